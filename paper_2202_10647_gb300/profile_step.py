"""Run a few ion_step calls on the nitrogen 3D workload, for profilers.

  python -m paper_2202_10647_gb300.profile_step [--nz 64] [--form f32|f64|both]
                                                [--steps 3]

The grid is nz x 256 x 512 cells (x fastest) of the 256 x 256 x 512 benchmark
workload's recipe (a few GB of device memory at most for nz <= 64); every
step starts from the same input state.  Meant to be wrapped by ncu with a
kernel filter and a launch count, e.g.
  ncu --set full --clock-control none -k regex:ion_step_f32 -s 2 -c 2 ...
"""
import argparse

import torch

from . import ionize, workloads


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nz", type=int, default=64)
    ap.add_argument("--form", default="both", choices=["f32", "f64", "both"])
    ap.add_argument("--steps", type=int, default=3)
    args = ap.parse_args()
    dev = torch.device("cuda")
    wl = workloads.nitrogen_3d(args.nz, 256, 512, seed=2, device=dev)
    n = wl.ncells
    sp = ionize.Species(wl.species.U, wl.species.l, wl.species.m)
    N0, lo0, hi0 = wl.N.clone(), wl.lo.clone(), wl.hi.clone()
    if args.form in ("f32", "both"):
        dne = torch.empty(n, device=dev)
        ws = ionize.workspace(n)
        for _ in range(args.steps):
            wl.N.copy_(N0)
            wl.lo.copy_(lo0)
            wl.hi.copy_(hi0)
            ionize.step(sp, wl.E, wl.N, wl.lo, wl.hi, 0.05, dne, ws=ws)
        torch.cuda.synchronize()
        print("f32: fp64-coefficient cells, invalid windows:", ionize.counters(ws),
              "stiff cells:", ionize.stiff_cells(ws))
    if args.form in ("f64", "both"):
        E64, N64 = wl.E.double(), N0.double()
        dne64 = torch.empty(n, dtype=torch.float64, device=dev)
        ws64 = ionize.workspace(n, ionize.ION_F64_PLAIN)
        for _ in range(args.steps):
            wl.lo.copy_(lo0)
            wl.hi.copy_(hi0)
            ionize.step(sp, E64, N64, wl.lo, wl.hi, 0.05, dne64, ws=ws64,
                        flags=ionize.ION_F64_PLAIN)
        torch.cuda.synchronize()
        print("f64 done")


if __name__ == "__main__":
    main()
