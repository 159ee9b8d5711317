"""Run a few steps on a reduced copy of a benchmark workload, for profilers.

  python profile_step.py [--nz 64]
        [--form f32|f64|both|surrogate|argon] [--steps 3] [--train-steps 1000]

f32/f64: the nitrogen 3D workload on nz x 256 x 512 cells (x fastest) of the
256 x 256 x 512 benchmark's recipe (a few GB of device memory at most for
nz <= 64).  argon: the Ar-like lognormal workload (the mixed-batch and
surrogate recipe) on as many cells, stepped by ion_step (FP32).  surrogate:
the same cells with a surrogate trained for --train-steps steps, stepped by
ion_step_surrogate.
Every step starts from the same input state.  Meant to be wrapped by ncu
with a kernel filter and a launch count, e.g.
  ncu --set full --clock-control none -k regex:ion_stream_kernel -s 1 -c 1 ...
"""
import argparse

import torch

from paper_2202_10647_gb300 import ionize, workloads


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nz", type=int, default=64)
    ap.add_argument("--form", default="both",
                    choices=["f32", "f64", "both", "surrogate", "argon"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--train-steps", type=int, default=1000)
    args = ap.parse_args()
    dev = torch.device("cuda")
    if args.form == "argon":
        sd = workloads.argon_like()
        sp = ionize.Species(sd.U, sd.l, sd.m)
        wl = workloads.ladder_cells(sd, args.nz * 256 * 512, 4, device=dev)
        n = wl.ncells
        N0, lo0, hi0 = wl.N.clone(), wl.lo.clone(), wl.hi.clone()
        dne = torch.empty(n, device=dev)
        ws = ionize.workspace(n)
        for _ in range(args.steps):
            wl.N.copy_(N0)
            wl.lo.copy_(lo0)
            wl.hi.copy_(hi0)
            ionize.step(sp, wl.E, wl.N, wl.lo, wl.hi, 0.05, dne, ws=ws)
        torch.cuda.synchronize()
        print("argon: fp64-coefficient cells, invalid windows:", ionize.counters(ws),
              "stiff cells:", ionize.stiff_cells(ws), "of", n)
        return
    if args.form == "surrogate":
        from paper_2202_10647_gb300 import surrogate
        sd = workloads.argon_like()
        sp = ionize.Species(sd.U, sd.l, sd.m)
        net, _, _ = surrogate.build(sp, steps=args.train_steps)
        wl = workloads.ladder_cells(sd, args.nz * 256 * 512, 4, device=dev)
        n = wl.ncells
        N0, lo0, hi0 = wl.N.clone(), wl.lo.clone(), wl.hi.clone()
        dne = torch.empty(n, device=dev)
        ws = ionize.workspace(n)
        for _ in range(args.steps):
            wl.N.copy_(N0)
            wl.lo.copy_(lo0)
            wl.hi.copy_(hi0)
            net.step(wl.E, wl.N, wl.lo, wl.hi, 0.05, dne, ws=ws)
        torch.cuda.synchronize()
        print("surrogate: (network cells, Eq. 1 cells, timeouts):",
              ionize.surrogate_counters(ws))
        return
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
