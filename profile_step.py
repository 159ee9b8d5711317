"""Run a few steps on a reduced copy of a benchmark workload, for profilers.

  python profile_step.py [--nz 64]
        [--form f32|f64|both|surrogate|argon|batched] [--steps 3] [--train-steps 1000]
        [--scale 0.25]

f32/f64: the nitrogen 3D workload on nz x 256 x 512 cells (x fastest) of the
256 x 256 x 512 benchmark's recipe (a few GB of device memory at most for
nz <= 64).  argon: the Ar-like lognormal workload (the mixed-batch and
surrogate recipe) on as many cells, stepped by ion_step (FP32).  batched:
the mixed-species workload (N, Ar-like, Kr-like) at --scale of its cell
counts, stepped by ion_step_batched in launch shape (1, 8, 0).  surrogate:
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
                    choices=["f32", "f64", "both", "surrogate", "argon", "batched"])
    ap.add_argument("--scale", type=float, default=0.25,
                    help="batched: fraction of the mixed-species cell counts")
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
    if args.form == "batched":
        wls = workloads.mixed_batch(scale=args.scale, seed=3, device=dev)
        sps = [ionize.Species(w.species.U, w.species.l, w.species.m) for w in wls]
        pristine = [(w.N.clone(), w.lo.clone(), w.hi.clone()) for w in wls]
        jobs = [(sp, w.E, w.N, w.lo, w.hi, torch.empty(w.ncells, device=dev))
                for sp, w in zip(sps, wls)]
        ws = ionize.batched_workspace(jobs)
        for _ in range(args.steps):
            for w, (n0, l0, h0) in zip(wls, pristine):
                w.N.copy_(n0)
                w.lo.copy_(l0)
                w.hi.copy_(h0)
            ionize.step_batched(jobs, 0.05, ws=ws, shape=(1, 8, 0))
        torch.cuda.synchronize()
        print("batched: fp64-coefficient cells, invalid windows:", ionize.counters(ws),
              "stiff cells:", ionize.stiff_cells(ws), "of", sum(w.ncells for w in wls))
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
