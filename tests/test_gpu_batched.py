"""The batched FP32 step (several species in one launch), every launch shape,
and the autotuner, against the FP64 oracle per species."""
import numpy as np
import pytest
import torch

from paper_2202_10647_gb300 import ionize, workloads as W
from test_gpu_step import check, oracle_species

pytestmark = pytest.mark.gpu


def make_jobs(cells=(3000, 2000, 1500), seed=41, block=64):
    """N, Ar-like and Kr-like cells (the mixed-species workload, scaled down);
    ragged counts so every job has a partial last chunk."""
    dev = "cuda"
    out = []
    for i, (sd, n) in enumerate(zip((W.nitrogen(), W.argon_like(), W.krypton_like()), cells)):
        wl = W.ladder_cells(sd, n + 7 * i + 3, seed + i, block=block)
        out.append(wl)
    gjobs = []
    for wl in out:
        sp = ionize.Species(wl.species.U, wl.species.l, wl.species.m)
        gjobs.append((sp, wl.E.to(dev), wl.N.to(dev), wl.lo.clone().to(dev),
                      wl.hi.clone().to(dev), torch.zeros(wl.ncells, device=dev)))
    return out, gjobs


def oracle_of(wl):
    import oracle
    n = wl.ncells
    No, loo, hio, dneo = oracle.step(oracle_species(wl.species), wl.E.double().numpy(),
                                     wl.N[:, :n].double().numpy(), wl.dt, wl.lo.numpy(),
                                     wl.hi.numpy())
    return dict(N=No, lo=loo, hi=hio, dne=dneo)


def gpu_out(job):
    sp, E, N, lo, hi, dne = job
    return dict(N=N.double().cpu().numpy(), lo=lo.cpu().numpy(), hi=hi.cpu().numpy(),
                dne=dne.double().cpu().numpy())


@pytest.mark.parametrize("shape", ionize.LAUNCH_SHAPES)
def test_batched_every_shape_matches_oracle(shape):
    wls, jobs = make_jobs()
    ws = ionize.step_batched(jobs, 0.05, shape=(shape[0], shape[1], 0))
    torch.cuda.synchronize()
    for wl, job in zip(wls, jobs):
        check(gpu_out(job), oracle_of(wl), wl.lo, wl.hi, ionize.ION_F32)
    assert ionize.counters(ws)[1] == 0


def test_batched_equals_separate_steps():
    wls, jobs = make_jobs(seed=43)
    _, jobs2 = make_jobs(seed=43)
    ionize.step_batched(jobs, 0.05)
    for sp, E, N, lo, hi, dne in jobs2:
        ionize.step(sp, E, N, lo, hi, 0.05, dne)
    torch.cuda.synchronize()
    for a, b in zip(jobs, jobs2):
        assert float((a[2] - b[2]).abs().max()) <= 2e-6
        assert torch.equal(a[3], b[3]) and torch.equal(a[4], b[4])


def test_batched_fp64_form():
    wls, jobs = make_jobs(seed=44)
    dev = "cuda"
    j64 = [(sp, E.double(), N.double(), lo, hi, dne.double()) for sp, E, N, lo, hi, dne in jobs]
    ionize.step_batched(j64, 0.05, flags=ionize.ION_F64_PLAIN)
    torch.cuda.synchronize()
    for wl, job in zip(wls, j64):
        check(gpu_out(job), oracle_of(wl), wl.lo, wl.hi, ionize.ION_F64_PLAIN)


def test_autotune_returns_a_built_shape():
    wls, jobs = make_jobs(cells=(20000, 8000, 2000), seed=45)
    best, ms = ionize.autotune(jobs, 0.05, reps=1)
    assert (best.cells_per_lane, best.warps_per_block) in ionize.LAUNCH_SHAPES
    assert 0 <= best.blocks_per_sm <= 4 and ms > 0


def test_batched_rejects_bad_arguments():
    wls, jobs = make_jobs(cells=(100, 100, 100), seed=46)
    with pytest.raises(ionize.IonError):
        ionize.step_batched(jobs, 0.05, shape=(3, 4, 0))
    with pytest.raises(ValueError):
        ionize.step_batched(jobs * 3, 0.05)
