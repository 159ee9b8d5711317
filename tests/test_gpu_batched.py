"""The batched FP32 step (several species in one launch), every launch shape,
and the autotuner, against the FP64 oracle per species."""
import numpy as np
import pytest
import torch

import oracle
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
        check(gpu_out(job), oracle_of(wl), wl.lo, wl.hi, ionize.ION_F32, sd=wl.species,
              E=wl.E.double().numpy())
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
        check(gpu_out(job), oracle_of(wl), wl.lo, wl.hi, ionize.ION_F64_PLAIN, sd=wl.species,
              E=wl.E.double().numpy())


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


def test_full_size_mixed_batch_sampled():
    """The mixed-species workload at its benchmark size (N 20M, Ar-like 8M,
    Kr-like 2M cells) in the autotuned launch shape: sampled cells of every
    species against the oracle, conservation over every cell."""
    dev = "cuda"
    wls = W.mixed_batch(scale=1.0, seed=3, device=dev)
    sps = [ionize.Species(w.species.U, w.species.l, w.species.m) for w in wls]
    dnes = [torch.empty(w.ncells, device=dev) for w in wls]
    jobs = [(sp, w.E, w.N, w.lo, w.hi, d) for sp, w, d in zip(sps, wls, dnes)]
    ws = ionize.batched_workspace(jobs)
    pristine = [(w.N.clone(), w.lo.clone(), w.hi.clone()) for w in wls]
    shape, _ = ionize.autotune(jobs, 0.05, ws=ws, reps=2)
    for w, (n0, l0, h0) in zip(wls, pristine):
        w.N.copy_(n0)
        w.lo.copy_(l0)
        w.hi.copy_(h0)
    rng = np.random.default_rng(11)
    samples = []
    for w in wls:
        ix = torch.tensor(np.sort(rng.choice(w.ncells, 3000, replace=False)), device=dev)
        samples.append((ix, w.E[ix].double().cpu().numpy(), w.N[:, ix].double().cpu().numpy(),
                        w.lo[ix].cpu().numpy(), w.hi[ix].cpu().numpy()))
    ionize.step_batched(jobs, 0.05, ws=ws, shape=shape)
    torch.cuda.synchronize()
    for w, (n0, _, _), (ix, Es, Ns, ls, hs) in zip(wls, pristine, samples):
        n = w.ncells
        tot = (w.N[:, :n].double().sum(0) - n0[:, :n].double().sum(0)).abs().max()
        assert float(tot) <= 1e-6
        No, loo, hio, dneo = oracle.step(oracle_species(w.species), Es, Ns, 0.05, ls, hs)
        err = np.abs(w.N[:, ix].double().cpu().numpy() - No).max()
        assert err <= 2e-6, (w.species.name, err)


@pytest.mark.parametrize("shape", [(1, 2), (1, 4), (1, 8), (2, 2), (2, 4), (2, 8)])
@pytest.mark.parametrize("name", ["nitrogen_3d", "Kr-like"])
def test_single_species_kernel_equals_general_kernel(shape, name):
    """A launch of one species under the paper's window rule takes the
    single-species streaming kernel; the same cells launched beside an empty
    second job take the general one.  Both run the same cell arithmetic, so
    the results are equal bit for bit, and both match the oracle."""
    if name == "nitrogen_3d":
        wl = W.nitrogen_3d(8, 32, 64, seed=47)
    else:
        wl = W.ladder_cells(W.krypton_like(), 6007, 48, block=64)
    n = wl.ncells
    dev = "cuda"
    sp = ionize.Species(wl.species.U, wl.species.l, wl.species.m)
    runs = []
    for extra in (False, True):
        E, N = wl.E.to(dev), wl.N.to(dev)
        lo, hi = wl.lo.clone().to(dev), wl.hi.clone().to(dev)
        dne = torch.full((n,), 9.0, device=dev)
        jobs = [(sp, E, N, lo, hi, dne)]
        if extra:
            z8 = torch.zeros(4, dtype=torch.uint8, device=dev)
            jobs.append((sp, torch.zeros(0, device=dev), torch.zeros((wl.species.Z + 1, 4), device=dev),
                         z8[:0], z8[:0], torch.zeros(0, device=dev)))
        ws = ionize.step_batched(jobs, 0.05, shape=(shape[0], shape[1], 0))
        torch.cuda.synchronize()
        runs.append((N, lo, hi, dne, ionize.counters(ws)))
    (Na, la, ha, da, ca), (Nb, lb, hb, db, cb) = runs
    assert torch.equal(Na, Nb) and torch.equal(la, lb) and torch.equal(ha, hb)
    assert torch.equal(da, db) and ca == cb
    check(dict(N=Na.double().cpu().numpy(), lo=la.cpu().numpy(), hi=ha.cpu().numpy(),
               dne=da.double().cpu().numpy()), oracle_of(wl), wl.lo, wl.hi, ionize.ION_F32,
          sd=wl.species, E=wl.E.double().numpy())


def fields_at_top_rate(sd, lo, hi, target, dt=0.05):
    """|E| per cell at which the largest rate of its window has W dt = target:
    the lowest field on a grid in log |E| where it exceeds the target, then
    bisection on the oracle's rates (Eq. 1 peaks and falls again at high
    fields, so the grid picks the rising side)."""
    osp = oracle_species(sd)
    n = lo.shape[0]

    def top(logE):
        Wr = oracle.rates(osp, 10.0 ** logE, 0, sd.Z) * dt
        k = np.arange(sd.Z)[:, None]
        inwin = (k >= lo[None, :]) & (k < hi[None, :])
        return np.where(inwin, Wr, 0.0).max(axis=0)

    grid = np.arange(0.0, 6.0001, 0.05)  # log10 |E| in GV/m
    above = np.stack([top(np.full(n, g)) > target for g in grid])
    assert not above[0].any() and above.any(axis=0).all()
    i = above.argmax(axis=0)
    a, b = grid[i - 1], grid[i]
    for _ in range(60):
        m = 0.5 * (a + b)
        up = top(m) > target
        b, a = np.where(up, m, b), np.where(up, a, m)
    E = (10.0 ** b).astype(np.float32)
    got = top(np.log10(E.astype(np.float64)))
    assert np.all(np.abs(got / target - 1.0) < 1e-4)
    return E


@pytest.mark.parametrize("general", [False, True])
def test_series_bound_by_cells_per_lane(general):
    """Cells whose largest window rate has 1 < W dt < 1.5 are finished by
    the Taylor series in the streaming kernel when a lane holds one cell (a
    warp's series then serves 32 cells) and become records for the Bateman
    form when it holds two; both match the oracle.  `general` launches two
    species at once (the general streaming kernel), otherwise one (the
    single-species kernel)."""
    dev = "cuda"
    rng = np.random.default_rng(53)
    wls = []
    for sd, n, seed in ((W.nitrogen(), 2053, 54), (W.argon_like(), 3001, 55)):
        wl = W.ladder_cells(sd, n, seed, block=64)
        target = rng.uniform(1.02, 1.48, n)
        wl.E.copy_(torch.from_numpy(fields_at_top_rate(sd, wl.lo.numpy().astype(int),
                                                       wl.hi.numpy().astype(int), target)))
        wls.append(wl)
    groups = [wls] if general else [[wl] for wl in wls]
    for shape, q in (((1, 8, 0), 1), ((2, 8, 0), 2)):
        for group in groups:
            jobs = []
            for wl in group:
                sp = ionize.Species(wl.species.U, wl.species.l, wl.species.m)
                jobs.append((sp, wl.E.to(dev), wl.N.to(dev), wl.lo.clone().to(dev),
                             wl.hi.clone().to(dev), torch.full((wl.ncells,), 9.0, device=dev)))
            ws = ionize.step_batched(jobs, 0.05, shape=shape)
            torch.cuda.synchronize()
            tails = sum(wl.ncells % (32 * q) for wl in group)
            want = tails if q == 1 else sum(wl.ncells for wl in group)
            assert ionize.stiff_cells(ws) == want, (shape, ionize.stiff_cells(ws), want)
            for wl, job in zip(group, jobs):
                check(gpu_out(job), oracle_of(wl), wl.lo, wl.hi, ionize.ION_F32,
                      sd=wl.species, E=wl.E.double().numpy())
