"""Multi-step runs: the conservation diagnostic, graph-captured steps, and the
Kr-like 16-beam workload (512x512x256 cells, 50 steps of 0.05 fs from N_0 = 1,
window [0, 3]) against the oracle on sampled cells."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_10647_gb300 import ionize, multistep, workloads as W
from test_gpu_step import gpu_species, oracle_species, window_ties

pytestmark = pytest.mark.gpu

EPS = 1e-6
DT = 0.05


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_conservation_kernel(dtype):
    g = torch.Generator().manual_seed(3)
    for planes, n, ld in ((37, 100003, 100004), (8, 5, 8), (1, 1000, 1000), (64, 3001, 3001),
                          (9, 0, 4)):
        N = torch.rand((planes, ld), generator=g, dtype=torch.float64).to(dtype)
        want = float((N[:, :n].double().sum(0) - 1.0).abs().max()) if n else 0.0
        out = torch.full((1,), 123.0, device="cuda")
        ionize.conservation(N.cuda(), out, ncells=n)
        got = float(out.cpu())
        assert got == pytest.approx(want, rel=1e-6, abs=1e-30), (planes, n)
    # a NaN anywhere makes the result NaN
    N = torch.full((5, 64), 0.2, dtype=dtype)
    N[3, 17] = float("nan")
    out = torch.zeros(1, device="cuda")
    ionize.conservation(N.cuda(), out)
    assert torch.isnan(out.cpu()).all()
    # exact sums give 0, other targets are honoured
    N = torch.full((4, 256), 0.25, dtype=dtype)
    ionize.conservation(N.cuda(), out)
    assert float(out.cpu()) == 0.0
    ionize.conservation(N.cuda(), out, target=0.5)
    assert float(out.cpu()) == 0.5
    for bad in (dict(nplanes=0), dict(nplanes=65), dict(ncells=300)):
        with pytest.raises(ionize.IonError):
            ionize.conservation(N.cuda(), out, **bad)


def small_krypton(nz=32, ny=64, nx=64, steps=50, device="cuda"):
    A, B = W.krypton_beam_terms(nz, ny, nx, device=device)
    S = W.krypton_scale(A)
    fields = [W.krypton_field(A, B, s * DT, S) for s in range(steps)]
    wl = W.krypton_initial(nz * ny * nx, device=device)
    return wl, fields


def test_graph_equals_eager():
    """50 captured steps give bit for bit what 50 eager calls give."""
    wl, fields = small_krypton()
    n = wl.ncells
    sp = gpu_species(wl.species)
    state = []
    for _ in range(2):
        state.append((wl.N.clone(), wl.lo.clone(), wl.hi.clone(),
                      torch.zeros(n, device="cuda")))
    N, lo, hi, dne = state[0]
    ws = ionize.workspace(n)
    for E in fields:
        ionize.step(sp, E, N, lo, hi, DT, dne, ws=ws)
    N2, lo2, hi2, dne2 = state[1]
    g = multistep.StepGraph(sp, fields, N2, lo2, hi2, dne2, DT)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(N, N2) and torch.equal(lo, lo2) and torch.equal(hi, hi2)
    assert torch.equal(dne, dne2)
    # each step keeps sum_k N_k to 1e-6; FP32 storage makes the drift add up
    bound = 1e-6 * torch.arange(1, len(fields) + 1, device="cuda")
    assert bool(torch.all(g.cons <= bound)), g.cons
    # the run did something: windows slid in part of the cells
    assert int((lo2 > 0).sum()) > 0


def oracle_run(sd, Es, N0, lo0, hi0):
    """The oracle's steps on the sampled cells, with the cells whose window
    decisions come within 2% of eps_shift (where FP32 and FP64 may decide
    differently) marked from that step on."""
    osp = oracle_species(sd)
    N, lo, hi = N0, lo0.astype(np.int64), hi0.astype(np.int64)
    n = N.shape[1]
    cols = np.arange(n)
    tie = np.zeros(n, bool)
    out = []
    for E in Es:
        N1, lo1, hi1, dne = oracle.step(osp, E, N, DT, lo.astype(np.uint8), hi.astype(np.uint8))
        lo1, hi1 = lo1.astype(np.int64), hi1.astype(np.int64)
        # the slide compared N1[k] with eps for k = lo..lo1
        for r in range(6):
            k = np.minimum(lo + r, sd.Z)
            v = N1[k, cols]
            near = (r <= lo1 - lo) & (np.abs(v / EPS - 1.0) < 0.02)
            tie |= near
        out.append((N1, lo1, hi1, dne, tie.copy()))
        N, lo, hi = N1, lo1, hi1
    return out


def test_krypton_full_size_sampled():
    """The 512x512x256 Kr-like run as the benchmark does it, step by step.
    Every step is held to the FP32 bar on its own: the oracle restarts from
    the GPU's sampled state (populations and windows) before each step, so
    step s is compared with the exact solution of step s from the same
    input.  Conservation is checked over every cell after every step, and
    the cumulative drift against an oracle run from t = 0 is reported."""
    dev = "cuda"
    nz, ny, nx = 256, 512, 512
    n = nz * ny * nx
    A, B = W.krypton_beam_terms(nz, ny, nx, device=dev)
    S = W.krypton_scale(A)
    amp = S * torch.sqrt(A * A + B * B)
    rng = np.random.default_rng(5)
    hot = torch.nonzero(amp > 2000.0).flatten().cpu().numpy()
    assert hot.size > 10000
    idx = np.unique(np.concatenate([rng.choice(n, 1000, replace=False),
                                    rng.choice(hot, 1000, replace=False)]))
    del amp
    idx_d = torch.tensor(idx, device=dev)
    wl = W.krypton_initial(n, device=dev)
    sd = wl.species
    sp = gpu_species(sd)
    osp = oracle_species(sd)
    dne = torch.zeros(n, device=dev)
    ws = ionize.workspace(n)
    cons = torch.zeros(50, device=dev)
    N0 = wl.N[:, idx_d].double().cpu().numpy()
    lo0, hi0 = wl.lo[idx_d].cpu().numpy(), wl.hi[idx_d].cpu().numpy()
    gpu, Es = [], []
    for s in range(50):
        E = W.krypton_field(A, B, s * DT, S)
        Es.append(E[idx_d].double().cpu().numpy())
        ionize.step(sp, E, wl.N, wl.lo, wl.hi, DT, dne, ws=ws)
        ionize.conservation(wl.N, cons[s:s + 1], ncells=n)
        gpu.append((wl.N[:, idx_d].double().cpu().numpy(), wl.lo[idx_d].cpu().numpy(),
                    wl.hi[idx_d].cpu().numpy(), dne[idx_d].double().cpu().numpy()))
        del E
    # each step keeps sum_k N_k to 1e-6; FP32 storage makes the drift add up
    assert bool(torch.all(cons <= 1e-6 * torch.arange(1, 51, device=dev))), cons
    # step by step from the GPU's own state: the FP32 bar at every step
    Np, lp, hp = N0, lo0, hi0
    per_step, ties = [], 0
    for s, (Ng, lg, hg, dg) in enumerate(gpu, start=1):
        No, lo_, ho, do = oracle.step(osp, Es[s - 1], Np, DT, lp, hp)
        err = float(np.abs(Ng - No).max())
        per_step.append(err)
        assert err <= 2e-6, (s, err)
        w = hp.astype(int) - lp.astype(int) + 1
        assert np.all(np.abs(dg - do) <= (w - 1) * 2e-6), (s, float(np.abs(dg - do).max()))
        t = window_ties(sd, Es[s - 1], Ng, No, lp, hp, lg, hg, lo_, ho, EPS, True)
        assert t <= max(2, idx.size // 100), (s, t)
        ties += t
        assert np.all(lg <= hg) and np.all(hg <= sd.Z) and np.all(hg - lg == 3)
        assert np.abs(Ng.sum(0) - 1.0).max() <= 1e-6 * s
        Np, lp, hp = Ng, lg, hg
    # cumulative drift against an oracle run from t = 0 (not the parity bar:
    # reported; cells whose window decisions came within 2% of eps_shift at
    # some step are left out, since the two runs may then follow different
    # windows)
    ref = oracle_run(sd, Es, N0, lo0, hi0)
    drift = []
    for s, ((Ng, lg, hg, dg), (No, lo_, ho, do, tie)) in enumerate(zip(gpu, ref), start=1):
        keep = ~tie
        drift.append(float(np.abs(Ng[:, keep] - No[:, keep]).max()))
        # exp(dt A) is column-stochastic (an L1 contraction): local errors
        # (at most 2e-6 on each of 4 states, in the L1 norm 8e-6) add up at most
        assert drift[-1] <= 8e-6 * s, (s, drift[-1])
    # the pulse ionized the hot cells well past the first window
    assert np.mean(gpu[-1][1][np.isin(idx, hot)] > 0) > 0.5
    print(f"per-step max |N - oracle| (oracle restarted from the GPU state): "
          f"max {max(per_step):.2e}, last {per_step[-1]:.2e}; window ties {ties} over 50 "
          f"steps of {idx.size} cells; cumulative drift from t = 0: step 1 {drift[0]:.2e}, "
          f"step 50 {drift[-1]:.2e} ({int(ref[-1][4].sum())} cells left out); max |sum N - 1| "
          f"after step 1 {float(cons[0]):.2e}, after 50 {float(cons[-1]):.2e}")


@pytest.mark.parametrize("case", ["nitrogen_3d", "Ar-like", "Ar-like adaptive", "nitrogen FP64"])
def test_step_conservation_measure(case):
    """ION_CONSERVATION_CHECK: the step's own measure, the largest change of
    a cell's total population max_c |sum_k N'_k - sum_k N_k|, equals the same
    quantity computed on the host in FP64 from the populations before and
    after the step (every kernel of the step contributes: the streaming or
    single-species kernel, the records, the FP64-coefficient queue)."""
    dev = "cuda"
    window = None
    flags = ionize.ION_CONSERVATION_CHECK
    if case.startswith("nitrogen"):
        wl = W.nitrogen_3d(8, 32, 64, seed=51)
    else:
        wl = W.ladder_cells(W.argon_like(), 30011, 52, block=64)
    if case.endswith("adaptive"):
        window = dict(w_min=2, w_max=6, eps_grow=1e-6)
    dt_ = torch.float32
    if case.endswith("FP64"):
        flags |= ionize.ION_F64_PLAIN
        dt_ = torch.float64
    n = wl.ncells
    sp = gpu_species(wl.species)
    E, N = wl.E.to(dt_).to(dev), wl.N.to(dt_).to(dev)
    lo, hi = wl.lo.clone().to(dev), wl.hi.clone().to(dev)
    dne = torch.zeros(n, dtype=dt_, device=dev)
    N0 = N.clone()
    ws = ionize.step(sp, E, N, lo, hi, 0.05, dne, flags=flags, window=window)
    torch.cuda.synchronize()
    got = ionize.conservation_change(ws)
    want = float((N[:, :n].double().sum(0) - N0[:, :n].double().sum(0)).abs().max())
    assert got == pytest.approx(want, rel=1e-5, abs=1e-15), (got, want)
    assert 0.0 < got <= 1e-6 or dt_ == torch.float64
    # without the flag the word stays 0, and the step is the same
    N2, lo2, hi2 = N0.clone(), wl.lo.clone().to(dev), wl.hi.clone().to(dev)
    dne2 = torch.zeros(n, dtype=dt_, device=dev)
    ws2 = ionize.step(sp, E, N2, lo2, hi2, 0.05, dne2,
                      flags=flags & ~ionize.ION_CONSERVATION_CHECK, window=window)
    torch.cuda.synchronize()
    assert ionize.conservation_change(ws2) == 0.0
    assert torch.equal(N, N2) and torch.equal(lo, lo2) and torch.equal(hi, hi2)


def test_graph_with_fused_conservation():
    """The 50-step graph with the fused check: the populations are those of
    the graph with the full check after every step, the fused measure of
    step 1 equals the full check after step 1 (the run starts from
    sum_k N_k = 1 exactly), and the full check after step 50 stays within
    the sum of the 50 fused measures."""
    wl, fields = small_krypton()
    n = wl.ncells
    sp = gpu_species(wl.species)
    runs = {}
    for mode in ("full", "fused"):
        N, lo, hi = wl.N.clone(), wl.lo.clone(), wl.hi.clone()
        dne = torch.zeros(n, device="cuda")
        g = multistep.StepGraph(sp, fields, N, lo, hi, dne, DT, conservation=mode)
        g.replay()
        torch.cuda.synchronize()
        runs[mode] = (N, lo, hi, dne, g)
    Nf, lf, hf, df, gf = runs["full"]
    Nu, lu, hu, du, gu = runs["fused"]
    assert torch.equal(Nf, Nu) and torch.equal(lf, lu) and torch.equal(hf, hu)
    assert torch.equal(df, du)
    c, full = gu.cons.double().cpu().numpy(), gu.cons_full.double().cpu().numpy()
    assert full[0] == pytest.approx(c[0], rel=1e-5, abs=1e-15)
    assert full[0] == pytest.approx(float(gf.cons[0]), rel=1e-6, abs=1e-15)
    assert full[1] == pytest.approx(float(gf.cons[-1]), rel=1e-6, abs=1e-15)
    assert full[1] <= c.sum() * (1 + 1e-5) + 1e-12
    assert np.all(c <= 1e-6)
