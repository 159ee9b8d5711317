"""Parity of the CUDA step with the FP64 oracle, through the C ABI.

Tolerances (per cell, per population, Sigma_k N_k = 1):
  FP32 form          |N - N_oracle| <= 2e-6, |dne - dne_oracle| <= (w-1) 2e-6
  plain FP64 form    |N - N_oracle| <= 1e-12, |dne - dne_oracle| <= 1e-11
Inputs are identical on both sides: the oracle gets the GPU's fp32 inputs
promoted to double.  Window decisions are compared exactly except for cells
whose lowest-state population lies within the tolerance of eps_shift.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2202_10647_gb300 import ionize, workloads as W

pytestmark = pytest.mark.gpu

TOL = {ionize.ION_F32: 2e-6, ionize.ION_F64_PLAIN: 1e-12}


def gpu_species(sd):
    return ionize.Species(sd.U, sd.l, sd.m)


def oracle_species(sd):
    return oracle.Species(sd.U, sd.l, sd.m)


def run_both(sd, E, N, lo, hi, dt=0.05, flags=ionize.ION_F32, n=None, eps=1e-6,
             gap=1e-3, update=True, n_gas=None):
    """Run one GPU step and the oracle on the same inputs.  E (float32 [n]),
    N (float32 [Z+1, ld]), lo/hi (uint8) are CPU tensors."""
    n = E.numel() if n is None else n
    f64 = bool(flags & ionize.ION_F64_PLAIN)
    dt_ = torch.float64 if f64 else torch.float32
    dev = torch.device("cuda")
    sp = gpu_species(sd)
    Eg = E.to(dt_).to(dev)
    Ng = N.to(dt_).to(dev)
    log, hig = lo.clone().to(dev), hi.clone().to(dev)
    dne = torch.full((max(n, 1),), float("nan"), dtype=dt_, device=dev)
    ng = None if n_gas is None else n_gas.to(dt_).to(dev)
    upd = 0 if update else ionize.ION_NO_WINDOW_UPDATE
    ws = ionize.step(sp, Eg, Ng, log, hig, dt, dne, n_gas=ng, eps_shift=eps,
                     degen_gap=gap, flags=flags | upd, ncells=n)
    torch.cuda.synchronize()
    out = dict(N=Ng.double().cpu().numpy(), lo=log.cpu().numpy(), hi=hig.cpu().numpy(),
               dne=dne[:n].double().cpu().numpy(), counters=ionize.counters(ws),
               sd=sd, E=E.to(dt_).double().numpy()[:n], update=update, eps=eps)
    # the oracle sees exactly the values the GPU read
    Ein = E.to(dt_).double().numpy()[:n]
    Nin = N.to(dt_).double().numpy()[:, :n]
    No, loo, hio, dneo = oracle.step(oracle_species(sd), Ein, Nin, dt, lo.numpy()[:n],
                                     hi.numpy()[:n], None if n_gas is None else
                                     n_gas.to(dt_).double().numpy()[:n],
                                     eps_shift=eps, window_update=update)
    ref = dict(N=No, lo=loo, hi=hio, dne=dneo)
    return out, ref


def window_ties(sd, E, out_N, ref_N, lo, hi, out_lo, out_hi, ref_lo, ref_hi, eps, f32,
                policy=None):
    """Window decisions against the oracle.  The GPU applies the rule to its
    own populations, so (1) its windows must equal the oracle's rule run on
    the GPU's post-step populations (dt = 0 leaves them as they are), bit
    for bit; then (2) a window that differs from the oracle's own must come
    from a population the rule compared that lies on the other side of its
    threshold on the two sides.  Returns the number of such cells."""
    n = out_lo.shape[0]
    eps_r = float(np.float32(eps)) if f32 else eps
    kw = {}
    if policy is not None:
        kw = dict(policy=oracle.WINDOW_ADAPTIVE, w_min=policy["w_min"], w_max=policy["w_max"],
                  eps_grow=float(np.float32(policy["eps_grow"])) if f32 else policy["eps_grow"])
    _, slo, shi, _ = oracle.step(oracle_species(sd), E, out_N, 0.0, lo, hi, eps_shift=eps_r, **kw)
    assert np.array_equal(slo, out_lo) and np.array_equal(shi, out_hi), \
        f"{int(((slo != out_lo) | (shi != out_hi)).sum())} windows break the rule on the GPU's own values"
    diff = np.nonzero((out_lo != ref_lo) | (out_hi != ref_hi))[0]
    for c in diff:
        a, b = int(lo[c]), int(hi[c])
        g, o = out_N[a:b, c], ref_N[a:b, c]
        straddle = np.any((g < eps_r) != (o < eps))
        if policy is not None:
            e2 = policy["eps_grow"]
            straddle = straddle or ((out_N[b, c] > e2) != (ref_N[b, c] > e2))
        assert straddle, f"cell {c}: windows differ with no population across a threshold"
    return len(diff)


def check(out, ref, lo, hi, flags, eps=1e-6, n=None, sd=None, E=None, max_ties=None):
    """Populations within the tolerance per cell and state, dne within (w-1)
    tolerances (one per internal boundary of the window: dne is the sum of
    the population that crossed them), windows as `window_ties` states.
    With sd and E given (the species and the fields the GPU read), the
    windows are checked against the rule on the GPU's own values; at most
    max(1, n/1000) cells may then differ from the oracle's windows."""
    tol = TOL[flags & ionize.ION_F64_PLAIN]
    n = ref["N"].shape[1] if n is None else n
    Ng = out["N"][:, :n]
    err = np.abs(Ng - ref["N"]).max(axis=0)
    assert err.max() <= tol, f"max |N - oracle| = {err.max():g} at cell {err.argmax()}"
    lo_, hi_ = lo.numpy()[:n], hi.numpy()[:n]
    w = hi_.astype(int) - lo_.astype(int) + 1
    derr = np.abs(out["dne"] - ref["dne"])
    dtol = np.maximum(w - 1, 1) * tol
    assert np.all(derr <= dtol), f"max |dne - oracle| = {derr.max():g} (cell {derr.argmax()})"
    sd = out.get("sd") if sd is None else sd
    E = out.get("E") if E is None else E
    eps = out.get("eps", eps)
    if sd is None or not out.get("update", True):
        assert np.array_equal(out["lo"][:n], ref["lo"]) and np.array_equal(out["hi"][:n], ref["hi"])
        return 0
    f32 = not flags & ionize.ION_F64_PLAIN
    ties = window_ties(sd, np.asarray(E, dtype=np.float64)[:n], Ng, ref["N"], lo_, hi_,
                       out["lo"][:n], out["hi"][:n], ref["lo"], ref["hi"], eps, f32)
    limit = max(1, n // 1000) if max_ties is None else max_ties
    assert ties <= limit, f"{ties} window decisions differ from the oracle's (limit {limit})"
    return ties


def cells_of(wl, n=None):
    n = wl.ncells if n is None else n
    return wl.E[:n], wl.N, wl.lo[:n], wl.hi[:n]


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F64_PLAIN])
def test_nitrogen_grid_parity(flags):
    wl = W.nitrogen_3d(16, 32, 64, seed=11)
    n = wl.ncells - 3  # ragged tail: not a multiple of the 4 cells per thread
    E, N, lo, hi = cells_of(wl, n)
    out, ref = run_both(wl.species, E, N, lo, hi, flags=flags, n=n)
    check(out, ref, lo, hi, flags, n=n)
    # planes past the last cell are untouched
    assert np.array_equal(out["N"][:, n:], wl.N[:, n:].double().numpy())


@pytest.mark.parametrize("flags", [ionize.ION_F32 | ionize.ION_NO_FP64_FALLBACK,
                                   ionize.ION_F32 | ionize.ION_FORCE_FP64_COEF])
def test_fp32_coefficient_modes(flags):
    wl = W.nitrogen_3d(8, 32, 64, seed=12)
    E, N, lo, hi = cells_of(wl)
    out, ref = run_both(wl.species, E, N, lo, hi, flags=flags)
    check(out, ref, lo, hi, ionize.ION_F32)
    fb, bad = out["counters"]
    assert bad == 0
    if flags & ionize.ION_FORCE_FP64_COEF:
        # every cell that takes the Bateman form (some rate W dt > 1) is
        # computed with FP64 coefficients; the others take the Taylor form
        w = (hi.long() - lo.long() + 1)
        assert 0 < fb <= int((w >= 2).sum())
    else:
        assert fb == 0


@pytest.mark.parametrize("name", ["Ar-like", "Kr-like"])
@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F64_PLAIN])
def test_ladder_parity(name, flags):
    sd = W.argon_like() if name == "Ar-like" else W.krypton_like()
    wl = W.ladder_cells(sd, 20000, seed=21, block=64)
    E, N, lo, hi = cells_of(wl)
    out, ref = run_both(sd, E, N, lo, hi, flags=flags)
    check(out, ref, lo, hi, flags)


def adversarial(sd, seed=0):
    """Every window width 1..6 at the bottom, middle and top of the ladder
    against fields from 0 to 1e6 GV/m, plus fields at which two rates of a
    window cross (equal and nearly equal rates)."""
    Z = sd.Z
    Es = [0.0, 1e-7, 1e-3, 1.0, 30.0, 100.0, 300.0, 700.0, 1000.0, 2000.0, 4000.0,
          6000.0, 1e4, 1e5, 1e6]
    # crossings of W_i and W_j for i < j in the same 6-wide window
    osp = oracle_species(sd)
    grid = np.exp(np.linspace(math.log(20), math.log(2e4), 4000))
    Wg = np.log(np.maximum(oracle.rates(osp, grid, 0, Z), 1e-300))
    for i in range(Z):
        for j in range(i + 1, min(Z, i + 5)):
            d = Wg[i] - Wg[j]
            ok = (Wg[i] > -200) & (Wg[j] > -200)
            s = np.nonzero((np.sign(d[:-1]) != np.sign(d[1:])) & ok[:-1])[0]
            for t in s[:2]:
                a, b = grid[t], grid[t + 1]
                for _ in range(60):
                    c = math.sqrt(a * b)
                    dc = (math.log(max(oracle.adk_rate(c, sd.U[i], sd.l[i], sd.m[i], i + 1), 1e-300))
                          - math.log(max(oracle.adk_rate(c, sd.U[j], sd.l[j], sd.m[j], j + 1), 1e-300)))
                    if np.sign(dc) == np.sign(d[t]):
                        a = c
                    else:
                        b = c
                for rel in (0.0, 1e-9, 1e-6, 1e-4, 1e-3, 3e-3, 1e-2, 0.1):
                    Es.append(float(np.float32(a * (1 + rel))))
    E, lo, hi = [], [], []
    for e in Es:
        for w in range(1, 7):
            for base in sorted({0, Z // 3, Z // 2, Z + 1 - w}):
                if base + w - 1 > Z or base < 0:
                    continue
                E.append(e)
                lo.append(base)
                hi.append(base + w - 1)
    n = len(E)
    ld = (n + 3) // 4 * 4
    lo_t = torch.tensor(lo, dtype=torch.uint8)
    p = torch.tensor([h - l + 1 for l, h in zip(lo, hi)])
    N = W.populations(seed, lo_t, p, Z, ld)
    return torch.tensor(E, dtype=torch.float32), N, lo_t, torch.tensor(hi, dtype=torch.uint8)


@pytest.mark.parametrize("name", ["N", "Ar-like", "Kr-like"])
@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F32 | ionize.ION_NO_FP64_FALLBACK,
                                   ionize.ION_F64_PLAIN])
def test_adversarial_cells(name, flags):
    sd = {"N": W.nitrogen(), "Ar-like": W.argon_like(), "Kr-like": W.krypton_like()}[name]
    E, N, lo, hi = adversarial(sd)
    out, ref = run_both(sd, E, N, lo, hi, flags=flags)
    check(out, ref, lo, hi, flags)
    assert np.all(np.isfinite(out["N"]))
    tot_in = N.double().numpy().sum(0)[:E.numel()]
    tot_out = out["N"].sum(0)[:E.numel()]
    assert np.abs(tot_out - tot_in).max() <= (1e-6 if not flags & 1 else 1e-14)


@pytest.mark.parametrize("dt", [0.0, 1e-4, 0.05, 1.0])
def test_time_steps_and_gas_density(dt):
    wl = W.nitrogen_3d(8, 16, 32, seed=13)
    E, N, lo, hi = cells_of(wl)
    ng = 1.0 + torch.arange(wl.ncells, dtype=torch.float32) % 7
    for flags in (ionize.ION_F32, ionize.ION_F64_PLAIN):
        out, ref = run_both(wl.species, E, N, lo, hi, dt=dt, flags=flags, n_gas=ng)
        check(out, ref, lo, hi, flags)
        if dt == 0.0:
            assert np.array_equal(out["N"], N.to(torch.float64 if flags else torch.float32).double().numpy())
            assert np.all(out["dne"] == 0.0)


def test_invalid_windows_are_skipped_and_counted():
    sd = W.nitrogen()
    E = torch.full((8,), 1500.0)
    lo = torch.tensor([0, 3, 5, 2, 0, 1, 4, 6], dtype=torch.uint8)
    hi = torch.tensor([3, 2, 9, 8, 6, 4, 7, 7], dtype=torch.uint8)  # 1: lo>hi, 2: hi>Z, 3,4: w>6
    N = W.populations(1, lo.clamp(max=7), torch.full((8,), 2), 7, 8)
    dev = "cuda"
    sp = gpu_species(sd)
    Ng = N.to(dev)
    log, hig = lo.to(dev), hi.to(dev)
    dne = torch.full((8,), -7.0, device=dev)
    ws = ionize.step(sp, E.to(dev), Ng, log, hig, 0.05, dne)
    fb, bad = ionize.counters(ws)
    assert bad == 4
    for c in (1, 2, 3, 4):
        assert torch.equal(Ng[:, c].cpu(), N[:, c])
        assert float(dne[c]) == -7.0
        assert int(log[c]) == int(lo[c]) and int(hig[c]) == int(hi[c])
    assert float(dne[0]) != -7.0


def test_guard_planes_untouched():
    """Canaries: planes and cells around the arrays stay bit-identical."""
    wl = W.nitrogen_3d(8, 16, 32, seed=14)
    n = wl.ncells
    dev = "cuda"
    Z = 7
    guard = 12
    big = torch.full((Z + 3, n + 2 * guard), 12345.0, device=dev)
    big[1:Z + 2, guard:guard + n] = wl.N[:, :n].to(dev)
    # view with ld = n + 2*guard starting at plane 1, cell `guard`
    N = big[1:Z + 2]
    sp = gpu_species(wl.species)
    E = torch.full((n + 2 * guard,), 777.0, device=dev)
    E[guard:guard + n] = wl.E.to(dev)
    lo = torch.full((n + 2 * guard,), 200, dtype=torch.uint8, device=dev)
    hi = lo.clone()
    lo[guard:guard + n] = wl.lo.to(dev)
    hi[guard:guard + n] = wl.hi.to(dev)
    dne = torch.full((n + 2 * guard,), 5.5, device=dev)
    lib = ionize.lib()
    ws = ionize.workspace(n)
    import ctypes
    off = guard
    rc = lib.ion_step(sp.handle, ctypes.c_void_p(E.data_ptr() + 4 * off),
                      ctypes.c_void_p(N.data_ptr() + 4 * off), N.shape[1], n, 0.05,
                      ctypes.c_void_p(lo.data_ptr() + off), ctypes.c_void_p(hi.data_ptr() + off),
                      ctypes.c_void_p(dne.data_ptr() + 4 * off), None, None, 0,
                      ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.ion_last_error()
    torch.cuda.synchronize()
    b = big.cpu()
    assert torch.all(b[0] == 12345.0) and torch.all(b[Z + 2] == 12345.0)
    assert torch.all(b[:, :guard] == 12345.0) and torch.all(b[:, guard + n:] == 12345.0)
    d = dne.cpu()
    assert torch.all(d[:guard] == 5.5) and torch.all(d[guard + n:] == 5.5)
    assert torch.all(lo.cpu()[:guard] == 200) and torch.all(lo.cpu()[guard + n:] == 200)


def test_argument_validation():
    sd = W.nitrogen()
    sp = gpu_species(sd)
    dev = "cuda"
    n = 64
    E = torch.full((n,), 100.0, device=dev)
    N = torch.zeros((8, n), device=dev)
    lo = torch.zeros(n, dtype=torch.uint8, device=dev)
    hi = torch.full((n,), 3, dtype=torch.uint8, device=dev)
    dne = torch.empty(n, device=dev)
    ws = ionize.workspace(n)
    ok = dict(sp=sp, E=E, N=N, k_lo=lo, k_hi=hi, dt=0.05, dne=dne, ws=ws)
    ionize.step(**ok)
    bad = [dict(dt=-1.0), dict(dt=float("inf")), dict(ws=ws[:100]), dict(eps_shift=-1.0),
           dict(degen_gap=1.5), dict(flags=0x100),
           dict(flags=ionize.ION_NO_FP64_FALLBACK | ionize.ION_FORCE_FP64_COEF)]
    for b in bad:
        args = dict(ok)
        args.update(b)
        with pytest.raises(ionize.IonError) as ei:
            ionize.step(**args)
        assert ei.value.code == ionize.ION_EINVAL
    # E misaligned to its element size, and ld < ncells
    import ctypes
    lib = ionize.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.ion_step(sp.handle, ctypes.c_void_p(E.data_ptr() + 1), ctypes.c_void_p(N.data_ptr()),
                      n, n - 1, 0.05, ctypes.c_void_p(lo.data_ptr()), ctypes.c_void_p(hi.data_ptr()),
                      ctypes.c_void_p(dne.data_ptr()), None, None, 0, ctypes.c_void_p(ws.data_ptr()),
                      ws.numel(), st)
    assert rc == ionize.ION_EINVAL
    rc = lib.ion_step(sp.handle, ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(N.data_ptr()),
                      n - 2, n, 0.05, ctypes.c_void_p(lo.data_ptr()), ctypes.c_void_p(hi.data_ptr()),
                      ctypes.c_void_p(dne.data_ptr()), None, None, 0, ctypes.c_void_p(ws.data_ptr()),
                      ws.numel(), st)
    assert rc == ionize.ION_EINVAL
    # empty input is a no-op
    ionize.step(sp, E[:0], N, lo[:0], hi[:0], 0.05, dne[:0], ws=ws, ncells=0)


@pytest.mark.parametrize("dtype,rtol", [(torch.float32, 2e-6), (torch.float64, 1e-12)])
def test_rates_parity(dtype, rtol):
    for sd in (W.nitrogen(), W.argon_like(), W.krypton_like()):
        E = torch.tensor(np.exp(np.linspace(math.log(1e-7), math.log(2e5), 3001)), dtype=dtype)
        E[0] = 0.0
        sp = gpu_species(sd)
        Wg = ionize.rates(sp, E.cuda(), 0, sd.Z).double().cpu().numpy()
        Wo = oracle.rates(oracle_species(sd), E.double().numpy(), 0, sd.Z)
        big = Wo * 0.05 > 1e-30
        rel = np.abs(Wg[big] - Wo[big]) / Wo[big]
        assert rel.max() <= rtol, rel.max()
        # where the oracle says 0 the GPU agrees, up to values no step can see
        assert np.all(Wg[Wo == 0] * 0.05 <= 1e-30)
        assert np.all(np.abs(Wg[~big]) * 0.05 <= 2e-30)


def test_nitrogen_pulse_200_steps_fp64():
    """The 2D nitrogen run: 200 steps of 0.05 fs from N_0 = 1, window [0,3],
    with window updates; FP64 parity at every step."""
    sd = W.nitrogen()
    wl = W.nitrogen_2d_initial()
    n = wl.ncells
    dev = "cuda"
    sp = gpu_species(sd)
    osp = oracle_species(sd)
    N = wl.N.double().to(dev)
    lo, hi = wl.lo.clone().to(dev), wl.hi.clone().to(dev)
    dne = torch.empty(n, dtype=torch.float64, device=dev)
    ws = ionize.workspace(n, ionize.ION_F64_PLAIN)
    No = wl.N[:, :n].double().numpy()
    loo, hio = wl.lo.numpy().copy(), wl.hi.numpy().copy()
    worst = 0.0
    for s in range(200):
        E = W.nitrogen_pulse_2d(s * 0.05)
        ionize.step(sp, E.double().to(dev), N, lo, hi, 0.05, dne, ws=ws,
                    flags=ionize.ION_F64_PLAIN)
        No, loo, hio, dneo = oracle.step(osp, E.double().numpy(), No, 0.05, loo, hio)
        if s % 10 == 9 or s == 199:
            Ng = N[:, :n].cpu().numpy()
            worst = max(worst, float(np.abs(Ng - No).max()))
            assert worst <= 1e-12, (s, worst)
            assert np.array_equal(lo.cpu().numpy(), loo) and np.array_equal(hi.cpu().numpy(), hio)
            assert np.abs(dne.cpu().numpy() - dneo).max() <= 1e-11
    # something happened: the front ionized at least the first two levels
    assert float(N[0, :n].min()) < 1e-3


def test_full_size_nitrogen_sampled():
    """The 256x256x512 nitrogen workload as the benchmark runs it: sampled
    cells against the oracle, and properties over every cell."""
    dev = "cuda"
    wl = W.nitrogen_3d(device=dev)
    n = wl.ncells
    rng = np.random.default_rng(0)
    idx = torch.tensor(np.sort(rng.choice(n, 20000, replace=False)), device=dev)
    E_s, N_s = wl.E[idx].cpu(), wl.N[:, idx].cpu()
    lo_s, hi_s = wl.lo[idx].cpu(), wl.hi[idx].cpu()
    tot0 = wl.N[:, :n].double().sum(0)
    sp = gpu_species(wl.species)
    dne = torch.empty(n, device=dev)
    ws = ionize.step(sp, wl.E, wl.N, wl.lo, wl.hi, 0.05, dne)
    torch.cuda.synchronize()
    fb, bad = ionize.counters(ws)
    assert bad == 0 and fb < n // 50
    tot1 = wl.N[:, :n].double().sum(0)
    assert float((tot1 - tot0).abs().max()) <= 1e-6
    assert float(wl.N[:, :n].min()) >= -1e-6
    assert bool(torch.all(wl.hi <= 7)) and bool(torch.all(wl.lo <= wl.hi))
    No, loo, hio, dneo = oracle.step(oracle_species(wl.species), E_s.double().numpy(),
                                     N_s.double().numpy(), 0.05, lo_s.numpy(), hi_s.numpy())
    Ng = wl.N[:, idx].double().cpu().numpy()
    assert np.abs(Ng - No).max() <= 2e-6
    assert np.abs(dne[idx].double().cpu().numpy() - dneo).max() <= 1e-5


def test_cell_ranges_with_offset():
    """Stepping cell ranges through `offset` gives what one whole call gives
    (ranges on 64-cell boundaries take the same kernel path)."""
    wl = W.nitrogen_3d(8, 16, 64, device="cuda")
    n = wl.ncells
    sp = gpu_species(wl.species)
    N1, lo1, hi1 = wl.N.clone(), wl.lo.clone(), wl.hi.clone()
    d1 = torch.zeros(n, device="cuda")
    ionize.step(sp, wl.E, N1, lo1, hi1, 0.05, d1)
    N2, lo2, hi2 = wl.N.clone(), wl.lo.clone(), wl.hi.clone()
    d2 = torch.zeros(n, device="cuda")
    for c0 in range(0, n, 2048):
        ionize.step(sp, wl.E, N2, lo2, hi2, 0.05, d2, offset=c0, ncells=min(2048, n - c0))
    assert torch.equal(N1, N2) and torch.equal(lo1, lo2) and torch.equal(hi1, hi2)
    assert torch.equal(d1, d2)
    with pytest.raises(ValueError):
        ionize.step(sp, wl.E, N2, lo2, hi2, 0.05, d2, offset=n - 10, ncells=20)


def _field_at_rate(osp, k, log2_rate, dt=0.05):
    """|E| at which the oracle's W_k dt equals 2^log2_rate (bisection in
    log E; W_k increases with |E| below that point)."""
    a, b = 1e-3, 1e7
    for _ in range(200):
        m = math.sqrt(a * b)
        w = oracle.rates(osp, np.array([m]), k, k + 1)[0, 0] * dt
        if w > 0 and math.log2(w) >= log2_rate:
            b = m
        else:
            a = m
    return a


def test_cold_chunks():
    """Chunks of cells whose window rates all have W dt far below the first
    Taylor term's threshold keep N bit for bit and free no electron; a cell
    in such a chunk whose lowest states hold less than eps_shift still
    slides (twice where two states are below it), and a chunk with one hot
    cell takes the full step.  All of it matches the oracle."""
    sd = W.nitrogen()
    osp = oracle_species(sd)
    n = 64 * 40 + 17
    idx = torch.arange(n)
    lo = (W.uniform(11, 1, idx) * 5).long().clamp(max=4)
    hi = lo + 2
    root = [_field_at_rate(osp, k, -30.0) for k in range(7)]
    E = torch.tensor([0.5 * root[int(k)] for k in lo], dtype=torch.float32)
    E[idx % 3 == 0] *= 0.01
    E[idx % 7 == 0] = 0.0
    hot = 11 * 64 + 5
    E[hot] = 3.0 * root[int(lo[hot])]
    ld = (n + 3) // 4 * 4
    N = torch.zeros((8, ld), dtype=torch.float32)
    p = W.uniform(11, 2, idx).to(torch.float32) * 0.5 + 0.25
    N[lo, idx] = p
    N[lo + 1, idx] = (1 - p) * 0.75
    N[lo + 2, idx] = 1 - p - (1 - p) * 0.75
    slides = [3 * 64 + 9, 7 * 64 + 40]
    for c in slides:
        N[lo[c], c] = 1e-8
        N[lo[c] + 1, c] = 1 - 1e-8 - N[lo[c] + 2, c]
    c2 = 9 * 64 + 17  # two states below eps_shift: slides twice
    lo[c2], hi[c2] = 1, 3
    E[c2] = 0.5 * root[1]
    N[:, c2] = 0.0
    N[1, c2], N[2, c2], N[3, c2] = 1e-8, 2e-8, 1 - 3e-8
    slides.append(c2)
    out, ref = run_both(sd, E, N, lo.to(torch.uint8), hi.to(torch.uint8))
    check(out, ref, lo.to(torch.uint8), hi.to(torch.uint8), ionize.ION_F32)
    cold = np.ones(n, bool)
    cold[11 * 64:12 * 64] = False
    cold[slides] = False
    cold[64 * 40:] = False  # the ragged tail takes the record path
    Nin = N.numpy()
    assert np.array_equal(out["N"][:, :n][:, cold].astype(np.float32), Nin[:, :n][:, cold])
    assert np.all(out["dne"][cold] == 0.0)
    assert np.array_equal(out["lo"], ref["lo"]) and np.array_equal(out["hi"], ref["hi"])
    for c in slides[:2]:
        assert out["lo"][c] == lo[c] + 1
    assert out["lo"][c2] == 3 and out["hi"][c2] == 5
    assert out["dne"][hot] > 0.0


@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F64_PLAIN])
def test_stiff_windows_rate_order(flags):
    """Stiff windows (some W dt > 1) of every width whose rates fall or rise
    along the window (the contiguous-range divided differences) and whose
    rates do neither (a ladder with potentials that go down and up again:
    every subset of the rates), both against the oracle; each record class
    of the FP32 path (windows of up to 4 states, and wider) is filled."""
    rising = W.SpeciesData("rising", [12.0, 18.0, 26.0, 35.0, 47.0, 60.0, 75.0],
                           [1, 1, 1, 1, 1, 0, 0], [0] * 7)
    zigzag = W.SpeciesData("zigzag", [20.0, 14.0, 30.0, 22.0, 40.0, 31.0, 55.0],
                           [1, 0, 1, 0, 1, 0, 1], [0] * 7)
    for sd in (rising, zigzag):
        n = 64 * 24 + 11
        idx = torch.arange(n)
        w = 2 + (idx % 5)                       # widths 2..6
        lo = (W.uniform(21, 1, idx) * (8 - w).double()).long()
        hi = lo + w - 1
        # fields from well below to far above the windows' first thresholds
        E = (10.0 ** (1.5 + 2.0 * W.uniform(21, 2, idx))).to(torch.float32)
        ld = (n + 3) // 4 * 4
        N = torch.zeros((8, ld), dtype=torch.float32)
        p = W.uniform(21, 3, idx).to(torch.float32)
        for r in range(6):
            on = (r < w - 1)
            share = (p * (r + 1)) % 1.0 + 0.05
            N[(lo + r).clamp(max=7)[on], idx[on]] = share[on]
        tot = N[:, :n].sum(0)
        N[:, :n] /= tot
        lo8, hi8 = lo.to(torch.uint8), hi.to(torch.uint8)
        out, ref = run_both(sd, E, N, lo8, hi8, flags=flags)
        check(out, ref, lo8, hi8, flags)
        osp = oracle_species(sd)
        Wr = oracle.rates(osp, E.double().numpy(), 0, 7) * 0.05
        stiff = np.array([Wr[int(lo[c]):int(hi[c]), c].max() > 1.0 for c in range(n)])
        assert stiff[(w <= 4).numpy()].sum() > 50 and stiff[(w > 4).numpy()].sum() > 50


def test_cold_cells_fp64():
    """The FP64 form's cold cells (every window rate below W dt = 2^-58):
    N is kept bit for bit, no electron is freed, windows whose lowest states
    hold less than eps_shift slide (once or twice), and hot cells in the same
    warps take the full step; all against the oracle."""
    sd = W.nitrogen()
    osp = oracle_species(sd)
    n = 32 * 30 + 7
    idx = torch.arange(n)
    lo = (W.uniform(12, 1, idx) * 5).long().clamp(max=4)
    hi = lo + 2
    root = [_field_at_rate(osp, k, -58.0) for k in range(7)]
    E = torch.tensor([0.5 * root[int(k)] for k in lo], dtype=torch.float32)
    E[idx % 5 == 0] = 0.0
    hot = idx % 32 == 7
    E[hot] = torch.tensor([3.0 * root[int(k)] for k in lo[hot]], dtype=torch.float32)
    ld = (n + 3) // 4 * 4
    N = torch.zeros((8, ld), dtype=torch.float32)
    p = W.uniform(12, 2, idx).to(torch.float32) * 0.5 + 0.25
    N[lo, idx] = p
    N[lo + 1, idx] = (1 - p) * 0.75
    N[lo + 2, idx] = 1 - p - (1 - p) * 0.75
    one, two = 3 * 32 + 9, 11 * 32 + 20
    N[lo[one], one] = 1e-8
    N[lo[one] + 1, one] = 1 - 1e-8 - N[lo[one] + 2, one]
    lo[two], hi[two] = 1, 3
    E[two] = 0.5 * root[1]
    N[:, two] = 0.0
    N[1, two], N[2, two], N[3, two] = 1e-8, 2e-8, 1 - 3e-8
    lo8, hi8 = lo.to(torch.uint8), hi.to(torch.uint8)
    out, ref = run_both(sd, E, N, lo8, hi8, flags=ionize.ION_F64_PLAIN)
    check(out, ref, lo8, hi8, ionize.ION_F64_PLAIN)
    cold = ~hot.numpy()
    Nin = N.double().numpy()[:, :n]
    assert np.array_equal(out["N"][:, :n][:, cold], Nin[:, cold])
    assert np.all(out["dne"][cold] == 0.0)
    assert np.all(out["dne"][hot.numpy()] > 0.0)
    assert out["lo"][one] == lo[one] + 1
    assert out["lo"][two] == 3 and out["hi"][two] == 5
    assert np.array_equal(out["lo"], ref["lo"]) and np.array_equal(out["hi"], ref["hi"])


def crossings(sd, dt=0.05):
    """Every field E with W_i(E) = W_j(E) dt > 1 for states i < j <= i + 4
    (bisection on the oracle's Eq. 1): (i, j, E)."""
    osp = oracle_species(sd)
    Z = sd.Z
    grid = np.exp(np.linspace(math.log(20), math.log(2e5), 20000))
    Wg = oracle.rates(osp, grid, 0, Z) * dt
    cross = []
    for i in range(Z):
        for j in range(i + 1, min(Z, i + 5)):
            d = np.log(np.maximum(Wg[i], 1e-300)) - np.log(np.maximum(Wg[j], 1e-300))
            for t in np.nonzero(np.sign(d[:-1]) != np.sign(d[1:]))[0]:
                if Wg[i, t] <= 1.0:
                    continue
                a, b = grid[t], grid[t + 1]
                for _ in range(80):
                    c = math.sqrt(a * b)
                    w = oracle.rates(osp, np.array([c]), 0, Z)[:, 0]
                    if np.sign(math.log(w[i]) - math.log(w[j])) == np.sign(d[t]):
                        a = c
                    else:
                        b = c
                cross.append((i, j, a))
    return cross


def degenerate_cells(sd, n_per=24, seed=3):
    """Stiff cells (some W dt > 1) whose windows hold a nearly equal pair of
    rates: at every crossing W_i(E) = W_j(E) with W dt > 1 (found by
    bisection on the oracle's Eq. 1), fields E (1 + d) for relative offsets d
    that put the pair's gap |W_i - W_j| / max from 0 to a few 1e-3, in
    windows of 3 to 6 states that contain both states.  Returns E, N, lo,
    hi and the oracle's smallest pair gap and largest W dt per cell."""
    osp = oracle_species(sd)
    Z = sd.Z
    cross = crossings(sd)
    E, lo, hi = [], [], []
    rel = [0.0, 1e-6, 1e-5, 3e-5, 1e-4, 2e-4, 5e-4, 1e-3, 3e-3, -1e-5, -1e-4, -5e-4]
    for q, (i, j, e0) in enumerate(cross):
        for r in rel:
            for w in range(max(3, j - i + 1), 7):
                a = max(0, min(i - (q + w) % 2, Z + 1 - w))
                if not (a <= i and j <= a + w - 2):
                    a = max(0, min(i, Z + 1 - w))
                if a + w - 1 > Z or j > a + w - 2:
                    continue
                E.append(float(np.float32(e0 * (1 + r))))
                lo.append(a)
                hi.append(a + w - 1)
    n = len(E)
    ld = (n + 3) // 4 * 4
    lo_t = torch.tensor(lo, dtype=torch.uint8)
    hi_t = torch.tensor(hi, dtype=torch.uint8)
    N = W.populations(seed, lo_t, hi_t.long() - lo_t.long(), Z, ld)
    Et = torch.tensor(E, dtype=torch.float32)
    Wc = oracle.rates(osp, Et.double().numpy(), 0, Z) * 0.05
    gap = np.full(n, np.inf)
    lmax = np.zeros(n)
    for c in range(n):
        lam = Wc[lo[c]:hi[c], c]
        lmax[c] = lam.max()
        for x in range(len(lam)):
            for y in range(x + 1, len(lam)):
                m = max(lam[x], lam[y])
                if m > 0:
                    gap[c] = min(gap[c], abs(lam[x] - lam[y]) / m)
    return Et, N, lo_t, hi_t, gap, lmax


@pytest.mark.parametrize("name", ["N", "Ar-like", "Kr-like"])
def test_near_degenerate_pairs_take_fp64_coefficients(name):
    """Under the default ION_F32 flags, stiff cells with a pair of window
    rates closer than 1e-3 relative (the divided differences of Eqs. 4-5
    divide by W_i - W_j) are queued for FP64 coefficients and match the
    oracle within the FP32 bar; the same cells with ION_NO_FP64_FALLBACK
    (FP32 divided differences with their Taylor switch) are reported."""
    sd = {"N": W.nitrogen(), "Ar-like": W.argon_like(), "Kr-like": W.krypton_like()}[name]
    E, N, lo, hi, gap, lmax = degenerate_cells(sd)
    n = E.numel()
    out, ref = run_both(sd, E, N, lo, hi)
    check(out, ref, lo, hi, ionize.ION_F32)
    fb, bad = out["counters"]
    assert bad == 0
    stiff = lmax > 1.01
    sure = int((stiff & (gap < 5e-4)).sum())
    maybe = int((stiff & (gap < 2e-3)).sum())
    assert sure > 20, sure
    assert sure <= fb <= maybe, (sure, fb, maybe)
    err_fb = float(np.abs(out["N"][:, :n] - ref["N"]).max())
    out2, _ = run_both(sd, E, N, lo, hi, flags=ionize.ION_F32 | ionize.ION_NO_FP64_FALLBACK)
    assert out2["counters"][0] == 0
    err_nofb = np.abs(out2["N"][:, :n] - ref["N"]).max(axis=0)
    sel = stiff & (gap < 1e-3)
    print(f"{name}: {n} cells, {fb} queued for FP64 coefficients "
          f"({sure} with an oracle gap below 5e-4); max |N - oracle| "
          f"{err_fb:.2e} with them, {float(err_nofb[sel].max()):.2e} on the same "
          f"near-degenerate cells without (ION_NO_FP64_FALLBACK)")


def end_gap_ratio(lam):
    """Largest spread / |z_i - z_j| over the contiguous ranges [j, i] of the
    nodes z = -lam whose spread is at least 1 (1 when the rates fall or rise
    along the window)."""
    z = -np.asarray(lam, dtype=np.float64)
    worst = 1.0
    for j in range(len(z)):
        for i in range(j + 2, len(z)):
            s = z[j:i + 1].max() - z[j:i + 1].min()
            if s >= 1.0:
                worst = max(worst, s / max(abs(z[i] - z[j]), 1e-300))
    return worst


@pytest.mark.parametrize("name", ["N", "Ar-like", "Kr-like"])
def test_close_ends_far_inner_node(name):
    """Windows whose rates do not fall or rise monotonically and where a
    range's end rates are close while an inner rate lies far off (near a
    crossing W_i = W_j, j >= i + 2, with a state between them): the
    end-removal recurrence of the divided differences would cancel there,
    so those ranges are evaluated on their sorted nodes.  Relative gaps of
    2e-3 to 0.1 keep the pair outside the FP64-coefficient criterion.  FP32
    (with and without the FP64 queue), the FP64-coefficient pass for every
    stiff cell, and the FP64 form all match the oracle."""
    sd = {"N": W.nitrogen(), "Ar-like": W.argon_like(), "Kr-like": W.krypton_like()}[name]
    osp = oracle_species(sd)
    Z = sd.Z
    E, lo, hi = [], [], []
    rel = [2e-3, -2e-3, 5e-3, -5e-3, 1e-2, -1e-2, 3e-2, -3e-2, 0.1, -0.1]
    for q, (i, j, e0) in enumerate(crossings(sd)):
        if j < i + 2:
            continue
        for r in rel:
            for w in range(j - i + 2, 7):
                a = max(0, min(i - (q + w) % 2, Z + 1 - w))
                if not (a <= i and j <= a + w - 2):
                    a = max(0, min(i, Z + 1 - w))
                if a + w - 1 > Z or j > a + w - 2:
                    continue
                E.append(float(np.float32(e0 * (1 + r))))
                lo.append(a)
                hi.append(a + w - 1)
    n = len(E)
    assert n > 0
    ld = (n + 3) // 4 * 4
    lo_t = torch.tensor(lo, dtype=torch.uint8)
    hi_t = torch.tensor(hi, dtype=torch.uint8)
    N = W.populations(7, lo_t, hi_t.long() - lo_t.long(), Z, ld)
    Et = torch.tensor(E, dtype=torch.float32)
    Wc = oracle.rates(osp, Et.double().numpy(), 0, Z) * 0.05
    ratio = np.array([end_gap_ratio(Wc[lo[c]:hi[c], c]) for c in range(n)])
    lmax = np.array([Wc[lo[c]:hi[c], c].max() for c in range(n)])
    far = int(((ratio > 16) & (lmax > 1.01)).sum())
    assert far >= 10, far
    for flags in (ionize.ION_F32, ionize.ION_F32 | ionize.ION_NO_FP64_FALLBACK,
                  ionize.ION_F32 | ionize.ION_FORCE_FP64_COEF, ionize.ION_F64_PLAIN):
        out, ref = run_both(sd, Et, N, lo_t, hi_t, flags=flags)
        check(out, ref, lo_t, hi_t, flags)
        assert out["counters"][1] == 0
        err = np.abs(out["N"][:, :n] - ref["N"]).max(axis=0)
        print(f"{name} flags {flags:#x}: {n} cells, {far} stiff with an end-gap ratio "
              f"above 16 (largest {ratio.max():.3g}); max |N - oracle| {err.max():.2e}")


def test_fp64_coefficients_for_many_cells():
    """ION_FORCE_FP64_COEF on 400,000 Ar-like cells: every stiff cell (about
    64,000, more than one pass of the FP64-coefficient kernel's warps) takes
    FP64 coefficients, and every cell matches the oracle."""
    sd = W.argon_like()
    wl = W.ladder_cells(sd, 400_000, 41)
    E, N, lo, hi = cells_of(wl)
    out, ref = run_both(sd, E, N, lo, hi, flags=ionize.ION_F32 | ionize.ION_FORCE_FP64_COEF)
    check(out, ref, lo, hi, ionize.ION_F32)
    fb, bad = out["counters"]
    assert bad == 0
    assert fb > 40_000, fb


@pytest.mark.parametrize("Z", [1, 2, 63])
@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F64_PLAIN])
def test_smallest_and_largest_species(Z, flags):
    """Species of 1, 2 and ION_MAX_Z = 63 transitions (synthetic ladders):
    every window width at the bottom, middle and top of the ladder against
    fields from 0 to 1e6 GV/m and rate crossings, in both forms."""
    assert Z <= ionize.ION_MAX_Z
    sd = W.synthetic_ladder(Z, 60 + Z)
    E, N, lo, hi = adversarial(sd, seed=Z)
    out, ref = run_both(sd, E, N, lo, hi, flags=flags)
    check(out, ref, lo, hi, flags)
    assert out["counters"][1] == 0


def test_batched_smallest_with_largest_species():
    """One batched launch over a 1-transition and a 63-transition species:
    each job matches its own oracle step."""
    jobs, refs = [], []
    for Z in (1, 63):
        sd = W.synthetic_ladder(Z, 70 + Z)
        E, N, lo, hi = adversarial(sd, seed=Z + 1)
        n = E.numel()
        No, loo, hio, dneo = oracle.step(oracle_species(sd), E.double().numpy(),
                                         N[:, :n].double().numpy(), 0.05, lo.numpy(), hi.numpy())
        jobs.append((gpu_species(sd), E.cuda(), N.cuda(), lo.clone().cuda(), hi.clone().cuda(),
                     torch.zeros(n, device="cuda")))
        refs.append((sd, E, lo, hi, dict(N=No, lo=loo, hi=hio, dne=dneo)))
    ionize.step_batched(jobs, 0.05)
    torch.cuda.synchronize()
    for (sp, Eg, Ng, log, hig, dne), (sd, E, lo, hi, ref) in zip(jobs, refs):
        out = dict(N=Ng.double().cpu().numpy(), lo=log.cpu().numpy(), hi=hig.cpu().numpy(),
                   dne=dne.double().cpu().numpy(), sd=sd, E=E.double().numpy())
        check(out, ref, lo, hi, ionize.ION_F32)
