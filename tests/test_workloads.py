"""Input recipes: deterministic, valid windows, normalized populations."""
import math

import torch

from paper_2202_10647_gb300 import workloads as W


def test_hash_is_deterministic_and_uniformish():
    idx = torch.arange(100000)
    a = W.uniform(1, 2, idx)
    b = W.uniform(1, 2, idx)
    assert torch.equal(a, b)
    assert not torch.equal(a, W.uniform(1, 3, idx))
    assert 0.0 < float(a.min()) and float(a.max()) < 1.0
    assert abs(float(a.mean()) - 0.5) < 0.01
    g = W.normal(4, 1, idx)
    assert abs(float(g.mean())) < 0.02 and abs(float(g.std()) - 1) < 0.02


def test_ladders():
    for sp, Z in ((W.argon_like(), 18), (W.krypton_like(), 36)):
        assert sp.Z == Z and sp.U[0] == 15.0
        assert all(b > a for a, b in zip(sp.U, sp.U[1:]))
        assert 3.0 <= sp.U[8] / sp.U[7] <= 5.0
        assert sp.l[6] == 0 and sp.l[7] == 0 and sp.l[5] == 1
    assert W.argon_like().U == W.argon_like().U


def check_cells(wl):
    n = wl.ncells
    lo, hi = wl.lo.long(), wl.hi.long()
    Z = wl.species.Z
    assert torch.all(lo <= hi) and torch.all(hi <= Z)
    w = hi - lo + 1
    assert torch.all(w <= 6) and torch.all(w >= 1)
    N = wl.N[:, :n].double()
    assert torch.allclose(N.sum(0), torch.ones(n, dtype=torch.float64), atol=1e-6)
    assert torch.all(N >= 0)
    k = torch.arange(Z + 1)[:, None]
    outside = (k < lo[None, :]) | (k > hi[None, :])
    assert float(N[outside].abs().max()) == 0.0
    assert torch.all(wl.E >= 0) and torch.all(torch.isfinite(wl.E))
    assert wl.N.shape[1] % 4 == 0


def test_nitrogen_3d_small():
    wl = W.nitrogen_3d(8, 16, 32, seed=1)
    check_cells(wl)
    w = (wl.hi.long() - wl.lo.long() + 1)
    assert set(w.unique().tolist()) <= {3, 4}
    assert float(wl.E.max()) <= 4000.0


def test_ladder_cells_and_batch():
    for wl in W.mixed_batch(scale=1e-3):
        check_cells(wl)
        assert 100.0 <= float(wl.E.min()) and float(wl.E.max()) <= 5000.0


def test_pulse_2d():
    E = W.nitrogen_pulse_2d(5.0)
    assert E.shape == (128 * 128,)
    # at t = t0 the peak sits at x = 0, y = 0: 2000 |cos(w t0)|
    w = 2 * math.pi * W.C_UM_PER_FS / 0.8
    peak = 2000 * abs(math.cos(w * 5.0))
    assert float(E.max()) <= peak + 1e-3


def test_krypton_beam_terms_match_the_direct_sum():
    """A cos(wt) + B sin(wt) equals the beam-by-beam superposition at any t."""
    nz, ny, nx = 6, 10, 12
    A, B = W.krypton_beam_terms(nz, ny, nx, dx=2.0)
    omega = 2 * math.pi / 0.8 * W.C_UM_PER_FS
    for t in (0.0, 0.37, 1.3, 2.45):
        direct = W.krypton_beams_direct(t, nz, ny, nx, dx=2.0)
        two = A * math.cos(omega * t) + B * math.sin(omega * t)
        assert torch.allclose(two, direct, rtol=0, atol=1e-12 * 16)
    # a subset of cells takes the grid's values there
    cells = torch.tensor([0, 5, 77, nz * ny * nx - 1])
    As, Bs = W.krypton_beam_terms(nz, ny, nx, dx=2.0, cells=cells)
    assert torch.equal(As, A[cells]) and torch.equal(Bs, B[cells])
    S = W.krypton_scale(A)
    E0 = W.krypton_field(A, B, 0.0, S)
    assert E0.dtype == torch.float32 and abs(float(E0.max()) - 6000.0) < 1e-3
    assert float(E0.min()) >= 0.0
