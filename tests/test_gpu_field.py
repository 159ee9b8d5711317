"""The step from field components (ion_field_magnitude, ion_step_field):
the magnitude against numpy, the step against the oracle on the magnitude
computed in FP64 from the same components, and against ion_step on the
magnitudes the library computed (equal bits)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_10647_gb300 import ionize, workloads as W
from test_gpu_step import TOL, check, gpu_species, oracle_species

pytestmark = pytest.mark.gpu


def components(E, ncomp, seed):
    """Split magnitudes |E| into ncomp signed components on a random
    direction per cell (float64)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(ncomp, E.size))
    d /= np.linalg.norm(d, axis=0)
    return [E * d[i] for i in range(ncomp)]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("ncomp", [1, 2, 3])
def test_field_magnitude(dtype, ncomp):
    rng = np.random.default_rng(ncomp)
    E = np.concatenate([10.0 ** rng.uniform(-3, 5, 30001), [0.0, 1e-7, 3e4]])
    comp = [torch.tensor(c, dtype=dtype, device="cuda") for c in components(E, ncomp, 5)]
    args = comp + [None] * (3 - ncomp)
    m = ionize.field_magnitude(*args).cpu().numpy().astype(np.float64)
    c64 = [c.double().cpu().numpy() for c in comp]
    ref = np.sqrt(sum(c * c for c in c64))
    if dtype == torch.float32:
        # fused multiply-adds and a correctly rounded sqrt in float32
        assert np.all(np.abs(m - ref) <= 3 * np.spacing(ref.astype(np.float32)) + 1e-45)
    else:
        assert np.all(np.abs(m - ref) <= 4 * np.spacing(ref) + 1e-300)
    if ncomp == 1:
        assert np.array_equal(m, np.abs(c64[0]))


@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F64_PLAIN])
@pytest.mark.parametrize("ncomp", [1, 3])
def test_step_field(flags, ncomp):
    sd = W.argon_like()
    wl = W.ladder_cells(sd, 50000, 17)
    n = wl.ncells
    f64 = bool(flags & ionize.ION_F64_PLAIN)
    dt_ = torch.float64 if f64 else torch.float32
    comp = [torch.tensor(c, dtype=dt_) for c in components(wl.E.double().numpy(), ncomp, 9)]
    sp = gpu_species(sd)
    gc = [c.cuda() for c in comp]
    N, lo, hi = wl.N.to(dt_).cuda(), wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne = torch.zeros(n, dtype=dt_, device="cuda")
    ionize.step_field(sp, gc, N, lo, hi, 0.05, dne, flags=flags)
    # the same step on the library's magnitudes: equal bits
    Em = ionize.field_magnitude(*(gc + [None] * (3 - ncomp)))
    N2, lo2, hi2 = wl.N.to(dt_).cuda(), wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne2 = torch.zeros(n, dtype=dt_, device="cuda")
    ionize.step(sp, Em, N2, lo2, hi2, 0.05, dne2, flags=flags)
    assert torch.equal(N, N2) and torch.equal(lo, lo2) and torch.equal(hi, hi2)
    assert torch.equal(dne, dne2)
    # the oracle on the magnitude of the same components in FP64
    Eo = np.sqrt(sum(c.double().numpy() ** 2 for c in comp))
    No, loo, hio, dneo = oracle.step(oracle_species(sd), Eo, wl.N.to(dt_).double().numpy()[:, :n],
                                     0.05, wl.lo.numpy(), wl.hi.numpy())
    out = dict(N=N.double().cpu().numpy(), lo=lo.cpu().numpy(), hi=hi.cpu().numpy(),
               dne=dne.double().cpu().numpy())
    check(out, dict(N=No, lo=loo, hi=hio, dne=dneo), wl.lo, wl.hi, flags, sd=sd,
          E=Em.double().cpu().numpy())


def test_step_field_arguments():
    sd = W.argon_like()
    sp = gpu_species(sd)
    n = 100
    Ex = torch.ones(n, device="cuda")
    N = torch.zeros((sd.Z + 1, n), device="cuda")
    N[0] = 1
    lo = torch.zeros(n, dtype=torch.uint8, device="cuda")
    hi = torch.full((n,), 3, dtype=torch.uint8, device="cuda")
    dne = torch.zeros(n, device="cuda")
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        ionize.step_field(sp, [Ex, Ex], N, lo, hi, 0.05, dne, ws=small)
    with pytest.raises(ValueError):
        ionize.field_magnitude(Ex, Ex.double())


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.uint8])
def test_copy_cells(dtype):
    """ion_copy_cells: a cell range of every plane, host to device and back,
    equal to the same slices copied plane by plane."""
    Z1, ld = 5, 1000
    g = torch.Generator().manual_seed(3)
    src = (torch.rand((Z1, ld), generator=g) * 200).to(dtype).pin_memory()
    dev = torch.zeros((Z1, ld + 24), dtype=dtype, device="cuda")[:, :ld]  # rows ld + 24 apart
    ionize.copy_cells(dev, src, 130, 517)
    torch.cuda.synchronize()
    want = torch.zeros((Z1, ld), dtype=dtype)
    want[:, 130:647] = src[:, 130:647]
    assert torch.equal(dev.cpu(), want)
    back = torch.full((Z1, ld), 7, dtype=dtype).pin_memory()
    ionize.copy_cells(back, dev, 100, 600)
    torch.cuda.synchronize()
    want2 = torch.full((Z1, ld), 7, dtype=dtype)
    want2[:, 100:700] = want[:, 100:700]
    assert torch.equal(back, want2)
    one = torch.zeros(ld, dtype=dtype, device="cuda")
    ionize.copy_cells(one, src[2].contiguous().pin_memory(), 0, ld)
    torch.cuda.synchronize()
    assert torch.equal(one.cpu(), src[2])
    with pytest.raises(ValueError):
        ionize.copy_cells(dev, src, 900, 200)
