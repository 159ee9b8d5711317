"""ion_step_noalloc, the entry point for callers that cannot allocate device
memory (code running under someone else's stream capture, hosts that forbid
device allocations, fixed-footprint codes).  It must give the results of
ion_step with a caller workspace, call after call, through the C ABI.

This file is collected last on purpose: the entry point shares one scratch
array per device for the life of the process, and its test must also pass
after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2202_10647_gb300 import ionize, workloads as W

pytestmark = pytest.mark.gpu

TOL = {ionize.ION_F32: 2e-6, ionize.ION_F64_PLAIN: 1e-12}


def _raw_noalloc(lib, sp, E, N, lo, hi, dne, n, flags):
    return lib.ion_step_noalloc(sp.handle, ctypes.c_void_p(E.data_ptr()),
                                ctypes.c_void_p(N.data_ptr()), N.shape[1], n, 0.05,
                                ctypes.c_void_p(lo.data_ptr()), ctypes.c_void_p(hi.data_ptr()),
                                ctypes.c_void_p(dne.data_ptr()), None, None, flags,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F64_PLAIN])
def test_noalloc_matches_workspace_step_on_two_calls(flags):
    dtype = torch.float64 if flags & ionize.ION_F64_PLAIN else torch.float32
    wl = W.nitrogen_3d(16, 32, 64, seed=31)
    n = wl.ncells - 5  # ragged: not a multiple of the 32-cell chunks
    dev = "cuda"
    sp = ionize.Species(wl.species.U, wl.species.l, wl.species.m)
    osp = oracle.Species(wl.species.U, wl.species.l, wl.species.m)
    lib = ionize.lib()
    E = wl.E.to(dtype).to(dev)
    # two copies of the state: one stepped through ion_step, one through
    # ion_step_noalloc, twice in a row
    Na, Nb = wl.N.to(dtype).to(dev), wl.N.to(dtype).to(dev)
    loa, hia = wl.lo.to(dev), wl.hi.to(dev)
    lob, hib = wl.lo.clone().to(dev), wl.hi.clone().to(dev)
    dnea = torch.zeros(n, dtype=dtype, device=dev)
    dneb = torch.full((n,), 7.0, dtype=dtype, device=dev)
    ws = ionize.workspace(n, flags)
    No = wl.N[:, :n].to(dtype).double().numpy()
    loo, hio = wl.lo[:n].numpy().copy(), wl.hi[:n].numpy().copy()
    Eo = wl.E[:n].to(dtype).double().numpy()
    tol = TOL[flags & ionize.ION_F64_PLAIN]
    for call in range(2):
        ionize.step(sp, E, Na, loa, hia, 0.05, dnea, ws=ws, flags=flags, ncells=n)
        rc = _raw_noalloc(lib, sp, E, Nb, lob, hib, dneb, n, flags)
        assert rc == ionize.ION_OK, lib.ion_last_error()
        torch.cuda.synchronize()
        # the same kernels on the same inputs: bit for bit, so that a counter
        # or record left in the shared array by an earlier call would show
        assert torch.equal(Na, Nb), call
        assert torch.equal(dnea, dneb), call
        assert torch.equal(loa, lob) and torch.equal(hia, hib), call
        # and within the tolerance of the oracle, started from the same state
        No, loo, hio, dneo = oracle.step(osp, Eo, No, 0.05, loo, hio)
        assert np.abs(Nb[:, :n].double().cpu().numpy() - No).max() <= tol, call
        No = Nb[:, :n].double().cpu().numpy()
        loo, hio = lob[:n].cpu().numpy(), hib[:n].cpu().numpy()
    # the state moved between the two calls (the second call saw new input)
    assert not torch.equal(Nb.cpu(), wl.N.to(dtype))


def test_noalloc_python_wrapper_and_its_size_checks():
    wl = W.nitrogen_3d(8, 16, 32, seed=33)
    dev = "cuda"
    sp = ionize.Species(wl.species.U, wl.species.l, wl.species.m)
    n = wl.ncells
    E, N, lo, hi = wl.E.to(dev), wl.N.to(dev), wl.lo.to(dev), wl.hi.to(dev)
    dne = torch.zeros(n, device=dev)
    Na, loa, hia = N.clone(), lo.clone(), hi.clone()
    dnea = torch.zeros(n, device=dev)
    ionize.step(sp, E, Na, loa, hia, 0.05, dnea)
    ionize.step_noalloc(sp, E, N, lo, hi, 0.05, dne)
    torch.cuda.synchronize()
    assert torch.equal(N, Na) and torch.equal(dne, dnea)
    assert torch.equal(lo, loa) and torch.equal(hi, hia)
    # ncells past one of the arrays is refused before any launch
    N0 = N.clone()
    for bad in (dict(k_lo=lo[:n - 1]), dict(dne=dne[:n - 8]), dict(ncells=n + 1),
                dict(ncells=-1), dict(n_gas=torch.ones(n - 1, device=dev))):
        args = dict(sp=sp, E=E, N=N, k_lo=lo, k_hi=hi, dt=0.05, dne=dne)
        args.update(bad)
        with pytest.raises(ValueError):
            ionize.step_noalloc(**args)
    torch.cuda.synchronize()
    assert torch.equal(N, N0)


def test_noalloc_rejects_too_many_cells():
    wl = W.nitrogen_3d(4, 8, 16, seed=32)
    sp = ionize.Species(wl.species.U, wl.species.l, wl.species.m)
    lib = ionize.lib()
    dev = "cuda"
    n = ionize.ION_STEP_NOALLOC_MAX_CELLS + 1
    E = torch.zeros(n, device=dev)
    N = torch.zeros((8, n), device=dev)
    lo = torch.zeros(n, dtype=torch.uint8, device=dev)
    hi = torch.zeros(n, dtype=torch.uint8, device=dev)
    dne = torch.zeros(n, device=dev)
    rc = _raw_noalloc(lib, sp, E, N, lo, hi, dne, n, ionize.ION_F32)
    assert rc == ionize.ION_EINVAL
    assert b"split" in lib.ion_last_error()
    # the maximum itself is accepted
    rc = _raw_noalloc(lib, sp, E, N, lo, hi, dne, n - 1, ionize.ION_F32)
    assert rc == ionize.ION_OK, lib.ion_last_error()
    torch.cuda.synchronize()
