"""Rate-model variants: the static-field ADK rate (Eq. 1 without its
cycle-averaging factor) and CODATA constants, on the GPU against the oracle
with the same choice."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_10647_gb300 import ionize, workloads as W
from test_gpu_step import check

pytestmark = pytest.mark.gpu

CASES = [(ionize.ION_ADK_STATIC, None), (ionize.ION_ADK_CYCLE_AVERAGED, "codata"),
         (ionize.ION_ADK_STATIC, "codata")]


def species_pair(sd, model, consts):
    c = ionize.CODATA_CONSTANTS if consts == "codata" else None
    g = ionize.Species(sd.U, sd.l, sd.m, constants=c, rate_model=model)
    o = oracle.Species(sd.U, sd.l, sd.m, constants=c, model=model)
    return g, o


@pytest.mark.parametrize("model,consts", CASES)
@pytest.mark.parametrize("dtype,rtol", [(torch.float32, 2e-6), (torch.float64, 1e-12)])
def test_rates(model, consts, dtype, rtol):
    sd = W.argon_like()
    sp, osp = species_pair(sd, model, consts)
    E = torch.pow(10.0, 1.0 + 3.7 * W.uniform(5, 1, torch.arange(20000))).to(dtype)
    Wg = ionize.rates(sp, E.cuda(), 0, sd.Z).double().cpu().numpy()
    Wo = oracle.rates(osp, E.double().numpy(), 0, sd.Z)
    big = Wo * 0.05 > 1e-30
    assert np.abs(Wg[big] / Wo[big] - 1).max() <= rtol
    # the static rate differs from the cycle-averaged one by the factor
    if model == ionize.ION_ADK_STATIC:
        sa, _ = species_pair(sd, ionize.ION_ADK_CYCLE_AVERAGED, consts)
        Wa = ionize.rates(sa, E.cuda(), 0, sd.Z).double().cpu().numpy()
        assert not np.allclose(Wa[big], Wg[big])


@pytest.mark.parametrize("model,consts", CASES)
@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F64_PLAIN])
def test_step(model, consts, flags):
    sd = W.argon_like()
    sp, osp = species_pair(sd, model, consts)
    wl = W.ladder_cells(sd, 6001, 31)
    n = wl.ncells
    f64 = bool(flags & ionize.ION_F64_PLAIN)
    dt_ = torch.float64 if f64 else torch.float32
    E, N = wl.E.to(dt_).cuda(), wl.N.to(dt_).cuda()
    lo, hi = wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne = torch.zeros(n, dtype=dt_, device="cuda")
    ionize.step(sp, E, N, lo, hi, 0.05, dne, flags=flags)
    No, loo, hio, dneo = oracle.step(osp, wl.E.to(dt_).double().numpy(),
                                     wl.N[:, :n].to(dt_).double().numpy(), 0.05,
                                     wl.lo.numpy(), wl.hi.numpy())
    out = dict(N=N.double().cpu().numpy(), lo=lo.cpu().numpy(), hi=hi.cpu().numpy(),
               dne=dne.double().cpu().numpy())
    check(out, dict(N=No, lo=loo, hi=hio, dne=dneo), wl.lo, wl.hi, flags, sd=sd,
          E=wl.E.to(dt_).double().numpy())
