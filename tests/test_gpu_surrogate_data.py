"""The surrogate's data preparation in library kernels: the FP64 log2 rates
of Eq. 1 (training targets) against the oracle, the input mapping and the
per-state standardization against numpy, and the validation bound
(ion_surrogate_validate) against the same reduction written out in numpy
over the network's rates and the oracle's."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2202_10647_gb300 import ionize, surrogate as S, workloads as W
from test_gpu_step import check, gpu_species, oracle_species
from test_gpu_surrogate import rand_P

pytestmark = pytest.mark.gpu

SPECIES = {"N": W.nitrogen, "Ar-like": W.argon_like, "Kr-like": W.krypton_like}


@pytest.mark.parametrize("name", list(SPECIES))
@pytest.mark.parametrize("floor", [-40.0, -200.0])
def test_log2_rates_match_oracle(name, floor):
    """max(log2 W_k, floor) from Eq. 1 in FP64: within 1e-10 of log2 of the
    oracle's rates (1e-12 relative in W is 1.4e-12 in log2), and exactly the
    floor where the oracle's rate is 0 or below it (zero field, the cutoff)."""
    sd = SPECIES[name]()
    sp = gpu_species(sd)
    rng = np.random.default_rng(3)
    E = np.concatenate([10.0 ** rng.uniform(-8, 6, 20000), [0.0, 1e-7, 1e-6, 2e-6, -250.0]])
    Ef = torch.tensor(E, dtype=torch.float32)
    y = ionize.log2_rates(sp, Ef.cuda(), 0, sd.Z, floor).cpu().numpy()  # (n, Z)
    Wo = oracle.rates(oracle_species(sd), Ef.double().numpy(), 0, sd.Z)  # (Z, n)
    with np.errstate(divide="ignore"):
        yo = np.maximum(np.log2(Wo), floor).T
    assert y.shape == yo.shape
    assert np.all(np.isfinite(y))
    assert np.abs(y - yo).max() <= 1e-10, np.abs(y - yo).max()
    assert np.all(y[yo == floor] == floor)
    # a sub-range of states, written with a row stride
    out = torch.full((Ef.numel(), 5), 7.0, dtype=torch.float64, device="cuda")
    part = ionize.log2_rates(sp, Ef.cuda(), 1, 4, floor, out=out[:, :3].contiguous())
    assert np.array_equal(part.cpu().numpy(), y[:, 1:4])


def test_log2_rates_argument_checks():
    sd = W.argon_like()
    sp = gpu_species(sd)
    E = torch.ones(10, device="cuda")
    with pytest.raises(RuntimeError):
        ionize.log2_rates(sp, E, 3, 3, -40.0)
    with pytest.raises(RuntimeError):
        ionize.log2_rates(sp, E, 0, sd.Z + 1, -40.0)
    with pytest.raises(RuntimeError):
        ionize.log2_rates(sp, E, 0, 2, float("nan"))


def test_mlp_inputs_match_numpy():
    rng = np.random.default_rng(4)
    E = np.concatenate([10.0 ** rng.uniform(0, 6, 50001), [0.0, -30.0, 1e30]]).astype(np.float32)
    l2lo, l2hi = S.log2_range()
    x = ionize.mlp_inputs(torch.tensor(E, device="cuda"), l2lo, l2hi).cpu().numpy()
    with np.errstate(divide="ignore"):
        l2 = np.log2(np.abs(E.astype(np.float64)))
    ref = np.clip(2.0 * (l2 - l2lo) / (l2hi - l2lo) - 1.0, -1.0, 1.0).astype(np.float32)
    assert np.array_equal(x, ref), np.abs(x - ref).max()
    assert x[-3] == -1.0 and x[-1] == 1.0


@pytest.mark.parametrize("n,K", [(2, 1), (1000, 18), (100003, 7), (4099, 63)])
def test_mlp_standardize_matches_numpy(n, K):
    """Column means and (n-1)-normalized standard deviations in FP64 (a
    constant column takes min_scale), the standardized targets rounded to
    float, and equal bits on a repeat."""
    rng = np.random.default_rng(n + K)
    Y = rng.normal(0.0, 1.0, (n, K)) * rng.uniform(0.1, 30.0, K) + rng.uniform(-60, 5, K)
    if K > 1:
        Y[:, 1] = -40.0  # a state clamped at the floor everywhere
    Yd = torch.tensor(Y, device="cuda")
    mean, scale, T = ionize.mlp_standardize(Yd, 1e-3)
    m = Y.mean(0)
    sdv = np.maximum(Y.std(0, ddof=1), 1e-3)
    assert np.allclose(mean.cpu().numpy(), m, rtol=1e-12, atol=1e-12)
    assert np.allclose(scale.cpu().numpy(), sdv, rtol=1e-12, atol=0)
    Tr = ((Y - mean.cpu().numpy()) / scale.cpu().numpy()).astype(np.float32)
    assert np.array_equal(T.cpu().numpy(), Tr)
    mean2, scale2, T2 = ionize.mlp_standardize(Yd, 1e-3)
    assert torch.equal(mean, mean2) and torch.equal(scale, scale2) and torch.equal(T, T2)


def bound_numpy(sd, net, nbins, per_bin, margin, floor_add, floor):
    """The validation bound written out: the sample points, the network's
    rates from the GPU, Eq. 1 from the oracle, the per-bin maximum."""
    l2lo, l2hi = S.log2_range()
    j = np.arange(nbins * per_bin)
    b, i = j // per_bin, j % per_bin
    E = np.exp2(l2lo + (l2hi - l2lo) * (b + i / (per_bin - 1)) / nbins).astype(np.float32)
    Wn = net.rates(torch.tensor(E, device="cuda")).double().cpu().numpy()  # (Z, n)
    Wo = oracle.rates(oracle_species(sd), E.astype(np.float64), 0, sd.Z)
    with np.errstate(divide="ignore"):
        yn = np.maximum(np.log2(Wn), floor)
        yo = np.maximum(np.log2(Wo), floor)
    d = np.abs(yn - yo).reshape(sd.Z, nbins, per_bin).max(2).T  # (nbins, Z)
    return d * margin + floor_add


def test_validate_bound_matches_numpy():
    sd = W.argon_like()
    sp = gpu_species(sd)
    P = torch.tensor(rand_P(sd.Z, 5, 0.3), dtype=torch.float32, device="cuda")
    l2lo, l2hi = S.log2_range()
    rng = np.random.default_rng(6)
    norm = {"log2E_min": l2lo, "log2E_max": l2hi, "y_floor": -40.0,
            "y_mean": list(rng.uniform(-30, 0, sd.Z)), "y_scale": list(rng.uniform(2, 9, sd.Z))}
    net = ionize.Surrogate(sp, P, norm)
    for nbins, per_bin, margin, add in ((64, 16, 1.25, 2e-3), (300, 7, 1.0, 0.0)):
        b = net.validate(nbins=nbins, per_bin=per_bin, margin=margin, floor_add=add)
        ref = bound_numpy(sd, net, nbins, per_bin, margin, add, -40.0)
        assert b.shape == (nbins, sd.Z)
        assert np.allclose(b, ref, rtol=1e-6, atol=1e-9), np.abs(b - ref).max()
    # the installed bound decides trust: a network with random weights misses
    # Eq. 1 by whole powers of two except where both clamp at the floor, so
    # at pop_tol 1e-6 the few cells on its rates are cells with vanishing
    # rates, and the step stays within the FP32 bar of the oracle
    net.validate()
    wl = W.ladder_cells(sd, 20000, 31)
    n = wl.ncells
    N, lo, hi = wl.N.cuda(), wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne = torch.zeros(n, device="cuda")
    ws = net.step(wl.E.cuda(), N, lo, hi, 0.05, dne, pop_tol=1e-6)
    n_net, n_plain, timeout = ionize.surrogate_counters(ws)
    assert timeout == 0 and n_net < n // 100 and n_plain > 0
    No, loo, hio, dneo = oracle.step(oracle_species(sd), wl.E.double().numpy(),
                                     wl.N[:, :n].double().numpy(), 0.05, wl.lo.numpy(),
                                     wl.hi.numpy())
    out = dict(N=N.double().cpu().numpy(), lo=lo.cpu().numpy(), hi=hi.cpu().numpy(),
               dne=dne.double().cpu().numpy())
    check(out, dict(N=No, lo=loo, hi=hio, dne=dneo), wl.lo, wl.hi, ionize.ION_F32, sd=sd,
          E=wl.E.double().numpy())
    with pytest.raises(RuntimeError):
        net.validate(nbins=0)
    with pytest.raises(RuntimeError):
        net.validate(per_bin=1)
    with pytest.raises(RuntimeError):
        net.validate(margin=0.5)


def test_validate_gives_up_with_the_wait():
    """A tensor-core wait that gives up (test hook) fails validation with
    ION_ETIMEOUT and leaves the installed bound; the next validation runs."""
    sd = W.argon_like()
    sp = gpu_species(sd)
    P = torch.tensor(rand_P(sd.Z, 8, 0.3), dtype=torch.float32, device="cuda")
    l2lo, l2hi = S.log2_range()
    norm = {"log2E_min": l2lo, "log2E_max": l2hi, "y_floor": -40.0,
            "y_mean": [0.0] * sd.Z, "y_scale": [1.0] * sd.Z}
    net = ionize.Surrogate(sp, P, norm)
    b0 = net.validate(nbins=32, per_bin=8)
    net.test_timeout(True)
    try:
        with pytest.raises(RuntimeError, match="gave up"):
            net.validate(nbins=16, per_bin=8)
    finally:
        net.test_timeout(False)
    b1 = net.validate(nbins=32, per_bin=8)
    assert np.array_equal(b0, b1)
