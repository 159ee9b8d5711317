"""The adaptive window policy (ION_WINDOW_ADAPTIVE) on the GPU against the
oracle with the same policy: FP32, FP64, batched and surrogate paths."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_10647_gb300 import ionize, workloads as W
from test_gpu_step import TOL, gpu_species, oracle_species, window_ties

pytestmark = pytest.mark.gpu

POLICIES = [dict(w_min=2, w_max=6, eps_grow=1e-6), dict(w_min=3, w_max=5, eps_grow=1e-4)]


def run_oracle(sd, E, N, lo, hi, win, dt=0.05):
    return oracle.step(oracle_species(sd), E, N, dt, lo, hi, policy=oracle.WINDOW_ADAPTIVE,
                       w_min=win["w_min"], w_max=win["w_max"], eps_grow=win["eps_grow"])


def check_policy(out, ref, lo, hi, win, tol, sd, E, f32):
    """Populations within tol, dne within (w-1) tol, windows by the rule on
    the GPU's own values and, where they differ from the oracle's, through a
    compared population on the other side of its threshold (window_ties).
    Returns the number of such cells."""
    Ng, lg, hg, dg = out
    No, lo_, ho, do = ref
    assert np.abs(Ng - No).max() <= tol, np.abs(Ng - No).max()
    w = hi.astype(int) - lo.astype(int) + 1
    derr = np.abs(dg - do)
    assert np.all(derr <= np.maximum(w - 1, 1) * tol), derr.max()
    return window_ties(sd, E, Ng, No, lo, hi, lg, hg, lo_, ho, 1e-6, f32, policy=win)


@pytest.mark.parametrize("win", POLICIES)
@pytest.mark.parametrize("flags", [ionize.ION_F32, ionize.ION_F64_PLAIN])
@pytest.mark.parametrize("name", ["N", "argon_like", "krypton_like"])
def test_adaptive_policy_matches_oracle(win, flags, name):
    sd = {"N": W.nitrogen(), "argon_like": W.argon_like(),
          "krypton_like": W.krypton_like()}[name]
    wl = W.ladder_cells(sd, 9001, 41)
    n = wl.ncells
    f64 = bool(flags & ionize.ION_F64_PLAIN)
    dt_ = torch.float64 if f64 else torch.float32
    sp = gpu_species(sd)
    E, N = wl.E.to(dt_).cuda(), wl.N.to(dt_).cuda()
    lo, hi = wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne = torch.zeros(n, dtype=dt_, device="cuda")
    ionize.step(sp, E, N, lo, hi, 0.05, dne, flags=flags, window=win)
    ref = run_oracle(sd, wl.E.to(dt_).double().numpy(), wl.N[:, :n].to(dt_).double().numpy(),
                     wl.lo.numpy(), wl.hi.numpy(), win)
    out = (N[:, :n].double().cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy(),
           dne.double().cpu().numpy())
    ties = check_policy(out, ref, wl.lo.numpy(), wl.hi.numpy(), win, TOL[flags], sd,
                        wl.E.to(dt_).double().numpy(), not f64)
    assert ties <= n // 1000
    # the policy did something: some windows changed width
    w0 = wl.hi.numpy().astype(int) - wl.lo.numpy().astype(int)
    w1 = out[2].astype(int) - out[1].astype(int)
    assert (w0 != w1).any()


def test_adaptive_policy_batched_and_surrogate():
    """The batched launch and the surrogate step apply the same rule."""
    win = POLICIES[0]
    sd = W.argon_like()
    sp = gpu_species(sd)
    wl = W.ladder_cells(sd, 5000, 43)
    n = wl.ncells
    ref = run_oracle(sd, wl.E.double().numpy(), wl.N[:, :n].double().numpy(),
                     wl.lo.numpy(), wl.hi.numpy(), win)
    for shape in [(1, 2, 0), (2, 8, 0), (4, 4, 0)]:
        E, N = wl.E.cuda(), wl.N.cuda()
        lo, hi = wl.lo.clone().cuda(), wl.hi.clone().cuda()
        dne = torch.zeros(n, device="cuda")
        ionize.step_batched([(sp, E, N, lo, hi, dne)], 0.05, shape=shape, window=win)
        out = (N[:, :n].double().cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy(),
               dne.double().cpu().numpy())
        ties = check_policy(out, ref, wl.lo.numpy(), wl.hi.numpy(), win, TOL[ionize.ION_F32],
                            sd, wl.E.double().numpy(), True)
        assert ties <= n // 1000
    # surrogate: an untrained network trusted nowhere (pop_tol 0), so every
    # cell takes Eq. 1 and the result is the plain step's
    P = torch.zeros(ionize.mlp_nparams(sd.Z), device="cuda")
    norm = {"log2E_min": 3.0, "log2E_max": 17.0, "y_floor": -40.0,
            "y_mean": [0.0] * sd.Z, "y_scale": [1.0] * sd.Z}
    net = ionize.Surrogate(sp, P, norm)
    E, N = wl.E.cuda(), wl.N.cuda()
    lo, hi = wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne = torch.zeros(n, device="cuda")
    net.step(E, N, lo, hi, 0.05, dne, pop_tol=0.0, window=win)
    out = (N[:, :n].double().cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy(),
           dne.double().cpu().numpy())
    ties = check_policy(out, ref, wl.lo.numpy(), wl.hi.numpy(), win, TOL[ionize.ION_F32], sd,
                        wl.E.double().numpy(), True)
    assert ties <= n // 1000


def test_adaptive_policy_argument_checks():
    sd = W.nitrogen()
    sp = gpu_species(sd)
    E = torch.zeros(8, device="cuda")
    N = torch.zeros((8, 8), device="cuda")
    lo = torch.zeros(8, dtype=torch.uint8, device="cuda")
    hi = torch.full((8,), 3, dtype=torch.uint8, device="cuda")
    dne = torch.zeros(8, device="cuda")
    for bad in (dict(w_min=1, w_max=4), dict(w_min=4, w_max=3), dict(w_min=2, w_max=7),
                dict(w_min=2, w_max=6, eps_grow=-1.0)):
        with pytest.raises(ionize.IonError):
            ionize.step(sp, E, N, lo, hi, 0.05, dne, window=bad)
