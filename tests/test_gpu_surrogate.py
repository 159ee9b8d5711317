"""The rate surrogate: training kernels against the FP64 reference network,
the tensor-core inference against the CUDA-core forward pass, the trained
network against Eq. 1, and the surrogate step against the oracle."""
import math
import time

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as omlp
from paper_2202_10647_gb300 import ionize, surrogate as S, workloads as W
from test_gpu_step import check, gpu_species, oracle_species

pytestmark = pytest.mark.gpu


def rand_P(K, seed, scale=0.5):
    return np.random.default_rng(seed).normal(0.0, scale, omlp.nparams(K))


@pytest.mark.parametrize("K,B", [(18, 1000), (36, 777), (7, 4096), (63, 130)])
def test_loss_grad_matches_oracle(K, B):
    rng = np.random.default_rng(K)
    P = rand_P(K, K + 1)
    x = rng.uniform(-1, 1, B)
    t = rng.normal(0, 1, (B, K))
    L, g = omlp.loss_grad(P, K, x, t)
    Pd = torch.tensor(P, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    # the oracle on the float32-rounded inputs the GPU sees
    L32, g32 = omlp.loss_grad(Pd.double().cpu().numpy(), K, xd.double().cpu().numpy(),
                              td.double().cpu().numpy())
    loss, grad = ionize.mlp_loss_grad(Pd, K, xd, td)
    assert float(loss) == pytest.approx(L32, rel=2e-5)
    gg = grad.double().cpu().numpy()
    assert np.abs(gg - g32).max() <= 2e-5 * np.abs(g32).max(), np.abs(gg - g32).max()
    # deterministic: the same call gives the same bits
    _, grad2 = ionize.mlp_loss_grad(Pd, K, xd, td)
    assert torch.equal(grad, grad2)
    # the inference arithmetic (bf16, straight-through) stays close
    _, gq = ionize.mlp_loss_grad(Pd, K, xd, td, flags=ionize.ION_MLP_BF16)
    assert float((gq - grad).abs().max()) <= 0.05 * float(grad.abs().max())


def test_forward_and_adam_match_oracle():
    K, B = 18, 513
    rng = np.random.default_rng(2)
    P = rand_P(K, 3)
    x = rng.uniform(-1, 1, B)
    Pd = torch.tensor(P, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    y, _ = omlp.forward(Pd.double().cpu().numpy(), K, xd.double().cpu().numpy())
    yg = ionize.mlp_forward(Pd, K, xd).double().cpu().numpy()
    assert np.abs(yg - y).max() <= 1e-5 * max(1.0, np.abs(y).max())
    # three Adam steps
    g = [rng.normal(size=P.size) for _ in range(3)]
    Po, m, v = Pd.double().cpu().numpy(), np.zeros(P.size), np.zeros(P.size)
    md, vd = torch.zeros_like(Pd), torch.zeros_like(Pd)
    for s in range(1, 4):
        gd = torch.tensor(g[s - 1], dtype=torch.float32, device="cuda")
        Po, m, v = omlp.adam(Po, gd.double().cpu().numpy(), m, v, 1e-2, 0.9, 0.999, 1e-8, s)
        ionize.mlp_adam(Pd, gd, md, vd, 1e-2, s)
    assert np.abs(Pd.double().cpu().numpy() - Po).max() <= 2e-6 * np.abs(Po).max()


@pytest.mark.parametrize("Z,n", [(7, 1000), (18, 300_000), (36, 4099), (63, 257)])
def test_tensor_core_inference_matches_cuda_core_forward(Z, n):
    """The tcgen05 kernel (bf16-pair operands, FP32 accumulators in tensor
    memory) against ion_mlp_forward in the same arithmetic on CUDA cores:
    equal up to the accumulation order and the lo*lo' products the tensor
    cores leave out."""
    sd = W.synthetic_ladder(Z, 90 + Z)
    sp = gpu_species(sd)
    P = torch.tensor(rand_P(Z, Z, 0.3), dtype=torch.float32, device="cuda")
    l2lo, l2hi = S.log2_range()
    norm = {"log2E_min": l2lo, "log2E_max": l2hi, "y_floor": -1000.0,
            "y_mean": [0.0] * Z, "y_scale": [1.0] * Z}
    net = ionize.Surrogate(sp, P, norm)
    g = torch.Generator(device="cuda").manual_seed(Z)
    E = torch.exp2(l2lo + (l2hi - l2lo) * torch.rand(n, generator=g, device="cuda"))
    Wn = net.rates(E)  # 2^y
    y_tc = torch.log2(Wn.double()).T
    x = S.scaled_input(E, l2lo, l2hi)
    y_cc = ionize.mlp_forward(P, Z, x, flags=ionize.ION_MLP_BF16).double()
    d = (y_tc - y_cc).abs()
    y32 = ionize.mlp_forward(P, Z, x).double()
    d32 = (y_tc - y32).abs()
    print(f"Z={Z}: |tensor cores - CUDA-core inference arithmetic| max {float(d.max()):.2e}, "
          f"median {float(d.median()):.2e}; against plain FP32 max {float(d32.max()):.2e}")
    assert float(d.max()) <= 2e-4, float(d.max())
    assert float(d.median()) <= 1e-5, float(d.median())
    # against plain FP32 (tanhf, no rounding): the SFU tanh's error only
    assert float(d32.max()) <= 2e-3


def bf16(a):
    """Round to bfloat16 (through float32, nearest even), as the kernel's
    conversions do; returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_pair(a):
    """The value a bf16 pair carries: hi = bf16(a), lo = bf16(a - hi), hi + lo
    (the rounding of a - hi in float32, as the kernel forms it)."""
    hi = bf16(a)
    d = (np.asarray(a, dtype=np.float32).astype(np.float64) - hi).astype(np.float32)
    return hi + bf16(d)


def forward_bf16(P, K, x):
    """The FP64 reference network (oracle/mlp.py) with the tensor-core
    arithmetic's roundings written in: W2, W3 and the hidden activations h1
    and h2 as bf16 pairs (hi + lo) before each product, the products summed
    in FP64 (the kernel sums hi*hi' + hi*lo' + lo*hi' in FP32)."""
    W1, b1, W2, b2, W3, b3 = omlp.unpack(P, K)
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    h1 = bf16_pair(omlp.gelu(x[:, None] * W1[None, :] + b1[None, :]))
    h2 = bf16_pair(omlp.gelu(h1 @ bf16_pair(W2).T + b2[None, :]))
    return h2 @ bf16_pair(W3).T + b3[None, :]


# deviation of the tensor-core outputs from the bf16-pair reference (outputs
# of order one): per output, at the 99th percentile, in the median (measured
# on the GB300: at most 4.0e-5, 1.4e-5 and 2.8e-6 over Z = 7, 18, 36, 63)
TC_MAX, TC_P99, TC_MEDIAN = 2e-4, 5e-5, 1e-5


@pytest.mark.parametrize("Z,n", [(7, 4099), (18, 20000), (36, 4099), (63, 1031)])
def test_tensor_core_network_matches_oracle_with_bf16_rounding(Z, n):
    """The tcgen05 network element by element against the FP64 reference
    network with the bf16-pair rounding of W2, W3, h1 and h2 written in.
    What is left is the SFU tanh of the GELU (tanh.approx.f32, relative error
    up to about 2^-11), the dropped lo*lo' products (about 2^-16 relative)
    and the FP32 sums."""
    sd = W.synthetic_ladder(Z, 90 + Z)
    sp = gpu_species(sd)
    P32 = torch.tensor(rand_P(Z, 7 * Z, 0.3), dtype=torch.float32)
    P = P32.cuda()
    l2lo, l2hi = S.log2_range()
    norm = {"log2E_min": l2lo, "log2E_max": l2hi, "y_floor": -1000.0,
            "y_mean": [0.0] * Z, "y_scale": [1.0] * Z}
    net = ionize.Surrogate(sp, P, norm)
    E = torch.exp2(l2lo + (l2hi - l2lo) * W.uniform(Z, 9, torch.arange(n))).to(torch.float32)
    y_tc = np.log2(net.rates(E.cuda()).double().cpu().numpy()).T
    x = np.clip((2.0 * (np.log2(E.double().numpy()) - l2lo) / (l2hi - l2lo) - 1.0), -1.0, 1.0)
    Pd = P32.double().numpy()
    want = forward_bf16(Pd, Z, x)
    d = np.abs(y_tc - want)
    plain = np.abs(y_tc - omlp.forward(Pd, Z, x)[0])
    print(f"Z={Z}: |tensor cores - bf16 reference| max {d.max():.2e}, p99 "
          f"{np.quantile(d, 0.99):.2e}, median {np.median(d):.2e}; against the plain "
          f"FP64 network max {plain.max():.2e}, median {np.median(plain):.2e}")
    assert d.max() <= TC_MAX
    assert np.quantile(d, 0.99) <= TC_P99
    assert np.median(d) <= TC_MEDIAN


@pytest.fixture(scope="module")
def argon_net():
    sd = W.argon_like()
    sp = gpu_species(sd)
    t0 = time.time()
    net, tr, bound = S.build(sp)
    torch.cuda.synchronize()
    print(f"\ntrained in {time.time() - t0:.1f} s; loss {tr.losses[-1]}")
    return sd, sp, net, tr, bound


def test_trained_network_accuracy(argon_net):
    """The trained network's rates against the oracle's Eq. 1 on fresh
    inputs, and its bound holds there."""
    sd, sp, net, tr, bound = argon_net
    assert tr.losses[-1][1] < 1e-4, tr.losses
    n = 20000
    E = torch.pow(10.0, 1.0 + 4.0 * W.uniform(77, 1, torch.arange(n))).to(torch.float32)
    Wn = net.rates(E.cuda()).double().cpu().numpy()
    osp = oracle_species(sd)
    Wo = oracle.rates(osp, E.double().numpy(), 0, sd.Z)
    big = Wo * 0.05 > 1e-12
    rel = np.abs(Wn[big] / Wo[big] - 1.0)
    print(f"max rel rate error {rel.max():.3e}, median {np.median(rel):.3e}")
    # the bf16-pair arithmetic leaves the training error: below 1 % in the
    # median (single bf16 operands gave about 2 %)
    assert np.median(rel) < 0.01, np.median(rel)
    l2 = np.log2(E.double().numpy())
    lo, hi = S.log2_range()
    nb = bound.shape[0]
    b = np.clip(np.floor((l2 - lo) / (hi - lo) * nb).astype(int), 0, nb - 1)
    yn = np.maximum(np.log2(np.maximum(Wn, 1e-300)), S.Y_FLOOR)
    yo = np.maximum(np.log2(np.maximum(Wo, 1e-300)), S.Y_FLOOR)
    viol = np.abs(yn - yo) > bound[b].T
    assert viol.mean() < 1e-3, viol.mean()


def test_surrogate_step_matches_oracle(argon_net):
    """ion_step_surrogate on the Ar-like lognormal workload: every cell within
    the FP32 bar of the oracle (the bound keeps the network's rate error
    below pop_tol in the populations)."""
    sd, sp, net, tr, bound = argon_net
    wl = W.ladder_cells(sd, 40000, 21)
    n = wl.ncells
    E, N, lo, hi = wl.E.cuda(), wl.N.cuda(), wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne = torch.zeros(n, device="cuda")
    ws = net.step(E, N, lo, hi, 0.05, dne, pop_tol=1e-6)
    n_net, n_plain, timeout = ionize.surrogate_counters(ws)
    assert timeout == 0
    No, loo, hio, dneo = oracle.step(oracle_species(sd), wl.E.double().numpy(),
                                     wl.N[:, :n].double().numpy(), 0.05, wl.lo.numpy(),
                                     wl.hi.numpy())
    out = dict(N=N.double().cpu().numpy(), lo=lo.cpu().numpy(), hi=hi.cpu().numpy(),
               dne=dne.double().cpu().numpy())
    check(out, dict(N=No, lo=loo, hi=hio, dne=dneo), wl.lo, wl.hi,
          ionize.ION_F32, sd=sd, E=wl.E.double().numpy())
    print(f"cells on the network's rates: {n_net} of {n}; on Eq. 1: {n_plain}")
    assert n_net + n_plain <= n


def test_surrogate_everywhere_reports_its_error(argon_net):
    """With no bound (pop_tol huge) every in-range cell whose rates all have
    W dt <= 1 takes the network's rates (cells with larger rates always take
    Eq. 1): populations stay conserved and non-negative, and the error
    against the oracle is what the rate error implies."""
    sd, sp, net, tr, bound = argon_net
    wl = W.ladder_cells(sd, 20000, 22)
    n = wl.ncells
    E, N, lo, hi = wl.E.cuda(), wl.N.cuda(), wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne = torch.zeros(n, device="cuda")
    ws = net.step(E, N, lo, hi, 0.05, dne, pop_tol=1e30)
    n_net, n_plain, timeout = ionize.surrogate_counters(ws)
    w = (wl.hi.long() - wl.lo.long() + 1)
    assert timeout == 0 and n_net > 0
    assert n_net + n_plain == int((w >= 2).sum())
    tot = N[:, :n].double().sum(0)
    assert float((tot - wl.N[:, :n].double().sum(0).cuda()).abs().max()) <= 1e-6
    assert float(N.min()) >= -1e-6
    No, _, _, _ = oracle.step(oracle_species(sd), wl.E.double().numpy(),
                              wl.N[:, :n].double().numpy(), 0.05, wl.lo.numpy(), wl.hi.numpy())
    err = float(np.abs(N[:, :n].double().cpu().numpy() - No).max())
    print(f"population error with the network everywhere: {err:.3e}")
    assert err < 0.5


def test_surrogate_gain(argon_net):
    """What the network gains over the plain rates of Eq. 1 on the same
    cells: time per step of both forms, and how many cells the network may
    serve at the FP32 accuracy bar (it is reported, not required to win)."""
    sd, sp, net, tr, bound = argon_net
    wl = W.ladder_cells(sd, 2_000_000, 23, device="cuda")
    n = wl.ncells
    dne = torch.zeros(n, device="cuda")
    ws = ionize.workspace(n)
    N0, lo0, hi0 = wl.N.clone(), wl.lo.clone(), wl.hi.clone()

    def timed(fn, reps=10):
        ts = []
        for _ in range(reps + 2):
            wl.N.copy_(N0)
            wl.lo.copy_(lo0)
            wl.hi.copy_(hi0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts[2:]))

    t_plain = timed(lambda: ionize.step(sp, wl.E, wl.N, wl.lo, wl.hi, 0.05, dne, ws=ws))
    t_net = timed(lambda: net.step(wl.E, wl.N, wl.lo, wl.hi, 0.05, dne, ws=ws))
    n_net, n_plain, _ = ionize.surrogate_counters(ws)
    print(f"plain FP32 {t_plain:.3f} ms, surrogate {t_net:.3f} ms "
          f"(gain {t_plain / t_net:.2f}x); network rates for {n_net / n:.1%} of the cells")
    assert t_net > 0 and t_plain > 0


def test_full_size_surrogate_sampled(argon_net):
    """The surrogate form on the 33.5M-cell Ar-like workload: sampled cells
    within the FP32 bar of the oracle, conservation over every cell."""
    sd, sp, net, tr, bound = argon_net
    dev = "cuda"
    wl = W.ladder_cells(sd, 33_554_432, 4, device=dev)
    n = wl.ncells
    rng = np.random.default_rng(12)
    ix = torch.tensor(np.sort(rng.choice(n, 4000, replace=False)), device=dev)
    Es, Ns = wl.E[ix].double().cpu().numpy(), wl.N[:, ix].double().cpu().numpy()
    ls, hs = wl.lo[ix].cpu().numpy(), wl.hi[ix].cpu().numpy()
    tot0 = wl.N[:, :n].double().sum(0)
    dne = torch.empty(n, device=dev)
    ws = net.step(wl.E, wl.N, wl.lo, wl.hi, 0.05, dne)
    torch.cuda.synchronize()
    n_net, n_plain, timeout = ionize.surrogate_counters(ws)
    assert timeout == 0 and n_net > 0
    assert float((wl.N[:, :n].double().sum(0) - tot0).abs().max()) <= 1e-6
    No, _, _, _ = oracle.step(oracle_species(sd), Es, Ns, 0.05, ls, hs)
    assert np.abs(wl.N[:, ix].double().cpu().numpy() - No).max() <= 2e-6


def test_bounded_wait_gives_up_and_frees_tensor_memory():
    """The surrogate kernels' bounded mbarrier wait, made to give up by the
    test hook (the first wait of each tile polls a barrier nothing arrives
    at): the step leaves every cell untouched and sets header word 5, the
    rates kernel writes NaN, and each CTA still waits for the matrix
    products it skipped and frees its tensor memory, so that the next normal
    calls run and give the plain step's result."""
    sd = W.argon_like()
    sp = gpu_species(sd)
    P = torch.tensor(rand_P(sd.Z, 11, 0.3), dtype=torch.float32, device="cuda")
    l2lo, l2hi = S.log2_range()
    norm = {"log2E_min": l2lo, "log2E_max": l2hi, "y_floor": -40.0,
            "y_mean": [0.0] * sd.Z, "y_scale": [1.0] * sd.Z}
    net = ionize.Surrogate(sp, P, norm)
    wl = W.ladder_cells(sd, 50000, 25)
    n = wl.ncells
    E = wl.E.cuda()
    net.test_timeout(True)
    try:
        for rep in range(2):
            N, lo, hi = wl.N.cuda(), wl.lo.clone().cuda(), wl.hi.clone().cuda()
            dne = torch.full((n,), 5.0, device="cuda")
            ws = net.step(E, N, lo, hi, 0.05, dne, pop_tol=1.0)
            torch.cuda.synchronize()
            n_net, n_plain, timeout = ionize.surrogate_counters(ws)
            assert timeout > 0 and n_net == 0
            assert torch.equal(N.cpu(), wl.N) and torch.equal(lo.cpu(), wl.lo)
            assert torch.equal(hi.cpu(), wl.hi) and bool(torch.all(dne == 5.0))
            Wn = net.rates(E[:4096].contiguous())
            torch.cuda.synchronize()
            assert bool(torch.isnan(Wn).all())
    finally:
        net.test_timeout(False)
    # normal calls afterwards: tensor memory was freed, the network runs
    N, lo, hi = wl.N.cuda(), wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne = torch.zeros(n, device="cuda")
    ws = net.step(E, N, lo, hi, 0.05, dne, pop_tol=0.0)
    Wn = net.rates(E[:4096].contiguous())
    N2, lo2, hi2 = wl.N.cuda(), wl.lo.clone().cuda(), wl.hi.clone().cuda()
    dne2 = torch.zeros(n, device="cuda")
    ionize.step(sp, E, N2, lo2, hi2, 0.05, dne2)
    torch.cuda.synchronize()
    assert ionize.surrogate_counters(ws)[2] == 0
    assert bool(torch.isfinite(Wn).all())
    assert float((N - N2).abs().max()) <= 2e-6
    assert torch.equal(lo, lo2) and torch.equal(hi, hi2)
