"""Training and validation of the rate surrogate (the learned alternative to
evaluating Eq. 1 per state).

Pipeline (every arithmetic step on the GPU runs in the library's kernels;
torch only holds the tensors, draws the batch order and does the elementwise
scaling of inputs and targets):

  training_set   |E| with log10|E| ~ U[1, 5] (GV/m) from the counter-based
                 hash, the rates of every state from ion_rates in FP64 (the
                 plain evaluation of Eq. 1), targets log2 W clamped below at
                 y_floor.
  train          Adam on the mean squared error of the standardized targets
                 (ion_mlp_loss_grad, ion_mlp_adam), the last steps in the
                 inference arithmetic (bf16, straight-through).
  error_bound    the tensor-core network (ion_surrogate_rates) against
                 ion_rates in FP64 on a dense grid: per input bin and state,
                 the largest |log2 W_net - log2 W| (both clamped at y_floor),
                 widened by a safety margin.
  build          train, bound, and return the ion_surrogate that
                 ion_step_surrogate uses.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import ionize
from . import workloads as W

LOG10E_RANGE = (1.0, 5.0)
Y_FLOOR = -40.0  # log2 W [1/fs]; W dt < 5e-14 at dt = 0.05 fs: no population sees it


def log2_range(log10E=LOG10E_RANGE):
    return (log10E[0] * math.log2(10.0), log10E[1] * math.log2(10.0))


def scaled_input(E: torch.Tensor, l2lo: float, l2hi: float) -> torch.Tensor:
    """x = 2 (log2|E| - l2lo)/(l2hi - l2lo) - 1, float32."""
    l2 = torch.log2(E.abs().double())
    return (2.0 * (l2 - l2lo) / (l2hi - l2lo) - 1.0).to(torch.float32)


def plain_log2_rates(sp: ionize.Species, E: torch.Tensor, floor: float = Y_FLOOR):
    """max(log2 W_k(|E|), floor) for every state, (n, Z) float64, from
    ion_rates in FP64."""
    Wt = ionize.rates(sp, E.double().contiguous(), 0, sp.Z)  # (Z, n)
    return torch.log2(Wt).clamp(min=floor).T.contiguous()


def training_set(sp: ionize.Species, n: int = 1 << 20, seed: int = 11,
                 log10E=LOG10E_RANGE, device="cuda"):
    """(E float32 [n], log2 W float64 [n, Z])."""
    idx = torch.arange(n, device=device, dtype=torch.int64)
    u = W.uniform(seed, 60, idx)
    E = torch.pow(10.0, log10E[0] + (log10E[1] - log10E[0]) * u).to(torch.float32)
    return E, plain_log2_rates(sp, E)


def init_params(K: int, seed: int = 12, device="cuda") -> torch.Tensor:
    """Layer 1 spreads the kinks of its GELUs over the input range; layers 2
    and 3 start near the scale that keeps activations of order one."""
    H = ionize.ION_MLP_HIDDEN
    g = torch.Generator().manual_seed(seed)
    W1 = torch.randn(H, generator=g) * 4.0
    b1 = (torch.rand(H, generator=g) * 2 - 1) * 4.0
    W2 = torch.randn(H, H, generator=g) * math.sqrt(2.0 / H)
    b2 = torch.zeros(H)
    W3 = torch.randn(K, H, generator=g) * math.sqrt(1.0 / H)
    b3 = torch.zeros(K)
    P = torch.cat([W1, b1, W2.reshape(-1), b2, W3.reshape(-1), b3]).to(torch.float32)
    assert P.numel() == ionize.mlp_nparams(K)
    return P.to(device)


@dataclass
class Trained:
    P: torch.Tensor
    norm: dict
    losses: list
    steps: int


def train(sp: ionize.Species, n: int = 1 << 20, steps: int = 8000, batch: int = 8192,
          lr: float = 3e-3, lr_end: float = 3e-5, bf16_steps: int = 1500, seed: int = 11,
          device="cuda", E=None, Y=None) -> Trained:
    """Adam with a cosine learning-rate schedule from lr to lr_end; the last
    bf16_steps steps use the inference arithmetic."""
    Z = sp.Z
    if E is None:
        E, Y = training_set(sp, n, seed, device=device)
    l2lo, l2hi = log2_range()
    x = scaled_input(E, l2lo, l2hi)
    mean = Y.mean(0)
    scale = Y.std(0).clamp(min=1e-3)
    T = ((Y - mean) / scale).to(torch.float32).contiguous()
    P = init_params(Z, seed + 1, device)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    grad = torch.empty_like(P)
    loss = torch.empty(1, dtype=torch.float32, device=device)
    ws = ionize.mlp_workspace(Z, batch, device)
    gen = torch.Generator(device=device).manual_seed(seed + 2)
    n = x.numel()
    perm = torch.randperm(n, generator=gen, device=device)
    pos = 0
    losses = []
    xb = torch.empty(batch, dtype=torch.float32, device=device)
    tb = torch.empty((batch, Z), dtype=torch.float32, device=device)
    for s in range(1, steps + 1):
        if pos + batch > n:
            perm = torch.randperm(n, generator=gen, device=device)
            pos = 0
        ix = perm[pos:pos + batch]
        pos += batch
        torch.index_select(x, 0, ix, out=xb)
        torch.index_select(T, 0, ix, out=tb)
        flags = ionize.ION_MLP_BF16 if s > steps - bf16_steps else 0
        ionize.mlp_loss_grad(P, Z, xb, tb, flags, grad=grad, loss=loss, ws=ws)
        cur = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * (s - 1) / steps))
        ionize.mlp_adam(P, grad, m, v, cur, s)
        if s % 200 == 0 or s == steps:
            losses.append((s, float(loss)))
    norm = {"log2E_min": l2lo, "log2E_max": l2hi, "y_floor": Y_FLOOR,
            "y_mean": [float(a) for a in mean.cpu()], "y_scale": [float(a) for a in scale.cpu()]}
    return Trained(P, norm, losses, steps)


def error_bound(sp: ionize.Species, net: ionize.Surrogate, nbins: int = 4096,
                per_bin: int = 64, margin: float = 1.25, floor_add: float = 2e-3,
                device="cuda"):
    """(nbins, Z) bound on |log2 W_net - log2 W| per input bin (both clamped
    at y_floor), from per_bin points of each bin: the observed maximum
    times `margin` plus `floor_add`."""
    l2lo, l2hi = log2_range()
    j = torch.arange(nbins * per_bin, device=device, dtype=torch.float64)
    # points at the bin edges and spread inside each bin
    l2 = l2lo + (l2hi - l2lo) * (torch.floor(j / per_bin) + (j % per_bin) / (per_bin - 1)) / nbins
    E = torch.exp2(l2).to(torch.float32)
    Wn = net.rates(E)  # (Z, n)
    yn = torch.log2(Wn.double()).clamp(min=Y_FLOOR).T
    yt = plain_log2_rates(sp, E)
    d = (yn - yt).abs().reshape(nbins, per_bin, sp.Z).amax(1)
    return (d * margin + floor_add).cpu().numpy().astype(np.float32)


def build(sp: ionize.Species, steps: int = 8000, nbins: int = 4096, seed: int = 11,
          device="cuda", **kw):
    """Train, bound and create the surrogate: (Surrogate, Trained, bound)."""
    tr = train(sp, steps=steps, seed=seed, device=device, **kw)
    raw = ionize.Surrogate(sp, tr.P, tr.norm, None)
    bound = error_bound(sp, raw, nbins=nbins, device=device)
    raw.close()
    return ionize.Surrogate(sp, tr.P, tr.norm, bound), tr, bound
