"""Training and validation of the rate surrogate (the learned alternative to
evaluating Eq. 1 per state).

Pipeline (every arithmetic step runs in the library's kernels; torch holds
the tensors, draws the batch order and gathers the batches):

  training_set   |E| with log10|E| ~ U[1, 5] (GV/m) from the seeded input
                 generator, targets max(log2 W_k, y_floor) for every state
                 from ion_log2_rates (Eq. 1 in FP64, in its log2 form).
  train          inputs from ion_mlp_inputs, targets standardized per state
                 by ion_mlp_standardize; Adam on the mean squared error
                 (ion_mlp_loss_grad, ion_mlp_adam), the last steps in the
                 inference arithmetic (bf16 pairs, SFU tanh; straight-through).
  build          train, then ion_surrogate_validate: the tensor-core network
                 against Eq. 1 in FP64 on a dense grid, per input bin and
                 state the largest |log2 W_net - log2 W| (both clamped at
                 y_floor), widened by a safety margin, installed as the
                 bound that ion_step_surrogate trusts the network by.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import ionize
from . import workloads as W

LOG10E_RANGE = (1.0, 5.0)
Y_FLOOR = -40.0  # log2 W [1/fs]; W dt < 5e-14 at dt = 0.05 fs: no population sees it


def log2_range(log10E=LOG10E_RANGE):
    return (log10E[0] * math.log2(10.0), log10E[1] * math.log2(10.0))


def scaled_input(E: torch.Tensor, l2lo: float, l2hi: float) -> torch.Tensor:
    """x = clamp(2 (log2|E| - l2lo)/(l2hi - l2lo) - 1, -1, 1), float32
    (ion_mlp_inputs)."""
    return ionize.mlp_inputs(E.to(torch.float32).contiguous(), l2lo, l2hi)


def plain_log2_rates(sp: ionize.Species, E: torch.Tensor, floor: float = Y_FLOOR):
    """max(log2 W_k(|E|), floor) for every state, (n, Z) float64, from
    ion_log2_rates (Eq. 1 in FP64)."""
    return ionize.log2_rates(sp, E.to(torch.float32).contiguous(), 0, sp.Z, floor)


def training_set(sp: ionize.Species, n: int = 1 << 20, seed: int = 11,
                 log10E=LOG10E_RANGE, device="cuda"):
    """(E float32 [n], log2 W float64 [n, Z])."""
    E = W.log_uniform_fields(seed, 60, n, log10E[0], log10E[1], device=device)
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


def train(sp: ionize.Species, n: int = 1 << 20, steps: int = 40000, batch: int = 8192,
          lr: float = 1e-2, lr_end: float = 3e-5, bf16_steps: int = 2000, seed: int = 11,
          device="cuda", E=None, Y=None) -> Trained:
    """Adam with a cosine learning-rate schedule from lr to lr_end; the last
    bf16_steps steps use the inference arithmetic."""
    Z = sp.Z
    if E is None:
        E, Y = training_set(sp, n, seed, device=device)
    l2lo, l2hi = log2_range()
    x = scaled_input(E, l2lo, l2hi)
    mean, scale, T = ionize.mlp_standardize(Y.contiguous(), 1e-3)
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


def build(sp: ionize.Species, steps: int = 40000, nbins: int = 4096, seed: int = 11,
          device="cuda", per_bin: int = 64, margin: float = 1.25, floor_add: float = 2e-3,
          **kw):
    """Train, create and validate the surrogate: (Surrogate, Trained, bound),
    bound the (nbins, Z) array of log2-error bounds it trusts the network by
    (ion_surrogate_validate: per bin the largest |log2 W_net - log2 W| over
    per_bin points, times margin, plus floor_add)."""
    tr = train(sp, steps=steps, seed=seed, device=device, **kw)
    net = ionize.Surrogate(sp, tr.P, tr.norm, None)
    bound = net.validate(nbins=nbins, per_bin=per_bin, margin=margin, floor_add=floor_add)
    return net, tr, bound
