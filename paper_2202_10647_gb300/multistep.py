"""Multi-step runs of ion_step captured in one CUDA graph.

A PIC code calls the ionization step once per time step with that step's
field.  StepGraph records K such calls (and, optionally, the conservation
diagnostic after each) into one CUDA graph, so that replaying K steps costs
one graph launch instead of K times three kernel launches and their host
argument checks.  Argument checking happens once, during capture; the graph
then replays the same device pointers: the field tensors, populations,
windows, dne and workspace must stay alive and in place.
"""
from __future__ import annotations

import torch

from . import ionize


def _prime(sp: ionize.Species, flags: int, device) -> None:
    """One eager step on a few private cells, so that the library's one-time
    per-kernel set-up (shared-memory limits, occupancy) is done before any
    capture."""
    n = 256
    f64 = bool(flags & ionize.ION_F64_PLAIN)
    dt = torch.float64 if f64 else torch.float32
    E = torch.full((n,), 100.0, dtype=dt, device=device)
    N = torch.zeros((sp.Z + 1, n), dtype=dt, device=device)
    N[0] = 1.0
    lo = torch.zeros(n, dtype=torch.uint8, device=device)
    hi = torch.full((n,), min(sp.Z, 3), dtype=torch.uint8, device=device)
    dne = torch.empty(n, dtype=dt, device=device)
    ionize.step(sp, E, N, lo, hi, 0.05, dne, flags=flags)
    torch.cuda.synchronize(device)


class StepGraph:
    """K = len(fields) steps: step s advances N, k_lo, k_hi by dt with the
    field fields[s] and writes dne (ion_step, or ion_step_surrogate when a
    surrogate is given; `window` selects the adaptive window policy, as in
    ionize.step).

    conservation:
      True or "full"  after every step, ion_conservation reads all Z+1
                      planes: self.cons[s] = max_c |sum_k N_k - 1| after
                      step s;
      "fused"         (ion_step only) every step measures its own change of
                      each cell's total, max_c |sum_k N'_k - sum_k N_k|
                      (ION_CONSERVATION_CHECK; the states outside a window
                      are not touched), into self.cons[s]; ion_conservation
                      runs after the first and the last step only, into
                      self.cons_full[0] and self.cons_full[1].  The total
                      after step s then lies within sum_{t<=s} cons[t] of
                      its value before the first step;
      False           no check."""

    def __init__(self, sp: ionize.Species, fields, N: torch.Tensor, k_lo: torch.Tensor,
                 k_hi: torch.Tensor, dne: torch.Tensor, dt: float,
                 ws: torch.Tensor | None = None, flags: int = ionize.ION_F32,
                 conservation: bool | str = True, eps_shift: float = 1e-6,
                 degen_gap: float = 1e-3, surrogate: ionize.Surrogate | None = None,
                 pop_tol: float = 1e-6, window: dict | None = None):
        if not fields:
            raise ValueError("at least one field")
        dev = N.device
        n = fields[0].numel()
        if any(f.numel() != n for f in fields):
            raise ValueError("every field must have the same number of cells")
        self.steps = len(fields)
        self.fields = list(fields)
        self.ws = ws if ws is not None else ionize.workspace(n, flags, dev)
        self.cons = torch.zeros(self.steps, dtype=torch.float32, device=dev)
        self.cons_full = torch.zeros(2, dtype=torch.float32, device=dev)
        fused = conservation == "fused"
        if fused and surrogate is not None:
            raise ValueError("the fused check serves ion_step; use conservation='full'")
        step_flags = flags | (ionize.ION_CONSERVATION_CHECK if fused else 0)
        # the step's own measure: word 10 of the workspace header
        change = self.ws[40:44].view(torch.float32)
        _prime(sp, flags, dev)
        _prime(sp, step_flags, dev)
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.graph(self.graph, stream=side):
            for s, E in enumerate(self.fields):
                if surrogate is None:
                    ionize.step(sp, E, N, k_lo, k_hi, dt, dne, ws=self.ws, eps_shift=eps_shift,
                                degen_gap=degen_gap, flags=step_flags, window=window)
                else:
                    surrogate.step(E, N, k_lo, k_hi, dt, dne, ws=self.ws, eps_shift=eps_shift,
                                   degen_gap=degen_gap, pop_tol=pop_tol, window=window)
                if fused:
                    self.cons[s:s + 1].copy_(change)
                    if s == 0:
                        ionize.conservation(N, self.cons_full[0:1], ncells=n)
                    if s == self.steps - 1:
                        ionize.conservation(N, self.cons_full[1:2], ncells=n)
                elif conservation:
                    ionize.conservation(N, self.cons[s:s + 1], ncells=n)
        torch.cuda.current_stream(dev).wait_stream(side)
        self.conservation = conservation

    def replay(self) -> None:
        """Enqueue the K steps on the current stream."""
        self.graph.replay()
