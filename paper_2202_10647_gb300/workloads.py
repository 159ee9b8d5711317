"""Seeded synthetic inputs of the ionization step (input recipes only).

This module holds no part of the method's arithmetic (no ADK rate, no
Bateman update).  It builds species data, field magnitudes, populations and
windows with torch ops that run on the CPU or the GPU; randomness comes from
a counter-based hash of (seed, stream, index), so a value depends only on
its seed and position.  Tests compare the CUDA path with the oracle on the
exact inputs the GPU saw (copied back), so CPU/GPU rounding differences of
the recipes themselves never enter a parity check.

Workloads (the sizes and distributions of the five benchmark configurations)
  nitrogen_pulse_2d   N, 128x128 cells, dx = 0.5 um, Gaussian pulse field
                      E0 exp(-y^2/w^2) exp(-((t - x/c) - t0)^2/tau^2) cos(wt).
  nitrogen_3d         N, 256x256x512 cells, one step; pulse envelope with a
                      per-8^3-block E0 ~ U[500, 4000] GV/m and |cos| phase;
                      windows of width 3-4 placed at the states the local
                      envelope is burning through; Dirichlet(1) populations
                      on the 2-3 lowest window states.
  mixed_batch         N (20M), Ar-like (Z=18, 8M), Kr-like (Z=36, 2M) cells,
                      lognormal |E| in [100, 5000] GV/m, widths 2-6.
  argon_surrogate     Ar-like ladder on 33.5M cells, lognormal |E|.
  krypton_beams       Kr-like ladder, 512x512x256 cells, |E| from 16 seeded
                      Gaussian beams, N_0 = 1 and window [0, 3] at t = 0.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import torch

_M32 = 0xFFFFFFFF
C_UM_PER_FS = 0.299792458  # speed of light, um/fs

# ---------------------------------------------------------------------------
# counter-based randomness
# ---------------------------------------------------------------------------


def _mul32(x: torch.Tensor, c: int) -> torch.Tensor:
    """(x * c) mod 2^32 for int64 tensors holding uint32 values."""
    lo, hi = c & 0xFFFF, c >> 16
    return (x * lo + (((x * hi) & 0xFFFF) << 16)) & _M32


def hash32(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """A 32-bit mix (Wellons' lowbias32 finalizer) of seed, stream and idx."""
    x = (idx.to(torch.int64) & _M32) ^ ((seed * 0x9E3779B1 + stream * 0x85EBCA77) & _M32)
    for _ in range(2):
        x = x ^ (x >> 16)
        x = _mul32(x, 0x7FEB352D)
        x = x ^ (x >> 15)
        x = _mul32(x, 0x846CA68B)
        x = x ^ (x >> 16)
    return x


def uniform(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Uniform float64 in (0, 1) from the top 24 bits of the hash."""
    h = hash32(seed, stream, idx)
    return ((h >> 8).to(torch.float64) + 0.5) * (1.0 / (1 << 24))


def normal(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Standard normal by Box-Muller from two hashed uniforms."""
    u1 = uniform(seed, 2 * stream, idx)
    u2 = uniform(seed, 2 * stream + 1, idx)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


def log_uniform_fields(seed: int, stream: int, n: int, log10_lo: float, log10_hi: float,
                       device="cpu") -> torch.Tensor:
    """n fields |E| in GV/m with log10|E| uniform in [log10_lo, log10_hi],
    float32 (the surrogate's training and test inputs)."""
    idx = torch.arange(n, device=device, dtype=torch.int64)
    u = uniform(seed, stream, idx)
    return torch.pow(10.0, log10_lo + (log10_hi - log10_lo) * u).to(torch.float32)


# ---------------------------------------------------------------------------
# species
# ---------------------------------------------------------------------------


@dataclass
class SpeciesData:
    name: str
    U: list  # eV, transition k -> k+1, k = 0..Z-1
    l: list
    m: list

    @property
    def Z(self) -> int:
        return len(self.U)


def nitrogen() -> SpeciesData:
    """N: potentials (eV) of N -> N+ ... N6+ -> N7+, l = 1 for the first
    three transitions (2p electrons) and l = 0 for the rest, m = 0."""
    return SpeciesData("N", [14.53, 29.60, 47.45, 77.47, 97.89, 552.07, 667.05],
                       [1, 1, 1, 0, 0, 0, 0], [0] * 7)


def synthetic_ladder(Z: int, seed: int, name: str = None) -> SpeciesData:
    """Monotone synthetic ladder: U_1 = 15 eV, U_{i+1} = U_i (1 + u) with
    u ~ U(0.08, 0.25) inside a shell and a jump by U(3, 5) after 8 and after
    18 electrons removed.  In each shell segment ([1..8], [9..18], [19..Z])
    the last two electrons removed are s (l = 0), the others p (l = 1); m = 0."""
    idx = torch.arange(Z, dtype=torch.int64)
    g = uniform(seed, 11, idx)
    j = uniform(seed, 12, idx)
    U = [15.0]
    for i in range(1, Z):
        if i in (8, 18):
            U.append(U[-1] * (3.0 + 2.0 * float(j[i])))
        else:
            U.append(U[-1] * (1.08 + 0.17 * float(g[i])))
    bounds = [(0, min(8, Z)), (8, min(18, Z)), (18, Z)]
    l = [1] * Z
    for a, b in bounds:
        for i in range(max(a, b - 2), b):
            l[i] = 0
    return SpeciesData(name or f"ladder{Z}", U, l, [0] * Z)


def argon_like() -> SpeciesData:
    return synthetic_ladder(18, seed=18, name="Ar-like")


def krypton_like() -> SpeciesData:
    return synthetic_ladder(36, seed=36, name="Kr-like")


_THRESH_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                            "window_thresholds.json")


def window_thresholds(name: str) -> list:
    """Field (GV/m) above which W_k dt = 0.05 fs exceeds 1, per state k of
    the named species.  Only shapes the synthetic window placement; written
    by oracle/make_window_thresholds.py."""
    with open(_THRESH_PATH) as f:
        return json.load(f)[name]


# ---------------------------------------------------------------------------
# a workload instance
# ---------------------------------------------------------------------------


@dataclass
class Workload:
    name: str
    species: SpeciesData
    E: torch.Tensor          # float32 [ncells]
    N: torch.Tensor          # float32 [Z+1, ld]
    lo: torch.Tensor         # uint8 [ncells]
    hi: torch.Tensor         # uint8 [ncells]
    dt: float = 0.05
    meta: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return self.E.numel()


def _padded(n: int, mult: int = 4) -> int:
    return (n + mult - 1) // mult * mult


def populations(seed: int, lo: torch.Tensor, p: torch.Tensor, Z: int, ld: int,
                dtype=torch.float32, cells: torch.Tensor | None = None) -> torch.Tensor:
    """Dirichlet(1) populations on states lo..lo+p-1 of each cell, 0 elsewhere,
    as SoA planes (Z+1, ld).  `cells` are the global cell indices that seed
    the draws (default 0..n-1)."""
    n = lo.numel()
    dev = lo.device
    idx = torch.arange(n, device=dev, dtype=torch.int64) if cells is None else cells
    N = torch.zeros((Z + 1, ld), dtype=torch.float64, device=dev)
    pmax = int(p.max()) if n else 0
    g = []
    for r in range(pmax):
        x = -torch.log(uniform(seed, 100 + r, idx))
        g.append(torch.where(r < p, x, torch.zeros_like(x)))
    tot = torch.stack(g).sum(0) if g else torch.ones(n, device=dev, dtype=torch.float64)
    for r in range(pmax):
        k = (lo.to(torch.int64) + r).clamp(max=Z)
        val = torch.where(r < p, g[r] / tot, torch.zeros_like(tot))
        N[:, :n].scatter_add_(0, k[None, :], val[None, :])
    return N.to(dtype)


def place_windows(E_env: torch.Tensor, thresholds: list, w: torch.Tensor, Z: int):
    """lo = number of states whose threshold lies below the envelope field,
    clipped so that [lo, lo+w-1] fits in [0, Z]."""
    th = torch.tensor(thresholds, dtype=torch.float64, device=E_env.device)
    lo = (E_env.to(torch.float64)[:, None] > th[None, :]).sum(1)
    lo = torch.minimum(lo, Z + 1 - w.to(torch.int64))
    lo = lo.clamp(min=0)
    return lo.to(torch.uint8), (lo + w.to(torch.int64) - 1).to(torch.uint8)


def nitrogen_pulse_2d(t: float, nx: int = 128, ny: int = 128, dx: float = 0.5,
                      E0: float = 2000.0, waist: float = 8.0, tau: float = 10.0,
                      lam: float = 0.8, t0: float = 5.0, device="cpu") -> torch.Tensor:
    """|E| (GV/m, float32, y-major [ny*nx]) of the 2D pulse at time t (fs):
    cells x_i = (i + 1/2) dx, y_j = (j - (ny-1)/2) dx."""
    x = (torch.arange(nx, dtype=torch.float64, device=device) + 0.5) * dx
    y = (torch.arange(ny, dtype=torch.float64, device=device) - (ny - 1) / 2) * dx
    omega = 2 * math.pi * C_UM_PER_FS / lam
    env_x = torch.exp(-(((t - x / C_UM_PER_FS) - t0) / tau) ** 2)
    env_y = torch.exp(-(y / waist) ** 2)
    E = E0 * env_y[:, None] * env_x[None, :] * math.cos(omega * t)
    return E.abs().reshape(-1).to(torch.float32)


def nitrogen_2d_initial(nx: int = 128, ny: int = 128, device="cpu") -> Workload:
    """N_0 = 1 everywhere, window [0, 3] (p = 0, four levels)."""
    n = nx * ny
    ld = _padded(n)
    N = torch.zeros((8, ld), dtype=torch.float32, device=device)
    N[0, :n] = 1.0
    lo = torch.zeros(n, dtype=torch.uint8, device=device)
    hi = torch.full((n,), 3, dtype=torch.uint8, device=device)
    return Workload("nitrogen_pulse_2d", nitrogen(), nitrogen_pulse_2d(0.0, nx, ny, device=device),
                    N, lo, hi, 0.05, {"nx": nx, "ny": ny, "steps": 200})


def nitrogen_3d(nz: int = 256, ny: int = 256, nx: int = 512, seed: int = 2,
                device="cpu", block: int = 8, cells: torch.Tensor | None = None) -> Workload:
    """One step of N on an nz x ny x nx grid (x fastest).  The box spans
    +-2 waists (w = 8 um) transversely and +-4 c tau (tau = 10 fs)
    longitudinally around the pulse centre, lambda = 0.8 um.  `cells`
    selects a subset of the grid by global index (the values are those the
    full grid has there)."""
    dev = torch.device(device)
    c = (torch.arange(nz * ny * nx, device=dev, dtype=torch.int64) if cells is None
         else cells.to(dev, torch.int64))
    n = c.numel()
    ld = _padded(n)
    waist, tau, lam = 8.0, 10.0, 0.8
    Lx, Ly = 8 * C_UM_PER_FS * tau, 4 * waist
    ix, iy, iz = c % nx, (c // nx) % ny, c // (nx * ny)
    xi = ((ix.to(torch.float64) + 0.5) / nx - 0.5) * Lx
    y = ((iy.to(torch.float64) + 0.5) / ny - 0.5) * Ly
    z = ((iz.to(torch.float64) + 0.5) / nz - 0.5) * Ly
    blk = ((iz // block) * ((ny + block - 1) // block) + iy // block) * ((nx + block - 1) // block) + ix // block
    E0 = 500.0 + 3500.0 * uniform(seed, 1, blk)
    env = E0 * torch.exp(-(y * y + z * z) / waist ** 2) * torch.exp(-(xi / (C_UM_PER_FS * tau)) ** 2)
    E = (env * torch.abs(torch.cos(2 * math.pi * xi / lam))).to(torch.float32)
    p = 2 + (uniform(seed, 2, blk) < 0.5).to(torch.int64)  # populated states 2 or 3
    w = p + 1
    lo, hi = place_windows(env, window_thresholds("N"), w, 7)
    N = populations(seed, lo, p, 7, ld, cells=c)
    del xi, y, z, env, blk, ix, iy, iz
    return Workload("nitrogen_3d", nitrogen(), E, N, lo, hi, 0.05,
                    {"grid": [nz, ny, nx], "seed": seed})


def lognormal_field(seed: int, c: torch.Tensor, block: int = 512,
                    mu: float = 6.215, sigma: float = 0.759):
    """Per-block lognormal level ln E_b ~ N(mu, sigma) and per-cell
    E = E_b exp(0.2 g), both clipped to [100, 5000] GV/m, for the global
    cell indices c.  Returns (E float32, E_b float64)."""
    blk = c // block
    Eb = torch.exp(mu + sigma * normal(seed, 3, blk)).clamp(100.0, 5000.0)
    E = (Eb * torch.exp(0.2 * normal(seed, 4, c))).clamp(100.0, 5000.0)
    return E.to(torch.float32), Eb


def ladder_cells(sp: SpeciesData, n: int, seed: int, device="cpu",
                 block: int = 512, wmin: int = 2, wmax: int = 6,
                 cells: torch.Tensor | None = None) -> Workload:
    """Cells of one species for the batched and surrogate workloads: window
    width uniform in [wmin, wmax] per block of cells, placed at the states the
    block's field level burns through; Dirichlet(1) populations on the window
    minus its top state."""
    dev = torch.device(device)
    c = (torch.arange(n, device=dev, dtype=torch.int64) if cells is None
         else cells.to(dev, torch.int64))
    n = c.numel()
    ld = _padded(n)
    E, Eb = lognormal_field(seed, c, block)
    blk = c // block
    w = wmin + torch.floor(uniform(seed, 5, blk) * (wmax - wmin + 1)).to(torch.int64)
    w = w.clamp(max=sp.Z + 1)
    lo, hi = place_windows(Eb, window_thresholds(sp.name), w, sp.Z)
    p = (w - 1).clamp(min=1)
    N = populations(seed, lo, p, sp.Z, ld, cells=c)
    return Workload(f"{sp.name}_cells", sp, E, N, lo, hi, 0.05,
                    {"seed": seed, "block": block})


def mixed_batch(scale: float = 1.0, seed: int = 3, device="cpu"):
    """N (20M), Ar-like (8M) and Kr-like (2M) cells; `scale` shrinks the
    counts for tests."""
    specs = [(nitrogen(), 20_000_000), (argon_like(), 8_000_000), (krypton_like(), 2_000_000)]
    return [ladder_cells(sp, max(1, int(n * scale)), seed + i, device)
            for i, (sp, n) in enumerate(specs)]


def krypton_beam_terms(nz: int = 256, ny: int = 512, nx: int = 512, dx: float = 0.5,
                       seed: int = 5, lam: float = 0.8, device="cpu",
                       cells: torch.Tensor | None = None) -> tuple:
    """The two standing patterns of 16 seeded Gaussian beams on an
    nz x ny x nx grid (x fastest, cell centres at (i + 1/2) dx).  Beam b has
    a unit direction d_b, a centre, a waist w_b ~ U(4, 16) um and a phase
    phi_b; with g_b = exp(-rho_b^2/w_b^2) (rho_b the distance from the beam
    axis) and theta_b = k d_b.r + phi_b, the field of the superposition is
    sum_b g_b cos(theta_b - w t) = A cos(w t) + B sin(w t) with
    A = sum_b g_b cos(theta_b), B = sum_b g_b sin(theta_b), since all beams
    share lambda.  Returns (A, B) float64 for the cells `cells` (default:
    the whole grid)."""
    dev = torch.device(device)
    c = (torch.arange(nz * ny * nx, device=dev, dtype=torch.int64) if cells is None
         else cells.to(dev, torch.int64))
    x = ((c % nx).to(torch.float64) + 0.5) * dx
    y = (((c // nx) % ny).to(torch.float64) + 0.5) * dx
    z = ((c // (nx * ny)).to(torch.float64) + 0.5) * dx
    del c
    b = torch.arange(16, dtype=torch.int64)
    d = torch.stack([normal(seed, 20 + k, b) for k in range(3)])
    d = d / d.norm(dim=0, keepdim=True)
    L = torch.tensor([nx * dx, ny * dx, nz * dx], dtype=torch.float64)
    ctr = torch.stack([uniform(seed, 30 + k, b) for k in range(3)]) * L[:, None]
    wb = 4.0 + 12.0 * uniform(seed, 40, b)
    phi = 2 * math.pi * uniform(seed, 41, b)
    kL = 2 * math.pi / lam
    A = torch.zeros_like(x)
    B = torch.zeros_like(x)
    for j in range(16):
        rx, ry, rz = x - float(ctr[0, j]), y - float(ctr[1, j]), z - float(ctr[2, j])
        along = rx * float(d[0, j]) + ry * float(d[1, j]) + rz * float(d[2, j])
        rho2 = rx * rx + ry * ry + rz * rz - along * along
        del rx, ry, rz
        g = torch.exp(-rho2 / float(wb[j]) ** 2)
        theta = kL * along + float(phi[j])
        A += g * torch.cos(theta)
        B += g * torch.sin(theta)
        del along, rho2, g, theta
    return A, B


def krypton_beams_direct(t: float, nz: int, ny: int, nx: int, dx: float = 0.5,
                         seed: int = 5, lam: float = 0.8) -> torch.Tensor:
    """The same superposition evaluated beam by beam at time t (float64,
    unscaled, signed), for checking krypton_beam_terms on small grids."""
    c = torch.arange(nz * ny * nx, dtype=torch.int64)
    r = torch.stack([((c % nx).to(torch.float64) + 0.5) * dx,
                     (((c // nx) % ny).to(torch.float64) + 0.5) * dx,
                     ((c // (nx * ny)).to(torch.float64) + 0.5) * dx])
    b = torch.arange(16, dtype=torch.int64)
    d = torch.stack([normal(seed, 20 + k, b) for k in range(3)])
    d = d / d.norm(dim=0, keepdim=True)
    L = torch.tensor([nx * dx, ny * dx, nz * dx], dtype=torch.float64)
    ctr = torch.stack([uniform(seed, 30 + k, b) for k in range(3)]) * L[:, None]
    wb = 4.0 + 12.0 * uniform(seed, 40, b)
    phi = 2 * math.pi * uniform(seed, 41, b)
    kL = 2 * math.pi / lam
    omega = kL * C_UM_PER_FS
    acc = torch.zeros(r.shape[1], dtype=torch.float64)
    for j in range(16):
        rel = r - ctr[:, j][:, None]
        along = (rel * d[:, j][:, None]).sum(0)
        rho2 = (rel * rel).sum(0) - along * along
        acc += torch.exp(-rho2 / float(wb[j]) ** 2) * torch.cos(kL * along - omega * t + float(phi[j]))
    return acc


def krypton_scale(A: torch.Tensor, peak: float = 6000.0) -> float:
    """S such that the t = 0 maximum of S |A| is `peak` GV/m."""
    return peak / float(A.abs().max())


def krypton_field(A: torch.Tensor, B: torch.Tensor, t: float, scale: float,
                  lam: float = 0.8) -> torch.Tensor:
    """|E| (GV/m, float32) = S |A cos(w t) + B sin(w t)| at time t (fs)."""
    omega = 2 * math.pi / lam * C_UM_PER_FS
    return (scale * (A * math.cos(omega * t) + B * math.sin(omega * t)).abs()).to(torch.float32)


def krypton_initial(n: int, device="cpu") -> Workload:
    sp = krypton_like()
    ld = _padded(n)
    N = torch.zeros((sp.Z + 1, ld), dtype=torch.float32, device=device)
    N[0, :n] = 1.0
    lo = torch.zeros(n, dtype=torch.uint8, device=device)
    hi = torch.full((n,), 3, dtype=torch.uint8, device=device)
    E = torch.zeros(n, dtype=torch.float32, device=device)
    return Workload("krypton_beams", sp, E, N, lo, hi, 0.05, {})


def window_bytes_per_cell(lo: torch.Tensor, hi: torch.Tensor, elem: int = 4) -> torch.Tensor:
    """Algorithmic HBM bytes of one step per cell: |E|, lo, hi, the window
    planes read and written, dne, lo and hi written."""
    w = hi.to(torch.int64) - lo.to(torch.int64) + 1
    return elem + 2 + 2 * elem * w + elem + 2
