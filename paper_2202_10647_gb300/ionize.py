"""Thin Python binding of libionize.so (include/ionize.h).

Argument marshalling only: every function takes torch tensors, checks their
dtype/device/shape, and passes raw device pointers and the current CUDA
stream to the C ABI.  All arithmetic runs in the library's CUDA kernels.
There is no CPU path: without the library or a GPU these functions raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

ION_OK = 0
ION_EINVAL = -1
ION_ECUDA = -2
ION_ENOMEM = -3
ION_ETIMEOUT = -4

ION_F32 = 0x0
ION_F64_PLAIN = 0x1
ION_NO_WINDOW_UPDATE = 0x2
ION_NO_FP64_FALLBACK = 0x4
ION_FORCE_FP64_COEF = 0x8
ION_CONSERVATION_CHECK = 0x10

ION_DTYPE_F32 = 0
ION_DTYPE_F64 = 1

ION_MAX_Z = 63
ION_MAX_WINDOW = 6

#: every symbol include/ionize.h declares
EXPORTS = ("ion_species_init", "ion_species_destroy", "ion_species_z",
           "ion_rates", "ion_step_workspace_bytes", "ion_step", "ion_field_magnitude",
           "ion_step_field_workspace_bytes", "ion_step_field",
           "ion_step_batched_workspace_bytes", "ion_step_batched", "ion_autotune",
           "ion_step_noalloc", "ion_conservation", "ion_copy_cells", "ion_mlp_nparams",
           "ion_mlp_workspace_bytes", "ion_mlp_loss_grad", "ion_mlp_adam", "ion_mlp_forward",
           "ion_log2_rates", "ion_mlp_inputs", "ion_mlp_standardize",
           "ion_surrogate_create", "ion_surrogate_destroy", "ion_surrogate_rates",
           "ion_step_surrogate", "ion_surrogate_test_timeout", "ion_surrogate_validate",
           "ion_measure_peaks",
           "ion_binary_version",
           "ion_last_error")

#: forward pass in the tensor-core arithmetic (W2, W3, h1, h2 as bf16 pairs; SFU tanh)
ION_MLP_BF16 = 0x1
ION_MLP_HIDDEN = 64

ION_MAX_JOBS = 8
#: launch shapes the library is built with (cells per lane, warps per block)
LAUNCH_SHAPES = [(q, w) for q in (1, 2, 4) for w in (2, 4, 8)]

#: largest ncells of one ion_step_noalloc call
ION_STEP_NOALLOC_MAX_CELLS = 262144

_lock = threading.Lock()
_lib = None


class IonError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ionize error {code}: {msg}")
        self.code = code


class _Constants(ctypes.Structure):
    _fields_ = [("omega_a_per_s", ctypes.c_double), ("E_a_GVm", ctypes.c_double),
                ("U_H_eV", ctypes.c_double), ("rate_model", ctypes.c_int)]


#: rate models (ion_constants.rate_model)
ION_ADK_CYCLE_AVERAGED = 0
ION_ADK_STATIC = 1
#: the printed constants of Eq. 1 with U_H = 13.6 eV, and CODATA values
PAPER_CONSTANTS = (4.13e16, 510.0, 13.6)
CODATA_CONSTANTS = (4.1341374e16, 514.22067, 13.605693)


class _StepOpts(ctypes.Structure):
    _fields_ = [("eps_shift", ctypes.c_double), ("degen_gap", ctypes.c_double),
                ("window_policy", ctypes.c_int), ("w_min", ctypes.c_int),
                ("w_max", ctypes.c_int), ("eps_grow", ctypes.c_double)]


#: window policies (ion_step_opts.window_policy)
ION_WINDOW_FIXED = 0
ION_WINDOW_ADAPTIVE = 1


def _opts(eps_shift=1e-6, degen_gap=1e-3, window=None) -> _StepOpts:
    """ion_step_opts; window = None (the paper's rule) or a dict with
    w_min, w_max and eps_grow for the adaptive policy."""
    if window is None:
        return _StepOpts(float(eps_shift), float(degen_gap), ION_WINDOW_FIXED, 2, 6, 1e-6)
    return _StepOpts(float(eps_shift), float(degen_gap), ION_WINDOW_ADAPTIVE,
                     int(window.get("w_min", 2)), int(window.get("w_max", 6)),
                     float(window.get("eps_grow", 1e-6)))


class _BatchJob(ctypes.Structure):
    _fields_ = [("species", ctypes.c_void_p), ("E", ctypes.c_void_p), ("N", ctypes.c_void_p),
                ("ld", ctypes.c_int64), ("ncells", ctypes.c_int64), ("k_lo", ctypes.c_void_p),
                ("k_hi", ctypes.c_void_p), ("dne", ctypes.c_void_p), ("n_gas", ctypes.c_void_p)]


class _SurrogateNorm(ctypes.Structure):
    _fields_ = [("log2E_min", ctypes.c_double), ("log2E_max", ctypes.c_double),
                ("y_floor", ctypes.c_double), ("y_mean", ctypes.c_double * ION_MAX_Z),
                ("y_scale", ctypes.c_double * ION_MAX_Z)]


class LaunchShape(ctypes.Structure):
    _fields_ = [("cells_per_lane", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int)]

    def __repr__(self):
        return (f"LaunchShape(cells_per_lane={self.cells_per_lane}, "
                f"warps_per_block={self.warps_per_block}, blocks_per_sm={self.blocks_per_sm})")


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def _declare(lib):
    lib.ion_last_error.restype = ctypes.c_char_p
    lib.ion_last_error.argtypes = []
    lib.ion_species_init.restype = ctypes.c_int
    lib.ion_species_init.argtypes = [ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                     ctypes.POINTER(_Constants), ctypes.POINTER(_vp)]
    lib.ion_species_destroy.restype = ctypes.c_int
    lib.ion_species_destroy.argtypes = [_vp]
    lib.ion_species_z.restype = ctypes.c_int
    lib.ion_species_z.argtypes = [_vp]
    lib.ion_rates.restype = ctypes.c_int
    lib.ion_rates.argtypes = [_vp, _vp, _i64, ctypes.c_int, ctypes.c_int, _vp, _i64,
                              ctypes.c_int, _vp]
    lib.ion_step_workspace_bytes.restype = ctypes.c_size_t
    lib.ion_step_workspace_bytes.argtypes = [_i64, ctypes.c_int]
    lib.ion_step.restype = ctypes.c_int
    lib.ion_step.argtypes = [_vp, _vp, _vp, _i64, _i64, ctypes.c_double, _vp, _vp,
                             _vp, _vp, ctypes.POINTER(_StepOpts), ctypes.c_int, _vp,
                             ctypes.c_size_t, _vp]
    lib.ion_step_batched_workspace_bytes.restype = ctypes.c_size_t
    lib.ion_step_batched_workspace_bytes.argtypes = [ctypes.POINTER(_BatchJob), ctypes.c_int,
                                                     ctypes.c_int]
    lib.ion_step_batched.restype = ctypes.c_int
    lib.ion_step_batched.argtypes = [ctypes.POINTER(_BatchJob), ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(_StepOpts), ctypes.c_int,
                                     ctypes.POINTER(LaunchShape), _vp, ctypes.c_size_t, _vp]
    lib.ion_autotune.restype = ctypes.c_int
    lib.ion_autotune.argtypes = [ctypes.POINTER(_BatchJob), ctypes.c_int, ctypes.c_double,
                                 ctypes.POINTER(_StepOpts), ctypes.c_int, _vp, ctypes.c_size_t,
                                 ctypes.c_int, _vp, ctypes.POINTER(LaunchShape),
                                 ctypes.POINTER(ctypes.c_float)]
    lib.ion_conservation.restype = ctypes.c_int
    lib.ion_conservation.argtypes = [_vp, _i64, _i64, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, _vp, _vp]
    lib.ion_mlp_nparams.restype = ctypes.c_int64
    lib.ion_mlp_nparams.argtypes = [ctypes.c_int]
    lib.ion_mlp_workspace_bytes.restype = ctypes.c_size_t
    lib.ion_mlp_workspace_bytes.argtypes = [ctypes.c_int, _i64]
    lib.ion_mlp_loss_grad.restype = ctypes.c_int
    lib.ion_mlp_loss_grad.argtypes = [_vp, ctypes.c_int, _vp, _vp, _i64, ctypes.c_int, _vp, _vp,
                                      _vp, ctypes.c_size_t, _vp]
    lib.ion_mlp_adam.restype = ctypes.c_int
    lib.ion_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_float, ctypes.c_int, _vp]
    lib.ion_mlp_forward.restype = ctypes.c_int
    lib.ion_mlp_forward.argtypes = [_vp, ctypes.c_int, _vp, _i64, ctypes.c_int, _vp, _vp]
    lib.ion_copy_cells.restype = ctypes.c_int
    lib.ion_copy_cells.argtypes = [_vp, _i64, _vp, _i64, ctypes.c_int, _i64, _i64, ctypes.c_int,
                                   _vp]
    lib.ion_field_magnitude.restype = ctypes.c_int
    lib.ion_field_magnitude.argtypes = [_vp, _vp, _vp, _i64, ctypes.c_int, _vp, _vp]
    lib.ion_step_field_workspace_bytes.restype = ctypes.c_size_t
    lib.ion_step_field_workspace_bytes.argtypes = [_i64, ctypes.c_int]
    lib.ion_step_field.restype = ctypes.c_int
    lib.ion_step_field.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _i64, ctypes.c_double, _vp,
                                   _vp, _vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_size_t, _vp]
    lib.ion_log2_rates.restype = ctypes.c_int
    lib.ion_log2_rates.argtypes = [_vp, _vp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   _vp, _i64, _vp]
    lib.ion_mlp_inputs.restype = ctypes.c_int
    lib.ion_mlp_inputs.argtypes = [_vp, _i64, ctypes.c_double, ctypes.c_double, _vp, _vp]
    lib.ion_mlp_standardize.restype = ctypes.c_int
    lib.ion_mlp_standardize.argtypes = [_vp, _i64, ctypes.c_int, ctypes.c_double, _vp, _vp, _vp,
                                        _vp]
    lib.ion_surrogate_create.restype = ctypes.c_int
    lib.ion_surrogate_create.argtypes = [_vp, _vp, ctypes.POINTER(_SurrogateNorm),
                                         ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                         ctypes.POINTER(_vp)]
    lib.ion_surrogate_destroy.restype = ctypes.c_int
    lib.ion_surrogate_destroy.argtypes = [_vp]
    lib.ion_surrogate_rates.restype = ctypes.c_int
    lib.ion_surrogate_rates.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp]
    lib.ion_step_surrogate.restype = ctypes.c_int
    lib.ion_step_surrogate.argtypes = [_vp, _vp, _vp, _i64, _i64, ctypes.c_double, _vp, _vp,
                                       _vp, _vp, ctypes.POINTER(_StepOpts), ctypes.c_double,
                                       _vp, ctypes.c_size_t, _vp]
    lib.ion_surrogate_test_timeout.restype = ctypes.c_int
    lib.ion_surrogate_test_timeout.argtypes = [_vp, ctypes.c_int]
    lib.ion_surrogate_validate.restype = ctypes.c_int
    lib.ion_surrogate_validate.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, _vp, _vp]
    lib.ion_measure_peaks.restype = ctypes.c_int
    lib.ion_measure_peaks.argtypes = [ctypes.POINTER(ctypes.c_double)]
    lib.ion_binary_version.restype = ctypes.c_int
    lib.ion_binary_version.argtypes = []
    lib.ion_step_noalloc.restype = ctypes.c_int
    lib.ion_step_noalloc.argtypes = [_vp, _vp, _vp, _i64, _i64, ctypes.c_double, _vp, _vp,
                                     _vp, _vp, ctypes.POINTER(_StepOpts), ctypes.c_int, _vp]
    return lib


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libionize.so (compiling it first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"{path} is missing; run __graft_entry__.build()")
                _build.build()
            _lib = _declare(ctypes.CDLL(path))
    return _lib


def _check(rc: int):
    if rc != ION_OK:
        raise IonError(rc, lib().ion_last_error().decode())


def _stream(t: torch.Tensor):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _stream_of(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t, offset: int = 0):
    """Device address of element `offset` (along the last axis for the
    population planes, which keep their stride ld)."""
    return None if t is None else ctypes.c_void_p(t.data_ptr() + offset * t.element_size())


def _need(t: torch.Tensor, name: str, dtype, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Species:
    """ADK table of one gas (ion_species_init).  U, l, m are sequences of
    length Z for the Z ionizing transitions k -> k+1."""

    def __init__(self, U, l, m, constants=None, rate_model: int = ION_ADK_CYCLE_AVERAGED):
        U = [float(x) for x in U]
        l = [int(x) for x in l]
        m = [int(x) for x in m]
        Z = len(U)
        if len(l) != Z or len(m) != Z:
            raise ValueError("U, l and m must have the same length")
        self.Z = Z
        self.U, self.l, self.m = U, l, m
        Ua = (ctypes.c_double * Z)(*U)
        la = (ctypes.c_int * Z)(*l)
        ma = (ctypes.c_int * Z)(*m)
        c = None
        if constants is not None or rate_model != ION_ADK_CYCLE_AVERAGED:
            cs = PAPER_CONSTANTS if constants is None else constants
            c = ctypes.byref(_Constants(*[float(x) for x in cs][:3], int(rate_model)))
        self.rate_model = int(rate_model)
        h = _vp()
        _check(lib().ion_species_init(Ua, la, ma, Z, c, ctypes.byref(h)))
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ion_species_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rates(sp: Species, E: torch.Tensor, k_lo: int, k_hi: int,
          out: torch.Tensor | None = None) -> torch.Tensor:
    """W_k(|E|) in 1/fs for k in [k_lo, k_hi): tensor (k_hi-k_lo, ncells)."""
    if E.dtype not in (torch.float32, torch.float64):
        raise ValueError("E must be float32 or float64")
    _need(E, "E", E.dtype)
    n = E.numel()
    if out is None:
        out = torch.empty((k_hi - k_lo, n), dtype=E.dtype, device=E.device)
    _need(out, "out", E.dtype, E.device)
    ldw = out.shape[1] if out.dim() == 2 else n
    dtype = ION_DTYPE_F32 if E.dtype == torch.float32 else ION_DTYPE_F64
    _check(lib().ion_rates(sp.handle, _ptr(E), n, int(k_lo), int(k_hi), _ptr(out),
                           ldw, dtype, _stream(E)))
    return out


def copy_cells(dst: torch.Tensor, src: torch.Tensor, offset: int, ncells: int) -> None:
    """ion_copy_cells: cells [offset, offset + ncells) of every row of src
    (a 1-D array or a (planes, ld) SoA) into the same cells of dst, in one
    strided copy on the current stream of whichever tensor is on the GPU
    (host tensors should be pinned)."""
    if dst.dtype != src.dtype:
        raise ValueError("dst and src must have the same dtype")
    if dst.dim() != src.dim() or dst.dim() not in (1, 2):
        raise ValueError("dst and src must both be 1-D or both (planes, ld)")
    for name, t in (("dst", dst), ("src", src)):
        if t.stride(-1) != 1:
            raise ValueError(f"{name} rows must be contiguous")
    planes = 1 if dst.dim() == 1 else dst.shape[0]
    if dst.dim() == 2 and src.shape[0] != planes:
        raise ValueError("dst and src must have the same number of planes")
    ld_d = dst.shape[-1] if dst.dim() == 1 else dst.stride(0)
    ld_s = src.shape[-1] if src.dim() == 1 else src.stride(0)
    if offset < 0 or ncells < 0 or offset + ncells > min(dst.shape[-1], src.shape[-1]):
        raise ValueError("offset/ncells outside the arrays")
    dev = dst.device if dst.is_cuda else src.device
    if not dev.type == "cuda":
        raise ValueError("one of dst and src must be a CUDA tensor")
    _check(lib().ion_copy_cells(ctypes.c_void_p(dst.data_ptr()), ld_d,
                                ctypes.c_void_p(src.data_ptr()), ld_s, planes, int(offset),
                                int(ncells), dst.element_size(), _stream_of(dev)))


def field_magnitude(Ex: torch.Tensor, Ey: torch.Tensor | None = None,
                    Ez: torch.Tensor | None = None,
                    out: torch.Tensor | None = None) -> torch.Tensor:
    """ion_field_magnitude: |E| from 1-3 components (float32 or float64)."""
    if Ex.dtype not in (torch.float32, torch.float64):
        raise ValueError("Ex must be float32 or float64")
    _need(Ex, "Ex", Ex.dtype)
    for name, t in (("Ey", Ey), ("Ez", Ez)):
        if t is not None:
            _need(t, name, Ex.dtype, Ex.device)
            if t.numel() < Ex.numel():
                raise ValueError(f"{name} is shorter than Ex")
    out = torch.empty_like(Ex) if out is None else out
    _need(out, "out", Ex.dtype, Ex.device)
    dtype = ION_DTYPE_F32 if Ex.dtype == torch.float32 else ION_DTYPE_F64
    _check(lib().ion_field_magnitude(_ptr(Ex), _ptr(Ey), _ptr(Ez), Ex.numel(), dtype, _ptr(out),
                                     _stream(Ex)))
    return out


def step_field(sp: "Species", components, N: torch.Tensor, k_lo: torch.Tensor,
               k_hi: torch.Tensor, dt: float, dne: torch.Tensor,
               n_gas: torch.Tensor | None = None, ws: torch.Tensor | None = None,
               eps_shift: float = 1e-6, degen_gap: float = 1e-3, flags: int = ION_F32,
               window: dict | None = None) -> torch.Tensor:
    """ion_step_field: ion_step with the field as 1-3 component tensors
    (Ex, Ey, Ez; missing ones None or left out).  Returns the workspace."""
    comps = list(components) + [None] * (3 - len(components))
    Ex, Ey, Ez = comps[:3]
    f64 = bool(flags & ION_F64_PLAIN)
    dt_ = torch.float64 if f64 else torch.float32
    _need(Ex, "Ex", dt_)
    dev = Ex.device
    n = Ex.numel()
    for name, t in (("Ey", Ey), ("Ez", Ez)):
        if t is not None:
            _need(t, name, dt_, dev)
            if t.numel() < n:
                raise ValueError(f"{name} is shorter than Ex")
    _need(N, "N", dt_, dev)
    _need(k_lo, "k_lo", torch.uint8, dev)
    _need(k_hi, "k_hi", torch.uint8, dev)
    _need(dne, "dne", dt_, dev)
    if n_gas is not None:
        _need(n_gas, "n_gas", dt_, dev)
    if N.dim() != 2 or N.shape[0] != sp.Z + 1:
        raise ValueError(f"N must have shape (Z+1, ld) = ({sp.Z + 1}, ld)")
    if n > min(k_lo.numel(), k_hi.numel(), dne.numel(), N.shape[1]):
        raise ValueError("the arrays are shorter than Ex")
    if ws is None:
        nb = int(lib().ion_step_field_workspace_bytes(n, int(flags)))
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    _need(ws, "ws", torch.uint8, dev)
    opts = _opts(eps_shift, degen_gap, window)
    _check(lib().ion_step_field(sp.handle, _ptr(Ex), _ptr(Ey), _ptr(Ez), _ptr(N), N.shape[1], n,
                                float(dt), _ptr(k_lo), _ptr(k_hi), _ptr(dne), _ptr(n_gas),
                                ctypes.byref(opts), int(flags), _ptr(ws), ws.numel(),
                                _stream(Ex)))
    return ws


def workspace_bytes(ncells: int, flags: int = ION_F32) -> int:
    return int(lib().ion_step_workspace_bytes(int(ncells), int(flags)))


def workspace(ncells: int, flags: int = ION_F32, device=None) -> torch.Tensor:
    """A device buffer big enough for ion_step (256-byte aligned by torch)."""
    nb = workspace_bytes(ncells, flags)
    return torch.empty(nb, dtype=torch.uint8, device=device or "cuda")


def step(sp: Species, E: torch.Tensor, N: torch.Tensor, k_lo: torch.Tensor,
         k_hi: torch.Tensor, dt: float, dne: torch.Tensor,
         n_gas: torch.Tensor | None = None, ws: torch.Tensor | None = None,
         eps_shift: float = 1e-6, degen_gap: float = 1e-3, flags: int = ION_F32,
         ncells: int | None = None, window: dict | None = None,
         offset: int = 0) -> torch.Tensor:
    """One ion_step.  N is (Z+1, ld) and is updated in place, as are k_lo and
    k_hi; dne is written.  window: None (the paper's slide) or
    {"w_min": .., "w_max": .., "eps_grow": ..} for ION_WINDOW_ADAPTIVE.
    offset, ncells: step cells [offset, offset + ncells) of the arrays (the
    planes keep their stride).  Returns the workspace (its header holds the
    counters described in include/ionize.h)."""
    f64 = bool(flags & ION_F64_PLAIN)
    dt_ = torch.float64 if f64 else torch.float32
    _need(E, "E", dt_)
    dev = E.device
    _need(N, "N", dt_, dev)
    _need(k_lo, "k_lo", torch.uint8, dev)
    _need(k_hi, "k_hi", torch.uint8, dev)
    _need(dne, "dne", dt_, dev)
    if n_gas is not None:
        _need(n_gas, "n_gas", dt_, dev)
    if N.dim() != 2 or N.shape[0] != sp.Z + 1:
        raise ValueError(f"N must have shape (Z+1, ld) = ({sp.Z + 1}, ld)")
    off = int(offset)
    n = E.numel() - off if ncells is None else int(ncells)
    if off < 0 or n < 0 or off + n > min(E.numel(), k_lo.numel(), k_hi.numel(),
                                         dne.numel(), N.shape[1]):
        raise ValueError("offset/ncells outside the arrays")
    if n_gas is not None and off + n > n_gas.numel():
        raise ValueError("offset/ncells outside n_gas")
    if ws is None:
        ws = workspace(n, flags, dev)
    _need(ws, "ws", torch.uint8, dev)
    opts = _opts(eps_shift, degen_gap, window)
    _check(lib().ion_step(sp.handle, _ptr(E, off), _ptr(N, off), N.shape[1], n,
                          float(dt), _ptr(k_lo, off), _ptr(k_hi, off), _ptr(dne, off),
                          _ptr(n_gas, off), ctypes.byref(opts), int(flags), _ptr(ws),
                          ws.numel(), _stream(E)))
    return ws


def step_noalloc(sp: Species, E: torch.Tensor, N: torch.Tensor, k_lo: torch.Tensor,
                 k_hi: torch.Tensor, dt: float, dne: torch.Tensor,
                 n_gas: torch.Tensor | None = None, eps_shift: float = 1e-6,
                 degen_gap: float = 1e-3, flags: int = ION_F32,
                 ncells: int | None = None, window: dict | None = None) -> None:
    """ion_step_noalloc: the same step as `step`, with the library's own
    fixed scratch array instead of a workspace (at most
    ION_STEP_NOALLOC_MAX_CELLS cells per call)."""
    f64 = bool(flags & ION_F64_PLAIN)
    dt_ = torch.float64 if f64 else torch.float32
    _need(E, "E", dt_)
    dev = E.device
    _need(N, "N", dt_, dev)
    _need(k_lo, "k_lo", torch.uint8, dev)
    _need(k_hi, "k_hi", torch.uint8, dev)
    _need(dne, "dne", dt_, dev)
    if n_gas is not None:
        _need(n_gas, "n_gas", dt_, dev)
    if N.dim() != 2 or N.shape[0] != sp.Z + 1:
        raise ValueError(f"N must have shape (Z+1, ld) = ({sp.Z + 1}, ld)")
    n = E.numel() if ncells is None else int(ncells)
    if n < 0 or n > min(E.numel(), k_lo.numel(), k_hi.numel(), dne.numel(), N.shape[1]):
        raise ValueError("ncells outside the arrays")
    if n_gas is not None and n > n_gas.numel():
        raise ValueError("ncells outside n_gas")
    opts = _opts(eps_shift, degen_gap, window)
    _check(lib().ion_step_noalloc(sp.handle, _ptr(E), _ptr(N), N.shape[1], n, float(dt),
                                  _ptr(k_lo), _ptr(k_hi), _ptr(dne), _ptr(n_gas),
                                  ctypes.byref(opts), int(flags), _stream(E)))


def _jobs(jobs, f64=False):
    """jobs: sequence of (Species, E, N, k_lo, k_hi, dne[, n_gas])."""
    if not 1 <= len(jobs) <= ION_MAX_JOBS:
        raise ValueError(f"1..{ION_MAX_JOBS} jobs")
    dt_ = torch.float64 if f64 else torch.float32
    arr = (_BatchJob * len(jobs))()
    dev = None
    for i, jb in enumerate(jobs):
        sp, E, N, lo, hi, dne = jb[:6]
        ng = jb[6] if len(jb) > 6 else None
        _need(E, "E", dt_)
        dev = dev or E.device
        for t, nm in ((N, "N"), (dne, "dne")):
            _need(t, nm, dt_, dev)
        _need(lo, "k_lo", torch.uint8, dev)
        _need(hi, "k_hi", torch.uint8, dev)
        if ng is not None:
            _need(ng, "n_gas", dt_, dev)
        if N.dim() != 2 or N.shape[0] != sp.Z + 1:
            raise ValueError(f"job {i}: N must have shape (Z+1, ld)")
        arr[i] = _BatchJob(sp.handle.value, E.data_ptr(), N.data_ptr(), N.shape[1], E.numel(),
                           lo.data_ptr(), hi.data_ptr(), dne.data_ptr(),
                           ng.data_ptr() if ng is not None else None)
    return arr, dev


def batched_workspace(jobs, flags: int = ION_F32, device=None) -> torch.Tensor:
    n = sum(jb[1].numel() for jb in jobs)
    return workspace(n, flags, device or jobs[0][1].device)


def step_batched(jobs, dt: float, ws: torch.Tensor | None = None, eps_shift: float = 1e-6,
                 degen_gap: float = 1e-3, flags: int = ION_F32,
                 shape: LaunchShape | tuple | None = None,
                 window: dict | None = None) -> torch.Tensor:
    """ion_step_batched over jobs = [(Species, E, N, k_lo, k_hi, dne[, n_gas]), ...]."""
    arr, dev = _jobs(jobs, bool(flags & ION_F64_PLAIN))
    if ws is None:
        ws = batched_workspace(jobs, flags, dev)
    if shape is not None and not isinstance(shape, LaunchShape):
        shape = LaunchShape(*shape)
    opts = _opts(eps_shift, degen_gap, window)
    _check(lib().ion_step_batched(arr, len(jobs), float(dt), ctypes.byref(opts), int(flags),
                                  ctypes.byref(shape) if shape is not None else None,
                                  _ptr(ws), ws.numel(), _stream(jobs[0][1])))
    return ws


def autotune(jobs, dt: float, ws: torch.Tensor | None = None, reps: int = 3,
             eps_shift: float = 1e-6, degen_gap: float = 1e-3, flags: int = ION_F32,
             window: dict | None = None):
    """ion_autotune: (best LaunchShape, its median ms).  Steps the jobs' arrays."""
    arr, dev = _jobs(jobs)
    if ws is None:
        ws = batched_workspace(jobs, flags, dev)
    opts = _opts(eps_shift, degen_gap, window)
    best = LaunchShape()
    ms = ctypes.c_float()
    _check(lib().ion_autotune(arr, len(jobs), float(dt), ctypes.byref(opts), int(flags),
                              _ptr(ws), ws.numel(), int(reps), _stream(jobs[0][1]),
                              ctypes.byref(best), ctypes.byref(ms)))
    return best, float(ms.value)


def counters(ws: torch.Tensor):
    """(cells done with FP64 coefficients, cells skipped for invalid windows)
    of the last step that used `ws` (synchronizes)."""
    h = ws[:8].cpu().view(torch.int32)
    return int(h[0]), int(h[1])


def stiff_cells(ws: torch.Tensor) -> int:
    """Cells of the last FP32 step that used `ws` with some W dt > 1 (> 1.5
    under a launch shape of one cell per lane), finished on the long path;
    synchronizes."""
    return int(ws[8:12].cpu().view(torch.int32)[0])


def conservation_change(ws: torch.Tensor) -> float:
    """With ION_CONSERVATION_CHECK: the largest |sum_k N'_k - sum_k N_k| over
    the cells of the last step that used `ws` (synchronizes)."""
    return float(ws[40:44].cpu().view(torch.float32)[0])


def conservation(N: torch.Tensor, out: torch.Tensor, ncells: int | None = None,
                 nplanes: int | None = None, target: float = 1.0) -> torch.Tensor:
    """ion_conservation: writes max_c |sum_k N[k, c] - target| over the
    first `ncells` cells of the (planes, ld) SoA N into the device scalar
    `out` (float32)."""
    if N.dtype not in (torch.float32, torch.float64):
        raise ValueError("N must be float32 or float64")
    _need(N, "N", N.dtype)
    _need(out, "out", torch.float32, N.device)
    if N.dim() != 2 or out.numel() < 1:
        raise ValueError("N must be (planes, ld) and out non-empty")
    n = N.shape[1] if ncells is None else int(ncells)
    k = N.shape[0] if nplanes is None else int(nplanes)
    dtype = ION_DTYPE_F32 if N.dtype == torch.float32 else ION_DTYPE_F64
    _check(lib().ion_conservation(_ptr(N), N.shape[1], n, k, float(target), dtype, _ptr(out),
                                  _stream(N)))
    return out


# ---------------------------------------------------------------------------
# rate surrogate: training calls and inference
# ---------------------------------------------------------------------------
def mlp_nparams(K: int) -> int:
    n = int(lib().ion_mlp_nparams(int(K)))
    if n < 0:
        raise IonError(n, lib().ion_last_error().decode())
    return n


def mlp_workspace(K: int, B: int, device=None) -> torch.Tensor:
    nb = int(lib().ion_mlp_workspace_bytes(int(K), int(B)))
    if nb == 0:
        raise ValueError("K or B out of range")
    return torch.empty(nb, dtype=torch.uint8, device=device or "cuda")


def mlp_loss_grad(P: torch.Tensor, K: int, x: torch.Tensor, t: torch.Tensor, flags: int = 0,
                  grad: torch.Tensor | None = None, loss: torch.Tensor | None = None,
                  ws: torch.Tensor | None = None):
    """ion_mlp_loss_grad: (loss (device scalar), grad) of the batch (x, t)."""
    _need(P, "P", torch.float32)
    dev = P.device
    _need(x, "x", torch.float32, dev)
    _need(t, "t", torch.float32, dev)
    B = x.numel()
    if t.numel() != B * K:
        raise ValueError("t must hold B*K targets")
    grad = torch.empty_like(P) if grad is None else grad
    loss = torch.empty(1, dtype=torch.float32, device=dev) if loss is None else loss
    ws = mlp_workspace(K, B, dev) if ws is None else ws
    _need(grad, "grad", torch.float32, dev)
    _need(loss, "loss", torch.float32, dev)
    _check(lib().ion_mlp_loss_grad(_ptr(P), int(K), _ptr(x), _ptr(t), B, int(flags), _ptr(grad),
                                   _ptr(loss), _ptr(ws), ws.numel(), _stream(P)))
    return loss, grad


def mlp_adam(P: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float,
             t: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """ion_mlp_adam: one Adam step (t >= 1) on P in place."""
    for a, nm in ((P, "P"), (grad, "grad"), (m, "m"), (v, "v")):
        _need(a, nm, torch.float32, P.device)
    _check(lib().ion_mlp_adam(_ptr(P), _ptr(grad), _ptr(m), _ptr(v), P.numel(), float(lr),
                              float(beta1), float(beta2), float(eps), int(t), _stream(P)))


def mlp_forward(P: torch.Tensor, K: int, x: torch.Tensor, flags: int = 0,
                out: torch.Tensor | None = None) -> torch.Tensor:
    """ion_mlp_forward: outputs (B, K) on CUDA cores."""
    _need(P, "P", torch.float32)
    _need(x, "x", torch.float32, P.device)
    out = torch.empty((x.numel(), K), dtype=torch.float32, device=P.device) if out is None else out
    _need(out, "out", torch.float32, P.device)
    _check(lib().ion_mlp_forward(_ptr(P), int(K), _ptr(x), x.numel(), int(flags), _ptr(out),
                                 _stream(P)))
    return out


def log2_rates(sp: Species, E: torch.Tensor, k_lo: int, k_hi: int, floor: float,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """ion_log2_rates: max(log2 W_k(|E|), floor) in FP64 for k in [k_lo, k_hi),
    tensor (ncells, k_hi - k_lo) float64 (one row per cell)."""
    _need(E, "E", torch.float32)
    n = E.numel()
    if out is None:
        out = torch.empty((n, k_hi - k_lo), dtype=torch.float64, device=E.device)
    _need(out, "out", torch.float64, E.device)
    if out.dim() != 2 or out.shape[0] != n or out.stride(1) != 1:
        raise ValueError("out must be (ncells, k_hi - k_lo) with unit column stride")
    _check(lib().ion_log2_rates(sp.handle, _ptr(E), n, int(k_lo), int(k_hi), float(floor),
                                _ptr(out), out.stride(0), _stream(E)))
    return out


def mlp_inputs(E: torch.Tensor, l2lo: float, l2hi: float,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """ion_mlp_inputs: the network input of each field, float32 [n]."""
    _need(E, "E", torch.float32)
    out = torch.empty(E.numel(), dtype=torch.float32, device=E.device) if out is None else out
    _need(out, "out", torch.float32, E.device)
    _check(lib().ion_mlp_inputs(_ptr(E), E.numel(), float(l2lo), float(l2hi), _ptr(out),
                                _stream(E)))
    return out


def mlp_standardize(Y: torch.Tensor, min_scale: float):
    """ion_mlp_standardize of targets Y (n, K) float64: (mean [K], scale [K],
    T (n, K) float32), all on Y's device."""
    _need(Y, "Y", torch.float64)
    if Y.dim() != 2:
        raise ValueError("Y must be (n, K)")
    n, K = Y.shape
    mean = torch.empty(K, dtype=torch.float64, device=Y.device)
    scale = torch.empty(K, dtype=torch.float64, device=Y.device)
    T = torch.empty((n, K), dtype=torch.float32, device=Y.device)
    _check(lib().ion_mlp_standardize(_ptr(Y), n, K, float(min_scale), _ptr(mean), _ptr(scale),
                                     _ptr(T), _stream(Y)))
    return mean, scale, T


class Surrogate:
    """ion_surrogate_create: a trained network for species `sp`.

    norm: dict with log2E_min, log2E_max, y_floor, y_mean (Z), y_scale (Z).
    bound: None or an array (nbins, Z) of log2-error bounds."""

    def __init__(self, sp: Species, P: torch.Tensor, norm: dict, bound=None):
        _need(P, "P", torch.float32)
        Z = sp.Z
        nm = _SurrogateNorm()
        nm.log2E_min = float(norm["log2E_min"])
        nm.log2E_max = float(norm["log2E_max"])
        nm.y_floor = float(norm["y_floor"])
        for k in range(Z):
            nm.y_mean[k] = float(norm["y_mean"][k])
            nm.y_scale[k] = float(norm["y_scale"][k])
        bptr, nbins = None, 0
        if bound is not None:
            import numpy as _np
            b = _np.ascontiguousarray(_np.asarray(bound, dtype=_np.float32))
            if b.ndim != 2 or b.shape[1] != Z:
                raise ValueError("bound must be (nbins, Z)")
            nbins = b.shape[0]
            self._bound = b
            bptr = b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        h = _vp()
        _check(lib().ion_surrogate_create(sp.handle, _ptr(P), ctypes.byref(nm), bptr, nbins,
                                          ctypes.byref(h)))
        self._h = h
        self.Z = Z
        self.norm = dict(norm)
        self.device = P.device

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ion_surrogate_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def validate(self, nbins: int = 4096, per_bin: int = 64, margin: float = 1.25,
                 floor_add: float = 2e-3):
        """ion_surrogate_validate: compute the validation bound on the GPU and
        install it; returns it as a numpy array (nbins, Z)."""
        import numpy as _np
        b = _np.empty((int(nbins), self.Z), dtype=_np.float32)
        _check(lib().ion_surrogate_validate(self._h, int(nbins), int(per_bin), float(margin),
                                            float(floor_add),
                                            b.ctypes.data_as(ctypes.c_void_p),
                                            _stream_of(self.device)))
        self._bound = b
        return b

    def test_timeout(self, on: bool = True) -> None:
        """ion_surrogate_test_timeout: make the kernels' first tensor-core
        wait give up (on) or wait normally (off)."""
        _check(lib().ion_surrogate_test_timeout(self._h, int(bool(on))))

    def rates(self, E: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """W_k(|E|) in 1/fs from the network, (Z, ncells)."""
        _need(E, "E", torch.float32)
        n = E.numel()
        out = torch.empty((self.Z, n), dtype=torch.float32, device=E.device) if out is None else out
        _need(out, "out", torch.float32, E.device)
        _check(lib().ion_surrogate_rates(self._h, _ptr(E), n, _ptr(out), out.shape[1],
                                         _stream(E)))
        return out

    def step(self, E: torch.Tensor, N: torch.Tensor, k_lo: torch.Tensor, k_hi: torch.Tensor,
             dt: float, dne: torch.Tensor, n_gas: torch.Tensor | None = None,
             ws: torch.Tensor | None = None, eps_shift: float = 1e-6, degen_gap: float = 1e-3,
             pop_tol: float = 1e-6, window: dict | None = None) -> torch.Tensor:
        """ion_step_surrogate; returns the workspace (header words 3, 4, 5:
        cells on the network's rates, on Eq. 1's rates, timeout flag)."""
        _need(E, "E", torch.float32)
        dev = E.device
        _need(N, "N", torch.float32, dev)
        _need(k_lo, "k_lo", torch.uint8, dev)
        _need(k_hi, "k_hi", torch.uint8, dev)
        _need(dne, "dne", torch.float32, dev)
        if n_gas is not None:
            _need(n_gas, "n_gas", torch.float32, dev)
        if N.dim() != 2 or N.shape[0] != self.Z + 1:
            raise ValueError(f"N must have shape (Z+1, ld) = ({self.Z + 1}, ld)")
        n = E.numel()
        ws = workspace(n, ION_F32, dev) if ws is None else ws
        opts = _opts(eps_shift, degen_gap, window)
        _check(lib().ion_step_surrogate(self._h, _ptr(E), _ptr(N), N.shape[1], n, float(dt),
                                        _ptr(k_lo), _ptr(k_hi), _ptr(dne), _ptr(n_gas),
                                        ctypes.byref(opts), float(pop_tol), _ptr(ws),
                                        ws.numel(), _stream(E)))
        return ws


def surrogate_counters(ws: torch.Tensor):
    """(cells on the network's rates, cells on Eq. 1's rates, timeout flag)
    of the last ion_step_surrogate that used `ws` (synchronizes)."""
    h = ws[:24].cpu().view(torch.int32)
    return int(h[3]), int(h[4]), int(h[5])


def measure_peaks() -> dict:
    """ion_measure_peaks on the current device (synchronizes)."""
    out = (ctypes.c_double * 4)()
    _check(lib().ion_measure_peaks(out))
    return {"sfu_ex2_per_s": out[0], "sfu_tanh_per_s": out[1], "fp64_flops": out[2],
            "fp64_exp2_per_s": out[3]}
