"""FP64 CPU oracle for the multi-level ADK ionization step (arXiv 2202.10647).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the product library never
does.  The arithmetic lives in ``ion_oracle.c`` (plain C, double precision);
this module only compiles it with gcc and marshals numpy arrays.

Functions
---------
``adk_rate``  Eq. 1 for scalar arguments (1/fs).
``flm``       the (l,|m|) factor of Eq. 1.
``rates``     Eq. 1 for states k_lo..k_hi-1 of every cell (SoA).
``expm``      exp(M) by scaling and squaring (the definition of the analytic
              solution of Eqs. 4-5).
``step``      one windowed analytic step for every cell (Eqs. 3-9 with the
              window shift of Sec. 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "ion_oracle.c")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

#: printed constants of Eq. 1 (omega_a in 1/s, E_a in GV/m) and U_H = 13.6 eV
PAPER_CONSTANTS = (4.13e16, 510.0, 13.6)


def build(force: bool = False) -> str:
    """Compile ion_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_variant(replacements, tag: str) -> ctypes.CDLL:
    """Compile a modified copy of ion_oracle.c (each (old, new) text
    replacement must match exactly once) and load it.  The tests use this to
    plant a mistake in the oracle and show that the pins catch it."""
    os.makedirs(_BUILD, exist_ok=True)
    text = open(_SRC).read()
    for old, new in replacements:
        if text.count(old) != 1:
            raise ValueError(f"replacement target not unique: {old!r}")
        text = text.replace(old, new)
    src = os.path.join(_BUILD, f"variant_{tag}.c")
    out = os.path.join(_BUILD, f"liboracle_{tag}.so")
    with open(src, "w") as f:
        f.write(text)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           "-D_GNU_SOURCE", src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return _declare(ctypes.CDLL(out))


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    lib.or_flm.restype = ctypes.c_double
    lib.or_flm.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.or_adk_rate.restype = ctypes.c_double
    lib.or_adk_rate.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, _dp]
    lib.or_expm.restype = None
    lib.or_expm.argtypes = [ctypes.c_int, _dp, _dp]
    lib.or_rates.restype = ctypes.c_int
    lib.or_rates.argtypes = [ctypes.c_int, _dp, _ip, _ip, _dp, ctypes.c_int64,
                             _dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int]
    lib.or_step.restype = ctypes.c_int
    lib.or_step.argtypes = [ctypes.c_int, _dp, _ip, _ip, _dp, ctypes.c_int64,
                            _dp, _dp, ctypes.c_int64, ctypes.c_double, _u8p, _u8p,
                            _dp, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.or_num_threads.restype = ctypes.c_int
    lib.or_num_threads.argtypes = []
    return lib


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t)


#: rate models: Eq. 1 as printed (cycle-averaged), or the static-field rate
ADK_CYCLE_AVERAGED = 0
ADK_STATIC = 1


def _consts(constants, model: int = ADK_CYCLE_AVERAGED):
    c = list(constants if constants is not None else PAPER_CONSTANTS)[:3]
    return np.ascontiguousarray(c + [float(model)], dtype=np.float64)


def flm(l: int, m: int, _lib=None) -> float:
    return (_lib or lib()).or_flm(int(l), int(m))


def adk_rate(E: float, U: float, l: int, m: int, Q: int, constants=None,
             _lib=None, model: int = ADK_CYCLE_AVERAGED) -> float:
    """Eq. 1, W in 1/fs, for one transition with charge after ionization Q
    (model ADK_STATIC: without the cycle-averaging factor)."""
    c = _consts(constants, model)
    return (_lib or lib()).or_adk_rate(float(E), float(U), int(l), int(m),
                                       int(Q), _ptr(c, _dp))


def expm(M, _lib=None) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.float64)
    n = M.shape[0]
    X = np.zeros_like(M)
    (_lib or lib()).or_expm(n, _ptr(M, _dp), _ptr(X, _dp))
    return X


class Species:
    """Per-state data of one gas: U_k (eV), l_k, m_k for k = 0..Z-1, where
    state k is ionized to k+1 by the rate W_k."""

    def __init__(self, U, l, m, constants=None, model: int = ADK_CYCLE_AVERAGED):
        self.U = np.ascontiguousarray(U, dtype=np.float64)
        self.l = np.ascontiguousarray(l, dtype=np.int32)
        self.m = np.ascontiguousarray(m, dtype=np.int32)
        self.Z = int(self.U.shape[0])
        self.constants = _consts(constants, model)

    def _args(self):
        return (self.Z, _ptr(self.U, _dp), _ptr(self.l, _ip), _ptr(self.m, _ip),
                _ptr(self.constants, _dp))


def rates(sp: Species, E, k_lo: int, k_hi: int, nthreads: int = 0,
          _lib=None) -> np.ndarray:
    """W_k(E_c) in 1/fs for k in [k_lo, k_hi), shape (k_hi-k_lo, ncells)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    n = E.shape[0]
    W = np.zeros((k_hi - k_lo, n), dtype=np.float64)
    rc = (_lib or lib()).or_rates(*sp._args(), n, _ptr(E, _dp), int(k_lo),
                                  int(k_hi), _ptr(W, _dp), int(nthreads))
    if rc != 0:
        raise ValueError(f"or_rates rejected its arguments ({rc})")
    return W


#: window policies: the paper's shift rule, and the adaptive width
WINDOW_FIXED = 0
WINDOW_ADAPTIVE = 1


def step(sp: Species, E, N, dt: float, lo, hi, n_gas=None,
         eps_shift: float = 1e-6, window_update: bool = True,
         nthreads: int = 0, _lib=None, policy: int = WINDOW_FIXED,
         w_min: int = 2, w_max: int = 6, eps_grow: float = 1e-6):
    """One windowed analytic step.  Returns (N', lo', hi', dne) as new arrays;
    N has shape (Z+1, ncells).  policy WINDOW_ADAPTIVE: after the step, while
    the lowest state holds less than eps_shift it is dropped (width above
    w_min) or the window slides; then, if the old top state holds more than
    eps_grow, the state above joins (width at most w_max)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    N = np.array(N, dtype=np.float64, order="C", copy=True)
    lo = np.array(lo, dtype=np.uint8, copy=True)
    hi = np.array(hi, dtype=np.uint8, copy=True)
    n = E.shape[0]
    if N.shape != (sp.Z + 1, n):
        raise ValueError("N must have shape (Z+1, ncells)")
    dne = np.zeros(n, dtype=np.float64)
    ng = None if n_gas is None else np.ascontiguousarray(n_gas, dtype=np.float64)
    rc = (_lib or lib()).or_step(*sp._args(), n, _ptr(E, _dp), _ptr(N, _dp), n,
                                 float(dt), _ptr(lo, _u8p), _ptr(hi, _u8p),
                                 _ptr(dne, _dp),
                                 None if ng is None else _ptr(ng, _dp),
                                 float(eps_shift), int(bool(window_update)),
                                 int(policy), int(w_min), int(w_max), float(eps_grow),
                                 int(nthreads))
    if rc != 0:
        raise ValueError(f"or_step rejected its arguments ({rc})")
    return N, lo, hi, dne


def num_threads() -> int:
    return lib().or_num_threads()
