"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every symbol include/ionize.h declares, and rejects bad arguments on the host
before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_2202_10647_gb300 import build as B
from paper_2202_10647_gb300 import ionize

HEADER = os.path.join(B.INCLUDE, "ionize.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"ION_API\s+[\w\s\*]+?\b(ion_\w+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(ionize.EXPORTS)


def test_library_loads_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm_103a_only():
    # one -gencode, sm_103a, both for the CUDA library and in what build()
    # passes to every nvcc call
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.gpu
def test_loaded_device_code_is_sm_103():
    # the CUDA runtime's own view of the loaded module (no binary tools)
    lib = ionize.lib()
    assert lib.ion_binary_version() == 103, lib.ion_last_error()


def test_host_side_rejections():
    lib = ionize.lib()
    d = (ctypes.c_double * 3)(10.0, 20.0, 30.0)
    i3 = (ctypes.c_int * 3)(0, 1, 0)
    m_bad = (ctypes.c_int * 3)(0, 2, 0)   # |m| > l
    h = ctypes.c_void_p()
    assert lib.ion_species_init(d, i3, i3, 0, None, ctypes.byref(h)) == ionize.ION_EINVAL
    assert lib.ion_species_init(d, i3, i3, 64, None, ctypes.byref(h)) == ionize.ION_EINVAL
    assert lib.ion_species_init(d, i3, m_bad, 3, None, ctypes.byref(h)) == ionize.ION_EINVAL
    assert b"m" in lib.ion_last_error()
    neg = (ctypes.c_double * 3)(10.0, -1.0, 30.0)
    assert lib.ion_species_init(neg, i3, i3, 3, None, ctypes.byref(h)) == ionize.ION_EINVAL
    assert lib.ion_species_init(d, i3, i3, 3, None, None) == ionize.ION_EINVAL
    # an unknown rate model and bad constants are rejected before any CUDA call
    bad_model = ionize._Constants(4.13e16, 510.0, 13.6, 7)
    assert lib.ion_species_init(d, i3, i3, 3, ctypes.byref(bad_model),
                                ctypes.byref(h)) == ionize.ION_EINVAL
    assert b"rate_model" in lib.ion_last_error()
    bad_const = ionize._Constants(4.13e16, -510.0, 13.6, ionize.ION_ADK_STATIC)
    assert lib.ion_species_init(d, i3, i3, 3, ctypes.byref(bad_const),
                                ctypes.byref(h)) == ionize.ION_EINVAL
    # NULL species is rejected before anything else
    assert lib.ion_step(None, None, None, 0, 0, 0.05, None, None, None, None, None, 0,
                        None, 0, None) == ionize.ION_EINVAL
    assert lib.ion_rates(None, None, 0, 0, 0, None, 0, 0, None) == ionize.ION_EINVAL
    assert lib.ion_species_z(None) == ionize.ION_EINVAL
    assert lib.ion_species_destroy(None) == ionize.ION_OK


def test_workspace_sizes():
    assert ionize.workspace_bytes(0) == 256
    # header + FP64 queue (5 B/cell) + stiff records (35 B/cell), each of the
    # seven sections 256-byte aligned
    for n in (1, 31, 32, 1000, 33554432):
        assert 256 + 40 * n <= ionize.workspace_bytes(n) <= 256 + 40 * n + 7 * 256
    assert ionize.workspace_bytes(1000, ionize.ION_F64_PLAIN) == 256
