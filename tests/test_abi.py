"""C ABI checks that need no GPU: the library builds and loads, exports every function that
the headers under include/ declare, and its host-side argument validation returns the documented status
codes without touching the device."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    txt = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"^(?:lisa_status|size_t|int32_t|const char\*)\s+(lisa_\w+)\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_06300_gb300 import binding
    return binding.load()


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2507_06300_gb300 import binding
    assert sorted(binding.EXPORTS) == declared_functions()


def test_status_strings(lib):
    for code in range(9):
        assert lib.lisa_status_string(code)
    assert b"unknown" in lib.lisa_status_string(99)


def test_null_arguments_are_rejected_on_the_host(lib):
    from paper_2507_06300_gb300 import binding as B
    LISA_ERR_NULL = 1
    out = ctypes.c_void_p()
    assert lib.lisa_data_create(None, None, ctypes.byref(out)) == LISA_ERR_NULL
    assert lib.lisa_data_destroy(None) == LISA_ERR_NULL
    assert lib.lisa_spline_setup(None, None, 0, None, 0, None, None) == LISA_ERR_NULL
    assert lib.lisa_psd_loglike(None, None, None, 0, 0, None, None, 0, 0, None) == LISA_ERR_NULL
    assert lib.lisa_psd_loglike_noalloc(None, None, None, 0, 0, None, 0, None) == LISA_ERR_NULL
    assert lib.lisa_model_psd(None, None, None, 0, 0, None, None) == LISA_ERR_NULL
    assert lib.lisa_spline_buf_bytes(None, 4, 0) == 0
    assert lib.lisa_workspace_bytes(None, 4, 0, 0) == 0
    assert lib.lisa_pipe_rates(2048, 1, None, None) == LISA_ERR_NULL
    assert lib.lisa_data_set_profiling(None, 1) == LISA_ERR_NULL
    assert lib.lisa_data_kernel_ms(None, None) == LISA_ERR_NULL


def test_pipe_rates_validates_before_touching_the_device(lib):
    LISA_ERR_VALUE = 2
    out = (ctypes.c_double * 5)()
    assert lib.lisa_pipe_rates(8, 1, out, None) == LISA_ERR_VALUE
    assert lib.lisa_pipe_rates(2048, 0, out, None) == LISA_ERR_VALUE


def test_bad_descriptions_are_rejected_before_any_device_work(lib):
    import numpy as np
    from paper_2507_06300_gb300 import binding as B
    d = B.lisa_data_desc()
    d.n_datasets, d.n_channels, d.sgwb_model, d.tdi_form = 1, 4, 1, 0      # 4 channels: invalid
    out = ctypes.c_void_p()
    assert lib.lisa_data_create(ctypes.byref(d), None, ctypes.byref(out)) == 2   # LISA_ERR_VALUE
    d.n_channels = 3
    assert lib.lisa_data_create(ctypes.byref(d), None, ctypes.byref(out)) == 1   # NULL arrays
    # unordered frequencies -> LISA_ERR_DATA, found by the host validation
    N = 4
    arr = {k: np.ascontiguousarray(v) for k, v in dict(
        bo=np.array([0, N], np.int64), so=np.array([0, 1], np.int64), f=np.array([1e-3, 2e-3, 1.5e-3, 3e-3]),
        nu=np.ones(N), P=np.ones(3 * N), R=np.ones(3 * N), xlo=np.array([-4.0]), xhi=np.array([-1.0]),
        fr=np.array([1e-3])).items()}
    P64 = ctypes.POINTER(ctypes.c_double)
    d.bin_offset = arr["bo"].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.state_offset = arr["so"].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    for fld, key in (("freq", "f"), ("nu", "nu"), ("periodogram", "P"), ("response", "R"), ("x_lo", "xlo"),
                     ("x_hi", "xhi"), ("f_ref", "fr")):
        setattr(d, fld, arr[key].ctypes.data_as(P64))
    assert lib.lisa_data_create(ctypes.byref(d), None, ctypes.byref(out)) == 4   # LISA_ERR_DATA


def test_release_build_has_no_index_checks(lib):
    """The release library compiles the index checks away: it reports them off, refuses the
    self-test without launching anything, and rejects a null report pointer on the host."""
    assert lib.lisa_debug_bounds_enabled() == 0
    LISA_ERR_NULL, LISA_ERR_VALUE = 1, 2
    assert lib.lisa_debug_bounds(0, None) == LISA_ERR_NULL
    assert lib.lisa_debug_bounds_selftest(None) == LISA_ERR_VALUE
