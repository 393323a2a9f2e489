"""Thin Python binding of ``include/lisa_psd.h`` (ctypes; argument marshalling only).

Every step of the likelihood runs in the CUDA library ``lib/liblisa_psd.so``; this module only
passes device pointers (from torch tensors) and the current CUDA stream.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.

Names follow the C ABI: ``Dataset`` wraps ``lisa_data`` (create / destroy / tiling),
``Dataset.spline_setup`` -> ``lisa_spline_setup``, ``Dataset.psd_loglike`` -> ``lisa_psd_loglike``,
``Dataset.psd_loglike_grad`` -> ``lisa_psd_loglike_grad``, ``Dataset.model_psd`` -> ``lisa_model_psd``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

FP32, FP64 = 0, 1
AKIMA, NATURAL = 0, 1
SGWB_NONE, SGWB_POWER_LAW, SGWB_BROKEN = 0, 1, 2
TDI_PRINTED, TDI_SIN2_2U = 0, 1
COV_DIAGONAL, COV_FULL = 0, 1
N_THETA = 5
MAX_KNOTS = 62

STATE_BITS = {1: "bad_count", 2: "bad_position", 4: "duplicate", 8: "bad_amplitude", 16: "bad_theta",
              32: "nonfinite"}

_c_i32, _c_i64, _c_dbl, _c_vp, _c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_P_i64 = ctypes.POINTER(_c_i64)
_P_dbl = ctypes.POINTER(_c_dbl)


class lisa_data_desc(ctypes.Structure):
    _fields_ = [("n_datasets", _c_i32), ("n_channels", _c_i32), ("sgwb_model", _c_i32), ("tdi_form", _c_i32),
                ("bin_offset", _P_i64), ("state_offset", _P_i64), ("freq", _P_dbl), ("nu", _P_dbl),
                ("periodogram", _P_dbl), ("response", _P_dbl), ("x_lo", _P_dbl), ("x_hi", _P_dbl),
                ("f_ref", _P_dbl), ("cov_model", _c_i32), ("periodogram_cross", _P_dbl)]


class lisa_params(ctypes.Structure):
    _fields_ = [("n_states", _c_i32), ("theta_dev", _c_vp)]


class lisa_knots(ctypes.Structure):
    _fields_ = [("n_states", _c_i32), ("n_splines", _c_i32), ("kmax", _c_i32), ("kind", _c_i32),
                ("count_dev", _c_vp), ("x_dev", _c_vp), ("w_dev", _c_vp)]


class lisa_bounds_report(ctypes.Structure):
    _fields_ = [("count", _c_i64), ("first_index", _c_i64), ("first_line", _c_i32),
                ("first_file", ctypes.c_char * 96)]


class lisa_tiling(ctypes.Structure):
    _fields_ = [("tile_bins", _c_i32), ("states_per_cta", _c_i32), ("group", _c_i32), ("ctas_per_sm", _c_i32)]


class lisa_data_info(ctypes.Structure):
    _fields_ = [("n_bins", _c_i64), ("n_states", _c_i64), ("n_datasets", _c_i32), ("n_channels", _c_i32),
                ("n_splines", _c_i32), ("sgwb_model", _c_i32), ("n_items", _c_i64), ("n_sm", _c_i32),
                ("tiling", lisa_tiling)]


EXPORTS = ["lisa_data_create", "lisa_data_destroy", "lisa_data_get_info", "lisa_data_set_tiling",
           "lisa_spline_buf_bytes", "lisa_spline_setup", "lisa_workspace_bytes", "lisa_psd_loglike",
           "lisa_psd_loglike_grad", "lisa_model_psd", "lisa_psd_loglike_noalloc", "lisa_status_string",
           "lisa_pipe_rates", "lisa_data_set_profiling", "lisa_data_kernel_ms", "lisa_fd_synthesize",
           "lisa_averaged_periodogram", "lisa_workspace_status", "lisa_data_set_test_wait",
           "lisa_debug_bounds_enabled", "lisa_debug_bounds", "lisa_debug_bounds_selftest"]
PIPE_OPS = ("ex2", "rcp", "lg2_ex2", "ffma", "ffma2", "dfma", "mix")   # order of lisa_pipe_op
NOALLOC_SCRATCH_BYTES = 4 * 1024 * 1024

_lock = threading.Lock()
_lib = None


class LisaError(RuntimeError):
    pass


def debug_requested() -> bool:
    """True when the environment asks for the bounds-checked library (``LISA_DEBUG_BOUNDS=1``)."""
    return os.environ.get("LISA_DEBUG_BOUNDS", "") not in ("", "0")


def library_path() -> str:
    return _build.LIB_DEBUG if debug_requested() else _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads the CUDA library (building it in-tree if needed): ``liblisa_psd.so``, or the
    bounds-checked ``liblisa_psd_debug.so`` when ``LISA_DEBUG_BOUNDS=1`` is set before the first
    call.  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        debug = debug_requested()
        path = library_path()
        if not os.path.exists(path) or not _build.up_to_date(debug):
            if not build_if_missing:
                raise LisaError(f"CUDA library not built: {path}")
            _build.build(debug=debug)
        lib = ctypes.CDLL(path)
        S = _c_i32  # enum lisa_status
        lib.lisa_data_create.argtypes = [ctypes.POINTER(lisa_data_desc), _c_vp, ctypes.POINTER(_c_vp)]
        lib.lisa_data_create.restype = S
        lib.lisa_data_destroy.argtypes = [_c_vp]
        lib.lisa_data_destroy.restype = S
        lib.lisa_data_get_info.argtypes = [_c_vp, ctypes.POINTER(lisa_data_info)]
        lib.lisa_data_get_info.restype = S
        lib.lisa_data_set_tiling.argtypes = [_c_vp, ctypes.POINTER(lisa_tiling)]
        lib.lisa_data_set_tiling.restype = S
        lib.lisa_spline_buf_bytes.argtypes = [_c_vp, _c_i32, _c_i32]
        lib.lisa_spline_buf_bytes.restype = _c_sz
        lib.lisa_spline_setup.argtypes = [_c_vp, ctypes.POINTER(lisa_knots), _c_i32, _c_vp, _c_sz, _c_vp, _c_vp]
        lib.lisa_spline_setup.restype = S
        lib.lisa_workspace_bytes.argtypes = [_c_vp, _c_i32, _c_i32, _c_i32]
        lib.lisa_workspace_bytes.restype = _c_sz
        lib.lisa_psd_loglike.argtypes = [_c_vp, ctypes.POINTER(lisa_params), _c_vp, _c_sz, _c_i32, _c_vp, _c_vp,
                                         _c_sz, _c_i32, _c_vp]
        lib.lisa_psd_loglike.restype = S
        lib.lisa_psd_loglike_grad.argtypes = [_c_vp, ctypes.POINTER(lisa_params), ctypes.POINTER(lisa_knots), _c_vp,
                                              _c_sz, _c_vp, _c_vp, _c_vp, _c_sz, _c_i32, _c_vp]
        lib.lisa_psd_loglike_grad.restype = S
        lib.lisa_model_psd.argtypes = [_c_vp, ctypes.POINTER(lisa_params), _c_vp, _c_sz, _c_i32, _c_vp, _c_vp]
        lib.lisa_model_psd.restype = S
        lib.lisa_psd_loglike_noalloc.argtypes = [_c_vp, ctypes.POINTER(lisa_params), _c_vp, _c_sz, _c_i32, _c_vp,
                                                 _c_i32, _c_vp]
        lib.lisa_psd_loglike_noalloc.restype = S
        lib.lisa_status_string.argtypes = [_c_i32]
        lib.lisa_status_string.restype = ctypes.c_char_p
        lib.lisa_pipe_rates.argtypes = [_c_i32, _c_i32, ctypes.POINTER(_c_dbl), _c_vp]
        lib.lisa_pipe_rates.restype = S
        lib.lisa_data_set_profiling.argtypes = [_c_vp, _c_i32]
        lib.lisa_data_set_profiling.restype = S
        lib.lisa_data_kernel_ms.argtypes = [_c_vp, ctypes.POINTER(ctypes.c_float)]
        lib.lisa_data_kernel_ms.restype = S
        lib.lisa_fd_synthesize.argtypes = [_c_vp, _c_vp, _c_i32, _c_i64, _c_vp, _c_vp]
        lib.lisa_fd_synthesize.restype = S
        lib.lisa_averaged_periodogram.argtypes = [_c_vp, _c_i32, _c_i64, _c_dbl, _c_dbl, _c_vp, _c_i64, _c_vp, _c_vp,
                                                  _c_vp, _c_vp]
        lib.lisa_averaged_periodogram.restype = S
        lib.lisa_workspace_status.argtypes = [_c_vp, _c_vp]
        lib.lisa_workspace_status.restype = S
        lib.lisa_data_set_test_wait.argtypes = [_c_vp, _c_i32, ctypes.c_uint32]
        lib.lisa_data_set_test_wait.restype = S
        lib.lisa_debug_bounds_enabled.argtypes = []
        lib.lisa_debug_bounds_enabled.restype = _c_i32
        lib.lisa_debug_bounds.argtypes = [_c_i32, ctypes.POINTER(lisa_bounds_report)]
        lib.lisa_debug_bounds.restype = S
        lib.lisa_debug_bounds_selftest.argtypes = [_c_vp]
        lib.lisa_debug_bounds_selftest.restype = S
        _lib = lib
        return lib


def debug_bounds_enabled() -> bool:
    """``lisa_debug_bounds_enabled``: whether the loaded library checks its indices."""
    return bool(load().lisa_debug_bounds_enabled())


def debug_bounds(reset: bool = False) -> dict:
    """``lisa_debug_bounds``: index violations since the last reset (synchronises the device)."""
    r = lisa_bounds_report()
    _check(load().lisa_debug_bounds(1 if reset else 0, ctypes.byref(r)), "lisa_debug_bounds")
    return {"count": int(r.count), "first_index": int(r.first_index), "first_line": int(r.first_line),
            "first_file": r.first_file.decode(errors="replace")}


def debug_bounds_selftest(stream=None) -> None:
    """``lisa_debug_bounds_selftest`` on ``stream`` (a torch stream; default: the current one)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(load().lisa_debug_bounds_selftest(ctypes.c_void_p(st.cuda_stream)), "lisa_debug_bounds_selftest")


def _check(st: int, what: str):
    if st != 0:
        msg = load().lisa_status_string(st).decode()
        raise LisaError(f"{what} failed: status {st} ({msg})")


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise LisaError("no CUDA device: the lisa_psd library runs on the GPU only")
    return torch


def _stream_handle(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _np_ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Dataset:
    """A ``lisa_data`` object: one or more datasets with their bins and states.

    Host arrays (numpy, FP64): freq [N], nu [N], periodogram [C, N], response [C, N] (or None for
    the noise-only model), bin_offset / state_offset [D+1], x_lo / x_hi / f_ref [D]; with
    cov_model=COV_FULL also periodogram_cross [3, N], the real parts of P_AE, P_AT, P_ET."""

    def __init__(self, *, n_channels, freq, nu, periodogram, response=None, bin_offset=None, state_offset=None,
                 n_states=None, x_lo, x_hi, f_ref, sgwb_model=SGWB_POWER_LAW, tdi_form=TDI_PRINTED,
                 cov_model=COV_DIAGONAL, periodogram_cross=None, stream=None):
        lib = load()
        torch = _torch()
        self.device = torch.cuda.current_device()
        freq = np.ascontiguousarray(freq, np.float64).ravel()
        N = freq.size
        if bin_offset is None:
            bin_offset = np.array([0, N], np.int64)
        if state_offset is None:
            state_offset = np.array([0, int(n_states)], np.int64)
        self._keep = dict(
            bin_offset=np.ascontiguousarray(bin_offset, np.int64), state_offset=np.ascontiguousarray(state_offset, np.int64),
            freq=freq, nu=np.ascontiguousarray(np.broadcast_to(np.asarray(nu, np.float64), (N,))),
            P=np.ascontiguousarray(periodogram, np.float64).reshape(n_channels, N),
            R=None if response is None else np.ascontiguousarray(response, np.float64).reshape(n_channels, N),
            x_lo=np.atleast_1d(np.ascontiguousarray(x_lo, np.float64)),
            x_hi=np.atleast_1d(np.ascontiguousarray(x_hi, np.float64)),
            f_ref=np.atleast_1d(np.ascontiguousarray(f_ref, np.float64)),
            X=None if periodogram_cross is None else np.ascontiguousarray(periodogram_cross, np.float64).reshape(3, N))
        k = self._keep
        D = k["bin_offset"].size - 1
        desc = lisa_data_desc(
            n_datasets=D, n_channels=int(n_channels), sgwb_model=int(sgwb_model), tdi_form=int(tdi_form),
            bin_offset=_np_ptr(k["bin_offset"], _c_i64), state_offset=_np_ptr(k["state_offset"], _c_i64),
            freq=_np_ptr(k["freq"], _c_dbl), nu=_np_ptr(k["nu"], _c_dbl), periodogram=_np_ptr(k["P"], _c_dbl),
            response=None if k["R"] is None else _np_ptr(k["R"], _c_dbl), x_lo=_np_ptr(k["x_lo"], _c_dbl),
            x_hi=_np_ptr(k["x_hi"], _c_dbl), f_ref=_np_ptr(k["f_ref"], _c_dbl), cov_model=int(cov_model),
            periodogram_cross=None if k["X"] is None else _np_ptr(k["X"], _c_dbl))
        h = _c_vp()
        _check(lib.lisa_data_create(ctypes.byref(desc), _stream_handle(stream), ctypes.byref(h)), "lisa_data_create")
        self._h = h
        self.n_channels = int(n_channels)
        self.sgwb_model = int(sgwb_model)
        self.cov_model = int(cov_model)
        self.n_splines = self.n_channels + (1 if sgwb_model else 0) + (3 if cov_model == COV_FULL else 0)
        self.n_states = int(k["state_offset"][-1])
        self.n_bins = N
        self.n_datasets = D
        self.bin_offset = k["bin_offset"]
        self.state_offset = k["state_offset"]

    @classmethod
    def from_workload(cls, wl, periodogram, **kw):
        """Dataset object for a ``synth.Workload`` with the given periodogram: [C, N] (diagonal
        covariance) or, for the full covariance, the nine rows P_AA, P_EE, P_TT, Re / Im of P_AE,
        P_AT, P_ET (only the real parts are passed on)."""
        P = np.asarray(periodogram)
        if P.shape[0] == 9:
            kw.setdefault("cov_model", COV_FULL)
            kw.setdefault("periodogram_cross", P[[3, 5, 7]])
            P = P[:3]
        return cls(n_channels=wl.n_channels, freq=wl.f, nu=wl.nu, periodogram=P,
                   response=wl.R if wl.sgwb_model else None, bin_offset=wl.bin_offset, state_offset=wl.state_offset,
                   x_lo=wl.x_lo, x_hi=wl.x_hi, f_ref=wl.f_ref, sgwb_model=wl.sgwb_model, tdi_form=wl.tdi_form, **kw)

    # ---- lifetime -------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lisa_data_destroy(self._h)
            self._h = _c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = lisa_data_info()
        _check(load().lisa_data_get_info(self._h, ctypes.byref(inf)), "lisa_data_get_info")
        t = inf.tiling
        return {"n_bins": inf.n_bins, "n_states": inf.n_states, "n_datasets": inf.n_datasets,
                "n_channels": inf.n_channels, "n_splines": inf.n_splines, "sgwb_model": inf.sgwb_model,
                "n_items": inf.n_items, "n_sm": inf.n_sm,
                "tiling": {"tile_bins": t.tile_bins, "states_per_cta": t.states_per_cta, "group": t.group,
                           "ctas_per_sm": t.ctas_per_sm}}

    def set_tiling(self, tile_bins=512, states_per_cta=128, group=4, ctas_per_sm=0):
        t = lisa_tiling(int(tile_bins), int(states_per_cta), int(group), int(ctas_per_sm))
        _check(load().lisa_data_set_tiling(self._h, ctypes.byref(t)), "lisa_data_set_tiling")

    def set_profiling(self, enable=True):
        """``lisa_data_set_profiling``: record per-kernel events in uncaptured likelihood calls."""
        _check(load().lisa_data_set_profiling(self._h, int(bool(enable))), "lisa_data_set_profiling")

    def kernel_ms(self):
        """``lisa_data_kernel_ms`` of the last recorded call: (main, compensated, finalize) in ms."""
        ms = (ctypes.c_float * 3)()
        _check(load().lisa_data_kernel_ms(self._h, ms), "lisa_data_kernel_ms")
        return tuple(float(v) for v in ms)

    # ---- sizes ----------------------------------------------------------------------------
    def spline_buf_bytes(self, kmax, precision):
        return int(load().lisa_spline_buf_bytes(self._h, int(kmax), int(precision)))

    def workspace_bytes(self, kmax, precision, with_grad=False):
        return int(load().lisa_workspace_bytes(self._h, int(kmax), int(precision), int(bool(with_grad))))

    # ---- entry points -----------------------------------------------------------------------
    def _knots(self, count, x, w, kmax, kind):
        return lisa_knots(self.n_states, self.n_splines, int(kmax), int(kind), count.data_ptr(),
                          x.data_ptr() if x.numel() else None, w.data_ptr())

    def spline_setup(self, count, x, w, kmax, kind=AKIMA, precision=FP32, buf=None, status=None, stream=None):
        """``lisa_spline_setup`` on device tensors count [S, nsp] int32, x [S, nsp, kmax] f64,
        w [S, nsp, kmax+2] f64.  Returns (spline buffer, per-state status int32)."""
        torch = _torch()
        nb = self.spline_buf_bytes(kmax, precision)
        if buf is None:
            buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
        if status is None:
            status = torch.empty(self.n_states, dtype=torch.int32, device="cuda")
        kn = self._knots(count, x, w, kmax, kind)
        _check(load().lisa_spline_setup(self._h, ctypes.byref(kn), int(precision), buf.data_ptr(), buf.numel(),
                                        status.data_ptr(), _stream_handle(stream)), "lisa_spline_setup")
        return buf, status

    def routed_states(self, buf):
        """Number of states the last FP32 lisa_spline_setup on ``buf`` routed to the compensated
        kernel (diagnostic; synchronises)."""
        a256 = lambda b: (b + 255) // 256 * 256
        off = a256(4 * self.n_states) + a256(4 * self.n_states * self.n_splines)
        return int(buf[off:off + 4].cpu().view(dtype=__import__("torch").int32)[0])

    def routed_list(self, buf):
        """State indices the last FP32 lisa_spline_setup on ``buf`` routed to the compensated
        kernel, ascending (diagnostic; synchronises)."""
        torch = _torch()
        a256 = lambda b: (b + 255) // 256 * 256
        off = a256(4 * self.n_states) + a256(4 * self.n_states * self.n_splines)
        words = buf[off:off + 4 * (self.n_states + 1)].cpu().view(dtype=torch.int32).numpy()
        return np.sort(words[1:1 + int(words[0])]).astype(np.int64)

    def psd_loglike(self, theta, buf, kmax, precision=FP32, out=None, workspace=None, stream=None):
        """``lisa_psd_loglike``: theta [S, 5] f64 device -> log L [S] f64 device."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.n_states, dtype=torch.float64, device="cuda")
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes(kmax, precision), dtype=torch.uint8, device="cuda")
        pr = lisa_params(self.n_states, theta.data_ptr())
        _check(load().lisa_psd_loglike(self._h, ctypes.byref(pr), buf.data_ptr(), buf.numel(), int(kmax),
                                       out.data_ptr(), workspace.data_ptr(), workspace.numel(), int(precision),
                                       _stream_handle(stream)), "lisa_psd_loglike")
        return out

    def workspace_status(self, workspace, stream=None):
        """``lisa_workspace_status``: synchronises the stream and returns the device-side status
        of the last likelihood call that used ``workspace`` (0, or 8 = LISA_ERR_TIMEOUT)."""
        return int(load().lisa_workspace_status(workspace.data_ptr(), _stream_handle(stream)))

    def set_test_wait(self, skip_copies=False, wait_limit=1 << 20):
        """``lisa_data_set_test_wait`` (tests of the timeout path only)."""
        _check(load().lisa_data_set_test_wait(self._h, int(bool(skip_copies)), int(wait_limit)),
               "lisa_data_set_test_wait")

    def psd_loglike_noalloc(self, theta, buf, kmax, precision=FP32, out=None, stream=None):
        """``lisa_psd_loglike_noalloc``: the same result as ``psd_loglike`` for callers that cannot
        allocate a workspace; the scratch lives in a fixed 4 MiB array inside the library (shared
        by all calls on the device, so calls must not overlap on the GPU)."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.n_states, dtype=torch.float64, device="cuda")
        pr = lisa_params(self.n_states, theta.data_ptr())
        _check(load().lisa_psd_loglike_noalloc(self._h, ctypes.byref(pr), buf.data_ptr(), buf.numel(), int(kmax),
                                               out.data_ptr(), int(precision), _stream_handle(stream)),
               "lisa_psd_loglike_noalloc")
        return out

    def psd_loglike_grad(self, theta, count, x, w, kmax, kind, buf, precision=FP32, out=None, grad=None,
                         workspace=None, stream=None):
        """``lisa_psd_loglike_grad``: returns (log L [S], grad [S, 5 + nsp*(2 kmax + 2)])."""
        torch = _torch()
        G = N_THETA + self.n_splines * (2 * int(kmax) + 2)
        if out is None:
            out = torch.empty(self.n_states, dtype=torch.float64, device="cuda")
        if grad is None:
            grad = torch.empty((self.n_states, G), dtype=torch.float64, device="cuda")
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes(kmax, precision, True), dtype=torch.uint8, device="cuda")
        pr = lisa_params(self.n_states, theta.data_ptr())
        kn = self._knots(count, x, w, kmax, kind)
        _check(load().lisa_psd_loglike_grad(self._h, ctypes.byref(pr), ctypes.byref(kn), buf.data_ptr(), buf.numel(),
                                            out.data_ptr(), grad.data_ptr(), workspace.data_ptr(), workspace.numel(),
                                            int(precision), _stream_handle(stream)), "lisa_psd_loglike_grad")
        return out, grad

    def model_psd(self, theta, buf64, kmax, out=None, stream=None):
        """``lisa_model_psd``: physical S_c(f_i) per state (FP64 spline buffer)."""
        torch = _torch()
        n = int(sum(self.n_channels * (self.state_offset[d + 1] - self.state_offset[d]) *
                    (self.bin_offset[d + 1] - self.bin_offset[d]) for d in range(self.n_datasets)))
        if out is None:
            out = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
        pr = lisa_params(self.n_states, theta.data_ptr())
        _check(load().lisa_model_psd(self._h, ctypes.byref(pr), buf64.data_ptr(), buf64.numel(), int(kmax),
                                     out.data_ptr(), _stream_handle(stream)), "lisa_model_psd")
        return out


def fd_synthesize(psd, normal, out=None, stream=None):
    """``lisa_fd_synthesize``: frequency-domain data d = sqrt(S/2) (z0 + i z1).  psd [C, N] and
    normal [C, N, 2] FP64 device tensors; returns d [C, N, 2] (FP64, interleaved re/im)."""
    torch = _torch()
    C, N = psd.shape
    if out is None:
        out = torch.empty((C, N, 2), dtype=torch.float64, device="cuda")
    _check(load().lisa_fd_synthesize(psd.data_ptr(), normal.data_ptr(), int(C), int(N), out.data_ptr(),
                                     _stream_handle(stream)), "lisa_fd_synthesize")
    return out


def averaged_periodogram(d, f0, df, bin_offset, stream=None):
    """``lisa_averaged_periodogram``: d [C, N, 2] FP64 device tensor, bin_offset [n_bins + 1]
    int64 device tensor; returns (P [C, n_bins], f [n_bins], nu [n_bins]) device tensors."""
    torch = _torch()
    C, N = d.shape[0], d.shape[1]
    nb = bin_offset.numel() - 1
    P = torch.empty((C, max(nb, 0)), dtype=torch.float64, device="cuda")
    f = torch.empty(max(nb, 0), dtype=torch.float64, device="cuda")
    nu = torch.empty(max(nb, 0), dtype=torch.float64, device="cuda")
    _check(load().lisa_averaged_periodogram(d.data_ptr(), int(C), int(N), float(f0), float(df), bin_offset.data_ptr(),
                                            int(nb), P.data_ptr(), f.data_ptr(), nu.data_ptr(),
                                            _stream_handle(stream)), "lisa_averaged_periodogram")
    return P, f, nu


def pipe_rates(iters=2048, reps=3, stream=None) -> dict:
    """``lisa_pipe_rates``: measured lane operations per second of the MUFU, FP32 and FP64 pipes on
    the current device, keyed by PIPE_OPS (a packed FMA counts two), and under "mix" the
    state-bins per second that the fused kernel's instruction mix allows.  Synchronises."""
    out = (_c_dbl * len(PIPE_OPS))()
    _check(load().lisa_pipe_rates(int(iters), int(reps), out, _stream_handle(stream)), "lisa_pipe_rates")
    return {k: float(out[i]) for i, k in enumerate(PIPE_OPS)}


def knots_to_device(knots, device="cuda"):
    """(count int32, x f64, w f64) device tensors from a synth.Knots / dict of numpy arrays."""
    torch = _torch()
    k = knots.as_dict() if hasattr(knots, "as_dict") else knots
    kmax = int(k["kmax"])
    count = torch.as_tensor(np.ascontiguousarray(k["count"], np.int32), device=device)
    x = torch.as_tensor(np.ascontiguousarray(np.asarray(k["x"], np.float64)[..., :kmax]), device=device)
    w = torch.as_tensor(np.ascontiguousarray(k["w"], np.float64), device=device)
    return count, x.contiguous(), w, kmax, int(k.get("kind", 0))


class Evaluator:
    """Preallocated hot path for one Dataset: knots / theta in, log L out.

    ``step()`` runs lisa_spline_setup + lisa_psd_loglike on device-resident inputs (the MCMC
    inner loop when the sampler lives on the GPU); ``loglike_host()`` is the end-to-end call of a
    host-side sampler: pinned host inputs are copied to the device, evaluated, and log L is copied
    back into pinned host memory.  ``capture()`` records step() into a CUDA graph;
    ``capture_host()`` records the whole host call (copies included) into one."""

    def __init__(self, dataset: Dataset, kmax: int, kind: int = AKIMA, precision: int = FP32):
        torch = _torch()
        self.ds, self.kmax, self.kind, self.precision = dataset, int(kmax), int(kind), int(precision)
        S, nsp = dataset.n_states, dataset.n_splines
        dev = "cuda"
        # the inputs live in one device block (and, for host callers, one pinned host block with
        # the same layout, see host_inputs), so the end-to-end call copies them in one transfer
        shapes = [((S, N_THETA), torch.float64), ((S, nsp), torch.int32), ((S, nsp, self.kmax), torch.float64),
                  ((S, nsp, self.kmax + 2), torch.float64)]
        self._in_layout, off = [], 0
        for shape, dt in shapes:
            n = int(np.prod(shape)) * torch.empty((), dtype=dt).element_size()
            self._in_layout.append((off, n, shape, dt))
            off += (n + 255) // 256 * 256
        self.inputs = torch.zeros(max(off, 256), dtype=torch.uint8, device=dev)
        self.theta, self.count, self.x, self.w = self._views(self.inputs)
        self.h_inputs = None
        self.buf = torch.empty(dataset.spline_buf_bytes(kmax, precision), dtype=torch.uint8, device=dev)
        self.status = torch.empty(S, dtype=torch.int32, device=dev)
        self.ws = torch.empty(dataset.workspace_bytes(kmax, precision), dtype=torch.uint8, device=dev)
        self.out = torch.empty(S, dtype=torch.float64, device=dev)
        self.graph = None

    def _views(self, block):
        return tuple(block[o:o + n].view(dt).view(shape) for o, n, shape, dt in self._in_layout)

    def host_inputs(self):
        """Pinned host tensors (theta, count, x, w) laid out like the device inputs: a host sampler
        that writes its proposals into them gets them to the device in one copy per call."""
        torch = _torch()
        if self.h_inputs is None:
            self.h_inputs = torch.zeros(self.inputs.numel(), dtype=torch.uint8).pin_memory()
            self.h_views = self._views(self.h_inputs)
        return self.h_views

    def load(self, theta, count, x, w):
        self.theta.copy_(theta)
        self.count.copy_(count)
        self.x.copy_(x)
        self.w.copy_(w)

    def setup(self, stream=None):
        self.ds.spline_setup(self.count, self.x, self.w, self.kmax, self.kind, self.precision, buf=self.buf,
                             status=self.status, stream=stream)

    def loglike(self, stream=None):
        return self.ds.psd_loglike(self.theta, self.buf, self.kmax, self.precision, out=self.out,
                                   workspace=self.ws, stream=stream)

    def step(self, stream=None):
        self.setup(stream)
        return self.loglike(stream)

    def capture(self):
        """Captures setup and log-likelihood as two CUDA graphs (so they can be timed apart)."""
        torch = _torch()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()  # warm (sets kernel attributes outside capture)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.g_setup, self.g_ll = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.g_setup):
            self.setup()
        with torch.cuda.graph(self.g_ll):
            self.loglike()
        self.graph = True
        return self

    def replay(self):
        self.g_setup.replay()
        self.g_ll.replay()
        return self.out

    @staticmethod
    def _require_pinned(*ts):
        # asynchronous copies from pageable memory silently become synchronous (eager calls) or
        # fail partway through a graph capture: the host path takes pinned tensors only
        for t in ts:
            if t.device.type != "cpu" or not t.is_pinned():
                raise LisaError("host tensors of the end-to-end call must be pinned CPU tensors "
                                "(torch.Tensor.pin_memory(), or the views host_inputs() returns)")

    def _host_step(self, theta, count, x, w, out, eager=False):
        mine = self.h_inputs is not None and all(a is b for a, b in zip(self.h_views, (theta, count, x, w)))
        if mine:
            self.inputs.copy_(self.h_inputs, non_blocking=True)
        else:
            self.theta.copy_(theta, non_blocking=True)
            self.count.copy_(count, non_blocking=True)
            self.x.copy_(x, non_blocking=True)
            self.w.copy_(w, non_blocking=True)
        if self.graph and not eager:
            self.replay()
        else:
            self.step()
        out.copy_(self.out, non_blocking=True)

    def capture_host(self, theta, count, x, w, out):
        """Captures the whole end-to-end call for these pinned host tensors as one CUDA graph:
        the copies in, spline setup, log-likelihood and the copy of log L into ``out``.  Later
        ``loglike_host`` calls with the same tensors replay it (one launch); the copies read
        whatever the tensors hold at that time, so a sampler refills them in place each step."""
        torch = _torch()
        self._require_pinned(theta, count, x, w, out)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._host_step(theta, count, x, w, out, eager=True)   # warm (kernel attributes set outside capture)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._host_step(theta, count, x, w, out, eager=True)
        self.g_host, self.host_args = g, (theta, count, x, w, out)
        return self

    def loglike_host(self, theta, count, x, w, out):
        """End-to-end: pinned host tensors in (theta [S,5] f64, count [S,nsp] i32, x, w f64),
        log L written into the pinned host tensor ``out`` [S]; returns ``out`` after the copy."""
        torch = _torch()
        self._require_pinned(theta, count, x, w, out)
        held = getattr(self, "host_args", None)
        if held is not None and all(a is b for a, b in zip(held, (theta, count, x, w, out))):
            self.g_host.replay()
        else:
            self._host_step(theta, count, x, w, out)
        torch.cuda.current_stream().synchronize()
        return out


def _make_autograd():
    import torch

    class PsdLogLike(torch.autograd.Function):
        """log L(theta, knot amplitudes, knot positions) for every state, differentiable.

        forward runs lisa_spline_setup and, when a gradient is wanted, lisa_psd_loglike_grad (the
        hand-written adjoint, which also returns log L; the spline coefficients are recomputed
        from the knots, nothing per bin is stored), else lisa_psd_loglike.  backward only scales
        the stored per-state gradient rows by the incoming gradient.  Knot counts (the
        reversible-jump dimension) are not differentiable."""

        @staticmethod
        def forward(ctx, theta, w, x, dataset, count, kmax, kind, precision):
            need = ctx.needs_input_grad[0] or ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
            theta_c, w_c, x_c = theta.detach().contiguous(), w.detach().contiguous(), x.detach().contiguous()
            buf, _ = dataset.spline_setup(count, x_c, w_c, kmax, kind, precision)
            if not need:
                return dataset.psd_loglike(theta_c, buf, kmax, precision)
            out, grad = dataset.psd_loglike_grad(theta_c, count, x_c, w_c, kmax, kind, buf, precision)
            ctx.save_for_backward(grad)
            ctx.shape = (dataset.n_splines, int(kmax))
            return out

        @staticmethod
        def backward(ctx, g_out):
            (grad,) = ctx.saved_tensors
            nsp, kmax = ctx.shape
            S = grad.shape[0]
            g = grad * g_out.reshape(S, 1)
            per = 2 * kmax + 2
            body = g[:, N_THETA:].reshape(S, nsp, per)
            g_theta = g[:, :N_THETA]
            g_w = body[:, :, :kmax + 2]
            g_x = body[:, :, kmax + 2:]
            return g_theta, g_w, g_x, None, None, None, None, None

    return PsdLogLike


_PsdLogLike = None


def psd_loglike(dataset, theta, w, x, count, kmax, kind=AKIMA, precision=FP32):
    """Differentiable log-likelihood of every state (see PsdLogLike): theta [S,5], w [S,nsp,kmax+2],
    x [S,nsp,kmax] (device tensors, FP64, requires_grad allowed), count [S,nsp] int32."""
    global _PsdLogLike
    if _PsdLogLike is None:
        _PsdLogLike = _make_autograd()
    return _PsdLogLike.apply(theta, w, x, dataset, count, int(kmax), int(kind), int(precision))
