"""ctypes binding of the srw C ABI (``include/srw.h``).

Argument marshalling only: every computation runs in the CUDA library
``libsrw.so``.  The functions carry the C names.  Host arguments are numpy
arrays; device arguments are CUDA tensors (anything with ``data_ptr()`` and
``is_cuda``), in which case the call is stream-ordered on the given stream
(default: torch's current stream).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SRW_LIB=debug selects the debug build (bounds checks compiled in, SRW_ECHECK)
LIB_PATH = os.path.join(_HERE, "libsrw_debug.so" if os.environ.get("SRW_LIB") == "debug" else "libsrw.so")

SRW_OK, SRW_EINVAL, SRW_ENOMEM, SRW_ECUDA, SRW_ENODATA, SRW_EDOMAIN, SRW_ETIMEOUT, SRW_EUNSUPPORTED, SRW_ECHECK = range(9)
SRW_HOST, SRW_DEVICE = 0, 1
SRW_FP32, SRW_BF16, SRW_BF16X3, SRW_FP16X3 = 0, 1, 2, 3
SRW_SCAN_FLAG_CELLS, SRW_SCAN_ERROR_BARS = 0, 1
SRW_RANK8 = 16  # srw_surrogate_scan_exact: the exact rank-8 evaluator
PRECISIONS = {"fp32": SRW_FP32, "bf16": SRW_BF16, "bf16x3": SRW_BF16X3, "fp16x3": SRW_FP16X3}

# Entry points declared in include/srw.h (checked by the test-suite).
EXPORTS = ("srw_create", "srw_set_data", "srw_spectrum", "srw_spectrum_batch", "srw_loglik", "srw_loglik_points", "srw_get_basis",
           "srw_autotune", "srw_info", "srw_set_reference", "srw_profile", "srw_profile_read", "srw_last_error", "srw_status_string",
           "srw_destroy", "srw_loglik_point_noalloc", "srw_noalloc_last_error", "srw_group_create", "srw_group_loglik",
           "srw_group_autotune", "srw_group_set_schedule", "srw_group_schedule", "srw_group_profile", "srw_group_profile_read",
           "srw_group_last_error", "srw_group_destroy", "srw_surrogate_create", "srw_surrogate_set_weights",
           "srw_surrogate_get_weights", "srw_surrogate_forward", "srw_surrogate_gradients", "srw_surrogate_train_step",
           "srw_surrogate_last_error", "srw_surrogate_destroy", "srw_surrogate_fit", "srw_surrogate_loglik",
           "srw_surrogate_scan", "srw_surrogate_scan_exact", "srw_surrogate_sobol", "srw_surrogate_get_standardization",
           "srw_diag_wait_timeout", "srw_loglik_linear", "srw_loglik_profiled", "srw_create_joint", "srw_joint_layout",
           "srw_fold_work", "srw_fault_inject", "srw_fault_pending", "srw_fault_parse", "srw_fold_config",
           "srw_set_fold_config", "srw_check", "srw_get_fold_config",
           "srw_surrogate_save", "srw_surrogate_load", "srw_surrogate_fit_resume", "srw_surrogate_scan_chunked",
           "srw_gemv_work")


class SrwError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("srw status %d: %s" % (status, message))
        self.status = status


class _Binning(ctypes.Structure):
    _fields_ = [("n_t", ctypes.c_int), ("t_edges", ctypes.POINTER(ctypes.c_double)), ("n_rec", ctypes.c_int),
                ("t_min", ctypes.c_double), ("midpoint", ctypes.c_int)]


class _Source(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int), ("e", ctypes.POINTER(ctypes.c_double)),
                ("w", ctypes.POINTER(ctypes.c_double)), ("pee", ctypes.POINTER(ctypes.c_double))]


class _Options(ctypes.Structure):
    _fields_ = [("sin2w", ctypes.c_double), ("f_tau", ctypes.c_double), ("exposure", ctypes.c_double),
                ("e_true_sm", ctypes.POINTER(ctypes.c_double))]


class _JointResponse(ctypes.Structure):
    _fields_ = [("hist", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("mask", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("scale", ctypes.POINTER(ctypes.c_double)), ("live", ctypes.POINTER(ctypes.c_double)),
                ("events", ctypes.POINTER(ctypes.c_double))]


class _Info(ctypes.Structure):
    _fields_ = [("n_t", ctypes.c_int), ("n_rec", ctypes.c_int), ("n_nodes", ctypes.c_int), ("k_pad", ctypes.c_int),
                ("device", ctypes.c_int), ("sm_count", ctypes.c_int), ("tensor_path", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("device_bytes", ctypes.c_size_t)]


_lib = None


class _FitOpts(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("epochs", ctypes.c_int), ("lr", ctypes.c_float), ("lr_final", ctypes.c_float),
                ("precision", ctypes.c_int)]


class _ScanOpts(ctypes.Structure):
    _fields_ = [("first", ctypes.c_longlong), ("n_points", ctypes.c_longlong), ("keep_frac", ctypes.c_double),
                ("check_theta", ctypes.c_void_p), ("n_check", ctypes.c_int), ("tol", ctypes.c_double),
                ("cells_per_dim", ctypes.c_int), ("precision", ctypes.c_int), ("rule", ctypes.c_int),
                ("margin_factor", ctypes.c_double)]


class _ScanResult(ctypes.Structure):
    _fields_ = [("best_value", ctypes.c_double), ("best_index", ctypes.c_longlong), ("best_theta", ctypes.c_float * 5),
                ("surrogate_min", ctypes.c_double), ("n_kept", ctypes.c_longlong), ("n_selected", ctypes.c_longlong),
                ("n_rescued", ctypes.c_longlong),
                ("n_cells", ctypes.c_int), ("n_flagged_cells", ctypes.c_int), ("check_max_abs_d", ctypes.c_double),
                ("ms_check", ctypes.c_float), ("ms_surrogate", ctypes.c_float), ("ms_select", ctypes.c_float),
                ("ms_exact", ctypes.c_float)]


def lib():
    """Load ``libsrw.so``; fails loudly if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsrw.so is not built (run paper_2607_00488_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp, fp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
        L.srw_create.argtypes = [ctypes.POINTER(_Binning), ctypes.POINTER(_Source), ip, vp,
                                 ctypes.POINTER(_Options), ctypes.POINTER(vp)]
        L.srw_create_joint.argtypes = [ctypes.POINTER(_Binning), ctypes.POINTER(_Source), ip,
                                       ctypes.POINTER(_JointResponse), ctypes.POINTER(_Options), ctypes.POINTER(vp)]
        L.srw_joint_layout.argtypes = [vp, ctypes.POINTER(ctypes.c_int), vp, vp]
        L.srw_fold_work.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_double)]
        L.srw_gemv_work.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
        L.srw_set_data.argtypes = [vp, dp, dp, ip, vp]
        L.srw_spectrum.argtypes = [vp, fp, ip, fp, ip, vp]
        L.srw_loglik.argtypes = [vp, fp, ip, vp, ip, ip, vp]
        L.srw_spectrum_batch.argtypes = [vp, fp, ip, vp, ip, ip, vp]
        L.srw_loglik_points.argtypes = [vp, fp, ip, vp, ip, vp]
        L.srw_get_basis.argtypes = [vp, dp]
        L.srw_autotune.argtypes = [vp, ip, ip, ctypes.c_char_p, vp, ctypes.POINTER(ctypes.c_int)]
        L.srw_info.argtypes = [vp, ctypes.POINTER(_Info)]
        L.srw_set_reference.argtypes = [vp, vp]
        L.srw_profile.argtypes = [vp, ip]
        L.srw_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        L.srw_last_error.argtypes = [vp]
        L.srw_last_error.restype = ctypes.c_char_p
        L.srw_status_string.argtypes = [ip]
        L.srw_status_string.restype = ctypes.c_char_p
        L.srw_destroy.argtypes = [vp]
        L.srw_loglik_point_noalloc.argtypes = [vp, ip, ip, vp, vp, vp, vp, vp, vp]
        L.srw_noalloc_last_error.argtypes = []
        L.srw_noalloc_last_error.restype = ctypes.c_char_p
        ipp = ctypes.POINTER(ctypes.c_int)
        L.srw_group_create.argtypes = [vp, ip, vp, ctypes.POINTER(vp)]
        L.srw_group_loglik.argtypes = [vp, vp, vp, ip, ip, vp]
        L.srw_group_autotune.argtypes = [vp, ip, vp, ipp]
        L.srw_group_set_schedule.argtypes = [vp, ip, ip]
        L.srw_group_schedule.argtypes = [vp, ip, ipp, ipp, ipp, ipp, ipp]
        L.srw_group_profile.argtypes = [vp, ip]
        L.srw_group_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        L.srw_group_last_error.argtypes = [vp]
        L.srw_group_last_error.restype = ctypes.c_char_p
        L.srw_group_destroy.argtypes = [vp]
        L.srw_surrogate_create.argtypes = [vp, vp, vp, vp, ctypes.POINTER(vp)]
        L.srw_surrogate_set_weights.argtypes = [vp, vp]
        L.srw_surrogate_get_weights.argtypes = [vp, vp]
        L.srw_surrogate_forward.argtypes = [vp, vp, ip, vp]
        L.srw_surrogate_gradients.argtypes = [vp, vp, vp, ip, vp, ctypes.POINTER(ctypes.c_double)]
        L.srw_surrogate_train_step.argtypes = [vp, vp, vp, ip, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
        L.srw_surrogate_fit.argtypes = [vp, vp, ctypes.c_longlong, ctypes.POINTER(_FitOpts), vp]
        L.srw_surrogate_loglik.argtypes = [vp, vp, ip, vp, ip, vp]
        L.srw_surrogate_scan.argtypes = [vp, ctypes.POINTER(_ScanOpts), ctypes.POINTER(_ScanResult)]
        L.srw_surrogate_scan_chunked.argtypes = [vp, ctypes.POINTER(_ScanOpts), ctypes.c_longlong, ctypes.c_char_p, ip,
                                                 ctypes.POINTER(_ScanResult), ctypes.POINTER(ctypes.c_int)]
        L.srw_surrogate_save.argtypes = [vp, ctypes.c_char_p]
        L.srw_surrogate_load.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong)]
        L.srw_surrogate_fit_resume.argtypes = [vp, vp, ctypes.c_longlong, ctypes.POINTER(_FitOpts), ip, ip,
                                               ctypes.c_char_p, vp]
        L.srw_surrogate_scan_exact.argtypes = [vp, ctypes.c_longlong, ctypes.c_longlong, ip,
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                               ctypes.POINTER(ctypes.c_float)]
        L.srw_surrogate_sobol.argtypes = [vp, ctypes.c_longlong, ip, vp]
        L.srw_surrogate_get_standardization.argtypes = [vp, vp, vp]
        L.srw_diag_wait_timeout.argtypes = [ctypes.c_uint]
        L.srw_fault_inject.argtypes = [ip, ctypes.c_longlong]
        L.srw_fold_config.argtypes = [ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]
        L.srw_set_fold_config.argtypes = [vp, ip, ip]
        L.srw_get_fold_config.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.srw_check.argtypes = [vp, vp]
        L.srw_fault_pending.argtypes = [ctypes.POINTER(ctypes.c_int)]
        L.srw_fault_parse.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]
        L.srw_loglik_linear.argtypes = [vp, vp, ip, vp, vp, ip, vp]
        L.srw_loglik_profiled.argtypes = [vp, vp, ip, ctypes.c_double, vp, vp, ip, vp]
        L.srw_surrogate_last_error.argtypes = [vp]
        L.srw_surrogate_last_error.restype = ctypes.c_char_p
        L.srw_surrogate_destroy.argtypes = [vp]
        for name in EXPORTS:
            if name not in ("srw_last_error", "srw_status_string", "srw_noalloc_last_error", "srw_group_last_error",
                            "srw_surrogate_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status, h):
    if status != SRW_OK:
        raise SrwError(status, lib().srw_last_error(h).decode(errors="replace"))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _is_device(x):
    return hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# The library takes every size from its integer arguments and the handle, so
# the buffers behind the pointers are checked here, before any call.
def _device_args(named):
    """Each (name, tensor, dtype, minimum number of values) must be a
    contiguous CUDA tensor of that dtype holding at least that many values,
    all on one device; ValueError otherwise."""
    devices = set()
    for name, t, dtype, n_min in named:
        if not _is_device(t):
            raise ValueError("%s must be a CUDA tensor" % name)
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if str(t.dtype) != "torch." + dtype:
            raise ValueError("%s must be %s, got %s" % (name, dtype, str(t.dtype).replace("torch.", "")))
        if t.numel() < n_min:
            raise ValueError("%s holds %d values, the call needs %d" % (name, t.numel(), n_min))
        devices.add(t.device)
    if len(devices) > 1:
        raise ValueError("all tensors must be on one device")


def _device_points(theta):
    """Number of points in a device theta (float32, 5 values a point)."""
    _device_args([("theta", theta, "float32", 0)])
    if theta.numel() % 5 != 0:
        raise ValueError("theta must hold 5 values a point, got %d values" % theta.numel())
    return theta.numel() // 5


def _device_out(out, like, n, dtype):
    """`out`, or a new tensor of n values on `like`'s device."""
    if out is None:
        import torch
        out = torch.empty(n, dtype=getattr(torch, dtype), device=like.device)
    return out


def _host_out(out, n, dtype, name="out"):
    """`out` (a writeable C-contiguous numpy array of `dtype` holding at least
    n values), or a new one; ValueError otherwise."""
    if out is None:
        return np.empty(n, dtype=dtype)
    if not isinstance(out, np.ndarray) or out.dtype != np.dtype(dtype):
        raise ValueError("%s must be a numpy %s array" % (name, dtype))
    if not (out.flags.c_contiguous and out.flags.writeable):
        raise ValueError("%s must be writeable and contiguous" % name)
    if out.size < int(np.prod(n)):
        raise ValueError("%s holds %d values, the call needs %d" % (name, out.size, int(np.prod(n))))
    return out


def _need(cond, msg, *args):
    if not cond:
        raise ValueError(msg % args)


def _spectrum_len(h, stage):
    if int(stage) not in (0, 1, 2, 3):
        raise ValueError("stage must be 0, 1, 2 or 3, got %r" % (stage,))
    info = srw_info(h)
    return info["n_t"] if int(stage) <= 1 else info["n_rec"]


# ------------------------------------------------------------------ entry points
def _sources(sources, keep):
    srcs = (_Source * len(sources))()
    for k, s in enumerate(sources):
        e = np.ascontiguousarray(s["e"], dtype=np.float64).reshape(-1)
        w = np.ascontiguousarray(s["w"], dtype=np.float64).reshape(-1)
        p = np.ascontiguousarray(s["pee"], dtype=np.float64).reshape(-1)
        _need(e.size >= 1 and w.size == e.size and p.size == e.size,
              "source %d: e, w and pee must hold the same number (>= 1) of nodes, got %d, %d, %d", k, e.size, w.size,
              p.size)
        keep += [e, w, p]
        srcs[k] = _Source(e.size, _dptr(e), _dptr(w), _dptr(p))
    return srcs


def srw_create(t_edges, n_rec, sources, R, exposure, t_min=1e-3, midpoint=False, sin2w=0.23121, f_tau=0.5,
               e_true_sm=None):
    """Create a context (see srw_create in include/srw.h).  Returns the handle."""
    t_edges = np.ascontiguousarray(t_edges, dtype=np.float64).reshape(-1)
    R = np.ascontiguousarray(R, dtype=np.float32)
    n_t = t_edges.size - 1
    _need(n_t >= 1, "t_edges must hold n_t + 1 >= 2 edges")
    _need(R.shape == (int(n_rec), n_t), "R must be n_rec x n_t = %d x %d, got %s", int(n_rec), n_t, R.shape)
    _need(e_true_sm is None or np.size(e_true_sm) == n_t, "e_true_sm must hold n_t = %d values", n_t)
    L = lib()
    keep = [t_edges, R]
    srcs = _sources(sources, keep)
    b = _Binning(t_edges.size - 1, _dptr(t_edges), int(n_rec), float(t_min), 1 if midpoint else 0)
    esm = None
    if e_true_sm is not None:
        esm = np.ascontiguousarray(e_true_sm, dtype=np.float64)
        keep.append(esm)
    o = _Options(float(sin2w), float(f_tau), float(exposure), _dptr(esm) if esm is not None else None)
    h = ctypes.c_void_p()
    st = L.srw_create(ctypes.byref(b), srcs, len(sources), R.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o),
                      ctypes.byref(h))
    _check(st, None)
    return h


def srw_create_joint(t_edges, components, hist, exposure, mask=None, scale=None, live=None, events=None, t_min=1e-3,
                     midpoint=False, sin2w=0.23121, f_tau=0.5):
    """Create a context with one joint response per component (see
    srw_create_joint in include/srw.h): hist[k] is component k's [n_rec, n_t]
    Monte Carlo histogram, mask[k] its live-time correction (or None)."""
    L = lib()
    t_edges = np.ascontiguousarray(t_edges, dtype=np.float64).reshape(-1)
    keep = [t_edges]
    srcs = _sources(components, keep)
    n_src = len(components)
    hs = [np.ascontiguousarray(x, dtype=np.float64) for x in hist]
    if len(hs) != n_src:
        raise ValueError("one histogram per component")
    n_t = t_edges.size - 1
    _need(n_t >= 1 and hs[0].ndim == 2, "t_edges must hold n_t + 1 >= 2 edges and hist[0] be 2-D")
    n_rec = hs[0].shape[0]
    for k, x in enumerate(hs):
        _need(x.shape == (n_rec, n_t), "hist[%d] must be n_rec x n_t = %d x %d, got %s", k, n_rec, n_t, x.shape)
    if mask is not None:
        _need(len(mask) == n_src, "one live-time correction (or None) per component")
        for k, m in enumerate(mask):
            _need(m is None or np.size(m) == n_rec, "mask[%d] must hold n_rec = %d values", k, n_rec)
    for name, a, n in (("scale", scale, n_src), ("events", events, n_src), ("live", live, n_rec)):
        _need(a is None or np.size(a) == n, "%s must hold %d values", name, n)
    keep += hs
    dpp = ctypes.POINTER(ctypes.c_double)
    harr = (dpp * n_src)(*[_dptr(x) for x in hs])
    marr = None
    if mask is not None:
        ms = [None if m is None else np.ascontiguousarray(m, dtype=np.float64) for m in mask]
        keep += [m for m in ms if m is not None]
        marr = (dpp * n_src)(*[None if m is None else _dptr(m) for m in ms])

    def opt(a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return _dptr(a)
    jr = _JointResponse(harr, marr, opt(scale), opt(live), opt(events))
    b = _Binning(t_edges.size - 1, _dptr(t_edges), int(n_rec), float(t_min), 1 if midpoint else 0)
    o = _Options(float(sin2w), float(f_tau), float(exposure), None)
    h = ctypes.c_void_p()
    st = L.srw_create_joint(ctypes.byref(b), srcs, n_src, ctypes.byref(jr), ctypes.byref(o), ctypes.byref(h))
    _check(st, None)
    return h


def srw_joint_layout(h):
    """(component, true bin) of every column of the fold axis, as two int arrays."""
    n = ctypes.c_int()
    _check(lib().srw_joint_layout(h, ctypes.byref(n), None, None), h)
    src = np.empty(n.value, dtype=np.int32)
    b = np.empty(n.value, dtype=np.int32)
    _check(lib().srw_joint_layout(h, ctypes.byref(n), src.ctypes.data_as(ctypes.c_void_p),
                                  b.ctypes.data_as(ctypes.c_void_p)), h)
    return src, b


def srw_set_data(h, counts, bkg=None, mask=None):
    n_rec = srw_info(h)["n_rec"]
    counts = np.ascontiguousarray(counts, dtype=np.float64).reshape(-1)
    _need(counts.size == n_rec, "counts must hold n_rec = %d values, got %d", n_rec, counts.size)
    n_bkg = 0
    bptr = None
    if bkg is not None:
        bkg = np.ascontiguousarray(np.atleast_2d(bkg), dtype=np.float64)
        _need(bkg.ndim == 2 and bkg.shape[1] == n_rec, "bkg must be n_bkg x n_rec (n_rec = %d), got %s", n_rec,
              bkg.shape)
        n_bkg = bkg.shape[0]
        bptr = _dptr(bkg)
    mptr = None
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        _need(mask.size == n_rec, "mask must hold n_rec = %d values, got %d", n_rec, mask.size)
        mptr = mask.ctypes.data_as(ctypes.c_void_p)
    _check(lib().srw_set_data(h, _dptr(counts), bptr, n_bkg, mptr), h)


def srw_spectrum(h, theta, stage, out=None, stream=None):
    """Spectrum stage 0..3 at one point.  Host theta -> numpy result; device
    theta (CUDA tensor) -> result written into ``out`` (CUDA float32 tensor,
    allocated when None)."""
    n = _spectrum_len(h, stage)
    if _is_device(theta):
        _device_args([("theta", theta, "float32", 5)])
        out = _device_out(out, theta, n, "float32")
        _device_args([("theta", theta, "float32", 5), ("out", out, "float32", n)])
        _check(lib().srw_spectrum(h, ctypes.c_void_p(theta.data_ptr()), int(stage), ctypes.c_void_p(out.data_ptr()),
                                  SRW_DEVICE, _stream(stream)), h)
        return out
    th = np.ascontiguousarray(theta, dtype=np.float32).reshape(5)
    res = _host_out(out, n, np.float32)
    _check(lib().srw_spectrum(h, th.ctypes.data_as(ctypes.c_void_p), int(stage), res.ctypes.data_as(ctypes.c_void_p),
                              SRW_HOST, None), h)
    return res


def _loglik(fn, h, theta, precision, out, stream, extra_prec=True):
    if _is_device(theta):
        P = _device_points(theta)
        out = _device_out(out, theta, P, "float64")
        _device_args([("theta", theta, "float32", 5 * P), ("out", out, "float64", P)])
        args = [h, ctypes.c_void_p(theta.data_ptr()), P, ctypes.c_void_p(out.data_ptr()), SRW_DEVICE]
        if extra_prec:
            args.append(int(precision))
        args.append(_stream(stream))
        _check(fn(*args), h)
        return out
    th = np.ascontiguousarray(theta, dtype=np.float32).reshape(-1, 5)
    P = th.shape[0]
    res = _host_out(out, P, np.float64)
    args = [h, th.ctypes.data_as(ctypes.c_void_p), P, res.ctypes.data_as(ctypes.c_void_p), SRW_HOST]
    if extra_prec:
        args.append(int(precision))
    args.append(None)
    st = fn(*args)
    if st == SRW_EDOMAIN:
        return res  # +inf marks the points outside the domain
    _check(st, h)
    return res


def srw_loglik(h, theta, precision=SRW_FP32, out=None, stream=None):
    """-2 ln L for P points (theta: P x 5 float32)."""
    return _loglik(lib().srw_loglik, h, theta, precision, out, stream)


def srw_loglik_points(h, theta, out=None, stream=None):
    """The plain single-point path applied to each point in turn."""
    return _loglik(lib().srw_loglik_points, h, theta, None, out, stream, extra_prec=False)


def srw_loglik_linear(h, theta, out=None, grad=False, grad_out=None, stream=None):
    """Exact rank-8 evaluation: -2 ln L for P points (and, with grad=True or a
    grad_out, the gradient [P, 5]).  Host theta -> numpy results; CUDA tensors
    -> written into out (and grad_out), allocated when None."""
    if _is_device(theta):
        P = _device_points(theta)
        out = _device_out(out, theta, P, "float64")
        if grad and grad_out is None:
            grad_out = _device_out(None, theta, 5 * P, "float64").view(P, 5)
        named = [("theta", theta, "float32", 5 * P), ("out", out, "float64", P)]
        if grad_out is not None:
            named.append(("grad_out", grad_out, "float64", 5 * P))
        _device_args(named)
        gp = ctypes.c_void_p(grad_out.data_ptr()) if grad_out is not None else None
        _check(lib().srw_loglik_linear(h, ctypes.c_void_p(theta.data_ptr()), P, ctypes.c_void_p(out.data_ptr()), gp,
                                       SRW_DEVICE, _stream(stream)), h)
        return (out, grad_out) if grad_out is not None else out
    th = np.ascontiguousarray(theta, dtype=np.float32).reshape(-1, 5)
    P = th.shape[0]
    res = _host_out(out, P, np.float64)
    grad = grad or grad_out is not None
    g = _host_out(grad_out, (P, 5), np.float64, "grad_out") if grad else None
    st = lib().srw_loglik_linear(h, th.ctypes.data_as(ctypes.c_void_p), P, res.ctypes.data_as(ctypes.c_void_p),
                                 g.ctypes.data_as(ctypes.c_void_p) if grad else None, SRW_HOST, None)
    if st != SRW_EDOMAIN:
        _check(st, h)
    return (res, g) if grad else res


def srw_loglik_profiled(h, theta, sigma_alpha=0.0):
    """-2 ln L with the signal normalisation profiled (host theta [P, 5]);
    returns (values, alpha-hat)."""
    th = np.ascontiguousarray(theta, dtype=np.float32).reshape(-1, 5)
    P = th.shape[0]
    res = np.empty(P, dtype=np.float64)
    a = np.empty(P, dtype=np.float64)
    st = lib().srw_loglik_profiled(h, th.ctypes.data_as(ctypes.c_void_p), P, float(sigma_alpha),
                                   res.ctypes.data_as(ctypes.c_void_p), a.ctypes.data_as(ctypes.c_void_p), SRW_HOST,
                                   None)
    if st != SRW_EDOMAIN:
        _check(st, h)
    return res, a


def srw_spectrum_batch(h, theta, precision=SRW_FP32, out=None, stream=None):
    """Folded signal spectra [P, n_rec] (float32) from the batched fold."""
    n_rec = srw_info(h)["n_rec"]
    if _is_device(theta):
        P = _device_points(theta)
        out = _device_out(out, theta, P * n_rec, "float32")
        if out.dim() == 1 and out.numel() == P * n_rec:
            out = out.view(P, n_rec)
        _device_args([("theta", theta, "float32", 5 * P), ("out", out, "float32", P * n_rec)])
        _check(lib().srw_spectrum_batch(h, ctypes.c_void_p(theta.data_ptr()), P, ctypes.c_void_p(out.data_ptr()),
                                        SRW_DEVICE, int(precision), _stream(stream)), h)
        return out
    th = np.ascontiguousarray(theta, dtype=np.float32).reshape(-1, 5)
    P = th.shape[0]
    res = _host_out(out, (P, n_rec), np.float32)
    _check(lib().srw_spectrum_batch(h, th.ctypes.data_as(ctypes.c_void_p), P, res.ctypes.data_as(ctypes.c_void_p),
                                    SRW_HOST, int(precision), None), h)
    return res


def srw_get_basis(h):
    info = srw_info(h)
    out = np.empty((8, info["n_t"]), dtype=np.float64)
    _check(lib().srw_get_basis(h, _dptr(out)), h)
    return out


def srw_autotune(h, P, precision, cache_path=None, stream=None):
    chosen = ctypes.c_int(-1)
    cp = cache_path.encode() if cache_path else None
    _check(lib().srw_autotune(h, int(P), int(precision), cp, _stream(stream) if stream is not None else None,
                              ctypes.byref(chosen)), h)
    return chosen.value


def srw_fold_config(index):
    """(tile, k_block, stages) of tensor-core fold configuration `index`; None past the last."""
    t, k, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    if lib().srw_fold_config(int(index), ctypes.byref(t), ctypes.byref(k), ctypes.byref(st)) != SRW_OK:
        return None
    return t.value, k.value, st.value


def srw_fold_configs():
    """All tensor-core fold configurations as (index, tile, k_block, stages)."""
    out, i = [], 0
    while True:
        c = srw_fold_config(i)
        if c is None:
            return out
        out.append((i,) + c)
        i += 1


def srw_get_fold_config(h, precision):
    """(configuration index in use, candidates timed by the last autotune)."""
    i, t = ctypes.c_int(), ctypes.c_int()
    _check(lib().srw_get_fold_config(h, int(precision), ctypes.byref(i), ctypes.byref(t)), h)
    return i.value, t.value


def srw_set_fold_config(h, precision, index):
    _check(lib().srw_set_fold_config(h, int(precision), int(index)), h)


def srw_gemv_work(h):
    """Bytes of R the single-point GEMV streams per call (its rows' nonzero bands)."""
    b = ctypes.c_longlong()
    _check(lib().srw_gemv_work(h, ctypes.byref(b)), h)
    return b.value


def srw_fold_work(h, precision, tile=0):
    """Fraction of the (rec tile, K block) pairs the batched fold executes
    (tile 0: the handle's configured rec-tile width)."""
    f = ctypes.c_double()
    _check(lib().srw_fold_work(h, int(precision), int(tile), ctypes.byref(f)), h)
    return f.value


def srw_info(h):
    i = _Info()
    _check(lib().srw_info(h, ctypes.byref(i)), h)
    return {"n_t": i.n_t, "n_rec": i.n_rec, "n_nodes": i.n_nodes, "k_pad": i.k_pad, "device": i.device,
            "sm_count": i.sm_count, "tensor_path": bool(i.tensor_path), "lambda": i.lambda_,
            "device_bytes": i.device_bytes}


def srw_set_reference(h, theta_ref):
    """Reference point of the folds (5 values), or None to fold directly."""
    if theta_ref is None:
        _check(lib().srw_set_reference(h, None), h)
        return
    t = np.ascontiguousarray(theta_ref, dtype=np.float32).reshape(5)
    _check(lib().srw_set_reference(h, t.ctypes.data_as(ctypes.c_void_p)), h)


def srw_profile(h, enable):
    _check(lib().srw_profile(h, 1 if enable else 0), h)


def srw_profile_read(h):
    """Device milliseconds of the fold launch of the last srw_loglik call."""
    ms = ctypes.c_float()
    _check(lib().srw_profile_read(h, ctypes.byref(ms)), h)
    return ms.value


def _check_noalloc_args(R, W, counts, out, bkg, mask):
    """Host-side checks of srw_loglik_point_noalloc's tensors (no device work)."""
    named = [("R", R, "float32"), ("W", W, "float32"), ("counts", counts, "float64"), ("out", out, "float64")]
    if bkg is not None:
        named.append(("bkg", bkg, "float64"))
    if mask is not None:
        named.append(("mask", mask, "uint8"))
    devices = set()
    for name, t, dtype in named:
        if not (hasattr(t, "data_ptr") and getattr(t, "is_cuda", False)):
            raise ValueError("%s must be a CUDA tensor" % name)
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if str(t.dtype) != "torch." + dtype:
            raise ValueError("%s must be %s, got %s" % (name, dtype, str(t.dtype).replace("torch.", "")))
        devices.add(t.device)
    if len(devices) != 1:
        raise ValueError("all tensors must be on one device")
    if R.dim() != 2:
        raise ValueError("R must be 2-D (n_rec, ld)")
    n_rec, ld = R.shape
    if W.numel() < ld:
        raise ValueError("W holds %d values, R's rows %d" % (W.numel(), ld))
    for name, t in (("counts", counts), ("bkg", bkg), ("mask", mask)):
        if t is not None and t.numel() != n_rec:
            raise ValueError("%s must hold n_rec = %d values, got %d" % (name, n_rec, t.numel()))
    if out.numel() < 1:
        raise ValueError("out must hold at least one value")


SRW_FAULT_NONE, SRW_FAULT_ALLOC, SRW_FAULT_LAUNCH, SRW_FAULT_TIMEOUT = 0, 1, 2, 3
FAULT_KINDS = {"none": SRW_FAULT_NONE, "alloc": SRW_FAULT_ALLOC, "launch": SRW_FAULT_LAUNCH,
               "timeout": SRW_FAULT_TIMEOUT}


def srw_fault_inject(kind, skip=0):
    """Arm a one-shot host-side fault ("alloc", "launch", "timeout" or "none"):
    it fires at the (skip+1)-th matching event and then disarms."""
    k = FAULT_KINDS[kind] if isinstance(kind, str) else int(kind)
    st = lib().srw_fault_inject(k, int(skip))
    if st != SRW_OK:
        raise SrwError(st, "bad fault kind or skip")


def srw_fault_pending():
    """The armed fault kind (0 when none is armed)."""
    k = ctypes.c_int()
    lib().srw_fault_pending(ctypes.byref(k))
    return k.value


def srw_fault_parse(spec):
    """(kind, skip) of an SRW_FAULT specification; SrwError if it is not one."""
    k, n = ctypes.c_int(), ctypes.c_longlong()
    st = lib().srw_fault_parse(spec.encode(), ctypes.byref(k), ctypes.byref(n))
    if st != SRW_OK:
        raise SrwError(st, "not a fault specification: %r" % spec)
    return k.value, n.value


def srw_loglik_point_noalloc(R, W, counts, out, bkg=None, mask=None, stream=None):
    """Allocation-free single-point -2 ln L: every argument a CUDA tensor.
    R: (n_rec, ld) float32 with ld a multiple of 64; W: (ld,) float32;
    counts, bkg: (n_rec,) float64; mask: (n_rec,) uint8 or None; out: (1,) float64.

    The library reads every size from n_rec and ld, so each tensor is checked
    here first (ValueError): CUDA, contiguous, one device, the dtypes above,
    and long enough for the reads the kernels make.  A timed-out device wait
    leaves NaN in out[0] (the call itself is asynchronous and returns first)."""
    _check_noalloc_args(R, W, counts, out, bkg, mask)
    n_rec, ld = R.shape
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    st = lib().srw_loglik_point_noalloc(ptr(R), int(n_rec), int(ld), ptr(W), ptr(counts), ptr(bkg), ptr(mask),
                                        ptr(out), _stream(stream))
    if st != SRW_OK:
        raise SrwError(st, lib().srw_noalloc_last_error().decode(errors="replace"))
    return out


def _gcheck(status, g):
    if status != SRW_OK:
        msg = (lib().srw_group_last_error(g) if g else lib().srw_status_string(status)).decode(errors="replace")
        raise SrwError(status, msg)


def srw_group_create(handles, P):
    """Group handles with P[g] points each (see srw_group_create in include/srw.h)."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    pv = np.ascontiguousarray(P, dtype=np.int32).reshape(-1)
    _need(pv.size == n, "one point count per handle: %d handles, %d counts", n, pv.size)
    g = ctypes.c_void_p()
    _gcheck(lib().srw_group_create(hs, n, pv.ctypes.data_as(ctypes.c_void_p), ctypes.byref(g)), None)
    return g


def srw_group_loglik(g, theta, precision=SRW_BF16X3, out=None, stream=None, n_points=None):
    """-2 ln L of all points of all configurations (theta: sum(P) x 5,
    concatenated).  The library reads sum(P) points: pass that as n_points
    (GroupedLikelihood does) to have theta's and out's lengths checked."""
    if _is_device(theta):
        P = _device_points(theta)
        if n_points is not None and P != n_points:
            raise ValueError("theta holds %d points, the group %d" % (P, n_points))
        out = _device_out(out, theta, P, "float64")
        _device_args([("theta", theta, "float32", 5 * P), ("out", out, "float64", P)])
        _gcheck(lib().srw_group_loglik(g, ctypes.c_void_p(theta.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       SRW_DEVICE, int(precision), _stream(stream)), g)
        return out
    th = np.ascontiguousarray(theta, dtype=np.float32).reshape(-1, 5)
    if n_points is not None and th.shape[0] != n_points:
        raise ValueError("theta holds %d points, the group %d" % (th.shape[0], n_points))
    res = _host_out(out, th.shape[0], np.float64)
    st = lib().srw_group_loglik(g, th.ctypes.data_as(ctypes.c_void_p), res.ctypes.data_as(ctypes.c_void_p),
                                SRW_HOST, int(precision), None)
    if st == SRW_EDOMAIN:
        return res
    _gcheck(st, g)
    return res


def srw_group_autotune(g, precision, stream=None):
    chosen = ctypes.c_int(-1)
    _gcheck(lib().srw_group_autotune(g, int(precision), _stream(stream) if stream is not None else None,
                                     ctypes.byref(chosen)), g)
    return chosen.value


def srw_group_set_schedule(g, precision, candidate):
    _gcheck(lib().srw_group_set_schedule(g, int(precision), int(candidate)), g)


def srw_group_schedule(g, precision, n_groups):
    bn_max, n_items, n_cta, cand = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    bn = (ctypes.c_int * n_groups)()
    _gcheck(lib().srw_group_schedule(g, int(precision), ctypes.byref(bn_max), bn, ctypes.byref(n_items),
                                     ctypes.byref(n_cta), ctypes.byref(cand)), g)
    return {"bn_max": bn_max.value, "bn": list(bn), "n_items": n_items.value, "n_cta": n_cta.value,
            "candidate": cand.value}


def srw_group_profile(g, enable):
    _gcheck(lib().srw_group_profile(g, 1 if enable else 0), g)


def srw_group_profile_read(g):
    ms = ctypes.c_float()
    _gcheck(lib().srw_group_profile_read(g, ctypes.byref(ms)), g)
    return ms.value


def srw_group_destroy(g):
    if g:
        lib().srw_group_destroy(g)


def _scheck(status, sg):
    if status != SRW_OK:
        msg = (lib().srw_surrogate_last_error(sg) if sg else lib().srw_status_string(status)).decode(errors="replace")
        raise SrwError(status, msg)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr_array(arrays):
    """ctypes array of 8 pointers to float32 host arrays (kept alive by the caller)."""
    return (ctypes.c_void_p * len(arrays))(*[a.ctypes.data for a in arrays])


_HIDDEN = 256  # the surrogate's hidden width (fixed by the library)


def _check_weights(params, n_out):
    """The four layers' (W, b) as the library reads them: W1 [256][5], W2 and
    W3 [256][256], W4 [n_out][256], each b as long as its W has rows."""
    _need(len(params) == 4, "four layers (W, b), got %d", len(params))
    shapes = [(_HIDDEN, 5), (_HIDDEN, _HIDDEN), (_HIDDEN, _HIDDEN), (n_out, _HIDDEN)]
    for k, ((W, b), want) in enumerate(zip(params, shapes)):
        _need(np.shape(W) == want, "layer %d: W must be %s, got %s", k + 1, want, np.shape(W))
        _need(np.size(b) == want[0], "layer %d: b must hold %d values, got %d", k + 1, want[0], np.size(b))


def srw_surrogate_create(h, centre, half_width, params):
    """params: [(W, b), ...] of the four layers (float32 host arrays)."""
    _check_weights(params, srw_info(h)["n_rec"])
    _need(np.size(centre) == 5 and np.size(half_width) == 5, "centre and half_width must hold 5 values each")
    flat = [_f32(x) for W, b in params for x in (W, b)]
    c, hw = _f32(centre), _f32(half_width)
    out = ctypes.c_void_p()
    _scheck(lib().srw_surrogate_create(h, c.ctypes.data, hw.ctypes.data, _ptr_array(flat), ctypes.byref(out)), None)
    return out


def srw_surrogate_set_weights(sg, params, n_out=None):
    """Replace the weights; with n_out (the handle's n_rec) their shapes are checked."""
    if n_out is not None:
        _check_weights(params, n_out)
    flat = [_f32(x) for W, b in params for x in (W, b)]
    _scheck(lib().srw_surrogate_set_weights(sg, _ptr_array(flat)), sg)


def _like(params):
    return [np.empty_like(_f32(x)) for W, b in params for x in (W, b)]


def _pairs(flat):
    return [(flat[2 * k], flat[2 * k + 1]) for k in range(len(flat) // 2)]


def srw_surrogate_get_weights(sg, shapes_like):
    flat = _like(shapes_like)
    _scheck(lib().srw_surrogate_get_weights(sg, _ptr_array(flat)), sg)
    return _pairs(flat)


def srw_surrogate_forward(sg, theta, n_out):
    th = _f32(theta).reshape(-1, 5)
    y = np.empty((th.shape[0], n_out), dtype=np.float32)
    _scheck(lib().srw_surrogate_forward(sg, th.ctypes.data, th.shape[0], y.ctypes.data), sg)
    return y


def srw_surrogate_gradients(sg, theta, targets, shapes_like):
    th = _f32(theta).reshape(-1, 5)
    t = _f32(targets)
    n_out = np.size(shapes_like[-1][1])
    _need(t.size == th.shape[0] * n_out, "targets must be P x n_out = %d x %d", th.shape[0], n_out)
    flat = _like(shapes_like)
    loss = ctypes.c_double()
    _scheck(lib().srw_surrogate_gradients(sg, th.ctypes.data, t.ctypes.data, th.shape[0], _ptr_array(flat),
                                          ctypes.byref(loss)), sg)
    return loss.value, _pairs(flat)


def srw_surrogate_train_step(sg, theta, targets, lr, n_out=None):
    th = _f32(theta).reshape(-1, 5)
    t = _f32(targets)
    _need(n_out is None or t.size == th.shape[0] * n_out, "targets must be P x n_out = %d x %s", th.shape[0], n_out)
    loss = ctypes.c_double()
    _scheck(lib().srw_surrogate_train_step(sg, th.ctypes.data, t.ctypes.data, th.shape[0], ctypes.c_float(lr),
                                           ctypes.byref(loss)), sg)
    return loss.value


def srw_surrogate_destroy(sg):
    if sg:
        lib().srw_surrogate_destroy(sg)


def srw_check(h, stream=None):
    """Device-side status of the handle's device-pointer calls (raises SrwError)."""
    _check(lib().srw_check(h, _stream(stream) if stream is not None else None), h)


def srw_last_error(h):
    return lib().srw_last_error(h).decode(errors="replace")


def srw_destroy(h):
    if h:
        lib().srw_destroy(h)


# ------------------------------------------------------------------ convenience
class Likelihood:
    """Owns one srw context built from a workload dict (see ``workloads``):
    a conditional response ``R`` (srw_create), or per-component Monte Carlo
    histograms ``hist`` (srw_create_joint)."""

    def __init__(self, wl, counts=None, midpoint=False, e_true_sm=None, mask=None):
        if "hist" in wl:
            self.handle = srw_create_joint(wl["t_edges"], wl["components"], wl["hist"], wl["exposure"],
                                           mask=wl.get("mc_mask"), scale=wl.get("scale"), live=wl.get("live"),
                                           events=wl.get("events"), t_min=wl["t_min"], midpoint=midpoint,
                                           sin2w=wl["sin2w"], f_tau=wl["f_tau"])
        else:
            self.handle = srw_create(wl["t_edges"], wl["R"].shape[0], wl["sources"], wl["R"], wl["exposure"],
                                     t_min=wl["t_min"], midpoint=midpoint, sin2w=wl["sin2w"], f_tau=wl["f_tau"],
                                     e_true_sm=e_true_sm)
        if counts is not None:
            try:
                srw_set_data(self.handle, counts, wl.get("bkg"), mask)
            except Exception:
                srw_destroy(self.handle)
                self.handle = None
                raise

    def spectrum(self, theta, stage, out=None, stream=None):
        return srw_spectrum(self.handle, theta, stage, out, stream)

    def loglik(self, theta, precision=SRW_FP32, out=None, stream=None):
        return srw_loglik(self.handle, theta, precision, out, stream)

    def spectrum_batch(self, theta, precision=SRW_FP32, out=None, stream=None):
        return srw_spectrum_batch(self.handle, theta, precision, out, stream)

    def loglik_linear(self, theta, out=None, grad=False, grad_out=None, stream=None):
        return srw_loglik_linear(self.handle, theta, out, grad, grad_out, stream)

    def loglik_profiled(self, theta, sigma_alpha=0.0):
        return srw_loglik_profiled(self.handle, theta, sigma_alpha)

    def loglik_points(self, theta, out=None, stream=None):
        return srw_loglik_points(self.handle, theta, out, stream)

    def check(self, stream=None):
        """Raise SrwError if a device-pointer call since the last check timed out
        (its affected values are NaN) or produced +inf."""
        srw_check(self.handle, stream)

    def set_fold_config(self, precision, index):
        srw_set_fold_config(self.handle, precision, index)

    def set_reference(self, theta_ref):
        srw_set_reference(self.handle, theta_ref)

    def basis(self):
        return srw_get_basis(self.handle)

    def layout(self):
        return srw_joint_layout(self.handle)

    def gemv_work(self):
        return srw_gemv_work(self.handle)

    def fold_work(self, precision, tile=0):
        return srw_fold_work(self.handle, precision, tile)

    def info(self):
        return srw_info(self.handle)

    def close(self):
        if self.handle:
            srw_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GroupedLikelihood:
    """Several configurations (``Likelihood`` objects) evaluated in one
    persistent launch; ``P[g]`` points for configuration g."""

    def __init__(self, likelihoods, P):
        self.members = list(likelihoods)  # the group does not own the handles; keep them alive
        self.P = [int(p) for p in P]
        self.handle = srw_group_create([lk.handle for lk in self.members], self.P)

    @property
    def offsets(self):
        return np.concatenate([[0], np.cumsum(self.P)]).astype(np.int64)

    def loglik(self, theta, precision=SRW_BF16X3, out=None, stream=None):
        return srw_group_loglik(self.handle, theta, precision, out, stream, n_points=sum(self.P))

    def autotune(self, precision, stream=None):
        return srw_group_autotune(self.handle, precision, stream)

    def set_schedule(self, precision, candidate):
        srw_group_set_schedule(self.handle, precision, candidate)

    def schedule(self, precision):
        return srw_group_schedule(self.handle, precision, len(self.members))

    def profile(self, enable):
        srw_group_profile(self.handle, enable)

    def profile_read(self):
        return srw_group_profile_read(self.handle)

    def close(self):
        if self.handle:
            srw_group_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """The learned surrogate of one likelihood context (``Likelihood``)."""

    def __init__(self, likelihood, params, centre, half_width):
        self.lk = likelihood  # the surrogate does not own the handle; keep it alive
        self.shapes = [(np.zeros_like(_f32(W)), np.zeros_like(_f32(b))) for W, b in params]
        self.n_out = self.shapes[-1][1].size
        self.handle = srw_surrogate_create(likelihood.handle, centre, half_width, params)

    def set_weights(self, params):
        srw_surrogate_set_weights(self.handle, params, self.n_out)

    def weights(self):
        return srw_surrogate_get_weights(self.handle, self.shapes)

    def forward(self, theta):
        return srw_surrogate_forward(self.handle, theta, self.n_out)

    def gradients(self, theta, targets):
        return srw_surrogate_gradients(self.handle, theta, targets, self.shapes)

    def train_step(self, theta, targets, lr):
        return srw_surrogate_train_step(self.handle, theta, targets, lr, self.n_out)

    def fit(self, theta, epochs, batch=8192, lr=1e-3, lr_final=1e-5, precision=None):
        """Train on the exact path's spectra at theta (host [n, 5]); returns the per-epoch losses."""
        th = _f32(theta).reshape(-1, 5)
        o = _FitOpts(int(batch), int(epochs), float(lr), float(lr_final),
                     int(SRW_FP16X3 if precision is None else precision))
        losses = np.zeros(max(1, int(epochs)), dtype=np.float32)
        _scheck(lib().srw_surrogate_fit(self.handle, th.ctypes.data, th.shape[0], ctypes.byref(o), losses.ctypes.data),
                self.handle)
        return losses[:int(epochs)]

    def save(self, path):
        """Checkpoint the whole training state (srw_surrogate_save)."""
        _scheck(lib().srw_surrogate_save(self.handle, os.fsencode(path)), self.handle)

    def load(self, path):
        """Restore a checkpoint; returns the completed epochs it records."""
        done = ctypes.c_longlong()
        _scheck(lib().srw_surrogate_load(self.handle, os.fsencode(path), ctypes.byref(done)), self.handle)
        return done.value

    def fit_resumable(self, theta, epochs, checkpoint, batch=8192, lr=1e-3, lr_final=1e-5, precision=None,
                      stop_after=None):
        """The fit of fit() with a checkpoint after every epoch: if `checkpoint`
        exists it is loaded and the fit continues after its last completed
        epoch.  stop_after (epochs of this call) ends the call early, as an
        interruption would.  Returns the losses of the epochs this call ran."""
        th = _f32(theta).reshape(-1, 5)
        first = self.load(checkpoint) if os.path.exists(checkpoint) else 0
        stop = int(epochs) if stop_after is None else min(int(epochs), first + int(stop_after))
        o = _FitOpts(int(batch), int(epochs), float(lr), float(lr_final),
                     int(SRW_FP16X3 if precision is None else precision))
        losses = np.zeros(max(1, int(epochs)), dtype=np.float32)
        if stop > first:
            _scheck(lib().srw_surrogate_fit_resume(self.handle, th.ctypes.data, th.shape[0], ctypes.byref(o), first,
                                                   stop, os.fsencode(checkpoint), losses.ctypes.data), self.handle)
        return losses[first:stop]

    def scan_chunked(self, n_points, state_path, chunk_points, first=0, keep_frac=0.01, check_theta=None, tol=0.05,
                     cells_per_dim=4, precision=None, rule=SRW_SCAN_FLAG_CELLS, margin_factor=2.0, max_new_chunks=0):
        """srw_surrogate_scan_chunked: returns (result dict, complete)."""
        chk = None if check_theta is None else _f32(check_theta).reshape(-1, 5)
        o = _ScanOpts(int(first), int(n_points), float(keep_frac), chk.ctypes.data if chk is not None else None,
                      0 if chk is None else chk.shape[0], float(tol), int(cells_per_dim),
                      int(SRW_FP16X3 if precision is None else precision), int(rule), float(margin_factor))
        r = _ScanResult()
        done = ctypes.c_int()
        _scheck(lib().srw_surrogate_scan_chunked(self.handle, ctypes.byref(o), int(chunk_points),
                                                 os.fsencode(state_path), int(max_new_chunks), ctypes.byref(r),
                                                 ctypes.byref(done)), self.handle)
        res = {name: (list(getattr(r, name)) if name == "best_theta" else getattr(r, name)) for name, _ in r._fields_}
        return res, bool(done.value)

    def loglik(self, theta, out=None, stream=None):
        """Surrogate -2 ln L (host theta -> numpy; CUDA tensors -> written into out)."""
        if _is_device(theta):
            P = _device_points(theta)
            out = _device_out(out, theta, P, "float64")
            _device_args([("theta", theta, "float32", 5 * P), ("out", out, "float64", P)])
            _scheck(lib().srw_surrogate_loglik(self.handle, ctypes.c_void_p(theta.data_ptr()), P,
                                               ctypes.c_void_p(out.data_ptr()), SRW_DEVICE, _stream(stream)),
                    self.handle)
            return out
        th = _f32(theta).reshape(-1, 5)
        res = _host_out(out, th.shape[0], np.float64)
        _scheck(lib().srw_surrogate_loglik(self.handle, th.ctypes.data, th.shape[0], res.ctypes.data, SRW_HOST, None),
                self.handle)
        return res

    def scan(self, n_points, first=0, keep_frac=0.01, check_theta=None, tol=0.05, cells_per_dim=4, precision=None,
             rule=SRW_SCAN_FLAG_CELLS, margin_factor=2.0):
        chk = None if check_theta is None else _f32(check_theta).reshape(-1, 5)
        o = _ScanOpts(int(first), int(n_points), float(keep_frac), chk.ctypes.data if chk is not None else None,
                      0 if chk is None else chk.shape[0], float(tol), int(cells_per_dim),
                      int(SRW_FP16X3 if precision is None else precision), int(rule), float(margin_factor))
        r = _ScanResult()
        _scheck(lib().srw_surrogate_scan(self.handle, ctypes.byref(o), ctypes.byref(r)), self.handle)
        return {name: (list(getattr(r, name)) if name == "best_theta" else getattr(r, name)) for name, _ in r._fields_}

    def scan_exact(self, n_points, first=0, precision=None):
        v, i, ms = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_float()
        _scheck(lib().srw_surrogate_scan_exact(self.handle, int(first), int(n_points),
                                               int(SRW_FP16X3 if precision is None else precision), ctypes.byref(v),
                                               ctypes.byref(i), ctypes.byref(ms)), self.handle)
        return {"best_value": v.value, "best_index": i.value, "ms": ms.value}

    def sobol(self, first, count):
        out = np.empty((int(count), 5), dtype=np.float32)
        _scheck(lib().srw_surrogate_sobol(self.handle, int(first), int(count), out.ctypes.data), self.handle)
        return out

    def standardization(self):
        m = np.empty(self.n_out, dtype=np.float32)
        sd = np.empty(self.n_out, dtype=np.float32)
        _scheck(lib().srw_surrogate_get_standardization(self.handle, m.ctypes.data, sd.ctypes.data), self.handle)
        return m, sd

    def close(self):
        if self.handle:
            srw_surrogate_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
