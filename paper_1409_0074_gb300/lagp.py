"""ctypes binding of the C ABI in include/lagp.h (liblagp_gb300.so).

Argument marshalling only: every step of local approximate GP prediction runs
in the CUDA kernels of the library.  PyTorch supplies device memory and
streams.  The binding refuses to run without the compiled library; there is no
CPU fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblagp_gb300.so")

LAGP_EXHAUSTIVE, LAGP_RAY, LAGP_RAY_FULL = 0, 1, 2
LAGP_FP64, LAGP_FP32_SCORE, LAGP_FP32_SCORE_TC = 0, 1, 2
LAGP_PROMOTE = 16
LAGP_PROMOTE_PIVOT = 3e-5
SEARCH = {"exhaustive": LAGP_EXHAUSTIVE, "ray": LAGP_RAY, "ray_full": LAGP_RAY_FULL}
# "_promote": the FP32 form re-solves its ill-conditioned locations in binary64
PRECISION = {"fp64": LAGP_FP64, "fp32": LAGP_FP32_SCORE, "fp32_tc": LAGP_FP32_SCORE_TC,
             "fp32_promote": LAGP_FP32_SCORE | LAGP_PROMOTE,
             "fp32_tc_promote": LAGP_FP32_SCORE_TC | LAGP_PROMOTE}
ERRORS = {-1: "invalid argument", -2: "workspace too small", -3: "CUDA error",
          -4: "device reported a failure"}
STATUS_BITS = {1: "timeout", 2: "kNN tie capacity", 4: "numeric (v <= 0)"}

LAGP_BUSY = 1

EXPORTED = ("laGP_workspace_bytes", "laGP_build_and_predict", "laGP_knn_workspace_bytes",
            "laGP_knn", "laGP_status", "laGP_host_workspace_bytes",
            "laGP_build_and_predict_host", "laGP_profile", "laGP_profile_read",
            "laGP_autotune", "laGP_tune_get", "laGP_tune_set", "laGP_plan_create",
            "laGP_plan_launch", "laGP_plan_destroy", "laGP_ctx_design_bytes",
            "laGP_ctx_request_bytes", "laGP_ctx_create", "laGP_ctx_submit", "laGP_ctx_poll",
            "laGP_ctx_wait", "laGP_ctx_capacity", "laGP_ctx_destroy", "laGP_mle_predict",
            "laGP_mle_workspace_bytes", "laGP_build_and_predict_mle", "laGP_promoted",
            "laGP_sep_mle_workspace_bytes", "laGP_sep_mle", "laGP_prescale")

_lib = None


class LagpError(RuntimeError):
    def __init__(self, fn, rc, status=0):
        bits = [v for k, v in STATUS_BITS.items() if status & k]
        super().__init__("%s failed: %s (%d)%s" % (fn, ERRORS.get(rc, "error"), rc,
                                                   (" status: " + ", ".join(bits)) if bits else ""))
        self.rc, self.status = rc, status


def load():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblagp_gb300.so is not built: run __graft_entry__.build() or "
                           "python paper_1409_0074_gb300/build.py")
    lib = C.CDLL(LIB_PATH)
    i64, i32, vp, sz, dbl = C.c_int64, C.c_int, C.c_void_p, C.c_size_t, C.c_double
    lib.laGP_workspace_bytes.restype = sz
    lib.laGP_workspace_bytes.argtypes = [i64, i32, i64, i32, i32, i32, i32, i32]
    lib.laGP_host_workspace_bytes.restype = sz
    lib.laGP_host_workspace_bytes.argtypes = [i64, i32, i64, i32, i32, i32, i32, i32]
    lib.laGP_knn_workspace_bytes.restype = sz
    lib.laGP_knn_workspace_bytes.argtypes = [i64, i32, i64, i32]
    full = [vp, vp, i64, i32, vp, i64, i32, i32, i32, dbl, dbl, i32, i32, i32, vp, vp, vp, vp,
            vp, vp, vp, vp, sz, vp]
    lib.laGP_build_and_predict.restype = i32
    lib.laGP_build_and_predict.argtypes = full
    lib.laGP_build_and_predict_host.restype = i32
    lib.laGP_build_and_predict_host.argtypes = full
    lib.laGP_knn.restype = i32
    lib.laGP_knn.argtypes = [vp, i64, i32, vp, i64, i32, vp, vp, sz, vp]
    lib.laGP_status.restype = i32
    lib.laGP_status.argtypes = [vp, vp, C.POINTER(C.c_uint)]
    lib.laGP_promoted.restype = i32
    lib.laGP_promoted.argtypes = [vp, vp, C.POINTER(C.c_int64)]
    lib.laGP_profile.restype = i32
    lib.laGP_profile.argtypes = [i32]
    lib.laGP_profile_read.restype = i32
    lib.laGP_profile_read.argtypes = [i32, C.c_char_p, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int32)]
    ip = C.POINTER(C.c_int)
    lib.laGP_autotune.restype = i32
    lib.laGP_autotune.argtypes = [vp, vp, i64, i32, vp, i64, i32, i32, i32, dbl, dbl, i32, i32,
                                  i32, vp, vp, vp, vp, vp, sz, vp, ip]
    lib.laGP_tune_get.restype = i32
    lib.laGP_tune_get.argtypes = [i32, i32, i32, i32, i32, i32, ip]
    lib.laGP_tune_set.restype = i32
    lib.laGP_tune_set.argtypes = [i32, i32, i32, i32, i32, i32, i32]
    lib.laGP_plan_create.restype = i32
    lib.laGP_plan_create.argtypes = full[:-1] + [C.POINTER(vp)]
    lib.laGP_plan_launch.restype = i32
    lib.laGP_plan_launch.argtypes = [vp, vp]
    lib.laGP_plan_destroy.restype = i32
    lib.laGP_plan_destroy.argtypes = [vp]
    lib.laGP_ctx_design_bytes.restype = sz
    lib.laGP_ctx_design_bytes.argtypes = [i64, i32]
    lib.laGP_ctx_request_bytes.restype = sz
    lib.laGP_ctx_request_bytes.argtypes = [i64, i32, i64, i32, i32, i32, i32, i32, i32]
    lib.laGP_ctx_create.restype = i32
    lib.laGP_ctx_create.argtypes = [vp, vp, i64, i32, dbl, dbl, i32, i32, i32, i32, i32, vp, sz,
                                    i32, C.POINTER(vp)]
    lib.laGP_ctx_submit.restype = i32
    lib.laGP_ctx_submit.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, C.POINTER(C.c_int64)]
    lib.laGP_ctx_poll.restype = i32
    lib.laGP_ctx_poll.argtypes = [vp, C.c_int64, ip]
    lib.laGP_ctx_wait.restype = i32
    lib.laGP_ctx_wait.argtypes = [vp, C.c_int64]
    lib.laGP_ctx_capacity.restype = i32
    lib.laGP_ctx_capacity.argtypes = [vp, C.POINTER(C.c_size_t), ip]
    lib.laGP_ctx_destroy.restype = i32
    lib.laGP_ctx_destroy.argtypes = [vp]
    lib.laGP_mle_workspace_bytes.restype = sz
    lib.laGP_mle_workspace_bytes.argtypes = [i64, i32, i64, i32, i32, i32, i32, i32]
    lib.laGP_build_and_predict_mle.restype = i32
    lib.laGP_build_and_predict_mle.argtypes = [vp, vp, i64, i32, vp, i64, i32, i32, i32, dbl,
                                               dbl, dbl, dbl, i32, i32, i32, i32, vp, vp, vp,
                                               vp, vp, sz, vp]
    lib.laGP_mle_predict.restype = i32
    lib.laGP_mle_predict.argtypes = [vp, vp, i64, i32, vp, i64, vp, i32, dbl, dbl, dbl, dbl,
                                     vp, vp, vp, vp, vp, vp]
    lib.laGP_sep_mle_workspace_bytes.restype = sz
    lib.laGP_sep_mle_workspace_bytes.argtypes = [i32, i32]
    lib.laGP_sep_mle.restype = i32
    lib.laGP_sep_mle.argtypes = [vp, vp, i64, i32, vp, i32, dbl, dbl, dbl, dbl, i32, vp, vp, vp,
                                 sz, vp]
    lib.laGP_prescale.restype = i32
    lib.laGP_prescale.argtypes = [vp, i64, i32, vp, vp, vp]
    _lib = lib
    return lib


def _ptr(t, dtype=None, n=None):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    if n is not None and t.numel() < n:
        raise ValueError("tensor too small: %d < %d" % (t.numel(), n))
    return t.data_ptr()


def _hptr(a, dtype, n=None):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous):
        raise ValueError("expected a C-contiguous numpy array of %s" % dtype)
    if n is not None and a.size < n:
        raise ValueError("array too small")
    return a.ctypes.data


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check(name, rc):
    if rc != 0:
        raise LagpError(name, rc)


def laGP_workspace_bytes(N, p, M, n, N_close, nrays, search, precision):
    return load().laGP_workspace_bytes(N, p, M, n, N_close, nrays, search, precision)


def laGP_host_workspace_bytes(N, p, M, n, N_close, nrays, search, precision):
    return load().laGP_host_workspace_bytes(N, p, M, n, N_close, nrays, search, precision)


def laGP_knn_workspace_bytes(N, p, M, N_close):
    return load().laGP_knn_workspace_bytes(N, p, M, N_close)


def laGP_build_and_predict(design, y, xref, n0, n, N_close, theta, g, search, nrays, precision,
                           mean, s2, workspace, n_loc=None, nclose_loc=None, selected=None,
                           tie_gap=None, nevals=None, stream=None):
    """Enqueue the whole path on `stream` (torch tensors on the GPU)."""
    import torch
    N, p = design.shape
    M = xref.shape[0]
    lib = load()
    rc = lib.laGP_build_and_predict(
        _ptr(design, torch.float64), _ptr(y, torch.float64, N), N, p, _ptr(xref, torch.float64),
        M, n0, n, N_close, float(theta), float(g), search, nrays, precision,
        _ptr(n_loc, torch.int32, M), _ptr(nclose_loc, torch.int32, M),
        _ptr(mean, torch.float64, M), _ptr(s2, torch.float64, M),
        _ptr(selected, torch.int32, M * n), _ptr(tie_gap, torch.float64, M * n),
        _ptr(nevals, torch.int32, M * n), _ptr(workspace), workspace.numel() * workspace.element_size(),
        _stream(stream))
    _check("laGP_build_and_predict", rc)


def laGP_knn(design, xref, N_close, cand, workspace, stream=None):
    import torch
    N, p = design.shape
    M = xref.shape[0]
    rc = load().laGP_knn(_ptr(design, torch.float64), N, p, _ptr(xref, torch.float64), M,
                         N_close, _ptr(cand, torch.int32, M * N_close), _ptr(workspace),
                         workspace.numel() * workspace.element_size(), _stream(stream))
    _check("laGP_knn", rc)


def laGP_mle_predict(design, y, xref, sel, theta0, g, tmin, tmax, theta_out, mean, s2,
                     status, iters=None, stream=None):
    """Local maximum-likelihood lengthscale on the designs `sel` [M][n] and the
    predictive equations at it (device tensors; asynchronous on `stream`)."""
    import torch
    N, p = design.shape
    M, n = sel.shape
    rc = load().laGP_mle_predict(_ptr(design, torch.float64), _ptr(y, torch.float64, N), N, p,
                                 _ptr(xref, torch.float64, M * p), M, _ptr(sel, torch.int32),
                                 n, float(theta0), float(g), float(tmin), float(tmax),
                                 _ptr(theta_out, torch.float64, M), _ptr(mean, torch.float64, M),
                                 _ptr(s2, torch.float64, M), _ptr(iters, torch.int32, M),
                                 _ptr(status, torch.int32, 1), _stream(stream))
    _check("laGP_mle_predict", rc)


def laGP_sep_mle_workspace_bytes(n_sub, p):
    return load().laGP_sep_mle_workspace_bytes(n_sub, p)


def laGP_sep_mle(design, y, subset, g, theta0, tmin, tmax, maxit, theta_out, workspace,
                 info=None, stream=None):
    """Separable global lengthscales on the design rows `subset` (blocks until
    the fit ends)."""
    import torch
    N, p = design.shape
    n = subset.shape[0]
    rc = load().laGP_sep_mle(_ptr(design, torch.float64), _ptr(y, torch.float64, N), N, p,
                             _ptr(subset, torch.int32, n), n, float(g), float(theta0),
                             float(tmin), float(tmax), int(maxit),
                             _ptr(theta_out, torch.float64, p), _ptr(info, torch.int32, 3),
                             _ptr(workspace), workspace.numel() * workspace.element_size(),
                             _stream(stream))
    _check("laGP_sep_mle", rc)


def laGP_prescale(X, theta, X_out, stream=None):
    import torch
    rows, p = X.shape
    _check("laGP_prescale", load().laGP_prescale(_ptr(X, torch.float64), rows, p,
                                                 _ptr(theta, torch.float64, p),
                                                 _ptr(X_out, torch.float64, rows * p),
                                                 _stream(stream)))


def sep_mle(design, y, subset, g, theta0, tmin, tmax, maxit=200, stream=None):
    """Convenience wrapper of laGP_sep_mle: returns (theta [p] CUDA tensor,
    (iterations, evaluations, status))."""
    import torch
    p = design.shape[1]
    wsb = laGP_sep_mle_workspace_bytes(subset.shape[0], p)
    if wsb == 0:
        raise LagpError("laGP_sep_mle_workspace_bytes", -1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=design.device)
    th = torch.empty(p, dtype=torch.float64, device=design.device)
    info = torch.zeros(3, dtype=torch.int32, device=design.device)
    laGP_sep_mle(design, y, subset, g, theta0, tmin, tmax, maxit, th, ws, info=info,
                 stream=stream)
    return th, tuple(int(v) for v in info.cpu())


def prescale(X, theta, stream=None):
    """X / sqrt(theta) as a new CUDA tensor."""
    import torch
    out = torch.empty_like(X)
    laGP_prescale(X, theta, out, stream=stream)
    return out


def mle_predict(design, y, xref, sel, theta0, g, tmin, tmax, stream=None):
    """Convenience wrapper: allocates the outputs, runs laGP_mle_predict and
    checks the device status.  Returns a dict of CUDA tensors (theta, mean, s2,
    iters)."""
    import torch
    M = xref.shape[0]
    dev = design.device
    out = dict(theta=torch.empty(M, dtype=torch.float64, device=dev),
               mean=torch.empty(M, dtype=torch.float64, device=dev),
               s2=torch.empty(M, dtype=torch.float64, device=dev),
               iters=torch.empty(M, dtype=torch.int32, device=dev))
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    laGP_mle_predict(design, y, xref, sel, theta0, g, tmin, tmax, out["theta"], out["mean"],
                     out["s2"], st, iters=out["iters"], stream=stream)
    stv = int(st.cpu()[0])
    if stv:
        raise LagpError("laGP_mle_predict (device)", -4, stv)
    return out


def laGP_mle_workspace_bytes(N, p, M, n, N_close, nrays, search, precision):
    return load().laGP_mle_workspace_bytes(N, p, M, n, N_close, nrays, search, precision)


def laGP_build_and_predict_mle(design, y, xref, n0, n, N_close, theta0, g, tmin, tmax, stages,
                               search, nrays, precision, theta_out, mean, s2, workspace,
                               selected=None, stream=None):
    """Enqueue designs coupled with local inference for theta (one or two
    stages) on `stream` (torch tensors on the GPU)."""
    import torch
    N, p = design.shape
    M = xref.shape[0]
    rc = load().laGP_build_and_predict_mle(
        _ptr(design, torch.float64), _ptr(y, torch.float64, N), N, p, _ptr(xref, torch.float64),
        M, n0, n, N_close, float(theta0), float(g), float(tmin), float(tmax), int(stages),
        search, nrays, precision, _ptr(theta_out, torch.float64, M),
        _ptr(mean, torch.float64, M), _ptr(s2, torch.float64, M),
        _ptr(selected, torch.int32, M * n), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(stream))
    _check("laGP_build_and_predict_mle", rc)


def predict_mle(design, y, xref, n0, n, N_close, theta0, g, tmin, tmax, stages=1,
                search="ray", nrays=0, precision="fp64", want_selected=False,
                want_promoted=False, stream=None):
    """Convenience wrapper of laGP_build_and_predict_mle: allocates outputs and
    workspace, checks the device status; returns a dict of CUDA tensors (and,
    with want_promoted, the int "promoted")."""
    import torch
    dev = design.device
    M = xref.shape[0]
    N, p = design.shape
    s, pr = SEARCH[search], PRECISION[precision]
    wsb = laGP_mle_workspace_bytes(N, p, M, n, N_close, nrays, s, pr)
    if wsb == 0:
        raise LagpError("laGP_mle_workspace_bytes", -1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    out = {k: torch.empty(M, dtype=torch.float64, device=dev) for k in ("theta", "mean", "s2")}
    if want_selected:
        out["selected"] = torch.empty((M, n), dtype=torch.int32, device=dev)
    laGP_build_and_predict_mle(design, y, xref, n0, n, N_close, theta0, g, tmin, tmax, stages,
                               s, nrays, pr, out["theta"], out["mean"], out["s2"], ws,
                               selected=out.get("selected"), stream=stream)
    rc, st = laGP_status(ws, stream)
    if rc != 0:
        raise LagpError("laGP_build_and_predict_mle (device)", rc, st)
    if want_promoted:
        out["promoted"] = laGP_promoted(ws, stream)
    return out


def laGP_status(workspace, stream=None):
    st = C.c_uint(0)
    rc = load().laGP_status(_ptr(workspace), _stream(stream), C.byref(st))
    return rc, st.value


def laGP_promoted(workspace, stream=None):
    """Locations the last call on this workspace re-solved in binary64."""
    cnt = C.c_int64(0)
    _check("laGP_promoted", load().laGP_promoted(_ptr(workspace), _stream(stream), C.byref(cnt)))
    return cnt.value


def laGP_profile(enable):
    _check("laGP_profile", load().laGP_profile(1 if enable else 0))


def laGP_profile_read(max_kernels=32):
    """{kernel name: (total ms, launches)} of the events recorded since laGP_profile(1)."""
    names = C.create_string_buffer(32 * max_kernels)
    ms = (C.c_double * max_kernels)()
    cnt = (C.c_int32 * max_kernels)()
    k = load().laGP_profile_read(max_kernels, names, ms, cnt)
    if k < 0:
        raise LagpError("laGP_profile_read", k)
    raw = names.raw
    out = {}
    for i in range(k):
        nm = raw[32 * i: 32 * i + 32].split(b"\0", 1)[0].decode()
        out[nm] = (ms[i], cnt[i])
    return out


def laGP_build_and_predict_host(design, y, xref, n0, n, N_close, theta, g, search, nrays,
                                precision, mean, s2, workspace, n_loc=None, nclose_loc=None,
                                selected=None, tie_gap=None, nevals=None, stream=None):
    """Host-buffer form (numpy arrays; pinned memory recommended)."""
    N, p = design.shape
    M = xref.shape[0]
    rc = load().laGP_build_and_predict_host(
        _hptr(design, np.float64), _hptr(y, np.float64, N), N, p, _hptr(xref, np.float64), M, n0,
        n, N_close, float(theta), float(g), search, nrays, precision,
        _hptr(n_loc, np.int32, M), _hptr(nclose_loc, np.int32, M), _hptr(mean, np.float64, M),
        _hptr(s2, np.float64, M), _hptr(selected, np.int32, M * n),
        _hptr(tie_gap, np.float64, M * n), _hptr(nevals, np.int32, M * n), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(stream))
    _check("laGP_build_and_predict_host", rc)


def predict(design, y, xref, n0, n, N_close, theta, g, search="ray", nrays=0, precision="fp32",
            n_loc=None, nclose_loc=None, want_trace=False, want_promoted=False, stream=None):
    """Convenience wrapper: allocates outputs and workspace with torch, enqueues
    the path, checks the device status.  Returns a dict of CUDA tensors (and,
    with want_promoted, the int "promoted": locations re-solved in binary64)."""
    import torch
    dev = design.device
    M = xref.shape[0]
    N, p = design.shape
    s, pr = SEARCH[search], PRECISION[precision]
    wsb = laGP_workspace_bytes(N, p, M, n, N_close, nrays, s, pr)
    if wsb == 0:
        raise LagpError("laGP_workspace_bytes", -1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    out = dict(mean=torch.empty(M, dtype=torch.float64, device=dev),
               s2=torch.empty(M, dtype=torch.float64, device=dev))
    if want_trace:
        out["selected"] = torch.empty((M, n), dtype=torch.int32, device=dev)
        out["tie_gap"] = torch.empty((M, n), dtype=torch.float64, device=dev)
        out["nevals"] = torch.empty((M, n), dtype=torch.int32, device=dev)
    laGP_build_and_predict(design, y, xref, n0, n, N_close, theta, g, s, nrays, pr, out["mean"],
                           out["s2"], ws, n_loc=n_loc, nclose_loc=nclose_loc,
                           selected=out.get("selected"), tie_gap=out.get("tie_gap"),
                           nevals=out.get("nevals"), stream=stream)
    rc, st = laGP_status(ws, stream)
    if rc != 0:
        raise LagpError("laGP_build_and_predict (device)", rc, st)
    if want_promoted:
        out["promoted"] = laGP_promoted(ws, stream)
    return out


def _args_common(design, y, xref, n0, n, N_close, theta, g, search, nrays, precision, n_loc,
                 nclose_loc):
    import torch
    N, p = design.shape
    M = xref.shape[0]
    return [_ptr(design, torch.float64), _ptr(y, torch.float64, N), N, p,
            _ptr(xref, torch.float64), M, n0, n, N_close, float(theta), float(g), search, nrays,
            precision, _ptr(n_loc, torch.int32, M), _ptr(nclose_loc, torch.int32, M)]


def laGP_autotune(design, y, xref, n0, n, N_close, theta, g, search, nrays, precision, mean, s2,
                  workspace, n_loc=None, nclose_loc=None, stream=None):
    """Times the launch choices on these locations; returns the stored choice code."""
    import torch
    M = xref.shape[0]
    choice = C.c_int(0)
    rc = load().laGP_autotune(*_args_common(design, y, xref, n0, n, N_close, theta, g, search,
                                            nrays, precision, n_loc, nclose_loc),
                              _ptr(mean, torch.float64, M), _ptr(s2, torch.float64, M),
                              _ptr(workspace), workspace.numel() * workspace.element_size(),
                              _stream(stream), C.byref(choice))
    _check("laGP_autotune", rc)
    return choice.value


def laGP_tune_get(p, n, N_close, nrays, search, uneven):
    choice = C.c_int(0)
    _check("laGP_tune_get", load().laGP_tune_get(p, n, N_close, nrays, search, int(uneven),
                                                 C.byref(choice)))
    return choice.value


def laGP_tune_set(p, n, N_close, nrays, search, uneven, choice):
    _check("laGP_tune_set", load().laGP_tune_set(p, n, N_close, nrays, search, int(uneven),
                                                 int(choice)))


class Plan:
    """A captured launch sequence (laGP_plan_create); keeps references to its
    tensors so that they outlive the plan."""

    def __init__(self, design, y, xref, n0, n, N_close, theta, g, search, nrays, precision, mean,
                 s2, workspace, n_loc=None, nclose_loc=None, selected=None, tie_gap=None,
                 nevals=None):
        import torch
        M = xref.shape[0]
        self._keep = (design, y, xref, mean, s2, workspace, n_loc, nclose_loc, selected, tie_gap,
                      nevals)
        h = C.c_void_p(0)
        rc = load().laGP_plan_create(
            *_args_common(design, y, xref, n0, n, N_close, theta, g, search, nrays, precision,
                          n_loc, nclose_loc),
            _ptr(mean, torch.float64, M), _ptr(s2, torch.float64, M),
            _ptr(selected, torch.int32, M * n), _ptr(tie_gap, torch.float64, M * n),
            _ptr(nevals, torch.int32, M * n), _ptr(workspace),
            workspace.numel() * workspace.element_size(), C.byref(h))
        _check("laGP_plan_create", rc)
        self._h = h

    def launch(self, stream=None):
        _check("laGP_plan_launch", load().laGP_plan_launch(self._h, _stream(stream)))

    def close(self):
        if self._h:
            load().laGP_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Serving context (laGP_ctx_*): device-resident design in a torch-allocated
    arena, requests admitted into in-flight slots by free arena space."""

    def __init__(self, design, y, theta, g, n0, N_close, search, nrays, precision, arena_bytes,
                 max_inflight=8):
        import torch
        N, p = design.shape
        self.N, self.p, self.N_close, self.nrays = N, p, N_close, nrays
        self.search, self.precision = search, precision
        self._arena = torch.empty(arena_bytes, dtype=torch.uint8, device=design.device)
        self._keep = (design, y)
        h = C.c_void_p(0)
        rc = load().laGP_ctx_create(_ptr(design, torch.float64), _ptr(y, torch.float64, N), N, p,
                                    float(theta), float(g), n0, N_close, search, nrays, precision,
                                    _ptr(self._arena), arena_bytes, max_inflight, C.byref(h))
        _check("laGP_ctx_create", rc)
        self._h = h

    def request_bytes(self, M, n, want_selected=False):
        return load().laGP_ctx_request_bytes(self.N, self.p, M, n, self.N_close, self.nrays,
                                             self.search, self.precision, int(want_selected))

    def submit(self, xref, n, mean, s2, n_loc=None, selected=None):
        """xref [M][p] float64, n_loc [M] int32 or None, outputs: numpy arrays
        (page-locked for asynchronous copies).  Returns a ticket, or None when
        the context is busy (LAGP_BUSY)."""
        M = xref.shape[0]
        t = C.c_int64(0)
        rc = load().laGP_ctx_submit(self._h, _hptr(xref, np.float64, M * self.p), M, n,
                                    _hptr(n_loc, np.int32, M), _hptr(mean, np.float64, M),
                                    _hptr(s2, np.float64, M), _hptr(selected, np.int32, M * n),
                                    C.byref(t))
        if rc == LAGP_BUSY:
            return None
        _check("laGP_ctx_submit", rc)
        return t.value

    def poll(self, ticket):
        """True once the request's outputs are in its host arrays (raises on a
        device-reported failure)."""
        done = C.c_int(0)
        rc = load().laGP_ctx_poll(self._h, ticket, C.byref(done))
        _check("laGP_ctx_poll", rc)
        return bool(done.value)

    def wait(self, ticket):
        _check("laGP_ctx_wait", load().laGP_ctx_wait(self._h, ticket))

    def capacity(self):
        free = C.c_size_t(0)
        slots = C.c_int(0)
        _check("laGP_ctx_capacity", load().laGP_ctx_capacity(self._h, C.byref(free),
                                                             C.byref(slots)))
        return free.value, slots.value

    def close(self):
        if self._h:
            load().laGP_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
