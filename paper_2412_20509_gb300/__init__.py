"""Python binding of ``libgmf.so``, the GB300 (sm_103a) library for block-wise
adaptive SGD on generalized matrix factorization models (arXiv 2412.20509).

Argument marshalling only: every step of the fit runs in the library's CUDA
kernels behind the C ABI declared in ``include/gmf.h``. PyTorch provides
device memory and streams. There is no CPU fallback: importing this package
without a built ``libgmf.so`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgmf.so")

GMF_OK, GMF_ERR_ARG, GMF_ERR_CUDA, GMF_ERR_OOM, GMF_ERR_TIMEOUT, GMF_ERR_NONFINITE, GMF_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
GMF_POISSON, GMF_NEGBIN, GMF_GAUSSIAN, GMF_BINOMIAL, GMF_GAMMA, GMF_INVGAUSS = 0, 1, 2, 3, 4, 5
GMF_Y_INT32, GMF_Y_UINT16, GMF_Y_FLOAT32 = 0, 1, 2
GMF_PREC_FP32, GMF_PREC_MIXED = 0, 1
GMF_ORTH_B1, GMF_ORTH_B2, GMF_ORTH_B3 = 1, 2, 3
GMF_FLAG_NO_CLUSTER, GMF_FLAG_PERSIST, GMF_FLAG_SIMT_DEVIANCE, GMF_FLAG_STAGED_UPLOAD = 1, 2, 4, 8
GMF_SWEEP_SEQUENTIAL, GMF_SWEEP_PERSISTENT = -1, -3
GMF_EPOCH_SEPARATE, GMF_EPOCH_CLUSTER, GMF_EPOCH_PERSISTENT = 0, 1, 2
EPOCH_MODES = {GMF_EPOCH_SEPARATE: "separate", GMF_EPOCH_CLUSTER: "cluster", GMF_EPOCH_PERSISTENT: "persistent"}

FAMILIES = {"poisson": GMF_POISSON, "negbin": GMF_NEGBIN, "gaussian": GMF_GAUSSIAN, "binomial": GMF_BINOMIAL,
            "gamma": GMF_GAMMA, "invgauss": GMF_INVGAUSS}
PRECISIONS = {"fp32": GMF_PREC_FP32, "mixed": GMF_PREC_MIXED}
ORTH = {"B1": GMF_ORTH_B1, "B2": GMF_ORTH_B2, "B3": GMF_ORTH_B3}

# Every function declared in include/gmf.h.
EXPORTS = ("gmf_config_default", "gmf_init", "gmf_update_y", "gmf_update_y_async", "gmf_num_sweeps",
           "gmf_launches_per_sweep", "gmf_epoch_mode", "gmf_strip_schedule", "gmf_count_buffers",
           "gmf_sgd_epoch", "gmf_sgd_sweeps",
           "gmf_deviance", "gmf_deviance_async", "gmf_get_params", "gmf_set_params", "gmf_get_ema", "gmf_set_ema",
           "gmf_orthogonalize", "gmf_project_cells", "gmf_trace", "gmf_trace_read", "gmf_deviance_noalloc",
           "gmf_set_wait_limit", "gmf_set_flow_lag", "gmf_sgd_sweep_blocks", "gmf_chunk_bytes", "gmf_chunk_state", "gmf_holdout",
           "gmf_loglik", "gmf_initialize", "gmf_fit_loadings", "gmf_set_gene_shapes", "gmf_get_gene_shapes", "gmf_gene_shape_moments",
           "gmf_gene_shape_ml",
           "gmf_sweep_init", "gmf_sweep_epoch", "gmf_sweep_set_group", "gmf_sweep_group", "gmf_sweep_autotune",
           "gmf_sweep_model", "gmf_sweep_free", "gmf_mlp_create",
           "gmf_mlp_set_params", "gmf_mlp_get_params", "gmf_mlp_get_grads", "gmf_mlp_forward", "gmf_mlp_loss_grad",
           "gmf_mlp_adam", "gmf_mlp_set_precision", "gmf_mlp_train", "gmf_mlp_free", "gmf_free", "gmf_last_error",
           "gmf_version")


class GmfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class gmf_config(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("p", C.c_int32), ("q", C.c_int32), ("d", C.c_int32),
                ("family", C.c_int32), ("nb_row", C.c_int32), ("nb_col", C.c_int32), ("bias_corr", C.c_int32),
                ("alpha_mode", C.c_int32), ("precision", C.c_int32), ("flags", C.c_int32), ("missing", C.c_int32),
                ("lambda_", C.c_double * 4), ("a1", C.c_double), ("a2", C.c_double), ("k0", C.c_double),
                ("k1", C.c_double), ("tau", C.c_double), ("damping", C.c_double), ("eps", C.c_double),
                ("eta_clamp", C.c_double)]


_lib = None
VP = C.c_void_p


def lib():
    """Load libgmf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgmf.so not found at {LIB_PATH}; build it with __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    sig = {
        "gmf_config_default": (None, [C.POINTER(gmf_config), C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                      C.c_int32, C.c_int32, C.c_int32]),
        "gmf_init": (C.c_int, [C.POINTER(VP), C.POINTER(gmf_config), VP, C.c_int32, C.c_int32, VP, VP, VP, VP, VP, VP,
                               VP, VP, VP, VP, C.c_double, VP]),
        "gmf_update_y": (C.c_int, [VP, VP, C.c_int32, VP]),
        "gmf_update_y_async": (C.c_int, [VP, VP, VP]),
        "gmf_num_sweeps": (C.c_int32, [VP]),
        "gmf_launches_per_sweep": (C.c_int32, [VP]),
        "gmf_epoch_mode": (C.c_int32, [VP]),
        "gmf_count_buffers": (C.c_int32, [VP]),
        "gmf_strip_schedule": (C.c_int, [C.c_int32, C.c_int32, VP, C.c_int32, C.c_int32, VP]),
        "gmf_sgd_epoch": (C.c_int, [VP, VP, VP]),
        "gmf_sgd_sweeps": (C.c_int, [VP, VP, C.c_int32, C.c_int32, VP]),
        "gmf_deviance": (C.c_int, [VP, C.POINTER(C.c_double), VP]),
        "gmf_deviance_async": (C.c_int, [VP, VP, VP]),
        "gmf_holdout": (C.c_int, [VP, VP, VP, VP]),
        "gmf_loglik": (C.c_int, [VP, VP, VP]),
        "gmf_initialize": (C.c_int, [VP, C.c_int32, C.c_uint64, VP, VP]),
        "gmf_fit_loadings": (C.c_int, [VP, C.c_int32, VP, VP]),
        "gmf_set_gene_shapes": (C.c_int, [VP, VP, VP]),
        "gmf_get_gene_shapes": (C.c_int, [VP, VP, VP]),
        "gmf_gene_shape_moments": (C.c_int, [VP, C.c_double, C.c_double, VP, VP]),
        "gmf_gene_shape_ml": (C.c_int, [VP, VP, C.c_int32, C.c_double, C.c_double, C.c_double, VP,
                                        C.POINTER(C.c_int32), VP]),
        "gmf_get_params": (C.c_int, [VP, VP, VP, VP, VP, VP, VP]),
        "gmf_set_params": (C.c_int, [VP, VP, VP, VP, VP, VP, VP]),
        "gmf_get_ema": (C.c_int, [VP, VP, VP, VP, VP, VP, VP, VP, VP]),
        "gmf_set_ema": (C.c_int, [VP, VP, VP, VP, VP, VP, VP, VP, VP]),
        "gmf_orthogonalize": (C.c_int, [VP, C.c_int32, VP]),
        "gmf_project_cells": (C.c_int, [VP, VP, C.c_int32, C.c_int64, VP, VP, VP, C.c_int32, VP, VP, VP, VP]),
        "gmf_set_wait_limit": (C.c_int, [VP, C.c_int64, C.c_int32]),
        "gmf_set_flow_lag": (C.c_int, [VP, C.c_int32]),
        "gmf_sgd_sweep_blocks": (C.c_int, [VP, VP, C.c_int32, VP, C.c_int32, VP]),
        "gmf_chunk_bytes": (C.c_int64, [VP, C.c_int32, C.c_int32]),
        "gmf_chunk_state": (C.c_int, [VP, C.c_int32, C.c_int32, VP, C.c_int32, VP]),
        "gmf_trace": (C.c_int, [VP, C.c_int32]),
        "gmf_trace_read": (C.c_int, [VP, C.POINTER(C.c_double), C.POINTER(C.c_int64), VP]),
        "gmf_deviance_noalloc": (C.c_int, [VP, C.c_int32, VP, C.c_int64, C.c_int64, VP, VP, C.c_int32, C.c_int32,
                                          C.c_int32, C.c_float, C.c_float, VP, VP]),
        "gmf_sweep_init": (C.c_int, [C.POINTER(VP), C.POINTER(gmf_config), VP, C.c_int32, VP, C.c_int32, C.c_int32, VP,
                                     VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP]),
        "gmf_sweep_epoch": (C.c_int, [VP, VP, VP]),
        "gmf_sweep_set_group": (C.c_int, [VP, C.c_int32]),
        "gmf_sweep_group": (C.c_int32, [VP]),
        "gmf_sweep_autotune": (C.c_int, [VP, VP, C.c_int32, VP, VP, VP]),
        "gmf_sweep_model": (VP, [VP, C.c_int32]),
        "gmf_sweep_free": (None, [VP]),
        "gmf_mlp_create": (C.c_int, [C.POINTER(VP), C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, VP]),
        "gmf_mlp_set_params": (C.c_int, [VP] * 8),
        "gmf_mlp_get_params": (C.c_int, [VP] * 8),
        "gmf_mlp_get_grads": (C.c_int, [VP] * 8),
        "gmf_mlp_forward": (C.c_int, [VP, VP, C.c_int32, C.c_int64, VP, VP]),
        "gmf_mlp_loss_grad": (C.c_int, [VP, VP, C.c_int32, C.c_int64, VP, VP, VP]),
        "gmf_mlp_adam": (C.c_int, [VP, C.c_float, C.c_float, C.c_float, C.c_float, VP]),
        "gmf_mlp_set_precision": (C.c_int, [VP, C.c_int32, VP]),
        "gmf_mlp_train": (C.c_int, [VP, VP, C.c_int32, C.c_int64, VP, C.c_int32, C.c_int32, C.c_float, C.c_uint64, VP,
                                    VP]),
        "gmf_mlp_free": (None, [VP]),
        "gmf_free": (None, [VP]),
        "gmf_last_error": (C.c_char_p, []),
        "gmf_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(rc):
    if rc != GMF_OK:
        raise GmfError(rc, lib().gmf_last_error().decode())
    return rc


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _torch_ydt(Y):
    """Response type of a torch tensor: int32, 16-bit counts (uint16, or their int16 view), or float32."""
    import torch
    if Y.dtype == torch.int32:
        return GMF_Y_INT32
    if Y.dtype == torch.float32:
        return GMF_Y_FLOAT32
    if Y.dtype == torch.int16 or (hasattr(torch, "uint16") and Y.dtype == torch.uint16):
        return GMF_Y_UINT16
    raise TypeError("responses must be int32, 16-bit counts (uint16 / int16 view) or float32")


def strip_schedule(r, s, sigma, w_begin=0, w_end=None):
    """need[w - w_begin, k]: earlier visits (within [w_begin, w)) of the moving
    strip of block k of sweep w -- the dependency counts of a persistent sweep
    range (host computation, gmf_strip_schedule)."""
    sigma = np.ascontiguousarray(sigma, dtype=np.int32)
    w_end = len(sigma) if w_end is None else w_end
    out = np.zeros((max(w_end - w_begin, 0), min(r, s)), dtype=np.int32)
    check(lib().gmf_strip_schedule(int(r), int(s), sigma.ctypes.data, int(w_begin), int(w_end), out.ctypes.data))
    return out


def make_config(n, m, p, q, d, family, nb_row, nb_col, settings, precision="fp32", flags=0):
    cfg = gmf_config()
    lib().gmf_config_default(C.byref(cfg), n, m, p, q, d, FAMILIES[family], nb_row, nb_col)
    s = settings
    cfg.lambda_ = (C.c_double * 4)(*s["lambda_"])
    for k in ("a1", "a2", "k0", "k1", "tau", "damping", "eps", "eta_clamp"):
        setattr(cfg, k, float(s[k]))
    cfg.bias_corr = int(s["bias_corr"])
    cfg.alpha_mode = int(s["alpha_mode"])
    cfg.missing = int(s.get("missing", 0))
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.flags = int(flags)
    return cfg


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        a = a.reshape(shape)
    return a


class Model:
    """One GMF fit held on the GPU (a ``gmf_model`` handle)."""

    def __init__(self, Y, X, Z, offset, start, *, family, nb_row, nb_col, row_perm, col_perm, settings,
                 precision="fp32", W=None, stream=None, flags=0):
        import torch
        self._h = VP()
        on_dev = isinstance(Y, torch.Tensor) and Y.is_cuda
        if isinstance(Y, torch.Tensor):
            n, m = Y.shape
            ydt = _torch_ydt(Y)
            Y = Y.contiguous()
        else:
            Y = np.ascontiguousarray(Y)
            n, m = Y.shape
            ydt = {np.dtype(np.int32): GMF_Y_INT32, np.dtype(np.uint16): GMF_Y_UINT16,
                   np.dtype(np.float32): GMF_Y_FLOAT32}.get(Y.dtype)
            if ydt is None:
                raise TypeError("Y must be int32, uint16 or float32")
        X = np.ascontiguousarray(X, dtype=np.float64)
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        p, q = X.shape[1], Z.shape[1]
        d = np.asarray(start["U"]).shape[1]
        self.dims = (n, m, p, q, d)
        self.cfg = make_config(n, m, p, q, d, family, nb_row, nb_col, settings, precision, flags)
        off = None if offset is None else np.ascontiguousarray(offset, dtype=np.float64)
        B0 = _f64(start["B"], (m, p)); G0 = _f64(start["Gamma"], (n, q))
        U0 = _f64(start["U"], (n, d)); V0 = _f64(start["V"], (m, d))
        rp = np.ascontiguousarray(row_perm, dtype=np.int32)
        cp = np.ascontiguousarray(col_perm, dtype=np.int32)
        if W is not None:
            if on_dev:
                W = W.to(torch.float32).contiguous()
            else:
                W = np.ascontiguousarray(W, dtype=np.float32)
        self._keep = (Y, W)
        check(lib().gmf_init(C.byref(self._h), C.byref(self.cfg), _ptr(Y), ydt, int(on_dev), _ptr(W), _ptr(X), _ptr(Z),
                             _ptr(off), _ptr(rp), _ptr(cp), _ptr(B0), _ptr(G0), _ptr(U0), _ptr(V0),
                             float(start.get("alpha", 1.0)), _stream(stream)))
        self._keep = None
        self.y_dtype = ydt

    @classmethod
    def _borrow(cls, handle, dims, owner):
        """A view of a handle owned by someone else (e.g. one model of a Sweep)."""
        obj = cls.__new__(cls)
        obj._h = VP(handle)
        obj.dims = dims
        obj._owner = owner
        obj._borrowed = True
        return obj

    def __del__(self):
        h = getattr(self, "_h", None)
        if getattr(self, "_borrowed", False):
            return
        if h is not None and h.value and _lib is not None:
            _lib.gmf_free(h)
            self._h = VP()

    close = __del__

    @property
    def num_sweeps(self):
        return lib().gmf_num_sweeps(self._h)

    @property
    def launches_per_sweep(self):
        """Kernel launches per sweep: 1 in cluster mode, 2 with a separate update
        launch, 0 when a sweep range is one persistent launch."""
        return lib().gmf_launches_per_sweep(self._h)

    @property
    def epoch_mode(self):
        """'separate', 'cluster' or 'persistent' (how gmf_sgd_epoch launches)."""
        return EPOCH_MODES[lib().gmf_epoch_mode(self._h)]

    def epoch(self, sigma, stream=None):
        sigma = np.ascontiguousarray(sigma, dtype=np.int32)
        check(lib().gmf_sgd_epoch(self._h, sigma.ctypes.data, _stream(stream)))

    def sweeps(self, sigma, w_begin, w_end, stream=None):
        sigma = np.ascontiguousarray(sigma, dtype=np.int32)
        check(lib().gmf_sgd_sweeps(self._h, sigma.ctypes.data, int(w_begin), int(w_end), _stream(stream)))

    def update_y(self, Y, stream=None):
        import torch
        on_dev = isinstance(Y, torch.Tensor) and Y.is_cuda
        if not on_dev:
            Y = np.ascontiguousarray(Y) if not isinstance(Y, torch.Tensor) else Y.contiguous()
        check(lib().gmf_update_y(self._h, _ptr(Y), int(on_dev), _stream(stream)))

    def update_y_async(self, Y, stream=None):
        """Counts from a host tensor or array without waiting (see gmf_update_y_async: pinned memory is read
        directly by the GPU); keep Y unchanged until the stream has passed this call's work."""
        check(lib().gmf_update_y_async(self._h, _ptr(Y), _stream(stream)))

    @property
    def count_buffers(self):
        """Count buffers held on the device (2 once gmf_update_y_async took the direct path)."""
        return lib().gmf_count_buffers(self._h)

    def deviance(self, stream=None):
        out = C.c_double()
        check(lib().gmf_deviance(self._h, C.byref(out), _stream(stream)))
        return out.value

    def holdout(self, Ytrue, stream=None):
        """Out-of-sample error and relative Poisson deviance on the entries marked missing (gmf_holdout);
        Ytrue: CUDA tensor of the complete counts in the caller's order (int32, or 16-bit counts)."""
        out = (C.c_double * 4)()
        check(lib().gmf_holdout(self._h, Ytrue.data_ptr(), out, _stream(stream)))
        return {"error": out[0], "deviance": out[1], "ybar": out[2], "n_heldout": int(out[3])}

    def set_gene_shapes(self, alpha, stream=None):
        """Per-gene NB shapes (alpha_mode 2), the caller's gene order."""
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        check(lib().gmf_set_gene_shapes(self._h, a.ctypes.data, _stream(stream)))

    def get_gene_shapes(self, stream=None):
        out = np.empty(self.dims[1])
        check(lib().gmf_get_gene_shapes(self._h, out.ctypes.data, _stream(stream)))
        return out

    def gene_shape_moments(self, eps=1e-8, cap=1e6, stream=None):
        """App. B's moment estimator per gene at the current parameters (gmf_gene_shape_moments)."""
        out = np.empty(self.dims[1])
        check(lib().gmf_gene_shape_moments(self._h, float(eps), float(cap), out.ctypes.data, _stream(stream)))
        return out

    def gene_shape_ml(self, start=None, iters=30, tol=1e-6, lo=1e-3, hi=1e4, stream=None):
        """Maximum-likelihood NB shape per gene at the current means (gmf_gene_shape_ml); returns
        (shapes in the caller's gene order, Newton passes made)."""
        out = np.empty(self.dims[1])
        st = None if start is None else np.ascontiguousarray(start, dtype=np.float64)
        done = C.c_int32(0)
        check(lib().gmf_gene_shape_ml(self._h, None if st is None else st.ctypes.data, int(iters), float(tol),
                                      float(lo), float(hi), out.ctypes.data, C.byref(done), _stream(stream)))
        return out, int(done.value)

    def initialize(self, power_iters=2, seed=0, stream=None):
        """The least-squares start of Sec. 4.1 (gmf_initialize); returns the residual's d leading singular values."""
        d = self.dims[4]
        sv = np.zeros(max(d, 1))
        check(lib().gmf_initialize(self._h, int(power_iters), int(seed), sv.ctypes.data, _stream(stream)))
        return sv[:d]

    def fit_loadings(self, n_steps=8, stream=None):
        """Column GLMs for V given U, B and Gamma, the last step of Sec. 4.1 (gmf_fit_loadings); returns the summed
        objective 0.5 deviance + 0.5 lambda_V |V|^2 at the result."""
        out = C.c_double()
        check(lib().gmf_fit_loadings(self._h, int(n_steps), C.addressof(out), _stream(stream)))
        return out.value

    def loglik(self, stream=None):
        """Log-likelihood, Pearson statistic and observed-entry count at the current parameters (gmf_loglik)."""
        out = (C.c_double * 3)()
        check(lib().gmf_loglik(self._h, out, _stream(stream)))
        return {"loglik": out[0], "pearson": out[1], "n_obs": int(out[2])}

    def deviance_async(self, out, stream=None):
        """Write the FP64 deviance into a 1-element CUDA float64 tensor."""
        check(lib().gmf_deviance_async(self._h, out.data_ptr(), _stream(stream)))

    def get_params(self, stream=None):
        n, m, p, q, d = self.dims
        B, G, U, V = np.empty((m, p)), np.empty((n, q)), np.empty((n, d)), np.empty((m, d))
        a = C.c_double()
        check(lib().gmf_get_params(self._h, _ptr(B), _ptr(G), _ptr(U), _ptr(V), C.addressof(a), _stream(stream)))
        return dict(B=B, Gamma=G, U=U, V=V, alpha=a.value)

    def set_params(self, params, stream=None):
        n, m, p, q, d = self.dims
        arr = [None if params.get(k) is None else _f64(params[k], s)
               for k, s in (("B", (m, p)), ("Gamma", (n, q)), ("U", (n, d)), ("V", (m, d)))]
        a = None if params.get("alpha") is None else C.c_double(float(params["alpha"]))
        check(lib().gmf_set_params(self._h, *[_ptr(x) for x in arr], None if a is None else C.addressof(a),
                                   _stream(stream)))

    def get_ema(self, stream=None):
        n, m, p, q, d = self.dims
        out = dict(Gb_row=np.empty((n, q + d)), Hb_row=np.empty((n, q + d)), Gb_col=np.empty((m, p + d)),
                   Hb_col=np.empty((m, p + d)), cnt_row=np.empty(n, dtype=np.int64), cnt_col=np.empty(m, dtype=np.int64))
        t = C.c_int64()
        check(lib().gmf_get_ema(self._h, *[_ptr(out[k]) for k in ("Gb_row", "Hb_row", "Gb_col", "Hb_col", "cnt_row",
                                                                  "cnt_col")], C.addressof(t), _stream(stream)))
        out["t"] = t.value
        return out

    def set_ema(self, ema, stream=None):
        n, m, p, q, d = self.dims
        shapes = dict(Gb_row=(n, q + d), Hb_row=(n, q + d), Gb_col=(m, p + d), Hb_col=(m, p + d))
        arrs = [None if ema.get(k) is None else _f64(ema[k], s) for k, s in shapes.items()]
        cnts = [None if ema.get(k) is None else np.ascontiguousarray(ema[k], dtype=np.int64)
                for k in ("cnt_row", "cnt_col")]
        t = None if ema.get("t") is None else C.c_int64(int(ema["t"]))
        check(lib().gmf_set_ema(self._h, *[_ptr(x) for x in arrs], *[_ptr(x) for x in cnts],
                                None if t is None else C.addressof(t), _stream(stream)))

    def state_dict(self):
        """Complete checkpoint (parameters + optimiser state) as numpy arrays."""
        s = self.get_params()
        s.update(self.get_ema())
        return s

    def load_state_dict(self, s):
        self.set_params(s)
        self.set_ema(s)

    def sweep_blocks(self, sigma, w, blocks, stream=None):
        """Sweep w restricted to the listed blocks (gmf_sgd_sweep_blocks); t advances by the whole sweep."""
        sigma = np.ascontiguousarray(sigma, dtype=np.int32)
        b = np.ascontiguousarray(sorted(int(k) for k in blocks), dtype=np.int32)
        check(lib().gmf_sgd_sweep_blocks(self._h, sigma.ctypes.data, int(w), b.ctypes.data if len(b) else None,
                                         len(b), _stream(stream)))

    def chunk_floats(self, side, chunk):
        """Floats of the packed state of row chunk (side 0) or column chunk (side 1)."""
        nb = lib().gmf_chunk_bytes(self._h, int(side), int(chunk))
        if nb < 0:
            raise GmfError(GMF_ERR_ARG, f"chunk {chunk} of side {side} out of range")
        return nb // 4

    def get_chunk(self, side, chunk, out, stream=None):
        """Packed state of a chunk into a CUDA float32 tensor of chunk_floats() elements (asynchronous)."""
        check(lib().gmf_chunk_state(self._h, int(side), int(chunk), out.data_ptr(), 0, _stream(stream)))

    def set_chunk(self, side, chunk, buf, stream=None):
        """Packed state of a chunk from a CUDA float32 tensor (asynchronous)."""
        check(lib().gmf_chunk_state(self._h, int(side), int(chunk), buf.data_ptr(), 1, _stream(stream)))

    def set_wait_limit(self, limit_ns=0, need_extra=0):
        """Testing hook of the persistent epoch's bounded strip waits (gmf_set_wait_limit)."""
        check(lib().gmf_set_wait_limit(self._h, int(limit_ns), int(need_extra)))

    def set_flow_lag(self, lag):
        """Item order of the dataflow epoch: a block's updates trail its tiles by
        `lag` tile groups (gmf_set_flow_lag; bitwise the same results)."""
        check(lib().gmf_set_flow_lag(self._h, int(lag)))

    def trace(self, enable=True):
        """Time every block-step launch with CUDA events on its stream."""
        check(lib().gmf_trace(self._h, int(bool(enable))))

    def trace_read(self, stream=None):
        """(summed kernel milliseconds, launches) since the last read."""
        ms, n = C.c_double(), C.c_int64()
        check(lib().gmf_trace_read(self._h, C.byref(ms), C.byref(n), _stream(stream)))
        return ms.value, n.value

    def orthogonalize(self, mode="B1", stream=None):
        check(lib().gmf_orthogonalize(self._h, ORTH[mode] if isinstance(mode, str) else int(mode), _stream(stream)))

    def project_cells(self, Ynew, Xnew, offset_new=None, U_start=None, n_steps=3, with_dev=True, stream=None):
        """Per-cell Fisher scoring of new rows; inputs are CUDA tensors."""
        import torch
        n_new = Ynew.shape[0]
        _, m, p, q, d = self.dims
        ydt = _torch_ydt(Ynew)
        dev = Ynew.device
        U = torch.empty((n_new, d), dtype=torch.float32, device=dev)
        G = torch.empty((n_new, q), dtype=torch.float32, device=dev)
        D = torch.empty((n_new,), dtype=torch.float32, device=dev) if with_dev else None
        Yc = Ynew.contiguous()
        Xf = Xnew.to(torch.float32).contiguous()
        of = None if offset_new is None else offset_new.to(torch.float32).contiguous()
        us = None if U_start is None else U_start.to(torch.float32).contiguous()
        check(lib().gmf_project_cells(self._h, _ptr(Yc), ydt, n_new, _ptr(Xf), _ptr(of), _ptr(us),
                                      int(n_steps), _ptr(U), _ptr(G), _ptr(D), _stream(stream)))
        self._keep_proj = (Yc, Xf, of, us)
        return U, G, D


class Sweep:
    """Fits of several latent ranks on one count matrix, advanced together by
    one launch per sweep (a ``gmf_sweep`` handle)."""

    def __init__(self, Y, X, Z, offset, starts, d_list, *, family, nb_row, nb_col, row_perm, col_perm, settings,
                 precision="fp32", W=None, stream=None):
        import torch
        self._h = VP()
        on_dev = isinstance(Y, torch.Tensor) and Y.is_cuda
        if isinstance(Y, torch.Tensor):
            n, m = Y.shape
            ydt = _torch_ydt(Y)
            Y = Y.contiguous()
        else:
            Y = np.ascontiguousarray(Y)
            n, m = Y.shape
            ydt = GMF_Y_INT32 if Y.dtype == np.int32 else GMF_Y_UINT16
        X = np.ascontiguousarray(X, dtype=np.float64)
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        p, q = X.shape[1], Z.shape[1]
        d_list = [int(d) for d in d_list]
        nm = len(d_list)
        cfg = make_config(n, m, p, q, 0, family, nb_row, nb_col, settings, precision)
        off = None if offset is None else np.ascontiguousarray(offset, dtype=np.float64)
        arrs = [dict(B=_f64(st["B"], (m, p)), G=_f64(st["Gamma"], (n, q)), U=_f64(st["U"], (n, d)),
                     V=_f64(st["V"], (m, d))) for st, d in zip(starts, d_list)]
        ptrs = {k: (C.c_void_p * nm)(*[a[k].ctypes.data for a in arrs]) for k in ("B", "G", "U", "V")}
        alph = np.array([float(st.get("alpha", 1.0)) for st in starts])
        dl = np.array(d_list, dtype=np.int32)
        rp = np.ascontiguousarray(row_perm, dtype=np.int32)
        cp = np.ascontiguousarray(col_perm, dtype=np.int32)
        if W is not None:
            W = W.to(torch.float32).contiguous() if on_dev else np.ascontiguousarray(W, dtype=np.float32)
        check(lib().gmf_sweep_init(C.byref(self._h), C.byref(cfg), dl.ctypes.data, nm, _ptr(Y), ydt, int(on_dev),
                                   _ptr(W), _ptr(X), _ptr(Z), _ptr(off), _ptr(rp), _ptr(cp), C.addressof(ptrs["B"]),
                                   C.addressof(ptrs["G"]), C.addressof(ptrs["U"]), C.addressof(ptrs["V"]),
                                   alph.ctypes.data, _stream(stream)))
        self.models = [Model._borrow(lib().gmf_sweep_model(self._h, i), (n, m, p, q, d), self)
                       for i, d in enumerate(d_list)]
        self.d_list = d_list

    def epoch(self, sigma, stream=None):
        sigma = np.ascontiguousarray(sigma, dtype=np.int32)
        check(lib().gmf_sweep_epoch(self._h, sigma.ctypes.data, _stream(stream)))

    @property
    def group(self):
        """Models per launch group (see gmf_sweep_set_group)."""
        return lib().gmf_sweep_group(self._h)

    @group.setter
    def group(self, g):
        check(lib().gmf_sweep_set_group(self._h, int(g)))

    def autotune(self, sigma, n_sweeps=None, stream=None):
        """Time the launch groupings, the sequential setting and (mixed precision) the persistent launch on
        sweeps of the epoch sigma from the models' current state (restored afterwards) and keep the fastest;
        returns (group, {group: ms}), group GMF_SWEEP_SEQUENTIAL (-1) for the sequential setting and
        GMF_SWEEP_PERSISTENT (-3) for the persistent launch."""
        sigma = np.ascontiguousarray(sigma, dtype=np.int32)
        n_sweeps = len(sigma) if n_sweeps is None else int(n_sweeps)
        nm = len(self.models)
        g = C.c_int32()
        ms = np.empty(nm + 2, dtype=np.float32)
        check(lib().gmf_sweep_autotune(self._h, sigma.ctypes.data, n_sweeps, C.addressof(g), ms.ctypes.data,
                                       _stream(stream)))
        times = {i + 1: float(v) for i, v in enumerate(ms[:nm]) if v >= 0}
        if ms[nm] >= 0:
            times[GMF_SWEEP_SEQUENTIAL] = float(ms[nm])
        if ms[nm + 1] >= 0:
            times[GMF_SWEEP_PERSISTENT] = float(ms[nm + 1])
        return g.value, times

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.gmf_sweep_free(h)
            self._h = VP()


MLP_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


class MLP:
    """The warm-start encoder (a ``gmf_mlp`` handle): log1p(counts) -> scores."""

    def __init__(self, n_in, n_h1, n_h2, n_out, max_batch=1024, stream=None):
        self._h = VP()
        self.shapes = dict(W1=(n_h1, n_in), b1=(n_h1,), W2=(n_h2, n_h1), b2=(n_h2,), W3=(n_out, n_h2), b3=(n_out,))
        self.n_in, self.n_out, self.max_batch = n_in, n_out, max_batch
        check(lib().gmf_mlp_create(C.byref(self._h), n_in, n_h1, n_h2, n_out, max_batch, _stream(stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.gmf_mlp_free(h)
            self._h = VP()

    def set_params(self, P, stream=None):
        arrs = [np.ascontiguousarray(P[k], dtype=np.float32).reshape(self.shapes[k]) for k in MLP_NAMES]
        check(lib().gmf_mlp_set_params(self._h, *[a.ctypes.data for a in arrs], _stream(stream)))

    def _get(self, fn, stream):
        out = {k: np.empty(self.shapes[k], dtype=np.float32) for k in MLP_NAMES}
        check(fn(self._h, *[out[k].ctypes.data for k in MLP_NAMES], _stream(stream)))
        return out

    def get_params(self, stream=None):
        return self._get(lib().gmf_mlp_get_params, stream)

    def get_grads(self, stream=None):
        return self._get(lib().gmf_mlp_get_grads, stream)

    @staticmethod
    def _ydt(Y):
        return _torch_ydt(Y)

    def forward(self, Y, stream=None):
        import torch
        Yc = Y.contiguous()
        out = torch.empty((Y.shape[0], self.n_out), dtype=torch.float32, device=Y.device)
        check(lib().gmf_mlp_forward(self._h, Yc.data_ptr(), self._ydt(Y), Y.shape[0], out.data_ptr(), _stream(stream)))
        return out

    def loss_grad(self, Y, target, stream=None):
        import torch
        Yc, Tc = Y.contiguous(), target.to(torch.float32).contiguous()
        loss = torch.zeros(1, dtype=torch.float32, device=Y.device)
        check(lib().gmf_mlp_loss_grad(self._h, Yc.data_ptr(), self._ydt(Y), Y.shape[0], Tc.data_ptr(),
                                      loss.data_ptr(), _stream(stream)))
        return loss

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        check(lib().gmf_mlp_adam(self._h, lr, beta1, beta2, eps, _stream(stream)))

    def set_precision(self, precision, stream=None):
        """"fp32" (default) or "mixed": the first layer on the tensor cores with BF16 W1 and inputs."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        check(lib().gmf_mlp_set_precision(self._h, p, _stream(stream)))

    def train(self, Y, target, epochs, batch, lr, seed=0, stream=None):
        import torch
        Yc, Tc = Y.contiguous(), target.to(torch.float32).contiguous()
        losses = np.zeros(max(epochs, 1), dtype=np.float32)
        check(lib().gmf_mlp_train(self._h, Yc.data_ptr(), self._ydt(Y), Y.shape[0], Tc.data_ptr(), epochs, batch,
                                  lr, seed, losses.ctypes.data, _stream(stream)))
        return losses[:epochs]
