"""FP64 oracle for block-wise adaptive SGD on GMF models (arXiv 2412.20509).

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA library is
checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. It
shares no code with the CUDA package and never imports it.

The SGD loop, the block estimators and the deviance live in ``gmf_oracle.c``
(plain C, FP64, single thread); this module loads it through ctypes and keeps
the state in numpy arrays. Algorithm 2 (identifiability projection) is in
``oracle.orth``; per-cell Fisher scoring in ``oracle.project``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(finite differences, closed forms, brute force, invariants).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmf_oracle.c")
_LIB = os.path.join(_HERE, "libgmf_oracle.so")


def build(force=False):
    """Compile the C oracle with gcc (FP64, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Config(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("p", C.c_int32), ("q", C.c_int32),
                ("d", C.c_int32), ("family", C.c_int32), ("nb_row", C.c_int32), ("nb_col", C.c_int32),
                ("bias_corr", C.c_int32), ("alpha_mode", C.c_int32), ("missing", C.c_int32),
                ("lambda_", C.c_double * 4),
                ("a1", C.c_double), ("a2", C.c_double), ("k0", C.c_double), ("k1", C.c_double),
                ("tau", C.c_double), ("damping", C.c_double), ("eps", C.c_double),
                ("eta_clamp", C.c_double)]


class _Data(C.Structure):
    _fields_ = [("Y", C.c_void_p), ("y_dtype", C.c_int32), ("W", C.c_void_p), ("X", C.c_void_p),
                ("Z", C.c_void_p), ("offset", C.c_void_p), ("row_perm", C.c_void_p),
                ("col_perm", C.c_void_p), ("alpha_col", C.c_void_p)]


class _State(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("B", "G", "U", "V", "Gb_row", "Hb_row", "Gb_col", "Hb_col",
                                            "cnt_row", "cnt_col", "alpha", "t")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.gmfo_entry.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib.gmfo_entry.restype = None
        _lib.gmfo_entry_deviance.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        _lib.gmfo_entry_deviance.restype = C.c_double
        _lib.gmfo_block_grad.argtypes = ([C.c_void_p] * 3 + [C.c_double] +
                                         [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64] + [C.c_void_p] * 5)
        _lib.gmfo_block_grad.restype = C.c_int
        _lib.gmfo_sgd_epoch.argtypes = [C.c_void_p] * 4
        _lib.gmfo_sgd_epoch.restype = C.c_int
        _lib.gmfo_sgd_sweeps.argtypes = [C.c_void_p] * 4 + [C.c_int64, C.c_int64]
        _lib.gmfo_sgd_sweeps.restype = C.c_int
        _lib.gmfo_sgd_sweep_blocks.argtypes = [C.c_void_p] * 4 + [C.c_int64, C.c_void_p, C.c_int64]
        _lib.gmfo_sgd_sweep_blocks.restype = C.c_int
        _lib.gmfo_deviance.argtypes = [C.c_void_p] * 3
        _lib.gmfo_deviance.restype = C.c_double
        _lib.gmfo_eta_entries.argtypes = [C.c_void_p] * 5 + [C.c_int64, C.c_void_p]
        _lib.gmfo_eta_entries.restype = None
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def entry(family, y, eta, w=1.0, alpha=1.0, clamp=30.0):
    """(mu, Ddot, Dddot) of one entry (Sec. 3); alpha is the family's scalar (NB shape or dispersion phi)."""
    mu, dd, ddd = C.c_double(), C.c_double(), C.c_double()
    lib().gmfo_entry(int(family), float(y), float(eta), float(w), float(alpha), float(clamp),
                     C.byref(mu), C.byref(dd), C.byref(ddd))
    return mu.value, dd.value, ddd.value


def entry_deviance(family, y, mu, w=1.0, alpha=1.0):
    return lib().gmfo_entry_deviance(int(family), float(y), float(mu), float(w), float(alpha))


# Table S1: log link for the count families, the Gamma and the inverse Gaussian; identity (Gaussian) and
# logit (Bernoulli, "binomial") as their canonical links
FAMILIES = {"poisson": 0, "negbin": 1, "gaussian": 2, "binomial": 3, "gamma": 4, "invgauss": 5}
Y_DTYPES = {np.dtype(np.int32): 0, np.dtype(np.uint16): 1, np.dtype(np.float32): 2}


class OracleFit:
    """State of one fit: parameters in the original row/column order, the
    smoothed derivatives of eq. 12, visit counters, the family's scalar (NB
    shape or dispersion phi, in ``alpha``) and t. Y: int32 / uint16 counts,
    or float32 responses (NaN = missing)."""

    def __init__(self, Y, X, Z, offset, start, *, family, nb_row, nb_col, row_perm, col_perm,
                 settings, W=None, alpha_col=None):
        self.Y = np.ascontiguousarray(Y)
        if self.Y.dtype not in Y_DTYPES:
            raise TypeError("Y must be int32, uint16 or float32")
        n, m = self.Y.shape
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.Z = np.ascontiguousarray(Z, dtype=np.float64)
        p, q = self.X.shape[1], self.Z.shape[1]
        d = np.asarray(start["U"]).shape[1]
        self.offset = None if offset is None else np.ascontiguousarray(offset, dtype=np.float64)
        self.W = None if W is None else np.ascontiguousarray(W, dtype=np.float64)
        # per-gene NB shapes (alpha_mode 2), in the original gene order
        self.alpha_col = None if alpha_col is None else np.ascontiguousarray(alpha_col, dtype=np.float64)
        self.row_perm = np.ascontiguousarray(row_perm, dtype=np.int32)
        self.col_perm = np.ascontiguousarray(col_perm, dtype=np.int32)
        self.B = np.array(start["B"], dtype=np.float64, order="C").reshape(m, p)
        self.G = np.array(start["Gamma"], dtype=np.float64, order="C").reshape(n, q)
        self.U = np.array(start["U"], dtype=np.float64, order="C").reshape(n, d)
        self.V = np.array(start["V"], dtype=np.float64, order="C").reshape(m, d)
        self.Gb_row = np.zeros((n, q + d))
        self.Hb_row = np.zeros((n, q + d))
        self.Gb_col = np.zeros((m, p + d))
        self.Hb_col = np.zeros((m, p + d))
        self.cnt_row = np.zeros(n, dtype=np.int64)
        self.cnt_col = np.zeros(m, dtype=np.int64)
        self.alpha = np.array([float(start.get("alpha", 1.0))])
        self.t = np.zeros(1, dtype=np.int64)
        s = settings
        self.cfg = _Config(n=n, m=m, p=p, q=q, d=d, family=FAMILIES[family] if isinstance(family, str) else int(family),
                           nb_row=int(nb_row), nb_col=int(nb_col), bias_corr=int(s["bias_corr"]),
                           alpha_mode=int(s["alpha_mode"]), missing=int(s.get("missing", 0)),
                           lambda_=(C.c_double * 4)(*s["lambda_"]),
                           a1=s["a1"], a2=s["a2"], k0=s["k0"], k1=s["k1"], tau=s["tau"],
                           damping=s["damping"], eps=s["eps"], eta_clamp=s["eta_clamp"])
        self._data = _Data(Y=self.Y.ctypes.data, y_dtype=Y_DTYPES[self.Y.dtype],
                           W=_p(self.W), X=_p(self.X), Z=_p(self.Z), offset=_p(self.offset),
                           row_perm=_p(self.row_perm), col_perm=_p(self.col_perm), alpha_col=_p(self.alpha_col))
        self._state = _State(**{k: getattr(self, k).ctypes.data for k, _ in _State._fields_})

    @property
    def dims(self):
        c = self.cfg
        return c.n, c.m, c.p, c.q, c.d

    def epoch(self, sigma):
        sigma = np.ascontiguousarray(sigma, dtype=np.int32)
        rc = lib().gmfo_sgd_epoch(C.byref(self.cfg), C.byref(self._data), C.byref(self._state), sigma.ctypes.data)
        if rc:
            raise RuntimeError(f"oracle epoch failed ({rc})")

    def sweeps(self, sigma, w0, w1):
        sigma = np.ascontiguousarray(sigma, dtype=np.int32)
        rc = lib().gmfo_sgd_sweeps(C.byref(self.cfg), C.byref(self._data), C.byref(self._state),
                                   sigma.ctypes.data, int(w0), int(w1))
        if rc:
            raise RuntimeError(f"oracle sweeps failed ({rc})")

    def sweep_blocks(self, sigma, w, blocks):
        """Sweep w restricted to the listed blocks; t advances by the whole sweep."""
        sigma = np.ascontiguousarray(sigma, dtype=np.int32)
        b = np.ascontiguousarray(sorted(int(k) for k in blocks), dtype=np.int32)
        rc = lib().gmfo_sgd_sweep_blocks(C.byref(self.cfg), C.byref(self._data), C.byref(self._state),
                                         sigma.ctypes.data, int(w), b.ctypes.data, len(b))
        if rc:
            raise RuntimeError(f"oracle sweep_blocks failed ({rc})")

    def deviance(self):
        return lib().gmfo_deviance(C.byref(self.cfg), C.byref(self._data), C.byref(self._state))

    def block_grad(self, I, J, alpha=None):
        """Block estimators of eq. 15 / App. B (no penalty, no damping)."""
        n, m, p, q, d = self.dims
        I = np.ascontiguousarray(I, dtype=np.int32)
        J = np.ascontiguousarray(J, dtype=np.int32)
        Grow = np.zeros((len(I), q + d)); Hrow = np.zeros_like(Grow)
        Gcol = np.zeros((len(J), p + d)); Hcol = np.zeros_like(Gcol)
        sums = np.zeros(2)
        lib().gmfo_block_grad(C.byref(self.cfg), C.byref(self._data), C.byref(self._state),
                              float(self.alpha[0] if alpha is None else alpha),
                              I.ctypes.data, len(I), J.ctypes.data, len(J),
                              Grow.ctypes.data, Hrow.ctypes.data, Gcol.ctypes.data, Hcol.ctypes.data,
                              sums.ctypes.data)
        return Grow, Hrow, Gcol, Hcol, sums

    def eta_entries(self, ii, jj):
        ii = np.ascontiguousarray(ii, dtype=np.int64)
        jj = np.ascontiguousarray(jj, dtype=np.int64)
        out = np.empty(len(ii))
        lib().gmfo_eta_entries(C.byref(self.cfg), C.byref(self._data), C.byref(self._state),
                               ii.ctypes.data, jj.ctypes.data, len(ii), out.ctypes.data)
        return out

    def eta(self):
        """Full linear predictor (numpy; for small problems and tests)."""
        e = self.X @ self.B.T + self.G @ self.Z.T + self.U @ self.V.T
        if self.offset is not None:
            e = e + self.offset[:, None]
        return e

    def params(self):
        return dict(B=self.B.copy(), Gamma=self.G.copy(), U=self.U.copy(), V=self.V.copy(),
                    alpha=float(self.alpha[0]))
