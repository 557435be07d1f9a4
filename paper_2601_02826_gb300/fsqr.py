"""Thin ctypes binding of the C ABI in include/fsqr.h (libfsqr.so).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels. Device arrays are torch CUDA tensors (float64 / uint8 / int8,
contiguous); host arrays are numpy. The in-tree library must have been built
(paper_2601_02826_gb300.build.build()); nothing here falls back to any other
implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOCONV, ETIMEOUT, ENUMERIC, ECUDA, ENOMEM = range(7)
DENSE_F64, INT8, TWOBIT = 0, 1, 2
FP64, MIXED, MIXED_SIMT = 0, 1, 2
WARM_NONE, WARM_GIVEN, WARM_PATH = 0, 1, 2
PEN_SCAD, PEN_MCP = 1, 2

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOCONV", 3: "ETIMEOUT", 4: "ENUMERIC", 5: "ECUDA", 6: "ENOMEM"}


class Design(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_int64), ("c", C.c_int64),
                ("geno_format", C.c_int32), ("standardize", C.c_int32),
                ("geno", C.c_void_p), ("geno_ld", C.c_int64), ("cov", C.c_void_p),
                ("col_mean", C.c_void_p), ("col_sd", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("check_every", C.c_int32),
                ("mu", C.c_double), ("eta", C.POINTER(C.c_double)), ("eta_margin", C.c_double),
                ("power_iters", C.c_int32), ("power_tol", C.c_double), ("precision", C.c_int32),
                ("warm", C.c_int32), ("digits", C.c_int32), ("max_group", C.c_int32),
                ("timeout_ms", C.c_int64), ("warm_params", C.c_void_p), ("ridge", C.c_double),
                ("screen", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("kkt", C.c_double),
                ("r_p", C.c_double), ("r_z", C.c_double), ("r_beta", C.c_double),
                ("r_1", C.c_double), ("primal", C.c_double), ("dual", C.c_double),
                ("gap", C.c_double), ("lambda_", C.c_double), ("lambda_max", C.c_double),
                ("mu", C.c_double), ("active", C.c_int64), ("t_setup_ms", C.c_double),
                ("t_solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(C.Structure):
    _fields_ = [("col_samples", C.c_int64), ("col_ms", C.c_double), ("xb_samples", C.c_int64),
                ("xb_ms", C.c_double), ("vec_samples", C.c_int64), ("vec_ms", C.c_double),
                ("iterations", C.c_int64), ("kernel_launches", C.c_int64), ("col_bytes", C.c_int64),
                ("tuned_group", C.c_int64), ("tc_groups", C.c_int64), ("simt_groups", C.c_int64),
                ("wide_groups", C.c_int64), ("screen_kept", C.c_int64), ("screen_total", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["fsqr_version", "fsqr_opts_default", "fsqr_create", "fsqr_destroy", "fsqr_last_error",
           "fsqr_col_stats", "fsqr_lambda_max", "fsqr_eta", "fsqr_fit", "fsqr_fit_batch",
           "fsqr_fit_batch_host", "fsqr_fit_lla", "fsqr_path_stats", "fsqr_interval_coverage", "fsqr_kkt", "fsqr_predict", "fsqr_back_transform",
           "fsqr_profile_enable", "fsqr_profile_get", "fsqr_profile_reset", "fsqr_wait_selftest",
           "fsqr_lambda_max_noalloc", "fsqr_mlp_param_count", "fsqr_mlp_init", "fsqr_mlp_forward",
           "fsqr_mlp_grad", "fsqr_mlp_train", "fsqr_warm_features", "fsqr_warm_start"]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Loads libfsqr.so (building it first if needed); raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        _build.build()
    L = C.CDLL(p)
    vp, i32, i64, dbl, pd = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.POINTER(C.c_double)
    pD, pO, pI = C.POINTER(Design), C.POINTER(Opts), C.POINTER(Info)
    pi64 = C.POINTER(C.c_int64)
    L.fsqr_version.restype = i32
    L.fsqr_opts_default.argtypes = [pO]
    L.fsqr_opts_default.restype = None
    L.fsqr_create.argtypes = [C.POINTER(vp), i32, vp]
    L.fsqr_destroy.argtypes = [vp]
    L.fsqr_last_error.argtypes = [vp]
    L.fsqr_last_error.restype = C.c_char_p
    L.fsqr_col_stats.argtypes = [vp, pD, vp, vp]
    L.fsqr_lambda_max.argtypes = [vp, pD, vp, dbl, vp, pd]
    L.fsqr_lambda_max_noalloc.argtypes = [vp, pD, vp, dbl, vp, pd]
    L.fsqr_eta.argtypes = [vp, pD, pi64, i32, dbl, dbl, i32, dbl, pd]
    L.fsqr_fit.argtypes = [vp, pD, vp, dbl, dbl, vp, pi64, i32, pO, vp, vp, vp, pI]
    L.fsqr_fit_batch.argtypes = [vp, pD, vp, i32, pd, i32, pd, vp, pi64, i32, pO, vp, vp, vp, pI]
    L.fsqr_fit_batch_host.argtypes = [vp, pD, vp, i32, pd, i32, pd, vp, pi64, i32, pO, vp, vp, vp, pI]
    L.fsqr_fit_lla.argtypes = [vp, pD, vp, dbl, dbl, vp, pi64, i32, i32, dbl, i32, pO, vp, vp, vp, vp, pI]
    L.fsqr_path_stats.argtypes = [vp, pD, vp, i32, pd, vp, pd, pi64, pd]
    L.fsqr_interval_coverage.argtypes = [vp, pD, vp, vp, vp, pd, pd, pi64]
    L.fsqr_kkt.argtypes = [vp, pD, vp, dbl, dbl, vp, dbl, vp, vp, vp, pI]
    L.fsqr_predict.argtypes = [vp, pD, vp, i32, vp]
    L.fsqr_back_transform.argtypes = [vp, pD, vp, i32, vp]
    L.fsqr_profile_enable.argtypes = [vp, i32]
    L.fsqr_wait_selftest.argtypes = [vp, i64, i32, C.POINTER(C.c_int)]
    L.fsqr_profile_get.argtypes = [vp, C.POINTER(Profile)]
    L.fsqr_profile_reset.argtypes = [vp]
    u64, flt = C.c_uint64, C.c_float
    L.fsqr_mlp_param_count.argtypes = []
    L.fsqr_mlp_init.argtypes = [vp, vp, u64]
    L.fsqr_mlp_forward.argtypes = [vp, vp, vp, i64, vp]
    L.fsqr_mlp_grad.argtypes = [vp, vp, vp, vp, vp, i64, vp, pd]
    L.fsqr_mlp_train.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, i64, i32, i32, flt, u64, pd]
    L.fsqr_warm_features.argtypes = [vp, pD, vp, dbl, dbl, vp, vp, pd]
    L.fsqr_warm_start.argtypes = [vp, pD, vp, dbl, dbl, vp, vp, vp, vp, vp]
    for f in EXPORTS:
        if f not in ("fsqr_opts_default", "fsqr_last_error", "fsqr_version"):
            getattr(L, f).restype = i32
    L.fsqr_mlp_param_count.restype = i64
    _lib = L
    return L


class FsqrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _host_ptr(a):
    """Host address of a numpy array or a CPU (ideally pinned) torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def default_opts(**kw) -> Opts:
    L = load()
    o = Opts()
    L.fsqr_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "eta":
            continue
        setattr(o, k, v)
    return o


class Context:
    """A library context bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self.L = load()
        h = C.c_void_p()
        s = C.c_void_p(stream) if stream else None
        rc = self.L.fsqr_create(C.byref(h), device, s)
        if rc != OK:
            raise FsqrError(rc, "fsqr_create failed")
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            self.L.fsqr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allowed=(OK,)):
        if rc not in allowed:
            raise FsqrError(rc, self.L.fsqr_last_error(self.h).decode())
        return rc

    # ------------------------------------------------------------- designs
    def design(self, n, p, c, fmt, geno, ld, cov=None, col_mean=None, col_sd=None, standardize=1,
               host=False):
        d = Design()
        d.n, d.p, d.c = n, p, c
        d.geno_format, d.standardize = fmt, standardize
        ptr = _host_ptr if host else _ptr
        d.geno = ptr(geno) if geno is not None else None
        d.geno_ld = ld
        d.cov = ptr(cov) if (cov is not None and c > 0) else None
        d.col_mean = ptr(col_mean) if col_mean is not None else None
        d.col_sd = ptr(col_sd) if col_sd is not None else None
        self._keep.append((geno, cov, col_mean, col_sd))
        return d

    # ---------------------------------------------------------- functions
    def col_stats(self, d, mean_out, sd_out):
        """fsqr_col_stats: column means and population sds (standardisation, Section 7)."""
        self._check(self.L.fsqr_col_stats(self.h, C.byref(d), _ptr(mean_out), _ptr(sd_out)))

    def lambda_max(self, d, y, tau, omega) -> float:
        """fsqr_lambda_max: the smallest lambda with beta_{1..} = 0 optimal (penalty path, Section 7)."""
        out = C.c_double()
        self._check(self.L.fsqr_lambda_max(self.h, C.byref(d), _ptr(y), tau, _ptr(omega), C.byref(out)))
        return out.value

    def lambda_max_noalloc(self, d, y, tau, omega) -> float:
        """fsqr_lambda_max_noalloc: as lambda_max, on the library's static
        device scratch instead of its workspace (no device allocation)."""
        out = C.c_double()
        self._check(self.L.fsqr_lambda_max_noalloc(self.h, C.byref(d), _ptr(y), tau, _ptr(omega),
                                                   C.byref(out)))
        return out.value

    def eta(self, d, block_ptr, mu, margin=0.05, max_iter=100, tol=1e-6) -> np.ndarray:
        """fsqr_eta: eta_g = (1 + margin) mu Lambda_hat(X~_g^T X~_g) by the power method (Section 4)."""
        bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
        G = len(bp) - 1
        out = np.zeros(max(G, 1))
        self._check(self.L.fsqr_eta(self.h, C.byref(d), bp.ctypes.data_as(C.POINTER(C.c_int64)), G,
                                    mu, margin, max_iter, tol, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out[:G]

    def _opts(self, opts: dict | None, G: int):
        o = default_opts(**(opts or {}))
        eta = None
        if opts and opts.get("eta") is not None:
            eta = np.ascontiguousarray(opts["eta"], dtype=np.float64)
            assert len(eta) == G
            o.eta = eta.ctypes.data_as(C.POINTER(C.c_double))
        return o, eta

    def fit(self, d, y, tau, lam, omega, block_ptr, beta, z, theta, opts=None,
            allowed=(OK, ENOCONV, ETIMEOUT)):
        """fsqr_fit: one FS-QRPPA fit (Algorithm 1); beta, z, theta receive the result (and hold the start when opts warm = 1)."""
        bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
        G = len(bp) - 1
        o, keep = self._opts(opts, G)
        info = Info()
        rc = self.L.fsqr_fit(self.h, C.byref(d), _ptr(y), tau, lam, _ptr(omega),
                             bp.ctypes.data_as(C.POINTER(C.c_int64)), G, C.byref(o),
                             _ptr(beta), _ptr(z), _ptr(theta), C.byref(info))
        self._check(rc, allowed)
        return rc, info

    def fit_batch(self, d, y, taus, lambdas, omega, block_ptr, beta, z, theta, opts=None,
                  allowed=(OK, ENOCONV, ETIMEOUT), host=False):
        """fsqr_fit_batch (host=True: fsqr_fit_batch_host): a tau x lambda grid of fits."""
        taus = np.ascontiguousarray(taus, dtype=np.float64)
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        n_tau = len(taus)
        n_lambda = lam.size // n_tau
        assert lam.size == n_tau * n_lambda
        bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
        G = len(bp) - 1
        o, keep = self._opts(opts, G)
        infos = (Info * (n_tau * n_lambda))()
        fn = self.L.fsqr_fit_batch_host if host else self.L.fsqr_fit_batch
        ptr = _host_ptr if host else _ptr
        rc = fn(self.h, C.byref(d), ptr(y), n_tau, taus.ctypes.data_as(C.POINTER(C.c_double)),
                n_lambda, lam.ctypes.data_as(C.POINTER(C.c_double)), ptr(omega),
                bp.ctypes.data_as(C.POINTER(C.c_int64)), G, C.byref(o), ptr(beta), ptr(z), ptr(theta),
                infos)
        self._check(rc, allowed)
        return rc, list(infos)

    def fit_lla(self, d, y, tau, lam, omega, block_ptr, penalty, a, L, beta, z, theta, lam_out=None,
                opts=None, allowed=(OK, ENOCONV, ETIMEOUT)):
        """fsqr_fit_lla: L-step LLA for SCAD (PEN_SCAD) or MCP (PEN_MCP)."""
        bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
        G = len(bp) - 1
        o, keep = self._opts(opts, G)
        info = Info()
        rc = self.L.fsqr_fit_lla(self.h, C.byref(d), _ptr(y), tau, lam, _ptr(omega),
                                 bp.ctypes.data_as(C.POINTER(C.c_int64)), G, penalty, a, L, C.byref(o),
                                 _ptr(beta), _ptr(z), _ptr(theta), _ptr(lam_out), C.byref(info))
        self._check(rc, allowed)
        return rc, info

    def path_stats(self, d, y, taus, beta):
        """fsqr_path_stats: (loss, active, hbic) of B fits (numpy arrays)."""
        taus = np.ascontiguousarray(taus, dtype=np.float64)
        B = len(taus)
        loss, hb = np.zeros(B), np.zeros(B)
        act = np.zeros(B, dtype=np.int64)
        self._check(self.L.fsqr_path_stats(self.h, C.byref(d), _ptr(y), B,
                                           taus.ctypes.data_as(C.POINTER(C.c_double)), _ptr(beta),
                                           loss.ctypes.data_as(C.POINTER(C.c_double)),
                                           act.ctypes.data_as(C.POINTER(C.c_int64)),
                                           hb.ctypes.data_as(C.POINTER(C.c_double))))
        return loss, act, hb

    def interval_coverage(self, d, y, beta_lo, beta_hi):
        """fsqr_interval_coverage: (coverage, mean width, crossings)."""
        cov, wid = C.c_double(), C.c_double()
        cr = C.c_int64()
        self._check(self.L.fsqr_interval_coverage(self.h, C.byref(d), _ptr(y), _ptr(beta_lo), _ptr(beta_hi),
                                                  C.byref(cov), C.byref(wid), C.byref(cr)))
        return cov.value, wid.value, cr.value

    def kkt(self, d, y, tau, lam, omega, lam_norm, beta, z, theta) -> Info:
        """fsqr_kkt: stop-test residuals, primal, dual and gap of a given iterate (Proposition 1)."""
        info = Info()
        self._check(self.L.fsqr_kkt(self.h, C.byref(d), _ptr(y), tau, lam, _ptr(omega), lam_norm,
                                    _ptr(beta), _ptr(z), _ptr(theta), C.byref(info)))
        return info

    # ---- learned warm start (float32 device tensors for the network)

    def mlp_param_count(self) -> int:
        """fsqr_mlp_param_count: floats in the warm-start network."""
        return int(self.L.fsqr_mlp_param_count())

    def mlp_init(self, params, seed: int):
        """fsqr_mlp_init: seeded initial parameters of the warm-start network."""
        self._check(self.L.fsqr_mlp_init(self.h, _ptr(params), seed))

    def mlp_forward(self, params, x, out):
        """fsqr_mlp_forward: the network on the rows of x (FP32, device)."""
        self._check(self.L.fsqr_mlp_forward(self.h, _ptr(params), _ptr(x), x.shape[0], _ptr(out)))

    def mlp_grad(self, params, x, t, w, grad) -> float:
        """fsqr_mlp_grad: weighted squared loss and its gradient; returns the loss."""
        loss = C.c_double()
        self._check(self.L.fsqr_mlp_grad(self.h, _ptr(params), _ptr(x), _ptr(t), _ptr(w), x.shape[0],
                                         _ptr(grad), C.byref(loss)))
        return loss.value

    def mlp_train(self, params, m, v, step0, x, t, w, steps, batch, lr, seed) -> np.ndarray:
        """fsqr_mlp_train: Adam steps on batches drawn on the device; returns the losses."""
        losses = np.zeros(max(steps, 1))
        self._check(self.L.fsqr_mlp_train(self.h, _ptr(params), _ptr(m), _ptr(v), step0, _ptr(x), _ptr(t),
                                          _ptr(w), x.shape[0], steps, batch, lr, seed,
                                          losses.ctypes.data_as(C.POINTER(C.c_double))))
        return losses[:steps]

    def warm_features(self, d, y, tau, lam_frac, omega, u) -> float:
        """fsqr_warm_features: the network inputs of every feature column; returns lambda_max."""
        lmax = C.c_double()
        self._check(self.L.fsqr_warm_features(self.h, C.byref(d), _ptr(y), tau, lam_frac, _ptr(omega), _ptr(u),
                                              C.byref(lmax)))
        return lmax.value

    def warm_start(self, d, y, tau, lam_frac, omega, params, beta, z, theta):
        """fsqr_warm_start: the start (beta, z, theta) the network proposes for one fit."""
        self._check(self.L.fsqr_warm_start(self.h, C.byref(d), _ptr(y), tau, lam_frac, _ptr(omega),
                                           _ptr(params), _ptr(beta), _ptr(z), _ptr(theta)))

    def predict(self, d, beta, B, out):
        """fsqr_predict: x~_i^T beta of B coefficient vectors (Section 7.1)."""
        self._check(self.L.fsqr_predict(self.h, C.byref(d), _ptr(beta), B, _ptr(out)))

    def back_transform(self, d, beta_std, B, out):
        """fsqr_back_transform: standardised coefficients on the original scale (Section 7)."""
        self._check(self.L.fsqr_back_transform(self.h, C.byref(d), _ptr(beta_std), B, _ptr(out)))

    def profile(self, enable: bool | None = None, reset: bool = False) -> Profile:
        """fsqr_profile_*: switch kernel sampling, read the counters, optionally reset them."""
        if enable is not None:
            self.L.fsqr_profile_enable(self.h, 1 if enable else 0)
        if reset:
            self.L.fsqr_profile_reset(self.h)
        p = Profile()
        self.L.fsqr_profile_get(self.h, C.byref(p))
        return p

    def wait_selftest(self, budget_cycles: int, arrive: bool):
        """fsqr_wait_selftest: (status, wait_ok)."""
        ok = C.c_int(0)
        rc = self.L.fsqr_wait_selftest(self.h, budget_cycles, 1 if arrive else 0, C.byref(ok))
        self._check(rc, (OK, ETIMEOUT))
        return rc, ok.value

    def last_error(self) -> str:
        """fsqr_last_error: message of the last failed call."""
        return self.L.fsqr_last_error(self.h).decode()
