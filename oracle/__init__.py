"""FP64 CPU oracle for SRCD (NMF with KL divergence) -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package. The CUDA library neither imports nor links it, and
the two share no code. It wraps ``srcd_oracle.c`` (plain sequential FP64 C,
compiled with gcc on first use) and works in the paper's orientation:
W is r x n, F is r x m, V ~= W^T F (Section 1).

Functions follow the paper:
  philox4x64_10  -- the counter-based generator behind the coordinate order
  perm           -- "ids", a random permutation of the r coordinates (Algorithm 1)
  alg2           -- Algorithm 2 on one subproblem min_{x>=0} D(v||Ax)+a/2|x|^2+b|x|_1
  half_F/half_W  -- one half of Algorithm 1 (all columns of F, all rows of W)
  objective      -- Eq. 1 (and the regularizer of Eq. 2)
  fit            -- Algorithm 1 for a number of sweeps, with the KL trajectory
  foldin         -- F for new documents under a fixed W, per-document stopping
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srcd_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compiles srcd_oracle.c with gcc into oracle/lib/liboracle.so."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        r = subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                            "-ffp-contract=off", _SRC, "-o", tmp, "-lm"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(ctypes.Structure):
    """Parameters of Algorithm 2 for one side (see srcd_oracle.c)."""
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("eps_grad", ctypes.c_double), ("eps_div", ctypes.c_double),
                ("eps_x", ctypes.c_double), ("max_inner", ctypes.c_int32),
                ("grad_mode", ctypes.c_int32), ("break_mode", ctypes.c_int32),
                ("perm_mode", ctypes.c_int32), ("perturb", ctypes.c_double),
                ("perturb_seed", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("coords", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("cap_hits", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def cfg(alpha=0.0, beta=0.0, eps_grad=1e-6, eps_div=1e-6, eps_x=0.1, max_inner=16,
        grad_mode=0, break_mode=0, perm_mode=0, perturb=0.0, perturb_seed=0) -> Cfg:
    """Defaults: eps_x = 0.1 (Section 3); the rest are this project's readings.
    perturb > 0 turns on the Monte Carlo arithmetic probe (see srcd_oracle.c)."""
    return Cfg(alpha, beta, eps_grad, eps_div, eps_x, max_inner, grad_mode, break_mode, perm_mode,
               perturb, perturb_seed)


def tight_cfg(**kw) -> Cfg:
    """Each coordinate solved to its 1-D minimiser (tiny eps_x, high cap)."""
    base = dict(eps_x=1e-9, max_inner=64, eps_grad=1e-13)
    base.update(kw)
    return cfg(**base)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        cp = ctypes.POINTER(Cfg)
        sp = ctypes.POINTER(Stats)
        lib.oracle_philox4x64_10.argtypes = [vp, vp, vp]
        lib.oracle_perm.argtypes = [u64, i64, i32, i64, i32, i32, vp]
        lib.oracle_uniform_init.argtypes = [u64, i32, i64, vp]
        lib.oracle_alg2.argtypes = [i64, vp, vp, vp, vp, i32, vp, cp, vp, sp]
        lib.oracle_rowsum.argtypes = [vp, i32, i64, vp]
        lib.oracle_derivatives.argtypes = [i64, vp, vp, i32, vp, i32, f64, f64, cp, vp, vp]
        lib.oracle_half.argtypes = [i32, i64, vp, vp, vp, vp, i64, vp, i32, u64, i64, cp, i32, sp]
        lib.oracle_objective.argtypes = [i64, i64, i32, vp, vp, vp, vp, vp, f64, f64, f64, f64, f64,
                                         vp, vp]
        lib.oracle_column_objective.argtypes = [i64, i64, i32, vp, vp, vp, vp, vp, vp, i64, f64, f64, f64]
        lib.oracle_column_objective.restype = f64
        lib.oracle_fit.argtypes = [i64, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, u64, i64, i32,
                                   cp, cp, i32, vp, sp]
        lib.oracle_foldin.argtypes = [i64, i64, i32, vp, vp, vp, vp, vp, u64, f64, i32, cp, vp]
        for f in ("oracle_philox4x64_10", "oracle_perm", "oracle_uniform_init", "oracle_alg2",
                  "oracle_rowsum", "oracle_derivatives", "oracle_half", "oracle_objective", "oracle_fit", "oracle_foldin"):
            getattr(lib, f).restype = None
        _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    _load().oracle_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def perm(seed: int, sweep: int, side: int, col: int, r: int, perm_mode: int = 0) -> np.ndarray:
    out = np.empty(r, dtype=np.int32)
    _load().oracle_perm(seed, sweep, side, col, perm_mode, r, _p(out))
    return out


def uniform_init(seed: int, which: int, r: int, cols: int) -> np.ndarray:
    out = np.empty((r, cols), dtype=np.float64)
    _load().oracle_uniform_init(seed, which, r * cols, _p(out))
    return out


def alg2(v, A, sumA, x, ids, c: Cfg | None = None):
    """Algorithm 2 on one subproblem. v: (L,), A: (L, r) rows at the nonzeros,
    sumA: (r,), x: (r,) start, ids: coordinate order. Returns (x, stats)."""
    c = c or cfg()
    v = _f64(v)
    A = _f64(A)
    L, r = A.shape
    x = _f64(x).copy()
    sumA = _f64(sumA)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    ax = np.empty(max(L, 1), dtype=np.float64)
    st = Stats()
    _load().oracle_alg2(L, _p(v), _p(A), _p(sumA), _p(x), r, _p(ids), ctypes.byref(c), _p(ax),
                        ctypes.byref(st))
    return x, st.as_dict()


def derivatives(v, A, Ax, k, sumA_k, x_k, c: Cfg | None = None):
    """(g_k, h_k) of Eq. Partial at the given [Ax] on the nonzeros."""
    c = c or cfg()
    v = _f64(v)
    A = _f64(A)
    Ax = _f64(Ax)
    g = np.zeros(1)
    h = np.zeros(1)
    _load().oracle_derivatives(A.shape[0], _p(v), _p(A), A.shape[1], _p(Ax), k, sumA_k, x_k,
                               ctypes.byref(c), _p(g), _p(h))
    return float(g[0]), float(h[0])


def rowsum(M) -> np.ndarray:
    M = _f64(M)
    r, cols = M.shape
    out = np.empty(r, dtype=np.float64)
    _load().oracle_rowsum(_p(M), r, cols, _p(out))
    return out


def half_F(V, W, F, seed, sweep, c: Cfg | None = None, threads: int = 1):
    """F half of Algorithm 1: every column of F, W fixed. Returns (F, stats)."""
    c = c or cfg()
    W = _f64(W)
    F = _f64(F).copy()
    r = W.shape[0]
    st = Stats()
    _load().oracle_half(0, V.m, _p(V.colptr), _p(V.rowidx), _p(V.val), _p(W), V.n, _p(F), r,
                        seed, sweep, ctypes.byref(c), threads, ctypes.byref(st))
    return F, st.as_dict()


def half_W(V, W, F, seed, sweep, c: Cfg | None = None, threads: int = 1):
    """W half of Algorithm 1: every row of W, F fixed. Returns (W, stats)."""
    c = c or cfg()
    F = _f64(F)
    W = _f64(W).copy()
    r = F.shape[0]
    st = Stats()
    _load().oracle_half(1, V.n, _p(V.rowptr), _p(V.colidx), _p(V.rval), _p(F), V.m, _p(W), r,
                        seed, sweep, ctypes.byref(c), threads, ctypes.byref(st))
    return W, st.as_dict()


def objective(V, W, F, eps_div=1e-6, a1=0.0, a2=0.0, b1=0.0, b2=0.0):
    """(Eq. 1 value, Eq. 2 regularizer) at W (r x n), F (r x m)."""
    W = _f64(W)
    F = _f64(F)
    kl = ctypes.c_double()
    reg = ctypes.c_double()
    _load().oracle_objective(V.n, V.m, W.shape[0], _p(V.colptr), _p(V.rowidx), _p(V.val), _p(W),
                             _p(F), eps_div, a1, a2, b1, b2, ctypes.byref(kl), ctypes.byref(reg))
    return kl.value, reg.value


def column_objective(V, W, F, j, alpha=0.0, beta=0.0, eps_div=1e-6) -> float:
    W = _f64(W)
    F = _f64(F)
    sumW = rowsum(W)
    return _load().oracle_column_objective(V.n, V.m, W.shape[0], _p(V.colptr), _p(V.rowidx),
                                           _p(V.val), _p(W), _p(sumW), _p(F), j, eps_div,
                                           alpha, beta)


@dataclass
class FitResult:
    W: np.ndarray
    F: np.ndarray
    kl: np.ndarray
    stats: dict


def fit(V, W0, F0, seed, sweeps, cF: Cfg | None = None, cW: Cfg | None = None, threads: int = 1,
        sweep0: int = 0, trace: bool = True) -> FitResult:
    """Algorithm 1 for `sweeps` sweeps from (W0, F0); kl[s] is Eq. 1 after sweep s."""
    cF = cF or cfg()
    cW = cW or cfg()
    W = _f64(W0).copy()
    F = _f64(F0).copy()
    r = W.shape[0]
    kl = np.zeros(max(sweeps, 1), dtype=np.float64)
    st = Stats()
    _load().oracle_fit(V.n, V.m, r, _p(V.colptr), _p(V.rowidx), _p(V.val), _p(V.rowptr),
                       _p(V.colidx), _p(V.rval), _p(W), _p(F), seed, sweep0, sweeps,
                       ctypes.byref(cF), ctypes.byref(cW), threads,
                       _p(kl) if trace else None, ctypes.byref(st))
    return FitResult(W, F, kl[:sweeps], st.as_dict())


def foldin(V, W, F0, seed, rel_tol=1e-5, max_sweeps=100, c: Cfg | None = None):
    """F (r x m) for the documents (columns) of V under fixed W; returns (F, sweeps per doc)."""
    c = c or cfg()
    W = _f64(W)
    F = _f64(F0).copy()
    r = W.shape[0]
    done = np.zeros(max(V.m, 1), dtype=np.int32)
    _load().oracle_foldin(V.n, V.m, r, _p(V.colptr), _p(V.rowidx), _p(V.val), _p(W), _p(F), seed,
                          rel_tol, max_sweeps, ctypes.byref(c), _p(done))
    return F, done[:V.m]
