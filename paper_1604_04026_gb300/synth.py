"""Seeded synthetic inputs shaped like the paper's sparse count workloads.

The paper evaluates on document/word count and tf-idf matrices (Table 1:
Digits, Reuters21578, TDT2, RCV1_4Class). None of those datasets ships with
this project, so every workload here is synthetic and seeded:

* ``poisson_lowrank`` -- V = mask * Poisson(Wt^T Ft) with Gamma(0.3, 1) factors
  and a Bernoulli mask, the small low-rank count matrix used for parity.
* ``docs`` -- a topic-model corpus: Zipf(1.1) word laws per topic over a
  random permutation of the vocabulary, Dirichlet(0.1) topic weights per
  document, log-normal document lengths (mean 150 tokens, sigma 1.0).
* ``foldin_docs`` -- new documents for fold-in: distinct-word counts drawn
  from Pareto(x_m=5, alpha=1.5) truncated at 5000 by resampling, words drawn
  from the same corpus; also returns the K topic-word distributions.
* ``digits`` -- a dense-ish image set shaped like the paper's Digits (MNIST:
  784 pixels x 60,000 images, ~19% nonzero, intensities 1..255): each image
  a Dirichlet mixture of stroke prototypes on the 28 x 28 grid, cut at the
  density's quantile and quantized.
* ``uniform_init`` -- FP32 Uniform(0, 1) starting factors.

This module only draws random numbers and builds CSC/CSR storage; it holds
none of the factorization arithmetic. Both the CUDA library and the FP64
oracle consume what it produces.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import _build

_lib = None


def _synth_lib():
    global _lib
    if _lib is None:
        path = _build.synth_library_path()
        if not os.path.exists(path):
            _build.build_synth()
        lib = ctypes.CDLL(path)
        vp, i64, i32, f64, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
        lib.synth_docs.restype = vp
        lib.synth_docs.argtypes = [i64, i64, i32, f64, f64, f64, f64, u64, i32]
        lib.synth_docs_distinct.restype = vp
        lib.synth_docs_distinct.argtypes = [i64, i64, i32, f64, f64, vp, u64, i32]
        lib.synth_nnz.restype = i64
        lib.synth_nnz.argtypes = [vp]
        lib.synth_fetch.restype = None
        lib.synth_fetch.argtypes = [vp, vp, vp, vp]
        lib.synth_topics.restype = None
        lib.synth_topics.argtypes = [i64, i32, f64, u64, vp]
        lib.synth_lowrank_means.restype = None
        lib.synth_lowrank_means.argtypes = [i64, i32, vp, vp, vp, vp, vp, i32]
        lib.synth_transpose.restype = None
        lib.synth_transpose.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class CountMatrix:
    """V (n x m) in both CSC (columns = documents) and CSR (rows = words).

    Indices are 0-based int32, offsets int64, values float32 > 0, indices
    sorted within each column (CSC) and row (CSR).
    """
    n: int
    m: int
    colptr: np.ndarray
    rowidx: np.ndarray
    val: np.ndarray
    rowptr: np.ndarray
    colidx: np.ndarray
    rval: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.m), dtype=np.float64)
        cols = np.repeat(np.arange(self.m), np.diff(self.colptr))
        d[self.rowidx, cols] = self.val
        return d

    def col_nnz(self) -> np.ndarray:
        return np.diff(self.colptr)

    def row_nnz(self) -> np.ndarray:
        return np.diff(self.rowptr)


def from_csc(n: int, m: int, colptr, rowidx, val) -> CountMatrix:
    """Builds the CSR twin of a CSC matrix (counting sort, order preserved)."""
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float32)
    nnz = int(colptr[-1])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    colidx = np.empty(nnz, dtype=np.int32)
    rval = np.empty(nnz, dtype=np.float32)
    _synth_lib().synth_transpose(n, m, _ptr(colptr), _ptr(rowidx), _ptr(val),
                                 _ptr(rowptr), _ptr(colidx), _ptr(rval))
    return CountMatrix(n, m, colptr, rowidx, val, rowptr, colidx, rval)


def from_dense(v: np.ndarray) -> CountMatrix:
    """CSC/CSR of the nonzeros of a dense array (column-major scan)."""
    v = np.asarray(v)
    n, m = v.shape
    cols, rows = np.nonzero(v.T)
    colptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=m), out=colptr[1:])
    return from_csc(n, m, colptr, rows.astype(np.int32), v[rows, cols].astype(np.float32))


def poisson_lowrank(n: int, m: int, r: int, shape: float = 0.3, density: float = 0.01,
                    seed: int = 0) -> CountMatrix:
    """V_ij = M_ij * Poisson([Wt^T Ft]_ij), Wt, Ft ~ Gamma(shape, 1), M ~ Bernoulli(density).

    Zeros (masked out or a zero Poisson draw) are dropped, so the realized
    density is below ``density``.
    """
    g = np.random.Generator(np.random.PCG64([seed, 0x5EED01]))
    wt = g.gamma(shape, 1.0, size=(r, n))
    ft = g.gamma(shape, 1.0, size=(r, m))
    mask = g.random((n, m)) < density
    lam = wt.T @ ft
    v = np.where(mask, g.poisson(lam), 0).astype(np.float32)
    return from_dense(v)


def poisson_lowrank_sparse(n: int, m: int, r: int, shape: float = 0.3, density: float = 0.01,
                           seed: int = 0) -> CountMatrix:
    """The law of poisson_lowrank (V_ij = M_ij * Poisson([Wt^T Ft]_ij),
    Gamma(shape, 1) factors) drawn without the dense n x m matrix: per column
    Binomial(n, density) rows drawn uniformly with replacement, duplicates
    merged (so the mask is Bernoulli with a slightly lower rate at high
    density), then the Poisson counts at those entries only (zeros dropped)."""
    g = np.random.Generator(np.random.PCG64([seed, 0x5EED02]))
    wt = g.gamma(shape, 1.0, size=(r, n))
    ft = g.gamma(shape, 1.0, size=(r, m))
    cnt = g.binomial(n, density, size=m)
    cols = np.repeat(np.arange(m, dtype=np.int64), cnt)
    key = np.sort(cols * n + g.integers(0, n, size=cols.size))
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    cols, rows = key // n, key % n
    lam = np.empty(cols.size)
    wtT, ftT = np.ascontiguousarray(wt.T), np.ascontiguousarray(ft.T)
    cols, rows = np.ascontiguousarray(cols), np.ascontiguousarray(rows)
    _synth_lib().synth_lowrank_means(cols.size, r, _ptr(wtT), _ptr(ftT), _ptr(rows), _ptr(cols), _ptr(lam),
                                     min(32, os.cpu_count() or 1))
    v = g.poisson(lam).astype(np.float32)
    keep = v > 0
    cols, rows, v = cols[keep], rows[keep], v[keep]
    colptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=m), out=colptr[1:])
    return from_csc(n, m, colptr, rows.astype(np.int32), v)


def docs(n: int, m: int, K: int, zipf_s: float = 1.1, dir_a: float = 0.1,
         mean_len: float = 150.0, sigma: float = 1.0, seed: int = 0,
         threads: int | None = None) -> CountMatrix:
    """Topic-model corpus (documents are columns); see the module docstring."""
    lib = _synth_lib()
    threads = threads or min(32, os.cpu_count() or 1)
    mu = math.log(mean_len) - 0.5 * sigma * sigma
    h = lib.synth_docs(n, m, K, zipf_s, dir_a, mu, sigma, seed, threads)
    if not h:
        raise ValueError("synth_docs: invalid arguments")
    nnz = lib.synth_nnz(h)
    colptr = np.empty(m + 1, dtype=np.int64)
    rowidx = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float32)
    lib.synth_fetch(h, _ptr(colptr), _ptr(rowidx), _ptr(val))
    return from_csc(n, m, colptr, rowidx, val)


def pareto_distinct(m: int, xm: float = 5.0, alpha: float = 1.5, cap: int = 5000,
                    seed: int = 0) -> np.ndarray:
    """Distinct-word counts ~ Pareto(xm, alpha), resampled until <= cap."""
    g = np.random.Generator(np.random.PCG64([seed, 0x9A2E70]))
    out = np.empty(m, dtype=np.int64)
    todo = np.arange(m)
    while todo.size:
        d = np.floor(xm * (1.0 - g.random(todo.size)) ** (-1.0 / alpha)).astype(np.int64)
        ok = d <= cap
        out[todo[ok]] = d[ok]
        todo = todo[~ok]
    return out.astype(np.int32)


def foldin_docs(n: int, m: int, K: int, zipf_s: float = 1.1, dir_a: float = 0.1,
                xm: float = 5.0, alpha: float = 1.5, cap: int = 5000, seed: int = 0,
                threads: int | None = None):
    """(topics, V): topics is the K x n FP32 topic-word matrix of the corpus,
    V the CSC/CSR of m new documents with Pareto distinct-word counts."""
    lib = _synth_lib()
    threads = threads or min(32, os.cpu_count() or 1)
    distinct = np.minimum(pareto_distinct(m, xm, alpha, cap, seed), n).astype(np.int32)
    h = lib.synth_docs_distinct(n, m, K, zipf_s, dir_a, _ptr(distinct), seed, threads)
    if not h:
        raise ValueError("synth_docs_distinct: invalid arguments")
    nnz = lib.synth_nnz(h)
    colptr = np.empty(m + 1, dtype=np.int64)
    rowidx = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float32)
    lib.synth_fetch(h, _ptr(colptr), _ptr(rowidx), _ptr(val))
    topics = np.empty((K, n), dtype=np.float32)
    lib.synth_topics(n, K, zipf_s, seed, _ptr(topics))
    return topics, from_csc(n, m, colptr, rowidx, val)


def digits(m: int = 60_000, K: int = 30, density: float = 0.19, alpha: float = 0.3, seed: int = 0,
           side: int = 28, chunk: int = 8192) -> CountMatrix:
    """Images as columns of a (side*side) x m count matrix, MNIST-shaped.

    K prototypes, each the sum of three isotropic Gaussian blobs (sigma 1.5 to
    3 pixels) centred uniformly in the middle 20 x 20 pixels; image j =
    sum_k theta_jk P_k with theta_j ~ Dirichlet(alpha 1_K), scaled to a peak of
    1; pixels at or below the (1 - density) quantile c of the intensities are
    dropped and a kept intensity t maps to round(255 (t - c) / (1 - c)), at
    least 1 (soft stroke edges, as in anti-aliased digits). Seeded; the
    realized density is `density` up to sampling of the quantile."""
    g = np.random.Generator(np.random.PCG64([seed, 0xD161]))
    n = side * side
    yy, xx = np.mgrid[0:side, 0:side]
    P = np.zeros((K, n))
    for k in range(K):
        for _ in range(3):
            cy, cx = g.uniform(4, side - 4, size=2)
            s = g.uniform(1.5, 3.0)
            P[k] += np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * s * s)).ravel()
    theta = g.dirichlet(alpha * np.ones(K), size=m)  # m x K
    # the threshold: the (1 - density) quantile over a sample of images
    samp = theta[: min(m, 4096)] @ P
    samp /= samp.max(axis=1, keepdims=True)
    cut = float(np.quantile(samp, 1.0 - density))
    cols, rows, vals = [], [], []
    for j0 in range(0, m, chunk):
        img = theta[j0:j0 + chunk] @ P  # images x n
        img /= img.max(axis=1, keepdims=True)
        jj, ii = np.nonzero(img > cut)
        cols.append(jj + j0)
        rows.append(ii)
        vals.append(np.maximum(1.0, np.rint(255.0 * (img[jj, ii] - cut) / (1.0 - cut))))
    cols = np.concatenate(cols)
    rows = np.concatenate(rows).astype(np.int32)
    vals = np.concatenate(vals).astype(np.float32)
    colptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=m), out=colptr[1:])
    return from_csc(n, m, colptr, rows, vals)


def uniform_init(r: int, cols: int, seed: int = 0, tag: int = 0) -> np.ndarray:
    """FP32 Uniform[0, 1) matrix of shape (r, cols) (starting W or F)."""
    g = np.random.Generator(np.random.PCG64([seed, 0x1A17, tag]))
    return g.random((r, cols), dtype=np.float32)
