"""The seeded synthetic inputs follow the recipe the workloads are stated in:
CSC and CSR hold the same matrix, documents are topic mixtures with
log-normal lengths and Zipf word laws, fold-in documents have Pareto
distinct-word counts, and every draw is reproducible from its seed."""
import numpy as np
import pytest

from paper_1604_04026_gb300 import synth


def _dense_from_csr(V):
    d = np.zeros((V.n, V.m), dtype=np.float64)
    rows = np.repeat(np.arange(V.n), np.diff(V.rowptr))
    d[rows, V.colidx] = V.rval
    return d


def _strictly_sorted(ptr, idx):
    for u in range(ptr.size - 1):
        seg = idx[ptr[u]:ptr[u + 1]]
        if seg.size > 1 and not np.all(np.diff(seg) > 0):
            return False
    return True


@pytest.fixture(scope="module")
def corpus():
    return synth.docs(2000, 3000, 10, seed=1, threads=4)


def test_csc_and_csr_hold_the_same_counts(corpus):
    V = corpus
    assert np.array_equal(V.dense(), _dense_from_csr(V))
    assert _strictly_sorted(V.colptr, V.rowidx) and _strictly_sorted(V.rowptr, V.colidx)
    assert V.colptr[0] == 0 and V.colptr[-1] == V.nnz == V.rowptr[-1]
    assert (V.val > 0).all() and np.array_equal(V.val, np.round(V.val))  # token counts


def test_documents_have_lognormal_lengths_and_at_least_one_token(corpus):
    V = corpus
    tokens = np.add.reduceat(V.val.astype(np.float64), V.colptr[:-1])
    assert (np.diff(V.colptr) >= 1).all()
    # LogNormal(ln 150 - 1/2, 1): mean 150, median 150 / e^(1/2)
    assert abs(tokens.mean() / 150.0 - 1.0) < 0.15
    assert abs(np.median(tokens) / (150.0 * np.exp(-0.5)) - 1.0) < 0.2


def test_word_frequencies_have_a_zipf_head(corpus):
    # the 1% most frequent words (20 of 2,000) occur in several times their share
    # of the (word, document) pairs, and the longest row is ~10x the median
    rows = np.sort(corpus.row_nnz())[::-1]
    assert rows[:20].sum() > 5 * 0.01 * rows.sum()
    assert rows[0] > 8 * np.median(rows)


def test_draws_are_reproducible_from_the_seed():
    a = synth.docs(500, 400, 5, seed=7, threads=2)
    b = synth.docs(500, 400, 5, seed=7, threads=2)
    c = synth.docs(500, 400, 5, seed=8, threads=2)
    assert np.array_equal(a.colptr, b.colptr) and np.array_equal(a.rowidx, b.rowidx) and np.array_equal(a.val, b.val)
    assert not (np.array_equal(a.colptr, c.colptr) and np.array_equal(a.rowidx, c.rowidx))
    # the corpus does not depend on how many host threads draw it
    t = synth.docs(500, 400, 5, seed=7, threads=1)
    assert np.array_equal(a.colptr, t.colptr) and np.array_equal(a.rowidx, t.rowidx) and np.array_equal(a.val, t.val)
    p = synth.poisson_lowrank(80, 60, 3, density=0.2, seed=4)
    q = synth.poisson_lowrank(80, 60, 3, density=0.2, seed=4)
    assert np.array_equal(p.dense(), q.dense())


def test_poisson_lowrank_counts_and_density():
    V = synth.poisson_lowrank(400, 300, 5, density=0.05, seed=2)
    assert np.array_equal(V.val, np.round(V.val)) and (V.val >= 1).all()
    # zeros dropped: realized density at most the mask density (and not far below it
    # for Gamma(0.3, 1) factors at rank 5)
    dens = V.nnz / (400 * 300)
    assert 0.005 < dens <= 0.05 * 1.1


def test_pareto_distinct_word_counts():
    d = synth.pareto_distinct(200_000, seed=3)
    assert d.min() >= 5 and d.max() <= 5000
    # Pareto(5, 1.5): mean 15 before truncation, floor() and the cap take a little off
    assert 12.5 < d.mean() < 15.5


def test_foldin_topics_are_zipf_laws():
    topics, V = synth.foldin_docs(3000, 200, 4, seed=5, threads=2)
    assert np.allclose(topics.sum(axis=1), 1.0, atol=1e-4)
    for t in topics:
        s = np.sort(t)[::-1]
        assert abs(s[0] / s[1] - 2.0 ** 1.1) < 0.05  # p(k) proportional to k^-1.1
    assert V.m == 200 and (np.diff(V.colptr) >= 1).all()


def test_digits_shape_density_and_values():
    """The Digits-like set: 784 x m, ~19% nonzero, integer intensities in
    [1, 255], both layouts agree, and the draw is reproducible."""
    V = synth.digits(m=3000, seed=4)
    assert (V.n, V.m) == (784, 3000)
    assert abs(V.nnz / (V.n * V.m) - 0.19) < 0.01
    assert V.val.min() >= 1 and V.val.max() <= 255 and np.all(V.val == np.rint(V.val))
    assert V.val.min() < 20  # soft stroke edges reach low intensities
    assert np.array_equal(np.sort(V.rval), np.sort(V.val))
    W = synth.digits(m=3000, seed=4)
    assert np.array_equal(V.rowidx, W.rowidx) and np.array_equal(V.val, W.val)
