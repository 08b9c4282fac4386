"""Fold-in (Algorithm 1's F half alone under a fixed W, each new column run to
its own stopping point) through the C ABI, against the FP64 oracle's
fold-in on the same seeded inputs.

Bars:
  * one pass from the same start in tight mode: every entry within 1e-4
    relative + 1e-6 x the column's largest entry + 4 x its FP32 sensitivity
    (Monte Carlo arithmetic probes of the oracle), as for the F half;
  * the full fold-in at the paper's constants and rel_tol 1e-5: every
    column's objective (Eq. kl, recomputed in FP64 from the returned F)
    within 1e-4 relative of the oracle's, and the reported objective within
    1e-5 of that recomputation;
  * the three launch schemes, graph replays, and a column submitted alone or
    inside a larger batch: bit-identical.
"""
import numpy as np
import pytest

import oracle
import paper_1604_04026_gb300 as nk
from paper_1604_04026_gb300 import synth

from _util import PROBE_FACTOR, TIGHT, assert_parity, cfg_for, fp32_sensitivity, params, unit_objectives

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def corpus():
    """K=20 topic-word laws over n=3000 words and 1500 new documents with
    Pareto(5, 1.5) distinct-word counts capped at 2000 (every length class up
    to the 2048 one)."""
    topics, V = synth.foldin_docs(3000, 1500, 20, cap=2000, seed=7, threads=8)
    return topics, V


def _model(W, p):
    r, n = W.shape
    m = nk.NMFKL(n, 1, params=p)
    m.init(np.ascontiguousarray(W, dtype=np.float32), np.zeros((r, 1), dtype=np.float32))
    return m


def _subset(V, cols):
    cols = np.asarray(cols)
    lens = np.diff(V.colptr)[cols]
    colptr = np.zeros(len(cols) + 1, dtype=np.int64)
    colptr[1:] = np.cumsum(lens)
    rowidx = np.concatenate([V.rowidx[V.colptr[j]:V.colptr[j + 1]] for j in cols]).astype(np.int32)
    val = np.concatenate([V.val[V.colptr[j]:V.colptr[j + 1]] for j in cols]).astype(np.float32)
    return synth.from_csc(V.n, len(cols), colptr, rowidx, val)


def test_one_pass_matches_oracle_tight(corpus):
    W, V = corpus
    r = W.shape[0]
    p = params(r, seed=5, **TIGHT)
    F0 = synth.uniform_init(r, V.m, 11, 1)
    with _model(W, p) as m:
        F, sweeps, obj = m.foldin(V, F0=F0, rel_tol=0.0, max_sweeps=1)
    assert (sweeps == 1).all()
    c = cfg_for(p, 0)
    Fo, done = oracle.foldin(V, W, F0, p.seed, rel_tol=0.0, max_sweeps=1, c=c)
    assert (done == 1).all()
    dev, _ = fp32_sensitivity(V, W, F0, 0, p, Fo)
    assert_parity("foldin_one_pass_tight/F", F, Fo, slack=PROBE_FACTOR * dev)


def test_full_foldin_objective_parity(corpus):
    W, V = corpus
    r = W.shape[0]
    p = params(r, seed=9)
    F0 = synth.uniform_init(r, V.m, 12, 1)
    with _model(W, p) as m:
        F, sweeps, obj = m.foldin(V, F0=F0, rel_tol=1e-5, max_sweeps=200)
    Fo, done = oracle.foldin(V, W, F0, p.seed, rel_tol=1e-5, max_sweeps=200, c=cfg_for(p, 0))
    dg = unit_objectives(V, W, F, 0)
    do = unit_objectives(V, W, Fo, 0)
    rel = np.abs(dg - do) / np.abs(do)
    assert rel.max() <= 1e-4, (rel.max(), int(rel.argmax()))
    # the objective the kernel reports is the one of the F it returns
    rep = np.abs(obj - dg) / np.abs(dg)
    assert rep.max() <= 1e-5, rep.max()
    # the stopping rule is the same; a column whose last relative change sits
    # on the threshold may stop one pass earlier or later in FP32
    same = (sweeps == done).mean()
    assert same >= 0.9, same
    assert (np.abs(sweeps.astype(np.int64) - done) <= 3).mean() >= 0.99
    assert (sweeps >= 1).all() and (F >= 0).all()


def test_launch_schemes_and_graph_replay_bit_identical(corpus):
    W, V = corpus
    r = W.shape[0]
    p = params(r, seed=3)
    F0 = synth.uniform_init(r, V.m, 13, 1)
    F0b = synth.uniform_init(r, V.m, 14, 1)
    with _model(W, p) as m:
        g1 = m.foldin(V, F0=F0, launch_mode=0)
        g2 = m.foldin(V, F0=F0, launch_mode=0)       # replay of the captured graph
        plain = m.foldin(V, F0=F0, launch_mode=1)
        per_doc = m.foldin(V, F0=F0, launch_mode=2)
        gb = m.foldin(V, F0=F0b, launch_mode=0)      # same sizes, new start: replay
        pb = m.foldin(V, F0=F0b, launch_mode=1)
    for other in (g2, plain, per_doc):
        for a, b in zip(g1, other):
            assert np.array_equal(a, b)
    for a, b in zip(gb, pb):
        assert np.array_equal(a, b)
    assert not np.array_equal(g1[0], gb[0])


def test_same_result_alone_and_in_a_batch(corpus):
    W, V = corpus
    r = W.shape[0]
    p = params(r, seed=21)
    A = np.arange(0, 300)
    B = np.arange(700, 1500)
    VA, VAB = _subset(V, A), _subset(V, np.concatenate([B, A]))
    F0 = synth.uniform_init(r, V.m, 15, 1)
    ids_AB = np.concatenate([10_000 + np.arange(len(B)), np.arange(len(A))]).astype(np.int64)
    with _model(W, p) as m:
        FA, sA, oA = m.foldin(VA, F0=F0[:, A])
        FAB, sAB, oAB = m.foldin(VAB, F0=np.concatenate([F0[:, B], F0[:, A]], axis=1), doc_ids=ids_AB)
    k = len(B)
    assert np.array_equal(FA, FAB[:, k:])
    assert np.array_equal(sA, sAB[k:])
    assert np.array_equal(oA, oAB[k:])


def test_device_inputs_match_host(torch, corpus):
    W, V = corpus
    r = W.shape[0]
    p = params(r, seed=4)
    F0 = synth.uniform_init(r, V.m, 16, 1)
    with _model(W, p) as m:
        Fh, sh, oh = m.foldin(V, F0=F0)
        d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        Fd, sd, od = m.foldin(colptr=d(V.colptr), rowidx=d(V.rowidx), val=d(V.val), F0=d(F0))
    assert np.array_equal(Fh, Fd.cpu().numpy())
    assert np.array_equal(sh, sd.cpu().numpy())
    assert np.array_equal(oh, od.cpu().numpy())


def test_random_start_matches_oracle_draw(corpus):
    W, V = corpus
    r = W.shape[0]
    p = params(r, seed=77)
    with _model(W, p) as m:
        F, _, _ = m.foldin(V, max_sweeps=0)
    assert np.array_equal(F.astype(np.float64), oracle.uniform_init(77, 2, r, V.m))


def test_edge_cases(torch):
    rng = np.random.default_rng(0)
    n, r = 9000, 8
    W = rng.random((r, n), dtype=np.float32)
    lens = [0, 1, 8192, 5, 0]
    cols = [np.sort(rng.choice(n, size=L, replace=False)) for L in lens]
    colptr = np.zeros(len(lens) + 1, dtype=np.int64)
    colptr[1:] = np.cumsum(lens)
    rowidx = np.concatenate(cols).astype(np.int32)
    val = rng.integers(1, 5, size=rowidx.size).astype(np.float32)
    V = synth.from_csc(n, len(lens), colptr, rowidx, val)
    p = params(r, seed=1)
    F0 = synth.uniform_init(r, V.m, 2, 1)
    with _model(W, p) as m:
        F, s, o = m.foldin(V, F0=F0, rel_tol=1e-6, max_sweeps=50)
        Fo, done = oracle.foldin(V, W, F0, p.seed, rel_tol=1e-6, max_sweeps=50, c=cfg_for(p, 0))
        # an empty column has no data term: every coordinate goes to 0 in one pass
        assert (F[:, 0] == 0).all() and (F[:, 4] == 0).all()
        dg, do = unit_objectives(V, W, F, 0), unit_objectives(V, W, Fo, 0)
        assert (np.abs(dg - do) <= 1e-4 * np.abs(do) + 1e-9).all(), (dg, do)
        # nothing to do
        F_empty, s_empty, _ = m.foldin(colptr=np.zeros(1, dtype=np.int64), rowidx=np.zeros(0, dtype=np.int32),
                                       val=np.zeros(0, dtype=np.float32))
        assert F_empty.shape == (r, 0) and s_empty.shape == (0,)
        # beyond the longest length class: refused, host and device inputs
        big = np.sort(rng.choice(n, size=8193, replace=False)).astype(np.int32)
        cp = np.array([0, 8193], dtype=np.int64)
        vv = np.ones(8193, dtype=np.float32)
        with pytest.raises(nk.NMFKLError) as e:
            m.foldin(colptr=cp, rowidx=big, val=vv)
        assert e.value.status_name == "EINVAL"
        d = lambda x: torch.from_numpy(x).cuda()
        with pytest.raises(nk.NMFKLError) as e:
            m.foldin(colptr=d(cp), rowidx=d(big), val=d(vv))
        assert e.value.status_name == "EINVAL"
        # still usable after a refusal
        F2, _, _ = m.foldin(V, F0=F0, rel_tol=1e-6, max_sweeps=50)
        assert np.array_equal(F, F2)
