"""Serving loop (nmfkl_server_*): requests submitted together run in merged
fold-in batches and concurrent factorizations, and every result is
bit-identical to the same request run alone (nmfkl_foldin / nmfkl_fit on a
context of its own). Also memory admission and queue limits."""
import time

import numpy as np
import pytest

import paper_1604_04026_gb300 as nk
from paper_1604_04026_gb300 import synth

from _util import params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def model():
    topics, V = synth.foldin_docs(3000, 1200, 16, cap=1500, seed=3, threads=8)
    return topics, V


def _subset(V, cols):
    cols = np.asarray(cols)
    lens = np.diff(V.colptr)[cols]
    colptr = np.zeros(len(cols) + 1, dtype=np.int64)
    colptr[1:] = np.cumsum(lens)
    rowidx = np.concatenate([V.rowidx[V.colptr[j]:V.colptr[j + 1]] for j in cols]).astype(np.int32)
    val = np.concatenate([V.val[V.colptr[j]:V.colptr[j + 1]] for j in cols]).astype(np.float32)
    return synth.from_csc(V.n, len(cols), colptr, rowidx, val)


def _fold_alone(W, p, Vq, rel_tol, max_sweeps):
    with nk.NMFKL(W.shape[1], 1, params=p) as m:
        m.init(W, np.zeros((W.shape[0], 1), dtype=np.float32))
        return m.foldin(Vq, rel_tol=rel_tol, max_sweeps=max_sweeps)


def _fit_alone(p, Vq, r, seed, rel_tol, max_sweeps):
    pp = nk.default_params(r, seed=seed)
    for f in ("alpha_W", "beta_W", "alpha_F", "beta_F", "eps_grad", "eps_div", "eps_x", "max_inner",
              "grad_mode", "break_mode", "perm_mode"):
        setattr(pp, f, getattr(p, f))
    with nk.NMFKL(Vq.n, Vq.m, params=pp) as m:
        m.set_data(Vq)
        m.init()
        trace, done = m.fit(max_sweeps, rel_tol)
        return m.get_F(), m.get_W(), done, trace[done - 1]


def test_mixed_requests_match_alone(model):
    W, V = model
    r = W.shape[0]
    p = params(r, seed=5)
    rng = np.random.default_rng(0)
    fold_sets = []
    start = 0
    for size in (1, 40, 300, 7, 120, 500, 2):
        fold_sets.append(np.arange(start, start + size))
        start += size
    fits = [(synth.poisson_lowrank(400, 700, 5, density=0.02, seed=11), 6, 101),
            (synth.poisson_lowrank(900, 500, 8, density=0.01, seed=12), 10, 102)]
    with nk.Server(W, params=p, slots=3) as srv:
        tickets = []
        order = list(range(len(fold_sets) + len(fits)))
        rng.shuffle(order)
        for i in order:
            if i < len(fold_sets):
                tickets.append(("fold", i, srv.submit_foldin(_subset(V, fold_sets[i]), rel_tol=1e-5, max_sweeps=80)))
            else:
                Vq, rq, seed = fits[i - len(fold_sets)]
                tickets.append(("fit", i, srv.submit_fit(Vq, rq, seed=seed, rel_tol=1e-4, max_sweeps=12)))
        for _, _, t in tickets:
            srv.wait(t)
            assert t.status == "OK"
        stats = srv.stats()
    assert stats["pending"] == 0 and stats["mem_in_use"] == 0
    for kind, i, t in tickets:
        if kind == "fold":
            F, s, o = _fold_alone(W, p, _subset(V, fold_sets[i]), 1e-5, 80)
            assert np.array_equal(t.F, F) and np.array_equal(t.sweeps, s) and np.array_equal(t.obj, o), i
        else:
            Vq, rq, seed = fits[i - len(fold_sets)]
            F, Wf, done, kl = _fit_alone(p, Vq, rq, seed, 1e-4, 12)
            assert np.array_equal(t.F, F) and np.array_equal(t.W, Wf), i
            assert t.sweeps[0] == done and t.obj[0] == kl


def test_requests_arriving_during_work_are_batched(model):
    W, V = model
    r = W.shape[0]
    p = params(r, seed=6)
    with nk.Server(W, params=p, slots=1) as srv:
        # a factorization occupies the only slot while fold-in requests queue up behind it
        big = synth.poisson_lowrank(3000, 3000, 8, density=0.02, seed=1)
        t0 = srv.submit_fit(big, 16, seed=1, rel_tol=0.0, max_sweeps=100)
        ts = [srv.submit_foldin(_subset(V, np.arange(10 * i, 10 * i + 10))) for i in range(20)]
        for t in [t0] + ts:
            srv.wait(t)
            assert t.status == "OK"
        stats = srv.stats()
    # the queued fold-in requests ran merged, in fewer batches than requests
    assert stats["batches"] < 20 and stats["batched_requests"] == 20
    assert max(t.batch_requests for t in ts) > 1


def test_admission_limits_and_bad_requests(model):
    W, V = model
    r = W.shape[0]
    p = params(r, seed=7)
    with nk.Server(W, params=p, slots=1, mem_budget=64 << 20, max_pending=2) as srv:
        # 200,000 x 200,000 with r = 100: the factors alone are above the 64 MiB budget
        huge = synth.from_csc(200_000, 200_000, np.concatenate([[0], np.ones(200_000, dtype=np.int64)]).cumsum(),
                              np.arange(200_000, dtype=np.int32), np.ones(200_000, dtype=np.float32))
        with pytest.raises(nk.NMFKLError) as e:
            srv.submit_fit(huge, 100)
        assert e.value.status_name == "EINVAL"
        # a long factorization holds the only slot
        busy_fit = srv.submit_fit(synth.poisson_lowrank(3000, 3000, 8, density=0.02, seed=1), 16, seed=1,
                                  rel_tol=0.0, max_sweeps=400)
        time.sleep(0.1)
        # a malformed column (zero value) fails its own request only
        bad = _subset(V, np.arange(0, 5))
        bad.val[0] = 0.0
        good = _subset(V, np.arange(5, 10))
        tb = srv.submit_foldin(bad)
        tg = srv.submit_foldin(good, rel_tol=1e-6)   # other settings: not merged with the bad one
        # the queue holds max_pending = 2 requests: the next one is refused for now
        with pytest.raises(nk.NMFKLError) as e:
            srv.submit_foldin(_subset(V, np.arange(20, 21)))
        assert e.value.status_name == "EBUSY"
        for t in (busy_fit, tb, tg):
            srv.wait(t)
        assert busy_fit.status == "OK" and tb.status == "EINVAL" and tg.status == "OK"
        F, s, o = _fold_alone(W, p, good, 1e-6, 100)
        assert np.array_equal(tg.F, F)


def test_cancel_withdraws_only_queued_requests(model):
    W, V = model
    r = W.shape[0]
    p = params(r, seed=8)
    with nk.Server(W, params=p, slots=1) as srv:
        # a long factorization (a second or more) holds the only slot; fold-in
        # requests wait behind it
        busy = srv.submit_fit(synth.poisson_lowrank(6000, 6000, 8, density=0.02, seed=1), 16, seed=1,
                              rel_tol=0.0, max_sweeps=3000)
        time.sleep(0.1)
        ts = [srv.submit_foldin(_subset(V, np.arange(10 * i, 10 * i + 10)), rel_tol=1e-6) for i in range(3)]
        assert srv.cancel(ts[1])          # still queued: withdrawn
        assert not srv.cancel(busy)       # running: it completes as usual
        assert srv.stats()["pending"] == 2
        for t in [busy] + ts:
            srv.wait(t)
        assert busy.status == "OK" and ts[0].status == "OK" and ts[2].status == "OK"
        assert ts[1].status == "ECANCELED" and ts[1].message
        assert not ts[1].F.any()          # its outputs were never written
        # the others are what they are alone
        for i in (0, 2):
            F, _, _ = _fold_alone(W, p, _subset(V, np.arange(10 * i, 10 * i + 10)), 1e-6, 100)
            assert np.array_equal(ts[i].F, F)
        # a collected ticket is unknown
        with pytest.raises(nk.NMFKLError) as e:
            srv.cancel(ts[1])
        assert e.value.status_name == "EINVAL"
