"""Launch plans on the GPU: the captured step graph, the per-class kernel
choice of the list plan, and the autotuner.

* The step (F half, W half, objective) replays as one CUDA graph; with kernel
  timing on, the same launches are issued one by one. Both give the same W,
  F and objective bit for bit, step after step.
* Units of at most 256 nonzeros have two kernels in the list plan (dense tile
  or sub-warp groups over the compressed rows); the group kernels meet the
  same tight-mode parity bar against the FP64 oracle.
* The autotuner measures both kernels per class from the current state,
  leaves W and F as they were, applies the faster ones, and caches them: a
  second call with the same cache applies the stored choice without
  measuring.
"""
import json

import numpy as np
import pytest

import paper_1604_04026_gb300 as nk
from paper_1604_04026_gb300 import synth

from _util import TIGHT, model, params, start

pytestmark = pytest.mark.gpu

ALL_GROUP = [[1, 1, 1, 1], [1, 1, 1, 1]]


@pytest.fixture(scope="module")
def docs():
    return synth.docs(3000, 2000, 20, seed=3, threads=8)


@pytest.mark.parametrize("list_mode", [0, 1, 2])
def test_graph_replay_equals_eager_launches(docs, list_mode):
    V, r = docs, 20
    W0, F0 = start(V, r, seed=2)
    out = []
    for timing in (False, True):
        m = model(V, W0, F0, params(r, seed=3, list_mode=list_mode))
        m.set_timing(timing)
        kls = [m.step(s) for s in range(4)]
        out.append((kls, m.get_W(), m.get_F()))
        m.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_plan_choice_round_trip_and_validation(docs):
    m = model(docs, *start(docs, 8, seed=1), params(8))
    pc = m.plan_choice()
    assert pc["list_threshold"] == 0.5 and pc["short_kernel"] == [[0] * 4, [0] * 4]
    m.set_plan_choice(list_threshold=0.3, short_kernel=[[1, 0, 1, 0], [0, 1, 0, 1]])
    assert m.plan_choice() == {"list_threshold": 0.3, "short_kernel": [[1, 0, 1, 0], [0, 1, 0, 1]]}
    for bad in (dict(list_threshold=1.5), dict(short_kernel=[[2, 0, 0, 0], [0, 0, 0, 0]])):
        with pytest.raises(nk.NMFKLError, match="EINVAL"):
            m.set_plan_choice(**bad)
    assert m.plan_choice()["list_threshold"] == 0.3
    m.close()


def test_group_kernels_run_when_chosen(docs):
    V, r = docs, 16
    m = model(V, *start(V, r, seed=2), params(r, seed=5, list_mode=2))
    m.set_plan_choice(short_kernel=ALL_GROUP)
    m.step(0)
    ran = {b["kernel"] for b in m.plan() if b["ran_last"]}
    assert any(k.startswith("group_") for k in ran), ran
    assert not any(k.startswith("sweep_warp_k") and b["list_plan"] for b in m.plan() if b["ran_last"]
                   for k in [b["kernel"]]), ran
    m.close()


def test_autotune_applies_caches_and_leaves_state(docs, tmp_path):
    V, r = docs, 16
    W0, F0 = start(V, r, seed=4)
    cache = str(tmp_path / "tune.jsonl")
    m = model(V, W0, F0, params(r, seed=6))
    for s in range(3):
        m.step(s)
    W1, F1 = m.get_W(), m.get_F()
    res = m.autotune(sweep=3, reps=1, cache_path=cache)
    assert not res["from_cache"]
    assert np.array_equal(m.get_W(), W1) and np.array_equal(m.get_F(), F1)
    assert m.plan_choice()["short_kernel"] == res["short_kernel"]
    times = [t for side in res["ms"] for cls in side for t in cls]
    assert any(t > 0 for t in times)
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and json.loads(lines[0])["short_kernel"] == res["short_kernel"]
    # the same configuration again: taken from the cache, nothing appended
    res2 = m.autotune(sweep=3, reps=1, cache_path=cache)
    assert res2["from_cache"] and res2["short_kernel"] == res["short_kernel"]
    assert len(open(cache).read().strip().splitlines()) == 1
    # a tuned context steps like any other: the same result as one set by hand
    kl_a = m.step(3)
    m.close()
    m2 = model(V, W1, F1, params(r, seed=6))
    m2.set_plan_choice(short_kernel=res["short_kernel"])
    assert m2.step(3) == kl_a
    m2.close()


def test_metrics_one_line_per_step(docs, tmp_path):
    V, r = docs, 12
    W0, F0 = start(V, r, seed=2)
    path = str(tmp_path / "metrics.jsonl")
    m = model(V, W0, F0, params(r, seed=3))
    m.set_metrics(path)
    kls = [m.step(s) for s in range(3)]
    W, F = m.get_W(), m.get_F()
    m.set_metrics(None)
    m.step(3)  # not recorded
    lines = [json.loads(x) for x in open(path).read().splitlines()]
    assert [x["sweep"] for x in lines] == [0, 1, 2]
    assert [x["kl"] for x in lines] == kls
    last = lines[-1]
    assert last["zeros_W_pct"] == pytest.approx(100.0 * (W == 0).mean(), rel=1e-5, abs=1e-9)
    assert last["zeros_F_pct"] == pytest.approx(100.0 * (F == 0).mean(), rel=1e-5, abs=1e-9)
    for x in lines:
        assert x["ms"] > 0 and x["updates_per_s"] == pytest.approx(2 * V.nnz * r / (x["ms"] / 1e3), rel=1e-4)
        assert x["evals_per_coord"] >= 1.0 and 0.0 <= x["steps_per_coord"] <= x["evals_per_coord"]
        assert x["plan"][0] in ("dense", "list") and x["plan"][1] in ("dense", "list")
    # fit: one line per sweep it ran
    m.set_metrics(path)
    trace = m.fit(sweep0=4, max_sweeps=2, rel_tol=0.0)
    m.close()
    lines = [json.loads(x) for x in open(path).read().splitlines()]
    assert [x["sweep"] for x in lines[3:]] == [4, 5]
