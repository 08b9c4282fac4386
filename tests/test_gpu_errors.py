"""Error paths of the C ABI on the GPU, made on the host side or by a bounded
wait running out (no fault, trap or endless loop is ever provoked).

* ETIMEOUT: the CTAs of a thread-block cluster exchange partial sums through
  distributed shared memory and wait for their peers with a bounded loop. A
  wait limit of one cycle makes those waits give up; the half must return
  ETIMEOUT (not hang), and the context must stay usable: with the default
  limit restored the same half matches the FP64 oracle.
* ENUMERIC: a NaN planted in the starting factors reaches a factor entry or
  the objective; the sweep or step that meets it must say so.
"""
import numpy as np
import pytest

import oracle
import paper_1604_04026_gb300 as nk
from paper_1604_04026_gb300 import synth

from _util import PROBE_FACTOR, TIGHT, assert_parity, cfg_for, fp32_sensitivity, model, params, start

pytestmark = pytest.mark.gpu


def _long_rows(seed=4):
    """64 rows; the first six hold 20k..99k nonzeros, so the W half runs the
    cluster kernels of both plans."""
    rng = np.random.default_rng(seed)
    n, m = 64, 100_000
    lens = [20_000, 30_000, 45_000, 60_000, 80_000, 99_000]
    rows, cols = [], []
    for i, L in enumerate(lens):
        rows.append(np.full(L, i))
        cols.append(np.sort(rng.choice(m, size=L, replace=False)))
    extra = rng.integers(0, m, size=2 * m)
    rows.append(rng.integers(len(lens), n, size=extra.size))
    cols.append(extra)
    R = np.concatenate(rows)
    C = np.concatenate(cols)
    key = np.unique(C.astype(np.int64) * n + R)
    C, R = key // n, key % n
    colptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(C, minlength=m), out=colptr[1:])
    return synth.from_csc(n, m, colptr, R.astype(np.int32), rng.integers(1, 6, size=R.size).astype(np.float32))


@pytest.mark.parametrize("list_mode", [1, 2])
def test_cluster_wait_limit_gives_etimeout_then_recovers(list_mode):
    V = _long_rows()
    r = 12
    W0, F0 = start(V, r, seed=3)
    p = params(r, seed=8, list_mode=list_mode, **TIGHT)
    m = model(V, W0, F0, p)
    kinds = {b["kernel"] for b in m.plan() if b["side"] == 1 and b["list_plan"] == (list_mode == 2)}
    assert any("cluster" in k for k in kinds), kinds
    m.set_wait_limit(1)
    with pytest.raises(nk.NMFKLError) as e:
        m.sweep_W(0)
    assert e.value.status_name == "ETIMEOUT"
    # the context is still usable: restore the default limit and the start
    m.set_wait_limit(0)
    m.init(W0, F0)
    m.sweep_W(0)
    Wg = m.get_W()
    m.close()
    Wo, _ = oracle.half_W(V, W0, F0, 8, 0, cfg_for(p, 1), threads=8)
    dev, _ = fp32_sensitivity(V, W0, F0, 1, p, Wo)
    assert_parity("after_timeout/lm%d/W" % list_mode, Wg, Wo, slack=PROBE_FACTOR * dev)


def test_wait_limit_rejects_negative():
    V = synth.poisson_lowrank(50, 40, 2, density=0.3, seed=0)
    with nk.NMFKL(V.n, V.m, params=params(4)) as m:
        with pytest.raises(nk.NMFKLError, match="EINVAL"):
            m.set_wait_limit(-1)


@pytest.mark.parametrize("list_mode", [1, 2])
def test_nan_in_start_is_reported(list_mode):
    V = synth.docs(3000, 2000, 20, seed=3, threads=8)
    r = 16
    W0, F0 = start(V, r, seed=5)
    p = params(r, seed=2, list_mode=list_mode)
    # a NaN in F: the F half writes it back (Algorithm 2 cannot move it) and reports it
    Fbad = F0.copy()
    Fbad[3, 7] = np.nan
    m = model(V, W0, Fbad, p)
    with pytest.raises(nk.NMFKLError) as e:
        m.sweep_F(0)
    assert e.value.status_name == "ENUMERIC"
    # a NaN in W: the step (both halves and the objective) reports it
    Wbad = W0.copy()
    Wbad[5, int(V.rowidx[0])] = np.nan
    m.init(Wbad, F0)
    with pytest.raises(nk.NMFKLError) as e:
        m.step(0)
    assert e.value.status_name == "ENUMERIC"
    # and Algorithm 1 stops at the first sweep that meets it
    m.init(Wbad, F0)
    with pytest.raises(nk.NMFKLError) as e:
        m.fit(3)
    assert e.value.status_name == "ENUMERIC"
    # a clean start on the same context runs
    m.init(W0, F0)
    assert np.isfinite(m.step(0))
    m.close()
