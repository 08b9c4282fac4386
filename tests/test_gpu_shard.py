"""The sharded half on the GPU (Eq. 3: the subproblems of a half are
independent). Two contexts on one GPU stand in for two ranks, run one after
the other: each sweeps its nonzero-balanced unit range (nmfkl_sweep_range),
the updated unit-major rows are exchanged through the contexts' factor views
(the all-gather of shard.exchange_units, done here by copies), and the result
equals the unsharded step bit for bit; Eq. 1 assembled from the ranks' data
terms and the linear term equals the unsharded objective to FP64 rounding."""
import numpy as np
import pytest

import paper_1604_04026_gb300 as nk
from paper_1604_04026_gb300 import shard, synth

from _util import model, params, start

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def docs():
    return synth.docs(3000, 2000, 20, seed=3, threads=8)


def _exchange(torch, views, parts):
    for k, vk in enumerate(views):
        for j, vj in enumerate(views):
            if j != k:
                lo, hi = parts[j]
                vk[lo:hi] = vj[lo:hi]
    torch.cuda.synchronize()


@pytest.mark.parametrize("list_mode", [0, 1, 2])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_step_equals_unsharded(docs, list_mode, world):
    import torch
    V, r = docs, 16
    W0, F0 = start(V, r, seed=5)
    p = params(r, seed=7, list_mode=list_mode)
    ref = model(V, W0, F0, p)
    kls_ref = [ref.step(s) for s in range(2)]
    Wr, Fr = ref.get_W(), ref.get_F()
    ref.close()
    parts = [shard.partition(V.colptr, world), shard.partition(V.rowptr, world)]
    ranks = [model(V, W0, F0, p) for _ in range(world)]
    for s in range(2):
        for k, m in enumerate(ranks):
            m.sweep_range(0, s, *parts[0][k])
        _exchange(torch, [m.factor_unit_major(0) for m in ranks], parts[0])
        data = [m.sweep_range(1, s, *parts[1][k]) for k, m in enumerate(ranks)]
        _exchange(torch, [m.factor_unit_major(1) for m in ranks], parts[1])
        kl = sum(data) + ranks[0].linear_term()
        assert kl == pytest.approx(kls_ref[s], rel=1e-11)
    for m in ranks:
        assert np.array_equal(m.get_W(), Wr) and np.array_equal(m.get_F(), Fr)
        m.close()


def test_full_range_equals_half_and_validation(docs):
    V, r = docs, 12
    W0, F0 = start(V, r, seed=1)
    a, b = model(V, W0, F0, params(r)), model(V, W0, F0, params(r))
    a.sweep_F(3)
    assert b.sweep_range(0, 3, 0, V.m) == 0.0
    assert np.array_equal(a.get_F(), b.get_F())
    # an empty range leaves everything as it was
    F1 = b.get_F()
    b.sweep_range(0, 4, 5, 5)
    assert np.array_equal(b.get_F(), F1)
    for bad in ((0, 0, -1, 3), (0, 0, 5, 4), (0, 0, 0, V.m + 1), (1, 0, 0, V.n + 1), (2, 0, 0, 1)):
        with pytest.raises(nk.NMFKLError, match="EINVAL"):
            b.sweep_range(*bad)
    view = b.factor_unit_major(1)
    assert tuple(view.shape) == (V.n, (r + 3) // 4 * 4)
    assert np.array_equal(view[:, :r].cpu().numpy().T, b.get_W())
    a.close()
    b.close()
