"""Sharded halves on CPU (torch.distributed gloo, world size 2): each rank
solves the subproblems of its nonzero-balanced unit range (Eq. 3: they are
independent), the unit-major blocks are all-gathered, and the assembled half
equals the unsharded one bit for bit (the coordinate orders are keyed by the
global unit id). The per-unit solver here is the FP64 oracle's Algorithm 2;
on the GPU the same partition and gather wrap the CUDA half. A whole sharded
step (shard.sharded_step: both halves, both all-gathers and the all-reduced
objective) runs here over a model whose per-unit solver is the oracle's."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1604_04026_gb300 import shard, synth


def test_partition_covers_and_balances():
    rng = np.random.default_rng(0)
    for units, world in [(0, 2), (1, 3), (10, 2), (1000, 4), (1000, 7)]:
        lens = rng.integers(0, 50, size=units)
        ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        parts = shard.partition(ptr, world)
        assert len(parts) == world and parts[0][0] == 0 and parts[-1][1] == units
        for (a, b), (c, d) in zip(parts, parts[1:]):
            assert b == c and a <= b
        if units:
            nnz = ptr[-1]
            for a, b in parts:
                # a range misses its share by less than one unit's nonzeros
                assert abs((ptr[b] - ptr[a]) - nnz / world) <= lens.max() + nnz / world


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, side, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        V = synth.poisson_lowrank(300, 240, 4, density=0.05, seed=3)
        r, seed, sweep = 6, 17, 2
        W0 = synth.uniform_init(r, V.n, 1, 0).astype(np.float64)
        F0 = synth.uniform_init(r, V.m, 1, 1).astype(np.float64)
        if side == 0:
            ptr, idx, val, A_of, X0, sumA = V.colptr, V.rowidx, V.val, W0, F0, oracle.rowsum(W0)
        else:
            ptr, idx, val, A_of, X0, sumA = V.rowptr, V.colidx, V.rval, F0, W0, oracle.rowsum(F0)
        parts = shard.partition(ptr, world)
        lo, hi = parts[rank]
        block = np.zeros((hi - lo, r))
        for u in range(lo, hi):
            a, b = ptr[u], ptr[u + 1]
            ids = oracle.perm(seed, sweep, side, u, r)
            x, _ = oracle.alg2(val[a:b], A_of[:, idx[a:b]].T, sumA, X0[:, u], ids)
            block[u - lo] = x
        full = shard.gather_units(torch.from_numpy(block), parts, rank).numpy().T
        if side == 0:
            ref, _ = oracle.half_F(V, W0, F0, seed, sweep)
        else:
            ref, _ = oracle.half_W(V, W0, F0, seed, sweep)
        q.put((rank, bool(np.array_equal(full, ref)), (hi - lo)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("side", [0, 1])
def test_sharded_half_equals_unsharded_gloo(side):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, side, q)) for k in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    results = sorted(q.get(timeout=5) for _ in procs)
    assert all(p.exitcode == 0 for p in procs)
    assert [r[0] for r in results] == [0, 1]
    assert all(r[1] for r in results), results
    assert all(r[2] > 0 for r in results)


class _OracleModel:
    """The interface shard.sharded_step drives (sweep_range, factor_unit_major,
    linear_term), with the FP64 oracle's Algorithm 2 per unit and the factors
    held unit-major in torch tensors (CPU)."""

    def __init__(self, V, W0, F0, seed, eps_div=1e-6):
        import torch
        self.V, self.seed, self.eps = V, seed, eps_div
        self.Wt = torch.from_numpy(np.ascontiguousarray(W0.T))  # n x r
        self.Ft = torch.from_numpy(np.ascontiguousarray(F0.T))  # m x r

    def factor_unit_major(self, side):
        return self.Ft if side == 0 else self.Wt

    def sweep_range(self, side, sweep, lo, hi):
        V = self.V
        W, F = self.Wt.numpy().T, self.Ft.numpy().T
        if side == 0:
            ptr, idx, val, A_of, X, sumA = V.colptr, V.rowidx, V.val, W, self.Ft.numpy(), oracle.rowsum(W)
        else:
            ptr, idx, val, A_of, X, sumA = V.rowptr, V.colidx, V.rval, F, self.Wt.numpy(), oracle.rowsum(F)
        r = X.shape[1]
        data = 0.0
        for u in range(lo, hi):
            a, b = ptr[u], ptr[u + 1]
            ids = oracle.perm(self.seed, sweep, side, u, r)
            A = A_of[:, idx[a:b]].T
            x, _ = oracle.alg2(val[a:b], A, sumA, X[u].copy(), ids)
            X[u] = x
            if side == 1:
                v = val[a:b].astype(np.float64)
                data += float(np.sum(v * np.log(v / (A @ x + self.eps)) - v))
        return data

    def linear_term(self):
        return float(self.Wt.numpy().sum(axis=0) @ self.Ft.numpy().sum(axis=0))


def _step_rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        V = synth.poisson_lowrank(200, 160, 4, density=0.06, seed=5)
        r, seed, sweep = 5, 23, 1
        W0 = synth.uniform_init(r, V.n, 2, 0).astype(np.float64)
        F0 = synth.uniform_init(r, V.m, 2, 1).astype(np.float64)
        parts = [shard.partition(V.colptr, world), shard.partition(V.rowptr, world)]
        m = _OracleModel(V, W0, F0, seed)
        kl = shard.sharded_step(m, sweep, parts, rank)
        F1, _ = oracle.half_F(V, W0, F0, seed, sweep)
        W1, _ = oracle.half_W(V, W0, F1, seed, sweep)
        ref_kl, _ = oracle.objective(V, W1, F1)
        same = bool(np.array_equal(m.Ft.numpy().T, F1) and np.array_equal(m.Wt.numpy().T, W1))
        q.put((rank, same, abs(kl - ref_kl) / ref_kl))
    finally:
        dist.destroy_process_group()


def test_sharded_step_gloo():
    """The whole sharded step on two gloo ranks: W and F equal the unsharded
    oracle step bit for bit, Eq. 1 to FP64 rounding."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_step_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    results = sorted(q.get(timeout=5) for _ in procs)
    assert all(p.exitcode == 0 for p in procs)
    assert all(r[1] for r in results), results
    assert all(r[2] < 1e-12 for r in results), results
