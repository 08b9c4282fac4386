"""Parity at the benchmark's full size: the large document-like corpus (n =
100,000 words, m = 1,000,000 documents, ~126M nnz), r = 100, default
parameters, the kernels and launch plans bench.py times.

Sampled outputs are recomputed one by one by the FP64 oracle's Algorithm 2
from the same state:
  * F half from the Uniform start (drawn by the same Philox rule on both
    sides): sampled columns of every length class, compared per entry;
  * W half from (W0, F1) with F1 the oracle's own full F half (an oracle
    value, computed for all columns): sampled rows, the longest ones included.
Bars as in the paper-constant parity tests: at least 99% of the sampled
entries within 1e-4 relative + 1e-6 x the unit's largest entry + 4 x the
entry's FP32 sensitivity (Monte Carlo arithmetic probes of the oracle), that
slack capped at 10 x the plain bound; the fraction within the plain bar is
reported beside it; and
every sampled unit's subproblem objective within 1e-5 of the magnitude of
its terms (+ 4 x its probe spread).
"""
import numpy as np
import pytest

import oracle
import paper_1604_04026_gb300 as nk
from paper_1604_04026_gb300 import synth

from _util import PROBE_FACTOR, U32, cfg_for, parity_report

pytestmark = pytest.mark.gpu

N, M, K, R, SEED = 100_000, 1_000_000, 100, 100, 0


@pytest.fixture(scope="module")
def large():
    return synth.docs(N, M, K, seed=SEED, threads=16)


def _sample_units(ptr, count, rng):
    """Units of every length class (quantiles), the longest, and random ones."""
    lens = np.diff(ptr)
    order = np.argsort(lens, kind="stable")
    picks = set(order[np.linspace(0, lens.size - 1, count // 2).astype(int)].tolist())
    picks.update(order[-4:].tolist())
    picks.update(rng.choice(lens.size, size=count - len(picks), replace=False).tolist())
    return np.array(sorted(picks))


def _unit_obj(v, A, x, sumA, eps):
    ax = A @ x
    return float(np.sum(v * np.log(v / (ax + eps)) - v) + sumA @ x)


def _unit_scale(v, A, x, sumA, eps):
    ax = A @ x
    return float(np.sum(v * (np.abs(np.log(v / (ax + eps))) + 1.0)) + sumA @ np.abs(x))


def _check_sampled(units, ptr, idx, val, A_full, X0, sumA, got, p, side, name="full_size_sampled"):
    c = cfg_for(p, side)
    G, O, S = [], [], []
    for u in units:
        a, b = ptr[u], ptr[u + 1]
        v = val[a:b].astype(np.float64)
        A = A_full[:, idx[a:b]].T
        ids = oracle.perm(p.seed, 0, side, int(u), R)
        ref, _ = oracle.alg2(v, A, sumA, X0[:, u], ids, c)
        dev = np.zeros(R)
        probe_obj = []
        for s in range(8):
            cp = cfg_for(p, side)
            cp.perturb = U32
            cp.perturb_seed = 1 + s + 1000 * int(u)
            xp, _ = oracle.alg2(v, A, sumA, X0[:, u], ids, cp)
            dev = np.maximum(dev, np.abs(xp - ref))
            probe_obj.append(_unit_obj(v, A, xp, sumA, p.eps_div))
        g = got[:, u].astype(np.float64)
        G.append(g)
        O.append(ref)
        S.append(PROBE_FACTOR * dev)
        d_ref = _unit_obj(v, A, ref, sumA, p.eps_div)
        spread = max(abs(x - d_ref) for x in probe_obj)
        err = abs(_unit_obj(v, A, g, sumA, p.eps_div) - d_ref)
        assert err <= 1e-5 * _unit_scale(v, A, ref, sumA, p.eps_div) + PROBE_FACTOR * spread, (side, int(u), err)
        assert (g >= 0).all()
    # columns are the sampled units; at the paper's constants a break or clamp
    # decision may flip between FP32 and FP64, so the gate is a fraction
    rep = parity_report("%s/%s" % (name, "F" if side == 0 else "W"), np.stack(G, axis=1),
                        np.stack(O, axis=1), slack=np.stack(S, axis=1))
    assert 1.0 - rep["beyond_cap"] / rep["entries"] >= 0.99, rep


def test_full_size_sampled_parity(large):
    V = large
    p = nk.default_params(R, seed=SEED)
    rng = np.random.default_rng(7)
    W0 = oracle.uniform_init(SEED, 0, R, V.n)
    F0 = oracle.uniform_init(SEED, 1, R, V.m)
    sumW = oracle.rowsum(W0)
    with nk.NMFKL(V.n, V.m, params=p) as m:
        m.set_data(V)
        m.init()  # the same Philox draw as W0, F0 above
        assert {b["kernel"] for b in m.plan()}, "no plan"
        m.sweep_F(0)
        F1g = m.get_F()
    cols = _sample_units(V.colptr, 48, rng)
    _check_sampled(cols, V.colptr, V.rowidx, V.val, W0, F0, sumW, F1g, p, 0)

    # W half from (W0, F1), F1 the oracle's F half over every column
    F1, _ = oracle.half_F(V, W0, F0, SEED, 0, cfg_for(p, 0), threads=16)
    with nk.NMFKL(V.n, V.m, params=p) as m:
        m.set_data(V)
        m.init(W0.astype(np.float32), F1.astype(np.float32))
        m.sweep_W(0)
        W1g = m.get_W()
        kinds = {b["kernel"] for b in m.plan() if b["side"] == 1 and b["ran_last"]}
    # the longest rows (~95k nonzeros) run split over clusters (or the giant kernels)
    assert any(k.startswith(("sparse_cluster", "sweep_cluster", "sparse_giant", "sweep_giant")) for k in kinds), kinds
    F1_32 = F1.astype(np.float32).astype(np.float64)
    rows = _sample_units(V.rowptr, 24, rng)
    _check_sampled(rows, V.rowptr, V.colidx, V.rval, F1_32, W0, oracle.rowsum(F1_32), W1g, p, 1)


def test_full_size_sampled_parity_regularized(large):
    """Eq. 2 with a1, a2, b1, b2 > 0 at the benchmark's size: the F half from
    the Uniform start and the W half from the same start (W0, F0), sampled
    columns and rows against the oracle's Algorithm 2 one by one."""
    V = large
    # weights comparable with the linear terms they join: from the Uniform
    # start sumW_k ~ n / 2 = 50,000 (F half) and sumF_k ~ m / 2 = 500,000
    # (W half); beta is a tenth of that, alpha x about as much at x ~ 0.5
    reg = dict(alpha_W=1e5, beta_W=5e4, alpha_F=1e4, beta_F=5e3)
    p = nk.default_params(R, seed=SEED, **reg)
    rng = np.random.default_rng(11)
    W0 = oracle.uniform_init(SEED, 0, R, V.n)
    F0 = oracle.uniform_init(SEED, 1, R, V.m)
    with nk.NMFKL(V.n, V.m, params=p) as m:
        m.set_data(V)
        m.init()
        m.sweep_F(0)
        F1g = m.get_F()
        m.init()
        m.sweep_W(0)
        W1g = m.get_W()
    _check_sampled(_sample_units(V.colptr, 32, rng), V.colptr, V.rowidx, V.val, W0, F0, oracle.rowsum(W0), F1g,
                   p, 0, name="full_size_sampled_regularized")
    _check_sampled(_sample_units(V.rowptr, 16, rng), V.rowptr, V.colidx, V.rval, F0, W0, oracle.rowsum(F0), W1g,
                   p, 1, name="full_size_sampled_regularized")
