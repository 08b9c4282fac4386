"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one part of the oracle to a library routine, a closed form,
brute force or an invariant that the paper and the mathematics fix:

* Philox4x64-10      -> numpy.random.Philox (an independent implementation)
* ids                -> bijective, uniform over all r! orders (chi-square)
* Eq. Partial        -> central finite differences of scipy.special.kl_div
* Eq. 1              -> dense scipy.special.kl_div sum; D = 0 at V = W^T F
* Algorithm 2, r = 1 -> closed-form minimiser of the 1-D subproblem
* Algorithm 2, r > 1 -> scipy L-BFGS-B on the dense objective; brute-force grid;
                        Lee-Seung multiplicative updates (a textbook method)
* Algorithm 1        -> nonnegativity, monotone KL per half, KKT at convergence,
                        exact-fit recovery, exact zeros appear (Table 2)
"""
import itertools
import math

import numpy as np
import pytest
from scipy import optimize, special, stats

import oracle
from paper_1604_04026_gb300 import synth


# ----------------------------------------------------------------- Philox / ids
def test_philox_matches_numpy():
    rng = np.random.default_rng(1)
    for _ in range(20):
        ctr = [int(x) for x in rng.integers(0, 2**62, size=4, dtype=np.int64)]
        key = [int(x) for x in rng.integers(0, 2**62, size=2, dtype=np.int64)]
        # numpy's Philox increments the counter before producing a block
        g = np.random.Philox(counter=[ctr[0] - 1] + ctr[1:], key=key)
        want = g.random_raw(4)
        got = oracle.philox4x64_10(ctr, key)
        assert np.array_equal(got, want)


def test_perm_is_bijection_and_deterministic():
    for r in (1, 2, 7, 10, 50, 100, 200, 256):
        for col in range(5):
            p = oracle.perm(3, 2, 1, col, r)
            assert sorted(p.tolist()) == list(range(r))
            assert np.array_equal(p, oracle.perm(3, 2, 1, col, r))
    assert not np.array_equal(oracle.perm(0, 0, 0, 0, 50), oracle.perm(0, 0, 0, 1, 50))
    assert not np.array_equal(oracle.perm(0, 0, 0, 0, 50), oracle.perm(0, 1, 0, 0, 50))
    assert not np.array_equal(oracle.perm(0, 0, 0, 0, 50), oracle.perm(0, 0, 1, 0, 50))
    assert not np.array_equal(oracle.perm(0, 0, 0, 0, 50), oracle.perm(1, 0, 0, 0, 50))


def test_perm_shared_mode_is_one_order_per_sweep():
    a = oracle.perm(7, 3, 0, 11, 40, perm_mode=1)
    assert np.array_equal(a, oracle.perm(7, 3, 1, 999, 40, perm_mode=1))
    assert not np.array_equal(a, oracle.perm(7, 4, 0, 11, 40, perm_mode=1))


def test_perm_uniform_over_all_orders():
    r = 4
    counts = {}
    N = 24 * 400
    for col in range(N):
        counts[tuple(oracle.perm(5, 0, 0, col, r))] = counts.get(tuple(oracle.perm(5, 0, 0, col, r)), 0) + 1
    assert len(counts) == math.factorial(r)
    obs = np.array([counts[p] for p in itertools.permutations(range(r))])
    _, pval = stats.chisquare(obs)
    assert pval > 1e-3


def test_perm_positions_uniform_large_r():
    r = 100
    pos = np.zeros((r, r))
    for col in range(3000):
        p = oracle.perm(9, 1, 0, col, r)
        pos[np.arange(r), p] += 1
    _, pval = stats.chisquare(pos.ravel())
    assert pval > 1e-3


def test_uniform_init_range_and_fp32_exact():
    x = oracle.uniform_init(0, 1, 7, 33)
    assert x.min() >= 0.0 and x.max() < 1.0
    assert np.array_equal(x.astype(np.float32).astype(np.float64), x)
    assert abs(x.mean() - 0.5) < 0.1


# ----------------------------------------------------------------- Eq. Partial
def _dense_f(v_all, A_all, x, alpha, beta):
    """Subproblem objective (Eq. kl) over ALL rows, via scipy's generalized KL."""
    return special.kl_div(v_all, A_all @ x).sum() + 0.5 * alpha * x @ x + beta * np.abs(x).sum()


@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (0.3, 0.2)])
def test_derivatives_match_finite_differences(alpha, beta):
    rng = np.random.default_rng(2)
    n, r = 30, 5
    A_all = rng.gamma(1.0, 1.0, size=(n, r))
    v_all = np.where(rng.random(n) < 0.4, rng.poisson(3.0, size=n) + 1.0, 0.0)
    nz = np.nonzero(v_all)[0]
    x = rng.uniform(0.2, 1.5, size=r)
    c = oracle.cfg(alpha=alpha, beta=beta, eps_div=0.0)
    sumA = A_all.sum(axis=0)
    Ax = A_all[nz] @ x
    for k in range(r):
        g, h = oracle.derivatives(v_all[nz], A_all[nz], Ax, k, sumA[k], x[k], c)
        e = np.zeros(r)
        d = 1e-5
        e[k] = d
        fp, f0, fm = (_dense_f(v_all, A_all, x + e, alpha, beta), _dense_f(v_all, A_all, x, alpha, beta),
                      _dense_f(v_all, A_all, x - e, alpha, beta))
        g_fd = (fp - fm) / (2 * d)
        h_fd = (fp - 2 * f0 + fm) / (d * d)
        assert abs(g - g_fd) <= 1e-6 * max(1.0, abs(g_fd))
        assert abs(h - h_fd) <= 1e-3 * max(1.0, abs(h_fd))


# ----------------------------------------------------------------- Eq. 1
def test_objective_matches_dense_kl_div():
    V = synth.poisson_lowrank(60, 40, 4, density=0.2, seed=3)
    rng = np.random.default_rng(3)
    W = rng.uniform(0, 1, size=(4, V.n))
    F = rng.uniform(0, 1, size=(4, V.m))
    kl, reg = oracle.objective(V, W, F, eps_div=0.0, a1=0.5, a2=0.25, b1=0.1, b2=0.2)
    want = special.kl_div(V.dense(), W.T @ F).sum()
    assert kl == pytest.approx(want, rel=1e-12)
    want_reg = 0.25 * (W ** 2).sum() + 0.125 * (F ** 2).sum() + 0.1 * W.sum() + 0.2 * F.sum()
    assert reg == pytest.approx(want_reg, rel=1e-12)


def test_objective_zero_at_exact_fit():
    rng = np.random.default_rng(4)
    W = rng.uniform(0.1, 1, size=(3, 12))
    F = rng.uniform(0.1, 1, size=(3, 9))
    V = synth.from_dense((W.T @ F).astype(np.float32))
    Wf = W.astype(np.float32).astype(np.float64)
    Ff = F.astype(np.float32).astype(np.float64)
    # V holds W^T F rounded to FP32, so D is at the level of that rounding
    kl, _ = oracle.objective(V, Wf, Ff, eps_div=0.0)
    assert abs(kl) < 1e-9 * V.val.sum()


# ----------------------------------------------------------------- Algorithm 2
def _closed_form_r1(sv, S, alpha, beta):
    if alpha == 0.0:
        return sv / (S + beta)
    return (-(S + beta) + math.sqrt((S + beta) ** 2 + 4 * alpha * sv)) / (2 * alpha)


@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (0.5, 0.0), (0.0, 0.7), (1.3, 0.4)])
def test_alg2_r1_closed_form(alpha, beta):
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = 15
        a_all = rng.gamma(1.0, 1.0, size=(n, 1))
        v_all = np.where(rng.random(n) < 0.5, rng.poisson(4.0, size=n) + 1.0, 0.0)
        v_all[0] = 2.0
        nz = np.nonzero(v_all)[0]
        S = a_all.sum()
        xs = _closed_form_r1(v_all.sum(), S, alpha, beta)
        x0 = np.array([xs * rng.uniform(0.3, 1.8)])  # inside the Newton basin (below 2 x*)
        x, st = oracle.alg2(v_all[nz], a_all[nz], [S], x0, [0],
                            oracle.tight_cfg(alpha=alpha, beta=beta, eps_div=0.0))
        assert x[0] == pytest.approx(xs, rel=1e-10)
        assert st["cap_hits"] == 0


def test_alg2_one_coordinate_is_exact_1d_minimiser():
    """Each coordinate step of tight Algorithm 2 lands on the argmin over x_k >= 0
    of the dense objective with the other coordinates held (bounded Brent)."""
    rng = np.random.default_rng(6)
    n, r = 25, 4
    for trial in range(10):
        A_all = rng.gamma(0.7, 1.0, size=(n, r))
        v_all = np.where(rng.random(n) < 0.5, rng.poisson(3.0, size=n) + 1.0, 0.0)
        v_all[:2] = 1.0
        nz = np.nonzero(v_all)[0]
        x0 = rng.uniform(0.1, 1.0, size=r)
        k = trial % r
        rest = A_all @ x0 - A_all[:, k] * x0[k]
        # two coordinates: k, and the others folded into one column held at 1;
        # ids visits k first, so x[0] is the result of k's Newton loop alone
        A2 = np.stack([A_all[:, k], rest], axis=1)
        x, _ = oracle.alg2(v_all[nz], A2[nz], A2.sum(axis=0), [x0[k], 1.0], [0, 1],
                           oracle.tight_cfg(eps_div=0.0))

        def f1(t):
            return special.kl_div(v_all, rest + A_all[:, k] * t).sum()

        res = optimize.minimize_scalar(f1, bounds=(0.0, 50.0), method="bounded",
                                       options={"xatol": 1e-12})
        xb = max(res.x, 0.0)
        # rest > 0 on the support here, so the minimiser may sit at 0
        assert abs(x[0] - xb) <= 1e-6 * max(1.0, xb)


def _solve_full(v_all, A_all, alpha, beta, sweeps=200):
    nz = np.nonzero(v_all)[0]
    r = A_all.shape[1]
    x = np.full(r, 0.5)
    S = A_all.sum(axis=0)
    c = oracle.tight_cfg(alpha=alpha, beta=beta, eps_div=0.0)
    for s in range(sweeps):
        x, _ = oracle.alg2(v_all[nz], A_all[nz], S, x, oracle.perm(1, s, 0, 0, r), c)
    return x


@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (0.2, 0.3)])
def test_alg2_converges_to_lbfgsb_minimiser(alpha, beta):
    rng = np.random.default_rng(7)
    n, r = 40, 5
    A_all = rng.gamma(0.5, 1.0, size=(n, r))
    v_all = np.where(rng.random(n) < 0.5, rng.poisson(5.0, size=n) + 1.0, 0.0)
    x = _solve_full(v_all, A_all, alpha, beta)
    res = optimize.minimize(lambda z: _dense_f(v_all, A_all, z, alpha, beta), np.full(r, 0.5),
                            method="L-BFGS-B", bounds=[(0, None)] * r,
                            options={"ftol": 1e-15, "gtol": 1e-10, "maxiter": 5000})
    f_ours = _dense_f(v_all, A_all, x, alpha, beta)
    assert f_ours <= res.fun + 1e-7 * abs(res.fun)
    assert np.allclose(x, res.x, atol=2e-3 * max(1.0, np.abs(res.x).max()))


def test_alg2_brute_force_grid_r2():
    rng = np.random.default_rng(8)
    n, r = 8, 2
    A_all = rng.gamma(1.0, 1.0, size=(n, r))
    v_all = np.array([3, 0, 1, 4, 0, 2, 5, 1], dtype=float)
    x = _solve_full(v_all, A_all, 0.0, 0.0, sweeps=100)
    g = np.linspace(0, 12, 1201)
    X, Y = np.meshgrid(g, g, indexing="ij")
    Ax = A_all[:, 0][None, None, :] * X[..., None] + A_all[:, 1][None, None, :] * Y[..., None]
    f = special.kl_div(v_all[None, None, :], Ax).sum(-1)
    i, j = np.unravel_index(np.argmin(f), f.shape)
    assert abs(x[0] - g[i]) <= 0.02 and abs(x[1] - g[j]) <= 0.02
    assert _dense_f(v_all, A_all, x, 0, 0) <= f[i, j] + 1e-12


def test_alg2_matches_lee_seung_mu():
    """Lee & Seung's multiplicative update for KL, x <- x * (A^T (v/Ax)) / (A^T 1),
    run to convergence on the same convex subproblem (a textbook method)."""
    rng = np.random.default_rng(9)
    n, r = 50, 4
    A_all = rng.gamma(2.0, 1.0, size=(n, r))
    xt = rng.uniform(0.5, 2.0, size=r)
    v_all = rng.poisson(A_all @ xt).astype(float)
    x = _solve_full(v_all, A_all, 0.0, 0.0)
    z = np.ones(r)
    for _ in range(200000):
        z = z * (A_all.T @ (v_all / (A_all @ z))) / A_all.sum(axis=0)
    assert np.allclose(x, z, rtol=1e-5, atol=1e-6)


def test_alg2_h_zero_case():
    """alpha = 0 and the coordinate's column is zero on the support: the
    objective is linear in x_k with slope sumA_k >= 0, so x_k goes to 0."""
    A = np.array([[1.0, 0.0], [2.0, 0.0]])
    v = np.array([1.0, 3.0])
    x, st = oracle.alg2(v, A, [5.0, 2.0], [0.5, 0.8], [1, 0], oracle.cfg())
    assert x[1] == 0.0
    assert st["cap_hits"] == 0
    # zero slope too (sumA_k = 0): every x_k is optimal, x_k stays
    x, _ = oracle.alg2(v, A, [5.0, 0.0], [0.5, 0.8], [1, 0], oracle.cfg())
    assert x[1] == 0.8


def test_alg2_empty_subproblem():
    """No nonzeros: f(x) = sumA.x + alpha/2|x|^2 + beta|x|_1, minimised at 0."""
    x, _ = oracle.alg2(np.zeros(0), np.zeros((0, 3)), [1.0, 2.0, 0.5], [0.3, 0.0, 2.0], [2, 0, 1],
                       oracle.cfg(alpha=0.1))
    assert np.array_equal(x, np.zeros(3))


# ----------------------------------------------------------------- Algorithm 1
def test_half_thread_count_independent():
    V = synth.docs(300, 400, 5, seed=1, threads=2)
    r = 8
    W0 = synth.uniform_init(r, V.n, 0, 0)
    F0 = synth.uniform_init(r, V.m, 0, 1)
    a, _ = oracle.half_F(V, W0, F0, 0, 0, threads=1)
    b, _ = oracle.half_F(V, W0, F0, 0, 0, threads=4)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("mode", ["default", "literal"])
def test_fit_invariants_c1(mode):
    """Nonnegativity and monotone KL after every half on the small Poisson
    workload (n=1000, m=500, r=10, 20 sweeps)."""
    V = synth.poisson_lowrank(1000, 500, 10, seed=0)
    assert V.nnz > 1000
    r = 10
    W = synth.uniform_init(r, V.n, 0, 0).astype(np.float64)
    F = synth.uniform_init(r, V.m, 0, 1).astype(np.float64)
    c = oracle.cfg() if mode == "default" else oracle.cfg(grad_mode=1, eps_grad=1e-10, break_mode=1,
                                                          perm_mode=1)
    kl0 = prev = oracle.objective(V, W, F)[0]
    # The default |dx| break runs each Newton loop until its step is small, so
    # every half lowers D. The literal signed break stops right after a
    # Newton overshoot (g is concave in x_k, so a step from the right lands
    # left of the minimiser), which can raise D on a half; there only the
    # overall descent is checked.
    strict = mode == "default"
    for s in range(20):
        F, _ = oracle.half_F(V, W, F, 0, s, c)
        kl = oracle.objective(V, W, F)[0]
        assert kl <= prev * (1 + 1e-12) or not strict
        prev = kl
        W, _ = oracle.half_W(V, W, F, 0, s, c)
        kl = oracle.objective(V, W, F)[0]
        assert kl <= prev * (1 + 1e-12) or not strict
        prev = kl
        assert W.min() >= 0 and F.min() >= 0
    assert prev < 0.5 * kl0
    # sparse factors appear (cf. Table 2)
    assert (F == 0).mean() > 0.2 and (W == 0).mean() > 0.2


def test_fit_trajectory_matches_halves():
    V = synth.poisson_lowrank(200, 150, 5, density=0.05, seed=2)
    r = 5
    W0 = synth.uniform_init(r, V.n, 1, 0)
    F0 = synth.uniform_init(r, V.m, 1, 1)
    res = oracle.fit(V, W0, F0, seed=4, sweeps=3)
    W, F = W0.astype(np.float64), F0.astype(np.float64)
    for s in range(3):
        F, _ = oracle.half_F(V, W, F, 4, s)
        W, _ = oracle.half_W(V, W, F, 4, s)
        assert res.kl[s] == oracle.objective(V, W, F)[0]
    assert np.array_equal(res.W, W) and np.array_equal(res.F, F)


def _kkt_violation(V, W, F, side):
    """max_k |min(x_k, g_k)| / (sumA_k) over all subproblems of one side."""
    r = W.shape[0]
    worst = 0.0
    if side == 0:
        sumA = W.sum(axis=1)
        for j in range(V.m):
            sl = slice(V.colptr[j], V.colptr[j + 1])
            A = W[:, V.rowidx[sl]].T
            x = F[:, j]
            Ax = A @ x
            for k in range(r):
                g, _ = oracle.derivatives(V.val[sl], A, Ax, k, sumA[k], x[k], oracle.cfg(eps_div=0.0))
                worst = max(worst, abs(min(x[k], g)) / sumA[k])
    else:
        sumA = F.sum(axis=1)
        for i in range(V.n):
            sl = slice(V.rowptr[i], V.rowptr[i + 1])
            A = F[:, V.colidx[sl]].T
            x = W[:, i]
            Ax = A @ x
            for k in range(r):
                g, _ = oracle.derivatives(V.rval[sl], A, Ax, k, sumA[k], x[k], oracle.cfg(eps_div=0.0))
                worst = max(worst, abs(min(x[k], g)) / sumA[k])
    return worst


def test_kkt_at_convergence():
    V = synth.poisson_lowrank(60, 50, 3, density=0.3, seed=5)
    r = 3
    W = synth.uniform_init(r, V.n, 2, 0) + 0.1
    F = synth.uniform_init(r, V.m, 2, 1) + 0.1
    c = oracle.tight_cfg(eps_div=0.0)
    res = oracle.fit(V, W, F, seed=0, sweeps=400, cF=c, cW=c, trace=False)
    # F was just solved with W fixed: its KKT holds to the solver tolerance
    W2, F2 = res.W, res.F
    F3, _ = oracle.half_F(V, W2, F2, 0, 999, c)
    assert _kkt_violation(V, W2, F3, 0) < 1e-6
    W3, _ = oracle.half_W(V, W2, F3, 0, 999, c)
    assert _kkt_violation(V, W3, F3, 1) < 1e-6
    # and the alternating fit itself is near a stationary point
    assert _kkt_violation(V, W3, F3, 0) < 1e-3


def test_foldin_recovers_exact_fit():
    rng = np.random.default_rng(11)
    r, n, m = 4, 40, 12
    W = rng.uniform(0.05, 1.0, size=(r, n))
    Ft = rng.uniform(0.2, 2.0, size=(r, m))
    V = synth.from_dense(W.T @ Ft)  # every entry stored, FP32-rounded values
    F0 = np.full((r, m), 0.5)
    F, done = oracle.foldin(V, W, F0, seed=3, rel_tol=1e-14, max_sweeps=3000,
                            c=oracle.tight_cfg(eps_div=0.0))
    assert np.allclose(F, Ft, rtol=1e-4, atol=1e-5)
    assert done.max() <= 3000


def _column_objectives(V, W, F, eps_div=1e-6):
    """Eq. kl of every column (data term over its nonzeros plus the linear
    term sum_k sumW_k F_kj), straight from the dense products in numpy."""
    out = np.zeros(V.m)
    sumW = W.sum(axis=1)
    for j in range(V.m):
        a, b = V.colptr[j], V.colptr[j + 1]
        v = V.val[a:b].astype(np.float64)
        x = W[:, V.rowidx[a:b]].T @ F[:, j]
        out[j] = np.sum(v * np.log(v / (x + eps_div)) - v) + sumW @ F[:, j]
    return out


def test_foldin_stops_on_relative_change():
    """Each document stops after the first pass whose objective changed by at
    most rel_tol times the previous value, and not before: the objectives
    after exactly t passes (fixed pass counts, rel_tol = 0) show that the last
    pass met the test and the one before it did not."""
    topics, V = synth.foldin_docs(500, 30, 6, seed=2, threads=2)
    W = topics.astype(np.float64)
    F0 = synth.uniform_init(6, V.m, 0, 1)
    tol = 1e-5
    F, done = oracle.foldin(V, W, F0, seed=0, rel_tol=tol, max_sweeps=200)
    assert (done >= 1).all() and (done < 200).all()
    assert (done >= 3).sum() >= V.m // 2  # most documents need several passes
    D = []
    for t in range(int(done.max()) + 1):
        Ft, dt = oracle.foldin(V, W, F0, seed=0, rel_tol=0.0, max_sweeps=t)
        # with rel_tol = 0 a document stops early only on an exactly unchanged
        # objective (every coordinate already optimal), and stays there
        assert (dt <= t).all()
        D.append(_column_objectives(V, W, Ft))
        for j in np.nonzero(done == t)[0]:
            # the stopped result is the state after exactly `done` passes
            assert np.array_equal(Ft[:, j], F[:, j]), j
    D = np.array(D)  # D[t, j]: objective of document j after t passes
    slop = 1e-12  # evaluation-order rounding between the oracle's sum and numpy's
    for j in range(V.m):
        d = int(done[j])
        assert abs(D[d - 1, j] - D[d, j]) <= tol * abs(D[d - 1, j]) * (1 + slop) + slop * abs(D[d, j]), j
        if d >= 2:
            assert abs(D[d - 2, j] - D[d - 1, j]) > tol * abs(D[d - 2, j]) * (1 - slop), j


def test_probe_magnitude_matches_first_order_closed_form():
    """The Monte Carlo arithmetic probe perturbs each x_p by a relative
    eps*xi, xi ~ U(-1, 1), after its initial sum. On an r = 1 column of L unit
    counts with W = 1 on every row (S = sum W = n = L) and eps_div = 0, one
    Newton step from f0 gives f1 = f0 + f0 (U1 - S f0) / U2 with U1 = sum
    1/(1+d_p), U2 = sum 1/(1+d_p)^2, so to first order in the perturbations
    d_p, df1 = f0 (L - 2 S f0) / L^2 * sum_p d_p, whose standard deviation is
    |f0 (L - 2 S f0)| / L^2 * eps * sqrt(L / 3). The spread of the probe runs
    must match it (a probe that over- or under-perturbs fails)."""
    L, f0, eps = 400, 0.3, 2.0 ** -24
    dense = np.ones((L, 1), dtype=np.float32)
    V = synth.from_dense(dense)
    W = np.ones((1, L))
    F0 = np.full((1, 1), f0)
    base = dict(eps_div=0.0, eps_x=0.0, eps_grad=0.0, max_inner=1)
    ref, st = oracle.half_F(V, W, F0, 0, 0, oracle.cfg(**base))
    assert st["steps"] == 1
    S = float(L)
    assert ref[0, 0] == pytest.approx(f0 + f0 * (L - S * f0) / L, rel=1e-14)
    devs = []
    for s in range(256):
        x, _ = oracle.half_F(V, W, F0, 0, 0, oracle.cfg(perturb=eps, perturb_seed=1 + s, **base))
        devs.append(x[0, 0] - ref[0, 0])
    devs = np.array(devs)
    predicted = abs(f0 * (L - 2 * S * f0)) / L ** 2 * eps * np.sqrt(L / 3.0)
    measured = devs.std()
    # sampling error of a standard deviation from 256 runs is ~4.4%
    assert 0.8 * predicted <= measured <= 1.25 * predicted, (measured, predicted)
    assert abs(devs.mean()) <= 4 * predicted / np.sqrt(len(devs))


def test_rounding_probe_off_by_default_and_deterministic():
    """The Monte Carlo arithmetic probe (used only to size FP32 bars) leaves
    the FP64 path untouched at perturb = 0, is reproducible per seed and
    independent of the thread count, and moves results by a small amount."""
    V = synth.docs(400, 300, 5, seed=2, threads=2)
    r = 8
    W0 = synth.uniform_init(r, V.n, 0, 0)
    F0 = synth.uniform_init(r, V.m, 0, 1)
    base, _ = oracle.half_F(V, W0, F0, 1, 0, oracle.cfg())
    same, _ = oracle.half_F(V, W0, F0, 1, 0, oracle.cfg(perturb=0.0, perturb_seed=7))
    assert np.array_equal(base, same)
    a, _ = oracle.half_F(V, W0, F0, 1, 0, oracle.cfg(perturb=2**-24, perturb_seed=7), threads=1)
    b, _ = oracle.half_F(V, W0, F0, 1, 0, oracle.cfg(perturb=2**-24, perturb_seed=7), threads=4)
    c, _ = oracle.half_F(V, W0, F0, 1, 0, oracle.cfg(perturb=2**-24, perturb_seed=8))
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c) and not np.array_equal(a, base)
    assert np.abs(a - base).max() < 1e-2 * np.abs(base).max()
