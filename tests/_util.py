"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

import oracle
import paper_1604_04026_gb300 as nk
from paper_1604_04026_gb300 import synth

# Per-entry bar of one sweep from an identical state: |gpu - oracle| <=
# RTOL |oracle| + FLOOR * max_k |oracle[:, unit]| (relative 1e-4, with a
# floor scaled to the unit's largest entry for values near zero).
RTOL = 1e-4
FLOOR = 1e-6

# Each coordinate solved to its 1-D minimiser: the Newton loop runs until its
# step is below 1e-7 relative (reachable in FP32; quadratic convergence puts
# the FP64 result ~1e-14 from the minimiser), the gradient test is far below
# FP32 noise, and the cap is high enough for the log-barrier regrowth from 0.
TIGHT = dict(eps_x=1e-7, max_inner=64, eps_grad=1e-9)


def params(r, **kw):
    return nk.default_params(r, **kw)


def cfg_for(p, side):
    """Oracle parameters of one side from the library parameters."""
    alpha = p.alpha_F if side == 0 else p.alpha_W
    beta = p.beta_F if side == 0 else p.beta_W
    return oracle.cfg(alpha=alpha, beta=beta, eps_grad=p.eps_grad, eps_div=p.eps_div, eps_x=p.eps_x,
                      max_inner=p.max_inner, grad_mode=p.grad_mode, break_mode=p.break_mode,
                      perm_mode=p.perm_mode)


def model(V, W0, F0, p):
    m = nk.NMFKL(V.n, V.m, params=p)
    m.set_data(V)
    m.init(np.ascontiguousarray(W0, dtype=np.float32), np.ascontiguousarray(F0, dtype=np.float32))
    return m


def unit_objectives(V, W, F, side, alpha=0.0, beta=0.0, eps_div=1e-6):
    """Subproblem objective (Eq. kl) of every unit at (W, F), in FP64 numpy:
    side 0: per column j of F, side 1: per row i of W."""
    W = np.asarray(W, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    if side == 0:
        units, ptr, idx, val = V.m, V.colptr, V.rowidx, V.val
        other_of = np.repeat(np.arange(units), np.diff(ptr))
        x = np.einsum("kp,kp->p", W[:, idx], F[:, other_of])
        X, S = F, W.sum(axis=1)
    else:
        units, ptr, idx, val = V.n, V.rowptr, V.colidx, V.rval
        other_of = np.repeat(np.arange(units), np.diff(ptr))
        x = np.einsum("kp,kp->p", F[:, idx], W[:, other_of])
        X, S = W, F.sum(axis=1)
    v = val.astype(np.float64)
    terms = v * np.log(v / (x + eps_div)) - v
    data = np.zeros(units)
    np.add.at(data, other_of, terms)
    return data + S @ X + 0.5 * alpha * (X * X).sum(axis=0) + beta * np.abs(X).sum(axis=0)


def _unit_layout(V, W, F, side):
    W = np.asarray(W, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    if side == 0:
        return V.m, V.colptr, V.rowidx, V.val.astype(np.float64), W, F
    return V.n, V.rowptr, V.colidx, V.rval.astype(np.float64), F, W


def objective_scale(V, W, F, side, alpha=0.0, beta=0.0, eps_div=1e-6):
    """Per unit, the sum of the magnitudes of the terms of Eq. kl: the scale
    at which FP32 evaluation of the unit's objective is accurate."""
    units, ptr, idx, v, A, X = _unit_layout(V, W, F, side)
    owner = np.repeat(np.arange(units), np.diff(ptr))
    x = np.einsum("kp,kp->p", A[:, idx], X[:, owner])
    terms = v * (np.abs(np.log(v / (x + eps_div))) + 1.0)
    mag = np.zeros(units)
    np.add.at(mag, owner, terms)
    return mag + A.sum(axis=1) @ np.abs(X) + 0.5 * alpha * (X * X).sum(axis=0) + beta * np.abs(X).sum(axis=0)


def objective_rel(V, Wg, Fg, Wo, Fo, side, alpha=0.0, beta=0.0, eps_div=1e-6):
    """max over units of |D_u(gpu) - D_u(oracle)| / (magnitude of D_u's terms)."""
    dg = unit_objectives(V, Wg, Fg, side, alpha, beta, eps_div)
    do = unit_objectives(V, Wo, Fo, side, alpha, beta, eps_div)
    scale = objective_scale(V, Wo, Fo, side, alpha, beta, eps_div)
    return float((np.abs(dg - do) / np.maximum(scale, 1e-30)).max())


U32 = 2.0 ** -24
PROBE_RUNS = 8
PROBE_FACTOR = 4.0


def fp32_sensitivity(V, W, F, side, p, ref, runs=PROBE_RUNS, threads=8):
    """Per entry, how far the oracle's half moves when the model values x_p
    are perturbed at FP32's unit roundoff after every update (Monte Carlo
    arithmetic, Parker 1997): max over `runs` seeded probe runs of
    |probe - ref|, and the probe results. `ref` is the unperturbed oracle
    half from the same state."""
    dev = np.zeros_like(np.asarray(ref, dtype=np.float64))
    probes = []
    for s in range(runs):
        c = cfg_for(p, side)
        c.perturb = U32
        c.perturb_seed = 1 + s
        if side == 0:
            x, _ = oracle.half_F(V, W, F, p.seed, 0, c, threads=threads)
        else:
            x, _ = oracle.half_W(V, W, F, p.seed, 0, c, threads=threads)
        dev = np.maximum(dev, np.abs(x - ref))
        probes.append(x)
    return dev, probes


def trajectory_sensitivity(V, W0, F0, p, sweeps, ref_kl, runs=4, threads=8):
    """Per sweep, max over `runs` Monte Carlo arithmetic runs of the oracle fit
    (x_p perturbed at FP32's unit roundoff, as in fp32_sensitivity) of
    |KL_probe - KL_ref|: how far FP32-level rounding moves the nonconvex
    trajectory of Algorithm 1."""
    dev = np.zeros(sweeps)
    for s in range(runs):
        cF, cW = cfg_for(p, 0), cfg_for(p, 1)
        for c in (cF, cW):
            c.perturb = U32
            c.perturb_seed = 101 + s
        res = oracle.fit(V, W0, F0, p.seed, sweeps, cF, cW, threads=threads)
        dev = np.maximum(dev, np.abs(res.kl - ref_kl))
    return dev


def within(g, o, rtol=RTOL, floor=FLOOR, slack=None):
    """Boolean mask of entries inside the per-entry bar (columns are units):
    |g - o| <= rtol |o| + floor * max_k |o[:, unit]| (+ the FP32 slack)."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    scale = np.abs(o).max(axis=0, keepdims=True)
    bound = rtol * np.abs(o) + floor * scale
    if slack is not None:
        bound = bound + slack
    return np.abs(g - o) <= bound


# The FP32 slack of the per-entry bar is capped: an entry may exceed the plain
# bar (1e-4 relative + the column-scaled floor) by its measured FP32
# sensitivity, but never by more than SLACK_CAP times the plain bound in all,
# and at most SLACK_FRACTION of a result's entries may need the slack.
# An entry whose measured sensitivity alone exceeds the cap is ill-conditioned:
# perturbing its subproblem's model values x_p at FP32's unit roundoff moves
# the FP64 oracle's own entry by more than 10x the plain bound, so no FP32
# computation can be held to that bar per entry. Only such entries may lie
# outside the capped bar: at most SLACK_FRACTION of a result's entries, each
# within PROBE_FACTOR x its own sensitivity, and their units held to the
# per-unit objective bar. Their count is reported (it measures the input's
# conditioning, not the kernel).
SLACK_CAP = 10.0
SLACK_FRACTION = 0.005


def parity_report(name, g, o, slack=None, rtol=RTOL, floor=FLOOR):
    """Per-entry parity of a result against the oracle, on the plain bar and
    on the capped slackened bar. Returns a dict:
      plain_frac     entries within |g-o| <= rtol|o| + floor*max_k|o[:, unit]|
      need_slack     entries outside the plain bar but within the slackened one
      beyond_cap     entries outside the slackened bar (capped at SLACK_CAP x the plain bound)
      max_ratio      max over entries of |g-o| / plain bound
      max_rel_err    max over entries with o != 0 of |g-o|/|o|
    and, when PARITY_REPORT names a file, appends it there as one JSON line."""
    import json
    import os
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    scale = np.abs(o).max(axis=0, keepdims=True)
    plain = rtol * np.abs(o) + floor * scale
    err = np.abs(g - o)
    extra = np.zeros_like(o) if slack is None else np.asarray(slack, dtype=np.float64)
    capped = np.minimum(plain + extra, SLACK_CAP * plain)
    in_plain = err <= plain
    in_capped = err <= capped
    ill = extra > (SLACK_CAP - 1.0) * plain
    nz = o != 0
    rep = {"name": name, "entries": int(o.size), "plain_frac": float(in_plain.mean()),
           "need_slack": int((~in_plain & in_capped).sum()), "beyond_cap": int((~in_capped).sum()),
           "ill_conditioned": int(ill.sum()),
           "beyond_cap_well_conditioned": int((~in_capped & ~ill).sum()),
           "ill_beyond_their_slack": int((ill & (err > plain + extra)).sum()),
           "max_ratio": float((err / np.maximum(plain, 1e-300)).max()) if o.size else 0.0,
           "max_rel_err": float((err[nz] / np.abs(o[nz])).max()) if nz.any() else 0.0}
    print("PARITY", json.dumps(rep))
    path = os.environ.get("PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rep) + "\n")
    return rep


def report_trajectory(name, rel_err, rel_spread):
    """Records the per-sweep relative KL error of a trajectory against the
    oracle's (and the FP32 spread of the oracle's own trajectory) as
    parity_report does."""
    import json
    import os
    rep = {"name": name, "sweeps": int(len(rel_err)), "max_rel_err": float(np.max(rel_err)),
           "plain_frac": float(np.mean(np.asarray(rel_err) <= RTOL)),
           "max_rel_spread": float(np.max(rel_spread))}
    print("PARITY", json.dumps(rep))
    path = os.environ.get("PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rep) + "\n")
    return rep


def assert_parity(name, g, o, slack=None, fraction=None):
    """The per-entry gate: every entry within the capped slackened bar and at
    most SLACK_FRACTION of them outside the plain bar; or, with `fraction`
    (the paper's constants, where a threshold decision may flip), at least
    that fraction within the capped slackened bar."""
    rep = parity_report(name, g, o, slack)
    n = max(rep["entries"], 1)
    if fraction is None:
        assert rep["beyond_cap_well_conditioned"] == 0, rep
        assert rep["ill_beyond_their_slack"] == 0, rep
        assert rep["beyond_cap"] <= SLACK_FRACTION * n, rep
        assert rep["need_slack"] <= SLACK_FRACTION * n, rep
    else:
        assert 1.0 - rep["beyond_cap"] / n >= fraction, rep
    return rep


def start(V, r, seed=0):
    return synth.uniform_init(r, V.n, seed, 0), synth.uniform_init(r, V.m, seed, 1)


def designed_matrix(n, m, col_lengths, row_lengths, seed=0):
    """Count matrix whose first columns have the given lengths and whose
    first rows have the given lengths (both at once), plus a sprinkle of
    entries elsewhere; values are small counts >= 1."""
    rng = np.random.default_rng(seed)
    d = {}
    for j, L in enumerate(col_lengths):
        for i in rng.choice(n, size=min(L, n), replace=False):
            d[(int(i), j)] = float(rng.integers(1, 6))
    for i, L in enumerate(row_lengths):
        for j in rng.choice(m, size=min(L, m), replace=False):
            d[(n - 1 - i, int(j))] = float(rng.integers(1, 6))
    for _ in range(3 * (n + m)):
        d[(int(rng.integers(n)), int(rng.integers(m)))] = float(rng.integers(1, 4))
    # exact column lengths for the designed columns: drop extras beyond L
    items = sorted(d.items(), key=lambda t: (t[0][1], t[0][0]))
    cols = [[] for _ in range(m)]
    for (i, j), v in items:
        cols[j].append((i, v))
    for j, L in enumerate(col_lengths):
        if len(cols[j]) > L:
            keep = rng.choice(len(cols[j]), size=L, replace=False)
            cols[j] = sorted(cols[j][k] for k in keep)
    colptr = np.zeros(m + 1, dtype=np.int64)
    colptr[1:] = np.cumsum([len(c) for c in cols])
    rowidx = np.array([i for c in cols for i, _ in c], dtype=np.int32)
    val = np.array([v for c in cols for _, v in c], dtype=np.float32)
    return synth.from_csc(n, m, colptr, rowidx, val)
