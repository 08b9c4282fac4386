/*
 * FP64 CPU oracle for sparse randomized coordinate descent (SRCD) on NMF with
 * KL divergence -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file's library. The CUDA library never calls it, and it shares no
 * code with the CUDA library.
 *
 * What it computes (Nguyen & Ho, "Fast parallel randomized algorithm for
 * nonnegative matrix factorization with KL divergence for large sparse
 * datasets"):
 *   V (n x m) ~= W^T F, W (r x n) >= 0, F (r x m) >= 0.
 *   Eq. 1   D(V || W^T F) = sum_ij V_ij log(V_ij / x_ij) - V_ij + x_ij,  x = W^T F
 *   Eq. 2   plus a1/2 |W|^2 + a2/2 |F|^2 + b1 |W|_1 + b2 |F|_1
 *   Eq. 3   D splits into independent per-column (F) and per-row (W) terms
 *   Eq. Partial (first and second derivative of the subproblem in x_k)
 *     g_k = -sum_i v_i A_ik / [Ax]_i + sum_i A_ik + alpha x_k + beta
 *     h_k =  sum_i v_i (A_ik / [Ax]_i)^2 + alpha
 *   projected Newton step  x_k <- max(0, x_k - g_k / h_k)   (Section 2)
 *   Algorithm 2: per-coordinate Newton loop in a random coordinate order
 *   Algorithm 1: alternate all columns of F, then all rows of W.
 *
 * Everything is plain sequential double-precision code in the paper's order;
 * sums run over the nonzeros of v in storage order. Only rows with v_i > 0
 * enter the data terms, and sum_i A_ik (all rows) is precomputed as sumA
 * (Algorithm 1 computes sumW = W 1 and sumF = F 1 before each half).
 *
 * Readings of points the paper leaves open (each is a parameter):
 *   - epsilon of Algorithm 2 is split in two: eps_div guards every
 *     denominator and log ([Ax]_i + eps_div); eps_grad is the gradient
 *     tolerance of the while test. grad_mode 0 (default) scales it as
 *     eps_grad * (sumA_k + beta) and tests x_k > 0; grad_mode 1 is the
 *     paper-literal absolute epsilon used in both places.
 *   - the inner break test uses |dx| < eps_x * xs (break_mode 0, default);
 *     break_mode 1 is the literal signed test dx < eps_x * xs.
 *   - the inner loop is capped at max_inner Newton steps per coordinate.
 *   - h_k = 0 (alpha = 0 and v_i A_ik = 0 on the support): the data term is
 *     flat in x_k, so x_k moves to 0 when g_k > 0 and stays otherwise.
 *   - the W half passes sumF, alpha1, beta1 (Algorithm 1 prints sumW,
 *     alpha2, beta2 there; Eq. 2 fixes which belong to W).
 *   - ids: a uniform random permutation of {0..r-1} by Fisher-Yates driven
 *     by Philox4x64-10 (Salmon et al., SC'11), keyed by the seed and
 *     counted by (block, column, sweep, side); perm_mode 1 shares one
 *     permutation per sweep across every column and row, as Algorithm 1
 *     draws ids once per outer iteration.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* Philox4x64-10, from the published round function: two 64x64->128      */
/* multiplications per round, a Weyl-sequence key schedule, 10 rounds.    */
/* ---------------------------------------------------------------------- */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL /* golden ratio */
#define PHILOX_W1 0xBB67AE8584CAA73BULL /* sqrt(3) - 1 */

void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0; k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Key and counter layout of the coordinate order (Algorithm 1, "ids"):
 *   key     = (seed, 0x5352434400000000 | purpose) with purpose 1 = ids
 *   counter = (block, column, sweep, side)
 * Random word t (t = 0, 1, ...) is word t % 4 of block t / 4. */
#define KEY_TAG_IDS 0x5352434400000001ULL
#define KEY_TAG_INIT 0x5352434400000002ULL

/* Fisher-Yates from the identity: for i = r-1 down to 1 take the next
 * 64-bit word u, j = floor(u * (i+1) / 2^64), swap ids[i], ids[j]. */
void oracle_perm(uint64_t seed, int64_t sweep, int32_t side, int64_t col, int32_t perm_mode,
                 int32_t r, int32_t *ids) {
    uint64_t key[2] = {seed, KEY_TAG_IDS};
    uint64_t ctr[4] = {0, (uint64_t)col, (uint64_t)sweep, (uint64_t)side};
    if (perm_mode == 1) { ctr[1] = 0; ctr[3] = 2; }
    for (int32_t i = 0; i < r; ++i) ids[i] = i;
    uint64_t words[4];
    int t = 0;
    for (int32_t i = r - 1; i >= 1; --i, ++t) {
        if (t % 4 == 0) { ctr[0] = (uint64_t)(t / 4); oracle_philox4x64_10(ctr, key, words); }
        uint64_t u = words[t % 4];
        int32_t j = (int32_t)(((unsigned __int128)u * (uint64_t)(i + 1)) >> 64);
        int32_t tmp = ids[i]; ids[i] = ids[j]; ids[j] = tmp;
    }
}

/* Uniform[0,1) starting values, FP32-representable (24-bit):
 * entry e of matrix `which` (0 = W, 1 = F) uses word e % 4 of the block
 * with counter (e / 4, which, 0, 0) and key (seed, KEY_TAG_INIT). */
void oracle_uniform_init(uint64_t seed, int32_t which, int64_t count, double *out) {
    uint64_t key[2] = {seed, KEY_TAG_INIT};
    uint64_t words[4];
    for (int64_t e = 0; e < count; ++e) {
        if (e % 4 == 0) {
            uint64_t ctr[4] = {(uint64_t)(e / 4), (uint64_t)which, 0, 0};
            oracle_philox4x64_10(ctr, key, words);
        }
        out[e] = (double)(words[e % 4] >> 40) * (1.0 / 16777216.0);
    }
}

/* ---------------------------------------------------------------------- */
/* Algorithm 2 on one subproblem                                          */
/* ---------------------------------------------------------------------- */
typedef struct {
    double alpha, beta;    /* L2 and L1 weights of this side (Eq. kl) */
    double eps_grad;       /* gradient tolerance (see grad_mode) */
    double eps_div;        /* guard added to [Ax]_i in divisions and logs */
    double eps_x;          /* inner-loop relative step break, 0.1 in Section 3 */
    int32_t max_inner;     /* cap on Newton steps per coordinate */
    int32_t grad_mode;     /* 0: eps_grad*(sumA_k+beta) and x_k>0; 1: absolute eps both places */
    int32_t break_mode;    /* 0: |dx| < eps_x*xs; 1: dx < eps_x*xs */
    int32_t perm_mode;     /* 0: ids per (sweep, side, column); 1: one ids per sweep */
    double perturb;        /* 0 (default): exact FP64. > 0: Monte Carlo arithmetic
                              probe (Parker 1997): [Ax]_p is multiplied by
                              (1 + perturb*xi), xi ~ U(-1, 1), after every update,
                              and by (1 + sqrt(r)*perturb*xi) after the initial sum,
                              keeping [Ax]_p >= 0 and exactly 0 when all its terms
                              A_pk x_k are 0 (it is a sum of nonnegative terms), to
                              measure how far rounding of x at that relative level
                              moves each result (tests use perturb = 2^-24, FP32's
                              unit roundoff). */
    uint64_t perturb_seed; /* stream of the probe; each unit mixes in its index, sweep and side */
} oracle_cfg;

typedef struct {
    int64_t coords;        /* coordinates visited */
    int64_t evals;         /* derivative evaluations (passes over the nonzeros) */
    int64_t steps;         /* Newton steps taken */
    int64_t cap_hits;      /* coordinates stopped by max_inner */
} oracle_stats;

/* Eq. Partial restricted to the nonzeros p of v (v_p > 0): the dense part
 * sum_i A_ik is sumA_k. A is L x r row-major, Ax holds [Ax]_p. */
void oracle_derivatives(int64_t L, const double *v, const double *A, int32_t r, const double *Ax,
                        int32_t k, double sumA_k, double x_k, const oracle_cfg *c,
                        double *g, double *h) {
    double s1 = 0.0, s2 = 0.0;
    for (int64_t p = 0; p < L; ++p) {
        double t = A[p * r + k] / (Ax[p] + c->eps_div);
        s1 += v[p] * t;
        s2 += v[p] * t * t;
    }
    *g = -s1 + sumA_k + c->alpha * x_k + c->beta;
    *h = s2 + c->alpha;
}

/* Uniform(-1, 1) from a splitmix64 stream (probe only). */
static double probe_xi(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

/* Updates x (length r) in place. ids is the coordinate order. Ax is scratch
 * of length L. */
void oracle_alg2(int64_t L, const double *v, const double *A, const double *sumA, double *x,
                 int32_t r, const int32_t *ids, const oracle_cfg *c, double *Ax, oracle_stats *st) {
    uint64_t probe = c->perturb_seed;
    /* Probe only: the number of positive terms A_pk x_k of each [Ax]_p. [Ax]_p
     * is a sum of nonnegative terms, so it is exactly 0 when that count is 0
     * and never negative; the perturbed values keep both properties. */
    int32_t *terms = NULL;
    if (c->perturb > 0.0) terms = (int32_t *)calloc((size_t)(L > 0 ? L : 1), sizeof(int32_t));
    /* Compute Ax on the nonzeros (Algorithm 2, first step). */
    for (int64_t p = 0; p < L; ++p) {
        double s = 0.0;
        for (int32_t k = 0; k < r; ++k) s += A[p * r + k] * x[k];
        Ax[p] = s;
        if (terms) {
            for (int32_t k = 0; k < r; ++k) terms[p] += (A[p * r + k] > 0.0 && x[k] > 0.0);
            Ax[p] = terms[p] == 0 ? 0.0 : Ax[p] * (1.0 + sqrt((double)r) * c->perturb * probe_xi(&probe));
        }
    }
    for (int32_t kk = 0; kk < r; ++kk) {
        int32_t k = ids[kk];
        double g, h;
        oracle_derivatives(L, v, A, r, Ax, k, sumA[k], x[k], c, &g, &h);
        if (st) { st->coords++; st->evals++; }
        double tol = c->grad_mode == 0 ? c->eps_grad * (sumA[k] + c->beta) : c->eps_grad;
        double xfloor = c->grad_mode == 0 ? 0.0 : c->eps_grad;
        int32_t it = 0;
        while (g < -tol || (fabs(g) > tol && x[k] > xfloor)) {
            if (it == c->max_inner) { if (st) st->cap_hits++; break; }
            ++it;
            double xn;
            if (h > 0.0) { xn = x[k] - g / h; if (xn < 0.0) xn = 0.0; }
            else xn = g > 0.0 ? 0.0 : x[k];
            double dx = xn - x[k];
            for (int64_t p = 0; p < L; ++p) Ax[p] += dx * A[p * r + k];
            if (terms) {
                const double xnew = x[k] + dx;
                const int dc = (x[k] == 0.0 && xnew > 0.0) ? 1 : ((x[k] > 0.0 && xnew == 0.0) ? -1 : 0);
                for (int64_t p = 0; p < L; ++p) {
                    if (A[p * r + k] > 0.0) terms[p] += dc;
                    if (terms[p] == 0) Ax[p] = 0.0;
                    else {
                        Ax[p] *= 1.0 + c->perturb * probe_xi(&probe);
                        if (Ax[p] < 0.0) Ax[p] = 0.0;
                    }
                }
            }
            double xs = x[k];
            x[k] = x[k] + dx;
            if (st) st->steps++;
            int brk = c->break_mode == 0 ? (fabs(dx) < c->eps_x * xs) : (dx < c->eps_x * xs);
            if (brk) break;
            oracle_derivatives(L, v, A, r, Ax, k, sumA[k], x[k], c, &g, &h);
            if (st) st->evals++;
        }
    }
    free(terms);
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 halves                                                      */
/* ---------------------------------------------------------------------- */
/* sumA_k = sum over the `cols` columns of M (r x cols row-major). */
void oracle_rowsum(const double *M, int32_t r, int64_t cols, double *out) {
    for (int32_t k = 0; k < r; ++k) {
        double s = 0.0;
        for (int64_t c = 0; c < cols; ++c) s += M[(int64_t)k * cols + c];
        out[k] = s;
    }
}

typedef struct {
    /* The half solves, for each unit u in [u0, u1), the subproblem with
     * v = val[ptr[u]..ptr[u+1]), A rows p = columns idx[p] of Aside (r x na),
     * x = column u of X (r x nx). */
    const int64_t *ptr; const int32_t *idx; const float *val;
    const double *Aside; int64_t na;
    double *X; int64_t nx;
    const double *sumA;
    int32_t r, side; int64_t sweep; uint64_t seed;
    const oracle_cfg *cfg;
    int64_t u0, u1;
    oracle_stats st;
} half_job;

static void *half_worker(void *arg) {
    half_job *J = (half_job *)arg;
    int32_t r = J->r;
    int64_t Lmax = 0;
    for (int64_t u = J->u0; u < J->u1; ++u) { int64_t L = J->ptr[u + 1] - J->ptr[u]; if (L > Lmax) Lmax = L; }
    double *v = (double *)malloc(sizeof(double) * (size_t)(Lmax + 1));
    double *A = (double *)malloc(sizeof(double) * (size_t)(Lmax + 1) * (size_t)r);
    double *Ax = (double *)malloc(sizeof(double) * (size_t)(Lmax + 1));
    double *x = (double *)malloc(sizeof(double) * (size_t)r);
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)r);
    for (int64_t u = J->u0; u < J->u1; ++u) {
        int64_t b = J->ptr[u], L = J->ptr[u + 1] - b;
        for (int64_t p = 0; p < L; ++p) {
            v[p] = (double)J->val[b + p];
            int64_t col = J->idx[b + p];
            for (int32_t k = 0; k < r; ++k) A[p * r + k] = J->Aside[(int64_t)k * J->na + col];
        }
        for (int32_t k = 0; k < r; ++k) x[k] = J->X[(int64_t)k * J->nx + u];
        oracle_perm(J->seed, J->sweep, J->side, u, J->cfg->perm_mode, r, ids);
        oracle_cfg cu = *J->cfg;
        cu.perturb_seed = J->cfg->perturb_seed ^ ((uint64_t)u * 0xD1B54A32D192ED03ULL) ^
                          ((uint64_t)(J->sweep + 1) * 0x9E3779B97F4A7C15ULL) ^ ((uint64_t)J->side << 62);
        oracle_alg2(L, v, A, J->sumA, x, r, ids, &cu, Ax, &J->st);
        for (int32_t k = 0; k < r; ++k) J->X[(int64_t)k * J->nx + u] = x[k];
    }
    free(v); free(A); free(Ax); free(x); free(ids);
    return NULL;
}

/* One half of Algorithm 1.
 * side 0 (F half): units are the m columns of V (CSC ptr/idx/val), A = W^T,
 *                  sumA = sumW = W 1, X = F (r x m), alpha2/beta2 in cfg.
 * side 1 (W half): units are the n rows of V (CSR), A = F^T, sumA = sumF,
 *                  X = W (r x n), alpha1/beta1 in cfg.
 * `other` is the fixed factor (W for side 0, F for side 1) with `n_other`
 * columns. Runs on `threads` threads over contiguous unit ranges; the result
 * does not depend on the thread count. stats may be NULL. */
void oracle_half(int32_t side, int64_t units, const int64_t *ptr, const int32_t *idx, const float *val,
                 const double *other, int64_t n_other, double *X, int32_t r, uint64_t seed,
                 int64_t sweep, const oracle_cfg *cfg, int32_t threads, oracle_stats *stats) {
    double *sumA = (double *)malloc(sizeof(double) * (size_t)r);
    oracle_rowsum(other, r, n_other, sumA);
    if (threads < 1) threads = 1;
    if (threads > units && units > 0) threads = (int32_t)units;
    half_job *jobs = (half_job *)calloc((size_t)threads, sizeof(half_job));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int32_t t = 0; t < threads; ++t) {
        half_job *J = &jobs[t];
        J->ptr = ptr; J->idx = idx; J->val = val; J->Aside = other; J->na = n_other;
        J->X = X; J->nx = units; J->sumA = sumA; J->r = r; J->side = side; J->sweep = sweep;
        J->seed = seed; J->cfg = cfg;
        J->u0 = units * t / threads; J->u1 = units * (t + 1) / threads;
        if (threads == 1) half_worker(J); else pthread_create(&th[t], NULL, half_worker, J);
    }
    if (threads > 1) for (int32_t t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    if (stats) {
        for (int32_t t = 0; t < threads; ++t) {
            stats->coords += jobs[t].st.coords; stats->evals += jobs[t].st.evals;
            stats->steps += jobs[t].st.steps; stats->cap_hits += jobs[t].st.cap_hits;
        }
    }
    free(jobs); free(th); free(sumA);
}

/* ---------------------------------------------------------------------- */
/* Objective, Eq. 1 and Eq. 2                                              */
/* ---------------------------------------------------------------------- */
/* kl = sum over nonzeros of V of [v log(v / (x + eps_div)) - v] + sum_ij x_ij,
 * where the last sum is sum_k (W 1)_k (F 1)_k since sum_ij [W^T F]_ij
 * factors that way; zero entries of V contribute x_ij only (0 log 0 = 0).
 * reg = a1/2 |W|^2 + a2/2 |F|^2 + b1 |W|_1 + b2 |F|_1. */
void oracle_objective(int64_t n, int64_t m, int32_t r, const int64_t *colptr, const int32_t *rowidx,
                      const float *val, const double *W, const double *F, double eps_div,
                      double a1, double a2, double b1, double b2, double *kl, double *reg) {
    double s = 0.0;
    for (int64_t j = 0; j < m; ++j)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            int64_t i = rowidx[p];
            double x = 0.0;
            for (int32_t k = 0; k < r; ++k) x += W[(int64_t)k * n + i] * F[(int64_t)k * m + j];
            double v = (double)val[p];
            s += v * log(v / (x + eps_div)) - v;
        }
    double *sw = (double *)malloc(sizeof(double) * (size_t)r);
    double *sf = (double *)malloc(sizeof(double) * (size_t)r);
    oracle_rowsum(W, r, n, sw);
    oracle_rowsum(F, r, m, sf);
    for (int32_t k = 0; k < r; ++k) s += sw[k] * sf[k];
    free(sw); free(sf);
    double w2 = 0.0, w1 = 0.0, f2 = 0.0, f1 = 0.0;
    for (int64_t e = 0; e < (int64_t)r * n; ++e) { w2 += W[e] * W[e]; w1 += fabs(W[e]); }
    for (int64_t e = 0; e < (int64_t)r * m; ++e) { f2 += F[e] * F[e]; f1 += fabs(F[e]); }
    *kl = s;
    *reg = 0.5 * a1 * w2 + 0.5 * a2 * f2 + b1 * w1 + b2 * f1;
}

/* Subproblem objective of Eq. kl for one column j (F side) at the current
 * F: sum_p [v log(v/(x_p+eps)) - v] + sum_k sumW_k F_kj + alpha/2|f|^2 + beta|f|_1. */
double oracle_column_objective(int64_t n, int64_t m, int32_t r, const int64_t *colptr,
                               const int32_t *rowidx, const float *val, const double *W,
                               const double *sumW, const double *F, int64_t j, double eps_div,
                               double alpha, double beta) {
    double s = 0.0;
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
        int64_t i = rowidx[p];
        double x = 0.0;
        for (int32_t k = 0; k < r; ++k) x += W[(int64_t)k * n + i] * F[(int64_t)k * m + j];
        double v = (double)val[p];
        s += v * log(v / (x + eps_div)) - v;
    }
    for (int32_t k = 0; k < r; ++k) {
        double f = F[(int64_t)k * m + j];
        s += sumW[k] * f + 0.5 * alpha * f * f + beta * fabs(f);
    }
    return s;
}

/* Algorithm 1: `sweeps` outer iterations from the given W, F (updated in
 * place). One sweep is the F half followed by the W half; sweep indices
 * start at sweep0. kl_trace[s] (may be NULL) receives Eq. 1 after sweep s. */
void oracle_fit(int64_t n, int64_t m, int32_t r, const int64_t *colptr, const int32_t *rowidx,
                const float *val, const int64_t *rowptr, const int32_t *colidx, const float *rval,
                double *W, double *F, uint64_t seed, int64_t sweep0, int32_t sweeps,
                const oracle_cfg *cfgF, const oracle_cfg *cfgW, int32_t threads,
                double *kl_trace, oracle_stats *stats) {
    for (int32_t s = 0; s < sweeps; ++s) {
        oracle_half(0, m, colptr, rowidx, val, W, n, F, r, seed, sweep0 + s, cfgF, threads, stats);
        oracle_half(1, n, rowptr, colidx, rval, F, m, W, r, seed, sweep0 + s, cfgW, threads, stats);
        if (kl_trace) {
            double kl, reg;
            oracle_objective(n, m, r, colptr, rowidx, val, W, F, cfgF->eps_div,
                             cfgW->alpha, cfgF->alpha, cfgW->beta, cfgF->beta, &kl, &reg);
            kl_trace[s] = kl;
        }
    }
}

/* Fold-in: W fixed, solve F for m new documents (columns). Document j runs
 * F-half sweeps s = 0, 1, ... on its own column until the change of its
 * subproblem objective (Eq. kl) is at most rel_tol times its previous value,
 * or max_sweeps.
 * sweeps_done[j] (may be NULL) receives the count. */
void oracle_foldin(int64_t n, int64_t m, int32_t r, const int64_t *colptr, const int32_t *rowidx,
                   const float *val, const double *W, double *F, uint64_t seed, double rel_tol,
                   int32_t max_sweeps, const oracle_cfg *cfg, int32_t *sweeps_done) {
    double *sumW = (double *)malloc(sizeof(double) * (size_t)r);
    oracle_rowsum(W, r, n, sumW);
    int64_t Lmax = 0;
    for (int64_t j = 0; j < m; ++j) { int64_t L = colptr[j + 1] - colptr[j]; if (L > Lmax) Lmax = L; }
    double *v = (double *)malloc(sizeof(double) * (size_t)(Lmax + 1));
    double *A = (double *)malloc(sizeof(double) * (size_t)(Lmax + 1) * (size_t)r);
    double *Ax = (double *)malloc(sizeof(double) * (size_t)(Lmax + 1));
    double *x = (double *)malloc(sizeof(double) * (size_t)r);
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)r);
    for (int64_t j = 0; j < m; ++j) {
        int64_t b = colptr[j], L = colptr[j + 1] - b;
        for (int64_t p = 0; p < L; ++p) {
            v[p] = (double)val[b + p];
            for (int32_t k = 0; k < r; ++k) A[p * r + k] = W[(int64_t)k * n + rowidx[b + p]];
        }
        for (int32_t k = 0; k < r; ++k) x[k] = F[(int64_t)k * m + j];
        double prev = oracle_column_objective(n, m, r, colptr, rowidx, val, W, sumW, F, j,
                                              cfg->eps_div, cfg->alpha, cfg->beta);
        int32_t s = 0;
        while (s < max_sweeps) {
            oracle_perm(seed, s, 0, j, cfg->perm_mode, r, ids);
            oracle_alg2(L, v, A, sumW, x, r, ids, cfg, Ax, NULL);
            for (int32_t k = 0; k < r; ++k) F[(int64_t)k * m + j] = x[k];
            ++s;
            double cur = oracle_column_objective(n, m, r, colptr, rowidx, val, W, sumW, F, j,
                                                 cfg->eps_div, cfg->alpha, cfg->beta);
            double change = fabs(prev - cur);
            int done = change <= rel_tol * fabs(prev);
            prev = cur;
            if (done) break;
        }
        if (sweeps_done) sweeps_done[j] = s;
    }
    free(sumW); free(v); free(A); free(Ax); free(x); free(ids);
}
