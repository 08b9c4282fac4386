/*
 * Seeded synthetic count matrices shaped like document/word data.
 *
 * This file is the input generator shared by the tests, the benchmark and the
 * oracle's callers. It draws random numbers and builds sparse storage only; it
 * contains none of the factorization arithmetic.
 *
 * Corpus model (the paper's workloads are tf-idf / count document sets, Table 1):
 *   - K topics; topic z is a Zipf(s) law over its own random permutation of
 *     the n-word vocabulary (rank t has mass t^-s / H, t = 1..n).
 *   - document j: topic weights theta_j ~ Dirichlet(a0 * 1_K); length
 *     L_j ~ LogNormal(mu, sigma) rounded, at least 1 token; each token picks a
 *     topic from theta_j and then a word from that topic; token counts are
 *     aggregated per (word, document).
 *   - fold-in documents instead fix the number of DISTINCT words d_j
 *     (drawn by the caller) and draw tokens until d_j distinct words are seen
 *     (or a token cap of 400*d_j is reached).
 * Output is CSC (document = column): colptr int64[m+1], rowidx int32[nnz]
 * sorted within each column, val float32[nnz] > 0.
 *
 * Every document draws from its own stream (xoshiro256** seeded by splitmix64
 * of (seed, document index)), so the output does not depend on the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- random streams ---------------- */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static void rng_seed(rng_t *g, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ULL + 0x2545F4914F6CDD1DULL);
    for (int i = 0; i < 4; ++i) g->s[i] = splitmix64(&x);
}
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t rng_next(rng_t *g) {
    uint64_t *s = g->s;
    uint64_t out = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return out;
}
/* uniform in (0,1): never exactly 0, so logs and powers are safe */
static inline double rng_u01(rng_t *g) { return ((double)(rng_next(g) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
static double rng_normal(rng_t *g) {
    double u1 = rng_u01(g), u2 = rng_u01(g);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
/* Gamma(shape a, scale 1): Marsaglia & Tsang (2000); a < 1 via the U^(1/a) boost. */
static double rng_gamma(rng_t *g, double a) {
    if (a < 1.0) {
        double u = rng_u01(g);
        return rng_gamma(g, a + 1.0) * pow(u, 1.0 / a);
    }
    double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
    for (;;) {
        double z, v;
        do { z = rng_normal(g); v = 1.0 + c * z; } while (v <= 0.0);
        v = v * v * v;
        double u = rng_u01(g);
        if (u < 1.0 - 0.0331 * z * z * z * z) return d * v;
        if (log(u) < 0.5 * z * z + d * (1.0 - v + log(v))) return d * v;
    }
}

/* ---------------- corpus tables ---------------- */
typedef struct {
    int64_t n;          /* vocabulary size */
    int K;              /* topics */
    double *zcdf;       /* n: cumulative Zipf mass, zcdf[n-1] = 1 */
    int32_t *perm;      /* K*n: perm[z*n + t] = word of rank t in topic z */
} corpus_t;

static void corpus_build(corpus_t *c, int64_t n, int K, double s, uint64_t seed) {
    c->n = n; c->K = K;
    c->zcdf = (double *)malloc(sizeof(double) * (size_t)n);
    c->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)K);
    double acc = 0.0;
    for (int64_t t = 0; t < n; ++t) { acc += pow((double)(t + 1), -s); c->zcdf[t] = acc; }
    for (int64_t t = 0; t < n; ++t) c->zcdf[t] /= acc;
    c->zcdf[n - 1] = 1.0;
    for (int z = 0; z < K; ++z) {
        rng_t g; rng_seed(&g, seed, 0xC0FFEE00ULL + (uint64_t)z);
        int32_t *p = c->perm + (size_t)z * (size_t)n;
        for (int64_t t = 0; t < n; ++t) p[t] = (int32_t)t;
        for (int64_t t = n - 1; t > 0; --t) {
            int64_t u = (int64_t)(rng_u01(&g) * (double)(t + 1));
            if (u > t) u = t;
            int32_t tmp = p[t]; p[t] = p[u]; p[u] = tmp;
        }
    }
}
static void corpus_free(corpus_t *c) { free(c->zcdf); free(c->perm); }

static inline int64_t zipf_rank(const corpus_t *c, rng_t *g) {
    double u = rng_u01(g);
    int64_t lo = 0, hi = c->n - 1;
    while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (c->zcdf[mid] < u) lo = mid + 1; else hi = mid; }
    return lo;
}

/* ---------------- per-thread output buffers ---------------- */
typedef struct {
    int32_t *idx; float *val; int64_t len, cap;
} buf_t;
static void buf_push(buf_t *b, int32_t i, float v) {
    if (b->len == b->cap) {
        b->cap = b->cap ? b->cap * 2 : 1 << 16;
        b->idx = (int32_t *)realloc(b->idx, sizeof(int32_t) * (size_t)b->cap);
        b->val = (float *)realloc(b->val, sizeof(float) * (size_t)b->cap);
    }
    b->idx[b->len] = i; b->val[b->len] = v; b->len++;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

typedef struct {
    const corpus_t *c;
    uint64_t seed;
    int64_t j0, j1;             /* documents [j0, j1) */
    double dir_a, mu, sigma;    /* Dirichlet concentration, lognormal length */
    const int32_t *distinct;    /* fold-in: target distinct words per doc (NULL: lengths) */
    int64_t *col_nnz;           /* out: per-document nnz (global array) */
    buf_t out;
} job_t;

static void *doc_worker(void *arg) {
    job_t *J = (job_t *)arg;
    const corpus_t *c = J->c;
    int K = c->K;
    double *cth = (double *)malloc(sizeof(double) * (size_t)K);
    int64_t tcap = 1024;
    int32_t *tok = (int32_t *)malloc(sizeof(int32_t) * (size_t)tcap);
    uint8_t *seen = J->distinct ? (uint8_t *)calloc((size_t)c->n, 1) : NULL;
    for (int64_t j = J->j0; j < J->j1; ++j) {
        rng_t g; rng_seed(&g, J->seed, (uint64_t)j);
        double tot = 0.0;
        for (int z = 0; z < K; ++z) { double x = rng_gamma(&g, J->dir_a); tot += x; cth[z] = tot; }
        if (!(tot > 0.0)) { for (int z = 0; z < K; ++z) cth[z] = (double)(z + 1); tot = (double)K; }
        int64_t L = 0, target = 0, distinct = 0, cap_tokens = 0;
        if (J->distinct) { target = J->distinct[j]; cap_tokens = 400 * target; }
        else {
            double len = exp(J->mu + J->sigma * rng_normal(&g));
            L = (int64_t)floor(len + 0.5);
            if (L < 1) L = 1;
        }
        int64_t nt = 0;
        for (;;) {
            if (J->distinct) { if (distinct >= target || nt >= cap_tokens) break; }
            else if (nt >= L) break;
            double u = rng_u01(&g) * tot;
            int z = 0;
            while (z < K - 1 && cth[z] < u) ++z;
            int64_t t = zipf_rank(c, &g);
            int32_t w = c->perm[(size_t)z * (size_t)c->n + (size_t)t];
            if (nt == tcap) { tcap *= 2; tok = (int32_t *)realloc(tok, sizeof(int32_t) * (size_t)tcap); }
            tok[nt++] = w;
            if (seen && !seen[w]) { seen[w] = 1; ++distinct; }
        }
        qsort(tok, (size_t)nt, sizeof(int32_t), cmp_i32);
        int64_t cnt = 0;
        for (int64_t a = 0; a < nt;) {
            int64_t b = a;
            while (b < nt && tok[b] == tok[a]) ++b;
            buf_push(&J->out, tok[a], (float)(b - a));
            if (seen) seen[tok[a]] = 0;
            ++cnt; a = b;
        }
        J->col_nnz[j] = cnt;
    }
    free(cth); free(tok); free(seen);
    return NULL;
}

typedef struct {
    int64_t m, nnz;
    int64_t *col_nnz;
    int nthreads;
    job_t *jobs;
} synth_handle;

static synth_handle *run_docs(int64_t n, int64_t m, int K, double zipf_s, double dir_a,
                              double mu, double sigma, const int32_t *distinct,
                              uint64_t seed, int nthreads) {
    if (n <= 0 || m < 0 || K <= 0 || nthreads <= 0) return NULL;
    corpus_t *c = (corpus_t *)malloc(sizeof(corpus_t));
    corpus_build(c, n, K, zipf_s, seed);
    synth_handle *h = (synth_handle *)calloc(1, sizeof(synth_handle));
    h->m = m; h->nthreads = nthreads;
    h->col_nnz = (int64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(int64_t));
    h->jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        job_t *J = &h->jobs[t];
        J->c = c; J->seed = seed; J->dir_a = dir_a; J->mu = mu; J->sigma = sigma;
        J->distinct = distinct; J->col_nnz = h->col_nnz;
        J->j0 = m * t / nthreads; J->j1 = m * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, doc_worker, J);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    h->nnz = 0;
    for (int t = 0; t < nthreads; ++t) h->nnz += h->jobs[t].out.len;
    corpus_free(c); free(c);
    return h;
}

/* Generates a corpus; returns an opaque handle (NULL on bad arguments).
 * Length mode: L ~ LogNormal(mu, sigma). */
void *synth_docs(int64_t n, int64_t m, int32_t K, double zipf_s, double dir_a,
                 double mu, double sigma, uint64_t seed, int32_t nthreads) {
    return run_docs(n, m, K, zipf_s, dir_a, mu, sigma, NULL, seed, nthreads);
}
/* Fold-in mode: distinct[j] distinct words for document j. */
void *synth_docs_distinct(int64_t n, int64_t m, int32_t K, double zipf_s, double dir_a,
                          const int32_t *distinct, uint64_t seed, int32_t nthreads) {
    return run_docs(n, m, K, zipf_s, dir_a, 0.0, 0.0, distinct, seed, nthreads);
}
int64_t synth_nnz(void *hv) { return hv ? ((synth_handle *)hv)->nnz : -1; }
/* Copies the CSC arrays out and frees the handle. */
void synth_fetch(void *hv, int64_t *colptr, int32_t *rowidx, float *val) {
    synth_handle *h = (synth_handle *)hv;
    colptr[0] = 0;
    for (int64_t j = 0; j < h->m; ++j) colptr[j + 1] = colptr[j] + h->col_nnz[j];
    int64_t off = 0;
    for (int t = 0; t < h->nthreads; ++t) {
        buf_t *b = &h->jobs[t].out;
        if (b->len) {
            memcpy(rowidx + off, b->idx, sizeof(int32_t) * (size_t)b->len);
            memcpy(val + off, b->val, sizeof(float) * (size_t)b->len);
        }
        off += b->len;
        free(b->idx); free(b->val);
    }
    free(h->jobs); free(h->col_nnz); free(h);
}

/* Topic-word distributions (K x n, row-major, each row sums to 1) of the same
 * corpus tables the documents are drawn from with this seed. */
void synth_topics(int64_t n, int32_t K, double zipf_s, uint64_t seed, float *W) {
    corpus_t c; corpus_build(&c, n, K, zipf_s, seed);
    for (int z = 0; z < K; ++z) {
        float *row = W + (size_t)z * (size_t)n;
        double prev = 0.0;
        for (int64_t t = 0; t < n; ++t) {
            row[c.perm[(size_t)z * (size_t)n + (size_t)t]] = (float)(c.zcdf[t] - prev);
            prev = c.zcdf[t];
        }
    }
    corpus_free(&c);
}

/* CSC (n x m) -> CSR of the same matrix (counting sort; indices stay sorted). */
void synth_transpose(int64_t n, int64_t m, const int64_t *colptr, const int32_t *rowidx,
                     const float *val, int64_t *rowptr, int32_t *colidx, float *rval) {
    memset(rowptr, 0, sizeof(int64_t) * (size_t)(n + 1));
    int64_t nnz = colptr[m];
    for (int64_t p = 0; p < nnz; ++p) rowptr[rowidx[p] + 1]++;
    for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    memcpy(fill, rowptr, sizeof(int64_t) * (size_t)n);
    for (int64_t j = 0; j < m; ++j)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            int64_t q = fill[rowidx[p]]++;
            colidx[q] = (int32_t)j; rval[q] = val[p];
        }
    free(fill);
}

/* Poisson means of a masked low-rank count matrix at given entries:
 * lam[p] = sum_k wtT[rows[p]*r + k] * ftT[cols[p]*r + k] (unit-major factors),
 * split over `threads` threads by entry range. */
typedef struct {
    int64_t p0, p1;
    int32_t r;
    const double *wtT, *ftT;
    const int64_t *rows, *cols;
    double *lam;
} lam_job;

static void *lam_worker(void *arg) {
    lam_job *J = (lam_job *)arg;
    for (int64_t p = J->p0; p < J->p1; ++p) {
        const double *a = J->wtT + J->rows[p] * J->r, *b = J->ftT + J->cols[p] * J->r;
        double s = 0.0;
        for (int32_t k = 0; k < J->r; ++k) s += a[k] * b[k];
        J->lam[p] = s;
    }
    return NULL;
}

void synth_lowrank_means(int64_t nnz, int32_t r, const double *wtT, const double *ftT, const int64_t *rows,
                         const int64_t *cols, double *lam, int32_t nthreads) {
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    lam_job *jobs = (lam_job *)malloc(sizeof(lam_job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].p0 = nnz * t / nthreads;
        jobs[t].p1 = nnz * (t + 1) / nthreads;
        jobs[t].r = r;
        jobs[t].wtT = wtT;
        jobs[t].ftT = ftT;
        jobs[t].rows = rows;
        jobs[t].cols = cols;
        jobs[t].lam = lam;
        pthread_create(&th[t], NULL, lam_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
}
