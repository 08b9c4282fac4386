// Supporting kernels: sumA (Algorithm 1's sumW = W 1, sumF = F 1), the
// objective of Eq. 1/2, random initialisation, layout transposes and input
// validation. Every reduction runs in a fixed order (block partials, then
// one ordered pass), so results are bitwise reproducible.
#include "common.cuh"

#include <cmath>

namespace nmfkl {

namespace {

constexpr int kColsumBlocks = 1024;
constexpr int kObjBlocks = 2048;

// Stage 1 of sum over rows of At (rows x ldr, ldr a multiple of 4): block b
// covers a contiguous row range; thread t owns the four columns 4g..4g+3, g =
// t % (ldr / 4), of rows t / (ldr / 4), + rpi, ... (16-byte loads, four
// independent FP64 sums per thread); the block then adds its row groups in
// order.
__global__ void colsum_partial_kernel(const float *At, int64_t rows, int ldr, double *part) {
    __shared__ double4 acc[256];
    const int t = threadIdx.x;
    const int nf4 = ldr >> 2;
    const int rpi = 256 / nf4;
    const int g = t % nf4, ro = t / nf4;
    const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(rows, r0 + per);
    double4 s = make_double4(0.0, 0.0, 0.0, 0.0);
    if (ro < rpi) {
        const float4 *src = reinterpret_cast<const float4 *>(At) + g;
        for (int64_t row = r0 + ro; row < r1; row += rpi) {
            const float4 v = __ldg(src + row * nf4);
            s.x += (double)v.x;
            s.y += (double)v.y;
            s.z += (double)v.z;
            s.w += (double)v.w;
        }
    }
    acc[t] = s;
    __syncthreads();
    if (t < nf4) {
        double4 tot = make_double4(0.0, 0.0, 0.0, 0.0);
        for (int j = 0; j < rpi; ++j) {
            const double4 v = acc[j * nf4 + t];
            tot.x += v.x;
            tot.y += v.y;
            tot.z += v.z;
            tot.w += v.w;
        }
        double *out = part + (int64_t)blockIdx.x * ldr + 4 * t;
        out[0] = tot.x;
        out[1] = tot.y;
        out[2] = tot.z;
        out[3] = tot.w;
    }
}

__global__ void colsum_final_kernel(const double *part, int nblocks, int ldr, int r, float *out,
                                    double *out_d) {
    for (int k = threadIdx.x; k < ldr; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * ldr + k];
        if (out) out[k] = k < r ? (float)s : 0.f;
        if (out_d) out_d[k] = k < r ? s : 0.0;
    }
}

// Eq. 1 over the nonzeros: one warp per column j (CSC), F^T row j in shared
// memory, one lane per nonzero computing x_ij = <W^T_i, F^T_j> in FP32 and
// the term v log(v / (x + eps)) - v in FP32, accumulated in FP64.
__global__ void objective_nnz_kernel(const int64_t *colptr, const int32_t *rowidx, const float *val,
                                     const float *Wt, const float *Ft, int64_t m, int ldr, float eps_div,
                                     double *part) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ double wsum[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *frow = reinterpret_cast<float4 *>(fsm + w * ldr);
    const int nf4 = ldr >> 2;
    double acc = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * 8 + w; j < m; j += (int64_t)gridDim.x * 8) {
        __syncwarp();
        for (int f = lane; f < nf4; f += 32) frow[f] = reinterpret_cast<const float4 *>(Ft + j * ldr)[f];
        __syncwarp();
        for (int64_t p = colptr[j] + lane; p < colptr[j + 1]; p += 32) {
            const float4 *wr = reinterpret_cast<const float4 *>(Wt + (int64_t)rowidx[p] * ldr);
            float x = 0.f;
            for (int f = 0; f < nf4; ++f) {
                const float4 a = __ldg(wr + f), b = frow[f];
                x = fmaf(a.x, b.x, x);
                x = fmaf(a.y, b.y, x);
                x = fmaf(a.z, b.z, x);
                x = fmaf(a.w, b.w, x);
            }
            const float v = val[p];
            acc += (double)(v * logf(v / (x + eps_div)) - v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) wsum[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += wsum[i];
        part[blockIdx.x] = s;
    }
}

// Sums of squares and absolute values of a unit-major factor (pads are 0).
__global__ void sq_abs_kernel(const float *X, int64_t count, double *part2, double *part1) {
    __shared__ double s2[256], s1[256];
    double a2 = 0.0, a1 = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < count; e += (int64_t)gridDim.x * 256) {
        const double v = (double)X[e];
        a2 += v * v;
        a1 += fabs(v);
    }
    s2[threadIdx.x] = a2;
    s1[threadIdx.x] = a1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s2[threadIdx.x] += s2[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part2[blockIdx.x] = s2[0];
        part1[blockIdx.x] = s1[0];
    }
}

// kl = sum of nnz partials + sum_k sumW_k sumF_k;
// reg = a1/2 |W|^2 + a2/2 |F|^2 + b1 |W|_1 + b2 |F|_1.
__global__ void objective_final_kernel(const double *nnzpart, int nb, const double *sw, const double *sf,
                                       int r, const double *regpart, int nreg, double a1, double a2,
                                       double b1, double b2, double *out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += nnzpart[b];
    for (int k = 0; k < r; ++k) s += sw[k] * sf[k];
    double w2 = 0.0, w1 = 0.0, f2 = 0.0, f1 = 0.0;
    for (int b = 0; b < nreg; ++b) {
        w2 += regpart[b];
        w1 += regpart[nreg + b];
        f2 += regpart[2 * nreg + b];
        f1 += regpart[3 * nreg + b];
    }
    out[0] = s;
    out[1] = 0.5 * a1 * w2 + 0.5 * a2 * f2 + b1 * w1 + b2 * f1;
}

// Uniform[0,1) from Philox: entry e (row-major r x cols) -> X[c*ldr + k].
__global__ void uniform_init_kernel(float *X, int r, int64_t cols, int ldr, uint64_t seed, int which) {
    const int64_t total = (int64_t)r * cols;
    for (int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; blk * 4 < total;
         blk += (int64_t)gridDim.x * blockDim.x) {
        uint64_t c[4] = {(uint64_t)blk, (uint64_t)which, 0ull, 0ull};
        philox4x64_10(c, seed, kKeyInit);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t e = blk * 4 + j;
            if (e < total) {
                const int64_t k = e / cols, col = e - k * cols;
                X[col * ldr + k] = (float)(c[j] >> 40) * (1.0f / 16777216.0f);
            }
        }
    }
}

// r x cols row-major  <->  cols x ldr unit-major (pad columns zero).
__global__ void to_unit_major_kernel(const float *src, float *dst, int r, int64_t cols, int ldr) {
    __shared__ float t[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int k = k0 + i;
        const int64_t c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (k < r && c < cols) ? src[(int64_t)k * cols + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t c = c0 + i;
        const int k = k0 + threadIdx.x;
        if (c < cols && k < ldr) dst[c * ldr + k] = t[threadIdx.x][i];
    }
}

__global__ void from_unit_major_kernel(const float *src, float *dst, int r, int64_t cols, int ldr) {
    __shared__ float t[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t c = c0 + i;
        const int k = k0 + threadIdx.x;
        t[i][threadIdx.x] = (c < cols && k < r) ? src[c * ldr + k] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int k = k0 + i;
        const int64_t c = c0 + threadIdx.x;
        if (k < r && c < cols) dst[(int64_t)k * cols + c] = t[threadIdx.x][i];
    }
}

// flag bit 1: offsets not monotone or out of [0, nnz]; 2: index out of range
// or not strictly increasing; 4: value not finite or <= 0.
// One warp per unit, lanes over its entries (coalesced; a unit of any length
// costs its entries / 32 steps): offsets in [0, nnz] and non-decreasing (flag
// 1), indices in [0, extent) and strictly increasing within the unit (2),
// values finite and > 0 (4).
__global__ void validate_kernel(int64_t units, int64_t extent, int64_t nnz, const int64_t *ptr,
                                const int32_t *idx, const float *val, int32_t *flag) {
    // nnz is the caller's count (the size of idx and val), not ptr[units]:
    // offsets past it are refused before any entry is read
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += warps) {
        const int64_t b = ptr[u], e = ptr[u + 1];
        if (b > e || b < 0 || e > nnz) {
            if (lane == 0) atomicOr(flag, 1);
            continue;
        }
        int bad = 0;
        for (int64_t p = b + lane; p < e; p += 32) {
            const int32_t i = idx[p];
            if (i < 0 || i >= extent || (p > b && idx[p - 1] >= i)) bad |= 2;
            const float v = val[p];
            if (!(v > 0.f) || !isfinite(v)) bad |= 4;
        }
        bad = __reduce_or_sync(0xffffffffu, bad);
        if (lane == 0 && bad) atomicOr(flag, bad);
    }
}

}  // namespace

nmfkl_status launch_colsum(nmfkl_ctx *c, const float *At, int64_t rows, float *out, double *out_d) {
    const int tok = timer_begin(c, "colsum");
    colsum_partial_kernel<<<kColsumBlocks, 256, 0, c->stream>>>(At, rows, c->ldr, c->dpart);
    colsum_final_kernel<<<1, 256, 0, c->stream>>>(c->dpart, kColsumBlocks, c->ldr, c->p.r, out, out_d);
    timer_end(c, tok);
    return cuda_ok(c, cudaGetLastError(), "colsum") ? NMFKL_OK : NMFKL_ECUDA;
}

nmfkl_status launch_objective(nmfkl_ctx *c, double *kl, double *reg) {
    const int ldr = c->ldr, r = c->p.r;
    // dpart layout: [colsum partials kColsumBlocks*ldr][sumW_d ldr][sumF_d ldr][nnz kObjBlocks][reg 4*kObjBlocks]
    double *sw = c->dpart + (int64_t)kColsumBlocks * ldr;
    double *sf = sw + ldr;
    double *nnzp = sf + ldr;
    double *regp = nnzp + kObjBlocks;
    const int tok = timer_begin(c, "objective");
    colsum_partial_kernel<<<kColsumBlocks, 256, 0, c->stream>>>(c->Wt, c->n, ldr, c->dpart);
    colsum_final_kernel<<<1, 256, 0, c->stream>>>(c->dpart, kColsumBlocks, ldr, r, nullptr, sw);
    colsum_partial_kernel<<<kColsumBlocks, 256, 0, c->stream>>>(c->Ft, c->m, ldr, c->dpart);
    colsum_final_kernel<<<1, 256, 0, c->stream>>>(c->dpart, kColsumBlocks, ldr, r, nullptr, sf);
    objective_nnz_kernel<<<kObjBlocks, 256, 8 * ldr * sizeof(float), c->stream>>>(
        c->colptr, c->rowidx, c->val, c->Wt, c->Ft, c->m, ldr, (float)c->p.eps_div, nnzp);
    sq_abs_kernel<<<kObjBlocks, 256, 0, c->stream>>>(c->Wt, c->n * ldr, regp, regp + kObjBlocks);
    sq_abs_kernel<<<kObjBlocks, 256, 0, c->stream>>>(c->Ft, c->m * ldr, regp + 2 * kObjBlocks,
                                                      regp + 3 * kObjBlocks);
    objective_final_kernel<<<1, 32, 0, c->stream>>>(nnzp, kObjBlocks, sw, sf, r, regp, kObjBlocks,
                                                    c->p.alpha_W, c->p.alpha_F, c->p.beta_W, c->p.beta_F,
                                                    c->dscalar);
    timer_end(c, tok);
    if (!cuda_ok(c, cudaGetLastError(), "objective")) return NMFKL_ECUDA;
    double h[2];
    if (!cuda_ok(c, cudaMemcpyAsync(h, c->dscalar, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy objective"))
        return NMFKL_ECUDA;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream), "objective sync")) return NMFKL_ECUDA;
    if (kl) *kl = h[0];
    if (reg) *reg = h[1];
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) {
        c->err = "objective is not finite";
        return NMFKL_ENUMERIC;
    }
    return NMFKL_OK;
}

// Eq. 1 after a W half: the per-row data terms the W half left in unit_obj
// (summed in row order) plus the closed form sum_k sumW_k sumF_k.
__global__ void fused_objective_kernel(const double *unit_obj, int64_t n, const double *sw, const double *sf,
                                       int r, double *out) {
    __shared__ double acc[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += unit_obj[i];
    acc[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) acc[threadIdx.x] += acc[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double t = acc[0];
        for (int k = 0; k < r; ++k) t += sw[k] * sf[k];
        out[0] = t;
    }
}

void launch_colsum_raw(cudaStream_t stream, const float *At, int64_t rows, int ldr, int r, double *part,
                       float *out, double *out_d) {
    colsum_partial_kernel<<<kColsumBlocks, 256, 0, stream>>>(At, rows, ldr, part);
    colsum_final_kernel<<<1, 256, 0, stream>>>(part, kColsumBlocks, ldr, r, out, out_d);
}

namespace {
// Sum of x[0..n) in FP64 by one block, in a fixed order (strided partial sums,
// then a tree over the threads).
__global__ void range_sum_kernel(const double *x, int64_t n, double *out) {
    __shared__ double part[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}
}  // namespace

nmfkl_status launch_range_sum(nmfkl_ctx *c, const double *x, int64_t n, double *out) {
    range_sum_kernel<<<1, 1024, 0, c->stream>>>(x, n, out);
    return cuda_ok(c, cudaGetLastError(), "range sum") ? NMFKL_OK : NMFKL_ECUDA;
}

nmfkl_status enqueue_fused_objective(nmfkl_ctx *c) {
    // sumF (FP64) is current from the W half; sumW changed in it, so sum W again.
    nmfkl_status st = launch_colsum(c, c->Wt, c->n, c->sumW, c->dsum[0]);
    if (st != NMFKL_OK) return st;
    const int tok = timer_begin(c, "objective_fused");
    fused_objective_kernel<<<1, 1024, 0, c->stream>>>(c->unit_obj, c->n, c->dsum[0], c->dsum[1], c->p.r, c->dscalar);
    timer_end(c, tok);
    return cuda_ok(c, cudaGetLastError(), "fused objective") ? NMFKL_OK : NMFKL_ECUDA;
}

nmfkl_status launch_fused_objective(nmfkl_ctx *c, double *kl) {
    nmfkl_status st = enqueue_fused_objective(c);
    if (st != NMFKL_OK) return st;
    double h = 0.0;
    if (!cuda_ok(c, cudaMemcpyAsync(&h, c->dscalar, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy objective") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "objective sync"))
        return NMFKL_ECUDA;
    if (kl) *kl = h;
    if (!std::isfinite(h)) {
        c->err = "objective is not finite";
        return NMFKL_ENUMERIC;
    }
    return NMFKL_OK;
}

int64_t dpart_required(int ldr) { return (int64_t)kColsumBlocks * ldr + 2 * ldr + 5 * kObjBlocks + 64; }

nmfkl_status launch_uniform_init(nmfkl_ctx *c, int which, float *X, int64_t cols) {
    const int tok = timer_begin(c, "uniform_init");
    uniform_init_kernel<<<1024, 256, 0, c->stream>>>(X, c->p.r, cols, c->ldr, c->p.seed, which);
    timer_end(c, tok);
    return cuda_ok(c, cudaGetLastError(), "uniform_init") ? NMFKL_OK : NMFKL_ECUDA;
}

void uniform_init_raw(cudaStream_t st, float *X, int r, int64_t cols, int ldr, uint64_t seed, int which) {
    uniform_init_kernel<<<1024, 256, 0, st>>>(X, r, cols, ldr, seed, which);
}

nmfkl_status launch_to_unit_major(nmfkl_ctx *c, const float *src, float *dst, int64_t cols) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((c->ldr + 31) / 32));
    const int tok = timer_begin(c, "transpose");
    to_unit_major_kernel<<<grid, dim3(32, 8), 0, c->stream>>>(src, dst, c->p.r, cols, c->ldr);
    timer_end(c, tok);
    return cuda_ok(c, cudaGetLastError(), "to_unit_major") ? NMFKL_OK : NMFKL_ECUDA;
}

nmfkl_status launch_from_unit_major(nmfkl_ctx *c, const float *src, float *dst, int64_t cols) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((c->p.r + 31) / 32));
    const int tok = timer_begin(c, "transpose");
    from_unit_major_kernel<<<grid, dim3(32, 8), 0, c->stream>>>(src, dst, c->p.r, cols, c->ldr);
    timer_end(c, tok);
    return cuda_ok(c, cudaGetLastError(), "from_unit_major") ? NMFKL_OK : NMFKL_ECUDA;
}

void launch_from_unit_major_raw(cudaStream_t st, const float *src, float *dst, int r, int64_t cols, int ldr) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((r + 31) / 32));
    from_unit_major_kernel<<<grid, dim3(32, 8), 0, st>>>(src, dst, r, cols, ldr);
}

__global__ void density_kernel(const float *At, int64_t rows, int ldr, int r, const int64_t *ptr,
                               unsigned long long *out) {
    // one warp per row: lanes read the row's coordinates, a ballot counts the positive ones
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < rows; i += warps) {
        const float *row = At + i * ldr;
        unsigned c = 0;
        for (int k0 = 0; k0 < r; k0 += 32) {
            const int k = k0 + lane;
            c += __popc(__ballot_sync(0xffffffffu, k < r && row[k] > 0.f));
        }
        acc += (unsigned long long)c * (unsigned long long)(ptr[i + 1] - ptr[i]);
    }
    if (lane == 0 && acc) atomicAdd(out, acc);
}

void launch_density(cudaStream_t st, const float *At, int64_t rows, int ldr, int r, const int64_t *ptr,
                    unsigned long long *out) {
    density_kernel<<<1024, 256, 0, st>>>(At, rows, ldr, r, ptr, out);
}

nmfkl_status launch_validate(nmfkl_ctx *c, int64_t units, int64_t extent, int64_t nnz, const int64_t *ptr,
                             const int32_t *idx, const float *val, int32_t *flag) {
    validate_kernel<<<4 * c->num_sms, 256, 0, c->stream>>>(units, extent, nnz, ptr, idx, val, flag);
    return cuda_ok(c, cudaGetLastError(), "validate") ? NMFKL_OK : NMFKL_ECUDA;
}

}  // namespace nmfkl
