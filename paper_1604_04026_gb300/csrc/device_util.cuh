// Device helpers shared by the sweep kernels of libnmfkl (sweep.cu and
// group.cu): asynchronous copies, coordinate orders, the x_p step, the
// projected Newton loop of Algorithm 2 and small reductions.
#pragma once

#include "common.cuh"

namespace nmfkl {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ constexpr int odd_stride(int r) { return (r & 1) ? r : r + 1; }
__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// 4-byte global -> shared copy; src_bytes 0 writes a zero.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, int src_bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
// 16-byte global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
// 16-byte copy of which only the first src_bytes (0..16) are read; the rest of
// the destination is zero-filled (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16z(void *dst, const void *src, int src_bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Swap index of Fisher-Yates step t over {0..r-1} (position i = r-1-t, n =
// i + 1 = r - t): j = floor(w n / 2^64) for the step's Philox word w, formed
// from the word's 32-bit halves (n < 2^32): the low half's product only
// carries its high half into the sum, and the sum stays below 2^64.
__device__ __forceinline__ int swap_index(uint64_t w, uint32_t n) {
    const uint64_t hi = (uint64_t)(uint32_t)(w >> 32) * n + __umulhi((uint32_t)w, n);
    return (int)(hi >> 32);
}

// Fisher-Yates over {0..r-1} from the identity: step t swaps position
// i = r-1-t with swaps[t] (from ids_swaps_warp).
__device__ __forceinline__ void fisher_yates(uint8_t *perm, const uint8_t *swaps, int r) {
    // the identity, four entries per 32-bit store (perm is 4-byte aligned and
    // holds r rounded up to a multiple of 4 bytes)
    for (int i = 0; i < r; i += 4) *reinterpret_cast<uint32_t *>(perm + i) = 0x03020100u + 0x01010101u * (uint32_t)i;
    int t = 0;
    for (int i = r - 1; i >= 1; --i, ++t) {
        const int j = swaps[t];
        const uint8_t tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
    }
}

// The r-1 swap indices of a unit's order, one byte each (r <= 256), from its
// r-1 Philox words, generated by `nlanes` lanes in parallel, so that the
// sequential shuffle (one lane) only moves entries.
__device__ __forceinline__ void ids_swaps_warp(uint8_t *swaps, int r, int64_t unit, int64_t sweep,
                                               int side, int perm_mode, uint64_t seed, int lane,
                                               int nlanes = 32) {
    const int nw = r - 1;
    const int nblk = (nw + 3) / 4;
    for (int b = lane; b < nblk; b += nlanes) {
        uint64_t c[4];
        ids_counter(c, (uint64_t)b, unit, sweep, side, perm_mode);
        philox4x64_10(c, seed, kKeyIds);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = 4 * b + j;
            if (t < nw) swaps[t] = (uint8_t)swap_index(c[j], (uint32_t)(r - t));
        }
    }
}

// x_p after a step of coordinate k: x_p + d A_pk, where `dc` (+1, -1 or 0)
// records whether x_k just became positive or just became zero. x_p is a
// sum of nonnegative terms A_pk x_k; `terms` counts the positive ones. When
// it reaches 0 the exact value is 0, and any FP32 residual left by the
// incremental updates is dropped; otherwise the value is kept >= 0.
__device__ __forceinline__ float step_x(float x, float av, float d, int dc, int &terms) {
    x = fmaf(d, av, x);
    if (dc == 0) return fmaxf(x, 0.f);  // no term appears or vanishes (dc is group-uniform)
    if (av > 0.f) terms += dc;
    return terms == 0 ? 0.f : fmaxf(x, 0.f);
}

// 1 / (x + eps) with the hardware approximation (relative error ~1 ulp;
// x + eps >= eps > 0, so no denormal or zero input).
__device__ __forceinline__ float recip(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The rest of step_x once x + d A_pk has been formed (by a packed fma).
__device__ __forceinline__ float finish_x(float x, float av, int dc, int &terms) {
    if (dc == 0) return fmaxf(x, 0.f);
    if (av > 0.f) terms += dc;
    return terms == 0 ? 0.f : fmaxf(x, 0.f);
}

// Packed FP32 pairs: one instruction performs two IEEE operations, each half
// rounded exactly as the scalar fmaf / multiplication / addition (sm_100 and
// later), so the per-nonzero loops issue half the arithmetic instructions.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(lo), "f"(hi));
    return v;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return make_float2(lo, hi);
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long fmul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// (a.x + b.x, a.y + b.y) in one packed instruction
__device__ __forceinline__ float2 add_pair(float2 a, float2 b) {
    return unpack2(fadd2(pack2(a.x, a.y), pack2(b.x, b.y)));
}

// One lane's share of an evaluation (Eq. Partial) over its staged nonzeros
// s < ks: (sum_s w_s a_s, sum_s q_s a_s^2) with a_s = ac[s * STRIDE], or, for
// kPiece (K a multiple of 4), a_s = ac[(s / 4) * STRIDE + s % 4], read as one
// float4 per piece of four (16-byte aligned). For even K the even and odd s
// are accumulated in the two halves of packed registers and added at the
// end; the entry after the last (s = ks, when ks is odd) must hold a finite
// value, its w and q being 0.
template <int K, int STRIDE, bool kPiece = false>
__device__ __forceinline__ float2 lane_sums(const float *ac, const float (&wr)[K], const float (&qr)[K], int ks) {
    static_assert(!kPiece || K % 4 == 0, "pieces of four entries");
    if constexpr (kPiece) {
        unsigned long long g = 0ull, h = 0ull;  // (+0, +0)
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const int s = 4 * q;
            if (s < ks) {
                const float4 v = *reinterpret_cast<const float4 *>(ac + q * STRIDE);
                const unsigned long long a01 = pack2(v.x, v.y), a23 = pack2(v.z, v.w);
                g = ffma2(pack2(wr[s], wr[s + 1]), a01, g);
                h = ffma2(fmul2(pack2(qr[s], qr[s + 1]), a01), a01, h);
                if (s + 2 < ks) {
                    g = ffma2(pack2(wr[s + 2], wr[s + 3]), a23, g);
                    h = ffma2(fmul2(pack2(qr[s + 2], qr[s + 3]), a23), a23, h);
                }
            }
        }
        const float2 gg = unpack2(g), hh = unpack2(h);
        return make_float2(gg.x + gg.y, hh.x + hh.y);
    } else if constexpr (K % 2 == 1) {
        float sg = 0.f, sh = 0.f;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (s < ks) {
                const float av = ac[s * STRIDE];
                sg = fmaf(wr[s], av, sg);
                sh = fmaf(qr[s] * av, av, sh);
            }
        }
        return make_float2(sg, sh);
    } else {
        unsigned long long g = 0ull, h = 0ull;  // (+0, +0)
#pragma unroll
        for (int s = 0; s < K; s += 2) {
            if (s < ks) {
                const unsigned long long a2 = pack2(ac[s * STRIDE], ac[(s + 1) * STRIDE]);
                g = ffma2(pack2(wr[s], wr[s + 1]), a2, g);
                h = ffma2(fmul2(pack2(qr[s], qr[s + 1]), a2), a2, h);
            }
        }
        const float2 gg = unpack2(g), hh = unpack2(h);
        return make_float2(gg.x + gg.y, hh.x + hh.y);
    }
}

// One pair of entries (s, s + 1) of an update, a0 and a1 their A entries.
template <int K>
__device__ __forceinline__ void pair_update(int s, float a0, float a1, float (&xr)[K], const float (&vr)[K],
                                            float (&wr)[K], float (&qr)[K], int (&cr)[K], unsigned long long d2,
                                            int dc, unsigned long long e2) {
    const float2 x = unpack2(ffma2(d2, pack2(a0, a1), pack2(xr[s], xr[s + 1])));
    xr[s] = finish_x(x.x, a0, dc, cr[s]);
    xr[s + 1] = finish_x(x.y, a1, dc, cr[s + 1]);
    const float2 t = unpack2(fadd2(pack2(xr[s], xr[s + 1]), e2));
    const unsigned long long ri = pack2(recip(t.x), recip(t.y));
    const unsigned long long w2 = fmul2(pack2(vr[s], vr[s + 1]), ri);
    const float2 w = unpack2(w2), q = unpack2(fmul2(w2, ri));
    wr[s] = w.x;
    wr[s + 1] = w.y;
    qr[s] = q.x;
    qr[s + 1] = q.y;
}

// One lane's share of an update (Algorithm 2, "Update Ax"): x_s += d a_s on
// its staged nonzeros s < ks with the positive-term counts, then w_s and q_s
// refreshed; the same operations, in the same rounding, as step_x and the
// scalar refresh. For even K the entry after the last (s = ks, ks odd) is
// updated too: its a_s is 0 and its state stays 0. a_s is addressed as in
// lane_sums.
template <int K, int STRIDE, bool kPiece = false>
__device__ __forceinline__ void lane_update(const float *ac, float (&xr)[K], const float (&vr)[K], float (&wr)[K],
                                            float (&qr)[K], int (&cr)[K], int ks, float d, int dc, float eps_div) {
    static_assert(!kPiece || K % 4 == 0, "pieces of four entries");
    if constexpr (kPiece) {
        const unsigned long long d2 = pack2(d, d), e2 = pack2(eps_div, eps_div);
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const int s = 4 * q;
            if (s < ks) {
                const float4 v = *reinterpret_cast<const float4 *>(ac + q * STRIDE);
                pair_update<K>(s, v.x, v.y, xr, vr, wr, qr, cr, d2, dc, e2);
                if (s + 2 < ks) pair_update<K>(s + 2, v.z, v.w, xr, vr, wr, qr, cr, d2, dc, e2);
            }
        }
    } else if constexpr (K % 2 == 1) {
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (s < ks) {
                xr[s] = step_x(xr[s], ac[s * STRIDE], d, dc, cr[s]);
                const float ri = recip(xr[s] + eps_div);
                wr[s] = vr[s] * ri;
                qr[s] = wr[s] * ri;
            }
        }
    } else {
        const unsigned long long d2 = pack2(d, d), e2 = pack2(eps_div, eps_div);
#pragma unroll
        for (int s = 0; s < K; s += 2) {
            if (s < ks) pair_update<K>(s, ac[s * STRIDE], ac[(s + 1) * STRIDE], xr, vr, wr, qr, cr, d2, dc, e2);
        }
    }
}

// Work counters of one thread (flushed once per kernel; a group processes far
// fewer than 2^32 coordinates).
struct Tally {
    unsigned coords = 0, evals = 0, steps = 0, caps = 0;
};

__device__ __forceinline__ void flush_tally(const HalfArgs &a, const Tally &t) {
    if (t.coords) atomicAdd(&a.counters[0], (unsigned long long)t.coords);
    if (t.evals) atomicAdd(&a.counters[1], (unsigned long long)t.evals);
    if (t.steps) atomicAdd(&a.counters[2], (unsigned long long)t.steps);
    if (t.caps) atomicAdd(&a.counters[3], (unsigned long long)t.caps);
}

// Drops the L2 lines of a finished tile (r rows of `len` floats, row stride
// lcap) without writing them back: the tile is dead once its unit is done.
// Whole 128-byte lines only; the partial lines at row ends are left alone.
__device__ __forceinline__ void discard_tile(float *tile, int r, int len, int lcap, int tid, int nthreads) {
    const int per_row = (len * 4) / 128;  // full lines from the row start (rows are 128-byte aligned)
    if (per_row == 0 || (lcap * 4) % 128 != 0) return;
    const int total = r * per_row;
    for (int i = tid; i < total; i += nthreads) {
        const int k = i / per_row, l = i - k * per_row;
        const char *addr = reinterpret_cast<const char *>(tile + (int64_t)k * lcap) + 128 * l;
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(addr) : "memory");
    }
}

// Eq. 1's data term of one nonzero at its final model value (FP32 term).
__device__ __forceinline__ float kl_term(float v, float x, float eps_div) {
    return v > 0.f ? v * logf(v / (x + eps_div)) - v : 0.f;
}

__device__ __forceinline__ double warp_sum_d(double t) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    return t;
}

// The projected Newton loop of Algorithm 2 for one coordinate. eval() returns
// (sum_p w_p A_pk, sum_p q_p A_pk^2) over the subproblem; update(d, dc)
// applies x_p += d A_pk (dc: x_k became positive (+1) or zero (-1)). Every
// thread of the group runs it with identical values.
template <class Eval, class Update>
__device__ __forceinline__ float newton_coordinate(const HalfArgs &a, float xk, float sAk, Eval &&eval,
                                                   Update &&update, Tally &t) {
    const float alpha = a.alpha, beta = a.beta;
    const float tol = a.grad_mode == 0 ? a.eps_grad * (sAk + beta) : a.eps_grad;
    const float xfloor = a.grad_mode == 0 ? 0.f : a.eps_grad;
    ++t.coords;
    // one evaluation site: every pass evaluates, tests, and steps
    for (int it = 0;; ++it) {
        const float2 s = eval();
        ++t.evals;
        const float g = -s.x + sAk + alpha * xk + beta;
        const float h = s.y + alpha;
        if (!(g < -tol || (fabsf(g) > tol && xk > xfloor))) break;
        if (it == a.max_inner) {
            ++t.caps;
            break;
        }
        float xn;
        if (h > 0.f) {
            xn = xk - (a.div_mode == 0 ? __fdiv_rn(g, h) : __fdividef(g, h));
            if (xn < 0.f) xn = 0.f;
        } else {
            xn = g > 0.f ? 0.f : xk;
        }
        const float d = xn - xk;
        const float xnew = xk + d;
        const int dc = (xk == 0.f && xnew > 0.f) ? 1 : ((xk > 0.f && xnew == 0.f) ? -1 : 0);
        if (d != 0.f) update(d, dc);
        const float xs = xk;
        xk = xnew;
        ++t.steps;
        const bool brk = a.break_mode == 0 ? (fabsf(d) < a.eps_x * xs) : (d < a.eps_x * xs);
        if (brk) break;
    }
    return xk;
}

// Programmatic dependent launch between the buckets of a half. The buckets
// work on disjoint units and read only what was complete before the first of
// them started, so a bucket lets the next one start at once
// (launch_dependents at entry): the next bucket's blocks take SMs as the
// current one's tail frees them, or SMs its clusters leave idle. Before it
// exits, every block waits for the previous bucket to complete (wait), so
// that the last bucket's completion still implies every earlier one's, and
// whatever follows the half in stream order sees all of its results. Both
// instructions are no-ops in a kernel launched without the attribute.
struct PdlScope {
    __device__ __forceinline__ PdlScope() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
    __device__ __forceinline__ ~PdlScope() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
};

// A bucket of the plan the half did not choose returns at once.
__device__ __forceinline__ bool plan_skip(const HalfArgs &a) { return a.plan_sel && *a.plan_sel != a.plan_id; }
// A unit outside the half's shard (when one is set) is left to another rank.
__device__ __forceinline__ bool out_of_range(const HalfArgs &a, int64_t u) {
    return a.u1 > a.u0 && (u < a.u0 || u >= a.u1);
}
// The sweep index of the half (from device memory in a captured step).
__device__ __forceinline__ int64_t sweep_of(const HalfArgs &a) { return a.sweep_dev ? *a.sweep_dev : a.sweep; }

}  // namespace dev
}  // namespace nmfkl
