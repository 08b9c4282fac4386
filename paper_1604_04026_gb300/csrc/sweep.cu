// Sweep kernels: one half of Algorithm 1, i.e. Algorithm 2 on every unit
// (column of F, or row of W) of a length bucket.
//
// Mapping (one subproblem = one "group": a warp, or a whole CTA):
//   1. stage: for each nonzero p of the unit, read the fixed factor's row
//      A_p = At[idx_p, 0:r] (one coalesced 4r-byte row), compute
//      x_p = [Ax]_p = sum_k A_pk x_k (Algorithm 2, first step), and write the
//      row transposed into the group's tile T[k][p] in global scratch, so
//      that every later access to column k of A is one coalesced sweep.
//   2. each thread keeps, for the nonzeros it owns (p = t + NT*s), x_p, v_p,
//      w_p = v_p / (x_p + eps) and q_p = w_p / (x_p + eps) in registers.
//      Then the Eq. Partial sums are sum_p w_p A_pk and sum_p q_p A_pk^2, and
//      a Newton step dx updates x_p += dx A_pk and refreshes w_p, q_p.
//   3. coordinates are visited in the Philox order ids (Algorithm 1) with the
//      projected Newton loop of Algorithm 2; column k of T is prefetched one
//      coordinate ahead into registers.
// Reductions are warp xor-butterflies (every lane ends with the same bits),
// plus for CTA groups one shared-memory exchange per evaluation.
#include "common.cuh"
#include "device_util.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

namespace nmfkl {

namespace {

using namespace dev;

// Per-group shared memory: perm (256 B) | x_init, x_out (ldr floats each) |
// staging rows (8 x odd_stride(r) floats per warp) | CTA partials.
__host__ __device__ inline size_t stage_offset(int ldr) { return align16(256 + 2 * (size_t)ldr * 4); }
__host__ __device__ inline size_t group_smem_bytes(int r, int ldr, int warps, bool cta) {
    size_t b = stage_offset(ldr) + (size_t)warps * 8 * odd_stride(r) * 4;
    if (cta) b += 2 * (size_t)warps * sizeof(float2);
    return align16(b);
}

// Shared memory of a ring group (warp, CTA, or CTA of a cluster):
//   perm (256 B) | x_init, x_out (ldr floats each) | Philox words, xpos flags |
//   ring of D tile columns (per thread: K floats per slot) | CTA partials
struct RingLayout {
    size_t aux_off, xpos_off, ring_off, red_off, bytes;
};
__host__ __device__ inline RingLayout ring_layout(int r, int ldr, int nt, int k, int d, bool cta) {
    RingLayout g{};
    size_t off = align16(256 + 2 * (size_t)ldr * 4);
    g.aux_off = off;
    off = align16(off + 8 * (size_t)(r > 1 ? r - 1 : 1));
    g.xpos_off = off;
    off = align16(off + 4 * (size_t)ldr);
    g.ring_off = off;
    off = align16(off + (size_t)d * nt * k * 4);
    g.red_off = off;
    if (cta) off = align16(off + 2 * ((size_t)nt / 32) * sizeof(float4));
    g.bytes = off;
    return g;
}

// x_p and the number of coordinates with A_pk > 0 and x_k > 0 (the positive
// terms of x_p) for one staged nonzero.
struct Staged {
    float x;
    int terms;
};

// Stages nonzero p (one per lane; `valid` false for lanes past the unit's
// end): streams the lane's A row (ldr floats, 16 bytes at a time),
// accumulates x_p = sum_k A_pk x_k and the number of positive terms
// (xpos[k] = 1 where x_k > 0), and writes the row into the tile transposed:
// for each k the warp's 32 lanes store 32 consecutive entries of row k.
__device__ __forceinline__ Staged stage_lane(const HalfArgs &a, float *tile, const float *x_init, const int *xpos,
                                             int p, bool valid, int idx) {
    const int r = a.r, nf4 = a.ldr >> 2;
    const int64_t lcap = a.lcap;
    const float4 *row = reinterpret_cast<const float4 *>(a.At + (int64_t)idx * a.ldr);
    const float4 *x4 = reinterpret_cast<const float4 *>(x_init);
    const int4 *p4 = reinterpret_cast<const int4 *>(xpos);
    float *tcol = tile + p;
    float acc = 0.f;
    int cnt = 0;
    // The row is read kStageBatch 16-byte pieces at a time, all issued before
    // the first is used, so that several gathers are in flight per lane. (8 at
    // a time measured slower: 108.8 vs 103.8 ms per step; the wider batch
    // costs registers the coordinate loop needs, and spills at K = 16.)
    constexpr int kStageBatch = 4;
    for (int f0 = 0; f0 < nf4; f0 += kStageBatch) {
        float4 buf[kStageBatch];
#pragma unroll
        for (int b = 0; b < kStageBatch; ++b)
            buf[b] = (valid && f0 + b < nf4) ? __ldg(row + f0 + b) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int b = 0; b < kStageBatch; ++b) {
            const int f = f0 + b;
            if (f < nf4) {
                const float4 av = buf[b];
                const float4 xv = x4[f];
                const int4 pv = p4[f];
                acc = fmaf(av.x, xv.x, acc);
                acc = fmaf(av.y, xv.y, acc);
                acc = fmaf(av.z, xv.z, acc);
                acc = fmaf(av.w, xv.w, acc);
                cnt += (av.x > 0.f ? pv.x : 0) + (av.y > 0.f ? pv.y : 0) + (av.z > 0.f ? pv.z : 0) +
                       (av.w > 0.f ? pv.w : 0);
                if (valid) {
                    const int k = 4 * f;
                    float *dst = tcol + (int64_t)k * lcap;
                    dst[0] = av.x;
                    if (k + 1 < r) dst[lcap] = av.y;
                    if (k + 2 < r) dst[2 * lcap] = av.z;
                    if (k + 3 < r) dst[3 * lcap] = av.w;
                }
            }
        }
    }
    return Staged{acc, cnt};
}

// Column of entry s of thread t in a tile row and in a ring slot of the dense
// kernels. With K = 4 or 8 the layout is piece-major: entries 4q..4q+3 of a
// thread are four adjacent columns, and the pieces of consecutive threads are
// adjacent (column 4 NT q + 4 t + s % 4), so that a thread moves a piece in
// one 16-byte access and a warp's pieces form one contiguous 512-byte run.
// A unit's last piece, when partial, is written whole, zeros standing for
// the entries without a nonzero, so its tile spans up to 4 NT - 1 columns
// more than its L nonzeros (more L2 footprint; writing that piece in the
// nonzeros' own order instead measured slower). Otherwise (and for K = 16,
// whose four-row staging would not fit the register budget) entry s of
// thread t is column NT s + t, its nonzero's position.
template <int K>
constexpr bool kPieceLayout = K % 4 == 0 && K <= 8;
template <int NT, int K>
__host__ __device__ constexpr int tile_col(int t, int s) {
    return kPieceLayout<K> ? 4 * NT * (s >> 2) + 4 * t + (s & 3) : NT * s + t;
}

// Stages the four nonzeros of one piece (entries 4q..4q+3 of a piece-major
// tile; bit j of `valid` set where entry 4q + j has a nonzero, idx[j] its row
// of A): the four A rows are streamed together, kRowBatch 16-byte pieces of
// each in flight; x_p and the positive-term count of each entry are formed by
// the same operations, in the same order, as in stage_lane; the piece of tile
// row k is written as one float4 at tcol + k * lcap (zeros for entries
// without a nonzero).
template <int kRowBatch>
__device__ __forceinline__ void stage_piece(const HalfArgs &a, float *tcol, const float *x_init, const int *xpos,
                                            const int (&idx)[4], unsigned valid, Staged (&out)[4]) {
    const int r = a.r, nf4 = a.ldr >> 2;
    const int64_t lcap = a.lcap;
    const float4 *row[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) row[j] = reinterpret_cast<const float4 *>(a.At + (int64_t)idx[j] * a.ldr);
    const float4 *x4 = reinterpret_cast<const float4 *>(x_init);
    const int4 *p4 = reinterpret_cast<const int4 *>(xpos);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int cnt[4] = {0, 0, 0, 0};
    for (int f0 = 0; f0 < nf4; f0 += kRowBatch) {
        float4 buf[kRowBatch][4];
#pragma unroll
        for (int b = 0; b < kRowBatch; ++b)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                buf[b][j] = (((valid >> j) & 1u) && f0 + b < nf4) ? __ldg(row[j] + f0 + b)
                                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int b = 0; b < kRowBatch; ++b) {
            const int f = f0 + b;
            if (f < nf4) {
                const float4 xv = x4[f];
                const int4 pv = p4[f];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 av = buf[b][j];
                    acc[j] = fmaf(av.x, xv.x, acc[j]);
                    acc[j] = fmaf(av.y, xv.y, acc[j]);
                    acc[j] = fmaf(av.z, xv.z, acc[j]);
                    acc[j] = fmaf(av.w, xv.w, acc[j]);
                    cnt[j] += (av.x > 0.f ? pv.x : 0) + (av.y > 0.f ? pv.y : 0) + (av.z > 0.f ? pv.z : 0) +
                              (av.w > 0.f ? pv.w : 0);
                }
                if (valid) {
                    const int k = 4 * f;
                    float4 *dst = reinterpret_cast<float4 *>(tcol + (int64_t)k * lcap);
                    dst[0] = make_float4(buf[b][0].x, buf[b][1].x, buf[b][2].x, buf[b][3].x);
                    if (k + 1 < r)
                        *reinterpret_cast<float4 *>(tcol + (int64_t)(k + 1) * lcap) =
                            make_float4(buf[b][0].y, buf[b][1].y, buf[b][2].y, buf[b][3].y);
                    if (k + 2 < r)
                        *reinterpret_cast<float4 *>(tcol + (int64_t)(k + 2) * lcap) =
                            make_float4(buf[b][0].z, buf[b][1].z, buf[b][2].z, buf[b][3].z);
                    if (k + 3 < r)
                        *reinterpret_cast<float4 *>(tcol + (int64_t)(k + 3) * lcap) =
                            make_float4(buf[b][0].w, buf[b][1].w, buf[b][2].w, buf[b][3].w);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j] = Staged{acc[j], cnt[j]};
}

// ---------------------------------------------------------------------------
// Register-resident groups: NT threads (32 = one warp per subproblem, several
// per block; otherwise one CTA), K nonzeros per thread, so L <= NT*K.
// ---------------------------------------------------------------------------
// Kernel modes: one half sweep, the allocation-free F half (units are the
// column indices themselves), and fold-in (each column runs its own sweeps of
// Algorithm 2 until its objective settles, with the tile staged once).
constexpr int kModeHalf = 0, kModeFree = 1, kModeFold = 2;

// Block shape of the one-warp-per-unit kernels: threads per block and the
// minimum resident blocks per SM, which sets the register budget. In a half,
// K = 4 runs 7-warp blocks four to an SM (28 warps, 72 registers) and K = 8
// 5-warp blocks four to an SM (20 warps, 96 registers): 81.1 -> 80.8 and
// -> 80.3 ms per step against 8-warp blocks (24 and 16 warps; 6-warp blocks
// three to an SM for K = 8: 80.6, 7-warp blocks three to an SM: spills). Otherwise 8
// warps per block, 64 registers for K <= 2 (32 warps per SM), 80 for K = 4,
// 128 for the rest. (K = 4 at 64 and K = 8 at 80 registers with 8-warp blocks
// spill and were measured slower; so was a deeper tile ring: the warp kernels
// run a 4-deep ring.) Fold-in and the allocation-free path keep 8-warp blocks.
__host__ __device__ constexpr int warp_block_threads(int K, int mode) {
    return mode != kModeHalf ? 256 : (K == 8 ? 160 : (K == 4 ? 224 : 256));
}
template <int NT, int K, int kMode = kModeHalf>
__host__ __device__ constexpr int min_blocks() {
    return NT == 32 ? (kMode == kModeHalf && K == 8 ? 4 : (K <= 2 || (kMode == kModeHalf && K == 4) ? 4 : (K == 4 ? 3 : 2)))
                    : (512 / NT > 1 ? 512 / NT : 1);
}

template <int NT, int K, int D, int kMode = kModeHalf>
__global__ void __launch_bounds__(NT == 32 ? warp_block_threads(K, kMode) : NT, min_blocks<NT, K, kMode>())
    sweep_kernel(HalfArgs a) {
    PdlScope pdl;
    if (plan_skip(a)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kCta = NT > 32;
    constexpr int kNW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int warp_in_block = threadIdx.x >> 5;
    const int group_in_block = kCta ? 0 : warp_in_block;
    const int groups_per_block = kCta ? 1 : (int)(blockDim.x >> 5);
    const int warp_in_group = kCta ? warp_in_block : 0;
    const int tid_g = kCta ? (int)threadIdx.x : lane;
    const int group_global = blockIdx.x * groups_per_block + group_in_block;

    const int r = a.r, ldr = a.ldr;
    const RingLayout lay = ring_layout(r, ldr, NT, K, D, kCta);
    unsigned char *gs = smem_raw + (size_t)group_in_block * lay.bytes;
    uint8_t *perm = gs;
    float *x_init = reinterpret_cast<float *>(gs + 256);
    float *x_out = x_init + ldr;
    uint64_t *words = reinterpret_cast<uint64_t *>(gs + lay.aux_off);
    int *xpos = reinterpret_cast<int *>(gs + lay.xpos_off);
    // ring slot d holds entry s of this thread at [d*K*NT + tile_col(tid_g, s)]
    constexpr bool kPiece = kPieceLayout<K>;
    constexpr int kRingStride = kPiece ? 4 * NT : NT;  // between pieces (kPiece) or entries
    float *myring = reinterpret_cast<float *>(gs + lay.ring_off) + tile_col<NT, K>(tid_g, 0);
    float2 *red = reinterpret_cast<float2 *>(gs + lay.red_off);
    __shared__ int s_q;

    float *tile = a.scratch + (int64_t)group_global * a.slot_floats;
    const int lcap = a.lcap;
    const float eps_div = a.eps_div;
    const int count = a.count_dev ? *a.count_dev : a.count;
    Tally tally;
    int parity = 0;

    auto group_sync = [&]() {
        if constexpr (kCta) __syncthreads(); else __syncwarp();
    };
    // Every CTA reduction (reduce, group_sum_d) uses 16-byte slots,
    // one per warp, in two halves used alternately (parity), so that a warp
    // that runs ahead never overwrites partials another warp still reads.
    float4 *red4 = reinterpret_cast<float4 *>(red);
    // Sum of one double per thread over the group, identical in every thread.
    auto group_sum_d = [&](double t) -> double {
        t = warp_sum_d(t);
        if constexpr (kCta) {
            float4 *rb = red4 + parity * kNW;
            if (lane == 0) *reinterpret_cast<double *>(&rb[warp_in_block]) = t;
            __syncthreads();
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < kNW; ++w) tot += *reinterpret_cast<const double *>(&rb[w]);
            parity ^= 1;
            return tot;
        } else {
            return t;
        }
    };

    for (;;) {
        int qi;
        if constexpr (kCta) {
            __syncthreads();
            if (threadIdx.x == 0) s_q = atomicAdd(a.queue, 1);
            __syncthreads();
            qi = s_q;
        } else {
            __syncwarp();
            int q = 0;
            if (lane == 0) q = atomicAdd(a.queue, 1);
            qi = __shfl_sync(kFull, q, 0);
        }
        if (qi >= count) break;
        const int64_t u = kMode == kModeFree ? (int64_t)qi : (int64_t)a.units[qi];
        if (out_of_range(a, u)) continue;
        const int64_t base = a.ptr[u];
        const int L = (int)(a.ptr[u + 1] - base);
        const int64_t perm_unit = a.unit_ids ? a.unit_ids[u] : u;
        if constexpr (kMode != kModeHalf) {
            // no host-side length buckets on these paths: a unit beyond NT*K nonzeros is refused
            if (L > NT * K || L < 0) {
                if (tid_g == 0) atomicOr(a.err, kErrLength);
                continue;
            }
        }
        const int ks = (L + NT - 1) / NT;
        // ring entries filled per coordinate: for even K a whole number of
        // pairs (the extra entry is zero-filled: its nonzeros lie past L)
        const int ks2 = K % 2 == 0 ? ks + (ks & 1) : ks;
        // entries of this thread with a nonzero: s < nvalid (nonzero NT s + tid_g < L)
        const int nvalid = tid_g < L ? (L - tid_g + NT - 1) / NT : 0;

        for (int k = tid_g; k < ldr; k += NT) {
            const float xv = a.X[u * ldr + k];
            x_init[k] = xv;
            xpos[k] = xv > 0.f ? 1 : 0;
        }
        group_sync();

        // ---- stage A rows, x_p, and the per-nonzero state
        float xr[K], vr[K], wr[K], qr[K];
        int cr[K];
        if constexpr (kPiece) {
#pragma unroll
            for (int s = 0; s < K; ++s) {
                xr[s] = 0.f; vr[s] = 0.f; wr[s] = 0.f; qr[s] = 0.f; cr[s] = 0;
            }
            // the four indices and values of a piece are loaded one piece
            // ahead, before the rows of the current piece are streamed
            int id4[4];
            float v4[4];
            auto load_piece = [&](int q, int (&ids)[4], float (&vs)[4]) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int pl = 32 * warp_in_group + NT * (4 * q + j) + lane;
                    ids[j] = 0;
                    vs[j] = 0.f;
                    if (pl < L) {
                        ids[j] = a.idx[base + pl];
                        vs[j] = a.val[base + pl];
                    }
                }
            };
            load_piece(0, id4, v4);
#pragma unroll
            for (int q = 0; q < K / 4; ++q) {
                const int p0 = 32 * warp_in_group + NT * 4 * q;
                if (p0 < L) {
                    int idn[4];
                    float vn[4];
                    if (q + 1 < K / 4) load_piece(q + 1, idn, vn);
                    unsigned valid = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (p0 + NT * j + lane < L) valid |= 1u << j;
                    Staged st[4];
                    stage_piece<1>(a, tile + tile_col<NT, K>(tid_g, 4 * q), x_init, xpos, id4, valid,
                                                   st);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if ((valid >> j) & 1u) {
                            const int s = 4 * q + j;
                            const float x_l = st[j].terms == 0 ? 0.f : st[j].x;
                            xr[s] = x_l;
                            cr[s] = st[j].terms;
                            vr[s] = v4[j];
                            const float ri = recip(x_l + eps_div);
                            wr[s] = v4[j] * ri;
                            qr[s] = wr[s] * ri;
                        }
                    }
                    if (q + 1 < K / 4) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            id4[j] = idn[j];
                            v4[j] = vn[j];
                        }
                    }
                }
            }
        } else {
            // the K indices and values are loaded first, so that the row gathers
            // of later rounds do not wait on them
            int ir[K];
#pragma unroll
            for (int s = 0; s < K; ++s) {
                ir[s] = 0;
                vr[s] = 0.f;
                const int pl = 32 * warp_in_group + NT * s + lane;
                if (s < ks && pl < L) {
                    ir[s] = a.idx[base + pl];
                    vr[s] = a.val[base + pl];
                }
            }
#pragma unroll
            for (int s = 0; s < K; ++s) {
                const float v_l = vr[s];
                xr[s] = 0.f; vr[s] = 0.f; wr[s] = 0.f; qr[s] = 0.f; cr[s] = 0;
                if (s < ks) {
                    const int p0 = 32 * warp_in_group + NT * s;
                    if (p0 < L) {
                        const int pl = p0 + lane;
                        const int idx_l = ir[s];
                        const Staged st = stage_lane(a, tile, x_init, xpos, pl, pl < L, idx_l);
                        if (pl < L) {
                            const float x_l = st.terms == 0 ? 0.f : st.x;
                            xr[s] = x_l;
                            cr[s] = st.terms;
                            vr[s] = v_l;
                            const float ri = recip(x_l + eps_div);
                            wr[s] = v_l * ri;
                            qr[s] = wr[s] * ri;
                        }
                    }
                }
            }
        }

        // ---- one pass of Algorithm 2 over the unit's coordinates (order of `sweep`)
        auto run_coordinates = [&](int64_t sweep) {
            if (warp_in_group == 0) {
                ids_swaps_warp(reinterpret_cast<uint8_t *>(words), r, perm_unit, sweep, a.side, a.perm_mode, a.seed, lane);
                __syncwarp();
                if (lane == 0) fisher_yates(perm, reinterpret_cast<const uint8_t *>(words), r);
                __syncwarp();
            }
            group_sync();
            // Each thread copies the tile entries it owns for the coordinate D-1
            // positions ahead into its ring slots (cp.async; no other thread
            // reads them), so the column is in shared memory when its turn comes.
            auto issue = [&](int pos) {
                if (pos < r) {
                    const float *col = tile + (int64_t)perm[pos] * lcap + tile_col<NT, K>(tid_g, 0);
                    float *dst = myring + (pos % D) * K * NT;
                    if constexpr (kPiece) {
                        // whole pieces, the entries without a nonzero zero-filled
#pragma unroll
                        for (int q = 0; q < K / 4; ++q)
                            if (4 * q < ks2)
                                cp_async16z(dst + q * kRingStride, col + q * kRingStride,
                                            4 * min(max(nvalid - 4 * q, 0), 4));
                    } else {
#pragma unroll
                        for (int s = 0; s < K; ++s)
                            if (s < ks2) cp_async4(dst + s * NT, col + NT * s, s < nvalid ? 4 : 0);
                    }
                }
                cp_async_commit();
            };
            auto reduce = [&](float sg, float sh) -> float2 {
                // butterfly over the warp, both sums added by one packed instruction
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ga = __shfl_xor_sync(kFull, sg, o), ha = __shfl_xor_sync(kFull, sh, o);
                    const float2 t = unpack2(fadd2(pack2(sg, sh), pack2(ga, ha)));
                    sg = t.x;
                    sh = t.y;
                }
                if constexpr (kCta) {
                    float4 *rb = red4 + parity * kNW;
                    if (lane == 0) rb[warp_in_block] = make_float4(sg, sh, 0.f, 0.f);
                    __syncthreads();
                    float2 t = make_float2(0.f, 0.f);
#pragma unroll
                    for (int w = 0; w < kNW; ++w) {
                        const float4 v = rb[w];
                        t = add_pair(t, make_float2(v.x, v.y));
                    }
                    parity ^= 1;
                    return t;
                } else {
                    return make_float2(sg, sh);
                }
            };
#pragma unroll
            for (int i = 0; i < D - 1; ++i) issue(i);
            for (int kk = 0; kk < r; ++kk) {
                issue(kk + D - 1);
                cp_async_wait<D - 1>();
                const float *ac = myring + (kk % D) * K * NT;
                const int k = perm[kk];
                auto eval = [&]() -> float2 {
                    const float2 t = lane_sums<K, kRingStride, kPiece>(ac, wr, qr, ks);
                    return reduce(t.x, t.y);
                };
                auto update = [&](float d, int dc) {
                    lane_update<K, kRingStride, kPiece>(ac, xr, vr, wr, qr, cr, ks, d, dc, eps_div);
                };
                const float xk = newton_coordinate(a, x_init[k], a.sumA[k], eval, update, tally);
                if (tid_g == 0) x_out[k] = xk;
            }
            cp_async_wait<0>();
        };

        if constexpr (kMode == kModeFold) {
            // The column objective: Eq. 1's data term over the column's nonzeros
            // (FP32 terms at the current x_p, FP64 sum) plus the linear and
            // regularization terms of its r coordinates (FP64).
            auto column_objective = [&]() -> double {
                float t = 0.f;
#pragma unroll
                for (int s = 0; s < K; ++s)
                    if (s < ks) t += kl_term(vr[s], xr[s], eps_div);
                double d = (double)t;
                for (int k = tid_g; k < r; k += NT) {
                    const double f = (double)x_init[k];
                    d += a.sumA64[k] * f + 0.5 * (double)a.alpha * f * f + (double)a.beta * fabs(f);
                }
                return group_sum_d(d);
            };
            // Algorithm 2's first step at the start of a later pass: x_p from the
            // tile and the current coordinates, in the staging order.
            auto recompute = [&]() {
#pragma unroll
                for (int s = 0; s < K; ++s) {
                    if (s < ks) {
                        const int p = tid_g + NT * s;
                        if (p < L) {
                            const float *col = tile + tile_col<NT, K>(tid_g, s);
                            float acc = 0.f;
                            int cnt = 0;
#pragma unroll 4
                            for (int k = 0; k < r; ++k) {
                                const float av = col[(int64_t)k * lcap];
                                const float xv = x_init[k];
                                acc = fmaf(av, xv, acc);
                                cnt += (av > 0.f && xv > 0.f) ? 1 : 0;
                            }
                            const float x_l = cnt == 0 ? 0.f : acc;
                            xr[s] = x_l;
                            cr[s] = cnt;
                            const float ri = recip(x_l + eps_div);
                            wr[s] = vr[s] * ri;
                            qr[s] = wr[s] * ri;
                        }
                    }
                }
            };
            group_sync();
            double prev = column_objective();
            int done_sweeps = 0;
            while (done_sweeps < a.max_sweeps) {
                run_coordinates(done_sweeps);
                group_sync();
                for (int k = tid_g; k < r; k += NT) x_init[k] = x_out[k];
                group_sync();
                ++done_sweeps;
                recompute();
                const double cur = column_objective();
                const bool settled = fabs(prev - cur) <= a.rel_tol * fabs(prev);
                prev = cur;
                if (settled) break;
            }
            group_sync();
            for (int k = tid_g; k < r; k += NT) x_out[k] = x_init[k];
            if (tid_g == 0) {
                a.sweeps_done[u] = done_sweeps;
                a.unit_final[u] = prev;
            }
        } else {
            run_coordinates(sweep_of(a));
            if (a.unit_obj) {
                float t = 0.f;
#pragma unroll
                for (int s = 0; s < K; ++s)
                    if (s < ks) t += kl_term(vr[s], xr[s], eps_div);
                const double tot = group_sum_d((double)t);
                if (tid_g == 0) a.unit_obj[u] = tot;
            }
        }
        group_sync();
        // the columns in use: the first L, or the first ceil(ks/4) pieces
        discard_tile(tile, r, kPiece ? min(lcap, (ks + 3) / 4 * 4 * NT) : L, lcap, tid_g, NT);
        for (int k = tid_g; k < r; k += NT) {
            const float xv = x_out[k];
            if (!(xv == xv)) atomicOr(a.err, kErrNaN);
            a.X[u * ldr + k] = xv;
        }
    }
    if (tid_g == 0) flush_tally(a, tally);
}

// ---------------------------------------------------------------------------
// Sub-warp groups on the dense tile: units of at most G*K nonzeros with G
// lanes per unit (G < 32) and 32/G units per warp. The warp takes its units
// together and visits their coordinates in step (each unit in its own order),
// with one warp-wide barrier per coordinate so that every instruction serves
// all of them; the group reductions are log2(G) shuffles. A one-warp group on
// a unit of a few dozen nonzeros spends most of each evaluation on the
// 32-lane reduction and the scalar Newton step, which here are shared by
// 32/G units. Staging and the tile ring are those of sweep_kernel.
// ---------------------------------------------------------------------------
template <int G, int K>
__host__ __device__ constexpr int sub_min_blocks() {
    return K <= 4 ? 3 : 2;
}

template <int G, int K, int D>
__global__ void __launch_bounds__(256, sub_min_blocks<G, K>()) sweep_sub_kernel(HalfArgs a) {
    static_assert(G == 4 || G == 8 || G == 16, "sub-warp groups of 4, 8 or 16 lanes");
    PdlScope pdl;
    if (plan_skip(a)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kPerWarp = 32 / G;
    const int lane = threadIdx.x & 31;
    const int glane = lane & (G - 1);
    const unsigned gmask = ((1u << G) - 1u) << (lane & ~(G - 1));
    const int group_in_block = threadIdx.x / G;
    const int groups_per_block = blockDim.x / G;
    const int group_global = blockIdx.x * groups_per_block + group_in_block;

    const int r = a.r, ldr = a.ldr;
    const RingLayout lay = ring_layout(r, ldr, G, K, D, false);
    unsigned char *gs = smem_raw + (size_t)group_in_block * lay.bytes;
    uint8_t *perm = gs;
    float *x_init = reinterpret_cast<float *>(gs + 256);
    float *x_out = x_init + ldr;
    uint64_t *words = reinterpret_cast<uint64_t *>(gs + lay.aux_off);
    int *xpos = reinterpret_cast<int *>(gs + lay.xpos_off);
    // ring slot d holds entry s of this lane at [d*K*G + tile_col(glane, s)]
    constexpr bool kPiece = kPieceLayout<K>;
    constexpr int kRingStride = kPiece ? 4 * G : G;
    float *myring = reinterpret_cast<float *>(gs + lay.ring_off) + tile_col<G, K>(glane, 0);

    float *tile = a.scratch + (int64_t)group_global * a.slot_floats;
    const int lcap = a.lcap;
    const float eps_div = a.eps_div;
    const int count = a.count_dev ? *a.count_dev : a.count;
    const int64_t sweep = sweep_of(a);
    Tally tally;

    for (;;) {
        __syncwarp();
        int q = 0;
        if (lane == 0) q = atomicAdd(a.queue, kPerWarp);
        q = __shfl_sync(kFull, q, 0);
        if (q >= count) break;
        // a group without a unit (the last batch) still runs the warp-wide
        // coordinate loop, without work
        const int qi = q + lane / G;
        bool work = qi < count;
        int64_t u = 0, base = 0;
        int L = 0;
        if (work) {
            u = a.units[qi];
            if (out_of_range(a, u)) {
                work = false;
            } else {
                base = a.ptr[u];
                L = (int)(a.ptr[u + 1] - base);
                if (L > G * K || L < 0) {  // cannot happen with a consistent plan; refuse rather than overrun
                    if (glane == 0) atomicOr(a.err, kErrLength);
                    work = false;
                    L = 0;
                }
            }
        }
        const int ks = work ? (L + G - 1) / G : 0;
        const int ks2 = K % 2 == 0 ? ks + (ks & 1) : ks;  // whole pairs, the extra entry zero-filled
        const int nvalid = glane < L ? (L - glane + G - 1) / G : 0;  // entries with a nonzero (L is 0 without work)
        if (work) {
            for (int k = glane; k < ldr; k += G) {
                const float xv = a.X[u * ldr + k];
                x_init[k] = xv;
                xpos[k] = xv > 0.f ? 1 : 0;
            }
        }
        __syncwarp();

        // ---- stage A rows, x_p, and the per-nonzero state (nonzero p = G s + glane)
        float xr[K], vr[K], wr[K], qr[K];
        int cr[K];
        if constexpr (kPiece) {
#pragma unroll
            for (int s = 0; s < K; ++s) {
                xr[s] = 0.f; vr[s] = 0.f; wr[s] = 0.f; qr[s] = 0.f; cr[s] = 0;
            }
#pragma unroll
            for (int q = 0; q < K / 4; ++q) {
                if (4 * q < ks) {
                    unsigned valid = 0;
                    int id4[4];
                    float v4[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int pl = G * (4 * q + j) + glane;
                        id4[j] = 0;
                        v4[j] = 0.f;
                        if (pl < L) {
                            id4[j] = a.idx[base + pl];
                            v4[j] = a.val[base + pl];
                            valid |= 1u << j;
                        }
                    }
                    Staged st[4];
                    stage_piece<1>(a, tile + tile_col<G, K>(glane, 4 * q), x_init, xpos, id4, valid, st);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if ((valid >> j) & 1u) {
                            const int s = 4 * q + j;
                            const float x_l = st[j].terms == 0 ? 0.f : st[j].x;
                            xr[s] = x_l;
                            cr[s] = st[j].terms;
                            vr[s] = v4[j];
                            const float ri = recip(x_l + eps_div);
                            wr[s] = v4[j] * ri;
                            qr[s] = wr[s] * ri;
                        }
                    }
                }
            }
        } else {
#pragma unroll
            for (int s = 0; s < K; ++s) {
                xr[s] = 0.f; vr[s] = 0.f; wr[s] = 0.f; qr[s] = 0.f; cr[s] = 0;
                if (s < ks) {
                    const int pl = G * s + glane;
                    int idx_l = 0;
                    float v_l = 0.f;
                    if (pl < L) {
                        idx_l = a.idx[base + pl];
                        v_l = a.val[base + pl];
                    }
                    const Staged st = stage_lane(a, tile, x_init, xpos, pl, pl < L, idx_l);
                    if (pl < L) {
                        const float x_l = st.terms == 0 ? 0.f : st.x;
                        xr[s] = x_l;
                        cr[s] = st.terms;
                        vr[s] = v_l;
                        const float ri = recip(x_l + eps_div);
                        wr[s] = v_l * ri;
                        qr[s] = wr[s] * ri;
                    }
                }
            }
        }
        if (work) {
            const int64_t perm_unit = a.unit_ids ? a.unit_ids[u] : u;
            ids_swaps_warp(reinterpret_cast<uint8_t *>(words), r, perm_unit, sweep, a.side, a.perm_mode, a.seed, glane, G);
            __syncwarp(gmask);
            if (glane == 0) fisher_yates(perm, reinterpret_cast<const uint8_t *>(words), r);
        }
        __syncwarp();

        // ---- Algorithm 2 over the units' coordinates, in step
        auto issue = [&](int pos) {
            if (work && pos < r) {
                const float *col = tile + (int64_t)perm[pos] * lcap + tile_col<G, K>(glane, 0);
                float *dst = myring + (pos % D) * K * G;
                if constexpr (kPiece) {
#pragma unroll
                    for (int q = 0; q < K / 4; ++q)
                        if (4 * q < ks2)
                            cp_async16z(dst + q * kRingStride, col + q * kRingStride,
                                        4 * min(max(nvalid - 4 * q, 0), 4));
                } else {
#pragma unroll
                    for (int s = 0; s < K; ++s)
                        if (s < ks2) cp_async4(dst + s * G, col + G * s, s < nvalid ? 4 : 0);
                }
            }
            cp_async_commit();
        };
#pragma unroll
        for (int i = 0; i < D - 1; ++i) issue(i);
        for (int kk = 0; kk < r; ++kk) {
            issue(kk + D - 1);
            cp_async_wait<D - 1>();
            if (work) {
                const float *ac = myring + (kk % D) * K * G;
                const int k = perm[kk];
                auto eval = [&]() -> float2 {
                    const float2 t = lane_sums<K, kRingStride, kPiece>(ac, wr, qr, ks);
                    float sg = t.x, sh = t.y;
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) {
                        const float ga = __shfl_xor_sync(gmask, sg, o), ha = __shfl_xor_sync(gmask, sh, o);
                        const float2 u = unpack2(fadd2(pack2(sg, sh), pack2(ga, ha)));
                        sg = u.x;
                        sh = u.y;
                    }
                    return make_float2(sg, sh);
                };
                auto update = [&](float d, int dc) {
                    lane_update<K, kRingStride, kPiece>(ac, xr, vr, wr, qr, cr, ks, d, dc, eps_div);
                };
                const float xk = newton_coordinate(a, x_init[k], a.sumA[k], eval, update, tally);
                if (glane == 0) x_out[k] = xk;
            }
            __syncwarp();
        }
        cp_async_wait<0>();
        if (work) {
            if (a.unit_obj) {
                float t = 0.f;
#pragma unroll
                for (int s = 0; s < K; ++s)
                    if (s < ks) t += kl_term(vr[s], xr[s], eps_div);
                double dt = (double)t;
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) dt += __shfl_xor_sync(gmask, dt, o);
                if (glane == 0) a.unit_obj[u] = dt;
            }
            __syncwarp(gmask);
            discard_tile(tile, r, kPiece ? min(lcap, (ks + 3) / 4 * 4 * G) : L, lcap, glane, G);
            for (int k = glane; k < r; k += G) {
                const float xv = x_out[k];
                if (!(xv == xv)) atomicOr(a.err, kErrNaN);
                a.X[u * ldr + k] = xv;
            }
        }
    }
    if (glane == 0) flush_tally(a, tally);
}

// ---------------------------------------------------------------------------
// Giant units (L beyond the register-resident buckets): one CTA per unit,
// per-nonzero state in the group's global scratch slot:
//   [T: r x lcap][x: lcap][v: lcap][w: lcap][q: lcap][terms: lcap]
// ---------------------------------------------------------------------------
constexpr int kGiantNT = 512;

__global__ void __launch_bounds__(kGiantNT) sweep_giant_kernel(HalfArgs a) {
    PdlScope pdl;
    if (plan_skip(a)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kNW = kGiantNT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = a.r, ldr = a.ldr, S = odd_stride(r), lcap = a.lcap;
    uint8_t *perm = smem_raw;
    float *x_init = reinterpret_cast<float *>(smem_raw + 256);
    float *x_out = x_init + ldr;
    float *stg_base = reinterpret_cast<float *>(smem_raw + stage_offset(ldr));
    float *stg = stg_base + warp * 8 * S;
    float2 *red = reinterpret_cast<float2 *>(stg_base + kNW * 8 * S);
    uint64_t *words = reinterpret_cast<uint64_t *>(stg_base);
    int *xpos = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(stg_base) + align16(8 * (size_t)r));
    __shared__ int s_q;

    float *tile = a.scratch + (int64_t)blockIdx.x * a.slot_floats;
    float *gx = tile + (int64_t)r * lcap;
    float *gv = gx + lcap;
    float *gw = gv + lcap;
    float *gq = gw + lcap;
    int *gc = reinterpret_cast<int *>(gq + lcap);
    const float eps_div = a.eps_div;
    Tally tally;
    int parity = 0;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_q = atomicAdd(a.queue, 1);
        __syncthreads();
        const int qi = s_q;
        if (qi >= a.count) break;
        const int64_t u = a.units[qi];
        if (out_of_range(a, u)) continue;
        const int64_t base = a.ptr[u];
        const int L = (int)(a.ptr[u + 1] - base);
        for (int k = threadIdx.x; k < ldr; k += kGiantNT) {
            const float xv = a.X[u * ldr + k];
            x_init[k] = xv;
            xpos[k] = xv > 0.f ? 1 : 0;
        }
        __syncthreads();
        for (int p0 = 32 * warp; p0 < L; p0 += kGiantNT) {
            const int pl = p0 + lane;
            int idx_l = 0;
            float v_l = 0.f;
            if (pl < L) {
                idx_l = a.idx[base + pl];
                v_l = a.val[base + pl];
            }
            const Staged st = stage_lane(a, tile, x_init, xpos, pl, pl < L, idx_l);
            if (pl < L) {
                const float x_l = st.terms == 0 ? 0.f : st.x;
                const float ri = recip(x_l + eps_div);
                gc[pl] = st.terms;
                gx[pl] = x_l;
                gv[pl] = v_l;
                gw[pl] = v_l * ri;
                gq[pl] = v_l * ri * ri;
            }
        }
        if (warp == 0) {
            ids_swaps_warp(reinterpret_cast<uint8_t *>(words), r, u, sweep_of(a), a.side, a.perm_mode, a.seed, lane);
            __syncwarp();
            if (lane == 0) fisher_yates(perm, reinterpret_cast<const uint8_t *>(words), r);
            __syncwarp();
        }
        __syncthreads();
        for (int kk = 0; kk < r; ++kk) {
            const int k = perm[kk];
            const float *col = tile + (int64_t)k * lcap;
            auto eval = [&]() -> float2 {
                float sg = 0.f, sh = 0.f;
                for (int p = threadIdx.x; p < L; p += kGiantNT) {
                    const float av = __ldcg(col + p);
                    sg = fmaf(__ldcg(gw + p), av, sg);
                    sh = fmaf(__ldcg(gq + p) * av, av, sh);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sg += __shfl_xor_sync(kFull, sg, o);
                    sh += __shfl_xor_sync(kFull, sh, o);
                }
                float2 *rb = red + parity * kNW;
                if (lane == 0) rb[warp] = make_float2(sg, sh);
                __syncthreads();
                float tg = 0.f, th = 0.f;
#pragma unroll
                for (int w = 0; w < kNW; ++w) {
                    const float2 v = rb[w];
                    tg += v.x;
                    th += v.y;
                }
                parity ^= 1;
                return make_float2(tg, th);
            };
            auto update = [&](float d, int dc) {
                for (int p = threadIdx.x; p < L; p += kGiantNT) {
                    int terms = __ldcg(gc + p);
                    const float xv = step_x(__ldcg(gx + p), __ldcg(col + p), d, dc, terms);
                    gc[p] = terms;
                    const float ri = recip(xv + eps_div);
                    const float wv = __ldcg(gv + p) * ri;
                    gx[p] = xv;
                    gw[p] = wv;
                    gq[p] = wv * ri;
                }
            };
            const float xk = newton_coordinate(a, x_init[k], a.sumA[k], eval, update, tally);
            if (threadIdx.x == 0) x_out[k] = xk;
        }
        if (a.unit_obj) {
            float t = 0.f;
            for (int p = threadIdx.x; p < L; p += kGiantNT) t += kl_term(__ldcg(gv + p), __ldcg(gx + p), eps_div);
            const double dt = warp_sum_d((double)t);
            double *rd = reinterpret_cast<double *>(red + parity * kNW);
            if (lane == 0) rd[warp] = dt;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < kNW; ++w) tot += rd[w];
                a.unit_obj[u] = tot;
            }
            parity ^= 1;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < r; k += kGiantNT) {
            const float xv = x_out[k];
            if (!(xv == xv)) atomicOr(a.err, kErrNaN);
            a.X[u * ldr + k] = xv;
        }
    }
    if (threadIdx.x == 0) flush_tally(a, tally);
}


// ---------------------------------------------------------------------------
// Cluster groups: a unit too long for one CTA's registers is split across the
// CL CTAs of a thread-block cluster (one CTA per SM). CTA c stages and owns
// the contiguous slice [c*Lc, (c+1)*Lc) of the unit's nonzeros (Lc =
// ceil(L / CL)) with K of them per thread in registers. Every evaluation
// reduces inside the CTA, then exchanges the CTA partials through
// distributed shared memory: each CTA stores its partial into slot[rank] of
// every CTA of the cluster and arrives on that CTA's mbarrier; each CTA
// waits on its own mbarrier (bounded by a clock limit: on timeout it sets
// the error flag and every later exchange is skipped) and sums the slots in
// rank order, so all CTAs hold identical totals and take identical Newton
// decisions. Units are assigned to clusters round-robin, longest first.
// ---------------------------------------------------------------------------
constexpr int kClusterMax = 16;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(rank));
    return out;
}
__device__ __forceinline__ void st_cluster_u64(uint32_t addr, unsigned long long v) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long pack_f2(float x, float y) {
    return (static_cast<unsigned long long>(__float_as_uint(y)) << 32) | __float_as_uint(x);
}
__device__ __forceinline__ float2 unpack_f2(unsigned long long v) {
    return make_float2(__uint_as_float(static_cast<unsigned>(v & 0xffffffffull)),
                       __uint_as_float(static_cast<unsigned>(v >> 32)));
}
__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    return done != 0;
}

template <int NT, int K, int D>
__global__ void __launch_bounds__(NT, 1) sweep_cluster_kernel(HalfArgs a) {
    PdlScope pdl;
    if (plan_skip(a)) return;  // uniform over the cluster: every CTA reads the same selection
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t crank = cluster.block_rank();
    const uint32_t csize = cluster.num_blocks();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kNW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = a.r, ldr = a.ldr, S = odd_stride(r);
    const RingLayout lay = ring_layout(r, ldr, NT, K, D, true);
    uint8_t *perm = smem_raw;
    float *x_init = reinterpret_cast<float *>(smem_raw + 256);
    float *x_out = x_init + ldr;
    uint64_t *words = reinterpret_cast<uint64_t *>(smem_raw + lay.aux_off);
    int *xpos = reinterpret_cast<int *>(smem_raw + lay.xpos_off);
    float *myring = reinterpret_cast<float *>(smem_raw + lay.ring_off) + threadIdx.x;
    float2 *red = reinterpret_cast<float2 *>(smem_raw + lay.red_off);
    unsigned long long *slots = reinterpret_cast<unsigned long long *>(smem_raw + lay.bytes);  // [2][kClusterMax]
    unsigned long long *mbar = slots + 2 * kClusterMax;                                         // [2]
    __shared__ int s_abort;

    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&mbar[0]), csize);
        mbar_init(smem_addr(&mbar[1]), csize);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster.sync();

    float *tile = a.scratch + (int64_t)blockIdx.x * a.slot_floats;
    const int lcap = a.lcap;
    const float eps_div = a.eps_div;
    Tally tally;
    int par = 0;
    uint32_t phase[2] = {0u, 0u};
    const int nclusters = gridDim.x / csize;
    const int cid = blockIdx.x / csize;

    // Sum of one 64-bit contribution per CTA of the cluster (rank order).
    auto exchange = [&](unsigned long long mine, auto &&combine) {
        if (warp == 0) {
            const bool live = !s_abort;
            const uint32_t my_bar = smem_addr(&mbar[par]);
            if (live && lane < (int)csize) {
                // lane c stores this CTA's partial into CTA c, then arrives there
                const uint32_t my_slot = smem_addr(&slots[par * kClusterMax + crank]);
                st_cluster_u64(map_rank(my_slot, lane), mine);
                mbar_arrive_remote(map_rank(my_bar, lane));
            }
            if (live && lane == 0) {
                // the clock is checked before every try, so a limit shorter
                // than one clock read gives up at once
                const long long t0 = clock64();
                for (;;) {
                    if (clock64() - t0 > a.wait_cycles) {
                        s_abort = 1;
                        atomicOr(a.err, kErrTimeout);
                        break;
                    }
                    if (mbar_try_wait(my_bar, phase[par])) break;
                }
            }
            __syncwarp();
        }
        __syncthreads();
        // After a timeout a late peer may still store into the slots while
        // they are read: an aborted CTA combines no slot at all, so every one
        // of its threads gets the same (zero) total and takes the same
        // decisions (s_abort was written before the barrier above).
        combine(slots + par * kClusterMax, s_abort ? 0u : csize);
        phase[par] ^= 1u;
        par ^= 1;
    };

    for (int qi = cid; qi < a.count; qi += nclusters) {
        const int64_t u = a.units[qi];
        if (out_of_range(a, u)) continue;  // uniform over the cluster
        const int64_t ubase = a.ptr[u];
        const int Lall = (int)(a.ptr[u + 1] - ubase);
        const int Lc = (Lall + (int)csize - 1) / (int)csize;
        const int my0 = (int)crank * Lc;
        const int L = max(0, min(Lc, Lall - my0));
        const int64_t base = ubase + my0;
        const int ks = (L + NT - 1) / NT;

        for (int k = threadIdx.x; k < ldr; k += NT) {
            const float xv = a.X[u * ldr + k];
            x_init[k] = xv;
            xpos[k] = xv > 0.f ? 1 : 0;
        }
        __syncthreads();
        float xr[K], vr[K], wr[K], qr[K];
        int cr[K];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            xr[s] = 0.f; vr[s] = 0.f; wr[s] = 0.f; qr[s] = 0.f; cr[s] = 0;
            if (s < ks) {
                const int p0 = 32 * warp + NT * s;
                if (p0 < L) {
                    const int pl = p0 + lane;
                    int idx_l = 0;
                    float v_l = 0.f;
                    if (pl < L) {
                        idx_l = a.idx[base + pl];
                        v_l = a.val[base + pl];
                    }
                    const Staged st = stage_lane(a, tile, x_init, xpos, pl, pl < L, idx_l);
                    if (pl < L) {
                        const float x_l = st.terms == 0 ? 0.f : st.x;
                        xr[s] = x_l;
                        cr[s] = st.terms;
                        vr[s] = v_l;
                        const float ri = recip(x_l + eps_div);
                        wr[s] = v_l * ri;
                        qr[s] = wr[s] * ri;
                    }
                }
            }
        }
        if (warp == 0) {
            ids_swaps_warp(reinterpret_cast<uint8_t *>(words), r, u, sweep_of(a), a.side, a.perm_mode, a.seed, lane);
            __syncwarp();
            if (lane == 0) fisher_yates(perm, reinterpret_cast<const uint8_t *>(words), r);
            __syncwarp();
        }
        __syncthreads();

        auto issue = [&](int pos) {
            if (pos < r) {
                const float *col = tile + (int64_t)perm[pos] * lcap + threadIdx.x;
                float *dst = myring + (pos % D) * K * NT;
#pragma unroll
                for (int s = 0; s < K; ++s)
                    if (s < ks) cp_async4(dst + s * NT, col + NT * s, (int)threadIdx.x + NT * s < L ? 4 : 0);
            }
            cp_async_commit();
        };
        auto reduce = [&](float sg, float sh) -> float2 {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sg += __shfl_xor_sync(kFull, sg, o);
                sh += __shfl_xor_sync(kFull, sh, o);
            }
            float2 *rb = red + par * kNW;
            if (lane == 0) rb[warp] = make_float2(sg, sh);
            __syncthreads();
            float tg = 0.f, th = 0.f;
#pragma unroll
            for (int w = 0; w < kNW; ++w) {
                const float2 v = rb[w];
                tg += v.x;
                th += v.y;
            }
            float2 tot = make_float2(0.f, 0.f);
            const float2 mine = make_float2(tg, th);
            exchange(*reinterpret_cast<const unsigned long long *>(&mine),
                     [&](const unsigned long long *sl, uint32_t n) {
                         for (uint32_t c = 0; c < n; ++c) {
                             const float2 v = *reinterpret_cast<const float2 *>(&sl[c]);
                             tot.x += v.x;
                             tot.y += v.y;
                         }
                     });
            return tot;
        };

#pragma unroll
        for (int i = 0; i < D - 1; ++i) issue(i);
        for (int kk = 0; kk < r; ++kk) {
            issue(kk + D - 1);
            cp_async_wait<D - 1>();
            const float *ac = myring + (kk % D) * K * NT;
            const int k = perm[kk];
            auto eval = [&]() -> float2 {
                float sg = 0.f, sh = 0.f;
#pragma unroll
                for (int s = 0; s < K; ++s) {
                    if (s < ks) {
                        const float av = ac[s * NT];
                        sg = fmaf(wr[s], av, sg);
                        sh = fmaf(qr[s] * av, av, sh);
                    }
                }
                return reduce(sg, sh);
            };
            auto update = [&](float d, int dc) {
#pragma unroll
                for (int s = 0; s < K; ++s) {
                    if (s < ks) {
                        xr[s] = step_x(xr[s], ac[s * NT], d, dc, cr[s]);
                        const float ri = recip(xr[s] + eps_div);
                        wr[s] = vr[s] * ri;
                        qr[s] = wr[s] * ri;
                    }
                }
            };
            const float xk = newton_coordinate(a, x_init[k], a.sumA[k], eval, update, tally);
            if (threadIdx.x == 0) x_out[k] = xk;
        }
        cp_async_wait<0>();
        if (a.unit_obj) {
            float t = 0.f;
#pragma unroll
            for (int s = 0; s < K; ++s)
                if (s < ks) t += kl_term(vr[s], xr[s], eps_div);
            const double dt = warp_sum_d((double)t);
            double *rd = reinterpret_cast<double *>(red + par * kNW);
            if (lane == 0) rd[warp] = dt;
            __syncthreads();
            double cta = 0.0;
            for (int w = 0; w < kNW; ++w) cta += rd[w];
            double tot = 0.0;
            exchange(static_cast<unsigned long long>(__double_as_longlong(cta)),
                     [&](const unsigned long long *sl, uint32_t n) {
                         for (uint32_t c = 0; c < n; ++c) tot += __longlong_as_double(static_cast<long long>(sl[c]));
                     });
            if (crank == 0 && threadIdx.x == 0) a.unit_obj[u] = tot;
        }
        __syncthreads();
        discard_tile(tile, r, L, lcap, threadIdx.x, NT);
        if (crank == 0) {
            for (int k = threadIdx.x; k < r; k += NT) {
                const float xv = x_out[k];
                if (!(xv == xv)) atomicOr(a.err, kErrNaN);
                a.X[u * ldr + k] = xv;
            }
        }
    }
    if (crank == 0 && threadIdx.x == 0) flush_tally(a, tally);
    // no CTA may leave while a peer can still write into its shared memory
    cluster.sync();
}

// ---------------------------------------------------------------------------
// Sparse-list groups. A nonzero p with A_pk = 0 adds nothing to either sum of
// Eq. Partial for coordinate k and its x_p does not move when x_k does, so
// coordinate k only needs the nonzeros with A_pk > 0 (the paper's use of the
// sparsity of W and F, Section 2). Staging writes, per warp of the group and
// per k, the list of (p, A_pk) over that warp's nonzeros with A_pk > 0, in
// increasing p (one ballot per k per 32 nonzeros), into the group's scratch
// slot; the coordinate loop then visits only those entries. The per-nonzero
// state (x_p, v_p), (w_p, q_p) and the positive-term count is addressed by p:
// in shared memory, or for giant units in the scratch slot.
// Warp w of the group owns the chunks of 32 nonzeros c = w, w + NW, ...; its
// lists hold only its own nonzeros, so warps never touch each other's state.
// (In a cluster each CTA does the same on its own slice of the unit.)
// ---------------------------------------------------------------------------
// list entries per lane prefetched into registers: warp groups (8 for the
// 513..1,024-nonzero compact class, whose lists on the W half run past four
// entries per lane: 10.1 -> 9.6 ms per W half on the large corpus at a steady
// state; the 257..512 class measured slower with 8 on the F half), CTA groups
// (12 measured slower than 8)
constexpr int kSparseE = 4, kSparseE1k = 8, kSparseECta = 8;

constexpr int kSparseCapW = 256;  // list entries per warp staged in shared memory per coordinate

struct SparseLayout {
    size_t words_off, cnt_off, red_off, xv_off, wq_off, tm_off, lbuf_off, bytes;
};
// scap: nonzeros whose state is in shared memory (0: state in the slot, and a
// double-buffered shared copy of each warp's list for the current coordinate)
// compact: shared-memory state of (x_p, v_p) and the term count only
__host__ __device__ inline SparseLayout sparse_layout(int r, int ldr, int nt, int scap, bool compact) {
    SparseLayout g{};
    size_t off = align16(256 + 2 * (size_t)ldr * 4);  // perm | x_init | x_out
    g.words_off = off;
    off = align16(off + 8 * (size_t)(r > 1 ? r - 1 : 1));
    g.cnt_off = off;
    off = align16(off + 4 * (size_t)(nt / 32) * ldr);
    g.red_off = off;
    off = align16(off + 2 * (size_t)(nt / 32) * sizeof(float2));
    // state slots: the scap nonzeros and one dummy (index scap)
    const size_t ns = scap > 0 ? (size_t)scap + 1 : 0;
    g.xv_off = off;
    off = align16(off + 8 * ns);
    g.wq_off = off;
    if (!compact) off = align16(off + 8 * ns);
    g.tm_off = off;
    off = align16(off + 2 * ns);
    g.lbuf_off = off;
    if (scap == 0) off = align16(off + 3 * (size_t)(nt / 32) * kSparseCapW * sizeof(int2));
    g.bytes = off;
    return g;
}
// Scratch slot of a sparse group (floats): lists [NW][r][lcap/NW] of int2,
// then, when the state is not in shared memory, xv[lcap+1], wq[lcap+1]
// (float2) and tm[lcap+1] (the last of each is the dummy).
__host__ __device__ inline int64_t sparse_slot_floats(int r, int lcap, bool smem_state) {
    int64_t f = 2 * (int64_t)r * lcap;
    if (!smem_state) f += 4 * ((int64_t)lcap + 1) + (lcap + 2) / 2;
    return (f + 63) / 64 * 64;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Register budgets: two blocks of eight warps (128 registers) for warp
// groups. (85 registers and three blocks for the slot-state warp groups was
// measured slower: 153 vs 133 ms per step.)
template <int NT, bool kSmemState>
__host__ __device__ constexpr int sparse_min_blocks() {
    return NT == 32 ? 2 : (NT == 128 ? 4 : (NT == 256 ? 2 : 1));
}
// kCompact (shared state only): keep (x_p, v_p) and the term count, and form
// w_p, q_p where they are used; this holds 1.8x the nonzeros in the same
// shared memory for one reciprocal more per list entry and evaluation.
// kCluster (CTA groups with shared state): a unit is split over the CTAs of a
// thread-block cluster. CTA c stages and owns the contiguous slice [c*Lc,
// (c+1)*Lc) of the unit's nonzeros (Lc = ceil(L / cluster size)), with its
// own lists and state. Every evaluation reduces inside the CTA, then warp 0
// stores the CTA partial into slot [rank] of every CTA of the cluster through
// distributed shared memory and arrives on that CTA's mbarrier; each thread
// waits on its own CTA's mbarrier (bounded by a clock limit: on timeout the
// error flag is set and later exchanges are skipped) and sums the slots in
// rank order, so that all threads of all CTAs hold identical totals and take
// identical Newton decisions. (One store and arrival per warp instead, with
// no CTA barrier, was slower: 128 arrivals per mbarrier and evaluation at 8
// CTAs.) Clusters take units from the bucket's queue, longest first.
template <int NT, bool kSmemState, bool kCompact = false, bool kCluster = false>
__global__ void __launch_bounds__(NT == 32 ? 256 : NT, (sparse_min_blocks<NT, kSmemState>())) sparse_kernel(HalfArgs a) {
    PdlScope pdl;
    if (plan_skip(a)) return;  // uniform over a cluster: every CTA reads the same selection
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kCta = NT > 32;
    // lanes per warp-level group: the whole warp (groups of 8 or 16 lanes,
    // several units per warp, lost to the dense tile for units that short)
    constexpr int G = 32;
    static_assert(!kCluster || (kCta && kSmemState), "clusters split CTA groups with shared state");
    constexpr int kNW = NT / 32;
    constexpr int E = kCta ? kSparseECta : (kCompact ? kSparseE1k : kSparseE);
    constexpr int CH = kCta ? 32 : G;   // lanes per chunk of nonzeros (a warp, or the group)
    constexpr int GS = kCta ? NT : G;   // threads per group
    const int lane = threadIdx.x & 31;
    const int glane = lane & (CH - 1);
    const int gbase = lane & ~(CH - 1);
    const unsigned gmask = CH == 32 ? kFull : (((1u << CH) - 1u) << gbase);
    const int warp_in_block = threadIdx.x >> 5;
    const int group_in_block = kCta ? 0 : (int)(threadIdx.x / G);
    const int groups_per_block = kCta ? 1 : (int)(blockDim.x / G);
    const int w = kCta ? warp_in_block : 0;
    const int tid_g = kCta ? (int)threadIdx.x : glane;
    const int group_global = blockIdx.x * groups_per_block + group_in_block;

    const int r = a.r, ldr = a.ldr, lcap = a.lcap, nf4 = ldr >> 2;
    const int LW = lcap / kNW;
    const SparseLayout lay = sparse_layout(r, ldr, NT, kSmemState ? lcap : 0, kCompact);
    constexpr bool kWQ = !(kSmemState && kCompact);  // w_p, q_p stored
    unsigned char *gs = smem_raw + (size_t)group_in_block * lay.bytes;
    uint8_t *perm = gs;
    float *x_init = reinterpret_cast<float *>(gs + 256);
    float *x_out = x_init + ldr;
    uint64_t *words = reinterpret_cast<uint64_t *>(gs + lay.words_off);
    int *mycnt = reinterpret_cast<int *>(gs + lay.cnt_off) + w * ldr;
    float2 *red = reinterpret_cast<float2 *>(gs + lay.red_off);
    float *slot = a.scratch + (int64_t)group_global * a.slot_floats;
    int2 *mylists = reinterpret_cast<int2 *>(slot) + (int64_t)w * r * LW;
    float2 *xv, *wq = nullptr;
    uint16_t *tm;
    if constexpr (kSmemState) {
        // compact: w_p = v_p/(x_p+eps) and q_p = w_p/(x_p+eps) are formed
        // where they are used, with the same operations as where they are stored
        xv = reinterpret_cast<float2 *>(gs + lay.xv_off);
        if constexpr (!kCompact) wq = reinterpret_cast<float2 *>(gs + lay.wq_off);
        tm = reinterpret_cast<uint16_t *>(gs + lay.tm_off);
    } else {
        // interleaved (x_p, v_p, w_p, q_p) per nonzero: one 16-byte piece, so a
        // prefetch of the piece brings everything a later access to p needs
        xv = reinterpret_cast<float2 *>(slot + 2 * (int64_t)r * lcap);
        wq = xv + 1;
        tm = reinterpret_cast<uint16_t *>(xv + 2 * ((int64_t)lcap + 1));
    }
    constexpr int XS = kSmemState ? 1 : 2;  // float2 stride of xv and wq
    __shared__ int s_q;
    const float eps_div = a.eps_div;
    const int count = a.count_dev ? *a.count_dev : a.count;
    Tally tally;
    int parity = 0;
    if (tid_g == 0) {  // the dummy entry's state: zero, and it stays zero
        xv[XS * (lcap)] = make_float2(0.f, 0.f);
        if constexpr (kWQ) wq[XS * (lcap)] = make_float2(0.f, 0.f);
        tm[lcap] = 0;
    }

    // cluster exchange: slots [2][kClusterMax] and two mbarriers after the layout
    uint32_t crank = 0, csize = 1;
    unsigned long long *xslots = reinterpret_cast<unsigned long long *>(smem_raw + lay.bytes);
    unsigned long long *xbar = xslots + 2 * kClusterMax;
    uint32_t xphase[2] = {0u, 0u};
    int xpar = 0;
    bool aborted = false;  // a wait of this CTA gave up (the same in every thread of the CTA)
    if constexpr (kCluster) {
        cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
        crank = cluster.block_rank();
        csize = cluster.num_blocks();
        if (threadIdx.x == 0) {
            mbar_init(smem_addr(&xbar[0]), csize);
            mbar_init(smem_addr(&xbar[1]), csize);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        cluster.sync();
    }
    // Sum over the cluster of one 64-bit value per CTA (`mine`, meaningful in
    // warp 0); `combine` reads the slots of the first n ranks in rank order.
    // Each thread waits on its CTA's mbarrier with a bounded loop; one
    // CTA-wide vote then decides whether any of them gave up, so all threads
    // take the same path. An aborted CTA stops exchanging and combines no
    // slot (a late peer may still be storing into them): its threads keep
    // identical totals, and its peers give up on their next wait for it.
    auto cluster_sum = [&](unsigned long long mine, auto &&combine) {
        const uint32_t bar = smem_addr(&xbar[xpar]);
        if (!aborted) {
            if (warp_in_block == 0 && lane < (int)csize) {
                const uint32_t slot = smem_addr(&xslots[xpar * kClusterMax + crank]);
                st_cluster_u64(map_rank(slot, lane), mine);
                mbar_arrive_remote(map_rank(bar, lane));
            }
            // the clock is checked before every try, so a limit shorter than
            // one clock read gives up at once
            bool late = false;
            const long long t0 = clock64();
            for (;;) {
                if (clock64() - t0 > a.wait_cycles) {
                    late = true;
                    break;
                }
                if (mbar_try_wait(bar, xphase[xpar])) break;
            }
            if (__syncthreads_or(late)) {
                aborted = true;
                if (threadIdx.x == 0) atomicOr(a.err, kErrTimeout);
            }
        }
        combine(xslots + xpar * kClusterMax, aborted ? 0 : (int)csize);
        xphase[xpar] ^= 1u;
        xpar ^= 1;
    };

    auto group_sync = [&]() {
        if constexpr (kCta) __syncthreads(); else __syncwarp(gmask);
    };
    auto reduce = [&](float sg, float sh) -> float2 {
#pragma unroll
        for (int o = CH / 2; o > 0; o >>= 1) {
            const float ga = __shfl_xor_sync(gmask, sg, o), ha = __shfl_xor_sync(gmask, sh, o);
            const float2 u = unpack2(fadd2(pack2(sg, sh), pack2(ga, ha)));
            sg = u.x;
            sh = u.y;
        }
        if constexpr (kCluster) {
            float2 *rb = red + parity * kNW;
            if (lane == 0) rb[warp_in_block] = make_float2(sg, sh);
            __syncthreads();
            parity ^= 1;
            float2 c = make_float2(0.f, 0.f);
            if (warp_in_block == 0) {
#pragma unroll
                for (int i = 0; i < kNW; ++i) c = add_pair(c, rb[i]);
            }
            float2 tot = make_float2(0.f, 0.f);
            cluster_sum(pack_f2(c.x, c.y), [&](const unsigned long long *sl, int n) {
                for (int i = 0; i < n; ++i) tot = add_pair(tot, unpack_f2(sl[i]));
            });
            return tot;
        } else if constexpr (kCta) {
            float2 *rb = red + parity * kNW;
            if (lane == 0) rb[warp_in_block] = make_float2(sg, sh);
            __syncthreads();
            float2 t = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < kNW; ++i) t = add_pair(t, rb[i]);
            parity ^= 1;
            return t;
        } else {
            return make_float2(sg, sh);
        }
    };

    for (;;) {
        int qi;
        if constexpr (kCluster) {
            // rank 0 takes the next unit and hands it to every CTA of the
            // cluster (the first barrier: every CTA has read the last one)
            cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
            cluster.sync();
            if (crank == 0 && threadIdx.x < csize) {
                int q = 0;
                if (threadIdx.x == 0) q = atomicAdd(a.queue, 1);
                q = __shfl_sync((1u << csize) - 1u, q, 0);
                st_cluster_u32(map_rank(smem_addr(&s_q), threadIdx.x), (uint32_t)q);
            }
            cluster.sync();
            qi = s_q;
        } else if constexpr (kCta) {
            __syncthreads();
            if (threadIdx.x == 0) s_q = atomicAdd(a.queue, 1);
            __syncthreads();
            qi = s_q;
        } else {
            __syncwarp(gmask);
            int q = 0;
            if (glane == 0) q = atomicAdd(a.queue, 1);
            qi = __shfl_sync(gmask, q, gbase);
        }
        if (qi >= count) break;
        const int64_t u = a.units[qi];
        if (out_of_range(a, u)) continue;  // uniform over a cluster
        int64_t base = a.ptr[u];
        int L = (int)(a.ptr[u + 1] - base);
        const int64_t perm_unit = a.unit_ids ? a.unit_ids[u] : u;
        // clusters: this CTA's slice (the same Lc, hence the same test, on every rank)
        const int Lc = (L + (int)csize - 1) / (int)csize;
        if constexpr (kCluster) {
            const int my0 = min(L, (int)crank * Lc);
            base += my0;
            L = min(Lc, L - my0);
        }
        if (Lc > lcap) {  // cannot happen with a consistent plan; refuse rather than overrun
            if (tid_g == 0) atomicOr(a.err, kErrLength);
            continue;
        }
        for (int k = tid_g; k < ldr; k += GS) {
            const float xk = a.X[u * ldr + k];
            x_init[k] = xk;
            x_out[k] = xk;
        }
        for (int k = glane; k < ldr; k += CH) mycnt[k] = 0;
        group_sync();

        // ---- stage: x_p, the state, and this warp's lists
        const int nchunks = (L + CH - 1) / CH;
        const float4 *x4 = reinterpret_cast<const float4 *>(x_init);
        int4 *cnt4 = reinterpret_cast<int4 *>(mycnt);
        const unsigned lt = lanemask_lt() & gmask;
        // the index and value of the lane's nonzero in the warp's next chunk
        // are loaded while the current chunk is staged (its row gather waits
        // on them otherwise: 81.6 -> 81.1 ms per step)
        int idx_n = 0;
        float v_n = 0.f;
        if (CH * w + glane < L) {
            idx_n = a.idx[base + CH * w + glane];
            v_n = a.val[base + CH * w + glane];
        }
        for (int c = w; c < nchunks; c += kNW) {
            const int p = CH * c + glane;
            const bool valid = p < L;
            const int idx = idx_n;
            const float v = v_n;
            {
                const int pn = p + CH * kNW;
                idx_n = 0;
                v_n = 0.f;
                if (pn < L) {
                    idx_n = a.idx[base + pn];
                    v_n = a.val[base + pn];
                }
            }
            const float4 *row = reinterpret_cast<const float4 *>(a.At + (int64_t)idx * ldr);
            float acc = 0.f;
            int terms = 0;
            constexpr int kB = 8;
            for (int f0 = 0; f0 < nf4; f0 += kB) {
                float4 buf[kB];
#pragma unroll
                for (int b = 0; b < kB; ++b)
                    buf[b] = (valid && f0 + b < nf4) ? __ldg(row + f0 + b) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int f = f0 + b;
                    if (f < nf4) {
                        const float4 av = buf[b];
                        const float4 xk = x4[f];
                        const int4 c4 = cnt4[f];
                        acc = fmaf(av.x, xk.x, acc);
                        acc = fmaf(av.y, xk.y, acc);
                        acc = fmaf(av.z, xk.z, acc);
                        acc = fmaf(av.w, xk.w, acc);
                        terms += (av.x > 0.f && xk.x > 0.f) + (av.y > 0.f && xk.y > 0.f) +
                                 (av.z > 0.f && xk.z > 0.f) + (av.w > 0.f && xk.w > 0.f);
                        // padding columns (k >= r) hold 0 and never enter a list
                        const unsigned m0 = __ballot_sync(gmask, av.x > 0.f);
                        const unsigned m1 = __ballot_sync(gmask, av.y > 0.f);
                        const unsigned m2 = __ballot_sync(gmask, av.z > 0.f);
                        const unsigned m3 = __ballot_sync(gmask, av.w > 0.f);
                        int2 *l0 = mylists + (int64_t)(4 * f) * LW;
                        if (av.x > 0.f) l0[c4.x + __popc(m0 & lt)] = make_int2(p, __float_as_int(av.x));
                        if (av.y > 0.f) l0[LW + c4.y + __popc(m1 & lt)] = make_int2(p, __float_as_int(av.y));
                        if (av.z > 0.f) l0[2 * LW + c4.z + __popc(m2 & lt)] = make_int2(p, __float_as_int(av.z));
                        if (av.w > 0.f) l0[3 * LW + c4.w + __popc(m3 & lt)] = make_int2(p, __float_as_int(av.w));
                        if (glane == 0)
                            cnt4[f] = make_int4(c4.x + __popc(m0), c4.y + __popc(m1), c4.z + __popc(m2),
                                                c4.w + __popc(m3));
                    }
                }
            }
            if (valid) {
                const float xl = terms == 0 ? 0.f : acc;
                xv[XS * (p)] = make_float2(xl, v);
                if constexpr (kWQ) {
                    const float ri = recip(xl + eps_div);
                    wq[XS * (p)] = make_float2(v * ri, v * ri * ri);
                }
                tm[p] = (uint16_t)terms;
            }
            __syncwarp(gmask);
        }
        if (w == 0) {
            ids_swaps_warp(reinterpret_cast<uint8_t *>(words), r, perm_unit, sweep_of(a), a.side, a.perm_mode, a.seed, glane, CH);
            __syncwarp(gmask);
            if (glane == 0) fisher_yates(perm, reinterpret_cast<const uint8_t *>(words), r);
            __syncwarp(gmask);
        }
        group_sync();

        // ---- Algorithm 2 over this unit's coordinates, list entries only
        // ---- Algorithm 2 over this unit's coordinates, list entries only
        if constexpr (kSmemState) {
            // The list of the next coordinate is in flight in registers while
            // the current one is processed (two register sets used in turn, so
            // no register is copied while its load may be outstanding).
            int2 qa[E], qb[E];
            int ca = 0, cb = 0;
            // Prefetched slots past the list's end hold the dummy entry (index
            // lcap: state zero, A = 0), so evaluations and updates run over all
            // E slots without a branch (every load issued at once; the dummy
            // adds exact zeros and stays zero: 83.1 -> 81.6 ms per step).
            // The list two coordinates ahead is prefetched into L2: lists are
            // written at staging and have left L2 by the time their coordinate
            // comes, so without it the register prefetch one coordinate ahead
            // (and the tail beyond it) waits on DRAM. (86.5 -> 83.1 ms per step
            // on the large corpus at a steady state; 83.5 at four ahead.)
            auto fetch = [&](int pos, int2 (&dst)[E], int &cn) {
                cn = 0;
                if (pos < r) {
                    const int k = perm[pos];
                    cn = mycnt[k];
                    const int2 *lk = mylists + (int64_t)k * LW;
#pragma unroll
                    for (int t = 0; t < E; ++t) {
                        const int j = glane + CH * t;
                        dst[t] = j < cn ? __ldcg(lk + j) : make_int2(lcap, 0);
                    }
                }
                if (pos + 2 < r) {
                    const int k2 = perm[pos + 2];
                    const int c2 = mycnt[k2];
                    const char *l2 = reinterpret_cast<const char *>(mylists + (int64_t)k2 * LW);
                    for (int b = glane * 128; b < c2 * 8; b += CH * 128)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(l2 + b));
                }
            };
            // entries beyond the prefetched ones, four loads in flight per lane
            auto for_rest = [&](const int2 *lk, int cn, auto &&body) {
                for (int j0 = glane + CH * E; j0 < cn; j0 += 4 * CH) {
                    int2 e[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) e[t] = j0 + CH * t < cn ? __ldcg(lk + j0 + CH * t) : make_int2(0, 0);
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (j0 + CH * t < cn) body(e[t].x, __int_as_float(e[t].y));
                }
            };
            auto coordinate = [&](int kk, int2 (&cur)[E], int cn) {
                const int k = perm[kk];
                const int2 *lk = mylists + (int64_t)k * LW;
                auto eval = [&]() -> float2 {
                    float sg = 0.f, sh = 0.f;
                    auto acc = [&](int p, float av) {
                        if constexpr (kCompact) {
                            const float2 st = xv[p];
                            const float ri = recip(st.x + eps_div);
                            const float wp = st.y * ri, qp = wp * ri;
                            sg = fmaf(wp, av, sg);
                            sh = fmaf(qp * av, av, sh);
                        } else {
                            const float2 st = wq[p];
                            sg = fmaf(st.x, av, sg);
                            sh = fmaf(st.y * av, av, sh);
                        }
                    };
#pragma unroll
                    for (int t = 0; t < E; ++t) acc(cur[t].x, __int_as_float(cur[t].y));
                    for_rest(lk, cn, acc);
                    return reduce(sg, sh);
                };
                auto update = [&](float d, int dc) {
                    auto upd = [&](int p, float av) {
                        if constexpr (kCompact) {
                            const float x0 = xv[p].x;
                            int terms = dc != 0 ? (int)tm[p] : 0;
                            const float xn = step_x(x0, av, d, dc, terms);
                            if (dc != 0) tm[p] = (uint16_t)terms;
                            xv[p].x = xn;
                        } else {
                            const float2 st = xv[p];
                            int terms = dc != 0 ? (int)tm[p] : 0;
                            const float xn = step_x(st.x, av, d, dc, terms);
                            if (dc != 0) tm[p] = (uint16_t)terms;
                            const float ri = recip(xn + eps_div);
                            xv[p].x = xn;
                            wq[p] = make_float2(st.y * ri, st.y * ri * ri);
                        }
                    };
#pragma unroll
                    for (int t = 0; t < E; ++t) upd(cur[t].x, __int_as_float(cur[t].y));
                    for_rest(lk, cn, upd);
                    // the next evaluation may read these entries from other lanes
                    __syncwarp(gmask);
                };
                const float xk = newton_coordinate(a, x_init[k], a.sumA[k], eval, update, tally);
                if (tid_g == 0) x_out[k] = xk;
            };
            fetch(0, qa, ca);
            for (int kk = 0; kk < r; kk += 2) {
                fetch(kk + 1, qb, cb);
                coordinate(kk, qa, ca);
                if (kk + 1 < r) {
                    fetch(kk + 2, qa, ca);
                    coordinate(kk + 1, qb, cb);
                }
            }
        } else {
            // State in the slot: each warp copies the list of the next
            // coordinate into shared memory (cp.async, up to kSparseCapW
            // entries) while it works on the current one, and issues the state
            // loads eight at a time.
            // Lists are staged two coordinates ahead; once the next one has
            // landed, the 16-byte state pieces of its entries are prefetched
            // into L1, so the next evaluation finds them there (stores of the
            // current coordinate to the same pieces reach L1 too).
            int2 *lbuf = reinterpret_cast<int2 *>(gs + lay.lbuf_off) + (size_t)w * 3 * kSparseCapW;
            auto stage_list = [&](int pos) {
                if (pos < r) {
                    const int k = perm[pos];
                    const int cn = min(mycnt[k], kSparseCapW);
                    const int2 *src = mylists + (int64_t)k * LW;
                    int2 *dst = lbuf + (pos % 3) * kSparseCapW;
                    for (int c = glane; 2 * c < cn; c += CH) cp_async16(dst + 2 * c, src + 2 * c);
                }
                cp_async_commit();
            };
            auto prefetch_state = [&](int pos) {
                if (pos < r) {
                    const int cn = min(mycnt[perm[pos]], kSparseCapW);
                    const int2 *lb = lbuf + (pos % 3) * kSparseCapW;
                    for (int j = glane; j < cn; j += CH)
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(xv + XS * lb[j].x));
                }
            };
            constexpr int kU = 8;
            stage_list(0);
            stage_list(1);
            for (int kk = 0; kk < r; ++kk) {
                stage_list(kk + 2);
                cp_async_wait<1>();
                __syncwarp(gmask);
                prefetch_state(kk + 1);
                const int k = perm[kk];
                const int cn = mycnt[k];
                const int2 *lk = mylists + (int64_t)k * LW;
                const int2 *lb = lbuf + (kk % 3) * kSparseCapW;
                auto entry = [&](int j) -> int2 { return j < kSparseCapW ? lb[j] : __ldcg(lk + j); };
                auto eval = [&]() -> float2 {
                    float sg = 0.f, sh = 0.f;
                    for (int j0 = glane; j0 < cn; j0 += CH * kU) {
                        int2 e[kU];
                        float2 st[kU];
#pragma unroll
                        for (int t = 0; t < kU; ++t) e[t] = j0 + CH * t < cn ? entry(j0 + CH * t) : make_int2(0, 0);
#pragma unroll
                        for (int t = 0; t < kU; ++t) st[t] = j0 + CH * t < cn ? wq[XS * (e[t].x)] : make_float2(0.f, 0.f);
#pragma unroll
                        for (int t = 0; t < kU; ++t) {
                            const float av = __int_as_float(e[t].y);
                            sg = fmaf(st[t].x, av, sg);
                            sh = fmaf(st[t].y * av, av, sh);
                        }
                    }
                    return reduce(sg, sh);
                };
                auto update = [&](float d, int dc) {
                    for (int j0 = glane; j0 < cn; j0 += CH * kU) {
                        int2 e[kU];
                        float2 st[kU];
#pragma unroll
                        for (int t = 0; t < kU; ++t) e[t] = j0 + CH * t < cn ? entry(j0 + CH * t) : make_int2(0, 0);
#pragma unroll
                        for (int t = 0; t < kU; ++t) st[t] = j0 + CH * t < cn ? xv[XS * (e[t].x)] : make_float2(0.f, 0.f);
#pragma unroll
                        for (int t = 0; t < kU; ++t) {
                            if (j0 + CH * t < cn) {
                                const int p = e[t].x;
                                int terms = dc != 0 ? (int)tm[p] : 0;
                                const float xn = step_x(st[t].x, __int_as_float(e[t].y), d, dc, terms);
                                if (dc != 0) tm[p] = (uint16_t)terms;
                                const float ri = recip(xn + eps_div);
                                xv[XS * (p)].x = xn;
                                wq[XS * (p)] = make_float2(st[t].y * ri, st[t].y * ri * ri);
                            }
                        }
                    }
                    __syncwarp(gmask);
                };
                const float xk = newton_coordinate(a, x_init[k], a.sumA[k], eval, update, tally);
                if (tid_g == 0) x_out[k] = xk;
                // the buffer just read is refilled two coordinates on
                __syncwarp(gmask);
            }
            cp_async_wait<0>();
        }
        if (a.unit_obj) {
            float t = 0.f;
            for (int c = w; c < nchunks; c += kNW) {
                const int p = CH * c + glane;
                if (p < L) {
                    const float2 s = xv[XS * (p)];
                    t += kl_term(s.y, s.x, eps_div);
                }
            }
            double dt = (double)t;
#pragma unroll
            for (int o = CH / 2; o > 0; o >>= 1) dt += __shfl_xor_sync(gmask, dt, o);
            if constexpr (kCluster) {
                double *rd = reinterpret_cast<double *>(red + parity * kNW);
                if (lane == 0) rd[warp_in_block] = dt;
                __syncthreads();
                parity ^= 1;
                double cta = 0.0;
                if (warp_in_block == 0)
                    for (int i = 0; i < kNW; ++i) cta += rd[i];
                cluster_sum(static_cast<unsigned long long>(__double_as_longlong(cta)),
                            [&](const unsigned long long *sl, int n) {
                                double tot = 0.0;
                                for (int i = 0; i < n; ++i) tot += __longlong_as_double(static_cast<long long>(sl[i]));
                                dt = tot;
                            });
            } else if constexpr (kCta) {
                double *rd = reinterpret_cast<double *>(red + parity * kNW);
                if (lane == 0) rd[warp_in_block] = dt;
                __syncthreads();
                double tot = 0.0;
#pragma unroll
                for (int i = 0; i < kNW; ++i) tot += rd[i];
                parity ^= 1;
                dt = tot;
            }
            if (tid_g == 0 && crank == 0) a.unit_obj[u] = dt;
        }
        group_sync();
        // drop this warp's finished list lines from L2 (whole lines only)
        for (int k = 0; k < r; ++k) {
            const int lines = (mycnt[k] * 8) / 128;
            const char *l0 = reinterpret_cast<const char *>(mylists + (int64_t)k * LW);
            for (int i = glane; i < lines; i += CH) asm volatile("discard.global.L2 [%0], 128;" ::"l"(l0 + 128 * i) : "memory");
        }
        if (crank == 0) {
            for (int k = tid_g; k < r; k += GS) {
                const float xk = x_out[k];
                if (!(xk == xk)) atomicOr(a.err, kErrNaN);
                a.X[u * ldr + k] = xk;
            }
        }
    }
    if (tid_g == 0 && crank == 0) flush_tally(a, tally);
    // no CTA of a cluster may leave while a peer can still write into its shared memory
    if constexpr (kCluster) cooperative_groups::this_cluster().sync();
}

// ---------------------------------------------------------------------------
// Host side: the bucket table and the plan.
// ---------------------------------------------------------------------------
struct KernelKind {
    const void *fn;
    int nt, k, cl;  // threads per CTA (32: warp groups), nonzeros per thread, CTAs per cluster
    int d;          // ring depth (tile columns in flight); 0 for the giant kernel
    const char *name;
};

constexpr int kClusterNT = 512, kClusterK = 12, kClusterD = 4;
const KernelKind kKinds[] = {
    // sub-warp groups (G lanes per unit) come first: for the lengths they hold
    // they replace the one-warp kernels below
    {(const void *)sweep_sub_kernel<8, 4, 4>, 8, 4, 1, 4, "sweep_sub_g8_k4"},
    {(const void *)sweep_sub_kernel<16, 4, 4>, 16, 4, 1, 4, "sweep_sub_g16_k4"},
    {(const void *)sweep_kernel<32, 1, 4>, 32, 1, 1, 4, "sweep_warp_k1"},
    {(const void *)sweep_kernel<32, 2, 4>, 32, 2, 1, 4, "sweep_warp_k2"},
    {(const void *)sweep_kernel<32, 4, 4>, 32, 4, 1, 4, "sweep_warp_k4"},
    {(const void *)sweep_kernel<32, 8, 4>, 32, 8, 1, 4, "sweep_warp_k8"},
    {(const void *)sweep_kernel<32, 16, 4>, 32, 16, 1, 4, "sweep_warp_k16"},
    {(const void *)sweep_kernel<128, 8, 8>, 128, 8, 1, 8, "sweep_cta128_k8"},
    {(const void *)sweep_kernel<256, 8, 6>, 256, 8, 1, 6, "sweep_cta256_k8"},
    {(const void *)sweep_kernel<512, 8, 4>, 512, 8, 1, 4, "sweep_cta512_k8"},
    {(const void *)sweep_kernel<512, 16, 3>, 512, 16, 1, 3, "sweep_cta512_k16"},
    {(const void *)sweep_cluster_kernel<kClusterNT, kClusterK, kClusterD>, kClusterNT, kClusterK, 2, kClusterD, "sweep_cluster2"},
    {(const void *)sweep_cluster_kernel<kClusterNT, kClusterK, kClusterD>, kClusterNT, kClusterK, 4, kClusterD, "sweep_cluster4"},
    {(const void *)sweep_cluster_kernel<kClusterNT, kClusterK, kClusterD>, kClusterNT, kClusterK, 8, kClusterD, "sweep_cluster8"},
    {(const void *)sweep_cluster_kernel<kClusterNT, kClusterK, kClusterD>, kClusterNT, kClusterK, 16, kClusterD, "sweep_cluster16"},
    {(const void *)sweep_giant_kernel, kGiantNT, 0, 1, 0, "sweep_giant"},
};
constexpr int kNumKinds = sizeof(kKinds) / sizeof(kKinds[0]);
constexpr int kGiantKind = kNumKinds - 1;

// First usable kind whose capacity holds L (giant beyond every capacity).
int kind_for_length(int64_t L, const std::vector<char> &usable) {
    for (int i = 0; i < kGiantKind; ++i)
        if (usable[i] && L <= (int64_t)kKinds[i].nt * kKinds[i].k * kKinds[i].cl) return i;
    return kGiantKind;
}

size_t cluster_smem_bytes(int r, int ldr) {
    return ring_layout(r, ldr, kClusterNT, kClusterK, kClusterD, true).bytes +
           (2 * kClusterMax + 2) * sizeof(unsigned long long);
}

// Clusters of `cl` CTAs of the cluster kernel that fit on the device at once.
int active_clusters(int cl, size_t smem) {
    const void *fn = kKinds[kGiantKind - 1].fn;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kClusterNT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

struct SparseKind {
    const void *fn;
    int nt;          // threads per CTA group, or 32 for warp-level groups
    int g;           // lanes per warp-level group (8, 16 or 32)
    int cap;         // longest unit (nonzeros) of the class; 0: no limit
    bool smem;       // per-nonzero state in shared memory (else in the slot)
    bool compact;    // shared state without w_p, q_p
    int cl;          // CTAs per cluster (1: no cluster)
    int max_groups;  // resident groups per SM at most (0: as many as fit)
    const char *name;
};
// List classes (units of more than kDenseBelow nonzeros): one warp per unit
// up to 1,024 nonzeros, then one CTA of 128 / 256 / 256 (compact state) /
// 512 threads per unit up to 2,048 / 4,096 / 8,192 / kSliceCap nonzeros (the
// compact 256-thread class fits two CTAs per SM where the 512-thread one fits
// one: 47.2 -> 46.5 ms per W half on the large corpus at a steady state; one
// compact warp per unit up to 2,048 measured slower, 49.8), then a cluster of 2, 3, 4, 6, 8 or
// 16 such 512-thread CTAs (the smallest whose slices hold kSliceCap), all
// with the per-nonzero state in shared memory; past that (or where no cluster
// can be scheduled) one 512-thread CTA per unit with the state in the slot.
// A class whose shared-memory layout does not fit passes its units on to the
// next one (at r <= 256 the 128- and 256-thread layouts always fit, the
// 512-thread one up to at least 20,992 nonzeros). One warp per unit with the
// state in the slot, for 1,025..8,192 nonzeros, measured 9% slower per step
// at r = 100.
// Nonzeros per 512-thread CTA (alone or in a cluster): at most 16,384, so that
// at a density of up to 1/4 a warp's list of a coordinate (<= 256 entries)
// fits the registers it prefetches into (longer lists read their tail from
// global memory in the dependent chain of every evaluation and update).
// Measured on the large corpus at r = 100: 117.6 ms per step at 16,384 vs
// 121.3 at 12,288 (more units in clusters, which leave SMs idle) and 120.4
// without a cap (22,016 by shared memory).
constexpr int kSliceCap = 16384;
#define NMFKL_SPARSE_CLU sparse_kernel<512, true, true, true>
const SparseKind kSparseKinds[] = {
    {(const void *)sparse_kernel<32, true>, 32, 32, 512, true, false, 1, 0, "sparse_warp"},
    {(const void *)sparse_kernel<32, true, true>, 32, 32, 1024, true, true, 1, 0, "sparse_warp_1k"},
    {(const void *)sparse_kernel<128, true>, 128, 32, 2048, true, false, 1, 0, "sparse_cta128"},
    {(const void *)sparse_kernel<256, true>, 256, 32, 4096, true, false, 1, 0, "sparse_cta256"},
    {(const void *)sparse_kernel<256, true, true>, 256, 32, 8192, true, true, 1, 0, "sparse_cta256c"},
    {(const void *)sparse_kernel<512, true, true>, 512, 32, kSliceCap, true, true, 1, 0, "sparse_cta512"},
    {(const void *)NMFKL_SPARSE_CLU, 512, 32, 2 * kSliceCap, true, true, 2, 0, "sparse_cluster2"},
    {(const void *)NMFKL_SPARSE_CLU, 512, 32, 3 * kSliceCap, true, true, 3, 0, "sparse_cluster3"},
    {(const void *)NMFKL_SPARSE_CLU, 512, 32, 4 * kSliceCap, true, true, 4, 0, "sparse_cluster4"},
    {(const void *)NMFKL_SPARSE_CLU, 512, 32, 6 * kSliceCap, true, true, 6, 0, "sparse_cluster6"},
    {(const void *)NMFKL_SPARSE_CLU, 512, 32, 8 * kSliceCap, true, true, 8, 0, "sparse_cluster8"},
    {(const void *)NMFKL_SPARSE_CLU, 512, 32, 16 * kSliceCap, true, true, 16, 0, "sparse_cluster16"},
    {(const void *)sparse_kernel<512, false>, 512, 32, 0, false, false, 1, 0, "sparse_giant"},
};
#undef NMFKL_SPARSE_CLU
constexpr int kNumSparseKinds = sizeof(kSparseKinds) / sizeof(kSparseKinds[0]);

// Row length of a unit of L nonzeros in a group of the kind: its slice (a
// cluster's CTAs split the unit) in whole chunks of every warp of the group.
int64_t sparse_lcap(const SparseKind &sk, int64_t L) {
    const int64_t chunk = sk.nt > 32 ? sk.nt : sk.g;
    const int64_t slice = (L + sk.cl - 1) / sk.cl;
    return std::max<int64_t>(chunk, (slice + chunk - 1) / chunk * chunk);
}

// Dynamic shared memory of one group of the kind at row length lcap: the
// layout, plus for clusters the exchange slots and mbarriers.
size_t sparse_group_smem(const SparseKind &sk, int r, int ldr, int64_t lcap) {
    size_t b = sparse_layout(r, ldr, sk.nt, sk.smem ? (int)lcap : 0, sk.compact).bytes;
    if (sk.cl > 1) b += (2 * (size_t)kClusterMax + 2) * sizeof(unsigned long long);
    return b;
}

// Clusters of the kind that can be resident at once at the given shared memory.
int sparse_active_clusters(const SparseKind &sk, size_t smem) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(sk.cl);
    cfg.blockDim = dim3(sk.nt);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = sk.cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, sk.fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// The first usable class whose cap holds L and, for shared-memory state,
// whose group layout fits the per-block limit.
int sparse_kind_for_length(int64_t L, int r, int ldr, int optin, const std::vector<char> &usable) {
    for (int i = 0; i < kNumSparseKinds - 1; ++i) {
        const SparseKind &sk = kSparseKinds[i];
        if (!usable[i] || L > sk.cap) continue;
        if (sk.smem && sparse_group_smem(sk, r, ldr, sparse_lcap(sk, L)) > (size_t)optin) continue;
        return i;
    }
    return kNumSparseKinds - 1;
}

}  // namespace

const char *kind_name(int kind) { return kKinds[kind].name; }
const char *bucket_name(const Bucket &b) {
    if (b.group) return group_kind(b.kind).name;
    return b.sparse ? kSparseKinds[b.kind].name : kKinds[b.kind].name;
}

// Kernel timer name of a bucket: "<kernel>/F" or "<kernel>/W", and for a
// dense-tile bucket that the list plan runs, "<kernel>/F/list" or
// "<kernel>/W/list" (static storage). Both plans' buckets are launched when
// the plan is chosen on the device, and the plan not chosen returns at once:
// the names keep those empty launches apart from the ones that ran.
const char *bucket_timer_name(const Bucket &b, int side) {
    static const std::vector<std::string> names = [] {
        std::vector<std::string> v;
        for (int s = 0; s < 2; ++s) {
            for (int i = 0; i < kNumKinds; ++i) v.push_back(std::string(kKinds[i].name) + (s ? "/W" : "/F"));
            for (int i = 0; i < kNumSparseKinds; ++i) v.push_back(std::string(kSparseKinds[i].name) + (s ? "/W" : "/F"));
            for (int i = 0; i < group_kind_count(); ++i) v.push_back(std::string(group_kind(i).name) + (s ? "/W" : "/F"));
            for (int i = 0; i < kNumKinds; ++i) v.push_back(std::string(kKinds[i].name) + (s ? "/W/list" : "/F/list"));
        }
        return v;
    }();
    const int per = kNumKinds + kNumSparseKinds + group_kind_count() + kNumKinds;
    const int idx = b.group ? kNumKinds + kNumSparseKinds + b.kind
                            : (b.sparse ? kNumKinds + b.kind
                                        : (b.borrowed ? kNumKinds + kNumSparseKinds + group_kind_count() + b.kind
                                                      : b.kind));
    return names[side * per + idx].c_str();
}



void free_plan(nmfkl_ctx *c) {
    for (int side = 0; side < 2; ++side) {
        for (auto *pl : {&c->plan[side], &c->plan_sparse[side]}) {
            for (auto &b : *pl)
                if (b.d_units && !b.borrowed) cudaFree(b.d_units);
            pl->clear();
        }
    }
}

namespace {

// Units in decreasing length, equal lengths in increasing unit id (the order
// the persistent kernels take them in), by a counting sort on the length.
std::vector<int32_t> order_by_length(const std::vector<int64_t> &ptr) {
    const int64_t units = (int64_t)ptr.size() - 1;
    int64_t max_len = 0;
    for (int64_t u = 0; u < units; ++u) max_len = std::max(max_len, ptr[u + 1] - ptr[u]);
    std::vector<int32_t> order(units);
    if (max_len > (int64_t)1 << 26) {  // a count array that large: compare instead
        for (int64_t u = 0; u < units; ++u) order[u] = (int32_t)u;
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
            return (ptr[x + 1] - ptr[x]) > (ptr[y + 1] - ptr[y]);
        });
        return order;
    }
    std::vector<int64_t> start(max_len + 2, 0);
    for (int64_t u = 0; u < units; ++u) start[max_len - (ptr[u + 1] - ptr[u]) + 1]++;
    for (int64_t i = 1; i <= max_len + 1; ++i) start[i] += start[i - 1];
    for (int64_t u = 0; u < units; ++u) order[start[max_len - (ptr[u + 1] - ptr[u])]++] = (int32_t)u;
    return order;
}

// Units of at most this many nonzeros have two alternatives in the list plan,
// chosen per length class (at most 32, 64, 128, 256 nonzeros): the dense-tile
// warp kernels of the dense plan, or the sub-warp group kernels over lists of
// the compressed factor rows. Measured by the autotuner on the large corpus at
// r = 100 after 25 sweeps, ms per F half: dense 2.3 / 4.6 / 9.3 / 12.3, group
// 10.4 / 20.8 / 56.1 / 68.9 (the group kernels' list building issues one
// scattered store per list entry); with Eq. 2 weights that leave the factors
// 99% zeros the group kernels win every class (the lists are nearly empty).
// The dense kernels are the default.
constexpr int64_t kDenseBelow = 256;

// Sparse-list plan of one half: the dense buckets of the units of at most
// kDenseBelow nonzeros, then one bucket per length class; a class's tile row
// length is its longest unit rounded up to whole chunks of every warp.
nmfkl_status plan_side_sparse(nmfkl_ctx *c, int side, const std::vector<int64_t> &ptr,
                              const std::vector<int32_t> &order, int optin) {
    const int64_t units = (int64_t)ptr.size() - 1;
    const int r = c->p.r, ldr = c->ldr;
    std::vector<std::vector<int32_t>> lists(kNumSparseKinds);
    std::vector<int64_t> maxlen(kNumSparseKinds, 0), nnz(kNumSparseKinds, 0);
    // cluster classes that the device can schedule (at the largest shared memory they may take)
    std::vector<char> usable(kNumSparseKinds, 1);
    std::vector<int> clusters_fit(kNumSparseKinds, 0);
    for (int i = 0; i < kNumSparseKinds; ++i) {
        if (kSparseKinds[i].cl <= 1) continue;
        clusters_fit[i] = sparse_active_clusters(kSparseKinds[i], (size_t)optin);
        usable[i] = clusters_fit[i] > 0;
    }
    // units of at most kDenseBelow nonzeros: the dense-tile warp buckets of the
    // dense plan, and the group kinds, by length (one alternative per class runs)
    for (const Bucket &d : c->plan[side]) {
        const KernelKind &kk = kKinds[d.kind];
        if (kk.cl == 1 && kk.k > 0 && kk.nt <= 32 && (int64_t)kk.nt * kk.k <= kDenseBelow) {
            Bucket b = d;
            b.borrowed = true;
            b.short_class = group_kind_for_length((int64_t)kk.nt * kk.k);
            c->plan_sparse[side].push_back(b);
        }
    }
    {
        const int ngk = group_kind_count();
        std::vector<std::vector<int32_t>> glists(ngk);
        std::vector<int64_t> gmax(ngk, 0), gnnz(ngk, 0);
        for (int32_t u : order) {
            const int64_t L = ptr[u + 1] - ptr[u];
            if (L > kDenseBelow) continue;
            const int gk = group_kind_for_length(L);
            glists[gk].push_back(u);
            gmax[gk] = std::max(gmax[gk], L);
            gnnz[gk] += L;
        }
        for (int gk = 0; gk < ngk; ++gk) {
            if (glists[gk].empty()) continue;
            const GroupKindInfo &info = group_kind(gk);
            Bucket b{};
            b.sparse = true;
            b.group = true;
            b.kind = gk;
            b.nt = info.g;
            b.k = 0;
            b.cl = 1;
            b.count = (int32_t)glists[gk].size();
            b.max_len = gmax[gk];
            b.nnz = gnnz[gk];
            b.lcap = info.lmax;
            b.short_class = gk;
            // groups per block: as many whole warps of groups as shared memory
            // holds, up to 256 threads; a class whose groups do not fit keeps
            // only its dense-tile alternative
            int gpb = 256 / info.g;
            while (gpb > 0 && group_block_smem(gk, r, ldr, gpb) > (size_t)optin) gpb -= 32 / info.g;
            if (gpb <= 0) continue;
            b.block = gpb * info.g;
            b.smem = group_block_smem(gk, r, ldr, gpb);
            int per_sm = 0;
            if (!cuda_ok(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, info.fn, b.block, b.smem),
                         "occupancy"))
                return NMFKL_ECUDA;
            if (per_sm < 1) {
                c->err = std::string("kernel ") + info.name + " cannot be resident";
                return NMFKL_EINVAL;
            }
            const int64_t need_blocks = (b.count + gpb - 1) / gpb;
            b.grid = (int)std::min<int64_t>(need_blocks, (int64_t)per_sm * c->num_sms);
            b.groups = b.grid * gpb;
            b.slot_floats = group_slot_floats(gk, r);
            if (!cuda_ok(c, cudaMalloc(&b.d_units, sizeof(int32_t) * glists[gk].size()), "alloc unit list"))
                return NMFKL_ENOMEM;
            if (!cuda_ok(c, cudaMemcpy(b.d_units, glists[gk].data(), sizeof(int32_t) * glists[gk].size(),
                                       cudaMemcpyHostToDevice),
                         "copy unit list"))
                return NMFKL_ECUDA;
            c->plan_sparse[side].push_back(b);
        }
    }
    // in decreasing length, so each class's list comes out longest first; the
    // class of a length is looked up once per distinct length
    int64_t last_len = -1;
    int kind = 0;
    for (int32_t u : order) {
        const int64_t L = ptr[u + 1] - ptr[u];
        if (L <= kDenseBelow) break;
        if (L != last_len) {
            kind = sparse_kind_for_length(L, r, ldr, optin, usable);
            last_len = L;
        }
        lists[kind].push_back(u);
        maxlen[kind] = std::max(maxlen[kind], L);
        nnz[kind] += L;
    }
    (void)units;
    for (int kind = 0; kind < kNumSparseKinds; ++kind) {
        auto &lst = lists[kind];
        if (lst.empty()) continue;
        const SparseKind &sk = kSparseKinds[kind];
        const bool smem_state = sk.smem;
        const bool cta = sk.nt > 32;
        Bucket b{};
        b.sparse = true;
        b.kind = kind;
        b.nt = sk.nt;
        b.k = 0;
        b.cl = sk.cl;
        b.count = (int32_t)lst.size();
        b.max_len = maxlen[kind];
        b.nnz = nnz[kind];
        b.lcap = (int32_t)sparse_lcap(sk, b.max_len);
        const size_t gbytes = sparse_group_smem(sk, r, ldr, b.lcap);
        int gpb = 1;
        if (!cta) {
            // warps per block: the most resident warps per SM that shared memory allows
            int sm_bytes = 0;
            cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device);
            int best = 0;
            for (int g = 256 / sk.g; g >= 1; --g) {
                if (gbytes * g > (size_t)optin) continue;
                const int blocks = std::min(2, (int)((size_t)sm_bytes / (gbytes * g + 1024)));
                if (blocks * g > best) {
                    best = blocks * g;
                    gpb = g;
                }
            }
        }
        b.block = cta ? sk.nt : sk.g * gpb;
        b.smem = gbytes * gpb;
        if (b.smem > (size_t)optin) {
            c->err = "sparse plan: shared memory exceeds the device limit";
            return NMFKL_EINVAL;
        }
        int per_sm = 0;
        if (!cuda_ok(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sk.fn, b.block, b.smem), "occupancy"))
            return NMFKL_ECUDA;
        if (per_sm < 1) {
            c->err = std::string("kernel ") + sk.name + " cannot be resident";
            return NMFKL_EINVAL;
        }
        if (sk.max_groups > 0) per_sm = std::max(1, std::min(per_sm, sk.max_groups / gpb));
        const int64_t need_blocks = (b.count + gpb - 1) / gpb;
        b.grid = (int)std::min<int64_t>(need_blocks, (int64_t)per_sm * c->num_sms);
        if (sk.cl > 1) {  // whole clusters, as many as can be resident (one unit each at a time)
            const int nclu = sparse_active_clusters(sk, b.smem);
            if (nclu < 1) {
                c->err = std::string("kernel ") + sk.name + " cannot be resident";
                return NMFKL_EINVAL;
            }
            b.grid = (int)std::min<int64_t>(b.count, nclu) * sk.cl;
        }
        b.groups = b.grid * gpb;
        b.slot_floats = sparse_slot_floats(r, b.lcap, smem_state);
        if (!cuda_ok(c, cudaMalloc(&b.d_units, sizeof(int32_t) * lst.size()), "alloc unit list")) return NMFKL_ENOMEM;
        if (!cuda_ok(c, cudaMemcpy(b.d_units, lst.data(), sizeof(int32_t) * lst.size(), cudaMemcpyHostToDevice),
                     "copy unit list"))
            return NMFKL_ECUDA;
        c->plan_sparse[side].push_back(b);
    }
    return NMFKL_OK;
}

}  // namespace

nmfkl_status plan_side(nmfkl_ctx *c, int side) {
    const int64_t units = side == 0 ? c->m : c->n;
    std::vector<int64_t> ptr(units + 1);
    const int64_t *dptr = side == 0 ? c->colptr : c->rowptr;
    if (!cuda_ok(c, cudaMemcpy(ptr.data(), dptr, sizeof(int64_t) * (units + 1), cudaMemcpyDeviceToHost),
                 "copy offsets"))
        return NMFKL_ECUDA;
    const int r0 = c->p.r, ldr0 = c->ldr;
    std::vector<char> usable(kNumKinds, 1);
    std::vector<int> clusters_fit(kNumKinds, 0);
    for (int kind = 0; kind < kGiantKind; ++kind) {
        if (kKinds[kind].cl <= 1) continue;
        clusters_fit[kind] = active_clusters(kKinds[kind].cl, cluster_smem_bytes(r0, ldr0));
        usable[kind] = clusters_fit[kind] > 0;
    }
    std::vector<std::vector<int32_t>> lists(kNumKinds);
    std::vector<int64_t> maxlen(kNumKinds, 0), nnz(kNumKinds, 0);
    const std::vector<int32_t> order = order_by_length(ptr);
    for (int32_t u : order) {  // each class's list comes out longest first
        const int64_t L = ptr[u + 1] - ptr[u];
        const int kind = kind_for_length(L, usable);
        lists[kind].push_back(u);
        maxlen[kind] = std::max(maxlen[kind], L);
        nnz[kind] += L;
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    optin -= 1024;  // headroom for the kernels' static shared memory
    const int r = c->p.r, ldr = c->ldr;
    for (int kind = 0; kind < kNumKinds; ++kind) {
        auto &lst = lists[kind];
        if (lst.empty()) continue;
        Bucket b{};
        b.kind = kind;
        b.nt = kKinds[kind].nt;
        b.k = kKinds[kind].k;
        b.count = (int32_t)lst.size();
        b.max_len = maxlen[kind];
        b.nnz = nnz[kind];
        b.cl = kKinds[kind].cl;
        if (b.cl > 1) {
            b.block = b.nt;
            b.smem = cluster_smem_bytes(r, ldr);
            const int nclu = (int)std::min<int64_t>(b.count, clusters_fit[kind]);
            b.grid = nclu * b.cl;
            b.groups = b.grid;
            b.lcap = b.nt * b.k;
            b.slot_floats = ((int64_t)r * b.lcap + 63) / 64 * 64;
            if (!cuda_ok(c, cudaMalloc(&b.d_units, sizeof(int32_t) * lst.size()), "alloc unit list"))
                return NMFKL_ENOMEM;
            if (!cuda_ok(c, cudaMemcpy(b.d_units, lst.data(), sizeof(int32_t) * lst.size(), cudaMemcpyHostToDevice),
                         "copy unit list"))
                return NMFKL_ECUDA;
            c->plan[side].push_back(b);
            continue;
        }
        const bool cta = b.nt > 32;
        const int warps = b.nt / 32;
        const size_t gbytes = kind == kGiantKind ? group_smem_bytes(r, ldr, warps, true)
                                                 : ring_layout(r, ldr, b.nt, b.k, kKinds[kind].d, cta).bytes;
        int groups_per_block = 1;
        if (!cta) {
            // warp groups: up to 8 per block; sub-warp groups: whole warps of
            // them, up to 256 threads
            const int step = b.nt < 32 ? 32 / b.nt : 1;
            groups_per_block = b.nt == 32 ? warp_block_threads(b.k, kModeHalf) / 32 : 256 / b.nt;
            while (groups_per_block > step && gbytes * groups_per_block > (size_t)optin) groups_per_block -= step;
        }
        b.block = cta ? b.nt : b.nt * groups_per_block;
        b.smem = gbytes * (cta ? 1 : groups_per_block);
        if (b.smem > (size_t)optin) {
            c->err = "shared memory plan exceeds the device limit";
            return NMFKL_EINVAL;
        }
        int per_sm = 0;
        if (!cuda_ok(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kKinds[kind].fn, b.block, b.smem),
                     "occupancy"))
            return NMFKL_ECUDA;
        if (per_sm < 1) {
            c->err = std::string("kernel ") + kKinds[kind].name + " cannot be resident";
            return NMFKL_EINVAL;
        }
        if (kind == kGiantKind) per_sm = 1;
        const int64_t need_blocks = (b.count + groups_per_block - 1) / groups_per_block;
        b.grid = (int)std::min<int64_t>(need_blocks, (int64_t)per_sm * c->num_sms);
        b.groups = b.grid * groups_per_block;
        if (kind == kGiantKind) {
            b.lcap = (int32_t)((b.max_len + 31) / 32 * 32);
            b.slot_floats = (int64_t)(r + 5) * b.lcap;
        } else {
            b.lcap = b.nt * b.k;
            b.slot_floats = (int64_t)r * b.lcap;
        }
        b.slot_floats = (b.slot_floats + 63) / 64 * 64;
        if (!cuda_ok(c, cudaMalloc(&b.d_units, sizeof(int32_t) * lst.size()), "alloc unit list"))
            return NMFKL_ENOMEM;
        if (!cuda_ok(c, cudaMemcpy(b.d_units, lst.data(), sizeof(int32_t) * lst.size(), cudaMemcpyHostToDevice),
                     "copy unit list"))
            return NMFKL_ECUDA;
        c->plan[side].push_back(b);
    }
    const nmfkl_status st = plan_side_sparse(c, side, ptr, order, optin);
    if (st != NMFKL_OK) return st;
    // Overlapped launches and scratch. A plan with cluster buckets runs its
    // buckets longest first, each launch allowed to start while the previous
    // one drains (programmatic dependent launch): the later buckets' blocks
    // fill the SMs that clusters leave idle and the earlier buckets' tails.
    // Its buckets may then run at once, so each gets scratch slots of its own
    // (128-byte aligned offsets). A plan without clusters runs its buckets
    // one after the other in the table's order and shares one scratch region.
    // (Measured on the large corpus at a steady state, W half: 48.8 ms in
    // sequence, 47.0 overlapped longest first, 54.6 overlapped shortest first;
    // F half, which has no clusters: 40.8 in sequence, 48.0 overlapped: the
    // concurrent dense-tile buckets contend for L2.) The two plans of a half
    // never both use their scratch (the one not chosen returns before
    // touching it), and halves run one after the other, so the buffer is the
    // largest plan's need.
    for (int lp = 0; lp < 2; ++lp) {
        std::vector<Bucket> &plan = lp ? c->plan_sparse[side] : c->plan[side];
        bool clusters = false;
        for (const Bucket &b : plan) clusters = clusters || b.cl > 1;
        c->overlap[side][lp] = c->pdl && clusters;
        int64_t off = 0, need = 0;
        for (Bucket &b : plan) {
            const int64_t fl = (b.slot_floats * b.groups + 31) / 32 * 32;
            b.scratch_off = c->overlap[side][lp] ? off : 0;
            off += fl;
            need = std::max(need, c->overlap[side][lp] ? off : fl);
        }
        c->scratch_floats = std::max<int64_t>(c->scratch_floats, need);
    }
    return NMFKL_OK;
}

// The kernel that runs a short length class of the list plan: the chosen one
// when the plan has it (a group kind that cannot be resident is left out).
int short_kernel(const nmfkl_ctx *c, int side, int cls) {
    if (c->short_choice[side][cls] == 0) return 0;
    for (const Bucket &b : c->plan_sparse[side])
        if (b.group && b.short_class == cls) return 1;
    return 0;
}

namespace {
// Launches one bucket of a half on stream st.
// One bucket's persistent launch. `pdl`: the launch may begin while the
// previous kernel on the stream is still running (programmatic dependent
// launch; every bucket kernel waits for its predecessor before it exits).
cudaError_t launch_bucket(const Bucket &b, HalfArgs &a, cudaStream_t st, bool pdl) {
    void *args[] = {&a};
    const void *fn = b.group ? group_kind(b.kind).fn : (b.sparse ? kSparseKinds[b.kind].fn : kKinds[b.kind].fn);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(b.grid);
    cfg.blockDim = dim3(b.block);
    cfg.dynamicSmemBytes = b.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (b.cl > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = b.cl;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    if (pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// The plan of a half from the fixed factor's density at the nonzeros of V
// (sum of row counts weighted by row lengths, over nnz * r): the lists below
// the threshold, else the dense tile.
__global__ void plan_select_kernel(const unsigned long long *dens, double denom, double threshold, int32_t *sel,
                                   double *dens_out) {
    const double d = denom > 0.0 ? (double)*dens / denom : 0.0;
    *dens_out = d;
    *sel = d < threshold ? 1 : 0;
}
}  // namespace

// One half of Algorithm 1 on the context stream, without any host
// synchronization (capturable): sumA, the compressed rows of the fixed
// factor and their density, the device-side choice of plan (list_mode 0),
// then every bucket of the plans that may run, in order; a bucket of the plan
// not chosen returns at once. With `sweep_dev` set the kernels read the sweep
// index from it (a captured step), else they take `sweep`.
nmfkl_status run_half(nmfkl_ctx *c, int side, int64_t sweep, const int64_t *sweep_dev, int64_t u0, int64_t u1) {
    TraceRange trace(side == 0 ? "F half" : "W half");
    const bool F = side == 0;
    const float *At = F ? c->Wt : c->Ft;
    float *X = F ? c->Ft : c->Wt;
    float *sumA = F ? c->sumW : c->sumF;
    nmfkl_status st = launch_colsum(c, At, F ? c->n : c->m, sumA, c->dsum[F ? 0 : 1]);
    if (st != NMFKL_OK) return st;
    HalfArgs a{};
    a.ptr = F ? c->colptr : c->rowptr;
    a.idx = F ? c->rowidx : c->colidx;
    a.val = F ? c->val : c->rval;
    a.At = At;
    a.X = X;
    a.sumA = sumA;
    a.r = c->p.r;
    a.ldr = c->ldr;
    a.alpha = (float)(F ? c->p.alpha_F : c->p.alpha_W);
    a.beta = (float)(F ? c->p.beta_F : c->p.beta_W);
    a.eps_grad = (float)c->p.eps_grad;
    a.eps_div = (float)c->p.eps_div;
    a.eps_x = (float)c->p.eps_x;
    a.max_inner = c->p.max_inner;
    a.grad_mode = c->p.grad_mode;
    a.break_mode = c->p.break_mode;
    a.div_mode = c->p.div_mode;
    a.perm_mode = c->p.perm_mode;
    a.seed = c->p.seed;
    a.sweep = sweep;
    a.sweep_dev = sweep_dev;
    a.u0 = u0;
    a.u1 = u1;
    a.side = side;
    a.scratch = c->scratch;
    a.counters = c->counters;
    a.err = c->err_flag;
    a.wait_cycles = c->wait_cycles;
    a.unit_obj = F ? nullptr : c->unit_obj;
    a.ccnt = c->crow_cnt;
    a.ck = c->crow_k;
    a.ca = c->crow_a;
    // The fixed factor's rows compressed to their positive entries (for the
    // group kernels of the list plan); the same pass measures the factor's
    // density at the nonzeros of V.
    if (!cuda_ok(c, cudaMemsetAsync(c->dens + side, 0, sizeof(unsigned long long), c->stream), "density reset"))
        return NMFKL_ECUDA;
    {
        const int tok = timer_begin(c, "compress_rows");
        launch_compress(c->stream, At, F ? c->n : c->m, c->ldr, c->p.r, F ? c->rowptr : c->colptr, c->crow_cnt,
                        c->crow_k, c->crow_a, c->dens + side);
        timer_end(c, tok);
        if (!cuda_ok(c, cudaGetLastError(), "compress rows")) return NMFKL_ECUDA;
    }
    // dense tile or sparse lists (list_mode): in automatic mode, chosen on the
    // device, the lists when the fixed factor is less dense than the threshold
    // at the nonzeros of V; 1 and 2 fix the plan
    bool run_plan[2] = {c->p.list_mode != 2, c->p.list_mode != 1};
    if (c->p.list_mode == 0) {
        const double denom = (double)c->nnz * c->p.r;
        plan_select_kernel<<<1, 1, 0, c->stream>>>(c->dens + side, denom, c->list_threshold, c->plan_sel + side,
                                                    c->dens_out + side);
        if (!cuda_ok(c, cudaGetLastError(), "plan select")) return NMFKL_ECUDA;
        a.plan_sel = c->plan_sel + side;
    } else {
        c->used_sparse[side] = c->p.list_mode == 2 ? 1 : 0;
    }
    // Buckets run one after another on the context stream. (Running them
    // concurrently on side streams, so that one bucket's tail overlaps the
    // next one's work, was measured slower: 139 vs 133 ms per step on the
    // large corpus; the concurrent persistent kernels contend for L2.)
    // Every work queue of the half is reset at once, so that the bucket
    // launches follow one another directly on the stream; in a plan marked
    // for overlap (see plan_side) they go longest first and each may start
    // while the one before drains its tail (not with kernel timing on, where
    // events separate the launches).
    if (!cuda_ok(c, cudaMemsetAsync(c->queues + side * kQueuesPerSide, 0, kQueuesPerSide * sizeof(int32_t),
                                    c->stream),
                 "reset queues"))
        return NMFKL_ECUDA;
    int qi = 0;
    bool first = true;
    for (int lp = 0; lp < 2; ++lp) {
        if (!run_plan[lp]) continue;
        a.plan_id = lp;
        const std::vector<Bucket> &plan = lp ? c->plan_sparse[side] : c->plan[side];
        const bool overlap = c->overlap[side][lp] && !c->timing;
        const int nb = (int)plan.size();
        for (int i = 0; i < nb; ++i) {
            const Bucket &b = plan[overlap ? nb - 1 - i : i];
            // the alternative of a short length class that was not chosen
            if (b.short_class >= 0 && (b.group ? 1 : 0) != short_kernel(c, side, b.short_class)) continue;
            if (qi >= kQueuesPerSide) {
                c->err = "run_half: more buckets than work queues";
                return NMFKL_EINVAL;
            }
            a.units = b.d_units;
            a.count = b.count;
            a.queue = c->queues + side * kQueuesPerSide + qi++;
            a.scratch = c->scratch + b.scratch_off;
            a.slot_floats = b.slot_floats;
            a.lcap = b.lcap;
            const int tok = timer_begin(c, bucket_timer_name(b, side));
            const cudaError_t e = launch_bucket(b, a, c->stream, overlap && !first);
            first = false;
            timer_end(c, tok);
            if (!cuda_ok(c, e, bucket_name(b))) return NMFKL_ECUDA;
        }
    }
    return NMFKL_OK;
}


// ---------------------------------------------------------------------------
// Fold-in (nmfkl_foldin): the F half alone under the context's fixed W, each
// new column running its own passes of Algorithm 2 until its objective
// settles. Columns are sorted into length classes on the device, so that the
// whole launch sequence (sums of W, classification, one persistent launch per
// class, output transpose) depends on no host-side knowledge of the lengths
// and is captured once into a CUDA graph.
// ---------------------------------------------------------------------------
namespace {

const KernelKind kFoldTable[kFoldKinds] = {
    {(const void *)sweep_kernel<32, 1, 8, kModeFold>, 32, 1, 1, 8, "foldin_warp_k1"},
    {(const void *)sweep_kernel<32, 2, 8, kModeFold>, 32, 2, 1, 8, "foldin_warp_k2"},
    {(const void *)sweep_kernel<32, 4, 8, kModeFold>, 32, 4, 1, 8, "foldin_warp_k4"},
    {(const void *)sweep_kernel<32, 8, 6, kModeFold>, 32, 8, 1, 6, "foldin_warp_k8"},
    {(const void *)sweep_kernel<32, 16, 4, kModeFold>, 32, 16, 1, 4, "foldin_warp_k16"},
    {(const void *)sweep_kernel<128, 8, 8, kModeFold>, 128, 8, 1, 8, "foldin_cta128_k8"},
    {(const void *)sweep_kernel<256, 8, 6, kModeFold>, 256, 8, 1, 6, "foldin_cta256_k8"},
    {(const void *)sweep_kernel<512, 8, 4, kModeFold>, 512, 8, 1, 4, "foldin_cta512_k8"},
    {(const void *)sweep_kernel<512, 16, 3, kModeFold>, 512, 16, 1, 3, "foldin_cta512_k16"},
};

__host__ __device__ inline int fold_kind_for_length(int64_t L) {
    constexpr int cap[kFoldKinds] = {32, 64, 128, 256, 512, 1024, 2048, 4096, 8192};
    for (int i = 0; i < kFoldKinds; ++i)
        if (L <= cap[i]) return i;
    return -1;
}

// Sorts the columns into the length classes; a column longer than the last
// class sets error bit 4 and is left out.
__global__ void fold_bucketize_kernel(const int64_t *colptr, int64_t m, int32_t *lists, int64_t cap_m,
                                      int32_t *counts, int32_t *err) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int kind = fold_kind_for_length(colptr[j + 1] - colptr[j]);
        if (kind < 0) {
            atomicOr(err, 4);
            continue;
        }
        const int pos = atomicAdd(&counts[kind], 1);
        lists[(int64_t)kind * cap_m + pos] = (int32_t)j;
    }
}

HalfArgs fold_args(nmfkl_ctx *c, FoldState &f, bool with_ids, double rel_tol, int32_t max_sweeps) {
    HalfArgs a{};
    a.ptr = f.colptr;
    a.idx = f.rowidx;
    a.val = f.val;
    a.At = c->Wt;
    a.X = f.Ft;
    a.sumA = c->sumW;
    a.r = c->p.r;
    a.ldr = c->ldr;
    a.alpha = (float)c->p.alpha_F;
    a.beta = (float)c->p.beta_F;
    a.eps_grad = (float)c->p.eps_grad;
    a.eps_div = (float)c->p.eps_div;
    a.eps_x = (float)c->p.eps_x;
    a.max_inner = c->p.max_inner;
    a.grad_mode = c->p.grad_mode;
    a.break_mode = c->p.break_mode;
    a.div_mode = c->p.div_mode;
    a.perm_mode = c->p.perm_mode;
    a.seed = c->p.seed;
    a.side = 0;
    a.scratch = f.scratch;
    a.counters = c->counters;
    a.err = f.ctl + 2 * kFoldKinds;
    a.wait_cycles = c->wait_cycles;
    a.unit_ids = with_ids ? f.ids : nullptr;
    a.max_sweeps = max_sweeps;
    a.rel_tol = rel_tol;
    a.sumA64 = c->dsum[0];
    a.sweeps_done = f.sweeps;
    a.unit_final = f.obj;
    return a;
}

// The fold-in launch sequence on `st` (capturable: no host synchronization,
// no allocation).
cudaError_t fold_enqueue(nmfkl_ctx *c, cudaStream_t st, int64_t m_new, bool with_ids, double rel_tol,
                         int32_t max_sweeps, bool timed) {
    FoldState &f = *c->fold;
    launch_colsum_raw(st, c->Wt, c->n, c->ldr, c->p.r, c->dpart, c->sumW, c->dsum[0]);
    cudaError_t e = cudaMemsetAsync(f.ctl, 0, sizeof(int32_t) * (2 * kFoldKinds + 1), st);
    if (e != cudaSuccess) return e;
    if (m_new > 0) {
        const int blocks = (int)std::min<int64_t>((m_new + 255) / 256, 4096);
        fold_bucketize_kernel<<<blocks, 256, 0, st>>>(f.colptr, m_new, f.lists, f.cap_m, f.ctl, f.ctl + 2 * kFoldKinds);
    }
    HalfArgs a = fold_args(c, f, with_ids, rel_tol, max_sweeps);
    for (int kind = 0; kind < kFoldKinds && m_new > 0; ++kind) {
        a.units = f.lists + (int64_t)kind * f.cap_m;
        a.count = 0;
        a.count_dev = f.ctl + kind;
        a.queue = f.ctl + kFoldKinds + kind;
        a.slot_floats = f.slot_floats[kind];
        a.lcap = f.lcap[kind];
        void *args[] = {&a};
        const int tok = timed ? timer_begin(c, kFoldTable[kind].name) : -1;
        e = cudaLaunchKernel(kFoldTable[kind].fn, dim3(f.grid[kind]), dim3(f.block[kind]), args, f.smem[kind], st);
        if (timed) timer_end(c, tok);
        if (e != cudaSuccess) return e;
    }
    if (m_new > 0) launch_from_unit_major_raw(st, f.Ft, f.Fout, c->p.r, m_new, c->ldr);
    return cudaGetLastError();
}

}  // namespace

int foldin_kind_for_length(int64_t L) { return fold_kind_for_length(L); }

void free_fold(nmfkl_ctx *c) {
    FoldState *f = c->fold;
    if (!f) return;
    if (f->graph) cudaGraphExecDestroy(f->graph);
    if (f->cap_stream) cudaStreamDestroy(f->cap_stream);
    cudaFree(f->colptr); cudaFree(f->ids); cudaFree(f->rowidx); cudaFree(f->val); cudaFree(f->Ft);
    cudaFree(f->Fout); cudaFree(f->lists); cudaFree(f->ctl); cudaFree(f->sweeps); cudaFree(f->obj);
    cudaFree(f->scratch);
    delete f;
    c->fold = nullptr;
}

// Sizes the per-class launches and the tile scratch once per context.
nmfkl_status fold_plan(nmfkl_ctx *c) {
    FoldState &f = *c->fold;
    if (f.planned) return NMFKL_OK;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    optin -= 1024;
    const int r = c->p.r, ldr = c->ldr;
    int64_t scratch = 0;
    for (int kind = 0; kind < kFoldKinds; ++kind) {
        const KernelKind &kk = kFoldTable[kind];
        const bool cta = kk.nt > 32;
        const size_t gbytes = ring_layout(r, ldr, kk.nt, kk.k, kk.d, cta).bytes;
        int gpb = 1;
        if (!cta) {
            gpb = 8;
            while (gpb > 1 && gbytes * gpb > (size_t)optin) --gpb;
        }
        f.block[kind] = cta ? kk.nt : 32 * gpb;
        f.smem[kind] = gbytes * (cta ? 1 : gpb);
        if (f.smem[kind] > (size_t)optin) {
            c->err = "fold-in: shared memory plan exceeds the device limit";
            return NMFKL_EINVAL;
        }
        int per_sm = 0;
        if (!cuda_ok(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kk.fn, f.block[kind], f.smem[kind]),
                     "fold-in occupancy"))
            return NMFKL_ECUDA;
        if (per_sm < 1) {
            c->err = std::string("fold-in kernel ") + kk.name + " cannot be resident";
            return NMFKL_EINVAL;
        }
        f.grid[kind] = per_sm * c->num_sms;
        f.groups[kind] = f.grid[kind] * gpb;
        f.lcap[kind] = kk.nt * kk.k;
        f.slot_floats[kind] = ((int64_t)r * f.lcap[kind] + 63) / 64 * 64;
        scratch = std::max<int64_t>(scratch, f.slot_floats[kind] * f.groups[kind]);
    }
    if (!cuda_ok(c, cudaMalloc(&f.scratch, sizeof(float) * (size_t)scratch), "fold-in scratch")) return NMFKL_ENOMEM;
    if (!cuda_ok(c, cudaMemset(f.scratch, 0, sizeof(float) * (size_t)scratch), "zero fold-in scratch"))
        return NMFKL_ECUDA;
    f.scratch_floats = scratch;
    if (!cuda_ok(c, cudaStreamCreateWithFlags(&f.cap_stream, cudaStreamNonBlocking), "fold-in capture stream"))
        return NMFKL_ECUDA;
    f.planned = true;
    return NMFKL_OK;
}

nmfkl_status foldin_run(nmfkl_ctx *c, int64_t m_new, bool with_ids, double rel_tol, int32_t max_sweeps,
                        bool use_graph) {
    nmfkl_status st = fold_plan(c);
    if (st != NMFKL_OK) return st;
    FoldState &f = *c->fold;
    if (!use_graph) {
        return cuda_ok(c, fold_enqueue(c, c->stream, m_new, with_ids, rel_tol, max_sweeps, c->timing), "fold-in launch")
                   ? NMFKL_OK
                   : NMFKL_ECUDA;
    }
    if (!f.graph || f.graph_m != m_new || f.graph_ids != with_ids || f.graph_tol != rel_tol ||
        f.graph_sweeps != max_sweeps) {
        if (f.graph) {
            cudaGraphExecDestroy(f.graph);
            f.graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        if (!cuda_ok(c, cudaStreamBeginCapture(f.cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture"))
            return NMFKL_ECUDA;
        const cudaError_t e = fold_enqueue(c, f.cap_stream, m_new, with_ids, rel_tol, max_sweeps, false);
        const cudaError_t e2 = cudaStreamEndCapture(f.cap_stream, &g);
        if (!cuda_ok(c, e, "fold-in capture") || !cuda_ok(c, e2, "end capture")) {
            if (g) cudaGraphDestroy(g);
            return NMFKL_ECUDA;
        }
        const cudaError_t e3 = cudaGraphInstantiate(&f.graph, g, 0);
        cudaGraphDestroy(g);
        if (!cuda_ok(c, e3, "instantiate fold-in graph")) {
            f.graph = nullptr;
            return NMFKL_ECUDA;
        }
        f.graph_m = m_new;
        f.graph_ids = with_ids;
        f.graph_tol = rel_tol;
        f.graph_sweeps = max_sweeps;
    }
    const int tok = timer_begin(c, "foldin_graph");
    const cudaError_t e = cudaGraphLaunch(f.graph, c->stream);
    timer_end(c, tok);
    return cuda_ok(c, e, "fold-in graph launch") ? NMFKL_OK : NMFKL_ECUDA;
}

// The plain scheme the batched launch is measured against: one launch per
// column (the same kernel, one group), in column order.
nmfkl_status foldin_per_doc(nmfkl_ctx *c, int64_t m_new, double rel_tol, int32_t max_sweeps) {
    nmfkl_status st = fold_plan(c);
    if (st != NMFKL_OK) return st;
    FoldState &f = *c->fold;
    std::vector<int64_t> ptr(m_new + 1);
    if (!cuda_ok(c, cudaMemcpyAsync(ptr.data(), f.colptr, sizeof(int64_t) * (m_new + 1), cudaMemcpyDeviceToHost,
                                    c->stream),
                 "copy fold-in offsets") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "fold-in offsets sync"))
        return NMFKL_ECUDA;
    // per column: a one-entry unit list (the column itself) and its own work counter
    std::vector<int32_t> iota(m_new);
    for (int64_t j = 0; j < m_new; ++j) iota[j] = (int32_t)j;
    if (!cuda_ok(c, cudaMemcpyAsync(f.lists, iota.data(), sizeof(int32_t) * m_new, cudaMemcpyHostToDevice, c->stream),
                 "fold-in unit ids") ||
        !cuda_ok(c, cudaMemsetAsync(f.lists + f.cap_m, 0, sizeof(int32_t) * m_new, c->stream), "fold-in counters") ||
        !cuda_ok(c, cudaMemsetAsync(f.ctl, 0, sizeof(int32_t) * (2 * kFoldKinds + 1), c->stream), "fold-in flags") ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream), "fold-in per-column setup"))
        return NMFKL_ECUDA;
    launch_colsum_raw(c->stream, c->Wt, c->n, c->ldr, c->p.r, c->dpart, c->sumW, c->dsum[0]);
    HalfArgs a = fold_args(c, f, false, rel_tol, max_sweeps);
    a.count = 1;
    for (int64_t j = 0; j < m_new; ++j) {
        const int kind = fold_kind_for_length(ptr[j + 1] - ptr[j]);
        if (kind < 0) {
            c->err = "fold-in: a column has more nonzeros than the longest length class";
            return NMFKL_EINVAL;
        }
        const KernelKind &kk = kFoldTable[kind];
        a.units = f.lists + j;
        a.queue = f.lists + f.cap_m + j;
        a.slot_floats = f.slot_floats[kind];
        a.lcap = f.lcap[kind];
        void *args[] = {&a};
        if (!cuda_ok(c, cudaLaunchKernel(kk.fn, dim3(1), dim3(kk.nt), args,
                                         ring_layout(c->p.r, c->ldr, kk.nt, kk.k, kk.d, kk.nt > 32).bytes, c->stream),
                     kk.name))
            return NMFKL_ECUDA;
    }
    launch_from_unit_major_raw(c->stream, f.Ft, f.Fout, c->p.r, m_new, c->ldr);
    return cuda_ok(c, cudaGetLastError(), "fold-in per-column launches") ? NMFKL_OK : NMFKL_ECUDA;
}


// ---------------------------------------------------------------------------
// Allocation-free F half (nmfkl_sweep_F_noalloc in include/nmfkl.h).
//
// Its scratch is the file-scope array below, held by every GPU that loads
// this library until the process exits:
//   [0, 2 MiB)        colsum partials (1024 blocks x up to 256 doubles)
//   [2 MiB, +4 KiB)   control: work counter, error flags, work counters,
//                     sumW (FP32 and FP64)
//   [2 MiB + 4 KiB, 32 MiB)  per-warp tiles (32*K x r floats each)
// Host code cannot use the array's name as a device address, so the address
// is taken with cudaGetSymbolAddress once per device (with that device
// current) on the first call there, and passed to the kernels.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocBytes = size_t(32) << 20;
constexpr size_t kNoAllocPartBytes = size_t(2) << 20;
constexpr size_t kNoAllocCtlBytes = 4096;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_ptr[kNoAllocMaxDevices] = {};

struct NoAllocCtl {  // lives at the start of the control block
    int32_t queue;
    int32_t err;
    unsigned long long counters[4];
};

const KernelKind kFreeKinds[] = {
    {(const void *)sweep_kernel<32, 1, 8, kModeFree>, 32, 1, 1, 8, "sweep_warp_k1_noalloc"},
    {(const void *)sweep_kernel<32, 2, 8, kModeFree>, 32, 2, 1, 8, "sweep_warp_k2_noalloc"},
    {(const void *)sweep_kernel<32, 4, 8, kModeFree>, 32, 4, 1, 8, "sweep_warp_k4_noalloc"},
    {(const void *)sweep_kernel<32, 8, 6, kModeFree>, 32, 8, 1, 6, "sweep_warp_k8_noalloc"},
};
}  // namespace

extern "C" nmfkl_status nmfkl_sweep_F_noalloc(const nmfkl_params *p, int64_t n, int64_t m, int32_t max_len,
                                              const int64_t *colptr, const int32_t *rowidx, const float *val,
                                              const float *Wt, float *Ft, int64_t sweep, void *stream) {
    if (!p || p->r < 1 || p->r > kMaxR || n < 1 || m < 1 || n > INT32_MAX || m > INT32_MAX || max_len < 0 ||
        max_len > 256 || !colptr || !Wt || !Ft || (max_len > 0 && (!rowidx || !val)))
        return NMFKL_EINVAL;
    // the factor rows are read and written 16 bytes at a time
    if ((reinterpret_cast<uintptr_t>(Wt) | reinterpret_cast<uintptr_t>(Ft)) % 16 != 0) return NMFKL_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return NMFKL_ECUDA;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return NMFKL_ECUDA;
            }
            g_noalloc_ptr[dev] = static_cast<unsigned char *>(ptr);
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int r = p->r, ldr = (r + 3) / 4 * 4;
    double *part = reinterpret_cast<double *>(base);
    unsigned char *ctl_bytes = base + kNoAllocPartBytes;
    NoAllocCtl *ctl = reinterpret_cast<NoAllocCtl *>(ctl_bytes);
    float *sumW = reinterpret_cast<float *>(ctl_bytes + 256);
    double *sumW_d = reinterpret_cast<double *>(ctl_bytes + 256 + 4 * kMaxR);
    float *tiles = reinterpret_cast<float *>(base + kNoAllocPartBytes + kNoAllocCtlBytes);
    const size_t tile_bytes = kNoAllocBytes - kNoAllocPartBytes - kNoAllocCtlBytes;

    int kind = 0;
    while (kind < 3 && max_len > 32 * kFreeKinds[kind].k) ++kind;
    const KernelKind &kk = kFreeKinds[kind];
    const int lcap = 32 * kk.k;
    const int64_t slot_floats = ((int64_t)r * lcap + 63) / 64 * 64;
    int optin = 0, sms = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return NMFKL_ECUDA;
    }
    optin -= 1024;
    const size_t gbytes = ring_layout(r, ldr, 32, kk.k, kk.d, false).bytes;
    int gpb = 8;
    while (gpb > 1 && gbytes * gpb > (size_t)optin) --gpb;
    const size_t smem = gbytes * gpb;
    if (kernel_attributes(dev) != cudaSuccess) return NMFKL_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kk.fn, 32 * gpb, smem) != cudaSuccess || per_sm < 1)
        return NMFKL_ECUDA;
    const int64_t slots = (int64_t)(tile_bytes / sizeof(float)) / slot_floats;
    const int64_t blocks_fit = slots / gpb;
    const int64_t grid = std::min<int64_t>(std::min<int64_t>((m + gpb - 1) / gpb, (int64_t)per_sm * sms), blocks_fit);
    if (grid < 1) return NMFKL_EINVAL;

    if (cudaMemsetAsync(ctl_bytes, 0, sizeof(NoAllocCtl), st) != cudaSuccess) return NMFKL_ECUDA;
    launch_colsum_raw(st, Wt, n, ldr, r, part, sumW, sumW_d);

    HalfArgs a{};
    a.ptr = colptr;
    a.idx = rowidx;
    a.val = val;
    a.At = Wt;
    a.X = Ft;
    a.sumA = sumW;
    a.r = r;
    a.ldr = ldr;
    a.alpha = (float)p->alpha_F;
    a.beta = (float)p->beta_F;
    a.eps_grad = (float)p->eps_grad;
    a.eps_div = (float)p->eps_div;
    a.eps_x = (float)p->eps_x;
    a.max_inner = p->max_inner;
    a.grad_mode = p->grad_mode;
    a.break_mode = p->break_mode;
    a.div_mode = p->div_mode;
    a.perm_mode = p->perm_mode;
    a.seed = p->seed;
    a.sweep = sweep;
    a.side = 0;
    a.units = nullptr;
    a.count = (int32_t)m;
    a.queue = &ctl->queue;
    a.scratch = tiles;
    a.slot_floats = slot_floats;
    a.lcap = lcap;
    a.counters = ctl->counters;
    a.err = &ctl->err;
    a.wait_cycles = kDefaultWaitCycles;
    a.unit_obj = nullptr;
    void *args[] = {&a};
    if (cudaLaunchKernel(kk.fn, dim3((unsigned)grid), dim3(32 * gpb), args, smem, st) != cudaSuccess)
        return NMFKL_ECUDA;
    int32_t err = 0;
    if (cudaMemcpyAsync(&err, &ctl->err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NMFKL_ECUDA;
    if (err & 4) return NMFKL_EINVAL;
    if (err & 1) return NMFKL_ENUMERIC;
    return NMFKL_OK;
}

// Coordinate orders exactly as the sweep kernels draw them (one warp per unit).
__global__ void debug_perm_kernel(const int64_t *cols, int64_t count, int r, int64_t sweep, int side,
                                  int perm_mode, uint64_t seed, int32_t *out) {
    __shared__ uint64_t words[8][kMaxR];
    __shared__ __align__(16) uint8_t perm[8][kMaxR];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * 8 + w;
    if (c >= count) return;
    ids_swaps_warp(reinterpret_cast<uint8_t *>(words[w]), r, cols[c], sweep, side, perm_mode, seed, lane);
    __syncwarp();
    if (lane == 0) fisher_yates(perm[w], reinterpret_cast<const uint8_t *>(words[w]), r);
    __syncwarp();
    for (int t = lane; t < r; t += 32) out[c * r + t] = perm[w][t];
}

nmfkl_status launch_debug_perm(nmfkl_ctx *c, int64_t sweep, int side, int64_t count, const int64_t *cols,
                               int32_t *out) {
    if (count <= 0) return NMFKL_OK;
    const int tok = timer_begin(c, "debug_perm");
    debug_perm_kernel<<<(unsigned)((count + 7) / 8), 256, 0, c->stream>>>(cols, count, c->p.r, sweep, side,
                                                                          c->p.perm_mode, c->p.seed, out);
    timer_end(c, tok);
    return cuda_ok(c, cudaGetLastError(), "debug_perm") ? NMFKL_OK : NMFKL_ECUDA;
}

namespace {
// The dynamic shared memory limit and the cluster-size permission are
// per-function state shared by every context in the process. Contexts that
// run at once on different streams or host threads (the serving loop) plan
// different sizes, so each kernel is given the device's opt-in maximum once,
// instead of each plan setting its own size.
constexpr int kMaxDevices = 64;
std::once_flag g_attr_once[kMaxDevices];
cudaError_t g_attr_err[kMaxDevices];

cudaError_t set_attrs_for(const void *fn, int optin) {
    // the limit covers dynamic shared memory only; the kernel's static part counts against the block total
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}
}  // namespace

cudaError_t kernel_attributes(int device) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_attr_once[device], [device] {
        int optin = 0;
        cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
        for (int i = 0; e == cudaSuccess && i < kNumKinds; ++i) e = set_attrs_for(kKinds[i].fn, optin);
        for (int i = 0; e == cudaSuccess && i < kFoldKinds; ++i) e = set_attrs_for(kFoldTable[i].fn, optin);
        for (int i = 0; e == cudaSuccess && i < kNumSparseKinds; ++i) e = set_attrs_for(kSparseKinds[i].fn, optin);
        for (const KernelKind &kk : kFreeKinds) {
            if (e != cudaSuccess) break;
            e = set_attrs_for(kk.fn, optin);
        }
        if (e == cudaSuccess) e = group_attributes(optin);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kKinds[kGiantKind - 1].fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        for (int i = 0; e == cudaSuccess && i < kNumSparseKinds; ++i)
            if (kSparseKinds[i].cl > 1)
                e = cudaFuncSetAttribute(kSparseKinds[i].fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        g_attr_err[device] = e;
    });
    return g_attr_err[device];
}

}  // namespace nmfkl
