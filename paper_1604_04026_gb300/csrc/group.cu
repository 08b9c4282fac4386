// Sub-warp group kernels: Algorithm 2 on short units (at most 256 nonzeros)
// with G lanes per unit and 32/G units per warp, visiting per coordinate only
// the nonzeros whose factor entry A_pk is positive.
//
// A term with A_pk = 0 adds nothing to either sum of Eq. Partial, and its x_p
// does not move when x_k does (Section 2 on the sparsity of W and F), so
// coordinate k needs only the list {(p, A_pk) : A_pk > 0}. At a typical fit
// the fixed factor is ~10-15% dense at a document's nonzeros, so a short
// unit's list holds a few entries per coordinate: one warp per unit (a
// 32-lane reduction per evaluation for a handful of entries) wastes most of
// its lanes and instructions, and a dense transposed tile per unit (r floats
// per nonzero, written and read back once) overflows L2 at the number of
// units in flight. Here:
//   * the fixed factor's rows are compressed once per half to their positive
//     entries in k order (compress_rows_kernel: count, k, value), so staging
//     touches only those;
//   * a group of G lanes owns one unit; a warp runs 32/G units of similar
//     length in step (their coordinates are visited in each unit's own order,
//     the group reductions are log2(G) shuffles);
//   * staging builds the unit's per-coordinate lists in the group's global
//     scratch slot, deterministically: pass A counts the entries of each
//     coordinate per lane (lane-private byte counters in shared memory) and
//     computes x_p; a scan gives each (coordinate, lane) its segment; pass B
//     writes the entries. List k is the lanes' segments in lane order, each in
//     increasing p, so the summation order is a fixed function of the data;
//   * the per-nonzero state (x_p, v_p, positive-term count) is in shared
//     memory; the list entries of the next two coordinates are loaded into
//     registers while the current one runs.
#include "common.cuh"
#include "device_util.cuh"

#include <algorithm>

namespace nmfkl {

namespace {

using namespace dev;

// Shared memory of one group, by offset:
//   x[ldr] (the unit's coordinates) | perm[r] | off[r+1] (int32 list starts) |
//   a region of max(cnt[r*G] bytes + state, 8 (r-1) bytes): first the Philox
//   words of the unit's order, then the per-(coordinate, lane) counts and the
//   state xs[LMAX] (float), vs[LMAX] (float), ts[LMAX] (uint16).
struct GroupLayout {
    size_t perm_off, off_off, cnt_off, xs_off, vs_off, ts_off, bytes;
};
__host__ __device__ inline GroupLayout group_layout(int r, int ldr, int g, int lmax) {
    GroupLayout y{};
    size_t o = align16(4 * (size_t)ldr);
    y.perm_off = o;
    o = align16(o + (size_t)r);
    y.off_off = o;
    o = align16(o + 4 * ((size_t)r + 1));
    y.cnt_off = o;
    const size_t cnt_bytes = align16((size_t)r * g);
    y.xs_off = o + cnt_bytes;
    y.vs_off = y.xs_off + 4 * (size_t)lmax;
    y.ts_off = y.vs_off + 4 * (size_t)lmax;
    const size_t state = cnt_bytes + 10 * (size_t)lmax, words = 8 * (size_t)(r > 1 ? r - 1 : 1);
    const size_t region = state > words ? state : words;
    y.bytes = align16(o + region);
    return y;
}

// List entries per lane held in registers for one coordinate (more are read
// from the slot as they are needed).
constexpr int kGroupE = 4;

struct ListSet {
    int j0 = 0, cnt = 0;
    int p[kGroupE];
    float a[kGroupE];
};

// Calls body(k, A_ik) for the positive entries of compressed row i (c of
// them), in k order. The row is read 16 entries at a time, every load of a
// batch issued before the first is used.
template <class Body>
__device__ __forceinline__ void row_entries(const float *__restrict__ ca, const uint8_t *__restrict__ ck, int64_t i,
                                            int ldr, int c, Body &&body) {
    const float4 *a4p = reinterpret_cast<const float4 *>(ca + i * ldr);
    const uint32_t *k4p = reinterpret_cast<const uint32_t *>(ck + i * ldr);
    for (int t0 = 0; t0 < c; t0 += 16) {
        float4 av[4];
        uint32_t kv[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            av[b] = make_float4(0.f, 0.f, 0.f, 0.f);
            kv[b] = 0u;
            if (t0 + 4 * b < c) {
                av[b] = __ldg(a4p + (t0 >> 2) + b);
                kv[b] = __ldg(k4p + (t0 >> 2) + b);
            }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float f[4] = {av[b].x, av[b].y, av[b].z, av[b].w};
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (t0 + 4 * b + s < c) body((int)((kv[b] >> (8 * s)) & 0xffu), f[s]);
        }
    }
}

// Calls body(p, i, v, c) for the nonzeros p = first, first + step, ... < L of
// a unit (row index i, value v, compressed-row count c), loading the next
// nonzero's index and count while the current one is processed.
template <class Body>
__device__ __forceinline__ void unit_nonzeros(const int32_t *__restrict__ idx, const float *__restrict__ val,
                                              const int32_t *__restrict__ cc, int64_t base, int L, int first,
                                              int step, Body &&body) {
    int p = first;
    if (p >= L) return;
    int i = __ldg(idx + base + p);
    float v = __ldg(val + base + p);
    int c = __ldg(cc + i);
    int i1 = 0;
    float v1 = 0.f;
    if (p + step < L) {
        i1 = __ldg(idx + base + p + step);
        v1 = __ldg(val + base + p + step);
    }
    for (; p < L; p += step) {
        int c1 = 0, i2 = 0;
        float v2 = 0.f;
        if (p + step < L) c1 = __ldg(cc + i1);
        if (p + 2 * step < L) {
            i2 = __ldg(idx + base + p + 2 * step);
            v2 = __ldg(val + base + p + 2 * step);
        }
        body(p, i, v, c);
        i = i1;
        v = v1;
        c = c1;
        i1 = i2;
        v1 = v2;
    }
}

template <int G, int LMAX>
__global__ void __launch_bounds__(256) group_kernel(HalfArgs a) {
    PdlScope pdl;
    if (plan_skip(a)) return;
    static_assert(G >= 4 && G <= 32 && (G & (G - 1)) == 0, "G: 4, 8, 16 or 32 lanes");
    static_assert(LMAX <= 256, "list entries hold p in 8 bits");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int glane = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << gbase);
    const int group_in_block = threadIdx.x / G;
    const int groups_per_block = blockDim.x / G;
    const int group_global = blockIdx.x * groups_per_block + group_in_block;
    constexpr int kPerWarp = 32 / G;

    const int r = a.r, ldr = a.ldr;
    const GroupLayout lay = group_layout(r, ldr, G, LMAX);
    // the block's copy of sumA, then one region per group
    float *sumA = reinterpret_cast<float *>(smem_raw);
    for (int k = threadIdx.x; k < r; k += blockDim.x) sumA[k] = a.sumA[k];
    __syncthreads();
    unsigned char *gs = smem_raw + align16(4 * (size_t)ldr) + (size_t)group_in_block * lay.bytes;
    float *x = reinterpret_cast<float *>(gs);
    uint8_t *perm = gs + lay.perm_off;
    int *off = reinterpret_cast<int *>(gs + lay.off_off);
    uint8_t *cnt = gs + lay.cnt_off;
    uint64_t *words = reinterpret_cast<uint64_t *>(gs + lay.cnt_off);
    float *xs = reinterpret_cast<float *>(gs + lay.xs_off);
    float *vs = reinterpret_cast<float *>(gs + lay.vs_off);
    uint16_t *ts = reinterpret_cast<uint16_t *>(gs + lay.ts_off);
    // the group's scratch slot: list values, then list positions p
    float *la = a.scratch + (int64_t)group_global * a.slot_floats;
    uint8_t *lp = reinterpret_cast<uint8_t *>(la + (int64_t)LMAX * r);

    const float eps_div = a.eps_div;
    const int count = a.count_dev ? *a.count_dev : a.count;
    Tally tally;

    for (;;) {
        __syncwarp();
        int q = 0;
        if (lane == 0) q = atomicAdd(a.queue, kPerWarp);
        q = __shfl_sync(kFull, q, 0);
        if (q >= count) break;
        const int qi = q + lane / G;
        // a group without a unit (the last batch) or with a unit it cannot hold
        // still runs the warp-wide coordinate loop below, without work
        bool work = qi < count;
        int64_t u = 0, base = 0;
        int L = 0;
        if (work) {
            u = a.units[qi];
            if (out_of_range(a, u)) work = false;
            base = a.ptr[u];
            L = (int)(a.ptr[u + 1] - base);
            if (L > LMAX || L < 0) {  // cannot happen with a consistent plan; refuse rather than overrun
                if (glane == 0) atomicOr(a.err, kErrLength);
                work = false;
            }
        }
        {
            if (work) {
                const int64_t perm_unit = a.unit_ids ? a.unit_ids[u] : u;
                // ---- the unit's coordinates and its order of Algorithm 1's ids
                for (int k = glane; k < ldr; k += G) x[k] = a.X[u * ldr + k];
                ids_swaps_warp(reinterpret_cast<uint8_t *>(words), r, perm_unit, sweep_of(a), a.side, a.perm_mode, a.seed, glane, G);
                __syncwarp(gmask);
                if (glane == 0) fisher_yates(perm, reinterpret_cast<const uint8_t *>(words), r);
                __syncwarp(gmask);
                // the words are consumed: the region now holds the counts and the state
                for (int i = glane; i < (r * G) / 4; i += G) reinterpret_cast<uint32_t *>(cnt)[i] = 0u;
                __syncwarp(gmask);

                // ---- pass A: x_p = sum_k A_pk x_k (Algorithm 2's first step, in k
                // order over the positive entries), its positive-term count, and
                // the number of list entries per (coordinate, lane)
                const int32_t *cc = a.ccnt;
                unit_nonzeros(a.idx, a.val, cc, base, L, glane, G, [&](int p, int i, float v, int c) {
                    float acc = 0.f;
                    int terms = 0;
                    row_entries(a.ca, a.ck, i, ldr, c, [&](int k, float av) {
                        const float xk = x[k];
                        acc = fmaf(av, xk, acc);
                        terms += xk > 0.f ? 1 : 0;
                        cnt[k * G + glane] += 1;
                    });
                    xs[p] = terms == 0 ? 0.f : acc;
                    vs[p] = v;
                    ts[p] = (uint16_t)terms;
                });
                __syncwarp(gmask);

                // ---- list starts: per coordinate the lanes' segments in lane
                // order (exclusive prefix over the lanes, kept in cnt), then an
                // exclusive scan of the per-coordinate totals over k into off
                for (int k = glane; k < r; k += G) {
                    uint8_t *row = cnt + k * G;
                    int run = 0;
#pragma unroll
                    for (int l = 0; l < G; ++l) {
                        const int cl = row[l];
                        row[l] = (uint8_t)run;
                        run += cl;
                    }
                    off[k] = run;
                }
                __syncwarp(gmask);
                {
                    const int chunk = (r + G - 1) / G;
                    const int k0 = glane * chunk, k1 = min(r, k0 + chunk);
                    int sum = 0;
                    for (int k = k0; k < k1; ++k) sum += off[k];
                    int incl = sum;
#pragma unroll
                    for (int d = 1; d < G; d <<= 1) {
                        const int y = __shfl_up_sync(gmask, incl, d, G);
                        if (glane >= d) incl += y;
                    }
                    int run = incl - sum;
                    __syncwarp(gmask);
                    for (int k = k0; k < k1; ++k) {
                        const int t = off[k];
                        off[k] = run;
                        run += t;
                    }
                    if (glane == G - 1) off[r] = incl;
                }
                __syncwarp(gmask);

                // ---- pass B: each lane writes its entries (p, A_pk) at its segment
                unit_nonzeros(a.idx, a.val, cc, base, L, glane, G, [&](int p, int i, float, int c) {
                    row_entries(a.ca, a.ck, i, ldr, c, [&](int k, float av) {
                        uint8_t &seg = cnt[k * G + glane];
                        const int pos = off[k] + seg;
                        seg = (uint8_t)(seg + 1);
                        la[pos] = av;
                        lp[pos] = (uint8_t)p;
                    });
                });
                __threadfence_block();
            }
            __syncwarp();
            {
                // ---- Algorithm 2 over the unit's coordinates, list entries only.
                // The warp's groups visit their coordinates in step: one warp-wide
                // barrier per coordinate keeps them converged, so that every
                // instruction serves all 32/G units.
                auto fetch = [&](int pos, ListSet &S) {
                    S.cnt = 0;
                    S.j0 = 0;
                    if (work && pos < r) {
                        const int k = perm[pos];
                        S.j0 = off[k];
                        S.cnt = off[k + 1] - S.j0;
#pragma unroll
                        for (int t = 0; t < kGroupE; ++t) {
                            const int j = glane + G * t;
                            if (j < S.cnt) {
                                S.p[t] = __ldcg(lp + S.j0 + j);
                                S.a[t] = __ldcg(la + S.j0 + j);
                            }
                        }
                    }
                };
                auto coordinate = [&](int kk, const ListSet &S) {
                    const int k = perm[kk];
                    auto term = [&](int p, float av, float &sg, float &sh) {
                        const float ri = recip(xs[p] + eps_div);
                        const float wp = vs[p] * ri;
                        const float qp = wp * ri;
                        sg = fmaf(wp, av, sg);
                        sh = fmaf(qp * av, av, sh);
                    };
                    auto eval = [&]() -> float2 {
                        float sg = 0.f, sh = 0.f;
#pragma unroll
                        for (int t = 0; t < kGroupE; ++t)
                            if (glane + G * t < S.cnt) term(S.p[t], S.a[t], sg, sh);
                        for (int j = glane + G * kGroupE; j < S.cnt; j += G)
                            term(__ldcg(lp + S.j0 + j), __ldcg(la + S.j0 + j), sg, sh);
#pragma unroll
                        for (int o = G / 2; o > 0; o >>= 1) {
                            sg += __shfl_xor_sync(gmask, sg, o);
                            sh += __shfl_xor_sync(gmask, sh, o);
                        }
                        return make_float2(sg, sh);
                    };
                    auto update = [&](float d, int dc) {
                        auto upd = [&](int p, float av) {
                            int terms = dc != 0 ? (int)ts[p] : 0;
                            const float xn = step_x(xs[p], av, d, dc, terms);
                            if (dc != 0) ts[p] = (uint16_t)terms;
                            xs[p] = xn;
                        };
#pragma unroll
                        for (int t = 0; t < kGroupE; ++t)
                            if (glane + G * t < S.cnt) upd(S.p[t], S.a[t]);
                        for (int j = glane + G * kGroupE; j < S.cnt; j += G)
                            upd(__ldcg(lp + S.j0 + j), __ldcg(la + S.j0 + j));
                        // the next evaluation reads these entries from other lanes
                        __syncwarp(gmask);
                    };
                    if (work) {
                        const float xk = newton_coordinate(a, x[k], sumA[k], eval, update, tally);
                        if (glane == 0) x[k] = xk;
                    }
                    __syncwarp();
                };
                ListSet S0, S1, S2;
                fetch(0, S0);
                fetch(1, S1);
                for (int kk = 0; kk < r; kk += 3) {
                    fetch(kk + 2, S2);
                    coordinate(kk, S0);
                    if (kk + 1 < r) {
                        fetch(kk + 3, S0);
                        coordinate(kk + 1, S1);
                    }
                    if (kk + 2 < r) {
                        fetch(kk + 4, S1);
                        coordinate(kk + 2, S2);
                    }
                }
            }
            if (work) {
                __syncwarp(gmask);
                // ---- Eq. 1's data term at the unit's final x (W half), write back
                if (a.unit_obj) {
                    float t = 0.f;
                    for (int p = glane; p < L; p += G) t += kl_term(vs[p], xs[p], eps_div);
                    double dt = (double)t;
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) dt += __shfl_xor_sync(gmask, dt, o);
                    if (glane == 0) a.unit_obj[u] = dt;
                }
                for (int k = glane; k < r; k += G) {
                    const float xv = x[k];
                    if (!(xv == xv)) atomicOr(a.err, kErrNaN);
                    a.X[u * ldr + k] = xv;
                }
                __syncwarp(gmask);
            }
        }
    }
    if (glane == 0) flush_tally(a, tally);
}

// One warp per row of At: the positive entries in k order (the padding
// columns k >= r hold 0 and never enter), their count, and the row's weight
// times its count added to *dens.
__global__ void __launch_bounds__(256) compress_rows_kernel(const float *At, int64_t rows, int ldr,
                                                            const int64_t *wptr, int32_t *cnt, uint8_t *ck,
                                                            float *ca, unsigned long long *dens) {
    const int lane = threadIdx.x & 31;
    const int nf4 = ldr >> 2;
    unsigned long long mine = 0;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
         row += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const float4 *src = reinterpret_cast<const float4 *>(At + row * ldr);
        uint8_t *dk = ck + row * ldr;
        float *da = ca + row * ldr;
        int base = 0;
        for (int f0 = 0; f0 < nf4; f0 += 32) {
            const int f = f0 + lane;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (f < nf4) v = __ldg(src + f);
            const int c = (v.x > 0.f) + (v.y > 0.f) + (v.z > 0.f) + (v.w > 0.f);
            int incl = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, d);
                if (lane >= d) incl += y;
            }
            int pos = base + incl - c;
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (vv[s] > 0.f) {
                    dk[pos] = (uint8_t)(4 * f + s);
                    da[pos] = vv[s];
                    ++pos;
                }
            }
            base += __shfl_sync(kFull, incl, 31);
        }
        if (lane == 0) {
            cnt[row] = base;
            mine += (unsigned long long)base * (unsigned long long)(wptr[row + 1] - wptr[row]);
        }
    }
    // one atomic per warp
    if (lane == 0 && mine) atomicAdd(dens, mine);
}

const GroupKindInfo kGroupKinds[] = {
    {(const void *)group_kernel<4, 32>, 4, 32, "group_g4_l32"},
    {(const void *)group_kernel<8, 64>, 8, 64, "group_g8_l64"},
    {(const void *)group_kernel<8, 128>, 8, 128, "group_g8_l128"},
    {(const void *)group_kernel<16, 256>, 16, 256, "group_g16_l256"},
};
constexpr int kNumGroupKinds = sizeof(kGroupKinds) / sizeof(kGroupKinds[0]);

}  // namespace

int group_kind_count() { return kNumGroupKinds; }
const GroupKindInfo &group_kind(int kind) { return kGroupKinds[kind]; }

size_t group_unit_smem(int kind, int r, int ldr) {
    const GroupKindInfo &gk = kGroupKinds[kind];
    return group_layout(r, ldr, gk.g, gk.lmax).bytes;
}

size_t group_block_smem(int kind, int r, int ldr, int groups) {
    return align16(4 * (size_t)ldr) + group_unit_smem(kind, r, ldr) * (size_t)groups;
}

int64_t group_slot_floats(int kind, int r) {
    const int64_t lmax = kGroupKinds[kind].lmax;
    const int64_t f = lmax * r + (lmax * r + 3) / 4;  // values, then one byte per position
    return (f + 63) / 64 * 64;
}

int group_kind_for_length(int64_t L) {
    for (int i = 0; i < kNumGroupKinds; ++i)
        if (L <= kGroupKinds[i].lmax) return i;
    return -1;
}

void launch_compress(cudaStream_t st, const float *At, int64_t rows, int ldr, int r, const int64_t *wptr,
                     int32_t *cnt, uint8_t *ck, float *ca, unsigned long long *dens) {
    (void)r;
    if (rows <= 0) return;
    const int64_t blocks = std::min<int64_t>((rows + 7) / 8, 152 * 16);
    compress_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(At, rows, ldr, wptr, cnt, ck, ca, dens);
}

cudaError_t group_attributes(int optin) {
    for (int i = 0; i < kNumGroupKinds; ++i) {
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, kGroupKinds[i].fn);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kGroupKinds[i].fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace nmfkl
