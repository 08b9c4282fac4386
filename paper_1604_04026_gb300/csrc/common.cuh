// Internal declarations shared by the CUDA translation units of libnmfkl.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "nmfkl.h"

namespace nmfkl {

constexpr int kMaxR = 256;
constexpr int kQueuesPerSide = 64;  // work counters per half (one per bucket of both plans)

// Device error flag bits, set by the kernels and read by the host after a half.
constexpr int32_t kErrNaN = 1;      // a factor entry came out NaN
constexpr int32_t kErrTimeout = 2;  // a bounded wait on a cluster peer gave up
constexpr int32_t kErrLength = 4;   // a unit longer than its kernel's capacity was refused
// Default limit of a bounded device wait, in SM clock cycles (~2 s at 2 GHz:
// a wait that long means a peer is gone).
constexpr long long kDefaultWaitCycles = 4000000000ll;

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): per round two 64x64 ->
// 128-bit products of counter words 0 and 2 by fixed multipliers, output
// words (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), key bumped by the Weyl
// constants (golden ratio, sqrt(3)-1); ten rounds.
// ---------------------------------------------------------------------------
constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ULL;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ULL;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ULL;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73BULL;
// Key word 1 tags what the stream is for.
constexpr uint64_t kKeyIds = 0x5352434400000001ULL;   // coordinate orders
constexpr uint64_t kKeyInit = 0x5352434400000002ULL;  // Uniform[0,1) starting factors

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t lo0 = kPhiloxM0 * c[0], hi0 = __umul64hi(kPhiloxM0, c[0]);
        const uint64_t lo1 = kPhiloxM1 * c[2], hi1 = __umul64hi(kPhiloxM1, c[2]);
        const uint64_t n0 = hi1 ^ c[1] ^ k0;
        const uint64_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
}

// Counter of block `blk` of the coordinate order of (sweep, side, unit).
// perm_mode 1 shares one order per sweep (column word 0, side word 2).
__device__ __forceinline__ void ids_counter(uint64_t c[4], uint64_t blk, int64_t unit, int64_t sweep,
                                            int side, int perm_mode) {
    c[0] = blk;
    c[1] = perm_mode == 1 ? 0ull : (uint64_t)unit;
    c[2] = (uint64_t)sweep;
    c[3] = perm_mode == 1 ? 2ull : (uint64_t)side;
}

// ---------------------------------------------------------------------------
// Arguments of one half sweep (Algorithm 1): the units are columns of V (F
// half, CSC, A = W^T) or rows of V (W half, CSR, A = F^T).
// ---------------------------------------------------------------------------
struct HalfArgs {
    const int64_t *ptr;   // unit offsets into idx/val
    const int32_t *idx;   // row of A (= the other factor's row) per nonzero
    const float *val;     // v per nonzero
    const float *At;      // fixed factor, one row of ldr floats per index (W^T or F^T)
    // the fixed factor's rows compressed to their positive entries, in k order
    // (row i: ccnt[i] entries at ck/ca[i * ldr ...]); used by the group kernels
    const int32_t *ccnt;
    const uint8_t *ck;
    const float *ca;
    float *X;             // updated factor, one row of ldr floats per unit (F^T or W^T)
    const float *sumA;    // r sums of the fixed factor's columns over its rows
    int32_t r, ldr;
    float alpha, beta, eps_grad, eps_div, eps_x;
    int32_t max_inner, grad_mode, break_mode, perm_mode;
    int32_t div_mode;  // 0: IEEE division in the Newton step, 1: fast division
    uint64_t seed;
    int64_t sweep;
    const int64_t *sweep_dev;  // if set, the sweep index is read here (a captured step replays with new ones)
    int32_t side;
    // if set, the plan (0: dense tile, 1: lists) the half runs, chosen on the
    // device from the fixed factor's density; a bucket of the other plan
    // (plan_id) returns at once
    const int32_t *plan_sel;
    int32_t plan_id;
    // if u1 > u0, only the units u0 <= u < u1 are updated (a shard of the half)
    int64_t u0, u1;
    // bucket
    const int32_t *units;  // unit ids of this bucket, longest first
    int32_t count;
    int32_t *queue;        // work counter, zero at launch
    float *scratch;        // per-group slots of slot_floats floats
    int64_t slot_floats;
    int32_t lcap;          // tile row length (max nonzeros of a unit in this bucket)
    unsigned long long *counters;  // coords, evals, steps, cap_hits
    int32_t *err;          // device error flag (kErr* bits)
    long long wait_cycles; // limit of each bounded wait on a cluster peer
    double *unit_obj;      // if set: per unit, sum over its nonzeros of v log(v/(x+eps)) - v
                           // at the unit's final x (Eq. 1's data term, fused into the W half)
    const int32_t *count_dev;  // if set, the bucket's unit count is read here (device-built buckets)
    const int64_t *unit_ids;   // if set, the unit id that keys the coordinate order (else the unit index)
    // fold-in (F half alone under a fixed W, every column to its own stopping point)
    int32_t max_sweeps;
    double rel_tol;
    const double *sumA64;  // FP64 column sums of the fixed factor (the objective's linear term)
    int32_t *sweeps_done;  // per unit
    double *unit_final;    // per unit: the column objective at the returned x
};

// One launch configuration of the sweep kernel family.
struct Bucket {
    // floats from the scratch base to this bucket's slots: every bucket of a
    // plan has slots of its own, since consecutive buckets may run at once
    int64_t scratch_off = 0;
    bool sparse = false;  // kernel table: the sparse-list kinds (else the dense-tile kinds)
    bool group = false;   // kernel table: the sub-warp group kinds (lists of compressed rows)
    int kind;         // index into the kernel table
    int nt;           // threads per subproblem group (32 = one warp)
    int k;            // nonzeros per thread held in registers (0 = giant)
    int cl;           // CTAs per cluster (1 = no cluster)
    int32_t count;    // units in the bucket
    int32_t lcap;     // tile row length
    int32_t *d_units; // device list of unit ids
    int grid;         // persistent blocks
    int block;        // threads per block
    size_t smem;      // dynamic shared memory per block
    int groups;       // subproblem groups in the grid
    int64_t slot_floats;
    int64_t max_len;
    int64_t nnz;      // nonzeros of the bucket's units
    bool borrowed = false;  // a dense bucket reused by the list plan (d_units owned by the dense plan)
    // list plan, units of at most 256 nonzeros: the length class (0..3 for at
    // most 32, 64, 128, 256) that this bucket is one alternative for (the
    // dense-tile warp kernel or the group kernel; the context's choice picks
    // one per class); -1 for every other bucket
    int short_class = -1;
};

// Device state of fold-in (nmfkl_foldin): input copies, per-length-class
// unit lists built on the device, tiles, and the captured launch graph.
constexpr int kFoldKinds = 9;
struct FoldState {
    int64_t cap_m = 0, cap_nnz = 0;
    int64_t *colptr = nullptr, *ids = nullptr;
    int32_t *rowidx = nullptr;
    float *val = nullptr;
    float *Ft = nullptr;       // cap_m x ldr, unit-major
    float *Fout = nullptr;     // r x cap_m, row-major
    int32_t *lists = nullptr;  // kFoldKinds x cap_m
    int32_t *ctl = nullptr;    // [counts kFoldKinds][queues kFoldKinds][err]
    int32_t *sweeps = nullptr;
    double *obj = nullptr;
    float *scratch = nullptr;
    int64_t scratch_floats = 0;
    bool planned = false;
    int grid[kFoldKinds] = {}, block[kFoldKinds] = {}, groups[kFoldKinds] = {};
    size_t smem[kFoldKinds] = {};
    int64_t slot_floats[kFoldKinds] = {};
    int32_t lcap[kFoldKinds] = {};
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_m = -1;
    bool graph_ids = false;
    double graph_tol = -1.0;
    int32_t graph_sweeps = -1;
};

struct KernelTimer {
    const char *name;  // string literal
    int64_t launches = 0;
    double ms = 0.0;
};

}  // namespace nmfkl

struct nmfkl_ctx {
    nmfkl_params p;
    int64_t n = 0, m = 0, nnz = 0;
    int32_t ldr = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::string err;
    bool have_data = false;
    // V
    int64_t *colptr = nullptr, *rowptr = nullptr;
    int32_t *rowidx = nullptr, *colidx = nullptr;
    float *val = nullptr, *rval = nullptr;
    // factors, unit-major with row stride ldr: Wt (n x ldr), Ft (m x ldr)
    float *Wt = nullptr, *Ft = nullptr;
    float *sumW = nullptr, *sumF = nullptr;
    double *dsum[2] = {nullptr, nullptr};  // FP64 sumW (0) and sumF (1) of the last colsum
    double *unit_obj = nullptr;            // n per-row data terms of the fused objective
    double *dpart = nullptr;       // reduction partials
    int64_t dpart_len = 0;
    double *dscalar = nullptr;     // small FP64 results
    unsigned long long *counters = nullptr;
    int32_t *queues = nullptr;     // one per bucket per side (kQueuesPerSide each)
    int32_t *err_flag = nullptr;
    long long wait_cycles = nmfkl::kDefaultWaitCycles;  // bounded device waits
    float *scratch = nullptr;
    int64_t scratch_floats = 0;
    float *tbuf = nullptr;         // transpose staging for get/set
    int64_t tbuf_floats = 0;
    std::vector<nmfkl::Bucket> plan[2];         // dense-tile kernels
    std::vector<nmfkl::Bucket> plan_sparse[2];  // sparse-list kernels
    unsigned long long *dens = nullptr;         // density numerators of the two halves
    // device control of a half: [0..1] the plan chosen per half, [2..3] unused,
    // then two doubles per half (density) and the sweep index (int64)
    int32_t *plan_sel = nullptr;
    double *dens_out = nullptr;
    int64_t *sweep_dev = nullptr;
    int64_t *h_sweep = nullptr;                 // pinned host copy of the sweep index
    double list_threshold = 0.5;                // density below which a half runs the list plan
    // the step (both halves and the objective) captured as one CUDA graph
    cudaGraphExec_t step_graph = nullptr;
    cudaStream_t cap_stream = nullptr;
    // the fixed factor of the current half compressed to its positive entries
    // (rows x ldr, rows = max(n, m)); rebuilt at the start of every half
    int32_t *crow_cnt = nullptr;
    uint8_t *crow_k = nullptr;
    float *crow_a = nullptr;
    double density[2] = {-1.0, -1.0};           // last measured density per half
    int used_sparse[2] = {-1, -1};              // which plan the last half ran
    // list plan: per half and short length class, 0 = dense-tile warp kernel,
    // 1 = group kernel over the compressed rows (set by nmfkl_set_plan_choice
    // or nmfkl_autotune)
    int8_t short_choice[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    // plans with cluster buckets launch longest first, each bucket allowed to
    // overlap the previous one's tail (set per half and plan at planning)
    bool pdl = true;
    bool overlap[2][2] = {{false, false}, {false, false}};
    nmfkl::FoldState *fold = nullptr;
    // timing
    bool timing = false;
    std::vector<nmfkl::KernelTimer> timers;
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { int timer; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    // per-step metrics (nmfkl_set_metrics): the file, the events around a
    // step, zero counts of W and F (device), the work counters at the last line
    std::FILE *metrics = nullptr;
    cudaEvent_t mev[2] = {nullptr, nullptr};
    unsigned long long *zeros_dev = nullptr;
    unsigned long long mprev[4] = {0, 0, 0, 0};
};

namespace nmfkl {

// Error helpers (host).
bool cuda_ok(nmfkl_ctx *c, cudaError_t e, const char *what);

// A named NVTX range over a host-side phase (a step, a half, fold-in, a
// serving batch): profilers show it as a span; without one attached the
// push and pop cost a few nanoseconds.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// trace.cu: one metrics line after a step whose work lies between c->mev[0]
// and c->mev[1] (no-op without a metrics file); freeing its state.
nmfkl_status write_metrics(nmfkl_ctx *c, int64_t sweep, double kl);
void free_metrics(nmfkl_ctx *c);

// Timing hooks around every kernel launch.
int timer_begin(nmfkl_ctx *c, const char *name);
void timer_end(nmfkl_ctx *c, int token);

// group.cu: sub-warp group kernels over lists of compressed factor rows
struct GroupKindInfo {
    const void *fn;
    int g;           // lanes per unit
    int lmax;        // longest unit (nonzeros)
    const char *name;
};
int group_kind_count();
const GroupKindInfo &group_kind(int kind);
// Dynamic shared memory of one group and its global scratch slot (floats).
size_t group_unit_smem(int kind, int r, int ldr);
size_t group_block_smem(int kind, int r, int ldr, int groups);
int64_t group_slot_floats(int kind, int r);
// The default group kind for units of at most L nonzeros (L <= 256), or -1.
int group_kind_for_length(int64_t L);
// Compresses the rows of At (rows x ldr) to their positive entries and adds
// sum_i (wptr[i+1] - wptr[i]) * count_i to *dens (zeroed by the caller).
void launch_compress(cudaStream_t st, const float *At, int64_t rows, int ldr, int r, const int64_t *wptr,
                     int32_t *cnt, uint8_t *ck, float *ca, unsigned long long *dens);
cudaError_t group_attributes(int optin);

// sweep.cu
// Gives every kernel the device's opt-in dynamic shared memory limit (once per
// device; the limit is process-wide per-function state).
cudaError_t kernel_attributes(int device);
nmfkl_status plan_side(nmfkl_ctx *c, int side);
nmfkl_status run_half(nmfkl_ctx *c, int side, int64_t sweep, const int64_t *sweep_dev = nullptr, int64_t u0 = 0,
                      int64_t u1 = 0);
void free_plan(nmfkl_ctx *c);
const char *kind_name(int kind);
const char *bucket_name(const Bucket &b);
// Kernel timer name of a bucket: "<kernel>/F" or "<kernel>/W" (static storage).
const char *bucket_timer_name(const Bucket &b, int side);
// The kernel (0 dense tile, 1 group) that runs short length class `cls` of
// the list plan of `side`: the context's choice, if the plan holds it.
int short_kernel(const nmfkl_ctx *c, int side, int cls);

// aux.cu
nmfkl_status launch_colsum(nmfkl_ctx *c, const float *At, int64_t rows, float *out, double *out_d);
nmfkl_status launch_fused_objective(nmfkl_ctx *c, double *kl);
// FP64 sum of x[0..n) into *out (device), one block, fixed order.
nmfkl_status launch_range_sum(nmfkl_ctx *c, const double *x, int64_t n, double *out);
// The fused objective's kernels alone (capturable); the value lands in c->dscalar[0].
nmfkl_status enqueue_fused_objective(nmfkl_ctx *c);
// colsum into caller buffers: part holds 1024 x ldr doubles.
void launch_colsum_raw(cudaStream_t stream, const float *At, int64_t rows, int ldr, int r, double *part,
                       float *out, double *out_d);
nmfkl_status launch_objective(nmfkl_ctx *c, double *kl, double *reg);
nmfkl_status launch_uniform_init(nmfkl_ctx *c, int which, float *X, int64_t cols);
nmfkl_status launch_to_unit_major(nmfkl_ctx *c, const float *src, float *dst, int64_t cols);
nmfkl_status launch_from_unit_major(nmfkl_ctx *c, const float *src, float *dst, int64_t cols);
void uniform_init_raw(cudaStream_t st, float *X, int r, int64_t cols, int ldr, uint64_t seed, int which);
void launch_from_unit_major_raw(cudaStream_t st, const float *src, float *dst, int r, int64_t cols, int ldr);
nmfkl_status launch_debug_perm(nmfkl_ctx *c, int64_t sweep, int side, int64_t count,
                               const int64_t *cols, int32_t *out);
int64_t dpart_required(int ldr);
// sweep.cu: fold-in
nmfkl_status foldin_run(nmfkl_ctx *c, int64_t m_new, bool with_ids, double rel_tol, int32_t max_sweeps,
                        bool use_graph);
nmfkl_status foldin_per_doc(nmfkl_ctx *c, int64_t m_new, double rel_tol, int32_t max_sweeps);
// api.cu: fold-in with the starting F given per segment of columns (serving)
struct FoldSegment {
    int64_t col0, m;
    const float *F0;  // host r x m row-major, or NULL: Uniform[0,1) drawn for the segment alone
};
nmfkl_status foldin_impl(nmfkl_ctx *c, int64_t m_new, int64_t nnz, const int64_t *colptr, const int32_t *rowidx,
                         const float *val, const int64_t *doc_ids, const float *F0,
                         const std::vector<FoldSegment> *segs, float *F_out, double rel_tol, int32_t max_sweeps,
                         int32_t *sweeps_done, double *doc_obj, int32_t launch_mode, int32_t mem_kind);
int foldin_kind_for_length(int64_t L);
void free_fold(nmfkl_ctx *c);
// Sum over the rows i of At of weight_i * #{k < r : At[i][k] > 0}, weight_i =
// ptr[i+1] - ptr[i], into *out (zeroed by the caller).
void launch_density(cudaStream_t st, const float *At, int64_t rows, int ldr, int r, const int64_t *ptr,
                    unsigned long long *out);
nmfkl_status launch_validate(nmfkl_ctx *c, int64_t units, int64_t extent, int64_t nnz, const int64_t *ptr,
                             const int32_t *idx, const float *val, int32_t *flag);

}  // namespace nmfkl
