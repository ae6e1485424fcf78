// bc_internal.cuh -- device-side types, exact integer helpers and the launch
// functions shared by the translation units of libbcgpu.so.
//
// State layout (row-major n x n, structure of arrays; Section 5 stores the triple
// (d, sigma, flag) per pair in one row-major array -- here each field is its own
// array so a pass reads only the fields it needs):
//   D   [n*n]  distance type DT (int32 or int64), INF = DT max
//   S   [n*n]  uint64 path counts sigma_st
//   Dl  [n*n]  dependencies delta_s.(t) as float-float pairs (ff.cuh), 0 on the diagonal
//   BC  [n]    fp64 pair (hi, lo): compensated running sums of the G_D scores
// E* superset ("E*+") -- every arc that lies on some shortest path, plus arcs that
// may no longer do so (Section 6: any superset of E* gives the right DAGs) -- is a
// CSR with per-vertex slack: arcs of vertex a sit in slots [off[a], off[a]+len[a]),
// followed by free slots (dst = -1).  A segment that fills up moves to the free region
// past the laid-out ones (off[a] changes, its old slots are emptied).  Each slot is a
// packed (dst, w) pair (Arc<DT>: 8 bytes for int32 distances, 16 for int64) so one load
// brings both; src[] repeats the tail of each slot for passes that run over the slots.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ff.cuh"

namespace bcg {

enum : int32_t { ERRF_OVERFLOW = 1, ERRF_DIST = 2, ERRF_TIMEOUT = 4, ERRF_ARG_DEVICE = 8 };

// Per-handle device counters: [0] rows re-accumulated [1] no-op updates [2] most rows of
// one update [3] updates [4] pairs lowered [5] pairs with new tied paths [6] rows scanned
// [7] rows re-accumulated in full [8] rows corrected pair by pair [9] (row, target) pairs
// of those corrections [10] pairs corrected by DAG walks [11] vertices those walks found
// [12] E* arcs they examined.
constexpr int kStats = 13;

// Saturation marker for a distance sum that does not fit: INT64_MAX.  For DT =
// int64 this equals INF, so callers test for it before comparing.
constexpr int64_t SAT = INT64_MAX;

template <typename DT> struct Inf;
template <> struct Inf<int32_t> { static constexpr int64_t v = INT32_MAX; };
template <> struct Inf<int64_t> { static constexpr int64_t v = INT64_MAX; };

// a + b for finite non-negative a, b; SAT when the sum is not a finite DT value.
template <typename DT>
__device__ __forceinline__ int64_t dsum(int64_t a, int64_t b) {
    if constexpr (sizeof(DT) == 4) {
        int64_t s = a + b;
        return s >= Inf<int32_t>::v ? SAT : s;
    } else {
        return (b > INT64_MAX - 1 - a) ? SAT : a + b;
    }
}

__device__ __forceinline__ void set_err(int32_t* err, int32_t f) { atomicOr(err, f); }

// Block-uniform read of the sticky error word: other CTAs of the same launch may set it
// at any time, so kernels that use barriers take one decision for the whole CTA.
// Every thread of the block must call it.
__device__ __forceinline__ bool block_err(const int32_t* err) {
    __shared__ int32_t s_err;
    __syncthreads();
    if (threadIdx.x == 0) s_err = *reinterpret_cast<const volatile int32_t*>(err);
    __syncthreads();
    return s_err != 0;
}

// 64 x 64 -> 64 product of path counts; flags overflow when the high word is used.
__device__ __forceinline__ uint64_t mul_chk(uint64_t a, uint64_t b, int32_t* err) {
    if (__umul64hi(a, b) != 0ull) set_err(err, ERRF_OVERFLOW);
    return a * b;
}

__device__ __forceinline__ uint64_t add_chk(uint64_t a, uint64_t b, int32_t* err) {
    uint64_t s = a + b;
    if (s < a) set_err(err, ERRF_OVERFLOW);
    return s;
}

template <typename DT> struct Arc;
template <> struct __align__(8) Arc<int32_t> { int32_t dst; int32_t w; };
template <> struct __align__(16) Arc<int64_t> { int64_t dst; int64_t w; };

constexpr int kPairCap = 128;   // changed targets of a row corrected pair by pair (k_pair.cu)

// The edges of one update as the DAG walks of the pair corrections need them: the
// updated vertex v, the other endpoints x_j and the weight of {v, x_j} before the
// update (-1: the edge is new).  Updates with more edges use the column test.
constexpr int kWalkMaxEdges = 32;
struct WalkUpd {
    int32_t v;
    int32_t k;
    int32_t x[kWalkMaxEdges];
    int64_t wold[kWalkMaxEdges];
};
constexpr int kWalkThreads = 256;
constexpr int kWalkCtasPerSm = 8;      // walks: latency-bound, 32 registers, a few KB of shared memory
constexpr int kWalkRowCtasPerSm = 8;
constexpr size_t kWalkSmemMax = 200 * 1024;
constexpr int kWalkBlock = 2048;     // walk buffer entries a warp reserves at a time
constexpr int kWalkDefaultMinN = 12288;   // undirected graphs with at least this many vertices walk by default

// One edge of a vertex update, as staged on the device (matches bc_vedge).
struct VEdge {
    int32_t x;
    int32_t dir;
    int64_t w;
};

// One write into the E*+ CSR (slot < 0: only the length of vertex a changes).
struct EOp {
    int32_t slot;
    int32_t a;
    int32_t b;
    int32_t len_a;
    int64_t w;
};
constexpr int kMaxEOps = 64;
struct EOps {
    int32_t count;
    int32_t pad;
    EOp op[kMaxEOps];
};
// Move of the E* segment of vertex a (len arcs) from slot from to slot to, in the free
// region past the laid-out segments.
struct EMove {
    int32_t a;
    int32_t from;
    int32_t to;
    int32_t len;
};
constexpr int kMaxEMoves = 32;
struct EMoves {
    int32_t count;
    int32_t pad;
    EMove mv[kMaxEMoves];
};

// Device state of one handle (plain pointers; owned by the host-side bc_graph).
struct Dev {
    int32_t n;
    int32_t dbytes;      // 4 or 8
    int32_t directed;
    int32_t nsm;
    void* D;
    uint64_t* S;
    ff* Dl;
    double* bc_hi;
    double* bc_lo;
    // full graph (G or G_D) CSR, used by the static computation
    int32_t* g_off;
    int32_t* g_src;
    int32_t* g_dst;
    void* g_w;
    int32_t* p_dst;      // static search: working copy of g_dst pruned to E* (NULL: no pruning)
    int32_t* s_order;    // static search: sources in order (NULL: 0 .. n-1)
    int64_t g_arcs;
    // E*+ CSR with slack
    int32_t* e_off;
    int32_t* e_len;
    int32_t* e_src;
    void* e_arc;         // Arc<DT>[e_cap]
    int64_t e_cap;
    // error word, counters
    int32_t* err;
    int64_t* stats;      // [0] rows re-accumulated [1] no-op updates [2] max rows [3] updates
                         // [4] pairs lowered [5] pairs with new ties [6] rows scanned
    // scratch
    uint8_t* mark;       // [n] rows that change in the current phase
    uint8_t* changed;    // [n] rows that changed in any phase of the current update
    int32_t* rows;       // [n] compacted rows of the current phase
    int32_t* acc_rows;   // [n] compacted rows to re-accumulate
    int32_t* counts;     // [0] phase rows [1] accumulation rows [3] full rows [4] pair pieces handed
                         // out [5] rows corrected pair by pair
    void* fD;            // [n] per-row distance to v after the phase (DT)
    uint64_t* fS;        // [n] per-row path count to v after the phase
    uint64_t* fM;        // [n] per-row multiplier of a tie
    void* cD;            // [n] per-column distances from v (DT)
    uint64_t* cS;        // [n] per-column path counts from v
    uint64_t* cM;        // [n] per-column multiplier of a tie
    void* cD2;           // [n] second column vector (fused undirected edge pass): distances (DT)
    uint64_t* cS2;       // [n] its path counts
    ff* partial;         // [nrb * n] column partial sums
    int32_t nrb_max;     // row blocks of the BC reduction
    int32_t acc_grid;    // CTAs of the accumulation kernel
    int32_t acc_smem;    // dynamic shared memory of the accumulation kernel
    int32_t acc_mask_smem;  // 1: the DAG slot mask lives in shared memory
    int32_t acc_threads;    // kAccThreadsWide: wide CTAs allowed for partial waves of sources
    int32_t acc_narrow_only;  // 1: never the wide CTAs (kept across launch-shape updates)
    int32_t acc_grid_wide;  // CTAs of the wide accumulation kernel (acc_grid: of the narrow one)
    int32_t* ws;         // accumulation work space, acc_grid * ws_stride ints
    int64_t ws_stride;
    // pair-dependency corrections (undirected graphs): the pairs changed by this update,
    // their values before it, and the changed targets of each row
    int32_t pair_on;
    int32_t tcap;        // targets recorded per row (kPairCap); more -> full re-accumulation
    uint32_t* chg;       // [n * chg_words] bit (s,t): pair changed in this update
    int32_t chg_words;   // (n + 31) / 32
    void* oldD;          // [n*n] d(s,t) before the update, valid where the bit is set (DT)
    uint64_t* oldS;      // [n*n] sigma_st before the update, likewise
    int32_t* tcnt;       // [n] changed targets of the row
    int32_t* tlist;      // [n * tcap]
    void* plan;          // [n * tcap] per-target scalars of the pair corrections (k_pair.cu)
    int64_t* pair_w;     // [n + 1] prefix of the pair corrections' work item weights
    int32_t* full_rows;  // [n] rows re-accumulated in full (counts[3])
    int32_t* pair_rows;  // [n] rows corrected pair by pair, most targets first (counts[5])
    int32_t pair_walk;   // 1: pair corrections by DAG walks (k_walk_units, k_walk_rows), scratch below
    int32_t* walk_list;      // [walk warps * n] per-warp vertex lists of a walk
    int32_t* walk_buf;       // [walk_cap] vertices found by the walks of an update
    int64_t walk_cap;
    int32_t* walk_useg;      // [n * tcap * 4] per (row, target): segments of the old and new walk
    int64_t* walk_acc2;      // [walk CTAs * 2n] per-CTA fixed-point column sums of a row (zero between rows)
    int32_t* walk_tl;        // [walk CTAs * n] per-CTA touched columns of a row
    int32_t* walk_ctl;       // [8] units and rows handed out, buffer used (64-bit), overflow
    int32_t* walk_rowE;      // [n] per listed row: vertices found by its walks
    int64_t* bcfix;      // [2n] BC change of the corrected rows in this update, per column a
                         // fixed-point pair (units of 2^-24, units of 2^-56); zero between updates
    cudaStream_t st;
    // a third stream for the heaviest rows of the DAG walks' phase 2 (undirected graphs):
    // forked from st after the walks, joined back before the BC fix-up
    cudaStream_t st3;
    cudaEvent_t ev3_fork, ev3_join;
};

constexpr int kRowsPerBlock = 64;   // rows per partial sum of the BC reduction
// Threads of an accumulation CTA (one source at a time): 1024 for the few rows over the
// target cap of an update on graphs of at least kAccWideMinN vertices (the level passes
// of one source spread over more threads), 256 otherwise (four sources in flight per SM:
// saturated serving of 64 graphs 1783 -> 2028 updates/s against 512 threads, 128 threads
// 1843); the batched path picks 128, 256 or 512 by autotuning.
constexpr int kAccThreadsWide = 1024;
constexpr int kAccThreadsNarrow = 256;
constexpr int kAccWideMinN = 4096;

// Accumulation launch shape for n and the current E* capacity (sets acc_grid, acc_smem,
// acc_mask_smem and ws_stride of d); the work space must then hold acc_grid * ws_stride.
void accum_config(Dev& d);

// Recording of changed pairs by the passes that write D and sigma (pair corrections).
struct PairRec {
    uint32_t* chg;
    int32_t chg_words;
    void* oldD;
    uint64_t* oldS;
    int32_t* tcnt;       // NULL: nothing is recorded
    int32_t* tlist;
    int32_t tcap;
    int32_t first;       // no pair has changed yet in this update (the IN phase; row v)
};

// The recording buffers of a handle with pair corrections.
__host__ __device__ inline PairRec make_pair_rec(const Dev& d) {
    PairRec r;
    r.chg = d.chg;
    r.chg_words = d.chg_words;
    r.oldD = d.oldD;
    r.oldS = d.oldS;
    r.tcnt = d.tcnt;
    r.tlist = d.tlist;
    r.tcap = d.tcap;
    r.first = 0;
    return r;
}

// Columns per thread of the pair-correction column test for n vertices: 16-byte (or two
// 16-byte) loads where every row starts on a 16-byte boundary.
constexpr int kPairVec32 = 8;   // columns per thread with int32 distances (4 or 8)
__host__ __device__ inline int pair_vn(int dbytes, int n) {
    if (dbytes == 4) return (kPairVec32 == 8 && n % 8 == 0) ? 8 : (n % 4 == 0 ? 4 : 1);
    return n % 2 == 0 ? 2 : 1;
}

// The first change of pair (s,t) in an update sets its bit, saves its old distance and
// path count, and lists t as a changed target of row s (targets beyond the capacity
// are only counted).  Later changes of the same pair (the OUT phase after the IN
// phase) keep the saved values.  Each pair is written by one thread per pass, and a
// bit set by an earlier pass is visible, so a plain read of the word decides; the bit
// is then set without waiting for the old word.
template <typename DT>
__device__ __forceinline__ void record_change(const PairRec& r, int n, int s, int t, int64_t d_old,
                                              uint64_t sig_old) {
    const uint32_t bit = 1u << (t & 31);
    uint32_t* w = r.chg + (size_t)s * r.chg_words + (t >> 5);
    if (!r.first && (*w & bit)) return;
    atomicOr(w, bit);
    const size_t i = (size_t)s * n + t;
    static_cast<DT*>(r.oldD)[i] = (DT)d_old;
    r.oldS[i] = sig_old;
    const int pos = atomicAdd(r.tcnt + s, 1);
    if (pos < r.tcap) r.tlist[(size_t)s * r.tcap + pos] = t;
}

// ---- programmatic dependent launch ----
// The kernels of an update run one after another on the handle's stream.  They are
// launched with programmatic stream serialization allowed, so the launch of the next
// kernel is processed while this one runs, and each one starts with pdl_enter(): a wait
// for the previous kernel's completion and memory before touching any data.  No kernel
// triggers its dependents early: the next kernel's CTAs are placed only as this grid's
// CTAs exit (an early trigger let every later kernel's CTAs occupy SMs while waiting,
// which slowed the running kernel).  Launched the ordinary way, or after a non-kernel
// operation, the wait has no effect.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---- launches (k_update.cu) ----
cudaError_t scan_setup();
void launch_estar_write(const Dev& d, const EOps& ops);
void launch_estar_move(const Dev& d, const EMoves& moves);
void launch_alg4_in(const Dev& d, int32_t v, const VEdge* e, int32_t k);
void launch_rows_out(const Dev& d, int32_t v, const VEdge* e, int32_t k);
void launch_alg4_out(const Dev& d, int32_t v, const VEdge* e, int32_t k);
void launch_compact(const Dev& d, const uint8_t* mark, int clear, int32_t* rows,
                    int32_t* count, int full, int stats);
void launch_scan_in(const Dev& d, int32_t v);
void launch_scan_out(const Dev& d, int32_t v);
void launch_write_row(const Dev& d, int32_t v);
void launch_edge_prep(const Dev& d, int32_t u, int32_t v, int64_t w);
void launch_edge_scan(const Dev& d);
void launch_estar_keep(const Dev& d, uint8_t* keep);
PairRec pair_rec(const Dev& d);
void launch_pair_lists(const Dev& d);
void launch_pairdep(const Dev& d, const WalkUpd* upd);   // upd: DAG walks (k_pairwalk), else column tests
size_t walk_smem(int n);
int64_t walk_warps(int nsm);
int64_t walk_ctas(int nsm);
// Kernel attributes of the pair corrections (the walks' and the weights pass's dynamic
// shared memory limits); bc_init_static sets them before it builds a handle.
cudaError_t walk_setup();
void launch_pair_clear(const Dev& d);
void launch_bc_fix(const Dev& d);

// ---- launches (k_accum.cu) ----
void launch_accum(const Dev& d, int is_static);
void launch_accum_rows(const Dev& d, const int32_t* rows, const int32_t* count);
void launch_bc_rows(const Dev& d, int sign, int is_static);
void launch_bc_rows_list(const Dev& d, int sign, const int32_t* rows, const int32_t* count);

// ---- launches (k_static.cu) ----
void launch_sssp(const Dev& d);
void launch_estar_flags(const Dev& d, uint8_t* flags);

}  // namespace bcg
