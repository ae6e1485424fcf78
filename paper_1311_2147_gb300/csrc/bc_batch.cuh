// bc_batch.cuh -- device-side records of a batch of graphs (k_batch.cu) and the launch
// entry points the host side of the batch calls.
#pragma once

#include "bc_internal.cuh"

namespace bcg {

// The r-th update of graph g (rounds x graphs, row-major by round).
struct BatchUpd {
    int32_t v;        // the updated vertex (an edge update (u, v) is one in-edge of v)
    int32_t k;        // its edges, entries[first .. first + k)
    int32_t kin;      // edges into v (IN phase), edges out of v (OUT phase)
    int32_t kout;
    int32_t present;  // 0: graph g has no r-th update
    int32_t pad;
    int64_t first;
};

struct BatchEOp {
    int32_t g;
    int32_t pad;
    EOp op;
};

struct BatchArgs {
    int32_t G;
    int32_t mask_in_smem;
    int32_t n_max;            // largest n of the batch
    const Dev* devs;          // [G]
    const BatchUpd* upd;      // [rounds * G]
    const VEdge* entries;
    const BatchEOp* eops;
    const int64_t* eop_off;   // [rounds + 1]
    const int64_t* voff;      // [rounds * 4 * (G + 1)]: per-vertex pass offsets
    const int64_t* coff;      // [G + 1]: column offsets (prefix of n_g)
    int64_t* plan_scan;       // [G + 1]
    int64_t* plan_bc;         // [G + 1]
    int64_t* plan_acc;        // [G + 1]
    int64_t* plan_pr;         // [G + 1]: rows listed for pair corrections (graphs with them)
    int64_t* plan_pw;         // [kPairClasses * (G + 1)]: column-test work per class of columns per thread
    int32_t* pctr;            // [kPairClasses]: column-test pieces handed out past the first wave
    int32_t* ws;              // accumulation work space, acc_grid * ws_stride ints
    int64_t ws_stride;
};

// Classes of the column test's columns per thread (pair_vn): int32 distances 8, 4, 1;
// int64 distances 2, 1.
constexpr int kPairClasses = 3;
__host__ __device__ inline int pair_class(int dbytes, int vn) {
    if (dbytes == 4) return vn == 8 ? 0 : (vn == 4 ? 1 : 2);
    return vn == 2 ? 0 : 1;
}

// Launch shape of a batch; the tunable part is what the autotuner varies.
struct BatchLaunch {
    int32_t nsm;
    int32_t vpass_ctas;   // CTAs per SM of the per-vertex passes      (tunable)
    int32_t scan_ctas;    // CTAs per SM of the rank-1 pass             (tunable)
    int32_t bc_ctas;      // CTAs per SM of the BC row sums             (tunable)
    int32_t acc_per_sm;   // cap on accumulation CTAs per SM, 0 = max   (tunable)
    int32_t scan_unroll;  // 16-byte vectors per thread per rank-1 item: the item's column
                          // chunk is 256 threads x this x the vector width (1, 2, 4, 8; tunable)
    int32_t scan_sched;   // 0: a contiguous block of items per CTA; 1: items dealt out in
                          // turn (item = CTA + k * grid)                (tunable)
    int32_t acc_threads;  // threads of an accumulation CTA: 512, 256 or 128 (more sources
                          // in flight per SM)                           (tunable)
    int32_t pair_classes; // bit c: some graph of the batch has pair corrections with columns
                          // per thread of class c (0: none; the round skips the pair kernels)
    int32_t acc_grid;
    int32_t acc_smem;
    int32_t mask_in_smem;
    int64_t ws_stride;
    int64_t max_eops;
};

// Graph g of task j: last g with off[g] <= j (off non-decreasing, off[0] = 0).
__device__ __forceinline__ int graph_of(const int64_t* off, int G, int64_t j) {
    int lo = 0, hi = G;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The rows a round re-accumulates by Algorithm 1 in graph d: with pair corrections the
// rows over the target cap, else every changed row.
__device__ __forceinline__ const int32_t* acc_list(const Dev& d) { return d.pair_on ? d.full_rows : d.acc_rows; }
__device__ __forceinline__ int32_t acc_list_count(const Dev& d) { return d.pair_on ? d.counts[3] : d.counts[1]; }

void batch_config(BatchLaunch& L, int dbytes, int n_max, int64_t cap_max);
void batch_launch_rounds(const BatchArgs& b, const BatchLaunch& L, int rounds, int dbytes, cudaStream_t st);
// Prefix offsets over graphs of one kind of per-graph work (kb_plan), and the pair
// corrections of round r (k_pair.cu).
void batch_plan(const BatchArgs& b, int r, int kind, int phase_active, int64_t* out, int scan_unroll,
                cudaStream_t st);
void batch_pair_lists(const BatchArgs& b, const BatchLaunch& L, int r, cudaStream_t st);
void batch_pair_launches(const BatchArgs& b, const BatchLaunch& L, int r, int dbytes, cudaStream_t st);

}  // namespace bcg
