// k_accum.cu -- dependency accumulation and the BC reduction.
//
// For each source s whose row changed (and, in the static computation, for every s):
//   * DAG'(s) is rebuilt implicitly: an arc (a,b) of the E* superset is in DAG'(s)
//     iff d'(s,a) is finite and d'(s,a) + w(a,b) = d'(s,b) (Eq. 1; Algorithm 6 step 4
//     applied to E'; Section 6 notes any superset of E* gives the same DAGs).
//   * A topological order of DAG'(s) is built level by level (Kahn): in-degrees are
//     counted first, then a vertex joins level L+1 when its last in-arc from level L
//     is consumed.  Section 2 notes that any reverse topological order serves
//     Algorithm 1 as well as the order by distance; level order keeps the sequential
//     chain as short as the DAG is deep.  In the static computation the same sweep
//     carries the path counts forward (sigma_sb = sum of sigma_sa over DAG in-arcs,
//     Algorithm 6 step 7).
//   * delta_s. is pulled in reverse level order (Eq. 4), in float-float (ff.cuh):
//         delta(a) = sum over DAG out-arcs (a,b) of sigma_sa / sigma_sb * (1 + delta(b))
//                  = sigma_sa * sum over the same arcs of rho(b),
//     with rho(b) = (1 + delta(b)) / sigma_sb kept per vertex.  The DAG out-arcs of a
//     level are flattened over the CTA (a block scan of the per-vertex arc counts, each
//     thread fetching rho of one arc, each vertex summing its own arcs in slot order);
//     vertices with more than kBigDag DAG out-arcs are summed by a warp over a fixed
//     stride and butterfly.  Either way the result does not depend on scheduling.
// The kernel stages in shared memory the source's distance row (16-bit when every
// finite distance of the row is below 65535, otherwise read from its row of D), the
// packed 16-bit Kahn counters, the 16-bit level order and a bit mask over the slots of
// the E* superset marking the arcs of DAG'(s): about 4n bytes plus one bit per slot,
// two CTAs per SM at n = 16384.  rho and the level bounds live in a per-CTA work space
// in global memory (L2-resident), and so does the slot mask when it is too large.
//
// BC is maintained as BC += sum over changed rows of (delta'_s - delta_s): the old rows
// are subtracted before the rows are rewritten and the new rows added after
// (Algorithm 3 step 1 recomputes BC from zero; rows that did not change contribute
// the same amount before and after, so only changed rows are touched).  Column sums
// run over row blocks in a fixed order into a compensated (hi, lo) pair.
#include "bc_device.cuh"

namespace bcg {

// One CTA per source at a time (shared memory as described at AccSmem; the per-round
// scratch of the level passes is static shared memory).
template <typename DT, bool STATIC, int T>
__global__ void __launch_bounds__(T, 1024 / T) k_accum_smem(AccArgs<DT> a) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LevelSmem<T> ls;
    __shared__ int s_tail, s_nbig;
    const AccSmem m = acc_smem(a, smem, a.ws + (size_t)blockIdx.x * a.ws_stride);
    const int total = STATIC ? a.n : *a.count;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        if (block_err(a.err)) return;
        dev_accum_source<DT, STATIC, T>(a, STATIC ? i : a.rows[i], m, ls, &s_tail, &s_nbig);
    }
}

__global__ void k_bc_partial(int n, const int32_t* rows, const int32_t* count, const ff* Dl,
                             ff* partial, const int32_t* err) {
    pdl_enter();
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = rows ? *count : n;
    for (int rb = blockIdx.y; rb * kRowsPerBlock < total; rb += gridDim.y)
        dev_bc_partial(t, rb, n, rows, total, Dl, partial);
}

// The same partial sums for two adjacent columns per thread (n even): 16-byte loads of
// both columns' float-float values, eight rows' loads issued before they are added;
// each column still adds its rows one by one in list order, as dev_bc_partial does, so
// the sums are bit-identical.
constexpr int kBcUnroll = 8;
__global__ void __launch_bounds__(256) k_bc_partial2(int n, const int32_t* rows, const int32_t* count,
                                                     const ff* Dl, ff* partial, const int32_t* err) {
    pdl_enter();
    if (*err) return;
    const int t = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int total = rows ? *count : n;
    if (t >= n) return;
    for (int rb = blockIdx.y; rb * kRowsPerBlock < total; rb += gridDim.y) {
        const int r0 = rb * kRowsPerBlock;
        const int r1 = min(total, r0 + kRowsPerBlock);
        ff a0{0.0f, 0.0f}, a1{0.0f, 0.0f};
        for (int r = r0; r < r1; r += kBcUnroll) {
            int sr[kBcUnroll];
            float4 v[kBcUnroll];
#pragma unroll
            for (int k = 0; k < kBcUnroll; ++k) sr[k] = r + k < r1 ? (rows ? rows[r + k] : r + k) : -1;
#pragma unroll
            for (int k = 0; k < kBcUnroll; ++k)
                if (sr[k] >= 0) v[k] = __ldcs(reinterpret_cast<const float4*>(Dl + (size_t)sr[k] * n + t));
#pragma unroll
            for (int k = 0; k < kBcUnroll; ++k) {
                if (sr[k] < 0) break;
                if (sr[k] != t) a0 = ff_add(a0, ff{v[k].x, v[k].y});
                if (sr[k] != t + 1) a1 = ff_add(a1, ff{v[k].z, v[k].w});
            }
        }
        partial[(size_t)rb * n + t] = a0;
        partial[(size_t)rb * n + t + 1] = a1;
    }
}

__global__ void k_bc_finish(int n, const int32_t* rows, const int32_t* count, const ff* partial,
                            double sign, int overwrite, double* hi, double* lo, const int32_t* err) {
    pdl_enter();
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dev_bc_finish(t, n, rows ? *count : n, partial, sign, overwrite, hi, lo);
}

// ------------------------------------------------------------------ launches

template <typename DT>
static AccArgs<DT> acc_args(const Dev& d, const int32_t* rows, const int32_t* count) {
    AccArgs<DT> a;
    a.n = d.n;
    a.D = (const DT*)d.D;
    a.S = d.S;
    a.Dl = d.Dl;
    a.e_off = d.e_off;
    a.e_len = d.e_len;
    a.e_src = d.e_src;
    a.e_arc = (const Arc<DT>*)d.e_arc;
    a.e_cap = d.e_cap;
    a.rows = rows;
    a.count = count;
    a.ws = d.ws;
    a.ws_stride = d.ws_stride;
    a.err = d.err;
    a.mask_in_smem = d.acc_mask_smem;
    return a;
}

// Shared memory of the accumulation kernel without / with the slot mask.
static size_t smem_base(int n) {
    const size_t np = ((size_t)n + 31) & ~(size_t)31;
    return 4 * np + 2 * (size_t)kBigCap;
}
static size_t mask_bytes(int64_t cap) { return 4 * (size_t)((cap + 31) / 32); }

constexpr size_t kSmemLimit = 180 * 1024;

template <typename DT, int T>
static int accum_occupancy(size_t smem) {
    const int maxs = (int)kSmemLimit;
    cudaFuncSetAttribute(k_accum_smem<DT, false, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
    cudaFuncSetAttribute(k_accum_smem<DT, true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_accum_smem<DT, false, T>, T, smem);
    return per_sm;
}

void accum_config(Dev& d) {
    const size_t base = smem_base(d.n);
    const size_t mb = mask_bytes(d.e_cap);
    const bool in_smem = base + mb <= kSmemLimit;
    const size_t smem = in_smem ? base + mb : base;
    int per_sm = d.dbytes == 4 ? accum_occupancy<int32_t, kAccThreadsNarrow>(smem)
                               : accum_occupancy<int64_t, kAccThreadsNarrow>(smem);
    int per_sm_w = d.dbytes == 4 ? accum_occupancy<int32_t, kAccThreadsWide>(smem)
                                 : accum_occupancy<int64_t, kAccThreadsWide>(smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm_w < 1) per_sm_w = 1;
    d.acc_threads = (d.n >= kAccWideMinN && !d.acc_narrow_only) ? kAccThreadsWide : kAccThreadsNarrow;
    d.acc_smem = (int32_t)smem;
    d.acc_mask_smem = in_smem ? 1 : 0;
    d.acc_grid = std::min(d.nsm * std::max(per_sm, per_sm_w), std::max(d.n, 1));
    d.acc_grid_wide = std::min(d.nsm * per_sm_w, d.acc_grid);
    // per CTA: rho (n float-float pairs) | level bounds (n + 2 ints) | slot mask if not in smem
    const int64_t head = ((3 * (int64_t)d.n + 2) + 3) & ~(int64_t)3;
    d.ws_stride = head + (in_smem ? 0 : (((int64_t)mb / 4 + 3) & ~(int64_t)3));
}

// Algorithm 1 for the sources listed in rows[0..*count), or for every source.
template <typename DT, int T>
static void accum_t(const Dev& d, int is_static, const int32_t* rows, const int32_t* count) {
    const int grid = T == kAccThreadsWide ? d.acc_grid_wide : d.acc_grid;
    const size_t smem = (size_t)d.acc_smem;
    if (is_static) launch_k(k_accum_smem<DT, true, T>, grid, T, smem, d.st, acc_args<DT>(d, rows, count));
    else launch_k(k_accum_smem<DT, false, T>, grid, T, smem, d.st, acc_args<DT>(d, rows, count));
}

// The wide CTAs serve a partial wave of sources (the rows over the target cap of an
// update with pair corrections: tens per update), where one source's latency is the
// time (BA n = 16384: 0.30 ms per update wide, 0.41 ms with 512-thread CTAs), and the
// static computation on the largest graphs (n = 16384: 139 ms wide, 141 ms with 512
// threads; n = 8192: 33.7 ms wide, 30.5 ms with 512 threads, 30.3 ms with 256).  Every
// changed row of an update without pair corrections (thousands of sources) is served
// faster by the narrow ones, several per SM.
constexpr int kAccStaticWideMinN = 16384;

static void accum(const Dev& d, int is_static, const int32_t* rows, const int32_t* count) {
    const bool wide = d.acc_threads == kAccThreadsWide && (is_static ? d.n >= kAccStaticWideMinN : d.pair_on != 0);
    if (d.dbytes == 4) {
        if (wide) accum_t<int32_t, kAccThreadsWide>(d, is_static, rows, count);
        else accum_t<int32_t, kAccThreadsNarrow>(d, is_static, rows, count);
    } else {
        if (wide) accum_t<int64_t, kAccThreadsWide>(d, is_static, rows, count);
        else accum_t<int64_t, kAccThreadsNarrow>(d, is_static, rows, count);
    }
}

void launch_accum(const Dev& d, int is_static) { accum(d, is_static, d.acc_rows, d.counts + 1); }

void launch_accum_rows(const Dev& d, const int32_t* rows, const int32_t* count) { accum(d, 0, rows, count); }

// sign = -1 / +1: subtract / add the rows listed in acc_rows; is_static: all rows,
// overwriting BC.
// The row blocks go to gridDim.y CTAs per column block in turn, about eight CTAs per SM
// in all (the count of listed rows is known only on the device).
static int bc_row_ctas(const Dev& d, int col_blocks) {
    return std::max(1, std::min(d.nrb_max, d.nsm * 8 / col_blocks));
}

static void bc_rows(const Dev& d, int sign, int is_static, const int32_t* rows, const int32_t* count) {
    const int tb = (d.n + 255) / 256;
    dim3 g1(tb, bc_row_ctas(d, tb));
    if (d.n % 2 == 0) {
        const int tb2 = (d.n / 2 + 255) / 256;
        dim3 g2(tb2, bc_row_ctas(d, tb2));
        launch_k(k_bc_partial2, g2, 256, 0, d.st, d.n, rows, count, d.Dl, d.partial, d.err);
    } else {
        launch_k(k_bc_partial, g1, 256, 0, d.st, d.n, rows, count, d.Dl, d.partial, d.err);
    }
    launch_k(k_bc_finish, tb, 256, 0, d.st, d.n, rows, count, d.partial, (double)sign, is_static, d.bc_hi, d.bc_lo,
                                      d.err);
}

void launch_bc_rows(const Dev& d, int sign, int is_static) {
    bc_rows(d, sign, is_static, is_static ? nullptr : d.acc_rows, d.counts + 1);
}

// The same for the rows listed in rows[0..*count).
void launch_bc_rows_list(const Dev& d, int sign, const int32_t* rows, const int32_t* count) {
    bc_rows(d, sign, 0, rows, count);
}

}  // namespace bcg
