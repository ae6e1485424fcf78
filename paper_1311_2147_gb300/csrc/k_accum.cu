// k_accum.cu -- dependency accumulation and the BC reduction.
//
// For each source s whose row changed (and, in the static computation, for every s):
//   * DAG'(s) is rebuilt implicitly: an arc (a,b) of the E* superset is in DAG'(s)
//     iff d'(s,a) is finite and d'(s,a) + w(a,b) = d'(s,b) (Eq. 1; Algorithm 6 step 4
//     applied to E'; Section 6 notes any superset of E* gives the same DAGs).
//   * A topological order of DAG'(s) is built level by level (Kahn): a vertex joins
//     level L+1 when its last in-arc from level L is consumed.  Section 2 notes that
//     any reverse topological order serves Algorithm 1 as well as the order by
//     distance; level order keeps the sequential chain as short as the DAG is deep.
//     In the static computation the same sweep carries the path counts forward
//     (sigma_sb = sum of sigma_sa over DAG in-arcs, Algorithm 6 step 7).
//   * delta_s. is pulled in reverse level order: delta(a) = sum over DAG out-arcs
//     (a,b) of sigma_sa / sigma_sb * (1 + delta(b))  (Eq. 4).  One warp per vertex,
//     lanes over its arcs, a fixed butterfly for the warp sum, so the result does
//     not depend on scheduling.
// BC is maintained as BC += sum over changed rows of (delta'_s - delta_s): the old rows
// are subtracted before the rows are rewritten and the new rows added after
// (Algorithm 3 step 1 recomputes BC from zero; rows that did not change contribute
// the same amount before and after, so only changed rows are touched).  Column sums
// run over row blocks in a fixed order into a compensated (hi, lo) pair.
#include "bc_internal.cuh"

namespace bcg {

template <typename DT>
struct AccArgs {
    int n;
    const DT* D;
    uint64_t* S;
    double* Dl;
    const int32_t* e_off;
    const int32_t* e_len;
    const int32_t* e_src;
    const int32_t* e_dst;
    const DT* e_w;
    int64_t e_cap;
    const int32_t* rows;
    const int32_t* count;
    int32_t* ws;
    int64_t ws_stride;
    int32_t* err;
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <typename DT, bool STATIC>
__global__ void __launch_bounds__(kAccThreads) k_accum(AccArgs<DT> a) {
    const int n = a.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = kAccThreads / 32;
    const int64_t INF = Inf<DT>::v;
    int32_t* cnt = a.ws + (size_t)blockIdx.x * a.ws_stride;
    int32_t* order = cnt + n;
    int32_t* lvl = order + n;   // n + 2 entries
    __shared__ int s_tail;
    const int total = STATIC ? n : *a.count;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        if (block_err(a.err)) return;
        const int s = STATIC ? i : a.rows[i];
        const DT* __restrict__ Ds = a.D + (size_t)s * n;
        uint64_t* Ss = a.S + (size_t)s * n;
        double* out = a.Dl + (size_t)s * n;
        for (int t = tid; t < n; t += kAccThreads) {
            cnt[t] = 0;
            out[t] = 0.0;
            if (STATIC) Ss[t] = (t == s) ? 1ull : 0ull;
        }
        __syncthreads();
        // in-degree of every vertex in DAG'(s), over the slots of the E* superset
        for (int64_t e = tid; e < a.e_cap; e += kAccThreads) {
            const int b = a.e_dst[e];
            if (b < 0) continue;
            const int64_t dx = Ds[a.e_src[e]];
            if (dx == INF) continue;
            if ((uint64_t)dx + (uint64_t)a.e_w[e] == (uint64_t)(int64_t)Ds[b]) atomicAdd(&cnt[b], 1);
        }
        if (tid == 0) {
            order[0] = s;
            lvl[0] = 0;
            lvl[1] = 1;
            s_tail = 1;
        }
        __syncthreads();
        // Kahn levels (and, statically, forward path counts)
        int L = 0;
        for (;;) {
            const int lo = lvl[L], hi = lvl[L + 1];
            for (int q = lo + warp; q < hi; q += nwarps) {
                const int x = order[q];
                const uint64_t dx = (uint64_t)(int64_t)Ds[x];
                const uint64_t sx = STATIC ? Ss[x] : 0ull;
                const int beg = a.e_off[x], end = beg + a.e_len[x];
                for (int e = beg + lane; e < end; e += 32) {
                    const int b = a.e_dst[e];
                    if (dx + (uint64_t)a.e_w[e] != (uint64_t)(int64_t)Ds[b]) continue;
                    if (STATIC) {
                        const unsigned long long old =
                            atomicAdd(reinterpret_cast<unsigned long long*>(Ss + b), (unsigned long long)sx);
                        if (old + sx < old) set_err(a.err, ERRF_OVERFLOW);
                    }
                    if (atomicSub(&cnt[b], 1) == 1) order[atomicAdd(&s_tail, 1)] = b;
                }
            }
            __syncthreads();
            if (tid == 0) lvl[L + 2] = s_tail;
            __syncthreads();
            if (lvl[L + 2] == hi) break;
            ++L;
        }
        // Eq. 4 in reverse level order (level 0 is s itself: delta_s.(s) is not kept)
        for (int Lq = L; Lq >= 1; --Lq) {
            const int lo = lvl[Lq], hi = lvl[Lq + 1];
            for (int q = lo + warp; q < hi; q += nwarps) {
                const int x = order[q];
                const uint64_t dx = (uint64_t)(int64_t)Ds[x];
                const double sx = (double)Ss[x];
                const int beg = a.e_off[x], end = beg + a.e_len[x];
                double acc = 0.0;
                for (int e = beg + lane; e < end; e += 32) {
                    const int b = a.e_dst[e];
                    if (dx + (uint64_t)a.e_w[e] != (uint64_t)(int64_t)Ds[b]) continue;
                    acc += sx / (double)Ss[b] * (1.0 + out[b]);
                }
                acc = warp_sum(acc);
                if (lane == 0) out[x] = acc;
            }
            __syncthreads();
        }
        __syncthreads();
    }
}

// partial[rb][t] = sum over rows r of row block rb of Dl[s_r][t] (t != s_r), rows in
// increasing order; rows = nullptr means all n rows.
__global__ void k_bc_partial(int n, const int32_t* rows, const int32_t* count, const double* Dl,
                             double* partial, const int32_t* err) {
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rb = blockIdx.y;
    const int total = rows ? *count : n;
    const int r0 = rb * kRowsPerBlock;
    if (r0 >= total || t >= n) return;
    const int r1 = min(total, r0 + kRowsPerBlock);
    double acc = 0.0;
    for (int r = r0; r < r1; ++r) {
        const int s = rows ? rows[r] : r;
        if (s != t) acc += Dl[(size_t)s * n + t];
    }
    partial[(size_t)rb * n + t] = acc;
}

// bc (hi, lo) += sign * (sum of the row-block partials in block order); overwrite
// starts from zero (the static computation).
__global__ void k_bc_finish(int n, const int32_t* rows, const int32_t* count, const double* partial,
                            double sign, int overwrite, double* hi, double* lo, const int32_t* err) {
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int total = rows ? *count : n;
    const int nrb = (total + kRowsPerBlock - 1) / kRowsPerBlock;
    if (nrb == 0 && !overwrite) return;
    double sum = 0.0;
    for (int rb = 0; rb < nrb; ++rb) sum += partial[(size_t)rb * n + t];
    sum *= sign;
    if (overwrite) {
        hi[t] = sum;
        lo[t] = 0.0;
        return;
    }
    // TwoSum (Knuth): h + x = s + e exactly
    const double h = hi[t];
    const double s = h + sum;
    const double bp = s - h;
    const double e = (h - (s - bp)) + (sum - bp);
    hi[t] = s;
    lo[t] += e;
}

// ------------------------------------------------------------------ launches

template <typename DT>
static AccArgs<DT> acc_args(const Dev& d) {
    AccArgs<DT> a;
    a.n = d.n;
    a.D = (const DT*)d.D;
    a.S = d.S;
    a.Dl = d.Dl;
    a.e_off = d.e_off;
    a.e_len = d.e_len;
    a.e_src = d.e_src;
    a.e_dst = d.e_dst;
    a.e_w = (const DT*)d.e_w;
    a.e_cap = d.e_cap;
    a.rows = d.acc_rows;
    a.count = d.counts + 1;
    a.ws = d.ws;
    a.ws_stride = d.ws_stride;
    a.err = d.err;
    return a;
}

void launch_accum(const Dev& d, int is_static) {
    const int grid = d.acc_grid;
    if (d.dbytes == 4) {
        if (is_static) k_accum<int32_t, true><<<grid, kAccThreads, 0, d.st>>>(acc_args<int32_t>(d));
        else k_accum<int32_t, false><<<grid, kAccThreads, 0, d.st>>>(acc_args<int32_t>(d));
    } else {
        if (is_static) k_accum<int64_t, true><<<grid, kAccThreads, 0, d.st>>>(acc_args<int64_t>(d));
        else k_accum<int64_t, false><<<grid, kAccThreads, 0, d.st>>>(acc_args<int64_t>(d));
    }
}

// sign = -1 / +1: subtract / add the rows listed in acc_rows; is_static: all rows,
// overwriting BC.
void launch_bc_rows(const Dev& d, int sign, int is_static) {
    const int tb = (d.n + 255) / 256;
    dim3 g1(tb, d.nrb_max);
    const int32_t* rows = is_static ? nullptr : d.acc_rows;
    k_bc_partial<<<g1, 256, 0, d.st>>>(d.n, rows, d.counts + 1, d.Dl, d.partial, d.err);
    k_bc_finish<<<tb, 256, 0, d.st>>>(d.n, rows, d.counts + 1, d.partial, (double)sign, is_static,
                                      d.bc_hi, d.bc_lo, d.err);
}

}  // namespace bcg
