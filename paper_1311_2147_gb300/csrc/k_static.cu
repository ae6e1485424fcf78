// k_static.cu -- the all-pairs distances of the static computation.
//
// bc_init_static needs d(s,t) for every pair before E* can be read off it.  Brandes
// (Appendix, Algorithm 7) runs Dijkstra from every source; a priority queue does not
// map well onto a CTA, so each CTA runs a label-correcting (Bellman-Ford) sweep from
// one source at a time with a frontier bitmap in shared memory: every round relaxes
// the out-arcs of the vertices whose distance dropped in the round before, until no
// distance drops.  With positive weights this ends after at most n-1 rounds with the
// same distances Dijkstra settles.  The distance row lives in shared memory when it
// fits, else in its row of D.
//
// E* (Section 1: arcs on some shortest path) is then {(a,b) : w(a,b) = d(a,b)}: the
// one-arc path a->b is shortest exactly when the arc lies on a shortest path (a
// sub-path of a shortest path is shortest).
//
// E* pruning (Section 6, Algorithm 6 step 1: the Hidden Paths algorithm examines only
// arcs of E*).  A search from s needs only the arcs of E* (every shortest path is made
// of them), and an arc (a,b) is known to be in E* or not as soon as the search from a
// has finished: w(a,b) = d(a,b).  So with pruning on, the CTA that finishes the
// search from a overwrites the head of every arc of a that is not in E* with -1 in a
// working copy of the arc heads, and every later search skips those arcs.  A search
// that reads a head while it is being overwritten sees either the head or -1; both are
// correct, since a search may use any set of arcs that contains E*.  The sources run in
// the given order, highest out-degree first, so that most arcs are decided early.
// (Hidden Paths settles the pairs of all sources in one global distance order and so
// never examines an arc outside E*; this form examines each arc at most until its
// tail's own search has finished.)
#include "bc_internal.cuh"

namespace bcg {

constexpr int kSsspThreads = 512;

template <typename DT>
__device__ __forceinline__ int64_t ld_relaxed(const DT* p) {
    return (int64_t)*reinterpret_cast<const volatile DT*>(p);
}

__device__ __forceinline__ int32_t atomic_min_dt(int32_t* p, int32_t v) { return atomicMin(p, v); }
__device__ __forceinline__ int64_t atomic_min_dt(int64_t* p, int64_t v) {
    return (int64_t)atomicMin(reinterpret_cast<long long*>(p), (long long)v);
}

// order: the sources in the order to run them (NULL: 0 .. n-1).  pdst: the working
// copy of the arc heads to prune (NULL: every arc is searched, dst is read).
template <typename DT, bool SMEM_DIST>
__global__ void __launch_bounds__(kSsspThreads)
k_sssp(int n, const int32_t* __restrict__ off, const int32_t* __restrict__ dst,
       const DT* __restrict__ w, DT* D, int32_t* err, const int32_t* __restrict__ order, int32_t* pdst) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int words = (n + 31) >> 5;
    DT* dist_s = reinterpret_cast<DT*>(smem);
    uint32_t* cur = reinterpret_cast<uint32_t*>(smem + (SMEM_DIST ? (((size_t)n * sizeof(DT) + 15) & ~(size_t)15) : 0));
    uint32_t* nxt = cur + words;
    __shared__ int s_sat;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = kSsspThreads / 32;
    const int64_t INF = Inf<DT>::v;
    const int32_t* heads = pdst ? pdst : dst;
    for (int si = blockIdx.x; si < n; si += gridDim.x) {
        if (block_err(err)) return;
        const int s = order ? order[si] : si;
        DT* dist = SMEM_DIST ? dist_s : D + (size_t)s * n;
        for (int t = tid; t < n; t += kSsspThreads) dist[t] = (t == s) ? (DT)0 : (DT)INF;
        for (int q = tid; q < words; q += kSsspThreads) {
            cur[q] = (q == (s >> 5)) ? (1u << (s & 31)) : 0u;
            nxt[q] = 0u;
        }
        if (tid == 0) s_sat = 0;
        __syncthreads();
        bool converged = false;
        for (int round = 0; round <= n; ++round) {
            for (int q = warp; q < words; q += nwarps) {
                uint32_t bits = cur[q];
                while (bits) {
                    const int x = (q << 5) + __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const int64_t dx = ld_relaxed(dist + x);
                    const int end = off[x + 1];
                    for (int e = off[x] + lane; e < end; e += 32) {
                        const int b = ld_relaxed(heads + e);
                        if (b < 0) continue;   // pruned: not in E*
                        const int64_t nd = dsum<DT>(dx, (int64_t)w[e]);
                        if (nd == SAT) {
                            s_sat = 1;
                            continue;
                        }
                        if (nd < ld_relaxed(dist + b)) {
                            const int64_t old = atomic_min_dt(dist + b, (DT)nd);
                            if (nd < old) atomicOr(nxt + (b >> 5), 1u << (b & 31));
                        }
                    }
                }
            }
            __syncthreads();
            int any = 0;
            for (int q = tid; q < words; q += kSsspThreads) {
                const uint32_t x = nxt[q];
                cur[q] = x;
                nxt[q] = 0u;
                any |= (x != 0u);
            }
            if (!__syncthreads_or(any)) {
                converged = true;
                break;
            }
        }
        // positive weights converge within n-1 rounds; anything else is reported
        if (!converged && tid == 0) set_err(err, ERRF_TIMEOUT);
        // A relaxation whose sum did not fit matters only if it was the way to reach a
        // vertex: then that vertex has a distance the type cannot hold.
        if (s_sat) {
            for (int x = warp; x < n; x += nwarps) {
                const int64_t dx = dist[x];
                if (dx == INF) continue;
                for (int e = off[x] + lane; e < off[x + 1]; e += 32)
                    if (dsum<DT>(dx, (int64_t)w[e]) == SAT && (int64_t)dist[dst[e]] == INF)
                        set_err(err, ERRF_DIST);
            }
        }
        if (SMEM_DIST) {
            DT* row = D + (size_t)s * n;
            for (int t = tid; t < n; t += kSsspThreads) row[t] = dist_s[t];
        }
        // the search from s is final: the arcs of s with w(s,b) > d(s,b) are not in E*
        if (pdst)
            for (int e = off[s] + tid; e < off[s + 1]; e += kSsspThreads) {
                const int b = dst[e];
                if ((int64_t)w[e] != ld_relaxed(dist + b)) pdst[e] = -1;
            }
        __syncthreads();
    }
}

template <typename DT>
__global__ void k_estar_flags(int n, int64_t arcs, const int32_t* g_src, const int32_t* g_dst,
                              const DT* g_w, const DT* D, uint8_t* flags) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= arcs) return;
    flags[e] = ((int64_t)D[(size_t)g_src[e] * n + g_dst[e]] == (int64_t)g_w[e]) ? 1 : 0;
}

template <typename DT>
static void sssp_dispatch(const Dev& d) {
    const size_t words = ((size_t)d.n + 31) / 32;
    const size_t bitmaps = 2 * words * sizeof(uint32_t);
    const size_t dist_bytes = (((size_t)d.n * sizeof(DT)) + 15) & ~(size_t)15;
    const size_t smem_cap = 200 * 1024;
    if (dist_bytes + bitmaps <= smem_cap) {
        const size_t smem = dist_bytes + bitmaps;
        cudaFuncSetAttribute(k_sssp<DT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sssp<DT, true>, kSsspThreads, smem);
        if (per_sm < 1) per_sm = 1;
        const int grid = (int)std::min<int64_t>((int64_t)d.nsm * per_sm, d.n);
        k_sssp<DT, true><<<grid, kSsspThreads, smem, d.st>>>(d.n, d.g_off, d.g_dst, (const DT*)d.g_w,
                                                             (DT*)d.D, d.err, d.s_order, d.p_dst);
    } else {
        const size_t smem = bitmaps;
        cudaFuncSetAttribute(k_sssp<DT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sssp<DT, false>, kSsspThreads, smem);
        if (per_sm < 1) per_sm = 1;
        const int grid = (int)std::min<int64_t>((int64_t)d.nsm * per_sm, d.n);
        k_sssp<DT, false><<<grid, kSsspThreads, smem, d.st>>>(d.n, d.g_off, d.g_dst, (const DT*)d.g_w,
                                                              (DT*)d.D, d.err, d.s_order, d.p_dst);
    }
}

void launch_sssp(const Dev& d) {
    if (d.dbytes == 4) sssp_dispatch<int32_t>(d);
    else sssp_dispatch<int64_t>(d);
}

void launch_estar_flags(const Dev& d, uint8_t* flags) {
    if (d.g_arcs <= 0) return;
    const int blocks = (int)((d.g_arcs + 255) / 256);
    if (d.dbytes == 4)
        k_estar_flags<int32_t><<<blocks, 256, 0, d.st>>>(d.n, d.g_arcs, d.g_src, d.g_dst,
                                                         (const int32_t*)d.g_w, (const int32_t*)d.D, flags);
    else
        k_estar_flags<int64_t><<<blocks, 256, 0, d.st>>>(d.n, d.g_arcs, d.g_src, d.g_dst,
                                                         (const int64_t*)d.g_w, (const int64_t*)d.D, flags);
}

}  // namespace bcg
