// k_update.cu -- the all-pairs part of an incremental update.
//
// Every update is handled as a vertex update of some vertex v (Section 4): an edge
// update (u, v, w') is the vertex update of v whose in-edge set E_i is {(u, v)}
// (Algorithm 4 with one edge gives exactly Lemma 2's three cases), and an undirected
// update is the vertex update of G_D whose E_i and E_o hold both arcs of each edge
// (Section 3, "Undirected graphs").  Per phase:
//
//   IN  (E_i):  k_alg4_in   Algorithm 4 for every source s -> d'(s,v), sigma'_sv,
//                           sigma-hat'_sv, and whether row s can change;
//               k_compact   rows that change, in increasing order;
//               k_scan      Lemma 4 over those rows: D(s,t) = d'(s,v) + d(v,t).
//   OUT (E_o):  k_alg4_out  Algorithm 4 on the reversed graph G'_R for every target t
//                           -> d''(v,t), sigma''_vt, sigma-hat''_vt (row v of the
//                           result; reads rows x_j of D', which are contiguous);
//               k_rows_out  rows s with d'(s,v) + w'(v,x_j) <= d'(s,x_j) for some j;
//               k_compact, k_scan  Lemma 4 read on G'_R: D(s,t) = d'(s,v) + d''(v,t);
//               k_write_row row v <- (d''(v,.), sigma''_v.).
//
// Lemma 1 (and its vertex analogue) makes the in-place scan race free: during the IN
// phase row v and column x_j are never written, during the OUT phase column v is not.
#include "bc_internal.cuh"

namespace bcg {

__global__ void k_estar_write(int32_t* e_src, void* e_arc, int32_t* e_len, int dbytes, EOps ops) {
    int i = threadIdx.x;
    if (i >= ops.count) return;
    const EOp o = ops.op[i];
    if (o.slot >= 0) {
        e_src[o.slot] = o.a;
        if (dbytes == 4) static_cast<Arc<int32_t>*>(e_arc)[o.slot] = Arc<int32_t>{o.b, (int32_t)o.w};
        else static_cast<Arc<int64_t>*>(e_arc)[o.slot] = Arc<int64_t>{(int64_t)o.b, o.w};
    }
    atomicMax(e_len + o.a, o.len_a);   // lengths only grow between rebuilds
}

// Algorithm 4 (Compute-Dist-to-v) for source s = this thread, over the in-edges
// (x_j, v) of the update, followed by the affected-row test of the IN phase: row s can
// change only if d'(s,v) < d(s,v) or new shortest paths reach v (sigma-hat > 0).
template <typename DT>
__global__ void k_alg4_in(int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                          int v, const VEdge* __restrict__ e, int k, int directed,
                          DT* fD, uint64_t* fS, uint64_t* fM, uint8_t* mark, uint8_t* changed,
                          int32_t* err) {
    if (*err) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t INF = Inf<DT>::v;
    const size_t rs = (size_t)s * n;
    const int64_t old = D[rs + v];
    int64_t cur = old;
    uint64_t sig = S[rs + v];
    uint64_t hat = 0;
    bool sat = false;
    for (int j = 0; j < k; ++j) {
        const VEdge ed = e[j];
        if (directed && ed.dir != 0) continue;
        const int64_t dx = D[rs + ed.x];
        if (dx == INF) continue;
        const int64_t dj = dsum<DT>(dx, ed.w);
        if (dj == SAT) {
            sat = true;
            continue;
        }
        const uint64_t sx = S[rs + ed.x];
        if (cur == dj) {
            sig = add_chk(sig, sx, err);
            hat += sx;
        } else if (cur > dj) {
            cur = dj;
            sig = sx;
        }
    }
    // v reachable from s only through a sum that does not fit: d'(s,v) overflows.
    if (sat && cur == INF) set_err(err, ERRF_DIST);
    const bool dec = cur < old;
    const bool aff = dec || hat != 0;
    fD[s] = (DT)cur;
    fS[s] = sig;
    fM[s] = dec ? sig : hat;
    mark[s] = aff ? 1 : 0;
    if (aff) changed[s] = 1;
}

// OUT phase, row test: row s (s != v) can change only through a new shortest path
// s ~> v -> x_j, i.e. d'(s,v) + w'(v,x_j) <= d'(s,x_j) for some out-edge of the update.
template <typename DT>
__global__ void k_rows_out(int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                           int v, const VEdge* __restrict__ e, int k, int directed,
                           DT* fD, uint64_t* fS, uint64_t* fM, uint8_t* mark, uint8_t* changed,
                           int32_t* err) {
    if (*err) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t INF = Inf<DT>::v;
    const size_t rs = (size_t)s * n;
    const int64_t dsv = D[rs + v];
    const uint64_t ssv = S[rs + v];
    bool aff = false;
    if (s != v && dsv != INF) {
        for (int j = 0; j < k; ++j) {
            const VEdge ed = e[j];
            if (directed && ed.dir != 1) continue;
            const int64_t dy = D[rs + ed.x];
            const int64_t c = dsum<DT>(dsv, ed.w);
            // A sum that does not fit can only matter where d'(s,x_j) is INF; the row is
            // then kept so that the scan decides (and reports a distance overflow).
            if (c == SAT) {
                if (dy == INF) aff = true;
                continue;
            }
            if (c <= dy) aff = true;
        }
    }
    fD[s] = (DT)dsv;
    fS[s] = ssv;
    fM[s] = ssv;
    mark[s] = aff ? 1 : 0;
    if (aff) changed[s] = 1;
}

// Algorithm 4 on the reversed graph G'_R, for "source" t of G'_R = target t of G: the
// out-edges (v, x_j) of the update are in-edges of v in G'_R, and d_R(t, x_j) is
// d'(x_j, t), read from row x_j.  Produces row v of the result.
template <typename DT>
__global__ void k_alg4_out(int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                           int v, const VEdge* __restrict__ e, int k, int directed,
                           DT* cD, uint64_t* cS, uint64_t* cM, uint8_t* changed, int32_t* err) {
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t INF = Inf<DT>::v;
    const size_t rv = (size_t)v * n;
    const int64_t old = D[rv + t];
    int64_t cur = old;
    uint64_t sig = S[rv + t];
    uint64_t hat = 0;
    bool sat = false;
    for (int j = 0; j < k; ++j) {
        const VEdge ed = e[j];
        if (directed && ed.dir != 1) continue;
        const size_t ry = (size_t)ed.x * n;
        const int64_t dy = D[ry + t];
        if (dy == INF) continue;
        const int64_t dj = dsum<DT>(ed.w, dy);
        if (dj == SAT) {
            sat = true;
            continue;
        }
        const uint64_t sy = S[ry + t];
        if (cur == dj) {
            sig = add_chk(sig, sy, err);
            hat += sy;
        } else if (cur > dj) {
            cur = dj;
            sig = sy;
        }
    }
    if (sat && cur == INF) set_err(err, ERRF_DIST);
    const bool dec = cur < old;
    cD[t] = (DT)cur;
    cS[t] = sig;
    cM[t] = dec ? sig : hat;
    if (dec || hat != 0) changed[v] = 1;
}

// Stable compaction of {s : mark[s]} (or of all s when full) into rows[], one CTA.
// Optionally clears mark[] and accumulates the per-update counters.
constexpr int kCompactThreads = 1024;
__global__ void __launch_bounds__(kCompactThreads)
k_compact(int n, uint8_t* mark, int clear, int32_t* rows, int32_t* count, int full,
          int64_t* stats, const int32_t* err) {
    __shared__ int32_t wsum[32];
    __shared__ int32_t s_total;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool bad = *err != 0;
    const unsigned lt = (1u << lane) - 1u;
    int base = 0;
    for (int tile = 0; tile < n; tile += kCompactThreads) {
        const int s = tile + tid;
        int f = 0;
        if (s < n) {
            f = (!bad && (full || mark[s] != 0)) ? 1 : 0;
            if (clear) mark[s] = 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int wpre = __popc(bal & lt);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        if (wid == 0) {
            const int x = wsum[lane];
            int incl = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            wsum[lane] = incl - x;
            if (lane == 31) s_total = incl;
        }
        __syncthreads();
        if (f) rows[base + wsum[wid] + wpre] = s;
        base += s_total;
        __syncthreads();
    }
    if (tid == 0) {
        *count = base;
        if (stats) {
            stats[0] += base;
            if (base == 0) stats[1] += 1;
            if (base > stats[2]) stats[2] = base;
            stats[3] += 1;
        }
    }
}

// Vector access of VEC consecutive distances (16 bytes).
template <typename DT> struct Vec;
template <> struct Vec<int32_t> {
    static constexpr int N = 4;
    using T = int4;
    __device__ static void unpack(const T& x, int64_t* o) { o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w; }
    __device__ static void set(T& x, int i, int64_t val) {
        if (i == 0) x.x = (int32_t)val; else if (i == 1) x.y = (int32_t)val;
        else if (i == 2) x.z = (int32_t)val; else x.w = (int32_t)val;
    }
};
template <> struct Vec<int64_t> {
    static constexpr int N = 2;
    using T = longlong2;
    __device__ static void unpack(const T& x, int64_t* o) { o[0] = x.x; o[1] = x.y; }
    __device__ static void set(T& x, int i, int64_t val) { if (i == 0) x.x = val; else x.y = val; }
};

constexpr int kScanThreads = 256;
constexpr int kScanUnroll = 4;

template <typename DT>
struct ScanArgs {
    int n;
    DT* D;
    uint64_t* S;
    const int32_t* rows;
    const int32_t* count;
    const DT* fD;          // per row s: distance to v (after the IN phase)
    const uint64_t* fS;    // per row s: path count to v
    const uint64_t* fM;    // per row s: multiplier of a tie
    const DT* cD;          // per column t: distance from v
    const uint64_t* cS;    // per column t: path count from v
    const uint64_t* cM;    // per column t: multiplier of a tie
    int skip_row;
    int32_t* err;
    int64_t* stats;        // [4] pairs with a lower distance [5] pairs with new tied paths [6] rows
};

// The rank-1 rule of Lemma 2 / Lemma 4 for one pair, given the candidate distance
// cand = rd + cd through v:  cand > d: unchanged;  cand == d: sigma += rowM * colM
// (new shortest paths through v);  cand < d: d = cand, sigma = rowS * colS.
template <typename DT>
__device__ __forceinline__ bool pair_rule(int64_t cand, int64_t old, size_t idx, uint64_t rs,
                                          uint64_t rm, uint64_t cs, uint64_t cm,
                                          uint64_t* S, int32_t* err, int64_t* newd, int* ties) {
    if (cand == SAT) {
        if (old == Inf<DT>::v) set_err(err, ERRF_DIST);
        return false;
    }
    if (cand > old) return false;
    if (cand < old) {
        S[idx] = mul_chk(rs, cs, err);
        *newd = cand;
        return true;
    }
    const uint64_t p = mul_chk(rm, cm, err);
    if (p != 0ull) {
        S[idx] = add_chk(S[idx], p, err);
        ++*ties;
    }
    return false;
}

// K2: in-place rank-1 min-plus / path-count pass over rows[0..count) x all columns.
// Work item = (row, chunk of CW columns).  Each CTA takes a contiguous block of items,
// so the per-row scalars are loaded once per row it meets; each thread issues all of
// its 16-byte loads of D and of the column vectors of an item before using any.  sigma
// is read only on ties and written only where the pair changes.
template <typename DT, bool VECTOR>
__global__ void __launch_bounds__(kScanThreads, 4) k_scan(ScanArgs<DT> a) {
    // warp-uniform early exit: the warp sum at the end needs every lane
    int bad = 0;
    if ((threadIdx.x & 31) == 0) bad = *reinterpret_cast<volatile int32_t*>(a.err);
    if (__shfl_sync(0xffffffffu, bad, 0)) return;
    using V = Vec<DT>;
    constexpr int VN = V::N;
    constexpr int CW = kScanThreads * VN * kScanUnroll;
    const int n = a.n;
    const int nchunks = (n + CW - 1) / CW;
    const int64_t total = (int64_t)(*a.count) * nchunks;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t it0 = (int64_t)blockIdx.x * per;
    const int64_t it1 = min(total, it0 + per);
    const int64_t INF = Inf<DT>::v;
    int n_changed = 0, n_ties = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 6),
                                                       (unsigned long long)(*a.count));
    int cur = -1, s = -1;
    int64_t rd = INF;
    uint64_t rs = 0, rm = 0;
    for (int64_t item = it0; item < it1; ++item) {
        const int i = (int)(item / nchunks);
        const int c = (int)(item - (int64_t)i * nchunks);
        if (i != cur) {
            cur = i;
            s = a.rows[i];
            rd = (s == a.skip_row) ? INF : (int64_t)a.fD[s];
            rs = a.fS[s];
            rm = a.fM[s];
        }
        if (rd == INF) continue;
        const size_t rowoff = (size_t)s * n;
        DT* __restrict__ Drow = a.D + rowoff;
        const int t0 = c * CW;
        if constexpr (VECTOR) {
            typename V::T dv[kScanUnroll], cv[kScanUnroll];
#pragma unroll
            for (int u = 0; u < kScanUnroll; ++u) {
                const int t = t0 + (u * kScanThreads + threadIdx.x) * VN;
                if (t < n) {
                    dv[u] = __ldcs(reinterpret_cast<const typename V::T*>(Drow + t));
                    cv[u] = __ldg(reinterpret_cast<const typename V::T*>(a.cD + t));
                }
            }
#pragma unroll
            for (int u = 0; u < kScanUnroll; ++u) {
                const int t = t0 + (u * kScanThreads + threadIdx.x) * VN;
                if (t >= n) break;
                bool any = false;
                if constexpr (sizeof(DT) == 4) {
                    // both terms are below 2^31, so their sum fits 32 bits: a pair can change
                    // only if the column term is finite and the sum does not exceed d (or d
                    // is INF, where a sum that does not fit must be reported)
                    const uint32_t r32 = (uint32_t)rd;
                    const int32_t* dp = reinterpret_cast<const int32_t*>(&dv[u]);
                    const int32_t* cp = reinterpret_cast<const int32_t*>(&cv[u]);
#pragma unroll
                    for (int q = 0; q < VN; ++q) {
                        const uint32_t sum = r32 + (uint32_t)cp[q];
                        any |= (cp[q] != INT32_MAX) & ((sum <= (uint32_t)dp[q]) | (dp[q] == INT32_MAX));
                    }
                } else {
                    int64_t dd0[VN], cd0[VN];
                    V::unpack(dv[u], dd0);
                    V::unpack(cv[u], cd0);
#pragma unroll
                    for (int q = 0; q < VN; ++q) {
                        if (cd0[q] == INF) continue;
                        const int64_t cand = dsum<DT>(rd, cd0[q]);
                        any |= (cand <= dd0[q]) || (cand == SAT);
                    }
                }
                if (!any) continue;
                int64_t dd[VN], cd[VN];
                V::unpack(dv[u], dd);
                V::unpack(cv[u], cd);
                bool wr = false;
#pragma unroll
                for (int q = 0; q < VN; ++q) {
                    if (cd[q] == INF) continue;
                    const int64_t cand = dsum<DT>(rd, cd[q]);
                    int64_t nd;
                    if (pair_rule<DT>(cand, dd[q], rowoff + t + q, rs, rm, a.cS[t + q], a.cM[t + q],
                                      a.S, a.err, &nd, &n_ties)) {
                        V::set(dv[u], q, nd);
                        wr = true;
                        ++n_changed;
                    }
                }
                if (wr) *reinterpret_cast<typename V::T*>(Drow + t) = dv[u];
            }
        } else {
            for (int t = t0 + threadIdx.x; t < t0 + CW && t < n; t += kScanThreads) {
                const int64_t cd = a.cD[t];
                if (cd == INF) continue;
                const int64_t old = Drow[t];
                const int64_t cand = dsum<DT>(rd, cd);
                int64_t nd;
                if (pair_rule<DT>(cand, old, rowoff + t, rs, rm, a.cS[t], a.cM[t], a.S, a.err, &nd, &n_ties)) {
                    Drow[t] = (DT)nd;
                    ++n_changed;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_changed += __shfl_xor_sync(0xffffffffu, n_changed, o);
        n_ties += __shfl_xor_sync(0xffffffffu, n_ties, o);
    }
    if ((threadIdx.x & 31) == 0 && (n_changed | n_ties)) {
        atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 4), (unsigned long long)n_changed);
        atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 5), (unsigned long long)n_ties);
    }
}

template <typename DT>
__global__ void k_write_row(int n, DT* D, uint64_t* S, int v, const DT* cD, const uint64_t* cS,
                            const int32_t* err) {
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    D[(size_t)v * n + t] = cD[t];
    S[(size_t)v * n + t] = cS[t];
}

// keep[e] = 1 when slot e holds an arc (a,b) with w(a,b) == d(a,b), i.e. an arc of E*
// (an arc lies on a shortest path exactly when it is one itself).
template <typename DT>
__global__ void k_estar_keep(int n, const DT* D, const int32_t* e_src, const Arc<DT>* e_arc,
                             int64_t cap, uint8_t* keep) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cap) return;
    const Arc<DT> a = e_arc[e];
    keep[e] = (a.dst >= 0 && (int64_t)D[(size_t)e_src[e] * n + a.dst] == (int64_t)a.w) ? 1 : 0;
}

// ------------------------------------------------------------------ launches

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

void launch_estar_write(const Dev& d, const EOps& ops) {
    if (ops.count <= 0) return;
    k_estar_write<<<1, kMaxEOps, 0, d.st>>>(d.e_src, d.e_arc, d.e_len, d.dbytes, ops);
}

void launch_alg4_in(const Dev& d, int32_t v, const VEdge* e, int32_t k) {
    if (d.dbytes == 4)
        k_alg4_in<int32_t><<<nblk(d.n, 256), 256, 0, d.st>>>(
            d.n, (const int32_t*)d.D, d.S, v, e, k, d.directed, (int32_t*)d.fD, d.fS, d.fM,
            d.mark, d.changed, d.err);
    else
        k_alg4_in<int64_t><<<nblk(d.n, 256), 256, 0, d.st>>>(
            d.n, (const int64_t*)d.D, d.S, v, e, k, d.directed, (int64_t*)d.fD, d.fS, d.fM,
            d.mark, d.changed, d.err);
}

void launch_rows_out(const Dev& d, int32_t v, const VEdge* e, int32_t k) {
    if (d.dbytes == 4)
        k_rows_out<int32_t><<<nblk(d.n, 256), 256, 0, d.st>>>(
            d.n, (const int32_t*)d.D, d.S, v, e, k, d.directed, (int32_t*)d.fD, d.fS, d.fM,
            d.mark, d.changed, d.err);
    else
        k_rows_out<int64_t><<<nblk(d.n, 256), 256, 0, d.st>>>(
            d.n, (const int64_t*)d.D, d.S, v, e, k, d.directed, (int64_t*)d.fD, d.fS, d.fM,
            d.mark, d.changed, d.err);
}

void launch_alg4_out(const Dev& d, int32_t v, const VEdge* e, int32_t k) {
    if (d.dbytes == 4)
        k_alg4_out<int32_t><<<nblk(d.n, 256), 256, 0, d.st>>>(
            d.n, (const int32_t*)d.D, d.S, v, e, k, d.directed, (int32_t*)d.cD, d.cS, d.cM,
            d.changed, d.err);
    else
        k_alg4_out<int64_t><<<nblk(d.n, 256), 256, 0, d.st>>>(
            d.n, (const int64_t*)d.D, d.S, v, e, k, d.directed, (int64_t*)d.cD, d.cS, d.cM,
            d.changed, d.err);
}

void launch_compact(const Dev& d, const uint8_t* mark, int clear, int32_t* rows, int32_t* count,
                    int full, int stats) {
    k_compact<<<1, kCompactThreads, 0, d.st>>>(d.n, const_cast<uint8_t*>(mark), clear, rows, count,
                                               full, stats ? d.stats : nullptr, d.err);
}

template <typename DT>
static void scan_dispatch(const Dev& d, ScanArgs<DT> a) {
    const int grid = d.nsm * 8;
    constexpr int VN = Vec<DT>::N;
    if (d.n % VN == 0)
        k_scan<DT, true><<<grid, kScanThreads, 0, d.st>>>(a);
    else
        k_scan<DT, false><<<grid, kScanThreads, 0, d.st>>>(a);
}

template <typename DT>
static ScanArgs<DT> scan_args(const Dev& d) {
    ScanArgs<DT> a;
    a.n = d.n;
    a.D = (DT*)d.D;
    a.S = d.S;
    a.rows = d.rows;
    a.count = d.counts;
    a.fD = (const DT*)d.fD;
    a.fS = d.fS;
    a.fM = d.fM;
    a.skip_row = -1;
    a.err = d.err;
    a.stats = d.stats;
    return a;
}

// IN phase: columns come from row v of the state (unchanged during this phase).
void launch_scan_in(const Dev& d, int32_t v) {
    if (d.dbytes == 4) {
        ScanArgs<int32_t> a = scan_args<int32_t>(d);
        a.cD = (const int32_t*)d.D + (size_t)v * d.n;
        a.cS = d.S + (size_t)v * d.n;
        a.cM = a.cS;
        scan_dispatch<int32_t>(d, a);
    } else {
        ScanArgs<int64_t> a = scan_args<int64_t>(d);
        a.cD = (const int64_t*)d.D + (size_t)v * d.n;
        a.cS = d.S + (size_t)v * d.n;
        a.cM = a.cS;
        scan_dispatch<int64_t>(d, a);
    }
}

// OUT phase: columns come from the new row v computed by k_alg4_out; row v itself is
// written afterwards by k_write_row.
void launch_scan_out(const Dev& d, int32_t v) {
    if (d.dbytes == 4) {
        ScanArgs<int32_t> a = scan_args<int32_t>(d);
        a.cD = (const int32_t*)d.cD;
        a.cS = d.cS;
        a.cM = d.cM;
        a.skip_row = v;
        scan_dispatch<int32_t>(d, a);
    } else {
        ScanArgs<int64_t> a = scan_args<int64_t>(d);
        a.cD = (const int64_t*)d.cD;
        a.cS = d.cS;
        a.cM = d.cM;
        a.skip_row = v;
        scan_dispatch<int64_t>(d, a);
    }
}

void launch_write_row(const Dev& d, int32_t v) {
    if (d.dbytes == 4)
        k_write_row<int32_t><<<nblk(d.n, 256), 256, 0, d.st>>>(d.n, (int32_t*)d.D, d.S, v,
                                                                (const int32_t*)d.cD, d.cS, d.err);
    else
        k_write_row<int64_t><<<nblk(d.n, 256), 256, 0, d.st>>>(d.n, (int64_t*)d.D, d.S, v,
                                                                (const int64_t*)d.cD, d.cS, d.err);
}

void launch_estar_keep(const Dev& d, uint8_t* keep) {
    if (d.e_cap <= 0) return;
    if (d.dbytes == 4)
        k_estar_keep<int32_t><<<nblk(d.e_cap, 256), 256, 0, d.st>>>(
            d.n, (const int32_t*)d.D, d.e_src, (const Arc<int32_t>*)d.e_arc, d.e_cap, keep);
    else
        k_estar_keep<int64_t><<<nblk(d.e_cap, 256), 256, 0, d.st>>>(
            d.n, (const int64_t*)d.D, d.e_src, (const Arc<int64_t>*)d.e_arc, d.e_cap, keep);
}

}  // namespace bcg
