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
#include "bc_device.cuh"

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

// One CTA per move: copy the segment, empty its old slots, point e_off[a] at the copy.
// Source and destination ranges of all moves are disjoint.
template <typename DT>
__global__ void k_estar_move(int32_t* e_off, int32_t* e_src, Arc<DT>* e_arc, EMoves moves) {
    if ((int)blockIdx.x >= moves.count) return;
    const EMove m = moves.mv[blockIdx.x];
    for (int i = threadIdx.x; i < m.len; i += blockDim.x) {
        e_arc[m.to + i] = e_arc[m.from + i];
        e_src[m.to + i] = m.a;
        e_arc[m.from + i].dst = -1;
    }
    if (threadIdx.x == 0) e_off[m.a] = m.to;
}

template <typename DT>
__global__ void k_alg4_in(int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                          int v, const VEdge* __restrict__ e, int k, int directed,
                          DT* fD, uint64_t* fS, uint64_t* fM, uint8_t* mark, uint8_t* changed,
                          int32_t* err) {
    if (*err) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    if (directed) dev_alg4_in<DT, false>(s, n, D, S, v, e, k, directed, fD, fS, fM, mark, changed, err);
    else dev_alg4_in<DT, true>(s, n, D, S, v, e, k, directed, fD, fS, fM, mark, changed, err);
}

template <typename DT>
__global__ void k_rows_out(int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                           int v, const VEdge* __restrict__ e, int k, int directed,
                           DT* fD, uint64_t* fS, uint64_t* fM, uint8_t* mark, uint8_t* changed,
                           int32_t* err) {
    if (*err) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) dev_rows_out<DT>(s, n, D, S, v, e, k, directed, fD, fS, fM, mark, changed, err);
}

template <typename DT>
__global__ void k_alg4_out(int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                           int v, const VEdge* __restrict__ e, int k, int directed,
                           DT* cD, uint64_t* cS, uint64_t* cM, uint8_t* changed, int32_t* err) {
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dev_alg4_out<DT>(t, n, D, S, v, e, k, directed, cD, cS, cM, changed, err);
}

__global__ void __launch_bounds__(kCompactThreads)
k_compact(int n, uint8_t* mark, int clear, int32_t* rows, int32_t* count, int full,
          int64_t* stats, const int32_t* err) {
    dev_compact(n, mark, clear, rows, count, full, stats, err);
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
    constexpr int CW = kScanThreads * Vec<DT>::N * kScanUnroll;
    const int nchunks = (a.n + CW - 1) / CW;
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
        dev_scan_item<DT, VECTOR>(a, s, rd, rs, rm, c, n_changed, n_ties);
    }
    scan_stats(a.stats, n_changed, n_ties);
}

// Row v <- the OUT phase's result; with rec.tcnt set, the pairs (v,t) whose distance or
// path count changes are recorded.
// K2, vector path (n a multiple of the vector width).  Work item = (chunk c of CW
// columns, row i) in chunk-major order, so the column vector of a chunk is staged in
// shared memory (with its largest finite value) once for all the rows a CTA meets in
// that chunk; CTAs take items in turn.  Each thread issues the kScanVecs 16-byte loads
// of its part of the row chunk before using any (the row of the next item is fetched a
// step ahead, so these loads do not wait for it), then applies the quick test of the
// rule to every vector and the rule itself (scan_vec) to the rare vectors that can
// change.  Changed vectors are written back to D.  (Measured alternatives: a bulk-copy
// (TMA) pipeline with 2-6 stages of 16 KB per CTA and a contiguous block of items per
// CTA were both slower on this pass.)
constexpr int kScanVecs = 8;
constexpr int kScanCtasPerSm = 4;

template <typename DT>
__global__ void __launch_bounds__(kScanThreads, kScanCtasPerSm) k_scan_cm(ScanArgs<DT> a) {
    using V = Vec<DT>;
    constexpr int VN = V::N;
    constexpr int CW = kScanThreads * VN * kScanVecs;
    extern __shared__ __align__(16) unsigned char smem[];
    DT* scd = reinterpret_cast<DT*>(smem);   // CW column values
    if (block_err(a.err)) return;
    const int tid = threadIdx.x;
    const int n = a.n;
    const int64_t INF = Inf<DT>::v;
    const int cnt = *a.count;
    const int nchunks = (n + CW - 1) / CW;
    const int total = cnt * nchunks;   // at most 32768 rows x 16 chunks
    if (blockIdx.x == 0 && tid == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 6), (unsigned long long)cnt);
    int n_changed = 0, n_ties = 0;
    {
        // CTAs take items in turn (item = block + k * grid): at any moment the CTAs
        // read neighbouring rows, which keeps the DRAM accesses of the whole grid local
        __shared__ int64_t s_cmax;
        int64_t cmax = 0;
        int cur_c = -1;
        int item = blockIdx.x;
        // the row of an item is fetched two items ahead and its distance to v one item
        // ahead, so neither the loads of D nor the distance load wait for a load issued
        // in the same item
        auto rd_of = [&](int r) { return (r == a.skip_row) ? INF : (int64_t)a.fD[r]; };
        auto row_of = [&](int it) { return it < total ? a.rows[it - (it / cnt) * cnt] : 0; };
        int s_next = row_of(item);
        int64_t rd_next = item < total ? rd_of(s_next) : INF;
        int s_next2 = row_of(item + (int)gridDim.x);
        for (; item < total; item += gridDim.x) {
            const int c = item / cnt;
            const int t0 = c * CW;
            const int s = s_next;
            const int64_t rd = rd_next;
            if (item + (int)gridDim.x < total) {
                s_next = s_next2;
                rd_next = rd_of(s_next);
                s_next2 = row_of(item + 2 * (int)gridDim.x);
            }
            if (c != cur_c) {   // block-uniform: stage the column chunk and its largest finite value
                cur_c = c;
                __syncthreads();   // the previous chunk is no longer read
                if (tid == 0) s_cmax = 0;
                __syncthreads();
                int64_t m = 0;
#pragma unroll
                for (int u = 0; u < kScanVecs; ++u) {
                    const int j = (u * kScanThreads + tid) * VN;
                    if (t0 + j < n) {
                        const typename V::T x = __ldg(reinterpret_cast<const typename V::T*>(a.cD + t0 + j));
                        *reinterpret_cast<typename V::T*>(scd + j) = x;
                        int64_t xv[VN];
                        V::unpack(x, xv);
#pragma unroll
                        for (int q = 0; q < VN; ++q)
                            if (xv[q] != INF && xv[q] > m) m = xv[q];
                    }
                }
                atomicMax(reinterpret_cast<unsigned long long*>(&s_cmax), (unsigned long long)m);
                __syncthreads();
                cmax = s_cmax;
            }
            if (rd != INF) {
                const size_t rowoff = (size_t)s * n;
                DT* Drow = a.D + rowoff;
                typename V::T dv[kScanVecs];
#pragma unroll
                for (int u = 0; u < kScanVecs; ++u) {
                    const int t = t0 + (u * kScanThreads + tid) * VN;
                    if (t < n) dv[u] = __ldcs(reinterpret_cast<const typename V::T*>(Drow + t));
                }
                // quick test of every vector first; the rare vectors that can change are
                // read again (from cache) by a loop that is not unrolled, so the rule's
                // code does not hold the registers of all kScanVecs vectors.  When no
                // finite sum of the row can exceed a finite distance bound (rd + the
                // chunk's largest finite column value < INF), the test is one add and
                // compare per pair.
                const bool small = rd + cmax < INF;
                unsigned cand = 0;
#pragma unroll
                for (int u = 0; u < kScanVecs; ++u) {
                    const int j = (u * kScanThreads + tid) * VN;
                    if (t0 + j >= n) break;
                    const typename V::T cv = *reinterpret_cast<const typename V::T*>(scd + j);
                    if (quick_vec<DT>(dv[u], cv, rd, small)) cand |= 1u << u;
                }
                if (cand) {
                    const uint64_t rs = a.fS[s], rm = a.fM[s];
                    while (cand) {
                        const int u = __ffs(cand) - 1;
                        cand &= cand - 1;
                        const int j = (u * kScanThreads + tid) * VN;
                        const int t = t0 + j;
                        typename V::T d1 = *reinterpret_cast<const typename V::T*>(Drow + t);
                        const typename V::T cv = *reinterpret_cast<const typename V::T*>(scd + j);
                        if (rule_vec<DT>(a, s, rowoff, t, d1, cv, rd, rs, rm, n_changed, n_ties))
                            *reinterpret_cast<typename V::T*>(Drow + t) = d1;
                    }
                }
            }
        }
    }
    scan_stats(a.stats, n_changed, n_ties);
}

template <typename DT>
__global__ void k_write_row(int n, DT* D, uint64_t* S, int v, const DT* cD, const uint64_t* cS, PairRec rec,
                            const int32_t* err) {
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (rec.tcnt) {
        const size_t i = (size_t)v * n + t;
        if (D[i] != cD[t] || S[i] != cS[t]) record_change<DT>(rec, n, v, t, D[i], S[i]);
    }
    dev_write_row<DT>(t, n, D, S, v, cD, cS, err);
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

void launch_estar_move(const Dev& d, const EMoves& moves) {
    if (moves.count <= 0) return;
    if (d.dbytes == 4)
        k_estar_move<int32_t><<<moves.count, 128, 0, d.st>>>(d.e_off, d.e_src, (Arc<int32_t>*)d.e_arc, moves);
    else
        k_estar_move<int64_t><<<moves.count, 128, 0, d.st>>>(d.e_off, d.e_src, (Arc<int64_t>*)d.e_arc, moves);
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

// Dynamic shared memory of k_scan_cm: one chunk of the column vector.
template <typename DT>
static constexpr size_t scan_cm_smem() {
    return (size_t)kScanThreads * Vec<DT>::N * kScanVecs * sizeof(DT);
}

// Allows the vector-path kernels their shared memory on the current device.
cudaError_t scan_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_scan_cm<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)scan_cm_smem<int32_t>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_scan_cm<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)scan_cm_smem<int64_t>());
    return e;
}

template <typename DT>
static void scan_dispatch(const Dev& d, ScanArgs<DT> a) {
    constexpr int VN = Vec<DT>::N;
    if (d.n % VN == 0) {
        k_scan_cm<DT><<<d.nsm * kScanCtasPerSm, kScanThreads, scan_cm_smem<DT>(), d.st>>>(a);
    } else {
        k_scan<DT, false><<<d.nsm * 8, kScanThreads, 0, d.st>>>(a);
    }
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
    a.rec = d.pair_on ? pair_rec(d) : PairRec{};
    return a;
}

// IN phase: columns come from row v of the state (unchanged during this phase).  It is
// the first pass of an update that writes pairs.
void launch_scan_in(const Dev& d, int32_t v) {
    if (d.dbytes == 4) {
        ScanArgs<int32_t> a = scan_args<int32_t>(d);
        a.rec.first = 1;
        a.cD = (const int32_t*)d.D + (size_t)v * d.n;
        a.cS = d.S + (size_t)v * d.n;
        a.cM = a.cS;
        scan_dispatch<int32_t>(d, a);
    } else {
        ScanArgs<int64_t> a = scan_args<int64_t>(d);
        a.rec.first = 1;
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

// Row v is never written before this in an update (Lemma 1 in the IN phase; the OUT
// phase's pass skips it), so its changes are first changes.
void launch_write_row(const Dev& d, int32_t v) {
    PairRec rec = d.pair_on ? pair_rec(d) : PairRec{};
    rec.first = 1;
    if (d.dbytes == 4)
        k_write_row<int32_t><<<nblk(d.n, 256), 256, 0, d.st>>>(d.n, (int32_t*)d.D, d.S, v,
                                                                (const int32_t*)d.cD, d.cS, rec, d.err);
    else
        k_write_row<int64_t><<<nblk(d.n, 256), 256, 0, d.st>>>(d.n, (int64_t*)d.D, d.S, v,
                                                                (const int64_t*)d.cD, d.cS, rec, d.err);
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
