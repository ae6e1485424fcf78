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
    pdl_enter();
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
    pdl_enter();
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
    pdl_enter();
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
    pdl_enter();
    if (*err) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) dev_rows_out<DT>(s, n, D, S, v, e, k, directed, fD, fS, fM, mark, changed, err);
}

template <typename DT>
__global__ void k_alg4_out(int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                           int v, const VEdge* __restrict__ e, int k, int directed,
                           DT* cD, uint64_t* cS, uint64_t* cM, uint8_t* changed, int32_t* err) {
    pdl_enter();
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dev_alg4_out<DT>(t, n, D, S, v, e, k, directed, cD, cS, cM, changed, err);
}

__global__ void __launch_bounds__(kCompactThreads)
k_compact(int n, uint8_t* mark, int clear, int32_t* rows, int32_t* count, int full,
          int64_t* stats, const int32_t* err) {
    pdl_enter();
    dev_compact(n, mark, clear, rows, count, full, stats, err);
}

// K2: in-place rank-1 min-plus / path-count pass over rows[0..count) x all columns.
// Work item = (row, chunk of CW columns).  Each CTA takes a contiguous block of items,
// so the per-row scalars are loaded once per row it meets; each thread issues all of
// its 16-byte loads of D and of the column vectors of an item before using any.  sigma
// is read only on ties and written only where the pair changes.
template <typename DT, bool VECTOR>
__global__ void __launch_bounds__(kScanThreads, 4) k_scan(ScanArgs<DT> a) {
    pdl_enter();
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

// K2, vector path (n a multiple of the vector width): column-stationary CTAs.  CTA b
// owns column chunk c = b mod nch (kCsThreads threads x kCsVpt 16-byte vectors) for
// the whole launch and walks the rows i = b / nch, + gridDim / nch, ... of the list.
// Its column values -- with the tie_cols bump, for the quick test -- sit in registers,
// loaded once; each thread streams its part of every row through a ring of kCsStages
// rows in shared memory filled by cp.async (16-byte copies that hold no registers
// while in flight, and that only the issuing thread reads back, so no CTA barrier is
// needed in the loop).  The rule itself runs only for the rare vectors that pass the
// quick test, with the true column values read from L2.  Changed vectors are written
// to D directly.
constexpr int kCsThreads = 256;
constexpr int kCsVpt = 4;
constexpr int kCsStages = 4;
constexpr int kCsCtasPerSm = 3;
constexpr size_t kCsRingBytes = (size_t)kCsStages * kCsVpt * kCsThreads * 16;
constexpr int kCsQueue = 32 + 32 * kCsVpt;   // a warp's candidate queue: < 32 left over plus one row

__device__ __forceinline__ void cs_copy16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global.L2::128B [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cs_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cs_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cs_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// WHOLE: n is a multiple of the chunk width, so no column of a chunk lies past n.
// DUAL: two row lists, each with its own column vector (a.rows2 set).
template <typename DT, bool WHOLE, bool DUAL>
__global__ void __launch_bounds__(kCsThreads, kCsCtasPerSm) k_scan_cs(ScanArgs<DT> a, int nch) {
    pdl_enter();
    using V = Vec<DT>;
    using VT = typename V::T;
    constexpr int VN = V::N;
    constexpr int CW = kCsThreads * kCsVpt * VN;
    constexpr int ST = kCsStages;
    extern __shared__ __align__(16) unsigned char cs_smem[];
    VT (*stage)[kCsVpt][kCsThreads] = reinterpret_cast<VT (*)[kCsVpt][kCsThreads]>(cs_smem);
    __shared__ unsigned long long s_cmax;
    if (block_err(a.err)) return;
    const int tid = threadIdx.x;
    const int n = a.n;
    const int64_t INF = Inf<DT>::v;
    int gpc = (int)gridDim.x / nch;   // CTAs per column chunk
    const int c = (int)blockIdx.x % nch;
    int r0 = (int)blockIdx.x / nch;
    int cnt = *a.count;
    bool second = false;   // this CTA works on the second list
    if (DUAL) {
        // two lists: the CTAs of a chunk are split between them in proportion to their
        // lengths (at least one each when both have rows); this CTA takes the second
        // list's column vector and rows when it falls in the second share
        const int cnt2 = *a.count2;
        int g1 = (cnt + cnt2) ? (int)(((int64_t)gpc * cnt + (cnt + cnt2) / 2) / (cnt + cnt2)) : gpc;
        if (cnt > 0 && cnt2 > 0) g1 = min(max(g1, 1), gpc - 1);
        if (blockIdx.x == 0 && tid == 0)
            atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 6), (unsigned long long)(cnt + cnt2));
        if (r0 >= g1) {
            r0 -= g1;
            gpc -= g1;
            cnt = cnt2;
            second = true;
        } else {
            gpc = g1;
        }
    } else if (blockIdx.x == 0 && tid == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 6), (unsigned long long)cnt);
    }
    if (gpc <= 0 || r0 >= gpc || r0 >= cnt) return;   // block-uniform: no rows for this CTA
    const int t0 = c * CW;
    // the column chunk: quick-test values in registers; cmax = largest finite TRUE value
    // (the bound that makes the one-compare quick test overflow-free)
    VT cq[kCsVpt];
    int64_t m = 0;
#pragma unroll
    for (int u = 0; u < kCsVpt; ++u) {
        const int t = t0 + (u * kCsThreads + tid) * VN;
        if (WHOLE || t < n) {
            VT x = __ldg(reinterpret_cast<const VT*>(((DUAL && second) ? a.cD2 : a.cD) + t));
            int64_t xv[VN];
            V::unpack(x, xv);
#pragma unroll
            for (int q = 0; q < VN; ++q) {
                if (xv[q] != INF && xv[q] > m) m = xv[q];
                if (a.tie_cols && xv[q] < INF - 1 && __ldg(((DUAL && second) ? a.cM2 : a.cM) + t + q) == 0ull) V::set(x, q, xv[q] + 1);
            }
            cq[u] = x;
        }
    }
    if (tid == 0) s_cmax = 0ull;
    __syncthreads();
    atomicMax(&s_cmax, (unsigned long long)m);
    __syncthreads();
    const int64_t cmax = (int64_t)s_cmax;
    // rows i_k = r0 + k * gpc of the list, k = 0 .. nk-1, ST of them in flight
    const int nk = (cnt - r0 + gpc - 1) / gpc;
    int n_changed = 0, n_ties = 0;
    // Row ids and per-row scalars come in batches of 32: lane j of every warp holds row
    // k0 + j of the current batch and of the next one (loaded a whole batch ahead, so
    // the issue never waits for them), and the issue takes its row's values by shuffle.
    // Per stage: the row it holds and that row's scalars (consumed ST rows later).
    const int lane = tid & 31;
    auto batch_row = [&](int k) { return k < nk ? ((DUAL && second) ? a.rows2 : a.rows)[r0 + k * gpc] : -1; };
    int cur_s = batch_row(lane), nxt_s = batch_row(32 + lane);
    DT cur_d = cur_s >= 0 ? a.fD[cur_s] : (DT)0;
    DT nxt_d = nxt_s >= 0 ? a.fD[nxt_s] : (DT)0;
    unsigned long long cur_m = (a.tie_rows && cur_s >= 0) ? a.fM[cur_s] : 1ull;
    unsigned long long nxt_m = (a.tie_rows && nxt_s >= 0) ? a.fM[nxt_s] : 1ull;
    int ring_s[ST];
    DT ring_d[ST];
    unsigned long long ring_m[ST];
    int k_issue = 0;
    auto issue = [&](int st) {
        const int j = k_issue & 31;
        if (j == 0 && k_issue > 0) {   // CTA-uniform: move to the next batch, fetch the one after
            cur_s = nxt_s;
            cur_d = nxt_d;
            cur_m = nxt_m;
            nxt_s = batch_row(k_issue + 32 + lane);
            nxt_d = nxt_s >= 0 ? a.fD[nxt_s] : (DT)0;
            nxt_m = (a.tie_rows && nxt_s >= 0) ? a.fM[nxt_s] : 1ull;
        }
        const int s = __shfl_sync(0xffffffffu, cur_s, j);
        ring_s[st] = s;
        ring_d[st] = __shfl_sync(0xffffffffu, cur_d, j);
        ring_m[st] = __shfl_sync(0xffffffffu, cur_m, j);
        if (s >= 0) {
            const DT* src = a.D + (size_t)s * n;
#pragma unroll
            for (int u = 0; u < kCsVpt; ++u) {
                const int t = t0 + (u * kCsThreads + tid) * VN;
                if (WHOLE || t < n) cs_copy16(&stage[st][u][tid], src + t);
            }
        }
        cs_commit();
        ++k_issue;
    };
    // Candidate vectors (s, t) of this warp, waiting for the rule: applying it takes a
    // few dependent memory round trips, which the 32 lanes then take together instead
    // of one candidate at a time while the warp's row stream waits.
    int2* wq = reinterpret_cast<int2*>(cs_smem + kCsRingBytes) + (tid >> 5) * kCsQueue;
    int qn = 0;   // warp-uniform
    auto run_queued = [&](int count) {
        int s = -1, t = 0;
        unsigned bits = 0;
        int64_t dold[VN];
        uint64_t sold[VN];
        if (lane < count) {
            const int2 e = wq[lane];
            s = e.x;
            t = e.y;
            const size_t rowoff = (size_t)s * n;
            const int64_t rd = (int64_t)a.fD[s];
            const uint64_t rs = a.fS[s], rm = a.fM[s];
            VT dv = *reinterpret_cast<const VT*>(a.D + rowoff + t);
            const VT cv = __ldg(reinterpret_cast<const VT*>(((DUAL && second) ? a.cD2 : a.cD) + t));
            const unsigned m = rule_vec_masked<DT>(a, second ? a.cS2 : a.cS, second ? a.cM2 : a.cM, rowoff, t, dv, cv,
                                                   rd, rs, rm, n_changed, n_ties, dold, sold);
            if (m & 0xffu) *reinterpret_cast<VT*>(a.D + rowoff + t) = dv;
            bits = (m | (m >> 8)) & 0xffu;
        }
        if (a.rec.tcnt) record_changes_warp<DT>(a.rec, n, s, t, bits, dold, sold);
    };
#pragma unroll
    for (int st = 0; st < ST; ++st) issue(st);
    for (int kb = 0; kb < nk; kb += ST) {
#pragma unroll
        for (int st = 0; st < ST; ++st) {
            if (kb + st >= nk) break;
            cs_wait<ST - 1>();
            const int s = ring_s[st];
            const int64_t rd = (s == a.skip_row) ? INF : (int64_t)ring_d[st];
            // the quick test's row term: rd + 1 where no tie of the row can add paths
            const int64_t rq = (rd < INF - 1 && ring_m[st] == 0ull) ? rd + 1 : rd;
            if (rd != INF) {
                const bool small = rd + cmax < INF;
                unsigned cand = 0;
                if (small) {
                    // no finite sum of the row reaches INF: a pair can change only if
                    // d - c >= rq, so one max over the thread's pairs decides whether
                    // any vector needs the per-vector test (d, c in [0, INF]: the
                    // differences fit DT)
                    DT mx = (DT)-Inf<DT>::v;
#pragma unroll
                    for (int u = 0; u < kCsVpt; ++u) {
                        const int t = t0 + (u * kCsThreads + tid) * VN;
                        if (WHOLE || t < n) {
                            const VT x = stage[st][u][tid];
                            const DT* xd = reinterpret_cast<const DT*>(&x);
                            const DT* cd = reinterpret_cast<const DT*>(&cq[u]);
#pragma unroll
                            for (int q = 0; q < VN; ++q) mx = max(mx, (DT)(xd[q] - cd[q]));
                        }
                    }
                    if ((int64_t)mx >= rq) {
#pragma unroll
                        for (int u = 0; u < kCsVpt; ++u) {
                            const int t = t0 + (u * kCsThreads + tid) * VN;
                            if ((WHOLE || t < n) && quick_vec<DT>(stage[st][u][tid], cq[u], rq, true)) cand |= 1u << u;
                        }
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < kCsVpt; ++u) {
                        const int t = t0 + (u * kCsThreads + tid) * VN;
                        if ((WHOLE || t < n) && quick_vec<DT>(stage[st][u][tid], cq[u], rq, false)) cand |= 1u << u;
                    }
                }
                // candidates go to the warp's queue (a row adds at most 32 x kCsVpt); the
                // rule runs 32 at a time, in one loop per row (inlined once per ring stage:
                // a flush inside the vector loop put 16 copies of the rule into the kernel,
                // too much code for the instruction cache on hub updates)
                if (__any_sync(0xffffffffu, cand != 0u)) {
#pragma unroll
                    for (int u = 0; u < kCsVpt; ++u) {
                        const bool mine = (cand >> u) & 1u;
                        const unsigned b = __ballot_sync(0xffffffffu, mine);
                        if (mine)
                            wq[qn + __popc(b & ((1u << lane) - 1u))] =
                                make_int2(s, t0 + (u * kCsThreads + tid) * VN);
                        qn += __popc(b);
                    }
                    while (qn >= 32) {
                        __syncwarp();
                        run_queued(32);
                        __syncwarp();
                        for (int i = lane; i < qn - 32; i += 32) wq[i] = wq[32 + i];
                        qn -= 32;
                        __syncwarp();
                    }
                }
            }
            // refill the stage just read with the row ST ahead (this thread's reads of
            // it are complete: their values were used above)
            issue(st);
        }
    }
    cs_wait_all();
    __syncwarp();
    run_queued(qn);
    scan_stats(a.stats, n_changed, n_ties);
}

template <typename DT>
__global__ void k_write_row(int n, DT* D, uint64_t* S, int v, const DT* cD, const uint64_t* cS, PairRec rec,
                            const int32_t* err) {
    pdl_enter();
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
    pdl_enter();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cap) return;
    const Arc<DT> a = e_arc[e];
    keep[e] = (a.dst >= 0 && (int64_t)D[(size_t)e_src[e] * n + a.dst] == (int64_t)a.w) ? 1 : 0;
}

// Fused pass of an undirected edge update {u, v} with weight w, preparation (one thread
// per row s): snapshot rows u and v of the state before the update (the column vectors
// of the pass; in G_D row x holds d(x, .) = d(., x), so position s of rows u and v also
// gives d(s,u) and d(s,v)), and put row s on one of two lists by the direction in which
// a new shortest path would use the edge:
//   list 1 (s ~> u -> v):  d(s,u) + w <= d(s,v);   list 2 (s ~> v -> u):  d(s,v) + w <= d(s,u).
// No row is on both (that would need 2w <= 0).  Per row it writes what Algorithm 4 with
// the one in-edge gives for the row's direction: the distance through the edge, the
// path count to the far endpoint and the tie multiplier (Lemma 2: on a tie only the new
// paths are added).  A shortest simple path uses the edge in at most one direction, and
// a candidate whose prefix already used the edge the other way is longer than d(s,t),
// so one pass with both candidates taken from the old state gives the two directed
// passes' d and sigma.  Rows are appended with one atomic per warp and list (the counts
// start at zero); the order of a list does not affect any result.
template <typename DT>
__global__ void k_edge_prep(int n, const DT* D, const uint64_t* S, int u, int v, int64_t w, DT* cDv,
                            uint64_t* cSv, DT* cDu, uint64_t* cSu, DT* fD, uint64_t* fS, uint64_t* fM,
                            int32_t* rows1, int32_t* count1, int32_t* rows2, int32_t* count2,
                            uint8_t* changed, int32_t* err) {
    pdl_enter();
    if (*reinterpret_cast<const volatile int32_t*>(err)) return;   // grid-uniform for this launch
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int64_t INF = Inf<DT>::v;
    bool in1 = false, in2 = false;
    if (s < n) {
        const int64_t du = D[(size_t)u * n + s], dv = D[(size_t)v * n + s];
        const uint64_t su = S[(size_t)u * n + s], sv = S[(size_t)v * n + s];
        cDu[s] = (DT)du;
        cSu[s] = su;
        cDv[s] = (DT)dv;
        cSv[s] = sv;
        int64_t rd = 0;
        uint64_t rs = 0, rm = 0;
        if (du != INF) {
            const int64_t c = dsum<DT>(du, w);
            if (c == SAT) {
                if (dv == INF) set_err(err, ERRF_DIST);
            } else if (c < dv) {
                in1 = true; rd = c; rs = su; rm = su;
            } else if (c == dv) {
                in1 = true; rd = c; rs = add_chk(sv, su, err); rm = su;
            }
        }
        if (!in1 && dv != INF) {
            const int64_t c = dsum<DT>(dv, w);
            if (c == SAT) {
                if (du == INF) set_err(err, ERRF_DIST);
            } else if (c < du) {
                in2 = true; rd = c; rs = sv; rm = sv;
            } else if (c == du) {
                in2 = true; rd = c; rs = add_chk(su, sv, err); rm = sv;
            }
        }
        if (in1 || in2) {
            fD[s] = (DT)rd;
            fS[s] = rs;
            fM[s] = rm;
            changed[s] = 1;
        }
    }
    const unsigned b1 = __ballot_sync(0xffffffffu, in1), b2 = __ballot_sync(0xffffffffu, in2);
    int p1 = 0, p2 = 0;
    if (lane == 0) {
        if (b1) p1 = atomicAdd(count1, __popc(b1));
        if (b2) p2 = atomicAdd(count2, __popc(b2));
    }
    p1 = __shfl_sync(0xffffffffu, p1, 0);
    p2 = __shfl_sync(0xffffffffu, p2, 0);
    const unsigned lt = (1u << lane) - 1u;
    if (in1) rows1[p1 + __popc(b1 & lt)] = s;
    if (in2) rows2[p2 + __popc(b2 & lt)] = s;
}

// ------------------------------------------------------------------ launches

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

void launch_estar_write(const Dev& d, const EOps& ops) {
    if (ops.count <= 0) return;
    launch_k(k_estar_write, 1, kMaxEOps, 0, d.st, d.e_src, d.e_arc, d.e_len, d.dbytes, ops);
}

void launch_estar_move(const Dev& d, const EMoves& moves) {
    if (moves.count <= 0) return;
    if (d.dbytes == 4)
        launch_k(k_estar_move<int32_t>, moves.count, 128, 0, d.st, d.e_off, d.e_src, (Arc<int32_t>*)d.e_arc, moves);
    else
        launch_k(k_estar_move<int64_t>, moves.count, 128, 0, d.st, d.e_off, d.e_src, (Arc<int64_t>*)d.e_arc, moves);
}

void launch_alg4_in(const Dev& d, int32_t v, const VEdge* e, int32_t k) {
    if (d.dbytes == 4)
        launch_k(k_alg4_in<int32_t>, nblk(d.n, 256), 256, 0, d.st, d.n, (const int32_t*)d.D, d.S, v, e, k, d.directed, (int32_t*)d.fD, d.fS, d.fM,
            d.mark, d.changed, d.err);
    else
        launch_k(k_alg4_in<int64_t>, nblk(d.n, 256), 256, 0, d.st, d.n, (const int64_t*)d.D, d.S, v, e, k, d.directed, (int64_t*)d.fD, d.fS, d.fM,
            d.mark, d.changed, d.err);
}

void launch_rows_out(const Dev& d, int32_t v, const VEdge* e, int32_t k) {
    if (d.dbytes == 4)
        launch_k(k_rows_out<int32_t>, nblk(d.n, 256), 256, 0, d.st, d.n, (const int32_t*)d.D, d.S, v, e, k, d.directed, (int32_t*)d.fD, d.fS, d.fM,
            d.mark, d.changed, d.err);
    else
        launch_k(k_rows_out<int64_t>, nblk(d.n, 256), 256, 0, d.st, d.n, (const int64_t*)d.D, d.S, v, e, k, d.directed, (int64_t*)d.fD, d.fS, d.fM,
            d.mark, d.changed, d.err);
}

void launch_alg4_out(const Dev& d, int32_t v, const VEdge* e, int32_t k) {
    if (d.dbytes == 4)
        launch_k(k_alg4_out<int32_t>, nblk(d.n, 256), 256, 0, d.st, d.n, (const int32_t*)d.D, d.S, v, e, k, d.directed, (int32_t*)d.cD, d.cS, d.cM,
            d.changed, d.err);
    else
        launch_k(k_alg4_out<int64_t>, nblk(d.n, 256), 256, 0, d.st, d.n, (const int64_t*)d.D, d.S, v, e, k, d.directed, (int64_t*)d.cD, d.cS, d.cM,
            d.changed, d.err);
}

void launch_compact(const Dev& d, const uint8_t* mark, int clear, int32_t* rows, int32_t* count,
                    int full, int stats) {
    launch_k(k_compact, 1, kCompactThreads, 0, d.st, d.n, const_cast<uint8_t*>(mark), clear, rows, count,
                                               full, stats ? d.stats : nullptr, d.err);
}

// Dynamic shared memory of k_scan_cs: its ring of kCsStages row chunks, then a queue
// of kCsQueue candidate vectors per warp.
constexpr size_t kCsSmem = kCsRingBytes + (size_t)(kCsThreads / 32) * kCsQueue * sizeof(int2);

// Allows the vector-path kernels their shared memory on the current device.
cudaError_t scan_setup() {
    const int b = (int)kCsSmem;
    const void* fns[] = {(const void*)k_scan_cs<int32_t, true, false>, (const void*)k_scan_cs<int32_t, false, false>,
                         (const void*)k_scan_cs<int64_t, true, false>, (const void*)k_scan_cs<int64_t, false, false>,
                         (const void*)k_scan_cs<int32_t, true, true>,  (const void*)k_scan_cs<int32_t, false, true>,
                         (const void*)k_scan_cs<int64_t, true, true>,  (const void*)k_scan_cs<int64_t, false, true>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename DT>
static void scan_dispatch(const Dev& d, ScanArgs<DT> a) {
    constexpr int VN = Vec<DT>::N;
    if (d.n % VN == 0) {
        constexpr int CW = kCsThreads * kCsVpt * VN;
        const int nch = (d.n + CW - 1) / CW;
        const int per = std::max(1, d.nsm * kCsCtasPerSm / nch);
        const bool whole = d.n % CW == 0;
        if (a.rows2) {
            if (whole) launch_k(k_scan_cs<DT, true, true>, nch * per, kCsThreads, kCsSmem, d.st, a, nch);
            else launch_k(k_scan_cs<DT, false, true>, nch * per, kCsThreads, kCsSmem, d.st, a, nch);
        } else {
            if (whole) launch_k(k_scan_cs<DT, true, false>, nch * per, kCsThreads, kCsSmem, d.st, a, nch);
            else launch_k(k_scan_cs<DT, false, false>, nch * per, kCsThreads, kCsSmem, d.st, a, nch);
        }
    } else {
        launch_k(k_scan<DT, false>, d.nsm * 8, kScanThreads, 0, d.st, a);
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
    a.tie_rows = 0;
    a.tie_cols = 0;
    a.rows2 = nullptr;
    a.count2 = nullptr;
    a.cD2 = nullptr;
    a.cS2 = a.cM2 = nullptr;
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
        a.tie_rows = 1;
        a.cD = (const int32_t*)d.D + (size_t)v * d.n;
        a.cS = d.S + (size_t)v * d.n;
        a.cM = a.cS;
        scan_dispatch<int32_t>(d, a);
    } else {
        ScanArgs<int64_t> a = scan_args<int64_t>(d);
        a.rec.first = 1;
        a.tie_rows = 1;
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
        a.tie_cols = 1;
        scan_dispatch<int32_t>(d, a);
    } else {
        ScanArgs<int64_t> a = scan_args<int64_t>(d);
        a.cD = (const int64_t*)d.cD;
        a.cS = d.cS;
        a.cM = d.cM;
        a.skip_row = v;
        a.tie_cols = 1;
        scan_dispatch<int64_t>(d, a);
    }
}

// Row v is never written before this in an update (Lemma 1 in the IN phase; the OUT
// phase's pass skips it), so its changes are first changes.
void launch_write_row(const Dev& d, int32_t v) {
    PairRec rec = d.pair_on ? pair_rec(d) : PairRec{};
    rec.first = 1;
    if (d.dbytes == 4)
        launch_k(k_write_row<int32_t>, nblk(d.n, 256), 256, 0, d.st, d.n, (int32_t*)d.D, d.S, v,
                                                                (const int32_t*)d.cD, d.cS, rec, d.err);
    else
        launch_k(k_write_row<int64_t>, nblk(d.n, 256), 256, 0, d.st, d.n, (int64_t*)d.D, d.S, v,
                                                                (const int64_t*)d.cD, d.cS, rec, d.err);
}

// The fused pass of an undirected edge update {u, v} with weight w: the row lists and
// column snapshots (k_edge_prep), then one rank-1 pass over both lists, each against its
// own column vector, every change a first change of the update.  List 1 goes to rows /
// counts[0] against row v; list 2 to acc_rows / counts[2] (free until the pair lists are
// built after the pass) against row u.
void launch_edge_prep(const Dev& d, int32_t u, int32_t v, int64_t w) {
    cudaMemsetAsync(d.counts, 0, 3 * sizeof(int32_t), d.st);   // counts[0..2]; [1] is rewritten later
    const int grid = (d.n + 255) / 256;
    if (d.dbytes == 4)
        launch_k(k_edge_prep<int32_t>, grid, 256, 0, d.st, d.n, (const int32_t*)d.D, d.S, u, v, w, (int32_t*)d.cD, d.cS, (int32_t*)d.cD2, d.cS2, (int32_t*)d.fD,
            d.fS, d.fM, d.rows, d.counts, d.acc_rows, d.counts + 2, d.changed, d.err);
    else
        launch_k(k_edge_prep<int64_t>, grid, 256, 0, d.st, d.n, (const int64_t*)d.D, d.S, u, v, w, (int64_t*)d.cD, d.cS, (int64_t*)d.cD2, d.cS2, (int64_t*)d.fD,
            d.fS, d.fM, d.rows, d.counts, d.acc_rows, d.counts + 2, d.changed, d.err);
}

template <typename DT>
static void edge_scan(const Dev& d) {
    ScanArgs<DT> a = scan_args<DT>(d);
    a.rec.first = 1;
    a.tie_rows = 1;
    a.cD = (const DT*)d.cD;
    a.cS = d.cS;
    a.cM = d.cS;
    a.rows2 = d.acc_rows;
    a.count2 = d.counts + 2;
    a.cD2 = (const DT*)d.cD2;
    a.cS2 = d.cS2;
    a.cM2 = d.cS2;
    scan_dispatch<DT>(d, a);
}

void launch_edge_scan(const Dev& d) {
    if (d.dbytes == 4) edge_scan<int32_t>(d);
    else edge_scan<int64_t>(d);
}

void launch_estar_keep(const Dev& d, uint8_t* keep) {
    if (d.e_cap <= 0) return;
    if (d.dbytes == 4)
        launch_k(k_estar_keep<int32_t>, nblk(d.e_cap, 256), 256, 0, d.st, d.n, (const int32_t*)d.D, d.e_src, (const Arc<int32_t>*)d.e_arc, d.e_cap, keep);
    else
        launch_k(k_estar_keep<int64_t>, nblk(d.e_cap, 256), 256, 0, d.st, d.n, (const int64_t*)d.D, d.e_src, (const Arc<int64_t>*)d.e_arc, d.e_cap, keep);
}

}  // namespace bcg
