// bc_device.cuh -- device functions shared by the single-graph kernels and the batched
// (many graphs per launch) kernels, so that both run the same arithmetic and give
// bit-identical results.  What each function computes is described at its definition;
// the translation units that launch them describe the method (k_update.cu: the
// all-pairs passes; k_accum.cu: the dependency accumulation and BC).
#pragma once

#include "bc_internal.cuh"

namespace bcg {

// Algorithm 4 (Compute-Dist-to-v) for source s = this thread, over the in-edges
// (x_j, v) of the update, followed by the affected-row test of the IN phase: row s can
// change only if d'(s,v) < d(s,v) or new shortest paths reach v (sigma-hat > 0).
// SYM: the graph is undirected and the state is the one before the update, whose d and
// sigma are symmetric, so d(s,x) is read as d(x,s) (consecutive threads then read
// consecutive entries of row x instead of one entry of each row).
template <typename DT, bool SYM = false>
__device__ __forceinline__ void dev_alg4_in(int s, int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                          int v, const VEdge* __restrict__ e, int k, int directed,
                          DT* fD, uint64_t* fS, uint64_t* fM, uint8_t* mark, uint8_t* changed,
                          int32_t* err) {
    const int64_t INF = Inf<DT>::v;
    const size_t rs = (size_t)s * n;
    auto at = [&](int x) { return SYM ? (size_t)x * n + s : rs + x; };
    const int64_t old = D[at(v)];
    int64_t cur = old;
    uint64_t sig = S[at(v)];
    uint64_t hat = 0;
    bool sat = false;
    for (int j = 0; j < k; ++j) {
        const VEdge ed = e[j];
        if (directed && ed.dir != 0) continue;
        const int64_t dx = D[at(ed.x)];
        if (dx == INF) continue;
        const int64_t dj = dsum<DT>(dx, ed.w);
        if (dj == SAT) {
            sat = true;
            continue;
        }
        const uint64_t sx = S[at(ed.x)];
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
__device__ __forceinline__ void dev_rows_out(int s, int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                           int v, const VEdge* __restrict__ e, int k, int directed,
                           DT* fD, uint64_t* fS, uint64_t* fM, uint8_t* mark, uint8_t* changed,
                           int32_t* err) {
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
__device__ __forceinline__ void dev_alg4_out(int t, int n, const DT* __restrict__ D, const uint64_t* __restrict__ S,
                           int v, const VEdge* __restrict__ e, int k, int directed,
                           DT* cD, uint64_t* cS, uint64_t* cM, uint8_t* changed, int32_t* err) {
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
// Optionally clears mark[] and accumulates the per-update counters.  A thread takes 16
// consecutive flags per tile (one 16-byte load where aligned), so n = 16384 is one tile:
// one block scan instead of one per 1024 flags.
constexpr int kCompactThreads = 1024;
constexpr int kCompactPerThread = 16;
// Every thread of the block calls it; blockDim.x is a multiple of 32 (at most 1024).
__device__ __forceinline__ void dev_compact(int n, uint8_t* mark, int clear, int32_t* rows, int32_t* count,
                                            int full, int64_t* stats, const int32_t* err) {
    constexpr int E = kCompactPerThread;
    __shared__ int32_t wsum[32];
    __shared__ int32_t s_total;
    const int nwarps = blockDim.x >> 5;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool bad = *err != 0;
    int base = 0;
    for (int tile = 0; tile < n; tile += (int)blockDim.x * E) {
        const int s0 = tile + tid * E;
        uint32_t fl = 0;   // bit e: flag of s0 + e
        if (s0 < n) {
            const bool vec = s0 + E <= n && ((reinterpret_cast<uintptr_t>(mark + s0) & 15) == 0);
            if (vec) {
                const uint4 v = *reinterpret_cast<const uint4*>(mark + s0);
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if ((w[e >> 2] >> (8 * (e & 3))) & 0xFFu) fl |= 1u << e;
                if (clear) *reinterpret_cast<uint4*>(mark + s0) = make_uint4(0u, 0u, 0u, 0u);
            } else {
                for (int e = 0; e < E && s0 + e < n; ++e) {
                    if (mark[s0 + e]) fl |= 1u << e;
                    if (clear) mark[s0 + e] = 0;
                }
            }
            if (full) fl = (s0 + E <= n) ? 0xFFFFu : ((1u << (n - s0)) - 1u);
            if (bad) fl = 0;
        }
        const int c = __popc(fl);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int x = lane < nwarps ? wsum[lane] : 0;
            int winc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, winc, o);
                if (lane >= o) winc += y;
            }
            if (lane < nwarps) wsum[lane] = winc - x;
            if (lane == 31) s_total = winc;
        }
        __syncthreads();
        int pos = base + wsum[wid] + incl - c;
        while (fl) {
            const int e = __ffs(fl) - 1;
            fl &= fl - 1;
            rows[pos++] = s0 + e;
        }
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
    // Ties with a zero tie multiplier add no paths (sigma += rowM * colM = 0), so for
    // integer distances such a pair can change only if cand < d, i.e. cand + 1 <= d.
    // tie_rows: rows with rowM = 0 take the quick test with rd + 1 (the IN phase, where
    // every finite column has colM = sigma(v,t) > 0);  tie_cols: columns with colM = 0
    // are staged as c + 1 (the OUT phase, where every finite row has rowM = sigma(s,v)
    // > 0).  Never both in one pass: cand + 2 <= d would miss an improvement by one.
    int tie_rows;
    int tie_cols;
    int32_t* err;
    int64_t* stats;        // [4] pairs with a lower distance [5] pairs with new tied paths [6] rows
    PairRec rec;           // when rec.tcnt is set: record the changed pairs (pair corrections)
    // Second row list with its own column vector (the fused pass of an undirected edge
    // update: the rows whose new paths use the edge as v -> u); rows2 = NULL: one list.
    const int32_t* rows2;
    const int32_t* count2;
    const DT* cD2;
    const uint64_t* cS2;
    const uint64_t* cM2;
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

// Quick test of the rank-1 rule on VN consecutive pairs (s, t .. t+VN-1) of row s with
// distances dv and column distances cv: can any of them change?  (False positives only
// cost time: scan_vec applies the exact rule.)
// small: rd plus every finite column value stays below INF, so no finite sum can
// overflow and a pair with d = INF and an INF column term cannot pass.
template <typename DT>
__device__ __forceinline__ bool quick_vec(const typename Vec<DT>::T& dv, const typename Vec<DT>::T& cv, int64_t rd,
                                          bool small = false) {
    using V = Vec<DT>;
    constexpr int VN = V::N;
    const int64_t INF = Inf<DT>::v;
    bool any = false;
    if constexpr (sizeof(DT) == 4) {
        // both terms are below 2^31, so their sum fits 32 bits: a pair can change only if
        // the sum does not exceed d (or d is INF, where a sum that does not fit must be
        // reported).  An INF column term passes only where d is INF or rd is 0; the rule
        // skips it.
        const uint32_t r32 = (uint32_t)rd;
        const int32_t* dp = reinterpret_cast<const int32_t*>(&dv);
        const int32_t* cp = reinterpret_cast<const int32_t*>(&cv);
        if (small) {
#pragma unroll
            for (int q = 0; q < VN; ++q) any |= r32 + (uint32_t)cp[q] <= (uint32_t)dp[q];
        } else {
#pragma unroll
            for (int q = 0; q < VN; ++q) {
                const uint32_t sum = r32 + (uint32_t)cp[q];
                any |= (sum <= (uint32_t)dp[q]) | (dp[q] == INT32_MAX);
            }
        }
    } else {
        int64_t dd0[VN], cd0[VN];
        V::unpack(dv, dd0);
        V::unpack(cv, cd0);
#pragma unroll
        for (int q = 0; q < VN; ++q) {
            if (cd0[q] == INF) continue;
            const int64_t cand = dsum<DT>(rd, cd0[q]);
            any |= (cand <= dd0[q]) || (cand == SAT);
        }
    }
    return any;
}

// The rank-1 rule on the VN consecutive pairs (s, t .. t+VN-1) of row s, given their
// distances dv (updated in place) and the column distances cv; sigma is read only on
// ties and written only where the pair changes.  Returns whether a distance changed
// (dv must then be written back).
template <typename DT>
__device__ __forceinline__ bool rule_vec(const ScanArgs<DT>& a, int s, size_t rowoff, int t, typename Vec<DT>::T& dv,
                                         const typename Vec<DT>::T& cv, int64_t rd, uint64_t rs, uint64_t rm,
                                         int& n_changed, int& n_ties) {
    using V = Vec<DT>;
    constexpr int VN = V::N;
    const int64_t INF = Inf<DT>::v;
    int64_t dd[VN], cd[VN];
    V::unpack(dv, dd);
    V::unpack(cv, cd);
    bool wr = false;
#pragma unroll
    for (int q = 0; q < VN; ++q) {
        if (cd[q] == INF) continue;
        const int64_t cand = dsum<DT>(rd, cd[q]);
        int64_t nd;
        const int ties0 = n_ties;
        const uint64_t sig0 = a.rec.tcnt ? a.S[rowoff + t + q] : 0ull;
        if (pair_rule<DT>(cand, dd[q], rowoff + t + q, rs, rm, a.cS[t + q], a.cM[t + q], a.S, a.err, &nd,
                          &n_ties)) {
            V::set(dv, q, nd);
            wr = true;
            ++n_changed;
            if (a.rec.tcnt) record_change<DT>(a.rec, a.n, s, t + q, dd[q], sig0);
        } else if (n_ties != ties0 && a.rec.tcnt) {
            record_change<DT>(a.rec, a.n, s, t + q, dd[q], sig0);
        }
    }
    return wr;
}

// VN consecutive path counts from a 16-byte aligned address, in 16-byte loads.
template <int VN>
__device__ __forceinline__ void load_u64s(const uint64_t* p, uint64_t* o) {
#pragma unroll
    for (int h = 0; h < VN / 2; ++h) {
        const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(p + 2 * h);
        o[2 * h] = x.x;
        o[2 * h + 1] = x.y;
    }
}

// The rank-1 rule on a vector like rule_vec, recording nothing: returns the mask of
// pairs q whose distance dropped (bits 0..7) or that gained paths at the same distance
// (bits 8..15), with their values before the rule in dold / sold, for a caller that
// records the changes of a whole warp together.  The vector's path counts and the
// column's counts and multipliers are loaded together (16-byte loads: t is a multiple
// of VN and so is n), and the changed counts written back together, so a vector costs
// one round trip to memory instead of one per pair.
template <typename DT>
__device__ __forceinline__ unsigned rule_vec_masked(const ScanArgs<DT>& a, const uint64_t* colS,
                                                    const uint64_t* colM, size_t rowoff, int t,
                                                    typename Vec<DT>::T& dv, const typename Vec<DT>::T& cv,
                                                    int64_t rd, uint64_t rs, uint64_t rm, int& n_changed,
                                                    int& n_ties, int64_t* dold, uint64_t* sold) {
    using V = Vec<DT>;
    constexpr int VN = V::N;
    const int64_t INF = Inf<DT>::v;
    int64_t dd[VN], cd[VN];
    uint64_t sg[VN], cs[VN], cm[VN];
    V::unpack(dv, dd);
    V::unpack(cv, cd);
    load_u64s<VN>(a.S + rowoff + t, sg);
    load_u64s<VN>(colS + t, cs);
    load_u64s<VN>(colM + t, cm);
    unsigned mask = 0;
#pragma unroll
    for (int q = 0; q < VN; ++q) {
        dold[q] = dd[q];
        sold[q] = sg[q];
        if (cd[q] == INF) continue;
        const int64_t cand = dsum<DT>(rd, cd[q]);
        if (cand == SAT) {
            if (dd[q] == INF) set_err(a.err, ERRF_DIST);
            continue;
        }
        if (cand > dd[q]) continue;
        if (cand < dd[q]) {
            sg[q] = mul_chk(rs, cs[q], a.err);
            V::set(dv, q, cand);
            ++n_changed;
            mask |= 1u << q;
        } else {
            const uint64_t p = mul_chk(rm, cm[q], a.err);
            if (p != 0ull) {
                sg[q] = add_chk(sg[q], p, a.err);
                ++n_ties;
                mask |= 1u << (q + 8);
            }
        }
    }
    if (mask) {
#pragma unroll
        for (int h = 0; h < VN / 2; ++h)
            *reinterpret_cast<ulonglong2*>(a.S + rowoff + t + 2 * h) = make_ulonglong2(sg[2 * h], sg[2 * h + 1]);
    }
    return mask;
}

// Records, for the whole warp, the changes one rule_vec_masked per lane found: lane
// holds row s (s < 0: nothing), the vector's first column t (a multiple of VN, so its
// pairs share one change-map word) and the changed pairs in bits; lanes with the same
// row must be consecutive.  One change-map OR per lane and one target-count atomic per
// run of lanes on the same row; the first change of a pair in the update saves its old
// values and lists it, as record_change does.  Every lane of the warp must call it.
template <typename DT>
__device__ __forceinline__ void record_changes_warp(const PairRec& r, int n, int s, int t, unsigned bits,
                                                    const int64_t* dold, const uint64_t* sold) {
    const int lane = threadIdx.x & 31;
    if (s >= 0 && bits) {
        uint32_t* w = r.chg + (size_t)s * r.chg_words + (t >> 5);
        unsigned wb = bits << (t & 31);
        if (!r.first) wb &= ~*w;   // pairs already recorded in this update keep their saved values
        bits = wb >> (t & 31);
        if (wb) atomicOr(w, wb);
        const size_t i0 = (size_t)s * n + t;
        for (unsigned b = bits; b; b &= b - 1) {
            const int q = __ffs(b) - 1;
            static_cast<DT*>(r.oldD)[i0 + q] = (DT)dold[q];
            r.oldS[i0 + q] = sold[q];
        }
    } else {
        bits = 0;
    }
    // segmented scan of the counts over runs of lanes with the same row
    const int c = __popc(bits);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int s_prev = __shfl_up_sync(0xffffffffu, s, 1);
    const unsigned starts = __ballot_sync(0xffffffffu, lane == 0 || s_prev != s);
    const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    const int start = 31 - __clz(starts & upto);
    const unsigned after = starts & ~upto;
    const int end = after ? __ffs(after) - 2 : 31;
    const int before = __shfl_sync(0xffffffffu, incl, start > 0 ? start - 1 : 0);
    const int base_incl = start > 0 ? before : 0;
    const int total = __shfl_sync(0xffffffffu, incl, end) - base_incl;
    int base = 0;
    if (lane == start && s >= 0 && total > 0) base = atomicAdd(r.tcnt + s, total);
    base = __shfl_sync(0xffffffffu, base, start);
    int pos = base + (incl - c - base_incl);
    for (unsigned b = bits; b; b &= b - 1, ++pos)
        if (pos < r.tcap) r.tlist[(size_t)s * r.tcap + pos] = t + __ffs(b) - 1;
}

template <typename DT>
__device__ __forceinline__ bool scan_vec(const ScanArgs<DT>& a, int s, size_t rowoff, int t, typename Vec<DT>::T& dv,
                                         const typename Vec<DT>::T& cv, int64_t rd, uint64_t rs, uint64_t rm,
                                         int& n_changed, int& n_ties) {
    if (!quick_vec<DT>(dv, cv, rd)) return false;
    return rule_vec<DT>(a, s, rowoff, t, dv, cv, rd, rs, rm, n_changed, n_ties);
}

// One work item of the rank-1 pass: row s (scalars rd, rs, rm), chunk c of CW columns.
template <typename DT, bool VECTOR, int U = kScanUnroll>
__device__ __forceinline__ void dev_scan_item(const ScanArgs<DT>& a, int s, int64_t rd, uint64_t rs, uint64_t rm,
                                              int c, int& n_changed, int& n_ties) {
    using V = Vec<DT>;
    constexpr int VN = V::N;
    constexpr int CW = kScanThreads * VN * U;
    const int n = a.n;
    const int64_t INF = Inf<DT>::v;
    const size_t rowoff = (size_t)s * n;
    DT* __restrict__ Drow = a.D + rowoff;
    const int t0 = c * CW;
    const int tid = threadIdx.x % kScanThreads;
    if constexpr (VECTOR) {
        typename V::T dv[U], cv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + (u * kScanThreads + tid) * VN;
            if (t < n) {
                dv[u] = __ldcs(reinterpret_cast<const typename V::T*>(Drow + t));
                cv[u] = __ldg(reinterpret_cast<const typename V::T*>(a.cD + t));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + (u * kScanThreads + tid) * VN;
            if (t >= n) break;
            if (scan_vec<DT>(a, s, rowoff, t, dv[u], cv[u], rd, rs, rm, n_changed, n_ties))
                *reinterpret_cast<typename V::T*>(Drow + t) = dv[u];
        }
    } else {
        for (int t = t0 + tid; t < t0 + CW && t < n; t += kScanThreads) {
            const int64_t cd = a.cD[t];
            if (cd == INF) continue;
            const int64_t old = Drow[t];
            const int64_t cand = dsum<DT>(rd, cd);
            int64_t nd;
            const int ties0 = n_ties;
            const uint64_t sig0 = a.rec.tcnt ? a.S[rowoff + t] : 0ull;
            if (pair_rule<DT>(cand, old, rowoff + t, rs, rm, a.cS[t], a.cM[t], a.S, a.err, &nd, &n_ties)) {
                Drow[t] = (DT)nd;
                ++n_changed;
                if (a.rec.tcnt) record_change<DT>(a.rec, n, s, t, old, sig0);
            } else if (n_ties != ties0 && a.rec.tcnt) {
                record_change<DT>(a.rec, n, s, t, old, sig0);
            }
        }
    }
}

// Fold the per-thread counters of the scan into the handle's statistics (whole warps).
__device__ __forceinline__ void scan_stats(int64_t* stats, int n_changed, int n_ties) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_changed += __shfl_xor_sync(0xffffffffu, n_changed, o);
        n_ties += __shfl_xor_sync(0xffffffffu, n_ties, o);
    }
    if ((threadIdx.x & 31) == 0 && (n_changed | n_ties)) {
        atomicAdd(reinterpret_cast<unsigned long long*>(stats + 4), (unsigned long long)n_changed);
        atomicAdd(reinterpret_cast<unsigned long long*>(stats + 5), (unsigned long long)n_ties);
    }
}

template <typename DT>
__device__ __forceinline__ void dev_write_row(int t, int n, DT* D, uint64_t* S, int v, const DT* cD, const uint64_t* cS,
                            const int32_t* err) {
    D[(size_t)v * n + t] = cD[t];
    S[(size_t)v * n + t] = cS[t];
}

template <typename DT>
struct AccArgs {
    int n;
    const DT* D;
    uint64_t* S;
    ff* Dl;
    const int32_t* e_off;
    const int32_t* e_len;
    const int32_t* e_src;
    const Arc<DT>* e_arc;
    int64_t e_cap;
    const int32_t* rows;
    const int32_t* count;
    int32_t* ws;
    int64_t ws_stride;
    int32_t* err;
    int mask_in_smem;
};

constexpr uint32_t FULL = 0xffffffffu;

// Distance of vertex i of the current source, with the row's own INF marker.
struct Dist16 {
    const uint16_t* p;
    static constexpr uint64_t INFV = 0xFFFFull;
    __device__ __forceinline__ uint64_t operator()(int i) const { return p[i]; }
};
template <typename DT>
struct DistG {
    const DT* p;
    static constexpr uint64_t INFV = (uint64_t)Inf<DT>::v;
    __device__ __forceinline__ uint64_t operator()(int i) const { return (uint64_t)(int64_t)__ldg(p + i); }
};

// Arc (x -> b, w) is in DAG'(s): d(x) finite (checked by the caller), d(b) finite and
// d(x) + w == d(b).
template <typename DA>
__device__ __forceinline__ bool on_dag(const DA& dist, uint64_t dx, int b, uint64_t w) {
    const uint64_t db = dist(b);
    return db != DA::INFV && dx + w == db;
}

// 16-bit in-degree counters, two to a 32-bit word (in-degrees stay below 65536).
__device__ __forceinline__ void cnt_inc(uint32_t* cnt, int b) {
    atomicAdd(cnt + (b >> 1), 1u << ((b & 1) << 4));
}
__device__ __forceinline__ bool cnt_last(uint32_t* cnt, int b) {
    const uint32_t sh = (b & 1) << 4;
    return ((atomicSub(cnt + (b >> 1), 1u << sh) >> sh) & 0xFFFFu) == 1u;
}

// Append the lanes' ready vertices to the order with one shared atomic per warp.
__device__ __forceinline__ void warp_append(bool ready, int b, uint16_t* order, int* tail) {
    const unsigned bal = __ballot_sync(FULL, ready);
    if (!bal) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(bal) - 1) base = atomicAdd(tail, __popc(bal));
    base = __shfl_sync(FULL, base, __ffs(bal) - 1);
    if (ready) order[base + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)b;
}

__device__ __forceinline__ ff warp_sum(ff x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = ff_add(x, ff_shfl_xor(x, o));
    return x;
}

// Finish vertex x: delta(x) = sigma_sx * acc, rho(x) = (1 + delta(x)) / sigma_sx
// = acc + 1 / sigma_sx.
__device__ __forceinline__ void finish_vertex(int x, ff acc, uint64_t sigma, ff* out, ff* rho) {
    const ff sx = ff_from_u64(sigma);
    out[x] = ff_mul(sx, acc);
    rho[x] = ff_add(acc, ff_rcp(sx));
}

// Passes 2 and 3 walk only the arcs of DAG'(s): pass 1 evaluates the predicate once per
// slot of the E* superset and records it in a bit mask (one warp ballot per 32 slots).
// Within a level, the DAG arcs of the level's vertices are spread evenly over the
// threads: a block scan of the vertices' DAG out-degrees gives each arc a rank, a
// thread finds the owner of its rank by binary search and the arc by selecting the
// right set bit of the owner's slot range.  In pass 3 the arcs' contributions go to a
// shared buffer and each owner adds its own in rank order (deterministic).  Vertices
// with more than kBigDag DAG out-arcs are taken by whole warps instead (lanes over
// their slots, fixed butterfly), so no owner loops long.
constexpr int kBigDag = 32;
constexpr int kBigCap = 2048;

__device__ __forceinline__ int count_bits(const uint32_t* m, int beg, int end) {
    if (beg >= end) return 0;
    const int w0 = beg >> 5, w1 = (end - 1) >> 5;
    int c = 0;
    for (int w = w0; w <= w1; ++w) {
        uint32_t b = m[w];
        if (w == w0) b &= 0xffffffffu << (beg & 31);
        if (w == w1) b &= 0xffffffffu >> (31 - ((end - 1) & 31));
        c += __popc(b);
    }
    return c;
}

// Slot of the r-th (0-based) set bit of m at or after slot beg.  Callers pass r below
// the number of set bits of the vertex's slot range, so the bit lies inside the range.
__device__ __forceinline__ int select_bit(const uint32_t* m, int beg, int r) {
    int w = beg >> 5;
    uint32_t b = m[w] & (0xffffffffu << (beg & 31));
    for (;;) {
        const int c = __popc(b);
        if (r < c) break;
        r -= c;
        b = m[++w];
    }
    for (; r > 0; --r) b &= b - 1u;
    return (w << 5) + __ffs(b) - 1;
}

// Exclusive block-wide prefix sum of v (all threads call it); *total gets the sum.
// s_ws needs T / 32 + 1 ints and must not be reused before a barrier (T threads).
template <int T>
__device__ __forceinline__ int block_excl_scan(int v, int* s_ws, int* total) {
    constexpr int NW = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int x = lane < NW ? s_ws[lane] : 0;
        int ix = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, ix, o);
            if (lane >= o) ix += y;
        }
        if (lane < NW) s_ws[lane] = ix - x;
        if (lane == NW - 1) s_ws[NW] = ix;
    }
    __syncthreads();
    *total = s_ws[NW];
    return s_ws[warp] + incl - v;
}

// Last index i in [0, T) with off[i] <= j (off non-decreasing, off[0] = 0).
template <int T>
__device__ __forceinline__ int owner_of(const int* off, int j) {
    int lo = 0, hi = T;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Append x to the big list when there is room (warp-aggregated); returns whether it was.
__device__ __forceinline__ bool big_push(bool want, int x, uint16_t* big, int* nbig) {
    const unsigned bal = __ballot_sync(FULL, want);
    if (!bal) return false;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(bal) - 1) base = atomicAdd(nbig, __popc(bal));
    base = __shfl_sync(FULL, base, __ffs(bal) - 1);
    const int pos = base + __popc(bal & ((1u << lane) - 1u));
    if (want && pos < kBigCap) {
        big[pos] = (uint16_t)x;
        return true;
    }
    return false;
}

template <typename DT, bool STATIC>
__device__ __forceinline__ void push_sigma(uint64_t* Ss, int b, uint64_t sx, int32_t* err) {
    if (STATIC) {
        const unsigned long long old =
            atomicAdd(reinterpret_cast<unsigned long long*>(Ss + b), (unsigned long long)sx);
        if (old + sx < old) set_err(err, ERRF_OVERFLOW);
    }
}

// Per-round shared scratch of the level passes.
// A round of a level pass gives every thread up to kPerThread vertices of the level.
constexpr int kPerThread = 2;

template <int T>
struct LevelSmem {
    int off[T];                  // first arc rank of the thread's vertices
    int beg[kPerThread][T];      // slot range start of each vertex
    int k0[T];                   // DAG out-arcs of the thread's first vertex
    uint64_t sx[kPerThread][T];  // path counts (static pass 2)
    ff buf[T];
    int ws[T / 32 + 1];
};

template <typename DT, bool STATIC, int T, typename DA>
__device__ __forceinline__ void accumulate_source(const AccArgs<DT>& a, const DA dist, int s, uint64_t* Ss,
                                                  ff* out, uint32_t* cnt, uint16_t* order, uint32_t* mask,
                                                  uint16_t* big, LevelSmem<T>& ls, ff* rho, int32_t* lvl,
                                                  int* s_tail, int* s_nbig) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = T / 32, U = 8;
    // ---- pass 1: DAG'(s) membership of every slot, and in-degrees (loads of U chunks
    // are issued before any of them is used)
    const int nchunk = (int)((a.e_cap + 31) >> 5);
    for (int c0 = warp; c0 < nchunk; c0 += U * NW) {
        Arc<DT> r[U];
        int src[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = ((int64_t)(c0 + u * NW) << 5) + lane;
            r[u].dst = -1;
            src[u] = 0;
            if (e < a.e_cap) {
                r[u] = a.e_arc[e];
                src[u] = a.e_src[e];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + u * NW;
            if (c >= nchunk) break;
            const int b = (int)r[u].dst;
            bool on = false;
            if (b >= 0) {
                const uint64_t dx = dist(src[u]);
                on = dx != DA::INFV && on_dag(dist, dx, b, (uint64_t)r[u].w);
            }
            if (on) cnt_inc(cnt, b);
            const unsigned word = __ballot_sync(FULL, on);
            if (lane == 0) mask[c] = word;
        }
    }
    __syncthreads();   // the distance row (aliased by order) is dead from here on
    if (tid == 0) {
        order[0] = (uint16_t)s;
        lvl[0] = 0;
        lvl[1] = 1;
        *s_tail = 1;
        *s_nbig = 0;
    }
    __syncthreads();
    // ---- pass 2: Kahn levels (statically also the forward path counts)
    int L = 0;
    for (;;) {
        const int lo = lvl[L], hi = lvl[L + 1];
        for (int qb = lo; qb < hi; qb += kPerThread * T) {
            int kk[kPerThread];
            int kt = 0;
#pragma unroll
            for (int v = 0; v < kPerThread; ++v) {
                const int q = qb + v * T + tid;
                int x = 0, beg = 0, k = 0;
                if (q < hi) {
                    x = order[q];
                    beg = a.e_off[x];
                    k = count_bits(mask, beg, beg + a.e_len[x]);
                }
                if (big_push(k > kBigDag, x, big, s_nbig)) k = 0;
                kk[v] = k;
                kt += k;
                ls.beg[v][tid] = beg;
                if (STATIC) ls.sx[v][tid] = k ? Ss[x] : 0ull;
            }
            int total;
            const int off = block_excl_scan<T>(kt, ls.ws, &total);
            ls.off[tid] = off;
            ls.k0[tid] = kk[0];
            __syncthreads();
            for (int jb = 0; jb < total; jb += T) {
                const int j = jb + tid;
                bool ready = false;
                int b = 0;
                if (j < total) {
                    const int o = owner_of<T>(ls.off, j);
                    int r = j - ls.off[o];
                    const int v = r < ls.k0[o] ? 0 : 1;
                    if (v) r -= ls.k0[o];
                    const int e = select_bit(mask, ls.beg[v][o], r);
                    b = (int)a.e_arc[e].dst;
                    push_sigma<DT, STATIC>(Ss, b, STATIC ? ls.sx[v][o] : 0ull, a.err);
                    ready = cnt_last(cnt, b);
                }
                warp_append(ready, b, order, s_tail);
            }
            __syncthreads();
        }
        const int nb = min(*s_nbig, kBigCap);
        for (int i = warp; i < nb; i += NW) {
            const int x = big[i];
            const int beg = a.e_off[x], end = beg + a.e_len[x];
            const uint64_t sx = STATIC ? Ss[x] : 0ull;
            for (int eb = beg; eb < end; eb += 32) {
                const int e = eb + lane;
                bool ready = false;
                int b = 0;
                if (e < end && ((mask[e >> 5] >> (e & 31)) & 1u)) {
                    b = (int)a.e_arc[e].dst;
                    push_sigma<DT, STATIC>(Ss, b, sx, a.err);
                    ready = cnt_last(cnt, b);
                }
                warp_append(ready, b, order, s_tail);
            }
        }
        __syncthreads();
        if (tid == 0) {
            lvl[L + 2] = *s_tail;
            *s_nbig = 0;
        }
        __syncthreads();
        if (lvl[L + 2] == hi) break;
        ++L;
    }
    // ---- pass 3: Eq. 4 in reverse level order (level 0 is s: delta_s.(s) is not kept)
    for (int Lq = L; Lq >= 1; --Lq) {
        const int lo = lvl[Lq], hi = lvl[Lq + 1];
        for (int qb = lo; qb < hi; qb += kPerThread * T) {
            int xs[kPerThread], kk[kPerThread];
            uint64_t sig[kPerThread];
            bool mine[kPerThread];
            int kt = 0;
#pragma unroll
            for (int v = 0; v < kPerThread; ++v) {
                const int q = qb + v * T + tid;
                int x = 0, beg = 0, k = 0;
                if (q < hi) {
                    x = order[q];
                    beg = a.e_off[x];
                    k = count_bits(mask, beg, beg + a.e_len[x]);
                }
                const bool is_big = big_push(k > kBigDag, x, big, s_nbig);
                if (is_big) k = 0;
                mine[v] = q < hi && !is_big;
                sig[v] = mine[v] ? Ss[x] : 1ull;
                xs[v] = x;
                kk[v] = k;
                kt += k;
                ls.beg[v][tid] = beg;
            }
            int total;
            const int off = block_excl_scan<T>(kt, ls.ws, &total);
            ls.off[tid] = off;
            ls.k0[tid] = kk[0];
            __syncthreads();
            ff acc[kPerThread];
#pragma unroll
            for (int v = 0; v < kPerThread; ++v) acc[v] = ff{0.0f, 0.0f};
            for (int jb = 0; jb < total; jb += T) {
                const int j = jb + tid;
                if (j < total) {
                    const int o = owner_of<T>(ls.off, j);
                    int r = j - ls.off[o];
                    const int v = r < ls.k0[o] ? 0 : 1;
                    if (v) r -= ls.k0[o];
                    const int e = select_bit(mask, ls.beg[v][o], r);
                    ls.buf[tid] = rho[a.e_arc[e].dst];
                }
                __syncthreads();
                int p = off;
#pragma unroll
                for (int v = 0; v < kPerThread; ++v) {
                    const int p0 = max(p, jb), p1 = min(p + kk[v], jb + T);
                    for (int pp = p0; pp < p1; ++pp) acc[v] = ff_add(acc[v], ls.buf[pp - jb]);
                    p += kk[v];
                }
                __syncthreads();
            }
#pragma unroll
            for (int v = 0; v < kPerThread; ++v)
                if (mine[v]) finish_vertex(xs[v], acc[v], sig[v], out, rho);
        }
        __syncthreads();
        const int nb = min(*s_nbig, kBigCap);
        for (int i = warp; i < nb; i += NW) {
            const int x = big[i];
            const int beg = a.e_off[x], end = beg + a.e_len[x];
            ff acc{0.0f, 0.0f};
            for (int e = beg + lane; e < end; e += 32)
                if ((mask[e >> 5] >> (e & 31)) & 1u) acc = ff_add(acc, rho[a.e_arc[e].dst]);
            acc = warp_sum(acc);
            if (lane == 0) finish_vertex(x, acc, Ss[x], out, rho);
        }
        __syncthreads();
        if (tid == 0) *s_nbig = 0;
        __syncthreads();
    }
}

// Shared-memory layout of the accumulation kernel for n vertices (n rounded to np):
// [d16 | order] (2np bytes; the distance row is dead once the slot mask is built, so
// the level order reuses it) | cnt (np/2 words) | big list | slot mask (here when it
// fits, else in the work space).
struct AccSmem {
    uint16_t* d16;
    uint16_t* order;
    uint32_t* cnt;
    uint16_t* big;
    uint32_t* mask;
    ff* rho;
    int32_t* lvl;
};

template <typename DT>
__device__ __forceinline__ AccSmem acc_smem(const AccArgs<DT>& a, unsigned char* smem, int32_t* wsb) {
    const int n = a.n;
    const int np = (n + 31) & ~31;
    AccSmem m;
    m.d16 = reinterpret_cast<uint16_t*>(smem);
    m.order = m.d16;
    m.cnt = reinterpret_cast<uint32_t*>(smem + 2 * (size_t)np);
    m.big = reinterpret_cast<uint16_t*>(smem + 4 * (size_t)np);
    m.rho = reinterpret_cast<ff*>(wsb);
    m.lvl = wsb + 2 * (size_t)n;
    m.mask = a.mask_in_smem ? reinterpret_cast<uint32_t*>(smem + 4 * (size_t)np + 2 * kBigCap)
                            : reinterpret_cast<uint32_t*>(wsb + ((3 * (int64_t)n + 2 + 3) & ~(int64_t)3));
    return m;
}

// Re-accumulate source s (whole block; every thread calls it): stage its distance row,
// rebuild DAG'(s), order it, pull Eq. 4, write its delta row (and, statically, its
// sigma row).
template <typename DT, bool STATIC, int T>
__device__ __forceinline__ void dev_accum_source(const AccArgs<DT>& a, int s, const AccSmem& m, LevelSmem<T>& ls,
                                                 int* s_tail, int* s_nbig) {
    const int n = a.n;
    const int np = (n + 31) & ~31;
    const int tid = threadIdx.x;
    const int64_t INF = Inf<DT>::v;
    const DT* Ds = a.D + (size_t)s * n;
    uint64_t* Ss = a.S + (size_t)s * n;
    ff* out = a.Dl + (size_t)s * n;
    int wide = 0;
    for (int t = tid; t < n; t += T) {
        const int64_t v = Ds[t];
        uint16_t c;
        if (v == INF) c = 0xFFFF;
        else if (v < 0xFFFF) c = (uint16_t)v;
        else { c = 0xFFFE; wide = 1; }
        m.d16[t] = c;
        out[t] = ff{0.0f, 0.0f};
        if (STATIC) Ss[t] = (t == s) ? 1ull : 0ull;
    }
    for (int t = tid; t < np / 2; t += T) m.cnt[t] = 0u;
    wide = __syncthreads_or(wide);
    if (!wide)
        accumulate_source<DT, STATIC, T>(a, Dist16{m.d16}, s, Ss, out, m.cnt, m.order, m.mask, m.big, ls, m.rho, m.lvl,
                                      s_tail, s_nbig);
    else
        accumulate_source<DT, STATIC, T>(a, DistG<DT>{Ds}, s, Ss, out, m.cnt, m.order, m.mask, m.big, ls, m.rho, m.lvl,
                                      s_tail, s_nbig);
    __syncthreads();
}

// partial[rb][t] = sum over rows r of row block rb of Dl[s_r][t] (t != s_r), rows in
// increasing order, in float-float (all terms are non-negative); rows = nullptr means
// all n rows.
__device__ __forceinline__ void dev_bc_partial(int t, int rb, int n, const int32_t* rows, int total,
                                               const ff* Dl, ff* partial) {
    const int r0 = rb * kRowsPerBlock;
    if (r0 >= total || t >= n) return;
    const int r1 = min(total, r0 + kRowsPerBlock);
    ff acc{0.0f, 0.0f};
    for (int r = r0; r < r1; ++r) {
        const int s = rows ? rows[r] : r;
        if (s != t) acc = ff_add(acc, Dl[(size_t)s * n + t]);
    }
    partial[(size_t)rb * n + t] = acc;
}

// bc (hi, lo) += sign * (sum of the row-block partials in block order): the partials are
// summed in float-float, the total is taken to fp64 and added with TwoSum; overwrite
// starts from zero (the static computation).
__device__ __forceinline__ void dev_bc_finish(int t, int n, int total, const ff* partial, double sign,
                                              int overwrite, double* hi, double* lo) {
    const int nrb = (total + kRowsPerBlock - 1) / kRowsPerBlock;
    if (nrb == 0 && !overwrite) return;
    ff acc{0.0f, 0.0f};
    for (int rb = 0; rb < nrb; ++rb) acc = ff_add(acc, partial[(size_t)rb * n + t]);
    const double sum = sign * ff_to_double(acc);
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

}  // namespace bcg
