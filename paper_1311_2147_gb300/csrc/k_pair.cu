// k_pair.cu -- dependency rows of an undirected update by pair corrections.
//
// delta_s(x) is the sum over targets t of the pair dependency
// delta_st(x) = sigma_sx * sigma_xt / sigma_st, taken where d(s,x) + d(x,t) = d(s,t) and
// x is neither s nor t (Section 2, the definition that Eq. 4 turns into a recurrence).
// Under a decrease, a pair (s,t) whose distance and path count are both unchanged keeps
// its whole set of shortest paths: no old shortest path uses a changed edge (it would
// now be shorter, so d(s,t) would have dropped), so each one keeps its weight and stays
// shortest, and since sigma_st did not grow no path joined them.  Every delta_st(x) of
// such a pair is unchanged, hence
//     delta'_s(x) = delta_s(x) + sum over changed pairs (s,t) of [delta'_st(x) - delta_st(x)].
// The passes that write D and sigma (the rank-1 passes of Lemma 2 / Lemma 4 and the
// write of row v) record each pair's first change in an update: a bit in the n x n
// change map, the pair's old distance and path count, and t in the target list of row
// s (record_change).  A row with at most kPairCap changed targets is corrected by the
// sum above.  The state before the update is the state after it except at the set
// bits, where the saved values hold, so both terms read the current rows plus a few
// saved values.  In G_D of an undirected graph d(x,t) = d(t,x) and sigma_xt = sigma_tx
// before and after the update, so the column t of the formula is row t, read
// contiguously.  Rows with more targets than the cap are re-accumulated by Algorithm 1.
#include "bc_batch.cuh"
#include "bc_device.cuh"
#include "ff.cuh"

static_assert(bcg::kPairCap <= 1024, "the targets of a row are sorted by one CTA");

namespace bcg {

constexpr int kPairThreads = 256;
constexpr int kPairCtasPerSm = 4;
// targets whose rows are loaded together: two with up to four columns per thread, one
// with eight (whose two loads per target already overlap)
template <int VN> struct PairGroup { static constexpr int value = VN >= 8 ? 1 : 2; };
constexpr int kPairPieces = 8;  // pieces of equal weight per CTA of the grid

// The row lists of an update's corrections in one pass over the changed-row flags (one
// CTA, kCompactPerThread flags per thread and tile, as k_compact): acc_rows = the
// changed rows, full_rows = those with more recorded targets than the cap (Algorithm 1
// in full), both in increasing order.  The flags are cleared and the per-update counters
// added as k_compact does for acc_rows.  A thread's two counts travel in one scan word
// (each tile holds at most 1024 x 16 < 2^16 rows).
// (CTA-wide; wsum and s_total in shared memory.)
__device__ __forceinline__ void dev_pair_lists(int n, uint8_t* changed, const int32_t* tcnt, int tcap,
                                               int32_t* acc_rows, int32_t* acc_count, int32_t* full_rows,
                                               int32_t* full_count, int64_t* stats, bool bad, int32_t* wsum,
                                               int32_t& s_total) {
    constexpr int E = kCompactPerThread;
    static_assert(kCompactThreads * E < (1 << 16), "a tile's counts fit 16 bits");
    const int nwarps = blockDim.x >> 5;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int base_a = 0, base_f = 0;
    for (int tile = 0; tile < n; tile += (int)blockDim.x * E) {
        const int s0 = tile + tid * E;
        uint32_t fl = 0, ffl = 0;   // bit e: row s0 + e changed / goes to the full path
        if (s0 < n) {
            if (s0 + E <= n && ((reinterpret_cast<uintptr_t>(changed + s0) & 15) == 0)) {
                const uint4 v = *reinterpret_cast<const uint4*>(changed + s0);
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if ((w[e >> 2] >> (8 * (e & 3))) & 0xFFu) fl |= 1u << e;
                *reinterpret_cast<uint4*>(changed + s0) = make_uint4(0u, 0u, 0u, 0u);
            } else {
                for (int e = 0; e < E && s0 + e < n; ++e) {
                    if (changed[s0 + e]) fl |= 1u << e;
                    changed[s0 + e] = 0;
                }
            }
            if (bad) fl = 0;
            for (uint32_t b = fl; b; b &= b - 1) {
                const int e = __ffs(b) - 1;
                if (tcnt[s0 + e] > tcap) ffl |= 1u << e;
            }
        }
        const int c = __popc(fl) | (__popc(ffl) << 16);
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
        const int excl = wsum[wid] + incl - c;
        int pa = base_a + (excl & 0xFFFF), pf = base_f + (excl >> 16);
        while (fl) {
            const int e = __ffs(fl) - 1;
            fl &= fl - 1;
            acc_rows[pa++] = s0 + e;
            if ((ffl >> e) & 1u) full_rows[pf++] = s0 + e;
        }
        base_a += s_total & 0xFFFF;
        base_f += s_total >> 16;
        __syncthreads();
    }
    if (tid == 0) {
        *acc_count = base_a;
        *full_count = base_f;
        stats[0] += base_a;
        if (base_a == 0) stats[1] += 1;
        if (base_a > stats[2]) stats[2] = base_a;
        stats[3] += 1;
    }
}

__global__ void __launch_bounds__(kCompactThreads) k_pair_lists(int n, uint8_t* changed, const int32_t* tcnt,
                                                                int tcap, int32_t* acc_rows, int32_t* acc_count,
                                                                int32_t* full_rows, int32_t* full_count,
                                                                int64_t* stats, const int32_t* err) {
    pdl_enter();
    __shared__ int32_t wsum[32];
    __shared__ int32_t s_total;
    dev_pair_lists(n, changed, tcnt, tcap, acc_rows, acc_count, full_rows, full_count, stats, *err != 0, wsum,
                   s_total);
}

// Per-update records of the rows listed in rows[0..count) back to zero (a pair (s,t)
// changes only in a changed row s), a warp per row: a row with at most tcap changed
// targets has its bits only in the words of its listed targets, a longer one is
// cleared whole.  The rows sent to the full path are added to stats[7].
__device__ __forceinline__ void dev_pair_clear_row(int s, int32_t* tcnt, const int32_t* tlist, int tcap,
                                                   uint32_t* chg, int words) {
    const int lane = threadIdx.x & 31;
    const int T = tcnt[s];
    uint32_t* row = chg + (size_t)s * words;
    if (T <= tcap) {
        for (int j = lane; j < T; j += 32) row[tlist[(size_t)s * tcap + j] >> 5] = 0u;
    } else {
        for (int j = lane; j < words; j += 32) row[j] = 0u;
    }
    __syncwarp();
    if (lane == 0) tcnt[s] = 0;
}

__global__ void k_pair_clear(const int32_t* rows, const int32_t* count, int32_t* tcnt, const int32_t* tlist,
                             int tcap, uint32_t* chg, int words, const int32_t* full_count, int64_t* stats) {
    pdl_enter();
    const int cnt = *count;
    if (blockIdx.x == 0 && threadIdx.x == 0) stats[7] += *full_count;
    const int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < cnt; i += gridDim.x * wpb)
        dev_pair_clear_row(rows[i], tcnt, tlist, tcap, chg, words);
}

// One changed target t of a row s, as prepared by k_pair_plan: the pair's distance and
// reciprocal path count before and after the update (-1: no path).
struct PairTgt {
    int32_t t;
    int32_t pad;
    int64_t dold;
    int64_t dnew;
    ff rold;
    ff rnew;
};
static_assert(sizeof(PairTgt) == 40, "the plan is allocated with 40 bytes per target");

template <typename DT>
struct PairArgs {
    int n;
    const DT* D;            // state after the update
    const uint64_t* S;
    const uint32_t* chg;    // change map: bit (s,x) set where the pair changed
    int words;
    const DT* oD;           // old values where the bit is set
    const uint64_t* oS;
    int32_t* tcnt;          // changed targets per row
    const int32_t* tlist;
    PairTgt* plan;          // [n * tcap]
    int64_t* wpre;          // [n + 1] prefix of the item weights of the listed rows
    int32_t* next_piece;    // pieces of the work handed out so far past the first wave
    const int32_t* prows;   // the rows corrected pair by pair, most targets first
    const int32_t* pcount;
    const int32_t* gate;    // when set: the column test runs only if *gate != 0 (walk overflow)
    int tcap;
    const int32_t* rows;
    const int32_t* count;
    ff* Dl;
    int64_t* bcfix;         // [2n] BC change of this update (fixed point, see bc_fix_add)
    int32_t* err;
};

// BC(x) += v for one corrected entry delta_s(x): v is added to the column's fixed-point
// pair (A in units of 2^-24, B in units of 2^-56) by two integer atomics, so the total
// does not depend on the order in which rows and CTAs add (the result is deterministic)
// and is exact up to the 2^-56 rounding of each entry.  Bounds: each pair term
// delta_st(x) lies in [0, 1] and a row has at most kPairCap targets, so |v| <= 128 and
// |A| <= 2^31, |B| <= 2^31 per entry (the DAG walks add a row's column sum with
// 0 <= B < 2^32); a column receives at most one entry per row, so for n < 2^20 both
// sums stay below 2^52 and k_bc_fix converts them exactly.
__device__ __forceinline__ void bc_fix_add(int64_t* fix, int x, ff v) {
    // in single precision, as fix_split: h = hi * 2^24 is exact (|h| <= 2^31) and so is
    // h - rint(h); (h - a) * 2^32 and lo * 2^56 (|lo| <= 2^-17) are exact scalings, each
    // rounded to an integer once, and a carry keeps |B| <= 2^31
    const float h = v.hi * 0x1p24f;
    const float a = rintf(h);
    long long b = __float2ll_rn((h - a) * 0x1p32f) + __float2ll_rn(v.lo * 0x1p56f);
    const long long c = (b + (1ll << 31)) >> 32;
    const long long A = __float2ll_rn(a) + c;
    b -= c << 32;
    unsigned long long* p = reinterpret_cast<unsigned long long*>(fix + 2 * (size_t)x);
    atomicAdd(p, (unsigned long long)A);
    if (b) atomicAdd(p + 1, (unsigned long long)b);
}

// One warp per listed row with 1..tcap changed targets (most rows have a few): rank
// them (the sums then run in a fixed order) and write the per-target scalars of the
// plan.  Every target of row s has its bit set, so its old values are the saved ones.
constexpr int kPlanThreads = 256;

// (One warp; sv: kPairCap ints of shared memory.)
template <typename DT>
__device__ __forceinline__ void dev_pair_plan_row(const PairArgs<DT>& a, int s, int32_t* sv) {
    const int n = a.n;
    const int64_t INF = Inf<DT>::v;
    const int lane = threadIdx.x & 31;
    const int T = a.tcnt[s];
    if (T == 0 || T > a.tcap) return;   // warp-uniform
    for (int j = lane; j < T; j += 32) sv[j] = a.tlist[(size_t)s * a.tcap + j];
    __syncwarp();
    for (int j = lane; j < T; j += 32) {
        const int val = sv[j];
        int pos = 0;
        for (int k = 0; k < T; ++k) pos += sv[k] < val;   // targets are distinct
        const size_t it = (size_t)s * n + val;
        const int64_t dol = a.oD[it], dnw = a.D[it];
        const uint64_t sol = a.oS[it], snw = a.S[it];
        PairTgt p;
        p.t = val;
        p.pad = 0;
        p.dold = (dol == INF || sol == 0) ? -1 : dol;
        p.dnew = (dnw == INF || snw == 0) ? -1 : dnw;
        p.rold = sol ? ff_rcp(ff_from_u64(sol)) : ff{0.f, 0.f};
        p.rnew = snw ? ff_rcp(ff_from_u64(snw)) : ff{0.f, 0.f};
        a.plan[(size_t)s * a.tcap + pos] = p;
    }
    __syncwarp();
}

template <typename DT>
__global__ void __launch_bounds__(kPlanThreads) k_pair_plan(PairArgs<DT> a) {
    pdl_enter();
    __shared__ int32_t s_val[kPlanThreads / 32][kPairCap];
    if (*a.err) return;
    const int cnt = *a.count;
    const int wib = threadIdx.x >> 5;
    const int nw = gridDim.x * (kPlanThreads / 32);
    for (int i = blockIdx.x * (kPlanThreads / 32) + wib; i < cnt; i += nw) dev_pair_plan_row<DT>(a, a.rows[i], s_val[wib]);
}

// sigma_sx * sigma_xt / sigma_st in float-float (the quotient as a product with the
// reciprocal of sigma_st).
__device__ __forceinline__ ff pair_term(uint64_t a, uint64_t b, const ff& rcp) {
    return ff_mul(ff_mul(ff_from_u64(a), ff_from_u64(b)), rcp);
}

// VN consecutive distances (one 16-byte load when VN > 1).
template <typename DT, int VN>
struct DVec {
    DT v[VN];
    __device__ __forceinline__ void load(const DT* p) {
        if constexpr (VN == 8) {
            const int4 x = *reinterpret_cast<const int4*>(p);
            const int4 y = *reinterpret_cast<const int4*>(p + 4);
            v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
            v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
        } else if constexpr (VN == 4) {
            const int4 x = *reinterpret_cast<const int4*>(p);
            v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        } else if constexpr (VN == 2) {
            const longlong2 x = *reinterpret_cast<const longlong2*>(p);
            v[0] = x.x; v[1] = x.y;
        } else {
            v[0] = p[0];
        }
    }
};

// Bits of columns x0 .. x0+VN-1 of row r in the change map (x0 is a multiple of VN, so
// they sit in one word).
template <int VN>
__device__ __forceinline__ unsigned chg_bits(const uint32_t* chg, int words, int r, int x0) {
    return (chg[(size_t)r * words + (x0 >> 5)] >> (x0 & 31)) & ((1u << VN) - 1u);
}

// The old values of row r at the columns whose bit is set (one vector load; the saved
// values at the other columns are stale and not used).
template <typename DT, int VN>
__device__ __forceinline__ void patch_old(DVec<DT, VN>& d, unsigned bits, const DT* oD_row, int x0) {
    DVec<DT, VN> o;
    o.load(oD_row + x0);
#pragma unroll
    for (int q = 0; q < VN; ++q)
        if ((bits >> q) & 1u) d.v[q] = o.v[q];
}

template <typename DT> struct Unsigned;
template <> struct Unsigned<int32_t> { using T = uint32_t; };
template <> struct Unsigned<int64_t> { using T = uint64_t; };

// Bit q set where column x0+q lies on a shortest s-t path of one state:
// d(s,x) + d(x,t) = d(s,t) and d(x,t) > 0 (x != t; x != s is ensured by the caller,
// which replaces d(s,s) by INF).  Distances are below INF = DT max, so their unsigned
// sum never wraps, and a sum with an INF term exceeds every finite d(s,t); "no path"
// is passed as all ones, which no sum equals.
template <typename DT, int VN>
__device__ __forceinline__ unsigned on_path(const DVec<DT, VN>& ds, const DVec<DT, VN>& dt,
                                            typename Unsigned<DT>::T dst) {
    using U = typename Unsigned<DT>::T;
    unsigned m = 0;
#pragma unroll
    for (int q = 0; q < VN; ++q)
        m |= (((U)ds.v[q] + (U)dt.v[q] == (U)dst) && dt.v[q] != 0) ? (1u << q) : 0u;
    return m;
}

// Per-target scalars of the row being processed, as staged in shared memory: what
// every column test reads (row t of D and of the change map, and the distances, with
// -1 for "no path": in unsigned arithmetic no sum of two distances equals it) and
// what only a matched column reads.
template <typename DT>
struct TgtFast {
    const DT* Dt;
    const uint32_t* Ct;
    DT dold, dnew;
};
struct TgtSlow {
    int64_t rt;      // t * n
    ff rold, rnew;
};


// Weight of one work item of a listed row: its targets plus one (the row's own loads),
// or 0 when the row takes the full path or has nothing to correct.
__device__ __forceinline__ int64_t item_weight(int T, int tcap) { return (T == 0 || T > tcap) ? 0 : T + 1; }

// prows[0..*pcount) = the listed rows with 1..tcap targets, most targets first;
// wpre[i] = total weight of the items of rows prows[0..i-1] (nchunks items per row).
// One CTA: a counting sort (the lanes of a warp with the same target count add to its
// bucket with one shared-memory atomic), then each warp scans a contiguous run of the
// sorted rows and one block scan joins the runs.
// Also adds the rows with a correction and their targets to stats[8], stats[9].
// Listed rows the weights pass stages in shared memory (up to n; none past the limit).
constexpr int kWeightsStageMax = 20480;   // 160 KB of row ids and counts
static int weights_stage(int n) { return n <= kWeightsStageMax ? n : 0; }

struct PairWeightsSmem {
    int64_t wsum[32];
    int64_t s_total;
    int64_t s_rows[32], s_tgts[32];
    int s_hist[kPairCap + 1];
};

// (CTA-wide, 1024 threads.)  s_r and s_T: scap ints each of shared memory; when the
// listed rows fit, they and their target counts are staged there first, every load
// issued before any is used (the passes below would otherwise wait on a row id and then
// on its count, tile after tile).  The sorted rows' counts are staged in wpre, which
// the last pass overwrites with the prefix.
__device__ __forceinline__ void dev_pair_weights(const int32_t* rows, const int32_t* count, const int32_t* tcnt,
                                                 int tcap, int nchunks, int32_t* prows, int32_t* pcount,
                                                 int64_t* wpre, int64_t* stats, int32_t* next_piece,
                                                 int32_t* walk_ctl, int32_t* walk_rowE, PairWeightsSmem& sm,
                                                 int32_t* s_r, int32_t* s_T, int scap) {
    int64_t* wsum = sm.wsum;
    int64_t& s_total = sm.s_total;
    int64_t* s_rows = sm.s_rows;
    int64_t* s_tgts = sm.s_tgts;
    int* s_hist = sm.s_hist;
    const int cnt_all = *count;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = blockDim.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    // the rows with 1..tcap targets, most targets first (a counting sort): the heaviest
    // items are handed out first and the light ones fill the end of the kernel.  The
    // order inside a bucket follows the atomics; a row's result does not depend on it.
    for (int b = tid; b <= kPairCap; b += blockDim.x) s_hist[b] = 0;
    const bool staged = cnt_all <= scap;
    if (staged) {
        for (int i = tid; i < cnt_all; i += blockDim.x) s_r[i] = rows[i];
        __syncthreads();
        for (int i = tid; i < cnt_all; i += blockDim.x) s_T[i] = tcnt[s_r[i]];
    }
    __syncthreads();
    for (int i0 = 0; i0 < cnt_all; i0 += blockDim.x) {   // warp-uniform bounds (the match)
        const int i = i0 + tid;
        const int T = i < cnt_all ? (staged ? s_T[i] : tcnt[rows[i]]) : 0;
        const bool ok = T > 0 && T <= tcap;
        const unsigned peers = __match_any_sync(0xffffffffu, ok ? T : -1);
        if (ok && lane == __ffs(peers) - 1) atomicAdd(&s_hist[T], __popc(peers));
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int b = kPairCap; b >= 1; --b) {
            const int h = s_hist[b];
            s_hist[b] = acc;
            acc += h;
        }
        s_hist[0] = acc;
        *pcount = acc;
    }
    __syncthreads();
    const int cnt = s_hist[0];
    if (walk_rowE)
        for (int i = tid; i < cnt_all; i += blockDim.x) walk_rowE[i] = 0;
    for (int i0 = 0; i0 < cnt_all; i0 += blockDim.x) {
        const int i = i0 + tid;
        const int r = i < cnt_all ? (staged ? s_r[i] : rows[i]) : 0;
        const int T = i < cnt_all ? (staged ? s_T[i] : tcnt[r]) : 0;
        const bool ok = T > 0 && T <= tcap;
        const unsigned peers = __match_any_sync(0xffffffffu, ok ? T : -1);
        const int leader = __ffs(peers) - 1;
        int p0 = 0;
        if (ok && lane == leader) p0 = atomicAdd(&s_hist[T], __popc(peers));
        p0 = __shfl_sync(0xffffffffu, p0, leader);
        if (ok) {
            const int pos = p0 + __popc(peers & below);
            prows[pos] = r;
            wpre[pos] = T;
        }
    }
    __syncthreads();
    int64_t my_rows = 0, my_tgts = 0;
    // a contiguous run of the sorted rows per warp, 32 rows per step
    const int per = (cnt + nw - 1) / nw;
    const int w0 = min(cnt, wid * per), w1 = min(cnt, w0 + per);
    auto warp_incl = [&](int64_t x) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        return x;
    };
    int64_t run = 0;
    for (int b0 = w0; b0 < w1; b0 += 32) {
        const int i = b0 + lane;
        const int64_t iw = i < w1 ? item_weight((int)wpre[i], tcap) : 0;
        if (iw) {
            ++my_rows;
            my_tgts += iw - 1;
        }
        run += __shfl_sync(0xffffffffu, warp_incl(iw * nchunks), 31);
    }
    if (lane == 0) wsum[wid] = run;
    __syncthreads();
    if (wid == 0) {
        const int64_t x = lane < nw ? wsum[lane] : 0;
        const int64_t winc = warp_incl(x);
        if (lane < nw) wsum[lane] = winc - x;
        if (lane == 31) s_total = winc;
    }
    __syncthreads();
    run = wsum[wid];
    for (int b0 = w0; b0 < w1; b0 += 32) {
        const int i = b0 + lane;
        const int64_t x = i < w1 ? item_weight((int)wpre[i], tcap) * nchunks : 0;
        const int64_t incl = warp_incl(x);
        if (i < w1) wpre[i] = run + incl - x;
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    const int64_t base = s_total;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_rows += __shfl_xor_sync(0xffffffffu, my_rows, o);
        my_tgts += __shfl_xor_sync(0xffffffffu, my_tgts, o);
    }
    if (lane == 0) {
        s_rows[wid] = my_rows;
        s_tgts[wid] = my_tgts;
    }
    __syncthreads();
    if (tid == 0) {
        int64_t r = 0, t = 0;
        for (int k = 0; k < nw; ++k) {
            r += s_rows[k];
            t += s_tgts[k];
        }
        wpre[cnt] = base;
        *next_piece = 0;
        if (walk_ctl)
            for (int k = 0; k < 8; ++k) walk_ctl[k] = 0;
        stats[8] += r;
        stats[9] += t;
    }
}

__global__ void __launch_bounds__(1024) k_pair_weights(const int32_t* rows, const int32_t* count,
                                                       const int32_t* tcnt, int tcap, int nchunks,
                                                       int32_t* prows, int32_t* pcount,
                                                       int64_t* wpre, int64_t* stats, int32_t* next_piece,
                                                       int32_t* walk_ctl, int32_t* walk_rowE, const int32_t* err,
                                                       int scap) {
    pdl_enter();
    __shared__ PairWeightsSmem sm;
    extern __shared__ int32_t s_stage[];   // 2 * scap ints
    if (*err) return;
    dev_pair_weights(rows, count, tcnt, tcap, nchunks, prows, pcount, wpre, stats, next_piece, walk_ctl, walk_rowE,
                     sm, s_stage, s_stage + scap, scap);
}

// Queue of one warp's matches: entry = lane (5 bits) | q (3) | target index u (7) |
// new state (1) | old d/sigma of s saved (1) | old d/sigma of t saved (1); the terms are
// evaluated by all lanes together and summed by the owning lane in queue order.
constexpr int kPairQueue = 64;
struct PairQueue {
    uint32_t e[kPairQueue];
    ff term[kPairQueue];
};

// One work item: the VN columns x0 .. x0+VN-1 of this thread in row s, whose U_
// targets are staged in s_fa / s_sl.  Targets go in groups of kPairGroup: the group's
// rows are loaded together (one memory round trip), then tested with one add and
// compare per column and state.  The matches (columns on a shortest s-t path of either
// state) are appended to the warp's queue in target order, old state first; when the
// queue is full and at the end of the item, the warp evaluates all queued terms at once
// (one match per lane, its two path counts loaded together with the others) and each
// lane adds its own terms to its column sums in queue order.  A column's sum thus runs
// in target order whatever the lanes' loads are -- one column on the paths to every
// target (a hub) no longer serialises its lane -- and does not depend on how the work
// is shared out.
template <typename DT, int VN>
__device__ __forceinline__ void pair_item(const PairArgs<DT>& a, int s, int U_, int x0, const TgtFast<DT>* s_fa,
                                          const TgtSlow* s_sl, ff (*s_acc)[kPairThreads], PairQueue& wq) {
    constexpr int kPairGroup = PairGroup<VN>::value;
    static_assert(2 * VN * kPairGroup <= 32 && VN <= 8, "a group's matches fit one 32-bit mask");
    using U = typename Unsigned<DT>::T;
    constexpr unsigned kMask = (1u << VN) - 1u;
    const int n = a.n;
    const int lane = threadIdx.x & 31;
    const size_t rs = (size_t)s * n;
    const bool active = x0 < n;   // the warp runs the item together (the queue needs every lane)
    DVec<DT, VN> dsn, dso;
    unsigned bs = 0;
    if (active) {
        dsn.load(a.D + rs + x0);
        bs = chg_bits<VN>(a.chg, a.words, s, x0);
        dso = dsn;
        if (bs) patch_old<DT, VN>(dso, bs, a.oD + rs, x0);
        if (s >= x0 && s < x0 + VN) {
#pragma unroll
            for (int q = 0; q < VN; ++q)
                if (x0 + q == s) dso.v[q] = dsn.v[q] = (DT)Inf<DT>::v;
        }
    }
    unsigned any = 0;   // bit q: s_acc[q][tid] holds the sum of column x0 + q
    int qlen = 0;       // warp-uniform
    const int lane_x0 = x0 - lane * VN;   // column of lane 0's first vector
    // evaluate the queued terms (all lanes), then add each lane's terms in queue order
    auto flush = [&]() {
        __syncwarp();
        for (int e = lane; e < qlen; e += 32) {
            const uint32_t en = wq.e[e];
            const int L = en & 31, q = (en >> 5) & 7, u = (en >> 8) & 127;
            const bool is_new = (en >> 15) & 1u;
            const int x = lane_x0 + L * VN + q;
            const TgtSlow& sl = s_sl[u];
            const size_t rt = (size_t)sl.rt;
            const uint64_t ssx = (!is_new && ((en >> 16) & 1u)) ? a.oS[rs + x] : a.S[rs + x];
            const uint64_t stx = (!is_new && ((en >> 17) & 1u)) ? a.oS[rt + x] : a.S[rt + x];
            ff t = pair_term(ssx, stx, is_new ? sl.rnew : sl.rold);
            if (!is_new) t = ff{-t.hi, -t.lo};
            wq.term[e] = t;
        }
        __syncwarp();
        for (int e = 0; e < qlen; ++e) {
            const uint32_t en = wq.e[e];
            if ((int)(en & 31) == lane) {
                const int q = (en >> 5) & 7;
                const ff prev = ((any >> q) & 1u) ? s_acc[q][threadIdx.x] : ff{0.f, 0.f};
                s_acc[q][threadIdx.x] = ff_add(prev, wq.term[e]);
                any |= 1u << q;
            }
        }
        __syncwarp();
        qlen = 0;
    };
    const int wofs = x0 >> 5, bsh = x0 & 31;
    for (int u0 = 0; u0 < U_; u0 += kPairGroup) {
        DVec<DT, VN> dtg[kPairGroup];
        unsigned btg[kPairGroup];
        if (active) {
#pragma unroll
            for (int k = 0; k < kPairGroup; ++k)
                if (u0 + k < U_) {
                    const TgtFast<DT> f = s_fa[u0 + k];
                    dtg[k].load(f.Dt + x0);
                    btg[k] = f.Ct[wofs];
                }
        }
        uint32_t mm = 0, btp = 0;
#pragma unroll
        for (int k = 0; k < kPairGroup; ++k) {
            if (!active || u0 + k >= U_) break;
            const TgtFast<DT> f = s_fa[u0 + k];
            const DVec<DT, VN>& dtn = dtg[k];
            const unsigned bt = (btg[k] >> bsh) & kMask;
            DVec<DT, VN> dto = dtn;
            bool hit = false;
            if (!(bs | bt)) {
                // no saved values at these columns: the old and new sums are the same
#pragma unroll
                for (int q = 0; q < VN; ++q) {
                    const U sum = (U)dsn.v[q] + (U)dtn.v[q];
                    hit |= (sum == (U)f.dold) | (sum == (U)f.dnew);
                }
            } else {
                if (bt) patch_old<DT, VN>(dto, bt, a.oD + (f.Dt - a.D), x0);
#pragma unroll
                for (int q = 0; q < VN; ++q) {
                    hit |= (U)dso.v[q] + (U)dto.v[q] == (U)f.dold;
                    hit |= (U)dsn.v[q] + (U)dtn.v[q] == (U)f.dnew;
                }
            }
            if (!hit) continue;
            const unsigned mo = on_path<DT, VN>(dso, dto, (U)f.dold);
            const unsigned mn = on_path<DT, VN>(dsn, dtn, (U)f.dnew);
            mm |= (mo | (mn << VN)) << (2 * VN * k);
            btp |= bt << (VN * k);
        }
        // append this group's matches, each lane's in (target, state, q) order; a group
        // that does not fit goes in parts, with a flush in between
        while (__any_sync(0xffffffffu, mm != 0)) {
            if (qlen == kPairQueue) flush();
            const int cnt = __popc(mm);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            const int space = kPairQueue - qlen;
            for (int pos = incl - cnt; mm && pos < space; ++pos) {
                const int b = __ffs(mm) - 1;
                mm &= mm - 1;
                const int k = b / (2 * VN), j = b - k * 2 * VN;
                const unsigned is_new = j >= VN ? 1u : 0u;
                const int q = is_new ? j - VN : j;
                wq.e[qlen + pos] = (uint32_t)lane | ((uint32_t)q << 5) | ((uint32_t)(u0 + k) << 8) | (is_new << 15) |
                                   (((bs >> q) & 1u) << 16) | (((btp >> (VN * k + q)) & 1u) << 17);
            }
            qlen += min(tot, space);
            __syncwarp();
        }
    }
    if (qlen) flush();
#pragma unroll
    for (int q = 0; q < VN; ++q)
        if ((any >> q) & 1u) {
            const ff acc = s_acc[q][threadIdx.x];
            ff* p = a.Dl + rs + x0 + q;
            *p = ff_add(*p, acc);
            bc_fix_add(a.bcfix, x0 + q, acc);
        }
}

// Work item = (listed row s, chunk of CW = threads x VN columns), in row-major order;
// an item weighs the row's targets plus one.  The items are cut into kPairPieces x grid
// pieces of equal weight (a piece runs the items whose start falls in it, so rows with
// many targets spread over several pieces).  The first wave of CTAs takes the first
// pieces and every CTA that finishes one takes the next from a counter: item costs
// vary more than their weights (the matches, the per-item loads), and a static share
// per CTA left half of the SMs idle for half of the kernel.  The plan of a row is
// staged in shared memory when the CTA meets the row.
template <typename DT, int VN>
__global__ void __launch_bounds__(kPairThreads, kPairCtasPerSm) k_pairdep(PairArgs<DT> a) {
    pdl_enter();
    __shared__ TgtFast<DT> s_fa[kPairCap];
    __shared__ TgtSlow s_sl[kPairCap];
    __shared__ ff s_acc[VN][kPairThreads];   // per thread: the sums of its VN columns
    __shared__ PairQueue s_wq[kPairThreads / 32];
    __shared__ int s_i, s_c, s_p;
    if (*a.err) return;
    if (a.gate && *a.gate == 0) return;
    constexpr int CW = kPairThreads * VN;
    const int n = a.n;
    const int nchunks = (n + CW - 1) / CW;
    const int cnt = *a.pcount;
    const int64_t W = a.wpre[cnt];
    const int npieces = gridDim.x * kPairPieces;
    int cur = -1, s = -1, U_ = 0;   // the row whose plan is staged
    for (int piece = blockIdx.x; piece < npieces;) {
        const int64_t lo = W * piece / npieces, hi = W * (piece + 1) / npieces;
        if (lo < hi) {   // block-uniform
            if (threadIdx.x == 0) {
                // last row whose items start at or before lo: wpre[L] <= lo < wpre[R]
                int L = 0, R = cnt;
                while (R - L > 1) {
                    const int m = (L + R) >> 1;
                    if (a.wpre[m] <= lo) L = m; else R = m;
                }
                const int64_t wc = (a.wpre[L + 1] - a.wpre[L]) / nchunks;   // > 0: lo lies in row L
                s_i = L;
                s_c = (int)((lo - a.wpre[L] + wc - 1) / wc);
            }
            __syncthreads();
            int i = s_i, c = s_c;
            int64_t wc = (a.wpre[i + 1] - a.wpre[i]) / nchunks;
            for (;;) {
                if (c >= nchunks) {   // next row with items (block-uniform)
                    do {
                        ++i;
                    } while (i < cnt && a.wpre[i + 1] == a.wpre[i]);
                    if (i >= cnt) break;
                    wc = (a.wpre[i + 1] - a.wpre[i]) / nchunks;
                    c = 0;
                }
                if (a.wpre[i] + (int64_t)c * wc >= hi) break;
                if (i != cur) {
                    cur = i;
                    s = a.prows[i];
                    U_ = (int)wc - 1;
                    __syncthreads();   // the previous row's plan is no longer read
                    if (threadIdx.x < U_) {
                        const PairTgt p = a.plan[(size_t)s * a.tcap + threadIdx.x];
                        const size_t rt = (size_t)p.t * n;
                        s_fa[threadIdx.x] =
                            TgtFast<DT>{a.D + rt, a.chg + (size_t)p.t * a.words, (DT)p.dold, (DT)p.dnew};
                        s_sl[threadIdx.x] = TgtSlow{(int64_t)rt, p.rold, p.rnew};
                    }
                    __syncthreads();
                }
                const int x0 = c * CW + threadIdx.x * VN;
                ++c;
                // a warp with at least one column in the row runs the item (all its lanes)
                if (x0 - (int)(threadIdx.x & 31) * VN < n)
                    pair_item<DT, VN>(a, s, U_, x0, s_fa, s_sl, s_acc, s_wq[threadIdx.x >> 5]);
            }
        }
        // the next piece: the first wave takes pieces 0 .. grid-1, later ones go in
        // order to the CTAs that finish first
        if (threadIdx.x == 0) s_p = gridDim.x + atomicAdd(a.next_piece, 1);
        __syncthreads();
        piece = s_p;
        __syncthreads();   // s_p is read by all before thread 0 writes it again
    }
}

// BC (hi, lo) += the fixed-point change of each column, then the pair is zeroed for the
// next update: B's high bits are carried into A (A' = A + (B >> 32), B' = B mod 2^32),
// so A' * 2^-24 and B' * 2^-56 are exact doubles, added with TwoSum as in
// dev_bc_finish.
__device__ __forceinline__ void dev_bc_fix(int t, int64_t* fix, double* hi, double* lo) {
    const longlong2 f = *reinterpret_cast<const longlong2*>(fix + 2 * (size_t)t);
    if (f.x == 0 && f.y == 0) return;
    *reinterpret_cast<longlong2*>(fix + 2 * (size_t)t) = make_longlong2(0, 0);
    const long long A = f.x + (f.y >> 32);
    const long long B = f.y & 0xFFFFFFFFll;
    const double x1 = (double)A * 0x1p-24;
    const double x2 = (double)B * 0x1p-56;
    const double h = hi[t];
    const double s = h + x1;
    const double bp = s - h;
    const double e = (h - (s - bp)) + (x1 - bp);
    hi[t] = s;
    lo[t] += e + x2;
}

__global__ void k_bc_fix(int n, int64_t* fix, double* hi, double* lo, const int32_t* err) {
    pdl_enter();
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dev_bc_fix(t, fix, hi, lo);
}

// ------------------------------------------------------------------ launches

PairRec pair_rec(const Dev& d) { return make_pair_rec(d); }

void launch_pair_lists(const Dev& d) {
    launch_k(k_pair_lists, 1, kCompactThreads, 0, d.st, d.n, d.changed, d.tcnt, d.tcap, d.acc_rows, d.counts + 1,
                                                  d.full_rows, d.counts + 3, d.stats, d.err);
}

void launch_pair_clear(const Dev& d) {
    launch_k(k_pair_clear, d.nsm * 4, 256, 0, d.st, d.acc_rows, d.counts + 1, d.tcnt, d.tlist, d.tcap, d.chg,
                                              d.chg_words, d.counts + 3, d.stats);
}

template <typename DT>
__host__ __device__ inline PairArgs<DT> pair_args(const Dev& d) {
    PairArgs<DT> a;
    a.n = d.n;
    a.D = (const DT*)d.D;
    a.S = d.S;
    a.chg = d.chg;
    a.words = d.chg_words;
    a.oD = (const DT*)d.oldD;
    a.oS = d.oldS;
    a.tcnt = d.tcnt;
    a.tlist = d.tlist;
    a.plan = reinterpret_cast<PairTgt*>(d.plan);
    a.wpre = d.pair_w;
    a.next_piece = d.counts + 4;
    a.prows = d.pair_rows;
    a.pcount = d.counts + 5;
    a.gate = nullptr;
    a.tcap = d.tcap;
    a.rows = d.acc_rows;
    a.count = d.counts + 1;
    a.Dl = d.Dl;
    a.bcfix = d.bcfix;
    a.err = d.err;
    return a;
}

// ------------------------------------------------------------------ batches
//
// The pair corrections of round r of a batch, for every graph that has them (the rest of
// the round is in k_batch.cu).  Each kernel runs the single-graph kernel's device
// function on the concatenated work of all graphs, a task mapped to its graph by binary
// search over prefix offsets, so a graph's result in a batch is bit-identical to its
// result alone.  The column test always serves a batch (the DAG walks are for graphs far
// larger than a batch's).

__device__ __forceinline__ bool batch_pair_graph(const BatchArgs& b, int r, int g) {
    const Dev& d = b.devs[g];
    return d.pair_on && b.upd[(int64_t)r * b.G + g].present && *d.err == 0;
}

// One CTA per graph in turn: the row lists of its corrections (k_pair_lists).
__global__ void __launch_bounds__(kCompactThreads) kb_pair_lists(BatchArgs b, int r) {
    __shared__ int32_t wsum[32];
    __shared__ int32_t s_total;
    for (int g = blockIdx.x; g < b.G; g += gridDim.x) {
        const Dev& d = b.devs[g];
        if (!d.pair_on || b.upd[(int64_t)r * b.G + g].present == 0) continue;   // block-uniform
        dev_pair_lists(d.n, d.changed, d.tcnt, d.tcap, d.acc_rows, d.counts + 1, d.full_rows, d.counts + 3, d.stats,
                       *d.err != 0, wsum, s_total);
        __syncthreads();
    }
}

// A warp per listed row of every graph (k_pair_plan); plan_pr offsets the rows.
template <typename DT>
__global__ void __launch_bounds__(kPlanThreads) kb_pair_plan(BatchArgs b) {
    __shared__ int32_t s_val[kPlanThreads / 32][kPairCap];
    const int G = b.G;
    const int64_t total = b.plan_pr[G];
    const int wib = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * (kPlanThreads / 32);
    for (int64_t j = (int64_t)blockIdx.x * (kPlanThreads / 32) + wib; j < total; j += nw) {
        const int g = graph_of(b.plan_pr, G, j);
        const Dev& d = b.devs[g];
        const PairArgs<DT> a = pair_args<DT>(d);
        dev_pair_plan_row<DT>(a, d.acc_rows[j - b.plan_pr[g]], s_val[wib]);
    }
}

// One CTA per graph in turn: rows most targets first and their weight prefix
// (k_pair_weights), with the graph's own columns per thread.
__global__ void __launch_bounds__(1024) kb_pair_weights(BatchArgs b, int r, int scap) {
    __shared__ PairWeightsSmem sm;
    extern __shared__ int32_t s_stage[];   // 2 * scap ints
    for (int g = blockIdx.x; g < b.G; g += gridDim.x) {
        if (!batch_pair_graph(b, r, g)) continue;   // block-uniform
        const Dev& d = b.devs[g];
        const int cw = kPairThreads * pair_vn(d.dbytes, d.n);
        const int nchunks = (d.n + cw - 1) / cw;
        dev_pair_weights(d.acc_rows, d.counts + 1, d.tcnt, d.tcap, nchunks, d.pair_rows, d.counts + 5, d.pair_w,
                         d.stats, d.counts + 4, nullptr, nullptr, sm, s_stage, s_stage + scap, scap);
        __syncthreads();
    }
}

// The column test (k_pairdep) over the graphs whose columns per thread are VN: their
// weight lines laid end to end (plan_pw of the class), cut into kPairPieces x grid pieces
// of equal weight; a piece runs the items whose start falls in it, across row and graph
// boundaries, and later pieces go to the CTAs that finish first (counter pctr).
template <typename DT, int VN>
__global__ void __launch_bounds__(kPairThreads, kPairCtasPerSm) kb_pairdep(BatchArgs b, int cls) {
    __shared__ TgtFast<DT> s_fa[kPairCap];
    __shared__ TgtSlow s_sl[kPairCap];
    __shared__ ff s_acc[VN][kPairThreads];
    __shared__ PairQueue s_wq[kPairThreads / 32];
    __shared__ int s_g, s_i, s_c, s_p;
    constexpr int CW = kPairThreads * VN;
    const int G = b.G;
    const int64_t* off = b.plan_pw + (int64_t)cls * (G + 1);
    const int64_t W = off[G];
    const int npieces = gridDim.x * kPairPieces;
    int cg = -1;                     // the graph whose arguments are loaded
    int sg = -1, cur = -1, s = -1;   // the graph and row whose plan is staged
    int U_ = 0, nchunks = 1, cnt = 0;
    PairArgs<DT> a{};
    for (int piece = blockIdx.x; piece < npieces;) {
        const int64_t lo = W * piece / npieces, hi = W * (piece + 1) / npieces;
        if (lo < hi) {   // block-uniform
            if (threadIdx.x == 0) {
                // the graph holding lo (off[g] <= lo < off[g + 1]), then its last row whose
                // items start at or before lo
                const int g = graph_of(off, G, lo);
                const Dev& d = b.devs[g];
                const int nch = (d.n + CW - 1) / CW;
                const int64_t l = lo - off[g];
                int L = 0, R = d.counts[5];
                while (R - L > 1) {
                    const int m = (L + R) >> 1;
                    if (d.pair_w[m] <= l) L = m; else R = m;
                }
                const int64_t wc = (d.pair_w[L + 1] - d.pair_w[L]) / nch;   // > 0: l lies in row L
                s_g = g;
                s_i = L;
                s_c = (int)((l - d.pair_w[L] + wc - 1) / wc);
            }
            __syncthreads();
            int g = s_g, i = s_i, c = s_c;
            if (g != cg) {
                cg = g;
                a = pair_args<DT>(b.devs[g]);
                nchunks = (a.n + CW - 1) / CW;
                cnt = *a.pcount;
            }
            int64_t wc = (a.wpre[i + 1] - a.wpre[i]) / nchunks;
            for (;;) {
                if (c >= nchunks) {   // next row with items, in this graph or the next ones (block-uniform)
                    do {
                        ++i;
                    } while (i < cnt && a.wpre[i + 1] == a.wpre[i]);
                    while (i >= cnt) {
                        do {
                            ++g;
                        } while (g < G && off[g + 1] == off[g]);
                        if (g >= G) break;
                        cg = g;
                        a = pair_args<DT>(b.devs[g]);
                        nchunks = (a.n + CW - 1) / CW;
                        cnt = *a.pcount;
                        i = 0;
                        while (i < cnt && a.wpre[i + 1] == a.wpre[i]) ++i;
                    }
                    if (g >= G) break;
                    wc = (a.wpre[i + 1] - a.wpre[i]) / nchunks;
                    c = 0;
                }
                if (off[g] + a.wpre[i] + (int64_t)c * wc >= hi) break;
                if (i != cur || g != sg) {
                    cur = i;
                    sg = g;
                    s = a.prows[i];
                    U_ = (int)wc - 1;
                    __syncthreads();   // the previous row's plan is no longer read
                    if (threadIdx.x < U_) {
                        const PairTgt p = a.plan[(size_t)s * a.tcap + threadIdx.x];
                        const size_t rt = (size_t)p.t * a.n;
                        s_fa[threadIdx.x] =
                            TgtFast<DT>{a.D + rt, a.chg + (size_t)p.t * a.words, (DT)p.dold, (DT)p.dnew};
                        s_sl[threadIdx.x] = TgtSlow{(int64_t)rt, p.rold, p.rnew};
                    }
                    __syncthreads();
                }
                const int x0 = c * CW + threadIdx.x * VN;
                ++c;
                if (x0 - (int)(threadIdx.x & 31) * VN < a.n)
                    pair_item<DT, VN>(a, s, U_, x0, s_fa, s_sl, s_acc, s_wq[threadIdx.x >> 5]);
            }
        }
        if (threadIdx.x == 0) s_p = gridDim.x + atomicAdd(b.pctr + cls, 1);
        __syncthreads();
        piece = s_p;
        __syncthreads();
    }
}

// BC += the fixed-point change of each column of every graph with corrections (k_bc_fix).
__global__ void kb_bc_fix(BatchArgs b, int r) {
    const int G = b.G;
    const int64_t total = b.coff[G];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int g = graph_of(b.coff, G, j);
        if (!batch_pair_graph(b, r, g)) continue;
        const Dev& d = b.devs[g];
        dev_bc_fix((int)(j - b.coff[g]), d.bcfix, d.bc_hi, d.bc_lo);
    }
}

// The per-update records back to zero, a warp per listed row (k_pair_clear).
__global__ void kb_pair_clear(BatchArgs b, int r) {
    const int G = b.G;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
        if (batch_pair_graph(b, r, g)) b.devs[g].stats[7] += b.devs[g].counts[3];
    const int64_t total = b.plan_pr[G];
    const int wpb = blockDim.x >> 5;
    for (int64_t j = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); j < total; j += (int64_t)gridDim.x * wpb) {
        const int g = graph_of(b.plan_pr, G, j);
        const Dev& d = b.devs[g];
        dev_pair_clear_row(d.acc_rows[j - b.plan_pr[g]], d.tcnt, d.tlist, d.tcap, d.chg, d.chg_words);
    }
}

void batch_pair_lists(const BatchArgs& b, const BatchLaunch& L, int r, cudaStream_t st) {
    kb_pair_lists<<<std::min(b.G, L.nsm * 2), kCompactThreads, 0, st>>>(b, r);
}

template <typename DT>
static void batch_pairs(const BatchArgs& b, const BatchLaunch& L, int r, cudaStream_t st) {
    const int G = b.G, nsm = L.nsm;
    batch_plan(b, r, 3, 2, b.plan_pr, L.scan_unroll, st);
    kb_pair_plan<DT><<<nsm * 8, kPlanThreads, 0, st>>>(b);
    const int scap = weights_stage(b.n_max);
    kb_pair_weights<<<std::min(G, nsm * 2), 1024, 2 * sizeof(int32_t) * (size_t)scap, st>>>(b, r, scap);
    const int pgrid = nsm * kPairCtasPerSm;
    for (int c = 0; c < kPairClasses; ++c) {
        if (!((L.pair_classes >> c) & 1)) continue;
        batch_plan(b, r, 4 + c, 2, b.plan_pw + (int64_t)c * (G + 1), L.scan_unroll, st);
        if constexpr (sizeof(DT) == 4) {
            if (c == 0) kb_pairdep<DT, 8><<<pgrid, kPairThreads, 0, st>>>(b, c);
            else if (c == 1) kb_pairdep<DT, 4><<<pgrid, kPairThreads, 0, st>>>(b, c);
            else kb_pairdep<DT, 1><<<pgrid, kPairThreads, 0, st>>>(b, c);
        } else {
            if (c == 0) kb_pairdep<DT, 2><<<pgrid, kPairThreads, 0, st>>>(b, c);
            else kb_pairdep<DT, 1><<<pgrid, kPairThreads, 0, st>>>(b, c);
        }
    }
    kb_bc_fix<<<nsm * 4, 256, 0, st>>>(b, r);
    kb_pair_clear<<<nsm * 4, 256, 0, st>>>(b, r);
}

void batch_pair_launches(const BatchArgs& b, const BatchLaunch& L, int r, int dbytes, cudaStream_t st) {
    if (dbytes == 4) batch_pairs<int32_t>(b, L, r, st);
    else batch_pairs<int64_t>(b, L, r, st);
}

// ------------------------------------------------------------------ DAG walks
//
// The same corrections with the columns found by walking the shortest-path DAG instead
// of testing every column.  The columns on a shortest s-t path of a state are the
// vertices from which t is reachable in DAG(s) of that state (Eq. 1: the arcs (x, y)
// with d(s,x) + w(x,y) = d(s,y)), so a walk backwards from t over those arcs visits
// exactly them -- about 20 per changed pair against n column tests.  In G_D of an
// undirected graph the arcs into y are y's own arcs reversed (same weight), read from
// the E* superset; before the update E*+ held every arc of the old E* (arcs are only
// added between re-layouts, and a re-layout keeps the arcs of the state it reads), and
// the arcs of the update itself carry their old weight from `upd` (or did not exist).
//
// Phase 1 (k_walk_units): a unit is one changed pair (row s, target); any free warp
// takes the next units, walks both states level by level (the arcs of a level's
// vertices spread over the lanes) and appends the vertices found -- t excluded -- to a
// global buffer, recording each walk's segment.  Phase 2 (k_walk_rows): one CTA per row;
// its warps share out the row's segments, evaluate the terms and add them to a per-CTA
// row of fixed-point column sums (integer atomics, so the sums do not depend on which
// warp adds first), which is then added to delta_s and to BC's fixed-point change.  If
// the buffer overflows, phase 2 does nothing and the column test runs instead.

template <typename DT>
struct WalkArgs {
    const int32_t* e_off;
    const int32_t* e_len;
    const Arc<DT>* e_arc;
    int32_t* list;      // [walk warps * n] vertices of a walk, level by level (phase 1)
    int32_t* buf;       // [cap] vertices found by the walks of the update's units
    int64_t cap;
    int32_t* useg;      // [n * tcap * 4] per unit: start and length of the old, then the new walk
    int64_t* acc2;      // [CTAs * 2n] per CTA: fixed-point column sums of a row (zero between rows)
    int32_t* tl;        // [CTAs * n] per CTA: columns of the row with a sum
    int32_t* ctl;       // [0] units handed out [1] rows handed out [2..3] buffer used (64-bit) [4] overflow
                        // [5] light rows handed out [6] mid-size rows handed out
    int32_t* rowE;      // [n] per listed row: vertices its walks found (zeroed by k_pair_weights)
    int64_t* stats;     // [10] pairs walked [11] vertices found [12] arcs examined
    int nchunks;        // items per row in the weight prefix wpre
    WalkUpd upd;
};

constexpr int kWalkWarps = kWalkThreads / 32;
constexpr int kWalkGrab = 1;         // units a warp takes at a time (unit costs vary too much for more)
constexpr int kWalkLightRowMax = 128;   // rows whose walks found at most this many vertices: light CTAs
constexpr int kWalkMidRowMax = 512;     // up to this many: mid-size CTAs; more: k_walk_rows

// d(s,x) and sigma_sx of a state: the saved values where the pair changed in this update
// (old state).  The change-map word and the current value are loaded together (one
// round trip); the saved value is read only where the bit is set, rarely.
template <typename DT>
__device__ __forceinline__ int64_t walk_d(const PairArgs<DT>& a, size_t rs, int s, int x, bool is_new) {
    const size_t i = rs + x;
    const int64_t cur = (int64_t)a.D[i];
    if (is_new) return cur;
    const uint32_t word = a.chg[(size_t)s * a.words + (x >> 5)];
    return ((word >> (x & 31)) & 1u) ? (int64_t)a.oD[i] : cur;
}
template <typename DT>
__device__ __forceinline__ uint64_t walk_sigma(const PairArgs<DT>& a, size_t rs, int s, int x, bool is_new) {
    const size_t i = rs + x;
    const uint64_t cur = a.S[i];
    if (is_new) return cur;
    const uint32_t word = a.chg[(size_t)s * a.words + (x >> 5)];
    return ((word >> (x & 31)) & 1u) ? a.oS[i] : cur;
}

// First unit of row index r: the targets of the rows before it (wpre counts T + 1 per
// row and item chunk).
template <typename DT>
__device__ __forceinline__ int64_t unit_start(const PairArgs<DT>& a, int nchunks, int r) {
    return a.wpre[r] / nchunks - r;
}

template <typename DT>
__global__ void __launch_bounds__(kWalkThreads, kWalkCtasPerSm) k_walk_units(PairArgs<DT> a, WalkArgs<DT> w) {
    pdl_enter();
    extern __shared__ uint32_t wbits[];   // per warp: visited bits
    if (*a.err) return;
    const int n = a.n, words = a.words;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t INF = Inf<DT>::v;
    uint32_t* vis = wbits + (size_t)wib * words;
    int32_t* list = w.list + ((size_t)blockIdx.x * kWalkWarps + wib) * n;
    for (int i = lane; i < words; i += 32) vis[i] = 0u;
    __syncwarp();
    const int cnt = *a.pcount;
    const int64_t nunits = unit_start<DT>(a, w.nchunks, cnt);
    const int v = w.upd.v;
    // this warp's block of the buffer: [bnext, bend)
    long long bnext = 0, bend = 0;
    __shared__ unsigned long long s_cnt[kWalkWarps][2];   // per warp: vertices found, arcs examined
    if (lane == 0) s_cnt[wib][0] = s_cnt[wib][1] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(w.stats + 10), (unsigned long long)nunits);
    for (;;) {
        int g0 = 0;
        if (lane == 0) g0 = atomicAdd(w.ctl, kWalkGrab);
        g0 = __shfl_sync(0xffffffffu, g0, 0);
        if (g0 >= nunits) break;
        for (int64_t id = g0; id < min((int64_t)g0 + kWalkGrab, nunits); ++id) {
            // the unit's row: the last r with unit_start(r) <= id, i.e. wpre[r] <= (id + r) *
            // nchunks (wpre[r] is a multiple of nchunks)
            int L = 0, R = cnt;
            while (R - L > 1) {
                const int m = (L + R) >> 1;
                if (a.wpre[m] <= (id + m) * w.nchunks) L = m; else R = m;
            }
            const int s = a.prows[L];
            const int u = (int)(id - unit_start<DT>(a, w.nchunks, L));
            const PairTgt& pt = a.plan[(size_t)s * a.tcap + u];
            const int t = pt.t;
            const size_t rs = (size_t)s * n;
            for (int stt = 0; stt < 2; ++stt) {
                const bool is_new = stt == 1;
                int found = 0;   // warp-uniform
                if ((is_new ? pt.dnew : pt.dold) >= 0) {
                    if (lane == 0) {
                        list[0] = t;
                        vis[t >> 5] |= 1u << (t & 31);
                    }
                    __syncwarp();
                    int head = 0, tail = 1;   // list[head, tail) is the current level
                    while (head < tail) {
                        const int l0 = head, l1 = tail;
                        head = l1;
                        for (int b0 = l0; b0 < l1; b0 += 32) {
                            const int nb = min(32, l1 - b0);
                            int y = 0, off = 0, len = 0;
                            int64_t dy = 0;
                            if (lane < nb) {
                                y = list[b0 + lane];
                                off = w.e_off[y];
                                len = w.e_len[y];
                                dy = walk_d<DT>(a, rs, s, y, is_new);
                            }
                            int incl = len;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const int z = __shfl_up_sync(0xffffffffu, incl, o);
                                if (lane >= o) incl += z;
                            }
                            const int tot = __shfl_sync(0xffffffffu, incl, 31);
                            const int excl = incl - len;
                            // first step of the owner search: the largest power of two below nb
                            const int top = nb > 1 ? 1 << (31 - __clz(nb - 1)) : 0;
                            if (lane == 0) s_cnt[wib][1] += (unsigned)tot;
                            for (int k0 = 0; k0 < tot; k0 += 32) {   // the batch's arcs, one per lane
                                const int k = k0 + lane;
                                int j = 0;   // owner: the last lane j < nb whose arcs start at or before k
                                for (int step = top; step >= 1; step >>= 1) {
                                    const int c = j + step;
                                    const int ex = __shfl_sync(0xffffffffu, excl, c & 31);
                                    if (c < nb && ex <= k) j = c;
                                }
                                const int yj = __shfl_sync(0xffffffffu, y, j);
                                const int offj = __shfl_sync(0xffffffffu, off, j);
                                const int exj = __shfl_sync(0xffffffffu, excl, j);
                                const int64_t dyj = __shfl_sync(0xffffffffu, dy, j);
                                bool fresh = false;
                                int x = -1;
                                if (k < tot) {
                                    const Arc<DT> arc = w.e_arc[offj + (k - exj)];
                                    x = (int)arc.dst;
                                    int64_t wv = (int64_t)arc.w;
                                    if (!is_new && (yj == v || x == v)) {
                                        const int o = yj == v ? x : yj;
                                        for (int e = 0; e < w.upd.k; ++e)
                                            if (w.upd.x[e] == o) wv = w.upd.wold[e];
                                    }
                                    if (x >= 0 && x != s && wv >= 0 && wv <= dyj) {   // else no predecessor
                                        const int64_t dx = walk_d<DT>(a, rs, s, x, is_new);
                                        if (dx != INF && dx + wv == dyj) {
                                            const uint32_t bit = 1u << (x & 31);
                                            fresh = !(atomicOr(&vis[x >> 5], bit) & bit);
                                        }
                                    }
                                }
                                const unsigned bal = __ballot_sync(0xffffffffu, fresh);
                                if (fresh) list[tail + __popc(bal & lt)] = x;
                                tail += __popc(bal);
                            }
                        }
                        __syncwarp();
                    }
                    found = tail - 1;
                    if (lane == 0) s_cnt[wib][0] += (unsigned)found;
                    // the walk's vertices (t excluded) into the buffer
                    // room in the warp's block, else a new block (a walk longer than a block
                    // gets a block of its own size); one atomic per block, not per walk
                    if (bnext + found > bend) {
                        const long long want = found > kWalkBlock ? found : kWalkBlock;
                        long long b = 0;
                        if (lane == 0)
                            b = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(w.ctl + 2),
                                                     (unsigned long long)want);
                        bnext = __shfl_sync(0xffffffffu, b, 0);
                        bend = bnext + want;
                    }
                    const long long base = bnext;
                    bnext += found;
                    if (base + found <= w.cap) {
                        for (int i = lane; i < found; i += 32) w.buf[base + i] = list[1 + i];
                    } else {
                        if (lane == 0) w.ctl[4] = 1;
                        found = 0;
                    }
                    if (lane == 0) w.useg[id * 4 + 2 * stt] = (int32_t)base;
                    for (int i = lane; i < tail; i += 32) vis[list[i] >> 5] = 0u;
                    __syncwarp();
                }
                if (lane == 0) {
                    w.useg[id * 4 + 2 * stt + 1] = found;
                    if (found) atomicAdd(w.rowE + L, found);
                }
            }
        }
    }
    if (lane == 0 && (s_cnt[wib][0] | s_cnt[wib][1])) {
        atomicAdd(reinterpret_cast<unsigned long long*>(w.stats + 11), s_cnt[wib][0]);
        atomicAdd(reinterpret_cast<unsigned long long*>(w.stats + 12), s_cnt[wib][1]);
    }
}

// A term v = hi + lo (|v| <= 1 + 2^-40, a pair dependency) as a fixed-point pair (units
// of 2^-24 and 2^-56, as in bc_fix_add) in single precision only (fp64 runs at a small
// fraction of the fp32 rate here): with h = hi * 2^24 and a = rint(h), h - a is exact
// (|h| <= 2^24 + 1), and (h - a) * 2^32 and lo * 2^56 are exact scalings, each rounded to
// an integer once, so B is within one unit of v * 2^56 - A * 2^32; a carry keeps
// |B| <= 2^31.
__device__ __forceinline__ void fix_split(ff v, long long* A, long long* B) {
    const float h = v.hi * 0x1p24f;
    const float a = rintf(h);
    long long b = __float2ll_rn((h - a) * 0x1p32f) + __float2ll_rn(v.lo * 0x1p56f);
    const long long c = (b + (1ll << 31)) >> 32;
    *A = (long long)__float2int_rn(a) + c;
    *B = b - (c << 32);
}

// A column's fixed-point sum (A in units of 2^-24 plus B in units of 2^-56, 0 <= B <
// 2^32, |A| < 2^47) as a float-float: four exactly representable parts, added with
// error-free sums.
__device__ __forceinline__ ff fix_to_ff(long long A, long long B) {
    const float p0 = (float)(int)(A >> 24);
    const float p1 = (float)(int)(A & 0xFFFFFF) * 0x1p-24f;
    const float p2 = (float)(int)(B >> 24) * 0x1p-32f;
    const float p3 = (float)(int)(B & 0xFFFFFF) * 0x1p-56f;
    return ff_add(two_sum(p0, p1), two_sum(p2, p3));
}

template <typename DT>
__global__ void __launch_bounds__(kWalkThreads, kWalkRowCtasPerSm) k_walk_rows(PairArgs<DT> a, WalkArgs<DT> w) {
    pdl_enter();
    extern __shared__ uint32_t tbits[];   // touched columns of the row
    __shared__ int s_r, s_nt;
    if (*a.err) return;
    if (*(volatile int32_t*)(w.ctl + 4)) return;   // overflow: the column test does the update
    const int n = a.n, words = a.words;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    long long* acc = reinterpret_cast<long long*>(w.acc2) + (size_t)blockIdx.x * 2 * n;
    int32_t* tl = w.tl + (size_t)blockIdx.x * n;
    for (int i = threadIdx.x; i < words; i += blockDim.x) tbits[i] = 0u;
    const int cnt = *a.pcount;
    for (;;) {
        if (threadIdx.x == 0) {
            s_r = atomicAdd(w.ctl + 1, 1);
            s_nt = 0;
        }
        __syncthreads();
        const int r = s_r;
        if (r >= cnt) break;
        if (w.rowE[r] <= kWalkMidRowMax) {   // none found, or taken by k_walk_rows_hash
            __syncthreads();
            continue;
        }
        const int s = a.prows[r];
        const int T = a.tcnt[s];
        const int64_t id0 = unit_start<DT>(a, w.nchunks, r);
        const size_t rs = (size_t)s * n;
        // the row's walks (2 per target) go to the warps in turn
        for (int q = wib; q < 2 * T; q += kWalkWarps) {
            const int u = q >> 1;
            const bool is_new = q & 1;
            const PairTgt& pt = a.plan[(size_t)s * a.tcap + u];
            const int64_t base = w.useg[(id0 + u) * 4 + 2 * (q & 1)];
            const int len = w.useg[(id0 + u) * 4 + 2 * (q & 1) + 1];
            const ff rcp = is_new ? pt.rnew : pt.rold;
            const size_t rt = (size_t)pt.t * n;
            for (int i = lane; i < len; i += 32) {
                const int x = w.buf[base + i];
                ff term = pair_term(walk_sigma<DT>(a, rs, s, x, is_new), walk_sigma<DT>(a, rt, pt.t, x, is_new), rcp);
                if (!is_new) term = ff{-term.hi, -term.lo};
                long long A, B;
                fix_split(term, &A, &B);
                atomicAdd(reinterpret_cast<unsigned long long*>(acc + 2 * x), (unsigned long long)A);
                if (B) atomicAdd(reinterpret_cast<unsigned long long*>(acc + 2 * x + 1), (unsigned long long)B);
                const uint32_t bit = 1u << (x & 31);
                if (!(atomicOr(&tbits[x >> 5], bit) & bit)) tl[atomicAdd(&s_nt, 1)] = x;
            }
        }
        __syncthreads();
        // the row's sums: delta_s and BC's change once per column, then the scratch back to zero
        const int nt = s_nt;
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            const int x = tl[i];
            const long long A0 = acc[2 * x], B0 = acc[2 * x + 1];
            acc[2 * x] = 0;
            acc[2 * x + 1] = 0;
            const long long A = A0 + (B0 >> 32), B = B0 & 0xFFFFFFFFll;   // 0 <= B < 2^32
            const ff v = fix_to_ff(A, B);
            ff* p = a.Dl + rs + x;
            *p = ff_add(*p, v);
            unsigned long long* bp = reinterpret_cast<unsigned long long*>(a.bcfix + 2 * (size_t)x);
            atomicAdd(bp, (unsigned long long)A);
            if (B) atomicAdd(bp + 1, (unsigned long long)B);
            tbits[x >> 5] = 0u;
        }
        __syncthreads();
    }
}

// The rows whose walks found at most kMaxE vertices (and more than kMinE) in CTAs of
// kThreads threads, many per SM so that many rows are in flight: the warps share out the
// row's walks and add the terms to a hash table of fixed-point column sums in shared
// memory (kHash slots, at least twice the vertices, so it never fills and every probe
// ends), which is then added to delta_s and to BC's change and emptied.  Two classes:
// light rows (at most 128 vertices; most rows, one to three changed targets) in 64-thread
// CTAs, 32 per SM, and mid-size rows (129 to 512 vertices) in 256-thread CTAs with a
// 1024-slot table, 8 per SM.  Rows with more vertices go to k_walk_rows.
template <int kThreads, int kCtas, int kHash, int kMinE, int kMaxE, int kCtl>
struct WalkHash {
    static constexpr int threads = kThreads, ctas = kCtas, hash = kHash, min_e = kMinE, max_e = kMaxE, ctl = kCtl;
    static_assert(kHash >= 2 * kMaxE, "the hash table stays at most half full");
    static_assert((kHash & (kHash - 1)) == 0, "a power of two");
    static constexpr int bits = kHash == 256 ? 8 : kHash == 512 ? 9 : kHash == 1024 ? 10 : kHash == 2048 ? 11 : 12;
    static_assert((1 << bits) == kHash, "table size");
    static constexpr size_t smem = (size_t)kHash * (2 * sizeof(unsigned long long) + sizeof(int32_t)) +
                                   (size_t)kMaxE * sizeof(int32_t);
};
using WalkLight = WalkHash<64, 32, 256, 0, kWalkLightRowMax, 5>;
using WalkMid = WalkHash<256, 8, 1024, kWalkLightRowMax, kWalkMidRowMax, 6>;
static_assert(WalkMid::smem * WalkMid::ctas <= 200 * 1024, "mid-size tables fit the SM");
static_assert(WalkMid::smem <= 48 * 1024 && WalkLight::smem <= 48 * 1024, "no opt-in shared memory needed");

template <typename DT, typename H>
__global__ void __launch_bounds__(H::threads, H::ctas) k_walk_rows_hash(PairArgs<DT> a, WalkArgs<DT> w) {
    pdl_enter();
    extern __shared__ unsigned long long hsm[];
    unsigned long long* hval = hsm;                                        // [2 * hash]
    int32_t* hkey = reinterpret_cast<int32_t*>(hsm + 2 * H::hash);         // [hash]
    int32_t* hused = hkey + H::hash;                                       // [max_e]
    __shared__ int s_r, s_nu;
    if (*a.err) return;
    if (*(volatile int32_t*)(w.ctl + 4)) return;   // overflow: the column test does the update
    const int n = a.n;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    constexpr int kW = H::threads / 32;
    for (int i = tid; i < H::hash; i += H::threads) {
        hkey[i] = -1;
        hval[2 * i] = 0ull;
        hval[2 * i + 1] = 0ull;
    }
    const int cnt = *a.pcount;
    for (;;) {
        if (tid == 0) {
            s_r = atomicAdd(w.ctl + H::ctl, 1);
            s_nu = 0;
        }
        __syncthreads();
        const int r = s_r;
        if (r >= cnt) break;
        const int e = w.rowE[r];
        if (e <= H::min_e || e > H::max_e || e == 0) {   // nothing found / another class
            __syncthreads();
            continue;
        }
        const int s = a.prows[r];
        const int T = a.tcnt[s];
        const int64_t id0 = unit_start<DT>(a, w.nchunks, r);
        const size_t rs = (size_t)s * n;
        for (int q = wib; q < 2 * T; q += kW) {
            const int u = q >> 1;
            const bool is_new = q & 1;
            const PairTgt& pt = a.plan[(size_t)s * a.tcap + u];
            const int64_t base = w.useg[(id0 + u) * 4 + 2 * (q & 1)];
            const int len = w.useg[(id0 + u) * 4 + 2 * (q & 1) + 1];
            const ff rcp = is_new ? pt.rnew : pt.rold;
            const size_t rt = (size_t)pt.t * n;
            for (int i = lane; i < len; i += 32) {
                const int x = w.buf[base + i];
                ff term = pair_term(walk_sigma<DT>(a, rs, s, x, is_new), walk_sigma<DT>(a, rt, pt.t, x, is_new), rcp);
                if (!is_new) term = ff{-term.hi, -term.lo};
                long long A, B;
                fix_split(term, &A, &B);
                int slot = (int)(((uint32_t)x * 2654435761u) >> (32 - H::bits));
                for (;;) {
                    const int old = atomicCAS(&hkey[slot], -1, x);
                    if (old == -1) {
                        hused[atomicAdd(&s_nu, 1)] = slot;
                        break;
                    }
                    if (old == x) break;
                    slot = (slot + 1) & (H::hash - 1);
                }
                atomicAdd(&hval[2 * slot], (unsigned long long)A);
                if (B) atomicAdd(&hval[2 * slot + 1], (unsigned long long)B);
            }
        }
        __syncthreads();
        const int nu = s_nu;
        for (int i = tid; i < nu; i += H::threads) {
            const int slot = hused[i];
            const int x = hkey[slot];
            const long long A0 = (long long)hval[2 * slot], B0 = (long long)hval[2 * slot + 1];
            hkey[slot] = -1;
            hval[2 * slot] = 0ull;
            hval[2 * slot + 1] = 0ull;
            const long long A = A0 + (B0 >> 32), B = B0 & 0xFFFFFFFFll;   // 0 <= B < 2^32
            const ff v = fix_to_ff(A, B);
            ff* p = a.Dl + rs + x;
            *p = ff_add(*p, v);
            unsigned long long* bp = reinterpret_cast<unsigned long long*>(a.bcfix + 2 * (size_t)x);
            atomicAdd(bp, (unsigned long long)A);
            if (B) atomicAdd(bp + 1, (unsigned long long)B);
        }
        __syncthreads();
    }
}

size_t walk_smem(int n) { return (size_t)kWalkWarps * (size_t)((n + 31) / 32) * sizeof(uint32_t); }
int64_t walk_warps(int nsm) { return (int64_t)nsm * kWalkCtasPerSm * kWalkWarps; }
int64_t walk_ctas(int nsm) { return (int64_t)nsm * kWalkRowCtasPerSm; }

cudaError_t walk_setup() {
    const int wmax = 2 * (int)sizeof(int32_t) * kWeightsStageMax;
    cudaError_t e0 = cudaFuncSetAttribute(k_pair_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, wmax);
    if (e0 == cudaSuccess) e0 = cudaFuncSetAttribute(kb_pair_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, wmax);
    if (e0 != cudaSuccess) return e0;
    cudaError_t e = cudaFuncSetAttribute(k_walk_units<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kWalkSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_walk_units<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kWalkSmemMax);
    return e;
}

template <typename DT>
static void launch_walks(const Dev& d, const WalkUpd& upd, int nchunks, int vn) {
    const int grid = d.nsm * kWalkCtasPerSm, rgrid = d.nsm * kWalkRowCtasPerSm;
    WalkArgs<DT> w{d.e_off, d.e_len, (const Arc<DT>*)d.e_arc, d.walk_list, d.walk_buf, d.walk_cap, d.walk_useg,
                   d.walk_acc2, d.walk_tl, d.walk_ctl, d.walk_rowE, d.stats, nchunks, upd};
    launch_k(k_walk_units<DT>, grid, kWalkThreads, walk_smem(d.n), d.st, pair_args<DT>(d), w);
    // phase 2: the heaviest rows (a few CTAs with a long tail) on the third stream beside
    // the two hash-table classes (disjoint rows, their own counters and scratch)
    const bool third = d.st3 != nullptr;
    cudaStream_t sr = d.st;
    if (third) {
        cudaEventRecord(d.ev3_fork, d.st);
        cudaStreamWaitEvent(d.st3, d.ev3_fork, 0);
        sr = d.st3;
    }
    launch_k(k_walk_rows<DT>, rgrid, kWalkThreads, (size_t)((d.n + 31) / 32) * sizeof(uint32_t), sr, pair_args<DT>(d), w);
    if (third) cudaEventRecord(d.ev3_join, d.st3);
    launch_k(k_walk_rows_hash<DT, WalkLight>, d.nsm * WalkLight::ctas, WalkLight::threads, WalkLight::smem, d.st, pair_args<DT>(d), w);
    launch_k(k_walk_rows_hash<DT, WalkMid>, d.nsm * WalkMid::ctas, WalkMid::threads, WalkMid::smem, d.st, pair_args<DT>(d), w);
    if (third) cudaStreamWaitEvent(d.st, d.ev3_join, 0);
    // the column test, which does nothing unless the walks' buffer overflowed
    PairArgs<DT> a = pair_args<DT>(d);
    a.gate = d.walk_ctl + 4;
    const int pgrid = d.nsm * kPairCtasPerSm;
    if constexpr (sizeof(DT) == 4) {
        if (vn == 8) launch_k(k_pairdep<DT, 8>, pgrid, kPairThreads, 0, d.st, a);
        else if (vn == 4) launch_k(k_pairdep<DT, 4>, pgrid, kPairThreads, 0, d.st, a);
        else launch_k(k_pairdep<DT, 1>, pgrid, kPairThreads, 0, d.st, a);
    } else {
        if (vn == 2) launch_k(k_pairdep<DT, 2>, pgrid, kPairThreads, 0, d.st, a);
        else launch_k(k_pairdep<DT, 1>, pgrid, kPairThreads, 0, d.st, a);
    }
}

void launch_pairdep(const Dev& d, const WalkUpd* upd) {
    const int pgrid = d.nsm * 8;
    if (d.dbytes == 4) launch_k(k_pair_plan<int32_t>, pgrid, kPlanThreads, 0, d.st, pair_args<int32_t>(d));
    else launch_k(k_pair_plan<int64_t>, pgrid, kPlanThreads, 0, d.st, pair_args<int64_t>(d));
    // columns per thread: 16-byte (or two 16-byte) loads where n allows them
    const int vn = pair_vn(d.dbytes, d.n);
    const int cw = kPairThreads * vn;
    const int nchunks = (d.n + cw - 1) / cw;
    const int scap = weights_stage(d.n);
    launch_k(k_pair_weights, 1, 1024, 2 * sizeof(int32_t) * (size_t)scap, d.st, d.acc_rows, d.counts + 1, d.tcnt,
             d.tcap, nchunks, d.pair_rows, d.counts + 5, d.pair_w, d.stats, d.counts + 4,
             upd ? d.walk_ctl : nullptr, upd ? d.walk_rowE : nullptr, d.err, scap);
    if (upd) {
        if (d.dbytes == 4) launch_walks<int32_t>(d, *upd, nchunks, vn);
        else launch_walks<int64_t>(d, *upd, nchunks, vn);
        return;
    }
    const int grid = d.nsm * kPairCtasPerSm;   // one resident wave; later pieces go to the first free CTA
    if (d.dbytes == 4) {
        if (vn == 8) launch_k(k_pairdep<int32_t, 8>, grid, kPairThreads, 0, d.st, pair_args<int32_t>(d));
        else if (vn == 4) launch_k(k_pairdep<int32_t, 4>, grid, kPairThreads, 0, d.st, pair_args<int32_t>(d));
        else launch_k(k_pairdep<int32_t, 1>, grid, kPairThreads, 0, d.st, pair_args<int32_t>(d));
    } else {
        if (vn == 2) launch_k(k_pairdep<int64_t, 2>, grid, kPairThreads, 0, d.st, pair_args<int64_t>(d));
        else launch_k(k_pairdep<int64_t, 1>, grid, kPairThreads, 0, d.st, pair_args<int64_t>(d));
    }
}

void launch_bc_fix(const Dev& d) {
    launch_k(k_bc_fix, (d.n + 255) / 256, 256, 0, d.st, d.n, d.bcfix, d.bc_hi, d.bc_lo, d.err);
}

}  // namespace bcg
