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
// The rank-1 passes record the changed targets t of every row s (Lemma 2 / Lemma 4:
// a lower distance, or new tied paths).  A row with at most kPairCap of them is
// corrected by this sum; the old terms read the rows as they were before the update,
// which k_snapshot saves before the first write to each row, and the new terms read
// the state after both phases.  In G_D of an undirected graph d(x,t) = d(t,x) and
// sigma_xt = sigma_tx before and after the update, so the column t of the formula is
// row t, read contiguously.  Rows with more targets, and row v (rewritten whole by the
// OUT phase, its targets unrecorded), are re-accumulated by Algorithm 1 instead.
#include "bc_device.cuh"
#include "ff.cuh"

namespace bcg {

constexpr int kSnapThreads = 256;
constexpr int kPairThreads = 256;

// Save rows[0..count) (and row extra_row when the OUT phase changes it) before their
// first write in this update.  A saved row of v is also sent to the full path by a
// target count above the cap.  The rows of one launch are distinct.
template <typename DT>
__global__ void __launch_bounds__(kSnapThreads)
k_snapshot(int n, const DT* __restrict__ D, const uint64_t* __restrict__ S, DT* sD, uint64_t* sS,
           uint8_t* snapped, const int32_t* rows, const int32_t* count, int extra_row,
           const uint8_t* changed, int32_t* tcnt, int tcap, const int32_t* err) {
    __shared__ int s_do;
    if (*err) return;
    const int cnt = *count;
    const int items = cnt + (extra_row >= 0 ? 1 : 0);
    for (int i = blockIdx.x; i < items; i += gridDim.x) {
        const int s = i < cnt ? rows[i] : extra_row;
        if (threadIdx.x == 0) {
            int go = snapped[s] == 0;
            if (i >= cnt) {
                go = go && changed[s] != 0;
                if (changed[s]) tcnt[s] = tcap + 1;
            }
            if (go) snapped[s] = 1;
            s_do = go;
        }
        __syncthreads();
        const bool go = s_do != 0;
        __syncthreads();
        if (!go) continue;
        const size_t off = (size_t)s * n;
        if ((n & 3) == 0 && sizeof(DT) == 4) {
            const int4* a = reinterpret_cast<const int4*>(D + off);
            int4* b = reinterpret_cast<int4*>(sD + off);
            for (int j = threadIdx.x; j < n / 4; j += blockDim.x) b[j] = __ldcs(a + j);
        } else {
            for (int j = threadIdx.x; j < n; j += blockDim.x) sD[off + j] = D[off + j];
        }
        if ((n & 1) == 0) {
            const ulonglong2* a = reinterpret_cast<const ulonglong2*>(S + off);
            ulonglong2* b = reinterpret_cast<ulonglong2*>(sS + off);
            for (int j = threadIdx.x; j < n / 2; j += blockDim.x) b[j] = __ldcs(a + j);
        } else {
            for (int j = threadIdx.x; j < n; j += blockDim.x) sS[off + j] = S[off + j];
        }
    }
}

// mark[s] = row s changed and has more recorded targets than the cap (or is row v).
__global__ void k_full_flags(int n, const uint8_t* changed, const int32_t* tcnt, int tcap, uint8_t* mark) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) mark[s] = (changed[s] != 0 && tcnt[s] > tcap) ? 1 : 0;
}

// Per-update flags of the rows listed in rows[0..count) back to zero; the rows sent to
// the full path are added to stats[7].
__global__ void k_pair_clear(const int32_t* rows, const int32_t* count, int32_t* tcnt, uint8_t* snapped,
                             const int32_t* full_count, int64_t* stats) {
    const int cnt = *count;
    if (blockIdx.x == 0 && threadIdx.x == 0) stats[7] += *full_count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int s = rows[i];
        tcnt[s] = 0;
        snapped[s] = 0;
    }
}

template <typename DT>
struct PairArgs {
    int n;
    const DT* D;            // state after the update
    const uint64_t* S;
    const DT* sD;           // rows saved before the update (where snapped)
    const uint64_t* sS;
    const uint8_t* snapped;
    const int32_t* tcnt;
    const int32_t* tlist;
    int tcap;
    const int32_t* rows;
    const int32_t* count;
    ff* Dl;
    int32_t* err;
};

// sigma_sx * sigma_xt / sigma_st in float-float (the quotient as a product with the
// reciprocal of sigma_st).
__device__ __forceinline__ ff pair_term(uint64_t a, uint64_t b, const ff& rcp) {
    return ff_mul(ff_mul(ff_from_u64(a), ff_from_u64(b)), rcp);
}

// Distances of VN consecutive columns (one 16-byte load when VN > 1).
template <typename DT, int VN>
__device__ __forceinline__ void load_d(const DT* p, int64_t* o) {
    if constexpr (VN == 1) {
        o[0] = p[0];
    } else {
        Vec<DT>::unpack(*reinterpret_cast<const typename Vec<DT>::T*>(p), o);
    }
}

// Adds sign * sigma_sx sigma_xt / sigma_st to acc[q] for the columns x = x0 + q on a
// shortest s-t path (d(s,x) + d(x,t) = d(s,t), x not in {s, t}) of one state (old or
// new).  Row t is read only when some column can be on such a path (d(s,x) < d(s,t)).
template <typename DT, int VN>
__device__ __forceinline__ void pair_terms(int x0, int s, int t, int64_t dst, const ff& rcp, float sign,
                                           const int64_t* ds, const DT* Dt, const uint64_t* St,
                                           const uint64_t* Ss, uint64_t* ss, unsigned& have, ff* acc,
                                           unsigned& any) {
    bool cand = false;
#pragma unroll
    for (int q = 0; q < VN; ++q) cand |= ds[q] < dst;
    if (!cand) return;
    int64_t dt[VN];
    load_d<DT, VN>(Dt + x0, dt);
#pragma unroll
    for (int q = 0; q < VN; ++q) {
        const int x = x0 + q;
        if (ds[q] >= dst || x == s || x == t || dt[q] == Inf<DT>::v) continue;
        // both terms are below 2^63: their unsigned sum is exact
        if ((uint64_t)ds[q] + (uint64_t)dt[q] != (uint64_t)dst) continue;
        if (!((have >> q) & 1u)) {
            ss[q] = Ss[x];
            have |= 1u << q;
        }
        const ff c = pair_term(ss[q], St[x], rcp);
        acc[q] = ff_add(acc[q], ff{sign * c.hi, sign * c.lo});
        any |= 1u << q;
    }
}

// One CTA per listed row s with 1..tcap recorded targets.  The targets are sorted and
// made unique by warp 0 (so the sum runs in a fixed order), then every thread takes VN
// consecutive columns x at a time and adds sum_t [delta'_st(x) - delta_st(x)] to
// delta_s(x).
template <typename DT, int VN>
__global__ void __launch_bounds__(kPairThreads) k_pairdep(PairArgs<DT> a) {
    __shared__ int32_t s_t[32];
    __shared__ int64_t s_dold[32], s_dnew[32];
    __shared__ ff s_rold[32], s_rnew[32];
    __shared__ const DT* s_pDo[32];
    __shared__ const uint64_t* s_pSo[32];
    __shared__ int s_u;
    if (*a.err) return;
    const int n = a.n;
    const int64_t INF = Inf<DT>::v;
    const int cnt = *a.count;
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
        const int s = a.rows[i];
        const int T = a.tcnt[s];
        if (T == 0 || T > a.tcap) continue;   // block-uniform
        const size_t rs = (size_t)s * n;
        const bool snap_s = a.snapped[s] != 0;
        const DT* Do_s = (snap_s ? a.sD : a.D) + rs;
        const uint64_t* So_s = (snap_s ? a.sS : a.S) + rs;
        const DT* Dn_s = a.D + rs;
        const uint64_t* Sn_s = a.S + rs;
        if (threadIdx.x < 32) {
            const int val = lane < T ? a.tlist[(size_t)s * a.tcap + lane] : INT32_MAX;
            bool dup = false;
            for (int j = 0; j < 32; ++j) {
                const int vj = __shfl_sync(0xffffffffu, val, j);
                dup |= (vj == val) && (j < lane);
            }
            const bool keep = !dup && val != INT32_MAX;
            const unsigned km = __ballot_sync(0xffffffffu, keep);
            int pos = 0;
            for (int j = 0; j < 32; ++j) {
                const int vj = __shfl_sync(0xffffffffu, val, j);
                pos += ((km >> j) & 1u) && vj < val;
            }
            if (keep) {
                const int t = val;
                const size_t rt = (size_t)t * n;
                const bool snap_t = a.snapped[t] != 0;
                s_t[pos] = t;
                s_pDo[pos] = (snap_t ? a.sD : a.D) + rt;
                s_pSo[pos] = (snap_t ? a.sS : a.S) + rt;
                const int64_t dol = Do_s[t], dnw = Dn_s[t];
                const uint64_t sol = So_s[t], snw = Sn_s[t];
                // -1: no shortest path (no column passes d(s,x) < -1)
                s_dold[pos] = (dol == INF || sol == 0) ? -1 : dol;
                s_dnew[pos] = (dnw == INF || snw == 0) ? -1 : dnw;
                s_rold[pos] = sol ? ff_rcp(ff_from_u64(sol)) : ff{0.f, 0.f};
                s_rnew[pos] = snw ? ff_rcp(ff_from_u64(snw)) : ff{0.f, 0.f};
            }
            if (lane == 0) s_u = __popc(km);
        }
        __syncthreads();
        const int U = s_u;
        for (int x0 = threadIdx.x * VN; x0 < n; x0 += blockDim.x * VN) {
            int64_t dso[VN], dsn[VN];
            load_d<DT, VN>(Do_s + x0, dso);
            load_d<DT, VN>(Dn_s + x0, dsn);
            ff acc[VN];
            uint64_t sso[VN], ssn[VN];
#pragma unroll
            for (int q = 0; q < VN; ++q) acc[q] = ff{0.f, 0.f};
            unsigned have_o = 0, have_n = 0, any = 0;
            for (int u = 0; u < U; ++u) {
                const int t = s_t[u];
                const size_t rt = (size_t)t * n;
                pair_terms<DT, VN>(x0, s, t, s_dold[u], s_rold[u], -1.f, dso, s_pDo[u], s_pSo[u], So_s, sso,
                                   have_o, acc, any);
                pair_terms<DT, VN>(x0, s, t, s_dnew[u], s_rnew[u], 1.f, dsn, a.D + rt, a.S + rt, Sn_s, ssn,
                                   have_n, acc, any);
            }
#pragma unroll
            for (int q = 0; q < VN; ++q)
                if ((any >> q) & 1u) a.Dl[rs + x0 + q] = ff_add(a.Dl[rs + x0 + q], acc[q]);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ launches

void launch_snapshot(const Dev& d, const int32_t* rows, const int32_t* count, int32_t extra_row) {
    const int grid = d.nsm * 4;
    if (d.dbytes == 4)
        k_snapshot<int32_t><<<grid, kSnapThreads, 0, d.st>>>(
            d.n, (const int32_t*)d.D, d.S, (int32_t*)d.snapD, d.snapS, d.snapped, rows, count, extra_row,
            d.changed, d.tcnt, d.tcap, d.err);
    else
        k_snapshot<int64_t><<<grid, kSnapThreads, 0, d.st>>>(
            d.n, (const int64_t*)d.D, d.S, (int64_t*)d.snapD, d.snapS, d.snapped, rows, count, extra_row,
            d.changed, d.tcnt, d.tcap, d.err);
}

void launch_full_flags(const Dev& d) {
    k_full_flags<<<(d.n + 255) / 256, 256, 0, d.st>>>(d.n, d.changed, d.tcnt, d.tcap, d.mark);
}

void launch_pair_clear(const Dev& d) {
    k_pair_clear<<<std::max(1, std::min(d.nsm, (d.n + 255) / 256)), 256, 0, d.st>>>(
        d.acc_rows, d.counts + 1, d.tcnt, d.snapped, d.counts + 3, d.stats);
}

template <typename DT>
static PairArgs<DT> pair_args(const Dev& d) {
    PairArgs<DT> a;
    a.n = d.n;
    a.D = (const DT*)d.D;
    a.S = d.S;
    a.sD = (const DT*)d.snapD;
    a.sS = d.snapS;
    a.snapped = d.snapped;
    a.tcnt = d.tcnt;
    a.tlist = d.tlist;
    a.tcap = d.tcap;
    a.rows = d.acc_rows;
    a.count = d.counts + 1;
    a.Dl = d.Dl;
    a.err = d.err;
    return a;
}

void launch_pairdep(const Dev& d) {
    const int grid = d.nsm * 8;
    if (d.dbytes == 4) {
        if (d.n % 4 == 0) k_pairdep<int32_t, 4><<<grid, kPairThreads, 0, d.st>>>(pair_args<int32_t>(d));
        else k_pairdep<int32_t, 1><<<grid, kPairThreads, 0, d.st>>>(pair_args<int32_t>(d));
    } else {
        if (d.n % 2 == 0) k_pairdep<int64_t, 2><<<grid, kPairThreads, 0, d.st>>>(pair_args<int64_t>(d));
        else k_pairdep<int64_t, 1><<<grid, kPairThreads, 0, d.st>>>(pair_args<int64_t>(d));
    }
}

}  // namespace bcg
