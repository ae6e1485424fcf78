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
//     with rho(b) = (1 + delta(b)) / sigma_sb kept per vertex.  Each vertex is summed by
//     a group of kGroup lanes (segments of at most kSmallDeg slots) or by a warp (longer
//     segments), each lane over a fixed stride of slots and a fixed butterfly across
//     the lanes, so the result does not depend on scheduling.
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
#include "bc_internal.cuh"

namespace bcg {

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
    const int32_t* e_big;
    int e_nbig;
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

// Slot of the r-th (0-based) set bit of m within [beg, end); the bit exists.
__device__ __forceinline__ int select_bit(const uint32_t* m, int beg, int end, int r) {
    const int w1 = (end - 1) >> 5;
    int w = beg >> 5;
    uint32_t b = m[w] & (0xffffffffu << (beg & 31));
    for (;;) {
        if (w == w1) b &= 0xffffffffu >> (31 - ((end - 1) & 31));
        const int c = __popc(b);
        if (r < c) break;
        r -= c;
        b = m[++w];
    }
    for (; r > 0; --r) b &= b - 1u;
    return (w << 5) + __ffs(b) - 1;
}

// Exclusive block-wide prefix sum of v (all threads call it); *total gets the sum.
// s_ws needs kAccThreads / 32 + 1 ints and must not be reused before a barrier.
__device__ __forceinline__ int block_excl_scan(int v, int* s_ws, int* total) {
    constexpr int NW = kAccThreads / 32;
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

// Last index i in [0, kAccThreads) with off[i] <= j (off non-decreasing, off[0] = 0).
__device__ __forceinline__ int owner_of(const int* off, int j) {
    int lo = 0, hi = kAccThreads;
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
struct LevelSmem {
    int off[kAccThreads];
    int beg[kAccThreads];
    int end[kAccThreads];
    uint64_t sx[kAccThreads];
    ff buf[kAccThreads];
    int ws[kAccThreads / 32 + 1];
};

template <typename DT, bool STATIC, typename DA>
__device__ __forceinline__ void accumulate_source(const AccArgs<DT>& a, const DA dist, int s, uint64_t* Ss,
                                                  ff* out, uint32_t* cnt, uint16_t* order, uint32_t* mask,
                                                  uint16_t* big, LevelSmem& ls, ff* rho, int32_t* lvl,
                                                  int* s_tail, int* s_nbig) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int T = kAccThreads, NW = kAccThreads / 32, U = 4;
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
        for (int qb = lo; qb < hi; qb += T) {
            const int q = qb + tid;
            int x = 0, beg = 0, end = 0, k = 0;
            if (q < hi) {
                x = order[q];
                beg = a.e_off[x];
                end = beg + a.e_len[x];
                k = count_bits(mask, beg, end);
            }
            if (big_push(k > kBigDag, x, big, s_nbig)) k = 0;
            int total;
            const int off = block_excl_scan(k, ls.ws, &total);
            ls.off[tid] = off;
            ls.beg[tid] = beg;
            ls.end[tid] = end;
            if (STATIC) ls.sx[tid] = k ? Ss[x] : 0ull;
            __syncthreads();
            for (int jb = 0; jb < total; jb += T) {
                const int j = jb + tid;
                bool ready = false;
                int b = 0;
                if (j < total) {
                    const int o = owner_of(ls.off, j);
                    const int e = select_bit(mask, ls.beg[o], ls.end[o], j - ls.off[o]);
                    b = (int)a.e_arc[e].dst;
                    push_sigma<DT, STATIC>(Ss, b, STATIC ? ls.sx[o] : 0ull, a.err);
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
        for (int qb = lo; qb < hi; qb += T) {
            const int q = qb + tid;
            int x = 0, beg = 0, end = 0, k = 0;
            if (q < hi) {
                x = order[q];
                beg = a.e_off[x];
                end = beg + a.e_len[x];
                k = count_bits(mask, beg, end);
            }
            const bool is_big = big_push(k > kBigDag, x, big, s_nbig);
            if (is_big) k = 0;
            const bool mine = q < hi && !is_big;
            const uint64_t sig = mine ? Ss[x] : 1ull;
            int total;
            const int off = block_excl_scan(k, ls.ws, &total);
            ls.off[tid] = off;
            ls.beg[tid] = beg;
            ls.end[tid] = end;
            __syncthreads();
            ff acc{0.0f, 0.0f};
            for (int jb = 0; jb < total; jb += T) {
                const int j = jb + tid;
                if (j < total) {
                    const int o = owner_of(ls.off, j);
                    const int e = select_bit(mask, ls.beg[o], ls.end[o], j - ls.off[o]);
                    ls.buf[tid] = rho[a.e_arc[e].dst];
                }
                __syncthreads();
                const int p0 = max(off, jb), p1 = min(off + k, jb + T);
                for (int p = p0; p < p1; ++p) acc = ff_add(acc, ls.buf[p - jb]);
                __syncthreads();
            }
            if (mine) finish_vertex(x, acc, sig, out, rho);
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

// One CTA per source at a time.  Shared memory: [d16 | order] (the distance row is dead
// once the slot mask is built, so the level order reuses it) | cnt (n/2 words) |
// big list | slot mask (here when it fits, else in the work space); the per-round
// scratch of the level passes is static shared memory.
template <typename DT, bool STATIC>
__global__ void __launch_bounds__(kAccThreads) k_accum_smem(AccArgs<DT> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LevelSmem ls;
    const int n = a.n;
    const int np = (n + 31) & ~31;
    uint16_t* d16 = reinterpret_cast<uint16_t*>(smem);
    uint16_t* order = d16;
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + 2 * (size_t)np);
    uint16_t* big = reinterpret_cast<uint16_t*>(smem + 4 * (size_t)np);
    int32_t* wsb = a.ws + (size_t)blockIdx.x * a.ws_stride;
    ff* rho = reinterpret_cast<ff*>(wsb);
    int32_t* lvl = wsb + 2 * (size_t)n;
    uint32_t* mask = a.mask_in_smem ? reinterpret_cast<uint32_t*>(smem + 4 * (size_t)np + 2 * kBigCap)
                                    : reinterpret_cast<uint32_t*>(wsb + ((3 * (int64_t)n + 2 + 3) & ~(int64_t)3));
    __shared__ int s_tail, s_nbig;
    const int tid = threadIdx.x;
    const int64_t INF = Inf<DT>::v;
    const int total = STATIC ? n : *a.count;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        if (block_err(a.err)) return;
        const int s = STATIC ? i : a.rows[i];
        const DT* Ds = a.D + (size_t)s * n;
        uint64_t* Ss = a.S + (size_t)s * n;
        ff* out = a.Dl + (size_t)s * n;
        int wide = 0;
        for (int t = tid; t < n; t += kAccThreads) {
            const int64_t v = Ds[t];
            uint16_t c;
            if (v == INF) c = 0xFFFF;
            else if (v < 0xFFFF) c = (uint16_t)v;
            else { c = 0xFFFE; wide = 1; }
            d16[t] = c;
            out[t] = ff{0.0f, 0.0f};
            if (STATIC) Ss[t] = (t == s) ? 1ull : 0ull;
        }
        for (int t = tid; t < np / 2; t += kAccThreads) cnt[t] = 0u;
        wide = __syncthreads_or(wide);
        if (!wide)
            accumulate_source<DT, STATIC>(a, Dist16{d16}, s, Ss, out, cnt, order, mask, big, ls, rho, lvl, &s_tail,
                                          &s_nbig);
        else
            accumulate_source<DT, STATIC>(a, DistG<DT>{Ds}, s, Ss, out, cnt, order, mask, big, ls, rho, lvl,
                                          &s_tail, &s_nbig);
        __syncthreads();
    }
}

// partial[rb][t] = sum over rows r of row block rb of Dl[s_r][t] (t != s_r), rows in
// increasing order, in float-float (all terms are non-negative); rows = nullptr means
// all n rows.
__global__ void k_bc_partial(int n, const int32_t* rows, const int32_t* count, const ff* Dl,
                             ff* partial, const int32_t* err) {
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rb = blockIdx.y;
    const int total = rows ? *count : n;
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
__global__ void k_bc_finish(int n, const int32_t* rows, const int32_t* count, const ff* partial,
                            double sign, int overwrite, double* hi, double* lo, const int32_t* err) {
    if (*err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int total = rows ? *count : n;
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
    a.e_arc = (const Arc<DT>*)d.e_arc;
    a.e_cap = d.e_cap;
    a.e_big = d.e_big;
    a.e_nbig = d.e_nbig;
    a.rows = d.acc_rows;
    a.count = d.counts + 1;
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

constexpr size_t kSmemLimit = 200 * 1024;

void accum_config(Dev& d) {
    const size_t base = smem_base(d.n);
    const size_t mb = mask_bytes(d.e_cap);
    const bool in_smem = base + mb <= kSmemLimit;
    const size_t smem = in_smem ? base + mb : base;
    int per_sm = 1;
    const int maxs = (int)kSmemLimit;
    if (d.dbytes == 4) {
        cudaFuncSetAttribute(k_accum_smem<int32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
        cudaFuncSetAttribute(k_accum_smem<int32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_accum_smem<int32_t, false>, kAccThreads, smem);
    } else {
        cudaFuncSetAttribute(k_accum_smem<int64_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
        cudaFuncSetAttribute(k_accum_smem<int64_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_accum_smem<int64_t, false>, kAccThreads, smem);
    }
    if (per_sm < 1) per_sm = 1;
    d.acc_smem = (int32_t)smem;
    d.acc_mask_smem = in_smem ? 1 : 0;
    d.acc_grid = std::min(d.nsm * per_sm, std::max(d.n, 1));
    // per CTA: rho (n float-float pairs) | level bounds (n + 2 ints) | slot mask if not in smem
    const int64_t head = ((3 * (int64_t)d.n + 2) + 3) & ~(int64_t)3;
    d.ws_stride = head + (in_smem ? 0 : (((int64_t)mb / 4 + 3) & ~(int64_t)3));
}

void launch_accum(const Dev& d, int is_static) {
    const int grid = d.acc_grid;
    const size_t smem = (size_t)d.acc_smem;
    if (d.dbytes == 4) {
        if (is_static) k_accum_smem<int32_t, true><<<grid, kAccThreads, smem, d.st>>>(acc_args<int32_t>(d));
        else k_accum_smem<int32_t, false><<<grid, kAccThreads, smem, d.st>>>(acc_args<int32_t>(d));
    } else {
        if (is_static) k_accum_smem<int64_t, true><<<grid, kAccThreads, smem, d.st>>>(acc_args<int64_t>(d));
        else k_accum_smem<int64_t, false><<<grid, kAccThreads, smem, d.st>>>(acc_args<int64_t>(d));
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
