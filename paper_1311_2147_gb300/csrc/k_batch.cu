// k_batch.cu -- many graphs, one launch per phase.
//
// A batch applies, to each of G graphs, its own list of updates; round r applies the
// r-th update of every graph that has one.  Within a round the phases of an update
// (k_update.cu: Algorithm 4 and the rank-1 pass of Lemma 2 / 4, both directions;
// k_accum.cu: DAG rebuild, Kahn levels, Eq. 4, BC update) run phase by phase over all
// graphs at once: each phase is one persistent kernel whose work is the concatenation
// of every graph's work for that phase, so a 64-vertex graph and a 2048-vertex graph
// share the GPU instead of each getting its own launches.  A task index is mapped to
// its graph by binary search over per-graph prefix offsets; offsets of work that is
// known only on the device (rows that changed) are computed by a one-CTA plan kernel
// just before the phase.  Every per-element, per-item and per-source body is the same
// device function the single-graph kernels call (bc_device.cuh), so a graph's result
// in a batch is bit-identical to its result alone.  The whole multi-round sequence is
// captured once into a CUDA graph and replayed with one graph launch per batch.
#include "bc_batch.cuh"
#include "bc_device.cuh"

namespace bcg {

// ---------------------------------------------------------------- E* writes

__global__ void kb_estar(BatchArgs b, int r) {
    const int64_t o0 = b.eop_off[r], o1 = b.eop_off[r + 1];
    for (int64_t j = o0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < o1;
         j += (int64_t)gridDim.x * blockDim.x) {
        const BatchEOp op = b.eops[j];
        const Dev& d = b.devs[op.g];
        if (op.op.slot >= 0) {
            d.e_src[op.op.slot] = op.op.a;
            if (d.dbytes == 4)
                static_cast<Arc<int32_t>*>(d.e_arc)[op.op.slot] = Arc<int32_t>{op.op.b, (int32_t)op.op.w};
            else
                static_cast<Arc<int64_t>*>(d.e_arc)[op.op.slot] = Arc<int64_t>{(int64_t)op.op.b, op.op.w};
        }
        atomicMax(d.e_len + op.op.a, op.op.len_a);
    }
}

// ---------------------------------------------------------------- per-vertex passes

// kind 0: Algorithm 4 forward (IN edges, per source); 1: OUT row test (per source);
// 2: Algorithm 4 on the reverse graph (per target); 3: write row v.
template <typename DT>
__global__ void kb_vertex_pass(BatchArgs b, int r, int kind) {
    const int G = b.G;
    const int64_t* off = b.voff + ((int64_t)r * 4 + kind) * (G + 1);
    const int64_t total = off[G];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int g = graph_of(off, G, j);
        const int x = (int)(j - off[g]);
        const Dev& d = b.devs[g];
        if (*d.err) continue;
        const BatchUpd u = b.upd[(int64_t)r * G + g];
        const VEdge* e = b.entries + u.first;
        const DT* D = (const DT*)d.D;
        switch (kind) {
            case 0:
                dev_alg4_in<DT>(x, d.n, D, d.S, u.v, e, u.k, d.directed, (DT*)d.fD, d.fS, d.fM, d.mark, d.changed,
                                d.err);
                break;
            case 1:
                dev_rows_out<DT>(x, d.n, D, d.S, u.v, e, u.k, d.directed, (DT*)d.fD, d.fS, d.fM, d.mark, d.changed,
                                 d.err);
                break;
            case 2:
                dev_alg4_out<DT>(x, d.n, D, d.S, u.v, e, u.k, d.directed, (DT*)d.cD, d.cS, d.cM, d.changed, d.err);
                break;
            default:
                if (d.pair_on) {
                    // row v is never written before this in an update: its changes are first changes
                    PairRec rec = make_pair_rec(d);
                    rec.first = 1;
                    const size_t i = (size_t)u.v * d.n + x;
                    if (D[i] != ((const DT*)d.cD)[x] || d.S[i] != d.cS[x])
                        record_change<DT>(rec, d.n, u.v, x, D[i], d.S[i]);
                }
                dev_write_row<DT>(x, d.n, (DT*)d.D, d.S, u.v, (const DT*)d.cD, d.cS, d.err);
        }
    }
}

// ---------------------------------------------------------------- compaction

// which 0: IN-phase rows, 1: OUT-phase rows, 2: rows to re-accumulate (clears changed;
// graphs with pair corrections list theirs in kb_pair_lists).
__global__ void __launch_bounds__(kCompactThreads) kb_compact(BatchArgs b, int r, int which) {
    for (int g = blockIdx.x; g < b.G; g += gridDim.x) {
        const BatchUpd u = b.upd[(int64_t)r * b.G + g];
        const Dev& d = b.devs[g];
        if (which == 0 && u.kin == 0) continue;
        if (which == 1 && u.kout == 0) continue;
        if (which == 2 && (u.present == 0 || d.pair_on)) continue;
        if (which < 2) dev_compact(d.n, d.mark, 0, d.rows, d.counts, 0, nullptr, d.err);
        else dev_compact(d.n, d.changed, 1, d.acc_rows, d.counts + 1, 0, d.stats, d.err);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- plans

// Per-graph work known only on the device, as exclusive prefix offsets over graphs:
// kind 0: scan items of the phase rows (rows x column chunks); 1: BC partial tasks
// (column blocks x row blocks of the rows to re-accumulate); 2: sources to
// re-accumulate; 3: rows listed for pair corrections; 4 + c: column-test weight of the
// graphs whose columns per thread are of class c (and its piece counter back to zero).
// One CTA.
__global__ void __launch_bounds__(1024) kb_plan(BatchArgs b, int r, int kind, int phase_active, int64_t* out,
                                                int scan_unroll) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t s_total, s_base;
    const int G = b.G, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int g0 = 0; g0 < G; g0 += 1024) {
        const int g = g0 + threadIdx.x;
        int64_t v = 0;
        if (g < G) {
            const Dev& d = b.devs[g];
            const BatchUpd u = b.upd[(int64_t)r * G + g];
            const bool on = (phase_active == 0) ? (u.kin != 0) : (phase_active == 1) ? (u.kout != 0) : (u.present != 0);
            if (on && *d.err == 0) {
                if (kind == 0) {
                    const int cw = kScanThreads * (d.dbytes == 4 ? 4 : 2) * scan_unroll;
                    v = (int64_t)d.counts[0] * ((d.n + cw - 1) / cw);
                    atomicAdd(reinterpret_cast<unsigned long long*>(d.stats + 6), (unsigned long long)d.counts[0]);
                } else if (kind == 1) {
                    v = (int64_t)((d.n + 255) / 256) * ((acc_list_count(d) + kRowsPerBlock - 1) / kRowsPerBlock);
                } else if (kind == 2) {
                    v = acc_list_count(d);
                } else if (kind == 3) {
                    v = d.pair_on ? d.counts[1] : 0;
                } else if (d.pair_on && pair_class(d.dbytes, pair_vn(d.dbytes, d.n)) == kind - 4) {
                    v = d.pair_w[d.counts[5]];
                }
            }
        }
        int64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int64_t x = wsum[lane];
            int64_t ix = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, ix, o);
                if (lane >= o) ix += y;
            }
            wsum[lane] = ix - x;
            if (lane == 31) s_total = ix;
        }
        __syncthreads();
        if (g < G) out[g] = s_base + wsum[wid] + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) s_base += s_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[G] = s_base;
        if (kind >= 4) b.pctr[kind - 4] = 0;
    }
}

// ---------------------------------------------------------------- rank-1 pass

template <typename DT>
__device__ __forceinline__ ScanArgs<DT> batch_scan_args(const Dev& d, const BatchUpd& u, int phase) {
    ScanArgs<DT> a;
    a.n = d.n;
    a.D = (DT*)d.D;
    a.S = d.S;
    a.rows = d.rows;
    a.count = d.counts;
    a.fD = (const DT*)d.fD;
    a.fS = d.fS;
    a.fM = d.fM;
    a.err = d.err;
    a.stats = d.stats;
    a.tie_rows = 0;
    a.tie_cols = 0;
    a.rec = d.pair_on ? make_pair_rec(d) : PairRec{};
    a.rows2 = nullptr;
    a.count2 = nullptr;
    a.cD2 = nullptr;
    a.cS2 = a.cM2 = nullptr;
    if (phase == 0) {
        a.cD = (const DT*)d.D + (size_t)u.v * d.n;
        a.cS = d.S + (size_t)u.v * d.n;
        a.cM = a.cS;
        a.skip_row = -1;
        a.rec.first = 1;   // the IN phase is the first pass of an update that writes pairs
    } else {
        a.cD = (const DT*)d.cD;
        a.cS = d.cS;
        a.cM = d.cM;
        a.skip_row = u.v;
    }
    return a;
}

// U: vectors per thread per item (the item's chunk width); sched 0: a contiguous block of
// items per CTA, 1: items dealt out in turn.
template <typename DT, int U>
__global__ void __launch_bounds__(kScanThreads, 4) kb_scan(BatchArgs b, int r, int phase, const int64_t* off,
                                                           int sched) {
    const int G = b.G;
    const int64_t total = off[G];
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t it0 = sched ? (int64_t)blockIdx.x : (int64_t)blockIdx.x * per;
    const int64_t it1 = sched ? total : min(total, it0 + per);
    const int64_t step = sched ? (int64_t)gridDim.x : 1;
    constexpr int VN = Vec<DT>::N;
    constexpr int CW = kScanThreads * VN * U;
    int cg = -1, cur = -1, s = -1, nchunks = 1;
    int64_t rd = Inf<DT>::v;
    uint64_t rs = 0, rm = 0;
    int n_changed = 0, n_ties = 0;
    ScanArgs<DT> a{};
    for (int64_t j = it0; j < it1; j += step) {
        int g = cg;
        if (g < 0 || j >= off[g + 1] || j < off[g]) {
            // flush the counters of the previous graph before moving on
            if (cg >= 0) {
                scan_stats(a.stats, n_changed, n_ties);
                n_changed = n_ties = 0;
            }
            g = graph_of(off, G, j);
            cg = g;
            cur = -1;
            const Dev& d = b.devs[g];
            a = batch_scan_args<DT>(d, b.upd[(int64_t)r * G + g], phase);
            nchunks = (d.n + CW - 1) / CW;
        }
        const int64_t item = j - off[g];
        const int i = (int)(item / nchunks);
        const int c = (int)(item - (int64_t)i * nchunks);
        if (i != cur) {
            cur = i;
            s = a.rows[i];
            rd = (s == a.skip_row) ? Inf<DT>::v : (int64_t)a.fD[s];
            rs = a.fS[s];
            rm = a.fM[s];
        }
        if (rd == Inf<DT>::v) continue;
        if (a.n % VN == 0) dev_scan_item<DT, true, U>(a, s, rd, rs, rm, c, n_changed, n_ties);
        else dev_scan_item<DT, false, U>(a, s, rd, rs, rm, c, n_changed, n_ties);
    }
    if (cg >= 0) scan_stats(a.stats, n_changed, n_ties);
    else scan_stats(b.devs[0].stats, 0, 0);
}

// ---------------------------------------------------------------- BC row sums

__global__ void kb_bc_partial(BatchArgs b, int r, const int64_t* off) {
    const int G = b.G;
    const int64_t total = off[G];
    for (int64_t j = blockIdx.x; j < total; j += gridDim.x) {
        const int g = graph_of(off, G, j);
        const Dev& d = b.devs[g];
        if (*d.err) continue;
        const int64_t task = j - off[g];
        const int tb = (d.n + 255) / 256;
        const int rb = (int)(task / tb);
        const int t = (int)(task - (int64_t)rb * tb) * 256 + threadIdx.x;
        dev_bc_partial(t, rb, d.n, acc_list(d), acc_list_count(d), d.Dl, d.partial);
    }
}

__global__ void kb_bc_finish(BatchArgs b, int r, double sign) {
    const int G = b.G;
    const int64_t* off = b.coff;
    const int64_t total = off[G];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int g = graph_of(off, G, j);
        const Dev& d = b.devs[g];
        if (*d.err || b.upd[(int64_t)r * G + g].present == 0) continue;
        const int t = (int)(j - off[g]);
        dev_bc_finish(t, d.n, acc_list_count(d), d.partial, sign, 0, d.bc_hi, d.bc_lo);
    }
}

// ---------------------------------------------------------------- accumulation

// One source per CTA of T threads (128, 256 or 512: a tile the autotuner picks), held to
// 64 registers so that 1024 threads share an SM.
template <typename DT, int T>
__global__ void __launch_bounds__(T, 1024 / T) kb_accum(BatchArgs b, int r, const int64_t* off) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LevelSmem<T> ls;
    __shared__ int s_tail, s_nbig;
    const int G = b.G;
    const int64_t total = off[G];
    int32_t* wsb = b.ws + (size_t)blockIdx.x * b.ws_stride;
    for (int64_t j = blockIdx.x; j < total; j += gridDim.x) {
        const int g = graph_of(off, G, j);
        const Dev& d = b.devs[g];
        if (block_err(d.err)) continue;
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
        a.rows = acc_list(d);
        a.count = d.pair_on ? d.counts + 3 : d.counts + 1;
        a.ws = b.ws;
        a.ws_stride = b.ws_stride;
        a.err = d.err;
        a.mask_in_smem = b.mask_in_smem;
        const AccSmem m = acc_smem(a, smem, wsb);
        dev_accum_source<DT, false, T>(a, a.rows[j - off[g]], m, ls, &s_tail, &s_nbig);
    }
}

// ---------------------------------------------------------------- launches

static inline int nb(int64_t x, int t) { return (int)std::max<int64_t>(1, (x + t - 1) / t); }

template <typename DT>
static void batch_scan(const BatchArgs& b, const BatchLaunch& L, int r, int phase, cudaStream_t st) {
    const int grid = L.nsm * L.scan_ctas;
    switch (L.scan_unroll) {
        case 1: kb_scan<DT, 1><<<grid, kScanThreads, 0, st>>>(b, r, phase, b.plan_scan, L.scan_sched); break;
        case 2: kb_scan<DT, 2><<<grid, kScanThreads, 0, st>>>(b, r, phase, b.plan_scan, L.scan_sched); break;
        case 8: kb_scan<DT, 8><<<grid, kScanThreads, 0, st>>>(b, r, phase, b.plan_scan, L.scan_sched); break;
        default: kb_scan<DT, 4><<<grid, kScanThreads, 0, st>>>(b, r, phase, b.plan_scan, L.scan_sched); break;
    }
}

template <typename DT>
static void round_launches(const BatchArgs& b, const BatchLaunch& L, int r, cudaStream_t st) {
    const int nsm = L.nsm;
    kb_estar<<<nb(L.max_eops, 256), 256, 0, st>>>(b, r);
    // IN phase
    kb_vertex_pass<DT><<<nsm * L.vpass_ctas, 256, 0, st>>>(b, r, 0);
    kb_compact<<<std::min(b.G, nsm * 2), kCompactThreads, 0, st>>>(b, r, 0);
    kb_plan<<<1, 1024, 0, st>>>(b, r, 0, 0, b.plan_scan, L.scan_unroll);
    batch_scan<DT>(b, L, r, 0, st);
    // OUT phase (graphs without out-edges in this round have no work)
    kb_vertex_pass<DT><<<nsm * L.vpass_ctas, 256, 0, st>>>(b, r, 2);
    kb_vertex_pass<DT><<<nsm * L.vpass_ctas, 256, 0, st>>>(b, r, 1);
    kb_compact<<<std::min(b.G, nsm * 2), kCompactThreads, 0, st>>>(b, r, 1);
    kb_plan<<<1, 1024, 0, st>>>(b, r, 0, 1, b.plan_scan, L.scan_unroll);
    batch_scan<DT>(b, L, r, 1, st);
    kb_vertex_pass<DT><<<nsm * L.vpass_ctas, 256, 0, st>>>(b, r, 3);
    // rows to re-accumulate, BC minus the old rows, accumulation, BC plus the new rows;
    // in graphs with pair corrections only the rows over the target cap, and the others
    // are corrected pair by pair after (the order of the single-graph path)
    kb_compact<<<std::min(b.G, nsm * 2), kCompactThreads, 0, st>>>(b, r, 2);
    if (L.pair_classes) batch_pair_lists(b, L, r, st);
    kb_plan<<<1, 1024, 0, st>>>(b, r, 1, 2, b.plan_bc, L.scan_unroll);
    kb_plan<<<1, 1024, 0, st>>>(b, r, 2, 2, b.plan_acc, L.scan_unroll);
    kb_bc_partial<<<nsm * L.bc_ctas, 256, 0, st>>>(b, r, b.plan_bc);
    kb_bc_finish<<<nsm * 2, 256, 0, st>>>(b, r, -1.0);
    if (L.acc_threads == 128) kb_accum<DT, 128><<<L.acc_grid, 128, L.acc_smem, st>>>(b, r, b.plan_acc);
    else if (L.acc_threads == 256) kb_accum<DT, 256><<<L.acc_grid, 256, L.acc_smem, st>>>(b, r, b.plan_acc);
    else kb_accum<DT, 512><<<L.acc_grid, 512, L.acc_smem, st>>>(b, r, b.plan_acc);
    kb_bc_partial<<<nsm * L.bc_ctas, 256, 0, st>>>(b, r, b.plan_bc);
    kb_bc_finish<<<nsm * 2, 256, 0, st>>>(b, r, +1.0);
    if (L.pair_classes) batch_pair_launches(b, L, r, sizeof(DT), st);
}

void batch_plan(const BatchArgs& b, int r, int kind, int phase_active, int64_t* out, int scan_unroll,
                cudaStream_t st) {
    kb_plan<<<1, 1024, 0, st>>>(b, r, kind, phase_active, out, scan_unroll);
}

void batch_config(BatchLaunch& L, int dbytes, int n_max, int64_t cap_max) {
    const size_t np = ((size_t)n_max + 31) & ~(size_t)31;
    const size_t base = 4 * np + 2 * (size_t)kBigCap;
    const size_t mb = 4 * (size_t)((cap_max + 31) / 32);
    const size_t limit = 180 * 1024;
    L.mask_in_smem = base + mb <= limit ? 1 : 0;
    L.acc_smem = (int)(L.mask_in_smem ? base + mb : base);
    int per_sm = 1;
    if (L.acc_threads != 128 && L.acc_threads != 256 && L.acc_threads != 512) L.acc_threads = kAccThreadsNarrow;
    auto occ = [&](auto kern, int threads) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, L.acc_smem);
    };
    if (dbytes == 4) {
        if (L.acc_threads == 128) occ(kb_accum<int32_t, 128>, 128);
        else if (L.acc_threads == 256) occ(kb_accum<int32_t, 256>, 256);
        else occ(kb_accum<int32_t, 512>, 512);
    } else {
        if (L.acc_threads == 128) occ(kb_accum<int64_t, 128>, 128);
        else if (L.acc_threads == 256) occ(kb_accum<int64_t, 256>, 256);
        else occ(kb_accum<int64_t, 512>, 512);
    }
    if (per_sm < 1) per_sm = 1;
    if (L.acc_per_sm > 0) per_sm = std::min(per_sm, L.acc_per_sm);
    L.acc_grid = L.nsm * per_sm;
    const int64_t head = ((3 * (int64_t)n_max + 2) + 3) & ~(int64_t)3;
    L.ws_stride = head + (L.mask_in_smem ? 0 : (((int64_t)mb / 4 + 3) & ~(int64_t)3));
}

void batch_launch_rounds(const BatchArgs& b, const BatchLaunch& L, int rounds, int dbytes, cudaStream_t st) {
    for (int r = 0; r < rounds; ++r) {
        if (dbytes == 4) round_launches<int32_t>(b, L, r, st);
        else round_launches<int64_t>(b, L, r, st);
    }
}

}  // namespace bcg
