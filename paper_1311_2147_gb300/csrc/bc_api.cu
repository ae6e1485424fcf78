// bc_api.cu -- host side of libbcgpu.so: handles, validation, the E* superset and the
// launch sequence of every update.  Declarations and conventions: include/bcgpu.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "bcgpu.h"
#include "bc_batch.cuh"
#include "bc_internal.cuh"

using namespace bcg;

namespace {

thread_local std::string g_init_error;

inline uint64_t arc_key(int32_t a, int32_t b) { return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b; }

struct HArc {
    int32_t a, b;
    int64_t w;
};

}  // namespace

struct bc_graph {
    Dev d{};
    int32_t n = 0;
    bool directed = true;
    int dbytes = 4;
    int64_t inf = INT32_MAX;
    bool poisoned = false;
    int poison_status = BC_OK;
    std::string last_error;
    bool full_scan = false;
    bool fused_edges = true;   // undirected edge updates in one pass over both directions
    // real weights (bc_init_static_f64): every weight is an integer number of units of
    // 2^w_exp; top_bits bounds their size (weights below 2^top_bits units)
    bool real_weights = false;
    int32_t w_exp = 0;
    int32_t top_bits = 0;
    // weights of every arc of G (G_D for undirected graphs)
    std::unordered_map<uint64_t, int64_t> wmap;
    // host mirror of the E* superset CSR
    // (slots [0, pool_top) hold the laid-out segments and moved ones; a vertex whose
    // segment fills up is moved to pool_top with room to grow, and E* is laid out
    // again only when the free region runs out)
    std::vector<int32_t> e_off, e_len, e_src, e_dst;
    std::vector<int32_t> e_capv;          // slots of each vertex's segment
    int64_t pool_top = 0;
    int64_t estar_rebuilds = 0;
    int64_t estar_moves = 0;
    std::vector<int64_t> e_w;
    std::unordered_map<uint64_t, int32_t> eslot;
    int64_t estar_arcs = 0;
    // staged batch
    std::vector<bc_update> staged;
    std::vector<int64_t> staged_first;   // first device entry of each staged update
    std::vector<int32_t> staged_k;
    std::vector<VEdge> h_entries;
    VEdge* d_entries = nullptr;
    int64_t d_entries_cap = 0;
    // bookkeeping
    int32_t* h_err = nullptr;             // pinned
    int64_t* h_stats = nullptr;           // pinned
    uint8_t* d_keep = nullptr;
    int64_t d_keep_cap = 0;
    int64_t ws_cap = 0;
    cudaEvent_t ev_done = nullptr;
    // second stream: full re-accumulation of some rows runs beside the pair corrections
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int64_t bytes = 0;
    double last_init_ms = 0.0;
    int64_t walk_cap_alloc = 0;   // entries allocated for the DAG walks' buffer
    std::vector<void*> allocs;
    std::vector<void*> allocs_async;   // stream-ordered (replaced while the handle lives)
    // launch accounting and optional per-class event timing
    int64_t launches = 0;
    bool profile = false;
    struct Rec {
        cudaEvent_t a, b;
        int cls, nl;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double prof_ms[BC_PROFILE_CLASSES] = {0};
    int64_t prof_launches[BC_PROFILE_CLASSES] = {0};
};

namespace {

int fail(bc_graph* g, int code, const std::string& msg) {
    if (g) g->last_error = msg;
    else g_init_error = msg;
    return code;
}

int cuda_fail(bc_graph* g, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(g, BC_ERR_OOM, m);
    return fail(g, BC_ERR_CUDA, m);
}

#define CK(g, call)                                               \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((g), e_, #call);  \
    } while (0)

template <typename T>
int dalloc(bc_graph* g, T** p, size_t count) {
    *p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) return cuda_fail(g, e, "cudaMalloc");
    g->allocs.push_back(*p);
    g->bytes += (int64_t)bytes;
    return BC_OK;
}

void dfree(bc_graph* g, void* p) {
    if (!p) return;
    auto it = std::find(g->allocs.begin(), g->allocs.end(), p);
    if (it != g->allocs.end()) g->allocs.erase(it);
    cudaFree(p);
}

// Stream-ordered allocation for the buffers that are replaced while the handle lives
// (the E* arrays, their keep flags, the accumulation work space): cudaFree waits for
// the whole device, the work of every other handle included, while a free ordered on
// this handle's stream waits only for this handle's earlier work.
template <typename T>
int dalloc_async(bc_graph* g, T** p, size_t count) {
    *p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), bytes, g->d.st);
    if (e != cudaSuccess) return cuda_fail(g, e, "cudaMallocAsync");
    g->allocs_async.push_back(*p);
    g->bytes += (int64_t)bytes;
    return BC_OK;
}

void dfree_async(bc_graph* g, void* p) {
    if (!p) return;
    auto it = std::find(g->allocs_async.begin(), g->allocs_async.end(), p);
    if (it != g->allocs_async.end()) g->allocs_async.erase(it);
    cudaFreeAsync(p, g->d.st);
}

int status_of_err(int32_t f) {
    if (f & ERRF_OVERFLOW) return BC_ERR_OVERFLOW;
    if (f & ERRF_DIST) return BC_ERR_DIST_OVERFLOW;
    if (f & ERRF_TIMEOUT) return BC_ERR_TIMEOUT;
    return BC_OK;
}

const char* status_text(int s) {
    switch (s) {
        case BC_ERR_OVERFLOW: return "a shortest-path count does not fit in 64 bits";
        case BC_ERR_DIST_OVERFLOW: return "a distance does not fit the distance type";
        case BC_ERR_TIMEOUT: return "a bounded device wait gave up";
        default: return "";
    }
}

cudaEvent_t take_event(bc_graph* g) {
    if (!g->pool.empty()) {
        cudaEvent_t e = g->pool.back();
        g->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Run one group of nl launches of kernel class cls, timed with events when profiling.
template <typename F>
void timed(bc_graph* g, int cls, int nl, F&& fn) {
    g->launches += nl;
    if (!g->profile) {
        fn();
        return;
    }
    cudaEvent_t a = take_event(g), b = take_event(g);
    cudaEventRecord(a, g->d.st);
    fn();
    cudaEventRecord(b, g->d.st);
    g->pending.push_back({a, b, cls, nl});
}

// Fold finished event pairs into the per-class sums (the stream has been synchronised).
void collect_profile(bc_graph* g) {
    for (auto& r : g->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) g->prof_ms[r.cls] += ms;
        g->prof_launches[r.cls] += r.nl;
        g->pool.push_back(r.a);
        g->pool.push_back(r.b);
    }
    g->pending.clear();
}

// Wait for the stream and turn a device-side error into a status (poisoning the handle).
int sync_check(bc_graph* g) {
    CK(g, cudaStreamSynchronize(g->d.st));
    collect_profile(g);
    CK(g, cudaMemcpy(g->h_err, g->d.err, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (*g->h_err) {
        g->poisoned = true;
        g->poison_status = status_of_err(*g->h_err);
        return fail(g, g->poison_status, status_text(g->poison_status));
    }
    return BC_OK;
}

// Lay the E* superset out with slack per vertex and upload it.  The device arrays get
// a quarter more slots than the layout needs: the free region where full segments move.
int estar_layout(bc_graph* g, const std::vector<HArc>& arcs, const std::vector<int32_t>* extra = nullptr) {
    const int32_t n = g->n;
    std::vector<int32_t> deg(n, 0);
    for (const HArc& x : arcs) deg[x.a]++;
    g->e_off.assign(n + 1, 0);
    g->e_len.assign(n, 0);
    g->e_capv.assign(n, 0);
    for (int32_t a = 0; a < n; ++a) {
        g->e_capv[a] = deg[a] + 2 + deg[a] / 8 + (extra ? (*extra)[a] : 0);
        g->e_off[a + 1] = g->e_off[a] + g->e_capv[a];
    }
    const int64_t cap = g->e_off[n];
    Dev& d = g->d;
    const size_t asz = g->dbytes == 4 ? sizeof(Arc<int32_t>) : sizeof(Arc<int64_t>);
    if (cap + cap / 8 > d.e_cap) {
        dfree_async(g, d.e_src);
        dfree_async(g, d.e_arc);
        d.e_src = nullptr;
        d.e_arc = nullptr;
        const int64_t ncap = cap + cap / 4 + 64;
        int rc;
        if ((rc = dalloc_async(g, &d.e_src, ncap))) return rc;
        unsigned char* p = nullptr;
        if ((rc = dalloc_async(g, &p, ncap * asz))) return rc;
        d.e_arc = p;
        d.e_cap = ncap;
    }
    g->pool_top = cap;
    g->e_src.assign(d.e_cap, 0);
    g->e_dst.assign(d.e_cap, -1);
    g->e_w.assign(d.e_cap, 0);
    g->eslot.clear();
    g->eslot.reserve(arcs.size() * 2 + 16);
    for (int32_t a = 0; a < n; ++a)
        for (int32_t s = g->e_off[a]; s < g->e_off[a + 1]; ++s) g->e_src[s] = a;
    for (const HArc& x : arcs) {
        const int32_t slot = g->e_off[x.a] + g->e_len[x.a]++;
        g->e_dst[slot] = x.b;
        g->e_w[slot] = x.w;
        g->eslot[arc_key(x.a, x.b)] = slot;
    }
    g->estar_arcs = (int64_t)arcs.size();
    std::vector<unsigned char> arc_bytes(d.e_cap * asz);
    if (g->dbytes == 4) {
        Arc<int32_t>* A = reinterpret_cast<Arc<int32_t>*>(arc_bytes.data());
        for (int64_t i = 0; i < d.e_cap; ++i) A[i] = Arc<int32_t>{g->e_dst[i], (int32_t)g->e_w[i]};
    } else {
        Arc<int64_t>* A = reinterpret_cast<Arc<int64_t>*>(arc_bytes.data());
        for (int64_t i = 0; i < d.e_cap; ++i) A[i] = Arc<int64_t>{(int64_t)g->e_dst[i], g->e_w[i]};
    }
    CK(g, cudaMemcpyAsync(d.e_off, g->e_off.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, d.st));
    CK(g, cudaMemcpyAsync(d.e_len, g->e_len.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, d.st));
    CK(g, cudaMemcpyAsync(d.e_src, g->e_src.data(), sizeof(int32_t) * d.e_cap, cudaMemcpyHostToDevice, d.st));
    CK(g, cudaMemcpyAsync(d.e_arc, arc_bytes.data(), arc_bytes.size(), cudaMemcpyHostToDevice, d.st));
    CK(g, cudaStreamSynchronize(d.st));
    // launch shape of the accumulation depends on the capacity: size its work space
    accum_config(d);
    const int64_t need = (int64_t)d.acc_grid * d.ws_stride;
    if (need > g->ws_cap) {
        dfree_async(g, d.ws);
        d.ws = nullptr;
        int rc;
        if ((rc = dalloc_async(g, &d.ws, need))) return rc;
        g->ws_cap = need;
    }
    return BC_OK;
}

// Rebuild the E* superset when a vertex runs out of slack: keep the arcs that are still
// in E* (w = d), add the pending arcs, lay out again.
int estar_rebuild(bc_graph* g, const std::vector<HArc>& pending) {
    int rc = sync_check(g);
    if (rc) return rc;
    Dev& d = g->d;
    if (d.e_cap > g->d_keep_cap) {
        dfree_async(g, g->d_keep);
        g->d_keep = nullptr;
        if ((rc = dalloc_async(g, &g->d_keep, d.e_cap))) return rc;
        g->d_keep_cap = d.e_cap;
    }
    launch_estar_keep(d, g->d_keep);
    std::vector<uint8_t> keep(d.e_cap);
    CK(g, cudaMemcpyAsync(keep.data(), g->d_keep, d.e_cap, cudaMemcpyDeviceToHost, d.st));
    CK(g, cudaStreamSynchronize(d.st));
    std::unordered_set<uint64_t> pend;
    for (const HArc& x : pending) pend.insert(arc_key(x.a, x.b));
    std::vector<HArc> arcs;
    arcs.reserve(g->estar_arcs + pending.size());
    const int64_t cap = (int64_t)g->e_dst.size();
    for (int64_t s = 0; s < cap; ++s) {
        if (g->e_dst[s] < 0 || !keep[s]) continue;
        if (pend.count(arc_key(g->e_src[s], g->e_dst[s]))) continue;
        arcs.push_back({g->e_src[s], g->e_dst[s], g->e_w[s]});
    }
    for (const HArc& x : pending) arcs.push_back(x);
    g->estar_rebuilds++;
    return estar_layout(g, arcs);
}

// Validate one update against the host weights and produce its edge entries (at vertex
// v).  Does not modify anything.
int validate_update(bc_graph* g, const bc_update& u, const bc_vedge* edges, int64_t n_edges,
                    int32_t* v_out, std::vector<VEdge>& ent) {
    ent.clear();
    const int32_t n = g->n;
    auto check_arc = [&](int32_t a, int32_t b, int64_t w) -> int {
        if (a < 0 || a >= n || b < 0 || b >= n || a == b)
            return fail(g, BC_ERR_ARG, "edge endpoint out of range or self-loop");
        if (w < 1 || w >= g->inf) return fail(g, BC_ERR_ARG, "weight outside [1, INF-1]");
        auto it = g->wmap.find(arc_key(a, b));
        if (it != g->wmap.end() && w >= it->second)
            return fail(g, BC_ERR_NOT_INCREMENTAL, "new weight is not below the current weight");
        return BC_OK;
    };
    if (u.kind == BC_UPD_EDGE) {
        int rc = check_arc(u.u, u.v, u.w);
        if (rc) return rc;
        *v_out = u.v;
        ent.push_back({u.u, 0, u.w});
        return BC_OK;
    }
    if (u.kind != BC_UPD_VERTEX) return fail(g, BC_ERR_ARG, "unknown update kind");
    if (u.v < 0 || u.v >= n) return fail(g, BC_ERR_ARG, "vertex out of range");
    if (u.k < 1) return fail(g, BC_ERR_ARG, "empty vertex update");
    if (!edges || u.first < 0 || u.first + u.k > n_edges) return fail(g, BC_ERR_ARG, "vertex update edges out of range");
    std::unordered_set<uint64_t> seen;
    for (int32_t j = 0; j < u.k; ++j) {
        const bc_vedge& e = edges[u.first + j];
        int32_t dir = g->directed ? e.dir : 0;
        if (g->directed && dir != 0 && dir != 1) return fail(g, BC_ERR_ARG, "edge direction must be 0 or 1");
        if (!seen.insert(arc_key(e.x, dir)).second) return fail(g, BC_ERR_ARG, "repeated edge in a vertex update");
        int rc = (dir == 0) ? check_arc(e.x, u.v, e.w) : check_arc(u.v, e.x, e.w);
        if (rc) return rc;
        ent.push_back({e.x, dir, e.w});
    }
    *v_out = u.v;
    return BC_OK;
}

// Move the segment of vertex a to the free region with room for want arcs (host mirror
// and a device move record).  False when the free region is too small.
bool estar_move(bc_graph* g, int32_t a, int32_t want, std::vector<EMove>& moves) {
    const int32_t len = g->e_len[a];
    const int64_t c = (int64_t)want + want / 2 + 8;
    if (g->pool_top + c > g->d.e_cap) return false;
    const int32_t from = g->e_off[a], to = (int32_t)g->pool_top;
    g->pool_top += c;
    for (int32_t i = 0; i < len; ++i) {
        g->e_dst[to + i] = g->e_dst[from + i];
        g->e_w[to + i] = g->e_w[from + i];
        g->eslot[arc_key(a, g->e_dst[to + i])] = to + i;
        g->e_dst[from + i] = -1;
    }
    for (int64_t i = 0; i < c; ++i) g->e_src[to + i] = a;
    g->e_off[a] = to;
    g->e_capv[a] = (int32_t)c;
    moves.push_back({a, from, to, len});
    g->estar_moves++;
    return true;
}

// Apply a validated update to the host weights and the E* superset mirror; fills the
// device moves and writes to make.  Sets *rebuild when a vertex has no room left and
// the free region cannot take its segment either.
void mirror_update(bc_graph* g, int32_t v, const std::vector<VEdge>& ent, std::vector<EOp>& ops,
                   std::vector<EMove>& moves, std::vector<HArc>& arcs, bool* rebuild) {
    arcs.clear();
    for (const VEdge& e : ent) {
        if (!g->directed) {
            arcs.push_back({e.x, v, e.w});
            arcs.push_back({v, e.x, e.w});
        } else if (e.dir == 0) {
            arcs.push_back({e.x, v, e.w});
        } else {
            arcs.push_back({v, e.x, e.w});
        }
    }
    *rebuild = false;
    ops.clear();
    moves.clear();
    // room first: segments that cannot take their new arcs move before any slot is written
    std::vector<std::pair<int32_t, int32_t>> need;   // (vertex, new arcs)
    for (const HArc& x : arcs) {
        if (g->eslot.count(arc_key(x.a, x.b))) continue;
        auto it = std::find_if(need.begin(), need.end(), [&](const std::pair<int32_t, int32_t>& p) {
            return p.first == x.a;
        });
        if (it == need.end()) need.push_back({x.a, 1});
        else it->second++;
    }
    for (const auto& p : need) {
        const int32_t a = p.first;
        if (g->e_len[a] + p.second <= g->e_capv[a]) continue;
        if (!estar_move(g, a, g->e_len[a] + p.second, moves)) {
            *rebuild = true;
            break;
        }
    }
    for (const HArc& x : arcs) {
        g->wmap[arc_key(x.a, x.b)] = x.w;
        if (*rebuild) continue;
        auto it = g->eslot.find(arc_key(x.a, x.b));
        if (it != g->eslot.end()) {
            g->e_w[it->second] = x.w;
            ops.push_back({it->second, x.a, x.b, g->e_len[x.a], x.w});
            continue;
        }
        const int32_t a = x.a;
        const int32_t slot = g->e_off[a] + g->e_len[a]++;
        g->e_src[slot] = a;
        g->e_dst[slot] = x.b;
        g->e_w[slot] = x.w;
        g->eslot[arc_key(a, x.b)] = slot;
        g->estar_arcs++;
        ops.push_back({slot, a, x.b, g->e_len[a], x.w});
    }
}

// Scratch of the DAG walks (per warp of the walk grid: a vertex list, a touched-column
// list and a row of column sums), allocated once per handle.
int walk_alloc(bc_graph* g) {
    Dev& d = g->d;
    if (d.walk_list) return BC_OK;
    if (walk_smem(d.n) > kWalkSmemMax) return fail(g, BC_ERR_ARG, "pair_walk: n too large for the walk's bit sets");
    const size_t n = (size_t)d.n;
    // expected use is ~25 entries per changed pair; every warp may leave part of a block unused
    d.walk_cap = (int64_t)(8u << 20) + 64 * (int64_t)n + walk_warps(d.nsm) * kWalkBlock;
    g->walk_cap_alloc = d.walk_cap;
    int rc;
    if ((rc = dalloc(g, &d.walk_list, (size_t)walk_warps(d.nsm) * n)) ||
        (rc = dalloc(g, &d.walk_buf, (size_t)d.walk_cap)) || (rc = dalloc(g, &d.walk_useg, n * kPairCap * 4)) ||
        (rc = dalloc(g, &d.walk_acc2, (size_t)walk_ctas(d.nsm) * 2 * n)) ||
        (rc = dalloc(g, &d.walk_tl, (size_t)walk_ctas(d.nsm) * n)) || (rc = dalloc(g, &d.walk_ctl, 8)) ||
        (rc = dalloc(g, &d.walk_rowE, n)))
        return rc;
    cudaError_t e = cudaMemsetAsync(d.walk_acc2, 0, sizeof(int64_t) * (size_t)walk_ctas(d.nsm) * 2 * n, d.st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.walk_ctl, 0, sizeof(int32_t) * 8, d.st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.walk_rowE, 0, sizeof(int32_t) * n, d.st);
    if (e != cudaSuccess) return cuda_fail(g, e, "cudaMemsetAsync");
    return BC_OK;
}

int enqueue_update(bc_graph* g, int32_t v, const std::vector<VEdge>& ent, const VEdge* d_ent) {
    Dev& d = g->d;
    std::vector<EOp> ops;
    std::vector<EMove> moves;
    std::vector<HArc> arcs;
    bool rebuild = false;
    // the DAG walks of the pair corrections need the update's edges with their old weights
    WalkUpd upd{};
    const bool walk = d.pair_on && d.pair_walk && !g->directed && (int)ent.size() <= kWalkMaxEdges;
    if (walk) {
        upd.v = v;
        upd.k = (int32_t)ent.size();
        for (int j = 0; j < upd.k; ++j) {
            upd.x[j] = ent[j].x;
            auto it = g->wmap.find(arc_key(ent[j].x, v));
            upd.wold[j] = it == g->wmap.end() ? -1 : it->second;
        }
    }
    mirror_update(g, v, ent, ops, moves, arcs, &rebuild);
    // moves made before a rebuild was found necessary are applied too: the rebuild reads
    // the device slots against the host mirror
    for (size_t i = 0; i < moves.size(); i += kMaxEMoves) {
        EMoves pack{};
        pack.count = (int32_t)std::min<size_t>(kMaxEMoves, moves.size() - i);
        for (int j = 0; j < pack.count; ++j) pack.mv[j] = moves[i + j];
        timed(g, 4, 1, [&] { launch_estar_move(d, pack); });
    }
    if (rebuild) {
        int rc = estar_rebuild(g, arcs);
        if (rc) return rc;
    } else {
        for (size_t i = 0; i < ops.size(); i += kMaxEOps) {
            EOps pack{};
            pack.count = (int32_t)std::min<size_t>(kMaxEOps, ops.size() - i);
            for (int j = 0; j < pack.count; ++j) pack.op[j] = ops[i + j];
            timed(g, 4, 1, [&] { launch_estar_write(d, pack); });
        }
    }
    int32_t kin = 0, kout = 0;
    for (const VEdge& e : ent) {
        if (!g->directed || e.dir == 0) kin++;
        if (!g->directed || e.dir == 1) kout++;
    }
    const int32_t k = (int32_t)ent.size();
    const int full = g->full_scan ? 1 : 0;
    const bool pair = d.pair_on != 0;
    // an undirected edge update: one pass over both directions (the vector path of the
    // rank-1 pass; every row's candidates taken from the state before the update)
    const bool fused = !g->directed && k == 1 && !g->full_scan && g->fused_edges && g->n % (16 / g->dbytes) == 0;
    if (fused) {
        kin = kout = 0;
        timed(g, 3, 1, [&] { launch_edge_prep(d, ent[0].x, v, ent[0].w); });
        timed(g, 0, 1, [&] { launch_edge_scan(d); });
    }
    if (kin) {
        timed(g, 3, 1, [&] { launch_alg4_in(d, v, d_ent, k); });
        timed(g, 4, 1, [&] { launch_compact(d, d.mark, 0, d.rows, d.counts, full, 0); });
        timed(g, 0, 1, [&] { launch_scan_in(d, v); });
    }
    if (kout) {
        timed(g, 3, 2, [&] {
            launch_alg4_out(d, v, d_ent, k);
            launch_rows_out(d, v, d_ent, k);
        });
        timed(g, 4, 1, [&] { launch_compact(d, d.mark, 0, d.rows, d.counts, full, 0); });
        timed(g, 0, 1, [&] { launch_scan_out(d, v); });
        timed(g, 3, 1, [&] { launch_write_row(d, v); });
    }
    if (pair) {
        // rows with more changed targets than kPairCap (and row v): Algorithm 1 in full;
        // the others: pair corrections of their dependency rows
        timed(g, 4, 1, [&] { launch_pair_lists(d); });
        // kernels of launch_pairdep: plan and weights, then the walks (units, two hash-table
        // row classes, whole-CTA rows) and the gated column test, or the column test alone
        const int pair_launches = walk ? 7 : 3;
        // BC: the full rows are subtracted before and added after their re-accumulation;
        // the corrected rows add their changes to BC's fixed-point change as they are
        // made, which k_bc_fix folds into BC at the end
        if (!g->profile) {
            // the two write disjoint dependency rows and only read the rest of the state:
            // the (latency-bound, partial-wave) accumulation of the full rows and their
            // new BC sums run on the second stream beside the pair corrections, which do
            // not touch BC itself until k_bc_fix, after the join.  The old rows' BC sums
            // are taken first on this stream, so that the accumulation is the first
            // kernel of the second stream: launched before the pair corrections, it gets
            // its SMs before their CTAs (which stay resident until all their work is
            // taken) fill the GPU.
            Dev ds = d;
            ds.st = g->side;
            launch_bc_rows_list(d, -1, d.full_rows, d.counts + 3);
            CK(g, cudaEventRecord(g->ev_fork, d.st));
            CK(g, cudaStreamWaitEvent(g->side, g->ev_fork, 0));
            launch_accum_rows(ds, d.full_rows, d.counts + 3);
            launch_bc_rows_list(ds, +1, d.full_rows, d.counts + 3);
            CK(g, cudaEventRecord(g->ev_join, g->side));
            launch_pairdep(d, walk ? &upd : nullptr);
            CK(g, cudaStreamWaitEvent(d.st, g->ev_join, 0));
            launch_bc_fix(d);
            g->launches += 6 + pair_launches;
        } else {
            timed(g, 2, 2, [&] { launch_bc_rows_list(d, -1, d.full_rows, d.counts + 3); });
            timed(g, 5, pair_launches, [&] { launch_pairdep(d, walk ? &upd : nullptr); });
            timed(g, 1, 1, [&] { launch_accum_rows(d, d.full_rows, d.counts + 3); });
            timed(g, 2, 3, [&] {
                launch_bc_rows_list(d, +1, d.full_rows, d.counts + 3);
                launch_bc_fix(d);
            });
        }
        timed(g, 4, 1, [&] { launch_pair_clear(d); });
    } else {
        timed(g, 4, 1, [&] { launch_compact(d, d.changed, 1, d.acc_rows, d.counts + 1, 0, 1); });
        timed(g, 2, 2, [&] { launch_bc_rows(d, -1, 0); });
        timed(g, 1, 1, [&] { launch_accum(d, 0); });
        timed(g, 2, 2, [&] { launch_bc_rows(d, +1, 0); });
    }
    CK(g, cudaGetLastError());
    return BC_OK;
}

void destroy_all(bc_graph* g) {
    if (!g) return;
    cudaStreamSynchronize(g->d.st);
    if (g->side) {
        cudaStreamSynchronize(g->side);
        cudaStreamDestroy(g->side);
    }
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->d.st3) {
        cudaStreamSynchronize(g->d.st3);
        cudaStreamDestroy(g->d.st3);
    }
    if (g->d.ev3_fork) cudaEventDestroy(g->d.ev3_fork);
    if (g->d.ev3_join) cudaEventDestroy(g->d.ev3_join);
    for (void* p : g->allocs_async) cudaFreeAsync(p, g->d.st);
    if (!g->allocs_async.empty()) cudaStreamSynchronize(g->d.st);
    g->allocs_async.clear();
    for (void* p : g->allocs) cudaFree(p);
    g->allocs.clear();
    if (g->h_err) cudaFreeHost(g->h_err);
    if (g->h_stats) cudaFreeHost(g->h_stats);
    if (g->ev_done) cudaEventDestroy(g->ev_done);
    for (auto& r : g->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : g->pool) cudaEventDestroy(e);
    delete g;
}

bool check_alive(bc_graph* g, int* rc) {
    if (!g) {
        *rc = BC_ERR_ARG;
        return false;
    }
    if (g->poisoned) {
        g->last_error = "handle poisoned by an earlier device-side error";
        *rc = BC_ERR_POISONED;
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

int bc_init_static(bc_graph** out, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                   const int64_t* w, uint32_t flags, void* cuda_stream) {
    if (!out) return fail(nullptr, BC_ERR_ARG, "out is NULL");
    *out = nullptr;
    const bool dir = (flags & BC_DIRECTED) != 0, und = (flags & BC_UNDIRECTED) != 0;
    const bool i32 = (flags & BC_DIST_I32) != 0, i64 = (flags & BC_DIST_I64) != 0;
    if (dir == und || i32 == i64) return fail(nullptr, BC_ERR_ARG, "flags need one of DIRECTED/UNDIRECTED and one of DIST_I32/DIST_I64");
    if (n < 1 || n > 32768) return fail(nullptr, BC_ERR_ARG, "n must be in [1, 32768]");
    if (m < 0 || (m > 0 && (!src || !dst || !w))) return fail(nullptr, BC_ERR_ARG, "bad edge arrays");
    bc_graph* g = new bc_graph();
    g->n = n;
    g->directed = dir;
    g->dbytes = i32 ? 4 : 8;
    g->inf = i32 ? (int64_t)INT32_MAX : INT64_MAX;
    Dev& d = g->d;
    d.n = n;
    d.dbytes = g->dbytes;
    d.directed = dir ? 1 : 0;
    d.st = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) {
        int rc = cuda_fail(nullptr, ce, "cudaGetDevice");
        delete g;
        return rc;
    }
    // ---- arcs of G (G_D), validated
    const int64_t arcs = dir ? m : 2 * m;
    std::vector<HArc> all;
    all.reserve(arcs);
    g->wmap.reserve(arcs * 2 + 16);
    for (int64_t i = 0; i < m; ++i) {
        const int32_t a = src[i], b = dst[i];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b || w[i] < 1 || w[i] >= g->inf) {
            destroy_all(g);
            return fail(nullptr, BC_ERR_ARG, "edge out of range, self-loop or weight outside [1, INF-1]");
        }
        if (!g->wmap.emplace(arc_key(a, b), w[i]).second || (!dir && !g->wmap.emplace(arc_key(b, a), w[i]).second)) {
            destroy_all(g);
            return fail(nullptr, BC_ERR_ARG, "repeated edge");
        }
        all.push_back({a, b, w[i]});
        if (!dir) all.push_back({b, a, w[i]});
    }
    // CSR of G by tail
    std::vector<int32_t> off(n + 1, 0), csrc(arcs), cdst(arcs);
    std::vector<int64_t> cw(arcs);
    for (const HArc& x : all) off[x.a + 1]++;
    for (int32_t a = 0; a < n; ++a) off[a + 1] += off[a];
    {
        std::vector<int32_t> pos(off.begin(), off.end() - 1);
        for (const HArc& x : all) {
            const int32_t p = pos[x.a]++;
            csrc[p] = x.a;
            cdst[p] = x.b;
            cw[p] = x.w;
        }
    }
    // ---- device memory
    const size_t nn = (size_t)n * n;
    int rc = BC_OK;
    d.nrb_max = (n + kRowsPerBlock - 1) / kRowsPerBlock;
    d.g_arcs = arcs;
    if (g->dbytes == 4) {
        int32_t *pD, *pfD, *pcD, *pcD2, *pgw;
        if ((rc = dalloc(g, &pD, nn)) || (rc = dalloc(g, &pfD, n)) || (rc = dalloc(g, &pcD, n)) ||
            (rc = dalloc(g, &pcD2, n)) || (rc = dalloc(g, &pgw, arcs))) {
            destroy_all(g);
            return fail(nullptr, rc, "device allocation failed");
        }
        d.D = pD; d.fD = pfD; d.cD = pcD; d.cD2 = pcD2; d.g_w = pgw;
    } else {
        int64_t *pD, *pfD, *pcD, *pcD2, *pgw;
        if ((rc = dalloc(g, &pD, nn)) || (rc = dalloc(g, &pfD, n)) || (rc = dalloc(g, &pcD, n)) ||
            (rc = dalloc(g, &pcD2, n)) || (rc = dalloc(g, &pgw, arcs))) {
            destroy_all(g);
            return fail(nullptr, rc, "device allocation failed");
        }
        d.D = pD; d.fD = pfD; d.cD = pcD; d.cD2 = pcD2; d.g_w = pgw;
    }
    if ((rc = dalloc(g, &d.S, nn)) || (rc = dalloc(g, &d.Dl, nn)) || (rc = dalloc(g, &d.bc_hi, n)) ||
        (rc = dalloc(g, &d.bc_lo, n)) || (rc = dalloc(g, &d.g_off, n + 1)) || (rc = dalloc(g, &d.g_src, arcs)) ||
        (rc = dalloc(g, &d.g_dst, arcs)) || (rc = dalloc(g, &d.e_off, n + 1)) || (rc = dalloc(g, &d.e_len, n)) ||
        (rc = dalloc(g, &d.err, 1)) || (rc = dalloc(g, &d.stats, kStats)) || (rc = dalloc(g, &d.mark, n)) ||
        (rc = dalloc(g, &d.changed, n)) || (rc = dalloc(g, &d.rows, n)) || (rc = dalloc(g, &d.acc_rows, n)) ||
        (rc = dalloc(g, &d.counts, 8)) || (rc = dalloc(g, &d.fS, n)) || (rc = dalloc(g, &d.fM, n)) ||
        (rc = dalloc(g, &d.cS, n)) || (rc = dalloc(g, &d.cM, n)) || (rc = dalloc(g, &d.cS2, n)) ||
        (rc = dalloc(g, &d.partial, (size_t)d.nrb_max * n))) {
        destroy_all(g);
        return fail(nullptr, rc, "device allocation failed");
    }
    // pair corrections (undirected graphs): change map, old values of changed pairs,
    // target lists and plans
    d.tcap = kPairCap;
    d.chg_words = (n + 31) / 32;
    if (!dir) {
        uint8_t* poD = nullptr;
        if ((rc = dalloc(g, &poD, nn * (size_t)g->dbytes)) || (rc = dalloc(g, &d.oldS, nn)) ||
            (rc = dalloc(g, &d.chg, (size_t)n * d.chg_words)) || (rc = dalloc(g, &d.tcnt, n)) ||
            (rc = dalloc(g, &d.tlist, (size_t)n * kPairCap)) || (rc = dalloc(g, &d.full_rows, n)) ||
            (rc = dalloc(g, &d.pair_rows, n)) ||
            (rc = dalloc(g, reinterpret_cast<uint8_t**>(&d.plan), (size_t)n * kPairCap * 40)) ||
            (rc = dalloc(g, &d.pair_w, (size_t)n + 1)) || (rc = dalloc(g, &d.bcfix, 2 * (size_t)n))) {
            destroy_all(g);
            return fail(nullptr, rc, "device allocation failed");
        }
        d.oldD = poD;
        d.pair_on = 1;
    }
    if (cudaMallocHost(&g->h_err, sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost(&g->h_stats, kStats * sizeof(int64_t)) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming) != cudaSuccess ||
        (!dir && (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess ||
                  cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                  cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess ||
                  cudaStreamCreateWithFlags(&g->d.st3, cudaStreamNonBlocking) != cudaSuccess ||
                  cudaEventCreateWithFlags(&g->d.ev3_fork, cudaEventDisableTiming) != cudaSuccess ||
                  cudaEventCreateWithFlags(&g->d.ev3_join, cudaEventDisableTiming) != cudaSuccess))) {
        destroy_all(g);
        return fail(nullptr, BC_ERR_OOM, "pinned host allocation, stream or event creation failed");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto bail = [&](int code, const std::string& msg) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        destroy_all(g);
        return fail(nullptr, code, msg);
    };
#define CKI(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bail(e_ == cudaErrorMemoryAllocation ? BC_ERR_OOM : BC_ERR_CUDA,        \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)
    CKI(scan_setup());
    CKI(walk_setup());
    if (!dir && n >= kWalkDefaultMinN) {
        if ((rc = walk_alloc(g))) return bail(rc, g->last_error);
        d.pair_walk = 1;
    }
    CKI(cudaMemsetAsync(d.err, 0, sizeof(int32_t), d.st));
    CKI(cudaMemsetAsync(d.stats, 0, kStats * sizeof(int64_t), d.st));
    CKI(cudaMemsetAsync(d.mark, 0, n, d.st));
    CKI(cudaMemsetAsync(d.changed, 0, n, d.st));
    CKI(cudaMemsetAsync(d.counts, 0, 8 * sizeof(int32_t), d.st));
    if (!dir) {
        CKI(cudaMemsetAsync(d.chg, 0, sizeof(uint32_t) * n * d.chg_words, d.st));
        CKI(cudaMemsetAsync(d.tcnt, 0, sizeof(int32_t) * n, d.st));
        CKI(cudaMemsetAsync(d.bcfix, 0, sizeof(int64_t) * 2 * n, d.st));
    }
    CKI(cudaStreamSynchronize(d.st));
    CKI(cudaEventRecord(e0, d.st));
    CKI(cudaMemcpyAsync(d.g_off, off.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, d.st));
    CKI(cudaMemcpyAsync(d.g_src, csrc.data(), sizeof(int32_t) * arcs, cudaMemcpyHostToDevice, d.st));
    CKI(cudaMemcpyAsync(d.g_dst, cdst.data(), sizeof(int32_t) * arcs, cudaMemcpyHostToDevice, d.st));
    std::vector<int32_t> w32;
    if (g->dbytes == 4) {
        w32.resize(arcs);
        for (int64_t i = 0; i < arcs; ++i) w32[i] = (int32_t)cw[i];
        CKI(cudaMemcpyAsync(d.g_w, w32.data(), sizeof(int32_t) * arcs, cudaMemcpyHostToDevice, d.st));
    } else {
        CKI(cudaMemcpyAsync(d.g_w, cw.data(), sizeof(int64_t) * arcs, cudaMemcpyHostToDevice, d.st));
    }
    // all-pairs distances, then E* read off them.  Unless asked for the search over every
    // arc, arcs found outside E* are pruned as the searches finish (k_static.cu), the
    // sources running highest out-degree first.
    const bool prune = (flags & BC_STATIC_ALL_ARCS) == 0 && arcs > 0;
    if (prune) {
        std::vector<int32_t> order(n);
        for (int32_t i = 0; i < n; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            return off[a + 1] - off[a] > off[b + 1] - off[b];
        });
        // scratch in the dependency rows (n^2 float-float pairs, >= 4 (arcs + n) bytes),
        // which the accumulation writes only after the searches: no allocation here (a
        // cudaFree waits for the whole device, other handles' work included)
        d.p_dst = reinterpret_cast<int32_t*>(d.Dl);
        d.s_order = d.p_dst + arcs;
        CKI(cudaMemcpyAsync(d.p_dst, d.g_dst, sizeof(int32_t) * arcs, cudaMemcpyDeviceToDevice, d.st));
        CKI(cudaMemcpyAsync(d.s_order, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, d.st));
    }
    launch_sssp(d);
    // the E* flags, also in the dependency rows' memory (free until the accumulation)
    uint8_t* d_flags = reinterpret_cast<uint8_t*>(d.Dl);
    launch_estar_flags(d, d_flags);
    std::vector<uint8_t> eflags(arcs);
    CKI(cudaMemcpyAsync(eflags.data(), d_flags, arcs, cudaMemcpyDeviceToHost, d.st));
    CKI(cudaStreamSynchronize(d.st));
    CKI(cudaGetLastError());
    d.p_dst = d.s_order = nullptr;
    {
        std::vector<HArc> estar;
        for (int64_t i = 0; i < arcs; ++i)
            if (eflags[i]) estar.push_back({csrc[i], cdst[i], cw[i]});
        if ((rc = estar_layout(g, estar))) return bail(rc, g->last_error);
    }
    // path counts, DAGs and dependencies of every source; BC as column sums
    launch_accum(d, 1);
    launch_bc_rows(d, +1, 1);
    CKI(cudaGetLastError());
    CKI(cudaEventRecord(e1, d.st));
    CKI(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    g->last_init_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
#undef CKI
    rc = sync_check(g);
    if (rc) {
        std::string msg = g->last_error;
        destroy_all(g);
        return fail(nullptr, rc, msg);
    }
    *out = g;
    return BC_OK;
}

int bc_stage_updates(bc_graph* g, int32_t count, const bc_update* ups, const bc_vedge* edges,
                     int64_t n_edges) {
    int rc;
    if (!check_alive(g, &rc)) return rc;
    if (count < 0 || (count > 0 && !ups) || n_edges < 0 || (n_edges > 0 && !edges))
        return fail(g, BC_ERR_ARG, "bad batch arrays");
    g->staged.assign(ups, ups + count);
    g->staged_first.assign(count, 0);
    g->staged_k.assign(count, 0);
    g->h_entries.clear();
    for (int32_t i = 0; i < count; ++i) {
        const bc_update& u = ups[i];
        g->staged_first[i] = (int64_t)g->h_entries.size();
        if (u.kind == BC_UPD_EDGE) {
            g->h_entries.push_back({u.u, 0, u.w});
            g->staged_k[i] = 1;
        } else if (u.kind == BC_UPD_VERTEX && u.k > 0 && u.first >= 0 && u.first + u.k <= n_edges) {
            for (int32_t j = 0; j < u.k; ++j) {
                const bc_vedge& e = edges[u.first + j];
                g->h_entries.push_back({e.x, g->directed ? e.dir : 0, e.w});
            }
            g->staged_k[i] = u.k;
        }
    }
    const int64_t need = (int64_t)g->h_entries.size();
    if (need > g->d_entries_cap) {
        CK(g, cudaStreamSynchronize(g->d.st));
        dfree(g, g->d_entries);
        g->d_entries = nullptr;
        const int64_t cap = std::max<int64_t>(need, 1024);
        if ((rc = dalloc(g, &g->d_entries, cap))) return rc;
        g->d_entries_cap = cap;
    }
    if (need > 0) {
        CK(g, cudaMemcpyAsync(g->d_entries, g->h_entries.data(), sizeof(VEdge) * need,
                              cudaMemcpyHostToDevice, g->d.st));
        CK(g, cudaStreamSynchronize(g->d.st));
    }
    // keep the caller's edges for validation in bc_run_staged
    g->h_entries.shrink_to_fit();
    return BC_OK;
}

int bc_run_staged(bc_graph* g, int32_t* n_done) {
    int rc;
    if (n_done) *n_done = 0;
    if (!check_alive(g, &rc)) return rc;
    std::vector<VEdge> ent;
    std::vector<bc_vedge> tmp;
    const int32_t count = (int32_t)g->staged.size();
    int32_t done = 0;
    rc = BC_OK;
    for (int32_t i = 0; i < count; ++i) {
        const bc_update& u = g->staged[i];
        // validation reads the staged entries (already in bc_vedge form)
        tmp.clear();
        bc_update uu = u;
        if (u.kind == BC_UPD_VERTEX) {
            if (g->staged_k[i] != u.k || u.k < 1) {
                rc = fail(g, BC_ERR_ARG, "vertex update edges out of range");
                break;
            }
            for (int32_t j = 0; j < u.k; ++j) {
                const VEdge& e = g->h_entries[g->staged_first[i] + j];
                tmp.push_back({e.x, e.dir, e.w});
            }
            uu.first = 0;
        }
        int32_t v = -1;
        rc = validate_update(g, uu, tmp.data(), (int64_t)tmp.size(), &v, ent);
        if (rc) break;
        rc = enqueue_update(g, v, ent, g->d_entries + g->staged_first[i]);
        if (rc) break;
        ++done;
    }
    if (n_done) *n_done = done;
    cudaEventRecord(g->ev_done, g->d.st);
    return rc;
}

int bc_synchronize(bc_graph* g) {
    int rc;
    if (!check_alive(g, &rc)) return rc;
    return sync_check(g);
}

int bc_query(bc_graph* g, int32_t* done) {
    int rc;
    if (!done) return fail(g, BC_ERR_ARG, "done is NULL");
    *done = 0;
    if (!check_alive(g, &rc)) return rc;
    cudaError_t e = cudaEventQuery(g->ev_done);
    if (e == cudaErrorNotReady) return BC_OK;
    if (e != cudaSuccess) return cuda_fail(g, e, "cudaEventQuery");
    *done = 1;
    return sync_check(g);
}

int bc_apply_updates(bc_graph* g, int32_t count, const bc_update* ups, const bc_vedge* edges,
                     int64_t n_edges, int32_t* n_done) {
    if (n_done) *n_done = 0;
    int rc = bc_stage_updates(g, count, ups, edges, n_edges);
    if (rc) return rc;
    rc = bc_run_staged(g, n_done);
    const int rs = bc_synchronize(g);
    return rc ? rc : rs;
}

int bc_apply_edge_update(bc_graph* g, int32_t u, int32_t v, int64_t w_new) {
    bc_update up{BC_UPD_EDGE, u, v, 0, w_new, 0};
    return bc_apply_updates(g, 1, &up, nullptr, 0, nullptr);
}

int bc_apply_vertex_update(bc_graph* g, int32_t v, int32_t k, const int32_t* nbr, const int64_t* w_new,
                           const uint8_t* dir) {
    int rc;
    if (!check_alive(g, &rc)) return rc;
    if (k < 1 || !nbr || !w_new || (g->directed && !dir)) return fail(g, BC_ERR_ARG, "bad vertex update arrays");
    std::vector<bc_vedge> e(k);
    for (int32_t j = 0; j < k; ++j) e[j] = {nbr[j], dir ? (int32_t)dir[j] : 0, w_new[j]};
    bc_update up{BC_UPD_VERTEX, -1, v, k, 0, 0};
    return bc_apply_updates(g, 1, &up, e.data(), k, nullptr);
}

// ---- real (fp64) weights
//
// A finite double w > 0 is exactly M * 2^e with M an odd integer below 2^53.  With E the
// smallest such e over the weights, every weight is the integer (w / 2^E) units of 2^E,
// exactly, and so is every path length: path lengths are compared, and ties decided, on
// the exact sums of the given doubles.  The state runs on these integers; BC does not
// depend on the unit.  The weights must span few enough binary orders of magnitude that
// n - 1 of the largest one fit the distance type.
static bool split_double(double w, int32_t* e_low, int32_t* e_top) {
    if (!(w > 0.0) || !std::isfinite(w)) return false;
    int x = 0;
    const double f = std::frexp(w, &x);                 // w = f * 2^x, f in [0.5, 1)
    uint64_t mant = (uint64_t)std::ldexp(f, 53);        // exact: w = mant * 2^(x - 53)
    int tz = 0;
    while (!(mant & 1ull)) { mant >>= 1; ++tz; }
    *e_low = x - 53 + tz;                               // w = odd * 2^e_low
    *e_top = x;                                         // w < 2^e_top
    return true;
}

static int bits_for(int64_t n) {
    int b = 0;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

// w as an integer number of units 2^e (exact), or -1 when it is not a multiple of the
// unit or not below 2^top units.
static int64_t to_units(double w, int32_t e, int32_t top) {
    int32_t lo = 0, hi = 0;
    if (!split_double(w, &lo, &hi) || lo < e || hi - e > top) return -1;
    return (int64_t)std::ldexp(w, -e);
}

int bc_init_static_f64(bc_graph** out, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                       const double* w, uint32_t flags, void* cuda_stream) {
    if (!out) return fail(nullptr, BC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || m < 0 || (m > 0 && (!src || !dst || !w))) return fail(nullptr, BC_ERR_ARG, "bad edge arrays");
    const bool i32 = (flags & BC_DIST_I32) != 0;
    int32_t e_min = INT32_MAX, top = INT32_MIN;
    for (int64_t i = 0; i < m; ++i) {
        int32_t lo = 0, hi = 0;
        if (!split_double(w[i], &lo, &hi)) return fail(nullptr, BC_ERR_ARG, "a weight is not a finite positive double");
        e_min = std::min(e_min, lo);
        top = std::max(top, hi);
    }
    if (m == 0) e_min = top = 0;
    // the largest weight is below 2^(top - e_min) units; n - 1 of them must stay below
    // INF of the distance type (2^31 - 1 or 2^63 - 1)
    const int32_t span = top - e_min;
    if (span + bits_for(n) > (i32 ? 30 : 62))
        return fail(nullptr, BC_ERR_ARG, "weights span too many binary orders of magnitude for exact sums");
    std::vector<int64_t> wi((size_t)m);
    for (int64_t i = 0; i < m; ++i) wi[i] = (int64_t)std::ldexp(w[i], -e_min);
    const int rc = bc_init_static(out, n, m, src, dst, wi.data(), flags, cuda_stream);
    if (rc) return rc;
    (*out)->real_weights = true;
    (*out)->w_exp = e_min;
    (*out)->top_bits = (i32 ? 30 : 62) - bits_for(n);
    return BC_OK;
}

int bc_apply_edge_update_f64(bc_graph* g, int32_t u, int32_t v, double w_new) {
    int rc;
    if (!check_alive(g, &rc)) return rc;
    if (!g->real_weights) return fail(g, BC_ERR_ARG, "the handle was not made by bc_init_static_f64");
    const int64_t x = to_units(w_new, g->w_exp, g->top_bits);
    if (x < 1) return fail(g, BC_ERR_ARG, "weight not representable exactly in the handle's unit");
    return bc_apply_edge_update(g, u, v, x);
}

int bc_apply_vertex_update_f64(bc_graph* g, int32_t v, int32_t k, const int32_t* nbr, const double* w_new,
                               const uint8_t* dir) {
    int rc;
    if (!check_alive(g, &rc)) return rc;
    if (!g->real_weights) return fail(g, BC_ERR_ARG, "the handle was not made by bc_init_static_f64");
    if (k < 1 || !w_new) return fail(g, BC_ERR_ARG, "bad vertex update arrays");
    std::vector<int64_t> xi(k);
    for (int32_t j = 0; j < k; ++j) {
        xi[j] = to_units(w_new[j], g->w_exp, g->top_bits);
        if (xi[j] < 1) return fail(g, BC_ERR_ARG, "weight not representable exactly in the handle's unit");
    }
    return bc_apply_vertex_update(g, v, k, nbr, xi.data(), dir);
}

int bc_get_weight_unit(bc_graph* g, int32_t* exp2) {
    int rc;
    if (!check_alive(g, &rc)) return rc;
    if (!exp2) return fail(g, BC_ERR_ARG, "exp2 is NULL");
    *exp2 = g->real_weights ? g->w_exp : 0;
    return BC_OK;
}

int bc_get_scores(bc_graph* g, double* out) {
    int rc;
    if (!check_alive(g, &rc)) return rc;
    if (!out) return fail(g, BC_ERR_ARG, "out is NULL");
    if ((rc = sync_check(g))) return rc;
    std::vector<double> hi(g->n), lo(g->n);
    CK(g, cudaMemcpy(hi.data(), g->d.bc_hi, sizeof(double) * g->n, cudaMemcpyDeviceToHost));
    CK(g, cudaMemcpy(lo.data(), g->d.bc_lo, sizeof(double) * g->n, cudaMemcpyDeviceToHost));
    const double f = g->directed ? 1.0 : 0.5;
    for (int32_t t = 0; t < g->n; ++t) out[t] = (hi[t] + lo[t]) * f;
    return BC_OK;
}

int bc_get_rows(bc_graph* g, int32_t s0, int32_t count, int64_t* d_out, uint64_t* sigma_out,
                double* delta_out) {
    int rc;
    if (!check_alive(g, &rc)) return rc;
    if (s0 < 0 || count < 0 || s0 + count > g->n) return fail(g, BC_ERR_ARG, "rows out of range");
    if ((rc = sync_check(g))) return rc;
    const size_t n = (size_t)g->n, off = (size_t)s0 * n, cnt = (size_t)count * n;
    if (d_out) {
        if (g->dbytes == 8) {
            CK(g, cudaMemcpy(d_out, (int64_t*)g->d.D + off, cnt * 8, cudaMemcpyDeviceToHost));
        } else {
            std::vector<int32_t> tmp(cnt);
            CK(g, cudaMemcpy(tmp.data(), (int32_t*)g->d.D + off, cnt * 4, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < cnt; ++i) d_out[i] = tmp[i] == INT32_MAX ? INT64_MAX : (int64_t)tmp[i];
        }
    }
    if (sigma_out) CK(g, cudaMemcpy(sigma_out, g->d.S + off, cnt * 8, cudaMemcpyDeviceToHost));
    if (delta_out) {
        std::vector<ff> tmp(cnt);
        CK(g, cudaMemcpy(tmp.data(), g->d.Dl + off, cnt * sizeof(ff), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < cnt; ++i) delta_out[i] = ff_to_double(tmp[i]);
    }
    return BC_OK;
}

int bc_get_edges(bc_graph* g, int64_t* m, int32_t* src, int32_t* dst, int64_t* w) {
    if (!g || !m) return BC_ERR_ARG;
    std::vector<std::pair<uint64_t, int64_t>> e;
    e.reserve(g->wmap.size());
    for (const auto& kv : g->wmap) {
        const int32_t a = (int32_t)(kv.first >> 32), b = (int32_t)(kv.first & 0xffffffffu);
        if (!g->directed && a > b) continue;
        e.push_back(kv);
    }
    std::sort(e.begin(), e.end());
    if (!src && !dst && !w) {
        *m = (int64_t)e.size();
        return BC_OK;
    }
    if (*m < (int64_t)e.size() || !src || !dst || !w) return fail(g, BC_ERR_ARG, "edge arrays too small");
    for (size_t i = 0; i < e.size(); ++i) {
        src[i] = (int32_t)(e[i].first >> 32);
        dst[i] = (int32_t)(e[i].first & 0xffffffffu);
        w[i] = e[i].second;
    }
    *m = (int64_t)e.size();
    return BC_OK;
}

int bc_get_info(bc_graph* g, bc_info* out) {
    if (!g || !out) return BC_ERR_ARG;
    CK(g, cudaStreamSynchronize(g->d.st));
    CK(g, cudaMemcpy(g->h_stats, g->d.stats, kStats * sizeof(int64_t), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->n = g->n;
    out->directed = g->directed ? 1 : 0;
    out->dist_bytes = g->dbytes;
    out->m = (int64_t)g->wmap.size();
    out->estar_arcs = g->estar_arcs;
    out->rows_reaccumulated = g->h_stats[0];
    out->noop_updates = g->h_stats[1];
    out->max_rows = g->h_stats[2];
    out->updates_applied = g->h_stats[3];
    out->pairs_lowered = g->h_stats[4];
    out->pairs_tied = g->h_stats[5];
    out->rows_scanned = g->h_stats[6];
    out->rows_full = g->h_stats[7];
    out->pair_rows = g->h_stats[8];
    out->pair_targets = g->h_stats[9];
    out->walk_pairs = g->h_stats[10];
    out->walk_vertices = g->h_stats[11];
    out->walk_arcs = g->h_stats[12];
    out->estar_rebuilds = g->estar_rebuilds;
    out->estar_moves = g->estar_moves;
    out->kernel_launches = g->launches;
    out->state_bytes = g->bytes;
    out->last_init_ms = g->last_init_ms;
    return BC_OK;
}

int bc_set_option(bc_graph* g, const char* name, int64_t value) {
    if (!g || !name) return BC_ERR_ARG;
    if (std::strcmp(name, "full_scan") == 0) {
        g->full_scan = value != 0;
        return BC_OK;
    }
    if (std::strcmp(name, "wide_accum") == 0) {
        // 1024-thread accumulation CTAs for the rows over the target cap (graphs of at
        // least 4096 vertices); 0: 256-thread ones, which share SMs better with the work of
        // other handles running at the same time (the server turns them off)
        g->d.acc_narrow_only = value != 0 ? 0 : 1;
        g->d.acc_threads = (value != 0 && g->n >= kAccWideMinN) ? kAccThreadsWide : kAccThreadsNarrow;
        return BC_OK;
    }
    if (std::strcmp(name, "fused_edges") == 0) {
        g->fused_edges = value != 0;
        return BC_OK;
    }
    if (std::strcmp(name, "profile") == 0) {
        g->profile = value != 0;
        return BC_OK;
    }
    if (std::strcmp(name, "pair_walk") == 0) {
        if (value != 0 && g->directed) return fail(g, BC_ERR_ARG, "pair_walk needs an undirected graph");
        if (value != 0) {
            const int rc = walk_alloc(g);
            if (rc) return rc;
        }
        g->d.pair_walk = value != 0 ? 1 : 0;
        return BC_OK;
    }
    if (std::strcmp(name, "walk_cap") == 0) {
        // entries of the walks' buffer to use (at most the allocated size; a test knob:
        // an update whose walks do not fit is done by the column test)
        if (!g->d.walk_list) return fail(g, BC_ERR_ARG, "walk_cap needs pair_walk on");
        if (value < 0 || value > g->walk_cap_alloc) return fail(g, BC_ERR_ARG, "walk_cap out of range");
        g->d.walk_cap = value;
        return BC_OK;
    }
    if (std::strcmp(name, "pair_updates") == 0) {
        if (value != 0 && g->directed) return fail(g, BC_ERR_ARG, "pair_updates needs an undirected graph");
        g->d.pair_on = value != 0 ? 1 : 0;
        return BC_OK;
    }
    return fail(g, BC_ERR_ARG, std::string("unknown option ") + name);
}

int bc_get_profile(bc_graph* g, double* ms, int64_t* launches, int32_t reset) {
    if (!g) return BC_ERR_ARG;
    CK(g, cudaStreamSynchronize(g->d.st));
    collect_profile(g);
    for (int c = 0; c < BC_PROFILE_CLASSES; ++c) {
        if (ms) ms[c] = g->prof_ms[c];
        if (launches) launches[c] = g->prof_launches[c];
        if (reset) {
            g->prof_ms[c] = 0.0;
            g->prof_launches[c] = 0;
        }
    }
    return BC_OK;
}

void bc_destroy(bc_graph* g) { destroy_all(g); }

const char* bc_last_error(const bc_graph* g) {
    return g ? g->last_error.c_str() : g_init_error.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------- batches

struct bc_batch {
    std::vector<bc_graph*> graphs;
    int32_t G = 0;
    int dbytes = 4;
    cudaStream_t st = nullptr;
    bool own_stream = false;   // the legacy default stream cannot be captured
    BatchLaunch L{};
    BatchArgs args{};
    int32_t n_max = 0;
    int64_t cap_max = 0;
    // device buffers (fixed while a captured graph refers to them)
    Dev* d_devs = nullptr;
    BatchUpd* d_upd = nullptr;
    VEdge* d_entries = nullptr;
    BatchEOp* d_eops = nullptr;
    int64_t* d_eop_off = nullptr;
    int64_t* d_voff = nullptr;
    int64_t* d_coff = nullptr;
    int64_t* d_plans = nullptr;
    int32_t* d_pctr = nullptr;
    int32_t* d_ws = nullptr;
    int64_t R_cap = 0, E_cap = 0, O_cap = 0, ws_cap = 0;
    cudaGraphExec_t exec = nullptr;
    int32_t exec_rounds = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double last_ms = 0.0;
    std::string last_error;
    std::vector<void*> allocs;
};

namespace {

int bfail(bc_batch* b, int code, const std::string& msg) {
    if (b) b->last_error = msg;
    return code;
}

#define CKB(b, call)                                                                           \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? BC_ERR_OOM : BC_ERR_CUDA,        \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

template <typename T>
int balloc(bc_batch* b, T** p, size_t count) {
    *p = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return bfail(b, BC_ERR_OOM, "cudaMalloc failed for a batch buffer");
    b->allocs.push_back(*p);
    return BC_OK;
}

void bfree(bc_batch* b, void* p) {
    if (!p) return;
    auto it = std::find(b->allocs.begin(), b->allocs.end(), p);
    if (it != b->allocs.end()) b->allocs.erase(it);
    cudaFree(p);
}

void drop_exec(bc_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->exec_rounds = -1;
}

// Arcs the update would add to the E* superset (not yet in it).
void new_arcs_of(bc_graph* g, int32_t v, const std::vector<VEdge>& ent, std::vector<int32_t>& need) {
    for (const VEdge& e : ent) {
        auto add = [&](int32_t a, int32_t bb) {
            if (!g->eslot.count(arc_key(a, bb))) need[a]++;
        };
        if (!g->directed) {
            add(e.x, v);
            add(v, e.x);
        } else if (e.dir == 0) {
            add(e.x, v);
        } else {
            add(v, e.x);
        }
    }
}

}  // namespace

extern "C" {

int bc_batch_create(bc_batch** out, int32_t count, bc_graph* const* graphs, void* cuda_stream) {
    if (!out || count < 1 || !graphs) return BC_ERR_ARG;
    *out = nullptr;
    bc_batch* b = new bc_batch();
    b->G = count;
    b->st = (cudaStream_t)cuda_stream;
    if (!b->st) {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return BC_ERR_CUDA;
        }
        b->own_stream = true;
    }
    b->graphs.assign(graphs, graphs + count);
    for (int32_t i = 0; i < count; ++i) {
        bc_graph* g = graphs[i];
        if (!g || g->poisoned || g->dbytes != graphs[0]->dbytes) {
            if (b->own_stream) cudaStreamDestroy(b->st);
            delete b;
            return BC_ERR_ARG;
        }
        b->n_max = std::max(b->n_max, g->n);
    }
    b->dbytes = graphs[0]->dbytes;
    b->L.nsm = graphs[0]->d.nsm;
    b->L.vpass_ctas = 4;
    b->L.scan_ctas = 8;
    b->L.bc_ctas = 8;
    b->L.acc_per_sm = 0;
    b->L.scan_unroll = 4;   // the single-graph item width (kScanUnroll)
    b->L.scan_sched = 0;
    b->L.acc_threads = kAccThreadsNarrow;
    int rc;
    if ((rc = balloc(b, &b->d_devs, count)) || (rc = balloc(b, &b->d_coff, count + 1)) ||
        (rc = balloc(b, &b->d_plans, (4 + (size_t)kPairClasses) * ((size_t)count + 1))) ||
        (rc = balloc(b, &b->d_pctr, kPairClasses))) {
        bc_batch_destroy(b);
        return rc;
    }
    cudaEventCreate(&b->e0);
    cudaEventCreate(&b->e1);
    std::vector<int64_t> coff(count + 1, 0);
    for (int32_t i = 0; i < count; ++i) coff[i + 1] = coff[i] + graphs[i]->n;
    if (cudaMemcpy(b->d_coff, coff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
        bc_batch_destroy(b);
        return BC_ERR_CUDA;
    }
    *out = b;
    return BC_OK;
}

int bc_batch_set_tiles(bc_batch* b, const int32_t* tiles, int32_t count) {
    if (!b || !tiles || count < 4) return BC_ERR_ARG;
    for (int i = 0; i < 4; ++i)
        if (tiles[i] < 0 || tiles[i] > 64) return bfail(b, BC_ERR_ARG, "tile value out of range");
    if (tiles[0] < 1 || tiles[1] < 1 || tiles[2] < 1) return bfail(b, BC_ERR_ARG, "tile value out of range");
    if (count >= 6 && ((tiles[4] != 1 && tiles[4] != 2 && tiles[4] != 4 && tiles[4] != 8) ||
                       (tiles[5] != 0 && tiles[5] != 1)))
        return bfail(b, BC_ERR_ARG, "rank-1 chunk (1, 2, 4, 8) or schedule (0, 1) out of range");
    if (count >= 7 && tiles[6] != 128 && tiles[6] != 256 && tiles[6] != 512)
        return bfail(b, BC_ERR_ARG, "accumulation CTA threads must be 128, 256 or 512");
    b->L.vpass_ctas = tiles[0];
    b->L.scan_ctas = tiles[1];
    b->L.bc_ctas = tiles[2];
    b->L.acc_per_sm = tiles[3];
    if (count >= 6) {
        b->L.scan_unroll = tiles[4];
        b->L.scan_sched = tiles[5];
    }
    if (count >= 7) b->L.acc_threads = tiles[6];
    b->cap_max = -1;   // forces a new launch configuration
    drop_exec(b);
    return BC_OK;
}

int bc_batch_apply(bc_batch* b, const int32_t* n_updates, const bc_update* ups, const bc_vedge* edges,
                   int64_t n_edges, int32_t* n_done) {
    if (!b || !n_updates || (!ups && n_edges > 0)) return BC_ERR_ARG;
    const int32_t G = b->G;
    int64_t first = 0;
    int32_t R = 0;
    for (int32_t g = 0; g < G; ++g) {
        if (n_updates[g] < 0) return bfail(b, BC_ERR_ARG, "negative update count");
        R = std::max(R, n_updates[g]);
        if (n_done) n_done[g] = 0;
    }
    for (bc_graph* g : b->graphs) {
        if (g->poisoned) return bfail(b, BC_ERR_POISONED, "a graph of the batch is poisoned");
        CKB(b, cudaStreamSynchronize(g->d.st));
    }
    int status = BC_OK;
    // ---- validate each graph's updates in order, size the slack, mirror them
    std::vector<std::vector<int32_t>> vtx(G);
    std::vector<std::vector<std::vector<VEdge>>> ents(G);
    std::vector<int32_t> ok(G, 0);
    int64_t base = 0;
    for (int32_t g = 0; g < G; ++g) {
        bc_graph* gr = b->graphs[g];
        // validation reads the host weights as they evolve: validate on a copy of the
        // weights first, then mirror for real once the slack is known to suffice
        std::unordered_map<uint64_t, int64_t> saved = gr->wmap;
        std::vector<int32_t> need(gr->n, 0);
        std::vector<VEdge> ent;
        for (int32_t k = 0; k < n_updates[g]; ++k) {
            const bc_update& u = ups[base + k];
            int32_t v = -1;
            int rc = validate_update(gr, u, edges, n_edges, &v, ent);
            if (rc) {
                if (status == BC_OK) status = rc;
                b->last_error = gr->last_error;
                break;
            }
            new_arcs_of(gr, v, ent, need);
            for (const VEdge& e : ent) {   // tentative weights so later updates validate against them
                if (!gr->directed) {
                    gr->wmap[arc_key(e.x, v)] = e.w;
                    gr->wmap[arc_key(v, e.x)] = e.w;
                } else if (e.dir == 0) {
                    gr->wmap[arc_key(e.x, v)] = e.w;
                } else {
                    gr->wmap[arc_key(v, e.x)] = e.w;
                }
            }
            vtx[g].push_back(v);
            ents[g].push_back(ent);
            ok[g]++;
        }
        gr->wmap.swap(saved);
        base += n_updates[g];
        bool short_slack = false;
        for (int32_t a = 0; a < gr->n && !short_slack; ++a)
            if (need[a] > gr->e_capv[a] - gr->e_len[a]) short_slack = true;
        if (short_slack) {
            std::vector<HArc> arcs;
            for (size_t s2 = 0; s2 < gr->e_dst.size(); ++s2)
                if (gr->e_dst[s2] >= 0) arcs.push_back({gr->e_src[s2], gr->e_dst[s2], gr->e_w[s2]});
            int rc = estar_layout(gr, arcs, &need);
            if (rc) return bfail(b, rc, gr->last_error);
        }
    }
    // ---- host records of every round
    std::vector<BatchUpd> upd((size_t)R * G);
    std::vector<VEdge> entries;
    std::vector<BatchEOp> eops;
    std::vector<int64_t> eop_off(R + 1, 0);
    std::vector<int64_t> voff((size_t)R * 4 * (G + 1), 0);
    std::vector<std::vector<EOp>> gops(G);
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t g = 0; g < G; ++g) {
            BatchUpd& u = upd[(size_t)r * G + g];
            u = BatchUpd{};
            if (r >= ok[g]) continue;
            bc_graph* gr = b->graphs[g];
            const std::vector<VEdge>& ent = ents[g][r];
            std::vector<EOp> ops;
            std::vector<EMove> moves;
            std::vector<HArc> arcs;
            bool rebuild = false;
            mirror_update(gr, vtx[g][r], ent, ops, moves, arcs, &rebuild);
            if (rebuild || !moves.empty()) return bfail(b, BC_ERR_CUDA, "internal: E* slack sized too small");
            u.v = vtx[g][r];
            u.k = (int32_t)ent.size();
            u.present = 1;
            u.first = (int64_t)entries.size();
            for (const VEdge& e : ent) {
                if (!gr->directed || e.dir == 0) u.kin++;
                if (!gr->directed || e.dir == 1) u.kout++;
                entries.push_back(e);
            }
            for (const EOp& op : ops) eops.push_back(BatchEOp{g, 0, op});
            gr->launches += 20;
        }
        eop_off[r + 1] = (int64_t)eops.size();
        for (int kind = 0; kind < 4; ++kind) {
            int64_t* o = &voff[((size_t)r * 4 + kind) * (G + 1)];
            for (int32_t g = 0; g < G; ++g) {
                const BatchUpd& u = upd[(size_t)r * G + g];
                const bool on = u.present && (kind == 0 ? u.kin > 0 : u.kout > 0);
                o[g + 1] = o[g] + (on ? b->graphs[g]->n : 0);
            }
        }
    }
    // ---- device buffers and launch shape
    // graphs with pair corrections (undirected, option on) by class of the column test's
    // columns per thread: the set of pair kernels a round launches
    int32_t pair_classes = 0;
    for (bc_graph* g : b->graphs)
        if (g->d.pair_on) pair_classes |= 1 << pair_class(g->dbytes, pair_vn(g->dbytes, g->n));
    if (pair_classes != b->L.pair_classes) {
        b->L.pair_classes = pair_classes;
        drop_exec(b);
    }
    int64_t cap_max = 0;
    for (bc_graph* g : b->graphs) cap_max = std::max(cap_max, g->d.e_cap);
    if (cap_max != b->cap_max) {
        b->cap_max = cap_max;
        batch_config(b->L, b->dbytes, b->n_max, cap_max);
        drop_exec(b);
    }
    int rc;
    const int64_t ws_need = (int64_t)b->L.acc_grid * b->L.ws_stride;
    if (ws_need > b->ws_cap) {
        bfree(b, b->d_ws);
        if ((rc = balloc(b, &b->d_ws, ws_need))) return rc;
        b->ws_cap = ws_need;
        drop_exec(b);
    }
    if (R > b->R_cap) {
        bfree(b, b->d_upd);
        bfree(b, b->d_eop_off);
        bfree(b, b->d_voff);
        const int64_t rc2 = std::max<int64_t>(R, 8);
        if ((rc = balloc(b, &b->d_upd, rc2 * G)) || (rc = balloc(b, &b->d_eop_off, rc2 + 1)) ||
            (rc = balloc(b, &b->d_voff, rc2 * 4 * (G + 1))))
            return rc;
        b->R_cap = rc2;
        drop_exec(b);
    }
    if ((int64_t)entries.size() > b->E_cap) {
        bfree(b, b->d_entries);
        const int64_t c = std::max<int64_t>((int64_t)entries.size() * 2, 1024);
        if ((rc = balloc(b, &b->d_entries, c))) return rc;
        b->E_cap = c;
        drop_exec(b);
    }
    if ((int64_t)eops.size() > b->O_cap) {
        bfree(b, b->d_eops);
        const int64_t c = std::max<int64_t>((int64_t)eops.size() * 2, 1024);
        if ((rc = balloc(b, &b->d_eops, c))) return rc;
        b->O_cap = c;
        drop_exec(b);
    }
    std::vector<Dev> devs(G);
    for (int32_t g = 0; g < G; ++g) devs[g] = b->graphs[g]->d;
    CKB(b, cudaMemcpyAsync(b->d_devs, devs.data(), sizeof(Dev) * G, cudaMemcpyHostToDevice, b->st));
    if (R > 0) {
        CKB(b, cudaMemcpyAsync(b->d_upd, upd.data(), sizeof(BatchUpd) * upd.size(), cudaMemcpyHostToDevice, b->st));
        CKB(b, cudaMemcpyAsync(b->d_eop_off, eop_off.data(), sizeof(int64_t) * eop_off.size(), cudaMemcpyHostToDevice,
                               b->st));
        CKB(b, cudaMemcpyAsync(b->d_voff, voff.data(), sizeof(int64_t) * voff.size(), cudaMemcpyHostToDevice, b->st));
    }
    if (!entries.empty())
        CKB(b, cudaMemcpyAsync(b->d_entries, entries.data(), sizeof(VEdge) * entries.size(), cudaMemcpyHostToDevice,
                               b->st));
    if (!eops.empty())
        CKB(b, cudaMemcpyAsync(b->d_eops, eops.data(), sizeof(BatchEOp) * eops.size(), cudaMemcpyHostToDevice, b->st));
    BatchArgs& a = b->args;
    a.G = G;
    a.mask_in_smem = b->L.mask_in_smem;
    a.n_max = b->n_max;
    a.devs = b->d_devs;
    a.upd = b->d_upd;
    a.entries = b->d_entries;
    a.eops = b->d_eops;
    a.eop_off = b->d_eop_off;
    a.voff = b->d_voff;
    a.coff = b->d_coff;
    a.plan_scan = b->d_plans;
    a.plan_bc = b->d_plans + (G + 1);
    a.plan_acc = b->d_plans + 2 * (G + 1);
    a.plan_pr = b->d_plans + 3 * (G + 1);
    a.plan_pw = b->d_plans + 4 * (G + 1);
    a.pctr = b->d_pctr;
    a.ws = b->d_ws;
    a.ws_stride = b->L.ws_stride;
    b->L.max_eops = std::max<int64_t>(b->L.max_eops, 256);
    if (R > 0 && (!b->exec || b->exec_rounds != R)) {
        drop_exec(b);
        cudaGraph_t graph = nullptr;
        CKB(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
        batch_launch_rounds(a, b->L, R, b->dbytes, b->st);
        CKB(b, cudaStreamEndCapture(b->st, &graph));
        cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(b, BC_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        b->exec_rounds = R;
    }
    CKB(b, cudaEventRecord(b->e0, b->st));
    if (R > 0) CKB(b, cudaGraphLaunch(b->exec, b->st));
    CKB(b, cudaEventRecord(b->e1, b->st));
    CKB(b, cudaStreamSynchronize(b->st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->e0, b->e1);
    b->last_ms = ms;
    for (int32_t g = 0; g < G; ++g) {
        bc_graph* gr = b->graphs[g];
        int rg = sync_check(gr);
        if (rg != BC_OK && status == BC_OK) {
            status = rg;
            b->last_error = gr->last_error;
        }
        if (n_done) n_done[g] = ok[g];
    }
    return status;
}

int bc_batch_last_ms(bc_batch* b, double* ms) {
    if (!b || !ms) return BC_ERR_ARG;
    *ms = b->last_ms;
    return BC_OK;
}

const char* bc_batch_last_error(const bc_batch* b) { return b ? b->last_error.c_str() : ""; }

void bc_batch_destroy(bc_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    drop_exec(b);
    for (void* p : b->allocs) cudaFree(p);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->own_stream) cudaStreamDestroy(b->st);
    delete b;
}

}  // extern "C"
