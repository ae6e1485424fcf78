// bc_server.cu -- serving many device-resident graphs with continuous batching.
//
// Built on the public C ABI.  Each admitted graph has its own handle and CUDA stream.
// Requests (incremental updates) queue per graph in arrival order; whenever a graph has
// no work on the device, every request queued for it is staged and launched at once
// (one bc_stage_updates + bc_run_staged), so requests that arrive while the graph is busy
// join its next launch, and the launches of different graphs overlap on the device.
// Admission: a graph's device state is about n^2 * (distance + 16) bytes; a graph is
// built on the device (bc_init_static) only when the server's budget and the device's
// free memory leave room for it.  When a graph with queued requests is waiting for room,
// idle resident graphs are evicted least-recently-used first; an evicted graph keeps its
// current edge list on the host and is rebuilt from it when it is needed again.  A
// request's latency runs from its submission to the poll that sees its launch finished.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "bcgpu.h"

namespace {

using clk = std::chrono::steady_clock;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(clk::now().time_since_epoch()).count();
}

struct Req {
    int64_t id;
    int64_t t_submit;
    bc_update up;
    std::vector<bc_vedge> edges;
};

struct GraphRec {
    int32_t n = 0;
    uint32_t flags = 0;
    std::vector<int32_t> src, dst;   // current edges (kept while evicted)
    std::vector<int64_t> w;
    bc_graph* h = nullptr;
    cudaStream_t st = nullptr;
    int64_t bytes = 0;
    std::deque<Req> queue;
    std::vector<Req> inflight;
    int64_t last_use = 0;
    int status = BC_OK;
};

}  // namespace

struct bc_server {
    int64_t budget = 0;
    int64_t used = 0;
    int32_t max_batch = 64;
    std::vector<GraphRec> graphs;
    std::vector<bc_result> done;
    int64_t next_id = 1;
    int64_t tick = 0;
    int64_t admissions = 0, evictions = 0, launches = 0;
    std::string last_error;
};

namespace {

int64_t state_bytes(int32_t n, uint32_t flags) {
    const int64_t sd = (flags & BC_DIST_I64) ? 8 : 4;
    // D, sigma, delta; undirected graphs also keep the old values of changed pairs and
    // the change map (one bit per pair) for pair corrections
    const bool und = (flags & BC_UNDIRECTED) != 0;
    const int64_t per_pair = (sd + 16) + (und ? sd + 8 : 0);
    return (int64_t)n * n * per_pair + (und ? (int64_t)n * n / 8 : 0) + (int64_t)n * 256 + (64 << 20);
}

int evict(bc_server* s, int32_t gid) {
    GraphRec& r = s->graphs[gid];
    if (!r.h) return BC_OK;
    int64_t m = 0;
    int rc = bc_get_edges(r.h, &m, nullptr, nullptr, nullptr);
    if (rc) return rc;
    r.src.resize(m);
    r.dst.resize(m);
    r.w.resize(m);
    rc = bc_get_edges(r.h, &m, r.src.data(), r.dst.data(), r.w.data());
    if (rc) return rc;
    bc_destroy(r.h);
    r.h = nullptr;
    s->used -= r.bytes;
    s->evictions++;
    return BC_OK;
}

// Try to build graph gid on the device, evicting idle graphs if needed.
int admit(bc_server* s, int32_t gid) {
    GraphRec& r = s->graphs[gid];
    if (r.h) return BC_OK;
    r.bytes = state_bytes(r.n, r.flags);
    for (;;) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const bool fits = s->used + r.bytes <= s->budget && (int64_t)free_b >= r.bytes;
        if (fits) break;
        // least recently used idle resident graph
        int32_t victim = -1;
        for (int32_t i = 0; i < (int32_t)s->graphs.size(); ++i) {
            const GraphRec& o = s->graphs[i];
            if (i == gid || !o.h || !o.inflight.empty() || !o.queue.empty()) continue;
            if (victim < 0 || o.last_use < s->graphs[victim].last_use) victim = i;
        }
        if (victim < 0) return BC_ERR_OOM;   // wait for room
        int rc = evict(s, victim);
        if (rc) return rc;
    }
    if (!r.st && cudaStreamCreateWithFlags(&r.st, cudaStreamNonBlocking) != cudaSuccess) return BC_ERR_CUDA;
    int rc = bc_init_static(&r.h, r.n, (int64_t)r.src.size(), r.src.data(), r.dst.data(), r.w.data(), r.flags, r.st);
    if (rc) {
        r.h = nullptr;
        return rc;
    }
    // resident graphs run side by side: narrow accumulation CTAs leave room on each SM
    bc_set_option(r.h, "wide_accum", 0);
    s->used += r.bytes;
    s->admissions++;
    return BC_OK;
}

void finish(bc_server* s, GraphRec& r, int status) {
    const int64_t t = now_ns();
    for (Req& q : r.inflight) {
        bc_result res{};
        res.request_id = q.id;
        res.graph_id = (int32_t)(&r - s->graphs.data());
        res.status = status;
        res.latency_ns = t - q.t_submit;
        s->done.push_back(res);
    }
    r.inflight.clear();
}

// Launch everything queued for graph gid (it is resident and idle).
int dispatch(bc_server* s, int32_t gid) {
    GraphRec& r = s->graphs[gid];
    const size_t k = std::min<size_t>(r.queue.size(), (size_t)s->max_batch);
    std::vector<bc_update> ups(k);
    std::vector<bc_vedge> edges;
    for (size_t i = 0; i < k; ++i) {
        Req& q = r.queue.front();
        ups[i] = q.up;
        if (q.up.kind == BC_UPD_VERTEX) {
            ups[i].first = (int64_t)edges.size();
            edges.insert(edges.end(), q.edges.begin(), q.edges.end());
        }
        r.inflight.push_back(std::move(q));
        r.queue.pop_front();
    }
    int rc = bc_stage_updates(r.h, (int32_t)k, ups.data(), edges.empty() ? nullptr : edges.data(),
                              (int64_t)edges.size());
    int32_t n_done = 0;
    if (!rc) rc = bc_run_staged(r.h, &n_done);
    r.last_use = ++s->tick;
    s->launches++;
    if (rc) {
        // the first n_done requests were enqueued; request n_done was rejected (state
        // untouched); the ones after it go back to the front of the queue in order
        std::vector<Req> ok(r.inflight.begin(), r.inflight.begin() + n_done);
        if ((size_t)n_done < r.inflight.size()) {
            std::vector<Req> bad(r.inflight.begin() + n_done, r.inflight.begin() + n_done + 1);
            for (size_t i = r.inflight.size(); i > (size_t)n_done + 1; --i) r.queue.push_front(r.inflight[i - 1]);
            r.inflight = bad;
            finish(s, r, rc);
        }
        r.inflight = ok;
    }
    return BC_OK;
}

}  // namespace

extern "C" {

int bc_server_create(bc_server** out, int64_t mem_budget_bytes, int32_t max_batch) {
    if (!out || mem_budget_bytes <= 0) return BC_ERR_ARG;
    bc_server* s = new bc_server();
    s->budget = mem_budget_bytes;
    if (max_batch > 0) s->max_batch = max_batch;
    *out = s;
    return BC_OK;
}

int bc_server_add_graph(bc_server* s, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                        const int64_t* w, uint32_t flags, int32_t* graph_id) {
    if (!s || !graph_id || n < 1 || m < 0 || (m > 0 && (!src || !dst || !w))) return BC_ERR_ARG;
    GraphRec r;
    r.n = n;
    r.flags = flags;
    r.src.assign(src, src + m);
    r.dst.assign(dst, dst + m);
    r.w.assign(w, w + m);
    s->graphs.push_back(std::move(r));
    *graph_id = (int32_t)s->graphs.size() - 1;
    int rc = admit(s, *graph_id);   // resident now if there is room; otherwise on demand
    return rc == BC_ERR_OOM ? BC_OK : rc;
}

int bc_server_submit(bc_server* s, int32_t graph_id, const bc_update* up, const bc_vedge* edges,
                     int64_t* request_id) {
    if (!s || !up || graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) return BC_ERR_ARG;
    Req q;
    q.id = s->next_id++;
    q.t_submit = now_ns();
    q.up = *up;
    if (up->kind == BC_UPD_VERTEX) {
        if (up->k < 1 || !edges) return BC_ERR_ARG;
        q.edges.assign(edges + up->first, edges + up->first + up->k);
        q.up.first = 0;
    }
    if (request_id) *request_id = q.id;
    s->graphs[graph_id].queue.push_back(std::move(q));
    return BC_OK;
}

int bc_server_poll(bc_server* s, int32_t max_results, bc_result* out, int32_t* n_out) {
    if (!s) return BC_ERR_ARG;
    // completions
    for (GraphRec& r : s->graphs) {
        if (r.inflight.empty() || !r.h) continue;
        int32_t fin = 0;
        int rc = bc_query(r.h, &fin);
        if (rc != BC_OK) finish(s, r, rc);
        else if (fin) finish(s, r, BC_OK);
    }
    // dispatch: every graph with queued requests and nothing in flight
    for (int32_t gid = 0; gid < (int32_t)s->graphs.size(); ++gid) {
        GraphRec& r = s->graphs[gid];
        if (r.queue.empty() || !r.inflight.empty()) continue;
        if (!r.h) {
            int rc = admit(s, gid);
            if (rc == BC_ERR_OOM) continue;   // no room yet
            if (rc) {
                r.inflight.assign(std::make_move_iterator(r.queue.begin()), std::make_move_iterator(r.queue.end()));
                r.queue.clear();
                finish(s, r, rc);
                continue;
            }
        }
        dispatch(s, gid);
    }
    int32_t k = 0;
    if (out && max_results > 0) {
        k = (int32_t)std::min<size_t>(s->done.size(), (size_t)max_results);
        std::memcpy(out, s->done.data(), sizeof(bc_result) * k);
        s->done.erase(s->done.begin(), s->done.begin() + k);
    }
    if (n_out) *n_out = k;
    return BC_OK;
}

int bc_server_pending(bc_server* s, int64_t* queued, int64_t* inflight) {
    if (!s) return BC_ERR_ARG;
    int64_t q = 0, f = 0;
    for (const GraphRec& r : s->graphs) {
        q += (int64_t)r.queue.size();
        f += (int64_t)r.inflight.size();
    }
    if (queued) *queued = q;
    if (inflight) *inflight = f + (int64_t)s->done.size();
    return BC_OK;
}

int bc_server_graph(bc_server* s, int32_t graph_id, bc_graph** handle) {
    if (!s || !handle || graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) return BC_ERR_ARG;
    GraphRec& r = s->graphs[graph_id];
    if (!r.h) {
        int rc = admit(s, graph_id);
        if (rc) return rc;
    }
    if (!r.inflight.empty()) {
        int rc = bc_synchronize(r.h);
        finish(s, r, rc);
        if (rc) return rc;
    }
    *handle = r.h;
    return BC_OK;
}

int bc_server_stats(bc_server* s, int64_t* stats) {
    if (!s || !stats) return BC_ERR_ARG;
    int64_t resident = 0;
    for (const GraphRec& r : s->graphs) resident += r.h ? 1 : 0;
    stats[0] = resident;
    stats[1] = s->used;
    stats[2] = s->admissions;
    stats[3] = s->evictions;
    stats[4] = s->launches;
    return BC_OK;
}

void bc_server_destroy(bc_server* s) {
    if (!s) return;
    for (GraphRec& r : s->graphs) {
        if (r.h) bc_destroy(r.h);
        if (r.st) cudaStreamDestroy(r.st);
    }
    delete s;
}

}  // extern "C"
