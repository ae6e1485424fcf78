// k_noalloc.cu -- static betweenness of a small graph without any device allocation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is owned by a
// framework's caching allocator or a serving runtime that reserves HBM up front and
// forbids further allocation (cudaMalloc may synchronise the device and stall other
// streams), or code that must not allocate once it has started.  For them
// bc_static_scores_noalloc runs the same static computation as bc_init_static --
// all-pairs distances, path counts, Algorithm 1 per source, BC as column sums -- on a
// graph the caller already holds in device memory, and writes the scores to a device
// buffer the caller provides.  Its scratch (the n x n state, packed arcs, work space)
// is one file-scope __device__ array of kScratchBytes, present on every GPU that loads
// the library until the process exits; it caps the graph at kMaxN vertices and
// kMaxArcs arcs.  Every arc of the graph is used as the superset of E* (any superset
// gives the same DAGs), so no host round trip is needed.
#include <mutex>

#include "bcgpu.h"
#include "bc_internal.cuh"

namespace bcg {

namespace {

constexpr int32_t kMaxN = 512;
constexpr int64_t kMaxArcs = 32768;
constexpr int kMaxDevices = 64;

// Byte offsets into the scratch array (every piece 256-byte aligned).
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffD = 0;
constexpr size_t kOffS = kOffD + al((size_t)kMaxN * kMaxN * 8);
constexpr size_t kOffDl = kOffS + al((size_t)kMaxN * kMaxN * 8);
constexpr size_t kOffHi = kOffDl + al((size_t)kMaxN * kMaxN * sizeof(ff));
constexpr size_t kOffLo = kOffHi + al((size_t)kMaxN * 8);
constexpr size_t kOffGw = kOffLo + al((size_t)kMaxN * 8);
constexpr size_t kOffArc = kOffGw + al((size_t)kMaxArcs * 8);
constexpr size_t kOffSrc = kOffArc + al((size_t)kMaxArcs * sizeof(Arc<int64_t>));
constexpr size_t kOffLen = kOffSrc + al((size_t)kMaxArcs * 4);
constexpr size_t kOffPart = kOffLen + al((size_t)kMaxN * 4);
constexpr size_t kOffErr = kOffPart + al((size_t)((kMaxN + kRowsPerBlock - 1) / kRowsPerBlock) * kMaxN * sizeof(ff));
constexpr size_t kOffCnt = kOffErr + 256;
constexpr size_t kOffStats = kOffCnt + 256;
constexpr size_t kOffWs = kOffStats + 256;
constexpr size_t kWsBytes = (size_t)4 << 20;
constexpr size_t kScratchBytes = kOffWs + kWsBytes;

}  // namespace

// The scratch itself.  Host code must not use this name as an address: it is only a
// host-side stand-in for the symbol; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Pack the caller's CSR into the slot format of the accumulation (every arc a slot),
// and check each arc: endpoints in range, no self-loop, weight in [1, INF-1].
template <typename DT>
__global__ void k_pack_graph(int n, int64_t arcs, const int32_t* off, const int32_t* dst, const int64_t* w,
                             DT* gw, Arc<DT>* arc, int32_t* src, int32_t* len, int32_t* err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int32_t a = off[i], b = off[i + 1];
        len[i] = b - a;
        if (a < 0 || b < a || b > arcs) set_err(err, ERRF_ARG_DEVICE);
        else
            for (int32_t e = a; e < b; ++e) {
                src[e] = (int32_t)i;
                if (dst[e] == (int32_t)i) set_err(err, ERRF_ARG_DEVICE);   // self-loop
            }
    }
    if (i < arcs) {
        const int32_t b = dst[i];
        const int64_t x = w[i];
        if (b < 0 || b >= n || x < 1 || x >= Inf<DT>::v) set_err(err, ERRF_ARG_DEVICE);
        gw[i] = (DT)x;
        arc[i] = Arc<DT>{(b >= 0 && b < n) ? (DT)b : (DT)-1, (DT)x};
    }
}

__global__ void k_scores_out(int n, const double* hi, const double* lo, double f, double* out, const int32_t* err) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n || *err) return;
    out[t] = (hi[t] + lo[t]) * f;
}

}  // namespace
}  // namespace bcg

using namespace bcg;

extern "C" int bc_static_scores_noalloc(int32_t n, int64_t arcs, const int32_t* d_off, const int32_t* d_dst,
                                        const int64_t* d_w, uint32_t flags, double* d_scores, void* cuda_stream) {
    const bool dir = (flags & BC_DIRECTED) != 0, und = (flags & BC_UNDIRECTED) != 0;
    const bool i32 = (flags & BC_DIST_I32) != 0, i64 = (flags & BC_DIST_I64) != 0;
    if (dir == und || i32 == i64) return BC_ERR_ARG;
    if (n < 1 || n > kMaxN || arcs < 0 || arcs > kMaxArcs) return BC_ERR_ARG;
    if (!d_off || !d_scores || (arcs > 0 && (!d_dst || !d_w))) return BC_ERR_ARG;
    unsigned char* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return BC_ERR_CUDA;
    Dev d{};
    d.n = n;
    d.dbytes = i32 ? 4 : 8;
    d.directed = dir ? 1 : 0;
    d.st = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return BC_ERR_CUDA;
    d.D = base + kOffD;
    d.S = reinterpret_cast<uint64_t*>(base + kOffS);
    d.Dl = reinterpret_cast<ff*>(base + kOffDl);
    d.bc_hi = reinterpret_cast<double*>(base + kOffHi);
    d.bc_lo = reinterpret_cast<double*>(base + kOffLo);
    d.g_off = const_cast<int32_t*>(d_off);
    d.g_dst = const_cast<int32_t*>(d_dst);
    d.g_w = base + kOffGw;
    d.g_arcs = arcs;
    d.e_off = const_cast<int32_t*>(d_off);
    d.e_len = reinterpret_cast<int32_t*>(base + kOffLen);
    d.e_src = reinterpret_cast<int32_t*>(base + kOffSrc);
    d.e_arc = base + kOffArc;
    d.e_cap = arcs;
    d.err = reinterpret_cast<int32_t*>(base + kOffErr);
    d.counts = reinterpret_cast<int32_t*>(base + kOffCnt);
    d.stats = reinterpret_cast<int64_t*>(base + kOffStats);
    d.partial = reinterpret_cast<ff*>(base + kOffPart);
    d.nrb_max = (n + kRowsPerBlock - 1) / kRowsPerBlock;
    accum_config(d);
    if ((size_t)d.acc_grid * (size_t)d.ws_stride * sizeof(int32_t) > kWsBytes) {
        // fewer CTAs keep the work space inside its share of the scratch
        d.acc_grid = (int32_t)(kWsBytes / ((size_t)d.ws_stride * sizeof(int32_t)));
        if (d.acc_grid < 1) return BC_ERR_ARG;
    }
    d.ws = reinterpret_cast<int32_t*>(base + kOffWs);
    // the error word and counters start at zero on every call (the scratch keeps the
    // previous call's contents)
    if (cudaMemsetAsync(d.err, 0, 256 * 3, d.st) != cudaSuccess) return BC_ERR_CUDA;
    const int blocks = (int)((std::max<int64_t>(n, arcs) + 255) / 256);
    if (d.dbytes == 4)
        k_pack_graph<int32_t><<<blocks, 256, 0, d.st>>>(n, arcs, d_off, d_dst, d_w, (int32_t*)d.g_w,
                                                         (Arc<int32_t>*)d.e_arc, d.e_src, d.e_len, d.err);
    else
        k_pack_graph<int64_t><<<blocks, 256, 0, d.st>>>(n, arcs, d_off, d_dst, d_w, (int64_t*)d.g_w,
                                                         (Arc<int64_t>*)d.e_arc, d.e_src, d.e_len, d.err);
    launch_sssp(d);
    launch_accum(d, 1);
    launch_bc_rows(d, +1, 1);
    k_scores_out<<<(n + 255) / 256, 256, 0, d.st>>>(n, d.bc_hi, d.bc_lo, dir ? 1.0 : 0.5, d_scores, d.err);
    if (cudaGetLastError() != cudaSuccess) return BC_ERR_CUDA;
    int32_t h_err = 0;
    if (cudaMemcpyAsync(&h_err, d.err, sizeof(int32_t), cudaMemcpyDeviceToHost, d.st) != cudaSuccess ||
        cudaStreamSynchronize(d.st) != cudaSuccess)
        return BC_ERR_CUDA;
    if (h_err & ERRF_ARG_DEVICE) return BC_ERR_ARG;
    if (h_err & ERRF_OVERFLOW) return BC_ERR_OVERFLOW;
    if (h_err & ERRF_DIST) return BC_ERR_DIST_OVERFLOW;
    if (h_err & ERRF_TIMEOUT) return BC_ERR_TIMEOUT;
    return BC_OK;
}
