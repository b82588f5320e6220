// gm_bfs_csr_noalloc: breadth-first search over caller-provided CSR arrays that
// allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// traversal: code whose device memory is all owned by its own caching allocator
// or a fixed arena (a cudaMalloc behind that allocator's back can fail once the
// arena has reserved the free memory, or fragments it), and latency-critical
// loops that must not pay for cudaMalloc/cudaFree, which can synchronise the
// device and fail under memory pressure.  This entry point keeps its scratch
// (two frontier queues and a few counters) in one file-scope device array of
// fixed size that every GPU holds for as long as the library is loaded.  The
// caller supplies the graph and the output buffer.
//
// The traversal gives the same result as gm_run with GM_BFS: depth 0 at the
// source, depth t+1 for every unvisited out-neighbour of a vertex reached in
// superstep t, one superstep per level plus the final one that finds nothing.
// Each superstep is one launch of a top-down (push) kernel over the current
// frontier queue, after which the host reads the next frontier's size (the
// call synchronises its stream once per superstep).
#include <mutex>

#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int64_t kNoAllocMaxVertices = 1 << 20;  // 1,048,576 vertices
constexpr int kCtl = 64;                          // control words at the start of the scratch
// Layout (uint32 words): [0, kCtl) counters, then queue A and queue B of
// kNoAllocMaxVertices entries each.  Total 8 MiB + 256 bytes.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kCtl + 2 * kNoAllocMaxVertices];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint32_t* g_scratch_ptr[kMaxDevices] = {nullptr};

__global__ void noalloc_init(uint32_t* scratch, uint32_t* depth, int64_t n, int32_t source) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        depth[v] = v == source ? 0u : kInf;
    if (blockIdx.x == 0 && threadIdx.x < kCtl) scratch[threadIdx.x] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scratch[kCtl] = (uint32_t)source;  // queue A holds the source
        scratch[0] = 1u;                   // length of queue A
    }
}

// One superstep: every frontier vertex (queue `cur`) pushes t+1 to its unvisited
// out-neighbours; the thread whose atomicCAS claims a vertex appends it to the
// other queue.  Counter words: [0] length of queue A, [1] length of queue B.
__global__ void noalloc_push(uint32_t* scratch, const int32_t* __restrict__ row_ptr,
                             const int32_t* __restrict__ col, uint32_t* depth, uint32_t t, int cur) {
    uint32_t* qcur = scratch + kCtl + (cur ? kNoAllocMaxVertices : 0);
    uint32_t* qnxt = scratch + kCtl + (cur ? 0 : kNoAllocMaxVertices);
    const uint32_t ncur = scratch[cur];
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gwarp; i < ncur; i += nwarps) {  // one warp per frontier vertex
        const int32_t u = (int32_t)qcur[i];
        const int32_t beg = row_ptr[u], end = row_ptr[u + 1];
        for (int32_t e = beg + lane; e < end; e += 32) {
            const int32_t v = col[e];
            if (depth[v] == kInf && atomicCAS(&depth[v], kInf, t + 1u) == kInf) {
                const uint32_t pos = atomicAdd(&scratch[cur ^ 1], 1u);
                qnxt[pos] = (uint32_t)v;
            }
        }
    }
}

// Device address of the scratch array on the current device (set up once per device).
gm_status scratch_for_current_device(uint32_t** out) {
    int dev = 0;
    GM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("gm_bfs_csr_noalloc: device ordinal %d not supported", dev);
        return GM_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("gm_bfs_csr_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return GM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_ptr[dev];
    return GM_OK;
}

}  // namespace

}  // namespace gm

using namespace gm;

extern "C" {

int64_t gm_bfs_csr_noalloc_max_vertices(void) { return kNoAllocMaxVertices; }

gm_status gm_bfs_csr_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col, int32_t source,
                             uint32_t* depth, int32_t* iters_done, void* stream) {
    if (n < 1 || !row_ptr || !col || !depth) {
        set_error("gm_bfs_csr_noalloc: need n >= 1 and non-NULL row_ptr, col, depth");
        return GM_ERR_INVALID_ARG;
    }
    if (n > kNoAllocMaxVertices) {
        set_error("gm_bfs_csr_noalloc: n = %lld exceeds the fixed scratch limit of %lld vertices",
                  (long long)n, (long long)kNoAllocMaxVertices);
        return GM_ERR_INVALID_ARG;
    }
    if (source < 0 || source >= n) {
        set_error("gm_bfs_csr_noalloc: source %d outside [0, %lld)", source, (long long)n);
        return GM_ERR_INVALID_ARG;
    }
    uint32_t* scratch = nullptr;
    GM_TRY(scratch_for_current_device(&scratch));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = num_sms() * 4;
    noalloc_init<<<blocks, 256, 0, s>>>(scratch, depth, n, source);
    g_launches++;
    GM_CUDA_TRY(cudaGetLastError());
    uint32_t count = 1;
    int32_t t = 0;
    int cur = 0;
    while (true) {  // a level-synchronous loop converges within n supersteps
        GM_CUDA_TRY(cudaMemsetAsync(scratch + (cur ^ 1), 0, sizeof(uint32_t), s));
        noalloc_push<<<blocks, 256, 0, s>>>(scratch, row_ptr, col, depth, (uint32_t)t, cur);
        g_launches++;
        GM_CUDA_TRY(cudaGetLastError());
        GM_CUDA_TRY(cudaMemcpyAsync(&count, scratch + (cur ^ 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        GM_CUDA_TRY(cudaStreamSynchronize(s));
        ++t;
        cur ^= 1;
        if (count == 0 || t > n) break;
    }
    if (iters_done) *iters_done = t;
    return GM_OK;
}

}  // extern "C"
