// Triangle counting (Section 3.IV; the two vertex programs of Section 4.2).
//
// The input is a directed acyclic graph: the symmetrised edge list oriented from
// lower to higher (degree, id) at ingest (GM_ORIENT_BY_DEGREE).  The paper's
// first program gives every vertex a sorted list of its neighbours; the second
// sends lists along the edges and intersects them at the receiver.  Here both
// lists of an edge u -> v are the out-lists of the oriented CSR (sorted by id at
// ingest): every w in out(u) and out(v) closes the triangle {u, v, w}, which the
// DAG holds exactly once.  With degree orientation every out-list has at most
// sqrt(2m) entries, so each intersection is short.  All three corners are
// credited, giving triangles incident to each vertex (uint64) and the total.
//
// One warp per edge: for the shorter list, lanes take 32 elements at a time and
// binary-search them in the longer list (L1/L2-resident for hubs); very short
// pairs are merged by one thread.
#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ bool contains(const int32_t* __restrict__ a, int32_t n, int32_t x) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && __ldg(a + lo) == x;
}

__global__ void __launch_bounds__(kThreads) tc_edges(const int32_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col,
                                                     const int32_t* __restrict__ esrc, int64_t m,
                                                     unsigned long long* __restrict__ count,
                                                     unsigned long long* __restrict__ total) {
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    unsigned long long mine = 0;
    for (int64_t e = gwarp; e < m; e += nwarps) {
        const int32_t u = esrc[e], v = col[e];
        const int32_t* A = col + row_ptr[u];
        const int32_t* B = col + row_ptr[v];
        int32_t na = row_ptr[u + 1] - row_ptr[u];
        int32_t nb = row_ptr[v + 1] - row_ptr[v];
        if (na > nb) {
            const int32_t* T = A; A = B; B = T;
            const int32_t tn = na; na = nb; nb = tn;
        }
        uint32_t c = 0;
        for (int32_t i0 = 0; i0 < na; i0 += 32) {
            const int32_t i = i0 + lane;
            bool hit = false;
            if (i < na) {
                const int32_t x = __ldg(A + i);
                hit = contains(B, nb, x);
                if (hit) atomicAdd(&count[x], 1ull);
            }
            c += (uint32_t)__popc(__ballot_sync(kFull, hit));
        }
        if (lane == 0 && c) {
            atomicAdd(&count[u], (unsigned long long)c);
            atomicAdd(&count[v], (unsigned long long)c);
            mine += c;
        }
    }
    if (lane == 0 && mine) atomicAdd(total, mine);
}

}  // namespace

gm_status tc_run(gm_graph* g, int32_t* iters_done) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n > 0 ? g->n : 1;
    GM_CUDA_TRY(cudaMemsetAsync(g->state.p, 0, sizeof(unsigned long long) * n, s));
    DevBuf esrc, tot;
    GM_TRY(dev_alloc(esrc, sizeof(int32_t) * (g->m > 0 ? g->m : 1), s));
    gm_status st = dev_alloc(tot, sizeof(unsigned long long), s);
    if (st == GM_OK) st = expand_rows(as<int32_t>(g->row_ptr), g->n, as<int32_t>(esrc), s);
    unsigned long long h = 0;
    if (st == GM_OK) {
        cudaMemsetAsync(tot.p, 0, sizeof(unsigned long long), s);
        if (g->m > 0) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_edges, kThreads, 0);
            if (per_sm <= 0) per_sm = 1;
            tc_edges<<<per_sm * num_sms(), kThreads, 0, s>>>(as<int32_t>(g->row_ptr), as<int32_t>(g->col),
                                                             as<int32_t>(esrc), g->m,
                                                             as<unsigned long long>(g->state),
                                                             as<unsigned long long>(tot));
            g_launches++;
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tot.p, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_error("triangle count: %s", cudaGetErrorString(e)); st = GM_ERR_CUDA; }
    }
    dev_free(esrc, s);
    dev_free(tot, s);
    if (st != GM_OK) return st;
    g->tc_total = h;
    g->stats = RunStats{};
    g->stats.supersteps = 2;
    if (iters_done) *iters_done = 2;  // the two vertex programs of Section 4.2, one superstep each
    return GM_OK;
}

}  // namespace gm
