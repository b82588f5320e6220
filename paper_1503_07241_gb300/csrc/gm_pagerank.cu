// PageRank supersteps (Eq. 1) as a pull SpMV over the CSC form with Apply fused:
//   x_{t+1}(v) = r + (1 - r) * sum_{u -> v} c_t(u),   c_t(u) = x_t(u) / deg(u).
// Every vertex is active in every superstep, so the sparse vector is dense and
// the pull form needs no frontier test and no atomics: each destination is
// reduced by exactly one thread group (a lane for in-degree < bin_small -- that bin
// is stored ordered by degree, so a warp's 32 destinations have about the same
// length -- a warp up to bin_large, a CTA beyond), four in-edges in flight per
// thread, in a fixed order, in FP32.  The Apply step writes both the new rank and
// the next contribution c_{t+1}(v).
#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kFull = 0xffffffffu;

struct PrArgs {
    const int32_t* col_ptr; const int32_t* row; const int32_t* out_deg;
    const int32_t* in_list; int64_t in_off[4];
    const int32_t* zero_in; int64_t zero_count;
    const float* x_cur; float* x_nxt;
    const float* c_cur; float* c_nxt;
    float r; int apply_all;
};

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ void pr_apply(const PrArgs& a, int32_t v, float sum) {
    const float x = a.r + (1.0f - a.r) * sum;
    a.x_nxt[v] = x;
    const int32_t d = a.out_deg[v];
    a.c_nxt[v] = d > 0 ? x / (float)d : 0.0f;
}

__global__ void __launch_bounds__(kThreads) pr_step(PrArgs a) {
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const uint32_t gwarp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
    __shared__ float s_red[kThreads / 32];

    // large in-degree: one CTA per vertex
    for (int64_t i = a.in_off[2] + blockIdx.x; i < a.in_off[3]; i += gridDim.x) {
        const int32_t v = a.in_list[i];
        const int32_t beg = a.col_ptr[v], end = a.col_ptr[v + 1];
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        int32_t e = beg + threadIdx.x;
        for (; e + 3 * kThreads < end; e += 4 * kThreads) {
            s0 += a.c_cur[a.row[e]];
            s1 += a.c_cur[a.row[e + kThreads]];
            s2 += a.c_cur[a.row[e + 2 * kThreads]];
            s3 += a.c_cur[a.row[e + 3 * kThreads]];
        }
        for (; e < end; e += kThreads) s0 += a.c_cur[a.row[e]];
        float s = warp_sum_f((s0 + s1) + (s2 + s3));
        if (lane == 0) s_red[wid] = s;
        __syncthreads();
        if (wid == 0) {
            float t = lane < kThreads / 32 ? s_red[lane] : 0.0f;
            t = warp_sum_f(t);
            if (lane == 0) pr_apply(a, v, t);
        }
        __syncthreads();
    }
    // medium: one warp per vertex
    for (int64_t i = a.in_off[1] + gwarp; i < a.in_off[2]; i += nwarps) {
        const int32_t v = a.in_list[i];
        const int32_t beg = a.col_ptr[v], end = a.col_ptr[v + 1];
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        int32_t e = beg + lane;
        for (; e + 96 < end; e += 128) {
            s0 += a.c_cur[a.row[e]];
            s1 += a.c_cur[a.row[e + 32]];
            s2 += a.c_cur[a.row[e + 64]];
            s3 += a.c_cur[a.row[e + 96]];
        }
        for (; e < end; e += 32) s0 += a.c_cur[a.row[e]];
        const float s = warp_sum_f((s0 + s1) + (s2 + s3));
        if (lane == 0) pr_apply(a, v, s);
    }
    // small: one lane per vertex, four in-edges in flight
    for (int64_t i = a.in_off[0] + (int64_t)gwarp * 32 + lane; i - lane < a.in_off[1]; i += (int64_t)nwarps * 32) {
        if (i >= a.in_off[1]) continue;
        const int32_t v = a.in_list[i];
        const int32_t beg = a.col_ptr[v], end = a.col_ptr[v + 1];
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        int32_t e = beg;
        for (; e + 3 < end; e += 4) {
            s0 += a.c_cur[a.row[e]];
            s1 += a.c_cur[a.row[e + 1]];
            s2 += a.c_cur[a.row[e + 2]];
            s3 += a.c_cur[a.row[e + 3]];
        }
        for (; e < end; ++e) s0 += a.c_cur[a.row[e]];
        pr_apply(a, v, (s0 + s1) + (s2 + s3));
    }
    // vertices without in-edges receive no message
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < a.zero_count;
         i += (int64_t)gridDim.x * kThreads) {
        const int32_t v = a.zero_in[i];
        if (a.apply_all) {
            pr_apply(a, v, 0.0f);
        } else {
            const float x = a.x_cur[v];
            a.x_nxt[v] = x;
            a.c_nxt[v] = a.c_cur[v];
        }
    }
}

__global__ void pr_init_contrib(const float* __restrict__ x, const int32_t* __restrict__ out_deg, int64_t n,
                                float* __restrict__ c) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = out_deg[v];
        c[v] = d > 0 ? x[v] / (float)d : 0.0f;
    }
}

__global__ void fill_f32(float* p, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

int pr_grid() {
    static int blocks = 0;
    if (blocks == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pr_step, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
        blocks = per_sm * num_sms();
    }
    return blocks;
}

PrArgs make_pr_args(gm_graph* g, int parity) {
    const int64_t n = g->n > 0 ? g->n : 1;
    float* X[2] = {as<float>(g->state), as<float>(g->work)};
    float* C[2] = {as<float>(g->work) + n, as<float>(g->work) + 2 * n};
    PrArgs a{};
    a.col_ptr = as<int32_t>(g->col_ptr);
    a.row = as<int32_t>(g->row);
    a.out_deg = as<int32_t>(g->out_deg);
    a.in_list = as<int32_t>(g->in_list);
    for (int b = 0; b < 4; ++b) a.in_off[b] = g->in_list_count[b];
    a.zero_in = as<int32_t>(g->zero_in_list);
    a.zero_count = g->zero_in_count;
    a.x_cur = X[parity];
    a.x_nxt = X[parity ^ 1];
    a.c_cur = C[parity];
    a.c_nxt = C[parity ^ 1];
    a.r = (float)g->params.r;
    a.apply_all = g->params.pr_apply_all;
    return a;
}

}  // namespace

gm_status pr_prepare(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n > 0 ? g->n : 1;
    GM_TRY(dev_alloc(g->state, sizeof(float) * n, s));
    GM_TRY(dev_alloc(g->work, sizeof(float) * 3 * n, s));
    g->work_bytes = (int64_t)(sizeof(float) * 3 * n);
    fill_f32<<<num_sms() * 4, 256, 0, s>>>(as<float>(g->state), g->n, 1.0f);
    g_launches++;
    GM_CUDA_TRY(cudaGetLastError());
    return GM_OK;
}

// `iters` supersteps, built as one CUDA graph of kernel nodes (no host round trips).
gm_status pr_run(gm_graph* g, int32_t iters, int32_t* iters_done) {
    cudaStream_t s = g->stream;
    g->stats = RunStats{};
    if (iters < 0) {
        set_error("gm_run: PageRank runs a fixed number of supersteps; max_iters must be >= 0");
        return GM_ERR_INVALID_ARG;
    }
    if (iters_done) *iters_done = iters;
    g->stats.supersteps = iters;
    if (iters == 0 || g->n == 0) return GM_OK;
    const int64_t n = g->n;
    pr_init_contrib<<<num_sms() * 4, 256, 0, s>>>(as<float>(g->state), as<int32_t>(g->out_deg), n,
                                                  as<float>(g->work) + n);
    g_launches++;
    GM_CUDA_TRY(cudaGetLastError());
    const int grid = pr_grid();
    if (g->tune.profile || g->tune.loop_mode == 1) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (g->tune.profile) {
            GM_CUDA_TRY(cudaEventCreate(&e0));
            GM_CUDA_TRY(cudaEventCreate(&e1));
        }
        for (int32_t it = 0; it < iters; ++it) {
            PrArgs a = make_pr_args(g, it & 1);
            if (e0) cudaEventRecord(e0, s);
            pr_step<<<grid, kThreads, 0, s>>>(a);
            if (e1) cudaEventRecord(e1, s);
            g_launches++;
            GM_CUDA_TRY(cudaGetLastError());
            if (e0) {
                GM_CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                g->stats.relax_ms += ms;
                g->stats.relax_launches++;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    } else {
        cudaGraph_t graph;
        GM_CUDA_TRY(cudaGraphCreate(&graph, 0));
        cudaGraphNode_t prev = nullptr;
        cudaError_t e = cudaSuccess;
        PrArgs args[2] = {make_pr_args(g, 0), make_pr_args(g, 1)};
        for (int32_t it = 0; it < iters && e == cudaSuccess; ++it) {
            void* kargs[] = {&args[it & 1]};
            cudaKernelNodeParams kp = {};
            kp.func = (void*)pr_step;
            kp.gridDim = dim3((unsigned)grid);
            kp.blockDim = dim3(kThreads);
            kp.kernelParams = kargs;
            cudaGraphNode_t node;
            e = cudaGraphAddKernelNode(&node, graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
            prev = node;
        }
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            set_error("PageRank graph: %s", cudaGetErrorString(e));
            return GM_ERR_CUDA;
        }
        g_launches += (uint64_t)iters;
    }
    if (iters & 1) GM_CUDA_TRY(cudaMemcpyAsync(g->state.p, g->work.p, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // namespace gm
