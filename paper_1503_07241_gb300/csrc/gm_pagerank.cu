// PageRank supersteps (Eq. 1) as a pull SpMV over the CSC form with Apply fused:
//   x_{t+1}(v) = r + (1 - r) * sum_{u -> v} c_t(u),   c_t(u) = x_t(u) / deg(u).
// Every vertex is active in every superstep, so the sparse vector is dense and
// the pull form needs no frontier test.  The in-edges are cut into fixed
// 256-edge warp tiles (pr_tiles), so a hub column is summed by many warps at
// once instead of one CTA walking its whole list; the pieces of a column that
// crosses tiles are combined by pr_cross.  FP32, every sum in a fixed order
// (deterministic); the Apply step writes both the new rank and the next
// contribution c_{t+1}(v).
#include <algorithm>
#include <cstring>
#include <new>

#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kFull = 0xffffffffu;

struct PrArgs {
    const int32_t* row; const int32_t* out_deg;
    const int32_t* dc_jc; const int32_t* dc_cp; const int32_t* dc_tile; const uint32_t* dc_head;
    int64_t ntiles, m;
    const int32_t* zero_in; int64_t zero_count;
    const float* x_cur; float* x_nxt;
    const float* c_cur; float* c_nxt;
    float* lead; float* trail;  // per tile: partial sums of the columns that cross tiles
    const int2* vd;             // per non-empty column: (vertex, out-degree)
    const int4* xk;             // per tile k: (t1, vertex, out-degree, -) of the crossing column starting in k, t1 = -1 if none
    float r; int apply_all;
};

__device__ __forceinline__ void pr_apply(const PrArgs& a, int32_t v, float sum) {
    const float x = a.r + (1.0f - a.r) * sum;
    a.x_nxt[v] = x;
    const int32_t d = a.out_deg[v];
    a.c_nxt[v] = d > 0 ? x / (float)d : 0.0f;
}

__device__ __forceinline__ void pr_apply_vd(const PrArgs& a, int32_t v, int32_t d, float sum) {
    const float x = a.r + (1.0f - a.r) * sum;
    a.x_nxt[v] = x;
    a.c_nxt[v] = d > 0 ? x / (float)d : 0.0f;
}

// Apply for the vertex of non-empty column col (one load for vertex and degree).
__device__ __forceinline__ void pr_apply_col(const PrArgs& a, int32_t col, float sum) {
    const int2 vd = __ldg(a.vd + col);
    pr_apply_vd(a, vd.x, vd.y, sum);
}

constexpr int kEPT = 8;  // in-edges per lane of a 256-edge warp tile (kWTile = 32 x 8)

// PageRank superstep over 256-edge warp tiles of the CSC (the doubly compressed
// CSC's tiles: dc_tile = column holding the tile's first edge, dc_head = one bit
// per in-edge marking a column's first).  Lane L takes edges 8L..8L+7 of the
// tile and sums c(u) over them in order, splitting at column starts; a
// segmented inclusive sum across the lanes (fixed shuffle order) joins the
// pieces of a column that spans lanes.  A column that begins and ends inside
// the tile is applied at once.  A column spread over tiles t0..t1 leaves a
// partial sum in each: trail[t0] (from its start to the end of t0) and lead[t]
// for t0 < t <= t1 (its part before the first column start of t, the whole
// tile for t < t1); pr_cross adds them up and applies.  No column's chain of
// dependent loads is longer than one tile's.
__global__ void __launch_bounds__(kThreads) pr_tiles(PrArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
    const uint32_t ntiles = (uint32_t)a.ntiles, m = (uint32_t)a.m;
    for (uint32_t k = gwarp; k < ntiles; k += nwarps) {
        const uint32_t e0 = k * 256u + (uint32_t)lane * kEPT;
        const uint32_t nv = e0 < m ? min((uint32_t)kEPT, m - e0) : 0u;
        int32_t src[kEPT];
        float cv[kEPT];
        if (nv == (uint32_t)kEPT) {
            const int4 lo = __ldg(reinterpret_cast<const int4*>(a.row + e0));
            const int4 hi = __ldg(reinterpret_cast<const int4*>(a.row + e0 + 4));
            src[0] = lo.x; src[1] = lo.y; src[2] = lo.z; src[3] = lo.w;
            src[4] = hi.x; src[5] = hi.y; src[6] = hi.z; src[7] = hi.w;
        } else {
#pragma unroll
            for (int q = 0; q < kEPT; ++q) src[q] = (uint32_t)q < nv ? __ldg(a.row + e0 + q) : 0;
        }
#pragma unroll
        for (int q = 0; q < kEPT; ++q) cv[q] = (uint32_t)q < nv ? __ldg(a.c_cur + src[q]) : 0.0f;
        const uint32_t hw = e0 < m ? __ldg(a.dc_head + (e0 >> 5)) : 0u;
        // the tile's last column ends in it when the next tile starts a column (or there is none)
        const bool ends_here = k + 1 >= ntiles || (__ldg(a.dc_head + (k + 1) * 8u) & 1u) != 0u;
        const uint32_t heads = (hw >> ((lane & 3) * 8)) & ((1u << nv) - 1u);
        const int32_t c0 = __ldg(a.dc_tile + k);
        // column numbering: column starts before this lane, and whether the tile starts one
        uint32_t hincl = (uint32_t)__popc(heads);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, hincl, o);
            if (lane >= o) hincl += y;
        }
        const uint32_t hex = hincl - (uint32_t)__popc(heads);
        const uint32_t bal_first = __ballot_sync(kFull, heads & 1u);
        const uint32_t bal_seen = __ballot_sync(kFull, heads != 0u);
        const uint32_t first_is_head = bal_first & 1u;
        const int32_t col_base = c0 + (int32_t)hex - (int32_t)first_is_head;
        // lane runs: F before the first start, complete runs applied, the last run open
        float F = 0.0f, run = 0.0f;
        int32_t run_col = col_base;
        const bool seen = heads != 0u;
#pragma unroll
        for (int q = 0; q < kEPT; ++q) {
            if ((heads >> q) & 1u) {
                if ((heads & ((1u << q) - 1u)) != 0u) pr_apply_col(a, run_col, run);  // inside this lane
                else F = run;
                run = 0.0f;
                run_col = col_base + (int32_t)__popc(heads & ((2u << q) - 1u));
            }
            run += cv[q];
        }
        if (!seen) F = run;
        float R = seen ? run : F;
        const uint32_t le = bal_seen & (0xFFFFFFFFu >> (31 - lane));
        const int seg0 = le ? 31 - __clz(le) : -1;  // -1: the segment began before the tile
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float Ru = __shfl_up_sync(kFull, R, o);
            if (lane - o >= max(seg0, 0)) R += Ru;
        }
        float Rprev = __shfl_up_sync(kFull, R, 1);
        if (lane == 0) Rprev = 0.0f;
        const bool fprev = lane > 0 && (bal_seen & ((1u << lane) - 1u)) != 0u;
        // the leading segment belongs to column c0, begun in an earlier tile
        float lead = 0.0f;
        bool lead_end = false;
        if (seen && !(heads & 1u)) {  // this lane's first edges finish a column begun to its left
            if (fprev) pr_apply_col(a, col_base, F + Rprev);
            else { lead = F + Rprev; lead_end = true; }
        }
        const bool next_head = lane < 31 && ((bal_first >> (lane + 1)) & 1u);
        if (lane == 31 || next_head) {
            const int32_t end_col = c0 + (int32_t)hincl - (int32_t)first_is_head;
            if (seg0 < 0) {
                lead = R;  // the leading segment ends here
                lead_end = true;
            } else if (lane < 31) {
                pr_apply_col(a, end_col, R);  // complete inside the tile
            } else if (ends_here) {  // the trailing segment: complete unless the column goes on
                pr_apply_col(a, end_col, R);
            } else {
                a.trail[k] = R;
            }
        }
        if (lead_end) a.lead[k] = lead;
    }
    // vertices without in-edges receive no message
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < a.zero_count;
         i += (int64_t)gridDim.x * kThreads) {
        const int32_t v = a.zero_in[i];
        if (a.apply_all) {
            pr_apply(a, v, 0.0f);
        } else {
            a.x_nxt[v] = a.x_cur[v];
            a.c_nxt[v] = a.c_cur[v];
        }
    }
}

constexpr int64_t kSerialTiles = 8;  // crossing columns over more tiles are summed by a whole warp

// The second half of a superstep: the columns that cross tiles, each found
// from the record xk[t0] of its first tile t0 (built once per graph).  One
// thread per tile sums trail[t0] + lead[t0+1] + ... + lead[t1] in that order
// when the column spans at most kSerialTiles tiles; longer ones (the hubs) are
// summed by the whole warp, each lane over a fixed stride of tiles, then a
// fixed shuffle tree.  Either way the order is fixed.
__global__ void __launch_bounds__(kThreads) pr_cross(PrArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t nt = a.ntiles;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t base = (int64_t)blockIdx.x * kThreads + (threadIdx.x & ~31); base < nt; base += stride) {
        const int64_t k = base + lane;
        const int4 x = k < nt ? __ldg(a.xk + k) : make_int4(-1, 0, 0, 0);
        const int64_t t1 = x.x;
        if (t1 >= 0 && t1 - k <= kSerialTiles) {
            float sum = __ldg(a.trail + k);
            for (int64_t t = k + 1; t <= t1; ++t) sum += __ldg(a.lead + t);
            pr_apply_vd(a, x.y, x.z, sum);
        }
        uint32_t big = __ballot_sync(kFull, t1 - k > kSerialTiles);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t kk = __shfl_sync(kFull, k, src);
            const int64_t tt = __shfl_sync(kFull, t1, src);
            float sum = lane == 0 ? __ldg(a.trail + kk) : 0.0f;
            for (int64_t t = kk + 1 + lane; t <= tt; t += 32) sum += __ldg(a.lead + t);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
            if (lane == src) pr_apply_vd(a, x.y, x.z, sum);
        }
    }
}

// Per-graph records for the supersteps: (vertex, out-degree) of each non-empty
// column, and for each tile k the column that starts in k and crosses into
// k + 1 (tile k + 1 starts with no column start, and that column's first edge
// lies in k), with the last tile it reaches.
__global__ void pr_records(PrArgs a, int64_t ncols, int2* vd, int4* xk) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += stride) {
        const int32_t v = a.dc_jc[c];
        vd[c] = make_int2(v, a.out_deg[v]);
    }
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.ntiles; k += stride) {
        int4 r = make_int4(-1, 0, 0, 0);
        if (k + 1 < a.ntiles && (a.dc_head[(k + 1) * 8] & 1u) == 0u) {
            const int32_t col = a.dc_tile[k + 1];
            if (((int64_t)a.dc_cp[col] >> 8) == k) {
                const int32_t v = a.dc_jc[col];
                r = make_int4((int32_t)(((int64_t)a.dc_cp[col + 1] - 1) >> 8), v, a.out_deg[v], 0);
            }
        }
        xk[k] = r;
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pr_tiles, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
        blocks = per_sm * num_sms();
    }
    return blocks;
}

int cross_grid(const gm_graph* g) {
    const int64_t blocks = (g->dc_ntiles + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms() * 8));
}

// Workspace, each part 16-byte aligned: the other rank array, two contribution
// arrays, per tile the leading and trailing partial sums, then the records
// (int2 per non-empty column, int4 per tile).
struct PrLayout {
    size_t lead, trail, vd, xk, total;
};

PrLayout pr_layout(const gm_graph* g) {
    const size_t n = (size_t)(g->n > 0 ? g->n : 1), nt = (size_t)(g->dc_ntiles > 0 ? g->dc_ntiles : 1);
    const size_t nc = (size_t)(g->dc_ncols > 0 ? g->dc_ncols : 1);
    auto up = [](size_t b) { return (b + 15) & ~(size_t)15; };
    PrLayout L;
    L.lead = up(sizeof(float) * 3 * n);
    L.trail = up(L.lead + sizeof(float) * nt);
    L.vd = up(L.trail + sizeof(float) * nt);
    L.xk = up(L.vd + sizeof(int2) * nc);
    L.total = L.xk + sizeof(int4) * nt;
    return L;
}

PrArgs make_pr_args(gm_graph* g, int parity) {
    const int64_t n = g->n > 0 ? g->n : 1;
    float* work = as<float>(g->work);
    char* wb = static_cast<char*>(g->work.p);
    const PrLayout L = pr_layout(g);
    float* X[2] = {as<float>(g->state), work};
    float* C[2] = {work + n, work + 2 * n};
    PrArgs a{};
    a.row = as<int32_t>(g->row);
    a.out_deg = as<int32_t>(g->out_deg);
    a.dc_jc = as<int32_t>(g->dc_jc);
    a.dc_cp = as<int32_t>(g->dc_cp);
    a.dc_tile = as<int32_t>(g->dc_tile);
    a.dc_head = as<uint32_t>(g->dc_head);
    a.ntiles = g->dc_ntiles;
    a.m = g->m;
    a.zero_in = as<int32_t>(g->zero_in_list);
    a.zero_count = g->zero_in_count;
    a.x_cur = X[parity];
    a.x_nxt = X[parity ^ 1];
    a.c_cur = C[parity];
    a.c_nxt = C[parity ^ 1];
    a.lead = reinterpret_cast<float*>(wb + L.lead);
    a.trail = reinterpret_cast<float*>(wb + L.trail);
    a.vd = reinterpret_cast<const int2*>(wb + L.vd);
    a.xk = reinterpret_cast<const int4*>(wb + L.xk);
    a.r = (float)g->params.r;
    a.apply_all = g->params.pr_apply_all;
    return a;
}

// The superstep graph of a run: `iters` pairs of nodes (pr_tiles, pr_cross), the arguments
// alternating between the two parities.  Kept on the handle and reused while
// the superstep count and the arguments (buffers, r, the apply rule) are
// unchanged.
struct PrGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t iters = 0;
    PrArgs args[2];
};

gm_status pr_graph_for(gm_graph* g, int32_t iters, int grid, int cgrid) {
    PrArgs args[2] = {make_pr_args(g, 0), make_pr_args(g, 1)};
    PrGraph* pg = static_cast<PrGraph*>(g->pr);
    if (pg && pg->exec && pg->iters == iters && std::memcmp(pg->args, args, sizeof(args)) == 0) return GM_OK;
    pr_release(g);
    pg = new (std::nothrow) PrGraph();
    if (!pg) { set_error("PageRank graph: host allocation failed"); return GM_ERR_OUT_OF_MEMORY; }
    std::memcpy(pg->args, args, sizeof(args));
    pg->iters = iters;
    cudaError_t e = cudaGraphCreate(&pg->graph, 0);
    cudaGraphNode_t prev = nullptr;
    for (int32_t it = 0; it < 2 * iters && e == cudaSuccess; ++it) {
        void* kargs[] = {&pg->args[(it >> 1) & 1]};
        cudaKernelNodeParams kp = {};
        kp.func = (it & 1) ? (void*)pr_cross : (void*)pr_tiles;
        kp.gridDim = dim3((unsigned)((it & 1) ? cgrid : grid));
        kp.blockDim = dim3(kThreads);
        kp.kernelParams = kargs;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, pg->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
        prev = node;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pg->exec, pg->graph, 0);
    g->pr = pg;
    if (e != cudaSuccess) {
        pr_release(g);
        set_error("PageRank graph: %s", cudaGetErrorString(e));
        return GM_ERR_CUDA;
    }
    return GM_OK;
}

}  // namespace

void pr_release(gm_graph* g) {
    PrGraph* pg = static_cast<PrGraph*>(g->pr);
    if (!pg) return;
    if (pg->exec) cudaGraphExecDestroy(pg->exec);
    if (pg->graph) cudaGraphDestroy(pg->graph);
    delete pg;
    g->pr = nullptr;
}

gm_status pr_reset(gm_graph* g) {
    fill_f32<<<num_sms() * 4, 256, 0, g->stream>>>(as<float>(g->state), g->n, 1.0f);
    g_launches++;
    GM_CUDA_TRY(cudaGetLastError());
    GM_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return GM_OK;
}

gm_status pr_prepare(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n > 0 ? g->n : 1;
    GM_TRY(dev_alloc(g->state, sizeof(float) * n, s));
    const PrLayout L = pr_layout(g);
    GM_TRY(dev_alloc(g->work, L.total, s));
    g->work_bytes = (int64_t)L.total;
    if (g->dc_ntiles > 0) {
        char* wb = static_cast<char*>(g->work.p);
        pr_records<<<num_sms() * 4, 256, 0, s>>>(make_pr_args(g, 0), g->dc_ncols, reinterpret_cast<int2*>(wb + L.vd),
                                                 reinterpret_cast<int4*>(wb + L.xk));
        g_launches++;
        GM_CUDA_TRY(cudaGetLastError());
    }
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
    const int grid = pr_grid(), cgrid = cross_grid(g);
    if (g->tune.profile || g->tune.loop_mode == 1) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (g->tune.profile) {
            GM_CUDA_TRY(cudaEventCreate(&e0));
            GM_CUDA_TRY(cudaEventCreate(&e1));
        }
        for (int32_t it = 0; it < iters; ++it) {
            PrArgs a = make_pr_args(g, it & 1);
            if (e0) cudaEventRecord(e0, s);
            pr_tiles<<<grid, kThreads, 0, s>>>(a);
            pr_cross<<<cgrid, kThreads, 0, s>>>(a);
            if (e1) cudaEventRecord(e1, s);
            g_launches += 2;
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
        GM_TRY(pr_graph_for(g, iters, grid, cgrid));
        GM_CUDA_TRY(cudaGraphLaunch(static_cast<PrGraph*>(g->pr)->exec, s));
        g_launches += 2ull * (uint64_t)iters;
    }
    if (iters & 1) GM_CUDA_TRY(cudaMemcpyAsync(g->state.p, g->work.p, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // namespace gm
