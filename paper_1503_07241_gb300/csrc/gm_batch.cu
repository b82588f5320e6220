// Batched traversal: many BFS / SSSP queries, on graphs of different sizes, in one
// device-driven superstep loop (an added form; each query follows Algorithm 2
// with the min semiring exactly as gm_run does).
//
// Queries of the same program on the same graph are bundled, up to 8 per bundle,
// and a bundle's queries advance in lockstep supersteps as one multi-source
// SpMSpV: a vertex's frontier membership for the bundle is one byte (bit q =
// in query q's frontier), and for SSSP its 8 messages are one 32-byte row
// (infinity for the queries whose frontier does not hold it).  Each superstep
// pulls over the in-edges (CSC) of every vertex once for the whole bundle:
//   BFS   new(v) = OR over in-edges u->v of front(u), minus the queries that
//         already reached v (the scan stops once every missing query is found);
//         depth_q(v) = t+1 for each new query q.
//   SSSP  acc_q(v) = min over in-edges of sat(msg_q(u) + w(u, v)), one 32-byte
//         gather per in-edge whose source is in any frontier; dist_q(v) =
//         min(dist_q(v), acc_q(v)); the changed queries form front(v) and
//         msg_q(v) of the next superstep.
// The work of a superstep is one queue of warp items over all bundles of all
// graphs: groups of 32 vertices of in-degree < bin_small (a lane each), single
// vertices of larger in-degree (a warp each, lanes over the in-edges, warp
// reductions), and groups of 32 vertices without in-edges (their next front
// byte is cleared).  A one-CTA plan kernel retires the queries whose next
// frontier is empty (recording their superstep counts) and stops the loop when
// no query runs.  Both kernels are captured in one CUDA graph whose conditional
// WHILE node repeats them.
#include <algorithm>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr int kSlots = 8;  // queries per bundle
constexpr uint32_t kFull = 0xffffffffu;

struct BGraph {
    const int32_t* col_ptr;
    const int32_t* row;
    const uint32_t* cw;   // uint32 in-edge weights, or nullptr
    const uint8_t* cw8;   // one-byte copy when every weight fits, or nullptr
    const int32_t* in_list;
    int64_t in_off[4];    // bins 1..3 of in_list at [in_off[b-1], in_off[b])
    const int32_t* zero_in;
    int64_t zero_count;
    int64_t n;
};

struct Bundle {
    int32_t graph, sssp, nq, pad;
    uint32_t* out[kSlots];   // the callers' depth / distance arrays (nullptr past nq)
    int32_t qid[kSlots];     // index of each slot's query in the call
    int32_t source[kSlots];
    uint8_t* front[2];       // per vertex, by superstep parity: bit q = in query q's frontier
    uint8_t* vis;            // BFS: bit q = reached by query q
    uint32_t* msg[2];        // SSSP: n rows of 8 messages, by superstep parity
    uint32_t item0;          // first work item of the bundle
    uint32_t n_small, n_big, n_zero;  // work items of each kind
    uint32_t active;         // queries still running (bits)
    uint32_t next_active;    // queries with a vertex in the next frontier (this superstep)
};

struct BCtl {
    uint32_t t;
    uint32_t any_active;
    uint32_t guard_hit;
    uint32_t max_iters;  // 0: until convergence
};

struct BArgs {
    const BGraph* graphs;
    Bundle* bundles;
    int32_t nb;
    uint32_t total_items;
    int32_t* iters;  // per query of the call
    BCtl* ctl;
    uint64_t guard;  // max n + 2
    cudaGraphConditionalHandle cond;
    int use_cond;
};

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return s < b ? kInf : s;
}

__device__ __forceinline__ uint32_t edge_weight(const BGraph& G, int32_t e) {
    return G.cw8 ? (uint32_t)G.cw8[e] : (G.cw ? G.cw[e] : 1u);
}

// The 8 messages of source u (two 16-byte loads).
__device__ __forceinline__ void load_msgs(const uint32_t* __restrict__ msg, int32_t u, uint32_t (&m)[kSlots]) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(msg + (int64_t)u * kSlots));
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(msg + (int64_t)u * kSlots + 4));
    m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w;
    m[4] = b.x; m[5] = b.y; m[6] = b.z; m[7] = b.w;
}

// Apply of SSSP at v: returns the changed queries; writes the next messages row.
__device__ __forceinline__ uint32_t sssp_apply(const Bundle& B, int32_t v, const uint32_t (&acc)[kSlots],
                                               uint32_t* __restrict__ msg_next) {
    uint32_t mask = 0u, nm[kSlots];
#pragma unroll
    for (int q = 0; q < kSlots; ++q) {
        nm[q] = kInf;
        if (q < B.nq && acc[q] != kInf && acc[q] < B.out[q][v]) {
            B.out[q][v] = acc[q];
            nm[q] = acc[q];
            mask |= 1u << q;
        }
    }
    uint4* row = reinterpret_cast<uint4*>(msg_next + (int64_t)v * kSlots);
    row[0] = make_uint4(nm[0], nm[1], nm[2], nm[3]);
    row[1] = make_uint4(nm[4], nm[5], nm[6], nm[7]);
    return mask;
}

// Apply of BFS at v: `found` = queries with an in-neighbour in their frontier.
__device__ __forceinline__ uint32_t bfs_apply(const Bundle& B, int32_t v, uint32_t vis_v, uint32_t found,
                                              uint32_t t) {
    const uint32_t nw = found & ~vis_v;
    if (nw) {
        B.vis[v] = (uint8_t)(vis_v | nw);
#pragma unroll
        for (int q = 0; q < kSlots; ++q)
            if ((nw >> q) & 1u) B.out[q][v] = t + 1u;
    }
    return nw;
}

__device__ __forceinline__ int32_t bundle_of(const Bundle* bs, int32_t nb, uint32_t item) {
    int32_t lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (bs[mid].item0 <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads) batch_pull(BArgs a) {
    const BCtl* c = a.ctl;
    if (c->any_active == 0u) return;
    const uint32_t t = c->t;
    const int cur = (int)(t & 1u), nxt = cur ^ 1;
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
    for (uint32_t item = gwarp; item < a.total_items; item += nwarps) {
        const int32_t bi = bundle_of(a.bundles, a.nb, item);
        Bundle& B = a.bundles[bi];
        if (B.active == 0u) continue;  // warp-uniform
        const BGraph& G = a.graphs[B.graph];
        const uint8_t* __restrict__ fc = B.front[cur];
        uint8_t* __restrict__ fn = B.front[nxt];
        uint32_t k = item - B.item0;
        uint32_t mask = 0u;
        if (k < B.n_small) {  // 32 vertices of small in-degree, a lane each
            const int64_t i = G.in_off[0] + (int64_t)k * 32 + lane;
            if (i < G.in_off[1]) {
                const int32_t v = G.in_list[i];
                const int32_t beg = G.col_ptr[v], end = G.col_ptr[v + 1];
                if (B.sssp) {
                    uint32_t acc[kSlots];
#pragma unroll
                    for (int q = 0; q < kSlots; ++q) acc[q] = kInf;
                    for (int32_t e = beg; e < end; ++e) {
                        const int32_t u = G.row[e];
                        if (!fc[u]) continue;
                        uint32_t m[kSlots];
                        load_msgs(B.msg[cur], u, m);
                        const uint32_t w = edge_weight(G, e);
#pragma unroll
                        for (int q = 0; q < kSlots; ++q) acc[q] = min(acc[q], sat_add(m[q], w));
                    }
                    mask = sssp_apply(B, v, acc, B.msg[nxt]);
                } else {
                    const uint32_t vis_v = B.vis[v];
                    const uint32_t need = B.active & ~vis_v;  // running queries that have not reached v
                    uint32_t found = 0u;
                    for (int32_t e = beg; e < end && (found & need) != need; ++e) found |= fc[G.row[e]];
                    mask = need ? bfs_apply(B, v, vis_v, found, t) : 0u;
                }
                fn[v] = (uint8_t)mask;
            }
        } else if ((k -= B.n_small) < B.n_big) {  // one vertex of larger in-degree, a warp
            const int32_t v = G.in_list[G.in_off[1] + k];
            const int32_t beg = G.col_ptr[v], end = G.col_ptr[v + 1];
            if (B.sssp) {
                uint32_t acc[kSlots];
#pragma unroll
                for (int q = 0; q < kSlots; ++q) acc[q] = kInf;
                for (int32_t e = beg + lane; e < end; e += 32) {
                    const int32_t u = G.row[e];
                    if (!fc[u]) continue;
                    uint32_t m[kSlots];
                    load_msgs(B.msg[cur], u, m);
                    const uint32_t w = edge_weight(G, e);
#pragma unroll
                    for (int q = 0; q < kSlots; ++q) acc[q] = min(acc[q], sat_add(m[q], w));
                }
#pragma unroll
                for (int q = 0; q < kSlots; ++q) acc[q] = __reduce_min_sync(kFull, acc[q]);
                if (lane == 0) {
                    mask = sssp_apply(B, v, acc, B.msg[nxt]);
                    fn[v] = (uint8_t)mask;
                }
            } else {
                const uint32_t vis_v = B.vis[v];
                const uint32_t need = B.active & ~vis_v;
                uint32_t found = 0u;
                for (int32_t e0 = beg; e0 < end && need; e0 += 32) {
                    if (e0 + lane < end) found |= fc[G.row[e0 + lane]];
                    found = __reduce_or_sync(kFull, found);
                    if ((found & need) == need) break;  // warp-uniform
                }
                if (lane == 0) {
                    mask = need ? bfs_apply(B, v, vis_v, found, t) : 0u;
                    fn[v] = (uint8_t)mask;
                }
            }
        } else {  // 32 vertices without in-edges: nothing reaches them
            k -= B.n_big;
            const int64_t i = (int64_t)k * 32 + lane;
            if (i < G.zero_count) fn[G.zero_in[i]] = 0u;
        }
        mask = __reduce_or_sync(kFull, mask);
        if (lane == 0 && mask) atomicOr(&B.next_active, mask);
    }
}

// One CTA: retire the queries whose next frontier is empty, stop at max_iters,
// advance the superstep and set the loop condition.
__global__ void batch_plan(BArgs a) {
    BCtl* c = a.ctl;
    __shared__ uint32_t s_any;
    if (c->any_active == 0u) return;
    const uint32_t t = c->t;
    if (threadIdx.x == 0) s_any = 0u;
    __syncthreads();
    const bool stop = (c->max_iters != 0u && t + 1u >= c->max_iters) || (uint64_t)t + 1u >= a.guard;
    for (int32_t b = threadIdx.x; b < a.nb; b += blockDim.x) {
        Bundle& B = a.bundles[b];
        if (B.active == 0u) continue;
        const uint32_t still = stop ? 0u : (B.active & B.next_active);
        const uint32_t ended = B.active & ~still;
        for (int q = 0; q < kSlots; ++q)
            if ((ended >> q) & 1u) a.iters[B.qid[q]] = (int32_t)(t + 1u);
        if (still == 0u && (B.active & B.next_active) != 0u && (uint64_t)t + 1u >= a.guard) c->guard_hit = 1u;
        B.active = still;
        B.next_active = 0u;
        if (still) atomicOr(&s_any, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        c->t = t + 1u;
        c->any_active = s_any;
        if (a.use_cond) cudaGraphSetConditional(a.cond, s_any ? 1u : 0u);
    }
}

// Every bundle's arrays at the start: fronts and reached bits clear, messages
// and outputs infinity (bundles strided over y, vertices over x).
__global__ void batch_clear(BArgs a) {
    for (int32_t b = blockIdx.y; b < a.nb; b += gridDim.y) {
    const Bundle& B = a.bundles[b];
    const int64_t n = a.graphs[B.graph].n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        B.front[0][v] = 0u;
        B.front[1][v] = 0u;
        if (!B.sssp) B.vis[v] = 0u;
        for (int q = 0; q < B.nq; ++q) B.out[q][v] = kInf;
        if (B.sssp)
            for (int s = 0; s < 2; ++s) {
                uint4* row = reinterpret_cast<uint4*>(B.msg[s] + v * kSlots);
                row[0] = make_uint4(kInf, kInf, kInf, kInf);
                row[1] = make_uint4(kInf, kInf, kInf, kInf);
            }
    }
    }
}

// The sources (one thread per bundle, after batch_clear).
__global__ void batch_seed(BArgs a) {
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < a.nb; b += gridDim.x * blockDim.x) {
        const Bundle& B = a.bundles[b];
        for (int q = 0; q < B.nq; ++q) {
            const int32_t s = B.source[q];
            B.out[q][s] = 0u;
            B.front[0][s] |= (uint8_t)(1u << q);
            if (B.sssp) B.msg[0][(int64_t)s * kSlots + q] = 0u;
            else B.vis[s] |= (uint8_t)(1u << q);
        }
    }
}

}  // namespace

}  // namespace gm

using namespace gm;

extern "C" {

gm_status gm_run_batch(gm_graph* const* graphs, int32_t n_graphs, const gm_query* queries, int32_t n_queries,
                       uint32_t* const* out_state, int32_t max_iters, int32_t* iters_done, void* stream) {
    if (n_queries < 0 || n_graphs < 0 || (n_queries > 0 && (!graphs || !queries || !out_state))) {
        set_error("gm_run_batch: NULL argument or negative count");
        return GM_ERR_INVALID_ARG;
    }
    if (max_iters < -1) { set_error("gm_run_batch: max_iters must be >= -1"); return GM_ERR_INVALID_ARG; }
    if (n_queries == 0) return GM_OK;
    for (int32_t gi = 0; gi < n_graphs; ++gi)
        if (!graphs[gi]) { set_error("gm_run_batch: graph %d is NULL", gi); return GM_ERR_INVALID_ARG; }
    for (int32_t i = 0; i < n_queries; ++i) {
        const gm_query& Q = queries[i];
        if (Q.graph < 0 || Q.graph >= n_graphs || (Q.kind != GM_BFS && Q.kind != GM_SSSP) || !out_state[i]) {
            set_error("gm_run_batch: query %d has a bad graph index, kind or output", i);
            return GM_ERR_INVALID_ARG;
        }
        const gm_graph* g = graphs[Q.graph];
        if (Q.source < 0 || Q.source >= g->n) {
            set_error("gm_run_batch: query %d source %d outside [0, %lld)", i, Q.source, (long long)g->n);
            return GM_ERR_INVALID_ARG;
        }
        if (Q.kind == GM_SSSP && g->wtype == GM_W_F32) {
            set_error("gm_run_batch: query %d: SSSP needs uint32 weights", i);
            return GM_ERR_INVALID_ARG;
        }
    }
    if (max_iters == 0) {
        for (int32_t i = 0; i < n_queries; ++i)
            if (iters_done) iters_done[i] = 0;
        return GM_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<BGraph> hg((size_t)n_graphs);
    int64_t max_n = 0;
    for (int32_t gi = 0; gi < n_graphs; ++gi) {
        const gm_graph* g = graphs[gi];
        BGraph& G = hg[gi];
        G.col_ptr = as<int32_t>(g->col_ptr);
        G.row = as<int32_t>(g->row);
        G.cw = g->wtype == GM_W_U32 ? as<uint32_t>(g->cw) : nullptr;
        G.cw8 = g->wtype == GM_W_U32 ? as<uint8_t>(g->cw8) : nullptr;
        G.in_list = as<int32_t>(g->in_list);
        for (int b = 0; b < 4; ++b) G.in_off[b] = g->in_list_count[b];
        G.zero_in = as<int32_t>(g->zero_in_list);
        G.zero_count = g->zero_in_count;
        G.n = g->n;
        max_n = std::max(max_n, g->n);
    }
    // bundles: queries of one program on one graph, up to kSlots each, in call order
    std::vector<Bundle> hb;
    {
        std::vector<int32_t> open((size_t)n_graphs * 2, -1);
        for (int32_t i = 0; i < n_queries; ++i) {
            const gm_query& Q = queries[i];
            const int key = Q.graph * 2 + (Q.kind == GM_SSSP ? 1 : 0);
            if (open[key] < 0 || hb[open[key]].nq == kSlots) {
                Bundle b{};
                b.graph = Q.graph;
                b.sssp = Q.kind == GM_SSSP ? 1 : 0;
                open[key] = (int32_t)hb.size();
                hb.push_back(b);
            }
            Bundle& b = hb[open[key]];
            b.out[b.nq] = out_state[i];
            b.qid[b.nq] = i;
            b.source[b.nq] = Q.source;
            b.nq++;
        }
    }
    // work items and workspace of every bundle
    auto round = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t ws = 0;
    uint64_t items = 0;
    std::vector<size_t> offs(hb.size());
    for (size_t b = 0; b < hb.size(); ++b) {
        Bundle& B = hb[b];
        const BGraph& G = hg[B.graph];
        const int64_t n = G.n > 0 ? G.n : 1;
        B.item0 = (uint32_t)items;
        B.n_small = (uint32_t)((G.in_off[1] - G.in_off[0] + 31) / 32);
        B.n_big = (uint32_t)(G.in_off[3] - G.in_off[1]);
        B.n_zero = (uint32_t)((G.zero_count + 31) / 32);
        items += (uint64_t)B.n_small + B.n_big + B.n_zero;
        B.active = (1u << B.nq) - 1u;
        offs[b] = ws;
        ws += 2 * round((size_t)n) + (B.sssp ? 2 * round(sizeof(uint32_t) * kSlots * (size_t)n) : round((size_t)n));
    }
    if (items >= (1ull << 32)) { set_error("gm_run_batch: too many work items"); return GM_ERR_INVALID_ARG; }
    DevBuf work, dgraphs, dbundles, diters, ctl;
    struct Scope {
        cudaStream_t s;
        DevBuf* b[5];
        ~Scope() { for (DevBuf* x : b) dev_free(*x, s); }
    } scope{s, {&work, &dgraphs, &dbundles, &diters, &ctl}};
    GM_TRY(dev_alloc(work, ws, s));
    for (size_t b = 0; b < hb.size(); ++b) {
        Bundle& B = hb[b];
        const int64_t n = hg[B.graph].n > 0 ? hg[B.graph].n : 1;
        char* p = static_cast<char*>(work.p) + offs[b];
        B.front[0] = reinterpret_cast<uint8_t*>(p);
        p += round((size_t)n);
        B.front[1] = reinterpret_cast<uint8_t*>(p);
        p += round((size_t)n);
        if (B.sssp) {
            B.msg[0] = reinterpret_cast<uint32_t*>(p);
            p += round(sizeof(uint32_t) * kSlots * (size_t)n);
            B.msg[1] = reinterpret_cast<uint32_t*>(p);
        } else {
            B.vis = reinterpret_cast<uint8_t*>(p);
        }
    }
    GM_TRY(dev_alloc(dgraphs, sizeof(BGraph) * hg.size(), s));
    GM_TRY(dev_alloc(dbundles, sizeof(Bundle) * hb.size(), s));
    GM_TRY(dev_alloc(diters, sizeof(int32_t) * (size_t)n_queries, s));
    GM_TRY(dev_alloc(ctl, sizeof(BCtl), s));
    GM_CUDA_TRY(cudaMemcpyAsync(dgraphs.p, hg.data(), sizeof(BGraph) * hg.size(), cudaMemcpyHostToDevice, s));
    GM_CUDA_TRY(cudaMemcpyAsync(dbundles.p, hb.data(), sizeof(Bundle) * hb.size(), cudaMemcpyHostToDevice, s));
    GM_CUDA_TRY(cudaMemsetAsync(diters.p, 0, sizeof(int32_t) * (size_t)n_queries, s));
    BCtl hc{};
    hc.any_active = 1u;
    hc.max_iters = max_iters > 0 ? (uint32_t)max_iters : 0u;
    GM_CUDA_TRY(cudaMemcpyAsync(ctl.p, &hc, sizeof(BCtl), cudaMemcpyHostToDevice, s));
    BArgs a{};
    a.graphs = as<BGraph>(dgraphs);
    a.bundles = as<Bundle>(dbundles);
    a.nb = (int32_t)hb.size();
    a.total_items = (uint32_t)items;
    a.iters = as<int32_t>(diters);
    a.ctl = as<BCtl>(ctl);
    a.guard = (uint64_t)max_n + 2u;
    {
        const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_n + 255) / 256, 256)),
                        (unsigned)std::min<size_t>(hb.size(), 65535));
        batch_clear<<<grid, 256, 0, s>>>(a);
        batch_seed<<<1, 128, 0, s>>>(a);
        g_launches += 2;
        GM_CUDA_TRY(cudaGetLastError());
    }
    // the superstep loop: WHILE { pull over every bundle; plan }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_pull, kThreads, 0);
    if (per_sm <= 0) per_sm = 1;
    cudaGraph_t graph;
    GM_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t cnode;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        a.cond = handle;
        a.use_cond = 1;
        void* kargs[] = {&a};
        cudaKernelNodeParams kp = {};
        kp.blockDim = dim3(kThreads);
        kp.kernelParams = kargs;
        cudaGraphNode_t n1, n2;
        kp.func = (void*)batch_pull;
        kp.gridDim = dim3((unsigned)(per_sm * num_sms()));
        e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &kp);
        if (e == cudaSuccess) {
            kp.func = (void*)batch_plan;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(1024);
            e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &kp);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
    }
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        set_error("gm_run_batch: superstep loop graph: %s", cudaGetErrorString(e));
        return GM_ERR_CUDA;
    }
    std::vector<int32_t> its((size_t)n_queries);
    GM_CUDA_TRY(cudaMemcpyAsync(its.data(), diters.p, sizeof(int32_t) * (size_t)n_queries, cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaMemcpyAsync(&hc, ctl.p, sizeof(BCtl), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    g_launches += 2ull * hc.t;
    if (iters_done)
        for (int32_t i = 0; i < n_queries; ++i) iters_done[i] = its[(size_t)i];
    if (hc.guard_hit) {
        set_error("gm_run_batch: superstep loop exceeded its bound (internal error)");
        return GM_ERR_TIMEOUT;
    }
    return GM_OK;
}

}  // extern "C"
