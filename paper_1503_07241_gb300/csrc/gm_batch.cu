// Batched traversal: many BFS / SSSP queries, on graphs of different sizes, in one
// device-driven superstep loop (an added form; each query follows Algorithm 2
// with the min semiring exactly as gm_run does).
//
// All queries advance in lockstep supersteps.  Superstep t is three kernels,
// captured once in a CUDA graph whose conditional WHILE node repeats them until
// every query has converged:
//   relax     a device work queue of items (query, vertex, edge chunk) over all
//             active queries' frontiers; a warp takes 32 consecutive items at a
//             time (one atomic per 32 items), concatenates their edge lists and
//             relaxes 8 edges per lane (atomicCAS for BFS, atomicMin for SSSP on
//             the query's own distance array); vertices that change go to the
//             query's next frontier (warp-aggregated per query with match_any).
//   plan      one CTA: per query, the next frontier's length; a query whose
//             frontier is empty has converged (its superstep count is t+1);
//             prefix sums of the item counts index the next work queue; the WHILE
//             condition is cleared once no query is active.
//   snapshot  SSSP messages of superstep t+1 (the distances fixed now) and
//             clearing of the "queued" bits, over the next work queue.
// A vertex with more than kBChunk out-edges is queued as one item per chunk of
// kBChunk edges, so no warp gets an unbounded edge list.
#include <algorithm>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kEPT = 8;
constexpr int kBChunk = 256;  // out-edges per work item
constexpr uint32_t kFull = 0xffffffffu;

struct BGraph {
    const int32_t* row_ptr;
    const int32_t* col;
    const uint32_t* w;  // nullptr: every weight is 1
    int64_t n;
};

struct BQuery {
    int32_t graph, sssp, source, pad;
    uint32_t* dist;   // caller's output, n of its graph
    uint32_t* msg;    // SSSP messages (n)
    uint32_t* qbits;  // "queued for the next superstep" bits (n/32 words)
    int2* q[2];       // frontier items (vertex, chunk) by superstep parity
    uint32_t cap;     // item capacity of each queue
};

struct BCtl {
    uint32_t t;
    uint32_t active;       // queries still running
    uint32_t item_next;    // work-queue head of the current superstep
    uint32_t total[2];     // items in the queues of each parity
    uint32_t guard_hit;
    uint32_t max_iters;    // 0: until convergence
    uint32_t pad;
};

struct BArgs {
    const BGraph* graphs;
    const BQuery* queries;
    int32_t nq;
    uint32_t* count;    // [nq][2] items queued per parity
    uint32_t* prefix;   // [2][nq + 1] exclusive prefix of count per parity
    uint32_t* done;     // [nq]
    int32_t* iters;     // [nq]
    BCtl* ctl;
    uint64_t guard;     // max n + 2
    cudaGraphConditionalHandle cond;
    int use_cond;
};

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return (s < a || s == kInf) ? kInf : s;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Largest q with pre[q] <= i (pre ascending, nq + 1 entries).
__device__ __forceinline__ int32_t query_of(const uint32_t* pre, int32_t nq, uint32_t i) {
    int32_t lo = 0, hi = nq - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint32_t chunks_of(const BGraph& g, int32_t v) {
    const int32_t d = g.row_ptr[v + 1] - g.row_ptr[v];
    return d <= 0 ? 1u : (uint32_t)((d + kBChunk - 1) / kBChunk);
}

__global__ void __launch_bounds__(kThreads) batch_relax(BArgs a) {
    BCtl* c = a.ctl;
    if (c->active == 0u) return;
    const uint32_t t = c->t;
    const int cur = (int)(t & 1u), nxt = cur ^ 1;
    const uint32_t total = c->total[cur];
    const uint32_t* pre = a.prefix + (size_t)cur * (a.nq + 1);
    const int lane = threadIdx.x & 31;
    __shared__ int32_t s_beg[kWarps][32];
    __shared__ uint32_t s_ex[kWarps][33];
    __shared__ uint32_t s_du[kWarps][32];
    __shared__ int32_t s_q[kWarps][32];
    int32_t* sb = s_beg[threadIdx.x >> 5];
    uint32_t* se = s_ex[threadIdx.x >> 5];
    uint32_t* sd = s_du[threadIdx.x >> 5];
    int32_t* sq = s_q[threadIdx.x >> 5];
    while (true) {
        uint32_t base = 0u;
        if (lane == 0) base = atomicAdd(&c->item_next, 32u);
        base = __shfl_sync(kFull, base, 0);
        if (base >= total) break;
        // this lane's item
        const uint32_t i = base + lane;
        int32_t qid = 0, beg = 0;
        uint32_t deg = 0u, du = 0u;
        if (i < total) {
            qid = query_of(pre, a.nq, i);
            const BQuery& Q = a.queries[qid];
            const BGraph& G = a.graphs[Q.graph];
            const int2 it = Q.q[cur][i - pre[qid]];
            const int32_t rb = G.row_ptr[it.x], re = G.row_ptr[it.x + 1];
            beg = rb + it.y * kBChunk;
            const int32_t end = min(re, beg + kBChunk);
            deg = end > beg ? (uint32_t)(end - beg) : 0u;
            du = Q.sssp ? Q.msg[it.x] : t;
        }
        const uint32_t incl = warp_incl_scan(deg);
        __syncwarp();
        sb[lane] = beg;
        se[lane] = incl - deg;
        sd[lane] = du;
        sq[lane] = qid;
        if (lane == 31) se[32] = incl;
        __syncwarp();
        const uint32_t tot = se[32];
        for (uint32_t b0 = 0; b0 < tot; b0 += 32 * kEPT) {
            const uint32_t j0 = b0 + (uint32_t)lane * kEPT;
            int o = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1)
                if (se[o + step] <= j0) o += step;
            int32_t vq[kEPT], qq[kEPT];
            uint32_t nd[kEPT];
            bool want[kEPT];
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                const uint32_t j = j0 + k;
                vq[k] = 0;
                qq[k] = -1;
                nd[k] = kInf;
                want[k] = false;
                if (j < tot) {
                    while (j >= se[o + 1]) ++o;
                    const int32_t e = sb[o] + (int32_t)(j - se[o]);
                    const BQuery& Q = a.queries[sq[o]];
                    const BGraph& G = a.graphs[Q.graph];
                    vq[k] = G.col[e];
                    qq[k] = sq[o];
                    nd[k] = Q.sssp ? sat_add(sd[o], G.w ? G.w[e] : 1u) : sd[o] + 1u;
                }
            }
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                if (qq[k] < 0) continue;
                const BQuery& Q = a.queries[qq[k]];
                uint32_t* dv = Q.dist + vq[k];
                if (nd[k] >= *dv) continue;
                if (Q.sssp) {
                    if (nd[k] < atomicMin(dv, nd[k])) {
                        const uint32_t bit = 1u << (vq[k] & 31);
                        want[k] = (atomicOr(Q.qbits + (vq[k] >> 5), bit) & bit) == 0u;
                    }
                } else {
                    want[k] = atomicCAS(dv, kInf, nd[k]) == kInf;
                }
            }
            // append to each query's next frontier, aggregated per query within the warp
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                uint32_t items = 0u;
                if (want[k]) items = chunks_of(a.graphs[a.queries[qq[k]].graph], vq[k]);
                const int key = want[k] ? qq[k] : -1 - lane;
                const uint32_t peers = __match_any_sync(kFull, key);
                if (!want[k]) continue;
                const int leader = __ffs(peers) - 1;
                // exclusive prefix of items among lower peers
                uint32_t before = 0u, sum = 0u;
                for (uint32_t m = peers; m; m &= m - 1) {
                    const int l = __ffs(m) - 1;
                    const uint32_t x = __shfl_sync(peers, items, l);
                    if (l < lane) before += x;
                    sum += x;
                }
                uint32_t pos = 0u;
                if (lane == leader) pos = atomicAdd(&a.count[qq[k] * 2 + nxt], sum);
                pos = __shfl_sync(peers, pos, leader) + before;
                const BQuery& Q = a.queries[qq[k]];
                if (pos + items <= Q.cap)
                    for (uint32_t ch = 0; ch < items; ++ch) Q.q[nxt][pos + ch] = make_int2(vq[k], (int32_t)ch);
            }
        }
    }
}

// One CTA: convergence, prefix sums of the next work queue, the loop condition.
__global__ void batch_plan(BArgs a) {
    BCtl* c = a.ctl;
    __shared__ uint32_t s_part[1024 / 32 + 1];
    __shared__ uint32_t s_active;
    if (c->active == 0u) return;
    const uint32_t t = c->t;
    const int nxt = (int)((t + 1u) & 1u);
    if (threadIdx.x == 0) s_active = 0u;
    __syncthreads();
    uint32_t* pre = a.prefix + (size_t)nxt * (a.nq + 1);
    uint32_t run = 0u;
    for (int32_t q0 = 0; q0 < a.nq; q0 += blockDim.x) {
        const int32_t q = q0 + (int32_t)threadIdx.x;
        uint32_t items = 0u;
        if (q < a.nq && !a.done[q]) {
            items = a.count[q * 2 + nxt];
            a.iters[q] = (int32_t)(t + 1u);
            bool stop = items == 0u || (c->max_iters > 0u && t + 1u >= c->max_iters);
            if (items > a.queries[q].cap) {  // cannot happen: each vertex is queued once per superstep
                c->guard_hit = 1u;
                stop = true;
            }
            if (stop) {
                a.done[q] = 1u;
                items = 0u;
            } else {
                atomicAdd(&s_active, 1u);
            }
            a.count[q * 2 + (nxt ^ 1)] = 0u;  // the consumed queue is refilled two supersteps on
        }
        // block-wide exclusive scan of items
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const uint32_t incl = warp_incl_scan(items);
        if (lane == 31) s_part[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const uint32_t nw = blockDim.x / 32;
            uint32_t v = lane < (int)nw ? s_part[lane] : 0u;
            const uint32_t vi = warp_incl_scan(v);
            if (lane < (int)nw) s_part[lane] = vi - v;
            if (lane == 31) s_part[32] = vi;
        }
        __syncthreads();
        if (q < a.nq) pre[q] = run + s_part[wid] + incl - items;
        run += s_part[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pre[a.nq] = run;
        c->total[nxt] = run;
        c->item_next = 0u;
        c->t = t + 1u;
        c->active = s_active;
        if ((uint64_t)t + 1u >= a.guard && s_active) {
            c->guard_hit = 1u;
            c->active = 0u;
        }
        if (a.use_cond) cudaGraphSetConditional(a.cond, c->active ? 1u : 0u);
    }
}

// Messages of the next superstep (SSSP) and clearing of the queued bits.
__global__ void batch_snapshot(BArgs a) {
    BCtl* c = a.ctl;
    if (c->active == 0u) return;
    const int cur = (int)(c->t & 1u);  // plan already advanced t
    const uint32_t total = c->total[cur];
    const uint32_t* pre = a.prefix + (size_t)cur * (a.nq + 1);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int32_t q = query_of(pre, a.nq, i);
        const BQuery& Q = a.queries[q];
        if (!Q.sssp) continue;
        const int2 it = Q.q[cur][i - pre[q]];
        if (it.y != 0) continue;
        Q.msg[it.x] = Q.dist[it.x];
        atomicAnd(Q.qbits + (it.x >> 5), ~(1u << (it.x & 31)));
    }
}

// Initial state: distances infinity except the source, the source queued.
__global__ void batch_seed(BArgs a) {
    const int32_t q = blockIdx.y;
    if (q >= a.nq) return;
    const BQuery& Q = a.queries[q];
    const BGraph& G = a.graphs[Q.graph];
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < G.n; v += (int64_t)gridDim.x * blockDim.x) {
        Q.dist[v] = v == Q.source ? 0u : kInf;
        if (Q.sssp && (v & 31) == 0) Q.qbits[v >> 5] = 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t nch = chunks_of(G, Q.source);
        for (uint32_t ch = 0; ch < nch; ++ch) Q.q[0][ch] = make_int2(Q.source, (int32_t)ch);
        if (Q.sssp) Q.msg[Q.source] = 0u;
        a.count[q * 2 + 0] = nch;
        a.count[q * 2 + 1] = 0u;
        a.done[q] = 0u;
        a.iters[q] = 0;
    }
}

__global__ void batch_prefix0(BArgs a) {  // single thread: prefix of the initial queues
    uint32_t run = 0u;
    for (int32_t q = 0; q < a.nq; ++q) {
        a.prefix[q] = run;
        run += a.count[q * 2];
    }
    a.prefix[a.nq] = run;
    BCtl* c = a.ctl;
    c->t = 0u;
    c->active = a.nq > 0 ? (uint32_t)a.nq : 0u;
    c->item_next = 0u;
    c->total[0] = run;
    c->total[1] = 0u;
    c->guard_hit = 0u;
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
        if (!g) { set_error("gm_run_batch: graph %d is NULL", gi); return GM_ERR_INVALID_ARG; }
        hg[gi] = BGraph{as<int32_t>(g->row_ptr), as<int32_t>(g->col),
                        g->wtype == GM_W_U32 ? as<uint32_t>(g->w) : nullptr, g->n};
        max_n = std::max(max_n, g->n);
    }
    // per-query workspace: messages, queued bits and two item queues
    std::vector<BQuery> hq((size_t)n_queries);
    std::vector<size_t> offs((size_t)n_queries);
    size_t total_bytes = 0;
    auto round = [](size_t b) { return (b + 255) & ~(size_t)255; };
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
        const int64_t n = g->n, cap = n + g->m / kBChunk + 2;
        offs[i] = total_bytes;
        total_bytes += round(sizeof(uint32_t) * n) + round(sizeof(uint32_t) * ((n + 31) / 32)) +
                       2 * round(sizeof(int2) * cap);
        hq[i] = BQuery{Q.graph, Q.kind == GM_SSSP ? 1 : 0, Q.source, 0, out_state[i], nullptr, nullptr,
                       {nullptr, nullptr}, (uint32_t)cap};
    }
    DevBuf work, dgraphs, dqueries, arrays, ctl;
    struct Scope {
        cudaStream_t s;
        DevBuf* b[5];
        ~Scope() { for (DevBuf* x : b) dev_free(*x, s); }
    } scope{s, {&work, &dgraphs, &dqueries, &arrays, &ctl}};
    GM_TRY(dev_alloc(work, total_bytes, s));
    char* base = static_cast<char*>(work.p);
    for (int32_t i = 0; i < n_queries; ++i) {
        const gm_graph* g = graphs[hq[i].graph];
        const int64_t n = g->n;
        char* p = base + offs[i];
        hq[i].msg = reinterpret_cast<uint32_t*>(p);
        p += round(sizeof(uint32_t) * n);
        hq[i].qbits = reinterpret_cast<uint32_t*>(p);
        p += round(sizeof(uint32_t) * ((n + 31) / 32));
        hq[i].q[0] = reinterpret_cast<int2*>(p);
        p += round(sizeof(int2) * hq[i].cap);
        hq[i].q[1] = reinterpret_cast<int2*>(p);
    }
    GM_TRY(dev_alloc(dgraphs, sizeof(BGraph) * (hg.size() + 1), s));
    GM_TRY(dev_alloc(dqueries, sizeof(BQuery) * hq.size(), s));
    const size_t nq = (size_t)n_queries;
    const size_t arr_bytes = sizeof(uint32_t) * (2 * nq + 2 * (nq + 1) + nq) + sizeof(int32_t) * nq;
    GM_TRY(dev_alloc(arrays, arr_bytes, s));
    GM_TRY(dev_alloc(ctl, sizeof(BCtl), s));
    GM_CUDA_TRY(cudaMemcpyAsync(dgraphs.p, hg.data(), sizeof(BGraph) * hg.size(), cudaMemcpyHostToDevice, s));
    GM_CUDA_TRY(cudaMemcpyAsync(dqueries.p, hq.data(), sizeof(BQuery) * hq.size(), cudaMemcpyHostToDevice, s));
    BCtl hc{};
    hc.max_iters = max_iters > 0 ? (uint32_t)max_iters : 0u;
    GM_CUDA_TRY(cudaMemcpyAsync(ctl.p, &hc, sizeof(BCtl), cudaMemcpyHostToDevice, s));
    BArgs a{};
    a.graphs = as<BGraph>(dgraphs);
    a.queries = as<BQuery>(dqueries);
    a.nq = n_queries;
    uint32_t* ab = as<uint32_t>(arrays);
    a.count = ab;
    a.prefix = ab + 2 * nq;
    a.done = a.prefix + 2 * (nq + 1);
    a.iters = reinterpret_cast<int32_t*>(a.done + nq);
    a.ctl = as<BCtl>(ctl);
    a.guard = (uint64_t)max_n + 2u;
    // seed every query, then build the initial work queue
    {
        dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_n + 255) / 256, 64)), (unsigned)n_queries);
        batch_seed<<<grid, 256, 0, s>>>(a);
        batch_prefix0<<<1, 1, 0, s>>>(a);
        g_launches += 2;
        GM_CUDA_TRY(cudaGetLastError());
    }
    // the superstep loop: WHILE { relax; plan; snapshot }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_relax, kThreads, 0);
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
        cudaGraphNode_t n1, n2, n3;
        kp.func = (void*)batch_relax;
        kp.gridDim = dim3((unsigned)(per_sm * num_sms()));
        e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &kp);
        if (e == cudaSuccess) {
            kp.func = (void*)batch_plan;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(1024);
            e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &kp);
        }
        if (e == cudaSuccess) {
            kp.func = (void*)batch_snapshot;
            kp.gridDim = dim3((unsigned)(num_sms() * 2));
            kp.blockDim = dim3(kThreads);
            e = cudaGraphAddKernelNode(&n3, body, &n2, 1, &kp);
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
    std::vector<int32_t> its(nq);
    GM_CUDA_TRY(cudaMemcpyAsync(its.data(), a.iters, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaMemcpyAsync(&hc, ctl.p, sizeof(BCtl), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    g_launches += 3ull * hc.t;
    if (iters_done)
        for (size_t i = 0; i < nq; ++i) iters_done[i] = its[i];
    if (hc.guard_hit) {
        set_error("gm_run_batch: superstep loop exceeded its bound (internal error)");
        return GM_ERR_TIMEOUT;
    }
    return GM_OK;
}

}  // extern "C"
