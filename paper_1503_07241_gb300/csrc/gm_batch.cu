// Batched traversal: many BFS / SSSP queries, on graphs of different sizes, in one
// device-driven superstep loop (an added form; each query follows Algorithm 2
// with the min semiring exactly as gm_run does).
//
// Queries of the same program on the same graph are bundled, up to 8 per bundle,
// and a bundle's queries advance in lockstep supersteps as one multi-source
// SpMSpV: a vertex's frontier membership for the bundle is one byte (bit q =
// in query q's frontier), and for SSSP its 8 messages are one 32-byte row
// (infinity for the queries whose frontier does not hold it).  Each superstep a
// bundle either pushes or pulls, chosen on the device from the out-edges of its
// frontier (the graph handle's switch point, so gm_autotune tunes it):
//   push  over the out-edges (CSR) of its frontier, kept as a list of pieces
//         (vertex, 256 out-edges); BFS: the queries of front(u) that have not
//         reached v reach it (an atomic OR on the reached byte decides which);
//         SSSP: atomicMin of sat(msg_q(u) + w) into dist_q(v) for q in front(u);
//         a vertex joins the next frontier for the queries that changed it.
//   pull  over the in-edges (CSC) of every vertex:
//         BFS   new(v) = OR over in-edges u->v of front(u), minus the queries that
//               already reached v (the scan stops once every missing query is found);
//         SSSP  acc_q(v) = min over in-edges of sat(msg_q(u) + w(u, v)), one 32-byte
//               gather per in-edge whose source is in any frontier.
// Both directions write the next frontier's bytes and count its out-edges; a
// push also lists it.  The work of a superstep is one queue of warp items over
// all bundles of all graphs (pull: groups of 32 vertices of small in-degree a
// lane each, single vertices of larger in-degree a warp each, groups of 32
// vertices without in-edges; push: one piece a warp).  A finish kernel then
// picks each bundle's next direction and prepares it: after a push it clears
// the frontier just consumed and, for SSSP, writes the next frontier's message
// rows from the values at the end of the superstep (as BSP requires); after a
// pull that a push follows it lists the next frontier from its bytes.  A
// one-CTA plan kernel retires the queries whose next frontier is empty
// (recording their superstep counts), lays out the next work queue and stops the
// loop when no query runs.  The pull and push kernels (side by side), finish
// and plan are the body of a CUDA graph's WHILE node.
#include <algorithm>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr int kSlots = 8;          // queries per bundle
constexpr int32_t kPiece = 256;    // out-edges per push work item (8 per lane)
constexpr int kPlanThreads = 1024;
constexpr uint32_t kFull = 0xffffffffu;

struct BGraph {
    const int32_t* col_ptr;
    const int32_t* row;
    const uint32_t* cw;   // uint32 in-edge weights, or nullptr
    const uint8_t* cw8;   // one-byte copy when every weight fits, or nullptr
    const int32_t* row_ptr;
    const int32_t* col;
    const uint32_t* w;    // uint32 out-edge weights, or nullptr (unit weights)
    const int32_t* out_deg;
    const int32_t* in_list;
    int64_t in_off[4];    // bins 1..3 of in_list at [in_off[b-1], in_off[b])
    const int32_t* zero_in;
    int64_t zero_count;
    int64_t n;
    unsigned long long pull_above_sssp;  // an SSSP bundle pulls when its frontier has more out-edges
    unsigned long long pull_above_bfs;   // the same for BFS
    int32_t dir_mode;     // 0 auto, 1 push only, 2 pull only (the handle's option)
};

struct Bundle {
    int32_t graph, sssp, nq, pad;
    uint32_t* out[kSlots];   // the callers' depth / distance arrays (nullptr past nq)
    int32_t qid[kSlots];     // index of each slot's query in the call
    int32_t source[kSlots];
    uint8_t* front[2];       // per vertex, by superstep parity: bit q = in query q's frontier
    uint8_t* vis;            // BFS: bit q = reached by query q
    uint32_t* msg[2];        // SSSP: n rows of 8 messages, by superstep parity
    int2* piece[2];          // frontier by parity: (vertex, piece) per 256 out-edges, (v, 0) if none
    uint32_t npiece[2];
    uint32_t item0[2];       // offset of this superstep's work items in the [0] push / [1] pull queue
    uint32_t n_items;        // this superstep's work items (in its direction's queue)
    uint32_t n_small, n_big, n_zero;  // pull work items of each kind
    uint32_t dir;            // this superstep: 0 push, 1 pull
    uint32_t next_dir;       // the next superstep's, decided when this one's frontier is known
    uint32_t active;         // queries still running (bits)
    uint32_t next_active;    // queries with a vertex in the next frontier (this superstep)
    unsigned long long next_medges;  // out-edges of the next frontier
};

struct BCtl {
    uint32_t t;
    uint32_t any_active;
    uint32_t guard_hit;
    uint32_t max_iters;    // 0: until convergence
    uint32_t total[2];     // work items of this superstep over all bundles: [0] push, [1] pull
};

struct BArgs {
    const BGraph* graphs;
    Bundle* bundles;
    int32_t nb;
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

__device__ __forceinline__ uint32_t in_weight(const BGraph& G, int32_t e) {
    return G.cw8 ? (uint32_t)G.cw8[e] : (G.cw ? G.cw[e] : 1u);
}

__device__ __forceinline__ uint32_t pieces_of(int32_t d) { return d > 0 ? (uint32_t)((d + kPiece - 1) / kPiece) : 1u; }

// The 8 messages of source u (two 16-byte loads).
__device__ __forceinline__ void load_msgs(const uint32_t* __restrict__ msg, int32_t u, uint32_t (&m)[kSlots]) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(msg + (int64_t)u * kSlots));
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(msg + (int64_t)u * kSlots + 4));
    m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w;
    m[4] = b.x; m[5] = b.y; m[6] = b.z; m[7] = b.w;
}

// Apply of SSSP at v after a pull: returns the changed queries; writes the next messages row.
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

// Apply of BFS at v after a pull: `found` = queries with an in-neighbour in their frontier.
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

// Atomic OR of `bits` into byte v of a byte array (through its 32-bit word; the
// arrays start 256-byte aligned); returns the byte's previous value.
__device__ __forceinline__ uint32_t byte_or(uint8_t* arr, int32_t v, uint32_t bits) {
    uint32_t* wd = reinterpret_cast<uint32_t*>(arr + (v & ~3));
    const uint32_t sh = 8u * (uint32_t)(v & 3);
    return (atomicOr(wd, bits << sh) >> sh) & 0xFFu;
}

// Append vertex v (lanes with `want`) to the next frontier's piece list and, if
// `count`, add its out-degree to the next frontier's edge count.  Warp-collective.
__device__ __forceinline__ void enqueue_next(Bundle& B, const BGraph& G, int nxt, int32_t v, bool want,
                                             bool count = true) {
    const int lane = threadIdx.x & 31;
    if (!__any_sync(kFull, want)) return;
    const int32_t d = want ? G.out_deg[v] : 0;
    const uint32_t np = want ? pieces_of(d) : 0u;
    uint32_t incl = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    unsigned long long de = (unsigned long long)d;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) de += __shfl_xor_sync(kFull, de, o);
    uint32_t base = 0u;
    if (lane == 31) {
        base = atomicAdd(&B.npiece[nxt], total);
        if (count && de) atomicAdd(&B.next_medges, de);
    }
    base = __shfl_sync(kFull, base, 31);
    int2* out = B.piece[nxt] + base + (incl - np);
    for (uint32_t p = 0; p < np; ++p) out[p] = make_int2(v, (int32_t)p);
}

// The bundle holding work item `item` of direction d's queue: the last bundle
// whose offset in that queue is at most `item` (offsets are exclusive prefixes
// over all bundles, a bundle of the other direction counting zero items, so it
// shares its offset with the next bundle and is never the last one found).
__device__ __forceinline__ int32_t bundle_of(const Bundle* bs, int32_t nb, int d, uint32_t item) {
    int32_t lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (bs[mid].item0[d] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Out-degree of the lanes' vertices that joined the next frontier, added to the
// next frontier's edge count (a pull lists the frontier only when a push follows).
// Warp-collective.
__device__ __forceinline__ void count_next(Bundle& B, const BGraph& G, int32_t v, bool want) {
    unsigned long long de = want ? (unsigned long long)G.out_deg[v] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) de += __shfl_xor_sync(kFull, de, o);
    if ((threadIdx.x & 31) == 0 && de) atomicAdd(&B.next_medges, de);
}

// One pull work item k of bundle B.  Warp-collective.
__device__ __forceinline__ void pull_item(Bundle& B, const BGraph& G, uint32_t k, uint32_t t, int cur, int nxt) {
    const int lane = threadIdx.x & 31;
    const uint8_t* __restrict__ fc = B.front[cur];
    uint8_t* __restrict__ fn = B.front[nxt];
    uint32_t mask = 0u;
    if (k < B.n_small) {  // 32 vertices of small in-degree, a lane each
        const int64_t i = G.in_off[0] + (int64_t)k * 32 + lane;
        int32_t v = 0;
        if (i < G.in_off[1]) {
            v = G.in_list[i];
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
                    const uint32_t w = in_weight(G, e);
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
        count_next(B, G, v, mask != 0u);
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
                const uint32_t w = in_weight(G, e);
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
        count_next(B, G, v, lane == 0 && mask != 0u);
    } else {  // 32 vertices without in-edges: nothing reaches them
        k -= B.n_big;
        const int64_t i = (int64_t)k * 32 + lane;
        if (i < G.zero_count) fn[G.zero_in[i]] = 0u;
    }
    mask = __reduce_or_sync(kFull, mask);
    if (lane == 0 && mask) atomicOr(&B.next_active, mask);
}

// One push work item k of bundle B: piece k of the frontier list, 8 out-edges a
// lane (strided across the warp).  Warp-collective.
__device__ __forceinline__ void push_item(Bundle& B, const BGraph& G, uint32_t k, uint32_t t, int cur, int nxt) {
    const int lane = threadIdx.x & 31;
    const int2 pc = B.piece[cur][k];
    const int32_t u = pc.x;
    const int32_t beg = G.row_ptr[u] + pc.y * kPiece;
    const int32_t end = min(G.row_ptr[u + 1], beg + kPiece);
    const uint32_t bits = B.front[cur][u];
    uint32_t m[kSlots];
    if (B.sssp) load_msgs(B.msg[cur], u, m);
    uint32_t changed_all = 0u;
    for (int j = 0; j < kPiece / 32; ++j) {
        const int32_t e = beg + j * 32 + lane;
        int32_t v = 0;
        uint32_t changed = 0u;
        if (e < end) {
            v = G.col[e];
            if (B.sssp) {
                const uint32_t w = G.w ? G.w[e] : 1u;
#pragma unroll
                for (int q = 0; q < kSlots; ++q) {
                    if (!((bits >> q) & 1u)) continue;
                    const uint32_t cand = sat_add(m[q], w);
                    if (cand < B.out[q][v] && cand < atomicMin(&B.out[q][v], cand)) changed |= 1u << q;
                }
            } else {
                const uint32_t nw = bits & ~(uint32_t)B.vis[v];
                if (nw) {
                    changed = nw & ~byte_or(B.vis, v, nw);  // the queries this thread brought to v first
#pragma unroll
                    for (int q = 0; q < kSlots; ++q)
                        if ((changed >> q) & 1u) B.out[q][v] = t + 1u;
                }
            }
        }
        const bool fresh = changed != 0u && byte_or(B.front[nxt], v, changed) == 0u;
        enqueue_next(B, G, nxt, v, fresh);
        changed_all |= changed;
    }
    changed_all = __reduce_or_sync(kFull, changed_all);
    if (lane == 0 && changed_all) atomicOr(&B.next_active, changed_all);
}

// The pull and push work of a superstep: two kernels (each compiled for its own
// register use), run side by side as two branches of the loop graph.
__global__ void __launch_bounds__(kThreads) batch_pull(BArgs a) {
    const BCtl* c = a.ctl;
    if (c->any_active == 0u) return;
    const uint32_t t = c->t, total = c->total[1];
    const int cur = (int)(t & 1u), nxt = cur ^ 1;
    const uint32_t gwarp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
    for (uint32_t item = gwarp; item < total; item += nwarps) {
        Bundle& B = a.bundles[bundle_of(a.bundles, a.nb, 1, item)];
        pull_item(B, a.graphs[B.graph], item - B.item0[1], t, cur, nxt);
    }
}

__global__ void __launch_bounds__(kThreads) batch_push(BArgs a) {
    const BCtl* c = a.ctl;
    if (c->any_active == 0u) return;
    const uint32_t t = c->t, total = c->total[0];
    const int cur = (int)(t & 1u), nxt = cur ^ 1;
    const uint32_t gwarp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
    for (uint32_t item = gwarp; item < total; item += nwarps) {
        Bundle& B = a.bundles[bundle_of(a.bundles, a.nb, 0, item)];
        push_item(B, a.graphs[B.graph], item - B.item0[0], t, cur, nxt);
    }
}

// Direction of the superstep after this one, from the next frontier's out-edges.
__device__ __forceinline__ uint32_t next_direction(const Bundle& B, const BGraph& G) {
    const unsigned long long lim = B.sssp ? G.pull_above_sssp : G.pull_above_bfs;
    return G.dir_mode == 1 ? 0u : (G.dir_mode == 2 ? 1u : (B.next_medges > lim ? 1u : 0u));
}

// After the relax, per bundle: decide the next direction; after a push, clear
// the frontier bytes just consumed (a push needs its output bytes clear, and
// these are the output two supersteps later) and, for SSSP, write the next
// frontier's message rows from the final distances of this superstep; after a
// pull followed by a push, list the next frontier from its bytes and clear the
// consumed bytes whole (a pull rewrites every byte, so it needs neither).
__global__ void __launch_bounds__(kThreads) batch_finish(BArgs a) {
    const BCtl* c = a.ctl;
    if (c->any_active == 0u) return;
    const int cur = (int)(c->t & 1u), nxt = cur ^ 1;
    const int lane = threadIdx.x & 31;
    const int64_t gtid = (int64_t)blockIdx.x * kThreads + threadIdx.x, gsize = (int64_t)gridDim.x * kThreads;
    const int64_t gwarp = gtid >> 5, nwarps = gsize >> 5;
    for (int32_t b = 0; b < a.nb; ++b) {
        Bundle& B = a.bundles[b];
        if (B.active == 0u) continue;
        const BGraph& G = a.graphs[B.graph];
        const uint32_t nd = next_direction(B, G);
        uint8_t* fc = B.front[cur];
        if (B.dir) {
            if (nd == 0u) {  // pull, then push
                const int64_t n = G.n;
                for (int64_t i = gtid; i < (n + 15) / 16; i += gsize)
                    reinterpret_cast<uint4*>(fc)[i] = make_uint4(0u, 0u, 0u, 0u);
                const uint8_t* fn = B.front[nxt];
                for (int64_t base = gwarp * 32; base < n; base += nwarps * 32) {
                    const int64_t v = base + lane;
                    enqueue_next(B, G, nxt, (int32_t)(v < n ? v : 0), v < n && fn[v] != 0u, false);
                }
            }
            if (gtid == 0) B.next_dir = nd;
            continue;
        }
        if (gtid == 0) B.next_dir = nd;
        for (int64_t i = gtid; i < (int64_t)B.npiece[cur]; i += gsize) {
            const int2 pc = B.piece[cur][i];
            if (pc.y == 0) fc[pc.x] = 0u;
        }
        if (!B.sssp) continue;
        const uint8_t* fn = B.front[nxt];
        for (int64_t i = gtid; i < (int64_t)B.npiece[nxt]; i += gsize) {
            const int2 pc = B.piece[nxt][i];
            if (pc.y != 0) continue;
            const int32_t v = pc.x;
            const uint32_t fb = fn[v];
            uint32_t r[kSlots];
#pragma unroll
            for (int q = 0; q < kSlots; ++q) r[q] = ((fb >> q) & 1u) ? B.out[q][v] : kInf;
            uint4* row = reinterpret_cast<uint4*>(B.msg[nxt] + (int64_t)v * kSlots);
            row[0] = make_uint4(r[0], r[1], r[2], r[3]);
            row[1] = make_uint4(r[4], r[5], r[6], r[7]);
        }
    }
}

// Exclusive prefixes of the bundles' n_items into the push and the pull queue
// offsets (item0[d]; a bundle counts in its direction's queue only), and the
// totals.  One CTA of kPlanThreads; every thread calls it.
__device__ void layout_items(BArgs& a, uint32_t* s_scan) {
    for (int d = 0; d < 2; ++d) {
        uint32_t base = 0u;
        for (int32_t b0 = 0; b0 < a.nb; b0 += kPlanThreads) {
            const int32_t b = b0 + (int32_t)threadIdx.x;
            const uint32_t x = (b < a.nb && a.bundles[b].dir == (uint32_t)d) ? a.bundles[b].n_items : 0u;
            s_scan[threadIdx.x] = x;
            __syncthreads();
            for (int o = 1; o < kPlanThreads; o <<= 1) {  // Hillis-Steele inclusive scan
                const uint32_t y = threadIdx.x >= (unsigned)o ? s_scan[threadIdx.x - o] : 0u;
                __syncthreads();
                s_scan[threadIdx.x] += y;
                __syncthreads();
            }
            if (b < a.nb) a.bundles[b].item0[d] = base + s_scan[threadIdx.x] - x;
            base += s_scan[kPlanThreads - 1];
            __syncthreads();
        }
        if (threadIdx.x == 0) a.ctl->total[d] = base;
    }
}

// Bundle B's next superstep in direction d: its work items.
__device__ __forceinline__ void plan_bundle(Bundle& B, uint32_t d, int nxt) {
    B.dir = d;
    B.n_items = d ? B.n_small + B.n_big + B.n_zero : B.npiece[nxt];
}

// One CTA: retire the queries whose next frontier is empty, stop at max_iters,
// pick each bundle's next direction, lay out the next work queue, advance the
// superstep and set the loop condition.
__global__ void __launch_bounds__(kPlanThreads) batch_plan(BArgs a) {
    BCtl* c = a.ctl;
    __shared__ uint32_t s_any;
    __shared__ uint32_t s_scan[kPlanThreads];
    if (c->any_active == 0u) return;
    const uint32_t t = c->t;
    const int cur = (int)(t & 1u), nxt = cur ^ 1;
    if (threadIdx.x == 0) s_any = 0u;
    __syncthreads();
    const bool stop = (c->max_iters != 0u && t + 1u >= c->max_iters) || (uint64_t)t + 1u >= a.guard;
    for (int32_t b = threadIdx.x; b < a.nb; b += blockDim.x) {
        Bundle& B = a.bundles[b];
        if (B.active == 0u) {
            B.n_items = 0u;
            continue;
        }
        const uint32_t still = stop ? 0u : (B.active & B.next_active);
        const uint32_t ended = B.active & ~still;
        for (int q = 0; q < kSlots; ++q)
            if ((ended >> q) & 1u) a.iters[B.qid[q]] = (int32_t)(t + 1u);
        if (still == 0u && (B.active & B.next_active) != 0u && (uint64_t)t + 1u >= a.guard) c->guard_hit = 1u;
        B.active = still;
        B.next_active = 0u;
        if (still) {
            plan_bundle(B, B.next_dir, nxt);
            atomicOr(&s_any, 1u);
        } else {
            B.n_items = 0u;
        }
        B.next_medges = 0ull;
        B.npiece[cur] = 0u;  // consumed; it collects the frontier of superstep t + 2
    }
    __syncthreads();
    layout_items(a, s_scan);
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
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
             v += (int64_t)gridDim.x * blockDim.x) {
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

// The sources (one CTA; a thread per bundle, after batch_clear), the first
// frontier's piece lists and directions, and the first work queue.
__global__ void __launch_bounds__(kPlanThreads) batch_seed(BArgs a) {
    __shared__ uint32_t s_scan[kPlanThreads];
    for (int32_t b = threadIdx.x; b < a.nb; b += blockDim.x) {
        Bundle& B = a.bundles[b];
        const BGraph& G = a.graphs[B.graph];
        uint32_t np = 0u;
        unsigned long long me = 0ull;
        for (int q = 0; q < B.nq; ++q) {
            const int32_t s = B.source[q];
            B.out[q][s] = 0u;
            if (B.front[0][s] == 0u) {  // a source not listed yet
                const int32_t d = G.out_deg[s];
                for (uint32_t p = 0; p < pieces_of(d); ++p) B.piece[0][np++] = make_int2(s, (int32_t)p);
                me += (unsigned long long)d;
            }
            B.front[0][s] |= (uint8_t)(1u << q);
            if (B.sssp) B.msg[0][(int64_t)s * kSlots + q] = 0u;
            else B.vis[s] |= (uint8_t)(1u << q);
        }
        B.npiece[0] = np;
        B.npiece[1] = 0u;
        B.next_medges = me;
        plan_bundle(B, next_direction(B, G), 0);
        B.next_medges = 0ull;
    }
    __syncthreads();
    layout_items(a, s_scan);
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
        const bool wu = g->wtype == GM_W_U32;
        G.col_ptr = as<int32_t>(g->col_ptr);
        G.row = as<int32_t>(g->row);
        G.cw = wu ? as<uint32_t>(g->cw) : nullptr;
        G.cw8 = wu ? as<uint8_t>(g->cw8) : nullptr;
        G.row_ptr = as<int32_t>(g->row_ptr);
        G.col = as<int32_t>(g->col);
        G.w = wu ? as<uint32_t>(g->w) : nullptr;
        G.out_deg = as<int32_t>(g->out_deg);
        G.in_list = as<int32_t>(g->in_list);
        for (int b = 0; b < 4; ++b) G.in_off[b] = g->in_list_count[b];
        G.zero_in = as<int32_t>(g->zero_in_list);
        G.zero_count = g->zero_in_count;
        G.n = g->n;
        // the handle's switch points: SSSP pulls above 4 x sssp_pull_frac of the
        // edges (one pull serves up to 8 queries; 4 x measured best on the 64-graph
        // workload), BFS above 1/alpha of them (the single-query rule with every
        // edge unvisited)
        G.pull_above_sssp = (unsigned long long)(std::min(1.0, 4.0 * g->tune.sssp_pull_frac) * (double)g->m);
        G.pull_above_bfs = (unsigned long long)((double)g->m / std::max(g->tune.alpha, 1e-9));
        G.dir_mode = g->tune.direction;
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
    auto pieces_cap = [&](const Bundle& B) {  // an entry per vertex and one per 256 out-edges
        const int64_t n = hg[B.graph].n > 0 ? hg[B.graph].n : 1;
        return (size_t)n + (size_t)(graphs[B.graph]->m / kPiece) + 2;
    };
    size_t ws = 0;
    std::vector<size_t> offs(hb.size());
    for (size_t b = 0; b < hb.size(); ++b) {
        Bundle& B = hb[b];
        const BGraph& G = hg[B.graph];
        const int64_t n = G.n > 0 ? G.n : 1;
        B.n_small = (uint32_t)((G.in_off[1] - G.in_off[0] + 31) / 32);
        B.n_big = (uint32_t)(G.in_off[3] - G.in_off[1]);
        B.n_zero = (uint32_t)((G.zero_count + 31) / 32);
        if ((uint64_t)B.n_small + B.n_big + B.n_zero >= (1ull << 31) || pieces_cap(B) >= (1ull << 31)) {
            set_error("gm_run_batch: graph %d is too large for the batched form", B.graph);
            return GM_ERR_INVALID_ARG;
        }
        B.active = (1u << B.nq) - 1u;
        offs[b] = ws;
        ws += 2 * round((size_t)n) + 2 * round(sizeof(int2) * pieces_cap(B)) +
              (B.sssp ? 2 * round(sizeof(uint32_t) * kSlots * (size_t)n) : round((size_t)n));
    }
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
        B.piece[0] = reinterpret_cast<int2*>(p);
        p += round(sizeof(int2) * pieces_cap(B));
        B.piece[1] = reinterpret_cast<int2*>(p);
        p += round(sizeof(int2) * pieces_cap(B));
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
    a.iters = as<int32_t>(diters);
    a.ctl = as<BCtl>(ctl);
    a.guard = (uint64_t)max_n + 2u;
    {
        const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_n + 255) / 256, 256)),
                        (unsigned)std::min<size_t>(hb.size(), 65535));
        batch_clear<<<grid, 256, 0, s>>>(a);
        batch_seed<<<1, kPlanThreads, 0, s>>>(a);
        g_launches += 2;
        GM_CUDA_TRY(cudaGetLastError());
    }
    // the superstep loop: WHILE { pull bundles || push bundles; finish; plan }
    int per_sm_pull = 0, per_sm_push = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_pull, batch_pull, kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_push, batch_push, kThreads, 0);
    per_sm_pull = std::max(per_sm_pull, 1);
    per_sm_push = std::max(per_sm_push, 1);
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
        cudaGraphNode_t nr[2] = {nullptr, nullptr}, n2 = nullptr, n3 = nullptr;
        kp.func = (void*)batch_pull;
        kp.gridDim = dim3((unsigned)(per_sm_pull * num_sms()));
        e = cudaGraphAddKernelNode(&nr[0], body, nullptr, 0, &kp);
        if (e == cudaSuccess) {
            kp.func = (void*)batch_push;
            kp.gridDim = dim3((unsigned)(per_sm_push * num_sms()));
            e = cudaGraphAddKernelNode(&nr[1], body, nullptr, 0, &kp);
        }
        if (e == cudaSuccess) {
            kp.func = (void*)batch_finish;
            kp.gridDim = dim3((unsigned)(2 * num_sms()));
            e = cudaGraphAddKernelNode(&n2, body, nr, 2, &kp);
        }
        if (e == cudaSuccess) {
            kp.func = (void*)batch_plan;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(kPlanThreads);
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
    std::vector<int32_t> its((size_t)n_queries);
    GM_CUDA_TRY(cudaMemcpyAsync(its.data(), diters.p, sizeof(int32_t) * (size_t)n_queries, cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaMemcpyAsync(&hc, ctl.p, sizeof(BCtl), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    g_launches += 4ull * hc.t;
    if (iters_done)
        for (int32_t i = 0; i < n_queries; ++i) iters_done[i] = its[(size_t)i];
    if (hc.guard_hit) {
        set_error("gm_run_batch: superstep loop exceeded its bound (internal error)");
        return GM_ERR_TIMEOUT;
    }
    return GM_OK;
}

}  // extern "C"
