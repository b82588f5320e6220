// BFS and SSSP supersteps (Algorithms 1 and 2 with the min semiring).
//
// One superstep is two kernels:
//   relax     the generalized SPMV with Process_Message/Reduce fused into the
//             update of the vertex property (Apply = min), either
//               push: over the out-edges (CSR) of the compacted frontier queue,
//                     atomicMin / atomicCAS on the destination, or
//               pull: over the in-edges (CSC) of every candidate vertex, testing
//                     the frontier bitvector (Section 4.3.2: the bitvector form
//                     of the sparse vector), no atomics on the property;
//             vertices whose property changed are written to the next frontier
//             (bitvector bit + queue entry, warp-aggregated) -- Algorithm 2's
//             "mark changed vertices active" without a separate scan.
//   finalize  SSSP: snapshot the messages (property values) of the next frontier;
//             the last CTA to finish counts the active vertices, stops at
//             convergence or max_iters, and picks push or pull for the next
//             superstep from the frontier size.
// Work inside a relax launch is split by degree bin: vertices of small degree
// are processed 32 to a warp with their edge lists concatenated, medium ones a
// warp each, large ones a CTA each.
//
// BSP semantics are exact: messages come from values fixed at the start of the
// superstep (BFS: the constant t+1; SSSP: the snapshot `msg`), so the property
// after each superstep and the superstep count equal Algorithm 2's.
#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kFull = 0xffffffffu;

struct TravCtlDev {
    TravCtl c;
    int32_t max_iters;   // < 0: until no vertex is active
    int32_t dir_mode;    // 0 auto, 1 push, 2 pull
    float alpha, beta, sssp_frac;
};

struct TravArgs {
    const int32_t* row_ptr; const int32_t* col; const uint32_t* w;
    const int32_t* col_ptr; const int32_t* row; const uint32_t* cw;
    const int32_t* out_deg; const int32_t* in_deg; const uint8_t* out_bin;
    const int32_t* in_list; int64_t in_off[4];
    int64_t n, m, nwords;
    uint32_t* dist; uint32_t* msg;
    uint32_t* bv[3];
    int32_t* q[3][4];        // [slot][bin], bin 1..3 used
    TravCtlDev* ctl;
    cudaGraphConditionalHandle cond;
    int use_cond;
};

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
    uint32_t s = a + b;
    return (s < a || s == kInf) ? kInf : s;
}

__device__ __forceinline__ bool test_bit(const uint32_t* bv, int32_t v) {
    return (__ldg(bv + (v >> 5)) >> (v & 31)) & 1u;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_min_u32(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Append the vertices with want == true (one per lane) to the next frontier of
// slot `nxt`, grouped by out-degree bin.  Must be called by all 32 lanes.
template <bool BFS>
__device__ __forceinline__ void warp_enqueue(const TravArgs& a, bool want, int32_t v, int nxt) {
    const uint32_t any = __ballot_sync(kFull, want);
    if (!any) return;
    const int lane = threadIdx.x & 31;
    uint32_t bin = 0, deg = 0, indeg = 0;
    if (want) {
        bin = a.out_bin[v];
        deg = (uint32_t)a.out_deg[v];
        if (BFS) indeg = (uint32_t)a.in_deg[v];
    }
    unsigned long long ds = warp_sum_u64(deg);
    unsigned long long is = BFS ? warp_sum_u64(indeg) : 0ull;
    TravCtl* c = &a.ctl->c;
    if (lane == 0) {
        if (ds) atomicAdd(&c->medges[nxt], ds);
        if (BFS && is) atomicAdd(&c->unvisited_in_edges, 0ull - is);
    }
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (uint32_t b = 0; b < 4; ++b) {
        const uint32_t mb = __ballot_sync(kFull, want && bin == b);
        if (!mb) continue;
        const int leader = __ffs(mb) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&c->count[nxt][b], (uint32_t)__popc(mb));
        base = __shfl_sync(kFull, base, leader);
        if (b > 0 && want && bin == b) a.q[nxt][b][base + __popc(mb & lt)] = v;
    }
}

// Push-side relaxation of edge (u -> v) with message du (SSSP) / t+1 (BFS).
// Returns true for the single caller that must enqueue v.
template <bool SSSP>
__device__ __forceinline__ bool push_edge(const TravArgs& a, int32_t v, uint32_t du, uint32_t wgt, uint32_t t,
                                          int nxt) {
    if (!SSSP) {
        if (a.dist[v] != kInf) return false;
        if (atomicCAS(&a.dist[v], kInf, t + 1) != kInf) return false;
        atomicOr(&a.bv[nxt][v >> 5], 1u << (v & 31));
        return true;
    } else {
        const uint32_t nd = sat_add(du, wgt);
        if (nd >= a.dist[v]) return false;
        const uint32_t old = atomicMin(&a.dist[v], nd);
        if (nd >= old) return false;
        const uint32_t bit = 1u << (v & 31);
        return (atomicOr(&a.bv[nxt][v >> 5], bit) & bit) == 0;
    }
}

// ---------------------------------------------------------------- push
template <bool SSSP>
__device__ void push_phase(const TravArgs& a, uint32_t t, int cur, int nxt, unsigned long long& scanned, unsigned long long& vcount) {
    const TravCtl* c = &a.ctl->c;
    const uint32_t nS = c->count[cur][1], nM = c->count[cur][2], nL = c->count[cur][3];
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kThreads) >> 5;

    // large: one CTA per vertex
    for (uint32_t i = blockIdx.x; i < nL; i += gridDim.x) {
        const int32_t u = a.q[cur][3][i];
        if (threadIdx.x == 0) ++vcount;
        const uint32_t du = SSSP ? a.msg[u] : 0u;
        const int32_t beg = a.row_ptr[u], end = a.row_ptr[u + 1];
        for (int32_t base = beg; base < end; base += kThreads) {
            const int32_t e = base + threadIdx.x;
            bool want = false;
            int32_t v = 0;
            if (e < end) {
                v = a.col[e];
                want = push_edge<SSSP>(a, v, du, SSSP ? a.w[e] : 0u, t, nxt);
                ++scanned;
            }
            warp_enqueue<!SSSP>(a, want, v, nxt);
        }
    }
    // medium: one warp per vertex
    for (uint32_t i = gwarp; i < nM; i += nwarps) {
        const int32_t u = a.q[cur][2][i];
        if (lane == 0) ++vcount;
        const uint32_t du = SSSP ? a.msg[u] : 0u;
        const int32_t beg = a.row_ptr[u], end = a.row_ptr[u + 1];
        for (int32_t base = beg; base < end; base += 32) {
            const int32_t e = base + lane;
            bool want = false;
            int32_t v = 0;
            if (e < end) {
                v = a.col[e];
                want = push_edge<SSSP>(a, v, du, SSSP ? a.w[e] : 0u, t, nxt);
                ++scanned;
            }
            warp_enqueue<!SSSP>(a, want, v, nxt);
        }
    }
    // small: 32 vertices per warp, edge lists concatenated
    for (uint32_t grp = gwarp; grp * 32u < nS; grp += nwarps) {
        const uint32_t i = grp * 32u + lane;
        int32_t beg = 0;
        uint32_t deg = 0, du = 0;
        if (i < nS) {
            const int32_t u = a.q[cur][1][i];
            ++vcount;
            beg = a.row_ptr[u];
            deg = (uint32_t)(a.row_ptr[u + 1] - beg);
            du = SSSP ? a.msg[u] : 0u;
        }
        const uint32_t incl = warp_incl_scan(deg);
        const uint32_t excl = incl - deg;
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t j = base + lane;
            int k = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const uint32_t ex = __shfl_sync(kFull, excl, k + step);
                if (ex <= j) k += step;
            }
            const int32_t bo = __shfl_sync(kFull, beg, k);
            const uint32_t eo = __shfl_sync(kFull, excl, k);
            const uint32_t duo = __shfl_sync(kFull, du, k);
            bool want = false;
            int32_t v = 0;
            if (j < total) {
                const int32_t e = bo + (int32_t)(j - eo);
                v = a.col[e];
                want = push_edge<SSSP>(a, v, duo, SSSP ? a.w[e] : 0u, t, nxt);
                ++scanned;
            }
            warp_enqueue<!SSSP>(a, want, v, nxt);
        }
    }
}

// ---------------------------------------------------------------- pull
// BFS: an unvisited vertex takes depth t+1 at its first in-neighbour in the
// frontier (early exit).  SSSP: min over in-neighbours in the frontier of
// msg[u] + w(u, v), applied with min.
template <bool SSSP>
__device__ void pull_phase(const TravArgs& a, uint32_t t, int cur, int nxt, unsigned long long& scanned, unsigned long long& vcount) {
    const int lane = threadIdx.x & 31;
    const int warp_in_cta = threadIdx.x >> 5;
    const uint32_t gwarp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
    const uint32_t* __restrict__ bvc = a.bv[cur];
    __shared__ uint32_t s_red[kThreads / 32];
    __shared__ uint32_t s_slot[kThreads / 32][32];

    // large: one CTA per vertex
    {
        const int64_t lo = a.in_off[2], hi = a.in_off[3];
        for (int64_t i = lo + blockIdx.x; i < hi; i += gridDim.x) {
            const int32_t v = a.in_list[i];
            if (!SSSP && a.dist[v] != kInf) continue;  // uniform over the CTA
            if (threadIdx.x == 0) ++vcount;
            const int32_t beg = a.col_ptr[v], end = a.col_ptr[v + 1];
            uint32_t best = kInf;
            for (int32_t base = beg; base < end; base += kThreads) {
                const int32_t e = base + threadIdx.x;
                bool hit = false;
                if (e < end) {
                    const int32_t u = a.row[e];
                    ++scanned;
                    if (test_bit(bvc, u)) {
                        hit = true;
                        if (SSSP) best = min(best, sat_add(a.msg[u], a.cw[e]));
                    }
                }
                if (!SSSP) {
                    if (__syncthreads_or(hit)) { best = t + 1; break; }
                }
            }
            if (SSSP) {
                best = warp_min_u32(best);
                if (lane == 0) s_red[warp_in_cta] = best;
                __syncthreads();
                if (warp_in_cta == 0) {
                    uint32_t b2 = lane < kThreads / 32 ? s_red[lane] : kInf;
                    best = warp_min_u32(b2);
                }
                __syncthreads();
            }
            if (warp_in_cta == 0) {
                bool want = false;
                if (lane == 0) {
                    if (best < a.dist[v]) {
                        a.dist[v] = best;
                        atomicOr(&a.bv[nxt][v >> 5], 1u << (v & 31));
                        want = true;
                    }
                }
                warp_enqueue<!SSSP>(a, want, v, nxt);
            }
            __syncthreads();
        }
    }
    // medium: one warp per vertex
    {
        const int64_t lo = a.in_off[1], hi = a.in_off[2];
        for (int64_t i = lo + gwarp; i < hi; i += nwarps) {
            const int32_t v = a.in_list[i];
            if (!SSSP && a.dist[v] != kInf) continue;  // uniform over the warp
            if (lane == 0) ++vcount;
            const int32_t beg = a.col_ptr[v], end = a.col_ptr[v + 1];
            uint32_t best = kInf;
            for (int32_t base = beg; base < end; base += 32) {
                const int32_t e = base + lane;
                bool hit = false;
                if (e < end) {
                    const int32_t u = a.row[e];
                    ++scanned;
                    if (test_bit(bvc, u)) {
                        hit = true;
                        if (SSSP) best = min(best, sat_add(a.msg[u], a.cw[e]));
                    }
                }
                if (!SSSP && __any_sync(kFull, hit)) { best = t + 1; break; }
            }
            if (SSSP) best = warp_min_u32(best);
            bool want = false;
            if (lane == 0 && best < a.dist[v]) {
                a.dist[v] = best;
                atomicOr(&a.bv[nxt][v >> 5], 1u << (v & 31));
                want = true;
            }
            warp_enqueue<!SSSP>(a, want, v, nxt);
        }
    }
    // small: 32 vertices per warp, in-edge lists concatenated
    {
        const int64_t lo = a.in_off[0], hi = a.in_off[1];
        uint32_t* slot = s_slot[warp_in_cta];
        for (int64_t g0 = lo + (int64_t)gwarp * 32; g0 < hi; g0 += (int64_t)nwarps * 32) {
            const int64_t i = g0 + lane;
            int32_t v = 0, beg = 0;
            uint32_t deg = 0;
            if (i < hi) {
                v = a.in_list[i];
                if (SSSP || a.dist[v] == kInf) {
                    ++vcount;
                    beg = a.col_ptr[v];
                    deg = (uint32_t)(a.col_ptr[v + 1] - beg);
                }
            }
            slot[lane] = kInf;
            __syncwarp();
            const uint32_t incl = warp_incl_scan(deg);
            const uint32_t excl = incl - deg;
            const uint32_t total = __shfl_sync(kFull, incl, 31);
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t j = base + lane;
                int k = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const uint32_t ex = __shfl_sync(kFull, excl, k + step);
                    if (ex <= j) k += step;
                }
                const int32_t bo = __shfl_sync(kFull, beg, k);
                const uint32_t eo = __shfl_sync(kFull, excl, k);
                if (j < total) {
                    const int32_t e = bo + (int32_t)(j - eo);
                    const int32_t u = a.row[e];
                    ++scanned;
                    if (test_bit(bvc, u)) {
                        if (SSSP) atomicMin(&slot[k], sat_add(a.msg[u], a.cw[e]));
                        else slot[k] = t + 1;
                    }
                }
            }
            __syncwarp();
            bool want = false;
            if (i < hi && deg > 0) {
                const uint32_t best = slot[lane];
                if (best < a.dist[v]) {
                    a.dist[v] = best;
                    atomicOr(&a.bv[nxt][v >> 5], 1u << (v & 31));
                    want = true;
                }
            }
            warp_enqueue<!SSSP>(a, want, v, nxt);
            __syncwarp();
        }
    }
}

template <bool SSSP>
__global__ void __launch_bounds__(kThreads) trav_relax(TravArgs a) {
    TravCtlDev* cd = a.ctl;
    if (cd->c.done) return;
    const uint32_t t = cd->c.iter;
    const int cur = (int)(t % 3u), nxt = (int)((t + 1u) % 3u), clr = (int)((t + 2u) % 3u);
    {   // clear the bitvector two supersteps back (it becomes "next" in superstep t+1)
        uint32_t* bz = a.bv[clr];
        for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < a.nwords;
             i += (int64_t)gridDim.x * kThreads)
            bz[i] = 0u;
    }
    unsigned long long scanned = 0, vcount = 0;
    if (cd->c.dir == 0) push_phase<SSSP>(a, t, cur, nxt, scanned, vcount);
    else pull_phase<SSSP>(a, t, cur, nxt, scanned, vcount);
    scanned = warp_sum_u64(scanned);
    vcount = warp_sum_u64(vcount);
    if ((threadIdx.x & 31) == 0) {
        if (scanned) atomicAdd(&cd->c.scanned_edges, scanned);
        if (vcount) atomicAdd(&cd->c.processed_vertices, vcount);
    }
}

template <bool SSSP>
__global__ void __launch_bounds__(kThreads) trav_finalize(TravArgs a) {
    TravCtlDev* cd = a.ctl;
    TravCtl* c = &cd->c;
    __shared__ uint32_t s_t, s_done, s_last;
    __shared__ uint32_t s_cnt[4];
    if (threadIdx.x == 0) {
        s_t = c->iter;
        s_done = c->done;
    }
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = c->count[(c->iter + 1u) % 3u][threadIdx.x];
    __syncthreads();
    if (s_done) return;
    const uint32_t t = s_t;
    const int nxt = (int)((t + 1u) % 3u);
    if (SSSP) {  // messages of the next superstep: property values fixed now
        const uint32_t n1 = s_cnt[1], n2 = s_cnt[2], n3 = s_cnt[3];
        const uint32_t tot = n1 + n2 + n3;
        for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < tot; i += gridDim.x * kThreads) {
            int32_t v;
            if (i < n1) v = a.q[nxt][1][i];
            else if (i < n1 + n2) v = a.q[nxt][2][i - n1];
            else v = a.q[nxt][3][i - n1 - n2];
            a.msg[v] = a.dist[v];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(&c->ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    // ---- last CTA: termination and direction for superstep t+1 ----
    __threadfence();
    c->ticket = 0;
    const unsigned long long active = (unsigned long long)s_cnt[0] + s_cnt[1] + s_cnt[2] + s_cnt[3];
    const uint32_t iters = t + 1u;
    if (c->dir == 0) c->pushes++;
    else c->pulls++;
    uint32_t done = (active == 0ull) ? 1u : 0u;
    if (cd->max_iters >= 0 && iters >= (uint32_t)cd->max_iters) done = 1u;
    // Min-semiring traversals with non-negative weights settle within n supersteps
    // (shortest paths have at most n-1 edges) plus one that finds no change.
    if (!done && (unsigned long long)iters >= (unsigned long long)a.n + 2ull) {
        done = 1u;
        c->guard_hit = 1u;
    }
    if (!done) {
        uint32_t dir = c->dir;
        const double mf = (double)c->medges[nxt];
        if (cd->dir_mode == 1) dir = 0;
        else if (cd->dir_mode == 2) dir = 1;
        else if (!SSSP) {
            if (dir == 0) dir = (mf > (double)c->unvisited_in_edges / cd->alpha) ? 1u : 0u;
            else dir = ((double)active < (double)a.n / cd->beta) ? 0u : 1u;
        } else {
            dir = (mf > cd->sssp_frac * (double)a.m) ? 1u : 0u;
        }
        c->dir = dir;
        const int clr = (int)((t + 2u) % 3u);
        for (int b = 0; b < 4; ++b) c->count[clr][b] = 0u;
        c->medges[clr] = 0ull;
    }
    c->iter = iters;
    c->iters_done = iters;
    c->done = done;
    if (a.use_cond) cudaGraphSetConditional(a.cond, done ? 0u : 1u);
}

// ---------------------------------------------------------------- frontier set-up
__global__ void seed_frontier(TravArgs a, const int32_t* __restrict__ verts, int64_t count, int bfs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool want = false;
    int32_t v = 0;
    if (i < count) v = verts[i];
    if (i < count && (v < 0 || v >= a.n)) {
        atomicAdd(&a.ctl->c.bad_ids, 1u);
    } else if (i < count) {
        a.dist[v] = 0u;
        a.msg[v] = 0u;
        const uint32_t bit = 1u << (v & 31);
        want = (atomicOr(&a.bv[0][v >> 5], bit) & bit) == 0;
    }
    if (bfs) warp_enqueue<true>(a, want, v, 0);
    else warp_enqueue<false>(a, want, v, 0);
}

__global__ void seed_all(TravArgs a, int bfs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool want = i < a.n;
    const int32_t v = want ? (int32_t)i : 0;
    if (want) {
        a.dist[v] = 0u;
        a.msg[v] = 0u;
        atomicOr(&a.bv[0][v >> 5], 1u << (v & 31));
    }
    if (bfs) warp_enqueue<true>(a, want, v, 0);
    else warp_enqueue<false>(a, want, v, 0);
}

__global__ void fill_u32(uint32_t* p, int64_t n, uint32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void reached_kernel(const uint32_t* __restrict__ dist, const int32_t* __restrict__ out_deg, int64_t n,
                               unsigned long long* out) {
    unsigned long long s = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (dist[v] != kInf) s += (unsigned long long)out_deg[v];
    s = warp_sum_u64(s);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// Workspace layout inside g->work for BFS/SSSP.
struct TravWork {
    uint32_t* msg;
    uint32_t* bv[3];
    int32_t* q[3][4];
};

TravWork work_layout(gm_graph* g) {
    TravWork w{};
    const int64_t n = g->n > 0 ? g->n : 1;
    const int64_t nwords = (n + 31) / 32;
    char* p = static_cast<char*>(g->work.p);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    };
    w.msg = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    for (int s = 0; s < 3; ++s) w.bv[s] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * nwords));
    for (int s = 0; s < 3; ++s) {
        w.q[s][0] = nullptr;
        for (int b = 1; b < 4; ++b) w.q[s][b] = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
    }
    return w;
}

size_t work_bytes(int64_t n) {
    n = n > 0 ? n : 1;
    const int64_t nwords = (n + 31) / 32;
    auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return r(sizeof(uint32_t) * n) + 3 * r(sizeof(uint32_t) * nwords) + 9 * r(sizeof(int32_t) * n);
}

TravArgs make_args(gm_graph* g) {
    TravArgs a{};
    TravWork w = work_layout(g);
    a.row_ptr = as<int32_t>(g->row_ptr);
    a.col = as<int32_t>(g->col);
    a.w = as<uint32_t>(g->w);
    a.col_ptr = as<int32_t>(g->col_ptr);
    a.row = as<int32_t>(g->row);
    a.cw = as<uint32_t>(g->cw);
    a.out_deg = as<int32_t>(g->out_deg);
    a.in_deg = as<int32_t>(g->in_deg);
    a.out_bin = as<uint8_t>(g->out_bin);
    a.in_list = as<int32_t>(g->in_list);
    for (int b = 0; b < 4; ++b) a.in_off[b] = g->in_list_count[b];
    a.n = g->n;
    a.m = g->m;
    a.nwords = (g->n + 31) / 32;
    a.dist = as<uint32_t>(g->state);
    a.msg = w.msg;
    for (int s = 0; s < 3; ++s) {
        a.bv[s] = w.bv[s];
        for (int b = 0; b < 4; ++b) a.q[s][b] = w.q[s][b];
    }
    a.ctl = as<TravCtlDev>(g->ctl_buf);
    a.use_cond = 0;
    return a;
}

int relax_grid() {
    static int blocks = 0;
    if (blocks == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trav_relax<true>, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
        blocks = per_sm * num_sms();
    }
    return blocks;
}

int finalize_grid() { return 2 * num_sms(); }

#define LAUNCH_OK()                                                                             \
    do {                                                                                        \
        cudaError_t _e = cudaGetLastError();                                                    \
        if (_e != cudaSuccess) {                                                                \
            set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(_e), __FILE__, __LINE__); \
            return GM_ERR_CUDA;                                                                 \
        }                                                                                       \
    } while (0)

// Reset the control block and the frontier before seeding.
gm_status reset_frontier(gm_graph* g) {
    cudaStream_t s = g->stream;
    TravWork w = work_layout(g);
    const int64_t nwords = ((g->n > 0 ? g->n : 1) + 31) / 32;
    for (int k = 0; k < 3; ++k) GM_CUDA_TRY(cudaMemsetAsync(w.bv[k], 0, sizeof(uint32_t) * nwords, s));
    TravCtlDev h{};
    h.c.dir = g->tune.direction == 2 ? 1u : 0u;
    h.c.unvisited_in_edges = (unsigned long long)g->m;
    h.max_iters = -1;
    h.dir_mode = g->tune.direction;
    h.alpha = (float)g->tune.alpha;
    h.beta = (float)g->tune.beta;
    h.sssp_frac = (float)g->tune.sssp_pull_frac;
    TravCtlDev* hp = static_cast<TravCtlDev*>(g->host_pinned);
    *hp = h;
    GM_CUDA_TRY(cudaMemcpyAsync(g->ctl_buf.p, hp, sizeof(TravCtlDev), cudaMemcpyHostToDevice, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));  // the pinned staging buffer is reused
    return GM_OK;
}

gm_status build_loop_graph(gm_graph* g, bool sssp) {
    if (g->loop_exec) {
        cudaGraphExecDestroy(g->loop_exec);
        g->loop_exec = nullptr;
    }
    if (g->loop_graph) {
        cudaGraphDestroy(g->loop_graph);
        g->loop_graph = nullptr;
    }
    cudaGraph_t graph;
    GM_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("cudaGraphConditionalHandleCreate: %s", cudaGetErrorString(e));
        return GM_ERR_CUDA;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("cudaGraphAddNode(conditional): %s", cudaGetErrorString(e));
        return GM_ERR_CUDA;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    TravArgs a = make_args(g);
    a.cond = handle;
    a.use_cond = 1;
    void* kargs[] = {&a};
    cudaKernelNodeParams kp = {};
    kp.func = sssp ? (void*)trav_relax<true> : (void*)trav_relax<false>;
    kp.gridDim = dim3((unsigned)relax_grid());
    kp.blockDim = dim3(kThreads);
    kp.kernelParams = kargs;
    cudaGraphNode_t n1, n2;
    e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &kp);
    if (e == cudaSuccess) {
        kp.func = sssp ? (void*)trav_finalize<true> : (void*)trav_finalize<false>;
        kp.gridDim = dim3((unsigned)finalize_grid());
        e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &kp);
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("superstep loop graph: %s", cudaGetErrorString(e));
        return GM_ERR_CUDA;
    }
    g->loop_graph = graph;
    g->loop_exec = exec;
    g->loop_graph_max_iters = sssp ? 1 : 0;  // records which program the graph was built for
    return GM_OK;
}

}  // namespace

gm_status trav_prepare(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n > 0 ? g->n : 1;
    GM_TRY(dev_alloc(g->state, sizeof(uint32_t) * n, s));
    GM_TRY(dev_alloc(g->work, work_bytes(g->n), s));
    g->work_bytes = (int64_t)work_bytes(g->n);
    GM_TRY(dev_alloc(g->ctl_buf, sizeof(TravCtlDev), s));
    fill_u32<<<num_sms() * 4, 256, 0, s>>>(as<uint32_t>(g->state), g->n, kInf);
    g_launches++;
    LAUNCH_OK();
    return reset_frontier(g);
}

gm_status trav_set_active(gm_graph* g, const int32_t* vertices_dev, int64_t count) {
    cudaStream_t s = g->stream;
    TravArgs a = make_args(g);
    const int bfs = g->kind == GM_BFS ? 1 : 0;
    if (count < 0) {
        if (g->n > 0) {
            seed_all<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(a, bfs);
            g_launches++;
            LAUNCH_OK();
        }
    } else if (count > 0) {
        seed_frontier<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(a, vertices_dev, count, bfs);
        g_launches++;
        LAUNCH_OK();
    }
    return GM_OK;
}

gm_status trav_run(gm_graph* g, int32_t max_iters, int32_t* iters_done) {
    cudaStream_t s = g->stream;
    const bool sssp = g->kind == GM_SSSP;
    g->stats = RunStats{};
    if (max_iters == 0) {
        if (iters_done) *iters_done = 0;
        return reset_frontier(g);
    }
    TravCtlDev* hp = static_cast<TravCtlDev*>(g->host_pinned);
    // parameters that may change between runs
    {
        int32_t params[2] = {max_iters, g->tune.direction};
        GM_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(g->ctl_buf.p) + offsetof(TravCtlDev, max_iters), params,
                                    sizeof(params), cudaMemcpyHostToDevice, s));
        float f[3] = {(float)g->tune.alpha, (float)g->tune.beta, (float)g->tune.sssp_pull_frac};
        GM_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(g->ctl_buf.p) + offsetof(TravCtlDev, alpha), f,
                                    sizeof(f), cudaMemcpyHostToDevice, s));
    }
    const bool host_loop = g->tune.loop_mode == 1 || g->tune.profile;
    if (!host_loop) {
        if (!g->loop_exec || g->loop_graph_max_iters != (sssp ? 1 : 0)) GM_TRY(build_loop_graph(g, sssp));
        GM_CUDA_TRY(cudaGraphLaunch(g->loop_exec, s));
    } else {
        TravArgs a = make_args(g);
        const int rg = relax_grid(), fg = finalize_grid();
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (g->tune.profile) {
            GM_CUDA_TRY(cudaEventCreate(&ev0));
            GM_CUDA_TRY(cudaEventCreate(&ev1));
        }
        unsigned long long prev_e = 0, prev_v = 0;
        for (int32_t it = 0;; ++it) {
            uint32_t dir_before = 0, frontier_before = 0;
            if (ev0) {  // direction and frontier size of this superstep, for the trace
                GM_CUDA_TRY(cudaMemcpyAsync(hp, g->ctl_buf.p, sizeof(TravCtlDev), cudaMemcpyDeviceToHost, s));
                GM_CUDA_TRY(cudaStreamSynchronize(s));
                dir_before = hp->c.dir;
                const uint32_t slot = hp->c.iter % 3u;
                frontier_before = hp->c.count[slot][0] + hp->c.count[slot][1] + hp->c.count[slot][2] +
                                  hp->c.count[slot][3];
            }
            if (ev0) cudaEventRecord(ev0, s);
            if (sssp) trav_relax<true><<<rg, kThreads, 0, s>>>(a);
            else trav_relax<false><<<rg, kThreads, 0, s>>>(a);
            if (ev1) cudaEventRecord(ev1, s);
            g_launches++;
            LAUNCH_OK();
            if (sssp) trav_finalize<true><<<fg, kThreads, 0, s>>>(a);
            else trav_finalize<false><<<fg, kThreads, 0, s>>>(a);
            g_launches++;
            LAUNCH_OK();
            GM_CUDA_TRY(cudaMemcpyAsync(&hp->c.done, &as<TravCtlDev>(g->ctl_buf)->c.done, sizeof(uint32_t),
                                        cudaMemcpyDeviceToHost, s));
            GM_CUDA_TRY(cudaStreamSynchronize(s));
            if (ev0) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev0, ev1);
                g->stats.relax_ms += ms;
                g->stats.relax_launches++;
                const uint32_t done = hp->c.done;
                GM_CUDA_TRY(cudaMemcpyAsync(hp, g->ctl_buf.p, sizeof(TravCtlDev), cudaMemcpyDeviceToHost, s));
                GM_CUDA_TRY(cudaStreamSynchronize(s));
                const double row[kTraceCols] = {(double)it, (double)dir_before, (double)frontier_before,
                                                (double)(hp->c.scanned_edges - prev_e),
                                                (double)(hp->c.processed_vertices - prev_v), (double)ms,
                                                (double)hp->c.medges[(it + 1) % 3]};
                prev_e = hp->c.scanned_edges;
                prev_v = hp->c.processed_vertices;
                g->stats.trace.insert(g->stats.trace.end(), row, row + kTraceCols);
                hp->c.done = done;
            }
            if (hp->c.done) break;
        }
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
    GM_CUDA_TRY(cudaMemcpyAsync(hp, g->ctl_buf.p, sizeof(TravCtlDev), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    if (!host_loop) g_launches += 2ull * hp->c.iters_done;
    g->stats.supersteps = (int32_t)hp->c.iters_done;
    g->stats.pushes = (int32_t)hp->c.pushes;
    g->stats.pulls = (int32_t)hp->c.pulls;
    g->stats.scanned_edges = (int64_t)hp->c.scanned_edges;
    g->stats.processed_vertices = (int64_t)hp->c.processed_vertices;
    if (iters_done) *iters_done = (int32_t)hp->c.iters_done;
    const uint32_t bad = hp->c.bad_ids;
    const uint32_t guard = hp->c.guard_hit;
    GM_TRY(reset_frontier(g));
    if (guard) {
        set_error("gm_run: superstep loop exceeded n + 1 supersteps (internal error)");
        return GM_ERR_TIMEOUT;
    }
    if (bad) {
        set_error("gm_run: %u active vertex ids given to gm_set_active were outside [0, %lld) and ignored", bad,
                  (long long)g->n);
        return GM_ERR_INVALID_ARG;
    }
    return GM_OK;
}

gm_status reached_edges(gm_graph* g, int64_t* out) {
    cudaStream_t s = g->stream;
    DevBuf acc;
    GM_TRY(dev_alloc(acc, sizeof(unsigned long long), s));
    gm_status st = GM_OK;
    cudaError_t e = cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess && g->n > 0) {
        reached_kernel<<<num_sms() * 4, 256, 0, s>>>(as<uint32_t>(g->state), as<int32_t>(g->out_deg), g->n,
                                                     as<unsigned long long>(acc));
        g_launches++;
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_error("reached_edges: %s", cudaGetErrorString(e)); st = GM_ERR_CUDA; }
    dev_free(acc, s);
    *out = (int64_t)h;
    return st;
}

void trav_release(gm_graph* g) {
    if (g->loop_exec) cudaGraphExecDestroy(g->loop_exec);
    if (g->loop_graph) cudaGraphDestroy(g->loop_graph);
    g->loop_exec = nullptr;
    g->loop_graph = nullptr;
    g->loop_graph_max_iters = -2;
}

}  // namespace gm
