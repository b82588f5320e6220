// BFS and SSSP supersteps (Algorithms 1 and 2 with the min semiring).
//
// One superstep is three kernels (push, pull, finalize); the direction not
// chosen on the device returns at once, and inside the device loop a one-CTA
// kernel (trav_small) first runs every superstep whose frontier is tiny:
//   relax     the generalized SPMV with Process_Message/Reduce fused into the
//             update of the vertex property (Apply = min), either
//               push: over the out-edges (CSR) of the compacted frontier queue,
//                     atomicCAS (BFS) / atomicMin (SSSP) on the destination, or
//               pull: over the in-edges (CSC) of every candidate vertex; BFS
//                     tests the frontier bitvector (Section 4.3.2's bitvector
//                     form of the sparse vector), SSSP gathers the message array
//                     (infinity off the frontier), the owner applies min;
//             vertices whose property changed join the next frontier (bitvector
//             bit + binned queue, warp-aggregated) -- Algorithm 2's "mark changed
//             vertices active" without a separate scan of the active array.
//   finalize  SSSP after a pull: Apply of the pull's per-column minima; SSSP
//             after a push: the messages of the next frontier; then the last
//             CTA to finish counts the active vertices, stops at convergence or
//             max_iters, and picks push or pull for the next superstep.
//
// Work decomposition for HBM bandwidth: every lane handles 8 edges per step with
// two 16-byte streaming loads per edge array, so each warp keeps 1-2 KB of edge
// data in flight.  Push: frontier vertices of small degree go 32 to a warp with
// their edge lists concatenated; the edges of medium vertices and of the
// 2048-edge chunks of large ones are cut into 256-edge pieces dealt to all
// warps.  Pull: fixed 256-edge warp tiles over the doubly compressed CSC,
// columns crossing tiles combined with atomics.
//
// BSP semantics are exact: messages come from values fixed at the start of the
// superstep (BFS: the constant t+1; SSSP: the message array), so the property
// after each superstep and the superstep count equal Algorithm 2's.
#include <algorithm>

#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kEPT = 8;                    // edges per lane per step
constexpr int kWarpSpan = 32 * kEPT;       // 256 edges per warp step
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
    const uint8_t* cw8;      // one byte per in-edge weight when all fit (nullptr otherwise)
    const int32_t* out_deg; const int32_t* in_deg; const uint8_t* out_bin;
    int32_t bin_small, bin_large;  // degree bins (out_bin[v] == out_bin_of(out_deg[v]))
    const int32_t* in_list; int64_t in_s0, in_s1, in_m1;  // small bin [in_s0, in_s1), medium [in_s1, in_m1)
    const int32_t* dc_jc; const int32_t* dc_cp; const int32_t* dc_tile;  // doubly compressed CSC + tiles
    int64_t dc_ncols, ntiles;
    int64_t n, m, nwords;
    uint32_t* dist;
    uint32_t* msg[2];        // SSSP messages of superstep t live in msg[t & 1], infinity elsewhere,
                             // indexed by source rank (msg[.][rank[v]] is vertex v's message)
    const int32_t* rank;     // SSSP: rank of each vertex by out-degree (descending)
    const int32_t* row_r;    // SSSP: CSC sources as ranks
    const uint32_t* oct_w;   // SSSP octet layout (or nullptr): (rank << 8) | weight per slot,
    const uint8_t* oct_meta; //   octet headers (real slots, first octet of a column),
    const int32_t* oct_c0;   //   first column of every tile of 32 octets
    int64_t oct_tiles;
    const int32_t* dc_rank;  // SSSP: rank of each non-empty column's vertex
    int32_t hot;             // SSSP pull: messages of ranks [0, hot) are staged in shared memory
    uint16_t* msg16;         // octet pull: the messages of ranks [0, hot16) as signed 16 bits (-1 = infinity),
    int32_t hot16;           //   written by the push launch of a pull superstep and staged instead of msg
    uint32_t stage_extra;    // test hook: bytes the staging barrier expects beyond its copies (0 or 16)
    uint32_t* lkey;          // sorted-list sparse vector (GM_OPT_SPARSE_LIST): indices, ascending
    uint32_t* lval;          //   and values (SSSP messages) of the current pull superstep's frontier
    uint32_t* ltile;         //   per-tile counts, then offsets, of the list build
    uint32_t* ycol;          // pull: reduced value per non-empty column, infinity between supersteps
    const uint32_t* dc_head; // pull: first-edge-of-column bits
    uint32_t* bv[3];         // frontier bitvectors, rotating by superstep
    int32_t* q[3][3];        // [slot][bin], bins 1 (small) and 2 (medium)
    int2* qc[3];             // [slot] large-bin work items (vertex, chunk)
    TravCtlDev* ctl;
    cudaGraphConditionalHandle cond;
    int use_cond;
};

constexpr uint32_t kStage = 256;  // per-warp staging capacity of each queue bin

// Per-warp staging of the next frontier in shared memory: bins 1 and 2 are
// appended here and copied to the global queue with one atomic per flush, so
// warps do not all serialise on the same few queue counters.
struct WarpQ {
    int32_t buf[2][kStage];
    uint32_t n[2];
};

// Per-thread statistics (reduced per CTA once per kernel) and the warp's stage.
struct Acc {
    unsigned long long scanned, verts, medges, unvis, n0;
    unsigned long long reached;  // out-degrees of vertices whose property went from infinity to finite
    WarpQ* wq;  // nullptr: enqueue straight to the global queue
};

// a + b, infinity when the sum reaches or passes UINT32_MAX (a sum equal to
// UINT32_MAX already is infinity; one that wrapped is below b).
__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return s < b ? kInf : s;
}

// Out-degree bin of a vertex from its out-degree (the rule that built out_bin).
__device__ __forceinline__ uint32_t out_bin_of(const TravArgs& a, uint32_t d) {
    return d == 0u ? 0u : (d < (uint32_t)a.bin_small ? 1u : (d < (uint32_t)a.bin_large ? 2u : 3u));
}

__device__ __forceinline__ bool test_bit(const uint32_t* bv, int32_t v) {
    return (__ldg(bv + (v >> 5)) >> (v & 31)) & 1u;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
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

// 8 consecutive 4-byte values at p[e0..e0+7]; e0 % 4 == 0, streaming (evict-first).
template <typename T>
__device__ __forceinline__ void load8(const T* p, int32_t e0, T (&x)[kEPT]) {
    const int4 lo = __ldcs(reinterpret_cast<const int4*>(p + e0));
    const int4 hi = __ldcs(reinterpret_cast<const int4*>(p + e0 + 4));
    x[0] = (T)lo.x; x[1] = (T)lo.y; x[2] = (T)lo.z; x[3] = (T)lo.w;
    x[4] = (T)hi.x; x[5] = (T)hi.y; x[6] = (T)hi.z; x[7] = (T)hi.w;
}

// Copy a warp's staged bin (1 or 2) to the global queue of slot nxt.  Warp-collective.
__device__ __forceinline__ void warp_flush(const TravArgs& a, WarpQ* wq, uint32_t b, int nxt) {
    const int lane = threadIdx.x & 31;
    const uint32_t n = wq->n[b - 1];
    if (n == 0u) return;
    uint32_t base = 0u;
    if (lane == 0) base = atomicAdd(&a.ctl->c.count[nxt][b], n);
    base = __shfl_sync(kFull, base, 0);
    int32_t* dst = a.q[nxt][b] + base;
    for (uint32_t i = lane; i < n; i += 32) dst[i] = wq->buf[b - 1][i];
    __syncwarp();
    if (lane == 0) wq->n[b - 1] = 0u;
    __syncwarp();
}

// Append the vertices v[k] with want[k] to the next frontier of slot `nxt`,
// grouped by out-degree bin (large vertices as one item per chunk); vb, vd and vin
// hold each wanted vertex's out-degree bin, out-degree and (BFS) in-degree, loaded
// by the caller ahead of time.  Warp-collective.
template <bool BFS>
__device__ __forceinline__ void enqueue_batch_pre(const TravArgs& a, const bool (&want)[kEPT],
                                                  const int32_t (&v)[kEPT], const uint32_t (&vb)[kEPT],
                                                  const uint32_t (&vd)[kEPT], const uint32_t (&vin)[kEPT], int nxt,
                                                  Acc& acc) {
    bool mine = false;
#pragma unroll
    for (int k = 0; k < kEPT; ++k) mine |= want[k];
    if (!__any_sync(kFull, mine)) return;
    const int lane = threadIdx.x & 31;
    uint32_t cnt[4] = {0u, 0u, 0u, 0u};
    uint32_t bin[kEPT], nch[kEPT];
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        bin[k] = 0u;
        nch[k] = 0u;
        if (want[k]) {
            const uint32_t b = vb[k];
            const uint32_t d = vd[k];
            acc.medges += d;
            if (BFS) {
                acc.unvis += vin[k];
                acc.reached += d;  // a BFS vertex joins a frontier once: when first reached
            }
            bin[k] = b;
            nch[k] = b == 3u ? (d + kChunk - 1u) / kChunk : 1u;
            cnt[b] += nch[k];
        }
    }
    TravCtl* c = &a.ctl->c;
#pragma unroll
    for (uint32_t b = 0; b < 4; ++b) {
        if (b == 0u && acc.wq) {  // no out-edges: counted as active, never pushed from
            acc.n0 += cnt[0];
            continue;
        }
        const uint32_t incl = warp_incl_scan(cnt[b]);
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        if (tot == 0u) continue;
        if (acc.wq && b < 3u) {
            WarpQ* wq = acc.wq;
            uint32_t n = wq->n[b - 1];
            if (n + tot > kStage) {
                warp_flush(a, wq, b, nxt);
                n = 0u;
            }
            uint32_t pos = n + incl - cnt[b];
#pragma unroll
            for (int k = 0; k < kEPT; ++k)
                if (want[k] && bin[k] == b) wq->buf[b - 1][pos++] = v[k];
            __syncwarp();
            if (lane == 0) wq->n[b - 1] = n + tot;
            __syncwarp();
            continue;
        }
        uint32_t base = 0u;
        if (lane == 31) base = atomicAdd(&c->count[nxt][b], tot);
        base = __shfl_sync(kFull, base, 31);
        if (b == 0u) continue;
        uint32_t pos = base + incl - cnt[b];
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            if (!want[k] || bin[k] != b) continue;
            if (b < 3u) {
                a.q[nxt][b][pos++] = v[k];
            } else {
                for (uint32_t ch = 0; ch < nch[k]; ++ch) a.qc[nxt][pos++] = make_int2(v[k], (int32_t)ch);
            }
        }
    }
}

// enqueue_batch_pre with the degree data loaded here.  Warp-collective.
template <bool BFS>
__device__ __forceinline__ void enqueue_batch(const TravArgs& a, const bool (&want)[kEPT], const int32_t (&v)[kEPT],
                                              int nxt, Acc& acc) {
    bool mine = false;
#pragma unroll
    for (int k = 0; k < kEPT; ++k) mine |= want[k];
    if (!__any_sync(kFull, mine)) return;
    uint32_t vb[kEPT], vd[kEPT], vin[kEPT];
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        vb[k] = want[k] ? (uint32_t)a.out_bin[v[k]] : 0u;
        vd[k] = want[k] ? (uint32_t)a.out_deg[v[k]] : 0u;
        vin[k] = (BFS && want[k]) ? (uint32_t)a.in_deg[v[k]] : 0u;
    }
    enqueue_batch_pre<BFS>(a, want, v, vb, vd, vin, nxt, acc);
}

// Push relaxation of up to 8 edges (u -> v[k]) with messages du[k]; `ok` masks
// valid edges.  Atomics are issued in phases so a lane keeps several in flight.
template <bool SSSP>
__device__ __forceinline__ void push_relax8(const TravArgs& a, const int32_t (&v)[kEPT], const uint32_t (&wt)[kEPT],
                                            const uint32_t (&du)[kEPT], uint32_t ok, uint32_t t, int nxt,
                                            bool (&want)[kEPT], Acc& acc) {
    uint32_t curd[kEPT];
#pragma unroll
    for (int k = 0; k < kEPT; ++k) curd[k] = ((ok >> k) & 1u) ? a.dist[v[k]] : 0u;
    if (!SSSP) {
        uint32_t old[kEPT];
#pragma unroll
        for (int k = 0; k < kEPT; ++k)
            old[k] = (((ok >> k) & 1u) && curd[k] == kInf) ? atomicCAS(&a.dist[v[k]], kInf, t + 1u) : 0u;
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            want[k] = ((ok >> k) & 1u) && curd[k] == kInf && old[k] == kInf;
            if (want[k]) atomicOr(&a.bv[nxt][v[k] >> 5], 1u << (v[k] & 31));
        }
    } else {
        uint32_t nd[kEPT], old[kEPT];
        bool tr[kEPT];
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            nd[k] = sat_add(du[k], wt[k]);
            tr[k] = ((ok >> k) & 1u) && nd[k] < curd[k];
        }
#pragma unroll
        for (int k = 0; k < kEPT; ++k) old[k] = tr[k] ? atomicMin(&a.dist[v[k]], nd[k]) : 0u;
        uint32_t prev[kEPT];
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            tr[k] = tr[k] && nd[k] < old[k];
            if (tr[k] && old[k] == kInf) acc.reached += (uint32_t)__ldg(a.out_deg + v[k]);
            prev[k] = tr[k] ? atomicOr(&a.bv[nxt][v[k] >> 5], 1u << (v[k] & 31)) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kEPT; ++k) want[k] = tr[k] && !((prev[k] >> (v[k] & 31)) & 1u);
    }
}

// Lane step over a contiguous edge range: edges e0..e0+7 masked to [beg, end).
template <bool SSSP>
__device__ __forceinline__ void push_contig(const TravArgs& a, int32_t e0, int32_t beg, int32_t end, uint32_t du,
                                            uint32_t t, int nxt, Acc& acc) {
    int32_t v[kEPT];
    uint32_t wt[kEPT], dv[kEPT];
    uint32_t ok = 0u;
    if (e0 < end) {
        load8(a.col, e0, v);
        if (SSSP) load8(a.w, e0, wt);
#pragma unroll
        for (int k = 0; k < kEPT; ++k)
            if (e0 + k >= beg && e0 + k < end) ok |= 1u << k;
    }
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
        if (!((ok >> k) & 1u)) { v[k] = 0; wt[k] = 0u; }
        if (!SSSP) wt[k] = 0u;
        dv[k] = du;
    }
    bool want[kEPT];
    push_relax8<SSSP>(a, v, wt, dv, ok, t, nxt, want, acc);
    acc.scanned += (unsigned)__popc(ok);
    enqueue_batch<!SSSP>(a, want, v, nxt, acc);
}

// Largest o in [0, 31] with ex[o] <= j (ex non-decreasing, 33 entries).
__device__ __forceinline__ int owner_of(const uint32_t* ex, uint32_t j) {
    int o = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
        if (ex[o + step] <= j) o += step;
    return o;
}

// ---------------------------------------------------------------- push
template <bool SSSP>
__device__ void push_phase(const TravArgs& a, uint32_t t, int cur, int nxt, Acc& acc, uint32_t* sw) {
    const TravCtl* c = &a.ctl->c;
    const uint32_t nS = c->count[cur][1], nM = c->count[cur][2], nC = c->count[cur][3];
    const uint32_t* __restrict__ msgc = a.msg[t & 1u];
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kThreads) >> 5;

    // Large chunks and medium vertices as warp pieces, dealt to every warp of the
    // grid so that no CTA or warp is left with a long serial tail: piece p of an
    // edge range [beg, end) is the 16-byte-aligned window
    // [(beg & ~3) + 256 p, + 256) clipped to the range (one warp step); a range
    // has at most kPiecesL (chunk of 2048) or pm (medium: degree < bin_large)
    // such windows, and windows past its end are empty.
    constexpr uint32_t kPiecesL = kChunk / kWarpSpan + 1;
    const uint32_t pm = (uint32_t)(((int64_t)a.bin_large + 2 + kWarpSpan - 1) / kWarpSpan);
    const uint64_t nL64 = (uint64_t)nC * kPiecesL, nMP64 = (uint64_t)nM * pm;
    // 32-bit piece numbers (always, short of graphs with ~2^28 frontier vertices);
    // else large chunks a CTA each and medium vertices a warp each
    const bool pieces = pm <= 16u && nL64 + nMP64 < (1ull << 32);
    const uint32_t nL = pieces ? (uint32_t)nL64 : 0u, nP = pieces ? (uint32_t)(nL64 + nMP64) : 0u;
    for (uint32_t i = gwarp; i < nP; i += nwarps) {
        int32_t u, beg, end;
        uint32_t p;
        bool first;
        if (i < nL) {
            const uint32_t c = i / kPiecesL;
            const int2 it = a.qc[cur][c];
            p = i - c * kPiecesL;
            u = it.x;
            beg = a.row_ptr[u] + it.y * kChunk;
            end = min(a.row_ptr[u + 1], beg + kChunk);
            first = it.y == 0 && p == 0u;
        } else {
            const uint32_t j = i - nL, vi = j / pm;
            p = j - vi * pm;
            u = a.q[cur][2][vi];
            beg = a.row_ptr[u];
            end = a.row_ptr[u + 1];
            first = p == 0u;
        }
        const int32_t base = (beg & ~3) + (int32_t)p * kWarpSpan;
        if (base >= end) continue;  // warp-uniform
        if (lane == 0 && first) acc.verts++;
        const uint32_t du = SSSP ? msgc[a.rank[u]] : 0u;
        push_contig<SSSP>(a, base + lane * kEPT, beg, end, du, t, nxt, acc);
    }
    if (!pieces) {
        for (uint32_t i = blockIdx.x; i < nC; i += gridDim.x) {  // large: one CTA per 2048-edge chunk
            const int2 it = a.qc[cur][i];
            const int32_t u = it.x;
            if (threadIdx.x == 0 && it.y == 0) acc.verts++;
            const int32_t beg = a.row_ptr[u] + it.y * kChunk;
            const int32_t end = min(a.row_ptr[u + 1], beg + kChunk);
            const uint32_t du = SSSP ? msgc[a.rank[u]] : 0u;
            for (int32_t base = beg & ~3; base < end; base += kThreads * kEPT)
                push_contig<SSSP>(a, base + (int32_t)threadIdx.x * kEPT, beg, end, du, t, nxt, acc);
        }
        // medium: one warp per vertex
        for (uint32_t i = gwarp; i < nM; i += nwarps) {
            const int32_t u = a.q[cur][2][i];
            if (lane == 0) acc.verts++;
            const int32_t beg = a.row_ptr[u], end = a.row_ptr[u + 1];
            const uint32_t du = SSSP ? msgc[a.rank[u]] : 0u;
            for (int32_t base = beg & ~3; base < end; base += kWarpSpan)
                push_contig<SSSP>(a, base + lane * kEPT, beg, end, du, t, nxt, acc);
        }
    }
    // small: 32 vertices per warp, edge lists concatenated
    int32_t* s_beg = reinterpret_cast<int32_t*>(sw);
    uint32_t* s_ex = sw + 32;  // 33 entries
    uint32_t* s_du = sw + 65;
    for (uint32_t grp = gwarp; grp * 32u < nS; grp += nwarps) {
        const uint32_t i = grp * 32u + lane;
        int32_t beg = 0;
        uint32_t deg = 0u, du = 0u;
        if (i < nS) {
            const int32_t u = a.q[cur][1][i];
            acc.verts++;
            beg = a.row_ptr[u];
            deg = (uint32_t)(a.row_ptr[u + 1] - beg);
            du = SSSP ? msgc[a.rank[u]] : 0u;
        }
        const uint32_t incl = warp_incl_scan(deg);
        __syncwarp();
        s_beg[lane] = beg;
        s_ex[lane] = incl - deg;
        s_du[lane] = du;
        if (lane == 31) s_ex[32] = incl;
        __syncwarp();
        const uint32_t total = s_ex[32];
        for (uint32_t base = 0; base < total; base += kWarpSpan) {
            const uint32_t j0 = base + (uint32_t)lane * kEPT;
            int o = owner_of(s_ex, j0);
            int32_t v[kEPT];
            uint32_t wt[kEPT], dv[kEPT];
            uint32_t ok = 0u;
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                const uint32_t j = j0 + k;
                v[k] = 0;
                wt[k] = 0u;
                dv[k] = 0u;
                if (j < total) {
                    while (j >= s_ex[o + 1]) ++o;
                    const int32_t e = s_beg[o] + (int32_t)(j - s_ex[o]);
                    v[k] = a.col[e];
                    if (SSSP) wt[k] = a.w[e];
                    dv[k] = s_du[o];
                    ok |= 1u << k;
                }
            }
            bool want[kEPT];
            push_relax8<SSSP>(a, v, wt, dv, ok, t, nxt, want, acc);
            acc.scanned += (unsigned)__popc(ok);
            enqueue_batch<!SSSP>(a, want, v, nxt, acc);
        }
    }
}

// Work every relax launch does first: clear the frontier of superstep t-1 (its
// bitvector becomes "next" in superstep t+1) and, for SSSP, its messages in
// msg[(t+1) & 1], which finalize refills.
template <bool SSSP>
__device__ __forceinline__ void relax_prologue(const TravArgs& a, const TravCtl* c, uint32_t t, int clr) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsize = (int64_t)gridDim.x * blockDim.x;
    uint32_t* bz = a.bv[clr];
    for (int64_t i = gtid; i < a.nwords; i += gsize) bz[i] = 0u;
    if (SSSP) {
        const uint32_t n1 = c->count[clr][1], n2 = c->count[clr][2], n3 = c->count[clr][3];
        uint32_t* mz = a.msg[(t + 1u) & 1u];
        for (int64_t i = gtid; i < (int64_t)n1 + n2 + n3; i += gsize) {
            int32_t v;
            if (i < n1) v = a.q[clr][1][i];
            else if (i < (int64_t)n1 + n2) v = a.q[clr][2][i - n1];
            else v = a.qc[clr][i - n1 - n2].x;
            mz[a.rank[v]] = kInf;
        }
    }
}

// End of a relax kernel: flush the warp's staged queue, then reduce the
// statistics over the CTA and add them to the control block with one atomic each.
// CTA-collective.
__device__ __forceinline__ void flush_acc(const TravArgs& a, Acc& acc, int nxt, bool bfs,
                                          unsigned long long* s_stat) {
    TravCtl* c = &a.ctl->c;
    if (acc.wq) {
        // one queue reservation per CTA and bin: the warps' staged counts are
        // summed in shared memory and each warp writes at its own offset
        __shared__ uint32_t s_off[kWarps][2];
        __shared__ uint32_t s_base[2];
        WarpQ* q0 = acc.wq - (threadIdx.x >> 5);
        __syncthreads();
        if (threadIdx.x < 2) {
            uint32_t tot = 0;
            for (int w = 0; w < kWarps; ++w) {
                s_off[w][threadIdx.x] = tot;
                tot += q0[w].n[threadIdx.x];
            }
            s_base[threadIdx.x] = tot ? atomicAdd(&c->count[nxt][threadIdx.x + 1], tot) : 0u;
        }
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int b = 0; b < 2; ++b) {
            const uint32_t n = acc.wq->n[b];
            int32_t* dst = a.q[nxt][b + 1] + s_base[b] + s_off[warp][b];
            for (uint32_t i = lane; i < n; i += 32) dst[i] = acc.wq->buf[b][i];
        }
        __syncwarp();
        if (lane < 2) acc.wq->n[lane] = 0u;
        __syncwarp();
    }
    unsigned long long vals[6] = {acc.scanned, acc.verts, acc.medges, acc.unvis, acc.n0, acc.reached};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        vals[i] = warp_sum_u64(vals[i]);
        if ((threadIdx.x & 31) == 0 && vals[i]) atomicAdd(&s_stat[i], vals[i]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_stat[0]) atomicAdd(&c->scanned_edges, s_stat[0]);
        if (s_stat[1]) atomicAdd(&c->processed_vertices, s_stat[1]);
        if (s_stat[2]) atomicAdd(&c->medges[nxt], s_stat[2]);
        if (bfs && s_stat[3]) atomicAdd(&c->unvisited_in_edges, 0ull - s_stat[3]);
        if (s_stat[4]) atomicAdd(&c->count[nxt][0], (uint32_t)s_stat[4]);
        if (s_stat[5]) atomicAdd(&c->reached, s_stat[5]);
    }
}

// ---------------------------------------------------------------- bulk copy (TMA)
constexpr int kPullThreads = 1024;
constexpr int32_t kHotMax = 49152;      // staged messages per CTA: at most 192 KB of shared memory
                                        // (pull_stage_messages caps the option at this)
constexpr uint32_t kBulkChunk = 32768;  // bytes per cp.async.bulk instruction

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make the initialised barrier visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy; completion is counted on the barrier in bytes.
// dst, src and bytes are multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the barrier's phase `parity` to complete, giving up after about one
// second (the global timer, read every 64 tries) or 2^22 tries, whichever comes
// first; each try may suspend the thread for a short, system-dependent time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 63u && global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

// ---------------------------------------------------------------- sorted-list sparse vector
// Section 4.3.2 names two forms of the sparse vector: a variable-sized array of
// (index, value) tuples sorted by index, and a bitvector of valid indices beside
// a dense value array; the paper keeps the second because the test "is j present
// in x" of Algorithm 1 becomes one bit lookup (its Fig. 7 measures the gain).
// The engine keeps the second form too (the frontier bitvector, and for SSSP a
// dense message array holding infinity off the frontier).  For that ablation the
// option GM_OPT_SPARSE_LIST rebuilds, at the start of every pull superstep, the
// frontier as the first form -- indices ascending (SSSP: source ranks with their
// messages; BFS: vertex ids) -- in three kernels (count per tile, scan of the
// tile counts, scatter), and the pull kernels find a source's message or
// membership by binary search in that list instead of one load.
constexpr int kListThreads = 256;
constexpr int kListPer = 8;
constexpr int kListTile = kListThreads * kListPer;  // 2048 indices per tile

template <bool SSSP>
__device__ __forceinline__ bool list_valid(const TravArgs& a, uint32_t t, int64_t i, uint32_t* val) {
    if (SSSP) {
        const uint32_t m = a.msg[t & 1u][i];
        *val = m;
        return m != kInf;
    }
    *val = 0u;
    return (a.bv[t % 3u][i >> 5] >> (i & 31)) & 1u;
}

// Entries of every tile of 2048 indices into ltile[tile].
template <bool SSSP>
__global__ void __launch_bounds__(kListThreads) list_count(TravArgs a) {
    TravCtlDev* cd = a.ctl;
    if (cd->c.done || cd->c.dir != 1u) return;
    const uint32_t t = cd->c.iter;
    __shared__ uint32_t s_w[kListThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ntiles = (a.n + kListTile - 1) / kListTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < kListPer; ++k) {
            const int64_t i = tile * kListTile + k * kListThreads + threadIdx.x;
            uint32_t v;
            if (i < a.n && list_valid<SSSP>(a, t, i, &v)) ++c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (lane == 0) s_w[wid] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < kListThreads / 32; ++w) tot += s_w[w];
            a.ltile[tile] = tot;
        }
        __syncthreads();
    }
}

// One CTA: exclusive scan of the tile counts in place; the total is the list length.
constexpr int kListScanThreads = 1024;
__global__ void __launch_bounds__(kListScanThreads) list_scan(TravArgs a) {
    TravCtlDev* cd = a.ctl;
    if (cd->c.done || cd->c.dir != 1u) return;
    __shared__ uint32_t s_w[kListScanThreads / 32];
    const int64_t ntiles = (a.n + kListTile - 1) / kListTile;
    const int64_t per = (ntiles + kListScanThreads - 1) / kListScanThreads;
    const int64_t b = threadIdx.x * per, e = min(b + per, ntiles);
    uint32_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += a.ltile[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = warp_incl_scan(sum);
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const uint32_t x = warp_incl_scan(s_w[lane]);
        s_w[lane] = x;
    }
    __syncthreads();
    uint32_t run = incl - sum + (wid > 0 ? s_w[wid - 1] : 0u);  // exclusive prefix of this thread
    for (int64_t i = b; i < e; ++i) {
        const uint32_t c = a.ltile[i];
        a.ltile[i] = run;
        run += c;
    }
    if (threadIdx.x == kListScanThreads - 1) cd->c.list_len = s_w[31];
}

// Every tile's entries at its offset, in index order (eight block-wide rounds of
// 256 consecutive indices, each ranked with a ballot).
template <bool SSSP>
__global__ void __launch_bounds__(kListThreads) list_scatter(TravArgs a) {
    TravCtlDev* cd = a.ctl;
    if (cd->c.done || cd->c.dir != 1u) return;
    const uint32_t t = cd->c.iter;
    __shared__ uint32_t s_w[kListThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ntiles = (a.n + kListTile - 1) / kListTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint32_t base = a.ltile[tile];
#pragma unroll 1
        for (int k = 0; k < kListPer; ++k) {
            const int64_t i = tile * kListTile + k * kListThreads + threadIdx.x;
            uint32_t v = 0;
            const bool f = i < a.n && list_valid<SSSP>(a, t, i, &v);
            const uint32_t bal = __ballot_sync(kFull, f);
            if (lane == 0) s_w[wid] = (uint32_t)__popc(bal);
            __syncthreads();
            uint32_t before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kListThreads / 32; ++w) {
                const uint32_t c = s_w[w];
                before += w < wid ? c : 0u;
                total += c;
            }
            if (f) {
                const uint32_t pos = base + before + (uint32_t)__popc(bal & ((1u << lane) - 1u));
                a.lkey[pos] = (uint32_t)i;
                if (SSSP) a.lval[pos] = v;
            }
            base += total;
            __syncthreads();
        }
    }
}

// Position of the first list entry whose index is >= k (binary search).
__device__ __forceinline__ uint32_t list_lower(const uint32_t* __restrict__ key, uint32_t len, uint32_t k) {
    uint32_t lo = 0, cnt = len;
    while (cnt > 0) {
        const uint32_t half = cnt >> 1;
        if (__ldg(key + lo + half) < k) {
            lo += half + 1u;
            cnt -= half + 1u;
        } else {
            cnt = half;
        }
    }
    return lo;
}

// Whether source u is in the frontier (BFS pull): bitvector, or list search.
template <bool LIST>
__device__ __forceinline__ bool in_frontier(const TravArgs& a, const uint32_t* bvc, uint32_t len, int32_t u) {
    if (!LIST) return test_bit(bvc, u);
    const uint32_t p = list_lower(a.lkey, len, (uint32_t)u);
    return p < len && __ldg(a.lkey + p) == (uint32_t)u;
}

// ---------------------------------------------------------------- pull
// Pull over the doubly compressed CSC (non-empty columns only).
//  pull_a  (SSSP) streams the in-edges in warp tiles of kWTile: each lane reads 8
//          consecutive edges with 16-byte loads (the next tile's edges are already
//          in flight), evaluates Process_Message for each (msg[u] + w(u, v), msg
//          infinity off the frontier), and Reduce(min)s them per column.  Columns are found
//          without any index loads: a bit marks the first edge of every column,
//          a warp prefix count of these bits numbers the columns, and a warp
//          segmented min-scan joins the pieces of columns that span lanes.
//          Complete columns are stored to y[column]; the (at most two) columns
//          crossing the tile border are combined with atomicMin.  Sources are
//          read as out-degree ranks and the messages are kept in rank order, so
//          the messages of the hottest sources (ranks [0, hot), about 60 % of the
//          in-edges of an RMAT graph) are one contiguous block: each CTA stages it
//          into shared memory with a bulk (TMA) copy, and only the other sources
//          are gathered through L1/L2.
//  pull_bu (BFS) the same reduction bottom-up: every message is t+1, so an
//          unvisited column needs only one in-neighbour in the frontier bitvector
//          and stops at the first; a visited column cannot change (its depth is
//          at most t) and is skipped.  The result per column equals the full
//          Reduce(min) wherever Apply can use it.
//          It applies directly (one lane owns a column).
//  pull_apply (SSSP, in the finalize kernel) applies y to the vertex properties
//          (Apply = min), makes changed vertices the next frontier and resets y
//          to infinity.
// One warp tile's streamed inputs per lane: 8 in-edge source ranks, their
// weights (one-byte weights stay packed in two words until used), the lane's 8
// first-edge bits and the tile's first column.
template <int WB>
struct PullTile {
    int32_t r[kEPT];
    uint32_t w[WB == 1 ? 2 : kEPT];
    uint32_t hw;
    int32_t c0;
    __device__ __forceinline__ int32_t rank(int q) const { return r[q]; }
    __device__ __forceinline__ uint32_t weight(int q) const {
        if (WB == 1) return (w[q >> 2] >> (8 * (q & 3))) & 0xFFu;
        return w[q];
    }
};

// Edge positions are 32-bit: m < 2^31, and a tile position is below m + kWTile.
template <int WB>
__device__ __forceinline__ void pull_load_tile(const TravArgs& a, uint32_t k, int lane, PullTile<WB>& x) {
    const uint32_t p = k * (uint32_t)kWTile + (uint32_t)lane * kEPT;
    if (p < (uint32_t)a.m) {
        load8(a.row_r, (int32_t)p, x.r);
        if (WB == 1) {
            const uint2 v = __ldcs(reinterpret_cast<const uint2*>(a.cw8 + p));
            x.w[0] = v.x;
            x.w[1] = v.y;
        } else {
            uint32_t (&w8)[kEPT] = *reinterpret_cast<uint32_t(*)[kEPT]>(&x.w[0]);
            load8(a.cw, (int32_t)p, w8);
        }
    }
    x.hw = __ldcs(a.dc_head + (p >> 5));
    x.c0 = __ldg(a.dc_tile + k);
}

// Number of a lane's 8 edges that lie below m.
__device__ __forceinline__ uint32_t lane_valid(uint32_t e0, uint32_t m) { return e0 < m ? min(8u, m - e0) : 0u; }

// Messages of a tile's sources: staged ranks from shared memory, the rest from
// global memory.  Only the last tile can hold edges at or past m: there
// (`last`) they read rank 0's message (present whenever there is an edge) and
// are masked later; every other tile skips the masking.
template <int WB>
__device__ __forceinline__ void pull_gather(const uint32_t* __restrict__ msgc, const uint32_t* s_hot, int32_t hlim,
                                            bool last, uint32_t nv, const PullTile<WB>& x, uint32_t (&mv)[kEPT]) {
    if (!last) {
#pragma unroll
        for (int q = 0; q < kEPT; ++q) {
            const int32_t rq = x.rank(q);
            mv[q] = rq < hlim ? s_hot[rq] : __ldg(msgc + rq);
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < kEPT; ++q) {
        const int32_t rq = (uint32_t)q < nv ? x.rank(q) : 0;
        mv[q] = rq < hlim ? s_hot[rq] : __ldg(msgc + rq);
    }
}

// Messages of a tile's sources looked up in the sorted list (GM_OPT_SPARSE_LIST):
// infinity for a source not in it.
template <int WB>
__device__ __forceinline__ void pull_gather_list(const TravArgs& a, uint32_t len, bool last, uint32_t nv,
                                                 const PullTile<WB>& x, uint32_t (&mv)[kEPT]) {
#pragma unroll
    for (int q = 0; q < kEPT; ++q) {
        const uint32_t rq = (last && (uint32_t)q >= nv) ? 0u : (uint32_t)x.rank(q);
        const uint32_t p = list_lower(a.lkey, len, rq);
        mv[q] = (p < len && __ldg(a.lkey + p) == rq) ? __ldg(a.lval + p) : kInf;
    }
}

// WB: bytes per in-edge weight read (1: the uint8 copy, 4: the uint32 array).
// LIST: sources are looked up in the sorted-list sparse vector (no shared-memory
// stage).
// One CTA of kPullThreads per SM; dynamic shared memory holds a.hot messages.
// Software pipeline per warp: while tile k is reduced, the messages of tile k+1
// are being gathered and the sources of tile k+2 streamed in.
template <int WB, bool LIST>
__global__ void __launch_bounds__(kPullThreads, 1) trav_pull_a(TravArgs a) {
    extern __shared__ __align__(128) uint32_t s_hot[];
    __shared__ __align__(8) uint64_t s_bar;
    TravCtlDev* cd = a.ctl;
    if (cd->c.done || cd->c.dir != 1u) return;
    const uint32_t t = cd->c.iter;
    const int clr = (int)((t + 2u) % 3u);
    const uint32_t* __restrict__ msgc = a.msg[t & 1u];
    const uint32_t llen = LIST ? cd->c.list_len : 0u;
    const int32_t hot = LIST ? 0 : a.hot;  // a multiple of 4, so the copy is whole 16-byte units
    if (threadIdx.x == 0 && hot > 0) {
        mbar_init(&s_bar, 1u);
        fence_mbar_init();
        const uint32_t bytes = (uint32_t)hot * 4u;
        mbar_arrive_expect_tx(&s_bar, bytes + a.stage_extra);
        for (uint32_t off = 0; off < bytes; off += kBulkChunk)
            bulk_copy_g2s(reinterpret_cast<char*>(s_hot) + off, reinterpret_cast<const char*>(msgc) + off,
                          min(kBulkChunk, bytes - off), &s_bar);
    }
    relax_prologue<true>(a, &cd->c, t, clr);
    const int lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * kPullThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kPullThreads) >> 5;
    const uint32_t ntiles = (uint32_t)a.ntiles, m = (uint32_t)a.m;
    uint32_t* __restrict__ y = a.ycol;
    unsigned long long scanned = 0;

    // the warp's first two tiles stream in while the staging copy runs
    PullTile<WB> cur, nxt;
    if (gwarp < ntiles) pull_load_tile<WB>(a, gwarp, lane, cur);
    if (gwarp + nwarps < ntiles) pull_load_tile<WB>(a, gwarp + nwarps, lane, nxt);
    __syncthreads();  // the barrier is initialised before anyone waits on it
    bool staged = hot > 0 && mbar_wait_bounded(&s_bar, 0u);
    staged = __syncthreads_and(staged) != 0;
    if (!staged && hot > 0 && threadIdx.x == 0) atomicAdd(&cd->c.stage_timeouts, 1u);
    const int32_t hlim = staged ? hot : 0;  // without the staged block every message is gathered
    uint32_t mv[kEPT];
    if (gwarp < ntiles) {
        if (LIST)
            pull_gather_list<WB>(a, llen, gwarp + 1 == ntiles, lane_valid(gwarp * kWTile + lane * kEPT, m), cur, mv);
        else
            pull_gather<WB>(msgc, s_hot, hlim, gwarp + 1 == ntiles, lane_valid(gwarp * kWTile + lane * kEPT, m), cur,
                            mv);
    }

    for (uint32_t k = gwarp; k < ntiles; k += nwarps) {
        const uint32_t nv = lane_valid(k * kWTile + lane * kEPT, m);
        const uint32_t vmask = (1u << nv) - 1u;
        uint32_t cand[kEPT];
        if (k + 1 < ntiles) {  // a full tile (warp-uniform)
#pragma unroll
            for (int q = 0; q < kEPT; ++q) cand[q] = sat_add(mv[q], cur.weight(q));
        } else {
#pragma unroll
            for (int q = 0; q < kEPT; ++q) cand[q] = (uint32_t)q < nv ? sat_add(mv[q], cur.weight(q)) : kInf;
        }
        const uint32_t heads = (cur.hw >> ((lane & 3) * 8)) & vmask;
        const int32_t c0 = cur.c0;
        // pipeline: gather tile k+1's messages, stream tile k+2's sources
        const uint32_t k1 = k + nwarps, k2 = k1 + nwarps;
        if (k1 < ntiles) {
            if (LIST)
                pull_gather_list<WB>(a, llen, k1 + 1 == ntiles, lane_valid(k1 * kWTile + lane * kEPT, m), nxt, mv);
            else
                pull_gather<WB>(msgc, s_hot, hlim, k1 + 1 == ntiles, lane_valid(k1 * kWTile + lane * kEPT, m), nxt,
                                mv);
        }
        cur = nxt;
        if (k2 < ntiles) pull_load_tile<WB>(a, k2, lane, nxt);
        scanned += nv;

        // column numbering: heads before this lane, and whether the tile starts a column
        const uint32_t nh = (uint32_t)__popc(heads);
        const uint32_t hincl = warp_incl_scan(nh);
        const uint32_t hex = hincl - nh;
        const uint32_t bal_first = __ballot_sync(kFull, heads & 1u);  // lanes whose first edge starts a column
        const uint32_t bal_seen = __ballot_sync(kFull, heads != 0u);  // lanes holding a column start
        const uint32_t first_is_head = bal_first & 1u;
        // column of edge q of this lane: c0 + (heads in the tile up to and including
        // edge q) - (1 if the tile's first edge is a head)
        const int32_t col_base = c0 + (int32_t)hex - (int32_t)first_is_head;
        const int32_t lane_col = col_base;  // column continued by the lane's first edges (no head at bit 0)
        // lane runs: F before the first head, interior runs complete, L from the last head
        uint32_t F = kInf, run = kInf;
        int32_t run_col = lane_col;
        const bool seen = heads != 0u;
#pragma unroll
        for (int q = 0; q < kEPT; ++q) {
            if ((heads >> q) & 1u) {
                if ((heads & ((1u << q) - 1u)) != 0u) {  // an earlier head in this lane
                    if (run != kInf) y[run_col] = run;   // column entirely inside this lane
                } else {
                    F = run;
                }
                run = kInf;
                run_col = col_base + (int32_t)__popc(heads & ((2u << q) - 1u));
            }
            run = min(run, cand[q]);
        }
        if (!seen) F = run;
        // segmented min-scan across lanes: a lane holding a column start begins a
        // segment; its start lane comes from the ballot, so only values move
        uint32_t R = seen ? run : F;
        const uint32_t le = bal_seen & (0xFFFFFFFFu >> (31 - lane));  // seen lanes <= this one
        const int seg0 = le ? 31 - __clz(le) : -1;                    // -1: began before the tile
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t Ru = __shfl_up_sync(kFull, R, o);
            if (lane - o >= max(seg0, 0)) R = min(R, Ru);
        }
        uint32_t Rprev = __shfl_up_sync(kFull, R, 1);
        const bool fprev = lane > 0 && (bal_seen & ((1u << lane) - 1u)) != 0u;  // lane-1's segment began in the tile
        if (lane == 0) Rprev = kInf;
        if (seen && !(heads & 1u)) {  // this lane's first edges finish a column begun to its left
            const uint32_t total = min(F, Rprev);
            if (total != kInf) {
                if (fprev) y[lane_col] = total;            // begun inside this tile: complete here
                else atomicMin(&y[lane_col], total);       // begun in an earlier tile
            }
        }
        // The segment ending with this lane is complete when the next lane starts a
        // new column; the tile's last segment may continue in the next tile.
        const bool next_head = lane < 31 && ((bal_first >> (lane + 1)) & 1u);
        if (R != kInf && (lane == 31 || next_head)) {
            const int32_t end_col = c0 + (int32_t)hincl - (int32_t)first_is_head;
            if (lane < 31 && seg0 >= 0) y[end_col] = R;  // its first edge lies in this tile
            else atomicMin(&y[end_col], R);
        }
    }
    scanned = warp_sum_u64(scanned);
    if (lane == 0 && scanned) atomicAdd(&cd->c.scanned_edges, scanned);
    if (!staged && hot > 0) mbar_wait_bounded(&s_bar, 0u);  // let a late copy land before the CTA exits
}

// ---------------------------------------------------------------- pull over octets
// pull_o (SSSP, octet layout): the same Reduce(min) per column as pull_a, over
// in-edge lists padded to whole octets so that a lane's 8 slots always belong to
// one column.  A lane takes the minimum of its (up to 8) candidates msg[u] + w
// with no per-edge column logic; one segmented min-scan across the warp joins
// the lanes of a column (a header bit marks a column's first octet), and the
// last lane of each column stores it -- with atomicMin when the column began in
// an earlier tile or may continue into the next.  Padding slots gather nothing.
// The hot messages are staged as 16 bits (twice as many sources in the same
// shared memory as pull_a's 4-byte stage: on RMAT scale 22 the 81,920 hottest
// sources carry 66.7 % of the in-edges instead of 56.5 %), copied by TMA from
// the 16-bit array the superstep's push launch wrote.
struct OctTile {
    uint32_t w[kOctet];  // (rank << 8) | weight
    uint32_t meta;       // real slots | 0x80 at a column's first octet; 0 past the end
    int32_t c0;          // column of the tile's first octet
};

// A lane's octet of tile k: slots 0-3 and 4-7 are each one 16-byte load that
// the warp makes over 512 consecutive bytes (the tile is stored slot-quad-major).
__device__ __forceinline__ void oct_load(const TravArgs& a, uint32_t k, int lane, OctTile& x) {
    const uint32_t o = k * (uint32_t)kOctTile + (uint32_t)lane;  // octets fill whole tiles: in bounds
    const int4* t = reinterpret_cast<const int4*>(a.oct_w + (size_t)k * (kOctTile * kOctet));
    const int4 lo = __ldcs(t + lane), hi = __ldcs(t + kOctTile + lane);
    x.w[0] = (uint32_t)lo.x; x.w[1] = (uint32_t)lo.y; x.w[2] = (uint32_t)lo.z; x.w[3] = (uint32_t)lo.w;
    x.w[4] = (uint32_t)hi.x; x.w[5] = (uint32_t)hi.y; x.w[6] = (uint32_t)hi.z; x.w[7] = (uint32_t)hi.w;
    x.meta = __ldcs(a.oct_meta + o);
    x.c0 = __ldg(a.oct_c0 + k);
}

// Messages of an octet's slots: staged ranks from shared memory (signed 16 bits,
// -1 = infinity), the rest from global memory, or (LIST) from the sorted
// list.  Padding slots hold rank 0 (staged, or one shared address) and are
// masked to infinity by the caller, so the loads need no branch.
template <bool LIST>
__device__ __forceinline__ void oct_gather(const TravArgs& a, const uint32_t* __restrict__ msgc,
                                           const uint32_t* s_hot, int32_t hlim, uint32_t llen, const OctTile& x,
                                           uint32_t (&mv)[kOctet]) {
#pragma unroll
    for (int q = 0; q < kOctet; ++q) {
        const uint32_t rq = x.w[q] >> 8;
        if (LIST) {
            const uint32_t p = list_lower(a.lkey, llen, rq);
            mv[q] = (p < llen && __ldg(a.lkey + p) == rq) ? __ldg(a.lval + p) : kInf;
        } else {
            // shared memory is read only for staged ranks (with no stage the
            // kernel has no dynamic shared memory at all)
            // (a signed 16-bit read: 0xFFFF, infinity, widens to 0xFFFFFFFF; the
            // other sources are read through L2 only: about 2 % of them would hit L1)
            mv[q] = (int32_t)rq < hlim ? (uint32_t)(int32_t)reinterpret_cast<const int16_t*>(s_hot)[rq]
                                       : __ldcg(msgc + rq);
        }
    }
}

template <bool LIST>
__global__ void __launch_bounds__(kPullThreads, 1) trav_pull_o(TravArgs a) {
    extern __shared__ __align__(128) uint32_t s_hot[];
    __shared__ __align__(8) uint64_t s_bar;
    TravCtlDev* cd = a.ctl;
    if (cd->c.done || cd->c.dir != 1u) return;
    const uint32_t t = cd->c.iter;
    const int clr = (int)((t + 2u) % 3u);
    const uint32_t* __restrict__ msgc = a.msg[t & 1u];
    const uint32_t llen = LIST ? cd->c.list_len : 0u;
    // the 16-bit hot messages (a multiple of 8, so the copy is whole 16-byte
    // units), unless some did not fit 16 bits in this superstep
    const int32_t hot = (LIST || cd->c.stage16_off == t + 1u) ? 0 : a.hot16;
    if (threadIdx.x == 0 && hot > 0) {
        mbar_init(&s_bar, 1u);
        fence_mbar_init();
        const uint32_t bytes = (uint32_t)hot * 2u;
        mbar_arrive_expect_tx(&s_bar, bytes + a.stage_extra);
        for (uint32_t off = 0; off < bytes; off += kBulkChunk)
            bulk_copy_g2s(reinterpret_cast<char*>(s_hot) + off, reinterpret_cast<const char*>(a.msg16) + off,
                          min(kBulkChunk, bytes - off), &s_bar);
    }
    relax_prologue<true>(a, &cd->c, t, clr);
    const int lane = threadIdx.x & 31;
    const uint32_t lane_le = 0xFFFFFFFFu >> (31 - lane);  // lanes <= this one
    const uint32_t gwarp = (blockIdx.x * kPullThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kPullThreads) >> 5;
    const uint32_t ntiles = (uint32_t)a.oct_tiles;
    uint32_t* __restrict__ y = a.ycol;
    unsigned long long scanned = 0;

    // the warp's first two tiles stream in while the staging copy runs
    OctTile cur, nxt;
    if (gwarp < ntiles) oct_load(a, gwarp, lane, cur);
    if (gwarp + nwarps < ntiles) oct_load(a, gwarp + nwarps, lane, nxt);
    __syncthreads();  // the barrier is initialised before anyone waits on it
    bool staged = hot > 0 && mbar_wait_bounded(&s_bar, 0u);
    staged = __syncthreads_and(staged) != 0;
    if (!staged && hot > 0 && threadIdx.x == 0) atomicAdd(&cd->c.stage_timeouts, 1u);
    const int32_t hlim = staged ? hot : 0;  // without the staged block every message is gathered
    uint32_t mv[kOctet];
    if (gwarp < ntiles) oct_gather<LIST>(a, msgc, s_hot, hlim, llen, cur, mv);

    for (uint32_t k = gwarp; k < ntiles; k += nwarps) {
        // the lane's candidates msg[u] + w(u, v), all of one column (padding slots,
        // q >= the octet's real count, masked out)
        const uint32_t meta = cur.meta;
        const uint32_t real = meta & 0xFu;
        uint32_t R = kInf;
#pragma unroll
        for (int q = 0; q < kOctet; ++q) {
            // msg + w saturating at infinity: with n <= 2^24 and weights below
            // 256 no finite sum reaches 2^32 - 1, so only infinity wraps, and
            // the max keeps it
            const uint32_t c = max(mv[q], mv[q] + (cur.w[q] & 0xFFu));
            R = min(R, (uint32_t)q < real ? c : kInf);
        }
        const int32_t c0 = cur.c0;
        // pipeline: gather tile k+1's messages, stream tile k+2's in-edges
        const uint32_t k1 = k + nwarps, k2 = k1 + nwarps;
        if (k1 < ntiles) oct_gather<LIST>(a, msgc, s_hot, hlim, llen, nxt, mv);
        cur = nxt;
        if (k2 < ntiles) oct_load(a, k2, lane, nxt);
        scanned += meta & 0xFu;

        // lanes holding a column's first octet start a segment
        const uint32_t heads = __ballot_sync(kFull, (meta & 0x80u) != 0u);
        if ((heads & ~1u) == 0u) {  // the whole tile lies in one column (warp-uniform)
            const uint32_t Rt = __reduce_min_sync(kFull, R);
            if (lane == 0 && Rt != kInf) atomicMin(&y[c0], Rt);
            continue;
        }
        const uint32_t le = heads & lane_le;
        const int seg0 = le ? 31 - __clz(le) : -1;  // -1: the column began before this tile
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t Ru = __shfl_up_sync(kFull, R, o);
            if (lane - o >= max(seg0, 0)) R = min(R, Ru);
        }
        // the segment's last lane holds its minimum
        const bool last = lane == 31 || ((heads >> (lane + 1)) & 1u);
        if (last && R != kInf) {
            const int32_t col = c0 + __popc(le & ~1u);
            if (lane < 31 && seg0 >= 0) y[col] = R;  // the whole column lies in this tile
            else atomicMin(&y[col], R);
        }
    }
    scanned = warp_sum_u64(scanned);
    if (lane == 0 && scanned) atomicAdd(&cd->c.scanned_edges, scanned);
    if (!staged && hot > 0) mbar_wait_bounded(&s_bar, 0u);  // let a late copy land before the CTA exits
}

// Next-frontier bits of one warp's 32 columns (vertex v per lane, ascending across
// lanes; lanes past the last column carry v = INT32_MAX): lanes sharing a bitvector
// word are adjacent, so a segmented OR-scan leaves one atomic per word.  Warp-collective.
__device__ __forceinline__ void warp_set_bits(uint32_t* bv, int32_t v, bool want) {
    const int lane = threadIdx.x & 31;
    const int32_t wd = v >> 5;
    const int32_t wd_prev = __shfl_up_sync(kFull, wd, 1);
    uint32_t R = want ? 1u << (v & 31) : 0u;
    uint32_t f = (lane == 0 || wd_prev != wd) ? 1u : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t Ru = __shfl_up_sync(kFull, R, o);
        const uint32_t fu = __shfl_up_sync(kFull, f, o);
        if (lane >= o && !f) R |= Ru;
        if (lane >= o) f |= fu;
    }
    const int32_t wd_next = __shfl_down_sync(kFull, wd, 1);
    if (R != 0u && (lane == 31 || wd_next != wd)) atomicOr(&bv[wd], R);
}

constexpr int kBuShort = 8;      // in-edges a lane checks alone before its warp helps
constexpr int kColsPerLane = 4;  // columns a lane handles per step in the SSSP apply kernel
constexpr int kBuCols = 2;       // the same in the bottom-up BFS pull (more state per column)

// BFS pull superstep in one kernel: the bottom-up search and Apply.  A column is
// owned by one lane, so the depth is written and the vertex queued directly.
template <bool LIST>
__global__ void __launch_bounds__(kThreads, 4) trav_pull_bu(TravArgs a) {
    TravCtlDev* cd = a.ctl;
    if (cd->c.done || cd->c.dir != 1u) return;
    const uint32_t t = cd->c.iter;
    const int cur = (int)(t % 3u), nxt = (int)((t + 1u) % 3u), clr = (int)((t + 2u) % 3u);
    const uint32_t llen = LIST ? cd->c.list_len : 0u;
    relax_prologue<false>(a, &cd->c, t, clr);
    __shared__ WarpQ s_q[kWarps];
    __shared__ unsigned long long s_stat[6];
    if (threadIdx.x < 6) s_stat[threadIdx.x] = 0ull;
    if ((threadIdx.x & 31) < 2) s_q[threadIdx.x >> 5].n[threadIdx.x & 31] = 0u;
    __syncthreads();
    Acc acc = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, &s_q[threadIdx.x >> 5]};
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    const uint32_t* __restrict__ bvc = a.bv[cur];
    const int32_t* __restrict__ row = a.row;
    constexpr int kSpan = 32 * kBuCols;
    // kBuCols columns per lane (32 apart, so each group is coalesced and
    // ascending across the warp), their loads issued together
    for (int64_t base = gwarp * kSpan; base < a.dc_ncols; base += nwarps * kSpan) {
        int32_t v[kBuCols], p[kBuCols], end[kBuCols];
        uint32_t dv[kBuCols];
#pragma unroll
        for (int k = 0; k < kBuCols; ++k) {
            const int64_t c = base + 32 * k + lane;
            v[k] = c < a.dc_ncols ? __ldg(a.dc_jc + c) : 0x7fffffff;  // past the last column: a word of its own
        }
#pragma unroll
        for (int k = 0; k < kBuCols; ++k) dv[k] = v[k] != 0x7fffffff ? a.dist[v[k]] : 0u;
        // for unvisited columns: the in-edge range, and the degree data the enqueue needs
        uint32_t vb[kEPT] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u}, vd[kEPT] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        uint32_t vin[kEPT] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < kBuCols; ++k) {
            p[k] = end[k] = 0;
            if (dv[k] == kInf) {
                const int64_t c = base + 32 * k + lane;
                p[k] = __ldg(a.dc_cp + c);
                end[k] = __ldg(a.dc_cp + c + 1);
                vb[k] = __ldg(a.out_bin + v[k]);
                vd[k] = (uint32_t)__ldg(a.out_deg + v[k]);
                vin[k] = (uint32_t)(end[k] - p[k]);  // the in-degree: the column's in-edges
                acc.verts++;
            }
        }
        // each lane alone: up to kBuShort in-edges per column, in rounds of four
        // edges of every column (independent loads)
        bool found[kBuCols];
#pragma unroll
        for (int k = 0; k < kBuCols; ++k) found[k] = false;
#pragma unroll
        for (int rnd = 0; rnd < kBuShort / 4; ++rnd) {
            int32_t u[kBuCols][4];
#pragma unroll
            for (int k = 0; k < kBuCols; ++k)
#pragma unroll
                for (int j = 0; j < 4; ++j) u[k][j] = (!found[k] && p[k] + j < end[k]) ? __ldg(row + p[k] + j) : -1;
#pragma unroll
            for (int k = 0; k < kBuCols; ++k) {
                const int32_t nn = found[k] ? 0 : min(4, end[k] - p[k]);  // edges loaded this round
                if (nn > 0) {
                    acc.scanned += (unsigned)nn;
                    p[k] += nn;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) found[k] |= u[k][j] >= 0 && in_frontier<LIST>(a, bvc, llen, u[k][j]);
            }
        }
        // the rest of long unvisited columns, one column at a time by the whole warp
#pragma unroll
        for (int k = 0; k < kBuCols; ++k) {
            uint32_t rest = __ballot_sync(kFull, !found[k] && p[k] < end[k]);
            while (rest) {
                const int L = __ffs(rest) - 1;
                rest &= rest - 1u;
                const int32_t pb = __shfl_sync(kFull, p[k], L), pe = __shfl_sync(kFull, end[k], L);
                bool hit = false;
                for (int32_t q0 = pb; q0 < pe && !hit; q0 += 128) {
                    bool h = false;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int32_t q = q0 + j * 32 + lane;
                        if (q < pe) {
                            h |= in_frontier<LIST>(a, bvc, llen, __ldg(row + q));
                            acc.scanned++;
                        }
                    }
                    hit = __any_sync(kFull, h);
                }
                if (lane == L) found[k] = hit;
            }
        }
        bool wa[kEPT] = {false, false, false, false, false, false, false, false};
        int32_t va[kEPT] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < kBuCols; ++k) {
            if (found[k]) a.dist[v[k]] = t + 1u;
            warp_set_bits(a.bv[nxt], v[k], found[k]);
            wa[k] = found[k];
            va[k] = found[k] ? v[k] : 0;
        }
        enqueue_batch_pre<true>(a, wa, va, vb, vd, vin, nxt, acc);
    }
    flush_acc(a, acc, nxt, true, s_stat);
}

// SSSP Apply after trav_pull_a (run by the SSSP finalize kernel in a pull
// superstep): four columns per lane per step (independent loads in flight),
// coalesced across the warp for each of the four.  CTA-collective.
__device__ __forceinline__ void pull_apply(const TravArgs& a, uint32_t t, WarpQ* s_q, unsigned long long* s_stat) {
    const int nxt = (int)((t + 1u) % 3u);
    if (threadIdx.x < 6) s_stat[threadIdx.x] = 0ull;
    if ((threadIdx.x & 31) < 2) s_q[threadIdx.x >> 5].n[threadIdx.x & 31] = 0u;
    __syncthreads();
    Acc acc = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, &s_q[threadIdx.x >> 5]};
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    uint32_t* __restrict__ y = a.ycol;
    uint32_t* __restrict__ msgn = a.msg[(t + 1u) & 1u];
    constexpr int kSpan = 32 * kColsPerLane;
    // column data of a step: reduced value, vertex and source rank (independent
    // loads); the next step's are loaded while this step's vertices are read
    uint32_t b[kColsPerLane];
    int32_t v[kColsPerLane], rk[kColsPerLane];
    auto load_cols = [&](int64_t base) {
#pragma unroll
        for (int k = 0; k < kColsPerLane; ++k) {
            const int64_t c = base + 32 * k + lane;
            const bool in = c < a.dc_ncols;
            b[k] = in ? y[c] : kInf;
            v[k] = in ? __ldg(a.dc_jc + c) : 0x7fffffff;
            rk[k] = in ? __ldg(a.dc_rank + c) : 0;
        }
    };
    int64_t base = gwarp * kSpan;
    if (base < a.dc_ncols) load_cols(base);
    for (; base < a.dc_ncols; base += nwarps * kSpan) {
        uint32_t dv[kColsPerLane];
        // the out-degree the enqueue needs is loaded together with the property
        uint32_t vb[kEPT] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u}, vd[kEPT] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        const uint32_t vin[kEPT] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < kColsPerLane; ++k) {
            dv[k] = b[k] != kInf ? a.dist[v[k]] : 0u;
            vd[k] = b[k] != kInf ? (uint32_t)__ldg(a.out_deg + v[k]) : 0u;
        }
        bool wa[kEPT] = {false, false, false, false, false, false, false, false};
        int32_t va[kEPT] = {0, 0, 0, 0, 0, 0, 0, 0};
        uint32_t bc[kColsPerLane];
        int32_t rc[kColsPerLane], vc[kColsPerLane];
#pragma unroll
        for (int k = 0; k < kColsPerLane; ++k) {
            bc[k] = b[k];
            rc[k] = rk[k];
            vc[k] = v[k];
        }
        const int64_t next = base + nwarps * kSpan;
        if (next < a.dc_ncols) load_cols(next);
#pragma unroll
        for (int k = 0; k < kColsPerLane; ++k) {
            if (bc[k] != kInf) {
                y[base + 32 * k + lane] = kInf;
                acc.verts++;
                if (bc[k] < dv[k]) {
                    if (dv[k] == kInf) acc.reached += vd[k];
                    a.dist[vc[k]] = bc[k];
                    msgn[rc[k]] = bc[k];  // superstep t+1's message (finalize skips pulls)
                    wa[k] = true;
                    va[k] = vc[k];
                    vb[k] = out_bin_of(a, vd[k]);
                }
            }
        }
        // (no frontier bits: an SSSP superstep reads its frontier from the queues
        // and the message array, never from the bitvector)
        enqueue_batch_pre<false>(a, wa, va, vb, vd, vin, nxt, acc);
    }
    flush_acc(a, acc, nxt, false, s_stat);
}

// The push launch of a pull superstep (which has no push work) writes the 16-bit
// copy of the hot messages that the octet pull stages, as signed 16-bit values:
// -1 (0xFFFF) for infinity, which a signed read widens to 0xFFFFFFFF, and the
// distance itself below 0x7FFF.  A finite distance of 0x7FFF or more cannot be
// held; then stage16_off is set to t + 1 and that pull stages nothing (every
// message comes from global memory, results unchanged).  Kept out of line so
// that the push's own register allocation does not carry it.
__device__ __noinline__ void pack_stage16(const TravArgs& a, TravCtl* c, uint32_t t) {
    const uint4* m4 = reinterpret_cast<const uint4*>(a.msg[t & 1u]);
    uint2* o2 = reinterpret_cast<uint2*>(a.msg16);
    bool wide = false;
    auto enc = [&wide](uint32_t x) {
        wide |= x != kInf && x >= 0x7FFFu;
        return x == kInf ? 0xFFFFu : min(x, 0x7FFEu);
    };
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.hot16 / 4; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 m = m4[i];
        o2[i] = make_uint2(enc(m.x) | (enc(m.y) << 16), enc(m.z) | (enc(m.w) << 16));
    }
    if (wide) c->stage16_off = t + 1u;
}

// Occupancy: the push waits on chains of dependent loads (ending in an atomic
// minimum for SSSP), so more resident warps pay.  SSSP at most 64 registers,
// four CTAs per SM (RMAT-22: 28.5 -> 25.7 us per launch against three at 80, a
// few spilled words included); BFS at most 80, three CTAs (two at its natural
// 96; 16 BFS queries 5.25 -> 5.16 ms).
template <bool SSSP>
__global__ void __launch_bounds__(kThreads, SSSP ? 4 : 3) trav_push(TravArgs a) {

    TravCtlDev* cd = a.ctl;
    if (cd->c.done) return;
    if (cd->c.dir != 0u) {
        if (SSSP && a.hot16 > 0) pack_stage16(a, &cd->c, cd->c.iter);
        return;
    }
    const uint32_t t = cd->c.iter;
    const int cur = (int)(t % 3u), nxt = (int)((t + 1u) % 3u), clr = (int)((t + 2u) % 3u);
    relax_prologue<SSSP>(a, &cd->c, t, clr);
    __shared__ uint32_t s_w[kWarps][100];
    __shared__ WarpQ s_q[kWarps];
    __shared__ unsigned long long s_stat[6];
    if (threadIdx.x < 6) s_stat[threadIdx.x] = 0ull;
    if ((threadIdx.x & 31) < 2) s_q[threadIdx.x >> 5].n[threadIdx.x & 31] = 0u;
    __syncthreads();
    Acc acc = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, &s_q[threadIdx.x >> 5]};
    push_phase<SSSP>(a, t, cur, nxt, acc, s_w[threadIdx.x >> 5]);
    flush_acc(a, acc, nxt, !SSSP, s_stat);
}

// End of superstep t (one thread, once every relax of the superstep is
// complete): counts the next frontier (cnt[b] = its vertices of out-degree bin
// b), stops at convergence, max_iters or the guard, picks push or pull for
// superstep t+1 and clears the counters of the slot superstep t+2 fills.  The
// control block is accessed through volatile so that values other threads of
// the same kernel wrote with atomics are read from L2.  Returns done.
template <bool SSSP>
__device__ uint32_t finish_superstep(const TravArgs& a, TravCtlDev* cdp, uint32_t t, const uint32_t* cnt) {
    volatile TravCtlDev* cd = cdp;
    volatile TravCtl* c = &cd->c;
    const int nxt = (int)((t + 1u) % 3u);
    const unsigned long long active = (unsigned long long)cnt[0] + cnt[1] + cnt[2] + cnt[3];
    const uint32_t iters = t + 1u;
    if (c->dir == 0) c->pushes = c->pushes + 1u;
    else c->pulls = c->pulls + 1u;
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
    return done;
}

// Last kernel of a superstep.  SSSP: after a pull, Apply (pull_apply); after a
// push, the messages of superstep t+1.  Then each CTA takes a ticket and the
// last one applies the end-of-superstep rule to the next frontier's counts.
template <bool SSSP>
__global__ void __launch_bounds__(kThreads, 4) trav_finalize(TravArgs a) {
    TravCtlDev* cd = a.ctl;
    TravCtl* c = &cd->c;
    __shared__ uint32_t s_t, s_done, s_last, s_dir;
    __shared__ uint32_t s_cnt[4];
    __shared__ WarpQ s_q[SSSP ? kWarps : 1];
    __shared__ unsigned long long s_stat[6];
    if (threadIdx.x == 0) {
        s_t = c->iter;
        s_done = c->done;
        s_dir = c->dir;
    }
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = c->count[(c->iter + 1u) % 3u][threadIdx.x];
    __syncthreads();
    if (s_done) return;
    const uint32_t t = s_t;
    const int nxt = (int)((t + 1u) % 3u);
    if (SSSP && s_dir == 1u) {
        pull_apply(a, t, s_q, s_stat);
    } else if (SSSP) {  // messages of superstep t+1 after a push (pull_apply writes its own)
        const uint32_t n1 = s_cnt[1], n2 = s_cnt[2], n3 = s_cnt[3];
        uint32_t* ms = a.msg[(t + 1u) & 1u];
        for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < (int64_t)n1 + n2 + n3;
             i += (int64_t)gridDim.x * kThreads) {
            int32_t v;
            if (i < n1) v = a.q[nxt][1][i];
            else if (i < (int64_t)n1 + n2) v = a.q[nxt][2][i - n1];
            else {
                const int2 it = a.qc[nxt][i - n1 - n2];
                if (it.y != 0) continue;
                v = it.x;
            }
            ms[a.rank[v]] = a.dist[v];
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
    if (SSSP && s_dir == 1u) {  // counted by pull_apply in this kernel: read them from L2
        volatile uint32_t* vc = c->count[nxt];
        for (int b = 0; b < 4; ++b) s_cnt[b] = vc[b];
    }
    const uint32_t done = finish_superstep<SSSP>(a, cd, t, s_cnt);
    if (a.use_cond) cudaGraphSetConditional(a.cond, done ? 0u : 1u);
}

// ---------------------------------------------------------------- small supersteps
// Supersteps whose frontier is tiny cost little work but a full superstep's
// launches (push, pull, finalize, each with hundreds of CTAs, plus the loop's
// own overhead).  trav_small, the first node of every loop iteration, runs such
// supersteps itself, one after another, in one CTA: while the next superstep is
// a push over at most kSmallItems work items and kSmallEdges out-edges, it does
// exactly what push + finalize would (same relaxation, same queues, counters,
// bitvectors and messages, same termination and direction rule), then returns
// and the other nodes run the first superstep it did not take (or nothing, once
// done).  All reads of data this kernel itself changed go to L2 (ld.global.cg
// or volatile), since the SM's L1 is not coherent with atomics.
constexpr int kSmallThreads = 1024;
constexpr uint32_t kSmallItems = 2 * kSmallThreads;  // frontier vertices / large-vertex chunks
constexpr uint32_t kSmallEdges = 16384;              // frontier out-edges
constexpr uint32_t kSmallClear = 65536;              // SSSP: messages of the previous frontier to clear
constexpr uint32_t kSmallList = 2048;                // vertices whose frontier bit a superstep set, kept to clear
constexpr int64_t kSmallFullClearWords = 1 << 19;    // largest bitvector the CTA clears whole (2 MB)

template <bool SSSP>
__global__ void __launch_bounds__(kSmallThreads, 1) trav_small(TravArgs a) {
    __shared__ uint32_t s_ex[kSmallItems + 1];  // exclusive prefix of the items' edge counts
    __shared__ int32_t s_beg[kSmallItems];      // first out-edge of each item
    __shared__ uint32_t s_du[kSmallItems];      // SSSP: message of each item's vertex
    // vertices whose bit in bv[slot] superstep t set, by t's parity (superstep
    // t+2 clears exactly those words); a count above kSmallList: not known
    __shared__ int32_t s_list[2][kSmallList];
    __shared__ uint32_t s_nlist[2];
    __shared__ uint32_t s_wsum[kSmallThreads / 32];
    __shared__ unsigned long long s_stat[6];
    __shared__ uint32_t s_go, s_t, s_total, s_cnt[4];
    TravCtlDev* cd = a.ctl;
    TravCtl* c = &cd->c;
    volatile TravCtl* vc = c;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        vc->loops = vc->loops + 1u;
        s_nlist[0] = s_nlist[1] = kSmallList + 1u;  // bits set by the launches before: clear whole
    }
    for (;;) {
        if (tid == 0) {
            uint32_t go = 0u;
            const uint32_t t = vc->iter;
            if (!vc->done && vc->dir == 0u) {
                const int cur = (int)(t % 3u), clr = (int)((t + 2u) % 3u);
                const uint32_t items = vc->count[cur][1] + vc->count[cur][2] + vc->count[cur][3];
                const uint32_t prev = vc->count[clr][1] + vc->count[clr][2] + vc->count[clr][3];
                const bool listed = s_nlist[t & 1u] <= kSmallList;
                go = (items <= kSmallItems && vc->medges[cur] <= (unsigned long long)kSmallEdges &&
                      (!SSSP || prev <= kSmallClear) && (listed || a.nwords <= kSmallFullClearWords))
                         ? 1u
                         : 0u;
            }
            s_go = go;
            s_t = t;
        }
        if (tid < 6) s_stat[tid] = 0ull;
        __syncthreads();
        if (!s_go) return;
        const uint32_t t = s_t;
        const int cur = (int)(t % 3u), nxt = (int)((t + 1u) % 3u), clr = (int)((t + 2u) % 3u);
        const uint32_t par = t & 1u;

        // ---- the relax prologue: clear the frontier bits superstep t-2 set and
        // (SSSP) the messages of superstep t-1
        uint32_t* bz = a.bv[clr];
        const uint32_t nl = s_nlist[par];
        if (nl <= kSmallList) {
            for (uint32_t i = tid; i < nl; i += kSmallThreads) bz[s_list[par][i] >> 5] = 0u;
        } else {
            const int64_t n4 = a.nwords >> 2;
            for (int64_t i = tid; i < n4; i += kSmallThreads) reinterpret_cast<uint4*>(bz)[i] = make_uint4(0, 0, 0, 0);
            for (int64_t i = (n4 << 2) + tid; i < a.nwords; i += kSmallThreads) bz[i] = 0u;
        }
        if (SSSP) {
            const uint32_t p1 = __ldcg(&c->count[clr][1]), p2 = __ldcg(&c->count[clr][2]),
                           p3 = __ldcg(&c->count[clr][3]);
            uint32_t* mz = a.msg[(t + 1u) & 1u];
            for (uint32_t i = tid; i < p1 + p2 + p3; i += kSmallThreads) {
                int32_t v;
                if (i < p1) v = __ldcg(a.q[clr][1] + i);
                else if (i < p1 + p2) v = __ldcg(a.q[clr][2] + (i - p1));
                else v = __ldcg(&a.qc[clr][i - p1 - p2].x);
                mz[a.rank[v]] = kInf;
            }
        }

        // ---- the frontier's work items, their edge ranges and messages
        const uint32_t n1 = __ldcg(&c->count[cur][1]), n2 = __ldcg(&c->count[cur][2]),
                       n3 = __ldcg(&c->count[cur][3]);
        const uint32_t ni = n1 + n2 + n3;
        const uint32_t* __restrict__ msgc = a.msg[t & 1u];
        Acc acc = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, nullptr};
        uint32_t d2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t i = 2u * (uint32_t)tid + (uint32_t)h;
            d2[h] = 0u;
            if (i < ni) {
                int32_t u, beg, end;
                if (i < n1 + n2) {
                    u = i < n1 ? __ldcg(a.q[cur][1] + i) : __ldcg(a.q[cur][2] + (i - n1));
                    beg = a.row_ptr[u];
                    end = a.row_ptr[u + 1];
                    acc.verts++;
                } else {
                    const int2 it = __ldcg(&a.qc[cur][i - n1 - n2]);
                    u = it.x;
                    beg = a.row_ptr[u] + it.y * kChunk;
                    end = min(a.row_ptr[u + 1], beg + kChunk);
                    if (it.y == 0) acc.verts++;
                }
                s_beg[i] = beg;
                s_du[i] = SSSP ? __ldcg(msgc + a.rank[u]) : 0u;
                d2[h] = (uint32_t)(end - beg);
            }
        }
        // exclusive scan of the edge counts over the items (two per thread)
        const uint32_t x = d2[0] + d2[1];
        const uint32_t incl = warp_incl_scan(x);
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const uint32_t w = s_wsum[lane];
            s_wsum[lane] = warp_incl_scan(w) - w;
        }
        __syncthreads();
        const uint32_t ex = s_wsum[wid] + incl - x;
        if (2u * tid < ni) s_ex[2 * tid] = ex;
        if (2u * tid + 1u < ni) s_ex[2 * tid + 1] = ex + d2[0];
        if (tid == kSmallThreads - 1) {
            s_total = ex + x;
            s_ex[ni] = ex + x;
        }
        if (tid == 0) s_nlist[par] = 0u;
        __syncthreads();

        // ---- relax: 8 consecutive edges per thread, as push_phase does
        const uint32_t total = s_total;
        for (uint32_t base = 0; base < total; base += kSmallThreads * kEPT) {
            const uint32_t j0 = base + (uint32_t)tid * kEPT;
            int32_t v[kEPT];
            uint32_t wt[kEPT], du[kEPT];
            uint32_t ok = 0u;
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                v[k] = 0;
                wt[k] = 0u;
                du[k] = 0u;
            }
            if (j0 < total) {
                int32_t lo = 0, hi = (int32_t)ni - 1;  // the item holding edge j0: last with s_ex <= j0
                while (lo < hi) {
                    const int32_t mid = (lo + hi + 1) >> 1;
                    if (s_ex[mid] <= j0) lo = mid;
                    else hi = mid - 1;
                }
                int32_t o = lo;
#pragma unroll
                for (int k = 0; k < kEPT; ++k) {
                    const uint32_t j = j0 + (uint32_t)k;
                    if (j < total) {
                        while (j >= s_ex[o + 1]) ++o;
                        const int32_t e = s_beg[o] + (int32_t)(j - s_ex[o]);
                        v[k] = a.col[e];
                        if (SSSP) wt[k] = a.w[e];
                        du[k] = s_du[o];
                        ok |= 1u << k;
                    }
                }
            }
            bool want[kEPT];
            push_relax8<SSSP>(a, v, wt, du, ok, t, nxt, want, acc);
            acc.scanned += (unsigned)__popc(ok);
#pragma unroll
            for (int k = 0; k < kEPT; ++k)
                if (want[k]) {
                    const uint32_t pos = atomicAdd(&s_nlist[par], 1u);
                    if (pos < kSmallList) s_list[par][pos] = v[k];
                }
            enqueue_batch<!SSSP>(a, want, v, nxt, acc);
        }
        flush_acc(a, acc, nxt, !SSSP, s_stat);
        __syncthreads();

        // ---- finalize: messages of superstep t+1, then termination and direction
        if (tid < 4) s_cnt[tid] = __ldcg(&c->count[nxt][tid]);
        __syncthreads();
        if (SSSP) {
            const uint32_t m1 = s_cnt[1], m2 = s_cnt[2], m3 = s_cnt[3];
            uint32_t* ms = a.msg[(t + 1u) & 1u];
            for (uint32_t i = tid; i < m1 + m2 + m3; i += kSmallThreads) {
                int32_t v;
                if (i < m1) v = __ldcg(a.q[nxt][1] + i);
                else if (i < m1 + m2) v = __ldcg(a.q[nxt][2] + (i - m1));
                else {
                    const int2 it = __ldcg(&a.qc[nxt][i - m1 - m2]);
                    if (it.y != 0) continue;
                    v = it.x;
                }
                ms[a.rank[v]] = __ldcg(a.dist + v);
            }
        }
        if (tid == 0) {
            __threadfence();  // this thread's statistics atomics land before the counters are read
            const uint32_t done = finish_superstep<SSSP>(a, cd, t, s_cnt);
            if (done && a.use_cond) cudaGraphSetConditional(a.cond, 0u);
        }
        __syncthreads();
    }
}

// Run parameters of the control block; `fresh` also sets the start-of-run
// fields (the direction of superstep 0 and the unvisited in-edge count).
__global__ void ctl_params(TravCtlDev* cd, int32_t max_iters, int32_t dir_mode, float alpha, float beta,
                           float sssp_frac, unsigned long long m, int fresh) {
    cd->max_iters = max_iters;
    cd->dir_mode = dir_mode;
    cd->alpha = alpha;
    cd->beta = beta;
    cd->sssp_frac = sssp_frac;
    if (fresh) cd->c.unvisited_in_edges = m;
    if (cd->c.iter == 0u) cd->c.dir = dir_mode == 2 ? 1u : 0u;
}

// ---------------------------------------------------------------- frontier set-up
__global__ void seed_frontier(TravArgs a, const int32_t* __restrict__ verts, int64_t count, int bfs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool want = false;
    int32_t v = 0;
    uint32_t first = 0u;  // out-degree of a source reached here for the first time
    if (i < count) v = verts[i];
    if (i < count && (v < 0 || v >= a.n)) {
        atomicAdd(&a.ctl->c.bad_ids, 1u);
        v = 0;
    } else if (i < count) {
        if (atomicExch(&a.dist[v], 0u) == kInf) first = (uint32_t)a.out_deg[v];
        if (!bfs) a.msg[0][a.rank[v]] = 0u;
        const uint32_t bit = 1u << (v & 31);
        want = (atomicOr(&a.bv[0][v >> 5], bit) & bit) == 0u;
    }
    Acc acc = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, nullptr};
    bool wa[kEPT] = {want, false, false, false, false, false, false, false};
    int32_t va[kEPT] = {v, 0, 0, 0, 0, 0, 0, 0};
    if (bfs) enqueue_batch<true>(a, wa, va, 0, acc);
    else enqueue_batch<false>(a, wa, va, 0, acc);
    acc.medges = warp_sum_u64(acc.medges);
    acc.unvis = warp_sum_u64(acc.unvis);
    const unsigned long long reached = warp_sum_u64(first);
    if ((threadIdx.x & 31) == 0) {
        if (acc.medges) atomicAdd(&a.ctl->c.medges[0], acc.medges);
        if (bfs && acc.unvis) atomicAdd(&a.ctl->c.unvisited_in_edges, 0ull - acc.unvis);
        if (reached) atomicAdd(&a.ctl->c.reached, reached);
    }
}

__global__ void seed_all(TravArgs a, int bfs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool want = i < a.n;
    const int32_t v = want ? (int32_t)i : 0;
    uint32_t first = 0u;
    if (want) {
        if (atomicExch(&a.dist[v], 0u) == kInf) first = (uint32_t)a.out_deg[v];
        if (!bfs) a.msg[0][a.rank[v]] = 0u;
        atomicOr(&a.bv[0][v >> 5], 1u << (v & 31));
    }
    Acc acc = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, nullptr};
    bool wa[kEPT] = {want, false, false, false, false, false, false, false};
    int32_t va[kEPT] = {v, 0, 0, 0, 0, 0, 0, 0};
    if (bfs) enqueue_batch<true>(a, wa, va, 0, acc);
    else enqueue_batch<false>(a, wa, va, 0, acc);
    acc.medges = warp_sum_u64(acc.medges);
    acc.unvis = warp_sum_u64(acc.unvis);
    const unsigned long long reached = warp_sum_u64(first);
    if ((threadIdx.x & 31) == 0) {
        if (acc.medges) atomicAdd(&a.ctl->c.medges[0], acc.medges);
        if (bfs && acc.unvis) atomicAdd(&a.ctl->c.unvisited_in_edges, 0ull - acc.unvis);
        if (reached) atomicAdd(&a.ctl->c.reached, reached);
    }
}

// The frontier's reset state in one launch: the three bitvectors clear, (SSSP)
// both message arrays infinity, and a fresh control block holding the run
// parameters (the superstep-0 direction from dir_mode).  Arrays start 256-byte
// aligned: 16-byte stores, then the tail.
__global__ void reset_kernel(TravCtlDev* cd, uint32_t* bv0, uint32_t* bv1, uint32_t* bv2, int64_t nwords,
                             uint32_t* m0, uint32_t* m1, int64_t n, int32_t dir_mode, float alpha, float beta,
                             float sssp_frac, unsigned long long m) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u), f = make_uint4(kInf, kInf, kInf, kInf);
    for (int64_t i = tid; i < nwords >> 2; i += stride) {
        reinterpret_cast<uint4*>(bv0)[i] = z;
        reinterpret_cast<uint4*>(bv1)[i] = z;
        reinterpret_cast<uint4*>(bv2)[i] = z;
    }
    for (int64_t i = ((nwords >> 2) << 2) + tid; i < nwords; i += stride) bv0[i] = bv1[i] = bv2[i] = 0u;
    if (m0) {
        for (int64_t i = tid; i < n >> 2; i += stride) {
            reinterpret_cast<uint4*>(m0)[i] = f;
            reinterpret_cast<uint4*>(m1)[i] = f;
        }
        for (int64_t i = ((n >> 2) << 2) + tid; i < n; i += stride) m0[i] = m1[i] = kInf;
    }
    if (tid == 0) {
        TravCtlDev c = {};
        c.max_iters = -1;
        c.dir_mode = dir_mode;
        c.alpha = alpha;
        c.beta = beta;
        c.sssp_frac = sssp_frac;
        c.c.unvisited_in_edges = m;
        c.c.dir = dir_mode == 2 ? 1u : 0u;
        *cd = c;
    }
}

__global__ void fill_u32(uint32_t* p, int64_t n, uint32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// Sum of out-degrees of reached vertices; 16-byte loads of both arrays (both
// start 256-byte aligned), the last n % 4 vertices one by one.
__global__ void reached_kernel(const uint32_t* __restrict__ dist, const int32_t* __restrict__ out_deg, int64_t n,
                               unsigned long long* out) {
    unsigned long long s = 0;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n >> 2;
    for (int64_t i = tid; i < n4; i += stride) {
        const uint4 d = reinterpret_cast<const uint4*>(dist)[i];
        const int4 o = __ldg(reinterpret_cast<const int4*>(out_deg) + i);
        s += (d.x != kInf ? (uint32_t)o.x : 0u) + (unsigned long long)(d.y != kInf ? (uint32_t)o.y : 0u) +
             (unsigned long long)(d.z != kInf ? (uint32_t)o.z : 0u) + (unsigned long long)(d.w != kInf ? (uint32_t)o.w : 0u);
    }
    for (int64_t v = (n4 << 2) + tid; v < n; v += stride)
        if (dist[v] != kInf) s += (unsigned long long)out_deg[v];
    s = warp_sum_u64(s);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// Workspace layout inside g->work for BFS/SSSP.
struct TravWork {
    uint32_t* msg[2];
    uint32_t* lkey;
    uint32_t* lval;
    uint32_t* ltile;
    uint32_t* ycol;
    uint16_t* msg16;
    uint32_t* bv[3];
    int32_t* q[3][3];
    int2* qc[3];
};

int64_t chunk_capacity(int64_t n, int64_t m) { return n + m / kChunk + 2; }

TravWork work_layout(gm_graph* g, size_t* total_bytes = nullptr) {
    TravWork w{};
    const int64_t n = g->n > 0 ? g->n : 1;
    const int64_t nwords = (n + 31) / 32;
    char* p = static_cast<char*>(g->work.p);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* r = p ? p + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return r;
    };
    for (int s = 0; s < 2; ++s) w.msg[s] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    w.ycol = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    w.msg16 = reinterpret_cast<uint16_t*>(take(sizeof(uint16_t) * 2 * kHotMax));
    w.lkey = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    w.lval = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    w.ltile = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * ((n + kListTile - 1) / kListTile + 1)));
    for (int s = 0; s < 3; ++s) w.bv[s] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * nwords));
    for (int s = 0; s < 3; ++s) {
        w.q[s][0] = nullptr;
        for (int b = 1; b < 3; ++b) w.q[s][b] = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
        w.qc[s] = reinterpret_cast<int2*>(take(sizeof(int2) * chunk_capacity(n, g->m)));
    }
    if (total_bytes) *total_bytes = off;
    return w;
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
    a.cw8 = as<uint8_t>(g->cw8);
    a.out_deg = as<int32_t>(g->out_deg);
    a.in_deg = as<int32_t>(g->in_deg);
    a.out_bin = as<uint8_t>(g->out_bin);
    a.bin_small = g->tune.bin_small;
    a.bin_large = g->tune.bin_large;
    a.in_list = as<int32_t>(g->in_list);
    a.in_s0 = g->in_list_count[0];
    a.in_s1 = g->in_list_count[1];
    a.in_m1 = g->in_list_count[2];
    a.dc_jc = as<int32_t>(g->dc_jc);
    a.dc_cp = as<int32_t>(g->dc_cp);
    a.dc_tile = as<int32_t>(g->dc_tile);
    a.dc_ncols = g->dc_ncols;
    a.ntiles = g->dc_ntiles;
    a.n = g->n;
    a.m = g->m;
    a.nwords = (g->n + 31) / 32;
    a.dist = as<uint32_t>(g->state);
    for (int s = 0; s < 2; ++s) a.msg[s] = w.msg[s];
    a.ycol = w.ycol;
    a.lkey = w.lkey;
    a.lval = w.lval;
    a.ltile = w.ltile;
    a.dc_head = as<uint32_t>(g->dc_head);
    for (int s = 0; s < 3; ++s) {
        a.bv[s] = w.bv[s];
        for (int b = 0; b < 3; ++b) a.q[s][b] = w.q[s][b];
        a.qc[s] = w.qc[s];
    }
    a.rank = as<int32_t>(g->src_rank);
    a.row_r = as<int32_t>(g->row_r);
    a.oct_w = as<uint32_t>(g->oct_w);
    a.oct_meta = as<uint8_t>(g->oct_meta);
    a.oct_c0 = as<int32_t>(g->oct_c0);
    a.oct_tiles = g->oct_tiles;
    a.dc_rank = as<int32_t>(g->dc_rank);
    a.hot = g->src_rank.p ? (int32_t)pull_stage_messages(g) : 0;
    a.msg16 = w.msg16;
    a.hot16 = (a.oct_w && a.hot > 0) ? (int32_t)pull_stage16_messages(g) : 0;
    a.stage_extra = g->tune.test_stall_stage ? 16u : 0u;
    a.ctl = as<TravCtlDev>(g->ctl_buf);
    a.use_cond = 0;
    return a;
}

template <typename K>
int grid_for(K kernel) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
    if (per_sm <= 0) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    return per_sm * num_sms();
}

int push_grid() {
    static int blocks = grid_for(trav_push<true>);
    return blocks;
}

// trav_pull_a runs one CTA of kPullThreads per SM with up to kHotMax * 4 bytes of
// dynamic shared memory; the attribute is set once per process.
int pull_grid() {
    static int blocks = [] {
        const int bytes = (int)(kHotMax * sizeof(uint32_t));
        cudaFuncSetAttribute(trav_pull_o<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(trav_pull_a<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(trav_pull_a<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        return num_sms();
    }();
    return blocks;
}

// The SSSP pull variant for the handle's in-edge layout (and the sorted-list
// sparse vector of the ablation).
const void* pull_a_kernel(const TravArgs& a, bool list = false) {
    if (a.oct_w) return list ? (const void*)trav_pull_o<true> : (const void*)trav_pull_o<false>;
    if (list) return a.cw8 ? (const void*)trav_pull_a<1, true> : (const void*)trav_pull_a<4, true>;
    return a.cw8 ? (const void*)trav_pull_a<1, false> : (const void*)trav_pull_a<4, false>;
}

int pull_bu_grid() {
    static int blocks = grid_for(trav_pull_bu<false>);
    return blocks;
}

// SSSP's finalize applies a pull or writes the next messages after a push
// (grid-stride loops); BFS's only elects the last CTA, so one CTA is enough.
int finalize_grid(bool sssp) {
    static int blocks = grid_for(trav_finalize<true>);
    return sssp ? blocks : 1;
}

#define LAUNCH_OK()                                                                             \
    do {                                                                                        \
        cudaError_t _e = cudaGetLastError();                                                    \
        if (_e != cudaSuccess) {                                                                \
            set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(_e), __FILE__, __LINE__); \
            return GM_ERR_CUDA;                                                                 \
        }                                                                                       \
    } while (0)

// Reset the control block and the frontier before seeding.
// Host side of a frontier reset (the bookkeeping that goes with reset_kernel).
void reset_frontier_flags(gm_graph* g) {
    if (g->reached_pending) {  // seeds counted in the control block that is about to be cleared
        g->reached_valid = false;
        g->reached_pending = false;
    }
    g->frontier_clean = true;
    if (g->kind == GM_SSSP) g->msg_clean = true;
}

gm_status reset_frontier(gm_graph* g) {
    cudaStream_t s = g->stream;
    TravWork w = work_layout(g);
    const int64_t n = g->n > 0 ? g->n : 1;
    const int64_t nwords = (n + 31) / 32;
    const bool sssp = g->kind == GM_SSSP;
    reset_kernel<<<num_sms() * 4, 256, 0, s>>>(as<TravCtlDev>(g->ctl_buf), w.bv[0], w.bv[1], w.bv[2], nwords,
                                               sssp ? w.msg[0] : nullptr, sssp ? w.msg[1] : nullptr, n,
                                               g->tune.direction, (float)g->tune.alpha, (float)g->tune.beta,
                                               (float)g->tune.sssp_pull_frac, (unsigned long long)g->m);
    g_launches++;
    LAUNCH_OK();
    reset_frontier_flags(g);
    return GM_OK;
}

gm_status build_loop_graph(gm_graph* g, bool sssp) {
    const int slot = sssp ? 1 : 0;
    if (g->loop_exec[slot]) {
        cudaGraphExecDestroy(g->loop_exec[slot]);
        g->loop_exec[slot] = nullptr;
    }
    if (g->loop_graph[slot]) {
        cudaGraphDestroy(g->loop_graph[slot]);
        g->loop_graph[slot] = nullptr;
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
    // run parameters (set per run), then the loop, then the copy of the control
    // block to the host and the frontier reset for the next run
    cudaGraphNode_t pnode = nullptr;
    {
        TravCtlDev* cd = as<TravCtlDev>(g->ctl_buf);
        int32_t mi = -1, dm = g->tune.direction;
        float al = (float)g->tune.alpha, be = (float)g->tune.beta, fr = (float)g->tune.sssp_pull_frac;
        unsigned long long mm = (unsigned long long)g->m;
        int fresh = 0;
        void* pargs[] = {&cd, &mi, &dm, &al, &be, &fr, &mm, &fresh};
        cudaKernelNodeParams pp = {};
        pp.func = (void*)ctl_params;
        pp.gridDim = dim3(1);
        pp.blockDim = dim3(1);
        pp.kernelParams = pargs;
        e = cudaGraphAddKernelNode(&pnode, graph, nullptr, 0, &pp);
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, graph, &pnode, nullptr, 1, &cp);
    cudaGraphNode_t copy_node = nullptr, reset_node = nullptr;
    if (e == cudaSuccess)
        e = cudaGraphAddMemcpyNode1D(&copy_node, graph, &cnode, 1, g->host_pinned, g->ctl_buf.p, sizeof(TravCtlDev),
                                     cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        TravWork w = work_layout(g);
        TravCtlDev* cd = as<TravCtlDev>(g->ctl_buf);
        const int64_t n = g->n > 0 ? g->n : 1;
        int64_t nwords = (n + 31) / 32, nn = n;
        uint32_t* m0 = sssp ? w.msg[0] : nullptr;
        uint32_t* m1 = sssp ? w.msg[1] : nullptr;
        int32_t dm = g->tune.direction;
        float al = (float)g->tune.alpha, be = (float)g->tune.beta, fr = (float)g->tune.sssp_pull_frac;
        unsigned long long mm = (unsigned long long)g->m;
        void* rargs[] = {&cd, &w.bv[0], &w.bv[1], &w.bv[2], &nwords, &m0, &m1, &nn, &dm, &al, &be, &fr, &mm};
        cudaKernelNodeParams rp = {};
        rp.func = (void*)reset_kernel;
        rp.gridDim = dim3((unsigned)(num_sms() * 4));
        rp.blockDim = dim3(256);
        rp.kernelParams = rargs;
        e = cudaGraphAddKernelNode(&reset_node, graph, &copy_node, 1, &rp);
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("superstep loop graph: %s", cudaGetErrorString(e));
        return GM_ERR_CUDA;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    TravArgs a = make_args(g);
    a.cond = handle;
    a.use_cond = 1;
    void* kargs[] = {&a};
    cudaKernelNodeParams kp = {};
    kp.func = sssp ? (void*)trav_small<true> : (void*)trav_small<false>;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(kSmallThreads);
    kp.kernelParams = kargs;
    cudaGraphNode_t ns = nullptr, n0 = nullptr, n1 = nullptr, n2 = nullptr;
    e = cudaGraphAddKernelNode(&ns, body, nullptr, 0, &kp);
    kp.func = sssp ? (void*)trav_push<true> : (void*)trav_push<false>;
    kp.gridDim = dim3((unsigned)push_grid());
    kp.blockDim = dim3(kThreads);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n0, body, &ns, 1, &kp);
    cudaGraphNode_t n1b = nullptr;
    if (e == cudaSuccess) {
        kp.func = !sssp ? (void*)trav_pull_bu<false> : const_cast<void*>(pull_a_kernel(a));
        kp.gridDim = dim3((unsigned)(sssp ? pull_grid() : pull_bu_grid()));
        kp.blockDim = dim3(sssp ? kPullThreads : kThreads);
        kp.sharedMemBytes = sssp ? (unsigned)a.hot * 4u : 0u;
        e = cudaGraphAddKernelNode(&n1, body, &n0, 1, &kp);
        kp.blockDim = dim3(kThreads);
        kp.sharedMemBytes = 0u;
    }
    if (e == cudaSuccess) {
        n1b = n1;  // Apply: the BFS pull's own, the SSSP finalize's
    }
    if (e == cudaSuccess) {
        kp.func = sssp ? (void*)trav_finalize<true> : (void*)trav_finalize<false>;
        kp.gridDim = dim3((unsigned)finalize_grid(sssp));
        e = cudaGraphAddKernelNode(&n2, body, &n1b, 1, &kp);
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("superstep loop graph: %s", cudaGetErrorString(e));
        return GM_ERR_CUDA;
    }
    g->loop_graph[slot] = graph;
    g->loop_exec[slot] = exec;
    g->loop_params[slot] = pnode;
    return GM_OK;
}

}  // namespace

gm_status trav_prepare(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n > 0 ? g->n : 1;
    if (g->kind == GM_SSSP) GM_TRY(build_source_ranks(g));
    GM_TRY(dev_alloc(g->state, sizeof(uint32_t) * n, s));
    size_t wb = 0;
    g->work.p = nullptr;
    work_layout(g, &wb);
    GM_TRY(dev_alloc(g->work, wb, s));
    g->work_bytes = (int64_t)wb;
    g->frontier_clean = g->msg_clean = false;
    GM_TRY(dev_alloc(g->ctl_buf, sizeof(TravCtlDev), s));
    fill_u32<<<num_sms() * 4, 256, 0, s>>>(as<uint32_t>(g->state), g->n, kInf);
    g_launches++;
    LAUNCH_OK();
    // per-column pull results start at infinity; pull_apply restores that after every use
    GM_CUDA_TRY(cudaMemsetAsync(work_layout(g).ycol, 0xFF, sizeof(uint32_t) * n, s));
    GM_TRY(reset_frontier(g));
    g->reached_total = 0;  // every property is infinity
    g->reached_valid = true;
    return GM_OK;
}

// program_set between BFS and SSSP when the workspace of a traversal is already
// allocated: the buffers and the cached loop graphs stay, the properties go back
// to infinity and the frontier is reset if seeds are pending or the program
// changed (the message arrays are SSSP's alone).
gm_status trav_reuse(gm_graph* g) {
    cudaStream_t s = g->stream;
    // the SSSP loop graph needs the ranks and the pull's in-edge layout; build
    // them first (or again, after a failed rebuild of the layout)
    if (g->kind == GM_SSSP && (!g->src_rank.p || (!g->oct_w.p && !g->row_r.p))) {
        GM_TRY(build_source_ranks(g));
        trav_release(g);
    }
    fill_u32<<<num_sms() * 4, 256, 0, s>>>(as<uint32_t>(g->state), g->n, kInf);
    g_launches++;
    LAUNCH_OK();
    // gm_run leaves the frontier reset: no second reset unless seeds were set
    // since or the SSSP messages were last used (or never cleared)
    if (!g->frontier_clean || (g->kind == GM_SSSP && !g->msg_clean)) GM_TRY(reset_frontier(g));
    g->reached_total = 0;
    g->reached_valid = true;
    return GM_OK;
}

gm_status trav_set_active(gm_graph* g, const int32_t* vertices_dev, int64_t count) {
    cudaStream_t s = g->stream;
    g->frontier_clean = false;
    if (g->kind == GM_SSSP) g->msg_clean = false;
    g->reached_pending = true;  // the seeding kernel adds newly reached sources to the control block
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
    if (sssp && (!g->src_rank.p || (!g->oct_w.p && !g->row_r.p))) {
        set_error("gm_run: the SSSP pull's in-edge layout is missing (a previous call failed to build it); "
                  "call gm_program_set again");
        return GM_ERR_STATE;
    }
    g->stats = RunStats{};
    g->frontier_clean = false;
    if (sssp) g->msg_clean = false;
    if (max_iters == 0) {
        if (iters_done) *iters_done = 0;
        return reset_frontier(g);
    }
    TravCtlDev* hp = static_cast<TravCtlDev*>(g->host_pinned);
    const bool list = g->tune.sparse_list != 0;  // the ablation's sorted-list frontier: host-issued loop
    const bool host_loop = g->tune.loop_mode == 1 || g->tune.profile || list;
    if (!host_loop) {
        // one graph: the run parameters, the superstep loop, the copy of the
        // control block to hp and the frontier reset for the next run
        const int slot = sssp ? 1 : 0;
        if (!g->loop_exec[slot]) GM_TRY(build_loop_graph(g, sssp));
        TravCtlDev* cd = as<TravCtlDev>(g->ctl_buf);
        int32_t mi = max_iters, dm = g->tune.direction;
        float al = (float)g->tune.alpha, be = (float)g->tune.beta, fr = (float)g->tune.sssp_pull_frac;
        unsigned long long mm = (unsigned long long)g->m;
        int fresh = 0;
        void* pargs[] = {&cd, &mi, &dm, &al, &be, &fr, &mm, &fresh};
        cudaKernelNodeParams pp = {};
        pp.func = (void*)ctl_params;
        pp.gridDim = dim3(1);
        pp.blockDim = dim3(1);
        pp.kernelParams = pargs;
        GM_CUDA_TRY(cudaGraphExecKernelNodeSetParams(g->loop_exec[slot], g->loop_params[slot], &pp));
        GM_CUDA_TRY(cudaGraphLaunch(g->loop_exec[slot], s));
        g_launches += 2;  // parameters and reset
        g->reached_pending = false;  // seeds pending in the control block are in the copy
        reset_frontier_flags(g);
    } else {
        // parameters that may have changed since the frontier was reset
        ctl_params<<<1, 1, 0, s>>>(as<TravCtlDev>(g->ctl_buf), max_iters, g->tune.direction,
                                   (float)g->tune.alpha, (float)g->tune.beta, (float)g->tune.sssp_pull_frac,
                                   (unsigned long long)g->m, 0);
        g_launches++;
        LAUNCH_OK();
        TravArgs a = make_args(g);
        const int pg = push_grid(), lg = sssp ? pull_grid() : pull_bu_grid(), fg = finalize_grid(sssp);
        cudaEvent_t ev0 = nullptr, ev1 = nullptr, evA = nullptr, evB = nullptr;
        if (g->tune.profile) {
            GM_CUDA_TRY(cudaEventCreate(&ev0));
            GM_CUDA_TRY(cudaEventCreate(&ev1));
            GM_CUDA_TRY(cudaEventCreate(&evA));
            GM_CUDA_TRY(cudaEventCreate(&evB));
        }
        unsigned long long prev_e = 0, prev_v = 0;
        const int list_grid = num_sms() * 8;
        for (int32_t it = 0;; ++it) {
            uint32_t dir_before = 0, frontier_before = 0;
            if (ev0 || list) {  // direction and frontier size of this superstep (trace; list build)
                GM_CUDA_TRY(cudaMemcpyAsync(hp, g->ctl_buf.p, sizeof(TravCtlDev), cudaMemcpyDeviceToHost, s));
                GM_CUDA_TRY(cudaStreamSynchronize(s));
                dir_before = hp->c.dir;
                const uint32_t slot = hp->c.iter % 3u;
                frontier_before = hp->c.count[slot][0] + hp->c.count[slot][1] + hp->c.count[slot][2] +
                                  hp->c.count[slot][3];
            }
            if (ev0) cudaEventRecord(ev0, s);
            if (list && dir_before == 1u) {  // this pull superstep's frontier as a sorted list
                if (sssp) list_count<true><<<list_grid, kListThreads, 0, s>>>(a);
                else list_count<false><<<list_grid, kListThreads, 0, s>>>(a);
                list_scan<<<1, kListScanThreads, 0, s>>>(a);
                if (sssp) list_scatter<true><<<list_grid, kListThreads, 0, s>>>(a);
                else list_scatter<false><<<list_grid, kListThreads, 0, s>>>(a);
                g_launches += 3;
                LAUNCH_OK();
            }
            // both are launched; the one not matching the device-side direction returns at once
            if (sssp) trav_push<true><<<pg, kThreads, 0, s>>>(a);
            else trav_push<false><<<pg, kThreads, 0, s>>>(a);
            if (evA) cudaEventRecord(evA, s);
            if (sssp) {
                void* pargs[] = {&a};
                GM_CUDA_TRY(cudaLaunchKernel(pull_a_kernel(a, list), dim3(lg), dim3(kPullThreads), pargs,
                                             list ? 0 : (size_t)a.hot * 4u, s));
            } else if (list) {
                trav_pull_bu<true><<<lg, kThreads, 0, s>>>(a);
            } else {
                trav_pull_bu<false><<<lg, kThreads, 0, s>>>(a);
            }
            if (evB) cudaEventRecord(evB, s);
            g_launches += 2;
            LAUNCH_OK();
            if (sssp) trav_finalize<true><<<fg, kThreads, 0, s>>>(a);  // SSSP Apply runs here
            else trav_finalize<false><<<fg, kThreads, 0, s>>>(a);
            if (ev1) cudaEventRecord(ev1, s);
            g_launches++;
            LAUNCH_OK();
            GM_CUDA_TRY(cudaMemcpyAsync(&hp->c.done, &as<TravCtlDev>(g->ctl_buf)->c.done, sizeof(uint32_t),
                                        cudaMemcpyDeviceToHost, s));
            GM_CUDA_TRY(cudaStreamSynchronize(s));
            if (ev0) {
                float ms = 0.f, ms_pull = 0.f, ms_push = 0.f, ms_fin = 0.f;
                cudaEventElapsedTime(&ms, ev0, ev1);
                cudaEventElapsedTime(&ms_pull, evA, evB);
                cudaEventElapsedTime(&ms_push, ev0, evA);
                cudaEventElapsedTime(&ms_fin, evB, ev1);
                g->stats.relax_ms += ms;
                g->stats.relax_launches++;
                const uint32_t done = hp->c.done;
                GM_CUDA_TRY(cudaMemcpyAsync(hp, g->ctl_buf.p, sizeof(TravCtlDev), cudaMemcpyDeviceToHost, s));
                GM_CUDA_TRY(cudaStreamSynchronize(s));
                const double row[kTraceCols] = {(double)it, (double)dir_before, (double)frontier_before,
                                                (double)(hp->c.scanned_edges - prev_e),
                                                (double)(hp->c.processed_vertices - prev_v), (double)ms,
                                                (double)hp->c.medges[(it + 1) % 3], (double)ms_pull,
                                                (double)ms_push, (double)ms_fin};
                prev_e = hp->c.scanned_edges;
                prev_v = hp->c.processed_vertices;
                g->stats.trace.insert(g->stats.trace.end(), row, row + kTraceCols);
                hp->c.done = done;
            }
            if (hp->c.done) break;
        }
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (evA) cudaEventDestroy(evA);
        if (evB) cudaEventDestroy(evB);
    }
    if (host_loop) {
        GM_CUDA_TRY(cudaMemcpyAsync(hp, g->ctl_buf.p, sizeof(TravCtlDev), cudaMemcpyDeviceToHost, s));
        // the frontier reset for the next run goes into the stream behind that
        // copy, before the wait: seeds pending in the control block are in the copy
        g->reached_pending = false;
        GM_TRY(reset_frontier(g));
    }
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    if (!host_loop) g_launches += 4ull * hp->c.loops;
    g->stats.supersteps = (int32_t)hp->c.iters_done;
    g->stats.pushes = (int32_t)hp->c.pushes;
    g->stats.pulls = (int32_t)hp->c.pulls;
    g->stats.scanned_edges = (int64_t)hp->c.scanned_edges;
    g->stats.processed_vertices = (int64_t)hp->c.processed_vertices;
    if (iters_done) *iters_done = (int32_t)hp->c.iters_done;
    g->reached_total += (int64_t)hp->c.reached;  // seeds since the last reset and this run
    const uint32_t bad = hp->c.bad_ids;
    const uint32_t guard = hp->c.guard_hit;
    const uint32_t stage_to = hp->c.stage_timeouts;
    if (stage_to) {  // the results are still exact (those CTAs gathered every message from global memory)
        set_error("gm_run: %u pull CTAs timed out waiting for their shared-memory staging copy", stage_to);
        return GM_ERR_TIMEOUT;
    }
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
    if (g->reached_valid && !g->reached_pending) {  // kept by the traversal kernels
        *out = g->reached_total;
        return GM_OK;
    }
    if (!g->reached_buf.p) GM_TRY(dev_alloc(g->reached_buf, sizeof(unsigned long long), s));
    GM_CUDA_TRY(cudaMemsetAsync(g->reached_buf.p, 0, sizeof(unsigned long long), s));
    if (g->n > 0) {
        reached_kernel<<<num_sms() * 4, 256, 0, s>>>(as<uint32_t>(g->state), as<int32_t>(g->out_deg), g->n,
                                                     as<unsigned long long>(g->reached_buf));
        g_launches++;
        LAUNCH_OK();
    }
    unsigned long long h = 0;
    GM_CUDA_TRY(cudaMemcpyAsync(&h, g->reached_buf.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    *out = (int64_t)h;
    if (!g->reached_pending) {  // counted from the state itself: the traversal keeps it from here
        g->reached_total = (int64_t)h;
        g->reached_valid = true;
    }
    return GM_OK;
}

void trav_release(gm_graph* g) {
    for (int k = 0; k < 2; ++k) {
        if (g->loop_exec[k]) cudaGraphExecDestroy(g->loop_exec[k]);
        if (g->loop_graph[k]) cudaGraphDestroy(g->loop_graph[k]);
        g->loop_exec[k] = nullptr;
        g->loop_graph[k] = nullptr;
    }
}

}  // namespace gm
