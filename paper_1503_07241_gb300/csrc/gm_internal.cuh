// Internal declarations of the GraphMat GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <atomic>
#include <string>
#include <vector>

#include "graphmat_gb300.h"

namespace gm {

constexpr uint32_t kInf = 0xFFFFFFFFu;  // "infinite" BFS depth / SSSP distance
constexpr int kNumBins = 3;             // degree bins: small (warp-cooperative), medium (warp), large (CTA)
constexpr int kEdgePad = 16;            // per-edge arrays carry this many spare entries, so 16-byte
                                        // vector loads that start inside a row never leave the buffer
constexpr int kChunk = 2048;            // edges of one large-vertex work item (256 threads x 8 edges)
constexpr int kWTile = 256;             // in-edges of one warp tile of the pull side (32 lanes x 8 edges)
constexpr int64_t kPackedMaxVertices = 1ll << 24;  // ranks that fit the 24 bits of a packed in-edge word
constexpr int kOctet = 8;                          // slots of one octet (one lane's share of a tile)
constexpr int kOctTile = 32;                       // octets of one warp tile

// Library-wide count of kernel launches issued (a graph replay counts each
// kernel node it runs).
extern std::atomic<uint64_t> g_launches;

void set_error(const char* fmt, ...);

#define GM_CUDA_TRY(expr)                                                             \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess) {                                                      \
            ::gm::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e),    \
                            __FILE__, __LINE__);                                      \
            return _e == cudaErrorMemoryAllocation ? GM_ERR_OUT_OF_MEMORY : GM_ERR_CUDA; \
        }                                                                             \
    } while (0)

#define GM_TRY(expr)                          \
    do {                                      \
        gm_status _s = (expr);                \
        if (_s != GM_OK) return _s;           \
    } while (0)

// Device buffer owned by the library (cudaMallocAsync on the graph's stream).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

gm_status dev_alloc(DevBuf& b, size_t bytes, cudaStream_t s);
extern std::atomic<int64_t> g_alloc_budget;  // test hook of gm_debug_fail_allocations_after
void dev_free(DevBuf& b, cudaStream_t s);
template <typename T>
inline T* as(const DevBuf& b) { return static_cast<T*>(b.p); }

// ---- primitives (gm_primitives.cu) -------------------------------------------------
// Exclusive scan of n uint32 values; out[n] receives the total (out has n+1 slots).
gm_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the keys.
// keys/vals are sorted in place; the alternate buffers are scratch of the same size.
gm_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                           int64_t n, int bits, cudaStream_t s);
// Compact the indices i in [0, n) with flag[i] != 0 into out (ascending); count to *count_dev.
gm_status compact_indices(const uint32_t* flags, int64_t n, int32_t* out, uint32_t* count_dev,
                          cudaStream_t s);

int num_sms();

// ---- traversal control block (device memory) --------------------------------------
struct TravCtl {
    uint32_t iter;                // superstep index t
    uint32_t dir;                 // 0 = push (top-down over the queue), 1 = pull (bottom-up over in-edges)
    uint32_t done;                // 1 once converged or at max_iters
    uint32_t ticket;              // last-CTA election in the finalize kernel
    uint32_t count[3][4];         // active vertices per rotating slot and out-degree bin (0 = no out-edges)
    unsigned long long medges[3]; // sum of out-degrees of each slot's queue
    unsigned long long unvisited_in_edges;  // BFS: in-edges of still-unvisited vertices
    unsigned long long scanned_edges;       // edges read (statistics)
    unsigned long long processed_vertices;  // vertices whose edge list was read (statistics)
    uint32_t pushes, pulls;       // supersteps run in each direction
    uint32_t iters_done;
    uint32_t bad_ids;             // seeding saw vertex ids outside [0, n)
    uint32_t guard_hit;           // the loop passed n + 1 supersteps (impossible for valid runs)
    uint32_t stage_timeouts;      // pull CTAs whose shared-memory staging copy did not complete in time
    uint32_t loops;               // iterations of the device loop (for the launch count)
    unsigned long long reached;   // out-degrees of the vertices whose property became finite since the reset
    uint32_t list_len;            // sorted-list sparse vector: entries of the current superstep's list
    uint32_t stage16_off;         // superstep + 1 of the last pull whose staged messages did not all fit 16 bits
};

// Options and tuning knobs of a graph handle.
struct Tuning {
    int32_t bin_small = 32;     // degree < bin_small: warp-cooperative group of 32 vertices
    int32_t bin_large = 2048;   // degree >= bin_large: one CTA per vertex
    double alpha = 14.0;        // push -> pull when frontier edges > unvisited edges / alpha
    double beta = 24.0;         // pull -> push when frontier vertices < n / beta
    double sssp_pull_frac = 0.05;  // SSSP: pull when frontier edges > sssp_pull_frac * m
    int32_t pull_stage = 40960;    // SSSP pull: hottest messages staged in shared memory per CTA
    int32_t test_stall_stage = 0;  // test hook: the staging barrier waits for bytes that never come
    int32_t test_stall_sgd = 0;    // test hook: one CTA never arrives at the first SGD grid barrier
    int32_t pull_packed = 1;       // SSSP pull: rank and one-byte weight in one word per in-edge when possible
    int32_t sparse_list = 0;       // 1: pull supersteps look the frontier up in a sorted (index, value) list
    int32_t direction = 0;      // 0 auto, 1 push only, 2 pull only
    int32_t loop_mode = 0;      // 0 device loop (CUDA graph with a conditional WHILE node), 1 host loop
    int32_t profile = 0;        // 1: host loop with CUDA events around every relax launch
};

struct RunStats {
    int32_t supersteps = 0, pushes = 0, pulls = 0;
    int64_t scanned_edges = 0;
    int64_t processed_vertices = 0;
    double relax_ms = 0.0;      // profile mode: summed relax-kernel time
    int32_t relax_launches = 0;
    double finalize_ms = 0.0;
    int32_t finalize_launches = 0;
    // profile mode: one row per superstep (see gm_get_trace)
    std::vector<double> trace;
};
constexpr int kTraceCols = 10;

}  // namespace gm

// The opaque handle.
struct gm_graph {
    int64_t n = 0, m = 0, n_left = 0;
    uint32_t flags = 0;
    cudaStream_t stream = nullptr;
    int32_t wtype = GM_W_NONE;
    // CSR: out-edges sorted by (src, dst)
    gm::DevBuf row_ptr, col, w;      // w: uint32 or float per CSR edge (as wtype)
    // CSC: in-edges sorted by (dst, src)
    gm::DevBuf col_ptr, row, cw, csc_pos;  // cw: CSC copy of w; csc_pos: CSR index of each CSC edge
    gm::DevBuf cw8;                  // uint8 copy of cw when every uint32 weight is below 256 (else empty)
    // Sources ranked by out-degree (descending, ties by id), built on the first SSSP
    // program_set: the SSSP messages live in rank order so that the hottest sources'
    // messages are one contiguous prefix the pull can keep in shared memory.
    gm::DevBuf src_rank;             // rank of each vertex (int32[n])
    gm::DevBuf row_r;                // CSC sources as ranks (int32[m + pad]); empty when the octets are built
    // Octet layout of the SSSP pull's in-edges, built instead of row_r when every
    // weight fits a byte and n <= 2^24: each non-empty column's in-edges, in CSC
    // order, padded to a multiple of 8 slots, so that every octet (the 8 slots one
    // lane reads) belongs to one column; 32 octets form a warp tile.
    gm::DevBuf oct_w;                // uint32 per slot: (source rank << 8) | weight; padding slots 0;
                                     // per tile slots 0-3 of its 32 octets, then slots 4-7
    gm::DevBuf oct_meta;             // uint8 per octet: bits 0-3 real slots (1..8), bit 7 first octet of
                                     // its column; 0 for octets past the last (the tail of the last tile)
    gm::DevBuf oct_c0;               // int32 per tile: non-empty column index of the tile's first octet
    int64_t oct_tiles = 0;           // tiles of 32 octets
    int64_t oct_slots = 0;           // real + padding slots (octets x 8) before the last tile's tail
    gm::DevBuf dc_rank;              // rank of each non-empty column's vertex (int32[ncols])
    gm::DevBuf out_deg, in_deg;      // int32
    gm::DevBuf out_bin, in_bin;      // uint8 bin of each vertex by out/in degree (0 = degree zero)
    gm::DevBuf in_list;              // vertex ids with in_deg > 0, grouped by in-degree bin
    int64_t in_list_count[gm::kNumBins + 1] = {0};  // offsets of bins 1..3 inside in_list
    gm::DevBuf out_list;             // vertex ids with out_deg > 0, grouped by out-degree bin
    int64_t out_list_count[gm::kNumBins + 1] = {0};
    gm::DevBuf zero_out_list;        // vertex ids with out_deg == 0
    int64_t zero_out_count = 0;
    // Doubly compressed CSC (Section 4.3.1's DCSC): non-empty columns only, and the
    // column holding the first edge of every kWTile-edge tile of the in-edge array.
    gm::DevBuf dc_jc;                // vertex id of each non-empty column (ascending)
    gm::DevBuf dc_cp;                // in-edge offset of each non-empty column, plus m at the end
    gm::DevBuf dc_tile;              // column index holding edge k * kWTile
    gm::DevBuf dc_head;              // bit e set iff in-edge e is the first of its column (m bits)
    int64_t dc_ncols = 0, dc_ntiles = 0;
    gm::DevBuf zero_in_list;         // vertex ids with in_deg == 0
    int64_t zero_in_count = 0;
    gm::Tuning tune;
    gm::RunStats stats;
    // GM_SCALAR_REACHED_EDGES kept up to date by the traversal itself: the sum of
    // out-degrees of vertices with a finite property, valid when no change since
    // the last fold is unaccounted (seeds pending in the control block, a state
    // written by the caller)
    int64_t reached_total = 0;
    bool reached_valid = false;
    bool reached_pending = false;
    // traversal workspace already in its reset state (bitvectors clear, control
    // block fresh; msg_clean: the SSSP message arrays all infinity)
    bool frontier_clean = false;
    bool msg_clean = false;

    // program state
    int32_t kind = -1;
    gm_program_params params{};
    bool active_set = false;
    gm::DevBuf state;                // uint32 dist / float rank / uint64 count / float factors
    gm::DevBuf work;                 // program workspace (see each program)
    int64_t work_bytes = 0;
    gm::DevBuf ctl_buf;              // TravCtl
    void* host_pinned = nullptr;     // small pinned staging buffer
    // device-loop graph for traversal
    // device-loop graphs for traversal, one per program (0 BFS, 1 SSSP), kept until
    // an option that changes their launch shapes or the workspace is freed
    cudaGraph_t loop_graph[2] = {nullptr, nullptr};
    cudaGraphExec_t loop_exec[2] = {nullptr, nullptr};
    cudaGraphNode_t loop_params[2] = {nullptr, nullptr};  // the run-parameter node, set per gm_run
    gm::DevBuf reached_buf;          // counter of gm_get_scalar(GM_SCALAR_REACHED_EDGES)
    // results
    uint64_t tc_total = 0;
    void* wpr = nullptr;             // weighted-PageRank buffers (gm_wpr.cu)
    void* cf = nullptr;              // collaborative-filtering buffers (gm_cf.cu)
    void* pr = nullptr;              // PageRank's cached superstep graph (gm_pagerank.cu)
};

namespace gm {
// per-program entry points (implemented in gm_traverse.cu, gm_pagerank.cu, ...)
gm_status trav_prepare(gm_graph* g);
gm_status trav_reuse(gm_graph* g);  // program_set between BFS and SSSP with the workspace kept
gm_status build_source_ranks(gm_graph* g);  // gm_graph.cu
gm_status build_pull_edge_words(gm_graph* g);  // gm_graph.cu
gm_status balance_octets(gm_graph* g, int64_t staged);  // gm_graph.cu
// Messages the SSSP pull stages per CTA (ranks [0, result)): the stage option,
// at most 49,152 and n rounded down to a multiple of 4.
inline int64_t pull_stage_messages(const gm_graph* g) {
    return std::min<int64_t>(std::min<int64_t>(49152, g->tune.pull_stage), g->n & ~(int64_t)3);
}
// The octet pull stores its staged messages as 16 bits, so the same shared
// memory holds twice as many (a multiple of 8: whole 16-byte copies).
inline int64_t pull_stage16_messages(const gm_graph* g) {
    return std::min<int64_t>(2 * pull_stage_messages(g), g->n & ~(int64_t)7);
}
gm_status trav_set_active(gm_graph* g, const int32_t* vertices_dev, int64_t count);
gm_status trav_run(gm_graph* g, int32_t max_iters, int32_t* iters_done);
void trav_release(gm_graph* g);
gm_status pr_prepare(gm_graph* g);
gm_status pr_run(gm_graph* g, int32_t iters, int32_t* iters_done);
gm_status tc_run(gm_graph* g, int32_t* iters_done);
gm_status cf_prepare(gm_graph* g);
gm_status cf_run(gm_graph* g, int32_t iters, int32_t* iters_done);
gm_status cf_loss(gm_graph* g, double* out);
gm_status reached_edges(gm_graph* g, int64_t* out);
void wpr_release(gm_graph* g);
void cf_release(gm_graph* g);
void pr_release(gm_graph* g);
gm_status pr_reset(gm_graph* g);  // ranks back to 1.0, buffers kept
gm_status cc_prepare(gm_graph* g);  // gm_cc.cu
gm_status cc_run(gm_graph* g, int32_t max_iters, int32_t* iters_done);
// Per-edge source ids of a CSR (out[e] = v for e in [ptr[v], ptr[v+1])).
gm_status expand_rows(const int32_t* ptr, int64_t n, int32_t* out, cudaStream_t s);
}  // namespace gm
