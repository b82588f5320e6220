// Graph ingest: edge list -> cleaned CSR (out-edges) + CSC (in-edges) on the GPU,
// degrees and degree-binned vertex lists.  Section 4.3.1 stores G^T as DCSC
// partitions for OpenMP threads; on GB300 the whole graph sits in HBM as CSR (the
// push side of Algorithm 1: the columns of G^T) plus CSC (the pull side), int32
// indices, with vertices grouped by degree so each group gets a fitting
// thread/warp/CTA mapping.  Section 5.1 gives the cleaning steps.
#include <cstring>
#include <new>

#include "gm_internal.cuh"

namespace gm {

const char* last_error();

namespace {

__global__ void count_bad_ids(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                              int64_t n, unsigned long long* bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool b = false;
    if (i < m) b = src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n;
    unsigned mask = __ballot_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(bad, (unsigned long long)__popc(mask));
}

// Keys (src << b | dst); the reversed copies of a symmetrised list follow all
// originals.  Self-loops to drop get the all-ones key (sorted last).
__global__ void build_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                           int64_t total, int b, int drop_loops, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int64_t j = i < m ? i : i - m;
    uint32_t s = (uint32_t)(i < m ? src[j] : dst[j]);
    uint32_t d = (uint32_t)(i < m ? dst[j] : src[j]);
    uint64_t marker = (b >= 32) ? ~0ull : ((1ull << (2 * b)) - 1ull);
    keys[i] = (drop_loops && s == d) ? marker : (((uint64_t)s << b) | d);
    vals[i] = (uint32_t)j;
}

__global__ void keep_flags(const uint64_t* __restrict__ keys, int64_t total, int b, int drop_loops,
                           int dedup, uint32_t* __restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    uint64_t marker = ((1ull << (2 * b)) - 1ull);
    uint64_t k = keys[i];
    bool keep = !(drop_loops && k == marker);
    if (keep && dedup && i > 0 && keys[i - 1] == k) keep = false;
    flags[i] = keep ? 1u : 0u;
}

// Scatter kept edges: split key into (first, second) ids, carry the value.
__global__ void compact_edges(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                              const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos,
                              int64_t total, int b, int32_t* __restrict__ first, int32_t* __restrict__ second,
                              uint32_t* __restrict__ val_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total || !flags[i]) return;
    uint32_t p = pos[i];
    uint64_t k = keys[i];
    first[p] = (int32_t)(k >> b);
    second[p] = (int32_t)(k & ((1ull << b) - 1ull));
    val_out[p] = vals[i];
}

// ptr[v] = first position p with ids[p] >= v (ids non-decreasing), ptr[n] = len.
__global__ void fill_ptr(const int32_t* __restrict__ ids, int64_t len, int64_t n, int32_t* __restrict__ ptr) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > len) return;
    int64_t lo = p == 0 ? 0 : (int64_t)ids[p - 1] + 1;
    int64_t hi = p == len ? n : (int64_t)ids[p];
    for (int64_t v = lo; v <= hi; ++v) ptr[v] = (int32_t)p;
}

__global__ void orient_flags(const int32_t* __restrict__ esrc, const int32_t* __restrict__ edst, int64_t len,
                             const int32_t* __restrict__ ptr, uint32_t* __restrict__ flags) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= len) return;
    int32_t u = esrc[p], v = edst[p];
    int32_t du = ptr[u + 1] - ptr[u], dv = ptr[v + 1] - ptr[v];
    flags[p] = (du < dv || (du == dv && u < v)) ? 1u : 0u;
}

__global__ void compact_triples(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                                const uint32_t* __restrict__ c, const uint32_t* __restrict__ flags,
                                const uint32_t* __restrict__ pos, int64_t len, int32_t* __restrict__ ao,
                                int32_t* __restrict__ bo, uint32_t* __restrict__ co) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len || !flags[i]) return;
    uint32_t p = pos[i];
    ao[p] = a[i];
    bo[p] = b[i];
    co[p] = c[i];
}

// out[i] = in[i] as one byte; *wide = 1 if some in[i] does not fit.
__global__ void narrow_u8(const uint32_t* __restrict__ in, int64_t len, uint8_t* __restrict__ out,
                          uint32_t* __restrict__ wide) {
    bool big = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = in[i];
        big |= x > 255u;
        out[i] = (uint8_t)x;
    }
    if (__syncthreads_or(big) && threadIdx.x == 0) atomicOr(wide, 1u);
}

__global__ void gather_u32(const uint32_t* __restrict__ in, const uint32_t* __restrict__ idx, int64_t len,
                           uint32_t* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] = in[idx[i]];
}

// CSC keys from the CSR-ordered edges: the destination in the low 32 bits (the
// sort looks at its low b bits only; the bits above stay zero), the source in the
// high 32.  The edges arrive sorted by (src, dst), so a stable sort on the
// destination alone yields (dst, src) order.
__global__ void csc_keys(const int32_t* __restrict__ esrc, const int32_t* __restrict__ edst, int64_t len,
                         uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= len) return;
    keys[p] = ((uint64_t)(uint32_t)esrc[p] << 32) | (uint32_t)edst[p];
    vals[p] = (uint32_t)p;
}

__global__ void csc_split(const uint64_t* __restrict__ keys, int64_t len, int32_t* __restrict__ dst_ids,
                          int32_t* __restrict__ row) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= len) return;
    uint64_t k = keys[q];
    dst_ids[q] = (int32_t)(uint32_t)k;
    row[q] = (int32_t)(k >> 32);
}

__global__ void degrees_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ cp, int64_t n,
                               int32_t* __restrict__ od, int32_t* __restrict__ id) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    od[v] = rp[v + 1] - rp[v];
    id[v] = cp[v + 1] - cp[v];
}

__device__ __forceinline__ uint8_t degree_bin(int32_t d, int32_t small, int32_t large) {
    return d == 0 ? 0 : (d < small ? 1 : (d < large ? 2 : 3));
}

__global__ void bins_kernel(const int32_t* __restrict__ od, const int32_t* __restrict__ id, int64_t n,
                            int32_t small, int32_t large, uint8_t* __restrict__ ob, uint8_t* __restrict__ ib) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    ob[v] = degree_bin(od[v], small, large);
    ib[v] = degree_bin(id[v], small, large);
}

__global__ void bin_match_flags(const uint8_t* __restrict__ bins, int64_t n, uint8_t want,
                                uint32_t* __restrict__ flags) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) flags[v] = bins[v] == want ? 1u : 0u;
}

__global__ void positive_flags(const int32_t* __restrict__ deg, int64_t n, uint32_t* __restrict__ flags) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) flags[v] = deg[v] > 0 ? 1u : 0u;
}

__global__ void dcsc_cp_kernel(const int32_t* __restrict__ jc, int64_t ncols, const int32_t* __restrict__ col_ptr,
                               int64_t m, int32_t* __restrict__ cp) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncols) cp[c] = col_ptr[jc[c]];
    if (c == ncols) cp[c] = (int32_t)m;
}

// tile[k] = the column holding edge k * kWTile (columns are non-empty, so exactly one).
__global__ void dcsc_tile_kernel(const int32_t* __restrict__ cp, int64_t ncols, int32_t* __restrict__ tile) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const int64_t b = cp[c], e = cp[c + 1];
    for (int64_t k = (b + kWTile - 1) / kWTile; k * kWTile < e; ++k) tile[k] = (int32_t)c;
}

__global__ void dcsc_head_kernel(const int32_t* __restrict__ cp, int64_t ncols, uint32_t* __restrict__ head) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const int64_t e = cp[c];
    atomicOr(&head[e >> 5], 1u << (e & 31));
}

inline unsigned blocks_for(int64_t n, int t = 256) {
    int64_t b = (n + t - 1) / t;
    return (unsigned)(b > 0 ? b : 1);
}

int bits_for(int64_t n) {
    int b = 1;
    while (b < 31 && (1ll << b) < n) ++b;
    return b;
}

#define LAUNCH_CHECK()                                                                     \
    do {                                                                                   \
        g_launches++;                                                                      \
        cudaError_t _e = cudaGetLastError();                                               \
        if (_e != cudaSuccess) {                                                           \
            set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(_e), __FILE__, \
                      __LINE__);                                                           \
            return GM_ERR_CUDA;                                                            \
        }                                                                                  \
    } while (0)

}  // namespace

__global__ void degree_keys(const int32_t* __restrict__ list, int64_t len, const int32_t* __restrict__ deg,
                            uint64_t* __restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint64_t)(uint32_t)deg[list[i]];
}

// Sort list[0, len) by deg (stable: ties keep ascending ids), so that 32
// consecutive small-bin rows, which row passes give one lane each, have about
// the same length.
static gm_status sort_by_degree(int32_t* list, int64_t len, const int32_t* deg, int bits, cudaStream_t s) {
    if (len < 2) return GM_OK;
    struct Tmp {
        cudaStream_t s;
        DevBuf b[3];
        ~Tmp() { for (DevBuf& x : b) dev_free(x, s); }
    } tmp{s};
    GM_TRY(dev_alloc(tmp.b[0], sizeof(uint64_t) * len, s));
    GM_TRY(dev_alloc(tmp.b[1], sizeof(uint64_t) * len, s));
    GM_TRY(dev_alloc(tmp.b[2], sizeof(uint32_t) * len, s));
    degree_keys<<<blocks_for(len), 256, 0, s>>>(list, len, deg, as<uint64_t>(tmp.b[0]));
    LAUNCH_CHECK();
    GM_TRY(radix_sort_pairs(as<uint64_t>(tmp.b[0]), reinterpret_cast<uint32_t*>(list), as<uint64_t>(tmp.b[1]),
                            as<uint32_t>(tmp.b[2]), len, bits, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));  // the temporaries are freed on return
    return GM_OK;
}

// Compact the vertices of each degree bin 1..3 (consecutive in `list`, offsets in
// off[0..3]) and the degree-0 vertices (into `zero`, count in *zero_count).  Bin 1
// is ordered by degree (see sort_by_degree); bins 2 and 3 by id.
static gm_status bin_lists(gm_graph* g, const uint8_t* bins, const int32_t* deg, int32_t* list, int64_t* off,
                           int32_t* zero, int64_t* zero_count) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n;
    DevBuf flags, cnt;
    GM_TRY(dev_alloc(flags, sizeof(uint32_t) * (n > 0 ? n : 1), s));
    gm_status st = dev_alloc(cnt, sizeof(uint32_t) * 4, s);
    uint32_t hc[4] = {0, 0, 0, 0};
    int64_t pos = 0;
    for (int bin = 0; bin <= 3 && st == GM_OK; ++bin) {
        if (n > 0) {
            bin_match_flags<<<blocks_for(n), 256, 0, s>>>(bins, n, (uint8_t)bin, as<uint32_t>(flags));
            g_launches++;
        }
        int32_t* dst = bin == 0 ? zero : list + pos;
        st = compact_indices(as<uint32_t>(flags), n, dst, as<uint32_t>(cnt) + bin, s);
        if (st != GM_OK) break;
        cudaError_t e = cudaMemcpyAsync(&hc[bin], as<uint32_t>(cnt) + bin, sizeof(uint32_t),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_error("bins: %s", cudaGetErrorString(e)); st = GM_ERR_CUDA; break; }
        if (bin == 1) st = sort_by_degree(list, hc[1], deg, bits_for((int64_t)g->tune.bin_small + 1), s);
        if (bin > 0) pos += hc[bin];
    }
    dev_free(flags, s);
    dev_free(cnt, s);
    if (st != GM_OK) return st;
    *zero_count = hc[0];
    off[0] = 0;
    off[1] = hc[1];
    off[2] = hc[1] + hc[2];
    off[3] = hc[1] + hc[2] + hc[3];
    return GM_OK;
}

// Rebuild degree bins and the binned vertex lists (by in-degree for pull-side
// passes over the CSC, by out-degree for passes over the CSR rows).
gm_status build_bins(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n;
    GM_TRY(dev_alloc(g->out_bin, n > 0 ? n : 1, s));
    GM_TRY(dev_alloc(g->in_bin, n > 0 ? n : 1, s));
    if (n > 0) {
        bins_kernel<<<blocks_for(n), 256, 0, s>>>(as<int32_t>(g->out_deg), as<int32_t>(g->in_deg), n,
                                                  g->tune.bin_small, g->tune.bin_large,
                                                  as<uint8_t>(g->out_bin), as<uint8_t>(g->in_bin));
        LAUNCH_CHECK();
    }
    GM_TRY(dev_alloc(g->in_list, sizeof(int32_t) * (n > 0 ? n : 1), s));
    GM_TRY(dev_alloc(g->zero_in_list, sizeof(int32_t) * (n > 0 ? n : 1), s));
    GM_TRY(dev_alloc(g->out_list, sizeof(int32_t) * (n > 0 ? n : 1), s));
    GM_TRY(dev_alloc(g->zero_out_list, sizeof(int32_t) * (n > 0 ? n : 1), s));
    GM_TRY(bin_lists(g, as<uint8_t>(g->in_bin), as<int32_t>(g->in_deg), as<int32_t>(g->in_list), g->in_list_count,
                     as<int32_t>(g->zero_in_list), &g->zero_in_count));
    GM_TRY(bin_lists(g, as<uint8_t>(g->out_bin), as<int32_t>(g->out_deg), as<int32_t>(g->out_list),
                     g->out_list_count, as<int32_t>(g->zero_out_list), &g->zero_out_count));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    return GM_OK;
}

// The doubly compressed CSC of the pull side and its edge tiles.
static gm_status build_dcsc(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n, m = g->m;
    DevBuf flags, cnt;
    GM_TRY(dev_alloc(g->dc_jc, sizeof(int32_t) * (n > 0 ? n : 1), s));
    GM_TRY(dev_alloc(flags, sizeof(uint32_t) * (n > 0 ? n : 1), s));
    gm_status st = dev_alloc(cnt, sizeof(uint32_t), s);
    uint32_t ncols = 0;
    if (st == GM_OK && n > 0) {
        positive_flags<<<blocks_for(n), 256, 0, s>>>(as<int32_t>(g->in_deg), n, as<uint32_t>(flags));
        g_launches++;
    }
    if (st == GM_OK) st = compact_indices(as<uint32_t>(flags), n, as<int32_t>(g->dc_jc), as<uint32_t>(cnt), s);
    if (st == GM_OK) {
        cudaError_t e = cudaMemcpyAsync(&ncols, cnt.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_error("dcsc: %s", cudaGetErrorString(e)); st = GM_ERR_CUDA; }
    }
    dev_free(flags, s);
    dev_free(cnt, s);
    if (st != GM_OK) return st;
    g->dc_ncols = ncols;
    g->dc_ntiles = (m + kWTile - 1) / kWTile;
    GM_TRY(dev_alloc(g->dc_cp, sizeof(int32_t) * (ncols + 1), s));
    GM_TRY(dev_alloc(g->dc_tile, sizeof(int32_t) * (g->dc_ntiles + 1), s));
    dcsc_cp_kernel<<<blocks_for((int64_t)ncols + 1), 256, 0, s>>>(as<int32_t>(g->dc_jc), ncols,
                                                                 as<int32_t>(g->col_ptr), m, as<int32_t>(g->dc_cp));
    LAUNCH_CHECK();
    // head bits, padded so a warp tile's words can always be read
    const int64_t hwords = (m + 31) / 32 + kWTile / 32 + 1;
    GM_TRY(dev_alloc(g->dc_head, sizeof(uint32_t) * hwords, s));
    GM_CUDA_TRY(cudaMemsetAsync(g->dc_head.p, 0, sizeof(uint32_t) * hwords, s));
    if (ncols > 0) {
        dcsc_tile_kernel<<<blocks_for(ncols), 256, 0, s>>>(as<int32_t>(g->dc_cp), ncols, as<int32_t>(g->dc_tile));
        LAUNCH_CHECK();
        dcsc_head_kernel<<<blocks_for(ncols), 256, 0, s>>>(as<int32_t>(g->dc_cp), ncols, as<uint32_t>(g->dc_head));
        LAUNCH_CHECK();
    }
    return GM_OK;
}

static gm_status ingest(gm_graph* g, const gm_edge_list* el, uint32_t flags) {
    cudaStream_t s = g->stream;
    const int64_t n = el->n_vertices, m = el->n_edges;
    const bool sym = flags & GM_SYMMETRIZE, drop = flags & GM_DROP_SELF_LOOPS, dedup = flags & GM_DEDUP,
               orient = flags & GM_ORIENT_BY_DEGREE;
    const int64_t total = sym ? 2 * m : m;
    const int b = bits_for(n);

    // ---- upload the raw list ----
    DevBuf d_src, d_dst, d_w;
    const int32_t* src = el->src;
    const int32_t* dst = el->dst;
    const uint32_t* win = static_cast<const uint32_t*>(el->weight);
    struct Scope {
        cudaStream_t s;
        DevBuf* bufs[24];
        int k = 0;
        ~Scope() { for (int i = 0; i < k; ++i) dev_free(*bufs[i], s); }
        void add(DevBuf& b) { bufs[k++] = &b; }
    } scope{s};
    DevBuf wide;  // flag: some weight needs more than 8 bits
    scope.add(d_src); scope.add(d_dst); scope.add(d_w); scope.add(wide);
    // The weights are not needed until the edges are sorted, so from host memory
    // they are copied on a side stream while the sort runs; the handle's stream
    // waits for that copy before it first reads them, and in any case before
    // this function returns (the guard is destroyed before the buffers are freed).
    struct SideCopy {
        cudaStream_t main, side = nullptr;
        cudaEvent_t done = nullptr;
        bool joined = true;
        cudaError_t join() {
            cudaError_t e = cudaSuccess;
            if (!joined) e = cudaStreamWaitEvent(main, done, 0);
            joined = true;
            return e;
        }
        ~SideCopy() {
            join();
            if (done) cudaEventDestroy(done);
            if (side) cudaStreamDestroy(side);
        }
    } wcopy{s};
    if (!el->on_device && m > 0) {
        GM_TRY(dev_alloc(d_src, sizeof(int32_t) * m, s));
        GM_TRY(dev_alloc(d_dst, sizeof(int32_t) * m, s));
        if (g->wtype != GM_W_NONE) GM_TRY(dev_alloc(d_w, sizeof(uint32_t) * m, s));
        GM_CUDA_TRY(cudaMemcpyAsync(d_src.p, el->src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        GM_CUDA_TRY(cudaMemcpyAsync(d_dst.p, el->dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        src = as<int32_t>(d_src);
        dst = as<int32_t>(d_dst);
        if (g->wtype != GM_W_NONE) {
            GM_CUDA_TRY(cudaStreamCreateWithFlags(&wcopy.side, cudaStreamNonBlocking));
            GM_CUDA_TRY(cudaEventCreateWithFlags(&wcopy.done, cudaEventDisableTiming));
            GM_CUDA_TRY(cudaEventRecord(wcopy.done, s));  // d_w is allocated (stream-ordered) before the copy
            GM_CUDA_TRY(cudaStreamWaitEvent(wcopy.side, wcopy.done, 0));
            GM_CUDA_TRY(cudaMemcpyAsync(d_w.p, el->weight, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, wcopy.side));
            GM_CUDA_TRY(cudaEventRecord(wcopy.done, wcopy.side));
            wcopy.joined = false;
            win = as<uint32_t>(d_w);
        }
    }

    // ---- validate ids ----
    DevBuf bad;
    scope.add(bad);
    GM_TRY(dev_alloc(bad, sizeof(unsigned long long), s));
    GM_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(unsigned long long), s));
    if (m > 0) {
        count_bad_ids<<<blocks_for(m), 256, 0, s>>>(src, dst, m, n, as<unsigned long long>(bad));
        LAUNCH_CHECK();
    }
    unsigned long long hbad = 0;
    GM_CUDA_TRY(cudaMemcpyAsync(&hbad, bad.p, sizeof(hbad), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) {
        set_error("gm_graph_create: %llu edge endpoints outside [0, %lld)", hbad, (long long)n);
        return GM_ERR_INVALID_ARG;
    }

    // ---- sort (src, dst), clean ----
    DevBuf keys, vals, keys2, vals2, fl, pos;
    scope.add(keys); scope.add(vals); scope.add(keys2); scope.add(vals2); scope.add(fl); scope.add(pos);
    GM_TRY(dev_alloc(keys, sizeof(uint64_t) * (total > 0 ? total : 1), s));
    GM_TRY(dev_alloc(vals, sizeof(uint32_t) * (total > 0 ? total : 1), s));
    GM_TRY(dev_alloc(keys2, sizeof(uint64_t) * (total > 0 ? total : 1), s));
    GM_TRY(dev_alloc(vals2, sizeof(uint32_t) * (total > 0 ? total : 1), s));
    GM_TRY(dev_alloc(fl, sizeof(uint32_t) * (total > 0 ? total : 1), s));
    GM_TRY(dev_alloc(pos, sizeof(uint32_t) * (total + 1), s));
    if (total > 0) {
        build_keys<<<blocks_for(total), 256, 0, s>>>(src, dst, m, total, b, drop ? 1 : 0, as<uint64_t>(keys),
                                                     as<uint32_t>(vals));
        LAUNCH_CHECK();
        GM_TRY(radix_sort_pairs(as<uint64_t>(keys), as<uint32_t>(vals), as<uint64_t>(keys2),
                                as<uint32_t>(vals2), total, 2 * b, s));
        keep_flags<<<blocks_for(total), 256, 0, s>>>(as<uint64_t>(keys), total, b, drop ? 1 : 0, dedup ? 1 : 0,
                                                     as<uint32_t>(fl));
        LAUNCH_CHECK();
    }
    GM_TRY(scan_exclusive_u32(as<uint32_t>(fl), as<uint32_t>(pos), total, s));
    uint32_t m1 = 0;
    GM_CUDA_TRY(cudaMemcpyAsync(&m1, as<uint32_t>(pos) + total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));

    DevBuf esrc, edst, perm, esrc2, edst2, perm2;  // function scope: the cleanup list points at them
    scope.add(esrc); scope.add(edst); scope.add(perm);
    scope.add(esrc2); scope.add(edst2); scope.add(perm2);
    GM_TRY(dev_alloc(esrc, sizeof(int32_t) * (m1 > 0 ? m1 : 1), s));
    GM_TRY(dev_alloc(edst, sizeof(int32_t) * (m1 > 0 ? m1 : 1), s));
    GM_TRY(dev_alloc(perm, sizeof(uint32_t) * (m1 > 0 ? m1 : 1), s));
    if (total > 0) {
        compact_edges<<<blocks_for(total), 256, 0, s>>>(as<uint64_t>(keys), as<uint32_t>(vals), as<uint32_t>(fl),
                                                        as<uint32_t>(pos), total, b, as<int32_t>(esrc),
                                                        as<int32_t>(edst), as<uint32_t>(perm));
        LAUNCH_CHECK();
    }
    GM_TRY(dev_alloc(g->row_ptr, sizeof(int32_t) * (n + 1), s));
    fill_ptr<<<blocks_for((int64_t)m1 + 1), 256, 0, s>>>(as<int32_t>(esrc), m1, n, as<int32_t>(g->row_ptr));
    LAUNCH_CHECK();

    int64_t mm = m1;
    if (orient && mm > 0) {
        orient_flags<<<blocks_for(mm), 256, 0, s>>>(as<int32_t>(esrc), as<int32_t>(edst), mm,
                                                    as<int32_t>(g->row_ptr), as<uint32_t>(fl));
        LAUNCH_CHECK();
        GM_TRY(scan_exclusive_u32(as<uint32_t>(fl), as<uint32_t>(pos), mm, s));
        uint32_t m2 = 0;
        GM_CUDA_TRY(cudaMemcpyAsync(&m2, as<uint32_t>(pos) + mm, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        GM_CUDA_TRY(cudaStreamSynchronize(s));
        GM_TRY(dev_alloc(esrc2, sizeof(int32_t) * (m2 > 0 ? m2 : 1), s));
        GM_TRY(dev_alloc(edst2, sizeof(int32_t) * (m2 > 0 ? m2 : 1), s));
        GM_TRY(dev_alloc(perm2, sizeof(uint32_t) * (m2 > 0 ? m2 : 1), s));
        compact_triples<<<blocks_for(mm), 256, 0, s>>>(as<int32_t>(esrc), as<int32_t>(edst), as<uint32_t>(perm),
                                                       as<uint32_t>(fl), as<uint32_t>(pos), mm, as<int32_t>(esrc2),
                                                       as<int32_t>(edst2), as<uint32_t>(perm2));
        LAUNCH_CHECK();
        std::swap(esrc, esrc2);
        std::swap(edst, edst2);
        std::swap(perm, perm2);
        mm = m2;
        fill_ptr<<<blocks_for(mm + 1), 256, 0, s>>>(as<int32_t>(esrc), mm, n, as<int32_t>(g->row_ptr));
        LAUNCH_CHECK();
    }
    g->m = mm;

    // ---- CSR arrays ----
    GM_TRY(dev_alloc(g->col, sizeof(int32_t) * (mm + kEdgePad), s));
    if (mm > 0)
        GM_CUDA_TRY(cudaMemcpyAsync(g->col.p, edst.p, sizeof(int32_t) * mm, cudaMemcpyDeviceToDevice, s));
    if (g->wtype != GM_W_NONE) {
        GM_TRY(dev_alloc(g->w, sizeof(uint32_t) * (mm + kEdgePad), s));
        GM_CUDA_TRY(wcopy.join());
        if (mm > 0) {
            gather_u32<<<blocks_for(mm), 256, 0, s>>>(win, as<uint32_t>(perm), mm, as<uint32_t>(g->w));
            LAUNCH_CHECK();
        }
    }

    // ---- CSC by a second sort on (dst, src) ----
    GM_TRY(dev_alloc(g->col_ptr, sizeof(int32_t) * (n + 1), s));
    GM_TRY(dev_alloc(g->row, sizeof(int32_t) * (mm + kEdgePad), s));
    GM_TRY(dev_alloc(g->csc_pos, sizeof(uint32_t) * (mm > 0 ? mm : 1), s));
    if (mm > 0) {
        csc_keys<<<blocks_for(mm), 256, 0, s>>>(as<int32_t>(esrc), as<int32_t>(edst), mm, as<uint64_t>(keys),
                                                as<uint32_t>(vals));
        LAUNCH_CHECK();
        GM_TRY(radix_sort_pairs(as<uint64_t>(keys), as<uint32_t>(vals), as<uint64_t>(keys2), as<uint32_t>(vals2),
                                mm, b, s));
        csc_split<<<blocks_for(mm), 256, 0, s>>>(as<uint64_t>(keys), mm, as<int32_t>(esrc), as<int32_t>(g->row));
        LAUNCH_CHECK();
        GM_CUDA_TRY(cudaMemcpyAsync(g->csc_pos.p, vals.p, sizeof(uint32_t) * mm, cudaMemcpyDeviceToDevice, s));
    }
    fill_ptr<<<blocks_for(mm + 1), 256, 0, s>>>(as<int32_t>(esrc), mm, n, as<int32_t>(g->col_ptr));
    LAUNCH_CHECK();
    if (g->wtype != GM_W_NONE) {
        GM_TRY(dev_alloc(g->cw, sizeof(uint32_t) * (mm + kEdgePad), s));
        if (mm > 0) {
            gather_u32<<<blocks_for(mm), 256, 0, s>>>(as<uint32_t>(g->w), as<uint32_t>(g->csc_pos), mm,
                                                      as<uint32_t>(g->cw));
            LAUNCH_CHECK();
        }
        if (g->wtype == GM_W_U32 && mm > 0) {  // one byte per in-edge for the pull when the weights allow
            GM_TRY(dev_alloc(wide, sizeof(uint32_t), s));
            GM_CUDA_TRY(cudaMemsetAsync(wide.p, 0, sizeof(uint32_t), s));
            GM_TRY(dev_alloc(g->cw8, (size_t)(mm + kEdgePad), s));
            GM_CUDA_TRY(cudaMemsetAsync(g->cw8.p, 0, (size_t)(mm + kEdgePad), s));
            narrow_u8<<<num_sms() * 8, 256, 0, s>>>(as<uint32_t>(g->cw), mm, as<uint8_t>(g->cw8), as<uint32_t>(wide));
            LAUNCH_CHECK();
            uint32_t h_wide = 1u;
            GM_CUDA_TRY(cudaMemcpyAsync(&h_wide, wide.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            GM_CUDA_TRY(cudaStreamSynchronize(s));
            if (h_wide) dev_free(g->cw8, s);
        }
    }

    // ---- degrees and bins ----
    GM_TRY(dev_alloc(g->out_deg, sizeof(int32_t) * (n > 0 ? n : 1), s));
    GM_TRY(dev_alloc(g->in_deg, sizeof(int32_t) * (n > 0 ? n : 1), s));
    if (n > 0) {
        degrees_kernel<<<blocks_for(n), 256, 0, s>>>(as<int32_t>(g->row_ptr), as<int32_t>(g->col_ptr), n,
                                                     as<int32_t>(g->out_deg), as<int32_t>(g->in_deg));
        LAUNCH_CHECK();
    }
    GM_TRY(build_bins(g));
    GM_TRY(build_dcsc(g));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    return GM_OK;
}

// ---- source ranks for the SSSP pull ----
__global__ void rank_keys(const int32_t* __restrict__ out_deg, int64_t n, uint64_t* __restrict__ keys,
                          uint32_t* __restrict__ vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = 0xFFFFFFFFull - (uint32_t)out_deg[i];  // ascending key = descending degree
        vals[i] = (uint32_t)i;
    }
}

__global__ void invert_order(const uint32_t* __restrict__ order, int64_t n, int32_t* __restrict__ rank) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rank[order[i]] = (int32_t)i;
}

__global__ void gather_i32(const int32_t* __restrict__ idx, int64_t len, const int32_t* __restrict__ table,
                           int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = table[idx[i]];
}

// Octets of every non-empty column c: ceil(in-degree / 8), into cnt[c] (cnt[ncols] = 0).
__global__ void octet_counts(const int32_t* __restrict__ cp, int64_t ncols, uint32_t* __restrict__ cnt) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= ncols; c += (int64_t)gridDim.x * blockDim.x)
        cnt[c] = c < ncols ? (uint32_t)((cp[c + 1] - cp[c] + kOctet - 1) / kOctet) : 0u;
}

// The octet layout is built in three steps.  octet_starts marks each column's
// first octet (header bit 0x80); octet_tile_starts counts the marks of every
// tile of 32 octets, and an exclusive scan of those counts gives, for each tile,
// the column of its first octet; octet_fill, one warp per tile and one lane per
// octet, finds its column from that and its lane's marks, and writes the
// octet's in-edges as one word each -- the source's rank in the high 24 bits and
// the one-byte weight in the low 8 (padding slots 0) -- the octet header (real
// slots, and the mark) and the tile's first column.  Within a tile the words are
// stored slot-quad-major: slots 0-3 of octets 0..31, then slots 4-7 of octets
// 0..31, so a lane's octet is two 16-byte stores and the warp's are 512
// consecutive bytes each.
__global__ void octet_starts(const uint32_t* __restrict__ ooff, int64_t ncols, uint8_t* __restrict__ meta) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += (int64_t)gridDim.x * blockDim.x)
        meta[ooff[c]] = 0x80;
}

__global__ void octet_tile_starts(const uint8_t* __restrict__ meta, int64_t octets, int64_t tiles,
                                  uint32_t* __restrict__ tcnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < tiles; k += nw) {
        const int64_t o = k * kOctTile + lane;
        const uint32_t ball = __ballot_sync(0xffffffffu, o < octets && (meta[o] & 0x80));
        if (lane == 0) tcnt[k] = (uint32_t)__popc(ball);
    }
}

__global__ void octet_fill(const int32_t* __restrict__ cp, const uint32_t* __restrict__ ooff, int64_t octets,
                           int64_t tiles, const uint32_t* __restrict__ tpre, const int32_t* __restrict__ row,
                           const uint8_t* __restrict__ w8, const int32_t* __restrict__ rank,
                           uint32_t* __restrict__ ow, uint8_t* __restrict__ meta, int32_t* __restrict__ c0) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < tiles; k += nw) {
        const int64_t o = k * kOctTile + lane;
        const bool here = o < octets;
        const bool start = here && (meta[o] & 0x80);
        const uint32_t ball = __ballot_sync(0xffffffffu, start);
        if (!here) continue;  // the tail of the last tile stays zero
        const int64_t col = (int64_t)tpre[k] + __popc(ball & (0xffffffffu >> (31 - lane))) - 1;
        const int64_t eb = (int64_t)cp[col] + (o - (int64_t)ooff[col]) * kOctet;
        const int real = (int)min((int64_t)kOctet, (int64_t)cp[col + 1] - eb);
        uint32_t wd[kOctet];
#pragma unroll
        for (int q = 0; q < kOctet; ++q)
            wd[q] = q < real ? ((uint32_t)rank[row[eb + q]] << 8) | (uint32_t)w8[eb + q] : 0u;
        uint4* tw = reinterpret_cast<uint4*>(ow + k * (kOctTile * kOctet));
        tw[lane] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        tw[kOctTile + lane] = make_uint4(wd[4], wd[5], wd[6], wd[7]);
        meta[o] = (uint8_t)(real | (start ? 0x80 : 0));
        if (lane == 0) c0[k] = (int32_t)col;
    }
}

// Slot order inside each octet, chosen so that the warp's shared-memory reads of
// staged messages (sources of rank < staged, two 16-bit messages per 4-byte
// bank word, so rank r sits in bank (r / 2) mod 32) spread over the 32 banks:
// for every tile one thread takes the octets in lane order and puts each staged
// source of an octet into the still-free slot (one of its real slots) whose
// warp-wide read has used that source's bank least so far; the other sources
// fill the slots left.  Any order of an octet's real slots gives the same
// minimum; on RMAT scale 22 (40,960 4-byte messages then) it took the reads from
// 2.3 to 1.2 bank-conflict wavefronts per warp-wide read.  Padding slots stay last.
constexpr int kBalanceThreads = 64;
__global__ void __launch_bounds__(kBalanceThreads) octet_balance(uint32_t* __restrict__ ow,
                                                                const uint8_t* __restrict__ meta, int64_t tiles,
                                                                uint32_t staged) {
    __shared__ uint8_t s_use[kBalanceThreads][kOctet][32];
    uint8_t (*use)[32] = s_use[threadIdx.x];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t* u32 = reinterpret_cast<uint32_t*>(&use[0][0]);
#pragma unroll
        for (int i = 0; i < kOctet * 32 / 4; ++i) u32[i] = 0u;
        // the tile is slot-quad-major: octet L's slots 0-3 are 16-byte word L, slots 4-7 word 32 + L
        uint4* tw = reinterpret_cast<uint4*>(ow + t * (kOctTile * kOctet));
        for (int L = 0; L < kOctTile; ++L) {
            const uint32_t real = meta[t * kOctTile + L] & 0xFu;
            const uint4 lo = tw[L], hi = tw[kOctTile + L];
            const uint32_t w[kOctet] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
            const uint32_t slots = (1u << real) - 1u;
            uint32_t taken = 0u;   // slots assigned so far
            uint32_t assign = 0u;  // 3 bits per slot: the source placed there
#pragma unroll
            for (int j = 0; j < kOctet; ++j) {  // staged sources first, each where its bank is used least
                const uint32_t r = w[j] >> 8;
                if ((uint32_t)j < real && r < staged) {
                    const uint32_t b = (r >> 1) & 31u;
                    int best = 0;
                    uint32_t bu = 0xFFFFu;
#pragma unroll
                    for (int q = 0; q < kOctet; ++q) {
                        const uint32_t u = use[q][b];
                        if ((((slots & ~taken) >> q) & 1u) && u < bu) {
                            best = q;
                            bu = u;
                        }
                    }
                    taken |= 1u << best;
                    assign |= (uint32_t)j << (3 * best);
                    use[best][b] = (uint8_t)(bu + 1u);
                }
            }
#pragma unroll
            for (int j = 0; j < kOctet; ++j) {  // the others into the free slots, in order
                if ((uint32_t)j < real && (w[j] >> 8) >= staged) {
                    const int q = __ffs(slots & ~taken) - 1;
                    taken |= 1u << q;
                    assign |= (uint32_t)j << (3 * q);
                }
            }
            uint32_t out[kOctet];
#pragma unroll
            for (int q = 0; q < kOctet; ++q) {
                const uint32_t j = (assign >> (3 * q)) & 7u;
                uint32_t v = w[0];
#pragma unroll
                for (int i = 1; i < kOctet; ++i) v = j == (uint32_t)i ? w[i] : v;
                out[q] = (uint32_t)q < real ? v : w[q];  // padding slots stay last
            }
            tw[L] = make_uint4(out[0], out[1], out[2], out[3]);
            tw[kOctTile + L] = make_uint4(out[4], out[5], out[6], out[7]);
        }
    }
}

// Re-orders the octets' slots for a stage of `staged` messages (octet_balance).
gm_status balance_octets(gm_graph* g, int64_t staged) {
    if (!g->oct_w.p || g->oct_tiles == 0) return GM_OK;
    cudaStream_t s = g->stream;
    const int64_t blocks = std::min<int64_t>((g->oct_tiles + kBalanceThreads - 1) / kBalanceThreads, 65535);
    octet_balance<<<(unsigned)blocks, kBalanceThreads, 0, s>>>(as<uint32_t>(g->oct_w), as<uint8_t>(g->oct_meta),
                                                               g->oct_tiles, (uint32_t)std::max<int64_t>(staged, 0));
    LAUNCH_CHECK();
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    return GM_OK;
}

// The SSSP pull's in-edge stream from the source ranks: the octet layout
// (oct_w, oct_meta, oct_c0) when every weight fits a byte, n <= 2^24 and the
// layout option allows it; otherwise the ranks alone (row_r), the weights then
// coming from cw8 or cw.  Replaces whichever exists.
namespace {
void free_pull_edge_words(gm_graph* g) {
    cudaStream_t s = g->stream;
    dev_free(g->row_r, s);
    dev_free(g->oct_w, s);
    dev_free(g->oct_meta, s);
    dev_free(g->oct_c0, s);
    g->oct_tiles = g->oct_slots = 0;
}

gm_status build_pull_edge_words_impl(gm_graph* g);
}  // namespace

// All or nothing: a failure leaves neither layout (the SSSP pull then refuses
// to run until the next gm_program_set builds it).
gm_status build_pull_edge_words(gm_graph* g) {
    const gm_status st = build_pull_edge_words_impl(g);
    if (st != GM_OK) free_pull_edge_words(g);
    return st;
}

namespace {
gm_status build_pull_edge_words_impl(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int64_t m = g->m, ncols = g->dc_ncols;
    free_pull_edge_words(g);
    const bool packed = g->tune.pull_packed && g->cw8.p != nullptr && g->n <= kPackedMaxVertices;
    if (!packed) {
        GM_TRY(dev_alloc(g->row_r, sizeof(int32_t) * (m + kEdgePad), s));
        GM_CUDA_TRY(cudaMemsetAsync(g->row_r.p, 0, sizeof(int32_t) * (m + kEdgePad), s));
        if (m > 0) {
            gather_i32<<<blocks_for(m), 256, 0, s>>>(as<int32_t>(g->row), m, as<int32_t>(g->src_rank),
                                                     as<int32_t>(g->row_r));
            LAUNCH_CHECK();
        }
        return GM_OK;
    }
    // octet offsets of the columns: an exclusive scan of their octet counts
    struct Tmp {
        cudaStream_t s;
        DevBuf b[4];
        ~Tmp() { for (DevBuf& x : b) dev_free(x, s); }
    } tmp{s};
    DevBuf &cnt = tmp.b[0], &ooff = tmp.b[1];
    GM_TRY(dev_alloc(cnt, sizeof(uint32_t) * (ncols + 1), s));
    GM_TRY(dev_alloc(ooff, sizeof(uint32_t) * (ncols + 2), s));
    octet_counts<<<blocks_for(ncols + 1), 256, 0, s>>>(as<int32_t>(g->dc_cp), ncols, as<uint32_t>(cnt));
    LAUNCH_CHECK();
    GM_TRY(scan_exclusive_u32(as<uint32_t>(cnt), as<uint32_t>(ooff), ncols + 1, s));
    uint32_t octets = 0;
    GM_CUDA_TRY(cudaMemcpyAsync(&octets, as<uint32_t>(ooff) + ncols, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t tiles = ((int64_t)octets + kOctTile - 1) / kOctTile;
    const int64_t octs_alloc = std::max<int64_t>(tiles, 1) * kOctTile;  // whole tiles: the tail reads in bounds
    GM_TRY(dev_alloc(g->oct_w, sizeof(uint32_t) * octs_alloc * kOctet, s));
    GM_TRY(dev_alloc(g->oct_meta, (size_t)octs_alloc, s));
    GM_TRY(dev_alloc(g->oct_c0, sizeof(int32_t) * std::max<int64_t>(tiles, 1), s));
    GM_CUDA_TRY(cudaMemsetAsync(g->oct_w.p, 0, sizeof(uint32_t) * octs_alloc * kOctet, s));
    GM_CUDA_TRY(cudaMemsetAsync(g->oct_meta.p, 0, (size_t)octs_alloc, s));
    GM_CUDA_TRY(cudaMemsetAsync(g->oct_c0.p, 0, sizeof(int32_t) * std::max<int64_t>(tiles, 1), s));
    if (ncols > 0) {
        DevBuf &tcnt = tmp.b[2], &tpre = tmp.b[3];
        GM_TRY(dev_alloc(tcnt, sizeof(uint32_t) * tiles, s));
        GM_TRY(dev_alloc(tpre, sizeof(uint32_t) * (tiles + 1), s));
        octet_starts<<<blocks_for(ncols), 256, 0, s>>>(as<uint32_t>(ooff), ncols, as<uint8_t>(g->oct_meta));
        LAUNCH_CHECK();
        const unsigned wb = (unsigned)std::min<int64_t>((tiles + 7) / 8, (int64_t)num_sms() * 16);
        octet_tile_starts<<<wb, 256, 0, s>>>(as<uint8_t>(g->oct_meta), octets, tiles, as<uint32_t>(tcnt));
        LAUNCH_CHECK();
        GM_TRY(scan_exclusive_u32(as<uint32_t>(tcnt), as<uint32_t>(tpre), tiles, s));
        octet_fill<<<wb, 256, 0, s>>>(as<int32_t>(g->dc_cp), as<uint32_t>(ooff), octets, tiles, as<uint32_t>(tpre),
                                      as<int32_t>(g->row), as<uint8_t>(g->cw8), as<int32_t>(g->src_rank),
                                      as<uint32_t>(g->oct_w), as<uint8_t>(g->oct_meta), as<int32_t>(g->oct_c0));
        LAUNCH_CHECK();
    }
    GM_CUDA_TRY(cudaStreamSynchronize(s));  // the temporaries are freed on return
    g->oct_tiles = tiles;
    g->oct_slots = (int64_t)octets * kOctet;
    return balance_octets(g, pull_stage16_messages(g));
}
}  // namespace

namespace {
gm_status build_source_ranks_impl(gm_graph* g);
}  // namespace

// All or nothing: on failure the ranks and the in-edge layout are freed, so the
// next SSSP gm_program_set builds them again.
gm_status build_source_ranks(gm_graph* g) {
    if (g->src_rank.p) {  // ranks exist; the layout too unless its last rebuild failed
        if (g->oct_w.p || g->row_r.p) return GM_OK;
        return build_pull_edge_words(g);
    }
    const gm_status st = build_source_ranks_impl(g);
    if (st != GM_OK) {
        dev_free(g->src_rank, g->stream);
        dev_free(g->dc_rank, g->stream);
        free_pull_edge_words(g);
    }
    return st;
}

namespace {
gm_status build_source_ranks_impl(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n, m = g->m;
    struct Tmp {
        cudaStream_t s;
        DevBuf b[4];
        ~Tmp() { for (DevBuf& x : b) dev_free(x, s); }
    } tmp{s};
    DevBuf &keys = tmp.b[0], &vals = tmp.b[1], &keys2 = tmp.b[2], &vals2 = tmp.b[3];
    const int64_t n1 = n > 0 ? n : 1;
    GM_TRY(dev_alloc(g->src_rank, sizeof(int32_t) * n1, s));
    GM_TRY(dev_alloc(g->dc_rank, sizeof(int32_t) * (g->dc_ncols > 0 ? g->dc_ncols : 1), s));
    if (n > 0) {
        GM_TRY(dev_alloc(keys, sizeof(uint64_t) * n, s));
        GM_TRY(dev_alloc(vals, sizeof(uint32_t) * n, s));
        GM_TRY(dev_alloc(keys2, sizeof(uint64_t) * n, s));
        GM_TRY(dev_alloc(vals2, sizeof(uint32_t) * n, s));
        rank_keys<<<blocks_for(n), 256, 0, s>>>(as<int32_t>(g->out_deg), n, as<uint64_t>(keys), as<uint32_t>(vals));
        LAUNCH_CHECK();
        GM_TRY(radix_sort_pairs(as<uint64_t>(keys), as<uint32_t>(vals), as<uint64_t>(keys2), as<uint32_t>(vals2), n,
                                32, s));
        invert_order<<<blocks_for(n), 256, 0, s>>>(as<uint32_t>(vals), n, as<int32_t>(g->src_rank));
        LAUNCH_CHECK();
    }
    GM_TRY(build_pull_edge_words(g));
    if (g->dc_ncols > 0) {
        gather_i32<<<blocks_for(g->dc_ncols), 256, 0, s>>>(as<int32_t>(g->dc_jc), g->dc_ncols, as<int32_t>(g->src_rank),
                                                           as<int32_t>(g->dc_rank));
        LAUNCH_CHECK();
    }
    GM_CUDA_TRY(cudaStreamSynchronize(s));  // the temporaries are freed on return
    return GM_OK;
}
}  // namespace

void release_graph(gm_graph* g);

}  // namespace gm

using namespace gm;

extern "C" {

gm_status gm_graph_create(const gm_edge_list* el, uint32_t flags, void* stream, gm_graph** out) {
    if (out) *out = nullptr;
    if (!el || !out) { set_error("gm_graph_create: NULL argument"); return GM_ERR_INVALID_ARG; }
    if (el->n_vertices < 0 || el->n_vertices >= (1ll << 31) - 1 || el->n_edges < 0) {
        set_error("gm_graph_create: n_vertices must be in [0, 2^31-1) and n_edges >= 0");
        return GM_ERR_INVALID_ARG;
    }
    if (el->n_edges > 0 && (!el->src || !el->dst)) {
        set_error("gm_graph_create: NULL src/dst with n_edges > 0");
        return GM_ERR_INVALID_ARG;
    }
    if (el->weight_type < GM_W_NONE || el->weight_type > GM_W_F32 ||
        (el->weight_type != GM_W_NONE && el->n_edges > 0 && !el->weight)) {
        set_error("gm_graph_create: bad weight_type or NULL weight");
        return GM_ERR_INVALID_ARG;
    }
    if (flags & ~(uint32_t)(GM_DROP_SELF_LOOPS | GM_DEDUP | GM_SYMMETRIZE | GM_ORIENT_BY_DEGREE)) {
        set_error("gm_graph_create: unknown flag bits");
        return GM_ERR_INVALID_ARG;
    }
    const int64_t total = (flags & GM_SYMMETRIZE) ? 2 * el->n_edges : el->n_edges;
    if (total >= (1ll << 31) - 1) {
        set_error("gm_graph_create: %lld edges exceed the int32 edge-offset limit", (long long)total);
        return GM_ERR_UNSUPPORTED;
    }
    if (el->n_left < 0 || el->n_left > el->n_vertices) {
        set_error("gm_graph_create: n_left outside [0, n]");
        return GM_ERR_INVALID_ARG;
    }
    gm_graph* g = new (std::nothrow) gm_graph();
    if (!g) { set_error("gm_graph_create: host allocation failed"); return GM_ERR_OUT_OF_MEMORY; }
    g->n = el->n_vertices;
    g->n_left = el->n_left;
    g->flags = flags;
    g->stream = static_cast<cudaStream_t>(stream);
    g->wtype = el->weight_type;
    gm_status st = ingest(g, el, flags);
    if (st != GM_OK) {
        cudaStreamSynchronize(g->stream);
        release_graph(g);
        return st;
    }
    *out = g;
    return GM_OK;
}

gm_status gm_graph_destroy(gm_graph* g) {
    if (!g) return GM_OK;
    release_graph(g);
    return GM_OK;
}

gm_status gm_graph_info(const gm_graph* g, int64_t* n_vertices, int64_t* n_edges) {
    if (!g) { set_error("gm_graph_info: NULL handle"); return GM_ERR_INVALID_ARG; }
    if (n_vertices) *n_vertices = g->n;
    if (n_edges) *n_edges = g->m;
    return GM_OK;
}

gm_status gm_graph_get_edges(const gm_graph* g, int32_t* src, int32_t* dst, void* weight, int dst_is_device) {
    if (!g) { set_error("gm_graph_get_edges: NULL handle"); return GM_ERR_INVALID_ARG; }
    cudaStream_t s = g->stream;
    cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (src && g->m > 0) {
        // expand row_ptr into per-edge sources
        DevBuf tmp;
        int32_t* target = src;
        if (!dst_is_device) {
            GM_TRY(dev_alloc(tmp, sizeof(int32_t) * g->m, s));
            target = as<int32_t>(tmp);
        }
        gm_status st = expand_rows(as<int32_t>(g->row_ptr), g->n, target, s);
        if (st == GM_OK && !dst_is_device) {
            cudaError_t e = cudaMemcpyAsync(src, target, sizeof(int32_t) * g->m, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) { set_error("gm_graph_get_edges: %s", cudaGetErrorString(e)); st = GM_ERR_CUDA; }
        }
        cudaStreamSynchronize(s);
        dev_free(tmp, s);
        if (st != GM_OK) return st;
    }
    if (dst && g->m > 0) GM_CUDA_TRY(cudaMemcpyAsync(dst, g->col.p, sizeof(int32_t) * g->m, k, s));
    if (weight && g->m > 0 && g->w.p) GM_CUDA_TRY(cudaMemcpyAsync(weight, g->w.p, sizeof(uint32_t) * g->m, k, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    return GM_OK;
}

gm_status gm_graph_get_degrees(const gm_graph* g, int32_t* out_deg, int32_t* in_deg, int dst_is_device) {
    if (!g) { set_error("gm_graph_get_degrees: NULL handle"); return GM_ERR_INVALID_ARG; }
    cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (out_deg && g->n > 0) GM_CUDA_TRY(cudaMemcpyAsync(out_deg, g->out_deg.p, sizeof(int32_t) * g->n, k, g->stream));
    if (in_deg && g->n > 0) GM_CUDA_TRY(cudaMemcpyAsync(in_deg, g->in_deg.p, sizeof(int32_t) * g->n, k, g->stream));
    GM_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return GM_OK;
}

uint64_t gm_kernel_launch_count(void) { return g_launches.load(); }

const char* gm_status_string(gm_status s) {
    switch (s) {
        case GM_OK: return "GM_OK";
        case GM_ERR_INVALID_ARG: return "GM_ERR_INVALID_ARG";
        case GM_ERR_OUT_OF_MEMORY: return "GM_ERR_OUT_OF_MEMORY";
        case GM_ERR_CUDA: return "GM_ERR_CUDA";
        case GM_ERR_STATE: return "GM_ERR_STATE";
        case GM_ERR_TIMEOUT: return "GM_ERR_TIMEOUT";
        case GM_ERR_UNSUPPORTED: return "GM_ERR_UNSUPPORTED";
    }
    return "GM_ERR_UNKNOWN";
}

const char* gm_last_error(void) { return gm::last_error(); }

}  // extern "C"

namespace gm {

__global__ void expand_rows_kernel(const int32_t* __restrict__ ptr, int64_t n, int32_t* __restrict__ out) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    for (int32_t e = ptr[v]; e < ptr[v + 1]; ++e) out[e] = (int32_t)v;
}

gm_status expand_rows(const int32_t* ptr, int64_t n, int32_t* out, cudaStream_t s) {
    if (n <= 0) return GM_OK;
    expand_rows_kernel<<<blocks_for(n), 256, 0, s>>>(ptr, n, out);
    LAUNCH_CHECK();
    return GM_OK;
}

void release_graph(gm_graph* g) {
    cudaStream_t s = g->stream;
    trav_release(g);
    wpr_release(g);
    cf_release(g);
    pr_release(g);
    DevBuf* bufs[] = {&g->row_ptr, &g->col, &g->w, &g->col_ptr, &g->row, &g->cw, &g->cw8, &g->csc_pos,
                      &g->out_deg, &g->in_deg, &g->out_bin, &g->in_bin, &g->in_list, &g->zero_in_list,
                      &g->out_list, &g->zero_out_list, &g->dc_jc, &g->dc_cp, &g->dc_tile, &g->dc_head,
                      &g->src_rank, &g->row_r, &g->oct_w, &g->oct_meta, &g->oct_c0, &g->dc_rank, &g->state, &g->work, &g->ctl_buf,
                      &g->reached_buf};
    for (DevBuf* b : bufs) dev_free(*b, s);
    if (g->host_pinned) cudaFreeHost(g->host_pinned);
    cudaStreamSynchronize(s);
    delete g;
}

}  // namespace gm
