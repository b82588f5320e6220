// Device-wide primitives used by graph ingest: exclusive scan, stable LSD radix
// sort of (uint64 key, uint32 value) pairs, and index compaction.  Written for
// sm_103a: 32-wide warps, warp match/ballot for stable digit ranking.
#include <algorithm>
#include <cstdarg>
#include <cstdio>

#include <atomic>
#include <mutex>

#include "gm_internal.cuh"

namespace gm {

std::atomic<uint64_t> g_launches{0};

static thread_local char t_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
}

const char* last_error() { return t_err; }

// Test hook: >= 0 allocations left before every further one fails (see
// gm_debug_fail_allocations_after); < 0 disables.
std::atomic<int64_t> g_alloc_budget{-1};

// The library's stream-ordered memory pool on the current device, created on
// first use.  Freed memory stays in the pool, up to an eighth of the device's
// memory, so the next graph build or program set reuses it instead of mapping
// new pages: graph ingest allocates and frees gigabytes of temporaries, and the
// default pool hands them back to the system at every synchronisation
// (RMAT-22: graph creation 25.6 -> 17.0 ms).  An allocation the pool cannot
// satisfy trims the pool and is tried once more.  nullptr: no pool (the
// default pool is used).
cudaMemPool_t library_pool() {
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDev] = {};
    static bool tried[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!tried[dev]) {
        tried[dev] = true;
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            size_t free_b = 0, total_b = 0;
            uint64_t keep = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess ? (uint64_t)total_b / 8 : 0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            pools[dev] = pool;
        } else {
            cudaGetLastError();  // fall back to the default pool
        }
    }
    return pools[dev];
}

gm_status dev_alloc(DevBuf& b, size_t bytes, cudaStream_t s) {
    dev_free(b, s);
    if (bytes == 0) bytes = 16;
    for (int64_t left = g_alloc_budget.load(); left >= 0;) {
        if (left == 0) {
            set_error("device allocation of %zu bytes failed: injected by gm_debug_fail_allocations_after", bytes);
            return GM_ERR_OUT_OF_MEMORY;
        }
        if (g_alloc_budget.compare_exchange_weak(left, left - 1)) break;
    }
    cudaMemPool_t pool = library_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&b.p, bytes, pool, s) : cudaMallocAsync(&b.p, bytes, s);
    if (e == cudaErrorMemoryAllocation && pool) {  // give the cached memory back and try once more
        cudaGetLastError();
        cudaStreamSynchronize(s);
        cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocFromPoolAsync(&b.p, bytes, pool, s);
    }
    if (e != cudaSuccess) {
        b.p = nullptr;
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GM_ERR_OUT_OF_MEMORY : GM_ERR_CUDA;
    }
    b.bytes = bytes;
    return GM_OK;
}

void dev_free(DevBuf& b, cudaStream_t s) {
    if (b.p) cudaFreeAsync(b.p, s);
    b.p = nullptr;
    b.bytes = 0;
}

// SM count of the current device, cached per device ordinal (grids sized from
// it must fit the device they run on, e.g. a cooperative launch).
int num_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cacheable = dev >= 0 && dev < kMaxDev;
    int sms = cacheable ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (sms == 0) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        if (cacheable) cache[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

// ------------------------------------------------------------------------------
// Exclusive scan (three phases: tile sums, scan of tile sums, tile scans).
// ------------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096 values per CTA

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* smem_warp, uint32_t& excl) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = warp_incl_scan(v);
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < (kScanThreads / 32) ? smem_warp[lane] : 0;
        uint32_t ti = warp_incl_scan(t);
        if (lane < (kScanThreads / 32)) smem_warp[lane] = ti - t;
        if (lane == 31) smem_warp[kScanThreads / 32] = ti;
    }
    __syncthreads();
    excl = smem_warp[warp] + incl - v;
    uint32_t total = smem_warp[kScanThreads / 32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_sums(const uint32_t* __restrict__ in, int64_t n,
                                                               uint32_t* __restrict__ sums) {
    __shared__ uint32_t sw[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) acc += in[i];
    }
    uint32_t excl;
    uint32_t tot = block_excl_scan(acc, sw, excl);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Each thread scans kScanItems consecutive values (blocked arrangement).
__global__ void __launch_bounds__(kScanThreads) scan_tiles(const uint32_t* __restrict__ in, int64_t n,
                                                           const uint32_t* __restrict__ tile_off,
                                                           uint32_t* __restrict__ out, int write_total) {
    __shared__ uint32_t sw[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : 0u;
        acc += v[k];
    }
    uint32_t excl;
    uint32_t tot = block_excl_scan(acc, sw, excl);
    uint32_t run = excl + (tile_off ? tile_off[blockIdx.x] : 0u);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (write_total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) {
        out[n] = (tile_off ? tile_off[blockIdx.x] : 0u) + tot;
    }
}

gm_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        GM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint32_t), s));
        return GM_OK;
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        scan_tiles<<<1, kScanThreads, 0, s>>>(in, n, nullptr, out, 1);
        g_launches++;
        GM_CUDA_TRY(cudaGetLastError());
        return GM_OK;
    }
    DevBuf sums, offs;
    GM_TRY(dev_alloc(sums, sizeof(uint32_t) * tiles, s));
    gm_status st = dev_alloc(offs, sizeof(uint32_t) * (tiles + 1), s);
    if (st != GM_OK) { dev_free(sums, s); return st; }
    scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, as<uint32_t>(sums));
    g_launches++;
    st = scan_exclusive_u32(as<uint32_t>(sums), as<uint32_t>(offs), tiles, s);
    if (st == GM_OK) {
        scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, as<uint32_t>(offs), out, 1);
        g_launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { set_error("scan: %s", cudaGetErrorString(e)); st = GM_ERR_CUDA; }
    }
    dev_free(sums, s);
    dev_free(offs, s);
    return st;
}

// ------------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits, one kernel per pass.  Before the passes,
// one kernel counts every pass's digits over all keys (the digit order does not
// change a digit's total), which gives each digit's first output position.  A
// pass then needs, per tile and digit, the count of that digit in all earlier
// tiles: each tile publishes its own counts as soon as it has ranked its keys,
// and looks back over the tiles before it, adding their counts until it finds
// one that has already published a running total (decoupled look-back).  Tiles
// take their numbers from an atomic counter in the order they start, so the
// tiles a tile waits for are running or done.  The waits are bounded; a tile
// that gives up writes nothing and the sort reports GM_ERR_TIMEOUT.
// Within a tile, keys are ranked with __match_any_sync (warp w owns a
// contiguous sub-range of the tile and walks it 32 keys at a time in input
// order), placed digit by digit in shared memory, and written out from there in
// order: consecutive threads write consecutive positions of each digit's run.
// ------------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 15;  // 32-key rounds per warp: 3840-key tiles, 55 KB of shared memory, 4 CTAs per SM
constexpr int kSortTile = kSortThreads * kSortRounds;     // keys per CTA
constexpr int kRadix = 256;
constexpr int kMaxSortPasses = 8;
// dynamic shared memory of a pass: the tile's keys and values, per-warp digit
// counts, the tile's digit offsets
constexpr size_t kScatterSmem = (size_t)kSortTile * (sizeof(uint64_t) + sizeof(uint32_t)) +
                                sizeof(uint32_t) * (kSortWarps * kRadix + 2 * kRadix);
// A tile's status word per digit: the pass's tag (pass + 1) in bits 56-63, what
// the value is in bits 54-55 (1: the tile's own count, 2: the total over this
// tile and all before it), the value in bits 0-53.  Words of an earlier pass
// carry another tag and read as "not yet published".
constexpr uint64_t kStTagMask = 0xFFull << 56;
constexpr uint64_t kStOwn = 1ull << 54, kStTotal = 2ull << 54, kStKind = 3ull << 54;
constexpr uint64_t kStValue = (1ull << 54) - 1ull;

__global__ void __launch_bounds__(kSortThreads) radix_hist_all(const uint64_t* __restrict__ keys, int64_t n,
                                                               int passes, uint32_t* __restrict__ ghist) {
    __shared__ uint32_t h[kMaxSortPasses * kRadix];
    for (int i = threadIdx.x; i < kMaxSortPasses * kRadix; i += kSortThreads) h[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kSortThreads) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p * kRadix + (int)((k >> (8 * p)) & 0xFF)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads)
        if (h[i]) atomicAdd(&ghist[i], h[i]);
}

// First output position of every digit of every pass (exclusive scan over digits).
__global__ void __launch_bounds__(kSortThreads) radix_bases(const uint32_t* __restrict__ ghist, int passes,
                                                            uint32_t* __restrict__ gbase) {
    __shared__ uint32_t sw[kScanThreads / 32 + 1];
    for (int p = 0; p < passes; ++p) {
        uint32_t excl;
        block_excl_scan(ghist[p * kRadix + threadIdx.x], sw, excl);
        gbase[p * kRadix + threadIdx.x] = excl;
    }
}

__device__ __forceinline__ uint64_t sort_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kSortThreads) radix_pass(const uint64_t* __restrict__ keys_in,
                                                           const uint32_t* __restrict__ vals_in, int64_t n,
                                                           int shift, uint64_t tag,
                                                           const uint32_t* __restrict__ gbase,
                                                           unsigned long long* status, uint32_t* tile_ctr,
                                                           uint64_t* __restrict__ keys_out,
                                                           uint32_t* __restrict__ vals_out, uint32_t* err) {
    extern __shared__ __align__(16) unsigned char sort_smem[];
    uint64_t* skey = reinterpret_cast<uint64_t*>(sort_smem);
    uint32_t* sval = reinterpret_cast<uint32_t*>(skey + kSortTile);
    uint32_t (*wcnt)[kRadix] = reinterpret_cast<uint32_t (*)[kRadix]>(sval + kSortTile);
    uint32_t* toff = &wcnt[kSortWarps][0];  // digit offsets inside the tile
    uint32_t* goff = toff + kRadix;         // digit offsets in the output
    __shared__ uint32_t s_tile, s_gave_up;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(tile_ctr, 1u);
        s_gave_up = 0u;
    }
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();

    const int64_t tile = s_tile;
    const int64_t tbase = tile * kSortTile;
    const int64_t tlen = min((int64_t)kSortTile, n - tbase);  // keys in this tile
    const int wofs = warp * (32 * kSortRounds);                // the warp's sub-range in the tile
    uint32_t rank[kSortRounds];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int j = wofs + r * 32 + lane;
        const bool valid = j < tlen;
        const uint64_t k = valid ? keys_in[tbase + j] : 0ull;
        // invalid lanes get a digit value no valid key has (256)
        const uint32_t d = valid ? (uint32_t)((k >> shift) & 0xFF) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t base = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        rank[r] = 0u;
        if (valid) {
            rank[r] = base + __popc(peers & lt_mask);
            if (lane == __ffs(peers) - 1) wcnt[warp][d] = base + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit (thread = digit): exclusive prefix over warps, and the tile's count
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = tot;
        tot += c;
    }
    volatile unsigned long long* mine = status + tile * kRadix + threadIdx.x;
    *mine = tag | (tile == 0 ? kStTotal : kStOwn) | tot;
    // exclusive scan of the digit counts over the CTA (kRadix == kSortThreads)
    uint32_t my_toff;
    {
        uint32_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        toff[threadIdx.x] = x;  // inclusive within the warp
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < warp; ++w) add += toff[w * 32 + 31];
        __syncthreads();
        my_toff = add + x - tot;  // exclusive over the CTA
    }
    // each warp's first position for this digit inside the tile (one shared read per key below)
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) wcnt[w][threadIdx.x] += my_toff;
    // look back: this digit's count in all earlier tiles
    uint64_t before = 0;
    if (tile > 0) {
        int64_t j = tile - 1;
        const uint64_t t0 = sort_ns();
        for (uint32_t tries = 0;;) {
            const unsigned long long v = reinterpret_cast<volatile unsigned long long*>(status)[j * kRadix + threadIdx.x];
            if ((v & kStTagMask) == tag && (v & kStKind) != 0ull) {
                before += v & kStValue;
                if ((v & kStKind) == kStTotal || j == 0) break;
                --j;
                continue;
            }
            if (++tries > (1u << 22) || ((tries & 63u) == 0u && sort_ns() - t0 > 1000000000ull)) {
                s_gave_up = 1u;
                atomicOr(err, 1u);
                break;
            }
            __nanosleep(32);
        }
        *mine = tag | kStTotal | (before + tot);
    }
    // output position of tile position lp of this digit = goff[digit] + lp (mod 2^32)
    goff[threadIdx.x] = gbase[threadIdx.x] + (uint32_t)before - my_toff;
    __syncthreads();
    if (s_gave_up) return;
    // place each key at its position inside the tile (digit-major, stable)
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int j = wofs + r * 32 + lane;
        if (j < tlen) {
            const uint64_t k = keys_in[tbase + j];
            const uint32_t d = (uint32_t)((k >> shift) & 0xFF);
            const uint32_t lp = wcnt[warp][d] + rank[r];
            skey[lp] = k;
            sval[lp] = vals_in[tbase + j];
        }
    }
    __syncthreads();
    // write out in tile order: position = the digit's output offset + the rank in its run
    for (int lp = threadIdx.x; lp < tlen; lp += kSortThreads) {
        const uint64_t k = skey[lp];
        const uint32_t d = (uint32_t)((k >> shift) & 0xFF);
        const uint32_t pos = goff[d] + (uint32_t)lp;
        if (pos < (uint64_t)n) {
            keys_out[pos] = k;
            vals_out[pos] = sval[lp];
        }
    }
}

gm_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                           int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return GM_OK;
    if (n >= (int64_t)0xFFFFFFFFll) {
        set_error("radix sort: %lld keys, at most 2^32 - 2", (long long)n);
        return GM_ERR_INVALID_ARG;
    }
    static const cudaError_t attr_ok =
        cudaFuncSetAttribute(radix_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
    if (attr_ok != cudaSuccess) { set_error("radix sort: %s", cudaGetErrorString(attr_ok)); return GM_ERR_CUDA; }
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    const int passes = std::min((bits + 7) / 8, kMaxSortPasses);
    // ghist, gbase (passes x kRadix each), a tile counter per pass, the error flag
    const size_t meta_words = 2 * (size_t)kMaxSortPasses * kRadix + kMaxSortPasses + 1;
    DevBuf meta, status;
    GM_TRY(dev_alloc(meta, sizeof(uint32_t) * meta_words, s));
    gm_status st = dev_alloc(status, sizeof(unsigned long long) * kRadix * (size_t)tiles, s);
    if (st != GM_OK) { dev_free(meta, s); return st; }
    uint32_t* ghist = as<uint32_t>(meta);
    uint32_t* gbase = ghist + kMaxSortPasses * kRadix;
    uint32_t* ctr = gbase + kMaxSortPasses * kRadix;
    uint32_t* err = ctr + kMaxSortPasses;
    cudaError_t e = cudaMemsetAsync(meta.p, 0, sizeof(uint32_t) * meta_words, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status.p, 0, sizeof(unsigned long long) * kRadix * (size_t)tiles, s);
    if (e == cudaSuccess) {
        const int64_t hb = std::min<int64_t>(tiles, (int64_t)num_sms() * 4);
        radix_hist_all<<<(unsigned)hb, kSortThreads, 0, s>>>(keys, n, passes, ghist);
        radix_bases<<<1, kSortThreads, 0, s>>>(ghist, passes, gbase);
        g_launches += 2;
        e = cudaGetLastError();
    }
    uint64_t* kin = keys; uint32_t* vin = vals;
    uint64_t* kout = keys_alt; uint32_t* vout = vals_alt;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        radix_pass<<<(unsigned)tiles, kSortThreads, kScatterSmem, s>>>(
            kin, vin, n, 8 * p, (uint64_t)(p + 1) << 56, gbase + p * kRadix,
            as<unsigned long long>(status), ctr + p, kout, vout, err);
        g_launches++;
        e = cudaGetLastError();
        uint64_t* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    if (e == cudaSuccess && kin != keys) {
        e = cudaMemcpyAsync(keys, kin, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, vin, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
    uint32_t h_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(meta, s);
    dev_free(status, s);
    if (e != cudaSuccess) {
        set_error("radix sort: %s", cudaGetErrorString(e));
        return GM_ERR_CUDA;
    }
    if (h_err) {
        set_error("radix sort: a tile waited more than a second for the tiles before it");
        return GM_ERR_TIMEOUT;
    }
    return GM_OK;
}

// ------------------------------------------------------------------------------
// Compaction of flagged indices (stable).
// ------------------------------------------------------------------------------
__global__ void compact_scatter(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos,
                                int64_t n, int32_t* __restrict__ out, uint32_t* __restrict__ count_dev) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flags[i]) out[pos[i]] = (int32_t)i;
    if (i == 0) *count_dev = pos[n];
}

gm_status compact_indices(const uint32_t* flags, int64_t n, int32_t* out, uint32_t* count_dev,
                          cudaStream_t s) {
    DevBuf pos;
    GM_TRY(dev_alloc(pos, sizeof(uint32_t) * (n + 1), s));
    gm_status st = scan_exclusive_u32(flags, as<uint32_t>(pos), n, s);
    if (st == GM_OK) {
        int64_t blocks = (n + 255) / 256;
        if (blocks == 0) blocks = 1;
        compact_scatter<<<(unsigned)blocks, 256, 0, s>>>(flags, as<uint32_t>(pos), n, out, count_dev);
        g_launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { set_error("compact: %s", cudaGetErrorString(e)); st = GM_ERR_CUDA; }
    }
    dev_free(pos, s);
    return st;
}

}  // namespace gm
