// Collaborative filtering by stochastic gradient descent (Section 3.III: the
// updates of Eqs. 4-5 without their sums, applied one rating at a time, each
// from the factor values before that rating):
//   e   = G_uv - p_u . p_v
//   p_u = p_u + gamma (e p_v - lambda p_u)
//   p_v = p_v + gamma (e p_u - lambda p_v)
//
// Order.  Section 3.III asks for a random order; one serial order has no
// parallelism, so the ratings run in the stratified order of distributed SGD
// (Gemulla, Nijkamp, Haas and Sismanis, KDD 2011).  User u lies in block
// u mod P, item v in block (v - n_left) mod P, and the rating (u, v) in stratum
// (item block - user block) mod P.  An epoch runs the strata 0..P-1 in turn.
// The P blocks of a stratum (user block b with item block (b + s) mod P) share
// no user and no item, so they run at the same time, one warp each, and give
// the factors of the serial order -- strata, then user blocks, then ratings in
// (user, item) order -- up to FP32 rounding.
//
// Layout.  gm_program_set sorts the ratings once (stable radix sort on stratum
// and user block) into 16-byte records {user, item slot in its block, rating,
// item}, with the first record of every (stratum, block) in blk[s * P + b].
//
// Kernel.  One cooperative launch runs every epoch.  Lane k of a warp holds
// factor component k (and k + 32 when K > 32).  A warp copies its block's item
// rows into its part of shared memory (when they fit; else it works on them in
// L2), keeps the current user and the item last used in registers, and loads
// the user rows of the next window of ratings one window ahead: a user's row is
// not written in a stratum before its first rating there, and no other warp
// touches it in that stratum.  Every lane reads and writes only its own
// components, in shared memory too, so a warp needs no barrier of its own.
// The critical path of an epoch is the chain of updates of the most-rated
// item: its ratings are serial in every order that reproduces serial SGD.
// Strata are separated by a grid barrier whose wait gives up after about ten
// seconds (or 2^30 tries), sets an error flag and ends the kernel; the host
// then returns GM_ERR_TIMEOUT.  The test option GM_OPT_TEST_STALL_SGD keeps one
// CTA from arriving at the first barrier and cuts the limit to half a second.
#include <algorithm>
#include <cmath>

#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kSgdThreads = 256;
constexpr int kSgdWarps = kSgdThreads / 32;
constexpr uint32_t kFull = 0xffffffffu;
constexpr int32_t kMaxStrata = 4096;
constexpr size_t kSgdSmemCap = 192 * 1024;  // item rows per CTA

struct SgdSync {
    unsigned count, gen, error, pad;
};

struct SgdState {
    DevBuf rec, blk, sync;
    int32_t P = 0;
    int32_t J = 0;  // items in the largest item block
    bool smem = false;
    int grid = 0;
    size_t smem_bytes = 0;
};

__device__ __forceinline__ uint64_t sgd_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Stratum and user block of every rating, packed as (user << 32) | (s * P + bu),
// its edge index, and the rating count of every (stratum, block).  One warp per
// user row.  Ratings whose item is not in [n_left, n) are counted in *bad.
__global__ void sgd_keys(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t n_left,
                         int64_t n, int32_t P, uint64_t* __restrict__ key, uint32_t* __restrict__ val,
                         uint32_t* __restrict__ count, uint32_t* __restrict__ bad) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n_left; u += nw) {
        const int64_t bu = u % P;
        const int64_t e1 = row_ptr[u + 1];
        for (int64_t e = row_ptr[u] + lane; e < e1; e += 32) {
            const int64_t v = col[e];
            uint32_t k = 0;
            if (v < n_left || v >= n) {
                atomicAdd(bad, 1u);
            } else {
                const int64_t s = ((v - n_left) % P - bu + P) % P;
                k = (uint32_t)(s * P + bu);
            }
            key[e] = ((uint64_t)u << 32) | k;
            val[e] = (uint32_t)e;
            atomicAdd(count + k, 1u);
        }
    }
}

__global__ void sgd_records(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, int64_t m,
                            const int32_t* __restrict__ col, const uint32_t* __restrict__ w, int64_t n_left,
                            int32_t P, int4* __restrict__ rec) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = val[i];
        const int32_t v = col[e];
        rec[i] = make_int4((int32_t)(key[i] >> 32), (int32_t)((v - n_left) / P), __float_as_int((float)w[e]), v);
    }
}

// Grid barrier between strata (all CTAs are resident: cooperative launch).
// Returns false, with the error flag set, when the wait gave up or another CTA
// gave up.  The wait gives up after wait_ns by the global timer or 2^30 tries.
// `skip_arrival` (the test hook) makes this CTA wait without arriving, so no
// CTA's wait can end but by its limit.
__device__ __forceinline__ bool sgd_grid_sync(SgdSync* sy, unsigned& gen, int* s_ok, bool skip_arrival,
                                              uint64_t wait_ns) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = gen + 1u;
        int ok = 1;
        if (!skip_arrival && atomicAdd(&sy->count, 1u) == gridDim.x - 1u) {
            atomicExch(&sy->count, 0u);
            __threadfence();
            atomicExch(&sy->gen, target);
        } else {
            const uint64_t t0 = sgd_ns();
            for (uint32_t i = 0;; ++i) {
                if (*(volatile unsigned*)&sy->gen == target) break;
                if (*(volatile unsigned*)&sy->error != 0u) { ok = 0; break; }
                if (i >= (1u << 30) || ((i & 63u) == 63u && sgd_ns() - t0 > wait_ns)) {
                    atomicExch(&sy->error, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        gen = target;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <int KL>
__device__ __forceinline__ void load_row(const float* __restrict__ row, int lane, int K, float (&x)[KL]) {
#pragma unroll
    for (int c = 0; c < KL; ++c) {
        const int k = lane + 32 * c;
        x[c] = k < K ? __ldcg(row + k) : 0.0f;
    }
}

template <int KL>
__device__ __forceinline__ void store_row(float* __restrict__ row, int lane, int K, const float (&x)[KL]) {
#pragma unroll
    for (int c = 0; c < KL; ++c) {
        const int k = lane + 32 * c;
        if (k < K) __stcg(row + k, x[c]);
    }
}

// The ratings [lo, hi) of one block; item block bv.  W ratings per window.
template <int KL, bool kSmem>
__device__ __forceinline__ void sgd_block(const int4* __restrict__ rec, uint32_t lo, uint32_t hi, int64_t bv,
                                          int32_t P, float* __restrict__ p, int64_t n_left, int64_t n_items,
                                          int K, float gamma, float lambda, float* __restrict__ my, int lane) {
    constexpr int W = 32 / KL;
    const int64_t item0 = n_left + bv;  // item of slot j: item0 + j * P
    const int32_t Jb = bv < n_items ? (int32_t)((n_items - 1 - bv) / P + 1) : 0;
    if (kSmem) {
#pragma unroll 4
        for (int32_t j = 0; j < Jb; ++j) {
            const float* row = p + (item0 + (int64_t)j * P) * K;
#pragma unroll
            for (int c = 0; c < KL; ++c) {
                const int k = lane + 32 * c;
                if (k < K) my[j * K + k] = __ldcg(row + k);
            }
        }
    }
    const uint32_t n = hi - lo;
    const int4 none = make_int4(-1, 0, 0, 0);
    int4 ra = (uint32_t)lane < min(n, (uint32_t)W) ? __ldg(rec + lo + lane) : none;
    int4 rb = (lane < W && (uint32_t)(W + lane) < n) ? __ldg(rec + lo + W + lane) : none;
    float pre_a[W][KL], pre_b[W][KL];
#pragma unroll
    for (int t = 0; t < W; ++t) {
        const int u = __shfl_sync(kFull, ra.x, t);
        if (u >= 0) load_row<KL>(p + (int64_t)u * K, lane, K, pre_a[t]);
    }
    int cur_u = -1, cur_j = -1;
    float pu[KL], pv[KL];
#pragma unroll
    for (int c = 0; c < KL; ++c) pu[c] = pv[c] = 0.0f;
    for (uint32_t base = 0; base < n; base += W) {
        const uint32_t cnt = min(n - base, (uint32_t)W);
        // one window ahead: the next window's user rows, two ahead: its records
#pragma unroll
        for (int t = 0; t < W; ++t) {
            const int u = __shfl_sync(kFull, rb.x, t);
            if (u >= 0) load_row<KL>(p + (int64_t)u * K, lane, K, pre_b[t]);
        }
        const int4 rc = (lane < W && base + 2 * W + lane < n) ? __ldg(rec + lo + base + 2 * W + lane) : none;
#pragma unroll
        for (int t = 0; t < W; ++t) {
            if ((uint32_t)t < cnt) {
                const int u = __shfl_sync(kFull, ra.x, t);
                const int j = __shfl_sync(kFull, ra.y, t);
                const float g = __int_as_float(__shfl_sync(kFull, ra.z, t));
                if (u != cur_u) {
                    if (cur_u >= 0) store_row<KL>(p + (int64_t)cur_u * K, lane, K, pu);
#pragma unroll
                    for (int c = 0; c < KL; ++c) pu[c] = pre_a[t][c];
                    cur_u = u;
                }
                if (j != cur_j) {
#pragma unroll
                    for (int c = 0; c < KL; ++c) {
                        const int k = lane + 32 * c;
                        if (kSmem) {
                            if (k < K) {
                                if (cur_j >= 0) my[cur_j * K + k] = pv[c];
                                pv[c] = my[j * K + k];
                            }
                        } else {
                            if (k < K) {
                                if (cur_j >= 0) __stcg(p + (item0 + (int64_t)cur_j * P) * K + k, pv[c]);
                                pv[c] = __ldcg(p + (item0 + (int64_t)j * P) * K + k);
                            }
                        }
                    }
                    cur_j = j;
                }
                float d = 0.0f;
#pragma unroll
                for (int c = 0; c < KL; ++c) d = fmaf(pu[c], pv[c], d);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
                const float e = g - d;
#pragma unroll
                for (int c = 0; c < KL; ++c) {
                    const float a = pu[c], b = pv[c];
                    pu[c] = a + gamma * (e * b - lambda * a);
                    pv[c] = b + gamma * (e * a - lambda * b);
                }
            }
        }
        ra = rb;
        rb = rc;
#pragma unroll
        for (int t = 0; t < W; ++t)
#pragma unroll
            for (int c = 0; c < KL; ++c) pre_a[t][c] = pre_b[t][c];
    }
    if (cur_u >= 0) store_row<KL>(p + (int64_t)cur_u * K, lane, K, pu);
    if (cur_j >= 0) {
#pragma unroll
        for (int c = 0; c < KL; ++c) {
            const int k = lane + 32 * c;
            if (k < K) {
                if (kSmem) my[cur_j * K + k] = pv[c];
                else __stcg(p + (item0 + (int64_t)cur_j * P) * K + k, pv[c]);
            }
        }
    }
    if (kSmem) {
#pragma unroll 4
        for (int32_t j = 0; j < Jb; ++j) {
            float* row = p + (item0 + (int64_t)j * P) * K;
#pragma unroll
            for (int c = 0; c < KL; ++c) {
                const int k = lane + 32 * c;
                if (k < K) __stcg(row + k, my[j * K + k]);
            }
        }
    }
}

template <int KL, bool kSmem>
__global__ void __launch_bounds__(kSgdThreads, 1)
    cf_sgd_epochs(const int4* __restrict__ rec, const uint32_t* __restrict__ blk, int32_t P, int32_t J,
                  float* __restrict__ p, int64_t n_left, int64_t n_items, int K, float gamma, float lambda,
                  int32_t epochs, SgdSync* __restrict__ sync, int32_t stall_cta, uint64_t wait_ns) {
    extern __shared__ float sgd_items[];
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t warp = (int64_t)blockIdx.x * kSgdWarps + wib;
    const int64_t nwarps = (int64_t)gridDim.x * kSgdWarps;
    float* my = kSmem ? sgd_items + (size_t)wib * J * K : nullptr;
    unsigned gen = 0;
    for (int32_t ep = 0; ep < epochs; ++ep) {
        for (int32_t s = 0; s < P; ++s) {
            for (int64_t b = warp; b < P; b += nwarps) {
                const uint32_t lo = blk[(int64_t)s * P + b], hi = blk[(int64_t)s * P + b + 1];
                if (lo < hi)
                    sgd_block<KL, kSmem>(rec, lo, hi, (b + s) % P, P, p, n_left, n_items, K, gamma, lambda, my,
                                         lane);
            }
            const bool skip = (int32_t)blockIdx.x == stall_cta && gen == 0u;  // test hook: first barrier only
            if (!sgd_grid_sync(sync, gen, &s_ok, skip, wait_ns)) return;
        }
    }
}

template <int KL, bool kSmem>
gm_status sgd_launch(const SgdState* st, gm_graph* g, int32_t epochs) {
    const int4* rec = as<int4>(st->rec);
    const uint32_t* blk = as<uint32_t>(st->blk);
    int32_t P = st->P, J = st->J;
    float* p = as<float>(g->state);
    int64_t n_left = g->n_left, n_items = g->n - g->n_left;
    int K = g->params.K;
    float gamma = (float)g->params.gamma, lambda = (float)g->params.lambda;
    SgdSync* sync = as<SgdSync>(st->sync);
    // the barrier's wait limit: about ten seconds (a stratum of a very skewed
    // matrix may legitimately take long), half a second under the test hook,
    // which keeps the last CTA from arriving at the first barrier
    int32_t stall_cta = g->tune.test_stall_sgd ? st->grid - 1 : -1;
    uint64_t wait_ns = g->tune.test_stall_sgd ? 500000000ull : 10000000000ull;
    void* args[] = {&rec, &blk, &P, &J, &p, &n_left, &n_items, &K, &gamma, &lambda, &epochs, &sync,
                    &stall_cta, &wait_ns};
    GM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)cf_sgd_epochs<KL, kSmem>, dim3(st->grid),
                                            dim3(kSgdThreads), args, st->smem_bytes, g->stream));
    g_launches++;
    return GM_OK;
}

template <typename F>
gm_status by_variant(int K, bool smem, F f) {
    if (K <= 32) return smem ? f(std::integral_constant<int, 1>(), std::true_type())
                             : f(std::integral_constant<int, 1>(), std::false_type());
    return smem ? f(std::integral_constant<int, 2>(), std::true_type())
                : f(std::integral_constant<int, 2>(), std::false_type());
}

template <int KL, bool kSmem>
gm_status sgd_configure(SgdState* st) {
    const auto kern = cf_sgd_epochs<KL, kSmem>;
    // opt in whenever rows go to shared memory: without it, dynamic plus static
    // shared memory must stay within 48 KB (an exactly 48 KB request does not fit)
    if (kSmem)
        GM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st->smem_bytes));
    int per_sm = 0;
    GM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSgdThreads, st->smem_bytes));
    if (per_sm < 1) {
        set_error("gm_program_set: the SGD kernel does not fit on an SM");
        return GM_ERR_UNSUPPORTED;
    }
    const int64_t want = ((int64_t)st->P + kSgdWarps - 1) / kSgdWarps;
    st->grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * num_sms()));
    return GM_OK;
}

// Blocks per side when the caller leaves the choice: about sqrt(m) / 10 rounded
// to a power of two.  Fewer, longer strata cost fewer grid barriers; more
// strata spread the most-rated items' ratings over more, shorter blocks.  On
// the 100M-rating, 480,000 x 17,800 workload P = 128 / 256 / 512 / 1024 / 2048
// took 290 / 205 / 167 / 151 / 162 ms per epoch.
int32_t default_strata(int64_t m) {
    const double x = std::sqrt((double)std::max<int64_t>(m, 1)) / 10.0;
    int32_t P = 1;
    while (P < kMaxStrata && (double)P * 1.41421356 < x) P *= 2;
    return P;
}

}  // namespace

void sgd_release(void* state, cudaStream_t s) {
    SgdState* st = static_cast<SgdState*>(state);
    if (!st) return;
    dev_free(st->rec, s);
    dev_free(st->blk, s);
    dev_free(st->sync, s);
    delete st;
}

gm_status sgd_prepare(gm_graph* g, void** out) {
    cudaStream_t s = g->stream;
    const int64_t m = g->m, n = g->n, n_left = g->n_left, n_items = n - n_left;
    const int K = g->params.K;
    int32_t P = g->params.cf_strata;
    if (P < 0 || P > kMaxStrata) {
        set_error("gm_program_set: cf_strata outside [0, %d]", kMaxStrata);
        return GM_ERR_INVALID_ARG;
    }
    if (m >= (int64_t)UINT32_MAX) {
        set_error("gm_program_set: SGD supports fewer than 2^32 ratings");
        return GM_ERR_UNSUPPORTED;
    }
    int32_t users_end = 0;
    GM_CUDA_TRY(cudaMemcpyAsync(&users_end, as<int32_t>(g->row_ptr) + n_left, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    if ((int64_t)users_end != m) {
        set_error("gm_program_set: SGD needs every rating to go from a user [0, n_left) to an item");
        return GM_ERR_INVALID_ARG;
    }
    if (P == 0) P = default_strata(m);
    SgdState* st = new (std::nothrow) SgdState();
    if (!st) { set_error("gm_program_set: host allocation failed"); return GM_ERR_OUT_OF_MEMORY; }
    *out = st;
    st->P = P;
    st->J = (int32_t)((n_items + P - 1) / P);
    const size_t rows = (size_t)kSgdWarps * (size_t)st->J * (size_t)K * sizeof(float);
    st->smem = rows <= kSgdSmemCap;
    st->smem_bytes = st->smem ? rows : 0;
    GM_TRY(by_variant(K, st->smem, [&](auto kl, auto sm) { return sgd_configure<decltype(kl)::value, decltype(sm)::value>(st); }));
    const int64_t nb = (int64_t)P * P;
    GM_TRY(dev_alloc(st->rec, sizeof(int4) * (size_t)std::max<int64_t>(m, 1), s));
    GM_TRY(dev_alloc(st->blk, sizeof(uint32_t) * (size_t)(nb + 1), s));
    GM_TRY(dev_alloc(st->sync, sizeof(SgdSync), s));
    DevBuf key, key_alt, val, val_alt, count, bad;
    auto release = [&] {
        dev_free(key, s); dev_free(key_alt, s); dev_free(val, s); dev_free(val_alt, s);
        dev_free(count, s); dev_free(bad, s);
    };
    gm_status r = GM_OK;
    const size_t mm = (size_t)std::max<int64_t>(m, 1);
    if (r == GM_OK) r = dev_alloc(key, sizeof(uint64_t) * mm, s);
    if (r == GM_OK) r = dev_alloc(key_alt, sizeof(uint64_t) * mm, s);
    if (r == GM_OK) r = dev_alloc(val, sizeof(uint32_t) * mm, s);
    if (r == GM_OK) r = dev_alloc(val_alt, sizeof(uint32_t) * mm, s);
    if (r == GM_OK) r = dev_alloc(count, sizeof(uint32_t) * (size_t)nb, s);
    if (r == GM_OK) r = dev_alloc(bad, sizeof(uint32_t), s);
    if (r != GM_OK) { release(); return r; }
    uint32_t h_bad = 0;
    cudaError_t ce = cudaMemsetAsync(count.p, 0, sizeof(uint32_t) * (size_t)nb, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(bad.p, 0, sizeof(uint32_t), s);
    if (ce == cudaSuccess && m > 0) {
        sgd_keys<<<num_sms() * 8, 256, 0, s>>>(as<int32_t>(g->row_ptr), as<int32_t>(g->col), n_left, n, P,
                                               as<uint64_t>(key), as<uint32_t>(val), as<uint32_t>(count),
                                               as<uint32_t>(bad));
        g_launches++;
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_bad, bad.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
        set_error("gm_program_set (SGD keys): %s", cudaGetErrorString(ce));
        release();
        return GM_ERR_CUDA;
    }
    if (h_bad != 0) {
        set_error("gm_program_set: SGD needs every rating to go from a user to an item in [n_left, n)");
        release();
        return GM_ERR_INVALID_ARG;
    }
    int bits = 0;
    while (bits < 64 && ((uint64_t)1 << bits) < (uint64_t)nb) ++bits;
    r = radix_sort_pairs(as<uint64_t>(key), as<uint32_t>(val), as<uint64_t>(key_alt), as<uint32_t>(val_alt), m,
                         bits, s);
    if (r == GM_OK) r = scan_exclusive_u32(as<uint32_t>(count), as<uint32_t>(st->blk), nb, s);
    if (r == GM_OK && m > 0) {
        sgd_records<<<num_sms() * 8, 256, 0, s>>>(as<uint64_t>(key), as<uint32_t>(val), m, as<int32_t>(g->col),
                                                  as<uint32_t>(g->w), n_left, P, as<int4>(st->rec));
        g_launches++;
        ce = cudaGetLastError();
        if (ce != cudaSuccess) { set_error("gm_program_set (SGD records): %s", cudaGetErrorString(ce)); r = GM_ERR_CUDA; }
    }
    if (r == GM_OK) {
        ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { set_error("gm_program_set (SGD): %s", cudaGetErrorString(ce)); r = GM_ERR_CUDA; }
    }
    release();
    if (r == GM_OK) g->params.cf_strata = P;
    return r;
}

gm_status sgd_run(gm_graph* g, void* state, int32_t epochs) {
    SgdState* st = static_cast<SgdState*>(state);
    cudaStream_t s = g->stream;
    if (epochs == 0 || g->m == 0) return GM_OK;
    GM_CUDA_TRY(cudaMemsetAsync(st->sync.p, 0, sizeof(SgdSync), s));
    GM_TRY(by_variant(g->params.K, st->smem,
                      [&](auto kl, auto sm) { return sgd_launch<decltype(kl)::value, decltype(sm)::value>(st, g, epochs); }));
    SgdSync h{};
    GM_CUDA_TRY(cudaMemcpyAsync(&h, st->sync.p, sizeof(SgdSync), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.error) {
        set_error(g->tune.test_stall_sgd ? "gm_run: an SGD grid barrier wait gave up (test hook: one CTA never arrived)"
                                         : "gm_run: an SGD grid barrier wait gave up (a stratum took over ten seconds)");
        return GM_ERR_TIMEOUT;
    }
    return GM_OK;
}

}  // namespace gm
