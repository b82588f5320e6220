// Collaborative filtering by full-batch gradient descent (Section 3.III, Eqs. 2-5).
//
// Users are vertices [0, n_left), items [n_left, n); every rating is an edge
// user -> item with its value G_uv.  One superstep (Jacobi, all factors of step t):
//   e_uv  = G_uv - p_u . p_v                                   (Eq. 3)
//   p_u  <- p_u + gamma [ sum_v e_uv p_v - lambda p_u ]         (Eq. 4)
//   p_v  <- p_v + gamma [ sum_u e_uv p_u - lambda p_v ]         (Eq. 5)
// As vertex programs: every vertex sends its factor vector, Process_Message
// computes e_uv from the message, the rating and the receiver's own factors
// (the destination-property access Section 4.2 highlights), Reduce sums, and
// Apply takes the gradient step.
//
// Kernels: a user pass over the CSR (one warp per chunk of <= 512 ratings of a
// user; for K = 8, 16, 32, 64 each rating is handled by K/8 lanes with 8 factor
// components each, so a warp has 32/(K/8) ratings in flight, other K spread the
// components over the 32 lanes, one rating at a time) computes and stores e_uv and
// accumulates sum_v e_uv p_v.  Item degrees are skewed, so for K = 8..64 the
// factor rows of the most-rated items are first copied into each CTA's shared
// memory (one 1024-thread CTA per SM; for K = 32, 1792 rows carrying about 57 %
// of the ratings of the Zipf-shaped workload) and each rating's item is stored
// as a code: its row's slot there, or -1 - the item, so the gathers of those
// ratings read shared memory instead of L2; an item pass over the CSC computes
// e_uv again from the rating (a one-byte CSC copy when the ratings fit) and the
// user's row -- the same products summed in the same order by the same lane
// grouping, so the same value -- and accumulates sum_u e_uv p_u; an update
// kernel applies Eqs. 4-5 to every vertex.  Recomputing e_uv costs one more
// K-wide dot product per rating and saves storing it and gathering it back in
// CSC order (a random 4-byte read from a 4-bytes-per-rating array, one 32-byte
// sector per rating).  Chunks of one long row are combined with float atomics.
// Arithmetic in FP32 on CUDA cores: every product is one K-wide dot product per
// rating, not a dense tile.
#include <algorithm>
#include <vector>

#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kFull = 0xffffffffu;
constexpr int kCfChunk = 512;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Counter-based normal draws for the initial factors: SplitMix64 (Steele, Lea
// and Flood, OOPSLA 2014) gives two 53-bit uniforms per value, combined by the
// Box-Muller transform (cosine branch), value index i = vertex * K + k.
__device__ __forceinline__ uint64_t sm_mix(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void cf_init(float* __restrict__ p, int64_t count, uint64_t seed, double sigma) {
    const uint64_t key = sm_mix(seed ^ sm_mix(9ULL * 0xD1B54A32D192ED03ULL));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t w1 = sm_mix(key ^ ((uint64_t)(2 * i) * 0x9E3779B97F4A7C15ULL));
        const uint64_t w2 = sm_mix(key ^ ((uint64_t)(2 * i + 1) * 0x9E3779B97F4A7C15ULL));
        const double u1 = ((double)(w1 >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        const double u2 = (double)(w2 >> 11) * (1.0 / 9007199254740992.0);
        p[i] = (float)(sigma * sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2));
    }
}

// KP = factor components per lane (K <= 32 * KP).
template <int KP>
__global__ void __launch_bounds__(kThreads) cf_user_pass(const int4* __restrict__ chunks, int64_t nchunks,
                                                         const int32_t* __restrict__ col,
                                                         const uint32_t* __restrict__ rating,
                                                         const float* __restrict__ p, int K,
                                                         float* __restrict__ acc,
                                                         double* __restrict__ sq_err) {
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    double sq = 0.0;
    for (int64_t c = gwarp; c < nchunks; c += nwarps) {
        const int4 ch = chunks[c];
        const int32_t u = ch.x;
        float pu[KP], ac[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) {
            const int k = lane + 32 * j;
            pu[j] = k < K ? p[(int64_t)u * K + k] : 0.0f;
            ac[j] = 0.0f;
        }
        for (int32_t e = ch.y; e < ch.z; ++e) {
            const int32_t v = __ldg(col + e);
            float pv[KP];
            float part = 0.0f;
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                const int k = lane + 32 * j;
                pv[j] = k < K ? __ldg(p + (int64_t)v * K + k) : 0.0f;
                part = fmaf(pu[j], pv[j], part);
            }
            const float err = (float)__ldg(rating + e) - warp_sum_f(part);
#pragma unroll
            for (int j = 0; j < KP; ++j) ac[j] += err * pv[j];
            if (lane == 0) sq += (double)err * (double)err;
        }
        if (acc) {
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                const int k = lane + 32 * j;
                if (k < K) atomicAdd(&acc[(int64_t)u * K + k], ac[j]);
            }
        }
    }
    if (sq_err && lane == 0 && sq != 0.0) atomicAdd(sq_err, sq);
}

// Rating q (CSC order) of the item pass: the one-byte copy when the ratings fit.
__device__ __forceinline__ float csc_rating(const uint8_t* __restrict__ r8, const uint32_t* __restrict__ r32,
                                            int32_t q) {
    return r8 ? (float)__ldg(r8 + q) : (float)__ldg(r32 + q);
}

template <int KP>
__global__ void __launch_bounds__(kThreads) cf_item_pass(const int4* __restrict__ chunks, int64_t nchunks,
                                                         const int32_t* __restrict__ row,
                                                         const uint8_t* __restrict__ r8,
                                                         const uint32_t* __restrict__ r32,
                                                         const float* __restrict__ p, int K,
                                                         float* __restrict__ acc) {
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    for (int64_t c = gwarp; c < nchunks; c += nwarps) {
        const int4 ch = chunks[c];
        const int32_t v = ch.x;
        float ac[KP], pv[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) {
            const int k = lane + 32 * j;
            pv[j] = k < K ? __ldg(p + (int64_t)v * K + k) : 0.0f;
            ac[j] = 0.0f;
        }
        for (int32_t q = ch.y; q < ch.z; ++q) {
            const int32_t u = __ldg(row + q);
            float pu[KP];
            float part = 0.0f;  // the user pass's dot product, term for term
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                const int k = lane + 32 * j;
                pu[j] = k < K ? __ldg(p + (int64_t)u * K + k) : 0.0f;
                part = fmaf(pu[j], pv[j], part);
            }
            const float err = csc_rating(r8, r32, q) - warp_sum_f(part);
#pragma unroll
            for (int j = 0; j < KP; ++j) ac[j] += err * pu[j];
        }
#pragma unroll
        for (int j = 0; j < KP; ++j) {
            const int k = lane + 32 * j;
            if (k < K) atomicAdd(&acc[(int64_t)v * K + k], ac[j]);
        }
    }
}

// Grouped forms for K = 8 L (L = 1, 2, 4, 8): L lanes share a rating, 8 factor
// components per lane (two 16-byte loads), so a warp keeps 32 / L ratings in
// flight instead of one, and a dot product needs log2(L) shuffles instead of 5.
template <int L>
__device__ __forceinline__ void load8f(const float* __restrict__ p, int64_t off, float (&x)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p + off));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p + off + 4));
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}

// Sum of x over the 32 / L groups of a warp (lanes with the same component slice).
template <int L>
__device__ __forceinline__ void group_reduce8(float (&x)[8]) {
#pragma unroll
    for (int o = L; o < 32; o <<= 1)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] += __shfl_xor_sync(kFull, x[j], o);
}

template <int L>
__global__ void __launch_bounds__(kThreads) cf_user_pass_g(const int4* __restrict__ chunks, int64_t nchunks,
                                                           const int32_t* __restrict__ col,
                                                           const uint32_t* __restrict__ rating,
                                                           const float* __restrict__ p,
                                                           float* __restrict__ acc,
                                                           double* __restrict__ sq_err) {
    constexpr int K = 8 * L, R = 32 / L;
    const int lane = threadIdx.x & 31, grp = lane / L, sub = lane % L;
    const int64_t gwarp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    double sq = 0.0;
    for (int64_t c = gwarp; c < nchunks; c += nwarps) {
        const int4 ch = chunks[c];
        const int32_t u = ch.x;
        float pu[8], ac[8];
        load8f<L>(p, (int64_t)u * K + 8 * sub, pu);
#pragma unroll
        for (int j = 0; j < 8; ++j) ac[j] = 0.0f;
        for (int32_t e0 = ch.y; e0 < ch.z; e0 += R) {
            const int32_t e = e0 + grp;
            const bool ok = e < ch.z;
            const int32_t v = ok ? __ldg(col + e) : u;  // a valid row to read; its terms are dropped
            const float g = ok ? (float)__ldg(rating + e) : 0.0f;
            float pv[8];
            load8f<L>(p, (int64_t)v * K + 8 * sub, pv);
            float part = 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) part = fmaf(pu[j], pv[j], part);
#pragma unroll
            for (int o = L / 2; o >= 1; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
            const float err = ok ? g - part : 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) ac[j] += err * pv[j];
            if (ok && sub == 0) sq += (double)err * (double)err;
        }
        if (acc) {
            group_reduce8<L>(ac);
            if (grp == 0)
#pragma unroll
                for (int j = 0; j < 8; ++j) atomicAdd(&acc[(int64_t)u * K + 8 * sub + j], ac[j]);
        }
    }
    if (sq_err) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
        if (lane == 0 && sq != 0.0) atomicAdd(sq_err, sq);
    }
}

template <int L>
__global__ void __launch_bounds__(kThreads) cf_item_pass_g(const int4* __restrict__ chunks, int64_t nchunks,
                                                           const int32_t* __restrict__ row,
                                                           const uint8_t* __restrict__ r8,
                                                           const uint32_t* __restrict__ r32,
                                                           const float* __restrict__ p, float* __restrict__ acc) {
    constexpr int K = 8 * L, R = 32 / L;
    const int lane = threadIdx.x & 31, grp = lane / L, sub = lane % L;
    const int64_t gwarp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    for (int64_t c = gwarp; c < nchunks; c += nwarps) {
        const int4 ch = chunks[c];
        const int32_t v = ch.x;
        float ac[8], pv[8];
        load8f<L>(p, (int64_t)v * K + 8 * sub, pv);
#pragma unroll
        for (int j = 0; j < 8; ++j) ac[j] = 0.0f;
        for (int32_t q0 = ch.y; q0 < ch.z; q0 += R) {
            const int32_t q = q0 + grp;
            const bool ok = q < ch.z;
            const int32_t u = ok ? __ldg(row + q) : 0;
            const float g = ok ? csc_rating(r8, r32, q) : 0.0f;
            float pu[8];
            load8f<L>(p, (int64_t)u * K + 8 * sub, pu);
            // e_uv as the user pass computes it: the same products, summed in the
            // same order over the same lanes
            float part = 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) part = fmaf(pu[j], pv[j], part);
#pragma unroll
            for (int o = L / 2; o >= 1; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
            const float err = ok ? g - part : 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) ac[j] += err * pu[j];
        }
        group_reduce8<L>(ac);
        if (grp == 0)
#pragma unroll
            for (int j = 0; j < 8; ++j) atomicAdd(&acc[(int64_t)v * K + 8 * sub + j], ac[j]);
    }
}

// cf_user_pass_g with the factor rows of the hottest items in shared memory:
// code[e] >= 0 is rating e's item row in s_hot, else the item is -1 - code[e].
// The same values in the same order as cf_user_pass_g, so the same results.
template <int L>
__global__ void __launch_bounds__(1024, 1) cf_user_pass_hot(const int4* __restrict__ chunks, int64_t nchunks,
                                                            const int32_t* __restrict__ code,
                                                            const uint32_t* __restrict__ rating,
                                                            const float* __restrict__ p,
                                                            const int32_t* __restrict__ hot_ids, int32_t n_hot,
                                                            float* __restrict__ acc) {
    constexpr int K = 8 * L, R = 32 / L, K4 = K / 4;
    extern __shared__ float4 s_hot[];  // n_hot rows of K floats
    for (int32_t i = threadIdx.x; i < n_hot * K4; i += blockDim.x) {
        const int32_t r = i / K4;
        s_hot[i] = __ldg(reinterpret_cast<const float4*>(p) + (int64_t)hot_ids[r] * K4 + (i - r * K4));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, grp = lane / L, sub = lane % L;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = gwarp; c < nchunks; c += nwarps) {
        const int4 ch = chunks[c];
        const int32_t u = ch.x;
        float pu[8], ac[8];
        load8f<L>(p, (int64_t)u * K + 8 * sub, pu);
#pragma unroll
        for (int j = 0; j < 8; ++j) ac[j] = 0.0f;
        for (int32_t e0 = ch.y; e0 < ch.z; e0 += R) {
            const int32_t e = e0 + grp;
            const bool ok = e < ch.z;
            const int32_t cd = ok ? __ldg(code + e) : -1 - u;  // a valid row to read; its terms are dropped
            const float g = ok ? (float)__ldg(rating + e) : 0.0f;
            float pv[8];
            if (cd >= 0) {
                const float4 a = s_hot[cd * K4 + 2 * sub], b = s_hot[cd * K4 + 2 * sub + 1];
                pv[0] = a.x; pv[1] = a.y; pv[2] = a.z; pv[3] = a.w;
                pv[4] = b.x; pv[5] = b.y; pv[6] = b.z; pv[7] = b.w;
            } else {
                load8f<L>(p, (int64_t)(-1 - cd) * K + 8 * sub, pv);
            }
            float part = 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) part = fmaf(pu[j], pv[j], part);
#pragma unroll
            for (int o = L / 2; o >= 1; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
            const float err = ok ? g - part : 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) ac[j] += err * pv[j];
        }
        group_reduce8<L>(ac);
        if (grp == 0)
#pragma unroll
            for (int j = 0; j < 8; ++j) atomicAdd(&acc[(int64_t)u * K + 8 * sub + j], ac[j]);
    }
}

// code[e] = slot of rating e's item among the staged rows, or -1 - the item.
__global__ void cf_codes(const int32_t* __restrict__ col, int64_t m, const int32_t* __restrict__ slot_of,
                         int32_t* __restrict__ code) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = col[e];
        const int32_t s = slot_of[v];
        code[e] = s >= 0 ? s : -1 - v;
    }
}

constexpr int kHotSmem = 224 * 1024;  // shared memory for staged item rows per CTA

// p <- p + gamma (acc - lambda p); acc <- 0
__global__ void cf_update(float* __restrict__ p, float* __restrict__ acc, int64_t count, float gamma, float lambda) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = p[i];
        p[i] = x + gamma * (acc[i] - lambda * x);
        acc[i] = 0.0f;
    }
}

__global__ void sum_squares(const float* __restrict__ p, int64_t count, double* __restrict__ out) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)p[i] * (double)p[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}

// Work items (row, first edge, end edge, 0) of at most kCfChunk edges per row.
std::vector<int4> make_chunks(const std::vector<int32_t>& ptr, int64_t r0, int64_t r1) {
    std::vector<int4> out;
    for (int64_t r = r0; r < r1; ++r)
        for (int32_t e = ptr[r]; e < ptr[r + 1]; e += kCfChunk)
            out.push_back(make_int4((int32_t)r, e, std::min(ptr[r + 1], e + kCfChunk), 0));
    return out;
}

struct CfState {
    DevBuf user_chunks, item_chunks, acc, scalar;
    DevBuf hot_ids, code;     // staged item rows (grouped K): their vertex ids; per-rating codes
    int32_t n_hot = 0;
    int64_t n_user_chunks = 0, n_item_chunks = 0;
    void* sgd = nullptr;      // stochastic gradient descent (gm_cf_sgd.cu)
};

int grid_cf() { return num_sms() * 8; }

template <typename F>
gm_status by_kp(int K, F f) {
    if (K <= 32) return f(std::integral_constant<int, 1>());
    return f(std::integral_constant<int, 2>());
}

// K = 8, 16, 32, 64 take the grouped kernels (L = K / 8 lanes per rating).
bool grouped(int K) { return K == 8 || K == 16 || K == 32 || K == 64; }

template <typename F>
gm_status by_group(int K, F f) {
    switch (K) {
        case 8: return f(std::integral_constant<int, 1>());
        case 16: return f(std::integral_constant<int, 2>());
        case 32: return f(std::integral_constant<int, 4>());
        default: return f(std::integral_constant<int, 8>());
    }
}

}  // namespace

// Stochastic gradient descent (gm_cf_sgd.cu): rating records in the stratified
// order, and the epochs.
gm_status sgd_prepare(gm_graph* g, void** state);
gm_status sgd_run(gm_graph* g, void* state, int32_t epochs);
void sgd_release(void* state, cudaStream_t s);

void cf_release(gm_graph* g) {
    CfState* c = static_cast<CfState*>(g->cf);
    if (!c) return;
    sgd_release(c->sgd, g->stream);
    c->sgd = nullptr;
    DevBuf* bufs[] = {&c->user_chunks, &c->item_chunks, &c->acc, &c->scalar, &c->hot_ids, &c->code};
    for (DevBuf* b : bufs) dev_free(*b, g->stream);
    delete c;
    g->cf = nullptr;
}

gm_status cf_prepare(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int K = g->params.K;
    const int64_t n = g->n;
    cf_release(g);
    CfState* c = new (std::nothrow) CfState();
    if (!c) { set_error("cf: host allocation failed"); return GM_ERR_OUT_OF_MEMORY; }
    g->cf = c;
    std::vector<int32_t> rp((size_t)n + 1), cp((size_t)n + 1);
    GM_CUDA_TRY(cudaMemcpyAsync(rp.data(), g->row_ptr.p, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaMemcpyAsync(cp.data(), g->col_ptr.p, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    const std::vector<int4> uc = make_chunks(rp, 0, g->n_left);
    const std::vector<int4> ic = make_chunks(cp, g->n_left, n);
    c->n_user_chunks = (int64_t)uc.size();
    c->n_item_chunks = (int64_t)ic.size();
    GM_TRY(dev_alloc(c->user_chunks, sizeof(int4) * (uc.size() + 1), s));
    GM_TRY(dev_alloc(c->item_chunks, sizeof(int4) * (ic.size() + 1), s));
    if (!uc.empty())
        GM_CUDA_TRY(cudaMemcpyAsync(c->user_chunks.p, uc.data(), sizeof(int4) * uc.size(), cudaMemcpyHostToDevice, s));
    if (!ic.empty())
        GM_CUDA_TRY(cudaMemcpyAsync(c->item_chunks.p, ic.data(), sizeof(int4) * ic.size(), cudaMemcpyHostToDevice, s));
    const bool sgd = g->kind == GM_CF_SGD;
    // the most-rated items' rows are staged in shared memory by the user pass
    if (!sgd && grouped(K) && g->m > 0 && n > g->n_left) {
        const int64_t n_items = n - g->n_left;
        const int32_t cap = (int32_t)std::min<int64_t>(n_items, kHotSmem / (int64_t)(sizeof(float) * K));
        std::vector<int32_t> items((size_t)n_items);
        for (int64_t i = 0; i < n_items; ++i) items[(size_t)i] = (int32_t)(g->n_left + i);
        std::stable_sort(items.begin(), items.end(), [&](int32_t a, int32_t b) {
            return cp[(size_t)a + 1] - cp[(size_t)a] > cp[(size_t)b + 1] - cp[(size_t)b];
        });
        items.resize((size_t)cap);
        std::vector<int32_t> slot_of((size_t)n, -1);
        for (int32_t i = 0; i < cap; ++i) slot_of[(size_t)items[(size_t)i]] = i;
        DevBuf dslot;
        GM_TRY(dev_alloc(c->hot_ids, sizeof(int32_t) * (size_t)std::max<int32_t>(cap, 1), s));
        GM_TRY(dev_alloc(c->code, sizeof(int32_t) * (size_t)g->m, s));
        GM_TRY(dev_alloc(dslot, sizeof(int32_t) * (size_t)n, s));
        GM_CUDA_TRY(cudaMemcpyAsync(c->hot_ids.p, items.data(), sizeof(int32_t) * (size_t)cap, cudaMemcpyHostToDevice, s));
        GM_CUDA_TRY(cudaMemcpyAsync(dslot.p, slot_of.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
        cf_codes<<<num_sms() * 8, 256, 0, s>>>(as<int32_t>(g->col), g->m, as<int32_t>(dslot), as<int32_t>(c->code));
        g_launches++;
        GM_CUDA_TRY(cudaGetLastError());
        GM_CUDA_TRY(cudaStreamSynchronize(s));  // the host copies above come from stack vectors
        dev_free(dslot, s);
        c->n_hot = cap;
    }
    if (sgd) {
        GM_TRY(sgd_prepare(g, &c->sgd));
    } else {
        GM_TRY(dev_alloc(c->acc, sizeof(float) * (n > 0 ? n : 1) * K, s));
        GM_CUDA_TRY(cudaMemsetAsync(c->acc.p, 0, sizeof(float) * (n > 0 ? n : 1) * K, s));
    }
    GM_TRY(dev_alloc(c->scalar, sizeof(double) * 2, s));
    GM_TRY(dev_alloc(g->state, sizeof(float) * (n > 0 ? n : 1) * K, s));
    if (n > 0) {
        cf_init<<<num_sms() * 4, 256, 0, s>>>(as<float>(g->state), n * K, g->params.seed, g->params.init_sigma);
        g_launches++;
        GM_CUDA_TRY(cudaGetLastError());
    }
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    return GM_OK;
}

gm_status cf_run(gm_graph* g, int32_t iters, int32_t* iters_done) {
    if (iters < 0) {
        set_error("gm_run: CF runs a fixed number of supersteps; max_iters must be >= 0");
        return GM_ERR_INVALID_ARG;
    }
    CfState* c = static_cast<CfState*>(g->cf);
    cudaStream_t s = g->stream;
    const int K = g->params.K;
    const int64_t nk = g->n * K;
    float* p = as<float>(g->state);
    if (g->kind == GM_CF_SGD) {
        GM_TRY(sgd_run(g, c->sgd, iters));
        g->stats = RunStats{};
        g->stats.supersteps = iters;
        if (iters_done) *iters_done = iters;
        return GM_OK;
    }
    for (int32_t it = 0; it < iters; ++it) {
        if (grouped(K)) {
            GM_TRY(by_group(K, [&](auto lc) -> gm_status {
                constexpr int L = decltype(lc)::value;
                if (c->n_user_chunks > 0 && c->n_hot > 0) {
                    const size_t smem = sizeof(float) * 8 * L * (size_t)c->n_hot;
                    static const bool attr = [] {
                        cudaFuncSetAttribute(cf_user_pass_hot<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kHotSmem);
                        return true;
                    }();
                    (void)attr;
                    cf_user_pass_hot<L><<<num_sms(), 1024, smem, s>>>(
                        as<int4>(c->user_chunks), c->n_user_chunks, as<int32_t>(c->code), as<uint32_t>(g->w), p,
                        as<int32_t>(c->hot_ids), c->n_hot, as<float>(c->acc));
                    g_launches++;
                } else if (c->n_user_chunks > 0) {
                    cf_user_pass_g<L><<<grid_cf(), kThreads, 0, s>>>(as<int4>(c->user_chunks), c->n_user_chunks,
                                                                      as<int32_t>(g->col), as<uint32_t>(g->w), p,
                                                                      as<float>(c->acc), nullptr);
                    g_launches++;
                }
                if (c->n_item_chunks > 0) {
                    cf_item_pass_g<L><<<grid_cf(), kThreads, 0, s>>>(as<int4>(c->item_chunks), c->n_item_chunks,
                                                                      as<int32_t>(g->row), as<uint8_t>(g->cw8),
                                                                      as<uint32_t>(g->cw), p, as<float>(c->acc));
                    g_launches++;
                }
                GM_CUDA_TRY(cudaGetLastError());
                return GM_OK;
            }));
        } else GM_TRY(by_kp(K, [&](auto kp) -> gm_status {
            constexpr int KP = decltype(kp)::value;
            if (c->n_user_chunks > 0) {
                cf_user_pass<KP><<<grid_cf(), kThreads, 0, s>>>(as<int4>(c->user_chunks), c->n_user_chunks,
                                                                 as<int32_t>(g->col), as<uint32_t>(g->w), p, K,
                                                                 as<float>(c->acc), nullptr);
                g_launches++;
            }
            if (c->n_item_chunks > 0) {
                cf_item_pass<KP><<<grid_cf(), kThreads, 0, s>>>(as<int4>(c->item_chunks), c->n_item_chunks,
                                                                 as<int32_t>(g->row), as<uint8_t>(g->cw8),
                                                                 as<uint32_t>(g->cw), p, K, as<float>(c->acc));
                g_launches++;
            }
            GM_CUDA_TRY(cudaGetLastError());
            return GM_OK;
        }));
        if (nk > 0) {
            cf_update<<<num_sms() * 8, 256, 0, s>>>(p, as<float>(c->acc), nk, (float)g->params.gamma,
                                                    (float)g->params.lambda);
            g_launches++;
            GM_CUDA_TRY(cudaGetLastError());
        }
    }
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    g->stats = RunStats{};
    g->stats.supersteps = iters;
    if (iters_done) *iters_done = iters;
    return GM_OK;
}

// Eq. 2 with the regulariser once per vertex, at the current factors, in FP64 sums.
gm_status cf_loss(gm_graph* g, double* out) {
    CfState* c = static_cast<CfState*>(g->cf);
    cudaStream_t s = g->stream;
    const int K = g->params.K;
    double* d = as<double>(c->scalar);
    GM_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(double) * 2, s));
    if (grouped(K)) {
        GM_TRY(by_group(K, [&](auto lc) -> gm_status {
            constexpr int L = decltype(lc)::value;
            if (c->n_user_chunks > 0) {
                cf_user_pass_g<L><<<grid_cf(), kThreads, 0, s>>>(as<int4>(c->user_chunks), c->n_user_chunks,
                                                                  as<int32_t>(g->col), as<uint32_t>(g->w),
                                                                  as<float>(g->state), nullptr, d);
                g_launches++;
            }
            return GM_OK;
        }));
    } else GM_TRY(by_kp(K, [&](auto kp) -> gm_status {
        constexpr int KP = decltype(kp)::value;
        if (c->n_user_chunks > 0) {
            cf_user_pass<KP><<<grid_cf(), kThreads, 0, s>>>(as<int4>(c->user_chunks), c->n_user_chunks,
                                                             as<int32_t>(g->col), as<uint32_t>(g->w),
                                                             as<float>(g->state), K, nullptr, d);
            g_launches++;
        }
        return GM_OK;
    }));
    if (g->n > 0) {
        sum_squares<<<num_sms() * 4, 256, 0, s>>>(as<float>(g->state), g->n * K, d + 1);
        g_launches++;
    }
    double h[2] = {0.0, 0.0};
    GM_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    *out = h[0] + g->params.lambda * h[1];
    return GM_OK;
}

}  // namespace gm
