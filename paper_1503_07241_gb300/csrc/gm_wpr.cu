// Differentiable weighted PageRank: Eq. 1 with learnable, row-normalised edge
// weights, and its hand-written adjoint.
//
//   S_u = sum_v w_uv,  P_uv = w_uv / S_u,
//   x^0 = 1,  x^{t+1}_v = r + (1 - r) sum_{u -> v} P_uv x^t_u        (t < T)
//
// Forward: a pull SpMV per superstep over the CSC (per-edge weight P in CSC order),
// storing x^t every `ckpt_every` supersteps.  Backward, given lambda^T = dL/dx^T:
//   gbar_uv  += (1 - r) x^t_u lambda^{t+1}_v                (edge gradient, SDDMM form)
//   lambda^t_u = (1 - r) sum_v P_uv lambda^{t+1}_v           (reverse SpMV over the CSR)
// for t = T-1 .. 0, recomputing each checkpoint segment's states forward first.
// Within a segment the lambda steps are pure reverse SpMVs that keep the segment's
// lambdas vertex-major, and one edge pass per segment adds up its gbar terms, so
// the per-edge accumulator is read and written once per segment, not per step;
// then the row-normalisation chain rule dL/dw_uv = (gbar_uv - sum_v' P_uv' gbar_uv') / S_u.
// Every pass is a row reduction over rows binned by length (32 short rows per
// warp, a warp per medium row, a CTA per long row), in FP32, in a fixed order.
#include <algorithm>
#include <new>

#include "gm_internal.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kFull = 0xffffffffu;

// Rows of a compressed matrix with their lists binned by length.
struct RowSet {
    const int32_t* ptr;     // row r's entries are [ptr[r], ptr[r+1])
    const int32_t* list;    // rows with >= 1 entry, bins 1..3 at [off[b-1], off[b])
    int64_t off[4];
    const int32_t* zero;    // rows without entries
    int64_t nzero;
};

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// For every row r: s = sum over its entries e of f.edge(r, e); then f.finish(r, s).
template <class F>
__global__ void __launch_bounds__(kThreads) row_pass(RowSet rs, F f) {
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t gwarp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    __shared__ float s_red[kWarps];
    __shared__ float s_acc[kWarps][32];
    // long rows: one CTA each
    for (int64_t i = rs.off[2] + blockIdx.x; i < rs.off[3]; i += gridDim.x) {
        const int32_t r = rs.list[i];
        const int32_t beg = rs.ptr[r], end = rs.ptr[r + 1];
        float s = 0.0f;
        for (int32_t e = beg + threadIdx.x; e < end; e += kThreads) s += f.edge(r, e);
        s = warp_sum_f(s);
        if (lane == 0) s_red[wid] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tot = 0.0f;
            for (int w2 = 0; w2 < kWarps; ++w2) tot += s_red[w2];
            f.finish(r, tot);
        }
        __syncthreads();
    }
    // medium rows: one warp each
    for (int64_t i = rs.off[1] + gwarp; i < rs.off[2]; i += nwarps) {
        const int32_t r = rs.list[i];
        const int32_t beg = rs.ptr[r], end = rs.ptr[r + 1];
        float s = 0.0f;
        for (int32_t e = beg + lane; e < end; e += 32) s += f.edge(r, e);
        s = warp_sum_f(s);
        if (lane == 0) f.finish(r, s);
    }
    // short rows: 32 per warp, entries concatenated, segmented sums in a fixed order
    float* acc = s_acc[wid];
    for (int64_t g0 = rs.off[0] + gwarp * 32; g0 < rs.off[1]; g0 += nwarps * 32) {
        const int64_t i = g0 + lane;
        int32_t r = 0, beg = 0;
        uint32_t len = 0u;
        if (i < rs.off[1]) {
            r = rs.list[i];
            beg = rs.ptr[r];
            len = (uint32_t)(rs.ptr[r + 1] - beg);
        }
        acc[lane] = 0.0f;
        __syncwarp();
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - len;
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
            const int32_t ro = __shfl_sync(kFull, r, k);
            const bool valid = j < total;
            float val = valid ? f.edge(ro, bo + (int32_t)(j - eo)) : 0.0f;
            const int owner = valid ? k : 32 + lane;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {  // inclusive segmented scan by owner
                const float y = __shfl_up_sync(kFull, val, o);
                const int ko = __shfl_up_sync(kFull, owner, o);
                if (lane >= o && ko == owner) val += y;
            }
            const int next_owner = __shfl_down_sync(kFull, owner, 1);
            if (valid && (lane == 31 || next_owner != owner)) acc[k] += val;
            __syncwarp();
        }
        if (i < rs.off[1]) f.finish(r, acc[lane]);
        __syncwarp();
    }
    // rows without entries
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < rs.nzero; i += (int64_t)gridDim.x * kThreads)
        f.finish(rs.zero[i], 0.0f);
}

// ---- the passes -------------------------------------------------------------------
struct RowSumF {  // S_u = sum_e w_e
    const float* w; float* S;
    __device__ float edge(int32_t, int32_t e) const { return w[e]; }
    __device__ void finish(int32_t u, float s) const { S[u] = s; }
};
struct NormalizeF {  // P_e = w_e / S_u (CSR order)
    const float* w; const float* S; float* P;
    __device__ float edge(int32_t u, int32_t e) const { P[e] = w[e] / S[u]; return 0.0f; }
    __device__ void finish(int32_t, float) const {}
};
struct ForwardF {  // x'_v = r + (1-r) sum_{u->v} Pc_q x_u (CSC order)
    const int32_t* row; const float* Pc; const float* x; float* xn; float r;
    __device__ float edge(int32_t, int32_t q) const { return Pc[q] * x[row[q]]; }
    __device__ void finish(int32_t v, float s) const { xn[v] = r + (1.0f - r) * s; }
};
// lambda^t_u = (1-r) sum_e P_e lambda^{t+1}_v (reverse SpMV over the CSR).  The
// lambdas of one checkpoint segment are kept vertex-major: lamT[v * kk + j].
struct LamF {
    const int32_t* col; const float* P; const float* lam; int kk, j_in; float* lamn; int kn, j_out; float r;
    __device__ float edge(int32_t, int32_t e) const { return P[e] * lam[(int64_t)col[e] * kk + j_in]; }
    __device__ void finish(int32_t u, float s) const { lamn[(int64_t)u * kn + j_out] = (1.0f - r) * s; }
};
// Edge gradient of one segment, supersteps t = c .. c+len-1 (SDDMM form):
// gbar_e += (1-r) x^t_u lambda^{t+1}_v with x^t in xs[(t-c) * n + u] and
// lambda^{t+1} in lamT[v * kk + (t - c)], added one superstep at a time from the
// last to the first, so the rounding is the same for every checkpoint interval.
struct GbarF {
    const int32_t* col; const float* xs; int64_t n; const float* lamT; int kk, len; float* gbar; float r;
    __device__ float edge(int32_t u, int32_t e) const {
        const float* lv = lamT + (int64_t)col[e] * kk;
        float acc = gbar[e];
        for (int j = len - 1; j >= 0; --j) acc += (1.0f - r) * xs[(int64_t)j * n + u] * lv[j];
        gbar[e] = acc;
        return 0.0f;
    }
    __device__ void finish(int32_t, float) const {}
};
struct RowDotF {  // d_u = sum_e P_e gbar_e
    const float* P; const float* gbar; float* d;
    __device__ float edge(int32_t, int32_t e) const { return P[e] * gbar[e]; }
    __device__ void finish(int32_t u, float s) const { d[u] = s; }
};
struct GradF {  // dL/dw_e = (gbar_e - d_u) / S_u
    const float* gbar; const float* d; const float* S; float* grad;
    __device__ float edge(int32_t u, int32_t e) const { grad[e] = (gbar[e] - d[u]) / S[u]; return 0.0f; }
    __device__ void finish(int32_t, float) const {}
};

__global__ void gather_f32(const float* __restrict__ in, const uint32_t* __restrict__ idx, int64_t len,
                           float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[idx[i]];
}

// out[v * stride + j] = in[v]
__global__ void scatter_strided_f32(const float* __restrict__ in, int64_t n, float* __restrict__ out,
                                    int stride, int j) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i * stride + j] = in[i];
}

__global__ void fill_f32_k(float* p, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

template <class F>
int pass_grid() {
    static int blocks = 0;
    if (blocks == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, row_pass<F>, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
        blocks = per_sm * num_sms();
    }
    return blocks;
}

template <class F>
gm_status launch_pass(const RowSet& rs, const F& f, cudaStream_t s) {
    row_pass<F><<<pass_grid<F>(), kThreads, 0, s>>>(rs, f);
    g_launches++;
    GM_CUDA_TRY(cudaGetLastError());
    return GM_OK;
}

RowSet csr_rows(const gm_graph* g) {
    RowSet rs{};
    rs.ptr = as<int32_t>(g->row_ptr);
    rs.list = as<int32_t>(g->out_list);
    for (int b = 0; b < 4; ++b) rs.off[b] = g->out_list_count[b];
    rs.zero = as<int32_t>(g->zero_out_list);
    rs.nzero = g->zero_out_count;
    return rs;
}

RowSet csc_rows(const gm_graph* g) {
    RowSet rs{};
    rs.ptr = as<int32_t>(g->col_ptr);
    rs.list = as<int32_t>(g->in_list);
    for (int b = 0; b < 4; ++b) rs.off[b] = g->in_list_count[b];
    rs.zero = as<int32_t>(g->zero_in_list);
    rs.nzero = g->zero_in_count;
    return rs;
}

}  // namespace

// Buffers of the weighted-PageRank forms (owned by the graph handle).
struct WprState {
    DevBuf S, P, Pc, gbar, ckpt, seg, lam, lamT, d;
    int32_t steps = -1, every = 0;
    float r = 0.15f;
    bool have_forward = false;
};

void wpr_release(gm_graph* g) {
    WprState* w = static_cast<WprState*>(g->wpr);
    if (!w) return;
    DevBuf* bufs[] = {&w->S, &w->P, &w->Pc, &w->gbar, &w->ckpt, &w->seg, &w->lam, &w->lamT, &w->d};
    for (DevBuf* b : bufs) dev_free(*b, g->stream);
    delete w;
    g->wpr = nullptr;
}

// x^{t+1} from x^t (both device float[n]).
static gm_status wpr_step(gm_graph* g, WprState* w, const float* x, float* xn) {
    ForwardF f{as<int32_t>(g->row), as<float>(w->Pc), x, xn, w->r};
    return launch_pass(csc_rows(g), f, g->stream);
}

}  // namespace gm

using namespace gm;

extern "C" {

gm_status gm_wpagerank_forward(gm_graph* g, const float* w_dev, double r, int32_t steps, int32_t ckpt_every,
                               float* x_out_dev) {
    if (!g || !w_dev || !x_out_dev) { set_error("gm_wpagerank_forward: NULL argument"); return GM_ERR_INVALID_ARG; }
    if (steps < 0 || ckpt_every < 1 || !(r >= 0.0 && r <= 1.0)) {
        set_error("gm_wpagerank_forward: need steps >= 0, ckpt_every >= 1, r in [0, 1]");
        return GM_ERR_INVALID_ARG;
    }
    cudaStream_t s = g->stream;
    const int64_t n = g->n > 0 ? g->n : 1, m = g->m > 0 ? g->m : 1;
    WprState* w = static_cast<WprState*>(g->wpr);
    if (!w) {
        w = new (std::nothrow) WprState();
        if (!w) { set_error("gm_wpagerank_forward: host allocation failed"); return GM_ERR_OUT_OF_MEMORY; }
        g->wpr = w;
        GM_TRY(dev_alloc(w->S, sizeof(float) * n, s));
        GM_TRY(dev_alloc(w->P, sizeof(float) * m, s));
        GM_TRY(dev_alloc(w->Pc, sizeof(float) * m, s));
        GM_TRY(dev_alloc(w->gbar, sizeof(float) * m, s));
        GM_TRY(dev_alloc(w->lam, sizeof(float) * 2 * n, s));
        GM_TRY(dev_alloc(w->d, sizeof(float) * n, s));
    }
    const int32_t nck = steps / ckpt_every + 1;
    if (w->every != ckpt_every || w->steps != steps) {
        GM_TRY(dev_alloc(w->ckpt, sizeof(float) * n * nck, s));
        GM_TRY(dev_alloc(w->seg, sizeof(float) * n * (ckpt_every + 1), s));
        GM_TRY(dev_alloc(w->lamT, sizeof(float) * n * ckpt_every, s));
    }
    w->steps = steps;
    w->every = ckpt_every;
    w->r = (float)r;
    const RowSet rows = csr_rows(g);
    GM_TRY(launch_pass(rows, RowSumF{w_dev, as<float>(w->S)}, s));
    GM_TRY(launch_pass(rows, NormalizeF{w_dev, as<float>(w->S), as<float>(w->P)}, s));
    if (g->m > 0) {
        gather_f32<<<num_sms() * 4, 256, 0, s>>>(as<float>(w->P), as<uint32_t>(g->csc_pos), g->m, as<float>(w->Pc));
        g_launches++;
    }
    // x^0 = 1 is checkpoint 0; two ping-pong vectors live in seg
    float* ck = as<float>(w->ckpt);
    fill_f32_k<<<num_sms() * 4, 256, 0, s>>>(ck, g->n, 1.0f);
    g_launches++;
    float* a = as<float>(w->seg);
    float* b = a + n;
    GM_CUDA_TRY(cudaMemcpyAsync(a, ck, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
    for (int32_t t = 0; t < steps; ++t) {
        GM_TRY(wpr_step(g, w, a, b));
        std::swap(a, b);
        if ((t + 1) % ckpt_every == 0 && (t + 1) / ckpt_every < nck)
            GM_CUDA_TRY(cudaMemcpyAsync(ck + n * ((t + 1) / ckpt_every), a, sizeof(float) * g->n,
                                        cudaMemcpyDeviceToDevice, s));
    }
    GM_CUDA_TRY(cudaMemcpyAsync(x_out_dev, a, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    w->have_forward = true;
    return GM_OK;
}

gm_status gm_wpagerank_backward(gm_graph* g, const float* dLdx_dev, float* dLdw_dev) {
    if (!g || !dLdx_dev || !dLdw_dev) { set_error("gm_wpagerank_backward: NULL argument"); return GM_ERR_INVALID_ARG; }
    WprState* w = static_cast<WprState*>(g->wpr);
    if (!w || !w->have_forward) { set_error("gm_wpagerank_backward: call gm_wpagerank_forward first"); return GM_ERR_STATE; }
    cudaStream_t s = g->stream;
    const int64_t n = g->n > 0 ? g->n : 1;
    const int32_t T = w->steps, k = w->every;
    const RowSet rows = csr_rows(g);
    // lam: lambda at the current segment's end (dense, stride 1); lamT: the
    // segment's lambda^{c+1} .. lambda^{e}, vertex-major with stride k.
    float* lam = as<float>(w->lam);
    float* lamT = as<float>(w->lamT);
    const int32_t* col = as<int32_t>(g->col);
    const float* P = as<float>(w->P);
    GM_CUDA_TRY(cudaMemcpyAsync(lam, dLdx_dev, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
    if (g->m > 0) GM_CUDA_TRY(cudaMemsetAsync(w->gbar.p, 0, sizeof(float) * g->m, s));
    float* seg = as<float>(w->seg);
    const float* ck = as<float>(w->ckpt);
    for (int32_t c = ((T - 1) / k) * k; T > 0 && c >= 0; c -= k) {
        const int32_t e = std::min(c + k, T);  // segment holds x^c .. x^{e-1}
        const int32_t len = e - c;
        GM_CUDA_TRY(cudaMemcpyAsync(seg, ck + n * (c / k), sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
        for (int32_t t = c; t + 1 < e; ++t) GM_TRY(wpr_step(g, w, seg + n * (t - c), seg + n * (t + 1 - c)));
        // lambda^{e} into slot len-1, then lambda^{t} for t = e-1 .. c+1 into slot t-c-1
        scatter_strided_f32<<<num_sms() * 4, 256, 0, s>>>(lam, g->n, lamT, k, len - 1);
        g_launches++;
        for (int32_t t = e - 1; t > c; --t)
            GM_TRY(launch_pass(rows, LamF{col, P, lamT, k, t - c, lamT, k, t - c - 1, w->r}, s));
        GM_TRY(launch_pass(rows, GbarF{col, seg, n, lamT, k, len, as<float>(w->gbar), w->r}, s));
        // lambda^{c} for the next (earlier) segment
        if (c > 0) GM_TRY(launch_pass(rows, LamF{col, P, lamT, k, 0, lam, 1, 0, w->r}, s));
    }
    GM_TRY(launch_pass(rows, RowDotF{as<float>(w->P), as<float>(w->gbar), as<float>(w->d)}, s));
    GM_TRY(launch_pass(rows, GradF{as<float>(w->gbar), as<float>(w->d), as<float>(w->S), dLdw_dev}, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // extern "C"
