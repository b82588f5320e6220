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
// for t = T-1 .. 0 in one fused pass per superstep (the gradient term reuses the
// lambda gather of the reverse SpMV), recomputing each checkpoint segment's states
// forward first -- except the last segment, whose states the forward leaves in
// place; then the row-normalisation chain rule
// dL/dw_uv = (gbar_uv - sum_v' P_uv' gbar_uv') / S_u.
// Every pass is a row reduction over rows binned by length (a lane per short row,
// the short bin ordered by length; a warp per medium row; a CTA per long row),
// four entries in flight per thread, in FP32, in a fixed order.
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
// Run by `nblk` CTAs numbered `blk`; CTA-collective.
template <class F>
__device__ __forceinline__ void row_pass_body(const RowSet& rs, const F& f, int64_t blk, int64_t nblk) {
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t gwarp = (blk * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = (nblk * kThreads) >> 5;
    __shared__ float s_red[kWarps];
    // long rows: one CTA each
    for (int64_t i = rs.off[2] + blk; i < rs.off[3]; i += nblk) {
        const int32_t r = rs.list[i];
        const int32_t beg = rs.ptr[r], end = rs.ptr[r + 1];
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;  // four entries in flight per thread
        int32_t e = beg + threadIdx.x;
        for (; e + 3 * kThreads < end; e += 4 * kThreads) {
            s0 += f.edge(r, e);
            s1 += f.edge(r, e + kThreads);
            s2 += f.edge(r, e + 2 * kThreads);
            s3 += f.edge(r, e + 3 * kThreads);
        }
        for (; e < end; e += kThreads) s0 += f.edge(r, e);
        float s = warp_sum_f((s0 + s1) + (s2 + s3));
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
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;  // four entries in flight per lane
        int32_t e = beg + lane;
        for (; e + 96 < end; e += 128) {
            s0 += f.edge(r, e);
            s1 += f.edge(r, e + 32);
            s2 += f.edge(r, e + 64);
            s3 += f.edge(r, e + 96);
        }
        for (; e < end; e += 32) s0 += f.edge(r, e);
        const float s = warp_sum_f((s0 + s1) + (s2 + s3));
        if (lane == 0) f.finish(r, s);
    }
    // short rows: one lane each; the bin is ordered by length, so a warp's 32 rows
    // take about the same number of steps; four entries in flight per lane
    for (int64_t i = rs.off[0] + gwarp * 32 + lane; i - lane < rs.off[1]; i += nwarps * 32) {
        if (i >= rs.off[1]) continue;
        const int32_t r = rs.list[i];
        const int32_t beg = rs.ptr[r], end = rs.ptr[r + 1];
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        int32_t e = beg;
        for (; e + 3 < end; e += 4) {
            s0 += f.edge(r, e);
            s1 += f.edge(r, e + 1);
            s2 += f.edge(r, e + 2);
            s3 += f.edge(r, e + 3);
        }
        for (; e < end; ++e) s0 += f.edge(r, e);
        f.finish(r, (s0 + s1) + (s2 + s3));
    }
    // rows without entries
    for (int64_t i = blk * kThreads + threadIdx.x; i < rs.nzero; i += nblk * kThreads) f.finish(rs.zero[i], 0.0f);
}

template <class F>
__global__ void __launch_bounds__(kThreads) row_pass(RowSet rs, F f) {
    row_pass_body(rs, f, blockIdx.x, gridDim.x);
}

// Two independent passes in one launch (CTAs [0, nblk1) run the first): an adjoint
// superstep and a recompute superstep of the next segment share the GPU, so each
// hides the other's memory latency.
template <class F1, class F2>
__global__ void __launch_bounds__(kThreads) row_pass2(RowSet rs1, F1 f1, int nblk1, RowSet rs2, F2 f2) {
    if ((int)blockIdx.x < nblk1) row_pass_body(rs1, f1, blockIdx.x, nblk1);
    else row_pass_body(rs2, f2, blockIdx.x - nblk1, gridDim.x - nblk1);
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
// One adjoint superstep over the CSR rows u (reverse SpMV fused with the edge
// gradient in SDDMM form), for t = T-1 .. 0:
//   gbar_e += (1-r) x^t_u lambda^{t+1}_v,   lambda^t_u = (1-r) sum_e P_e lambda^{t+1}_v.
// Each edge's gradient terms are added one superstep at a time from the last to
// the first, so the rounding does not depend on the checkpoint interval.  All
// reads are non-coherent loads: gbar_e is read and then written by one thread
// only, so the compiler may issue the loads of several edges before their stores.
struct BackwardF {
    const int32_t* col; const float* P; const float* x; const float* lam; float* lamn; float* gbar; float r;
    __device__ float edge(int32_t u, int32_t e) const {
        const float lv = __ldg(lam + __ldg(col + e));
        const float g0 = __ldg(gbar + e);
        gbar[e] = g0 + (1.0f - r) * __ldg(x + u) * lv;
        return __ldg(P + e) * lv;
    }
    __device__ void finish(int32_t u, float s) const { lamn[u] = (1.0f - r) * s; }
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

template <class F1, class F2>
gm_status launch_pass2(const RowSet& rs1, const F1& f1, const RowSet& rs2, const F2& f2, cudaStream_t s) {
    const int b1 = pass_grid<F1>(), b2 = pass_grid<F2>();
    row_pass2<F1, F2><<<b1 + b2, kThreads, 0, s>>>(rs1, f1, b1, rs2, f2);
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
    DevBuf S, P, Pc, gbar, ckpt, seg, seg2, lam, d;  // seg2: the next segment, recomputed alongside
    int32_t steps = -1, every = 0;
    int32_t seg_c = -1;  // >= 0: seg holds x^seg_c .. x^steps from the last forward (its last segment)
    float r = 0.15f;
    bool have_forward = false;
};

void wpr_release(gm_graph* g) {
    WprState* w = static_cast<WprState*>(g->wpr);
    if (!w) return;
    DevBuf* bufs[] = {&w->S, &w->P, &w->Pc, &w->gbar, &w->ckpt, &w->seg, &w->seg2, &w->lam, &w->d};
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
        GM_TRY(dev_alloc(w->seg2, sizeof(float) * n * (ckpt_every + 1), s));
    }
    w->steps = steps;
    w->every = ckpt_every;
    w->seg_c = -1;
    w->have_forward = false;
    w->r = (float)r;
    const RowSet rows = csr_rows(g);
    GM_TRY(launch_pass(rows, RowSumF{w_dev, as<float>(w->S)}, s));
    GM_TRY(launch_pass(rows, NormalizeF{w_dev, as<float>(w->S), as<float>(w->P)}, s));
    if (g->m > 0) {
        gather_f32<<<num_sms() * 4, 256, 0, s>>>(as<float>(w->P), as<uint32_t>(g->csc_pos), g->m, as<float>(w->Pc));
        g_launches++;
    }
    // x^0 = 1 is checkpoint 0.  Up to the last segment two ping-pong vectors live in
    // seg; the last segment's states x^c_last .. x^steps are kept in seg's slots
    // 0 .. steps - c_last, so the adjoint starts without recomputing them.
    float* ck = as<float>(w->ckpt);
    fill_f32_k<<<num_sms() * 4, 256, 0, s>>>(ck, g->n, 1.0f);
    g_launches++;
    float* seg = as<float>(w->seg);
    const int32_t c_last = steps > 0 ? ((steps - 1) / ckpt_every) * ckpt_every : 0;
    float* a = seg;
    float* b = a + n;
    GM_CUDA_TRY(cudaMemcpyAsync(a, ck, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
    for (int32_t t = 0; t < steps; ++t) {
        if (t == c_last && a != seg) {  // x^c_last into slot 0
            GM_CUDA_TRY(cudaMemcpyAsync(seg, a, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
            a = seg;
        }
        if (t >= c_last) b = seg + n * (t + 1 - c_last);
        GM_TRY(wpr_step(g, w, a, b));
        std::swap(a, b);
        if ((t + 1) % ckpt_every == 0 && (t + 1) / ckpt_every < nck)
            GM_CUDA_TRY(cudaMemcpyAsync(ck + n * ((t + 1) / ckpt_every), a, sizeof(float) * g->n,
                                        cudaMemcpyDeviceToDevice, s));
    }
    w->seg_c = c_last;
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
    float* lam = as<float>(w->lam);  // lambda^{t+1} and lambda^t, ping-pong
    float* lamn = lam + n;
    GM_CUDA_TRY(cudaMemcpyAsync(lam, dLdx_dev, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
    if (g->m > 0) GM_CUDA_TRY(cudaMemsetAsync(w->gbar.p, 0, sizeof(float) * g->m, s));
    // Segments from the last to the first.  `cur` holds the states of the segment
    // being differentiated; the next (earlier) segment's states are recomputed into
    // `nxt` by forward steps launched together with the adjoint steps.
    float* cur = as<float>(w->seg);
    float* nxt = as<float>(w->seg2);
    const float* ck = as<float>(w->ckpt);
    const RowSet ccols = csc_rows(g);
    const int32_t c_top = T > 0 ? ((T - 1) / k) * k : -1;
    if (T > 0 && c_top != w->seg_c) {  // the last segment is not in place: recompute it first
        GM_CUDA_TRY(cudaMemcpyAsync(cur, ck + n * (c_top / k), sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
        for (int32_t t = c_top; t + 1 < T; ++t) GM_TRY(wpr_step(g, w, cur + n * (t - c_top), cur + n * (t + 1 - c_top)));
    }
    w->seg_c = -1;  // the segment buffers are overwritten from here on
    for (int32_t c = c_top; c >= 0; c -= k) {
        const int32_t e = std::min(c + k, T);  // cur holds x^c .. x^{e-1}
        const int32_t cp = c - k;               // the next segment: x^cp .. x^{c-1} (k states)
        if (cp >= 0)
            GM_CUDA_TRY(cudaMemcpyAsync(nxt, ck + n * (cp / k), sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
        int32_t done = 0;  // recompute steps of the next segment issued
        for (int32_t t = e - 1; t >= c; --t) {
            const BackwardF bf{as<int32_t>(g->col), as<float>(w->P), cur + n * (t - c), lam, lamn,
                               as<float>(w->gbar), w->r};
            if (cp >= 0 && done + 1 < k) {
                const ForwardF ff{as<int32_t>(g->row), as<float>(w->Pc), nxt + n * done, nxt + n * (done + 1), w->r};
                GM_TRY(launch_pass2(rows, bf, ccols, ff, s));
                ++done;
            } else {
                GM_TRY(launch_pass(rows, bf, s));
            }
            std::swap(lam, lamn);
        }
        for (; cp >= 0 && done + 1 < k; ++done) GM_TRY(wpr_step(g, w, nxt + n * done, nxt + n * (done + 1)));
        std::swap(cur, nxt);
    }
    GM_TRY(launch_pass(rows, RowDotF{as<float>(w->P), as<float>(w->gbar), as<float>(w->d)}, s));
    GM_TRY(launch_pass(rows, GradF{as<float>(w->gbar), as<float>(w->d), as<float>(w->S), dLdw_dev}, s));
    GM_CUDA_TRY(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // extern "C"
