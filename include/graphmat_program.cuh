/*
 * graphmat_program.cuh -- user-defined vertex programs on the GPU.
 *
 * The generalized SpMSpV of Algorithm 1 inside the superstep loop of Algorithm 2
 * (Section 4.1-4.2) for any vertex program written as the four functions of
 * Section 4 / Figure 2 and the appendix API: Send_Message, Process_Message,
 * Reduce and Apply.  A program is a struct compiled ahead of time with nvcc
 * (include this header in a .cu file); it runs on a graph handle of the C ABI
 * through the read-only device view gm_graph_device_view() returns.
 *
 * A program type P provides
 *   using Prop = ...;   vertex property            (trivially copyable)
 *   using Msg  = ...;   message                    (trivially copyable)
 *   using Acc  = ...;   processed / reduced value  (trivially copyable, size a multiple of 4)
 *   static constexpr bool kAllActive;   every vertex is active in every superstep
 *   static constexpr bool kApplyToAll;  Apply also vertices without a message (with identity())
 *   __device__ bool send(int32_t v, const Prop& p, Msg& m) const;             Send_Message; false: nothing
 *   __device__ Acc process(const Msg& m, uint32_t w, const Prop& dst) const;  Process_Message (w = 1 when
 *                                                                             the graph has no weights)
 *   __device__ Acc reduce(const Acc& a, const Acc& b) const;                   Reduce (associative, commutative)
 *   __device__ Acc identity() const;                                           Reduce's identity
 *   __device__ bool apply(const Acc& y, Prop& p) const;                        Apply; true if p changed
 *
 * Semantics (Algorithm 2): in superstep t every active vertex u sends m_u;
 * every vertex v with at least one in-edge from a sender reduces
 * process(m_u, w_uv, p_v) over those edges (p_v as it was at the start of the
 * superstep) and applies the result; the vertices whose property changed are
 * the active set of superstep t+1.  The loop ends after max_iters supersteps or
 * after the first superstep that changes no vertex (that superstep is counted).
 *
 * Execution: a send kernel (one thread per 32 vertices writes that word of the
 * message-present bitvector), then a pull kernel over the in-edges (CSC): a lane
 * per destination of in-degree < bin_small (the bin is ordered by degree), a
 * warp per larger destination with a warp-shuffle Reduce, so no atomics are
 * needed for any Reduce; the owner of a destination applies.  Reductions are in
 * a fixed order for a given graph and bin thresholds.
 *
 * Memory: the caller owns `props` (device, n values) and `active` (device,
 * ceil(n/32) words, bit v = vertex v active; updated in place).  run() allocates
 * its workspace (n messages + two bitvectors) with cudaMallocAsync on `stream`
 * and frees it before returning.  Errors: GM_ERR_INVALID_ARG for a NULL
 * argument, GM_ERR_CUDA for a failed launch or allocation.
 */
#ifndef GRAPHMAT_PROGRAM_CUH
#define GRAPHMAT_PROGRAM_CUH

#include <cuda_runtime.h>
#include <stdint.h>

#include "graphmat_gb300.h"

namespace gm_program {

constexpr int kThreads = 256;
constexpr unsigned kFullMask = 0xffffffffu;

// Warp shuffle (xor) of a value whose size is a multiple of 4 bytes.
template <class T>
__device__ __forceinline__ T shfl_xor_any(const T& v, int mask) {
    static_assert(sizeof(T) % 4 == 0, "Acc must be a multiple of 4 bytes");
    union U {
        T t;
        uint32_t w[sizeof(T) / 4];
        __device__ U() {}
    } a, b;
    a.t = v;
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) b.w[i] = __shfl_xor_sync(kFullMask, a.w[i], mask);
    return b.t;
}

__device__ __forceinline__ bool test_bit(const uint32_t* bv, int32_t v) { return (bv[v >> 5] >> (v & 31)) & 1u; }

// Send_Message of every active vertex; thread i owns vertices [32 i, 32 i + 32).
template <class P>
__global__ void __launch_bounds__(kThreads) send_kernel(P prog, int64_t n, const typename P::Prop* __restrict__ props,
                                                        const uint32_t* __restrict__ active,
                                                        typename P::Msg* __restrict__ msgs,
                                                        uint32_t* __restrict__ has_msg) {
    const int64_t nwords = (n + 31) / 32;
    for (int64_t wd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wd < nwords;
         wd += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t act = P::kAllActive ? 0xffffffffu : active[wd];
        uint32_t out = 0u;
        for (int b = 0; b < 32; ++b) {
            const int64_t v = wd * 32 + b;
            if (v >= n || !((act >> b) & 1u)) continue;
            typename P::Msg m;
            if (prog.send((int32_t)v, props[v], m)) {
                msgs[v] = m;
                out |= 1u << b;
            }
        }
        has_msg[wd] = out;
    }
}

// Reduce over the in-edges of v from senders, then Apply; returns whether v changed.
template <class P>
__device__ __forceinline__ void finish_vertex(const P& prog, int32_t v, bool any, const typename P::Acc& y,
                                              typename P::Prop* props, uint32_t* next_active,
                                              unsigned long long* n_active) {
    if (!any && !P::kApplyToAll) return;
    typename P::Prop p = props[v];
    const bool changed = prog.apply(any ? y : prog.identity(), p);
    props[v] = p;
    if (changed) {
        atomicOr(&next_active[v >> 5], 1u << (v & 31));
        atomicAdd(n_active, 1ull);
    }
}

template <class P>
__global__ void __launch_bounds__(kThreads) pull_kernel(P prog, gm_device_view V,
                                                        const typename P::Msg* __restrict__ msgs,
                                                        const uint32_t* __restrict__ has_msg,
                                                        typename P::Prop* props, uint32_t* next_active,
                                                        unsigned long long* n_active) {
    using Acc = typename P::Acc;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    // destinations of in-degree >= bin_small: one warp each
    for (int64_t i = V.in_off[1] + gwarp; i < V.in_off[3]; i += nwarps) {
        const int32_t v = V.in_list[i];
        const typename P::Prop dst = props[v];
        Acc acc = prog.identity();
        bool any = false;
        for (int32_t e = V.col_ptr[v] + lane; e < V.col_ptr[v + 1]; e += 32) {
            const int32_t u = V.row[e];
            if (test_bit(has_msg, u)) {
                acc = prog.reduce(acc, prog.process(msgs[u], V.cw ? V.cw[e] : 1u, dst));
                any = true;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = prog.reduce(acc, shfl_xor_any(acc, o));
        any = __any_sync(kFullMask, any);
        if (lane == 0) finish_vertex(prog, v, any, acc, props, next_active, n_active);
    }
    // destinations of in-degree < bin_small: one lane each
    for (int64_t i = V.in_off[0] + (int64_t)blockIdx.x * kThreads + threadIdx.x; i < V.in_off[1];
         i += (int64_t)gridDim.x * kThreads) {
        const int32_t v = V.in_list[i];
        const typename P::Prop dst = props[v];
        Acc acc = prog.identity();
        bool any = false;
        for (int32_t e = V.col_ptr[v]; e < V.col_ptr[v + 1]; ++e) {
            const int32_t u = V.row[e];
            if (test_bit(has_msg, u)) {
                acc = prog.reduce(acc, prog.process(msgs[u], V.cw ? V.cw[e] : 1u, dst));
                any = true;
            }
        }
        finish_vertex(prog, v, any, acc, props, next_active, n_active);
    }
    // destinations without in-edges receive no message
    if (P::kApplyToAll)
        for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < V.zero_in_count;
             i += (int64_t)gridDim.x * kThreads)
            finish_vertex(prog, V.zero_in[i], false, prog.identity(), props, next_active, n_active);
}

// Runs the program from the active set in `active` (updated to the final active
// set).  *iters_done receives the number of supersteps run.
template <class P>
gm_status run(const gm_device_view& V, const P& prog, typename P::Prop* props, uint32_t* active, int32_t max_iters,
              int32_t* iters_done, cudaStream_t stream) {
    if (!props || !active || max_iters < -1) return GM_ERR_INVALID_ARG;
    if (P::kAllActive && max_iters < 0) return GM_ERR_INVALID_ARG;  // it would never stop
    const int64_t n = V.n > 0 ? V.n : 1;
    const int64_t nwords = (n + 31) / 32;
    typename P::Msg* msgs = nullptr;
    uint32_t* bits = nullptr;  // has_msg, next_active
    unsigned long long* cnt = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&msgs), sizeof(typename P::Msg) * n, stream) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&bits), sizeof(uint32_t) * 2 * nwords, stream) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&cnt), sizeof(unsigned long long), stream) != cudaSuccess) {
        if (msgs) cudaFreeAsync(msgs, stream);
        if (bits) cudaFreeAsync(bits, stream);
        return GM_ERR_CUDA;
    }
    uint32_t* has_msg = bits;
    uint32_t* next = bits + nwords;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(sms * 4);
    gm_status st = GM_OK;
    int32_t it = 0;
    for (; (max_iters < 0 || it < max_iters) && V.n > 0; ++it) {
        unsigned long long h = 0;
        send_kernel<P><<<grid, kThreads, 0, stream>>>(prog, V.n, props, active, msgs, has_msg);
        cudaMemsetAsync(next, 0, sizeof(uint32_t) * nwords, stream);
        cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), stream);
        pull_kernel<P><<<grid, kThreads, 0, stream>>>(prog, V, msgs, has_msg, props, next, cnt);
        if (cudaGetLastError() != cudaSuccess) { st = GM_ERR_CUDA; break; }
        cudaMemcpyAsync(active, next, sizeof(uint32_t) * nwords, cudaMemcpyDeviceToDevice, stream);
        if (cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            st = GM_ERR_CUDA;
            break;
        }
        if (h == 0 && !P::kAllActive) { ++it; break; }  // the superstep that changed nothing is counted
    }
    cudaFreeAsync(msgs, stream);
    cudaFreeAsync(bits, stream);
    cudaFreeAsync(cnt, stream);
    if (iters_done) *iters_done = it;
    return st;
}

}  // namespace gm_program

#endif  // GRAPHMAT_PROGRAM_CUH
