// Connected components by label propagation: a vertex program outside the
// paper's five, written with the user-program API of graphmat_program.cuh
// (Section 4's Send_Message / Process_Message / Reduce / Apply):
//   send: the vertex's label;  process: the label received;  reduce: min;
//   apply: label(v) = min(label(v), reduced), active if it fell.
// Labels start at the vertex id with every vertex active; on a symmetrised
// graph they converge to the smallest id of each connected component, on a
// directed graph to the smallest id of any vertex with a path to v.
#include "gm_internal.cuh"
#include "graphmat_program.cuh"

namespace gm {

namespace {

struct LabelProp {
    using Prop = uint32_t;
    using Msg = uint32_t;
    using Acc = uint32_t;
    static constexpr bool kAllActive = false;
    static constexpr bool kApplyToAll = false;
    __device__ bool send(int32_t, const uint32_t& p, uint32_t& m) const {
        m = p;
        return true;
    }
    __device__ uint32_t process(const uint32_t& m, uint32_t, const uint32_t&) const { return m; }
    __device__ uint32_t reduce(const uint32_t& a, const uint32_t& b) const { return a < b ? a : b; }
    __device__ uint32_t identity() const { return 0xFFFFFFFFu; }
    __device__ bool apply(const uint32_t& y, uint32_t& p) const {
        if (y < p) {
            p = y;
            return true;
        }
        return false;
    }
};

// label[v] = v; every vertex active (bits past n stay clear).
__global__ void cc_init(uint32_t* __restrict__ label, uint32_t* __restrict__ active, int64_t n) {
    const int64_t nwords = (n + 31) / 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        label[i] = (uint32_t)i;
    for (int64_t wd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wd < nwords;
         wd += (int64_t)gridDim.x * blockDim.x) {
        const int64_t left = n - wd * 32;
        active[wd] = left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
    }
}

}  // namespace

// State: uint32 labels; workspace: the active bitvector.
gm_status cc_prepare(gm_graph* g) {
    cudaStream_t s = g->stream;
    const int64_t n = g->n > 0 ? g->n : 1;
    GM_TRY(dev_alloc(g->state, sizeof(uint32_t) * n, s));
    GM_TRY(dev_alloc(g->work, sizeof(uint32_t) * ((n + 31) / 32), s));
    g->work_bytes = (int64_t)(sizeof(uint32_t) * ((n + 31) / 32));
    if (g->n > 0) {
        cc_init<<<num_sms() * 4, 256, 0, s>>>(as<uint32_t>(g->state), as<uint32_t>(g->work), g->n);
        g_launches++;
        GM_CUDA_TRY(cudaGetLastError());
    }
    return GM_OK;
}

gm_status cc_run(gm_graph* g, int32_t max_iters, int32_t* iters_done) {
    gm_device_view V;
    GM_TRY(gm_graph_device_view(g, &V));
    int32_t it = 0;
    const gm_status st = gm_program::run(V, LabelProp{}, as<uint32_t>(g->state), as<uint32_t>(g->work), max_iters,
                                         &it, g->stream);
    if (st != GM_OK) {
        set_error("gm_run: connected components: %s", st == GM_ERR_CUDA ? "CUDA error" : "invalid argument");
        return st;
    }
    g_launches += 2ull * (uint64_t)it;
    g->stats = RunStats{};
    g->stats.supersteps = it;
    if (iters_done) *iters_done = it;
    return GM_OK;
}

}  // namespace gm
