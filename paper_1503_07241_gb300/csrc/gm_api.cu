// C ABI: program selection, activity, the superstep driver and state access
// (Algorithm 2's Run_Graph_Program and the appendix's graph_program_init /
// run_graph_program / vertexproperty[] / active[] interface).
#include <cstring>

#include "gm_internal.cuh"

namespace gm {

gm_status build_bins(gm_graph* g);

namespace {

__global__ void fill_u32_k(uint32_t* p, int64_t n, uint32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

int64_t state_bytes(const gm_graph* g) {
    switch (g->kind) {
        case GM_BFS:
        case GM_SSSP: return 4 * g->n;
        case GM_PAGERANK: return 4 * g->n;
        case GM_TRIANGLE_COUNT: return 8 * g->n;
        case GM_CF:
        case GM_CF_SGD: return 4 * g->n * (int64_t)g->params.K;
        case GM_CONNECTED_COMPONENTS: return 4 * g->n;
        default: return -1;
    }
}

gm_status ensure_pinned(gm_graph* g) {
    if (!g->host_pinned) GM_CUDA_TRY(cudaMallocHost(&g->host_pinned, 4096));
    return GM_OK;
}

// SSSP on an unweighted graph relaxes with weight 1.
gm_status ensure_unit_weights(gm_graph* g) {
    if (g->w.p) return GM_OK;
    const int64_t m = g->m + kEdgePad;
    GM_TRY(dev_alloc(g->w, sizeof(uint32_t) * m, g->stream));
    GM_TRY(dev_alloc(g->cw, sizeof(uint32_t) * m, g->stream));
    fill_u32_k<<<num_sms() * 4, 256, 0, g->stream>>>(as<uint32_t>(g->w), g->m, 1u);
    fill_u32_k<<<num_sms() * 4, 256, 0, g->stream>>>(as<uint32_t>(g->cw), g->m, 1u);
    g_launches += 2;
    GM_CUDA_TRY(cudaGetLastError());
    GM_TRY(dev_alloc(g->cw8, (size_t)m, g->stream));  // unit weights fit in one byte
    GM_CUDA_TRY(cudaMemsetAsync(g->cw8.p, 1, (size_t)m, g->stream));
    g->wtype = GM_W_U32;
    return GM_OK;
}

}  // namespace
}  // namespace gm

using namespace gm;

extern "C" {

gm_status gm_program_set(gm_graph* g, int32_t kind, const gm_program_params* params) {
    if (!g) { set_error("gm_program_set: NULL handle"); return GM_ERR_INVALID_ARG; }
    gm_program_params p{};
    p.r = 0.15;
    p.pr_apply_all = 1;
    p.K = 32;
    p.lambda = 0.05;
    p.gamma = 1e-3;
    p.init_sigma = 0.1;
    p.seed = 0;
    p.cf_strata = 0;
    if (params) p = *params;
    switch (kind) {
        case GM_PAGERANK:
            if (!(p.r >= 0.0 && p.r <= 1.0)) { set_error("gm_program_set: r outside [0, 1]"); return GM_ERR_INVALID_ARG; }
            break;
        case GM_BFS:
        case GM_SSSP:
            break;
        case GM_TRIANGLE_COUNT:
        case GM_CONNECTED_COMPONENTS:
            break;
        case GM_CF:
        case GM_CF_SGD:
            if (g->n_left <= 0 || g->n_left >= g->n) {
                set_error("gm_program_set: CF needs a bipartite graph with 0 < n_left < n");
                return GM_ERR_INVALID_ARG;
            }
            if (g->wtype != GM_W_U32) {
                set_error("gm_program_set: CF needs uint32 ratings as edge values");
                return GM_ERR_INVALID_ARG;
            }
            if (p.K < 1 || p.K > 64 || !(p.gamma >= 0.0) || !(p.lambda >= 0.0) || !(p.init_sigma >= 0.0)) {
                set_error("gm_program_set: CF needs 1 <= K <= 64 and non-negative gamma, lambda, init_sigma");
                return GM_ERR_INVALID_ARG;
            }
            break;
        default:
            set_error("gm_program_set: unknown program kind %d", kind);
            return GM_ERR_INVALID_ARG;
    }
    GM_TRY(ensure_pinned(g));
    const bool traversal = kind == GM_BFS || kind == GM_SSSP;
    if (traversal && (g->kind == GM_BFS || g->kind == GM_SSSP) && g->state.p && g->work.p && g->ctl_buf.p) {
        // BFS <-> SSSP: keep the workspace and the cached loop graphs (same sizes)
        g->kind = kind;
        g->params = p;
        g->stats = RunStats{};
        gm_status st = kind == GM_SSSP ? ensure_unit_weights(g) : GM_OK;
        if (st == GM_OK) st = trav_reuse(g);
        if (st != GM_OK) g->kind = -1;
        return st;
    }
    if (kind == GM_PAGERANK && g->kind == GM_PAGERANK && g->state.p && g->work.p) {
        // PageRank again: keep the buffers and the cached superstep graph (it is
        // rebuilt at the next run only if r or the apply rule changed)
        g->params = p;
        g->stats = RunStats{};
        const gm_status st = pr_reset(g);
        if (st != GM_OK) g->kind = -1;
        return st;
    }
    trav_release(g);
    cf_release(g);
    pr_release(g);
    dev_free(g->state, g->stream);
    dev_free(g->work, g->stream);
    g->kind = kind;
    g->params = p;
    g->stats = RunStats{};
    gm_status st = GM_OK;
    if (kind == GM_BFS || kind == GM_SSSP) {
        if (kind == GM_SSSP) st = ensure_unit_weights(g);
        if (st == GM_OK) st = trav_prepare(g);
    } else if (kind == GM_PAGERANK) {
        st = pr_prepare(g);
    } else if (kind == GM_TRIANGLE_COUNT) {
        g->tc_total = 0;
        st = dev_alloc(g->state, sizeof(uint64_t) * (g->n > 0 ? g->n : 1), g->stream);
        if (st == GM_OK && g->n > 0) {
            cudaError_t e = cudaMemsetAsync(g->state.p, 0, sizeof(uint64_t) * g->n, g->stream);
            if (e != cudaSuccess) { set_error("gm_program_set: %s", cudaGetErrorString(e)); st = GM_ERR_CUDA; }
        }
    } else if (kind == GM_CF || kind == GM_CF_SGD) {
        st = cf_prepare(g);
    } else if (kind == GM_CONNECTED_COMPONENTS) {
        st = cc_prepare(g);
    }
    if (st != GM_OK) { g->kind = -1; return st; }
    GM_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return GM_OK;
}

gm_status gm_set_active(gm_graph* g, const int32_t* vertices, int64_t count, int src_is_device) {
    if (!g) { set_error("gm_set_active: NULL handle"); return GM_ERR_INVALID_ARG; }
    if (g->kind < 0) { set_error("gm_set_active: call gm_program_set first"); return GM_ERR_STATE; }
    if (count > 0 && !vertices) { set_error("gm_set_active: NULL vertices"); return GM_ERR_INVALID_ARG; }
    if (g->kind != GM_BFS && g->kind != GM_SSSP) return GM_OK;  // every vertex is always active
    if (count <= 0) return count < 0 ? trav_set_active(g, nullptr, -1) : GM_OK;
    cudaStream_t s = g->stream;
    if (src_is_device) {
        // ids are range-checked by the seeding kernel; a bad id fails the next gm_run
        return trav_set_active(g, vertices, count);
    }
    for (int64_t i = 0; i < count; ++i)
        if (vertices[i] < 0 || vertices[i] >= g->n) {
            set_error("gm_set_active: vertex id %d outside [0, %lld)", vertices[i], (long long)g->n);
            return GM_ERR_INVALID_ARG;
        }
    DevBuf tmp;
    GM_TRY(dev_alloc(tmp, sizeof(int32_t) * count, s));
    cudaError_t e = cudaMemcpyAsync(tmp.p, vertices, sizeof(int32_t) * count, cudaMemcpyHostToDevice, s);
    gm_status st = GM_OK;
    if (e != cudaSuccess) { set_error("gm_set_active: %s", cudaGetErrorString(e)); st = GM_ERR_CUDA; }
    if (st == GM_OK) st = trav_set_active(g, as<int32_t>(tmp), count);
    dev_free(tmp, s);  // stream-ordered: freed after the seeding kernel has read it
    return st;
}

gm_status gm_run(gm_graph* g, int32_t max_iters, int32_t* iters_done) {
    if (!g) { set_error("gm_run: NULL handle"); return GM_ERR_INVALID_ARG; }
    if (g->kind < 0) { set_error("gm_run: call gm_program_set first"); return GM_ERR_STATE; }
    if (max_iters < -1) { set_error("gm_run: max_iters must be >= -1"); return GM_ERR_INVALID_ARG; }
    switch (g->kind) {
        case GM_BFS:
        case GM_SSSP: return trav_run(g, max_iters, iters_done);
        case GM_PAGERANK: return pr_run(g, max_iters, iters_done);
        case GM_TRIANGLE_COUNT: return tc_run(g, iters_done);
        case GM_CF:
        case GM_CF_SGD: return cf_run(g, max_iters, iters_done);
        case GM_CONNECTED_COMPONENTS: return cc_run(g, max_iters, iters_done);
        default: break;
    }
    set_error("gm_run: program not available");
    return GM_ERR_UNSUPPORTED;
}

void gm_debug_fail_allocations_after(int64_t n) { g_alloc_budget.store(n < 0 ? -1 : n); }

gm_status gm_graph_device_view(const gm_graph* g, gm_device_view* out) {
    if (!g || !out) { set_error("gm_graph_device_view: NULL argument"); return GM_ERR_INVALID_ARG; }
    gm_device_view v{};
    v.n = g->n;
    v.m = g->m;
    v.col_ptr = as<int32_t>(g->col_ptr);
    v.row = as<int32_t>(g->row);
    v.cw = g->wtype == GM_W_U32 ? as<uint32_t>(g->cw) : nullptr;
    v.row_ptr = as<int32_t>(g->row_ptr);
    v.col = as<int32_t>(g->col);
    v.w = g->wtype == GM_W_U32 ? as<uint32_t>(g->w) : nullptr;
    v.in_list = as<int32_t>(g->in_list);
    for (int b = 0; b < 4; ++b) v.in_off[b] = g->in_list_count[b];
    v.zero_in = as<int32_t>(g->zero_in_list);
    v.zero_in_count = g->zero_in_count;
    *out = v;
    return GM_OK;
}

gm_status gm_get_vertex_state(gm_graph* g, void* dst, int64_t bytes, int dst_is_device) {
    if (!g) { set_error("gm_get_vertex_state: NULL handle"); return GM_ERR_INVALID_ARG; }
    if (g->kind < 0) { set_error("gm_get_vertex_state: no program set"); return GM_ERR_STATE; }
    const int64_t need = state_bytes(g);
    if (bytes != need || (need > 0 && !dst)) {
        set_error("gm_get_vertex_state: expected %lld bytes", (long long)need);
        return GM_ERR_INVALID_ARG;
    }
    if (need > 0)
        GM_CUDA_TRY(cudaMemcpyAsync(dst, g->state.p, (size_t)need,
                                    dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    GM_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return GM_OK;
}

gm_status gm_set_vertex_state(gm_graph* g, const void* src, int64_t bytes, int src_is_device) {
    if (!g) { set_error("gm_set_vertex_state: NULL handle"); return GM_ERR_INVALID_ARG; }
    if (g->kind < 0) { set_error("gm_set_vertex_state: no program set"); return GM_ERR_STATE; }
    const int64_t need = state_bytes(g);
    if (bytes != need || (need > 0 && !src)) {
        set_error("gm_set_vertex_state: expected %lld bytes", (long long)need);
        return GM_ERR_INVALID_ARG;
    }
    g->reached_valid = false;  // a property set by the caller: count reached vertices from the state
    if (need > 0)
        GM_CUDA_TRY(cudaMemcpyAsync(g->state.p, src, (size_t)need,
                                    src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    GM_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return GM_OK;
}

gm_status gm_get_scalar(gm_graph* g, int32_t which, void* out) {
    if (!g || !out) { set_error("gm_get_scalar: NULL argument"); return GM_ERR_INVALID_ARG; }
    switch (which) {
        case GM_SCALAR_TC_TOTAL:
            if (g->kind != GM_TRIANGLE_COUNT) { set_error("gm_get_scalar: not a triangle-count program"); return GM_ERR_STATE; }
            *static_cast<uint64_t*>(out) = g->tc_total;
            return GM_OK;
        case GM_SCALAR_CF_LOSS:
            if (g->kind != GM_CF && g->kind != GM_CF_SGD) {
                set_error("gm_get_scalar: not a CF program");
                return GM_ERR_STATE;
            }
            return cf_loss(g, static_cast<double*>(out));
        case GM_SCALAR_CF_STRATA:
            if (g->kind != GM_CF_SGD) { set_error("gm_get_scalar: not an SGD program"); return GM_ERR_STATE; }
            *static_cast<int32_t*>(out) = g->params.cf_strata;
            return GM_OK;
        case GM_SCALAR_REACHED_EDGES:
            if (g->kind != GM_BFS && g->kind != GM_SSSP) { set_error("gm_get_scalar: not a traversal program"); return GM_ERR_STATE; }
            return reached_edges(g, static_cast<int64_t*>(out));
        case GM_SCALAR_SUPERSTEPS: *static_cast<int32_t*>(out) = g->stats.supersteps; return GM_OK;
        case GM_SCALAR_PUSH_STEPS: *static_cast<int32_t*>(out) = g->stats.pushes; return GM_OK;
        case GM_SCALAR_PULL_STEPS: *static_cast<int32_t*>(out) = g->stats.pulls; return GM_OK;
        case GM_SCALAR_SCANNED_EDGES: *static_cast<int64_t*>(out) = g->stats.scanned_edges; return GM_OK;
        case GM_SCALAR_RELAX_MS: *static_cast<double*>(out) = g->stats.relax_ms; return GM_OK;
        case GM_SCALAR_RELAX_LAUNCHES: *static_cast<int32_t*>(out) = g->stats.relax_launches; return GM_OK;
        case GM_SCALAR_PROCESSED_VERTICES: *static_cast<int64_t*>(out) = g->stats.processed_vertices; return GM_OK;
        case GM_SCALAR_PULL_WEIGHT_BYTES:
            *static_cast<int32_t*>(out) = g->wtype == GM_W_NONE ? 0 : g->cw8.p ? 1 : 4;
            return GM_OK;
        case GM_SCALAR_PULL_STREAM_BYTES: {
            // in-edge data of one SSSP pull in the layout build_pull_edge_words built
            int64_t b = 0;
            if (g->oct_w.p) {
                b = g->oct_slots * 4 + g->oct_slots / kOctet + g->oct_tiles * 4;
            } else if (g->row_r.p) {
                const int64_t wb = g->cw8.p ? 1 : 4;
                b = g->m * (4 + wb) + (g->m + 7) / 8 + g->dc_ntiles * 4;
            }
            *static_cast<int64_t*>(out) = b;
            return GM_OK;
        }
        default: break;
    }
    set_error("gm_get_scalar: unknown scalar %d", which);
    return GM_ERR_INVALID_ARG;
}

gm_status gm_get_trace(gm_graph* g, double* rows, int32_t max_rows, int32_t* n_rows) {
    if (!g || (max_rows > 0 && !rows)) { set_error("gm_get_trace: NULL argument"); return GM_ERR_INVALID_ARG; }
    const int64_t avail = (int64_t)(g->stats.trace.size() / kTraceCols);
    if (n_rows) *n_rows = (int32_t)avail;
    const int64_t k = max_rows < avail ? max_rows : avail;
    for (int64_t i = 0; i < k * kTraceCols; ++i) rows[i] = g->stats.trace[(size_t)i];
    return GM_OK;
}

gm_status gm_set_option(gm_graph* g, int32_t option, int64_t value) {
    if (!g) { set_error("gm_set_option: NULL handle"); return GM_ERR_INVALID_ARG; }
    Tuning& t = g->tune;
    switch (option) {
        case GM_OPT_DIRECTION:
            if (value < 0 || value > 2) break;
            t.direction = (int32_t)value;
            return GM_OK;
        case GM_OPT_LOOP_MODE:
            if (value < 0 || value > 1) break;
            t.loop_mode = (int32_t)value;
            return GM_OK;
        case GM_OPT_PROFILE:
            t.profile = value ? 1 : 0;
            return GM_OK;
        case GM_OPT_BIN_SMALL:
        case GM_OPT_BIN_LARGE: {
            int64_t small = option == GM_OPT_BIN_SMALL ? value : t.bin_small;
            int64_t large = option == GM_OPT_BIN_LARGE ? value : t.bin_large;
            if (small < 1 || small > 4096 || large < small || large > (1ll << 30)) break;
            t.bin_small = (int32_t)small;
            t.bin_large = (int32_t)large;
            trav_release(g);  // the loop graph bakes the bin offsets in
            return build_bins(g);
        }
        case GM_OPT_ALPHA_X1000:
            if (value <= 0) break;
            t.alpha = value / 1000.0;
            return GM_OK;
        case GM_OPT_BETA_X1000:
            if (value <= 0) break;
            t.beta = value / 1000.0;
            return GM_OK;
        case GM_OPT_SSSP_PULL_PPM:
            if (value < 0 || value > 1000000) break;
            t.sssp_pull_frac = value * 1e-6;
            return GM_OK;
        case GM_OPT_PULL_STAGE:
            if (value < 0 || value > 49152) break;
            if (t.pull_stage == (int32_t)(value & ~(int64_t)3)) return GM_OK;
            t.pull_stage = (int32_t)(value & ~(int64_t)3);
            trav_release(g);  // the loop graph bakes the shared-memory size in
            return balance_octets(g, pull_stage16_messages(g));  // slot order for the new stage
        case GM_OPT_TEST_STALL_STAGE:
            if (value < 0 || value > 1) break;
            t.test_stall_stage = (int32_t)value;
            trav_release(g);
            return GM_OK;
        case GM_OPT_TEST_STALL_SGD:
            if (value < 0 || value > 1) break;
            t.test_stall_sgd = (int32_t)value;
            return GM_OK;
        case GM_OPT_SPARSE_LIST:
            if (value < 0 || value > 1) break;
            t.sparse_list = (int32_t)value;
            return GM_OK;
        case GM_OPT_PULL_PACKED:
            if (value < 0 || value > 1) break;
            if (t.pull_packed == (int32_t)value) return GM_OK;
            t.pull_packed = (int32_t)value;
            trav_release(g);  // the loop graph bakes the pull variant in
            if (g->src_rank.p) {  // ranks exist: rebuild the in-edge stream in the chosen layout
                GM_TRY(build_pull_edge_words(g));
                GM_CUDA_TRY(cudaStreamSynchronize(g->stream));
            }
            return GM_OK;
        default:
            set_error("gm_set_option: unknown option %d", option);
            return GM_ERR_INVALID_ARG;
    }
    set_error("gm_set_option: value %lld out of range for option %d", (long long)value, option);
    return GM_ERR_INVALID_ARG;
}

}  // extern "C"
