// Autotuner for the single-query traversal engine: picks the push/pull switch
// points and the degree-bin thresholds of a graph handle by timing real runs.
//
// Coordinate descent over small candidate sets, one knob at a time, each
// candidate timed with CUDA events on the handle's stream over the given sample
// sources (program set + seed + run, as a user would call them), best of three
// timed passes after one untimed pass.  The best value
// of each knob is kept before the next knob is tuned; the final choice is left
// set on the handle.  Results never depend on these knobs (they only change the
// work decomposition), so tuning cannot change any vertex property.
#include <algorithm>
#include <vector>

#include "gm_internal.cuh"

using namespace gm;

namespace {

gm_status time_once(gm_graph* g, int32_t kind, const int32_t* sources, int32_t n_sources, double* ms) {
    cudaEvent_t e0, e1;
    GM_CUDA_TRY(cudaEventCreate(&e0));
    GM_CUDA_TRY(cudaEventCreate(&e1));
    gm_status st = GM_OK;
    cudaEventRecord(e0, g->stream);
    for (int32_t i = 0; i < n_sources && st == GM_OK; ++i) {
        st = gm_program_set(g, kind, nullptr);
        if (st == GM_OK) st = gm_set_active(g, sources + i, 1, 0);
        if (st == GM_OK) st = gm_run(g, -1, nullptr);
    }
    cudaEventRecord(e1, g->stream);
    cudaEventSynchronize(e1);
    float f = 0.f;
    cudaEventElapsedTime(&f, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = f;
    return st;
}

// One untimed pass (a changed option may rebuild the loop graph), then the best of three.
gm_status time_sample(gm_graph* g, int32_t kind, const int32_t* sources, int32_t n_sources, double* ms) {
    double t = 0.0, best = 1e300;
    GM_TRY(time_once(g, kind, sources, n_sources, &t));
    for (int rep = 0; rep < 3; ++rep) {
        GM_TRY(time_once(g, kind, sources, n_sources, &t));
        best = std::min(best, t);
    }
    *ms = best;
    return GM_OK;
}

}  // namespace

extern "C" {

gm_status gm_autotune(gm_graph* g, int32_t kind, const int32_t* sources, int32_t n_sources, gm_tuning* out) {
    if (!g || !sources || n_sources < 1) { set_error("gm_autotune: NULL argument or no sources"); return GM_ERR_INVALID_ARG; }
    if (kind != GM_BFS && kind != GM_SSSP) { set_error("gm_autotune: only GM_BFS and GM_SSSP are tuned"); return GM_ERR_INVALID_ARG; }
    for (int32_t i = 0; i < n_sources; ++i)
        if (sources[i] < 0 || sources[i] >= g->n) { set_error("gm_autotune: source outside [0, n)"); return GM_ERR_INVALID_ARG; }
    const int32_t saved_loop = g->tune.loop_mode, saved_prof = g->tune.profile, saved_dir = g->tune.direction;
    g->tune.loop_mode = 0;
    g->tune.profile = 0;
    g->tune.direction = 0;
    double best = 0.0;
    GM_TRY(time_sample(g, kind, sources, n_sources, &best));
    // knob, candidates (x1000 for the real-valued ones)
    struct Knob { int32_t opt; std::vector<int64_t> vals; };
    std::vector<Knob> knobs;
    if (kind == GM_SSSP) {
        knobs.push_back({GM_OPT_SSSP_PULL_PPM, {5000, 20000, 50000, 100000, 200000, 350000, 1000000}});
        knobs.push_back({GM_OPT_PULL_STAGE, {0, 16384, 32768, 40960, 49152}});
    } else {
        knobs.push_back({GM_OPT_ALPHA_X1000, {2000, 6000, 14000, 30000, 80000}});
        knobs.push_back({GM_OPT_BETA_X1000, {6000, 24000, 96000}});
    }
    knobs.push_back({GM_OPT_BIN_LARGE, {256, 1024, 2048, 8192}});
    knobs.push_back({GM_OPT_BIN_SMALL, {8, 16, 32}});
    for (const Knob& k : knobs) {
        int64_t cur = 0;
        switch (k.opt) {
            case GM_OPT_SSSP_PULL_PPM: cur = (int64_t)(g->tune.sssp_pull_frac * 1e6 + 0.5); break;
            case GM_OPT_ALPHA_X1000: cur = (int64_t)(g->tune.alpha * 1e3 + 0.5); break;
            case GM_OPT_BETA_X1000: cur = (int64_t)(g->tune.beta * 1e3 + 0.5); break;
            case GM_OPT_BIN_LARGE: cur = g->tune.bin_large; break;
            case GM_OPT_BIN_SMALL: cur = g->tune.bin_small; break;
            case GM_OPT_PULL_STAGE: cur = g->tune.pull_stage; break;
        }
        int64_t best_v = cur;
        for (int64_t v : k.vals) {
            if (v == cur) continue;
            if (k.opt == GM_OPT_BIN_SMALL && v > g->tune.bin_large) continue;
            if (k.opt == GM_OPT_BIN_LARGE && v < g->tune.bin_small) continue;
            GM_TRY(gm_set_option(g, k.opt, v));
            double ms = 0.0;
            GM_TRY(time_sample(g, kind, sources, n_sources, &ms));
            if (ms < best) {
                best = ms;
                best_v = v;
            }
        }
        GM_TRY(gm_set_option(g, k.opt, best_v));
    }
    g->tune.loop_mode = saved_loop;
    g->tune.profile = saved_prof;
    g->tune.direction = saved_dir;
    if (out) {
        out->alpha = g->tune.alpha;
        out->beta = g->tune.beta;
        out->sssp_pull_frac = g->tune.sssp_pull_frac;
        out->bin_small = g->tune.bin_small;
        out->bin_large = g->tune.bin_large;
        out->best_ms = best;
        out->pull_stage = g->tune.pull_stage;
    }
    return GM_OK;
}

}  // extern "C"
