/*
 * graphmat_gb300.h -- C ABI of the GraphMat superstep engine for NVIDIA GB300 (sm_103a).
 *
 * GraphMat (Sundaram et al., VLDB 2015) runs a vertex program as a sequence of
 * supersteps (Algorithm 2).  Each superstep turns the send_message outputs of the
 * active vertices into a sparse vector x, multiplies the transposed adjacency
 * matrix by x with process_message as the multiply and reduce as the add
 * (Algorithm 1, the generalized SPMV), applies the reduced values to the vertex
 * properties, and makes the vertices whose property changed active for the next
 * superstep.  This library runs that loop on one GPU for the built-in programs of
 * Section 3 (PageRank, BFS, SSSP, triangle counting, collaborative filtering).
 *
 * Conventions for every call:
 *  - Every call returns a gm_status; nothing aborts, traps or prints.
 *    gm_last_error() gives a one-line description of the last failure on the
 *    calling thread.
 *  - Input arrays are copied; the caller keeps ownership.  Outputs go to buffers
 *    the caller provides.  A handle and all device memory it owns are released
 *    only by gm_graph_destroy.
 *  - Pointers flagged "on_device"/"is_device" are CUDA device pointers of the
 *    current device; otherwise they are host pointers (pageable or pinned).
 *  - All GPU work of a handle is ordered on the CUDA stream given at creation
 *    (NULL = legacy default stream).  Calls that return data to the host
 *    synchronise that stream.  A handle must not be used by two host threads at
 *    once.
 *  - Vertex ids are int32 in [0, n); n < 2^31 and edge counts < 2^31 - 1.
 */
#ifndef GRAPHMAT_GB300_H
#define GRAPHMAT_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define GM_API __attribute__((visibility("default")))
#else
#define GM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gm_graph gm_graph;

typedef enum gm_status {
    GM_OK = 0,
    GM_ERR_INVALID_ARG = 1,    /* bad pointer, size, vertex id or program parameter */
    GM_ERR_OUT_OF_MEMORY = 2,  /* a device or pinned allocation failed */
    GM_ERR_CUDA = 3,           /* a CUDA runtime call failed (see gm_last_error) */
    GM_ERR_STATE = 4,          /* calls in the wrong order, e.g. gm_run before gm_program_set */
    GM_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    GM_ERR_UNSUPPORTED = 6     /* valid request the library does not handle */
} gm_status;

typedef enum gm_weight_type {
    GM_W_NONE = 0, /* unweighted: every edge value is 1 */
    GM_W_U32 = 1,  /* uint32 edge values (SSSP weights, CF ratings) */
    GM_W_F32 = 2   /* float edge values (weighted PageRank) */
} gm_weight_type;

/* An edge list: edge i goes from src[i] to dst[i] with value weight[i]. */
typedef struct gm_edge_list {
    int64_t n_vertices;   /* n */
    int64_t n_edges;      /* number of entries in src/dst/weight */
    const int32_t* src;
    const int32_t* dst;
    const void* weight;   /* NULL, or n_edges values of weight_type */
    int32_t weight_type;  /* gm_weight_type */
    int32_t on_device;    /* 1: src/dst/weight are device pointers; 0: host pointers */
    int64_t n_left;       /* collaborative filtering: users are [0, n_left), items [n_left, n) */
} gm_edge_list;

/* Ingest flags (Section 5.1 preprocessing). */
enum {
    GM_DROP_SELF_LOOPS = 1,   /* remove edges v -> v */
    GM_DEDUP = 2,             /* keep the first occurrence (input order) of each (src, dst) */
    GM_SYMMETRIZE = 4,        /* add dst -> src for every edge (after all originals, same value) */
    GM_ORIENT_BY_DEGREE = 8   /* keep u -> v only if (deg(u), u) < (deg(v), v): a DAG for triangle counting */
};

/*
 * gm_graph_create -- ingest an edge list into CSR (out-edges) and CSC (in-edges)
 * form on the GPU, with out/in-degrees and degree-binned vertex lists.
 * Paper: Section 4.3.1 (the matrix store; DCSC there, CSR + CSC here) and
 * Section 5.1 (self-loop removal, symmetrisation, orientation).
 *   el      edge list; ids outside [0, n) give GM_ERR_INVALID_ARG.
 *   flags   GM_* ingest flags, applied in the order symmetrise, drop self-loops,
 *           dedup, orient.
 *   stream  cudaStream_t for all work of this handle (NULL = default stream).
 *   out     receives the handle on GM_OK, NULL otherwise.
 * The call synchronises `stream` before returning.
 */
GM_API gm_status gm_graph_create(const gm_edge_list* el, uint32_t flags, void* stream, gm_graph** out);

/* Release the handle and all its device memory (synchronises its stream). NULL is a no-op. */
GM_API gm_status gm_graph_destroy(gm_graph* g);

/* Vertex count and edge count after cleaning. */
GM_API gm_status gm_graph_info(const gm_graph* g, int64_t* n_vertices, int64_t* n_edges);

/* Copy the cleaned edges in CSR order (sorted by (src, dst)): src, dst as int32
 * and, if the graph is weighted and `weight` is not NULL, the 4-byte values.
 * Any output pointer may be NULL.  Per-edge arrays of gm_wpagerank_* use this order. */
GM_API gm_status gm_graph_get_edges(const gm_graph* g, int32_t* src, int32_t* dst, void* weight,
                             int dst_is_device);

/* Out-degree and in-degree of every vertex (int32[n] each; either may be NULL). */
GM_API gm_status gm_graph_get_degrees(const gm_graph* g, int32_t* out_deg, int32_t* in_deg,
                               int dst_is_device);

typedef enum gm_program_kind {
    GM_PAGERANK = 0,        /* Eq. 1 */
    GM_BFS = 1,             /* Section 3.II */
    GM_SSSP = 2,            /* Section 3.V and the appendix program */
    GM_TRIANGLE_COUNT = 3,  /* Section 3.IV, two vertex programs (Section 4.2) */
    GM_CF = 4,              /* Section 3.III, Eqs. 2-5, gradient descent */
    GM_CONNECTED_COMPONENTS = 5, /* not one of the paper's programs: label propagation written with the
                                    user-program API of graphmat_program.cuh (Section 4's four functions);
                                    label(v) = min(label(v), labels received), labels start at the vertex
                                    id, every vertex active at the start; uint32 labels.  On a symmetrised
                                    graph the result is the smallest id of each connected component. */
    GM_CF_SGD = 6           /* Section 3.III, stochastic gradient descent: Eqs. 4-5 without their
                               sums, one rating at a time, each from the factors before that rating.
                               Order (Section 3.III asks for a random one): the stratified order of
                               distributed SGD -- user u in block u mod P, item v in block
                               (v - n_left) mod P, rating (u, v) in stratum (item block - user block)
                               mod P; an epoch runs strata 0..P-1, in a stratum user blocks 0..P-1,
                               in a block the ratings in (user, item) order.  gm_run(g, E) runs E
                               epochs.  Same state, parameters and loss as GM_CF, plus cf_strata. */
} gm_program_kind;

typedef struct gm_program_params {
    double r;              /* PageRank random-surf probability r of Eq. 1 (damping 0.85 -> r = 0.15) */
    int32_t pr_apply_all;  /* PageRank: 1 = Eq. 1 for every vertex (a vertex without in-edges gets r);
                              0 = Algorithm 2, apply only to vertices that received a message */
    int32_t K;             /* CF latent dimension (1..64) */
    double lambda;         /* CF regularisation weight of Eqs. 2, 4, 5 */
    double gamma;          /* CF step size of Eqs. 4, 5 */
    double init_sigma;     /* CF initial factors ~ N(0, init_sigma) */
    uint64_t seed;         /* CF initial-factor seed (counter-based SplitMix64 + Box-Muller) */
    int32_t cf_strata;     /* GM_CF_SGD: blocks per side P of the stratified order, 1..4096; 0 = about
                              sqrt(ratings) / 10 rounded to a power of two (GM_SCALAR_CF_STRATA
                              reads the value used) */
} gm_program_params;

/*
 * gm_program_set -- select the vertex program and (re)initialise the vertex
 * property of every vertex: PageRank 1.0 (Section 3.I), BFS/SSSP infinity =
 * UINT32_MAX (Sections 3.II, 3.V; appendix run_sssp), triangle counts 0, CF
 * factors N(0, init_sigma) drawn from `seed`.  No vertex is active afterwards
 * (except PageRank and CF, where all vertices are active every superstep).
 * `params` may be NULL for BFS, SSSP and triangle counting.
 * SSSP needs a GM_W_U32 graph (an unweighted graph uses weight 1); CF needs
 * n_left > 0 and GM_W_U32 ratings; GM_CF_SGD also needs every rating to go from
 * a user [0, n_left) to an item [n_left, n) (else GM_ERR_INVALID_ARG) and fewer
 * than 2^32 ratings.  GM_CF_SGD sorts the ratings into the stratified order here
 * (device memory: 16 bytes per rating kept, about 24 more during the sort, and
 * 4 (P^2 + 1) bytes of block pointers).
 */
GM_API gm_status gm_program_set(gm_graph* g, int32_t kind, const gm_program_params* params);

/*
 * Read-only device view of a graph handle for user-defined vertex programs
 * (graphmat_program.cuh).  Every pointer is device memory owned by the handle,
 * valid until gm_graph_destroy or an option that rebuilds the degree bins
 * (GM_OPT_BIN_SMALL / GM_OPT_BIN_LARGE).  CSC: the in-edges of v are
 * [col_ptr[v], col_ptr[v+1]) with sources row[] and uint32 weights cw[] (cw is
 * NULL unless the graph has GM_W_U32 weights); CSR likewise with row_ptr, col, w.
 * in_list holds the vertices with in-degree >= 1, bin b (1: < bin_small, ordered
 * by in-degree; 2: < bin_large; 3: the rest) at [in_off[b-1], in_off[b]);
 * zero_in lists the vertices without in-edges.  Errors: GM_ERR_INVALID_ARG for
 * a NULL argument.
 */
typedef struct gm_device_view {
    int64_t n, m;
    const int32_t* col_ptr;
    const int32_t* row;
    const uint32_t* cw;
    const int32_t* row_ptr;
    const int32_t* col;
    const uint32_t* w;
    const int32_t* in_list;
    int64_t in_off[4];
    const int32_t* zero_in;
    int64_t zero_in_count;
} gm_device_view;
GM_API gm_status gm_graph_device_view(const gm_graph* g, gm_device_view* out);

/*
 * gm_set_active -- mark vertices active for the next gm_run (appendix run_sssp:
 * the source gets distance 0 and is marked active).  BFS/SSSP: each listed
 * vertex gets property 0 and is active; several vertices make a multi-source
 * traversal.  count < 0 marks every vertex active (vertices is ignored).
 * Duplicate ids are allowed.  `src_is_device` says where `vertices` lives.
 */
GM_API gm_status gm_set_active(gm_graph* g, const int32_t* vertices, int64_t count, int src_is_device);

/*
 * gm_run -- Algorithm 2: run supersteps until no vertex is active or
 * `max_iters` supersteps have run (max_iters = -1: until no vertex is active, as
 * run_graph_program(..., -1, ...) in the appendix).  PageRank and CF run exactly
 * max_iters >= 0 supersteps (GM_CF_SGD: epochs, all in one cooperative launch).
 * Triangle counting runs its two programs and ignores max_iters.  iters_done
 * (may be NULL) receives the number of supersteps executed, counting the final
 * one that found no active vertex.  The call synchronises the stream.
 * Errors: GM_ERR_STATE before gm_program_set; GM_ERR_INVALID_ARG for
 * max_iters < -1 (and for -1 with PageRank or CF); GM_ERR_TIMEOUT when a bounded
 * device wait or guard gave up: an SSSP pull CTA's wait for its shared-memory
 * staging copy (the results stay exact: that CTA read the messages from global
 * memory), the traversal's n + 2 superstep guard (an internal error), or a
 * GM_CF_SGD grid barrier between strata that waited about ten seconds (the
 * factors are then unspecified; gm_program_set makes the handle usable again).
 */
GM_API gm_status gm_run(gm_graph* g, int32_t max_iters, int32_t* iters_done);

/*
 * Copy the vertex property array out: BFS/SSSP uint32[n], PageRank float[n],
 * triangle counting uint64[n] (triangles incident to each vertex), CF (both forms) float[n*K]
 * row-major.  `bytes` must equal that size.
 */
GM_API gm_status gm_get_vertex_state(gm_graph* g, void* dst, int64_t bytes, int dst_is_device);

/* Overwrite the vertex property array (same layout and size as above); used to
 * resume a run or to start CF from given factors.  Activity is not changed. */
GM_API gm_status gm_set_vertex_state(gm_graph* g, const void* src, int64_t bytes, int src_is_device);

enum {
    GM_SCALAR_TC_TOTAL = 1,       /* uint64: triangles in the graph */
    GM_SCALAR_CF_LOSS = 2,        /* double: Eq. 2 loss at the current factors (regulariser once per vertex) */
    GM_SCALAR_REACHED_EDGES = 3,  /* int64: sum of out-degrees of vertices with finite BFS/SSSP property */
    GM_SCALAR_SUPERSTEPS = 4,     /* int32: supersteps of the last gm_run */
    GM_SCALAR_PUSH_STEPS = 5,     /* int32: supersteps of the last gm_run run top-down (push) */
    GM_SCALAR_PULL_STEPS = 6,     /* int32: supersteps run bottom-up (pull) */
    GM_SCALAR_SCANNED_EDGES = 7,  /* int64: edges read by the relax kernels in the last gm_run */
    GM_SCALAR_RELAX_MS = 8,       /* double: profile mode, summed superstep-kernel time (CUDA events) */
    GM_SCALAR_RELAX_LAUNCHES = 9, /* int32: profile mode, relax-kernel launches timed */
    GM_SCALAR_PROCESSED_VERTICES = 10, /* int64: vertices whose edge lists the relax kernels read */
    GM_SCALAR_PULL_WEIGHT_BYTES = 11,  /* int32: bytes per in-edge weight the SSSP pull reads: 1 when
                                          every uint32 weight is below 256 (a one-byte copy is kept),
                                          4 otherwise, 0 for an unweighted graph; set at creation */
    GM_SCALAR_CF_STRATA = 12,          /* int32: blocks per side P of the GM_CF_SGD order in use */
    GM_SCALAR_PULL_STREAM_BYTES = 13   /* int64: bytes of in-edge data one SSSP pull superstep streams, for
                                          the layout in use: with GM_OPT_PULL_PACKED, 4 B per slot of the
                                          column lists padded to whole octets of 8 slots, a header byte per
                                          octet and 4 B per tile of 32 octets; otherwise 4 B + the weight
                                          width per in-edge, a first-edge bit per in-edge and 4 B per tile
                                          of 256 in-edges.  0 until an SSSP gm_program_set has built it. */
};
GM_API gm_status gm_get_scalar(gm_graph* g, int32_t which, void* out);

/*
 * Per-superstep trace of the last gm_run in profile mode (GM_OPT_PROFILE = 1):
 * up to max_rows rows of 10 doubles -- superstep index, direction (0 push, 1 pull),
 * active work items at its start, edges read, vertices whose edge lists were read,
 * time of the superstep's kernels in ms (push, pull and finalize, which holds the
 * SSSP Apply after a pull; CUDA events), the out-edges of the next frontier, the
 * time of the pull kernel alone (SSSP: the in-edge streaming kernel, BFS: the
 * bottom-up kernel, which counts in-edges checked), the time of the push kernel
 * alone and the time of the finalize kernel alone.  Both directions' kernels are
 * launched every superstep and the one not chosen returns at once, so the push
 * time of a pull superstep (and the pull time of a push superstep) is that early
 * return.
 * *n_rows receives the number of rows available.
 */
GM_API gm_status gm_get_trace(gm_graph* g, double* rows, int32_t max_rows, int32_t* n_rows);

/*
 * Differentiable weighted PageRank (an added form with no counterpart in the paper's
 * programs): Eq. 1 with learnable edge weights w normalised per source row,
 *   P_uv = w_uv / sum_v' w_uv',  x^0 = 1,  x^{t+1}_v = r + (1 - r) sum_{u->v} P_uv x^t_u.
 * gm_wpagerank_forward runs `steps` supersteps and writes x^steps; it keeps x^t
 * every `ckpt_every` supersteps (and the normalised weights) inside the handle.
 * gm_wpagerank_backward takes dL/dx^steps and writes dL/dw for the same w: a
 * reverse SpMV over the out-edges per superstep plus an edge-gradient
 * accumulation, recomputing each checkpoint segment, then the chain rule of the
 * row normalisation.
 *   w, dLdw   float[m] in the CSR edge order of gm_graph_get_edges, device memory;
 *             weights must be positive.
 *   x, dLdx   float[n], device memory.
 * The graph's own edge values are not used.  Calls synchronise the stream.
 */
GM_API gm_status gm_wpagerank_forward(gm_graph* g, const float* w, double r, int32_t steps, int32_t ckpt_every,
                                      float* x_out);
GM_API gm_status gm_wpagerank_backward(gm_graph* g, const float* dLdx, float* dLdw);

/*
 * gm_run_batch -- many BFS / SSSP queries (an added form: the programs of
 * Sections 3.II and 3.V) over one or more graphs, in one device-driven superstep
 * loop.  Queries of one program on one graph are bundled, up to 8 per bundle,
 * and run as one multi-source SpMSpV: a frontier byte per vertex (a bit per
 * query) and, for SSSP, a 32-byte row of 8 messages per vertex, so one pass over
 * the edges per superstep serves the whole bundle.  Each bundle pushes over its
 * frontier's out-edges or pulls over every in-edge, chosen on the device each
 * superstep from the frontier's out-edges and the graph handle's switch point
 * and direction option (gm_set_option / gm_autotune: SSSP pulls above
 * 4 x sssp_pull_frac of the edges, BFS above 1/alpha of them).  All bundles advance
 * in lockstep supersteps; a device work queue hands work of every bundle to the
 * warps; the loop is one CUDA graph whose conditional node stops when no query
 * is active.  Each query's result and superstep count equal gm_run's for the
 * same graph, program and single source.
 *   graphs     n_graphs handles (their programs and states are not touched).
 *   queries    n_queries entries: graph index, GM_BFS or GM_SSSP, source vertex.
 *   out_state  n_queries device pointers, uint32[n of the query's graph] each:
 *              depth / distance per vertex (UINT32_MAX = unreached).
 *   max_iters  -1: every query until convergence; k > 0: at most k supersteps.
 *   iters_done NULL or int32[n_queries] (host): supersteps of each query.
 *   stream     cudaStream_t (NULL = default); the call synchronises it.
 * Workspace (per bundle: two frontier bytes and two frontier lists of 8-byte
 * entries per vertex and per 256 edges, and a reached byte per vertex for BFS
 * or two 32-byte message rows per vertex for SSSP) is allocated
 * for the call and released before it returns.
 */
typedef struct gm_query {
    int32_t graph;   /* index into graphs */
    int32_t kind;    /* GM_BFS or GM_SSSP */
    int32_t source;  /* source vertex */
    int32_t reserved;
} gm_query;
GM_API gm_status gm_run_batch(gm_graph* const* graphs, int32_t n_graphs, const gm_query* queries, int32_t n_queries,
                              uint32_t* const* out_state, int32_t max_iters, int32_t* iters_done, void* stream);

/*
 * gm_bfs_csr_noalloc -- BFS over caller-provided CSR arrays that allocates no
 * memory.  The paper has no counterpart: this is a library convenience for callers
 * that cannot allocate device memory when they need a traversal, such as code
 * whose device memory is all owned by its own arena or caching allocator (a
 * cudaMalloc outside it can fail once the arena has reserved the free memory),
 * and latency-critical loops that must not pay for cudaMalloc/cudaFree (which can
 * synchronise the device and can fail under memory pressure).
 *
 * The result equals gm_run with GM_BFS from one source on the same edges:
 * depth[v] = number of edges on a shortest path from `source`, UINT32_MAX if
 * unreachable; *iters_done (may be NULL) = supersteps executed, counting the
 * final one that finds no new vertex.
 *   n        vertices, 1 <= n <= gm_bfs_csr_noalloc_max_vertices() (1,048,576);
 *            larger n returns GM_ERR_INVALID_ARG without touching the GPU.
 *   row_ptr  device int32[n+1], col device int32[row_ptr[n]]: out-edges of each
 *            vertex; ids in [0, n).  Read only; owned by the caller.
 *   depth    device uint32[n], written.
 *   stream   cudaStream_t for all work (NULL = default stream); the call copies
 *            the next frontier's size to the host and synchronises the stream
 *            once per superstep.
 * Scratch: two frontier queues and counters live in one fixed device array of
 * 8 MiB + 256 bytes that each GPU holds until the library is unloaded.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Every call shares the array and clears what it needs at
 * the start, so calls that overlap on the GPU (on different streams or host
 * threads) race and must not be issued.
 */
GM_API gm_status gm_bfs_csr_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col, int32_t source,
                                    uint32_t* depth, int32_t* iters_done, void* stream);
/* The largest n gm_bfs_csr_noalloc accepts (the size of its fixed scratch). */
GM_API int64_t gm_bfs_csr_noalloc_max_vertices(void);

/* Engine options (not program parameters). */
enum {
    GM_OPT_DIRECTION = 1,     /* 0 auto push/pull switch (default), 1 push only, 2 pull only */
    GM_OPT_LOOP_MODE = 2,     /* 0 superstep loop inside one CUDA graph (default), 1 host loop */
    GM_OPT_PROFILE = 3,       /* 1: host loop with CUDA events around every relax launch */
    GM_OPT_BIN_SMALL = 4,     /* degree below which vertices are processed 32 per warp */
    GM_OPT_BIN_LARGE = 5,     /* degree from which a whole CTA processes one vertex */
    GM_OPT_ALPHA_X1000 = 6,   /* BFS push->pull switch: frontier edges > unvisited in-edges / alpha */
    GM_OPT_BETA_X1000 = 7,    /* BFS pull->push switch: frontier vertices < n / beta */
    GM_OPT_SSSP_PULL_PPM = 8, /* SSSP: pull when frontier edges > ppm * 1e-6 * m */
    GM_OPT_PULL_STAGE = 9,    /* SSSP pull: messages of the highest-out-degree sources each CTA stages in
                                 shared memory, 0..49152 (rounded down to a multiple of 4; default 40960),
                                 counted as 4-byte messages; the pull over octets (one-byte weights) stores
                                 them as 16 bits and so stages twice as many sources in the same bytes */
    GM_OPT_TEST_STALL_STAGE = 10, /* test hook, 0 or 1: the SSSP pull's staging barrier expects 16 bytes more
                                     than its copies bring, so every CTA's bounded wait (about a second)
                                     runs out; those CTAs gather every message from global memory, the
                                     results stay exact, and gm_run returns GM_ERR_TIMEOUT */
    GM_OPT_TEST_STALL_SGD = 11,   /* test hook, 0 or 1: in GM_CF_SGD runs one CTA never arrives at the
                                     first grid barrier between strata and the barrier's wait limit is
                                     cut from about ten seconds to about half a second, so every CTA's
                                     wait runs out, the kernel ends, gm_run returns GM_ERR_TIMEOUT and
                                     the factors are left part-way through the first stratum */
    GM_OPT_PULL_PACKED = 12,      /* SSSP pull in-edge layout: 1 (default) one 32-bit word per in-edge,
                                     source rank << 8 | weight, when every weight is below 256 and
                                     n <= 2^24; 0 the source rank and the weight as separate arrays.
                                     Results are identical. */
    GM_OPT_SPARSE_LIST = 13       /* ablation of the sparse-vector form (Section 4.3.2, Fig. 7): 1 keeps
                                     each pull superstep's frontier as a sorted array of (index, value)
                                     tuples, rebuilt at its start, and the BFS/SSSP pull finds a source
                                     by binary search in it instead of one bitvector / dense-array load;
                                     runs the superstep loop from the host (as GM_OPT_LOOP_MODE = 1).
                                     0 (default): bitvector + dense array.  Results are identical. */
};
GM_API gm_status gm_set_option(gm_graph* g, int32_t option, int64_t value);

/*
 * gm_autotune -- pick the push/pull switch points (BFS: GM_OPT_ALPHA_X1000 and
 * GM_OPT_BETA_X1000; SSSP: GM_OPT_SSSP_PULL_PPM) and the degree-bin thresholds
 * (GM_OPT_BIN_SMALL, GM_OPT_BIN_LARGE) of this handle by timing gm_program_set +
 * gm_set_active + gm_run on the given host `sources` (coordinate descent over
 * small candidate sets, CUDA events on the handle's stream).  The chosen values
 * stay set on the handle and are reported in *out (may be NULL).  Tuning changes
 * only the work decomposition, never a result.  The current program state is
 * overwritten.
 */
typedef struct gm_tuning {
    double alpha, beta, sssp_pull_frac;
    int32_t bin_small, bin_large;
    double best_ms;  /* time of the sample with the chosen values */
    int32_t pull_stage;  /* GM_OPT_PULL_STAGE chosen (SSSP) */
} gm_tuning;
GM_API gm_status gm_autotune(gm_graph* g, int32_t kind, const int32_t* sources, int32_t n_sources, gm_tuning* out);

/*
 * Test hook for failure paths: after `n` more successful device allocations by
 * this library, every further allocation fails with GM_ERR_OUT_OF_MEMORY (the
 * calling entry point returns that status and frees what it allocated); n < 0
 * turns the hook off.  No GPU call fails: the check happens before the
 * allocation is requested.  Process-wide, all threads.
 */
GM_API void gm_debug_fail_allocations_after(int64_t n);

/* Number of kernel launches this library has issued since load (all handles). */
GM_API uint64_t gm_kernel_launch_count(void);

/* Readable name of a status code (static string). */
GM_API const char* gm_status_string(gm_status s);

/* One-line description of the last error on the calling thread ("" if none). */
GM_API const char* gm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GRAPHMAT_GB300_H */
