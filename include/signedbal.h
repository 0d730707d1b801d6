/*
 * signedbal.h -- C ABI of the GB300 (sm_103a) graphBpp / graphL library.
 *
 * Method: Shebaro & Tesic, "Scaling Frustration Index and Corresponding
 * Balanced State Discovery for Real Signed Graphs" (arXiv 2311.00869).
 *
 * Conventions for every entry point
 *   - Pointers are plain host or device pointers; sizes are int64_t.  Unless a
 *     function says otherwise, array arguments are DEVICE pointers on the
 *     context's device (a torch tensor's data_ptr() works).  Output arrays
 *     may instead be host pointers where marked "host or device": the library
 *     then copies through cudaMemcpyAsync and synchronises the stream.
 *   - The caller owns every buffer it passes.  The context owns the loaded
 *     graph, the labels of the last sampled batch, the cloud and its scratch.
 *   - Work is enqueued on the context's stream.  Calls that return host
 *     scalars (n_out, m_out, n_states_out, fr_min_out) synchronise it.
 *   - Errors are returned as negative sb_status codes; no C++ exception
 *     crosses the ABI.  sb_last_error() gives a one-line reason.  After
 *     SB_ERR_CUDA the context should be destroyed.
 *   - One context must not be used from two host threads at once.
 */
#ifndef SIGNEDBAL_H
#define SIGNEDBAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sb_ctx sb_ctx;
typedef int32_t sb_status;

#define SB_OK 0
#define SB_ERR_ARG (-1)          /* bad argument or size                              */
#define SB_ERR_CUDA (-2)         /* CUDA runtime error                                */
#define SB_ERR_OOM (-3)          /* allocation failed                                 */
#define SB_ERR_SELF_LOOP (-4)    /* input edge (v, v)                                 */
#define SB_ERR_BAD_SIGN (-5)     /* sign not +1 / -1                                  */
#define SB_ERR_INCONSISTENT (-6) /* same vertex pair present with both signs          */
#define SB_ERR_DUPLICATE (-7)    /* repeated pair and SB_LOAD_MERGE_DUP not set       */
#define SB_ERR_DISCONNECTED (-8) /* several components and SB_LOAD_LCC not set        */
#define SB_ERR_RANGE (-9)        /* vertex id outside [0, n)                          */
#define SB_ERR_STATE (-10)       /* call out of order (no graph, no sampled batch)    */
#define SB_ERR_CLOUD_FULL (-11)  /* cloud reached its state capacity                  */
#define SB_ERR_TIMEOUT (-12)     /* a bounded device wait gave up                     */
#define SB_ERR_DEVICE_CHECK (-13)/* a device-side consistency check failed            */

/* sb_load_graph flags */
#define SB_LOAD_LCC 1u        /* keep the largest connected component              */
#define SB_LOAD_MERGE_DUP 2u  /* merge repeated pairs of equal sign                */

/* Device memory hooks: alloc(bytes, stream, user) -> device pointer or NULL;
   free(ptr, stream, user). */
typedef void* (*sb_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*sb_free_fn)(void* ptr, void* stream, void* user);

/* One entry of the frustration cloud, Alg. 1 and Eq. 1: a distinct balanced
   state with its switch count S, its count C, the first tree that produced
   it, and its 64-bit state hash. */
typedef struct sb_cloud_entry {
    uint64_t hash;       /* sum of vertex weights over vertices labelled 1, mod 2^64 */
    int32_t S;           /* edge signs switched to reach the state (Algorithm 1)   */
    int32_t count;       /* trees that produced the state (Algorithm 1)           */
    int64_t first_tree;  /* global index of the first such tree                      */
} sb_cloud_entry;

/* ---------------------------------------------------------------- context */

/* Creates a context on CUDA device `device`; `cuda_stream` is a cudaStream_t
   (NULL = the legacy default stream).  *out is NULL on failure. */
sb_status sb_create(sb_ctx** out, int device, void* cuda_stream);
void sb_destroy(sb_ctx* ctx);
const char* sb_status_str(sb_status s);
const char* sb_last_error(const sb_ctx* ctx);
/* Replaces cudaMalloc/cudaFree for context-owned buffers (e.g. with a
   framework's caching allocator).  Call before sb_load_graph. */
sb_status sb_set_allocator(sb_ctx* ctx, sb_alloc_fn alloc, sb_free_fn free_fn, void* user);
/* Waits for the stream and reports any pending device error, including a
   device wait that ran out during sb_batch_steps (SB_ERR_TIMEOUT). */
sb_status sb_sync(sb_ctx* ctx);

/* Kernel families timed by the profiler (sb_profile / sb_profile_read). */
#define SB_PROF_BFS 0      /* tree sampler + labeller (cooperative BFS)        */
#define SB_PROF_SCORE 1    /* frustration counts                              */
#define SB_PROF_HASH 2     /* state hash                                      */
#define SB_PROF_CLOUD 3    /* cloud insertion and checks                      */
#define SB_PROF_INGEST 4   /* graph ingest                                    */
#define SB_PROF_GL_ROWS 5  /* graphL adjoint / descent step over CSR rows     */
#define SB_PROF_GL_FWD 6   /* graphL edge-parallel loss                       */
#define SB_PROF_OTHER 7    /* set-up and small kernels                        */
#define SB_PROF_N 8

/* Enables (1) or disables (0) CUDA-event timing of every kernel launch on the
   context's stream, by family.  Off by default. */
sb_status sb_profile(sb_ctx* ctx, int enable);
/* Waits for the stream, then writes the device time (ms) and number of
   kernel launches per family since the last read (host arrays of SB_PROF_N
   entries, nullable), and resets them.  Launch counts are kept even when
   timing is off. */
sb_status sb_profile_read(sb_ctx* ctx, double* ms_out, int64_t* launches_out);

/* Run-time tuning knobs (chosen by the package's autotuner; 0 = default):
   SB_TUNE_BFS_WORDS         64-tree words grown per BFS launch (1..32; 32)
   SB_TUNE_SCORE_BLOCKS_SM   scorer blocks per SM (0 = as many as fit)
   SB_TUNE_GL_LANES          graphL lanes per row segment: 8 (32 columns),
                             16 (64 columns) or 32 (128 columns) when
                             R % 4 == 0 (8)
   SB_TUNE_BFS_GROUP         lanes that share one vertex in the BFS, a power
                             of two in [1, 32]; used when it is at most twice
                             the launch's words rounded up to a power of two
                             (0 or otherwise: that power of two)
   SB_TUNE_WAIT_US           limit of every bounded device wait (the BFS grid
                             barrier between levels, the scorer's tile
                             copies), in microseconds at the device's SM
                             clock, 1 .. 6e7 (0 = 10 s).  A wait that runs
                             out makes its kernel stop early and the next
                             sb_label / sb_frustration return SB_ERR_TIMEOUT;
                             the context stays usable.
   SB_TUNE_STALL_TEST        1: the grid barriers of the next sb_sample_trees
                             call wait for one block more than the launch
                             has, so that every barrier wait runs out (a
                             test of the timeout path; no fault, nothing is
                             left running).  Reset to 0 by that call.
   SB_TUNE_MST_WORDS         64-tree words per pass of the Kruskal sampler,
                             1 .. 64 (0 = as many as its scratch budget of
                             32 GiB, at most half the free memory, holds)
   Results never depend on the first four, nor on SB_TUNE_MST_WORDS.
   sb_get_tuning returns the current value. */
#define SB_TUNE_BFS_WORDS 0
#define SB_TUNE_SCORE_BLOCKS_SM 1
#define SB_TUNE_GL_LANES 2
#define SB_TUNE_BFS_GROUP 3
#define SB_TUNE_WAIT_US 4
#define SB_TUNE_STALL_TEST 5
#define SB_TUNE_MST_WORDS 6
#define SB_TUNE_N 7
sb_status sb_set_tuning(sb_ctx* ctx, int32_t knob, int64_t value);
sb_status sb_get_tuning(sb_ctx* ctx, int32_t knob, int64_t* value);

/* Work counters of the last sb_sample_trees call (host array, n entries,
   n <= SB_STATS_N): [0] BFS levels (largest over its launches), [1] BFS
   launches, [2] neighbour entries scanned (per vertex-word lane),
   [3] hashed parent candidates of whole rows, [4] always 0 (kept so that
   the layout stays; every row is scanned in one pass), [5] hashed parent
   candidates of split rows.  All zero after sb_sample_trees_kruskal.
   Synchronises the stream. */
#define SB_STATS_N 6
sb_status sb_stats(sb_ctx* ctx, int64_t* out, int32_t n);

/* Measures the integer-ALU ceiling of the BFS's hash work on the context's
   device: a full grid evaluates, for `seconds` (0 < seconds <= 60), the
   parent-key hash of sb_sample_trees (one add of the tree salt, the 32-bit
   MurmurHash3 finaliser, one running minimum) on independent chains and
   nothing else, timed with CUDA events on the context's stream.
   *hashes_per_s_out (host) receives hashes per second.  Synchronous; for
   benchmarks (the roofline of the BFS sampler). */
sb_status sb_hash_peak(sb_ctx* ctx, double seconds, double* hashes_per_s_out);

/* ------------------------------------------------------------ graph ingest */

/*
 * Loads an undirected signed graph (Def. "Signed graph", Sec. 2) from a COO
 * list: edge i joins src[i] and dst[i] with sign[i] in {+1, -1}.  The
 * appendix "Implementation" paragraph describes the cleaning: self-loops and
 * invalid signs are errors, a pair with both signs is an inconsistency,
 * repeated pairs (either orientation) are merged with SB_LOAD_MERGE_DUP,
 * and with SB_LOAD_LCC the largest connected component is kept (most
 * vertices; ties go to the component with the smallest vertex id), its
 * vertices renumbered in increasing original id.  The first offending input
 * edge decides among range / self-loop / sign errors.
 * src, dst, sign: host or device, m entries each.  n >= 1, 2*m < 2^31.
 * Outputs (host pointers): *n_out, *m_out after cleaning.  vmap_out (host or
 * device, n entries, nullable) receives old id -> new id or -1.
 * Synchronous.  Replaces any previous graph and clears the cloud.
 */
sb_status sb_load_graph(sb_ctx* ctx, int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                        const int8_t* sign, uint32_t flags, int64_t* n_out, int64_t* m_out, int32_t* vmap_out);

/* Exports the cleaned edge list: u < v, lexicographic order, neg = 1 for a
   negative edge.  Each pointer host or device, m_out entries, nullable. */
sb_status sb_graph_edges(sb_ctx* ctx, int32_t* u_out, int32_t* v_out, int8_t* neg_out);

/* Exports the CSR (rows sorted ascending): rowptr n+1 entries, col and neg
   2m entries.  Host or device, nullable. */
sb_status sb_graph_csr(sb_ctx* ctx, int32_t* rowptr_out, int32_t* col_out, int8_t* neg_out);

/*
 * Loads a batch of G signed graphs as one disjoint union, to run thousands of
 * small uneven graphs through the same launches (each sb_* call then works on
 * every graph at once).  Graph g has nv[g] vertices with local ids
 * [0, nv[g]) and the input edges [eofs[g], eofs[g+1]) of src / dst / sign
 * (host or device, local ids).  Each graph is cleaned on its own exactly as
 * sb_load_graph cleans one graph (with SB_LOAD_LCC: its own largest
 * component); errors name the first offending edge of the whole input.
 * nv, eofs: host, G and G+1 entries (eofs[0] = 0).  Outputs (host, G entries,
 * nullable): vertices and edges of each cleaned graph.  Cleaned graph g holds
 * the union's vertices [sum of earlier nv_out, ...) in order.
 * In a batch, sb_sample_trees(seed, t0, K) samples K trees in EVERY graph:
 * tree t of graph g is exactly tree t of sb_load_graph(graph g) with the
 * same seed (ids are taken inside each graph).  sb_frustration then returns
 * G x K counts / hashes (graph-major), and sb_label canonicalises each graph
 * by its own vertex 0.  graphL runs on the union (the graphs share no edge,
 * so rows and gradients are per graph); every per-column output becomes
 * per (graph, column), G x R graph-major: sb_graphL_fwd's loss and F,
 * sb_graphL_round's F, and sb_graphL_descent's exps, F_trace rows and
 * F_final, whose renormalisation is decided per graph and column.
 * sb_cloud is not available on a batch: use sb_batch_cloud.
 */
sb_status sb_load_batch(sb_ctx* ctx, int64_t n_graphs, const int64_t* nv, const int64_t* eofs, const int32_t* src,
                        const int32_t* dst, const int8_t* sign, uint32_t flags, int64_t* nv_out, int64_t* m_out);

/*
 * Frustration cloud of every graph of a batch for the trees of the last
 * sb_sample_trees (K <= 1024): the distinct states of each graph's K trees,
 * checked bit for bit on every hash match (Algorithm 1).  Host or
 * device outputs: n_states_out[G], fr_min_out[G] (= min S, Eq. 1), and
 * entries_out[G x K] (nullable): graph g's states at [g*K, g*K + n_states[g])
 * in order of first appearance.
 */
sb_status sb_batch_cloud(sb_ctx* ctx, int32_t* n_states_out, int32_t* fr_min_out, sb_cloud_entry* entries_out);

/*
 * `steps` graphBpp steps on the loaded batch of graphs (Algorithm 1 on every
 * graph at once) with no host synchronisation: step i samples the BFS trees
 * [tree_begin + i K, tree_begin + (i + 1) K) in every graph, counts and
 * hashes their states and builds each graph's cloud of the step's trees,
 * exactly as sb_sample_trees, sb_frustration and sb_batch_cloud do.
 * use_graph = 1 runs the first step directly, captures the second into a CUDA
 * graph (once; it is replayed while seed, K, the batch and the tuning stay the
 * same) and replays it for the remaining steps; the device holds the first
 * tree of the current step and every replay moves it on by K.  use_graph = 0
 * enqueues every step's kernels directly.  The results are the same.
 * Outputs (device, G entries, nullable): fr_min_out[g] = the smallest S of
 * graph g over all the steps' trees; n_states_out[g] = the distinct states of
 * graph g in the last step.  The call only enqueues work on the context's
 * stream: the outputs are ready, and a device wait that ran out during the
 * steps is reported (SB_ERR_TIMEOUT), by sb_sync.  Afterwards sb_label,
 * sb_frustration and sb_batch_cloud see the last step's trees.
 * K in [1, 1024], steps >= 1; SB_ERR_STATE without a batch of graphs.
 */
sb_status sb_batch_steps(sb_ctx* ctx, uint64_t seed, int64_t tree_begin, int64_t K, int32_t steps, int32_t use_graph,
                         int32_t* fr_min_out, int32_t* n_states_out);

/* ---------------------------------------------------------------- graphBpp */

/*
 * Samples trees [tree_begin, tree_begin + K) and their balanced states
 * (Algorithm 1; appendix graphB+ algorithm).  Tree t is the
 * randomized BFS tree defined by
 *     S   = mix64(seed + G),  K_t = mix64(S + (t + 1) G),  G = 0x9E3779B97F4A7C15
 *     root r_t = ((K_t >> 32) * n) >> 32
 *     parent of v = argmin over neighbours u one BFS level up of
 *                   (fmix32((u ^ y_v) + lo32(K_t)) << 32) | u,
 *     y_v = hi32(mix64(v ^ S ^ 0xD1B54A32D192ED03))
 * (mix64 = SplitMix64 finaliser, fmix32 = MurmurHash3 finaliser), and its
 * state labels each vertex with the parity of negative tree edges on its
 * root path, canonicalised so vertex 0 has label 0.  A tree is a pure
 * function of (seed, t): splitting a range gives the same trees.
 * K >= 1 (at most 64 * 64 per call).  parents_out (device, K x n int32,
 * nullable; -1 at the root) costs extra shared memory: meant for checks on
 * small graphs.  Replaces the previous batch.
 */
sb_status sb_sample_trees(sb_ctx* ctx, uint64_t seed, int64_t tree_begin, int64_t K, int32_t* parents_out);

/*
 * Samples trees [tree_begin, tree_begin + K) with the randomized Kruskal
 * sampler (appendix, tree samplers: Kruskal's algorithm on random edge
 * weights drawn afresh for every tree) and their balanced states, in place of
 * sb_sample_trees: sb_label, sb_frustration and sb_cloud then work on these
 * trees the same way.  Tree t is the minimum spanning tree under the weights
 *     w_t(u, v) = mix64(((u << 32) | v) ^ K_t)
 * of the cleaned edges (u < v; ids local to each graph in a batch; K_t as in
 * sb_sample_trees).  mix64 is a bijection, so the weights of one tree are
 * distinct and the tree is unique (Prim's algorithm on the same weights finds
 * it too).  The state labels each vertex with the parity of negative tree
 * edges between it and vertex 0 (canonical: vertex 0 has label 0).  A tree is
 * a pure function of (seed, t).  Works on a single graph and on a batch.
 * K >= 1 (at most 64 * 64 per call).  in_tree_out (device, K x m bytes,
 * nullable; edge order of sb_graph_edges): 1 where the edge is in the tree.
 * Scratch: 36 bytes per (vertex, tree); a pass of trees takes at most
 * 16 GiB and half the free device memory (at least 64 trees per pass).  The
 * context keeps it for the next call until a graph is loaded or the context
 * is destroyed.
 * Errors: SB_ERR_ARG, SB_ERR_STATE (no graph), SB_ERR_OOM; a tree that does
 * not span its graph (an internal error) is reported as SB_ERR_DEVICE_CHECK
 * by the next sb_label / sb_frustration.  Replaces the previous batch.
 */
sb_status sb_sample_trees_kruskal(sb_ctx* ctx, uint64_t seed, int64_t tree_begin, int64_t K, uint8_t* in_tree_out);

/* Canonical labels of the last batch, bit-packed vertex-major:
   labels_out[v * W + w] bit b = label of tree tree_begin + 64 w + b at vertex v,
   W = ceil(K / 64); bits of trees >= K are 0.  Host or device. */
sb_status sb_label(sb_ctx* ctx, uint64_t* labels_out);

/* Algorithm 1 for each tree of the last batch: counts_out[i] = number of
   edges whose sign differs between the graph and the state of tree
   tree_begin + i (label(u) XOR label(v) XOR neg).  hashes_out[i] = state
   hash.  Host or device; hashes_out nullable. */
sb_status sb_frustration(sb_ctx* ctx, int32_t* counts_out, uint64_t* hashes_out);

/*
 * Inserts the last batch into the context's frustration cloud (Alg. 1 lines
 * 8-14; the key is the canonical state, checked bit for bit whenever two
 * trees share a hash) and exports it: entries in order of first appearance.
 * out: host or device, cap entries; out = NULL with cap = 0 only inserts
 * and reports.  Host outputs: *n_states_out, *fr_min_out = min S (Eq. 1;
 * nullable).  Returns SB_ERR_CLOUD_FULL when the cloud's capacity was
 * reached (entries beyond it are dropped and counted nowhere) or when
 * 0 < cap < n_states (then only cap entries are written).  The cloud accumulates across batches until
 * sb_cloud_reset or sb_load_graph.
 */
sb_status sb_cloud(sb_ctx* ctx, sb_cloud_entry* out, int64_t cap, int64_t* n_states_out, int32_t* fr_min_out);

/* Empties the cloud; max_states (0 = 4096) sets its capacity in states.
   hash_bits in [1, 64] (0 = 64) truncates the table key for testing the
   collision path; exported hashes stay full. */
sb_status sb_cloud_reset(sb_ctx* ctx, int64_t max_states, int32_t hash_bits);

/* Empties the cloud and switches it to the scalable rule of the paper's
   appendix algorithm for large graphs (alg-scale), with room for f_max states
   (1 <= f_max <= 2^30): trees are taken in order; the first stored state opens
   the cloud; after that a tree counts only when its S is below the largest
   stored S, raising the count of its stored state, or else adding its state
   while fewer than f_max are stored, or else replacing a stored state of
   largest S (the paper's argmin there would replace the best state; the
   lowest index among equal S goes).  A state's first_tree is the tree that
   stored it.  Trees that do not count are not errors (no SB_ERR_CLOUD_FULL);
   two different states with one 64-bit hash give SB_ERR_DEVICE_CHECK.
   sb_cloud_reset returns to the unbounded cloud. */
sb_status sb_cloud_reset_scalable(sb_ctx* ctx, int64_t f_max);

/* Canonical labels of cloud state `idx` (order of sb_cloud), bit-packed:
   bits_out[v / 64] bit (v % 64) = label of vertex v.  ceil(n/64) words,
   host or device. */
sb_status sb_cloud_state(sb_ctx* ctx, int64_t idx, uint64_t* bits_out);

/* The edges that cloud state `idx` (order of sb_cloud) switches to reach its
   balanced signing -- the paper's output "list of edges to switch" (Sec. 3,
   the frustration cloud; Sec. 6): bit e % 64 of edge_bits_out[e / 64] is 1
   when edge e (order of sb_graph_edges) has lab[u] ^ lab[v] ^ neg = 1.
   ceil(m/64) words, host or device; n_switched_out (host, nullable)
   receives their number, which equals the state's S.  Not available on a
   batch of graphs (SB_ERR_STATE); synchronises the stream. */
sb_status sb_cloud_switch(sb_ctx* ctx, int64_t idx, uint64_t* edge_bits_out, int64_t* n_switched_out);

/* ------------------------------------------------------------------ graphL */

/*
 * Relaxed loss of Eq. 3 and discrete loss of Eq. 2 (Algorithm 2) for R
 * starting points at once: gamma is n x R float32 row-major (gamma[v*R + r]).
 * loss_out[r] = sum over edges (1 - e_uv G_u G_v) / 2, each undirected edge
 * once; F_out[r] = edges with e_uv theta_u theta_v = -1, theta = +1 iff
 * G >= 0 (nullable).  Edge-parallel, deterministic.  Device pointers.
 */
sb_status sb_graphL_fwd(sb_ctx* ctx, const float* gamma, int32_t R, float* loss_out, int32_t* F_out);

/*
 * Adjoint of sb_graphL_fwd (Eq. 4): grad_out[v*R + r] =
 * -1/2 * gout[g*R + r] * sum_{j in N(v)} e_vj gamma[j*R + r], g = the graph
 * of v (0 for one graph; gout is G x R in a batch, like the losses),
 * summed over CSR rows in a fixed order (no float atomics; bitwise
 * reproducible).  Device pointers.
 */
sb_status sb_graphL_bwd(sb_ctx* ctx, const float* gamma, int32_t R, const float* gout, float* grad_out);

/*
 * Alg. 2 descent from gamma0 for `steps` updates G <- G - alpha dL/dG (every
 * start point weighted 1).  After each update a column whose largest |G|
 * reached 2^renorm_log2 is scaled by 2^-renorm_log2 and exps_out[r] grows by
 * renorm_log2 (0 disables; powers of two keep every sign and every rounded
 * value).  gamma_out receives the final G (n x R); exps_out (int32 R);
 * F_trace (int32 steps x R, nullable) the discrete loss before each update;
 * F_final (int32 R, nullable) the discrete loss of the final G (Alg. 2 lines
 * 11-24).  Device pointers; gamma0 and gamma_out may alias.
 */
sb_status sb_graphL_descent(sb_ctx* ctx, const float* gamma0, float* gamma_out, int32_t R, float alpha, int32_t steps,
                            int32_t renorm_log2, int32_t* exps_out, int32_t* F_trace, int32_t* F_final);

/*
 * Alg. 2 final loop: theta = +1 iff G >= 0, F_out[r] = frustrated edges
 * (exact integer), flip_out (nullable) bit-packed per start point:
 * flip_out[r * ceil(m/64) + i/64] bit i%64 = 1 when edge i (order of
 * sb_graph_edges) must switch sign.  Device pointers.
 */
sb_status sb_graphL_round(sb_ctx* ctx, const float* gamma, int32_t R, int32_t* F_out, uint64_t* flip_out);

/*
 * Allocation-free variant of sb_graphL_fwd (the paper has no counterpart;
 * this is an integration convenience).  For callers that cannot allocate
 * device memory at call time because their memory is fixed ahead of time:
 * hosts that hand the library a fixed memory budget up front, plugins whose
 * host application owns every allocator, and loops that must not enter the
 * CUDA allocator while they run.  It takes no context
 * and calls no cudaMalloc, cudaFree or allocating library routine; its
 * scratch is a fixed device array of about 2.4 MiB that every GPU loading the
 * library keeps until exit.
 *   edges: device array of m (u, v | neg << 31) int32 pairs, the cleaned edge
 *          list in the layout of the context's own (u < v; neg = 1 for a
 *          negative edge; sb_graph_edges gives its parts).
 *   gamma (n x R float32), loss_out (R), F_out (R, nullable): device, as for
 *          sb_graphL_fwd, on the current CUDA device.
 *   cuda_stream: cudaStream_t (NULL = legacy default stream).
 * Limits: 1 <= R <= 1024 and 0 <= m < 2^31, else SB_ERR_ARG and nothing runs.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) and should come before any stream capture.  That
 * address is kept per device for the life of the process, so every call must
 * run in the device's primary context (the CUDA runtime's own); a driver
 * context made current by the caller, or a cudaDeviceReset between calls,
 * is not supported.  All calls on a device share the scratch and it keeps the
 * last call's contents: calls that overlap on the GPU race and must be
 * serialised by the caller.  A CUDA error already pending when the call is
 * made (from the caller's earlier work) is left in place and the call returns
 * SB_ERR_CUDA without launching anything.
 */
sb_status sb_graphL_fwd_static(const int32_t* edges, int64_t m, const float* gamma, int32_t R, float* loss_out,
                               int32_t* F_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SIGNEDBAL_H */
