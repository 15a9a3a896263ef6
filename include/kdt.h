/*
 * kdt.h - C ABI of the GB300 k-d tree query library.
 *
 * Find-closest-point (fcp) and k-nearest-neighbour (kNN) queries over a
 * left-balanced, complete k-d tree stored in level order, traversed with the
 * stack-free (curr, prev) state machine of Wald, "A Stack-Free Traversal
 * Algorithm for Left-Balanced k-d Trees" (arXiv 2210.12859), Sec. 3.
 *
 * Conventions shared by every entry point:
 *   - Pointers prefixed d_ are DEVICE pointers on the current CUDA device,
 *     owned by the caller; pointers prefixed h_ are HOST pointers owned by the
 *     caller.  Point and query arrays are dense row-major float32 [count][D].
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue their work on it and return without waiting,
 *     unless the entry point says it synchronises.
 *   - Every call returns KDT_OK (0) or a negative KDT_E* status; the text of
 *     the last failure on the calling host thread is kdt_last_error().
 *   - IDs are indices of the input points (within their own cloud for the
 *     batched calls), not node indices.  Result rows are sorted ascending by
 *     (squared distance, id); empty slots hold id -1 and distance +inf.
 *   - Squared distances are FP32: d2 = ((t_0 + t_1) + t_2) + ..., with
 *     t_j = (p_j - q_j)^2 each rounded to float, no fused multiply-add.  A
 *     point is a candidate iff d2 <= max_radius * max_radius (rounded to
 *     float); ties in d2 go to the smaller id.  The result is the exact
 *     k-best set under that order whatever flags are used.
 *   - Objects (kdt_tree, kdt_forest) are not thread-safe: serialise calls
 *     that use one object on one stream.
 */
#ifndef KDT_H
#define KDT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define KDT_OK          0
#define KDT_EINVAL     -1  /* bad argument: N < 1, D outside [1,8], k outside [1,64], Q < 0,
                              max_radius < 0 or NaN, N >= 2^30, NULL pointer, ... */
#define KDT_ENONFINITE -2  /* a point coordinate is NaN or infinite */
#define KDT_ENOMEM     -3  /* device or host allocation failed */
#define KDT_ECUDA      -4  /* a CUDA runtime call failed */
#define KDT_ETRAVERSAL -5  /* a traversal exceeded its step bound (never for a valid tree) */
#define KDT_ENOMODEL   -6  /* KDT_LEARNED requested but the tree has no trained radius model */
#define KDT_EIO        -7  /* model file could not be read or written, or has a bad header */

/* ---- query flags ------------------------------------------------------- */
#define KDT_ORDERED    0x0 /* close child first (Sec. 3, ordered traversal), the default */
#define KDT_UNORDERED  0x1 /* left child first; a child is entered iff the query is on its
                              side or the splitting plane is within the cull radius
                              (Sec. 3: unordered traversal as a simplification) */
#define KDT_MORTON     0x2 /* sort queries along a 30-bit Morton curve before traversal so
                              that the threads of a warp walk nearby paths; results are
                              written to the caller's query order */
#define KDT_LEARNED    0x4 /* seed each query's cull radius with the trained radius model
                              and re-run the queries that find fewer than k points with
                              the caller's radius (not in the paper; results unchanged) */
#define KDT_NO_STAGE   0x8 /* do not stage the top tree levels in shared memory */
#define KDT_COST_ORDER 0x20 /* with KDT_MORTON, single trees with D <= 3: run the queries in cost
                              classes, most expensive first (judged by how far the greedy
                              descent ends from its leaf point, relative to the mean point
                              spacing: one class per power of two of that squared distance
                              beyond 64 spacings squared, three below), Morton order within a
                              class.  Pays when a few queries cost far more than the rest
                              (queries outside the data); costs one descent per query */
/* Traversal ablations (ordered kNN / fcp, k <= 16, D <= 4; at most one; not
 * with KDT_UNORDERED or KDT_LEARNED).  Same results as without them; they
 * measure the choices around Sec. 3's stack-free traversal, for which the
 * paper makes no speed claim against a stack-based one: */
#define KDT_PLAIN_STEP  0x40  /* the stack-free machine as stated: one node per step, no
                                 inlined bottom subtrees */
#define KDT_CLOSE_FIRST 0x80  /* process a node after its close subtree instead of before
                                 it (the order swap the footnote of Sec. 3.1 allows) */
#define KDT_STACK       0x100 /* a stack-based traversal (far child pushed with its plane
                                 distance, culled when popped): the recursion of Sec. 3.1
                                 with an explicit per-thread stack */

/* ---- build options ----------------------------------------------------- */
#define KDT_BUILD_ASYNC 0x1 /* kdt_build_ex: do not synchronise to check the points for
                               NaN / inf; the check result is reported by kdt_status */
#define KDT_BUILD_WIDEST 0x2 /* kdt_build_ex, D <= 3: store a split dimension in every node
                               instead of using level mod D (Sec. 3 leaves splitDimOf open
                               between the two): the dimension of widest extent (largest
                               max - min, rounded to float) of the node's points, ties to the
                               lowest dimension; otherwise the same median rule */

typedef struct kdt_tree kdt_tree;
typedef struct kdt_forest kdt_forest;

/* Text of the last failure on the calling thread ("" if none). */
const char *kdt_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices).  Kernels inside the CUDA graph that kdt_knn_batched
 * replays are counted when the graph is captured, not at each replay. */
int64_t kdt_launch_count(void);

/* ---- single tree ------------------------------------------------------- */

/* Build the left-balanced complete tree of N points of dimension D in level
 * order (Sec. 3: node n has children 2n+1 and 2n+2).  Split dimension of a
 * node on level l is l mod D; the point stored at a node is the element of
 * rank L(n) (the complete tree's left-subtree size) of its subtree's points in
 * (coordinate, input index) order, so the tree is the one any serial median
 * builder produces (Sec. 4).
 *   d_points: float32 [N][D], read only during the call's stream work.
 *   N in [1, 2^30), D in [1, 8].
 *   *out receives a library-owned tree; release it with kdt_free.
 * Synchronises `stream` once to report KDT_ENONFINITE. */
int kdt_build(const float *d_points, int64_t N, int D, void *stream, kdt_tree **out);

/* As kdt_build; opts = 0 or a combination of KDT_BUILD_ASYNC (no
 * synchronisation) and KDT_BUILD_WIDEST (stored split dimensions, D <= 3;
 * KDT_EINVAL for D > 3). */
int kdt_build_ex(const float *d_points, int64_t N, int D, int opts, void *stream, kdt_tree **out);

/* Rebuild `tree` in place from new points with the same N and D, reusing its
 * device memory (a trained radius model is kept; a payload set with
 * kdt_tree_set_payload is dropped, as it follows the old node order).  The
 * split-dimension rule is the tree's own (KDT_BUILD_WIDEST in opts is
 * ignored); opts as for kdt_build_ex otherwise. */
int kdt_rebuild(kdt_tree *tree, const float *d_points, int opts, void *stream);

/* Split dimension of every level-order node: d_dims uint8 [N] (level mod D, or
 * the stored dimension of a KDT_BUILD_WIDEST tree). */
int kdt_tree_split_dims(const kdt_tree *tree, uint8_t *d_dims, void *stream);

/* N and D of a tree (host values, no synchronisation). */
int kdt_tree_info(const kdt_tree *tree, int64_t *N, int *D);

/* Copy the level-order tree: d_coords float32 [N][D] (coordinates of the
 * point at each node) and d_ids int32 [N] (its input index). */
int kdt_tree_export(const kdt_tree *tree, float *d_coords, int32_t *d_ids, void *stream);

/* Save a tree as its level-order arrays (coordinates, input indices, bounding
 * box) with a header and a checksum; load it back as a new tree without
 * rebuilding (synchronous; KDT_EIO for a missing, foreign or damaged file).
 * A radius model is not part of the tree file (kdt_radius_model_save). */
int kdt_tree_save(const kdt_tree *tree, const char *path);
int kdt_tree_load(const char *path, void *stream, kdt_tree **out);

/* Find-closest-point (Sec. 4, fcp): kNN with k = 1.
 *   d_queries float32 [Q][D]; d_ids int32 [Q]; d_d2 float32 [Q]. */
int kdt_fcp(const kdt_tree *tree, const float *d_queries, int64_t Q, float max_radius,
            int flags, int32_t *d_ids, float *d_d2, void *stream);

/* k nearest neighbours within max_radius (inclusive; +inf = unbounded) with a
 * shrinking cull radius (Sec. 3).  k in [1, 64].
 *   d_queries float32 [Q][D]; d_ids int32 [Q][k]; d_d2 float32 [Q][k].
 * Q = 0 is a no-op. */
int kdt_knn(const kdt_tree *tree, const float *d_queries, int64_t Q, int k, float max_radius,
            int flags, int32_t *d_ids, float *d_d2, void *stream);

/* Per-query count of processed nodes (first visits, the processNode calls of
 * Sec. 3.2) of the traversal kdt_knn would run with the same arguments.  With
 * KDT_LEARNED: nodes of the bounded pass plus, for re-run queries, of the
 * re-run (results are not written).  d_visits int32 [Q]. */
int kdt_knn_visits(const kdt_tree *tree, const float *d_queries, int64_t Q, int k,
                   float max_radius, int flags, int32_t *d_visits, void *stream);

/* ---- range queries ---------------------------------------------------------
 * Every point within a radius of a query point (ball, inclusive, the same FP32
 * squared distance as kdt_knn: d2 <= fl(radius * radius)) or inside an
 * axis-aligned box (inclusive bounds; lo > hi in any dimension gives none),
 * found with the unordered stack-free traversal and a fixed range (Sec. 3:
 * other query primitives change only the range test and processNode).
 * Queries float [Q][D] (ball centres, box lower / upper corners), device.
 * Two passes: *_count writes d_counts int32 [Q]; kdt_offsets turns counts into
 * d_offsets int64 [Q+1] (exclusive prefix sums, offsets[Q] = total); *_fill
 * writes query q's point ids (and, for balls, squared distances if d_d2 is not
 * NULL) to [offsets[q], offsets[q+1]) in traversal order, the same on every
 * call.  flags: 0 or KDT_MORTON (queries run in Morton order; results are the
 * same), plus KDT_RANGE_VISITS for the count calls; any other bit is
 * KDT_EINVAL.  A fill whose hits do not match its
 * offsets writes nothing outside the query's slice and is reported by
 * kdt_status.  Buffers are the caller's; nothing is kept after the call. */
int kdt_radius_count(const kdt_tree *tree, const float *d_queries, int64_t Q, float radius, int flags,
                     int32_t *d_counts, void *stream);
int kdt_radius_fill(const kdt_tree *tree, const float *d_queries, int64_t Q, float radius, int flags,
                    const int64_t *d_offsets, int32_t *d_ids, float *d_d2, void *stream);
int kdt_box_count(const kdt_tree *tree, const float *d_lo, const float *d_hi, int64_t Q, int flags,
                  int32_t *d_counts, void *stream);
int kdt_box_fill(const kdt_tree *tree, const float *d_lo, const float *d_hi, int64_t Q, int flags,
                 const int64_t *d_offsets, int32_t *d_ids, void *stream);
/* flags bit for kdt_radius_count / kdt_box_count only: write each query's
 * number of processed nodes (first visits of the traversal) instead of its
 * number of hits (the per-query work, for measurement). */
#define KDT_RANGE_VISITS 0x200

/* Exclusive prefix sum of counts into d_offsets int64 [Q+1]; if h_total is not
 * NULL the stream is synchronised and *h_total receives offsets[Q]. */
int kdt_offsets(const int32_t *d_counts, int64_t Q, int64_t *d_offsets, int64_t *h_total, void *stream);

/* ---- payloads and reductions ------------------------------------------------
 * Sec. 3: the point type may carry payload data (its example: surface normal
 * and photon power for photon mapping, the application Sec. 1 cites).  A
 * payload is C floats per point (1 <= C <= KDT_PAYLOAD_MAX_C), given in input
 * order float [N][C]; the tree keeps its own copy in node order (N*C*4 + N*4
 * bytes, freed with the tree, dropped by kdt_rebuild).  Synchronises `stream`.
 * Reductions sum a payload over each query's hits, in FP32, one addition at a
 * time, in a fixed order, and write d_out float [Q][C]:
 *   KDT_REDUCE_SUM      the sum;
 *   KDT_REDUCE_MEAN     the sum / the number of hits;
 *   KDT_REDUCE_DENSITY  the sum / fl(pi * R2), the photon-map density estimate
 *                       (R2: kdt_radius_reduce fl(radius^2), the gather disc;
 *                       kdt_knn_reduce the largest d2 found, the disc through
 *                       the farthest neighbour);
 * a query with no hit gets 0 in every mode.  kdt_radius_reduce sums over the
 * ball's hits in traversal order (d_counts int32 [Q] may be NULL; flags as for
 * the range queries); kdt_knn_reduce over the kNN result in ascending (d2, id)
 * order (k, max_radius and flags as kdt_knn). */
#define KDT_PAYLOAD_MAX_C 8
#define KDT_REDUCE_SUM 0
#define KDT_REDUCE_MEAN 1
#define KDT_REDUCE_DENSITY 2
int kdt_tree_set_payload(kdt_tree *tree, const float *d_payload, int C, void *stream);
int kdt_radius_reduce(const kdt_tree *tree, const float *d_queries, int64_t Q, float radius, int flags, int mode,
                      float *d_out, int32_t *d_counts, void *stream);
int kdt_knn_reduce(const kdt_tree *tree, const float *d_queries, int64_t Q, int k, float max_radius, int flags,
                   int mode, float *d_out, void *stream);

/* Synchronise `stream` and report device-side failures recorded on the tree
 * since the last call: KDT_ENONFINITE (asynchronous build), KDT_ETRAVERSAL, or
 * KDT_EINVAL (a range fill whose offsets did not match its hits).  Clears the
 * recorded state. */
int kdt_status(kdt_tree *tree, void *stream);

/* Release a tree and its device memory (synchronises the device first). */
void kdt_free(kdt_tree *tree);

/* One call from host memory to host memory: copies h_points to the device,
 * builds the tree, runs kdt_knn on h_queries and writes the results into
 * h_ids int32 [Q][k] and h_d2 float32 [Q][k], and frees everything.
 * Synchronous.  Page-locked (pinned or registered) query and result buffers
 * are used in place: the query kernels read the queries and store the results
 * through the host link themselves, with no staging copy; other host buffers
 * are copied to and from device scratch. */
int kdt_knn_host(const float *h_points, int64_t N, int D, const float *h_queries, int64_t Q,
                 int k, float max_radius, int flags, int32_t *h_ids, float *h_d2);

/* kdt_knn without any device allocation.  The paper has no counterpart: this
 * serves callers that must not enter the CUDA allocator while they query
 * (an application whose own pool owns all device memory, a real-time loop
 * that cannot afford the synchronisation of cudaMalloc / cudaFree, a plugin
 * host that forbids library allocations).  Scratch lives in one fixed device
 * array inside the library (about 4.3 MB per GPU that loads it, held until the
 * process exits), so Q is limited to KDT_STATIC_MAX_Q per call; larger Q gives
 * KDT_EINVAL.  KDT_LEARNED is not accepted.  Same arguments, results and
 * flags as kdt_knn otherwise.
 * Every call looks up the array's device address in the current device's
 * context (cudaGetSymbolAddress, which allocates nothing); on a device whose
 * module is not loaded yet, make the first call before any stream capture.
 * Every call reuses the same array: calls whose GPU work overlaps (other
 * streams, other host threads) race and must be serialised.  The work counter
 * is cleared by each call; the rest is overwritten before it is read.
 * kdt_profile_enable / kdt_profile_read do not time these calls. */
#define KDT_STATIC_MAX_Q (1 << 18)
int kdt_knn_static(const kdt_tree *tree, const float *d_queries, int64_t Q, int k, float max_radius,
                   int flags, int32_t *d_ids, float *d_d2, void *stream);

/* ---- learned radius proposal (not in the paper) ------------------------- */

/* Which queries of a KDT_LEARNED call take the proposed radius (no paper
 * counterpart; results are the same for every choice).  A proposal saves
 * work only where the plain traversal wastes it: queries far from the data
 * process many nodes, and a tight initial radius removes some of them, while
 * queries inside the data find their neighbours at once and only pay for the
 * features and the network. */
#define KDT_GATE_AUTO 0 /* training option: choose among the forms below from the training queries (see
                           kdt_train_opts.gate) */
#define KDT_GATE_ALL  1 /* every query */
#define KDT_GATE_FAR  2 /* queries whose greedy descent ends more than 8 mean point spacings from its leaf point
                           (the far cost classes of KDT_COST_ORDER, which the call then uses); the others run the
                           plain traversal */
#define KDT_GATE_NONE 3 /* no query: the call runs the plain traversal */

typedef struct kdt_train_opts {
    int epochs;           /* passes over the training queries (default 6 if <= 0) */
    int batch;            /* minibatch size (default 1024 if <= 0; rounded down to a multiple of 64) */
    float lr;             /* Adam step size (default 2e-3 if <= 0) */
    uint64_t seed;        /* weight initialisation seed */
    float margin;         /* cull radius = margin * predicted radius; if <= 0 the margin is
                             calibrated after training so that a fraction fallback_target of
                             the training queries would fall back */
    float fallback_target;/* see margin (default 0.02 if <= 0) */
    int uniform_weights;  /* 0 (default): weight each training query by the work the plain
                             traversal spends on it (processed nodes plus a floor of a tenth of
                             the mean), by resampling the training set with those
                             probabilities; the margin's fallback target is then a share of
                             that work.  1: every query weighs the same */
    int gate;             /* KDT_GATE_* (default KDT_GATE_AUTO: on up to 2^20 of the training
                             queries, with query_flags, the processed nodes of the plain traversal
                             and of the learned forms (all queries gated, the far ones) are counted,
                             and the network pass's cost per gated query is measured in
                             processed-node equivalents (its time per query over the plain
                             traversal's time per processed node); a gated call's nodes are
                             charged 1.08 plain nodes each (the bounded pass's measured
                             per-node overhead, rounded up); the form that saves the most
                             nodes net of these costs is kept, KDT_GATE_NONE when none saves
                             any) */
    int query_flags;      /* flags of the queries the automatic gate is judged with (default
                             KDT_MORTON | KDT_COST_ORDER) */
} kdt_train_opts;

/* Width of the two hidden layers of the radius model. */
#define KDT_MLP_HIDDEN 64
/* Number of float parameters: W1[64][4] b1[64] W2[64][64] b2[64] w3[64] b3. */
#define KDT_MLP_PARAMS (64 * 4 + 64 + 64 * 64 + 64 + 64 + 1)

/* Train the radius model of `tree` on Qt training queries for k neighbours:
 * labels are 0.5*log(d2 of the exact k-th neighbour) from kdt_knn; features
 * are the query coordinates and log(max(d2 to the greedy-descent leaf, 1e-30))
 * (the leaf is where repeated close-child steps from the root end), normalised
 * by their training mean and standard deviation; the MLP 4 -> 64 -> 64 -> 1
 * (ReLU) runs with BF16-rounded weights and FP32 accumulation and is fitted by
 * Adam (step size decaying along a half cosine) on the mean squared error over
 * the (by default cost-weighted) training sample, entirely by the library's
 * kernels.
 * Synchronous.  *final_loss (may be NULL) receives the last epoch's mean loss. */
int kdt_radius_model_train(kdt_tree *tree, const float *d_train_queries, int64_t Qt, int k,
                           const kdt_train_opts *opts, float *final_loss, void *stream);

/* Copy the model out of / into the tree (host buffers).
 *   h_params float32 [KDT_MLP_PARAMS] (FP32 master weights), h_norm float32 [8]
 *   (feature mean[4], std[4]), *margin. */
int kdt_radius_model_get(const kdt_tree *tree, float *h_params, float *h_norm, float *margin);
int kdt_radius_model_set(kdt_tree *tree, const float *h_params, const float *h_norm, float margin);

/* The gate of the tree's radius model (KDT_GATE_ALL / FAR / NONE), and a way
 * to set it after training or loading. */
int kdt_radius_model_gate(const kdt_tree *tree, int *gate);
int kdt_radius_model_set_gate(kdt_tree *tree, int gate);

/* Save / load the model as a small versioned binary file (the gate included;
 * files of the first version load with KDT_GATE_ALL). */
int kdt_radius_model_save(const kdt_tree *tree, const char *path);
int kdt_radius_model_load(kdt_tree *tree, const char *path);

/* Per-query features: d_feat float32 [Q][4] = (q_0, q_1, q_2, log(max(d2_leaf, 1e-30)))
 * before normalisation (3-D trees only). */
int kdt_descent_features(const kdt_tree *tree, const float *d_queries, int64_t Q,
                         float *d_feat, void *stream);

/* Model forward on normalised features: d_x float32 [n][4] -> d_y float32 [n],
 * the inference path of the learned query: h_params (FP32) with weights
 * rounded to BF16; layer 1 in FP32, hidden activations rounded to BF16, the
 * 64 x 64 layer on the tensor cores (tcgen05.mma, FP32 accumulation), output
 * layer in FP32.  Synchronous. */
int kdt_mlp_forward(const float *h_params, const float *d_x, int64_t n, float *d_y, void *stream);

/* Mean squared error of the model on (d_x, d_label) and its gradient with
 * respect to the BF16-rounded parameters: h_grad float32 [KDT_MLP_PARAMS].
 * The training path: the three 64 x 64 contractions of the step (hidden
 * layer forward, back-propagation through it, its weight gradient) run on the
 * tensor cores (tcgen05.mma) with BF16 operands (weights, hidden activations,
 * back-propagated gradients) and FP32 accumulation; the rest in FP32, sums in
 * a fixed order.  Synchronous. */
int kdt_mlp_loss_grad(const float *h_params, const float *d_x, const float *d_label, int64_t n,
                      float *h_loss, float *h_grad, void *stream);

/* Learned-path statistics of the last KDT_LEARNED query on this tree:
 * number of queries re-run with the caller's radius, and the mean of
 * (proposed radius / true k-th neighbour radius) over the gated queries that
 * did not fall back.  Synchronises `stream`. */
int kdt_learned_stats(const kdt_tree *tree, int64_t *fallbacks, double *radius_ratio, void *stream);

/* Number of queries of the last KDT_LEARNED call on this tree that took the
 * proposed radius (all of them, the far ones or none, by the model's gate).
 * Synchronises `stream`. */
int kdt_learned_gated(const kdt_tree *tree, int64_t *gated, void *stream);

/* ---- batched: many independent trees ------------------------------------ */

/* Build T trees at once.  Cloud i is d_points rows [h_offsets[i], h_offsets[i+1])
 * (h_offsets int64 [T+1], h_offsets[0] = 0, non-decreasing; empty clouds are
 * allowed).  Each tree is exactly the tree kdt_build makes of its cloud. */
int kdt_build_batched(const float *d_points, const int64_t *h_offsets, int T, int D,
                      void *stream, kdt_forest **out);

/* kNN of each query set against its own tree: queries of tree i are rows
 * [h_qoffsets[i], h_qoffsets[i+1]) of d_queries; result rows follow the query
 * rows; ids are indices within cloud i.  One persistent launch serves all
 * trees (captured once into a CUDA graph and replayed while the arguments are
 * unchanged).  With KDT_PER_TREE the same kernel is launched once per tree
 * instead (for comparison). */
#define KDT_PER_TREE 0x10
int kdt_knn_batched(kdt_forest *forest, const float *d_queries, const int64_t *h_qoffsets,
                    int k, float max_radius, int flags, int32_t *d_ids, float *d_d2, void *stream);

/* Level-order arrays of all trees, concatenated in cloud order:
 * d_coords float32 [sum N_i][D], d_ids int32 [sum N_i] (ids within the cloud). */
int kdt_forest_export(const kdt_forest *forest, float *d_coords, int32_t *d_ids, void *stream);

/* Launch parameters of the batched query: threads per block (0 = 128, else a
 * multiple of 32 up to 128), traversal steps between two claim rounds of a
 * warp (0 = the default for k, 32 for k = 1 and 64 otherwise; up to 256), the
 * inline depth (0 = default 2, or 1; see kdt_set_inline_depth) and the light
 * run (0 = default 1, up to 64; see kdt_set_light_run).
 * Shared-memory staging does not apply to forests: the lanes of a warp walk
 * different trees.  The next kdt_knn_batched re-captures its graph. */
int kdt_forest_set_launch(kdt_forest *forest, int threads, int claim_steps, int inline_depth, int light_run);

/* Processed nodes (first visits) of every query of a kdt_knn_batched call
 * (same arguments; KDT_UNORDERED respected, the other flags do not change
 * the counts): d_visits int32 [total queries], 0 for queries of an empty
 * cloud.  Counts the traversal of Sec. 3.2 as kdt_knn_visits does for one
 * tree (the roofline's V_q of the batched form); one launch per tree. */
int kdt_knn_batched_visits(kdt_forest *forest, const float *d_queries, const int64_t *h_query_offsets, int k,
                           float max_radius, int flags, int32_t *d_visits, void *stream);

/* Time the batched query (kdt_knn_batched with these arguments, graph
 * included; it writes d_ids / d_d2 like that call) for inline depths {2, 1},
 * light runs {1, 4, 8}, block sizes {128, 64}, then claim steps {16, 32, 64,
 * 128}, one warm-up and
 * one timed run each, and keep the fastest on the forest (a candidate must win
 * by 2 %).  Synchronous.  The out pointers may be NULL. */
int kdt_forest_autotune(kdt_forest *forest, const float *d_queries, const int64_t *h_query_offsets, int k,
                        float max_radius, int flags, int32_t *d_ids, float *d_d2, int *best_threads,
                        int *best_claim, int *best_inline, int *best_light, float *best_ms, void *stream);

/* Release a forest and its device memory (synchronises the device first). */
void kdt_forest_free(kdt_forest *forest);

/* ---- launch tuning -------------------------------------------------------- */

/* The traversal kernels copy the top `levels` levels of the tree (2^levels - 1
 * nodes) into shared memory once per block.  Staging trades L1 capacity (the
 * same on-chip array) for the latency of the top-level loads; the best depth
 * depends on the tree and the queries.  -1 restores the automatic choice (the
 * tuned value for this tree's shape if kdt_autotune or kdt_tuning_load set
 * one, else 0: no staging).  levels in [-1, 16]. */
int kdt_set_stage_levels(kdt_tree *tree, int levels);

/* Traversal steps a lane takes between two claim rounds of its warp (a lane
 * whose query ends waits for the round to take its next one): large values
 * amortise the claim vote for long queries, small ones idle less behind short
 * queries.  -1 restores the tuned or default value (32 for k = 1, 64
 * otherwise).  Range 1..256. */
int kdt_set_claim_steps(kdt_tree *tree, int steps);

/* Depth of the bottom subtrees one traversal step processes whole, with their
 * loads issued together: 2 (default) saves steps on long queries; 3 also
 * takes the node above two such subtrees into the same step (the second
 * subtree's loads issued when the traversal enters it), saving the steps
 * between them; 1 avoids loads that short queries rarely use; 0 selects the
 * simplest kernel (one node per step; ordered kNN with k <= 16 and D <= 4
 * without staging, else depth 1 is used); -1 restores the tuned or default
 * value.  Staged launches use depth 2.  Results and processed nodes are the
 * same for every depth. */
int kdt_set_inline_depth(kdt_tree *tree, int depth);

/* Traversal steps a lane may take in one call while they are light (a heavy
 * step enters a node whose bottom subtree is processed whole): with values
 * above 1 the heavy steps of a warp's lanes tend to start their calls
 * together.  1 (default) suits long queries; 4 or 8 pay for short ones.  -1
 * restores the tuned or default value.  Range 1..64.  Results and processed
 * nodes are the same for every value. */
int kdt_set_light_run(kdt_tree *tree, int steps);

/* Where the k-best lists of queries with k > 16 live (no paper counterpart; a
 * placement choice of the GPU kernel, results and processed nodes are the same
 * for every choice).  KDT_LIST_SHARED: a per-thread binary max-heap in shared
 * memory (k x 8 bytes per thread, which limits the resident blocks and takes
 * the on-chip array that L1 shares).  KDT_LIST_GLOBAL: the same heap in a
 * per-thread slice of a scratch buffer in device memory (about
 * SMs x 1024 x k x 8 bytes per call, allocated with the call's scratch),
 * cached in L1 / L2 beside the tree.  -1 restores the default. */
#define KDT_LIST_SHARED 0
#define KDT_LIST_GLOBAL 1
/* KDT_LIST_GROUP4 / 8: a sorted list spread over a group of 4 (8) lanes that
 * walk the query together, k / 4 (k / 8) keys in each lane's registers,
 * insertion by warp shuffles (ordered and unordered kNN and visit counts;
 * other calls use the shared-memory heap). */
#define KDT_LIST_GROUP4 2
#define KDT_LIST_GROUP8 3
int kdt_set_large_k_list(kdt_tree *tree, int placement);
/* The placement kdt_knn uses for this tree and k: set on the tree, else tuned
 * for its shape (for k > 16 kdt_autotune takes the global heap when its query
 * sample processes at least 1024 nodes per query, the shared-memory heap
 * otherwise), else KDT_LIST_SHARED. */
int kdt_large_k_list(const kdt_tree *tree, int k, int *placement);

/* The launch parameters kdt_knn uses for this tree and k: set on the tree,
 * else tuned for its shape (kdt_autotune / kdt_tuning_load), else defaults
 * (no staging, 32 claim steps for k = 1 and 64 otherwise, inline depth 2,
 * light run 1).  Any out pointer may be NULL. */
int kdt_tuned_params(const kdt_tree *tree, int k, int *stage_levels, int *claim_steps, int *inline_depth,
                     int *light_run);

/* Time the plain traversal of up to 2^20 of the given queries and remember
 * the fastest launch parameters for this tree's shape (GPU name, D, k bucket,
 * floor(log2 N)): a coordinate search over the inline depth {2, 1, 0}, the
 * light run {1, 4, 8}, then the claim steps {16, 32, 64, 128}, then the
 * staging depth {0, 4, 6, 8}, each
 * candidate timed over two launches after a warm-up and taken only when it is
 * faster than the best so far by 2 % (staging: 5 %).  Later queries on trees of that shape use the choice unless
 * the kdt_set_* calls override.  Synchronous.  *best_levels and *best_ms (may
 * be NULL) receive the staging depth and the best time per launch;
 * kdt_tuned_params reports all three. */
int kdt_autotune(kdt_tree *tree, const float *d_queries, int64_t Q, int k, int flags, int *best_levels,
                 float *best_ms, void *stream);

/* Write / read the remembered tuning choices as a small JSON file. */
int kdt_tuning_save(const char *path);
int kdt_tuning_load(const char *path);

/* ---- failure injection (tests) ------------------------------------------
 * Host-side hooks that make the library's error paths reachable without a
 * device fault.  kdt_debug_fail_allocs(n): the next n device allocations the
 * library makes (tree arrays, per-call scratch) fail with KDT_ENOMEM; 0
 * clears.  kdt_debug_set_step_cap(tree, cap): traversals of kdt_knn /
 * kdt_fcp / kdt_knn_visits on this tree stop after about cap steps (the bound
 * is checked once per claim round) and report KDT_ETRAVERSAL through
 * kdt_status, as a traversal exceeding the 3N + 3 bound would; 0 restores
 * the bound.  No paper counterpart. */
int kdt_debug_fail_allocs(int n);
int kdt_debug_set_step_cap(kdt_tree *tree, uint32_t cap);

/* ---- profiling ----------------------------------------------------------- */

/* Accumulate device time of the traversal kernels launched by kdt_knn /
 * kdt_fcp on `tree` (CUDA events recorded on the launching stream around each
 * traversal launch) while enabled. */
int kdt_profile_enable(kdt_tree *tree, int enable);
/* Synchronise, then return the accumulated milliseconds and launch count of the
 * traversal kernels since profiling was enabled, and reset them. */
int kdt_profile_read(kdt_tree *tree, double *ms, int64_t *launches);

/* L2 read bandwidth of the current GPU in GB/s, measured by the library's own
 * kernel (no paper counterpart): a device buffer of `bytes` (1 MiB to 1 GiB;
 * small enough to stay in L2 for the figure to mean L2) is read once, then
 * `reps` times with 16-byte loads that bypass L1, by 8 blocks of 256 threads
 * per SM; *gbs = bytes x reps over the fastest of three timed launches.  The
 * buffer is allocated and freed on `stream`.  Synchronous.  This is the
 * denominator of the L2 fractions the benchmark reports. */
int kdt_l2_read_bandwidth(int64_t bytes, int reps, double *gbs, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KDT_H */
