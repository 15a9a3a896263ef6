/*
 * CPU oracle for the left-balanced k-d tree queries of Wald, "A Stack-Free
 * Traversal Algorithm for Left-Balanced k-d Trees" (arXiv 2210.12859).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * library and is deliberately plain and slow.
 *
 * Compile with -O2 -ffp-contract=off and without fast-math, so that every
 * float expression below is evaluated as written: one IEEE-754 binary32
 * operation at a time, round-to-nearest-even, no fused multiply-add, no
 * flush-to-zero.
 *
 * Contents, each citing the part of the paper it follows:
 *   orc_left_size       subtree size of a complete tree (Sec. 3, level-order
 *                       assumption; needed by the builder of Sec. 4)
 *   orc_build           recursive median builder (Sec. 4: the tree any serial
 *                       builder produces), round-robin split dimension
 *   orc_build_widest    the same with a stored per-node split dimension (the
 *                       other splitDimOf variant Sec. 3 names): widest extent
 *   orc_build_par       either builder with the two subtrees of the top few
 *                       nodes built in separate threads (the same recursion)
 *   orc_knn_brute       plain definition of the fcp / kNN result (exact method,
 *                       Sec. 3 "shrinking max radius"), FP32 distances
 *   orc_knn_brute_f64   the same selection with distances in FP64
 *   orc_knn_recursive   the recursive ordered / unordered traversal (Sec. 3.1)
 *   orc_knn_stackfree   the (curr, prev) state machine (Sec. 3.2)
 *   orc_radius_brute    every point within a radius / inside a box (the plain
 *   orc_box_brute       definition of the range queries Sec. 3 mentions)
 *   orc_range_stackfree the same queries through the unordered stack-free
 *                       machine with a fixed range (Sec. 3: other primitives
 *                       change only the range test and processNode), hits in
 *                       traversal order; orc_range_visits its processed nodes
 *   orc_range_reduce    per-query reductions of a per-point payload over those
 *   orc_knn_reduce      hits / over a kNN result (Sec. 3: point types with
 *                       payload such as photon power; the photon-map density
 *                       estimate of the photon-mapping application it cites)
 *   orc_descent_leaf    greedy close-child descent (feature of the learned
 *                       radius proposal; not in the paper)
 *   orc_mlp_*           FP64 forward / backward of the radius MLP (not in the
 *                       paper), and both with a bound on the error of a
 *                       BF16-in / FP32-accumulate evaluation (per sample for
 *                       the forward, per parameter for the gradient): parity
 *                       targets for the tensor-core inference and training
 *                       kernels
 *
 * Parity status: every function above is pinned by tests under tests/ against
 * values fixed by the paper (the six-point example of Figure 1), closed forms,
 * brute force on tiny inputs, library routines and invariants; a mutation
 * test compiles copies of this file with one planted mistake each and checks
 * that those pins reject every copy.
 */
#define _GNU_SOURCE 1 /* qsort_r */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Tree topology (Sec. 3: level order, lChild = 2n+1, rChild = 2n+2).       */
/* ------------------------------------------------------------------------ */

static int orc_level(int64_t node)
{
    /* level(n) = floor(log2(n + 1)) */
    int l = 0;
    int64_t v = node + 1;
    while (v > 1) {
        v >>= 1;
        ++l;
    }
    return l;
}

/* Size of the left subtree of the root of a complete binary tree of n nodes
 * whose last level is filled from the left.  h = floor(log2 n) is the depth of
 * the last level; the levels above it hold 2^h - 1 nodes; `last` nodes sit on
 * the last level, and the left subtree receives up to 2^(h-1) of them. */
int64_t orc_left_size(int64_t n)
{
    if (n <= 1)
        return 0;
    int h = 0;
    while (((int64_t)1 << (h + 1)) <= n)
        ++h;
    int64_t half = (int64_t)1 << (h - 1);
    int64_t last = n - (((int64_t)1 << h) - 1);
    return (half - 1) + (last < half ? last : half);
}

/* ------------------------------------------------------------------------ */
/* Builder (Sec. 4 cites a parallel builder and states that it emits the same */
/* tree as any serial builder; this is that serial builder).                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    const float *pts;
    int D;
    int dim;
} orc_sort_ctx;

/* order by (coordinate in `dim`, input index); float `<`, so -0 == +0 */
static int orc_cmp_coord_idx(const void *a, const void *b, void *vctx)
{
    const orc_sort_ctx *c = (const orc_sort_ctx *)vctx;
    int32_t ia = *(const int32_t *)a;
    int32_t ib = *(const int32_t *)b;
    float ca = c->pts[(int64_t)ia * c->D + c->dim];
    float cb = c->pts[(int64_t)ib * c->D + c->dim];
    if (ca < cb)
        return -1;
    if (cb < ca)
        return 1;
    return (ia > ib) - (ia < ib);
}

/* dimension of widest extent (max - min, rounded to float) of the points S,
 * ties to the lowest dimension index */
static int orc_widest_dim(const float *pts, int D, const int32_t *S, int64_t n)
{
    int best = 0;
    float best_ext = -1.0f;
    for (int e = 0; e < D; ++e) {
        float lo = pts[(int64_t)S[0] * D + e], hi = lo;
        for (int64_t i = 1; i < n; ++i) {
            float v = pts[(int64_t)S[i] * D + e];
            if (v < lo)
                lo = v;
            if (v > hi)
                hi = v;
        }
        float ext = hi - lo;
        if (ext > best_ext) {
            best_ext = ext;
            best = e;
        }
    }
    return best;
}

/* node_dim NULL: split dimension level mod D; else the widest dimension of the
 * node's points, recorded in node_dim[node] */
static int orc_build_rec(const float *pts, int64_t N, int D, int32_t *S,
                         int64_t n, int64_t node, int32_t *node_pid, uint8_t *node_dim)
{
    if (n == 0)
        return 0;
    if (node >= N)
        return -1; /* subtree sizes disagree with the complete tree */
    int dim = node_dim ? orc_widest_dim(pts, D, S, n) : orc_level(node) % D;
    if (node_dim)
        node_dim[node] = (uint8_t)dim;
    orc_sort_ctx ctx = {pts, D, dim};
    qsort_r(S, (size_t)n, sizeof(int32_t), orc_cmp_coord_idx, &ctx);
    int64_t L = orc_left_size(n);
    node_pid[node] = S[L];
    if (orc_build_rec(pts, N, D, S, L, 2 * node + 1, node_pid, node_dim))
        return -1;
    return orc_build_rec(pts, N, D, S + L + 1, n - L - 1, 2 * node + 2, node_pid, node_dim);
}

/* The same recursion, with the left subtree of each node in the top `spawn`
 * levels built by a new thread while the calling thread builds the right one.
 * The subtrees write disjoint parts of S and of the output arrays. */
typedef struct {
    const float *pts;
    int64_t N;
    int D;
    int32_t *S;
    int64_t n;
    int64_t node;
    int32_t *node_pid;
    uint8_t *node_dim;
    int spawn;
    int rc;
} orc_build_task;

static void *orc_build_task_run(void *arg)
{
    orc_build_task *t = (orc_build_task *)arg;
    if (t->spawn <= 0 || t->n < 4096) {
        t->rc = orc_build_rec(t->pts, t->N, t->D, t->S, t->n, t->node, t->node_pid, t->node_dim);
        return NULL;
    }
    t->rc = 0;
    if (t->n == 0)
        return NULL;
    if (t->node >= t->N) {
        t->rc = -1;
        return NULL;
    }
    int dim = t->node_dim ? orc_widest_dim(t->pts, t->D, t->S, t->n) : orc_level(t->node) % t->D;
    if (t->node_dim)
        t->node_dim[t->node] = (uint8_t)dim;
    orc_sort_ctx ctx = {t->pts, t->D, dim};
    qsort_r(t->S, (size_t)t->n, sizeof(int32_t), orc_cmp_coord_idx, &ctx);
    int64_t L = orc_left_size(t->n);
    t->node_pid[t->node] = t->S[L];
    orc_build_task left = {t->pts, t->N, t->D, t->S, L, 2 * t->node + 1, t->node_pid, t->node_dim, t->spawn - 1, 0};
    orc_build_task right = {t->pts, t->N, t->D, t->S + L + 1, t->n - L - 1, 2 * t->node + 2, t->node_pid,
                            t->node_dim, t->spawn - 1, 0};
    pthread_t th;
    int spawned = pthread_create(&th, NULL, orc_build_task_run, &left) == 0;
    if (!spawned)
        orc_build_task_run(&left);
    orc_build_task_run(&right);
    if (spawned)
        pthread_join(th, NULL);
    t->rc = (left.rc || right.rc) ? -1 : 0;
    return NULL;
}

static int orc_build_any(const float *pts, int64_t N, int D, int32_t *node_pid, uint8_t *node_dim, int threads)
{
    if (N < 1 || D < 1 || D > 8)
        return -1;
    for (int64_t i = 0; i < N * D; ++i)
        if (!isfinite(pts[i]))
            return -1;
    int32_t *S = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!S)
        return -1;
    for (int64_t i = 0; i < N; ++i)
        S[i] = (int32_t)i;
    int rc;
    if (threads > 1) {
        int spawn = 0;
        while ((1 << spawn) < threads && spawn < 12)
            ++spawn;
        orc_build_task root = {pts, N, D, S, N, 0, node_pid, node_dim, spawn, 0};
        orc_build_task_run(&root);
        rc = root.rc;
    } else {
        rc = orc_build_rec(pts, N, D, S, N, 0, node_pid, node_dim);
    }
    free(S);
    return rc;
}

/* node_pid[t] = input index of the point stored at level-order node t, split
 * dimension level mod D.  Returns 0 on success, -1 on bad arguments or a
 * non-finite coordinate. */
int orc_build(const float *pts, int64_t N, int D, int32_t *node_pid)
{
    return orc_build_any(pts, N, D, node_pid, NULL, 1);
}

/* The same builder with the split dimension of every node stored in the node
 * (Sec. 3 leaves splitDimOf open: stored per node or fixed by level): the
 * dimension of widest extent of the node's points, ties to the lowest index;
 * node_dim[t] receives it. */
int orc_build_widest(const float *pts, int64_t N, int D, int32_t *node_pid, uint8_t *node_dim)
{
    return orc_build_any(pts, N, D, node_pid, node_dim, 1);
}

/* orc_build (node_dim NULL) or orc_build_widest with up to about `threads`
 * threads building subtrees in parallel: the same tree. */
int orc_build_par(const float *pts, int64_t N, int D, int32_t *node_pid, uint8_t *node_dim, int threads)
{
    return orc_build_any(pts, N, D, node_pid, node_dim, threads);
}

/* ------------------------------------------------------------------------ */
/* Distances and the k-best list.                                           */
/* ------------------------------------------------------------------------ */

/* d2(p, q) = ((t_0 + t_1) + t_2) + ..., t_j = fl(fl(p_j - q_j)^2), FP32 */
static float orc_d2(const float *p, const float *q, int D)
{
    float diff = p[0] - q[0];
    float s = diff * diff;
    for (int j = 1; j < D; ++j) {
        float dj = p[j] - q[j];
        float tj = dj * dj;
        s = s + tj;
    }
    return s;
}

/* (da, ia) < (db, ib) lexicographically */
static int orc_pair_less(float da, int32_t ia, float db, int32_t ib)
{
    if (da < db)
        return 1;
    if (db < da)
        return 0;
    return ia < ib;
}

typedef struct {
    int k;
    int count;
    float r2;
    float *d2;
    int32_t *id;
} orc_list;

/* processNode of fcp / kNN: accept iff d2 <= r2 and the list has room or the
 * pair beats the current worst; keep the list sorted ascending by (d2, id). */
static void orc_list_offer(orc_list *L, float d2, int32_t id)
{
    if (!(d2 <= L->r2))
        return;
    if (L->count == L->k && !orc_pair_less(d2, id, L->d2[L->k - 1], L->id[L->k - 1]))
        return;
    int pos = L->count < L->k ? L->count : L->k - 1;
    while (pos > 0 && orc_pair_less(d2, id, L->d2[pos - 1], L->id[pos - 1])) {
        L->d2[pos] = L->d2[pos - 1];
        L->id[pos] = L->id[pos - 1];
        --pos;
    }
    L->d2[pos] = d2;
    L->id[pos] = id;
    if (L->count < L->k)
        L->count++;
}

/* the shrinking cull radius (squared): the k-th best once the list is full */
static float orc_list_cull(const orc_list *L)
{
    return L->count == L->k ? L->d2[L->k - 1] : L->r2;
}

static void orc_list_emit(const orc_list *L, int32_t *ids, float *d2)
{
    for (int i = 0; i < L->k; ++i) {
        if (i < L->count) {
            ids[i] = L->id[i];
            d2[i] = L->d2[i];
        } else {
            ids[i] = -1;
            d2[i] = INFINITY;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Plain definition: k lexicographically smallest (d2, id) with d2 <= r2.   */
/* ------------------------------------------------------------------------ */

void orc_knn_brute(const float *pts, int64_t N, int D, const float *qs, int64_t Q,
                   int k, float max_radius, int32_t *ids, float *d2)
{
    float r2 = max_radius * max_radius;
    float *ld = (float *)malloc((size_t)k * sizeof(float));
    int32_t *li = (int32_t *)malloc((size_t)k * sizeof(int32_t));
    for (int64_t q = 0; q < Q; ++q) {
        orc_list L = {k, 0, r2, ld, li};
        for (int64_t i = 0; i < N; ++i)
            orc_list_offer(&L, orc_d2(pts + i * D, qs + q * D, D), (int32_t)i);
        orc_list_emit(&L, ids + q * k, d2 + q * k);
    }
    free(ld);
    free(li);
}

/* FP64 cross-check: distances of the FP32 inputs computed in double. */
void orc_knn_brute_f64(const float *pts, int64_t N, int D, const float *qs, int64_t Q,
                       int k, int32_t *ids, double *d2)
{
    for (int64_t q = 0; q < Q; ++q) {
        int32_t *oi = ids + q * k;
        double *od = d2 + q * k;
        int count = 0;
        for (int64_t i = 0; i < N; ++i) {
            double s = 0.0;
            for (int j = 0; j < D; ++j) {
                double dj = (double)pts[i * D + j] - (double)qs[q * D + j];
                s += dj * dj;
            }
            if (count == k && !(s < od[k - 1] || (s == od[k - 1] && i < oi[k - 1])))
                continue;
            int pos = count < k ? count : k - 1;
            while (pos > 0 && (s < od[pos - 1] || (s == od[pos - 1] && i < oi[pos - 1]))) {
                od[pos] = od[pos - 1];
                oi[pos] = oi[pos - 1];
                --pos;
            }
            od[pos] = s;
            oi[pos] = (int32_t)i;
            if (count < k)
                ++count;
        }
        for (int i = count; i < k; ++i) {
            oi[i] = -1;
            od[i] = INFINITY;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Traversals over a built tree.  The tree is given as node -> input index; */
/* node coordinates are read from the input points.                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    const float *pts;
    const int32_t *node_pid;
    int64_t N;
    int D;
    const float *q;
    int ordered;       /* 0 unordered, 1 ordered (node before its close child),
                          2 ordered with the node after its close subtree */
    orc_list *L;
    int32_t *visits;   /* first visits (processNode calls), may be NULL */
    int64_t nvisits;
    int64_t vcap;
    int32_t *steps;    /* every node the traversal is "at", may be NULL */
    int64_t nsteps;
    int64_t scap;
    const uint8_t *node_dim; /* stored split dimensions, or NULL: level mod D */
} orc_trav;

static int orc_split_dim(const orc_trav *T, int64_t node)
{
    return T->node_dim ? T->node_dim[node] : orc_level(node) % T->D;
}

static void orc_log(int32_t *buf, int64_t *n, int64_t cap, int64_t node)
{
    if (buf && *n < cap)
        buf[*n] = (int32_t)node;
    ++*n;
}

static void orc_process(orc_trav *T, int64_t node)
{
    int32_t pid = T->node_pid[node];
    float d2 = orc_d2(T->pts + (int64_t)pid * T->D, T->q, T->D);
    orc_list_offer(T->L, d2, pid);
    orc_log(T->visits, &T->nvisits, T->vcap, node);
}

/* Sec. 3.1, second formulation: empty subtree -> return; process; close child;
 * far child if it still overlaps the (possibly shrunk) query range.  The
 * unordered variant always takes the left child first and enters a child iff
 * the query lies on its side or the plane is within the cull radius.  With
 * ordered == 2 the node is processed after its close subtree instead of
 * before it (the swap of root and close subtree that the footnote of Sec. 3.1
 * allows). */
static void orc_rec(orc_trav *T, int64_t node)
{
    orc_log(T->steps, &T->nsteps, T->scap, node);
    if (node >= T->N)
        return;
    if (T->ordered != 2)
        orc_process(T, node);
    int dim = orc_split_dim(T, node);
    float split = T->pts[(int64_t)T->node_pid[node] * T->D + dim];
    float sd = T->q[dim] - split;
    if (T->ordered) {
        int close_side = sd > 0.0f;
        int64_t close_child = 2 * node + 1 + close_side;
        int64_t far_child = 2 * node + 2 - close_side;
        orc_rec(T, close_child);
        orc_log(T->steps, &T->nsteps, T->scap, node);
        if (T->ordered == 2)
            orc_process(T, node);
        if (sd * sd <= orc_list_cull(T->L)) {
            orc_rec(T, far_child);
            orc_log(T->steps, &T->nsteps, T->scap, node);
        }
    } else {
        if (sd <= 0.0f || sd * sd <= orc_list_cull(T->L)) {
            orc_rec(T, 2 * node + 1);
            orc_log(T->steps, &T->nsteps, T->scap, node);
        }
        if (sd > 0.0f || sd * sd <= orc_list_cull(T->L)) {
            orc_rec(T, 2 * node + 2);
            orc_log(T->steps, &T->nsteps, T->scap, node);
        }
    }
}

/* Sec. 3.2: the traversal keeps only the node it is at and the node it came
 * from; the pair says which of three situations it is in.
 *
 *   arrived from the parent   the node is processed (unless ordered == 2),
 *                             then the first child is entered if it is in
 *                             range, else the second, else back to the parent
 *   back from the first child the second child is entered if it is in range,
 *                             else back to the parent
 *   back from the second      back to the parent
 *
 * The two children of a node are ranked per node: the ordered traversal puts
 * the child on the query's side of the plane first, the unordered one puts
 * the left child first.  Either way a child is in range iff the query lies on
 * its side of the plane or the plane is within the current cull radius, so
 * the ordered traversal always enters its first child.  Entering a missing
 * child (index >= N) is one step down and one straight back up.  Going up
 * from the root ends the traversal.  With ordered == 2 a node is processed
 * when the machine is back from its first child, and the second child is then
 * judged against the radius that processing left. */
enum { ORC_FROM_PARENT, ORC_FROM_FIRST, ORC_FROM_SECOND };

/* whether the machine enters `child` of a node whose plane lies at signed
 * distance sd from the query (sd > 0: the query is on the right) */
static int orc_enters(const orc_trav *T, int64_t child, int64_t left, float sd)
{
    int query_side = child == left ? sd <= 0.0f : sd > 0.0f;
    return query_side || sd * sd <= orc_list_cull(T->L);
}

static int orc_stackfree(orc_trav *T)
{
    int64_t at = 0;
    int64_t from = -1;
    int64_t bound = 3 * (2 * T->N + 1) + 8;
    for (int64_t step = 0; step < bound; ++step) {
        orc_log(T->steps, &T->nsteps, T->scap, at);
        int64_t up = at == 0 ? -1 : (at - 1) / 2;
        if (at >= T->N) {
            from = at;
            at = up;
            continue;
        }
        int dim = orc_split_dim(T, at);
        float sd = T->q[dim] - T->pts[(int64_t)T->node_pid[at] * T->D + dim];
        int64_t left = 2 * at + 1;
        int64_t right = left + 1;
        int64_t first = T->ordered && sd > 0.0f ? right : left;
        int64_t second = first == left ? right : left;
        int arrival = from == up ? ORC_FROM_PARENT : (from == first ? ORC_FROM_FIRST : ORC_FROM_SECOND);
        int64_t next = up;
        switch (arrival) {
        case ORC_FROM_PARENT:
            if (T->ordered != 2)
                orc_process(T, at);
            if (orc_enters(T, first, left, sd))
                next = first;
            else if (orc_enters(T, second, left, sd))
                next = second;
            break;
        case ORC_FROM_FIRST:
            if (T->ordered == 2)
                orc_process(T, at);
            if (orc_enters(T, second, left, sd))
                next = second;
            break;
        default: /* ORC_FROM_SECOND */
            break;
        }
        if (next < 0)
            return 0;
        from = at;
        at = next;
    }
    return -1; /* step bound exceeded: cannot happen for a correct machine */
}

static int orc_knn_tree(const float *pts, const int32_t *node_pid, const uint8_t *node_dim, int64_t N, int D,
                        const float *q, int k, float max_radius, int ordered,
                        int stackfree, int32_t *ids, float *d2,
                        int32_t *visits, int64_t vcap, int64_t *nvisits,
                        int32_t *steps, int64_t scap, int64_t *nsteps)
{
    float *ld = (float *)malloc((size_t)k * sizeof(float));
    int32_t *li = (int32_t *)malloc((size_t)k * sizeof(int32_t));
    orc_list L = {k, 0, max_radius * max_radius, ld, li};
    orc_trav T = {pts, node_pid, N, D, q, ordered, &L, visits, 0, vcap, steps, 0, scap, node_dim};
    int rc = 0;
    if (stackfree)
        rc = orc_stackfree(&T);
    else
        orc_rec(&T, 0);
    orc_list_emit(&L, ids, d2);
    if (nvisits)
        *nvisits = T.nvisits;
    if (nsteps)
        *nsteps = T.nsteps;
    free(ld);
    free(li);
    return rc;
}

/* One query, recursive traversal, with optional visit / step logs. */
int orc_knn_recursive(const float *pts, const int32_t *node_pid, int64_t N, int D,
                      const float *q, int k, float max_radius, int ordered,
                      int32_t *ids, float *d2, int32_t *visits, int64_t vcap,
                      int64_t *nvisits, int32_t *steps, int64_t scap, int64_t *nsteps)
{
    return orc_knn_tree(pts, node_pid, NULL, N, D, q, k, max_radius, ordered, 0, ids, d2,
                        visits, vcap, nvisits, steps, scap, nsteps);
}

/* One query, stack-free state machine, with optional visit / step logs. */
int orc_knn_stackfree(const float *pts, const int32_t *node_pid, int64_t N, int D,
                      const float *q, int k, float max_radius, int ordered,
                      int32_t *ids, float *d2, int32_t *visits, int64_t vcap,
                      int64_t *nvisits, int32_t *steps, int64_t scap, int64_t *nsteps)
{
    return orc_knn_tree(pts, node_pid, NULL, N, D, q, k, max_radius, ordered, 1, ids, d2,
                        visits, vcap, nvisits, steps, scap, nsteps);
}

/* Many queries through the stack-free machine; per-query first-visit counts.
 * node_dim: stored split dimensions, or NULL for level mod D. */
int orc_knn_stackfree_batch_dims(const float *pts, const int32_t *node_pid, const uint8_t *node_dim, int64_t N,
                                 int D, const float *qs, int64_t Q, int k, float max_radius,
                                 int ordered, int32_t *ids, float *d2, int32_t *nvisit)
{
    int rc = 0;
    for (int64_t i = 0; i < Q; ++i) {
        int64_t nv = 0;
        if (orc_knn_tree(pts, node_pid, node_dim, N, D, qs + i * D, k, max_radius, ordered, 1,
                         ids + i * k, d2 + i * k, NULL, 0, &nv, NULL, 0, NULL))
            rc = -1;
        if (nvisit)
            nvisit[i] = (int32_t)nv;
    }
    return rc;
}

int orc_knn_stackfree_batch(const float *pts, const int32_t *node_pid, int64_t N, int D,
                            const float *qs, int64_t Q, int k, float max_radius,
                            int ordered, int32_t *ids, float *d2, int32_t *nvisit)
{
    return orc_knn_stackfree_batch_dims(pts, node_pid, NULL, N, D, qs, Q, k, max_radius, ordered, ids, d2,
                                        nvisit);
}

/* ------------------------------------------------------------------------ */
/* Learned radius proposal (not in the paper).                              */
/* ------------------------------------------------------------------------ */

/* Greedy descent from the root, always to the close child (the child on the
 * query's side, Sec. 3.2 closeSide rule), until that child does not exist.
 * Returns the FP32 squared distance from q to the last valid node's point.
 * node_dim NULL: split dimension level mod D; else the dimension stored per
 * node by orc_build_widest (Sec. 3.1's stored-split variant). */
float orc_descent_leaf(const float *pts, const int32_t *node_pid, const uint8_t *node_dim, int64_t N, int D,
                       const float *q)
{
    int64_t node = 0;
    for (;;) {
        int dim = node_dim ? node_dim[node] : orc_level(node) % D;
        float sd = q[dim] - pts[(int64_t)node_pid[node] * D + dim];
        int64_t child = 2 * node + 1 + (sd > 0.0f);
        if (child >= N)
            break;
        node = child;
    }
    return orc_d2(pts + (int64_t)node_pid[node] * D, q, D);
}

/* Round a float to the nearest bfloat16 (ties to even), returned as float.
 * bfloat16 keeps the top 16 bits of binary32; finite inputs only. */
float orc_round_bf16(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u = u + 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

/* MLP 4 -> H -> H -> 1 with ReLU, parameters laid out as
 *   W1[H][4], b1[H], W2[H][H], b2[H], w3[H], b3
 * (row-major, W[out][in]); evaluated in FP64 on the given parameter values
 * (the caller passes BF16-rounded weights to mirror the device model). */
void orc_mlp_forward(const double *params, int H, const double *x, int64_t n, double *y)
{
    const double *W1 = params;
    const double *b1 = W1 + (int64_t)H * 4;
    const double *W2 = b1 + H;
    const double *b2 = W2 + (int64_t)H * H;
    const double *w3 = b2 + H;
    const double *b3 = w3 + H;
    double *h1 = (double *)malloc((size_t)H * sizeof(double));
    double *h2 = (double *)malloc((size_t)H * sizeof(double));
    for (int64_t s = 0; s < n; ++s) {
        const double *xs = x + s * 4;
        for (int i = 0; i < H; ++i) {
            double a = b1[i];
            for (int j = 0; j < 4; ++j)
                a += W1[i * 4 + j] * xs[j];
            h1[i] = a > 0.0 ? a : 0.0;
        }
        for (int i = 0; i < H; ++i) {
            double a = b2[i];
            for (int j = 0; j < H; ++j)
                a += W2[(int64_t)i * H + j] * h1[j];
            h2[i] = a > 0.0 ? a : 0.0;
        }
        double o = b3[0];
        for (int i = 0; i < H; ++i)
            o += w3[i] * h2[i];
        y[s] = o;
    }
    free(h1);
    free(h2);
}

/* Loss = (1/n) * sum_s (y_s - label_s)^2 and its gradient with respect to every
 * parameter (same layout as params), by the chain rule through the ReLUs.
 * Returns the loss. */
double orc_mlp_loss_grad(const double *params, int H, const double *x,
                         const double *label, int64_t n, double *grad)
{
    const double *W1 = params;
    const double *b1 = W1 + (int64_t)H * 4;
    const double *W2 = b1 + H;
    const double *b2 = W2 + (int64_t)H * H;
    const double *w3 = b2 + H;
    const double *b3 = w3 + H;
    int64_t P = (int64_t)H * 4 + H + (int64_t)H * H + H + H + 1;
    double *gW1 = grad;
    double *gb1 = gW1 + (int64_t)H * 4;
    double *gW2 = gb1 + H;
    double *gb2 = gW2 + (int64_t)H * H;
    double *gw3 = gb2 + H;
    double *gb3 = gw3 + H;
    for (int64_t i = 0; i < P; ++i)
        grad[i] = 0.0;
    double *z1 = (double *)malloc((size_t)H * sizeof(double));
    double *h1 = (double *)malloc((size_t)H * sizeof(double));
    double *z2 = (double *)malloc((size_t)H * sizeof(double));
    double *h2 = (double *)malloc((size_t)H * sizeof(double));
    double *g2 = (double *)malloc((size_t)H * sizeof(double));
    double *g1 = (double *)malloc((size_t)H * sizeof(double));
    double loss = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        const double *xs = x + s * 4;
        for (int i = 0; i < H; ++i) {
            double a = b1[i];
            for (int j = 0; j < 4; ++j)
                a += W1[i * 4 + j] * xs[j];
            z1[i] = a;
            h1[i] = a > 0.0 ? a : 0.0;
        }
        for (int i = 0; i < H; ++i) {
            double a = b2[i];
            for (int j = 0; j < H; ++j)
                a += W2[(int64_t)i * H + j] * h1[j];
            z2[i] = a;
            h2[i] = a > 0.0 ? a : 0.0;
        }
        double o = b3[0];
        for (int i = 0; i < H; ++i)
            o += w3[i] * h2[i];
        double e = o - label[s];
        loss += e * e;
        double go = 2.0 * e / (double)n;   /* dLoss / dy_s */
        gb3[0] += go;
        for (int i = 0; i < H; ++i) {
            gw3[i] += go * h2[i];
            g2[i] = z2[i] > 0.0 ? go * w3[i] : 0.0;   /* dLoss / dz2_i */
        }
        for (int i = 0; i < H; ++i) {
            gb2[i] += g2[i];
            for (int j = 0; j < H; ++j)
                gW2[(int64_t)i * H + j] += g2[i] * h1[j];
        }
        for (int j = 0; j < H; ++j) {
            double a = 0.0;
            for (int i = 0; i < H; ++i)
                a += W2[(int64_t)i * H + j] * g2[i];
            g1[j] = z1[j] > 0.0 ? a : 0.0;             /* dLoss / dz1_j */
        }
        for (int i = 0; i < H; ++i) {
            gb1[i] += g1[i];
            for (int j = 0; j < 4; ++j)
                gW1[i * 4 + j] += g1[i] * xs[j];
        }
    }
    free(z1);
    free(h1);
    free(z2);
    free(h2);
    free(g2);
    free(g1);
    return loss / (double)n;
}

/* The model's forward (as orc_mlp_forward, FP64) together with, per sample, a
 * bound on how far from it an evaluation in the precision the radius model is
 * specified in can land: the hidden activations rounded to bfloat16 as the
 * operands of the 64 x 64 contraction (BF16 in), everything else in FP32
 * (FP32 accumulation), in any order, each FP32 operation with a relative error
 * of at most 2^-23 (round to nearest gives 2^-24; the bound also admits
 * truncating accumulation).  params hold bfloat16-valued weights, x values
 * exact in FP32.  With g(m) = m e / (1 - m e), e = 2^-23, for m operations and
 * b = 2^-8 the unit roundoff of bfloat16 (8 significant bits):
 *   layer 1: |z1' - z1| <= g(10) S1, S1 = |b1| + sum |W1 x|; the activation
 *            relu(z1') rounded to bfloat16 is within
 *            e1 = b (h1 + g(10) S1) + g(10) S1 of h1 (relu is 1-Lipschitz);
 *   layer 2: e2 = sum_i |W2_ji| e1_i + g(2H + 2) (|b2_j| + sum_i |W2_ji| (h1_i + e1_i));
 *   output:  e3 = sum_j |w3_j| e2_j + g(2H + 2) (|b3| + sum_j |w3_j| (h2_j + e2_j)). */
static double orc_gamma(int m)
{
    const double e = 1.0 / 8388608.0;
    return m * e / (1.0 - m * e);
}

void orc_mlp_forward_bound(const double *params, int H, const double *x, int64_t n, double *y, double *bound)
{
    const double *W1 = params;
    const double *b1 = W1 + (int64_t)H * 4;
    const double *W2 = b1 + H;
    const double *b2 = W2 + (int64_t)H * H;
    const double *w3 = b2 + H;
    const double *b3 = w3 + H;
    const double ub = 1.0 / 256.0;
    const double g1 = orc_gamma(10), g2 = orc_gamma(2 * H + 2);
    double *h1 = (double *)malloc((size_t)H * sizeof(double));
    double *e1 = (double *)malloc((size_t)H * sizeof(double));
    double *h2 = (double *)malloc((size_t)H * sizeof(double));
    double *e2 = (double *)malloc((size_t)H * sizeof(double));
    for (int64_t s = 0; s < n; ++s) {
        const double *xs = x + s * 4;
        for (int i = 0; i < H; ++i) {
            double z = b1[i], S = fabs(b1[i]);
            for (int j = 0; j < 4; ++j) {
                z += W1[i * 4 + j] * xs[j];
                S += fabs(W1[i * 4 + j] * xs[j]);
            }
            h1[i] = z > 0.0 ? z : 0.0;
            e1[i] = ub * (h1[i] + g1 * S) + g1 * S;
        }
        for (int j = 0; j < H; ++j) {
            double z = b2[j], A = fabs(b2[j]), prop = 0.0;
            for (int i = 0; i < H; ++i) {
                double w = W2[(int64_t)j * H + i];
                z += w * h1[i];
                A += fabs(w) * (h1[i] + e1[i]);
                prop += fabs(w) * e1[i];
            }
            h2[j] = z > 0.0 ? z : 0.0;
            e2[j] = prop + g2 * A;
        }
        double o = b3[0], A = fabs(b3[0]), prop = 0.0;
        for (int j = 0; j < H; ++j) {
            o += w3[j] * h2[j];
            A += fabs(w3[j]) * (h2[j] + e2[j]);
            prop += fabs(w3[j]) * e2[j];
        }
        y[s] = o;
        bound[s] = prop + g2 * A;
    }
    free(h1);
    free(e1);
    free(h2);
    free(e2);
}

/* The loss and gradient of orc_mlp_loss_grad (FP64) together with, per
 * parameter, a bound on how far from it an evaluation in the training
 * precision of the radius model can land: the forward as for
 * orc_mlp_forward_bound (hidden activations rounded to bfloat16 where they
 * enter the 64 x 64 contraction), and in the backward pass the gradient at the
 * hidden layer's pre-activations rounded to bfloat16 where it enters the two
 * contractions (G2 W2 and G2^T H1), everything else in FP32 in any order, each
 * FP32 operation with a relative error of at most 2^-23.  A ReLU whose input
 * lies within its error bound of 0 may switch either way; the bound then
 * admits both values.  Per sample s, with e the FP32 allowance and b = 2^-8:
 *   output error     de = e3 + e (|err| + e3); dgo = 2 de / n + 3 e 2 (|err| + de) / n
 *   g2_i             dg2 = (|go| + dgo) |w3_i| (1 + e) if |z2_i| <= e2_i, else
 *                    [z2_i > 0] (dgo + e (|go| + dgo)) |w3_i|; |g2_i| <= M2_i;
 *                    as a BF16 operand dg2b = dg2 + b M2
 *   dH1_j            d = sum_i dg2b |W2_ij| + g(2H+2) sum_i M2b |W2_ij|, magnitude MH
 *   g1_j             dg1 = MH + d if |z1_j| <= g(10) S1_j, else [z1_j > 0] d
 * and the parameter bounds sum these over the samples with the summation
 * allowance g(2n) of their magnitudes.  bound[P] bounds the loss. */
double orc_mlp_loss_grad_bound(const double *params, int H, const double *x, const double *label, int64_t n,
                               double *grad, double *bound)
{
    const double *W1 = params;
    const double *b1 = W1 + (int64_t)H * 4;
    const double *W2 = b1 + H;
    const double *b2 = W2 + (int64_t)H * H;
    const double *w3 = b2 + H;
    const double *b3 = w3 + H;
    int64_t P = (int64_t)H * 4 + H + (int64_t)H * H + H + H + 1;
    double *bW1 = bound;
    double *bb1 = bW1 + (int64_t)H * 4;
    double *bW2 = bb1 + H;
    double *bb2 = bW2 + (int64_t)H * H;
    double *bw3 = bb2 + H;
    double *bb3 = bw3 + H;
    const double ub = 1.0 / 256.0, uf = 1.0 / 8388608.0;
    const double g10 = orc_gamma(10), gH = orc_gamma(2 * H + 2), gn = orc_gamma((int)(2 * n + 2 < 2000000000 ? 2 * n + 2 : 2000000000));
    double loss = orc_mlp_loss_grad(params, H, x, label, n, grad);
    /* per-parameter sums over the samples: propagated errors and magnitudes */
    double *acc = (double *)calloc((size_t)(2 * (P + 1)), sizeof(double));
    double *mag = acc + P + 1;
    double *z1 = (double *)malloc((size_t)H * 8), *h1 = (double *)malloc((size_t)H * 8);
    double *E1 = (double *)malloc((size_t)H * 8), *e1 = (double *)malloc((size_t)H * 8);
    double *z2 = (double *)malloc((size_t)H * 8), *h2 = (double *)malloc((size_t)H * 8);
    double *e2 = (double *)malloc((size_t)H * 8);
    double *dg2b = (double *)malloc((size_t)H * 8), *M2b = (double *)malloc((size_t)H * 8);
    for (int64_t s = 0; s < n; ++s) {
        const double *xs = x + s * 4;
        for (int j = 0; j < H; ++j) {
            double z = b1[j], S = fabs(b1[j]);
            for (int m = 0; m < 4; ++m) {
                z += W1[j * 4 + m] * xs[m];
                S += fabs(W1[j * 4 + m] * xs[m]);
            }
            z1[j] = z;
            h1[j] = z > 0.0 ? z : 0.0;
            E1[j] = g10 * S;
            e1[j] = ub * (h1[j] + E1[j]) + E1[j];
        }
        double y = b3[0], A3 = fabs(b3[0]), p3 = 0.0;
        for (int i = 0; i < H; ++i) {
            double z = b2[i], A = fabs(b2[i]), pr = 0.0;
            for (int j = 0; j < H; ++j) {
                double w = W2[(int64_t)i * H + j];
                z += w * h1[j];
                A += fabs(w) * (h1[j] + e1[j]);
                pr += fabs(w) * e1[j];
            }
            z2[i] = z;
            h2[i] = z > 0.0 ? z : 0.0;
            e2[i] = pr + gH * A;
            y += w3[i] * h2[i];
            A3 += fabs(w3[i]) * (h2[i] + e2[i]);
            p3 += fabs(w3[i]) * e2[i];
        }
        const double e3 = p3 + gH * A3;
        const double err = y - label[s];
        const double de = e3 + uf * (fabs(err) + e3);
        const double go = 2.0 * err / (double)n;
        const double dgo = 2.0 * de / (double)n + 3.0 * uf * 2.0 * (fabs(err) + de) / (double)n;
        const double ago = fabs(go) + dgo;
        /* output layer and its bias */
        acc[P - 1] += dgo;
        mag[P - 1] += ago;
        for (int i = 0; i < H; ++i) {
            acc[(bw3 - bound) + i] += fabs(go) * e2[i] + dgo * (h2[i] + e2[i]) + uf * ago * (h2[i] + e2[i]);
            mag[(bw3 - bound) + i] += ago * (h2[i] + e2[i]);
            const int amb = fabs(z2[i]) <= e2[i];
            const int on = z2[i] > 0.0 || amb;
            const double M2 = on ? ago * fabs(w3[i]) * (1.0 + uf) : 0.0;
            const double dg2 = amb ? M2 : (z2[i] > 0.0 ? (dgo + uf * ago) * fabs(w3[i]) : 0.0);
            acc[(bb2 - bound) + i] += dg2;
            mag[(bb2 - bound) + i] += M2;
            dg2b[i] = dg2 + ub * M2;
            M2b[i] = M2 * (1.0 + ub);
        }
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < H; ++j) {
                acc[(bW2 - bound) + (int64_t)i * H + j] += dg2b[i] * (h1[j] + e1[j]) + M2b[i] * e1[j];
                mag[(bW2 - bound) + (int64_t)i * H + j] += M2b[i] * (h1[j] + e1[j]);
            }
        for (int j = 0; j < H; ++j) {
            double d = 0.0, MH = 0.0;
            for (int i = 0; i < H; ++i) {
                d += dg2b[i] * fabs(W2[(int64_t)i * H + j]);
                MH += M2b[i] * fabs(W2[(int64_t)i * H + j]);
            }
            d += gH * MH;
            MH *= 1.0 + gH;
            const int amb = fabs(z1[j]) <= E1[j];
            const int on = z1[j] > 0.0 || amb;
            const double dg1 = amb ? MH + d : (z1[j] > 0.0 ? d : 0.0);
            const double M1 = on ? MH + d : 0.0;
            acc[(bb1 - bound) + j] += dg1;
            mag[(bb1 - bound) + j] += M1;
            for (int m = 0; m < 4; ++m) {
                acc[(bW1 - bound) + j * 4 + m] += dg1 * fabs(xs[m]) + uf * M1 * fabs(xs[m]);
                mag[(bW1 - bound) + j * 4 + m] += M1 * fabs(xs[m]);
            }
        }
        acc[P] += (2.0 * fabs(err) * de + de * de) / (double)n;
        mag[P] += (fabs(err) + de) * (fabs(err) + de) / (double)n;
    }
    for (int64_t q = 0; q <= P; ++q)
        bound[q] = acc[q] + gn * mag[q];
    (void)bb3;
    free(acc);
    free(z1);
    free(h1);
    free(E1);
    free(e1);
    free(z2);
    free(h2);
    free(e2);
    free(dg2b);
    free(M2b);
    return loss;
}

/* ------------------------------------------------------------------------ */
/* Range queries (Sec. 3: a point / sphere or a box as query primitive).     */
/* ------------------------------------------------------------------------ */

/* Every point with d2 <= fl(r * r) (FP32 distance as orc_d2), per query in
 * input-index order.  counts[q] receives the number; when ids is not NULL,
 * query q's ids (and d2 when not NULL) are written at offsets[q]. */
void orc_radius_brute(const float *pts, int64_t N, int D, const float *qs, int64_t Q, float radius,
                      int32_t *counts, const int64_t *offsets, int32_t *ids, float *d2)
{
    float r2 = radius * radius;
    for (int64_t q = 0; q < Q; ++q) {
        int64_t c = 0;
        for (int64_t i = 0; i < N; ++i) {
            float v = orc_d2(pts + i * D, qs + q * D, D);
            if (v <= r2) {
                if (ids) {
                    ids[offsets[q] + c] = (int32_t)i;
                    if (d2)
                        d2[offsets[q] + c] = v;
                }
                ++c;
            }
        }
        counts[q] = (int32_t)c;
    }
}

/* Every point p with lo_j <= p_j <= hi_j for all j, per query in input-index
 * order (counts / offsets / ids as orc_radius_brute). */
void orc_box_brute(const float *pts, int64_t N, int D, const float *lo, const float *hi, int64_t Q,
                   int32_t *counts, const int64_t *offsets, int32_t *ids)
{
    for (int64_t q = 0; q < Q; ++q) {
        int64_t c = 0;
        for (int64_t i = 0; i < N; ++i) {
            int in = 1;
            for (int j = 0; j < D; ++j) {
                float v = pts[i * D + j];
                if (!(lo[q * D + j] <= v && v <= hi[q * D + j])) {
                    in = 0;
                    break;
                }
            }
            if (in) {
                if (ids)
                    ids[offsets[q] + c] = (int32_t)i;
                ++c;
            }
        }
        counts[q] = (int32_t)c;
    }
}

/* Range queries over a built tree through the (curr, prev) machine of
 * Sec. 3.2, unordered (left child first), with a fixed range instead of a
 * shrinking one.  kind 0: the ball d2 <= r2 around a; kind 1: the box
 * [a, b].  Children are entered as in the unordered kNN traversal: a child
 * whose side holds the query, or whose plane is within range.  Missing
 * children are stepped into and left, as in orc_stackfree.  Writes the hits'
 * input indices (and d2 for balls) in traversal order, up to cap of them, and
 * returns their number (or -1 if the step bound was exceeded). */
static int64_t orc_range_one(const float *pts, const int32_t *node_pid, const uint8_t *node_dim, int64_t N, int D,
                             int kind, const float *a, const float *b, float r2, int32_t *ids, float *d2, int64_t cap,
                             int64_t *nvisits)
{
    int64_t curr = 0, prev = -1, count = 0, visits = 0;
    int64_t bound = 3 * (2 * N + 1) + 8;
    for (int64_t step = 0; step < bound; ++step) {
        int64_t parent = (curr + 1) / 2 - 1;
        if (curr >= N) {
            prev = curr;
            curr = parent;
            continue;
        }
        const float *p = pts + (int64_t)node_pid[curr] * D;
        int from_parent = prev < curr;
        if (from_parent) {
            ++visits;
            int hit;
            float v = 0.0f;
            if (kind == 0) {
                v = orc_d2(p, a, D);
                hit = v <= r2;
            } else {
                hit = 1;
                for (int j = 0; j < D; ++j)
                    if (!(a[j] <= p[j] && p[j] <= b[j]))
                        hit = 0;
            }
            if (hit) {
                if (count < cap) {
                    ids[count] = node_pid[curr];
                    if (d2)
                        d2[count] = v;
                }
                ++count;
            }
        }
        int dim = node_dim ? node_dim[curr] : orc_level(curr) % D;
        float split = p[dim];
        int left_in, right_in;
        if (kind == 0) {
            float sd = a[dim] - split;
            left_in = sd <= 0.0f || sd * sd <= r2;
            right_in = sd > 0.0f || sd * sd <= r2;
        } else {
            left_in = a[dim] <= split;   /* left subtree: coordinates <= split */
            right_in = b[dim] >= split;  /* right subtree: coordinates >= split */
        }
        int64_t lc = 2 * curr + 1, rc = 2 * curr + 2, next;
        if (from_parent)
            next = left_in ? lc : (right_in ? rc : parent);
        else if (prev == lc)
            next = right_in ? rc : parent;
        else
            next = parent;
        if (next == -1) {
            if (nvisits)
                *nvisits = visits;
            return count;
        }
        prev = curr;
        curr = next;
    }
    return -1;
}

/* Many range queries; counts[q] = hits of query q; when ids is not NULL,
 * query q's hits go to ids[offsets[q] ...] (and d2 for balls) in traversal
 * order.  qb: upper corners (boxes) or NULL (balls).  Returns -1 if any
 * traversal exceeded its step bound. */
int orc_range_stackfree(const float *pts, const int32_t *node_pid, const uint8_t *node_dim, int64_t N, int D,
                        int kind, const float *qa, const float *qb, int64_t Q, float radius, int32_t *counts,
                        const int64_t *offsets, int32_t *ids, float *d2)
{
    float r2 = radius * radius;
    int rc = 0;
    for (int64_t q = 0; q < Q; ++q) {
        int64_t c;
        if (ids)
            c = orc_range_one(pts, node_pid, node_dim, N, D, kind, qa + q * D, kind ? qb + q * D : NULL, r2,
                              ids + offsets[q], d2 ? d2 + offsets[q] : NULL, offsets[q + 1] - offsets[q], NULL);
        else
            c = orc_range_one(pts, node_pid, node_dim, N, D, kind, qa + q * D, kind ? qb + q * D : NULL, r2,
                              NULL, NULL, 0, NULL);
        if (c < 0)
            rc = -1;
        counts[q] = (int32_t)c;
    }
    return rc;
}

/* Processed nodes (first visits) of each range query's traversal. */
int orc_range_visits(const float *pts, const int32_t *node_pid, const uint8_t *node_dim, int64_t N, int D, int kind,
                     const float *qa, const float *qb, int64_t Q, float radius, int32_t *visits)
{
    float r2 = radius * radius;
    int rc = 0;
    for (int64_t q = 0; q < Q; ++q) {
        int64_t nv = 0;
        if (orc_range_one(pts, node_pid, node_dim, N, D, kind, qa + q * D, kind ? qb + q * D : NULL, r2, NULL, NULL, 0,
                          &nv) < 0)
            rc = -1;
        visits[q] = (int32_t)nv;
    }
    return rc;
}

/* Reductions of a payload (C floats per input point, input order).  The sum
 * runs in FP32 over the hits in the order given, one addition at a time.
 * mode 0: the sum; 1: the sum / count; 2: density, the sum / fl(pi_f * R2)
 * with R2 the squared radius of the disc the hits were gathered from.  No
 * hit: 0 in every mode. */
#define ORC_PI_F 3.14159265358979323846f

static void orc_reduce_one(const float *payload, int C, const int32_t *hits, int64_t n, int mode, float R2,
                           float *out)
{
    for (int c = 0; c < C; ++c) {
        float s = 0.0f;
        for (int64_t i = 0; i < n; ++i)
            s = s + payload[(int64_t)hits[i] * C + c];
        if (n == 0)
            s = 0.0f;
        else if (mode == 1)
            s = s / (float)n;
        else if (mode == 2)
            s = s / (ORC_PI_F * R2);
        out[c] = s;
    }
}

/* Ball queries (radius r, R2 = fl(r * r)) through orc_range_one, reduced in
 * traversal order: out [Q][C]; counts [Q] may be NULL. */
int orc_range_reduce(const float *pts, const int32_t *node_pid, const uint8_t *node_dim, int64_t N, int D,
                     const float *qs, int64_t Q, float radius, const float *payload, int C, int mode, float *out,
                     int32_t *counts)
{
    float r2 = radius * radius;
    int32_t *hits = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
    int rc = 0;
    for (int64_t q = 0; q < Q; ++q) {
        int64_t n = orc_range_one(pts, node_pid, node_dim, N, D, 0, qs + q * D, NULL, r2, hits, NULL, N, NULL);
        if (n < 0) {
            rc = -1;
            n = 0;
        }
        orc_reduce_one(payload, C, hits, n, mode, r2, out + q * C);
        if (counts)
            counts[q] = (int32_t)n;
    }
    free(hits);
    return rc;
}

/* Reductions over kNN results (ids / d2 [Q][k], ascending, -1 = empty), in
 * list order; R2 = the largest d2 found (the disc through the farthest
 * neighbour, as in the photon-map radiance estimate). */
void orc_knn_reduce(const int32_t *ids, const float *d2, int64_t Q, int k, const float *payload, int C, int mode,
                    float *out)
{
    for (int64_t q = 0; q < Q; ++q) {
        int64_t n = 0;
        while (n < k && ids[q * k + n] >= 0)
            ++n;
        float R2 = n ? d2[q * k + n - 1] : 0.0f;
        orc_reduce_one(payload, C, ids + q * k, n, mode, R2, out + q * C);
    }
}
