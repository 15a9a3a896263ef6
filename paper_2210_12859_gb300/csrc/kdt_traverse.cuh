// Device-side traversal core shared by the plain, learned and batched query
// kernels: node fetch for the three node layouts, the FP32 squared distance,
// the k-best lists and the stack-free (curr, prev) state machine of Sec. 3.2.
#pragma once

#include "kdt_internal.cuh"

namespace kdt {

// number of coordinate slots per layout (padding slots hold 0 in both the
// node and the query, and add exactly +0 to a distance)
template <int LAYOUT> struct LayoutTraits;
template <> struct LayoutTraits<0> { static constexpr int NC = 3; static constexpr int NF = 1; };
template <> struct LayoutTraits<1> { static constexpr int NC = 4; static constexpr int NF = 1; };
template <> struct LayoutTraits<2> { static constexpr int NC = 8; static constexpr int NF = 2; };
template <> struct LayoutTraits<3> { static constexpr int NC = 3; static constexpr int NF = 1; };

template <int LAYOUT>
struct NodeVal {
    float c[LayoutTraits<LAYOUT>::NC];
    uint32_t id;  // layouts 0 and 3 (the node's id word)
};

// split dimension of a node: stored in the id word (layout 3), else the
// dimension the walker tracks (level mod D)
template <int LAYOUT>
__device__ __forceinline__ int split_dim_of(const NodeVal<LAYOUT> &nd, int tracked)
{
    if constexpr (LAYOUT == 3)
        return (int)(nd.id >> NODE_DIM_SHIFT);
    else
        return tracked;
}

__device__ __forceinline__ float4 ldg_f4(const float4 *p) { return __ldg(p); }

// Fetch node `curr` (from shared memory when it is among the `staged` first
// nodes).  nodes: the tree's node array (already offset to the tree's base).
template <int LAYOUT, bool STAGE = true>
__device__ __forceinline__ NodeVal<LAYOUT> fetch(const float4 *__restrict__ nodes, const float4 *s_nodes, int staged,
                                                 int curr)
{
    NodeVal<LAYOUT> v;
    if constexpr (LAYOUT == 2) {
        float4 a, b;
        if (STAGE && curr < staged) {
            a = s_nodes[2 * curr];
            b = s_nodes[2 * curr + 1];
        } else {
            a = ldg_f4(nodes + 2 * curr);
            b = ldg_f4(nodes + 2 * curr + 1);
        }
        v.c[0] = a.x; v.c[1] = a.y; v.c[2] = a.z; v.c[3] = a.w;
        v.c[4] = b.x; v.c[5] = b.y; v.c[6] = b.z; v.c[7] = b.w;
        v.id = 0;
    } else {
        float4 a = (STAGE && curr < staged) ? s_nodes[curr] : ldg_f4(nodes + curr);
        v.c[0] = a.x; v.c[1] = a.y; v.c[2] = a.z;
        if constexpr (LAYOUT == 1) {
            v.c[3] = a.w;
            v.id = 0;
        } else {
            v.id = __float_as_uint(a.w);
        }
    }
    return v;
}

template <int NC>
__device__ __forceinline__ float select_dim(const float (&c)[NC], int dim)
{
    float r = c[0];
#pragma unroll
    for (int j = 1; j < NC; ++j)
        r = dim == j ? c[j] : r;
    return r;
}

// d2 = ((t_0 + t_1) + t_2) + ..., t_j = fl(fl(p_j - q_j)^2); the _rn
// intrinsics are never contracted into fused multiply-adds.
template <int NC>
__device__ __forceinline__ float dist2(const float (&p)[NC], const float (&q)[NC])
{
    float d = __fsub_rn(p[0], q[0]);
    float s = __fmul_rn(d, d);
#pragma unroll
    for (int j = 1; j < NC; ++j) {
        float dj = __fsub_rn(p[j], q[j]);
        s = __fadd_rn(s, __fmul_rn(dj, dj));
    }
    return s;
}

// (d2, id) packed so that unsigned 64-bit order is the lexicographic order:
// d2 >= +0 or NaN, whose float bits order like unsigned integers.
__device__ __forceinline__ unsigned long long pack_key(float d2, uint32_t id)
{
    return ((unsigned long long)__float_as_uint(d2) << 32) | id;
}
__device__ __forceinline__ float key_d2(unsigned long long k) { return __uint_as_float((uint32_t)(k >> 32)); }

constexpr uint32_t EMPTY_ID = 0xffffffffu;

// Register-resident sorted k-best list of capacity K.  A query for k <= K
// neighbours fills the first K-k slots with key 0 (below every real key), so
// they never move, and the k real slots start at (r2, EMPTY_ID): a candidate
// is accepted iff its key is below the last slot, which is exactly
// "d2 <= r2 and (list not full or (d2, id) < worst)"; the last slot's d2 is
// the shrinking cull radius (r2 until k points are held).
template <int K>
struct RegList {
    unsigned long long L[K];
    __device__ __forceinline__ void init(int k, float r2)
    {
        unsigned long long s = pack_key(r2, EMPTY_ID);
#pragma unroll
        for (int i = 0; i < K; ++i)
            L[i] = i < K - k ? 0ull : s;
    }
    __device__ __forceinline__ float cull() const { return key_d2(L[K - 1]); }
    __device__ __forceinline__ unsigned long long worst() const { return L[K - 1]; }
    __device__ __forceinline__ void insert(unsigned long long c)
    {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            unsigned long long a = L[i];
            bool sw = c < a;
            L[i] = sw ? c : a;
            c = sw ? a : c;
        }
    }
    __device__ __forceinline__ void store(int k, int32_t *ids, float *d2) const
    {
        if constexpr (K % 4 == 0) {
            // a full row on 16-byte boundaries: four 16-byte stores instead of
            // 2K word stores (fewer transactions, which matters most when the
            // outputs are host memory written through the C2C link)
            if (k == K && ((reinterpret_cast<uintptr_t>(ids) | reinterpret_cast<uintptr_t>(d2)) & 15u) == 0) {
#pragma unroll
                for (int i = 0; i < K; i += 4) {
                    int32_t vi[4];
                    float vd[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t id = (uint32_t)L[i + j];
                        const bool empty = id == EMPTY_ID;
                        vi[j] = empty ? -1 : (int32_t)id;
                        vd[j] = empty ? __int_as_float(0x7f800000) : key_d2(L[i + j]);
                    }
                    *reinterpret_cast<int4 *>(ids + i) = make_int4(vi[0], vi[1], vi[2], vi[3]);
                    *reinterpret_cast<float4 *>(d2 + i) = make_float4(vd[0], vd[1], vd[2], vd[3]);
                }
                return;
            }
        }
#pragma unroll
        for (int i = 0; i < K; ++i) {
            int o = i - (K - k);
            if (o >= 0) {
                uint32_t id = (uint32_t)L[i];
                bool empty = id == EMPTY_ID;
                ids[o] = empty ? -1 : (int32_t)id;
                d2[o] = empty ? __int_as_float(0x7f800000) : key_d2(L[i]);
            }
        }
    }
    __device__ __forceinline__ bool full(int) const { return (uint32_t)L[K - 1] != EMPTY_ID; }
};

// k-best set for 16 < k <= 64: a binary max-heap of packed (d2, id) keys per
// thread, in shared memory (slot i of thread t at s[i * stride + t], so
// consecutive threads hit consecutive banks) or in a per-thread slice of a
// global scratch buffer (stride 1: the thread's k keys contiguous).  The root is the worst key, i.e.
// the cull radius; an accepted key replaces the root and sifts down (log2 k
// levels instead of k/2 shifts of a sorted list).  The k slots start at
// (r2, EMPTY_ID) like the register list, which gives the same acceptance rule.
// store() sorts the heap once (heapsort, ascending).
struct SmemList {
    unsigned long long *s;
    int stride;
    int k;
    unsigned long long w;  // root (worst key) mirrored in a register
    __device__ __forceinline__ void init(int k_, float r2)
    {
        k = k_;
        w = pack_key(r2, EMPTY_ID);
        for (int i = 0; i < k; ++i)
            s[i * stride] = w;
    }
    __device__ __forceinline__ float cull() const { return key_d2(w); }
    __device__ __forceinline__ unsigned long long worst() const { return w; }
    // replace the root by c (c < root) and restore the heap on [0, n)
    __device__ __forceinline__ static void sift(unsigned long long *h, int stride, int n, unsigned long long c)
    {
        int i = 0;
        for (;;) {
            const int l = 2 * i + 1;
            if (l >= n)
                break;
            unsigned long long big = h[l * stride];
            int j = l;
            if (l + 1 < n) {
                const unsigned long long r = h[(l + 1) * stride];
                if (r > big) {
                    big = r;
                    j = l + 1;
                }
            }
            if (!(big > c))
                break;
            h[i * stride] = big;
            i = j;
        }
        h[i * stride] = c;
    }
    __device__ __forceinline__ void insert(unsigned long long c)
    {
        sift(s, stride, k, c);
        w = s[0];
    }
    __device__ __forceinline__ void store(int, int32_t *ids, float *d2)
    {
        // heapsort: move the maximum to the end, shrink, repeat
        for (int n = k; n > 1; --n) {
            const unsigned long long top = s[0];
            const unsigned long long last = s[(n - 1) * stride];
            s[(n - 1) * stride] = top;
            sift(s, stride, n - 1, last);
        }
        for (int i = 0; i < k; ++i) {
            unsigned long long key = s[i * stride];
            uint32_t id = (uint32_t)key;
            bool empty = id == EMPTY_ID;
            ids[i] = empty ? -1 : (int32_t)id;
            d2[i] = empty ? __int_as_float(0x7f800000) : key_d2(key);
        }
    }
    // whether k points are held: the root is a real point
    __device__ __forceinline__ bool full(int) const { return (uint32_t)w != EMPTY_ID; }
};

// k-best list spread over a group of G lanes that walk one query together
// (every lane of the group runs the same steps on the same values).  The
// list is sorted across the group: lane j of the group holds positions
// [j M, (j + 1) M) in registers, sorted.  Inserting c shifts everything after
// c's place by one position: lane j takes in max(c, last key of lane j - 1)
// (c for lane 0; the blocks are contiguous, so that is the key leaving lane
// j - 1), one warp shuffle, and runs the compare-swap chain of RegList on its
// block, whose largest key leaves.  The group's last key, the worst (the cull
// radius), is then broadcast from the group's last lane.  As in RegList, the
// first G M - k positions hold key 0 and the k real ones start at
// (r2, EMPTY_ID).  Shuffles use the group's lane mask: the group's lanes are
// converged wherever the list is touched.
template <int M, int G>
struct GroupList {
    unsigned long long L[M];
    unsigned long long w;  // worst key of the group's list
    int li;                // lane within the group
    unsigned gmask;        // the group's lanes
    __device__ __forceinline__ void init(int k, float r2)
    {
        const int lane = threadIdx.x & 31;
        li = lane % G;
        gmask = ((1u << G) - 1u) << (lane - li);
        const unsigned long long s = pack_key(r2, EMPTY_ID);
        const int pad = G * M - k;
#pragma unroll
        for (int i = 0; i < M; ++i)
            L[i] = li * M + i < pad ? 0ull : s;
        w = s;
    }
    __device__ __forceinline__ float cull() const { return key_d2(w); }
    __device__ __forceinline__ unsigned long long worst() const { return w; }
    __device__ __forceinline__ void insert(unsigned long long c)
    {
        const unsigned long long left_last = __shfl_up_sync(gmask, L[M - 1], 1, G);
        unsigned long long in = (li == 0 || c > left_last) ? c : left_last;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const unsigned long long a = L[i];
            const bool sw = in < a;
            L[i] = sw ? in : a;
            in = sw ? a : in;
        }
        w = __shfl_sync(gmask, L[M - 1], G - 1, G);
    }
    __device__ __forceinline__ void store(int k, int32_t *ids, float *d2) const
    {
        const int pad = G * M - k;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int o = li * M + i - pad;
            if (o >= 0) {
                const uint32_t id = (uint32_t)L[i];
                const bool empty = id == EMPTY_ID;
                ids[o] = empty ? -1 : (int32_t)id;
                d2[o] = empty ? __int_as_float(0x7f800000) : key_d2(L[i]);
            }
        }
    }
    __device__ __forceinline__ bool full(int) const { return (uint32_t)w != EMPTY_ID; }
};

// processNode of fcp / kNN for node `n` (values nd)
template <int LAYOUT, class List>
__device__ __forceinline__ void process(const NodeVal<LAYOUT> &nd, int n, const int32_t *__restrict__ ids,
                                        const float (&q)[LayoutTraits<LAYOUT>::NC], List &list)
{
    const float d2 = dist2<LayoutTraits<LAYOUT>::NC>(nd.c, q);
    if (d2 <= key_d2(list.worst())) {
        const uint32_t id = LAYOUT == 0 ? nd.id : (LAYOUT == 3 ? (nd.id & NODE_ID_MASK) : (uint32_t)__ldg(ids + n));
        const unsigned long long key = pack_key(d2, id);
        if (key < list.worst())
            list.insert(key);
    }
}

// The stack-free state machine of Sec. 3.2 for one query, advanced one step
// at a time so that a persistent lane can interleave queries.
//
// Two shortcuts leave the sequence of processed nodes unchanged:
//  * a missing child is never stepped into: stepping into it and straight back
//    only sets prev to that child, so the machine continues as if it had been
//    visited;
//  * when the subtree below a node is at most INLINE_DEPTH levels deep, it is
//    processed in the node's own step, in the order the machine would visit
//    it (close child, its subtree, then the far child and its subtree if the
//    plane is still within the cull radius; unordered: left then right, each
//    if in range), and the step returns to the parent - the same processed
//    nodes in the same order, without the steps into and out of them.
// Depth of the bottom subtrees processed inside one step (1: a node whose
// children are leaves; 2: also a node whose grandchildren are leaves; 3 and 4:
// also a node whose subtree below is three or four levels deep, as blocks of
// depth 2 whose seven loads are issued when the machine enters them).  Depth 2 pays when queries
// process many nodes; for short queries the four extra up-front loads cost
// more than the steps they save, and depth 1 is faster; depth 3 saves the two
// steps between the halves (the tuner measures which).
constexpr int INLINE_DEPTH = 2;

template <int LAYOUT, bool ORDERED, int INLINE = INLINE_DEPTH>
struct Walker {
    static constexpr int NC = LayoutTraits<LAYOUT>::NC;
    int curr, prev, dim;
    uint32_t steps;

    __device__ __forceinline__ void start()
    {
        curr = 0;
        prev = -1;
        dim = 0;
        steps = 0;
    }

    // Whole bottom subtrees: the keys (d2, id) of all their nodes and the
    // children's split offsets are computed first, from the values loaded at
    // once; the machine's order is then followed on these scalars (a node's
    // key is offered to the list when the machine would process it), which
    // needs far fewer registers and selects than carrying whole node values.
    __device__ __forceinline__ static unsigned long long node_key(const NodeVal<LAYOUT> &nd, int n,
                                                                   const int32_t *__restrict__ ids,
                                                                   const float (&q)[NC])
    {
        const float d2 = dist2<NC>(nd.c, q);
        const uint32_t id = LAYOUT == 0 ? nd.id : (LAYOUT == 3 ? (nd.id & NODE_ID_MASK) : (uint32_t)__ldg(ids + n));
        return pack_key(d2, id);
    }
    template <class List>
    __device__ __forceinline__ static void offer(List &list, unsigned long long k)
    {
        if (k < list.worst())
            list.insert(k);
    }
    // leaves lcc (key ka) and lcc + 1 (key kb, valid iff lcc + 1 < N) below a
    // node whose split offset is sdc, in the machine's order: ordered, close
    // leaf first and the far one if the plane is still within the cull
    // radius; unordered, left then right, each if on the query's side or in range
    template <class List>
    __device__ __forceinline__ static void eager_leaf_pair(float sdc, float sdc2, int lcc, unsigned long long ka,
                                                           unsigned long long kb, int N, List &list, int &visits)
    {
        const bool rcc_ok = lcc + 1 < N;
        if constexpr (ORDERED) {
            const bool rf = sdc > 0.f;
            if (!rf || rcc_ok) {
                ++visits;
                offer(list, rf ? kb : ka);
            }
            if ((rf || rcc_ok) && sdc2 <= list.cull()) {
                ++visits;
                offer(list, rf ? ka : kb);
            }
        } else {
            if (sdc <= 0.f || sdc2 <= list.cull()) {
                ++visits;
                offer(list, ka);
            }
            if (rcc_ok && (sdc > 0.f || sdc2 <= list.cull())) {
                ++visits;
                offer(list, kb);
            }
        }
    }
    template <class List>
    __device__ __forceinline__ static void eager_leaf_parent(int c, unsigned long long kc, float sdc,
                                                             unsigned long long ka, unsigned long long kb, int N,
                                                             List &list, int &visits)
    {
        ++visits;
        offer(list, kc);
        const int lcc = 2 * c + 1;
        if (lcc < N)
            eager_leaf_pair(sdc, __fmul_rn(sdc, sdc), lcc, ka, kb, N, list, visits);
    }

    // The subtree below a node x of depth at most 2 (x's grandchildren are
    // leaves or missing) as scalars: the keys of x's two children and four
    // grandchildren and the children's split offsets.  The six node indices
    // follow from x alone, so all loads are issued first (indices clamped to
    // N - 1; values of missing nodes are never used).  dim1: the split
    // dimension of x's children (level mod D).  LEAF_OK: x may be a leaf
    // (else its left child is known to exist).
    struct Below2 {
        unsigned long long k_c0, k_c1, k_g00, k_g01, k_g10, k_g11;
        float sdc0, sdc1;
    };
    template <bool STAGE, bool LEAF_OK>
    __device__ __forceinline__ static Below2 load_below2(int x, int dim1, const float4 *__restrict__ nodes,
                                                         const int32_t *__restrict__ ids, const float4 *s_nodes,
                                                         int staged, int N, const float (&q)[NC])
    {
        const int last = N - 1;
        const int lc = 2 * x + 1, rc = lc + 1;
        const int g0 = 2 * lc + 1;
        const int lcx = LEAF_OK ? min(lc, last) : lc;
        const NodeVal<LAYOUT> c0 = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, lcx);
        const NodeVal<LAYOUT> c1 = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, min(rc, last));
        const NodeVal<LAYOUT> g00 = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, min(g0, last));
        const NodeVal<LAYOUT> g01 = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, min(g0 + 1, last));
        const NodeVal<LAYOUT> g10 = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, min(g0 + 2, last));
        const NodeVal<LAYOUT> g11 = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, min(g0 + 3, last));
        Below2 b;
        b.k_c0 = node_key(c0, lcx, ids, q);
        b.k_c1 = node_key(c1, min(rc, last), ids, q);
        b.k_g00 = node_key(g00, min(g0, last), ids, q);
        b.k_g01 = node_key(g01, min(g0 + 1, last), ids, q);
        b.k_g10 = node_key(g10, min(g0 + 2, last), ids, q);
        b.k_g11 = node_key(g11, min(g0 + 3, last), ids, q);
        const int d0 = split_dim_of<LAYOUT>(c0, dim1), d1 = split_dim_of<LAYOUT>(c1, dim1);
        b.sdc0 = __fsub_rn(select_dim<NC>(q, d0), select_dim<NC>(c0.c, d0));
        b.sdc1 = __fsub_rn(select_dim<NC>(q, d1), select_dim<NC>(c1.c, d1));
        return b;
    }
    // the machine's order over that subtree, x already processed, sd: x's
    // split offset
    template <bool LEAF_OK, class List>
    __device__ __forceinline__ static void walk_below2(int x, float sd, const Below2 &b, int N, List &list,
                                                       int &visits)
    {
        const int lc = 2 * x + 1, rc = lc + 1;
        const bool lc_ok = !LEAF_OK || lc < N, rc_ok = rc < N;
        const float sd2 = __fmul_rn(sd, sd);
        if constexpr (ORDERED) {
            const bool right_first = sd > 0.f;
            if (right_first ? rc_ok : lc_ok)
                eager_leaf_parent(right_first ? rc : lc, right_first ? b.k_c1 : b.k_c0, right_first ? b.sdc1 : b.sdc0,
                                  right_first ? b.k_g10 : b.k_g00, right_first ? b.k_g11 : b.k_g01, N, list, visits);
            if ((right_first ? lc_ok : rc_ok) && sd2 <= list.cull())
                eager_leaf_parent(right_first ? lc : rc, right_first ? b.k_c0 : b.k_c1, right_first ? b.sdc0 : b.sdc1,
                                  right_first ? b.k_g00 : b.k_g10, right_first ? b.k_g01 : b.k_g11, N, list, visits);
        } else {
            if (lc_ok && (sd <= 0.f || sd2 <= list.cull()))
                eager_leaf_parent(lc, b.k_c0, b.sdc0, b.k_g00, b.k_g01, N, list, visits);
            if (rc_ok && (sd > 0.f || sd2 <= list.cull()))
                eager_leaf_parent(rc, b.k_c1, b.sdc1, b.k_g10, b.k_g11, N, list, visits);
        }
    }


    // The subtree below a processed node x of depth at most L >= 2, in the
    // machine's order: for L = 2 the six-node block above; otherwise each
    // child in turn (close child first, or left first unordered; a child only
    // when it exists and is in range), its key offered and the subtree below
    // it walked the same way.  A child's own node is loaded together with the
    // first block below it.  dimc: the split dimension of x's children.
    // MIN: a lower bound on the depth of x's subtree (x is a leaf only when
    // MIN = 0); a child's subtree is at most two levels shallower than its
    // parent's lower bound (the right one may be a level shallower than the
    // left, which is one shallower than the parent).
    template <int L, bool STAGE, int MIN, class List>
    __device__ __forceinline__ static void walk_below(int x, float sd, int dimc, int D,
                                                      const float4 *__restrict__ nodes,
                                                      const int32_t *__restrict__ ids, const float4 *s_nodes,
                                                      int staged, int N, const float (&q)[NC], List &list,
                                                      int &visits)
    {
        if constexpr (L <= 2) {
            walk_below2<MIN < 1>(x, sd, load_below2<STAGE, (MIN < 1)>(x, dimc, nodes, ids, s_nodes, staged, N, q), N,
                                 list, visits);
        } else {
            const int lc = 2 * x + 1;
            const int dimg = dimc + 1 == D ? 0 : dimc + 1;
            const bool first_right = ORDERED && sd > 0.f;
            const int fc = lc + (int)first_right, sc = lc + 1 - (int)first_right;
            const float sd2 = __fmul_rn(sd, sd);
            if (fc < N && (ORDERED || sd <= 0.f || sd2 <= list.cull())) {
                const NodeVal<LAYOUT> nf = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, fc);
                ++visits;
                offer(list, node_key(nf, fc, ids, q));
                const int df = split_dim_of<LAYOUT>(nf, dimc);
                walk_below<L - 1, STAGE, (MIN >= 2 ? MIN - 2 : 0)>(fc, __fsub_rn(select_dim<NC>(q, df), select_dim<NC>(nf.c, df)), dimg, D,
                                         nodes, ids, s_nodes, staged, N, q, list, visits);
            }
            if (sc < N && ((!ORDERED && sd > 0.f) || sd2 <= list.cull())) {
                const NodeVal<LAYOUT> ns = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, sc);
                ++visits;
                offer(list, node_key(ns, sc, ids, q));
                const int ds = split_dim_of<LAYOUT>(ns, dimc);
                walk_below<L - 1, STAGE, (MIN >= 2 ? MIN - 2 : 0)>(sc, __fsub_rn(select_dim<NC>(q, ds), select_dim<NC>(ns.c, ds)), dimg, D,
                                         nodes, ids, s_nodes, staged, N, q, list, visits);
            }
        }
    }

    // The subtree below node c is at least L levels deep iff its leftmost
    // descendant L levels down, (c + 1) 2^L - 1, exists, i.e. iff
    // c < floor(N / 2^L) = N >> L: the depth tests of a step are compares
    // against these thresholds.

    // One or more steps; returns true when the traversal has finished.  With
    // RUNS and light_run > 1 a call continues with further steps while the next one is
    // light (not entering a node whose bottom subtree is processed whole), at
    // most light_run steps, so the heavy steps of a warp's lanes tend to
    // start their calls together (the same steps in the same order; pays for
    // short queries, not for long ones: tuned).  The caller bounds a
    // traversal by checking `steps` against 3N + 3 once per claim round (and
    // reports an overrun through *overflow).  STAGE: the first `staged` nodes
    // are read from shared memory.
    template <bool STAGE, bool RUNS, class List>
    __device__ __forceinline__ bool step(const float4 *__restrict__ nodes, const int32_t *__restrict__ ids,
                                         const float4 *s_nodes, int staged, int N, int D, const float (&q)[NC],
                                         List &list, int &visits, bool &overflow, int light_run = 1)
    {
      for (int g = 0;; ++g) {
        ++steps;
        const NodeVal<LAYOUT> nd = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, curr);
        const bool from_parent = prev < curr;
        if (from_parent) {
            ++visits;
            process<LAYOUT>(nd, curr, ids, q, list);
        }
        const int sdim = split_dim_of<LAYOUT>(nd, dim);
        const float sd = __fsub_rn(select_dim<NC>(q, sdim), select_dim<NC>(nd.c, sdim));
        const float sd2 = __fmul_rn(sd, sd);
        const int lc = 2 * curr + 1;
        const int parent = (curr - 1) >> 1;  // -1 for the root
        int next;
        const int rc = lc + 1;
        const int dim1 = dim + 1 == D ? 0 : dim + 1;
        // whole subtrees below at most INLINE (and at least one) levels deep
        // are processed in this step
        // (for INLINE <= 2 from the children's indices, which keeps the
        // depth-2 kernel at 64 registers)
        bool inl;
        if constexpr (INLINE >= 3)
            inl = from_parent && curr < (N >> 1) && curr >= (N >> (INLINE + 1));
        else if constexpr (INLINE == 2)
            inl = from_parent && lc < N && 2u * (2u * (uint32_t)lc + 1u) + 1u >= (uint32_t)N;
        else
            inl = INLINE == 1 && from_parent && lc < N && 2 * lc + 1 >= N;
        if (INLINE >= 4 && inl && curr < (N >> 4)) {
            // the subtree below is four levels deep: its two depth-3 halves,
            // each as two depth-2 blocks of seven loads issued together
            walk_below<4, STAGE, 4>(curr, sd, dim1, D, nodes, ids, s_nodes, staged, N, q, list, visits);
            next = parent;
        } else if (INLINE >= 3 && inl && curr < (N >> 3)) {
            // three levels deep: both children (each with the depth-1 or
            // depth-2 subtree below it) in the machine's order, each child's
            // seven nodes loaded at once when the machine enters that child
            walk_below<3, STAGE, 3>(curr, sd, dim1, D, nodes, ids, s_nodes, staged, N, q, list, visits);
            next = parent;
        } else if (INLINE >= 2 && inl && (INLINE >= 3 ? curr < (N >> 2) : 2 * lc + 1 < N)) {
            // the children have only leaves below them: the whole depth-2
            // subtree in the machine's order, its six loads issued first
            walk_below<2, STAGE, 2>(curr, sd, dim1, D, nodes, ids, s_nodes, staged, N, q, list, visits);
            next = parent;
        } else if (inl) {
            // both children are leaves (the right one may be missing): both
            // loads first
            const NodeVal<LAYOUT> a = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, lc);
            const NodeVal<LAYOUT> b = fetch<LAYOUT, STAGE>(nodes, s_nodes, staged, min(rc, N - 1));
            eager_leaf_pair(sd, sd2, lc, node_key(a, lc, ids, q), node_key(b, min(rc, N - 1), ids, q), N, list,
                            visits);
            next = parent;
        } else {
            const float cull = list.cull();
            if constexpr (ORDERED) {
                const int close_side = sd > 0.f;
                const int close_child = lc + close_side;
                const int far_child = lc + 1 - close_side;
                const bool far_ok = sd2 <= cull && far_child < N;
                if (from_parent)
                    next = close_child < N ? close_child : (far_ok ? far_child : parent);
                else if (prev == close_child)
                    next = far_ok ? far_child : parent;
                else
                    next = parent;
            } else {
                const int rc = lc + 1;
                const bool left_ok = (sd <= 0.f || sd2 <= cull) && lc < N;
                const bool right_ok = (sd > 0.f || sd2 <= cull) && rc < N;
                if (from_parent)
                    next = left_ok ? lc : (right_ok ? rc : parent);
                else if (prev == lc)
                    next = right_ok ? rc : parent;
                else
                    next = parent;
            }
        }
        if (next < 0)
            return true;
        if (next == parent)
            dim = dim == 0 ? D - 1 : dim - 1;
        else
            dim = dim + 1 == D ? 0 : dim + 1;
        prev = curr;
        curr = next;
        if constexpr (!RUNS)
            return false;
        if (g + 1 >= light_run)
            return false;
        // stop before a heavy step (entering a node whose bottom subtree is
        // processed whole), so that it starts the next call
        if (curr > prev && 2 * curr + 1 < N &&
            (INLINE >= 3 ? curr >= (N >> (INLINE + 1))
                         : (INLINE == 2 ? 2u * (2u * (2u * (uint32_t)curr + 1u) + 1u) + 1u >= (uint32_t)N
                                        : 2 * (2 * curr + 1) + 1 >= N)))
            return false;
      }
    }
};


template <int LAYOUT>
__device__ __forceinline__ void load_query(const float *__restrict__ queries, int64_t qi, int D,
                                           float (&q)[LayoutTraits<LAYOUT>::NC])
{
    constexpr int NC = LayoutTraits<LAYOUT>::NC;
#pragma unroll
    for (int j = 0; j < NC; ++j)
        q[j] = j < D ? __ldg(queries + qi * D + j) : 0.f;
}

// stage the first `staged` nodes of a tree into shared memory (whole block)
template <int LAYOUT>
__device__ __forceinline__ void stage_nodes(const float4 *__restrict__ nodes, float4 *s_nodes, int staged)
{
    constexpr int NF = LayoutTraits<LAYOUT>::NF;
    for (int i = threadIdx.x; i < staged * NF; i += blockDim.x)
        s_nodes[i] = ldg_f4(nodes + i);
}

// Greedy close-child descent from the root (Sec. 3.2's closeSide rule at every
// node) until that child does not exist; returns the FP32 squared distance to
// the last node reached (layout 0 / 3 trees, D <= 3; stored: split dimension
// stored in the node).
__device__ __forceinline__ float descent_leaf_d2(const float4 *__restrict__ nodes, const float4 *s_nodes, int staged,
                                                 int N, int D, const float (&q)[3], bool stored = false)
{
    int node = 0, dim = 0;
    NodeVal<0> nd = fetch<0>(nodes, s_nodes, staged, 0);
    for (;;) {
        const int sdim = stored ? (int)(nd.id >> NODE_DIM_SHIFT) : dim;
        const float sd = __fsub_rn(select_dim<3>(q, sdim), select_dim<3>(nd.c, sdim));
        const int child = 2 * node + 1 + (sd > 0.f);
        if (child >= N)
            break;
        node = child;
        dim = dim + 1 == D ? 0 : dim + 1;
        nd = fetch<0>(nodes, s_nodes, staged, node);
    }
    return dist2<3>(nd.c, q);
}

__device__ __forceinline__ uint32_t lane_mask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace kdt
