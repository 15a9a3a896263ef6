// Range queries and payload reductions.
//
// Ball: every point within a fixed radius of a query point; box: every point
// inside an axis-aligned box.  Sec. 3 notes that other query primitives only
// change the in-range test and what processNode does, and that a non-ordered
// traversal is a simplification of the ordered one; both queries use the
// unordered stack-free machine (left child first, a child is entered iff it
// can hold a point in range) with a fixed range instead of a shrinking one.
// The kernel is templated over the processNode action:
//   ACT_COUNT   count the hits;
//   ACT_FILL    write the hits to the query's slice [offsets[q], offsets[q+1])
//               in traversal order (count and fill walk the same nodes in the
//               same order, so no atomics are needed); hits from the first
//               16-byte boundary of the slice on are collected four at a time
//               in registers and written as 16-byte stores, the slice's
//               unaligned head and its last partial group one word at a time;
//   ACT_REDUCE  sum a per-point payload over the hits in traversal order (the
//               point types with payload, e.g. photon power, that Sec. 3 names;
//               the fixed-radius photon-map density estimate on top).
// A payload is attached to the tree in node order, so that its loads follow
// the node loads of the traversal; kNN reductions gather it through the
// inverse permutation after an ordinary kNN query.
#include <string.h>

#include "kdt_learned.cuh"
#include "kdt_query.cuh"

namespace kdt {
namespace {

constexpr int RANGE_THREADS = 128;
// traversal steps between two claim rounds of a warp (as for kNN, 64 beats 16)
constexpr int RANGE_CLAIM_STEPS = 64;
// levels below a bottom node that one traversal step walks with it, per
// processNode action.  Measured on the clustered 2^24 set (2^22 ball queries):
// one level takes the count pass from 103 to 74 ms at r = 0.004 (3852 nodes
// per query) and leaves it unchanged at r = 0.001 (172 nodes); two levels gain
// more on long queries (59 ms) but cost registers, and so resident warps, on
// short ones (+9 %).  The fill, whose hit staging already holds more
// registers, is fastest without inlining at r = 0.001 and within 6 % of the
// best at r = 0.004.
constexpr int RANGE_COUNT_LEVELS = 1;
constexpr int RANGE_FILL_LEVELS = 0;
constexpr int RANGE_REDUCE_LEVELS = 1;
enum : int { ACT_COUNT = 0, ACT_FILL = 1, ACT_REDUCE = 2 };
// binary32 rounding of pi
constexpr float PI_F = 3.14159265358979323846f;

struct RangeArgs {
    const float4 *nodes;
    const int32_t *ids;
    int N, D;
    const float *a;  // ball: centres; box: lower corners   [Q][D]
    const float *b;  // box: upper corners                  [Q][D]
    int64_t Q;
    const uint32_t *perm;  // traversal order -> query index, or NULL
    float r2;
    int32_t *counts;
    const int64_t *offsets;
    int32_t *out_ids;
    float *out_d2;
    const float *payload;  // [N][C] in node order (ACT_REDUCE)
    int C;
    int mode;              // KDT_REDUCE_*
    float *out;            // [Q][C] (ACT_REDUCE)
    bool count_visits;     // ACT_COUNT: count processed nodes instead of hits
    bool vec_fill;         // ACT_FILL: outputs 16-byte aligned, groups of four hits stored at once
    int *err;
    unsigned long long *counter;
};

template <int LAYOUT>
__device__ __forceinline__ uint32_t node_id(const NodeVal<LAYOUT> &nd, const int32_t *__restrict__ ids, int n)
{
    if constexpr (LAYOUT == 0)
        return nd.id;
    else if constexpr (LAYOUT == 3)
        return nd.id & NODE_ID_MASK;
    else
        return (uint32_t)__ldg(ids + n);
}

// Final value of a reduction: no hit -> 0; mean: / count; density: / fl(pi * R2).
__device__ __forceinline__ float finish_reduce(float s, int64_t n, int mode, float R2)
{
    if (n == 0)
        return 0.f;
    if (mode == KDT_REDUCE_MEAN)
        return __fdiv_rn(s, (float)n);
    if (mode == KDT_REDUCE_DENSITY)
        return __fdiv_rn(s, __fmul_rn(PI_F, R2));
    return s;
}

// One lane's range query: the query box / ball and the processNode action's
// state.  node() is processNode for a node entered from its parent; cull()
// gives which children can hold a point in range (their existence is the
// caller's test).  The fill's pending group of up to three hits waits in
// registers (a staging buffer in shared memory measured slower: the carve-out
// it takes shrinks the L1 that neighbouring lanes share nodes through).
// fill: the last `ns` hits (ns < 4) not yet written, newest in the last slot
template <bool FILL>
struct FillStage {
};
template <>
struct FillStage<true> {
    int64_t base;
    int32_t limit;
    int32_t sid0, sid1, sid2, sid3;
    float sd20, sd21, sd22, sd23;
    int ns;
};

template <int LAYOUT, int KIND, int ACT>
struct RangeLane : FillStage<ACT == ACT_FILL> {
    static constexpr int NC = LayoutTraits<LAYOUT>::NC;
    float lo[NC], hi[KIND == 1 ? NC : 1];
    float acc[ACT == ACT_REDUCE ? KDT_PAYLOAD_MAX_C : 1];
    int32_t count, visits;  // hits and nodes of one query are below N < 2^30

    __device__ __forceinline__ void start(const RangeArgs &a, int64_t qi)
    {
        load_query<LAYOUT>(a.a, qi, a.D, lo);
        if constexpr (KIND == 1)
            load_query<LAYOUT>(a.b, qi, a.D, hi);
        count = 0;
        visits = 0;
        if constexpr (ACT == ACT_FILL) {
            this->base = a.offsets[qi];
            // saturated: a slice longer than any hit count, or negative, still
            // ends with count != limit and the range error
            const int64_t len = a.offsets[qi + 1] - this->base;
            this->limit = (int32_t)(len < 0 ? -1 : (len > INT32_MAX ? INT32_MAX : len));
            this->ns = 0;
        }
        if constexpr (ACT == ACT_REDUCE) {
#pragma unroll
            for (int c = 0; c < KDT_PAYLOAD_MAX_C; ++c)
                acc[c] = 0.f;
        }
    }

    __device__ __forceinline__ void node(const RangeArgs &a, const NodeVal<LAYOUT> &nd, int n)
    {
        if constexpr (ACT == ACT_COUNT)
            ++visits;
        bool hit;
        float d2 = 0.f;
        if constexpr (KIND == 0) {
            d2 = dist2<NC>(nd.c, lo);
            hit = d2 <= a.r2;
        } else {
            hit = true;
#pragma unroll
            for (int j = 0; j < NC; ++j)
                hit = hit && lo[j] <= nd.c[j] && nd.c[j] <= hi[j];
        }
        if (!hit)
            return;
        if constexpr (ACT == ACT_FILL) {
            if (count < this->limit) {
                const int32_t id = (int32_t)node_id<LAYOUT>(nd, a.ids, n);
                const int64_t pos = this->base + count;
                if (!a.vec_fill || (this->ns == 0 && (pos & 3) != 0)) {
                    // before the slice's first 16-byte boundary (or unaligned outputs)
                    a.out_ids[pos] = id;
                    if (KIND == 0 && a.out_d2)
                        a.out_d2[pos] = d2;
                } else {
                    this->sid0 = this->sid1; this->sid1 = this->sid2; this->sid2 = this->sid3; this->sid3 = id;
                    this->sd20 = this->sd21; this->sd21 = this->sd22; this->sd22 = this->sd23; this->sd23 = d2;
                    if (++this->ns == 4) {  // positions pos - 3 .. pos, pos - 3 on a 16-byte boundary
                        *reinterpret_cast<int4 *>(a.out_ids + pos - 3) =
                            make_int4(this->sid0, this->sid1, this->sid2, this->sid3);
                        if (KIND == 0 && a.out_d2)
                            *reinterpret_cast<float4 *>(a.out_d2 + pos - 3) =
                                make_float4(this->sd20, this->sd21, this->sd22, this->sd23);
                        this->ns = 0;
                    }
                }
            }
        }
        if constexpr (ACT == ACT_REDUCE) {
            const float *p = a.payload + (int64_t)n * a.C;
#pragma unroll
            for (int c = 0; c < KDT_PAYLOAD_MAX_C; ++c)
                if (c < a.C)
                    acc[c] = __fadd_rn(acc[c], __ldg(p + c));
        }
        ++count;
    }

    __device__ __forceinline__ void cull(const RangeArgs &a, const NodeVal<LAYOUT> &nd, int sdim, bool &left_ok,
                                         bool &right_ok) const
    {
        const float split = select_dim<NC>(nd.c, sdim);
        if constexpr (KIND == 0) {
            const float sd = __fsub_rn(select_dim<NC>(lo, sdim), split);
            const float sd2 = __fmul_rn(sd, sd);
            left_ok = sd <= 0.f || sd2 <= a.r2;
            right_ok = sd > 0.f || sd2 <= a.r2;
        } else {
            // left subtree coordinates are <= split, right ones >= split
            left_ok = select_dim<NC>(lo, sdim) <= split;
            right_ok = select_dim<NC>(hi, sdim) >= split;
        }
    }

    // the query's end: the last partial group of the fill, the count or the
    // reduction written out
    __device__ __forceinline__ void finish(const RangeArgs &a, int64_t qi)
    {
        if constexpr (ACT == ACT_FILL) {
            // the newest ns hits end at position base + min(count, limit) - 1
            const int64_t end = this->base + (count < this->limit ? count : this->limit);
            if (this->ns >= 3) {
                a.out_ids[end - 3] = this->sid1;
                if (KIND == 0 && a.out_d2)
                    a.out_d2[end - 3] = this->sd21;
            }
            if (this->ns >= 2) {
                a.out_ids[end - 2] = this->sid2;
                if (KIND == 0 && a.out_d2)
                    a.out_d2[end - 2] = this->sd22;
            }
            if (this->ns >= 1) {
                a.out_ids[end - 1] = this->sid3;
                if (KIND == 0 && a.out_d2)
                    a.out_d2[end - 1] = this->sd23;
            }
            this->ns = 0;
            if (count != this->limit)
                atomicOr(a.err, ERR_RANGE);
        } else {
            if (a.counts)
                a.counts[qi] = ACT == ACT_COUNT && a.count_visits ? visits : count;
            if constexpr (ACT == ACT_REDUCE) {
#pragma unroll
                for (int c = 0; c < KDT_PAYLOAD_MAX_C; ++c)
                    if (c < a.C)
                        a.out[qi * a.C + c] = finish_reduce(acc[c], count, a.mode, a.r2);
            }
        }
    }
};

// KIND 0: ball of squared radius r2 around a[q]; KIND 1: box [a[q], b[q]].
// Persistent blocks; every lane claims its next query when its current one
// ends (checked every RANGE_CLAIM_STEPS steps), as in the kNN kernel; the step
// bound 3N + 3 is checked once per round.  A node entered from its parent
// whose subtree spans at most L + 1 levels (L the action's level constant; index >=
// floor(N / 2^(L+1)) for L levels below it: its leftmost descendant L + 1
// levels down, 2^(L+1) (i + 1) - 1, does not exist) is walked whole in one
// step: its descendants are loaded together, then entered in the machine's
// order (node, left subtree, right subtree) under the same cull tests, and
// the step returns to the parent as the machine would after the node's right
// subtree.  Hits, their order and the processed nodes are those of the
// one-node-per-step machine.
template <int LAYOUT, int KIND, int ACT>
__global__ void __launch_bounds__(RANGE_THREADS) range_kernel(const RangeArgs a)
{
    // levels below a node walked within its step (two float4 per node in layout 2: no inlining there)
    constexpr int LEVELS =
        ACT == ACT_COUNT ? RANGE_COUNT_LEVELS : (ACT == ACT_FILL ? RANGE_FILL_LEVELS : RANGE_REDUCE_LEVELS);
    constexpr int INL = LAYOUT != 2 ? LEVELS : 0;
    RangeLane<LAYOUT, KIND, ACT> L;
    int64_t qi = -1;
    bool exhausted = false;
    int curr = 0, prev = -1, dim = 0;
    uint32_t steps = 0;
    const uint32_t cap = 3u * (uint32_t)a.N + 3u;
    const int last = a.N - 1, bottom = a.N >> (INL + 1);
    for (;;) {
        const bool need = qi < 0 && !exhausted;
        const int64_t slot = claim_slot(need, a.counter);
        if (need) {
            if (slot < a.Q) {
                qi = a.perm ? (int64_t)a.perm[slot] : slot;
                L.start(a, qi);
                curr = 0;
                prev = -1;
                dim = 0;
                steps = 0;
            } else {
                exhausted = true;
            }
        }
        if (__all_sync(0xffffffffu, qi < 0))
            break;
        if (qi < 0)
            continue;
        bool done = false;
        if (steps > cap) {
            atomicOr(a.err, ERR_TRAVERSAL);
            done = true;
        }
        for (int s = 0; s < RANGE_CLAIM_STEPS && !done; ++s) {
            ++steps;
            const NodeVal<LAYOUT> nd = fetch<LAYOUT, false>(a.nodes, nullptr, 0, curr);
            const bool from_parent = prev < curr;
            const int lc = 2 * curr + 1, rc = lc + 1;
            const int parent = (curr - 1) >> 1;
            int next;
            if (INL > 0 && from_parent && curr >= bottom) {
                // children lc, rc (one 32-byte sector); with two levels also
                // the grandchildren 2 lc + 1 .. 2 rc + 2 (indices clamped to
                // the last node for the loads, tested before use)
                const int c1 = min(lc, last), c2 = min(rc, last);
                const NodeVal<LAYOUT> n1 = fetch<LAYOUT, false>(a.nodes, nullptr, 0, c1);
                const NodeVal<LAYOUT> n2 = fetch<LAYOUT, false>(a.nodes, nullptr, 0, c2);
                NodeVal<LAYOUT> m1, m2, m3, m4;
                if constexpr (INL >= 2) {
                    m1 = fetch<LAYOUT, false>(a.nodes, nullptr, 0, min(2 * c1 + 1, last));
                    m2 = fetch<LAYOUT, false>(a.nodes, nullptr, 0, min(2 * c1 + 2, last));
                    m3 = fetch<LAYOUT, false>(a.nodes, nullptr, 0, min(2 * c2 + 1, last));
                    m4 = fetch<LAYOUT, false>(a.nodes, nullptr, 0, min(2 * c2 + 2, last));
                }
                const int dim1 = dim + 1 == a.D ? 0 : dim + 1;
                bool l, r, l1, r1;
                L.node(a, nd, curr);
                L.cull(a, nd, split_dim_of<LAYOUT>(nd, dim), l, r);
                if (l && lc < a.N) {
                    L.node(a, n1, lc);
                    if constexpr (INL >= 2) {
                        L.cull(a, n1, split_dim_of<LAYOUT>(n1, dim1), l1, r1);
                        if (l1 && 2 * lc + 1 < a.N)
                            L.node(a, m1, 2 * lc + 1);
                        if (r1 && 2 * lc + 2 < a.N)
                            L.node(a, m2, 2 * lc + 2);
                    }
                }
                if (r && rc < a.N) {
                    L.node(a, n2, rc);
                    if constexpr (INL >= 2) {
                        L.cull(a, n2, split_dim_of<LAYOUT>(n2, dim1), l1, r1);
                        if (l1 && 2 * rc + 1 < a.N)
                            L.node(a, m3, 2 * rc + 1);
                        if (r1 && 2 * rc + 2 < a.N)
                            L.node(a, m4, 2 * rc + 2);
                    }
                }
                next = parent;
            } else {
                if (from_parent)
                    L.node(a, nd, curr);
                bool left_ok, right_ok;
                L.cull(a, nd, split_dim_of<LAYOUT>(nd, dim), left_ok, right_ok);
                left_ok = left_ok && lc < a.N;
                right_ok = right_ok && rc < a.N;
                if (from_parent)
                    next = left_ok ? lc : (right_ok ? rc : parent);
                else if (prev == lc)
                    next = right_ok ? rc : parent;
                else
                    next = parent;
            }
            if (next < 0) {
                done = true;
                break;
            }
            if (next == parent)
                dim = dim == 0 ? a.D - 1 : dim - 1;
            else
                dim = dim + 1 == a.D ? 0 : dim + 1;
            prev = curr;
            curr = next;
        }
        if (!done)
            continue;
        L.finish(a, qi);
        qi = -1;
    }
}

template <int LAYOUT, int KIND, int ACT>
int launch_one(const RangeArgs &a, cudaStream_t s)
{
    const int grid = grid_for_kernel((const void *)range_kernel<LAYOUT, KIND, ACT>, RANGE_THREADS, 0);
    KDT_LAUNCH range_kernel<LAYOUT, KIND, ACT><<<grid, RANGE_THREADS, 0, s>>>(a);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

template <int LAYOUT>
int launch_range_layout(int kind, int act, const RangeArgs &a, cudaStream_t s)
{
    if (kind == 0) {
        if (act == ACT_COUNT)
            return launch_one<LAYOUT, 0, ACT_COUNT>(a, s);
        if (act == ACT_FILL)
            return launch_one<LAYOUT, 0, ACT_FILL>(a, s);
        return launch_one<LAYOUT, 0, ACT_REDUCE>(a, s);
    }
    if (act == ACT_COUNT)
        return launch_one<LAYOUT, 1, ACT_COUNT>(a, s);
    return launch_one<LAYOUT, 1, ACT_FILL>(a, s);
}

int run_range(const kdt_tree *t, int kind, int act, int flags, RangeArgs a, cudaStream_t s)
{
    pool_setup_once();
    const bool morton = flags & KDT_MORTON;
    Scratch sc(s);
    KDT_TRY(sc.alloc(carve_size({64}) + (morton ? morton_scratch_bytes(a.Q) : 0)));
    Carve c{(char *)sc.p};
    a.counter = c.take<unsigned long long>(8);
    a.nodes = t->nodes;
    a.ids = t->ids;
    a.N = (int)t->N;
    a.D = t->D;
    a.err = t->err;
    a.perm = nullptr;
    if (morton)
        KDT_TRY(morton_order(a.a, a.Q, t->D, t->bbox, 1, nullptr, 0, nullptr, t->N, t->layout == 3, c.base + c.off,
                             const_cast<uint32_t **>(&a.perm), s));
    KDT_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s));
    switch (t->layout) {
    case 0: return launch_range_layout<0>(kind, act, a, s);
    case 1: return launch_range_layout<1>(kind, act, a, s);
    case 3: return launch_range_layout<3>(kind, act, a, s);
    default: return launch_range_layout<2>(kind, act, a, s);
    }
}

__global__ void counts_to_u64_kernel(const int32_t *__restrict__ counts, int64_t Q, unsigned long long *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= Q; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = i < Q ? (unsigned long long)(counts[i] > 0 ? counts[i] : 0) : 0ull;
}

// payload[id][C] (input order) -> node order; node_of[id] = node
template <int LAYOUT>
__global__ void payload_permute_kernel(const float4 *__restrict__ nodes, const int32_t *__restrict__ ids, int64_t N,
                                       const float *__restrict__ in, int C, float *__restrict__ out,
                                       int32_t *__restrict__ node_of)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const NodeVal<LAYOUT> nd = fetch<LAYOUT, false>(nodes, nullptr, 0, (int)n);
        const int64_t id = node_id<LAYOUT>(nd, ids, (int)n);
        for (int c = 0; c < C; ++c)
            out[n * C + c] = in[id * C + c];
        node_of[id] = (int32_t)n;
    }
}

// Sum of the payload over each query's kNN list in list order (ascending
// (d2, id)); density radius R2 = the farthest found neighbour's d2.
__global__ void knn_reduce_kernel(const int32_t *__restrict__ ids, const float *__restrict__ d2, int64_t Q, int k,
                                  const int32_t *__restrict__ node_of, const float *__restrict__ payload, int C,
                                  int mode, float *__restrict__ out)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *row = ids + q * k;
        int n = 0;
        while (n < k && row[n] >= 0)
            ++n;
        const float R2 = n ? d2[q * k + n - 1] : 0.f;
        float acc[KDT_PAYLOAD_MAX_C];
#pragma unroll
        for (int c = 0; c < KDT_PAYLOAD_MAX_C; ++c)
            acc[c] = 0.f;
        for (int i = 0; i < n; ++i) {
            const float *p = payload + (int64_t)node_of[row[i]] * C;
#pragma unroll
            for (int c = 0; c < KDT_PAYLOAD_MAX_C; ++c)
                if (c < C)
                    acc[c] = __fadd_rn(acc[c], __ldg(p + c));
        }
#pragma unroll
        for (int c = 0; c < KDT_PAYLOAD_MAX_C; ++c)
            if (c < C)
                out[q * C + c] = finish_reduce(acc[c], n, mode, R2);
    }
}

unsigned grid_for(int64_t n)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16));
}

int check_range(const kdt_tree *t, int64_t Q, const void *a, const void *b, bool need_b, int flags)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (Q < 0 || Q >= ((int64_t)1 << 32))
        return set_error(KDT_EINVAL, "Q must be in [0, 2^32)");
    if (Q > 0 && (!a || (need_b && !b)))
        return set_error(KDT_EINVAL, "NULL query pointer");
    if (flags & ~(KDT_MORTON | KDT_RANGE_VISITS))
        return set_error(KDT_EINVAL, "range queries take no flag but KDT_MORTON and KDT_RANGE_VISITS (got %#x)",
                         flags);
    return KDT_OK;
}

int check_radius(float radius)
{
    if (!(radius >= 0.f))
        return set_error(KDT_EINVAL, "radius must be >= 0 (got %g)", (double)radius);
    return KDT_OK;
}

RangeArgs blank_args()
{
    RangeArgs a;
    memset(&a, 0, sizeof(a));
    return a;
}

// 16-byte stores of the fill pass only into 16-byte aligned outputs
bool fill_vectorizable(const int32_t *ids, const float *d2)
{
    return ((uintptr_t)ids & 15u) == 0 && ((uintptr_t)d2 & 15u) == 0;
}

}  // namespace
}  // namespace kdt

using namespace kdt;

extern "C" {

int kdt_radius_count(const kdt_tree *t, const float *d_q, int64_t Q, float radius, int flags, int32_t *d_counts,
                     void *stream)
{
    KDT_TRY(check_range(t, Q, d_q, nullptr, false, flags));
    KDT_TRY(check_radius(radius));
    if (Q > 0 && !d_counts)
        return set_error(KDT_EINVAL, "NULL counts");
    if (Q == 0)
        return KDT_OK;
    RangeArgs a = blank_args();
    a.a = d_q;
    a.Q = Q;
    a.r2 = radius * radius;
    a.counts = d_counts;
    a.count_visits = flags & KDT_RANGE_VISITS;
    return run_range(t, 0, ACT_COUNT, flags, a, (cudaStream_t)stream);
}

int kdt_radius_fill(const kdt_tree *t, const float *d_q, int64_t Q, float radius, int flags, const int64_t *d_offsets,
                    int32_t *d_ids, float *d_d2, void *stream)
{
    KDT_TRY(check_range(t, Q, d_q, nullptr, false, flags));
    if (flags & KDT_RANGE_VISITS)
        return set_error(KDT_EINVAL, "KDT_RANGE_VISITS applies to the count calls only");
    KDT_TRY(check_radius(radius));
    if (Q > 0 && (!d_offsets || !d_ids))
        return set_error(KDT_EINVAL, "NULL offsets / ids");
    if (Q == 0)
        return KDT_OK;
    RangeArgs a = blank_args();
    a.a = d_q;
    a.Q = Q;
    a.r2 = radius * radius;
    a.offsets = d_offsets;
    a.out_ids = d_ids;
    a.out_d2 = d_d2;
    a.vec_fill = fill_vectorizable(d_ids, d_d2);
    return run_range(t, 0, ACT_FILL, flags, a, (cudaStream_t)stream);
}

int kdt_box_count(const kdt_tree *t, const float *d_lo, const float *d_hi, int64_t Q, int flags, int32_t *d_counts,
                  void *stream)
{
    KDT_TRY(check_range(t, Q, d_lo, d_hi, true, flags));
    if (Q > 0 && !d_counts)
        return set_error(KDT_EINVAL, "NULL counts");
    if (Q == 0)
        return KDT_OK;
    RangeArgs a = blank_args();
    a.a = d_lo;
    a.b = d_hi;
    a.Q = Q;
    a.counts = d_counts;
    a.count_visits = flags & KDT_RANGE_VISITS;
    return run_range(t, 1, ACT_COUNT, flags, a, (cudaStream_t)stream);
}

int kdt_box_fill(const kdt_tree *t, const float *d_lo, const float *d_hi, int64_t Q, int flags,
                 const int64_t *d_offsets, int32_t *d_ids, void *stream)
{
    KDT_TRY(check_range(t, Q, d_lo, d_hi, true, flags));
    if (flags & KDT_RANGE_VISITS)
        return set_error(KDT_EINVAL, "KDT_RANGE_VISITS applies to the count calls only");
    if (Q > 0 && (!d_offsets || !d_ids))
        return set_error(KDT_EINVAL, "NULL offsets / ids");
    if (Q == 0)
        return KDT_OK;
    RangeArgs a = blank_args();
    a.a = d_lo;
    a.b = d_hi;
    a.Q = Q;
    a.offsets = d_offsets;
    a.out_ids = d_ids;
    a.vec_fill = fill_vectorizable(d_ids, nullptr);
    return run_range(t, 1, ACT_FILL, flags, a, (cudaStream_t)stream);
}

int kdt_offsets(const int32_t *d_counts, int64_t Q, int64_t *d_offsets, int64_t *h_total, void *stream)
{
    if (Q < 0 || !d_offsets || (Q > 0 && !d_counts))
        return set_error(KDT_EINVAL, "bad offsets arguments");
    cudaStream_t s = (cudaStream_t)stream;
    pool_setup_once();
    unsigned long long *out = (unsigned long long *)d_offsets;
    const int64_t n = Q + 1;
    Scratch sc(s);
    KDT_TRY(sc.alloc((scan_scratch_elems(n) + 1) * sizeof(unsigned long long)));
    KDT_LAUNCH counts_to_u64_kernel<<<grid_for(n), 256, 0, s>>>(d_counts, Q, out);
    KDT_TRY(exclusive_scan_u64(out, n, (unsigned long long *)sc.p, s));
    if (h_total) {
        KDT_CUDA(cudaMemcpyAsync(h_total, d_offsets + Q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KDT_CUDA(cudaStreamSynchronize(s));
    }
    return KDT_OK;
}

int kdt_tree_set_payload(kdt_tree *t, const float *d_payload, int C, void *stream)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (C < 1 || C > KDT_PAYLOAD_MAX_C || (t->N > 0 && !d_payload))
        return set_error(KDT_EINVAL, "payload: C must be in [1, %d] and the pointer non-NULL", KDT_PAYLOAD_MAX_C);
    cudaStream_t s = (cudaStream_t)stream;
    KDT_CUDA(cudaStreamSynchronize(s));
    cudaFree(t->payload);
    cudaFree(t->node_of);
    t->payload = nullptr;
    t->node_of = nullptr;
    t->payload_c = 0;
    const int64_t N = std::max<int64_t>(t->N, 1);
    KDT_CUDA(cudaMalloc(&t->payload, (size_t)N * C * sizeof(float)));
    KDT_CUDA(cudaMalloc(&t->node_of, (size_t)N * sizeof(int32_t)));
    if (t->N > 0) {
        const unsigned g = grid_for(t->N);
        switch (t->layout) {
        case 0: KDT_LAUNCH payload_permute_kernel<0><<<g, 256, 0, s>>>(t->nodes, t->ids, t->N, d_payload, C,
                                                                     t->payload, t->node_of); break;
        case 1: KDT_LAUNCH payload_permute_kernel<1><<<g, 256, 0, s>>>(t->nodes, t->ids, t->N, d_payload, C,
                                                                     t->payload, t->node_of); break;
        case 3: KDT_LAUNCH payload_permute_kernel<3><<<g, 256, 0, s>>>(t->nodes, t->ids, t->N, d_payload, C,
                                                                     t->payload, t->node_of); break;
        default: KDT_LAUNCH payload_permute_kernel<2><<<g, 256, 0, s>>>(t->nodes, t->ids, t->N, d_payload, C,
                                                                      t->payload, t->node_of); break;
        }
        KDT_CUDA(cudaGetLastError());
    }
    t->payload_c = C;
    return KDT_OK;
}

int kdt_radius_reduce(const kdt_tree *t, const float *d_q, int64_t Q, float radius, int flags, int mode, float *d_out,
                      int32_t *d_counts, void *stream)
{
    KDT_TRY(check_range(t, Q, d_q, nullptr, false, flags));
    if (flags & KDT_RANGE_VISITS)
        return set_error(KDT_EINVAL, "KDT_RANGE_VISITS applies to the count calls only");
    KDT_TRY(check_radius(radius));
    if (mode < KDT_REDUCE_SUM || mode > KDT_REDUCE_DENSITY)
        return set_error(KDT_EINVAL, "unknown reduction mode %d", mode);
    if (t->payload_c == 0)
        return set_error(KDT_EINVAL, "the tree has no payload (kdt_tree_set_payload)");
    if (Q > 0 && !d_out)
        return set_error(KDT_EINVAL, "NULL output");
    if (Q == 0)
        return KDT_OK;
    RangeArgs a = blank_args();
    a.a = d_q;
    a.Q = Q;
    a.r2 = radius * radius;
    a.counts = d_counts;
    a.payload = t->payload;
    a.C = t->payload_c;
    a.mode = mode;
    a.out = d_out;
    return run_range(t, 0, ACT_REDUCE, flags, a, (cudaStream_t)stream);
}

int kdt_knn_reduce(const kdt_tree *t, const float *d_q, int64_t Q, int k, float max_radius, int flags, int mode,
                   float *d_out, void *stream)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (mode < KDT_REDUCE_SUM || mode > KDT_REDUCE_DENSITY)
        return set_error(KDT_EINVAL, "unknown reduction mode %d", mode);
    if (t->payload_c == 0)
        return set_error(KDT_EINVAL, "the tree has no payload (kdt_tree_set_payload)");
    if (k < 1 || k > 64)
        return set_error(KDT_EINVAL, "k must be in [1, 64] (got %d)", k);
    if (Q < 0 || (Q > 0 && (!d_q || !d_out)))
        return set_error(KDT_EINVAL, "bad query count or NULL pointer");
    if (Q == 0)
        return KDT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    pool_setup_once();
    Scratch sc(s);
    KDT_TRY(sc.alloc(carve_size({(size_t)Q * k * 4, (size_t)Q * k * 4})));
    Carve c{(char *)sc.p};
    int32_t *ids = c.take<int32_t>((size_t)Q * k);
    float *d2 = c.take<float>((size_t)Q * k);
    KDT_TRY(kdt_knn(t, d_q, Q, k, max_radius, flags, ids, d2, stream));
    KDT_LAUNCH knn_reduce_kernel<<<grid_for(Q), 256, 0, s>>>(ids, d2, Q, k, t->node_of, t->payload, t->payload_c, mode,
                                                             d_out);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

}  // extern "C"
