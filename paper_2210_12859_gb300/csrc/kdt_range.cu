// Range queries: every point within a fixed radius of a query point (ball), or
// inside an axis-aligned box.  Sec. 3 notes that other query primitives only
// change the in-range test and what processNode does, and that a non-ordered
// traversal is a simplification of the ordered one; both queries use the
// unordered stack-free machine (left child first, a child is entered iff it
// can hold a point in range) with a fixed range instead of a shrinking one.
//
// Output protocol: a count pass writes each query's number of hits; the
// caller (or kdt_offsets) turns the counts into exclusive prefix offsets; a
// fill pass writes query q's hits to [offsets[q], offsets[q+1]) in traversal
// order.  A fill whose hits disagree with its offsets writes nothing beyond
// its slice and records the mismatch for kdt_status.
#include <algorithm>

#include "kdt_learned.cuh"
#include "kdt_query.cuh"

namespace kdt {
namespace {

constexpr int RANGE_THREADS = 128;

struct RangeArgs {
    const float4 *nodes;
    const int32_t *ids;
    int N, D;
    const float *a;  // ball: centres; box: lower corners   [Q][D]
    const float *b;  // box: upper corners                  [Q][D]
    int64_t Q;
    float r2;
    int32_t *counts;
    const int64_t *offsets;
    int32_t *out_ids;
    float *out_d2;
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

__device__ __forceinline__ int64_t claim(bool need, unsigned long long *counter)
{
    const unsigned m = __ballot_sync(0xffffffffu, need);
    int64_t slot = INT64_MAX;
    if (m) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader)
            base = atomicAdd(counter, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (need)
            slot = (int64_t)(base + __popc(m & lane_mask_lt()));
    }
    return slot;
}

// KIND 0: ball of squared radius r2 around a[q]; KIND 1: box [a[q], b[q]].
template <int LAYOUT, int KIND, bool FILL>
__global__ void __launch_bounds__(RANGE_THREADS) range_kernel(const RangeArgs a)
{
    constexpr int NC = LayoutTraits<LAYOUT>::NC;
    int64_t qi = -1;
    bool exhausted = false;
    float lo[NC], hi[NC];
    int curr = 0, prev = -1, dim = 0;
    uint32_t steps = 0;
    int64_t count = 0, base = 0, limit = 0;
    const uint32_t cap = 3u * (uint32_t)a.N + 3u;
    for (;;) {
        const bool need = qi < 0 && !exhausted;
        const int64_t slot = claim(need, a.counter);
        if (need) {
            if (slot < a.Q) {
                qi = slot;
                load_query<LAYOUT>(a.a, qi, a.D, lo);
                if (KIND == 1)
                    load_query<LAYOUT>(a.b, qi, a.D, hi);
                curr = 0;
                prev = -1;
                dim = 0;
                steps = 0;
                count = 0;
                if (FILL) {
                    base = a.offsets[qi];
                    limit = a.offsets[qi + 1] - base;
                }
            } else {
                exhausted = true;
            }
        }
        if (__all_sync(0xffffffffu, qi < 0))
            break;
        if (qi < 0)
            continue;
        bool done = false;
        for (int s = 0; s < STEPS_PER_CLAIM && !done; ++s) {
            if (++steps > cap) {
                atomicOr(a.err, ERR_TRAVERSAL);
                done = true;
                break;
            }
            const NodeVal<LAYOUT> nd = fetch<LAYOUT, false>(a.nodes, nullptr, 0, curr);
            const bool from_parent = prev < curr;
            if (from_parent) {
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
                if (hit) {
                    if (FILL && count < limit) {
                        a.out_ids[base + count] = (int32_t)node_id<LAYOUT>(nd, a.ids, curr);
                        if (KIND == 0 && a.out_d2)
                            a.out_d2[base + count] = d2;
                    }
                    ++count;
                }
            }
            const int sdim = split_dim_of<LAYOUT>(nd, dim);
            const float split = select_dim<NC>(nd.c, sdim);
            bool left_ok, right_ok;
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
            const int lc = 2 * curr + 1, rc = lc + 1;
            const int parent = (curr - 1) >> 1;
            left_ok = left_ok && lc < a.N;
            right_ok = right_ok && rc < a.N;
            int next;
            if (from_parent)
                next = left_ok ? lc : (right_ok ? rc : parent);
            else if (prev == lc)
                next = right_ok ? rc : parent;
            else
                next = parent;
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
        if (FILL) {
            if (count != limit)
                atomicOr(a.err, ERR_RANGE);
        } else {
            a.counts[qi] = (int32_t)count;
        }
        qi = -1;
    }
}

template <int LAYOUT>
int launch_range_layout(int kind, bool fill, const RangeArgs &a, cudaStream_t s)
{
    const void *fn;
    if (kind == 0)
        fn = fill ? (const void *)range_kernel<LAYOUT, 0, true> : (const void *)range_kernel<LAYOUT, 0, false>;
    else
        fn = fill ? (const void *)range_kernel<LAYOUT, 1, true> : (const void *)range_kernel<LAYOUT, 1, false>;
    const int grid = grid_for_kernel(fn, RANGE_THREADS, 0);
    KDT_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s));
    if (kind == 0 && fill)
        KDT_LAUNCH range_kernel<LAYOUT, 0, true><<<grid, RANGE_THREADS, 0, s>>>(a);
    else if (kind == 0)
        KDT_LAUNCH range_kernel<LAYOUT, 0, false><<<grid, RANGE_THREADS, 0, s>>>(a);
    else if (fill)
        KDT_LAUNCH range_kernel<LAYOUT, 1, true><<<grid, RANGE_THREADS, 0, s>>>(a);
    else
        KDT_LAUNCH range_kernel<LAYOUT, 1, false><<<grid, RANGE_THREADS, 0, s>>>(a);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

int run_range(const kdt_tree *t, int kind, bool fill, const float *qa, const float *qb, int64_t Q, float r2,
              int32_t *counts, const int64_t *offsets, int32_t *out_ids, float *out_d2, cudaStream_t s)
{
    unsigned long long *counter = nullptr;
    KDT_CUDA(cudaMallocAsync(&counter, 256, s));
    RangeArgs a{t->nodes, t->ids, (int)t->N, t->D, qa, qb, Q, r2, counts, offsets, out_ids, out_d2, t->err, counter};
    int rc;
    switch (t->layout) {
    case 0: rc = launch_range_layout<0>(kind, fill, a, s); break;
    case 1: rc = launch_range_layout<1>(kind, fill, a, s); break;
    case 3: rc = launch_range_layout<3>(kind, fill, a, s); break;
    default: rc = launch_range_layout<2>(kind, fill, a, s); break;
    }
    cudaFreeAsync(counter, s);
    return rc;
}

__global__ void counts_to_u64_kernel(const int32_t *__restrict__ counts, int64_t Q, unsigned long long *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= Q; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = i < Q ? (unsigned long long)(counts[i] > 0 ? counts[i] : 0) : 0ull;
}

int check_range(const kdt_tree *t, int64_t Q, const void *a, const void *b, bool need_b)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (Q < 0 || Q >= ((int64_t)1 << 32))
        return set_error(KDT_EINVAL, "Q must be in [0, 2^32)");
    if (Q > 0 && (!a || (need_b && !b)))
        return set_error(KDT_EINVAL, "NULL query pointer");
    return KDT_OK;
}

}  // namespace
}  // namespace kdt

using namespace kdt;

extern "C" {

int kdt_radius_count(const kdt_tree *t, const float *d_q, int64_t Q, float radius, int32_t *d_counts, void *stream)
{
    KDT_TRY(check_range(t, Q, d_q, nullptr, false));
    if (!(radius >= 0.f) || (Q > 0 && !d_counts))
        return set_error(KDT_EINVAL, "bad radius or NULL counts");
    if (Q == 0)
        return KDT_OK;
    return run_range(t, 0, false, d_q, nullptr, Q, radius * radius, d_counts, nullptr, nullptr, nullptr,
                     (cudaStream_t)stream);
}

int kdt_radius_fill(const kdt_tree *t, const float *d_q, int64_t Q, float radius, const int64_t *d_offsets,
                    int32_t *d_ids, float *d_d2, void *stream)
{
    KDT_TRY(check_range(t, Q, d_q, nullptr, false));
    if (!(radius >= 0.f) || (Q > 0 && (!d_offsets || !d_ids)))
        return set_error(KDT_EINVAL, "bad radius or NULL offsets / ids");
    if (Q == 0)
        return KDT_OK;
    return run_range(t, 0, true, d_q, nullptr, Q, radius * radius, nullptr, d_offsets, d_ids, d_d2,
                     (cudaStream_t)stream);
}

int kdt_box_count(const kdt_tree *t, const float *d_lo, const float *d_hi, int64_t Q, int32_t *d_counts,
                  void *stream)
{
    KDT_TRY(check_range(t, Q, d_lo, d_hi, true));
    if (Q > 0 && !d_counts)
        return set_error(KDT_EINVAL, "NULL counts");
    if (Q == 0)
        return KDT_OK;
    return run_range(t, 1, false, d_lo, d_hi, Q, 0.f, d_counts, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

int kdt_box_fill(const kdt_tree *t, const float *d_lo, const float *d_hi, int64_t Q, const int64_t *d_offsets,
                 int32_t *d_ids, void *stream)
{
    KDT_TRY(check_range(t, Q, d_lo, d_hi, true));
    if (Q > 0 && (!d_offsets || !d_ids))
        return set_error(KDT_EINVAL, "NULL offsets / ids");
    if (Q == 0)
        return KDT_OK;
    return run_range(t, 1, true, d_lo, d_hi, Q, 0.f, nullptr, d_offsets, d_ids, nullptr, (cudaStream_t)stream);
}

int kdt_offsets(const int32_t *d_counts, int64_t Q, int64_t *d_offsets, int64_t *h_total, void *stream)
{
    if (Q < 0 || !d_offsets || (Q > 0 && !d_counts))
        return set_error(KDT_EINVAL, "bad offsets arguments");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *out = (unsigned long long *)d_offsets;
    const int64_t n = Q + 1;
    unsigned long long *scratch = nullptr;
    KDT_CUDA(cudaMallocAsync(&scratch, (scan_scratch_elems(n) + 1) * sizeof(unsigned long long), s));
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16));
    KDT_LAUNCH counts_to_u64_kernel<<<g, 256, 0, s>>>(d_counts, Q, out);
    int rc = exclusive_scan_u64(out, n, scratch, s);
    cudaFreeAsync(scratch, s);
    if (rc != KDT_OK)
        return rc;
    if (h_total) {
        KDT_CUDA(cudaMemcpyAsync(h_total, d_offsets + Q, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KDT_CUDA(cudaStreamSynchronize(s));
    }
    return KDT_OK;
}

}  // extern "C"
