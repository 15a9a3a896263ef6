// Query kernels, instantiated once per node layout by kdt_query_l{0,1,2}.cu.
#pragma once

#include <algorithm>
#include <type_traits>

#include "kdt_query.cuh"

namespace kdt {

// Single tree.  Persistent blocks stage the top levels once; every lane then
// runs queries back to back: when its query ends it claims the next one
// (persistent threads with replacement), so a lane never idles while a slow
// neighbour in its warp is still traversing, until the work runs out.
// Register-list kernels with k <= 8 are built for at least 6 resident blocks
// per SM (at most 85 registers a thread; without the bound the depth-2 kernel
// once took 82 registers and 5 blocks fit), the learned radius's bounded
// kernel included, so that it runs with the plain kernel's occupancy.  With
// the bottom subtrees handled as scalar keys the depth-2 kernel needs 64
// registers (8 blocks) and the depth-3 one 79, both without spills, so the
// bounds only guard against regressions.
//
// G > 1 (k > 16): a group of G lanes walks one query together and holds its
// k-best list spread over the group (GroupList, insertion by warp shuffles);
// the group's first lane claims the query for the group.
template <int LAYOUT, int K, bool ORDERED, int MODE, bool STAGE, int INLINE, bool RUNS = false, int G = 1>
__global__ void __launch_bounds__(K <= MAX_REG_K ? REG_THREADS : SMEM_THREADS, K <= 8 ? 6 : 1)
    knn_kernel(const QueryArgs a)
{
    constexpr int NC = LayoutTraits<LAYOUT>::NC;
    constexpr int NF = LayoutTraits<LAYOUT>::NF;
    using List = typename std::conditional<
        (G > 1), GroupList<(G > 1 ? K / G : 1), (G > 1 ? G : 2)>,
        typename std::conditional<(K <= MAX_REG_K), RegList<K <= MAX_REG_K ? K : 1>, SmemList>::type>::type;
    extern __shared__ float4 s_dyn[];
    float4 *s_nodes = s_dyn;
    if (STAGE) {
        stage_nodes<LAYOUT>(a.nodes, s_nodes, a.staged);
        __syncthreads();
    }
    const int64_t Qn = a.Q;
    // learned radius: the traversal-order slots below n_gate take the
    // proposal, the others the caller's radius
    const int64_t ngate = (MODE == MODE_BOUNDED && a.n_gate) ? (int64_t)*a.n_gate : INT64_MAX;
    bool gated = false;
    double ratio = 0.0;
    int64_t qi = -1;
    bool exhausted = false;
    float q[NC];
    float r2 = 0.f;
    int visits = 0;
    List list;
    if constexpr (K > MAX_REG_K && G == 1) {
        if (a.heap) {  // this thread's k entries, contiguous
            list.s = a.heap + ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * (size_t)a.k;
            list.stride = 1;
        } else {
            list.s = reinterpret_cast<unsigned long long *>(s_nodes + (size_t)a.staged * NF) + threadIdx.x;
            list.stride = blockDim.x;
        }
    }
    Walker<LAYOUT, ORDERED, INLINE> w;
    const int glane = (threadIdx.x & 31) % G;
    for (;;) {
        const bool need = qi < 0 && !exhausted;
        int64_t slot = claim_slot(need && glane == 0, a.counter);
        if constexpr (G > 1)
            slot = __shfl_sync(0xffffffffu, slot, (threadIdx.x & 31) - glane);
        if (need) {
            if (slot < Qn) {
                qi = a.perm ? (int64_t)a.perm[slot] : slot;
                gated = MODE == MODE_BOUNDED && slot < ngate;
                r2 = gated ? a.r2q[qi] : a.r2;
                load_query<LAYOUT>(a.queries, qi, a.D, q);
                list.init(a.k, r2);
                w.start();
                visits = 0;
            } else {
                exhausted = true;
            }
        }
        if (__all_sync(0xffffffffu, qi < 0))
            break;
        if (qi < 0)
            continue;
        // up to claim_steps steps between claims: amortises the warp vote
        bool overflow = false;
        bool fin = false;
        for (int s = 0; s < a.claim_steps && !fin; ++s)
            fin = w.template step<STAGE, RUNS>(a.nodes, a.ids, s_nodes, a.staged, a.N, a.D, q, list, visits,
                                               overflow, a.light_run);
        if (!fin && w.steps > (a.step_cap ? a.step_cap : 3u * (uint32_t)a.N + 3u)) {
            overflow = true;
            fin = true;
        }
        if (!fin)
            continue;
        // query finished
        if (overflow)
            atomicOr(a.err, ERR_TRAVERSAL);
        const bool full = list.full(a.k);
        // a bounded query is exact when its list is full (every point outside
        // the proposed radius is farther than all k held) or when the proposal
        // did not shrink the caller's radius; the others restart at once in the
        // same lane with the caller's radius (the plain traversal): no second
        // launch, and the re-run stays next to its Morton neighbours
        const bool fallback = MODE == MODE_BOUNDED && !(full || r2 == a.r2);
        if (fallback) {
            atomicAdd(a.fb_count, 1ull);
            gated = false;
            r2 = a.r2;
            list.init(a.k, r2);
            w.start();
            continue;
        }
        if (MODE != MODE_VISITS && a.out_ids)
            list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
        if (MODE == MODE_VISITS || (MODE == MODE_BOUNDED && a.visits))
            a.visits[qi] = overflow ? -1 : visits;
        if (MODE == MODE_BOUNDED && gated && full && list.cull() > 0.f && r2 < __int_as_float(0x7f800000))
            ratio += sqrt((double)r2 / (double)list.cull());
        qi = -1;
    }
    if (MODE == MODE_BOUNDED) {
        for (int o = 16; o > 0; o >>= 1)
            ratio += __shfl_down_sync(0xffffffffu, ratio, o);
        if ((threadIdx.x & 31) == 0 && ratio != 0.0)
            atomicAdd(a.ratio_sum, ratio);
    }
}

// Forest: a lane's query finds its tree by binary search over the query
// offsets; no shared-memory staging (neighbouring lanes may walk different
// trees).  Same lane-refill scheme as knn_kernel.
template <int LAYOUT, int K, bool ORDERED, int INLINE, bool RUNS = false>
__global__ void __launch_bounds__(K <= MAX_REG_K ? REG_THREADS : SMEM_THREADS)
    knn_forest_kernel(const QueryArgs a)
{
    constexpr int NC = LayoutTraits<LAYOUT>::NC;
    constexpr int NF = LayoutTraits<LAYOUT>::NF;
    using List = typename std::conditional<(K <= MAX_REG_K), RegList<K <= MAX_REG_K ? K : 1>, SmemList>::type;
    extern __shared__ float4 s_dyn[];
    int64_t qi = -1;
    bool exhausted = false;
    float q[NC];
    int visits = 0;
    int N = 0;
    const float4 *nodes = nullptr;
    const int32_t *ids = nullptr;
    List list;
    if constexpr (K > MAX_REG_K) {
        list.s = reinterpret_cast<unsigned long long *>(s_dyn) + threadIdx.x;
        list.stride = blockDim.x;
    }
    Walker<LAYOUT, ORDERED, INLINE> w;
    for (;;) {
        const bool need = qi < 0 && !exhausted;
        const int64_t slot = claim_slot(need, a.counter);
        if (need) {
            if (slot < a.Q) {
                qi = a.perm ? (int64_t)a.perm[slot] : slot;
                int lo = 0, hi = a.T - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.q_off[mid] <= qi)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                const int64_t nb = a.node_off[lo];
                N = (int)(a.node_off[lo + 1] - nb);
                nodes = a.nodes + nb * NF;
                ids = a.ids ? a.ids + nb : nullptr;
                load_query<LAYOUT>(a.queries, qi, a.D, q);
                list.init(a.k, a.r2);
                w.start();
                visits = 0;
                if (N == 0) {  // empty cloud: empty result
                    list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
                    qi = -1;
                }
            } else {
                exhausted = true;
            }
        }
        if (__all_sync(0xffffffffu, qi < 0))
            break;
        if (qi < 0)
            continue;
        bool overflow = false;
        bool fin = false;
        for (int s = 0; s < a.claim_steps && !fin; ++s)
            fin = w.template step<false, RUNS>(nodes, ids, nullptr, 0, N, a.D, q, list, visits, overflow, a.light_run);
        if (!fin && w.steps > 3u * (uint32_t)N + 3u) {
            overflow = true;
            fin = true;
        }
        if (!fin)
            continue;
        if (overflow)
            atomicOr(a.err, ERR_TRAVERSAL);
        list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
        qi = -1;
    }
}

template <typename Kern>
inline int launch_kernel(Kern fn, int threads, size_t smem, const QueryArgs &a, cudaStream_t s)
{
    if (smem > 48 * 1024)
        KDT_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = grid_for_kernel((const void *)fn, threads, smem);
    if (a.heap && (int64_t)grid * threads > a.heap_threads)
        grid = (int)std::max<int64_t>(1, a.heap_threads / threads);
    KDT_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s));
    KDT_LAUNCH fn<<<grid, threads, smem, s>>>(a);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

template <int LAYOUT, int K, bool STAGE, int INLINE>
inline int launch_mode(const QueryArgs &a, bool ordered, int mode, int threads, size_t smem, cudaStream_t s)
{
    switch (mode) {
    case MODE_VISITS:
        if (ordered)
            return launch_kernel(knn_kernel<LAYOUT, K, true, MODE_VISITS, STAGE, INLINE>, threads, smem, a, s);
        return launch_kernel(knn_kernel<LAYOUT, K, false, MODE_VISITS, STAGE, INLINE>, threads, smem, a, s);
    case MODE_BOUNDED:
        if constexpr (LAYOUT == 0 || LAYOUT == 3) {
            // light runs as for the plain traversal (the same tuned value)
            if constexpr (!STAGE) {
                if (a.light_run > 1) {
                    if (ordered)
                        return launch_kernel(knn_kernel<LAYOUT, K, true, MODE_BOUNDED, false, INLINE, true>, threads,
                                             smem, a, s);
                    return launch_kernel(knn_kernel<LAYOUT, K, false, MODE_BOUNDED, false, INLINE, true>, threads,
                                         smem, a, s);
                }
            }
            if (ordered)
                return launch_kernel(knn_kernel<LAYOUT, K, true, MODE_BOUNDED, STAGE, INLINE>, threads, smem, a, s);
            return launch_kernel(knn_kernel<LAYOUT, K, false, MODE_BOUNDED, STAGE, INLINE>, threads, smem, a, s);
        } else {
            return set_error(KDT_EINVAL, "the learned radius path needs D <= 3");
        }
    default:
        // light runs (tuned for short queries) have their own instantiation
        // so that the default kernel keeps its single-step code
        if constexpr (!STAGE) {
            if (a.light_run > 1) {
                if (ordered)
                    return launch_kernel(knn_kernel<LAYOUT, K, true, MODE_RESULTS, false, INLINE, true>, threads,
                                         smem, a, s);
                return launch_kernel(knn_kernel<LAYOUT, K, false, MODE_RESULTS, false, INLINE, true>, threads, smem,
                                     a, s);
            }
        }
        if (ordered)
            return launch_kernel(knn_kernel<LAYOUT, K, true, MODE_RESULTS, STAGE, INLINE>, threads, smem, a, s);
        return launch_kernel(knn_kernel<LAYOUT, K, false, MODE_RESULTS, STAGE, INLINE>, threads, smem, a, s);
    }
}

template <int LAYOUT, int K>
inline int launch_k(const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s)
{
    constexpr int NF = LayoutTraits<LAYOUT>::NF;
    const int threads = batched && a.threads > 0 ? a.threads : (K <= MAX_REG_K ? REG_THREADS : SMEM_THREADS);
    size_t list_bytes = (K <= MAX_REG_K || (a.heap && !batched)) ? 0 : (size_t)a.k * threads * 8;
    if (batched) {
        if constexpr (LAYOUT == 3)
            return set_error(KDT_EINVAL, "forests store no per-node split dimensions");
        const bool runs = a.light_run > 1;
        if (a.inline_depth == 1) {
            if (runs)
                return ordered ? launch_kernel(knn_forest_kernel<LAYOUT, K, true, 1, true>, threads, list_bytes, a, s)
                               : launch_kernel(knn_forest_kernel<LAYOUT, K, false, 1, true>, threads, list_bytes, a, s);
            return ordered ? launch_kernel(knn_forest_kernel<LAYOUT, K, true, 1>, threads, list_bytes, a, s)
                           : launch_kernel(knn_forest_kernel<LAYOUT, K, false, 1>, threads, list_bytes, a, s);
        }
        if (runs)
            return ordered ? launch_kernel(knn_forest_kernel<LAYOUT, K, true, 2, true>, threads, list_bytes, a, s)
                           : launch_kernel(knn_forest_kernel<LAYOUT, K, false, 2, true>, threads, list_bytes, a, s);
        return ordered ? launch_kernel(knn_forest_kernel<LAYOUT, K, true, 2>, threads, list_bytes, a, s)
                       : launch_kernel(knn_forest_kernel<LAYOUT, K, false, 2>, threads, list_bytes, a, s);
    }
    if constexpr (K > MAX_REG_K) {
        // k-best lists spread over groups of lanes: plain results and visit counts
        if (a.group > 1 && (mode == MODE_RESULTS || mode == MODE_VISITS)) {
            const bool vis = mode == MODE_VISITS;
            const int d = a.inline_depth == 3 ? 3 : 2;
#define KDT_GROUP_LAUNCH(GG, DD)                                                                                  \
    return ordered ? (vis ? launch_kernel(knn_kernel<LAYOUT, K, true, MODE_VISITS, false, DD, false, GG>, threads, 0, a, s)   \
                          : launch_kernel(knn_kernel<LAYOUT, K, true, MODE_RESULTS, false, DD, false, GG>, threads, 0, a, s)) \
                   : (vis ? launch_kernel(knn_kernel<LAYOUT, K, false, MODE_VISITS, false, DD, false, GG>, threads, 0, a, s)  \
                          : launch_kernel(knn_kernel<LAYOUT, K, false, MODE_RESULTS, false, DD, false, GG>, threads, 0, a, s))
            if (a.group == 8) {
                if (d == 3)
                    KDT_GROUP_LAUNCH(8, 3);
                KDT_GROUP_LAUNCH(8, 2);
            }
            if (d == 3)
                KDT_GROUP_LAUNCH(4, 3);
            KDT_GROUP_LAUNCH(4, 2);
#undef KDT_GROUP_LAUNCH
        }
    }
    size_t smem = (size_t)a.staged * NF * 16 + list_bytes;
    // staging is paired with depth-2 inlining only (both serve long queries)
    if (a.staged > 0)
        return launch_mode<LAYOUT, K, true, 2>(a, ordered, mode, threads, smem, s);
    if (a.inline_depth == 1)
        return launch_mode<LAYOUT, K, false, 1>(a, ordered, mode, threads, smem, s);
    if (a.inline_depth == 3)
        return launch_mode<LAYOUT, K, false, 3>(a, ordered, mode, threads, smem, s);
    if (a.inline_depth == 4)
        return launch_mode<LAYOUT, K, false, 4>(a, ordered, mode, threads, smem, s);
    return launch_mode<LAYOUT, K, false, 2>(a, ordered, mode, threads, smem, s);
}

template <int LAYOUT>
inline int launch_query_impl(const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s)
{
    if (a.k <= 1)
        return launch_k<LAYOUT, 1>(a, ordered, mode, batched, s);
    if (a.k <= 2)
        return launch_k<LAYOUT, 2>(a, ordered, mode, batched, s);
    if (a.k <= 4)
        return launch_k<LAYOUT, 4>(a, ordered, mode, batched, s);
    if (a.k <= 8)
        return launch_k<LAYOUT, 8>(a, ordered, mode, batched, s);
    if (a.k <= 16)
        return launch_k<LAYOUT, 16>(a, ordered, mode, batched, s);
    return launch_k<LAYOUT, 64>(a, ordered, mode, batched, s);
}

}  // namespace kdt
