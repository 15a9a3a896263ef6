// Query kernels, instantiated once per node layout by kdt_query_l{0,1,2}.cu.
#pragma once

#include "kdt_query.cuh"

namespace kdt {

// Single tree.  Persistent blocks stage the top levels once, then every warp
// repeatedly claims the next 32 query slots from a global counter, so the
// slow lanes of a warp hold up only that warp and the tail stays short.
template <int LAYOUT, int K, bool ORDERED, bool COUNT>
__global__ void __launch_bounds__(K <= MAX_REG_K ? REG_THREADS : SMEM_THREADS)
    knn_kernel(const QueryArgs a)
{
    constexpr int NC = LayoutTraits<LAYOUT>::NC;
    constexpr int NF = LayoutTraits<LAYOUT>::NF;
    extern __shared__ float4 s_dyn[];
    float4 *s_nodes = s_dyn;
    stage_nodes<LAYOUT>(a.nodes, s_nodes, a.staged);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0)
            b = atomicAdd(a.counter, 32ull);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= (unsigned long long)a.Q)
            break;
        const int64_t i = (int64_t)b + lane;
        if (i >= a.Q)
            continue;
        const int64_t qi = a.perm ? (int64_t)a.perm[i] : i;
        float q[NC];
        load_query<LAYOUT>(a.queries, qi, a.D, q);
        int v;
        if constexpr (K <= MAX_REG_K) {
            RegList<K> list;
            list.init(a.k, a.r2);
            v = traverse<LAYOUT, ORDERED>(a.nodes, a.ids, s_nodes, a.staged, a.N, a.D, q, list);
            if (!COUNT)
                list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
        } else {
            SmemList list;
            list.s = reinterpret_cast<unsigned long long *>(s_nodes + (size_t)a.staged * NF) + threadIdx.x;
            list.stride = blockDim.x;
            list.init(a.k, a.r2);
            v = traverse<LAYOUT, ORDERED>(a.nodes, a.ids, s_nodes, a.staged, a.N, a.D, q, list);
            if (!COUNT)
                list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
        }
        if (v < 0)
            atomicOr(a.err, ERR_TRAVERSAL);
        if (COUNT)
            a.visits[qi] = v;
    }
}

// Forest: every query slot finds its tree by binary search over the query
// offsets; no shared-memory staging (trees differ between neighbouring slots).
template <int LAYOUT, int K, bool ORDERED>
__global__ void __launch_bounds__(K <= MAX_REG_K ? REG_THREADS : SMEM_THREADS)
    knn_forest_kernel(const QueryArgs a)
{
    constexpr int NC = LayoutTraits<LAYOUT>::NC;
    constexpr int NF = LayoutTraits<LAYOUT>::NF;
    extern __shared__ float4 s_dyn[];
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0)
            b = atomicAdd(a.counter, 32ull);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= (unsigned long long)a.Q)
            break;
        const int64_t i = (int64_t)b + lane;
        if (i >= a.Q)
            continue;
        const int64_t qi = a.perm ? (int64_t)a.perm[i] : i;
        int lo = 0, hi = a.T - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (a.q_off[mid] <= qi)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t nb = a.node_off[lo];
        const int N = (int)(a.node_off[lo + 1] - nb);
        float q[NC];
        load_query<LAYOUT>(a.queries, qi, a.D, q);
        const float4 *nodes = a.nodes + nb * NF;
        const int32_t *ids = a.ids ? a.ids + nb : nullptr;
        int v = 0;
        if constexpr (K <= MAX_REG_K) {
            RegList<K> list;
            list.init(a.k, a.r2);
            if (N > 0)
                v = traverse<LAYOUT, ORDERED>(nodes, ids, nullptr, 0, N, a.D, q, list);
            list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
        } else {
            SmemList list;
            list.s = reinterpret_cast<unsigned long long *>(s_dyn) + threadIdx.x;
            list.stride = blockDim.x;
            list.init(a.k, a.r2);
            if (N > 0)
                v = traverse<LAYOUT, ORDERED>(nodes, ids, nullptr, 0, N, a.D, q, list);
            list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
        }
        if (v < 0)
            atomicOr(a.err, ERR_TRAVERSAL);
    }
}

template <typename Kern>
inline int launch_kernel(Kern fn, int threads, size_t smem, const QueryArgs &a, cudaStream_t s)
{
    if (smem > 48 * 1024)
        KDT_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = grid_for_kernel((const void *)fn, threads, smem);
    KDT_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s));
    fn<<<grid, threads, smem, s>>>(a);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

template <int LAYOUT, int K>
inline int launch_k(const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s)
{
    constexpr int NF = LayoutTraits<LAYOUT>::NF;
    const int threads = K <= MAX_REG_K ? REG_THREADS : SMEM_THREADS;
    size_t list_bytes = K <= MAX_REG_K ? 0 : (size_t)a.k * threads * 8;
    if (batched) {
        if (ordered)
            return launch_kernel(knn_forest_kernel<LAYOUT, K, true>, threads, list_bytes, a, s);
        return launch_kernel(knn_forest_kernel<LAYOUT, K, false>, threads, list_bytes, a, s);
    }
    size_t smem = (size_t)a.staged * NF * 16 + list_bytes;
    if (mode == 1) {
        if (ordered)
            return launch_kernel(knn_kernel<LAYOUT, K, true, true>, threads, smem, a, s);
        return launch_kernel(knn_kernel<LAYOUT, K, false, true>, threads, smem, a, s);
    }
    if (ordered)
        return launch_kernel(knn_kernel<LAYOUT, K, true, false>, threads, smem, a, s);
    return launch_kernel(knn_kernel<LAYOUT, K, false, false>, threads, smem, a, s);
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
