// Query kernels, instantiated once per node layout by kdt_query_l{0,1,2}.cu.
#pragma once

#include "kdt_query.cuh"

namespace kdt {

// Single tree.  Persistent blocks stage the top levels once, then every warp
// repeatedly claims the next 32 query slots from a global counter, so the
// slow lanes of a warp hold up only that warp and the tail stays short.
template <int LAYOUT, int K, bool ORDERED, int MODE>
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
    const int64_t Qn = MODE == MODE_FALLBACK ? (int64_t)*a.fb_count : a.Q;
    double ratio = 0.0;
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0)
            b = atomicAdd(a.counter, 32ull);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= (unsigned long long)Qn)
            break;
        const int64_t i = (int64_t)b + lane;
        bool fallback = false;
        int64_t qi = 0;
        if (i < Qn) {
            if (MODE == MODE_FALLBACK)
                qi = a.fb_list[i];
            else
                qi = a.perm ? (int64_t)a.perm[i] : i;
            const float r2 = MODE == MODE_BOUNDED ? a.r2q[qi] : a.r2;
            float q[NC];
            load_query<LAYOUT>(a.queries, qi, a.D, q);
            int v;
            bool full;
            float worst;
            if constexpr (K <= MAX_REG_K) {
                RegList<K> list;
                list.init(a.k, r2);
                v = traverse<LAYOUT, ORDERED>(a.nodes, a.ids, s_nodes, a.staged, a.N, a.D, q, list);
                full = list.full(a.k);
                worst = list.cull();
                fallback = MODE == MODE_BOUNDED && !(full || r2 == a.r2);
                if (MODE != MODE_VISITS && !fallback && a.out_ids)
                    list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
            } else {
                SmemList list;
                list.s = reinterpret_cast<unsigned long long *>(s_nodes + (size_t)a.staged * NF) + threadIdx.x;
                list.stride = blockDim.x;
                list.init(a.k, r2);
                v = traverse<LAYOUT, ORDERED>(a.nodes, a.ids, s_nodes, a.staged, a.N, a.D, q, list);
                full = list.full(a.k);
                worst = list.cull();
                fallback = MODE == MODE_BOUNDED && !(full || r2 == a.r2);
                if (MODE != MODE_VISITS && !fallback && a.out_ids)
                    list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
            }
            if (v < 0)
                atomicOr(a.err, ERR_TRAVERSAL);
            if (MODE == MODE_VISITS || (MODE == MODE_BOUNDED && a.visits))
                a.visits[qi] = v;
            if (MODE == MODE_FALLBACK && a.visits)
                a.visits[qi] += v;
            // a query is exact when its list is full (every point outside the
            // proposed radius is farther than all k held) or when the proposal
            // did not shrink the caller's radius; for the others the k-best set
            // may lie beyond the proposal and they are re-run
            if (MODE == MODE_BOUNDED && !fallback && full && worst > 0.f && r2 < __int_as_float(0x7f800000))
                ratio += sqrt((double)r2 / (double)worst);
        }
        if (MODE == MODE_BOUNDED) {
            // warp-aggregated append of the queries to re-run (all lanes here)
            const unsigned m = __ballot_sync(0xffffffffu, fallback);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long base = 0;
                if (lane == leader)
                    base = atomicAdd(a.fb_count, (unsigned long long)__popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (fallback)
                    a.fb_list[base + __popc(m & ((1u << lane) - 1))] = (uint32_t)qi;
            }
        }
    }
    if (MODE == MODE_BOUNDED) {
        for (int o = 16; o > 0; o >>= 1)
            ratio += __shfl_down_sync(0xffffffffu, ratio, o);
        if (lane == 0 && ratio != 0.0)
            atomicAdd(a.ratio_sum, ratio);
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
    KDT_LAUNCH fn<<<grid, threads, smem, s>>>(a);
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
    switch (mode) {
    case MODE_VISITS:
        if (ordered)
            return launch_kernel(knn_kernel<LAYOUT, K, true, MODE_VISITS>, threads, smem, a, s);
        return launch_kernel(knn_kernel<LAYOUT, K, false, MODE_VISITS>, threads, smem, a, s);
    case MODE_BOUNDED:
    case MODE_FALLBACK:
        if constexpr (LAYOUT == 0) {
            if (mode == MODE_BOUNDED) {
                if (ordered)
                    return launch_kernel(knn_kernel<LAYOUT, K, true, MODE_BOUNDED>, threads, smem, a, s);
                return launch_kernel(knn_kernel<LAYOUT, K, false, MODE_BOUNDED>, threads, smem, a, s);
            }
            if (ordered)
                return launch_kernel(knn_kernel<LAYOUT, K, true, MODE_FALLBACK>, threads, smem, a, s);
            return launch_kernel(knn_kernel<LAYOUT, K, false, MODE_FALLBACK>, threads, smem, a, s);
        } else {
            return set_error(KDT_EINVAL, "the learned radius path needs D <= 3");
        }
    default:
        if (ordered)
            return launch_kernel(knn_kernel<LAYOUT, K, true, MODE_RESULTS>, threads, smem, a, s);
        return launch_kernel(knn_kernel<LAYOUT, K, false, MODE_RESULTS>, threads, smem, a, s);
    }
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
