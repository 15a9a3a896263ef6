// Device-wide primitives used by the builder and the query reordering:
// an exclusive prefix sum over u32 and a stable LSD radix sort of
// (u32 key, u32 value) pairs, 8 bits per pass.
//
// Both are three-phase (per-tile reduce, scan of tile totals, per-tile scan
// and scatter) so that every pass is a plain streaming read of its input.
#include <algorithm>

#include "kdt_internal.cuh"

namespace kdt {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
static_assert(SCAN_TILE == SCAN_TILE_ELEMS, "scan tile and the scratch-size formula disagree");

constexpr int RADIX_THREADS = 256;
constexpr int RADIX_ITEMS = 8;
constexpr int RADIX_TILE = RADIX_THREADS * RADIX_ITEMS;
static_assert(RADIX_TILE == RADIX_TILE_KEYS, "radix tile and the scratch-size formula disagree");
constexpr int RADIX_WARPS = RADIX_THREADS / 32;

template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += u;
    }
    return v;
}

// exclusive block scan of one value per thread; returns the exclusive prefix
// and writes the block total to *total (all threads)
template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T *s_warp, T *total)
{
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    T inc = warp_inclusive_sum(v);
    if (lane == 31)
        s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        T x = lane < nw ? s_warp[lane] : T(0);
        T xi = warp_inclusive_sum(x);
        if (lane < nw)
            s_warp[lane] = xi - x;
        if (lane == nw - 1)
            s_warp[32] = xi;
    }
    __syncthreads();
    T r = s_warp[w] + inc - v;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(const T *__restrict__ data, int64_t n,
                                                                     T *__restrict__ partials)
{
    __shared__ T s_warp[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n)
            sum += data[i];
    }
    T total;
    block_exclusive_sum(sum, s_warp, &total);
    if (threadIdx.x == 0)
        partials[blockIdx.x] = total;
}

// single block: exclusive scan of the tile totals, in chunks
template <typename T>
__global__ void __launch_bounds__(1024) scan_partials_kernel(T *__restrict__ partials, int64_t np)
{
    __shared__ T s_warp[33];
    T carry = 0;
    for (int64_t base = 0; base < np; base += 1024) {
        int64_t i = base + threadIdx.x;
        T v = i < np ? partials[i] : T(0);
        T total;
        T ex = block_exclusive_sum(v, s_warp, &total);
        if (i < np)
            partials[i] = carry + ex;
        carry += total;
    }
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_downsweep_kernel(T *__restrict__ data, int64_t n,
                                                                        const T *__restrict__ partials)
{
    __shared__ T s_warp[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + j;
        v[j] = i < n ? data[i] : T(0);
        sum += v[j];
    }
    T total;
    T run = block_exclusive_sum(sum, s_warp, &total) + partials[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + j;
        if (i < n)
            data[i] = run;
        run += v[j];
    }
}

template <typename T>
int exclusive_scan_t(T *data, int64_t n, T *scratch, cudaStream_t s)
{
    if (n <= 0)
        return KDT_OK;
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    KDT_LAUNCH scan_reduce_kernel<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(data, n, scratch);
    KDT_LAUNCH scan_partials_kernel<T><<<1, 1024, 0, s>>>(scratch, tiles);
    KDT_LAUNCH scan_downsweep_kernel<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(data, n, scratch);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

// ---- radix sort

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(RADIX_THREADS) radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t n,
                                                                     int shift, int64_t tiles,
                                                                     uint32_t *__restrict__ hist)
{
    __shared__ uint32_t s_cnt[256];
    s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RADIX_TILE;
#pragma unroll
    for (int j = 0; j < RADIX_ITEMS; ++j) {
        int64_t i = base + (int64_t)j * RADIX_THREADS + threadIdx.x;
        uint32_t d = i < n ? (keys[i] >> shift) & 255u : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (d < 256 && (peers & lanemask_lt()) == 0)
            atomicAdd(&s_cnt[d], __popc(peers));
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = s_cnt[threadIdx.x];
}

// Stable scatter.  Items of a tile are taken in rounds j = 0..RADIX_ITEMS-1,
// round j holding elements base + j*256 + tid, so index order is round-major,
// then warp, then lane.  Within a round every warp groups equal digits with
// match_any; per-digit prefix counts over the warps (plus the counts of earlier
// rounds) give each element its rank among equal digits of the tile.
__global__ void __launch_bounds__(RADIX_THREADS) radix_scatter_kernel(
    const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n, int shift, int64_t tiles,
    const uint32_t *__restrict__ offsets, uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out)
{
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_warp[RADIX_WARPS][256];
    const int tid = threadIdx.x;
    const int w = tid >> 5;
    s_off[tid] = offsets[(int64_t)tid * tiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RADIX_TILE;
    const uint32_t lt = lanemask_lt();
    for (int j = 0; j < RADIX_ITEMS; ++j) {
#pragma unroll
        for (int w2 = 0; w2 < RADIX_WARPS; ++w2)
            s_warp[w2][tid] = 0;
        int64_t i = base + (int64_t)j * RADIX_THREADS + tid;
        bool valid = i < n;
        uint32_t key = valid ? keys[i] : 0;
        uint32_t val = valid ? vals[i] : 0;
        uint32_t d = valid ? (key >> shift) & 255u : 256u;
        __syncthreads();
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0)
            s_warp[w][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = s_off[tid];
#pragma unroll
            for (int w2 = 0; w2 < RADIX_WARPS; ++w2) {
                uint32_t c = s_warp[w2][tid];
                s_warp[w2][tid] = run;
                run += c;
            }
            s_off[tid] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t dst = s_warp[w][d] + rank;
            if (dst < n) {  // always true for a consistent histogram
                keys_out[dst] = key;
                vals_out[dst] = val;
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t scan_scratch_elems(int64_t n)
{
    return scan_scratch_elems_of(n);
}

int exclusive_scan_u32(uint32_t *data, int64_t n, uint32_t *scratch, cudaStream_t s)
{
    return exclusive_scan_t<uint32_t>(data, n, scratch, s);
}

int exclusive_scan_u64(unsigned long long *data, int64_t n, unsigned long long *scratch, cudaStream_t s)
{
    return exclusive_scan_t<unsigned long long>(data, n, scratch, s);
}

size_t radix_scratch_elems(int64_t n)
{
    return radix_scratch_elems_of(n);
}

int radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_k, uint32_t *tmp_v, int64_t n, int bits,
                     uint32_t *scratch, cudaStream_t s)
{
    if (n <= 1)
        return KDT_OK;
    int64_t tiles = (n + RADIX_TILE - 1) / RADIX_TILE;
    uint32_t *hist = scratch;
    uint32_t *scan_tmp = scratch + 256 * tiles;
    int passes = (bits + 7) / 8;
    uint32_t *ka = keys, *va = vals, *kb = tmp_k, *vb = tmp_v;
    for (int p = 0; p < passes; ++p) {
        KDT_LAUNCH radix_hist_kernel<<<(unsigned)tiles, RADIX_THREADS, 0, s>>>(ka, n, 8 * p, tiles, hist);
        KDT_TRY(exclusive_scan_u32(hist, 256 * tiles, scan_tmp, s));
        KDT_LAUNCH radix_scatter_kernel<<<(unsigned)tiles, RADIX_THREADS, 0, s>>>(ka, va, n, 8 * p, tiles, hist, kb, vb);
        KDT_CUDA(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        KDT_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        KDT_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    return KDT_OK;
}

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0)
            sms = 1;
    }
    return sms;
}

}  // namespace kdt
