// L2 read bandwidth of this GPU, measured by the library's own kernel (no
// paper counterpart): the denominator of the L2 fraction that the benchmark
// reports beside the HBM fraction.  A buffer small enough to stay in L2 is
// read once to bring it in, then read `reps` times with 16-byte loads that
// bypass L1 (ld.global.cg), by a grid of 8 blocks of 256 threads per SM; the
// rate is the bytes read over the CUDA-event time of the timed passes.
#include "kdt_internal.cuh"

namespace kdt {
namespace {

__global__ void __launch_bounds__(256) l2_read_kernel(const float4 *__restrict__ p, int64_t n4, int reps,
                                                      float *__restrict__ sink)
{
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(p + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    }
    // the buffer holds zeros; the store never happens but keeps the loads
    if (acc != 0.f)
        sink[threadIdx.x] = acc;
}

}  // namespace
}  // namespace kdt

using namespace kdt;

extern "C" int kdt_l2_read_bandwidth(int64_t bytes, int reps, double *gbs, void *stream)
{
    if (bytes < (1 << 20) || bytes > ((int64_t)1 << 30) || reps < 1 || reps > 100000 || !gbs)
        return set_error(KDT_EINVAL, "bytes must be in [1 MiB, 1 GiB], reps in [1, 100000], gbs not NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n4 = bytes / 16;
    void *buf = nullptr;
    KDT_CUDA(cudaMallocAsync(&buf, (size_t)n4 * 16 + 1024, s));
    float4 *p = (float4 *)buf;
    float *sink = (float *)((char *)buf + n4 * 16);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = KDT_OK;
    float best = 3.4e38f;
    if (cudaMemsetAsync(buf, 0, (size_t)n4 * 16 + 1024, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = set_error(KDT_ECUDA, "probe set-up failed");
    const int grid = num_sms() * 8;
    if (rc == KDT_OK)
        KDT_LAUNCH l2_read_kernel<<<grid, 256, 0, s>>>(p, n4, 1, sink);  // bring the buffer into L2
    for (int t = 0; t < 3 && rc == KDT_OK; ++t) {
        float ms = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess)
            rc = set_error(KDT_ECUDA, "event record");
        if (rc == KDT_OK)
            KDT_LAUNCH l2_read_kernel<<<grid, 256, 0, s>>>(p, n4, reps, sink);
        if (rc == KDT_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = set_error(KDT_ECUDA, "probe timing failed");
        if (rc == KDT_OK && ms < best)
            best = ms;
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFreeAsync(buf, s);
    if (rc != KDT_OK)
        return rc;
    *gbs = (double)n4 * 16.0 * reps / (best * 1e-3) / 1e9;
    return KDT_OK;
}
