// Learned radius proposal (not in the paper).
#include "kdt_learned.cuh"

namespace kdt {

__global__ void fill_inf_kernel(float *p, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = __int_as_float(0x7f800000);
}

void fill_inf(float *p, int64_t n, cudaStream_t s)
{
    if (n > 0)
        fill_inf_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(p, n);
}

int run_learned_query(kdt_tree *t, const float *, int64_t, int, float, int, int32_t *, float *, cudaStream_t)
{
    if (!t->model.trained)
        return set_error(KDT_ENOMODEL, "the tree has no trained radius model");
    return set_error(KDT_EINVAL, "learned queries are not available in this build");
}

void free_model(kdt_tree *t)
{
    if (t->model.d_params)
        cudaFree(t->model.d_params);
    t->model.d_params = nullptr;
}

}  // namespace kdt
