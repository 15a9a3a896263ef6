// Query kernels for node layout 3 (see kdt_query_impl.cuh).
#include "kdt_query_impl.cuh"

namespace kdt {
int launch_query_layout3(const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s)
{
    return launch_query_impl<3>(a, ordered, mode, batched, s);
}
}  // namespace kdt
