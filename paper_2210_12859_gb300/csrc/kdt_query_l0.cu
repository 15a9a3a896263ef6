// Query kernels for node layout 0 (see kdt_query_impl.cuh).
#include "kdt_query_impl.cuh"

namespace kdt {
int launch_query_layout0(const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s)
{
    return launch_query_impl<0>(a, ordered, mode, batched, s);
}
}  // namespace kdt
