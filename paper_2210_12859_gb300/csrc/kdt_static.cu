// kdt_knn_static: kdt_knn for callers that cannot allocate device memory.
//
// Some callers are not allowed to enter the CUDA allocator while they query:
// an application that hands all device memory to its own pool at start-up
// and leaves nothing for a library's cudaMalloc; a real-time loop in which
// the implicit synchronisation of cudaMalloc / cudaFree would stall other
// work; a plugin whose host forbids device allocations from inside a frame.
// For them this entry point keeps its scratch (the warp work counter and the
// Morton keys, permutation and radix-sort temporaries) in one file-scope
// device array of fixed size instead of allocating it per call.  The array
// lives in every GPU that loads the library until the process exits.
//
// The array is shared by all calls: a call clears what must start at zero (the
// work counter) and overwrites the rest before reading it.  Two calls whose
// work overlaps on the GPU (different streams, or host threads racing) use
// the same bytes and race; serialise them.
#include "kdt_query.cuh"

namespace kdt {


namespace {

constexpr int64_t STATIC_MAX_Q = KDT_STATIC_MAX_Q;
constexpr size_t STATIC_COUNTER_BYTES = 256;
// the work counter block, then the Morton keys, permutation and radix-sort
// temporaries of the largest call (the same formula run_query sizes its
// scratch with, evaluated at compile time)
constexpr size_t STATIC_BYTES = STATIC_COUNTER_BYTES + morton_scratch_bytes_of(STATIC_MAX_Q);
static_assert(STATIC_BYTES < (size_t)8 << 20, "static scratch grew beyond its documented few MB");

__device__ __align__(256) unsigned char g_static_scratch[STATIC_BYTES];

// Device address of g_static_scratch in the current device's context.  In
// host code the symbol name is only a host-side stand-in, so the address is
// looked up on every call (cheap, allocates nothing) rather than cached: a
// cached pointer would go stale if the context were torn down and recreated.
int static_scratch(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
        return cuda_error(e, "cudaGetSymbolAddress(g_static_scratch)", __FILE__, __LINE__);
    *out = p;
    return KDT_OK;
}

}  // namespace
}  // namespace kdt

using namespace kdt;

extern "C" int kdt_knn_static(const kdt_tree *t, const float *d_q, int64_t Q, int k, float max_radius, int flags,
                              int32_t *d_ids, float *d_d2, void *stream)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (Q < 0)
        return set_error(KDT_EINVAL, "Q must be >= 0 (got %lld)", (long long)Q);
    if (Q > STATIC_MAX_Q)
        return set_error(KDT_EINVAL, "kdt_knn_static serves at most %lld queries per call (got %lld)",
                         (long long)STATIC_MAX_Q, (long long)Q);
    if (k < 1 || k > 64)
        return set_error(KDT_EINVAL, "k must be in [1, 64] (got %d)", k);
    if (!(max_radius >= 0.f))
        return set_error(KDT_EINVAL, "max_radius must be >= 0 (got %g)", (double)max_radius);
    if (flags & (KDT_LEARNED | KDT_PLAIN_STEP | KDT_CLOSE_FIRST | KDT_STACK))
        return set_error(KDT_EINVAL, "kdt_knn_static takes neither KDT_LEARNED nor the traversal ablations");
    if (Q > 0 && (!d_q || !d_ids || !d_d2))
        return set_error(KDT_EINVAL, "NULL query or output pointer");
    if (Q == 0)
        return KDT_OK;
    if (STATIC_COUNTER_BYTES + morton_scratch_bytes(Q) > STATIC_BYTES)
        return set_error(KDT_EINVAL, "static scratch too small for %lld queries", (long long)Q);
    void *base = nullptr;
    KDT_TRY(static_scratch(&base));
    cudaStream_t s = (cudaStream_t)stream;

    QueryArgs a;
    a.counter = (unsigned long long *)base;  // zeroed by the launch
    if (flags & KDT_MORTON)
        KDT_TRY(morton_order(d_q, Q, t->D, t->bbox, 1, nullptr, 0, (flags & KDT_COST_ORDER) ? t->nodes : nullptr, t->N,
                             t->layout == 3, (char *)base + STATIC_COUNTER_BYTES,
                             const_cast<uint32_t **>(&a.perm), s));
    a.nodes = t->nodes;
    a.ids = t->ids;
    a.N = (int)t->N;
    a.D = t->D;
    a.queries = d_q;
    a.Q = Q;
    a.k = k;
    a.r2 = max_radius * max_radius;
    a.out_ids = d_ids;
    a.out_d2 = d_d2;
    a.err = t->err;
    a.staged = (flags & KDT_NO_STAGE) ? 0 : staged_for_levels(t->N, stage_levels_for(t, k));
    a.claim_steps = claim_steps_for(t, k);
    a.light_run = light_run_for(t, k);
    a.step_cap = t->debug_step_cap;
    a.inline_depth = inline_depth_for(t, k) >= 2 ? inline_depth_for(t, k) : 1;  // depth 0 is plain-query only
    return launch_query(t->layout, a, !(flags & KDT_UNORDERED), MODE_RESULTS, false, s);
}
