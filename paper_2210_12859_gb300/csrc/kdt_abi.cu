// C ABI of the library (declared in include/kdt.h): argument checking, object
// lifetimes, scratch memory, the query reordering and kernel dispatch.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "kdt_learned.cuh"
#include "kdt_query.cuh"
#include "kdt_traverse.cuh"

namespace kdt {

// ---------------------------------------------------------------- errors

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    int code = e == cudaErrorMemoryAllocation ? KDT_ENOMEM : KDT_ECUDA;
    const char *f = strrchr(file, '/');
    return set_error(code, "%s:%d: %s failed: %s", f ? f + 1 : file, line, what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------- helpers

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int grid_for_kernel(const void *fn, int threads, size_t smem)
{
    static std::mutex mu;
    static std::unordered_map<const void *, std::unordered_map<size_t, int>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto &m = cache[fn];
    const size_t key = smem * 2048 + (size_t)threads;
    auto it = m.find(key);
    if (it != m.end())
        return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int g = per_sm * num_sms();
    m[key] = g;
    return g;
}

static bool bad_radius(float r) { return !(r >= 0.f); }

static std::atomic<int> g_fail_allocs{0};

bool debug_alloc_fails()
{
    int n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1))
            return true;
    return false;
}

// ---------------------------------------------------------------- Morton order

__device__ __forceinline__ uint32_t spread3(uint32_t x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// 30-bit Morton code of the first min(D,3) coordinates quantised to 10 bits
// inside the bounding box of the query's tree.  With `nodes` (a single tree
// of D <= 3), the key is a 5-bit cost class above a 27-bit Morton code (9 bits
// per coordinate), most expensive class first: a query whose greedy descent
// ends far from its leaf point, relative to the tree's mean point spacing,
// lies outside the data and processes many nodes, more the farther it ends.
// With r = d2(leaf) / spacing^2, queries with r > 64 are classed by
// floor(log2 r) (larger first), the others in three classes (r > 8, r > 1,
// the rest).  Starting the longest queries first keeps them out of the end of
// the launch, where too few lanes are left to hide their latency.
__global__ void morton_kernel(const float *__restrict__ qs, int64_t Q, int D, const float *__restrict__ bbox, int T,
                              const int64_t *__restrict__ q_off, const float4 *__restrict__ nodes, int64_t N,
                              bool stored, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                              unsigned long long *__restrict__ n_far)
{
    float spacing2 = 0.f;
    if (nodes) {
        float vol = 1.f;
        for (int j = 0; j < D; ++j)
            vol *= fmaxf(bbox[3 + j] - bbox[j], 1e-30f);
        spacing2 = powf(vol / (float)N, 2.f / (float)D);
    }
    // every thread of the grid runs the same number of iterations, so the
    // warp vote that counts far queries sees full warps
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t iters = (Q + stride - 1) / stride;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t i = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        bool far = false;
        if (i < Q) {
            int t = 0;
            if (T > 1) {
                int lo = 0, hi = T - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (q_off[mid] <= i)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                t = lo;
            }
            const float *bb = bbox + 6 * t;
            uint32_t code = 0;
            const float cells = nodes ? 512.f : 1024.f;
            for (int j = 0; j < 3 && j < D; ++j) {
                float ext = bb[3 + j] - bb[j];
                float x = ext > 0.f ? (qs[i * D + j] - bb[j]) / ext : 0.f;
                x = fminf(fmaxf(x, 0.f), 1.f);
                uint32_t c = (uint32_t)fminf(x * cells, cells - 1.f);
                code |= spread3(c) << (2 - j);
            }
            if (nodes) {
                float q[3];
                load_query<0>(qs, i, D, q);
                const float r = descent_leaf_d2(nodes, nullptr, 0, (int)N, D, q, stored) / spacing2;
                uint32_t cls;
                if (r > 64.f) {  // floor(log2 r) >= 6: classes 28 (r < 128) down to 0
                    const int e = ilogbf(r);
                    cls = (uint32_t)(28 - min(e - 6, 28));
                    far = true;
                } else {
                    cls = r > 8.f ? 29u : (r > 1.f ? 30u : 31u);  // NaN: 31
                }
                code |= cls << 27;
            }
            keys[i] = code;
            vals[i] = (uint32_t)i;
        }
        if (n_far) {
            const unsigned m = __ballot_sync(0xffffffffu, far);
            if ((threadIdx.x & 31) == 0 && m)
                atomicAdd(n_far, (unsigned long long)__popc(m));
        }
    }
}

__global__ void tree_of_query_kernel(const uint32_t *__restrict__ vals, int64_t Q, const int64_t *__restrict__ q_off,
                                     int T, uint32_t *__restrict__ keys)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t qi = vals[i];
        int lo = 0, hi = T - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (q_off[mid] <= qi)
                lo = mid;
            else
                hi = mid - 1;
        }
        keys[i] = (uint32_t)lo;
    }
}

static unsigned grid_1d(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * 32));
}

size_t morton_scratch_bytes(int64_t Q)
{
    return morton_scratch_bytes_of(Q);
}

// permutation of the queries along the Morton curve (stable: equal codes keep
// their index order); perm receives traversal order -> query index
int morton_order(const float *d_q, int64_t Q, int D, const float *bbox, int T, const int64_t *d_qoff, int tbits,
                 const float4 *nodes, int64_t N, bool stored, void *scratch, uint32_t **perm_out, cudaStream_t s,
                 unsigned long long *n_far)
{
    Carve c{(char *)scratch};
    uint32_t *keys = c.take<uint32_t>(Q);
    uint32_t *perm = c.take<uint32_t>(Q);
    uint32_t *tk = c.take<uint32_t>(Q);
    uint32_t *tv = c.take<uint32_t>(Q);
    uint32_t *rs = c.take<uint32_t>(radix_scratch_elems(Q));
    const bool cost = nodes && D <= 3 && T == 1;
    if (n_far)
        KDT_CUDA(cudaMemsetAsync(n_far, 0, sizeof(unsigned long long), s));
    KDT_LAUNCH morton_kernel<<<grid_1d(Q), 256, 0, s>>>(d_q, Q, D, bbox, T, d_qoff, cost ? nodes : nullptr, N, stored,
                                                        keys, perm, cost ? n_far : nullptr);
    KDT_TRY(radix_sort_pairs(keys, perm, tk, tv, Q, cost ? 32 : 30, rs, s));
    if (T > 1) {
        KDT_LAUNCH tree_of_query_kernel<<<grid_1d(Q), 256, 0, s>>>(perm, Q, d_qoff, T, keys);
        KDT_TRY(radix_sort_pairs(keys, perm, tk, tv, Q, tbits, rs, s));
    }
    KDT_CUDA(cudaGetLastError());
    *perm_out = perm;
    return KDT_OK;
}

// ---------------------------------------------------------------- profiling

struct Prof {
    std::vector<cudaEvent_t> ev;   // pairs
    size_t used = 0;
};

static int prof_begin(kdt_tree *t, cudaStream_t s, cudaEvent_t *stop)
{
    *stop = nullptr;
    if (!t->profiling)
        return KDT_OK;
    Prof *p = (Prof *)t->prof;
    if (p->used + 2 > p->ev.size()) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t e;
            KDT_CUDA(cudaEventCreate(&e));
            p->ev.push_back(e);
        }
    }
    KDT_CUDA(cudaEventRecord(p->ev[p->used], s));
    *stop = p->ev[p->used + 1];
    p->used += 2;
    return KDT_OK;
}

// ---------------------------------------------------------------- queries

int run_query(const kdt_tree *t, const float *d_q, int64_t Q, int k, float r2, int flags, int mode,
              int32_t *d_ids, float *d_d2, int32_t *d_visits, cudaStream_t s)
{
    pool_setup_once();
    const bool morton = flags & KDT_MORTON;
    const bool gheap = heap_in_global(t, k);
    const size_t heap_bytes = gheap ? (size_t)heap_scratch_threads() * k * 8 : 0;
    size_t bytes = carve_size({64, heap_bytes}) + (morton ? morton_scratch_bytes(Q) : 0);
    Scratch sc(s);
    KDT_TRY(sc.alloc(bytes));
    Carve c{(char *)sc.p};
    unsigned long long *counter = c.take<unsigned long long>(8);
    QueryArgs a;
    if (gheap) {
        a.heap = c.take<unsigned long long>(heap_bytes / 8);
        a.heap_threads = heap_scratch_threads();
    }
    a.group = list_group_for(t, k);
    if (morton)
        KDT_TRY(morton_order(d_q, Q, t->D, t->bbox, 1, nullptr, 0, (flags & KDT_COST_ORDER) ? t->nodes : nullptr,
                             t->N, t->layout == 3, c.base + c.off, const_cast<uint32_t **>(&a.perm),
                             s));
    a.nodes = t->nodes;
    a.ids = t->ids;
    a.N = (int)t->N;
    a.D = t->D;
    a.queries = d_q;
    a.Q = Q;
    a.k = k;
    a.r2 = r2;
    a.out_ids = d_ids;
    a.out_d2 = d_d2;
    a.visits = d_visits;
    a.err = t->err;
    a.counter = counter;
    a.staged = (flags & KDT_NO_STAGE) ? 0 : staged_for_levels(t->N, stage_levels_for(t, k));
    a.claim_steps = claim_steps_for(t, k);
    a.light_run = light_run_for(t, k);
    a.step_cap = t->debug_step_cap;
    a.inline_depth = inline_depth_for(t, k);
    cudaEvent_t stop;
    KDT_TRY(prof_begin(const_cast<kdt_tree *>(t), s, &stop));
    // inline depth 0: the one-node-per-step kernel, where it applies
    const bool simple = a.inline_depth == 0 && a.staged == 0 && !(flags & KDT_UNORDERED) && k <= 16 &&
                        t->layout != 2 && (mode == MODE_RESULTS || mode == MODE_VISITS);
    if (a.inline_depth == 0 && !simple)
        a.inline_depth = 1;
    if (flags & (KDT_PLAIN_STEP | KDT_CLOSE_FIRST | KDT_STACK))
        KDT_TRY(launch_ablation(t->layout, a, flags, mode, s));
    else if (simple)
        KDT_TRY(launch_ablation(t->layout, a, KDT_PLAIN_STEP, mode, s));
    else
        KDT_TRY(launch_query(t->layout, a, !(flags & KDT_UNORDERED), mode, false, s));
    if (stop)
        KDT_CUDA(cudaEventRecord(stop, s));
    return KDT_OK;
}

// the traversal ablations are ordered plain-radius variants of kdt_knn
static int check_ablation_flags(int flags)
{
    const int abl = flags & (KDT_PLAIN_STEP | KDT_CLOSE_FIRST | KDT_STACK);
    if (!abl)
        return KDT_OK;
    if (abl & (abl - 1))
        return set_error(KDT_EINVAL, "at most one of KDT_PLAIN_STEP, KDT_CLOSE_FIRST, KDT_STACK");
    if (flags & (KDT_UNORDERED | KDT_LEARNED))
        return set_error(KDT_EINVAL, "the traversal ablations are ordered and take no learned radius");
    return KDT_OK;
}

// o2 may be NULL when the call has a single output
static int check_query_args(const kdt_tree *t, const float *d_q, int64_t Q, int k, float max_radius, const void *o1,
                            const void *o2, bool one_output = false)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (Q < 0)
        return set_error(KDT_EINVAL, "Q must be >= 0 (got %lld)", (long long)Q);
    if (k < 1 || k > 64)
        return set_error(KDT_EINVAL, "k must be in [1, 64] (got %d)", k);
    if (bad_radius(max_radius))
        return set_error(KDT_EINVAL, "max_radius must be >= 0 (got %g)", (double)max_radius);
    if (Q > 0 && (!d_q || !o1 || (!one_output && !o2)))
        return set_error(KDT_EINVAL, "NULL query or output pointer");
    if (Q >= ((int64_t)1 << 32))
        return set_error(KDT_EINVAL, "Q must be < 2^32");
    return KDT_OK;
}

// ---------------------------------------------------------------- export

__global__ void export_kernel(const float4 *__restrict__ nodes, const int32_t *__restrict__ ids, int64_t n, int D,
                              float *__restrict__ coords, int32_t *__restrict__ out_ids)
{
    const int NF = D <= 4 ? 1 : 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        float v[8];
        float4 a = nodes[t * NF];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        if (NF == 2) {
            float4 b = nodes[t * NF + 1];
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        }
        if (coords)
            for (int j = 0; j < D; ++j)
                coords[t * D + j] = v[j];
        if (out_ids)
            out_ids[t] = D <= 3 ? (int32_t)(__float_as_uint(a.w) & NODE_ID_MASK) : ids[t];
    }
}

__global__ void split_dims_kernel(const float4 *__restrict__ nodes, int64_t n, int D, bool stored,
                                  uint8_t *__restrict__ dims)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dims[t] = stored ? (uint8_t)(__float_as_uint(nodes[t].w) >> NODE_DIM_SHIFT)
                         : (uint8_t)(Topo::level(t) % D);
}

}  // namespace kdt

using namespace kdt;

// ======================================================================== ABI

extern "C" {

const char *kdt_last_error(void) { return g_err; }

int64_t kdt_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

__attribute__((visibility("hidden"))) int kdt_tree_alloc_internal(int64_t N, int D, kdt_tree **out)
{
    kdt_tree *t = new (std::nothrow) kdt_tree();
    if (!t)
        return set_error(KDT_ENOMEM, "host allocation failed");
    t->N = N;
    t->D = D;
    t->layout = layout_of(D);
    cudaGetDevice(&t->device);
    t->prof = new Prof();
    if (debug_alloc_fails()) {
        kdt_free(t);
        return set_error(KDT_ENOMEM, "device allocation failed (injected)");
    }
    const int nf = float4_per_node(D);
    cudaError_t e = cudaMalloc(&t->nodes_alloc, ((size_t)N * nf + (nf == 1 ? 1 : 0)) * sizeof(float4));
    t->nodes = t->nodes_alloc + (nf == 1 ? 1 : 0);
    if (e == cudaSuccess && t->layout > 0)
        e = cudaMalloc(&t->ids, (size_t)N * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMalloc(&t->bbox, 6 * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&t->err, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemset(t->err, 0, sizeof(int));
    if (e != cudaSuccess) {
        kdt_free(t);
        return cuda_error(e, "tree allocation", __FILE__, __LINE__);
    }
    *out = t;
    return KDT_OK;
}

static int check_build_args(const float *d_points, int64_t N, int D)
{
    if (!d_points)
        return set_error(KDT_EINVAL, "d_points is NULL");
    if (N < 1 || N >= ((int64_t)1 << 30))
        return set_error(KDT_EINVAL, "N must be in [1, 2^30) (got %lld)", (long long)N);
    if (D < 1 || D > 8)
        return set_error(KDT_EINVAL, "D must be in [1, 8] (got %d)", D);
    return KDT_OK;
}

static int finish_build(kdt_tree *t, int opts, cudaStream_t s)
{
    if (opts & KDT_BUILD_ASYNC)
        return KDT_OK;
    int h = 0;
    KDT_CUDA(cudaMemcpyAsync(&h, t->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KDT_CUDA(cudaStreamSynchronize(s));
    if (h & ERR_NONFINITE)
        return set_error(KDT_ENONFINITE, "a point coordinate is NaN or infinite");
    return KDT_OK;
}

int kdt_build_ex(const float *d_points, int64_t N, int D, int opts, void *stream, kdt_tree **out)
{
    if (!out)
        return set_error(KDT_EINVAL, "out is NULL");
    *out = nullptr;
    KDT_TRY(check_build_args(d_points, N, D));
    const bool widest = opts & KDT_BUILD_WIDEST;
    if (widest && D > 3)
        return set_error(KDT_EINVAL, "KDT_BUILD_WIDEST needs D <= 3 (got %d)", D);
    pool_setup_once();
    cudaStream_t s = (cudaStream_t)stream;
    kdt_tree *t = nullptr;
    KDT_TRY(kdt_tree_alloc_internal(N, D, &t));
    if (widest)
        t->layout = 3;
    int64_t off[2] = {0, N};
    int rc = build_forest(d_points, off, 1, D, t->nodes, t->ids, t->bbox, t->err, s, widest);
    if (rc == KDT_OK)
        rc = finish_build(t, opts, s);
    if (rc != KDT_OK) {
        kdt_free(t);
        return rc;
    }
    *out = t;
    return KDT_OK;
}

int kdt_build(const float *d_points, int64_t N, int D, void *stream, kdt_tree **out)
{
    return kdt_build_ex(d_points, N, D, 0, stream, out);
}

int kdt_rebuild(kdt_tree *t, const float *d_points, int opts, void *stream)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    KDT_TRY(check_build_args(d_points, t->N, t->D));
    cudaStream_t s = (cudaStream_t)stream;
    if (t->payload_c) {
        // the payload follows the old node order: drop it
        KDT_CUDA(cudaStreamSynchronize(s));
        cudaFree(t->payload);
        cudaFree(t->node_of);
        t->payload = nullptr;
        t->node_of = nullptr;
        t->payload_c = 0;
    }
    int64_t off[2] = {0, t->N};
    KDT_TRY(build_forest(d_points, off, 1, t->D, t->nodes, t->ids, t->bbox, t->err, s, t->layout == 3));
    return finish_build(t, opts, s);
}

int kdt_debug_fail_allocs(int n)
{
    if (n < 0)
        return set_error(KDT_EINVAL, "n must be >= 0");
    g_fail_allocs.store(n);
    return KDT_OK;
}

int kdt_debug_set_step_cap(kdt_tree *t, uint32_t cap)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    t->debug_step_cap = cap;
    return KDT_OK;
}

int kdt_tree_info(const kdt_tree *t, int64_t *N, int *D)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (N)
        *N = t->N;
    if (D)
        *D = t->D;
    return KDT_OK;
}

int kdt_tree_export(const kdt_tree *t, float *d_coords, int32_t *d_ids, void *stream)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    KDT_LAUNCH export_kernel<<<grid_1d(t->N), 256, 0, s>>>(t->nodes, t->ids, t->N, t->D, d_coords, d_ids);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

int kdt_tree_split_dims(const kdt_tree *t, uint8_t *d_dims, void *stream)
{
    if (!t || !d_dims)
        return set_error(KDT_EINVAL, "NULL tree or output");
    KDT_LAUNCH split_dims_kernel<<<grid_1d(t->N), 256, 0, (cudaStream_t)stream>>>(t->nodes, t->N, t->D,
                                                                                   t->layout == 3, d_dims);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

int kdt_knn(const kdt_tree *t, const float *d_q, int64_t Q, int k, float max_radius, int flags, int32_t *d_ids,
            float *d_d2, void *stream)
{
    KDT_TRY(check_query_args(t, d_q, Q, k, max_radius, d_ids, d_d2));
    if (Q == 0)
        return KDT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    KDT_TRY(check_ablation_flags(flags));
    float r2 = max_radius * max_radius;
    if (flags & KDT_LEARNED)
        return run_learned_query(const_cast<kdt_tree *>(t), d_q, Q, k, r2, flags, d_ids, d_d2, nullptr, s);
    return run_query(t, d_q, Q, k, r2, flags, 0, d_ids, d_d2, nullptr, s);
}

int kdt_fcp(const kdt_tree *t, const float *d_q, int64_t Q, float max_radius, int flags, int32_t *d_ids, float *d_d2,
            void *stream)
{
    return kdt_knn(t, d_q, Q, 1, max_radius, flags, d_ids, d_d2, stream);
}

int kdt_knn_visits(const kdt_tree *t, const float *d_q, int64_t Q, int k, float max_radius, int flags,
                   int32_t *d_visits, void *stream)
{
    KDT_TRY(check_query_args(t, d_q, Q, k, max_radius, d_visits, nullptr, true));
    KDT_TRY(check_ablation_flags(flags));
    if (Q == 0)
        return KDT_OK;
    if (flags & KDT_LEARNED)
        return run_learned_query(const_cast<kdt_tree *>(t), d_q, Q, k, max_radius * max_radius, flags, nullptr,
                                 nullptr, d_visits, (cudaStream_t)stream);
    return run_query(t, d_q, Q, k, max_radius * max_radius, flags, 1, nullptr, nullptr, d_visits,
                     (cudaStream_t)stream);
}

int kdt_status(kdt_tree *t, void *stream)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    KDT_CUDA(cudaStreamSynchronize(s));
    KDT_CUDA(cudaMemcpy(&h, t->err, sizeof(int), cudaMemcpyDeviceToHost));
    KDT_CUDA(cudaMemset(t->err, 0, sizeof(int)));
    if (h & ERR_NONFINITE)
        return set_error(KDT_ENONFINITE, "a point coordinate is NaN or infinite");
    if (h & ERR_TRAVERSAL)
        return set_error(KDT_ETRAVERSAL, "a traversal exceeded its step bound");
    if (h & ERR_RANGE)
        return set_error(KDT_EINVAL, "a range fill found a different number of points than its offsets allow");
    return KDT_OK;
}

void kdt_free(kdt_tree *t)
{
    if (!t)
        return;
    cudaDeviceSynchronize();
    cudaFree(t->nodes_alloc);
    cudaFree(t->ids);
    cudaFree(t->bbox);
    cudaFree(t->err);
    cudaFree(t->payload);
    cudaFree(t->node_of);
    free_model(t);
    if (t->prof) {
        Prof *p = (Prof *)t->prof;
        for (cudaEvent_t e : p->ev)
            cudaEventDestroy(e);
        delete p;
    }
    delete t;
}

// device address of a host buffer the GPU can address directly (page-locked
// or registered host memory), else NULL; unregistered memory is copied
static void *mapped_host(const void *p)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int kdt_knn_host(const float *h_points, int64_t N, int D, const float *h_q, int64_t Q, int k, float max_radius,
                 int flags, int32_t *h_ids, float *h_d2)
{
    if (!h_points || (Q > 0 && (!h_q || !h_ids || !h_d2)))
        return set_error(KDT_EINVAL, "NULL host pointer");
    KDT_TRY(check_build_args(h_points, N, D));
    if (k < 1 || k > 64 || Q < 0 || bad_radius(max_radius))
        return set_error(KDT_EINVAL, "bad k, Q or max_radius");
    if (flags & KDT_LEARNED)
        return set_error(KDT_EINVAL, "kdt_knn_host builds a fresh tree, which has no radius model");
    pool_setup_once();
    cudaStream_t s;
    KDT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int rc = KDT_OK;
    kdt_tree *t = nullptr;
    {
        // page-locked queries are read and page-locked outputs written in
        // place through the host link (the kernels' own loads and stores,
        // spread over the query launch); other host buffers are copied
        float *mq = Q > 0 ? (float *)mapped_host(h_q) : nullptr;
        int32_t *mi = Q > 0 ? (int32_t *)mapped_host(h_ids) : nullptr;
        float *md = Q > 0 ? (float *)mapped_host(h_d2) : nullptr;
        const bool direct_out = mi && md;
        Scratch sc(s);
        size_t pb = (size_t)N * D * 4, qb = mq ? 0 : (size_t)Q * D * 4, ob = direct_out ? 0 : (size_t)Q * k * 4;
        rc = sc.alloc(carve_size({pb, qb, ob, ob}));
        if (rc == KDT_OK) {
            Carve c{(char *)sc.p};
            float *dp = c.take<float>((size_t)N * D);
            float *dq = mq ? mq : c.take<float>((size_t)Q * D);
            int32_t *di = direct_out ? mi : c.take<int32_t>((size_t)Q * k);
            float *dd = direct_out ? md : c.take<float>((size_t)Q * k);
            cudaError_t e = cudaMemcpyAsync(dp, h_points, pb, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && Q > 0 && !mq)
                e = cudaMemcpyAsync(dq, h_q, qb, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess)
                rc = cuda_error(e, "host to device copy", __FILE__, __LINE__);
            if (rc == KDT_OK)
                rc = kdt_build_ex(dp, N, D, 0, s, &t);
            if (rc == KDT_OK && Q > 0)
                rc = kdt_knn(t, dq, Q, k, max_radius, flags, di, dd, s);
            if (rc == KDT_OK && Q > 0 && !direct_out) {
                e = cudaMemcpyAsync(h_ids, di, ob, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(h_d2, dd, ob, cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess)
                    rc = cuda_error(e, "device to host copy", __FILE__, __LINE__);
            }
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (rc == KDT_OK && e != cudaSuccess)
        rc = cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    if (rc == KDT_OK && t)
        rc = kdt_status(t, s);
    kdt_free(t);
    cudaStreamDestroy(s);
    return rc;
}

int kdt_profile_enable(kdt_tree *t, int enable)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    t->profiling = enable != 0;
    return KDT_OK;
}

int kdt_profile_read(kdt_tree *t, double *ms, int64_t *launches)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    Prof *p = (Prof *)t->prof;
    double total = 0;
    for (size_t i = 0; i + 1 < p->used; i += 2) {
        KDT_CUDA(cudaEventSynchronize(p->ev[i + 1]));
        float m = 0;
        KDT_CUDA(cudaEventElapsedTime(&m, p->ev[i], p->ev[i + 1]));
        total += m;
    }
    if (ms)
        *ms = total;
    if (launches)
        *launches = (int64_t)(p->used / 2);
    p->used = 0;
    return KDT_OK;
}

// ---------------------------------------------------------------- forests

struct ForestGraph {
    cudaGraphExec_t exec = nullptr;
    const float *q = nullptr;
    int32_t *ids = nullptr;
    float *d2 = nullptr;
    int k = 0;
    float r2 = 0;
    int flags = 0;
    std::vector<int64_t> qoff;
    void *scratch = nullptr;   // persistent scratch referenced by the graph
    size_t scratch_bytes = 0;
    int threads = 0;           // launch parameters the graph was captured with
    int claim_steps = 0;
    int inline_depth = 0;
    int light_run = 0;
};

int kdt_build_batched(const float *d_points, const int64_t *h_off, int T, int D, void *stream, kdt_forest **out)
{
    if (!out)
        return set_error(KDT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d_points || !h_off || T < 1 || D < 1 || D > 8)
        return set_error(KDT_EINVAL, "bad forest arguments (T=%d, D=%d)", T, D);
    if (h_off[0] != 0)
        return set_error(KDT_EINVAL, "offsets must start at 0");
    for (int i = 0; i < T; ++i) {
        int64_t n = h_off[i + 1] - h_off[i];
        if (n < 0 || n >= ((int64_t)1 << 30))
            return set_error(KDT_EINVAL, "cloud %d has bad size %lld", i, (long long)n);
    }
    if (h_off[T] >= ((int64_t)1 << 32))
        return set_error(KDT_EINVAL, "total points must be < 2^32");
    pool_setup_once();
    cudaStream_t s = (cudaStream_t)stream;
    kdt_forest *f = new (std::nothrow) kdt_forest();
    if (!f)
        return set_error(KDT_ENOMEM, "host allocation failed");
    f->f.T = T;
    f->f.D = D;
    f->f.total = h_off[T];
    f->h_offsets = new int64_t[T + 1];
    memcpy(f->h_offsets, h_off, (T + 1) * sizeof(int64_t));
    int64_t total = std::max<int64_t>(h_off[T], 1);
    cudaError_t e = cudaMalloc(&f->nodes, (size_t)total * float4_per_node(D) * sizeof(float4));
    if (e == cudaSuccess && layout_of(D) > 0)
        e = cudaMalloc(&f->ids, (size_t)total * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMalloc(&f->bbox, (size_t)T * 6 * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&f->f.d_offsets, (size_t)(T + 1) * sizeof(int64_t));
    if (e == cudaSuccess)
        e = cudaMalloc(&f->err, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(f->err, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f->f.d_offsets, h_off, (T + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    int rc = e == cudaSuccess ? KDT_OK : cuda_error(e, "forest allocation", __FILE__, __LINE__);
    if (rc == KDT_OK)
        rc = build_forest(d_points, h_off, T, D, f->nodes, f->ids, f->bbox, f->err, s);
    if (rc == KDT_OK) {
        int h = 0;
        e = cudaMemcpyAsync(&h, f->err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            rc = cuda_error(e, "forest build", __FILE__, __LINE__);
        else if (h & ERR_NONFINITE)
            rc = set_error(KDT_ENONFINITE, "a point coordinate is NaN or infinite");
    }
    if (rc != KDT_OK) {
        kdt_forest_free(f);
        return rc;
    }
    *out = f;
    return KDT_OK;
}

static int forest_enqueue(kdt_forest *f, ForestGraph *g, const float *d_q, int64_t Q, const int64_t *d_qoff, int k,
                          float r2, int flags, int32_t *d_ids, float *d_d2, cudaStream_t s)
{
    const int T = f->f.T;
    Carve c{(char *)g->scratch};
    unsigned long long *counter = c.take<unsigned long long>(8);
    c.take<int64_t>(T + 1);  // query offsets (filled before)
    QueryArgs a;
    if (flags & KDT_MORTON) {
        int tbits = T > 1 ? floor_log2((uint64_t)(T - 1)) + 1 : 0;
        KDT_TRY(morton_order(d_q, Q, f->f.D, f->bbox, T, d_qoff, tbits, nullptr, 0, false, c.base + c.off,
                             const_cast<uint32_t **>(&a.perm), s));
    }
    a.nodes = f->nodes;
    a.ids = f->ids;
    a.D = f->f.D;
    a.queries = d_q;
    a.Q = Q;
    a.k = k;
    a.r2 = r2;
    a.out_ids = d_ids;
    a.out_d2 = d_d2;
    a.err = f->err;
    a.counter = counter;
    a.T = T;
    a.node_off = f->f.d_offsets;
    a.q_off = d_qoff;
    a.threads = f->threads;
    a.claim_steps = f->claim_steps > 0 ? f->claim_steps : default_claim_steps_k(k);
    a.inline_depth = f->inline_depth == 1 ? 1 : 2;
    a.light_run = f->light_run > 0 ? f->light_run : 1;
    return launch_query(layout_of(f->f.D), a, !(flags & KDT_UNORDERED), 0, true, s);
}

int kdt_knn_batched_visits(kdt_forest *f, const float *d_q, const int64_t *h_qoff, int k, float max_radius,
                           int flags, int32_t *d_visits, void *stream)
{
    if (!f || !h_qoff)
        return set_error(KDT_EINVAL, "NULL forest or offsets");
    const int T = f->f.T;
    if (k < 1 || k > 64 || bad_radius(max_radius))
        return set_error(KDT_EINVAL, "bad k or max_radius");
    if (flags & (KDT_LEARNED | KDT_PLAIN_STEP | KDT_CLOSE_FIRST | KDT_STACK))
        return set_error(KDT_EINVAL, "forest visit counts are for the plain traversal");
    if (h_qoff[0] != 0)
        return set_error(KDT_EINVAL, "query offsets must start at 0");
    for (int i = 0; i < T; ++i)
        if (h_qoff[i + 1] < h_qoff[i])
            return set_error(KDT_EINVAL, "query offsets must be non-decreasing");
    if (h_qoff[T] == 0)
        return KDT_OK;
    if (!d_q || !d_visits)
        return set_error(KDT_EINVAL, "NULL query or visits pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    KDT_TRY(sc.alloc(256));
    const int layout = layout_of(f->f.D);
    const int NF = float4_per_node(f->f.D);
    // one counting launch per tree: the counts do not depend on how the
    // queries are scheduled
    for (int i = 0; i < T; ++i) {
        const int64_t nq = h_qoff[i + 1] - h_qoff[i];
        const int64_t nb = f->h_offsets[i];
        const int64_t n = f->h_offsets[i + 1] - nb;
        if (nq == 0)
            continue;
        if (n == 0) {
            KDT_CUDA(cudaMemsetAsync(d_visits + h_qoff[i], 0, nq * 4, s));
            continue;
        }
        QueryArgs a;
        a.nodes = f->nodes + nb * NF;
        a.ids = f->ids ? f->ids + nb : nullptr;
        a.N = (int)n;
        a.D = f->f.D;
        a.queries = d_q + h_qoff[i] * f->f.D;
        a.Q = nq;
        a.k = k;
        a.r2 = max_radius * max_radius;
        a.visits = d_visits + h_qoff[i];
        a.err = f->err;
        a.counter = (unsigned long long *)sc.p;
        a.claim_steps = default_claim_steps_k(k);
        KDT_TRY(launch_query(layout, a, !(flags & KDT_UNORDERED), MODE_VISITS, false, s));
    }
    return KDT_OK;
}

int kdt_knn_batched(kdt_forest *f, const float *d_q, const int64_t *h_qoff, int k, float max_radius, int flags,
                    int32_t *d_ids, float *d_d2, void *stream)
{
    if (!f || !h_qoff)
        return set_error(KDT_EINVAL, "NULL forest or offsets");
    const int T = f->f.T;
    if (k < 1 || k > 64 || bad_radius(max_radius))
        return set_error(KDT_EINVAL, "bad k or max_radius");
    if (flags & KDT_LEARNED)
        return set_error(KDT_EINVAL, "KDT_LEARNED is not supported for forests");
    if (flags & (KDT_PLAIN_STEP | KDT_CLOSE_FIRST | KDT_STACK))
        return set_error(KDT_EINVAL, "the traversal ablations are single-tree only");
    if (h_qoff[0] != 0)
        return set_error(KDT_EINVAL, "query offsets must start at 0");
    for (int i = 0; i < T; ++i)
        if (h_qoff[i + 1] < h_qoff[i])
            return set_error(KDT_EINVAL, "query offsets must be non-decreasing");
    const int64_t Q = h_qoff[T];
    if (Q >= ((int64_t)1 << 32))
        return set_error(KDT_EINVAL, "total queries must be < 2^32");
    if (Q == 0)
        return KDT_OK;
    if (!d_q || !d_ids || !d_d2)
        return set_error(KDT_EINVAL, "NULL query or output pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const float r2 = max_radius * max_radius;

    if (flags & KDT_PER_TREE) {
        // the same traversal, one launch per tree
        Scratch sc(s);
        KDT_TRY(sc.alloc(256));
        unsigned long long *counter = (unsigned long long *)sc.p;
        const int layout = layout_of(f->f.D);
        const int NF = float4_per_node(f->f.D);
        for (int i = 0; i < T; ++i) {
            int64_t nq = h_qoff[i + 1] - h_qoff[i];
            int64_t nb = f->h_offsets[i];
            int64_t n = f->h_offsets[i + 1] - nb;
            if (nq == 0)
                continue;
            if (n == 0) {
                KDT_CUDA(cudaMemsetAsync(d_ids + h_qoff[i] * k, 0xff, nq * k * 4, s));
                fill_inf(d_d2 + h_qoff[i] * k, nq * k, s);
                continue;
            }
            QueryArgs a;
            a.nodes = f->nodes + nb * NF;
            a.ids = f->ids ? f->ids + nb : nullptr;
            a.N = (int)n;
            a.D = f->f.D;
            a.queries = d_q + h_qoff[i] * f->f.D;
            a.Q = nq;
            a.k = k;
            a.r2 = r2;
            a.out_ids = d_ids + h_qoff[i] * k;
            a.out_d2 = d_d2 + h_qoff[i] * k;
            a.err = f->err;
            a.counter = counter;
            a.staged = (flags & KDT_NO_STAGE) ? 0 : staged_for_levels(n, 6);
            a.claim_steps = default_claim_steps_k(k);
            KDT_TRY(launch_query(layout, a, !(flags & KDT_UNORDERED), 0, false, s));
        }
        return KDT_OK;
    }

    ForestGraph *g = (ForestGraph *)f->graph;
    if (!g) {
        g = new ForestGraph();
        f->graph = g;
    }
    const bool same = g->exec && g->q == d_q && g->ids == d_ids && g->d2 == d_d2 && g->k == k && g->r2 == r2 &&
                      g->flags == flags && g->threads == f->threads && g->claim_steps == f->claim_steps &&
                      g->inline_depth == f->inline_depth && g->light_run == f->light_run &&
                      g->qoff.size() == (size_t)T + 1 &&
                      std::equal(g->qoff.begin(), g->qoff.end(), h_qoff);
    if (!same) {
        if (g->exec) {
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
        size_t need = carve_size({64, (size_t)(T + 1) * 8}) + ((flags & KDT_MORTON) ? morton_scratch_bytes(Q) : 0);
        if (need > g->scratch_bytes) {
            KDT_CUDA(cudaStreamSynchronize(s));
            cudaFree(g->scratch);
            g->scratch = nullptr;
            g->scratch_bytes = 0;
            KDT_CUDA(cudaMalloc(&g->scratch, need));
            g->scratch_bytes = need;
        }
        g->q = d_q;
        g->ids = d_ids;
        g->d2 = d_d2;
        g->k = k;
        g->r2 = r2;
        g->flags = flags;
        g->threads = f->threads;
        g->claim_steps = f->claim_steps;
        g->inline_depth = f->inline_depth;
        g->light_run = f->light_run;
        g->qoff.assign(h_qoff, h_qoff + T + 1);
    }
    Carve c{(char *)g->scratch};
    c.take<unsigned long long>(8);
    int64_t *d_qoff = c.take<int64_t>(T + 1);
    if (!same)
        KDT_CUDA(cudaMemcpyAsync(d_qoff, h_qoff, (T + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));

    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    KDT_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone || s == nullptr)
        return forest_enqueue(f, g, d_q, Q, d_qoff, k, r2, flags, d_ids, d_d2, s);
    if (!g->exec) {
        cudaGraph_t graph = nullptr;
        KDT_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = forest_enqueue(f, g, d_q, Q, d_qoff, k, r2, flags, d_ids, d_d2, s);
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (rc != KDT_OK) {
            if (graph)
                cudaGraphDestroy(graph);
            return rc;
        }
        KDT_CUDA(e);
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        KDT_CUDA(e);
    }
    KDT_CUDA(cudaGraphLaunch(g->exec, s));
    return KDT_OK;
}

int kdt_forest_set_launch(kdt_forest *f, int threads, int claim_steps, int inline_depth, int light_run)
{
    if (!f)
        return set_error(KDT_EINVAL, "forest is NULL");
    if (inline_depth < 0 || inline_depth > 2)
        return set_error(KDT_EINVAL, "inline_depth must be 0 (default), 1 or 2 (got %d)", inline_depth);
    if (light_run < 0 || light_run > 64)
        return set_error(KDT_EINVAL, "light_run must be in [0, 64] (got %d)", light_run);
    if (threads < 0 || threads > REG_THREADS || threads % 32 != 0)
        return set_error(KDT_EINVAL, "threads must be 0 or a multiple of 32 up to %d (got %d)", REG_THREADS, threads);
    if (claim_steps < 0 || claim_steps > 256)
        return set_error(KDT_EINVAL, "claim_steps must be in [0, 256] (got %d)", claim_steps);
    f->threads = threads;
    f->claim_steps = claim_steps;
    f->inline_depth = inline_depth;
    f->light_run = light_run;
    return KDT_OK;
}

// Coordinate search over the batched launch: inline depth {2, 1}, light run
// {1, 4, 8}, block size {128, 64}, then claim steps {16, 32, 64, 128}; each
// candidate is the whole
// batched query (graph included), one warm-up and one timed run, and is taken
// when it is faster than the best so far by 2 %.
int kdt_forest_autotune(kdt_forest *f, const float *d_q, const int64_t *h_qoff, int k, float max_radius, int flags,
                        int32_t *d_ids, float *d_d2, int *best_threads, int *best_claim, int *best_inline,
                        int *best_light, float *best_ms, void *stream)
{
    if (!f || !h_qoff || !d_q || !d_ids || !d_d2)
        return set_error(KDT_EINVAL, "NULL forest, query, offset or output pointer");
    if (flags & KDT_PER_TREE)
        return set_error(KDT_EINVAL, "autotune the batched launch (no KDT_PER_TREE)");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    KDT_CUDA(cudaEventCreate(&e0));
    KDT_CUDA(cudaEventCreate(&e1));
    const int saved_t = f->threads, saved_c = f->claim_steps, saved_i = f->inline_depth, saved_l = f->light_run;
    int bt = 0, bc = 0, bi = 2, bl = 1, rc = KDT_OK;
    float best = 3.4e38f;
    auto trial = [&](int th, int cs, int inl, int lr) {
        if (rc != KDT_OK)
            return;
        f->threads = th;
        f->claim_steps = cs;
        f->inline_depth = inl;
        f->light_run = lr;
        rc = kdt_knn_batched(f, d_q, h_qoff, k, max_radius, flags, d_ids, d_d2, stream);
        float ms = 0.f;
        if (rc == KDT_OK && cudaEventRecord(e0, s) != cudaSuccess)
            rc = set_error(KDT_ECUDA, "event record");
        if (rc == KDT_OK)
            rc = kdt_knn_batched(f, d_q, h_qoff, k, max_radius, flags, d_ids, d_d2, stream);
        if (rc == KDT_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = set_error(KDT_ECUDA, "event timing failed");
        if (rc == KDT_OK && ms < best * 0.98f) {
            best = ms;
            bt = th;
            bc = cs;
            bi = inl;
            bl = lr;
        }
    };
    trial(0, 0, 2, 1);
    trial(0, 0, 1, 1);
    const int i_best = bi;
    trial(0, 0, i_best, 4);
    trial(0, 0, i_best, 8);
    const int l_best = bl;
    trial(64, 0, i_best, l_best);
    const int t_best = bt;
    for (int cs : {16, 32, 64, 128})
        if (cs != default_claim_steps_k(k))
            trial(t_best, cs, i_best, l_best);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != KDT_OK) {
        f->threads = saved_t;
        f->claim_steps = saved_c;
        f->inline_depth = saved_i;
        f->light_run = saved_l;
        return rc;
    }
    f->threads = bt;
    f->claim_steps = bc;
    f->inline_depth = bi;
    f->light_run = bl;
    if (best_inline)
        *best_inline = bi;
    if (best_light)
        *best_light = bl;
    if (best_threads)
        *best_threads = bt ? bt : REG_THREADS;
    if (best_claim)
        *best_claim = bc ? bc : default_claim_steps_k(k);
    if (best_ms)
        *best_ms = best;
    return KDT_OK;
}

int kdt_forest_export(const kdt_forest *f, float *d_coords, int32_t *d_ids, void *stream)
{
    if (!f)
        return set_error(KDT_EINVAL, "forest is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (f->f.total == 0)
        return KDT_OK;
    KDT_LAUNCH export_kernel<<<grid_1d(f->f.total), 256, 0, s>>>(f->nodes, f->ids, f->f.total, f->f.D, d_coords, d_ids);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

void kdt_forest_free(kdt_forest *f)
{
    if (!f)
        return;
    cudaDeviceSynchronize();
    if (f->graph) {
        ForestGraph *g = (ForestGraph *)f->graph;
        if (g->exec)
            cudaGraphExecDestroy(g->exec);
        cudaFree(g->scratch);
        delete g;
    }
    cudaFree(f->nodes);
    cudaFree(f->ids);
    cudaFree(f->bbox);
    cudaFree(f->f.d_offsets);
    cudaFree(f->err);
    delete[] f->h_offsets;
    delete f;
}

}  // extern "C"
