// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <initializer_list>
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kdt.h"

namespace kdt {

// ---------------------------------------------------------------- errors

int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what, const char *file, int line);

#define KDT_CUDA(call)                                                          \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess)                                                  \
            return ::kdt::cuda_error(e_, #call, __FILE__, __LINE__);            \
    } while (0)

#define KDT_TRY(call)                                                           \
    do {                                                                        \
        int rc_ = (call);                                                       \
        if (rc_ != KDT_OK)                                                      \
            return rc_;                                                         \
    } while (0)

// every kernel launch of the library goes through KDT_LAUNCH, which counts it
void note_launch();
#define KDT_LAUNCH ::kdt::note_launch(),

// device error word bits
enum : int { ERR_NONFINITE = 1, ERR_TRAVERSAL = 2, ERR_RANGE = 4 };

// ---------------------------------------------------------------- topology
// A complete, left-balanced tree of n nodes in level order (root 0, children
// 2t+1 and 2t+2).  H = floor(log2 n) is the last level and M the number of
// nodes on it.  In a perfect tree of H+1 levels the in-order index of the
// j-th node of level l is (2j+1)*2^(H-l) - 1; the complete tree lacks the
// last-level nodes j >= M, whose perfect in-order indices are the even numbers
// 2j, so an in-order index shifts down by the number of missing nodes before
// it.

__host__ __device__ __forceinline__ int floor_log2(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return 63 - __clzll((long long)v);
#else
    return 63 - __builtin_clzll(v);
#endif
}

__host__ __device__ __forceinline__ int count_tz(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return __ffsll((long long)v) - 1;
#else
    return __builtin_ctzll(v);
#endif
}

struct Topo {
    int64_t n;
    int H;
    int64_t M;
    __host__ __device__ __forceinline__ explicit Topo(int64_t n_) : n(n_)
    {
        H = n_ > 0 ? floor_log2((uint64_t)n_) : 0;
        M = n_ - (((int64_t)1 << H) - 1);
    }
    __host__ __device__ __forceinline__ static int level(int64_t t) { return floor_log2((uint64_t)(t + 1)); }

    // in-order index of node t (t < n)
    __host__ __device__ __forceinline__ int64_t inorder(int64_t t) const
    {
        int l = level(t);
        int64_t j = t - (((int64_t)1 << l) - 1);
        int64_t P = ((2 * j + 1) << (H - l)) - 1;
        int64_t half = (P + 1) >> 1;
        int64_t full = (int64_t)1 << H;
        int64_t missing = (half < full ? half : full) - M;
        return P - (missing > 0 ? missing : 0);
    }
    // node at in-order index p (p < n)
    __host__ __device__ __forceinline__ int64_t node_at(int64_t p) const
    {
        int64_t P = p < 2 * M ? p : 2 * (p - M) + 1;
        int tz = count_tz((uint64_t)(P + 1));
        int l = H - tz;
        int64_t j = (P + 1) >> (tz + 1);
        return (((int64_t)1 << l) - 1) + j;
    }
    // rightmost node of the subtree of t
    __host__ __device__ __forceinline__ int64_t rightmost(int64_t t) const
    {
        int m = H - level(t);
        int64_t u = ((t + 2) << m) - 2;
        if (u >= n)
            u = ((t + 2) << (m - 1)) - 2;
        return u;
    }
    // leftmost node of the subtree of t
    __host__ __device__ __forceinline__ int64_t leftmost(int64_t t) const
    {
        int m = H - level(t);
        int64_t u = ((t + 1) << m) - 1;
        if (u >= n)
            u = ((t + 1) << (m - 1)) - 1;
        return u;
    }
    // ancestor of u on level l (level(u) >= l)
    __host__ __device__ __forceinline__ static int64_t ancestor(int64_t u, int lu, int l)
    {
        return ((u + 1) >> (lu - l)) - 1;
    }
};

// order-preserving unsigned key of a finite float; -0 is mapped to +0 first
__host__ __device__ __forceinline__ uint32_t float_key(float x)
{
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(x);
#else
    __builtin_memcpy(&u, &x, 4);
#endif
    if (u == 0x80000000u)
        u = 0;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// ---------------------------------------------------------------- layouts
// Node storage:
//   layout 0 (D <= 3): float4 {x, y, z, id bits} per node, unused coords = 0
//   layout 1 (D == 4): float4 {c0..c3} per node + int32 ids[N]
//   layout 2 (D 5..8): 2 x float4 {c0..c7} per node + int32 ids[N], unused = 0
//   layout 3 (D <= 3, split dimension stored per node): as layout 0 with the
//            node's split dimension in the two high bits of the id word
constexpr uint32_t NODE_ID_MASK = 0x3fffffffu;
constexpr int NODE_DIM_SHIFT = 30;
__host__ __device__ __forceinline__ int layout_of(int D) { return D <= 3 ? 0 : (D == 4 ? 1 : 2); }
__host__ __device__ __forceinline__ int float4_per_node(int D) { return D <= 4 ? 1 : 2; }

// ---------------------------------------------------------------- primitives
// Stable LSD radix sort of (u32 key, u32 value) pairs on bits [0, bits).
// keys/vals hold the input and receive the output; tmp_k / tmp_v are scratch of
// n elements each, `scratch` holds radix_scratch_elems(n) elements.
size_t radix_scratch_elems(int64_t n);
int radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_k, uint32_t *tmp_v, int64_t n,
                     int bits, uint32_t *scratch, cudaStream_t s);

// exclusive prefix sum of u32 in place (n elements), scratch of
// scan_scratch_elems(n) elements
size_t scan_scratch_elems(int64_t n);
int exclusive_scan_u32(uint32_t *data, int64_t n, uint32_t *scratch, cudaStream_t s);
int exclusive_scan_u64(unsigned long long *data, int64_t n, unsigned long long *scratch, cudaStream_t s);

int num_sms();

// permutation of queries along the Morton curve (traversal order -> query index);
// with cost classes (nodes given), n_far (device, may be NULL) receives the
// number of queries in the far classes, which come first in the permutation
int morton_order(const float *d_q, int64_t Q, int D, const float *bbox, int T, const int64_t *d_qoff, int tbits,
                 const float4 *nodes, int64_t N, bool stored, void *scratch, uint32_t **perm_out, cudaStream_t s,
                 unsigned long long *n_far = nullptr);
size_t morton_scratch_bytes(int64_t Q);

// ---------------------------------------------------------------- scratch

// failure injection for tests: true while kdt_debug_fail_allocs has failures
// left (each call consumes one)
bool debug_alloc_fails();

inline void pool_setup_once()
{
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev])
        return;
    done[dev] = true;
    // keep freed scratch in the stream-ordered pool of this process instead of
    // returning it to the driver after every call
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
}

// stream-ordered scratch released at scope exit
struct Scratch {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    explicit Scratch(cudaStream_t s_) : s(s_) {}
    int alloc(size_t bytes)
    {
        if (debug_alloc_fails())
            return set_error(KDT_ENOMEM, "device allocation failed (injected)");
        KDT_CUDA(cudaMallocAsync(&p, std::max<size_t>(bytes, 256), s));
        return KDT_OK;
    }
    ~Scratch()
    {
        if (p)
            cudaFreeAsync(p, s);
    }
};

struct Carve {
    char *base;
    size_t off = 0;
    template <class T> T *take(size_t n)
    {
        T *r = (T *)(base + off);
        off += (n * sizeof(T) + 255) & ~(size_t)255;
        return r;
    }
};

constexpr size_t carve_size(std::initializer_list<size_t> bytes)
{
    size_t s = 0;
    for (size_t b : bytes)
        s += (b + 255) & ~(size_t)255;
    return s;
}

// Tile sizes of the device-wide scan and radix sort (kdt_sort.cu), here so
// that scratch sizes can be computed at compile time.
constexpr int SCAN_TILE_ELEMS = 2048;   // elements per tile of the exclusive scan
constexpr int RADIX_TILE_KEYS = 2048;   // keys per tile of the radix sort
constexpr size_t scan_scratch_elems_of(int64_t n)
{
    return (size_t)((n + SCAN_TILE_ELEMS - 1) / SCAN_TILE_ELEMS) + 1;
}
constexpr size_t radix_scratch_elems_of(int64_t n)
{
    const int64_t tiles = (n + RADIX_TILE_KEYS - 1) / RADIX_TILE_KEYS;
    const size_t h = (size_t)256 * (size_t)(tiles > 1 ? tiles : 1);
    return h + scan_scratch_elems_of((int64_t)h);
}
// Morton keys, permutation and two sort temporaries of Q u32 each, plus the
// radix sort's histograms and scan partials
constexpr size_t morton_scratch_bytes_of(int64_t Q)
{
    return carve_size({(size_t)Q * 4, (size_t)Q * 4, (size_t)Q * 4, (size_t)Q * 4, radix_scratch_elems_of(Q) * 4});
}


// ---------------------------------------------------------------- objects

struct Model {
    bool trained = false;
    float *d_params = nullptr;     // FP32 master weights [KDT_MLP_PARAMS]
    float norm[8] = {0, 0, 0, 0, 1, 1, 1, 1};
    float margin = 1.25f;
    int k_trained = 0;
    int gate = KDT_GATE_ALL;       // which queries get the proposal
    float gate_cost = 0.f;         // network pass per query in processed-node equivalents (automatic gate)
};

struct ForestDesc {
    int T = 1;
    int D = 3;
    int64_t total = 0;
    int64_t *d_offsets = nullptr;  // [T+1] node offsets of each tree
};

}  // namespace kdt

struct kdt_tree {
    int64_t N = 0;
    int D = 0;
    int layout = 0;                // 3: split dimension stored per node (widest extent)
    int device = 0;
    float4 *nodes = nullptr;       // N * float4_per_node(D), node t at nodes[t * float4_per_node(D)]
    float4 *nodes_alloc = nullptr; // allocation; 16-byte nodes start one slot in, so that the siblings
                                   // 2c+1 and 2c+2 share one 32-byte sector
    int32_t *ids = nullptr;        // layout > 0
    float *bbox = nullptr;         // device [2][3]: lo, hi of the first min(D,3) dims
    int *err = nullptr;            // device error word
    kdt::Model model;
    // learned-path statistics of the last learned query
    int64_t *stats = nullptr;      // device [2]: fallback count, sum of radius ratios (double bits)
    int64_t last_learned_q = 0;
    int last_learned_gate = KDT_GATE_ALL;
    // top tree levels staged in shared memory by the traversal kernels
    // (-1: the tuned or default depth for this tree's shape)
    int stage_levels = -1;
    // traversal steps between two claim rounds of a warp (-1: the tuned or
    // default value for this tree's shape)
    int claim_steps = -1;
    // depth of the bottom subtrees a traversal step processes whole (1 or 2;
    // -1: tuned or default)
    int inline_depth = -1;
    // steps a lane may take per call while they are light (-1: tuned or 1)
    int light_run = -1;
    // where the k-best heaps of k > 16 live (KDT_LIST_*; -1: the default)
    int large_k_list = -1;
    // test hook: traversal step bound (0: 3N + 3)
    uint32_t debug_step_cap = 0;
    // per-point payload in node order [N][payload_c] and node_of[input index]
    // (kdt_tree_set_payload; dropped by a rebuild)
    float *payload = nullptr;
    int32_t *node_of = nullptr;
    int payload_c = 0;
    // profiling
    bool profiling = false;
    void *prof = nullptr;
};

struct kdt_forest {
    kdt::ForestDesc f;
    float4 *nodes = nullptr;
    int32_t *ids = nullptr;
    float *bbox = nullptr;         // [T][2][3]
    int64_t *h_offsets = nullptr;  // host copy [T+1]
    int *err = nullptr;
    void *graph = nullptr;         // cached graph of the batched query
    int threads = 0;               // block size of the batched kernel (0: default 128)
    int claim_steps = 0;           // traversal steps between claim rounds (0: default for k)
    int inline_depth = 0;          // bottom-subtree depth per step (0: default 2)
    int light_run = 0;             // light steps per call (0: default 1)
};

// allocate an empty tree object with device arrays for N nodes of dimension D
extern "C" int kdt_tree_alloc_internal(int64_t N, int D, kdt_tree **out);

namespace kdt {
// staging depth (levels) for a query on tree t with k neighbours: the tree's
// own setting, else the tuned value for its shape, else the default
int stage_levels_for(const kdt_tree *t, int k);
int claim_steps_for(const kdt_tree *t, int k);
// default claim steps for k neighbours (no tuning)
int default_claim_steps_k(int k);
int inline_depth_for(const kdt_tree *t, int k);
int light_run_for(const kdt_tree *t, int k);
// whether a query for k neighbours keeps its heap in global scratch
bool heap_in_global(const kdt_tree *t, int k);
// lanes per query of the shuffle-inserted group list (1: one lane per query)
int list_group_for(const kdt_tree *t, int k);
// per-thread heap scratch for the traversal kernels (threads x k keys)
inline int64_t heap_scratch_threads() { return (int64_t)num_sms() * 1024; }
// builder shared by kdt_build and kdt_build_batched: fills nodes / ids / bbox
// widest: split dimension per node = widest extent of its points (T == 1,
// D <= 3), stored in the node (layout 3); else level mod D
int build_forest(const float *d_points, const int64_t *h_offsets, int T, int D, float4 *nodes,
                 int32_t *ids, float *bbox, int *err, cudaStream_t s, bool widest = false);
}  // namespace kdt
