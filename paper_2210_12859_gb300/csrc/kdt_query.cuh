// Query kernels (plain single-tree and batched forests) and their launcher
// interface.  Each node layout is instantiated in its own translation unit.
#pragma once

#include "kdt_traverse.cuh"

namespace kdt {

constexpr int REG_THREADS = 128;   // block size of the register-list kernels
constexpr int SMEM_THREADS = 128;  // block size of the shared-memory-list kernels
constexpr int MAX_REG_K = 16;
constexpr int STEPS_PER_CLAIM = 16; // traversal steps between two query claims of a warp

struct QueryArgs {
    const float4 *nodes = nullptr;     // single tree: its nodes; batched: all nodes
    const int32_t *ids = nullptr;
    int N = 0;                         // single tree size
    int D = 0;
    const float *queries = nullptr;
    int64_t Q = 0;
    const uint32_t *perm = nullptr;    // traversal order -> query index (optional)
    int k = 1;
    float r2 = 0.f;
    int32_t *out_ids = nullptr;
    float *out_d2 = nullptr;
    int32_t *visits = nullptr;         // COUNT variants
    int *err = nullptr;
    int staged = 0;                    // nodes staged in shared memory
    int claim_steps = STEPS_PER_CLAIM; // traversal steps a lane takes between two claim rounds
    int inline_depth = 2;              // bottom-subtree depth processed within one step (1, 2 or 3)
    int threads = 0;                   // block size of the forest kernel (0: the kernel's default)
    int light_run = 1;                 // steps a lane may take per call while they are light
    uint32_t step_cap = 0;             // traversal step bound (0: 3N + 3; a test hook lowers it)
    unsigned long long *counter = nullptr;  // dynamic work counter, zeroed before launch
    // k > 16: the per-thread heaps in global memory (k entries per thread, for
    // at most heap_threads threads; the grid is clamped to that), else (NULL)
    // in shared memory
    unsigned long long *heap = nullptr;
    int64_t heap_threads = 0;
    int group = 1;                     // k > 16: lanes per query holding a shuffle-inserted list (1: one lane)
    // batched forests
    int T = 1;
    const int64_t *node_off = nullptr; // [T+1]
    const int64_t *q_off = nullptr;    // [T+1]
    // learned radius proposal
    const float *r2q = nullptr;        // per-query cull radius of the bounded pass (mode 2)
    const unsigned long long *n_gate = nullptr;  // mode 2: only slots below *n_gate take r2q (NULL: all)
    unsigned long long *fb_count = nullptr;
    double *ratio_sum = nullptr;       // sum of proposed / true k-th radius (mode 2, exact queries)
};

// Claim the next queries for the lanes of the warp that need one: one atomic
// per warp, consecutive slots in lane order.  Returns the slot of this lane
// (or a value >= limit when the work is exhausted); all 32 lanes must call.
__device__ __forceinline__ int64_t claim_slot(bool need, unsigned long long *counter)
{
    const unsigned m = __ballot_sync(0xffffffffu, need);
    int64_t slot = INT64_MAX;
    if (m) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader)
            base = atomicAdd(counter, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (need)
            slot = (int64_t)(base + __popc(m & lane_mask_lt()));
    }
    return slot;
}

// kernel modes: results, visit counts, learned bounded pass, fallback pass
// (MODE_BOUNDED: per-query cull radius r2q; a query whose list is not full
// restarts in the same lane with the caller's radius)
enum : int { MODE_RESULTS = 0, MODE_VISITS = 1, MODE_BOUNDED = 2 };

// Ablation kernels (kdt_ablation.cu): flags select the variant
int launch_ablation(int layout, const QueryArgs &a, int flags, int mode, cudaStream_t s);

// Launch a traversal for one layout (mode: MODE_*).
int launch_query_layout0(const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s);
int launch_query_layout1(const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s);
int launch_query_layout2(const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s);
int launch_query_layout3(const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s);

inline int launch_query(int layout, const QueryArgs &a, bool ordered, int mode, bool batched, cudaStream_t s)
{
    switch (layout) {
    case 0: return launch_query_layout0(a, ordered, mode, batched, s);
    case 1: return launch_query_layout1(a, ordered, mode, batched, s);
    case 3: return launch_query_layout3(a, ordered, mode, batched, s);
    default: return launch_query_layout2(a, ordered, mode, batched, s);
    }
}

// nodes staged in shared memory for `levels` top levels of a tree of n nodes
inline int staged_for_levels(int64_t n, int levels)
{
    if (levels <= 0)
        return 0;
    int64_t cap = ((int64_t)1 << levels) - 1;
    return (int)(n < cap ? n : cap);
}

int grid_for_kernel(const void *fn, int threads, size_t smem);

}  // namespace kdt
