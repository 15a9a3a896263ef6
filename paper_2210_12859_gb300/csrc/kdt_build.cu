// GPU builder of left-balanced, complete, level-order k-d trees.
//
// The tree is the one a serial median builder produces (Sec. 4 states that a
// parallel builder emits exactly that tree): for a subtree of n points at
// level l the points are ordered by (coordinate l mod D, input index), the
// element of rank L(n) (left-subtree size of a complete tree of n nodes)
// becomes the node, the lower ranks form the left subtree and the higher ranks
// the right subtree.
//
// Design.  For every dimension e the builder keeps a list of point indices
// sorted by (coordinate e, input index) (one stable radix sort per dimension).
// Positions of every list are laid out in IN-ORDER: the points of the subtree
// of node t always occupy the in-order range of t's subtree.  Then, at level l
// with split dimension d:
//   * the list of d needs no work: within a segment the element at in-order
//     position p goes left iff p lies in the left subtree's in-order range,
//     becomes the node iff p is t's own in-order position, else goes right.
//     That is purely topological (closed-form in-order <-> node maps), so one
//     pass over the list writes each point's side and emits the level's nodes;
//   * every other list still needed later is stably partitioned inside each
//     segment into [left | node | right] with a segmented scan of the side
//     flags, which keeps each part sorted by its own key.
// All of it is streaming passes over arrays of N elements plus gathers of a
// 1-byte side array (N bytes, resident in L2).  T > 1 trees are built in the
// same passes: lists are first sorted by (tree, coordinate, index) and every
// position knows its tree.
#include <algorithm>
#include <vector>

#include "kdt_internal.cuh"

namespace kdt {
namespace {

constexpr int BT = 256;          // threads per block, builder kernels
constexpr int PITEMS = 4;        // items per thread, partition scan
constexpr int PTILE = BT * PITEMS;

enum : uint8_t { SIDE_LEFT = 0, SIDE_NODE = 1, SIDE_RIGHT = 2 };

struct Where {
    int64_t base;   // first position of the position's tree
    int64_t n;      // size of that tree
};

__device__ __forceinline__ Where locate(int64_t p, int T, const int64_t *__restrict__ off,
                                        const int32_t *__restrict__ tree_of, int64_t total)
{
    if (T == 1)
        return {0, total};
    int i = tree_of[p];
    int64_t b = off[i];
    return {b, off[i + 1] - b};
}

__global__ void prep_keys_kernel(const float *__restrict__ pts, int64_t total, int D, int e,
                                 uint32_t *__restrict__ keys, uint32_t *__restrict__ vals, int *__restrict__ err)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        float x = pts[i * D + e];
        if (!isfinite(x))
            atomicOr(err, ERR_NONFINITE);
        keys[i] = float_key(x);
        vals[i] = (uint32_t)i;
    }
}

__global__ void tree_keys_kernel(const uint32_t *__restrict__ vals, const int32_t *__restrict__ tree_of, int64_t total,
                                 uint32_t *__restrict__ keys)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint32_t)tree_of[vals[i]];
}

__global__ void tree_of_kernel(const int64_t *__restrict__ off, int T, int64_t total, int32_t *__restrict__ tree_of)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        // last tree whose offset is <= i (empty trees are skipped by taking the last)
        int lo = 0, hi = T - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= i)
                lo = mid;
            else
                hi = mid - 1;
        }
        tree_of[i] = lo;
    }
}

// bounding box of the first min(D,3) dims of each tree: the extremes of the
// per-dimension sorted lists
__global__ void bbox_kernel(const float *__restrict__ pts, int D, const uint32_t *const *lists,
                            const int64_t *__restrict__ off, int T, float *__restrict__ bbox)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T)
        return;
    int64_t a = off[i], b = off[i + 1];
    for (int e = 0; e < 3; ++e) {
        float lo = 0.f, hi = 0.f;
        if (e < D && b > a) {
            lo = pts[(int64_t)lists[e][a] * D + e];
            hi = pts[(int64_t)lists[e][b - 1] * D + e];
        }
        bbox[i * 6 + e] = lo;
        bbox[i * 6 + 3 + e] = hi;
    }
}

// Level l, split list: record each point's side and emit the level's nodes.
__global__ void assign_kernel(const uint32_t *__restrict__ list, int64_t total, int l, int T,
                              const int64_t *__restrict__ off, const int32_t *__restrict__ tree_of,
                              const float *__restrict__ pts, int D, uint8_t *__restrict__ side,
                              float4 *__restrict__ nodes, int32_t *__restrict__ ids)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
        Where w = locate(p, T, off, tree_of, total);
        Topo tp(w.n);
        if (l > tp.H)
            continue;
        int64_t u = tp.node_at(p - w.base);
        int lu = Topo::level(u);
        if (lu < l)
            continue;
        uint32_t pid = list[p];
        if (lu == l) {
            side[pid] = SIDE_NODE;
            const float *c = pts + (int64_t)pid * D;
            int32_t local = (int32_t)(pid - (uint32_t)w.base);
            int64_t node = w.base + u;
            if (D <= 3) {
                float4 v = make_float4(c[0], D > 1 ? c[1] : 0.f, D > 2 ? c[2] : 0.f, __int_as_float(local));
                nodes[node] = v;
            } else if (D == 4) {
                nodes[node] = make_float4(c[0], c[1], c[2], c[3]);
                ids[node] = local;
            } else {
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = j < D ? c[j] : 0.f;
                nodes[2 * node] = make_float4(v[0], v[1], v[2], v[3]);
                nodes[2 * node + 1] = make_float4(v[4], v[5], v[6], v[7]);
                ids[node] = local;
            }
        } else {
            int bit = (int)(((u + 1) >> (lu - l - 1)) & 1);
            side[pid] = bit ? SIDE_RIGHT : SIDE_LEFT;
        }
    }
}

// ---- stored split dimension (widest extent of the node's points)

struct ListPtrs {
    const uint32_t *p[8];
};

// split dimension of every node of level l: within the node's segment each
// list is sorted by its coordinate, so its first and last elements give the
// extent; the widest dimension wins, ties to the lowest index
__global__ void widest_kernel(ListPtrs lists, int64_t n, int l, const float *__restrict__ pts, int D,
                              uint8_t *__restrict__ node_dim)
{
    const int64_t first = ((int64_t)1 << l) - 1;
    const int64_t count = (first + 1 < n - first) ? first + 1 : n - first;
    const Topo tp(n);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = first + i;
        const int64_t a = tp.inorder(tp.leftmost(t));
        const int64_t b = tp.inorder(tp.rightmost(t));
        int best = 0;
        float best_ext = -1.f;
        for (int e = 0; e < D; ++e) {
            const float lo = pts[(int64_t)lists.p[e][a] * D + e];
            const float hi = pts[(int64_t)lists.p[e][b] * D + e];
            const float ext = __fsub_rn(hi, lo);
            if (ext > best_ext) {
                best_ext = ext;
                best = e;
            }
        }
        node_dim[t] = (uint8_t)best;
    }
}

// level l with per-node split dimensions: the element at in-order position p
// of its segment's split list decides the side (single tree, D <= 3)
__global__ void assign_widest_kernel(ListPtrs lists, int64_t n, int l, const uint8_t *__restrict__ node_dim,
                                     const float *__restrict__ pts, int D, uint8_t *__restrict__ side,
                                     float4 *__restrict__ nodes)
{
    const Topo tp(n);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        if (l > tp.H)
            continue;
        const int64_t u = tp.node_at(p);
        const int lu = Topo::level(u);
        if (lu < l)
            continue;
        const int64_t t = Topo::ancestor(u, lu, l);
        const int e = node_dim[t];
        const uint32_t pid = lists.p[e][p];
        if (lu == l) {
            side[pid] = SIDE_NODE;
            const float *c = pts + (int64_t)pid * D;
            const uint32_t word = pid | ((uint32_t)e << NODE_DIM_SHIFT);
            nodes[u] = make_float4(c[0], D > 1 ? c[1] : 0.f, D > 2 ? c[2] : 0.f, __uint_as_float(word));
        } else {
            const int bit = (int)(((u + 1) >> (lu - l - 1)) & 1);
            side[pid] = bit ? SIDE_RIGHT : SIDE_LEFT;
        }
    }
}

// ---- segmented stable partition of a non-split list

struct Seg {
    uint32_t f;                 // segment head inside the range
    unsigned long long v;       // left count (low 32) | right count (high 32)
};

__device__ __forceinline__ Seg seg_op(Seg a, Seg b)
{
    Seg r;
    r.f = a.f | b.f;
    r.v = b.f ? b.v : a.v + b.v;
    return r;
}

struct Item {
    Seg s;          // value of this position
    int64_t dest;   // -1: copy through
    uint32_t pid;
    uint8_t side;
    int64_t s_t, in_t;  // segment start and node in-order position (relative)
    int64_t base, n;
};

__device__ __forceinline__ void load_item(const uint32_t *__restrict__ in, int64_t p, int64_t total, int l, int T,
                                          const int64_t *__restrict__ off, const int32_t *__restrict__ tree_of,
                                          const uint8_t *__restrict__ side, Item &it)
{
    it.s.f = 1;
    it.s.v = 0;
    it.dest = -1;
    if (p >= total)
        return;
    it.pid = in[p];
    Where w = locate(p, T, off, tree_of, total);
    Topo tp(w.n);
    if (l > tp.H)
        return;
    int64_t lp = p - w.base;
    int64_t u = tp.node_at(lp);
    int lu = Topo::level(u);
    if (lu < l)
        return;
    int64_t t = Topo::ancestor(u, lu, l);
    it.s_t = tp.inorder(tp.leftmost(t));
    it.in_t = tp.inorder(t);
    it.base = w.base;
    it.n = w.n;
    it.side = side[it.pid];
    it.s.f = lp == it.s_t;
    it.s.v = (it.side == SIDE_LEFT ? 1ull : 0ull) | (it.side == SIDE_RIGHT ? (1ull << 32) : 0ull);
    it.dest = 0;
}

__device__ __forceinline__ Seg shfl_up_seg(Seg x, int o)
{
    Seg r;
    r.f = __shfl_up_sync(0xffffffffu, x.f, o);
    r.v = __shfl_up_sync(0xffffffffu, x.v, o);
    return r;
}

// exclusive segmented block scan of one Seg per thread; *agg = block total
__device__ __forceinline__ Seg block_exclusive_seg(Seg x, Seg *s_warp, Seg *agg)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    Seg inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Seg y = shfl_up_seg(inc, o);
        if (lane >= o)
            inc = seg_op(y, inc);
    }
    Seg ex = shfl_up_seg(inc, 1);
    if (lane == 0)
        ex = Seg{0, 0};
    if (lane == 31)
        s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        Seg a = lane < nw ? s_warp[lane] : Seg{0, 0};
        Seg ai = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Seg y = shfl_up_seg(ai, o);
            if (lane >= o)
                ai = seg_op(y, ai);
        }
        Seg ae = shfl_up_seg(ai, 1);
        if (lane == 0)
            ae = Seg{0, 0};
        if (lane < nw)
            s_warp[lane] = ae;
        if (lane == nw - 1)
            s_warp[32] = ai;
    }
    __syncthreads();
    Seg r = seg_op(s_warp[w], ex);
    *agg = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(BT) part_reduce_kernel(const uint32_t *__restrict__ in, int64_t total, int l, int T,
                                                         const int64_t *__restrict__ off,
                                                         const int32_t *__restrict__ tree_of,
                                                         const uint8_t *__restrict__ side, Seg *__restrict__ tiles)
{
    __shared__ Seg s_warp[33];
    const int64_t base = (int64_t)blockIdx.x * PTILE + (int64_t)threadIdx.x * PITEMS;
    Seg acc{0, 0};
#pragma unroll
    for (int j = 0; j < PITEMS; ++j) {
        Item it;
        load_item(in, base + j, total, l, T, off, tree_of, side, it);
        acc = seg_op(acc, it.s);
    }
    Seg agg;
    block_exclusive_seg(acc, s_warp, &agg);
    if (threadIdx.x == 0)
        tiles[blockIdx.x] = agg;
}

__global__ void __launch_bounds__(1024) part_tiles_kernel(Seg *__restrict__ tiles, int64_t nt)
{
    __shared__ Seg s_warp[33];
    Seg carry{0, 0};
    for (int64_t b = 0; b < nt; b += 1024) {
        int64_t i = b + threadIdx.x;
        Seg x = i < nt ? tiles[i] : Seg{0, 0};
        Seg agg;
        Seg ex = block_exclusive_seg(x, s_warp, &agg);
        if (i < nt)
            tiles[i] = seg_op(carry, ex);
        carry = seg_op(carry, agg);
    }
}

__global__ void __launch_bounds__(BT) part_scatter_kernel(const uint32_t *__restrict__ in, int64_t total, int l, int T,
                                                          const int64_t *__restrict__ off,
                                                          const int32_t *__restrict__ tree_of,
                                                          const uint8_t *__restrict__ side,
                                                          const Seg *__restrict__ tiles, uint32_t *__restrict__ out)
{
    __shared__ Seg s_warp[33];
    const int64_t base = (int64_t)blockIdx.x * PTILE + (int64_t)threadIdx.x * PITEMS;
    Item it[PITEMS];
    Seg acc{0, 0};
#pragma unroll
    for (int j = 0; j < PITEMS; ++j) {
        load_item(in, base + j, total, l, T, off, tree_of, side, it[j]);
        acc = seg_op(acc, it[j].s);
    }
    Seg agg;
    Seg run = seg_op(tiles[blockIdx.x], block_exclusive_seg(acc, s_warp, &agg));
#pragma unroll
    for (int j = 0; j < PITEMS; ++j) {
        int64_t p = base + j;
        if (p >= total)
            break;
        // run is the exclusive prefix of this item within its segment (a head
        // starts from zero)
        Seg ex = it[j].s.f ? Seg{1, 0} : run;
        if (it[j].dest < 0) {
            out[p] = it[j].pid;
        } else {
            uint32_t lb = (uint32_t)(ex.v & 0xffffffffu);
            uint32_t rb = (uint32_t)(ex.v >> 32);
            int64_t d;
            if (it[j].side == SIDE_NODE)
                d = it[j].in_t;
            else if (it[j].side == SIDE_LEFT)
                d = it[j].s_t + lb;
            else
                d = it[j].in_t + 1 + rb;
            if (d >= 0 && d < it[j].n)  // always true for consistent side flags
                out[it[j].base + d] = it[j].pid;
        }
        run = seg_op(run, it[j].s);
    }
}

inline unsigned grid_for(int64_t n)
{
    int64_t b = (n + BT - 1) / BT;
    int64_t cap = (int64_t)num_sms() * 16;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf()
    {
        if (p)
            cudaFreeAsync(p, s);
    }
};

}  // namespace

int build_forest(const float *d_points, const int64_t *h_off, int T, int D, float4 *nodes, int32_t *ids, float *bbox,
                 int *err, cudaStream_t s, bool widest)
{
    const int64_t total = h_off[T];
    int maxH = 0;
    for (int i = 0; i < T; ++i) {
        int64_t n = h_off[i + 1] - h_off[i];
        if (n > 0)
            maxH = std::max(maxH, floor_log2((uint64_t)n));
    }
    if (total == 0)
        return KDT_OK;

    // scratch: D lists + spare + 2 key arrays (u32), side (u8), tree_of (i32),
    // offsets (i64), tiles (Seg), radix scratch
    const int64_t ptiles = (total + PTILE - 1) / PTILE;
    const size_t rs = radix_scratch_elems(total);
    size_t bytes = 0;
    auto take = [&](size_t b) {
        size_t o = bytes;
        bytes += (b + 255) & ~(size_t)255;
        return o;
    };
    size_t o_lists = take((size_t)(D + 1) * total * 4);
    size_t o_keys = take((size_t)2 * total * 4);
    size_t o_side = take((size_t)total);
    size_t o_tree = take(T > 1 ? (size_t)total * 4 : 0);
    size_t o_off = take((size_t)(T + 1) * 8);
    size_t o_tiles = take((size_t)ptiles * sizeof(Seg));
    size_t o_rs = take(rs * 4);
    size_t o_lptr = take((size_t)8 * sizeof(uint32_t *));
    size_t o_dim = take(widest ? (size_t)total : 0);
    DevBuf buf;
    buf.s = s;
    KDT_CUDA(cudaMallocAsync(&buf.p, bytes, s));
    char *B = (char *)buf.p;
    uint32_t *lists[9];
    for (int e = 0; e <= D; ++e)
        lists[e] = (uint32_t *)(B + o_lists) + (size_t)e * total;
    uint32_t *spare = lists[D];
    uint32_t *k0 = (uint32_t *)(B + o_keys);
    uint32_t *k1 = k0 + total;
    uint8_t *side = (uint8_t *)(B + o_side);
    int32_t *tree_of = T > 1 ? (int32_t *)(B + o_tree) : nullptr;
    int64_t *d_off = (int64_t *)(B + o_off);
    Seg *tiles = (Seg *)(B + o_tiles);
    uint32_t *rscr = (uint32_t *)(B + o_rs);
    uint32_t **d_lptr = (uint32_t **)(B + o_lptr);
    uint8_t *node_dim = (uint8_t *)(B + o_dim);

    KDT_CUDA(cudaMemcpyAsync(d_off, h_off, (T + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const unsigned g = grid_for(total);
    if (T > 1)
        KDT_LAUNCH tree_of_kernel<<<g, BT, 0, s>>>(d_off, T, total, tree_of);
    int tbits = T > 1 ? floor_log2((uint64_t)(T - 1)) + 1 : 0;

    // per-dimension lists sorted by (tree, coordinate, index)
    for (int e = 0; e < D; ++e) {
        KDT_LAUNCH prep_keys_kernel<<<g, BT, 0, s>>>(d_points, total, D, e, k0, lists[e], err);
        KDT_TRY(radix_sort_pairs(k0, lists[e], k1, spare, total, 32, rscr, s));
        if (T > 1) {
            KDT_LAUNCH tree_keys_kernel<<<g, BT, 0, s>>>(lists[e], tree_of, total, k0);
            KDT_TRY(radix_sort_pairs(k0, lists[e], k1, spare, total, tbits, rscr, s));
        }
    }
    KDT_CUDA(cudaMemcpyAsync(d_lptr, lists, 8 * sizeof(uint32_t *), cudaMemcpyHostToDevice, s));
    KDT_LAUNCH bbox_kernel<<<(T + 127) / 128, 128, 0, s>>>(d_points, D, d_lptr, d_off, T, bbox);

    if (widest) {
        // per-node split dimensions: every list may be a node's split list,
        // so every list is partitioned at every level that has a successor
        for (int l = 0; l <= maxH; ++l) {
            ListPtrs lp;
            for (int e = 0; e < 8; ++e)
                lp.p[e] = e < D ? lists[e] : nullptr;
            const int64_t level_nodes = std::min<int64_t>((int64_t)1 << l, total - (((int64_t)1 << l) - 1));
            KDT_LAUNCH widest_kernel<<<grid_for(level_nodes), BT, 0, s>>>(lp, total, l, d_points, D, node_dim);
            KDT_LAUNCH assign_widest_kernel<<<g, BT, 0, s>>>(lp, total, l, node_dim, d_points, D, side, nodes);
            if (l < maxH) {
                for (int e = 0; e < D; ++e) {
                    KDT_LAUNCH part_reduce_kernel<<<(unsigned)ptiles, BT, 0, s>>>(lists[e], total, l, T, d_off, tree_of,
                                                                                  side, tiles);
                    KDT_LAUNCH part_tiles_kernel<<<1, 1024, 0, s>>>(tiles, ptiles);
                    KDT_LAUNCH part_scatter_kernel<<<(unsigned)ptiles, BT, 0, s>>>(lists[e], total, l, T, d_off,
                                                                                   tree_of, side, tiles, spare);
                    std::swap(lists[e], spare);
                }
            }
            KDT_CUDA(cudaGetLastError());
        }
        return KDT_OK;
    }
    for (int l = 0; l <= maxH; ++l) {
        const int d = l % D;
        KDT_LAUNCH assign_kernel<<<g, BT, 0, s>>>(lists[d], total, l, T, d_off, tree_of, d_points, D, side, nodes, ids);
        for (int e = 0; e < D; ++e) {
            if (e == d)
                continue;
            // next level that splits on e
            int nl = l + ((e - d + D) % D);
            if (nl > maxH)
                continue;
            KDT_LAUNCH part_reduce_kernel<<<(unsigned)ptiles, BT, 0, s>>>(lists[e], total, l, T, d_off, tree_of, side, tiles);
            KDT_LAUNCH part_tiles_kernel<<<1, 1024, 0, s>>>(tiles, ptiles);
            KDT_LAUNCH part_scatter_kernel<<<(unsigned)ptiles, BT, 0, s>>>(lists[e], total, l, T, d_off, tree_of, side, tiles,
                                                                spare);
            std::swap(lists[e], spare);
        }
        KDT_CUDA(cudaGetLastError());
    }
    return KDT_OK;
}

}  // namespace kdt
