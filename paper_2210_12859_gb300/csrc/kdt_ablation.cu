// Ablation kernels for the traversal (ordered kNN / fcp, k <= 16, D <= 4).
//
// They exist to measure the choices around the stack-free traversal, which
// Sec. 3 presents without a speed claim against a stack-based one:
//   ABL_PLAIN        the stack-free machine of Sec. 3.2 as stated: one node per
//                    step, node before its close child, no inlined subtrees;
//   ABL_CLOSE_FIRST  the same machine with the node processed after its close
//                    subtree (the swap the footnote of Sec. 3.1 allows);
//   ABL_STACK        a stack-based traversal: process a node, push its far
//                    child with fl(sd^2), descend to the close child; a popped
//                    entry is culled against the radius at pop time.  This is
//                    the recursion of Sec. 3.1 with an explicit stack, so it
//                    processes the same nodes in the same order as ABL_PLAIN.
// All three keep the production kernel's lane refill and distance arithmetic,
// so results are bit-identical to kdt_knn's and visit counts to the oracle's.
#include "kdt_query_impl.cuh"

namespace kdt {
namespace {

constexpr int ABL_THREADS = 128;
enum : int { ABL_PLAIN = 0, ABL_CLOSE_FIRST = 1, ABL_STACK = 2 };
// far children pushed at most once per level of the current path (N < 2^30)
constexpr int STACK_DEPTH = 32;

__device__ __forceinline__ int level_of(int n) { return 31 - __clz(n + 1); }

template <int LAYOUT, int K, int VAR, bool VISITS>
__global__ void __launch_bounds__(ABL_THREADS) ablation_kernel(const QueryArgs a)
{
    constexpr int NC = LayoutTraits<LAYOUT>::NC;
    int64_t qi = -1;
    bool exhausted = false;
    float q[NC];
    RegList<K> list;
    int curr = 0, prev = -1, dim = 0, visits = 0, sp = 0;
    bool bad = false;
    uint32_t steps = 0;
    int stk_node[VAR == ABL_STACK ? STACK_DEPTH : 1];
    float stk_sd2[VAR == ABL_STACK ? STACK_DEPTH : 1];
    const uint32_t cap = 3u * (uint32_t)a.N + 3u;
    for (;;) {
        const bool need = qi < 0 && !exhausted;
        const int64_t slot = claim_slot(need, a.counter);
        if (need) {
            if (slot < a.Q) {
                qi = a.perm ? (int64_t)a.perm[slot] : slot;
                load_query<LAYOUT>(a.queries, qi, a.D, q);
                list.init(a.k, a.r2);
                curr = 0;
                prev = -1;
                dim = 0;
                visits = 0;
                sp = 0;
                steps = 0;
                bad = false;
            } else {
                exhausted = true;
            }
        }
        if (__all_sync(0xffffffffu, qi < 0))
            break;
        if (qi < 0)
            continue;
        bool done = false;
        for (int s = 0; s < a.claim_steps && !done; ++s) {
            if (++steps > cap) {
                bad = true;
                done = true;
                break;
            }
            if constexpr (VAR == ABL_STACK) {
                if (curr < 0) {
                    if (sp == 0) {
                        done = true;
                        break;
                    }
                    --sp;
                    curr = stk_node[sp];
                    if (stk_sd2[sp] > list.cull()) {
                        curr = -1;
                        continue;
                    }
                    dim = LAYOUT == 3 ? 0 : level_of(curr) % a.D;
                }
                const NodeVal<LAYOUT> nd = fetch<LAYOUT, false>(a.nodes, nullptr, 0, curr);
                process<LAYOUT>(nd, curr, a.ids, q, list);
                ++visits;
                const int sdim = split_dim_of<LAYOUT>(nd, dim);
                const float sd = __fsub_rn(select_dim<NC>(q, sdim), select_dim<NC>(nd.c, sdim));
                const int close = 2 * curr + 1 + (sd > 0.f);
                const int far = 2 * curr + 2 - (sd > 0.f);  // the other child; no 4 * curr (overflows past 2^29)
                if (far < a.N) {
                    if (sp < STACK_DEPTH) {
                        stk_node[sp] = far;
                        stk_sd2[sp] = __fmul_rn(sd, sd);
                        ++sp;
                    } else {
                        bad = true;
                    }
                }
                curr = close < a.N ? close : -1;
                dim = dim + 1 == a.D ? 0 : dim + 1;
            } else {
                const NodeVal<LAYOUT> nd = fetch<LAYOUT, false>(a.nodes, nullptr, 0, curr);
                const bool from_parent = prev < curr;
                if (VAR == ABL_PLAIN && from_parent) {
                    process<LAYOUT>(nd, curr, a.ids, q, list);
                    ++visits;
                }
                const int sdim = split_dim_of<LAYOUT>(nd, dim);
                const float sd = __fsub_rn(select_dim<NC>(q, sdim), select_dim<NC>(nd.c, sdim));
                const int close = 2 * curr + 1 + (sd > 0.f);
                const int far = 2 * curr + 2 - (sd > 0.f);  // the other child; no 4 * curr (overflows past 2^29)
                const int parent = (curr - 1) >> 1;
                int next;
                if (from_parent && close < a.N) {
                    next = close;
                } else if (from_parent || prev == close) {
                    // the close subtree is done (or missing, which the machine
                    // would step into and straight back out of)
                    if (VAR == ABL_CLOSE_FIRST) {
                        process<LAYOUT>(nd, curr, a.ids, q, list);
                        ++visits;
                    }
                    next = far < a.N && __fmul_rn(sd, sd) <= list.cull() ? far : parent;
                } else {
                    next = parent;
                }
                if (next < 0) {
                    done = true;
                    break;
                }
                if (next == parent)
                    dim = dim == 0 ? a.D - 1 : dim - 1;
                else
                    dim = dim + 1 == a.D ? 0 : dim + 1;
                prev = curr;
                curr = next;
            }
        }
        if (!done)
            continue;
        if (bad)
            atomicOr(a.err, ERR_TRAVERSAL);
        if (VISITS)
            a.visits[qi] = bad ? -1 : visits;
        else
            list.store(a.k, a.out_ids + qi * a.k, a.out_d2 + qi * a.k);
        qi = -1;
    }
}

template <int LAYOUT, int K>
int launch_abl_k(const QueryArgs &a, int var, bool visits, cudaStream_t s)
{
    switch (var * 2 + (visits ? 1 : 0)) {
    case 0: return launch_kernel(ablation_kernel<LAYOUT, K, ABL_PLAIN, false>, ABL_THREADS, 0, a, s);
    case 1: return launch_kernel(ablation_kernel<LAYOUT, K, ABL_PLAIN, true>, ABL_THREADS, 0, a, s);
    case 2: return launch_kernel(ablation_kernel<LAYOUT, K, ABL_CLOSE_FIRST, false>, ABL_THREADS, 0, a, s);
    case 3: return launch_kernel(ablation_kernel<LAYOUT, K, ABL_CLOSE_FIRST, true>, ABL_THREADS, 0, a, s);
    case 4: return launch_kernel(ablation_kernel<LAYOUT, K, ABL_STACK, false>, ABL_THREADS, 0, a, s);
    default: return launch_kernel(ablation_kernel<LAYOUT, K, ABL_STACK, true>, ABL_THREADS, 0, a, s);
    }
}

template <int LAYOUT>
int launch_abl_layout(const QueryArgs &a, int var, bool visits, cudaStream_t s)
{
    if (a.k <= 1)
        return launch_abl_k<LAYOUT, 1>(a, var, visits, s);
    if (a.k <= 8)
        return launch_abl_k<LAYOUT, 8>(a, var, visits, s);
    return launch_abl_k<LAYOUT, 16>(a, var, visits, s);
}

}  // namespace

int launch_ablation(int layout, const QueryArgs &a, int flags, int mode, cudaStream_t s)
{
    const int sel = flags & (KDT_PLAIN_STEP | KDT_CLOSE_FIRST | KDT_STACK);
    const int var = sel == KDT_PLAIN_STEP ? ABL_PLAIN : sel == KDT_CLOSE_FIRST ? ABL_CLOSE_FIRST : ABL_STACK;
    if (sel != KDT_PLAIN_STEP && sel != KDT_CLOSE_FIRST && sel != KDT_STACK)
        return set_error(KDT_EINVAL, "at most one of KDT_PLAIN_STEP, KDT_CLOSE_FIRST, KDT_STACK");
    if (flags & (KDT_UNORDERED | KDT_LEARNED))
        return set_error(KDT_EINVAL, "the traversal ablations are ordered and take no learned radius");
    if (a.k > 16)
        return set_error(KDT_EINVAL, "the traversal ablations take k <= 16 (got %d)", a.k);
    if (mode != MODE_RESULTS && mode != MODE_VISITS)
        return set_error(KDT_EINVAL, "unsupported ablation mode");
    const bool visits = mode == MODE_VISITS;
    switch (layout) {
    case 0: return launch_abl_layout<0>(a, var, visits, s);
    case 1: return launch_abl_layout<1>(a, var, visits, s);
    case 3: return launch_abl_layout<3>(a, var, visits, s);
    default: return set_error(KDT_EINVAL, "the traversal ablations take D <= 4");
    }
}

}  // namespace kdt
