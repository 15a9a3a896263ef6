// Learned radius proposal (not in the paper; results never change).
//
// A small MLP predicts, per query, the radius of its k-th nearest neighbour.
// The proposal r_p = margin * exp(y) seeds the cull radius of the ordered
// traversal (Sec. 3's shrinking radius then starts small instead of at the
// caller's radius).  The result is exact for every query whose list is full
// at the end (any point outside r_p is farther than the k points found inside
// it) or whose proposal did not shrink the caller's radius; the remaining
// queries are re-run with the caller's radius.
//
// Features: the query coordinates and log(max(d2_leaf, 1e-30)), where d2_leaf
// is the squared distance to the node where a greedy close-child descent from
// the root ends, normalised by training mean and standard deviation.
// Network: 4 -> 64 -> 64 -> 1 with ReLU, weights rounded to BF16, biases in
// FP32; the 64 x 64 contractions take BF16 operands (weights and hidden
// activations / gradients) with FP32 accumulation on the tensor cores
// (kdt_mlp_tc.cu), everything else is FP32.  Training: MSE against
// 0.5*log(d2 of the exact k-th neighbour), Adam, deterministic reductions.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "kdt_learned.cuh"
#include "kdt_query.cuh"

namespace kdt {


namespace {

constexpr int H = KDT_MLP_HIDDEN;
constexpr int P = KDT_MLP_PARAMS;
constexpr int OW1 = 0;
constexpr int OB1 = OW1 + H * 4;
constexpr int OW2 = OB1 + H;
constexpr int OB2 = OW2 + H * H;
constexpr int OW3 = OB2 + H;
constexpr int OB3 = OW3 + H;
static_assert(OB3 + 1 == P, "parameter layout");
static_assert(OW2 % 4 == 0, "W2 must be float4 aligned");

constexpr int TS = 64;  // minibatch sizes are multiples of this

__host__ __device__ inline bool is_weight(int i)
{
    return i < OB1 || (i >= OW2 && i < OB2) || (i >= OW3 && i < OB3);
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// master and rounded may be the same buffer (element-wise, in place), so
// neither pointer is restrict-qualified
__global__ void round_params_kernel(const float *master, float *rounded)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P)
        rounded[i] = is_weight(i) ? bf16_round(master[i]) : master[i];
}

__device__ __forceinline__ float leaf_feature(float d2) { return logf(fmaxf(d2, 1e-30f)); }

struct Norm {
    float mu[4];
    float sd[4];
};

__global__ void __launch_bounds__(256) features_kernel(const float4 *__restrict__ nodes, int N, int D,
                                                       const float *__restrict__ qs, int64_t Q, int staged,
                                                       bool stored, float *__restrict__ feat)
{
    extern __shared__ float4 s_nodes[];
    stage_nodes<0>(nodes, s_nodes, staged);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q; i += (int64_t)gridDim.x * blockDim.x) {
        float q[3];
        load_query<0>(qs, i, D, q);
        const float d2 = descent_leaf_d2(nodes, s_nodes, staged, N, D, q, stored);
        float4 f = make_float4(q[0], q[1], q[2], leaf_feature(d2));
        reinterpret_cast<float4 *>(feat)[i] = f;
    }
}

// fixed-order sum over blocks: grad[i] = sum_b partial[b][i]
__global__ void grad_reduce_kernel(const float *__restrict__ partial, int nb, float *__restrict__ grad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > P)
        return;
    float a = 0.f;
    for (int b = 0; b < nb; ++b)
        a = __fadd_rn(a, partial[(size_t)b * (P + 1) + i]);
    grad[i] = a;
}

__global__ void adam_kernel(float *__restrict__ master, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ grad, float lr, float bc1, float bc2,
                            float *__restrict__ rounded, double *__restrict__ loss_acc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0)
        *loss_acc += (double)grad[P];
    if (i >= P)
        return;
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    const float step = lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    const float wi = master[i] - step;
    master[i] = wi;
    rounded[i] = is_weight(i) ? bf16_round(wi) : wi;
}

__global__ void label_kernel(const float *__restrict__ d2, int64_t n, int k, float *__restrict__ label)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float v = d2[i * k + k - 1];
        v = v == v && v < 1e30f ? v : 1e30f;
        label[i] = 0.5f * logf(fmaxf(v, 1e-30f));
    }
}

// per-block sums (double) of x_j and x_j^2 for the 4 features and of the labels
constexpr int STAT_BLOCKS = 256;
__global__ void stats_kernel(const float *__restrict__ feat, const float *__restrict__ label, int64_t n,
                             double *__restrict__ out /* [STAT_BLOCKS][10] */)
{
    __shared__ double s[256][10];
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int j = 0; j < 4; ++j) {
            double x = feat[i * 4 + j];
            acc[j] += x;
            acc[4 + j] += x * x;
        }
        acc[8] += label[i];
        acc[9] += 1.0;
    }
    for (int j = 0; j < 10; ++j)
        s[threadIdx.x][j] = acc[j];
    __syncthreads();
    if (threadIdx.x < 10) {
        double a = 0;
        for (int t = 0; t < 256; ++t)
            a += s[t][threadIdx.x];
        out[blockIdx.x * 10 + threadIdx.x] = a;
    }
}

__global__ void normalize_kernel(float *__restrict__ feat, int64_t n, Norm nm)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < 4; ++j)
            feat[i * 4 + j] = __fdiv_rn(__fsub_rn(feat[i * 4 + j], nm.mu[j]), nm.sd[j]);
}

// ---- cost-weighted resampling of the training set
// The proposal exists to save traversal work, so each training query is
// weighted by the work the plain method spends on it: its processed nodes
// plus a floor (a tenth of the mean), which keeps cheap queries represented.
// Systematic resampling draws Qt samples with those probabilities (sample j
// takes the query whose cumulative-weight interval holds (j + u) / Qt of the
// total); a sort by hashed keys then shuffles them so that minibatches mix.

__global__ void visits_to_u64_kernel(const int32_t *__restrict__ v, int64_t n, unsigned long long *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = i < n ? (unsigned long long)(v[i] > 0 ? v[i] : 0) : 0ull;
}

__device__ __forceinline__ uint32_t hash32(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return (uint32_t)x;
}

// cdf: exclusive prefix sums of the visits [n+1]; weight of query i =
// visits_i + floor, so its interval is [cdf[i] + floor*i, cdf[i+1] + floor*(i+1))
__global__ void resample_kernel(const unsigned long long *__restrict__ cdf, int64_t n, double floor_w, double u,
                                uint64_t seed, uint32_t *__restrict__ keys, uint32_t *__restrict__ idx)
{
    const double total = (double)cdf[n] + floor_w * (double)n;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double target = ((double)j + u) * total / (double)n;
        int64_t lo = 0, hi = n - 1;  // largest i with start(i) <= target
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if ((double)cdf[mid] + floor_w * (double)mid <= target)
                lo = mid;
            else
                hi = mid - 1;
        }
        idx[j] = (uint32_t)lo;
        keys[j] = hash32(seed * 0x9e3779b97f4a7c15ull + (uint64_t)j);
    }
}

__global__ void gather_samples_kernel(const uint32_t *__restrict__ idx, int64_t n, const float4 *__restrict__ feat,
                                      const float *__restrict__ lab, float4 *__restrict__ feat_out,
                                      float *__restrict__ lab_out)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = idx[j];
        feat_out[j] = feat[i];
        lab_out[j] = lab[i];
    }
}

__global__ void fill_inf_kernel(float *p, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = __int_as_float(0x7f800000);
}

unsigned grid_of(int64_t n)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16));
}

struct Dev {
    void *p = nullptr;
    cudaStream_t s;
    explicit Dev(cudaStream_t s_) : s(s_) {}
    ~Dev()
    {
        if (p)
            cudaFreeAsync(p, s);
    }
};

uint64_t splitmix(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int ensure_params(kdt_tree *t)
{
    if (!t->model.d_params)
        KDT_CUDA(cudaMalloc(&t->model.d_params, P * sizeof(float)));
    return KDT_OK;
}

int ensure_stats(kdt_tree *t)
{
    if (!t->stats)
        KDT_CUDA(cudaMalloc(&t->stats, 4 * sizeof(int64_t)));
    return KDT_OK;
}

int upload_rounded(const float *h_params, float *d_rounded, cudaStream_t s)
{
    KDT_CUDA(cudaMemcpyAsync(d_rounded, h_params, P * sizeof(float), cudaMemcpyHostToDevice, s));
    KDT_LAUNCH round_params_kernel<<<(P + 255) / 256, 256, 0, s>>>(d_rounded, d_rounded);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

int check_learned_tree(const kdt_tree *t)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (t->D > 3)
        return set_error(KDT_EINVAL, "the radius model needs D <= 3 (tree has D = %d)", t->D);
    return KDT_OK;
}

// queries of the last learned call that took the proposal (counted: the far
// queries the Morton pass counted, for KDT_GATE_FAR)
int64_t learned_gated(const kdt_tree *t, int64_t counted)
{
    switch (t->last_learned_gate) {
    case KDT_GATE_FAR: return counted;
    case KDT_GATE_NONE: return 0;
    default: return t->last_learned_q;
    }
}

}  // namespace

void fill_inf(float *p, int64_t n, cudaStream_t s)
{
    if (n > 0)
        KDT_LAUNCH fill_inf_kernel<<<grid_of(n), 256, 0, s>>>(p, n);
}

void free_model(kdt_tree *t)
{
    if (t->model.d_params)
        cudaFree(t->model.d_params);
    t->model.d_params = nullptr;
    if (t->stats)
        cudaFree(t->stats);
    t->stats = nullptr;
}

int run_learned_query(kdt_tree *t, const float *d_q, int64_t Q, int k, float r2, int flags, int32_t *d_ids,
                      float *d_d2, int32_t *d_visits, cudaStream_t s)
{
    KDT_TRY(check_learned_tree(t));
    if (!t->model.trained)
        return set_error(KDT_ENOMODEL, "the tree has no trained radius model");
    KDT_TRY(ensure_stats(t));
    const int gate = t->model.gate;
    t->last_learned_q = Q;
    t->last_learned_gate = gate;
    // stats slots: [0] fallback count, [1] ratio sum (double bits), [2] gated queries
    KDT_CUDA(cudaMemsetAsync(t->stats, 0, 3 * sizeof(int64_t), s));
    if (gate == KDT_GATE_NONE)  // the proposal pays on none of these queries: the plain traversal
        return run_query(t, d_q, Q, k, r2, flags & ~KDT_LEARNED, d_ids ? MODE_RESULTS : MODE_VISITS, d_ids, d_d2,
                         d_visits, s);
    // far queries only: their cost classes come first in the traversal order,
    // and the Morton pass counts them
    if (gate == KDT_GATE_FAR)
        flags |= KDT_MORTON | KDT_COST_ORDER;
    const bool morton = flags & KDT_MORTON;
    const size_t heap_bytes = heap_in_global(t, k) ? (size_t)heap_scratch_threads() * k * 8 : 0;
    size_t off_w = 0, off_r2 = 1 << 15;
    size_t off_h = off_r2 + (((size_t)Q * 4 + 255) & ~(size_t)255);
    size_t off_m = off_h + heap_bytes;
    size_t bytes = off_m + (morton ? morton_scratch_bytes(Q) : 0);
    Dev sc(s);
    KDT_CUDA(cudaMallocAsync(&sc.p, bytes, s));
    char *B = (char *)sc.p;
    float *wts = (float *)(B + off_w);                                  // P floats
    unsigned long long *counter = (unsigned long long *)(B + 20480);    // 3 x u64 after the weights
    unsigned long long *n_far = gate == KDT_GATE_FAR ? (unsigned long long *)(B + 20736) : nullptr;
    float *r2q = (float *)(B + off_r2);
    uint32_t *perm = nullptr;
    if (morton)
        KDT_TRY(morton_order(d_q, Q, t->D, t->bbox, 1, nullptr, 0, (flags & KDT_COST_ORDER) ? t->nodes : nullptr,
                             t->N, t->layout == 3, B + off_m, &perm, s, n_far));
    KDT_LAUNCH round_params_kernel<<<(P + 255) / 256, 256, 0, s>>>(t->model.d_params, wts);
    KDT_TRY(tc_radius(t, wts, d_q, Q, perm, r2, r2q, s, n_far));
    if (n_far)
        KDT_CUDA(cudaMemcpyAsync(t->stats + 2, n_far, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));

    QueryArgs a;
    a.nodes = t->nodes;
    a.ids = t->ids;
    a.N = (int)t->N;
    a.D = t->D;
    a.queries = d_q;
    a.Q = Q;
    a.perm = perm;
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
    a.inline_depth = inline_depth_for(t, k) >= 2 ? inline_depth_for(t, k) : 1;  // depth 0 is plain-query only
    a.r2q = r2q;
    a.n_gate = n_far;
    if (heap_bytes) {
        a.heap = (unsigned long long *)(B + off_h);
        a.heap_threads = heap_scratch_threads();
    }
    a.fb_count = (unsigned long long *)t->stats;
    a.ratio_sum = (double *)(t->stats + 1);
    const bool ordered = !(flags & KDT_UNORDERED);
    KDT_TRY(launch_query(t->layout, a, ordered, MODE_BOUNDED, false, s));
    return KDT_OK;
}

// The automatic gate, from the training queries: the processed nodes the
// plain traversal needs and those the learned forms need (all queries gated,
// or the far ones), counted exactly, and the cost of the network pass (the
// descent for the features, the MLP) per gated query in processed-node
// equivalents: its time per query over the plain traversal's time per
// processed node.  A form's score is the nodes it saves minus that cost times
// the queries it gates; the best positive score wins, else no query is gated.
// (Timing the whole forms on the training set does not transfer: at 2^20
// queries the traversal's launch tail weighs differently than at full size.)
int choose_gate(kdt_tree *t, const float *d_q, int64_t n, int k, int qflags, cudaStream_t s)
{
    qflags &= ~(KDT_LEARNED | KDT_PLAIN_STEP | KDT_CLOSE_FIRST | KDT_STACK);
    Dev buf(s);
    const size_t vis_b = ((size_t)n * 4 + 255) & ~(size_t)255;
    const size_t out_b = ((size_t)n * k * 4 + 255) & ~(size_t)255;
    KDT_CUDA(cudaMallocAsync(&buf.p, vis_b + 2 * out_b + 3 * vis_b + (1 << 15), s));
    char *B = (char *)buf.p;
    int32_t *vis = (int32_t *)B;
    int32_t *ids = (int32_t *)(B + vis_b);
    float *d2 = (float *)(B + vis_b + out_b);
    float *r2q = (float *)(B + vis_b + 2 * out_b);
    float *wts = (float *)(B + 4 * vis_b + 2 * out_b);
    std::vector<int32_t> hv(n);
    int rc = KDT_OK;
    auto total = [&](double *out) {
        if (rc != KDT_OK)
            return;
        if (cudaMemcpyAsync(hv.data(), vis, (size_t)n * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = set_error(KDT_ECUDA, "visit count copy failed");
            return;
        }
        double sum = 0.0;
        for (int64_t i = 0; i < n; ++i)
            sum += hv[i];
        *out = sum;
    };
    double v_plain = 0, v_all = 0, v_far = 0;
    rc = run_query(t, d_q, n, k, INFINITY, qflags, MODE_VISITS, nullptr, nullptr, vis, s);
    total(&v_plain);
    t->model.gate = KDT_GATE_ALL;
    if (rc == KDT_OK)
        rc = run_learned_query(t, d_q, n, k, INFINITY, qflags, nullptr, nullptr, vis, s);
    total(&v_all);
    t->model.gate = KDT_GATE_FAR;
    if (rc == KDT_OK)
        rc = run_learned_query(t, d_q, n, k, INFINITY, qflags, nullptr, nullptr, vis, s);
    total(&v_far);
    int64_t stats[3] = {0, 0, 0};
    if (rc == KDT_OK && (cudaMemcpyAsync(stats, t->stats, sizeof(stats), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                         cudaStreamSynchronize(s) != cudaSuccess))
        rc = set_error(KDT_ECUDA, "stats copy failed");
    const double n_far = (double)stats[2];
    // times: the plain query, and the network pass over all n queries
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == KDT_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = set_error(KDT_ECUDA, "event create");
    if (rc == KDT_OK)
        KDT_LAUNCH round_params_kernel<<<(P + 255) / 256, 256, 0, s>>>(t->model.d_params, wts);
    auto best_of = [&](bool net, float *best) {
        *best = 3.4e38f;
        for (int rep = 0; rep < 4 && rc == KDT_OK; ++rep) {
            float ms = 0.f;
            if (cudaEventRecord(e0, s) != cudaSuccess)
                rc = set_error(KDT_ECUDA, "event record");
            if (rc == KDT_OK)
                rc = net ? tc_radius(t, wts, d_q, n, nullptr, INFINITY, r2q, s)
                         : run_query(t, d_q, n, k, INFINITY, qflags, MODE_RESULTS, ids, d2, nullptr, s);
            if (rc == KDT_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                 cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = set_error(KDT_ECUDA, "event timing failed");
            if (rep > 0 && ms < *best)
                *best = ms;
        }
    };
    float t_plain = 0.f, t_net = 0.f;
    best_of(false, &t_plain);
    best_of(true, &t_net);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (rc != KDT_OK)
        return rc;
    // network pass per query, in processed-node equivalents of the plain traversal
    const double c = (t_net / (double)n) / (t_plain / std::max(v_plain, 1.0));
    // every query of a gated call, gated or not, runs in the bounded pass, and
    // a node there costs more than one of the plain traversal (restart state
    // and its registers): fitted to two full-size forms (clustered k = 8 with
    // the far gate, surface k = 32 with every query gated) as 5.9 % per node
    // beside a fixed per-query part, taken as 8 % so that a gate is chosen
    // only for a clear saving
    constexpr double BOUNDED_NODE_COST = 1.08;
    const double score_all = v_plain - BOUNDED_NODE_COST * v_all - c * (double)n;
    const double score_far = v_plain - BOUNDED_NODE_COST * v_far - c * n_far;
    int best = KDT_GATE_NONE;
    double best_score = 0.0;
    if (score_all > best_score) {
        best = KDT_GATE_ALL;
        best_score = score_all;
    }
    if (score_far > best_score)
        best = KDT_GATE_FAR;
    t->model.gate = best;
    t->model.gate_cost = (float)c;
    return KDT_OK;
}

}  // namespace kdt

using namespace kdt;

extern "C" {

int kdt_descent_features(const kdt_tree *t, const float *d_q, int64_t Q, float *d_feat, void *stream)
{
    KDT_TRY(check_learned_tree(t));
    if (Q < 0 || (Q > 0 && (!d_q || !d_feat)))
        return set_error(KDT_EINVAL, "bad query or feature arguments");
    if (Q == 0)
        return KDT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int staged = staged_for_levels(t->N, stage_levels_for(t, 8));
    KDT_LAUNCH features_kernel<<<grid_of(Q), 256, staged * 16, s>>>(t->nodes, (int)t->N, t->D, d_q, Q, staged,
                                                                        t->layout == 3, d_feat);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

int kdt_mlp_forward(const float *h_params, const float *d_x, int64_t n, float *d_y, void *stream)
{
    if (!h_params || n < 0 || (n > 0 && (!d_x || !d_y)))
        return set_error(KDT_EINVAL, "bad MLP arguments");
    if (n == 0)
        return KDT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Dev w(s);
    const size_t wb = ((P * 4 + 255) & ~(size_t)255);
    KDT_CUDA(cudaMallocAsync(&w.p, wb + 256, s));
    int *err = (int *)((char *)w.p + wb);
    KDT_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    KDT_TRY(upload_rounded(h_params, (float *)w.p, s));
    KDT_TRY(tc_forward((const float *)w.p, d_x, n, d_y, err, s));
    int h = 0;
    KDT_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KDT_CUDA(cudaStreamSynchronize(s));
    if (h)
        return set_error(KDT_ECUDA, "the tensor-core MMA did not signal completion in time");
    return KDT_OK;
}

// loss and gradient on the tensor cores (BF16 operands, FP32 accumulation),
// then the fixed-order sum over the blocks
static int loss_grad_dev(const float *d_w, const float *d_x, const float *d_label, int64_t begin, int64_t count,
                         float *d_partial, float *d_grad, int *d_err, cudaStream_t s)
{
    int nb = 0;
    KDT_TRY(tc_loss_grad(d_w, d_x, d_label, begin, count, d_partial, d_err, s, &nb));
    KDT_LAUNCH grad_reduce_kernel<<<(P + 1 + 255) / 256, 256, 0, s>>>(d_partial, nb, d_grad);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

int kdt_mlp_loss_grad(const float *h_params, const float *d_x, const float *d_label, int64_t n, float *h_loss,
                      float *h_grad, void *stream)
{
    if (!h_params || n < 1 || !d_x || !d_label || !h_grad)
        return set_error(KDT_EINVAL, "bad MLP gradient arguments");
    if (n > (1 << 24))
        return set_error(KDT_EINVAL, "n must be <= 2^24");
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((n + 127) / 128);
    Dev buf(s);
    size_t wb = ((P * 4 + 255) & ~(size_t)255);
    KDT_CUDA(cudaMallocAsync(&buf.p, 2 * wb + 256 + (size_t)nb * (P + 1) * 4, s));
    float *w = (float *)buf.p;
    float *grad = (float *)((char *)buf.p + wb);
    int *err = (int *)((char *)buf.p + 2 * wb);
    float *partial = (float *)((char *)buf.p + 2 * wb + 256);
    KDT_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    KDT_TRY(upload_rounded(h_params, w, s));
    KDT_TRY(loss_grad_dev(w, d_x, d_label, 0, n, partial, grad, err, s));
    std::vector<float> g(P + 1);
    int h = 0;
    KDT_CUDA(cudaMemcpyAsync(g.data(), grad, (P + 1) * sizeof(float), cudaMemcpyDeviceToHost, s));
    KDT_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KDT_CUDA(cudaStreamSynchronize(s));
    if (h)
        return set_error(KDT_ECUDA, "the tensor-core MMA did not signal completion in time");
    memcpy(h_grad, g.data(), P * sizeof(float));
    if (h_loss)
        *h_loss = g[P] / (float)n;
    return KDT_OK;
}

int kdt_radius_model_train(kdt_tree *t, const float *d_q, int64_t Qt, int k, const kdt_train_opts *opts,
                           float *final_loss, void *stream)
{
    KDT_TRY(check_learned_tree(t));
    if (Qt < 1 || !d_q || k < 1 || k > 64)
        return set_error(KDT_EINVAL, "bad training arguments");
    if (Qt > ((int64_t)1 << 26))
        return set_error(KDT_EINVAL, "at most 2^26 training queries");
    cudaStream_t s = (cudaStream_t)stream;
    kdt_train_opts o{6, 1024, 2e-3f, 1, 0.f, 0.02f, 0, KDT_GATE_AUTO, 0};
    if (opts) {
        if (opts->epochs > 0)
            o.epochs = opts->epochs;
        if (opts->batch > 0)
            o.batch = opts->batch;
        if (opts->lr > 0)
            o.lr = opts->lr;
        o.seed = opts->seed;
        if (opts->margin > 0)
            o.margin = opts->margin;
        if (opts->fallback_target > 0)
            o.fallback_target = std::min(opts->fallback_target, 0.5f);
        o.uniform_weights = opts->uniform_weights;
        o.gate = opts->gate;
        o.query_flags = opts->query_flags;
    }
    if (o.gate < KDT_GATE_AUTO || o.gate > KDT_GATE_NONE)
        return set_error(KDT_EINVAL, "gate must be one of KDT_GATE_* (got %d)", o.gate);
    o.batch = std::max(TS, (o.batch / TS) * TS);
    KDT_TRY(ensure_params(t));

    // buffers: d2 [Qt][k] + ids (for labels), features, labels, weights, Adam state, partials, stats
    const int nbmax = (o.batch + TS - 1) / TS;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t o_d2 = 0, o_ids = o_d2 + al((size_t)Qt * k * 4), o_feat = o_ids + al((size_t)Qt * k * 4);
    size_t o_lab = o_feat + al((size_t)Qt * 16), o_w = o_lab + al((size_t)Qt * 4), o_m = o_w + al(P * 4);
    size_t o_v = o_m + al(P * 4), o_g = o_v + al(P * 4), o_part = o_g + al((P + 1) * 4);
    size_t o_stat = o_part + al((size_t)nbmax * (P + 1) * 4), o_loss = o_stat + al(STAT_BLOCKS * 10 * 8);
    // resampling: visits, cdf + scan scratch, keys / idx / sort temporaries, resampled features and labels
    const bool weighted = !o.uniform_weights;
    size_t o_vis = o_loss + 256, o_cdf = o_vis + al((size_t)Qt * 4);
    size_t o_scan = o_cdf + al(((size_t)Qt + 1) * 8), o_keys = o_scan + al((scan_scratch_elems(Qt + 1) + 1) * 8);
    size_t o_idx = o_keys + al((size_t)Qt * 4), o_tk = o_idx + al((size_t)Qt * 4), o_tv = o_tk + al((size_t)Qt * 4);
    size_t o_rs = o_tv + al((size_t)Qt * 4), o_f2 = o_rs + al((radix_scratch_elems(Qt) + 1) * 4);
    size_t o_l2 = o_f2 + al((size_t)Qt * 16);
    size_t bytes = weighted ? o_l2 + al((size_t)Qt * 4) : o_loss + 256;
    Dev buf(s);
    KDT_CUDA(cudaMallocAsync(&buf.p, bytes, s));
    char *B = (char *)buf.p;
    float *d2 = (float *)(B + o_d2);
    int32_t *ids = (int32_t *)(B + o_ids);
    float *feat = (float *)(B + o_feat);
    float *lab = (float *)(B + o_lab);
    float *w = (float *)(B + o_w);
    float *m = (float *)(B + o_m);
    float *v = (float *)(B + o_v);
    float *grad = (float *)(B + o_g);
    float *part = (float *)(B + o_part);
    double *stat = (double *)(B + o_stat);
    double *loss_acc = (double *)(B + o_loss);

    // exact labels from the plain method
    KDT_TRY(run_query(t, d_q, Qt, k, INFINITY, KDT_MORTON, MODE_RESULTS, ids, d2, nullptr, s));
    KDT_LAUNCH label_kernel<<<grid_of(Qt), 256, 0, s>>>(d2, Qt, k, lab);
    KDT_TRY(kdt_descent_features(t, d_q, Qt, feat, s));
    if (weighted) {
        int32_t *vis = (int32_t *)(B + o_vis);
        unsigned long long *cdf = (unsigned long long *)(B + o_cdf);
        uint32_t *keys = (uint32_t *)(B + o_keys), *idx = (uint32_t *)(B + o_idx);
        KDT_TRY(run_query(t, d_q, Qt, k, INFINITY, KDT_MORTON, MODE_VISITS, nullptr, nullptr, vis, s));
        KDT_LAUNCH visits_to_u64_kernel<<<grid_of(Qt + 1), 256, 0, s>>>(vis, Qt, cdf);
        KDT_TRY(exclusive_scan_u64(cdf, Qt + 1, (unsigned long long *)(B + o_scan), s));
        unsigned long long total = 0;
        KDT_CUDA(cudaMemcpyAsync(&total, cdf + Qt, 8, cudaMemcpyDeviceToHost, s));
        KDT_CUDA(cudaStreamSynchronize(s));
        const double floor_w = std::max(1.0, 0.1 * (double)total / (double)Qt);
        uint64_t su = o.seed * 0xD1B54A32D192ED03ull + 99;
        const double u = (double)(splitmix(su) >> 11) * (1.0 / 9007199254740992.0);
        KDT_LAUNCH resample_kernel<<<grid_of(Qt), 256, 0, s>>>(cdf, Qt, floor_w, u, o.seed, keys, idx);
        KDT_TRY(radix_sort_pairs(keys, idx, (uint32_t *)(B + o_tk), (uint32_t *)(B + o_tv), Qt, 32,
                                 (uint32_t *)(B + o_rs), s));
        float *feat2 = (float *)(B + o_f2), *lab2 = (float *)(B + o_l2);
        KDT_LAUNCH gather_samples_kernel<<<grid_of(Qt), 256, 0, s>>>(idx, Qt, (const float4 *)feat, lab,
                                                                     (float4 *)feat2, lab2);
        feat = feat2;
        lab = lab2;
    }
    KDT_LAUNCH stats_kernel<<<STAT_BLOCKS, 256, 0, s>>>(feat, lab, Qt, stat);
    std::vector<double> hs(STAT_BLOCKS * 10);
    KDT_CUDA(cudaMemcpyAsync(hs.data(), stat, hs.size() * 8, cudaMemcpyDeviceToHost, s));
    KDT_CUDA(cudaStreamSynchronize(s));
    double sum[10] = {0};
    for (int b = 0; b < STAT_BLOCKS; ++b)
        for (int j = 0; j < 10; ++j)
            sum[j] += hs[b * 10 + j];
    Norm nm;
    for (int j = 0; j < 4; ++j) {
        double mu = sum[j] / sum[9];
        double var = std::max(sum[4 + j] / sum[9] - mu * mu, 0.0);
        nm.mu[j] = (float)mu;
        nm.sd[j] = (float)std::max(sqrt(var), 1e-6);
    }
    const double label_mean = sum[8] / sum[9];
    KDT_LAUNCH normalize_kernel<<<grid_of(Qt), 256, 0, s>>>(feat, Qt, nm);

    // He-uniform initial weights, zero biases, output bias at the label mean
    std::vector<float> h(P, 0.f);
    uint64_t st = o.seed * 0x2545F4914F6CDD1Dull + 12345;
    auto uni = [&](float lim) { return (float)(((splitmix(st) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * lim; };
    for (int i = 0; i < H * 4; ++i)
        h[OW1 + i] = uni(sqrtf(6.f / 4.f));
    for (int i = 0; i < H * H; ++i)
        h[OW2 + i] = uni(sqrtf(6.f / H));
    for (int i = 0; i < H; ++i)
        h[OW3 + i] = uni(sqrtf(6.f / H)) * 0.1f;
    h[OB3] = (float)label_mean;
    KDT_CUDA(cudaMemcpyAsync(t->model.d_params, h.data(), P * 4, cudaMemcpyHostToDevice, s));
    KDT_LAUNCH round_params_kernel<<<(P + 255) / 256, 256, 0, s>>>(t->model.d_params, w);
    KDT_CUDA(cudaMemsetAsync(m, 0, P * 4, s));
    KDT_CUDA(cudaMemsetAsync(v, 0, P * 4, s));

    double b1t = 1.0, b2t = 1.0;
    float last = 0.f;
    // step size decays along a half cosine from lr to 0 over the run
    const int64_t steps_total = (int64_t)o.epochs * ((Qt + o.batch - 1) / o.batch);
    int64_t step = 0;
    for (int ep = 0; ep < o.epochs; ++ep) {
        KDT_CUDA(cudaMemsetAsync(loss_acc, 0, 8, s));
        for (int64_t b0 = 0; b0 < Qt; b0 += o.batch) {
            const int64_t cnt = std::min<int64_t>(o.batch, Qt - b0);
            KDT_TRY(loss_grad_dev(w, feat, lab, b0, cnt, part, grad, t->err, s));
            b1t *= 0.9;
            b2t *= 0.999;
            const float lr = (float)(0.5 * o.lr * (1.0 + cos(M_PI * (double)step / (double)steps_total)));
            ++step;
            KDT_LAUNCH adam_kernel<<<(P + 255) / 256, 256, 0, s>>>(t->model.d_params, m, v, grad, lr, (float)(1.0 - b1t),
                                                       (float)(1.0 - b2t), w, loss_acc);
        }
        KDT_CUDA(cudaGetLastError());
        double l = 0;
        KDT_CUDA(cudaMemcpyAsync(&l, loss_acc, 8, cudaMemcpyDeviceToHost, s));
        KDT_CUDA(cudaStreamSynchronize(s));
        last = (float)(l / (double)Qt);
    }
    float margin = o.margin;
    if (!(margin > 0.f)) {
        // calibrate: the proposal falls short for a query iff its residual
        // label - prediction exceeds log(margin); take the (1 - target)
        // quantile of the training residuals (of the cost-weighted sample:
        // re-runs then cost about a fraction `target` of the plain work)
        float *pred = d2;  // reuse: Qt floats
        KDT_TRY(tc_forward(w, feat, Qt, pred, t->err, s));
        std::vector<float> hp(Qt), hl(Qt);
        KDT_CUDA(cudaMemcpyAsync(hp.data(), pred, Qt * 4, cudaMemcpyDeviceToHost, s));
        KDT_CUDA(cudaMemcpyAsync(hl.data(), lab, Qt * 4, cudaMemcpyDeviceToHost, s));
        KDT_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < Qt; ++i)
            hp[i] = hl[i] - hp[i];
        int64_t at = std::min<int64_t>(Qt - 1, (int64_t)((1.0 - o.fallback_target) * (double)Qt));
        std::nth_element(hp.begin(), hp.begin() + at, hp.end());
        margin = expf(std::min(std::max(hp[at], -0.7f), 2.8f));
    }
    for (int j = 0; j < 4; ++j) {
        t->model.norm[j] = nm.mu[j];
        t->model.norm[4 + j] = nm.sd[j];
    }
    t->model.margin = margin;
    t->model.k_trained = k;
    t->model.trained = true;
    if (o.gate != KDT_GATE_AUTO) {
        t->model.gate = o.gate;
    } else {
        const int qf = o.query_flags ? o.query_flags : (KDT_MORTON | KDT_COST_ORDER);
        KDT_TRY(choose_gate(t, d_q, std::min<int64_t>(Qt, (int64_t)1 << 20), k, qf, s));
    }
    if (final_loss)
        *final_loss = last;
    return KDT_OK;
}

int kdt_radius_model_get(const kdt_tree *t, float *h_params, float *h_norm, float *margin)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (!t->model.trained)
        return set_error(KDT_ENOMODEL, "the tree has no radius model");
    if (h_params)
        KDT_CUDA(cudaMemcpy(h_params, t->model.d_params, P * sizeof(float), cudaMemcpyDeviceToHost));
    if (h_norm)
        memcpy(h_norm, t->model.norm, sizeof(t->model.norm));
    if (margin)
        *margin = t->model.margin;
    return KDT_OK;
}

int kdt_radius_model_set(kdt_tree *t, const float *h_params, const float *h_norm, float margin)
{
    KDT_TRY(check_learned_tree(t));
    if (!h_params || !h_norm || !(margin > 0.f))
        return set_error(KDT_EINVAL, "bad model arguments");
    for (int j = 0; j < 4; ++j)
        if (!(h_norm[4 + j] > 0.f))
            return set_error(KDT_EINVAL, "feature standard deviations must be > 0");
    KDT_TRY(ensure_params(t));
    KDT_CUDA(cudaMemcpy(t->model.d_params, h_params, P * sizeof(float), cudaMemcpyHostToDevice));
    memcpy(t->model.norm, h_norm, sizeof(t->model.norm));
    t->model.margin = margin;
    t->model.trained = true;
    return KDT_OK;
}

static const char MODEL_MAGIC[8] = {'K', 'D', 'T', 'R', 'A', 'D', 'M', '1'};

int kdt_radius_model_save(const kdt_tree *t, const char *path)
{
    if (!path)
        return set_error(KDT_EINVAL, "path is NULL");
    std::vector<float> p(P);
    float norm[8], margin;
    KDT_TRY(kdt_radius_model_get(t, p.data(), norm, &margin));
    FILE *f = fopen(path, "wb");
    if (!f)
        return set_error(KDT_EIO, "cannot open %s for writing", path);
    int32_t hdr[4] = {2, H, P, t->model.k_trained};
    const int32_t gate = t->model.gate;
    bool ok = fwrite(MODEL_MAGIC, 1, 8, f) == 8 && fwrite(hdr, 4, 4, f) == 4 && fwrite(norm, 4, 8, f) == 8 &&
              fwrite(&margin, 4, 1, f) == 1 && fwrite(p.data(), 4, P, f) == (size_t)P && fwrite(&gate, 4, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    return ok ? KDT_OK : set_error(KDT_EIO, "write to %s failed", path);
}

int kdt_radius_model_load(kdt_tree *t, const char *path)
{
    KDT_TRY(check_learned_tree(t));
    if (!path)
        return set_error(KDT_EINVAL, "path is NULL");
    FILE *f = fopen(path, "rb");
    if (!f)
        return set_error(KDT_EIO, "cannot open %s", path);
    char magic[8];
    int32_t hdr[4];
    float norm[8], margin;
    std::vector<float> p(P);
    // version 1: no gate (every query takes the proposal); version 2: the gate follows the parameters
    int32_t gate = KDT_GATE_ALL;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, MODEL_MAGIC, 8) == 0 && fread(hdr, 4, 4, f) == 4 &&
              (hdr[0] == 1 || hdr[0] == 2) && hdr[1] == H && hdr[2] == P && fread(norm, 4, 8, f) == 8 &&
              fread(&margin, 4, 1, f) == 1 && fread(p.data(), 4, P, f) == (size_t)P &&
              (hdr[0] == 1 || (fread(&gate, 4, 1, f) == 1 && gate >= KDT_GATE_ALL && gate <= KDT_GATE_NONE));
    fclose(f);
    if (!ok)
        return set_error(KDT_EIO, "%s is not a radius model file of a known version", path);
    KDT_TRY(kdt_radius_model_set(t, p.data(), norm, margin));
    t->model.k_trained = hdr[3];
    t->model.gate = gate;
    return KDT_OK;
}

int kdt_radius_model_gate(const kdt_tree *t, int *gate)
{
    if (!t || !gate)
        return set_error(KDT_EINVAL, "tree or out pointer is NULL");
    if (!t->model.trained)
        return set_error(KDT_ENOMODEL, "the tree has no radius model");
    *gate = t->model.gate;
    return KDT_OK;
}

int kdt_radius_model_set_gate(kdt_tree *t, int gate)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (!t->model.trained)
        return set_error(KDT_ENOMODEL, "the tree has no radius model");
    if (gate < KDT_GATE_ALL || gate > KDT_GATE_NONE)
        return set_error(KDT_EINVAL, "gate must be KDT_GATE_ALL, KDT_GATE_FAR or KDT_GATE_NONE (got %d)", gate);
    t->model.gate = gate;
    return KDT_OK;
}

int kdt_learned_gated(const kdt_tree *t, int64_t *gated, void *stream)
{
    if (!t || !gated)
        return set_error(KDT_EINVAL, "tree or out pointer is NULL");
    if (!t->stats)
        return set_error(KDT_ENOMODEL, "no learned query has run on this tree");
    int64_t h[3];
    KDT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    KDT_CUDA(cudaMemcpy(h, t->stats, sizeof(h), cudaMemcpyDeviceToHost));
    *gated = learned_gated(t, h[2]);
    return KDT_OK;
}

int kdt_learned_stats(const kdt_tree *t, int64_t *fallbacks, double *radius_ratio, void *stream)
{
    if (!t)
        return set_error(KDT_EINVAL, "tree is NULL");
    if (!t->stats)
        return set_error(KDT_ENOMODEL, "no learned query has run on this tree");
    int64_t h[3];
    KDT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    KDT_CUDA(cudaMemcpy(h, t->stats, sizeof(h), cudaMemcpyDeviceToHost));
    double ratio_sum;
    memcpy(&ratio_sum, &h[1], 8);
    const int64_t gated = learned_gated(t, h[2]);
    const int64_t exact = gated - h[0];
    if (fallbacks)
        *fallbacks = h[0];
    if (radius_ratio)
        *radius_ratio = exact > 0 ? ratio_sum / (double)exact : 0.0;
    return KDT_OK;
}

}  // extern "C"
