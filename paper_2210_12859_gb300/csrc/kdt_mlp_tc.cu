// Radius-model inference on the 5th-generation tensor cores (not in the paper).
//
// The model is 4 -> 64 -> 64 -> 1 (ReLU).  Layers 1 and 3 are 256 + 64
// multiply-adds per query and stay on the CUDA cores; the 64 x 64 hidden layer
// (4096 multiply-adds per query) is a dense contraction and runs as
// tcgen05.mma: a CTA of 128 threads takes 128 queries at a time, each thread
// writes its query's 64 hidden activations (BF16) as one row of the A tile in
// shared memory, one thread issues four M=128 N=64 K=16 MMAs against W2 (BF16,
// the B tile, loaded once per CTA) into a 128 x 64 FP32 accumulator in tensor
// memory, and each thread reads its own row back with tcgen05.ld.
//
// Shared-memory operands use the no-swizzle K-major layout: 8 x 16-byte core
// matrices, consecutive along K at 128 bytes (leading byte offset), 8-row
// groups at 1024 bytes (stride byte offset).
#include <cuda_bf16.h>

#include <algorithm>

#include "kdt_learned.cuh"
#include "kdt_query.cuh"
#include "kdt_traverse.cuh"

namespace kdt {
namespace {

constexpr int H = KDT_MLP_HIDDEN;
constexpr int OW1 = 0, OB1 = OW1 + H * 4, OW2 = OB1 + H, OB2 = OW2 + H * H;
static_assert(OB2 + 2 * H + 1 == KDT_MLP_PARAMS, "parameter layout");

constexpr int TILE_M = 128;                    // queries per MMA tile = threads per CTA
constexpr int A_BYTES = TILE_M * H * 2;        // 16 KB
constexpr int B_BYTES = H * H * 2;             // 8 KB
constexpr int SMEM_FIXED = A_BYTES + B_BYTES + 4096;  // + small weights, barrier, TMEM slot
constexpr uint32_t TMEM_COLS = 64;
constexpr long long WAIT_LIMIT = 1ll << 26;   // mbarrier polls before giving up

// instruction descriptor, kind::f16: D = F32 (bits 4-5), A = B = BF16 (bits
// 7-9, 10-12), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                           ((uint32_t)(TILE_M >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4, leading byte offset >> 4 (bits
// 16-29), stride byte offset >> 4 (bits 32-45), descriptor version 1 (bit 46),
// no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// byte offset of element (row r, k) in a K-major no-swizzle tile with K = 64
__device__ __forceinline__ uint32_t kmajor_offset(int r, int k)
{
    return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// true once the phase with the given parity has completed; false after
// WAIT_LIMIT polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done)
            return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    const float *wts;          // rounded parameters (P floats)
    int64_t n;                 // queries / samples
    // radius mode
    const float4 *nodes;
    int N, D;
    bool stored;               // split dimension stored in the nodes
    const float *queries;
    const uint32_t *perm;
    float mu[4], sd[4];
    float margin, r2_user;
    float *r2q;
    const unsigned long long *n_lim;  // radius mode: only the first *n_lim entries of perm (NULL: all n)
    // forward mode
    const float *x;            // normalised features [n][4]
    float *y;
    int *err;
};

// MODE 0: descent features -> normalise -> MLP -> per-query cull radius.
// MODE 1: given normalised features -> MLP output.
template <int MODE>
__global__ void __launch_bounds__(TILE_M) mlp_tc_kernel(const TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;
    unsigned char *sB = smem + A_BYTES;
    float *sw = reinterpret_cast<float *>(smem + A_BYTES + B_BYTES);  // W1, b1, b2, w3, b3
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + A_BYTES + B_BYTES + 3584);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + A_BYTES + B_BYTES + 3600);
    int *abort_flag = reinterpret_cast<int *>(smem + A_BYTES + B_BYTES + 3608);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    // operands that stay for the whole launch
    for (int i = tid; i < H * H; i += TILE_M) {
        const int nrow = i / H, k = i % H;  // B[k][n] = W2[n][k]: row n of the K-major tile
        *reinterpret_cast<__nv_bfloat16 *>(sB + kmajor_offset(nrow, k)) = __float2bfloat16_rn(a.wts[OW2 + i]);
    }
    for (int i = tid; i < OW2; i += TILE_M)
        sw[i] = a.wts[i];
    for (int i = tid; i < 2 * H + 1; i += TILE_M)
        sw[OW2 + i] = a.wts[OB2 + i];  // b2, w3, b3
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;
    const float *b2 = sw + OW2;
    const float *w3 = b2 + H;
    const float b3 = w3[H];

    uint32_t phase = 0;
    int64_t n = a.n;
    if (MODE == 0 && a.n_lim)
        n = min(n, (int64_t)*a.n_lim);
    const int64_t tiles = (n + TILE_M - 1) / TILE_M;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t i = tile * TILE_M + tid;
        const bool valid = i < n;
        int64_t qi = 0;
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (valid) {
            if constexpr (MODE == 0) {
                qi = a.perm ? (int64_t)a.perm[i] : i;
                float q[3];
                load_query<0>(a.queries, qi, a.D, q);
                const float d2 = descent_leaf_d2(a.nodes, nullptr, 0, a.N, a.D, q, a.stored);
                const float f[4] = {q[0], q[1], q[2], logf(fmaxf(d2, 1e-30f))};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    x[j] = __fdiv_rn(__fsub_rn(f[j], a.mu[j]), a.sd[j]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    x[j] = a.x[i * 4 + j];
            }
        }
        // layer 1 on the CUDA cores, ReLU, BF16 row of the A tile
#pragma unroll
        for (int g = 0; g < H / 8; ++g) {
            __align__(16) __nv_bfloat16 h[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int o = g * 8 + e;
                float acc = sw[OB1 + o];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc = __fmaf_rn(sw[OW1 + 4 * o + j], x[j], acc);
                h[e] = __float2bfloat16_rn(fmaxf(acc, 0.f));
            }
            *reinterpret_cast<uint4 *>(sA + kmajor_offset(tid, g * 8)) = *reinterpret_cast<const uint4 *>(h);
        }
        // make the tile visible to the tensor cores, then one thread issues
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
#pragma unroll
            for (int ks = 0; ks < H / 16; ++ks) {
                const uint64_t ad = smem_desc(a0 + ks * 256, 128, 1024);
                const uint64_t bd = smem_desc(b0 + ks * 256, 128, 1024);
                const uint32_t acc = ks > 0;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(bar))
                         : "memory");
            if (!mbar_wait(bar, phase))
                *abort_flag = 1;
        }
        __syncthreads();
        if (*abort_flag)
            break;
        phase ^= 1u;
        tc_fence_after();
        // each warp reads its 32 TMEM lanes: thread tid holds row tid = its query
        float y = b3;
#pragma unroll
        for (int c = 0; c < H; c += 16) {
            float v[16];
            tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 16; ++e)
                y = __fmaf_rn(w3[c + e], fmaxf(__fadd_rn(v[e], b2[c + e]), 0.f), y);
        }
        if (valid) {
            if constexpr (MODE == 0) {
                const float r = __fmul_rn(a.margin, expf(y));
                const float rp2 = __fmul_rn(r, r);
                a.r2q[qi] = (rp2 == rp2 && rp2 < a.r2_user) ? rp2 : a.r2_user;
            } else {
                a.y[i] = y;
            }
        }
        tc_fence_before();
        __syncthreads();  // A tile and accumulator free for the next tile
    }
    if (*abort_flag) {
        // the MMAs did not signal in time: record it, give them one more
        // bounded wait before the accumulator is released
        if (tid == 0) {
            atomicOr(a.err, ERR_TRAVERSAL);
            mbar_wait(bar, phase);
        }
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------- training
//
// Loss and gradient of the model on the tensor cores, BF16 operands and FP32
// accumulation, one CTA of 128 threads per tile of 128 samples (thread r holds
// sample r).  With H1 the hidden activations of layer 1 (BF16) and G2 the
// gradient at the pre-activations of the hidden layer (BF16), three
// contractions of the validated shape (M = 128, N = 64, both operands K-major
// in shared memory, FP32 accumulator in TMEM):
//   Z2  = H1 . W2^T           rows = samples, K = 64   (TMEM columns 0..63)
//   dH1 = G2 . W2             rows = samples, K = 64   (columns 64..127)
//   dW2 = G2^T . H1           rows = the 64 hidden units (padded to 128 with
//                             zero rows), K = 128 samples  (columns 128..191)
// Layers 1 and 3, the ReLU masks and the sums over the tile's samples of the
// small gradients (W1, b1, b2, w3, b3, the loss) run on the CUDA cores in
// FP32, in a fixed order.  partial[blockIdx.x][P + 1] receives the tile's sums
// (slot P: the squared errors).
constexpr int GK = TILE_M;                      // samples per tile: K of the weight-gradient contraction
constexpr int RED_LD = H + 1;                   // row stride of the FP32 reduction buffer (no bank conflicts)
constexpr int G_W2 = 0;                         // B of Z2: row i, K = j
constexpr int G_W2T = G_W2 + H * H * 2;         // B of dH1: row j, K = i
constexpr int G_H1 = G_W2T + H * H * 2;         // A of Z2: row r, K = j
constexpr int G_G2 = G_H1 + TILE_M * H * 2;     // A of dH1: row r, K = i
constexpr int G_G2T = G_G2 + TILE_M * H * 2;    // A of dW2: row i (64..127 zero), K = r
constexpr int G_H1T = G_G2T + 128 * GK * 2;     // B of dW2: row j, K = r
constexpr int G_RED = G_H1T + H * GK * 2;       // FP32 [128][RED_LD]
constexpr int G_SW = G_RED + ((TILE_M * RED_LD * 4 + 1023) & ~1023);  // W1, b1, b2, w3, b3 (FP32)
constexpr int G_BAR = G_SW + 2048;              // mbarrier, TMEM slot, abort flag
constexpr int G_SMEM = G_BAR + 64;
constexpr uint32_t G_TMEM_COLS = 256;
static_assert(G_H1 % 1024 == 0 && G_G2 % 1024 == 0 && G_G2T % 1024 == 0 && G_H1T % 1024 == 0, "tile alignment");
static_assert(4 * H + 3 * H + 1 <= 2048 / 4, "small weights");

// byte offset of element (row r, k) in a K-major no-swizzle tile with K columns
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// ksteps MMAs of K = 16 into the accumulator at taddr (the first one
// overwrites it); sbo: the tiles' 8-row group strides (K * 16 bytes)
__device__ __forceinline__ void mma_k_major(uint32_t taddr, uint32_t a0, uint32_t b0, int ksteps, uint32_t sbo_a,
                                            uint32_t sbo_b)
{
    for (int ks = 0; ks < ksteps; ++ks) {
        const uint64_t ad = smem_desc(a0 + ks * 256, 128, sbo_a);
        const uint64_t bd = smem_desc(b0 + ks * 256, 128, sbo_b);
        const uint32_t acc = ks > 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
    }
}

// column sums of the reduction buffer in row order: thread t < H sums column t
__device__ __forceinline__ float column_sum(const float *red, int t)
{
    float a = 0.f;
    for (int r = 0; r < TILE_M; ++r)
        a = __fadd_rn(a, red[r * RED_LD + t]);
    return a;
}

__global__ void __launch_bounds__(TILE_M) mlp_tc_grad_kernel(const float *__restrict__ wts, const float *__restrict__ x,
                                                             const float *__restrict__ label, int64_t begin,
                                                             int64_t count, float inv_count,
                                                             float *__restrict__ partial, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    float *red = reinterpret_cast<float *>(smem + G_RED);
    float *sw = reinterpret_cast<float *>(smem + G_SW);  // W1 [4H], b1 [H], b2 [H], w3 [H], b3
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + G_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + G_BAR + 16);
    int *abort_flag = reinterpret_cast<int *>(smem + G_BAR + 24);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    float *out = partial + (size_t)blockIdx.x * (KDT_MLP_PARAMS + 1);

    for (int e = tid; e < H * H; e += TILE_M) {
        const int i = e / H, j = e % H;
        const __nv_bfloat16 v = __float2bfloat16_rn(wts[OW2 + e]);  // W2[i][j] (BF16-valued already)
        *reinterpret_cast<__nv_bfloat16 *>(smem + G_W2 + kmajor_off(i, j, H)) = v;
        *reinterpret_cast<__nv_bfloat16 *>(smem + G_W2T + kmajor_off(j, i, H)) = v;
    }
    for (int e = tid; e < 64 * GK; e += TILE_M)
        *reinterpret_cast<__nv_bfloat16 *>(smem + G_G2T + kmajor_off(64 + e / GK, e % GK, GK)) = __float2bfloat16_rn(0.f);
    for (int i = tid; i < 5 * H; i += TILE_M)
        sw[i] = wts[i];  // W1, b1
    for (int i = tid; i < 2 * H + 1; i += TILE_M)
        sw[5 * H + i] = wts[OB2 + i];  // b2, w3, b3
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(G_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const float *W1 = sw;
    const float *b1 = sw + 4 * H;
    const float *b2 = sw + 5 * H;
    const float *w3 = sw + 6 * H;
    const float b3v = wts[OB2 + 2 * H];

    const int64_t idx = begin + (int64_t)blockIdx.x * TILE_M + tid;
    const bool valid = idx < begin + count;
    float xs[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        xs[j] = valid ? x[idx * 4 + j] : 0.f;
    const float lab = valid ? label[idx] : 0.f;
    __syncthreads();  // small weights in place

    // layer 1 (FP32), ReLU, BF16 rows of H1 and columns of H1^T
    uint64_t mask1 = 0;  // z1_j > 0
#pragma unroll
    for (int g = 0; g < H / 8; ++g) {
        __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = g * 8 + e;
            float a = b1[j];
#pragma unroll
            for (int m = 0; m < 4; ++m)
                a = __fmaf_rn(W1[4 * j + m], xs[m], a);
            const bool on = valid && a > 0.f;
            mask1 |= (uint64_t)on << j;
            hb[e] = __float2bfloat16_rn(on ? a : 0.f);
            *reinterpret_cast<__nv_bfloat16 *>(smem + G_H1T + kmajor_off(j, tid, GK)) = hb[e];
        }
        *reinterpret_cast<uint4 *>(smem + G_H1 + kmajor_off(tid, g * 8, H)) = *reinterpret_cast<const uint4 *>(hb);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;
    const uint32_t s0 = smem_addr(smem);
    if (tid == 0) {
        mma_k_major(taddr, s0 + G_H1, s0 + G_W2, H / 16, H * 16, H * 16);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(bar))
                     : "memory");
        if (!mbar_wait(bar, 0))
            *abort_flag = 1;
    }
    __syncthreads();
    uint32_t pending = 0;  // parity of the MMA batch being waited for
    if (!*abort_flag) {
        pending = 1;
        tc_fence_after();
        // epilogue of Z2: hidden layer, output, error
        float z2[H];
#pragma unroll
        for (int c = 0; c < H; c += 16) {
            float v[16];
            tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 16; ++e)
                z2[c + e] = __fadd_rn(v[e], b2[c + e]);
        }
        float y = b3v;
#pragma unroll
        for (int i = 0; i < H; ++i)
            y = __fmaf_rn(w3[i], fmaxf(z2[i], 0.f), y);
        const float err_s = valid ? __fsub_rn(y, lab) : 0.f;
        const float go = __fmul_rn(__fmul_rn(2.f, err_s), inv_count);
        // dLoss/dw3 = sum of go * h2, dLoss/db2 = sum of g2 (FP32)
#pragma unroll
        for (int i = 0; i < H; ++i)
            red[tid * RED_LD + i] = __fmul_rn(go, fmaxf(z2[i], 0.f));
        __syncthreads();
        if (tid < H)
            out[OB2 + H + tid] = column_sum(red, tid);  // w3 follows b2
        __syncthreads();
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const float g2 = (valid && z2[i] > 0.f) ? __fmul_rn(go, w3[i]) : 0.f;
            red[tid * RED_LD + i] = g2;
            const __nv_bfloat16 gb = __float2bfloat16_rn(g2);
            *reinterpret_cast<__nv_bfloat16 *>(smem + G_G2 + kmajor_off(tid, i, H)) = gb;
            *reinterpret_cast<__nv_bfloat16 *>(smem + G_G2T + kmajor_off(i, tid, GK)) = gb;
        }
        __syncthreads();
        if (tid < H)
            out[OB2 + tid] = column_sum(red, tid);
        __syncthreads();
        red[tid * RED_LD + 0] = go;
        red[tid * RED_LD + 1] = __fmul_rn(err_s, err_s);
        __syncthreads();
        if (tid == 0) {
            float gb3 = 0.f, l = 0.f;
            for (int r = 0; r < TILE_M; ++r) {
                gb3 = __fadd_rn(gb3, red[r * RED_LD + 0]);
                l = __fadd_rn(l, red[r * RED_LD + 1]);
            }
            out[OB2 + 2 * H] = gb3;
            out[KDT_MLP_PARAMS] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            mma_k_major(taddr + 64, s0 + G_G2, s0 + G_W2T, H / 16, H * 16, H * 16);
            mma_k_major(taddr + 128, s0 + G_G2T, s0 + G_H1T, GK / 16, GK * 16, GK * 16);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(bar))
                         : "memory");
            if (!mbar_wait(bar, 1))
                *abort_flag = 1;
        }
        __syncthreads();
    }
    if (!*abort_flag) {
        tc_fence_after();
        // g1 = relu'(z1) * (G2 W2) row of this sample
        float g1[H];
#pragma unroll
        for (int c = 0; c < H; c += 16) {
            float v[16];
            tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(64 + c), v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 16; ++e)
                g1[c + e] = ((mask1 >> (c + e)) & 1ull) ? v[e] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < H; ++j)
            red[tid * RED_LD + j] = g1[j];
        __syncthreads();
        if (tid < H)
            out[OB1 + tid] = column_sum(red, tid);
        for (int m = 0; m < 4; ++m) {
            __syncthreads();
#pragma unroll
            for (int j = 0; j < H; ++j)
                red[tid * RED_LD + j] = __fmul_rn(g1[j], xs[m]);
            __syncthreads();
            if (tid < H)
                out[OW1 + 4 * tid + m] = column_sum(red, tid);
        }
        // dW2: TMEM lanes 0..63 (warps 0 and 1) hold rows i = 0..63
        if (warp < 2) {
#pragma unroll
            for (int c = 0; c < H; c += 16) {
                float v[16];
                tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(128 + c), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    out[OW2 + tid * H + c + e] = v[e];
            }
        }
    } else {
        // an MMA did not signal in time: record it, give the pending ones one
        // more bounded wait before the accumulator is released
        if (tid == 0) {
            atomicOr(err, ERR_TRAVERSAL);
            mbar_wait(bar, pending);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(G_TMEM_COLS) : "memory");
}

constexpr size_t tc_smem_bytes() { return SMEM_FIXED; }

int launch_tc(int mode, const TcArgs &a, cudaStream_t s)
{
    const size_t smem = tc_smem_bytes();
    const void *fn = mode == 0 ? (const void *)mlp_tc_kernel<0> : (const void *)mlp_tc_kernel<1>;
    KDT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // at most 4 resident CTAs per SM (4 x 64 TMEM columns of 512)
    const int64_t tiles = (a.n + TILE_M - 1) / TILE_M;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * 4));
    if (mode == 0)
        KDT_LAUNCH mlp_tc_kernel<0><<<grid, TILE_M, smem, s>>>(a);
    else
        KDT_LAUNCH mlp_tc_kernel<1><<<grid, TILE_M, smem, s>>>(a);
    KDT_CUDA(cudaGetLastError());
    return KDT_OK;
}

}  // namespace

int tc_radius(const kdt_tree *t, const float *wts, const float *d_q, int64_t Q, const uint32_t *perm, float r2_user,
              float *r2q, cudaStream_t s, const unsigned long long *n_lim)
{
    TcArgs a{};
    a.n_lim = n_lim;
    a.wts = wts;
    a.n = Q;
    a.nodes = t->nodes;
    a.N = (int)t->N;
    a.D = t->D;
    a.stored = t->layout == 3;
    a.queries = d_q;
    a.perm = perm;
    for (int j = 0; j < 4; ++j) {
        a.mu[j] = t->model.norm[j];
        a.sd[j] = t->model.norm[4 + j];
    }
    a.margin = t->model.margin;
    a.r2_user = r2_user;
    a.r2q = r2q;
    a.err = t->err;
    return launch_tc(0, a, s);
}

int tc_forward(const float *wts, const float *d_x, int64_t n, float *d_y, int *d_err, cudaStream_t s)
{
    TcArgs a{};
    a.wts = wts;
    a.n = n;
    a.x = d_x;
    a.y = d_y;
    a.err = d_err;
    return launch_tc(1, a, s);
}

int tc_loss_grad(const float *wts, const float *d_x, const float *d_label, int64_t begin, int64_t count,
                 float *d_partial, int *d_err, cudaStream_t s, int *blocks)
{
    const int nb = (int)((count + TILE_M - 1) / TILE_M);
    KDT_CUDA(cudaFuncSetAttribute((const void *)mlp_tc_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  G_SMEM));
    KDT_LAUNCH mlp_tc_grad_kernel<<<nb, TILE_M, G_SMEM, s>>>(wts, d_x, d_label, begin, count, 1.0f / (float)count,
                                                            d_partial, d_err);
    KDT_CUDA(cudaGetLastError());
    *blocks = nb;
    return KDT_OK;
}

}  // namespace kdt
