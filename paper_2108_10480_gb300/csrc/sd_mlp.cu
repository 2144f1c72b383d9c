// Learned far-field surrogate: a Fourier-feature MLP trained on samples of
// the Barnes-Hut smooth distance, and its use behind a certified lower bound.
//
// Network (parameters flattened in this order, fp32 master copy):
//   xh = (x - c) / h;  f = [xh, sin(pi B xh), cos(pi B xh)]     B: [32,3]
//   z1 = W1 f + b1, a1 = silu(z1)      W1: [128,67]
//   z2 = W2 a1 + b2, a2 = silu(z2)     W2: [128,128]
//   z3 = W3 a2 + b3, a3 = silu(z3)     W3: [128,128]
//   y = s (w4 . a3 + b4)
// Weight matrices and w4 are used rounded to bfloat16 with fp32 accumulation.
//
// Training (sd_mlp_train_step): layer-by-layer fp32 SIMT GEMMs over a batch
// in device memory, mean-squared-error gradient, Adam; every reduction runs
// in a fixed order, so a step is deterministic.
// Inference (sd_mlp_forward): one fused kernel per 128-query tile on the
// tcgen05 tensor cores (bf16 operands in shared memory, fp32 accumulators in
// tensor memory), weights staged once per CTA, and the input gradient dy/dx
// by back-propagation through the same weights.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sd_common.cuh"
#include "sd_sort.cuh"

namespace {

constexpr int NF = 32, HID = 128, NIN = 67;
constexpr int OFF_B = 0, OFF_W1 = 96, OFF_B1 = OFF_W1 + HID * NIN, OFF_W2 = OFF_B1 + HID;
constexpr int OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID;
constexpr int OFF_W4 = OFF_B3 + HID, OFF_B4 = OFF_W4 + HID, NPARAMS = OFF_B4 + 1;
static_assert(NPARAMS == 41953, "parameter layout");
constexpr int KF = 68;   // feature row length in the training buffers (67 + 1 zero)

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

struct Frame {
    float c[3];
    float h[3], s;
};

// ---------------------------------------------------------------------------
// training: features, SIMT GEMM, elementwise pieces, Adam
// ---------------------------------------------------------------------------
__global__ void k_features(const float* __restrict__ x, int n, const float* __restrict__ P, Frame fr,
                           float* __restrict__ F)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float xh[3];
    for (int j = 0; j < 3; ++j) xh[j] = (x[3 * r + j] - fr.c[j]) / fr.h[j];
    float* f = F + (size_t)r * KF;
    f[0] = xh[0]; f[1] = xh[1]; f[2] = xh[2];
    for (int m = 0; m < NF; ++m) {
        const float* b = P + OFF_B + 3 * m;
        float p = fmaf(b[0], xh[0], fmaf(b[1], xh[1], b[2] * xh[2]));
        float sv, cv;
        sincospif(p, &sv, &cv);
        f[3 + m] = sv;
        f[3 + NF + m] = cv;
    }
    f[67] = 0.f;
}

// C(m,n) = sum_k A(m,k) B(k,n) over the split's k range; A(m,k) = A[m*am + k*ak],
// B(k,n) = B[k*bk + n*bn]; B rounded to bf16 when rb. EPI 1: z = acc + bias[n],
// C = z, act = silu(z). With splits the split s writes C + s*M*ldc.
template <int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, long am, long ak,
                                              const float* __restrict__ B, long bk, long bn, int rb,
                                              float* __restrict__ C, long ldc, const float* __restrict__ bias,
                                              float* __restrict__ act, int kchunk)
{
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int k0 = blockIdx.z * kchunk, k1 = min(K, k0 + kchunk);
    float acc[4][4] = {};
    for (int kk = k0; kk < k1; kk += 16) {
        for (int i = 0; i < 4; ++i) {
            int e = tid + 256 * i;
            int k = (ak == 1) ? (e & 15) : (e >> 6), m = (ak == 1) ? (e >> 4) : (e & 63);
            int gm = m0 + m, gk = kk + k;
            As[k][m] = (gm < M && gk < k1) ? A[gm * am + gk * ak] : 0.f;
            int kb = (bk == 1) ? (e & 15) : (e >> 6), nb = (bk == 1) ? (e >> 4) : (e & 63);
            int gn = n0 + nb, gkb = kk + kb;
            float v = (gn < N && gkb < k1) ? B[gkb * bk + gn * bn] : 0.f;
            Bs[kb][nb] = rb ? bf16r(v) : v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[k][ty * 4 + i]; b[i] = Bs[k][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* Cs = C + (size_t)blockIdx.z * M * ldc;
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty * 4 + i;
        if (gm >= M) continue;
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx * 4 + j;
            if (gn >= N) continue;
            float v = acc[i][j];
            if (EPI == 1) {
                v += bias[gn];
                act[(size_t)gm * ldc + gn] = silu(v);
            }
            Cs[(size_t)gm * ldc + gn] = v;
        }
    }
}

// sum of `splits` partial [M,N] blocks, in split order, into out (row stride N)
__global__ void k_sum_splits(const float* __restrict__ part, int splits, int MN, float* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MN) return;
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * MN + i];
    out[i] = s;
}

// y = s (w4 . a3 + b4), dy = 2 (y - t) / n
__global__ void k_out(const float* __restrict__ A3, int n, const float* __restrict__ P, float s,
                      const float* __restrict__ t, float* __restrict__ y, float* __restrict__ dy)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float acc = 0.f;
    for (int o = 0; o < HID; ++o) acc = fmaf(A3[(size_t)r * HID + o], bf16r(P[OFF_W4 + o]), acc);
    float v = s * (acc + P[OFF_B4]);
    y[r] = v;
    dy[r] = 2.f * (v - t[r]) / (float)n;
}

// d3 = s dy w4 dsilu(z3)
__global__ void k_back_out(const float* __restrict__ dy, const float* __restrict__ Z3, int n,
                           const float* __restrict__ P, float s, float* __restrict__ D3)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * HID) return;
    int r = i / HID, o = i - r * HID;
    D3[i] = s * dy[r] * bf16r(P[OFF_W4 + o]) * dsilu(Z3[i]);
}

__global__ void k_mul_dsilu(float* __restrict__ D, const float* __restrict__ Z, int total)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) D[i] *= dsilu(Z[i]);
}

// per-column sums in row order: out[o] = scale * sum_r w_r D[r][o] (w = 1 if null)
__global__ void k_colsum(const float* __restrict__ D, int n, int ncol, const float* __restrict__ w, float scale,
                         float* __restrict__ out)
{
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= ncol) return;
    float acc = 0.f;
    for (int r = 0; r < n; ++r) acc = fmaf(w ? w[r] : 1.f, D[(size_t)r * ncol + o], acc);
    out[o] = scale * acc;
}

// loss = mean (y - t)^2, one thread, fixed order
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, int n, float* __restrict__ loss)
{
    if (threadIdx.x || blockIdx.x) return;
    double acc = 0.0;
    for (int r = 0; r < n; ++r) {
        double d = (double)y[r] - (double)t[r];
        acc += d * d;
    }
    *loss = (float)(acc / n);
}

// Adam (Kingma & Ba) on every parameter except the Fourier frequencies
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                       float* __restrict__ v, int step, float lr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAMS || i < OFF_W1) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float g = G[i];
    float mi = b1 * m[i] + (1.f - b1) * g;
    float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / (1.f - powf(b1, (float)step));
    float vh = vi / (1.f - powf(b2, (float)step));
    P[i] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
// fused inference on the 5th-generation tensor cores (tcgen05): value and
// input gradient of 128-query tiles
// ---------------------------------------------------------------------------
// One CTA per SM; its 16 warps form two groups of 8 that walk alternate
// 128-row tiles, so one group's activation work overlaps the other's tensor
// work. The six GEMMs of a tile (three layers forward, three back for dy/dx)
// are single-thread-issued tcgen05.mma (kind::f16, bf16 operands, fp32
// accumulation, M = 128) with both operands in shared memory and the
// accumulator in tensor memory (TMEM); completion is signalled through the
// group's mbarrier by tcgen05.commit. Between GEMMs the group's 256 threads
// (thread = TMEM lane (row) x half of the columns) read the accumulator with
// tcgen05.ld, apply bias and activation and write the next A operand back to
// the group's shared-memory buffer; dsilu(z1), dsilu(z2) wait in TMEM as
// packed binary16 pairs (tcgen05.st) for the backward pass. Operands use the
// no-swizzle layout of 8 x 16-byte core matrices. The weights are staged
// once per CTA as stored ([out][in], K-major for the forward GEMMs); the
// backward GEMMs read the same copy as an MN-major B operand. Rounding
// points: features, a1, a2 and the back-propagated factors in bf16,
// dsilu(z1), dsilu(z2) in binary16, everything else fp32.
constexpr int TM = 128;                 // rows per tile = TMEM lanes
constexpr int TC_THREADS = 512;         // 2 groups x 8 warps: lane quarter (warp % 4) x column half
constexpr int TC_GROUP = 256;
constexpr int KF1 = 80;                 // layer-1 K (67 features + zero padding to a multiple of 16)
constexpr int TMEM_COLS = 512;          // per group (256 columns each): accumulator [0,128),
                                        // dsilu(z1) [128,192), dsilu(z2) [192,256) (binary16 pairs)
constexpr int SZ_W1 = HID * KF1 * 2, SZ_W = HID * HID * 2, SZ_X = TM * HID * 2;
// per group, the complementary sine or cosine of every Fourier feature
// column (fp32, [64 columns][128 rows]) kept from the forward pass for dy/dx
constexpr int SZ_FC = TM * 2 * NF * 4;
constexpr int O_W1 = 0, O_W2 = O_W1 + SZ_W1, O_W3 = O_W2 + SZ_W, O_X = O_W3 + SZ_W, O_FC = O_X + 2 * SZ_X,
              O_F32 = O_FC + 2 * SZ_FC;
// fp32 area: b1, b2, b3, w4 (bf16-rounded) [4 x 128], B [96], b4, then per
// group the second column half's partial sums: y [128], dy/dxh [128 x 3],
// then s * w4 [128]
constexpr int F_BIAS = 0, F_BQ = 4 * HID, F_B4 = F_BQ + 96, F_YP = F_B4 + 4, F_GP = F_YP + 2 * TM,
              F_SW4 = F_GP + 6 * TM, F_END = F_SW4 + HID;     // s * w4 [128] last
constexpr int O_BAR = O_F32 + 4 * F_END;
constexpr size_t TC_SMEM = (size_t)O_BAR + 32;    // 2 mbarriers, TMEM address, 2 wait flags
static_assert(O_X % 1024 == 0 && O_BAR % 8 == 0 && TC_SMEM <= 232448, "tcgen05 MLP shared memory layout");
// mbarrier polls before a tile is abandoned (its group's remaining outputs
// become NaN), and polls of the drain that then waits for the GEMMs already
// issued before the tensor memory is freed
#ifndef SD_TC_WAIT_LIMIT
#define SD_TC_WAIT_LIMIT (1 << 24)
#endif
constexpr int TC_WAIT_LIMIT = SD_TC_WAIT_LIMIT;
constexpr int TC_DRAIN_LIMIT = 1 << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of a matrix with row extent kdim: core
// matrices of 8 rows x 8 elements (16 bytes per row, 128 bytes each),
// column-adjacent core matrices 128 bytes apart, row groups kdim * 16 bytes
// apart. Read with r as M/N and k as K this is the K-major operand layout;
// read with r as K and k as N it is the MN-major one.
__device__ __forceinline__ int core_off(int r, int k, int kdim)
{
    return ((r >> 3) * (kdim >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor (no swizzle): start, leading byte offset
// (between core matrices adjacent in K), stride byte offset (between core
// matrices adjacent in M/N), version 1
__device__ __forceinline__ uint64_t sm_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: fp32 D, bf16 A and B, A K-major, B
// K-major or MN-major, M = 128
__device__ __forceinline__ uint32_t tc_idesc(int N, bool b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (b_mn ? 1u << 16 : 0u) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(TM >> 4) << 24);
}

// forward GEMM: D[128 x N] (TMEM) = X[128 x K] * W[N x K]^T, W stored [N][K]
__device__ __forceinline__ void tc_gemm_fwd(uint32_t tmem_d, uint32_t xa, uint32_t wa, int K, int N)
{
    const uint32_t idesc = tc_idesc(N, false);
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint64_t da = sm_desc(xa + 256u * ks, 128u, sbo);
        const uint64_t db = sm_desc(wa + 256u * ks, 128u, sbo);
        const uint32_t accum = ks > 0 ? 1u : 0u;
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accum));
    }
}

// backward GEMM: D[128 x N] = X[128 x 128] * W[128 x N], W stored [128][N]
// (row = K): the stored copy read as an MN-major B operand
__device__ __forceinline__ void tc_gemm_bwd(uint32_t tmem_d, uint32_t xa, uint32_t wa, int N)
{
    const uint32_t idesc = tc_idesc(N, true);
    const uint32_t lbo = (uint32_t)(N / 8) * 128u;     // next 8 rows (K) of W
    for (int ks = 0; ks < HID / 16; ++ks) {
        const uint64_t da = sm_desc(xa + 256u * ks, 128u, (HID / 8) * 128u);
        const uint64_t db = sm_desc(wa + 2u * lbo * ks, lbo, 128u);
        const uint32_t accum = ks > 0 ? 1u : 0u;
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accum));
    }
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

// bounded wait for the mbarrier phase with parity `ph`
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t ph, int limit)
{
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(bar), "r"(ph));
    return done != 0;
}

#define TC_R8(v, o) "=r"(v[o]), "=r"(v[o + 1]), "=r"(v[o + 2]), "=r"(v[o + 3]), "=r"(v[o + 4]), "=r"(v[o + 5]), \
                    "=r"(v[o + 6]), "=r"(v[o + 7])
#define TC_W8(v, o) "r"(v[o]), "r"(v[o + 1]), "r"(v[o + 2]), "r"(v[o + 3]), "r"(v[o + 4]), "r"(v[o + 5]), \
                    "r"(v[o + 6]), "r"(v[o + 7])

// consecutive TMEM columns of this thread's lane; tm_wait_ld completes
// every load issued before it
__device__ __forceinline__ void tm_ld32(uint32_t ta, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : TC_R8(v, 0), TC_R8(v, 8), TC_R8(v, 16), TC_R8(v, 24) : "r"(ta));
}

__device__ __forceinline__ void tm_ld16(uint32_t ta, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : TC_R8(v, 0), TC_R8(v, 8) : "r"(ta));
}

__device__ __forceinline__ void tm_ld8(uint32_t ta, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : TC_R8(v, 0) : "r"(ta));
}

__device__ __forceinline__ void tm_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;");
}

__device__ __forceinline__ void tm_st16(uint32_t ta, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(ta), TC_W8(v, 0), TC_W8(v, 8));
    asm volatile("tcgen05.wait::st.sync.aligned;");
}

// 8 consecutive bf16 values into one 16-byte row of a core matrix
__device__ __forceinline__ void st_bf16x8(unsigned char* base, int off, const float* f)
{
    uint4 u;
    __nv_bfloat162 p0 = __floats2bfloat162_rn(f[0], f[1]), p1 = __floats2bfloat162_rn(f[2], f[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(f[4], f[5]), p3 = __floats2bfloat162_rn(f[6], f[7]);
    u.x = *reinterpret_cast<uint32_t*>(&p0);
    u.y = *reinterpret_cast<uint32_t*>(&p1);
    u.z = *reinterpret_cast<uint32_t*>(&p2);
    u.w = *reinterpret_cast<uint32_t*>(&p3);
    *reinterpret_cast<uint4*>(base + off) = u;
}

// sin(pi p), cos(pi p): p reduced exactly to [-1, 1] (p - 2 rint(p / 2)),
// then the hardware sine and cosine on [-pi, pi] (absolute error about
// 2^-21, far below the bfloat16 rounding of the features)
__device__ __forceinline__ void sincospi_tc(float p, float* sv, float* cv)
{
    const float rr = p - 2.f * rintf(0.5f * p);
    __sincosf(3.14159265358979f * rr, sv, cv);
}

// silu(z) and dsilu(z) from one logistic sigmoid (approximate reciprocal:
// relative error ~1e-7, far below the bfloat16 rounding that follows)
__device__ __forceinline__ void silu_pair(float z, float& a, float& da)
{
    const float sg = __fdividef(1.f, 1.f + __expf(-z));
    a = z * sg;
    da = sg * fmaf(z, 1.f - sg, 1.f);
}

// the group's named barrier (ids 1, 2; 256 threads)
__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(TC_GROUP));
}

// make this thread's shared-memory and TMEM writes visible to the next
// tensor-core operation of the group, then hand the issue to its thread 0
__device__ __forceinline__ void tc_sync_before_mma(int g)
{
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    group_sync(g);
    asm volatile("tcgen05.fence::after_thread_sync;");
}

// wait for the group's GEMMs: its issuing thread polls the mbarrier, the
// other threads sleep in the group barrier (no issue slots taken from the
// other group); returns whether the GEMMs completed
__device__ __forceinline__ bool group_wait(int g, bool issuer, uint32_t bar, uint32_t ph, volatile int* flag)
{
    if (issuer) *flag = bar_wait(bar, ph, TC_WAIT_LIMIT) ? 1 : 0;
    group_sync(g);
    const bool ok = *flag != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    return ok;
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi)
{
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_tc(const float* __restrict__ P, Frame fr,
                                                          const float* __restrict__ x, int n,
                                                          float* __restrict__ y, float* __restrict__ dydx)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    float* F32 = reinterpret_cast<float*>(smem + O_F32);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + O_BAR + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = warp >> 3, gw = warp & 7, gt = tid & (TC_GROUP - 1);
    const int row = (gw & 3) * 32 + lane, half = gw >> 2;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_addr(tmem_slot)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid < 2) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(smem + O_BAR + 8 * tid)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // the weights in bf16 as stored, [out][in]
    for (int i = tid; i < HID * KF1; i += TC_THREADS) {
        const int o = i / KF1, k = i - o * KF1;
        *reinterpret_cast<__nv_bfloat16*>(smem + O_W1 + core_off(o, k, KF1)) =
            __float2bfloat16_rn(k < NIN ? P[OFF_W1 + o * NIN + k] : 0.f);
    }
    for (int i = tid; i < HID * HID; i += TC_THREADS) {
        const int o = i / HID, k = i - o * HID;
        *reinterpret_cast<__nv_bfloat16*>(smem + O_W2 + core_off(o, k, HID)) = __float2bfloat16_rn(P[OFF_W2 + i]);
        *reinterpret_cast<__nv_bfloat16*>(smem + O_W3 + core_off(o, k, HID)) = __float2bfloat16_rn(P[OFF_W3 + i]);
    }
    for (int i = tid; i < HID; i += TC_THREADS) {
        F32[F_BIAS + i] = P[OFF_B1 + i];
        F32[F_BIAS + HID + i] = P[OFF_B2 + i];
        F32[F_BIAS + 2 * HID + i] = P[OFF_B3 + i];
        F32[F_BIAS + 3 * HID + i] = bf16r(P[OFF_W4 + i]);
        F32[F_SW4 + i] = fr.s * bf16r(P[OFF_W4 + i]);
    }
    for (int i = tid; i < 96; i += TC_THREADS) F32[F_BQ + i] = P[OFF_B + i];
    if (tid == 0) F32[F_B4] = P[OFF_B4];
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // this group's accumulator columns and this warp's lane quarter
    const uint32_t tg = *tmem_slot + (uint32_t)(g * 256);
    const uint32_t tl = tg + ((uint32_t)((gw & 3) * 32) << 16);
    const uint32_t bar_a = smem_addr(smem + O_BAR + 8 * g), xa = smem_addr(smem + O_X + g * SZ_X);
    const uint32_t w1a = smem_addr(smem + O_W1), w2a = smem_addr(smem + O_W2), w3a = smem_addr(smem + O_W3);
    unsigned char* X = smem + O_X + g * SZ_X;
    float* FC = reinterpret_cast<float*>(smem + O_FC + g * SZ_FC);
    const float* w4 = F32 + F_BIAS + 3 * HID;
    const float* Bq = F32 + F_BQ;
    float* yp_h = F32 + F_YP + g * TM;          // the second half's partial y
    float* gp_h = F32 + F_GP + g * 3 * TM;      // and partial dy/dxh
    const bool issuer = gt == 0;
    volatile int* wflag = reinterpret_cast<volatile int*>(smem + O_BAR + 24 + 4 * g);
    uint32_t ph = 0;
    const int ntiles = (n + TM - 1) / TM;
    const int t0 = 2 * (int)blockIdx.x + g, tstep = 2 * (int)gridDim.x;
    float xn[3] = {0.f, 0.f, 0.f};
    if (t0 < ntiles) {
        const int gr = min(t0 * TM + row, n - 1);
        for (int j = 0; j < 3; ++j) xn[j] = x[3 * gr + j];
    }
    for (int tile = t0; tile < ntiles; tile += tstep) {
        const int r = tile * TM + row;
        float xh[3];
        for (int j = 0; j < 3; ++j) xh[j] = (xn[j] - fr.c[j]) / fr.h[j];
        if (tile + tstep < ntiles) {                    // the next tile's query, early
            const int gr = min((tile + tstep) * TM + row, n - 1);
            for (int j = 0; j < 3; ++j) xn[j] = x[3 * gr + j];
        }
        // features: this half's 40 columns of [xh, sin(pi B xh), cos(pi B xh), 0...]
#pragma unroll 1
        for (int fc = 0; fc < 5; ++fc) {
            float f[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = half * 40 + fc * 8 + j;
                float v = 0.f;
                if (c < 3) {
                    v = xh[c];
                } else if (c < NIN) {
                    const int m = c < 3 + NF ? c - 3 : c - 3 - NF;
                    const float pp = fmaf(Bq[3 * m], xh[0], fmaf(Bq[3 * m + 1], xh[1], Bq[3 * m + 2] * xh[2]));
                    float sv, cv;
                    sincospi_tc(pp, &sv, &cv);
                    v = c < 3 + NF ? sv : cv;
                    FC[(c - 3) * TM + row] = c < 3 + NF ? cv : sv;   // what dy/dx needs for this column
                }
                f[j] = v;
            }
            st_bf16x8(X, core_off(row, half * 40 + fc * 8, KF1), f);
        }
        // forward: layers 1..3
#pragma unroll 1
        for (int layer = 0; layer < 3; ++layer) {
            tc_sync_before_mma(g);
            if (issuer) {
                if (layer == 0) tc_gemm_fwd(tg, xa, w1a, KF1, HID);
                else tc_gemm_fwd(tg, xa, layer == 1 ? w2a : w3a, HID, HID);
                tc_commit(bar_a);
            }
            if (!group_wait(g, issuer, bar_a, ph, wflag)) goto tile_failed;
            ph ^= 1u;
            const float4* bb = reinterpret_cast<const float4*>(F32 + F_BIAS + layer * HID);
            const float4* w4v = reinterpret_cast<const float4*>(w4);
            const float4* sw4v = reinterpret_cast<const float4*>(F32 + F_SW4);
            float yp = 0.f;
#pragma unroll 1
            for (int cc = 0; cc < 2; ++cc) {
                const int c0 = half * 64 + cc * 32;
                uint32_t v[32];
                tm_ld32(tl + c0, v);
                tm_wait_ld();
                float a[32];
                uint32_t hp[16];
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const float4 b4 = bb[(c0 + j) >> 2];
                    const float bz[4] = {b4.x, b4.y, b4.z, b4.w};
                    float sz[4], dz[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) silu_pair(__uint_as_float(v[j + e]) + bz[e], sz[e], dz[e]);
                    if (layer < 2) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) a[j + e] = sz[e];
                        hp[j >> 1] = pack_h2(dz[0], dz[1]);
                        hp[(j >> 1) + 1] = pack_h2(dz[2], dz[3]);
                    } else {
                        // layer 3: y partial from a3, the backward pass starts
                        // from g3 = s w4 dsilu(z3)
                        const float4 w = w4v[(c0 + j) >> 2], sw = sw4v[(c0 + j) >> 2];
                        yp = fmaf(sz[0], w.x, fmaf(sz[1], w.y, fmaf(sz[2], w.z, fmaf(sz[3], w.w, yp))));
                        a[j] = sw.x * dz[0];
                        a[j + 1] = sw.y * dz[1];
                        a[j + 2] = sw.z * dz[2];
                        a[j + 3] = sw.w * dz[3];
                    }
                }
                if (layer < 2) tm_st16(tl + (uint32_t)(HID + layer * 64 + (c0 >> 1)), hp);
#pragma unroll
                for (int kb = 0; kb < 4; ++kb) st_bf16x8(X, core_off(row, c0 + kb * 8, HID), a + 8 * kb);
            }
            if (layer == 2) {
                if (half) yp_h[row] = yp;
                group_sync(g);
                if (!half && r < n) y[r] = fr.s * ((yp + yp_h[row]) + F32[F_B4]);
            }
        }
        if (dydx) {
            // backward: g2 = (g3 W3) dsilu(z2), g1 = (g2 W2) dsilu(z1), gf = g1 W1
#pragma unroll 1
            for (int layer = 2; layer >= 0; --layer) {
                tc_sync_before_mma(g);
                if (issuer) {
                    if (layer == 0) tc_gemm_bwd(tg, xa, w1a, KF1);
                    else tc_gemm_bwd(tg, xa, layer == 2 ? w3a : w2a, HID);
                    tc_commit(bar_a);
                }
                if (!group_wait(g, issuer, bar_a, ph, wflag)) goto tile_failed;
                ph ^= 1u;
                if (layer > 0) {
#pragma unroll 1
                    for (int cc = 0; cc < 2; ++cc) {
                        const int c0 = half * 64 + cc * 32;
                        uint32_t v[32], d[16];
                        tm_ld32(tl + c0, v);
                        tm_ld16(tl + (uint32_t)(HID + (layer - 1) * 64 + (c0 >> 1)), d);
                        tm_wait_ld();
                        float a[32];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float2 dd = __half22float2(*reinterpret_cast<const __half2*>(&d[j]));
                            a[2 * j] = __uint_as_float(v[2 * j]) * dd.x;
                            a[2 * j + 1] = __uint_as_float(v[2 * j + 1]) * dd.y;
                        }
#pragma unroll
                        for (int kb = 0; kb < 4; ++kb) st_bf16x8(X, core_off(row, c0 + kb * 8, HID), a + 8 * kb);
                    }
                } else {
                    // features -> xh: columns [40 half, 40 half + 40) of gf
                    float gg[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
                    for (int cc = 0; cc < 2; ++cc) {
                        const int c0 = half * 40 + cc * 32;
                        uint32_t v[32];
                        if (cc == 0) tm_ld32(tl + c0, v);
                        else tm_ld8(tl + c0, v);
                        tm_wait_ld();
                        const int cn = cc == 0 ? 32 : 8;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (j >= cn) break;
                            const int c = c0 + j;
                            const float gv = __uint_as_float(v[j]);
                            if (c < 3) {
                                gg[c] += gv;
                            } else if (c < NIN) {
                                const int m = c < 3 + NF ? c - 3 : c - 3 - NF;
                                const float o = FC[(c - 3) * TM + row];   // cos for a sine column, sin for a cosine one
                                const float k = c < 3 + NF ? gv * 3.14159265358979f * o
                                                           : -gv * 3.14159265358979f * o;
                                gg[0] = fmaf(k, Bq[3 * m], gg[0]);
                                gg[1] = fmaf(k, Bq[3 * m + 1], gg[1]);
                                gg[2] = fmaf(k, Bq[3 * m + 2], gg[2]);
                            }
                        }
                    }
                    if (half)
                        for (int j = 0; j < 3; ++j) gp_h[3 * row + j] = gg[j];
                    group_sync(g);
                    if (!half && r < n)
                        for (int j = 0; j < 3; ++j)
                            dydx[3 * r + j] = (gg[j] + gp_h[3 * row + j]) / fr.h[j];
                }
            }
        }
        continue;
    tile_failed:
        // A wait ran out (the same verdict for the whole group): no further
        // GEMM is issued, this tile's rows and those of every later tile of
        // the group are NaN, and the issuing thread waits (bounded) for the
        // GEMM already committed before the tensor memory is freed.
        if (!half)
            for (int tt = tile; tt < ntiles; tt += tstep) {
                const int rr = tt * TM + row;
                if (rr >= n) break;
                y[rr] = __int_as_float(0x7fffffff);
                if (dydx) dydx[3 * rr] = dydx[3 * rr + 1] = dydx[3 * rr + 2] = __int_as_float(0x7fffffff);
            }
        if (issuer) bar_wait(bar_a, ph, TC_DRAIN_LIMIT);
        group_sync(g);
        break;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_slot), "r"(TMEM_COLS));
}

int sm_count_mlp()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

Frame make_frame(const float* frame)
{
    Frame f;
    for (int j = 0; j < 3; ++j) {
        f.c[j] = frame[j];
        f.h[j] = frame[3 + j];
    }
    f.s = frame[6];
    return f;
}

bool frame_ok(const float* frame)
{
    return frame[3] > 0.f && frame[4] > 0.f && frame[5] > 0.f && std::isfinite(frame[6]);
}

}  // namespace

extern "C" int64_t sd_mlp_num_params(void) { return NPARAMS; }

extern "C" size_t sd_mlp_workspace_bytes(int64_t n)
{
    // F [n,68], Z1..Z3 and A1..A3 [n,128], D [n,128] x2, y, dy [n], split partials
    size_t b = sizeof(float) * (size_t)n * (KF + 8 * HID + 2);
    b += sizeof(float) * (size_t)64 * HID * HID;   // up to 64 split-K partial blocks of 128 x 128
    return b + 4096;
}

extern "C" int sd_mlp_forward(const float* params, const float* frame, const float* x, int64_t n, float* y,
                              float* dydx, void* stream)
{
    if (!params || !frame || !frame_ok(frame) || n < 0 || (n > 0 && (!x || !y))) return SD_ERR_INVALID_ARG;
    if (n == 0) return SD_OK;
    if (n >= ((int64_t)1 << 31) / 3) return SD_ERR_TOO_LARGE;
    cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    Frame fr = make_frame(frame);
    const int tiles = (int)((n + TM - 1) / TM);
    const int blocks = std::max(1, std::min(sm_count_mlp(), (tiles + 1) / 2));
    k_mlp_tc<<<blocks, TC_THREADS, TC_SMEM, (cudaStream_t)stream>>>(params, fr, x, (int)n, y, dydx);
    sd_count_launches(1);
    return sd_cuda_status(cudaGetLastError());
}

extern "C" int sd_mlp_train_step(float* params, float* adam_m, float* adam_v, int32_t step, float lr,
                                 const float* frame, const float* x, const float* target, int64_t n, float* loss,
                                 float* grad, void* workspace, size_t ws_bytes, void* stream)
{
    if (!params || !frame || !frame_ok(frame) || !x || !target || n <= 0 || !workspace || !grad)
        return SD_ERR_INVALID_ARG;
    if (lr > 0.f && (!adam_m || !adam_v || step < 1)) return SD_ERR_INVALID_ARG;
    if (ws_bytes < sd_mlp_workspace_bytes(n)) return SD_ERR_INVALID_ARG;
    if (n > (1 << 24)) return SD_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)stream;
    Frame fr = make_frame(frame);
    const int N = (int)n;
    float* F = (float*)workspace;
    float* Z1 = F + (size_t)N * KF;
    float* Z2 = Z1 + (size_t)N * HID;
    float* Z3 = Z2 + (size_t)N * HID;
    float* A1 = Z3 + (size_t)N * HID;
    float* A2 = A1 + (size_t)N * HID;
    float* A3 = A2 + (size_t)N * HID;
    float* D = A3 + (size_t)N * HID;
    float* D2 = D + (size_t)N * HID;
    float* yv = D2 + (size_t)N * HID;
    float* dy = yv + N;
    float* part = dy + N;
    int nl = 0;
    auto gemm_grid = [](int M, int Nn, int splits) { return dim3((Nn + 63) / 64, (M + 63) / 64, splits); };
    // forward: z_l = a_{l-1} W_l^T + b_l with W rounded to bf16
    k_features<<<(N + 255) / 256, 256, 0, st>>>(x, N, params, fr, F); ++nl;
    k_gemm<1><<<gemm_grid(N, HID, 1), 256, 0, st>>>(N, HID, NIN, F, KF, 1, params + OFF_W1, 1, NIN, 1, Z1, HID,
                                                     params + OFF_B1, A1, NIN); ++nl;
    k_gemm<1><<<gemm_grid(N, HID, 1), 256, 0, st>>>(N, HID, HID, A1, HID, 1, params + OFF_W2, 1, HID, 1, Z2, HID,
                                                     params + OFF_B2, A2, HID); ++nl;
    k_gemm<1><<<gemm_grid(N, HID, 1), 256, 0, st>>>(N, HID, HID, A2, HID, 1, params + OFF_W3, 1, HID, 1, Z3, HID,
                                                     params + OFF_B3, A3, HID); ++nl;
    k_out<<<(N + 255) / 256, 256, 0, st>>>(A3, N, params, fr.s, target, yv, dy); ++nl;
    k_loss<<<1, 1, 0, st>>>(yv, target, N, loss); ++nl;
    // backward
    cudaMemsetAsync(grad, 0, sizeof(float) * OFF_W1, st);
    k_colsum<<<1, HID, 0, st>>>(A3, N, HID, dy, fr.s, grad + OFF_W4); ++nl;
    k_colsum<<<1, 1, 0, st>>>(dy, N, 1, nullptr, fr.s, grad + OFF_B4); ++nl;
    k_back_out<<<(N * HID + 255) / 256, 256, 0, st>>>(dy, Z3, N, params, fr.s, D); ++nl;
    const int splits = std::min(64, std::max(1, N / 256));
    const int kchunk = (N + splits - 1) / splits;
    const float* Ain[3] = {F, A1, A2};
    const int Kin[3] = {NIN, HID, HID};
    const long lda[3] = {KF, HID, HID};
    const int offW[3] = {OFF_W1, OFF_W2, OFF_W3};
    const int offb[3] = {OFF_B1, OFF_B2, OFF_B3};
    const float* Zs[3] = {Z1, Z2, Z3};
    float* dcur = D;
    float* dnext = D2;
    for (int l = 2; l >= 0; --l) {
        // dW_l = d_l^T a_{l-1} (sum over the batch, split-K, reduced in order)
        k_gemm<0><<<gemm_grid(HID, Kin[l], splits), 256, 0, st>>>(HID, Kin[l], N, dcur, 1, HID, Ain[l], lda[l], 1, 0,
                                                                   part, Kin[l], nullptr, nullptr, kchunk); ++nl;
        k_sum_splits<<<(HID * Kin[l] + 255) / 256, 256, 0, st>>>(part, splits, HID * Kin[l], grad + offW[l]); ++nl;
        k_colsum<<<1, HID, 0, st>>>(dcur, N, HID, nullptr, 1.f, grad + offb[l]); ++nl;
        if (l > 0) {
            // d_{l-1} = (d_l W_l) * dsilu(z_{l-1})
            k_gemm<0><<<gemm_grid(N, HID, 1), 256, 0, st>>>(N, HID, HID, dcur, HID, 1, params + offW[l], HID, 1, 1,
                                                             dnext, HID, nullptr, nullptr, HID); ++nl;
            k_mul_dsilu<<<(N * HID + 255) / 256, 256, 0, st>>>(dnext, Zs[l - 1], N * HID); ++nl;
            std::swap(dcur, dnext);
        }
    }
    if (lr > 0.f) {
        k_adam<<<(NPARAMS + 255) / 256, 256, 0, st>>>(params, grad, adam_m, adam_v, step, lr);
        ++nl;
    }
    sd_count_launches(nl);
    return sd_cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// certified lower bound over a top-of-tree cut, and routing
// ---------------------------------------------------------------------------
// For a cut C of the tree (nodes covering every primitive once),
//   LB(q) = -(1/alpha) log sum_{B in C} n_B (A kappa)^S e^{-alpha d(q, box B)}
// (n_B (A kappa)^S = nw_B kappa^S for nodes holding an edge or triangle; the
// bound multiplies every cut node by kappa^S >= 1, which only loosens it).
// Every exact term w_i e^{-alpha d_i} of a primitive in B has d_i >= d(q, box B)
// and w_i = (A w~_i)^S <= (A kappa)^S, with kappa >= max w~ (the largest
// Bernstein coefficient bounds a Bernstein polynomial). So LB is a lower
// bound of the exact d^ (Eq. 3). It is not one of the Barnes-Hut value: a far
// field taken at a node above the cut uses a nearer box than the cut nodes.
namespace {

constexpr int CUT_MAX = 64;

struct CutNode {
    float lo[3], hi[3], w;
};

__device__ __forceinline__ unsigned fkey(float f) { return __float_as_uint(f); }   // f >= 0

// kappa: bound of w~ over every primitive (1 for points and isolated primitives)
__global__ void k_kappa(SdParams P, unsigned* __restrict__ kbits)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.n_prims) return;
    float4 h = P.hdr[k];
    int kind = (int)h.w;
    float kap = 1.f;
    if (!P.unit_weights && kind == SD_KIND_SEG) {
        float u = P.ext[2 * k].w, v = P.ext[2 * k + 1].x;
        kap = fmaxf(fmaxf(u, v), (16.f - 5.f * u - 5.f * v) * (1.f / 6.f));
    } else if (!P.unit_weights && kind == SD_KIND_TRI) {
        float iv = P.ext[2 * k].w, ie = P.ext[2 * k + 1].w;
        if (iv != 1.f)
            for (int n = 0; n < 36; ++n)
                kap = fmaxf(kap, fmaf(ie, P.tri_de[n], fmaf(iv, P.tri_dv[n], P.tri_base[n])));
    }
    kap = fmaxf(kap, 1.f) * 1.0001f;   // margin for the fp32 rounding of the coefficients
    atomicMax(kbits, fkey(kap));
}

// the cut: breadth-first from the root while the next level has <= CUT_MAX nodes
__global__ void k_cut(SdParams P, const unsigned* __restrict__ kbits, CutNode* __restrict__ cut, int* __restrict__ ncut)
{
    if (threadIdx.x || blockIdx.x) return;
    int refs[2][CUT_MAX];
    CutNode nodes[2][CUT_MAX];
    int cur = 0, n = 0;
    auto read = [&](int rec, int slot, CutNode& c) {
        const float* f = reinterpret_cast<const float*>(&P.nodes[rec]);
        c.lo[0] = f[0 + slot]; c.lo[1] = f[2 + slot]; c.lo[2] = f[4 + slot];
        c.hi[0] = -f[6 + slot]; c.hi[1] = -f[8 + slot]; c.hi[2] = -f[10 + slot];
        c.w = exp2f(slot ? P.lw2[rec].y : P.lw2[rec].x);
    };
    refs[0][0] = P.nodes[P.root_record].d.x;
    read(P.root_record, 0, nodes[0][0]);
    n = 1;
    for (;;) {
        int nn = 0;
        for (int i = 0; i < n; ++i) nn += refs[cur][i] >= 0 ? 2 : 1;
        if (nn > CUT_MAX || nn == n) break;
        int o = 0;
        for (int i = 0; i < n; ++i) {
            int r = refs[cur][i];
            if (r < 0) {
                refs[cur ^ 1][o] = r;
                nodes[cur ^ 1][o++] = nodes[cur][i];
            } else {
                const int4 d = P.nodes[r].d;
                refs[cur ^ 1][o] = d.x; read(r, 0, nodes[cur ^ 1][o++]);
                refs[cur ^ 1][o] = d.y; read(r, 1, nodes[cur ^ 1][o++]);
            }
        }
        cur ^= 1;
        n = o;
    }
    const float kS = powf(__uint_as_float(*kbits), P.S);
    for (int i = 0; i < n; ++i) {
        cut[i] = nodes[cur][i];
        cut[i].w *= kS;
    }
    *ncut = n;
}

// LB per query in fp32 with a max shift, lowered by 1e-3 + 1e-5 |LB| to cover
// the fp32 rounding of the box distances and the sum (the bound stays
// certified); its gradient sum_B softmax_B (q - y_B) / d_B (y_B the closest
// point of box B; 0 inside a box); flag = LB > margin
__global__ void k_lower_bound(const CutNode* __restrict__ cut, const int* __restrict__ ncut, float alpha,
                              const float* __restrict__ q, int M, float margin, float* __restrict__ lb,
                              float* __restrict__ glb, int* __restrict__ flag)
{
    __shared__ CutNode sc[CUT_MAX];
    __shared__ float slw[CUT_MAX];
    __shared__ int sn;
    if (threadIdx.x == 0) sn = *ncut;
    __syncthreads();
    for (int i = threadIdx.x; i < sn; i += blockDim.x) {
        sc[i] = cut[i];
        slw[i] = logf(cut[i].w);
    }
    __syncthreads();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const float qx = q[3 * k], qy = q[3 * k + 1], qz = q[3 * k + 2];
    float m = -INFINITY, s = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    for (int i = 0; i < sn; ++i) {
        float dx = qx - fminf(fmaxf(qx, sc[i].lo[0]), sc[i].hi[0]);
        float dy = qy - fminf(fmaxf(qy, sc[i].lo[1]), sc[i].hi[1]);
        float dz = qz - fminf(fmaxf(qz, sc[i].lo[2]), sc[i].hi[2]);
        float d = sqrtf(dx * dx + dy * dy + dz * dz);
        float t = slw[i] - alpha * d;
        float inv = d > 0.f ? 1.f / d : 0.f;
        dx *= inv; dy *= inv; dz *= inv;
        if (t > m) {
            float r = expf(m - t);
            s = fmaf(s, r, 1.f);
            gx = fmaf(gx, r, dx); gy = fmaf(gy, r, dy); gz = fmaf(gz, r, dz);
            m = t;
        } else {
            float e = expf(t - m);
            s += e;
            gx = fmaf(e, dx, gx); gy = fmaf(e, dy, gy); gz = fmaf(e, dz, gz);
        }
    }
    float v = -(m + logf(s)) / alpha;
    v -= 1e-3f + 1e-5f * fabsf(v);
    if (lb) lb[k] = v;
    if (glb) {
        const float is = 1.f / s;
        glb[3 * k] = gx * is; glb[3 * k + 1] = gy * is; glb[3 * k + 2] = gz * is;
    }
    if (flag) flag[k] = (v > margin) ? 1 : 0;
}

__global__ void k_gather3(const float* __restrict__ q, const int* __restrict__ idx, int n, float* __restrict__ out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int s = idx[k];
    out[3 * k] = q[3 * s]; out[3 * k + 1] = q[3 * s + 1]; out[3 * k + 2] = q[3 * s + 2];
}

// results back to query order; the network's answers (positions >= nb)
// are residuals over the lower bound, so LB and its gradient are added back
__global__ void k_scatter(const int* __restrict__ idx, int n, int nb, const float* __restrict__ v,
                          const float* __restrict__ g, const float* __restrict__ lb, const float* __restrict__ glb,
                          float* __restrict__ value, float* __restrict__ grad)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int d = idx[k];
    const bool net = k >= nb;
    value[d] = net ? v[k] + lb[d] : v[k];
    if (grad)
        for (int j = 0; j < 3; ++j) grad[3 * d + j] = net ? g[3 * k + j] + glb[3 * d + j] : g[3 * k + j];
}

__global__ void k_iota_flagkey(const int* __restrict__ flag, int M, unsigned* __restrict__ key, int* __restrict__ val,
                               int* __restrict__ count)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    key[k] = (unsigned)flag[k];
    val[k] = k;
    if (flag[k]) atomicAdd(count, 1);
}

}  // namespace

// Forward declarations of the traversal entry (sd_query.cu) used below.
extern "C" int sd_query(const sd_tree* t, const float* q, int64_t M, float* value, float* grad,
                        const sd_query_opts* opts, void* stream);

extern "C" int sd_lower_bound(const sd_tree* t, const float* q, int64_t M, float margin, float* lb, float* lb_grad,
                              int32_t* flag, void* stream)
{
    if (!t || M < 0 || (M > 0 && !q)) return SD_ERR_INVALID_ARG;
    SdUse use_{t, (cudaStream_t)stream};
    if (M == 0 || t->info.n_prims == 0) return SD_OK;
    if (M >= ((int64_t)1 << 31) / 3) return SD_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)stream;
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, sizeof(CutNode) * CUT_MAX + 256, st);
    if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    CutNode* cut = (CutNode*)tmp;
    int* ncut = (int*)(cut + CUT_MAX);
    unsigned* kb = (unsigned*)(ncut + 1);
    cudaMemsetAsync(kb, 0, sizeof(unsigned), st);
    const int m = (int)M;
    k_kappa<<<(t->P.n_prims + 255) / 256, 256, 0, st>>>(t->P, kb);
    k_cut<<<1, 1, 0, st>>>(t->P, kb, cut, ncut);
    k_lower_bound<<<(m + 127) / 128, 128, 0, st>>>(cut, ncut, t->info.alpha, q, m, margin, lb, lb_grad, flag);
    sd_count_launches(3);
    e = cudaGetLastError();
    cudaFreeAsync(tmp, st);
    return sd_cuda_status(e);
}

extern "C" int sd_surrogate_query(const sd_tree* t, const float* params, const float* frame, float margin,
                                  const float* q, int64_t M, float* value, float* grad, int32_t* routed,
                                  int64_t* n_routed, void* stream)
{
    if (!t || !params || !frame || M < 0 || (M > 0 && (!q || !value))) return SD_ERR_INVALID_ARG;
    SdUse use_{t, (cudaStream_t)stream};
    if (n_routed) *n_routed = 0;
    if (M == 0) return SD_OK;
    if (M >= ((int64_t)1 << 31) / 3) return SD_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)stream;
    const int m = (int)M;
    if (t->info.n_prims == 0) return sd_query(t, q, M, value, grad, nullptr, stream);
    // scratch: flags, sort keys/values, gathered queries and results
    size_t bytes = sizeof(int) * 8 * (size_t)m + sizeof(float) * 11 * (size_t)m +
                   sizeof(uint32_t) * sdsort::hist_words(m, 1) + 4096;
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, bytes, st);
    if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    int* flag = (int*)tmp;
    unsigned* k0 = (unsigned*)(flag + m);
    unsigned* k1 = k0 + m;
    int* v0 = (int*)(k1 + m);
    int* v1 = v0 + m;
    int* cnt = v1 + m;
    float* qg = (float*)(cnt + 64);
    float* vg = qg + 3 * (size_t)m;
    float* gg = vg + m;
    float* lbv = gg + 3 * (size_t)m;
    float* lbg = lbv + m;
    uint32_t* hist = (uint32_t*)(lbg + 3 * (size_t)m);
    cudaMemsetAsync(cnt, 0, sizeof(int), st);
    int rc = sd_lower_bound(t, q, M, margin, lbv, grad ? lbg : nullptr, flag, stream);
    if (rc != SD_OK) { cudaFreeAsync(tmp, st); return rc; }
    k_iota_flagkey<<<(m + 255) / 256, 256, 0, st>>>(flag, m, k0, v0, cnt);
    int nl = 1;
    // stable partition: exact queries first, surrogate queries after
    int where = sdsort::sort_pairs<unsigned, int>(k0, v0, k1, v1, m, 1, hist, st, &nl);
    int* idx = where ? v1 : v0;
    int hcnt = 0;
    e = cudaMemcpyAsync(&hcnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFreeAsync(tmp, st); return sd_cuda_status(e); }
    const int nm = hcnt, nb = m - nm;
    if (routed) cudaMemcpyAsync(routed, flag, sizeof(int) * (size_t)m, cudaMemcpyDeviceToDevice, st);
    k_gather3<<<(m + 255) / 256, 256, 0, st>>>(q, idx, m, qg);
    ++nl;
    if (nb > 0) {
        rc = sd_query(t, qg, nb, vg, grad ? gg : nullptr, nullptr, stream);
        if (rc != SD_OK) { cudaFreeAsync(tmp, st); return rc; }
    }
    if (nm > 0) {
        rc = sd_mlp_forward(params, frame, qg + 3 * (size_t)nb, nm, vg + nb, grad ? gg + 3 * (size_t)nb : nullptr,
                            stream);
        if (rc != SD_OK) { cudaFreeAsync(tmp, st); return rc; }
    }
    k_scatter<<<(m + 255) / 256, 256, 0, st>>>(idx, m, nb, vg, grad ? gg : nullptr, lbv, lbg, value, grad);
    ++nl;
    sd_count_launches(nl);
    e = cudaGetLastError();
    cudaFreeAsync(tmp, st);
    if (n_routed) *n_routed = nm;
    return sd_cuda_status(e);
}
