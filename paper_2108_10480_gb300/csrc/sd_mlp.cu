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
// Inference (sd_mlp_forward): one fused kernel per 16-query tile and warp,
// bf16 tensor-core MMAs (mma.sync m16n8k16, fp32 accumulate), activations
// kept in registers between layers, weights in shared memory, and the input
// gradient dy/dx by back-propagation through the same weights.
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
// fused inference: bf16 tensor-core MLP, value and input gradient
// ---------------------------------------------------------------------------
constexpr int IW = 8;                   // warps per block
constexpr int S1 = 88;                  // W1 row stride (bf16): 80 used columns, conflict-free ldmatrix
constexpr int S2 = 136;                 // W2, W3 row stride (bf16)
constexpr int FS = 81;                  // per-warp feature row stride (fp32): 80 columns
constexpr int SMEM_W = HID * S1 + 2 * HID * S2;            // bf16 elements
constexpr int SMEM_STASH = 2 * 16 * HID;                   // fp16 dsilu of layers 1, 2 per warp
constexpr size_t SMEM_BYTES = sizeof(__nv_bfloat16) * SMEM_W + sizeof(float) * (4 * HID + 96 + 8) +
                              (size_t)IW * (sizeof(float) * 16 * FS + sizeof(__half) * SMEM_STASH);

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// acc[16][4] = A[16 x 16*KSTEPS] * W^T, W [128][stride] row-major (out, in):
// forward use, B(k = in, n = out) fragments by ldmatrix on W's rows
template <int KSTEPS, int STRIDE>
__device__ __forceinline__ void gemm_fwd(float (&acc)[16][4], const uint32_t (&A)[KSTEPS][4],
                                         const __nv_bfloat16* W, int lane)
{
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int mi = lane >> 3, ri = lane & 7;
#pragma unroll
    for (int kk = 0; kk < KSTEPS; ++kk) {
#pragma unroll
        for (int jp = 0; jp < 8; ++jp) {
            // matrices: (n0, k0), (n0, k0+8), (n0+8, k0), (n0+8, k0+8)
            const int n = jp * 16 + (mi >> 1) * 8 + ri;
            const int k = kk * 16 + (mi & 1) * 8;
            uint32_t b0, b1, b2, b3;
            ldsm_x4(smem_addr(W + n * STRIDE + k), b0, b1, b2, b3);
            mma(acc[2 * jp], A[kk], b0, b1);
            mma(acc[2 * jp + 1], A[kk], b2, b3);
        }
    }
}

// acc[NT][4] = G[16 x 128] * W, W [128][stride] (out, in): input-gradient use,
// B(k = out, n = in) fragments by transposing ldmatrix on W's rows
template <int NT, int STRIDE>
__device__ __forceinline__ void gemm_bwd(float (&acc)[NT][4], const uint32_t (&G)[8][4], const __nv_bfloat16* W,
                                         int lane)
{
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int mi = lane >> 3, ri = lane & 7;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
        for (int jp = 0; jp < NT / 2; ++jp) {
            // matrices: (k0, n0), (k0+8, n0), (k0, n0+8), (k0+8, n0+8)
            const int k = kk * 16 + (mi & 1) * 8 + ri;
            const int n = jp * 16 + (mi >> 1) * 8;
            uint32_t b0, b1, b2, b3;
            ldsm_x4_t(smem_addr(W + k * STRIDE + n), b0, b1, b2, b3);
            mma(acc[2 * jp], G[kk], b0, b1);
            mma(acc[2 * jp + 1], G[kk], b2, b3);
        }
    }
}

// C fragments [16 x 128] -> next layer's A fragments (8 k-steps)
__device__ __forceinline__ void c_to_a(const float (&v)[16][4], uint32_t (&A)[8][4])
{
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        A[kk][0] = pack_bf16(v[2 * kk][0], v[2 * kk][1]);
        A[kk][1] = pack_bf16(v[2 * kk][2], v[2 * kk][3]);
        A[kk][2] = pack_bf16(v[2 * kk + 1][0], v[2 * kk + 1][1]);
        A[kk][3] = pack_bf16(v[2 * kk + 1][2], v[2 * kk + 1][3]);
    }
}

__global__ void __launch_bounds__(IW * 32, 1) k_mlp_infer(const float* __restrict__ P, Frame fr,
                                                          const float* __restrict__ x, int n,
                                                          float* __restrict__ y, float* __restrict__ dydx)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* W1 = reinterpret_cast<__nv_bfloat16*>(smem);
    __nv_bfloat16* W2 = W1 + HID * S1;
    __nv_bfloat16* W3 = W2 + HID * S2;
    float* bias = reinterpret_cast<float*>(W3 + HID * S2);   // b1, b2, b3, w4 (bf16-rounded)
    float* Bq = bias + 4 * HID;                               // frequencies [32][3]
    float* misc = Bq + 96;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float* Fw = misc + 8 + warp * (16 * FS);
    __half* stash = reinterpret_cast<__half*>(misc + 8 + IW * 16 * FS) + warp * SMEM_STASH;
    // stage the weights (rounded to bf16) once per block
    for (int i = tid; i < HID * S1; i += blockDim.x) {
        int o = i / S1, k = i - o * S1;
        W1[i] = __float2bfloat16_rn(k < NIN ? P[OFF_W1 + o * NIN + k] : 0.f);
    }
    for (int i = tid; i < HID * S2; i += blockDim.x) {
        int o = i / S2, k = i - o * S2;
        W2[i] = __float2bfloat16_rn(k < HID ? P[OFF_W2 + o * HID + k] : 0.f);
        W3[i] = __float2bfloat16_rn(k < HID ? P[OFF_W3 + o * HID + k] : 0.f);
    }
    for (int i = tid; i < HID; i += blockDim.x) {
        bias[i] = P[OFF_B1 + i];
        bias[HID + i] = P[OFF_B2 + i];
        bias[2 * HID + i] = P[OFF_B3 + i];
        bias[3 * HID + i] = bf16r(P[OFF_W4 + i]);
    }
    for (int i = tid; i < 96; i += blockDim.x) Bq[i] = P[OFF_B + i];
    if (tid == 0) misc[0] = P[OFF_B4];
    __syncthreads();
    const int g = lane >> 2, t4 = lane & 3;
    const int ntiles = (n + 15) / 16;
    for (int tile = blockIdx.x * IW + warp; tile < ntiles; tile += gridDim.x * IW) {
        const int r0 = tile * 16;
        // features of the 16 rows: lanes 0..15 write xh, every lane 16 projections
        {
            const int row = lane >> 1, half = lane & 1;
            const int gr = min(r0 + row, n - 1);
            float xh[3];
            for (int j = 0; j < 3; ++j) xh[j] = (x[3 * gr + j] - fr.c[j]) / fr.h[j];
            float* f = Fw + row * FS;
            if (!half) { f[0] = xh[0]; f[1] = xh[1]; f[2] = xh[2]; }
            for (int mm = 0; mm < 16; ++mm) {
                const int m = half * 16 + mm;
                float p = fmaf(Bq[3 * m], xh[0], fmaf(Bq[3 * m + 1], xh[1], Bq[3 * m + 2] * xh[2]));
                float sv, cv;
                sincospif(p, &sv, &cv);
                f[3 + m] = sv;
                f[3 + NF + m] = cv;
            }
            if (!half) for (int c = NIN; c < 80; ++c) f[c] = 0.f;
        }
        __syncwarp();
        uint32_t A1[5][4];
#pragma unroll
        for (int kk = 0; kk < 5; ++kk) {
            const int c = kk * 16 + 2 * t4;
            A1[kk][0] = pack_bf16(Fw[g * FS + c], Fw[g * FS + c + 1]);
            A1[kk][1] = pack_bf16(Fw[(g + 8) * FS + c], Fw[(g + 8) * FS + c + 1]);
            A1[kk][2] = pack_bf16(Fw[g * FS + c + 8], Fw[g * FS + c + 9]);
            A1[kk][3] = pack_bf16(Fw[(g + 8) * FS + c + 8], Fw[(g + 8) * FS + c + 9]);
        }
        float acc[16][4];
        uint32_t A[8][4];
        uint32_t G[8][4];
        const float* w4 = bias + 3 * HID;
        // hidden layers 1, 2: z = acc + b, stash dsilu(z), a = silu(z)
        gemm_fwd<5, S1>(acc, A1, W1, lane);
#pragma unroll
        for (int layer = 0; layer < 2; ++layer) {
            if (layer == 1) gemm_fwd<8, S2>(acc, A, W2, lane);
            const float* b = bias + layer * HID;
            __half* st = stash + layer * 16 * HID;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = 8 * j + 2 * t4;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int row = g + (e >> 1) * 8, col = c + (e & 1);
                    const float z = acc[j][e] + b[col];
                    st[row * HID + col] = __float2half_rn(dsilu(z));
                    acc[j][e] = silu(z);
                }
            }
            c_to_a(acc, A);
        }
        // layer 3: a3 stays in acc; the input gradient starts from
        // g3 = s w4 dsilu(z3), packed straight into A fragments
        gemm_fwd<8, S2>(acc, A, W3, lane);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            float gv[2][4];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int j = 2 * kk + h2;
                const int c = 8 * j + 2 * t4;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int col = c + (e & 1);
                    const float z = acc[j][e] + bias[2 * HID + col];
                    gv[h2][e] = fr.s * w4[col] * dsilu(z);
                    acc[j][e] = silu(z);
                }
            }
            G[kk][0] = pack_bf16(gv[0][0], gv[0][1]);
            G[kk][1] = pack_bf16(gv[0][2], gv[0][3]);
            G[kk][2] = pack_bf16(gv[1][0], gv[1][1]);
            G[kk][3] = pack_bf16(gv[1][2], gv[1][3]);
        }
        // output: y = s (w4 . a3 + b4), rows g and g + 8
        float ya = 0.f, yb = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int c = 8 * j + 2 * t4;
            ya = fmaf(acc[j][0], w4[c], fmaf(acc[j][1], w4[c + 1], ya));
            yb = fmaf(acc[j][2], w4[c], fmaf(acc[j][3], w4[c + 1], yb));
        }
        ya += __shfl_xor_sync(0xffffffffu, ya, 1);
        ya += __shfl_xor_sync(0xffffffffu, ya, 2);
        yb += __shfl_xor_sync(0xffffffffu, yb, 1);
        yb += __shfl_xor_sync(0xffffffffu, yb, 2);
        if (t4 == 0) {
            if (r0 + g < n) y[r0 + g] = fr.s * (ya + misc[0]);
            if (r0 + g + 8 < n) y[r0 + g + 8] = fr.s * (yb + misc[0]);
        }
        __syncwarp();
        if (dydx) {
            // back through W3, W2 (times the stashed dsilu), W1
#pragma unroll
            for (int layer = 1; layer >= 0; --layer) {
                gemm_bwd<16, S2>(acc, G, layer == 1 ? W3 : W2, lane);
                const __half* st = stash + layer * 16 * HID;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = 8 * j + 2 * t4;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int row = g + (e >> 1) * 8, col = c + (e & 1);
                        acc[j][e] *= __half2float(st[row * HID + col]);
                    }
                }
                c_to_a(acc, G);
            }
            float gf[10][4];
            gemm_bwd<10, S1>(gf, G, W1, lane);
            // features -> xh: d f_j / d xh for xh, sin(pi B xh), cos(pi B xh)
            float ga[3] = {0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < 10; ++j) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int row = g + (e >> 1) * 8, col = 8 * j + 2 * t4 + (e & 1);
                    const float v = gf[j][e];
                    float* gg = (e >> 1) ? gb : ga;
                    if (col < 3) {
                        gg[col] += v;
                    } else if (col < 3 + NF) {
                        const int m = col - 3;
                        const float k = v * 3.14159265358979f * Fw[row * FS + 3 + NF + m];
                        gg[0] = fmaf(k, Bq[3 * m], gg[0]); gg[1] = fmaf(k, Bq[3 * m + 1], gg[1]);
                        gg[2] = fmaf(k, Bq[3 * m + 2], gg[2]);
                    } else if (col < NIN) {
                        const int m = col - 3 - NF;
                        const float k = -v * 3.14159265358979f * Fw[row * FS + 3 + m];
                        gg[0] = fmaf(k, Bq[3 * m], gg[0]); gg[1] = fmaf(k, Bq[3 * m + 1], gg[1]);
                        gg[2] = fmaf(k, Bq[3 * m + 2], gg[2]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                ga[j] += __shfl_xor_sync(0xffffffffu, ga[j], 1);
                ga[j] += __shfl_xor_sync(0xffffffffu, ga[j], 2);
                gb[j] += __shfl_xor_sync(0xffffffffu, gb[j], 1);
                gb[j] += __shfl_xor_sync(0xffffffffu, gb[j], 2);
            }
            if (t4 == 0) {
                if (r0 + g < n)
                    for (int j = 0; j < 3; ++j) dydx[3 * (r0 + g) + j] = ga[j] / fr.h[j];
                if (r0 + g + 8 < n)
                    for (int j = 0; j < 3; ++j) dydx[3 * (r0 + g + 8) + j] = gb[j] / fr.h[j];
            }
        }
        __syncwarp();
    }
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
    cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    Frame fr = make_frame(frame);
    int tiles = (int)((n + 15) / 16);
    int blocks = std::max(1, std::min(sm_count_mlp(), (tiles + IW - 1) / IW));
    k_mlp_infer<<<blocks, IW * 32, SMEM_BYTES, (cudaStream_t)stream>>>(params, fr, x, (int)n, y, dydx);
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
        c.w = slot ? P.nw2[rec].y : P.nw2[rec].x;
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
    int where = sdsort::sort_pairs<unsigned, int>(k0, v0, k1, v1, m, 1, hist, t->status, 1 << SD_ERR_TIMEOUT, st, &nl);
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
