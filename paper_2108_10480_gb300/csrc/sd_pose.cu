// Rigid-pose queries and their adjoint (Sec. 4.5, Eq. opt; Sec. 3.6,
// Eq. lse_full2 / Eq. dlse_full with point queries, n(g) = 0).
//
// A body's vertices are placed by x_k = R(theta) x0_k + p, theta a rotation
// vector (exponential map); the smooth distance and gradient of every x_k
// come from sd_query. The reduction then forms either
//   D = -(1/alpha_q) log sum_k exp(-alpha_q d^_k)   (alpha_q > 0), with
//   gamma_k = exp(-alpha_q d^_k) / sum_j exp(-alpha_q d^_j), or
//   sum_k gamma_k d^_k for caller-given gamma_k      (alpha_q <= 0),
// and the gradients
//   dD/dp = sum_k gamma_k g_k,
//   dD/dtheta = J_l(theta)^T sum_k gamma_k (R x0_k) x g_k,
//   dD/dx0_k = gamma_k R^T g_k,
// with g_k = grad d^(x_k) and J_l the left Jacobian of SO(3)
// (d(R x0) = -[R x0]_x J_l dtheta).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sd_common.cuh"

namespace {

struct PoseF {
    float R[9];   // row-major rotation
    float p[3];
    float J[9];   // row-major left Jacobian J_l(theta)
};

void pose_from_vector(const double* pose, PoseF& P)
{
    const double tx = pose[0], ty = pose[1], tz = pose[2];
    const double th = std::sqrt(tx * tx + ty * ty + tz * tz);
    // Rodrigues: R = I + a [t]x + b [t]x^2, J_l = I + b [t]x + c [t]x^2
    double a, b, c;
    if (th < 1e-4) {
        const double t2 = th * th;
        a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
        b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        c = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
    } else {
        a = std::sin(th) / th;
        b = (1.0 - std::cos(th)) / (th * th);
        c = (th - std::sin(th)) / (th * th * th);
    }
    const double K[9] = {0.0, -tz, ty, tz, 0.0, -tx, -ty, tx, 0.0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += K[3 * i + k] * K[3 * k + j];
            K2[3 * i + j] = s;
        }
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        P.R[i] = (float)(I + a * K[i] + b * K2[i]);
        P.J[i] = (float)(I + b * K[i] + c * K2[i]);
    }
    for (int j = 0; j < 3; ++j) P.p[j] = (float)pose[3 + j];
}

__device__ __forceinline__ float3 rot(const PoseF& P, float3 x)
{
    return f3(fmaf(P.R[0], x.x, fmaf(P.R[1], x.y, P.R[2] * x.z)),
              fmaf(P.R[3], x.x, fmaf(P.R[4], x.y, P.R[5] * x.z)),
              fmaf(P.R[6], x.x, fmaf(P.R[7], x.y, P.R[8] * x.z)));
}

__global__ void k_pose_transform(const float* __restrict__ X0, int M, PoseF P, float* __restrict__ X)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    float3 y = rot(P, f3(X0[3 * k], X0[3 * k + 1], X0[3 * k + 2]));
    X[3 * k] = y.x + P.p[0];
    X[3 * k + 1] = y.y + P.p[1];
    X[3 * k + 2] = y.z + P.p[2];
}

// partial sums of one block: LSE-shifted (m, s) and the weighted sums of
// g_k and y_k x g_k (8 floats)
struct Part {
    float m, s, v;      // max exponent, shifted weight sum, weighted value sum (linear mode)
    float gp[3], gt[3];
};

constexpr int RB = 256;

__device__ __forceinline__ void part_merge(Part& a, const Part& b)
{
    float mn = fmaxf(a.m, b.m);
    float ea = (a.m == -INFINITY) ? 0.f : __expf(a.m - mn);
    float eb = (b.m == -INFINITY) ? 0.f : __expf(b.m - mn);
    a.s = a.s * ea + b.s * eb;
    a.v = a.v * ea + b.v * eb;
    for (int j = 0; j < 3; ++j) {
        a.gp[j] = a.gp[j] * ea + b.gp[j] * eb;
        a.gt[j] = a.gt[j] * ea + b.gt[j] * eb;
    }
    a.m = mn;
}

__device__ __forceinline__ Part part_shfl(const Part& p, int o)
{
    Part q;
    q.m = __shfl_xor_sync(0xffffffffu, p.m, o);
    q.s = __shfl_xor_sync(0xffffffffu, p.s, o);
    q.v = __shfl_xor_sync(0xffffffffu, p.v, o);
    for (int j = 0; j < 3; ++j) {
        q.gp[j] = __shfl_xor_sync(0xffffffffu, p.gp[j], o);
        q.gt[j] = __shfl_xor_sync(0xffffffffu, p.gt[j], o);
    }
    return q;
}

// Every thread folds a strided set of vertices; warps and then the block
// combine in a fixed order, so the result does not depend on timing.
// lse: exponent t_k = -alpha_q d^_k; otherwise the weight is gamma_k
// (carried with exponent 0 so the same merge applies).
__global__ void __launch_bounds__(RB) k_pose_partials(const float* __restrict__ X0, const float* __restrict__ value,
                                                     const float* __restrict__ grad, const float* __restrict__ gamma,
                                                     int M, float alpha_q, PoseF P, Part* __restrict__ parts)
{
    __shared__ Part sp[RB / 32];
    Part a;
    a.m = -INFINITY; a.s = 0.f; a.v = 0.f;
    for (int j = 0; j < 3; ++j) a.gp[j] = a.gt[j] = 0.f;
    const bool lse = alpha_q > 0.f;
    for (int k = blockIdx.x * RB + threadIdx.x; k < M; k += gridDim.x * RB) {
        float d = value[k];
        float3 g = f3(grad[3 * k], grad[3 * k + 1], grad[3 * k + 2]);
        float3 y = rot(P, f3(X0[3 * k], X0[3 * k + 1], X0[3 * k + 2]));
        float3 t = f3(y.y * g.z - y.z * g.y, y.z * g.x - y.x * g.z, y.x * g.y - y.y * g.x);
        Part b;
        b.m = lse ? -alpha_q * d : 0.f;
        b.s = lse ? 1.f : gamma[k];
        b.v = b.s * d;
        b.gp[0] = b.s * g.x; b.gp[1] = b.s * g.y; b.gp[2] = b.s * g.z;
        b.gt[0] = b.s * t.x; b.gt[1] = b.s * t.y; b.gt[2] = b.s * t.z;
        part_merge(a, b);
    }
    for (int o = 1; o < 32; o <<= 1) {
        Part b = part_shfl(a, o);
        part_merge(a, b);
    }
    if ((threadIdx.x & 31) == 0) sp[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        Part r = sp[0];
        for (int w = 1; w < RB / 32; ++w) part_merge(r, sp[w]);
        parts[blockIdx.x] = r;
    }
}

// out = (D, dD/dp (3), dD/dtheta (3)), then the final shift m and shifted sum s
// (used by k_pose_dx0 to form the softmin weights)
__global__ void k_pose_final(const Part* __restrict__ parts, int nparts, float alpha_q, PoseF P,
                             float* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Part r = parts[0];
    for (int b = 1; b < nparts; ++b) part_merge(r, parts[b]);
    const bool lse = alpha_q > 0.f;
    float n = lse ? 1.f / r.s : 1.f;
    float D = lse ? -(r.m + logf(r.s)) / alpha_q : r.v;
    float gt[3] = {r.gt[0] * n, r.gt[1] * n, r.gt[2] * n};
    out[0] = D;
    for (int j = 0; j < 3; ++j) out[1 + j] = r.gp[j] * n;
    for (int j = 0; j < 3; ++j) out[4 + j] = P.J[0 * 3 + j] * gt[0] + P.J[1 * 3 + j] * gt[1] + P.J[2 * 3 + j] * gt[2];
    out[7] = r.m;
    out[8] = r.s;
}

// dL/dx0_k = w_k R^T g_k with w_k = gamma_k (linear) or the softmin weight
__global__ void k_pose_dx0(const float* __restrict__ value, const float* __restrict__ grad,
                           const float* __restrict__ gamma, int M, float alpha_q, PoseF P,
                           const float* __restrict__ fin, float* __restrict__ dX0)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    float w = alpha_q > 0.f ? __expf(-alpha_q * value[k] - fin[7]) / fin[8] : gamma[k];
    float3 g = f3(grad[3 * k] * w, grad[3 * k + 1] * w, grad[3 * k + 2] * w);
    dX0[3 * k] = P.R[0] * g.x + P.R[3] * g.y + P.R[6] * g.z;
    dX0[3 * k + 1] = P.R[1] * g.x + P.R[4] * g.y + P.R[7] * g.z;
    dX0[3 * k + 2] = P.R[2] * g.x + P.R[5] * g.y + P.R[8] * g.z;
}

}  // namespace

extern "C" int sd_pose_query(const sd_tree* t, const float* X0, int64_t M, const double* pose, float* X,
                             float* value, float* grad, const sd_query_opts* opts, void* stream)
{
    if (!t || !pose || M < 0 || (M > 0 && (!X0 || !X || !value))) return SD_ERR_INVALID_ARG;
    for (int j = 0; j < 6; ++j)
        if (!std::isfinite(pose[j])) return SD_ERR_NONFINITE;
    if (M == 0) return SD_OK;
    if (M >= ((int64_t)1 << 31) / 3) return SD_ERR_TOO_LARGE;
    PoseF P;
    pose_from_vector(pose, P);
    cudaStream_t st = (cudaStream_t)stream;
    int m = (int)M;
    k_pose_transform<<<(m + 255) / 256, 256, 0, st>>>(X0, m, P, X);
    sd_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sd_cuda_status(e);
    return sd_query(t, X, M, value, grad, opts, stream);
}

extern "C" int sd_pose_reduce(const float* X0, const float* value, const float* grad, const float* gamma,
                              int64_t M, const double* pose, float alpha_q, float* out, float* dX0, void* stream)
{
    if (!pose || !out || M <= 0 || !X0 || !value || !grad) return SD_ERR_INVALID_ARG;
    if (!(alpha_q > 0.f) && !gamma) return SD_ERR_INVALID_ARG;
    if (M >= ((int64_t)1 << 31) / 3) return SD_ERR_TOO_LARGE;
    for (int j = 0; j < 6; ++j)
        if (!std::isfinite(pose[j])) return SD_ERR_NONFINITE;
    PoseF P;
    pose_from_vector(pose, P);
    cudaStream_t st = (cudaStream_t)stream;
    int m = (int)M;
    int nparts = std::min((m + RB - 1) / RB, 1024);
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, sizeof(Part) * nparts + sizeof(float) * 16, st);
    if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    Part* parts = (Part*)tmp;
    float* fin = (float*)(parts + nparts);
    k_pose_partials<<<nparts, RB, 0, st>>>(X0, value, grad, gamma, m, alpha_q, P, parts);
    k_pose_final<<<1, 32, 0, st>>>(parts, nparts, alpha_q, P, fin);
    cudaMemcpyAsync(out, fin, sizeof(float) * 7, cudaMemcpyDeviceToDevice, st);
    int nl = 2;
    if (dX0) {
        k_pose_dx0<<<(m + 255) / 256, 256, 0, st>>>(value, grad, gamma, m, alpha_q, P, fin, dX0);
        ++nl;
    }
    sd_count_launches(nl);
    e = cudaGetLastError();
    cudaFreeAsync(tmp, st);
    return sd_cuda_status(e);
}
