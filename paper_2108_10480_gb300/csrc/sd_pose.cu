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
#include <vector>

#include "sd_common.cuh"

namespace {

struct PoseF {
    float R[9];   // row-major rotation
    float p[3];
    float J[9];   // row-major left Jacobian J_l(theta)
};

// R(theta) (Rodrigues) and the left Jacobian J_l(theta) in FP64, row-major
void pose_matrices(const double* pose, double* R, double* J)
{
    const double tx = pose[0], ty = pose[1], tz = pose[2];
    const double th = std::sqrt(tx * tx + ty * ty + tz * tz);
    // R = I + a [t]x + b [t]x^2, J_l = I + b [t]x + c [t]x^2
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
        R[i] = I + a * K[i] + b * K2[i];
        J[i] = I + b * K[i] + c * K2[i];
    }
}

void pose_from_vector(const double* pose, PoseF& P)
{
    double R[9], J[9];
    pose_matrices(pose, R, J);
    for (int i = 0; i < 9; ++i) {
        P.R[i] = (float)R[i];
        P.J[i] = (float)J[i];
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
    SdUse use_{t, (cudaStream_t)stream};
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

// One shard of a body's vertices (Sec. 3.6, the outer sum of Eq. lse_full2 /
// Eq. dlse_full is associative): its LSE-shifted partial (m, s, v, sum e g,
// sum e (R x0) x g) with e = exp(t_k - m), written to part[9] on the device.
namespace {

__global__ void k_pose_part_final(const Part* __restrict__ parts, int nparts, float* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Part r = parts[0];
    for (int b = 1; b < nparts; ++b) part_merge(r, parts[b]);
    out[0] = r.m; out[1] = r.s; out[2] = r.v;
    for (int j = 0; j < 3; ++j) { out[3 + j] = r.gp[j]; out[6 + j] = r.gt[j]; }
}

}  // namespace

extern "C" int sd_pose_partial(const float* X0, const float* value, const float* grad, const float* gamma,
                               int64_t M, const double* pose, float alpha_q, float* part, void* stream)
{
    if (!pose || !part || M < 0 || (M > 0 && (!X0 || !value || !grad))) return SD_ERR_INVALID_ARG;
    if (!(alpha_q > 0.f) && M > 0 && !gamma) return SD_ERR_INVALID_ARG;
    if (M >= ((int64_t)1 << 31) / 3) return SD_ERR_TOO_LARGE;
    for (int j = 0; j < 6; ++j)
        if (!std::isfinite(pose[j])) return SD_ERR_NONFINITE;
    cudaStream_t st = (cudaStream_t)stream;
    if (M == 0) {
        // the empty shard: the merge's neutral element
        const float empty[9] = {-INFINITY, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        return sd_cuda_status(cudaMemcpyAsync(part, empty, sizeof(empty), cudaMemcpyHostToDevice, st));
    }
    PoseF P;
    pose_from_vector(pose, P);
    int m = (int)M;
    int nparts = std::min((m + RB - 1) / RB, 1024);
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, sizeof(Part) * nparts, st);
    if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    k_pose_partials<<<nparts, RB, 0, st>>>(X0, value, grad, gamma, m, alpha_q, P, (Part*)tmp);
    k_pose_part_final<<<1, 32, 0, st>>>((const Part*)tmp, nparts, part);
    sd_count_launches(2);
    e = cudaGetLastError();
    cudaFreeAsync(tmp, st);
    return sd_cuda_status(e);
}

extern "C" int sd_pose_merge(const double* parts, int32_t n, const double* pose, float alpha_q, double* out)
{
    if (!parts || n <= 0 || !pose || !out) return SD_ERR_INVALID_ARG;
    for (int j = 0; j < 6; ++j)
        if (!std::isfinite(pose[j])) return SD_ERR_NONFINITE;
    const bool lse = alpha_q > 0.f;
    double mx = -INFINITY;
    for (int i = 0; i < n; ++i)
        if (parts[9 * i + 1] > 0.0 && parts[9 * i] > mx) mx = parts[9 * i];
    if (lse && !(mx > -INFINITY)) return SD_ERR_INVALID_ARG;    // every shard empty
    double r[9] = {0.0};
    for (int i = 0; i < n; ++i) {
        const double* p = parts + 9 * i;
        if (!(p[1] > 0.0) && lse) continue;                       // an empty shard adds nothing
        const double e = lse ? std::exp(p[0] - mx) : 1.0;
        for (int j = 1; j < 9; ++j) r[j] += p[j] * e;
    }
    double R[9], J[9];
    pose_matrices(pose, R, J);
    const double nrm = lse ? 1.0 / r[1] : 1.0;
    out[0] = lse ? -(mx + std::log(r[1])) / (double)alpha_q : r[2];
    for (int j = 0; j < 3; ++j) out[1 + j] = r[3 + j] * nrm;
    for (int j = 0; j < 3; ++j)
        out[4 + j] = (J[0 * 3 + j] * r[6] + J[1 * 3 + j] * r[7] + J[2 * 3 + j] * r[8]) * nrm;
    return SD_OK;
}

// ---------------------------------------------------------------------------
// Batched multi-body evaluation: many rigid bodies with uneven vertex counts
// against one data mesh. One pass places every body's vertices from a
// per-body pose table, orders all of them along one Morton curve, runs ONE
// persistent traversal launch over the flattened list, and reduces each body
// (outer LogSumExp and 6-DoF gradient). All buffers are allocated when the
// batch is created; sd_batch_run only enqueues work on the stream (no
// allocation, no synchronisation), so a caller can capture it in a CUDA
// graph and replay it.
// ---------------------------------------------------------------------------
struct sd_batch {
    const sd_tree* tree;
    int B;
    int M;
    const float* X0;
    void* mem;
    int* body_of;       // [M]
    float* X;           // [M,3]
    float* value;       // [M]
    float* grad;        // [M,3]
    int32_t* order;     // [M]
    void* oscratch;     // ordering scratch
    int* work;          // packet counter
    PoseF* poses;       // [B]
    int nchunks;
    int4* chunks;       // (start, end, body, 0) per chunk, bodies in order
    int* body_chunk;    // [B + 1] first chunk of each body
    Part* parts;        // [nchunks]
    float* fin;         // [B, 9]
    bool posed;
};

namespace {

constexpr int CHUNK = 4096;

__global__ void k_batch_place(const float* __restrict__ X0, const int* __restrict__ body_of, int M,
                              const PoseF* __restrict__ poses, float* __restrict__ X)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const PoseF& P = poses[body_of[k]];
    float3 y = rot(P, f3(X0[3 * k], X0[3 * k + 1], X0[3 * k + 2]));
    X[3 * k] = y.x + P.p[0];
    X[3 * k + 1] = y.y + P.p[1];
    X[3 * k + 2] = y.z + P.p[2];
}

// one block per chunk of one body: LSE-shifted partial sums
__global__ void __launch_bounds__(RB) k_batch_partials(const float* __restrict__ X0, const float* __restrict__ value,
                                                      const float* __restrict__ grad, const int4* __restrict__ chunks,
                                                      const PoseF* __restrict__ poses, float alpha_q,
                                                      Part* __restrict__ parts)
{
    __shared__ Part sp[RB / 32];
    const int4 ch = chunks[blockIdx.x];
    const PoseF& P = poses[ch.z];
    Part a;
    a.m = -INFINITY; a.s = 0.f; a.v = 0.f;
    for (int j = 0; j < 3; ++j) a.gp[j] = a.gt[j] = 0.f;
    for (int k = ch.x + threadIdx.x; k < ch.y; k += RB) {
        float d = value[k];
        float3 g = f3(grad[3 * k], grad[3 * k + 1], grad[3 * k + 2]);
        float3 y = rot(P, f3(X0[3 * k], X0[3 * k + 1], X0[3 * k + 2]));
        float3 t = f3(y.y * g.z - y.z * g.y, y.z * g.x - y.x * g.z, y.x * g.y - y.y * g.x);
        Part b;
        b.m = -alpha_q * d; b.s = 1.f; b.v = d;
        b.gp[0] = g.x; b.gp[1] = g.y; b.gp[2] = g.z;
        b.gt[0] = t.x; b.gt[1] = t.y; b.gt[2] = t.z;
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

// one thread per body: merge its chunks in order; out[b] = (D, dD/dp, dD/dtheta)
__global__ void k_batch_final(const Part* __restrict__ parts, const int* __restrict__ body_chunk, int B,
                              const PoseF* __restrict__ poses, float alpha_q, float* __restrict__ out)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    Part r = parts[body_chunk[b]];
    for (int c = body_chunk[b] + 1; c < body_chunk[b + 1]; ++c) part_merge(r, parts[c]);
    const PoseF& P = poses[b];
    float n = 1.f / r.s;
    float gt[3] = {r.gt[0] * n, r.gt[1] * n, r.gt[2] * n};
    float* o = out + 7 * b;
    o[0] = -(r.m + logf(r.s)) / alpha_q;
    for (int j = 0; j < 3; ++j) o[1 + j] = r.gp[j] * n;
    for (int j = 0; j < 3; ++j) o[4 + j] = P.J[0 * 3 + j] * gt[0] + P.J[1 * 3 + j] * gt[1] + P.J[2 * 3 + j] * gt[2];
}

__global__ void k_fill_body(int* __restrict__ body_of, int start, int end, int b)
{
    int k = start + blockIdx.x * blockDim.x + threadIdx.x;
    if (k < end) body_of[k] = b;
}

}  // namespace

extern "C" int sd_batch_create(const sd_tree* t, const float* X0, const int64_t* offsets, int32_t nbodies,
                               sd_batch** out)
{
    if (!out) return SD_ERR_INVALID_ARG;
    *out = nullptr;
    if (!t || !offsets || nbodies <= 0) return SD_ERR_INVALID_ARG;
    if (offsets[0] != 0) return SD_ERR_INVALID_ARG;
    for (int b = 0; b < nbodies; ++b)
        if (offsets[b + 1] <= offsets[b]) return SD_ERR_INVALID_ARG;   // every body has a vertex
    int64_t M64 = offsets[nbodies];
    if (!X0) return SD_ERR_INVALID_ARG;
    if (M64 >= ((int64_t)1 << 31) / 3) return SD_ERR_TOO_LARGE;
    const int M = (int)M64, B = nbodies;
    std::vector<int4> chunks;
    std::vector<int> body_chunk(B + 1);
    for (int b = 0; b < B; ++b) {
        body_chunk[b] = (int)chunks.size();
        for (int64_t s = offsets[b]; s < offsets[b + 1]; s += CHUNK)
            chunks.push_back(make_int4((int)s, (int)std::min<int64_t>(s + CHUNK, offsets[b + 1]), b, 0));
    }
    body_chunk[B] = (int)chunks.size();
    const int NC = (int)chunks.size();
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += al(std::max<size_t>(bytes, 1)); return o; };
    size_t o_body = carve(sizeof(int) * (size_t)M);
    size_t o_X = carve(sizeof(float) * 3 * (size_t)M);
    size_t o_v = carve(sizeof(float) * (size_t)M);
    size_t o_g = carve(sizeof(float) * 3 * (size_t)M);
    size_t o_ord = carve(sizeof(int32_t) * (size_t)M);
    size_t o_os = carve(sdint::order_scratch_bytes(M));
    size_t o_work = carve(sizeof(int));
    size_t o_pose = carve(sizeof(PoseF) * B);
    size_t o_ch = carve(sizeof(int4) * NC);
    size_t o_bc = carve(sizeof(int) * (B + 1));
    size_t o_parts = carve(sizeof(Part) * NC);
    size_t o_fin = carve(sizeof(float) * 9 * B);
    sd_batch* bt = new sd_batch();
    bt->tree = t; bt->B = B; bt->M = M; bt->X0 = X0; bt->nchunks = NC; bt->posed = false;
    cudaError_t e = cudaMalloc(&bt->mem, off);
    if (e != cudaSuccess) { delete bt; cudaGetLastError(); return SD_ERR_OOM; }
    char* base = (char*)bt->mem;
    bt->body_of = (int*)(base + o_body);
    bt->X = (float*)(base + o_X);
    bt->value = (float*)(base + o_v);
    bt->grad = (float*)(base + o_g);
    bt->order = (int32_t*)(base + o_ord);
    bt->oscratch = base + o_os;
    bt->work = (int*)(base + o_work);
    bt->poses = (PoseF*)(base + o_pose);
    bt->chunks = (int4*)(base + o_ch);
    bt->body_chunk = (int*)(base + o_bc);
    bt->parts = (Part*)(base + o_parts);
    bt->fin = (float*)(base + o_fin);
    e = cudaMemcpy(bt->chunks, chunks.data(), sizeof(int4) * NC, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->body_chunk, body_chunk.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice);
    for (int b = 0; b < B && e == cudaSuccess; ++b) {
        int n = (int)(offsets[b + 1] - offsets[b]);
        k_fill_body<<<(n + 255) / 256, 256>>>(bt->body_of, (int)offsets[b], (int)offsets[b + 1], b);
        e = cudaGetLastError();
    }
    sd_count_launches(B);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { cudaFree(bt->mem); delete bt; return sd_cuda_status(e); }
    *out = bt;
    return SD_OK;
}

extern "C" int sd_batch_set_poses(sd_batch* bt, const double* poses, void* stream)
{
    if (!bt || !poses) return SD_ERR_INVALID_ARG;
    std::vector<PoseF> P(bt->B);
    for (int b = 0; b < bt->B; ++b) {
        for (int j = 0; j < 6; ++j)
            if (!std::isfinite(poses[6 * b + j])) return SD_ERR_NONFINITE;
        pose_from_vector(poses + 6 * b, P[b]);
    }
    // pageable source: the copy is staged before the call returns
    cudaError_t e = cudaMemcpyAsync(bt->poses, P.data(), sizeof(PoseF) * bt->B, cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return sd_cuda_status(e);
    bt->posed = true;
    return SD_OK;
}

extern "C" int sd_batch_run(sd_batch* bt, float alpha_q, int32_t block, float* body_out, void* stream)
{
    if (!bt || !body_out || !(alpha_q > 0.f) || !bt->posed) return SD_ERR_INVALID_ARG;
    SdUse use_{bt->tree, (cudaStream_t)stream};
    cudaStream_t st = (cudaStream_t)stream;
    const int M = bt->M;
    k_batch_place<<<(M + 255) / 256, 256, 0, st>>>(bt->X0, bt->body_of, M, bt->poses, bt->X);
    sd_count_launches(1);
    int rc = sdint::order_into(bt->tree, bt->X, M, bt->order, bt->oscratch, st);
    if (rc != SD_OK) return rc;
    rc = sdint::traverse(bt->tree, bt->X, M, bt->order, bt->value, bt->grad, block, bt->work, st);
    if (rc != SD_OK) return rc;
    k_batch_partials<<<bt->nchunks, RB, 0, st>>>(bt->X0, bt->value, bt->grad, bt->chunks, bt->poses, alpha_q,
                                                  bt->parts);
    k_batch_final<<<(bt->B + 63) / 64, 64, 0, st>>>(bt->parts, bt->body_chunk, bt->B, bt->poses, alpha_q,
                                                     body_out);
    sd_count_launches(2);
    return sd_cuda_status(cudaGetLastError());
}

extern "C" int sd_batch_vertex_outputs(const sd_batch* bt, const float** X, const float** value, const float** grad)
{
    if (!bt) return SD_ERR_INVALID_ARG;
    if (X) *X = bt->X;
    if (value) *value = bt->value;
    if (grad) *grad = bt->grad;
    return SD_OK;
}

extern "C" void sd_batch_free(sd_batch* bt)
{
    if (!bt) return;
    if (bt->mem) cudaFree(bt->mem);
    delete bt;
}
