// sd_mesh_reduce: the smooth distance between the data mesh and a query
// mesh, and its gradient per query vertex (Sec. 3.6, Eq. lse_full,
// Eq. lse_full2, Eq. dlse_full), from per-primitive d^_j and translation
// gradients grad d^_j (sd_query_prims):
//   D = -(1/alpha_q) log sum_j exp(-alpha_q d^_j),  gamma_j its softmin weights,
//   grad_k D = sum_{j incident to k} gamma_j / (n(g_j) + 1) grad d^_j.
// Every sum is taken in a fixed order: the (max, sum) pairs of blocks of
// primitives are merged in block order, and each vertex adds its incident
// primitives in slot order (slots j * k + c stably sorted by vertex).
#include <cuda_runtime.h>

#include <cmath>

#include "sd_common.cuh"
#include "sd_sort.cuh"

namespace {

constexpr int MB = 256;

struct MPart {
    float m, s;
};

// block b: max and shifted sum of t_j = -alpha_q d^_j over its primitives
__global__ void __launch_bounds__(MB) k_mesh_partials(const float* __restrict__ val, int m, float alpha_q,
                                                      MPart* __restrict__ parts)
{
    __shared__ float sm[MB];
    __shared__ float ss[MB];
    int j = blockIdx.x * MB + threadIdx.x;
    float t = j < m ? -alpha_q * val[j] : -INFINITY;
    sm[threadIdx.x] = t;
    __syncthreads();
    for (int o = MB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] = fmaxf(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    const float mx = sm[0];
    ss[threadIdx.x] = (j < m && mx > -INFINITY) ? expf(t - mx) : 0.f;
    __syncthreads();
    for (int o = MB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) ss[threadIdx.x] += ss[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = MPart{mx, ss[0]};
}

// one thread merges the block partials in order: out[0] = D; mz = (M, Z)
__global__ void k_mesh_final(const MPart* __restrict__ parts, int nparts, float alpha_q, float* out, float* mz)
{
    if (threadIdx.x || blockIdx.x) return;
    float M = -INFINITY;
    for (int b = 0; b < nparts; ++b) M = fmaxf(M, parts[b].m);
    float Z = 0.f;
    for (int b = 0; b < nparts; ++b)
        if (parts[b].m > -INFINITY) Z += parts[b].s * expf(parts[b].m - M);
    out[0] = -(M + logf(Z)) / alpha_q;
    mz[0] = M;
    mz[1] = Z;
}

// (vertex, slot) pairs of every primitive corner; indices outside [0, nv)
// get the key nv and are never read back
__global__ void k_mesh_slots(const int* __restrict__ F, int n, int nv, unsigned* __restrict__ key,
                             int* __restrict__ slot)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int v = F[i];
    key[i] = (v >= 0 && v < nv) ? (unsigned)v : (unsigned)nv;
    slot[i] = i;
}

// range [first, last) of each vertex in the sorted keys
__global__ void k_mesh_bounds(const unsigned* __restrict__ key, int n, int nv, int* __restrict__ first,
                              int* __restrict__ last)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned k = key[i];
    if (k >= (unsigned)nv) return;
    if (i == 0 || key[i - 1] != k) first[k] = i;
    if (i == n - 1 || key[i + 1] != k) last[k] = i + 1;
}

__global__ void k_mesh_vgrad(const unsigned* __restrict__ key, const int* __restrict__ slot,
                             const int* __restrict__ first, const int* __restrict__ last, int nv, int k,
                             const float* __restrict__ val, const float* __restrict__ grad, float alpha_q,
                             const float* __restrict__ mz, float* __restrict__ vgrad)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const float M = mz[0], iz = 1.f / (mz[1] * (float)k);
    float g[3] = {0.f, 0.f, 0.f};
    for (int i = first[v]; i < last[v]; ++i) {
        int j = slot[i] / k;
        float w = expf(-alpha_q * val[j] - M) * iz;
        for (int d = 0; d < 3; ++d) g[d] = fmaf(w, grad[3 * j + d], g[d]);
    }
    for (int d = 0; d < 3; ++d) vgrad[3 * v + d] = g[d];
}

}  // namespace

extern "C" int sd_mesh_reduce(const int32_t* QF, int32_t k, int64_t M, int64_t nqv, const float* value,
                              const float* grad, float alpha_q, float* out, float* vgrad, int32_t* status,
                              void* stream)
{
    if (k < 1 || k > 3 || M <= 0 || nqv < 0 || !QF || !value || !out || !(alpha_q > 0.f) || !std::isfinite(alpha_q))
        return SD_ERR_INVALID_ARG;
    if (vgrad && nqv > 0 && !grad) return SD_ERR_INVALID_ARG;
    if (k * M >= ((int64_t)1 << 31) / 2 || nqv >= ((int64_t)1 << 30)) return SD_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)stream;
    const int m = (int)M, n = (int)(k * M), nv = (int)nqv;
    const int nparts = (m + MB - 1) / MB;
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) <= nqv) ++bits;     // keys 0..nv
    const bool want_v = vgrad && nv > 0;
    size_t o_parts = 0, o_mz = o_parts + 16 * (((size_t)nparts * sizeof(MPart) + 15) / 16);
    size_t o_key = o_mz + 16;
    size_t o_rest = o_key;
    if (want_v) o_rest += sizeof(unsigned) * 4 * (size_t)n + sizeof(int) * 2 * (size_t)nv + 64;
    size_t o_hist = 16 * ((o_rest + 15) / 16);
    size_t bytes = o_hist + (want_v ? sizeof(uint32_t) * sdsort::hist_words(n, (bits + 7) / 8) : 0);
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, bytes, st);
    if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    char* b = (char*)tmp;
    MPart* parts = (MPart*)(b + o_parts);
    float* mz = (float*)(b + o_mz);
    int nl = 2;
    k_mesh_partials<<<nparts, MB, 0, st>>>(value, m, alpha_q, parts);
    k_mesh_final<<<1, 32, 0, st>>>(parts, nparts, alpha_q, out, mz);
    if (want_v) {
        unsigned* k0 = (unsigned*)(b + o_key);
        unsigned* k1 = k0 + n;
        int* s0 = (int*)(k1 + n);
        int* s1 = s0 + n;
        int* first = s1 + n;
        int* last = first + nv;
        uint32_t* hist = (uint32_t*)(b + o_hist);
        cudaMemsetAsync(first, 0, sizeof(int) * 2 * (size_t)nv, st);
        k_mesh_slots<<<(n + 255) / 256, 256, 0, st>>>(QF, n, nv, k0, s0);
        int where = sdsort::sort_pairs<unsigned, int>(k0, s0, k1, s1, n, bits, hist, st, &nl);
        const unsigned* sk = where ? k1 : k0;
        const int* sv = where ? s1 : s0;
        k_mesh_bounds<<<(n + 255) / 256, 256, 0, st>>>(sk, n, nv, first, last);
        k_mesh_vgrad<<<(nv + 255) / 256, 256, 0, st>>>(sk, sv, first, last, nv, k, value, grad, alpha_q, mz, vgrad);
        nl += 3;
    }
    sd_count_launches(nl);
    e = cudaGetLastError();
    cudaFreeAsync(tmp, st);
    return sd_cuda_status(e);
}
