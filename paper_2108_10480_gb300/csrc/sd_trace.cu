// sd_sphere_trace: sphere tracing of the zero isosurface of the smooth
// distance (Sec. 4.2; Hart 1996) through a pinhole camera, as a wavefront:
// every iteration evaluates d^ (Barnes-Hut, value only) at the current point
// of every ray still marching, in one traversal launch over a compacted list
// of rays, then advances each ray by its d^ and drops the rays that hit
// (d^ < eps) or left (t > t_max, or max_steps evaluations). The list keeps
// the rays' 8 x 4 pixel-tile order (a stable partition), so each warp packet
// marches 32 neighbouring rays.
#include <cuda_runtime.h>

#include <cmath>

#include "sd_common.cuh"
#include "sd_sort.cuh"

namespace {

struct Cam {
    float3 eye, f, r, u;
    float tx, ty;   // tan(fov_y / 2) * W / H, tan(fov_y / 2)
    int W, H;
};

__device__ __forceinline__ float3 ray_dir(const Cam& c, int p)
{
    const int i = p / c.W, j = p - i * c.W;
    const float x = (((float)j + 0.5f) / (float)c.W * 2.f - 1.f) * c.tx;
    const float y = (1.f - ((float)i + 0.5f) / (float)c.H * 2.f) * c.ty;
    float3 d = f3(c.f.x + x * c.r.x + y * c.u.x, c.f.y + x * c.r.y + y * c.u.y, c.f.z + x * c.r.z + y * c.u.z);
    const float inv = rsqrtf(dot(d, d));
    return scale(d, inv);
}

// rays in 8 x 4 pixel tiles, row-major tiles; slots outside the image get -1
__global__ void k_trace_init(Cam c, int nslots, int* __restrict__ act, float* __restrict__ tval,
                             float* __restrict__ depth, int* __restrict__ steps, float3* __restrict__ dirs)
{
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nslots) return;
    const int tpr = (c.W + 7) / 8;
    const int T = l >> 5, w = l & 31;
    const int px = (T % tpr) * 8 + (w & 7), py = (T / tpr) * 4 + (w >> 3);
    const bool ok = px < c.W && py < c.H;
    const int p = py * c.W + px;
    act[l] = ok ? p : -1;
    if (ok) {
        tval[p] = 0.f;
        depth[p] = INFINITY;
        if (steps) steps[p] = 0;
        dirs[p] = ray_dir(c, p);
    }
}

__global__ void k_trace_points(Cam c, const int* __restrict__ act, int n, const float* __restrict__ tval,
                               const float3* __restrict__ dirs, float* __restrict__ q)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = act[i];
    float3 x = c.eye;
    if (p >= 0) {
        const float t = tval[p];
        const float3 d = dirs[p];
        x = f3(fmaf(t, d.x, c.eye.x), fmaf(t, d.y, c.eye.y), fmaf(t, d.z, c.eye.z));
    }
    q[3 * i] = x.x;
    q[3 * i + 1] = x.y;
    q[3 * i + 2] = x.z;
}

// advance or retire each marching ray; key 0 = keeps marching
__global__ void k_trace_step(const int* __restrict__ act, int n, const float* __restrict__ v, float eps, float t_max,
                             int last, int k, float* __restrict__ tval, float* __restrict__ depth,
                             int* __restrict__ steps, unsigned* __restrict__ key, int* __restrict__ live)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = act[i];
    unsigned keep = 0u;
    if (p >= 0) {
        if (steps) steps[p] = k + 1;
        const float d = v[i];
        const float t = tval[p];
        if (d < eps) {
            depth[p] = t;
        } else {
            const float tn = t + d;
            tval[p] = tn;
            keep = (tn <= t_max && !last) ? 1u : 0u;
        }
    }
    key[i] = keep ? 0u : 1u;
    if (keep) atomicAdd(live, 1);
}

}  // namespace

extern "C" int sd_sphere_trace(const sd_tree* t, const sd_trace_opts* o, float* depth, int32_t* steps,
                               int64_t* evaluations, void* stream)
{
    if (!t || !o || !depth || o->width <= 0 || o->height <= 0 || !(o->eps > 0.f) || !(o->t_max > 0.f) ||
        o->max_steps <= 0 || !(o->fov_y > 0.f && o->fov_y < 3.1f))
        return SD_ERR_INVALID_ARG;
    if ((int64_t)o->width * o->height >= ((int64_t)1 << 28)) return SD_ERR_TOO_LARGE;
    if (o->block < 0 || o->block > 256 || (o->block % 32) != 0) return SD_ERR_INVALID_ARG;
    // camera basis in double, as the definition states it
    double e[3], f[3], up[3], r[3], u[3];
    for (int j = 0; j < 3; ++j) { e[j] = o->eye[j]; f[j] = (double)o->target[j] - o->eye[j]; up[j] = o->up[j]; }
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0.0)) return SD_ERR_INVALID_ARG;
    for (int j = 0; j < 3; ++j) f[j] /= fl;
    r[0] = f[1] * up[2] - f[2] * up[1]; r[1] = f[2] * up[0] - f[0] * up[2]; r[2] = f[0] * up[1] - f[1] * up[0];
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rl > 0.0)) return SD_ERR_INVALID_ARG;      // up parallel to the view direction
    for (int j = 0; j < 3; ++j) r[j] /= rl;
    u[0] = r[1] * f[2] - r[2] * f[1]; u[1] = r[2] * f[0] - r[0] * f[2]; u[2] = r[0] * f[1] - r[1] * f[0];
    Cam c;
    c.eye = make_float3((float)e[0], (float)e[1], (float)e[2]);
    c.f = make_float3((float)f[0], (float)f[1], (float)f[2]);
    c.r = make_float3((float)r[0], (float)r[1], (float)r[2]);
    c.u = make_float3((float)u[0], (float)u[1], (float)u[2]);
    const double th = std::tan(0.5 * (double)o->fov_y);
    c.W = o->width;
    c.H = o->height;
    c.tx = (float)(th * c.W / c.H);
    c.ty = (float)th;
    SdUse use_{t, (cudaStream_t)stream};
    cudaStream_t st = (cudaStream_t)stream;
    const int P = c.W * c.H;
    const int nslots = ((c.W + 7) / 8) * ((c.H + 3) / 4) * 32;
    // scratch
    size_t off = 0;
    auto carve = [&](size_t b) { size_t o2 = off; off += (b + 255) & ~(size_t)255; return o2; };
    size_t o_act0 = carve(sizeof(int) * nslots), o_act1 = carve(sizeof(int) * nslots);
    size_t o_k0 = carve(sizeof(unsigned) * nslots), o_k1 = carve(sizeof(unsigned) * nslots);
    size_t o_t = carve(sizeof(float) * P), o_dir = carve(sizeof(float3) * P);
    size_t o_q = carve(sizeof(float) * 3 * nslots), o_v = carve(sizeof(float) * nslots);
    size_t o_hist = carve(sizeof(uint32_t) * sdsort::hist_words(nslots, 1));
    size_t o_cnt = carve(sizeof(int) * 64);
    void* tmp = nullptr;
    cudaError_t ce = cudaMallocAsync(&tmp, off, st);
    if (ce != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    char* b = (char*)tmp;
    int* act = (int*)(b + o_act0);
    int* act1 = (int*)(b + o_act1);
    unsigned* k0 = (unsigned*)(b + o_k0);
    unsigned* k1 = (unsigned*)(b + o_k1);
    float* tval = (float*)(b + o_t);
    float3* dirs = (float3*)(b + o_dir);
    float* q = (float*)(b + o_q);
    float* v = (float*)(b + o_v);
    uint32_t* hist = (uint32_t*)(b + o_hist);
    int* cnt = (int*)(b + o_cnt);      // [0] rays still marching, [1] packet counter
    int nl = 1;
    k_trace_init<<<(nslots + 255) / 256, 256, 0, st>>>(c, nslots, act, tval, depth, steps, dirs);
    int n = nslots;
    int64_t evals = 0;
    int rc = SD_OK;
    for (int k = 0; k < o->max_steps && n > 0; ++k) {
        k_trace_points<<<(n + 255) / 256, 256, 0, st>>>(c, act, n, tval, dirs, q);
        rc = sdint::traverse(t, q, n, nullptr, v, nullptr, o->block, cnt + 1, st);
        if (rc != SD_OK) break;
        cudaMemsetAsync(cnt, 0, sizeof(int), st);
        k_trace_step<<<(n + 255) / 256, 256, 0, st>>>(act, n, v, o->eps, o->t_max, k + 1 == o->max_steps, k, tval,
                                                       depth, steps, k0, cnt);
        nl += 2;
        evals += k == 0 ? P : n;     // the first wavefront also holds the padding slots
        int where = sdsort::sort_pairs<unsigned, int>(k0, act, k1, act1, n, 1, hist, st, &nl);
        if (where) std::swap(act, act1);
        int live = 0;
        ce = cudaMemcpyAsync(&live, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rc = sd_cuda_status(ce); break; }
        n = live;
    }
    sd_count_launches(nl);
    if (rc == SD_OK) rc = sd_cuda_status(cudaGetLastError());
    cudaFreeAsync(tmp, st);
    if (evaluations) *evaluations = evals;
    return rc;
}
