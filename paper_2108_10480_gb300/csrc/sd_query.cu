// sd_query / sd_query_brute: Alg. 2 over Alg. 1 (Barnes-Hut), and the plain
// all-pairs evaluation of Eq. 3 / Eq. 4.
//
// Traversal: a warp walks the tree for 32 Morton-adjacent queries at once.
// Each popped record tests both children for every lane still interested in
// it (Barnes-Hut test first, also at leaves, as in Alg. 1): a far child adds
// n_B w_B e^{-alpha d_box} with gradient direction (q - y_B)/d_box (App. D),
// a near leaf adds its primitives' exact terms, a near internal child is
// pushed with the mask of lanes that need it. The LogSumExp is accumulated
// online in fp32 with a running max shift (no overflow or underflow for any
// alpha).
#include <cuda_runtime.h>

#include <algorithm>

#include "sd_common.cuh"
#include "sd_sort.cuh"

namespace {

// Warp-cooperative ("packet") traversal: the 32 lanes of a warp hold 32
// consecutive queries of the Morton order and walk the tree together on one
// warp-uniform stack of (record, lane mask) entries in shared memory. Every
// lane takes its own Barnes-Hut decisions (so each query gets exactly the
// terms of Alg. 1); a record is fetched once per warp and broadcast, a child
// is pushed if any lane needs it opened, and a leaf is evaluated by the lanes
// that reach it.
constexpr int PK_STACK = 128;     // > depth + 1 of any radix tree over 95-bit keys
constexpr int PK_MAX_THREADS = 256;

template <int KINDS, bool GRAD>
__device__ __forceinline__ void packet_child(const SdParams& P, float3 q, bool mine, float lx, float ly, float lz,
                                             float hx, float hy, float hz, int ref, float nw, Lse& acc,
                                             int2* st, int& sp, int lane, int& ntest, int& nfar, int& nleaf,
                                             bool& overflow)
{
    bool need = false, leaf = false;
    if (mine) {
        ++ntest;
        float dbox2;
        float3 off;
        if (bh_far(q, lx, ly, lz, hx, hy, hz, P.beta2, dbox2, off)) {
            // far field of App. D at the box's closest point y_B
            float rs = rsqrtf(dbox2);
            lse_add<GRAD>(acc, -P.alpha2 * (dbox2 * rs), nw, scale(off, rs));
            ++nfar;
        } else if (ref < 0) {
            leaf = true;
        } else {
            need = true;
        }
    }
    if (__ballot_sync(0xffffffffu, leaf)) {
        int k0 = (-ref - 1) * P.L;
        int k1 = min(k0 + P.L, P.n_prims);
        if (leaf) {
            for (int k = k0; k < k1; ++k) {
                float y, w;
                float3 v;
                leaf_term<KINDS, GRAD>(P, q, k, y, w, v);
                lse_add<GRAD>(acc, y, w, v);
            }
            nleaf += k1 - k0;
        }
    }
    unsigned pm = __ballot_sync(0xffffffffu, need);
    if (pm) {
        if (sp < PK_STACK) {
            if (lane == 0) st[sp] = make_int2(ref, (int)pm);
            ++sp;
        } else {
            overflow = true;
        }
    }
}

template <int KINDS, bool GRAD>
__global__ void __launch_bounds__(PK_MAX_THREADS) k_traverse(SdParams P, const float* __restrict__ qs, int M,
                                                             const int* __restrict__ order,
                                                             float* __restrict__ value, float* __restrict__ grad,
                                                             int* __restrict__ counts, int* __restrict__ status)
{
    extern __shared__ int2 stk[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int2* st = stk + wib * PK_STACK;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool inrange = t < M;
    int qi = inrange ? (order ? order[t] : t) : 0;
    float3 q = f3(0.f, 0.f, 0.f);
    if (inrange) q = f3(qs[3 * qi], qs[3 * qi + 1], qs[3 * qi + 2]);
    bool ok = inrange && isfinite(q.x) && isfinite(q.y) && isfinite(q.z);
    if (inrange && !ok) {
        atomicOr(status, 1 << SD_ERR_NONFINITE);
        value[qi] = __int_as_float(0x7fffffff);
        if (grad) grad[3 * qi] = grad[3 * qi + 1] = grad[3 * qi + 2] = __int_as_float(0x7fffffff);
        if (counts) counts[3 * qi] = counts[3 * qi + 1] = counts[3 * qi + 2] = 0;
    }
    unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (!mask) return;
    Lse acc;
    lse_init(acc);
    int ntest = 0, nfar = 0, nleaf = 0;
    bool overflow = false;
    int sp = 0;
    int rec = P.root_record;
    for (;;) {
        const SdNode& r = P.nodes[rec];
        float4 a = __ldg(&r.a), b = __ldg(&r.b), c = __ldg(&r.c);
        int4 d = __ldg(&r.d);
        bool mine = (mask >> lane) & 1u;
        packet_child<KINDS, GRAD>(P, q, mine, a.x, a.y, a.z, a.w, b.x, b.y, d.x, __int_as_float(d.z), acc, st, sp,
                                  lane, ntest, nfar, nleaf, overflow);
        if (d.y != SD_NO_CHILD)
            packet_child<KINDS, GRAD>(P, q, mine, b.z, b.w, c.x, c.y, c.z, c.w, d.y, __int_as_float(d.w), acc, st,
                                      sp, lane, ntest, nfar, nleaf, overflow);
        if (sp == 0) break;
        __syncwarp();
        int2 e = st[--sp];
        __syncwarp();
        rec = e.x;
        mask = (unsigned)e.y;
    }
    if (overflow && lane == 0) atomicOr(status, 1 << SD_ERR_TOO_LARGE);
    if (!ok) return;
    // Alg. 2: d^ = -log(c)/alpha, grad d^ = grad c / c (c >= 1 after the shift)
    value[qi] = -(acc.m + sd_lg2(acc.s)) * P.inv_alpha2;
    if (GRAD) {
        float is = 1.f / acc.s;
        grad[3 * qi] = acc.gx * is;
        grad[3 * qi + 1] = acc.gy * is;
        grad[3 * qi + 2] = acc.gz * is;
    }
    if (counts) {
        counts[3 * qi] = ntest;
        counts[3 * qi + 1] = nfar;
        counts[3 * qi + 2] = nleaf;
    }
}

// Plain method: every query against every primitive, primitives staged
// through shared memory in tiles.
constexpr int BT = 128;

template <int KINDS, bool GRAD>
__global__ void __launch_bounds__(BT) k_brute(SdParams P, const float* __restrict__ qs, int M,
                                              float* __restrict__ value, float* __restrict__ grad,
                                              int* __restrict__ status)
{
    __shared__ float4 sh[BT];
    __shared__ float4 sx[2 * BT];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool live = t < M;
    float3 q = live ? f3(qs[3 * t], qs[3 * t + 1], qs[3 * t + 2]) : f3(0.f, 0.f, 0.f);
    bool finite = isfinite(q.x) && isfinite(q.y) && isfinite(q.z);
    if (live && !finite) atomicOr(status, 1 << SD_ERR_NONFINITE);
    Lse acc;
    lse_init(acc);
    const bool has_ext = KINDS != SD_HAS_PTS;
    for (int k0 = 0; k0 < P.n_prims; k0 += BT) {
        int kk = k0 + threadIdx.x;
        __syncthreads();
        if (kk < P.n_prims) {
            sh[threadIdx.x] = P.hdr[kk];
            if (has_ext) {
                sx[2 * threadIdx.x] = P.ext[2 * kk];
                sx[2 * threadIdx.x + 1] = P.ext[2 * kk + 1];
            }
        }
        __syncthreads();
        int cnt = min(BT, P.n_prims - k0);
        if (!live || !finite) continue;
        for (int j = 0; j < cnt; ++j) {
            float4 h = sh[j];
            float y, w;
            float3 v;
            int kind = KINDS == SD_HAS_PTS ? SD_KIND_POINT : KINDS == SD_HAS_SEGS ? SD_KIND_SEG
                     : KINDS == SD_HAS_TRIS ? SD_KIND_TRI : (int)h.w;
            if (kind == SD_KIND_POINT) leaf_point(P, q, h, y, w, v);
            else if ((KINDS & SD_HAS_SEGS) && kind == SD_KIND_SEG) leaf_segment<GRAD>(P, q, h, sx[2 * j], sx[2 * j + 1], y, w, v);
            else leaf_triangle<GRAD>(P, q, h, sx[2 * j], sx[2 * j + 1], y, w, v);
            lse_add<GRAD>(acc, y, w, v);
        }
    }
    if (!live) return;
    if (!finite) {
        value[t] = __int_as_float(0x7fffffff);
        if (GRAD) grad[3 * t] = grad[3 * t + 1] = grad[3 * t + 2] = __int_as_float(0x7fffffff);
        return;
    }
    value[t] = -(acc.m + sd_lg2(acc.s)) * P.inv_alpha2;
    if (GRAD) {
        float is = 1.f / acc.s;
        grad[3 * t] = acc.gx * is;
        grad[3 * t + 1] = acc.gy * is;
        grad[3 * t + 2] = acc.gz * is;
    }
}

__global__ void k_fill_empty(float* value, float* grad, int M)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    value[t] = INFINITY;
    if (grad) grad[3 * t] = grad[3 * t + 1] = grad[3 * t + 2] = 0.f;
}

// 30-bit Morton code of each query relative to the scene box (clamped), the
// traversal order
__global__ void k_query_codes(const float* __restrict__ qs, int M, float3 lo, float3 inv_ext,
                              unsigned* __restrict__ keys, int* __restrict__ vals)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    float c[3] = {qs[3 * t], qs[3 * t + 1], qs[3 * t + 2]};
    float l[3] = {lo.x, lo.y, lo.z}, ie[3] = {inv_ext.x, inv_ext.y, inv_ext.z};
    unsigned k[3];
    for (int j = 0; j < 3; ++j) {
        float u = (c[j] - l[j]) * ie[j];
        u = fminf(fmaxf(u, 0.f), 1.f);          // NaN -> 0
        k[j] = min((unsigned)(u * 1024.f), 1023u);
    }
    unsigned code = 0;
    for (int b = 9; b >= 0; --b)
        code = (code << 3) | (((k[0] >> b) & 1u) << 2) | (((k[1] >> b) & 1u) << 1) | ((k[2] >> b) & 1u);
    keys[t] = code;
    vals[t] = t;
}

template <bool BRUTE, int KINDS, bool GRAD>
void launch_one(const sd_tree* t, const float* q, int M, const int* order, float* value, float* grad, int* counts,
                int block, cudaStream_t st)
{
    if (BRUTE) {
        k_brute<KINDS, GRAD><<<(M + BT - 1) / BT, BT, 0, st>>>(t->P, q, M, value, grad, t->status);
    } else {
        int B = block > 0 ? block : 128;
        size_t smem = sizeof(int2) * PK_STACK * (B / 32);
        k_traverse<KINDS, GRAD><<<(M + B - 1) / B, B, smem, st>>>(t->P, q, M, order, value, grad, counts, t->status);
    }
}

template <bool BRUTE>
void dispatch(const sd_tree* t, const float* q, int M, const int* order, float* value, float* grad, int* counts,
              int block, cudaStream_t st)
{
    bool g = grad != nullptr;
    switch (t->kinds) {
    case SD_HAS_PTS:
        g ? launch_one<BRUTE, SD_HAS_PTS, true>(t, q, M, order, value, grad, counts, block, st)
          : launch_one<BRUTE, SD_HAS_PTS, false>(t, q, M, order, value, grad, counts, block, st);
        break;
    case SD_HAS_SEGS:
        g ? launch_one<BRUTE, SD_HAS_SEGS, true>(t, q, M, order, value, grad, counts, block, st)
          : launch_one<BRUTE, SD_HAS_SEGS, false>(t, q, M, order, value, grad, counts, block, st);
        break;
    case SD_HAS_TRIS:
        g ? launch_one<BRUTE, SD_HAS_TRIS, true>(t, q, M, order, value, grad, counts, block, st)
          : launch_one<BRUTE, SD_HAS_TRIS, false>(t, q, M, order, value, grad, counts, block, st);
        break;
    default:
        g ? launch_one<BRUTE, 7, true>(t, q, M, order, value, grad, counts, block, st)
          : launch_one<BRUTE, 7, false>(t, q, M, order, value, grad, counts, block, st);
        break;
    }
}

int check_query_args(const sd_tree* t, const float* q, int64_t M, const float* value)
{
    if (!t || M < 0) return SD_ERR_INVALID_ARG;
    if (M > 0 && (!q || !value)) return SD_ERR_INVALID_ARG;
    if (M >= ((int64_t)1 << 31) / 3) return SD_ERR_TOO_LARGE;
    return SD_OK;
}

}  // namespace

namespace {

// Morton order of the queries into `order` (stream-ordered scratch).
int compute_order(const sd_tree* t, const float* q, int m, int32_t* order, cudaStream_t st)
{
    size_t hw = sdsort::hist_words(m);
    size_t bytes = sizeof(unsigned) * 2 * (size_t)m + sizeof(int) * (size_t)m + sizeof(uint32_t) * hw + 1024;
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, bytes, st);
    if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    unsigned* k0 = (unsigned*)tmp;
    unsigned* k1 = k0 + m;
    int* v1 = (int*)(k1 + m);
    uint32_t* hist = (uint32_t*)(v1 + m);
    const sd_tree_info& I = t->info;
    float3 lo = make_float3(I.scene_lo[0], I.scene_lo[1], I.scene_lo[2]);
    float ex[3];
    for (int j = 0; j < 3; ++j) ex[j] = I.scene_hi[j] - I.scene_lo[j];
    float3 ie = make_float3(ex[0] > 0 ? 1.f / ex[0] : 0.f, ex[1] > 0 ? 1.f / ex[1] : 0.f, ex[2] > 0 ? 1.f / ex[2] : 0.f);
    int nl = 1;
    k_query_codes<<<(m + 255) / 256, 256, 0, st>>>(q, m, lo, ie, k0, order);
    int where = sdsort::sort_pairs<unsigned, int>(k0, order, k1, v1, m, 30, hist, st, &nl);
    if (where) cudaMemcpyAsync(order, v1, sizeof(int) * (size_t)m, cudaMemcpyDeviceToDevice, st);
    sd_count_launches(nl);
    e = cudaGetLastError();
    cudaFreeAsync(tmp, st);
    return sd_cuda_status(e);
}

}  // namespace

extern "C" int sd_query_order(const sd_tree* t, const float* q, int64_t M, int32_t* order, void* stream)
{
    int rc = check_query_args(t, q, M, order ? (const float*)order : nullptr);
    if (rc != SD_OK) return rc;
    if (M == 0) return SD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int m = (int)M;
    if (m == 1) {
        int zero = 0;
        return sd_cuda_status(cudaMemcpyAsync(order, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    }
    return compute_order(t, q, m, order, st);
}

extern "C" int sd_query(const sd_tree* t, const float* q, int64_t M, float* value, float* grad,
                        const sd_query_opts* opts_in, void* stream)
{
    int rc = check_query_args(t, q, M, value);
    if (rc != SD_OK) return rc;
    sd_query_opts opts;
    if (opts_in) opts = *opts_in; else sd_default_query_opts(&opts);
    if (opts.block < 0 || opts.block > PK_MAX_THREADS || (opts.block % 32) != 0) return SD_ERR_INVALID_ARG;
    if (M == 0) return SD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int m = (int)M;
    if (t->info.n_prims == 0) {
        k_fill_empty<<<(m + 255) / 256, 256, 0, st>>>(value, grad, m);
        sd_count_launches(1);
        if (opts.counts) cudaMemsetAsync(opts.counts, 0, sizeof(int) * 3 * (size_t)m, st);
        return sd_cuda_status(cudaGetLastError());
    }
    const int* order = opts.order;
    void* tmp = nullptr;
    if (!order && opts.sort_queries && m > 1) {
        cudaError_t e = cudaMallocAsync(&tmp, sizeof(int) * (size_t)m, st);
        if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
        rc = compute_order(t, q, m, (int32_t*)tmp, st);
        if (rc != SD_OK) { cudaFreeAsync(tmp, st); return rc; }
        order = (const int*)tmp;
    }
    dispatch<false>(t, q, m, order, value, grad, opts.counts, opts.block, st);
    sd_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (tmp) cudaFreeAsync(tmp, st);
    return sd_cuda_status(e);
}

extern "C" int sd_query_brute(const sd_tree* t, const float* q, int64_t M, float* value, float* grad,
                              const sd_query_opts* opts, void* stream)
{
    (void)opts;
    int rc = check_query_args(t, q, M, value);
    if (rc != SD_OK) return rc;
    if (M == 0) return SD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int m = (int)M;
    if (t->info.n_prims == 0) {
        k_fill_empty<<<(m + 255) / 256, 256, 0, st>>>(value, grad, m);
        sd_count_launches(1);
        return sd_cuda_status(cudaGetLastError());
    }
    dispatch<true>(t, q, m, nullptr, value, grad, nullptr, 0, st);
    sd_count_launches(1);
    return sd_cuda_status(cudaGetLastError());
}

extern "C" int sd_query_status(const sd_tree* t, void* stream)
{
    if (!t) return SD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, t->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return sd_cuda_status(e);
    if (h) {
        cudaMemsetAsync(t->status, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        for (int c = 1; c < 31; ++c)
            if (h & (1 << c)) return c;
    }
    return SD_OK;
}
