// sd_build: the acceleration structure of Alg. 1 (Sec. 3.5, App. D) built on
// the GPU, plus the per-primitive weight parameters of App. C.
//
// Stream order of one build:
//   validate -> scene box -> incidence counts / weight parameters ->
//   Morton codes -> radix sort by (code, index) -> radix tree (Karras) ->
//   bottom-up AABBs, counts and far-field masses -> leaf-order gather.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstring>
#include <vector>

#include "sd_common.cuh"
#include "sd_sort.cuh"
#include "sd_wtab.h"

namespace {

enum { ST_NONFINITE = 1, ST_INDEX = 2 };

// scalars the build accumulates on the device
struct BuildScalars {
    unsigned box[6];   // scene box as order-preserving unsigned keys: lo.xyz (min), hi.xyz (max)
    int status;
    int A_E, A_T;
    int pad;
};

__device__ __forceinline__ unsigned f2key(float f)
{
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __host__ __forceinline__ float key2f(unsigned k)
{
    unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}

struct Geo {
    const float* P; int np;
    const float* EV; int nev; const int* E; int ne;
    const float* TV; int ntv; const int* F; int nf;
    int n;
};

__device__ __forceinline__ int clampi(int v, int n) { return min(max(v, 0), n - 1); }

// vertex j (0..2) of primitive i, as fp32 xyz. Indices are clamped into
// range: an out-of-range index is reported by the validation kernels and the
// build is discarded, but no kernel ever reads outside the inputs.
__device__ __forceinline__ float3 prim_vertex(const Geo& g, int i, int j)
{
    const float* p;
    if (i < g.np) p = g.P + 3 * i;
    else if (i < g.np + g.ne) p = g.EV + 3 * clampi(g.E[2 * (i - g.np) + j], g.nev);
    else p = g.TV + 3 * clampi(g.F[3 * (i - g.np - g.ne) + j], g.ntv);
    return make_float3(p[0], p[1], p[2]);
}
__device__ __forceinline__ int prim_nv(const Geo& g, int i) { return i < g.np ? 1 : (i < g.np + g.ne ? 2 : 3); }

// --- validation and scene box --------------------------------------------
__device__ __forceinline__ void check_vertices(const float* __restrict__ x, int nv, BuildScalars* bs)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
        for (int j = 0; j < 3; ++j) {
            float v = x[3 * i + j];
            bad |= !isfinite(v);
            lo[j] = fminf(lo[j], v);
            hi[j] = fmaxf(hi[j], v);
        }
    }
    if (bad) atomicOr(&bs->status, ST_NONFINITE);
    for (int j = 0; j < 3; ++j) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[j] = fminf(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], o));
            hi[j] = fmaxf(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int j = 0; j < 3; ++j) {
            if (lo[j] <= hi[j]) {
                atomicMin(&bs->box[j], f2key(lo[j]));
                atomicMax(&bs->box[3 + j], f2key(hi[j]));
            }
        }
    }
}

__device__ __forceinline__ void check_index(const int* __restrict__ idx, int64_t count, int nv, BuildScalars* bs)
{
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        int v = idx[i];
        bad |= v < 0 || v >= nv;
    }
    if (bad) atomicOr(&bs->status, ST_INDEX);
}

// every input check in one launch: blockIdx.y picks the array (points,
// edge-mesh vertices, triangle-mesh vertices, edge indices, triangle indices)
__global__ void k_validate(Geo g, BuildScalars* bs)
{
    sdsort::pdl_wait_and_release();     // (launched as k_init's dependent)
    switch (blockIdx.y) {
    case 0: check_vertices(g.P, g.np, bs); break;
    case 1: check_vertices(g.EV, g.nev, bs); break;
    case 2: check_vertices(g.TV, g.ntv, bs); break;
    case 3: check_index(g.E, 2 * (int64_t)g.ne, g.nev, bs); break;
    default: check_index(g.F, 3 * (int64_t)g.nf, g.ntv, bs); break;
    }
}

// zero / fill the build's working arrays and its scalars in one launch
struct InitJob {
    BuildScalars* bs;
    int* status;
    float* params; int nparams;
    int4* nodes; int nnodes4;
    int* ecnt; int nev;
    int* vcnt; int ntv;
    int* hcnt; unsigned long long* hkeys; int hcap;
    uint32_t* hist; int nhist;          // the primitive sort's scratch words
};

__global__ void k_init(InitJob J)
{
    sdsort::pdl_release();      // k_validate may launch
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    if (t0 == 0) {
        BuildScalars b;
        for (int j = 0; j < 3; ++j) { b.box[j] = 0xffffffffu; b.box[3 + j] = 0u; }
        b.status = 0;
        b.A_E = 1; b.A_T = 1;
        b.pad = 0;
        *J.bs = b;
        for (int j = 0; j < 4; ++j) J.status[j] = 0;
    }
    for (int i = t0; i < J.nparams; i += st) J.params[i] = 0.f;
    for (int i = t0; i < J.nnodes4; i += st) J.nodes[i] = make_int4(0, 0, 0, 0);
    for (int i = t0; i < J.nhist; i += st) J.hist[i] = 0u;
    for (int i = t0; i < J.nev; i += st) J.ecnt[i] = 0;
    for (int i = t0; i < J.ntv; i += st) J.vcnt[i] = 0;
    for (int i = t0; i < J.hcap; i += st) { J.hcnt[i] = 0; J.hkeys[i] = ~0ull; }
}

// --- incidence counts (App. C.2, C.3): one count per incidence slot -------
__global__ void k_count_slots(const int* __restrict__ idx, int64_t count, int nv, int* __restrict__ cnt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        int v = idx[i];
        if (v >= 0 && v < nv) atomicAdd(&cnt[v], 1);
    }
}

__device__ __forceinline__ unsigned long long edge_key(int a, int b)
{
    unsigned lo = (unsigned)min(a, b), hi = (unsigned)max(a, b);
    return ((unsigned long long)lo << 32) | hi;
}
__device__ __forceinline__ unsigned hash64(unsigned long long k, unsigned mask)
{
    k ^= k >> 33; k *= 0xff51afd7ed558ccdull; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull; k ^= k >> 33;
    return (unsigned)k & mask;
}

// open-addressing table: key per slot, count per slot; probing is bounded by
// the capacity (load factor <= 1/2, so a slot is always found)
__global__ void k_edge_insert(const int* __restrict__ F, int nf, unsigned long long* keys, int* counts, unsigned mask)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= 3 * nf) return;
    int t = s / 3, j = s - 3 * t;
    unsigned long long k = edge_key(F[3 * t + j], F[3 * t + (j + 1) % 3]);
    unsigned h = hash64(k, mask);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        unsigned long long prev = atomicCAS(&keys[h], ~0ull, k);
        if (prev == ~0ull || prev == k) { atomicAdd(&counts[h], 1); return; }
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ int edge_lookup(const unsigned long long* keys, const int* counts, unsigned mask,
                                           unsigned long long k)
{
    unsigned h = hash64(k, mask);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        unsigned long long v = keys[h];
        if (v == k) return counts[h];
        if (v == ~0ull) return 0;
        h = (h + 1) & mask;
    }
    return 0;
}

// triangle i: v_i = max vertex valence, e_i = max edge valence -> (1/v_i, 1/e_i)
__global__ void k_tri_params(const int* __restrict__ F, int nf, int ntv, const int* __restrict__ vcnt,
                             const unsigned long long* keys, const int* counts, unsigned mask,
                             float* __restrict__ params, int first, BuildScalars* bs)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf) return;
    int a = clampi(F[3 * t], ntv), b = clampi(F[3 * t + 1], ntv), c = clampi(F[3 * t + 2], ntv);
    int vm = max(max(vcnt[a], max(vcnt[b], vcnt[c])), 1);
    int em = max(edge_lookup(keys, counts, mask, edge_key(a, b)),
                 max(edge_lookup(keys, counts, mask, edge_key(b, c)), edge_lookup(keys, counts, mask, edge_key(c, a))));
    params[2 * (first + t)] = 1.f / (float)vm;
    params[2 * (first + t) + 1] = 1.f / (float)max(em, 1);
    atomicMax(&bs->A_T, vm);
}

// edge i: (u, v) = (1/|N_i0|, 1/|N_i1|)
__global__ void k_edge_params(const int* __restrict__ E, int ne, int nev, const int* __restrict__ cnt,
                              float* __restrict__ params, int first, BuildScalars* bs)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    int c0 = max(cnt[clampi(E[2 * e], nev)], 1), c1 = max(cnt[clampi(E[2 * e + 1], nev)], 1);
    params[2 * (first + e)] = 1.f / (float)c0;
    params[2 * (first + e) + 1] = 1.f / (float)c1;
    atomicMax(&bs->A_E, max(c0, c1));
}

// --- Morton codes (fp32 centroid in a fixed operation order) ---------------
// the Morton code of primitive i (written to codes, keys and its index to vals)
__device__ __forceinline__ unsigned long long morton_code(const Geo& g, const BuildScalars* bs, int i,
                                                          unsigned long long* codes, unsigned long long* keys,
                                                          int* vals)
{
    float lo[3], hi[3];
    for (int j = 0; j < 3; ++j) { lo[j] = key2f(bs->box[j]); hi[j] = key2f(bs->box[3 + j]); }
    int nvx = prim_nv(g, i);
    float3 a = prim_vertex(g, i, 0);
    float c[3] = {a.x, a.y, a.z};
    if (nvx == 2) {
        float3 b = prim_vertex(g, i, 1);
        c[0] = __fmul_rn(__fadd_rn(a.x, b.x), 0.5f);
        c[1] = __fmul_rn(__fadd_rn(a.y, b.y), 0.5f);
        c[2] = __fmul_rn(__fadd_rn(a.z, b.z), 0.5f);
    } else if (nvx == 3) {
        float3 b = prim_vertex(g, i, 1), d = prim_vertex(g, i, 2);
        const float third = 1.0f / 3.0f;
        c[0] = __fmul_rn(__fadd_rn(__fadd_rn(a.x, b.x), d.x), third);
        c[1] = __fmul_rn(__fadd_rn(__fadd_rn(a.y, b.y), d.y), third);
        c[2] = __fmul_rn(__fadd_rn(__fadd_rn(a.z, b.z), d.z), third);
    }
    unsigned k[3];
    for (int j = 0; j < 3; ++j) {
        float ext = __fsub_rn(hi[j], lo[j]);
        float u = 0.f;
        if (ext > 0.f) u = __fdiv_rn(__fsub_rn(c[j], lo[j]), ext);
        u = fminf(fmaxf(u, 0.f), 1.f);
        unsigned v = (unsigned)floorf(__fmul_rn(u, 2097152.0f));
        k[j] = min(v, 2097151u);
    }
    unsigned long long code = 0;
    for (int b = 20; b >= 0; --b) {
        code = (code << 1) | ((k[0] >> b) & 1u);
        code = (code << 1) | ((k[1] >> b) & 1u);
        code = (code << 1) | ((k[2] >> b) & 1u);
    }
    codes[i] = code;
    keys[i] = code;
    vals[i] = i;
    return code;
}

// (blocks of 256 threads over a grid-stride loop; each block also adds its
// codes' radix digits of all eight passes to the sort's digit totals, once
// per block, so that few blocks contend for the totals' words)
__global__ void __launch_bounds__(256) k_morton(Geo g, const BuildScalars* bs, unsigned long long* __restrict__ codes,
                                                unsigned long long* __restrict__ keys, int* __restrict__ vals,
                                                uint32_t* __restrict__ totals)
{
    __shared__ uint32_t h[8][256];
    sdsort::pdl_release();      // the sort's first pass may launch
    for (int p = 0; p < 8; ++p) h[p][threadIdx.x] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x)
        sdsort::count_key(h, morton_code(g, bs, i, codes, keys, vals), 8);
    __syncthreads();
    for (int p = 0; p < 8; ++p) {
        const uint32_t c = h[p][threadIdx.x];
        if (c) atomicAdd(&totals[256 * p + threadIdx.x], c);
    }
}

// --- binary radix tree over buckets (Karras 2012) --------------------------
__device__ __forceinline__ int bucket_prefix(const unsigned long long* sk, const int* sv, int L, int nb, int i, int j)
{
    if (j < 0 || j >= nb) return -1;
    unsigned long long a = sk[(size_t)i * L], b = sk[(size_t)j * L];
    if (a != b) return __clzll(a ^ b);
    return 64 + __clz(sv[(size_t)i * L] ^ sv[(size_t)j * L]);
}

// Record nb - 1 is the super-root: one child (the root, or leaf 0 when the
// tree is a single bucket) in slot 0; slot 1 is empty and never tested.
__device__ __forceinline__ void super_root_record(SdNode* nodes, float2* lw2, int nb)
{
    SdNode& r = nodes[nb - 1];
    r.d.x = nb > 1 ? 0 : -1;
    r.d.y = SD_NO_CHILD;
    float* f = reinterpret_cast<float*>(&r);
    for (int j = 1; j < 12; j += 2) f[j] = 0.f;
    f[15] = 0.f;
    lw2[nb - 1].y = 0.f;
}

// the tree's scalars from the build's atomics (one thread): the weight
// scales, and the validation bits folded into the tree's status word
__device__ __forceinline__ void finalize_scalars(const BuildScalars* bs, int unit, SdScalars* sc, int* status)
{
    sc->A_E = unit ? 1.f : (float)bs->A_E;
    sc->A_T = unit ? 1.f : (float)bs->A_T;
    sc->status = bs->status;
    if (bs->status & ST_INDEX) atomicOr(status, 1 << SD_ERR_INDEX);
    if (bs->status & ST_NONFINITE) atomicOr(status, 1 << SD_ERR_NONFINITE);
}

__device__ __forceinline__ void karras_node(int i, const unsigned long long* __restrict__ sk,
                                            const int* __restrict__ sv, int L, int nb, int* __restrict__ left,
                                            int* __restrict__ right, int* __restrict__ parent_int,
                                            int2* __restrict__ range, SdNode* __restrict__ nodes,
                                            float2* __restrict__ lw2)
{
    if (i >= nb - 1) return;
    int d = bucket_prefix(sk, sv, L, nb, i, i + 1) - bucket_prefix(sk, sv, L, nb, i, i - 1) > 0 ? 1 : -1;
    int dmin = bucket_prefix(sk, sv, L, nb, i, i - d);
    int lmax = 2;
    while (bucket_prefix(sk, sv, L, nb, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (bucket_prefix(sk, sv, L, nb, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = bucket_prefix(sk, sv, L, nb, i, j);
    int s = 0;
    int t = (l + 1) >> 1;
    for (;;) {
        if (bucket_prefix(sk, sv, L, nb, i, i + (s + t) * d) > dnode) s += t;
        if (t == 1) break;
        t = (t + 1) >> 1;
    }
    int gamma = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    int lref = (lo == gamma) ? -(gamma + 1) : gamma;
    int rref = (hi == gamma + 1) ? -(gamma + 2) : gamma + 1;
    left[i] = lref;
    right[i] = rref;
    range[i] = make_int2(lo, hi);
    if (i == 0) super_root_record(nodes, lw2, nb);
    if (lref >= 0) parent_int[gamma] = i;
    if (rref >= 0) parent_int[gamma + 1] = i;
    nodes[i].d.x = lref;
    nodes[i].d.y = rref;
    if (i == 0) parent_int[0] = -1;
}

// write child slot `slot` of record `rec` (interleaved AABB with negated upper
// corner, squared diagonal) and log2 of the child's far-field mass
__device__ __forceinline__ void write_slot(SdNode* nodes, float2* lw2, int rec, int slot, const float* lo,
                                           const float* hi, float nw)
{
    float* r = reinterpret_cast<float*>(&nodes[rec]);
    r[0 + slot] = lo[0];
    r[2 + slot] = lo[1];
    r[4 + slot] = lo[2];
    r[6 + slot] = -hi[0];
    r[8 + slot] = -hi[1];
    r[10 + slot] = -hi[2];
    r[14 + slot] = box_diag2(lo, hi);
    float* w = reinterpret_cast<float*>(&lw2[rec]);
    w[slot] = log2f(nw);
}

// Aggregates without a bottom-up climb. Every node of the radix tree covers a
// contiguous range of buckets, so its AABB (an exact fp32 min/max, the same
// in any order of reduction), its primitive count and whether it holds only
// points are reductions over that range. The bucket blocks of k_after_sort
// compute every bucket's own aggregates and, in each block of 1,024
// buckets, the unions over every aligned run of 2^k buckets (k = 0..10);
// k_nodes then assembles each
// internal node from at most 2 x 10 aligned runs plus whole runs of 1,024,
// loaded independently of one another. A run entry is two float4:
// (lo.x, lo.y, lo.z, 1 if points only else 0) and (hi.x, hi.y, hi.z, 0).
constexpr int AGG_T = 1024;
constexpr int AGG_LEVELS = 11;

// first entry of level k of the run table (levels 0..k-1 before it)
__host__ __device__ __forceinline__ int64_t run_level_offset(int nb, int k)
{
    int64_t off = 0;
    for (int j = 0; j < k; ++j) off += (nb + (1 << j) - 1) >> j;
    return off;
}

__device__ __forceinline__ float far_weight(const BuildScalars* bs, float S, int unit)
{
    if (unit) return 1.f;
    float A = (float)max(max(bs->A_E, bs->A_T), 1);
    return (S == 1.f) ? A : powf(A, S);
}

// (called by every thread of a block of AGG_T threads; blk = the block's
// index among the bucket blocks)
__device__ __forceinline__ void leaves_block(int blk, const Geo& g, const int* __restrict__ sorted, int L, int nb,
                                             float* __restrict__ leaf_box, int* __restrict__ leaf_count,
                                             float4* __restrict__ runs, SdNode* nodes, float2* lw2,
                                             const BuildScalars* bs, float S, int unit)
{
    __shared__ float s_lo[3][AGG_T], s_hi[3][AGG_T];
    __shared__ int s_pts[AGG_T];
    const int t = threadIdx.x;
    const int b = blk * AGG_T + t;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int pts = 1;
    if (b < nb) {
        const int k0 = b * L, k1 = min(k0 + L, g.n);
        for (int k = k0; k < k1; ++k) {
            const int p = sorted[k];
            const int nvx = prim_nv(g, p);
            if (nvx > 1) pts = 0;
            for (int j = 0; j < nvx; ++j) {
                const float3 v = prim_vertex(g, p, j);
                lo[0] = fminf(lo[0], v.x); lo[1] = fminf(lo[1], v.y); lo[2] = fminf(lo[2], v.z);
                hi[0] = fmaxf(hi[0], v.x); hi[1] = fmaxf(hi[1], v.y); hi[2] = fmaxf(hi[2], v.z);
            }
        }
        for (int j = 0; j < 3; ++j) { leaf_box[6 * b + j] = lo[j]; leaf_box[6 * b + 3 + j] = hi[j]; }
        leaf_count[b] = k1 - k0;
        runs[2 * (int64_t)b] = make_float4(lo[0], lo[1], lo[2], (float)pts);
        runs[2 * (int64_t)b + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
        if (nb == 1) {
            // the only bucket is the root: the super-root's one child
            const float nw = pts ? (float)(k1 - k0) : __fmul_rn((float)(k1 - k0), far_weight(bs, S, unit));
            write_slot(nodes, lw2, nb - 1, 0, lo, hi, nw);
        }
    }
    for (int j = 0; j < 3; ++j) { s_lo[j][t] = lo[j]; s_hi[j][t] = hi[j]; }
    s_pts[t] = pts;
    for (int k = 1; k < AGG_LEVELS; ++k) {
        __syncthreads();
        if (t < (AGG_T >> k)) {
            const int i0 = t << k, i1 = i0 + (1 << (k - 1));
            float a[3], c[3];
            for (int j = 0; j < 3; ++j) {
                a[j] = fminf(s_lo[j][i0], s_lo[j][i1]);
                c[j] = fmaxf(s_hi[j][i0], s_hi[j][i1]);
                s_lo[j][i0] = a[j];
                s_hi[j][i0] = c[j];
            }
            const int f = s_pts[i0] & s_pts[i1];
            s_pts[i0] = f;
            const int64_t r = (int64_t)blk * (AGG_T >> k) + t;             // run index at level k
            if ((r << k) < nb) {
                const int64_t e = run_level_offset(nb, k) + r;
                runs[2 * e] = make_float4(a[0], a[1], a[2], (float)f);
                runs[2 * e + 1] = make_float4(c[0], c[1], c[2], 0.f);
            }
        }
    }
}

// one thread per internal node: its aggregates, its slot in its parent's
// record (the super-root's for the root) and the slots of its leaf children
__global__ void k_nodes(int nb, int L, int n, const int2* __restrict__ range, const int* __restrict__ left,
                        const int* __restrict__ right, const int* __restrict__ parent_int,
                        const float4* __restrict__ runs, float* __restrict__ node_box, int* __restrict__ node_count,
                        SdNode* nodes, float2* lw2, const BuildScalars* bs, float S, int unit, SdScalars* sc,
                        int* status)
{
    __shared__ int64_t s_off[AGG_LEVELS];
    sdsort::pdl_wait_and_release();     // (launched as k_after_sort's dependent)
    if (blockIdx.x == 0 && threadIdx.x == 0) finalize_scalars(bs, unit, sc, status);
    if (threadIdx.x < AGG_LEVELS) s_off[threadIdx.x] = run_level_offset(nb, threadIdx.x);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < nb - 1;
    if (!__any_sync(0xffffffffu, live)) return;     // (a warp-uniform exit)
    const int lane = threadIdx.x & 31;
    int a = 0, e = 0;       // buckets [a, e)
    if (live) {
        const int2 rg = __ldg(&range[i]);
        a = rg.x;
        e = rg.y + 1;
    }
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float pts = 1.f;
    // The whole runs of 1,024 buckets in [a, e), [g0, g1): for a node with
    // more than eight of them the warp loads them together, one node at a
    // time, and reduces them with shuffles.
    constexpr int TOP = AGG_LEVELS - 1;
    const int m0 = (a + (1 << TOP) - 1) >> TOP, m1 = e >> TOP;
    const bool wide = live && m1 - m0 > 8;
    for (unsigned wm = __ballot_sync(0xffffffffu, wide); wm; wm &= wm - 1) {
        const int src = __ffs(wm) - 1;
        const int r0 = __shfl_sync(0xffffffffu, m0, src), r1 = __shfl_sync(0xffffffffu, m1, src);
        float l0 = INFINITY, l1 = INFINITY, l2 = INFINITY, h0 = -INFINITY, h1 = -INFINITY, h2 = -INFINITY, f = 1.f;
        for (int r = r0 + lane; r < r1; r += 32) {
            const float4 A = __ldg(&runs[2 * (s_off[TOP] + r)]), B = __ldg(&runs[2 * (s_off[TOP] + r) + 1]);
            l0 = fminf(l0, A.x); l1 = fminf(l1, A.y); l2 = fminf(l2, A.z);
            h0 = fmaxf(h0, B.x); h1 = fmaxf(h1, B.y); h2 = fmaxf(h2, B.z);
            f = fminf(f, A.w);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            l0 = fminf(l0, __shfl_xor_sync(0xffffffffu, l0, o));
            l1 = fminf(l1, __shfl_xor_sync(0xffffffffu, l1, o));
            l2 = fminf(l2, __shfl_xor_sync(0xffffffffu, l2, o));
            h0 = fmaxf(h0, __shfl_xor_sync(0xffffffffu, h0, o));
            h1 = fmaxf(h1, __shfl_xor_sync(0xffffffffu, h1, o));
            h2 = fmaxf(h2, __shfl_xor_sync(0xffffffffu, h2, o));
            f = fminf(f, __shfl_xor_sync(0xffffffffu, f, o));
        }
        if (lane == src) {
            lo[0] = l0; lo[1] = l1; lo[2] = l2;
            hi[0] = h0; hi[1] = h1; hi[2] = h2;
            pts = f;
        }
    }
    if (!live) return;
    const float wfar = far_weight(bs, S, unit);
    const int g0 = wide ? m0 << TOP : e, g1 = wide ? m1 << TOP : e;
    int x = a;
    while (x < e) {
        // the next eight aligned runs in [x, e) outside [g0, g1), largest
        // first at each step
        int64_t ent[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            ent[q] = -1;
            if (x == g0) x = g1;
            if (x < e) {
                const int lim = x < g0 ? g0 : e;
                int k = x ? __ffs(x) - 1 : AGG_LEVELS - 1;
                k = min(min(k, AGG_LEVELS - 1), 31 - __clz(lim - x));
                ent[q] = s_off[k] + (x >> k);
                x += 1 << k;
            }
        }
        float4 A[8], B[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (ent[q] >= 0) {
                A[q] = __ldg(&runs[2 * ent[q]]);
                B[q] = __ldg(&runs[2 * ent[q] + 1]);
            } else {
                A[q] = make_float4(INFINITY, INFINITY, INFINITY, 1.f);
                B[q] = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            lo[0] = fminf(lo[0], A[q].x); lo[1] = fminf(lo[1], A[q].y); lo[2] = fminf(lo[2], A[q].z);
            hi[0] = fmaxf(hi[0], B[q].x); hi[1] = fmaxf(hi[1], B[q].y); hi[2] = fmaxf(hi[2], B[q].z);
            pts = fminf(pts, A[q].w);
        }
        if (x == g0) x = g1;
    }
    const int count = min((int64_t)e * L, (int64_t)n) - a * L;
    for (int j = 0; j < 3; ++j) { node_box[6 * i + j] = lo[j]; node_box[6 * i + 3 + j] = hi[j]; }
    node_count[i] = count;
    const float nw = pts != 0.f ? (float)count : __fmul_rn((float)count, wfar);
    const int p = __ldg(&parent_int[i]);
    if (p < 0) write_slot(nodes, lw2, nb - 1, 0, lo, hi, nw);
    else write_slot(nodes, lw2, p, __ldg(&left[p]) == i ? 0 : 1, lo, hi, nw);
    // leaf children
    const int ch[2] = {__ldg(&left[i]), __ldg(&right[i])};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (ch[c] >= 0) continue;
        const int lb = -ch[c] - 1;
        const float4 la = __ldg(&runs[2 * (int64_t)lb]), lh = __ldg(&runs[2 * (int64_t)lb + 1]);
        const float llo[3] = {la.x, la.y, la.z}, lhi[3] = {lh.x, lh.y, lh.z};
        const int lc = min((lb + 1) * L, n) - lb * L;
        const float lw = la.w != 0.f ? (float)lc : __fmul_rn((float)lc, wfar);
        write_slot(nodes, lw2, i, c, llo, lhi, lw);
    }
}

// the super-root's own fields when the tree is a single bucket (with two
// or more buckets the topology kernel writes them)
__global__ void k_super_root(SdNode* nodes, float2* lw2, int nb)
{
    super_root_record(nodes, lw2, nb);
}

// the scene box into the tree's scalars, as soon as validation has reduced
// it (the query order needs nothing else of the tree)
__global__ void k_box(const BuildScalars* bs, int n, SdScalars* sc)
{
    sdsort::pdl_wait_and_release();     // (launched as k_validate's dependent)
    if (threadIdx.x || blockIdx.x) return;
    for (int j = 0; j < 3; ++j) {
        float lo = n ? key2f(bs->box[j]) : 0.f, hi = n ? key2f(bs->box[3 + j]) : 0.f;
        float ex = hi - lo;
        sc->lo[j] = lo;
        sc->hi[j] = hi;
        sc->inv_ex[j] = ex > 0.f ? 1.f / ex : 0.f;
    }
}

// the tree's scalars when there are no internal nodes (k_nodes does this
// otherwise)
__global__ void k_finalize(const BuildScalars* bs, int unit, SdScalars* sc, int* status)
{
    if (threadIdx.x || blockIdx.x) return;
    finalize_scalars(bs, unit, sc, status);
}

// primitives in leaf order
__device__ __forceinline__ void gather_prim(int k, const Geo& g, const int* __restrict__ sorted,
                                            const float* __restrict__ params, float4* __restrict__ hdr,
                                            float4* __restrict__ ext, int* __restrict__ sorted_out)
{
    if (k >= g.n) return;
    int p = sorted[k];
    sorted_out[k] = p;
    float3 a = prim_vertex(g, p, 0);
    if (p < g.np) {
        hdr[k] = make_float4(a.x, a.y, a.z, (float)SD_KIND_POINT);
        return;
    }
    if (p < g.np + g.ne) {
        float3 b = prim_vertex(g, p, 1);
        hdr[k] = make_float4(a.x, a.y, a.z, (float)SD_KIND_SEG);
        ext[2 * k] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, params[2 * p]);
        ext[2 * k + 1] = make_float4(params[2 * p + 1], 0.f, 0.f, 0.f);
        return;
    }
    float3 b = prim_vertex(g, p, 1), c = prim_vertex(g, p, 2);
    hdr[k] = make_float4(a.x, a.y, a.z, (float)SD_KIND_TRI);
    ext[2 * k] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, params[2 * p]);
    ext[2 * k + 1] = make_float4(c.x - a.x, c.y - a.y, c.z - a.z, params[2 * p + 1]);
}

// After the sort, in one launch: the radix tree's topology (Karras), every
// bucket's aggregates and aligned runs, and the primitives in leaf order.
// Blocks [0, nbk) take the topology, the next nbl blocks the buckets, the
// rest the gather (a block-uniform split; only the bucket blocks use
// barriers).
struct AfterSort {
    Geo g;
    const unsigned long long* sk; const int* sv; int L; int nb;
    int* left; int* right; int* parent_int; int2* range;
    SdNode* nodes; float2* lw2;
    float* leaf_box; int* leaf_count; float4* runs;
    const BuildScalars* bs; float S; int unit;
    const float* params; float4* hdr; float4* ext; int* sorted_out;
    int nbk, nbl;
};

__global__ void __launch_bounds__(AGG_T) k_after_sort(AfterSort A)
{
    sdsort::pdl_release();      // the node kernel may launch
    int blk = blockIdx.x;
    if (blk < A.nbk) {
        const int i = blk * AGG_T + threadIdx.x;
        karras_node(i, A.sk, A.sv, A.L, A.nb, A.left, A.right, A.parent_int, A.range, A.nodes, A.lw2);
        return;
    }
    blk -= A.nbk;
    if (blk < A.nbl) {
        leaves_block(blk, A.g, A.sv, A.L, A.nb, A.leaf_box, A.leaf_count, A.runs, A.nodes, A.lw2, A.bs, A.S, A.unit);
        return;
    }
    blk -= A.nbl;
    gather_prim(blk * AGG_T + threadIdx.x, A.g, A.sv, A.params, A.hdr, A.ext, A.sorted_out);
}

inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 1 << 20)); }

// The nested-Horner weight tables (sd_wtab.h) live in one static device
// array per device, filled once by a synchronous copy (the first build on a
// device must therefore not be under stream capture) and read by every
// tree's kernels through SdParams::wtab.
static __device__ __align__(16) float g_wtab[SD_WT_TOTAL];
std::mutex g_wtab_mu;
const float* g_wtab_addr[64] = {};

int weight_tables(cudaStream_t st, const float** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sd_cuda_status(e);
    if (dev < 0 || dev >= 64) return SD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_wtab_mu);
    if (!g_wtab_addr[dev]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            sd_set_last_error("the first sd_build on a device fills a constant table and cannot be captured");
            return SD_ERR_INVALID_ARG;
        }
        static std::vector<float> host;
        if (host.empty()) {
            host.resize(SD_WT_TOTAL);
            if (sd_weight_horner_tables(host.data()) != SD_OK ||
                sd_weight_horner_basis(host.data() + SD_WT_CLASSES) != SD_OK) {
                host.clear();
                return SD_ERR_INVALID_ARG;
            }
        }
        e = cudaMemcpyToSymbol(g_wtab, host.data(), sizeof(float) * SD_WT_TOTAL);
        if (e != cudaSuccess) return sd_cuda_status(e);
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_wtab);
        if (e != cudaSuccess) return sd_cuda_status(e);
        g_wtab_addr[dev] = (const float*)p;
    }
    *out = g_wtab_addr[dev];
    return SD_OK;
}

// the library's triangle weight basis as the three float tables of SdParams
int load_weight_basis(SdParams& P)
{
    double b[108];
    int rc = sd_weight_basis(b);
    if (rc != SD_OK) return rc;
    for (int n = 0; n < 36; ++n) {
        P.tri_base[n] = (float)b[72 + n];          // (v-1)/v column: the barycentre basis
        P.tri_dv[n] = (float)(b[n] - b[72 + n]);   // 1/v column minus the barycentre column
        P.tri_de[n] = (float)b[36 + n];            // 1/e column
    }
    return SD_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// One library-owned non-blocking stream per device for the build's
// independent branch (weight parameters and the leaf-order gather run there
// beside the Morton sort, the topology and the aggregates). Every build on
// the device shares it, so concurrent builds queue their branches behind
// one another; each build's own stream waits only for its own events.
static std::mutex g_side_mu;
static cudaStream_t g_side[64] = {};

static cudaStream_t side_stream(int dev)
{
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(g_side_mu);
    if (!g_side[dev]) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_side[dev] = s;
    }
    return g_side[dev];
}

static std::mutex g_use_mu;

void sd_mark_use(const sd_tree* tc, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) { cudaGetLastError(); return; }
    if (cs != cudaStreamCaptureStatusNone) return;
    sd_tree* t = const_cast<sd_tree*>(tc);
    std::lock_guard<std::mutex> g(g_use_mu);
    int i = 0;
    while (i < t->n_use && t->use_stream[i] != st) ++i;
    if (i == t->n_use) {
        if (t->n_use < 4) {
            if (cudaEventCreateWithFlags(&t->use_event[i], cudaEventDisableTiming) != cudaSuccess) {
                // no event: wait for the work now instead
                cudaGetLastError();
                cudaStreamSynchronize(st);
                return;
            }
            ++t->n_use;
        } else {
            // reuse the oldest slot once its stream's recorded work is done
            i = t->use_next;
            t->use_next = (t->use_next + 1) % 4;
            cudaEventSynchronize(t->use_event[i]);
        }
        t->use_stream[i] = st;
    }
    cudaEventRecord(t->use_event[i], st);
}

// the tree info fields that come from the device
static void fill_info(sd_tree* t, const SdScalars& hs)
{
    sd_tree_info& inf = t->info;
    inf.A_E = hs.A_E;
    inf.A_T = hs.A_T;
    float A = std::max(inf.A_E, inf.A_T);
    inf.w_far = t->weights_unit ? 1.f : (inf.S == 1.f ? A : std::pow(A, inf.S));
    for (int j = 0; j < 3; ++j) {
        inf.scene_lo[j] = hs.lo[j];
        inf.scene_hi[j] = hs.hi[j];
    }
    t->info_ready = true;
}

// Launches a kernel as the programmatic dependent of the kernel before it
// on `st` (it may start while that one finishes; the kernel itself waits
// for its predecessor before touching memory); an ordinary launch if the
// attribute is refused.
template <typename... P, typename... A>
void launch_dependent(void (*kern)(P...), dim3 grid, dim3 block, cudaStream_t st, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, args...) != cudaSuccess) {
        cudaGetLastError();
        kern<<<grid, block, 0, st>>>(args...);
    }
}

extern "C" int sd_build(const sd_geometry* g, float alpha, float beta, const sd_build_opts* opts_in,
                        void* stream, sd_tree** out)
{
    if (!out) return SD_ERR_INVALID_ARG;
    *out = nullptr;
    if (!g) return SD_ERR_INVALID_ARG;
    sd_build_opts opts;
    if (opts_in) opts = *opts_in; else sd_default_build_opts(&opts);
    if (!(alpha > 0.f) || !std::isfinite(alpha) || !(beta >= 0.f) || !std::isfinite(beta)) return SD_ERR_INVALID_ARG;
    if (opts.leaf_size < 1 || opts.leaf_size > 1024 || !(opts.alpha_u >= 0.f)) return SD_ERR_INVALID_ARG;
    if (g->pts.n < 0 || g->edges.nv < 0 || g->edges.ne < 0 || g->tris.nv < 0 || g->tris.nf < 0) return SD_ERR_INVALID_ARG;
    if ((g->pts.n && !g->pts.xyz) || (g->edges.ne && (!g->edges.V || !g->edges.E)) ||
        (g->tris.nf && (!g->tris.V || !g->tris.F)))
        return SD_ERR_INVALID_ARG;
    int64_t n64 = g->pts.n + g->edges.ne + g->tris.nf;
    const int64_t LIM = (int64_t)1 << 30;
    if (n64 >= LIM || g->edges.nv >= LIM || g->tris.nv >= LIM || 3 * g->tris.nf >= LIM) return SD_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    const float* wtab = nullptr;
    {
        int trc = weight_tables(st, &wtab);
        if (trc != SD_OK) return trc;
    }

    Geo geo;
    geo.P = g->pts.xyz; geo.np = (int)g->pts.n;
    geo.EV = g->edges.V; geo.nev = g->edges.ne ? (int)g->edges.nv : 0; geo.E = g->edges.E; geo.ne = (int)g->edges.ne;
    geo.TV = g->tris.V; geo.ntv = g->tris.nf ? (int)g->tris.nv : 0; geo.F = g->tris.F; geo.nf = (int)g->tris.nf;
    geo.n = (int)n64;
    const int n = geo.n;
    const int L = opts.leaf_size;
    const int nb = n > 0 ? (n + L - 1) / L : 0;
    const int ni = nb > 0 ? nb - 1 : 0;
    int kinds = (geo.np ? SD_HAS_PTS : 0) | (geo.ne ? SD_HAS_SEGS : 0) | (geo.nf ? SD_HAS_TRIS : 0);

    sd_tree* t = new sd_tree();
    std::memset(t, 0, sizeof(*t));
    t->device = dev;
    t->kinds = kinds;
    t->weights_unit = opts.weights == SD_WEIGHTS_UNIT;
    t->paper_metric = opts.paper_metric != 0;
    float S = alpha / std::max(alpha, opts.alpha_u);

    // persistent memory
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += align_up(std::max<size_t>(bytes, 1)); return o; };
    size_t o_nodes = carve(sizeof(SdNode) * std::max(nb, 1));
    size_t o_nw = carve(sizeof(float2) * std::max(nb, 1));
    size_t o_hdr = carve(sizeof(float4) * std::max(n, 1));
    size_t o_ext = carve((kinds & (SD_HAS_SEGS | SD_HAS_TRIS)) ? sizeof(float4) * 2 * (size_t)n : 16);
    size_t o_codes = carve(sizeof(uint64_t) * std::max(n, 1));
    size_t o_sorted = carve(sizeof(int) * std::max(n, 1));
    size_t o_left = carve(sizeof(int) * std::max(ni, 1));
    size_t o_right = carve(sizeof(int) * std::max(ni, 1));
    size_t o_nbox = carve(sizeof(float) * 6 * std::max(ni, 1));
    size_t o_ncnt = carve(sizeof(int) * std::max(ni, 1));
    size_t o_lbox = carve(sizeof(float) * 6 * std::max(nb, 1));
    size_t o_lcnt = carve(sizeof(int) * std::max(nb, 1));
    size_t o_params = carve(sizeof(float) * 2 * std::max(n, 1));
    size_t o_status = carve(sizeof(int) * 4);
    size_t o_sc = carve(sizeof(SdScalars));
    t->mem_bytes = off;
    cudaError_t ce = cudaMallocAsync(&t->mem, off, st);
    if (ce != cudaSuccess) { delete t; cudaGetLastError(); return SD_ERR_OOM; }
    char* base = (char*)t->mem;
    t->nodes = (SdNode*)(base + o_nodes);
    t->lw2 = (float2*)(base + o_nw);
    t->hdr = (float4*)(base + o_hdr);
    t->ext = (float4*)(base + o_ext);
    t->codes = (uint64_t*)(base + o_codes);
    t->sorted = (int32_t*)(base + o_sorted);
    t->left = (int32_t*)(base + o_left);
    t->right = (int32_t*)(base + o_right);
    t->node_box = (float*)(base + o_nbox);
    t->node_count = (int32_t*)(base + o_ncnt);
    t->leaf_box = (float*)(base + o_lbox);
    t->leaf_count = (int32_t*)(base + o_lcnt);
    t->params = (float*)(base + o_params);
    t->status = (int*)(base + o_status);
    t->sc = (SdScalars*)(base + o_sc);

    // temporary memory
    size_t toff = 0;
    auto tcarve = [&](size_t bytes) { size_t o = toff; toff += align_up(std::max<size_t>(bytes, 1)); return o; };
    unsigned hcap = 1;
    while (hcap < (unsigned)std::max(2 * 3 * geo.nf, 2)) hcap <<= 1;
    size_t t_bs = tcarve(sizeof(BuildScalars));
    size_t t_k1 = tcarve(sizeof(unsigned long long) * std::max(n, 1));
    size_t t_v0 = tcarve(sizeof(int) * std::max(n, 1));
    size_t t_v1 = tcarve(sizeof(int) * std::max(n, 1));
    size_t t_k0 = tcarve(sizeof(unsigned long long) * std::max(n, 1));
    size_t t_hist = tcarve(sizeof(uint32_t) * sdsort::hist_words(std::max(n, 1)));
    size_t t_ecnt = tcarve(sizeof(int) * std::max(geo.nev, 1));
    size_t t_vcnt = tcarve(sizeof(int) * std::max(geo.ntv, 1));
    size_t t_hkeys = tcarve(geo.nf ? sizeof(unsigned long long) * hcap : 8);
    size_t t_hcnt = tcarve(geo.nf ? sizeof(int) * hcap : 4);
    size_t t_pint = tcarve(sizeof(int) * std::max(nb, 1));
    size_t t_range = tcarve(sizeof(int2) * std::max(nb, 1));
    size_t t_runs = tcarve(2 * sizeof(float4) * (size_t)std::max<int64_t>(run_level_offset(nb, AGG_LEVELS), 1));
    void* tmp = nullptr;
    ce = cudaMallocAsync(&tmp, toff, st);
    if (ce != cudaSuccess) { cudaFreeAsync(t->mem, st); delete t; cudaGetLastError(); return SD_ERR_OOM; }
    char* tb = (char*)tmp;
    BuildScalars* bs = (BuildScalars*)(tb + t_bs);
    auto* k0 = (unsigned long long*)(tb + t_k0);
    auto* k1 = (unsigned long long*)(tb + t_k1);
    int* v0 = (int*)(tb + t_v0);
    int* v1 = (int*)(tb + t_v1);
    uint32_t* hist = (uint32_t*)(tb + t_hist);
    int* ecnt = (int*)(tb + t_ecnt);
    int* vcnt = (int*)(tb + t_vcnt);
    auto* hkeys = (unsigned long long*)(tb + t_hkeys);
    int* hcnt = (int*)(tb + t_hcnt);
    int* pint = (int*)(tb + t_pint);
    int2* range = (int2*)(tb + t_range);
    float4* runs = (float4*)(tb + t_runs);

    const int T = 256;
    int nl = 0;   // kernel launches of this build
    {
        InitJob J;
        J.bs = bs; J.status = t->status;
        J.params = t->params; J.nparams = 2 * std::max(n, 1);
        // every record of a non-empty tree is written in full below
        J.nodes = (int4*)t->nodes; J.nnodes4 = n > 0 ? 0 : 4 * std::max(nb, 1);
        J.ecnt = ecnt; J.nev = geo.ne ? geo.nev : 0;
        J.vcnt = vcnt; J.ntv = geo.nf ? geo.ntv : 0;
        J.hcnt = hcnt; J.hkeys = hkeys; J.hcap = geo.nf ? (int)hcap : 0;
        J.hist = hist; J.nhist = (int)sdsort::hist_words(std::max(n, 1));
        int work = std::max({J.nparams, J.nnodes4, J.nev, J.ntv, J.hcap, J.nhist});
        ++nl;
        k_init<<<std::min(nblk(work, T), 1024), T, 0, st>>>(J);
    }
    // validation + scene box over every vertex
    {
        int64_t most = std::max<int64_t>({geo.np, geo.nev, geo.ntv, 2 * (int64_t)geo.ne, 3 * (int64_t)geo.nf, 1});
        ++nl;
        launch_dependent(k_validate, dim3(std::min(nblk(most, T), 1024), 5), dim3(T), st, geo, bs);
        ++nl;
        launch_dependent(k_box, dim3(1), dim3(32), st, (const BuildScalars*)bs, n, t->sc);
        // with deferred checks the build returns at once: mark the point
        // after which the scene box is final (sd_query_order waits for it,
        // not for the whole build)
        if (opts.defer_checks) {
            ce = cudaEventCreateWithFlags(&t->box_ready, cudaEventDisableTiming);
            if (ce == cudaSuccess) ce = cudaEventRecord(t->box_ready, st);
            if (ce != cudaSuccess) {
                if (t->box_ready) cudaEventDestroy(t->box_ready);
                t->box_ready = nullptr;
                cudaGetLastError();
            }
        }
    }
    // validation results are read once, at the end of the build; the kernels
    // below clamp every index they dereference

    // The weight parameters (incidence counts, App. C.2-C.3) do not feed the
    // Morton codes, the sort or the topology: they run on the side stream
    // from here on, beside the Morton codes and the sort, and the build
    // stream waits for them after the sort (the leaf-order gather and the
    // aggregates need them). Without a side stream everything stays on `st`.
    cudaStream_t ps = st;
    cudaEvent_t ev_fork = nullptr, ev_params = nullptr;
    if (n > 0 && (geo.ne || geo.nf)) {
        cudaStream_t sd = side_stream(dev);
        if (sd && cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&ev_params, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventRecord(ev_fork, st) == cudaSuccess && cudaStreamWaitEvent(sd, ev_fork, 0) == cudaSuccess) {
            ps = sd;
        }
        cudaGetLastError();
    }

    // incidence counts and weight parameters
    if (geo.ne) {
        ++nl;
        k_count_slots<<<std::min(nblk(2 * (int64_t)geo.ne, T), 4096), T, 0, ps>>>(geo.E, 2 * (int64_t)geo.ne, geo.nev, ecnt);
        ++nl;
        k_edge_params<<<nblk(geo.ne, T), T, 0, ps>>>(geo.E, geo.ne, geo.nev, ecnt, t->params, geo.np, bs);
    }
    if (geo.nf) {
        ++nl;
        k_count_slots<<<std::min(nblk(3 * (int64_t)geo.nf, T), 4096), T, 0, ps>>>(geo.F, 3 * (int64_t)geo.nf, geo.ntv, vcnt);
        ++nl;
        k_edge_insert<<<nblk(3 * (int64_t)geo.nf, T), T, 0, ps>>>(geo.F, geo.nf, hkeys, hcnt, hcap - 1);
        ++nl;
        k_tri_params<<<nblk(geo.nf, T), T, 0, ps>>>(geo.F, geo.nf, geo.ntv, vcnt, hkeys, hcnt, hcap - 1, t->params,
                                                     geo.np + geo.ne, bs);
    }
    if (ps != st) cudaEventRecord(ev_params, ps);
    if (n > 0) {
        // Morton order
        ++nl;
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
            cudaGetLastError();
            nsm = 1;
        }
        k_morton<<<std::min(nblk(n, T), 2 * nsm), T, 0, st>>>(geo, bs, (unsigned long long*)t->codes, k0, v0,
                                                              sdsort::digit_totals(hist, n, 8));
        int where = sdsort::sort_pairs<unsigned long long, int>(k0, v0, k1, v1, n, 64, hist, st, &nl, true);
        unsigned long long* sk = where ? k1 : k0;
        int* sv = where ? v1 : v0;
        // topology, buckets and gather need the sorted order and (the last
        // two) the weight parameters
        if (ps != st) cudaStreamWaitEvent(st, ev_params, 0);
        AfterSort A;
        A.g = geo; A.sk = sk; A.sv = sv; A.L = L; A.nb = nb;
        A.left = t->left; A.right = t->right; A.parent_int = pint; A.range = range;
        A.nodes = t->nodes; A.lw2 = t->lw2;
        A.leaf_box = t->leaf_box; A.leaf_count = t->leaf_count; A.runs = runs;
        A.bs = bs; A.S = S; A.unit = t->weights_unit;
        A.params = t->params; A.hdr = t->hdr; A.ext = t->ext; A.sorted_out = t->sorted;
        A.nbk = nb > 1 ? nblk(nb - 1, AGG_T) : 0;
        A.nbl = nblk(nb, AGG_T);
        ++nl;
        k_after_sort<<<A.nbk + A.nbl + nblk(n, AGG_T), AGG_T, 0, st>>>(A);
        // internal nodes from the runs (far-field weights use A)
        if (nb > 1) {
            ++nl;
            launch_dependent(k_nodes, dim3(nblk(nb - 1, T)), dim3(T), st, nb, L, n, (const int2*)range,
                             (const int*)t->left, (const int*)t->right, (const int*)pint, (const float4*)runs,
                             t->node_box, t->node_count, t->nodes, t->lw2, (const BuildScalars*)bs, S,
                             t->weights_unit, t->sc, t->status);
        } else {
            ++nl;
            k_super_root<<<1, 1, 0, st>>>(t->nodes, t->lw2, nb);
        }
    }
    for (cudaEvent_t e : {ev_fork, ev_params})
        if (e) cudaEventDestroy(e);
    if (nb < 2) {
        ++nl;
        k_finalize<<<1, 32, 0, st>>>(bs, t->weights_unit, t->sc, t->status);
    }
    cudaFreeAsync(tmp, st);
    sd_count_launches(nl);

    sd_tree_info& inf = t->info;
    inf.n_prims = n; inf.n_points = geo.np; inf.n_edges = geo.ne; inf.n_tris = geo.nf;
    inf.n_buckets = nb; inf.leaf_size = L;
    inf.alpha = alpha; inf.beta = beta; inf.alpha_u = opts.alpha_u; inf.S = S;
    inf.device_bytes = (int64_t)t->mem_bytes;
    if (opts.defer_checks) {
        // return at once: the checks' outcome reaches the status word
        // (sd_query_status), the device scalars reach info on demand
        ce = cudaEventCreateWithFlags(&t->built, cudaEventDisableTiming);
        if (ce == cudaSuccess) ce = cudaEventRecord(t->built, st);
        if (ce == cudaSuccess) ce = cudaGetLastError();
        if (ce != cudaSuccess) {
            cudaStreamSynchronize(st);
            if (t->built) cudaEventDestroy(t->built);
            if (t->box_ready) cudaEventDestroy(t->box_ready);
            cudaFreeAsync(t->mem, st);
            delete t;
            return sd_cuda_status(ce);
        }
    } else {
        SdScalars hs;
        ce = cudaMemcpyAsync(&hs, t->sc, sizeof(hs), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce == cudaSuccess) ce = cudaGetLastError();
        int status = SD_OK;
        if (ce != cudaSuccess) status = sd_cuda_status(ce);
        else if (hs.status & ST_INDEX) status = SD_ERR_INDEX;
        else if (hs.status & ST_NONFINITE) status = SD_ERR_NONFINITE;
        if (status != SD_OK) {
            cudaFreeAsync(t->mem, st);
            delete t;
            return status;
        }
        fill_info(t, hs);
    }

    SdParams& P = t->P;
    int wrc = load_weight_basis(P);
    if (wrc != SD_OK) {
        cudaStreamSynchronize(st);
        if (t->built) cudaEventDestroy(t->built);
        if (t->box_ready) cudaEventDestroy(t->box_ready);
        cudaFreeAsync(t->mem, st);
        delete t;
        return wrc;
    }
    P.wtab = wtab;
    P.nodes = t->nodes;
    P.lw2 = t->lw2;
    P.hdr = t->hdr;
    P.ext = t->ext;
    P.root_record = nb - 1;
    P.n_prims = n;
    P.L = L;
    P.beta2 = beta * beta;
    const float LOG2E = 1.4426950408889634f;
    P.alpha2 = alpha * LOG2E;
    P.inv_alpha2 = 1.f / P.alpha2;
    P.S = S;
    P.sc = t->sc;
    P.kw = t->paper_metric ? S / (alpha * alpha) : S / alpha;
    P.unit_weights = t->weights_unit;
    P.s_is_one = S == 1.f;
    sd_mark_use(t, st);
    *out = t;
    return SD_OK;
}

extern "C" int sd_tree_get_info(const sd_tree* t, sd_tree_info* info)
{
    if (!t || !info) return SD_ERR_INVALID_ARG;
    if (!t->info_ready) {
        // a build with deferred checks: wait for it and read its scalars
        sd_tree* m = const_cast<sd_tree*>(t);
        SdScalars hs;
        cudaError_t e = cudaEventSynchronize(t->built);
        if (e == cudaSuccess) e = cudaMemcpy(&hs, t->sc, sizeof(hs), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return sd_cuda_status(e);
        fill_info(m, hs);
    }
    *info = t->info;
    return SD_OK;
}

extern "C" int sd_tree_export(const sd_tree* t, sd_tree_view* v)
{
    if (!t || !v) return SD_ERR_INVALID_ARG;
    int64_t n = t->info.n_prims, nb = t->info.n_buckets, ni = nb > 0 ? nb - 1 : 0;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        if (dst && bytes && e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
    };
    cp(v->codes, t->codes, sizeof(uint64_t) * n);
    cp(v->sorted, t->sorted, sizeof(int32_t) * n);
    cp(v->left, t->left, sizeof(int32_t) * ni);
    cp(v->right, t->right, sizeof(int32_t) * ni);
    cp(v->node_count, t->node_count, sizeof(int32_t) * ni);
    cp(v->leaf_count, t->leaf_count, sizeof(int32_t) * nb);
    cp(v->params, t->params, sizeof(float) * 2 * n);
    if (e == cudaSuccess && (v->node_lo || v->node_hi) && ni) {
        std::vector<float> box(6 * ni);
        cp(box.data(), t->node_box, sizeof(float) * 6 * ni);
        for (int64_t i = 0; i < ni; ++i)
            for (int j = 0; j < 3; ++j) {
                if (v->node_lo) v->node_lo[3 * i + j] = box[6 * i + j];
                if (v->node_hi) v->node_hi[3 * i + j] = box[6 * i + 3 + j];
            }
    }
    if (e == cudaSuccess && (v->leaf_lo || v->leaf_hi) && nb) {
        std::vector<float> box(6 * nb);
        cp(box.data(), t->leaf_box, sizeof(float) * 6 * nb);
        for (int64_t i = 0; i < nb; ++i)
            for (int j = 0; j < 3; ++j) {
                if (v->leaf_lo) v->leaf_lo[3 * i + j] = box[6 * i + j];
                if (v->leaf_hi) v->leaf_hi[3 * i + j] = box[6 * i + 3 + j];
            }
    }
    return e == cudaSuccess ? SD_OK : sd_cuda_status(e);
}

extern "C" void sd_free(sd_tree* t)
{
    if (!t) return;
    // the memory is stream-ordered (cudaMallocAsync), and cudaFree does not
    // wait for work still queued on it: wait for every recorded use first
    for (int i = 0; i < t->n_use; ++i) {
        cudaEventSynchronize(t->use_event[i]);
        cudaEventDestroy(t->use_event[i]);
    }
    if (t->built) {
        cudaEventSynchronize(t->built);
        cudaEventDestroy(t->built);
    }
    if (t->box_ready) cudaEventDestroy(t->box_ready);
    if (t->mem) cudaFree(t->mem);
    delete t;
}
