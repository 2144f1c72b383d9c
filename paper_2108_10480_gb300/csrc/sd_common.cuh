// Internal structures and device functions shared by the build and query
// translation units of libsd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sd.h"
#include "sd_wtab.h"

// ---------------------------------------------------------------------------
// tree layout in device memory
// ---------------------------------------------------------------------------
// One record per internal node of the binary radix tree (Karras numbering,
// 0 .. nb-2) plus a super-root record at index nb-1 whose child 0 is the
// root. Each record holds what the Barnes-Hut test of Alg. 1 / App. D needs
// for BOTH children, interleaved so that the two tests run as packed
// two-wide fp32 operations: lower corners, negated upper corners (so that
// q - hi is an exact packed add), child references and squared diagonals.
//   a = (c0.lo.x, c1.lo.x, c0.lo.y, c1.lo.y)
//   b = (c0.lo.z, c1.lo.z, -c0.hi.x, -c1.hi.x)
//   c = (-c0.hi.y, -c1.hi.y, -c0.hi.z, -c1.hi.z)
//   d = (ref0, ref1, bits(diag2_0), bits(diag2_1))
// ref >= 0: internal node; ref < 0: leaf bucket -(ref + 1); SD_NO_CHILD: none.
// log2 of the far-field masses n_B w_B of both children sits in lw2[record].
struct __align__(16) SdNode {
    float4 a, b, c;
    int4 d;
};
#define SD_NO_CHILD ((int)0x80000000)

// Primitive records in sorted (leaf) order:
//   hdr[k]   = (x, y, z, kind)        first vertex (point / a / v0), kind as float 0/1/2
//   ext[2k]  = segment (e.xyz, u)  | triangle (e1.xyz, 1/v_i)
//   ext[2k+1]= segment (v, 0, 0, 0)| triangle (e2.xyz, 1/e_i)
// with e = b - a, e1 = v1 - v0, e2 = v2 - v0 rounded to fp32.
enum { SD_KIND_POINT = 0, SD_KIND_SEG = 1, SD_KIND_TRI = 2 };
enum { SD_HAS_PTS = 1, SD_HAS_SEGS = 2, SD_HAS_TRIS = 4 };

// Tree scalars that the build computes on the device (read by the kernels,
// copied to the host only when the tree's info is asked for).
struct SdScalars {
    float A_E, A_T;         // weight scales A of App. C.2 / C.3 (1 for unit weights)
    float lo[3], inv_ex[3]; // scene box corner and 1 / extent (0 on a flat axis): query codes
    float hi[3];
    int status;             // build validation bits
    int pad[2];
};

// Parameters a traversal needs, passed by value to the kernels.
struct SdParams {
    const SdNode* nodes;
    const float2* lw2;    // log2 of the far-field masses n_B w_B of both children, per record
    const float4* hdr;
    const float4* ext;
    int root_record;      // nb - 1 (also the offset of bucket ids in nw)
    int n_prims;
    int L;
    float beta2;          // beta*beta rounded to fp32 (the Barnes-Hut test is taken in fp32)
    float alpha2;         // alpha * log2(e): exponents are kept in base 2
    float inv_alpha2;     // 1 / alpha2
    float S;              // attenuation exponent
    const SdScalars* sc;  // device-computed scalars (A_E, A_T, scene box)
    float kw;             // S / alpha (S / alpha^2 with the alpha-scaled metric)
    int unit_weights;
    int s_is_one;
    // triangle weight basis in Bernstein form (App. C.3): for a triangle,
    // b_n = tri_base[n] + (1/v) tri_dv[n] + (1/e) tri_de[n]; index of (i,j,k)
    // is r(r+1)/2 + k with r = j + k (see sd_weight_basis). Kernel parameters
    // live in the constant bank, so every lane reads them by broadcast.
    float tri_base[36];
    float tri_dv[36];
    float tri_de[36];
    // the same weights as nested-Horner tables per class (v, e) and
    // orientation, then the blend's three parts (sd_wtab.h)
    const float* wtab;
};

struct sd_tree {
    int device;
    sd_tree_info info;
    int kinds;
    int weights_unit, paper_metric;
    SdParams P;
    // persistent device memory (one allocation, carved)
    void* mem;
    size_t mem_bytes;
    SdNode* nodes;        // nb records (nb - 1 internal + super-root)
    float2* lw2;          // nb pairs of log2 far-field masses
    float4* hdr;          // n
    float4* ext;          // 2n (only when edges or triangles exist)
    uint64_t* codes;      // n, original order
    int32_t* sorted;      // n, sorted position -> original index
    int32_t* left;        // nb - 1
    int32_t* right;       // nb - 1
    float* node_box;      // (nb - 1) * 6: lo.xyz, hi.xyz
    int32_t* node_count;  // nb - 1
    float* leaf_box;      // nb * 6
    int32_t* leaf_count;  // nb
    float* params;        // 2n, original order
    int* status;          // device status word
    SdScalars* sc;        // device scalars written at the end of the build
    bool info_ready;      // info's device-derived fields (A, w_far, scene box) filled in
    cudaEvent_t built;    // recorded after the build's last kernel (deferred checks)
    cudaEvent_t box_ready;   // recorded once the scene box in sc is final (deferred checks)
    // streams that have enqueued work on the tree and an event recorded after
    // their latest such work: sd_free waits for these before releasing memory
    cudaStream_t use_stream[4];
    cudaEvent_t use_event[4];
    int n_use, use_next;
};

// Record that `st` has enqueued work reading the tree (outside stream capture;
// a captured graph's owner keeps the tree alive while the graph can run).
void sd_mark_use(const sd_tree* t, cudaStream_t st);

// Marks the tree's use on a stream when the enclosing API call returns.
struct SdUse {
    const sd_tree* t;
    cudaStream_t st;
    ~SdUse() { if (t) sd_mark_use(t, st); }
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sd_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sd_lg2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// a*b - c*d with one rounding error (Kahan's FMA difference of products,
// the cancellation-safe form the paper uses for its distance kernels).
__device__ __forceinline__ float sd_dop(float a, float b, float c, float d)
{
    float w = c * d;
    float e = fmaf(-c, d, w);
    float f = fmaf(a, b, -w);
    return f + e;
}

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 add(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 scale(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 axpy(float s, float3 x, float3 y) { return f3(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y), fmaf(s, x.z, y.z)); }
__device__ __forceinline__ float3 cross_k(float3 a, float3 b)
{
    return f3(sd_dop(a.y, b.z, a.z, b.y), sd_dop(a.z, b.x, a.x, b.z), sd_dop(a.x, b.y, a.y, b.x));
}

// Running LogSumExp state in base 2: the sum is s * 2^m, the gradient
// numerator g * 2^m (Eq. 4 numerator). m starts at -inf.
struct Lse {
    float m, s, gx, gy, gz;
};

__device__ __forceinline__ void lse_init(Lse& L)
{
    L.m = -INFINITY; L.s = 0.f; L.gx = L.gy = L.gz = 0.f;
}

// add w * 2^y with gradient vector v (weights carried multiplicatively)
template <bool GRAD>
__device__ __forceinline__ void lse_add(Lse& L, float y, float w, float3 v)
{
    float dl = y - L.m;
    float e = sd_ex2(-fabsf(dl));
    bool up = dl > 0.f;
    float a = up ? e : 1.f;
    float b = up ? w : w * e;
    L.s = fmaf(L.s, a, b);
    if (GRAD) {
        L.gx = fmaf(L.gx, a, b * v.x);
        L.gy = fmaf(L.gy, a, b * v.y);
        L.gz = fmaf(L.gz, a, b * v.z);
    }
    L.m = up ? y : L.m;
}

// fp32 sum of squares in the fixed order fma(z, z, fma(y, y, x * x)), each
// step rounded once (never re-associated or split by the compiler)
__device__ __forceinline__ float sumsq3(float x, float y, float z)
{
    return __fmaf_rn(z, z, __fmaf_rn(y, y, __fmul_rn(x, x)));
}

// squared diagonal |B|^2 of an AABB (App. D), stored in the tree records
__device__ __forceinline__ float box_diag2(const float* lo, const float* hi)
{
    return sumsq3(__fsub_rn(hi[0], lo[0]), __fsub_rn(hi[1], lo[1]), __fsub_rn(hi[2], lo[2]));
}

// The Barnes-Hut test |B|^2 < beta^2 d(y_B, q)^2 (App. D) in fp32 with a fixed
// operation order, so that its outcome is reproducible bit for bit. Returns
// dbox2 and the signed offset q - y_B (y_B = closest point of the box).
// (Scalar form, used by the brute-force-free paths and the build checks.)
__device__ __forceinline__ bool bh_far(float3 q, float lx, float ly, float lz, float hx, float hy, float hz,
                                       float diag2, float beta2, float& dbox2, float3& off)
{
    float ax = __fsub_rn(lx, q.x), bx = __fsub_rn(q.x, hx);
    float ay = __fsub_rn(ly, q.y), by = __fsub_rn(q.y, hy);
    float az = __fsub_rn(lz, q.z), bz = __fsub_rn(q.z, hz);
    float dx = fmaxf(fmaxf(ax, bx), 0.f);
    float dy = fmaxf(fmaxf(ay, by), 0.f);
    float dz = fmaxf(fmaxf(az, bz), 0.f);
    dbox2 = sumsq3(dx, dy, dz);
    // q > hi: offset +d (b > 0); q < lo: offset -d (b < 0); inside: 0
    off = f3(copysignf(dx, bx), copysignf(dy, by), copysignf(dz, bz));
    return diag2 < __fmul_rn(beta2, dbox2);
}

// A term that is absent has exponent SD_NEG (finite, so that differences
// never give NaN); the running max m of a packet walk starts at SD_FLOOR,
// far above SD_NEG and far below any real exponent, so that an absent
// term's factor 2^(SD_NEG - m) is exactly 0 and the first real term's
// rescale 2^(SD_FLOOR - y) is exactly 0 as well.
#define SD_NEG (-8.5e37f)
#define SD_FLOOR (-1e30f)

// merge a second LSE state (m2, s2, g2) into L
template <bool GRAD>
__device__ __forceinline__ void lse_merge(Lse& L, float m2, float s2, float gx2, float gy2, float gz2)
{
    float dl = m2 - L.m;
    float e = sd_ex2(-fabsf(dl));
    bool up = dl > 0.f;
    float a = up ? e : 1.f;
    float b = up ? 1.f : e;
    L.s = fmaf(L.s, a, s2 * b);
    if (GRAD) {
        L.gx = fmaf(L.gx, a, gx2 * b);
        L.gy = fmaf(L.gy, a, gy2 * b);
        L.gz = fmaf(L.gz, a, gz2 * b);
    }
    L.m = up ? m2 : L.m;
}

// ---------------------------------------------------------------------------
// weights (App. C) in Bernstein form
// ---------------------------------------------------------------------------
// Edge weight w~(t) with w~(0) = u, w~(1) = v, w~(1/2) = 1, w~'(0) = w~'(1) = 0
// (App. C.2) as a quartic in Bernstein form: control values (u, u, c, v, v)
// with c = (16 - 5u - 5v) / 6 (from w~(1/2) = (5u + 6c + 5v) / 16 = 1).
__device__ __forceinline__ float edge_weight(float t, float u, float v, float& dwdt)
{
    float s = 1.f - t;
    float c = (16.f - 5.f * u - 5.f * v) * (1.f / 6.f);
    float s2 = s * s, t2 = t * t, st = s * t;
    // B^4: s^4, 4 s^3 t, 6 s^2 t^2, 4 s t^3, t^4
    float w = u * (s2 * fmaf(4.f, st, s2)) + 6.f * c * s2 * t2 + v * (t2 * fmaf(4.f, st, t2));
    dwdt = 12.f * st * fmaf(c - u, s, (v - c) * t);
    return w;
}

// de Casteljau evaluation of the degree-7 triangle weight and its partial
// derivatives with respect to (phi1, phi2) (phi0 = 1 - phi1 - phi2).
__device__ __forceinline__ float tri_weight(const SdParams& P, float p1, float p2, float iv, float ie, float& d1,
                                            float& d2)
{
    float p0 = 1.f - p1 - p2;
    float b[36];
#pragma unroll
    for (int n = 0; n < 36; ++n) b[n] = fmaf(ie, P.tri_de[n], fmaf(iv, P.tri_dv[n], P.tri_base[n]));
    // reduce degree 7 -> 1; at degree r the entry (i,j,k) sits at
    // (j+k)(j+k+1)/2 + k, the same layout truncated to rows 0..r
#pragma unroll
    for (int deg = 7; deg > 1; --deg) {
#pragma unroll
        for (int rr = 0; rr < deg; ++rr) {
#pragma unroll
            for (int k = 0; k <= rr; ++k) {
                // child (i, j, k) of degree deg-1 with j + k = rr: combine
                // (i+1, j, k) [row rr], (i, j+1, k) [row rr+1, same k],
                // (i, j, k+1) [row rr+1, k+1]
                int o = rr * (rr + 1) / 2 + k;
                int r1 = (rr + 1) * (rr + 2) / 2;
                b[o] = fmaf(p0, b[o], fmaf(p1, b[r1 + k], p2 * b[r1 + k + 1]));
            }
        }
    }
    // degree 1: b[0] = (1,0,0), b[1] = (0,1,0), b[2] = (0,0,1)
    d1 = 7.f * (b[1] - b[0]);
    d2 = 7.f * (b[2] - b[0]);
    return fmaf(p0, b[0], fmaf(p1, b[1], p2 * b[2]));
}

// The same weight and partials by nested Horner evaluation (sd_wtab.h): with
// phi_o the largest barycentric and x, y the other two divided by it (both
// in [0, 1]), w~ = phi_o^7 sum c_ab x^a y^b and dw~/dphi_1,2 = phi_o^6 sum
// c'_ab x^a y^b, coefficients (Bernstein coefficient times multinomial) read
// in Horner order, row by row. 36 + 2 x 28 FMAs instead of de Casteljau's
// 84 x 3, and few coefficients live at a time; with the ratios in [0, 1] the
// rounding error stays of the order of de Casteljau's (a few ulps of the sum
// of the terms' magnitudes). BLEND: the class is outside the tables, and
// each coefficient is blended from the base, dv, de tables (sd_wtab.h) as
// base + iv dv + ie de.
template <bool BLEND>
__device__ __forceinline__ float wt_coef(const float* __restrict__ t, int n, float iv, float ie)
{
    if (!BLEND) return __ldg(t + n);
    const int part = 3 * SD_WT_FLOATS;
    return fmaf(ie, __ldg(t + 2 * part + n), fmaf(iv, __ldg(t + part + n), __ldg(t + n)));
}

template <bool BLEND>
__device__ __forceinline__ float tri_weight_horner(const float* __restrict__ T, float iv, float ie, float p1, float p2,
                                                   float& d1, float& d2)
{
    const float p0 = 1.f - p1 - p2;
    const bool o0 = p0 >= p1 && p0 >= p2, o1 = !o0 && p1 >= p2;
    const float base = o0 ? p0 : (o1 ? p1 : p2);
    const float x = o0 ? p1 : p0, y = o0 || o1 ? p2 : p1;
    const float ib = __frcp_rn(base);
    const float r = x * ib, s = y * ib;
    const float* t = T + (o0 ? 0 : (o1 ? 1 : 2)) * SD_WT_FLOATS;
    // value: powers of y from 7 down, each row a Horner polynomial in x
    float acc = 0.f;
    int n = 0;
#pragma unroll
    for (int bp = 7; bp >= 0; --bp) {
        float inner = wt_coef<BLEND>(t, n++, iv, ie);
#pragma unroll
        for (int ap = 7 - bp; ap > 0; --ap) inner = fmaf(inner, r, wt_coef<BLEND>(t, n++, iv, ie));
        acc = fmaf(acc, s, inner);
    }
    // the two partials (degree 6)
    float g1 = 0.f, g2 = 0.f;
#pragma unroll
    for (int bp = 6; bp >= 0; --bp) {
        float i1 = wt_coef<BLEND>(t, n, iv, ie), i2 = wt_coef<BLEND>(t, n + 28, iv, ie);
        ++n;
#pragma unroll
        for (int ap = 6 - bp; ap > 0; --ap) {
            i1 = fmaf(i1, r, wt_coef<BLEND>(t, n, iv, ie));
            i2 = fmaf(i2, r, wt_coef<BLEND>(t, n + 28, iv, ie));
            ++n;
        }
        g1 = fmaf(g1, s, i1);
        g2 = fmaf(g2, s, i2);
    }
    const float b2 = base * base, b3 = b2 * base, b6 = b3 * b3;
    d1 = g1 * b6;
    d2 = g2 * b6;
    return acc * (b6 * base);
}

// ---------------------------------------------------------------------------
// leaf terms (App. B distances + Sec. 3.3 weights). Each returns the base-2
// exponent y, the multiplicative weight w and the gradient vector v so that
// the term is w 2^y with gradient numerator w 2^y v (Eq. 4).
// ---------------------------------------------------------------------------
// (The *_rel forms take the query relative to the primitive's first vertex.)
__device__ __forceinline__ void leaf_point_rel(const SdParams& P, float3 d, float& y, float& w, float3& v)
{
    float d2 = dot(d, d);
    float dist = sqrtf(d2);
    float inv = dist > 0.f ? 1.f / dist : 0.f;
    y = -P.alpha2 * dist;
    w = 1.f;
    v = scale(d, inv);
}

__device__ __forceinline__ void leaf_point(const SdParams& P, float3 q, float4 h, float& y, float& w, float3& v)
{
    leaf_point_rel(P, sub(q, f3(h.x, h.y, h.z)), y, w, v);
}

// weight factor for a weighted primitive: w~ and grad w~ -> (y, w, v)
template <bool GRAD>
__device__ __forceinline__ void apply_weight(const SdParams& P, float A, float dist, float wt, float3 gwt,
                                             float3 gd, float& y, float& w, float3& v)
{
    y = -P.alpha2 * dist;
    if (P.unit_weights) {
        w = 1.f;
        v = gd;
        return;
    }
    wt = fmaxf(wt, 1e-6f);
    if (P.s_is_one) {
        w = A * wt;
    } else {
        y = fmaf(P.S, sd_lg2(A * wt), y);
        w = 1.f;
    }
    if (GRAD) {
        float k = P.kw / wt;
        v = f3(fmaf(-k, gwt.x, gd.x), fmaf(-k, gwt.y, gd.y), fmaf(-k, gwt.z, gd.z));
    }
}

template <bool GRAD>
__device__ __forceinline__ void leaf_segment_rel(const SdParams& P, float3 ap, float4 x0, float4 x1,
                                                 float& y, float& w, float3& v, bool touch = false)
{
    float3 e = f3(x0.x, x0.y, x0.z);
    float u = x0.w, vv = x1.x;
    float ee = dot(e, e);
    float t = ee > 0.f ? dot(ap, e) / ee : 0.f;
    bool inside = t > 0.f && t < 1.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    float3 diff = axpy(-t, e, ap);
    float dist = touch ? 0.f : sqrtf(dot(diff, diff));   // touch: a query primitive touching it
    float3 gd = scale(diff, dist > 0.f ? 1.f / dist : 0.f);
    float dw = 0.f;
    float wt = (u == 1.f && vv == 1.f) ? 1.f : edge_weight(t, u, vv, dw);
    float3 gwt = f3(0.f, 0.f, 0.f);
    if (GRAD && inside) gwt = scale(e, dw / ee);
    apply_weight<GRAD>(P, __ldg(&P.sc->A_E), dist, wt, gwt, gd, y, w, v);
}

template <bool GRAD>
__device__ __forceinline__ void leaf_segment(const SdParams& P, float3 q, float4 h, float4 x0, float4 x1,
                                             float& y, float& w, float3& v)
{
    leaf_segment_rel<GRAD>(P, sub(q, f3(h.x, h.y, h.z)), x0, x1, y, w, v);
}

// Closest point of a triangle by its Voronoi regions (vertex, edge, face),
// in coordinates relative to v0; differences of products use sd_dop.
template <bool GRAD>
__device__ __forceinline__ void leaf_triangle_rel(const SdParams& P, float3 ap, float4 x0, float4 x1,
                                                  float& y, float& w, float3& v, bool touch = false)
{
    float3 e1 = f3(x0.x, x0.y, x0.z);
    float3 e2 = f3(x1.x, x1.y, x1.z);
    float iv = x0.w, ie = x1.w;
    float d1 = dot(e1, ap), d2 = dot(e2, ap);
    float g00 = dot(e1, e1), g01 = dot(e1, e2), g11 = dot(e2, e2);
    float d3 = d1 - g00, d4 = d2 - g01;      // q - v1 against e1, e2
    float d5 = d1 - g01, d6 = d2 - g11;      // q - v2 against e1, e2
    float3 n = cross_k(e1, e2);
    float nn = dot(n, n);
    float p1, p2;                             // barycentrics of the closest point
    float3 gp1 = f3(0.f, 0.f, 0.f), gp2 = f3(0.f, 0.f, 0.f);
    float3 diff;
    // sin^2 of the corner angle below 1e-10 counts as zero area
    bool degenerate = !(nn > 1e-10f * g00 * g11);
    if (d1 <= 0.f && d2 <= 0.f) {                       // vertex v0
        p1 = 0.f; p2 = 0.f; diff = ap;
    } else if (d3 >= 0.f && d4 <= d3) {                 // vertex v1
        p1 = 1.f; p2 = 0.f; diff = sub(ap, e1);
    } else if (d6 >= 0.f && d5 <= d6) {                 // vertex v2
        p1 = 0.f; p2 = 1.f; diff = sub(ap, e2);
    } else {
        float vc = sd_dop(d1, d4, d3, d2);
        float vb = sd_dop(d5, d2, d1, d6);
        float va = sd_dop(d3, d6, d5, d4);
        if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {       // edge v0v1
            float t = d1 / (d1 - d3);
            p1 = t; p2 = 0.f; diff = axpy(-t, e1, ap);
            if (GRAD) gp1 = scale(e1, 1.f / g00);
        } else if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) { // edge v0v2
            float t = d2 / (d2 - d6);
            p1 = 0.f; p2 = t; diff = axpy(-t, e2, ap);
            if (GRAD) gp2 = scale(e2, 1.f / g11);
        } else if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {   // edge v1v2
            float t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
            float3 e12 = sub(e2, e1);
            p1 = 1.f - t; p2 = t;
            diff = axpy(-t, e12, sub(ap, e1));
            if (GRAD) { gp2 = scale(e12, 1.f / dot(e12, e12)); gp1 = scale(gp2, -1.f); }
        } else {                                        // face: project along the normal
            float den = 1.f / (va + vb + vc);
            p1 = vb * den; p2 = vc * den;
            diff = scale(n, dot(ap, n) / nn);
            if (GRAD) {
                float inn = 1.f / nn;
                gp1 = scale(cross_k(e2, n), inn);
                gp2 = scale(cross_k(n, e1), inn);
            }
        }
    }
    if (degenerate) {
        // zero-area triangle: closest of its three sides, no weight gradient
        float best = INFINITY;
        float3 sides[3] = {e1, e2, sub(e2, e1)};
        float3 starts[3] = {ap, ap, sub(ap, e1)};
        for (int s = 0; s < 3; ++s) {
            float ee = dot(sides[s], sides[s]);
            float t = ee > 0.f ? fminf(fmaxf(dot(starts[s], sides[s]) / ee, 0.f), 1.f) : 0.f;
            float3 dd = axpy(-t, sides[s], starts[s]);
            float l = dot(dd, dd);
            if (l < best) {
                best = l; diff = dd;
                p1 = s == 0 ? t : (s == 1 ? 0.f : 1.f - t);
                p2 = s == 0 ? 0.f : t;
            }
        }
        gp1 = gp2 = f3(0.f, 0.f, 0.f);
    }
    float dist = touch ? 0.f : sqrtf(dot(diff, diff));   // touch: a query primitive touching it
    float3 gd = scale(diff, dist > 0.f ? 1.f / dist : 0.f);
    float wt = 1.f;
    float3 gwt = f3(0.f, 0.f, 0.f);
    if (!P.unit_weights && iv != 1.f) {
        float dw1, dw2;
        // the class (v, e) from the stored 1/v, 1/e (exact small integers)
        const int cv = __float2int_rn(__frcp_rn(iv)), ce = __float2int_rn(__frcp_rn(ie));
        if (cv <= SD_WT_VMAX && ce >= 1 && ce <= SD_WT_EMAX)
            wt = tri_weight_horner<false>(P.wtab + ((cv - 1) * SD_WT_EMAX + (ce - 1)) * 3 * SD_WT_FLOATS, iv, ie, p1,
                                          p2, dw1, dw2);
        else
            wt = tri_weight_horner<true>(P.wtab + SD_WT_CLASSES, iv, ie, p1, p2, dw1, dw2);
        if (GRAD) gwt = f3(dw1 * gp1.x + dw2 * gp2.x, dw1 * gp1.y + dw2 * gp2.y, dw1 * gp1.z + dw2 * gp2.z);
        if (wt < 1e-6f) gwt = f3(0.f, 0.f, 0.f);
    }
    apply_weight<GRAD>(P, __ldg(&P.sc->A_T), dist, wt, gwt, gd, y, w, v);
}

template <bool GRAD>
__device__ __forceinline__ void leaf_triangle(const SdParams& P, float3 q, float4 h, float4 x0, float4 x1,
                                              float& y, float& w, float3& v)
{
    leaf_triangle_rel<GRAD>(P, sub(q, f3(h.x, h.y, h.z)), x0, x1, y, w, v);
}

// one primitive at sorted position k
template <int KINDS, bool GRAD>
__device__ __forceinline__ void leaf_term(const SdParams& P, float3 q, int k, float& y, float& w, float3& v)
{
    float4 h = __ldg(&P.hdr[k]);
    if (KINDS == SD_HAS_PTS) { leaf_point(P, q, h, y, w, v); return; }
    int kind = (KINDS == SD_HAS_SEGS) ? SD_KIND_SEG : (KINDS == SD_HAS_TRIS) ? SD_KIND_TRI : (int)h.w;
    if ((KINDS & SD_HAS_PTS) && kind == SD_KIND_POINT) { leaf_point(P, q, h, y, w, v); return; }
    float4 x0 = __ldg(&P.ext[2 * k]);
    float4 x1 = __ldg(&P.ext[2 * k + 1]);
    if ((KINDS & SD_HAS_SEGS) && kind == SD_KIND_SEG) { leaf_segment<GRAD>(P, q, h, x0, x1, y, w, v); return; }
    leaf_triangle<GRAD>(P, q, h, x0, x1, y, w, v);
}

// ---------------------------------------------------------------------------
// host-side error helpers
// ---------------------------------------------------------------------------
void sd_set_last_error(const char* msg);
int sd_cuda_status(cudaError_t e);
void sd_count_launches(int k);

// allocation-free pieces of the query path (sd_query.cu), used by the
// batched multi-body path
namespace sdint {
size_t order_scratch_bytes(int m);
int order_into(const sd_tree* t, const float* q, int m, int32_t* order, void* scratch, cudaStream_t st);
int traverse(const sd_tree* t, const float* q, int m, const int* order, float* value, float* grad, int block,
             int* work, cudaStream_t st);
}
