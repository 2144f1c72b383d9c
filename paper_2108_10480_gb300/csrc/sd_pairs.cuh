// Closest points between simplices in fp32, for edge and triangle queries
// (Sec. 3.4: the distance between a data primitive f and a query primitive
// g is the simplex-simplex QP of App. B; its exact term is the point term at
// g's point of a closest pair). Everything is expressed relative to the data
// primitive's first vertex, so near pairs keep the precision of their
// separation rather than of their absolute coordinates.
//
// Building blocks (standard constructions, written here from their
// definitions): the point-segment projection; the point-triangle closest
// point by Voronoi regions; the segment-segment closest pair by clamped line
// parameters (Ericson, Real-Time Collision Detection, Sec. 5.1.9); the
// segment-triangle crossing by Moller-Trumbore barycentrics. A segment and a
// triangle that do not cross have a closest pair on the boundary: an
// endpoint against the triangle or the segment against an edge; two
// triangles that do not cross, a vertex against the other triangle or an
// edge against an edge. A crossing segment and triangle share one point;
// crossing triangles share a segment, represented by the mean of the points
// where an edge of one pierces the other.
#pragma once

#include "sd_common.cuh"

namespace sdpair {

// closest point to p on the segment from o along d
__device__ __forceinline__ float3 seg_point(float3 o, float3 d, float3 p)
{
    float dd = dot(d, d);
    float t = dd > 0.f ? fminf(fmaxf(dot(sub(p, o), d) / dd, 0.f), 1.f) : 0.f;
    return axpy(t, d, o);
}

// closest point to p on the triangle (o, o + e1, o + e2)
__device__ __forceinline__ float3 tri_point(float3 o, float3 e1, float3 e2, float3 p)
{
    float3 ap = sub(p, o);
    float g00 = dot(e1, e1), g11 = dot(e2, e2);
    float3 n = cross_k(e1, e2);
    if (!(dot(n, n) > 1e-10f * g00 * g11)) {
        // zero area: the closest of its three sides
        float3 c0 = seg_point(o, e1, p), c1 = seg_point(o, e2, p), c2 = seg_point(add(o, e1), sub(e2, e1), p);
        float l0 = dot(sub(p, c0), sub(p, c0)), l1 = dot(sub(p, c1), sub(p, c1)), l2 = dot(sub(p, c2), sub(p, c2));
        return (l0 <= l1 && l0 <= l2) ? c0 : (l1 <= l2 ? c1 : c2);
    }
    float d1 = dot(e1, ap), d2 = dot(e2, ap);
    if (d1 <= 0.f && d2 <= 0.f) return o;
    float d3 = d1 - g00, d4 = d2 - dot(e1, e2);
    if (d3 >= 0.f && d4 <= d3) return add(o, e1);
    float vc = sd_dop(d1, d4, d3, d2);
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) return axpy(d1 / (d1 - d3), e1, o);
    float d5 = d1 - dot(e1, e2), d6 = d2 - g11;
    if (d6 >= 0.f && d5 <= d6) return add(o, e2);
    float vb = sd_dop(d5, d2, d1, d6);
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) return axpy(d2 / (d2 - d6), e2, o);
    float va = sd_dop(d3, d6, d5, d4);
    if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
        float t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        return axpy(t, sub(e2, e1), add(o, e1));
    }
    float den = 1.f / (va + vb + vc);
    return add(o, axpy(vb * den, e1, scale(e2, vc * den)));
}

// closest pair of the segments p1 + s d1 and p2 + t d2 (s, t in [0, 1]);
// returns the squared distance
__device__ __forceinline__ float seg_seg(float3 p1, float3 d1, float3 p2, float3 d2, float3& c1, float3& c2)
{
    float3 r = sub(p1, p2);
    float a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
    float s = 0.f, t = 0.f;
    if (a <= 0.f && e <= 0.f) {
        s = t = 0.f;
    } else if (a <= 0.f) {
        t = fminf(fmaxf(f / e, 0.f), 1.f);
    } else {
        float c = dot(d1, r);
        if (e <= 0.f) {
            s = fminf(fmaxf(-c / a, 0.f), 1.f);
        } else {
            float b = dot(d1, d2);
            float den = sd_dop(a, e, b, b);
            s = den > 0.f ? fminf(fmaxf(sd_dop(b, f, c, e) / den, 0.f), 1.f) : 0.f;
            t = fmaf(b, s, f) / e;
            if (t < 0.f) {
                t = 0.f;
                s = fminf(fmaxf(-c / a, 0.f), 1.f);
            } else if (t > 1.f) {
                t = 1.f;
                s = fminf(fmaxf((b - c) / a, 0.f), 1.f);
            }
        }
    }
    c1 = axpy(s, d1, p1);
    c2 = axpy(t, d2, p2);
    float3 dd = sub(c1, c2);
    return dot(dd, dd);
}

// does the segment p + s d (s in [0, 1]) cross the triangle (o, o + e1,
// o + e2)? If so x is the crossing point.
__device__ __forceinline__ bool seg_tri_cross(float3 p, float3 d, float3 o, float3 e1, float3 e2, float3& x)
{
    float3 h = cross_k(d, e2);
    float det = dot(e1, h);
    float3 n = cross_k(e1, e2);
    float nd = sqrtf(dot(n, n) * dot(d, d));
    if (!(fabsf(det) > 1e-6f * nd)) return false;     // parallel (or degenerate): no crossing point
    float inv = 1.f / det;
    float3 sv = sub(p, o);
    float u = inv * dot(sv, h);
    if (u < 0.f || u > 1.f) return false;
    float3 qv = cross_k(sv, e1);
    float v = inv * dot(d, qv);
    if (v < 0.f || u + v > 1.f) return false;
    float t = inv * dot(e2, qv);
    if (t < 0.f || t > 1.f) return false;
    x = axpy(t, d, p);
    return true;
}

// closest pair of the segment p + s d and the triangle (o, o + e1, o + e2);
// cs on the segment, ct on the triangle; true if they cross (distance 0)
__device__ __forceinline__ bool seg_tri(float3 p, float3 d, float3 o, float3 e1, float3 e2, float3& cs, float3& ct)
{
    float3 x;
    if (seg_tri_cross(p, d, o, e1, e2, x)) {
        cs = ct = x;
        return true;
    }
    float best = INFINITY;
    float3 a, b;
    float l;
    l = seg_seg(p, d, o, e1, a, b);
    if (l < best) { best = l; cs = a; ct = b; }
    l = seg_seg(p, d, o, e2, a, b);
    if (l < best) { best = l; cs = a; ct = b; }
    l = seg_seg(p, d, add(o, e1), sub(e2, e1), a, b);
    if (l < best) { best = l; cs = a; ct = b; }
    b = tri_point(o, e1, e2, p);
    l = dot(sub(p, b), sub(p, b));
    if (l < best) { best = l; cs = p; ct = b; }
    a = add(p, d);
    b = tri_point(o, e1, e2, a);
    l = dot(sub(a, b), sub(a, b));
    if (l < best) { cs = a; ct = b; }
    return false;
}

// closest pair of triangles A (a, a + a1, a + a2) and B (b, b + b1, b + b2);
// ca on A, cb on B; true if they cross (distance 0)
__device__ __forceinline__ bool tri_tri(float3 a, float3 a1, float3 a2, float3 b, float3 b1, float3 b2, float3& ca,
                                        float3& cb)
{
    const float3 ao[3] = {a, a, add(a, a1)}, ad[3] = {a1, a2, sub(a2, a1)};
    const float3 bo[3] = {b, b, add(b, b1)}, bd[3] = {b1, b2, sub(b2, b1)};
    // crossing triangles meet along a segment whose ends are where an edge
    // of one pierces the other: the point used is the mean of those piercing
    // points (the segment's midpoint in general position)
    float3 x, sum = f3(0.f, 0.f, 0.f);
    int hits = 0;
    for (int i = 0; i < 3; ++i) {
        if (seg_tri_cross(ao[i], ad[i], b, b1, b2, x)) { sum = add(sum, x); ++hits; }
        if (seg_tri_cross(bo[i], bd[i], a, a1, a2, x)) { sum = add(sum, x); ++hits; }
    }
    if (hits) {
        ca = cb = scale(sum, 1.f / (float)hits);
        return true;
    }
    float best = INFINITY;
    float3 p, q;
    float l;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            l = seg_seg(ao[i], ad[i], bo[j], bd[j], p, q);
            if (l < best) { best = l; ca = p; cb = q; }
        }
    const float3 av[3] = {a, add(a, a1), add(a, a2)}, bv[3] = {b, add(b, b1), add(b, b2)};
    for (int i = 0; i < 3; ++i) {
        q = tri_point(b, b1, b2, av[i]);
        l = dot(sub(av[i], q), sub(av[i], q));
        if (l < best) { best = l; ca = av[i]; cb = q; }
        p = tri_point(a, a1, a2, bv[i]);
        l = dot(sub(bv[i], p), sub(bv[i], p));
        if (l < best) { best = l; ca = p; cb = bv[i]; }
    }
    return false;
}

}  // namespace sdpair

// Exact term of data primitive k for a query primitive with QK vertices g[]
// (absolute fp32 coordinates): the point term at g's point of a closest pair.
template <int KINDS, bool GRAD, int QK>
__device__ __forceinline__ void leaf_term_q(const SdParams& P, const float3* g, int k, float& y, float& w, float3& v)
{
    static_assert(QK == 2 || QK == 3, "edge or triangle queries");
    using namespace sdpair;
    float4 h = __ldg(&P.hdr[k]);
    const float3 a = f3(h.x, h.y, h.z);
    float3 r[QK];
#pragma unroll
    for (int i = 0; i < QK; ++i) r[i] = sub(g[i], a);
    const float3 o = f3(0.f, 0.f, 0.f);
    int kind = (KINDS == SD_HAS_PTS) ? SD_KIND_POINT : (KINDS == SD_HAS_SEGS) ? SD_KIND_SEG
             : (KINDS == SD_HAS_TRIS) ? SD_KIND_TRI : (int)h.w;
    if (kind == SD_KIND_POINT) {
        float3 pg = QK == 2 ? seg_point(r[0], sub(r[1], r[0]), o) : tri_point(r[0], sub(r[1], r[0]), sub(r[QK - 1], r[0]), o);
        leaf_point_rel(P, pg, y, w, v);
        return;
    }
    float4 x0 = __ldg(&P.ext[2 * k]);
    float4 x1 = __ldg(&P.ext[2 * k + 1]);
    // touch: the primitives cross, the pair's distance is 0 and its gradient
    // 0 (as for d = 0 in Eq. dgrad); the weight is taken at the crossing
    float3 pf, pg;
    bool touch = false;
    if ((KINDS & SD_HAS_SEGS) && kind == SD_KIND_SEG) {
        const float3 e = f3(x0.x, x0.y, x0.z);
        if (QK == 2) seg_seg(o, e, r[0], sub(r[1], r[0]), pf, pg);
        else touch = seg_tri(o, e, r[0], sub(r[1], r[0]), sub(r[QK - 1], r[0]), pf, pg);
        leaf_segment_rel<GRAD>(P, pg, x0, x1, y, w, v, touch);
        return;
    }
    const float3 e1 = f3(x0.x, x0.y, x0.z), e2 = f3(x1.x, x1.y, x1.z);
    if (QK == 2) touch = seg_tri(r[0], sub(r[1], r[0]), o, e1, e2, pg, pf);
    else touch = tri_tri(o, e1, e2, r[0], sub(r[1], r[0]), sub(r[QK - 1], r[0]), pf, pg);
    leaf_triangle_rel<GRAD>(P, pg, x0, x1, y, w, v, touch);
}
