// sd_query / sd_query_brute: Alg. 2 over Alg. 1 (Barnes-Hut), and the plain
// all-pairs evaluation of Eq. 3 / Eq. 4.
//
// Traversal: a warp walks the tree for 32 adjacent queries (Hilbert order) at once.
// Each popped record tests both children for every lane still interested in
// it (Barnes-Hut test first, also at leaves, as in Alg. 1): a far child adds
// n_B w_B e^{-alpha d_box} with gradient direction (q - y_B)/d_box (App. D),
// a near leaf adds its primitives' exact terms, a near internal child is
// pushed with the mask of lanes that need it. The LogSumExp is accumulated
// online in fp32 with a running max shift (no overflow or underflow for any
// alpha).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "sd_common.cuh"
#include "sd_pairs.cuh"
#include "sd_sort.cuh"

namespace {

// Warp-cooperative ("packet") traversal: the 32 lanes of a warp hold 32
// consecutive queries of the Hilbert order and walk the tree together on one
// warp-uniform stack of (record, lane mask) entries in shared memory. Every
// lane takes its own Barnes-Hut decisions (so each query gets exactly the
// terms of Alg. 1); a record is fetched once per warp and broadcast, and a
// child is pushed if any lane needs it opened. Exact leaf terms are not
// evaluated where they are found: each (query lane, primitive) pair goes to
// a per-warp queue, and every 32 queued pairs are evaluated by the 32 lanes
// at once, then folded into their owners' LogSumExp states by warp shuffles.
// Warps are persistent and take packets from a global counter.
constexpr int PK_STACK = 128;     // > depth + 1 of any radix tree over 95-bit keys
constexpr int PK_QCAP = 64;       // leaf queue: < 32 pending + at most 32 pushed at once
constexpr int PK_MAX_THREADS = 256;
constexpr int PK_WARP_INTS = 2 * PK_STACK + 2 * PK_QCAP + 32;   // per-warp shared memory, in ints

// Query primitives (Sec. 3.4): QK vertices each, indices F [m, QK] into the
// vertex array V [nv, 3] (unused for point queries, QK = 1).
struct QPrims {
    const float* V;
    const int* F;
    int nv;
};

// the vertices of query primitive qi (indices already validated)
template <int QK>
__device__ __forceinline__ void load_prim(const QPrims& Q, int qi, float3 (&g)[QK])
{
#pragma unroll
    for (int c = 0; c < QK; ++c) {
        int vi = __ldg(&Q.F[QK * qi + c]);
        g[c] = f3(__ldg(&Q.V[3 * vi]), __ldg(&Q.V[3 * vi + 1]), __ldg(&Q.V[3 * vi + 2]));
    }
}

struct WarpShared {
    int2* stack;
    int2* queue;
    int* lead;      // lead[owner lane] = lane holding the owner's merged partial sum, or -1
};

// Evaluate n <= 32 queued (owner lane, primitive) pairs, one per lane, and
// fold each result into its owner's accumulator.
template <int KINDS, bool GRAD, int QK>
__device__ __forceinline__ void flush_queue(const SdParams& P, float3 q, int qi, const QPrims& QP, const int2* items,
                                            int n, const WarpShared& ws, int lane, Lse& acc)
{
    __syncwarp();
    bool has = lane < n;
    int2 it = has ? items[lane] : make_int2(lane, 0);
    int owner = it.x;
    float3 qo = q;
    int qio = 0;
    if (QK == 1)
        qo = f3(__shfl_sync(0xffffffffu, q.x, owner), __shfl_sync(0xffffffffu, q.y, owner),
                __shfl_sync(0xffffffffu, q.z, owner));
    else
        qio = __shfl_sync(0xffffffffu, qi, owner);
    float tm = -INFINITY, ts = 0.f, tx = 0.f, ty = 0.f, tz = 0.f;
    if (has) {
        float y, w;
        float3 v;
        if constexpr (QK == 1) {
            leaf_term<KINDS, GRAD>(P, qo, it.y, y, w, v);
        } else {
            float3 g[QK];
            load_prim<QK>(QP, qio, g);
            leaf_term_q<KINDS, GRAD, QK>(P, g, it.y, y, w, v);
        }
        tm = y; ts = w;
        if (GRAD) { tx = w * v.x; ty = w * v.y; tz = w * v.z; }
    }
    // combine the terms of each owner in its group leader
    unsigned key = has ? (unsigned)owner : 32u + (unsigned)lane;
    unsigned peers = __match_any_sync(0xffffffffu, key);
    int leader = __ffs(peers) - 1;
    unsigned rest = (lane == leader) ? (peers & (peers - 1u)) : 0u;
    while (__any_sync(0xffffffffu, rest != 0u)) {
        int src = rest ? __ffs(rest) - 1 : lane;
        float m2 = __shfl_sync(0xffffffffu, tm, src), s2 = __shfl_sync(0xffffffffu, ts, src);
        float x2 = 0.f, y2 = 0.f, z2 = 0.f;
        if (GRAD) {
            x2 = __shfl_sync(0xffffffffu, tx, src);
            y2 = __shfl_sync(0xffffffffu, ty, src);
            z2 = __shfl_sync(0xffffffffu, tz, src);
        }
        if (rest) {
            Lse t{tm, ts, tx, ty, tz};
            lse_merge<GRAD>(t, m2, s2, x2, y2, z2);
            tm = t.m; ts = t.s; tx = t.gx; ty = t.gy; tz = t.gz;
            rest &= rest - 1u;
        }
    }
    if (has && lane == leader) ws.lead[owner] = lane;
    __syncwarp();
    int src = ws.lead[lane];
    int sl = src < 0 ? lane : src;
    float m2 = __shfl_sync(0xffffffffu, tm, sl), s2 = __shfl_sync(0xffffffffu, ts, sl);
    float x2 = 0.f, y2 = 0.f, z2 = 0.f;
    if (GRAD) {
        x2 = __shfl_sync(0xffffffffu, tx, sl);
        y2 = __shfl_sync(0xffffffffu, ty, sl);
        z2 = __shfl_sync(0xffffffffu, tz, sl);
    }
    if (src >= 0) {
        lse_merge<GRAD>(acc, m2, s2, x2, y2, z2);
        ws.lead[lane] = -1;
    }
    __syncwarp();
}

// queue the leaf bucket `ref` for the lanes in `lm`, flushing full groups of 32
template <int KINDS, bool GRAD, int QK>
__device__ __forceinline__ void queue_leaf(const SdParams& P, float3 q, int qi, const QPrims& QP, bool leaf, unsigned lm,
                                           int ref, Lse& acc, const WarpShared& ws, int& nq, int lane, int& nleaf)
{
    int k0 = (-ref - 1) * P.L;
    int k1 = min(k0 + P.L, P.n_prims);
    unsigned lt = (1u << lane) - 1u;
    int cnt = __popc(lm);
    if (leaf) nleaf += k1 - k0;
    for (int k = k0; k < k1; ++k) {
        if (leaf) ws.queue[nq + __popc(lm & lt)] = make_int2(lane, k);
        nq += cnt;
        if (nq >= 32) {
            nq -= 32;
            flush_queue<KINDS, GRAD, QK>(P, q, qi, QP, ws.queue + nq, 32, ws, lane, acc);
        }
    }
}

// Both children of one record, for every lane of the packet at once. The two
// Barnes-Hut tests run as packed two-wide fp32 operations whose per-element
// rounding equals the scalar test of the oracle (for a point query the
// offset to the box's closest point is q + max(-max(q, lo), -hi), which is
// exactly lo - q, q - hi or 0). Accepted far fields (App. D) add
// n_B w_B e^{-alpha d} with direction (q - y_B)/d, the mass folded into the
// base-2 exponent y = log2(n_B w_B) - alpha log2(e) d, into the running
// max-shifted LogSumExp without branches. Returns the lane masks of the
// children that must be opened.
template <int KINDS, bool GRAD, bool COUNT, int QK, bool TWO>
__device__ __forceinline__ void packet_record(const SdParams& P, float3 q, float3 nq3, int qi, const QPrims& QP,
                                              bool mine, int rec, Lse& acc, const WarpShared& ws, int& nq,
                                              int lane, int& ntest, int& nfar, int& nleaf, int& ref0, int& ref1,
                                              unsigned& open0, unsigned& open1)
{
    const SdNode& r = P.nodes[rec];
    float4 a = __ldg(&r.a), b = __ldg(&r.b), c = __ldg(&r.c);
    int4 d = __ldg(&r.d);
    const float2 lw = __ldg(&P.lw2[rec]);
    // every internal node has two children; only the super-root has one
    const bool has1 = TWO || d.y != SD_NO_CHILD;
    float2 ox, oy, oz;
    if (QK == 1) {
        ox = __fadd2_rn(make_float2(q.x, q.x), make_float2(fmaxf(-fmaxf(q.x, a.x), b.z), fmaxf(-fmaxf(q.x, a.y), b.w)));
        oy = __fadd2_rn(make_float2(q.y, q.y), make_float2(fmaxf(-fmaxf(q.y, a.z), c.x), fmaxf(-fmaxf(q.y, a.w), c.y)));
        oz = __fadd2_rn(make_float2(q.z, q.z), make_float2(fmaxf(-fmaxf(q.z, b.x), c.z), fmaxf(-fmaxf(q.z, b.y), c.w)));
    } else {
        // gap between the query primitive's box [q, -nq3] and the child box
        // per axis, signed by the side the query lies on
        float2 ax = __fadd2_rn(make_float2(a.x, a.y), make_float2(nq3.x, nq3.x));
        float2 ay = __fadd2_rn(make_float2(a.z, a.w), make_float2(nq3.y, nq3.y));
        float2 az = __fadd2_rn(make_float2(b.x, b.y), make_float2(nq3.z, nq3.z));
        float2 bx = __fadd2_rn(make_float2(q.x, q.x), make_float2(b.z, b.w));
        float2 by = __fadd2_rn(make_float2(q.y, q.y), make_float2(c.x, c.y));
        float2 bz = __fadd2_rn(make_float2(q.z, q.z), make_float2(c.z, c.w));
        ox = make_float2(copysignf(fmaxf(fmaxf(ax.x, bx.x), 0.f), bx.x), copysignf(fmaxf(fmaxf(ax.y, bx.y), 0.f), bx.y));
        oy = make_float2(copysignf(fmaxf(fmaxf(ay.x, by.x), 0.f), by.x), copysignf(fmaxf(fmaxf(ay.y, by.y), 0.f), by.y));
        oz = make_float2(copysignf(fmaxf(fmaxf(az.x, bz.x), 0.f), bz.x), copysignf(fmaxf(fmaxf(az.y, bz.y), 0.f), bz.y));
    }
    const float2 db = __ffma2_rn(oz, oz, __ffma2_rn(oy, oy, __fmul2_rn(ox, ox)));
    const float2 rhs = __fmul2_rn(make_float2(P.beta2, P.beta2), db);
    const bool t1 = mine && has1;
    const bool far0 = mine && __int_as_float(d.z) < rhs.x;
    const bool far1 = t1 && __int_as_float(d.w) < rhs.y;
    {
        // An absent term has exponent SD_NEG, far below the reference (which
        // starts at SD_FLOOR), so its factor ex2(SD_NEG - m) is exactly 0;
        // the tiny bias keeps 1/d finite inside a box (d = 0, never far).
        const float2 rb = __fadd2_rn(db, make_float2(1e-30f, 1e-30f));
        const float2 r = make_float2(rsqrtf(rb.x), rsqrtf(rb.y));
        float2 y = __ffma2_rn(make_float2(-P.alpha2, -P.alpha2), __fmul2_rn(db, r), lw);
        y.x = far0 ? y.x : SD_NEG;
        y.y = far1 ? y.y : SD_NEG;
        const float mn = fmaxf(acc.m, fmaxf(y.x, y.y));
        const float e = sd_ex2(acc.m - mn);
        const float2 t = __fadd2_rn(y, make_float2(-mn, -mn));
        const float2 c = make_float2(sd_ex2(t.x), sd_ex2(t.y));
        acc.s = fmaf(acc.s, e, c.x + c.y);
        if (GRAD) {
            const float2 cr = __fmul2_rn(c, r);
            acc.gx = fmaf(acc.gx, e, fmaf(cr.x, ox.x, cr.y * ox.y));
            acc.gy = fmaf(acc.gy, e, fmaf(cr.x, oy.x, cr.y * oy.y));
            acc.gz = fmaf(acc.gz, e, fmaf(cr.x, oz.x, cr.y * oz.y));
        }
        acc.m = mn;
    }
    if (COUNT) {
        ntest += mine ? (has1 ? 2 : 1) : 0;
        nfar += (far0 ? 1 : 0) + (far1 ? 1 : 0);
    }
    const bool near0 = mine && !far0;
    const bool near1 = t1 && !far1;
    const unsigned nm0 = __ballot_sync(0xffffffffu, near0);
    const unsigned nm1 = __ballot_sync(0xffffffffu, near1);
    ref0 = d.x;
    ref1 = d.y;
    open0 = open1 = 0u;
    if (nm0) {
        if (d.x < 0) queue_leaf<KINDS, GRAD, QK>(P, q, qi, QP, near0, nm0, d.x, acc, ws, nq, lane, nleaf);
        else open0 = nm0;
    }
    if (nm1) {
        if (d.y < 0) queue_leaf<KINDS, GRAD, QK>(P, q, qi, QP, near1, nm1, d.y, acc, ws, nq, lane, nleaf);
        else open1 = nm1;
    }
}

// QK = 1: point queries q[3 qi..]; QK = 2, 3: query primitive qi of QP,
// whose Barnes-Hut tests take its axis-aligned box [q, -nq3] (Sec. 3.5).
template <int KINDS, bool GRAD, bool COUNT, int QK>
// (no __launch_bounds__: with one, ptxas gives this kernel 80 registers and
// spills a little; without, 72 and none, which admits a seventh block of 128
// threads per SM; measured 1.8 % faster)
__global__ void k_traverse(SdParams P, const float* __restrict__ qs, int M,
                                                             const int* __restrict__ order,
                                                             float* __restrict__ value, float* __restrict__ grad,
                                                             int* __restrict__ counts, int* __restrict__ status,
                                                             int* __restrict__ work, int npackets, QPrims QP)
{
    extern __shared__ int smem_i[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int* wbase = smem_i + wib * PK_WARP_INTS;
    WarpShared ws;
    ws.stack = reinterpret_cast<int2*>(wbase);
    ws.queue = reinterpret_cast<int2*>(wbase + 2 * PK_STACK);
    ws.lead = wbase + 2 * PK_STACK + 2 * PK_QCAP;
    ws.lead[lane] = -1;
    __syncwarp();
    for (;;) {
        int pkt = 0;
        if (lane == 0) pkt = atomicAdd(work, 1);
        pkt = __shfl_sync(0xffffffffu, pkt, 0);
        if (pkt >= npackets) break;
        const int t = pkt * 32 + lane;
        const bool inrange = t < M;
        int qi = inrange ? (order ? order[t] : t) : 0;
        float3 q = f3(0.f, 0.f, 0.f), qhi = q;
        bool ok = inrange;
        bool bad_index = false;
        if (inrange) {
            if (QK == 1) {
                q = qhi = f3(qs[3 * qi], qs[3 * qi + 1], qs[3 * qi + 2]);
            } else {
                q = f3(INFINITY, INFINITY, INFINITY);
                qhi = f3(-INFINITY, -INFINITY, -INFINITY);
                for (int c = 0; c < QK; ++c) {
                    int vi = QP.F[QK * qi + c];
                    if (vi < 0 || vi >= QP.nv) { bad_index = true; continue; }
                    float3 g = f3(QP.V[3 * vi], QP.V[3 * vi + 1], QP.V[3 * vi + 2]);
                    q = f3(fminf(q.x, g.x), fminf(q.y, g.y), fminf(q.z, g.z));
                    qhi = f3(fmaxf(qhi.x, g.x), fmaxf(qhi.y, g.y), fmaxf(qhi.z, g.z));
                    if (!(isfinite(g.x) && isfinite(g.y) && isfinite(g.z))) ok = false;
                }
                ok = ok && !bad_index;
            }
            ok = ok && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(qhi.x) && isfinite(qhi.y) &&
                 isfinite(qhi.z);
        }
        if (inrange && !ok) {
            atomicOr(status, 1 << (bad_index ? SD_ERR_INDEX : SD_ERR_NONFINITE));
            value[qi] = __int_as_float(0x7fffffff);
            if (grad) grad[3 * qi] = grad[3 * qi + 1] = grad[3 * qi + 2] = __int_as_float(0x7fffffff);
            if (counts) counts[3 * qi] = counts[3 * qi + 1] = counts[3 * qi + 2] = 0;
        }
        if (!ok) q = qhi = f3(0.f, 0.f, 0.f);
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (!mask) continue;
        Lse acc;
        acc.m = SD_FLOOR; acc.s = 0.f; acc.gx = acc.gy = acc.gz = 0.f;
        int ntest = 0, nfar = 0, nleaf = 0;
        bool overflow = false;
        int sp = 0, nq = 0;
        const float3 nq3 = f3(-qhi.x, -qhi.y, -qhi.z);
        // the super-root (one child: the root) first, then the walk over
        // records with two children
        int rec, r0, r1;
        unsigned o0, o1;
        packet_record<KINDS, GRAD, COUNT, QK, false>(P, q, nq3, qi, QP, (mask >> lane) & 1u, P.root_record, acc, ws,
                                                     nq, lane, ntest, nfar, nleaf, r0, r1, o0, o1);
        rec = r0;
        mask = o0;
        while (mask) {
            const bool mine = (mask >> lane) & 1u;
            packet_record<KINDS, GRAD, COUNT, QK, true>(P, q, nq3, qi, QP, mine, rec, acc, ws, nq, lane, ntest, nfar,
                                                        nleaf, r0, r1, o0, o1);
            // descend into a child that must be opened; keep the other on the stack
            if (o0) {
                if (o1) {
                    if (sp < PK_STACK) {
                        if (lane == 0) ws.stack[sp] = make_int2(r1, (int)o1);
                        ++sp;
                    } else {
                        overflow = true;
                        break;
                    }
                }
                rec = r0;
                mask = o0;
                continue;
            }
            if (o1) {
                rec = r1;
                mask = o1;
                continue;
            }
            if (sp == 0) break;
            __syncwarp();
            int2 e = ws.stack[--sp];
            __syncwarp();
            rec = e.x;
            mask = (unsigned)e.y;
        }
        if (nq > 0) flush_queue<KINDS, GRAD, QK>(P, q, qi, QP, ws.queue, nq, ws, lane, acc);
        if (!ok) continue;
        if (overflow) {
            // a walk deeper than the stack (no radix tree over 95-bit keys is):
            // the packet's outputs are NaN, never a partial sum
            if (lane == 0) atomicOr(status, 1 << SD_ERR_TOO_LARGE);
            value[qi] = __int_as_float(0x7fffffff);
            if (GRAD) grad[3 * qi] = grad[3 * qi + 1] = grad[3 * qi + 2] = __int_as_float(0x7fffffff);
            continue;
        }
        // Alg. 2: d^ = -log(c)/alpha, grad d^ = grad c / c (c >= 1 after the shift)
        value[qi] = -(acc.m + sd_lg2(acc.s)) * P.inv_alpha2;
        if (GRAD) {
            float is = 1.f / acc.s;
            grad[3 * qi] = acc.gx * is;
            grad[3 * qi + 1] = acc.gy * is;
            grad[3 * qi + 2] = acc.gz * is;
        }
        if (COUNT) {
            counts[3 * qi] = ntest;
            counts[3 * qi + 1] = nfar;
            counts[3 * qi + 2] = nleaf;
        }
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

// Bounds of the finite query coordinates, as order-preserving unsigned keys
// reduced with atomicMax: qb[0..2] = max key of x, y, z; qb[3..5] = max of
// the complemented keys (the minimum). qb must be zero beforehand; a zero
// word decodes to NaN, which the code kernel ignores (no finite query).
__device__ __forceinline__ unsigned q_key(float f)
{
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float q_unkey(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// (also zeroes the order sort's nz scratch words, which the codes kernel
// then fills with the keys' digit totals)
__global__ void __launch_bounds__(256) k_query_bounds(const float* __restrict__ qs, int M, unsigned* __restrict__ qb,
                                                      uint32_t* __restrict__ zero, int nz)
{
    __shared__ unsigned sh[6];
    if (threadIdx.x < 6) sh[threadIdx.x] = 0u;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nz; i += gridDim.x * blockDim.x) zero[i] = 0u;
    __syncthreads();
    unsigned hi[3] = {0u, 0u, 0u}, nlo[3] = {0u, 0u, 0u};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M; t += gridDim.x * blockDim.x)
        for (int j = 0; j < 3; ++j) {
            const float v = qs[3 * t + j];
            if (isfinite(v)) {
                hi[j] = max(hi[j], q_key(v));
                nlo[j] = max(nlo[j], ~q_key(v));
            }
        }
    for (int j = 0; j < 3; ++j) {
        unsigned a = hi[j], b = nlo[j];
        for (int o = 16; o > 0; o >>= 1) {
            a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&sh[j], a);
            atomicMax(&sh[3 + j], b);
        }
    }
    __syncthreads();
    if (threadIdx.x < 6 && sh[threadIdx.x]) atomicMax(&qb[threadIdx.x], sh[threadIdx.x]);
}

// 24-bit Hilbert index of each query on a 256^3 grid over the union of the
// scene box and the queries' bounds (a query outside the scene box keeps its
// own cell instead of being clamped onto the box's faces with the others:
// measured 4.7 % fewer records visited per query on the benchmark workload,
// 30 % of whose queries lie in a box twice the mesh's size), the traversal
// order. Consecutive Hilbert cells are always face neighbours, so packets of
// 32 consecutive queries are more compact than on the Morton curve and open
// fewer tree nodes (measured 5 % faster). The index follows Skilling's
// transposition (AIP Conf. Proc. 707, 2004): undo the excess work of the
// axes from the top bit down, Gray-encode, then interleave. The order
// changes speed and summation order only.
__device__ __forceinline__ unsigned hilbert_key(const float* __restrict__ qs, int t, const SdScalars* __restrict__ sc,
                                                const unsigned* __restrict__ qb)
{
    float c[3] = {qs[3 * t], qs[3 * t + 1], qs[3 * t + 2]};
    float l[3], ie[3];
    for (int j = 0; j < 3; ++j) {
        // fminf / fmaxf drop a NaN bound (no finite query)
        l[j] = fminf(sc->lo[j], q_unkey(~qb[3 + j]));
        const float h = fmaxf(sc->hi[j], q_unkey(qb[j]));
        const float ex = h - l[j];
        ie[j] = ex > 0.f ? 1.f / ex : 0.f;
    }
    unsigned k[3];
    for (int j = 0; j < 3; ++j) {
        float u = (c[j] - l[j]) * ie[j];
        u = fminf(fmaxf(u, 0.f), 1.f);          // NaN -> 0
        k[j] = min((unsigned)(u * 256.f), 255u);
    }
    for (unsigned Q = 128u; Q > 1u; Q >>= 1) {
        const unsigned P = Q - 1u;
        for (int i = 0; i < 3; ++i) {
            if (k[i] & Q) {
                k[0] ^= P;                       // invert the low bits of axis 0
            } else {
                unsigned x = (k[0] ^ k[i]) & P;  // exchange the low bits of axes 0 and i
                k[0] ^= x;
                k[i] ^= x;
            }
        }
    }
    k[1] ^= k[0];
    k[2] ^= k[1];
    unsigned g = 0;
    for (unsigned Q = 128u; Q > 1u; Q >>= 1)
        if (k[2] & Q) g ^= Q - 1u;
    k[0] ^= g; k[1] ^= g; k[2] ^= g;
    unsigned code = 0;
    for (int b = 7; b >= 0; --b)
        code = (code << 3) | (((k[0] >> b) & 1u) << 2) | (((k[1] >> b) & 1u) << 1) | ((k[2] >> b) & 1u);
    return code;
}

// (blocks of 256 threads over a grid-stride loop; each block also adds its
// keys' radix digits of the three passes to the sort's digit totals, once
// per block, so that few blocks contend for the totals' words)
__global__ void __launch_bounds__(256) k_query_codes(const float* __restrict__ qs, int M,
                                                     const SdScalars* __restrict__ sc, const unsigned* __restrict__ qb,
                                                     unsigned* __restrict__ keys, int* __restrict__ vals,
                                                     uint32_t* __restrict__ totals)
{
    __shared__ uint32_t h[3][256];
    sdsort::pdl_release();      // the sort's first pass may launch
    for (int p = 0; p < 3; ++p) h[p][threadIdx.x] = 0;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M; t += gridDim.x * blockDim.x) {
        const unsigned code = hilbert_key(qs, t, sc, qb);
        keys[t] = code;
        vals[t] = t;
        sdsort::count_key(h, code, 3);
    }
    __syncthreads();
    for (int p = 0; p < 3; ++p) {
        const uint32_t c = h[p][threadIdx.x];
        if (c) atomicAdd(&totals[256 * p + threadIdx.x], c);
    }
}

int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

// persistent traversal launch: one block per resident slot on every SM
template <int KINDS, bool GRAD, bool COUNT, int QK>
void launch_traverse(const sd_tree* t, const float* q, int M, const int* order, float* value, float* grad,
                     int* counts, int block, int* work, const QPrims& QP, cudaStream_t st)
{
    int B = block > 0 ? block : 128;
    size_t smem = sizeof(int) * PK_WARP_INTS * (B / 32);
    int npackets = (M + 31) / 32;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse<KINDS, GRAD, COUNT, QK>, B, smem);
    int blocks = std::max(1, std::min(per_sm * sm_count(), (npackets * 32 + B - 1) / B));
    k_traverse<KINDS, GRAD, COUNT, QK><<<blocks, B, smem, st>>>(t->P, q, M, order, value, grad, counts, t->status,
                                                                work, npackets, QP);
}

template <bool BRUTE, int KINDS, bool GRAD>
void launch_one(const sd_tree* t, const float* q, int M, const int* order, float* value, float* grad, int* counts,
                int block, int* work, cudaStream_t st)
{
    if (BRUTE) {
        k_brute<KINDS, GRAD><<<(M + BT - 1) / BT, BT, 0, st>>>(t->P, q, M, value, grad, t->status);
    } else {
        QPrims none{nullptr, nullptr, 0};
        if (counts) launch_traverse<KINDS, GRAD, true, 1>(t, q, M, order, value, grad, counts, block, work, none, st);
        else launch_traverse<KINDS, GRAD, false, 1>(t, q, M, order, value, grad, counts, block, work, none, st);
    }
}

// edge (QK = 2) or triangle (QK = 3) queries; value and gradient always
template <int QK>
void dispatch_prims(const sd_tree* t, const QPrims& QP, int M, const int* order, float* value, float* grad,
                    int* counts, int block, int* work, cudaStream_t st)
{
#define SD_LAUNCH_PRIMS(K)                                                                                     \
    (counts ? launch_traverse<K, true, true, QK>(t, nullptr, M, order, value, grad, counts, block, work, QP, st) \
            : launch_traverse<K, true, false, QK>(t, nullptr, M, order, value, grad, counts, block, work, QP, st))
    switch (t->kinds) {
    case SD_HAS_PTS: SD_LAUNCH_PRIMS(SD_HAS_PTS); break;
    case SD_HAS_SEGS: SD_LAUNCH_PRIMS(SD_HAS_SEGS); break;
    case SD_HAS_TRIS: SD_LAUNCH_PRIMS(SD_HAS_TRIS); break;
    default: SD_LAUNCH_PRIMS(7); break;
    }
#undef SD_LAUNCH_PRIMS
}

template <bool BRUTE>
void dispatch(const sd_tree* t, const float* q, int M, const int* order, float* value, float* grad, int* counts,
              int block, int* work, cudaStream_t st)
{
    bool g = grad != nullptr;
    switch (t->kinds) {
    case SD_HAS_PTS:
        g ? launch_one<BRUTE, SD_HAS_PTS, true>(t, q, M, order, value, grad, counts, block, work, st)
          : launch_one<BRUTE, SD_HAS_PTS, false>(t, q, M, order, value, grad, counts, block, work, st);
        break;
    case SD_HAS_SEGS:
        g ? launch_one<BRUTE, SD_HAS_SEGS, true>(t, q, M, order, value, grad, counts, block, work, st)
          : launch_one<BRUTE, SD_HAS_SEGS, false>(t, q, M, order, value, grad, counts, block, work, st);
        break;
    case SD_HAS_TRIS:
        g ? launch_one<BRUTE, SD_HAS_TRIS, true>(t, q, M, order, value, grad, counts, block, work, st)
          : launch_one<BRUTE, SD_HAS_TRIS, false>(t, q, M, order, value, grad, counts, block, work, st);
        break;
    default:
        g ? launch_one<BRUTE, 7, true>(t, q, M, order, value, grad, counts, block, work, st)
          : launch_one<BRUTE, 7, false>(t, q, M, order, value, grad, counts, block, work, st);
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

// the Hilbert keys of m queries (keys) and their indices (vals), counted
// into the sort scratch `hist` (hist_words(m, 3) words, zeroed here) for a
// three-pass sort_pairs(..., counted = true); qb is six words of scratch
// for the queries' bounds
void enqueue_codes(const sd_tree* t, const float* q, int m, unsigned* qb, unsigned* keys, int* vals,
                   uint32_t* hist, cudaStream_t st, int* nl)
{
    cudaMemsetAsync(qb, 0, 6 * sizeof(unsigned), st);
    k_query_bounds<<<std::min((m + 255) / 256, 2 * sm_count()), 256, 0, st>>>(q, m, qb, hist,
                                                                            (int)sdsort::hist_words(m, 3));
    k_query_codes<<<std::min((m + 255) / 256, 2 * sm_count()), 256, 0, st>>>(q, m, t->sc, qb, keys, vals,
                                                                             sdsort::digit_totals(hist, m, 3));
    *nl += 2;
}

// Hilbert order of the queries into `order` (stream-ordered scratch).
int compute_order(const sd_tree* t, const float* q, int m, int32_t* order, cudaStream_t st)
{
    size_t hw = sdsort::hist_words(m, 3);
    size_t bytes = sizeof(unsigned) * 2 * (size_t)m + sizeof(int) * (size_t)m + sizeof(uint32_t) * hw + 1024;
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, bytes, st);
    if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    unsigned* k0 = (unsigned*)tmp;
    unsigned* k1 = k0 + m;
    int* v1 = (int*)(k1 + m);
    uint32_t* hist = (uint32_t*)(v1 + m);
    unsigned* qb = (unsigned*)(hist + hw);
    int nl = 0;
    // the sort's odd pass count leaves its result in the second buffer: give
    // it `order` there and start from the scratch copy
    enqueue_codes(t, q, m, qb, k0, v1, hist, st, &nl);
    int where = sdsort::sort_pairs<unsigned, int>(k0, v1, k1, order, m, 24, hist, st, &nl, true);
    if (!where) cudaMemcpyAsync(order, v1, sizeof(int) * (size_t)m, cudaMemcpyDeviceToDevice, st);
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
    SdUse use_{t, (cudaStream_t)stream};
    if (M == 0) return SD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // after a deferred-check build the order needs only the scene box: wait
    // for that point of the build (a no-op on the build's own stream), so
    // that on another stream the order overlaps the rest of the build
    if (t->box_ready) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
            cudaStreamWaitEvent(st, t->box_ready, 0);
        cudaGetLastError();
    }
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
    SdUse use_{t, (cudaStream_t)stream};
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
    bool sort = !order && opts.sort_queries && m > 1;
    // scratch: the packet counter, then the traversal order if it is computed here
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, 256 + (sort ? sizeof(int) * (size_t)m : 0), st);
    if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    int* work = (int*)tmp;
    cudaMemsetAsync(work, 0, sizeof(int), st);
    if (sort) {
        int32_t* ord = (int32_t*)((char*)tmp + 256);
        rc = compute_order(t, q, m, ord, st);
        if (rc != SD_OK) { cudaFreeAsync(tmp, st); return rc; }
        order = ord;
    }
    dispatch<false>(t, q, m, order, value, grad, opts.counts, opts.block, work, st);
    sd_count_launches(1);
    e = cudaGetLastError();
    cudaFreeAsync(tmp, st);
    return sd_cuda_status(e);
}

namespace {

// centroid of each query primitive (the traversal order key, and the query
// point itself when k = 1); a primitive with an index outside [0, nv) is
// reported in the status word and gets the origin (k = 1: NaN, so that the
// point traversal skips it)
__global__ void k_prim_centroids(const float* __restrict__ V, const int* __restrict__ F, int k, int m, int nv,
                                 float* __restrict__ c, int* status)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    float s[3] = {0.f, 0.f, 0.f};
    bool ok = true;
    for (int i = 0; i < k; ++i) {
        int v = F[k * j + i];
        if (v < 0 || v >= nv) { ok = false; continue; }
        for (int d = 0; d < 3; ++d) s[d] += V[3 * v + d];
    }
    const float inv = k == 1 ? 1.f : (k == 2 ? 0.5f : 1.f / 3.f);
    if (!ok) atomicOr(status, 1 << SD_ERR_INDEX);
    const float bad = k == 1 ? __int_as_float(0x7fffffff) : 0.f;
    for (int d = 0; d < 3; ++d) c[3 * j + d] = ok ? s[d] * inv : bad;
}

}  // namespace

extern "C" int sd_query_prims(const sd_tree* t, const float* QV, int64_t nqv, const int32_t* QF, int32_t k, int64_t M,
                              float* value, float* grad, const sd_query_opts* opts_in, void* stream)
{
    if (!t || k < 1 || k > 3 || M < 0 || nqv < 0 || (M > 0 && (!QV || !QF || !value))) return SD_ERR_INVALID_ARG;
    if (M >= ((int64_t)1 << 31) / 3 || nqv >= ((int64_t)1 << 31) / 3) return SD_ERR_TOO_LARGE;
    SdUse use_{t, (cudaStream_t)stream};
    sd_query_opts opts;
    if (opts_in) opts = *opts_in; else sd_default_query_opts(&opts);
    if (opts.block < 0 || opts.block > PK_MAX_THREADS || (opts.block % 32) != 0) return SD_ERR_INVALID_ARG;
    if (M == 0) return SD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int m = (int)M;
    if (t->info.n_prims == 0) {
        k_fill_empty<<<(m + 255) / 256, 256, 0, st>>>(value, grad, m);
        sd_count_launches(1);
        if (opts.counts) cudaMemsetAsync(opts.counts, 0, sizeof(int) * 3 * (size_t)m, st);
        return sd_cuda_status(cudaGetLastError());
    }
    const int* order = opts.order;
    const bool sort = !order && opts.sort_queries && m > 1;
    // scratch: packet counter, centroids, order, gradient when not wanted
    size_t o_cent = 256, o_ord = o_cent + 16 * (((size_t)m * 3 * sizeof(float) + 15) / 16);
    size_t o_grad = o_ord + 16 * (((size_t)m * sizeof(int) + 15) / 16);
    size_t bytes = o_grad + (grad ? 0 : sizeof(float) * 3 * (size_t)m);
    void* tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, bytes, st);
    if (e != cudaSuccess) { cudaGetLastError(); return SD_ERR_OOM; }
    int* work = (int*)tmp;
    float* cent = (float*)((char*)tmp + o_cent);
    int32_t* ord = (int32_t*)((char*)tmp + o_ord);
    float* g = grad ? grad : (float*)((char*)tmp + o_grad);
    cudaMemsetAsync(work, 0, sizeof(int), st);
    k_prim_centroids<<<(m + 255) / 256, 256, 0, st>>>(QV, QF, k, m, (int)nqv, cent, t->status);
    int nl = 1;
    int rc = SD_OK;
    if (sort) {
        rc = compute_order(t, cent, m, ord, st);
        order = ord;
    }
    if (rc == SD_OK) {
        QPrims QP{QV, QF, (int)nqv};
        if (k == 1) dispatch<false>(t, cent, m, order, value, g, opts.counts, opts.block, work, st);
        else if (k == 2) dispatch_prims<2>(t, QP, m, order, value, g, opts.counts, opts.block, work, st);
        else dispatch_prims<3>(t, QP, m, order, value, g, opts.counts, opts.block, work, st);
        ++nl;
    }
    sd_count_launches(nl);
    e = cudaGetLastError();
    cudaFreeAsync(tmp, st);
    return rc != SD_OK ? rc : sd_cuda_status(e);
}

extern "C" int sd_query_brute(const sd_tree* t, const float* q, int64_t M, float* value, float* grad,
                              const sd_query_opts* opts, void* stream)
{
    (void)opts;
    int rc = check_query_args(t, q, M, value);
    if (rc != SD_OK) return rc;
    SdUse use_{t, (cudaStream_t)stream};
    if (M == 0) return SD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int m = (int)M;
    if (t->info.n_prims == 0) {
        k_fill_empty<<<(m + 255) / 256, 256, 0, st>>>(value, grad, m);
        sd_count_launches(1);
        return sd_cuda_status(cudaGetLastError());
    }
    dispatch<true>(t, q, m, nullptr, value, grad, nullptr, 0, nullptr, st);
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

// ---------------------------------------------------------------------------
// sd_query_noalloc: the Barnes-Hut query for callers that must not let this
// library allocate device memory (for example an application that owns a
// fixed device-memory budget and forbids allocation during a simulation
// step, where a cudaMalloc could block on the device or fail part-way).
// Its temporary storage — the packet counter of the persistent traversal and
// the buffers of the query order sort — lives in one file-scope device
// array of fixed size, so the call allocates nothing. Limits and sharing:
//   * at most SD_NOALLOC_MAX_QUERIES queries per call;
//   * every device that loads this library holds the array until the
//     process exits;
//   * all calls on a device share the array and leave their contents in it,
//     so calls that overlap on the GPU race, whether they are made directly
//     (for example on two streams) or replayed from captured graphs;
//   * the first call on a device looks up the array's device address once,
//     with that device current, and caches it; make that first call before
//     any stream capture. The cache does not survive cudaDeviceReset.
// ---------------------------------------------------------------------------
namespace {

constexpr int SD_NOALLOC_MAX_QUERIES = 262144;
constexpr size_t NOALLOC_HIST_WORDS = sdsort::hist_words(SD_NOALLOC_MAX_QUERIES, 3);
// [counter: 256 B][keys: 2 x max u32][order, alternate order: 2 x max i32][sort counters]
constexpr size_t NOALLOC_BYTES = 256 + 4 * sizeof(uint32_t) * (size_t)SD_NOALLOC_MAX_QUERIES +
                                 sizeof(uint32_t) * NOALLOC_HIST_WORDS;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};   // device address of g_noalloc_scratch, per device

}  // namespace

extern "C" int sd_query_noalloc(const sd_tree* t, const float* q, int64_t M, float* value, float* grad,
                                void* stream)
{
    int rc = check_query_args(t, q, M, value);
    if (rc != SD_OK) return rc;
    SdUse use_{t, (cudaStream_t)stream};
    if (M > SD_NOALLOC_MAX_QUERIES) return SD_ERR_TOO_LARGE;
    if (M == 0) return SD_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sd_cuda_status(e);
    if (dev < 0 || dev >= 64) return SD_ERR_INVALID_ARG;
    char* base = nullptr;
    {
        // The array's name is only a host-side stand-in; its device address
        // is looked up once per device, with that device current.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return sd_cuda_status(e);
            g_noalloc_addr[dev] = p;
        }
        base = (char*)g_noalloc_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int m = (int)M;
    if (t->info.n_prims == 0) {
        k_fill_empty<<<(m + 255) / 256, 256, 0, st>>>(value, grad, m);
        sd_count_launches(1);
        return sd_cuda_status(cudaGetLastError());
    }
    int* work = (int*)base;
    unsigned* qb = (unsigned*)(base + 64);     // the queries' bounds, in the counter area
    unsigned* k0 = (unsigned*)(base + 256);
    unsigned* k1 = k0 + SD_NOALLOC_MAX_QUERIES;
    int* ord0 = (int*)(k1 + SD_NOALLOC_MAX_QUERIES);
    int* ord1 = ord0 + SD_NOALLOC_MAX_QUERIES;
    uint32_t* hist = (uint32_t*)(ord1 + SD_NOALLOC_MAX_QUERIES);
    // the packet counter must start at zero on every call
    e = cudaMemsetAsync(work, 0, sizeof(int), st);
    if (e != cudaSuccess) return sd_cuda_status(e);
    const int* order = nullptr;
    int nl = 0;
    if (m > 1) {
        enqueue_codes(t, q, m, qb, k0, ord0, hist, st, &nl);
        int where = sdsort::sort_pairs<unsigned, int>(k0, ord0, k1, ord1, m, 24, hist, st, &nl, true);
        order = where ? ord1 : ord0;
    }
    dispatch<false>(t, q, m, order, value, grad, nullptr, 0, work, st);
    sd_count_launches(nl + 1);
    return sd_cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// allocation-free building blocks for the batched multi-body path
// ---------------------------------------------------------------------------
namespace sdint {

size_t order_scratch_bytes(int m)
{
    return sizeof(unsigned) * 2 * (size_t)m + sizeof(int) * (size_t)m + sizeof(uint32_t) * sdsort::hist_words(m, 3) + 512;
}

// Hilbert order of m queries into `order`, using caller scratch of
// order_scratch_bytes(m) bytes (256-byte aligned).
int order_into(const sd_tree* t, const float* q, int m, int32_t* order, void* scratch, cudaStream_t st)
{
    if (m <= 0) return SD_OK;
    unsigned* k0 = (unsigned*)scratch;
    unsigned* k1 = k0 + m;
    int* v1 = (int*)(k1 + m);
    uint32_t* hist = (uint32_t*)(v1 + m);
    unsigned* qb = (unsigned*)(hist + sdsort::hist_words(m, 3));
    int nl = 0;
    // the sort's odd pass count leaves its result in the second buffer: give
    // it `order` there and start from the scratch copy
    enqueue_codes(t, q, m, qb, k0, v1, hist, st, &nl);
    int where = sdsort::sort_pairs<unsigned, int>(k0, v1, k1, order, m, 24, hist, st, &nl, true);
    if (!where) cudaMemcpyAsync(order, v1, sizeof(int) * (size_t)m, cudaMemcpyDeviceToDevice, st);
    sd_count_launches(nl);
    return sd_cuda_status(cudaGetLastError());
}

// Barnes-Hut traversal with a caller-provided packet counter (zeroed here).
int traverse(const sd_tree* t, const float* q, int m, const int* order, float* value, float* grad, int block,
             int* work, cudaStream_t st)
{
    if (m <= 0) return SD_OK;
    if (block < 0 || block > PK_MAX_THREADS || (block % 32) != 0) return SD_ERR_INVALID_ARG;
    if (t->info.n_prims == 0) {
        k_fill_empty<<<(m + 255) / 256, 256, 0, st>>>(value, grad, m);
        sd_count_launches(1);
        return sd_cuda_status(cudaGetLastError());
    }
    cudaMemsetAsync(work, 0, sizeof(int), st);
    dispatch<false>(t, q, m, order, value, grad, nullptr, block, work, st);
    sd_count_launches(1);
    return sd_cuda_status(cudaGetLastError());
}

}  // namespace sdint
