/*
 * Smooth-distance oracle: a plain, slow FP64 CPU reference.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg load this library; the CUDA library shares no code with
 * it and never links it.
 *
 * What it computes (Madan & Levin, "Fast Evaluation of Smooth Distance
 * Constraints on Co-Dimensional Geometry"):
 *   - exact point/segment/triangle distances and closest-point barycentrics
 *     (App. B, Eq. distsq / dgrad);
 *   - the blending weights w_i = (A w~_i)^S with the App. C polynomials (the
 *     coefficient bases are solved in numpy and passed in) and the gradient
 *     chain rule of Eq. dw_new, attenuation S = alpha / max(alpha, alpha_U)
 *     (Sec. 3.3);
 *   - the LogSumExp smooth distance and its gradient (Eq. 3 / Eq. 4) by brute
 *     force over all primitives, evaluated in shifted form
 *     t_i = ln w_i - alpha d_i, m = max t_i;
 *   - the conservative Barnes-Hut evaluation of Alg. 1 / Alg. 2 with the far
 *     field of App. D (expansion centre = closest point of the node's AABB),
 *     on a binary radix tree over Morton codes that this file builds itself
 *     (top-down split at the highest differing key bit).
 *
 * Readings of the paper that this file takes (each listed in the design
 * notes): epsilon of Alg. 2 is 0 (the shifted sum is >= 1); incidence counts
 * are per slot; isolated triangles (v_i = 1) use w~ = 1; w~ is clamped to at
 * least 1e-6; far-field weight of a node is 1 if it holds only points, else
 * max(A_E, A_T)^S; the Barnes-Hut test is applied before the leaf test.
 *
 * Compile: gcc -O2 -ffp-contract=off -fPIC -shared -pthread sd_oracle.c -lm
 * (no FMA contraction: the FP32 Morton codes and FP32 Barnes-Hut decisions
 * below must be the exact IEEE results of the written operation order).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { K_POINT = 0, K_SEG = 1, K_TRI = 2 };

typedef struct {
    int kind;
    int64_t v[3];      /* indices into the scene's combined vertex array */
    double pa, pb;     /* segment: u, v = 1/|N_i0|, 1/|N_i1|; triangle: 1/v_i, 1/e_i */
    int isolated;      /* triangle whose largest vertex valence is 1 */
} prim_t;

typedef struct {
    int64_t nv;
    double *V;         /* combined vertices (points, edge-mesh V, triangle-mesh V), FP64 */
    float *Vf;         /* the same vertices as given (fp32) */
    int64_t n, np, ne, nt;
    prim_t *P;
    double A_E, A_T;
    double ebasis[5][3];
    double tbasis[36][3];
    int texp[36][2];
    /* tree */
    int L;
    int64_t nb;
    uint64_t *codes;   /* Morton code per primitive, original order */
    int64_t *sorted;   /* primitive index in sorted order */
    int32_t *left, *right;      /* internal nodes (nb-1); leaf child = -(bucket+1) */
    float (*nlo)[3], (*nhi)[3]; /* internal node AABBs */
    int64_t *ncount;
    int *npts_only;
    float (*llo)[3], (*lhi)[3]; /* leaf (bucket) AABBs */
    int64_t *lcount;
    int *lpts_only;
    float slo[3], shi[3];       /* scene AABB */
} scene_t;

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                     */
/* ------------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(double *o, const double *a, const double *b) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }

/* ------------------------------------------------------------------------ */
/* scene construction: primitives, incidence counts (valences)              */
/* ------------------------------------------------------------------------ */
static int cmp_u64pair(const void *a, const void *b)
{
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    return (x[0] < y[0]) ? -1 : (x[0] > y[0]) ? 1 : 0;
}

void *orc_scene_new(const float *pts, int64_t np,
                    const float *ev, int64_t nev, const int32_t *E, int64_t ne,
                    const float *tv, int64_t ntv, const int32_t *F, int64_t nf,
                    const double *ebasis15, const double *tbasis108)
{
    scene_t *s = (scene_t *)calloc(1, sizeof(scene_t));
    s->np = np; s->ne = ne; s->nt = nf;
    s->n = np + ne + nf;
    s->nv = np + nev + ntv;
    s->V = (double *)malloc(sizeof(double) * 3 * (s->nv ? s->nv : 1));
    s->Vf = (float *)malloc(sizeof(float) * 3 * (s->nv ? s->nv : 1));
    for (int64_t i = 0; i < np * 3; ++i) { s->Vf[i] = pts[i]; }
    for (int64_t i = 0; i < nev * 3; ++i) { s->Vf[np * 3 + i] = ev[i]; }
    for (int64_t i = 0; i < ntv * 3; ++i) { s->Vf[(np + nev) * 3 + i] = tv[i]; }
    for (int64_t i = 0; i < s->nv * 3; ++i) s->V[i] = (double)s->Vf[i];
    memcpy(s->ebasis, ebasis15, sizeof(s->ebasis));
    memcpy(s->tbasis, tbasis108, sizeof(s->tbasis));
    {
        int j = 0;
        for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b)
                if (a + b <= 7) { s->texp[j][0] = a; s->texp[j][1] = b; ++j; }
    }
    s->P = (prim_t *)calloc((size_t)(s->n ? s->n : 1), sizeof(prim_t));
    int64_t k = 0;
    for (int64_t i = 0; i < np; ++i, ++k) {
        s->P[k].kind = K_POINT; s->P[k].v[0] = i;
    }
    /* edge mesh: |N_k| = number of edge slots that reference vertex k */
    s->A_E = 1.0;
    if (ne > 0) {
        int64_t *cnt = (int64_t *)calloc((size_t)nev, sizeof(int64_t));
        for (int64_t i = 0; i < ne; ++i) { cnt[E[2 * i]]++; cnt[E[2 * i + 1]]++; }
        int64_t amax = 0;
        for (int64_t i = 0; i < nev; ++i) if (cnt[i] > amax) amax = cnt[i];
        s->A_E = (double)amax;
        for (int64_t i = 0; i < ne; ++i, ++k) {
            s->P[k].kind = K_SEG;
            s->P[k].v[0] = np + E[2 * i];
            s->P[k].v[1] = np + E[2 * i + 1];
            s->P[k].pa = 1.0 / (double)cnt[E[2 * i]];
            s->P[k].pb = 1.0 / (double)cnt[E[2 * i + 1]];
        }
        free(cnt);
    }
    /* triangle mesh: vertex valence = triangle slots referencing the vertex;
       edge valence = triangle edge slots with the same unordered vertex pair */
    s->A_T = 1.0;
    if (nf > 0) {
        int64_t *vc = (int64_t *)calloc((size_t)ntv, sizeof(int64_t));
        for (int64_t i = 0; i < nf * 3; ++i) vc[F[i]]++;
        uint64_t *ek = (uint64_t *)malloc(sizeof(uint64_t) * 2 * 3 * nf);
        for (int64_t i = 0; i < nf; ++i)
            for (int j = 0; j < 3; ++j) {
                uint64_t a = (uint64_t)F[3 * i + j], b = (uint64_t)F[3 * i + (j + 1) % 3];
                uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
                ek[2 * (3 * i + j)] = (lo << 32) | hi;
                ek[2 * (3 * i + j) + 1] = (uint64_t)(3 * i + j);
            }
        qsort(ek, (size_t)(3 * nf), 2 * sizeof(uint64_t), cmp_u64pair);
        int64_t *ecnt = (int64_t *)malloc(sizeof(int64_t) * 3 * nf);
        for (int64_t i = 0; i < 3 * nf;) {
            int64_t j = i;
            while (j < 3 * nf && ek[2 * j] == ek[2 * i]) ++j;
            for (int64_t t = i; t < j; ++t) ecnt[ek[2 * t + 1]] = j - i;
            i = j;
        }
        int64_t amax = 0;
        for (int64_t i = 0; i < nf; ++i, ++k) {
            int64_t vmax = 0, emax = 0;
            for (int j = 0; j < 3; ++j) {
                if (vc[F[3 * i + j]] > vmax) vmax = vc[F[3 * i + j]];
                if (ecnt[3 * i + j] > emax) emax = ecnt[3 * i + j];
            }
            if (vmax > amax) amax = vmax;
            s->P[k].kind = K_TRI;
            for (int j = 0; j < 3; ++j) s->P[k].v[j] = np + nev + F[3 * i + j];
            s->P[k].pa = 1.0 / (double)vmax;
            s->P[k].pb = 1.0 / (double)emax;
            s->P[k].isolated = (vmax == 1);
        }
        s->A_T = (double)amax;
        free(vc); free(ek); free(ecnt);
    }
    return s;
}

static void tree_free(scene_t *s)
{
    free(s->codes); free(s->sorted); free(s->left); free(s->right);
    free(s->nlo); free(s->nhi); free(s->ncount); free(s->npts_only);
    free(s->llo); free(s->lhi); free(s->lcount); free(s->lpts_only);
    s->codes = NULL; s->sorted = NULL; s->left = s->right = NULL;
    s->nlo = s->nhi = NULL; s->ncount = NULL; s->npts_only = NULL;
    s->llo = s->lhi = NULL; s->lcount = NULL; s->lpts_only = NULL;
    s->nb = 0;
}

void orc_scene_free(void *h)
{
    scene_t *s = (scene_t *)h;
    if (!s) return;
    tree_free(s);
    free(s->V); free(s->Vf); free(s->P); free(s);
}

void orc_scene_info(void *h, double *out)
{
    scene_t *s = (scene_t *)h;
    out[0] = s->A_E; out[1] = s->A_T;
    out[2] = (double)s->n; out[3] = (double)s->np; out[4] = (double)s->ne; out[5] = (double)s->nt;
}

void orc_prim_params(void *h, double *out, int32_t *kind, int32_t *iso)
{
    scene_t *s = (scene_t *)h;
    for (int64_t i = 0; i < s->n; ++i) {
        out[2 * i] = s->P[i].pa; out[2 * i + 1] = s->P[i].pb;
        kind[i] = s->P[i].kind; iso[i] = s->P[i].isolated;
    }
}

/* ------------------------------------------------------------------------ */
/* exact distances (App. B)                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    double d;          /* distance */
    double gd[3];      /* gradient of d w.r.t. q (Eq. dgrad), 0 when d == 0 */
    double phi[2];     /* barycentric coordinates of the closest point */
    double gphi[2][3]; /* gradients of phi w.r.t. q */
    int degenerate;    /* zero-area triangle: weight gradient forced to 0 */
} near_t;

/* closest point of segment a + t e, t in [0, 1]; returns t and whether the
   unconstrained parameter was clamped (then dt/dq = 0) */
static double seg_param(const double *a, const double *e, const double *q, int *clamped)
{
    double ee = dot3(e, e);
    if (ee == 0.0) { *clamped = 1; return 0.0; }
    double ap[3]; sub3(ap, q, a);
    double t = dot3(ap, e) / ee;
    if (t <= 0.0) { *clamped = 1; return 0.0; }
    if (t >= 1.0) { *clamped = 1; return 1.0; }
    *clamped = 0;
    return t;
}

static void finish_dist(near_t *r, const double *q, const double *pi)
{
    double dv[3]; sub3(dv, q, pi);
    r->d = sqrt(dot3(dv, dv));
    for (int j = 0; j < 3; ++j) r->gd[j] = r->d > 0.0 ? dv[j] / r->d : 0.0;
}

static void near_point(const double *p, const double *q, near_t *r)
{
    memset(r, 0, sizeof(*r));
    finish_dist(r, q, p);
}

static void near_segment(const double *a, const double *b, const double *q, near_t *r)
{
    memset(r, 0, sizeof(*r));
    double e[3]; sub3(e, b, a);
    int cl;
    double t = seg_param(a, e, q, &cl);
    double pi[3] = {a[0] + t * e[0], a[1] + t * e[1], a[2] + t * e[2]};
    r->phi[0] = t;
    if (!cl) {
        double ee = dot3(e, e);
        for (int j = 0; j < 3; ++j) r->gphi[0][j] = e[j] / ee;
    }
    finish_dist(r, q, pi);
}

/* Point-triangle distance as the QP of Eq. distsq over the simplex
   f(phi) = (1 - phi1 - phi2) v0 + phi1 v1 + phi2 v2: the unconstrained
   minimiser (2x2 normal equations) if it lies in the triangle, otherwise the
   best of the three boundary segments (the minimiser of a convex QP that is
   not interior lies on the boundary). */
static void near_triangle(const double *v0, const double *v1, const double *v2, const double *q, near_t *r)
{
    memset(r, 0, sizeof(*r));
    double e1[3], e2[3], ap[3];
    sub3(e1, v1, v0); sub3(e2, v2, v0); sub3(ap, q, v0);
    double g00 = dot3(e1, e1), g01 = dot3(e1, e2), g11 = dot3(e2, e2);
    double det = g00 * g11 - g01 * g01;
    double scale = g00 * g11;
    /* sin^2 of the corner angle below 1e-10 counts as zero area */
    int degenerate = !(det > 1e-10 * scale) || scale == 0.0;
    if (!degenerate) {
        double r0 = dot3(ap, e1), r1 = dot3(ap, e2);
        double p1 = (g11 * r0 - g01 * r1) / det;
        double p2 = (g00 * r1 - g01 * r0) / det;
        if (p1 >= 0.0 && p2 >= 0.0 && p1 + p2 <= 1.0) {
            double pi[3];
            for (int j = 0; j < 3; ++j) pi[j] = v0[j] + p1 * e1[j] + p2 * e2[j];
            r->phi[0] = p1; r->phi[1] = p2;
            for (int j = 0; j < 3; ++j) {
                r->gphi[0][j] = (g11 * e1[j] - g01 * e2[j]) / det;
                r->gphi[1][j] = (g00 * e2[j] - g01 * e1[j]) / det;
            }
            finish_dist(r, q, pi);
            return;
        }
    }
    /* boundary: edges v0v1 (phi = (t, 0)), v1v2 (phi = (1 - t, t)), v0v2 (phi = (0, t)) */
    near_t best; best.d = INFINITY;
    for (int k = 0; k < 3; ++k) {
        const double *a = k == 0 ? v0 : (k == 1 ? v1 : v0);
        const double *b = k == 0 ? v1 : (k == 1 ? v2 : v2);
        near_t c;
        memset(&c, 0, sizeof(c));
        double e[3]; sub3(e, b, a);
        int cl;
        double t = seg_param(a, e, q, &cl);
        double pi[3] = {a[0] + t * e[0], a[1] + t * e[1], a[2] + t * e[2]};
        finish_dist(&c, q, pi);
        double ee = dot3(e, e);
        double gt[3] = {0, 0, 0};
        if (!cl) for (int j = 0; j < 3; ++j) gt[j] = e[j] / ee;
        if (k == 0) { c.phi[0] = t; c.phi[1] = 0.0; for (int j = 0; j < 3; ++j) c.gphi[0][j] = gt[j]; }
        if (k == 1) { c.phi[0] = 1.0 - t; c.phi[1] = t; for (int j = 0; j < 3; ++j) { c.gphi[0][j] = -gt[j]; c.gphi[1][j] = gt[j]; } }
        if (k == 2) { c.phi[0] = 0.0; c.phi[1] = t; for (int j = 0; j < 3; ++j) c.gphi[1][j] = gt[j]; }
        if (c.d < best.d) best = c;
    }
    *r = best;
    r->degenerate = degenerate;
}

/* ------------------------------------------------------------------------ */
/* weights (Sec. 3.3, App. C)                                               */
/* ------------------------------------------------------------------------ */
#define W_MIN 1e-6

/* w~ and dw~/dphi for a primitive at barycentrics phi */
static void weight_tilde(const scene_t *s, const prim_t *p, const double *phi, double *wt, double *dw)
{
    dw[0] = dw[1] = 0.0;
    if (p->kind == K_SEG) {
        double c[5];
        for (int k = 0; k < 5; ++k) c[k] = s->ebasis[k][0] * p->pa + s->ebasis[k][1] * p->pb + s->ebasis[k][2];
        double x = phi[0], w = 0.0, d = 0.0;
        for (int k = 0; k < 5; ++k) w += c[k] * pow(x, k);
        for (int k = 1; k < 5; ++k) d += k * c[k] * pow(x, k - 1);
        *wt = w; dw[0] = d;
    } else if (p->kind == K_TRI) {
        if (p->isolated) { *wt = 1.0; return; }
        double x = phi[0], y = phi[1], w = 0.0, d1 = 0.0, d2 = 0.0;
        double rhs[3] = {p->pa, p->pb, 1.0 - p->pa};
        for (int j = 0; j < 36; ++j) {
            double c = s->tbasis[j][0] * rhs[0] + s->tbasis[j][1] * rhs[1] + s->tbasis[j][2] * rhs[2];
            int a = s->texp[j][0], b = s->texp[j][1];
            w += c * pow(x, a) * pow(y, b);
            if (a > 0) d1 += c * a * pow(x, a - 1) * pow(y, b);
            if (b > 0) d2 += c * b * pow(x, a) * pow(y, b - 1);
        }
        *wt = w; dw[0] = d1; dw[1] = d2;
    } else {
        *wt = 1.0;
    }
    if (*wt < W_MIN) { *wt = W_MIN; dw[0] = dw[1] = 0.0; }
}

/* One exact contribution: t = ln w - alpha d and the vector
   grad d - (1/alpha) grad(w) / w  (so that the numerator of Eq. 4 is
   sum_i w_i e^{-alpha d_i} * vector_i). */
typedef struct { double t; double v[3]; } term_t;

typedef struct {
    double alpha, S;
    int paper_metric;
    int unit;          /* unit weights: w_i = 1 for every primitive */
} params_t;

static void prim_near(const scene_t *s, const prim_t *p, const double *q, near_t *nr)
{
    const double *V = s->V;
    if (p->kind == K_POINT) near_point(V + 3 * p->v[0], q, nr);
    else if (p->kind == K_SEG) near_segment(V + 3 * p->v[0], V + 3 * p->v[1], q, nr);
    else near_triangle(V + 3 * p->v[0], V + 3 * p->v[1], V + 3 * p->v[2], q, nr);
}

static term_t prim_term(const scene_t *s, const prim_t *p, const double *q, const params_t *pr,
                        near_t *nr_out, double *wt_out, double *gwt_out)
{
    near_t nr;
    prim_near(s, p, q, &nr);
    term_t T;
    double wt = 1.0, dw[2] = {0, 0}, gwt[3] = {0, 0, 0};
    if (p->kind != K_POINT) {
        weight_tilde(s, p, nr.phi, &wt, dw);
        if (!nr.degenerate)
            for (int j = 0; j < 3; ++j) gwt[j] = dw[0] * nr.gphi[0][j] + dw[1] * nr.gphi[1][j];
        if (pr->paper_metric)
            for (int j = 0; j < 3; ++j) gwt[j] /= pr->alpha;
    }
    if (p->kind == K_POINT || pr->unit) {
        T.t = -pr->alpha * nr.d;
        for (int j = 0; j < 3; ++j) T.v[j] = nr.gd[j];
    } else {
        double A = p->kind == K_SEG ? s->A_E : s->A_T;
        double lw = pr->S * log(A * wt);
        T.t = lw - pr->alpha * nr.d;
        for (int j = 0; j < 3; ++j) T.v[j] = nr.gd[j] - (pr->S * gwt[j] / wt) / pr->alpha;
    }
    if (nr_out) *nr_out = nr;
    if (wt_out) *wt_out = wt;
    if (gwt_out) for (int j = 0; j < 3; ++j) gwt_out[j] = gwt[j];
    return T;
}

/* out: d, gd[3], phi[2], wt, gwt[3], t, v[3]  (14 doubles) */
void orc_prim_eval(void *h, int64_t i, double alpha, double alpha_u, int paper_metric,
                   const double *q, double *out)
{
    scene_t *s = (scene_t *)h;
    params_t pr = {alpha, alpha / (alpha > alpha_u ? alpha : alpha_u), paper_metric, 0};
    near_t nr; double wt, gwt[3];
    term_t T = prim_term(s, &s->P[i], q, &pr, &nr, &wt, gwt);
    out[0] = nr.d;
    for (int j = 0; j < 3; ++j) out[1 + j] = nr.gd[j];
    out[4] = nr.phi[0]; out[5] = nr.phi[1];
    out[6] = wt;
    for (int j = 0; j < 3; ++j) out[7 + j] = gwt[j];
    out[10] = T.t;
    for (int j = 0; j < 3; ++j) out[11 + j] = T.v[j];
}

/* LogSumExp of Eq. 3 / Eq. 4 over a list of terms (shifted by the max) */
static void lse_finish(const term_t *T, int64_t n, double alpha, double *val, double *grad)
{
    if (n == 0) { *val = INFINITY; grad[0] = grad[1] = grad[2] = 0.0; return; }
    double m = -INFINITY;
    for (int64_t i = 0; i < n; ++i) if (T[i].t > m) m = T[i].t;
    double sum = 0.0, g[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double e = exp(T[i].t - m);
        sum += e;
        for (int j = 0; j < 3; ++j) g[j] += e * T[i].v[j];
    }
    *val = -(m + log(sum)) / alpha;
    for (int j = 0; j < 3; ++j) grad[j] = g[j] / sum;
}

/* ------------------------------------------------------------------------ */
/* thread pool over queries                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    void (*fn)(void *ctx, int64_t i, void *scratch);
    void *ctx;
    int64_t m, next;
    size_t scratch_bytes;
    pthread_mutex_t mu;
} pool_t;

static void *pool_worker(void *arg)
{
    pool_t *p = (pool_t *)arg;
    void *scratch = p->scratch_bytes ? malloc(p->scratch_bytes) : NULL;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t i0 = p->next;
        p->next += 16;
        pthread_mutex_unlock(&p->mu);
        if (i0 >= p->m) break;
        int64_t i1 = i0 + 16 < p->m ? i0 + 16 : p->m;
        for (int64_t i = i0; i < i1; ++i) p->fn(p->ctx, i, scratch);
    }
    free(scratch);
    return NULL;
}

static void run_pool(void (*fn)(void *, int64_t, void *), void *ctx, int64_t m, size_t scratch, int nthreads)
{
    pool_t p;
    p.fn = fn; p.ctx = ctx; p.m = m; p.next = 0; p.scratch_bytes = scratch;
    pthread_mutex_init(&p.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, pool_worker, &p);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&p.mu);
}

/* ------------------------------------------------------------------------ */
/* brute force (Eq. 3 / Eq. 4 over every primitive)                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    const scene_t *s;
    params_t pr;
    const double *q;
    double *val, *grad, *dmin;
} brute_ctx;

static void brute_one(void *c_, int64_t i, void *scratch)
{
    brute_ctx *c = (brute_ctx *)c_;
    const scene_t *s = c->s;
    term_t *T = (term_t *)scratch;
    const double *q = c->q + 3 * i;
    double dm = INFINITY;
    for (int64_t k = 0; k < s->n; ++k) {
        near_t nr;
        T[k] = prim_term(s, &s->P[k], q, &c->pr, &nr, NULL, NULL);
        if (nr.d < dm) dm = nr.d;
    }
    lse_finish(T, s->n, c->pr.alpha, &c->val[i], &c->grad[3 * i]);
    if (c->dmin) c->dmin[i] = dm;
}

void orc_brute(void *h, double alpha, double alpha_u, int paper_metric, int unit,
               const double *q, int64_t m, double *val, double *grad, double *dmin, int nthreads)
{
    scene_t *s = (scene_t *)h;
    brute_ctx c = {s, {alpha, alpha / (alpha > alpha_u ? alpha : alpha_u), paper_metric, unit}, q, val, grad, dmin};
    run_pool(brute_one, &c, m, sizeof(term_t) * (size_t)(s->n ? s->n : 1), nthreads);
}

/* ------------------------------------------------------------------------ */
/* Morton codes and the binary radix tree                                   */
/* ------------------------------------------------------------------------ */
/* fp32 centroid in a fixed operation order (no contraction) */
static void centroid_f(const scene_t *s, const prim_t *p, float *c)
{
    const float *V = s->Vf;
    if (p->kind == K_POINT) {
        for (int j = 0; j < 3; ++j) c[j] = V[3 * p->v[0] + j];
    } else if (p->kind == K_SEG) {
        for (int j = 0; j < 3; ++j) c[j] = (V[3 * p->v[0] + j] + V[3 * p->v[1] + j]) * 0.5f;
    } else {
        const float third = 1.0f / 3.0f;
        for (int j = 0; j < 3; ++j) c[j] = ((V[3 * p->v[0] + j] + V[3 * p->v[1] + j]) + V[3 * p->v[2] + j]) * third;
    }
}

static uint64_t morton_of(const float *c, const float *lo, const float *hi)
{
    uint32_t k[3];
    for (int j = 0; j < 3; ++j) {
        float ext = hi[j] - lo[j];
        float u = 0.0f;
        if (ext > 0.0f) u = (c[j] - lo[j]) / ext;
        if (u < 0.0f) u = 0.0f;
        if (u > 1.0f) u = 1.0f;
        float f = floorf(u * 2097152.0f);
        uint32_t v = (uint32_t)f;
        k[j] = v > 2097151u ? 2097151u : v;
    }
    uint64_t code = 0;
    for (int b = 20; b >= 0; --b) {
        code = (code << 1) | ((k[0] >> b) & 1u);
        code = (code << 1) | ((k[1] >> b) & 1u);
        code = (code << 1) | ((k[2] >> b) & 1u);
    }
    return code;
}

static const scene_t *g_sort_scene;
static int cmp_sorted(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    uint64_t ci = g_sort_scene->codes[i], cj = g_sort_scene->codes[j];
    if (ci != cj) return ci < cj ? -1 : 1;
    return i < j ? -1 : (i > j ? 1 : 0);
}

/* common-prefix length of the augmented keys (64-bit code, 32-bit index) of
   buckets i and j (each keyed by its first sorted primitive) */
static int key_prefix(const scene_t *s, int64_t i, int64_t j)
{
    int64_t pi = s->sorted[i * s->L], pj = s->sorted[j * s->L];
    uint64_t a = s->codes[pi], b = s->codes[pj];
    if (a != b) return __builtin_clzll(a ^ b);
    uint32_t x = (uint32_t)pi, y = (uint32_t)pj;
    return 64 + __builtin_clz(x ^ y);   /* buckets are distinct, so x != y */
}

static void aabb_init(float *lo, float *hi) { for (int j = 0; j < 3; ++j) { lo[j] = INFINITY; hi[j] = -INFINITY; } }
static void aabb_addp(const scene_t *s, const prim_t *p, float *lo, float *hi)
{
    int nvtx = p->kind == K_POINT ? 1 : (p->kind == K_SEG ? 2 : 3);
    for (int a = 0; a < nvtx; ++a)
        for (int j = 0; j < 3; ++j) {
            float x = s->Vf[3 * p->v[a] + j];
            if (x < lo[j]) lo[j] = x;
            if (x > hi[j]) hi[j] = x;
        }
}

/* top-down construction of internal node `node` over buckets [first, last] */
static void build_range(scene_t *s, int64_t node, int64_t first, int64_t last)
{
    int dnode = key_prefix(s, first, last);
    int64_t split = first;
    for (int64_t i = first; i < last; ++i)
        if (key_prefix(s, first, i) > dnode) split = i;
    /* children numbered the Karras way: left = split, right = split + 1 */
    if (split == first) s->left[node] = -(int32_t)(split + 1);
    else { s->left[node] = (int32_t)split; build_range(s, split, first, split); }
    if (split + 1 == last) s->right[node] = -(int32_t)(split + 2);
    else { s->right[node] = (int32_t)(split + 1); build_range(s, split + 1, split + 1, last); }
}

static void agg_node(scene_t *s, int32_t child, float *lo, float *hi, int64_t *cnt, int *pts_only);
static void agg_internal(scene_t *s, int64_t node)
{
    float lo[3], hi[3];
    aabb_init(lo, hi);
    int64_t cnt = 0; int po = 1;
    int32_t ch[2] = {s->left[node], s->right[node]};
    for (int c = 0; c < 2; ++c) {
        float clo[3], chi[3]; int64_t cc; int cpo;
        agg_node(s, ch[c], clo, chi, &cc, &cpo);
        for (int j = 0; j < 3; ++j) { if (clo[j] < lo[j]) lo[j] = clo[j]; if (chi[j] > hi[j]) hi[j] = chi[j]; }
        cnt += cc; po = po && cpo;
    }
    memcpy(s->nlo[node], lo, sizeof(lo)); memcpy(s->nhi[node], hi, sizeof(hi));
    s->ncount[node] = cnt; s->npts_only[node] = po;
}

static void agg_node(scene_t *s, int32_t child, float *lo, float *hi, int64_t *cnt, int *pts_only)
{
    if (child < 0) {
        int64_t b = -(int64_t)child - 1;
        memcpy(lo, s->llo[b], sizeof(float) * 3); memcpy(hi, s->lhi[b], sizeof(float) * 3);
        *cnt = s->lcount[b]; *pts_only = s->lpts_only[b];
    } else {
        agg_internal(s, child);
        memcpy(lo, s->nlo[child], sizeof(float) * 3); memcpy(hi, s->nhi[child], sizeof(float) * 3);
        *cnt = s->ncount[child]; *pts_only = s->npts_only[child];
    }
}

int orc_tree_build(void *h, int L)
{
    scene_t *s = (scene_t *)h;
    tree_free(s);
    if (L < 1) return -1;
    s->L = L;
    int64_t n = s->n;
    /* scene box over every vertex */
    aabb_init(s->slo, s->shi);
    for (int64_t i = 0; i < s->nv; ++i)
        for (int j = 0; j < 3; ++j) {
            float x = s->Vf[3 * i + j];
            if (x < s->slo[j]) s->slo[j] = x;
            if (x > s->shi[j]) s->shi[j] = x;
        }
    s->codes = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    s->sorted = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        float c[3];
        centroid_f(s, &s->P[i], c);
        s->codes[i] = morton_of(c, s->slo, s->shi);
        s->sorted[i] = i;
    }
    g_sort_scene = s;
    qsort(s->sorted, (size_t)n, sizeof(int64_t), cmp_sorted);
    if (n == 0) { s->nb = 0; return 0; }
    int64_t nb = (n + L - 1) / L;
    s->nb = nb;
    s->llo = malloc(sizeof(float) * 3 * nb); s->lhi = malloc(sizeof(float) * 3 * nb);
    s->lcount = malloc(sizeof(int64_t) * nb); s->lpts_only = malloc(sizeof(int) * nb);
    for (int64_t b = 0; b < nb; ++b) {
        aabb_init(s->llo[b], s->lhi[b]);
        int64_t e = (b + 1) * L < n ? (b + 1) * L : n;
        int po = 1;
        for (int64_t k = b * L; k < e; ++k) {
            const prim_t *p = &s->P[s->sorted[k]];
            aabb_addp(s, p, s->llo[b], s->lhi[b]);
            if (p->kind != K_POINT) po = 0;
        }
        s->lcount[b] = e - b * L; s->lpts_only[b] = po;
    }
    int64_t ni = nb - 1;
    int64_t na = ni ? ni : 1;
    s->left = malloc(sizeof(int32_t) * na); s->right = malloc(sizeof(int32_t) * na);
    s->nlo = malloc(sizeof(float) * 3 * na); s->nhi = malloc(sizeof(float) * 3 * na);
    s->ncount = malloc(sizeof(int64_t) * na); s->npts_only = malloc(sizeof(int) * na);
    if (ni > 0) {
        build_range(s, 0, 0, nb - 1);
        agg_internal(s, 0);
    }
    return 0;
}

int64_t orc_tree_nb(void *h) { return ((scene_t *)h)->nb; }

void orc_tree_export(void *h, uint64_t *codes, int64_t *sorted, int32_t *left, int32_t *right,
                     float *nlo, float *nhi, int64_t *ncount, float *llo, float *lhi, int64_t *lcount,
                     float *scene_box)
{
    scene_t *s = (scene_t *)h;
    int64_t nb = s->nb, ni = nb > 0 ? nb - 1 : 0;
    memcpy(codes, s->codes, sizeof(uint64_t) * s->n);
    memcpy(sorted, s->sorted, sizeof(int64_t) * s->n);
    if (ni) {
        memcpy(left, s->left, sizeof(int32_t) * ni); memcpy(right, s->right, sizeof(int32_t) * ni);
        memcpy(nlo, s->nlo, sizeof(float) * 3 * ni); memcpy(nhi, s->nhi, sizeof(float) * 3 * ni);
        memcpy(ncount, s->ncount, sizeof(int64_t) * ni);
    }
    if (nb) {
        memcpy(llo, s->llo, sizeof(float) * 3 * nb); memcpy(lhi, s->lhi, sizeof(float) * 3 * nb);
        memcpy(lcount, s->lcount, sizeof(int64_t) * nb);
    }
    for (int j = 0; j < 3; ++j) { scene_box[j] = s->slo[j]; scene_box[3 + j] = s->shi[j]; }
}

/* ------------------------------------------------------------------------ */
/* query primitives (Sec. 3.4): an edge or a triangle as the query          */
/* ------------------------------------------------------------------------ */
/* Closest points of two simplices A (na vertices) and B (nb vertices): the
   minimum of |A(lambda) - B(mu)|^2 over both barycentric simplices (the QP
   of App. B). Every pair of faces (vertex subsets) is tried: the pair's
   unconstrained minimiser on its affine hulls, kept if its barycentric
   coordinates are feasible. The convex minimum lies in the relative interior
   of some face pair, where it is that pair's unconstrained minimiser; a pair
   whose normal equations are singular (parallel hulls) is skipped, since its
   minimum is then also reached on a smaller face pair. The first face pair
   in enumeration order that reaches the smallest distance gives pa, pb. */
double orc_simplex_closest(const double *A, int na, const double *B, int nb, double *pa, double *pb)
{
    double best = INFINITY;
    for (int sa = 1; sa < (1 << na); ++sa)
        for (int sb = 1; sb < (1 << nb); ++sb) {
            int ia[3] = {0, 0, 0}, ib[3] = {0, 0, 0}, ka = 0, kb = 0;
            for (int i = 0; i < na; ++i) if ((sa >> i) & 1) ia[ka++] = i;
            for (int j = 0; j < nb; ++j) if ((sb >> j) & 1) ib[kb++] = j;
            const double *a0 = A + 3 * ia[0], *b0 = B + 3 * ib[0];
            double M[3][4], r0[3];
            int m = 0;
            for (int i = 1; i < ka; ++i, ++m)
                for (int j = 0; j < 3; ++j) M[j][m] = A[3 * ia[i] + j] - a0[j];
            for (int i = 1; i < kb; ++i, ++m)
                for (int j = 0; j < 3; ++j) M[j][m] = -(B[3 * ib[i] + j] - b0[j]);
            for (int j = 0; j < 3; ++j) r0[j] = a0[j] - b0[j];
            double z[4] = {0, 0, 0, 0};
            if (m > 0) {
                /* normal equations (M^T M) z = -M^T r0 by Gaussian elimination */
                double G[4][5], scale = 0.0;
                for (int p = 0; p < m; ++p) {
                    for (int q = 0; q < m; ++q) {
                        double g = 0.0;
                        for (int j = 0; j < 3; ++j) g += M[j][p] * M[j][q];
                        G[p][q] = g;
                    }
                    double rhs = 0.0;
                    for (int j = 0; j < 3; ++j) rhs -= M[j][p] * r0[j];
                    G[p][m] = rhs;
                    if (G[p][p] > scale) scale = G[p][p];
                }
                int singular = scale <= 0.0;
                for (int col = 0; col < m && !singular; ++col) {
                    int piv = col;
                    for (int r = col + 1; r < m; ++r) if (fabs(G[r][col]) > fabs(G[piv][col])) piv = r;
                    if (fabs(G[piv][col]) <= 1e-13 * scale) { singular = 1; break; }
                    if (piv != col)
                        for (int q = 0; q <= m; ++q) { double t = G[col][q]; G[col][q] = G[piv][q]; G[piv][q] = t; }
                    for (int r = 0; r < m; ++r) {
                        if (r == col) continue;
                        double f = G[r][col] / G[col][col];
                        for (int q = col; q <= m; ++q) G[r][q] -= f * G[col][q];
                    }
                }
                if (singular) continue;
                for (int p = 0; p < m; ++p) z[p] = G[p][m] / G[p][p];
            }
            /* feasibility: barycentric coordinates of both points >= 0 */
            double la0 = 1.0, mb0 = 1.0;
            int ok = 1;
            for (int i = 0; i < ka - 1; ++i) { ok &= z[i] >= 0.0; la0 -= z[i]; }
            for (int i = 0; i < kb - 1; ++i) { ok &= z[ka - 1 + i] >= 0.0; mb0 -= z[ka - 1 + i]; }
            if (!ok || la0 < 0.0 || mb0 < 0.0) continue;
            double xa[3], xb[3];
            for (int j = 0; j < 3; ++j) {
                xa[j] = a0[j];
                xb[j] = b0[j];
                for (int i = 1; i < ka; ++i) xa[j] += z[i - 1] * (A[3 * ia[i] + j] - a0[j]);
                for (int i = 1; i < kb; ++i) xb[j] += z[ka - 1 + i - 1] * (B[3 * ib[i] + j] - b0[j]);
            }
            double d2 = 0.0;
            for (int j = 0; j < 3; ++j) d2 += (xa[j] - xb[j]) * (xa[j] - xb[j]);
            if (d2 < best) {
                best = d2;
                for (int j = 0; j < 3; ++j) { pa[j] = xa[j]; pb[j] = xb[j]; }
            }
        }
    return sqrt(best);
}

/* A query: its vertices (k = 1: a point) and its axis-aligned box. */
typedef struct { double v[9]; int k; double lo[3], hi[3]; } query_t;

static void query_point(query_t *Q, const double *q)
{
    Q->k = 1;
    for (int j = 0; j < 3; ++j) Q->v[j] = Q->lo[j] = Q->hi[j] = q[j];
}

static void query_prim(query_t *Q, const double *V, const int32_t *f, int k)
{
    Q->k = k;
    for (int j = 0; j < 3; ++j) { Q->lo[j] = INFINITY; Q->hi[j] = -INFINITY; }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < 3; ++j) {
            double x = V[3 * (int64_t)f[i] + j];
            Q->v[3 * i + j] = x;
            if (x < Q->lo[j]) Q->lo[j] = x;
            if (x > Q->hi[j]) Q->hi[j] = x;
        }
}

/* The exact term of data primitive p for query Q. For an edge or triangle
   query the term is the point term at g's point of a closest pair (Sec. 3.4
   takes the closest point on g wherever a single point is needed, as in the
   weights); its distance is the simplex distance and its gradient is that of
   a rigid translation of g. */
static term_t query_term(const scene_t *s, const prim_t *p, const query_t *Q, const params_t *pr, double *dist)
{
    if (Q->k == 1) {
        near_t nr;
        term_t T = prim_term(s, p, Q->v, pr, &nr, NULL, NULL);
        if (dist) *dist = nr.d;
        return T;
    }
    int nv = p->kind == K_POINT ? 1 : (p->kind == K_SEG ? 2 : 3);
    double F[9], pf[3], pg[3];
    for (int i = 0; i < nv; ++i)
        for (int j = 0; j < 3; ++j) F[3 * i + j] = s->V[3 * p->v[i] + j];
    double d = orc_simplex_closest(F, nv, Q->v, Q->k, pf, pg);
    if (dist) *dist = d;
    double scale = 1.0;
    for (int j = 0; j < 3; ++j) scale = fmax(scale, fabs(pg[j]));
    const double tol = 1e-12 * scale;
    if (d <= tol && nv == 3 && Q->k == 3) {
        /* crossing triangles touch along a segment: the point taken is the
           mean of the points where an edge of one pierces the other (the
           segment's midpoint in general position) */
        double sum[3] = {0, 0, 0};
        int hits = 0;
        for (int side = 0; side < 2; ++side)
            for (int e = 0; e < 3; ++e) {
                const double *T3 = side ? F : Q->v, *O3 = side ? Q->v : F;
                double E[6], a[3], b[3];
                for (int j = 0; j < 3; ++j) { E[j] = O3[3 * e + j]; E[3 + j] = O3[3 * ((e + 1) % 3) + j]; }
                if (orc_simplex_closest(E, 2, T3, 3, a, b) <= tol) {
                    for (int j = 0; j < 3; ++j) sum[j] += a[j];
                    ++hits;
                }
            }
        if (hits)
            for (int j = 0; j < 3; ++j) pg[j] = sum[j] / hits;
    }
    near_t nr;
    term_t T = prim_term(s, p, pg, pr, &nr, NULL, NULL);
    /* touching primitives: the point term at the touching point has a
       distance at rounding level with a meaningless direction; the pair's
       distance is 0 and, as for d = 0 in Eq. dgrad, its gradient is 0 */
    if (d <= tol) {
        T.t += pr->alpha * nr.d;
        for (int j = 0; j < 3; ++j) T.v[j] -= nr.gd[j];
    }
    return T;
}

typedef struct {
    const scene_t *s;
    params_t pr;
    const double *V;
    const int32_t *QF;
    int k;
    double *val, *grad, *dmin;
} qbrute_ctx;

static void qbrute_one(void *c_, int64_t i, void *scratch)
{
    qbrute_ctx *c = (qbrute_ctx *)c_;
    const scene_t *s = c->s;
    term_t *T = (term_t *)scratch;
    query_t Q;
    query_prim(&Q, c->V, c->QF + (int64_t)c->k * i, c->k);
    double dm = INFINITY;
    for (int64_t n = 0; n < s->n; ++n) {
        double d;
        T[n] = query_term(s, &s->P[n], &Q, &c->pr, &d);
        if (d < dm) dm = d;
    }
    lse_finish(T, s->n, c->pr.alpha, &c->val[i], &c->grad[3 * i]);
    if (c->dmin) c->dmin[i] = dm;
}

/* Eq. 3 / Eq. 4 with query primitives: m primitives of k vertices each
   (QF [m, k] indices into V [*, 3]); grad is that of a rigid translation. */
void orc_brute_prims(void *h, double alpha, double alpha_u, int paper_metric, int unit, const double *V,
                     const int32_t *QF, int k, int64_t m, double *val, double *grad, double *dmin, int nthreads)
{
    scene_t *s = (scene_t *)h;
    qbrute_ctx c = {s, {alpha, alpha / (alpha > alpha_u ? alpha : alpha_u), paper_metric, unit}, V, QF, k, val,
                    grad, dmin};
    run_pool(qbrute_one, &c, m, sizeof(term_t) * (size_t)(s->n ? s->n : 1), nthreads);
}

/* ------------------------------------------------------------------------ */
/* Barnes-Hut (Alg. 1 / Alg. 2, App. D)                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    const scene_t *s;
    params_t pr;
    double beta;
    float beta2f;
    int decision;          /* 0: fp32 squared test, 1: fp64 ratio test */
    double wfar;           /* max(A_E, A_T)^S */
    const double *q;       /* query points [m,3], or the query mesh's vertices */
    const int32_t *QF;     /* query primitives [m, qk] (NULL: point queries) */
    int qk;
    double *val, *grad;
    int64_t *counts;       /* [m, 3]: nodes tested, far-field accepts, leaf primitives */
    double *margin;        /* min over tested nodes of |ratio - beta| / beta */
} bh_ctx;

typedef struct { term_t *T; int64_t n, cap; int64_t tested, far, leafp; double margin; } acc_t;

static void acc_push(acc_t *a, term_t t)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 256;
        a->T = (term_t *)realloc(a->T, sizeof(term_t) * a->cap);
    }
    a->T[a->n++] = t;
}

/* The Barnes-Hut condition |B| / d(y_B, g) < beta with y_B the closest point
   of the box (Sec. 3.5, App. D). The query g is given by its axis-aligned
   box [qlo, qhi] (a point: qlo = qhi = q). For an edge or triangle query the
   halfspace test of Sec. 3.5 is taken on that box: the box halfspaces that g
   lies entirely outside of are those where g's box is beyond the node's, and
   the distance to the feature they identify is replaced by the distance
   between the two boxes, a lower bound of it (equal to it for one halfspace
   and for points), so the far field stays an underestimate. Decision mode 0
   takes the test in FP32 as diag^2 < beta^2 * dbox^2 with the operation
   order fixed below (squares summed as fma(z, z, fma(y, y, x * x)), each fma
   rounded once); mode 1 in FP64 as the ratio. Overlapping boxes (d = 0)
   always open the node. */
static int bh_condition(const bh_ctx *c, const float *lo, const float *hi, const double *qlo, const double *qhi,
                        double *margin)
{
    if (c->decision == 0) {
        float dx[3], ex[3];
        for (int j = 0; j < 3; ++j) {
            float a = lo[j] - (float)qhi[j], b = (float)qlo[j] - hi[j];
            float m = a > b ? a : b;
            dx[j] = m > 0.0f ? m : 0.0f;
            ex[j] = hi[j] - lo[j];
        }
        float x0 = dx[0] * dx[0];
        float dbox2 = fmaf(dx[2], dx[2], fmaf(dx[1], dx[1], x0));
        float y0 = ex[0] * ex[0];
        float diag2 = fmaf(ex[2], ex[2], fmaf(ex[1], ex[1], y0));
        float rhs = c->beta2f * dbox2;
        if (margin && dbox2 > 0.0f) {
            double r = sqrt((double)diag2) / sqrt((double)dbox2);
            double mg = fabs(r - c->beta) / (c->beta > 0 ? c->beta : 1.0);
            if (mg < *margin) *margin = mg;
        }
        return diag2 < rhs;
    } else {
        double d2 = 0.0, g2 = 0.0;
        for (int j = 0; j < 3; ++j) {
            double l = lo[j], h = hi[j];
            double gap = qhi[j] < l ? l - qhi[j] : (qlo[j] > h ? qlo[j] - h : 0.0);
            d2 += gap * gap;
            g2 += (h - l) * (h - l);
        }
        if (d2 <= 0.0) return 0;
        double r = sqrt(g2) / sqrt(d2);
        if (margin) {
            double mg = fabs(r - c->beta) / (c->beta > 0 ? c->beta : 1.0);
            if (mg < *margin) *margin = mg;
        }
        return r < c->beta;
    }
}

/* far-field term at the node box's nearest point to the query box: the
   offset is g's box minus the node's per axis (0 where they overlap) */
static void far_term(const bh_ctx *c, const float *lo, const float *hi, int64_t nB, int pts_only,
                     const double *qlo, const double *qhi, acc_t *a)
{
    double dv[3];
    for (int j = 0; j < 3; ++j) {
        double l = lo[j], h = hi[j];
        dv[j] = qhi[j] < l ? qhi[j] - l : (qlo[j] > h ? qlo[j] - h : 0.0);
    }
    double d = sqrt(dot3(dv, dv));
    double wB = pts_only ? 1.0 : c->wfar;
    term_t t;
    t.t = log((double)nB * wB) - c->pr.alpha * d;
    for (int j = 0; j < 3; ++j) t.v[j] = dv[j] / d;
    acc_push(a, t);
}

/* Alg. 1, recursive: the Barnes-Hut test first (also at leaves), else exact
   leaf terms, else both children. Q: the query (a point, or a primitive of
   Q->k vertices) and its box. */
static void collect(const bh_ctx *c, int32_t node, int is_leaf, const query_t *Q, acc_t *a)
{
    const scene_t *s = c->s;
    const float *lo, *hi; int64_t nB; int po;
    if (is_leaf) { lo = s->llo[node]; hi = s->lhi[node]; nB = s->lcount[node]; po = s->lpts_only[node]; }
    else { lo = s->nlo[node]; hi = s->nhi[node]; nB = s->ncount[node]; po = s->npts_only[node]; }
    a->tested++;
    if (bh_condition(c, lo, hi, Q->lo, Q->hi, c->margin ? &a->margin : NULL)) {
        a->far++;
        far_term(c, lo, hi, nB, po, Q->lo, Q->hi, a);
        return;
    }
    if (is_leaf) {
        int64_t e = ((int64_t)node + 1) * s->L < s->n ? ((int64_t)node + 1) * s->L : s->n;
        for (int64_t k = (int64_t)node * s->L; k < e; ++k) {
            acc_push(a, query_term(s, &s->P[s->sorted[k]], Q, &c->pr, NULL));
            a->leafp++;
        }
        return;
    }
    int32_t ch[2] = {s->left[node], s->right[node]};
    for (int k = 0; k < 2; ++k) {
        if (ch[k] < 0) collect(c, -ch[k] - 1, 1, Q, a);
        else collect(c, ch[k], 0, Q, a);
    }
}

static void bh_one(void *c_, int64_t i, void *scratch)
{
    bh_ctx *c = (bh_ctx *)c_;
    acc_t *a = (acc_t *)scratch;
    a->n = 0; a->tested = a->far = a->leafp = 0; a->margin = INFINITY;
    query_t Q;
    if (c->QF) query_prim(&Q, c->q, c->QF + (int64_t)c->qk * i, c->qk);
    else query_point(&Q, c->q + 3 * i);
    if (c->s->nb == 1) collect(c, 0, 1, &Q, a);
    else if (c->s->nb > 1) collect(c, 0, 0, &Q, a);
    lse_finish(a->T, a->n, c->pr.alpha, &c->val[i], &c->grad[3 * i]);
    if (c->counts) { c->counts[3 * i] = a->tested; c->counts[3 * i + 1] = a->far; c->counts[3 * i + 2] = a->leafp; }
    if (c->margin) c->margin[i] = a->margin;
}

typedef struct { bh_ctx *c; int64_t m, next; pthread_mutex_t mu; } bh_pool_t;

static void *bh_worker(void *arg)
{
    bh_pool_t *p = (bh_pool_t *)arg;
    acc_t a; memset(&a, 0, sizeof(a));
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t i0 = p->next; p->next += 16;
        pthread_mutex_unlock(&p->mu);
        if (i0 >= p->m) break;
        int64_t i1 = i0 + 16 < p->m ? i0 + 16 : p->m;
        for (int64_t i = i0; i < i1; ++i) bh_one(p->c, i, &a);
    }
    free(a.T);
    return NULL;
}

/* Barnes-Hut over m queries: points q [m,3] (qf_prims NULL) or primitives
   qf_prims [m, qk_prims] indexing the vertex array q. */
static int bh_run(void *h, double alpha, double alpha_u, double beta, int paper_metric, int unit, int decision,
                  const double *q, const int32_t *qf_prims, int qk_prims, int64_t m, double *val, double *grad,
                  int64_t *counts, double *margin, int nthreads)
{
    scene_t *s = (scene_t *)h;
    if (s->n > 0 && s->nb == 0) return -1;
    bh_ctx c;
    memset(&c, 0, sizeof(c));
    c.s = s;
    c.pr.alpha = alpha;
    c.pr.S = alpha / (alpha > alpha_u ? alpha : alpha_u);
    c.pr.paper_metric = paper_metric;
    c.pr.unit = unit;
    c.beta = beta;
    { float bf = (float)beta; c.beta2f = bf * bf; }
    c.decision = decision;
    double A = s->A_E > s->A_T ? s->A_E : s->A_T;
    c.wfar = unit ? 1.0 : pow(A, c.pr.S);
    c.q = q; c.val = val; c.grad = grad; c.counts = counts; c.margin = margin;
    c.QF = qf_prims; c.qk = qk_prims;
    bh_pool_t p; p.c = &c; p.m = m; p.next = 0;
    pthread_mutex_init(&p.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, bh_worker, &p);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&p.mu);
    return 0;
}

int orc_bh(void *h, double alpha, double alpha_u, double beta, int paper_metric, int unit, int decision,
           const double *q, int64_t m, double *val, double *grad, int64_t *counts, double *margin, int nthreads)
{
    return bh_run(h, alpha, alpha_u, beta, paper_metric, unit, decision, q, NULL, 1, m, val, grad, counts, margin,
                  nthreads);
}

int orc_bh_prims(void *h, double alpha, double alpha_u, double beta, int paper_metric, int unit, int decision,
                 const double *V, const int32_t *QF, int k, int64_t m, double *val, double *grad, int64_t *counts,
                 double *margin, int nthreads)
{
    return bh_run(h, alpha, alpha_u, beta, paper_metric, unit, decision, V, QF, k, m, val, grad, counts, margin,
                  nthreads);
}

/* ------------------------------------------------------------------------ */
/* certified lower bound of d^ over a top cut of the tree                   */
/* ------------------------------------------------------------------------ */
/* Every exact term w_i e^{-alpha d_i} of a primitive inside a node B has
   d_i >= d(q, box B) and w_i = (A w~_i)^S <= (A kappa)^S when kappa bounds
   w~ (a Bernstein polynomial lies below its largest coefficient), so
     LB(q) = -(1/alpha) ln sum_{B in cut} n_B w_B kappa^S e^{-alpha d(q, box B)}
   with w_B the far-field weight (1 for points-only nodes, max(A_E, A_T)^S
   otherwise) is below the exact d^ of Eq. 3 for any cut that covers every
   primitive once. The cut: breadth-first from the root, one level at a
   time, while the next level has at most 64 nodes (leaves stay). */
static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* largest Bernstein coefficient of w~ on one primitive, by the change of
   basis from the monomial form the weights are stored in:
   degree n in x:  beta_i = sum_{k<=i} C(i,k) / C(n,k) c_k;
   degree n on the triangle (1-x-y, x, y):
     beta_{.jk} = sum_{a<=j, b<=k} C(j,a) C(k,b) a! b! (n-a-b)! / n! c_{ab} */
static double prim_kappa(const scene_t *s, const prim_t *p, double *corner)
{
    corner[0] = corner[1] = corner[2] = 1.0;
    if (p->kind == K_SEG) {
        double c[5], best = -INFINITY;
        for (int k = 0; k < 5; ++k) c[k] = s->ebasis[k][0] * p->pa + s->ebasis[k][1] * p->pb + s->ebasis[k][2];
        for (int i = 0; i <= 4; ++i) {
            double b = 0.0;
            for (int k = 0; k <= i; ++k) b += binom(i, k) / binom(4, k) * c[k];
            if (b > best) best = b;
            if (i == 0) corner[0] = b;
            if (i == 4) corner[1] = b;
        }
        corner[2] = NAN;
        return best;
    }
    if (p->kind == K_TRI) {
        if (p->isolated) return 1.0;
        double c[8][8];
        memset(c, 0, sizeof(c));
        double rhs[3] = {p->pa, p->pb, 1.0 - p->pa};
        for (int j = 0; j < 36; ++j)
            c[s->texp[j][0]][s->texp[j][1]] +=
                s->tbasis[j][0] * rhs[0] + s->tbasis[j][1] * rhs[1] + s->tbasis[j][2] * rhs[2];
        double best = -INFINITY;
        for (int j = 0; j <= 7; ++j)
            for (int k = 0; j + k <= 7; ++k) {
                double b = 0.0;
                for (int a = 0; a <= j; ++a)
                    for (int bb = 0; bb <= k; ++bb)
                        b += binom(j, a) * binom(k, bb) / (binom(7, a) * binom(7 - a, bb)) * c[a][bb];
                if (b > best) best = b;
                if (j == 0 && k == 0) corner[0] = b;
                if (j == 7) corner[1] = b;
                if (k == 7) corner[2] = b;
            }
        return best;
    }
    return 1.0;
}

/* per primitive: largest Bernstein coefficient of w~ and the coefficients at
   the corners (x = 0, x = 1 [, y = 1]); out [n, 4] */
void orc_prim_kappa(void *h, double *out)
{
    scene_t *s = (scene_t *)h;
    for (int64_t i = 0; i < s->n; ++i) out[4 * i] = prim_kappa(s, &s->P[i], out + 4 * i + 1);
}

/* out: kappa, cut size. lb [m], grad [m,3] (grad may be NULL). */
int orc_lower_bound(void *h, double alpha, double alpha_u, int unit, const double *q, int64_t m, double *lb,
                    double *grad, double *info)
{
    scene_t *s = (scene_t *)h;
    if (s->n == 0 || s->nb == 0) return -1;
    double S = alpha / (alpha > alpha_u ? alpha : alpha_u);
    double kappa = 1.0;
    if (!unit)
        for (int64_t i = 0; i < s->n; ++i) {
            double corner[3];
            double k = prim_kappa(s, &s->P[i], corner);
            if (k > kappa) kappa = k;
        }
    double A = s->A_E > s->A_T ? s->A_E : s->A_T;
    double wfar = unit ? 1.0 : pow(A, S);
    enum { CUT = 64 };
    int32_t cur[CUT], nxt[CUT];  /* >= 0 internal node, < 0 leaf -(b+1) */
    int n = 1;
    cur[0] = s->nb > 1 ? 0 : -1;
    for (;;) {
        int nn = 0;
        for (int i = 0; i < n; ++i) nn += cur[i] >= 0 ? 2 : 1;
        if (nn > CUT || nn == n) break;
        int o = 0;
        for (int i = 0; i < n; ++i) {
            if (cur[i] < 0) nxt[o++] = cur[i];
            else { nxt[o++] = s->left[cur[i]]; nxt[o++] = s->right[cur[i]]; }
        }
        memcpy(cur, nxt, sizeof(int32_t) * o);
        n = o;
    }
    double lw[CUT];
    const float *lo[CUT], *hi[CUT];
    for (int i = 0; i < n; ++i) {
        int64_t cnt; int po;
        if (cur[i] < 0) {
            int64_t b = -(int64_t)cur[i] - 1;
            lo[i] = s->llo[b]; hi[i] = s->lhi[b]; cnt = s->lcount[b]; po = s->lpts_only[b];
        } else {
            lo[i] = s->nlo[cur[i]]; hi[i] = s->nhi[cur[i]]; cnt = s->ncount[cur[i]]; po = s->npts_only[cur[i]];
        }
        lw[i] = log((double)cnt * (po ? 1.0 : wfar)) + S * log(kappa);
    }
    for (int64_t k = 0; k < m; ++k) {
        const double *x = q + 3 * k;
        double t[CUT], dv[CUT][3], d[CUT], mx = -INFINITY;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < 3; ++j) {
                double l = lo[i][j], u = hi[i][j];
                double y = x[j] < l ? l : (x[j] > u ? u : x[j]);
                dv[i][j] = x[j] - y;
            }
            d[i] = sqrt(dot3(dv[i], dv[i]));
            t[i] = lw[i] - alpha * d[i];
            if (t[i] > mx) mx = t[i];
        }
        double sum = 0.0, g[3] = {0, 0, 0};
        for (int i = 0; i < n; ++i) {
            double e = exp(t[i] - mx);
            sum += e;
            if (d[i] > 0.0)
                for (int j = 0; j < 3; ++j) g[j] += e * dv[i][j] / d[i];
        }
        lb[k] = -(mx + log(sum)) / alpha;
        if (grad)
            for (int j = 0; j < 3; ++j) grad[3 * k + j] = g[j] / sum;
    }
    if (info) { info[0] = kappa; info[1] = (double)n; }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* rigid placement of query vertices in fp32                                */
/* ------------------------------------------------------------------------ */
/* x_k = R x0_k + p evaluated in fp32 in the fixed order
   fma(R_i0, x, fma(R_i1, y, R_i2 * z)) + p_i, with R and p rounded to fp32:
   the query points the GPU path evaluates (Sec. 4.5 places the query mesh by
   its pose; the rounding rule is part of this project's definition). */
void orc_pose_f32(const double *R9, const double *p3, const float *X0, int64_t m, float *X)
{
    float R[9], p[3];
    for (int i = 0; i < 9; ++i) R[i] = (float)R9[i];
    for (int i = 0; i < 3; ++i) p[i] = (float)p3[i];
    for (int64_t k = 0; k < m; ++k) {
        float x = X0[3 * k], y = X0[3 * k + 1], z = X0[3 * k + 2];
        for (int i = 0; i < 3; ++i)
            X[3 * k + i] = fmaf(R[3 * i], x, fmaf(R[3 * i + 1], y, R[3 * i + 2] * z)) + p[i];
    }
}
