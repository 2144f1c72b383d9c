/*
 * libsd: smooth distance and gradient on co-dimensional geometry, on one GPU.
 *
 * Computes, for a batch of query points q, the weighted LogSumExp smooth
 * minimum distance of Madan & Levin ("Fast Evaluation of Smooth Distance
 * Constraints on Co-Dimensional Geometry"), Eq. 3,
 *
 *     d^(q) = -(1/alpha) log sum_i w_i(q) exp(-alpha d_i(q)),
 *
 * and its gradient, Eq. 4, over a data mesh of points, edges and triangles,
 * with the blending weights of Sec. 3.3 / App. C and the conservative
 * Barnes-Hut far field of Sec. 3.5 / App. D (Alg. 1 and Alg. 2).
 *
 * Conventions for every entry point:
 *   - Returns an sd_status (SD_OK == 0); nothing is thrown across the ABI.
 *   - "device" pointers are CUDA device memory of the current device; the
 *     caller owns them and keeps them alive until the work on `stream` ends.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Arrays are row-major, contiguous: xyz triples are [n,3] float32,
 *     index tuples are [m,2] / [m,3] int32 (0-based into their own vertex
 *     array).
 */
#ifndef SD_H_
#define SD_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SD_OK = 0,
    SD_ERR_INVALID_ARG = 1, /* bad pointer/size/parameter; nothing was launched */
    SD_ERR_CUDA = 2,        /* a CUDA call failed (the library's last error text is kept) */
    SD_ERR_OOM = 3,         /* device allocation failed */
    SD_ERR_NONFINITE = 4,   /* a vertex or query coordinate is NaN/Inf */
    SD_ERR_INDEX = 5,       /* an edge/triangle index is outside its vertex array */
    SD_ERR_TOO_LARGE = 6,   /* a size exceeds what the library supports (2^31-1 primitives) */
    SD_ERR_TIMEOUT = 7      /* a bounded device-side wait ran out (the results of that call are invalid);
                               no entry point returns it at present: the sorts' waits fall back to an
                               exact direct count, and the tensor-core kernel marks its rows NaN */
} sd_status;

/* Geometry of the data mesh M_d = (V, F) (Sec. 3). Each part may be empty
   (count 0, pointer ignored). Primitive order: points, then edges, then
   triangles; "original index" below means this order. */
typedef struct { const float* xyz; int64_t n; } sd_points;                              /* device [n,3] */
typedef struct { const float* V; int64_t nv; const int32_t* E; int64_t ne; } sd_edges;   /* device [nv,3], [ne,2] */
typedef struct { const float* V; int64_t nv; const int32_t* F; int64_t nf; } sd_tris;    /* device [nv,3], [nf,3] */
typedef struct { sd_points pts; sd_edges edges; sd_tris tris; } sd_geometry;

enum { SD_WEIGHTS_PAPER = 0, SD_WEIGHTS_UNIT = 1 };

typedef struct {
    float alpha_u;        /* attenuation threshold alpha_U of Sec. 3.3: S = alpha / max(alpha, alpha_U); 0 => S = 1 */
    int32_t leaf_size;    /* L >= 1: primitives per leaf bucket (part of the tree's definition; the paper uses 1) */
    int32_t weights;      /* SD_WEIGHTS_PAPER: w_i = (A w~_i)^S of App. C; SD_WEIGHTS_UNIT: w_i = 1 */
    int32_t paper_metric; /* 1: barycentric gradients measured in the alpha-scaled metric of Sec. 3.3
                             (the weight-gradient term is divided by alpha once more); 0: exact gradient */
    int32_t defer_checks; /* 0 (default): sd_build waits for the device and returns data errors itself;
                             1: sd_build only enqueues work and returns SD_OK; data errors are reported
                             by sd_query_status, and sd_tree_get_info waits for the build */
} sd_build_opts;

typedef struct {
    int32_t sort_queries; /* 1 (default): traverse in Hilbert order of the queries (results change only by
                             summation order) */
    int32_t block;        /* threads per block of the traversal kernel: a multiple of 32 up to 256;
                             0 = library default (128) */
    int32_t* counts;      /* optional device [M,3] int32 output: Barnes-Hut tests, far-field accepts,
                             leaf primitives evaluated (the work counts of Alg. 1), or NULL */
    const int32_t* order; /* optional device [M] permutation of 0..M-1 giving the traversal order (as
                             written by sd_query_order); when set, sort_queries is ignored */
} sd_query_opts;

typedef struct sd_tree sd_tree;

/* Fill option structs with defaults (alpha_u 0, L 1, paper weights, exact
   metric; sorted queries, default block, no counts). */
void sd_default_build_opts(sd_build_opts* o);
void sd_default_query_opts(sd_query_opts* o);

/*
 * Build the acceleration structure for Alg. 1 (Sec. 3.5, App. D) on `stream`:
 * validation, incidence counts and weight parameters (App. C.2-C.3), 63-bit
 * Morton codes, a stable radix sort by (code, original index), a binary
 * radix tree over leaf buckets of L consecutive sorted primitives, per-node
 * AABBs, primitive counts n_B and far-field weights w_B (App. D), and the
 * primitives re-packed in leaf order.
 *   g      host pointer to the geometry (its arrays are device pointers)
 *   alpha  > 0, accuracy parameter of Eq. 3
 *   beta   >= 0, Barnes-Hut parameter (0 = exact evaluation, Sec. 3.5)
 *   opts   host pointer or NULL for defaults
 *   out    receives the new tree; the tree owns copies of everything it
 *          needs, so `g`'s arrays may be freed after the call returns.
 * By default synchronises `stream` before returning (it reports data errors
 * such as SD_ERR_NONFINITE / SD_ERR_INDEX, in which case *out is NULL). With
 * opts->defer_checks = 1 it returns after enqueueing the build: the same
 * kernels run (indices are clamped where they are dereferenced, so bad input
 * cannot fault) and their verdict is reported by sd_query_status.
 * The weight parameters run on a library-owned side stream of the device,
 * joined back into `stream` by an event after the sort; builds on several
 * streams of one device share that side
 * stream (their parameter phases queue behind one another), and a build
 * enqueued under stream capture takes the side stream into the capture, so
 * no other build may run on the device meanwhile.
 */
int sd_build(const sd_geometry* g, float alpha, float beta, const sd_build_opts* opts,
             void* stream, sd_tree** out);

/*
 * Barnes-Hut smooth distance and gradient (Alg. 2 over Alg. 1) at M queries.
 *   q      device [M,3] float32 query points
 *   value  device [M] float32 output d^(q); +inf for an empty data mesh
 *   grad   device [M,3] float32 output grad d^(q), or NULL for value only
 *   opts   host pointer or NULL for defaults
 * Asynchronous on `stream`. A non-finite query yields NaN outputs for that
 * query and sets the tree's status word to SD_ERR_NONFINITE (read it with
 * sd_query_status). Concurrent calls on one tree are safe; they share only
 * the status word.
 */
int sd_query(const sd_tree* t, const float* q, int64_t M, float* value, float* grad,
             const sd_query_opts* opts, void* stream);

/*
 * Traversal order for sd_query: writes to `order` (device [M] int32) the
 * query indices sorted by the 24-bit Hilbert index of each query relative to
 * the tree's scene box (stable; ties keep index order). Asynchronous on
 * `stream`; uses stream-ordered temporary device memory. For a tree built
 * with defer_checks, `stream` first waits (outside stream capture) for the
 * point of the build at which the scene box is final, so the order may be
 * computed on another stream than the build's, overlapping the rest of the
 * build; the queries themselves must be ready on `stream`.
 */
int sd_query_order(const sd_tree* t, const float* q, int64_t M, int32_t* order, void* stream);

/*
 * The plain method: Eq. 3 / Eq. 4 summed exactly over every primitive (no
 * tree pruning; equivalent to beta = 0), with the same weights as `t`.
 * Same arguments and behaviour as sd_query (opts->counts is ignored).
 */
int sd_query_brute(const sd_tree* t, const float* q, int64_t M, float* value, float* grad,
                   const sd_query_opts* opts, void* stream);

/*
 * sd_query without any device allocation by the library (the paper has no
 * counterpart; this is an integration entry point). For callers that own a
 * fixed device-memory budget and must not let a library call cudaMalloc
 * during their work, where an allocation could block on the device or fail
 * part-way. Same inputs and outputs as sd_query with default options
 * (Hilbert-ordered traversal, value and gradient, no counts).
 *   M      0 <= M <= 262144 (SD_ERR_TOO_LARGE beyond, nothing launched)
 * Its temporary storage (4,984,320 bytes, about 5.0 MB or 4.75 MiB) is one
 * static device array that every device loading the library keeps until
 * the process exits. All calls on a device share it, whether made directly
 * or replayed from a captured CUDA graph, so any two of them that overlap
 * on the GPU race: order them (one stream, or events). The first call on a
 * device looks up the array's address with that device current and caches
 * it: make that call before any stream capture, and do not call the entry
 * point again after resetting the device (cudaDeviceReset) in the same
 * process, since the cached address does not survive a reset.
 */
int sd_query_noalloc(const sd_tree* t, const float* q, int64_t M, float* value, float* grad, void* stream);

/*
 * Rigid-body queries (Sec. 4.5, Eq. opt): places a body's rest vertices by
 * x_k = R(theta) x0_k + p, theta a rotation vector (exponential map), and
 * evaluates d^ and grad d^ at every x_k with sd_query.
 *   X0     device [M,3] rest-pose vertices
 *   pose   host double[6] = (theta_x, theta_y, theta_z, p_x, p_y, p_z)
 *   X      device [M,3] output: the placed vertices (the queries)
 *   value, grad, opts, stream: as for sd_query
 */
int sd_pose_query(const sd_tree* t, const float* X0, int64_t M, const double* pose, float* X,
                  float* value, float* grad, const sd_query_opts* opts, void* stream);

/*
 * Reduction over a body's vertices and its pose adjoint (Sec. 3.6,
 * Eq. lse_full2 and Eq. dlse_full for point queries, n(g) = 0, weight 1):
 *   alpha_q > 0: D = -(1/alpha_q) log sum_k exp(-alpha_q d^_k), gamma_k its
 *                softmin weights (`gamma` ignored);
 *   alpha_q <= 0: D = sum_k gamma_k d^_k for the given device [M] gamma
 *                (an upstream gradient).
 * Writes device out[7] = (D, dD/dp (3), dD/dtheta (3)) with
 * dD/dp = sum_k gamma_k g_k and dD/dtheta = J_l(theta)^T sum_k gamma_k
 * (R x0_k) x g_k (J_l the left Jacobian of SO(3)); if dX0 is not NULL also
 * device [M,3] dD/dx0_k = gamma_k R^T g_k. value/grad are sd_pose_query's
 * outputs for the same X0 and pose. The sums are reduced in a fixed order
 * (deterministic). Uses stream-ordered temporary device memory.
 */
int sd_pose_reduce(const float* X0, const float* value, const float* grad, const float* gamma, int64_t M,
                   const double* pose, float alpha_q, float* out, float* dX0, void* stream);

/*
 * One shard of a body's vertices, for a reduction split across processes or
 * GPUs (Sec. 3.6: the outer sum of Eq. lse_full2 and Eq. dlse_full is
 * associative, so per-shard partials merge exactly up to rounding). Inputs
 * as for sd_pose_reduce, restricted to the shard's vertices; writes device
 * part[9] = (m, s, v, gp (3), gt (3)) with
 *   alpha_q > 0:  t_k = -alpha_q d^_k, m = max_k t_k, e_k = exp(t_k - m);
 *   alpha_q <= 0: m = 0, e_k = gamma_k (device [M]);
 *   s = sum e_k, v = sum e_k d^_k, gp = sum e_k g_k,
 *   gt = sum e_k (R x0_k) x g_k,
 * summed in a fixed order (deterministic). M = 0 writes the merge's neutral
 * element (m = -inf, the rest 0). Uses stream-ordered temporary memory.
 */
int sd_pose_partial(const float* X0, const float* value, const float* grad, const float* gamma, int64_t M,
                    const double* pose, float alpha_q, float* part, void* stream);

/*
 * Host-only (needs no GPU): merges n shard partials (host double [n,9] in
 * sd_pose_partial's layout, any grouping and order) and finalises them as
 * sd_pose_reduce does, in FP64: out[7] = (D, dD/dp (3), dD/dtheta (3)) with
 * M = max_i m_i, and S, V, GP, GT the shards' s, v, gp, gt scaled by
 * exp(m_i - M) and summed:
 *   alpha_q > 0:  D = -(M + log S)/alpha_q, dD/dp = GP/S,
 *                 dD/dtheta = J_l(theta)^T GT/S;
 *   alpha_q <= 0: D = V, dD/dp = GP, dD/dtheta = J_l(theta)^T GT.
 * SD_ERR_INVALID_ARG for n <= 0, a NULL pointer, or (alpha_q > 0) only
 * empty shards; SD_ERR_NONFINITE for a non-finite pose.
 */
int sd_pose_merge(const double* parts, int32_t n, const double* pose, float alpha_q, double* out);

/*
 * Batched rigid bodies against one data mesh (the multi-object evaluation
 * behind Sec. 4.5's simulations): B bodies with uneven vertex counts,
 * flattened into one vertex list. sd_batch_run places every vertex from a
 * per-body pose table, orders all of them on one Hilbert curve, evaluates
 * them in ONE persistent traversal launch and reduces each body to
 * (D_b, dD_b/dp (3), dD_b/dtheta (3)) with D_b the outer LogSumExp of
 * Eq. lse_full2 over the body's vertices (as sd_pose_reduce).
 *   sd_batch_create: X0 device [M,3] rest vertices of all bodies (kept by
 *     pointer; must outlive the batch), offsets host int64 [B+1] with
 *     offsets[0] = 0 and at least one vertex per body. Allocates all the
 *     batch's device buffers and synchronises the device.
 *   sd_batch_set_poses: host double [B,6] poses (theta, p); copied to the
 *     device on `stream` before the call returns.
 *   sd_batch_run: alpha_q > 0; block = traversal block size (0 default);
 *     body_out device [B,7]. Enqueues work on `stream` only: no allocation
 *     and no synchronisation, so it can be captured in a CUDA graph.
 *   sd_batch_vertex_outputs: device pointers to the batch's placed vertices
 *     [M,3], d^ [M] and grad d^ [M,3] of the last run.
 */
typedef struct sd_batch sd_batch;
int sd_batch_create(const sd_tree* t, const float* X0, const int64_t* offsets, int32_t nbodies, sd_batch** out);
int sd_batch_set_poses(sd_batch* b, const double* poses, void* stream);
int sd_batch_run(sd_batch* b, float alpha_q, int32_t block, float* body_out, void* stream);
int sd_batch_vertex_outputs(const sd_batch* b, const float** X, const float** value, const float** grad);
void sd_batch_free(sd_batch* b);

/*
 * Learned far-field surrogate (an extension of the method; the paper has none).
 * A Fourier-feature MLP, parameters in one fp32 vector of
 * sd_mlp_num_params() floats laid out (B [32,3], W1 [128,67], b1, W2
 * [128,128], b2, W3 [128,128], b3, w4 [128], b4):
 *   xh = (x - c)/h per axis, f = [xh, sin(pi B xh), cos(pi B xh)],
 *   a_l = silu(W_l a_{l-1} + b_l) (l = 1..3), y = s (w4 . a3 + b4),
 * W_l and w4 used rounded to bfloat16 with fp32 accumulation.
 * frame = host float[7] = (c_x, c_y, c_z, h_x, h_y, h_z, s): box centre,
 * half extents (> 0) and output scale; SD_ERR_INVALID_ARG otherwise.
 *   sd_mlp_forward: device x [n,3] -> y [n] and, if dydx is not NULL,
 *     dy/dx [n,3] (tcgen05 tensor-core kernel, one CTA with 224,176 bytes (218.9 KiB) of shared
 *     memory and all 512 tensor-memory columns per SM; features, a1, a2 and
 *     the back-propagated factors rounded to bfloat16, dsilu(z1), dsilu(z2)
 *     to binary16; input gradient by back-propagation). If a bounded wait
 *     for a 128-query tile's tensor-core work runs out, that tile and every
 *     later tile of its warp group get NaN outputs: the group issues no
 *     more work and waits (bounded) for what it already committed before
 *     the tensor memory is freed.
 *   sd_mlp_train_step: one mean-squared-error step on a device batch
 *     (x [n,3], target [n]): writes loss (device [1]) and the gradient
 *     (device [num_params], zero for B); if lr > 0 also an Adam step (step
 *     >= 1, moments adam_m/adam_v device [num_params]) on every parameter but
 *     B. workspace: device, >= sd_mlp_workspace_bytes(n). Deterministic.
 */
int64_t sd_mlp_num_params(void);
size_t sd_mlp_workspace_bytes(int64_t n);
int sd_mlp_forward(const float* params, const float* frame, const float* x, int64_t n, float* y, float* dydx,
                   void* stream);
int sd_mlp_train_step(float* params, float* adam_m, float* adam_v, int32_t step, float lr, const float* frame,
                      const float* x, const float* target, int64_t n, float* loss, float* grad, void* workspace,
                      size_t ws_bytes, void* stream);

/*
 * Certified lower bound of the exact d^ (Eq. 3) from a cut of at most 64
 * top nodes of the tree (breadth-first from the root while the next level
 * has at most 64 nodes):
 *   LB(q) = -(1/alpha) ln sum_{B in cut} n_B w_B kappa^S e^{-alpha d(q, box B)}
 * with w_B the far-field weight (1 for points-only nodes, max(A_E, A_T)^S
 * otherwise) and kappa >= 1 a bound of the blending polynomials w~ (their
 * largest Bernstein coefficient, times 1.0001 for fp32), lowered by
 * 1e-3 + 1e-5 |LB| for fp32 rounding. It does not bound the Barnes-Hut
 * value: a far field taken at a node above the cut sits at a nearer box and
 * can fall below LB (both stay below the exact d^).
 * Writes device lb [M], lb_grad [M,3] (the gradient of LB before the
 * rounding allowance: sum_B softmax_B (q - y_B)/|q - y_B|, y_B the closest
 * point of box B, 0 inside a box) and flag [M] = (LB > margin); any of the
 * three may be NULL. Uses stream-ordered temporary memory.
 */
int sd_lower_bound(const sd_tree* t, const float* q, int64_t M, float margin, float* lb, float* lb_grad,
                   int32_t* flag, void* stream);

/*
 * Surrogate-routed query: queries whose certified lower bound exceeds
 * `margin` are answered by LB plus the MLP (the network models the residual
 * d^ - LB; value and gradient), all others by the Barnes-Hut traversal, so
 * the constraint near contact is always the method itself. routed (device
 * [M], may be NULL) receives 1 for surrogate answers; *n_routed (host, may
 * be NULL) their count. Synchronises `stream` once (to size the two
 * groups). Uses stream-ordered temporary memory.
 */
int sd_surrogate_query(const sd_tree* t, const float* params, const float* frame, float margin, const float* q,
                       int64_t M, float* value, float* grad, int32_t* routed, int64_t* n_routed, void* stream);

/*
 * Edge and triangle queries (Sec. 3.4): the smooth distance of Eq. 3 from
 * each of M query primitives g_j to the data mesh, with the simplex-simplex
 * distance of App. B, the weights taken at g_j's point of a closest pair,
 * and the Barnes-Hut test of Sec. 3.5 on g_j's axis-aligned box (the box
 * halfspaces g_j lies entirely outside of; the distance to the feature they
 * identify lower-bounded by the gap between the boxes).
 *   QV     device [nqv,3] float32 query-mesh vertices
 *   QF     device [M,k] int32 vertex indices; k = 1 (points), 2 (edges) or
 *          3 (triangles)
 *   value  device [M] d^(g_j); grad device [M,3] (may be NULL) its gradient
 *          for a rigid translation of g_j
 *   opts   as for sd_query (sort_queries orders by the Hilbert index of each
 *          primitive's centroid; order, block, counts as for sd_query)
 * A primitive with an index outside [0, nqv) or a non-finite vertex gets NaN
 * outputs and sets the status word (SD_ERR_INDEX / SD_ERR_NONFINITE).
 * Asynchronous; uses stream-ordered temporary memory.
 */
int sd_query_prims(const sd_tree* t, const float* QV, int64_t nqv, const int32_t* QF, int32_t k, int64_t M,
                   float* value, float* grad, const sd_query_opts* opts, void* stream);

/*
 * Smooth distance between the data mesh and a query mesh (Sec. 3.6,
 * Eq. lse_full) from sd_query_prims' outputs, and its gradient per query
 * vertex (Eq. lse_full2 / Eq. dlse_full: each primitive's softmin share
 * split equally between its k vertices):
 *   out    device [1]: D = -(1/alpha_q) log sum_j exp(-alpha_q d^_j)
 *   vgrad  device [nqv,3] (may be NULL): dD/dv_k; vertices used by no
 *          primitive get 0; indices outside [0, nqv) are ignored
 *   status device int (may be NULL): never written (kept for the ABI; the
 *          vertex sort's bounded waits fall back to an exact direct count)
 * Sums run in a fixed order (deterministic). Asynchronous; uses
 * stream-ordered temporary memory.
 */
int sd_mesh_reduce(const int32_t* QF, int32_t k, int64_t M, int64_t nqv, const float* value, const float* grad,
                   float alpha_q, float* out, float* vgrad, int32_t* status, void* stream);

/*
 * Sphere tracing of the zero isosurface of d^ (Sec. 4.2; Hart 1996) through
 * a pinhole camera. Pixel (row i from the top, column j) looks along
 * normalize(f + x r + y u), f the unit view direction (target - eye), r the
 * unit f x up, u = r x f, x = ((j + 0.5) / W * 2 - 1) tan(fov_y / 2) W / H,
 * y = (1 - (i + 0.5) / H * 2) tan(fov_y / 2). Each ray starts at t = 0 from
 * eye; at every step d^(eye + t dir) is evaluated (Barnes-Hut with the
 * tree's alpha and beta, value only): d^ < eps is a hit at depth t,
 * otherwise t += d^, and the ray misses once t > t_max or after max_steps
 * evaluations.
 *   depth  device [H*W] float32, row-major: hit depth, +inf for a miss
 *   steps  device [H*W] int32 (may be NULL): evaluations spent on the ray
 *   evaluations host int64 (may be NULL): evaluations over all rays
 * Synchronises `stream` once per step (to size the next wavefront). Uses
 * stream-ordered temporary memory.
 */
typedef struct {
    float eye[3], target[3], up[3];
    float fov_y;          /* vertical field of view, radians, (0, 3.1) */
    int32_t width, height;
    float eps;            /* > 0 */
    float t_max;          /* > 0 */
    int32_t max_steps;    /* > 0 */
    int32_t block;        /* traversal block size, a multiple of 32 up to 256; 0 = default */
} sd_trace_opts;
int sd_sphere_trace(const sd_tree* t, const sd_trace_opts* opts, float* depth, int32_t* steps, int64_t* evaluations,
                    void* stream);

/* Synchronise `stream`, return and clear the tree's device status word. */
int sd_query_status(const sd_tree* t, void* stream);

typedef struct {
    int64_t n_prims, n_points, n_edges, n_tris;
    int64_t n_buckets;   /* leaf buckets nb = ceil(n/L); internal nodes nb - 1 */
    int32_t leaf_size;
    float alpha, beta, alpha_u, S;
    float A_E, A_T;      /* scale A of App. C.2 / C.3 (1 when the part is empty) */
    float w_far;         /* far-field weight max(A_E, A_T)^S for nodes holding an edge or triangle */
    float scene_lo[3], scene_hi[3];
    int64_t device_bytes;
} sd_tree_info;

int sd_tree_get_info(const sd_tree* t, sd_tree_info* info);

/* Host copies of the build's results, for tests. Every pointer is a host
   array the caller allocated with the size given (n = n_prims, nb =
   n_buckets, ni = nb - 1), or NULL to skip it.
     codes    [n]    uint64 Morton code of each primitive (original order)
     sorted   [n]    int32 original index of the primitive at each sorted position
     left/right [ni] int32 children of internal node i (Karras numbering; a
                     leaf child b is stored as -(b + 1))
     node_lo/node_hi [ni,3], node_count [ni]   internal node AABB and n_B
     leaf_lo/leaf_hi [nb,3], leaf_count [nb]   bucket AABB and n_B
     params   [n,2]  float per-primitive weight parameters in original order:
                     edges (1/|N_i0|, 1/|N_i1|), triangles (1/v_i, 1/e_i), points (0,0) */
typedef struct {
    uint64_t* codes; int32_t* sorted;
    int32_t* left; int32_t* right;
    float* node_lo; float* node_hi; int32_t* node_count;
    float* leaf_lo; float* leaf_hi; int32_t* leaf_count;
    float* params;
} sd_tree_view;

int sd_tree_export(const sd_tree* t, sd_tree_view* view);

/* Release the tree (synchronises the device). NULL is a no-op. */
void sd_free(sd_tree* t);

/* Number of CUDA kernels this library has launched in this process. */
int64_t sd_kernel_launches(void);

/* Static text for a status code; sd_last_error() holds the last CUDA error
   text seen by this thread. */
const char* sd_status_str(int status);
const char* sd_last_error(void);

/*
 * Host-only: the library's triangle weight basis (App. C.3) in Bernstein
 * form. out[3*36]: for unit right-hand sides (1/v, 1/e, (v-1)/v) in that
 * order, the 36 Bernstein-Bezier coefficients b_ijk of the degree-7
 * polynomial, (i,j,k) = exponents of (phi0, phi1, phi2), i+j+k = 7, in the
 * order i = 7..0 outer, j = 7-i..0 inner. Needs no GPU.
 */
int sd_weight_basis(double* out);

/*
 * Host-only: the same weights as the tables the kernels evaluate (App. C.3
 * has no evaluation scheme; this is the library's). For every class (v, e)
 * of vertex valence v = 1..16 and edge valence e = 1..4 (the blended
 * w~ = (1/v) P_V + (1/e) P_E + ((v-1)/v) P_B) and each orientation o = 0, 1,
 * 2 (phi_o, the largest barycentric, as the base variable; x, y the other
 * two, lower index first, divided by phi_o), 92 floats: 36 coefficients
 * c_ab with w~ = phi_o^7 sum c_ab x^a y^b, then 28 with
 * dw~/dphi1 = phi_o^6 sum c_ab x^a y^b and 28 with dw~/dphi2 likewise
 * (phi0 = 1 - phi1 - phi2), each c_ab a Bernstein coefficient times its
 * multinomial, in Horner order (powers of y from 7 or 6 down, within each
 * the powers of x from high to low). out[16 * 4 * 3 * 92], class (v, e),
 * orientation o at offset (((v - 1) * 4 + (e - 1)) * 3 + o) * 92. Computed
 * in FP64, rounded to fp32 once. Needs no GPU.
 */
int sd_weight_horner_tables(float* out);

/*
 * Pipe-throughput probe (a measurement aid; the paper has no counterpart).
 * The traversal is bound by the FP32 pipe with the MUFU (special-function)
 * pipe as a co-bound; this measures both rates at whatever clock the GPU
 * runs, as the roofline's denominators.
 *   kind   0: fma.rn.f32; 1: fma.rn.f32x2 (two FMAs per lane and
 *          instruction); 2: ex2.approx.ftz.f32 (each followed by one FMA on
 *          the FP32 pipe that keeps the chain bounded)
 *   blocks > 0 blocks of 256 threads; each thread runs iters x 16 steps of
 *          8 independent dependency chains
 *   sink   device [blocks*256] float32 output (keeps the chains live)
 *   ops    host: lane operations of the launch (FMAs, or exponentials)
 * Asynchronous on `stream`: time the launch with CUDA events. An FMA is
 * 2 flops. SD_ERR_INVALID_ARG for an unknown kind or a non-positive size.
 */
int sd_peak_probe(int32_t kind, int32_t blocks, int32_t iters, float* sink, double* ops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SD_H_ */
