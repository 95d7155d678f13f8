/*
 * reg.h - C ABI of the GB300 registration-scan library (libreg.so).
 *
 * The library registers every frame f_1..f_{N-1} of an image series to the
 * first frame f_0 by an inclusive prefix scan with the operator
 *
 *     phi_ij (.)_B phi_jk = B(phi_ij, phi_jk)                 [Sec. 3]
 *
 * where B composes the two known deformations into an initial guess
 * phi_jk o phi_ij and then minimises the normalised-cross-correlation
 * distance D(f_i, f_k o phi) by gradient flow on a coarse-to-fine pyramid
 * [Sec. 2.3.1, Sec. 2.3.2].  The neighbour registrations
 * A(f_{i-1}, f_i) start from the identity.
 *
 * Deformation models:
 *   REG_RIGID     phi(x) = Rot(alpha) (x - c) + c + G, c = ((W-1)/2, (H-1)/2),
 *                 pixel (r, c) at x = (c, r)                         [Sec. 2.3.1]
 *   REG_NONRIGID  phi(x) = x + u(x), u bilinear in control displacements c_j on
 *                 a grid of spacing s (finest pixels) at points (jx s, jy s),
 *                 jx < nx = ceil((W-1)/s) + 1; energy 1 - NCC + lambda/(2P) sum over
 *                 control-grid edges |c_a - c_b|^2 (an extension: the paper's
 *                 deformation is rigid).  Both frames enter this energy through the
 *                 quadratic B-spline model of their samples (extended by the mean), a
 *                 continuously differentiable image; the rigid energy samples the
 *                 frames bilinearly.  Control values are stored as (x, y) float
 *                 pairs, row-major [ny][nx]; dense fields as planes [2][H][W].
 *
 * Conventions common to every entry point:
 *   - Return value: REG_OK (0) or a negative REG_E* code; reg_strerror()
 *     names it and reg_last_error_message() gives the detail of the last
 *     failure on the calling thread.  Non-convergence is not an error: it is
 *     reported in reg_stats_t.stop[].
 *   - Pointers are host or device memory as stated per argument; where
 *     "host or device" is allowed the library detects the kind.
 *   - Caller-owned buffers are only borrowed for the duration of the call
 *     (the call returns after its work on `stream` has completed).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).
 *   - All computation runs in the library's CUDA kernels (sm_103a); there is
 *     no CPU fallback.  Without a usable GPU every compute entry point
 *     returns REG_ECUDA.
 *   - Every wait inside a kernel is bounded.  The persistent executor's wait
 *     for a ready operator gives up after 20 s (REG_QUEUE_TIMEOUT_MS in the
 *     environment overrides it), and reg_scan then returns REG_ETIMEOUT with the
 *     context still usable.  For tests, REG_FAULT_INJECT=stuck_op in the
 *     environment makes one operator of the next persistent reg_scan wait for
 *     an input that never arrives.
 */
#ifndef REG_H
#define REG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define REG_OK        0
#define REG_EINVAL   -1   /* bad argument (size, pointer, mode, adjacency of B's inputs) */
#define REG_ENOMEM   -2   /* device or host allocation failed */
#define REG_EBUDGET  -3   /* stream admission refused: memory budget or slots full; retry later */
#define REG_ETIMEOUT -4   /* a bounded wait gave up (device queue or host poll) */
#define REG_ECUDA    -5   /* CUDA runtime error, or no usable GPU */
#define REG_ESTATE   -6   /* object used in the wrong state */

/* ---- enums ------------------------------------------------------------ */
#define REG_RIGID    0
#define REG_NONRIGID 1

#define REG_F32  0        /* pyramid storage type; arithmetic is always FP32 */
#define REG_BF16 1
#define REG_F16  2

#define REG_SCHED_SEQ           0   /* left fold phi_{0,i} = phi_{0,i-1} (.) phi_{i-1,i}   [Sec. 3] */
#define REG_SCHED_BRENT_KUNG    1   /* work-efficient tree scan                        [Table 1] */
#define REG_SCHED_DISSEMINATION 2   /* recursive doubling, depth log2 N                [Table 1, Fig. 2] */
#define REG_SCHED_LADNER_FISCHER 3  /* Ladner-Fischer P_0                              [Table 1] */
#define REG_SCHED_BLELLOCH      4   /* exclusive tree scan with the identity      [Table 1]; mock only */
/* online scan with a look-back of k leaves: window products of the last k leaves by doubling,
 * prefix p_j = p_{j-k} (.) (x_{j-k+1} .. x_j), so k chains of prefixes advance side by side
 * (p_j = p_{j-1} (.) x_j for j < k); the streaming service's schedule, see reg_stream_set_lookback */
#define REG_SCHED_LOOKBACK_2    17
#define REG_SCHED_LOOKBACK_4    18
#define REG_SCHED_LOOKBACK_8    19

#define REG_EXEC_PLAIN      0   /* one operator per kernel launch, DAG order on a stream pool */
#define REG_EXEC_LEVEL      1   /* one launch per DAG depth, all its operators batched */
#define REG_EXEC_PERSISTENT 2   /* one persistent launch, device ready-queue over the DAG */
#define REG_EXEC_GRAPH      3   /* the REG_EXEC_PLAIN launches captured once per plan as a CUDA
                                   graph and replayed: same kernels, same results, no per-call
                                   launch cost.  The graph is rebuilt when N, the schedule, the
                                   frame geometry or a workspace changes. */

/* OR into `exec` of reg_scan / reg_scan_batch (not with REG_EXEC_GRAPH): every neighbour
 * operator A runs to completion before the first B, and with timing enabled the two phases are
 * timed separately (reg_timing_t.leaf_ms, dag_ms).  The paper reports the scan of B alone and
 * the full registration with the A's before it (Sec. 5.2, its scan and full speedup bounds). */
#define REG_EXEC_SPLIT_PHASES 0x100

#define REG_MAX_LEVELS 8

/* why a level stopped (reg_stats_t.stop) */
#define REG_STOP_GRAD    0   /* metric gradient norm below tol_grad */
#define REG_STOP_REL     1   /* accepted step lowered E by less than tol_rel_e * |E| */
#define REG_STOP_LS      2   /* line search exhausted max_rejects rejected trials */
#define REG_STOP_MAXIT   3   /* max_iter accepted steps */

/* ---- data types --------------------------------------------------------- */

/* Scan element: deformation plus indices, 20 bytes [Sec. 5: the data a rank
 * exchanges per element].  Rigid parameters (alpha in radians, G in
 * pixels of the finest level).  For REG_NONRIGID the field lives in a separate
 * buffer and alpha/gx/gy hold the field's mean displacement (alpha = 0). */
typedef struct {
    int32_t i, k;        /* phi_{i,k}: f_k o phi ~ f_i */
    float alpha, gx, gy;
} reg_elem_t;

typedef struct {
    int    mode;          /* REG_RIGID or REG_NONRIGID */
    int    levels;        /* pyramid levels, 1..REG_MAX_LEVELS */
    int    max_iter;      /* accepted gradient-flow steps per level */
    int    max_rejects;   /* rejected Armijo trials allowed per step */
    double tol_grad;      /* stop: metric norm of the descent direction (default 3e-5) */
    double tol_rel_e;     /* stop: relative energy decrease of an accepted step; 0 (default)
                             stops only on an accepted step that does not lower E at all */
    double armijo_c;      /* sufficient-decrease constant */
    double tau0;          /* first trial step of each level */
    double step_cap;      /* largest step, pixels of the current level */
    double lambda;        /* regulariser weight (REG_NONRIGID) */
    int    storage;       /* REG_F32, REG_BF16 or REG_F16 pyramid storage */
    int    cluster;       /* CTAs cooperating on one operator (1,2,4,8,16); 0 = auto */
    int    workers;       /* persistent executor: operator slots in flight; 0 = auto */
    size_t mem_budget;    /* stream service: device bytes it may hold; 0 = unlimited */
    int    grid;          /* REG_NONRIGID control-grid spacing in finest pixels; 0 = auto (16,
                             doubled until at most 65 points per axis); a multiple of 2^(levels-1) */
    int    metric;        /* REG_NONRIGID scalar product of the gradient flow: REG_METRIC_GAUSS_NEWTON
                             (default), REG_METRIC_MEAN or REG_METRIC_H1 */
    int    unroll;        /* REG_NONRIGID energy passes: pixels in flight per lane (2 or 4); 0 = auto
                             (the autotuned value, else 4) */
    int    ctas_per_sm;   /* REG_NONRIGID operator kernels: register budget sized for 3 or 4 CTAs
                             per SM (80 or 64 registers a thread); 0 = auto (the autotuned value,
                             else 4 for 16-CTA operators and 3 below) */
    double sigma;         /* REG_METRIC_H1: smoothing length in control-grid spacings (>= 0; default 1) */
    double tol_coarse;    /* stop at every level above the finest: tol_coarse x tol_grad (a coarse
                             level only supplies the next level's initial guess); in [1, 1e6],
                             default 10 */
} reg_config_t;

/* Scalar product of the nonrigid gradient flow [Sec. 2.3.1 takes the flow with respect to a
 * scalar product it does not fix].  REG_METRIC_MEAN: the mean over control points.
 * REG_METRIC_GAUSS_NEWTON: per level, each control point and axis weighted by the Gauss-Newton
 * curvature of the data term at the level's initial deformation, sum_x w_j(x)^2 (dT/dp)^2 /
 * (P var T), plus the regulariser's lambda n_j / P (n_j neighbours), normalised by the mean and
 * floored at 1e-3 of it: each control point's step is scaled by its own curvature. */
#define REG_METRIC_MEAN         0
#define REG_METRIC_GAUSS_NEWTON 1
/* REG_METRIC_H1: <u, v> = (1/Nc) u^T (I + sigma^2 Lg) v per axis, Lg the Laplacian of the control
 * grid's graph (the neighbour edges the regulariser sums over): the flow's direction is the
 * gradient smoothed over about sigma grid spacings, d = -Nc (I + sigma^2 Lg)^-1 dE/dc.  Available
 * to reg_scan, reg_scan_batch and reg_pairwise (not to streams or reg_pairwise_noalloc: REG_EINVAL). */
#define REG_METRIC_H1           2

typedef struct {
    int32_t i, k;                      /* the element this operator produced */
    int32_t iters[REG_MAX_LEVELS];     /* accepted steps per level, index 0 = finest */
    int32_t evals[REG_MAX_LEVELS];     /* energy evaluations per level */
    int32_t stop[REG_MAX_LEVELS];      /* REG_STOP_* per level */
    int32_t rejects;                   /* Armijo rejections, all levels */
    int32_t status;                    /* REG_OK, or a device-side error code */
    double  energy;                    /* energy at the result, finest level */
    double  theta[3];                  /* the result: rigid (alpha, Gx, Gy) in FP64; nonrigid
                                          (0, mean u_x, mean u_y) */
} reg_stats_t;

typedef struct reg_ctx reg_ctx_t;
typedef struct reg_stream reg_stream_t;

typedef struct {
    uint64_t frame_id;     /* id given at submit */
    reg_elem_t elem;       /* phi_{0,i} of that frame (i = its position in the stream) */
    double submit_us;      /* host clock (us) at submit */
    double done_us;        /* host clock (us) when the result was seen complete */
    int32_t status;
} reg_result_t;

/* ---- configuration and context ----------------------------------------- */

/* Fill *cfg with the defaults (rigid, 2 levels, FP32 storage, auto tiles; stop on a metric
 * gradient norm below 3e-5, at most 500 accepted steps per level; Gauss-Newton scalar product
 * for the nonrigid flow). */
void reg_config_default(reg_config_t *cfg);

/* Create a context on CUDA device `device`.  The context owns its pyramids,
 * queues and workspaces; destroy it with reg_ctx_destroy.  Errors: REG_EINVAL
 * (bad config), REG_ECUDA (no device / no sm_103a GPU), REG_ENOMEM. */
int reg_ctx_create(const reg_config_t *cfg, int device, reg_ctx_t **out);
void reg_ctx_destroy(reg_ctx_t *ctx);

/* ---- the operators ------------------------------------------------------ */

/* Register template T onto reference R (A when init == NULL, else the
 * minimisation of B from `init`) [Sec. 2.3.1].
 *   R, T       fp32 images, H rows of `pitch` elements (pitch >= W), host or device.
 *   init       rigid initial deformation (host), NULL = identity.
 *   field_in   REG_NONRIGID initial field [2][H][W] fp32 (x plane then y), host or
 *              device, NULL = identity.
 *   out        result (host), i = 0, k = 1.
 *   field_out  REG_NONRIGID result field [2][H][W] (host or device); may be NULL
 *              for REG_RIGID.
 *   stats      optional (host).
 * Errors: REG_EINVAL (W or H < 2 at the coarsest level, pitch < W, NULL R/T/out). */
int reg_pairwise(reg_ctx_t *ctx, const float *R, const float *T, int W, int H, int pitch,
                 const reg_elem_t *init, const float *field_in,
                 reg_elem_t *out, float *field_out, reg_stats_t *stats, void *stream);

/* Register all frames to f_0 by the scan [Sec. 3]: the N-1 neighbour
 * operators A(f_{i-1}, f_i), then B along the DAG of `schedule`.
 *   frames     fp32 [N][H][pitch], host or device.  Host frames are staged on the device:
 *              page-locked memory mapped at the same address (cudaHostAlloc, or
 *              torch's pin_memory) is read over the CPU-GPU link by a copy kernel,
 *              other host memory is copied by cudaMemcpyAsync.
 *   out        N-1 elements phi_{0,1}..phi_{0,N-1} (host or device).
 *   fields_out REG_NONRIGID: [N-1][2][H][W] fp32 (host or device), or NULL to skip
 *              the dense fields (reg_scan_grids then gives the control values).
 *              NULL for rigid.
 *   per_op     optional host array of (N-1) + (#B operators of the schedule)
 *              stats, leaves first, then the B operators in DAG order
 *              (reg_scan_work() gives the count).
 * Errors: REG_EINVAL, REG_ENOMEM, REG_ECUDA, REG_ETIMEOUT (persistent queue). */
int reg_scan(reg_ctx_t *ctx, const float *frames, int N, int W, int H, int pitch,
             int schedule, int exec, reg_elem_t *out, float *fields_out,
             reg_stats_t *per_op, void *stream);

/* S independent series of N frames each (same W, H) registered in one call: the
 * operators of all series share the executor's launches (and, with
 * REG_EXEC_PERSISTENT, one device queue), so series with uneven iteration counts
 * fill the GPU together.  Each series is the scan of reg_scan [Sec. 3].
 *   frames     fp32 [S][N][H][pitch], host or device (host frames staged as in reg_scan).
 *   out        S x (N-1) elements, series-major; indices i, k are series-local.
 *   fields_out REG_NONRIGID: [S][N-1][2][H][W] or NULL.
 *   per_op     optional host array of S x (the per-series count of reg_scan),
 *              series-major, frame indices series-local.
 * reg_scan_grids afterwards returns S x (N-1) control grids.  Errors as reg_scan. */
int reg_scan_batch(reg_ctx_t *ctx, const float *frames, int S, int N, int W, int H, int pitch,
                   int schedule, int exec, reg_elem_t *out, float *fields_out,
                   reg_stats_t *per_op, void *stream);

/* Control values of the N-1 prefixes phi_{0,1}..phi_{0,N-1} of the last
 * successful REG_NONRIGID reg_scan on ctx: grids_out, device, [N-1][ny][nx]
 * (x, y) pairs, ny/nx from reg_grid_dims for that scan's W, H.  n_out (host,
 * optional) receives N-1.  A later reg_pairwise or reg_energy on ctx ends the
 * availability.  Errors: REG_ESTATE if ctx has no nonrigid scan result;
 * REG_EINVAL for a host grids_out. */
int reg_scan_grids(reg_ctx_t *ctx, float *grids_out, int *n_out, void *stream);

/* Control values of chosen operators' results of the last successful REG_NONRIGID reg_scan
 * or reg_scan_batch on ctx (inspection of the scan's intermediate deformations, e.g. a B
 * operator's inputs).  ops (host) holds n operator indices in the per_op order of that call:
 * leaves A(f_j, f_{j+1}) first, then the B operators in DAG order (series-major for a batch).
 * grids_out: device, [n][ny][nx] (x, y) pairs.  A later reg_pairwise or reg_energy on ctx
 * reuses the node storage and ends the availability.  Errors: REG_ESTATE without such a
 * result; REG_EINVAL for an index out of range or a host grids_out. */
int reg_scan_node_grids(reg_ctx_t *ctx, const int32_t *ops, int n, float *grids_out, void *stream);

/* Registered series and its average [Sec. 2: every frame of the series is
 * registered to the first one, then the series is averaged].
 *   out_k(x) = f_k(phi_{0,k}(x)), k = 0..N-1 (phi_{0,0} = identity), bilinear
 *   with clamp-to-edge, the sampling of the operator; mean(x) = (1/N) sum_k out_k(x),
 *   summed per chunk of 64 frames with compensation and over chunks in FP64, in
 *   a fixed order (bitwise reproducible).
 *   frames   device fp32 [N][H][pitch], N >= 1.
 *   elems    REG_RIGID: the N-1 prefixes from reg_scan (host or device), element
 *            k-1 = phi_{0,k}.  Ignored for REG_NONRIGID.
 *   grids    REG_NONRIGID: device [N-1][ny][nx] (x, y) control values of the
 *            prefixes, as reg_scan_grids writes them.  Ignored for REG_RIGID.
 *   out      device [N][H][W] fp32, or NULL.   mean  device [H][W] fp32, or NULL.
 * Source tiles are staged in shared memory by TMA when frames is 16-byte
 * aligned, pitch % 4 == 0 and W >= 80, H >= 40; otherwise samples are read from
 * global memory (same results).  The call returns after its work on `stream`
 * has completed.  Errors: REG_EINVAL (NULL or host frames/grids, both outputs
 * NULL, N < 1, W or H < 2), REG_ETIMEOUT (a bounded wait on a TMA load gave up),
 * REG_ECUDA. */
int reg_warp(reg_ctx_t *ctx, const float *frames, int N, int W, int H, int pitch,
             const reg_elem_t *elems, const float *grids, float *out, float *mean, void *stream);

/* Mock operator on the device executors [Sec. 5.1: an artificial operator of fixed or
 * exponentially distributed running time, to study the scan algorithms and the balance of their
 * load apart from the registration].  Element j holds values[j]; an operator of the schedule's
 * DAG adds its two inputs after spinning for its duration on the device clock, on one CTA.
 *   values     host, n doubles.
 *   op_us      host, one duration per operator of the DAG in DAG order (reg_scan_dag), in
 *              microseconds, each in [0, 1e5]; the caller draws them (fixed, or exponential
 *              with mean t for the paper's dynamic configuration).
 *   exec       REG_EXEC_PLAIN, REG_EXEC_LEVEL or REG_EXEC_PERSISTENT.
 *   prefix     host, n doubles: the inclusive prefix sums; for REG_SCHED_BLELLOCH the exclusive
 *              ones (prefix[0] = 0, the identity).
 *   elapsed_ms host, optional: device time of the operator phase (CUDA events).
 * Errors: REG_EINVAL (n < 1, a duration out of range, unknown schedule or executor). */
int reg_mock_scan(reg_ctx_t *ctx, int n, int schedule, int exec, const double *values, const float *op_us,
                  double *prefix, double *elapsed_ms);

/* Number of B applications the schedule uses for n = N-1 elements (host only,
 * no GPU needed).  Returns -1 for an unknown schedule. */
int reg_scan_work(int schedule, int n);

/* Write the schedule's DAG in SSA form (host only): op j creates node n+j =
 * node[left[j]] (.) node[right[j]]; out_node[i] holds x_0 (.) ... (.) x_i.
 * Arrays sized by reg_scan_work() and n.  Returns the op count or -1. */
int reg_scan_dag(int schedule, int n, int32_t *left, int32_t *right, int32_t *out_node);

/* Allocation-free rigid pairwise registration (the paper has no counterpart:
 * this serves callers that may not allocate device memory when they register,
 * e.g. a real-time acquisition loop where cudaMalloc/cudaFree would stall the
 * device, or an application that hands the GPU a fixed memory budget up front).
 * Same result as reg_pairwise for REG_RIGID, computed without any allocation:
 * pyramids and operator state live in one file-scope device array of about
 * 12.2 MB, sized for frames of at most 1,048,576 pixels (W, H <= 4096), which
 * every GPU that loads libreg keeps until the process exits.
 *   cfg      configuration (host); mode must be REG_RIGID; the other fields are
 *            checked by the rules of reg_ctx_create.
 *   device   CUDA device to run on (made current for the call, then restored).
 *   R, T     fp32 images, H rows of `pitch` elements, in device memory of `device`
 *            (or managed memory); host memory and memory of another GPU are
 *            rejected (REG_EINVAL): staging or peer access would need allocations.
 *   init     host, NULL = identity.  out (host) receives phi; stats (host) optional.
 *   stream   a stream of `device` (REG_EINVAL otherwise), or NULL.
 * Errors: REG_EINVAL for a nonrigid or otherwise invalid config, sizes beyond the
 * limit (with a message naming it), host, foreign-device or NULL pointers, a stream
 * of another device; REG_ECUDA for CUDA failures.
 * The first call for a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current.  The call waits for `stream`
 * several times (the level means come back to the host between the pyramid and the
 * operator) and returns after its work has completed, so it must not be made while
 * `stream` is being captured into a CUDA graph.  Every call shares the one array
 * and overwrites what the previous call left there: calls that overlap on the GPU
 * (other host threads, other streams) race and must be serialised by the caller. */
int reg_pairwise_noalloc(const reg_config_t *cfg, int device, const float *R, const float *T, int W, int H,
                         int pitch, const reg_elem_t *init, reg_elem_t *out, reg_stats_t *stats, void *stream);

/* ---- kernel-level entry points (one hot-path step each) ------------------- */

/* Pyramid build [Sec. 2.3.1, multilevel scheme]: 2x2 box average per level,
 * odd last row/column clamped.  frame: device fp32 [H][pitch].  out: device,
 * levels packed level 0 first, each W_l x H_l contiguous, in `storage` type
 * (4 or 2 bytes per pixel).  Returns REG_EINVAL for levels outside 1..8. */
int reg_pyramid(reg_ctx_t *ctx, const float *frame, int W, int H, int pitch,
                int levels, int storage, void *out, void *stream);

/* Energy and gradient at a given deformation (one fused warp+reduction pass,
 * as used inside the iteration) [Sec. 2.3.1].  R, T device or host fp32 [H][W].
 *   REG_RIGID:    theta[3] (host) = (alpha, Gx, Gy); grad[3] (host, optional).
 *   REG_NONRIGID: grid_values: control values [ny][nx] (x, y) pairs, device;
 *                 grad_values: dE/dc in the same layout, device, optional.
 *                 lambda and grid spacing from the context configuration.
 *   energy (host): E. */
int reg_energy(reg_ctx_t *ctx, const float *R, const float *T, int W, int H,
               const double *theta, const float *grid_values, double *energy,
               double *grad, float *grad_values, void *stream);

/* Control grid of a W x H frame for spacing `grid` (0 = auto) and `levels` (host only).
 * REG_EINVAL when the spacing is negative or not a multiple of 2^(levels-1), when the grid
 * has fewer than 2 x 2 points, or when one operator's grid state (4 x 8 B per point plus a
 * 16-byte control row per warp) would exceed 216 KB of shared memory. */
int reg_grid_dims(int W, int H, int grid, int levels, int *nx, int *ny, int *spacing);

/* Nonrigid composition at the control points (B's initial guess, Sec. 2.3.2):
 * out_j = q1_j + u2(X_j + q1_j), u2 the field of q2.  Device [ny][nx] (x, y) pairs. */
int reg_compose_grid(reg_ctx_t *ctx, const float *q1, const float *q2, int W, int H,
                     float *out, void *stream);

/* ---- streaming service ----------------------------------------------------- */

/* Open an acquisition stream of W x H fp32 frames.  The first submitted frame
 * is f_0; each later frame f_i yields phi_{0,i} via A(f_{i-1}, f_i) and
 * B(phi_{0,i-1}, phi_{i-1,i}), run on the device while other frames and other
 * streams are in flight.  Errors: REG_EBUDGET if the stream's resident state
 * does not fit the context's memory budget. */
int reg_stream_open(reg_ctx_t *ctx, int W, int H, reg_stream_t **out);

/* Submit one frame (host or device, [H][W] fp32; copied before return).
 * REG_EBUDGET: no slot or memory free right now; retry after polling. */
int reg_stream_submit(reg_stream_t *s, const float *frame, uint64_t frame_id);

/* The online scan of the stream (call before the first submit): with a look-back of k leaves
 * (k in {1, 2, 4, 8}; default 1, the sequential recursion phi_{0,i} = B(phi_{0,i-1}, A_i)), frame
 * i also brings the window operators of REG_SCHED_LOOKBACK_k and its prefix is
 * phi_{0,i} = B(phi_{0,i-k}, phi_{i-k,i}), so k chains of prefixes advance side by side: a stream
 * whose single B takes longer than its frame interval keeps up with about k times the rate, at
 * 1 + log2 k extra B operators per frame.  The results equal reg_scan with that schedule.
 * Errors: REG_EINVAL for another k; REG_ESTATE after the first submit. */
int reg_stream_set_lookback(reg_stream_t *s, int k);

/* REG_NONRIGID streams: the control values of every result, not only its mean displacement.
 * ring: caller-owned device memory of `capacity` grids [capacity][ny][nx] (x, y) pairs (ny, nx
 * from reg_grid_dims for the stream's W, H and the context's configuration).  The control values
 * of phi_{0,i} are in ring[i % capacity] by the time frame i's result is reported by
 * reg_stream_poll (elem.k = i; f_0 gets the identity), and stay there until the result of frame
 * i + capacity is computed: capacity must cover the frames in flight plus those not yet
 * consumed.  Call before the first submit.  Errors: REG_EINVAL for a rigid stream, a host ring
 * or capacity < 1; REG_ESTATE after the first submit. */
int reg_stream_grids(reg_stream_t *s, float *ring, int capacity);

/* Collect up to `max` finished results in submission order; waits up to
 * timeout_us for at least one (0 = do not wait).  *n_out = number written.
 * REG_ETIMEOUT if none finished in time (n_out = 0). */
int reg_stream_poll(reg_stream_t *s, reg_result_t *out, int max, int *n_out, int timeout_us);

/* Finish all submitted frames and release the stream. */
int reg_stream_close(reg_stream_t *s);

/* ---- autotuner ----------------------------------------------------------- */

/* Choose the launch shape of the operator kernels (the "tile") for this frame size, mode,
 * storage type and executor, by timing reg_scan on `frames` (each candidate twice, after one
 * untimed run; nonrigid scans are timed without dense fields, whose kernel costs the same for
 * every candidate) and keeping the fastest:
 *   1. CTAs per operator (rows of each pyramid level per CTA): 1, 2, 4, 8 and 16, for
 *      REG_NONRIGID each with either register form (3 or 4 CTAs per SM);
 *   2. REG_NONRIGID, at the chosen pair: pixels per lane of the energy passes (4, then 2).
 * Fields of cfg that are set (cluster, unroll, ctas_per_sm > 0) are not tuned.  Later reg_scan
 * calls on the context with a matching shape (same W, H, mode, storage, executor and
 * floor(log2 N)) use the choice for every field the config leaves at 0.  Arguments as reg_scan;
 * best (host, optional) receives the CTAs per operator.  A candidate the device cannot schedule
 * ends the search with the choices so far.  The paper has no counterpart (its operator runs on
 * one CPU core). */
int reg_autotune(reg_ctx_t *ctx, const float *frames, int N, int W, int H, int pitch,
                 int schedule, int exec, int *best);

/* The autotuned shape for (N, W, H, exec) at the context's mode and storage (host outputs,
 * each optional): CTAs per operator, energy-pass pixels per lane (0 for REG_RIGID) and the
 * register form.  REG_EINVAL if there is none. */
int reg_autotune_get(reg_ctx_t *ctx, int N, int W, int H, int exec, int *cluster, int *unroll,
                     int *ctas_per_sm);

/* Write / read the context's autotuned choices as JSON lines (host files). */
int reg_autotune_save(reg_ctx_t *ctx, const char *path);
int reg_autotune_load(reg_ctx_t *ctx, const char *path);

/* ---- measurement ----------------------------------------------------------- */

/* Device-side accounting of the last reg_scan / reg_pairwise call on a context. */
typedef struct {
    int32_t op_launches;       /* operator-kernel launches */
    int32_t pyramid_launches;  /* pyramid-build launches (level copy, box averages, level means) */
    double  op_kernel_ms;      /* device time of the operator kernels: CUDA events recorded on the
                                  launching stream around each launch (per-DAG-depth executor) or
                                  around the whole operator phase (stream-pool and persistent
                                  executors); 0 unless timing is enabled */
    double  pyramid_ms;        /* device time of the pyramid build, same method */
    int32_t graph_captures;    /* REG_EXEC_GRAPH: 1 if this call captured a new graph, 0 if it
                                  replayed the cached one (always 0 for the other executors) */
    int32_t tma_staged;        /* reg_warp: 1 if the source tiles were staged in shared memory
                                  by TMA, 0 if sampled from global memory */
    int32_t leaf_ops, dag_ops; /* REG_EXEC_SPLIT_PHASES: operators A (DAG depth 0) and B */
    double  leaf_ms, dag_ms;   /* REG_EXEC_SPLIT_PHASES with timing: device time of the A phase and
                                  of the B phase (same method as op_kernel_ms) */
    int32_t cluster;           /* launch shape of the last operator launch: CTAs per operator, */
    int32_t unroll;            /* energy-pass pixels per lane (0 for REG_RIGID), */
    int32_t ctas_per_sm;       /* and the register form (CTAs per SM it is sized for) */
    int32_t h2d_path;          /* host frames staged by: 0 none (device frames), 1 cudaMemcpyAsync,
                                  2 the SMs reading mapped page-locked memory */
    double  h2d_ms;            /* with timing: device time of that staging (0 for device frames) */
} reg_timing_t;

/* Enable (1) or disable (0) event timing of the kernels launched by later calls. */
int reg_ctx_set_timing(reg_ctx_t *ctx, int enable);

/* Copy the accounting of the last call into *out (host). */
int reg_ctx_last_timing(reg_ctx_t *ctx, reg_timing_t *out);

/* ---- diagnostics ----------------------------------------------------------- */
const char *reg_strerror(int code);
const char *reg_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* REG_H */
