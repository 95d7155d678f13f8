/*
 * FP64 CPU oracle of the registration scan operator (arXiv 2010.12478).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no
 * code, header, table or constant generator with the CUDA path: every step is
 * written out here from the paper's definitions, in plain double-precision
 * loops, with no blocking, fusion or reordering.
 *
 * What it computes (paper section / definition in brackets):
 *   - the image pyramid of the multilevel scheme            [Sec. 2.3.1]
 *   - the normalised-cross-correlation distance D(R, T o phi) and its
 *     gradient, for the rigid map phi(x) = R(alpha)(x - c) + c + G
 *                                                          [Sec. 2.3.1]
 *   - a nonrigid extension phi(x) = x + u(x) (not in the paper) with energy
 *     1 - NCC + lambda/(2P) * sum over grid edges of |u(a) - u(b)|^2
 *   - the gradient-flow minimiser with Armijo backtracking, run coarse to
 *     fine                                                  [Sec. 2.3.1]
 *   - the composition phi_jk o phi_ij used as initial guess of B [Sec. 2.3.2]
 *   - the registered frame T o phi on the reference grid, from which the
 *     registered series and its average are formed            [Sec. 2]
 *
 * The scan itself (sequential recursion, tree DAGs) is driven from Python
 * (oracle/__init__.py), one operator call at a time.
 *
 * Conventions (readings where the paper is silent):
 *   pixel (r, c) sits at x = (c, r); centre c0 = ((W-1)/2, (H-1)/2);
 *   rigid map and registered frames: bilinear sampling with clamp-to-edge;
 *   the derivative is the analytic derivative of the interpolant in the
 *   cell, 0 along a clamped axis; cell choice x0 = min(floor(px), W-2) so
 *   that W >= 2 and H >= 2 suffice;
 *   nonrigid field: both frames are taken through the quadratic B-spline
 *   model of their samples, extended beyond the border by the frame's mean,
 *   a continuously differentiable image, so that the energy of the local
 *   control values has a continuous gradient (see or_sample_q).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_LEVELS 8

typedef struct {
    int levels;        /* number of pyramid levels L */
    int max_iter;      /* accepted steps allowed per level */
    int max_rejects;   /* rejected line-search trials allowed per iteration */
    double tol_grad;   /* stop when the metric gradient norm falls below */
    double tol_rel_e;  /* stop when an accepted step lowers E by less than tol_rel_e*|E| */
    double armijo_c;   /* sufficient-decrease constant */
    double tau0;       /* first trial step of each level */
    double step_cap;   /* largest step, in pixels of the current level */
    double lambda;     /* regulariser weight (nonrigid only) */
    int metric;        /* nonrigid flow's scalar product: 0 mean over control points, 1 Gauss-Newton diagonal,
                          2 H1 (identity plus sigma^2 times the control grid's Laplacian) */
    double sigma;      /* metric 2: smoothing length in control-grid spacings */
    double tol_coarse; /* factor on tol_grad at every level above the finest (a coarse level only
                          supplies the next level's initial guess) */
} or_cfg_t;

typedef struct {
    int iters[OR_MAX_LEVELS];   /* accepted steps per level (index 0 = finest) */
    int evals[OR_MAX_LEVELS];   /* energy evaluations per level (with and without gradient) */
    int stop[OR_MAX_LEVELS];    /* why each level stopped, see OR_STOP_* */
    int rejects;                /* line-search rejections, all levels */
    double energy;              /* energy at the returned deformation, finest level */
} or_stats_t;

enum { OR_STOP_GRAD = 0, OR_STOP_REL = 1, OR_STOP_LS = 2, OR_STOP_MAXIT = 3 };

/* ------------------------------------------------------------------------ */
/* Multilevel scheme: 2x2 box average; an odd last row/column is clamped.   */
/* ------------------------------------------------------------------------ */

void or_downsample(const double *src, int W, int H, double *dst)
{
    int w2 = (W + 1) / 2, h2 = (H + 1) / 2;
    for (int r = 0; r < h2; ++r) {
        int r0 = 2 * r, r1 = 2 * r + 1 < H ? 2 * r + 1 : H - 1;
        for (int c = 0; c < w2; ++c) {
            int c0 = 2 * c, c1 = 2 * c + 1 < W ? 2 * c + 1 : W - 1;
            dst[r * w2 + c] = 0.25 * (src[r0 * W + c0] + src[r0 * W + c1] +
                                      src[r1 * W + c0] + src[r1 * W + c1]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Bilinear interpolation of T at (px, py) and its derivative.              */
/* out[0] = T(p), out[1] = dT/dpx, out[2] = dT/dpy.                         */
/* ------------------------------------------------------------------------ */

static double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Step-size rule of the line search (Armijo backtracking with safeguarded quadratic
 * interpolation, Nocedal and Wright, Numerical Optimization, Sec. 3.5).  After a trial at
 * step tau with energy Et, tq minimises the parabola through E(0) = E, E'(0) = slope and
 * E(tau) = Et.  A rejected trial retries at tq clamped to [0.1 tau, 0.5 tau]; an accepted one
 * starts the next line search at tq clamped to [0.5 tau, 4 tau].  Without positive curvature
 * (den <= 0) the rule falls back to halving / doubling.                                     */
static double or_next_tau(double E, double slope, double tau, double Et, int accepted)
{
    const double den = Et - E - slope * tau;
    if (!(den > 0.0)) return accepted ? 2.0 * tau : 0.5 * tau;
    const double tq = -slope * tau * tau / (2.0 * den);
    return accepted ? fmin(fmax(tq, 0.5 * tau), 4.0 * tau) : fmin(fmax(tq, 0.1 * tau), 0.5 * tau);
}

/* The step rule by itself (for its pins). */
double or_step_size(double E, double slope, double tau, double Et, int accepted)
{
    return or_next_tau(E, slope, tau, Et, accepted);
}

/* First trial step of a line search after an accepted step (Barzilai and Borwein, "Two-point step
 * size gradient methods", IMA J. Numer. Anal. 8, 1988, their second step): with the previous
 * step s = tau_acc d_prev and the change of the descent direction y = d_prev - d (directions in the
 * metric M, d = -M^-1 grad E), tau = <s, y>_M / <y, y>_M.  M weighs component 0 by m0 (rigid,
 * m0 = rho^2) and every component by 1 otherwise (pass m0 = 1).  Without positive curvature along
 * y (<s, y> <= 0 or <y, y> = 0) the step of the quadratic rule, tau_q, stays.                 */
static double or_bb_step(double tau_q, double tau_acc, const double *dprev, const double *d, const double *w, int n)
{
    double num = 0.0, den = 0.0;
    for (int k = 0; k < n; ++k) {
        const double wk = w ? w[k] : 1.0, y = dprev[k] - d[k];
        num += wk * dprev[k] * y;
        den += wk * y * y;
    }
    return (num > 0.0 && den > 0.0) ? tau_acc * num / den : tau_q;
}

/* The first-trial rule by itself (for its pins), metric diag(m0, 1, 1, ...). */
double or_bb_first_step(double tau_q, double tau_acc, const double *dprev, const double *d, int n, double m0)
{
    double *w = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int k = 0; k < n; ++k) w[k] = k == 0 ? m0 : 1.0;
    const double t = or_bb_step(tau_q, tau_acc, dprev, d, w, n);
    free(w);
    return t;
}

void or_sample(const double *T, int W, int H, double px, double py, double out[3])
{
    double qx = clampd(px, 0.0, (double)(W - 1));
    double qy = clampd(py, 0.0, (double)(H - 1));
    int x0 = (int)floor(qx), y0 = (int)floor(qy);
    if (x0 > W - 2) x0 = W - 2;
    if (y0 > H - 2) y0 = H - 2;
    double fx = qx - x0, fy = qy - y0;
    double t00 = T[y0 * W + x0], t01 = T[y0 * W + x0 + 1];
    double t10 = T[(y0 + 1) * W + x0], t11 = T[(y0 + 1) * W + x0 + 1];
    double top = (1.0 - fx) * t00 + fx * t01;
    double bot = (1.0 - fx) * t10 + fx * t11;
    out[0] = (1.0 - fy) * top + fy * bot;
    out[1] = (px < 0.0 || px > W - 1) ? 0.0 : (1.0 - fy) * (t01 - t00) + fy * (t11 - t10);
    out[2] = (py < 0.0 || py > H - 1) ? 0.0 : bot - top;
}

/* ------------------------------------------------------------------------ */
/* Quadratic B-spline model of the samples T_k (k on the integer grid):     */
/*   T(p) = sum_k T_k b(px - kx) b(py - ky),                                  */
/*   b(t) = 3/4 - t^2 (|t| <= 1/2), (|t| - 3/2)^2 / 2 (1/2 <= |t| <= 3/2), 0 */
/* with T_k = `outside` for k outside the frame (the energy passes the      */
/* frame's mean: beyond its border a frame carries no information, and its  */
/* centred value there is 0).  The model is continuously differentiable     */
/* everywhere (b is C1), reproduces affine images away from the border, and */
/* at a pixel centre equals the separable filter (1/8, 3/4, 1/8) of the     */
/* samples with derivative the central difference.                         */
/* out[0] = T(p), out[1] = dT/dpx, out[2] = dT/dpy.                         */
/* ------------------------------------------------------------------------ */

/* The three nonzero weights b(t + 1), b(t), b(t - 1) at offset t in [-1/2, 1/2) from the
 * nearest sample, and their derivatives. */
static void bspline2_weights(double t, double w[3], double dw[3])
{
    w[0] = 0.5 * (0.5 - t) * (0.5 - t);
    w[1] = 0.75 - t * t;
    w[2] = 0.5 * (0.5 + t) * (0.5 + t);
    dw[0] = -(0.5 - t);
    dw[1] = -2.0 * t;
    dw[2] = 0.5 + t;
}

void or_sample_q(const double *T, int W, int H, double outside, double px, double py, double out[3])
{
    const int nx = (int)floor(px + 0.5), ny = (int)floor(py + 0.5);   /* nearest sample */
    double wx[3], dwx[3], wy[3], dwy[3];
    bspline2_weights(px - nx, wx, dwx);
    bspline2_weights(py - ny, wy, dwy);
    double v = 0.0, gx = 0.0, gy = 0.0;
    for (int j = 0; j < 3; ++j) {
        const int y = ny - 1 + j;
        for (int i = 0; i < 3; ++i) {
            const int x = nx - 1 + i;
            const double t = (x < 0 || x >= W || y < 0 || y >= H) ? outside : T[y * W + x];
            v += wx[i] * wy[j] * t;
            gx += dwx[i] * wy[j] * t;
            gy += wx[i] * dwy[j] * t;
        }
    }
    out[0] = v;
    out[1] = gx;
    out[2] = gy;
}

/* ------------------------------------------------------------------------ */
/* Normalised cross-correlation from the five moments.                      */
/* Returns 1 (degenerate) when either image is constant to 1e-12 variance. */
/* ------------------------------------------------------------------------ */

typedef struct {
    double P, sR, sT, sRR, sTT, sRT;
} or_moments_t;

typedef struct {
    double ncc;     /* S'_RT / sqrt(S'_RR S'_TT) */
    double a, b;    /* dNCC/dTw(x) = a (R - Rbar) - b (Tw - Tbar) */
    double rbar, tbar;
    int degenerate;
} or_ncc_t;

static or_ncc_t or_ncc(const or_moments_t *m)
{
    or_ncc_t o;
    double srr = m->sRR - m->sR * m->sR / m->P;
    double stt = m->sTT - m->sT * m->sT / m->P;
    double srt = m->sRT - m->sR * m->sT / m->P;
    o.rbar = m->sR / m->P;
    o.tbar = m->sT / m->P;
    if (srr < 1e-12 * m->P || stt < 1e-12 * m->P) {
        o.ncc = 0.0; o.a = 0.0; o.b = 0.0; o.degenerate = 1;
        return o;
    }
    double root = sqrt(srr * stt);
    o.ncc = srt / root;
    o.a = 1.0 / root;
    o.b = o.ncc / stt;
    o.degenerate = 0;
    return o;
}

/* ------------------------------------------------------------------------ */
/* Rigid energy E = 1 - NCC(R, T o phi) and its gradient in (alpha, Gx, Gy). */
/* phi(x) = R(alpha)(x - c0) + c0 + G                      [Sec. 2.3.1]        */
/* ------------------------------------------------------------------------ */

int or_rigid_energy(const double *R, const double *T, int W, int H,
                    const double th[3], double *E, double *grad)
{
    const double cx = 0.5 * (W - 1), cy = 0.5 * (H - 1);
    const double ca = cos(th[0]), sa = sin(th[0]);
    or_moments_t m = {(double)W * H, 0, 0, 0, 0, 0};
    double sRg[3] = {0, 0, 0}, sTg[3] = {0, 0, 0}, sg[3] = {0, 0, 0};
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            double xc = c - cx, yc = r - cy;
            double px = ca * xc - sa * yc + cx + th[1];
            double py = sa * xc + ca * yc + cy + th[2];
            double s[3];
            or_sample(T, W, H, px, py, s);
            double rv = R[r * W + c], tv = s[0];
            m.sR += rv; m.sT += tv; m.sRR += rv * rv; m.sTT += tv * tv; m.sRT += rv * tv;
            if (grad) {
                /* g_k = grad T(phi(x)) . d phi / d theta_k */
                double dpx_da = -sa * xc - ca * yc, dpy_da = ca * xc - sa * yc;
                double g[3] = {s[1] * dpx_da + s[2] * dpy_da, s[1], s[2]};
                for (int k = 0; k < 3; ++k) {
                    sRg[k] += rv * g[k]; sTg[k] += tv * g[k]; sg[k] += g[k];
                }
            }
        }
    }
    or_ncc_t n = or_ncc(&m);
    if (n.degenerate) {
        *E = 1.0;
        if (grad) grad[0] = grad[1] = grad[2] = 0.0;
        return 1;
    }
    *E = 1.0 - n.ncc;
    if (grad) {
        for (int k = 0; k < 3; ++k) {
            double dncc = n.a * (sRg[k] - n.rbar * sg[k]) - n.b * (sTg[k] - n.tbar * sg[k]);
            grad[k] = -dncc;
        }
    }
    return 0;
}

/* Rigid composition phi2 o phi1 in centred coordinates: alpha1 + alpha2,
 * G = R(alpha2) G1 + G2.                                   [Sec. 2.3.2]   */
void or_rigid_compose(const double a[3], const double b[3], double out[3])
{
    double ca = cos(b[0]), sa = sin(b[0]);
    out[0] = a[0] + b[0];
    out[1] = ca * a[1] - sa * a[2] + b[1];
    out[2] = sa * a[1] + ca * a[2] + b[2];
}

/* One level of gradient flow with Armijo backtracking, rigid parameters.
 * Metric M = diag(rho^2, 1, 1), rho = (W + H) / 4: alpha is measured as an
 * arc length in pixels.                                                   */
static void or_rigid_level(const double *R, const double *T, int W, int H,
                           const or_cfg_t *cfg, double th[3], or_stats_t *st, int lvl)
{
    const double rho = 0.25 * (W + H), m0 = rho * rho;
    double E, g[3];
    or_rigid_energy(R, T, W, H, th, &E, g);
    st->evals[lvl] += 1;
    double tau = cfg->tau0;
    double dprev[3] = {0.0, 0.0, 0.0}, tau_acc = 0.0;
    int have_prev = 0;
    int stop = OR_STOP_MAXIT;
    for (int it = 0; it < cfg->max_iter; ++it) {
        double d[3] = {-g[0] / m0, -g[1], -g[2]};
        double slope = g[0] * d[0] + g[1] * d[1] + g[2] * d[2];
        double gn = sqrt(-slope);
        if (!(gn >= cfg->tol_grad * (lvl > 0 ? cfg->tol_coarse : 1.0))) { stop = OR_STOP_GRAD; break; }
        if (have_prev) {
            const double w[3] = {m0, 1.0, 1.0};
            tau = or_bb_step(tau, tau_acc, dprev, d, w, 3);
        }
        if (tau * gn > cfg->step_cap) tau = cfg->step_cap / gn;
        int accepted = 0;
        double tt[3], Et = 0.0;
        for (int rej = 0; rej <= cfg->max_rejects; ++rej) {
            for (int k = 0; k < 3; ++k) tt[k] = th[k] + tau * d[k];
            or_rigid_energy(R, T, W, H, tt, &Et, NULL);
            st->evals[lvl] += 1;
            if (Et <= E + cfg->armijo_c * tau * slope) { accepted = 1; break; }
            st->rejects += 1;
            tau = or_next_tau(E, slope, tau, Et, 0);
        }
        if (!accepted) { stop = OR_STOP_LS; break; }
        th[0] = tt[0]; th[1] = tt[1]; th[2] = tt[2];
        st->iters[lvl] += 1;
        tau_acc = tau;
        dprev[0] = d[0]; dprev[1] = d[1]; dprev[2] = d[2];
        have_prev = 1;
        double Eold = E;
        tau = or_next_tau(E, slope, tau, Et, 1);
        E = Et;
        if (Eold - Et <= cfg->tol_rel_e * fabs(Eold)) { stop = OR_STOP_REL; break; }
        or_rigid_energy(R, T, W, H, th, &E, g);
        st->evals[lvl] += 1;
    }
    st->stop[lvl] = stop;
    if (lvl == 0) st->energy = E;
}

/* Multilevel rigid registration: coarsest level first; G halves per level
 * going down (centred coordinates scale by exactly 2 for even sizes).     */
void or_rigid_register(const double *const *Rp, const double *const *Tp,
                       const int *Ws, const int *Hs, const or_cfg_t *cfg,
                       const double init[3], double out[3], or_stats_t *st)
{
    int L = cfg->levels;
    memset(st, 0, sizeof(*st));
    double th[3] = {init[0], ldexp(init[1], -(L - 1)), ldexp(init[2], -(L - 1))};
    for (int l = L - 1; l >= 0; --l) {
        or_rigid_level(Rp[l], Tp[l], Ws[l], Hs[l], cfg, th, st, l);
        if (l > 0) { th[1] *= 2.0; th[2] *= 2.0; }
    }
    out[0] = th[0]; out[1] = th[1]; out[2] = th[2];
}

/* ------------------------------------------------------------------------ */
/* Nonrigid extension (not in the paper): phi(x) = x + u(x) with u a         */
/* free-form field, bilinear in control displacements c_j on a grid of       */
/* spacing s (finest-level pixels), points X_j = (jx s, jy s),               */
/* jx = 0..nx-1, jy = 0..ny-1, nx = ceil((W0-1)/s) + 1.                      */
/* At level l, pixel x of the level sits at finest coordinate                */
/* X = 2^l x + (2^l - 1)/2 and the level's control values are c / 2^l        */
/* (displacements in pixels of that level).                                  */
/* E = 1 - NCC(R, T o phi) + lambda/(2 P_l) sum over control-grid edges of   */
/* |c_a - c_b|^2  (c in pixels of the level).                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, s;      /* control grid and spacing (finest pixels) */
    int W0, H0;         /* finest level size */
} or_grid_t;

/* Cell and bilinear weights of the finest-level coordinate (X, Y), clamped to the grid. */
static void or_grid_cell(const or_grid_t *g, double X, double Y, int *jx, int *jy, double *wx, double *wy)
{
    double gx = clampd(X / g->s, 0.0, (double)(g->nx - 1));
    double gy = clampd(Y / g->s, 0.0, (double)(g->ny - 1));
    int ix = (int)floor(gx), iy = (int)floor(gy);
    if (ix > g->nx - 2) ix = g->nx - 2;
    if (iy > g->ny - 2) iy = g->ny - 2;
    *jx = ix; *jy = iy;
    *wx = gx - ix; *wy = gy - iy;
}

/* u at finest coordinate (X, Y) from control values cx, cy ([ny][nx]). */
static void or_grid_eval(const or_grid_t *g, const double *cx, const double *cy, double X, double Y,
                         double *ux, double *uy)
{
    int jx, jy;
    double wx, wy;
    or_grid_cell(g, X, Y, &jx, &jy, &wx, &wy);
    int i = jy * g->nx + jx;
    double w00 = (1 - wx) * (1 - wy), w01 = wx * (1 - wy), w10 = (1 - wx) * wy, w11 = wx * wy;
    *ux = w00 * cx[i] + w01 * cx[i + 1] + w10 * cx[i + g->nx] + w11 * cx[i + g->nx + 1];
    *uy = w00 * cy[i] + w01 * cy[i + 1] + w10 * cy[i + g->nx] + w11 * cy[i + g->nx + 1];
}

double or_grid_regulariser(const or_grid_t *g, const double *cx, const double *cy, double lambda, double P)
{
    double s = 0.0;
    for (int jy = 0; jy < g->ny; ++jy) {
        for (int jx = 0; jx < g->nx; ++jx) {
            int i = jy * g->nx + jx;
            if (jx + 1 < g->nx) {
                double a = cx[i + 1] - cx[i], b = cy[i + 1] - cy[i];
                s += a * a + b * b;
            }
            if (jy + 1 < g->ny) {
                double a = cx[i + g->nx] - cx[i], b = cy[i + g->nx] - cy[i];
                s += a * a + b * b;
            }
        }
    }
    return 0.5 * lambda * s / P;
}

static double or_mean(const double *A, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += A[i];
    return s / n;
}

/* Energy at level l (images R, T of that level, W x H) for control values c
 * given in pixels of that level; gradient dE/dc (same units) if gx/gy given.
 * Both frames are taken through the quadratic B-spline model (or_sample_q),
 * each extended by its own mean: the reference at its pixel centres, the
 * template at x + u(x).                                                     */
int or_grid_energy(const double *R, const double *T, int W, int H, int l, const or_grid_t *g,
                   const double *cx, const double *cy, double lambda, double *E, double *gx, double *gy)
{
    const int P = W * H, Nc = g->nx * g->ny;
    const double scale = ldexp(1.0, l), off = 0.5 * (scale - 1.0);
    or_moments_t m = {(double)P, 0, 0, 0, 0, 0};
    double *tw = NULL, *dtx = NULL, *dty = NULL;
    /* the reference through the same image model, at its pixel centres */
    double *Rm = (double *)malloc(sizeof(double) * P);
    const double mR = or_mean(R, P), mT = or_mean(T, P);
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            double s[3];
            or_sample_q(R, W, H, mR, (double)c, (double)r, s);
            Rm[r * W + c] = s[0];
        }
    if (gx) {
        tw = (double *)malloc(sizeof(double) * P);
        dtx = (double *)malloc(sizeof(double) * P);
        dty = (double *)malloc(sizeof(double) * P);
    }
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            int i = r * W + c;
            double ux, uy, s[3];
            or_grid_eval(g, cx, cy, scale * c + off, scale * r + off, &ux, &uy);
            or_sample_q(T, W, H, mT, c + ux, r + uy, s);
            double rv = Rm[i], tv = s[0];
            m.sR += rv; m.sT += tv; m.sRR += rv * rv; m.sTT += tv * tv; m.sRT += rv * tv;
            if (gx) { tw[i] = tv; dtx[i] = s[1]; dty[i] = s[2]; }
        }
    }
    or_ncc_t n = or_ncc(&m);
    *E = (n.degenerate ? 1.0 : 1.0 - n.ncc) + or_grid_regulariser(g, cx, cy, lambda, (double)P);
    if (gx) {
        for (int j = 0; j < Nc; ++j) { gx[j] = 0.0; gy[j] = 0.0; }
        if (!n.degenerate) {
            for (int r = 0; r < H; ++r) {
                for (int c = 0; c < W; ++c) {
                    int i = r * W + c, jx, jy;
                    double wx, wy;
                    or_grid_cell(g, scale * c + off, scale * r + off, &jx, &jy, &wx, &wy);
                    double f = -(n.a * (Rm[i] - n.rbar) - n.b * (tw[i] - n.tbar));
                    double ax = f * dtx[i], ay = f * dty[i];
                    int j = jy * g->nx + jx;
                    double w[4] = {(1 - wx) * (1 - wy), wx * (1 - wy), (1 - wx) * wy, wx * wy};
                    int idx[4] = {j, j + 1, j + g->nx, j + g->nx + 1};
                    for (int q = 0; q < 4; ++q) { gx[idx[q]] += w[q] * ax; gy[idx[q]] += w[q] * ay; }
                }
            }
        }
        /* d/dc_j of lambda/(2P) sum over grid edges |c_a - c_b|^2 */
        const double k = lambda / (double)P;
        for (int jy = 0; jy < g->ny; ++jy) {
            for (int jx = 0; jx < g->nx; ++jx) {
                int j = jy * g->nx + jx;
                double lx = 0.0, ly = 0.0;
                if (jx > 0)         { lx += cx[j] - cx[j - 1];     ly += cy[j] - cy[j - 1]; }
                if (jx + 1 < g->nx) { lx += cx[j] - cx[j + 1];     ly += cy[j] - cy[j + 1]; }
                if (jy > 0)         { lx += cx[j] - cx[j - g->nx]; ly += cy[j] - cy[j - g->nx]; }
                if (jy + 1 < g->ny) { lx += cx[j] - cx[j + g->nx]; ly += cy[j] - cy[j + g->nx]; }
                gx[j] += k * lx;
                gy[j] += k * ly;
            }
        }
        free(tw); free(dtx); free(dty);
    }
    free(Rm);
    return n.degenerate;
}

/* Scalar product of the nonrigid flow (cfg->metric = 1): per control point and axis the
 * Gauss-Newton curvature of the data term plus the regulariser's,
 *   m_j^x = sum_x w_j(x)^2 (dT/dpx)^2 / (P var T) + lambda n_j / P   (likewise for y),
 * with w_j the bilinear weight of control point j at pixel x, dT the derivative of the image
 * model at x + u(x) for the level's initial control values, var T the variance of those samples
 * and n_j the number of grid neighbours of j; normalised by the mean of all 2 Nc values and
 * floored at 1e-3 of it.  <u, v> = (1/Nc) sum_j (m_j^x u_j^x v_j^x + m_j^y u_j^y v_j^y): a fixed
 * scalar product per level in which every control point's step is scaled by its own curvature
 * (control points outside the overlap of the two frames are held by the regulariser alone).   */
void or_grid_metric(const double *T, int W, int H, int l, const or_grid_t *g, const double *cx,
                    const double *cy, double lambda, double *mx, double *my)
{
    const int P = W * H, Nc = g->nx * g->ny;
    const double scale = ldexp(1.0, l), off = 0.5 * (scale - 1.0);
    double st = 0.0, stt = 0.0;
    const double mT = or_mean(T, P);
    for (int j = 0; j < Nc; ++j) { mx[j] = 0.0; my[j] = 0.0; }
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            int jx, jy;
            double ux, uy, wx, wy, s[3];
            or_grid_eval(g, cx, cy, scale * c + off, scale * r + off, &ux, &uy);
            or_sample_q(T, W, H, mT, c + ux, r + uy, s);
            st += s[0];
            stt += s[0] * s[0];
            or_grid_cell(g, scale * c + off, scale * r + off, &jx, &jy, &wx, &wy);
            const int j = jy * g->nx + jx;
            const double w[4] = {(1 - wx) * (1 - wy), wx * (1 - wy), (1 - wx) * wy, wx * wy};
            const int idx[4] = {j, j + 1, j + g->nx, j + g->nx + 1};
            for (int q = 0; q < 4; ++q) {
                mx[idx[q]] += w[q] * w[q] * s[1] * s[1];
                my[idx[q]] += w[q] * w[q] * s[2] * s[2];
            }
        }
    }
    const double var = stt / P - (st / P) * (st / P);
    const double dk = var > 0.0 ? 1.0 / (P * var) : 0.0;
    double mean = 0.0;
    for (int jy = 0; jy < g->ny; ++jy)
        for (int jx = 0; jx < g->nx; ++jx) {
            const int j = jy * g->nx + jx;
            const int nb = (jx > 0) + (jx + 1 < g->nx) + (jy > 0) + (jy + 1 < g->ny);
            mx[j] = mx[j] * dk + lambda * nb / P;
            my[j] = my[j] * dk + lambda * nb / P;
            mean += mx[j] + my[j];
        }
    mean /= 2.0 * Nc;
    for (int j = 0; j < Nc; ++j) {
        if (!(mean > 0.0)) { mx[j] = 1.0; my[j] = 1.0; continue; }
        mx[j] = fmax(mx[j] / mean, 1e-3);
        my[j] = fmax(my[j] / mean, 1e-3);
    }
}

/* H1 scalar product on control-point fields (metric 2; Sec. 2.3.1 leaves the flow's scalar product
 * open): <u, v> = (1/Nc) u^T M v per axis with M = I + sigma^2 Lg, Lg the Laplacian of the control
 * grid's graph (the horizontal and vertical neighbour edges the regulariser sums over):
 * (Lg v)_j = sum over neighbours k of j of (v_j - v_k).  The flow's direction d = -Nc M^-1 dE/dc is
 * the gradient smoothed over about sigma grid spacings.                                          */
void or_h1_apply(const or_grid_t *g, double sigma, const double *v, double *out)
{
    const double s2 = sigma * sigma;
    for (int jy = 0; jy < g->ny; ++jy)
        for (int jx = 0; jx < g->nx; ++jx) {
            const int j = jy * g->nx + jx;
            double lap = 0.0;
            if (jx > 0) lap += v[j] - v[j - 1];
            if (jx + 1 < g->nx) lap += v[j] - v[j + 1];
            if (jy > 0) lap += v[j] - v[j - g->nx];
            if (jy + 1 < g->ny) lap += v[j] - v[j + g->nx];
            out[j] = v[j] + s2 * lap;
        }
}

/* M = I + sigma^2 Lg as a symmetric band matrix (half-bandwidth nx, the row-major neighbour
 * offsets 1 and nx), factored M = C C^T by Cholesky in band storage: C[i][j] at
 * band[i (nx + 1) + j - i + nx] for i - nx <= j <= i.  M is positive definite (Lg is positive
 * semidefinite), so every pivot is at least 1.                                                   */
double *or_h1_factor(const or_grid_t *g, double sigma)
{
    const int n = g->nx * g->ny, p = g->nx, w = p + 1;
    double *b = (double *)calloc((size_t)n * w, sizeof(double));
    const double s2 = sigma * sigma;
    /* lower half of M: diagonal 1 + s2 deg_j, -s2 for each neighbour below the diagonal */
    for (int jy = 0; jy < g->ny; ++jy)
        for (int jx = 0; jx < g->nx; ++jx) {
            const int i = jy * g->nx + jx;
            const int deg = (jx > 0) + (jx + 1 < g->nx) + (jy > 0) + (jy + 1 < g->ny);
            b[(size_t)i * w + p] = 1.0 + s2 * deg;
            if (jx > 0) b[(size_t)i * w + p - 1] = -s2;
            if (jy > 0) b[(size_t)i * w + 0] = -s2;
        }
    for (int i = 0; i < n; ++i) {
        const int j0 = i - p > 0 ? i - p : 0;
        for (int j = j0; j <= i; ++j) {
            double acc = b[(size_t)i * w + j - i + p];
            const int k0 = (i - p > j - p ? i - p : j - p) > 0 ? (i - p > j - p ? i - p : j - p) : 0;
            for (int k = k0; k < j; ++k) acc -= b[(size_t)i * w + k - i + p] * b[(size_t)j * w + k - j + p];
            if (j == i) b[(size_t)i * w + p] = sqrt(acc);
            else b[(size_t)i * w + j - i + p] = acc / b[(size_t)j * w + p];
        }
    }
    return b;
}

/* x = M^-1 rhs with the factor of or_h1_factor: C y = rhs, then C^T x = y. */
void or_h1_solve(const or_grid_t *g, const double *band, const double *rhs, double *x)
{
    const int n = g->nx * g->ny, p = g->nx, w = p + 1;
    for (int i = 0; i < n; ++i) {
        double acc = rhs[i];
        for (int k = (i - p > 0 ? i - p : 0); k < i; ++k) acc -= band[(size_t)i * w + k - i + p] * x[k];
        x[i] = acc / band[(size_t)i * w + p];
    }
    for (int i = n - 1; i >= 0; --i) {
        double acc = x[i];
        for (int k = i + 1; k <= (i + p < n - 1 ? i + p : n - 1); ++k) acc -= band[(size_t)k * w + i - k + p] * x[k];
        x[i] = acc / band[(size_t)i * w + p];
    }
}

/* The solve by itself (for its pins): x = (I + sigma^2 Lg)^-1 rhs. */
void or_h1_inverse(const or_grid_t *g, double sigma, const double *rhs, double *x)
{
    double *band = or_h1_factor(g, sigma);
    or_h1_solve(g, band, rhs, x);
    free(band);
}

/* One level of gradient flow for the control values (pixels of level l).
 * Metric: cfg->metric 1, the Gauss-Newton diagonal of or_grid_metric; 0, the
 * mean over control points, <v, w> = (1/Nc) sum v.w; 2, the H1 product of
 * or_h1_apply.  The descent direction is d = -M^-1 dE/dc (in the metric's
 * 1/Nc normalisation: d = -Nc M^-1 g) and tau |d_j| is a move in pixels.   */
static void or_grid_level(const double *R, const double *T, int W, int H, int l, const or_grid_t *g,
                          const or_cfg_t *cfg, double *cx, double *cy, or_stats_t *st)
{
    const int Nc = g->nx * g->ny;
    double *gx = (double *)malloc(sizeof(double) * Nc), *gy = (double *)malloc(sizeof(double) * Nc);
    double *dx = (double *)malloc(sizeof(double) * Nc), *dy = (double *)malloc(sizeof(double) * Nc);
    double *tx = (double *)malloc(sizeof(double) * Nc), *ty = (double *)malloc(sizeof(double) * Nc);
    /* previous direction, both components in one array (x plane then y plane) */
    double *dp = (double *)malloc(sizeof(double) * 2 * Nc), *dc = (double *)malloc(sizeof(double) * 2 * Nc);
    /* the level's scalar product, per control point and axis (interleaved like dc) */
    double *mx = (double *)malloc(sizeof(double) * Nc), *my = (double *)malloc(sizeof(double) * Nc);
    double *mw = (double *)malloc(sizeof(double) * 2 * Nc);
    double E, Et = 0.0, tau_acc = 0.0;
    int have_prev = 0;
    /* H1: the factor of M and work arrays for M^-1 g and M applied to directions */
    const int h1 = cfg->metric == 2;
    double *band = h1 ? or_h1_factor(g, cfg->sigma) : NULL;
    double *h1a = (double *)malloc(sizeof(double) * Nc), *h1b = (double *)malloc(sizeof(double) * Nc);
    double *dpx = (double *)malloc(sizeof(double) * Nc), *dpy = (double *)malloc(sizeof(double) * Nc);
    if (cfg->metric == 1) {
        or_grid_metric(T, W, H, l, g, cx, cy, cfg->lambda, mx, my);
    } else {
        for (int j = 0; j < Nc; ++j) { mx[j] = 1.0; my[j] = 1.0; }
    }
    for (int j = 0; j < Nc; ++j) { mw[2 * j] = mx[j]; mw[2 * j + 1] = my[j]; }
    or_grid_energy(R, T, W, H, l, g, cx, cy, cfg->lambda, &E, gx, gy);
    st->evals[l] += 1;
    double tau = cfg->tau0;
    int stop = OR_STOP_MAXIT;
    for (int it = 0; it < cfg->max_iter; ++it) {
        /* d = -M^-1 grad E; ss = Nc |d|_M^2 = sum_j (m^x dx^2 + m^y dy^2); dmax = max_j |d_j| in px */
        double ss = 0.0, dmax = 0.0;
        if (h1) {
            /* d = -Nc M^-1 g per axis, ss = d^T M d */
            or_h1_solve(g, band, gx, dx);
            or_h1_solve(g, band, gy, dy);
            for (int j = 0; j < Nc; ++j) { dx[j] *= -(double)Nc; dy[j] *= -(double)Nc; }
            or_h1_apply(g, cfg->sigma, dx, h1a);
            or_h1_apply(g, cfg->sigma, dy, h1b);
            for (int j = 0; j < Nc; ++j) {
                const double q = dx[j] * dx[j] + dy[j] * dy[j];
                ss += dx[j] * h1a[j] + dy[j] * h1b[j];
                if (q > dmax) dmax = q;
            }
        } else {
            for (int j = 0; j < Nc; ++j) {
                dx[j] = -(double)Nc * gx[j] / mx[j];
                dy[j] = -(double)Nc * gy[j] / my[j];
                double q = dx[j] * dx[j] + dy[j] * dy[j];
                ss += mx[j] * dx[j] * dx[j] + my[j] * dy[j] * dy[j];
                if (q > dmax) dmax = q;
            }
        }
        dmax = sqrt(dmax);
        double slope = -ss / (double)Nc;
        double gn = sqrt(ss / (double)Nc);
        if (!(gn >= cfg->tol_grad * (l > 0 ? cfg->tol_coarse : 1.0))) { stop = OR_STOP_GRAD; break; }
        for (int j = 0; j < Nc; ++j) { dc[2 * j] = dx[j]; dc[2 * j + 1] = dy[j]; }
        /* the metric's common factor 1/Nc cancels in the ratio */
        if (have_prev && h1) {
            /* <s, y>_M / <y, y>_M with y = d_prev - d, through M applied to y */
            double num = 0.0, den = 0.0;
            for (int j = 0; j < Nc; ++j) { h1a[j] = dpx[j] - dx[j]; h1b[j] = dpy[j] - dy[j]; }
            double *ya = tx, *yb = ty;   /* trial buffers are free here */
            or_h1_apply(g, cfg->sigma, h1a, ya);
            or_h1_apply(g, cfg->sigma, h1b, yb);
            for (int j = 0; j < Nc; ++j) {
                num += dpx[j] * ya[j] + dpy[j] * yb[j];
                den += h1a[j] * ya[j] + h1b[j] * yb[j];
            }
            tau = (num > 0.0 && den > 0.0) ? tau_acc * num / den : tau;
        } else if (have_prev) {
            tau = or_bb_step(tau, tau_acc, dp, dc, mw, 2 * Nc);
        }
        if (tau * dmax > cfg->step_cap) tau = cfg->step_cap / dmax;
        int accepted = 0;
        for (int rej = 0; rej <= cfg->max_rejects; ++rej) {
            for (int j = 0; j < Nc; ++j) { tx[j] = cx[j] + tau * dx[j]; ty[j] = cy[j] + tau * dy[j]; }
            or_grid_energy(R, T, W, H, l, g, tx, ty, cfg->lambda, &Et, NULL, NULL);
            st->evals[l] += 1;
            if (Et <= E + cfg->armijo_c * tau * slope) { accepted = 1; break; }
            st->rejects += 1;
            tau = or_next_tau(E, slope, tau, Et, 0);
        }
        if (!accepted) { stop = OR_STOP_LS; break; }
        memcpy(cx, tx, sizeof(double) * Nc);
        memcpy(cy, ty, sizeof(double) * Nc);
        st->iters[l] += 1;
        tau_acc = tau;
        memcpy(dp, dc, sizeof(double) * 2 * Nc);
        memcpy(dpx, dx, sizeof(double) * Nc);
        memcpy(dpy, dy, sizeof(double) * Nc);
        have_prev = 1;
        double Eold = E;
        tau = or_next_tau(E, slope, tau, Et, 1);
        E = Et;
        if (Eold - Et <= cfg->tol_rel_e * fabs(Eold)) { stop = OR_STOP_REL; break; }
        or_grid_energy(R, T, W, H, l, g, cx, cy, cfg->lambda, &E, gx, gy);
        st->evals[l] += 1;
    }
    st->stop[l] = stop;
    if (l == 0) st->energy = E;
    free(gx); free(gy); free(dx); free(dy); free(tx); free(ty); free(dp); free(dc); free(mx); free(my); free(mw);
    free(band); free(h1a); free(h1b); free(dpx); free(dpy);
}

/* Multilevel nonrigid registration on the control grid.  init (finest-level
 * pixels, NULL = identity) is scaled to the coarsest level by 2^-(L-1); each
 * finer level starts from twice the coarser result (same grid, exact).     */
void or_grid_register(const double *const *Rp, const double *const *Tp, const int *Ws, const int *Hs,
                      const or_cfg_t *cfg, const or_grid_t *g, const double *init_x, const double *init_y,
                      double *out_x, double *out_y, or_stats_t *st)
{
    const int L = cfg->levels, Nc = g->nx * g->ny;
    memset(st, 0, sizeof(*st));
    double *cx = (double *)calloc(Nc, sizeof(double)), *cy = (double *)calloc(Nc, sizeof(double));
    if (init_x) {
        for (int j = 0; j < Nc; ++j) { cx[j] = ldexp(init_x[j], -(L - 1)); cy[j] = ldexp(init_y[j], -(L - 1)); }
    }
    for (int l = L - 1; l >= 0; --l) {
        or_grid_level(Rp[l], Tp[l], Ws[l], Hs[l], l, g, cfg, cx, cy, st);
        if (l > 0)
            for (int j = 0; j < Nc; ++j) { cx[j] *= 2.0; cy[j] *= 2.0; }
    }
    memcpy(out_x, cx, sizeof(double) * Nc);
    memcpy(out_y, cy, sizeof(double) * Nc);
    free(cx); free(cy);
}

/* Composition at the control points (B's initial guess, Sec. 2.3.2):
 * c(X_j) = c1_j + u2(X_j + c1_j), u2 the field of c2 (finest-level pixels). */
void or_grid_compose(const or_grid_t *g, const double *c1x, const double *c1y, const double *c2x,
                     const double *c2y, double *ox, double *oy)
{
    for (int jy = 0; jy < g->ny; ++jy) {
        for (int jx = 0; jx < g->nx; ++jx) {
            int j = jy * g->nx + jx;
            double ux, uy;
            or_grid_eval(g, c2x, c2y, jx * (double)g->s + c1x[j], jy * (double)g->s + c1y[j], &ux, &uy);
            ox[j] = c1x[j] + ux;
            oy[j] = c1y[j] + uy;
        }
    }
}

/* Field of level l (W x H pixels of that level) for control values in pixels of that level. */
void or_grid_level_dense(const or_grid_t *g, const double *cx, const double *cy, int l, int W, int H,
                         double *ux, double *uy)
{
    const double scale = ldexp(1.0, l), off = 0.5 * (scale - 1.0);
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c)
            or_grid_eval(g, cx, cy, scale * c + off, scale * r + off, &ux[r * W + c], &uy[r * W + c]);
}

/* Dense finest-level field of the control values. */
void or_grid_dense(const or_grid_t *g, const double *cx, const double *cy, double *ux, double *uy)
{
    for (int r = 0; r < g->H0; ++r)
        for (int c = 0; c < g->W0; ++c)
            or_grid_eval(g, cx, cy, (double)c, (double)r, &ux[r * g->W0 + c], &uy[r * g->W0 + c]);
}

/* ------------------------------------------------------------------------ */
/* Registered frame: T resampled onto the reference grid by phi,            */
/* out(x) = T(phi(x)), bilinear with clamp-to-edge.  The series is          */
/* registered to its first frame and then averaged            [Sec. 2].    */
/* ------------------------------------------------------------------------ */
void or_warp_rigid(const double *T, int W, int H, const double theta[3], double *out)
{
    const double cx = 0.5 * (W - 1), cy = 0.5 * (H - 1);
    const double ca = cos(theta[0]), sa = sin(theta[0]);
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            double xc = c - cx, yc = r - cy, v[3];
            or_sample(T, W, H, ca * xc - sa * yc + cx + theta[1], sa * xc + ca * yc + cy + theta[2], v);
            out[r * W + c] = v[0];
        }
}

void or_warp_grid(const or_grid_t *g, const double *T, const double *cx, const double *cy, double *out)
{
    for (int r = 0; r < g->H0; ++r)
        for (int c = 0; c < g->W0; ++c) {
            double ux, uy, v[3];
            or_grid_eval(g, cx, cy, (double)c, (double)r, &ux, &uy);
            or_sample(T, g->W0, g->H0, c + ux, r + uy, v);
            out[r * g->W0 + c] = v[0];
        }
}
