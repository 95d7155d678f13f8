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
 *
 * The scan itself (sequential recursion, tree DAGs) is driven from Python
 * (oracle/__init__.py), one operator call at a time.
 *
 * Conventions (readings where the paper is silent):
 *   pixel (r, c) sits at x = (c, r); centre c0 = ((W-1)/2, (H-1)/2);
 *   bilinear sampling with clamp-to-edge; the derivative is the analytic
 *   derivative of the interpolant in the cell, 0 along a clamped axis;
 *   cell choice x0 = min(floor(px), W-2) so that W >= 2 and H >= 2 suffice.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_LEVELS 8

typedef struct {
    int levels;        /* number of pyramid levels L */
    int max_iter;      /* accepted steps allowed per level */
    int max_rejects;   /* line-search halvings allowed per iteration */
    double tol_grad;   /* stop when the metric gradient norm falls below */
    double tol_rel_e;  /* stop when an accepted step lowers E by less than tol_rel_e*|E| */
    double armijo_c;   /* sufficient-decrease constant */
    double tau0;       /* first trial step of each level */
    double step_cap;   /* largest step, in pixels of the current level */
    double lambda;     /* regulariser weight (nonrigid only) */
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
    int stop = OR_STOP_MAXIT;
    for (int it = 0; it < cfg->max_iter; ++it) {
        double d[3] = {-g[0] / m0, -g[1], -g[2]};
        double slope = g[0] * d[0] + g[1] * d[1] + g[2] * d[2];
        double gn = sqrt(-slope);
        if (!(gn >= cfg->tol_grad)) { stop = OR_STOP_GRAD; break; }
        if (tau * gn > cfg->step_cap) tau = cfg->step_cap / gn;
        int accepted = 0;
        double tt[3], Et = 0.0;
        for (int rej = 0; rej <= cfg->max_rejects; ++rej) {
            for (int k = 0; k < 3; ++k) tt[k] = th[k] + tau * d[k];
            or_rigid_energy(R, T, W, H, tt, &Et, NULL);
            st->evals[lvl] += 1;
            if (Et <= E + cfg->armijo_c * tau * slope) { accepted = 1; break; }
            st->rejects += 1;
            tau *= 0.5;
        }
        if (!accepted) { stop = OR_STOP_LS; break; }
        th[0] = tt[0]; th[1] = tt[1]; th[2] = tt[2];
        st->iters[lvl] += 1;
        double Eold = E;
        E = Et;
        tau *= 2.0;
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
/* Nonrigid extension: phi(x) = x + u(x), u = (ux, uy) on the pixel grid.   */
/* E = 1 - NCC(R, T o phi) + lambda/(2P) sum |forward differences of u|^2   */
/* ------------------------------------------------------------------------ */

double or_regulariser(const double *ux, const double *uy, int W, int H, double lambda)
{
    double s = 0.0;
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            int i = r * W + c;
            if (c + 1 < W) {
                double ax = ux[i + 1] - ux[i], ay = uy[i + 1] - uy[i];
                s += ax * ax + ay * ay;
            }
            if (r + 1 < H) {
                double bx = ux[i + W] - ux[i], by = uy[i + W] - uy[i];
                s += bx * bx + by * by;
            }
        }
    }
    return 0.5 * lambda * s / ((double)W * H);
}

/* E and, if gx/gy are given, dE/du(x) per pixel. */
int or_nonrigid_energy(const double *R, const double *T, int W, int H,
                       const double *ux, const double *uy, double lambda,
                       double *E, double *gx, double *gy)
{
    const int P = W * H;
    or_moments_t m = {(double)P, 0, 0, 0, 0, 0};
    double *tw = NULL, *dtx = NULL, *dty = NULL;
    if (gx) {
        tw = (double *)malloc(sizeof(double) * P);
        dtx = (double *)malloc(sizeof(double) * P);
        dty = (double *)malloc(sizeof(double) * P);
    }
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            int i = r * W + c;
            double s[3];
            or_sample(T, W, H, c + ux[i], r + uy[i], s);
            double rv = R[i], tv = s[0];
            m.sR += rv; m.sT += tv; m.sRR += rv * rv; m.sTT += tv * tv; m.sRT += rv * tv;
            if (gx) { tw[i] = tv; dtx[i] = s[1]; dty[i] = s[2]; }
        }
    }
    or_ncc_t n = or_ncc(&m);
    double Ed = n.degenerate ? 1.0 : 1.0 - n.ncc;
    *E = Ed + or_regulariser(ux, uy, W, H, lambda);
    if (gx) {
        const double k = lambda / (double)P;
        for (int r = 0; r < H; ++r) {
            for (int c = 0; c < W; ++c) {
                int i = r * W + c;
                double f = n.degenerate ? 0.0 : -(n.a * (R[i] - n.rbar) - n.b * (tw[i] - n.tbar));
                /* d/du(x) of lambda/(2P) sum over grid edges (u(a)-u(b))^2 */
                double lx = 0.0, ly = 0.0;
                if (c > 0)     { lx += ux[i] - ux[i - 1]; ly += uy[i] - uy[i - 1]; }
                if (c + 1 < W) { lx += ux[i] - ux[i + 1]; ly += uy[i] - uy[i + 1]; }
                if (r > 0)     { lx += ux[i] - ux[i - W]; ly += uy[i] - uy[i - W]; }
                if (r + 1 < H) { lx += ux[i] - ux[i + W]; ly += uy[i] - uy[i + W]; }
                gx[i] = f * dtx[i] + k * lx;
                gy[i] = f * dty[i] + k * ly;
            }
        }
        free(tw); free(dtx); free(dty);
    }
    return n.degenerate;
}

/* Composition of displacement fields: (phi2 o phi1)(x) = x + u1(x) + u2(x + u1(x)). */
void or_nonrigid_compose(const double *u1x, const double *u1y,
                         const double *u2x, const double *u2y, int W, int H,
                         double *ox, double *oy)
{
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            int i = r * W + c;
            double px = c + u1x[i], py = r + u1y[i], sx[3], sy[3];
            or_sample(u2x, W, H, px, py, sx);
            or_sample(u2y, W, H, px, py, sy);
            ox[i] = u1x[i] + sx[0];
            oy[i] = u1y[i] + sy[0];
        }
    }
}

/* Coarse-to-fine transfer: a coarse pixel (rc, cc) covers fine pixels 2rc, 2rc+1,
 * so fine pixel (r, c) sits at coarse coordinate ((c - 0.5)/2, (r - 0.5)/2);
 * displacements double.                                                      */
void or_prolong(const double *src, int Wc, int Hc, double *dst, int W, int H)
{
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            double s[3];
            or_sample(src, Wc, Hc, 0.5 * (c - 0.5), 0.5 * (r - 0.5), s);
            dst[r * W + c] = 2.0 * s[0];
        }
    }
}

/* Fine-to-coarse transfer of an initial displacement: box average, halved. */
void or_restrict(const double *src, int W, int H, double *dst)
{
    int w2 = (W + 1) / 2, h2 = (H + 1) / 2;
    or_downsample(src, W, H, dst);
    for (int i = 0; i < w2 * h2; ++i) dst[i] *= 0.5;
}

/* One level of gradient flow for the field u.  Metric: the mean-L2 product
 * <v, w> = (1/P) sum v.w, so the descent direction is d = -P dE/du and a
 * step tau moves pixel x by tau |d(x)| pixels.                             */
static void or_nonrigid_level(const double *R, const double *T, int W, int H,
                              const or_cfg_t *cfg, double *ux, double *uy,
                              or_stats_t *st, int lvl)
{
    const int P = W * H;
    double *gx = (double *)malloc(sizeof(double) * P), *gy = (double *)malloc(sizeof(double) * P);
    double *dx = (double *)malloc(sizeof(double) * P), *dy = (double *)malloc(sizeof(double) * P);
    double *tx = (double *)malloc(sizeof(double) * P), *ty = (double *)malloc(sizeof(double) * P);
    double E, Et = 0.0;
    or_nonrigid_energy(R, T, W, H, ux, uy, cfg->lambda, &E, gx, gy);
    st->evals[lvl] += 1;
    double tau = cfg->tau0;
    int stop = OR_STOP_MAXIT;
    for (int it = 0; it < cfg->max_iter; ++it) {
        double ss = 0.0, dmax = 0.0;
        for (int i = 0; i < P; ++i) {
            dx[i] = -(double)P * gx[i];
            dy[i] = -(double)P * gy[i];
            double q = dx[i] * dx[i] + dy[i] * dy[i];
            ss += q;
            if (q > dmax) dmax = q;
        }
        dmax = sqrt(dmax);
        double slope = -ss / (double)P;       /* dE/du . d */
        double gn = sqrt(ss / (double)P);      /* metric norm of d */
        if (!(gn >= cfg->tol_grad)) { stop = OR_STOP_GRAD; break; }
        if (tau * dmax > cfg->step_cap) tau = cfg->step_cap / dmax;
        int accepted = 0;
        for (int rej = 0; rej <= cfg->max_rejects; ++rej) {
            for (int i = 0; i < P; ++i) { tx[i] = ux[i] + tau * dx[i]; ty[i] = uy[i] + tau * dy[i]; }
            or_nonrigid_energy(R, T, W, H, tx, ty, cfg->lambda, &Et, NULL, NULL);
            st->evals[lvl] += 1;
            if (Et <= E + cfg->armijo_c * tau * slope) { accepted = 1; break; }
            st->rejects += 1;
            tau *= 0.5;
        }
        if (!accepted) { stop = OR_STOP_LS; break; }
        memcpy(ux, tx, sizeof(double) * P);
        memcpy(uy, ty, sizeof(double) * P);
        st->iters[lvl] += 1;
        double Eold = E;
        E = Et;
        tau *= 2.0;
        if (Eold - Et <= cfg->tol_rel_e * fabs(Eold)) { stop = OR_STOP_REL; break; }
        or_nonrigid_energy(R, T, W, H, ux, uy, cfg->lambda, &E, gx, gy);
        st->evals[lvl] += 1;
    }
    st->stop[lvl] = stop;
    if (lvl == 0) st->energy = E;
    free(gx); free(gy); free(dx); free(dy); free(tx); free(ty);
}

/* Multilevel nonrigid registration.  init_x/init_y: finest-level initial
 * displacement (NULL = identity); it is restricted to the coarsest level,
 * and each level's result is prolonged to start the next finer level.     */
void or_nonrigid_register(const double *const *Rp, const double *const *Tp,
                          const int *Ws, const int *Hs, const or_cfg_t *cfg,
                          const double *init_x, const double *init_y,
                          double *out_x, double *out_y, or_stats_t *st)
{
    int L = cfg->levels;
    memset(st, 0, sizeof(*st));
    double *ux[OR_MAX_LEVELS] = {0}, *uy[OR_MAX_LEVELS] = {0};
    for (int l = 0; l < L; ++l) {
        ux[l] = (double *)calloc((size_t)Ws[l] * Hs[l], sizeof(double));
        uy[l] = (double *)calloc((size_t)Ws[l] * Hs[l], sizeof(double));
    }
    if (init_x) {
        memcpy(ux[0], init_x, sizeof(double) * Ws[0] * Hs[0]);
        memcpy(uy[0], init_y, sizeof(double) * Ws[0] * Hs[0]);
        for (int l = 1; l < L; ++l) {
            or_restrict(ux[l - 1], Ws[l - 1], Hs[l - 1], ux[l]);
            or_restrict(uy[l - 1], Ws[l - 1], Hs[l - 1], uy[l]);
        }
    }
    for (int l = L - 1; l >= 0; --l) {
        or_nonrigid_level(Rp[l], Tp[l], Ws[l], Hs[l], cfg, ux[l], uy[l], st, l);
        if (l > 0) {
            or_prolong(ux[l], Ws[l], Hs[l], ux[l - 1], Ws[l - 1], Hs[l - 1]);
            or_prolong(uy[l], Ws[l], Hs[l], uy[l - 1], Ws[l - 1], Hs[l - 1]);
        }
    }
    memcpy(out_x, ux[0], sizeof(double) * Ws[0] * Hs[0]);
    memcpy(out_y, uy[0], sizeof(double) * Ws[0] * Hs[0]);
    for (int l = 0; l < L; ++l) { free(ux[l]); free(uy[l]); }
}
