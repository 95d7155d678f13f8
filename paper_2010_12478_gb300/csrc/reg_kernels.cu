// Device kernels of libreg: pyramid build and the registration operator.
//
// Design (GB300, sm_103a):
//   * One operator application (A or B, Sec. 2.3.1-2.3.2) runs start to finish
//     inside ONE thread-block cluster: every level, every gradient-flow
//     iteration and every Armijo trial.  The C CTAs of the cluster split the
//     rows of each pyramid level; their partial sums meet through distributed
//     shared memory, so an iteration costs one cluster barrier and never a
//     kernel launch or a grid-wide synchronisation.
//   * Per pixel the work is FP32 (warp, bilinear sample, derivative, moment
//     products).  Sums are accumulated per thread in FP32 over chunks of 32
//     pixels, then carried as float-float pairs (error-free transformations on
//     the FP32 pipes: GB300's FP64 rate is a small fraction of FP32) through the
//     warp and CTA stages, and in FP64 across the cluster.  Reduction order is
//     fixed, so results are bitwise reproducible for a given cluster size.
//   * The step controller (NCC from the moments, gradient, Armijo test, step
//     size, stop rules) is FP64 and runs on thread 0 of every CTA of the
//     cluster on identical totals, so all CTAs take identical decisions.
//   * Images are read through the read-only path; the nonrigid fields, which
//     the cluster rewrites between passes, through L2 (ld/st .cg) with a fence
//     before each cluster barrier.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "reg_internal.h"

namespace cg = cooperative_groups;

namespace reg {

constexpr int kWarps = kThreads / 32;
constexpr int kNM = 16;        // moment slots per reduction
constexpr int kChunk = 32;     // pixels per thread between float-float flushes

// ------------------------------------------------------------------ loads
template <typename S> __device__ __forceinline__ float ldS(const S *p);
template <> __device__ __forceinline__ float ldS<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldS<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float ldS<__half>(const __half *p) { return __half2float(__ldg(p)); }

template <typename S> __device__ __forceinline__ S toS(float v);
template <> __device__ __forceinline__ float toS<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 toS<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half toS<__half>(float v) { return __float2half_rn(v); }

// ------------------------------------------------------------------ float-float
// (hi, lo) += x, exactly up to the final rounding of lo (Knuth's TwoSum).
__device__ __forceinline__ void ff_acc(float &hi, float &lo, float x)
{
    float s = __fadd_rn(hi, x);
    float bp = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// (hi, lo) += (h2, l2), renormalised.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float h2, float l2)
{
    float s = __fadd_rn(hi, h2);
    float bp = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(h2, bp));
    e = __fadd_rn(e, __fadd_rn(lo, l2));
    float h = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(h, s));
    hi = h;
}

// ------------------------------------------------------------------ shared state
struct Smem {
    float2 warp[kWarps][kNM];   // per-warp (hi, lo) partials
    double part[2][kNM];        // this CTA's partials, read by the whole cluster
    double tot[kNM];            // cluster totals
    float pm[16];               // pass parameters broadcast by thread 0
    int action;
    int idata[4];
};

// Reduce NM per-thread float-float partials over the cluster into sm.tot.
// If MAXLAST, slot NM-1 holds a non-negative value combined by max (hi only).
template <int NM, bool MAXLAST>
__device__ __forceinline__ void cluster_reduce(float (&hi)[NM], float (&lo)[NM], Smem &sm,
                                               int &buf, const cg::cluster_group &cl, bool fence)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            float h2 = __shfl_xor_sync(0xffffffffu, hi[m], off);
            float l2 = __shfl_xor_sync(0xffffffffu, lo[m], off);
            if (MAXLAST && m == NM - 1) hi[m] = fmaxf(hi[m], h2);
            else ff_add(hi[m], lo[m], h2, l2);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int m = 0; m < NM; ++m) sm.warp[w][m] = make_float2(hi[m], lo[m]);
    }
    __syncthreads();
    if (tid < NM) {
        float h = 0.f, l = 0.f;
        for (int k = 0; k < kWarps; ++k) {
            float2 v = sm.warp[k][tid];
            if (MAXLAST && tid == NM - 1) h = fmaxf(h, v.x);
            else ff_add(h, l, v.x, v.y);
        }
        sm.part[buf][tid] = (double)h + (double)l;
    }
    if (fence) __threadfence();
    cl.sync();
    if (tid < NM) {
        double s = 0.0;
        const unsigned C = cl.num_blocks();
        for (unsigned r = 0; r < C; ++r) {
            double v = *cl.map_shared_rank(&sm.part[buf][tid], r);
            if (MAXLAST && tid == NM - 1) s = fmax(s, v);
            else s = __dadd_rn(s, v);
        }
        sm.tot[tid] = s;
    }
    buf ^= 1;
    __syncthreads();
}

__device__ __forceinline__ void cluster_barrier(const cg::cluster_group &cl)
{
    __threadfence();
    cl.sync();
}

// ------------------------------------------------------------------ NCC (FP64)
struct Ncc {
    double ncc, a, b, rbar, tbar;   // means of the shifted samples
    int degenerate;
};

// NCC = S'_RT / sqrt(S'_RR S'_TT) from shifted sums; dNCC/dTw(x) = a (r - rbar) - b (t - tbar).
// Explicit round-to-nearest operations keep the result independent of FMA contraction,
// so identical inputs (t == r) give exactly NCC = 1 and a zero gradient.
__device__ Ncc ncc_terms(double P, double sr, double st, double srr, double stt, double srt)
{
    Ncc o;
    double Srr = __dsub_rn(srr, __ddiv_rn(__dmul_rn(sr, sr), P));
    double Stt = __dsub_rn(stt, __ddiv_rn(__dmul_rn(st, st), P));
    double Srt = __dsub_rn(srt, __ddiv_rn(__dmul_rn(sr, st), P));
    o.rbar = __ddiv_rn(sr, P);
    o.tbar = __ddiv_rn(st, P);
    if (Srr < 1e-12 * P || Stt < 1e-12 * P) {
        o.ncc = 0.0; o.a = 0.0; o.b = 0.0; o.degenerate = 1;
        return o;
    }
    double root = __dsqrt_rn(__dmul_rn(Srr, Stt));
    o.ncc = __ddiv_rn(Srt, root);
    o.a = __ddiv_rn(1.0, root);
    o.b = __ddiv_rn(o.ncc, Stt);
    o.degenerate = 0;
    return o;
}

// ------------------------------------------------------------------ level access
struct Lvl {
    const void *R, *T;
    int W, H, Rp, Tp;
    float cR;   // shift constant (mean of the reference level)
};

__device__ __forceinline__ void strip_rows(int H, int rank, int C, int &r0, int &r1)
{
    int per = (H + C - 1) / C;
    r0 = min(H, rank * per);
    r1 = min(H, r0 + per);
}

// Iterate the pixels of rows [r0, r1): f(r, c) per pixel; flush_fast() after every
// kFast pixels of this thread and flush() after every kChunk pixels (and at the end).
constexpr int kFast = 8;
template <typename F, typename G, typename Q>
__device__ __forceinline__ void for_pixels2(int W, int r0, int r1, F &&f, Q &&flush_fast, G &&flush)
{
    const int tid = threadIdx.x;
    int i = r0 * W + tid;
    const int end = r1 * W;
    int r = i / W, c = i - r * W;
    const int dr = kThreads / W, dc = kThreads - dr * W;
    while (i < end) {
#pragma unroll 1
        for (int q = 0; q < kChunk / kFast && i < end; ++q) {
#pragma unroll 1
            for (int k = 0; k < kFast && i < end; ++k) {
                f(r, c);
                i += kThreads;
                c += dc; r += dr;
                if (c >= W) { c -= W; r += 1; }
            }
            flush_fast();
        }
        flush();
    }
}

template <typename F, typename G>
__device__ __forceinline__ void for_pixels(int W, int r0, int r1, F &&f, G &&flush)
{
    for_pixels2(W, r0, r1, f, []() {}, flush);
}

// Bilinear sample of T (storage S, pitch Tp) at p = (xi + vx, yi + vy) with clamp-to-edge,
// where (xi, yi) is an integer pixel and (vx, vy) a small FP32 offset.  Splitting the
// position keeps the FP32 fractional part exact to the precision of the offset, not
// of the absolute coordinate.  Cell choice and clamping follow floor(p) clamped to
// [0, W-2]; the derivative along a clamped axis (p < 0 or p > W-1) is 0.
template <typename S, bool DERIV>
__device__ __forceinline__ float sample_at(const S *T, int W, int H, int Tp, int xi, int yi, float vx, float vy,
                                           float &dtx, float &dty)
{
    vx = fminf(fmaxf(vx, -1.0e6f), 1.0e6f);   // also maps NaN into range: every access stays in bounds
    vy = fminf(fmaxf(vy, -1.0e6f), 1.0e6f);
    const float flx = floorf(vx), fly = floorf(vy);
    int x = xi + (int)flx, y = yi + (int)fly;
    float fx = vx - flx, fy = vy - fly;
    bool clx = false, cly = false;
    if (x < 0) { x = 0; fx = 0.f; clx = true; }
    else if (x > W - 2) { clx = (x > W - 1) || (fx > 0.f); x = W - 2; fx = 1.f; }
    if (y < 0) { y = 0; fy = 0.f; cly = true; }
    else if (y > H - 2) { cly = (y > H - 1) || (fy > 0.f); y = H - 2; fy = 1.f; }
    const S *row = T + (size_t)y * Tp + x;
    float t00 = ldS<S>(row), t01 = ldS<S>(row + 1);
    float t10 = ldS<S>(row + Tp), t11 = ldS<S>(row + Tp + 1);
    float gx = 1.f - fx, gy = 1.f - fy;
    float top = fmaf(fx, t01, gx * t00);
    float bot = fmaf(fx, t11, gx * t10);
    if (DERIV) {
        dtx = clx ? 0.f : fmaf(fy, t11 - t10, gy * (t01 - t00));
        dty = cly ? 0.f : (bot - top);
    }
    return fmaf(fy, bot, gy * top);
}

// Bilinear value (no derivative) of an fp32 field read through L2, at (xi + vx, yi + vy).
__device__ __forceinline__ float sample_cg(const float *F, int W, int H, int xi, int yi, float vx, float vy)
{
    vx = fminf(fmaxf(vx, -1.0e6f), 1.0e6f);
    vy = fminf(fmaxf(vy, -1.0e6f), 1.0e6f);
    const float flx = floorf(vx), fly = floorf(vy);
    int x = xi + (int)flx, y = yi + (int)fly;
    float fx = vx - flx, fy = vy - fly;
    if (x < 0) { x = 0; fx = 0.f; } else if (x > W - 2) { x = W - 2; fx = 1.f; }
    if (y < 0) { y = 0; fy = 0.f; } else if (y > H - 2) { y = H - 2; fy = 1.f; }
    const float *row = F + (size_t)y * W + x;
    float t00 = __ldcg(row), t01 = __ldcg(row + 1), t10 = __ldcg(row + W), t11 = __ldcg(row + W + 1);
    float gx = 1.f - fx;
    float top = fmaf(fx, t01, gx * t00);
    float bot = fmaf(fx, t11, gx * t10);
    return fmaf(fy, bot, (1.f - fy) * top);
}

// ================================================================== rigid
// Moment slots: 0 St, 1 Stt, 2 Srt, 3 Sr, 4 Srr, 5..7 Srg_k, 8..10 Stg_k, 11..13 Sg_k.
template <typename S, int NM, bool GRAD>
__device__ void eval_rigid(const Lvl &L, int r0, int r1, const float *pm, Smem &sm, int &buf,
                           const cg::cluster_group &cl)
{
    // pm: cos(alpha) - 1, sin(alpha), fractional translation (x, y), integer translation (x, y)
    const float cm1 = pm[0], sa = pm[1], gfx = pm[2], gfy = pm[3];
    const int gix = (int)pm[4], giy = (int)pm[5];
    const float cx = 0.5f * (float)(L.W - 1), cy = 0.5f * (float)(L.H - 1);
    const S *R = (const S *)L.R, *T = (const S *)L.T;
    float hi[NM], lo[NM], a[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) { hi[m] = 0.f; lo[m] = 0.f; a[m] = 0.f; }
    for_pixels2(
        L.W, r0, r1,
        [&](int r, int c) {
            float xc = (float)c - cx, yc = (float)r - cy;
            // phi(x) - x - integer translation: small, so FP32 keeps it to ~1e-7 relative
            float vx = fmaf(cm1, xc, fmaf(-sa, yc, gfx));
            float vy = fmaf(sa, xc, fmaf(cm1, yc, gfy));
            float dtx, dty;
            float tw = sample_at<S, GRAD>(T, L.W, L.H, L.Tp, c + gix, r + giy, vx, vy, dtx, dty);
            float rv = ldS<S>(R + (size_t)r * L.Rp + c) - L.cR;
            float tv = tw - L.cR;
            a[0] += tv;
            a[1] = fmaf(tv, tv, a[1]);
            a[2] = fmaf(rv, tv, a[2]);
            if constexpr (NM > 3) {
                a[3] += rv;
                a[4] = fmaf(rv, rv, a[4]);
            }
            if constexpr (GRAD) {
                // g_alpha = dT . dphi/dalpha, dphi/dalpha = Rot'(alpha) (x - c)
                const float ca = 1.f + cm1;
                float g0 = fmaf(dty, fmaf(ca, xc, -sa * yc), -dtx * fmaf(sa, xc, ca * yc));
                a[5] = fmaf(rv, g0, a[5]);
                a[6] = fmaf(rv, dtx, a[6]);
                a[7] = fmaf(rv, dty, a[7]);
                a[8] = fmaf(tv, g0, a[8]);
                a[9] = fmaf(tv, dtx, a[9]);
                a[10] = fmaf(tv, dty, a[10]);
                a[11] += g0;
                a[12] += dtx;
                a[13] += dty;
            }
        },
        [&]() {
            // energy moments: short FP32 runs keep 1 - NCC accurate to ~1e-9
#pragma unroll
            for (int m = 0; m < (NM < 5 ? NM : 5); ++m) { ff_acc(hi[m], lo[m], a[m]); a[m] = 0.f; }
        },
        [&]() {
#pragma unroll
            for (int m = 5; m < NM; ++m) { ff_acc(hi[m], lo[m], a[m]); a[m] = 0.f; }
        });
    cluster_reduce<NM, false>(hi, lo, sm, buf, cl, false);
}

enum Action { kActGrad = 0, kActTrial = 1, kActDone = 2, kActEnergy = 3, kActField = 4 };

struct RigidCtl {
    double th[3], tt[3], d[3];
    double E, tau, slope, sr, srr, m0, P, cx, cy;
    int nrej, iters, evals, stop, rejects;
};

__device__ void rigid_params(const RigidCtl &k, const double *th, float *pm)
{
    const float a = (float)th[0];
    const float h = sinf(0.5f * a);
    pm[0] = -2.f * h * h;            // cos(a) - 1 without cancellation
    pm[1] = sinf(a);
    const double ix = rint(th[1]), iy = rint(th[2]);
    pm[2] = (float)(th[1] - ix);
    pm[3] = (float)(th[2] - iy);
    pm[4] = (float)fmax(-4.0e6, fmin(4.0e6, ix));
    pm[5] = (float)fmax(-4.0e6, fmin(4.0e6, iy));
    (void)k;
}

// Thread-0 controller step after a GRAD (first == true: the level's first) or TRIAL pass.
// Returns the next action and writes the pass parameters.
__device__ int rigid_step(RigidCtl &k, const Config &cfg, const double *tot, int action, bool first,
                          float *pm)
{
    if (action == kActGrad) {
        if (first) { k.sr = tot[3]; k.srr = tot[4]; }
        Ncc n = ncc_terms(k.P, k.sr, tot[0], k.srr, tot[1], tot[2]);
        double g[3];
        if (n.degenerate) {
            k.E = 1.0; g[0] = g[1] = g[2] = 0.0;
        } else {
            k.E = __dsub_rn(1.0, n.ncc);
            for (int q = 0; q < 3; ++q) {
                double x = __dsub_rn(tot[5 + q], __dmul_rn(n.rbar, tot[11 + q]));
                double y = __dsub_rn(tot[8 + q], __dmul_rn(n.tbar, tot[11 + q]));
                g[q] = -__dsub_rn(__dmul_rn(n.a, x), __dmul_rn(n.b, y));
            }
        }
        k.evals += 1;
        if (k.iters >= cfg.max_iter) { k.stop = REG_STOP_MAXIT; return kActDone; }
        k.d[0] = -g[0] / k.m0; k.d[1] = -g[1]; k.d[2] = -g[2];
        k.slope = g[0] * k.d[0] + g[1] * k.d[1] + g[2] * k.d[2];
        double gn = sqrt(-k.slope);
        if (!(gn >= cfg.tol_grad)) { k.stop = REG_STOP_GRAD; return kActDone; }
        if (k.tau * gn > cfg.step_cap) k.tau = cfg.step_cap / gn;
        k.nrej = 0;
        for (int q = 0; q < 3; ++q) k.tt[q] = k.th[q] + k.tau * k.d[q];
        rigid_params(k, k.tt, pm);
        return kActTrial;
    }
    // trial
    Ncc n = ncc_terms(k.P, k.sr, tot[0], k.srr, tot[1], tot[2]);
    double Et = n.degenerate ? 1.0 : __dsub_rn(1.0, n.ncc);
    k.evals += 1;
    if (Et <= k.E + cfg.armijo_c * k.tau * k.slope) {
        for (int q = 0; q < 3; ++q) k.th[q] = k.tt[q];
        k.iters += 1;
        double Eold = k.E;
        k.E = Et;
        k.tau *= 2.0;
        if (Eold - Et <= cfg.tol_rel_e * fabs(Eold)) { k.stop = REG_STOP_REL; return kActDone; }
        rigid_params(k, k.th, pm);
        return kActGrad;
    }
    k.rejects += 1;
    k.nrej += 1;
    k.tau *= 0.5;
    if (k.nrej > cfg.max_rejects) { k.stop = REG_STOP_LS; return kActDone; }
    for (int q = 0; q < 3; ++q) k.tt[q] = k.th[q] + k.tau * k.d[q];
    rigid_params(k, k.tt, pm);
    return kActTrial;
}

__device__ __forceinline__ Lvl level_of(const Params &p, int ref, int tmpl, int l)
{
    const LevelDesc &a = p.levels[ref * p.cfg.levels + l];
    const LevelDesc &b = p.levels[tmpl * p.cfg.levels + l];
    Lvl L;
    L.R = a.ptr; L.T = b.ptr; L.W = a.W; L.H = a.H; L.Rp = a.pitch; L.Tp = b.pitch; L.cR = a.mean;
    return L;
}

template <typename S>
__device__ void run_rigid(const Params &p, const OpDesc &op, int op_index, Smem &sm,
                          const cg::cluster_group &cl)
{
    const int tid = threadIdx.x;
    const int C = cl.num_blocks(), rank = cl.block_rank();
    const Config &cfg = p.cfg;
    int buf = 0;
    RigidCtl k;
    if (tid == 0) {
        memset(&k, 0, sizeof(k));
        double th0[3] = {0.0, 0.0, 0.0};
        if (op.left >= 0) {
            // B's initial guess phi_jk o phi_ij in centred coordinates (Sec. 2.3.2)
            // node states come from other clusters: read through L2, never a stale L1 line
            const double *pa = p.node_theta + 3 * op.left, *pb = p.node_theta + 3 * op.right;
            double a[3] = {__ldcg(pa), __ldcg(pa + 1), __ldcg(pa + 2)};
            double b[3] = {__ldcg(pb), __ldcg(pb + 1), __ldcg(pb + 2)};
            float s, c;
            sincosf((float)b[0], &s, &c);
            double cb = c, sb = s;
            th0[0] = a[0] + b[0];
            th0[1] = cb * a[1] - sb * a[2] + b[1];
            th0[2] = sb * a[1] + cb * a[2] + b[2];
        } else if (op.init_node >= 0) {
            const double *pa = p.node_theta + 3 * op.init_node;
            th0[0] = __ldcg(pa); th0[1] = __ldcg(pa + 1); th0[2] = __ldcg(pa + 2);
        }
        k.th[0] = th0[0];
        k.th[1] = ldexp(th0[1], -(cfg.levels - 1));
        k.th[2] = ldexp(th0[2], -(cfg.levels - 1));
    }
    int stops[kMaxLevels], iters[kMaxLevels], evals[kMaxLevels];
    for (int l = cfg.levels - 1; l >= 0; --l) {
        const Lvl L = level_of(p, op.ref, op.tmpl, l);
        int r0, r1;
        strip_rows(L.H, rank, C, r0, r1);
        if (tid == 0) {
            k.P = (double)L.W * (double)L.H;
            k.cx = 0.5 * (L.W - 1);
            k.cy = 0.5 * (L.H - 1);
            double rho = 0.25 * (L.W + L.H);
            k.m0 = rho * rho;
            k.tau = cfg.tau0;
            k.iters = 0; k.evals = 0; k.stop = REG_STOP_MAXIT;
            rigid_params(k, k.th, sm.pm);
            sm.action = kActGrad;
        }
        bool first = true;
        for (;;) {
            __syncthreads();
            const int act = sm.action;
            if (act == kActDone) break;
            float pm[6] = {sm.pm[0], sm.pm[1], sm.pm[2], sm.pm[3], sm.pm[4], sm.pm[5]};
            if (act == kActGrad) {
                eval_rigid<S, 14, true>(L, r0, r1, pm, sm, buf, cl);
            } else {
                eval_rigid<S, 3, false>(L, r0, r1, pm, sm, buf, cl);
            }
            if (tid == 0) sm.action = rigid_step(k, cfg, sm.tot, act, first && act == kActGrad, sm.pm);
            if (act == kActGrad) first = false;
        }
        if (tid == 0) {
            stops[l] = k.stop; iters[l] = k.iters; evals[l] = k.evals;
            if (l > 0) { k.th[1] *= 2.0; k.th[2] *= 2.0; }
        }
        __syncthreads();
    }
    if (tid == 0 && rank == 0) {
        double *o = p.node_theta + 3 * op.out;
        __stcg(o, k.th[0]); __stcg(o + 1, k.th[1]); __stcg(o + 2, k.th[2]);
        OpStats &st = p.stats[op_index];
        st.i = op.ref;
        st.k = op.tmpl;
        for (int l = 0; l < kMaxLevels; ++l) {
            bool v = l < cfg.levels;
            st.iters[l] = v ? iters[l] : 0;
            st.evals[l] = v ? evals[l] : 0;
            st.stop[l] = v ? stops[l] : 0;
        }
        st.rejects = k.rejects;
        st.status = kDevOk;
        st.energy = k.E;
        st.theta[0] = o[0]; st.theta[1] = o[1]; st.theta[2] = o[2];
    }
}

// ================================================================== nonrigid
// Work buffers of one slot: per level l, 8 planes of W_l*H_l floats:
// U0x U0y U1x U1y D0x D0y D1x D1y.
struct FieldLvl {
    float *base;
    int W, H;
    __device__ float *U(int b, int comp) const { return base + (size_t)(2 * b + comp) * W * H; }
    __device__ float *D(int b, int comp) const { return base + (size_t)(4 + 2 * b + comp) * W * H; }
};

__device__ __forceinline__ FieldLvl field_level(const Params &p, int slot, int l)
{
    size_t off = 0;
    int W = 0, H = 0;
    for (int q = 0; q <= l; ++q) {
        const LevelDesc &d = p.levels[q];   // frame 0's geometry: every frame has the same size
        if (q < l) off += (size_t)8 * d.W * d.H;
        W = d.W; H = d.H;
    }
    FieldLvl f;
    f.base = p.scratch + (size_t)slot * p.scratch_floats + off;
    f.W = W; f.H = H;
    return f;
}

// u(x) = U(x) + tau * D(x) (tau == 0: D is not read)
__device__ __forceinline__ float2 u_at(const FieldLvl &F, int b, size_t i, float tau)
{
    float ux = __ldcg(F.U(b, 0) + i), uy = __ldcg(F.U(b, 1) + i);
    if (tau != 0.f) {
        ux = fmaf(tau, __ldcg(F.D(b, 0) + i), ux);
        uy = fmaf(tau, __ldcg(F.D(b, 1) + i), uy);
    }
    return make_float2(ux, uy);
}

// Energy of the field U_b + tau D_b: slots 0 St, 1 Stt, 2 Srt, 3 Sr, 4 Srr, 5 sum |forward diff|^2.
template <typename S>
__device__ void eval_field_energy(const Lvl &L, const FieldLvl &F, int b, float tau, int r0, int r1,
                                  Smem &sm, int &buf, const cg::cluster_group &cl)
{
    const S *R = (const S *)L.R, *T = (const S *)L.T;
    constexpr int NM = 6;
    float hi[NM], lo[NM], a[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) { hi[m] = 0.f; lo[m] = 0.f; a[m] = 0.f; }
    const int W = L.W, H = L.H;
    for_pixels2(
        W, r0, r1,
        [&](int r, int c) {
            size_t i = (size_t)r * W + c;
            float2 u = u_at(F, b, i, tau);
            float dtx, dty;
            float tw = sample_at<S, false>(T, W, H, L.Tp, c, r, u.x, u.y, dtx, dty);
            float rv = ldS<S>(R + (size_t)r * L.Rp + c) - L.cR;
            float tv = tw - L.cR;
            a[0] += tv;
            a[1] = fmaf(tv, tv, a[1]);
            a[2] = fmaf(rv, tv, a[2]);
            a[3] += rv;
            a[4] = fmaf(rv, rv, a[4]);
            float reg = 0.f;
            if (c + 1 < W) {
                float2 v = u_at(F, b, i + 1, tau);
                float ex = v.x - u.x, ey = v.y - u.y;
                reg = fmaf(ex, ex, fmaf(ey, ey, reg));
            }
            if (r + 1 < H) {
                float2 v = u_at(F, b, i + W, tau);
                float ex = v.x - u.x, ey = v.y - u.y;
                reg = fmaf(ex, ex, fmaf(ey, ey, reg));
            }
            a[5] += reg;
        },
        [&]() {
#pragma unroll
            for (int m = 0; m < 5; ++m) { ff_acc(hi[m], lo[m], a[m]); a[m] = 0.f; }
        },
        [&]() { ff_acc(hi[5], lo[5], a[5]); a[5] = 0.f; });
    cluster_reduce<NM, false>(hi, lo, sm, buf, cl, false);
}

// Field pass: u = U_b + tau D_b materialised into U_{1-b}; descent direction
// d = -P dE/du = -(fP grad T(x + u) + lambda * sum_nbrs (u(x) - u(y))) into D_{1-b};
// reduces sum |d|^2 and max |d|^2.  pm: tau, aP, bP, rbar, tbar, lambda.
template <typename S>
__device__ void eval_field_grad(const Lvl &L, const FieldLvl &F, int b, const float *pm, int r0, int r1,
                                Smem &sm, int &buf, const cg::cluster_group &cl)
{
    const S *R = (const S *)L.R, *T = (const S *)L.T;
    const float tau = pm[0], aP = pm[1], bP = pm[2], rb = pm[3], tb = pm[4], lam = pm[5];
    constexpr int NM = 2;
    float hi[NM] = {0.f, 0.f}, lo[NM] = {0.f, 0.f}, a[NM] = {0.f, 0.f};
    const int W = L.W, H = L.H;
    const int nb = 1 - b;
    for_pixels(
        W, r0, r1,
        [&](int r, int c) {
            size_t i = (size_t)r * W + c;
            float2 u = u_at(F, b, i, tau);
            float lx = 0.f, ly = 0.f;
            if (c > 0)     { float2 v = u_at(F, b, i - 1, tau); lx += u.x - v.x; ly += u.y - v.y; }
            if (c + 1 < W) { float2 v = u_at(F, b, i + 1, tau); lx += u.x - v.x; ly += u.y - v.y; }
            if (r > 0)     { float2 v = u_at(F, b, i - W, tau); lx += u.x - v.x; ly += u.y - v.y; }
            if (r + 1 < H) { float2 v = u_at(F, b, i + W, tau); lx += u.x - v.x; ly += u.y - v.y; }
            float dtx, dty;
            float tw = sample_at<S, true>(T, W, H, L.Tp, c, r, u.x, u.y, dtx, dty);
            float rv = ldS<S>(R + (size_t)r * L.Rp + c) - L.cR;
            float tv = tw - L.cR;
            // fP = P * dE_data/dTw = -(aP (r - rbar) - bP (t - tbar)), no contraction
            float fP = -__fsub_rn(__fmul_rn(aP, rv - rb), __fmul_rn(bP, tv - tb));
            float dx = -fmaf(fP, dtx, lam * lx);
            float dy = -fmaf(fP, dty, lam * ly);
            __stcg(F.U(nb, 0) + i, u.x);
            __stcg(F.U(nb, 1) + i, u.y);
            __stcg(F.D(nb, 0) + i, dx);
            __stcg(F.D(nb, 1) + i, dy);
            float q = fmaf(dx, dx, dy * dy);
            a[0] += q;
            a[1] = fmaxf(a[1], q);
        },
        [&]() {
            ff_acc(hi[0], lo[0], a[0]);
            a[0] = 0.f;
            hi[1] = fmaxf(hi[1], a[1]);
        });
    cluster_reduce<NM, true>(hi, lo, sm, buf, cl, true);
}

struct FieldCtl {
    double E, tau, tau_pend, slope, P, sr, srr;
    double a, b, rbar, tbar;      // NCC terms at the current field
    double ta, tb, trbar, ttbar;  // at the trial field
    int degen, tdegen;
    int nrej, iters, evals, stop, rejects, cur;
};

__device__ double field_energy(FieldCtl &k, const Config &cfg, const double *tot, bool trial)
{
    Ncc n = ncc_terms(k.P, k.sr, tot[0], k.srr, tot[1], tot[2]);
    double Ed = n.degenerate ? 1.0 : __dsub_rn(1.0, n.ncc);
    double E = Ed + 0.5 * cfg.lambda * tot[5] / k.P;
    if (trial) { k.ta = n.a; k.tb = n.b; k.trbar = n.rbar; k.ttbar = n.tbar; k.tdegen = n.degenerate; }
    else { k.a = n.a; k.b = n.b; k.rbar = n.rbar; k.tbar = n.tbar; k.degen = n.degenerate; }
    return E;
}

__device__ void field_params(const FieldCtl &k, const Config &cfg, float tau, float *pm)
{
    pm[0] = tau;
    pm[1] = (float)(k.a * k.P);
    pm[2] = (float)(k.b * k.P);
    pm[3] = (float)k.rbar;
    pm[4] = (float)k.tbar;
    pm[5] = (float)cfg.lambda;
}

// Thread-0 controller of the nonrigid level loop; mirrors rigid_step with the
// field passes (ENERGY at level start, FIELD = gradient, TRIAL = Armijo trial).
__device__ int field_step(FieldCtl &k, const Config &cfg, const double *tot, int action, float *pm)
{
    if (action == kActEnergy) {
        k.sr = tot[3]; k.srr = tot[4];
        k.E = field_energy(k, cfg, tot, false);
        k.tau_pend = 0.0;
        field_params(k, cfg, 0.f, pm);
        return kActField;
    }
    if (action == kActField) {
        k.evals += 1;
        k.cur ^= 1;
        k.tau_pend = 0.0;
        if (k.iters >= cfg.max_iter) { k.stop = REG_STOP_MAXIT; return kActDone; }
        double ss = tot[0], dmax = sqrt(tot[1]);
        k.slope = -ss / k.P;
        double gn = sqrt(ss / k.P);
        if (!(gn >= cfg.tol_grad)) { k.stop = REG_STOP_GRAD; return kActDone; }
        if (k.tau * dmax > cfg.step_cap) k.tau = cfg.step_cap / dmax;
        k.nrej = 0;
        pm[0] = (float)k.tau;
        return kActTrial;
    }
    // trial
    double Et = field_energy(k, cfg, tot, true);
    k.evals += 1;
    if (Et <= k.E + cfg.armijo_c * k.tau * k.slope) {
        k.iters += 1;
        double Eold = k.E;
        k.E = Et;
        k.a = k.ta; k.b = k.tb; k.rbar = k.trbar; k.tbar = k.ttbar; k.degen = k.tdegen;
        k.tau_pend = (double)(float)k.tau;   // the step the trial pass applied
        k.tau *= 2.0;
        if (Eold - Et <= cfg.tol_rel_e * fabs(Eold)) { k.stop = REG_STOP_REL; return kActDone; }
        field_params(k, cfg, (float)k.tau_pend, pm);
        return kActField;
    }
    k.rejects += 1;
    k.nrej += 1;
    k.tau *= 0.5;
    if (k.nrej > cfg.max_rejects) { k.stop = REG_STOP_LS; return kActDone; }
    pm[0] = (float)k.tau;
    return kActTrial;
}

// Composition (B's initial guess) into U_0 of level 0: u1(x) + u2(x + u1(x)).
__device__ void field_compose(const float *u1, const float *u2, const FieldLvl &F, int r0, int r1)
{
    const int W = F.W, H = F.H;
    const size_t P = (size_t)W * H;
    for_pixels(
        W, r0, r1,
        [&](int r, int c) {
            size_t i = (size_t)r * W + c;
            float ax = __ldcg(u1 + i), ay = __ldcg(u1 + P + i);
            __stcg(F.U(0, 0) + i, ax + sample_cg(u2, W, H, c, r, ax, ay));
            __stcg(F.U(0, 1) + i, ay + sample_cg(u2 + P, W, H, c, r, ax, ay));
        },
        []() {});
}

// Restriction of an initial field, level l -> l+1: box average, halved.
__device__ void field_restrict(const FieldLvl &Ff, const FieldLvl &Fc, int r0, int r1)
{
    for_pixels(
        Fc.W, r0, r1,
        [&](int r, int c) {
            int ra = 2 * r, rb = min(2 * r + 1, Ff.H - 1), ca = 2 * c, cb = min(2 * c + 1, Ff.W - 1);
            for (int comp = 0; comp < 2; ++comp) {
                const float *s = Ff.U(0, comp);
                float v = (__ldcg(s + (size_t)ra * Ff.W + ca) + __ldcg(s + (size_t)ra * Ff.W + cb)) +
                          (__ldcg(s + (size_t)rb * Ff.W + ca) + __ldcg(s + (size_t)rb * Ff.W + cb));
                __stcg(Fc.U(0, comp) + (size_t)r * Fc.W + c, 0.125f * v);
            }
        },
        []() {});
}

// Prolongation, level l+1 -> l: u_l(x) = 2 bilinear(u_{l+1}, ((c - 0.5)/2, (r - 0.5)/2)),
// u_{l+1} = U_b + tau D_b of the coarse level.
__device__ void field_prolong(const FieldLvl &Fc, int b, float tau, const FieldLvl &Ff, int r0, int r1)
{
    for_pixels(
        Ff.W, r0, r1,
        [&](int r, int c) {
            float px = 0.5f * ((float)c - 0.5f), py = 0.5f * ((float)r - 0.5f);
            float qx = fminf(fmaxf(px, 0.f), (float)(Fc.W - 1));
            float qy = fminf(fmaxf(py, 0.f), (float)(Fc.H - 1));
            int x0 = min((int)qx, Fc.W - 2), y0 = min((int)qy, Fc.H - 2);
            float fx = qx - (float)x0, fy = qy - (float)y0;
            size_t i00 = (size_t)y0 * Fc.W + x0;
            float2 t00 = u_at(Fc, b, i00, tau), t01 = u_at(Fc, b, i00 + 1, tau);
            float2 t10 = u_at(Fc, b, i00 + Fc.W, tau), t11 = u_at(Fc, b, i00 + Fc.W + 1, tau);
            float gx = 1.f - fx, gy = 1.f - fy;
            float topx = fmaf(fx, t01.x, gx * t00.x), botx = fmaf(fx, t11.x, gx * t10.x);
            float topy = fmaf(fx, t01.y, gx * t00.y), boty = fmaf(fx, t11.y, gx * t10.y);
            size_t i = (size_t)r * Ff.W + c;
            __stcg(Ff.U(0, 0) + i, 2.f * fmaf(fy, botx, gy * topx));
            __stcg(Ff.U(0, 1) + i, 2.f * fmaf(fy, boty, gy * topy));
        },
        []() {});
}

template <typename S>
__device__ void run_nonrigid(const Params &p, const OpDesc &op, int op_index, int slot, Smem &sm,
                             const cg::cluster_group &cl)
{
    const int tid = threadIdx.x;
    const int C = cl.num_blocks(), rank = cl.block_rank();
    const Config &cfg = p.cfg;
    const int Lc = cfg.levels;
    int buf = 0;
    const FieldLvl F0 = field_level(p, slot, 0);
    const size_t P0 = (size_t)F0.W * F0.H;
    // initial field at level 0 (U_0), then restricted down to the coarsest level
    {
        int r0, r1;
        strip_rows(F0.H, rank, C, r0, r1);
        bool have_init = true;
        if (op.left >= 0) {
            field_compose(p.node_field + 2 * P0 * op.left, p.node_field + 2 * P0 * op.right, F0, r0, r1);
        } else if (op.init_node >= 0) {
            const float *src = p.node_field + 2 * P0 * op.init_node;
            for_pixels(F0.W, r0, r1, [&](int r, int c) {
                size_t i = (size_t)r * F0.W + c;
                __stcg(F0.U(0, 0) + i, __ldcg(src + i));
                __stcg(F0.U(0, 1) + i, __ldcg(src + P0 + i));
            }, []() {});
        } else {
            have_init = false;
        }
        if (have_init) {
            for (int l = 0; l + 1 < Lc; ++l) {
                cluster_barrier(cl);
                FieldLvl Ff = field_level(p, slot, l), Fc = field_level(p, slot, l + 1);
                int q0, q1;
                strip_rows(Fc.H, rank, C, q0, q1);
                field_restrict(Ff, Fc, q0, q1);
            }
        } else {
            FieldLvl Fc = field_level(p, slot, Lc - 1);
            int q0, q1;
            strip_rows(Fc.H, rank, C, q0, q1);
            for_pixels(Fc.W, q0, q1, [&](int r, int c) {
                size_t i = (size_t)r * Fc.W + c;
                __stcg(Fc.U(0, 0) + i, 0.f);
                __stcg(Fc.U(0, 1) + i, 0.f);
            }, []() {});
        }
        cluster_barrier(cl);
    }
    FieldCtl k;
    if (tid == 0) memset(&k, 0, sizeof(k));
    int stops[kMaxLevels], iters[kMaxLevels], evals[kMaxLevels];
    int cur = 0;
    float tau_pend = 0.f;
    for (int l = Lc - 1; l >= 0; --l) {
        const Lvl L = level_of(p, op.ref, op.tmpl, l);
        const FieldLvl F = field_level(p, slot, l);
        int r0, r1;
        strip_rows(L.H, rank, C, r0, r1);
        if (tid == 0) {
            k.P = (double)L.W * (double)L.H;
            k.tau = cfg.tau0;
            k.iters = 0; k.evals = 0; k.stop = REG_STOP_MAXIT;
            k.cur = 0;
            sm.action = kActEnergy;
            sm.pm[0] = 0.f;
            sm.idata[0] = 0;
        }
        for (;;) {
            __syncthreads();
            const int act = sm.action;
            if (act == kActDone) break;
            float pm[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) pm[q] = sm.pm[q];
            cur = sm.idata[0];
            if (act == kActEnergy) eval_field_energy<S>(L, F, 0, 0.f, r0, r1, sm, buf, cl);
            else if (act == kActTrial) eval_field_energy<S>(L, F, cur, pm[0], r0, r1, sm, buf, cl);
            else eval_field_grad<S>(L, F, cur, pm, r0, r1, sm, buf, cl);
            if (tid == 0) {
                sm.action = field_step(k, cfg, sm.tot, act, sm.pm);
                sm.idata[0] = k.cur;
                sm.pm[8] = (float)k.tau_pend;
            }
        }
        cur = sm.idata[0];
        tau_pend = sm.pm[8];
        if (tid == 0) { stops[l] = k.stop; iters[l] = k.iters; evals[l] = k.evals; }
        if (l > 0) {
            const FieldLvl Ff = field_level(p, slot, l - 1);
            int q0, q1;
            strip_rows(Ff.H, rank, C, q0, q1);
            field_prolong(F, cur, tau_pend, Ff, q0, q1);
            cluster_barrier(cl);
            if (tid == 0) { sm.idata[0] = 0; sm.pm[8] = 0.f; }
            __syncthreads();
        }
    }
    // output: node field = U_cur + tau_pend D_cur at level 0; mean displacement reduced
    {
        int r0, r1;
        strip_rows(F0.H, rank, C, r0, r1);
        float *o = p.node_field + 2 * P0 * op.out;
        float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f}, a[2] = {0.f, 0.f};
        for_pixels(
            F0.W, r0, r1,
            [&](int r, int c) {
                size_t i = (size_t)r * F0.W + c;
                float2 u = u_at(F0, cur, i, tau_pend);
                __stcg(o + i, u.x);
                __stcg(o + P0 + i, u.y);
                a[0] += u.x;
                a[1] += u.y;
            },
            [&]() {
                ff_acc(hi[0], lo[0], a[0]); ff_acc(hi[1], lo[1], a[1]);
                a[0] = a[1] = 0.f;
            });
        cluster_reduce<2, false>(hi, lo, sm, buf, cl, true);
    }
    if (tid == 0 && rank == 0) {
        double *o = p.node_theta + 3 * op.out;
        o[0] = 0.0;
        o[1] = sm.tot[0] / (double)P0;
        o[2] = sm.tot[1] / (double)P0;
        OpStats &st = p.stats[op_index];
        st.i = op.ref;
        st.k = op.tmpl;
        for (int l = 0; l < kMaxLevels; ++l) {
            bool v = l < Lc;
            st.iters[l] = v ? iters[l] : 0;
            st.evals[l] = v ? evals[l] : 0;
            st.stop[l] = v ? stops[l] : 0;
        }
        st.rejects = k.rejects;
        st.status = kDevOk;
        st.energy = k.E;
        st.theta[0] = o[0]; st.theta[1] = o[1]; st.theta[2] = o[2];
    }
}

// ================================================================== kernels
__device__ bool op_valid(const Params &p, const OpDesc &op)
{
    auto node_ok = [&](int n) { return n >= 0 && n < p.n_nodes; };
    if (op.ref < 0 || op.ref >= p.n_frames || op.tmpl < 0 || op.tmpl >= p.n_frames) return false;
    if (!node_ok(op.out)) return false;
    if (op.left >= 0 && !(node_ok(op.left) && node_ok(op.right))) return false;
    if (op.left < 0 && op.init_node >= 0 && !node_ok(op.init_node)) return false;
    return true;
}

template <int MODE, typename S>
__device__ void run_op(const Params &p, int op_index, int slot, Smem &sm, const cg::cluster_group &cl)
{
    const OpDesc op = p.ops[op_index];
    if (!op_valid(p, op)) {
        if (threadIdx.x == 0 && cl.block_rank() == 0) {
            p.stats[op_index].status = kDevBadOp;
            atomicCAS(p.status, 0, (int)kDevBadOp);
        }
        return;
    }
    if constexpr (MODE == REG_RIGID) run_rigid<S>(p, op, op_index, sm, cl);
    else run_nonrigid<S>(p, op, op_index, slot, sm, cl);
}

// Batched launch: cluster q of the grid runs operator op_base + q.
template <int MODE, typename S>
__global__ void __launch_bounds__(kThreads, 2) op_kernel(Params p)
{
    __shared__ Smem sm;
    cg::cluster_group cl = cg::this_cluster();
    const int q = blockIdx.x / cl.num_blocks();
    run_op<MODE, S>(p, p.op_base + q, q, sm, cl);
    cl.sync();   // no CTA leaves while a peer may still read its shared memory
}

// Persistent launch: each cluster claims ready operators from the device queue
// until all n_ops have been claimed.  Every wait is bounded by queue.timeout_ns.
template <int MODE, typename S>
__global__ void __launch_bounds__(kThreads, 2) persistent_kernel(Params p)
{
    __shared__ Smem sm;
    cg::cluster_group cl = cg::this_cluster();
    const int worker = blockIdx.x / cl.num_blocks();
    const bool leader = cl.block_rank() == 0 && threadIdx.x == 0;
    for (;;) {
        if (leader) {
            int slot = atomicAdd(p.queue.head, 1);
            int op = -1;
            if (slot < p.n_ops) {
                volatile int *vs = p.queue.slots;
                long long t0 = (long long)clock64();
                unsigned long long start;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(start));
                unsigned ns = 64;
                for (;;) {
                    op = vs[slot];
                    if (op >= 0) break;
                    unsigned long long now;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                    if ((long long)(now - start) > p.queue.timeout_ns || *((volatile int *)p.status) != 0) {
                        atomicCAS(p.status, 0, (int)kDevQueueTimeout);
                        op = -2;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 4096) ns *= 2;
                }
                (void)t0;
                __threadfence();
            }
            sm.idata[1] = op;
        }
        cl.sync();
        const int op = *cl.map_shared_rank(&sm.idata[1], 0);
        cl.sync();
        if (op < 0) break;
        run_op<MODE, S>(p, op, worker, sm, cl);
        cl.sync();
        if (leader) {
            // publish the produced node and release its consumers
            __threadfence();
            const int node = p.ops[op].out;
            for (int e = p.queue.cons_start[node]; e < p.queue.cons_start[node + 1]; ++e) {
                int c = p.queue.consumers[e];
                if (atomicSub(p.queue.pending + c, 1) == 1) {
                    int t = atomicAdd(p.queue.tail, 1);
                    __threadfence();
                    atomicExch(p.queue.slots + t, c);
                }
            }
            atomicAdd(p.queue.done, 1);
        }
    }
    cl.sync();
}

// Energy/gradient at a given deformation for a single pair (one cluster of 1 CTA).
template <int MODE, typename S>
__global__ void __launch_bounds__(kThreads) energy_kernel(Params p, const double *theta, const float *field,
                                                          double *out, float *grad_field)
{
    __shared__ Smem sm;
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x;
    int buf = 0;
    const Lvl L = level_of(p, 0, 1, 0);
    if constexpr (MODE == REG_RIGID) {
        RigidCtl k;
        memset(&k, 0, sizeof(k));
        k.cx = 0.5 * (L.W - 1);
        k.cy = 0.5 * (L.H - 1);
        float pm[6];
        rigid_params(k, theta, pm);
        eval_rigid<S, 14, true>(L, 0, L.H, pm, sm, buf, cl);
        if (tid == 0) {
            double P = (double)L.W * L.H;
            Ncc n = ncc_terms(P, sm.tot[3], sm.tot[0], sm.tot[4], sm.tot[1], sm.tot[2]);
            out[0] = n.degenerate ? 1.0 : __dsub_rn(1.0, n.ncc);
            for (int q = 0; q < 3; ++q) {
                double x = __dsub_rn(sm.tot[5 + q], __dmul_rn(n.rbar, sm.tot[11 + q]));
                double y = __dsub_rn(sm.tot[8 + q], __dmul_rn(n.tbar, sm.tot[11 + q]));
                out[1 + q] = n.degenerate ? 0.0 : -__dsub_rn(__dmul_rn(n.a, x), __dmul_rn(n.b, y));
            }
        }
    } else {
        // field energy at U_0 of slot 0 (the caller's field is staged there by the host)
        const FieldLvl F = field_level(p, 0, 0);
        eval_field_energy<S>(L, F, 0, 0.f, 0, L.H, sm, buf, cl);
        FieldCtl k;
        if (tid == 0) {
            memset(&k, 0, sizeof(k));
            k.P = (double)L.W * L.H;
            k.sr = sm.tot[3]; k.srr = sm.tot[4];
            out[0] = field_energy(k, p.cfg, sm.tot, false);
            field_params(k, p.cfg, 0.f, sm.pm);
        }
        __syncthreads();
        if (grad_field) {
            float pm[6];
            for (int q = 0; q < 6; ++q) pm[q] = sm.pm[q];
            eval_field_grad<S>(L, F, 0, pm, 0, L.H, sm, buf, cl);
            // D_1 holds d = -P dE/du; report dE/du
            const size_t P = (size_t)L.W * L.H;
            const float s = -1.f / (float)P;
            for (size_t i = tid; i < P; i += kThreads) {
                grad_field[i] = s * __ldcg(F.D(1, 0) + i);
                grad_field[P + i] = s * __ldcg(F.D(1, 1) + i);
            }
        }
    }
    (void)field;
}

// ================================================================== pyramid
// All kernels take a batch of frames (grid.z or grid.x = frame).
template <typename S>
__global__ void pyr_level0(const float *frames, size_t fstride, int W, int H, int pitch, S *out, size_t ostride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    const size_t f = blockIdx.z;
    if (c < W && r < H) out[f * ostride + (size_t)r * W + c] = toS<S>(__ldg(frames + f * fstride + (size_t)r * pitch + c));
}

// Level l+1 from level l: 2x2 box average, last odd row/column clamped.
template <typename S>
__global__ void pyr_down(const S *src, size_t sstride, int W, int H, S *dst, size_t dstride)
{
    const int w2 = (W + 1) / 2, h2 = (H + 1) / 2;
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= w2 || r >= h2) return;
    src += blockIdx.z * sstride;
    dst += blockIdx.z * dstride;
    int r0 = 2 * r, r1 = min(2 * r + 1, H - 1), c0 = 2 * c, c1 = min(2 * c + 1, W - 1);
    float v = ((ldS<S>(src + (size_t)r0 * W + c0) + ldS<S>(src + (size_t)r0 * W + c1)) +
               ldS<S>(src + (size_t)r1 * W + c0)) + ldS<S>(src + (size_t)r1 * W + c1);
    dst[(size_t)r * w2 + c] = toS<S>(0.25f * v);
}

// Mean of one level of each frame (one CTA per frame), deterministic float-float sum.
template <typename S>
__global__ void __launch_bounds__(kThreads) level_mean(const S *img, size_t stride, int n, float *mean, int mstride)
{
    __shared__ float2 ws[kWarps];
    img += blockIdx.x * stride;
    float hi = 0.f, lo = 0.f;
    for (int base = 0; base < n; base += kThreads * kChunk) {
        float a = 0.f;
        const int e = min(n, base + kThreads * kChunk);
        for (int i = base + threadIdx.x; i < e; i += kThreads) a += ldS<S>(img + i);
        ff_acc(hi, lo, a);
    }
    for (int off = 16; off > 0; off >>= 1) {
        float h2 = __shfl_xor_sync(0xffffffffu, hi, off), l2 = __shfl_xor_sync(0xffffffffu, lo, off);
        ff_add(hi, lo, h2, l2);
    }
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = make_float2(hi, lo);
    __syncthreads();
    if (threadIdx.x == 0) {
        float h = 0.f, l = 0.f;
        for (int k = 0; k < kWarps; ++k) ff_add(h, l, ws[k].x, ws[k].y);
        mean[(size_t)blockIdx.x * mstride] = (float)(((double)h + (double)l) / (double)n);
    }
}

// Nonrigid composition of two fields (standalone entry point).
__global__ void compose_kernel(const float *u1, const float *u2, int W, int H, float *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= W || r >= H) return;
    const size_t P = (size_t)W * H, i = (size_t)r * W + c;
    float ax = u1[i], ay = u1[P + i];
    out[i] = ax + sample_cg(u2, W, H, c, r, ax, ay);
    out[P + i] = ay + sample_cg(u2 + P, W, H, c, r, ax, ay);
}

// ================================================================== host launchers
template <typename S>
static cudaError_t pyramid_t(const float *frames, int N, size_t fstride, int W, int H, int pitch, int levels,
                             void *const *level_base, const size_t *level_stride, float *means, cudaStream_t s)
{
    pyr_level0<S><<<dim3((W + 127) / 128, H, N), 128, 0, s>>>(frames, fstride, W, H, pitch,
                                                              (S *)level_base[0], level_stride[0]);
    int w = W, h = H;
    for (int l = 0; l + 1 < levels; ++l) {
        int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
        pyr_down<S><<<dim3((w2 + 127) / 128, h2, N), 128, 0, s>>>((const S *)level_base[l], level_stride[l], w, h,
                                                                  (S *)level_base[l + 1], level_stride[l + 1]);
        w = w2; h = h2;
    }
    if (means) {
        w = W; h = H;
        for (int l = 0; l < levels; ++l) {
            level_mean<S><<<N, kThreads, 0, s>>>((const S *)level_base[l], level_stride[l], w * h, means + l, levels);
            w = (w + 1) / 2; h = (h + 1) / 2;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_pyramid(const float *frames, int N, size_t fstride, int W, int H, int pitch, int levels,
                           int storage, void *const *level_base, const size_t *level_stride, float *means,
                           cudaStream_t s)
{
    switch (storage) {
    case REG_F32: return pyramid_t<float>(frames, N, fstride, W, H, pitch, levels, level_base, level_stride, means, s);
    case REG_BF16:
        return pyramid_t<__nv_bfloat16>(frames, N, fstride, W, H, pitch, levels, level_base, level_stride, means, s);
    case REG_F16: return pyramid_t<__half>(frames, N, fstride, W, H, pitch, levels, level_base, level_stride, means, s);
    }
    return cudaErrorInvalidValue;
}

template <typename K>
static cudaError_t launch_cluster(K kernel, int blocks, int cluster, cudaStream_t s, const Params &p)
{
    if (cluster > 8) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(blocks);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = 0;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, kernel, p);
}

cudaError_t launch_ops(const Params &p, int storage, int cluster, int n_launch_ops, cudaStream_t s)
{
    const int blocks = n_launch_ops * cluster;
    if (p.cfg.mode == REG_RIGID) {
        switch (storage) {
        case REG_F32: return launch_cluster(op_kernel<REG_RIGID, float>, blocks, cluster, s, p);
        case REG_BF16: return launch_cluster(op_kernel<REG_RIGID, __nv_bfloat16>, blocks, cluster, s, p);
        case REG_F16: return launch_cluster(op_kernel<REG_RIGID, __half>, blocks, cluster, s, p);
        }
    } else {
        switch (storage) {
        case REG_F32: return launch_cluster(op_kernel<REG_NONRIGID, float>, blocks, cluster, s, p);
        case REG_BF16: return launch_cluster(op_kernel<REG_NONRIGID, __nv_bfloat16>, blocks, cluster, s, p);
        case REG_F16: return launch_cluster(op_kernel<REG_NONRIGID, __half>, blocks, cluster, s, p);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_persistent(const Params &p, int storage, int cluster, int workers, cudaStream_t s)
{
    const int blocks = workers * cluster;
    if (p.cfg.mode == REG_RIGID) {
        switch (storage) {
        case REG_F32: return launch_cluster(persistent_kernel<REG_RIGID, float>, blocks, cluster, s, p);
        case REG_BF16: return launch_cluster(persistent_kernel<REG_RIGID, __nv_bfloat16>, blocks, cluster, s, p);
        case REG_F16: return launch_cluster(persistent_kernel<REG_RIGID, __half>, blocks, cluster, s, p);
        }
    } else {
        switch (storage) {
        case REG_F32: return launch_cluster(persistent_kernel<REG_NONRIGID, float>, blocks, cluster, s, p);
        case REG_BF16: return launch_cluster(persistent_kernel<REG_NONRIGID, __nv_bfloat16>, blocks, cluster, s, p);
        case REG_F16: return launch_cluster(persistent_kernel<REG_NONRIGID, __half>, blocks, cluster, s, p);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_energy(const Params &p, int storage, const double *theta_dev, const float *field,
                          double *out_dev, float *grad_field, cudaStream_t s)
{
    (void)storage;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(1);
    lc.blockDim = dim3(kThreads);
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (p.cfg.mode == REG_RIGID)
        return cudaLaunchKernelEx(&lc, energy_kernel<REG_RIGID, float>, p, theta_dev, field, out_dev, grad_field);
    return cudaLaunchKernelEx(&lc, energy_kernel<REG_NONRIGID, float>, p, theta_dev, field, out_dev, grad_field);
}

cudaError_t launch_compose(const float *u1, const float *u2, int W, int H, float *out, cudaStream_t s)
{
    compose_kernel<<<dim3((W + 127) / 128, H), 128, 0, s>>>(u1, u2, W, H, out);
    return cudaGetLastError();
}

size_t scratch_floats_per_slot(const int *W, const int *H, int levels)
{
    size_t n = 0;
    for (int l = 0; l < levels; ++l) n += (size_t)8 * W[l] * H[l];
    return n;
}

int max_cluster_size() { return 16; }

}  // namespace reg
