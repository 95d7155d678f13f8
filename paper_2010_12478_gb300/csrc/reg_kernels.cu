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
#include "reg_f2.cuh"

namespace cg = cooperative_groups;

namespace reg {

constexpr int kWarps = kThreads / 32;
constexpr int kNM = 8;         // moment slots per reduction (at most 6 are used)
constexpr int kMaxCluster = 16; // CTAs per operator at most (non-portable cluster size)
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

// acc += x*y with the exact rounding error of the product kept in err (the error of a
// product of two floats is exactly representable: fmaf(x, y, -p)).
__device__ __forceinline__ void acc_prod(float &acc, float &err, float x, float y)
{
    const float p = __fmul_rn(x, y);
    err += fmaf(x, y, -p);
    acc = __fadd_rn(acc, p);
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
// Step-controller state (FP64), used by thread 0 of each CTA only: kept in shared memory so
// it does not occupy registers of every thread.
struct RigidCtl {
    double th[3], tt[3], d[3], dp[3];   // dp: the direction of the last accepted step
    double E, tau, slope, sr, srr, m0, P, cx, cy, invP, inv_m0;
    double tau_acc;                // length of the last accepted step (along dp)
    double a, b, rbar, tbar;       // NCC terms at th
    double ta, tb, trbar, ttbar;   // at the trial point tt
    int nrej, iters, evals, stop, rejects, have_prev;
    double tolg;   // the level's stop tolerance (tol_grad, times tol_coarse above the finest level)
};

struct FieldCtl {
    double E, tau, tau_pend, tau_acc, slope, P, Nc, sr, srr, invP, invNc;
    double a, b, rbar, tbar;      // NCC terms at the current field
    double ta, tb, trbar, ttbar;  // at the trial field
    int degen, tdegen;
    int nrej, iters, evals, stop, rejects, have_prev;
    double tolg;   // the level's stop tolerance (tol_grad, times tol_coarse above the finest level)
};

// First trial of a line search after an accepted step (Barzilai and Borwein, "Two-point step size
// gradient methods", 1988, their second step): tau = tau_acc <d_prev, d_prev - d> / |d_prev - d|^2
// in the flow's metric, given num = <d_prev, d_prev - d> and den = |d_prev - d|^2; without positive
// curvature the quadratic rule's tau_q stays.  The ratio needs no more than FP32 relative precision.
__device__ __forceinline__ double bb_tau(double tau_q, double tau_acc, double num, double den)
{
    if (!(num > 0.0 && den > 0.0)) return tau_q;
    return tau_acc * num * (double)__frcp_rn((float)den);
}

struct Smem {
    float2 warp[kWarps][kNM];   // per-warp (hi, lo) partials
    double part[2][kMaxCluster][kNM];   // every CTA's partials, pushed here by each CTA
    double tot[kNM];            // cluster totals
    float pm[16];               // pass parameters broadcast by thread 0
    int action;
    int idata[4];
    union {
        RigidCtl rctl;
        FieldCtl fctl;
    };
};

// Reduce NM per-thread float-float partials over the cluster into sm.tot.
// If MAXLAST, slot NM-1 holds a non-negative value combined by max (hi only).
template <int NM, bool MAXLAST>
__device__ __forceinline__ void cluster_reduce(float (&hi)[NM], float (&lo)[NM], Smem &sm,
                                               int &buf, const cg::cluster_group &cl, bool fence)
{
    static_assert(NM <= kNM, "reduction slots");
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
    const unsigned C = cl.num_blocks(), me = cl.block_rank();
    if (tid < NM) {
        float h = 0.f, l = 0.f;
        for (int k = 0; k < kWarps; ++k) {
            float2 v = sm.warp[k][tid];
            if (MAXLAST && tid == NM - 1) h = fmaxf(h, v.x);
            else ff_add(h, l, v.x, v.y);
        }
        // push this CTA's partial into slot `me` of every CTA of the cluster (remote stores do
        // not wait; the cluster barrier below makes them visible)
        const double v = (double)h + (double)l;
        for (unsigned r = 0; r < C; ++r) *cl.map_shared_rank(&sm.part[buf][me][tid], r) = v;
    }
    if (fence) __threadfence();
    cl.sync();
    if (tid < NM) {
        // every CTA adds the same values in rank order: identical totals everywhere
        double s = 0.0;
        for (unsigned r = 0; r < C; ++r) {
            const double v = sm.part[buf][r][tid];
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
// 1/sqrt(q) for a positive normal q without a double-precision divide or square root (both
// are long dependent instruction sequences on this GPU's narrow FP64 unit): the hardware
// reciprocal-square-root approximation, then two Newton-Raphson steps y <- y (3 - q y^2) / 2,
// each squaring the relative error (about 1e-7 -> 1e-14 -> double rounding).
__device__ __forceinline__ double rsqrt_nr(double q)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(q));
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double t = __dmul_rn(q, __dmul_rn(y, y));
        y = __dmul_rn(y, __fma_rn(-0.5, t, 1.5));
    }
    return y;
}

// NCC and its gradient coefficients from the shifted sums (invP = 1/P, formed once per level).
// Explicit round-to-nearest operations keep the result independent of FMA contraction; when
// S'_rt == S'_rr == S'_tt (T o phi equals R up to the shift: identical inputs) the result is
// exactly NCC = 1 with a == b, so the gradient vanishes exactly.
__device__ Ncc ncc_terms(double P, double invP, double sr, double st, double srr, double stt, double srt)
{
    Ncc o;
    const double Srr = __dsub_rn(srr, __dmul_rn(__dmul_rn(sr, sr), invP));
    const double Stt = __dsub_rn(stt, __dmul_rn(__dmul_rn(st, st), invP));
    const double Srt = __dsub_rn(srt, __dmul_rn(__dmul_rn(sr, st), invP));
    o.rbar = __dmul_rn(sr, invP);
    o.tbar = __dmul_rn(st, invP);
    if (Srr < 1e-12 * P || Stt < 1e-12 * P) {
        o.ncc = 0.0; o.a = 0.0; o.b = 0.0; o.degenerate = 1;
        return o;
    }
    const double a = rsqrt_nr(__dmul_rn(Srr, Stt));   // 1 / sqrt(S'_rr S'_tt)
    o.a = a;
    if (Srt == Srr && Srr == Stt) {
        o.ncc = 1.0;
        o.b = a;
    } else {
        o.ncc = __dmul_rn(Srt, a);
        o.b = __dmul_rn(__dmul_rn(o.ncc, Srr), __dmul_rn(a, a));   // NCC / S'_tt
    }
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

// Row-major traversal for the fused evaluation passes: warp w walks rows r0 + w, r0 + w + kWarps,
// ...; in a row, lane l takes columns l + 32 u (u < U) per step, so each thread has U independent
// samples in flight and a warp's loads stay coalesced.  row(r) runs once per row; px(r, c) per
// pixel; flush_fast() after every kFast pixels of a thread, flush() after every kChunk (and at
// the end).  U must divide kFast.
template <int U, typename RowF, typename PixF, typename Q, typename G>
__device__ __forceinline__ void for_rows(int W, int r0, int r1, RowF &&row, PixF &&px, Q &&flush_fast, G &&flush)
{
    static_assert(kFast % U == 0, "U must divide kFast");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cnt = 0;
    for (int r = r0 + warp; r < r1; r += kWarps) {
        row(r);
        for (int c0 = lane; c0 < W; c0 += 32 * U) {
            if (c0 + 32 * (U - 1) < W) {
#pragma unroll
                for (int u = 0; u < U; ++u) px(r, c0 + 32 * u);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (c0 + 32 * u < W) px(r, c0 + 32 * u);
            }
            cnt += U;
            if ((cnt & (kFast - 1)) == 0) flush_fast();
            if ((cnt & (kChunk - 1)) == 0) flush();
        }
    }
    flush_fast();
    flush();
}

// for_rows with the pixels of a step taken in pairs: px2(r, c, c + 32) for columns 32 apart (U
// even); a row's partial last step goes pixel by pixel through px(r, c).
template <int U, typename RowF, typename Pix2F, typename PixF, typename Q, typename G>
__device__ __forceinline__ void for_rows2(int W, int r0, int r1, RowF &&row, Pix2F &&px2, PixF &&px, Q &&flush_fast,
                                          G &&flush)
{
    static_assert(kFast % U == 0 && U % 2 == 0, "U even, dividing kFast");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cnt = 0;
    for (int r = r0 + warp; r < r1; r += kWarps) {
        row(r);
        for (int c0 = lane; c0 < W; c0 += 32 * U) {
            if (c0 + 32 * (U - 1) < W) {
#pragma unroll
                for (int u = 0; u < U; u += 2) px2(r, c0 + 32 * u, c0 + 32 * u + 32);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (c0 + 32 * u < W) px(r, c0 + 32 * u);
            }
            cnt += U;
            if ((cnt & (kFast - 1)) == 0) flush_fast();
            if ((cnt & (kChunk - 1)) == 0) flush();
        }
    }
    flush_fast();
    flush();
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

// Quadratic B-spline model of the samples of T (storage S) at p = (xi + vx, yi + vy), with the
// samples beyond the border equal to the level's mean: the image model of the nonrigid energy,
// continuously differentiable everywhere.  With n the nearest sample and t = p - n in
// [-1/2, 1/2) per axis, the three taps n - 1, n, n + 1 carry the weights (1/2 - t)^2 / 2,
// 3/4 - t^2, (1/2 + t)^2 / 2 and, for the derivative, t - 1/2, -2 t, t + 1/2.  T addresses
// pixel (0, 0) of a level stored with a border of kPad >= 3 samples holding its mean (row pitch
// Tp): n clamped to [-2, W + 1] x [-2, H + 1] keeps the window inside the border, and a window
// clamped there lies wholly in the border, as the true one does: the mean-extended model for any p.
template <typename S, bool DERIV>
__device__ __forceinline__ float sample_q(const S *T, int W, int H, int Tp, int xi, int yi, float vx, float vy,
                                          float &dtx, float &dty)
{
    // nearest sample n = floor(v + 1/2), t = v - n: within rounding of [-1/2, 1/2) (at a tie either
    // window gives the same value and derivative, the model being C1).  A NaN or huge offset
    // converts to 0 or a saturated integer, the sum wraps, and the clamp keeps the window inside
    // the border whatever the offset.
    const float fnx = floorf(vx + 0.5f), fny = floorf(vy + 0.5f);
    const float tx = vx - fnx, ty = vy - fny;
    int nx = (int)((unsigned)xi + (unsigned)__float2int_rz(fnx));
    int ny = (int)((unsigned)yi + (unsigned)__float2int_rz(fny));
    nx = min(max(nx, -2), W + 1);
    ny = min(max(ny, -2), H + 1);
    const S *p0 = T + (ptrdiff_t)(ny - 1) * Tp + nx;
    const S *p1 = p0 + Tp, *p2 = p1 + Tp;
    // weights (1/2 - t)^2 / 2, 3/4 - t^2, (1/2 + t)^2 / 2; the last is the first plus t
    const float ax = 0.5f - tx, ay = 0.5f - ty;
    const float wx0 = (0.5f * ax) * ax, wx1 = fmaf(-tx, tx, 0.75f), wx2 = wx0 + tx;
    const float wy0 = (0.5f * ay) * ay, wy1 = fmaf(-ty, ty, 0.75f), wy2 = wy0 + ty;
    const float t00 = ldS<S>(p0 - 1), t01 = ldS<S>(p0), t02 = ldS<S>(p0 + 1);
    const float t10 = ldS<S>(p1 - 1), t11 = ldS<S>(p1), t12 = ldS<S>(p1 + 1);
    const float t20 = ldS<S>(p2 - 1), t21 = ldS<S>(p2), t22 = ldS<S>(p2 + 1);
    const float a0 = fmaf(wx2, t02, fmaf(wx1, t01, wx0 * t00));
    const float a1 = fmaf(wx2, t12, fmaf(wx1, t11, wx0 * t10));
    const float a2 = fmaf(wx2, t22, fmaf(wx1, t21, wx0 * t20));
    if (DERIV) {
        // derivative weights t - 1/2, -2 t, t + 1/2
        const float m2x = -2.f * tx, bx = 0.5f + tx;
        const float b0 = fmaf(bx, t02, fmaf(m2x, t01, -ax * t00));
        const float b1 = fmaf(bx, t12, fmaf(m2x, t11, -ax * t10));
        const float b2 = fmaf(bx, t22, fmaf(m2x, t21, -ax * t20));
        dtx = fmaf(wy2, b2, fmaf(wy1, b1, wy0 * b0));
        dty = fmaf(0.5f + ty, a2, fmaf(-2.f * ty, a1, -ay * a0));
    }
    return fmaf(wy2, a2, fmaf(wy1, a1, wy0 * a0));
}

// Two samples of the model at once, pixel a in the .x and pixel b in the .y of every float2: the
// steps of sample_q with each floating-point operation done on both in one packed FP32x2
// instruction (each lane rounded as the scalar operation, so the values equal two sample_q calls).
template <typename S, bool DERIV>
__device__ __forceinline__ float2 sample_q2(const S *T, int W, int H, int Tp, int2 xi, int2 yi, float2 vx, float2 vy,
                                            float2 &dtx, float2 &dty)
{
    const float2 h = make_float2(0.5f, 0.5f);
    const float2 px = __fadd2_rn(vx, h), py = __fadd2_rn(vy, h);
    const float2 fnx = make_float2(floorf(px.x), floorf(px.y)), fny = make_float2(floorf(py.x), floorf(py.y));
    const float2 tx = __fadd2_rn(vx, make_float2(-fnx.x, -fnx.y)), ty = __fadd2_rn(vy, make_float2(-fny.x, -fny.y));
    const int nxa = min(max((int)((unsigned)xi.x + (unsigned)__float2int_rz(fnx.x)), -2), W + 1);
    const int nxb = min(max((int)((unsigned)xi.y + (unsigned)__float2int_rz(fnx.y)), -2), W + 1);
    const int nya = min(max((int)((unsigned)yi.x + (unsigned)__float2int_rz(fny.x)), -2), H + 1);
    const int nyb = min(max((int)((unsigned)yi.y + (unsigned)__float2int_rz(fny.y)), -2), H + 1);
    const S *pa = T + (ptrdiff_t)(nya - 1) * Tp + nxa, *pb = T + (ptrdiff_t)(nyb - 1) * Tp + nxb;
    const float2 ax = __fadd2_rn(h, make_float2(-tx.x, -tx.y)), ay = __fadd2_rn(h, make_float2(-ty.x, -ty.y));
    const float2 wx0 = __fmul2_rn(__fmul2_rn(h, ax), ax), wy0 = __fmul2_rn(__fmul2_rn(h, ay), ay);
    const float2 q34 = make_float2(0.75f, 0.75f);
    const float2 wx1 = __ffma2_rn(make_float2(-tx.x, -tx.y), tx, q34), wy1 = __ffma2_rn(make_float2(-ty.x, -ty.y), ty, q34);
    const float2 wx2 = __fadd2_rn(wx0, tx), wy2 = __fadd2_rn(wy0, ty);
    float2 tr[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) tr[r][k] = make_float2(ldS<S>(pa + r * Tp + k - 1), ldS<S>(pb + r * Tp + k - 1));
    float2 a[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) a[r] = __ffma2_rn(wx2, tr[r][2], __ffma2_rn(wx1, tr[r][1], __fmul2_rn(wx0, tr[r][0])));
    if (DERIV) {
        // derivative weights t - 1/2, -2 t, t + 1/2
        const float2 m2 = make_float2(-2.f, -2.f);
        const float2 nax = make_float2(-ax.x, -ax.y), bx = __fadd2_rn(h, tx);
        float2 b[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            b[r] = __ffma2_rn(bx, tr[r][2], __ffma2_rn(__fmul2_rn(m2, tx), tr[r][1], __fmul2_rn(nax, tr[r][0])));
        dtx = __ffma2_rn(wy2, b[2], __ffma2_rn(wy1, b[1], __fmul2_rn(wy0, b[0])));
        dty = __ffma2_rn(__fadd2_rn(h, ty), a[2], __ffma2_rn(__fmul2_rn(m2, ty), a[1],
                                                                 __fmul2_rn(make_float2(-ay.x, -ay.y), a[0])));
    }
    return __ffma2_rn(wy2, a[2], __ffma2_rn(wy1, a[1], __fmul2_rn(wy0, a[0])));
}

// ================================================================== rigid
// Energy pass moment slots: 0 St, 1 Stt, 2 Srt (t = T(phi(x)) - cR, r = R(x) - cR), and with
// RSTAT (first pass of a level) 3 Sr, 4 Srr.
template <typename S, bool RSTAT>
__device__ void eval_rigid_energy(const Lvl &L, int r0, int r1, const float *pm, Smem &sm, int &buf,
                                  const cg::cluster_group &cl)
{
    constexpr int NM = RSTAT ? 5 : 3;
    // pm: cos(alpha) - 1, sin(alpha), fractional translation (x, y), integer translation (x, y)
    const float cm1 = pm[0], sa = pm[1], gfx = pm[2], gfy = pm[3];
    const int gix = (int)pm[4], giy = (int)pm[5];
    const float cx = 0.5f * (float)(L.W - 1), cy = 0.5f * (float)(L.H - 1);
    const S *R = (const S *)L.R, *T = (const S *)L.T;
    float hi[NM], lo[NM], a[NM];
    float e1 = 0.f, e2 = 0.f, e4 = 0.f;   // exact product rounding errors of slots 1, 2, 4
#pragma unroll
    for (int m = 0; m < NM; ++m) { hi[m] = 0.f; lo[m] = 0.f; a[m] = 0.f; }
    // per-row terms of phi(x) - x - integer translation (small, so FP32 keeps ~1e-7 relative)
    float bx = 0.f, by = 0.f;
    const S *Rrow = R;
    int yi = 0;
    for_rows<4>(
        L.W, r0, r1,
        [&](int r) {
            const float yc = (float)r - cy;
            bx = fmaf(-sa, yc, gfx);
            by = fmaf(cm1, yc, gfy);
            Rrow = R + (size_t)r * L.Rp;
            yi = r + giy;
        },
        [&](int r, int c) {
            (void)r;
            const float xc = (float)c - cx;
            float dtx, dty;
            const float tw = sample_at<S, false>(T, L.W, L.H, L.Tp, c + gix, yi, fmaf(cm1, xc, bx),
                                                 fmaf(sa, xc, by), dtx, dty);
            const float rv = ldS<S>(Rrow + c) - L.cR;
            const float tv = tw - L.cR;
            a[0] += tv;
            acc_prod(a[1], e1, tv, tv);
            acc_prod(a[2], e2, rv, tv);
            if constexpr (RSTAT) {
                a[3] += rv;
                acc_prod(a[4], e4, rv, rv);
            }
        },
        [&]() {
            // short FP32 runs plus the exact product errors keep 1 - NCC accurate to ~1e-9
#pragma unroll
            for (int m = 0; m < NM; ++m) { ff_acc(hi[m], lo[m], a[m]); a[m] = 0.f; }
            lo[1] += e1; lo[2] += e2;
            e1 = 0.f; e2 = 0.f;
            if constexpr (RSTAT) { lo[4] += e4; e4 = 0.f; }
        },
        []() {});
    cluster_reduce<NM, false>(hi, lo, sm, buf, cl, false);
}

// Gradient pass at a point whose NCC terms are known (from the energy pass or the accepted
// trial at the same point): slots k = 0..2 sum F(x) g_k(x), F = P dE/dTw =
// -(aP (r - rbar) - bP (t - tbar)), g_k = grad T(phi(x)) . dphi/dtheta_k.
// pm[6..9] = aP, bP, rbar, tbar (rbar, tbar: means of the shifted samples).
template <typename S>
__device__ void eval_rigid_grad(const Lvl &L, int r0, int r1, const float *pm, Smem &sm, int &buf,
                                const cg::cluster_group &cl)
{
    constexpr int NM = 3;
    const float cm1 = pm[0], sa = pm[1], gfx = pm[2], gfy = pm[3];
    const int gix = (int)pm[4], giy = (int)pm[5];
    const float aP = pm[6], bP = pm[7], rb = pm[8], tb = pm[9];
    const float ca = 1.f + cm1;
    const float cx = 0.5f * (float)(L.W - 1), cy = 0.5f * (float)(L.H - 1);
    const S *R = (const S *)L.R, *T = (const S *)L.T;
    float hi[NM], lo[NM], a[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) { hi[m] = 0.f; lo[m] = 0.f; a[m] = 0.f; }
    float bx = 0.f, by = 0.f, gax = 0.f, gay = 0.f;
    const S *Rrow = R;
    int yi = 0;
    for_rows<4>(
        L.W, r0, r1,
        [&](int r) {
            const float yc = (float)r - cy;
            bx = fmaf(-sa, yc, gfx);
            by = fmaf(cm1, yc, gfy);
            gax = -sa * yc;   // terms in yc of dphi/dalpha = Rot'(alpha) (x - c)
            gay = ca * yc;
            Rrow = R + (size_t)r * L.Rp;
            yi = r + giy;
        },
        [&](int r, int c) {
            (void)r;
            const float xc = (float)c - cx;
            float dtx, dty;
            const float tw = sample_at<S, true>(T, L.W, L.H, L.Tp, c + gix, yi, fmaf(cm1, xc, bx),
                                                fmaf(sa, xc, by), dtx, dty);
            const float rv = ldS<S>(Rrow + c) - L.cR;
            const float tv = tw - L.cR;
            // no contraction: identical r and t give F == 0 exactly
            const float F = -__fsub_rn(__fmul_rn(aP, rv - rb), __fmul_rn(bP, tv - tb));
            const float g0 = fmaf(dty, fmaf(ca, xc, gax), -dtx * fmaf(sa, xc, gay));
            a[0] = fmaf(F, g0, a[0]);
            a[1] = fmaf(F, dtx, a[1]);
            a[2] = fmaf(F, dty, a[2]);
        },
        []() {},
        [&]() {
#pragma unroll
            for (int m = 0; m < NM; ++m) { ff_acc(hi[m], lo[m], a[m]); a[m] = 0.f; }
        });
    cluster_reduce<NM, false>(hi, lo, sm, buf, cl, false);
}

enum Action { kActGrad = 0, kActTrial = 1, kActDone = 2, kActEnergy = 3, kActField = 4, kActMetric = 5 };


__device__ void rigid_params(const double *th, float *pm)
{
    const float a = (float)th[0];
    float h, ch;
    sincosf(0.5f * a, &h, &ch);
    pm[0] = -2.f * h * h;            // cos(a) - 1 without cancellation
    pm[1] = 2.f * h * ch;            // sin(a)
    const double ix = rint(th[1]), iy = rint(th[2]);
    pm[2] = (float)(th[1] - ix);
    pm[3] = (float)(th[2] - iy);
    pm[4] = (float)fmax(-4.0e6, fmin(4.0e6, ix));
    pm[5] = (float)fmax(-4.0e6, fmin(4.0e6, iy));
}

__device__ void rigid_grad_params(const RigidCtl &k, float *pm)
{
    rigid_params(k.th, pm);
    pm[6] = (float)(k.a * k.P);
    pm[7] = (float)(k.b * k.P);
    pm[8] = (float)k.rbar;
    pm[9] = (float)k.tbar;
}

// Step-size rule of the line search: Armijo backtracking with safeguarded quadratic
// interpolation (Nocedal and Wright, Numerical Optimization, Sec. 3.5).  tq minimises the
// parabola through E(0) = E, E'(0) = slope and E(tau) = Et; a rejected trial retries at tq
// clamped to [0.1 tau, 0.5 tau], an accepted one starts the next search at tq clamped to
// [0.5 tau, 4 tau]; without positive curvature the rule halves / doubles.
__device__ __forceinline__ double next_tau(double E, double slope, double tau, double Et, bool accepted)
{
    const double den = Et - E - slope * tau;
    if (!(den > 0.0)) return accepted ? 2.0 * tau : 0.5 * tau;
    // a step-size estimate needs no more than FP32 relative precision once den is formed
    const double tq = (-slope * tau * tau) * (double)__frcp_rn((float)(2.0 * den));
    return accepted ? fmin(fmax(tq, 0.5 * tau), 4.0 * tau) : fmin(fmax(tq, 0.1 * tau), 0.5 * tau);
}

// Thread-0 controller after an ENERGY (level start), GRAD or TRIAL pass.  Returns the next
// action and writes its parameters.  Same rules as the oracle's level loop.
__device__ int rigid_step(RigidCtl &k, const Config &cfg, const double *tot, int action, float *pm)
{
    if (action == kActEnergy) {
        k.sr = tot[3];
        k.srr = tot[4];
        const Ncc n = ncc_terms(k.P, k.invP, k.sr, tot[0], k.srr, tot[1], tot[2]);
        k.E = n.degenerate ? 1.0 : __dsub_rn(1.0, n.ncc);
        k.a = n.a; k.b = n.b; k.rbar = n.rbar; k.tbar = n.tbar;
        rigid_grad_params(k, pm);
        return kActGrad;
    }
    if (action == kActGrad) {
        double g[3];
        for (int q = 0; q < 3; ++q) g[q] = tot[q] * k.invP;
        k.evals += 1;
        if (k.iters >= cfg.max_iter) { k.stop = REG_STOP_MAXIT; return kActDone; }
        k.d[0] = -g[0] * k.inv_m0; k.d[1] = -g[1]; k.d[2] = -g[2];
        k.slope = g[0] * k.d[0] + g[1] * k.d[1] + g[2] * k.d[2];
        // |g|_M = sqrt(-slope); the tests compare squares (no square root unless the cap applies)
        const double gn2 = -k.slope;
        if (!(gn2 >= k.tolg * k.tolg)) { k.stop = REG_STOP_GRAD; return kActDone; }
        if (k.have_prev) {
            double num = 0.0, den = 0.0;
            for (int q = 0; q < 3; ++q) {
                const double w = q == 0 ? k.m0 : 1.0, y = k.dp[q] - k.d[q];
                num += w * k.dp[q] * y;
                den += w * y * y;
            }
            k.tau = bb_tau(k.tau, k.tau_acc, num, den);
        }
        if (k.tau * k.tau * gn2 > cfg.step_cap * cfg.step_cap) k.tau = cfg.step_cap / sqrt(gn2);
        k.nrej = 0;
        for (int q = 0; q < 3; ++q) k.tt[q] = k.th[q] + k.tau * k.d[q];
        rigid_params(k.tt, pm);
        return kActTrial;
    }
    // trial
    const Ncc n = ncc_terms(k.P, k.invP, k.sr, tot[0], k.srr, tot[1], tot[2]);
    const double Et = n.degenerate ? 1.0 : __dsub_rn(1.0, n.ncc);
    k.evals += 1;
    if (Et <= k.E + cfg.armijo_c * k.tau * k.slope) {
        for (int q = 0; q < 3; ++q) { k.th[q] = k.tt[q]; k.dp[q] = k.d[q]; }
        k.tau_acc = k.tau;
        k.have_prev = 1;
        k.iters += 1;
        const double Eold = k.E;
        k.tau = next_tau(k.E, k.slope, k.tau, Et, true);
        k.E = Et;
        k.a = n.a; k.b = n.b; k.rbar = n.rbar; k.tbar = n.tbar;
        if (Eold - Et <= cfg.tol_rel_e * fabs(Eold)) { k.stop = REG_STOP_REL; return kActDone; }
        rigid_grad_params(k, pm);
        return kActGrad;
    }
    k.rejects += 1;
    k.nrej += 1;
    k.tau = next_tau(k.E, k.slope, k.tau, Et, false);
    if (k.nrej > cfg.max_rejects) { k.stop = REG_STOP_LS; return kActDone; }
    for (int q = 0; q < 3; ++q) k.tt[q] = k.th[q] + k.tau * k.d[q];
    rigid_params(k.tt, pm);
    return kActTrial;
}

__device__ __forceinline__ Lvl level_of(const Params &p, int ref, int tmpl, int l)
{
    const LevelDesc &a = p.levels[ref * p.cfg.levels + l];
    const LevelDesc &b = p.levels[tmpl * p.cfg.levels + l];
    Lvl L;
    L.R = a.rptr; L.T = b.ptr; L.W = a.W; L.H = a.H; L.Rp = a.rpitch; L.Tp = b.pitch; L.cR = a.mean;
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
    RigidCtl &k = sm.rctl;
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
            k.invP = 1.0 / k.P;
            k.cx = 0.5 * (L.W - 1);
            k.cy = 0.5 * (L.H - 1);
            double rho = 0.25 * (L.W + L.H);
            k.m0 = rho * rho;
            k.inv_m0 = 1.0 / k.m0;
            k.tau = cfg.tau0;
            k.have_prev = 0;
            k.iters = 0; k.evals = 0; k.stop = REG_STOP_MAXIT;
            // a coarse level only supplies the next level's initial guess: a looser stop
            k.tolg = cfg.tol_grad * (l > 0 ? cfg.tol_coarse : 1.0);
            rigid_params(k.th, sm.pm);
            sm.action = kActEnergy;
        }
        for (;;) {
            __syncthreads();
            const int act = sm.action;
            if (act == kActDone) break;
            float pm[10];
#pragma unroll
            for (int q = 0; q < 10; ++q) pm[q] = sm.pm[q];
            if (act == kActEnergy) eval_rigid_energy<S, true>(L, r0, r1, pm, sm, buf, cl);
            else if (act == kActGrad) eval_rigid_grad<S>(L, r0, r1, pm, sm, buf, cl);
            else eval_rigid_energy<S, false>(L, r0, r1, pm, sm, buf, cl);
            if (tid == 0) sm.action = rigid_step(k, cfg, sm.tot, act, sm.pm);
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
// Free-form field: u(x) bilinear in control values c_j on a grid of spacing s
// (finest-level pixels), points (jx s, jy s).  At level l a pixel x sits at
// finest coordinate X = 2^l x + (2^l - 1)/2, and the level works on c in its
// own pixels (c / 2^l).  Every CTA of the cluster holds the whole grid in
// shared memory: c (current), d (descent direction), mt (scalar product) and gp
// (this CTA's partial gradient); a trial's values c + tau d are formed where read.

struct Grid {
    int nx, ny, s;   // points per axis, spacing in finest pixels
};

struct GridLvl {
    int W, H, l;     // level size and index
    float scale_inv; // 1 / s in level-coordinate units: g = (2^l x + off) / s
    float off;       // (2^l - 1) / 2
    float pl;        // 2^l
};

// Cell and weights of level pixel (x, y); matches the clamped cell choice of the oracle.
__device__ __forceinline__ void grid_cell(const Grid &G, const GridLvl &L, int x, int y, int &ix, int &iy,
                                          float &wx, float &wy)
{
    float gx = fmaf(L.pl, (float)x, L.off) * L.scale_inv;
    float gy = fmaf(L.pl, (float)y, L.off) * L.scale_inv;
    gx = fminf(gx, (float)(G.nx - 1));
    gy = fminf(gy, (float)(G.ny - 1));
    ix = min((int)gx, G.nx - 2);
    iy = min((int)gy, G.ny - 2);
    wx = gx - (float)ix;
    wy = gy - (float)iy;
}

__device__ __forceinline__ float2 grid_eval(const float2 *c, int nx, int ix, int iy, float wx, float wy)
{
    const float2 a = c[iy * nx + ix], b = c[iy * nx + ix + 1], e = c[(iy + 1) * nx + ix], f = c[(iy + 1) * nx + ix + 1];
    const float gx = 1.f - wx, gy = 1.f - wy;
    float2 u;
    u.x = fmaf(wy, fmaf(wx, f.x, gx * e.x), gy * fmaf(wx, b.x, gx * a.x));
    u.y = fmaf(wy, fmaf(wx, f.y, gx * e.y), gy * fmaf(wx, b.y, gx * a.y));
    return u;
}

// Rows and band of control-cell rows owned by a CTA: cell rows [k q, (k+1) q), q = ceil((ny-1)/C);
// level pixel rows of those cells (the last CTA also takes rows clamped into the last cell row).
// Partial-gradient buffer of one CTA: the control rows of its band of cell rows, [cr0, cr1].
__host__ __device__ __forceinline__ int grid_band_elems(int gnx, int gny, int C)
{
    return ((gny - 1 + C - 1) / C + 1) * gnx;
}

// Dynamic shared memory of the nonrigid kernels, in float2 units: c, d, mt (whole grid each; mt the
// flow's scalar product per control point and axis, or with the H1 product its right-hand side),
// with the H1 product two more whole-grid buffers t and u for its solve, the band of partial
// gradients, then (16-byte aligned) one row of gnx - 1 float4 per warp: the control values of the
// warp's pixel row interpolated along y, (u_j, u_{j+1} - u_j).
struct GridLayout {
    int c, d, mt, t, u, gp, crow;
};
__host__ __device__ __forceinline__ GridLayout grid_layout(int gnx, int gny, int C, bool h1)
{
    const int Nc = gnx * gny;
    GridLayout g;
    g.c = 0;
    g.d = Nc;
    g.mt = 2 * Nc;
    int o = 3 * Nc;
    g.t = h1 ? o : -1;
    g.u = h1 ? o + Nc : -1;
    if (h1) o += 2 * Nc;
    g.gp = o;
    o += grid_band_elems(gnx, gny, C);
    g.crow = o + (o & 1);
    return g;
}

__device__ __forceinline__ void grid_rows(const Grid &G, const GridLvl &L, int rank, int C, int &cr0, int &cr1,
                                          int &r0, int &r1)
{
    const int cells = G.ny - 1;
    const int q = (cells + C - 1) / C;
    cr0 = min(cells, rank * q);
    cr1 = min(cells, cr0 + q);
    const int sl = G.s >> L.l;   // cell height in level pixels
    r0 = min(L.H, cr0 * sl);
    r1 = (cr1 == cells) ? L.H : min(L.H, cr1 * sl);
    if (cr0 == cr1) r0 = r1 = L.H;
}

// Energy moments of the field ct = c + tau d (TRIAL; else ct = c): slots 0 St, 1 Stt, 2 Srt, with
// RSTAT (first pass of a level) 3 Sr, 4 Srr; slot 5 = sum over control edges |dct|^2 (rank 0 only,
// so the cluster sum counts it once).  Each warp first interpolates the control values of its row
// along y into crow (u_j and u_{j+1} - u_j for the nx - 1 cells), so a pixel only interpolates
// along x.  The trial values are formed where they are read, fmaf(tau, d_j, c_j), the expression
// an accepted step stores into c.
template <typename S, bool RSTAT, int U, bool TRIAL>
__device__ void grid_energy_pass(const Lvl &L, const Grid &G, const GridLvl &GL, const float2 *c, const float2 *d,
                                 float tau, float4 *crow_all, int r0, int r1, Smem &sm, int &buf,
                                 const cg::cluster_group &cl)
{
    auto ct = [&](int j) {
        const float2 a = c[j];
        if constexpr (TRIAL) {
            const float2 b = d[j];
            return make_float2(fmaf(tau, b.x, a.x), fmaf(tau, b.y, a.y));
        } else {
            return a;
        }
    };
    const S *R = (const S *)L.R, *T = (const S *)L.T;
    constexpr int NM = 6;
    float hi[NM], lo[NM];
    // per-lane partial sums of the current kFast pixels, in pairs (.x and .y: the two pixels of a
    // packed step); e: the exact rounding errors of the products of slots 1, 2 and 4
    float2 a[5], e1 = make_float2(0.f, 0.f), e2 = e1, e4 = e1;
#pragma unroll
    for (int m = 0; m < NM; ++m) { hi[m] = 0.f; lo[m] = 0.f; }
#pragma unroll
    for (int m = 0; m < 5; ++m) a[m] = make_float2(0.f, 0.f);
    const int lane = threadIdx.x & 31;
    float4 *crow = crow_all + (threadIdx.x >> 5) * (G.nx - 1);
    const S *Rrow = R;
    auto row = [&](int r) {
        Rrow = R + (size_t)r * L.Rp;
        const float gyf = fminf(fmaf(GL.pl, (float)r, GL.off) * GL.scale_inv, (float)(G.ny - 1));
        const int iy = min((int)gyf, G.ny - 2);
        const float wy = gyf - (float)iy, hy = 1.f - wy;
        __syncwarp();
        for (int j = lane; j < G.nx - 1; j += 32) {
            const float2 a0 = ct(iy * G.nx + j), a1 = ct((iy + 1) * G.nx + j);
            const float2 b0 = ct(iy * G.nx + j + 1), b1 = ct((iy + 1) * G.nx + j + 1);
            const float ux0 = fmaf(wy, a1.x, hy * a0.x), uy0 = fmaf(wy, a1.y, hy * a0.y);
            const float ux1 = fmaf(wy, b1.x, hy * b0.x), uy1 = fmaf(wy, b1.y, hy * b0.y);
            crow[j] = make_float4(ux0, uy0, ux1 - ux0, uy1 - uy0);
        }
        __syncwarp();
    };
    const float2 ncr = make_float2(-L.cR, -L.cR);
    // two pixels (r, ca) and (r, cb) with displacements (ux.x, uy.x) and (ux.y, uy.y)
    auto pixel2 = [&](int r, int ca, int cb, float2 ux, float2 uy) {
        float2 dtx, dty;
        const float2 tw = sample_q2<S, false>(T, L.W, L.H, L.Tp, make_int2(ca, cb), make_int2(r, r), ux, uy, dtx, dty);
        const float2 rv = __fadd2_rn(make_float2(ldS<S>(Rrow + ca), ldS<S>(Rrow + cb)), ncr);
        const float2 tv = __fadd2_rn(tw, ncr);
        a[0] = __fadd2_rn(a[0], tv);
        acc_prod2(a[1], e1, tv, tv);
        acc_prod2(a[2], e2, rv, tv);
        if constexpr (RSTAT) {
            a[3] = __fadd2_rn(a[3], rv);
            acc_prod2(a[4], e4, rv, rv);
        }
    };
    // one pixel (a row's ragged end), into the .x partial sums
    auto pixel = [&](int r, int c, float ux, float uy) {
        float dtx, dty;
        const float tw = sample_q<S, false>(T, L.W, L.H, L.Tp, c, r, ux, uy, dtx, dty);
        const float rv = ldS<S>(Rrow + c) - L.cR;
        const float tv = tw - L.cR;
        a[0].x += tv;
        acc_prod(a[1].x, e1.x, tv, tv);
        acc_prod(a[2].x, e2.x, rv, tv);
        if constexpr (RSTAT) {
            a[3].x += rv;
            acc_prod(a[4].x, e4.x, rv, rv);
        }
    };
    auto flush_fast = [&]() {
#pragma unroll
        for (int m = 0; m < (RSTAT ? 5 : 3); ++m) {
            ff_acc(hi[m], lo[m], a[m].x + a[m].y);
            a[m] = make_float2(0.f, 0.f);
        }
        lo[1] += e1.x + e1.y; lo[2] += e2.x + e2.y;
        e1 = make_float2(0.f, 0.f); e2 = e1;
        if constexpr (RSTAT) { lo[4] += e4.x + e4.y; e4 = e1; }
    };
    // A lane's columns are 32 apart.  When the cell width sl at this level is a power of two
    // dividing 32, the spacing a power of two and no column reaches the grid's last line, every
    // column of a lane has the same offset in its cell: the weight along x is fixed per lane and
    // the cell index is a shift.  Both are exact, so the values equal the general form's.
    const int sl = G.s >> GL.l;
    const bool fast = sl >= 1 && sl <= 32 && (sl & (sl - 1)) == 0 && (sl << GL.l) == G.s &&
                      fmaf(GL.pl, (float)(L.W - 1), GL.off) * GL.scale_inv < (float)(G.nx - 1);
    if (fast) {
        const int lgl = 31 - __clz(sl);
        const float wxl = fmaf(GL.pl, (float)(lane & (sl - 1)), GL.off) * GL.scale_inv;
        const float2 wxl2 = make_float2(wxl, wxl);
        for_rows2<U>(
            L.W, r0, r1, row,
            [&](int r, int ca, int cb) {
                const float4 qa = crow[ca >> lgl], qb = crow[cb >> lgl];
                pixel2(r, ca, cb, __ffma2_rn(wxl2, make_float2(qa.z, qb.z), make_float2(qa.x, qb.x)),
                       __ffma2_rn(wxl2, make_float2(qa.w, qb.w), make_float2(qa.y, qb.y)));
            },
            [&](int r, int c) {
                const float4 q = crow[c >> lgl];
                pixel(r, c, fmaf(wxl, q.z, q.x), fmaf(wxl, q.w, q.y));
            },
            flush_fast, []() {});
    } else {
        auto cellx = [&](int c, float &wx) {
            const float gxf = fminf(fmaf(GL.pl, (float)c, GL.off) * GL.scale_inv, (float)(G.nx - 1));
            const int ix = min((int)gxf, G.nx - 2);
            wx = gxf - (float)ix;
            return crow[ix];
        };
        for_rows2<U>(
            L.W, r0, r1, row,
            [&](int r, int ca, int cb) {
                float wa, wb;
                const float4 qa = cellx(ca, wa), qb = cellx(cb, wb);
                const float2 w2 = make_float2(wa, wb);
                pixel2(r, ca, cb, __ffma2_rn(w2, make_float2(qa.z, qb.z), make_float2(qa.x, qb.x)),
                       __ffma2_rn(w2, make_float2(qa.w, qb.w), make_float2(qa.y, qb.y)));
            },
            [&](int r, int c) {
                float wx;
                const float4 q = cellx(c, wx);
                pixel(r, c, fmaf(wx, q.z, q.x), fmaf(wx, q.w, q.y));
            },
            flush_fast, []() {});
    }
    if (cl.block_rank() == 0) {
        const int Nc = G.nx * G.ny;
        float e = 0.f;
        int k = 0;
        for (int j = threadIdx.x; j < Nc; j += kThreads) {
            const int jx = j % G.nx;
            const float2 v = ct(j);
            if (jx + 1 < G.nx) {
                const float2 w = ct(j + 1);
                e = fmaf(w.x - v.x, w.x - v.x, fmaf(w.y - v.y, w.y - v.y, e));
            }
            if (j + G.nx < Nc) {
                const float2 w = ct(j + G.nx);
                e = fmaf(w.x - v.x, w.x - v.x, fmaf(w.y - v.y, w.y - v.y, e));
            }
            if (++k == kFast) { ff_acc(hi[5], lo[5], e); e = 0.f; k = 0; }
        }
        ff_acc(hi[5], lo[5], e);
    }
    cluster_reduce<NM, false>(hi, lo, sm, buf, cl, false);
}

// Sum eight per-lane values over aligned segments of S lanes (S = 8, 16 or 32) by halving
// exchanges: on return every lane holds its segment's total of value index 4 B1 + 2 B2 + B3, where
// B1, B2, B3 are the lane's bits at S/2, S/4 and S/8 (the same in the S/8 lanes sharing them).
// 2 log2(S) + 1 shuffles for S = 32 instead of 40; fixed order, so deterministic.
template <int S>
__device__ __forceinline__ float seg_reduce_scatter8(const float (&v)[8], int lane)
{
    constexpr int o1 = S / 2, o2 = S / 4, o3 = S / 8;
    const bool b1 = lane & o1, b2 = lane & o2, b3 = lane & o3;
    float a4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = b1 ? v[k] : v[k + 4], keep = b1 ? v[k + 4] : v[k];
        a4[k] = keep + __shfl_xor_sync(0xffffffffu, send, o1);
    }
    float a2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = b2 ? a4[k] : a4[k + 2], keep = b2 ? a4[k + 2] : a4[k];
        a2[k] = keep + __shfl_xor_sync(0xffffffffu, send, o2);
    }
    const float send = b3 ? a2[0] : a2[1], keep = b3 ? a2[1] : a2[0];
    float t = keep + __shfl_xor_sync(0xffffffffu, send, o3);
#pragma unroll
    for (int o = o3 / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// Value index a lane holds after seg_reduce_scatter8<S>, and whether it is the segment's writer.
template <int S>
__device__ __forceinline__ int seg_index8(int lane)
{
    return ((lane & (S / 2)) ? 4 : 0) + ((lane & (S / 4)) ? 2 : 0) + ((lane & (S / 8)) ? 1 : 0);
}

// Buffers of the H1 scalar product (B null: another product): B the right-hand side -Nc dE/dc,
// T and U work grids, q the cosine bases and eigenvalues of the control grid (Qx [nx][nx],
// Qy [ny][ny], lx [nx], ly [ny], device memory), s2 = sigma^2.
struct H1Bufs {
    float2 *B = nullptr, *T = nullptr, *U = nullptr;
    const float *q = nullptr;
    float s2 = 0.f;
};

// U = (I + s2 Lg)^-1 B per axis, Lg the control grid's graph Laplacian, through its eigenbasis:
// Lg = (Qy (x) Qx) diag(ly_m + lx_k) (Qy (x) Qx)^T with Qx, Qy the orthonormal DCT-II bases
// (free-end path graphs), so U = Qy [(Qy^T B Qx) / (1 + s2 (ly_m + lx_k))] Qx^T: four small matrix
// products over the grid, every CTA of the cluster the same work in the same order.
__device__ void h1_solve(const H1Bufs &h, int nx, int ny)
{
    const float *Qx = h.q, *Qy = h.q + nx * nx, *lx = Qy + ny * ny, *ly = lx + nx;
    const int Nc = nx * ny;
    // T = B Qx
    for (int i = threadIdx.x; i < Nc; i += kThreads) {
        const int jy = i / nx, k = i - jy * nx;
        float ax = 0.f, ay = 0.f;
        for (int jx = 0; jx < nx; ++jx) {
            const float qv = __ldg(Qx + jx * nx + k);
            const float2 b = h.B[jy * nx + jx];
            ax = fmaf(b.x, qv, ax);
            ay = fmaf(b.y, qv, ay);
        }
        h.T[i] = make_float2(ax, ay);
    }
    __syncthreads();
    // U = (Qy^T T) / (1 + s2 (ly_m + lx_k))
    for (int i = threadIdx.x; i < Nc; i += kThreads) {
        const int m = i / nx, k = i - m * nx;
        float ax = 0.f, ay = 0.f;
        for (int jy = 0; jy < ny; ++jy) {
            const float qv = __ldg(Qy + jy * ny + m);
            const float2 t = h.T[jy * nx + k];
            ax = fmaf(qv, t.x, ax);
            ay = fmaf(qv, t.y, ay);
        }
        const float den = fmaf(h.s2, __ldg(ly + m) + __ldg(lx + k), 1.f);
        h.U[i] = make_float2(ax / den, ay / den);
    }
    __syncthreads();
    // T = Qy U
    for (int i = threadIdx.x; i < Nc; i += kThreads) {
        const int jy = i / nx, k = i - jy * nx;
        float ax = 0.f, ay = 0.f;
        for (int m = 0; m < ny; ++m) {
            const float qv = __ldg(Qy + jy * ny + m);
            const float2 u = h.U[m * nx + k];
            ax = fmaf(qv, u.x, ax);
            ay = fmaf(qv, u.y, ay);
        }
        h.T[i] = make_float2(ax, ay);
    }
    __syncthreads();
    // U = T Qx^T
    for (int i = threadIdx.x; i < Nc; i += kThreads) {
        const int jy = i / nx, jx = i - jy * nx;
        float ax = 0.f, ay = 0.f;
        for (int k = 0; k < nx; ++k) {
            const float qv = __ldg(Qx + jx * nx + k);
            const float2 t = h.T[jy * nx + k];
            ax = fmaf(t.x, qv, ax);
            ay = fmaf(t.y, qv, ay);
        }
        h.U[i] = make_float2(ax, ay);
    }
    __syncthreads();
}

// Gradient pass at c: this CTA's cells in four parity phases (no two cells of a phase share a
// corner, so each corner is updated by one warp at a time, in a fixed order); then every CTA
// assembles the whole gradient from the (at most two) CTAs whose band holds each control row,
// and forms d = -(Nc/P) [sum F grad T w + lambda sum_nbrs (c_j - c_k)], F = P dE/dTw.
// d = -M^-1 grad E with the scalar product mt.  pm: aP, bP, rbar, tbar, lambda.  Returns
// sum_j m_j |d_j|^2 (float-float, in sm.tot[0]), max |d_j|^2 (sm.tot[1]), and with the direction
// d held before the call, <d_old, d_old - d>_M (sm.tot[2]) and |d_old - d|_M^2 (sm.tot[3]);
// identical in every CTA.
//
// METRIC: instead of the gradient, the flow's scalar product at c (the level's initial control
// values): per control point and axis m = dk sum_x w_j(x)^2 (dT/dp)^2 + rk n_j (pm[0] = dk =
// 1/(P var T), pm[1] = rk = lambda/P, n_j the neighbours of j), normalised by the mean of all
// 2 Nc values and floored at 1e-3 of it, written to mt.
template <typename S, bool METRIC>
__device__ void grid_grad_pass(const Lvl &L, const Grid &G, const GridLvl &GL, const float2 *c, float2 *d,
                               float2 *mt, float2 *gp, const float *pm, int cr0, int cr1, Smem &sm,
                               const cg::cluster_group &cl, const H1Bufs &h1)
{
    const S *R = (const S *)L.R, *T = (const S *)L.T;
    const float aP = pm[0], bP = pm[1], rb = pm[2], tb = pm[3], lam = pm[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int Nc = G.nx * G.ny, ncx = G.nx - 1, ncy = G.ny - 1;
    const int sl = G.s >> GL.l;
    const int lg = 31 - __clz(max(sl, 1));   // log2 of sl when sl is a power of two (the fast path below)
    // fast path: cell width a power of two dividing 32, spacing a power of two
    const bool pow2 = sl >= 1 && sl <= 32 && (sl & (sl - 1)) == 0 && (sl << GL.l) == G.s;
    const float dwy = (float)(32 >> lg) * GL.pl * GL.scale_inv;   // weight step between a lane's rows
    // cells of width 16 or 8: G = 32 / sl cells per warp (below)
    const int grp = (pow2 && (sl == 16 || sl == 8)) ? 32 / sl : 1;
    float *gpf = (float *)gp;   // band-local: control row cr0 + i at gp[i nx .. (i + 1) nx)
    for (int j = tid; j < (cr1 - cr0 + 1) * G.nx; j += kThreads) gp[j] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int phase = 0; phase < 4; ++phase) {
        const int px = phase & 1, py = phase >> 1;
        const int first_row = cr0 + ((py - cr0) % 2 + 2) % 2;
        const int rows = first_row < cr1 ? (cr1 - first_row + 1) / 2 : 0;
        const int cols = (ncx - px + 1) / 2;
        // cells taken G at a time by a warp (all but a last column narrower than sl), then the rest
        // one per warp
        const bool has_last = ncx - 1 - px >= 0 && ((ncx - 1 - px) & 1) == 0;
        const int gcols = grp > 1 ? cols - ((has_last && L.W - (ncx - 1) * sl != sl) ? 1 : 0) : 0;
        const int gpr = (gcols + grp - 1) / grp;   // groups per phase row
        const int ngroup = rows * gpr, rc = cols - gcols;
        for (int q = warp; q < ngroup + rows * rc; q += kWarps) {
            if (q < ngroup) {
                // lane: column lane mod sl of cell k = lane / sl of the group, through all its rows;
                // weights and x-interpolated control values as in the single-cell form below
                const int ri = q / gpr, ci = (q - ri * gpr) * grp + (lane >> lg);
                const bool valid = ci < gcols;
                const int cyy = first_row + 2 * ri, cxx = px + 2 * min(ci, gcols - 1);
                const int x = cxx * sl + (lane & (sl - 1));
                const int y0 = cyy * sl, y1 = (cyy == ncy - 1) ? L.H : min(L.H, y0 + sl);
                const int j0 = cyy * G.nx + cxx;
                const float2 c00 = c[j0], c01 = c[j0 + 1], c10 = c[j0 + G.nx], c11 = c[j0 + G.nx + 1];
                const float wx = fminf(fmaf(GL.pl, (float)x, GL.off) * GL.scale_inv, (float)(G.nx - 1)) - (float)cxx;
                const float tx = fmaf(wx, c01.x - c00.x, c00.x), ty = fmaf(wx, c01.y - c00.y, c00.y);
                const float bx = fmaf(wx, c11.x - c10.x, c10.x), by = fmaf(wx, c11.y - c10.y, c10.y);
                const float ex = bx - tx, ey = by - ty;
                const float wmax = (float)(G.ny - 1 - cyy), dw1 = GL.pl * GL.scale_inv;
                float wyk = GL.off * GL.scale_inv;   // g(y0) - cyy, exact
                float st_x = 0.f, st_y = 0.f, sb_x = 0.f, sb_y = 0.f;
#pragma unroll 4
                for (int y = y0; y < y1; ++y) {
                    const float wy = fminf(wyk, wmax);
                    wyk += dw1;
                    float dtx, dty;
                    const float tw = sample_q<S, true>(T, L.W, L.H, L.Tp, x, y, fmaf(wy, ex, tx), fmaf(wy, ey, ty),
                                                       dtx, dty);
                    const float hy = 1.f - wy;
                    if constexpr (METRIC) {
                        (void)tw;
                        const float gx = dtx * dtx, gy = dty * dty, hy2 = hy * hy, wy2 = wy * wy;
                        st_x = fmaf(hy2, gx, st_x); st_y = fmaf(hy2, gy, st_y);
                        sb_x = fmaf(wy2, gx, sb_x); sb_y = fmaf(wy2, gy, sb_y);
                    } else {
                        const float rv = ldS<S>(R + (size_t)y * L.Rp + x) - L.cR;
                        const float tv = tw - L.cR;
                        const float F = -__fsub_rn(__fmul_rn(aP, rv - rb), __fmul_rn(bP, tv - tb));
                        const float gx = F * dtx, gy = F * dty;
                        st_x = fmaf(hy, gx, st_x); st_y = fmaf(hy, gy, st_y);
                        sb_x = fmaf(wy, gx, sb_x); sb_y = fmaf(wy, gy, sb_y);
                    }
                }
                const float hx = METRIC ? (1.f - wx) * (1.f - wx) : 1.f - wx, vx = METRIC ? wx * wx : wx;
                const float m = valid ? 1.f : 0.f;
                float acc[8] = {m * hx * st_x, m * hx * st_y, m * vx * st_x, m * vx * st_y,
                                m * hx * sb_x, m * hx * sb_y, m * vx * sb_x, m * vx * sb_y};
                const float tot = sl == 16 ? seg_reduce_scatter8<16>(acc, lane) : seg_reduce_scatter8<8>(acc, lane);
                const bool writer = sl == 16 ? (lane & 1) == 0 : true;
                if (valid && writer) {
                    const int vi = sl == 16 ? seg_index8<16>(lane) : seg_index8<8>(lane);
                    const int corner = vi >> 1;
                    const int jc = (cyy + (corner >> 1) - cr0) * G.nx + cxx + (corner & 1);
                    gpf[2 * jc + (vi & 1)] += tot;
                }
                continue;
            }
            const int r = q - ngroup;
            const int cyy = first_row + 2 * (r / rc), cxx = px + 2 * (gcols + r % rc);
            const int x0 = cxx * sl, x1 = (cxx == ncx - 1) ? L.W : min(L.W, x0 + sl);
            const int y0 = cyy * sl, y1 = (cyy == ncy - 1) ? L.H : min(L.H, y0 + sl);
            const int w = x1 - x0, npx = w * (y1 - y0);
            const int j0 = cyy * G.nx + cxx;
            const float2 c00 = c[j0], c01 = c[j0 + 1], c10 = c[j0 + G.nx], c11 = c[j0 + G.nx + 1];
            const float2 dtop = make_float2(c01.x - c00.x, c01.y - c00.y);
            const float2 dbot = make_float2(c11.x - c10.x, c11.y - c10.y);
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (w == sl && pow2) {
                // Full-width cell whose width (a power of two) divides the warp: every lane keeps one column
                // (x = x0 + lane mod sl) and walks rows 32/sl apart, so the weight along x and
                // the x-interpolated control values are fixed per lane; the y weights are summed
                // and the x weights applied once at the end (the bilinear weight factorises).
                // With a power-of-two spacing the weights are exact dyadic values, so the weight
                // along y advances by a constant and equals the per-row formula
                // min(g(y), ny - 1) - cyy, g(y) = (2^l y + off) / s.
                const int x = x0 + (lane & (sl - 1)), dy = 32 >> lg;
                const float wx = fminf(fmaf(GL.pl, (float)x, GL.off) * GL.scale_inv, (float)(G.nx - 1)) - (float)cxx;
                const float tx = fmaf(wx, dtop.x, c00.x), ty = fmaf(wx, dtop.y, c00.y);
                const float bx = fmaf(wx, dbot.x, c10.x), by = fmaf(wx, dbot.y, c10.y);
                const float ex = bx - tx, ey = by - ty;
                const float wmax = (float)(G.ny - 1 - cyy);
                float wyk = fmaf(GL.pl, (float)(lane >> lg), GL.off) * GL.scale_inv;
                float st_x = 0.f, st_y = 0.f, sb_x = 0.f, sb_y = 0.f;
#pragma unroll 4
                for (int y = y0 + (lane >> lg); y < y1; y += dy) {
                    const float wy = fminf(wyk, wmax);
                    wyk += dwy;
                    float dtx, dty;
                    const float tw = sample_q<S, true>(T, L.W, L.H, L.Tp, x, y, fmaf(wy, ex, tx), fmaf(wy, ey, ty),
                                                       dtx, dty);
                    const float hy = 1.f - wy;
                    if constexpr (METRIC) {
                        // squared weights: w^2 = hx^2 hy^2 factorises like w
                        (void)tw;
                        const float gx = dtx * dtx, gy = dty * dty, hy2 = hy * hy, wy2 = wy * wy;
                        st_x = fmaf(hy2, gx, st_x); st_y = fmaf(hy2, gy, st_y);
                        sb_x = fmaf(wy2, gx, sb_x); sb_y = fmaf(wy2, gy, sb_y);
                    } else {
                        const float rv = ldS<S>(R + (size_t)y * L.Rp + x) - L.cR;
                        const float tv = tw - L.cR;
                        // F = P dE/dTw = -(aP (r - rbar) - bP (t - tbar)), no contraction
                        const float F = -__fsub_rn(__fmul_rn(aP, rv - rb), __fmul_rn(bP, tv - tb));
                        const float gx = F * dtx, gy = F * dty;
                        st_x = fmaf(hy, gx, st_x); st_y = fmaf(hy, gy, st_y);
                        sb_x = fmaf(wy, gx, sb_x); sb_y = fmaf(wy, gy, sb_y);
                    }
                }
                const float hx = METRIC ? (1.f - wx) * (1.f - wx) : 1.f - wx, vx = METRIC ? wx * wx : wx;
                acc[0] = hx * st_x; acc[1] = hx * st_y; acc[2] = vx * st_x; acc[3] = vx * st_y;
                acc[4] = hx * sb_x; acc[5] = hx * sb_y; acc[6] = vx * sb_x; acc[7] = vx * sb_y;
            } else
            for (int i = lane; i < npx; i += 32) {
                const int y = y0 + i / w, x = x0 + i % w;
                const float gxf = fminf(fmaf(GL.pl, (float)x, GL.off) * GL.scale_inv, (float)(G.nx - 1));
                const float gyf = fminf(fmaf(GL.pl, (float)y, GL.off) * GL.scale_inv, (float)(G.ny - 1));
                const float wx = gxf - (float)cxx, wy = gyf - (float)cyy;
                const float tx = fmaf(wx, dtop.x, c00.x), ty = fmaf(wx, dtop.y, c00.y);
                const float bx = fmaf(wx, dbot.x, c10.x), by = fmaf(wx, dbot.y, c10.y);
                const float ux = fmaf(wy, bx - tx, tx), uy = fmaf(wy, by - ty, ty);
                float dtx, dty;
                const float tw = sample_q<S, true>(T, L.W, L.H, L.Tp, x, y, ux, uy, dtx, dty);
                float gx, gy;
                if constexpr (METRIC) {
                    (void)tw;
                    gx = dtx * dtx;
                    gy = dty * dty;
                } else {
                    const float rv = ldS<S>(R + (size_t)y * L.Rp + x) - L.cR;
                    const float tv = tw - L.cR;
                    // F = P dE/dTw = -(aP (r - rbar) - bP (t - tbar)), no contraction
                    const float F = -__fsub_rn(__fmul_rn(aP, rv - rb), __fmul_rn(bP, tv - tb));
                    gx = F * dtx;
                    gy = F * dty;
                }
                const float hx = 1.f - wx, hy = 1.f - wy;
                float w00 = hx * hy, w01 = wx * hy, w10 = hx * wy, w11 = wx * wy;
                if constexpr (METRIC) { w00 *= w00; w01 *= w01; w10 *= w10; w11 *= w11; }
                acc[0] = fmaf(w00, gx, acc[0]); acc[1] = fmaf(w00, gy, acc[1]);
                acc[2] = fmaf(w01, gx, acc[2]); acc[3] = fmaf(w01, gy, acc[3]);
                acc[4] = fmaf(w10, gx, acc[4]); acc[5] = fmaf(w10, gy, acc[5]);
                acc[6] = fmaf(w11, gx, acc[6]); acc[7] = fmaf(w11, gy, acc[7]);
            }
            const float tot8 = seg_reduce_scatter8<32>(acc, lane);
            if ((lane & 3) == 0) {
                const int vi = seg_index8<32>(lane);
                const int corner = vi >> 1;
                const int jc = (cyy + (corner >> 1) - cr0) * G.nx + cxx + (corner & 1);
                gpf[2 * jc + (vi & 1)] += tot8;
            }
        }
        __syncthreads();
    }
    cl.sync();   // every CTA's partial gradient is complete and visible in the cluster
    const int C = cl.num_blocks();
    const int q = (ncy + C - 1) / C;
    const float scale = -(float)Nc / ((float)L.W * (float)L.H);
    if constexpr (METRIC) {
        // m_j = dk sum w^2 dT^2 + rk n_j per axis, then its mean over all 2 Nc values
        const float dk = pm[0], rk = pm[1];
        float mh = 0.f, ml = 0.f, mrun = 0.f;
        int kk = 0;
        for (int j = tid; j < Nc; j += kThreads) {
            const int jy = j / G.nx, jx = j - jy * G.nx;
            const int rlo = jy > 0 ? min(C - 1, (jy - 1) / max(q, 1)) : 0;
            const int rhi = min(C - 1, jy / max(q, 1));
            float2 h = *cl.map_shared_rank(gp + (jy - min(ncy, rlo * q)) * G.nx + jx, rlo);
            if (rhi != rlo) {
                const float2 h2 = *cl.map_shared_rank(gp + (jy - min(ncy, rhi * q)) * G.nx + jx, rhi);
                h.x += h2.x;
                h.y += h2.y;
            }
            const float nb = (float)((jx > 0) + (jx + 1 < G.nx) + (jy > 0) + (jy + 1 < G.ny));
            const float2 m = make_float2(fmaf(dk, h.x, rk * nb), fmaf(dk, h.y, rk * nb));
            mt[j] = m;
            mrun += m.x + m.y;
            if (++kk == kFast) { ff_acc(mh, ml, mrun); mrun = 0.f; kk = 0; }
        }
        ff_acc(mh, ml, mrun);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, mh, off), l2 = __shfl_xor_sync(0xffffffffu, ml, off);
            ff_add(mh, ml, h2, l2);
        }
        if (lane == 0) sm.warp[warp][0] = make_float2(mh, ml);
        __syncthreads();
        if (tid == 0) {
            float h = 0.f, l = 0.f;
            for (int w2 = 0; w2 < kWarps; ++w2) ff_add(h, l, sm.warp[w2][0].x, sm.warp[w2][0].y);
            sm.tot[0] = ((double)h + (double)l) / (2.0 * Nc);
        }
        __syncthreads();
        const double mean = sm.tot[0];
        const float inv = mean > 0.0 ? (float)(1.0 / mean) : 0.f;
        for (int j = tid; j < Nc; j += kThreads) {
            const float2 m = mt[j];
            mt[j] = mean > 0.0 ? make_float2(fmaxf(m.x * inv, 1e-3f), fmaxf(m.y * inv, 1e-3f)) : make_float2(1.f, 1.f);
        }
        // no CTA may overwrite its band (next gradient pass) while a peer still reads it
        cl.sync();
        return;
    }
    float ssh = 0.f, ssl = 0.f, mx = 0.f, run = 0.f;
    // <d_prev, d_prev - d> and |d_prev - d|^2 for the first trial step (d still holds d_prev)
    float nmh = 0.f, nml = 0.f, dnh = 0.f, dnl = 0.f, nrun = 0.f, drun = 0.f;
    int k = 0;
    constexpr int kBatch = 4;   // points per thread whose remote loads are in flight together
    if (h1.B) {
        // H1 product: b = scale (lambda lap + g) = -Nc dE/dc into B, d = M^-1 b into U; then
        // |d|_M^2 = d.b, and for the first trial <d_prev, y>_M, |y|_M^2 with y = d_prev - d, M y
        // taken as the stencil y + s2 Lg y
        for (int j = tid; j < Nc; j += kThreads) {
            const int jy = j / G.nx, jx = j - jy * G.nx;
            const int rlo = jy > 0 ? min(C - 1, (jy - 1) / max(q, 1)) : 0;
            const int rhi = min(C - 1, jy / max(q, 1));
            float2 g = *cl.map_shared_rank(gp + (jy - min(ncy, rlo * q)) * G.nx + jx, rlo);
            if (rhi != rlo) {
                const float2 w2 = *cl.map_shared_rank(gp + (jy - min(ncy, rhi * q)) * G.nx + jx, rhi);
                g.x += w2.x;
                g.y += w2.y;
            }
            const float2 cj = c[j];
            float lx = 0.f, ly = 0.f;
            if (jx > 0)        { const float2 v = c[j - 1];    lx += cj.x - v.x; ly += cj.y - v.y; }
            if (jx + 1 < G.nx) { const float2 v = c[j + 1];    lx += cj.x - v.x; ly += cj.y - v.y; }
            if (jy > 0)        { const float2 v = c[j - G.nx]; lx += cj.x - v.x; ly += cj.y - v.y; }
            if (jy + 1 < G.ny) { const float2 v = c[j + G.nx]; lx += cj.x - v.x; ly += cj.y - v.y; }
            h1.B[j] = make_float2(scale * fmaf(lam, lx, g.x), scale * fmaf(lam, ly, g.y));
        }
        __syncthreads();
        h1_solve(h1, G.nx, G.ny);
        auto yv = [&](int i) {
            const float2 a = d[i], b = h1.U[i];
            return make_float2(a.x - b.x, a.y - b.y);
        };
        for (int j = tid; j < Nc; j += kThreads) {
            const int jy = j / G.nx, jx = j - jy * G.nx;
            const float2 dj = h1.U[j], bj = h1.B[j], dold = d[j], y = yv(j);
            float lx = 0.f, ly = 0.f;
            if (jx > 0)        { const float2 v = yv(j - 1);    lx += y.x - v.x; ly += y.y - v.y; }
            if (jx + 1 < G.nx) { const float2 v = yv(j + 1);    lx += y.x - v.x; ly += y.y - v.y; }
            if (jy > 0)        { const float2 v = yv(j - G.nx); lx += y.x - v.x; ly += y.y - v.y; }
            if (jy + 1 < G.ny) { const float2 v = yv(j + G.nx); lx += y.x - v.x; ly += y.y - v.y; }
            const float myx = fmaf(h1.s2, lx, y.x), myy = fmaf(h1.s2, ly, y.y);
            run = fmaf(dj.x, bj.x, fmaf(dj.y, bj.y, run));
            nrun = fmaf(dold.x, myx, fmaf(dold.y, myy, nrun));
            drun = fmaf(y.x, myx, fmaf(y.y, myy, drun));
            mx = fmaxf(mx, fmaf(dj.x, dj.x, dj.y * dj.y));
            if (++k == kFast) {
                ff_acc(ssh, ssl, run); run = 0.f;
                ff_acc(nmh, nml, nrun); nrun = 0.f;
                ff_acc(dnh, dnl, drun); drun = 0.f;
                k = 0;
            }
        }
        __syncthreads();   // every d_prev was read before d is replaced
        for (int j = tid; j < Nc; j += kThreads) d[j] = h1.U[j];
    } else
    for (int j0 = tid; j0 < Nc; j0 += kBatch * kThreads) {
        float2 gb[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            const int j = j0 + b * kThreads;
            gb[b] = make_float2(0.f, 0.f);
            if (j < Nc) {
                const int jy = j / G.nx;
                // bands: rank r owns cell rows [r q, (r+1) q) and so control rows [r q, (r+1) q]
                const int rlo = jy > 0 ? min(C - 1, (jy - 1) / max(q, 1)) : 0;
                const int rhi = min(C - 1, jy / max(q, 1));
                const int jx = j - jy * G.nx;
                const float2 v = *cl.map_shared_rank(gp + (jy - min(ncy, rlo * q)) * G.nx + jx, rlo);
                gb[b].x += v.x;
                gb[b].y += v.y;
                if (rhi != rlo) {
                    const float2 w2 = *cl.map_shared_rank(gp + (jy - min(ncy, rhi * q)) * G.nx + jx, rhi);
                    gb[b].x += w2.x;
                    gb[b].y += w2.y;
                }
            }
        }
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
        const int j = j0 + b * kThreads;
        if (j >= Nc) break;
        const int jy = j / G.nx, jx = j - jy * G.nx;
        const float2 g = gb[b];
        const float2 cj = c[j];
        float lx = 0.f, ly = 0.f;
        if (jx > 0)        { const float2 v = c[j - 1];    lx += cj.x - v.x; ly += cj.y - v.y; }
        if (jx + 1 < G.nx) { const float2 v = c[j + 1];    lx += cj.x - v.x; ly += cj.y - v.y; }
        if (jy > 0)        { const float2 v = c[j - G.nx]; lx += cj.x - v.x; ly += cj.y - v.y; }
        if (jy + 1 < G.ny) { const float2 v = c[j + G.nx]; lx += cj.x - v.x; ly += cj.y - v.y; }
        // d = -M^-1 grad E with the level's scalar product M (per axis)
        const float2 mj = mt[j];
        float2 dj;
        dj.x = scale * fmaf(lam, lx, g.x) / mj.x;
        dj.y = scale * fmaf(lam, ly, g.y) / mj.y;
        const float2 dold = d[j];
        d[j] = dj;
        const float qd = fmaf(dj.x, dj.x, dj.y * dj.y);
        const float yx = dold.x - dj.x, yy = dold.y - dj.y;
        run = fmaf(mj.x * dj.x, dj.x, fmaf(mj.y * dj.y, dj.y, run));
        nrun = fmaf(mj.x * dold.x, yx, fmaf(mj.y * dold.y, yy, nrun));
        drun = fmaf(mj.x * yx, yx, fmaf(mj.y * yy, yy, drun));
        mx = fmaxf(mx, qd);
        if (++k == kFast) {
            ff_acc(ssh, ssl, run); run = 0.f;
            ff_acc(nmh, nml, nrun); nrun = 0.f;
            ff_acc(dnh, dnl, drun); drun = 0.f;
            k = 0;
        }
        }
    }
    ff_acc(ssh, ssl, run);
    ff_acc(nmh, nml, nrun);
    ff_acc(dnh, dnl, drun);
    // block reduction (identical in every CTA: same inputs, same order)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        float h2 = __shfl_xor_sync(0xffffffffu, ssh, off), l2 = __shfl_xor_sync(0xffffffffu, ssl, off);
        ff_add(ssh, ssl, h2, l2);
        h2 = __shfl_xor_sync(0xffffffffu, nmh, off); l2 = __shfl_xor_sync(0xffffffffu, nml, off);
        ff_add(nmh, nml, h2, l2);
        h2 = __shfl_xor_sync(0xffffffffu, dnh, off); l2 = __shfl_xor_sync(0xffffffffu, dnl, off);
        ff_add(dnh, dnl, h2, l2);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) {
        sm.warp[warp][0] = make_float2(ssh, ssl);
        sm.warp[warp][1] = make_float2(mx, 0.f);
        sm.warp[warp][2] = make_float2(nmh, nml);
        sm.warp[warp][3] = make_float2(dnh, dnl);
    }
    __syncthreads();
    if (tid < 4 && tid != 1) {
        float h = 0.f, l = 0.f;
        for (int w2 = 0; w2 < kWarps; ++w2) ff_add(h, l, sm.warp[w2][tid].x, sm.warp[w2][tid].y);
        sm.tot[tid] = (double)h + (double)l;
    } else if (tid == 1) {
        float m = 0.f;
        for (int w2 = 0; w2 < kWarps; ++w2) m = fmaxf(m, sm.warp[w2][1].x);
        sm.tot[1] = (double)m;
    }
    __syncthreads();
}

__device__ double field_energy(FieldCtl &k, const Config &cfg, const double *tot, bool trial)
{
    Ncc n = ncc_terms(k.P, k.invP, k.sr, tot[0], k.srr, tot[1], tot[2]);
    double Ed = n.degenerate ? 1.0 : __dsub_rn(1.0, n.ncc);
    double E = Ed + 0.5 * cfg.lambda * tot[5] * k.invP;
    if (trial) { k.ta = n.a; k.tb = n.b; k.trbar = n.rbar; k.ttbar = n.tbar; k.tdegen = n.degenerate; }
    else { k.a = n.a; k.b = n.b; k.rbar = n.rbar; k.tbar = n.tbar; k.degen = n.degenerate; }
    return E;
}

// Gradient-pass parameters from the current NCC terms: aP, bP, rbar, tbar, lambda.
__device__ void field_grad_params(const FieldCtl &k, const Config &cfg, float *pm)
{
    pm[0] = (float)(k.a * k.P);
    pm[1] = (float)(k.b * k.P);
    pm[2] = (float)k.rbar;
    pm[3] = (float)k.tbar;
    pm[4] = (float)cfg.lambda;
}

// Thread-0 controller of the nonrigid level loop (same rules as the rigid one): ENERGY at level
// start, GRAD = gradient pass, TRIAL = Armijo trial at c + tau d.  pm[0] of a trial is tau.
__device__ int field_step(FieldCtl &k, const Config &cfg, const double *tot, int action, float *pm)
{
    if (action == kActEnergy) {
        k.sr = tot[3]; k.srr = tot[4];
        k.E = field_energy(k, cfg, tot, false);
        if (cfg.metric == 1) {
            // the level's scalar product at its initial control values: 1/(P var T) and lambda/P
            const double vt = (tot[1] - tot[0] * tot[0] * k.invP) * k.invP;
            pm[0] = vt > 0.0 ? (float)(k.invP / vt) : 0.f;
            pm[1] = (float)(cfg.lambda * k.invP);
            return kActMetric;
        }
        field_grad_params(k, cfg, pm);
        return kActGrad;
    }
    if (action == kActMetric) {
        field_grad_params(k, cfg, pm);
        return kActGrad;
    }
    if (action == kActGrad) {
        k.evals += 1;
        if (k.iters >= cfg.max_iter) { k.stop = REG_STOP_MAXIT; return kActDone; }
        // |g| = sqrt(ss / Nc) and the largest control step dmax = sqrt(tot[1]): compared squared
        const double ss = tot[0], dmax2 = tot[1];
        k.slope = -ss * k.invNc;
        if (!(ss * k.invNc >= k.tolg * k.tolg)) { k.stop = REG_STOP_GRAD; return kActDone; }
        // the metric (mean over control points) is a common factor of tot[2] and tot[3]
        if (k.have_prev) k.tau = bb_tau(k.tau, k.tau_acc, tot[2], tot[3]);
        if (k.tau * k.tau * dmax2 > cfg.step_cap * cfg.step_cap) k.tau = cfg.step_cap / sqrt(dmax2);
        k.nrej = 0;
        pm[0] = (float)k.tau;
        return kActTrial;
    }
    // trial
    const double Et = field_energy(k, cfg, tot, true);
    k.evals += 1;
    if (Et <= k.E + cfg.armijo_c * k.tau * k.slope) {
        k.iters += 1;
        const double Eold = k.E;
        k.tau_pend = (double)(float)k.tau;
        k.tau_acc = k.tau_pend;   // the step applied: c + (float)tau d
        k.have_prev = 1;
        k.tau = next_tau(k.E, k.slope, k.tau, Et, true);
        k.E = Et;
        k.a = k.ta; k.b = k.tb; k.rbar = k.trbar; k.tbar = k.ttbar; k.degen = k.tdegen;
        if (Eold - Et <= cfg.tol_rel_e * fabs(Eold)) { k.stop = REG_STOP_REL; return kActDone; }
        field_grad_params(k, cfg, pm);
        return kActGrad;   // c is advanced to ct before the gradient pass
    }
    k.rejects += 1;
    k.nrej += 1;
    k.tau = next_tau(k.E, k.slope, k.tau, Et, false);
    k.tau_pend = 0.0;
    if (k.nrej > cfg.max_rejects) { k.stop = REG_STOP_LS; return kActDone; }
    pm[0] = (float)k.tau;
    return kActTrial;
}

// FFD value of the grid q (finest-pixel values) at finest coordinate (X, Y), read through L2.
__device__ __forceinline__ float2 grid_eval_global(const float2 *q, const Grid &G, float X, float Y)
{
    float gx = fminf(fmaxf(X / (float)G.s, 0.f), (float)(G.nx - 1));
    float gy = fminf(fmaxf(Y / (float)G.s, 0.f), (float)(G.ny - 1));
    int ix = min((int)gx, G.nx - 2), iy = min((int)gy, G.ny - 2);
    float wx = gx - (float)ix, wy = gy - (float)iy;
    const float2 *p = q + iy * G.nx + ix;
    float2 a = __ldcg(p), b = __ldcg(p + 1), e = __ldcg(p + G.nx), f = __ldcg(p + G.nx + 1);
    float hx = 1.f - wx, hy = 1.f - wy;
    float2 u;
    u.x = fmaf(wy, fmaf(wx, f.x, hx * e.x), hy * fmaf(wx, b.x, hx * a.x));
    u.y = fmaf(wy, fmaf(wx, f.y, hx * e.y), hy * fmaf(wx, b.y, hx * a.y));
    return u;
}

template <typename S, int U>
__device__ void run_nonrigid(const Params &p, const OpDesc &op, int op_index, Smem &sm, float2 *gbuf,
                             const cg::cluster_group &cl)
{
    const int tid = threadIdx.x;
    const int C = cl.num_blocks(), rank = cl.block_rank();
    const Config &cfg = p.cfg;
    const int Lc = cfg.levels;
    const Grid G{p.gnx, p.gny, p.gs};
    const int Nc = G.nx * G.ny;
    const bool h1 = cfg.metric == REG_METRIC_H1;
    const GridLayout lay = grid_layout(G.nx, G.ny, C, h1);
    float2 *c = gbuf + lay.c, *d = gbuf + lay.d, *mt = gbuf + lay.mt, *gp = gbuf + lay.gp;
    float4 *crow = (float4 *)(gbuf + lay.crow);
    // H1 product: mt holds the right-hand side of its solve
    const H1Bufs hb{h1 ? mt : nullptr, h1 ? gbuf + lay.t : nullptr, h1 ? gbuf + lay.u : nullptr, p.h1q,
                    (float)(cfg.sigma * cfg.sigma)};
    int buf = 0;
    // initial control values (finest px), scaled to the coarsest level
    {
        const float sc = ldexpf(1.f, -(Lc - 1));
        if (op.left >= 0) {
            // B's initial guess phi_jk o phi_ij at the control points (Sec. 2.3.2)
            const float2 *q1 = p.node_grid + (size_t)Nc * op.left, *q2 = p.node_grid + (size_t)Nc * op.right;
            for (int j = tid; j < Nc; j += kThreads) {
                const int jy = j / G.nx, jx = j - jy * G.nx;
                const float2 a = __ldcg(q1 + j);
                const float2 u = grid_eval_global(q2, G, (float)(jx * G.s) + a.x, (float)(jy * G.s) + a.y);
                c[j] = make_float2(sc * (a.x + u.x), sc * (a.y + u.y));
            }
        } else if (op.init_node >= 0) {
            const float2 *q = p.node_grid + (size_t)Nc * op.init_node;
            for (int j = tid; j < Nc; j += kThreads) {
                const float2 a = __ldcg(q + j);
                c[j] = make_float2(sc * a.x, sc * a.y);
            }
        } else {
            for (int j = tid; j < Nc; j += kThreads) c[j] = make_float2(0.f, 0.f);
        }
    }
    FieldCtl &k = sm.fctl;
    if (tid == 0) {
        memset(&k, 0, sizeof(k));
        k.Nc = (double)Nc;
        k.invNc = 1.0 / k.Nc;
    }
    int stops[kMaxLevels], iters[kMaxLevels], evals[kMaxLevels];
    for (int l = Lc - 1; l >= 0; --l) {
        const Lvl L = level_of(p, op.ref, op.tmpl, l);
        GridLvl GL;
        GL.W = L.W; GL.H = L.H; GL.l = l;
        GL.pl = ldexpf(1.f, l);
        GL.off = 0.5f * (GL.pl - 1.f);
        GL.scale_inv = 1.f / (float)G.s;
        int cr0, cr1, r0, r1;
        grid_rows(G, GL, rank, C, cr0, cr1, r0, r1);
        for (int j = tid; j < Nc; j += kThreads) mt[j] = make_float2(1.f, 1.f);
        if (tid == 0) {
            k.P = (double)L.W * (double)L.H;
            k.invP = 1.0 / k.P;
            k.tau = cfg.tau0;
            k.tau_pend = 0.0;
            k.have_prev = 0;
            k.iters = 0; k.evals = 0; k.stop = REG_STOP_MAXIT;
            // a coarse level only supplies the next level's initial guess: a looser stop
            k.tolg = cfg.tol_grad * (l > 0 ? cfg.tol_coarse : 1.0);
            sm.action = kActEnergy;
        }
        for (;;) {
            __syncthreads();
            const int act = sm.action;
            if (act == kActDone) break;
            float pm[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) pm[q] = sm.pm[q];
            if (act == kActEnergy) {
                grid_energy_pass<S, true, U, false>(L, G, GL, c, d, 0.f, crow, r0, r1, sm, buf, cl);
            } else if (act == kActTrial) {
                grid_energy_pass<S, false, U, true>(L, G, GL, c, d, pm[0], crow, r0, r1, sm, buf, cl);
            } else if (act == kActMetric) {
                grid_grad_pass<S, true>(L, G, GL, c, d, mt, gp, pm, cr0, cr1, sm, cl, hb);
            } else {
                grid_grad_pass<S, false>(L, G, GL, c, d, mt, gp, pm, cr0, cr1, sm, cl, hb);
            }
            if (tid == 0) {
                const int next = field_step(k, cfg, sm.tot, act, sm.pm);
                sm.action = next;
                sm.idata[0] = (act == kActTrial && k.tau_pend != 0.0) ? 1 : 0;   // accepted: c <- ct
            }
            __syncthreads();
            if (sm.idata[0]) {
                // the accepted trial: c + tau d with the trial's tau, as the trial pass formed it
                for (int j = tid; j < Nc; j += kThreads) {
                    const float2 a = c[j], b = d[j];
                    c[j] = make_float2(fmaf(pm[0], b.x, a.x), fmaf(pm[0], b.y, a.y));
                }
                __syncthreads();
                if (tid == 0) { sm.idata[0] = 0; k.tau_pend = 0.0; }
            }
        }
        if (tid == 0) { stops[l] = k.stop; iters[l] = k.iters; evals[l] = k.evals; }
        if (l > 0) {
            for (int j = tid; j < Nc; j += kThreads) c[j] = make_float2(2.f * c[j].x, 2.f * c[j].y);
        }
        __syncthreads();
    }
    if (rank == 0) {
        float2 *o = p.node_grid + (size_t)Nc * op.out;
        for (int j = tid; j < Nc; j += kThreads) __stcg(o + j, c[j]);
    }
    if (tid == 0 && rank == 0) {
        double mx = 0.0, my = 0.0;
        for (int j = 0; j < Nc; ++j) { mx += c[j].x; my += c[j].y; }
        double *o = p.node_theta + 3 * op.out;
        o[0] = 0.0;
        o[1] = mx / Nc;
        o[2] = my / Nc;
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
// Mock operator (Sec. 5.1): the two input values are added after a spin of the operator's given
// duration on %globaltimer (at most 100 ms, and a bounded number of sleeps), as the paper's
// artificial operator of fixed or exponentially distributed running time.  left < 0 is the
// identity (0), which the exclusive Blelloch scan feeds in.
__device__ void run_mock(const Params &p, const OpDesc &op, int op_index, const cg::cluster_group &cl)
{
    if (threadIdx.x != 0 || cl.block_rank() != 0) return;
    const double a = op.left >= 0 ? __ldcg(p.node_theta + 3 * op.left) : 0.0;
    const double b = __ldcg(p.node_theta + 3 * op.right);
    const long long dur = (long long)(fminf(fmaxf(p.mock_us[op_index], 0.f), 1.0e5f) * 1000.0f);
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int it = 0; it < (1 << 24); ++it) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if ((long long)(t - t0) >= dur) break;
        __nanosleep(100);
    }
    __stcg(p.node_theta + 3 * op.out, a + b);
    OpStats &st = p.stats[op_index];
    st.i = op.ref;
    st.k = op.tmpl;
    st.status = kDevOk;
    st.energy = a + b;
}

__device__ bool op_valid(const Params &p, const OpDesc &op)
{
    if (p.cfg.mode == kModeMock) {
        auto ok = [&](int n) { return n >= 0 && n < p.n_nodes; };
        return ok(op.out) && ok(op.right) && (op.left < 0 || ok(op.left));
    }
    auto node_ok = [&](int n) { return n >= 0 && n < p.n_nodes; };
    if (p.cfg.mode == REG_NONRIGID && p.cfg.metric == REG_METRIC_H1 && !p.h1q) return false;
    if (op.ref < 0 || op.ref >= p.n_frames || op.tmpl < 0 || op.tmpl >= p.n_frames) return false;
    if (!node_ok(op.out)) return false;
    if (op.left >= 0 && !(node_ok(op.left) && node_ok(op.right))) return false;
    if (op.left < 0 && op.init_node >= 0 && !node_ok(op.init_node)) return false;
    return true;
}

template <int MODE, typename S, int U>
__device__ void run_op(const Params &p, int op_index, Smem &sm, float2 *gbuf, const cg::cluster_group &cl)
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
    else if constexpr (MODE == kModeMock) run_mock(p, op, op_index, cl);
    else run_nonrigid<S, U>(p, op, op_index, sm, gbuf, cl);
}

// Batched launch: cluster q of the grid runs operator op_base + q.  MINB: CTAs per SM the
// register budget is sized for (the nonrigid kernels come in a 3-CTA form without spills and a
// 4-CTA form with a few spilled registers, faster once the clusters are large).  U: pixels in
// flight per lane in the nonrigid energy passes (2 or 4, the tile shape reg_autotune chooses).
template <int MODE, typename S, int MINB, int U = 4>
__global__ void __launch_bounds__(kThreads, MINB) op_kernel(Params p)
{
    __shared__ Smem sm;
    extern __shared__ __align__(16) float2 gbuf[];   // nonrigid: control grid c, d, ct, gp
    cg::cluster_group cl = cg::this_cluster();
    const int q = blockIdx.x / cl.num_blocks();
    run_op<MODE, S, U>(p, p.op_base + q, sm, gbuf, cl);
    cl.sync();   // no CTA leaves while a peer may still read its shared memory
}

// Persistent launch: each cluster claims ready operators from the device queue
// until all n_ops have been claimed.  Every wait is bounded by queue.timeout_ns.
template <int MODE, typename S, int MINB, int U = 4>
__global__ void __launch_bounds__(kThreads, MINB) persistent_kernel(Params p)
{
    __shared__ Smem sm;
    extern __shared__ __align__(16) float2 gbuf[];
    cg::cluster_group cl = cg::this_cluster();
    const bool leader = cl.block_rank() == 0 && threadIdx.x == 0;
    for (;;) {
        if (leader) {
            // claim the first ready operator of the most urgent non-empty class; every operator
            // claimed (all classes): leave.  Waiting for work gives up after queue.timeout_ns
            // without any operator finishing; the wait for a claimed slot's writer is bounded too.
            const Queue &Q = p.queue;
            volatile int *vh = Q.head, *vt = Q.tail, *vs = Q.slots, *vc = Q.claimed, *vd = Q.done;
            unsigned long long start;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(start));
            unsigned ns = 64;
            int op = -1, seen = *vd;
            // the wait has run out once timeout_ns passed with no operator finishing (the finished
            // count is read only then, so spinning workers do not crowd its line), or on an error
            auto wait_expired = [&](unsigned long long now) {
                if (*((volatile int *)p.status) != 0) return true;
                if ((long long)(now - start) <= Q.timeout_ns) return false;
                const int dn = *vd;
                if (dn == seen) return true;
                seen = dn;
                start = now;
                return false;
            };
            // the mock operator's kernel keeps to the FIFO (the class scan's registers would halve its
            // resident CTAs)
            constexpr bool kClassQueue = MODE != kModeMock;
            if (!kClassQueue || Q.n_class == 1) {
                // one class, a plain FIFO: take a ticket, then wait for that slot to be written (the
                // form for short operators, where polling every class's head would crowd one line)
                const int slot = atomicAdd(Q.head, 1);
                while (slot < p.n_ops && (op = vs[slot]) < 0) {
                    unsigned long long now;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                    if (wait_expired(now)) {
                        atomicCAS(p.status, 0, (int)kDevQueueTimeout);
                        op = -2;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 1024) ns *= 2;
                }
            }
            for (; kClassQueue && Q.n_class > 1;) {
                if (*vc >= p.n_ops) break;
                // every class's head and tail in one round of loads; the first class with a ready
                // operator is claimed with an atomic on its head (no compare-and-swap: under
                // contention a worker may draw a slot past the tail, which a later release of that
                // class fills; a draw past the class's last operator is void)
                int hs[kQueueClasses], ts[kQueueClasses];
#pragma unroll
                for (int c = 0; c < kQueueClasses; ++c) hs[c] = c < Q.n_class ? vh[c] : 0;
#pragma unroll
                for (int c = 0; c < kQueueClasses; ++c) ts[c] = c < Q.n_class ? vt[c] : 0;
                int slot = -1;
                bool void_draw = false;
#pragma unroll
                for (int c = 0; c < kQueueClasses; ++c)
                    if (slot < 0 && !void_draw && hs[c] < ts[c]) {
                        const int h = atomicAdd(Q.head + c, 1);
                        if (h < Q.class_off[c + 1] - Q.class_off[c]) slot = Q.class_off[c] + h;
                        else void_draw = true;   // the class is used up: look again at once
                    }
                if (void_draw) continue;
                if (slot >= 0) {
                    atomicAdd(Q.claimed, 1);
                    // the releaser bumps the tail before it writes the slot; a slot drawn past the
                    // tail is written by a later release of its class
                    while ((op = vs[slot]) < 0) {
                        unsigned long long now;
                        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                        if (wait_expired(now)) {
                            atomicCAS(p.status, 0, (int)kDevQueueTimeout);
                            op = -2;
                            break;
                        }
                        __nanosleep(32);
                    }
                    break;
                }
                unsigned long long now;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                if (wait_expired(now)) {
                    atomicCAS(p.status, 0, (int)kDevQueueTimeout);
                    op = -2;
                    break;
                }
                __nanosleep(ns);
                if (ns < 1024) ns *= 2;
            }
            __threadfence();
            sm.idata[1] = op;
        }
        cl.sync();
        const int op = *cl.map_shared_rank(&sm.idata[1], 0);
        cl.sync();
        if (op < 0) break;
        run_op<MODE, S, U>(p, op, sm, gbuf, cl);
        cl.sync();
        if (cl.block_rank() == 0) {
            // publish the produced node and release its consumers, spread over the CTA's threads (a
            // node of a Ladner-Fischer scan has up to n/2 consumers); the lanes of a warp that make
            // consumers of one class ready claim their slots with one atomic on that class's tail
            const int node = p.ops[op].out;
            const int cb = p.queue.cons_start[node], ce = p.queue.cons_start[node + 1];
            const int lane = threadIdx.x & 31;
            // only warps with consumers take part (most nodes have one or two: warp 0 alone); each
            // orders the cluster's writes of the node, seen through cl.sync, before its releases
            if (cb + (int)(threadIdx.x & ~31) < ce) __threadfence();
            for (int base = cb + (int)(threadIdx.x & ~31); base < ce; base += kThreads) {
                const int e = base + lane;
                int c = -1;
                bool ready = false;
                if (e < ce) {
                    c = p.queue.consumers[e];
                    ready = atomicSub(p.queue.pending + c, 1) == 1;
                }
                if (__ballot_sync(0xffffffffu, ready)) {
                    // lanes releasing into the same class take consecutive slots of it
                    const int cls = ready ? p.queue.op_class[c] : -1;
                    const unsigned grp = __match_any_sync(0xffffffffu, cls);
                    if (ready) {
                        const int first = __ffs(grp) - 1;
                        int t0 = 0;
                        if (lane == first) t0 = atomicAdd(p.queue.tail + cls, __popc(grp));
                        t0 = __shfl_sync(grp, t0, first);
                        atomicExch(p.queue.slots + p.queue.class_off[cls] + t0 + __popc(grp & ((1u << lane) - 1)), c);
                    }
                }
            }
            if (threadIdx.x == 0) atomicAdd(p.queue.done, 1);
        }
    }
    cl.sync();
}

// Energy/gradient at a given deformation for a single pair (one cluster of 1 CTA).
// Rigid: theta (device) -> out[0] = E, out[1..3] = dE/dtheta.  Nonrigid: control values cgrid
// (finest px, level 0) -> out[0] = E and grad_c = dE/dc.
template <int MODE, typename S>
__global__ void __launch_bounds__(kThreads) energy_kernel(Params p, const double *theta, const float2 *cgrid,
                                                          double *out, float2 *grad_c)
{
    __shared__ Smem sm;
    extern __shared__ __align__(16) float2 gbuf[];
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x;
    int buf = 0;
    const Lvl L = level_of(p, 0, 1, 0);
    if constexpr (MODE == REG_RIGID) {
        RigidCtl &k = sm.rctl;
        if (tid == 0) memset(&k, 0, sizeof(k));
        __syncthreads();
        k.P = (double)L.W * L.H;
        k.invP = 1.0 / k.P;
        k.th[0] = theta[0]; k.th[1] = theta[1]; k.th[2] = theta[2];
        float pm[10];
        rigid_params(k.th, pm);
        eval_rigid_energy<S, true>(L, 0, L.H, pm, sm, buf, cl);
        if (tid == 0) {
            rigid_step(k, p.cfg, sm.tot, kActEnergy, sm.pm);
            out[0] = k.E;
        }
        __syncthreads();
        for (int q = 0; q < 10; ++q) pm[q] = sm.pm[q];
        eval_rigid_grad<S>(L, 0, L.H, pm, sm, buf, cl);
        if (tid == 0)
            for (int q = 0; q < 3; ++q) out[1 + q] = sm.tot[q] / k.P;
    } else {
        const Grid G{p.gnx, p.gny, p.gs};
        const int Nc = G.nx * G.ny;
        const GridLayout lay = grid_layout(G.nx, G.ny, 1, false);
        float2 *c = gbuf + lay.c, *d = gbuf + lay.d, *mt = gbuf + lay.mt, *gp = gbuf + lay.gp;
        float4 *crow = (float4 *)(gbuf + lay.crow);
        for (int j = tid; j < Nc; j += kThreads) { c[j] = cgrid[j]; mt[j] = make_float2(1.f, 1.f); }
        __syncthreads();
        GridLvl GL;
        GL.W = L.W; GL.H = L.H; GL.l = 0; GL.pl = 1.f; GL.off = 0.f; GL.scale_inv = 1.f / (float)G.s;
        int cr0, cr1, r0, r1;
        grid_rows(G, GL, 0, 1, cr0, cr1, r0, r1);
        grid_energy_pass<S, true, 4, false>(L, G, GL, c, c, 0.f, crow, r0, r1, sm, buf, cl);
        FieldCtl &k = sm.fctl;
        if (tid == 0) {
            memset(&k, 0, sizeof(k));
            k.P = (double)L.W * L.H;
            k.invP = 1.0 / k.P;
            k.Nc = Nc;
            k.invNc = 1.0 / k.Nc;
            k.sr = sm.tot[3]; k.srr = sm.tot[4];
            out[0] = field_energy(k, p.cfg, sm.tot, false);
            field_grad_params(k, p.cfg, sm.pm);
        }
        __syncthreads();
        if (grad_c) {
            float pm[5];
            for (int q = 0; q < 5; ++q) pm[q] = sm.pm[q];
            grid_grad_pass<S, false>(L, G, GL, c, d, mt, gp, pm, cr0, cr1, sm, cl, H1Bufs{});
            // d = -Nc dE/dc (unit scalar product)
            const float s = -1.f / (float)Nc;
            for (int j = tid; j < Nc; j += kThreads) grad_c[j] = make_float2(s * d[j].x, s * d[j].y);
        }
    }
}

// ================================================================== pyramid
// All kernels take a batch of frames (grid.z or grid.x = frame).  Level pointers address pixel
// (0, 0) of frame 0; rows are `pitch` elements apart and frames `stride` elements apart.
// Level 0 in storage type: a CTA of kL0Threads covers kL0Rows rows of kL0Cols columns, each thread
// kL0Rows x (kL0Cols / kL0Threads) samples with every load issued before the first store.
constexpr int kL0Threads = 256, kL0Rows = 4, kL0Cols = 1024;
template <typename S>
__global__ void __launch_bounds__(kL0Threads) pyr_level0(const float *frames, size_t fstride, int W, int H,
                                                         int pitch, S *out, size_t ostride, int opitch)
{
    constexpr int CB = kL0Cols / kL0Threads;
    const int c0 = blockIdx.x * kL0Cols + threadIdx.x, r0 = blockIdx.y * kL0Rows;
    const float *src = frames + blockIdx.z * fstride;
    S *dst = out + blockIdx.z * ostride;
    float v[kL0Rows][CB];
#pragma unroll
    for (int i = 0; i < kL0Rows; ++i)
#pragma unroll
        for (int j = 0; j < CB; ++j) {
            const int r = r0 + i, c = c0 + j * kL0Threads;
            v[i][j] = r < H && c < W ? __ldg(src + (size_t)r * pitch + c) : 0.f;
        }
#pragma unroll
    for (int i = 0; i < kL0Rows; ++i)
#pragma unroll
        for (int j = 0; j < CB; ++j) {
            const int r = r0 + i, c = c0 + j * kL0Threads;
            if (r < H && c < W) dst[(size_t)r * opitch + c] = toS<S>(v[i][j]);
        }
}

// Level l+1 from level l: 2x2 box average, last odd row/column clamped.  A thread makes kDnRows
// samples of one column, every load issued before the first store.
constexpr int kDnThreads = 128, kDnRows = 8;
template <typename S>
__global__ void __launch_bounds__(kDnThreads) pyr_down(const S *src, size_t sstride, int spitch, int W, int H,
                                                       S *dst, size_t dstride, int dpitch)
{
    const int w2 = (W + 1) / 2, h2 = (H + 1) / 2;
    const int c = blockIdx.x * kDnThreads + threadIdx.x, rb = blockIdx.y * kDnRows;
    if (c >= w2) return;
    src += blockIdx.z * sstride;
    dst += blockIdx.z * dstride;
    const int c0 = 2 * c, c1 = min(2 * c + 1, W - 1);
    float v[kDnRows];
#pragma unroll
    for (int k = 0; k < kDnRows; ++k) {
        v[k] = 0.f;
        const int r = rb + k;
        if (r < h2) {
            const int r0 = 2 * r, r1 = min(2 * r + 1, H - 1);
            v[k] = ((ldS<S>(src + (size_t)r0 * spitch + c0) + ldS<S>(src + (size_t)r0 * spitch + c1)) +
                    ldS<S>(src + (size_t)r1 * spitch + c0)) + ldS<S>(src + (size_t)r1 * spitch + c1);
        }
    }
#pragma unroll
    for (int k = 0; k < kDnRows; ++k)
        if (rb + k < h2) dst[(size_t)(rb + k) * dpitch + c] = toS<S>(0.25f * v[k]);
}

// Border of `pad` samples around a W x H level (pitch W + 2 pad) holding the level's mean (frame
// f's at mean[f * mstride]): beyond its border a frame is taken to be its mean.  Thread t covers one
// border sample, the top and bottom bands first, then the left and right bands.
template <typename S>
__global__ void pyr_border(S *lvl, size_t stride, int W, int H, int pad, const float *mean, int mstride)
{
    const int pitch = W + 2 * pad;
    const int bands = 2 * pad * pitch, sides = 2 * pad * H;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= bands + sides) return;
    lvl += blockIdx.z * stride;
    int r, c;
    if (t < bands) {
        const int q = t / pitch;                      // 0 .. 2 pad - 1
        r = q < pad ? q - pad : H + (q - pad);        // -pad .. -1, then H .. H + pad - 1
        c = t - q * pitch - pad;                      // -pad .. W + pad - 1
    } else {
        const int u = t - bands, q = u / H;           // 0 .. 2 pad - 1
        r = u - q * H;
        c = q < pad ? q - pad : W + (q - pad);
    }
    lvl[(ptrdiff_t)r * pitch + c] = toS<S>(mean[(size_t)blockIdx.z * mstride]);
}

// The quadratic B-spline model at the pixel centres: the separable filter (1/8, 3/4, 1/8) of a
// bordered level (its border, the level's mean, supplies the outer taps), with the operations of
// sample_q at a zero offset, so that a frame registered to itself matches bit for bit.  Written
// as a plain W x H level.  A thread walks kSmoothRows rows down one column and carries the
// horizontal filter of the rows above and at the current one, so each output row reads one row
// of three taps.
constexpr int kSmoothRows = 16;
template <typename S>
__global__ void pyr_smooth(const S *src, size_t sstride, int spitch, int W, int H, S *dst, size_t dstride)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r0 = blockIdx.y * kSmoothRows;
    if (c >= W || r0 >= H) return;
    const S *p = src + blockIdx.z * sstride + (ptrdiff_t)r0 * spitch + c;
    S *q = dst + blockIdx.z * dstride + (size_t)r0 * W + c;
    // the horizontal filter of row r0 + k of the bordered level (k = -1 .. kSmoothRows)
    auto hrow = [&](int k) {
        const S *x = p + (ptrdiff_t)k * spitch;
        return fmaf(0.125f, ldS<S>(x + 1), fmaf(0.75f, ldS<S>(x), 0.125f * ldS<S>(x - 1)));
    };
    float a = hrow(-1), b = hrow(0);
#pragma unroll
    for (int k = 0; k < kSmoothRows; ++k) {
        if (r0 + k >= H) break;
        const float d = hrow(k + 1);
        q[(size_t)k * W] = toS<S>(fmaf(0.125f, d, fmaf(0.75f, b, 0.125f * a)));
        a = b;
        b = d;
    }
}

// Mean of one level of each frame (one CTA per frame), deterministic float-float sum.
template <typename S>
__global__ void __launch_bounds__(kThreads) level_mean(const S *img, size_t stride, int W, int H, int pitch,
                                                       float *mean, int mstride)
{
    __shared__ float2 ws[kWarps];
    img += blockIdx.x * stride;
    const int n = W * H;
    float hi = 0.f, lo = 0.f;
    for (int base = 0; base < n; base += kThreads * kChunk) {
        // a thread's kChunk samples of the chunk, loaded first, then summed in index order
        float x[kChunk];
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
            const int i = base + threadIdx.x + k * kThreads;
            x[k] = 0.f;
            if (i < n) {
                const int r = i / W;
                x[k] = ldS<S>(img + (size_t)r * pitch + (i - r * W));
            }
        }
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < kChunk; ++k) a += x[k];
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

// The level means of a freshly built pyramid into its rows of a level table.
__global__ void set_level_means_kernel(LevelDesc *tab, const float *means, int L)
{
    const int l = threadIdx.x;
    if (l < L) tab[l].mean = means[l];
}

cudaError_t launch_set_level_means(LevelDesc *tab, const float *means, int L, cudaStream_t s)
{
    set_level_means_kernel<<<1, 32, 0, s>>>(tab, means, L);
    return cudaGetLastError();
}

// Composition of two control grids at the control points (standalone entry point).
__global__ void grid_compose_kernel(const float2 *q1, const float2 *q2, Grid G, float2 *out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= G.nx * G.ny) return;
    const int jy = j / G.nx, jx = j - jy * G.nx;
    const float2 a = q1[j];
    const float2 u = grid_eval_global(q2, G, (float)(jx * G.s) + a.x, (float)(jy * G.s) + a.y);
    out[j] = make_float2(a.x + u.x, a.y + u.y);
}

// Dense finest-level fields [2][H][W] of control grids (grid nodes[blockIdx.z]), four pixels per
// thread written with one float4 store per plane where the row allows it.
__global__ void grid_dense_kernel(const float2 *grids, const int *nodes, Grid G, int W, int H, float *out)
{
    const int Nc = G.nx * G.ny;
    const float2 *q = grids + (size_t)Nc * nodes[blockIdx.z];
    float *ox = out + (size_t)blockIdx.z * 2 * W * H, *oy = ox + (size_t)W * H;
    const int r = blockIdx.y, c0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (c0 >= W) return;
    float vx[4], vy[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float2 u = grid_eval_global(q, G, (float)min(c0 + t, W - 1), (float)r);
        vx[t] = u.x;
        vy[t] = u.y;
    }
    const size_t i = (size_t)r * W + c0;
    if (c0 + 3 < W && (((size_t)(ox + i) | (size_t)(oy + i)) & 15) == 0) {
        __stcs((float4 *)(ox + i), make_float4(vx[0], vx[1], vx[2], vx[3]));
        __stcs((float4 *)(oy + i), make_float4(vy[0], vy[1], vy[2], vy[3]));
    } else {
        for (int t = 0; t < 4 && c0 + t < W; ++t) { ox[i + t] = vx[t]; oy[i + t] = vy[t]; }
    }
}

// Control values sampled from a dense finest-level field [2][H][W] (clamped at the border).
__global__ void grid_from_dense_kernel(const float *u, int W, int H, Grid G, float2 *out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= G.nx * G.ny) return;
    const int jy = j / G.nx, jx = j - jy * G.nx;
    const int x = min(jx * G.s, W - 1), y = min(jy * G.s, H - 1);
    out[j] = make_float2(u[(size_t)y * W + x], u[(size_t)W * H + (size_t)y * W + x]);
}

// ================================================================== host launchers
template <typename S>
static cudaError_t pyramid_t(const float *frames, int N, size_t fstride, int W, int H, int pitch, int levels,
                             const PyrOut &o, float *means, cudaStream_t s)
{
    S *lv[kMaxLevels];
    int w = W, h = H;
    for (int l = 0; l < levels; ++l) {
        lv[l] = (S *)o.raw[l] + level_origin(w, o.pad);
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    pyr_level0<S><<<dim3((W + kL0Cols - 1) / kL0Cols, (H + kL0Rows - 1) / kL0Rows, N), kL0Threads, 0, s>>>(
        frames, fstride, W, H, pitch, lv[0], o.raw_stride[0], level_pitch(W, o.pad));
    w = W; h = H;
    for (int l = 0; l + 1 < levels; ++l) {
        int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
        pyr_down<S><<<dim3((w2 + kDnThreads - 1) / kDnThreads, (h2 + kDnRows - 1) / kDnRows, N), kDnThreads, 0, s>>>(
            lv[l], o.raw_stride[l], level_pitch(w, o.pad), w, h, lv[l + 1], o.raw_stride[l + 1], level_pitch(w2, o.pad));
        w = w2; h = h2;
    }
    w = W; h = H;
    for (int l = 0; l < levels; ++l) {
        if (means)
            level_mean<S><<<N, kThreads, 0, s>>>(lv[l], o.raw_stride[l], w, h, level_pitch(w, o.pad), means + l,
                                                 levels);
        if (o.pad > 0) {
            const int nb = 2 * o.pad * level_pitch(w, o.pad) + 2 * o.pad * h;
            pyr_border<S><<<dim3((nb + 127) / 128, 1, N), 128, 0, s>>>(lv[l], o.raw_stride[l], w, h, o.pad,
                                                                       means + l, levels);
            if (o.smooth[l])
                pyr_smooth<S><<<dim3((w + 127) / 128, (h + kSmoothRows - 1) / kSmoothRows, N), 128, 0, s>>>(
                    lv[l], o.raw_stride[l], level_pitch(w, o.pad), w, h, (S *)o.smooth[l], o.smooth_stride[l]);
        }
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    return cudaGetLastError();
}

cudaError_t launch_pyramid(const float *frames, int N, size_t fstride, int W, int H, int pitch, int levels,
                           int storage, const PyrOut &out, float *means, cudaStream_t s)
{
    if (out.pad != 0) {
        // the smoothed levels read the 3x3 window of a bordered level; the border holds the mean
        if (out.pad < 1 || !means) return cudaErrorInvalidValue;
    } else {
        for (int l = 0; l < levels; ++l)
            if (out.smooth[l]) return cudaErrorInvalidValue;
    }
    switch (storage) {
    case REG_F32: return pyramid_t<float>(frames, N, fstride, W, H, pitch, levels, out, means, s);
    case REG_BF16: return pyramid_t<__nv_bfloat16>(frames, N, fstride, W, H, pitch, levels, out, means, s);
    case REG_F16: return pyramid_t<__half>(frames, N, fstride, W, H, pitch, levels, out, means, s);
    }
    return cudaErrorInvalidValue;
}

// Dynamic shared memory of the nonrigid kernels (layout of grid_layout).
static size_t grid_smem(const Params &p, int cluster)
{
    if (p.cfg.mode != REG_NONRIGID) return 0;
    return sizeof(float2) * (size_t)grid_layout(p.gnx, p.gny, cluster, p.cfg.metric == REG_METRIC_H1).crow +
           sizeof(float4) * (size_t)kWarps * (p.gnx - 1);
}

template <typename K>
static cudaError_t launch_cluster(K kernel, int blocks, int cluster, cudaStream_t s, const Params &p)
{
    if (cluster > 8) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = grid_smem(p, cluster);
    if (smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(blocks);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = smem;
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

typedef void (*OpKernelFn)(Params);

// The nonrigid kernel for a storage type, launch form, register form and energy-pass unroll.
template <typename S>
static OpKernelFn nonrigid_fn(bool persistent, bool minb4, int unroll)
{
    const bool u2 = unroll == 2;
    if (persistent) {
        if (minb4) return u2 ? persistent_kernel<REG_NONRIGID, S, 4, 2> : persistent_kernel<REG_NONRIGID, S, 4, 4>;
        return u2 ? persistent_kernel<REG_NONRIGID, S, 3, 2> : persistent_kernel<REG_NONRIGID, S, 3, 4>;
    }
    if (minb4) return u2 ? op_kernel<REG_NONRIGID, S, 4, 2> : op_kernel<REG_NONRIGID, S, 4, 4>;
    return u2 ? op_kernel<REG_NONRIGID, S, 3, 2> : op_kernel<REG_NONRIGID, S, 3, 4>;
}

static OpKernelFn nonrigid_kernel(int storage, bool persistent, bool minb4, int unroll)
{
    switch (storage) {
    case REG_F32: return nonrigid_fn<float>(persistent, minb4, unroll);
    case REG_BF16: return nonrigid_fn<__nv_bfloat16>(persistent, minb4, unroll);
    case REG_F16: return nonrigid_fn<__half>(persistent, minb4, unroll);
    }
    return nullptr;
}

cudaError_t launch_ops(const Params &p, int storage, int cluster, int n_launch_ops, cudaStream_t s)
{
    const bool minb4 = p.minb > 0 ? p.minb == 4 : cluster >= 16;   // nonrigid register form
    const int blocks = n_launch_ops * cluster;
    if (p.cfg.mode == kModeMock) return launch_cluster(op_kernel<kModeMock, float, 8>, blocks, cluster, s, p);
    if (p.cfg.mode == REG_RIGID) {
        switch (storage) {
        case REG_F32: return launch_cluster(op_kernel<REG_RIGID, float, 4>, blocks, cluster, s, p);
        case REG_BF16: return launch_cluster(op_kernel<REG_RIGID, __nv_bfloat16, 4>, blocks, cluster, s, p);
        case REG_F16: return launch_cluster(op_kernel<REG_RIGID, __half, 4>, blocks, cluster, s, p);
        }
    } else {
        OpKernelFn k = nonrigid_kernel(storage, false, minb4, p.unroll);
        if (k) return launch_cluster(k, blocks, cluster, s, p);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_persistent(const Params &p, int storage, int cluster, int workers, cudaStream_t s)
{
    const bool minb4 = p.minb > 0 ? p.minb == 4 : cluster >= 16;   // nonrigid register form
    const int blocks = workers * cluster;
    if (p.cfg.mode == kModeMock) return launch_cluster(persistent_kernel<kModeMock, float, 8>, blocks, cluster, s, p);
    if (p.cfg.mode == REG_RIGID) {
        switch (storage) {
        case REG_F32: return launch_cluster(persistent_kernel<REG_RIGID, float, 4>, blocks, cluster, s, p);
        case REG_BF16: return launch_cluster(persistent_kernel<REG_RIGID, __nv_bfloat16, 4>, blocks, cluster, s, p);
        case REG_F16: return launch_cluster(persistent_kernel<REG_RIGID, __half, 4>, blocks, cluster, s, p);
        }
    } else {
        OpKernelFn k = nonrigid_kernel(storage, true, minb4, p.unroll);
        if (k) return launch_cluster(k, blocks, cluster, s, p);
    }
    return cudaErrorInvalidValue;
}

template <typename K>
static int resident_clusters(K kernel, int cluster, const Params &p)
{
    if (cluster > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return -1;
    const size_t smem = grid_smem(p, cluster);
    if (smem > 0 && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cluster);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &lc) != cudaSuccess) return -1;
    return n;
}

int persistent_resident_clusters(const Params &p, int storage, int cluster)
{
    const bool minb4 = p.minb > 0 ? p.minb == 4 : cluster >= 16;   // nonrigid register form
    int n = -1;
    if (p.cfg.mode == kModeMock) {
        n = resident_clusters(persistent_kernel<kModeMock, float, 8>, cluster, p);
    } else if (p.cfg.mode == REG_RIGID) {
        switch (storage) {
        case REG_F32: n = resident_clusters(persistent_kernel<REG_RIGID, float, 4>, cluster, p); break;
        case REG_BF16: n = resident_clusters(persistent_kernel<REG_RIGID, __nv_bfloat16, 4>, cluster, p); break;
        case REG_F16: n = resident_clusters(persistent_kernel<REG_RIGID, __half, 4>, cluster, p); break;
        }
    } else {
        OpKernelFn k = nonrigid_kernel(storage, true, minb4, p.unroll);
        if (k) n = resident_clusters(k, cluster, p);
    }
    if (n < 0) cudaGetLastError();
    return n;
}

cudaError_t launch_energy(const Params &p, int storage, const double *theta_dev, const float2 *grid_dev,
                          double *out_dev, float2 *grad_dev, cudaStream_t s)
{
    (void)storage;
    const size_t smem = grid_smem(p, 1);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(1);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (p.cfg.mode == REG_RIGID)
        return cudaLaunchKernelEx(&lc, energy_kernel<REG_RIGID, float>, p, theta_dev, grid_dev, out_dev, grad_dev);
    cudaError_t e = cudaFuncSetAttribute(energy_kernel<REG_NONRIGID, float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&lc, energy_kernel<REG_NONRIGID, float>, p, theta_dev, grid_dev, out_dev, grad_dev);
}

cudaError_t launch_grid_compose(const float2 *q1, const float2 *q2, int nx, int ny, int spacing, float2 *out,
                                cudaStream_t s)
{
    const int Nc = nx * ny;
    grid_compose_kernel<<<(Nc + 127) / 128, 128, 0, s>>>(q1, q2, Grid{nx, ny, spacing}, out);
    return cudaGetLastError();
}

cudaError_t launch_grid_dense(const float2 *grids, const int *nodes, int n, int nx, int ny, int spacing, int W,
                              int H, float *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    dim3 grid((W / 4 + 1 + 63) / 64, H, n);
    grid_dense_kernel<<<grid, 64, 0, s>>>(grids, nodes, Grid{nx, ny, spacing}, W, H, out);
    return cudaGetLastError();
}

cudaError_t launch_grid_from_dense(const float *u, int W, int H, int nx, int ny, int spacing, float2 *out,
                                   cudaStream_t s)
{
    const int Nc = nx * ny;
    grid_from_dense_kernel<<<(Nc + 127) / 128, 128, 0, s>>>(u, W, H, Grid{nx, ny, spacing}, out);
    return cudaGetLastError();
}

int max_cluster_size() { return 16; }

}  // namespace reg
