// Registered series (reg_warp): every frame resampled onto the first frame's pixel grid by
// its prefix deformation phi_{0,k}, out_k(x) = f_k(phi_{0,k}(x)), and the mean of the
// registered series [Sec. 2: the series is registered to its first frame and averaged].
//
// The kernel is bound by HBM: each frame is read once and (optionally) written once.
// A block owns a 64 x 32 output tile and walks a chunk of frames, warp-specialised: a
// producer warp computes, for each frame, the source box the tile's samples can touch (from
// the rigid parameters, or from the min/max of the control values of the cells under the
// tile: bilinear interpolation is a convex combination, so the field over a cell lies between
// its corner values) and issues a TMA load of an 80 x 40 box of the frame into a 4-stage
// shared-memory ring; eight consumer warps sample from the ring.  Full/empty mbarriers with
// bounded waits hand the stages back and forth, so no block-wide barrier sits in the frame
// loop.  A frame whose box does not fit (a large rotation or a strongly varying field under
// the tile) is sampled from global memory instead.  Per-pixel sums of the chunk go to a
// partial buffer (FP32 runs of 16 frames folded into float-float); a second kernel adds the
// chunks in a fixed order and scales by 1/N, so the mean does not depend on the launch shape.
#include <cuda.h>   // CUtensorMap and the tensor-map encoder's types (resolved at run time)

#include <cstring>
#include <mutex>

#include "reg_f2.cuh"
#include "reg_internal.h"

namespace reg {
namespace {

constexpr int kTW = 64, kTH = 32;          // output tile
constexpr int kBW = 80, kBH = 40;          // staged source box (tile + margins; kBW % 4 == 0)
constexpr int kStages = 4;
constexpr int kConsumers = 8;              // consumer warps; one more warp produces
constexpr int kRun = 16;                   // frames summed in FP32 before the float-float fold
constexpr int kWinX = 12, kWinY = 8;       // control points under a tile (spacing >= 8)
constexpr int kWThreads = 32 * (kConsumers + 1);
constexpr unsigned kBoxBytes = kBW * kBH * 4;
constexpr unsigned kMaxTap = kBW * kBH - kBW - 2;   // largest top-left tap index in a box

// How a (frame, tile) is sampled.
enum : int {
    kGlobal = 0,          // from global memory with the full clamp logic (box does not fit)
    kStagedClamped = 1,   // from the staged box, samples may reach the frame edge
    kInterior = 2         // from the staged box, every sample strictly inside the frame
};

struct WarpArgs {
    const float *frames;
    int N, W, H, pitch;
    int mode;
    const float4 *rigid;       // per frame: cos(a) - 1, sin(a), gx, gy (frame 0: identity)
    const float2 *grids;       // nonrigid: frames 1..N-1, [ny][nx] each
    int nx, ny, s;
    float inv_s;
    int window;                // control window staged in shared memory (spacing >= 8)
    float *out;                // [N][H][W] or null
    float2 *part;              // [chunks][H][W] compensated sums, or null
    int chunk;                 // frames per chunk
    int *status;
    int use_tma;
    long long timeout_ns;
};

struct __align__(128) WarpSmem {
    float buf[kStages][kBH * kBW];
    unsigned long long full[kStages];    // producer -> consumers: parameters written, box landed
    unsigned long long empty[kStages];   // consumers -> producer: stage read by all consumer warps
    int2 org[kStages];
    int fit[kStages];
    float4 rp[kStages];
    float2 win[kStages][kWinY * kWinX];  // control points under the tile
    float2 xint[kStages][kWinY][kTW];   // control rows of the window interpolated along x at each tile column
    int2 wo[kStages];
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ long long gtime()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the mbarrier completes the phase of parity `ph`; false after timeout_ns.
__device__ bool mbar_wait(uint32_t bar, uint32_t ph, long long timeout_ns)
{
    long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(ph)
            : "memory");
        if (done) return true;
        if ((it & 31) == 0) {
            const long long t = gtime();
            if (it == 0) t0 = t;
            else if (t - t0 > timeout_ns) return false;
        }
    }
}

__device__ __forceinline__ int cell_of(float gf, int n)
{
    return min((int)gf, n - 2);
}

// Control points under the tile (x0, y0): first cell column / row and the point counts.
struct Window {
    int cx0, cy0, wx, wy;
};

__device__ __forceinline__ Window window_of(const WarpArgs &a, int x0, int y0)
{
    const int x1 = min(x0 + kTW, a.W) - 1, y1 = min(y0 + kTH, a.H) - 1;
    Window w;
    w.cx0 = cell_of(fminf((float)x0 * a.inv_s, (float)(a.nx - 1)), a.nx);
    w.cy0 = cell_of(fminf((float)y0 * a.inv_s, (float)(a.ny - 1)), a.ny);
    w.wx = cell_of(fminf((float)x1 * a.inv_s, (float)(a.nx - 1)), a.nx) + 2 - w.cx0;   // <= kWinX for spacing >= 8
    w.wy = cell_of(fminf((float)y1 * a.inv_s, (float)(a.ny - 1)), a.ny) + 2 - w.cy0;   // <= kWinY
    return w;
}

// What the producer needs from global memory for one frame, loaded a frame ahead so that the
// load latency overlaps the previous frame's work: the rigid parameters, or this lane's share
// (up to 3 points) of the control window.
struct Prefetch {
    float4 q;
    float2 v[3];
};

__device__ __forceinline__ Prefetch fetch(const WarpArgs &a, const Window &w, int k)
{
    Prefetch f;
    const int lane = threadIdx.x & 31;
    if (a.mode == REG_RIGID) {
        f.q = a.rigid[k];
        return f;
    }
    f.q = make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 *g = k > 0 ? a.grids + (size_t)(k - 1) * a.nx * a.ny : nullptr;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int j = lane + 32 * t;
        f.v[t] = make_float2(0.f, 0.f);
        if (a.window && g && j < w.wx * w.wy) {
            const int jy = j / w.wx, jx = j - jy * w.wx;
            f.v[t] = g[(size_t)(w.cy0 + jy) * a.nx + w.cx0 + jx];
        }
    }
    return f;
}

// Warp 0: stage the parameters of frame k for the tile (x0, y0) into ring slot st and start
// the TMA load of its source box.
__device__ void prepare(const WarpArgs &a, const CUtensorMap *tmap, WarpSmem &sm, int k, int st, int x0, int y0,
                        const Window &win, const Prefetch &f)
{
    const int lane = threadIdx.x & 31;
    const int x1 = min(x0 + kTW, a.W) - 1, y1 = min(y0 + kTH, a.H) - 1;
    float pxlo, pxhi, pylo, pyhi;
    if (a.mode == REG_RIGID) {
        const float4 q = f.q;
        const float cx = 0.5f * (float)(a.W - 1), cy = 0.5f * (float)(a.H - 1);
        pxlo = pylo = 3.0e38f;
        pxhi = pyhi = -3.0e38f;
        for (int c = 0; c < 4; ++c) {
            const float xx = (float)((c & 1) ? x1 : x0), yy = (float)((c & 2) ? y1 : y0);
            const float xc = xx - cx, yc = yy - cy;
            float vx = fmaf(q.x, xc, fmaf(-q.y, yc, q.z)), vy = fmaf(q.y, xc, fmaf(q.x, yc, q.w));
            vx = fminf(fmaxf(vx, -1.0e6f), 1.0e6f);
            vy = fminf(fmaxf(vy, -1.0e6f), 1.0e6f);
            pxlo = fminf(pxlo, xx + vx); pxhi = fmaxf(pxhi, xx + vx);
            pylo = fminf(pylo, yy + vy); pyhi = fmaxf(pyhi, yy + vy);
        }
        if (lane == 0) sm.rp[st] = q;
    } else {
        float uxlo = 0.f, uxhi = 0.f, uylo = 0.f, uyhi = 0.f;
        if (a.window) {
            const int cx0 = win.cx0, cy0 = win.cy0, wx = win.wx, wy = win.wy;
            uxlo = uylo = 3.0e38f;
            uxhi = uyhi = -3.0e38f;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int j = lane + 32 * t;
                if (j < wx * wy) {
                    const int jy = j / wx, jx = j - jy * wx;
                    const float2 v = f.v[t];
                    sm.win[st][jy * kWinX + jx] = v;
                    uxlo = fminf(uxlo, v.x); uxhi = fmaxf(uxhi, v.x);
                    uylo = fminf(uylo, v.y); uyhi = fmaxf(uyhi, v.y);
                }
            }
            // each window control row interpolated along x at the tile's columns (a column past
            // the frame edge uses the last one), so a consumer pixel only interpolates along y
            __syncwarp();
#pragma unroll 4
            for (int j = lane; j < wy * kTW; j += 32) {
                const int jy = j / kTW, col = j - jy * kTW;
                const int c = min(x0 + col, a.W - 1);
                const float gxf = fminf((float)c * a.inv_s, (float)(a.nx - 1));
                const int ix = cell_of(gxf, a.nx);
                const float2 *q = sm.win[st] + jy * kWinX + (ix - cx0);
                const float2 p0 = q[0], p1 = q[1];
                sm.xint[st][jy][col] = __ffma2_rn(f2(gxf - (float)ix), f2sub(p1, p0), p0);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                uxlo = fminf(uxlo, __shfl_xor_sync(0xffffffffu, uxlo, o));
                uxhi = fmaxf(uxhi, __shfl_xor_sync(0xffffffffu, uxhi, o));
                uylo = fminf(uylo, __shfl_xor_sync(0xffffffffu, uylo, o));
                uyhi = fmaxf(uyhi, __shfl_xor_sync(0xffffffffu, uyhi, o));
            }
            if (lane == 0) sm.wo[st] = make_int2(cx0, cy0);
        } else {
            uxlo = uylo = -1.0e6f;   // no bound without the window: sample from global memory
            uxhi = uyhi = 1.0e6f;
        }
        uxlo = fmaxf(uxlo, -1.0e6f); uxhi = fminf(uxhi, 1.0e6f);
        uylo = fmaxf(uylo, -1.0e6f); uyhi = fminf(uyhi, 1.0e6f);
        pxlo = (float)x0 + uxlo; pxhi = (float)x1 + uxhi;
        pylo = (float)y0 + uylo; pyhi = (float)y1 + uyhi;
    }
    __syncwarp();   // the window written by every lane is ordered before lane 0's arrive
    if (lane == 0) {
        // taps the samples can read: cells floor(p) clamped to [0, W-2] and their right/lower
        // neighbours, widened by one pixel against rounding in the per-pixel arithmetic
        const int nxlo = max(0, min((int)floorf(pxlo), a.W - 2) - 1);
        const int nxhi = min(a.W - 1, max(0, min((int)floorf(pxhi), a.W - 2)) + 2);
        const int nylo = max(0, min((int)floorf(pylo), a.H - 2) - 1);
        const int nyhi = min(a.H - 1, max(0, min((int)floorf(pyhi), a.H - 2)) + 2);
        const int ox = nxlo & ~3;   // TMA: the innermost coordinate x 4 bytes must be 16-byte aligned
        const int oy = nylo;
        sm.org[st] = make_int2(ox, oy);
        const bool fit = a.use_tma && (nxhi - ox < kBW) && (nyhi - oy < kBH);
        // interior: every sample lies at least one pixel inside the frame, so no edge clamp
        // (and no cell clamp at W-2) can apply
        const bool interior = pxlo >= 1.f && pxhi <= (float)(a.W - 2) && pylo >= 1.f && pyhi <= (float)(a.H - 2);
        sm.fit[st] = fit ? (interior ? kInterior : kStagedClamped) : kGlobal;
        const uint32_t bar = smem_u32(&sm.full[st]);
        if (a.use_tma) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBoxBytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];" ::"r"(smem_u32(sm.buf[st])),
                "l"((unsigned long long)tmap), "r"(ox), "r"(oy), "r"(k), "r"(bar)
                : "memory");
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
        }
    }
}

// Bilinear value at (c + vx, r + vy), clamp-to-edge, cell floor(p) clamped to [0, W-2].
__device__ __forceinline__ float sample(const WarpArgs &a, const WarpSmem &sm, int st, bool fit, const float *frame,
                                        int c, int r, float vx, float vy)
{
    vx = fminf(fmaxf(vx, -1.0e6f), 1.0e6f);
    vy = fminf(fmaxf(vy, -1.0e6f), 1.0e6f);
    const float flx = floorf(vx), fly = floorf(vy);
    int x = c + (int)flx, y = r + (int)fly;
    float fx = vx - flx, fy = vy - fly;
    if (x < 0) { x = 0; fx = 0.f; }
    else if (x > a.W - 2) { x = a.W - 2; fx = 1.f; }
    if (y < 0) { y = 0; fy = 0.f; }
    else if (y > a.H - 2) { y = a.H - 2; fy = 1.f; }
    float t00, t01, t10, t11;
    if (fit) {
        const int sx = min(max(x - sm.org[st].x, 0), kBW - 2), sy = min(max(y - sm.org[st].y, 0), kBH - 2);
        const float *b = sm.buf[st] + sy * kBW + sx;
        t00 = b[0]; t01 = b[1]; t10 = b[kBW]; t11 = b[kBW + 1];
    } else {
        const float *b = frame + (size_t)y * a.pitch + x;
        t00 = __ldg(b); t01 = __ldg(b + 1); t10 = __ldg(b + a.pitch); t11 = __ldg(b + a.pitch + 1);
    }
    // (1 - f) a + f b as f b + (a - f a): exact at f = 0 and f = 1, so integer positions
    // (the identity, whole-pixel shifts, the clamped edge) return pixel values unchanged
    const float top = fmaf(fx, t01, fmaf(-fx, t00, t00)), bot = fmaf(fx, t11, fmaf(-fx, t10, t10));
    return fmaf(fy, bot, fmaf(-fy, top, top));
}

// Per-thread pixel columns: c0 = x0 + lane and c1 = c0 + 32, processed as one float2 pair.
struct Cols {
    int c0, c1;                // clamped to the last column; in0/in1 say which are real
    int col0, col1;            // the same columns relative to the tile's first one
    bool in0, in1;
    float2 xc;                 // rigid: columns relative to the rotation centre
    int ix0, ix1;              // nonrigid: control cell of each column
    float2 wx;                 //           and the weight along x
};

// The two pixels' displacements on row r of frame slot st.
template <int MODE, bool WINDOW>
__device__ __forceinline__ void displacement(const WarpArgs &a, const WarpSmem &sm, int st, int k, const Cols &cl,
                                             int r, float2 &vx, float2 &vy)
{
    if (MODE == REG_RIGID) {
        const float4 q = sm.rp[st];
        const float yc = (float)r - 0.5f * (float)(a.H - 1);
        vx = __ffma2_rn(f2(q.x), cl.xc, f2(fmaf(-q.y, yc, q.z)));
        vy = __ffma2_rn(f2(q.y), cl.xc, f2(fmaf(q.x, yc, q.w)));
    } else {
        const float gyf = fminf((float)r * a.inv_s, (float)(a.ny - 1));
        const int iy = cell_of(gyf, a.ny);
        const float2 wy = f2(gyf - (float)iy);
        float2 u[2];
        if constexpr (WINDOW) {
            // x-interpolated control rows iy, iy + 1 at this lane's two columns
            const float2 *t = sm.xint[st][iy - sm.wo[st].y], *b = sm.xint[st][iy - sm.wo[st].y + 1];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = h ? cl.col1 : cl.col0;
                const float2 tv = t[col], bv = b[col];
                u[h] = __ffma2_rn(wy, f2sub(bv, tv), tv);
            }
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ix = h ? cl.ix1 : cl.ix0;
                float2 p00, p01, p10, p11;
                if (k > 0) {
                    const float2 *g = a.grids + (size_t)(k - 1) * a.nx * a.ny + (size_t)iy * a.nx + ix;
                    p00 = g[0]; p01 = g[1]; p10 = g[a.nx]; p11 = g[a.nx + 1];
                } else {
                    p00 = p01 = p10 = p11 = make_float2(0.f, 0.f);
                }
                const float2 wx = f2(h ? cl.wx.y : cl.wx.x);
                const float2 top = __ffma2_rn(wx, f2sub(p01, p00), p00), bot = __ffma2_rn(wx, f2sub(p11, p10), p10);
                u[h] = __ffma2_rn(wy, f2sub(bot, top), top);
            }
        }
        vx = make_float2(u[0].x, u[1].x);
        vy = make_float2(u[0].y, u[1].y);
    }
}

// Sample the two pixels of a row from the staged box (KIND kInterior or kStagedClamped).
// sx, sy: sample positions in box coordinates.
template <int KIND>
__device__ __forceinline__ float2 staged_pair(const WarpArgs &a, const WarpSmem &sm, int st, float2 sx, float2 sy)
{
    float2 fl, gl;
    if (KIND == kStagedClamped) {
        // clamp to the frame (box coordinates of columns 0 .. W-1), cell at most W-2
        const int2 org = sm.org[st];
        const float xlo = (float)(-org.x), xhi = (float)(a.W - 1 - org.x);
        const float ylo = (float)(-org.y), yhi = (float)(a.H - 1 - org.y);
        sx = make_float2(fminf(fmaxf(sx.x, xlo), xhi), fminf(fmaxf(sx.y, xlo), xhi));
        sy = make_float2(fminf(fmaxf(sy.x, ylo), yhi), fminf(fmaxf(sy.y, ylo), yhi));
        fl = make_float2(fminf(floorf(sx.x), xhi - 1.f), fminf(floorf(sx.y), xhi - 1.f));
        gl = make_float2(fminf(floorf(sy.x), yhi - 1.f), fminf(floorf(sy.y), yhi - 1.f));
    } else {
        fl = make_float2(floorf(sx.x), floorf(sx.y));
        gl = make_float2(floorf(sy.x), floorf(sy.y));
    }
    const float2 fx = f2sub(sx, fl), fy = f2sub(sy, gl);
    // top-left tap of each pixel; the unsigned clamp keeps any index inside the box
    const unsigned i0 = min((unsigned)__float2int_rn(fmaf(gl.x, (float)kBW, fl.x)), kMaxTap);
    const unsigned i1 = min((unsigned)__float2int_rn(fmaf(gl.y, (float)kBW, fl.y)), kMaxTap);
    const float *b = sm.buf[st];
    const float2 t00 = make_float2(b[i0], b[i1]), t01 = make_float2(b[i0 + 1], b[i1 + 1]);
    const float2 t10 = make_float2(b[i0 + kBW], b[i1 + kBW]), t11 = make_float2(b[i0 + kBW + 1], b[i1 + kBW + 1]);
    if (KIND == kStagedClamped) {
        // (1 - f) a + f b as f b + (a - f a): exact at f = 1 (the clamped last cell)
        const float2 nfx = f2sub(fl, sx), nfy = f2sub(gl, sy);
        const float2 top = __ffma2_rn(fx, t01, __ffma2_rn(nfx, t00, t00));
        const float2 bot = __ffma2_rn(fx, t11, __ffma2_rn(nfx, t10, t10));
        return __ffma2_rn(fy, bot, __ffma2_rn(nfy, top, top));
    }
    // interior: f < 1, and a + f (b - a) is exact at f = 0
    const float2 top = __ffma2_rn(fx, f2sub(t01, t00), t00), bot = __ffma2_rn(fx, f2sub(t11, t10), t10);
    return __ffma2_rn(fy, f2sub(bot, top), top);
}

// One frame of the tile for one consumer warp: rows warp, warp + 8, warp + 16, warp + 24.
template <int MODE, bool WINDOW, int KIND>
__device__ __forceinline__ void tile_frame(const WarpArgs &a, const WarpSmem &sm, int st, int k, const Cols &cl,
                                           int y0, float2 (&run)[4])
{
    const int warp = threadIdx.x >> 5;
    const float *frame = a.frames + (size_t)k * a.H * a.pitch;
    float *o = a.out ? a.out + (size_t)k * a.H * a.W : nullptr;
    const int2 org = sm.org[st];
    const float2 colx = make_float2((float)(cl.c0 - org.x), (float)(cl.c1 - org.x));
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = y0 + warp + 8 * j;
        if (r >= a.H) continue;
        float2 vx, vy;
        displacement<MODE, WINDOW>(a, sm, st, k, cl, r, vx, vy);
        float2 v;
        if (KIND == kGlobal) {
            v.x = sample(a, sm, st, false, frame, cl.c0, r, vx.x, vy.x);
            v.y = sample(a, sm, st, false, frame, cl.c1, r, vx.y, vy.y);
        } else {
            v = staged_pair<KIND>(a, sm, st, __fadd2_rn(vx, colx), __fadd2_rn(vy, f2((float)(r - org.y))));
        }
        if (o) {
            if (cl.in0) o[(size_t)r * a.W + cl.c0] = v.x;
            if (cl.in1) o[(size_t)r * a.W + cl.c1] = v.y;
        }
        run[j] = __fadd2_rn(run[j], v);
    }
}

// Fold an FP32 run into the float-float sums (hi, lo): TwoSum of hi and the run, error into lo.
__device__ __forceinline__ void fold(float2 &hi, float2 &lo, float2 &run)
{
    const float2 s = __fadd2_rn(hi, run);
    const float2 bp = f2sub(s, hi);
    const float2 err = __fadd2_rn(f2sub(hi, f2sub(s, bp)), f2sub(run, bp));
    hi = s;
    lo = __fadd2_rn(lo, err);
    run = make_float2(0.f, 0.f);
}

template <int MODE, bool WINDOW>
__global__ void __launch_bounds__(kWThreads, 3) warp_kernel(const WarpArgs a, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    WarpSmem &sm = *reinterpret_cast<WarpSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = (a.W + kTW - 1) / kTW;
    const int x0 = (blockIdx.x % tiles_x) * kTW, y0 = (blockIdx.x / tiles_x) * kTH;
    const int kb = blockIdx.y * a.chunk, ke = min(a.N, kb + a.chunk);
    const int n = ke - kb;
    if (tid == 0) {
        sm.abort = 0;
        for (int st = 0; st < kStages; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.full[st])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.empty[st])), "r"(kConsumers)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int *abort = &sm.abort;

    if (warp == kConsumers) {
        // ---- producer: parameters and the TMA load of each frame, up to kStages ahead
        int issued = 0;
        const Window win = window_of(a, x0, y0);
        Prefetch cur = fetch(a, win, kb);
        for (int i = 0; i < n; ++i) {
            const int st = i % kStages;
            Prefetch nxt = cur;
            if (i + 1 < n) nxt = fetch(a, win, kb + i + 1);   // in flight while this frame is prepared
            if (i >= kStages) {
                // every lane acquires: lane 0 reuses the box, all lanes rewrite the window
                const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&sm.empty[st]),
                                                                  (uint32_t)(((i / kStages) + 1) & 1), a.timeout_ns));
                if (!ok) {
                    if (lane == 0) { atomicExch(a.status, kDevWaitTimeout); *abort = 1; }
                    break;
                }
            }
            if (*abort) break;
            prepare(a, &tmap, sm, kb + i, st, x0, y0, win, cur);
            issued = i + 1;
            cur = nxt;
        }
        __syncthreads();
        if (*abort && lane == 0 && a.use_tma) {
            // let the loads still in flight land before the block's shared memory is released
            for (int j = max(0, issued - kStages); j < issued; ++j)
                mbar_wait(smem_u32(&sm.full[j % kStages]), (uint32_t)((j / kStages) & 1), a.timeout_ns);
        }
        return;
    }

    // ---- consumers
    Cols cl;   // a column past the frame edge samples the last one; it is neither stored nor summed
    cl.in0 = x0 + lane < a.W;
    cl.in1 = x0 + lane + 32 < a.W;
    cl.c0 = min(x0 + lane, a.W - 1);
    cl.c1 = min(x0 + lane + 32, a.W - 1);
    cl.col0 = cl.c0 - x0;
    cl.col1 = cl.c1 - x0;
    cl.xc = make_float2((float)cl.c0 - 0.5f * (float)(a.W - 1), (float)cl.c1 - 0.5f * (float)(a.W - 1));
    if (MODE == REG_NONRIGID) {
        const float g0 = fminf((float)cl.c0 * a.inv_s, (float)(a.nx - 1));
        const float g1 = fminf((float)cl.c1 * a.inv_s, (float)(a.nx - 1));
        cl.ix0 = cell_of(g0, a.nx);
        cl.ix1 = cell_of(g1, a.nx);
        cl.wx = make_float2(g0 - (float)cl.ix0, g1 - (float)cl.ix1);
    }
    float2 hi[4], lo[4], run[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) { hi[j] = lo[j] = run[j] = make_float2(0.f, 0.f); }
    for (int i = 0; i < n; ++i) {
        const int k = kb + i, st = i % kStages;
        // every lane waits (acquire) before reading the stage
        const bool ok = __all_sync(0xffffffffu,
                                   mbar_wait(smem_u32(&sm.full[st]), (uint32_t)((i / kStages) & 1), a.timeout_ns));
        if (!ok) {
            if (lane == 0) { atomicExch(a.status, kDevWaitTimeout); *abort = 1; }
            break;
        }
        if (*abort) break;
        const int kind = sm.fit[st];
        if (kind == kInterior) tile_frame<MODE, WINDOW, kInterior>(a, sm, st, k, cl, y0, run);
        else if (kind == kStagedClamped) tile_frame<MODE, WINDOW, kStagedClamped>(a, sm, st, k, cl, y0, run);
        else tile_frame<MODE, WINDOW, kGlobal>(a, sm, st, k, cl, y0, run);
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&sm.empty[st])) : "memory");
        if ((i % kRun) == kRun - 1) {
#pragma unroll
            for (int j = 0; j < 4; ++j) fold(hi[j], lo[j], run[j]);
        }
    }
    __syncthreads();
    if (*abort || !a.part) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) fold(hi[j], lo[j], run[j]);
    float2 *p = a.part + (size_t)blockIdx.y * a.H * a.W;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = y0 + warp + 8 * j;
        if (r >= a.H) continue;
        if (cl.in0) p[(size_t)r * a.W + cl.c0] = make_float2(hi[j].x, lo[j].x);
        if (cl.in1) p[(size_t)r * a.W + cl.c1] = make_float2(hi[j].y, lo[j].y);
    }
}

// mean = (1/N) sum over chunks, in chunk order; four pixels per thread (float4 store) when
// the row length allows it.
__global__ void mean_kernel(const float2 *part, int chunks, int W, int H, double inv_n, float *mean)
{
    const size_t P = (size_t)W * H;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((W & 3) == 0 && (((uintptr_t)mean) & 15) == 0) {
        const size_t i0 = 4 * q;
        if (i0 >= P) return;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int c = 0; c < chunks; ++c) {
            const float4 *v = (const float4 *)(part + c * P + i0);
            const float4 u0 = v[0], u1 = v[1];
            s0 += (double)u0.x + (double)u0.y;
            s1 += (double)u0.z + (double)u0.w;
            s2 += (double)u1.x + (double)u1.y;
            s3 += (double)u1.z + (double)u1.w;
        }
        *(float4 *)(mean + i0) = make_float4((float)(s0 * inv_n), (float)(s1 * inv_n), (float)(s2 * inv_n),
                                             (float)(s3 * inv_n));
    } else {
        for (size_t i = 4 * q; i < min(P, 4 * q + 4); ++i) {
            double s = 0.0;
            for (int c = 0; c < chunks; ++c) s += (double)part[c * P + i].x + (double)part[c * P + i].y;
            mean[i] = (float)(s * inv_n);
        }
    }
}

// Per-frame rigid parameters from the scan elements (frame 0: identity).
// cos(a) - 1 = -2 sin^2(a/2) keeps the small-angle term accurate.
__global__ void rigid_prep_kernel(const reg_elem_t *e, int N, float4 *prm)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    if (k == 0) {
        prm[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const reg_elem_t v = e[k - 1];
    const float h = sinf(0.5f * v.alpha);
    prm[k] = make_float4(-2.f * h * h, sinf(v.alpha), v.gx, v.gy);
}

__global__ void grid_gather_kernel(const float2 *src, const int *nodes, int n, int Nc, float2 *dst)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * Nc) return;
    const int i = (int)(t / Nc), j = (int)(t - (size_t)i * Nc);
    dst[t] = src[(size_t)nodes[i] * Nc + j];
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
        cudaGetLastError();
    });
    return fn;
}

}  // namespace

int warp_chunk_frames()
{
    return 64;
}

size_t warp_workspace_bytes(int N, int W, int H, bool mean)
{
    const size_t chunks = (size_t)(N + warp_chunk_frames() - 1) / warp_chunk_frames();
    size_t b = 256 * (((size_t)N * sizeof(float4) + 255) / 256);
    if (mean) b += chunks * (size_t)W * H * sizeof(float2);
    return b;
}

cudaError_t launch_warp(const WarpJob &j, cudaStream_t s, int *used_tma)
{
    const int chunk = warp_chunk_frames();
    const int chunks = (j.N + chunk - 1) / chunk;
    WarpArgs a;
    memset(&a, 0, sizeof(a));
    a.frames = j.frames;
    a.N = j.N;
    a.W = j.W;
    a.H = j.H;
    a.pitch = j.pitch;
    a.mode = j.mode;
    a.nx = j.nx;
    a.ny = j.ny;
    a.s = j.s;
    a.inv_s = j.s > 0 ? 1.0f / (float)j.s : 0.f;
    a.window = j.mode == REG_NONRIGID && j.s >= 8;
    a.out = j.out;
    a.chunk = chunk;
    a.status = j.status;
    a.timeout_ns = j.timeout_ns;
    char *ws = (char *)j.ws;
    float4 *prm = (float4 *)ws;
    a.rigid = prm;
    a.grids = j.grids;
    a.part = j.mean ? (float2 *)(ws + 256 * (((size_t)j.N * sizeof(float4) + 255) / 256)) : nullptr;
    if (j.mode == REG_RIGID) {
        rigid_prep_kernel<<<(j.N + 127) / 128, 128, 0, s>>>(j.elems, j.N, prm);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // TMA needs a 16-byte aligned base, 16-byte multiple strides and a box no larger than the frame
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    EncodeTiled enc = encoder();
    a.use_tma = enc && (((uintptr_t)j.frames) & 15) == 0 && (j.pitch % 4) == 0 && j.W >= kBW && j.H >= kBH;
    if (a.use_tma) {
        const cuuint64_t dims[3] = {(cuuint64_t)j.W, (cuuint64_t)j.H, (cuuint64_t)j.N};
        const cuuint64_t strides[2] = {(cuuint64_t)j.pitch * 4, (cuuint64_t)j.pitch * 4 * j.H};
        const cuuint32_t box[3] = {kBW, kBH, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)j.frames, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            a.use_tma = 0;
    }
    if (used_tma) *used_tma = a.use_tma;
    const int tiles = ((j.W + kTW - 1) / kTW) * ((j.H + kTH - 1) / kTH);
    dim3 grid(tiles, chunks);
    auto kern = j.mode == REG_RIGID ? warp_kernel<REG_RIGID, false>
                : (a.window ? warp_kernel<REG_NONRIGID, true> : warp_kernel<REG_NONRIGID, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WarpSmem));
    if (e != cudaSuccess) return e;
    kern<<<grid, kWThreads, sizeof(WarpSmem), s>>>(a, tmap);
    e = cudaGetLastError();
    if (e != cudaSuccess || !j.mean) return e;
    const size_t quads = ((size_t)j.W * j.H + 3) / 4;
    mean_kernel<<<(unsigned)((quads + 255) / 256), 256, 0, s>>>(a.part, chunks, j.W, j.H, 1.0 / j.N, j.mean);
    return cudaGetLastError();
}

cudaError_t launch_grid_gather(const float2 *src, const int *nodes, int n, int Nc, float2 *dst, cudaStream_t s)
{
    const size_t t = (size_t)n * Nc;
    if (t == 0) return cudaSuccess;
    grid_gather_kernel<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(src, nodes, n, Nc, dst);
    return cudaGetLastError();
}

}  // namespace reg
