// Internal declarations shared by the kernel and host translation units of libreg.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/reg.h"

namespace reg {

constexpr int kMaxLevels = REG_MAX_LEVELS;
constexpr int kThreads = 256;          // threads per CTA of the operator kernels

// One pyramid level of one frame, as the operator kernels read it.
struct LevelDesc {
    const void *ptr;    // template role: storage-typed samples, row-major, pixel (0, 0)
    const void *rptr;   // reference role: the same samples (rigid model) or the B-spline model
                        // at the pixel centres (nonrigid model)
    int W, H, pitch;    // pitch of ptr, in elements
    int rpitch;         // pitch of rptr, in elements
    float mean;         // level mean (FP32 shift constant of the moment sums)
};

// Pyramid layout.  The nonrigid model samples the quadratic B-spline of a level's samples
// extended by the level's mean; storing every level of that model with a border of kPad samples
// holding the mean lets a 3x3 tap window at a nearest sample clamped to [-2, W + 1] x [-2, H + 1]
// read without per-tap clamps and still equal the mean-extended model everywhere.
constexpr int kPad = 3;
inline int level_pitch(int W, int pad) { return W + 2 * pad; }
inline size_t level_elems(int W, int H, int pad) { return (size_t)(W + 2 * pad) * (H + 2 * pad); }
inline size_t level_origin(int W, int pad) { return (size_t)pad * (W + 2 * pad) + pad; }

// Where launch_pyramid writes the levels of frame 0 (frame f at + f * stride elements).
struct PyrOut {
    void *raw[kMaxLevels];            // start of level l's block (border included)
    size_t raw_stride[kMaxLevels];
    void *smooth[kMaxLevels];         // B-spline model at the pixel centres, W_l x H_l, or null
    size_t smooth_stride[kMaxLevels];
    int pad;                          // 0, or kPad border samples (the level's mean) around each level
};

// One operator application.  left < 0: A(f_ref, f_tmpl) from the identity (or
// from `init_node` when >= 0); otherwise B(node[left], node[right]).
struct OpDesc {
    int ref, tmpl;     // frame indices
    int left, right;   // input nodes of B, -1 for A
    int out;           // node written
    int init_node;     // A only: node holding the initial deformation, -1 = identity
};

// Per-operator record written by the device (mirrors reg_stats_t).
struct OpStats {
    int32_t i, k;
    int32_t iters[kMaxLevels], evals[kMaxLevels], stop[kMaxLevels];
    int32_t rejects, status;
    double energy;
    double theta[3];
};
static_assert(sizeof(OpStats) == sizeof(reg_stats_t), "stats layout");

// Device-side error codes in OpStats::status and the kernel status word.
enum DevStatus : int32_t {
    kDevOk = 0,
    kDevBadOp = 1,       // operator descriptor out of range / non-adjacent
    kDevQueueTimeout = 2, // bounded wait on the ready queue gave up
    kDevWaitTimeout = 3   // bounded wait on a TMA load (mbarrier) gave up
};

// Operator model of a launch beyond REG_RIGID / REG_NONRIGID: the mock operator of reg_mock_scan.
constexpr int kModeMock = 2;

struct Config {
    int mode, levels, max_iter, max_rejects;
    double tol_grad, tol_rel_e, armijo_c, tau0, step_cap, lambda;
    int metric;   // nonrigid scalar product: REG_METRIC_MEAN, REG_METRIC_GAUSS_NEWTON or REG_METRIC_H1
    double sigma; // REG_METRIC_H1: smoothing length in control-grid spacings
    double tol_coarse;   // factor on tol_grad at every level above the finest
};

// Ready-queue state of the persistent executor (device memory): one FIFO per priority class,
// class 0 first.  An operator's class is its rank by bottom level (the longest estimated path
// from it to the end of the DAG), so operators on long chains start before ones with slack.
constexpr int kQueueClasses = 16;
struct Queue {
    int *head;         // [kQueueClasses] next slot to claim in each class
    int *tail;         // [kQueueClasses] next slot to fill in each class
    int *slots;        // class c at slots[class_off[c] ...]: op indices in ready order, -1 = not yet filled
    const int *op_class;   // per op: its class
    const int *class_off;  // [kQueueClasses + 1] first slot of each class, then the slot count
    int *pending;      // per op: inputs not yet produced
    int *consumers;    // CSR list of ops consuming each node
    int *cons_start;   // [n_nodes + 1]
    int *done;         // number of finished ops
    int *claimed;      // number of claimed ops, all classes
    int n_class;       // classes in use (1: a plain FIFO)
    long long timeout_ns;
};

struct Params {
    Config cfg;
    const LevelDesc *levels;   // [n_frames][cfg.levels]
    int n_frames;
    const OpDesc *ops;
    int n_ops;
    int op_base;               // first op of this launch (batched launches)
    double *node_theta;        // [n_nodes][3]: rigid (alpha, Gx, Gy); nonrigid (0, mean c_x, mean c_y)
    float2 *node_grid;         // nonrigid: [n_nodes][gny * gnx] control values (finest px)
    const float *mock_us;      // mock operator (kModeMock): duration of each operator, microseconds
    const float *h1q;          // REG_METRIC_H1: the control grid's cosine bases and eigenvalues (Qx, Qy, lx, ly)
    int unroll;                // nonrigid energy passes: pixels in flight per lane (2 or 4; 0 = 4)
    int minb;                  // nonrigid register form: CTAs per SM (3 or 4; 0 = 4 at 16 CTAs per
                               // operator, else 3)
    int gnx, gny, gs;          // nonrigid control grid: points per axis and spacing (finest px)
    int n_nodes;
    OpStats *stats;            // [n_ops]
    int *status;               // kernel status word (first device error)
    Queue queue;               // persistent executor only
};

// Launch shape of the operator kernels (0 = not chosen): CTAs per operator, energy-pass pixels
// per lane, and register form (CTAs per SM the kernel's register budget is sized for).
struct TileShape {
    int cluster = 0, unroll = 0, minb = 0;
};

// Host launchers (reg_kernels.cu).
// Pyramids of N frames (frame f at frames + f * fstride, rows of `pitch`) into the layout `out`
// (storage-typed); means[f * levels + l] = mean of level l of frame f (or null).
cudaError_t launch_pyramid(const float *frames, int N, size_t fstride, int W, int H, int pitch, int levels,
                           int storage, const PyrOut &out, float *means, cudaStream_t s);
// tab[l].mean = means[l] for l < L (a slot's level table rows after its pyramid build).
cudaError_t launch_set_level_means(LevelDesc *tab, const float *means, int L, cudaStream_t s);
cudaError_t launch_ops(const Params &p, int storage, int cluster, int n_launch_ops,
                       cudaStream_t s);
cudaError_t launch_persistent(const Params &p, int storage, int cluster, int workers,
                              cudaStream_t s);
// Clusters of `cluster` CTAs of the persistent kernel that fit on the device at once
// (occupancy query), or -1 if the query fails.
int persistent_resident_clusters(const Params &p, int storage, int cluster);

// Registered series (reg_warp): out_k = f_k o phi_{0,k} and their mean.
struct WarpJob {
    const float *frames;       // device [N][H][pitch]
    int N, W, H, pitch;
    int mode;
    const reg_elem_t *elems;   // rigid: N-1 device elements phi_{0,k}, k = 1..N-1
    const float2 *grids;       // nonrigid: N-1 device control grids [ny][nx]
    int nx, ny, s;
    float *out;                // device [N][H][W] or null
    float *mean;               // device [H][W] or null
    void *ws;                  // warp_workspace_bytes() of device memory
    int *status;               // device status word (kDevWaitTimeout on a timed-out load)
    long long timeout_ns;
};
size_t warp_workspace_bytes(int N, int W, int H, bool mean);
// *used_tma = 1 when the source boxes were staged by TMA (aligned frames, pitch % 4 == 0).
cudaError_t launch_warp(const WarpJob &j, cudaStream_t s, int *used_tma);
// dst (device) = bytes of src, host memory the device reads at the same address; both 16-byte
// aligned, bytes a multiple of 16 (else cudaErrorInvalidValue).  `blocks` CTAs of 256 threads.
cudaError_t launch_stage_copy(void *dst, const void *src, size_t bytes, int blocks, cudaStream_t s);
cudaError_t launch_grid_gather(const float2 *src, const int *nodes, int n, int Nc, float2 *dst, cudaStream_t s);
cudaError_t launch_energy(const Params &p, int storage, const double *theta_dev,
                          const float2 *grid_dev, double *out_dev, float2 *grad_dev,
                          cudaStream_t s);
cudaError_t launch_grid_compose(const float2 *q1, const float2 *q2, int nx, int ny, int spacing,
                                float2 *out, cudaStream_t s);
cudaError_t launch_grid_dense(const float2 *grids, const int *nodes, int n, int nx, int ny,
                              int spacing, int W, int H, float *out, cudaStream_t s);
cudaError_t launch_grid_from_dense(const float *u, int W, int H, int nx, int ny, int spacing,
                                   float2 *out, cudaStream_t s);
// Set the calling thread's message returned by reg_last_error_message().
void set_last_error(const char *msg);
int max_cluster_size();

}  // namespace reg
