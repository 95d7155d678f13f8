// Host side of libreg: the C ABI declared in include/reg.h, the scan DAG
// builders, the executors and device memory management.
#include <algorithm>
#include <chrono>
#include <map>
#include <tuple>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>   // cuPointerGetAttribute's types (resolved at run time)

#include "reg_internal.h"
#include "reg_host.h"

using namespace reg;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CU(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? REG_ENOMEM : REG_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

#define CHECK(expr)                \
    do {                           \
        int r_ = (expr);           \
        if (r_ != REG_OK) return r_; \
    } while (0)

extern "C" const char *reg_strerror(int code)
{
    switch (code) {
    case REG_OK: return "ok";
    case REG_EINVAL: return "invalid argument";
    case REG_ENOMEM: return "out of memory";
    case REG_EBUDGET: return "memory budget or slots exhausted";
    case REG_ETIMEOUT: return "bounded wait timed out";
    case REG_ECUDA: return "CUDA error";
    case REG_ESTATE: return "invalid state";
    }
    return "unknown error";
}

extern "C" const char *reg_last_error_message(void) { return g_last_error.c_str(); }

void reg::set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

int reg::host_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

// ------------------------------------------------------------------ device buffers
namespace {

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    ~DevBuf() { release(); }
    void release()
    {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    int reserve(size_t n)
    {
        if (n <= bytes) return REG_OK;
        release();
        size_t want = std::max(n, (size_t)256);
        cudaError_t e = cudaMalloc(&ptr, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
            return fail(REG_ENOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
        }
        bytes = want;
        return REG_OK;
    }
    template <typename T> T *as() const { return (T *)ptr; }
};

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

using PointerAttrFn = CUresult (*)(void *, CUpointer_attribute, CUdeviceptr);
PointerAttrFn pointer_attr_fn()
{
    static PointerAttrFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (PointerAttrFn) nullptr;
        }
        return (PointerAttrFn)f;
    }();
    return fn;
}

// p when [p, p + bytes) lies in one page-locked host allocation that the current device reads
// at the same address (mapped under unified addressing), else null.
const void *mapped_host_ptr(const void *p, size_t bytes)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer != p) return nullptr;
    PointerAttrFn fn = pointer_attr_fn();
    CUdeviceptr start = 0;
    size_t size = 0;
    if (!fn || fn(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)p) != CUDA_SUCCESS ||
        fn(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)p) != CUDA_SUCCESS)
        return nullptr;
    const uintptr_t b = (uintptr_t)p;
    return b >= start && b - start <= size && bytes <= size - (b - start) ? p : nullptr;
}

size_t storage_bytes(int storage) { return storage == REG_F32 ? 4 : 2; }

}  // namespace

// ------------------------------------------------------------------ scan DAGs
// SSA form: leaves 0..n-1 are x_0..x_{n-1}; op j makes node n+j = node[l] (.) node[r].
namespace {

struct Dag {
    std::vector<int> left, right, out;
};

struct DagBuilder {
    int n;
    Dag d;
    explicit DagBuilder(int n_) : n(n_) {}
    int op(int l, int r)
    {
        d.left.push_back(l);
        d.right.push_back(r);
        return n + (int)d.left.size() - 1;
    }
};

// Sequential recursion phi_{0,i} = phi_{0,i-1} (.) phi_{i-1,i} (Sec. 3).
Dag dag_seq(int n)
{
    DagBuilder b(n);
    std::vector<int> cur(n);
    for (int i = 0; i < n; ++i) cur[i] = i;
    for (int i = 1; i < n; ++i) cur[i] = b.op(cur[i - 1], cur[i]);
    b.d.out = cur;
    return b.d;
}

// Brent-Kung: reduction tree over strides 1, 2, 4, ..., then a reverse tree
// that completes the prefixes between the tree nodes (Table 1 family).
Dag dag_brent_kung(int n)
{
    DagBuilder b(n);
    std::vector<int> cur(n);
    for (int i = 0; i < n; ++i) cur[i] = i;
    int stride = 1;
    for (; stride < n; stride *= 2)
        for (int i = 2 * stride - 1; i < n; i += 2 * stride) cur[i] = b.op(cur[i - stride], cur[i]);
    int top = 1;
    while (top * 4 <= n) top *= 2;   // largest stride whose reverse step can apply
    for (int s = top; s >= 1; s /= 2)
        for (int i = 3 * s - 1; i < n; i += 2 * s) cur[i] = b.op(cur[i - s], cur[i]);
    b.d.out = cur;
    return b.d;
}

// Dissemination: in round r every element combines with the one 2^r before it (Fig. 2).
Dag dag_dissemination(int n)
{
    DagBuilder b(n);
    std::vector<int> cur(n), prev;
    for (int i = 0; i < n; ++i) cur[i] = i;
    for (int s = 1; s < n; s *= 2) {
        prev = cur;
        for (int i = s; i < n; ++i) cur[i] = b.op(prev[i - s], prev[i]);
    }
    b.d.out = cur;
    return b.d;
}

// Ladner-Fischer P_k recursion (Table 1): P_0 = P_1 on the left half, P_0 on the
// right half, then the left total applied to every right prefix; P_k (k >= 1)
// pairs neighbours, recurses with P_{k-1} on the pairs and fills even positions.
std::vector<int> lf_rec(DagBuilder &b, const std::vector<int> &xs, int k)
{
    const int m = (int)xs.size();
    if (m == 1) return xs;
    if (m == 2) return {xs[0], b.op(xs[0], xs[1])};
    std::vector<int> res;
    if (k == 0) {
        int h = (m + 1) / 2;
        std::vector<int> L = lf_rec(b, std::vector<int>(xs.begin(), xs.begin() + h), 1);
        std::vector<int> R = lf_rec(b, std::vector<int>(xs.begin() + h, xs.end()), 0);
        res = L;
        for (int r : R) res.push_back(b.op(L.back(), r));
        return res;
    }
    std::vector<int> pairs;
    for (int i = 0; i + 1 < m; i += 2) pairs.push_back(b.op(xs[i], xs[i + 1]));
    std::vector<int> sub = lf_rec(b, pairs, k - 1);
    res.push_back(xs[0]);
    for (int i = 1; i < m; ++i) res.push_back(i % 2 ? sub[i / 2] : b.op(sub[i / 2 - 1], xs[i]));
    return res;
}

Dag dag_ladner_fischer(int n)
{
    DagBuilder b(n);
    std::vector<int> xs(n);
    for (int i = 0; i < n; ++i) xs[i] = i;
    b.d.out = n > 0 ? lf_rec(b, xs, 0) : std::vector<int>();
    return b.d;
}

// Online scan with a look-back of k leaves (k a power of two): as leaf j arrives, window nodes
// w_m(j) = w_{m-1}(j - 2^(m-1)) (.) w_{m-1}(j) for j >= 2^m - 1, m = 1..log2 k, then the prefix
// p_j = p_{j-1} (.) x_j for 0 < j < k and p_j = p_{j-k} (.) w_{log2 k}(j) for j >= k: k chains of
// prefixes advance side by side (the streaming service's schedule; k = 1 is the sequential one).
Dag dag_lookback(int n, int k)
{
    DagBuilder b(n);
    int m = 0;
    while ((1 << m) < k) ++m;
    std::vector<std::vector<int>> w(m + 1, std::vector<int>(n, -1));
    for (int j = 0; j < n; ++j) w[0][j] = j;
    std::vector<int> p(n, -1);
    for (int j = 0; j < n; ++j) {
        for (int lev = 1; lev <= m; ++lev)
            if (j >= (1 << lev) - 1) w[lev][j] = b.op(w[lev - 1][j - (1 << (lev - 1))], w[lev - 1][j]);
        if (j == 0) p[0] = 0;
        else if (j < k) p[j] = b.op(p[j - 1], j);
        else p[j] = b.op(p[j - k], w[m][j]);
    }
    b.d.out = p;
    return b.d;
}

// Blelloch: the reduction tree, then the root set to the identity (node -1) and a down-sweep that
// hands every left child its parent's value and every right child the parent's value combined
// with the left child's sum: an exclusive scan, out[i] = x_0 (.) ... (.) x_{i-1}.  The tree spans
// the next power of two P >= n with identity elements past n; an application with such an operand
// (x (.) e = x) is not made, nor one whose value only reaches positions >= n.  Table 1 counts the
// identity applications of the down-sweep: work 2 (n - 1).
Dag dag_blelloch(int n)
{
    DagBuilder b(n);
    int P = 1;
    while (P < n) P *= 2;
    std::vector<int> cur(P, -1);
    for (int i = 0; i < n; ++i) cur[i] = i;
    int d = 1;
    for (; d < P; d *= 2)
        for (int i = 2 * d - 1; i < P; i += 2 * d)
            if (cur[i] != -1) cur[i] = b.op(cur[i - d], cur[i]);
            else cur[i] = cur[i - d];   // padding is a suffix: the left operand alone
    if (n > 0) cur[P - 1] = -1;
    for (d = P / 2; d >= 1; d /= 2)
        for (int i = 2 * d - 1; i < P; i += 2 * d) {
            const int left = cur[i - d], parent = cur[i];
            cur[i - d] = parent;
            cur[i] = (left != -1 && i - d + 1 < n) ? b.op(parent, left) : parent;
        }
    cur.resize(n);
    b.d.out = cur;
    return b.d;
}

bool make_dag(int schedule, int n, Dag &d)
{
    switch (schedule) {
    case REG_SCHED_BLELLOCH: d = dag_blelloch(n); return true;
    case REG_SCHED_LOOKBACK_2: d = dag_lookback(n, 2); return true;
    case REG_SCHED_LOOKBACK_4: d = dag_lookback(n, 4); return true;
    case REG_SCHED_LOOKBACK_8: d = dag_lookback(n, 8); return true;
    case REG_SCHED_SEQ: d = dag_seq(n); return true;
    case REG_SCHED_BRENT_KUNG: d = dag_brent_kung(n); return true;
    case REG_SCHED_DISSEMINATION: d = dag_dissemination(n); return true;
    case REG_SCHED_LADNER_FISCHER: d = dag_ladner_fischer(n); return true;
    }
    return false;
}

}  // namespace

extern "C" int reg_scan_work(int schedule, int n)
{
    if (n < 0) return -1;
    Dag d;
    if (!make_dag(schedule, n, d)) return -1;
    return (int)d.left.size();
}

extern "C" int reg_scan_dag(int schedule, int n, int32_t *left, int32_t *right, int32_t *out_node)
{
    if (n < 0) return -1;
    Dag d;
    if (!make_dag(schedule, n, d)) return -1;
    for (size_t j = 0; j < d.left.size(); ++j) {
        if (left) left[j] = d.left[j];
        if (right) right[j] = d.right[j];
    }
    if (out_node)
        for (int i = 0; i < n; ++i) out_node[i] = d.out[i];
    return (int)d.left.size();
}

// ------------------------------------------------------------------ context
// Streams of the one-launch-per-operator executor: enough concurrent operators to fill every
// CTA slot of the GPU (152 SMs x 3-4 CTAs / 16 CTAs per operator = 28-38 operators).
constexpr int kPoolStreams = 64;

struct reg_ctx {
    reg_config_t cfg;
    int device = 0;
    int num_sms = 0;
    std::mutex mu;
    // workspaces
    DevBuf frames_dev;      // host-supplied frames staged on the device
    DevBuf pyr[kMaxLevels]; // pyramid levels of all frames (nonrigid: with a border holding the mean)
    DevBuf spyr[kMaxLevels]; // nonrigid: the B-spline model of every level at its pixel centres
    DevBuf means, level_tab, ops, stats, node_theta, node_grid, status, node_ids;
    DevBuf q_slots, q_pending, q_cons, q_cons_start, q_ctr, q_class;
    DevBuf h1q;   // REG_METRIC_H1: cosine bases and eigenvalues of the control grid
    DevBuf tmp;
    cudaStream_t pool[kPoolStreams] = {};
    cudaEvent_t ev_pool_done[kPoolStreams] = {};
    std::vector<cudaEvent_t> op_events;
    bool pool_ready = false;
    // REG_EXEC_GRAPH: the captured plain-path launches and the plan they were captured for
    // last successful nonrigid reg_scan: prefixes' node indices are in node_ids
    int last_n = 0, last_gnx = 0, last_gny = 0;
    std::vector<int> last_op_nodes;   // node produced by each operator, in per_op order
    DevBuf pick_ids;                  // reg_scan_node_grids: node indices of one request
    DevBuf warp_ws;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture = nullptr;   // graphs are captured here (the caller's stream may be the legacy one)
    uint64_t graph_key = 0;
    int graph_captures = 0;
    // autotuned launch shapes, keyed by (W, H, mode, storage, exec, floor(log2 N))
    std::map<std::tuple<int, int, int, int, int, int>, TileShape> tuned;
    // measurement
    bool timing = false;
    std::vector<cudaEvent_t> tev;   // timing events, used in pairs
    size_t tev_used = 0;
    std::vector<std::pair<int, int>> op_pairs, pyr_pairs;
    std::pair<int, int> h2d_pair = {-1, -1};   // copy of host frames to the device
    size_t split_from = 0, split_at = 0;   // REG_EXEC_SPLIT_PHASES: op_pairs [from, at) = A, [at, end) = B
    bool split = false;
    reg_timing_t last = {};
};

extern "C" void reg_config_default(reg_config_t *c)
{
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->mode = REG_RIGID;
    c->levels = 2;
    c->max_iter = 500;
    c->max_rejects = 30;
    c->tol_grad = 3e-5;
    c->tol_rel_e = 0.0;
    c->metric = REG_METRIC_GAUSS_NEWTON;
    c->sigma = 1.0;
    c->tol_coarse = 10.0;
    c->armijo_c = 0.25;
    c->tau0 = 1.0;
    c->step_cap = 0.5;
    c->lambda = 2.0;
    c->grid = 0;
    c->storage = REG_F32;
    c->cluster = 0;
    c->workers = 0;
    c->mem_budget = 0;
}

static int validate_cfg(const reg_config_t &c)
{
    if (c.mode != REG_RIGID && c.mode != REG_NONRIGID) return fail(REG_EINVAL, "mode %d", c.mode);
    if (c.levels < 1 || c.levels > kMaxLevels) return fail(REG_EINVAL, "levels %d not in 1..%d", c.levels, kMaxLevels);
    if (c.max_iter < 0 || c.max_rejects < 0) return fail(REG_EINVAL, "negative iteration limits");
    if (!(c.tau0 > 0) || !(c.step_cap > 0) || !(c.armijo_c > 0 && c.armijo_c < 1))
        return fail(REG_EINVAL, "tau0/step_cap/armijo_c out of range");
    if (!(c.tol_grad >= 0) || !(c.tol_rel_e >= 0)) return fail(REG_EINVAL, "tol_grad/tol_rel_e must be >= 0");
    if (c.storage != REG_F32 && c.storage != REG_BF16 && c.storage != REG_F16)
        return fail(REG_EINVAL, "storage %d", c.storage);
    if (c.cluster != 0 && c.cluster != 1 && c.cluster != 2 && c.cluster != 4 && c.cluster != 8 && c.cluster != 16)
        return fail(REG_EINVAL, "cluster %d not in {0,1,2,4,8,16}", c.cluster);
    if (c.lambda < 0) return fail(REG_EINVAL, "lambda < 0");
    if (c.grid < 0) return fail(REG_EINVAL, "grid < 0");
    if (c.metric != REG_METRIC_MEAN && c.metric != REG_METRIC_GAUSS_NEWTON && c.metric != REG_METRIC_H1)
        return fail(REG_EINVAL, "metric %d", c.metric);
    if (!(c.sigma >= 0.0 && c.sigma <= 1.0e3)) return fail(REG_EINVAL, "sigma %g not in [0, 1000]", c.sigma);
    if (!(c.tol_coarse >= 1.0 && c.tol_coarse <= 1.0e6))
        return fail(REG_EINVAL, "tol_coarse %g not in [1, 1e6]", c.tol_coarse);
    if (c.unroll != 0 && c.unroll != 2 && c.unroll != 4) return fail(REG_EINVAL, "unroll %d not in {0,2,4}", c.unroll);
    if (c.ctas_per_sm != 0 && c.ctas_per_sm != 3 && c.ctas_per_sm != 4)
        return fail(REG_EINVAL, "ctas_per_sm %d not in {0,3,4}", c.ctas_per_sm);
    return REG_OK;
}

int reg::validate_config(const reg_config_t &c) { return validate_cfg(c); }

extern "C" int reg_ctx_create(const reg_config_t *cfg, int device, reg_ctx_t **out)
{
    if (!out) return fail(REG_EINVAL, "out is NULL");
    *out = nullptr;
    reg_config_t c;
    if (cfg) c = *cfg;
    else reg_config_default(&c);
    CHECK(validate_cfg(c));
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= device || device < 0) {
        cudaGetLastError();
        return fail(REG_ECUDA, "no CUDA device %d (count %d)", device, n);
    }
    cudaDeviceProp prop;
    CU(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(REG_ECUDA, "device %d is sm_%d%d; this build targets sm_103a (GB300)", device, prop.major,
                    prop.minor);
    CU(cudaSetDevice(device));
    reg_ctx *ctx = new reg_ctx();
    ctx->cfg = c;
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    *out = ctx;
    return REG_OK;
}

reg_config_t reg::host_config(reg_ctx_t *ctx) { return ctx->cfg; }
int reg::host_device(reg_ctx_t *ctx) { return ctx->device; }

extern "C" void reg_ctx_destroy(reg_ctx_t *ctx)
{
    if (!ctx) return;
    stop_stream_service(ctx);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->pool_ready) {
        for (int i = 0; i < kPoolStreams; ++i) {
            cudaStreamDestroy(ctx->pool[i]);
            cudaEventDestroy(ctx->ev_pool_done[i]);
        }
        cudaStreamDestroy(ctx->capture);
    }
    for (cudaEvent_t e : ctx->op_events) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    delete ctx;
}

// ------------------------------------------------------------------ shared pieces
namespace {

// Timing: event pairs recorded on the launching stream, resolved after the call.
void timing_reset(reg_ctx *ctx)
{
    ctx->tev_used = 0;
    ctx->op_pairs.clear();
    ctx->pyr_pairs.clear();
    ctx->split = false;
    ctx->split_from = ctx->split_at = 0;
    ctx->h2d_pair = {-1, -1};
    memset(&ctx->last, 0, sizeof(ctx->last));
}

int timing_mark(reg_ctx *ctx, cudaStream_t s)
{
    if (!ctx->timing) return -1;
    if (ctx->tev_used == ctx->tev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        ctx->tev.push_back(e);
    }
    int id = (int)ctx->tev_used++;
    if (cudaEventRecord(ctx->tev[id], s) != cudaSuccess) return -1;
    return id;
}

void timing_resolve(reg_ctx *ctx)
{
    if (!ctx->timing) return;
    auto sum = [&](const std::vector<std::pair<int, int>> &v) {
        double t = 0.0;
        for (auto &pr : v) {
            float ms = 0.f;
            if (pr.first >= 0 && pr.second >= 0 && cudaEventElapsedTime(&ms, ctx->tev[pr.first], ctx->tev[pr.second]) == cudaSuccess)
                t += ms;
        }
        return t;
    };
    ctx->last.op_kernel_ms = sum(ctx->op_pairs);
    ctx->last.pyramid_ms = sum(ctx->pyr_pairs);
    ctx->last.h2d_ms = sum(std::vector<std::pair<int, int>>{ctx->h2d_pair});
    if (ctx->split) {
        std::vector<std::pair<int, int>> a(ctx->op_pairs.begin() + ctx->split_from, ctx->op_pairs.begin() + ctx->split_at);
        std::vector<std::pair<int, int>> b(ctx->op_pairs.begin() + ctx->split_at, ctx->op_pairs.end());
        ctx->last.leaf_ms = sum(a);
        ctx->last.dag_ms = sum(b);
    }
}

struct Geometry {
    int W[kMaxLevels], H[kMaxLevels], levels;
};

int geometry(int W, int H, int levels, Geometry &g)
{
    g.levels = levels;
    int w = W, h = H;
    for (int l = 0; l < levels; ++l) {
        if (w < 2 || h < 2)
            return fail(REG_EINVAL, "level %d of a %dx%d frame is %dx%d; every level needs >= 2x2", l, W, H, w, h);
        g.W[l] = w;
        g.H[l] = h;
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    return REG_OK;
}

struct GridDims {
    int nx, ny, s;
};

// Control grid of the nonrigid field: spacing 16 finest pixels doubled until at most 65 points per
// axis (grid == 0), or the configured spacing; every level needs a spacing of at least one pixel.
int grid_dims(int W, int H, int grid, int levels, GridDims &g)
{
    if (grid < 0) return fail(REG_EINVAL, "grid spacing %d < 0", grid);
    int sp = grid > 0 ? grid : 16;
    if (grid == 0)
        while ((W - 1 + sp - 1) / sp + 1 > 65 || (H - 1 + sp - 1) / sp + 1 > 65) sp *= 2;
    g.s = sp;
    g.nx = (W - 1 + sp - 1) / sp + 1;
    g.ny = (H - 1 + sp - 1) / sp + 1;
    if (g.nx < 2 || g.ny < 2) return fail(REG_EINVAL, "control grid needs >= 2x2 points");
    if ((sp >> (levels - 1)) < 1 || (sp & ((1 << (levels - 1)) - 1)) != 0)
        return fail(REG_EINVAL, "grid spacing %d must be a multiple of 2^(levels-1)", sp);
    // dynamic shared memory of a one-CTA operator (the largest band): c, d, ct, the scalar product
    // and the band as float2, then one float4 control row per warp; the static part stays under 8 KB
    const size_t nc = (size_t)g.nx * g.ny;
    if (8 * (5 * nc + 1) + 16 * (size_t)(kThreads / 32) * (g.nx - 1) > 216 * 1024)
        return fail(REG_EINVAL, "control grid %dx%d does not fit shared memory; use a larger spacing", g.nx, g.ny);
    return REG_OK;
}

Config dev_config(const reg_config_t &c)
{
    Config d;
    d.mode = c.mode;
    d.levels = c.levels;
    d.max_iter = c.max_iter;
    d.max_rejects = c.max_rejects;
    d.tol_grad = c.tol_grad;
    d.tol_rel_e = c.tol_rel_e;
    d.armijo_c = c.armijo_c;
    d.tau0 = c.tau0;
    d.step_cap = c.step_cap;
    d.lambda = c.lambda;
    d.metric = c.metric;
    d.sigma = c.sigma;
    d.tol_coarse = c.tol_coarse;
    return d;
}

// Build the pyramids of `nf` frames (device fp32, frame f at frames + f*fstride,
// rows of `pitch`) into ctx->pyr starting at frame slot `first`, and fill the
// level table rows of those frames.  `total` frames are reserved.  The nonrigid
// model stores every level with a border holding its mean (its B-spline window) and the
// model at the pixel centres (its reference role) beside it.
int build_pyramids(reg_ctx *ctx, const Geometry &g, const float *frames, int nf, size_t fstride, int pitch,
                   int first, int total, cudaStream_t s)
{
    const int L = g.levels;
    const size_t sb = storage_bytes(ctx->cfg.storage);
    const bool nonrigid = ctx->cfg.mode == REG_NONRIGID;
    PyrOut o;
    memset(&o, 0, sizeof(o));
    o.pad = nonrigid ? kPad : 0;
    for (int l = 0; l < L; ++l) {
        o.raw_stride[l] = level_elems(g.W[l], g.H[l], o.pad);
        CHECK(ctx->pyr[l].reserve(o.raw_stride[l] * sb * total));
        o.raw[l] = (char *)ctx->pyr[l].ptr + o.raw_stride[l] * sb * first;
        if (nonrigid) {
            o.smooth_stride[l] = (size_t)g.W[l] * g.H[l];
            CHECK(ctx->spyr[l].reserve(o.smooth_stride[l] * sb * total));
            o.smooth[l] = (char *)ctx->spyr[l].ptr + o.smooth_stride[l] * sb * first;
        }
    }
    CHECK(ctx->means.reserve(sizeof(float) * (size_t)total * L));
    int e0 = timing_mark(ctx, s);
    CU(launch_pyramid(frames, nf, fstride, g.W[0], g.H[0], pitch, L, ctx->cfg.storage, o,
                      ctx->means.as<float>() + (size_t)first * L, s));
    ctx->pyr_pairs.push_back({e0, timing_mark(ctx, s)});
    ctx->last.pyramid_launches += (nonrigid ? 4 : 2) * L;
    return REG_OK;
}

// Level table for `total` frames (means are read on the device side via a copy).
int build_level_table(reg_ctx *ctx, const Geometry &g, int total, cudaStream_t s)
{
    const int L = g.levels;
    const size_t sb = storage_bytes(ctx->cfg.storage);
    const int pad = ctx->cfg.mode == REG_NONRIGID ? kPad : 0;
    std::vector<float> means((size_t)total * L);
    CU(cudaMemcpyAsync(means.data(), ctx->means.ptr, sizeof(float) * means.size(), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    std::vector<LevelDesc> tab((size_t)total * L);
    for (int f = 0; f < total; ++f)
        for (int l = 0; l < L; ++l) {
            LevelDesc &d = tab[(size_t)f * L + l];
            const size_t raw = level_elems(g.W[l], g.H[l], pad);
            d.ptr = (const char *)ctx->pyr[l].ptr + (raw * f + level_origin(g.W[l], pad)) * sb;
            d.W = g.W[l];
            d.H = g.H[l];
            d.pitch = level_pitch(g.W[l], pad);
            if (pad) {
                d.rptr = (const char *)ctx->spyr[l].ptr + (size_t)g.W[l] * g.H[l] * sb * f;
                d.rpitch = g.W[l];
            } else {
                d.rptr = d.ptr;
                d.rpitch = d.pitch;
            }
            d.mean = means[(size_t)f * L + l];
        }
    CHECK(ctx->level_tab.reserve(sizeof(LevelDesc) * tab.size()));
    CU(cudaMemcpyAsync(ctx->level_tab.ptr, tab.data(), sizeof(LevelDesc) * tab.size(), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    return REG_OK;
}

int log2_floor(int v)
{
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return l;
}

// Launch shape chosen by reg_autotune for this frame size and executor (zeros if none), with
// every field the config fixes taken from the config.
TileShape tuned_shape(const reg_ctx *ctx, int W, int H, int exec, int N)
{
    TileShape t;
    auto it = ctx->tuned.find(std::make_tuple(W, H, ctx->cfg.mode, ctx->cfg.storage, exec, log2_floor(N)));
    if (it != ctx->tuned.end()) t = it->second;
    if (ctx->cfg.cluster > 0) t.cluster = ctx->cfg.cluster;
    if (ctx->cfg.unroll > 0) t.unroll = ctx->cfg.unroll;
    if (ctx->cfg.ctas_per_sm > 0) t.minb = ctx->cfg.ctas_per_sm;
    return t;
}

// Record the shape of an operator launch in the context's accounting.
void note_shape(reg_ctx *ctx, const Params &p, int C)
{
    ctx->last.cluster = C;
    ctx->last.unroll = p.cfg.mode == REG_NONRIGID ? (p.unroll == 2 ? 2 : 4) : 0;
    ctx->last.ctas_per_sm = p.cfg.mode == REG_NONRIGID ? (p.minb > 0 ? p.minb : (C >= 16 ? 4 : 3)) : 4;
}

int pow2_floor(int v)
{
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

// CTAs per operator for a launch of `n_ops` concurrent operators: enough to fill
// the GPU twice over (two CTAs per SM), at most 8, unless fixed by the config.
int auto_cluster(const reg_ctx *ctx, int n_ops)
{
    if (ctx->cfg.cluster > 0) return ctx->cfg.cluster;
    int slots = 2 * ctx->num_sms;
    int c = pow2_floor(std::max(1, slots / std::max(1, n_ops)));
    return std::min(8, c);
}

struct ScanPlan {
    std::vector<OpDesc> ops;       // execution order (grouped by depth)
    std::vector<int> user_index;   // execution index -> index in the user's stats order
    std::vector<int> depth_start;  // ops[depth_start[d] .. depth_start[d+1]) have depth d
    std::vector<int> node_i, node_k;
    std::vector<int> out_nodes;
    int n_nodes = 0;
};

int plan_scan(int N, const Dag &d, ScanPlan &p)
{
    const int n = N - 1, m = (int)d.left.size();
    p.n_nodes = n + m;
    p.node_i.assign(p.n_nodes, 0);
    p.node_k.assign(p.n_nodes, 0);
    std::vector<OpDesc> user(n + m);
    std::vector<int> depth(p.n_nodes, 0), op_depth(n + m, 0);
    for (int i = 0; i < n; ++i) {
        p.node_i[i] = i;
        p.node_k[i] = i + 1;
        user[i] = OpDesc{i, i + 1, -1, -1, i, -1};
    }
    for (int j = 0; j < m; ++j) {
        int l = d.left[j], r = d.right[j], o = n + j;
        if (l < 0 || r < 0 || l >= o || r >= o) return fail(REG_EINVAL, "malformed DAG");
        if (p.node_k[l] != p.node_i[r])
            return fail(REG_EINVAL, "B needs adjacent elements: (%d,%d) (.) (%d,%d)", p.node_i[l], p.node_k[l],
                        p.node_i[r], p.node_k[r]);
        p.node_i[o] = p.node_i[l];
        p.node_k[o] = p.node_k[r];
        depth[o] = 1 + std::max(depth[l], depth[r]);
        user[n + j] = OpDesc{p.node_i[l], p.node_k[r], l, r, o, -1};
        op_depth[n + j] = depth[o];
    }
    int maxd = 0;
    for (int v : op_depth) maxd = std::max(maxd, v);
    p.depth_start.assign(maxd + 2, 0);
    for (int v : op_depth) p.depth_start[v + 1]++;
    for (int q = 0; q <= maxd; ++q) p.depth_start[q + 1] += p.depth_start[q];
    std::vector<int> fill(p.depth_start.begin(), p.depth_start.end() - 1);
    p.ops.resize(n + m);
    p.user_index.resize(n + m);
    for (int u = 0; u < n + m; ++u) {
        int e = fill[op_depth[u]]++;
        p.ops[e] = user[u];
        p.user_index[e] = u;
    }
    p.out_nodes = d.out;
    return REG_OK;
}

int ensure_pool(reg_ctx *ctx)
{
    if (ctx->pool_ready) return REG_OK;
    for (int i = 0; i < kPoolStreams; ++i) {
        CU(cudaStreamCreateWithFlags(&ctx->pool[i], cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&ctx->ev_pool_done[i], cudaEventDisableTiming));
    }
    CU(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
    ctx->pool_ready = true;
    return REG_OK;
}

int ensure_op_events(reg_ctx *ctx, size_t n)
{
    while (ctx->op_events.size() < n) {
        cudaEvent_t e;
        CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->op_events.push_back(e);
    }
    return REG_OK;
}

// Allocate node storage and stats; fill Params.
int prepare_params(reg_ctx *ctx, const Geometry &g, int n_frames, int n_nodes, int n_ops, Params &p, cudaStream_t s)
{
    memset(&p, 0, sizeof(p));
    p.cfg = dev_config(ctx->cfg);
    p.levels = ctx->level_tab.as<LevelDesc>();
    p.n_frames = n_frames;
    p.n_ops = n_ops;
    p.n_nodes = n_nodes;
    CHECK(ctx->ops.reserve(sizeof(OpDesc) * std::max(1, n_ops)));
    p.ops = ctx->ops.as<OpDesc>();
    CHECK(ctx->stats.reserve(sizeof(OpStats) * std::max(1, n_ops)));
    p.stats = ctx->stats.as<OpStats>();
    CHECK(ctx->node_theta.reserve(sizeof(double) * 3 * std::max(1, n_nodes)));
    p.node_theta = ctx->node_theta.as<double>();
    CHECK(ctx->status.reserve(sizeof(int) * 4));
    p.status = ctx->status.as<int>();
    CU(cudaMemsetAsync(p.status, 0, sizeof(int) * 4, s));
    CU(cudaMemsetAsync(p.stats, 0, sizeof(OpStats) * std::max(1, n_ops), s));
    if (ctx->cfg.mode == REG_NONRIGID) {
        GridDims gd;
        CHECK(grid_dims(g.W[0], g.H[0], ctx->cfg.grid, g.levels, gd));
        p.gnx = gd.nx;
        p.gny = gd.ny;
        p.gs = gd.s;
        CHECK(ctx->node_grid.reserve(sizeof(float2) * (size_t)gd.nx * gd.ny * std::max(1, n_nodes)));
        p.node_grid = ctx->node_grid.as<float2>();
        if (ctx->cfg.metric == REG_METRIC_H1) {
            // orthonormal DCT-II bases Q[j][k] = a_k cos(pi k (j + 1/2) / n) of the free-end path
            // graphs, a_0 = sqrt(1/n), a_k = sqrt(2/n), and their Laplacian eigenvalues 2 - 2 cos(pi k / n)
            std::vector<float> q;
            for (int n : {gd.nx, gd.ny})
                for (int j = 0; j < n; ++j)
                    for (int k = 0; k < n; ++k)
                        q.push_back((float)(std::sqrt((k == 0 ? 1.0 : 2.0) / n) * std::cos(M_PI * k * (j + 0.5) / n)));
            for (int n : {gd.nx, gd.ny})
                for (int k = 0; k < n; ++k) q.push_back((float)(2.0 - 2.0 * std::cos(M_PI * k / n)));
            CHECK(ctx->h1q.reserve(sizeof(float) * q.size()));
            CU(cudaMemcpyAsync(ctx->h1q.ptr, q.data(), sizeof(float) * q.size(), cudaMemcpyHostToDevice, s));
            p.h1q = ctx->h1q.as<float>();
        }
    }
    return REG_OK;
}

int check_device_status(reg_ctx *ctx, cudaStream_t s)
{
    int st[4];
    CU(cudaMemcpyAsync(st, ctx->status.ptr, sizeof(st), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (st[0] == kDevQueueTimeout) return fail(REG_ETIMEOUT, "device ready-queue wait timed out");
    if (st[0] != 0) return fail(REG_EINVAL, "device rejected an operator descriptor (code %d)", st[0]);
    return REG_OK;
}

uint64_t fnv1a(const void *data, size_t n, uint64_t h)
{
    const unsigned char *b = (const unsigned char *)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ULL;
    }
    return h;
}

// One launch per operator on the stream pool, in plan order; an operator waits for the
// events of the two operators that produce its inputs.  The pool forks from and joins back
// into s, so the whole sequence can also be captured from s as one graph.
int launch_plain(reg_ctx *ctx, const ScanPlan &plan, const Params &p, int C, cudaStream_t s)
{
    const int n_ops = (int)plan.ops.size();
    const int storage = ctx->cfg.storage;
    std::vector<int> node_op(p.n_nodes, -1);
    for (int e = 0; e < n_ops; ++e) node_op[plan.ops[e].out] = e;
    CU(cudaEventRecord(ctx->ev_pool_done[0], s));
    for (int i = 0; i < kPoolStreams; ++i) CU(cudaStreamWaitEvent(ctx->pool[i], ctx->ev_pool_done[0], 0));
    for (int e = 0; e < n_ops; ++e) {
        cudaStream_t ls = ctx->pool[e % kPoolStreams];
        const OpDesc &op = plan.ops[e];
        // inputs produced by an earlier launch on s are complete: the pool forked from s after it
        if (op.left >= 0 && node_op[op.left] >= 0) CU(cudaStreamWaitEvent(ls, ctx->op_events[node_op[op.left]], 0));
        if (op.right >= 0 && node_op[op.right] >= 0) CU(cudaStreamWaitEvent(ls, ctx->op_events[node_op[op.right]], 0));
        Params q = p;
        q.op_base = e;
        CU(launch_ops(q, storage, C, 1, ls));
        CU(cudaEventRecord(ctx->op_events[e], ls));
    }
    for (int i = 0; i < kPoolStreams; ++i) {
        CU(cudaEventRecord(ctx->ev_pool_done[i], ctx->pool[i]));
        CU(cudaStreamWaitEvent(s, ctx->ev_pool_done[i], 0));
    }
    return REG_OK;
}

// Execute the planned operators.
int execute(reg_ctx *ctx, const ScanPlan &plan, Params &p, int exec, const TileShape &tuned, cudaStream_t s)
{
    const int n_ops = (int)plan.ops.size();
    const int storage = ctx->cfg.storage;
    const int n_depth = (int)plan.depth_start.size() - 1;
    p.unroll = tuned.unroll;
    p.minb = tuned.minb;
    if (exec == REG_EXEC_LEVEL) {
        for (int dpt = 0; dpt < n_depth; ++dpt) {
            int b = plan.depth_start[dpt], e = plan.depth_start[dpt + 1];
            int C = tuned.cluster > 0 ? tuned.cluster : auto_cluster(ctx, e - b);
            note_shape(ctx, p, C);
            int chunk = std::max(1, e - b);
            for (int q = b; q < e; q += chunk) {
                p.op_base = q;
                int e0 = timing_mark(ctx, s);
                CU(launch_ops(p, storage, C, std::min(chunk, e - q), s));
                ctx->op_pairs.push_back({e0, timing_mark(ctx, s)});
                ctx->last.op_launches += 1;
            }
        }
        return REG_OK;
    }
    if (exec == REG_EXEC_PLAIN) {
        CHECK(ensure_pool(ctx));
        CHECK(ensure_op_events(ctx, n_ops));
        const int C = tuned.cluster > 0 ? tuned.cluster : 8;
        note_shape(ctx, p, C);
        const int t0 = timing_mark(ctx, s);
        CHECK(launch_plain(ctx, plan, p, C, s));
        ctx->op_pairs.push_back({t0, timing_mark(ctx, s)});
        ctx->last.op_launches += n_ops;
        return REG_OK;
    }
    if (exec == REG_EXEC_GRAPH) {
        CHECK(ensure_pool(ctx));
        CHECK(ensure_op_events(ctx, n_ops));
        const int C = tuned.cluster > 0 ? tuned.cluster : 8;
        note_shape(ctx, p, C);
        // The graph bakes in the kernel arguments (workspace pointers, config) and the
        // dependency edges; the descriptors themselves are read from device memory when it runs.
        p.op_base = 0;
        uint64_t key = fnv1a(&p, sizeof(p), 1469598103934665603ULL);
        key = fnv1a(plan.ops.data(), sizeof(OpDesc) * plan.ops.size(), key);
        int hdr[4] = {C, storage, ctx->cfg.mode, n_ops};
        key = fnv1a(hdr, sizeof(hdr), key);
        if (!ctx->graph || ctx->graph_key != key) {
            if (ctx->graph) {
                CU(cudaGraphExecDestroy(ctx->graph));
                ctx->graph = nullptr;
            }
            // Relaxed mode: the launcher sets kernel attributes (not stream work) while capturing.
            CU(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeRelaxed));
            const int rc = launch_plain(ctx, plan, p, C, ctx->capture);
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(ctx->capture, &g);
            if (rc != REG_OK || ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return rc != REG_OK ? rc : fail(REG_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
            }
            const cudaError_t ie = cudaGraphInstantiate(&ctx->graph, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                ctx->graph = nullptr;
                cudaGetLastError();
                return fail(REG_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
            }
            ctx->graph_key = key;
            ctx->graph_captures += 1;
            ctx->last.graph_captures = 1;
        }
        const int t0 = timing_mark(ctx, s);
        CU(cudaGraphLaunch(ctx->graph, s));
        ctx->op_pairs.push_back({t0, timing_mark(ctx, s)});
        ctx->last.op_launches += n_ops;
        return REG_OK;
    }
    if (exec == REG_EXEC_PERSISTENT) {
        // consumers (CSR by node) and pending counts
        // an operator waits for the inputs that operators of this launch produce (inputs of an
        // earlier launch on the same stream are complete)
        std::vector<int> pending(n_ops, 0), cstart(p.n_nodes + 1, 0), cons, node_made(p.n_nodes, 0);
        std::vector<int> ready;
        for (int e = 0; e < n_ops; ++e) node_made[plan.ops[e].out] = 1;
        for (int e = 0; e < n_ops; ++e) {
            const OpDesc &op = plan.ops[e];
            for (int v : {op.left, op.right})
                if (v >= 0 && node_made[v]) {
                    pending[e] += 1;
                    cstart[v + 1]++;
                }
            if (pending[e] == 0) ready.push_back(e);
        }
        for (int v = 0; v < p.n_nodes; ++v) cstart[v + 1] += cstart[v];
        cons.assign(std::max(1, cstart[p.n_nodes]), 0);
        std::vector<int> fillp(cstart.begin(), cstart.end() - 1);
        for (int e = 0; e < n_ops; ++e) {
            const OpDesc &op = plan.ops[e];
            for (int v : {op.left, op.right})
                if (v >= 0 && node_made[v]) cons[fillp[v]++] = e;
        }
        // Host-side fault injection for tests: REG_FAULT_INJECT=stuck_op keeps the last operator
        // waiting for an input that never arrives, so the device queue's bounded wait must give
        // up and report REG_ETIMEOUT; REG_QUEUE_TIMEOUT_MS shortens that wait.
        const char *inj = getenv("REG_FAULT_INJECT");
        if (inj && strcmp(inj, "stuck_op") == 0 && n_ops > 0) {
            const int last = n_ops - 1;
            if (pending[last] == 0) ready.erase(std::remove(ready.begin(), ready.end(), last), ready.end());
            pending[last] += 1;
        }
        // priority classes: bottom level with the cost of an operator estimated from its span (the
        // frames it registers across; evaluations grow with the drift to undo), ranked into
        // kQueueClasses equal groups.  Consumers come after their producers in the plan.
        std::vector<double> blev(n_ops);
        for (int e = n_ops - 1; e >= 0; --e) {
            const OpDesc &op = plan.ops[e];
            double tail = 0.0;
            for (int q = cstart[op.out]; q < cstart[op.out + 1]; ++q) tail = std::max(tail, blev[cons[q]]);
            blev[e] = 1.0 + std::abs(op.tmpl - op.ref) / 64.0 + tail;
        }
        // the mock operator (Sec. 5.1, microseconds each) takes the plain FIFO: the paper's dynamic
        // scheduling without priorities, and no polling of every class
        const int n_class = p.cfg.mode == kModeMock ? 1 : kQueueClasses;
        std::vector<int> order(n_ops), op_class(n_ops), class_cnt(kQueueClasses, 0);
        for (int e = 0; e < n_ops; ++e) order[e] = e;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return blev[a] > blev[b]; });
        for (int r = 0; r < n_ops; ++r) {
            const int c = (int)((long long)r * n_class / std::max(1, n_ops));
            op_class[order[r]] = c;
            class_cnt[c] += 1;
        }
        // class_off[c] .. class_off[c + 1]: the slots of class c (kQueueClasses + 1 offsets)
        std::vector<int> class_off(kQueueClasses + 1, 0), class_tail(kQueueClasses, 0);
        for (int c = 1; c <= kQueueClasses; ++c) class_off[c] = class_off[c - 1] + class_cnt[c - 1];
        std::vector<int> slots(n_ops, -1);
        for (int e : ready) {
            const int c = op_class[e];
            slots[class_off[c] + class_tail[c]++] = e;
        }
        std::vector<int> cls_buf(op_class);
        cls_buf.insert(cls_buf.end(), class_off.begin(), class_off.end());
        CHECK(ctx->q_slots.reserve(sizeof(int) * std::max(1, n_ops)));
        CHECK(ctx->q_pending.reserve(sizeof(int) * std::max(1, n_ops)));
        CHECK(ctx->q_cons.reserve(sizeof(int) * cons.size()));
        CHECK(ctx->q_cons_start.reserve(sizeof(int) * cstart.size()));
        CHECK(ctx->q_class.reserve(sizeof(int) * cls_buf.size()));
        CHECK(ctx->q_ctr.reserve(sizeof(int) * (2 * kQueueClasses + 2)));
        CU(cudaMemcpyAsync(ctx->q_slots.ptr, slots.data(), sizeof(int) * n_ops, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(ctx->q_pending.ptr, pending.data(), sizeof(int) * n_ops, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(ctx->q_cons.ptr, cons.data(), sizeof(int) * cons.size(), cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(ctx->q_cons_start.ptr, cstart.data(), sizeof(int) * cstart.size(), cudaMemcpyHostToDevice,
                           s));
        CU(cudaMemcpyAsync(ctx->q_class.ptr, cls_buf.data(), sizeof(int) * cls_buf.size(), cudaMemcpyHostToDevice, s));
        // counters: heads, tails, done, claimed
        std::vector<int> ctr(2 * kQueueClasses + 2, 0);
        for (int c = 0; c < kQueueClasses; ++c) ctr[kQueueClasses + c] = class_tail[c];
        CU(cudaMemcpyAsync(ctx->q_ctr.ptr, ctr.data(), sizeof(int) * ctr.size(), cudaMemcpyHostToDevice, s));
        p.queue.head = ctx->q_ctr.as<int>();
        p.queue.tail = ctx->q_ctr.as<int>() + kQueueClasses;
        p.queue.done = ctx->q_ctr.as<int>() + 2 * kQueueClasses;
        p.queue.claimed = ctx->q_ctr.as<int>() + 2 * kQueueClasses + 1;
        p.queue.n_class = n_class;
        p.queue.op_class = ctx->q_class.as<int>();
        p.queue.class_off = ctx->q_class.as<int>() + n_ops;
        p.queue.slots = ctx->q_slots.as<int>();
        p.queue.pending = ctx->q_pending.as<int>();
        p.queue.consumers = ctx->q_cons.as<int>();
        p.queue.cons_start = ctx->q_cons_start.as<int>();
        p.queue.timeout_ns = 20LL * 1000 * 1000 * 1000;
        if (const char *t = getenv("REG_QUEUE_TIMEOUT_MS")) {
            long long ms = atoll(t);
            if (ms > 0) p.queue.timeout_ns = ms * 1000 * 1000;
        }
        const int C = tuned.cluster > 0 ? tuned.cluster : 8;
        note_shape(ctx, p, C);
        int workers = ctx->cfg.workers;
        if (workers <= 0) {
            // one worker per cluster slot the device holds at once; extra workers would only wait
            const int resident = persistent_resident_clusters(p, storage, C);
            workers = resident > 0 ? resident : std::max(1, 2 * ctx->num_sms / C);
        }
        workers = std::max(1, std::min(workers, n_ops));
        p.op_base = 0;
        int e0 = timing_mark(ctx, s);
        CU(launch_persistent(p, storage, C, workers, s));
        ctx->op_pairs.push_back({e0, timing_mark(ctx, s)});
        ctx->last.op_launches += 1;
        return REG_OK;
    }
    return fail(REG_EINVAL, "exec %d", exec);
}

// The operators [b, e) of a plan (whole DAG depths) as a plan of their own, with Params whose
// descriptors and stats start at operator b.
void sub_plan(const ScanPlan &plan, const Params &p, int b, int e, ScanPlan &sub, Params &q)
{
    sub.ops.assign(plan.ops.begin() + b, plan.ops.begin() + e);
    sub.user_index.assign(plan.user_index.begin() + b, plan.user_index.begin() + e);
    sub.depth_start.clear();
    for (int v : plan.depth_start)
        if (v >= b && v <= e && (sub.depth_start.empty() || v - b != sub.depth_start.back()))
            sub.depth_start.push_back(v - b);
    sub.n_nodes = plan.n_nodes;
    sub.out_nodes = plan.out_nodes;
    q = p;
    q.ops = p.ops + b;
    q.stats = p.stats + b;
    q.n_ops = e - b;
}

// REG_EXEC_SPLIT_PHASES: every A leaf (DAG depth 0) runs to completion before the first B,
// and the two phases are timed separately (the paper's "full" vs "scan" registration).
int execute_split(reg_ctx *ctx, const ScanPlan &plan, Params &p, int exec, const TileShape &tuned, cudaStream_t s)
{
    const int n_ops = (int)plan.ops.size();
    const int nl = plan.depth_start.size() > 1 ? plan.depth_start[1] : n_ops;
    const size_t k0 = ctx->op_pairs.size();
    ctx->split_at = k0;
    for (int phase = 0; phase < 2; ++phase) {
        const int b = phase == 0 ? 0 : nl, e = phase == 0 ? nl : n_ops;
        if (b == e) continue;
        ScanPlan sub;
        Params q;
        sub_plan(plan, p, b, e, sub, q);
        CHECK(execute(ctx, sub, q, exec, tuned, s));
        if (phase == 0) ctx->split_at = ctx->op_pairs.size();
    }
    ctx->split_from = k0;
    ctx->last.leaf_ops = nl;
    ctx->last.dag_ops = n_ops - nl;
    return REG_OK;
}

int copy_out(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (!dst) return REG_OK;
    CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    return REG_OK;
}

}  // namespace

// ------------------------------------------------------------------ reg_scan
namespace {

// S independent series of N frames in one plan: series s owns frames s N .. s N + N - 1 and
// nodes s n_nodes .. (s + 1) n_nodes - 1 of the single-series plan; operators are grouped by
// DAG depth across series, so every executor runs the series side by side.
int plan_batch(int S, int N, const Dag &d, ScanPlan &p)
{
    ScanPlan one;
    CHECK(plan_scan(N, d, one));
    if (S == 1) {
        p = std::move(one);
        return REG_OK;
    }
    const int nops = (int)one.ops.size(), nn = one.n_nodes, n = N - 1;
    p.n_nodes = S * nn;
    p.node_i.resize(p.n_nodes);
    p.node_k.resize(p.n_nodes);
    p.out_nodes.resize((size_t)S * n);
    for (int sr = 0; sr < S; ++sr) {
        for (int v = 0; v < nn; ++v) {
            p.node_i[sr * nn + v] = one.node_i[v] + sr * N;
            p.node_k[sr * nn + v] = one.node_k[v] + sr * N;
        }
        for (int i = 0; i < n; ++i) p.out_nodes[(size_t)sr * n + i] = one.out_nodes[i] + sr * nn;
    }
    const int nd = (int)one.depth_start.size() - 1;
    p.depth_start.assign(nd + 1, 0);
    p.ops.clear();
    p.user_index.clear();
    for (int dpt = 0; dpt < nd; ++dpt) {
        p.depth_start[dpt] = (int)p.ops.size();
        for (int sr = 0; sr < S; ++sr)
            for (int e = one.depth_start[dpt]; e < one.depth_start[dpt + 1]; ++e) {
                OpDesc op = one.ops[e];
                op.ref += sr * N;
                op.tmpl += sr * N;
                if (op.left >= 0) op.left += sr * nn;
                if (op.right >= 0) op.right += sr * nn;
                op.out += sr * nn;
                p.ops.push_back(op);
                p.user_index.push_back(sr * nops + one.user_index[e]);
            }
    }
    p.depth_start[nd] = (int)p.ops.size();
    return REG_OK;
}

int scan_impl(reg_ctx_t *ctx, const float *frames, int S, int N, int W, int H, int pitch, int schedule, int exec,
              reg_elem_t *out, float *fields_out, reg_stats_t *per_op, void *stream)
{
    if (!ctx) return fail(REG_EINVAL, "ctx is NULL");
    if (!frames || !out) return fail(REG_EINVAL, "frames/out is NULL");
    if (S < 1) return fail(REG_EINVAL, "need S >= 1 series, got %d", S);
    if (N < 2) return fail(REG_EINVAL, "need N >= 2 frames, got %d", N);
    if (pitch < W) return fail(REG_EINVAL, "pitch %d < W %d", pitch, W);
    const bool split = (exec & REG_EXEC_SPLIT_PHASES) != 0;
    exec &= ~REG_EXEC_SPLIT_PHASES;
    if (exec != REG_EXEC_PLAIN && exec != REG_EXEC_LEVEL && exec != REG_EXEC_PERSISTENT && exec != REG_EXEC_GRAPH)
        return fail(REG_EINVAL, "exec %d", exec);
    if (split && exec == REG_EXEC_GRAPH)
        return fail(REG_EINVAL, "REG_EXEC_SPLIT_PHASES is not available with REG_EXEC_GRAPH");
    std::lock_guard<std::mutex> lock(ctx->mu);
    CU(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    Geometry g;
    CHECK(geometry(W, H, ctx->cfg.levels, g));
    if (ctx->cfg.mode == REG_NONRIGID) {
        GridDims gd;
        CHECK(grid_dims(W, H, ctx->cfg.grid, ctx->cfg.levels, gd));
    }
    Dag dag;
    if (schedule == REG_SCHED_BLELLOCH)
        return fail(REG_EINVAL, "the Blelloch scan is exclusive: available to reg_mock_scan, not to registration");
    if (!make_dag(schedule, N - 1, dag)) return fail(REG_EINVAL, "schedule %d", schedule);
    ScanPlan plan;
    CHECK(plan_batch(S, N, dag, plan));
    timing_reset(ctx);
    const int NF = S * N;   // frames of all series

    const float *dframes = frames;
    if (!is_device_ptr(frames)) {
        size_t bytes = sizeof(float) * (size_t)NF * H * pitch;
        CHECK(ctx->frames_dev.reserve(bytes));
        const int c0 = timing_mark(ctx, s);
        const void *mapped = mapped_host_ptr(frames, bytes);
        if (mapped && bytes % 16 == 0 && (uintptr_t)mapped % 16 == 0) {
            CU(launch_stage_copy(ctx->frames_dev.ptr, mapped, bytes, 8 * ctx->num_sms, s));
            ctx->last.h2d_path = 2;
        } else {
            CU(cudaMemcpyAsync(ctx->frames_dev.ptr, frames, bytes, cudaMemcpyHostToDevice, s));
            ctx->last.h2d_path = 1;
        }
        ctx->h2d_pair = {c0, timing_mark(ctx, s)};
        dframes = ctx->frames_dev.as<float>();
    }
    CHECK(build_pyramids(ctx, g, dframes, NF, (size_t)H * pitch, pitch, 0, NF, s));
    CHECK(build_level_table(ctx, g, NF, s));

    const int n_ops = (int)plan.ops.size();
    Params p;
    CHECK(prepare_params(ctx, g, NF, plan.n_nodes, n_ops, p, s));
    CU(cudaMemcpyAsync(ctx->ops.ptr, plan.ops.data(), sizeof(OpDesc) * n_ops, cudaMemcpyHostToDevice, s));
    const TileShape tuned = tuned_shape(ctx, W, H, exec, NF);
    if (split) {
        ctx->split = true;
        CHECK(execute_split(ctx, plan, p, exec, tuned, s));
    } else {
        CHECK(execute(ctx, plan, p, exec, tuned, s));
    }
    CU(cudaGetLastError());
    CHECK(check_device_status(ctx, s));

    // results (element indices are series-local: frame s N + i is frame i of series s)
    const int n = N - 1, nout = S * n, nops1 = n_ops / S;
    std::vector<double> th((size_t)3 * plan.n_nodes);
    CU(cudaMemcpyAsync(th.data(), p.node_theta, sizeof(double) * th.size(), cudaMemcpyDeviceToHost, s));
    std::vector<OpStats> st(n_ops);
    CU(cudaMemcpyAsync(st.data(), p.stats, sizeof(OpStats) * n_ops, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    std::vector<reg_elem_t> el(nout);
    for (int q = 0; q < nout; ++q) {
        const int node = plan.out_nodes[q], base = (q / n) * N;
        el[q].i = plan.node_i[node] - base;
        el[q].k = plan.node_k[node] - base;
        el[q].alpha = (float)th[3 * node];
        el[q].gx = (float)th[3 * node + 1];
        el[q].gy = (float)th[3 * node + 2];
    }
    CHECK(copy_out(out, el.data(), sizeof(reg_elem_t) * nout, s));
    ctx->last_n = 0;
    if (ctx->cfg.mode == REG_NONRIGID) {
        CHECK(ctx->node_ids.reserve(sizeof(int) * nout));
        CU(cudaMemcpyAsync(ctx->node_ids.ptr, plan.out_nodes.data(), sizeof(int) * nout, cudaMemcpyHostToDevice, s));
    }
    if (ctx->cfg.mode == REG_NONRIGID && fields_out) {
        // dense finest-level fields of the prefixes, written by one kernel
        const size_t fb = sizeof(float) * 2 * (size_t)W * H;
        float *dst = (float *)fields_out;
        const bool direct = is_device_ptr(fields_out);
        if (!direct) {
            CHECK(ctx->frames_dev.reserve(fb * nout + (size_t)sizeof(float) * NF * H * pitch));
            dst = (float *)((char *)ctx->frames_dev.ptr + (size_t)sizeof(float) * NF * H * pitch);
        }
        CU(launch_grid_dense(p.node_grid, ctx->node_ids.as<int>(), nout, p.gnx, p.gny, p.gs, W, H, dst, s));
        if (!direct) CU(cudaMemcpyAsync(fields_out, dst, fb * nout, cudaMemcpyDeviceToHost, s));
    }
    if (per_op) {
        for (int e = 0; e < n_ops; ++e) {
            reg_stats_t r;
            memcpy(&r, &st[e], sizeof(r));
            const int base = (plan.user_index[e] / nops1) * N;
            r.i -= base;
            r.k -= base;
            per_op[plan.user_index[e]] = r;
        }
    }
    CU(cudaStreamSynchronize(s));
    timing_resolve(ctx);
    for (int e = 0; e < n_ops; ++e)
        if (st[e].status != kDevOk) return fail(REG_EINVAL, "operator %d failed on the device (%d)", e, st[e].status);
    if (ctx->cfg.mode == REG_NONRIGID) {
        ctx->last_n = nout;
        ctx->last_gnx = p.gnx;
        ctx->last_gny = p.gny;
        ctx->last_op_nodes.assign(n_ops, 0);
        for (int e = 0; e < n_ops; ++e) ctx->last_op_nodes[plan.user_index[e]] = plan.ops[e].out;
    }
    return REG_OK;
}

}  // namespace

extern "C" int reg_scan(reg_ctx_t *ctx, const float *frames, int N, int W, int H, int pitch, int schedule, int exec,
                        reg_elem_t *out, float *fields_out, reg_stats_t *per_op, void *stream)
{
    return scan_impl(ctx, frames, 1, N, W, H, pitch, schedule, exec, out, fields_out, per_op, stream);
}

extern "C" int reg_scan_batch(reg_ctx_t *ctx, const float *frames, int S, int N, int W, int H, int pitch,
                              int schedule, int exec, reg_elem_t *out, float *fields_out, reg_stats_t *per_op,
                              void *stream)
{
    return scan_impl(ctx, frames, S, N, W, H, pitch, schedule, exec, out, fields_out, per_op, stream);
}

// ------------------------------------------------------------------ mock operator
extern "C" int reg_mock_scan(reg_ctx_t *ctx, int n, int schedule, int exec, const double *values, const float *op_us,
                             double *prefix, double *elapsed_ms)
{
    if (!ctx || !values || !op_us || !prefix) return fail(REG_EINVAL, "NULL argument");
    if (n < 1) return fail(REG_EINVAL, "need n >= 1 elements");
    if (exec != REG_EXEC_PLAIN && exec != REG_EXEC_LEVEL && exec != REG_EXEC_PERSISTENT)
        return fail(REG_EINVAL, "exec %d (plain, level or persistent)", exec);
    Dag dag;
    if (!make_dag(schedule, n, dag)) return fail(REG_EINVAL, "schedule %d", schedule);
    const int m = (int)dag.left.size();
    for (int j = 0; j < m; ++j)
        if (!(op_us[j] >= 0.f && op_us[j] <= 1.0e5f)) return fail(REG_EINVAL, "duration of operator %d not in [0, 1e5] us", j);
    std::lock_guard<std::mutex> lock(ctx->mu);
    CU(cudaSetDevice(ctx->device));
    timing_reset(ctx);
    // plan: the DAG's operators by depth (the identity, node -1, has depth 0)
    ScanPlan plan;
    plan.n_nodes = n + m;
    std::vector<int> depth(plan.n_nodes, 0), op_depth(m);
    std::vector<OpDesc> user(m);
    for (int j = 0; j < m; ++j) {
        const int l = dag.left[j], r = dag.right[j], o = n + j;
        depth[o] = 1 + std::max(l >= 0 ? depth[l] : 0, depth[r]);
        op_depth[j] = depth[o] - 1;
        user[j] = OpDesc{0, 0, l, r, o, -1};
    }
    int maxd = 0;
    for (int v : op_depth) maxd = std::max(maxd, v);
    plan.depth_start.assign(maxd + 2, 0);
    for (int v : op_depth) plan.depth_start[v + 1]++;
    for (int q = 0; q <= maxd; ++q) plan.depth_start[q + 1] += plan.depth_start[q];
    std::vector<int> fill(plan.depth_start.begin(), plan.depth_start.end() - 1);
    plan.ops.resize(m);
    plan.user_index.resize(m);
    for (int j = 0; j < m; ++j) {
        const int e = fill[op_depth[j]]++;
        plan.ops[e] = user[j];
        plan.user_index[e] = j;
    }
    plan.out_nodes = dag.out;
    std::vector<float> us(std::max(1, m));
    for (int e = 0; e < m; ++e) us[e] = op_us[plan.user_index[e]];
    // device state: descriptors, durations, node values (component 0 of node_theta)
    cudaStream_t s = nullptr;
    Params p;
    memset(&p, 0, sizeof(p));
    p.cfg.mode = kModeMock;
    p.n_ops = m;
    p.n_nodes = plan.n_nodes;
    CHECK(ctx->ops.reserve(sizeof(OpDesc) * std::max(1, m)));
    CHECK(ctx->stats.reserve(sizeof(OpStats) * std::max(1, m)));
    CHECK(ctx->node_theta.reserve(sizeof(double) * 3 * plan.n_nodes));
    CHECK(ctx->tmp.reserve(sizeof(float) * us.size()));
    CHECK(ctx->status.reserve(sizeof(int) * 4));
    ctx->last_n = 0;   // the node storage of the last scan is reused here
    p.ops = ctx->ops.as<OpDesc>();
    p.stats = ctx->stats.as<OpStats>();
    p.node_theta = ctx->node_theta.as<double>();
    p.mock_us = ctx->tmp.as<float>();
    p.status = ctx->status.as<int>();
    std::vector<double> th((size_t)3 * plan.n_nodes, 0.0);
    for (int j = 0; j < n; ++j) th[3 * j] = values[j];
    CU(cudaMemcpyAsync(p.node_theta, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, s));
    if (m > 0) {
        CU(cudaMemcpyAsync(ctx->ops.ptr, plan.ops.data(), sizeof(OpDesc) * m, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync((void *)p.mock_us, us.data(), sizeof(float) * m, cudaMemcpyHostToDevice, s));
    }
    CU(cudaMemsetAsync(p.status, 0, sizeof(int) * 4, s));
    const bool timing = ctx->timing;
    ctx->timing = true;
    TileShape one;
    one.cluster = 1;   // one CTA per mock operator
    int rc = REG_OK;
    if (m > 0) rc = execute(ctx, plan, p, exec, one, s);
    if (rc == REG_OK && cudaGetLastError() != cudaSuccess) rc = fail(REG_ECUDA, "mock operator launch failed");
    if (rc == REG_OK) rc = check_device_status(ctx, s);
    if (rc == REG_OK && cudaMemcpyAsync(th.data(), p.node_theta, sizeof(double) * th.size(), cudaMemcpyDeviceToHost,
                                        s) != cudaSuccess)
        rc = fail(REG_ECUDA, "mock scan: copy of the node values");
    if (rc == REG_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = fail(REG_ECUDA, "mock scan: synchronize");
    if (rc == REG_OK) timing_resolve(ctx);   // the events are read while timing is still on
    ctx->timing = timing;
    CHECK(rc);
    for (int i = 0; i < n; ++i) prefix[i] = dag.out[i] >= 0 ? th[3 * dag.out[i]] : 0.0;
    if (elapsed_ms) *elapsed_ms = ctx->last.op_kernel_ms;
    return REG_OK;
}

// ------------------------------------------------------------------ reg_scan_grids / reg_warp
extern "C" int reg_scan_grids(reg_ctx_t *ctx, float *grids_out, int *n_out, void *stream)
{
    if (!ctx || !grids_out) return fail(REG_EINVAL, "ctx/grids_out is NULL");
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (ctx->last_n <= 0) return fail(REG_ESTATE, "no nonrigid scan result on this context");
    CU(cudaSetDevice(ctx->device));
    if (!is_device_ptr(grids_out)) return fail(REG_EINVAL, "grids_out must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    CU(launch_grid_gather(ctx->node_grid.as<float2>(), ctx->node_ids.as<int>(), ctx->last_n,
                          ctx->last_gnx * ctx->last_gny, (float2 *)grids_out, s));
    CU(cudaStreamSynchronize(s));
    if (n_out) *n_out = ctx->last_n;
    return REG_OK;
}

extern "C" int reg_scan_node_grids(reg_ctx_t *ctx, const int32_t *ops, int n, float *grids_out, void *stream)
{
    if (!ctx || !ops || !grids_out || n < 1) return fail(REG_EINVAL, "NULL argument or n < 1");
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (ctx->last_n <= 0) return fail(REG_ESTATE, "no nonrigid scan result on this context");
    CU(cudaSetDevice(ctx->device));
    if (!is_device_ptr(grids_out)) return fail(REG_EINVAL, "grids_out must be device memory");
    std::vector<int> nodes(n);
    for (int q = 0; q < n; ++q) {
        if (ops[q] < 0 || ops[q] >= (int)ctx->last_op_nodes.size())
            return fail(REG_EINVAL, "operator %d not in 0..%zu", ops[q], ctx->last_op_nodes.size() - 1);
        nodes[q] = ctx->last_op_nodes[ops[q]];
    }
    cudaStream_t s = (cudaStream_t)stream;
    CHECK(ctx->pick_ids.reserve(sizeof(int) * n));
    CU(cudaMemcpyAsync(ctx->pick_ids.ptr, nodes.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CU(launch_grid_gather(ctx->node_grid.as<float2>(), ctx->pick_ids.as<int>(), n, ctx->last_gnx * ctx->last_gny,
                          (float2 *)grids_out, s));
    CU(cudaStreamSynchronize(s));
    return REG_OK;
}

extern "C" int reg_warp(reg_ctx_t *ctx, const float *frames, int N, int W, int H, int pitch,
                        const reg_elem_t *elems, const float *grids, float *out, float *mean, void *stream)
{
    if (!ctx || !frames) return fail(REG_EINVAL, "ctx/frames is NULL");
    if (!out && !mean) return fail(REG_EINVAL, "out and mean are both NULL");
    if (N < 1) return fail(REG_EINVAL, "need N >= 1 frames, got %d", N);
    if (W < 2 || H < 2 || pitch < W) return fail(REG_EINVAL, "need W, H >= 2 and pitch >= W");
    const bool nonrigid = ctx->cfg.mode == REG_NONRIGID;
    if (N > 1 && !nonrigid && !elems) return fail(REG_EINVAL, "elems is NULL");
    if (N > 1 && nonrigid && !grids) return fail(REG_EINVAL, "grids is NULL");
    std::lock_guard<std::mutex> lock(ctx->mu);
    CU(cudaSetDevice(ctx->device));
    if (!is_device_ptr(frames) || (N > 1 && nonrigid && !is_device_ptr(grids)) || (out && !is_device_ptr(out)) ||
        (mean && !is_device_ptr(mean)))
        return fail(REG_EINVAL, "frames, grids, out and mean must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    WarpJob j;
    memset(&j, 0, sizeof(j));
    j.frames = frames;
    j.N = N;
    j.W = W;
    j.H = H;
    j.pitch = pitch;
    j.mode = ctx->cfg.mode;
    j.out = out;
    j.mean = mean;
    if (nonrigid) {
        GridDims gd;
        CHECK(grid_dims(W, H, ctx->cfg.grid, ctx->cfg.levels, gd));
        j.nx = gd.nx;
        j.ny = gd.ny;
        j.s = gd.s;
        j.grids = (const float2 *)grids;
    }
    // workspace: per-frame parameters and chunk partial sums, then the rigid elements and status
    const size_t wb = warp_workspace_bytes(N, W, H, mean != nullptr);
    const size_t eb = 256 * (((size_t)std::max(1, N - 1) * sizeof(reg_elem_t) + 255) / 256);
    CHECK(ctx->warp_ws.reserve(wb + eb + 256));
    char *ws = (char *)ctx->warp_ws.ptr;
    j.ws = ws;
    j.status = (int *)(ws + wb + eb);
    if (!nonrigid && N > 1) {
        reg_elem_t *de = (reg_elem_t *)(ws + wb);
        CU(cudaMemcpyAsync(de, elems, sizeof(reg_elem_t) * (N - 1), cudaMemcpyDefault, s));
        j.elems = de;
    }
    j.timeout_ns = 2LL * 1000 * 1000 * 1000;
    CU(cudaMemsetAsync(j.status, 0, sizeof(int), s));
    int used_tma = 0;
    CU(launch_warp(j, s, &used_tma));
    int st = 0;
    CU(cudaMemcpyAsync(&st, j.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (st == kDevWaitTimeout) return fail(REG_ETIMEOUT, "a bounded wait on a TMA load gave up");
    memset(&ctx->last, 0, sizeof(ctx->last));
    ctx->last.op_launches = (N > 1 && !nonrigid) + 1 + (mean != nullptr);   // parameter prep, warp, mean
    ctx->last.tma_staged = used_tma;
    return REG_OK;
}

// ------------------------------------------------------------------ reg_pairwise
extern "C" int reg_pairwise(reg_ctx_t *ctx, const float *R, const float *T, int W, int H, int pitch,
                            const reg_elem_t *init, const float *field_in, reg_elem_t *out, float *field_out,
                            reg_stats_t *stats, void *stream)
{
    if (!ctx) return fail(REG_EINVAL, "ctx is NULL");
    if (!R || !T || !out) return fail(REG_EINVAL, "R/T/out is NULL");
    if (pitch < W) return fail(REG_EINVAL, "pitch %d < W %d", pitch, W);
    const bool nonrigid = ctx->cfg.mode == REG_NONRIGID;
    if (nonrigid && !field_out) return fail(REG_EINVAL, "field_out is NULL for nonrigid");
    std::lock_guard<std::mutex> lock(ctx->mu);
    CU(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    Geometry g;
    CHECK(geometry(W, H, ctx->cfg.levels, g));
    timing_reset(ctx);
    ctx->last_n = 0;   // the node storage of the last scan is reused below
    const size_t fbytes = sizeof(float) * (size_t)H * pitch;
    // staged R and T, then (nonrigid) one dense field for the initial guess or the result
    CHECK(ctx->frames_dev.reserve(2 * fbytes + (nonrigid ? sizeof(float) * 2 * (size_t)W * H : 0)));
    float *stage = ctx->frames_dev.as<float>();
    const float *src[2] = {R, T};
    for (int f = 0; f < 2; ++f) {
        CU(cudaMemcpyAsync((char *)stage + f * fbytes, src[f], fbytes, cudaMemcpyDefault, s));
    }
    CHECK(build_pyramids(ctx, g, stage, 2, (size_t)H * pitch, pitch, 0, 2, s));
    CHECK(build_level_table(ctx, g, 2, s));
    Params p;
    CHECK(prepare_params(ctx, g, 2, 2, 1, p, s));
    const bool has_init = nonrigid ? field_in != nullptr : init != nullptr;
    OpDesc op{0, 1, -1, -1, 0, has_init ? 1 : -1};
    CU(cudaMemcpyAsync(ctx->ops.ptr, &op, sizeof(op), cudaMemcpyHostToDevice, s));
    if (has_init) {
        if (nonrigid) {
            // dense initial field -> control values sampled at the control points (node 1)
            const size_t fb = sizeof(float) * 2 * (size_t)W * H;
            float *u = (float *)((char *)ctx->frames_dev.ptr + 2 * fbytes);
            CU(cudaMemcpyAsync(u, field_in, fb, cudaMemcpyDefault, s));
            CU(launch_grid_from_dense(u, W, H, p.gnx, p.gny, p.gs, p.node_grid + (size_t)p.gnx * p.gny, s));
        } else {
            double th[3] = {init->alpha, init->gx, init->gy};
            CU(cudaMemcpyAsync(p.node_theta + 3, th, sizeof(th), cudaMemcpyHostToDevice, s));
            CU(cudaStreamSynchronize(s));
        }
    }
    int C = ctx->cfg.cluster > 0 ? ctx->cfg.cluster : 8;
    p.op_base = 0;
    p.unroll = ctx->cfg.unroll;
    p.minb = ctx->cfg.ctas_per_sm;
    note_shape(ctx, p, C);
    int e0 = timing_mark(ctx, s);
    CU(launch_ops(p, ctx->cfg.storage, C, 1, s));
    ctx->op_pairs.push_back({e0, timing_mark(ctx, s)});
    ctx->last.op_launches += 1;
    CU(cudaGetLastError());
    CHECK(check_device_status(ctx, s));
    double th[3];
    OpStats st;
    CU(cudaMemcpyAsync(th, p.node_theta, sizeof(th), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(&st, p.stats, sizeof(st), cudaMemcpyDeviceToHost, s));
    if (nonrigid) {
        const size_t fb = sizeof(float) * 2 * (size_t)W * H;
        CHECK(ctx->node_ids.reserve(sizeof(int)));
        CU(cudaMemsetAsync(ctx->node_ids.ptr, 0, sizeof(int), s));
        float *u = (float *)((char *)ctx->frames_dev.ptr + 2 * fbytes);
        CU(launch_grid_dense(p.node_grid, ctx->node_ids.as<int>(), 1, p.gnx, p.gny, p.gs, W, H, u, s));
        CHECK(copy_out(field_out, u, fb, s));
    }
    CU(cudaStreamSynchronize(s));
    timing_resolve(ctx);
    out->i = 0;
    out->k = 1;
    out->alpha = (float)th[0];
    out->gx = (float)th[1];
    out->gy = (float)th[2];
    if (stats) memcpy(stats, &st, sizeof(st));
    if (st.status != kDevOk) return fail(REG_EINVAL, "operator failed on the device (%d)", st.status);
    return REG_OK;
}

// ------------------------------------------------------------------ kernel-level entry points
extern "C" int reg_pyramid(reg_ctx_t *ctx, const float *frame, int W, int H, int pitch, int levels, int storage,
                           void *out, void *stream)
{
    if (!ctx || !frame || !out) return fail(REG_EINVAL, "NULL argument");
    if (levels < 1 || levels > kMaxLevels) return fail(REG_EINVAL, "levels %d", levels);
    if (storage != REG_F32 && storage != REG_BF16 && storage != REG_F16) return fail(REG_EINVAL, "storage");
    if (pitch < W) return fail(REG_EINVAL, "pitch < W");
    if (!is_device_ptr(frame) || !is_device_ptr(out)) return fail(REG_EINVAL, "frame and out must be device memory");
    Geometry g;
    CHECK(geometry(W, H, levels, g));
    std::lock_guard<std::mutex> lock(ctx->mu);
    CU(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    PyrOut o;
    memset(&o, 0, sizeof(o));
    size_t off = 0;
    for (int l = 0; l < levels; ++l) {
        o.raw_stride[l] = (size_t)g.W[l] * g.H[l];
        o.raw[l] = (char *)out + off;
        off += o.raw_stride[l] * storage_bytes(storage);
    }
    CU(launch_pyramid(frame, 1, (size_t)H * pitch, W, H, pitch, levels, storage, o, nullptr, s));
    CU(cudaStreamSynchronize(s));
    return REG_OK;
}

extern "C" int reg_energy(reg_ctx_t *ctx, const float *R, const float *T, int W, int H, const double *theta,
                          const float *grid_values, double *energy, double *grad, float *grad_values, void *stream)
{
    if (!ctx || !R || !T || !energy) return fail(REG_EINVAL, "NULL argument");
    const bool nonrigid = ctx->cfg.mode == REG_NONRIGID;
    if (nonrigid ? !grid_values : !theta) return fail(REG_EINVAL, "deformation is NULL");
    if (W < 2 || H < 2) return fail(REG_EINVAL, "W, H >= 2");
    if (nonrigid && (!is_device_ptr(grid_values) || (grad_values && !is_device_ptr(grad_values))))
        return fail(REG_EINVAL, "control values and their gradient must be device memory");
    std::lock_guard<std::mutex> lock(ctx->mu);
    CU(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    reg_config_t saved = ctx->cfg;
    ctx->last_n = 0;   // the node storage of the last scan is reused below
    ctx->cfg.levels = 1;
    ctx->cfg.storage = REG_F32;
    Geometry g;
    int rc = geometry(W, H, 1, g);
    const size_t fbytes = sizeof(float) * (size_t)W * H;
    Params p;
    if (rc == REG_OK) rc = ctx->frames_dev.reserve(2 * fbytes);
    if (rc == REG_OK) {
        float *stage = ctx->frames_dev.as<float>();
        cudaMemcpyAsync(stage, R, fbytes, cudaMemcpyDefault, s);
        cudaMemcpyAsync((char *)stage + fbytes, T, fbytes, cudaMemcpyDefault, s);
        rc = build_pyramids(ctx, g, stage, 2, (size_t)W * H, W, 0, 2, s);
    }
    if (rc == REG_OK) rc = build_level_table(ctx, g, 2, s);
    if (rc == REG_OK) rc = prepare_params(ctx, g, 2, 1, 1, p, s);
    if (rc == REG_OK) rc = ctx->tmp.reserve(sizeof(double) * 8);
    if (rc == REG_OK) {
        double *dv = ctx->tmp.as<double>();
        if (!nonrigid) cudaMemcpyAsync(dv + 4, theta, sizeof(double) * 3, cudaMemcpyHostToDevice, s);
        cudaError_t e = launch_energy(p, REG_F32, dv + 4, (const float2 *)grid_values, dv, (float2 *)grad_values, s);
        double res[4] = {0, 0, 0, 0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(res, dv, sizeof(res), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(REG_ECUDA, "energy kernel: %s", cudaGetErrorString(e));
        else {
            *energy = res[0];
            if (grad && !nonrigid) { grad[0] = res[1]; grad[1] = res[2]; grad[2] = res[3]; }
        }
    }
    ctx->cfg = saved;
    return rc;
}

extern "C" int reg_grid_dims(int W, int H, int grid, int levels, int *nx, int *ny, int *spacing)
{
    if (levels < 1 || levels > kMaxLevels) return fail(REG_EINVAL, "levels %d", levels);
    GridDims g;
    CHECK(grid_dims(W, H, grid, levels, g));
    if (nx) *nx = g.nx;
    if (ny) *ny = g.ny;
    if (spacing) *spacing = g.s;
    return REG_OK;
}

extern "C" int reg_compose_grid(reg_ctx_t *ctx, const float *q1, const float *q2, int W, int H, float *out,
                                void *stream)
{
    if (!ctx || !q1 || !q2 || !out) return fail(REG_EINVAL, "NULL argument");
    if (W < 2 || H < 2) return fail(REG_EINVAL, "W, H >= 2");
    if (!is_device_ptr(q1) || !is_device_ptr(q2) || !is_device_ptr(out))
        return fail(REG_EINVAL, "q1, q2 and out must be device memory");
    GridDims g;
    CHECK(grid_dims(W, H, ctx->cfg.grid, ctx->cfg.levels, g));
    CU(cudaSetDevice(ctx->device));
    CU(launch_grid_compose((const float2 *)q1, (const float2 *)q2, g.nx, g.ny, g.s, (float2 *)out,
                           (cudaStream_t)stream));
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    return REG_OK;
}

// ------------------------------------------------------------------ measurement
extern "C" int reg_ctx_set_timing(reg_ctx_t *ctx, int enable)
{
    if (!ctx) return fail(REG_EINVAL, "ctx is NULL");
    ctx->timing = enable != 0;
    return REG_OK;
}

extern "C" int reg_ctx_last_timing(reg_ctx_t *ctx, reg_timing_t *out)
{
    if (!ctx || !out) return fail(REG_EINVAL, "NULL argument");
    *out = ctx->last;
    return REG_OK;
}

// ------------------------------------------------------------------ autotuner
extern "C" int reg_autotune(reg_ctx_t *ctx, const float *frames, int N, int W, int H, int pitch, int schedule,
                            int exec, int *best)
{
    if (!ctx || !frames) return fail(REG_EINVAL, "NULL argument");
    if (N < 2) return fail(REG_EINVAL, "need N >= 2 frames");
    const reg_config_t saved = ctx->cfg;
    const int n = N - 1;
    std::vector<reg_elem_t> out(n);
    // no dense fields while timing: their kernel runs after the scan and costs the same for
    // every candidate, and for long series the buffer would take gigabytes
    float *fields = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return fail(REG_ECUDA, "autotune: cudaEventCreate: %s", cudaGetErrorString(e));
    }
    // time one candidate (the config's fields as set): best of two runs after an untimed one
    auto trial = [&](float &ms_min) {
        ms_min = 1e30f;
        int rc = reg_scan(ctx, frames, N, W, H, pitch, schedule, exec, out.data(), fields, nullptr, s);
        for (int rep = 0; rep < 2 && rc == REG_OK; ++rep) {
            cudaEventRecord(e0, s);
            rc = reg_scan(ctx, frames, N, W, H, pitch, schedule, exec, out.data(), fields, nullptr, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_min = std::min(ms_min, ms);
        }
        return rc;
    };
    // the tuned entry is cleared first, so a candidate's unset fields take the built-in rule
    const auto key = std::make_tuple(W, H, saved.mode, saved.storage, exec, log2_floor(N));
    ctx->tuned.erase(key);
    TileShape bestT;
    int rc = REG_OK;
    float best_ms = 1e30f;
    // 1. CTAs per operator (nonrigid: with either register form), at the default pixels per lane
    const bool nonrigid = saved.mode == REG_NONRIGID;
    const int clusters[] = {1, 2, 4, 8, 16};
    for (int c : clusters) {
        if (saved.cluster > 0 && c != saved.cluster) continue;
        bool stop = false;
        for (int mb : {3, 4}) {
            if (!nonrigid && mb == 4) continue;
            if (nonrigid && saved.ctas_per_sm > 0 && mb != saved.ctas_per_sm) continue;
            ctx->cfg.cluster = c;
            if (nonrigid) ctx->cfg.ctas_per_sm = mb;
            float ms;
            rc = trial(ms);
            if (rc != REG_OK) { stop = true; break; }   // e.g. a cluster size the device cannot schedule
            if (ms < best_ms) {
                best_ms = ms;
                bestT.cluster = c;
                bestT.minb = nonrigid ? mb : 0;
            }
        }
        if (stop) break;
    }
    // 2. nonrigid: the other pixels per lane at that shape
    if (bestT.cluster > 0 && nonrigid) {
        ctx->cfg.cluster = bestT.cluster;
        ctx->cfg.ctas_per_sm = bestT.minb;
        bestT.unroll = saved.unroll > 0 ? saved.unroll : 4;
        if (saved.unroll == 0) {
            ctx->cfg.unroll = 2;
            float ms;
            if (trial(ms) == REG_OK && ms < best_ms) {
                best_ms = ms;
                bestT.unroll = 2;
            }
        }
    }
    ctx->cfg = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bestT.cluster == 0) return rc != REG_OK ? rc : fail(REG_ECUDA, "autotune: no candidate ran");
    ctx->tuned[key] = bestT;
    if (best) *best = bestT.cluster;
    return REG_OK;
}

extern "C" int reg_autotune_get(reg_ctx_t *ctx, int N, int W, int H, int exec, int *cluster, int *unroll,
                                int *ctas_per_sm)
{
    if (!ctx) return fail(REG_EINVAL, "ctx is NULL");
    auto it = ctx->tuned.find(std::make_tuple(W, H, ctx->cfg.mode, ctx->cfg.storage, exec, log2_floor(N)));
    if (it == ctx->tuned.end()) return fail(REG_EINVAL, "no autotuned shape for %dx%d, %d frames, exec %d", W, H, N, exec);
    if (cluster) *cluster = it->second.cluster;
    if (unroll) *unroll = it->second.unroll;
    if (ctas_per_sm) *ctas_per_sm = it->second.minb;
    return REG_OK;
}

extern "C" int reg_autotune_save(reg_ctx_t *ctx, const char *path)
{
    if (!ctx || !path) return fail(REG_EINVAL, "NULL argument");
    FILE *f = fopen(path, "w");
    if (!f) return fail(REG_EINVAL, "cannot write %s", path);
    for (auto &kv : ctx->tuned) {
        int W, H, mode, storage, exec, lg;
        std::tie(W, H, mode, storage, exec, lg) = kv.first;
        fprintf(f, "{\"W\": %d, \"H\": %d, \"mode\": %d, \"storage\": %d, \"exec\": %d, \"log2_frames\": %d, "
                   "\"cluster\": %d, \"unroll\": %d, \"ctas_per_sm\": %d}\n", W, H, mode, storage, exec, lg,
                kv.second.cluster, kv.second.unroll, kv.second.minb);
    }
    fclose(f);
    return REG_OK;
}

extern "C" int reg_autotune_load(reg_ctx_t *ctx, const char *path)
{
    if (!ctx || !path) return fail(REG_EINVAL, "NULL argument");
    FILE *f = fopen(path, "r");
    if (!f) return fail(REG_EINVAL, "cannot read %s", path);
    char line[512];
    int loaded = 0;
    while (fgets(line, sizeof(line), f)) {
        int W, H, mode, storage, exec, lg, c, u = 0, m = 0;
        // lines written before the energy-pass shape was tuned end after "cluster"
        const int got = sscanf(line, "{\"W\": %d, \"H\": %d, \"mode\": %d, \"storage\": %d, \"exec\": %d, "
                                     "\"log2_frames\": %d, \"cluster\": %d, \"unroll\": %d, \"ctas_per_sm\": %d}",
                               &W, &H, &mode, &storage, &exec, &lg, &c, &u, &m);
        if ((got == 7 || got == 9) && (c == 1 || c == 2 || c == 4 || c == 8 || c == 16) &&
            (u == 0 || u == 2 || u == 4) && (m == 0 || m == 3 || m == 4)) {
            TileShape t;
            t.cluster = c;
            t.unroll = u;
            t.minb = m;
            ctx->tuned[std::make_tuple(W, H, mode, storage, exec, lg)] = t;
            ++loaded;
        }
    }
    fclose(f);
    return loaded > 0 ? REG_OK : fail(REG_EINVAL, "no autotune entries in %s", path);
}
