// Streaming service of libreg (reg_stream_*): online registration of frames
// as they arrive, with continuous batching on one GPU.
//
// Each acquisition stream registers frame f_i to its first frame f_0 by the
// sequential recursion of Sec. 3, phi_{0,i} = B(phi_{0,i-1}, A(f_{i-1}, f_i)).
// A service thread (one per context) launches every operator as soon as its
// inputs are complete, one operator per launch on a pool of CUDA streams, so
// the operators of new frames and of other streams run on the device while
// earlier ones are still in flight (continuous batching: the hardware runs the
// concurrent launches side by side).  Frames live in a fixed ring of device
// slots per stream; submit refuses a frame with REG_EBUDGET while every slot is
// in use, and opening a stream is refused when its resident state would exceed
// the context's memory budget.  Results come back in submission order.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "reg_internal.h"
#include "reg_host.h"

using namespace reg;

namespace {

constexpr int kLanes = 32;          // CUDA streams the service launches operators on
constexpr int kSlots = 24;          // frame slots per stream (frames in flight)
// CTAs per operator unless the config sets them (fixed: results do not depend on load).  A
// stream's operators are latency-bound: a frame's result waits for its A, its window operators
// and its prefix B one after another, and a few streams keep only tens of operators in flight, so
// every operator takes the largest cluster (measured on eight mixed streams: 16 CTAs for A and B
// gave p99 21 ms from arrival, A on 4 CTAs and B on 16 gave 1.2 s).
constexpr int kClusterA = 16;
constexpr int kClusterB = 16;
// Operators of one frame slot: A at 0, the look-back windows at 1..log2 k, the prefix at kOpP.
constexpr int kMaxLookbackLog = 3;              // look-back k <= 8
constexpr int kOpsPerSlot = kMaxLookbackLog + 2;
constexpr int kOpP = kOpsPerSlot - 1;

double now_us()
{
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Slot {
    bool used = false;
    long long index = -1;       // frame index within the stream (1 ..)
    uint64_t frame_id = 0;
    double submit_us = 0.0;
    cudaEvent_t ready = nullptr; // pyramid built
    cudaEvent_t ev[kOpsPerSlot] = {};
    bool launched[kOpsPerSlot] = {}, fin[kOpsPerSlot] = {};
    bool emitted = false;
};

}  // namespace

struct reg_stream {
    reg_ctx_t *ctx = nullptr;
    int W = 0, H = 0, L = 0, storage = REG_F32, mode = REG_RIGID;
    int gnx = 0, gny = 0, gs = 0;
    int lookback = 1, nlev = 0;  // look-back k of the online scan and log2 k
    size_t bytes = 0;
    // device memory (owned)
    void *pyr[kMaxLevels] = {};        // levels of every slot (nonrigid: with a border holding the mean)
    void *spyr[kMaxLevels] = {};       // nonrigid: the B-spline model at the pixel centres
    size_t lvl_elems[kMaxLevels] = {};
    int pad = 0;
    int Wl[kMaxLevels] = {}, Hl[kMaxLevels] = {};
    float *stage[2] = {};        // fp32 frames being copied in (two, used in turn)
    cudaEvent_t stage_free[2] = {};   // the pyramid build that read stage[b] is done
    int next_stage = 0;
    float *means = nullptr;      // level means of the frame being staged
    LevelDesc *table = nullptr;  // [kSlots + 1][L]; slot 0 holds f_0
    OpDesc *ops = nullptr;       // [2 (kSlots + 1)]: A of slot s at 2s, B at 2s + 1
    OpStats *stats = nullptr;
    double *theta = nullptr;     // nodes, one per op
    float2 *grid = nullptr;
    float2 *ring = nullptr;      // caller's ring of prefix control grids (reg_stream_grids), or null
    int ring_cap = 0;
    int *status = nullptr;
    // pinned host mirrors
    OpDesc *h_ops = nullptr;
    double *h_theta = nullptr;
    OpStats *h_stats = nullptr;
    cudaStream_t copy = nullptr;     // input copies
    cudaStream_t build = nullptr;    // pyramid builds (after their copy)
    cudaEvent_t copied = nullptr;    // the last submitted frame has been read
    // host state (guarded by the service mutex)
    Slot slots[kSlots + 1];
    long long submitted = 0;     // frames submitted, f_0 included
    bool have_f0 = false;
    cudaEvent_t f0_ready = nullptr;
    std::deque<reg_result_t> results;
    bool closing = false;
    int error = REG_OK;
};

namespace {

struct Service {
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::thread th;
    bool stop = false;
    std::vector<reg_stream *> streams;
    // lanes [0, kLanes/2): B operators at the highest stream priority (each stream's chain
    // phi_{0,i-1} -> phi_{0,i} is its critical path); [kLanes/2, kLanes): A operators at the lowest
    cudaStream_t lanes[kLanes] = {};
    int next_lane_a = 0, next_lane_b = 0;
    int device = 0;
    size_t used_bytes = 0;
};

std::mutex g_services_mu;
std::vector<std::pair<reg_ctx_t *, Service *>> g_services;

Service *service_of(reg_ctx_t *ctx, bool create);

int slot_of(long long index) { return (int)((index - 1) % kSlots) + 1; }

Params stream_params(reg_stream *s)
{
    Params p;
    memset(&p, 0, sizeof(p));
    reg_config_t c = host_config(s->ctx);
    p.cfg.mode = c.mode;
    p.cfg.levels = c.levels;
    p.cfg.max_iter = c.max_iter;
    p.cfg.max_rejects = c.max_rejects;
    p.cfg.tol_grad = c.tol_grad;
    p.cfg.tol_coarse = c.tol_coarse;
    p.cfg.tol_rel_e = c.tol_rel_e;
    p.cfg.armijo_c = c.armijo_c;
    p.cfg.tau0 = c.tau0;
    p.cfg.step_cap = c.step_cap;
    p.cfg.lambda = c.lambda;
    p.cfg.metric = c.metric;
    p.levels = s->table;
    p.n_frames = kSlots + 1;
    p.ops = s->ops;
    p.n_ops = kOpsPerSlot * (kSlots + 1);
    p.node_theta = s->theta;
    p.node_grid = s->grid;
    p.gnx = s->gnx;
    p.gny = s->gny;
    p.gs = s->gs;
    p.n_nodes = kOpsPerSlot * (kSlots + 1);
    p.stats = s->stats;
    p.status = s->status;
    return p;
}

// Launch one operator (op index e) on a service lane; results to pinned memory; event after.
// prefix >= 0: the operator produces phi_{0,prefix}, whose control values go to the caller's ring.
int launch_op(Service *sv, reg_stream *s, int e, const OpDesc &op, cudaEvent_t ev, long long prefix)
{
    cudaStream_t ls;
    if (op.left >= 0) {
        ls = sv->lanes[sv->next_lane_b];
        sv->next_lane_b = (sv->next_lane_b + 1) % (kLanes / 2);
    } else {
        ls = sv->lanes[kLanes / 2 + sv->next_lane_a];
        sv->next_lane_a = (sv->next_lane_a + 1) % (kLanes / 2);
    }
    s->h_ops[e] = op;
    if (cudaMemcpyAsync(s->ops + e, s->h_ops + e, sizeof(OpDesc), cudaMemcpyHostToDevice, ls) != cudaSuccess)
        return REG_ECUDA;
    Params p = stream_params(s);
    p.op_base = e;
    const int C = host_config(s->ctx).cluster > 0 ? host_config(s->ctx).cluster : (op.left >= 0 ? kClusterB : kClusterA);
    if (launch_ops(p, s->storage, C, 1, ls) != cudaSuccess) return REG_ECUDA;
    if (cudaMemcpyAsync(s->h_theta + 3 * e, s->theta + 3 * e, 3 * sizeof(double), cudaMemcpyDeviceToHost, ls) !=
        cudaSuccess)
        return REG_ECUDA;
    if (cudaMemcpyAsync(s->h_stats + e, s->stats + e, sizeof(OpStats), cudaMemcpyDeviceToHost, ls) != cudaSuccess)
        return REG_ECUDA;
    if (prefix >= 0 && s->ring) {
        const size_t nc = (size_t)s->gnx * s->gny;
        if (cudaMemcpyAsync(s->ring + (size_t)(prefix % s->ring_cap) * nc, s->grid + (size_t)e * nc,
                            sizeof(float2) * nc, cudaMemcpyDeviceToDevice, ls) != cudaSuccess)
            return REG_ECUDA;
    }
    if (cudaEventRecord(ev, ls) != cudaSuccess) return REG_ECUDA;
    return REG_OK;
}

bool done(cudaEvent_t e)
{
    cudaError_t r = cudaEventQuery(e);
    if (r == cudaErrorNotReady) return false;
    if (r != cudaSuccess) cudaGetLastError();
    return true;
}

void emit(reg_stream *s, Slot &sl, int node, bool identity)
{
    reg_result_t r;
    memset(&r, 0, sizeof(r));
    r.frame_id = sl.frame_id;
    r.elem.i = 0;
    r.elem.k = (int32_t)sl.index;
    if (!identity) {
        r.elem.alpha = (float)s->h_theta[3 * node];
        r.elem.gx = (float)s->h_theta[3 * node + 1];
        r.elem.gy = (float)s->h_theta[3 * node + 2];
        r.status = s->h_stats[node].status;
    }
    r.submit_us = sl.submit_us;
    r.done_us = now_us();
    s->results.push_back(r);
    sl.emitted = true;
}

// One pass of the service over a stream: launch ready operators, note completions,
// emit results in order, free slots.  Called with the service mutex held.
//
// The online scan with a look-back of k leaves (REG_SCHED_LOOKBACK_k; k = 1 is the sequential
// recursion of Sec. 3): frame i (leaf j = i - 1) brings A_i = A(f_{i-1}, f_i), window operators
// W_m(i) = B(W_{m-1}(i - 2^(m-1)), W_{m-1}(i)) registering f_{i-2^m} to f_i for i >= 2^m
// (W_0 = A), and its prefix P(i) = phi_{0,i}: A_1 for i = 1, B(P(i-1), A_i) for i <= k, else
// B(P(i-k), W_log2k(i)).  k chains of prefixes advance side by side.
void advance(Service *sv, reg_stream *s)
{
    if (s->error != REG_OK) return;
    // frames in index order
    std::vector<Slot *> order;
    for (int q = 1; q <= kSlots; ++q)
        if (s->slots[q].used) order.push_back(&s->slots[q]);
    std::sort(order.begin(), order.end(), [](const Slot *a, const Slot *b) { return a->index < b->index; });
    const int k = s->lookback, m = s->nlev;
    auto frame = [&](long long f) -> Slot * {   // the live slot of frame f >= 1, or null
        Slot *q = &s->slots[slot_of(f)];
        return (q->used && q->index == f) ? q : nullptr;
    };
    auto op_of = [&](long long f, int o) { return kOpsPerSlot * slot_of(f) + o; };
    auto frame_slot = [&](long long f) { return f == 0 ? 0 : slot_of(f); };   // pyramid slot of f_f
    // node of P(f) and whether it is complete
    auto prefix_node = [&](long long f) { return f == 1 ? op_of(1, 0) : op_of(f, kOpP); };
    auto prefix_done = [&](long long f) {
        Slot *q = frame(f);
        return q && (f == 1 ? q->fin[0] : q->fin[kOpP]);
    };
    for (Slot *sl : order) {
        const long long i = sl->index;
        const int si = slot_of(i);
        Slot *prev = i > 1 ? frame(i - 1) : nullptr;
        const bool prev_frame_ready = i == 1 ? done(s->f0_ready) : (prev != nullptr);
        // A(f_{i-1}, f_i)
        if (!sl->launched[0] && done(sl->ready) && prev_frame_ready && (i == 1 || done(prev->ready))) {
            OpDesc op{frame_slot(i - 1), si, -1, -1, op_of(i, 0), -1};
            if (launch_op(sv, s, op_of(i, 0), op, sl->ev[0], i == 1 ? 1 : -1) != REG_OK) { s->error = REG_ECUDA; return; }
            sl->launched[0] = true;
        }
        for (int o = 0; o < kOpsPerSlot; ++o)
            if (sl->launched[o] && !sl->fin[o] && done(sl->ev[o])) sl->fin[o] = true;
        // windows W_lev(i), lev = 1..m, for i >= 2^lev
        for (int lev = 1; lev <= m; ++lev) {
            if (sl->launched[lev] || i < (1LL << lev)) continue;
            const long long h = 1LL << (lev - 1);
            Slot *lf = frame(i - h);
            if (!lf || !lf->fin[lev - 1] || !sl->fin[lev - 1]) continue;
            OpDesc op{frame_slot(i - (1LL << lev)), si, op_of(i - h, lev - 1), op_of(i, lev - 1), op_of(i, lev), -1};
            if (launch_op(sv, s, op_of(i, lev), op, sl->ev[lev], -1) != REG_OK) { s->error = REG_ECUDA; return; }
            sl->launched[lev] = true;
        }
        // the prefix P(i), registering f_i onto f_0
        if (i > 1 && !sl->launched[kOpP]) {
            const long long back = i <= k ? i - 1 : i - k;
            const int win = i <= k ? 0 : m;
            if (prefix_done(back) && sl->fin[win]) {
                OpDesc op{0, si, prefix_node(back), op_of(i, win), op_of(i, kOpP), -1};
                if (launch_op(sv, s, op_of(i, kOpP), op, sl->ev[kOpP], i) != REG_OK) { s->error = REG_ECUDA; return; }
                sl->launched[kOpP] = true;
            }
        }
        // results in submission order
        const bool mine = i == 1 ? sl->fin[0] : sl->fin[kOpP];
        if (mine && !sl->emitted && (i == 1 || (prev && prev->emitted)))
            emit(s, *sl, i == 1 ? op_of(1, 0) : op_of(i, kOpP), false);
    }
    // a frame is done when every operator it brings has completed
    auto frame_done = [&](long long f) {
        Slot *q = frame(f);
        if (!q || !q->fin[0]) return false;
        for (int lev = 1; lev <= m; ++lev)
            if (f >= (1LL << lev) && !q->fin[lev]) return false;
        return f == 1 || q->fin[kOpP];
    };
    // free frame i's slot once frames i+1 .. i+k, the only ones that read its pyramid or nodes, are done
    for (Slot *sl : order) {
        if (!sl->used || !sl->emitted) continue;
        const long long i = sl->index;
        bool free_it = true;
        for (long long f = i + 1; f <= i + k && free_it; ++f) free_it = frame_done(f);
        if (free_it) sl->used = false;
    }
}

void service_loop(Service *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lock(sv->mu);
    while (!sv->stop) {
        for (reg_stream *s : sv->streams) advance(sv, s);
        sv->done_cv.notify_all();
        sv->cv.wait_for(lock, std::chrono::microseconds(50));
    }
}

Service *service_of(reg_ctx_t *ctx, bool create)
{
    std::lock_guard<std::mutex> g(g_services_mu);
    for (auto &pr : g_services)
        if (pr.first == ctx) return pr.second;
    if (!create) return nullptr;
    Service *sv = new Service();
    sv->device = host_device(ctx);
    cudaSetDevice(sv->device);
    int prio_low = 0, prio_high = 0;   // numerically smaller is higher
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_low = prio_high = 0;
    }
    for (int i = 0; i < kLanes; ++i)
        cudaStreamCreateWithPriority(&sv->lanes[i], cudaStreamNonBlocking, i < kLanes / 2 ? prio_high : prio_low);
    sv->th = std::thread(service_loop, sv);
    g_services.push_back({ctx, sv});
    return sv;
}

void free_stream(reg_stream *s)
{
    for (int l = 0; l < kMaxLevels; ++l) {
        if (s->pyr[l]) cudaFree(s->pyr[l]);
        if (s->spyr[l]) cudaFree(s->spyr[l]);
    }
    void *dev[] = {s->stage[0], s->stage[1], s->means, s->table, s->ops, s->stats, s->theta, s->grid, s->status};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (s->h_ops) cudaFreeHost(s->h_ops);
    if (s->h_theta) cudaFreeHost(s->h_theta);
    if (s->h_stats) cudaFreeHost(s->h_stats);
    for (int k = 0; k <= kSlots; ++k) {
        if (s->slots[k].ready) cudaEventDestroy(s->slots[k].ready);
        for (int o = 0; o < kOpsPerSlot; ++o)
            if (s->slots[k].ev[o]) cudaEventDestroy(s->slots[k].ev[o]);
    }
    if (s->f0_ready) cudaEventDestroy(s->f0_ready);
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->build) cudaStreamDestroy(s->build);
    if (s->copied) cudaEventDestroy(s->copied);
    for (int b = 0; b < 2; ++b)
        if (s->stage_free[b]) cudaEventDestroy(s->stage_free[b]);
    delete s;
}

}  // namespace

// Called by reg_ctx_destroy: stop the service thread of the context.
void reg::stop_stream_service(reg_ctx_t *ctx)
{
    Service *sv = nullptr;
    {
        std::lock_guard<std::mutex> g(g_services_mu);
        for (size_t i = 0; i < g_services.size(); ++i)
            if (g_services[i].first == ctx) {
                sv = g_services[i].second;
                g_services.erase(g_services.begin() + i);
                break;
            }
    }
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    sv->th.join();
    for (reg_stream *s : sv->streams) free_stream(s);
    for (int i = 0; i < kLanes; ++i) cudaStreamDestroy(sv->lanes[i]);
    delete sv;
}

extern "C" int reg_stream_open(reg_ctx_t *ctx, int W, int H, reg_stream_t **out)
{
    if (!ctx || !out) return host_fail(REG_EINVAL, "NULL argument");
    *out = nullptr;
    const reg_config_t c = host_config(ctx);
    int Wl[kMaxLevels], Hl[kMaxLevels];
    {
        int w = W, h = H;
        for (int l = 0; l < c.levels; ++l) {
            if (w < 2 || h < 2) return host_fail(REG_EINVAL, "every pyramid level needs at least 2x2 pixels");
            Wl[l] = w;
            Hl[l] = h;
            w = (w + 1) / 2;
            h = (h + 1) / 2;
        }
    }
    int gnx = 0, gny = 0, gs = 0;
    if (c.mode == REG_NONRIGID && c.metric == REG_METRIC_H1)
        return host_fail(REG_EINVAL, "the H1 scalar product is available to reg_scan, reg_scan_batch and reg_pairwise");
    if (c.mode == REG_NONRIGID) {
        int rc = reg_grid_dims(W, H, c.grid, c.levels, &gnx, &gny, &gs);
        if (rc != REG_OK) return rc;
    }
    const size_t sb = c.storage == REG_F32 ? 4 : 2;
    const int pad = c.mode == REG_NONRIGID ? kPad : 0;
    size_t pyr_bytes = 0;
    for (int l = 0; l < c.levels; ++l)
        pyr_bytes += (level_elems(Wl[l], Hl[l], pad) + (pad ? (size_t)Wl[l] * Hl[l] : 0)) * sb;
    const int nops = kOpsPerSlot * (kSlots + 1);
    const size_t bytes = pyr_bytes * (kSlots + 1) + 2 * sizeof(float) * (size_t)W * H + sizeof(LevelDesc) * (kSlots + 1) * c.levels +
                         (sizeof(OpDesc) + sizeof(OpStats) + 3 * sizeof(double)) * nops +
                         sizeof(float2) * (size_t)gnx * gny * nops + 4096;
    Service *sv = service_of(ctx, true);
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        if (c.mem_budget > 0 && sv->used_bytes + bytes > c.mem_budget)
            return host_fail(REG_EBUDGET, "stream needs %zu bytes; %zu of the %zu-byte budget in use", bytes,
                             sv->used_bytes, c.mem_budget);
        sv->used_bytes += bytes;
    }
    if (cudaSetDevice(host_device(ctx)) != cudaSuccess) return host_fail(REG_ECUDA, "cudaSetDevice");
    reg_stream *s = new reg_stream();
    s->ctx = ctx;
    s->W = W;
    s->H = H;
    s->L = c.levels;
    s->storage = c.storage;
    s->mode = c.mode;
    s->gnx = gnx;
    s->gny = gny;
    s->gs = gs;
    s->bytes = bytes;
    bool ok = true;
    s->pad = pad;
    for (int l = 0; l < c.levels && ok; ++l) {
        s->Wl[l] = Wl[l];
        s->Hl[l] = Hl[l];
        s->lvl_elems[l] = level_elems(Wl[l], Hl[l], pad);
        ok = cudaMalloc(&s->pyr[l], s->lvl_elems[l] * sb * (kSlots + 1)) == cudaSuccess;
        if (ok && pad) ok = cudaMalloc(&s->spyr[l], (size_t)Wl[l] * Hl[l] * sb * (kSlots + 1)) == cudaSuccess;
    }
    for (int b = 0; b < 2 && ok; ++b) ok = cudaMalloc(&s->stage[b], sizeof(float) * (size_t)W * H) == cudaSuccess;
    ok = ok && cudaMalloc(&s->means, sizeof(float) * kMaxLevels) == cudaSuccess;
    ok = ok && cudaMalloc(&s->table, sizeof(LevelDesc) * (kSlots + 1) * c.levels) == cudaSuccess;
    ok = ok && cudaMalloc(&s->ops, sizeof(OpDesc) * nops) == cudaSuccess;
    ok = ok && cudaMalloc(&s->stats, sizeof(OpStats) * nops) == cudaSuccess;
    ok = ok && cudaMalloc(&s->theta, sizeof(double) * 3 * nops) == cudaSuccess;
    ok = ok && cudaMalloc(&s->status, sizeof(int) * 4) == cudaSuccess;
    if (ok && gnx > 0) ok = cudaMalloc(&s->grid, sizeof(float2) * (size_t)gnx * gny * nops) == cudaSuccess;
    ok = ok && cudaMallocHost(&s->h_ops, sizeof(OpDesc) * nops) == cudaSuccess;
    ok = ok && cudaMallocHost(&s->h_theta, sizeof(double) * 3 * nops) == cudaSuccess;
    ok = ok && cudaMallocHost(&s->h_stats, sizeof(OpStats) * nops) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&s->build, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&s->copied, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaEventCreateWithFlags(&s->stage_free[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventRecord(s->stage_free[b], s->build) == cudaSuccess;
    for (int k = 0; k <= kSlots && ok; ++k) {
        ok = cudaEventCreateWithFlags(&s->slots[k].ready, cudaEventDisableTiming) == cudaSuccess;
        for (int o = 0; o < kOpsPerSlot && ok; ++o)
            ok = cudaEventCreateWithFlags(&s->slots[k].ev[o], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaEventCreateWithFlags(&s->f0_ready, cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaMemset(s->status, 0, sizeof(int) * 4) == cudaSuccess &&
                 cudaMemset(s->stats, 0, sizeof(OpStats) * nops) == cudaSuccess;
    if (ok) {
        // the level table of every slot: fixed pointers and sizes; each submit writes the means
        const size_t sbs = c.storage == REG_F32 ? 4 : 2;
        std::vector<LevelDesc> tab((size_t)(kSlots + 1) * c.levels);
        for (int k = 0; k <= kSlots; ++k)
            for (int l = 0; l < c.levels; ++l) {
                LevelDesc &d = tab[(size_t)k * c.levels + l];
                memset(&d, 0, sizeof(d));
                d.ptr = (char *)s->pyr[l] + (s->lvl_elems[l] * k + level_origin(Wl[l], pad)) * sbs;
                d.W = Wl[l];
                d.H = Hl[l];
                d.pitch = level_pitch(Wl[l], pad);
                d.rptr = pad ? (char *)s->spyr[l] + (size_t)Wl[l] * Hl[l] * sbs * k : d.ptr;
                d.rpitch = pad ? Wl[l] : d.pitch;
            }
        ok = cudaMemcpy(s->table, tab.data(), sizeof(LevelDesc) * tab.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        free_stream(s);
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->used_bytes -= bytes;
        return host_fail(REG_ENOMEM, "stream allocation failed");
    }
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->streams.push_back(s);
    }
    *out = s;
    return REG_OK;
}

extern "C" int reg_stream_submit(reg_stream_t *s, const float *frame, uint64_t frame_id)
{
    if (!s || !frame) return host_fail(REG_EINVAL, "NULL argument");
    Service *sv = service_of(s->ctx, false);
    if (!sv) return host_fail(REG_ESTATE, "stream service is not running");
    const double t_submit = now_us();
    long long index;
    int slot;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        if (s->closing) return host_fail(REG_ESTATE, "stream is closing");
        if (s->error != REG_OK) return host_fail(s->error, "stream failed earlier");
        index = s->submitted;
        slot = index == 0 ? 0 : slot_of(index);
        if (index > 0 && s->slots[slot].used) return host_fail(REG_EBUDGET, "all %d frame slots are in flight", kSlots);
    }
    if (cudaSetDevice(host_device(s->ctx)) != cudaSuccess) return host_fail(REG_ECUDA, "cudaSetDevice");
    // copy the frame in and build its pyramid (the caller's buffer is free on return)
    const size_t fb = sizeof(float) * (size_t)s->W * s->H;
    const size_t sb = s->storage == REG_F32 ? 4 : 2;
    PyrOut o;
    memset(&o, 0, sizeof(o));
    o.pad = s->pad;
    for (int l = 0; l < s->L; ++l) {
        o.raw[l] = (char *)s->pyr[l] + s->lvl_elems[l] * sb * slot;
        o.raw_stride[l] = s->lvl_elems[l];
        if (s->pad) {
            o.smooth_stride[l] = (size_t)s->Wl[l] * s->Hl[l];
            o.smooth[l] = (char *)s->spyr[l] + o.smooth_stride[l] * sb * slot;
        }
    }
    // the copy reads the caller's frame into one of two staging buffers (once the build that last
    // read that buffer is done); the pyramid is built on its own stream after the copy, and only
    // the copy is waited for here
    const int b = s->next_stage;
    s->next_stage ^= 1;
    cudaError_t e = cudaStreamWaitEvent(s->copy, s->stage_free[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->stage[b], frame, fb, cudaMemcpyDefault, s->copy);
    if (e == cudaSuccess) e = cudaEventRecord(s->copied, s->copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->build, s->copied, 0);
    if (e == cudaSuccess)
        e = launch_pyramid(s->stage[b], 1, (size_t)s->W * s->H, s->W, s->H, s->W, s->L, s->storage, o, s->means,
                           s->build);
    if (e == cudaSuccess) e = launch_set_level_means(s->table + (size_t)slot * s->L, s->means, s->L, s->build);
    if (e == cudaSuccess && index == 0 && s->ring)   // phi_{0,0} is the identity
        e = cudaMemsetAsync(s->ring, 0, sizeof(float2) * (size_t)s->gnx * s->gny, s->build);
    cudaEvent_t ready = index == 0 ? s->f0_ready : s->slots[slot].ready;
    if (e == cudaSuccess) e = cudaEventRecord(s->stage_free[b], s->build);
    if (e == cudaSuccess) e = cudaEventRecord(ready, s->build);
    if (e == cudaSuccess) e = cudaEventSynchronize(s->copied);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return host_fail(REG_ECUDA, "staging the frame failed: %s", cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        s->submitted = index + 1;
        if (index == 0) {
            s->have_f0 = true;
            reg_result_t r;
            memset(&r, 0, sizeof(r));
            r.frame_id = frame_id;
            r.submit_us = t_submit;
            r.done_us = now_us();
            s->results.push_back(r);   // phi_{0,0} is the identity
        } else {
            Slot &sl = s->slots[slot];
            sl.used = true;
            sl.index = index;
            sl.frame_id = frame_id;
            sl.submit_us = t_submit;
            for (int o = 0; o < kOpsPerSlot; ++o) sl.launched[o] = sl.fin[o] = false;
            sl.emitted = false;
        }
    }
    sv->cv.notify_all();
    return REG_OK;
}

extern "C" int reg_stream_set_lookback(reg_stream_t *s, int k)
{
    if (!s) return host_fail(REG_EINVAL, "NULL stream");
    if (k != 1 && k != 2 && k != 4 && k != 8) return host_fail(REG_EINVAL, "look-back %d not in {1, 2, 4, 8}", k);
    Service *sv = service_of(s->ctx, false);
    if (!sv) return host_fail(REG_ESTATE, "stream service is not running");
    std::lock_guard<std::mutex> lock(sv->mu);
    if (s->submitted > 0) return host_fail(REG_ESTATE, "set the look-back before the first submit");
    s->lookback = k;
    s->nlev = k == 1 ? 0 : (k == 2 ? 1 : (k == 4 ? 2 : 3));
    return REG_OK;
}

extern "C" int reg_stream_grids(reg_stream_t *s, float *ring, int capacity)
{
    if (!s || !ring || capacity < 1) return host_fail(REG_EINVAL, "NULL ring or capacity < 1");
    if (s->mode != REG_NONRIGID) return host_fail(REG_EINVAL, "control grids exist for REG_NONRIGID streams only");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ring) != cudaSuccess ||
        !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return host_fail(REG_EINVAL, "the ring must be device memory");
    }
    Service *sv = service_of(s->ctx, false);
    if (!sv) return host_fail(REG_ESTATE, "stream service is not running");
    std::lock_guard<std::mutex> lock(sv->mu);
    if (s->submitted > 0) return host_fail(REG_ESTATE, "set the ring before the first submit");
    s->ring = (float2 *)ring;
    s->ring_cap = capacity;
    return REG_OK;
}

extern "C" int reg_stream_poll(reg_stream_t *s, reg_result_t *out, int max, int *n_out, int timeout_us)
{
    if (!s || (!out && max > 0) || !n_out) return host_fail(REG_EINVAL, "NULL argument");
    *n_out = 0;
    Service *sv = service_of(s->ctx, false);
    if (!sv) return host_fail(REG_ESTATE, "stream service is not running");
    std::unique_lock<std::mutex> lock(sv->mu);
    if (s->results.empty() && timeout_us > 0)
        sv->done_cv.wait_for(lock, std::chrono::microseconds(timeout_us), [&] { return !s->results.empty() || s->error; });
    int n = 0;
    while (n < max && !s->results.empty()) {
        out[n++] = s->results.front();
        s->results.pop_front();
    }
    *n_out = n;
    if (s->error != REG_OK) return host_fail(s->error, "stream failed on the device");
    if (n == 0) return host_fail(REG_ETIMEOUT, "no result within %d us", timeout_us);
    return REG_OK;
}

extern "C" int reg_stream_close(reg_stream_t *s)
{
    if (!s) return host_fail(REG_EINVAL, "NULL argument");
    Service *sv = service_of(s->ctx, false);
    if (!sv) return host_fail(REG_ESTATE, "stream service is not running");
    int rc = REG_OK;
    {
        std::unique_lock<std::mutex> lock(sv->mu);
        s->closing = true;
        // every submitted frame finishes; bounded wait
        auto all_done = [&] {
            if (s->error != REG_OK) return true;
            for (int k = 1; k <= kSlots; ++k)
                if (s->slots[k].used && !s->slots[k].emitted) return false;
            return true;
        };
        if (!sv->done_cv.wait_for(lock, std::chrono::seconds(120), all_done)) rc = REG_ETIMEOUT;
        sv->streams.erase(std::remove(sv->streams.begin(), sv->streams.end(), s), sv->streams.end());
        sv->used_bytes -= s->bytes;
    }
    cudaSetDevice(host_device(s->ctx));
    for (int i = 0; i < kLanes; ++i) cudaStreamSynchronize(sv->lanes[i]);
    cudaStreamSynchronize(s->copy);
    cudaStreamSynchronize(s->build);
    free_stream(s);
    return rc == REG_OK ? REG_OK : host_fail(rc, "stream close timed out waiting for its frames");
}
