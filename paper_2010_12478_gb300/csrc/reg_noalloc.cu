// Allocation-free rigid pairwise registration (reg_pairwise_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a
// registration: an acquisition loop with a real-time budget (cudaMalloc and
// cudaFree can synchronise the whole device and stall the detector readout),
// or a host application that hands the GPU a fixed memory pool up front and
// forbids later allocations.  This entry point serves them: everything it
// needs beyond the caller's inputs and outputs lives in one file-scope device
// array, sized once for frames of up to kMaxPixels pixels, which every GPU
// that loads the library holds until the process exits.  The call waits for
// its stream several times (the level means come back to the host between
// the pyramid and the operator), so it is not meant to be recorded into a
// CUDA graph: a caller must not make it while `stream` is being captured.
#include <cstring>
#include <mutex>

#include "reg_host.h"
#include "reg_internal.h"

namespace {

using namespace reg;

// Largest frame the scratch array is sized for (W * H), and the array itself.
constexpr long long kMaxPixels = 1LL << 20;   // e.g. 1024 x 1024
constexpr int kMaxDevices = 64;

// Byte layout: two pyramids (reference, template) of fp32 levels, then the
// small records the operator kernel reads and writes.
constexpr size_t kPyrBytes = 4 * ((kMaxPixels * 4) / 3 + 4 * 4096 * kMaxLevels + 256);
constexpr size_t kOffR = 0;
constexpr size_t kOffT = kPyrBytes;
constexpr size_t kOffTab = 2 * kPyrBytes;
constexpr size_t kOffOp = kOffTab + 256 * ((sizeof(LevelDesc) * 2 * kMaxLevels + 255) / 256);
constexpr size_t kOffStats = kOffOp + 256;
constexpr size_t kOffTheta = kOffStats + 256 * ((sizeof(OpStats) + 255) / 256);
constexpr size_t kOffStatus = kOffTheta + 256;
constexpr size_t kOffMeans = kOffStatus + 256;
constexpr size_t kScratchBytes = kOffMeans + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, resolved on the first call
// made for that device (with the device current).
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mu;

int noalloc_fail(int code, const char *msg)
{
    set_last_error(msg);   // reported by reg_last_error_message()
    return code;
}

// Device memory of `device` itself, or managed memory.  Memory of another GPU is refused: the
// pyramid kernels would read it directly, without peer access.
bool on_device(const void *p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" int reg_pairwise_noalloc(const reg_config_t *cfg, int device, const float *R, const float *T, int W,
                                    int H, int pitch, const reg_elem_t *init, reg_elem_t *out, reg_stats_t *stats,
                                    void *stream)
{
    if (!cfg || !R || !T || !out) return noalloc_fail(REG_EINVAL, "cfg, R, T and out are required");
    // the configuration rules of reg_ctx_create, so that every config reg_pairwise rejects is rejected here
    const int vrc = validate_config(*cfg);
    if (vrc != REG_OK) return vrc;
    if (cfg->mode != REG_RIGID) return noalloc_fail(REG_EINVAL, "the allocation-free entry point is rigid only");
    if (W < 2 || H < 2 || pitch < W) return noalloc_fail(REG_EINVAL, "need W, H >= 2 and pitch >= W");
    if ((long long)W * H > kMaxPixels || W > 4096 || H > 4096)
        return noalloc_fail(REG_EINVAL,
                            "frame too large for the allocation-free scratch: W*H must be <= 1048576 and W, H <= 4096");
    if (device < 0 || device >= kMaxDevices) return noalloc_fail(REG_EINVAL, "device index out of range");

    // level geometry
    int Wl[kMaxLevels], Hl[kMaxLevels];
    size_t off_l[kMaxLevels];
    const size_t sb = cfg->storage == REG_F32 ? 4 : 2;
    size_t used = 0;
    {
        int w = W, h = H;
        for (int l = 0; l < cfg->levels; ++l) {
            if (w < 2 || h < 2) return noalloc_fail(REG_EINVAL, "every pyramid level needs at least 2x2 pixels");
            Wl[l] = w;
            Hl[l] = h;
            off_l[l] = used;
            used += ((size_t)w * h * sb + 255) / 256 * 256;
            w = (w + 1) / 2;
            h = (h + 1) / 2;
        }
    }
    if (used > kPyrBytes) return noalloc_fail(REG_EINVAL, "pyramid does not fit the allocation-free scratch");

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(REG_ECUDA, "no CUDA device");
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(REG_ECUDA, "cudaSetDevice failed");
    }
    int rc = REG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    do {
        if (!on_device(R, device) || !on_device(T, device)) {
            rc = noalloc_fail(REG_EINVAL, "R and T must be device memory of `device` (or managed memory)");
            break;
        }
        if (stream) {
            int sdev = -1;
            if (cudaStreamGetDevice(s, &sdev) != cudaSuccess || sdev != device) {
                cudaGetLastError();
                rc = noalloc_fail(REG_EINVAL, "stream does not belong to `device`");
                break;
            }
        }
        unsigned char *base = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_setup_mu);
            if (!g_scratch_addr[device]) {
                void *p = nullptr;
                cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
                if (e != cudaSuccess || !p) {
                    cudaGetLastError();
                    rc = noalloc_fail(REG_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
                    break;
                }
                g_scratch_addr[device] = p;
            }
            base = (unsigned char *)g_scratch_addr[device];
        }
        LevelDesc *tab = (LevelDesc *)(base + kOffTab);
        OpDesc *op = (OpDesc *)(base + kOffOp);
        OpStats *st = (OpStats *)(base + kOffStats);
        double *theta = (double *)(base + kOffTheta);
        int *status = (int *)(base + kOffStatus);
        float *means = (float *)(base + kOffMeans);

        // the array keeps the previous call's contents: clear what must start at zero
        cudaError_t e = cudaMemsetAsync(st, 0, sizeof(OpStats), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 4 * sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(theta, 0, 6 * sizeof(double), s);
        // pyramids of R and T, then their level means back to the host for the level table
        void *lr[kMaxLevels], *lt[kMaxLevels];
        PyrOut orr, ot;
        memset(&orr, 0, sizeof(orr));
        memset(&ot, 0, sizeof(ot));
        for (int l = 0; l < cfg->levels; ++l) {
            lr[l] = base + kOffR + off_l[l];
            lt[l] = base + kOffT + off_l[l];
            orr.raw[l] = lr[l];
            ot.raw[l] = lt[l];
            orr.raw_stride[l] = ot.raw_stride[l] = (size_t)Wl[l] * Hl[l];
        }
        if (e == cudaSuccess)
            e = launch_pyramid(R, 1, (size_t)H * pitch, W, H, pitch, cfg->levels, cfg->storage, orr, means, s);
        if (e == cudaSuccess)
            e = launch_pyramid(T, 1, (size_t)H * pitch, W, H, pitch, cfg->levels, cfg->storage, ot,
                               means + cfg->levels, s);
        float hmeans[2 * kMaxLevels];
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hmeans, means, sizeof(float) * 2 * cfg->levels, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = noalloc_fail(REG_ECUDA, "pyramid build failed");
            break;
        }
        LevelDesc htab[2 * kMaxLevels];
        for (int f = 0; f < 2; ++f)
            for (int l = 0; l < cfg->levels; ++l) {
                LevelDesc &d = htab[f * cfg->levels + l];
                d.ptr = f == 0 ? lr[l] : lt[l];
                d.rptr = d.ptr;
                d.W = Wl[l];
                d.H = Hl[l];
                d.pitch = Wl[l];
                d.rpitch = Wl[l];
                d.mean = hmeans[f * cfg->levels + l];
            }
        OpDesc hop{0, 1, -1, -1, 0, init ? 1 : -1};
        double hinit[3] = {init ? init->alpha : 0.0, init ? init->gx : 0.0, init ? init->gy : 0.0};
        e = cudaMemcpyAsync(tab, htab, sizeof(LevelDesc) * 2 * cfg->levels, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(op, &hop, sizeof(hop), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && init) e = cudaMemcpyAsync(theta + 3, hinit, sizeof(hinit), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host staging arrays leave scope below
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = noalloc_fail(REG_ECUDA, "staging the operator failed");
            break;
        }
        Params p;
        memset(&p, 0, sizeof(p));
        p.cfg.mode = cfg->mode;
        p.cfg.levels = cfg->levels;
        p.cfg.max_iter = cfg->max_iter;
        p.cfg.max_rejects = cfg->max_rejects;
        p.cfg.tol_grad = cfg->tol_grad;
        p.cfg.tol_coarse = cfg->tol_coarse;
        p.cfg.tol_rel_e = cfg->tol_rel_e;
        p.cfg.armijo_c = cfg->armijo_c;
        p.cfg.tau0 = cfg->tau0;
        p.cfg.step_cap = cfg->step_cap;
        p.cfg.lambda = cfg->lambda;
        p.cfg.metric = cfg->metric;
        p.levels = tab;
        p.n_frames = 2;
        p.ops = op;
        p.n_ops = 1;
        p.op_base = 0;
        p.node_theta = theta;
        p.n_nodes = 2;
        p.stats = st;
        p.status = status;
        const int C = cfg->cluster > 0 ? cfg->cluster : 8;
        e = launch_ops(p, cfg->storage, C, 1, s);
        OpStats hst;
        double hth[3];
        int hstatus[4];
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hth, theta, sizeof(hth), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hstatus, status, sizeof(hstatus), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = noalloc_fail(REG_ECUDA, "operator kernel failed");
            break;
        }
        if (hstatus[0] != 0 || hst.status != kDevOk) {
            rc = noalloc_fail(REG_EINVAL, "the operator kernel rejected its descriptor");
            break;
        }
        out->i = 0;
        out->k = 1;
        out->alpha = (float)hth[0];
        out->gx = (float)hth[1];
        out->gy = (float)hth[2];
        if (stats) memcpy(stats, &hst, sizeof(hst));
    } while (0);
    cudaSetDevice(prev);
    return rc;
}
