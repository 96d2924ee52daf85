// An allocation-free entry point: the joint LM fit of asp_fit_active_set
// without a context, its device scratch held in one file-scope array.
//
// Some callers cannot create device allocations of their own: code that runs
// inside another framework's memory pool (the pool owns the device memory
// budget and every byte outside it is an accounting error), real-time
// pipelines that forbid allocation after start-up (cudaMalloc can
// synchronise the device and take milliseconds), and host threads that may
// run while another thread captures a CUDA graph in global mode, where
// cudaMalloc is an illegal call.  asp_fit_static serves them: the caller
// passes the image and gets the fit back; the only device memory it touches
// besides the caller's image is g_fit_scratch below.
//
// g_fit_scratch is a __device__ array: every GPU that loads this library
// holds its ASP_STATIC_SCRATCH_BYTES until the process exits.  Every call on
// a device shares it and it keeps the last call's contents, so the entry
// point clears what must start at zero (the grid-barrier counter and the fit
// output) on each call; calls that overlap on the GPU race on it.
#include <cmath>
#include <cstring>
#include <mutex>

#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {
namespace {

// Layout of the scratch array (offsets in bytes, each 256-aligned).
constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t OFF_DESC = 0;
constexpr size_t OFF_OUT = align256(OFF_DESC + sizeof(FitDesc));
constexpr size_t OFF_BAR = align256(OFF_OUT + sizeof(FitOut));
constexpr size_t OFF_SUMS = align256(OFF_BAR + sizeof(unsigned));
constexpr size_t OFF_PART = align256(OFF_SUMS + (size_t)SUMS_DOUBLES * sizeof(double));
constexpr size_t STATIC_BYTES = align256(OFF_PART + (size_t)ASP_STATIC_GRID_MAX * NACC_MAX * sizeof(double));
constexpr int STATIC_NB = ((4 * ASP_STATIC_KMAX + 1) + 3) / 4;
static_assert(STATIC_NB * (STATIC_NB + 1) / 2 <= FIT_THREADS, "the one-tile-per-thread fit variant must cover K");
static_assert(STATIC_BYTES == ASP_STATIC_SCRATCH_BYTES, "ASP_STATIC_SCRATCH_BYTES in asp.h is out of date");

constexpr int MAX_DEVICES = 64;

struct DeviceSetup {
    unsigned char* scratch = nullptr;   // device address of g_fit_scratch on this device
    int g_max = 0;                      // co-resident CTAs the fit may use
    bool ready = false;
};

DeviceSetup g_setup[MAX_DEVICES];
std::mutex g_setup_mutex;

}  // namespace

// The scratch itself: FitDesc, FitOut, barrier counter, two sum buffers and
// ASP_STATIC_GRID_MAX CTA partial rows.
static __device__ __align__(256) unsigned char g_fit_scratch[ASP_STATIC_SCRATCH_BYTES];

namespace {

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in) and the fit kernel's
// co-residency limit.
asp_status setup_device(int dev, DeviceSetup** out) {
    if (dev < 0 || dev >= MAX_DEVICES) return ASP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.ready) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_fit_scratch) != cudaSuccess || ptr == nullptr) return ASP_ERR_CUDA;
        int bps = 0;
        if (fit_configure(1, &bps) != cudaSuccess || bps < 1) return ASP_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ASP_ERR_CUDA;
        s.scratch = static_cast<unsigned char*>(ptr);
        s.g_max = sms * bps < ASP_STATIC_GRID_MAX ? sms * bps : ASP_STATIC_GRID_MAX;
        s.ready = true;
    }
    *out = &s;
    return ASP_OK;
}

}  // namespace
}  // namespace aspd

using namespace aspd;

extern "C" asp_status asp_fit_static(const float* image_dev, int H, int W, const asp_gauss* init, int n, int n_old,
                                     double omega_min, const asp_params* lm, asp_gauss* out, asp_fit_info* info,
                                     void* stream) {
    if (!image_dev || !init || !out || !lm || H < 1 || W < 1 || n < 1 || n_old < 0 || n_old > n)
        return ASP_ERR_INVALID_ARG;
    if (n > ASP_STATIC_KMAX) return ASP_ERR_UNSUPPORTED;
    if (!(omega_min >= 0.0) || lm->lm_max_iter < 0 || !(lm->lm_lambda0 > 0) || !(lm->lm_rtol >= 0) ||
        !(lm->lm_xtol >= 0))
        return ASP_ERR_INVALID_ARG;
    // window: bounding box of the members' boxes, clipped to the image
    long long wx0 = 0, wx1 = 0, wy0 = 0, wy1 = 0;
    for (int k = 0; k < n; ++k) {
        const asp_gauss& g = init[k];
        // finite values and a positive width, as asp_fit_active_set requires
        // (an infinite centre or width would reach member_box's integer casts)
        if (!std::isfinite(g.amp) || !std::isfinite(g.x) || !std::isfinite(g.y) || !std::isfinite(g.width) ||
            !(g.width > 0))
            return ASP_ERR_INVALID_ARG;
        long long b[4];
        member_box(g.x, g.y, g.width, b);
        if (k == 0) { wx0 = b[0]; wx1 = b[1]; wy0 = b[2]; wy1 = b[3]; }
        wx0 = b[0] < wx0 ? b[0] : wx0; wx1 = b[1] > wx1 ? b[1] : wx1;
        wy0 = b[2] < wy0 ? b[2] : wy0; wy1 = b[3] > wy1 ? b[3] : wy1;
    }
    wx0 = wx0 < 0 ? 0 : wx0; wy0 = wy0 < 0 ? 0 : wy0;
    wx1 = wx1 > W - 1 ? W - 1 : wx1; wy1 = wy1 > H - 1 ? H - 1 : wy1;
    if (wx0 > wx1 || wy0 > wy1) return ASP_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ASP_ERR_CUDA;
    DeviceSetup* ds = nullptr;
    asp_status st = setup_device(dev, &ds);
    if (st != ASP_OK) return st;

    FitDesc d;
    memset(&d, 0, sizeof(d));
    d.K = n;
    d.n_old = n_old;
    d.wx0 = (int)wx0; d.wy0 = (int)wy0;
    d.ww = (int)(wx1 - wx0 + 1); d.wh = (int)(wy1 - wy0 + 1);
    d.omega_min = omega_min;
    d.omega_max = (double)(d.ww > d.wh ? d.ww : d.wh);
    d.bx0 = (double)wx0; d.bx1 = (double)wx1; d.by0 = (double)wy0; d.by1 = (double)wy1;
    for (int k = 0; k < n; ++k) {
        d.theta0[4 * k] = init[k].amp;
        d.theta0[4 * k + 1] = init[k].x;
        d.theta0[4 * k + 2] = init[k].y;
        d.theta0[4 * k + 3] = init[k].width;
    }
    int smem_ok = 0;
    d.grid = fit_grid((long long)d.ww * d.wh, n, 0, ds->g_max, &smem_ok);
    if (!smem_ok) return ASP_ERR_UNSUPPORTED;   // the window must fit the CTAs' shared memory
    d.smem_ok = 1;
    d.active = 1;

    LMConst lmc{};
    lmc.lambda0 = lm->lm_lambda0;
    lmc.lambda_up = 10.0;
    lmc.lambda_down = 10.0;
    lmc.lambda_min = 1e-12;
    lmc.lambda_max = 1e12;
    lmc.rtol = lm->lm_rtol;
    lmc.xtol = lm->lm_xtol;
    lmc.max_iter = lm->lm_max_iter;
    lmc.px_per_cta = 0;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    FitDesc* desc_dev = reinterpret_cast<FitDesc*>(ds->scratch + OFF_DESC);
    FitOut* out_dev = reinterpret_cast<FitOut*>(ds->scratch + OFF_OUT);
    unsigned* bar = reinterpret_cast<unsigned*>(ds->scratch + OFF_BAR);
    double* sums = reinterpret_cast<double*>(ds->scratch + OFF_SUMS);
    double* partials = reinterpret_cast<double*>(ds->scratch + OFF_PART);
    if (cudaMemcpyAsync(desc_dev, &d, sizeof(d), cudaMemcpyHostToDevice, s) != cudaSuccess) return ASP_ERR_CUDA;
    if (cudaMemsetAsync(out_dev, 0, sizeof(FitOut), s) != cudaSuccess) return ASP_ERR_CUDA;
    // launch_lm_fit clears the barrier counter before the kernel
    if (launch_lm_fit(1, ds->g_max, image_dev, W, desc_dev, lmc, out_dev, partials, sums, bar, nullptr, s) !=
        cudaSuccess)
        return ASP_ERR_CUDA;
    FitOut fo;
    if (cudaMemcpyAsync(&fo, out_dev, sizeof(FitOut), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ASP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ASP_ERR_CUDA;
    // FitOut.error carries the asp_status the kernel recorded (a bounded
    // grid-barrier wait that gave up sets ASP_ERR_TIMEOUT)
    if (fo.error) return fo.error > ASP_OK && fo.error <= ASP_ERR_CAPACITY ? (asp_status)fo.error : ASP_ERR_CUDA;
    for (int k = 0; k < n; ++k) {
        out[k].amp = fo.theta[4 * k];
        out[k].x = fo.theta[4 * k + 1];
        out[k].y = fo.theta[4 * k + 2];
        out[k].width = fo.theta[4 * k + 3];
    }
    if (info) {
        info->iters = fo.iters;
        info->passes = fo.passes;
        info->status = fo.status;
        info->k = n;
        info->x0 = (int)wx0; info->x1 = (int)wx1; info->y0 = (int)wy0; info->y1 = (int)wy1;
        info->chi2_init = fo.chi2_init;
        info->chi2_final = fo.chi2;
        info->lambda = fo.lambda;
        info->pixel_evals = fo.pixel_evals;
    }
    return ASP_OK;
}
