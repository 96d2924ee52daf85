// C-ABI of libasp: context life cycle, argument checking, device memory, and
// the launch sequence of the minor cycle (captured once into a CUDA graph and
// replayed; every step runs in the kernels of asp_fit.cu, asp_image.cu and
// asp_cycle.cu).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "asp_dev.cuh"
#include "asp_internal.h"

using namespace aspd;

// Kernel classes timed by asp_set_profiling.
enum KernelClass {
    KC_BEGIN, KC_SMOOTH_H, KC_SMOOTH_V, KC_SELECT, KC_FIT, KC_UPDATE, KC_WEIGHTS, KC_SUB_H, KC_SUB_V, KC_ARGMAX,
    KC_MLP, KC_LEARNED, KC_HARVEST, KC_SUB_GAUSS, KC_MAJOR, KC_SUB_FFT, KC_COUNT
};
static const char* const KC_NAMES[KC_COUNT] = {
    "k_cycle_begin", "k_smooth_h", "k_smooth_v_argmax", "k_select", "k_lm_fit", "k_update", "k_build_weights",
    "k_sub_h", "k_sub_v_argmax", "k_argmax_abs", "mlp_infer (tcgen05)", "k_learned_*", "k_harvest",
    "k_sub_gauss", "major cycle (FFT)", "subtraction (FFT)"};
static const int MAJOR_KERNELS = 6;     // own kernels of one major cycle (5 and the argmax; the 2 cuFFT calls not counted)
static const int SUB_FFT_KERNELS = 3;   // own kernels of one FFT residual update (the 2 cuFFT calls not counted)
static const int KERNELS_PER_ITER = 9;   // kernels one minor-cycle iteration enqueues

struct ProfMark {
    int cls;
    cudaEvent_t a, b;
};

struct asp_ctx {
    int dev = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    asp_params p{};
    Params dp{};
    int H = 0, W = 0;
    long long N = 0;
    float* R = nullptr;
    float* B = nullptr;
    double alpha_b = 0, omega_b = 0, xb = 0, yb = 0;
    double noise = 0;
    CycleState* st = nullptr;
    asp_component* comps = nullptr;
    asp_component* comp_stage = nullptr;
    asp_iter_record* hist = nullptr;
    float* wbuf = nullptr;
    float* T1 = nullptr;
    int terms_cap = 0;
    float* S1 = nullptr;
    float* taps_dev = nullptr;
    SmoothTaps taps{};
    double smooth_flops = 0.0;   // 2 passes x 2 flops x taps x pixels, all scales
    size_t taps_cap = 0;
    size_t s1_cap = 0;              // floats of S1
    double* partials = nullptr;
    double* sums = nullptr;
    unsigned* bar = nullptr;
    float* Tg = nullptr;
    ArgRes* part = nullptr;
    unsigned* ticket = nullptr;
    unsigned long long* hist256 = nullptr;
    double* dscalar = nullptr;
    int g_max = 1, tpt = 1, grid_img = 1;
    int grid_sh = 1, grid_sv = 1;   // smoothing passes: resident blocks (<= grid_img)
    unsigned* sched = nullptr;      // smoothing task counters: row pass [0, 1], column pass [2, 3]
    int g_alloc = 1;   // fit CTAs the partial-sum buffer holds (g_max may be capped below it)
    cudaGraphExec_t gexec = nullptr;
    int graph_unroll = 8;
    int graph_state = 0;   // 0 untried, 1 usable, -1 unavailable (direct launches)
    int profiling = 0;
    std::vector<ProfMark> marks;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[KC_COUNT] = {};
    long long prof_n[KC_COUNT] = {};
    long long launches = 0;
    int graph_kernels = 8 * KERNELS_PER_ITER;   // kernels one graph replay launches
    // learned initial values
    int learned = 0;
    float* mlpP = nullptr;                 // FP32 parameter vector
    void* W1b = nullptr;                   // BF16 copies of W1, W2
    void* W2b = nullptr;
    void* Xinf = nullptr;                  // 128 x 1024 BF16 network input (row 0 used)
    void* H1b = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Yinf = nullptr;
    unsigned* mlp_err = nullptr;
    // training-data harvest
    float* harvest_p = nullptr;
    float* harvest_t = nullptr;
    int harvest_cap = 0;
    // the plain start's fit beside the learned one (learned initial values)
    double* partials2 = nullptr;
    double* sums2 = nullptr;
    unsigned* bar2 = nullptr;
    float* Tg2 = nullptr;
    // minor/major split (asp_params.major_every > 0): the dirty image, the
    // PSF's transform, FFT buffers and plans, per-component normalisations
    float* D = nullptr;
    float* fft_in = nullptr;
    float* fft_out = nullptr;
    cufftComplex* fft_work = nullptr;
    cufftComplex* bhat = nullptr;
    float2* norms = nullptr;
    cufftHandle r2c = 0, c2r = 0;
    bool plans = false;
    bool sub_fft = false;   // per-iteration residual update by FFT (asp_params.sub_mode)
    Fit2004Buffers* f2004 = nullptr;   // Asp-Clean2004's objective, allocated by its first call
    unsigned char* ell_buf = nullptr;  // elliptical deconvolution in/out, allocated by its first call
    int broken = 0;
    std::string err;
    std::vector<void*> allocs;
};

namespace {

// The public totals of a control block.
void fill_stats(const CycleState& h, asp_cycle_stats* out) {
    memset(out, 0, sizeof(*out));
    out->iterations = h.t;
    out->components = h.n_comp;
    out->pixel_evals = h.pixel_evals;
    out->lm_iters = h.lm_iters;
    out->lm_passes = h.lm_passes;
    out->peak_abs = std::fabs((double)h.peak.val);
    out->stop_reason = h.stop_reason;
    out->fit_flops = h.fit_flops;
    out->sub_flops = h.sub_flops;
    out->sub_bytes = h.sub_bytes;
    out->smooth_flops = h.smooth_flops;
    out->fit_pass_ms = h.fit_ns_pass * 1e-6;
    out->fit_reduce_ms = h.fit_ns_reduce * 1e-6;
    out->fit_solve_ms = h.fit_ns_solve * 1e-6;
    out->fit_factor_ms = h.fit_ns_factor * 1e-6;
    out->fit_subst_ms = h.fit_ns_subst * 1e-6;
    out->fit_refinements = h.fit_refinements;
    out->fit_fallbacks = h.fit_fallbacks;
    out->learned_fits = h.learned_fits;
    out->learned_refits = h.learned_refits;
    out->learned_kept = h.learned_kept;
    out->fit_ex2 = h.fit_ex2;
    out->smooth_iters = h.smooth_iters;
}

asp_status fail(asp_ctx* c, asp_status s, const std::string& msg) {
    if (c) {
        c->err = msg;
        if (s == ASP_ERR_CUDA || s == ASP_ERR_TIMEOUT) c->broken = 1;
    }
    return s;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? ASP_ERR_OOM : ASP_ERR_CUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

#define CHECK_CTX()                                                                                \
    do {                                                                                           \
        if (!ctx) return ASP_ERR_INVALID_ARG;                                                      \
        if (ctx->broken) return ASP_ERR_STATE;                                                     \
        cudaSetDevice(ctx->dev);                                                                   \
    } while (0)

template <class T>
cudaError_t dalloc(asp_ctx* ctx, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) return e;
    ctx->allocs.push_back(q);
    *p = reinterpret_cast<T*>(q);
    return cudaSuccess;
}

LMConst lmconst_from(const asp_params& p, int max_iter_override = -1) {
    LMConst l{};
    l.lambda0 = p.lm_lambda0;
    l.lambda_up = 10.0;
    l.lambda_down = 10.0;
    l.lambda_min = 1e-12;
    l.lambda_max = 1e12;
    l.rtol = p.lm_rtol;
    l.xtol = p.lm_xtol;
    l.max_iter = max_iter_override >= 0 ? max_iter_override : p.lm_max_iter;
    l.px_per_cta = p.fit_px_per_cta;
    return l;
}

asp_status validate_params(const asp_params* p) {
    if (!p) return ASP_ERR_INVALID_ARG;
    if (!(p->gain > 0.f && p->gain <= 1.f)) return ASP_ERR_INVALID_ARG;
    if (p->k_max < 1) return ASP_ERR_INVALID_ARG;
    if (p->k_max > ASP_KMAX) return ASP_ERR_UNSUPPORTED;
    if (p->lm_max_iter < 0 || p->n_scales < 1 || p->n_scales > MAX_SCALES) return ASP_ERR_INVALID_ARG;
    if (!(p->lm_lambda0 > 0) || !(p->lm_rtol >= 0) || !(p->lm_xtol >= 0)) return ASP_ERR_INVALID_ARG;
    if (p->fit_px_per_cta < 0 || p->major_every < 0) return ASP_ERR_INVALID_ARG;
    if (p->sub_mode < ASP_SUB_AUTO || p->sub_mode > ASP_SUB_FFT) return ASP_ERR_INVALID_ARG;
    if (p->init_mode < 0 || p->init_mode > 2) return ASP_ERR_INVALID_ARG;
    if (p->retained_cap < 0 || p->retained_cap > RET_MAX) return ASP_ERR_UNSUPPORTED;
    if (p->max_components < 0) return ASP_ERR_INVALID_ARG;
    return ASP_OK;
}

asp_status read_state(asp_ctx* ctx, CycleState* h) {
    CK(cudaMemcpyAsync(h, ctx->st, sizeof(CycleState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ASP_OK;
}

// Field-wise host->device update of the control block.
template <class T>
asp_status put_field(asp_ctx* ctx, T* dev_field, const T& v) {
    CK(cudaMemcpyAsync(dev_field, &v, sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ASP_OK;
}

cudaEvent_t take_event(asp_ctx* ctx) {
    cudaEvent_t e = nullptr;
    if (!ctx->event_pool.empty()) {
        e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
    } else {
        cudaEventCreate(&e);
    }
    return e;
}

// Brackets one kernel launch with events when profiling (direct launches only).
struct Mark {
    asp_ctx* ctx;
    int cls;
    cudaEvent_t a = nullptr;
    Mark(asp_ctx* c, int k) : ctx(c), cls(k) {
        ctx->launches += 1;
        if (ctx->profiling) {
            a = take_event(ctx);
            cudaEventRecord(a, ctx->stream);
        }
    }
    ~Mark() {
        if (a) {
            cudaEvent_t b = take_event(ctx);
            cudaEventRecord(b, ctx->stream);
            ctx->marks.push_back({cls, a, b});
        }
    }
};

// Folds recorded event pairs into the per-class totals (stream synchronised).
void collect_marks(asp_ctx* ctx) {
    for (const ProfMark& m : ctx->marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            ctx->prof_ms[m.cls] += ms;
            ctx->prof_n[m.cls] += 1;
        }
        ctx->event_pool.push_back(m.a);
        ctx->event_pool.push_back(m.b);
    }
    ctx->marks.clear();
}

asp_status refresh_peak(asp_ctx* ctx) {
    Mark m(ctx, KC_ARGMAX);
    CK(launch_argmax(ctx->R, ctx->N, ctx->grid_img, ctx->part, ctx->ticket, &ctx->st->peak, &ctx->st->nonfinite,
                     nullptr, ctx->stream));
    return ASP_OK;
}

// One minor-cycle iteration as a fixed launch sequence (device-side gating).
asp_status enqueue_iteration(asp_ctx* ctx) {
    const int H = ctx->H, W = ctx->W;
    CycleState* st = ctx->st;
    cudaStream_t s = ctx->stream;
    { Mark m(ctx, KC_BEGIN); CK(launch_cycle_begin(st, ctx->dp, H, W, ctx->smooth_flops, s)); }
    { Mark m(ctx, KC_SMOOTH_H); CK(launch_smooth_h(ctx->R, H, W, ctx->taps, &st->skip_smooth, -1, ctx->S1, ctx->grid_sh, ctx->sched, s)); }
    { Mark m(ctx, KC_SMOOTH_V);
      CK(launch_smooth_v(ctx->S1, H, W, ctx->taps, st, &st->skip_smooth, -1, nullptr, ctx->grid_sv, ctx->part,
                         ctx->ticket, ctx->sched + 2, s)); }
    { Mark m(ctx, KC_SELECT); CK(launch_select(st, ctx->comps, ctx->dp, H, W, ctx->g_max, s)); }
    if (ctx->learned) {
        // the network's proposal, then the fits from the learned and the
        // plain start side by side in one launch, and the lower chi^2 kept
        { Mark m(ctx, KC_LEARNED); CK(launch_learned_prep(st, ctx->R, H, W, ctx->Xinf, s)); }
        {
            Mark m(ctx, KC_MLP);
            ctx->launches += mlp_infer_kernels() - 1;
            CK(launch_mlp_infer(ctx->Xinf, ctx->W1b, ctx->W2b, ctx->mlpP, ctx->Z1, ctx->H1b, ctx->Z2, ctx->H2, ctx->Yinf,
                                ctx->mlp_err, s));
        }
        { Mark m(ctx, KC_LEARNED); CK(launch_learned_apply(st, ctx->Yinf, ctx->g_max, s)); }
        { Mark m(ctx, KC_FIT);
          CK(launch_lm_fit_pair(ctx->tpt, ctx->g_max, ctx->R, W, ctx->dp.lm, &st->fit, &st->fout, ctx->partials,
                                ctx->sums, ctx->bar, ctx->Tg, &st->fit2, &st->fout2, ctx->partials2, ctx->sums2,
                                ctx->bar2, ctx->Tg2, s)); }
        { Mark m(ctx, KC_LEARNED); CK(launch_learned_pick(st, s)); }
    } else {
        Mark m(ctx, KC_FIT);
        CK(launch_lm_fit(ctx->tpt, ctx->g_max, ctx->R, W, &st->fit, ctx->dp.lm, &st->fout, ctx->partials, ctx->sums,
                         ctx->bar, ctx->Tg, s));
    }
    { Mark m(ctx, KC_UPDATE); CK(launch_update(st, ctx->comps, ctx->hist, ctx->dp, H, W, s)); }
    if (ctx->harvest_p) {
        Mark m(ctx, KC_HARVEST);
        CK(launch_harvest(st, ctx->R, H, W, ctx->harvest_p, ctx->harvest_t, ctx->harvest_cap, s));
    }
    if (ctx->p.major_every > 0) {
        // minor/major split: the terms' single-Gaussian-beam images, then the
        // next peak of the (approximate) residual
        { Mark m(ctx, KC_SUB_GAUSS); CK(launch_sub_gauss(ctx->R, H, W, st, ctx->grid_img, s)); }
        { Mark m(ctx, KC_ARGMAX);
          CK(launch_argmax(ctx->R, ctx->N, ctx->grid_img, ctx->part, ctx->ticket, &st->peak, &st->nonfinite,
                           &st->stopped, s)); }
        return ASP_OK;
    }
    { Mark m(ctx, KC_WEIGHTS); CK(launch_build_weights(st, &st->stopped, ctx->wbuf, s)); }
    if (ctx->sub_fft) {
        Mark m(ctx, KC_SUB_FFT);
        ctx->launches += SUB_FFT_KERNELS - 1;
        CK(launch_sub_fft(st, &st->stopped, ctx->wbuf, H, W, ctx->fft_in, ctx->fft_work, ctx->bhat, ctx->fft_out, ctx->R,
                          ctx->r2c, ctx->c2r, ctx->grid_img, ctx->part, ctx->ticket, s));
        return ASP_OK;
    }
    { Mark m(ctx, KC_SUB_H); CK(launch_sub_h(ctx->B, H, W, st, &st->stopped, ctx->wbuf, ctx->T1, ctx->grid_img, ctx->taps, s)); }
    { Mark m(ctx, KC_SUB_V);
      CK(launch_sub_v(ctx->R, ctx->B, H, W, st, &st->stopped, ctx->wbuf, ctx->T1, ctx->grid_img, ctx->part, ctx->ticket,
                      s)); }
    return ASP_OK;
}

// The major cycle: R = D - B * M exactly (FFT convolution), applied if a
// minor iteration ran since the last one, then the next peak.
asp_status enqueue_major(asp_ctx* ctx) {
    CycleState* st = ctx->st;
    {
        Mark m(ctx, KC_MAJOR);
        ctx->launches += MAJOR_KERNELS - 2;
        CK(launch_major(ctx->comps, ctx->norms, st, ctx->H, ctx->W, ctx->fft_in, ctx->fft_work, ctx->bhat,
                        ctx->fft_out, ctx->R, ctx->D, ctx->r2c, ctx->c2r, ctx->grid_img, ctx->stream));
    }
    { Mark m(ctx, KC_ARGMAX);
      CK(launch_argmax(ctx->R, ctx->N, ctx->grid_img, ctx->part, ctx->ticket, &st->peak, &st->nonfinite,
                       &st->major_skip, ctx->stream)); }
    return ASP_OK;
}

asp_status build_graph(asp_ctx* ctx) {
    if (ctx->graph_state != 0) return ASP_OK;
    if (getenv("ASP_NO_GRAPH")) { ctx->graph_state = -1; return ASP_OK; }
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = ctx->stream;
    ctx->stream = cs;
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    asp_status s = ASP_OK;
    const long long launches_before = ctx->launches;
    if (ok) {
        for (int i = 0; i < ctx->graph_unroll && s == ASP_OK; ++i) s = enqueue_iteration(ctx);
        if (s == ASP_OK && ctx->p.major_every > 0) s = enqueue_major(ctx);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        ok = (s == ASP_OK) && e == cudaSuccess && g != nullptr;
    }
    ctx->graph_kernels = (int)(ctx->launches - launches_before);
    ctx->stream = saved;
    ctx->launches = launches_before;
    ctx->broken = 0;
    ctx->err.clear();
    if (ok && cudaGraphInstantiate(&ctx->gexec, g, 0) == cudaSuccess) {
        ctx->graph_state = 1;
    } else {
        ctx->graph_state = -1;
        cudaGetLastError();
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return ASP_OK;
}

void host_member_box(double x, double y, double w, long long* b) { member_box(x, y, w, b); }

}  // namespace

// Beam (alpha_b, omega_b): LM fit of one Gaussian to the PSF main lobe
// (Sect. 3).  Leaves the result in ctx and in the control block.
asp_status fit_beam(asp_ctx* ctx) {
    const int H = ctx->H, W = ctx->W;
    CK(launch_beam_init(&ctx->st->fit, ctx->B, H, W, ctx->g_max, ctx->stream));
    CK(cudaMemsetAsync(&ctx->st->fout, 0, sizeof(FitOut), ctx->stream));
    {
        Mark m(ctx, KC_FIT);
        CK(launch_lm_fit(ctx->tpt, ctx->g_max, ctx->B, 2 * W, &ctx->st->fit, ctx->dp.lm, &ctx->st->fout,
                         ctx->partials, ctx->sums, ctx->bar, ctx->Tg, ctx->stream));
    }
    FitOut fo;
    CK(cudaMemcpyAsync(&fo, &ctx->st->fout, sizeof(FitOut), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (fo.error) return fail(ctx, ASP_ERR_TIMEOUT, "beam fit: device wait timed out");
    if (!(fo.theta[3] > 0) || !std::isfinite(fo.theta[0]) || fo.theta[0] == 0.0 || !std::isfinite(fo.theta[3]))
        return fail(ctx, ASP_ERR_NAN, "beam fit failed (no main lobe to fit)");
    ctx->alpha_b = fo.theta[0];
    ctx->xb = fo.theta[1];
    ctx->yb = fo.theta[2];
    ctx->omega_b = fo.theta[3];
    double ab_wb[2] = {ctx->alpha_b, ctx->omega_b};
    CK(cudaMemcpyAsync(&ctx->st->alpha_b, ab_wb, sizeof(ab_wb), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ASP_OK;
}

// Smoothing scales s_j = omega_b 2^j, kept while s_j <= min(H, W) / 8, with
// unit-L2 1-D taps exp(-u^2 / 2 s^2), |u| <= ceil(4 s).
asp_status setup_taps(asp_ctx* ctx) {
    const int H = ctx->H, W = ctx->W;
    const long long N = ctx->N;
    std::vector<float> taps;
    SmoothTaps t{};
    double sflops = 0.0;
    int m_max = 0;
    for (int j = 0; j < ctx->p.n_scales; ++j) {
        double s_j = ctx->omega_b * std::ldexp(1.0, j);
        if (j > 0 && s_j > std::min(H, W) / 8.0) continue;
        int m = (int)std::ceil(4.0 * s_j);
        std::vector<double> e(2 * m + 1);
        double ss = 0;
        for (int u = -m; u <= m; ++u) {
            e[u + m] = std::exp(-(double)u * u / (2.0 * s_j * s_j));
            ss += e[u + m] * e[u + m];
        }
        double inv = 1.0 / std::sqrt(ss);
        t.off[t.n] = (int)taps.size();
        t.m[t.n] = m;
        t.t8[t.n] = (2 * m + 1 + 7) & ~7;
        t.scale[t.n] = s_j;
        for (double v : e) taps.push_back((float)(v * inv));
        t.t8max = std::max(t.t8max, t.t8[t.n]);
        m_max = std::max(m_max, m);
        t.n++;
        sflops += 2.0 * 2.0 * (2 * m + 1) * (double)N;
    }
    // register-blocked pass geometry: 8 outputs per thread
    const int per_row = (W + 7) / 8;
    t.tpr = std::min(RED_THREADS, (per_row + 31) / 32 * 32);
    t.rpb = RED_THREADS / t.tpr;
    t.nseg = (W + 8 * t.tpr - 1) / (8 * t.tpr);
    {
        const int last = 8 * t.tpr + t.t8max + 7;          // largest staged index
        t.blen = last + (last >> 3) + 1;
    }
    // the paired row pass doubles the taps and the segment buffers
    t.pair_h = 2 * ((size_t)t.t8max + (size_t)t.rpb * t.blen) * sizeof(float) <= 48 * 1024;
    t.mpad = ((m_max + 7) & ~7) + 8;
    t.s1rows = (long long)H + 2LL * t.mpad + 8;
    if (taps.size() > ctx->taps_cap) {
        float* p = nullptr;
        CK(dalloc(ctx, &p, taps.size()));
        ctx->taps_dev = p;
        ctx->taps_cap = taps.size();
    }
    const size_t s1_need = (size_t)t.n * (size_t)t.s1rows * (size_t)W;
    if (s1_need > ctx->s1_cap) {
        float* p = nullptr;
        CK(dalloc(ctx, &p, s1_need));
        ctx->S1 = p;
        ctx->s1_cap = s1_need;
    }
    // the halo rows stay zero: only interior rows are ever written
    CK(cudaMemset(ctx->S1, 0, s1_need * sizeof(float)));
    if (smooth_h_smem(t) > 48 * 1024) return ASP_ERR_UNSUPPORTED;
    ctx->grid_sh = smooth_grid_h(t, ctx->num_sms, ctx->grid_img);
    ctx->grid_sv = smooth_grid_v(t, ctx->num_sms, ctx->grid_img);
    CK(cudaMemcpy(ctx->taps_dev, taps.data(), taps.size() * sizeof(float), cudaMemcpyHostToDevice));
    t.k = ctx->taps_dev;
    ctx->taps = t;
    ctx->smooth_flops = sflops;
    return ASP_OK;
}

// =====================================================================
extern "C" {

const char* asp_status_string(asp_status s) {
    switch (s) {
        case ASP_OK: return "ok";
        case ASP_ERR_INVALID_ARG: return "invalid argument";
        case ASP_ERR_CUDA: return "CUDA error";
        case ASP_ERR_OOM: return "out of device memory";
        case ASP_ERR_NAN: return "non-finite value";
        case ASP_ERR_TIMEOUT: return "device wait timed out";
        case ASP_ERR_NOT_CONVERGED: return "not converged";
        case ASP_ERR_STATE: return "context unusable after an earlier error";
        case ASP_ERR_UNSUPPORTED: return "size beyond a compiled-in limit";
        case ASP_ERR_CAPACITY: return "component list full";
    }
    return "unknown status";
}

void asp_default_params(asp_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->gain = 0.35f;
    p->k_max = 5;
    p->lm_max_iter = 50;
    p->lm_lambda0 = 1e-3;
    p->lm_rtol = 1e-7;
    p->lm_xtol = 1e-7;
    p->noise_sigma = 0.f;
    p->stop_ksigma = 3.f;
    p->n_scales = 6;
    p->area_frac = 0.05f;
    p->init_mode = ASP_INIT_AUTO;
    p->tau = 1e-3;
    p->retained_cap = 0;
    p->max_components = 0;
}

const char* asp_last_error(const asp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static asp_status init_common(const asp_params* pin, int H, int W, const float* dirty, const float* psf, int on_host,
                              void* stream, asp_ctx** out) {
    if (!out) return ASP_ERR_INVALID_ARG;
    *out = nullptr;
    asp_status vs = validate_params(pin);
    if (vs != ASP_OK) return vs;
    if (H < 1 || W < 1 || !dirty || !psf) return ASP_ERR_INVALID_ARG;
    if ((long long)H * W > (1LL << 31) / 4 || H > (1 << 20) || W > (1 << 20)) return ASP_ERR_UNSUPPORTED;
    asp_ctx* ctx = new asp_ctx();
    ctx->p = *pin;
    if (ctx->p.retained_cap == 0) ctx->p.retained_cap = std::min(RET_MAX, 8 * ctx->p.k_max);
    if (ctx->p.max_components == 0) ctx->p.max_components = 65536;
    ctx->H = H;
    ctx->W = W;
    ctx->N = (long long)H * W;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    asp_status s = ASP_OK;
    auto bail = [&](asp_status st) { asp_destroy(ctx); return st; };
    if (cudaGetDevice(&ctx->dev) != cudaSuccess) return bail(ASP_ERR_CUDA);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, ctx->dev) != cudaSuccess) return bail(ASP_ERR_CUDA);
    ctx->num_sms = prop.multiProcessorCount;
    ctx->grid_img = ctx->num_sms * 4;
    ctx->tpt = fit_tpt_for(ctx->p.k_max);
    int bps = 0;
    if (fit_configure(ctx->tpt, &bps) != cudaSuccess || bps < 1) return bail(ASP_ERR_CUDA);
    ctx->g_max = std::min(ctx->num_sms * bps, FIT_GRID_MAX);
    ctx->g_alloc = ctx->g_max;

    // device parameters
    ctx->dp.gain = ctx->p.gain;
    ctx->dp.area_frac = ctx->p.area_frac;
    ctx->dp.k_max = ctx->p.k_max;
    ctx->dp.init_mode = ctx->p.init_mode;
    ctx->dp.retained_cap = ctx->p.retained_cap;
    ctx->dp.n_scales = ctx->p.n_scales;
    ctx->dp.tau = ctx->p.tau;
    ctx->dp.major_every = ctx->p.major_every;
    ctx->dp.lm = lmconst_from(ctx->p);

    const long long N = ctx->N;
    ctx->sub_fft = ctx->p.major_every == 0 &&
                   (ctx->p.sub_mode == ASP_SUB_FFT || (ctx->p.sub_mode == ASP_SUB_AUTO && N >= ASP_SUB_FFT_MIN_PIXELS));
    ctx->terms_cap = std::max(2 * ctx->p.k_max - 1, 1);
    const int cap = ctx->p.max_components;
#define AL(ptr, n) if (dalloc(ctx, &(ptr), (size_t)(n)) != cudaSuccess) return bail(ASP_ERR_OOM)
    AL(ctx->R, N);
    AL(ctx->B, 4 * N);
    AL(ctx->st, 1);
    AL(ctx->comps, cap);
    AL(ctx->comp_stage, MAX_TERMS);
    AL(ctx->hist, cap);
    AL(ctx->wbuf, (size_t)MAX_TERMS * wslot_stride(W, H));
    // the direct update's row-pass buffer (the FFT update needs none; slack
    // rows: see k_sub_v_argmax)
    const size_t t1_rows = (ctx->sub_fft ? 0 : (size_t)ctx->terms_cap * (2 * H - 1)) + T1_SLACK_ROWS;
    AL(ctx->T1, t1_rows * W);
    if (cudaMemset(ctx->T1, 0, t1_rows * W * sizeof(float)) != cudaSuccess)
        return bail(ASP_ERR_CUDA);
    AL(ctx->partials, (size_t)ctx->g_max * NACC_MAX);
    AL(ctx->sums, SUMS_DOUBLES);
    AL(ctx->bar, 1);
    AL(ctx->Tg, 4 * N);   // window targets beyond shared memory (image or PSF windows)
    AL(ctx->part, std::max(ctx->grid_img, ctx->g_max));
    AL(ctx->ticket, 1);
    AL(ctx->sched, 4);
    AL(ctx->hist256, 260);
    AL(ctx->dscalar, 4);
#undef AL
    cudaMemcpyKind kind = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpyAsync(ctx->R, dirty, N * sizeof(float), kind, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(ctx->B, psf, 4 * N * sizeof(float), kind, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->st, 0, sizeof(CycleState), ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->ticket, 0, sizeof(unsigned), ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->sched, 0, 4 * sizeof(unsigned), ctx->stream) != cudaSuccess)
        return bail(ASP_ERR_CUDA);

    if (ctx->p.major_every > 0 || ctx->sub_fft) {
        // the FFT buffers and plans of the 2H x 2W grid and the PSF's
        // transform; the minor/major split adds the dirty image and the
        // components' normalisations
        const size_t nc = (size_t)(2 * H) * (W + 1);
        if (dalloc(ctx, &ctx->fft_in, (size_t)4 * N) != cudaSuccess ||
            dalloc(ctx, &ctx->fft_out, (size_t)4 * N) != cudaSuccess || dalloc(ctx, &ctx->fft_work, nc) != cudaSuccess ||
            dalloc(ctx, &ctx->bhat, nc) != cudaSuccess)
            return bail(ASP_ERR_OOM);
        if (ctx->p.major_every > 0 &&
            (dalloc(ctx, &ctx->D, (size_t)N) != cudaSuccess || dalloc(ctx, &ctx->norms, (size_t)cap) != cudaSuccess))
            return bail(ASP_ERR_OOM);
        if (cufftPlan2d(&ctx->r2c, 2 * H, 2 * W, CUFFT_R2C) != CUFFT_SUCCESS) return bail(ASP_ERR_CUDA);
        if (cufftPlan2d(&ctx->c2r, 2 * H, 2 * W, CUFFT_C2R) != CUFFT_SUCCESS) {
            cufftDestroy(ctx->r2c);
            return bail(ASP_ERR_CUDA);
        }
        ctx->plans = true;
        if ((ctx->D && cudaMemcpyAsync(ctx->D, ctx->R, N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream) !=
                           cudaSuccess) ||
            compute_psf_transform(ctx->B, H, W, ctx->fft_in, ctx->bhat, ctx->r2c, ctx->stream) != cudaSuccess)
            return bail(ASP_ERR_CUDA);
        if (ctx->p.major_every > 0) ctx->graph_unroll = ctx->p.major_every;
    }
    s = fit_beam(ctx);
    if (s != ASP_OK) return bail(s);
    s = setup_taps(ctx);
    if (s != ASP_OK) return bail(s);

    // ---- noise level: given, or 1.4826 x MAD of the dirty image
    if (ctx->p.noise_sigma > 0.f) {
        ctx->noise = ctx->p.noise_sigma;
    } else {
        double med = 0, mad = 0;
        if (launch_radix_median(ctx->R, N, 0, 0.0, ctx->hist256, ctx->dscalar, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(&med, ctx->dscalar, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return bail(ASP_ERR_CUDA);
        if (launch_radix_median(ctx->R, N, 1, med, ctx->hist256, ctx->dscalar, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(&mad, ctx->dscalar, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return bail(ASP_ERR_CUDA);
        ctx->noise = 1.4826 * mad;
    }

    // ---- control block
    CycleState h;
    memset(&h, 0, sizeof(h));
    h.cap_comp = cap;
    h.thr = (double)ctx->p.stop_ksigma * ctx->noise;
    h.alpha_b = ctx->alpha_b;
    h.omega_b = ctx->omega_b;
    h.t_stop = 0;
    if (cudaMemcpyAsync(ctx->st, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        return bail(ASP_ERR_CUDA);
    s = refresh_peak(ctx);
    if (s != ASP_OK) return bail(s);
    CycleState chk;
    s = read_state(ctx, &chk);
    if (s != ASP_OK) return bail(s);
    if (chk.nonfinite) { ctx->err = "non-finite value in the dirty image"; return bail(ASP_ERR_NAN); }
    *out = ctx;
    return ASP_OK;
}

asp_status asp_init(const asp_params* p, int H, int W, const float* dirty_dev, const float* psf_dev, void* stream,
                    asp_ctx** out) {
    return init_common(p, H, W, dirty_dev, psf_dev, 0, stream, out);
}

asp_status asp_init_host(const asp_params* p, int H, int W, const float* dirty_host, const float* psf_host,
                         void* stream, asp_ctx** out) {
    return init_common(p, H, W, dirty_host, psf_host, 1, stream, out);
}

asp_status asp_destroy(asp_ctx* ctx) {
    if (!ctx) return ASP_ERR_INVALID_ARG;
    cudaSetDevice(ctx->dev);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->plans) { cufftDestroy(ctx->r2c); cufftDestroy(ctx->c2r); }
    if (ctx->f2004) {
        Fit2004Buffers* fb = ctx->f2004;
        if (fb->r2c1) cufftDestroy(fb->r2c1);
        if (fb->c2r1) cufftDestroy(fb->c2r1);
        if (fb->r2cN) cufftDestroy(fb->r2cN);
        if (fb->c2rN) cufftDestroy(fb->c2rN);
        delete fb;
    }
    collect_marks(ctx);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    for (void* q : ctx->allocs) cudaFree(q);
    delete ctx;
    return ASP_OK;
}

asp_status asp_get_beam(asp_ctx* ctx, double* alpha_b, double* omega_b, double* x_b, double* y_b) {
    CHECK_CTX();
    if (alpha_b) *alpha_b = ctx->alpha_b;
    if (omega_b) *omega_b = ctx->omega_b;
    if (x_b) *x_b = ctx->xb;
    if (y_b) *y_b = ctx->yb;
    return ASP_OK;
}

asp_status asp_find_peak(asp_ctx* ctx, int mode, asp_peak* out) {
    CHECK_CTX();
    if (!out || (mode != ASP_PEAK_SIMPLE && mode != ASP_PEAK_SMOOTH)) return ASP_ERR_INVALID_ARG;
    CycleState h;
    if (mode == ASP_PEAK_SIMPLE) {
        asp_status s = refresh_peak(ctx);
        if (s != ASP_OK) return s;
        s = read_state(ctx, &h);
        if (s != ASP_OK) return s;
        out->index = h.peak.idx;
        out->x = (int32_t)(h.peak.idx % ctx->W);
        out->y = (int32_t)(h.peak.idx / ctx->W);
        out->value = h.peak.val;
        out->scale = 0.f;
        out->mode = ASP_PEAK_SIMPLE;
        out->scale_index = -1;
        out->a0 = h.peak.val;
        out->x0 = out->x;
        out->y0 = out->y;
        out->w0 = ctx->omega_b;
        return ASP_OK;
    }
    {
        Mark m(ctx, KC_SMOOTH_H);
        CK(launch_smooth_h(ctx->R, ctx->H, ctx->W, ctx->taps, nullptr, -1, ctx->S1, ctx->grid_sh, ctx->sched, ctx->stream));
    }
    {
        Mark m(ctx, KC_SMOOTH_V);
        CK(launch_smooth_v(ctx->S1, ctx->H, ctx->W, ctx->taps, ctx->st, nullptr, -1, nullptr, ctx->grid_sv, ctx->part,
                           ctx->ticket, ctx->sched + 2, ctx->stream));
    }
    asp_status s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    out->index = h.speak.idx;
    out->x = (int32_t)(h.speak.idx % ctx->W);
    out->y = (int32_t)(h.speak.idx / ctx->W);
    out->value = h.speak.val;
    out->scale = (float)ctx->taps.scale[h.speak.j];
    out->mode = ASP_PEAK_SMOOTH;
    out->scale_index = h.speak.j;
    out->a0 = h.init[0];
    out->x0 = h.init[1];
    out->y0 = h.init[2];
    out->w0 = h.init[3];
    return ASP_OK;
}

static asp_status run_fit(asp_ctx* ctx, const asp_gauss* init, int n, int n_old, int x0, int x1, int y0, int y1,
                          int max_iter, FitOut* fo, double lambda0 = 0.0, const asp_gauss* start = nullptr) {
    FitDesc d;
    memset(&d, 0, sizeof(d));
    d.K = n;
    d.n_old = n_old;
    d.wx0 = x0;
    d.wy0 = y0;
    d.ww = x1 - x0 + 1;
    d.wh = y1 - y0 + 1;
    d.omega_min = 0.25 * ctx->omega_b;
    d.omega_max = (double)std::max(d.ww, d.wh);
    d.bx0 = x0; d.bx1 = x1; d.by0 = y0; d.by1 = y1;
    for (int k = 0; k < n; ++k) {
        d.theta0[4 * k] = init[k].amp;
        d.theta0[4 * k + 1] = init[k].x;
        d.theta0[4 * k + 2] = init[k].y;
        d.theta0[4 * k + 3] = init[k].width;
        if (start) {
            d.start[4 * k] = start[k].amp;
            d.start[4 * k + 1] = start[k].x;
            d.start[4 * k + 2] = start[k].y;
            d.start[4 * k + 3] = start[k].width;
        }
    }
    d.has_start = start != nullptr;
    LMConst lmc = ctx->dp.lm;
    if (max_iter >= 0) lmc.max_iter = max_iter;
    if (lambda0 > 0.0) lmc.lambda0 = lambda0;
    int smem_ok = 1;
    d.grid = fit_grid((long long)d.ww * d.wh, n, lmc.px_per_cta, ctx->g_max, &smem_ok);
    d.smem_ok = smem_ok;
    d.active = 1;
    CK(cudaMemcpyAsync(&ctx->st->fit, &d, sizeof(d), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(&ctx->st->fout, 0, sizeof(FitOut), ctx->stream));
    {
        Mark m(ctx, KC_FIT);
        CK(launch_lm_fit(ctx->tpt, ctx->g_max, ctx->R, ctx->W, &ctx->st->fit, lmc, &ctx->st->fout, ctx->partials,
                         ctx->sums, ctx->bar, ctx->Tg, ctx->stream));
    }
    CK(cudaMemcpyAsync(fo, &ctx->st->fout, sizeof(FitOut), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (fo->error) return fail(ctx, ASP_ERR_TIMEOUT, "fit: grid barrier timed out");
    return ASP_OK;
}

static bool gauss_ok(const asp_gauss& g) {
    return std::isfinite(g.amp) && std::isfinite(g.x) && std::isfinite(g.y) && std::isfinite(g.width) && g.width > 0;
}

static asp_status fit_common(asp_ctx* ctx, const asp_gauss* init, int n, int n_old, const asp_gauss* start,
                             double lambda0, int max_iter, asp_gauss* out, asp_fit_info* info, asp_gauss* trial,
                             double* chi2_trial) {
    if (!init || !out || n < 1 || n > ctx->p.k_max || n_old < 0 || n_old > n) return ASP_ERR_INVALID_ARG;
    if (start)
        for (int k = 0; k < n; ++k)
            if (!gauss_ok(start[k])) return ASP_ERR_INVALID_ARG;
    long long wx0 = 0, wx1 = 0, wy0 = 0, wy1 = 0;
    for (int k = 0; k < n; ++k) {
        if (!gauss_ok(init[k])) return ASP_ERR_INVALID_ARG;
        long long b[4];
        host_member_box(init[k].x, init[k].y, init[k].width, b);
        if (k == 0) { wx0 = b[0]; wx1 = b[1]; wy0 = b[2]; wy1 = b[3]; }
        wx0 = std::min(wx0, b[0]); wx1 = std::max(wx1, b[1]);
        wy0 = std::min(wy0, b[2]); wy1 = std::max(wy1, b[3]);
    }
    wx0 = std::max(wx0, 0LL); wy0 = std::max(wy0, 0LL);
    wx1 = std::min(wx1, (long long)ctx->W - 1); wy1 = std::min(wy1, (long long)ctx->H - 1);
    if (wx0 > wx1 || wy0 > wy1) return ASP_ERR_INVALID_ARG;
    FitOut fo;
    asp_status s = run_fit(ctx, init, n, n_old, (int)wx0, (int)wx1, (int)wy0, (int)wy1, max_iter, &fo, lambda0, start);
    if (s != ASP_OK) return s;
    for (int k = 0; k < n; ++k) {
        out[k].amp = fo.theta[4 * k];
        out[k].x = fo.theta[4 * k + 1];
        out[k].y = fo.theta[4 * k + 2];
        out[k].width = fo.theta[4 * k + 3];
        if (trial) {
            trial[k].amp = fo.trial[4 * k];
            trial[k].x = fo.trial[4 * k + 1];
            trial[k].y = fo.trial[4 * k + 2];
            trial[k].width = fo.trial[4 * k + 3];
        }
    }
    if (chi2_trial) *chi2_trial = fo.chi2_trial;
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

asp_status asp_fit_active_set(asp_ctx* ctx, const asp_gauss* init, int n, int n_old, asp_gauss* out,
                              asp_fit_info* info) {
    CHECK_CTX();
    return fit_common(ctx, init, n, n_old, nullptr, 0.0, -1, out, info, nullptr, nullptr);
}

asp_status asp_fit_lm(asp_ctx* ctx, const asp_gauss* init, int n, int n_old, const asp_gauss* start, double lambda0,
                      int max_iter, asp_gauss* out, asp_fit_info* info, asp_gauss* trial_out, double* chi2_trial) {
    CHECK_CTX();
    if (!(lambda0 > 0.0) || !std::isfinite(lambda0) || max_iter < 0) return ASP_ERR_INVALID_ARG;
    return fit_common(ctx, init, n, n_old, start, lambda0, max_iter, out, info, trial_out, chi2_trial);
}

// ---------------------------------------------------------------- elliptical variant

static bool gauss_ell_ok(const asp_gauss_ell& g) {
    if (!(std::isfinite(g.amp) && std::isfinite(g.x) && std::isfinite(g.y) && std::isfinite(g.pxx) &&
          std::isfinite(g.pxy) && std::isfinite(g.pyy)))
        return false;
    return g.pxx > 0 && g.pyy > 0 && g.pxx * g.pyy - g.pxy * g.pxy > 0;
}

// Major principal width 1 / sqrt(mu_min) of a positive-definite precision matrix.
static double ell_sigma_max(const asp_gauss_ell& g) {
    const double h = 0.5 * (g.pxx + g.pyy), r = std::hypot(0.5 * (g.pxx - g.pyy), g.pxy);
    return 1.0 / std::sqrt(h - r);
}

// One elliptical fit launch: the fit variant for 6n parameters (that of
// ceil(6n / 4) circular members), configured on first use, at most the
// context's grid.
static asp_status ell_variant(asp_ctx* ctx, int K, int* tpt, int* g_max) {
    *tpt = fit_tpt_for((6 * K + 3) / 4);
    int bps = 0;
    if (fit_configure_model(1, *tpt, &bps) != cudaSuccess || bps < 1) return fail(ctx, ASP_ERR_CUDA, "fit variant");
    *g_max = std::min(std::min(ctx->num_sms * bps, FIT_GRID_MAX), ctx->g_max);
    return ASP_OK;
}

static asp_status run_fit_ell(asp_ctx* ctx, FitDesc& d, int K, const float* src, int src_w, FitOut* fo) {
    int tpt = 1, g_max = 1;
    asp_status vs = ell_variant(ctx, K, &tpt, &g_max);
    if (vs != ASP_OK) return vs;
    LMConst lmc = ctx->dp.lm;
    if (d.active) {
        int smem_ok = 1;
        d.grid = fit_grid((long long)d.ww * d.wh, d.K, lmc.px_per_cta, g_max, &smem_ok);
        d.smem_ok = smem_ok;
        CK(cudaMemcpyAsync(&ctx->st->fit, &d, sizeof(d), cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaMemsetAsync(&ctx->st->fout, 0, sizeof(FitOut), ctx->stream));
    {
        Mark m(ctx, KC_FIT);
        CK(launch_lm_fit_model(1, tpt, g_max, src, src_w, &ctx->st->fit, lmc, &ctx->st->fout, ctx->partials,
                               ctx->sums, ctx->bar, ctx->Tg, ctx->stream));
    }
    CK(cudaMemcpyAsync(fo, &ctx->st->fout, sizeof(FitOut), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (fo->error) return fail(ctx, ASP_ERR_TIMEOUT, "fit: grid barrier timed out");
    return ASP_OK;
}

asp_status asp_fit_elliptical(asp_ctx* ctx, const asp_gauss_ell* init, int n, int n_old, asp_gauss_ell* out,
                              asp_fit_info* info) {
    CHECK_CTX();
    if (!init || !out || n < 1 || n_old < 0 || n_old > n) return ASP_ERR_INVALID_ARG;
    if (n > ASP_ELL_KMAX) return ASP_ERR_UNSUPPORTED;
    long long wx0 = 0, wx1 = 0, wy0 = 0, wy1 = 0;
    for (int k = 0; k < n; ++k) {
        if (!gauss_ell_ok(init[k])) return ASP_ERR_INVALID_ARG;
        long long b[4];
        host_member_box(init[k].x, init[k].y, ell_sigma_max(init[k]), b);
        if (k == 0) { wx0 = b[0]; wx1 = b[1]; wy0 = b[2]; wy1 = b[3]; }
        wx0 = std::min(wx0, b[0]); wx1 = std::max(wx1, b[1]);
        wy0 = std::min(wy0, b[2]); wy1 = std::max(wy1, b[3]);
    }
    wx0 = std::max(wx0, 0LL); wy0 = std::max(wy0, 0LL);
    wx1 = std::min(wx1, (long long)ctx->W - 1); wy1 = std::min(wy1, (long long)ctx->H - 1);
    if (wx0 > wx1 || wy0 > wy1) return ASP_ERR_INVALID_ARG;
    FitDesc d;
    memset(&d, 0, sizeof(d));
    d.K = n;
    d.n_old = n_old;
    d.model = 1;
    d.wx0 = (int)wx0; d.wy0 = (int)wy0;
    d.ww = (int)(wx1 - wx0 + 1); d.wh = (int)(wy1 - wy0 + 1);
    d.omega_min = 0.25 * ctx->omega_b;
    d.omega_max = (double)std::max(d.ww, d.wh);
    d.bx0 = (double)wx0; d.bx1 = (double)wx1; d.by0 = (double)wy0; d.by1 = (double)wy1;
    for (int k = 0; k < n; ++k) {
        double* t = d.theta0 + 6 * k;
        t[0] = init[k].amp; t[1] = init[k].x; t[2] = init[k].y;
        t[3] = init[k].pxx; t[4] = init[k].pxy; t[5] = init[k].pyy;
    }
    d.active = 1;
    FitOut fo;
    asp_status s = run_fit_ell(ctx, d, n, ctx->R, ctx->W, &fo);
    if (s != ASP_OK) return s;
    for (int k = 0; k < n; ++k) {
        const double* t = fo.theta + 6 * k;
        out[k] = asp_gauss_ell{t[0], t[1], t[2], t[3], t[4], t[5]};
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

asp_status asp_fit_beam_elliptical(asp_ctx* ctx, asp_gauss_ell* out) {
    CHECK_CTX();
    if (!out) return ASP_ERR_INVALID_ARG;
    // the circular beam's region and bounds (k_beam_init, its grid sized
    // for the launch below), then the elliptical start from the circular beam
    int tpt = 1, g_max = 1;
    asp_status s = ell_variant(ctx, 1, &tpt, &g_max);
    if (s != ASP_OK) return s;
    CK(launch_beam_init(&ctx->st->fit, ctx->B, ctx->H, ctx->W, g_max, ctx->stream));
    CK(launch_beam_ell_desc(&ctx->st->fit, ctx->alpha_b, ctx->xb, ctx->yb, ctx->omega_b, ctx->stream));
    FitDesc d;
    memset(&d, 0, sizeof(d));   // inactive: run_fit_ell keeps the device's descriptor
    FitOut fo;
    s = run_fit_ell(ctx, d, 1, ctx->B, 2 * ctx->W, &fo);
    if (s != ASP_OK) return s;
    const asp_gauss_ell g{fo.theta[0], fo.theta[1], fo.theta[2], fo.theta[3], fo.theta[4], fo.theta[5]};
    if (!gauss_ell_ok(g) || g.amp == 0.0)
        return fail(ctx, ASP_ERR_NAN, "elliptical beam fit failed (no positive-definite main lobe)");
    *out = g;
    return ASP_OK;
}

asp_status asp_deconvolve_elliptical(asp_ctx* ctx, const asp_gauss_ell* in, int n, const asp_gauss_ell* beam,
                                     asp_component_ell* out) {
    CHECK_CTX();
    if (!in || !beam || !out || n < 0) return ASP_ERR_INVALID_ARG;
    if (n > ASP_ELL_KMAX) return ASP_ERR_UNSUPPORTED;
    if (!gauss_ell_ok(*beam) || beam->amp == 0.0) return ASP_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        if (!gauss_ell_ok(in[k])) return ASP_ERR_INVALID_ARG;
    if (n == 0) return ASP_OK;
    const size_t in_bytes = sizeof(asp_gauss_ell) * (ASP_ELL_KMAX + 1);
    if (!ctx->ell_buf) CK(dalloc(ctx, &ctx->ell_buf, in_bytes + sizeof(asp_component_ell) * ASP_ELL_KMAX));
    asp_gauss_ell* din = reinterpret_cast<asp_gauss_ell*>(ctx->ell_buf);
    asp_component_ell* dout = reinterpret_cast<asp_component_ell*>(ctx->ell_buf + in_bytes);
    CK(cudaMemcpyAsync(din, beam, sizeof(asp_gauss_ell), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(din + 1, in, sizeof(asp_gauss_ell) * n, cudaMemcpyHostToDevice, ctx->stream));
    { Mark m(ctx, KC_UPDATE); CK(launch_deconvolve_ell(din, n, dout, ctx->stream)); }
    CK(cudaMemcpyAsync(out, dout, sizeof(asp_component_ell) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ASP_OK;
}

// ---------------------------------------------------------------- Asp-Clean2004's objective (Eq. 3)

static asp_status f2004_setup(asp_ctx* ctx, int K) {
    const int H = ctx->H, W = ctx->W;
    const int nb = 4 * K + 1;
    if (!ctx->f2004) {
        Fit2004Buffers* fb = new Fit2004Buffers();
        ctx->f2004 = fb;
        const size_t nimg = (size_t)4 * ctx->N, nc = (size_t)(2 * H) * (W + 1);
        fb->grid = ctx->grid_img;
        fb->ne_blocks = ctx->grid_img;
        CK(dalloc(ctx, &fb->imgs, nimg * FIT2004_NA));
        CK(dalloc(ctx, &fb->conv, nimg * FIT2004_NA));
        CK(dalloc(ctx, &fb->work, nc * FIT2004_NA));
        CK(dalloc(ctx, &fb->bhat, nc));
        CK(dalloc(ctx, &fb->T, (size_t)ctx->N));
        CK(dalloc(ctx, &fb->partials, (size_t)fb->ne_blocks * FIT2004_NACC));
        CK(dalloc(ctx, &fb->sums, (size_t)FIT2004_NACC));
        CK(dalloc(ctx, &fb->theta, (size_t)4 * FIT2004_KMAX));
        CK(cudaMemsetAsync(fb->imgs, 0, sizeof(float) * nimg * FIT2004_NA, ctx->stream));
        if (cufftPlan2d(&fb->r2c1, 2 * H, 2 * W, CUFFT_R2C) != CUFFT_SUCCESS ||
            cufftPlan2d(&fb->c2r1, 2 * H, 2 * W, CUFFT_C2R) != CUFFT_SUCCESS)
            return fail(ctx, ASP_ERR_CUDA, "cuFFT plan");
        CK(psf_transform_2004(*fb, ctx->B, H, W, ctx->stream));
    }
    Fit2004Buffers* fb = ctx->f2004;
    if (fb->nb != nb) {
        if (fb->r2cN) { cufftDestroy(fb->r2cN); fb->r2cN = 0; }
        if (fb->c2rN) { cufftDestroy(fb->c2rN); fb->c2rN = 0; }
        int n[2] = {2 * H, 2 * W};
        const int dist_r = 4 * H * W, dist_c = 2 * H * (W + 1);
        if (cufftPlanMany(&fb->r2cN, 2, n, nullptr, 1, dist_r, nullptr, 1, dist_c, CUFFT_R2C, nb) != CUFFT_SUCCESS ||
            cufftPlanMany(&fb->c2rN, 2, n, nullptr, 1, dist_c, nullptr, 1, dist_r, CUFFT_C2R, nb) != CUFFT_SUCCESS)
            return fail(ctx, ASP_ERR_CUDA, "cuFFT batched plan");
        fb->nb = nb;
    }
    return ASP_OK;
}

// One evaluation of Eq. 3 at theta (host, 4K values): with full, the packed
// upper triangle of [J | r]^T [J | r] into A (K4 x K4, full), g and chi2;
// else chi2 only.
static asp_status f2004_eval(asp_ctx* ctx, const double* theta, int K, bool full, double* A, double* g, double* chi2) {
    Fit2004Buffers* fb = ctx->f2004;
    const int P = 4 * K, NA = full ? P + 1 : 1, nacc = NA * (NA + 1) / 2;
    CK(cudaMemcpyAsync(fb->theta, theta, sizeof(double) * P, cudaMemcpyHostToDevice, ctx->stream));
    CK(eval_2004(*fb, fb->theta, K, NA, ctx->H, ctx->W, ctx->R, false, ctx->stream));
    std::vector<double> sums((size_t)nacc);
    CK(cudaMemcpyAsync(sums.data(), fb->sums, sizeof(double) * nacc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    auto at = [&](int i, int j) {                       // packed upper triangle, row-major
        if (i > j) std::swap(i, j);
        return sums[(size_t)i * NA - (size_t)i * (i - 1) / 2 + (j - i)];
    };
    *chi2 = at(NA - 1, NA - 1);
    if (full) {
        for (int i = 0; i < P; ++i) {
            g[i] = at(i, P);
            for (int j = 0; j < P; ++j) A[(size_t)i * P + j] = at(i, j);
        }
    }
    return ASP_OK;
}

// (A + lam diag(d)) delta = g by FP64 Cholesky, d_i = A_ii (1 where A_ii <=
// 0); false if not positive definite.
static bool f2004_solve(const std::vector<double>& A, const std::vector<double>& g, double lam, int P,
                        std::vector<double>& delta) {
    std::vector<double> L((size_t)P * P, 0.0);
    for (int i = 0; i < P; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = A[(size_t)i * P + j];
            if (i == j) {
                const double d = A[(size_t)i * P + i] > 0 ? A[(size_t)i * P + i] : 1.0;
                v += lam * d;
            }
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * P + k] * L[(size_t)j * P + k];
            if (i == j) {
                if (!(v > 0) || !std::isfinite(v)) return false;
                L[(size_t)i * P + i] = std::sqrt(v);
            } else {
                L[(size_t)i * P + j] = v / L[(size_t)j * P + j];
            }
        }
    std::vector<double> z((size_t)P);
    for (int i = 0; i < P; ++i) {
        double v = g[i];
        for (int k = 0; k < i; ++k) v -= L[(size_t)i * P + k] * z[k];
        z[i] = v / L[(size_t)i * P + i];
    }
    delta.assign((size_t)P, 0.0);
    for (int i = P - 1; i >= 0; --i) {
        double v = z[i];
        for (int k = i + 1; k < P; ++k) v -= L[(size_t)k * P + i] * delta[k];
        delta[i] = v / L[(size_t)i * P + i];
        if (!std::isfinite(delta[i])) return false;
    }
    return true;
}

asp_status asp_fit_2004(asp_ctx* ctx, const asp_gauss* init, int n, int n_old, double omega_min, asp_gauss* out,
                        asp_fit_info* info) {
    CHECK_CTX();
    if (!init || !out || n < 1 || n_old < 0 || n_old > n || !(omega_min >= 0.0)) return ASP_ERR_INVALID_ARG;
    if (n > FIT2004_KMAX) return ASP_ERR_UNSUPPORTED;
    for (int k = 0; k < n; ++k)
        if (!gauss_ok(init[k])) return ASP_ERR_INVALID_ARG;
    asp_status s = f2004_setup(ctx, n);
    if (s != ASP_OK) return s;
    Fit2004Buffers* fb = ctx->f2004;
    const int H = ctx->H, W = ctx->W, P = 4 * n;
    // target: the residual with the last n_old members added back through B
    if (n_old > 0) {
        std::vector<double> th_old((size_t)4 * n_old);
        for (int k = 0; k < n_old; ++k) {
            const asp_gauss& q = init[n - n_old + k];
            th_old[4 * k] = q.amp; th_old[4 * k + 1] = q.x; th_old[4 * k + 2] = q.y; th_old[4 * k + 3] = q.width;
        }
        CK(cudaMemcpyAsync(fb->theta, th_old.data(), sizeof(double) * 4 * n_old, cudaMemcpyHostToDevice, ctx->stream));
        CK(eval_2004(*fb, fb->theta, n_old, 1, H, W, ctx->R, true, ctx->stream));
    } else {
        CK(cudaMemcpyAsync(fb->T, ctx->R, sizeof(float) * ctx->N, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    const LMConst lm = ctx->dp.lm;
    std::vector<double> theta((size_t)P), A((size_t)P * P), g((size_t)P), delta, trial((size_t)P);
    for (int k = 0; k < n; ++k) {
        theta[4 * k] = init[k].amp; theta[4 * k + 1] = init[k].x; theta[4 * k + 2] = init[k].y;
        theta[4 * k + 3] = init[k].width;
    }
    double chi2 = 0.0;
    s = f2004_eval(ctx, theta.data(), n, true, A.data(), g.data(), &chi2);
    if (s != ASP_OK) return s;
    const double chi2_init = chi2, omega_max = (double)std::max(H, W);
    int passes = 1, iters = 0, status = ASP_LM_CAP;
    double lam = lm.lambda0;
    while (true) {
        if (iters >= lm.max_iter) { status = ASP_LM_CAP; break; }
        const bool ok = f2004_solve(A, g, lam, P, delta);
        ++iters;
        if (!ok) {
            lam *= lm.lambda_up;
            if (lam > lm.lambda_max) { status = ASP_LM_STALLED; break; }
            continue;
        }
        // predicted decrease d.g + lam d.D.d of the damped step (Marquardt)
        double pred = 0.0;
        for (int i = 0; i < P; ++i) {
            const double d = A[(size_t)i * P + i] > 0 ? A[(size_t)i * P + i] : 1.0;
            pred += delta[i] * g[i] + lam * d * delta[i] * delta[i];
        }
        if (pred <= lm.rtol * chi2) { status = ASP_LM_CONVERGED; break; }
        bool valid = true;
        for (int i = 0; i < P; ++i) {
            trial[i] = theta[i] + delta[i];
            valid = valid && std::isfinite(trial[i]);
        }
        for (int k = 0; k < n && valid; ++k) {
            const double x = trial[4 * k + 1], y = trial[4 * k + 2], w = trial[4 * k + 3];
            valid = w > omega_min && !(w > omega_max) && x >= 0 && x <= W - 1 && y >= 0 && y <= H - 1;
        }
        if (!valid) {
            lam *= lm.lambda_up;
            if (lam > lm.lambda_max) { status = ASP_LM_STALLED; break; }
            continue;
        }
        double chi2_t = 0.0;
        s = f2004_eval(ctx, trial.data(), n, false, nullptr, nullptr, &chi2_t);
        if (s != ASP_OK) return s;
        ++passes;
        if (chi2_t < chi2) {
            const double rel = chi2 > 0 ? (chi2 - chi2_t) / chi2 : 0.0;
            bool small = true;
            for (int i = 0; i < P; ++i) {
                double sc = (i & 3) == 0 ? std::fabs(theta[i]) : theta[(i & ~3) + 3];
                if (sc == 0.0) sc = 1.0;
                small = small && std::fabs(delta[i]) < lm.xtol * sc;
            }
            theta = trial;
            s = f2004_eval(ctx, theta.data(), n, true, A.data(), g.data(), &chi2);
            if (s != ASP_OK) return s;
            lam = std::max(lam / lm.lambda_down, lm.lambda_min);
            if (rel < lm.rtol || small) { status = ASP_LM_CONVERGED; break; }
        } else {
            lam *= lm.lambda_up;
            if (lam > lm.lambda_max) { status = ASP_LM_STALLED; break; }
        }
    }
    for (int k = 0; k < n; ++k) {
        out[k].amp = theta[4 * k]; out[k].x = theta[4 * k + 1]; out[k].y = theta[4 * k + 2];
        out[k].width = theta[4 * k + 3];
    }
    if (info) {
        info->iters = iters;
        info->passes = passes;
        info->status = status;
        info->k = n;
        info->x0 = 0; info->x1 = W - 1; info->y0 = 0; info->y1 = H - 1;
        info->chi2_init = chi2_init;
        info->chi2_final = chi2;
        info->lambda = lam;
        info->pixel_evals = (int64_t)passes * ctx->N;
    }
    return ASP_OK;
}

asp_status asp_eval_normal_equations(asp_ctx* ctx, const asp_gauss* theta, int n, int n_old, int x0, int x1, int y0,
                                     int y1, double* A_host, double* g_host, double* chi2_host) {
    CHECK_CTX();
    if (!theta || n < 1 || n > ASP_KMAX || n > ctx->p.k_max || n_old < 0 || n_old > n) return ASP_ERR_INVALID_ARG;
    x0 = std::max(x0, 0); y0 = std::max(y0, 0);
    x1 = std::min(x1, ctx->W - 1); y1 = std::min(y1, ctx->H - 1);
    if (x0 > x1 || y0 > y1) return ASP_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        if (!gauss_ok(theta[k])) return ASP_ERR_INVALID_ARG;
    FitOut fo;
    asp_status s = run_fit(ctx, theta, n, n_old, x0, x1, y0, y1, 0, &fo);
    if (s != ASP_OK) return s;
    // after the single pass the sums live in buffer 1
    const int P = 4 * n, NAp = ((P + 1) + 3) & ~3, nb = NAp / 4;
    std::vector<double> acc((size_t)fit_tiles(n) * 16);
    CK(cudaMemcpy(acc.data(), ctx->sums + NACC_MAX, acc.size() * sizeof(double), cudaMemcpyDeviceToHost));
    auto at = [&](int i, int j) {
        if (i > j) std::swap(i, j);
        int bi = i >> 2, bj = j >> 2;
        int t = bi * nb - bi * (bi - 1) / 2 + (bj - bi);
        return acc[(size_t)t * 16 + (i & 3) * 4 + (j & 3)];
    };
    for (int i = 0; i < P; ++i) {
        if (A_host)
            for (int j = 0; j < P; ++j) A_host[(size_t)i * P + j] = at(i, j);
        if (g_host) g_host[i] = at(i, P);
    }
    if (chi2_host) *chi2_host = at(P, P);
    return ASP_OK;
}

asp_status asp_subtract(asp_ctx* ctx, const asp_component* comps, int n, float gain) {
    CHECK_CTX();
    if (!comps || n < 0 || n > ctx->terms_cap || !std::isfinite(gain)) return ASP_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(comps[i].flux) || !std::isfinite(comps[i].x) || !std::isfinite(comps[i].y) ||
            !std::isfinite(comps[i].width) || comps[i].width < 0)
            return ASP_ERR_INVALID_ARG;
    if (n == 0) return ASP_OK;
    CK(cudaMemcpyAsync(ctx->comp_stage, comps, n * sizeof(asp_component), cudaMemcpyHostToDevice, ctx->stream));
    { Mark m(ctx, KC_UPDATE); CK(launch_terms_from_components(ctx->st, ctx->comp_stage, n, gain, ctx->H, ctx->W, ctx->stream)); }
    { Mark m(ctx, KC_WEIGHTS); CK(launch_build_weights(ctx->st, nullptr, ctx->wbuf, ctx->stream)); }
    if (ctx->sub_fft) {
        Mark m(ctx, KC_SUB_FFT);
        ctx->launches += SUB_FFT_KERNELS - 1;
        CK(launch_sub_fft(ctx->st, nullptr, ctx->wbuf, ctx->H, ctx->W, ctx->fft_in, ctx->fft_work, ctx->bhat,
                          ctx->fft_out, ctx->R, ctx->r2c, ctx->c2r, ctx->grid_img, ctx->part, ctx->ticket, ctx->stream));
    } else {
    { Mark m(ctx, KC_SUB_H); CK(launch_sub_h(ctx->B, ctx->H, ctx->W, ctx->st, nullptr, ctx->wbuf, ctx->T1, ctx->grid_img, ctx->taps, ctx->stream)); }
    {
        Mark m(ctx, KC_SUB_V);
        CK(launch_sub_v(ctx->R, ctx->B, ctx->H, ctx->W, ctx->st, nullptr, ctx->wbuf, ctx->T1, ctx->grid_img, ctx->part,
                        ctx->ticket, ctx->stream));
    }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return ASP_OK;
}

asp_status asp_subtract_beam(asp_ctx* ctx, const asp_component* comps, int n, float gain) {
    CHECK_CTX();
    if (!comps || n < 0 || n > MAX_TERMS || !std::isfinite(gain)) return ASP_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(comps[i].flux) || !std::isfinite(comps[i].x) || !std::isfinite(comps[i].y) ||
            !std::isfinite(comps[i].width) || comps[i].width < 0)
            return ASP_ERR_INVALID_ARG;
    if (n == 0) return ASP_OK;
    CK(cudaMemcpyAsync(ctx->comp_stage, comps, n * sizeof(asp_component), cudaMemcpyHostToDevice, ctx->stream));
    { Mark m(ctx, KC_UPDATE); CK(launch_terms_from_components(ctx->st, ctx->comp_stage, n, gain, ctx->H, ctx->W, ctx->stream)); }
    { Mark m(ctx, KC_SUB_GAUSS); CK(launch_sub_gauss(ctx->R, ctx->H, ctx->W, ctx->st, ctx->grid_img, ctx->stream)); }
    CK(cudaStreamSynchronize(ctx->stream));
    return refresh_peak(ctx);
}

asp_status asp_minor_cycle(asp_ctx* ctx, int n_iter, asp_cycle_stats* out) {
    CHECK_CTX();
    if (n_iter < 0) return ASP_ERR_INVALID_ARG;
    CycleState h;
    asp_status s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    const int t0 = h.t;
    struct { int t_stop, stopped, stop_reason; } ctl = {t0 + n_iter, 0, 0};
    CK(cudaMemcpyAsync(&ctx->st->t_stop, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, ctx->stream));
    if (!ctx->profiling) {
        s = build_graph(ctx);
        if (s != ASP_OK) return s;
    }
    if (n_iter > 0) {
        if (ctx->graph_state == 1 && !ctx->profiling) {
            const int reps = (n_iter + ctx->graph_unroll - 1) / ctx->graph_unroll;
            for (int r = 0; r < reps; ++r) CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
            ctx->launches += (long long)reps * ctx->graph_kernels;
        } else {
            const int me = ctx->p.major_every;
            for (int i = 0; i < n_iter; ++i) {
                s = enqueue_iteration(ctx);
                if (s != ASP_OK) return s;
                if (me > 0 && ((i + 1) % me == 0 || i + 1 == n_iter)) {
                    s = enqueue_major(ctx);
                    if (s != ASP_OK) return s;
                }
            }
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    collect_marks(ctx);
    s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    if (h.error == ASP_ERR_TIMEOUT) return fail(ctx, ASP_ERR_TIMEOUT, "fit: grid barrier timed out");
    if (ctx->learned && ctx->mlp_err) {
        unsigned me = 0;
        CK(cudaMemcpy(&me, ctx->mlp_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
        if (me) return fail(ctx, ASP_ERR_TIMEOUT, "network inference: tensor-core wait timed out");
    }
    if (h.error == ASP_ERR_NAN || h.nonfinite) return fail(ctx, ASP_ERR_NAN, "non-finite value in the residual");
    if (out) fill_stats(h, out);
    if (h.stop_reason == ASP_STOP_CAPACITY) return fail(ctx, ASP_ERR_CAPACITY, "component list full");
    return ASP_OK;
}

asp_status asp_get_stats(asp_ctx* ctx, asp_cycle_stats* out) {
    CHECK_CTX();
    if (!out) return ASP_ERR_INVALID_ARG;
    CycleState h;
    asp_status s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    fill_stats(h, out);
    return ASP_OK;
}

asp_status asp_num_scales(asp_ctx* ctx, int* n, double* scales_host) {
    CHECK_CTX();
    if (!n) return ASP_ERR_INVALID_ARG;
    *n = ctx->taps.n;
    if (scales_host)
        for (int j = 0; j < ctx->taps.n; ++j) scales_host[j] = ctx->taps.scale[j];
    return ASP_OK;
}

asp_status asp_smooth(asp_ctx* ctx, int scale_index, float* out_dev) {
    CHECK_CTX();
    if (scale_index < 0 || scale_index >= ctx->taps.n || !out_dev) return ASP_ERR_INVALID_ARG;
    {
        Mark m(ctx, KC_SMOOTH_H);
        CK(launch_smooth_h(ctx->R, ctx->H, ctx->W, ctx->taps, nullptr, scale_index, ctx->S1, ctx->grid_sh, ctx->sched,
                           ctx->stream));
    }
    {
        Mark m(ctx, KC_SMOOTH_V);
        CK(launch_smooth_v(ctx->S1, ctx->H, ctx->W, ctx->taps, ctx->st, nullptr, scale_index, out_dev, ctx->grid_sv,
                           ctx->part, ctx->ticket, ctx->sched + 2, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return ASP_OK;
}

asp_status asp_residual_ptr(asp_ctx* ctx, float** residual_dev) {
    CHECK_CTX();
    if (!residual_dev) return ASP_ERR_INVALID_ARG;
    *residual_dev = ctx->R;
    return ASP_OK;
}

asp_status asp_copy_residual(asp_ctx* ctx, float* dst, int dst_on_host) {
    CHECK_CTX();
    if (!dst) return ASP_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(dst, ctx->R, ctx->N * sizeof(float),
                       dst_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ASP_OK;
}

asp_status asp_set_residual(asp_ctx* ctx, const float* src, int src_on_host) {
    CHECK_CTX();
    if (!src) return ASP_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(ctx->R, src, ctx->N * sizeof(float),
                       src_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream));
    return asp_refresh_peak(ctx);
}

asp_status asp_refresh_peak(asp_ctx* ctx) {
    CHECK_CTX();
    asp_status s = refresh_peak(ctx);
    if (s != ASP_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return ASP_OK;
}

asp_status asp_get_components(asp_ctx* ctx, asp_component* out_host, int cap, int* count) {
    CHECK_CTX();
    if (!count || cap < 0 || (cap > 0 && !out_host)) return ASP_ERR_INVALID_ARG;
    CycleState h;
    asp_status s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    *count = h.n_comp;
    const int n = std::min(cap, h.n_comp);
    if (n > 0) CK(cudaMemcpy(out_host, ctx->comps, n * sizeof(asp_component), cudaMemcpyDeviceToHost));
    return ASP_OK;
}

asp_status asp_get_history(asp_ctx* ctx, asp_iter_record* out_host, int cap, int* count) {
    CHECK_CTX();
    if (!count || cap < 0 || (cap > 0 && !out_host)) return ASP_ERR_INVALID_ARG;
    CycleState h;
    asp_status s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    const int total = std::min(h.t, ctx->p.max_components);
    *count = total;
    const int n = std::min(cap, total);
    if (n > 0) CK(cudaMemcpy(out_host, ctx->hist, n * sizeof(asp_iter_record), cudaMemcpyDeviceToHost));
    return ASP_OK;
}

asp_status asp_get_state(asp_ctx* ctx, asp_component* comps, int comp_cap, int* n_comp, int* retained, int ret_cap,
                         int* n_ret, int64_t* t, double* last_wi, double* last_w0) {
    CHECK_CTX();
    CycleState h;
    asp_status s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    if (n_comp) *n_comp = h.n_comp;
    if (comps && comp_cap > 0) {
        const int n = std::min(comp_cap, h.n_comp);
        if (n > 0) CK(cudaMemcpy(comps, ctx->comps, n * sizeof(asp_component), cudaMemcpyDeviceToHost));
    }
    if (n_ret) *n_ret = h.n_ret;
    if (retained && ret_cap > 0)
        for (int i = 0; i < std::min(ret_cap, h.n_ret); ++i) retained[i] = h.ret[i];
    if (t) *t = h.t;
    if (last_wi) *last_wi = h.last_wi;
    if (last_w0) *last_w0 = h.last_w0;
    return ASP_OK;
}

asp_status asp_set_state(asp_ctx* ctx, const asp_component* comps, int n_comp, const int* retained, int n_ret,
                         int64_t t, double last_wi, double last_w0) {
    CHECK_CTX();
    if (n_comp < 0 || n_comp > ctx->p.max_components || (n_comp > 0 && !comps)) return ASP_ERR_INVALID_ARG;
    if (n_ret < 0 || n_ret > ctx->p.retained_cap || (n_ret > 0 && !retained) || t < 0 || t > (1LL << 30))
        return ASP_ERR_INVALID_ARG;
    for (int i = 0; i < n_ret; ++i)
        if (retained[i] < 0 || retained[i] >= n_comp) return ASP_ERR_INVALID_ARG;
    CycleState h;
    asp_status s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    if (n_comp > 0) CK(cudaMemcpy(ctx->comps, comps, n_comp * sizeof(asp_component), cudaMemcpyHostToDevice));
    h.n_comp = n_comp;
    h.n_ret = n_ret;
    for (int i = 0; i < n_ret; ++i) h.ret[i] = retained[i];
    h.t = (int)t;
    h.t_stop = (int)t;
    h.last_wi = last_wi;
    h.last_w0 = last_w0;
    h.stopped = 0;
    h.stop_reason = 0;
    h.pixel_evals = h.lm_iters = h.lm_passes = 0;
    h.fit_flops = h.sub_flops = h.sub_bytes = h.smooth_flops = h.fit_ex2 = 0.0;
    h.smooth_iters = 0;
    h.fit_ns_pass = h.fit_ns_reduce = h.fit_ns_solve = h.fit_ns_factor = h.fit_ns_subst = 0;
    h.fit_refinements = h.fit_fallbacks = 0;
    CK(cudaMemcpyAsync(ctx->st, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    return asp_refresh_peak(ctx);
}

asp_status asp_get_last_fit(asp_ctx* ctx, asp_gauss* out, int cap, int* n, asp_fit_info* info) {
    CHECK_CTX();
    if (!n || cap < 0 || (cap > 0 && !out)) return ASP_ERR_INVALID_ARG;
    CycleState h;
    asp_status s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    const int K = h.fit.K;
    *n = K;
    for (int k = 0; k < std::min(cap, K); ++k) {
        out[k].amp = h.fout.theta[4 * k];
        out[k].x = h.fout.theta[4 * k + 1];
        out[k].y = h.fout.theta[4 * k + 2];
        out[k].width = h.fout.theta[4 * k + 3];
    }
    if (info) {
        info->iters = h.fout.iters;
        info->passes = h.fout.passes;
        info->status = h.fout.status;
        info->k = K;
        info->x0 = h.fit.wx0; info->x1 = h.fit.wx0 + h.fit.ww - 1;
        info->y0 = h.fit.wy0; info->y1 = h.fit.wy0 + h.fit.wh - 1;
        info->chi2_init = h.fout.chi2_init;
        info->chi2_final = h.fout.chi2;
        info->lambda = h.fout.lambda;
        info->pixel_evals = h.fout.pixel_evals;
    }
    return ASP_OK;
}

asp_status asp_reset(asp_ctx* ctx, const float* dirty, int dirty_on_host, const float* psf, int psf_on_host) {
    CHECK_CTX();
    if (!dirty) return ASP_ERR_INVALID_ARG;
    if (psf) {
        CK(cudaMemcpyAsync(ctx->B, psf, 4 * ctx->N * sizeof(float),
                           psf_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream));
        const double wb_old = ctx->omega_b;
        asp_status s = fit_beam(ctx);
        if (s != ASP_OK) return s;
        if (ctx->omega_b != wb_old) {
            s = setup_taps(ctx);
            if (s != ASP_OK) return s;
            ctx->graph_state = ctx->gexec ? 0 : ctx->graph_state;   // taps are baked into the graph
            if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
        }
    }
    CK(cudaMemcpyAsync(ctx->R, dirty, ctx->N * sizeof(float),
                       dirty_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream));
    if (ctx->p.major_every > 0)
        CK(cudaMemcpyAsync(ctx->D, ctx->R, ctx->N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    if (psf && ctx->plans) CK(compute_psf_transform(ctx->B, ctx->H, ctx->W, ctx->fft_in, ctx->bhat, ctx->r2c, ctx->stream));
    if (psf && ctx->f2004) CK(psf_transform_2004(*ctx->f2004, ctx->B, ctx->H, ctx->W, ctx->stream));
    { Mark m(ctx, KC_BEGIN); CK(launch_reset_state(ctx->st, ctx->stream)); }
    return refresh_peak(ctx);
}

asp_status asp_set_profiling(asp_ctx* ctx, int on) {
    CHECK_CTX();
    CK(cudaStreamSynchronize(ctx->stream));
    collect_marks(ctx);
    ctx->profiling = on ? 1 : 0;
    for (int k = 0; k < KC_COUNT; ++k) { ctx->prof_ms[k] = 0.0; ctx->prof_n[k] = 0; }
    return ASP_OK;
}

asp_status asp_get_kernel_times(asp_ctx* ctx, asp_kernel_time* out, int cap, int* n) {
    CHECK_CTX();
    if (!n || cap < 0 || (cap > 0 && !out)) return ASP_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    collect_marks(ctx);
    *n = KC_COUNT;
    for (int k = 0; k < std::min(cap, (int)KC_COUNT); ++k) {
        memset(out[k].name, 0, sizeof(out[k].name));
        strncpy(out[k].name, KC_NAMES[k], sizeof(out[k].name) - 1);
        out[k].launches = ctx->prof_n[k];
        out[k].total_ms = ctx->prof_ms[k];
    }
    return ASP_OK;
}

asp_status asp_launch_count(asp_ctx* ctx, int64_t* n) {
    CHECK_CTX();
    if (!n) return ASP_ERR_INVALID_ARG;
    *n = ctx->launches;
    return ASP_OK;
}

static const uint32_t STATE_MAGIC = 0x41535031u;   // "ASP1"

asp_status asp_set_mlp(asp_ctx* ctx, const float* params_host, int enable) {
    CHECK_CTX();
    if (enable && !params_host) return ASP_ERR_INVALID_ARG;
    if (enable) {
        if (!ctx->mlpP) {
            const long long np = mlp_num_params();
#define AL(ptr, n) if (dalloc(ctx, &(ptr), (size_t)(n)) != cudaSuccess) return fail(ctx, ASP_ERR_OOM, "asp_set_mlp")
            float* P = nullptr;
            uint16_t *w1 = nullptr, *w2 = nullptr, *x = nullptr, *h1 = nullptr;
            AL(P, np);
            AL(w1, 256 * 1024);
            AL(w2, 256 * 256);
            AL(x, 128 * 1024);
            AL(h1, 128 * 256);
            AL(ctx->Z1, 128 * 256);
            AL(ctx->Z2, 128 * 256);
            AL(ctx->H2, 128 * 256);
            AL(ctx->Yinf, 128 * 4);
            AL(ctx->mlp_err, 1);
            // the plain start's fit runs beside the learned one
            AL(ctx->partials2, (size_t)ctx->g_max * NACC_MAX);
            AL(ctx->sums2, SUMS_DOUBLES);
            AL(ctx->bar2, 1);
            AL(ctx->Tg2, 4 * ctx->N);
#undef AL
            ctx->mlpP = P;
            ctx->W1b = w1;
            ctx->W2b = w2;
            ctx->Xinf = x;
            ctx->H1b = h1;
            CK(cudaMemsetAsync(ctx->Xinf, 0, 128 * 1024 * sizeof(uint16_t), ctx->stream));
            CK(cudaMemsetAsync(ctx->mlp_err, 0, sizeof(unsigned), ctx->stream));
            // the plain start's fit descriptor starts inactive
            CK(cudaMemsetAsync(&ctx->st->fit2, 0, sizeof(FitDesc), ctx->stream));
        }
        CK(cudaMemcpyAsync(ctx->mlpP, params_host, mlp_num_params() * sizeof(float), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(mlp_prepare(ctx->mlpP, ctx->W1b, ctx->W2b, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (ctx->learned != (enable ? 1 : 0)) {
        ctx->learned = enable ? 1 : 0;
        if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
        ctx->graph_state = 0;
    }
    return ASP_OK;
}

asp_status asp_set_harvest(asp_ctx* ctx, float* patches_dev, float* targets_dev, int capacity) {
    CHECK_CTX();
    if (patches_dev && (!targets_dev || capacity < 1)) return ASP_ERR_INVALID_ARG;
    const bool was = ctx->harvest_p != nullptr, now = patches_dev != nullptr;
    ctx->harvest_p = patches_dev;
    ctx->harvest_t = now ? targets_dev : nullptr;
    ctx->harvest_cap = now ? capacity : 0;
    if (was || now) {   // the pointers are baked into the captured graph
        if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
        ctx->graph_state = 0;
    }
    return ASP_OK;
}

asp_status asp_save_state(asp_ctx* ctx, const char* path) {
    CHECK_CTX();
    if (!path) return ASP_ERR_INVALID_ARG;
    CycleState h;
    asp_status s = read_state(ctx, &h);
    if (s != ASP_OK) return s;
    std::vector<float> R(ctx->N);
    std::vector<asp_component> comps(h.n_comp);
    CK(cudaMemcpy(R.data(), ctx->R, ctx->N * sizeof(float), cudaMemcpyDeviceToHost));
    if (h.n_comp) CK(cudaMemcpy(comps.data(), ctx->comps, h.n_comp * sizeof(asp_component), cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) return fail(ctx, ASP_ERR_INVALID_ARG, std::string("cannot open ") + path);
    int32_t hdr[6] = {(int32_t)STATE_MAGIC, ctx->H, ctx->W, h.n_comp, h.n_ret, h.t};
    bool ok = fwrite(hdr, sizeof(hdr), 1, f) == 1;
    double dd[6] = {h.last_wi, h.last_w0, ctx->alpha_b, ctx->omega_b, 0.0, 0.0};
    ok = ok && fwrite(dd, sizeof(dd), 1, f) == 1;
    ok = ok && fwrite(R.data(), sizeof(float), R.size(), f) == R.size();
    if (h.n_comp) ok = ok && fwrite(comps.data(), sizeof(asp_component), comps.size(), f) == comps.size();
    if (h.n_ret) ok = ok && fwrite(h.ret, sizeof(int), h.n_ret, f) == (size_t)h.n_ret;
    ok = (fclose(f) == 0) && ok;
    return ok ? ASP_OK : fail(ctx, ASP_ERR_INVALID_ARG, "short write");
}

asp_status asp_load_state(asp_ctx* ctx, const char* path) {
    CHECK_CTX();
    if (!path) return ASP_ERR_INVALID_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(ctx, ASP_ERR_INVALID_ARG, std::string("cannot open ") + path);
    int32_t hdr[6];
    double dd[6];
    bool ok = fread(hdr, sizeof(hdr), 1, f) == 1 && fread(dd, sizeof(dd), 1, f) == 1;
    if (!ok || hdr[0] != (int32_t)STATE_MAGIC || hdr[1] != ctx->H || hdr[2] != ctx->W || hdr[3] < 0 ||
        hdr[3] > ctx->p.max_components || hdr[4] < 0 || hdr[4] > RET_MAX) {
        fclose(f);
        return fail(ctx, ASP_ERR_INVALID_ARG, "state file does not match this context");
    }
    std::vector<float> R(ctx->N);
    std::vector<asp_component> comps(hdr[3]);
    std::vector<int> ret(hdr[4]);
    ok = fread(R.data(), sizeof(float), R.size(), f) == R.size();
    if (hdr[3]) ok = ok && fread(comps.data(), sizeof(asp_component), comps.size(), f) == comps.size();
    if (hdr[4]) ok = ok && fread(ret.data(), sizeof(int), ret.size(), f) == ret.size();
    fclose(f);
    if (!ok) return fail(ctx, ASP_ERR_INVALID_ARG, "short read");
    CK(cudaMemcpy(ctx->R, R.data(), ctx->N * sizeof(float), cudaMemcpyHostToDevice));
    return asp_set_state(ctx, comps.data(), hdr[3], ret.data(), std::min(hdr[4], ctx->p.retained_cap), hdr[5], dd[0],
                         dd[1]);
}

}  // extern "C"

// =====================================================================
// Batches: independent images advanced together, one launch per kernel of
// the iteration (images on grid.y) and one cooperative launch for all the
// images' LM fits (image i owns a fixed CTA group).
struct asp_batch {
    int dev = 0, num_sms = 0, g_total = 0;
    cudaStream_t stream = nullptr;
    std::vector<asp_ctx*> imgs;
    std::vector<float*> dirty;           // device copies of the dirty images (resets)
    std::vector<ImgDesc> h_desc;
    ImgDesc* d_desc = nullptr;
    unsigned* bars = nullptr;
    int* dmap = nullptr;                 // CTA ranges of the batched fit (device, n + 1)
    int tpt = 1, grid_x = 1;
    int px_per_cta = 0, share_policy = 0;
    size_t smem_smooth_h = 0, smem_smooth_v = 0, smem_sub_h = 0;
    cudaGraphExec_t gexec = nullptr;
    int graph_unroll = 8, graph_state = 0;
    long long launches = 0;
    int broken = 0;
    // learned initial values for the whole batch: one network input row per image
    int learned = 0, mlp_rows = 0;
    float* mlpP = nullptr;
    void *W1b = nullptr, *W2b = nullptr, *Xinf = nullptr, *H1b = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Yinf = nullptr;
    unsigned* mlp_err = nullptr;
    std::vector<void*> mlp_allocs;
    // joint wide-band fit (asp_batch_fit_joint): channel pointers, beams,
    // targets, Eq. 8 output; allocated by its first call
    const float** j_src = nullptr;
    double* j_wb2 = nullptr;     // omega_b^2 then alpha_b per channel
    float* j_T = nullptr;
    double* j_flux = nullptr;    // PMAX fluxes then PMAX point flags (as doubles)
    // work queue (asp_batch_run_queue): lane streams, the lane count and
    // window tile the images' graphs were built for
    std::vector<cudaStream_t> lanes;
    int q_lanes = 0, q_px = -1;
};

namespace {

const int BATCH_KERNELS_PER_ITER = 10;   // the 9 of an iteration plus the CTA map of the fit
const int BATCH_LEARNED_KERNELS = 11;   // prep, chi^2 fit, 5 inference kernels, apply, check, refit, pick

asp_status batch_fail(asp_batch* b, asp_status s) {
    if (b && (s == ASP_ERR_CUDA || s == ASP_ERR_TIMEOUT)) b->broken = 1;
    return s;
}

#define BK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return batch_fail(b, e_ == cudaErrorMemoryAllocation ? ASP_ERR_OOM : ASP_ERR_CUDA);    \
    } while (0)

// Caps on each image's CTA group for the batched fit: 0 equal shares, 1
// shares proportional to the image areas (each at least one CTA, summing to
// at most g_total), 2 on demand (every image may ask for all g_total CTAs;
// k_fit_map_b scales the requests of each iteration down to g_total).
void batch_shares(asp_batch* b) {
    const int n = (int)b->imgs.size();
    std::vector<int> share(n, 1);
    if (b->share_policy == 0) {
        for (int i = 0; i < n; ++i) share[i] += (b->g_total - n) / n;
    } else if (b->share_policy == 1) {
        double tot = 0;
        for (asp_ctx* c : b->imgs) tot += (double)c->N;
        for (int i = 0; i < n; ++i)
            share[i] += (int)std::floor((double)(b->g_total - n) * b->imgs[i]->N / tot);
    } else {
        for (int i = 0; i < n; ++i) share[i] = b->g_total;
    }
    for (int i = 0; i < n; ++i) b->h_desc[i].g_share = share[i];
}

asp_status batch_upload(asp_batch* b) {
    for (size_t i = 0; i < b->h_desc.size(); ++i) b->h_desc[i].dp.lm.px_per_cta = b->px_per_cta;
    BK(cudaMemcpyAsync(b->d_desc, b->h_desc.data(), b->h_desc.size() * sizeof(ImgDesc), cudaMemcpyHostToDevice,
                       b->stream));
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    b->graph_state = 0;
    return ASP_OK;
}

asp_status batch_enqueue_iteration(asp_batch* b, cudaStream_t s) {
    const int n = (int)b->imgs.size();
    BK(launch_cycle_begin_b(b->d_desc, n, s));
    BK(launch_smooth_h_b(b->d_desc, n, b->grid_x, b->smem_smooth_h, s));
    BK(launch_smooth_v_b(b->d_desc, n, b->grid_x, b->smem_smooth_v, s));
    BK(launch_select_b(b->d_desc, n, s));
    BK(launch_fit_map_b(b->d_desc, n, b->g_total, b->dmap, s));
    if (b->learned) {
        BK(launch_learned_b(b->d_desc, n, 0, s));
        BK(launch_mlp_infer(b->Xinf, b->W1b, b->W2b, b->mlpP, b->Z1, b->H1b, b->Z2, b->H2, b->Yinf, b->mlp_err, s,
                            b->mlp_rows));
        BK(launch_learned_b(b->d_desc, n, 1, s));
    }
    BK(launch_lm_fit_batched(b->tpt, b->d_desc, b->dmap, n, b->g_total, b->bars, s));
    if (b->learned) {
        BK(launch_lm_fit_batched(b->tpt, b->d_desc, b->dmap, n, b->g_total, b->bars, s, 1, -1));  // the plain start's fit
        BK(launch_learned_b(b->d_desc, n, 2, s));
    }
    BK(launch_update_b(b->d_desc, n, s));
    BK(launch_build_weights_b(b->d_desc, n, s));
    BK(launch_sub_h_b(b->d_desc, n, b->grid_x, b->smem_sub_h, s));
    BK(launch_sub_v_b(b->d_desc, n, b->grid_x, s));
    return ASP_OK;
}

asp_status batch_build_graph(asp_batch* b) {
    if (b->graph_state != 0) return ASP_OK;
    if (getenv("ASP_NO_GRAPH")) { b->graph_state = -1; return ASP_OK; }
    cudaStream_t cs = nullptr;
    BK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    asp_status s = ASP_OK;
    if (ok) {
        for (int i = 0; i < b->graph_unroll && s == ASP_OK; ++i) s = batch_enqueue_iteration(b, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        ok = (s == ASP_OK) && e == cudaSuccess && g != nullptr;
    }
    b->broken = 0;
    if (ok && cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess) {
        b->graph_state = 1;
    } else {
        b->graph_state = -1;
        cudaGetLastError();
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return ASP_OK;
}

asp_status batch_run(asp_batch* b, int n_iter) {
    const int n = (int)b->imgs.size();
    BK(launch_arm_b(b->d_desc, n, n_iter, b->stream));
    asp_status s = batch_build_graph(b);
    if (s != ASP_OK) return s;
    if (n_iter > 0) {
        if (b->graph_state == 1) {
            const int reps = (n_iter + b->graph_unroll - 1) / b->graph_unroll;
            for (int r = 0; r < reps; ++r) BK(cudaGraphLaunch(b->gexec, b->stream));
            b->launches += (long long)reps * b->graph_unroll *
                           (BATCH_KERNELS_PER_ITER + (b->learned ? BATCH_LEARNED_KERNELS : 0));
        } else {
            for (int i = 0; i < n_iter; ++i) {
                s = batch_enqueue_iteration(b, b->stream);
                if (s != ASP_OK) return s;
            }
            b->launches += (long long)n_iter * (BATCH_KERNELS_PER_ITER + (b->learned ? BATCH_LEARNED_KERNELS : 0));
        }
    }
    BK(cudaStreamSynchronize(b->stream));
    return ASP_OK;
}

#undef BK

}  // namespace

#define BK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return batch_fail(b, e_ == cudaErrorMemoryAllocation ? ASP_ERR_OOM : ASP_ERR_CUDA);    \
    } while (0)

extern "C" {

asp_status asp_batch_fit_joint(asp_batch* b, const double* init, int n, int n_old, double* out, double* flux,
                               int* is_point, asp_fit_info* info) {
    if (!b || b->broken) return b ? ASP_ERR_STATE : ASP_ERR_INVALID_ARG;
    const int C = (int)b->imgs.size();
    if (!init || !out || n < 1 || n_old < 0 || n_old > n) return ASP_ERR_INVALID_ARG;
    if ((long long)n * (3 + C) > PMAX) return ASP_ERR_UNSUPPORTED;
    asp_ctx* c0 = b->imgs[0];
    const int H = c0->H, W = c0->W;
    for (asp_ctx* c : b->imgs)
        if (c->H != H || c->W != W) return ASP_ERR_UNSUPPORTED;
    const int NPM = 3 + C;
    for (int i = 0; i < n * NPM; ++i)
        if (!std::isfinite(init[i])) return ASP_ERR_INVALID_ARG;
    if (cudaSetDevice(b->dev) != cudaSuccess) return ASP_ERR_CUDA;
    if (!b->j_src) {
        BK(cudaMalloc(&b->j_src, sizeof(float*) * C));
        BK(cudaMalloc(&b->j_wb2, sizeof(double) * 2 * C));
        BK(cudaMalloc(&b->j_T, sizeof(float) * (size_t)C * c0->N));
        BK(cudaMalloc(&b->j_flux, sizeof(double) * 2 * PMAX));
    }
    std::vector<const float*> srcs(C);
    std::vector<double> wb(2 * C);
    double max_wb2 = 0.0;
    for (int c = 0; c < C; ++c) {
        srcs[c] = b->imgs[c]->R;
        wb[c] = b->imgs[c]->omega_b * b->imgs[c]->omega_b;
        wb[C + c] = b->imgs[c]->alpha_b;
        max_wb2 = std::max(max_wb2, wb[c]);
    }
    // the shared window: member boxes of the widest convolved width
    long long wx0 = 0, wx1 = 0, wy0 = 0, wy1 = 0;
    for (int k = 0; k < n; ++k) {
        const double* r = init + (size_t)k * NPM;
        long long bx[4];
        host_member_box(r[0], r[1], std::sqrt(r[2] * r[2] + max_wb2), bx);
        if (k == 0) { wx0 = bx[0]; wx1 = bx[1]; wy0 = bx[2]; wy1 = bx[3]; }
        wx0 = std::min(wx0, bx[0]); wx1 = std::max(wx1, bx[1]);
        wy0 = std::min(wy0, bx[2]); wy1 = std::max(wy1, bx[3]);
    }
    wx0 = std::max(wx0, 0LL); wy0 = std::max(wy0, 0LL);
    wx1 = std::min(wx1, (long long)W - 1); wy1 = std::min(wy1, (long long)H - 1);
    if (wx0 > wx1 || wy0 > wy1) return ASP_ERR_INVALID_ARG;
    FitDesc d;
    memset(&d, 0, sizeof(d));
    d.K = n;
    d.n_old = n_old;
    d.model = 2;
    d.n_chan = C;
    d.chan_src = b->j_src;
    d.chan_wb2 = b->j_wb2;
    d.max_wb2 = max_wb2;
    d.wx0 = (int)wx0; d.wy0 = (int)wy0;
    d.ww = (int)(wx1 - wx0 + 1); d.wh = (int)(wy1 - wy0 + 1);
    d.omega_min = 0.0;
    d.omega_max = (double)std::max(d.ww, d.wh);
    d.bx0 = (double)wx0; d.bx1 = (double)wx1; d.by0 = (double)wy0; d.by1 = (double)wy1;
    for (int i = 0; i < n * NPM; ++i) d.theta0[i] = init[i];
    const int tpt = fit_tpt_for((n * NPM + 3) / 4);
    int bps = 0;
    if (fit_configure_model(2, tpt, &bps) != cudaSuccess || bps < 1) return batch_fail(b, ASP_ERR_CUDA);
    const int g_max = std::min(std::min(b->num_sms * bps, FIT_GRID_MAX), c0->g_max);
    LMConst lmc = c0->dp.lm;
    int smem_ok = 1;
    d.grid = fit_grid((long long)d.ww * d.wh * C, n, lmc.px_per_cta, g_max, &smem_ok);
    d.smem_ok = smem_ok;
    d.active = 1;
    cudaStream_t s = b->stream;
    BK(cudaMemcpyAsync(b->j_src, srcs.data(), sizeof(float*) * C, cudaMemcpyHostToDevice, s));
    BK(cudaMemcpyAsync(b->j_wb2, wb.data(), sizeof(double) * 2 * C, cudaMemcpyHostToDevice, s));
    BK(cudaMemcpyAsync(&c0->st->fit, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    BK(cudaMemsetAsync(&c0->st->fout, 0, sizeof(FitOut), s));
    BK(launch_lm_fit_model(2, tpt, g_max, c0->R, W, &c0->st->fit, lmc, &c0->st->fout, c0->partials, c0->sums,
                           c0->bar, b->j_T, s));
    BK(launch_joint_flux(&c0->st->fout, n, C, b->j_wb2, b->j_flux, s));
    b->launches += 2;
    FitOut fo;
    std::vector<double> fl(2 * PMAX);
    BK(cudaMemcpyAsync(&fo, &c0->st->fout, sizeof(FitOut), cudaMemcpyDeviceToHost, s));
    BK(cudaMemcpyAsync(fl.data(), b->j_flux, sizeof(double) * 2 * PMAX, cudaMemcpyDeviceToHost, s));
    BK(cudaStreamSynchronize(s));
    if (fo.error) return batch_fail(b, ASP_ERR_TIMEOUT);
    for (int i = 0; i < n * NPM; ++i) out[i] = fo.theta[i];
    if (flux)
        for (int i = 0; i < n * C; ++i) flux[i] = fl[i];
    if (is_point)
        for (int k = 0; k < n; ++k) is_point[k] = fl[PMAX + k] != 0.0;
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

asp_status asp_batch_destroy(asp_batch* b) {
    if (!b) return ASP_ERR_INVALID_ARG;
    cudaSetDevice(b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (asp_ctx* c : b->imgs) asp_destroy(c);
    for (float* d : b->dirty) cudaFree(d);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->bars) cudaFree(b->bars);
    if (b->dmap) cudaFree(b->dmap);
    for (void* q : b->mlp_allocs) cudaFree(q);
    for (cudaStream_t l : b->lanes) cudaStreamDestroy(l);
    if (b->j_src) cudaFree(b->j_src);
    if (b->j_wb2) cudaFree(b->j_wb2);
    if (b->j_T) cudaFree(b->j_T);
    if (b->j_flux) cudaFree(b->j_flux);
    delete b;
    return ASP_OK;
}

asp_status asp_batch_create(const asp_params* params, int n, const int* H, const int* W,
                            const float* const* dirty, const float* const* psf, int on_host, void* stream,
                            asp_batch** out) {
    if (!out) return ASP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || n < 1 || n > MAX_BATCH || !H || !W || !dirty || !psf) return ASP_ERR_INVALID_ARG;
    if (params->major_every != 0) return ASP_ERR_UNSUPPORTED;   // the minor/major split is per context
    if (params->sub_mode == ASP_SUB_FFT) return ASP_ERR_UNSUPPORTED;   // batch iterations subtract directly
    for (int i = 0; i < n; ++i)
        if (H[i] < 1 || W[i] < 1 || !dirty[i] || !psf[i]) return ASP_ERR_INVALID_ARG;
    asp_batch* b = new asp_batch();
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    auto bail = [&](asp_status st) { asp_batch_destroy(b); return st; };
    if (cudaGetDevice(&b->dev) != cudaSuccess) return bail(ASP_ERR_CUDA);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, b->dev) != cudaSuccess) return bail(ASP_ERR_CUDA);
    b->num_sms = prop.multiProcessorCount;
    asp_params ip = *params;
    ip.sub_mode = ASP_SUB_DIRECT;   // the images' contexts hold no FFT buffers
    for (int i = 0; i < n; ++i) {
        asp_ctx* c = nullptr;
        asp_status s = on_host ? asp_init_host(&ip, H[i], W[i], dirty[i], psf[i], stream, &c)
                               : asp_init(&ip, H[i], W[i], dirty[i], psf[i], stream, &c);
        if (s != ASP_OK) return bail(s);
        b->imgs.push_back(c);
        float* d = nullptr;
        if (cudaMalloc(&d, (size_t)c->N * sizeof(float)) != cudaSuccess) return bail(ASP_ERR_OOM);
        b->dirty.push_back(d);
        if (cudaMemcpyAsync(d, dirty[i], (size_t)c->N * sizeof(float),
                            on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
            return bail(ASP_ERR_CUDA);
    }
    b->tpt = b->imgs[0]->tpt;
    b->px_per_cta = params->fit_px_per_cta;
    int bps = 0;
    if (fit_configure(b->tpt, &bps) != cudaSuccess || bps < 1) return bail(ASP_ERR_CUDA);
    b->g_total = std::min(b->num_sms * bps, FIT_GRID_MAX);
    if (n > b->g_total) return bail(ASP_ERR_UNSUPPORTED);
    if (cudaMalloc(&b->bars, sizeof(unsigned) * n) != cudaSuccess ||
        cudaMalloc(&b->dmap, sizeof(int) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&b->d_desc, sizeof(ImgDesc) * n) != cudaSuccess)
        return bail(ASP_ERR_OOM);
    long long n_max = 0;
    b->h_desc.resize(n);
    for (int i = 0; i < n; ++i) {
        asp_ctx* c = b->imgs[i];
        ImgDesc& g = b->h_desc[i];
        memset(&g, 0, sizeof(g));
        g.R = c->R; g.B = c->B; g.H = c->H; g.W = c->W;
        g.st = c->st; g.comps = c->comps; g.hist = c->hist;
        g.wbuf = c->wbuf; g.T1 = c->T1; g.S1 = c->S1;
        g.taps = c->taps; g.smooth_flops = c->smooth_flops;
        g.partials = c->partials; g.sums = c->sums; g.bar = b->bars + i; g.Tg = c->Tg;
        g.part = c->part; g.ticket = c->ticket;
        g.dp = c->dp;
        g.sub_blen = sub_h_blen(c->W, c->taps);
        b->smem_smooth_h = std::max(b->smem_smooth_h, smooth_h_smem(c->taps));
        b->smem_smooth_v = std::max(b->smem_smooth_v, smooth_v_smem(c->taps));
        b->smem_sub_h = std::max(b->smem_sub_h, (size_t)c->taps.rpb * g.sub_blen * sizeof(float));
        n_max = std::max(n_max, c->N);
    }
    if (b->smem_smooth_h > 48 * 1024 || b->smem_sub_h > 48 * 1024) return bail(ASP_ERR_UNSUPPORTED);
    // image-wide kernels: enough blocks per image for the largest one (64k
    // pixels a block); smaller images leave most of theirs idle
    b->grid_x = (int)std::min<long long>(std::max<long long>((n_max + 65535) / 65536, 4), b->imgs[0]->grid_img);
    batch_shares(b);
    asp_status s = batch_upload(b);
    if (s != ASP_OK) return bail(s);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bail(ASP_ERR_CUDA);
    *out = b;
    return ASP_OK;
}

asp_status asp_batch_reset(asp_batch* b) {
    if (!b) return ASP_ERR_INVALID_ARG;
    if (b->broken) return ASP_ERR_STATE;
    cudaSetDevice(b->dev);
    for (size_t i = 0; i < b->imgs.size(); ++i) {
        asp_ctx* c = b->imgs[i];
        // the image's statistics restart with it
        asp_status s = asp_reset(c, b->dirty[i], 0, nullptr, 0);
        if (s != ASP_OK) return batch_fail(b, s);
    }
    BK(cudaStreamSynchronize(b->stream));
    return ASP_OK;
}

asp_status asp_batch_minor_cycle(asp_batch* b, int n_iter, asp_cycle_stats* stats) {
    if (!b || n_iter < 0) return ASP_ERR_INVALID_ARG;
    if (b->broken) return ASP_ERR_STATE;
    cudaSetDevice(b->dev);
    asp_status s = batch_run(b, n_iter);
    if (s != ASP_OK) return s;
    if (b->learned) {
        unsigned me = 0;
        BK(cudaMemcpy(&me, b->mlp_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
        if (me) { b->broken = 1; return ASP_ERR_TIMEOUT; }
    }
    asp_status first_err = ASP_OK;
    for (size_t i = 0; i < b->imgs.size(); ++i) {
        asp_ctx* c = b->imgs[i];
        CycleState h;
        BK(cudaMemcpyAsync(&h, c->st, sizeof(CycleState), cudaMemcpyDeviceToHost, b->stream));
        BK(cudaStreamSynchronize(b->stream));
        if (h.error == ASP_ERR_TIMEOUT) { b->broken = 1; return ASP_ERR_TIMEOUT; }
        if ((h.error == ASP_ERR_NAN || h.nonfinite) && first_err == ASP_OK) first_err = ASP_ERR_NAN;
        if (h.stop_reason == ASP_STOP_CAPACITY && first_err == ASP_OK) first_err = ASP_ERR_CAPACITY;
        if (stats) {
            fill_stats(h, &stats[i]);
        }
    }
    return first_err;
}

asp_status asp_batch_run_queue(asp_batch* b, int n_iter, int n_lanes, int px_per_cta, asp_cycle_stats* stats) {
    if (!b || n_iter < 0 || n_lanes < 1 || n_lanes > 64 || px_per_cta < 0) return ASP_ERR_INVALID_ARG;
    if (b->broken) return ASP_ERR_STATE;
    if (b->learned) return ASP_ERR_UNSUPPORTED;   // the batch's network runs in the lock-step iteration
    cudaSetDevice(b->dev);
    const int n = (int)b->imgs.size();
    // lane streams, and each image's fit grid capped so that the lanes'
    // cooperative fits fit the GPU side by side; the graphs are rebuilt for
    // the cap (and the window tile) once per configuration
    while ((int)b->lanes.size() < n_lanes) {
        cudaStream_t l = nullptr;
        BK(cudaStreamCreateWithFlags(&l, cudaStreamNonBlocking));
        b->lanes.push_back(l);
    }
    if (b->q_lanes != n_lanes || b->q_px != px_per_cta) {
        const int cap = std::max(1, (b->num_sms + n_lanes - 1) / n_lanes);
        for (asp_ctx* c : b->imgs) {
            c->g_max = std::min(c->g_alloc, cap);
            c->dp.lm.px_per_cta = px_per_cta > 0 ? px_per_cta : c->p.fit_px_per_cta;
            if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
            c->graph_state = 0;
            asp_status gs = build_graph(c);
            if (gs != ASP_OK) return gs;
        }
        b->q_lanes = n_lanes;
        b->q_px = px_per_cta;
    }
    // lanes start after the batch stream's earlier work
    cudaEvent_t ev0;
    BK(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
    BK(cudaEventRecord(ev0, b->stream));
    for (int l = 0; l < n_lanes; ++l) BK(cudaStreamWaitEvent(b->lanes[l], ev0, 0));
    cudaEventDestroy(ev0);
    // longest first onto the least-loaded lane (cost: image pixels)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->imgs[a]->N > b->imgs[c]->N; });
    std::vector<long long> load(n_lanes, 0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += b->imgs[i]->N;
        asp_ctx* c = b->imgs[i];
        cudaStream_t saved = c->stream;
        c->stream = b->lanes[l];
        asp_status es = ASP_OK;
        if (launch_arm_b(b->d_desc + i, 1, n_iter, c->stream) != cudaSuccess) es = ASP_ERR_CUDA;
        b->launches += 1;
        if (es == ASP_OK && n_iter > 0) {
            if (c->graph_state == 1) {
                const int reps = (n_iter + c->graph_unroll - 1) / c->graph_unroll;
                for (int r = 0; r < reps && es == ASP_OK; ++r)
                    if (cudaGraphLaunch(c->gexec, c->stream) != cudaSuccess) es = ASP_ERR_CUDA;
                b->launches += (long long)reps * c->graph_kernels;
            } else {
                const long long l0 = c->launches;
                for (int it = 0; it < n_iter && es == ASP_OK; ++it) es = enqueue_iteration(c);
                b->launches += c->launches - l0;
            }
        }
        c->stream = saved;
        if (es != ASP_OK) return batch_fail(b, es);
    }
    for (int l = 0; l < n_lanes; ++l) {
        cudaEvent_t ev;
        BK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        BK(cudaEventRecord(ev, b->lanes[l]));
        BK(cudaStreamWaitEvent(b->stream, ev, 0));
        cudaEventDestroy(ev);
    }
    BK(cudaStreamSynchronize(b->stream));
    asp_status first_err = ASP_OK;
    for (int i = 0; i < n; ++i) {
        CycleState h;
        BK(cudaMemcpyAsync(&h, b->imgs[i]->st, sizeof(CycleState), cudaMemcpyDeviceToHost, b->stream));
        BK(cudaStreamSynchronize(b->stream));
        if (h.error == ASP_ERR_TIMEOUT) { b->broken = 1; return ASP_ERR_TIMEOUT; }
        if ((h.error == ASP_ERR_NAN || h.nonfinite) && first_err == ASP_OK) first_err = ASP_ERR_NAN;
        if (h.stop_reason == ASP_STOP_CAPACITY && first_err == ASP_OK) first_err = ASP_ERR_CAPACITY;
        if (stats) fill_stats(h, &stats[i]);
    }
    return first_err;
}

asp_status asp_batch_autotune(asp_batch* b, int n_trial_iter, asp_batch_tuning* out) {
    if (!b || n_trial_iter < 1) return ASP_ERR_INVALID_ARG;
    if (b->broken) return ASP_ERR_STATE;
    cudaSetDevice(b->dev);
    const int cand_px[] = {0, 48, 192, 384, 768, 1536};   // pixels per CTA (0: the default, 96)
    const int n_px = (int)(sizeof(cand_px) / sizeof(cand_px[0]));
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    double best = 1e300, dflt = 0.0;
    int best_px = 0, best_pol = 0, tried = 0;
    asp_status s = ASP_OK;
    for (int pol = 0; pol < 3 && s == ASP_OK; ++pol)
        for (int k = 0; k < n_px && s == ASP_OK; ++k) {
            b->share_policy = pol;
            b->px_per_cta = cand_px[k];
            batch_shares(b);
            s = batch_upload(b);
            if (s == ASP_OK) s = asp_batch_reset(b);
            if (s == ASP_OK) s = batch_build_graph(b);
            if (s != ASP_OK) break;
            BK(cudaEventRecord(e0, b->stream));
            s = batch_run(b, n_trial_iter);
            BK(cudaEventRecord(e1, b->stream));
            BK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BK(cudaEventElapsedTime(&ms, e0, e1));
            ++tried;
            if (pol == 0 && k == 0) dflt = ms;
            if (ms < best) { best = ms; best_px = cand_px[k]; best_pol = pol; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != ASP_OK) return s;
    b->share_policy = best_pol;
    b->px_per_cta = best_px;
    batch_shares(b);
    s = batch_upload(b);
    if (s == ASP_OK) s = asp_batch_reset(b);
    if (s != ASP_OK) return s;
    if (out) {
        out->px_per_cta = best_px;
        out->share_policy = best_pol;
        out->n_candidates = tried;
        out->best_ms = best;
        out->default_ms = dflt;
    }
    return ASP_OK;
}

asp_status asp_batch_set_mlp(asp_batch* b, const float* params_host, int enable) {
    if (!b || (enable && !params_host)) return ASP_ERR_INVALID_ARG;
    if (b->broken) return ASP_ERR_STATE;
    cudaSetDevice(b->dev);
    const int n = (int)b->imgs.size();
    if (enable) {
        if (!b->mlpP) {
            b->mlp_rows = ((n + 127) / 128) * 128;
            const size_t R = b->mlp_rows;
            auto al = [&](void** p, size_t bytes) -> bool {
                if (cudaMalloc(p, bytes) != cudaSuccess) return false;
                b->mlp_allocs.push_back(*p);
                return true;
            };
            void *P = nullptr, *z1 = nullptr, *z2 = nullptr, *h2 = nullptr, *y = nullptr, *er = nullptr;
            if (!al(&P, mlp_num_params() * sizeof(float)) || !al(&b->W1b, 256 * 1024 * 2) || !al(&b->W2b, 256 * 256 * 2) ||
                !al(&b->Xinf, R * 1024 * 2) || !al(&b->H1b, R * 256 * 2) || !al(&z1, R * 256 * 4) ||
                !al(&z2, R * 256 * 4) || !al(&h2, R * 256 * 4) || !al(&y, R * 4 * 4) || !al(&er, sizeof(unsigned)))
                return ASP_ERR_OOM;
            b->mlpP = (float*)P; b->Z1 = (float*)z1; b->Z2 = (float*)z2; b->H2 = (float*)h2; b->Yinf = (float*)y;
            b->mlp_err = (unsigned*)er;
            BK(cudaMemsetAsync(b->Xinf, 0, R * 1024 * 2, b->stream));
            BK(cudaMemsetAsync(b->mlp_err, 0, sizeof(unsigned), b->stream));
            for (int i = 0; i < n; ++i) {
                BK(cudaMemsetAsync(&b->imgs[i]->st->fit2, 0, sizeof(FitDesc), b->stream));
                b->h_desc[i].Xrow = static_cast<uint16_t*>(b->Xinf) + (size_t)i * 1024;
                b->h_desc[i].Yrow = b->Yinf + (size_t)i * 4;
            }
        }
        BK(cudaMemcpyAsync(b->mlpP, params_host, mlp_num_params() * sizeof(float), cudaMemcpyHostToDevice, b->stream));
        BK(mlp_prepare(b->mlpP, b->W1b, b->W2b, b->stream));
    }
    b->learned = enable ? 1 : 0;
    asp_status s = batch_upload(b);
    if (s != ASP_OK) return s;
    BK(cudaStreamSynchronize(b->stream));
    return ASP_OK;
}

asp_status asp_batch_image(asp_batch* b, int i, asp_ctx** ctx) {
    if (!b || !ctx || i < 0 || i >= (int)b->imgs.size()) return ASP_ERR_INVALID_ARG;
    *ctx = b->imgs[i];
    return ASP_OK;
}

asp_status asp_batch_launch_count(asp_batch* b, int64_t* n) {
    if (!b || !n) return ASP_ERR_INVALID_ARG;
    *n = b->launches;
    return ASP_OK;
}

}  // extern "C"
#undef BK
