// Internal device-side definitions of libasp (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/asp.h"

namespace aspd {

// ---------------------------------------------------------------- limits
constexpr int KMAX = ASP_KMAX;                     // members per fit
constexpr int PMAX = 4 * KMAX;                     // parameters per fit
constexpr int NAP_MAX = PMAX + 4;                  // [J | r] columns padded to 4
constexpr int NB_MAX = NAP_MAX / 4;                // 4x4 tiles per side
constexpr int NTILES_MAX = NB_MAX * (NB_MAX + 1) / 2;
constexpr int NACC_MAX = NTILES_MAX * 16;          // accumulator entries (tile order)
constexpr int FIT_GRID_MAX = 1024;                 // CTAs of one fit group (at most)
// fit sums: two FP64 buffers, their two FP32 copies, then each CTA's chi^2
// partial pair (two buffers of FIT_GRID_MAX float2)
constexpr int SUMS_DOUBLES = 3 * NACC_MAX + 2 * FIT_GRID_MAX;
constexpr int MAX_TERMS = 2 * KMAX;                // subtraction terms per iteration
constexpr int T1_SLACK_ROWS = 32;                  // rows behind the last subtraction term (the column pass's prefetch)
constexpr int MAX_SCALES = 8;                      // smoothing scales
constexpr int FIT_THREADS = 256;
constexpr int PX_SMEM = 12288;                     // target pixels one CTA keeps in smem
constexpr int FIT_PX_PER_CTA = 96;                 // default fit tile: window pixels per CTA (measured best on the 1024^2 workload)
constexpr int RET_MAX = 1024;                      // retained-list capacity
constexpr int RED_THREADS = 256;                   // threads of the image-wide kernels
constexpr unsigned SPIN_LIMIT = 1u << 22;          // bounded grid-barrier wait (polls of ~0.3 us: ~1-2 s)

constexpr double LOG2E = 1.4426950408889634074;

// Asp-Clean2004's objective (asp_fit_2004): members per fit and the packed
// upper triangle of [J | r]^T [J | r] at that size.
constexpr int FIT2004_KMAX = 8;
constexpr int FIT2004_NA = 4 * FIT2004_KMAX + 1;
constexpr int FIT2004_NACC = FIT2004_NA * (FIT2004_NA + 1) / 2;

// ---------------------------------------------------------------- structs
struct LMConst {
    double lambda0, lambda_up, lambda_down, lambda_min, lambda_max, rtol, xtol;
    int max_iter;
    int px_per_cta;   // launch-shape knob: target window pixels per CTA
};

// One joint fit: K members, the trailing n_old of which are added back into
// the target (at their theta0 values).  Window in source-image coordinates.
struct FitDescHead {
    int K, n_old;
    int wx0, wy0, ww, wh;
    int use_mask, grid;
    double mcx, mcy, mr2;          // optional circular pixel mask (beam fit)
    double omega_min, omega_max;   // trial widths must lie in (omega_min, omega_max]
    double bx0, bx1, by0, by1;     // trial centres must stay inside this box
    int active, smem_ok;
    int model, pad_model;          // 0: circular members (a, x, y, omega); 1: elliptical (a, x, y, A, B, C);
                                   // 2: joint over n_chan channels (x, y, s, a_1 .. a_C)
    int n_chan, pad_chan;          // model 2: channels, each an image of the same size (row stride src_w)
    const float* const* chan_src;  // model 2: the channels' images (device array of n_chan pointers)
    const double* chan_wb2;        // model 2: omega_b^2 of each channel's beam (device)
    double max_wb2;                // model 2: the largest of them
    double theta0[PMAX];
};
// The fit's description plus an optional LM start other than theta0 (which
// still defines the added-back members' images in the target, the window
// and the trial bounds): restarting LM from any point of a fit.  The fit
// kernel keeps only the head in shared memory and reads the start once.
struct FitDesc : FitDescHead {
    int has_start, pad_start;
    double start[PMAX];
};

struct FitOut {
    double theta[PMAX];
    double chi2_init, chi2, lambda;
    int iters, passes, status, error;
    long long pixel_evals;
    long long ns_pass, ns_reduce, ns_solve;   // time split of the fit (CTA 0)
    long long ns_factor, ns_subst;            // parts of ns_solve: damped solves, LM logic
    int refinements, fallbacks;               // FP64 refinement steps, FP64-factor fallbacks
    double trial[PMAX];                       // the last proposed point (theta + delta of the last solve)
    double chi2_trial;                        // chi^2 of the last pixel pass (at the last evaluated point)
};

// A separable subtraction term: image value scale * wx[i] * wy[j] at
// (qx0 + i, qy0 + j).
struct TermDesc {
    int qx0, nx, qy0, ny;          // clipped support
    float scale;                   // signed flux
    int woff_x, woff_y;            // offsets of wx, wy in the weight buffer
    int r0;                        // first PSF row the horizontal pass needs
    long long t1off;               // offset of this term's rows in the T1 buffer
    double cx, cy, w;              // component centre and width
    int bilinear;                  // 1: bilinear point deposit, 0: sampled Gaussian
    int ux0, ux1, uy0, uy1;        // unclipped support (normalisation range)
    int pad;
};

// One bilinear point deposit of dC: weight w at image pixel (qx, qy).
struct Deposit {
    int qx, qy;
    float w;
    int pad;
};
constexpr int MAX_DEPOSITS = 4 * MAX_TERMS;

struct ArgRes {                    // argmax of |v| with its signed value
    float val;
    int j;                         // scale index (smoothing) or 0
    long long idx;
};

// Minor-cycle control block (device memory).
struct CycleState {
    int t, t_stop, stopped, stop_reason;
    int mode, error, n_comp, cap_comp;
    int n_ret, n_terms, K, skip_smooth;
    double last_wi, last_w0;
    double thr;                    // stop threshold on max|R|
    double alpha_b, omega_b;
    double init[4];
    int init_scale, pad1;
    float init_value, init_s;
    ArgRes peak;                   // argmax |R| of the current residual
    ArgRes speak;                  // argmax |S_j| of the last smoothing
    int members[KMAX];             // component index of each fit member (-1: new)
    long long pixel_evals, lm_iters, lm_passes;
    double fit_flops, sub_flops, sub_bytes, smooth_flops;   // algorithmic work totals
    double fit_ex2;                                         // exponentials of the LM passes (K per pixel evaluation)
    long long smooth_iters;                                 // iterations that ran the smoothing peak search
    long long fit_ns_pass, fit_ns_reduce, fit_ns_solve;     // fit time split
    long long fit_ns_factor, fit_ns_subst;
    long long fit_refinements, fit_fallbacks;
    unsigned cnt_argmax, cnt_smooth, nonfinite, pad2;
    int ret[RET_MAX];
    TermDesc terms[MAX_TERMS];
    int n_dep, pad3;
    Deposit dep[MAX_DEPOSITS];     // point-like terms as bilinear deposits
    FitDesc fit;
    FitOut fout;
    // learned initial values: the plain start, a second fit (chi^2 at the
    // plain start, then the fallback refit) and the counters
    FitDesc fit2;
    FitOut fout2;
    double plain_theta[4];
    double learned_rp;             // R(p*) at the plain peak
    int learned_px, learned_py;    // the plain peak pixel
    int learned_used, need_plain;
    long long learned_fits, learned_refits, learned_kept;
    // minor/major split: minor iterations since the last exact residual,
    // whether the current major cycle is skipped, major cycles applied
    int since_major, major_skip;
    long long major_cycles;
    // FFT residual update: the change image's box of the last update (the
    // next one clears it) and of the current one (x0, x1, y0, y1; empty
    // when x0 > x1)
    int dbox[4], dbox_next[4];
};

struct Params {                    // device copy of asp_params plus derived values
    float gain, area_frac;
    int k_max, init_mode, retained_cap, n_scales;
    int major_every, pad_p;
    double tau;
    LMConst lm;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ long long round_half_up(double v) { return (long long)floor(v + 0.5); }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Arrival with release semantics (orders this thread's earlier writes, and
// those it observed through a block barrier, before the increment).
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// |a| beats |b|, ties: lower scale index, then lower flat index.
__device__ __forceinline__ bool arg_better(float av, int aj, long long ai, float bv, int bj, long long bi) {
    float fa = fabsf(av), fb = fabsf(bv);
    if (fa > fb) return true;
    if (!(fa >= fb)) return false;   // smaller, or a NaN on either side

    if (aj != bj) return aj < bj;
    return ai < bi;
}

__device__ __forceinline__ void arg_warp_reduce(float& v, int& j, long long& i) {
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_down_sync(0xffffffffu, v, o);
        int oj = __shfl_down_sync(0xffffffffu, j, o);
        long long oi = __shfl_down_sync(0xffffffffu, i, o);
        if (arg_better(ov, oj, oi, v, j, i)) { v = ov; j = oj; i = oi; }
    }
}

// Member box of the fit window: half-width max(5, ceil(4 w)) around the
// rounded centre (inclusive, unclipped).
// Axis weights of one subtraction term in the weight buffer: wx then wy,
// each stored reversed and zero-padded to a multiple of 8 taps, each
// region 16-byte aligned.
__device__ __host__ inline int wslot_x_len(int W) { return (W + 8 + 3) & ~3; }
__device__ __host__ inline int wslot_stride(int W, int H) { return wslot_x_len(W) + ((H + 8 + 3) & ~3); }

__device__ __host__ inline void member_box(double x, double y, double w, long long* b) {
    long long h = (long long)ceil(4.0 * w);
    if (h < 5) h = 5;
    long long rx = (long long)floor(x + 0.5), ry = (long long)floor(y + 0.5);
    b[0] = rx - h; b[1] = rx + h; b[2] = ry - h; b[3] = ry + h;
}

// Algorithmic FP32 work of one LM pixel evaluation with K members: per
// member 15 flops (offsets, r^2, exponent argument, g, model sum, three
// Jacobian products) plus one ex2; one residual subtraction; and the upper
// triangle of [J | r]^T [J | r] as FMAs, (P + 1)(P + 2) / 2 of them (P = 4K).
__device__ __host__ inline double pixel_eval_flops(int K) {
    const double P = 4.0 * K;
    return 15.0 * K + 1.0 + (P + 1.0) * (P + 2.0);
}

__device__ __host__ inline int fit_tiles(int K) {
    int NA = 4 * K + 1;
    int NAp = (NA + 3) & ~3;
    int nb = NAp / 4;
    return nb * (nb + 1) / 2;
}

// CTAs a fit of K members over Wn pixels uses: one CTA per px_per_cta
// window pixels (default FIT_PX_PER_CTA), capped at g_max.  An LM iteration
// is latency-bound (grid barriers and the serial solve dominate), so the
// accumulation phase is spread as thin as the barriers allow; windows below
// one tile run on a single CTA without grid barriers.
// CTAs of a fit group of G that hold window pixels: with three or more,
// the last one holds none and solves the damped system speculatively (the
// step a rejected trial asks for next) while the others run the pass.
__device__ __host__ inline int fit_pixel_ctas(int G) { return G >= 3 ? G - 1 : G; }

// Whether the window's pixel slices (split over the group's pixel CTAs) fit
// each CTA's shared-memory target buffer.
__device__ __host__ inline int fit_smem_ok(long long Wn, int G) {
    const long long gp = fit_pixel_ctas(G);
    return ((Wn + gp - 1) / gp) <= PX_SMEM;
}

__device__ __host__ inline int fit_grid(long long Wn, int K, int px_per_cta, int g_max, int* smem_ok) {
    (void)K;   // one tile size serves every active-set size (measured)
    long long target = px_per_cta > 0 ? px_per_cta : FIT_PX_PER_CTA;
    if (target < 32) target = 32;
    if (target > PX_SMEM) target = PX_SMEM;
    long long g = (Wn + target - 1) / target;
    if (g < 1) g = 1;
    if (g > g_max) g = g_max;
    *smem_ok = fit_smem_ok(Wn, (int)g);
    return (int)g;
}

}  // namespace aspd
