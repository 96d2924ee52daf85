// Host-side launchers shared between the translation units of libasp.
#pragma once
#include <cuda_runtime.h>
#include <cufft.h>

#include "asp_dev.cuh"

namespace aspd {

struct SmoothTaps {          // unit-L2 1-D smoothing kernels, passed by value
    const float* k;          // all taps, scale j at k + off[j], length 2 m[j] + 1
    int off[MAX_SCALES];
    int m[MAX_SCALES];
    int t8[MAX_SCALES];      // 2 m[j] + 1 rounded up to 8 (zero taps beyond 2 m[j])
    double scale[MAX_SCALES];
    int n;
    int t8max;               // max over scales of t8
    // launch geometry of the register-blocked passes (8 outputs per thread)
    int tpr;                 // row pass: threads per row segment (multiple of 32, <= 256)
    int rpb;                 // row pass: row segments per block (256 / tpr)
    int nseg;                // row pass: segments per image row
    int blen;                // row pass: shared floats per segment buffer (bank-padded)
    int pair_h;              // row pass takes two rows per thread (packed FMAs) when its buffers fit
    int mpad;                // zero halo rows above and below each scale's row-pass image
    long long s1rows;        // rows of each scale's row-pass image (H + 2 mpad + 8)
};

// One image of a batch as the batched kernels see it (device memory).
struct ImgDesc {
    float* R;
    const float* B;
    int H, W;
    CycleState* st;
    asp_component* comps;
    asp_iter_record* hist;
    float* wbuf;
    float* T1;
    float* S1;
    SmoothTaps taps;
    double smooth_flops;
    double* partials;
    double* sums;
    unsigned* bar;
    float* Tg;
    ArgRes* part;
    unsigned* ticket;
    Params dp;
    int g_share;        // CTAs of the batched fit given to this image
    int sub_blen;       // floats of one row-pass buffer of the subtraction
    void* Xrow;         // learned initial values: this image's row of the shared network input (BF16)
    const float* Yrow;  // and of the network output (4 floats)
};

constexpr int MAX_BATCH = 256;

int sub_h_blen(int W, const SmoothTaps& geo);
size_t smooth_h_smem(const SmoothTaps& t);   // dynamic shared bytes of the row pass (its chosen form)
size_t smooth_v_smem(const SmoothTaps& t);   // ... of the column pass
int smooth_grid_h(const SmoothTaps& t, int num_sms, int cap);   // resident blocks of the row pass (<= cap)
int smooth_grid_v(const SmoothTaps& t, int num_sms, int cap);   // ... of the column pass

// asp_fit.cu
size_t fit_smem_bytes();
size_t fit_smem_bytes(int variant);
int fit_tpt_for(int k_max);
cudaError_t fit_configure(int tpt, int* blocks_per_sm);
// the elliptical (model 1) and joint wide-band (model 2) fit kernels
cudaError_t fit_configure_model(int model, int variant, int* blocks_per_sm);
cudaError_t launch_lm_fit_model(int model, int tpt, int grid, const float* src, int src_w, const FitDesc* desc,
                                const LMConst& lmc, FitOut* out, double* partials, double* sums, unsigned* bar,
                                float* Tg, cudaStream_t s);
cudaError_t launch_lm_fit_batched(int tpt, const ImgDesc* imgs, const int* dmap, int n, int g_total, unsigned* bars,
                                  cudaStream_t s, int which = 0, int max_iter_override = -1);
cudaError_t launch_lm_fit_pair(int tpt, int grid, const float* src, int src_w, const LMConst& lmc, const FitDesc* dA,
                               FitOut* oA, double* pA, double* sA, unsigned* bA, float* tA, const FitDesc* dB,
                               FitOut* oB, double* pB, double* sB, unsigned* bB, float* tB, cudaStream_t s);
cudaError_t launch_lm_fit(int tpt, int grid, const float* src, int src_w, const FitDesc* desc, const LMConst& lmc,
                          FitOut* out, double* partials, double* sums, unsigned* bar, float* Tg, cudaStream_t s);

// asp_image.cu (one kernel per launcher)
cudaError_t launch_argmax(const float* R, long long N, int grid, ArgRes* part, unsigned* ticket, ArgRes* res,
                          unsigned* nonfinite, const int* gate, cudaStream_t s);
cudaError_t launch_sub_h(const float* B, int H, int W, const CycleState* st, const int* gate, const float* wbuf,
                          float* T1, int grid, const SmoothTaps& geo, cudaStream_t s);
cudaError_t launch_sub_v(float* R, const float* B, int H, int W, CycleState* st, const int* gate, const float* wbuf,
                         const float* T1, int grid, ArgRes* part, unsigned* ticket, cudaStream_t s);
// sched: two zeroed unsigned task counters of this pass (nullptr: static order)
cudaError_t launch_smooth_h(const float* R, int H, int W, const SmoothTaps& taps, const int* gate, int only_scale,
                            float* S1, int grid, unsigned* sched, cudaStream_t s);
cudaError_t launch_smooth_v(const float* S1, int H, int W, const SmoothTaps& taps, CycleState* st, const int* gate,
                            int only_scale, float* out_S, int grid, ArgRes* part, unsigned* ticket, unsigned* sched,
                            cudaStream_t s);

// asp_major.cu (minor/major split)
cudaError_t launch_sub_gauss(float* R, int H, int W, CycleState* st, int grid, cudaStream_t s);
cudaError_t launch_fft_sub_argmax(float* R, const float* conv, int H, int W, CycleState* st, const int* gate, int grid,
                                  ArgRes* part, unsigned* ticket, cudaStream_t s);
cudaError_t launch_sub_fft(CycleState* st, const int* gate, const float* wbuf, int H, int W, float* pad_in,
                           cufftComplex* work, const cufftComplex* bhat, float* conv_out, float* R, cufftHandle r2c,
                           cufftHandle c2r, int grid, ArgRes* part, unsigned* ticket, cudaStream_t s);
cudaError_t launch_major(const asp_component* comps, float2* norms, CycleState* st, int H, int W, float* pad_in,
                         cufftComplex* work, const cufftComplex* bhat, float* conv_out, float* R, const float* D,
                         cufftHandle r2c, cufftHandle c2r, int grid, cudaStream_t s);
cudaError_t compute_psf_transform(const float* B, int H, int W, float* pad_in, cufftComplex* bhat, cufftHandle r2c,
                                  cudaStream_t s);

// asp_2004.cu (Asp-Clean2004's objective)
struct Fit2004Buffers {
    float* imgs = nullptr;          // FIT2004_NA zero-padded 2H x 2W images
    float* conv = nullptr;          // their PSF convolutions (same layout)
    cufftComplex* work = nullptr;   // FIT2004_NA transforms of 2H x (W + 1)
    cufftComplex* bhat = nullptr;   // the PSF's transform
    float* T = nullptr;             // target image H x W
    float2* partials = nullptr;     // ne_blocks x FIT2004_NACC pairs
    double* sums = nullptr;         // FIT2004_NACC
    double* theta = nullptr;        // 4 FIT2004_KMAX
    cufftHandle r2c1 = 0, c2r1 = 0, r2cN = 0, c2rN = 0;
    int nb = 0;                     // batch of the N plans (4K + 1)
    int grid = 0, ne_blocks = 0;
};
cudaError_t eval_2004(const Fit2004Buffers& fb, const double* theta_dev, int K, int n_img, int H, int W,
                      const float* R, bool target_only, cudaStream_t s);
cudaError_t psf_transform_2004(const Fit2004Buffers& fb, const float* B, int H, int W, cudaStream_t s);

// asp_cycle.cu
cudaError_t launch_cycle_begin(CycleState* st, const Params& p, int H, int W, double smooth_flops, cudaStream_t s);
cudaError_t launch_select(CycleState* st, const asp_component* comps, const Params& p, int H, int W, int g_max,
                          cudaStream_t s);
cudaError_t launch_update(CycleState* st, asp_component* comps, asp_iter_record* hist, const Params& p, int H,
                          int W, cudaStream_t s);
cudaError_t launch_build_weights(CycleState* st, const int* gate, float* wbuf, cudaStream_t s);
cudaError_t launch_terms_from_components(CycleState* st, const asp_component* comps, int n, float gain, int H,
                                         int W, cudaStream_t s);
cudaError_t launch_reset_state(CycleState* st, cudaStream_t s);

// asp_setup.cu
// batched iteration kernels (grid.y = image; grid_x blocks per image)
cudaError_t launch_cycle_begin_b(const ImgDesc* imgs, int n, cudaStream_t s);
cudaError_t launch_smooth_h_b(const ImgDesc* imgs, int n, int grid_x, size_t smem, cudaStream_t s);
cudaError_t launch_smooth_v_b(const ImgDesc* imgs, int n, int grid_x, size_t smem, cudaStream_t s);
cudaError_t launch_select_b(const ImgDesc* imgs, int n, cudaStream_t s);
cudaError_t launch_update_b(const ImgDesc* imgs, int n, cudaStream_t s);
cudaError_t launch_build_weights_b(const ImgDesc* imgs, int n, cudaStream_t s);
cudaError_t launch_sub_h_b(const ImgDesc* imgs, int n, int grid_x, size_t smem, cudaStream_t s);
cudaError_t launch_sub_v_b(const ImgDesc* imgs, int n, int grid_x, cudaStream_t s);
cudaError_t launch_arm_b(const ImgDesc* imgs, int n, int n_iter, cudaStream_t s);
cudaError_t launch_fit_map_b(const ImgDesc* imgs, int n, int g_total, int* dmap, cudaStream_t s);
// learned initial values (asp_mlp.cu, asp_cycle.cu)
cudaError_t launch_mlp_infer(const void* X, const void* W1b, const void* W2b, const float* P, float* Z1, void* H1b,
                             float* Z2, float* H2, float* Y, unsigned* err, cudaStream_t s, int rows = 128);
cudaError_t launch_learned_b(const ImgDesc* imgs, int n, int step, cudaStream_t s);
int mlp_infer_kernels();
cudaError_t mlp_prepare(const float* P, void* W1b, void* W2b, cudaStream_t s);
long long mlp_num_params();
cudaError_t launch_learned_prep(CycleState* st, const float* R, int H, int W, void* Xrow, cudaStream_t s);
cudaError_t launch_learned_apply(CycleState* st, const float* y, int g_pair, cudaStream_t s);
cudaError_t launch_learned_pick(CycleState* st, cudaStream_t s);
cudaError_t launch_harvest(const CycleState* st, const float* R, int H, int W, float* patches, float* targets,
                           int capacity, cudaStream_t s);
cudaError_t launch_beam_init(FitDesc* desc, const float* B, int H, int W, int g_max, cudaStream_t s);
cudaError_t launch_beam_ell_desc(FitDesc* d, double a, double x, double y, double w, cudaStream_t s);
cudaError_t launch_joint_flux(const FitOut* fo, int K, int C, const double* wb, double* out, cudaStream_t s);
cudaError_t launch_deconvolve_ell(const asp_gauss_ell* beam_then_in, int n, asp_component_ell* out, cudaStream_t s);
cudaError_t launch_radix_median(const float* v, long long n, int absdev, double center, unsigned long long* ws,
                                double* out, cudaStream_t s);

}  // namespace aspd
