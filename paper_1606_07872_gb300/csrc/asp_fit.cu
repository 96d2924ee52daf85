// Launch code of the LM fit kernel (asp_fit_body.cuh): the circular model
// of the minor cycle, its pair and batched forms, shared-memory sizes and
// the variant choice.
#include "asp_fit_body.cuh"

namespace aspd {

// Fit variants: 1 = one tile per thread (K <= 7), 3 = three tiles per
// thread (K <= 32), 4 = the large variant (three tiles per thread in rounds,
// A read from L2; K <= KMAX).
size_t fit_smem_bytes(int variant) {
    if (variant == 4) return (size_t)PX_SMEM * sizeof(float) + (size_t)UNI_L_FLOATS * sizeof(float);
    return (size_t)PX_SMEM * sizeof(float) + (size_t)NACC_S * (sizeof(double) + sizeof(float)) +
           (size_t)JC_FLOATS * sizeof(float);
}
size_t fit_smem_bytes() { return fit_smem_bytes(1); }

static const void* fit_kernel_ptr(int variant) {
    return variant == 1 ? (const void*)k_lm_fit<1, false, 0>
                        : variant == 3 ? (const void*)k_lm_fit<3, false, 0> : (const void*)k_lm_fit<3, true, 0>;
}
static const void* fit_kernel_b_ptr(int variant) {
    return variant == 1 ? (const void*)k_lm_fit_b<1, false>
                        : variant == 3 ? (const void*)k_lm_fit_b<3, false> : (const void*)k_lm_fit_b<3, true>;
}

int fit_tpt_for(int k_max) {
    if (fit_tiles(k_max) <= FIT_THREADS) return 1;
    return k_max <= KMAX_S ? 3 : 4;
}

static const void* fit_kernel_pair_ptr(int variant) {
    return variant == 1 ? (const void*)k_lm_fit_pair<1, false>
                        : variant == 3 ? (const void*)k_lm_fit_pair<3, false> : (const void*)k_lm_fit_pair<3, true>;
}

cudaError_t fit_configure(int variant, int* blocks_per_sm) {
    const int smem = (int)fit_smem_bytes(variant);
    cudaError_t e = cudaFuncSetAttribute(fit_kernel_ptr(variant), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fit_kernel_b_ptr(variant), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fit_kernel_pair_ptr(variant), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fit_kernel_ptr(variant), FIT_THREADS, smem);
}

cudaError_t launch_lm_fit_batched(int tpt, const ImgDesc* imgs, const int* dmap, int n, int g_total, unsigned* bars,
                                  cudaStream_t s, int which, int max_iter_override) {
    cudaError_t e = cudaMemsetAsync(bars, 0, sizeof(unsigned) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g_total);
    cfg.blockDim = dim3(FIT_THREADS);
    cfg.dynamicSmemBytes = fit_smem_bytes(tpt);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (tpt == 1) return cudaLaunchKernelEx(&cfg, k_lm_fit_b<1, false>, imgs, dmap, n, which, max_iter_override);
    if (tpt == 3) return cudaLaunchKernelEx(&cfg, k_lm_fit_b<3, false>, imgs, dmap, n, which, max_iter_override);
    return cudaLaunchKernelEx(&cfg, k_lm_fit_b<3, true>, imgs, dmap, n, which, max_iter_override);
}

cudaError_t launch_lm_fit_pair(int tpt, int grid, const float* src, int src_w, const LMConst& lmc, const FitDesc* dA,
                               FitOut* oA, double* pA, double* sA, unsigned* bA, float* tA, const FitDesc* dB,
                               FitOut* oB, double* pB, double* sB, unsigned* bB, float* tB, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bA, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(bB, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(FIT_THREADS);
    cfg.dynamicSmemBytes = fit_smem_bytes(tpt);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (tpt == 1)
        return cudaLaunchKernelEx(&cfg, k_lm_fit_pair<1, false>, src, src_w, lmc, dA, oA, pA, sA, bA, tA, dB, oB, pB,
                                  sB, bB, tB);
    if (tpt == 3)
        return cudaLaunchKernelEx(&cfg, k_lm_fit_pair<3, false>, src, src_w, lmc, dA, oA, pA, sA, bA, tA, dB, oB, pB,
                                  sB, bB, tB);
    return cudaLaunchKernelEx(&cfg, k_lm_fit_pair<3, true>, src, src_w, lmc, dA, oA, pA, sA, bA, tA, dB, oB, pB, sB,
                              bB, tB);
}

cudaError_t launch_lm_fit(int tpt, int grid, const float* src, int src_w, const FitDesc* desc, const LMConst& lmc,
                          FitOut* out, double* partials, double* sums, unsigned* bar, float* Tg,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(FIT_THREADS);
    cfg.dynamicSmemBytes = fit_smem_bytes(tpt);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (tpt == 1)
        return cudaLaunchKernelEx(&cfg, k_lm_fit<1, false, 0>, src, src_w, desc, lmc, out, partials, sums, bar, Tg);
    if (tpt == 3)
        return cudaLaunchKernelEx(&cfg, k_lm_fit<3, false, 0>, src, src_w, desc, lmc, out, partials, sums, bar, Tg);
    return cudaLaunchKernelEx(&cfg, k_lm_fit<3, true, 0>, src, src_w, desc, lmc, out, partials, sums, bar, Tg);
}

}  // namespace aspd
