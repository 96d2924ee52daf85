// The LM fit kernel (asp_fit_body.cuh) for the elliptical members (model 1:
// a, x, y and the precision matrix A, B, C) and the joint wide-band members
// (model 2: x, y, s shared by the channels, an amplitude per channel), in a
// translation unit of their own so that the build compiles them beside the
// circular model's instantiations.
#include "asp_fit_body.cuh"

namespace aspd {

namespace {

template <int MODEL>
const void* model_kernel_ptr(int variant) {
    return variant == 1 ? (const void*)k_lm_fit<1, false, MODEL>
                        : variant == 3 ? (const void*)k_lm_fit<3, false, MODEL> : (const void*)k_lm_fit<3, true, MODEL>;
}

template <int MODEL>
cudaError_t launch_model(cudaLaunchConfig_t& cfg, int tpt, const float* src, int src_w, const FitDesc* desc,
                         const LMConst& lmc, FitOut* out, double* partials, double* sums, unsigned* bar, float* Tg) {
    if (tpt == 1)
        return cudaLaunchKernelEx(&cfg, k_lm_fit<1, false, MODEL>, src, src_w, desc, lmc, out, partials, sums, bar, Tg);
    if (tpt == 3)
        return cudaLaunchKernelEx(&cfg, k_lm_fit<3, false, MODEL>, src, src_w, desc, lmc, out, partials, sums, bar, Tg);
    return cudaLaunchKernelEx(&cfg, k_lm_fit<3, true, MODEL>, src, src_w, desc, lmc, out, partials, sums, bar, Tg);
}

}  // namespace

cudaError_t fit_configure_model(int model, int variant, int* blocks_per_sm) {
    if (model != 1 && model != 2) return cudaErrorInvalidValue;
    const void* k = model == 1 ? model_kernel_ptr<1>(variant) : model_kernel_ptr<2>(variant);
    const int smem = (int)fit_smem_bytes(variant);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, FIT_THREADS, smem);
}

cudaError_t launch_lm_fit_model(int model, int tpt, int grid, const float* src, int src_w, const FitDesc* desc,
                                const LMConst& lmc, FitOut* out, double* partials, double* sums, unsigned* bar,
                                float* Tg, cudaStream_t s) {
    if (model != 1 && model != 2) return cudaErrorInvalidValue;
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
    return model == 1 ? launch_model<1>(cfg, tpt, src, src_w, desc, lmc, out, partials, sums, bar, Tg)
                      : launch_model<2>(cfg, tpt, src, src_w, desc, lmc, out, partials, sums, bar, Tg);
}

}  // namespace aspd
