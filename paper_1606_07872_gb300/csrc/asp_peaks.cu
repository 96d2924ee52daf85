// Issue-rate microbenchmarks of the two pipes the LM pixel pass runs on:
// FP32 fused multiply-add (the model, Jacobian and the [J | r]^T [J | r]
// accumulation) and the MUFU ex2 unit (one exponential per member and pixel).
// They give the measured denominators of the pass's ALU roofline.
//
// Each kernel runs one full wave (every SM at full occupancy) of threads that
// each advance 8 independent dependency chains, long enough (~10^8 issues
// per SM) that launch overhead is negligible; CUDA events time the launch and
// clock64 deltas of every CTA give the SM clock the work ran at.
#include <cstring>

#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {
namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void record_cycles(unsigned long long c0, unsigned long long* cyc) {
    const unsigned long long dc = clock64() - c0;
    if (threadIdx.x == 0) atomicMax(cyc, dc);
}

// 8 chains x 8 unrolled FMAs per loop trip; x -> x * a + b stays bounded for
// |a| < 1.  The sum is stored only if it equals a value it cannot reach, so
// the chains are live but nothing is written.
__global__ void __launch_bounds__(PK_THREADS) k_peak_fma(int trips, float a, float b, float* sink,
                                                          unsigned long long* cyc) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    const unsigned long long c0 = clock64();
#pragma unroll 1
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    record_cycles(c0, cyc);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

// The same with Blackwell's packed two-lane FP32 FMA (fma.rn.f32x2 on a
// 64-bit register pair): 2 FMAs per instruction.
__global__ void __launch_bounds__(PK_THREADS) k_peak_fma2(int trips, float a, float b, float* sink,
                                                           unsigned long long* cyc) {
    unsigned long long x[PK_CHAINS / 2];
    unsigned long long av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < PK_CHAINS / 2; ++c) {
        const float lo = (float)(threadIdx.x + 2 * c) * 1e-3f, hi = (float)(threadIdx.x + 2 * c + 1) * 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    const unsigned long long c0 = clock64();
#pragma unroll 1
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < PK_CHAINS / 2; ++c)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
    record_cycles(c0, cyc);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS / 2; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

// 8 chains of x -> ex2(-x) (values stay in (0, 1]): MUFU issue rate.
__global__ void __launch_bounds__(PK_THREADS) k_peak_ex2(int trips, float* sink, unsigned long long* cyc) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    const unsigned long long c0 = clock64();
#pragma unroll 1
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = ex2_approx(-x[c]);
    }
    record_cycles(c0, cyc);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace aspd

using namespace aspd;

extern "C" asp_status asp_measure_alu_peaks(asp_alu_peaks* out) {
    if (!out) return ASP_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ASP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ASP_ERR_CUDA;
    int bps_fma = 0, bps_fma2 = 0, bps_ex2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_fma, k_peak_fma, PK_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_fma2, k_peak_fma2, PK_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_ex2, k_peak_ex2, PK_THREADS, 0) != cudaSuccess)
        return ASP_ERR_CUDA;
    if (bps_fma < 1 || bps_fma2 < 1 || bps_ex2 < 1) return ASP_ERR_CUDA;
    float* sink = nullptr;
    unsigned long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    asp_status st = ASP_OK;
    if (cudaMalloc(&sink, sizeof(float) * (size_t)sms * 64) != cudaSuccess) return ASP_ERR_OOM;
    if (cudaMalloc(&cyc, sizeof(unsigned long long)) != cudaSuccess) { cudaFree(sink); return ASP_ERR_OOM; }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // kind 0: FP32 FMA, 1: packed FP32 FMA, 2: ex2; ops per thread and trip
    const int trips[3] = {1 << 15, 1 << 14, 1 << 13};
    const double ops_per_trip[3] = {64.0, 64.0, 32.0};
    const int bps[3] = {bps_fma, bps_fma2, bps_ex2};
    double rate[3] = {0, 0, 0}, mhz[3] = {0, 0, 0};
    for (int kind = 0; kind < 3 && st == ASP_OK; ++kind) {
        const int grid = sms * bps[kind];
        for (int rep = 0; rep < 3 && st == ASP_OK; ++rep) {       // first launch warms up
            cudaMemset(cyc, 0, sizeof(unsigned long long));
            cudaEventRecord(e0);
            if (kind == 0) k_peak_fma<<<grid, PK_THREADS>>>(trips[0], 0.999f, 1e-3f, sink, cyc);
            if (kind == 1) k_peak_fma2<<<grid, PK_THREADS>>>(trips[1], 0.999f, 1e-3f, sink, cyc);
            if (kind == 2) k_peak_ex2<<<grid, PK_THREADS>>>(trips[2], sink, cyc);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = ASP_ERR_CUDA; break; }
            float ms = 0.f;
            unsigned long long c = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
            const double ops = (double)grid * PK_THREADS * trips[kind] * ops_per_trip[kind];
            const double r = ops / (ms * 1e-3);
            if (rep > 0 && r > rate[kind]) {
                rate[kind] = r;
                mhz[kind] = (double)c / (ms * 1e-3) / 1e6;
            }
        }
    }
    if (cudaGetLastError() != cudaSuccess && st == ASP_OK) st = ASP_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(cyc);
    if (st != ASP_OK) return st;
    out->sms = sms;
    out->fp32_fma_tflops = 2.0 * rate[0] / 1e12;
    out->fp32_fma2_tflops = 2.0 * rate[1] / 1e12;
    out->ex2_gops = rate[2] / 1e9;
    out->sm_mhz_fma = mhz[0];
    out->sm_mhz_fma2 = mhz[1];
    out->sm_mhz_ex2 = mhz[2];
    out->fma_per_sm_clk = rate[0] / (sms * mhz[0] * 1e6);
    out->fma2_per_sm_clk = rate[1] / (sms * mhz[1] * 1e6);
    out->ex2_per_sm_clk = rate[2] / (sms * mhz[2] * 1e6);
    return ASP_OK;
}
