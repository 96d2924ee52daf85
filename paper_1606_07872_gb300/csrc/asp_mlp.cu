// Learned initial values: the 1024-256-256-4 GELU network that proposes a
// new component's starting point from the residual patch at the plain
// method's peak, trained and run on the GPU.  The two wide layers (and their
// gradients) are BF16 products on the 5th-generation tensor cores:
// tcgen05.mma with both operands in shared memory (canonical K-major layout,
// no swizzle) and the FP32 accumulator tile in tensor memory, read back with
// tcgen05.ld.  The 256 -> 4 output layer, GELU, the loss and Adam run on the
// CUDA cores in FP32.
//
// Every wait is bounded: the kernel that issues the MMAs waits on an
// mbarrier for at most MBAR_SPIN rounds, then records an error, gives the
// tensor core a second bounded wait, frees its tensor memory and returns.
#include <cstdint>
#include <cstring>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {

namespace {

constexpr int GM_THREADS = 128;          // one warpgroup: warp w owns TMEM lanes 32w .. 32w+31
constexpr int GM_TM = 128;               // M of one MMA / one CTA tile
constexpr int GM_TN = 256;               // N of one MMA / one CTA tile (TMEM columns)
constexpr int GM_KC = 64;                // K staged per round (4 MMAs of K = 16)
constexpr int GM_A_BYTES = GM_TM * GM_KC * 2;            // 16 KB
constexpr int GM_B_BYTES = GM_TN * GM_KC * 2;            // 32 KB
constexpr int GM_SMEM = 100 * 1024;      // > 2 x the stage: at most 2 CTAs (512 TMEM columns) per SM
constexpr long long MBAR_SPIN = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between core matrices adjacent along K), stride byte offset
// (between 8-row core-matrix groups along M or N), descriptor version 1,
// no swizzle.  Offsets are encoded in 16-byte units.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t mma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(phase)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t phase) {
    for (long long it = 0; it < MBAR_SPIN; ++it)
        if (mbar_try_wait(addr, phase)) return true;
    return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) of a 128- or 256-row operand stage in the
// canonical K-major layout without swizzle: per K step of 16 (kk) a block of
// rows/8 core-matrix groups; a group holds two 8x16-byte core matrices (the
// two K halves, LBO = 128 bytes apart); groups are SBO = 256 bytes apart.
__device__ __forceinline__ int stage_off(int row, int ku, int rows) {
    // ku: 16-byte unit along K within the 64-wide stage (0..7)
    return (ku >> 1) * (rows * 32) + (row >> 3) * 256 + (ku & 1) * 128 + (row & 7) * 16;
}

}  // namespace

// C[M x N] (FP32, row-major, ldc) = A[M x K] (BF16, row-major, lda) x
// B[N x K]^T (BF16, row-major, ldb).  Grid (N / 256, M / 128), 128 threads.
// M % 128 == 0, N % 256 == 0, K % 64 == 0, lda and ldb multiples of 8.
__global__ void __launch_bounds__(GM_THREADS, 1)
k_gemm_bf16_tc(const __nv_bfloat16* __restrict__ A, int lda, const __nv_bfloat16* __restrict__ B, int ldb,
               float* __restrict__ C, int ldc, int K, unsigned* err) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    unsigned char* sA = gsm;
    unsigned char* sB = gsm + GM_A_BYTES;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * GM_TM, n0 = blockIdx.x * GM_TN;
    const uint32_t mbar_a = smem_u32(&mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(GM_TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mbar_a, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = mma_idesc_bf16(GM_TM, GM_TN);
    uint32_t phase = 0;

    for (int k0 = 0; k0 < K; k0 += GM_KC) {
        // stage A rows m0.., B rows n0.., columns k0 .. k0+63: 16-byte units
        for (int u = tid; u < GM_TM * 8; u += GM_THREADS) {
            const int r = u >> 3, ku = u & 7;
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * lda + k0 + ku * 8));
            *reinterpret_cast<uint4*>(sA + stage_off(r, ku, GM_TM)) = v;
        }
        for (int u = tid; u < GM_TN * 8; u += GM_THREADS) {
            const int r = u >> 3, ku = u & 7;
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(B + (size_t)(n0 + r) * ldb + k0 + ku * 8));
            *reinterpret_cast<uint4*>(sB + stage_off(r, ku, GM_TN)) = v;
        }
        // generic-proxy stores must be visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < GM_KC / 16; ++kk) {
                const uint64_t ad = smem_desc(smem_u32(sA) + kk * (GM_TM * 32), 128, 256);
                const uint64_t bd = smem_desc(smem_u32(sB) + kk * (GM_TN * 32), 128, 256);
                mma_bf16(tmem, ad, bd, idesc, (k0 > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(mbar_a);
        }
        // the MMAs read the stage: wait for them before it is overwritten
        const bool ok = mbar_wait_bounded(mbar_a, phase);
        phase ^= 1u;
        if (!ok) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        const int row = m0 + 32 * warp + lane;
        float* crow = C + (size_t)row * ldc + n0;
#pragma unroll 1
        for (int c = 0; c < GM_TN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int q = 0; q < 16; q += 4)
                *reinterpret_cast<float4*>(crow + c + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        }
    } else if (tid == 0) {
        atomicExch(err, 1u);
        // give MMAs still in flight a second bounded wait before freeing their accumulator
        mbar_wait_bounded(mbar_a, phase ^ 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GM_TN) : "memory");
    }
}

cudaError_t gemm_bf16_configure() {
    return cudaFuncSetAttribute(k_gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, GM_SMEM);
}

cudaError_t launch_gemm_bf16(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M, int N, int K,
                             unsigned* err, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0 || M % GM_TM || N % GM_TN || K % GM_KC || lda % 8 || ldb % 8 || ldc % 4 ||
        lda < K || ldb < K || ldc < N)
        return cudaErrorInvalidValue;
    k_gemm_bf16_tc<<<dim3(N / GM_TN, M / GM_TM), GM_THREADS, GM_SMEM, s>>>(
        reinterpret_cast<const __nv_bfloat16*>(A), lda, reinterpret_cast<const __nv_bfloat16*>(B), ldb, C, ldc, K, err);
    return cudaGetLastError();
}

}  // namespace aspd

using namespace aspd;

extern "C" asp_status asp_mlp_gemm(const void* A_dev, int lda, const void* B_dev, int ldb, float* C_dev, int ldc,
                                   int M, int N, int K, void* stream) {
    if (!A_dev || !B_dev || !C_dev) return ASP_ERR_INVALID_ARG;
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 256 || K % 64 || lda % 8 || ldb % 8 || ldc % 4 || lda < K ||
        ldb < K || ldc < N)
        return ASP_ERR_INVALID_ARG;
    static unsigned* err = nullptr;
    if (!err) {
        if (cudaMalloc(&err, sizeof(unsigned)) != cudaSuccess) return ASP_ERR_OOM;
        if (gemm_bf16_configure() != cudaSuccess) return ASP_ERR_CUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) return ASP_ERR_CUDA;
    if (launch_gemm_bf16(A_dev, lda, B_dev, ldb, C_dev, ldc, M, N, K, err, s) != cudaSuccess) return ASP_ERR_CUDA;
    unsigned h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ASP_ERR_CUDA;
    return h ? ASP_ERR_TIMEOUT : ASP_OK;
}

// =====================================================================
// Training and batched inference of the network.
namespace aspd {
namespace {

constexpr int NI = 1024, NH = 256, NO = 4;

int ew_grid(long long n) { return (int)(n + 255) / 256 < 4096 ? (int)((n + 255) / 256) : 4096; }
constexpr size_t OFF_W1 = 0, OFF_B1 = OFF_W1 + (size_t)NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + (size_t)NH * NH,
                 OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + (size_t)NO * NH, N_PARAMS = OFF_B3 + NO;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// rows r < bn: X[idx[r]] (and its target); rows bn .. B-1: zeros.  Writes the
// batch row-major and transposed (BF16) for the two products that read it.
__global__ void k_gather_batch(const __nv_bfloat16* __restrict__ Xall, const float* __restrict__ Tall,
                               const int* __restrict__ idx, int bn, int B, __nv_bfloat16* __restrict__ Xb,
                               __nv_bfloat16* __restrict__ XbT, float* __restrict__ Tb) {
    const long long total = (long long)B * NI;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(q / NI), c = (int)(q % NI);
        const __nv_bfloat16 v = r < bn ? Xall[(size_t)idx[r] * NI + c] : __float2bfloat16(0.f);
        Xb[q] = v;
        XbT[(size_t)c * B + r] = v;
        if (c < NO) Tb[r * NO + c] = r < bn ? Tall[(size_t)idx[r] * NO + c] : 0.f;
    }
}

// z += b (kept for the backward pass); h = GELU(z) into any of: BF16
// row-major, BF16 transposed (ld B), FP32 row-major.
__global__ void k_bias_gelu(float* __restrict__ Z, const float* __restrict__ b, int B, __nv_bfloat16* __restrict__ Hb,
                            __nv_bfloat16* __restrict__ HbT, float* __restrict__ Hf) {
    const long long total = (long long)B * NH;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(q / NH), c = (int)(q % NH);
        const float z = Z[q] + b[c];
        Z[q] = z;
        const float h = gelu_f(z);
        if (Hb) Hb[q] = __float2bfloat16(h);
        if (HbT) HbT[(size_t)c * B + r] = __float2bfloat16(h);
        if (Hf) Hf[q] = h;
    }
}

// Output layer (FP32): Y[r] = W3 h2[r] + b3, one warp per row.
__global__ void k_out_fwd(const float* __restrict__ H2, const float* __restrict__ W3, const float* __restrict__ b3, int B,
                          float* __restrict__ Y) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    float acc[NO] = {0.f, 0.f, 0.f, 0.f};
    for (int j = lane; j < NH; j += 32) {
        const float h = H2[(size_t)warp * NH + j];
#pragma unroll
        for (int o = 0; o < NO; ++o) acc[o] = fmaf(W3[o * NH + j], h, acc[o]);
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        float v = acc[o];
        for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
        if (lane == 0) Y[warp * NO + o] = v + b3[o];
    }
}

// Mean squared error over the bn real rows and dL/dY (zero on padding rows);
// one block, loss written to *loss.
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ T, int bn, int B, float* __restrict__ dY,
                            float* __restrict__ loss) {
    __shared__ float red[256];
    const float scale = 2.0f / (float)(bn * NO);
    float s = 0.f;
    for (int q = threadIdx.x; q < B * NO; q += blockDim.x) {
        float d = 0.f;
        if (q < bn * NO) {
            d = Y[q] - T[q];
            s = fmaf(d, d, s);
        }
        dY[q] = scale * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (float)(bn * NO);
}

// Output-layer backward: gW3 = dY^T H2, gb3 = column sums of dY (thread per
// weight, rows in order); dH2 = dY W3 (thread per element).
__global__ void k_out_bwd(const float* __restrict__ dY, const float* __restrict__ H2, const float* __restrict__ W3, int B,
                          float* __restrict__ gW3, float* __restrict__ gb3, float* __restrict__ dH2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < NO * NH) {
        const int o = t / NH, j = t % NH;
        float s = 0.f;
        for (int r = 0; r < B; ++r) s = fmaf(dY[r * NO + o], H2[(size_t)r * NH + j], s);
        gW3[t] = s;
    }
    if (t < NO) {
        float s = 0.f;
        for (int r = 0; r < B; ++r) s += dY[r * NO + t];
        gb3[t] = s;
    }
    const long long total = (long long)B * NH;
    for (long long q = t; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(q / NH), j = (int)(q % NH);
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < NO; ++o) s = fmaf(dY[r * NO + o], W3[o * NH + j], s);
        dH2[q] = s;
    }
}

// dz = dh GELU'(z) into FP32 (for the bias sums) and BF16 row-major and/or
// transposed (ld B) for the products.
__global__ void k_gelu_bwd(const float* __restrict__ dH, const float* __restrict__ Z, int B, float* __restrict__ dZ,
                           __nv_bfloat16* __restrict__ dZb, __nv_bfloat16* __restrict__ dZbT) {
    const long long total = (long long)B * NH;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(q / NH), c = (int)(q % NH);
        const float d = dH[q] * gelu_grad_f(Z[q]);
        dZ[q] = d;
        if (dZb) dZb[q] = __float2bfloat16(d);
        if (dZbT) dZbT[(size_t)c * B + r] = __float2bfloat16(d);
    }
}

// Column sums (bias gradients), rows in order.
__global__ void k_colsum(const float* __restrict__ D, int B, int ncol, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    float s = 0.f;
    for (int r = 0; r < B; ++r) s += D[(size_t)r * ncol + c];
    out[c] = s;
}

// Adam on the FP32 masters (bias-corrected), then the BF16 copies the
// products read: W1, W2 and W2 transposed.
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ Mm, float* __restrict__ Vv,
                       long long n, float lr, float beta1, float beta2, float eps, float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = beta1 * Mm[i] + (1.f - beta1) * g;
        const float v = beta2 * Vv[i] + (1.f - beta2) * g * g;
        Mm[i] = m;
        Vv[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

__global__ void k_refresh_bf16(const float* __restrict__ P, __nv_bfloat16* __restrict__ W1b, __nv_bfloat16* __restrict__ W2b,
                               __nv_bfloat16* __restrict__ W2Tb) {
    const long long n1 = (long long)NH * NI, n2 = (long long)NH * NH;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2; i += (long long)gridDim.x * blockDim.x) {
        if (i < n1) {
            W1b[i] = __float2bfloat16(P[OFF_W1 + i]);
        } else {
            const long long q = i - n1;
            const int r = (int)(q / NH), c = (int)(q % NH);
            const __nv_bfloat16 v = __float2bfloat16(P[OFF_W2 + q]);
            W2b[q] = v;
            W2Tb[(size_t)c * NH + r] = v;
        }
    }
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16(src[i]);
}

}  // namespace
}  // namespace aspd

namespace aspd {

// In-cycle inference for up to 128 patches (rows of X, BF16; unused rows
// zero): two tensor-core products and the FP32 output layer, Y (128 x 4).
cudaError_t launch_mlp_infer(const void* X, const void* W1b, const void* W2b, const float* P, float* Z1, void* H1b,
                             float* Z2, float* H2, float* Y, unsigned* err, cudaStream_t s, int rows) {
    if (rows < 128 || rows % 128) return cudaErrorInvalidValue;
    cudaError_t e = launch_gemm_bf16(X, NI, W1b, NI, Z1, NH, rows, NH, NI, err, s);
    if (e != cudaSuccess) return e;
    k_bias_gelu<<<ew_grid((long long)rows * NH), 256, 0, s>>>(Z1, P + OFF_B1, rows,
                                                              reinterpret_cast<__nv_bfloat16*>(H1b), nullptr, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_gemm_bf16(H1b, NH, W2b, NH, Z2, NH, rows, NH, NH, err, s)) != cudaSuccess) return e;
    k_bias_gelu<<<ew_grid((long long)rows * NH), 256, 0, s>>>(Z2, P + OFF_B2, rows, nullptr, nullptr, H2);
    k_out_fwd<<<(rows * 32 + 255) / 256, 256, 0, s>>>(H2, P + OFF_W3, P + OFF_B3, rows, Y);
    return cudaGetLastError();
}
int mlp_infer_kernels() { return 5; }

// BF16 copies of W1 and W2 from the FP32 parameter vector P (device).
cudaError_t mlp_prepare(const float* P, void* W1b, void* W2b, cudaStream_t s) {
    cudaError_t e = gemm_bf16_configure();
    if (e != cudaSuccess) return e;
    k_to_bf16<<<ew_grid((long long)NH * NI), 256, 0, s>>>(P + OFF_W1, reinterpret_cast<__nv_bfloat16*>(W1b),
                                                            (long long)NH * NI);
    k_to_bf16<<<ew_grid((long long)NH * NH), 256, 0, s>>>(P + OFF_W2, reinterpret_cast<__nv_bfloat16*>(W2b),
                                                            (long long)NH * NH);
    return cudaGetLastError();
}
long long mlp_num_params() { return (long long)N_PARAMS; }

}  // namespace aspd

struct asp_mlp {
    int B = 0;                    // batch capacity (multiple of 128)
    cudaStream_t stream = nullptr;
    float *P = nullptr, *G = nullptr, *Mm = nullptr, *Vv = nullptr;   // masters, gradients, Adam moments
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2Tb = nullptr;
    __nv_bfloat16* Xall = nullptr;
    float* Tall = nullptr;
    long long n_data = 0;
    int* idx = nullptr;
    __nv_bfloat16 *Xb = nullptr, *XbT = nullptr, *H1b = nullptr, *H1Tb = nullptr, *dZ2b = nullptr, *dZ2Tb = nullptr,
                  *dZ1Tb = nullptr;
    float *Tb = nullptr, *Z1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *dH2 = nullptr,
          *dH1 = nullptr, *dZ = nullptr, *loss = nullptr;
    unsigned* err = nullptr;
    int t = 0;                    // Adam steps taken
    std::vector<void*> allocs;
};

namespace {

template <class T>
cudaError_t malloc_m(asp_mlp* m, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) return e;
    m->allocs.push_back(q);
    *p = reinterpret_cast<T*>(q);
    return cudaSuccess;
}


// forward (and backward) of the batch already gathered into m->Xb/XbT/Tb
asp_status mlp_pass(asp_mlp* m, int bn, bool backward) {
    using namespace aspd;
    const int B = ((bn + 127) / 128) * 128;
    cudaStream_t s = m->stream;
#define MC(call) do { if ((call) != cudaSuccess) return ASP_ERR_CUDA; } while (0)
    MC(launch_gemm_bf16(m->Xb, NI, m->W1b, NI, m->Z1, NH, B, NH, NI, m->err, s));
    k_bias_gelu<<<ew_grid((long long)B * NH), 256, 0, s>>>(m->Z1, m->P + OFF_B1, B, m->H1b, m->H1Tb, nullptr);
    MC(cudaGetLastError());
    MC(launch_gemm_bf16(m->H1b, NH, m->W2b, NH, m->Z2, NH, B, NH, NH, m->err, s));
    k_bias_gelu<<<ew_grid((long long)B * NH), 256, 0, s>>>(m->Z2, m->P + OFF_B2, B, nullptr, nullptr, m->H2);
    k_out_fwd<<<(B * 32 + 255) / 256, 256, 0, s>>>(m->H2, m->P + OFF_W3, m->P + OFF_B3, B, m->Y);
    MC(cudaGetLastError());
    if (!backward) return ASP_OK;
    k_loss_grad<<<1, 256, 0, s>>>(m->Y, m->Tb, bn, B, m->dY, m->loss);
    k_out_bwd<<<ew_grid((long long)B * NH), 256, 0, s>>>(m->dY, m->H2, m->P + OFF_W3, B, m->G + OFF_W3, m->G + OFF_B3,
                                                       m->dH2);
    k_gelu_bwd<<<ew_grid((long long)B * NH), 256, 0, s>>>(m->dH2, m->Z2, B, m->dZ, m->dZ2b, m->dZ2Tb);
    k_colsum<<<1, NH, 0, s>>>(m->dZ, B, NH, m->G + OFF_B2);
    MC(cudaGetLastError());
    MC(launch_gemm_bf16(m->dZ2Tb, B, m->H1Tb, B, m->G + OFF_W2, NH, NH, NH, B, m->err, s));   // gW2 = dz2^T h1
    MC(launch_gemm_bf16(m->dZ2b, NH, m->W2Tb, NH, m->dH1, NH, B, NH, NH, m->err, s));        // dh1 = dz2 W2
    k_gelu_bwd<<<ew_grid((long long)B * NH), 256, 0, s>>>(m->dH1, m->Z1, B, m->dZ, nullptr, m->dZ1Tb);
    k_colsum<<<1, NH, 0, s>>>(m->dZ, B, NH, m->G + OFF_B1);
    MC(cudaGetLastError());
    MC(launch_gemm_bf16(m->dZ1Tb, B, m->XbT, B, m->G + OFF_W1, NI, NH, NI, B, m->err, s));   // gW1 = dz1^T x
#undef MC
    return ASP_OK;
}

asp_status mlp_sync_check(asp_mlp* m) {
    unsigned h = 0;
    if (cudaMemcpyAsync(&h, m->err, sizeof(unsigned), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return ASP_ERR_CUDA;
    return h ? ASP_ERR_TIMEOUT : ASP_OK;
}

}  // namespace

extern "C" {

asp_status asp_mlp_destroy(asp_mlp* m) {
    if (!m) return ASP_ERR_INVALID_ARG;
    if (m->stream) cudaStreamSynchronize(m->stream);
    else cudaDeviceSynchronize();
    for (void* q : m->allocs) cudaFree(q);
    delete m;
    return ASP_OK;
}

asp_status asp_mlp_create(const float* params_host, int max_batch, void* stream, asp_mlp** out) {
    using namespace aspd;
    if (!out) return ASP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params_host || max_batch < 1 || max_batch > (1 << 16)) return ASP_ERR_INVALID_ARG;
    asp_mlp* m = new asp_mlp();
    m->B = ((max_batch + 127) / 128) * 128;
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    auto bail = [&](asp_status st) { asp_mlp_destroy(m); return st; };
    if (gemm_bf16_configure() != cudaSuccess) return bail(ASP_ERR_CUDA);
    const size_t B = m->B;
#define MA(p, n) if (malloc_m(m, &(p), (size_t)(n)) != cudaSuccess) return bail(ASP_ERR_OOM)
    MA(m->P, N_PARAMS); MA(m->G, N_PARAMS); MA(m->Mm, N_PARAMS); MA(m->Vv, N_PARAMS);
    MA(m->W1b, (size_t)NH * NI); MA(m->W2b, (size_t)NH * NH); MA(m->W2Tb, (size_t)NH * NH);
    MA(m->idx, B);
    MA(m->Xb, B * NI); MA(m->XbT, B * NI); MA(m->H1b, B * NH); MA(m->H1Tb, B * NH);
    MA(m->dZ2b, B * NH); MA(m->dZ2Tb, B * NH); MA(m->dZ1Tb, B * NH);
    MA(m->Tb, B * NO); MA(m->Z1, B * NH); MA(m->Z2, B * NH); MA(m->H2, B * NH); MA(m->Y, B * NO); MA(m->dY, B * NO);
    MA(m->dH2, B * NH); MA(m->dH1, B * NH); MA(m->dZ, B * NH); MA(m->loss, 1); MA(m->err, 1);
#undef MA
    if (cudaMemcpyAsync(m->P, params_host, N_PARAMS * sizeof(float), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->Mm, 0, N_PARAMS * sizeof(float), m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->Vv, 0, N_PARAMS * sizeof(float), m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->err, 0, sizeof(unsigned), m->stream) != cudaSuccess)
        return bail(ASP_ERR_CUDA);
    k_refresh_bf16<<<ew_grid((long long)NH * (NI + NH)), 256, 0, m->stream>>>(m->P, m->W1b, m->W2b, m->W2Tb);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess) return bail(ASP_ERR_CUDA);
    *out = m;
    return ASP_OK;
}

asp_status asp_mlp_num_params(long long* n) {
    if (!n) return ASP_ERR_INVALID_ARG;
    *n = (long long)aspd::N_PARAMS;
    return ASP_OK;
}

asp_status asp_mlp_set_data(asp_mlp* m, const float* X_host, const float* T_host, long long n) {
    using namespace aspd;
    if (!m || !X_host || !T_host || n < 1) return ASP_ERR_INVALID_ARG;
    if (n > m->n_data) {
        float* tmp = nullptr;
        if (malloc_m(m, &m->Xall, (size_t)n * NI) != cudaSuccess || malloc_m(m, &m->Tall, (size_t)n * NO) != cudaSuccess)
            return ASP_ERR_OOM;
        (void)tmp;
    }
    m->n_data = n;
    float* stage = nullptr;
    if (cudaMalloc(&stage, (size_t)n * NI * sizeof(float)) != cudaSuccess) return ASP_ERR_OOM;
    asp_status st = ASP_OK;
    if (cudaMemcpyAsync(stage, X_host, (size_t)n * NI * sizeof(float), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(m->Tall, T_host, (size_t)n * NO * sizeof(float), cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        st = ASP_ERR_CUDA;
    if (st == ASP_OK) {
        k_to_bf16<<<ew_grid(n * NI), 256, 0, m->stream>>>(stage, m->Xall, n * NI);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess) st = ASP_ERR_CUDA;
    }
    cudaFree(stage);
    return st;
}

// One forward/backward pass on rows idx[0 .. bn) of the data set; with
// update, one Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8).  loss_out
// and grads_out (N_PARAMS floats, parameter order W1 b1 W2 b2 W3 b3) are
// host pointers and may be NULL.
asp_status asp_mlp_step(asp_mlp* m, const int* idx_host, int bn, float lr, int update, float* loss_out,
                        float* grads_out) {
    using namespace aspd;
    if (!m || !idx_host || bn < 1 || bn > m->B || m->n_data < 1) return ASP_ERR_INVALID_ARG;
    for (int i = 0; i < bn; ++i)
        if (idx_host[i] < 0 || idx_host[i] >= m->n_data) return ASP_ERR_INVALID_ARG;
    const int B = ((bn + 127) / 128) * 128;
    if (cudaMemcpyAsync(m->idx, idx_host, bn * sizeof(int), cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        return ASP_ERR_CUDA;
    k_gather_batch<<<ew_grid((long long)B * NI), 256, 0, m->stream>>>(m->Xall, m->Tall, m->idx, bn, B, m->Xb, m->XbT,
                                                                       m->Tb);
    if (cudaGetLastError() != cudaSuccess) return ASP_ERR_CUDA;
    asp_status s = mlp_pass(m, bn, true);
    if (s != ASP_OK) return s;
    if (update) {
        m->t += 1;
        const float c1 = 1.f - powf(0.9f, (float)m->t), c2 = 1.f - powf(0.999f, (float)m->t);
        k_adam<<<ew_grid((long long)N_PARAMS), 256, 0, m->stream>>>(m->P, m->G, m->Mm, m->Vv, (long long)N_PARAMS, lr, 0.9f,
                                                                   0.999f, 1e-8f, c1, c2);
        k_refresh_bf16<<<ew_grid((long long)NH * (NI + NH)), 256, 0, m->stream>>>(m->P, m->W1b, m->W2b, m->W2Tb);
        if (cudaGetLastError() != cudaSuccess) return ASP_ERR_CUDA;
    }
    if (loss_out && cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return ASP_ERR_CUDA;
    if (grads_out &&
        cudaMemcpyAsync(grads_out, m->G, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return ASP_ERR_CUDA;
    return mlp_sync_check(m);
}

// Batched inference: Y (n x 4, host) for X (n x 1024, host), n <= capacity.
asp_status asp_mlp_predict(asp_mlp* m, const float* X_host, int n, float* Y_host) {
    using namespace aspd;
    if (!m || !X_host || !Y_host || n < 1 || n > m->B) return ASP_ERR_INVALID_ARG;
    const int B = ((n + 127) / 128) * 128;
    float* stage = nullptr;
    if (cudaMalloc(&stage, (size_t)B * NI * sizeof(float)) != cudaSuccess) return ASP_ERR_OOM;
    asp_status st = ASP_OK;
    if (cudaMemsetAsync(stage, 0, (size_t)B * NI * sizeof(float), m->stream) != cudaSuccess ||
        cudaMemcpyAsync(stage, X_host, (size_t)n * NI * sizeof(float), cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        st = ASP_ERR_CUDA;
    if (st == ASP_OK) {
        k_to_bf16<<<ew_grid((long long)B * NI), 256, 0, m->stream>>>(stage, m->Xb, (long long)B * NI);
        if (cudaGetLastError() != cudaSuccess) st = ASP_ERR_CUDA;
    }
    if (st == ASP_OK) st = mlp_pass(m, n, false);
    if (st == ASP_OK &&
        cudaMemcpyAsync(Y_host, m->Y, (size_t)n * NO * sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        st = ASP_ERR_CUDA;
    if (st == ASP_OK) st = mlp_sync_check(m);
    cudaFree(stage);
    return st;
}

asp_status asp_mlp_get_params(asp_mlp* m, float* params_host) {
    if (!m || !params_host) return ASP_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(params_host, m->P, aspd::N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, m->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return ASP_ERR_CUDA;
    return ASP_OK;
}

}  // extern "C"
