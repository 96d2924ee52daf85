// Asp-Clean2004's objective (Sect. 2, Eq. 3), the system the paper
// accelerates: chi^2 = || T - B * sum_k g_k ||^2 over the whole image, g_k
// the unconvolved component a exp(-r^2 / 2 omega^2) sampled at the pixel
// centres and B the full PSF, so every evaluation is an FFT convolution of
// the image (Sect. 2: N (3 log2 N + 1) per convolution).  Kernels of one
// evaluation:
//   k_images_2004   the model image and its 4K derivative images (FP32,
//                   integer-centre frames) into the image corner of
//                   zero-padded 2H x 2W buffers;
//   (cuFFT R2C, batched) -> k_fft_mul_batch with the PSF's transform ->
//   (cuFFT C2R, batched);
//   k_ne_2004       the upper triangle of [J | r]^T [J | r] over the image
//                   pixels, r = T - (B * model): per-block FP32 leaves with
//                   Kahan across chunks, written as (sum, -compensation)
//                   pairs;
//   k_ne_reduce     each entry summed over the blocks in FP64, fixed order.
// The LM iterations themselves run on the host (asp_fit_2004 in
// asp_api.cu): a trial needs only the model's convolution, an accepted
// point the 4K Jacobian convolutions as well.
#include <cufft.h>

#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {

namespace {
constexpr int NE_CH = 64;          // pixels per staged chunk of k_ne_2004
constexpr int NE_THREADS = 256;
}  // namespace

// imgs: n_img buffers of 2H x 2W floats (stride img_stride), image region
// rows 0..H-1, columns 0..W-1.  n_img = 1: the model only; 4K + 1: the model
// then d/da, d/dx, d/dy, d/domega of each member.
__global__ void k_images_2004(const double* __restrict__ theta, int K, int H, int W, float* __restrict__ imgs,
                              long long img_stride, int n_img) {
    __shared__ float fa[FIT2004_KMAX], fc[FIT2004_KMAX], fiw2[FIT2004_KMAX], fiw3[FIT2004_KMAX], ffx[FIT2004_KMAX],
        ffy[FIT2004_KMAX];
    __shared__ int icx[FIT2004_KMAX], icy[FIT2004_KMAX];
    if (threadIdx.x < K) {
        const int k = threadIdx.x;
        const double a = theta[4 * k], x = theta[4 * k + 1], y = theta[4 * k + 2], w = theta[4 * k + 3];
        const double cx = floor(x + 0.5), cy = floor(y + 0.5), iw = 1.0 / w, iw2 = iw * iw;
        fa[k] = (float)a;
        fc[k] = (float)(0.5 * LOG2E * iw2);
        fiw2[k] = (float)iw2;
        fiw3[k] = (float)(iw2 * iw);
        ffx[k] = (float)(x - cx);
        ffy[k] = (float)(y - cy);
        icx[k] = (int)cx;
        icy[k] = (int)cy;
    }
    __syncthreads();
    const long long N = (long long)H * W;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i % W);
        const long long o = (long long)y * (2 * W) + x;
        float model = 0.f;
        for (int k = 0; k < K; ++k) {
            const float dx = (float)(x - icx[k]) - ffx[k], dy = (float)(y - icy[k]) - ffy[k];
            const float r2 = dx * dx + dy * dy;
            const float e = exp2f(-r2 * fc[k]);
            const float g = fa[k] * e;
            model += g;
            if (n_img > 1) {
                imgs[(1 + 4 * k) * img_stride + o] = e;
                imgs[(2 + 4 * k) * img_stride + o] = g * dx * fiw2[k];
                imgs[(3 + 4 * k) * img_stride + o] = g * dy * fiw2[k];
                imgs[(4 + 4 * k) * img_stride + o] = g * r2 * fiw3[k];
            }
        }
        imgs[o] = model;
    }
}

__global__ void k_fft_mul_batch(cufftComplex* __restrict__ a, const cufftComplex* __restrict__ b, long long nc,
                                int batch) {
    const long long n = nc * batch;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const cufftComplex u = a[i], v = b[i % nc];
        a[i] = make_cuComplex(u.x * v.x - u.y * v.y, u.x * v.y + u.y * v.x);
    }
}

// T = R + sc * conv0 (the members' previous contributions added back through
// B); conv0 is the inverse transform of the model's product (pixel p at p +
// (H, W) of the 2H x 2W grid).
__global__ void k_target_2004(const float* __restrict__ R, const float* __restrict__ conv, int H, int W, float sc,
                              float* __restrict__ T) {
    const long long N = (long long)H * W;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i % W);
        T[i] = R[i] + sc * conv[(long long)(y + H) * (2 * W) + x + W];
    }
}

// Upper triangle of [J | r]^T [J | r] (NA = n_img columns: J_0..J_{P-1}, r
// last; n_img = 1: chi^2 only) over the image pixels.  Entry e of the packed
// upper triangle (row-major) is handled by threads e, e + 256, ...; the
// chunk's rows are staged in shared memory.
__global__ void __launch_bounds__(NE_THREADS) k_ne_2004(const float* __restrict__ conv, long long img_stride,
                                                       const float* __restrict__ T, int H, int W, float sc, int n_img,
                                                       float2* __restrict__ partials) {
    extern __shared__ float rows[];                 // NE_CH x NA
    __shared__ short ei[FIT2004_NACC], ej[FIT2004_NACC];
    const int NA = n_img;                           // J columns 0..NA-2, r at NA-1 (model is conv image 0)
    const int nacc = NA * (NA + 1) / 2;
    for (int e = threadIdx.x; e < nacc; e += blockDim.x) {
        int i = 0, rem = e;
        while (rem >= NA - i) { rem -= NA - i; ++i; }
        ei[e] = (short)i;
        ej[e] = (short)(i + rem);
    }
    constexpr int EPT = (FIT2004_NACC + NE_THREADS - 1) / NE_THREADS;
    float s[EPT], c[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) { s[q] = 0.f; c[q] = 0.f; }
    __syncthreads();
    const long long N = (long long)H * W;
    for (long long p0 = (long long)blockIdx.x * NE_CH; p0 < N; p0 += (long long)gridDim.x * NE_CH) {
        const int cn = (int)min((long long)NE_CH, N - p0);
        for (int t = threadIdx.x; t < NE_CH * NA; t += blockDim.x) {
            const int l = t / NA, col = t % NA;
            float v = 0.f;
            if (l < cn) {
                const long long p = p0 + l;
                const int y = (int)(p / W), x = (int)(p % W);
                const long long o = (long long)(y + H) * (2 * W) + x + W;
                if (col == NA - 1) v = T[p] - sc * conv[o];               // residual: model is image 0
                else v = sc * conv[(1 + col) * img_stride + o];           // Jacobian column col
            }
            rows[l * NA + col] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int e = threadIdx.x + q * NE_THREADS;
            if (e < nacc) {
                const int i = ei[e], j = ej[e];
                float acc = 0.f;
                for (int l = 0; l < cn; ++l) acc = fmaf(rows[l * NA + i], rows[l * NA + j], acc);
                const float yv = acc - c[q];
                const float tv = s[q] + yv;
                c[q] = (tv - s[q]) - yv;
                s[q] = tv;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const int e = threadIdx.x + q * NE_THREADS;
        if (e < nacc) partials[(size_t)blockIdx.x * FIT2004_NACC + e] = make_float2(s[q], -c[q]);
    }
}

__global__ void k_ne_reduce(const float2* __restrict__ partials, int nblocks, int nacc, double* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nacc; e += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            const float2 v = partials[(size_t)b * FIT2004_NACC + e];
            acc += (double)v.x + (double)v.y;
        }
        out[e] = acc;
    }
}

// One evaluation: images at theta, their PSF convolutions, and (unless
// target_only) the normal equations into sums (packed upper triangle of
// [J | r]^T [J | r], or chi^2 alone for n_img = 1).  target_only: T = R +
// conv of the model (the added-back members) instead of the sums.
cudaError_t eval_2004(const Fit2004Buffers& fb, const double* theta_dev, int K, int n_img, int H, int W,
                      const float* R, bool target_only, cudaStream_t s) {
    const long long stride = 4LL * H * W;
    const long long nc = (long long)(2 * H) * (W + 1);
    const int grid = fb.grid;
    k_images_2004<<<grid, 256, 0, s>>>(theta_dev, K, H, W, fb.imgs, stride, n_img);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cufftHandle r2c = n_img == 1 ? fb.r2c1 : fb.r2cN, c2r = n_img == 1 ? fb.c2r1 : fb.c2rN;
    if (cufftSetStream(r2c, s) != CUFFT_SUCCESS || cufftSetStream(c2r, s) != CUFFT_SUCCESS) return cudaErrorUnknown;
    if (cufftExecR2C(r2c, fb.imgs, fb.work) != CUFFT_SUCCESS) return cudaErrorUnknown;
    k_fft_mul_batch<<<grid, 256, 0, s>>>(fb.work, fb.bhat, nc, n_img);
    if (cufftExecC2R(c2r, fb.work, fb.conv) != CUFFT_SUCCESS) return cudaErrorUnknown;
    const float sc = 1.0f / (4.0f * (float)H * (float)W);
    if (target_only) {
        k_target_2004<<<grid, 256, 0, s>>>(R, fb.conv, H, W, sc, fb.T);
        return cudaGetLastError();
    }
    const int NA = n_img;   // [J | r]: n_img - 1 Jacobian columns and r
    const size_t smem = sizeof(float) * NE_CH * NA;
    k_ne_2004<<<fb.ne_blocks, NE_THREADS, smem, s>>>(fb.conv, stride, fb.T, H, W, sc, n_img, fb.partials);
    k_ne_reduce<<<8, 256, 0, s>>>(fb.partials, fb.ne_blocks, NA * (NA + 1) / 2, fb.sums);
    return cudaGetLastError();
}

cudaError_t psf_transform_2004(const Fit2004Buffers& fb, const float* B, int H, int W, cudaStream_t s) {
    // the PSF through the single forward plan, staged in the first image
    // buffer (which the next evaluation rewrites; its padding is zeroed back)
    cudaError_t e = cudaMemcpyAsync(fb.imgs, B, sizeof(float) * 4 * (size_t)H * W, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    if (cufftSetStream(fb.r2c1, s) != CUFFT_SUCCESS) return cudaErrorUnknown;
    if (cufftExecR2C(fb.r2c1, fb.imgs, fb.bhat) != CUFFT_SUCCESS) return cudaErrorUnknown;
    return cudaMemsetAsync(fb.imgs, 0, sizeof(float) * 4 * (size_t)H * W, s);
}

}  // namespace aspd
