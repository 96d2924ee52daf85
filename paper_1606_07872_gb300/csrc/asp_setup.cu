// Set-up kernels run once per context:
//  * the initial guess and fit region of the single-Gaussian beam (Sect. 3:
//    the PSF approximated as one Gaussian (alpha_b, omega_b)): half-maximum
//    crossings along the four axes from the zero lag give omega_init; the fit
//    uses the pixels within radius ceil(3 omega_init);
//  * the noise level for the stopping rule (Sect. 2 step 4) when none is
//    given: 1.4826 x median absolute deviation, each median by an exact
//    8-pass radix select on FP64 order-preserving keys.
#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {

namespace {

__device__ __forceinline__ unsigned long long order_key(double d) {
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

__device__ __forceinline__ double key_value(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k;
    return __longlong_as_double((long long)b);
}

struct RadixWs {                      // laid out after the 256 histogram bins
    unsigned long long prefix, mask, k, pad;
};

}  // namespace

__global__ void k_beam_init(FitDesc* d, const float* __restrict__ B, int H, int W, int g_max) {
    if (threadIdx.x != 0) return;
    const int W2 = 2 * W;
    const double peak = B[(long long)H * W2 + W];
    const double half = 0.5 * peak;
    const int lim = H < W ? H : W;
    const int dirs[4][2] = {{0, 1}, {0, -1}, {1, 0}, {-1, 0}};
    double sum = 0.0;
    for (int q = 0; q < 4; ++q) {
        double prev = peak, rad = (double)(lim - 1);
        for (int s = 1; s < lim; ++s) {
            const double v = B[(long long)(H + dirs[q][0] * s) * W2 + (W + dirs[q][1] * s)];
            if (v < half) { rad = (s - 1) + (prev - half) / (prev - v); break; }
            prev = v;
        }
        sum += rad;
    }
    const double w0 = (sum / 4.0) / sqrt(2.0 * log(2.0));
    const int r = (int)ceil(3.0 * w0);
    const int x0 = max(0, W - r), x1 = min(W2 - 1, W + r);
    const int y0 = max(0, H - r), y1 = min(2 * H - 1, H + r);
    d->K = 1;
    d->n_old = 0;
    d->has_start = 0;
    d->model = 0;
    d->wx0 = x0; d->wy0 = y0; d->ww = x1 - x0 + 1; d->wh = y1 - y0 + 1;
    d->use_mask = 1;
    d->mcx = W; d->mcy = H; d->mr2 = (double)r * r;
    d->omega_min = 0.25 * w0;
    d->omega_max = (double)(2 * r + 1);
    d->bx0 = W - r; d->bx1 = W + r; d->by0 = H - r; d->by1 = H + r;
    d->theta0[0] = peak; d->theta0[1] = W; d->theta0[2] = H; d->theta0[3] = w0;
    int smem_ok = 1;
    d->grid = fit_grid((long long)d->ww * d->wh, 1, 0, g_max, &smem_ok);
    d->smem_ok = smem_ok;
    d->active = 1;
}

// The elliptical beam's fit: the circular beam's region and bounds, the
// elliptical model started from the circular beam (A = C = 1 / omega_b^2,
// B = 0).
__global__ void k_beam_ell_desc(FitDesc* d, double a, double x, double y, double w) {
    if (threadIdx.x != 0) return;
    d->model = 1;
    d->theta0[0] = a; d->theta0[1] = x; d->theta0[2] = y;
    d->theta0[3] = 1.0 / (w * w); d->theta0[4] = 0.0; d->theta0[5] = 1.0 / (w * w);
}

cudaError_t launch_beam_ell_desc(FitDesc* d, double a, double x, double y, double w, cudaStream_t s) {
    k_beam_ell_desc<<<1, 32, 0, s>>>(d, a, x, y, w);
    return cudaGetLastError();
}

__global__ void k_radix_reset(unsigned long long* ws, long long rank) {
    RadixWs* r = reinterpret_cast<RadixWs*>(ws + 256);
    if (threadIdx.x < 256) ws[threadIdx.x] = 0;
    if (threadIdx.x == 0) { r->prefix = 0; r->mask = 0; r->k = (unsigned long long)rank; }
}

__global__ void __launch_bounds__(256)
k_radix_hist(const float* __restrict__ v, long long n, int absdev, double center, int shift, unsigned long long* ws) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const RadixWs* r = reinterpret_cast<const RadixWs*>(ws + 256);
    const unsigned long long prefix = r->prefix, mask = r->mask;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double x = (double)v[i];
        if (absdev) x = fabs(x - center);
        const unsigned long long key = order_key(x);
        if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&ws[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

__global__ void k_radix_step(unsigned long long* ws, int shift) {
    if (threadIdx.x != 0) return;
    RadixWs* r = reinterpret_cast<RadixWs*>(ws + 256);
    unsigned long long k = r->k, cum = 0;
    int b = 255;
    for (int i = 0; i < 256; ++i) {
        if (cum + ws[i] > k) { b = i; break; }
        cum += ws[i];
    }
    r->k = k - cum;
    r->prefix |= (unsigned long long)b << shift;
    r->mask |= 255ULL << shift;
    for (int i = 0; i < 256; ++i) ws[i] = 0;
}

__global__ void k_radix_store(unsigned long long* ws, double* out, int slot) {
    if (threadIdx.x != 0) return;
    const RadixWs* r = reinterpret_cast<const RadixWs*>(ws + 256);
    out[slot] = key_value(r->prefix);
}

__global__ void k_radix_finish(double* out, int even) {
    if (threadIdx.x != 0) return;
    out[0] = even ? 0.5 * (out[1] + out[2]) : out[1];
}

cudaError_t launch_beam_init(FitDesc* desc, const float* B, int H, int W, int g_max, cudaStream_t s) {
    k_beam_init<<<1, 32, 0, s>>>(desc, B, H, W, g_max);
    return cudaGetLastError();
}

// Median of v (or of |v - center| when absdev) written to out[0]; ws holds
// 256 bins + 4 words; out needs 3 doubles.
cudaError_t launch_radix_median(const float* v, long long n, int absdev, double center, unsigned long long* ws,
                                double* out, cudaStream_t s) {
    const bool even = (n % 2) == 0;
    const long long ranks[2] = {even ? n / 2 - 1 : n / 2, n / 2};
    for (int q = 0; q < (even ? 2 : 1); ++q) {
        k_radix_reset<<<1, 256, 0, s>>>(ws, ranks[q]);
        for (int pass = 0; pass < 8; ++pass) {
            const int shift = 56 - 8 * pass;
            k_radix_hist<<<256, 256, 0, s>>>(v, n, absdev, center, shift, ws);
            k_radix_step<<<1, 32, 0, s>>>(ws, shift);
        }
        k_radix_store<<<1, 32, 0, s>>>(ws, out, 1 + q);
    }
    k_radix_finish<<<1, 32, 0, s>>>(out, even ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace aspd
