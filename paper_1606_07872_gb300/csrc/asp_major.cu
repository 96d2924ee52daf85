// Minor and major cycles split in the manner of Clark CLEAN (the paper's
// Sect. 1 and Sect. 3 comparison: Clark subtracts with an approximate PSF in
// the minor cycle, Asp-Clean2016 uses its single-Gaussian approximation in
// the estimation step).  With asp_params.major_every = n > 0:
//   * minor cycle: the residual update of Sect. 2 step 3 is made with the
//     PSF approximated by its fitted Gaussian (alpha_b, omega_b): a
//     component of flux F and width omega subtracts its single-Gaussian-beam
//     image alpha_b omega_b^2 F / omega_ic^2 exp(-r^2 / 2 omega_ic^2),
//     omega_ic^2 = omega^2 + omega_b^2 (Eqs. 7-8 inverted), over the box
//     |q - centre|_inf <= ceil(5 omega_ic) + 1 -- local and cheap;
//   * major cycle, after every n minor iterations and at the end of each
//     asp_minor_cycle call: the residual is recomputed exactly, R = D - B *
//     M (Sect. 2 step 3 with the full PSF), M the model image of every
//     component sampled as in the per-iteration subtraction, the
//     convolution as an FFT product on the 2H x 2W grid with the PSF's
//     transform cached per context (cuFFT).
#include <cufft.h>

#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {

namespace {

constexpr int MT = 32;   // model-image tile side

__device__ __forceinline__ void gauss_beam_box(double cx, double cy, double w, double wb, int H, int W, int& x0,
                                               int& x1, int& y0, int& y1, double& wic2) {
    wic2 = w * w + wb * wb;
    const double h = ceil(5.0 * sqrt(wic2)) + 1.0;
    const double bx0 = fmax(ceil(cx - h), 0.0), bx1 = fmin(floor(cx + h), (double)(W - 1));
    const double by0 = fmax(ceil(cy - h), 0.0), by1 = fmin(floor(cy + h), (double)(H - 1));
    x0 = (int)bx0; x1 = (int)bx1; y0 = (int)by0; y1 = (int)by1;
}

}  // namespace

// Minor-cycle subtraction with the Gaussian beam: every pixel of the union
// box of the iteration's terms subtracts the sum of the terms' beam images
// (one thread per pixel, terms in their fixed order).  One block first
// computes the union box into shared memory.
__global__ void __launch_bounds__(256) k_sub_gauss(float* __restrict__ R, int H, int W, CycleState* st) {
    if (st->stopped) return;
    __shared__ int bx0, bx1, by0, by1, nt;
    __shared__ double sab, swb;
    if (threadIdx.x == 0) {
        nt = st->n_terms;
        sab = st->alpha_b;
        swb = st->omega_b;
        int a0 = W, a1 = -1, b0 = H, b1 = -1;
        for (int t = 0; t < nt; ++t) {
            const TermDesc& td = st->terms[t];
            int x0, x1, y0, y1;
            double wic2;
            gauss_beam_box(td.cx, td.cy, td.w, swb, H, W, x0, x1, y0, y1, wic2);
            if (x0 > x1 || y0 > y1) continue;
            a0 = min(a0, x0); a1 = max(a1, x1); b0 = min(b0, y0); b1 = max(b1, y1);
        }
        bx0 = a0; bx1 = a1; by0 = b0; by1 = b1;
    }
    __syncthreads();
    if (bx0 > bx1 || by0 > by1) return;
    const long long bw = bx1 - bx0 + 1, bh = by1 - by0 + 1;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < bw * bh;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = by0 + (int)(i / bw), x = bx0 + (int)(i % bw);
        float acc = 0.f;
        for (int t = 0; t < nt; ++t) {
            const TermDesc& td = st->terms[t];
            int x0, x1, y0, y1;
            double wic2;
            gauss_beam_box(td.cx, td.cy, td.w, swb, H, W, x0, x1, y0, y1, wic2);
            if (x < x0 || x > x1 || y < y0 || y > y1) continue;
            // centre as integer + fraction, so the offsets carry no cancellation
            const double fx = floor(td.cx), fy = floor(td.cy);
            const float dx = (float)(x - (long long)fx) - (float)(td.cx - fx);
            const float dy = (float)(y - (long long)fy) - (float)(td.cy - fy);
            const float amp = (float)(sab * swb * swb / wic2) * td.scale;
            acc = fmaf(amp, expf(-(dx * dx + dy * dy) * (float)(0.5 / wic2)), acc);
        }
        R[(long long)y * W + x] -= acc;
    }
}

// Axis normalisations of every extended component (the sampled Gaussian on
// |q - centre|_inf <= ceil(5 omega) + 1 has unit sum per axis, as in the
// per-iteration subtraction): one warp per component, FP32 samples.
__global__ void __launch_bounds__(256) k_comp_norms(const asp_component* __restrict__ comps, const CycleState* st,
                                                   float2* __restrict__ norms) {
    const int n = st->n_comp;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int c = warp; c < n; c += nw) {
        const asp_component cp = comps[c];
        float2 out = make_float2(1.f, 1.f);
        if (!(cp.is_point || cp.width < 0.5)) {
            const double h = ceil(5.0 * cp.width) + 1.0;
            const float iw = (float)(1.0 / (2.0 * cp.width * cp.width));
            float s[2];
            for (int axis = 0; axis < 2; ++axis) {
                const double ce = axis == 0 ? cp.x : cp.y;
                const long long u0 = (long long)ceil(ce - h), u1 = (long long)floor(ce + h);
                const double fc = floor(ce);
                const long long ic = (long long)fc;
                const float fr = (float)(ce - fc);
                float a = 0.f;
                for (long long q = u0 + lane; q <= u1; q += 32) {
                    const float d = (float)(q - ic) - fr;
                    a += expf(-d * d * iw);
                }
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                s[axis] = a;
            }
            out = make_float2(s[0], s[1]);
        }
        if (lane == 0) norms[c] = out;
    }
}

// Model image M (every component sampled as in the subtraction: extended
// ones as unit-sum sampled Gaussians of flux F over their box, the rest as
// bilinear deposits of F) written into the image corner of the zero-padded
// 2H x 2W FFT input.  One block per 32 x 32 tile: the components touching
// the tile are collected in index order (ballot compaction), then each
// thread sums them for its pixels -- a fixed order, no atomics.
__global__ void __launch_bounds__(256) k_model_image(const asp_component* __restrict__ comps,
                                                    const float2* __restrict__ norms, const CycleState* st, int H,
                                                    int W, float* __restrict__ pad) {
    __shared__ int list[1024];
    __shared__ int count;
    __shared__ int wcount[8];
    const int n = st->n_comp;
    const int ntx = (W + MT - 1) / MT, nty = (H + MT - 1) / MT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
        const int tx0 = (tile % ntx) * MT, ty0 = (tile / ntx) * MT;
        const int tx1 = min(tx0 + MT - 1, W - 1), ty1 = min(ty0 + MT - 1, H - 1);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int c0 = 0; c0 < n; c0 += 1024) {
            // collect up to 1024 components of this chunk that touch the tile
            if (threadIdx.x == 0) count = 0;
            __syncthreads();
            for (int r0 = 0; r0 < 1024 && c0 + r0 < n; r0 += blockDim.x) {
                const int c = c0 + r0 + threadIdx.x;
                bool hit = false;
                if (c < n && r0 + threadIdx.x < 1024) {
                    const asp_component cp = comps[c];
                    double lx, hx, ly, hy;
                    if (cp.is_point || cp.width < 0.5) {
                        lx = floor(cp.x); hx = lx + 1.0; ly = floor(cp.y); hy = ly + 1.0;
                    } else {
                        const double h = ceil(5.0 * cp.width) + 1.0;
                        lx = ceil(cp.x - h); hx = floor(cp.x + h); ly = ceil(cp.y - h); hy = floor(cp.y + h);
                    }
                    hit = cp.flux != 0.0 && !(hx < tx0 || lx > tx1 || hy < ty0 || ly > ty1);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (lane == 0) wcount[warp] = __popc(bal);
                __syncthreads();
                int off = 0;
                for (int w = 0; w < warp; ++w) off += wcount[w];
                if (hit) list[count + off + __popc(bal & ((1u << lane) - 1u))] = c;
                __syncthreads();
                if (threadIdx.x == 0) {
                    int tot = 0;
                    for (int w = 0; w < 8; ++w) tot += wcount[w];
                    count += tot;
                }
                __syncthreads();
            }
            const int nl = count;
            // each thread: 4 pixels of the tile (rows warp*4 .. +3, column lane)
            for (int k = 0; k < nl; ++k) {
                const int c = list[k];
                const asp_component cp = comps[c];
                const int x = tx0 + lane;
                if (x > tx1) continue;
                if (cp.is_point || cp.width < 0.5) {
                    const double fx0 = floor(cp.x), fy0 = floor(cp.y);
                    const double fx = cp.x - fx0, fy = cp.y - fy0;
                    double wxv = 0.0;
                    if (x == (long long)fx0) wxv = 1.0 - fx;
                    else if (x == (long long)fx0 + 1) wxv = fx;
                    if (wxv == 0.0) continue;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int y = ty0 + warp * 4 + r;
                        double wyv = 0.0;
                        if (y == (long long)fy0) wyv = 1.0 - fy;
                        else if (y == (long long)fy0 + 1) wyv = fy;
                        acc[r] += (float)(cp.flux * wxv * wyv);
                    }
                } else {
                    const double h = ceil(5.0 * cp.width) + 1.0;
                    const float iw = (float)(1.0 / (2.0 * cp.width * cp.width));
                    const double fcx = floor(cp.x), fcy = floor(cp.y);
                    if (x < ceil(cp.x - h) || x > floor(cp.x + h)) continue;
                    const float dx = (float)(x - (long long)fcx) - (float)(cp.x - fcx);
                    const float2 nm = norms[c];
                    const float ax = (float)cp.flux * expf(-dx * dx * iw) / (nm.x * nm.y);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int y = ty0 + warp * 4 + r;
                        if (y < ceil(cp.y - h) || y > floor(cp.y + h)) continue;
                        const float dy = (float)(y - (long long)fcy) - (float)(cp.y - fcy);
                        acc[r] = fmaf(ax, expf(-dy * dy * iw), acc[r]);
                    }
                }
            }
            __syncthreads();
        }
        const int x = tx0 + lane;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int y = ty0 + warp * 4 + r;
            if (x <= tx1 && y <= ty1) pad[(long long)y * (2 * W) + x] = acc[r];
        }
    }
}

// Pointwise product with the PSF's transform (the FFT convolution's middle).
__global__ void k_fft_mul(cufftComplex* __restrict__ a, const cufftComplex* __restrict__ b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const cufftComplex u = a[i], v = b[i];
        a[i] = make_cuComplex(u.x * v.x - u.y * v.y, u.x * v.y + u.y * v.x);
    }
}

// Whether this major cycle applies: only if a minor iteration ran since the
// last one.  Decided once, before the other major-cycle kernels read it.
__global__ void k_major_gate(CycleState* st) {
    if (threadIdx.x != 0) return;
    st->major_skip = st->since_major == 0;
    st->since_major = 0;
    if (!st->major_skip) st->major_cycles += 1;
}

// R = D - (B * M)(p + (H, W)) / (4 H W): the inverse transform is
// unnormalised; the zero lag of B sits at [H, W], so the output pixel p of
// the circular 2H x 2W convolution is p + (H, W) (no wrap-around: p - q + H
// stays in [1, 2H - 1] for image pixels p, q).
__global__ void k_major_residual(float* __restrict__ R, const float* __restrict__ D, const float* __restrict__ conv,
                                 int H, int W, const CycleState* st) {
    if (st->major_skip) return;
    const float sc = 1.0f / (4.0f * (float)H * (float)W);
    const long long N = (long long)H * W;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i % W);
        R[i] = D[i] - conv[(long long)(y + H) * (2 * W) + x + W] * sc;
    }
}

// ------------------------------------------------------------------ FFT residual update
// The per-iteration update of Sect. 2 step 3, R -= B * dC with the full PSF,
// as one FFT convolution of the change image dC (sub_mode FFT) instead of
// the direct separable passes: dC is the same sum of the same terms, each
// extended term scale_t wx_t(x) wy_t(y) with the axis weights
// k_build_weights samples, each point-like term its bilinear deposits, so
// both forms compute one definition and differ only in rounding.
//
// k_delta_image writes dC into the image corner of the zero-padded 2H x 2W
// FFT input.  dC is zero outside the terms' boxes, so only the 32 x 32
// tiles meeting the union of this update's box and the previous update's
// box are written (the previous terms' samples are overwritten, by zeros
// where nothing of the new update lies).  Per tile the terms meeting it are
// listed in index order (ballot compaction); each thread sums them for 4
// pixels of one column, then adds the deposits in their order.
__global__ void __launch_bounds__(256) k_delta_image(CycleState* st, const int* gate, const float* __restrict__ wbuf,
                                                    int H, int W, float* __restrict__ pad) {
    if (gate && *gate) return;
    __shared__ int tq[MAX_TERMS][4];     // qx0, nx, qy0, ny (nx = ny = 0 for point-like terms)
    __shared__ int tw[MAX_TERMS][2];     // woff_x, woff_y
    __shared__ float ts[MAX_TERMS];      // scale
    __shared__ Deposit sdep[MAX_DEPOSITS];
    __shared__ int list[MAX_TERMS];
    __shared__ int wcount[8];
    __shared__ int ub[4], count;
    const int nt = min(st->n_terms, MAX_TERMS), nd = min(st->n_dep, MAX_DEPOSITS);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < nt; t += blockDim.x) {
        const TermDesc& td = st->terms[t];
        const bool ext = !td.bilinear;
        tq[t][0] = td.qx0; tq[t][1] = ext ? td.nx : 0; tq[t][2] = td.qy0; tq[t][3] = ext ? td.ny : 0;
        tw[t][0] = td.woff_x; tw[t][1] = td.woff_y;
        ts[t] = td.scale;
    }
    for (int i = tid; i < nd; i += blockDim.x) sdep[i] = st->dep[i];
    __syncthreads();
    if (tid == 0) {
        int x0 = W, x1 = -1, y0 = H, y1 = -1;
        for (int t = 0; t < nt; ++t) {
            if (tq[t][1] <= 0 || tq[t][3] <= 0) continue;
            x0 = min(x0, tq[t][0]); x1 = max(x1, tq[t][0] + tq[t][1] - 1);
            y0 = min(y0, tq[t][2]); y1 = max(y1, tq[t][2] + tq[t][3] - 1);
        }
        for (int d = 0; d < nd; ++d) {
            x0 = min(x0, sdep[d].qx); x1 = max(x1, sdep[d].qx);
            y0 = min(y0, sdep[d].qy); y1 = max(y1, sdep[d].qy);
        }
        if (blockIdx.x == 0) {
            st->dbox_next[0] = x0; st->dbox_next[1] = x1; st->dbox_next[2] = y0; st->dbox_next[3] = y1;
        }
        const int p0 = st->dbox[0], p1 = st->dbox[1], q0 = st->dbox[2], q1 = st->dbox[3];
        if (p0 <= p1 && q0 <= q1) {
            x0 = min(x0, p0); x1 = max(x1, p1); y0 = min(y0, q0); y1 = max(y1, q1);
        }
        ub[0] = max(x0, 0); ub[1] = min(x1, W - 1); ub[2] = max(y0, 0); ub[3] = min(y1, H - 1);
    }
    __syncthreads();
    if (ub[0] > ub[1] || ub[2] > ub[3]) return;
    const int tx0 = ub[0] / MT, tx1 = ub[1] / MT, ty0 = ub[2] / MT, ty1 = ub[3] / MT;
    const int ntx = tx1 - tx0 + 1, ntiles = ntx * (ty1 - ty0 + 1);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int px0 = (tx0 + tile % ntx) * MT, py0 = (ty0 + tile / ntx) * MT;
        const int px1 = min(px0 + MT - 1, W - 1), py1 = min(py0 + MT - 1, H - 1);
        // the terms meeting the tile, in index order (nt <= MAX_TERMS <= 4 warps)
        bool hit = false;
        if (tid < nt)
            hit = tq[tid][1] > 0 && tq[tid][3] > 0 && tq[tid][0] <= px1 && tq[tid][0] + tq[tid][1] - 1 >= px0 &&
                  tq[tid][2] <= py1 && tq[tid][2] + tq[tid][3] - 1 >= py0;
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int w = 0; w < warp; ++w) off += wcount[w];
        if (hit) list[off + __popc(bal & ((1u << lane) - 1u))] = tid;
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wcount[w];
            count = tot;
        }
        __syncthreads();
        const int x = px0 + lane;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (x <= px1) {
            for (int k = 0; k < count; ++k) {
                const int t = list[k];
                const int qx0 = tq[t][0], nx = tq[t][1], qy0 = tq[t][2], ny = tq[t][3];
                if (x < qx0 || x >= qx0 + nx) continue;
                // weights are stored reversed: tap i (pixel q0 + i) at n - 1 - i
                const float wx = ts[t] * __ldg(wbuf + tw[t][0] + (nx - 1 - (x - qx0)));
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int y = py0 + warp * 4 + r;
                    if (y >= qy0 && y < qy0 + ny) acc[r] = fmaf(wx, __ldg(wbuf + tw[t][1] + (ny - 1 - (y - qy0))), acc[r]);
                }
            }
            for (int d = 0; d < nd; ++d) {
                if (sdep[d].qx != x) continue;
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (sdep[d].qy == py0 + warp * 4 + r) acc[r] += sdep[d].w;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int y = py0 + warp * 4 + r;
                if (y <= py1) pad[(long long)y * (2 * W) + x] = acc[r];
            }
        }
        __syncthreads();   // list and count are rebuilt for the next tile
    }
}

cudaError_t launch_sub_gauss(float* R, int H, int W, CycleState* st, int grid, cudaStream_t s) {
    k_sub_gauss<<<grid, 256, 0, s>>>(R, H, W, st);
    return cudaGetLastError();
}

// The major cycle's launches: gate, component norms, model image into the
// padded FFT input, forward transform, product with the PSF's transform,
// inverse transform, residual.  The argmax of the new residual follows
// (gated on the same flag) in the caller.
cudaError_t launch_major(const asp_component* comps, float2* norms, CycleState* st, int H, int W, float* pad_in,
                         cufftComplex* work, const cufftComplex* bhat, float* conv_out, float* R, const float* D,
                         cufftHandle r2c, cufftHandle c2r, int grid, cudaStream_t s) {
    k_major_gate<<<1, 32, 0, s>>>(st);
    k_comp_norms<<<grid, 256, 0, s>>>(comps, st, norms);
    k_model_image<<<grid, 256, 0, s>>>(comps, norms, st, H, W, pad_in);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (cufftSetStream(r2c, s) != CUFFT_SUCCESS || cufftSetStream(c2r, s) != CUFFT_SUCCESS) return cudaErrorUnknown;
    if (cufftExecR2C(r2c, pad_in, work) != CUFFT_SUCCESS) return cudaErrorUnknown;
    k_fft_mul<<<grid, 256, 0, s>>>(work, bhat, (long long)(2 * H) * (W + 1));
    if (cufftExecC2R(c2r, work, conv_out) != CUFFT_SUCCESS) return cudaErrorUnknown;
    k_major_residual<<<grid, 256, 0, s>>>(R, D, conv_out, H, W, st);
    return cudaGetLastError();
}

// FFT residual update: dC into the padded input, forward transform, product
// with the PSF's transform, inverse transform, then R -= conv / (4 H W)
// with the next argmax (k_fft_sub_argmax, asp_image.cu).  The transforms
// run whether or not the gate is set (a stopped cycle transforms a stale
// dC and discards it).
cudaError_t launch_sub_fft(CycleState* st, const int* gate, const float* wbuf, int H, int W, float* pad_in,
                           cufftComplex* work, const cufftComplex* bhat, float* conv_out, float* R, cufftHandle r2c,
                           cufftHandle c2r, int grid, ArgRes* part, unsigned* ticket, cudaStream_t s) {
    // grid = 4 blocks per SM: the change image (often a few tiles) with one
    // block per SM, so few blocks stage the terms for nothing; the residual
    // pass with two per SM, several float4 per thread and fewer argmax
    // partials for the last block to reduce
    const int g_sm = grid >= 4 ? grid / 4 : 1, g_sub = grid >= 2 ? grid / 2 : 1;
    k_delta_image<<<g_sm, 256, 0, s>>>(st, gate, wbuf, H, W, pad_in);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (cufftSetStream(r2c, s) != CUFFT_SUCCESS || cufftSetStream(c2r, s) != CUFFT_SUCCESS) return cudaErrorUnknown;
    if (cufftExecR2C(r2c, pad_in, work) != CUFFT_SUCCESS) return cudaErrorUnknown;
    k_fft_mul<<<grid, 256, 0, s>>>(work, bhat, (long long)(2 * H) * (W + 1));
    if (cufftExecC2R(c2r, work, conv_out) != CUFFT_SUCCESS) return cudaErrorUnknown;
    return launch_fft_sub_argmax(R, conv_out, H, W, st, gate, g_sub, part, ticket, s);
}

// The PSF's transform: B (2H x 2W) through the forward plan into bhat, with
// pad_in as staging (zeroed again afterwards for the model images).
cudaError_t compute_psf_transform(const float* B, int H, int W, float* pad_in, cufftComplex* bhat, cufftHandle r2c,
                                  cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(pad_in, B, sizeof(float) * 4 * (size_t)H * W, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    if (cufftSetStream(r2c, s) != CUFFT_SUCCESS) return cudaErrorUnknown;
    if (cufftExecR2C(r2c, pad_in, bhat) != CUFFT_SUCCESS) return cudaErrorUnknown;
    return cudaMemsetAsync(pad_in, 0, sizeof(float) * 4 * (size_t)H * W, s);
}

}  // namespace aspd
