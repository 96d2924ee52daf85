// Levenberg-Marquardt fit of an active set of PSF-convolved Gaussians to the
// residual image: the Eq. 6 objective chi^2 = || I_res - sum_k g_k ||^2 with
// g_k = a_k exp(-((x-x_k)^2 + (y-y_k)^2) / (2 w_k^2)) (Sect. 3), minimised
// by Marquardt's damped Gauss-Newton method (Marquardt 1963, cited in Sect. 1).
//
// One persistent cooperative kernel runs the whole fit.  Each CTA owns a
// fixed slice of the window pixels and keeps its target values in shared
// memory for all iterations.  Per LM iteration:
//   1. pixel pass (FP32): per pixel the K Gaussians, the residual r and the
//      4K Jacobian entries, accumulated as the upper triangle of
//      [J | r]^T [J | r] (J^T J, J^T r and r^T r) in 4x4 register tiles,
//      leaf sums of <= 64 pixels, Kahan-compensated across leaves;
//   2. CTA partials (FP64) -> grid barrier -> column-split FP64 reduction ->
//      grid barrier;
//   3. every CTA redundantly runs the LM decision logic and the FP64
//      Cholesky solve of (A + lambda diag A) delta = g, so no third barrier
//      is needed to broadcast the next trial point.
// Grid barriers are bounded spins; on timeout the kernel records an error
// and returns.
#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {

namespace {

constexpr int CH_SMALL = 256;   // chunk pixels when NAp <= 64
constexpr int CH_LARGE = 128;   // chunk pixels otherwise
constexpr int JC_FLOATS = 128 * NAP_MAX;   // >= 256 * 64
constexpr int M_DOUBLES = PMAX * (PMAX + 1) / 2;

struct MemberFrame {
    float a, c, iw2, iw3, fx, fy;   // c = log2(e) / (2 w^2)
    int cx, cy;
};

__device__ __forceinline__ int pidx(int i, int j) { return i * (i + 1) / 2 + j; }   // packed lower, j <= i

__device__ __forceinline__ int tile_index(int bi, int bj, int nb) { return bi * nb - bi * (bi - 1) / 2 + (bj - bi); }

// Accumulator entry of (i, j) of [J | r]^T [J | r].
__device__ __forceinline__ int acc_index(int i, int j, int nb) {
    if (i > j) { int t = i; i = j; j = t; }
    return tile_index(i >> 2, j >> 2, nb) * 16 + (i & 3) * 4 + (j & 3);
}

__device__ void grid_barrier(unsigned* bar, unsigned target, int* s_err, int* g_err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        unsigned spins = 0;
        while (ld_acquire_u32(bar) < target) {
            if (++spins > SPIN_LIMIT) {
                *s_err = 1;
                atomicExch(g_err, ASP_ERR_TIMEOUT);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
}

// Frame of member k for the FP32 pass: integer centre plus fractional offset
// so dx = (px - cx) - fx is computed without cancellation.
__device__ __forceinline__ void make_frame(const double* th, MemberFrame& f) {
    double a = th[0], x = th[1], y = th[2], w = th[3];
    double cx = floor(x + 0.5), cy = floor(y + 0.5);
    f.a = (float)a;
    f.c = (float)(LOG2E / (2.0 * w * w));
    f.iw2 = (float)(1.0 / (w * w));
    f.iw3 = (float)(1.0 / (w * w * w));
    f.fx = (float)(x - cx);
    f.fy = (float)(y - cy);
    f.cx = (int)cx;
    f.cy = (int)cy;
}

// Cholesky factorisation of the packed lower matrix M (P x P) in place, all
// threads of the block.  Returns false if a pivot is not positive.
__device__ bool cholesky_packed(double* M, int P, double* inv_diag, int* s_flag) {
    const int tid = threadIdx.x;
    for (int j = 0; j < P; ++j) {
        if (tid == 0) {
            double d = M[pidx(j, j)];
            if (!(d > 0.0) || !isfinite(d)) {
                *s_flag = 1;
            } else {
                double l = sqrt(d);
                M[pidx(j, j)] = l;
                inv_diag[j] = 1.0 / l;
            }
        }
        __syncthreads();
        if (*s_flag) return false;
        const double il = inv_diag[j];
        for (int i = j + 1 + tid; i < P; i += blockDim.x) M[pidx(i, j)] *= il;
        __syncthreads();
        const int m = P - j - 1;
        const int total = m * (m + 1) / 2;
        for (int q = tid; q < total; q += blockDim.x) {
            int ii = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
            while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
            while (ii * (ii + 1) / 2 > q) --ii;
            int kk = q - ii * (ii + 1) / 2;
            int i = j + 1 + ii, k = j + 1 + kk;
            M[pidx(i, k)] -= M[pidx(i, j)] * M[pidx(k, j)];
        }
        __syncthreads();
    }
    return true;
}

// Solve L L^T x = b with warp 0 (b overwritten by x).
__device__ void chol_solve_warp(const double* M, int P, const double* inv_diag, double* b) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    for (int j = 0; j < P; ++j) {                 // L y = b
        double yj = b[j] * inv_diag[j];
        __syncwarp();
        if (lane == 0) b[j] = yj;
        for (int i = j + 1 + lane; i < P; i += 32) b[i] -= M[pidx(i, j)] * yj;
        __syncwarp();
    }
    for (int j = P - 1; j >= 0; --j) {            // L^T x = y
        double xj = b[j] * inv_diag[j];
        __syncwarp();
        if (lane == 0) b[j] = xj;
        for (int i = lane; i < j; i += 32) b[i] -= M[pidx(j, i)] * xj;
        __syncwarp();
    }
}

}  // namespace

template <int TPT>
__global__ void __launch_bounds__(FIT_THREADS, 1)
k_lm_fit(const float* __restrict__ src, int src_w, const FitDesc* __restrict__ descp, LMConst lmc,
         FitOut* __restrict__ out, double* __restrict__ partials, double* __restrict__ sums,
         unsigned* __restrict__ bar, float* __restrict__ Tg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Ts = reinterpret_cast<float*>(smem_raw);                          // PX_SMEM floats
    float* Jc = Ts + PX_SMEM;                                                // union region
    double* Mp = reinterpret_cast<double*>(Jc);
    float* red = Jc;

    __shared__ FitDesc d;
    __shared__ MemberFrame fr[KMAX];
    __shared__ short2 ttab[NTILES_MAX];
    __shared__ double theta[PMAX], trial[PMAX], delta[PMAX], gvec[PMAX], dvec[PMAX], inv_diag[PMAX];
    __shared__ double s_lam, s_chi2, s_chi2_init;
    __shared__ int s_cur, s_iters, s_passes, s_status, s_done, s_err, s_flag, s_go;

    const int tid = threadIdx.x;
    {
        const int* srcw = reinterpret_cast<const int*>(descp);
        int* dstw = reinterpret_cast<int*>(&d);
        for (int i = tid; i < (int)(sizeof(FitDesc) / sizeof(int)); i += blockDim.x) dstw[i] = srcw[i];
    }
    __syncthreads();
    if (!d.active) return;
    const int G = d.grid;
    const int b = blockIdx.x;
    if (b >= G) return;

    const int K = d.K, P = 4 * K, NA = P + 1, NAp = (NA + 3) & ~3, nb = NAp / 4;
    const int ntiles = nb * (nb + 1) / 2;
    const int nacc = ntiles * 16;
    const long long Wn = (long long)d.ww * d.wh;
    const long long s0 = Wn * b / G, s1 = Wn * (b + 1) / G;
    const int slen = (int)(s1 - s0);
    const bool in_smem = d.smem_ok != 0;
    const int CH = (NAp <= 64) ? CH_SMALL : CH_LARGE;
    const int chi_idx = acc_index(P, P, nb);

    // ---- tile table and thread -> (tile, group) assignment
    for (int t = tid; t < ntiles; t += blockDim.x) {
        int bi = 0, rem = t;
        while (rem >= nb - bi) { rem -= nb - bi; ++bi; }
        ttab[t] = make_short2((short)bi, (short)(bi + rem));
    }
    int n_groups, my_group, my_tile0;
    if (ntiles >= (int)blockDim.x) {
        n_groups = 1; my_group = 0; my_tile0 = tid;
    } else {
        n_groups = blockDim.x / ntiles;
        my_group = tid / ntiles;
        my_tile0 = tid % ntiles;
        if (my_group >= n_groups) my_group = -1;
    }

    // ---- stage the target T = src + sum of the added-back members
    if (tid < K) make_frame(&d.theta0[4 * tid], fr[tid]);
    __syncthreads();
    for (int i = tid; i < slen; i += blockDim.x) {
        long long gi = s0 + i;
        int y = d.wy0 + (int)(gi / d.ww), x = d.wx0 + (int)(gi % d.ww);
        float v = src[(long long)y * src_w + x];
        for (int m = K - d.n_old; m < K; ++m) {
            const MemberFrame& f = fr[m];
            float dx = (float)(x - f.cx) - f.fx, dy = (float)(y - f.cy) - f.fy;
            v += f.a * exp2f(-(dx * dx + dy * dy) * f.c);
        }
        if (in_smem) Ts[i] = v; else Tg[gi] = v;
    }
    if (tid == 0) {
        for (int i = 0; i < P; ++i) theta[i] = d.theta0[i];
        s_lam = lmc.lambda0; s_cur = 0; s_iters = 0; s_passes = 0; s_status = ASP_LM_CAP;
        s_done = 0; s_err = 0; s_flag = 0;
    }
    for (int i = tid; i < P; i += blockDim.x) trial[i] = d.theta0[i];
    __syncthreads();

    unsigned epoch = 0;
    bool first = true;
    while (true) {
        // ================= pixel pass at trial[] =================
        if (tid < K) make_frame(&trial[4 * tid], fr[tid]);
        __syncthreads();
        float acc[TPT][16], ks[TPT][16], kc[TPT][16];
#pragma unroll
        for (int q = 0; q < TPT; ++q)
#pragma unroll
            for (int e = 0; e < 16; ++e) { acc[q][e] = 0.f; ks[q][e] = 0.f; kc[q][e] = 0.f; }

        for (int c0 = 0; c0 < slen; c0 += CH) {
            const int cn = min(CH, slen - c0);
            // phase A: one pixel row of [J | r] per thread
            if (tid < CH) {
                float* row = Jc + tid * NAp;
                bool live = tid < cn;
                int x = 0, y = 0;
                if (live) {
                    long long gi = s0 + c0 + tid;
                    y = d.wy0 + (int)(gi / d.ww);
                    x = d.wx0 + (int)(gi % d.ww);
                    if (d.use_mask) {
                        double ddx = x - d.mcx, ddy = y - d.mcy;
                        live = ddx * ddx + ddy * ddy <= d.mr2;
                    }
                }
                if (live) {
                    float model = 0.f;
                    for (int k = 0; k < K; ++k) {
                        const MemberFrame& f = fr[k];
                        float dx = (float)(x - f.cx) - f.fx, dy = (float)(y - f.cy) - f.fy;
                        float r2 = dx * dx + dy * dy;
                        float e = exp2f(-r2 * f.c);
                        float g = f.a * e;
                        model += g;
                        float4 jr = make_float4(e, g * dx * f.iw2, g * dy * f.iw2, g * r2 * f.iw3);
                        *reinterpret_cast<float4*>(row + 4 * k) = jr;
                    }
                    float t = in_smem ? Ts[c0 + tid] : Tg[s0 + c0 + tid];
                    row[P] = t - model;
                    for (int c = P + 1; c < NAp; ++c) row[c] = 0.f;
                } else {
                    for (int c = 0; c < NAp; ++c) row[c] = 0.f;
                }
            }
            __syncthreads();
            // phase B: SYRK of the chunk into the register tiles
            if (my_group >= 0) {
                const int per = (cn + n_groups - 1) / n_groups;
                const int pa = my_group * per, pb = min(cn, pa + per);
                for (int l0 = pa; l0 < pb; l0 += 64) {
                    const int l1 = min(pb, l0 + 64);
#pragma unroll
                    for (int q = 0; q < TPT; ++q) {
                        const int t = my_tile0 + q * (int)blockDim.x;
                        if (t < ntiles) {
                            const short2 bij = ttab[t];
                            for (int l = l0; l < l1; ++l) {
                                const float4 av = *reinterpret_cast<const float4*>(Jc + l * NAp + 4 * bij.x);
                                const float4 bv = *reinterpret_cast<const float4*>(Jc + l * NAp + 4 * bij.y);
                                const float aa[4] = {av.x, av.y, av.z, av.w};
                                const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                                for (int i = 0; i < 4; ++i)
#pragma unroll
                                    for (int j = 0; j < 4; ++j) acc[q][i * 4 + j] = fmaf(aa[i], bb[j], acc[q][i * 4 + j]);
                            }
                            // Kahan flush of the leaf
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                float yv = acc[q][e] - kc[q][e];
                                float tv = ks[q][e] + yv;
                                kc[q][e] = (tv - ks[q][e]) - yv;
                                ks[q][e] = tv;
                                acc[q][e] = 0.f;
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }

        // ---- CTA total of each accumulator entry (FP64 across pixel groups)
        const int nxt = 1 - s_cur;
        double* sums_nxt = sums + (size_t)nxt * NACC_MAX;
        if (n_groups == 1) {
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                const int t = my_tile0 + q * (int)blockDim.x;
                if (my_group == 0 && t < ntiles) {
                    double* dst = (G == 1) ? (sums_nxt + t * 16) : (partials + (size_t)b * NACC_MAX + t * 16);
#pragma unroll
                    for (int e = 0; e < 16; ++e) dst[e] = (double)ks[q][e] - (double)kc[q][e];
                }
            }
        } else {
            if (my_group >= 0) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    red[(my_group * ntiles + my_tile0) * 16 + e] = ks[0][e];
                    red[(n_groups * ntiles + my_group * ntiles + my_tile0) * 16 + e] = kc[0][e];
                }
            }
            __syncthreads();
            for (int e = tid; e < nacc; e += blockDim.x) {
                double s = 0.0;
                for (int g = 0; g < n_groups; ++g)
                    s += (double)red[g * nacc + e] - (double)red[(n_groups + g) * nacc + e];
                if (G == 1) sums_nxt[e] = s; else partials[(size_t)b * NACC_MAX + e] = s;
            }
        }

        // ---- cross-CTA reduction (FP64, fixed order -> identical in every CTA)
        if (G > 1) {
            ++epoch;
            grid_barrier(bar, epoch * (unsigned)G, &s_err, &out->error);
            if (s_err) return;
            for (int e = b * (int)blockDim.x + tid; e < nacc; e += G * (int)blockDim.x) {
                double s = 0.0;
                for (int c = 0; c < G; ++c) s += __ldcg(partials + (size_t)c * NACC_MAX + e);
                sums_nxt[e] = s;
            }
            ++epoch;
            grid_barrier(bar, epoch * (unsigned)G, &s_err, &out->error);
            if (s_err) return;
        } else {
            __syncthreads();
        }

        // ================= LM decision (identical in every CTA) =================
        if (tid == 0) {
            s_passes += 1;
            const double chi2_t = __ldcg(sums_nxt + chi_idx);
            if (first) {
                s_cur = nxt;
                s_chi2 = chi2_t;
                s_chi2_init = chi2_t;
            } else if (chi2_t < s_chi2) {
                const double rel = s_chi2 > 0.0 ? (s_chi2 - chi2_t) / s_chi2 : 0.0;
                double mx = 0.0;
                for (int k = 0; k < K; ++k) {
                    double w = theta[4 * k + 3];
                    double sa = fabs(theta[4 * k]);
                    if (sa == 0.0) sa = 1.0;
                    mx = fmax(mx, fabs(delta[4 * k]) / sa);
                    mx = fmax(mx, fabs(delta[4 * k + 1]) / w);
                    mx = fmax(mx, fabs(delta[4 * k + 2]) / w);
                    mx = fmax(mx, fabs(delta[4 * k + 3]) / w);
                }
                for (int i = 0; i < P; ++i) theta[i] = trial[i];
                s_cur = nxt;
                s_chi2 = chi2_t;
                s_lam = fmax(s_lam / lmc.lambda_down, lmc.lambda_min);
                if (rel < lmc.rtol || mx < lmc.xtol) { s_status = ASP_LM_CONVERGED; s_done = 1; }
            } else {
                s_lam *= lmc.lambda_up;
                if (s_lam > lmc.lambda_max) { s_status = ASP_LM_STALLED; s_done = 1; }
            }
        }
        first = false;
        __syncthreads();

        // ---- propose the next trial point (solves without a pass loop here)
        const double* sc = sums + (size_t)s_cur * NACC_MAX;
        while (!s_done) {
            if (tid == 0 && s_iters >= lmc.max_iter) { s_status = ASP_LM_CAP; s_done = 1; }
            __syncthreads();
            if (s_done) break;
            // damped matrix (packed lower) and right-hand side
            for (int i = tid; i < P; i += blockDim.x) {
                double dd = __ldcg(sc + acc_index(i, i, nb));
                dvec[i] = dd > 0.0 ? dd : 1.0;
                gvec[i] = __ldcg(sc + acc_index(i, P, nb));
            }
            __syncthreads();
            const double lam = s_lam;
            for (int q = tid; q < P * (P + 1) / 2; q += blockDim.x) {
                int i = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
                while ((i + 1) * (i + 2) / 2 <= q) ++i;
                while (i * (i + 1) / 2 > q) --i;
                int j = q - i * (i + 1) / 2;
                double v = __ldcg(sc + acc_index(i, j, nb));
                if (i == j) v += lam * dvec[i];
                Mp[q] = v;
            }
            if (tid == 0) s_flag = 0;
            __syncthreads();
            const bool ok = cholesky_packed(Mp, P, inv_diag, &s_flag);
            if (ok) {
                for (int i = tid; i < P; i += blockDim.x) delta[i] = gvec[i];
                __syncthreads();
                chol_solve_warp(Mp, P, inv_diag, delta);
            }
            __syncthreads();
            if (tid == 0) {
                s_iters += 1;
                s_go = 0;
                bool fin = ok;
                for (int i = 0; ok && i < P; ++i) fin = fin && isfinite(delta[i]);
                if (!fin) {
                    s_lam *= lmc.lambda_up;
                    if (s_lam > lmc.lambda_max) { s_status = ASP_LM_STALLED; s_done = 1; }
                } else {
                    double dg = 0.0, dd2 = 0.0;
                    for (int i = 0; i < P; ++i) { dg += delta[i] * gvec[i]; dd2 += dvec[i] * delta[i] * delta[i]; }
                    const double pred = dg + lam * dd2;
                    if (pred <= lmc.rtol * s_chi2) {
                        s_status = ASP_LM_CONVERGED; s_done = 1;
                    } else {
                        bool valid = true;
                        for (int k = 0; k < K; ++k) {
                            double a = theta[4 * k] + delta[4 * k];
                            double x = theta[4 * k + 1] + delta[4 * k + 1];
                            double y = theta[4 * k + 2] + delta[4 * k + 2];
                            double w = theta[4 * k + 3] + delta[4 * k + 3];
                            trial[4 * k] = a; trial[4 * k + 1] = x; trial[4 * k + 2] = y; trial[4 * k + 3] = w;
                            if (!(w > d.omega_min) || w > d.omega_max || !isfinite(a) || !isfinite(x) ||
                                !isfinite(y) || !isfinite(w) ||
                                x < d.bx0 || x > d.bx1 || y < d.by0 || y > d.by1)
                                valid = false;
                        }
                        if (valid) {
                            s_go = 1;
                        } else {
                            s_lam *= lmc.lambda_up;
                            if (s_lam > lmc.lambda_max) { s_status = ASP_LM_STALLED; s_done = 1; }
                        }
                    }
                }
            }
            __syncthreads();
            if (s_go) break;
        }
        __syncthreads();
        if (s_done) break;
    }

    if (b == 0 && tid == 0) {
        for (int i = 0; i < P; ++i) out->theta[i] = theta[i];
        out->chi2_init = s_chi2_init;
        out->chi2 = s_chi2;
        out->lambda = s_lam;
        out->iters = s_iters;
        out->passes = s_passes;
        out->status = s_status;
        out->pixel_evals = (long long)s_passes * Wn;
    }
}

size_t fit_smem_bytes() {
    size_t jc = (size_t)JC_FLOATS * sizeof(float);
    size_t m = (size_t)M_DOUBLES * sizeof(double);
    size_t red = (size_t)2 * FIT_THREADS * 16 * sizeof(float);
    size_t u = jc > m ? jc : m;
    if (red > u) u = red;
    return (size_t)PX_SMEM * sizeof(float) + u;
}

static const void* fit_kernel_ptr(int tpt) {
    return tpt == 1 ? (const void*)k_lm_fit<1> : (const void*)k_lm_fit<3>;
}

int fit_tpt_for(int k_max) { return fit_tiles(k_max) <= FIT_THREADS ? 1 : 3; }

cudaError_t fit_configure(int tpt, int* blocks_per_sm) {
    const void* fn = fit_kernel_ptr(tpt);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fit_smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, FIT_THREADS, fit_smem_bytes());
}

cudaError_t launch_lm_fit(int tpt, int grid, const float* src, int src_w, const FitDesc* desc, const LMConst& lmc,
                          FitOut* out, double* partials, double* sums, unsigned* bar, float* Tg,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(FIT_THREADS);
    cfg.dynamicSmemBytes = fit_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (tpt == 1)
        return cudaLaunchKernelEx(&cfg, k_lm_fit<1>, src, src_w, desc, lmc, out, partials, sums, bar, Tg);
    return cudaLaunchKernelEx(&cfg, k_lm_fit<3>, src, src_w, desc, lmc, out, partials, sums, bar, Tg);
}

}  // namespace aspd
