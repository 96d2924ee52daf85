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
//      leaf sums of <= 64 pixels, Kahan-compensated across leaves; each CTA
//      writes its partial sums as FP32 (sum, -compensation) pairs;
//   2. grid barrier -> every CTA combines the CTAs' chi^2 pairs and takes the
//      LM decision (all CTAs identically);
//   3. accepted steps only: error-free FP32 pair reduction of every entry
//      over the CTAs, one FP64 value (and its FP32 rounding) per entry ->
//      grid barrier; a rejected step keeps the current point's sums;
//   4. every CTA redundantly solves (A + lambda diag A) delta = g (scaled
//      FP32 Cholesky, FP64 refinement when a pivot is small), so no further
//      barrier is needed to broadcast the next trial point.
// Grid barriers are bounded spins; on timeout the kernel records an error
// and returns.
// This header holds the fit kernel itself (helpers, the body and the kernel
// templates); asp_fit.cu instantiates the circular model and the launch
// code, asp_fit_models.cu the elliptical and joint models.
#pragma once
#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {

namespace {

constexpr int CH_SMALL = 256;   // chunk pixels when NAp <= 64
constexpr int CH_LARGE = 128;   // chunk pixels when NAp <= PMAX_S + 4
constexpr int CH_XL = 64;       // chunk pixels of the large-active-set variant
// Two shared-memory layouts.  Variant S (K <= KMAX_S) caches A of the
// current point in shared memory; variant L (K <= KMAX) reads A from the
// L2-resident sums buffer and gives the union region to the J chunk or the
// FP32 factor with its panel.
constexpr int KMAX_S = 32;
constexpr int PMAX_S = 4 * KMAX_S;
constexpr int NB_S = (PMAX_S + 4) / 4;
constexpr int NACC_S = NB_S * (NB_S + 1) / 2 * 16;            // cached sums of S, tile order (FP64 and FP32)
constexpr int UNI_L_FLOATS = ((PMAX + 1) * (PMAX + 2) / 2 + 3) / 4 * 4 + 8 * (PMAX + 4);
// Speculation block in the speculating CTA's partial row (doubles from
// SPEC_OFF): two broadcast records of the pixel CTAs' LM state (8 doubles
// each), then two speculative steps (lambda, ok, delta[PMAX]).  Above the
// FP64 fallback factor the same row can hold (P (P+1) / 2 doubles).
constexpr int SPEC_BC = 8;
constexpr int SPEC_STEP = PMAX + 8;
constexpr int SPEC_OFF = NACC_MAX - 2 * SPEC_BC - 2 * SPEC_STEP;
static_assert(SPEC_OFF >= PMAX * (PMAX + 1) / 2, "the speculation block must not overlap the FP64 fallback factor");
static_assert(UNI_L_FLOATS >= CH_XL * (NAP_MAX + 4), "J chunk of the large variant must fit its union region");

// 64 bytes, 16-byte aligned: the circular fields come first, so the pixel
// loop of the circular fit reads its frame with two 16-byte loads.
struct __align__(16) MemberFrame {
    float a, c, iw2, iw3;           // circular: c = log2(e) / (2 w^2); elliptical: c = log2(e) A / 2
    float fx, fy;
    int cx, cy;
    float cb, cc;                   // elliptical: log2(e) B, log2(e) C / 2 (exponent coefficients)
    float pa, pb, pc;               // elliptical: A, B, C (Jacobian); joint: pa = s
    float pad0, pad1, pad2;
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int pidx(int i, int j) { return i * (i + 1) / 2 + j; }   // packed lower, j <= i

// Error-free FP32 sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// Add the FP32 pair (hi, lo) into the running pair (s, c), in FP32.
__device__ __forceinline__ void pair_add(float& s, float& c, float hi, float lo) {
    float e;
    two_sum(s, hi, s, e);
    c += e + lo;
}

__device__ __forceinline__ int tile_index(int bi, int bj, int nb) { return bi * nb - bi * (bi - 1) / 2 + (bj - bi); }

// Accumulator entry of (i, j) of [J | r]^T [J | r].
__device__ __forceinline__ int acc_index(int i, int j, int nb) {
    if (i > j) { int t = i; i = j; j = t; }
    return tile_index(i >> 2, j >> 2, nb) * 16 + (i & 3) * 4 + (j & 3);
}

// Grid barrier of the fit group: a release increment and acquire polls by
// thread 0, block barriers around them (the block barrier makes the CTA's
// writes visible to thread 0; release and acquire are cumulative).  Bounded:
// after SPIN_LIMIT polls the CTA records a timeout and returns.
__device__ void grid_barrier(unsigned* bar, unsigned target, int* s_err, int* g_err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add_u32(bar, 1u);
        unsigned spins = 0;
        while (ld_acquire_u32(bar) < target) {
            if (++spins > SPIN_LIMIT) {
                *s_err = 1;
                atomicExch(g_err, ASP_ERR_TIMEOUT);
                break;
            }
        }
    }
    __syncthreads();
}

// Frame of member k for the FP32 pass: integer centre plus fractional offset
// so dx = (px - cx) - fx is computed without cancellation.
__device__ __forceinline__ void make_frame(const double* th, MemberFrame& f) {
    double a = th[0], x = th[1], y = th[2], w = th[3];
    double cx = floor(x + 0.5), cy = floor(y + 0.5);
    const double iw = 1.0 / w, iw2 = iw * iw;
    f.a = (float)a;
    f.c = (float)(0.5 * LOG2E * iw2);
    f.iw2 = (float)iw2;
    f.iw3 = (float)(iw2 * iw);
    f.fx = (float)(x - cx);
    f.fy = (float)(y - cy);
    f.cx = (int)cx;
    f.cy = (int)cy;
}

// Elliptical member (a, x, y, A, B, C): a exp(-(A dx^2 + 2 B dx dy + C
// dy^2) / 2) = a exp2(-(c dx^2 + cb dx dy + cc dy^2)), same centre frame.
__device__ __forceinline__ void make_frame_ell(const double* th, MemberFrame& f) {
    const double a = th[0], x = th[1], y = th[2], A = th[3], B = th[4], C = th[5];
    const double cx = floor(x + 0.5), cy = floor(y + 0.5);
    f.a = (float)a;
    f.c = (float)(0.5 * LOG2E * A);
    f.cb = (float)(LOG2E * B);
    f.cc = (float)(0.5 * LOG2E * C);
    f.pa = (float)A;
    f.pb = (float)B;
    f.pc = (float)C;
    f.fx = (float)(x - cx);
    f.fy = (float)(y - cy);
    f.cx = (int)cx;
    f.cy = (int)cy;
}

// Joint member (x, y, s, a_1 .. a_C): the centre frame only; the
// per-channel amplitude and 1 / omega_kc^2 live in the pass's channel
// tables.  pa carries s (the Jacobian's d/ds = g r^2 s / omega^4).
__device__ __forceinline__ void make_frame_mc(const double* th, MemberFrame& f) {
    const double x = th[0], y = th[1];
    const double cx = floor(x + 0.5), cy = floor(y + 0.5);
    f.pa = (float)th[2];
    f.fx = (float)(x - cx);
    f.fy = (float)(y - cy);
    f.cx = (int)cx;
    f.cy = (int)cy;
}

// Eigenvalues (mu-, mu+) of the precision matrix [[A, B], [B, C]].
__device__ __forceinline__ void prec_eig(double A, double B, double C, double& mm, double& mp) {
    const double h = 0.5 * (A + C), r = hypot(0.5 * (A - C), B);
    mm = h - r;
    mp = h + r;
}

// Pivot l = sqrt(d) and 1/l.  FP32 (the refined factor): rsqrtf, whose
// few-ulp error the FP64 refinement removes; FP64: correctly rounded.
__device__ __forceinline__ void pivot(double d, double& l, double& il) { l = sqrt(d); il = 1.0 / l; }

// Cholesky factorisation of the packed lower matrix M in place: columns
// 0..P-1 of rows 0..nrows-1 (nrows = P + 1 carries a right-hand side b as
// row P, which comes out as L^-1 b: the forward substitution fused into the
// factorisation).  Blocked right-looking with 4-column panels: thread 0
// factors the 4x4 diagonal block, one thread per row solves the panel, and
// the trailing rank-4 update runs one row per warp, one column per lane.
// Three block barriers per panel.  Returns false if a pivot is not positive.
template <class T>
__device__ bool cholesky_packed(T* M, int P, int nrows, T* inv_diag, int* s_flag) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
#pragma unroll 1
    for (int j0 = 0; j0 < P; j0 += 4) {
        const int nbk = min(4, P - j0);
        if (tid == 0) {
#pragma unroll 1
            for (int c = 0; c < nbk; ++c) {
                const int jc = j0 + c;
                const T d = M[pidx(jc, jc)];
                if (!(d > T(0)) || !isfinite(d)) { *s_flag = 1; break; }
                T l, il;
                pivot(d, l, il);
                M[pidx(jc, jc)] = l;
                inv_diag[jc] = il;
                for (int r = c + 1; r < nbk; ++r) M[pidx(j0 + r, jc)] *= il;
                for (int r = c + 1; r < nbk; ++r)
                    for (int s = c + 1; s <= r; ++s) M[pidx(j0 + r, j0 + s)] -= M[pidx(j0 + r, jc)] * M[pidx(j0 + s, jc)];
            }
        }
        __syncthreads();
        if (*s_flag) return false;
        const int r0 = j0 + nbk;
        for (int i = r0 + tid; i < nrows; i += blockDim.x) {      // panel rows below the block
            T* row = M + pidx(i, 0);
#pragma unroll 1
            for (int c = 0; c < nbk; ++c) {
                T v = row[j0 + c];
                for (int t = 0; t < c; ++t) v -= row[j0 + t] * M[pidx(j0 + c, j0 + t)];
                row[j0 + c] = v * inv_diag[j0 + c];
            }
        }
        __syncthreads();
        for (int i = r0 + warp; i < nrows; i += nwarp) {         // trailing rank-nbk update
            T* row = M + pidx(i, 0);
            T li[4];
            for (int c = 0; c < 4; ++c) li[c] = c < nbk ? row[j0 + c] : T(0);
            const int kmax = min(i, P - 1);
            for (int k = r0 + lane; k <= kmax; k += 32) {
                const T* rk = M + pidx(k, 0) + j0;
                T acc = row[k];
                for (int c = 0; c < nbk; ++c) acc -= li[c] * rk[c];
                row[k] = acc;
            }
        }
        __syncthreads();
    }
    return true;
}

// Triangular solves with warp 0, the right-hand side held in registers
// (lane l owns entries l, l+32, l+64, l+96), four unknowns per step: the
// four are broadcast by shuffle, every lane solves the 4x4 diagonal block
// redundantly, then updates its own entries.  No warp barriers (a
// __syncwarp round costs ~200 cycles on this part, a shuffle ~30).
// mode 1: forward (L y = b), 2: backward (L^T x = y), 3: both.
template <class T>
__device__ __forceinline__ T slot_get(const T (&v)[4], int s) { return s == 0 ? v[0] : s == 1 ? v[1] : s == 2 ? v[2] : v[3]; }

template <class T>
__device__ void trsv_warp(const T* __restrict__ M, int P, const T* __restrict__ inv_diag, T* b, int mode) {
    if (threadIdx.x >= 32) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x;
    T v[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) v[s] = lane + 32 * s < P ? b[lane + 32 * s] : T(0);
    if (mode & 1) {
#pragma unroll 1
        for (int j0 = 0; j0 < P; j0 += 4) {
            const int nb = min(4, P - j0), slot = j0 >> 5, l0 = j0 & 31;
            const T vs = slot_get(v, slot);
            T y[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) y[c] = __shfl_sync(FULL, vs, l0 + c);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c < nb) {
                    T a = y[c];
#pragma unroll
                    for (int t = 0; t < c; ++t) a -= M[pidx(j0 + c, j0 + t)] * y[t];
                    y[c] = a * inv_diag[j0 + c];
                } else {
                    y[c] = T(0);
                }
            }
            // owners keep the solved values; everyone below updates
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int i = lane + 32 * s;
                if (s == slot && i >= j0 && i < j0 + nb) v[s] = slot_get(y, i - j0);
                if (i >= j0 + nb && i < P) {
                    const T* ri = M + pidx(i, 0) + j0;
                    T a = v[s];
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (c < nb) a -= ri[c] * y[c];
                    v[s] = a;
                }
            }
        }
    }
    if (mode & 2) {
        const int last = ((P - 1) / 4) * 4;
#pragma unroll 1
        for (int j0 = last; j0 >= 0; j0 -= 4) {
            const int nb = min(4, P - j0), slot = j0 >> 5, l0 = j0 & 31;
            const T vs = slot_get(v, slot);
            T x[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) x[c] = __shfl_sync(FULL, vs, l0 + c);
#pragma unroll
            for (int c = 3; c >= 0; --c) {
                if (c < nb) {
                    T a = x[c];
#pragma unroll
                    for (int t = c + 1; t < 4; ++t)
                        if (t < nb) a -= M[pidx(j0 + t, j0 + c)] * x[t];
                    x[c] = a * inv_diag[j0 + c];
                } else {
                    x[c] = T(0);
                }
            }
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int i = lane + 32 * s;
                if (s == slot && i >= j0 && i < j0 + nb) v[s] = slot_get(x, i - j0);
                if (i < j0) {
                    T a = v[s];
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (c < nb) a -= M[pidx(j0 + c, i)] * x[c];
                    v[s] = a;
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (lane + 32 * s < P) b[lane + 32 * s] = v[s];
}

// The FP32 factor (packed lower, P4 + 1 rows with the right-hand side row;
// P4 = P padded with identity rows to a multiple of the panel width, 4 for
// P <= 32 and 8 above: narrow panels keep the pivot chain short for small
// P, wide ones halve the barriers for large P) is followed by its panel Lp
// (PB columns of ld lp_ld >= P + 1) at a 4-float-aligned offset.
__host__ __device__ constexpr int lp_offset(int P4) { return ((P4 + 1) * (P4 + 2) / 2 + 3) & ~3; }
// Union region of S: the J chunk (rows x NAp floats, rows chosen to fit),
// the FP32 factor of P4 <= PMAX_S with its 8-column panel, or the CTA's leaf
// sums of several pixel groups (2 x FIT_THREADS x 17 floats).
constexpr int JC_FLOATS = lp_offset(PMAX_S) + 8 * (PMAX_S + 4);
static_assert(JC_FLOATS >= 2 * FIT_THREADS * 17, "parked leaf sums (17 floats a tile) must fit the union region");
static_assert(JC_FLOATS / (PMAX_S + 8) >= 64, "the J chunk of S must hold 64 rows");

// Factor the PBxPB diagonal block at r0 (lower, packed in M) in registers,
// every lane of the calling warp redundantly; lane 0 stores the factor and
// its inverse pivots.  If Lp is given, the panel rows r0..r0+PB-1 (PB columns
// of ld LP_LD) are first subtracted (panel columns in ascending order).  The
// elimination is right-looking, the trailing entries updated at once, so the
// chain from one pivot to the next is one multiply, one FMA and the
// reciprocal square root.  Returns false if a pivot is not positive and
// finite.
template <int PB>
__device__ __forceinline__ bool factor_diag_rl(float* __restrict__ M, const float* __restrict__ Lp, int LP_LD,
                                               float* __restrict__ inv_diag, int r0, int lane) {
    float d[PB][PB];
#pragma unroll
    for (int r = 0; r < PB; ++r)
#pragma unroll
        for (int t = 0; t <= r; ++t) d[r][t] = M[pidx(r0 + r, r0 + t)];
    if (Lp) {
#pragma unroll
        for (int c = 0; c < PB; ++c) {
            float l[PB];
#pragma unroll
            for (int q = 0; q < PB; q += 4) {
                const float4 v = *reinterpret_cast<const float4*>(Lp + c * LP_LD + r0 + q);
                l[q] = v.x; l[q + 1] = v.y; l[q + 2] = v.z; l[q + 3] = v.w;
            }
#pragma unroll
            for (int r = 0; r < PB; ++r)
#pragma unroll
                for (int t = 0; t <= r; ++t) d[r][t] = fmaf(-l[r], l[t], d[r][t]);
        }
    }
    // The next pivot's update and reciprocal square root are issued first in
    // each column (warps issue in program order), the rest of the column's
    // update while it is in flight.  v > 0 && v < inf also rejects NaN.
    float inv[PB];
    bool ok = (d[0][0] > 0.f) & (d[0][0] < INFINITY);
    float il = rsqrtf(d[0][0]);
#pragma unroll
    for (int c = 0; c < PB; ++c) {
        inv[c] = il;
        d[c][c] = d[c][c] * il;
        float il_next = 0.f;
        if (c + 1 < PB) {
            d[c + 1][c] *= il;
            d[c + 1][c + 1] = fmaf(-d[c + 1][c], d[c + 1][c], d[c + 1][c + 1]);
            const float vn = d[c + 1][c + 1];
            ok = ok & (vn > 0.f) & (vn < INFINITY);
            il_next = rsqrtf(vn);
        }
#pragma unroll
        for (int r = c + 2; r < PB; ++r) d[r][c] *= il;
#pragma unroll
        for (int r = c + 2; r < PB; ++r)
#pragma unroll
            for (int t = c + 1; t <= r; ++t) d[r][t] = fmaf(-d[r][c], d[t][c], d[r][t]);
        il = il_next;
    }
    __syncwarp();   // every lane has read the block
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < PB; ++c) {
#pragma unroll
            for (int t = 0; t <= c; ++t) M[pidx(r0 + c, r0 + t)] = d[c][t];
            inv_diag[r0 + c] = inv[c];
        }
    }
    return ok;
}

// Cholesky factorisation of the packed lower FP32 matrix M in place: rows
// 0..P (row P carries a right-hand side b and comes out as L^-1 b, the
// forward substitution fused into the factorisation), P a multiple of the
// panel width PB.  Blocked right-looking with look-ahead; per panel:
//   (A) one thread per row below the diagonal block solves its panel
//       entries against the factored block, stored in place and column-major
//       in Lp (PB columns of ld LP_LD, 16-byte aligned);
//   (B) warps 0..nwarp-2 apply the trailing update on 4x4 register tiles
//       (two 16-byte panel loads per panel column for 16 FMAs), rows
//       r0 + 4 bi (bi >= PB / 4) and columns r0 + 4 bj, bj <= bi, while the
//       last warp takes the next diagonal block with this panel's update and
//       factors it (factor_diag_rl).
// Two block barriers per panel.  *s_flag must be 0 on entry; returns false
// if a pivot fails.
template <int PB>
__device__ bool chol_tiled(float* __restrict__ M, float* __restrict__ Lp, int P, float* __restrict__ inv_diag,
                           int* s_flag, const int LP_LD) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int nrows = P + 1;
    const int nupd = (nwarp - 1) * 32;
    if (warp == nwarp - 1 && !factor_diag_rl<PB>(M, nullptr, LP_LD, inv_diag, 0, lane) && lane == 0) *s_flag = 1;
    __syncthreads();
    if (*s_flag) return false;
#pragma unroll 1
    for (int j0 = 0; j0 < P; j0 += PB) {
        const int r0 = j0 + PB;
        // A: panel rows below the diagonal block
        const int i = r0 + tid;
        if (i < nrows) {
            float a[PB], iv[PB];
#pragma unroll
            for (int c = 0; c < PB; ++c) { a[c] = M[pidx(i, j0 + c)]; iv[c] = inv_diag[j0 + c]; }
            float l[PB][PB];
#pragma unroll
            for (int c = 1; c < PB; ++c)
#pragma unroll
                for (int t = 0; t < c; ++t) l[c][t] = M[pidx(j0 + c, j0 + t)];
#pragma unroll
            for (int c = 0; c < PB; ++c) {
                a[c] *= iv[c];
#pragma unroll
                for (int r = c + 1; r < PB; ++r) a[r] = fmaf(-l[r][c], a[c], a[r]);
            }
#pragma unroll
            for (int c = 0; c < PB; ++c) {
                M[pidx(i, j0 + c)] = a[c];
                Lp[c * LP_LD + i] = a[c];
            }
        }
        __syncthreads();
        if (warp == nwarp - 1) {
            if (r0 < P && !factor_diag_rl<PB>(M, Lp, LP_LD, inv_diag, r0, lane) && lane == 0) *s_flag = 1;
        } else {
            const int nbr = (nrows - r0 + 3) >> 2;
            const int T0 = (PB / 4) * (PB / 4 + 1) / 2;
            const int ntile = nbr * (nbr + 1) / 2 - T0;
            for (int u = tid; u < ntile; u += nupd) {
                const int uu = u + T0;
                int bi = (int)((sqrtf(8.f * (float)uu + 1.f) - 1.f) * 0.5f);
                while (bi * (bi + 1) / 2 > uu) --bi;
                while ((bi + 1) * (bi + 2) / 2 <= uu) ++bi;
                const int bj = uu - bi * (bi + 1) / 2;
                const int i0 = r0 + 4 * bi, k0 = r0 + 4 * bj;
                float acc[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ii = i0 + r, kk = k0 + q;
                        acc[r][q] = (ii < nrows && kk <= ii && kk < P) ? M[pidx(ii, kk)] : 0.f;
                    }
#pragma unroll
                for (int c = 0; c < PB; ++c) {
                    const float4 li = *reinterpret_cast<const float4*>(Lp + c * LP_LD + i0);
                    const float4 lk = *reinterpret_cast<const float4*>(Lp + c * LP_LD + k0);
                    const float lr[4] = {li.x, li.y, li.z, li.w};
                    const float lq[4] = {lk.x, lk.y, lk.z, lk.w};
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(-lr[r], lq[q], acc[r][q]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ii = i0 + r, kk = k0 + q;
                        if (ii < nrows && kk <= ii && kk < P) M[pidx(ii, kk)] = acc[r][q];
                    }
            }
        }
        __syncthreads();
        if (*s_flag) return false;
    }
    return true;
}

// Back substitution L^T x = y with L from chol_tiled (P a multiple of PB),
// all threads, PB-row blocks from the bottom, one block barrier per block:
// every thread solves the block's 8 unknowns redundantly from the (already
// updated) y entries, then thread i < jb removes them from y_i.  y is
// destroyed; x must not alias y.
template <int PB>
__device__ void trsv_back_block(const float* __restrict__ M, int P, const float* __restrict__ inv_diag,
                                float* __restrict__ y, float* __restrict__ x) {
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int jb = P - PB; jb >= 0; jb -= PB) {
        if (tid < max(jb, PB)) {     // warps without rows to update skip the loads
        float xb[PB], iv[PB], l[PB][PB];
#pragma unroll
        for (int c = 0; c < PB; ++c) { xb[c] = y[jb + c]; iv[c] = inv_diag[jb + c]; }
#pragma unroll
        for (int c = 1; c < PB; ++c)
#pragma unroll
            for (int t = 0; t < c; ++t) l[c][t] = M[pidx(jb + c, jb + t)];
        const int i = tid < jb ? tid : jb;   // others load a row nobody writes in this block
        float lr[PB];
#pragma unroll
        for (int c = 0; c < PB; ++c) lr[c] = M[pidx(jb + c, i)];
        float yi = y[i];
#pragma unroll
        for (int c = PB - 1; c >= 0; --c) {
            xb[c] *= iv[c];
#pragma unroll
            for (int t = 0; t < c; ++t) xb[t] = fmaf(-l[c][t], xb[c], xb[t]);
        }
        if (tid < PB) {
            float xv = xb[0];
#pragma unroll
            for (int c = 1; c < PB; ++c) xv = tid == c ? xb[c] : xv;
            x[jb + tid] = xv;
        }
        if (tid < jb) {
#pragma unroll
            for (int c = 0; c < PB; ++c) yi = fmaf(-lr[c], xb[c], yi);
            y[tid] = yi;
        }
        }
        __syncthreads();
    }
}

// Forward substitution L z = r, the mirror of trsv_back_block: blocks from
// the top, thread i >= jb + PB removes the block's unknowns from r_i.  r is
// destroyed; z must not alias r.
template <int PB>
__device__ void trsv_fwd_block(const float* __restrict__ M, int P, const float* __restrict__ inv_diag,
                               float* __restrict__ r, float* __restrict__ z) {
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int jb = 0; jb < P; jb += PB) {
        if (tid < max(P - jb - PB, PB)) {     // warps without rows to update skip the loads
        float zb[PB], iv[PB], l[PB][PB];
#pragma unroll
        for (int c = 0; c < PB; ++c) { zb[c] = r[jb + c]; iv[c] = inv_diag[jb + c]; }
#pragma unroll
        for (int c = 1; c < PB; ++c)
#pragma unroll
            for (int t = 0; t < c; ++t) l[c][t] = M[pidx(jb + c, jb + t)];
        const int i = jb + PB + tid;
        const bool upd = i < P;
        const int ir = upd ? i : jb + PB - 1;
        float lr[PB];
#pragma unroll
        for (int c = 0; c < PB; ++c) lr[c] = M[pidx(ir, jb + c)];
        float ri = r[ir];
#pragma unroll
        for (int c = 0; c < PB; ++c) {
            zb[c] *= iv[c];
#pragma unroll
            for (int t = c + 1; t < PB; ++t) zb[t] = fmaf(-l[t][c], zb[c], zb[t]);
        }
        if (tid < PB) {
            float zv = zb[0];
#pragma unroll
            for (int c = 1; c < PB; ++c) zv = tid == c ? zb[c] : zv;
            z[jb + tid] = zv;
        }
        if (upd) {
#pragma unroll
            for (int c = 0; c < PB; ++c) ri = fmaf(-lr[c], zb[c], ri);
            r[i] = ri;
        }
        }
        __syncthreads();
    }
}

// A (the normal-equation matrix of the current point, FP64, symmetric)
// as the solve reads it: the tile-ordered accumulator sums, copied to shared
// memory (variant S) or read from global memory / L2 (variant L).
struct SmemTileA {
    const double* p;
    int nb;
    __device__ __forceinline__ double operator()(int i, int j) const { return p[acc_index(i, j, nb)]; }
};
struct TileA {
    const double* p;
    int nb;
    __device__ __forceinline__ double operator()(int i, int j) const { return __ldcg(p + acc_index(i, j, nb)); }
};
// The FP32 copy of A (the reduction writes both) for the solve's setup: its
// tile-ordered entries (shared memory for variant S, global memory / L2 for
// variant L), the tile table (tile -> (bi, bj)) and the diagonal.
struct TiledA32 {
    const float* p;          // nacc entries, tile order
    const short2* ttab;
    const float* diag;       // A_ii, i < P
    int nacc;
    bool global;
};

constexpr float REFINE_INV_MAX = 10.0f;   // refine when some 1/L_jj of the scaled factor exceeds this

struct SolveWork {              // shared-memory scratch of solve_damped
    double bt[PMAX], ud[PMAX], inv64[PMAX];
    double rq[4][64];           // the refinement residual's column-quarter sums
    float sf[PMAX], mf[PMAX], xv[PMAX], zv[PMAX], cv[PMAX], inv32[PMAX];
    int flag, refinements, fallbacks, pad;
};

// FP32 scaled factor-and-refine solve (see solve_damped) with panel width
// PB; P4 = P rounded up to PB.  The scaled matrix is built from the FP32
// copy A32 of A (g32, dv32 likewise): no FP64 instruction outside the
// refinement.  Returns false if the FP32 factor fails.
template <int PB, class AT>
__device__ bool solve_scaled_fp32(const AT& A, const TiledA32& A32, const double* __restrict__ g,
                                  const float* __restrict__ g32, const double* __restrict__ dv,
                                  const float* __restrict__ dv32, double lam, int P, void* uni, SolveWork& w,
                                  double* __restrict__ delta) {
    const int tid = threadIdx.x;
    const int P4 = (P + PB - 1) & ~(PB - 1);   // padded with identity rows: every block of the factor is full
    float* L32 = reinterpret_cast<float*>(uni);
    float* Lp = L32 + lp_offset(P4);
    const int lp_ld = P4 + 4;
    const float lam32 = (float)lam;
    for (int i = tid; i < P4; i += blockDim.x) {
        float sc = 1.0f, m = 1.0f;
        if (i < P) {
            m = fmaf(lam32, dv32[i], A32.diag[i]);
            sc = m > 0.f ? rsqrtf(m) : 1.0f;
        }
        w.sf[i] = sc;
        w.mf[i] = m;
    }
    if (tid == 0) w.flag = 0;
    __syncthreads();
    // S (A + lam D) S into the packed lower factor, straight from the tile
    // order (entry e of tile (bi, bj), bi <= bj, is (i, j) = (4 bi + e/4 % 4,
    // 4 bj + e % 4); diagonal tiles also hold i > j, skipped)
#pragma unroll 4
    for (int e = tid; e < A32.nacc; e += blockDim.x) {
        const float a = A32.global ? __ldcg(A32.p + e) : A32.p[e];
        const short2 bij = A32.ttab[e >> 4];
        const int i = 4 * bij.x + ((e >> 2) & 3), j = 4 * bij.y + (e & 3);
        if (i <= j && j < P) L32[pidx(j, i)] = (i == j ? w.mf[j] : a) * w.sf[j] * w.sf[i];
    }
    // right-hand side row S g; identity padding rows P..P4-1
    for (int j = tid; j < P4; j += blockDim.x) L32[pidx(P4, j)] = j < P ? w.sf[j] * g32[j] : 0.f;
    for (int q = tid; q < (P4 - P) * P4; q += blockDim.x) {
        const int i = P + q / P4, j = q % P4;
        if (j <= i) L32[pidx(i, j)] = i == j ? 1.f : 0.f;
    }
    __syncthreads();
    if (chol_tiled<PB>(L32, Lp, P4, w.inv32, &w.flag, lp_ld)) {
        trsv_back_block<PB>(L32, P4, w.inv32, L32 + pidx(P4, 0), w.xv);      // x = L^-T (L^-1 S g)
        // The scaled matrix has a unit diagonal, so its Cholesky pivots
        // L_jj^2 lie in (0, 1] and a small one marks a near-dependency.  With
        // every pivot >= 1e-2 (1/L_jj <= 10) the FP32 solution is accurate to
        // a few 1e-5 relative -- the FP32 normal equations' own level -- and
        // the FP64 refinement is skipped.
        const int refine = __syncthreads_or(tid < P4 && !(w.inv32[tid] <= REFINE_INV_MAX));
        if (!refine) {
            for (int i = tid; i < P; i += blockDim.x) delta[i] = (double)w.sf[i] * (double)w.xv[i];
            __syncthreads();
            return true;
        }
        for (int i = tid; i < P4; i += blockDim.x) {
            w.ud[i] = (double)w.sf[i] * (double)w.xv[i];
            w.bt[i] = i < P ? (double)w.sf[i] * g[i] : 0.0;
        }
        __syncthreads();
        // refinement: c = (L L^T)^-1 (S g - S (A + lam D) S x), residual in
        // FP64.  Row i's columns are split in four quarters over the four
        // thread groups of 64 (so the FP64 work spreads over all the SM's
        // schedulers), each quarter as two FMA chains; the quarters are
        // added in order.  P4 > 64 takes further rows in later rounds.
        {
            const int nq = (int)blockDim.x / 64;          // 4 column quarters
            const int qi = tid / 64, ri = tid % 64;
            const int qlen = (P + nq - 1) / nq;
            const int ja = qi * qlen, jb = min(P, ja + qlen);
            for (int i0 = 0; i0 < P4; i0 += 64) {
                const int i = i0 + ri;
                double part = 0.0;
                if (i < P) {
                    double a0 = 0.0, a1 = 0.0;
                    int j = ja;
                    for (; j + 1 < jb; j += 2) {
                        const double v0 = A(i, j), v1 = A(i, j + 1);
                        a0 = fma(v0, w.ud[j], a0);
                        a1 = fma(v1, w.ud[j + 1], a1);
                    }
                    if (j < jb) a0 = fma(A(i, j), w.ud[j], a0);
                    part = a0 + a1;
                }
                w.rq[qi][ri] = part;
                __syncthreads();
                if (tid < 64 && i < P4) {
                    if (i >= P) {
                        w.cv[i] = 0.f;
                    } else {
                        const double mx = ((w.rq[0][ri] + w.rq[1][ri]) + (w.rq[2][ri] + w.rq[3][ri])) +
                                          lam * dv[i] * w.ud[i];
                        w.cv[i] = (float)(w.bt[i] - (double)w.sf[i] * mx);
                    }
                }
                __syncthreads();
            }
        }
        if (tid == 0) w.refinements += 1;
        __syncthreads();
        trsv_fwd_block<PB>(L32, P4, w.inv32, w.cv, w.zv);
        trsv_back_block<PB>(L32, P4, w.inv32, w.zv, w.cv);
        for (int i = tid; i < P; i += blockDim.x) delta[i] = (double)w.sf[i] * ((double)w.xv[i] + (double)w.cv[i]);
        __syncthreads();
        return true;
    }
    return false;
}

// Solve (A + lam diag(dv)) delta = g, all threads of the block; A is read
// through the FP64 accessor (tile-ordered sums in shared memory or L2) and
// its FP32 copy through A32.  With S = diag(A + lam D)^-1/2 rounded to FP32
// (any diagonal scaling serves; an FP32 one is exact in FP64 below), the
// matrix S (A + lam D) S, augmented by the row S g, is factored in FP32 (the
// forward substitution comes out of the factorisation); one back
// substitution gives x; when a pivot of the unit-diagonal factor is below
// 1e-2, one step of iterative refinement with the residual
// S g - S (A + lam D) S x evaluated in FP64 corrects it; delta = S x.  If the
// FP32 factor fails, an FP64 factor of the unscaled matrix is used, in m64
// (P (P+1) / 2 doubles: the CTA's partial row in global memory).  Returns
// false when the damped matrix is not positive definite.
template <class AT>
__device__ bool solve_damped(const AT& A, const TiledA32& A32, const double* __restrict__ g, const float* __restrict__ g32,
                             const double* __restrict__ dv, const float* __restrict__ dv32, double lam, int P,
                             void* uni, double* m64, SolveWork& w, double* __restrict__ delta) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    if (P <= 32 ? solve_scaled_fp32<4>(A, A32, g, g32, dv, dv32, lam, P, uni, w, delta)
                : solve_scaled_fp32<8>(A, A32, g, g32, dv, dv32, lam, P, uni, w, delta))
        return true;
    // FP64 factor of the unscaled damped matrix
    if (tid == 0) w.fallbacks += 1;
    double* M64 = m64;
    for (int i = warp; i < P; i += nwarp)
        for (int j = lane; j <= i; j += 32) {
            double v = A(i, j);
            if (i == j) v += lam * dv[i];
            M64[pidx(i, j)] = v;
        }
    if (tid == 0) w.flag = 0;
    __syncthreads();
    if (!cholesky_packed<double>(M64, P, P, w.inv64, &w.flag)) return false;
    for (int i = tid; i < P; i += blockDim.x) delta[i] = g[i];
    __syncthreads();
    trsv_warp<double>(M64, P, w.inv64, delta, 3);
    __syncthreads();
    return true;
}

}  // namespace

// The whole fit of one window, run by the CTAs of one fit group; b is this
// CTA's rank in the group (the group has d.grid CTAs).
template <int TPT, bool LARGE, int MODEL>
__device__ __forceinline__ void lm_fit_body(const float* __restrict__ src, int src_w, const FitDesc* __restrict__ descp,
                                            const LMConst& lmc, FitOut* __restrict__ out, double* __restrict__ partials,
                                            double* __restrict__ sums, unsigned* __restrict__ bar,
                                            float* __restrict__ Tg, const int b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Ts = reinterpret_cast<float*>(smem_raw);                          // PX_SMEM floats
    // variant S: A at the current point cached in shared memory; variant L:
    // A read from the sums buffer (L2), the union region follows Ts
    double* Ac = LARGE ? nullptr : reinterpret_cast<double*>(Ts + PX_SMEM);   // FP64 sums, tile order
    float* Ac32 = LARGE ? nullptr : reinterpret_cast<float*>(Ac + NACC_S);    // FP32 sums, tile order
    float* Jc = LARGE ? Ts + PX_SMEM : Ac32 + NACC_S;                          // union region
    float* red = Jc;
    float* sums32 = reinterpret_cast<float*>(sums + 2 * NACC_MAX);            // FP32 copies of both buffers
    float2* chib = reinterpret_cast<float2*>(sums + 3 * NACC_MAX);            // chi^2 partials, 2 x FIT_GRID_MAX

    __shared__ FitDescHead d;
    __shared__ MemberFrame fr[KMAX];
    __shared__ short2 ttab[NTILES_MAX];     // layout tile t -> (bi, bj), row-major upper triangle
    __shared__ short tperm[NTILES_MAX];     // SYRK thread order -> layout tile
    __shared__ double theta[PMAX], trial[PMAX], delta[PMAX], gvec[PMAX], dvec[PMAX];
    __shared__ float g32[PMAX], dv32[PMAX], a32d[PMAX];
    __shared__ SolveWork sw;
    __shared__ double s_lam, s_chi2, s_chi2_init;
    __shared__ double s_lam_acc, s_lam_rej, s_thr;   // the decision's FP64 terms, computed during the pass
    __shared__ double s_chi2_t;                       // chi^2 at the trial point
    __shared__ int s_cur, s_iters, s_passes, s_status, s_done, s_err, s_flag, s_go, s_acc, s_small, s_rej_stall;
    __shared__ float s_pred[2], s_thr32;   // predicted-decrease sums; rtol chi^2 of the current point
    __shared__ unsigned s_flags;          // post-solve flags: finite, valid, small
    __shared__ int s_use_spec;            // this solve takes the speculating CTA's step

    const int tid = threadIdx.x;
    {
        const int* srcw = reinterpret_cast<const int*>(descp);
        int* dstw = reinterpret_cast<int*>(&d);
        for (int i = tid; i < (int)(sizeof(FitDescHead) / sizeof(int)); i += blockDim.x) dstw[i] = srcw[i];
    }
    __syncthreads();
    if (!d.active) return;
    const int G = d.grid;
    if (b >= G) return;
    // Speculation.  With three or more CTAs the last one holds no pixels: it
    // solves the damped system at lambda_up x lambda, the step a rejected
    // trial asks for next, while the others run the trial's pixel pass, so a
    // rejected step costs no solve.  Gp CTAs split the window.
    const int Gp = fit_pixel_ctas(G);
    const bool spec_on = Gp != G;
    const bool is_spec = spec_on && b == Gp;
    double* const spec_blk = spec_on ? partials + (size_t)Gp * NACC_MAX + SPEC_OFF : nullptr;

    // the member model is a template parameter: the circular fit (the
    // minor cycle's) carries no branch of the other two
    constexpr bool ell = MODEL == 1, mch = MODEL == 2;
    const int NCH = mch ? d.n_chan : 1;   // channels of a joint fit
    const int NPM = ell ? 6 : mch ? 3 + NCH : 4;   // parameters per member
    const int K = d.K, P = NPM * K, NA = P + 1, NAp = (NA + 3) & ~3, nb = NAp / 4;
    const int ntiles = nb * (nb + 1) / 2;
    const int nacc = ntiles * 16;
    // a joint fit runs over the window of every channel, channel after channel
    const long long Wn1 = (long long)d.ww * d.wh, Wn = Wn1 * NCH;
    const long long s0 = is_spec ? Wn : Wn * b / Gp, s1 = is_spec ? Wn : Wn * (b + 1) / Gp;
    const int slen = (int)(s1 - s0);
    const bool in_smem = d.smem_ok != 0;
    // J rows: stride of an odd number of float4s, so the row-per-thread
    // stores of phase A hit distinct bank groups
    const int JS = (nb & 1) ? NAp : NAp + 4;
    const int CH = LARGE ? CH_XL : min(NAp <= 64 ? CH_SMALL : CH_LARGE, JC_FLOATS / JS);
    const int chi_idx = acc_index(P, P, nb);

    // ---- tile table and thread -> (tile, group) assignment
    for (int t = tid; t < ntiles; t += blockDim.x) {
        int bi = 0, rem = t;
        while (rem >= nb - bi) { rem -= nb - bi; ++bi; }
        ttab[t] = make_short2((short)bi, (short)(bi + rem));
    }
    // SYRK thread order: column blocks of 8 tile columns, rows ascending
    // within a block, so the 32 lanes of a warp cover about 4 tile rows x 8
    // tile columns and each pixel's two float4 J loads of a warp touch ~12
    // distinct float4 (2 shared-memory wavefronts instead of ~5 in row order)
    for (int t = tid; t < ntiles; t += blockDim.x) {
        int k = t, c0 = 0, c1 = 0, full = 0, nfull = 0;
        for (int C = 0;; ++C) {
            c0 = 8 * C;
            c1 = min(c0 + 7, nb - 1);
            full = c1 - c0 + 1;                    // rows 0..c0 span the block's full width
            nfull = c0 + 1;
            const int cnt = nfull * full + (full - 1) * full / 2;   // rows c0+1..c1: widths full-1..1
            if (k < cnt) break;
            k -= cnt;
        }
        int bi, bj;
        if (k < nfull * full) {
            bi = k / full;
            bj = c0 + k % full;
        } else {
            k -= nfull * full;
            int w = full - 1;
            bi = c0 + 1;
            while (k >= w) { k -= w; --w; ++bi; }
            bj = bi + k;
        }
        tperm[t] = (short)tile_index(bi, bj, nb);
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

    // joint fits: per (member, channel) amplitude and 1 / omega_kc^2, FP32,
    // in the step buffer's storage (free from the end of a solve loop to the
    // next solve)
    float* const mc_a = reinterpret_cast<float*>(delta);
    float* const mc_iw2 = mc_a + PMAX;

    // ---- stage the target T = src + sum of the added-back members
    if (tid < K) {
        if (ell) make_frame_ell(&d.theta0[NPM * tid], fr[tid]);
        else if (mch) make_frame_mc(&d.theta0[NPM * tid], fr[tid]);
        else make_frame(&d.theta0[NPM * tid], fr[tid]);
    }
    if (mch && tid < K * NCH) {
        const int k = tid / NCH, c = tid - k * NCH;
        const double sk = d.theta0[NPM * k + 2];
        mc_iw2[tid] = (float)(1.0 / (sk * sk + d.chan_wb2[c]));
        mc_a[tid] = (float)d.theta0[NPM * k + 3 + c];
    }
    __syncthreads();
    for (int i = tid; i < slen; i += blockDim.x) {
        long long gi = s0 + i;
        int ch = 0;
        if (mch) { ch = (int)(gi / Wn1); gi -= (long long)ch * Wn1; }
        int y = d.wy0 + (int)(gi / d.ww), x = d.wx0 + (int)(gi % d.ww);
        float v = mch ? d.chan_src[ch][(long long)y * src_w + x] : src[(long long)y * src_w + x];
        for (int m = K - d.n_old; m < K; ++m) {
            const MemberFrame& f = fr[m];
            float dx = (float)(x - f.cx) - f.fx, dy = (float)(y - f.cy) - f.fy;
            if (mch) {
                const int q = m * NCH + ch;
                v += mc_a[q] * exp2f(-(dx * dx + dy * dy) * (0.5f * (float)LOG2E) * mc_iw2[q]);
            } else {
                v += f.a * exp2f(ell ? -((f.c * dx + f.cb * dy) * dx + f.cc * dy * dy) : -(dx * dx + dy * dy) * f.c);
            }
        }
        if (in_smem) Ts[i] = v; else Tg[gi] = v;
    }
    const bool has_start = descp->has_start != 0;
    if (tid == 0) {
        for (int i = 0; i < P; ++i) theta[i] = has_start ? descp->start[i] : d.theta0[i];
        s_lam = lmc.lambda0; s_cur = 0; s_iters = 0; s_passes = 0; s_status = ASP_LM_CAP;
        s_done = 0; s_err = 0; s_flag = 0; s_use_spec = 0; s_small = 0;
        sw.refinements = 0; sw.fallbacks = 0;
    }
    for (int i = tid; i < P; i += blockDim.x) trial[i] = has_start ? descp->start[i] : d.theta0[i];
    __syncthreads();

    // phase A's threads per pixel row (circular members): the members of a
    // pixel split over TPP adjacent lanes, a power of two (at most 8) with
    // TPP times the rows a chunk holds (the slice's, if it is shorter than
    // a chunk) within the block, so narrow chunks and short slices keep the
    // threads busy
    int TPP = 1;
    if (!ell && !mch) {
        const int rows = max(1, min(CH, slen));   // rows a chunk of this slice fills
        while (rows * TPP * 2 <= (int)blockDim.x && TPP < 8) TPP *= 2;
    }
    const int lpix = tid / TPP, lq = tid - lpix * TPP;   // this thread's row and member offset
    // pixel coordinates of this thread's J row in the first chunk (the only
    // chunk when the slice fits one), computed once for all passes
    int x_first = 0, y_first = 0, c_first = 0;
    if (lpix < CH && lpix < slen) {
        long long gi = s0 + lpix;
        if (mch) { c_first = (int)(gi / Wn1); gi -= (long long)c_first * Wn1; }
        y_first = d.wy0 + (int)(gi / d.ww);
        x_first = d.wx0 + (int)(gi % d.ww);
    }

    unsigned epoch = 0;
    int npass = 0;
    bool first = true;
    // phase clocks (CTA 0, thread 0): pass, CTA + cross-CTA reduction, LM logic + solves
    unsigned long long t_pass = 0, t_red = 0, t_solve = 0, t_factor = 0, t_subst = 0, t0 = gtimer(), t1;
    while (true) {
        // ================= pixel pass at trial[] =================
        if (tid < K) {
            if (ell) make_frame_ell(&trial[NPM * tid], fr[tid]);
            else if (mch) make_frame_mc(&trial[NPM * tid], fr[tid]);
            else make_frame(&trial[NPM * tid], fr[tid]);
        }
        if (mch && tid < K * NCH) {
            const int k = tid / NCH, c = tid - k * NCH;
            const double sk = trial[NPM * k + 2];
            mc_iw2[tid] = (float)(1.0 / (sk * sk + d.chan_wb2[c]));
            mc_a[tid] = (float)trial[NPM * k + 3 + c];
        }
        if (tid == (int)blockDim.x - 1 && !first) {
            // the LM decision's FP64 arithmetic (a division among it), done
            // here by a thread without a J row so that it stays off the
            // critical path: lambda after an accepted or rejected step and
            // the flatness threshold rtol chi^2
            s_lam_acc = fmax(s_lam / lmc.lambda_down, lmc.lambda_min);
            s_lam_rej = s_lam * lmc.lambda_up;
            s_rej_stall = s_lam_rej > lmc.lambda_max;
            s_thr = lmc.rtol * s_chi2;
        }
        if (spec_on && b == 0 && tid == (int)blockDim.x - 1) {
            // the LM state the decision after this pass reads, for the
            // speculating CTA (which did not see this fit's solves)
            double* bc = spec_blk + (npass & 1) * SPEC_BC;
            bc[0] = s_lam; bc[1] = s_lam_acc; bc[2] = s_lam_rej; bc[3] = s_rej_stall;
            bc[4] = s_small; bc[5] = 0.0;
        }
        __syncthreads();
        const int nxt = 1 - s_cur;
        double* sums_nxt = sums + (size_t)nxt * NACC_MAX;
        // this pass's chi^2 partials: buffers alternate, so a CTA's write two
        // passes on follows every CTA's read (a grid barrier lies between)
        float2* chib_p = chib + (npass & 1) * FIT_GRID_MAX;
        const int chi_t = chi_idx >> 4, chi_e = chi_idx & 15;
        ++npass;
        float* sums32_nxt = sums32 + (size_t)nxt * NACC_MAX;
        // the tiles in rounds of TPT per thread (one round unless the active
        // set is large), re-evaluating the J rows each round
        const int tiles_per_round = TPT * (int)blockDim.x;
        const int n_rounds = n_groups == 1 ? (ntiles + tiles_per_round - 1) / tiles_per_round : 1;
        for (int round = 0; round < n_rounds; ++round) {
        const int tbase = my_tile0 + round * tiles_per_round;
        float acc[TPT][16], ks[TPT][16], kc[TPT][16];
#pragma unroll
        for (int q = 0; q < TPT; ++q)
#pragma unroll
            for (int e = 0; e < 16; ++e) { acc[q][e] = 0.f; ks[q][e] = 0.f; kc[q][e] = 0.f; }

        for (int c0 = 0; c0 < slen; c0 += CH) {
            const int cn = min(CH, slen - c0);
            // phase A: one pixel row of [J | r] per TPP threads
            if (lpix < CH) {
                float* row = Jc + lpix * JS;
                bool live = lpix < cn;
                int x = 0, y = 0, ch = 0;
                if (live) {
                    if (c0 == 0) {
                        x = x_first;
                        y = y_first;
                        ch = c_first;
                    } else {
                        long long gi = s0 + c0 + lpix;
                        if (mch) { ch = (int)(gi / Wn1); gi -= (long long)ch * Wn1; }
                        y = d.wy0 + (int)(gi / d.ww);
                        x = d.wx0 + (int)(gi % d.ww);
                    }
                    if (d.use_mask) {
                        double ddx = x - d.mcx, ddy = y - d.mcy;
                        live = ddx * ddx + ddy * ddy <= d.mr2;
                    }
                }
                if (live && mch) {
                    // joint members in channel ch: d/dx = g dx / w^2,
                    // d/dy = g dy / w^2, d/ds = g r^2 s / w^4, d/da_k,ch = E;
                    // every other channel's amplitude column is zero
                    for (int c = 0; c < NAp; ++c) row[c] = 0.f;
                    float model = 0.f;
                    for (int k = 0; k < K; ++k) {
                        const MemberFrame& f = fr[k];
                        const int q = k * NCH + ch;
                        const float dx = (float)(x - f.cx) - f.fx, dy = (float)(y - f.cy) - f.fy;
                        const float r2 = dx * dx + dy * dy, iw2 = mc_iw2[q];
                        const float e = exp2f(-r2 * (0.5f * (float)LOG2E) * iw2);
                        const float g = mc_a[q] * e, giw = g * iw2;
                        model += g;
                        float* rk = row + NPM * k;
                        rk[0] = giw * dx;
                        rk[1] = giw * dy;
                        rk[2] = giw * r2 * f.pa * iw2;
                        rk[3 + ch] = e;
                    }
                    float t = in_smem ? Ts[c0 + lpix] : Tg[s0 + c0 + lpix];
                    row[P] = t - model;
                } else if (live && ell) {
                    // elliptical members: d/da = E, d/dx0 = g (A dx + B dy),
                    // d/dy0 = g (B dx + C dy), d/dA = -g dx^2 / 2,
                    // d/dB = -g dx dy, d/dC = -g dy^2 / 2
                    float model = 0.f;
#pragma unroll 2
                    for (int k = 0; k < K; ++k) {
                        const MemberFrame& f = fr[k];
                        const float dx = (float)(x - f.cx) - f.fx, dy = (float)(y - f.cy) - f.fy;
                        const float e = exp2f(-((f.c * dx + f.cb * dy) * dx + f.cc * dy * dy));
                        const float g = f.a * e, hg = -0.5f * g;
                        model += g;
                        float2* r2p = reinterpret_cast<float2*>(row + 6 * k);
                        r2p[0] = make_float2(e, g * (f.pa * dx + f.pb * dy));
                        r2p[1] = make_float2(g * (f.pb * dx + f.pc * dy), hg * dx * dx);
                        r2p[2] = make_float2(-g * dx * dy, hg * dy * dy);
                    }
                    float t = in_smem ? Ts[c0 + lpix] : Tg[s0 + c0 + lpix];
                    row[P] = t - model;
                    for (int c = P + 1; c < NAp; ++c) row[c] = 0.f;
                } else if (live) {
                    // members lq, lq + TPP, ...; the TPP partial model sums
                    // meet in a butterfly over the row's lanes (every lane
                    // ends with the same value)
                    float model = 0.f;
#pragma unroll 4
                    for (int k = lq; k < K; k += TPP) {
                        const MemberFrame& f = fr[k];
                        float dx = (float)(x - f.cx) - f.fx, dy = (float)(y - f.cy) - f.fy;
                        float r2 = dx * dx + dy * dy;
                        float e = exp2f(-r2 * f.c);
                        float g = f.a * e;
                        model += g;
                        float4 jr = make_float4(e, g * dx * f.iw2, g * dy * f.iw2, g * r2 * f.iw3);
                        *reinterpret_cast<float4*>(row + 4 * k) = jr;
                    }
                    if (TPP > 1) {
                        const unsigned gm = ((1u << TPP) - 1u) << ((tid & 31) & ~(TPP - 1));
                        for (int o = TPP >> 1; o > 0; o >>= 1) model += __shfl_xor_sync(gm, model, o);
                    }
                    if (lq == 0) {
                        float t = in_smem ? Ts[c0 + lpix] : Tg[s0 + c0 + lpix];
                        row[P] = t - model;
                        for (int c = P + 1; c < NAp; ++c) row[c] = 0.f;
                    }
                } else {
                    for (int c = lq; c < NAp; c += TPP) row[c] = 0.f;
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
                        const int t = tbase + q * (int)blockDim.x;
                        if (t < ntiles) {
                            const short2 bij = ttab[tperm[t]];
                            // unrolled so the next pixels' loads issue ahead of the FMAs
#pragma unroll 4
                            for (int l = l0; l < l1; ++l) {
                                const float4 av = *reinterpret_cast<const float4*>(Jc + l * JS + 4 * bij.x);
                                const float4 bv = *reinterpret_cast<const float4*>(Jc + l * JS + 4 * bij.y);
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

        // ---- CTA total of each accumulator entry of this round
        // CTA partials stay FP32 pairs (hi, lo) = (Kahan sum, -compensation):
        // every FP64 operation or conversion costs the narrow FP64 pipe;
        // only a single-CTA fit writes its FP64 sums here
        if (is_spec) {
            // no pixels, no partial sums
        } else if (n_groups == 1) {
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                const int t = tbase + q * (int)blockDim.x;
                if (my_group == 0 && t < ntiles) {
                    const int slot = tperm[t];                // layout position of this tile
                    if (G == 1) {
                        double* dst = sums_nxt + slot * 16;
                        float* dst32 = sums32_nxt + slot * 16;
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            dst[e] = (double)ks[q][e] - (double)kc[q][e];
                            dst32[e] = ks[q][e] - kc[q][e];
                        }
                    } else {
                        float2* dst = reinterpret_cast<float2*>(partials + (size_t)b * NACC_MAX) + slot * 16;
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            dst[e] = make_float2(ks[q][e], -kc[q][e]);
                            if (slot == chi_t && e == chi_e) chib_p[b] = make_float2(ks[q][e], -kc[q][e]);
                        }
                    }
                }
            }
        } else if (my_group >= 0) {
            // several pixel groups per tile: park each group's leaf sums at
            // the tile's layout position, 17 floats per tile so that the
            // lanes' stores of one entry fall in distinct banks
            const int slot = tperm[my_tile0];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                red[(my_group * ntiles + slot) * 17 + e] = ks[0][e];
                red[(n_groups * ntiles + my_group * ntiles + slot) * 17 + e] = kc[0][e];
            }
        }
        }   // rounds
        t1 = gtimer(); t_pass += t1 - t0; t0 = t1;
        if (n_groups > 1 && !is_spec) {
            // the pixel groups' pairs combined error-free in FP32, in group order
            // (entry e = 16 slot + q of group g parked at (g ntiles + slot) 17 + q)
#define RS(g, e) red[((g) * ntiles + ((e) >> 4)) * 17 + ((e) & 15)]
#define RC(g, e) red[((n_groups + (g)) * ntiles + ((e) >> 4)) * 17 + ((e) & 15)]
            __syncthreads();
            for (int e = tid; e < nacc; e += blockDim.x) {
                // up to 4 groups in order; more as four chains (group g in
                // chain g % 4) joined pairwise
                float sh = 0.f, sl = 0.f;
                if (n_groups <= 4) {
                    for (int g = 0; g < n_groups; ++g) pair_add(sh, sl, RS(g, e), -RC(g, e));
                } else {
                    float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f, h3 = 0.f, l3 = 0.f;
                    int g = 0;
                    for (; g + 3 < n_groups; g += 4) {
                        pair_add(sh, sl, RS(g, e), -RC(g, e));
                        pair_add(h1, l1, RS(g + 1, e), -RC(g + 1, e));
                        pair_add(h2, l2, RS(g + 2, e), -RC(g + 2, e));
                        pair_add(h3, l3, RS(g + 3, e), -RC(g + 3, e));
                    }
                    for (; g < n_groups; ++g) pair_add(sh, sl, RS(g, e), -RC(g, e));
                    pair_add(sh, sl, h1, l1);
                    pair_add(h2, l2, h3, l3);
                    pair_add(sh, sl, h2, l2);
                }
                if (G == 1) { sums_nxt[e] = (double)sh + (double)sl; sums32_nxt[e] = sh + sl; }
                else {
                    reinterpret_cast<float2*>(partials + (size_t)b * NACC_MAX)[e] = make_float2(sh, sl);
                    if (e == chi_idx) chib_p[b] = make_float2(sh, sl);
                }
            }
#undef RS
#undef RC
        }

        // ---- chi^2 at the trial point first: after a grid barrier every CTA
        // combines the CTAs' chi^2 pairs (fixed order -> identical everywhere)
        if (G > 1) {
            ++epoch;
            grid_barrier(bar, epoch * (unsigned)G, &s_err, &out->error);
            if (s_err) return;
            if (tid < 32) {
                // lane l combines CTAs l, l + 32, ... (all loads in flight first)
                float h = 0.f, l = 0.f;
                for (int cb = tid; cb < Gp; cb += 8 * 32) {
                    float2 v[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int c = cb + 32 * k;
                        v[k] = c < Gp ? __ldcg(chib_p + c) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) pair_add(h, l, v[k].x, v[k].y);
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    const float hh = __shfl_down_sync(0xffffffffu, h, o);
                    const float ll = __shfl_down_sync(0xffffffffu, l, o);
                    pair_add(h, l, hh, ll);
                }
                if (tid == 0) s_chi2_t = (double)h + (double)l;
            }
        } else if (tid == 0) {
            s_chi2_t = 0.0;
        }
        __syncthreads();
        if (G == 1 && tid == 0) s_chi2_t = sums_nxt[chi_idx];
        if (is_spec && tid == 0) {
            const double* bc = spec_blk + ((npass - 1) & 1) * SPEC_BC;
            s_lam = __ldcg(bc + 0); s_lam_acc = __ldcg(bc + 1); s_lam_rej = __ldcg(bc + 2);
            s_rej_stall = __ldcg(bc + 3) != 0.0; s_small = __ldcg(bc + 4) != 0.0;
            s_thr = lmc.rtol * s_chi2;
            if (__ldcg(bc + 5) != 0.0) s_done = 1;    // the fit ended in the pixel CTAs' solve loop
        }
        if (is_spec) {
            __syncthreads();
            if (s_done) break;
        }
        // ================= LM decision (identical in every CTA) =================
        if (tid == 0) {
            const double chi2_t = s_chi2_t;                      // FP64 acceptance test
            s_passes += 1;
            s_acc = 0;
            if (first) {
                s_cur = nxt;
                s_chi2 = chi2_t;
                s_chi2_init = chi2_t;
            } else if (chi2_t < s_chi2) {
                // relative decrease below rtol: (chi2 - chi2_t) < rtol chi2
                const bool flat = !(s_chi2 - chi2_t >= s_thr) || !(s_chi2 > 0.0);
                s_acc = 1;
                s_cur = nxt;
                s_chi2 = chi2_t;
                s_lam = s_lam_acc;
                if (flat || s_small) { s_status = ASP_LM_CONVERGED; s_done = 1; }
            } else {
                s_lam = s_lam_rej;
                if (s_rej_stall) { s_status = ASP_LM_STALLED; s_done = 1; }
            }
            // a rejected trial asks for the step at the new lambda on the same
            // A: the speculating CTA solved it during this pass
            s_use_spec = 0;
            if (spec_on && !is_spec && !first && !s_acc && !s_done) {
                const double* st = spec_blk + 2 * SPEC_BC + ((npass - 1) & 1) * SPEC_STEP;
                s_use_spec = __ldcg(st + 0) == s_lam && __ldcg(st + 1) != 0.0;
            }
        }
        __syncthreads();
        // ---- the full cross-CTA reduction, only when the point moves (a
        // rejected step keeps the current point's sums)
        if (G > 1 && s_cur == nxt) {
            // T lanes per entry (a power of two <= 32 and <= G, as many as the
            // grid's threads allow): lane (e_local, s) of a warp holds entry
            // e0 + e_local and combines the CTAs s, s + T, ... as four FP32
            // pair chains; the T lanes' pairs then meet in a fixed shuffle
            // tree.  Same order in every CTA and every launch.
            const int nwarp = (int)blockDim.x >> 5, lane = tid & 31;
            int T = 1;
            while (T < 32 && 2 * T <= Gp && (long long)G * (int)blockDim.x >= (long long)nacc * 2 * T) T *= 2;
            const int E = 32 / T;
            const int el = lane & (E - 1), s0 = lane / E;
            const float2* pbase = reinterpret_cast<const float2*>(partials);
            const size_t stride = NACC_MAX;   // a partial row: NACC_MAX doubles = NACC_MAX float2
            for (int e0 = (b * nwarp + (tid >> 5)) * E; e0 < nacc; e0 += G * nwarp * E) {
                const int e = e0 + el;
                float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f, h3 = 0.f, l3 = 0.f;
                if (e < nacc) {
                    // batches of RB loads in flight, then four pair chains
                    // (chain k % 4); absent CTAs load nothing and add zero
                    constexpr int RB = 16;
                    const float2* pe = pbase + e;
                    for (int cb = s0; cb < Gp; cb += RB * T) {
                        float2 v[RB];
#pragma unroll
                        for (int k = 0; k < RB; ++k) {
                            const int c = cb + k * T;
                            v[k] = c < Gp ? __ldcg(pe + (size_t)c * stride) : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int k = 0; k < RB; k += 4) {
                            pair_add(h0, l0, v[k].x, v[k].y);
                            pair_add(h1, l1, v[k + 1].x, v[k + 1].y);
                            pair_add(h2, l2, v[k + 2].x, v[k + 2].y);
                            pair_add(h3, l3, v[k + 3].x, v[k + 3].y);
                        }
                    }
                    pair_add(h0, l0, h1, l1);
                    pair_add(h2, l2, h3, l3);
                    pair_add(h0, l0, h2, l2);
                }
                for (int o = 16; o >= E; o >>= 1) {
                    const float hh = __shfl_down_sync(0xffffffffu, h0, o);
                    const float ll = __shfl_down_sync(0xffffffffu, l0, o);
                    pair_add(h0, l0, hh, ll);
                }
                if (s0 == 0 && e < nacc) {
                    sums_nxt[e] = (double)h0 + (double)l0;
                    sums32_nxt[e] = h0 + l0;      // the FP64 sum rounded to FP32
                }
            }
            ++epoch;
            grid_barrier(bar, epoch * (unsigned)G, &s_err, &out->error);
            if (s_err) return;
        }
        t1 = gtimer(); t_red += t1 - t0; t0 = t1;
        __syncthreads();
        if (s_acc && tid < P) theta[tid] = trial[tid];
        first = false;
        __syncthreads();
        // the current point moved (first pass or accepted step): variant S
        // copies its sums (FP64 and FP32, tile order) to shared memory, a
        // flat batched copy; both cache g, diag A and the Marquardt diagonal
        if (s_cur == nxt) {
            const double* sc = sums + (size_t)s_cur * NACC_MAX;
            const float* sc32 = sums32 + (size_t)s_cur * NACC_MAX;
            if (tid == (int)blockDim.x - 1) s_thr32 = (float)(lmc.rtol * s_chi2);   // for the post-solve test
            if (!LARGE) {
#pragma unroll 4
                for (int e = tid; e < nacc; e += blockDim.x) {
                    Ac[e] = __ldcg(sc + e);
                    Ac32[e] = __ldcg(sc32 + e);
                }
                __syncthreads();
            }
            const double* ad = LARGE ? sc : Ac;
            const float* af = LARGE ? sc32 : Ac32;
            for (int i = tid; i < P; i += blockDim.x) {
                const int qg = acc_index(i, P, nb), qd = acc_index(i, i, nb);
                gvec[i] = LARGE ? __ldcg(ad + qg) : ad[qg];
                g32[i] = LARGE ? __ldcg(af + qg) : af[qg];
                const double dd = LARGE ? __ldcg(ad + qd) : ad[qd];
                const float dd32 = LARGE ? __ldcg(af + qd) : af[qd];
                dvec[i] = dd > 0.0 ? dd : 1.0;
                a32d[i] = dd32;
                dv32[i] = dd32 > 0.f ? dd32 : 1.f;
            }
            __syncthreads();
        }

        // ---- the speculating CTA: the step at lambda_up x lambda on the
        // current A (what a rejected trial asks for next), published before
        // it meets the others at the next pass's barrier
        if (is_spec) {
            if (s_done) break;
            const double lam_s = s_lam * lmc.lambda_up;
            const bool ok =
                LARGE ? solve_damped(TileA{sums + (size_t)s_cur * NACC_MAX, nb},
                                     TiledA32{sums32 + (size_t)s_cur * NACC_MAX, ttab, a32d, nacc, true}, gvec, g32,
                                     dvec, dv32, lam_s, P, Jc, partials + (size_t)b * NACC_MAX, sw, delta)
                      : solve_damped(SmemTileA{Ac, nb}, TiledA32{Ac32, ttab, a32d, nacc, false}, gvec, g32, dvec,
                                     dv32, lam_s, P, Jc, partials + (size_t)b * NACC_MAX, sw, delta);
            double* st = spec_blk + 2 * SPEC_BC + (npass & 1) * SPEC_STEP;
            for (int i = tid; i < P; i += blockDim.x) st[2 + i] = delta[i];
            if (tid == 0) { st[0] = lam_s; st[1] = ok ? 1.0 : 0.0; }
            __syncthreads();
            continue;
        }
        // ---- propose the next trial point (solves without a pass loop here)
        const int done_before = s_done;
        while (!s_done) {
            if (tid == 0) {
                if (s_iters >= lmc.max_iter) { s_status = ASP_LM_CAP; s_done = 1; }
                s_pred[0] = 0.f;       // cleared here: the solve's barriers order them before the checks
                s_pred[1] = 0.f;
                s_flags = 7u;
            }
            __syncthreads();
            if (s_done) break;
            const double lam = s_lam;
            const unsigned long long tf0 = gtimer();
            bool ok;
            // the FP64 fallback factor goes to this CTA's partial row (consumed
            // by the reduction, rewritten by the next pass)
            if (s_use_spec) {
                // after a rejected trial: the speculating CTA's step at this lambda
                const double* st = spec_blk + 2 * SPEC_BC + ((npass - 1) & 1) * SPEC_STEP;
                for (int i = tid; i < P; i += blockDim.x) delta[i] = __ldcg(st + 2 + i);
                ok = true;
                __syncthreads();
                if (tid == 0) s_use_spec = 0;
            } else if (LARGE)
                ok = solve_damped(TileA{sums + (size_t)s_cur * NACC_MAX, nb},
                                  TiledA32{sums32 + (size_t)s_cur * NACC_MAX, ttab, a32d, nacc, true}, gvec, g32,
                                  dvec, dv32, lam, P, Jc,
                                  partials + (size_t)b * NACC_MAX, sw, delta);
            else
                ok = solve_damped(SmemTileA{Ac, nb}, TiledA32{Ac32, ttab, a32d, nacc, false}, gvec, g32, dvec, dv32, lam, P, Jc,
                                  partials + (size_t)b * NACC_MAX, sw, delta);
            const unsigned long long tf1 = gtimer();
            t_factor += tf1 - tf0;
            // predicted decrease d.g + lam d.D.d (FP32 sums), finiteness, validity
            int fin_i = 1, valid_i = 1, small_i = 1;
            float dg_i = 0.f, dd_i = 0.f;
            if (ok && tid < P) {
                const double di = delta[tid];
                fin_i = isfinite(di);
                // every step below xtol of its scale: |a|; w for centre and
                // width (circular); the major width for the centre and
                // (A + C) / 2 for A, B, C (elliptical)
                double sc;
                if (mch) {
                    // the widest convolved width for x, y, s; |a| for amplitudes
                    const int j = tid % NPM, base = tid - j;
                    sc = j < 3 ? sqrt(theta[base + 2] * theta[base + 2] + d.max_wb2) : fabs(theta[tid]);
                } else if (ell) {
                    const int j = tid % 6, base = tid - j;
                    if (j == 0) {
                        sc = fabs(theta[tid]);
                    } else {
                        const double A = theta[base + 3], C = theta[base + 5];
                        double mm, mp;
                        prec_eig(A, theta[base + 4], C, mm, mp);
                        sc = j <= 2 ? 1.0 / sqrt(mm) : 0.5 * (A + C);
                    }
                } else {
                    sc = (tid & 3) == 0 ? fabs(theta[tid]) : theta[(tid & ~3) + 3];
                }
                if (sc == 0.0) sc = 1.0;
                small_i = fabs(di) < lmc.xtol * sc;
                const float df = (float)di;
                dg_i = df * g32[tid];
                dd_i = dv32[tid] * df * df;
                trial[tid] = theta[tid] + di;
            }
            if (ok && tid < K && mch) {
                // centre in the box, every convolved width within the window
                const int o = NPM * tid;
                const double x = theta[o] + delta[o], y = theta[o + 1] + delta[o + 1], sv = theta[o + 2] + delta[o + 2];
                valid_i = isfinite(x) && isfinite(y) && isfinite(sv) && !(x < d.bx0) && !(x > d.bx1) &&
                          !(y < d.by0) && !(y > d.by1) && !(sv * sv + d.max_wb2 > d.omega_max * d.omega_max);
            } else if (ok && tid < K && ell) {
                // positive definite, principal widths 1 / sqrt(mu) in
                // (omega_min, omega_max], centre in the box
                const int o = 6 * tid;
                const double a = theta[o] + delta[o], x = theta[o + 1] + delta[o + 1], y = theta[o + 2] + delta[o + 2];
                const double A = theta[o + 3] + delta[o + 3], B = theta[o + 4] + delta[o + 4];
                const double C = theta[o + 5] + delta[o + 5];
                double mm, mp;
                prec_eig(A, B, C, mm, mp);
                valid_i = isfinite(a) && isfinite(x) && isfinite(y) && isfinite(A) && isfinite(B) && isfinite(C) &&
                          !(x < d.bx0) && !(x > d.bx1) && !(y < d.by0) && !(y > d.by1) && mm > 0.0 &&
                          mp < 1.0 / (d.omega_min * d.omega_min) && mm >= 1.0 / (d.omega_max * d.omega_max);
            } else if (ok && tid < K) {
                const double a = theta[4 * tid] + delta[4 * tid];
                const double x = theta[4 * tid + 1] + delta[4 * tid + 1];
                const double y = theta[4 * tid + 2] + delta[4 * tid + 2];
                const double w = theta[4 * tid + 3] + delta[4 * tid + 3];
                valid_i = (w > d.omega_min) && !(w > d.omega_max) && isfinite(a) && isfinite(x) && isfinite(y) &&
                          isfinite(w) && !(x < d.bx0) && !(x > d.bx1) && !(y < d.by0) && !(y > d.by1);
            }
            if ((tid & ~31) < P) {          // whole warps holding parameters (zeros beyond P)
                for (int o = 16; o > 0; o >>= 1) {
                    dg_i += __shfl_xor_sync(0xffffffffu, dg_i, o);
                    dd_i += __shfl_xor_sync(0xffffffffu, dd_i, o);
                }
                if ((tid & 31) == 0) { atomicAdd(&s_pred[0], dg_i); atomicAdd(&s_pred[1], dd_i); }
            }
            // the three block-wide ANDs in one barrier: warp AND, then a shared atomic
            {
                unsigned f = (fin_i ? 1u : 0u) | (valid_i ? 2u : 0u) | (small_i ? 4u : 0u);
                f = __reduce_and_sync(0xffffffffu, f);
                if ((tid & 31) == 0) atomicAnd(&s_flags, f);
            }
            const float lam32 = tid == 0 ? (float)lam : 0.f;   // the test below runs on thread 0
            __syncthreads();
            const int fin = (s_flags & 1u) && ok;
            const int valid = (s_flags & 2u) != 0u;
            const int small = (s_flags & 4u) != 0u;
            if (tid == 0) {
                s_iters += 1;
                s_go = 0;
                if (!fin) {
                    s_lam *= lmc.lambda_up;
                    if (s_lam > lmc.lambda_max) { s_status = ASP_LM_STALLED; s_done = 1; }
                } else if (fmaf(lam32, s_pred[1], s_pred[0]) <= s_thr32) {   // FP32 sums against FP32 rtol chi^2
                    s_status = ASP_LM_CONVERGED; s_done = 1;
                } else if (valid) {
                    s_go = 1;
                    s_small = small;
                } else {
                    s_lam *= lmc.lambda_up;
                    if (s_lam > lmc.lambda_max) { s_status = ASP_LM_STALLED; s_done = 1; }
                }
            }
            __syncthreads();
            t_subst += gtimer() - tf1;
            if (s_go) break;
        }
        __syncthreads();
        t1 = gtimer(); t_solve += t1 - t0; t0 = t1;
        if (s_done) {
            if (spec_on && !done_before) {
                // the fit ended in the solve loop: the speculating CTA waits at
                // the next pass's barrier and learns it there
                if (b == 0 && tid == 0) spec_blk[(npass & 1) * SPEC_BC + 5] = 1.0;
                ++epoch;
                grid_barrier(bar, epoch * (unsigned)G, &s_err, &out->error);
                if (s_err) return;
            }
            break;
        }
    }

    if (b == 0 && tid == 0) {
        out->ns_pass = (long long)t_pass;
        out->ns_reduce = (long long)t_red;
        out->ns_solve = (long long)t_solve;
        out->ns_factor = (long long)t_factor;
        out->ns_subst = (long long)t_subst;
        out->refinements = sw.refinements;
        out->fallbacks = sw.fallbacks;
        for (int i = 0; i < P; ++i) out->theta[i] = theta[i];
        out->chi2_init = s_chi2_init;
        out->chi2 = s_chi2;
        out->lambda = s_lam;
        out->iters = s_iters;
        out->passes = s_passes;
        out->status = s_status;
        out->pixel_evals = (long long)s_passes * Wn;
        for (int i = 0; i < P; ++i) out->trial[i] = trial[i];
        out->chi2_trial = s_chi2_t;
    }
}

// MODEL: 0 circular members (the minor cycle), 1 elliptical, 2 joint over
// channels (FitDescHead.model must agree); models 1 and 2 are instantiated
// in asp_fit_models.cu.
template <int TPT, bool LARGE, int MODEL>
__global__ void __launch_bounds__(FIT_THREADS, 1)
k_lm_fit(const float* __restrict__ src, int src_w, const FitDesc* __restrict__ descp, const __grid_constant__ LMConst lmc,
         FitOut* __restrict__ out, double* __restrict__ partials, double* __restrict__ sums,
         unsigned* __restrict__ bar, float* __restrict__ Tg) {
    lm_fit_body<TPT, LARGE, MODEL>(src, src_w, descp, lmc, out, partials, sums, bar, Tg, blockIdx.x);
}

// Two fits of one image side by side in one cooperative launch: CTAs
// [0, GA) run fit A (the learned start), [GA, GA + GB) fit B (the plain
// start), each with its own partials, sums, barrier counter and target
// buffer; G = 0 for an inactive fit.
template <int TPT, bool LARGE>
__global__ void __launch_bounds__(FIT_THREADS, 1)
k_lm_fit_pair(const float* __restrict__ src, int src_w, const __grid_constant__ LMConst lmc,
              const FitDesc* __restrict__ dA, FitOut* __restrict__ oA, double* __restrict__ pA, double* __restrict__ sA,
              unsigned* __restrict__ bA, float* __restrict__ tA, const FitDesc* __restrict__ dB,
              FitOut* __restrict__ oB, double* __restrict__ pB, double* __restrict__ sB, unsigned* __restrict__ bB,
              float* __restrict__ tB) {
    const int GA = dA->active ? dA->grid : 0;
    const int GB = dB->active ? dB->grid : 0;
    const int c = (int)blockIdx.x;
    if (c < GA) lm_fit_body<TPT, LARGE, 0>(src, src_w, dA, lmc, oA, pA, sA, bA, tA, c);
    else if (c - GA < GB) lm_fit_body<TPT, LARGE, 0>(src, src_w, dB, lmc, oB, pB, sB, bB, tB, c - GA);
}

// Batched: the fits of many images in one cooperative launch of g_total
// CTAs.  Image i owns CTAs [dmap[i], dmap[i+1]) (written on the device each
// iteration by k_fit_map_b); each group runs its own fit with its own
// barrier counter, partials and sums; CTAs beyond dmap[n] return.
template <int TPT, bool LARGE>
__global__ void __launch_bounds__(FIT_THREADS, 1)
k_lm_fit_b(const ImgDesc* __restrict__ imgs, const int* __restrict__ dmap, int n, int which, int max_iter_override) {
    const int c = (int)blockIdx.x;
    if (c >= dmap[n]) return;
    int lo = 0, hi = n - 1;                 // image i with dmap[i] <= c < dmap[i+1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (dmap[mid] <= c) lo = mid; else hi = mid - 1;
    }
    const ImgDesc& g = imgs[lo];
    // which = 1: the second fit (learned initial values: chi^2 at the plain
    // start, the fallback refit)
    LMConst lmc = g.dp.lm;
    if (max_iter_override >= 0) lmc.max_iter = max_iter_override;
    lm_fit_body<TPT, LARGE, 0>(g.R, g.W, which ? &g.st->fit2 : &g.st->fit, lmc, which ? &g.st->fout2 : &g.st->fout,
                            g.partials, g.sums, g.bar, g.Tg, c - dmap[lo]);
}

}  // namespace aspd
