// Image-wide kernels of the minor cycle:
//  * argmax |R| (the simple initial-value method and the noise stopping test,
//    Sect. 2 step 4 and Sect. 3),
//  * R -= B * dC with the full PSF, dC a sum of separable sampled components
//    (residual update, Sect. 2 step 3), with the next argmax fused in,
//  * multi-scale Gaussian smoothing of R with the global peak over all scales
//    fused in (initial values, Sect. 2 step 1).
// Grid-wide argmax uses per-block partials and a last-block-done reduction
// (an atomic ticket, no waiting).
#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {

namespace {

// Block-wide argmax; result valid in thread 0.
__device__ void block_arg_reduce(float& v, int& j, long long& i) {
    __shared__ float sv[32];
    __shared__ int sj[32];
    __shared__ long long si[32];
    arg_warp_reduce(v, j, i);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sv[w] = v; sj[w] = j; si[w] = i; }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = l < nw ? sv[l] : 0.f;
        j = l < nw ? sj[l] : 0x7fffffff;
        i = l < nw ? si[l] : 0x7fffffffffffffffLL;
        arg_warp_reduce(v, j, i);
    }
    __syncthreads();
}

// Publishes this block's partial; the last block to arrive reduces all of
// them into *res and re-arms the ticket.  Returns true in that block.
__device__ bool grid_arg_finish(float v, int j, long long i, ArgRes* part, unsigned* ticket, ArgRes* res) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        part[blockIdx.x].val = v;
        part[blockIdx.x].j = j;
        part[blockIdx.x].idx = i;
        __threadfence();
        unsigned n = atomicAdd(ticket, 1u);
        last = (n == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    float bv = 0.f;
    int bj = 0x7fffffff;
    long long bi = 0x7fffffffffffffffLL;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
        float ov = __ldcg(&part[k].val);
        int oj = __ldcg(&part[k].j);
        long long oi = __ldcg(&part[k].idx);
        if (arg_better(ov, oj, oi, bv, bj, bi)) { bv = ov; bj = oj; bi = oi; }
    }
    block_arg_reduce(bv, bj, bi);
    if (threadIdx.x == 0) {
        res->val = bv;
        res->j = bj;
        res->idx = bi;
        *ticket = 0;
    }
    return true;
}

}  // namespace

// ------------------------------------------------------------------ argmax
__global__ void __launch_bounds__(RED_THREADS)
k_argmax_abs(const float* __restrict__ R, long long N, ArgRes* part, unsigned* ticket, ArgRes* res,
             unsigned* nonfinite, const int* gate) {
    if (gate && *gate) return;
    float bv = 0.f;
    long long bi = 0x7fffffffffffffffLL;
    int bj = 0;
    const long long stride = (long long)gridDim.x * blockDim.x * 4;
    const bool vec = ((reinterpret_cast<uintptr_t>(R) & 15) == 0);
    unsigned bad = 0;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4; base < N; base += stride) {
        float v[4];
        if (vec && base + 3 < N) {
            float4 q = __ldg(reinterpret_cast<const float4*>(R + base));
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
            for (int k = 0; k < 4; ++k) v[k] = base + k < N ? R[base + k] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (base + k < N) {
                if (!isfinite(v[k])) bad = 1;
                if (arg_better(v[k], 0, base + k, bv, 0, bi)) { bv = v[k]; bi = base + k; }
            }
        }
    }
    if (bad && nonfinite) atomicOr(nonfinite, 1u);
    block_arg_reduce(bv, bj, bi);
    grid_arg_finish(bv, bj, bi, part, ticket, res);
}

// ------------------------------------------------------------------ subtraction
// Horizontal pass: T1_t[r][u] = sum_i wx_t[i] B[r0_t + r][u - qx0_t - i + W]
// for r < H + ny_t - 1, u < W, every term t.
__global__ void __launch_bounds__(RED_THREADS)
k_sub_h(const float* __restrict__ B, int H, int W, const CycleState* __restrict__ st, const int* gate,
        const float* __restrict__ wbuf, float* __restrict__ T1) {
    if (gate && *gate) return;
    const int nt = st->n_terms;
    const int W2 = 2 * W;
    for (int t = 0; t < nt; ++t) {
        const TermDesc td = st->terms[t];
        if (td.bilinear) continue;
        const long long nrows = H + td.ny - 1;
        const long long total = nrows * W;
        const float* wx = wbuf + td.woff_x;
        float* out = T1 + td.t1off;
        for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
             q += (long long)gridDim.x * blockDim.x) {
            const int r = (int)(q / W), u = (int)(q % W);
            const float* brow = B + (long long)(td.r0 + r) * W2 + (u - td.qx0 + W);
            float s = 0.f;
            for (int i = 0; i < td.nx; ++i) s = fmaf(wx[i], __ldg(brow - i), s);
            out[q] = s;
        }
    }
}

// Vertical pass + update + fused argmax:
// R[py][px] -= sum_t scale_t sum_j wy_t[j] T1_t[py - j + ny_t - 1][px]
//            + sum_d w_d B[py - qy_d + H][px - qx_d + W]      (point deposits)
// Each thread owns VROWS consecutive rows of one column: a sliding window
// over T1 gives VROWS FMAs per T1 load; lanes hold consecutive columns.
constexpr int VROWS = 8;

__global__ void __launch_bounds__(RED_THREADS)
k_sub_v_argmax(float* __restrict__ R, int H, int W, CycleState* st, const int* gate,
               const float* __restrict__ wbuf, const float* __restrict__ T1, const float* __restrict__ B,
               ArgRes* part, unsigned* ticket) {
    if (gate && *gate) return;
    __shared__ Deposit sdep[MAX_DEPOSITS];
    const int nt = st->n_terms;
    const int nd = st->n_dep;
    for (int i = threadIdx.x; i < nd; i += blockDim.x) sdep[i] = st->dep[i];
    __syncthreads();
    const int W2 = 2 * W;
    const long long nblk = (H + VROWS - 1) / VROWS;
    float bv = 0.f;
    long long bi = 0x7fffffffffffffffLL;
    int bj = 0;
    unsigned bad = 0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nblk * W;
         q += (long long)gridDim.x * blockDim.x) {
        const int px = (int)(q % W);
        const int py0 = (int)(q / W) * VROWS;
        float acc[VROWS];
#pragma unroll
        for (int o = 0; o < VROWS; ++o) acc[o] = 0.f;
        for (int t = 0; t < nt; ++t) {
            const TermDesc& td = st->terms[t];
            if (td.bilinear) continue;
            const int ny = td.ny;
            const long long nrows_t1 = H + ny - 1;
            const float* wy = wbuf + td.woff_y;
            const float* col = T1 + td.t1off + px;
            // window rows py0 + o + k for k = 0 .. ny-1 (tap j = ny - 1 - k)
            float win[VROWS], s[VROWS];
#pragma unroll
            for (int o = 0; o < VROWS; ++o) {
                const long long r = py0 + o;
                win[o] = r < nrows_t1 ? __ldg(col + r * W) : 0.f;
                s[o] = 0.f;
            }
            for (int k = 0; k < ny; ++k) {
                const float w = __ldg(wy + (ny - 1 - k));
#pragma unroll
                for (int o = 0; o < VROWS; ++o) s[o] = fmaf(w, win[o], s[o]);
#pragma unroll
                for (int o = 0; o < VROWS - 1; ++o) win[o] = win[o + 1];
                const long long r = (long long)py0 + VROWS + k;
                win[VROWS - 1] = r < nrows_t1 ? __ldg(col + r * W) : 0.f;
            }
#pragma unroll
            for (int o = 0; o < VROWS; ++o) acc[o] = fmaf(td.scale, s[o], acc[o]);
        }
#pragma unroll
        for (int o = 0; o < VROWS; ++o) {
            const int py = py0 + o;
            if (py < H) {
                float dsum = 0.f;
                for (int d = 0; d < nd; ++d)
                    dsum = fmaf(sdep[d].w, __ldg(B + (long long)(py - sdep[d].qy + H) * W2 + (px - sdep[d].qx + W)),
                                dsum);
                const long long p = (long long)py * W + px;
                const float v = R[p] - (acc[o] + dsum);
                R[p] = v;
                if (!isfinite(v)) bad = 1;
                if (arg_better(v, 0, p, bv, 0, bi)) { bv = v; bi = p; }
            }
        }
    }
    if (bad) atomicOr(&st->nonfinite, 1u);
    block_arg_reduce(bv, bj, bi);
    grid_arg_finish(bv, bj, bi, part, ticket, &st->peak);
}

// ------------------------------------------------------------------ smoothing
// Row pass for every scale: S1_j[y][x] = sum_u k_j[u] R[y][x + u - m_j].
__global__ void __launch_bounds__(RED_THREADS)
k_smooth_h(const float* __restrict__ R, int H, int W, const SmoothTaps taps, const int* gate,
           int only_scale, float* __restrict__ S1) {
    if (gate && *gate) return;
    const long long N = (long long)H * W;
    const int j0 = only_scale >= 0 ? only_scale : 0, j1 = only_scale >= 0 ? only_scale + 1 : taps.n;
    for (int j = j0; j < j1; ++j) {
        const float* k = taps.k + taps.off[j];
        const int m = taps.m[j];
        float* out = S1 + (long long)j * N;
        for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N;
             p += (long long)gridDim.x * blockDim.x) {
            const int y = (int)(p / W), x = (int)(p % W);
            const float* row = R + (long long)y * W;
            const int u0 = max(0, m - x), u1 = min(2 * m, W - 1 - x + m);
            float s = 0.f;
            for (int u = u0; u <= u1; ++u) s = fmaf(k[u], __ldg(row + x + u - m), s);
            out[p] = s;
        }
    }
}

// Column pass for every scale with the fused argmax of |S_j| over (j, p);
// the last block turns the winner into the initial values
// (S/(sqrt(pi) s), x*, y*, max(s, omega_b)).  out_S (optional) receives S_j.
__global__ void __launch_bounds__(RED_THREADS)
k_smooth_v_argmax(const float* __restrict__ S1, int H, int W, const SmoothTaps taps, CycleState* st,
                  const int* gate, int only_scale, float* __restrict__ out_S, ArgRes* part, unsigned* ticket) {
    if (gate && *gate) return;
    const long long N = (long long)H * W;
    const int j0 = only_scale >= 0 ? only_scale : 0, j1 = only_scale >= 0 ? only_scale + 1 : taps.n;
    float bv = 0.f;
    long long bi = 0x7fffffffffffffffLL;
    int bj = 0x7fffffff;
    for (int j = j0; j < j1; ++j) {
        const float* k = taps.k + taps.off[j];
        const int m = taps.m[j];
        const float* in = S1 + (long long)j * N;
        for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N;
             p += (long long)gridDim.x * blockDim.x) {
            const int y = (int)(p / W), x = (int)(p % W);
            const int u0 = max(0, m - y), u1 = min(2 * m, H - 1 - y + m);
            float s = 0.f;
            for (int u = u0; u <= u1; ++u) s = fmaf(k[u], __ldg(in + (long long)(y + u - m) * W + x), s);
            if (out_S) out_S[p] = s;
            if (arg_better(s, j, p, bv, bj, bi)) { bv = s; bj = j; bi = p; }
        }
    }
    block_arg_reduce(bv, bj, bi);
    if (grid_arg_finish(bv, bj, bi, part, ticket, &st->speak) && threadIdx.x == 0 && only_scale < 0) {
        // the grid-wide winner (not this block's partial)
        const float gv = st->speak.val;
        const int gj = st->speak.j;
        const long long gi = st->speak.idx;
        const double s = taps.scale[gj];
        st->init[0] = (double)gv / (1.7724538509055160273 * s);
        st->init[1] = (double)(gi % W);
        st->init[2] = (double)(gi / W);
        st->init[3] = fmax(s, st->omega_b);
        st->init_scale = gj;
        st->init_value = gv;
        st->init_s = (float)s;
    }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_argmax(const float* R, long long N, int grid, ArgRes* part, unsigned* ticket, ArgRes* res,
                          unsigned* nonfinite, const int* gate, cudaStream_t s) {
    k_argmax_abs<<<grid, RED_THREADS, 0, s>>>(R, N, part, ticket, res, nonfinite, gate);
    return cudaGetLastError();
}

cudaError_t launch_sub_h(const float* B, int H, int W, const CycleState* st, const int* gate, const float* wbuf,
                         float* T1, int grid, cudaStream_t s) {
    k_sub_h<<<grid, RED_THREADS, 0, s>>>(B, H, W, st, gate, wbuf, T1);
    return cudaGetLastError();
}

cudaError_t launch_sub_v(float* R, const float* B, int H, int W, CycleState* st, const int* gate, const float* wbuf,
                         const float* T1, int grid, ArgRes* part, unsigned* ticket, cudaStream_t s) {
    k_sub_v_argmax<<<grid, RED_THREADS, 0, s>>>(R, H, W, st, gate, wbuf, T1, B, part, ticket);
    return cudaGetLastError();
}

cudaError_t launch_smooth_h(const float* R, int H, int W, const SmoothTaps& taps, const int* gate, int only_scale,
                            float* S1, int grid, cudaStream_t s) {
    k_smooth_h<<<grid, RED_THREADS, 0, s>>>(R, H, W, taps, gate, only_scale, S1);
    return cudaGetLastError();
}

cudaError_t launch_smooth_v(const float* S1, int H, int W, const SmoothTaps& taps, CycleState* st, const int* gate,
                            int only_scale, float* out_S, int grid, ArgRes* part, unsigned* ticket, cudaStream_t s) {
    k_smooth_v_argmax<<<grid, RED_THREADS, 0, s>>>(S1, H, W, taps, st, gate, only_scale, out_S, part, ticket);
    return cudaGetLastError();
}

}  // namespace aspd
