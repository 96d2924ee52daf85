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

// Bank-padded shared-memory index of the row passes: thread t reads q = 8 (t + c) + i, padded 9 (t + c) + i,
// so the 32 lanes of a warp hit 32 different banks.
__device__ __forceinline__ int spad(int q) { return q + (q >> 3); }

// Task order of the smoothing passes.  Tasks are numbered scale by scale,
// and a task's cost grows with its scale (20x from the first scale to the
// sixth).  With a counter (sched[0]), thread 0 takes the next task,
// costliest first, so a block that finishes early takes more and the SMs
// end together.  The block that leaves last resets the counter and its exit
// count (sched[1]) for the next launch.  Without a counter the blocks stride
// over the tasks.  Both forms begin with the block barrier that orders the
// previous task's shared-memory reads before the next task's writes.
__device__ __forceinline__ long long next_task(unsigned* sched, long long r, long long total) {
    __shared__ long long s_task;
    __syncthreads();
    if (sched == nullptr) {
        const long long t = r * gridDim.x + blockIdx.x;
        return t < total ? t : -1;
    }
    if (threadIdx.x == 0) {
        const long long t = (long long)atomicAdd(sched, 1u);
        s_task = t < total ? total - 1 - t : -1;
    }
    __syncthreads();
    return s_task;
}
__device__ __forceinline__ void end_tasks(unsigned* sched) {
    if (sched == nullptr || threadIdx.x != 0) return;
    __threadfence();                                  // this block's last fetch before its exit count
    if (atomicAdd(sched + 1, 1u) == gridDim.x - 1) {
        __threadfence();
        atomicExch(sched, 0u);
        atomicExch(sched + 1, 0u);
    }
}

// 8 outputs x 8 taps of a correlation: acc[i] += sum_d k[d] x[i + d], the 16
// inputs x[0..15] given as two 8-register banks (lo, hi).
__device__ __forceinline__ void conv8k(float (&acc)[8], const float (&lo)[8], const float (&hi)[8],
                                       const float4 ka, const float4 kb) {
    const float kk[8] = {ka.x, ka.y, ka.z, ka.w, kb.x, kb.y, kb.z, kb.w};
#pragma unroll
    for (int d = 0; d < 8; ++d)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = fmaf(kk[d], i + d < 8 ? lo[i + d] : hi[i + d - 8], acc[i]);
}
// The same with the taps read from 8 consecutive floats of a 16-byte
// aligned, zero-padded weight row in global memory (L1-cached).
__device__ __forceinline__ void conv8(float (&acc)[8], const float (&lo)[8], const float (&hi)[8],
                                      const float* __restrict__ k8) {
    conv8k(acc, lo, hi, __ldg(reinterpret_cast<const float4*>(k8)), __ldg(reinterpret_cast<const float4*>(k8 + 4)));
}
// ... in shared memory.
__device__ __forceinline__ void conv8s(float (&acc)[8], const float (&lo)[8], const float (&hi)[8], const float* k8) {
    conv8k(acc, lo, hi, *reinterpret_cast<const float4*>(k8), *reinterpret_cast<const float4*>(k8 + 4));
}

// 8 consecutive rows of one column (row stride W) into a register bank.
__device__ __forceinline__ void load_rows8(float (&b)[8], const float* __restrict__ p, int W) {
#pragma unroll
    for (int i = 0; i < 8; ++i) b[i] = __ldg(p + (long long)i * W);
}

// conv8k for two independent output streams at once (two rows, or two
// columns) with Blackwell's packed two-lane FP32 FMA.  Each lane rounds
// like fmaf and the taps are applied in the same order, so every output has
// the bits of the scalar pass, with half the FMA instructions.  k16 holds
// the 8 taps each written twice (k0 k0 k1 k1 ...), 16-byte aligned.
__device__ __forceinline__ void conv8k2(float2 (&acc)[8], const float2 (&lo)[8], const float2 (&hi)[8],
                                        const float* k16) {
    const float4* k4 = reinterpret_cast<const float4*>(k16);
    float2 kk[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = k4[q];
        kk[2 * q] = make_float2(v.x, v.y);
        kk[2 * q + 1] = make_float2(v.z, v.w);
    }
#pragma unroll
    for (int d = 0; d < 8; ++d)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = __ffma2_rn(kk[d], i + d < 8 ? lo[i + d] : hi[i + d - 8], acc[i]);
}

// 8 consecutive rows of two adjacent columns (8-byte aligned) into a bank.
__device__ __forceinline__ void load_rows8x2(float2 (&b)[8], const float* __restrict__ p, int W) {
#pragma unroll
    for (int i = 0; i < 8; ++i) b[i] = __ldg(reinterpret_cast<const float2*>(p + (long long)i * W));
}

// ------------------------------------------------------------------ subtraction
// R -= B * dC (Sect. 2 step 3) with dC a sum of separable sampled terms:
// for term t with axis weights wx (nx taps from column qx0) and wy (ny taps
// from row qy0), T1_t = rows of B convolved with wx, then R -= scale_t *
// (T1_t convolved with wy).  Both passes are register-blocked like the
// smoothing: 8 consecutive outputs per thread, a 16-entry sliding window,
// 8 taps per step.  The weight buffer holds each axis reversed and
// zero-padded to a multiple of 8, so both passes are correlations
//   T1_t[r][u] = sum_i wxr[i] B[r0 + r][c0 + u + i],  c0 = W - qx0 - nx + 1,
//   dR[y][x]   = sum_k wyr[k] T1_t[y + k][x].

// Row pass.  A block task is rpb row segments (8 tpr outputs each) of one
// term's T1 rows; the B segment is staged in shared memory (bank-padded).
// The geometry (tpr, rpb, nseg) depends only on W and is shared with the
// smoothing row pass.
__device__ __forceinline__ void sub_h_body(const float* __restrict__ B, int H, int W, const CycleState* __restrict__ st, const int* gate,
        const float* __restrict__ wbuf, float* __restrict__ T1, int tpr, int rpb, int nseg, int blen) {
    if (gate && *gate) return;
    extern __shared__ __align__(16) float sm_sub[];
    const int tid = threadIdx.x;
    const int sub = tid / tpr, lt = tid - sub * tpr;
    float* buf = sm_sub + sub * blen;
    const int nt = st->n_terms;
    const int W2 = 2 * W;
    long long rows_total = 0;
    for (int t = 0; t < nt; ++t)
        if (!st->terms[t].bilinear) rows_total += (long long)(H + st->terms[t].ny - 1) * nseg;
    const long long btasks = (rows_total + rpb - 1) / rpb;
    for (long long task = blockIdx.x; task < btasks; task += gridDim.x) {
        long long rt = task * rpb + sub;
        const bool live = sub < rpb && rt < rows_total;
        // locate (term, row, segment) of this row task
        int t = 0;
        if (live) {
            for (; t < nt; ++t) {
                if (st->terms[t].bilinear) continue;
                const long long n = (long long)(H + st->terms[t].ny - 1) * nseg;
                if (rt < n) break;
                rt -= n;
            }
        }
        const TermDesc& td = st->terms[live ? t : 0];
        const int r = live ? (int)(rt / nseg) : 0;
        const int xs = live ? (int)(rt % nseg) * 8 * tpr : 0;
        const int nx8 = (td.nx + 7) & ~7;
        const int c0 = W - td.qx0 - td.nx + 1;
        __syncthreads();                                     // previous task's reads are done
        if (sub < rpb) {
            const float* brow = B + (long long)(td.r0 + r) * W2;
            const int len = 8 * tpr + nx8 + 8;
            for (int q = lt; q < len; q += tpr) {
                const int c = c0 + xs + q;
                buf[spad(q)] = (live && c >= 0 && c < W2) ? __ldg(brow + c) : 0.f;
            }
        }
        __syncthreads();
        const int x0 = xs + 8 * lt;
        if (!live || x0 >= W) continue;
        const float* wxr = wbuf + td.woff_x;
        // the 16-entry window lives in two 8-register banks whose roles swap
        // every 8 taps (the loop is unrolled by two), so no register moves
        float acc[8], wa[8], wb[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { acc[i] = 0.f; wa[i] = buf[spad(8 * lt + i)]; }
#pragma unroll 1
        for (int u0 = 0; u0 < nx8; u0 += 16) {
#pragma unroll
            for (int i = 0; i < 8; ++i) wb[i] = buf[spad(8 * lt + u0 + 8 + i)];
            conv8(acc, wa, wb, wxr + u0);
            if (u0 + 8 >= nx8) break;
#pragma unroll
            for (int i = 0; i < 8; ++i) wa[i] = buf[spad(8 * lt + u0 + 16 + i)];
            conv8(acc, wb, wa, wxr + u0 + 8);
        }
        float* out = T1 + td.t1off + (long long)r * W + x0;
        if (x0 + 8 <= W && (W & 3) == 0) {
            reinterpret_cast<float4*>(out)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            reinterpret_cast<float4*>(out)[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (x0 + i < W) out[i] = acc[i];
        }
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_sub_h(const float* __restrict__ B, int H, int W, const CycleState* __restrict__ st, const int* gate,
        const float* __restrict__ wbuf, float* __restrict__ T1, int tpr, int rpb, int nseg, int blen) { sub_h_body(B, H, W, st, gate, wbuf, T1, tpr, rpb, nseg, blen); }

// Column pass + update + fused argmax:
// R[y][x] -= sum_t scale_t sum_k wyr_t[k] T1_t[y + k][x]
//          + sum_d w_d B[y - qy_d + H][x - qx_d + W]      (point deposits)
// Each thread owns 8 consecutive rows of one column (lanes: consecutive
// columns), one block task is 32 columns x 64 rows.  The T1 buffer carries
// zeroed slack rows behind its last term, so the window (which runs up to
// 15 rows past a term's end under zero taps) needs no bounds tests.
__device__ __forceinline__ void sub_v_body(float* __restrict__ R, int H, int W, CycleState* st, const int* gate,
               const float* __restrict__ wbuf, const float* __restrict__ T1, const float* __restrict__ B,
               ArgRes* part, unsigned* ticket) {
    if (gate && *gate) return;
    __shared__ Deposit sdep[MAX_DEPOSITS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = st->n_terms;
    const int nd = st->n_dep;
    for (int i = tid; i < nd; i += blockDim.x) sdep[i] = st->dep[i];
    __syncthreads();
    const int W2 = 2 * W;
    const int ncb = (W + 31) / 32, nrb = (H + 63) / 64;
    float bv = 0.f;
    long long bi = 0x7fffffffffffffffLL;
    int bj = 0;
    unsigned bad = 0;
    for (long long task = blockIdx.x; task < (long long)ncb * nrb; task += gridDim.x) {
        const int rb = (int)(task / ncb), cb = (int)(task % ncb);
        const int px = cb * 32 + lane, py0 = rb * 64 + 8 * warp;
        if (px >= W || py0 >= H) continue;
        float acc[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o] = 0.f;
        for (int t = 0; t < nt; ++t) {
            const TermDesc& td = st->terms[t];
            if (td.bilinear) continue;
            const int ny8 = (td.ny + 7) & ~7;
            const float* wyr = wbuf + td.woff_y;
            const float* col = T1 + td.t1off + (long long)py0 * W + px;
            // three 8-row register banks rotate (the loop is unrolled by
            // three): each step computes on two and loads the next 8 rows
            // into the third, a full step before they are used, so the L2
            // latency of the column loads hides behind the FMAs.  The
            // prefetch reads up to 23 rows past a term's last tap (zero
            // taps; T1 keeps T1_SLACK_ROWS rows behind the last term).
            float s[8], b0[8], b1[8], b2[8];
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                s[o] = 0.f;
                b0[o] = __ldg(col + (long long)o * W);
                b1[o] = __ldg(col + (long long)(8 + o) * W);
            }
#pragma unroll 1
            for (int k0 = 0; k0 < ny8; k0 += 24) {
                load_rows8(b2, col + (long long)(k0 + 16) * W, W);
                conv8(s, b0, b1, wyr + k0);
                if (k0 + 8 >= ny8) break;
                load_rows8(b0, col + (long long)(k0 + 24) * W, W);
                conv8(s, b1, b2, wyr + k0 + 8);
                if (k0 + 16 >= ny8) break;
                load_rows8(b1, col + (long long)(k0 + 32) * W, W);
                conv8(s, b2, b0, wyr + k0 + 16);
            }
#pragma unroll
            for (int o = 0; o < 8; ++o) acc[o] = fmaf(td.scale, s[o], acc[o]);
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) {
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

__global__ void __launch_bounds__(RED_THREADS)
k_sub_v_argmax(float* __restrict__ R, int H, int W, CycleState* st, const int* gate,
               const float* __restrict__ wbuf, const float* __restrict__ T1, const float* __restrict__ B,
               ArgRes* part, unsigned* ticket) { sub_v_body(R, H, W, st, gate, wbuf, T1, B, part, ticket); }

// FFT residual update, last step: R -= conv(p + (H, W)) / (4 H W) (the
// inverse transform of dC's product with the PSF's transform, unnormalised;
// the PSF's zero lag at [H, W] puts image pixel p at p + (H, W) of the
// 2H x 2W grid) with the next argmax fused in, as k_sub_v_argmax does.  The
// block that finishes the argmax records dC's box for the next update.
__global__ void __launch_bounds__(RED_THREADS)
k_fft_sub_argmax(float* __restrict__ R, const float* __restrict__ conv, int H, int W, CycleState* st, const int* gate,
                 ArgRes* part, unsigned* ticket) {
    if (gate && *gate) return;
    const float sc = 1.0f / (4.0f * (float)H * (float)W);
    const long long N = (long long)H * W;
    const long long W2 = 2LL * W;
    float bv = 0.f;
    long long bi = 0x7fffffffffffffffLL;
    int bj = 0;
    unsigned bad = 0;
    if ((W & 3) == 0) {
        // 4 consecutive pixels of one row per thread: both rows are 16-byte aligned
        const long long nq = N >> 2;
        for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (long long)gridDim.x * blockDim.x) {
            const long long p = q << 2;
            const long long y = p / W, x = p - y * W;
            const float4 c = __ldg(reinterpret_cast<const float4*>(conv + (y + H) * W2 + x + W));
            float4 r = reinterpret_cast<const float4*>(R)[q];
            r.x -= c.x * sc; r.y -= c.y * sc; r.z -= c.z * sc; r.w -= c.w * sc;
            reinterpret_cast<float4*>(R)[q] = r;
            const float v[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!isfinite(v[k])) bad = 1;
                if (arg_better(v[k], 0, p + k, bv, 0, bi)) { bv = v[k]; bi = p + k; }
            }
        }
    } else {
        for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
            const long long y = p / W, x = p - y * W;
            const float v = R[p] - __ldg(conv + (y + H) * W2 + x + W) * sc;
            R[p] = v;
            if (!isfinite(v)) bad = 1;
            if (arg_better(v, 0, p, bv, 0, bi)) { bv = v; bi = p; }
        }
    }
    if (bad) atomicOr(&st->nonfinite, 1u);
    block_arg_reduce(bv, bj, bi);
    if (grid_arg_finish(bv, bj, bi, part, ticket, &st->peak) && threadIdx.x < 4) st->dbox[threadIdx.x] = st->dbox_next[threadIdx.x];
}

cudaError_t launch_fft_sub_argmax(float* R, const float* conv, int H, int W, CycleState* st, const int* gate, int grid,
                                  ArgRes* part, unsigned* ticket, cudaStream_t s) {
    k_fft_sub_argmax<<<grid, RED_THREADS, 0, s>>>(R, conv, H, W, st, gate, part, ticket);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ smoothing
// Separable Gaussian smoothing at every scale s_j (Sect. 2 step 1), zero
// padded at the image edges, as two register-blocked passes: each thread
// produces 8 consecutive outputs, keeping a 16-entry sliding window of the
// input in registers, so 8 taps cost 8 loads, 2 broadcast tap loads and 64
// FMAs.  Taps are zero-padded to a multiple of 8 (t8).  The paired forms
// give each thread two such output streams (two rows, or two columns) and
// run both with packed two-lane FMAs: the same bits, half the FMA
// instructions.

// Row pass: S1_j[y + mpad][x] = sum_u k_j[u] R[y][x + u - m_j].  A block
// task is rpb row segments of 8 tpr outputs each; the segment with its
// halo is staged in shared memory.  Blocks loop over the tasks of every
// scale (or only_scale).  This form takes one row per thread; the paired
// form below (the default where its buffers fit) two.
__device__ __forceinline__ void smooth_h_single(const float* __restrict__ R, int H, int W, const SmoothTaps& taps,
                                                int only_scale, float* __restrict__ S1, unsigned* sched) {
    extern __shared__ __align__(16) float sm_h[];
    float* ktap = sm_h;
    const int tid = threadIdx.x;
    const int tpr = taps.tpr, rpb = taps.rpb, nseg = taps.nseg;
    const int sub = tid / tpr, lt = tid - sub * tpr;
    float* buf = sm_h + taps.t8max + sub * taps.blen;
    const int j0 = only_scale >= 0 ? only_scale : 0, nj = only_scale >= 0 ? 1 : taps.n;
    const long long rowtasks = (long long)H * nseg;
    const long long btasks = (rowtasks + rpb - 1) / rpb;
    for (long long r = 0;; ++r) {
        const long long task = next_task(sched, r, nj * btasks);
        if (task < 0) break;
        const int j = j0 + (int)(task / btasks);
        const long long rt = (task % btasks) * rpb + sub;
        const int m = taps.m[j], t8 = taps.t8[j];
        const bool live = sub < rpb && rt < rowtasks;
        const int y = live ? (int)(rt / nseg) : 0;
        const int xs = live ? (int)(rt % nseg) * 8 * tpr : 0;
        const float* kj = taps.k + taps.off[j];
        for (int q = tid; q < t8; q += blockDim.x) ktap[q] = q < 2 * m + 1 ? kj[q] : 0.f;
        if (sub < rpb) {
            const float* row = R + (long long)y * W;
            const int len = 8 * tpr + t8 + 8;
            for (int q = lt; q < len; q += tpr) {
                const int x = xs - m + q;
                buf[spad(q)] = (live && x >= 0 && x < W) ? __ldg(row + x) : 0.f;
            }
        }
        __syncthreads();
        const int x0 = xs + 8 * lt;
        if (!live || x0 >= W) continue;
        // two 8-register window banks swap roles every 8 taps (no moves)
        float acc[8], wa[8], wb[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { acc[i] = 0.f; wa[i] = buf[spad(8 * lt + i)]; }
#pragma unroll 1
        for (int u0 = 0; u0 < t8; u0 += 16) {
#pragma unroll
            for (int i = 0; i < 8; ++i) wb[i] = buf[spad(8 * lt + u0 + 8 + i)];
            conv8s(acc, wa, wb, ktap + u0);
            if (u0 + 8 >= t8) break;
#pragma unroll
            for (int i = 0; i < 8; ++i) wa[i] = buf[spad(8 * lt + u0 + 16 + i)];
            conv8s(acc, wb, wa, ktap + u0 + 8);
        }
        float* out = S1 + ((long long)j * taps.s1rows + y + taps.mpad) * W + x0;
        if (x0 + 8 <= W && (W & 3) == 0) {
            reinterpret_cast<float4*>(out)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            reinterpret_cast<float4*>(out)[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (x0 + i < W) out[i] = acc[i];
        }
    }
}

// Paired row pass: each thread takes the same 8 outputs of rows y and y + 1
// (a row-pair task), the two rows staged interleaved as float2 so one
// shared load feeds both lanes of a packed FMA.  Same sums, same order, so
// the same bits as smooth_h_single.  Shared memory: the taps twice each
// (2 t8max floats), then rpb buffers of 2 blen floats.  The float2 index
// spad(q) puts a half-warp's 8-byte loads in distinct bank pairs.
__device__ __forceinline__ void smooth_h_pair(const float* __restrict__ R, int H, int W, const SmoothTaps& taps,
                                              int only_scale, float* __restrict__ S1, unsigned* sched) {
    extern __shared__ __align__(16) float sm_h[];
    float* ktap = sm_h;
    const int tid = threadIdx.x;
    const int tpr = taps.tpr, rpb = taps.rpb, nseg = taps.nseg;
    const int sub = tid / tpr, lt = tid - sub * tpr;
    float2* buf = reinterpret_cast<float2*>(sm_h + 2 * taps.t8max) + sub * taps.blen;
    const int j0 = only_scale >= 0 ? only_scale : 0, nj = only_scale >= 0 ? 1 : taps.n;
    const long long rowtasks = (long long)((H + 1) >> 1) * nseg;
    const long long btasks = (rowtasks + rpb - 1) / rpb;
    for (long long r = 0;; ++r) {
        const long long task = next_task(sched, r, nj * btasks);
        if (task < 0) break;
        const int j = j0 + (int)(task / btasks);
        const long long rt = (task % btasks) * rpb + sub;
        const int m = taps.m[j], t8 = taps.t8[j];
        const bool live = sub < rpb && rt < rowtasks;
        const int y = live ? 2 * (int)(rt / nseg) : 0;
        const bool live1 = live && y + 1 < H;
        const int xs = live ? (int)(rt % nseg) * 8 * tpr : 0;
        const float* kj = taps.k + taps.off[j];
        for (int q = tid; q < t8; q += blockDim.x) {
            const float v = q < 2 * m + 1 ? kj[q] : 0.f;
            reinterpret_cast<float2*>(ktap)[q] = make_float2(v, v);
        }
        if (sub < rpb) {
            const float* row = R + (long long)y * W;
            const int len = 8 * tpr + t8 + 8;
            for (int q = lt; q < len; q += tpr) {
                const int x = xs - m + q;
                const bool in = x >= 0 && x < W;
                buf[spad(q)] = make_float2((live && in) ? __ldg(row + x) : 0.f, (live1 && in) ? __ldg(row + W + x) : 0.f);
            }
        }
        __syncthreads();
        const int x0 = xs + 8 * lt;
        if (!live || x0 >= W) continue;
        float2 acc[8], wa[8], wb[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { acc[i] = make_float2(0.f, 0.f); wa[i] = buf[spad(8 * lt + i)]; }
#pragma unroll 1
        for (int u0 = 0; u0 < t8; u0 += 16) {
#pragma unroll
            for (int i = 0; i < 8; ++i) wb[i] = buf[spad(8 * lt + u0 + 8 + i)];
            conv8k2(acc, wa, wb, ktap + 2 * u0);
            if (u0 + 8 >= t8) break;
#pragma unroll
            for (int i = 0; i < 8; ++i) wa[i] = buf[spad(8 * lt + u0 + 16 + i)];
            conv8k2(acc, wb, wa, ktap + 2 * u0 + 16);
        }
        float* out = S1 + ((long long)j * taps.s1rows + y + taps.mpad) * W + x0;
        if (x0 + 8 <= W && (W & 3) == 0) {
            reinterpret_cast<float4*>(out)[0] = make_float4(acc[0].x, acc[1].x, acc[2].x, acc[3].x);
            reinterpret_cast<float4*>(out)[1] = make_float4(acc[4].x, acc[5].x, acc[6].x, acc[7].x);
            if (live1) {
                reinterpret_cast<float4*>(out + W)[0] = make_float4(acc[0].y, acc[1].y, acc[2].y, acc[3].y);
                reinterpret_cast<float4*>(out + W)[1] = make_float4(acc[4].y, acc[5].y, acc[6].y, acc[7].y);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (x0 + i < W) {
                    out[i] = acc[i].x;
                    if (live1) out[W + i] = acc[i].y;
                }
        }
    }
}

__device__ __forceinline__ void smooth_h_body(const float* __restrict__ R, int H, int W, const SmoothTaps& taps, const int* gate,
                                              int only_scale, float* __restrict__ S1, unsigned* sched) {
    if (gate && *gate) return;
    if (taps.pair_h) smooth_h_pair(R, H, W, taps, only_scale, S1, sched);
    else smooth_h_single(R, H, W, taps, only_scale, S1, sched);
    end_tasks(sched);
}

__global__ void __launch_bounds__(RED_THREADS, 4)
k_smooth_h(const float* __restrict__ R, int H, int W, const __grid_constant__ SmoothTaps taps, const int* gate,
           int only_scale, float* __restrict__ S1, unsigned* sched) { smooth_h_body(R, H, W, taps, gate, only_scale, S1, sched); }

// Column pass for every scale with the fused argmax of |S_j| over (j, p);
// the last block turns the winner into the initial values
// (S/(sqrt(pi) s), x*, y*, max(s, omega_b)).  out_S (optional) receives S_j.
// A block task is 32 columns x 64 rows of one scale: lane = column, warp w
// = rows 8w..8w+7.  The row-pass image has mpad zero rows above and below,
// so the sliding window needs no bounds tests.  This form serves odd W; the
// paired form below (even W) is the default.
__device__ __forceinline__ void smooth_v_single(const float* __restrict__ S1, int H, int W, const SmoothTaps& taps,
                                                int j0, int nj, float* __restrict__ out_S, float& bv, int& bj,
                                                long long& bi, unsigned* sched) {
    extern __shared__ __align__(16) float ktap[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncb = (W + 31) / 32, nrb = (H + 63) / 64;
    const long long per = (long long)ncb * nrb;
    for (long long r = 0;; ++r) {
        const long long task = next_task(sched, r, nj * per);
        if (task < 0) break;
        const int j = j0 + (int)(task / per);
        const int rem = (int)(task % per);
        const int rb = rem / ncb, cb = rem - rb * ncb;
        const int m = taps.m[j], t8 = taps.t8[j];
        const float* kj = taps.k + taps.off[j];
        for (int q = tid; q < t8; q += blockDim.x) ktap[q] = q < 2 * m + 1 ? kj[q] : 0.f;
        __syncthreads();
        const int x = cb * 32 + lane, y0 = rb * 64 + 8 * warp;
        if (x >= W || y0 >= H) continue;
        const float* col = S1 + ((long long)j * taps.s1rows + (y0 - m + taps.mpad)) * W + x;
        // three 8-row register banks rotate (the loop is unrolled by three):
        // each step computes on two and loads the next 8 rows into the
        // third a step ahead -- only rows the window will use, the same
        // rows as without the prefetch
        float acc[8], b0[8], b1[8], b2[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            acc[i] = 0.f;
            b0[i] = __ldg(col + (long long)i * W);
            b1[i] = __ldg(col + (long long)(8 + i) * W);
        }
#pragma unroll 1
        for (int u0 = 0; u0 < t8; u0 += 24) {
            if (u0 + 8 < t8) load_rows8(b2, col + (long long)(u0 + 16) * W, W);
            conv8s(acc, b0, b1, ktap + u0);
            if (u0 + 8 >= t8) break;
            if (u0 + 16 < t8) load_rows8(b0, col + (long long)(u0 + 24) * W, W);
            conv8s(acc, b1, b2, ktap + u0 + 8);
            if (u0 + 16 >= t8) break;
            if (u0 + 24 < t8) load_rows8(b1, col + (long long)(u0 + 32) * W, W);
            conv8s(acc, b2, b0, ktap + u0 + 16);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int y = y0 + i;
            if (y < H) {
                const long long p = (long long)y * W + x;
                if (out_S) out_S[p] = acc[i];
                if (arg_better(acc[i], j, p, bv, bj, bi)) { bv = acc[i]; bj = j; bi = p; }
            }
        }
    }
}

// Paired column pass (even W): a block task is 64 columns x 64 rows, lane l
// takes columns 2l and 2l + 1 with one 8-byte load per row and packed FMAs
// (the taps written twice each in shared memory).  Same sums in the same
// order as smooth_v_single, so the same S_j bits and the same winner
// (arg_better is a total order, so the visiting order does not matter).
__device__ __forceinline__ void smooth_v_pair(const float* __restrict__ S1, int H, int W, const SmoothTaps& taps,
                                              int j0, int nj, float* __restrict__ out_S, float& bv, int& bj,
                                              long long& bi, unsigned* sched) {
    extern __shared__ __align__(16) float ktap[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncb = (W + 63) / 64, nrb = (H + 63) / 64;
    const long long per = (long long)ncb * nrb;
    for (long long r = 0;; ++r) {
        const long long task = next_task(sched, r, nj * per);
        if (task < 0) break;
        const int j = j0 + (int)(task / per);
        const int rem = (int)(task % per);
        const int rb = rem / ncb, cb = rem - rb * ncb;
        const int m = taps.m[j], t8 = taps.t8[j];
        const float* kj = taps.k + taps.off[j];
        for (int q = tid; q < t8; q += blockDim.x) {
            const float v = q < 2 * m + 1 ? kj[q] : 0.f;
            reinterpret_cast<float2*>(ktap)[q] = make_float2(v, v);
        }
        __syncthreads();
        const int x = cb * 64 + 2 * lane, y0 = rb * 64 + 8 * warp;
        if (x >= W || y0 >= H) continue;                     // W even: x + 1 < W as well
        const float* col = S1 + ((long long)j * taps.s1rows + (y0 - m + taps.mpad)) * W + x;
        float2 acc[8], b0[8], b1[8], b2[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = make_float2(0.f, 0.f);
        load_rows8x2(b0, col, W);
        load_rows8x2(b1, col + (long long)8 * W, W);
#pragma unroll 1
        for (int u0 = 0; u0 < t8; u0 += 24) {
            if (u0 + 8 < t8) load_rows8x2(b2, col + (long long)(u0 + 16) * W, W);
            conv8k2(acc, b0, b1, ktap + 2 * u0);
            if (u0 + 8 >= t8) break;
            if (u0 + 16 < t8) load_rows8x2(b0, col + (long long)(u0 + 24) * W, W);
            conv8k2(acc, b1, b2, ktap + 2 * u0 + 16);
            if (u0 + 16 >= t8) break;
            if (u0 + 24 < t8) load_rows8x2(b1, col + (long long)(u0 + 32) * W, W);
            conv8k2(acc, b2, b0, ktap + 2 * u0 + 32);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int y = y0 + i;
            if (y < H) {
                const long long p = (long long)y * W + x;
                if (out_S) { out_S[p] = acc[i].x; out_S[p + 1] = acc[i].y; }   // caller's buffer: 4-byte alignment
                if (arg_better(acc[i].x, j, p, bv, bj, bi)) { bv = acc[i].x; bj = j; bi = p; }
                if (arg_better(acc[i].y, j, p + 1, bv, bj, bi)) { bv = acc[i].y; bj = j; bi = p + 1; }
            }
        }
    }
}

// Shared memory of the column pass: the taps written twice (paired form).
__device__ __forceinline__ void smooth_v_body(const float* __restrict__ S1, int H, int W, const SmoothTaps& taps, CycleState* st,
                  const int* gate, int only_scale, float* __restrict__ out_S, ArgRes* part, unsigned* ticket,
                  unsigned* sched) {
    if (gate && *gate) return;
    const int j0 = only_scale >= 0 ? only_scale : 0, nj = only_scale >= 0 ? 1 : taps.n;
    float bv = 0.f;
    long long bi = 0x7fffffffffffffffLL;
    int bj = 0x7fffffff;
    if ((W & 1) == 0) smooth_v_pair(S1, H, W, taps, j0, nj, out_S, bv, bj, bi, sched);
    else smooth_v_single(S1, H, W, taps, j0, nj, out_S, bv, bj, bi, sched);
    end_tasks(sched);
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

__global__ void __launch_bounds__(RED_THREADS, 3)
k_smooth_v_argmax(const float* __restrict__ S1, int H, int W, const __grid_constant__ SmoothTaps taps, CycleState* st,
                  const int* gate, int only_scale, float* __restrict__ out_S, ArgRes* part, unsigned* ticket,
                  unsigned* sched) { smooth_v_body(S1, H, W, taps, st, gate, only_scale, out_S, part, ticket, sched); }


// ------------------------------------------------------------------ batched wrappers
// grid.y = image; every image runs the same body with its own buffers.
__global__ void __launch_bounds__(RED_THREADS) k_smooth_h_b(const ImgDesc* __restrict__ imgs) {
    const ImgDesc& g = imgs[blockIdx.y];
    smooth_h_body(g.R, g.H, g.W, g.taps, &g.st->skip_smooth, -1, g.S1, nullptr);
}
__global__ void __launch_bounds__(RED_THREADS) k_smooth_v_b(const ImgDesc* __restrict__ imgs) {
    const ImgDesc& g = imgs[blockIdx.y];
    smooth_v_body(g.S1, g.H, g.W, g.taps, g.st, &g.st->skip_smooth, -1, nullptr, g.part, g.ticket, nullptr);
}
__global__ void __launch_bounds__(RED_THREADS) k_sub_h_b(const ImgDesc* __restrict__ imgs) {
    const ImgDesc& g = imgs[blockIdx.y];
    sub_h_body(g.B, g.H, g.W, g.st, &g.st->stopped, g.wbuf, g.T1, g.taps.tpr, g.taps.rpb, g.taps.nseg, g.sub_blen);
}
__global__ void __launch_bounds__(RED_THREADS) k_sub_v_b(const ImgDesc* __restrict__ imgs) {
    const ImgDesc& g = imgs[blockIdx.y];
    sub_v_body(g.R, g.H, g.W, g.st, &g.st->stopped, g.wbuf, g.T1, g.B, g.part, g.ticket);
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_smooth_h_b(const ImgDesc* imgs, int n, int grid_x, size_t smem, cudaStream_t s) {
    k_smooth_h_b<<<dim3(grid_x, n), RED_THREADS, smem, s>>>(imgs);
    return cudaGetLastError();
}
cudaError_t launch_smooth_v_b(const ImgDesc* imgs, int n, int grid_x, size_t smem, cudaStream_t s) {
    k_smooth_v_b<<<dim3(grid_x, n), RED_THREADS, smem, s>>>(imgs);
    return cudaGetLastError();
}
cudaError_t launch_sub_h_b(const ImgDesc* imgs, int n, int grid_x, size_t smem, cudaStream_t s) {
    k_sub_h_b<<<dim3(grid_x, n), RED_THREADS, smem, s>>>(imgs);
    return cudaGetLastError();
}
cudaError_t launch_sub_v_b(const ImgDesc* imgs, int n, int grid_x, cudaStream_t s) {
    k_sub_v_b<<<dim3(grid_x, n), RED_THREADS, 0, s>>>(imgs);
    return cudaGetLastError();
}

cudaError_t launch_argmax(const float* R, long long N, int grid, ArgRes* part, unsigned* ticket, ArgRes* res,
                          unsigned* nonfinite, const int* gate, cudaStream_t s) {
    k_argmax_abs<<<grid, RED_THREADS, 0, s>>>(R, N, part, ticket, res, nonfinite, gate);
    return cudaGetLastError();
}

// Row-pass buffer of the subtraction: 8 tpr outputs + up to roundup8(W)
// taps + 8 window slack, bank-padded.
int sub_h_blen(int W, const SmoothTaps& geo) {
    const int last = 8 * geo.tpr + ((W + 7) & ~7) + 7;
    return last + (last >> 3) + 1;
}

cudaError_t launch_sub_h(const float* B, int H, int W, const CycleState* st, const int* gate, const float* wbuf,
                          float* T1, int grid, const SmoothTaps& geo, cudaStream_t s) {
    const int blen = sub_h_blen(W, geo);
    const size_t smem = (size_t)geo.rpb * blen * sizeof(float);
    k_sub_h<<<grid, RED_THREADS, smem, s>>>(B, H, W, st, gate, wbuf, T1, geo.tpr, geo.rpb, geo.nseg, blen);
    return cudaGetLastError();
}

cudaError_t launch_sub_v(float* R, const float* B, int H, int W, CycleState* st, const int* gate, const float* wbuf,
                         const float* T1, int grid, ArgRes* part, unsigned* ticket, cudaStream_t s) {
    k_sub_v_argmax<<<grid, RED_THREADS, 0, s>>>(R, H, W, st, gate, wbuf, T1, B, part, ticket);
    return cudaGetLastError();
}

size_t smooth_h_smem(const SmoothTaps& t) {
    const size_t nr = t.pair_h ? 2 : 1;
    return nr * ((size_t)t.t8max + (size_t)t.rpb * t.blen) * sizeof(float);
}
size_t smooth_v_smem(const SmoothTaps& t) { return 2 * (size_t)t.t8max * sizeof(float); }

// Blocks of the smoothing passes: as many as are resident at once (blocks
// that draw tasks from the counter balance only while they all run), at
// most cap.
static int resident_grid(const void* fn, size_t smem, int num_sms, int cap) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, RED_THREADS, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return std::max(1, std::min(cap, per_sm * num_sms));
}
int smooth_grid_h(const SmoothTaps& t, int num_sms, int cap) {
    return resident_grid(reinterpret_cast<const void*>(&k_smooth_h), smooth_h_smem(t), num_sms, cap);
}
int smooth_grid_v(const SmoothTaps& t, int num_sms, int cap) {
    return resident_grid(reinterpret_cast<const void*>(&k_smooth_v_argmax), smooth_v_smem(t), num_sms, cap);
}

cudaError_t launch_smooth_h(const float* R, int H, int W, const SmoothTaps& taps, const int* gate, int only_scale,
                            float* S1, int grid, unsigned* sched, cudaStream_t s) {
    k_smooth_h<<<grid, RED_THREADS, smooth_h_smem(taps), s>>>(R, H, W, taps, gate, only_scale, S1, sched);
    return cudaGetLastError();
}

cudaError_t launch_smooth_v(const float* S1, int H, int W, const SmoothTaps& taps, CycleState* st, const int* gate,
                            int only_scale, float* out_S, int grid, ArgRes* part, unsigned* ticket, unsigned* sched,
                            cudaStream_t s) {
    k_smooth_v_argmax<<<grid, RED_THREADS, smooth_v_smem(taps), s>>>(S1, H, W, taps, st, gate, only_scale, out_S,
                                                                      part, ticket, sched);
    return cudaGetLastError();
}

}  // namespace aspd
