// Device-side control of one minor-cycle iteration (Sect. 2 steps 1-4 with
// the Sect. 3 changes), so a whole iteration runs without a host round trip:
//   k_cycle_begin  stopping tests (iteration cap, max|R| below the noise
//                  threshold) and the initial-value switch (simple method iff
//                  the last optimal component's area is < area_frac of the
//                  last initial guess's area, Sect. 3);
//   k_select       active set (new member + overlapping, not co-located
//                  retained members) and
//                  the joint fit window, written as a FitDesc;
//   k_update       Eqs. 7-8 deconvolution, loop gain on the new component,
//                  component list / retained list updates, and the separable
//                  subtraction terms dC = gain c_new + sum_old (c'_k - c_k);
//   k_build_weights the sampled, flux-normalised axis weights of each term.
// These are control kernels: one thread, one warp or one block (k_select
// scans the retained list with a block; k_build_weights takes a block per
// term).
#include <cuda_bf16.h>

#include "asp_dev.cuh"
#include "asp_internal.h"

namespace aspd {

namespace {

constexpr double TWO_PI = 6.283185307179586477;
constexpr int SELECT_THREADS = 256;   // k_select: retained members tested at once

// Single-Gaussian image of a component: (alpha_b omega_b^2 F / w_ic^2, x, y,
// w_ic) with w_ic^2 = w_i^2 + omega_b^2 (Eqs. 7-8 inverted).
__device__ void gauss_of(const asp_component& c, double ab, double wb, double* g) {
    double wic2 = c.width * c.width + wb * wb;
    g[0] = ab * wb * wb * c.flux / wic2;
    g[1] = c.x;
    g[2] = c.y;
    g[3] = sqrt(wic2);
}

// Eqs. 7-8 through the flux F = a_ic w_ic^2 / (alpha_b omega_b^2); a point
// when w_ic^2 <= omega_b^2 (1 + 1e-3).
// Word copy by the 32 lanes of a warp (bytes a multiple of 4).
__device__ __forceinline__ void copy_words_warp(void* dst, const void* src, int bytes, int lane) {
    int* d = reinterpret_cast<int*>(dst);
    const int* q = reinterpret_cast<const int*>(src);
    for (int i = lane; i < bytes / 4; i += 32) d[i] = q[i];
}

__device__ asp_component deconvolve(double a, double x, double y, double w, double ab, double wb, double gain) {
    asp_component c;
    double F = a * w * w / (ab * wb * wb);
    c.x = x;
    c.y = y;
    c.reserved = 0;
    if (w * w > wb * wb * (1.0 + 1e-3)) {
        double wi = sqrt(w * w - wb * wb);
        c.flux = gain * F;
        c.amp = gain * F / (TWO_PI * wi * wi);
        c.width = wi;
        c.is_point = 0;
    } else {
        c.flux = gain * F;
        c.amp = gain * F;
        c.width = 0.0;
        c.is_point = 1;
    }
    return c;
}

// Term descriptor of component c scaled by s; returns false if its support
// misses the image.
__device__ bool make_term(const asp_component& c, double s, int H, int W, int slot, TermDesc& td) {
    long long ux0, ux1, uy0, uy1;
    if (c.is_point || c.width < 0.5) {
        td.bilinear = 1;
        ux0 = (long long)floor(c.x); ux1 = ux0 + 1;
        uy0 = (long long)floor(c.y); uy1 = uy0 + 1;
    } else {
        td.bilinear = 0;
        double h = ceil(5.0 * c.width) + 1.0;
        ux0 = (long long)ceil(c.x - h); ux1 = (long long)floor(c.x + h);
        uy0 = (long long)ceil(c.y - h); uy1 = (long long)floor(c.y + h);
    }
    long long qx0 = ux0 < 0 ? 0 : ux0, qx1 = ux1 > W - 1 ? W - 1 : ux1;
    long long qy0 = uy0 < 0 ? 0 : uy0, qy1 = uy1 > H - 1 ? H - 1 : uy1;
    if (qx0 > qx1 || qy0 > qy1) return false;
    td.qx0 = (int)qx0; td.nx = (int)(qx1 - qx0 + 1);
    td.qy0 = (int)qy0; td.ny = (int)(qy1 - qy0 + 1);
    td.ux0 = (int)(ux0 < -(1LL << 30) ? -(1LL << 30) : ux0);
    td.ux1 = (int)(ux1 > (1LL << 30) ? (1LL << 30) : ux1);
    td.uy0 = (int)(uy0 < -(1LL << 30) ? -(1LL << 30) : uy0);
    td.uy1 = (int)(uy1 > (1LL << 30) ? (1LL << 30) : uy1);
    td.scale = (float)s;
    td.cx = c.x; td.cy = c.y; td.w = c.width;
    td.woff_x = slot * wslot_stride(W, H);
    td.woff_y = slot * wslot_stride(W, H) + wslot_x_len(W);
    td.r0 = H - td.qy0 - td.ny + 1;
    td.pad = 0;
    return true;
}

// Point-like terms become bilinear deposits (weights (1-f, f) per axis,
// clipped to the image); extended terms get T1 offsets for the separable
// passes.  Also the algorithmic work of R -= B * dC: per extended term
// 2 nx (H + ny - 1) W + 2 ny H W flops, per deposit 2 H W, plus 2 H W for the
// update; bytes: each term's PSF region read once, R read and written once.
// terms: the n_terms descriptors being built (in shared memory, so this
// single-thread loop does not wait on a global round trip per field).
// Warp-inclusive scan of a 64-bit count over the 32 lanes.
__device__ __forceinline__ long long warp_scan_ll(long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// finish_terms by the 32 lanes of a warp: each lane takes terms t = lane,
// lane + 32, ...; T1 offsets and deposit slots come from warp scans, in
// term order, so the result is the serial loop's (deposits beyond
// MAX_DEPOSITS dropped in the same order); the work totals are warp sums.
__device__ void finish_terms_warp(CycleState* st, TermDesc* terms, int n_terms, int H, int W, int lane) {
    long long off = 0;
    int nd = 0;
    double fl = 0.0, by = 0.0;
    for (int t0 = 0; t0 < n_terms; t0 += 32) {
        const int t = t0 + lane;
        long long rows = 0;
        int ndep = 0;
        unsigned dmask = 0;
        double qx[2] = {0, 0}, qy[2] = {0, 0}, wx[2] = {0, 0}, wy[2] = {0, 0};
        if (t < n_terms) {
            TermDesc& td = terms[t];
            if (td.bilinear) {
                const double fx0 = floor(td.cx), fy0 = floor(td.cy);
                const double fx = td.cx - fx0, fy = td.cy - fy0;
                for (int j = 0; j < 2; ++j)
                    for (int i = 0; i < 2; ++i) {
                        const long long ix = (long long)fx0 + i, iy = (long long)fy0 + j;
                        if (ix < 0 || ix >= W || iy < 0 || iy >= H) continue;
                        dmask |= 1u << (2 * j + i);
                        ++ndep;
                    }
                qx[0] = fx0; qy[0] = fy0; wx[0] = 1.0 - fx; wx[1] = fx; wy[0] = 1.0 - fy; wy[1] = fy;
            } else {
                rows = (long long)(H + td.ny - 1) * W;
                fl += 2.0 * td.nx * (double)(H + td.ny - 1) * W + 2.0 * td.ny * (double)H * W;
                by += 4.0 * (double)(H + td.ny - 1) * (W + td.nx - 1);
            }
        }
        const long long rows_incl = warp_scan_ll(rows, lane);
        const long long dep_incl = warp_scan_ll(ndep, lane);
        if (t < n_terms) {
            TermDesc& td = terms[t];
            if (td.bilinear) {
                td.t1off = -1;
                int slot = nd + (int)(dep_incl - ndep);
                for (int q = 0; q < 4; ++q) {
                    if (!(dmask & (1u << q))) continue;
                    if (slot < MAX_DEPOSITS) {
                        const int i = q & 1, j = q >> 1;
                        st->dep[slot].qx = (int)((long long)qx[0] + i);
                        st->dep[slot].qy = (int)((long long)qy[0] + j);
                        st->dep[slot].w = (float)((double)td.scale * wx[i] * wy[j]);
                        st->dep[slot].pad = 0;
                        fl += 2.0 * (double)H * W;
                        by += 4.0 * (double)H * W;
                    }
                    ++slot;
                }
            } else {
                td.t1off = off + rows_incl - rows;
            }
        }
        off += __shfl_sync(0xffffffffu, rows_incl, 31);
        nd += (int)__shfl_sync(0xffffffffu, dep_incl, 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fl += __shfl_xor_sync(0xffffffffu, fl, o);
        by += __shfl_xor_sync(0xffffffffu, by, o);
    }
    if (lane == 0) {
        st->n_dep = nd < MAX_DEPOSITS ? nd : MAX_DEPOSITS;
        st->sub_flops += fl + 2.0 * (double)H * W;
        st->sub_bytes += by + 8.0 * (double)H * W;
    }
}

__device__ void finish_terms(CycleState* st, TermDesc* terms, int n_terms, int H, int W) {
    long long off = 0;
    double fl = 0.0, by = 8.0 * (double)H * W;
    int nd = 0;
    for (int t = 0; t < n_terms; ++t) {
        TermDesc& td = terms[t];
        if (td.bilinear) {
            const double fx0 = floor(td.cx), fy0 = floor(td.cy);
            const double fx = td.cx - fx0, fy = td.cy - fy0;
            for (int j = 0; j < 2; ++j)
                for (int i = 0; i < 2; ++i) {
                    const long long qx = (long long)fx0 + i, qy = (long long)fy0 + j;
                    if (qx < 0 || qx >= W || qy < 0 || qy >= H || nd >= MAX_DEPOSITS) continue;
                    const double w = (double)td.scale * (i ? fx : 1.0 - fx) * (j ? fy : 1.0 - fy);
                    st->dep[nd].qx = (int)qx;
                    st->dep[nd].qy = (int)qy;
                    st->dep[nd].w = (float)w;
                    st->dep[nd].pad = 0;
                    ++nd;
                    fl += 2.0 * (double)H * W;
                    by += 4.0 * (double)H * W;
                }
            td.t1off = -1;
        } else {
            td.t1off = off;
            off += (long long)(H + td.ny - 1) * W;
            fl += 2.0 * td.nx * (double)(H + td.ny - 1) * W + 2.0 * td.ny * (double)H * W;
            by += 4.0 * (double)(H + td.ny - 1) * (W + td.nx - 1);
        }
    }
    st->n_dep = nd;
    st->sub_flops += fl + 2.0 * (double)H * W;
    st->sub_bytes += by;
}

}  // namespace

__device__ __forceinline__ void cycle_begin_body(CycleState* st, Params p, int H, int W, double smooth_flops) {
    if (threadIdx.x != 0) return;
    // every field read first, so the loads go out together instead of one
    // L2 round trip per test
    const int stopped = st->stopped;
    const unsigned nonfinite = st->nonfinite;
    const int t = st->t, t_stop = st->t_stop, n_comp = st->n_comp, cap_comp = st->cap_comp;
    const float pval = st->peak.val;
    const long long pidx = st->peak.idx;
    const double thr = st->thr, last_wi = st->last_wi, last_w0 = st->last_w0, omega_b = st->omega_b;
    st->fit.active = 0;
    st->skip_smooth = 1;
    if (stopped) return;
    if (nonfinite) { st->stopped = 1; st->error = ASP_ERR_NAN; return; }
    if (t >= t_stop) { st->stopped = 1; st->stop_reason = ASP_STOP_ITER; return; }
    if (fabs((double)pval) < thr) { st->stopped = 1; st->stop_reason = ASP_STOP_NOISE; return; }
    if (n_comp >= cap_comp) { st->stopped = 1; st->stop_reason = ASP_STOP_CAPACITY; return; }
    int mode;
    if (p.init_mode == ASP_INIT_SIMPLE) mode = ASP_PEAK_SIMPLE;
    else if (p.init_mode == ASP_INIT_SMOOTH) mode = ASP_PEAK_SMOOTH;
    else mode = (t > 0 && last_wi * last_wi < (double)p.area_frac * last_w0 * last_w0)
                    ? ASP_PEAK_SIMPLE : ASP_PEAK_SMOOTH;
    st->mode = mode;
    st->skip_smooth = mode != ASP_PEAK_SMOOTH;
    if (mode == ASP_PEAK_SMOOTH) { st->smooth_flops += smooth_flops; st->smooth_iters += 1; }
    if (mode == ASP_PEAK_SIMPLE) {
        const long long idx = pidx;
        st->init[0] = pval;
        st->init[1] = (double)(idx % W);
        st->init[2] = (double)(idx / W);
        st->init[3] = omega_b;
        st->init_scale = -1;
        st->init_value = pval;
        st->init_s = 0.f;
    }
}

__global__ void k_cycle_begin(CycleState* st, Params p, int H, int W, double smooth_flops) { cycle_begin_body(st, p, H, W, smooth_flops); }

__device__ __forceinline__ void select_body(CycleState* st, const asp_component* __restrict__ comps, Params p, int H, int W,
                         int g_max) {
    // the block's threads test blockDim.x retained members at a time; the
    // first ones in list order (most recent first) are taken, as in a
    // sequential scan: a member's rank is the number of overlapping members
    // before it in the list (warp ballots plus the warps before it)
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)(blockDim.x >> 5);
    __shared__ int s_cnt[2][32];      // per warp: overlapping members, taken members
    __shared__ int s_box[4][32];      // per warp: bounds of the taken members' boxes
    // the fields read before the first branch, so their loads go out together
    const int stopped = st->stopped, n_ret_ = st->n_ret;
    const double ab = st->alpha_b, wb = st->omega_b;
    const double ix = st->init[1], iy = st->init[2], iw = st->init[3];
    if (stopped) return;
    FitDesc& f = st->fit;
    long long nb[4];
    member_box(ix, iy, iw, nb);
    long long wx0 = nb[0], wx1 = nb[1], wy0 = nb[2], wy1 = nb[3];
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) f.theta0[i] = st->init[i];
        st->members[0] = -1;
    }
    int K = 1;
    const int n_ret = n_ret_;
    for (int base = 0; base < n_ret && K < p.k_max; base += blockDim.x) {
        const int r = base + tid;
        double g[4] = {0, 0, 0, 0};
        long long b[4] = {0, 0, 0, 0};
        int k = -1;
        bool ok = false;
        if (r < n_ret) {
            k = st->ret[r];
            gauss_of(comps[k], ab, wb, g);
            member_box(g[1], g[2], g[3], b);
            const double dx = g[1] - ix, dy = g[2] - iy;
            const double mw = fmax(iw, g[3]);
            // overlapping but not co-located (co-located members leave only
            // the sum of their amplitudes determined)
            ok = b[0] <= nb[1] && nb[0] <= b[1] && b[2] <= nb[3] && nb[2] <= b[3] && dx * dx + dy * dy > mw * mw;
        }
        const unsigned mask = __ballot_sync(FULL, ok);
        if (lane == 0) s_cnt[0][warp] = __popc(mask);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += s_cnt[0][w];
        // the first k_max - K overlapping entries in list order: each taken
        // thread writes its own member slot; the window grows by min/max
        // reductions over the taken threads' boxes (image coordinates fit int)
        const int rank = before + __popc(mask & ((1u << lane) - 1u));
        const bool take = ok && rank < p.k_max - K;
        if (take) {
            const int slot = K + rank;
            for (int i = 0; i < 4; ++i) f.theta0[4 * slot + i] = g[i];
            st->members[slot] = k;
        }
        const int big = 0x3fffffff;
        const int c0 = take ? (int)max(b[0], (long long)-big) : big, c1 = take ? (int)min(b[1], (long long)big) : -big;
        const int c2 = take ? (int)max(b[2], (long long)-big) : big, c3 = take ? (int)min(b[3], (long long)big) : -big;
        const int m0 = __reduce_min_sync(FULL, c0), m1 = __reduce_max_sync(FULL, c1);
        const int m2 = __reduce_min_sync(FULL, c2), m3 = __reduce_max_sync(FULL, c3);
        const int nt = __popc(__ballot_sync(FULL, take));
        if (lane == 0) {
            s_box[0][warp] = m0; s_box[1][warp] = m1; s_box[2][warp] = m2; s_box[3][warp] = m3;
            s_cnt[1][warp] = nt;
        }
        __syncthreads();
        for (int w = 0; w < nw; ++w) {
            K += s_cnt[1][w];
            wx0 = min(wx0, (long long)s_box[0][w]);
            wx1 = max(wx1, (long long)s_box[1][w]);
            wy0 = min(wy0, (long long)s_box[2][w]);
            wy1 = max(wy1, (long long)s_box[3][w]);
        }
        __syncthreads();                  // s_cnt and s_box are rewritten by the next chunk
    }
    if (tid != 0) return;
    wx0 = max(wx0, 0LL); wy0 = max(wy0, 0LL);
    wx1 = min(wx1, (long long)W - 1); wy1 = min(wy1, (long long)H - 1);
    f.K = K;
    f.n_old = K - 1;
    f.has_start = 0;
    f.model = 0;
    f.wx0 = (int)wx0; f.wy0 = (int)wy0;
    f.ww = (int)(wx1 - wx0 + 1); f.wh = (int)(wy1 - wy0 + 1);
    f.use_mask = 0;
    f.mcx = f.mcy = f.mr2 = 0.0;
    f.omega_min = 0.25 * wb;
    f.omega_max = (double)max(f.ww, f.wh);
    f.bx0 = (double)wx0; f.bx1 = (double)wx1; f.by0 = (double)wy0; f.by1 = (double)wy1;
    int smem_ok = 1;
    f.grid = fit_grid((long long)f.ww * f.wh, K, p.lm.px_per_cta, g_max, &smem_ok);
    f.smem_ok = smem_ok;
    f.active = 1;
    st->K = K;
    st->fout.error = 0;
}

__global__ void k_select(CycleState* st, const asp_component* __restrict__ comps, Params p, int H, int W,
                         int g_max) { select_body(st, comps, p, H, W, g_max); }

// One warp.  Lane m (1 <= m < K) deconvolves refit member m and tests its
// retention; lane 0 lays out the subtraction terms in the fixed order (new,
// then (refit, -old) per member), writes the history and the totals; the
// retained list is compacted by ballot.
__device__ __forceinline__ void update_body(CycleState* st, asp_component* comps, asp_iter_record* hist, Params p, int H, int W) {
    const int lane = threadIdx.x;
    if (lane >= 32) return;
    if (st->stopped) return;
    const FitOut& fo = st->fout;
    const FitDesc& f = st->fit;
    if (fo.error) {
        if (lane == 0) { st->stopped = 1; st->error = fo.error; st->n_terms = 0; }
        return;
    }
    __shared__ asp_component s_old[KMAX], s_new[KMAX];
    __shared__ int s_drop[KMAX];
    const double ab = st->alpha_b, wb = st->omega_b;
    const int K = f.K;
    const int ni = st->n_comp;
    // refit members in parallel: retention test (tau) and the deconvolved new value
    __shared__ int s_member[KMAX];
    for (int m = 1 + lane; m < K; m += 32) {
        const int k = st->members[m];
        s_member[m] = k;
        const double* g0 = &f.theta0[4 * m];
        const double* g1 = &fo.theta[4 * m];
        const double tau = p.tau;
        const bool keep = fabs(g1[0] - g0[0]) > tau * fabs(g0[0]) || fabs(g1[1] - g0[1]) > tau * g0[3] ||
                          fabs(g1[2] - g0[2]) > tau * g0[3] || fabs(g1[3] - g0[3]) > tau * g0[3];
        s_drop[m] = keep ? -1 : k;
        s_old[m] = comps[k];
        s_new[m] = deconvolve(g1[0], g1[1], g1[2], g1[3], ab, wb, 1.0);
    }
    __shared__ asp_component s_cn;
    if (lane == 0) {
        // new component with the loop gain (Sect. 3, after Eq. 8)
        s_cn = deconvolve(fo.theta[0], fo.theta[1], fo.theta[2], fo.theta[3], ab, wb, (double)p.gain);
        comps[ni] = s_cn;
        st->n_comp = ni + 1;
        st->last_wi = s_cn.width;
    }
    __syncwarp();
    // the terms in a fixed order -- the new component, then each refit
    // member's new value and its old value negated -- one candidate per
    // lane (u = 0; u = 2m - 1, 2m for member m), those whose support meets
    // the image kept in order by a ballot; old members are replaced by their
    // refit values
    __shared__ TermDesc s_terms[MAX_TERMS];
    const int n_cand = 2 * K - 1;
    int nt = 0;
    for (int u0 = 0; u0 < n_cand; u0 += 32) {
        const int u = u0 + lane;
        TermDesc td;
        bool ok = false;
        if (u < n_cand) {
            if (u == 0) {
                ok = make_term(s_cn, s_cn.flux, H, W, 0, td);
            } else {
                const int m = (u + 1) >> 1;
                if (u & 1) {
                    comps[s_member[m]] = s_new[m];
                    ok = make_term(s_new[m], s_new[m].flux, H, W, 0, td);
                } else {
                    ok = make_term(s_old[m], -s_old[m].flux, H, W, 0, td);
                }
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const int slot = nt + __popc(bal & ((1u << lane) - 1u));
            td.woff_x = slot * wslot_stride(W, H);
            td.woff_y = slot * wslot_stride(W, H) + wslot_x_len(W);
            s_terms[slot] = td;
        }
        nt += __popc(bal);
    }
    __syncwarp();
    if (lane == 0) st->n_terms = nt;
    // the separable full-PSF passes' layout and work; the minor/major split
    // subtracts the terms' beam images instead (k_sub_gauss)
    if (p.major_every == 0) finish_terms_warp(st, s_terms, nt, H, W, lane);
    __syncwarp();
    copy_words_warp(st->terms, s_terms, nt * (int)sizeof(TermDesc), lane);
    // retained list: new first, then the previous list minus members whose
    // fit moved no parameter by more than tau (order kept)
    const int n_old = st->n_ret;
    const int cap = p.retained_cap;
    __shared__ int s_ret[RET_MAX];
    for (int r = lane; r < n_old; r += 32) s_ret[r] = st->ret[r];   // staged: the list is rewritten in place
    __syncwarp();
    int out = 1;   // slot 0 is the new component
    for (int r0 = 0; r0 < n_old; r0 += 32) {
        const int r = r0 + lane;
        int k = -1;
        bool keep_r = false;
        if (r < n_old) {
            k = s_ret[r];
            keep_r = true;
            for (int m = 1; m < K; ++m)
                if (s_drop[m] == k) keep_r = false;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep_r);
        const int pos = out + __popc(bal & ((1u << lane) - 1u));
        if (keep_r && pos < cap) st->ret[pos] = k;
        out += __popc(bal);
    }
    if (lane == 0) {
        st->ret[0] = ni;
        st->n_ret = out < cap ? out : cap;
        // history
        if (st->t < st->cap_comp) {
            asp_iter_record* h = hist + st->t;
            h->t = st->t; h->mode = st->mode; h->k = K; h->status = fo.status;
            h->iters = fo.iters; h->passes = fo.passes;
            h->x0 = f.wx0; h->x1 = f.wx0 + f.ww - 1; h->y0 = f.wy0; h->y1 = f.wy0 + f.wh - 1;
            h->new_index = ni; h->n_terms = st->n_terms;
            h->peak_value = st->peak.val;
            h->init_scale = st->init_scale >= 0 ? st->init_s : 0.f;
            h->chi2_init = fo.chi2_init; h->chi2_final = fo.chi2;
            h->a0 = st->init[0]; h->x0_init = st->init[1]; h->y0_init = st->init[2]; h->w0 = st->init[3];
        }
        // switch statistics and totals
        st->last_w0 = st->init[3];
        st->pixel_evals += fo.pixel_evals;
        st->fit_flops += (double)fo.pixel_evals * pixel_eval_flops(K);
        st->fit_ex2 += (double)fo.pixel_evals * K;
        st->lm_iters += fo.iters;
        st->fit_ns_pass += fo.ns_pass;
        st->fit_ns_reduce += fo.ns_reduce;
        st->fit_ns_solve += fo.ns_solve;
        st->fit_ns_factor += fo.ns_factor;
        st->fit_ns_subst += fo.ns_subst;
        st->fit_refinements += fo.refinements;
        st->fit_fallbacks += fo.fallbacks;
        st->lm_passes += fo.passes;
        st->t += 1;
        st->since_major += 1;
    }
}

__global__ void k_update(CycleState* st, asp_component* comps, asp_iter_record* hist, Params p, int H, int W) { update_body(st, comps, hist, p, H, W); }

__global__ void k_terms_from_components(CycleState* st, const asp_component* __restrict__ comps, int n, float gain,
                                        int H, int W) {
    if (threadIdx.x != 0) return;
    int nt = 0;
    for (int i = 0; i < n && nt < MAX_TERMS; ++i)
        if (make_term(comps[i], (double)gain * comps[i].flux, H, W, nt, st->terms[nt])) ++nt;
    st->n_terms = nt;
    finish_terms(st, st->terms, nt, H, W);
}

// Axis weights of every term: sampled Gaussian normalised to unit sum over the
// unclipped support (so the component's discrete flux is its F), or the
// bilinear pair (1 - f, f).  One block per term.
__device__ __forceinline__ void build_weights_body(const CycleState* __restrict__ st, const int* gate, float* __restrict__ wbuf) {
    if (gate && *gate) return;
    const int t = blockIdx.x;
    if (t >= st->n_terms) return;
    const TermDesc td = st->terms[t];
    if (td.bilinear) return;          // applied as deposits, no axis weights
    __shared__ float red[256];
    for (int axis = 0; axis < 2; ++axis) {
        const double c = axis == 0 ? td.cx : td.cy;
        const int q0 = axis == 0 ? td.qx0 : td.qy0;
        const int n = axis == 0 ? td.nx : td.ny;
        const int u0 = axis == 0 ? td.ux0 : td.uy0;
        const int u1 = axis == 0 ? td.ux1 : td.uy1;
        float* out = wbuf + (axis == 0 ? td.woff_x : td.woff_y);
        {
            // FP32 samples exp(-dq^2 / 2 w^2) with dq = (q - q_c) - f, the
            // integer and fractional parts of the centre apart (no
            // cancellation); the normalising sum as per-thread partials and
            // a fixed tree (error ~ (taps / 256 + 8) u32, far inside the
            // subtraction's 1e-5 bar)
            const float iw = (float)(1.0 / (2.0 * td.w * td.w));
            const double cq = floor(c);
            const float fr = (float)(c - cq);
            const long long icq = (long long)cq;
            float sum = 0.f;
            for (long long q = (long long)u0 + threadIdx.x; q <= u1; q += blockDim.x) {
                const float dq = (float)(q - icq) - fr;
                sum += expf(-dq * dq * iw);
            }
            red[threadIdx.x] = sum;
            __syncthreads();
            for (int o = 128; o > 0; o >>= 1) {
                if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
                __syncthreads();
            }
            const float inv = 1.0f / red[0];
            __syncthreads();
            // reversed (tap i at n - 1 - i) and zero-padded to a multiple of 8
            const int n8 = (n + 7) & ~7;
            for (int i = threadIdx.x; i < n8; i += blockDim.x) {
                float v = 0.f;
                if (i < n) {
                    const float dq = (float)((long long)(q0 + i) - icq) - fr;
                    v = expf(-dq * dq * iw) * inv;
                }
                out[i < n ? n - 1 - i : i] = v;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
k_build_weights(const CycleState* __restrict__ st, const int* gate, float* __restrict__ wbuf) { build_weights_body(st, gate, wbuf); }

// Eqs. 7-8 for elliptical shapes, one thread per component (FP64):
// Sigma = P^-1 for the fitted Gaussian and the beam, Sigma_i = Sigma_ic -
// Sigma_b, flux F = a_ic sqrt(det Sigma_ic) / (alpha_b sqrt(det Sigma_b)),
// amp = F / (2 pi sqrt(det Sigma_i)); a point when the smaller eigenvalue of
// Sigma_i is at most 1e-3 times the smaller eigenvalue of Sigma_b.
// v[0] is the beam, v[1..n] the components.
__global__ void k_deconvolve_ell(const asp_gauss_ell* __restrict__ v, int n, asp_component_ell* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const asp_gauss_ell b = v[0], g = v[1 + k];
    auto cov = [](double A, double B, double C, double& sxx, double& sxy, double& syy, double& det) {
        const double dp = A * C - B * B;
        sxx = C / dp; sxy = -B / dp; syy = A / dp;
        det = 1.0 / dp;
    };
    auto eig_min = [](double sxx, double sxy, double syy) {
        return 0.5 * (sxx + syy) - hypot(0.5 * (sxx - syy), sxy);
    };
    double bxx, bxy, byy, bdet, cxx, cxy, cyy, cdet;
    cov(b.pxx, b.pxy, b.pyy, bxx, bxy, byy, bdet);
    cov(g.pxx, g.pxy, g.pyy, cxx, cxy, cyy, cdet);
    asp_component_ell c;
    c.x = g.x;
    c.y = g.y;
    c.reserved = 0;
    c.flux = g.amp * sqrt(cdet) / (b.amp * sqrt(bdet));
    const double ixx = cxx - bxx, ixy = cxy - bxy, iyy = cyy - byy;
    if (eig_min(ixx, ixy, iyy) <= 1e-3 * eig_min(bxx, bxy, byy)) {
        c.is_point = 1;
        c.amp = c.flux;
        c.sxx = c.sxy = c.syy = 0.0;
    } else {
        c.is_point = 0;
        c.sxx = ixx; c.sxy = ixy; c.syy = iyy;
        c.amp = c.flux / (TWO_PI * sqrt(ixx * iyy - ixy * ixy));
    }
    out[k] = c;
}

cudaError_t launch_deconvolve_ell(const asp_gauss_ell* beam_then_in, int n, asp_component_ell* out, cudaStream_t s) {
    k_deconvolve_ell<<<(n + 63) / 64, 64, 0, s>>>(beam_then_in, n, out);
    return cudaGetLastError();
}

// Eq. 8 per channel for a joint wide-band fit: member k's flux in channel c,
// F = a_kc w_kc^2 / (alpha_b_c omega_b_c^2) with w_kc^2 = s_k^2 +
// omega_b_c^2, and the point flag s_k^2 <= 1e-3 min_c omega_b_c^2.  wb
// holds omega_b_c^2 then alpha_b_c; out: K x C fluxes, then PMAX flags.
__global__ void k_joint_flux(const FitOut* __restrict__ fo, int K, int C, const double* __restrict__ wb,
                             double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * C) return;
    const int k = i / C, c = i - k * C, NPM = 3 + C;
    const double sk = fo->theta[NPM * k + 2], wb2 = wb[c];
    out[i] = fo->theta[NPM * k + 3 + c] * (sk * sk + wb2) / (wb[C + c] * wb2);
    if (c == 0) {
        double wmin = wb[0];
        for (int q = 1; q < C; ++q) wmin = fmin(wmin, wb[q]);
        out[PMAX + k] = sk * sk <= 1e-3 * wmin ? 1.0 : 0.0;
    }
}

cudaError_t launch_joint_flux(const FitOut* fo, int K, int C, const double* wb, double* out, cudaStream_t s) {
    k_joint_flux<<<(K * C + 127) / 128, 128, 0, s>>>(fo, K, C, wb, out);
    return cudaGetLastError();
}

// Clears the minor-cycle state (components, retained list, counters) while
// keeping the beam, the noise threshold and the capacities.
__global__ void k_reset_state(CycleState* st) {
    if (threadIdx.x != 0) return;
    st->t = 0; st->t_stop = 0; st->stopped = 0; st->stop_reason = 0;
    st->mode = 0; st->error = 0; st->n_comp = 0; st->n_ret = 0; st->n_terms = 0; st->K = 0;
    st->skip_smooth = 1;
    st->last_wi = 0.0; st->last_w0 = 0.0;
    st->pixel_evals = 0; st->lm_iters = 0; st->lm_passes = 0;
    st->fit_flops = 0.0; st->sub_flops = 0.0; st->sub_bytes = 0.0; st->smooth_flops = 0.0;
    st->fit_ex2 = 0.0; st->smooth_iters = 0;
    st->since_major = 0; st->major_skip = 1; st->major_cycles = 0;
    st->fit_ns_pass = 0; st->fit_ns_reduce = 0; st->fit_ns_solve = 0; st->fit_ns_factor = 0; st->fit_ns_subst = 0;
    st->fit_refinements = 0; st->fit_fallbacks = 0;
    st->nonfinite = 0;
    st->fit.active = 0;
    st->fit2.active = 0;
    st->learned_used = 0; st->need_plain = 0;
    st->learned_fits = 0; st->learned_refits = 0; st->learned_kept = 0;
}


// ------------------------------------------------------------------ batched wrappers (grid.y = image)
__global__ void k_cycle_begin_b(const ImgDesc* __restrict__ imgs) {
    const ImgDesc& g = imgs[blockIdx.y];
    cycle_begin_body(g.st, g.dp, g.H, g.W, g.smooth_flops);
}
__global__ void k_select_b(const ImgDesc* __restrict__ imgs) {
    const ImgDesc& g = imgs[blockIdx.y];
    select_body(g.st, g.comps, g.dp, g.H, g.W, g.g_share);
}
__global__ void k_update_b(const ImgDesc* __restrict__ imgs) {
    const ImgDesc& g = imgs[blockIdx.y];
    update_body(g.st, g.comps, g.hist, g.dp, g.H, g.W);
}
__global__ void __launch_bounds__(256) k_build_weights_b(const ImgDesc* __restrict__ imgs) {
    const ImgDesc& g = imgs[blockIdx.y];
    build_weights_body(g.st, &g.st->stopped, g.wbuf);
}
// Every image may run n_iter more iterations (the batch counterpart of the
// host-side stop reset of asp_minor_cycle).
__global__ void k_arm_b(const ImgDesc* __restrict__ imgs, int n, int n_iter) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    CycleState* st = imgs[i].st;
    st->t_stop = st->t + n_iter;
    st->stopped = 0;
    st->stop_reason = 0;
}

// CTA groups of the batched fit for this iteration: image i asks for its
// fit's grid (capped by its g_share when select ran); if the requests exceed
// g_total they are scaled down proportionally (at least one CTA each).  The
// granted grid is written back into the image's fit descriptor (and whether
// the window still fits the group's shared memory), the CTA ranges to dmap.
__global__ void k_fit_map_b(const ImgDesc* __restrict__ imgs, int n, int g_total, int* __restrict__ dmap) {
    __shared__ int req[MAX_BATCH];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const FitDesc& f = imgs[i].st->fit;
        req[i] = f.active ? max(f.grid, 1) : 0;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    long long total = 0;
    for (int i = 0; i < n; ++i) total += req[i];
    if (total > g_total) {
        long long sum = 0;
        for (int i = 0; i < n; ++i) {
            if (!req[i]) continue;
            const int sh = (int)((long long)req[i] * g_total / total);
            req[i] = sh > 1 ? sh : 1;
            sum += req[i];
        }
        while (sum > g_total) {                 // trim the largest groups (n <= g_total: this ends)
            int j = 0;
            for (int i = 1; i < n; ++i) if (req[i] > req[j]) j = i;
            if (req[j] <= 1) break;
            req[j] -= 1;
            sum -= 1;
        }
    }
    int acc = 0;
    for (int i = 0; i < n; ++i) {
        dmap[i] = acc;
        if (req[i]) {
            FitDesc& f = imgs[i].st->fit;
            const long long Wn = (long long)f.ww * f.wh;
            f.grid = req[i];
            f.smem_ok = fit_smem_ok(Wn, req[i]);
        }
        acc += req[i];
    }
    dmap[n] = acc;
}
cudaError_t launch_fit_map_b(const ImgDesc* imgs, int n, int g_total, int* dmap, cudaStream_t s) {
    k_fit_map_b<<<1, 256, 0, s>>>(imgs, n, g_total, dmap);
    return cudaGetLastError();
}

cudaError_t launch_cycle_begin_b(const ImgDesc* imgs, int n, cudaStream_t s) {
    k_cycle_begin_b<<<dim3(1, n), 32, 0, s>>>(imgs);
    return cudaGetLastError();
}
cudaError_t launch_select_b(const ImgDesc* imgs, int n, cudaStream_t s) {
    k_select_b<<<dim3(1, n), SELECT_THREADS, 0, s>>>(imgs);
    return cudaGetLastError();
}
cudaError_t launch_update_b(const ImgDesc* imgs, int n, cudaStream_t s) {
    k_update_b<<<dim3(1, n), 32, 0, s>>>(imgs);
    return cudaGetLastError();
}
cudaError_t launch_build_weights_b(const ImgDesc* imgs, int n, cudaStream_t s) {
    k_build_weights_b<<<dim3(MAX_TERMS, n), 256, 0, s>>>(imgs);
    return cudaGetLastError();
}
cudaError_t launch_arm_b(const ImgDesc* imgs, int n, int n_iter, cudaStream_t s) {
    k_arm_b<<<(n + 127) / 128, 128, 0, s>>>(imgs, n, n_iter);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ learned initial values
// (see asp_set_mlp).  The plain method has already chosen p*, the members
// and the window (k_select); these kernels only move the new member's LM
// start and apply the fallback rule.

namespace {
__device__ void copy_words(void* dst, const void* src, int bytes) {
    int* d = reinterpret_cast<int*>(dst);
    const int* q = reinterpret_cast<const int*>(src);
    for (int i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = q[i];
}
__device__ void account_fit(CycleState* st, const FitOut& fo, int K) {
    st->pixel_evals += fo.pixel_evals;
    st->fit_flops += (double)fo.pixel_evals * pixel_eval_flops(K);
    st->fit_ex2 += (double)fo.pixel_evals * K;
    st->lm_iters += fo.iters;
    st->lm_passes += fo.passes;
    st->fit_ns_pass += fo.ns_pass;
    st->fit_ns_reduce += fo.ns_reduce;
    st->fit_ns_solve += fo.ns_solve;
    st->fit_ns_factor += fo.ns_factor;
    st->fit_ns_subst += fo.ns_subst;
    st->fit_refinements += fo.refinements;
    st->fit_fallbacks += fo.fallbacks;
}
}  // namespace

// After k_select: keep the plain start (fit2 is the plain method's fit,
// armed once the proposal is known), and write the input patch (divided by
// |R(p*)|, BF16) to Xrow.  One block.
__device__ __forceinline__ void learned_prep_body(CycleState* st, const float* __restrict__ R, int H, int W,
                                                  __nv_bfloat16* __restrict__ Xrow) {
    const bool live = !st->stopped && st->fit.active;
    __syncthreads();
    if (!live) {
        if (threadIdx.x == 0) { st->fit2.active = 0; st->learned_used = 0; st->need_plain = 0; }
        for (int q = threadIdx.x; q < 1024; q += blockDim.x) Xrow[q] = __float2bfloat16(0.f);
        return;
    }
    copy_words(&st->fit2, &st->fit, (int)sizeof(FitDesc));
    const int px = (int)st->init[1], py = (int)st->init[2];
    const float rp = R[(long long)py * W + px];
    const float inv = rp != 0.f ? 1.0f / fabsf(rp) : 0.f;
    for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
        const int y = py - 16 + (q >> 5), x = px - 16 + (q & 31);
        const float v = (y >= 0 && y < H && x >= 0 && x < W) ? R[(long long)y * W + x] * inv : 0.f;
        Xrow[q] = __float2bfloat16(v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) st->plain_theta[i] = st->fit.theta0[i];
        st->learned_rp = rp;
        st->learned_px = px;
        st->learned_py = py;
        st->fit2.active = 0;
        st->learned_used = 0;
        st->need_plain = 0;
    }
}
__global__ void k_learned_prep(CycleState* st, const float* __restrict__ R, int H, int W, __nv_bfloat16* Xrow) {
    learned_prep_body(st, R, H, W, Xrow);
}

// After the network: the learned start of the new member (y = the network's
// 4 outputs), used when it is finite, inside the window and the width
// bounds.  Then both fits run -- fit from the learned start, fit2 from the
// plain one -- and the lower chi^2 is kept (k_learned_pick).  g_pair > 0
// (a context, both fits in one launch): each fit's group is capped at half
// of the g_pair co-resident CTAs.
__device__ __forceinline__ void learned_apply_body(CycleState* st, const float* __restrict__ y, int g_pair) {
    if (threadIdx.x != 0) return;
    FitDesc& f = st->fit;
    if (st->stopped || !f.active) return;
    const double a0 = (double)y[0] * st->learned_rp;
    const double w0 = st->omega_b * exp((double)y[1]);
    const double x0 = st->learned_px + (double)y[2];
    const double y0 = st->learned_py + (double)y[3];
    const bool ok = isfinite(a0) && isfinite(w0) && isfinite(x0) && isfinite(y0) && a0 != 0.0 && w0 > f.omega_min &&
                    !(w0 > f.omega_max) && !(x0 < f.bx0) && !(x0 > f.bx1) && !(y0 < f.by0) && !(y0 > f.by1);
    if (!ok) return;                                   // the plain fit alone
    f.theta0[0] = a0; f.theta0[1] = x0; f.theta0[2] = y0; f.theta0[3] = w0;
    st->learned_used = 1;
    st->learned_fits += 1;
    FitDesc& f2 = st->fit2;
    f2.active = 1;
    st->need_plain = 1;
    if (g_pair > 0) {
        const long long Wn = (long long)f.ww * f.wh;
        const int ga = g_pair / 2, gb = g_pair - ga;
        if (f.grid > ga) { f.grid = ga; f.smem_ok = fit_smem_ok(Wn, ga); }
        if (f2.grid > gb) { f2.grid = gb; f2.smem_ok = fit_smem_ok(Wn, gb); }
    }
}
__global__ void k_learned_apply(CycleState* st, const float* __restrict__ y, int g_pair) {
    learned_apply_body(st, y, g_pair);
}

// After both fits: the learned start's result is kept when it is finite,
// above the width bound and its chi^2 is not above the plain start's fit's;
// otherwise the plain fit is (the fallback).  The other fit's work is
// counted here (the kept one by k_update).
__device__ __forceinline__ void learned_pick_body(CycleState* st) {
    const bool go = st->need_plain != 0;
    __syncthreads();
    if (!go) return;
    const FitOut& fl = st->fout;
    const bool plain_better = !isfinite(fl.chi2) || !(fl.theta[3] > st->fit.omega_min) || !(fl.chi2 <= st->fout2.chi2);
    __syncthreads();
    if (threadIdx.x == 0) account_fit(st, plain_better ? st->fout : st->fout2, st->fit.K);
    __syncthreads();
    if (plain_better) copy_words(&st->fout, &st->fout2, (int)sizeof(FitOut));
    __syncthreads();
    if (threadIdx.x == 0) {
        if (plain_better) {
            for (int i = 0; i < 4; ++i) st->fit.theta0[i] = st->plain_theta[i];
            st->learned_refits += 1;
        } else {
            st->learned_kept += 1;
        }
        st->fit2.active = 0;
        st->need_plain = 0;
    }
}
__global__ void k_learned_pick(CycleState* st) { learned_pick_body(st); }

// Training-data harvest, after k_update (R not yet updated): record t-1.
__device__ __forceinline__ void harvest_body(const CycleState* __restrict__ st, const float* __restrict__ R, int H, int W,
                                             float* __restrict__ patches, float* __restrict__ targets, int capacity,
                                             int last_t) {
    const int t = st->t - 1;
    if (st->t == last_t || t < 0 || t >= capacity || !st->fit.active) return;   // no new iteration ran
    const int px = (int)st->init[1], py = (int)st->init[2];
    const double rp = R[(long long)py * W + px];
    const float inv = rp != 0.0 ? (float)(1.0 / fabs(rp)) : 0.f;
    float* pt = patches + (long long)t * 1024;
    for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
        const int y = py - 16 + (q >> 5), x = px - 16 + (q & 31);
        pt[q] = (y >= 0 && y < H && x >= 0 && x < W) ? R[(long long)y * W + x] * inv : 0.f;
    }
    if (threadIdx.x == 0) {
        const double* th = st->fout.theta;
        float* tg = targets + (long long)t * 8;
        tg[0] = (float)(th[0] / rp);
        tg[1] = (float)log(th[3] / st->omega_b);
        tg[2] = (float)(th[1] - px);
        tg[3] = (float)(th[2] - py);
        tg[4] = (float)rp;
        tg[5] = (float)px;
        tg[6] = (float)py;
        tg[7] = (float)st->fout.status;
    }
}
__global__ void k_harvest(const CycleState* __restrict__ st, const float* __restrict__ R, int H, int W, float* patches,
                          float* targets, int capacity) {
    harvest_body(st, R, H, W, patches, targets, capacity, -1);
}


// Batched learned-initial-value steps (grid.y = image): 0 prep, 1 apply,
// 2 check, 3 pick.
__global__ void k_learned_b(const ImgDesc* __restrict__ imgs, int step) {
    const ImgDesc& g = imgs[blockIdx.y];
    // step 0: patch; 1: the learned start (both fits run as two launches,
    // so no group caps); 2: keep the better fit
    if (step == 0) learned_prep_body(g.st, g.R, g.H, g.W, reinterpret_cast<__nv_bfloat16*>(g.Xrow));
    else if (step == 1) learned_apply_body(g.st, g.Yrow, 0);
    else learned_pick_body(g.st);
}
cudaError_t launch_learned_b(const ImgDesc* imgs, int n, int step, cudaStream_t s) {
    k_learned_b<<<dim3(1, n), 256, 0, s>>>(imgs, step);
    return cudaGetLastError();
}

cudaError_t launch_learned_prep(CycleState* st, const float* R, int H, int W, void* Xrow, cudaStream_t s) {
    k_learned_prep<<<1, 256, 0, s>>>(st, R, H, W, reinterpret_cast<__nv_bfloat16*>(Xrow));
    return cudaGetLastError();
}
cudaError_t launch_learned_apply(CycleState* st, const float* y, int g_pair, cudaStream_t s) {
    k_learned_apply<<<1, 32, 0, s>>>(st, y, g_pair);
    return cudaGetLastError();
}
cudaError_t launch_learned_pick(CycleState* st, cudaStream_t s) {
    k_learned_pick<<<1, 256, 0, s>>>(st);
    return cudaGetLastError();
}
cudaError_t launch_harvest(const CycleState* st, const float* R, int H, int W, float* patches, float* targets,
                           int capacity, cudaStream_t s) {
    k_harvest<<<1, 256, 0, s>>>(st, R, H, W, patches, targets, capacity);
    return cudaGetLastError();
}

cudaError_t launch_cycle_begin(CycleState* st, const Params& p, int H, int W, double smooth_flops, cudaStream_t s) {
    k_cycle_begin<<<1, 32, 0, s>>>(st, p, H, W, smooth_flops);
    return cudaGetLastError();
}

cudaError_t launch_select(CycleState* st, const asp_component* comps, const Params& p, int H, int W, int g_max,
                          cudaStream_t s) {
    k_select<<<1, SELECT_THREADS, 0, s>>>(st, comps, p, H, W, g_max);
    return cudaGetLastError();
}

cudaError_t launch_update(CycleState* st, asp_component* comps, asp_iter_record* hist, const Params& p, int H,
                          int W, cudaStream_t s) {
    k_update<<<1, 32, 0, s>>>(st, comps, hist, p, H, W);
    return cudaGetLastError();
}

cudaError_t launch_build_weights(CycleState* st, const int* gate, float* wbuf, cudaStream_t s) {
    k_build_weights<<<MAX_TERMS, 256, 0, s>>>(st, gate, wbuf);
    return cudaGetLastError();
}

cudaError_t launch_terms_from_components(CycleState* st, const asp_component* comps, int n, float gain, int H,
                                         int W, cudaStream_t s) {
    k_terms_from_components<<<1, 32, 0, s>>>(st, comps, n, gain, H, W);
    return cudaGetLastError();
}

cudaError_t launch_reset_state(CycleState* st, cudaStream_t s) {
    k_reset_state<<<1, 32, 0, s>>>(st);
    return cudaGetLastError();
}

}  // namespace aspd
