// One Gauss-Newton pass over a problem's patch chunks, for problems with at
// most kTcMaxFree free poses (Deep Patch Visual Odometry, Sec. 3.1, Eq. 6;
// reprojection Eq. 2-3; damping in the Appendix "Bundle Adjustment Layer").
//
// gn_pass_kernel, launch t of a solve (one CTA per work item = a range of
// chunks of one problem; 256 threads; two CTAs per SM):
//
//   (A, B) t > 0: back-substitution of iteration t-1's pose increment.  The
//          depth row of the normal equations gives
//              dd_k = (w_k - sum_a e_ak^T dxi_a) / C_k,
//          and sum_a e_ak^T dxi_a = sum over patch k's edges of
//          J_d^T W (J_i dxi_i + J_j dxi_j).  Instead of storing each patch's
//          coupling row e_k, every edge recomputes, at iterate t-1, the change
//          of its reprojected point along the increment,
//              dX = K_ij pbar + d h_ij,
//              K_ij = [w_j]x R_ij - R_ij [w_i]x,  h_ij = v_j + w_j x t_ij - R_ij v_i
//          (the left perturbations of poses j and i acting on X = R_ij pbar +
//          t_ij d), projects it with d pi / d X and weights it with J_d; C_k
//          and w_k come from iteration t-1's pass (two floats per patch).
//          Edges between two fixed poses contribute nothing here.
//   (C)    t < iters: linearisation at iterate t.  Thread (frame j, patch
//          group) walks the chunk's patches: residual, J_d and, where a pose
//          of the edge is free, J_j and the weighted products
//              M_j += J_j^T W J_j, v_j += J_j^T W r   (registers, per frame),
//              e_jk = J_j^T W J_d                     (operand column, FP32),
//          C_k, w_k and the anchor column's Y terms into per-slot sums.
//   (D)    per patch: C_k = lambda + sum C_e, w_k, the anchor column
//          e_ik = -[d Y; pbar x Y]; the patch's pose column scaled by
//          C_k^-1/2 is split into TF32 halves hi = rna(x), lo = rna(x - hi)
//          in a K-major tensor-core operand [lo; hi] (patches along K).
//   (E)    one thread issues tcgen05.mma kind::tf32, M = 128, N = 64: D = [lo;
//          hi] . hi^T accumulates lo.hi^T (TMEM lanes 0-63) and hi.hi^T (lanes
//          64-127) in FP32; rows 62/63 of hi carry C_k^-1/2 w_k in two halves,
//          so v' comes out of the same product.  The tensor core truncates
//          its FP32 accumulation, so the large hi.hi^T block is drained into
//          FP32 sums in shared memory every kGpDrainEvery chunks (a fresh
//          accumulation follows, which restarts both halves of D, so both are
//          drained).
//   Group end (the last chunk of an anchor's run): the per-frame sums M_j,
//          v_j are combined over patch groups and the pose-pair blocks
//          B_jj = M_j, B_ij = -Ad_ij^T M_j, B_ii = sum_j Ad_ij^T M_j Ad_ij go
//          into the CTA's FP64 partial of (S, v') in global memory.
//   End:   S -= hi.hi^T + lo.hi^T + (lo.hi^T)^T, v' -= its w columns, in the
//          partial (the strip layout the reduced solve reads).
//
// The last launch (t = iters) runs (A, B) only and writes the caller's
// inverse depths (and, in item 0, the poses).  No atomics: the result is
// bitwise reproducible.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "ba_common.cuh"
#include "kernels.cuh"
#include "se3.cuh"
#include "tc.cuh"

namespace dpvo {

constexpr int kGpDrainEvery = 2;       // chunks of MMAs accumulated in TMEM before hi.hi^T is drained
constexpr int kGpDaccLd = 68;          // row stride (floats) of the drained [lo.hi^T; hi.hi^T] sums
constexpr int kGpWin = 72;             // floats of window data per frame
constexpr int kGpMpHalf = 14;          // frame sums (of 27) parked per thread at a time at a group end

// Shared-memory layout of gn_pass_kernel for window cap W, chunk cap G, frames n_max.
struct GpSmem {
    int W, G, Gs, Gs1, Kc;
    uint32_t sbo;
    size_t off_pnew, off_pold, off_dxs, off_win, off_rjj, off_rtg, off_rwt, off_rpx, off_rpy, off_rdep, off_rseg,
        off_rcw, off_idx, off_u, off_sc1, off_pd, off_op, off_dacc, off_mc, bytes;
};

__host__ __device__ inline GpSmem gp_smem_layout(int W, int G, int n_max) {
    GpSmem s;
    s.W = W;
    s.G = G;
    s.Gs = G + ((2 - G) % 8 + 8) % 8;       // float4 slot stride (see lin_smem_layout)
    s.Gs1 = G + ((8 - G) % 16 + 16) % 16;   // float slot stride
    s.Kc = (G + 7) & ~7;
    s.sbo = (uint32_t)(s.Kc / 4) * 144u;
    const size_t EC = (size_t)W * G;
    const size_t slots4 = (size_t)W * s.Gs, slots1 = (size_t)W * s.Gs1;
    size_t o = 0;
    s.off_pnew = o; o = align16(o + (size_t)n_max * 7 * 4);
    s.off_pold = o; o = align16(o + (size_t)n_max * 7 * 4);
    s.off_dxs = o;  o = align16(o + (size_t)6 * kMaxFree * 4);
    s.off_win = o;  o = align16(o + (size_t)W * kGpWin * 4);
    s.off_rjj = o;  o = align16(o + (EC + 8) * 4);
    s.off_rtg = o;  o = align16(o + (EC + 2) * 8);
    s.off_rwt = o;  o = align16(o + (EC + 2) * 8);
    s.off_rpx = o;  o = align16(o + (size_t)G * 4);
    s.off_rpy = o;  o = align16(o + (size_t)G * 4);
    s.off_rdep = o; o = align16(o + (size_t)G * 4);
    s.off_rseg = o; o = align16(o + (size_t)(G + 1) * 4);
    s.off_rcw = o;  o = align16(o + (size_t)G * 8);
    s.off_idx = o;  o = align16(o + slots4 * 2);
    // union: per-slot sums (sc4 float4 | sc1 float, the back-substitution
    // terms sharing sc1) during a chunk; at a group end one half of the
    // per-thread frame sums at a time, then the anchor-pair products
    const size_t u_slots = align16(slots4 * 16) + slots1 * 4;
    const size_t u_mp = (size_t)kThreads * kGpMpHalf * 4;
    const size_t u_pair = align16((size_t)W * 42 * 4) * 2;
    size_t u = u_slots;
    if (u_mp > u) u = u_mp;
    if (u_pair > u) u = u_pair;
    s.off_u = o;
    s.off_sc1 = o + align16(slots4 * 16);
    o = align16(o + u);
    s.off_pd = o;   o = align16(o + (size_t)G * 16);
    s.off_op = o;   o = align16(o + (size_t)16 * s.sbo);
    s.off_dacc = o; o = align16(o + (size_t)2 * kTcRows * kGpDaccLd * 4);
    s.off_mc = o;   o = align16(o + (size_t)W * 27 * 4);
    s.bytes = o;
    return s;
}

// Start copying one chunk's inputs: frames, targets and weights of its edges
// (bulk copies on `bar` where aligned), its patches' centres and inverse
// depths (depth_src), patch -> edge offsets, the previous pass's (C_k, w_k)
// when cw != nullptr, and the descriptor of the chunk after it.
__device__ __forceinline__ void gp_prefetch(const Prob &pr, const Chunk &ch, const float *depth_src, int *rjj,
                                            float2 *rtg, float2 *rwt, float *rpx, float *rpy, float *rdep, int *rseg,
                                            float2 *rcw, const Chunk *desc_src, Chunk *desc_dst, uint32_t bar) {
    prefetch_chunk(pr, ch, depth_src, rjj, rtg, rwt, rpx, rpy, rdep, rseg, desc_src, desc_dst, bar);
    if (rcw) {
        const float2 *cw = reinterpret_cast<const float2 *>(pr.cw);
        for (int q = threadIdx.x; q < ch.count; q += kThreads) cp_async8(rcw + q, cw + ch.k0 + q);
        cp_async_commit();
    }
}

// Window data of frame jl (W frames from jlo, relative to the anchor):
//   [0, 12)  R_ij, t_ij at iterate t;   [12, 48) Ad(G_ij) at iterate t;
//   [48, 60) R_ij, t_ij at iterate t-1; [60, 72) K_ij (row-major), h_ij of
//   the back-substitution (iteration t-1's increment, zero for fixed poses).
__device__ __forceinline__ void gp_window(const Prob &pr, const float *pnew, const float *pold, const float *dxs,
                                          int anc, int jlo, int W, bool lin, bool bs, float *win) {
    for (int jl = threadIdx.x; jl < W; jl += kThreads) {
        float *wd = win + jl * kGpWin;
        const int j = jlo + jl;
        if (lin) {
            relative_pose(pnew + 7 * anc, pnew + 7 * j, wd, wd + 9);
            adjoint6(wd, wd + 9, wd + 12);
        }
        if (bs) {
            float *R = wd + 48, *tt = wd + 57, *K = wd + 60, *h = wd + 69;
            relative_pose(pold + 7 * anc, pold + 7 * j, R, tt);
            float vi[3] = {0.f, 0.f, 0.f}, wi[3] = {0.f, 0.f, 0.f}, vj[3] = {0.f, 0.f, 0.f}, wj[3] = {0.f, 0.f, 0.f};
            if (anc >= pr.t0)
                for (int m = 0; m < 3; ++m) { vi[m] = dxs[6 * (anc - pr.t0) + m]; wi[m] = dxs[6 * (anc - pr.t0) + 3 + m]; }
            if (j >= pr.t0)
                for (int m = 0; m < 3; ++m) { vj[m] = dxs[6 * (j - pr.t0) + m]; wj[m] = dxs[6 * (j - pr.t0) + 3 + m]; }
            // K = [wj]x R - R [wi]x
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    // ([wj]x R)_rc = (wj x R_col c)_r
                    const float a = wj[(r + 1) % 3] * R[3 * ((r + 2) % 3) + c] - wj[(r + 2) % 3] * R[3 * ((r + 1) % 3) + c];
                    // (R [wi]x)_rc = sum_m R_rm ([wi]x)_mc, ([wi]x)_mc = eps_{m i c} wi_i
                    const float b = R[3 * r + (c + 1) % 3] * wi[(c + 2) % 3] - R[3 * r + (c + 2) % 3] * wi[(c + 1) % 3];
                    K[3 * r + c] = a - b;
                }
            // h = vj + wj x t - R vi
            for (int r = 0; r < 3; ++r)
                h[r] = vj[r] + (wj[(r + 1) % 3] * tt[(r + 2) % 3] - wj[(r + 2) % 3] * tt[(r + 1) % 3]) -
                       (R[3 * r] * vi[0] + R[3 * r + 1] * vi[1] + R[3 * r + 2] * vi[2]);
        }
    }
}

// One edge's back-substitution term at iterate t-1: J_d^T W (d pi/d X) dX for
// dX = K pbar + d h (R, t the relative pose), or 0 if the edge takes no part.
__device__ __forceinline__ float gp_bs_term(const float *R, const float *K, float px, float py, float d, float w0,
                                            float w1, float fx2, float fy2, float z_min) {
    const float X = fmaf(R[9], d, fmaf(R[1], py, fmaf(R[0], px, R[2])));
    const float Y = fmaf(R[10], d, fmaf(R[4], py, fmaf(R[3], px, R[5])));
    const float Z = fmaf(R[11], d, fmaf(R[7], py, fmaf(R[6], px, R[8])));
    if (!(Z > z_min)) return 0.f;
    const float iz = 1.0f / Z;
    const float a = X * iz, b = Y * iz;
    const float dx = fmaf(K[9], d, fmaf(K[1], py, fmaf(K[0], px, K[2])));
    const float dy = fmaf(K[10], d, fmaf(K[4], py, fmaf(K[3], px, K[5])));
    const float dz = fmaf(K[11], d, fmaf(K[7], py, fmaf(K[6], px, K[8])));
    // J_d = (fx iz (t0 - a t2), fy iz (t1 - b t2)); (d pi/d X) dX = (fx iz (dx - a dz), fy iz (dy - b dz))
    const float u0 = fmaf(-a, R[11], R[9]), u1 = fmaf(-b, R[11], R[10]);
    const float g0 = fmaf(-a, dz, dx), g1 = fmaf(-b, dz, dy);
    return (iz * iz) * fmaf(w1 * fy2 * u1, g1, w0 * fx2 * u0 * g0);
}

// Add the TMEM accumulator D (128 lanes x 64 FP32 columns) into the FP32 sums
// dacc [128][kGpDaccLd]: warp w reads lanes 32 (w % 4) .. + 31 (the quarter it
// may access) and columns 32 (w / 4) .. + 31; a thread adds its row's 32
// values with 16-byte shared-memory accesses (the padded stride keeps a
// quarter warp's rows in distinct banks).
__device__ __forceinline__ void gp_drain(uint32_t tmem, float *dacc, int warp, int lane) {
    const int row = 32 * (warp & 3) + lane, c0 = 32 * (warp >> 2);
    float4 *dr = reinterpret_cast<float4 *>(dacc + row * kGpDaccLd + c0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + 16 * h), v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 a = dr[4 * h + q];
            a.x += v[4 * q]; a.y += v[4 * q + 1]; a.z += v[4 * q + 2]; a.w += v[4 * q + 3];
            dr[4 * h + q] = a;
        }
    }
}

__global__ void __launch_bounds__(kThreads, 2) gn_pass_kernel(const Prob *__restrict__ probs,
                                                              const Item *__restrict__ items, int t, int W_cap,
                                                              int G_cap, int n_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Item itm = items[blockIdx.x];
    const Prob &pr = probs[itm.prob];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (t > pr.iters) return;
    const bool do_bs = t > 0;
    const bool do_lin = t < pr.iters;
    __shared__ int s_st;
    if (tid == 0) s_st = *pr.status;
    __syncthreads();
    if (!do_lin && itm.item == 0 && tid == 0 && pr.status_user) *pr.status_user = s_st;
    if (s_st != 0) return;

    const GpSmem L = gp_smem_layout(W_cap, G_cap, n_max);
    float *pnew = reinterpret_cast<float *>(smem + L.off_pnew);
    float *pold = reinterpret_cast<float *>(smem + L.off_pold);
    float *dxs = reinterpret_cast<float *>(smem + L.off_dxs);
    float *win = reinterpret_cast<float *>(smem + L.off_win);
    int *rjj_s = reinterpret_cast<int *>(smem + L.off_rjj);
    float2 *rtg_s = reinterpret_cast<float2 *>(smem + L.off_rtg);
    float2 *rwt_s = reinterpret_cast<float2 *>(smem + L.off_rwt);
    float *rpx = reinterpret_cast<float *>(smem + L.off_rpx);
    float *rpy = reinterpret_cast<float *>(smem + L.off_rpy);
    float *rdep = reinterpret_cast<float *>(smem + L.off_rdep);
    int *rseg = reinterpret_cast<int *>(smem + L.off_rseg);
    float2 *rcw = reinterpret_cast<float2 *>(smem + L.off_rcw);
    short *sidx = reinterpret_cast<short *>(smem + L.off_idx);
    float4 *sc4 = reinterpret_cast<float4 *>(smem + L.off_u);
    float *sc1 = reinterpret_cast<float *>(smem + L.off_sc1);   // also the back-substitution terms
    float *Mp = reinterpret_cast<float *>(smem + L.off_u);      // group end: per-thread frame sums
    float *Aj = reinterpret_cast<float *>(smem + L.off_u);      // then the anchor-pair products
    float *Bp = reinterpret_cast<float *>(smem + L.off_u + align16((size_t)W_cap * 42 * 4));
    float4 *pd = reinterpret_cast<float4 *>(smem + L.off_pd);
    unsigned char *op = smem + L.off_op;
    float *dacc = reinterpret_cast<float *>(smem + L.off_dacc);   // drained [lo.hi^T; hi.hi^T]
    float *Mc = reinterpret_cast<float *>(smem + L.off_mc);
    const int Gs = L.Gs, Gs1 = L.Gs1;
    const uint32_t sbo = L.sbo;
    __shared__ float Bii[42];

    const int N = pr.N, t0 = pr.t0, nf = pr.nf, n6 = 6 * nf;
    const float fx = pr.fx, fy = pr.fy, cx = pr.cx, cy = pr.cy, z_min = pr.z_min, lam = pr.damping;
    const float ifx = 1.0f / fx, ify = 1.0f / fy, fx2 = fx * fx, fy2 = fy * fy;
    const float *pose_t = pr.pose_it + (size_t)t * N * 7;
    float *depth_t = pr.depth_it + (size_t)t * pr.P;
    const float *depth_src = pr.depth_it + (size_t)(do_bs ? t - 1 : t) * pr.P;

    const int nch = *pr.n_chunks;
    const int c_begin = (int)(((long long)itm.item * nch) / pr.n_items);
    const int c_end = (int)(((long long)(itm.item + 1) * nch) / pr.n_items);

    for (int q = tid; q < N * 7; q += kThreads) {
        pnew[q] = pose_t[q];
        if (do_bs) pold[q] = pose_t[q - N * 7];
    }
    if (do_bs)
        for (int q = tid; q < 6 * nf; q += kThreads) dxs[q] = (float)pr.dxi[(size_t)(t - 1) * nf * 6 + q];
    if (!do_lin && itm.item == 0 && !pr.no_writeback)
        for (int q = tid; q < N * 7; q += kThreads) pr.poses[q] = pose_t[q];

    // tensor-core state: 64 TMEM columns, the MMA-completion mbarrier
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ __align__(8) uint64_t s_ldbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_bad;
    const bool use_tc = do_lin && nf > 0;
    const uint32_t mbar = smem_u32(&s_mbar), ldbar = smem_u32(&s_ldbar);
    if (tid == 0) {
        mbar_init(ldbar, 1);
        if (use_tc) mbar_init(mbar, 1);
        s_bad = 0;
    }
    if (use_tc && warp == 0) tmem_alloc(&s_tmem, 64);
    if (use_tc) {
        uint4 *o4 = reinterpret_cast<uint4 *>(op);
        for (int q = tid; q < (int)(16 * sbo / 16); q += kThreads) o4[q] = make_uint4(0u, 0u, 0u, 0u);
        for (int q = tid; q < 2 * kTcRows * kGpDaccLd; q += kThreads) dacc[q] = 0.f;
    }
    if (do_lin) {
        double *part = pr.partial + (size_t)itm.item * pr.L;
        for (int q = tid; q < pr.L; q += kThreads) part[q] = 0.0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = use_tc ? s_tmem : 0u;

    __shared__ __align__(16) Chunk s_ch[2];
    if (c_begin < c_end) {
        if (tid == 0) s_ch[0] = pr.chunks[c_begin];
        __syncthreads();
        gp_prefetch(pr, s_ch[0], depth_src, rjj_s, rtg_s, rwt_s, rpx, rpy, rdep, rseg, do_bs ? rcw : nullptr,
                    c_begin + 1 < c_end ? pr.chunks + c_begin + 1 : nullptr, &s_ch[1], ldbar);
    }

    int cur = 0;
    bool group_open = false;
    int n_commit = 0;     // MMA batches committed (the same in every thread)
    int in_block = 0;     // chunks accumulated in TMEM since the last drain
    float M[21], V[6];
#pragma unroll
    for (int q = 0; q < 21; ++q) M[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 6; ++q) V[q] = 0.f;

    for (int c = c_begin; c < c_end; ++c) {
        const Chunk ch = s_ch[cur];
        const bool have_next = c + 1 < c_end;
        cp_async_wait_all();
        if (!mbar_wait(ldbar, (uint32_t)(c - c_begin) & 1u)) atomicOr(&s_bad, 1);
        // the previous chunk's MMAs read the operand, which this chunk rewrites
        if (use_tc && n_commit > 0 && !mbar_wait(mbar, (uint32_t)(n_commit - 1) & 1u)) atomicOr(&s_bad, 2);
        __syncthreads();
        if (s_bad) break;
        int o_jj, o_tw;
        staged_offsets(pr, ch, true, o_jj, o_tw);
        Chunk nx = ch;
        if (have_next) nx = s_ch[cur ^ 1];
        const bool group_next = have_next && nx.anchor == ch.anchor && nx.jlo == ch.jlo && nx.jhi == ch.jhi;
        const int k0 = ch.k0, cnt = ch.count, e0 = ch.e0;
        const int anc = ch.anchor, jlo = ch.jlo;
        const int W = ch.jhi - jlo + 1;
        const bool anc_free = anc >= t0;
        const int NG = kThreads / W;
        const int my_g = tid % NG, my_jl = tid / NG;
        const int my_j = jlo + my_jl;
        const bool edge_thread = my_jl < W;
        const bool j_free = my_j >= t0;
        const int fj = my_j - t0;
        const bool pose_terms = edge_thread && my_j != anc && (anc_free || j_free);
        int lp_sh = 2;
        const int LP = lanes_per_patch(cnt, &lp_sh);
        const int ps_sh = 8 - lp_sh, PSm = (1 << ps_sh) - 1;

        // -- (0) slot -> staged edge table, patch data, window, cleared operand columns
        {
            const int p = tid & PSm;
            if (p < cnt) {
                const int a = rseg[p] - e0, b = rseg[p + 1] - e0;
                int jf = 0, jz = -1;
                bool contig = true;
                if (b > a) {
                    jf = rjj_s[o_jj + a];
                    jz = rjj_s[o_jj + b - 1];
                    contig = jz - jf + 1 == b - a;
                }
                for (int jl = tid >> ps_sh; jl < W; jl += kThreads >> ps_sh) {
                    const int j = jlo + jl;
                    int idx = -1;
                    if (j >= jf && j <= jz) {
                        if (contig) {
                            idx = a + (j - jf);
                        } else {
                            int lo = a, hi = b - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (rjj_s[o_jj + mid] < j) lo = mid + 1; else hi = mid;
                            }
                            if (rjj_s[o_jj + lo] == j) idx = lo;
                        }
                    }
                    sidx[jl * Gs + p] = (short)(idx >= 0 ? idx + o_tw : -1);
                }
                if (use_tc)
                    for (int f = tid >> ps_sh; f < nf; f += kThreads >> ps_sh) {   // free frames outside the window
                        const int fr = t0 + f;
                        if (fr < jlo || fr > ch.jhi)
#pragma unroll
                            for (int m = 0; m < 6; ++m)
                                *reinterpret_cast<float *>(op + op_offset(kTcRows + 6 * f + m, p, sbo)) = 0.f;
                    }
            }
            for (int q = tid; q < cnt; q += kThreads)
                pd[q] = make_float4((rpx[q] - cx) * ifx, (rpy[q] - cy) * ify, rdep[q], 0.f);
            if (!group_open) gp_window(pr, pnew, pold, dxs, anc, jlo, W, do_lin, do_bs, win);
        }
        __syncthreads();

        if (do_bs) {
            // -- (A) back-substitution terms of iteration t-1, per slot
            if (edge_thread) {
                float Rb[12], Kb[12];
                const float *wd = win + my_jl * kGpWin;
#pragma unroll
                for (int q = 0; q < 12; ++q) { Rb[q] = wd[48 + q]; Kb[q] = wd[60 + q]; }
                for (int p = my_g; p < cnt; p += NG) {
                    float s = 0.f;
                    const int idx = sidx[my_jl * Gs + p];
                    if (pose_terms && idx >= 0) {
                        const float2 wv = rwt_s[idx];
                        const float4 q = pd[p];
                        s = gp_bs_term(Rb, Kb, q.x, q.y, q.z, wv.x, wv.y, fx2, fy2, z_min);
                    }
                    sc1[my_jl * Gs1 + p] = s;
                }
            }
            __syncthreads();
            // -- (B) dd_k = (w_k - sum) / C_k, the new inverse depth
            {
                const int p = tid >> lp_sh, sub = tid & (LP - 1);
                float s = 0.f;
                if (p < cnt)
                    for (int jl = sub; jl < W; jl += LP) s += sc1[jl * Gs1 + p];
                s = lane_group_sum(s, LP);
                if (sub == 0 && p < cnt) {
                    const float2 cw = rcw[p];
                    const float d = rdep[p] + (cw.y - s) / cw.x;
                    depth_t[k0 + p] = d;
                    pd[p].z = d;
                    if (!do_lin && !pr.no_writeback) pr.patches[3 * (k0 + p) + 2] = d;
                }
            }
            __syncthreads();
            if (!do_lin) {   // last launch: the staging buffers are free
                if (have_next)
                    gp_prefetch(pr, nx, depth_src, rjj_s, rtg_s, rwt_s, rpx, rpy, rdep, rseg, rcw,
                                c + 2 < c_end ? pr.chunks + c + 2 : nullptr, &s_ch[cur], ldbar);
                group_open = group_next;
                cur ^= 1;
                continue;
            }
        }

        // -- (C) linearise at iterate t
        if (edge_thread) {
            if (!group_open) {
#pragma unroll
                for (int q = 0; q < 21; ++q) M[q] = 0.f;
#pragma unroll
                for (int q = 0; q < 6; ++q) V[q] = 0.f;
            }
            float Rr[12];
            const float *wd = win + my_jl * kGpWin;
#pragma unroll
            for (int q = 0; q < 12; ++q) Rr[q] = wd[q];
            for (int p = my_g; p < cnt; p += NG) {
                const int idx = sidx[my_jl * Gs + p];
                float Ce = 0.f, we = 0.f, Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
                float4 elo = make_float4(0.f, 0.f, 0.f, 0.f), ehi = elo;
                if (idx >= 0 && my_j != anc) {
                    const float2 wv = rwt_s[idx];
                    if (wv.x != 0.f || wv.y != 0.f) {
                        const float2 tv = rtg_s[idx];
                        const float4 q = pd[p];
                        EdgeLin E;
                        if (edge_linearize(Rr, Rr + 9, q.x, q.y, q.z, tv.x, tv.y, fx, fy, cx, cy, z_min, E)) {
                            float wjd0, wjd1;
                            depth_terms(E, wv.x, wv.y, wjd0, wjd1, Ce, we);
                            if (anc_free) anchor_terms(E, Rr, wjd0, wjd1, Y0, Y1, Y2);
                            if (pose_terms) {
                                float wj0[6], wj1[6];
#pragma unroll
                                for (int m = 0; m < 6; ++m) { wj0[m] = wv.x * E.j0[m]; wj1[m] = wv.y * E.j1[m]; }
#pragma unroll
                                for (int r = 0; r < 6; ++r)
#pragma unroll
                                    for (int cc = r; cc < 6; ++cc) {
                                        float acc = M[sym6(r, cc)];
                                        if (r != 1 && cc != 1) acc = fmaf(wj0[r], E.j0[cc], acc);
                                        if (r != 0 && cc != 0) acc = fmaf(wj1[r], E.j1[cc], acc);
                                        M[sym6(r, cc)] = acc;
                                    }
#pragma unroll
                                for (int m = 0; m < 6; ++m) {
                                    float vv = V[m];
                                    if (m != 1) vv = fmaf(wj0[m], E.r0, vv);
                                    if (m != 0) vv = fmaf(wj1[m], E.r1, vv);
                                    V[m] = vv;
                                }
                                elo = make_float4(wj0[0] * E.jd0, wj1[1] * E.jd1,
                                                  fmaf(wj1[2], E.jd1, wj0[2] * E.jd0), 0.f);
                                ehi = make_float4(fmaf(wj1[3], E.jd1, wj0[3] * E.jd0),
                                                  fmaf(wj1[4], E.jd1, wj0[4] * E.jd0),
                                                  fmaf(wj1[5], E.jd1, wj0[5] * E.jd0), 0.f);
                            }
                        }
                    }
                }
                if (j_free && my_j != anc) {   // e_jk, unscaled FP32, into the hi half
                    const float ev[6] = {elo.x, elo.y, elo.z, ehi.x, ehi.y, ehi.z};
#pragma unroll
                    for (int m = 0; m < 6; ++m)
                        *reinterpret_cast<float *>(op + op_offset(kTcRows + 6 * fj + m, p, sbo)) = ev[m];
                }
                sc4[my_jl * Gs + p] = make_float4(Ce, we, Y0, Y1);
                sc1[my_jl * Gs1 + p] = Y2;
            }
        }
        __syncthreads();
        // the staging buffers are free: start the next chunk's copies
        if (have_next)
            gp_prefetch(pr, nx, depth_src, rjj_s, rtg_s, rwt_s, rpx, rpy, rdep, rseg, do_bs ? rcw : nullptr,
                        c + 2 < c_end ? pr.chunks + c + 2 : nullptr, &s_ch[cur], ldbar);

        // drain D (lane = row: warp w reads lanes 32 (w % 4) .., columns 32 (w / 4) ..)
        // before this chunk's MMAs start a fresh accumulation
        const bool drain = use_tc && in_block >= kGpDrainEvery;
        if (drain) {
            tc_fence_after();
            gp_drain(tmem, dacc, warp, lane);
            tc_fence_before();
            in_block = 0;
        }

        // -- (D) per patch: C_k, w_k, the anchor column; scale by C_k^-1/2 and split into TF32 halves
        {
            const int p = tid >> lp_sh, sub = tid & (LP - 1);
            float C = sub == 0 ? lam : 0.f, w = 0.f, Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
            if (p < cnt)
                for (int jl = sub; jl < W; jl += LP) {
                    const float4 v = sc4[jl * Gs + p];
                    C += v.x;
                    w += v.y;
                    Y0 += v.z;
                    Y1 += v.w;
                    Y2 += sc1[jl * Gs1 + p];
                }
            C = lane_group_sum(C, LP);
            w = lane_group_sum(w, LP);
            Y0 = lane_group_sum(Y0, LP);
            Y1 = lane_group_sum(Y1, LP);
            Y2 = lane_group_sum(Y2, LP);
            float q = 0.f;
            if (p < cnt) {
                q = sqrtf(1.0f / C);
                if (sub == 0) reinterpret_cast<float2 *>(pr.cw)[k0 + p] = make_float2(C, w);
                if (use_tc && anc_free && sub >= 1 && sub <= 2) {
                    const float4 qd = pd[p];
                    const float d = qd.z, px = qd.x, py = qd.y;
                    float3 v;
                    if (sub == 1) v = make_float3(-d * Y0, -d * Y1, -d * Y2);
                    else          // -(pbar x Y), pbar = (px, py, 1)
                        v = make_float3(-(py * Y2 - Y1), -(Y0 - px * Y2), -(px * Y1 - py * Y0));
                    const int r0 = kTcRows + 6 * (anc - t0) + 3 * (sub - 1);
                    *reinterpret_cast<float *>(op + op_offset(r0, p, sbo)) = v.x;
                    *reinterpret_cast<float *>(op + op_offset(r0 + 1, p, sbo)) = v.y;
                    *reinterpret_cast<float *>(op + op_offset(r0 + 2, p, sbo)) = v.z;
                }
            }
            __syncwarp();
            if (use_tc && p < L.Kc) {
                const bool in = p < cnt;
                for (int r = sub; r < kTcRows - 1; r += LP) {
                    if (r >= n6 && r != kTcRows - 2) continue;
                    const uint32_t off = op_offset(r, p, sbo);
                    uint32_t *lp = reinterpret_cast<uint32_t *>(op + off);
                    uint32_t *hp = reinterpret_cast<uint32_t *>(op + off + (kTcRows / 8) * sbo);
                    float x = 0.f;
                    if (in) x = r < n6 ? __uint_as_float(*hp) * q : q * w;
                    const uint32_t h = to_tf32(x);
                    const uint32_t lo = to_tf32(x - __uint_as_float(h));
                    if (r == kTcRows - 2) {          // hi rows 62, 63: hi and lo of C^-1/2 w
                        hp[0] = h;
                        hp[4] = lo;                  // row 63: 16 bytes on
                    } else {
                        *hp = h;
                        *lp = lo;
                    }
                }
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        // -- (E) the chunk's MMAs, one thread
        if (use_tc) {
            if (tid == 0) {
                tc_fence_after();
                const uint32_t base = smem_u32(op);
                constexpr uint32_t idesc = idesc_tf32(2 * kTcRows, kTcRows);
                const int Ksteps = (cnt + 7) >> 3;
                for (int st = 0; st < Ksteps; ++st) {
                    const uint64_t ad = smem_desc(base + st * 2 * kLbo, kLbo, sbo);
                    const uint64_t bd = smem_desc(base + (kTcRows / 8) * sbo + st * 2 * kLbo, kLbo, sbo);
                    mma_tf32(tmem, ad, bd, idesc, (in_block > 0 || st > 0) ? 1 : 0);
                }
                mma_commit(mbar);
            }
            ++n_commit;
            ++in_block;
        }

        // -- group end: the pose-pair blocks of this anchor's run go into the FP64 partial
        if (!group_next) {
            // combine the per-thread frame sums (M_j, v_j) over patch groups,
            // compensated, one half of the 27 values at a time
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m0 = h * kGpMpHalf, mn = h ? 27 - kGpMpHalf : kGpMpHalf;
                if (edge_thread) {
                    float *mp = Mp + (size_t)tid * kGpMpHalf;
#pragma unroll
                    for (int q = 0; q < kGpMpHalf; ++q) {
                        const int m = m0 + q;
                        if (q < mn) mp[q] = m < 21 ? M[m < 21 ? m : 0] : V[m >= 21 ? m - 21 : 0];
                    }
                }
                __syncthreads();
                for (int q = tid; q < W * mn; q += kThreads) {
                    const int jl = q / mn, m = q - jl * mn;
                    float s = 0.f, cc = 0.f;
                    for (int g = 0; g < NG; ++g) kahan_add(s, cc, Mp[(size_t)(jl * NG + g) * kGpMpHalf + m]);
                    Mc[jl * 27 + m0 + m] = s - cc;
                }
                __syncthreads();
            }
            if (anc_free) {
                for (int q = tid; q < W * 6; q += kThreads) {
                    const int jl = q / 6, r = q - jl * 6;
                    const float *Ad = win + jl * kGpWin + 12;
                    const float *Mj = Mc + jl * 27;
                    float *A = Aj + jl * 42;
                    float *B = Bp + jl * 42;
                    const bool self = jlo + jl == anc;
                    float row[6];
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) {
                        float s = 0.f;
#pragma unroll
                        for (int m = 0; m < 6; ++m) s = fmaf(Ad[6 * m + r], Mj[sym6(m, cc)], s);
                        row[cc] = s;
                        A[6 * r + cc] = s;
                    }
                    float s = 0.f;
#pragma unroll
                    for (int m = 0; m < 6; ++m) s = fmaf(Ad[6 * m + r], Mj[21 + m], s);
                    A[36 + r] = -s;
                    B[36 + r] = self ? 0.f : -s;
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) {
                        float b = 0.f;
#pragma unroll
                        for (int m = 0; m < 6; ++m) b = fmaf(row[m], Ad[6 * m + cc], b);
                        B[6 * r + cc] = self ? 0.f : b;
                    }
                }
                __syncthreads();
                if (tid < 42) {
                    float s = 0.f, cc = 0.f;
                    for (int jl = 0; jl < W; ++jl) kahan_add(s, cc, Bp[jl * 42 + tid]);
                    Bii[tid] = s - cc;
                }
                __syncthreads();
            }
            // each changed strip of the partial: per free pose f, its diagonal
            // block (two strips), its v' strip, and its pair with the anchor
            double *part = pr.partial + (size_t)itm.item * pr.L;
            const int fanc = anc - t0, nbs = 2 * n_block_pairs(nf);
            for (int it5 = tid; it5 < 5 * nf; it5 += kThreads) {
                const int f = it5 / 5, kind = it5 - 5 * f, fr = t0 + f;
                const bool in_w = fr >= jlo && fr < jlo + W;
                int a2 = f, b2 = f, h2 = kind & 1;
                bool vs = false;
                if (kind < 3) {
                    if (!in_w && fr != anc) continue;
                    vs = kind == 2;
                } else {
                    if (!anc_free || fr == anc || !in_w) continue;
                    a2 = min(f, fanc);
                    b2 = max(f, fanc);
                    h2 = kind - 3;
                }
                float add[18];
                if (!strip_block_add(a2, b2, h2, vs, t0, anc, jlo, W, Mc, Aj, Bii, add)) continue;
                if (vs) {
                    double *o = part + 18 * nbs + 6 * a2;
#pragma unroll
                    for (int q = 0; q < 6; ++q) o[q] += (double)add[q];
                } else {
                    const int st = 2 * (a2 * nf - a2 * (a2 - 1) / 2 + (b2 - a2)) + h2;
                    double *o = part + 18 * st;
#pragma unroll
                    for (int q = 0; q < 18; ++q) o[q] += (double)add[q];
                }
            }
            __syncthreads();   // Mp / Aj / Bp are read before the next chunk's slots overwrite them
        }
        group_open = group_next;
        cur ^= 1;
    }
    cp_async_wait_all();
    if (c_begin < c_end && s_bad) {
        // a copy or an MMA batch did not complete in time: report it and give
        // the copies one more bounded wait
        if (tid == 0) {
            atomicOr(pr.status, DPVO_BA_STATUS_TIMEOUT);
            mbar_wait(ldbar, 0u);
            mbar_wait(ldbar, 1u);
        }
    }

    if (use_tc) {
        bool have = n_commit > 0 && s_bad == 0;
        if (n_commit > 0 && !mbar_wait(mbar, (uint32_t)(n_commit - 1) & 1u)) {
            if (tid == 0) atomicOr(pr.status, DPVO_BA_STATUS_TIMEOUT);
            have = false;
        }
        __syncthreads();
        tc_fence_after();
        if (have && in_block > 0) gp_drain(tmem, dacc, warp, lane);   // the last block
        tc_fence_before();
        __syncthreads();
        if (have) {
            // S -= hi.hi^T + lo.hi^T + (lo.hi^T)^T;  v' -= the w columns (hi rows 62, 63)
            double *part = pr.partial + (size_t)itm.item * pr.L;
            const int nbs = 2 * n_block_pairs(nf);
            for (int q = tid; q < pr.L; q += kThreads) {
                float s;
                if (q < 18 * nbs) {
                    const int st = q / 18, e = q - 18 * st;
                    int a, b;
                    decode_pair(st >> 1, nf, a, b);
                    const int m = 6 * a + 3 * (st & 1) + e / 6, n = 6 * b + e % 6;
                    s = dacc[(kTcRows + m) * kGpDaccLd + n] + dacc[m * kGpDaccLd + n] + dacc[n * kGpDaccLd + m];
                } else {
                    const int m = q - 18 * nbs;
                    s = dacc[(kTcRows + m) * kGpDaccLd + kTcRows - 2] + dacc[(kTcRows + m) * kGpDaccLd + kTcRows - 1] +
                        dacc[m * kGpDaccLd + kTcRows - 2];
                }
                part[q] -= (double)s;
            }
        }
        if (warp == 0) {
            tc_fence_after();
            tmem_dealloc(tmem, 64);
        }
    }
}

}  // namespace dpvo
