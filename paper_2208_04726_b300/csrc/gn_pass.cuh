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
//          its FP32 accumulation, so D is drained into FP32 sums in shared
//          memory every kGpDrainEvery chunks (a fresh accumulation follows):
//          A += hi.hi^T / 2 + lo.hi^T over the pose columns (then S's Schur
//          term is A + A^T), and the w columns as v' needs them.
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
constexpr int kGpDaccLd = 68;          // row stride (floats) of the drained sums A (64 rows)
constexpr int kGpWin = 72;             // floats of window data per frame
constexpr int kGpMpHalf = 14;          // frame sums (of 27) parked per thread at a time at a group end

// Shared-memory layout of gn_pass_kernel for window cap W, chunk cap G, frames n_max.
struct GpSmem {
    int W, G, Gs, Gs1, Kc;
    uint32_t sbo;
    size_t off_pnew, off_pold, off_rot, off_dxs, off_win, off_stage, off_idx, off_u, off_sc1, off_pd, off_op,
        off_dacc, off_mc, bytes;
    // one chunk's staging buffers, offsets from a staging base
    size_t st_rjj, st_rtg, st_rwt, st_rpx, st_rpy, st_rdep, st_rseg, st_rcw, st_bytes;
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
    size_t q = 0;
    s.st_rjj = q;  q = align16(q + (EC + 8) * 4);
    s.st_rtg = q;  q = align16(q + (EC + 2) * 8);
    s.st_rwt = q;  q = align16(q + (EC + 2) * 8);
    s.st_rpx = q;  q = align16(q + (size_t)G * 4);
    s.st_rpy = q;  q = align16(q + (size_t)G * 4);
    s.st_rdep = q; q = align16(q + (size_t)G * 4);
    s.st_rseg = q; q = align16(q + (size_t)(G + 1) * 4);
    s.st_rcw = q;  q = align16(q + (size_t)G * 8);
    s.st_bytes = q;
    size_t o = 0;
    s.off_pnew = o; o = align16(o + (size_t)n_max * 7 * 4);
    s.off_pold = o; o = align16(o + (size_t)n_max * 7 * 4);
    s.off_rot = o;  o = align16(o + (size_t)n_max * 18 * 4);
    s.off_dxs = o;  o = align16(o + (size_t)6 * kMaxFree * 4);
    s.off_win = o;  o = align16(o + (size_t)W * kGpWin * 4);
    s.off_stage = o; o = align16(o + s.st_bytes);
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
    // the operand and the drained sums are contiguous: the last launch (no
    // linearisation) stages its next chunk there
    s.off_op = o;   o = align16(o + (size_t)16 * s.sbo);
    s.off_dacc = o; o = align16(o + (size_t)kTcRows * kGpDaccLd * 4);
    if (o - s.off_op < s.st_bytes) o = s.off_op + s.st_bytes;
    s.off_mc = o;   o = align16(o + (size_t)W * 27 * 4);
    s.bytes = o;
    return s;
}

// One chunk's staging buffers.
struct GpStage {
    int *rjj;
    float2 *rtg, *rwt;
    float *rpx, *rpy, *rdep;
    int *rseg;
    float2 *rcw;
};

__device__ __forceinline__ GpStage gp_stage(unsigned char *base, const GpSmem &L) {
    GpStage g;
    g.rjj = reinterpret_cast<int *>(base + L.st_rjj);
    g.rtg = reinterpret_cast<float2 *>(base + L.st_rtg);
    g.rwt = reinterpret_cast<float2 *>(base + L.st_rwt);
    g.rpx = reinterpret_cast<float *>(base + L.st_rpx);
    g.rpy = reinterpret_cast<float *>(base + L.st_rpy);
    g.rdep = reinterpret_cast<float *>(base + L.st_rdep);
    g.rseg = reinterpret_cast<int *>(base + L.st_rseg);
    g.rcw = reinterpret_cast<float2 *>(base + L.st_rcw);
    return g;
}

// TF32 (10 stored mantissa bits) nearest to x, ties away from zero, as bits:
// the 13 dropped bits round the kept ones by an integer add and mask.
__device__ __forceinline__ uint32_t gp_tf32(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

// Start copying one chunk's inputs: frames, targets and weights of its edges
// (bulk copies on `bar` where aligned), its patches' centres and inverse
// depths (depth_src), patch -> edge offsets, the previous pass's (C_k, w_k)
// when cw != nullptr, and the descriptor of the chunk after it.
__device__ __forceinline__ void gp_prefetch(const Prob &pr, const Chunk &ch, const float *depth_src, const GpStage &g,
                                            bool with_cw, const Chunk *desc_src, Chunk *desc_dst, uint32_t bar) {
    prefetch_chunk(pr, ch, depth_src, g.rjj, g.rtg, g.rwt, g.rpx, g.rpy, g.rdep, g.rseg, desc_src, desc_dst, bar);
    if (with_cw) {
        const float2 *cw = reinterpret_cast<const float2 *>(pr.cw);
        for (int q = threadIdx.x; q < ch.count; q += kThreads) cp_async8(g.rcw + q, cw + ch.k0 + q);
        cp_async_commit();
    }
}

// Window data of frame jl (W frames from jlo, relative to the anchor):
//   [0, 12)  R_ij, t_ij at iterate t;   [12, 48) Ad(G_ij) at iterate t;
//   [48, 60) R_ij, t_ij at iterate t-1; [60, 72) K_ij (row-major), h_ij of
//   the back-substitution (iteration t-1's increment, zero for fixed poses).
// Three threads per frame, one per row; rot holds each frame's rotation
// matrix at iterates t (rot) and t-1 (rot + 9 N).
// Step 1: R_ij = R_j R_i^T and t_ij = t_j - R_ij t_i.
__device__ __forceinline__ void gp_window1(const float *pnew, const float *pold, const float *rot, int N, int anc,
                                           int jlo, int W, bool lin, bool bs, float *win) {
    for (int q = threadIdx.x; q < 3 * W; q += kThreads) {
        const int jl = q / 3, r = q - 3 * jl, j = jlo + jl;
        float *wd = win + jl * kGpWin;
#pragma unroll
        for (int st = 0; st < 2; ++st) {
            if (st == 0 ? !lin : !bs) continue;
            const float *Rs = rot + st * 9 * N, *ps = st ? pold : pnew;
            const float *Ri = Rs + 9 * anc, *Rj = Rs + 9 * j;
            float R[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                R[c] = fmaf(Rj[3 * r + 2], Ri[3 * c + 2], fmaf(Rj[3 * r + 1], Ri[3 * c + 1], Rj[3 * r] * Ri[3 * c]));
            float *o = wd + (st ? 48 : 0);
            o[3 * r] = R[0];
            o[3 * r + 1] = R[1];
            o[3 * r + 2] = R[2];
            const float *ti = ps + 7 * anc;
            o[9 + r] = ps[7 * j + r] - fmaf(R[2], ti[2], fmaf(R[1], ti[1], R[0] * ti[0]));
        }
    }
}

// Step 2 (after a barrier): Ad(G_ij) rows r and r + 3; K_ij row r and h_ij[r]:
//   K = [w_j]x R - R [w_i]x,  h = v_j + w_j x t - R v_i.
__device__ __forceinline__ void gp_window2(const float *dxs, int t0, int anc, int jlo, int W, bool lin, bool bs,
                                           float *win) {
    for (int q = threadIdx.x; q < 3 * W; q += kThreads) {
        const int jl = q / 3, r = q - 3 * jl, j = jlo + jl;
        float *wd = win + jl * kGpWin;
        const int r1 = r == 2 ? 0 : r + 1, r2 = r == 0 ? 2 : r - 1;
        if (lin) {
            const float *R = wd, *tt = wd + 9;
            float *Ad = wd + 12;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Ad[6 * r + c] = R[3 * r + c];
                // ([t]x R)_rc = t_{r+1} R_{r+2,c} - t_{r+2} R_{r+1,c}
                Ad[6 * r + 3 + c] = fmaf(tt[r1], R[3 * r2 + c], -tt[r2] * R[3 * r1 + c]);
                Ad[6 * (r + 3) + c] = 0.f;
                Ad[6 * (r + 3) + 3 + c] = R[3 * r + c];
            }
        }
        if (bs) {
            const float *R = wd + 48, *tt = wd + 57;
            float *K = wd + 60, *h = wd + 69;
            float vi[3] = {0.f, 0.f, 0.f}, wi[3] = {0.f, 0.f, 0.f}, vj[3] = {0.f, 0.f, 0.f}, wj[3] = {0.f, 0.f, 0.f};
            if (anc >= t0)
#pragma unroll
                for (int m = 0; m < 3; ++m) { vi[m] = dxs[6 * (anc - t0) + m]; wi[m] = dxs[6 * (anc - t0) + 3 + m]; }
            if (j >= t0)
#pragma unroll
                for (int m = 0; m < 3; ++m) { vj[m] = dxs[6 * (j - t0) + m]; wj[m] = dxs[6 * (j - t0) + 3 + m]; }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
                // ([wj]x R)_rc = wj_{r+1} R_{r+2,c} - wj_{r+2} R_{r+1,c}
                const float a = fmaf(wj[r1], R[3 * r2 + c], -wj[r2] * R[3 * r1 + c]);
                // (R [wi]x)_rc = R_{r,c+1} wi_{c+2} - R_{r,c+2} wi_{c+1}
                const float b = fmaf(R[3 * r + c1], wi[c2], -R[3 * r + c2] * wi[c1]);
                K[3 * r + c] = a - b;
            }
            h[r] = vj[r] + fmaf(wj[r1], tt[r2], -wj[r2] * tt[r1]) -
                   fmaf(R[3 * r + 2], vi[2], fmaf(R[3 * r + 1], vi[1], R[3 * r] * vi[0]));
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

// Drain D (128 TMEM lanes x 64 FP32 columns) into the FP32 sums A [64][kGpDaccLd]
// in two passes (the two halves of D land on the same rows of A): first the
// hi.hi^T rows (lanes 64-127: warps 2, 3, 6, 7), halved on the pose columns,
// then, after a barrier, the lo.hi^T rows (lanes 0-63) without their column 63
// (lo.lo of the w column).  Warp w reads lanes 32 (w % 4) .. + 31, the quarter
// it may access, and columns 32 (w / 4) .. + 31.  All threads call it.
__device__ __forceinline__ void gp_drain(uint32_t tmem, float *acc, int warp, int lane) {
    const int q4 = warp & 3, c0 = 32 * (warp >> 2);
    const int row = 32 * q4 + lane - (q4 >= 2 ? kTcRows : 0);
    float4 *dr = reinterpret_cast<float4 *>(acc + row * kGpDaccLd + c0);
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        if ((q4 >= 2) == (pass == 0)) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(c0 + 16 * h), v);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int col = c0 + 16 * h + 4 * q + e;
                        float &x = v[4 * q + e];
                        if (pass == 0) x = col < kTcRows - 2 ? 0.5f * x : x;   // hi.hi^T: halved pose columns
                        else x = col == kTcRows - 1 ? 0.f : x;                  // lo.hi^T: no lo.lo of w
                    }
                    float4 a = dr[4 * h + q];
                    a.x += v[4 * q]; a.y += v[4 * q + 1]; a.z += v[4 * q + 2]; a.w += v[4 * q + 3];
                    dr[4 * h + q] = a;
                }
            }
        }
        if (pass == 0) __syncthreads();
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
    float *rot = reinterpret_cast<float *>(smem + L.off_rot);
    float *dxs = reinterpret_cast<float *>(smem + L.off_dxs);
    float *win = reinterpret_cast<float *>(smem + L.off_win);
    // staging: one buffer; the last launch alternates with a second one in the
    // (then unused) operand region, so that the next chunk's copies start as
    // soon as the current chunk's have landed
    unsigned char *const stage0 = smem + L.off_stage;
    unsigned char *const stage1 = smem + (do_lin ? L.off_stage : L.off_op);
    short *sidx = reinterpret_cast<short *>(smem + L.off_idx);
    float4 *sc4 = reinterpret_cast<float4 *>(smem + L.off_u);
    float *sc1 = reinterpret_cast<float *>(smem + L.off_sc1);   // also the back-substitution terms
    float *Mp = reinterpret_cast<float *>(smem + L.off_u);      // group end: per-thread frame sums
    float *Aj = reinterpret_cast<float *>(smem + L.off_u);      // then the anchor-pair products
    float *Bp = reinterpret_cast<float *>(smem + L.off_u + align16((size_t)W_cap * 42 * 4));
    float4 *pd = reinterpret_cast<float4 *>(smem + L.off_pd);
    unsigned char *op = smem + L.off_op;
    float *dacc = reinterpret_cast<float *>(smem + L.off_dacc);   // drained sums A
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
        for (int q = tid; q < kTcRows * kGpDaccLd; q += kThreads) dacc[q] = 0.f;
    }
    if (do_lin) {
        double *part = pr.partial + (size_t)itm.item * pr.L;
        for (int q = tid; q < pr.L; q += kThreads) part[q] = 0.0;
    }
    __syncthreads();                                 // poses staged
    for (int j = tid; j < N; j += kThreads) {        // per-frame rotations at iterates t and t-1
        if (do_lin) quat_to_rot(pnew + 7 * j + 3, rot + 9 * j);
        if (do_bs) quat_to_rot(pold + 7 * j + 3, rot + 9 * N + 9 * j);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = use_tc ? s_tmem : 0u;

    __shared__ __align__(16) Chunk s_ch[2];
    if (c_begin < c_end) {
        if (tid == 0) s_ch[0] = pr.chunks[c_begin];
        __syncthreads();
        gp_prefetch(pr, s_ch[0], depth_src, gp_stage(stage0, L), do_bs,
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
        const GpStage g = gp_stage(cur ? stage1 : stage0, L);
        cp_async_wait_all();
        if (!mbar_wait(ldbar, (uint32_t)(c - c_begin) & 1u)) atomicOr(&s_bad, 1);
        // the previous chunk's MMAs read the operand, which this chunk rewrites
        if (use_tc && n_commit > 0 && !mbar_wait(mbar, (uint32_t)(n_commit - 1) & 1u)) atomicOr(&s_bad, 2);
        __syncthreads();
        if (s_bad) break;
        Chunk nx = ch;
        if (have_next) nx = s_ch[cur ^ 1];
        if (!do_lin && have_next)   // the last launch: the next chunk's copies start now, into the other buffer
            gp_prefetch(pr, nx, depth_src, gp_stage(cur ? stage0 : stage1, L), true,
                        c + 2 < c_end ? pr.chunks + c + 2 : nullptr, &s_ch[cur], ldbar);
        int o_jj, o_tw;
        staged_offsets(pr, ch, true, o_jj, o_tw);
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

        // -- (0) the window at a group's first chunk (two steps), slot -> staged
        // edge table, patch data, cleared operand columns
        if (!group_open) {
            gp_window1(pnew, pold, rot, N, anc, jlo, W, do_lin, do_bs, win);
            __syncthreads();
            gp_window2(dxs, t0, anc, jlo, W, do_lin, do_bs, win);
        }
        {
            const int p = tid & PSm;
            if (p < cnt) {
                const int a = g.rseg[p] - e0, b = g.rseg[p + 1] - e0;
                int jf = 0, jz = -1;
                bool contig = true;
                if (b > a) {
                    jf = g.rjj[o_jj + a];
                    jz = g.rjj[o_jj + b - 1];
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
                                if (g.rjj[o_jj + mid] < j) lo = mid + 1; else hi = mid;
                            }
                            if (g.rjj[o_jj + lo] == j) idx = lo;
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
                pd[q] = make_float4((g.rpx[q] - cx) * ifx, (g.rpy[q] - cy) * ify, g.rdep[q], 0.f);
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
                        const float2 wv = g.rwt[idx];
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
                    const float2 cw = g.rcw[p];
                    const float d = g.rdep[p] + (cw.y - s) / cw.x;
                    depth_t[k0 + p] = d;
                    pd[p].z = d;
                    if (!do_lin && !pr.no_writeback) pr.patches[3 * (k0 + p) + 2] = d;
                }
            }
            __syncthreads();
            if (!do_lin) {
                group_open = group_next;
                cur ^= 1;
                continue;
            }
        }

        // -- (C) linearise at iterate t
        if (edge_thread) {
            float Rr[12];
            const float *wd = win + my_jl * kGpWin;
#pragma unroll
            for (int q = 0; q < 12; ++q) Rr[q] = wd[q];
            for (int p = my_g; p < cnt; p += NG) {
                const int idx = sidx[my_jl * Gs + p];
                float Ce = 0.f, we = 0.f, Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
                float4 elo = make_float4(0.f, 0.f, 0.f, 0.f), ehi = elo;
                if (idx >= 0 && my_j != anc) {
                    const float2 wv = g.rwt[idx];
                    if (wv.x != 0.f || wv.y != 0.f) {
                        const float2 tv = g.rtg[idx];
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
        // the staging buffer is free: start the next chunk's copies
        if (have_next)
            gp_prefetch(pr, nx, depth_src, gp_stage(stage0, L), do_bs, c + 2 < c_end ? pr.chunks + c + 2 : nullptr,
                        &s_ch[cur], ldbar);

        // drain D before this chunk's MMAs start a fresh accumulation
        if (use_tc && in_block >= kGpDrainEvery) {
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
                    const uint32_t h = gp_tf32(x);
                    const uint32_t lo = gp_tf32(x - __uint_as_float(h));
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
                if (h == 1) {   // the sums of the next group start from zero
#pragma unroll
                    for (int q = 0; q < 21; ++q) M[q] = 0.f;
#pragma unroll
                    for (int q = 0; q < 6; ++q) V[q] = 0.f;
                }
                for (int q = tid; q < W * mn; q += kThreads) {
                    const int jl = q / mn, m = q - jl * mn;
                    float s = 0.f, cc = 0.f;
                    for (int g2 = 0; g2 < NG; ++g2) kahan_add(s, cc, Mp[(size_t)(jl * NG + g2) * kGpMpHalf + m]);
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
            // block (two strips), its v' strip, and its pair with the anchor;
            // the 18 (or 6) entries are loaded together, added, stored
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
                const int n_e = vs ? 6 : 18;
                double *o = vs ? part + 18 * nbs + 6 * a2
                               : part + 18 * (2 * (a2 * nf - a2 * (a2 - 1) / 2 + (b2 - a2)) + h2);
                double2 *o2 = reinterpret_cast<double2 *>(o);
#pragma unroll
                for (int q0 = 0; q0 < 9; q0 += 3) {      // three 16-byte loads in flight, then their stores
                    if (2 * q0 >= n_e) break;
                    double2 cur2[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) cur2[q] = o2[q0 + q];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        cur2[q].x += (double)add[2 * (q0 + q)];
                        cur2[q].y += (double)add[2 * (q0 + q) + 1];
                        o2[q0 + q] = cur2[q];
                    }
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
        __shared__ int s_have;
        if (tid == 0) s_have = 1;
        __syncthreads();
        if (!have) s_have = 0;
        __syncthreads();
        const bool have_all = s_have != 0;
        tc_fence_after();
        if (have_all && in_block > 0) gp_drain(tmem, dacc, warp, lane);   // the last block
        tc_fence_before();
        __syncthreads();
        if (have_all) {
            // S -= A + A^T on the pose columns;  v' -= the w columns (62, 63)
            double *part = pr.partial + (size_t)itm.item * pr.L;
            const int nbs = 2 * n_block_pairs(nf);
            for (int q = tid; q < pr.L; q += kThreads) {
                float s;
                if (q < 18 * nbs) {
                    const int st = q / 18, e = q - 18 * st;
                    int a, b;
                    decode_pair(st >> 1, nf, a, b);
                    const int m = 6 * a + 3 * (st & 1) + e / 6, n = 6 * b + e % 6;
                    s = dacc[m * kGpDaccLd + n] + dacc[n * kGpDaccLd + m];
                } else {
                    const int m = q - 18 * nbs;
                    s = dacc[m * kGpDaccLd + kTcRows - 2] + dacc[m * kGpDaccLd + kTcRows - 1];
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
