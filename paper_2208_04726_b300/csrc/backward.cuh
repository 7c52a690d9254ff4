// Adjoint (backward) of the unrolled Gauss-Newton iterations (Deep Patch
// Visual Odometry, Sec. 3.1: the layer back-propagates through its
// Gauss-Newton iterations; the analytic gradients are derived here).
//
// Forward, per iteration t: linearise at x_t, H_t dx_t = g_t with
// H = sum J^T W J + damping, g = sum J^T W r, then x_{t+1} = x_t (+) dx_t
// (left SE(3) increment on the free poses, additive on the inverse depths).
// Backward, for a loss L(x_T), from t = T-1 down to 0:
//   retraction:  dxi_bar = J_l(dxi)^T eps_{t+1},  eps_t <- Ad(Exp(dxi))^T eps_{t+1}
//                dd_bar = dbar_{t+1}
//   solve:       y = H_t^-1 (dxi_bar, dd_bar), through the Schur complement with
//                the factor kept by the forward pass
//   edges:       u = J y, p = J dx_t, and for every active edge
//                dL/dtarget += W u,  dL/dweight += u * (r - p),
//                x_bar_t += -J^T W u + grad_x [ (W (r - p))^T J(x) y ]
//                                    - grad_x [ (W u)^T J(x) dx_t ]
// The last two terms are the derivative of the Jacobian itself (projection
// Hessian and the SE(3) perturbation terms), evaluated per edge in closed form.
#pragma once

#include "kernels.cuh"

namespace dpvo {

// ---------------------------------------------------------------- FP64 SE(3)

// R and t of Exp(xi), xi = (v, w), via the unit quaternion of R(w) and
// V(w) v = v + A w x v + B w x (w x v).
__device__ inline void se3_exp_rt(const double *xi, double *R, double *t) {
    const double v0 = xi[0], v1 = xi[1], v2 = xi[2];
    const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    const double th = sqrt(th2);
    double A, B, hs, hc;
    if (th < 1e-4) {
        A = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        B = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
        hs = 0.5 - th2 / 48.0 + th2 * th2 / 3840.0;
        hc = 1.0 - th2 / 8.0 + th2 * th2 / 384.0;
    } else {
        double s, c;
        sincos(th, &s, &c);
        A = (1.0 - c) / th2;
        B = (th - s) / (th2 * th);
        double s2, c2;
        sincos(0.5 * th, &s2, &c2);
        hs = s2 / th;
        hc = c2;
    }
    const double qx = hs * w0, qy = hs * w1, qz = hs * w2, qw = hc;
    R[0] = 1 - 2 * (qy * qy + qz * qz); R[1] = 2 * (qx * qy - qz * qw);     R[2] = 2 * (qx * qz + qy * qw);
    R[3] = 2 * (qx * qy + qz * qw);     R[4] = 1 - 2 * (qx * qx + qz * qz); R[5] = 2 * (qy * qz - qx * qw);
    R[6] = 2 * (qx * qz - qy * qw);     R[7] = 2 * (qy * qz + qx * qw);     R[8] = 1 - 2 * (qx * qx + qy * qy);
    const double c0 = w1 * v2 - w2 * v1, c1 = w2 * v0 - w0 * v2, c2 = w0 * v1 - w1 * v0;
    const double d0 = w1 * c2 - w2 * c1, d1 = w2 * c0 - w0 * c2, d2 = w0 * c1 - w1 * c0;
    t[0] = v0 + A * c0 + B * d0;
    t[1] = v1 + A * c1 + B * d1;
    t[2] = v2 + A * c2 + B * d2;
}

__device__ inline void cross3d(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// y = ad(xi)^T x for ad(xi) = [[w^, v^], [0, w^]]:
// y_v = x_v x w,  y_w = x_v x v + x_w x w.
__device__ inline void ad_transpose_times(const double *xi, const double *x, double *y) {
    double a[3], b[3];
    cross3d(x, xi + 3, y);
    cross3d(x, xi, a);
    cross3d(x + 3, xi + 3, b);
    y[3] = a[0] + b[0];
    y[4] = a[1] + b[1];
    y[5] = a[2] + b[2];
}

// J_l(xi)^T e = sum_n (ad^T)^n e / (n + 1)!  (series; |xi| of a Gauss-Newton
// increment is small, 24 terms reach FP64 rounding for |xi| up to ~2).
__device__ inline void left_jacobian_transpose_times(const double *xi, const double *e, double *out) {
    double term[6], nxt[6];
    for (int q = 0; q < 6; ++q) { term[q] = e[q]; out[q] = e[q]; }
    for (int n = 1; n < 24; ++n) {
        ad_transpose_times(xi, term, nxt);
        for (int q = 0; q < 6; ++q) {
            term[q] = nxt[q] / n;
            out[q] += term[q] / (n + 1);
        }
    }
}

// ---------------------------------------------------------------- per-problem kernels

// eps at the final poses from dL/d(t, q): v_bar = t_bar,
// w_bar = t x t_bar + (q_w q_bar_v + q_v x q_bar_v - q_bar_w q_v) / 2;
// dbar = dL/dd; the target and weight gradients start at zero.
__global__ void __launch_bounds__(kThreads) bw_init_kernel(const Prob *__restrict__ probs) {
    const Prob &pr = probs[blockIdx.x];
    const int tid = threadIdx.x;
    for (int e = tid; e < 2 * pr.E; e += kThreads) {
        pr.dL_dtarget[e] = 0.f;
        pr.dL_dweight[e] = 0.f;
    }
    if (block_status(pr.status) != 0) return;
    const float *pose = pr.pose_it + (size_t)pr.iters * pr.N * 7;
    for (int a = tid; a < pr.N; a += kThreads) {
        double *ep = pr.eps + 6 * a;
        if (a < pr.t0) {
            for (int q = 0; q < 6; ++q) ep[q] = 0.0;
            continue;
        }
        const float *g = pr.dL_dposes + 7 * a;
        const float *P = pose + 7 * a;
        const double t[3] = {P[0], P[1], P[2]}, tb[3] = {g[0], g[1], g[2]};
        const double qv[3] = {P[3], P[4], P[5]}, qbv[3] = {g[3], g[4], g[5]};
        const double qw = P[6], qbw = g[6];
        double c1[3], c2[3];
        cross3d(t, tb, c1);
        cross3d(qv, qbv, c2);
        for (int q = 0; q < 3; ++q) {
            ep[q] = tb[q];
            ep[3 + q] = c1[q] + 0.5 * (qw * qbv[q] + c2[q] - qbw * qv[q]);
        }
    }
    for (int k = tid; k < pr.P; k += kThreads) pr.dbar[k] = pr.dL_ddepth[k];
}

// Retraction adjoint of iteration t (first adding the pose-gradient partials
// of the edge pass of iteration t + 1).
__global__ void __launch_bounds__(kSolveThreads) bw_retract_kernel(const Prob *__restrict__ probs, int t) {
    const Prob &pr = probs[blockIdx.x];
    const int tid = threadIdx.x;
    if (t >= pr.iters || block_status(pr.status) != 0) return;
    const int N = pr.N, t0 = pr.t0;
    if (t < pr.iters - 1) {
        for (int q = tid; q < N * 6; q += kSolveThreads) {
            double acc = pr.eps[q];
            for (int it = 0; it < pr.n_items; ++it) acc += pr.pgrad[(size_t)it * N * 6 + q];
            pr.eps[q] = acc;
        }
        __syncthreads();
    }
    for (int f = tid; f < pr.nf; f += kSolveThreads) {
        const double *xi = pr.dxi + ((size_t)t * pr.nf + f) * 6;
        double *ep = pr.eps + 6 * (t0 + f);
        double e[6];
        for (int q = 0; q < 6; ++q) e[q] = ep[q];
        left_jacobian_transpose_times(xi, e, pr.dxibar + 6 * f);
        double R[9], tt[3];
        se3_exp_rt(xi, R, tt);
        // Ad(Exp(xi))^T e: v <- R^T e_v, w <- R^T (e_w - t x e_v)
        double c[3];
        cross3d(tt, e, c);
        const double w[3] = {e[3] - c[0], e[4] - c[1], e[5] - c[2]};
        for (int r = 0; r < 3; ++r) {
            ep[r] = R[r] * e[0] + R[3 + r] * e[1] + R[6 + r] * e[2];
            ep[3 + r] = R[r] * w[0] + R[3 + r] * w[1] + R[6 + r] * w[2];
        }
    }
}

// Adjoint solve of iteration t, pose part: S y = dxi_bar - sum_k E_k C_k^-1 dd_bar_k,
// with the factor U (S = U D^-1 U^T, D = diag U) kept by the forward pass.
__global__ void __launch_bounds__(kSolveThreads) bw_solve_kernel(const Prob *__restrict__ probs, int t) {
    const Prob &pr = probs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31;
    if (t >= pr.iters || block_status(pr.status) != 0) return;
    const int nf = pr.nf, n = 6 * nf;
    if (n == 0) return;
    __shared__ double b[6 * kMaxFree];
    const int Lp = pr.L, nparts = pr.n_parts, off = 18 * 2 * n_block_pairs(nf);
    for (int q = tid; q < n; q += kSolveThreads) {
        double acc = pr.dxibar[q];
        for (int part = 0; part < nparts; ++part) acc += pr.partial[(size_t)part * Lp + off + q];
        b[q] = acc;
    }
    __syncthreads();
    if (tid < 32) {
        const double *U = pr.ufac + (size_t)t * (n * (n + 1) / 2);
        // forward: c_i -= (U_ij / U_jj) c_j for i > j
        for (int j = 0; j < n; ++j) {
            double cj = 0.0;
            if (lane == 0) cj = b[j] / U[j * (j + 1) / 2 + j];
            cj = shfl_double(cj, 0);
            for (int i = j + 1 + lane; i < n; i += 32) b[i] -= U[i * (i + 1) / 2 + j] * cj;
            __syncwarp();
        }
        // back: x_j = (c_j - sum_{k>j} U_kj x_k) / U_jj
        for (int j = n - 1; j >= 0; --j) {
            double xj = 0.0;
            if (lane == 0) xj = b[j] / U[j * (j + 1) / 2 + j];
            xj = shfl_double(xj, 0);
            for (int i = lane; i < j; i += 32) b[i] -= U[j * (j + 1) / 2 + i] * xj;
            __syncwarp();
            if (lane == 0) b[j] = xj;
            __syncwarp();
        }
        for (int q = lane; q < n; q += 32) pr.yxi[q] = b[q];
    }
}

// ---------------------------------------------------------------- edge pass

struct BwSmem {
    int W, G, Gs, EC;
    size_t off_pose, off_rjj, off_rtg, off_rwt, off_rpx, off_rpy, off_rdep, off_rseg, off_rdep2, off_rdb, off_idx,
        off_sc, off_rel, off_pd, off_zy, off_ps, off_dy, off_dx, off_mp, off_pacc;
    size_t bytes;
};

__host__ __device__ inline BwSmem bw_smem_layout(int W, int G, int n_max) {
    BwSmem s;
    s.W = W;
    s.G = G;
    s.Gs = G | 1;
    s.EC = W * G;
    const size_t slots = (size_t)W * s.Gs;
    size_t o = 0;
    s.off_pose = o;  o = align16(o + (size_t)n_max * 7 * 4);
    s.off_rjj = o;   o = align16(o + (size_t)s.EC * 4);
    s.off_rtg = o;   o = align16(o + (size_t)s.EC * 8);
    s.off_rwt = o;   o = align16(o + (size_t)s.EC * 8);
    s.off_rpx = o;   o = align16(o + (size_t)G * 4);
    s.off_rpy = o;   o = align16(o + (size_t)G * 4);
    s.off_rdep = o;  o = align16(o + (size_t)G * 4);
    s.off_rseg = o;  o = align16(o + (size_t)(G + 1) * 4);
    s.off_rdep2 = o; o = align16(o + (size_t)G * 4);
    s.off_rdb = o;   o = align16(o + (size_t)G * 4);
    s.off_idx = o;   o = align16(o + slots * 2);
    s.off_sc = o;    o = align16(o + slots * 8);
    s.off_rel = o;   o = align16(o + (size_t)W * 12 * 4);
    s.off_pd = o;    o = align16(o + (size_t)G * 16);
    s.off_zy = o;    o = align16(o + (size_t)G * 16);
    s.off_ps = o;    o = align16(o + (size_t)G * 4);
    s.off_dy = o;    o = align16(o + kMaxFree * 6 * 4);
    s.off_dx = o;    o = align16(o + kMaxFree * 6 * 4);
    s.off_mp = o;    o = align16(o + (size_t)kThreads * 12 * 4);
    s.off_pacc = o;  o = align16(o + (size_t)n_max * 12 * 4);
    s.bytes = o;
    return s;
}

// dX along the state direction (pose-i twist ai, pose-j twist aj, depth ad):
// V = d nu_j + om_j x X - R (d nu_i + om_i x pbar) + t ad.  Also returns
// u_i = d nu_i + om_i x pbar.
__device__ __forceinline__ void dX_along(const float *R, const float *t, const float *X, const float *pb, float d,
                                         const float *ai, const float *aj, float ad, float *V, float *ui) {
    ui[0] = d * ai[0] + (ai[4] * pb[2] - ai[5] * pb[1]);
    ui[1] = d * ai[1] + (ai[5] * pb[0] - ai[3] * pb[2]);
    ui[2] = d * ai[2] + (ai[3] * pb[1] - ai[4] * pb[0]);
#pragma unroll
    for (int r = 0; r < 3; ++r) V[r] = d * aj[r] - (R[3 * r] * ui[0] + R[3 * r + 1] * ui[1] + R[3 * r + 2] * ui[2]) + t[r] * ad;
    V[0] += aj[4] * X[2] - aj[5] * X[1];
    V[1] += aj[5] * X[0] - aj[3] * X[2];
    V[2] += aj[3] * X[1] - aj[4] * X[0];
}

__device__ __forceinline__ void cross3f(const float *a, const float *b, float *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// gi, gj, gd += sgn * grad over the state of h = b^T (d pi / d X)(X) V_a(x)
__device__ __forceinline__ void add_second_order(float sgn, const float *R, const float *t, const float *X,
                                                 const float *pb, float d, float iz, float a, float b_, float fx,
                                                 float fy, const float *bb, const float *ai, const float *aj,
                                                 float ad, float *gi, float *gj, float &gd) {
    float V[3], ui[3];
    dX_along(R, t, X, pb, d, ai, aj, ad, V, ui);
    const float fxi = fx * iz, fyi = fy * iz, iz2 = iz * iz;
    const float beta[3] = {fxi * bb[0], fyi * bb[1], -(a * fxi * bb[0] + b_ * fyi * bb[1])};
    float kp[3];
    kp[0] = -fx * bb[0] * V[2] * iz2;
    kp[1] = -fy * bb[1] * V[2] * iz2;
    kp[2] = fx * bb[0] * iz2 * (2.f * a * V[2] - V[0]) + fy * bb[1] * iz2 * (2.f * b_ * V[2] - V[1]);
    float c[3];
    cross3f(beta, aj + 3, c);                       // + beta x om_j
    kp[0] += c[0]; kp[1] += c[1]; kp[2] += c[2];
    float Ru[3], RTk[3], RTb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        Ru[r] = R[3 * r] * ui[0] + R[3 * r + 1] * ui[1] + R[3 * r + 2] * ui[2];
        RTk[r] = R[r] * kp[0] + R[3 + r] * kp[1] + R[6 + r] * kp[2];
        RTb[r] = R[r] * beta[0] + R[3 + r] * beta[1] + R[6 + r] * beta[2];
    }
    float x1[3], x2[3], x3[3];
    cross3f(X, kp, x1);
    cross3f(beta, Ru, x2);
    cross3f(t, beta, x3);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        gj[r] += sgn * (d * kp[r] + ad * beta[r]);
        gj[3 + r] += sgn * (x1[r] + x2[r] + ad * x3[r]);
        gi[r] += sgn * (-d * RTk[r] - ad * RTb[r]);
    }
    cross3f(pb, RTk, x1);
    cross3f(ui, RTb, x2);
#pragma unroll
    for (int r = 0; r < 3; ++r) gi[3 + r] += sgn * (-x1[r] + x2[r]);
    const float Rnu[3] = {R[0] * ai[0] + R[1] * ai[1] + R[2] * ai[2], R[3] * ai[0] + R[4] * ai[1] + R[5] * ai[2],
                          R[6] * ai[0] + R[7] * ai[1] + R[8] * ai[2]};
    gd += sgn * (kp[0] * t[0] + kp[1] * t[1] + kp[2] * t[2] + beta[0] * (aj[0] - Rnu[0]) +
                 beta[1] * (aj[1] - Rnu[1]) + beta[2] * (aj[2] - Rnu[2]));
}

// Adjoint edge pass of iteration t at x_t: y_d per patch, then per edge the
// target / weight gradients and the state-gradient terms; inverse-depth
// gradients are updated in place, pose gradients go to per-CTA partials.
__global__ void __launch_bounds__(kThreads, 2) bw_edge_kernel(const Prob *__restrict__ probs,
                                                              const Item *__restrict__ items, int t, int W_cap,
                                                              int G_cap, int n_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Item itm = items[blockIdx.x];
    const Prob &pr = probs[itm.prob];
    const int tid = threadIdx.x;
    if (t >= pr.iters || block_status(pr.status) != 0) return;
    const BwSmem L = bw_smem_layout(W_cap, G_cap, n_max);
    float *spose = reinterpret_cast<float *>(smem + L.off_pose);
    int *rjj = reinterpret_cast<int *>(smem + L.off_rjj);
    float2 *rtg = reinterpret_cast<float2 *>(smem + L.off_rtg);
    float2 *rwt = reinterpret_cast<float2 *>(smem + L.off_rwt);
    float *rpx = reinterpret_cast<float *>(smem + L.off_rpx);
    float *rpy = reinterpret_cast<float *>(smem + L.off_rpy);
    float *rdep = reinterpret_cast<float *>(smem + L.off_rdep);
    int *rseg = reinterpret_cast<int *>(smem + L.off_rseg);
    float *rdep2 = reinterpret_cast<float *>(smem + L.off_rdep2);
    float *rdb = reinterpret_cast<float *>(smem + L.off_rdb);
    short *sidx = reinterpret_cast<short *>(smem + L.off_idx);
    float2 *sc = reinterpret_cast<float2 *>(smem + L.off_sc);
    float *rel = reinterpret_cast<float *>(smem + L.off_rel);
    float4 *pd = reinterpret_cast<float4 *>(smem + L.off_pd);
    float4 *zy = reinterpret_cast<float4 *>(smem + L.off_zy);
    float *yd = reinterpret_cast<float *>(smem + L.off_ps);
    float *dys = reinterpret_cast<float *>(smem + L.off_dy);
    float *dxs = reinterpret_cast<float *>(smem + L.off_dx);
    float *Mp = reinterpret_cast<float *>(smem + L.off_mp);
    float *pacc = reinterpret_cast<float *>(smem + L.off_pacc);   // [N][6] sum, [N][6] compensation
    const int Gs = L.Gs;
    const int N = pr.N, t0 = pr.t0, nf = pr.nf;
    const float fx = pr.fx, fy = pr.fy, cx = pr.cx, cy = pr.cy, z_min = pr.z_min, lam = pr.damping;
    const float ifx = 1.0f / fx, ify = 1.0f / fy;
    const float *pose_t = pr.pose_it + (size_t)t * N * 7;
    const float *depth_t = pr.depth_it + (size_t)t * pr.P;
    const float *depth_t1 = pr.depth_it + (size_t)(t + 1) * pr.P;

    const int nch = *pr.n_chunks;
    const int c_begin = (int)(((long long)itm.item * nch) / pr.n_items);
    const int c_end = (int)(((long long)(itm.item + 1) * nch) / pr.n_items);

    for (int q = tid; q < N * 7; q += kThreads) spose[q] = pose_t[q];
    for (int q = tid; q < nf * 6; q += kThreads) {
        dys[q] = (float)pr.yxi[q];
        dxs[q] = (float)pr.dxi[(size_t)t * nf * 6 + q];
    }
    for (int q = tid; q < N * 12; q += kThreads) pacc[q] = 0.f;

    __shared__ __align__(16) Chunk s_ch[2];
    auto prefetch = [&](const Chunk &ch, const Chunk *desc_src, Chunk *desc_dst) {
        prefetch_chunk(pr, ch, depth_t, rjj, rtg, rwt, rpx, rpy, rdep, rseg, desc_src, desc_dst);
        for (int q = tid; q < ch.count; q += kThreads) {
            cp_async4(rdep2 + q, depth_t1 + ch.k0 + q);
            cp_async4(rdb + q, pr.dbar + ch.k0 + q);
        }
        cp_async_commit();
    };
    if (c_begin < c_end) {
        if (tid == 0) s_ch[0] = pr.chunks[c_begin];
        __syncthreads();
        prefetch(s_ch[0], c_begin + 1 < c_end ? pr.chunks + c_begin + 1 : nullptr, &s_ch[1]);
    }
    int cur = 0;
    int prev_anchor = -1, prev_jlo = -1, prev_jhi = -1;
    for (int c = c_begin; c < c_end; ++c) {
        const Chunk ch = s_ch[cur];
        const bool have_next = c + 1 < c_end;
        cp_async_wait_all();
        __syncthreads();
        Chunk nx = ch;
        if (have_next) nx = s_ch[cur ^ 1];
        const int k0 = ch.k0, cnt = ch.count, e0 = ch.e0;
        const int anc = ch.anchor, jlo = ch.jlo;
        const int W = ch.jhi - jlo + 1;
        const bool anc_free = anc >= t0;
        const int NG = kThreads / W;
        const int my_g = tid % NG, my_jl = tid / NG;
        const int my_j = jlo + my_jl;
        const bool edge_thread = my_jl < W;
        const bool new_window = anc != prev_anchor || jlo != prev_jlo || ch.jhi != prev_jhi;

        // -- slot table, patch data (d_t, dd_t), z_y for the anchor term, window poses
        {
            const int p = tid & 63;
            if (p < cnt) {
                const int a = rseg[p] - e0, b = rseg[p + 1] - e0;
                int jf = 0, jz = -1;
                bool contig = true;
                if (b > a) {
                    jf = rjj[a];
                    jz = rjj[b - 1];
                    contig = jz - jf + 1 == b - a;
                }
                for (int jl = tid >> 6; jl < W; jl += kThreads / 64) {
                    const int j = jlo + jl;
                    int idx = -1;
                    if (j >= jf && j <= jz) {
                        if (contig) {
                            idx = a + (j - jf);
                        } else {
                            int lo = a, hi = b - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (rjj[mid] < j) lo = mid + 1; else hi = mid;
                            }
                            if (rjj[lo] == j) idx = lo;
                        }
                    }
                    sidx[jl * Gs + p] = (short)idx;
                }
                if (tid < 64) {
                    const float px = (rpx[p] - cx) * ifx, py = (rpy[p] - cy) * ify, d = rdep[p];
                    pd[p] = make_float4(px, py, d, rdep2[p] - d);
                    if (anc_free) {
                        const float *yi = dys + 6 * (anc - t0);
                        zy[p] = make_float4(fmaf(d, yi[0], yi[4] - yi[5] * py), fmaf(d, yi[1], yi[5] * px - yi[3]),
                                            fmaf(d, yi[2], yi[3] * py - yi[4] * px), 0.f);
                    }
                }
            }
        }
        if (new_window) window_poses(spose, anc, jlo, W, rel, nullptr);
        __syncthreads();

        // -- (1) per edge: C_e and e_jk . y_j - Y . z_y (as in the back-substitution)
        float Rr[12];
        if (edge_thread) {
#pragma unroll
            for (int q = 0; q < 12; ++q) Rr[q] = rel[my_jl * 12 + q];
            const bool jfree = my_j >= t0 && my_j != anc;
            const float *yj = dys + 6 * (jfree ? my_j - t0 : 0);
            for (int p = my_g; p < cnt; p += NG) {
                const int slot = my_jl * Gs + p;
                const int ei = sidx[slot];
                float Ce = 0.f, se = 0.f;
                if (ei >= 0 && my_j != anc) {
                    const float2 tv = rtg[ei], wv = rwt[ei];
                    const float4 q = pd[p];
                    EdgeLin E;
                    if ((wv.x != 0.f || wv.y != 0.f) &&
                        edge_linearize(Rr, Rr + 9, q.x, q.y, q.z, tv.x, tv.y, fx, fy, cx, cy, z_min, E)) {
                        float wjd0, wjd1, we;
                        depth_terms(E, wv.x, wv.y, wjd0, wjd1, Ce, we);
                        if (jfree) {
#pragma unroll
                            for (int m = 0; m < 6; ++m) se = fmaf(fmaf(E.j1[m], wjd1, E.j0[m] * wjd0), yj[m], se);
                        }
                        if (anc_free) {
                            float Y0, Y1, Y2;
                            anchor_terms(E, Rr, wjd0, wjd1, Y0, Y1, Y2);
                            const float4 z = zy[p];
                            se -= fmaf(Y2, z.z, fmaf(Y1, z.y, Y0 * z.x));
                        }
                    }
                }
                sc[slot] = make_float2(Ce, se);
            }
        }
        __syncthreads();
        {   // y_d,k = (dd_bar_k - e_k^T y) / C_k, four lanes per patch
            const int p = tid >> 2, sub = tid & 3;
            float C = sub == 0 ? lam : 0.f, s = 0.f;
            if (p < cnt)
                for (int jl = sub; jl < W; jl += 4) {
                    const float2 v = sc[jl * Gs + p];
                    C += v.x;
                    s += v.y;
                }
            C = quad_sum(C);
            s = quad_sum(s);
            if (sub == 0 && p < cnt) yd[p] = (rdb[p] - s) / C;
        }
        __syncthreads();

        // -- (2) per edge: u = J y, p = J dx, gradients
        float gi[6], gj[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) { gi[q] = 0.f; gj[q] = 0.f; }
        if (edge_thread) {
            const bool ifree = anc_free, jfree = my_j >= t0 && my_j != anc;
            float yi[6], yjv[6], Di[6], Dj[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                yi[q] = ifree ? dys[6 * (anc - t0) + q] : 0.f;
                Di[q] = ifree ? dxs[6 * (anc - t0) + q] : 0.f;
                yjv[q] = jfree ? dys[6 * (my_j - t0) + q] : 0.f;
                Dj[q] = jfree ? dxs[6 * (my_j - t0) + q] : 0.f;
            }
            for (int p = my_g; p < cnt; p += NG) {
                const int slot = my_jl * Gs + p;
                const int ei = sidx[slot];
                float gd = 0.f;
                if (ei >= 0 && my_j != anc) {
                    const float2 tv = rtg[ei], wv = rwt[ei];
                    const float4 q = pd[p];
                    EdgeLin E;
                    if ((wv.x != 0.f || wv.y != 0.f) &&
                        edge_linearize(Rr, Rr + 9, q.x, q.y, q.z, tv.x, tv.y, fx, fy, cx, cy, z_min, E)) {
                        const float pb[3] = {q.x, q.y, 1.f};
                        const float d = q.z;
                        const float X[3] = {fmaf(Rr[9], d, fmaf(Rr[1], q.y, fmaf(Rr[0], q.x, Rr[2]))),
                                            fmaf(Rr[10], d, fmaf(Rr[4], q.y, fmaf(Rr[3], q.x, Rr[5]))),
                                            fmaf(Rr[11], d, fmaf(Rr[7], q.y, fmaf(Rr[6], q.x, Rr[8])))};
                        const float iz = E.fxi / fx;
                        float V[3], ui[3];
                        dX_along(Rr, Rr + 9, X, pb, d, yi, yjv, yd[p], V, ui);
                        const float u0 = E.fxi * (V[0] - E.a * V[2]), u1 = E.fyi * (V[1] - E.b * V[2]);
                        dX_along(Rr, Rr + 9, X, pb, d, Di, Dj, q.w, V, ui);
                        const float p0 = E.fxi * (V[0] - E.a * V[2]), p1 = E.fyi * (V[1] - E.b * V[2]);
                        const int eg = e0 + ei;
                        pr.dL_dtarget[2 * eg] += wv.x * u0;
                        pr.dL_dtarget[2 * eg + 1] += wv.y * u1;
                        pr.dL_dweight[2 * eg] += u0 * (E.r0 - p0);
                        pr.dL_dweight[2 * eg + 1] += u1 * (E.r1 - p1);
                        // first order: -J^T W u
                        const float b2[2] = {wv.x * u0, wv.y * u1};
                        const float beta[3] = {-E.fxi * b2[0], -E.fyi * b2[1], E.a * E.fxi * b2[0] + E.b * E.fyi * b2[1]};
                        float c[3], RTb[3];
                        cross3f(X, beta, c);
#pragma unroll
                        for (int r = 0; r < 3; ++r) {
                            gj[r] += d * beta[r];
                            gj[3 + r] += c[r];
                            RTb[r] = Rr[r] * beta[0] + Rr[3 + r] * beta[1] + Rr[6 + r] * beta[2];
                            gi[r] -= d * RTb[r];
                        }
                        cross3f(pb, RTb, c);
#pragma unroll
                        for (int r = 0; r < 3; ++r) gi[3 + r] -= c[r];
                        gd += beta[0] * Rr[9] + beta[1] * Rr[10] + beta[2] * Rr[11];
                        // second order: + grad (W (r - p))^T J y - grad (W u)^T J dx
                        const float b1[2] = {wv.x * (E.r0 - p0), wv.y * (E.r1 - p1)};
                        add_second_order(1.f, Rr, Rr + 9, X, pb, d, iz, E.a, E.b, fx, fy, b1, yi, yjv, yd[p], gi, gj, gd);
                        add_second_order(-1.f, Rr, Rr + 9, X, pb, d, iz, E.a, E.b, fx, fy, b2, Di, Dj, q.w, gi, gj, gd);
                    }
                }
                sc[slot].x = gd;
            }
            float *mp = Mp + (size_t)tid * 12;
#pragma unroll
            for (int q = 0; q < 6; ++q) { mp[q] = gi[q]; mp[6 + q] = gj[q]; }
        }
        __syncthreads();
        {   // inverse-depth gradient: dbar_k += sum of the edge terms (four lanes per patch)
            const int p = tid >> 2, sub = tid & 3;
            float s = 0.f;
            if (p < cnt)
                for (int jl = sub; jl < W; jl += 4) s += sc[jl * Gs + p].x;
            s = quad_sum(s);
            if (sub == 0 && p < cnt) pr.dbar[k0 + p] = rdb[p] + s;
        }
        // pose gradients: frame j from the threads of its column, the anchor from all
        for (int q = tid; q < W * 6; q += kThreads) {
            const int jl = q / 6, m = q - jl * 6;
            float s = 0.f;
            for (int g = 0; g < NG; ++g) s += Mp[(size_t)(jl * NG + g) * 12 + 6 + m];
            float *ps = pacc + (jlo + jl) * 6 + m;
            kahan_add(ps[0], ps[N * 6], s);
        }
        __syncthreads();
        // the staging buffers (including the staged dbar) are free: start the next chunk's copies
        if (have_next) prefetch(nx, c + 2 < c_end ? pr.chunks + c + 2 : nullptr, &s_ch[cur]);
        if (tid < 6) {
            float s = 0.f, cc = 0.f;
            for (int q = 0; q < NG * W; ++q) kahan_add(s, cc, Mp[(size_t)q * 12 + tid]);
            float *ps = pacc + anc * 6 + tid;
            kahan_add(ps[0], ps[N * 6], s - cc);
        }
        __syncthreads();
        prev_anchor = anc;
        prev_jlo = jlo;
        prev_jhi = ch.jhi;
        cur ^= 1;
    }
    cp_async_wait_all();
    __syncthreads();
    double *out = pr.pgrad + (size_t)itm.item * N * 6;
    for (int q = tid; q < N * 6; q += kThreads) out[q] = (double)pacc[q] - (double)pacc[N * 6 + q];
}

}  // namespace dpvo
