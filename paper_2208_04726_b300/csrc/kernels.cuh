// Bundle-adjustment kernels (Deep Patch Visual Odometry, Sec. 3.1 Eq. 6).
//
//   plan_kernel       once per solve: validates indices and ordering, builds the
//                     patch -> edge offsets and the chunk table, copies the
//                     initial state into iterate 0.
//   linearize_kernel  once per iteration (and once more at the end): for each
//                     chunk of patches that share a source frame,
//                       (a) back-substitutes the previous iteration's inverse-
//                           depth increments dd_k = (w_k - e_k^T dxi) / C_k,
//                       (b) linearises every edge at the new state (Eq. 2-3
//                           reprojection, residual, pose-j / inverse-depth
//                           Jacobians) and reduces the pose-pair blocks
//                           B_jj += J_j^T W J_j by frame,
//                       (c) accumulates the Schur complement
//                           S = B - sum_k E_k C_k^-1 E_k^T, v' = v - sum_k E_k C_k^-1 w_k
//                           over the free poses, with compensated sums,
//                     and writes one FP64 partial of (S, v') per CTA.
//   solve_kernel      once per iteration: sums the partials in FP64, factorises
//                     S = L L^T in FP64 (pivot check -> NOT_SPD), solves for the
//                     pose increments and retracts T <- Exp(dxi) T.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "ba_common.cuh"
#include "se3.cuh"

namespace dpvo {

// ----------------------------------------------------------------------------
// Per-edge linearisation (Eq. 2-3 reprojection of the patch centre, residual
// r = target - pi(X), Jacobians of pi w.r.t. the left perturbation of pose j
// and the inverse depth).  X = R_ij pbar + t_ij d with pbar = K^-1 (x, y, 1);
// the homogeneous fourth coordinate is d.  Returns false if the edge takes no
// part (third coordinate <= z_min).
// ----------------------------------------------------------------------------
struct EdgeLin {
    float r0, r1;
    float a, b, fxi, fyi;       // X/Z, Y/Z, fx/Z, fy/Z
    float j0[6], j1[6];         // rows of J_j; j0[1] == j1[0] == 0
    float jd0, jd1;             // J_d
};

__device__ __forceinline__ bool edge_linearize(const float *Rij, const float *tij, float pbx, float pby,
                                               float d, float tx, float ty, float fx, float fy, float cx,
                                               float cy, float z_min, EdgeLin &L) {
    const float X = fmaf(tij[0], d, fmaf(Rij[1], pby, fmaf(Rij[0], pbx, Rij[2])));
    const float Y = fmaf(tij[1], d, fmaf(Rij[4], pby, fmaf(Rij[3], pbx, Rij[5])));
    const float Z = fmaf(tij[2], d, fmaf(Rij[7], pby, fmaf(Rij[6], pbx, Rij[8])));
    if (!(Z > z_min)) return false;
    const float iz = 1.0f / Z;
    const float a = X * iz, b = Y * iz;
    L.a = a;
    L.b = b;
    L.r0 = tx - fmaf(fx, a, cx);
    L.r1 = ty - fmaf(fy, b, cy);
    const float fxi = fx * iz, fyi = fy * iz;
    L.fxi = fxi;
    L.fyi = fyi;
    const float diz = d * iz;
    // d pi / d xi_j = d pi / d X  [d I, -[X]x]
    L.j0[0] = fx * diz;  L.j0[1] = 0.f;        L.j0[2] = -fx * a * diz;
    L.j0[3] = -fx * a * b; L.j0[4] = fx * fmaf(a, a, 1.f); L.j0[5] = -fx * b;
    L.j1[0] = 0.f;       L.j1[1] = fy * diz;   L.j1[2] = -fy * b * diz;
    L.j1[3] = -fy * fmaf(b, b, 1.f); L.j1[4] = fy * a * b; L.j1[5] = fy * a;
    // d pi / d d = d pi / d X  t_ij
    L.jd0 = fxi * fmaf(-a, tij[2], tij[0]);
    L.jd1 = fyi * fmaf(-b, tij[2], tij[1]);
    return true;
}

// Weighted inverse-depth terms of one edge: C_e = J_d^T W J_d, w_e = J_d^T W r.
__device__ __forceinline__ void depth_terms(const EdgeLin &L, float w0, float w1, float &wjd0, float &wjd1,
                                            float &Ce, float &we) {
    wjd0 = w0 * L.jd0;
    wjd1 = w1 * L.jd1;
    Ce = fmaf(wjd1, L.jd1, wjd0 * L.jd0);
    we = fmaf(wjd1, L.r1, wjd0 * L.r0);
}

// Y_e = R_ij^T (d pi / d X)^T W J_d: the anchor-pose column of E_k is
// e_ik = -[d Y; pbar x Y] summed over the patch's edges (from
// J_i = -(d pi / d X) R_ij [d I, -[pbar]x]).
__device__ __forceinline__ void anchor_terms(const EdgeLin &L, const float *Rij, float wjd0, float wjd1,
                                             float &Y0, float &Y1, float &Y2) {
    const float g0 = L.fxi * wjd0, g1 = L.fyi * wjd1;
    const float g2 = -fmaf(L.a, g0, L.b * g1);
    Y0 = fmaf(Rij[6], g2, fmaf(Rij[3], g1, Rij[0] * g0));
    Y1 = fmaf(Rij[7], g2, fmaf(Rij[4], g1, Rij[1] * g0));
    Y2 = fmaf(Rij[8], g2, fmaf(Rij[5], g1, Rij[2] * g0));
}

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int n, int key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ----------------------------------------------------------------------------
// plan_kernel: one CTA per problem.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) plan_kernel(const Prob *__restrict__ probs) {
    const Prob &pr = probs[blockIdx.x];
    const int tid = threadIdx.x;
    const int N = pr.N, P = pr.P, E = pr.E;
    __shared__ int s_bad;
    __shared__ int s_fstart[DPVO_BA_MAX_FRAMES + 1];
    __shared__ int s_choff[DPVO_BA_MAX_FRAMES + 1];
    if (tid == 0) s_bad = 0;
    __syncthreads();

    for (int i = tid; i < N * 7; i += kThreads) pr.pose_it[i] = pr.poses[i];
    for (int k = tid; k < P; k += kThreads) pr.depth_it[k] = pr.patches[3 * k + 2];

    int bad = 0;
    for (int k = tid; k < P; k += kThreads) {
        const int a = pr.anchor[k];
        if (a < 0 || a >= N) bad = 1;
        else if (k > 0 && pr.anchor[k - 1] > a) bad = 1;
    }
    for (int e = tid; e < E; e += kThreads) {
        const int k = pr.kk[e], j = pr.jj[e];
        if (k < 0 || k >= P || j < 0 || j >= N) { bad = 1; continue; }
        if (e > 0) {
            const int kp = pr.kk[e - 1];
            if (kp > k) bad = 1;
            else if (kp == k && pr.jj[e - 1] >= j) bad = 1;
        }
    }
    for (int i = tid; i < N * 7; i += kThreads)
        if (!isfinite(pr.poses[i])) bad = 1;
    if (bad) atomicOr(&s_bad, 1);
    __syncthreads();
    if (s_bad) {
        if (tid == 0) { *pr.status = DPVO_BA_STATUS_BAD_INPUT; *pr.n_chunks = 0; }
        return;
    }
    for (int k = tid; k <= P; k += kThreads) pr.seg[k] = lower_bound_i32(pr.kk, E, k);
    for (int i = tid; i <= N; i += kThreads) s_fstart[i] = lower_bound_i32(pr.anchor, P, i);
    __syncthreads();
    if (tid == 0) {
        int off = 0;
        for (int i = 0; i < N; ++i) {
            s_choff[i] = off;
            const int cnt = s_fstart[i + 1] - s_fstart[i];
            off += (cnt + pr.chunk_cap - 1) / pr.chunk_cap;
        }
        s_choff[N] = off;
        if (off > pr.max_chunks) s_bad = 1;
    }
    __syncthreads();
    for (int i = tid; i < N && !s_bad; i += kThreads) {
        const int cnt = s_fstart[i + 1] - s_fstart[i];
        const int nch = s_choff[i + 1] - s_choff[i];
        if (nch == 0) continue;
        const int base = cnt / nch, rem = cnt % nch;
        int k = s_fstart[i];
        for (int c = 0; c < nch; ++c) {
            const int sz = base + (c < rem ? 1 : 0);
            Chunk ch;
            ch.k0 = k;
            ch.count = sz;
            ch.e0 = pr.seg[k];
            ch.e1 = pr.seg[k + sz];
            ch.anchor = i;
            int jlo = i, jhi = i;
            for (int q = k; q < k + sz; ++q) {
                const int s0 = pr.seg[q], s1 = pr.seg[q + 1];
                if (s1 > s0) {
                    jlo = min(jlo, (int)pr.jj[s0]);
                    jhi = max(jhi, (int)pr.jj[s1 - 1]);
                }
            }
            ch.jlo = jlo;
            ch.jhi = jhi;
            ch.pad = 0;
            if (jhi - jlo + 1 > pr.win_cap) atomicOr(&s_bad, 1);
            pr.chunks[s_choff[i] + c] = ch;
            k += sz;
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_bad) { *pr.status = DPVO_BA_STATUS_BAD_INPUT; *pr.n_chunks = 0; }
        else { *pr.status = 0; *pr.n_chunks = s_choff[N]; }
    }
}

// ----------------------------------------------------------------------------
// linearize_kernel shared-memory carve-up (sizes depend on the batch's window
// and chunk caps, and on the largest number of free poses).
// ----------------------------------------------------------------------------
struct LinSmem {
    int W, G, ES;  // window cap, chunk cap, E-column stride
    size_t off_tw, off_sc4, off_sc1, off_ec, off_rel, off_adj, off_mc, off_aj, off_bii, off_pd, off_zk, off_dx;
    size_t bytes;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline LinSmem lin_smem_layout(int W, int G, int nf_max) {
    LinSmem s;
    s.W = W; s.G = G;
    int es = 6 * nf_max + 2;
    if ((es & 1) == 0) es += 1;
    s.ES = es;
    size_t o = 0;
    size_t tw = (size_t)W * G * 16, mp = (size_t)kThreads * 27 * 4;
    s.off_tw = o;  o = align16(o + (tw > mp ? tw : mp));
    s.off_sc4 = o; o = align16(o + (size_t)W * G * 16);
    s.off_sc1 = o; o = align16(o + (size_t)W * G * 4);
    s.off_ec = o;  o = align16(o + (size_t)G * es * 4);
    s.off_rel = o; o = align16(o + (size_t)W * 12 * 4);
    s.off_adj = o; o = align16(o + (size_t)W * 36 * 4);
    s.off_mc = o;  o = align16(o + (size_t)W * 27 * 4);
    s.off_aj = o;  o = align16(o + (size_t)W * 42 * 4);
    s.off_bii = o; o = align16(o + 42 * 4);
    s.off_pd = o;  o = align16(o + (size_t)G * 16);
    s.off_zk = o;  o = align16(o + (size_t)G * 16);
    s.off_dx = o;  o = align16(o + kMaxFree * 6 * 4);
    s.bytes = o;
    return s;
}

// Compensated (Kahan) update of a running sum (s, c) with the block sum blk.
__device__ __forceinline__ void kahan_add(float &s, float &c, float blk) {
    const float y = blk - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Compute relative poses (and adjoints) of the chunk's window frames w.r.t.
// the anchor at the pose set `poses`.
__device__ __forceinline__ void window_poses(const float *poses, int anchor, int jlo, int W, float *rel,
                                             float *adj) {
    for (int jl = threadIdx.x; jl < W; jl += kThreads) {
        float *R = rel + jl * 12;
        relative_pose(poses + 7 * anchor, poses + 7 * (jlo + jl), R, R + 9);
        adjoint6(R, R + 9, adj + jl * 36);
    }
}

// ----------------------------------------------------------------------------
// linearize_kernel: one CTA per work item (a range of chunks of one problem).
// t = iteration.  For t < iters: back-substitute iteration t-1 (if t > 0), then
// linearise at iterate t and accumulate the Schur partial.  For t == iters:
// back-substitute the last iteration and write the caller's outputs.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) linearize_kernel(const Prob *__restrict__ probs,
                                                             const Item *__restrict__ items, int t,
                                                             int W_cap, int G_cap, int nf_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Item itm = items[blockIdx.x];
    const Prob &pr = probs[itm.prob];
    const int tid = threadIdx.x;
    if (t > pr.iters) return;
    const bool do_bs = t > 0;
    const bool do_lin = t < pr.iters;
    const bool final_pass = t == pr.iters;
    {
        const int st = *pr.status;
        if (final_pass && itm.item == 0 && tid == 0 && pr.status_user) *pr.status_user = st;
        if (st != 0) return;
    }

    const LinSmem L = lin_smem_layout(W_cap, G_cap, nf_max);
    float4 *tw = reinterpret_cast<float4 *>(smem + L.off_tw);
    float *Mp = reinterpret_cast<float *>(smem + L.off_tw);   // aliases tw after the edge pass
    float4 *sc4 = reinterpret_cast<float4 *>(smem + L.off_sc4);
    float *sc1 = reinterpret_cast<float *>(smem + L.off_sc1);
    float *Ec = reinterpret_cast<float *>(smem + L.off_ec);
    float *rel = reinterpret_cast<float *>(smem + L.off_rel);
    float *adj = reinterpret_cast<float *>(smem + L.off_adj);
    float *Mc = reinterpret_cast<float *>(smem + L.off_mc);
    float *Aj = reinterpret_cast<float *>(smem + L.off_aj);
    float *Bii = reinterpret_cast<float *>(smem + L.off_bii);
    float4 *pd = reinterpret_cast<float4 *>(smem + L.off_pd);
    float4 *zk = reinterpret_cast<float4 *>(smem + L.off_zk);
    float *dxs = reinterpret_cast<float *>(smem + L.off_dx);
    const int Gs = G_cap, ES = L.ES;

    const int N = pr.N, t0 = pr.t0, nf = pr.nf;
    const float fx = pr.fx, fy = pr.fy, cx = pr.cx, cy = pr.cy, z_min = pr.z_min, lam = pr.damping;
    const float *pose_old = pr.pose_it + (size_t)(t > 0 ? t - 1 : 0) * N * 7;
    const float *pose_new = pr.pose_it + (size_t)t * N * 7;
    const float *depth_old = pr.depth_it + (size_t)(t > 0 ? t - 1 : 0) * pr.P;
    float *depth_new = pr.depth_it + (size_t)t * pr.P;

    // Work-item chunk range.
    const int nch = *pr.n_chunks;
    const int c_begin = (int)(((long long)itm.item * nch) / pr.n_items);
    const int c_end = (int)(((long long)(itm.item + 1) * nch) / pr.n_items);

    // Strip ownership for the Schur accumulation.
    const int nbp = n_block_pairs(nf);
    const int nbs = 2 * nbp;
    const int nst = nbs + nf;
    const int KS = pr.ks;
    const int my_strip = nst > 0 ? tid % nst : 0;
    const int my_ks = nst > 0 ? tid / nst : KS;
    const bool owns = do_lin && nst > 0 && my_ks < KS;
    const bool is_vstrip = my_strip >= nbs;
    int sa = 0, sb = 0, sh = 0;
    if (owns) {
        if (!is_vstrip) {
            decode_pair(my_strip >> 1, nf, sa, sb);
            sh = my_strip & 1;
        } else {
            sa = sb = my_strip - nbs;
        }
    }
    float acc_s[18], acc_c[18], blk[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) { acc_s[q] = 0.f; acc_c[q] = 0.f; blk[q] = 0.f; }

    if (do_bs) {
        const double *dx = pr.dxi + (size_t)(t - 1) * nf * 6;
        for (int q = tid; q < nf * 6; q += kThreads) dxs[q] = (float)dx[q];
    }

    __shared__ Chunk s_ch;
    for (int c = c_begin; c < c_end; ++c) {
        if (tid == 0) s_ch = pr.chunks[c];
        __syncthreads();
        const int k0 = s_ch.k0, cnt = s_ch.count, e0 = s_ch.e0, e1 = s_ch.e1;
        const int anc = s_ch.anchor, jlo = s_ch.jlo;
        const int W = s_ch.jhi - jlo + 1;
        const bool anc_free = anc >= t0;
        const int NG = kThreads / W;
        const int my_jl = tid % W, my_g = tid / W;
        const int my_j = jlo + my_jl;
        const bool edge_thread = my_g < NG;

        // -- stage: clear slots, load edges transposed to [frame][patch], patch data
        for (int q = tid; q < W * Gs; q += kThreads) tw[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int p = tid; p < cnt; p += kThreads) {
            const int k = k0 + p;
            const float x = pr.patches[3 * k], y = pr.patches[3 * k + 1];
            pd[p] = make_float4((x - cx) / fx, (y - cy) / fy, do_bs ? depth_old[k] : depth_new[k], 0.f);
        }
        window_poses(do_bs ? pose_old : pose_new, anc, jlo, W, rel, adj);
        __syncthreads();
        {
            const float2 *tg = reinterpret_cast<const float2 *>(pr.target);
            const float2 *wt = reinterpret_cast<const float2 *>(pr.weight);
            for (int e = e0 + tid; e < e1; e += kThreads) {
                const int p = pr.kk[e] - k0, jl = pr.jj[e] - jlo;
                const float2 a = tg[e], w = wt[e];
                tw[jl * Gs + p] = make_float4(a.x, a.y, w.x, w.y);
            }
        }
        if (do_bs && anc_free) {
            // z_k = d dxi_i,v + dxi_i,w x pbar for the anchor term of the back-substitution
            const float *di = dxs + 6 * (anc - t0);
            for (int p = tid; p < cnt; p += kThreads) {
                const float4 q = pd[p];
                const float px = q.x, py = q.y, pz = 1.f, d = q.z;
                zk[p] = make_float4(fmaf(d, di[0], di[4] * pz - di[5] * py),
                                    fmaf(d, di[1], di[5] * px - di[3] * pz),
                                    fmaf(d, di[2], di[3] * py - di[4] * px), 0.f);
            }
        }
        __syncthreads();

        // -- (a) back-substitution of the previous iteration at the old state
        if (do_bs) {
            if (edge_thread) {
                const float *R = rel + my_jl * 12;
                float Rr[12];
#pragma unroll
                for (int q = 0; q < 12; ++q) Rr[q] = R[q];
                const bool jfree = my_j >= t0 && my_j != anc;
                const float *dj = dxs + 6 * (my_j - t0);
                for (int p = my_g; p < cnt; p += NG) {
                    const int slot = my_jl * Gs + p;
                    const float4 tv = tw[slot];
                    float Ce = 0.f, we = 0.f, se = 0.f;
                    if (my_j != anc && (tv.z != 0.f || tv.w != 0.f)) {
                        const float4 q = pd[p];
                        EdgeLin E;
                        if (edge_linearize(Rr, Rr + 9, q.x, q.y, q.z, tv.x, tv.y, fx, fy, cx, cy, z_min, E)) {
                            float wjd0, wjd1;
                            depth_terms(E, tv.z, tv.w, wjd0, wjd1, Ce, we);
                            if (jfree) {
#pragma unroll
                                for (int m = 0; m < 6; ++m) se = fmaf(fmaf(E.j1[m], wjd1, E.j0[m] * wjd0), dj[m], se);
                            }
                            if (anc_free) {
                                float Y0, Y1, Y2;
                                anchor_terms(E, Rr, wjd0, wjd1, Y0, Y1, Y2);
                                const float4 z = zk[p];
                                se -= fmaf(Y2, z.z, fmaf(Y1, z.y, Y0 * z.x));
                            }
                        }
                    }
                    sc4[slot] = make_float4(Ce, we, se, 0.f);
                }
            }
            __syncthreads();
            for (int p = tid; p < cnt; p += kThreads) {
                float C = lam, w = 0.f, s = 0.f;
                for (int jl = 0; jl < W; ++jl) {
                    const float4 v = sc4[jl * Gs + p];
                    C += v.x;
                    w += v.y;
                    s += v.z;
                }
                const float dnew = pd[p].z + (w - s) / C;
                pd[p].z = dnew;
                depth_new[k0 + p] = dnew;
                if (final_pass) pr.patches[3 * (k0 + p) + 2] = dnew;
            }
            if (do_lin) window_poses(pose_new, anc, jlo, W, rel, adj);
            __syncthreads();
        }
        if (!do_lin) continue;

        // -- (b) linearise at the new state
        for (int q = tid; q < cnt * ES; q += kThreads) Ec[q] = 0.f;
        __syncthreads();
        float M[21], V[6];
#pragma unroll
        for (int q = 0; q < 21; ++q) M[q] = 0.f;
#pragma unroll
        for (int q = 0; q < 6; ++q) V[q] = 0.f;
        if (edge_thread) {
            const float *R = rel + my_jl * 12;
            float Rr[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) Rr[q] = R[q];
            const bool jfree = my_j >= t0 && my_j != anc;
            const int fj = my_j - t0;
            for (int p = my_g; p < cnt; p += NG) {
                const int slot = my_jl * Gs + p;
                const float4 tv = tw[slot];
                float Ce = 0.f, we = 0.f, Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
                if (my_j != anc && (tv.z != 0.f || tv.w != 0.f)) {
                    const float4 q = pd[p];
                    EdgeLin E;
                    if (edge_linearize(Rr, Rr + 9, q.x, q.y, q.z, tv.x, tv.y, fx, fy, cx, cy, z_min, E)) {
                        float wjd0, wjd1;
                        depth_terms(E, tv.z, tv.w, wjd0, wjd1, Ce, we);
                        anchor_terms(E, Rr, wjd0, wjd1, Y0, Y1, Y2);
                        float wj0[6], wj1[6];
#pragma unroll
                        for (int m = 0; m < 6; ++m) { wj0[m] = tv.z * E.j0[m]; wj1[m] = tv.w * E.j1[m]; }
                        // B_jj += J_j^T W J_j (the zero entries j0[1], j1[0] skipped)
#pragma unroll
                        for (int r = 0; r < 6; ++r)
#pragma unroll
                            for (int cc = r; cc < 6; ++cc) {
                                float acc = M[sym6(r, cc)];
                                if (r != 1 && cc != 1) acc = fmaf(wj0[r], E.j0[cc], acc);
                                if (r != 0 && cc != 0) acc = fmaf(wj1[r], E.j1[cc], acc);
                                M[sym6(r, cc)] = acc;
                            }
                        // v_j += J_j^T W r ; e_jk = J_j^T W J_d
#pragma unroll
                        for (int m = 0; m < 6; ++m) {
                            float vv = V[m];
                            if (m != 1) vv = fmaf(wj0[m], E.r0, vv);
                            if (m != 0) vv = fmaf(wj1[m], E.r1, vv);
                            V[m] = vv;
                        }
                        if (jfree) {
                            float *e = Ec + p * ES + 6 * fj;
                            e[0] = wj0[0] * E.jd0;
                            e[1] = wj1[1] * E.jd1;
#pragma unroll
                            for (int m = 2; m < 6; ++m) e[m] = fmaf(wj1[m], E.jd1, wj0[m] * E.jd0);
                        }
                    }
                }
                sc4[slot] = make_float4(Ce, we, Y0, Y1);
                sc1[slot] = Y2;
            }
        }
        __syncthreads();   // tw no longer read: Mp may overwrite it
        if (edge_thread) {
            float *mp = Mp + (size_t)(my_g * W + my_jl) * 27;
#pragma unroll
            for (int q = 0; q < 21; ++q) mp[q] = M[q];
#pragma unroll
            for (int q = 0; q < 6; ++q) mp[21 + q] = V[q];
        }
        // per-patch finalisation: C_k, w_k, anchor column, scaling by C_k^-1/2
        for (int p = tid; p < cnt; p += kThreads) {
            float C = lam, w = 0.f, Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
            for (int jl = 0; jl < W; ++jl) {
                const float4 v = sc4[jl * Gs + p];
                C += v.x;
                w += v.y;
                Y0 += v.z;
                Y1 += v.w;
                Y2 += sc1[jl * Gs + p];
            }
            float *e = Ec + p * ES;
            if (anc_free) {
                const float4 q = pd[p];
                const float d = q.z, px = q.x, py = q.y;
                float *ei = e + 6 * (anc - t0);
                ei[0] = -d * Y0;
                ei[1] = -d * Y1;
                ei[2] = -d * Y2;
                ei[3] = -(py * Y2 - Y1);          // -(pbar x Y), pbar = (px, py, 1)
                ei[4] = -(Y0 - px * Y2);
                ei[5] = -(px * Y1 - py * Y0);
            }
            const float sq = sqrtf(1.0f / C);
            for (int m = 0; m < 6 * nf; ++m) e[m] *= sq;
            e[6 * nf] = sq * w;
        }
        __syncthreads();
        // combine the per-thread frame sums (M_j, v_j) over patch groups, compensated
        for (int q = tid; q < W * 27; q += kThreads) {
            const int jl = q / 27, m = q % 27;
            float s = 0.f, cc = 0.f;
            for (int g = 0; g < NG; ++g) kahan_add(s, cc, Mp[(size_t)(g * W + jl) * 27 + m]);
            Mc[jl * 27 + m] = s - cc;
        }
        __syncthreads();
        // pose-pair blocks that involve the anchor:
        //   B_ij = -Ad_ij^T M_j,  B_ii = sum_j Ad_ij^T M_j Ad_ij,  v_i = -sum_j Ad_ij^T v_j
        if (anc_free) {
            for (int q = tid; q < W * 6; q += kThreads) {
                const int jl = q / 6, r = q % 6;
                const float *Ad = adj + jl * 36;
                const float *Mj = Mc + jl * 27;
                float *A = Aj + jl * 42;
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) {
                    float s = 0.f;
#pragma unroll
                    for (int m = 0; m < 6; ++m) s = fmaf(Ad[6 * m + r], Mj[sym6(m, cc)], s);
                    A[6 * r + cc] = s;
                }
                float s = 0.f;
#pragma unroll
                for (int m = 0; m < 6; ++m) s = fmaf(Ad[6 * m + r], Mj[21 + m], s);
                A[36 + r] = -s;
            }
            __syncthreads();
            if (tid < 42) {
                float s = 0.f, cc = 0.f;
                if (tid < 36) {
                    const int r = tid / 6, col = tid % 6;
                    for (int jl = 0; jl < W; ++jl) {
                        if (jlo + jl == anc) continue;
                        const float *A = Aj + jl * 42;
                        const float *Ad = adj + jl * 36;
                        float v = 0.f;
#pragma unroll
                        for (int m = 0; m < 6; ++m) v = fmaf(A[6 * r + m], Ad[6 * m + col], v);
                        kahan_add(s, cc, v);
                    }
                } else {
                    const int r = tid - 36;
                    for (int jl = 0; jl < W; ++jl) {
                        if (jlo + jl == anc) continue;
                        kahan_add(s, cc, Aj[jl * 42 + 36 + r]);
                    }
                }
                Bii[tid] = s - cc;
            }
            __syncthreads();
        }

        // -- (c) Schur accumulation over the chunk's patches, then the B blocks
        if (owns) {
            int since = 0;
            if (!is_vstrip) {
                for (int p = my_ks; p < cnt; p += KS) {
                    const float *e = Ec + p * ES;
                    float ea[3], eb[6];
#pragma unroll
                    for (int r = 0; r < 3; ++r) ea[r] = e[6 * sa + 3 * sh + r];
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) eb[cc] = e[6 * sb + cc];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int cc = 0; cc < 6; ++cc) blk[6 * r + cc] = fmaf(-ea[r], eb[cc], blk[6 * r + cc]);
                    if (++since == kFlushEvery) {
#pragma unroll
                        for (int q = 0; q < 18; ++q) { kahan_add(acc_s[q], acc_c[q], blk[q]); blk[q] = 0.f; }
                        since = 0;
                    }
                }
            } else {
                for (int p = my_ks; p < cnt; p += KS) {
                    const float *e = Ec + p * ES;
                    const float sw = e[6 * nf];
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) blk[cc] = fmaf(-e[6 * sa + cc], sw, blk[cc]);
                    if (++since == kFlushEvery) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) { kahan_add(acc_s[q], acc_c[q], blk[q]); blk[q] = 0.f; }
                        since = 0;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 18; ++q) { kahan_add(acc_s[q], acc_c[q], blk[q]); blk[q] = 0.f; }
            if (my_ks == 0) {
                const int fa = t0 + sa, fb = t0 + sb;
                const int ja = fa - jlo, jb = fb - jlo;
                const bool a_in = ja >= 0 && ja < W, b_in = jb >= 0 && jb < W;
                if (!is_vstrip) {
                    float add[18];
#pragma unroll
                    for (int q = 0; q < 18; ++q) add[q] = 0.f;
                    if (sa == sb) {
                        if (fa == anc) {
#pragma unroll
                            for (int r = 0; r < 3; ++r)
#pragma unroll
                                for (int cc = 0; cc < 6; ++cc) add[6 * r + cc] = Bii[6 * (3 * sh + r) + cc];
                        } else if (a_in) {
                            const float *Mj = Mc + ja * 27;
#pragma unroll
                            for (int r = 0; r < 3; ++r)
#pragma unroll
                                for (int cc = 0; cc < 6; ++cc) add[6 * r + cc] = Mj[sym6(3 * sh + r, cc)];
                        }
                    } else if (fa == anc && b_in) {
                        const float *A = Aj + jb * 42;          // block (i, j) = -Ad^T M_j
#pragma unroll
                        for (int r = 0; r < 3; ++r)
#pragma unroll
                            for (int cc = 0; cc < 6; ++cc) add[6 * r + cc] = -A[6 * (3 * sh + r) + cc];
                    } else if (fb == anc && a_in) {
                        const float *A = Aj + ja * 42;          // block (j, i) = -(Ad^T M_j)^T
#pragma unroll
                        for (int r = 0; r < 3; ++r)
#pragma unroll
                            for (int cc = 0; cc < 6; ++cc) add[6 * r + cc] = -A[6 * cc + 3 * sh + r];
                    }
#pragma unroll
                    for (int q = 0; q < 18; ++q) kahan_add(acc_s[q], acc_c[q], add[q]);
                } else {
                    float add[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q) add[q] = 0.f;
                    if (fa == anc) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) add[q] = Bii[36 + q];
                    } else if (a_in) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) add[q] = Mc[ja * 27 + 21 + q];
                    }
#pragma unroll
                    for (int q = 0; q < 6; ++q) kahan_add(acc_s[q], acc_c[q], add[q]);
                }
            }
        }
        __syncthreads();
    }

    // write this CTA's partial of (S, v')
    if (owns) {
        double *out = pr.partial + ((size_t)itm.item * KS + my_ks) * pr.L;
        if (!is_vstrip) {
            double *o = out + 18 * my_strip;
#pragma unroll
            for (int q = 0; q < 18; ++q) o[q] = (double)acc_s[q] - (double)acc_c[q];
        } else {
            double *o = out + 18 * nbs + 6 * sa;
#pragma unroll
            for (int q = 0; q < 6; ++q) o[q] = (double)acc_s[q] - (double)acc_c[q];
        }
    }
    if (final_pass && itm.item == 0) {
        for (int q = tid; q < N * 7; q += kThreads) pr.poses[q] = pose_new[q];
    }
}

// ----------------------------------------------------------------------------
// solve_kernel: one CTA per problem.  Sums the Schur partials in FP64, factors
// S = L L^T (FP64, right-looking, in shared memory), solves S dxi = v', and
// retracts the free poses.  If S_out is non-null, writes (S, v') there instead
// and changes nothing else.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) solve_kernel(const Prob *__restrict__ probs, int t,
                                                         double *S_out, double *v_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Prob &pr = probs[blockIdx.x];
    const int tid = threadIdx.x;
    if (t >= pr.iters) return;
    const int N = pr.N, t0 = pr.t0, nf = pr.nf, n = 6 * nf;
    const float *pose_cur = pr.pose_it + (size_t)t * N * 7;
    float *pose_next = pr.pose_it + (size_t)(t + 1) * N * 7;
    double *dxi = pr.dxi + (size_t)t * nf * 6;
    __shared__ int s_flag;
    if (tid == 0) s_flag = *pr.status;
    __syncthreads();
    if (s_flag != 0 || nf == 0) {
        if (S_out == nullptr) {
            for (int q = tid; q < N * 7; q += kThreads) pose_next[q] = pose_cur[q];
            for (int q = tid; q < nf * 6; q += kThreads) dxi[q] = 0.0;
        }
        return;
    }
    const int ld = n + 1;
    double *S = reinterpret_cast<double *>(smem);
    double *v = S + (size_t)n * ld;

    // FP64 sum of the partials in a fixed order (deterministic)
    const int Lp = pr.L, nparts = pr.n_items * pr.ks, nbs = 2 * n_block_pairs(nf);
    for (int q = tid; q < Lp; q += kThreads) {
        double acc = 0.0;
        for (int part = 0; part < nparts; ++part) acc += pr.partial[(size_t)part * Lp + q];
        if (q < 18 * nbs) {
            const int s = q / 18, e = q % 18;
            int a, b;
            decode_pair(s >> 1, nf, a, b);
            const int row = 6 * a + 3 * (s & 1) + e / 6, col = 6 * b + e % 6;
            S[row * ld + col] = acc;
            if (a != b) S[col * ld + row] = acc;
        } else {
            v[q - 18 * nbs] = acc;
        }
    }
    __syncthreads();
    if (S_out != nullptr) {
        for (int q = tid; q < n * n; q += kThreads) S_out[q] = S[(q / n) * ld + q % n];
        for (int q = tid; q < n; q += kThreads) v_out[q] = v[q];
        return;
    }
    // Cholesky, lower triangle, in place
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            const double piv = S[j * ld + j];
            if (!(piv > 0.0)) s_flag = DPVO_BA_STATUS_NOT_SPD;
            else S[j * ld + j] = sqrt(piv);
        }
        __syncthreads();
        if (s_flag) break;
        const double djj = S[j * ld + j];
        for (int i = j + 1 + tid; i < n; i += kThreads) S[i * ld + j] /= djj;
        __syncthreads();
        const int m = n - j - 1;
        for (int q = tid; q < m * m; q += kThreads) {
            const int ii = q / m, kk = q % m;
            if (kk <= ii) S[(j + 1 + ii) * ld + j + 1 + kk] -= S[(j + 1 + ii) * ld + j] * S[(j + 1 + kk) * ld + j];
        }
        __syncthreads();
    }
    if (!s_flag) {
        // L y = v'
        for (int j = 0; j < n; ++j) {
            if (tid == 0) v[j] /= S[j * ld + j];
            __syncthreads();
            for (int i = j + 1 + tid; i < n; i += kThreads) v[i] -= S[i * ld + j] * v[j];
            __syncthreads();
        }
        // L^T x = y
        for (int j = n - 1; j >= 0; --j) {
            if (tid == 0) v[j] /= S[j * ld + j];
            __syncthreads();
            for (int i = tid; i < j; i += kThreads) v[i] -= S[j * ld + i] * v[j];
            __syncthreads();
        }
        if (tid == 0) {
            for (int q = 0; q < n; ++q)
                if (!isfinite(v[q])) s_flag = DPVO_BA_STATUS_NONFINITE;
        }
        __syncthreads();
    }
    if (s_flag) {
        if (tid == 0) *pr.status = s_flag;
        for (int q = tid; q < N * 7; q += kThreads) pose_next[q] = pose_cur[q];
        for (int q = tid; q < nf * 6; q += kThreads) dxi[q] = 0.0;
        return;
    }
    for (int q = tid; q < n; q += kThreads) dxi[q] = v[q];
    for (int a = tid; a < N; a += kThreads) {
        if (a >= t0) se3_left_update(v + 6 * (a - t0), pose_cur + 7 * a, pose_next + 7 * a);
        else
            for (int q = 0; q < 7; ++q) pose_next[7 * a + q] = pose_cur[7 * a + q];
    }
}

}  // namespace dpvo
