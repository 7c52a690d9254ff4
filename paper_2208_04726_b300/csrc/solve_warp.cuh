// solve_warp_kernel: the reduced solve of the Gauss-Newton step (Sec. 3.1: the
// Schur-complement system over the free poses, solved by Cholesky, then the
// retraction of the poses) for at most kFusedMaxFree free poses (n = 6 x free
// poses <= 90), one CTA of four warps per problem.
//
// A reduced system this small is a chain of short dependent steps, and B300
// runs FP64 at a small fraction of its FP32 rate.  So the FP32 chain (the
// factorisation and the triangular solves) runs in ONE warp with no barrier
// wider than __syncwarp, and the FP64 sums (the partials, the refinement
// residuals) use all four warps, one per SM sub-partition:
//
//   1. (all warps) S and v' = the FP64 sum of the problem's Schur partials, in
//      the parts' order; an FP32 copy of the lower triangle of S alongside.
//   2. (warp 0) The FP32 copy factored as S = L D L^T (L unit lower, D the
//      pivots d_j: the square-root-free Cholesky form) by panels of kSwBlk
//      columns.  Every lane factors the panel's diagonal block itself, in
//      registers, from broadcast loads; lane l then eliminates its rows l,
//      l + 32, l + 64 below the block, stores their multipliers, and applies
//      the panel's rank-kSwBlk update to the trailing columns of its rows,
//      reading the multipliers of the trailing rows as broadcast loads.  Lanes
//      0..7 also form the inverse of the diagonal block (for step 4).  A pivot
//      <= 0, or a reciprocal that is not finite, hands the problem to step 5.
//   3. (warp 0) x = S32^-1 v', the triangular solves a block at a time: the
//      block's right-hand side times its inverse, then the other rows updated
//      with the block's solution, both exchanged through shared memory.
//   4. Refinement in FP64: r = v' - S x (all warps), x += S32^-1 r (warp 0),
//      until a correction is below kRefineTol of x, or the first correction is
//      below 1e-4 of x (the refinement then contracts by about that ratio, so
//      the next correction would be below 1e-8 of x).  A correction that does
//      not halve, a non-finite one, or kMaxRefine of them hand the problem to
//      step 5.
//   5. (fallback, warp 0) FP64 elimination of S and back substitution.
//   6. (warp 0) The pose increments (FP64) and the retraction T <- Exp(dxi) T
//      of the free poses (se3_left_update).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "ba_common.cuh"
#include "kernels.cuh"
#include "se3.cuh"

namespace dpvo {

constexpr int kSwThreads = 128;        // four warps
constexpr int kSwBlk = 8;              // panel width and diagonal block size
constexpr int kSwMLd = 12;             // row stride of an inverted diagonal block (16-byte rows)
constexpr int kSwMSize = kSwBlk * kSwMLd;
constexpr unsigned kSwFull = 0xffffffffu;

// Row stride of the FP32 factor: at least n rounded up to a panel, and 4 mod
// 32, so that 16-byte row segments of 8 consecutive rows fall in distinct
// bank groups.
__host__ __device__ inline int sw_ldf(int n) { return ((((n + 7) & ~7) - 4 + 31) / 32) * 32 + 4; }

// Shared-memory layout for n = 6 nf (byte offsets, 16-byte aligned): S (FP64,
// n x (n+1), both triangles), v' and x (FP64), the FP32 factor (n x ldf), the
// pivot reciprocals, each diagonal block's inverse and its transpose, two
// FP32 vectors of the solves, each warp's copy of a panel's multipliers.
struct SwLayout {
    size_t S, v, x, Sf, rp, Minv, yb, zs, Lc, bytes;
};
__host__ __device__ inline SwLayout sw_layout(int nf) {
    const size_t n = 6 * (size_t)nf, n8 = (n + 7) & ~size_t(7), nblk = n8 / kSwBlk;
    SwLayout L;
    L.S = 0;
    L.v = L.S + n * (n + 1) * 8;
    L.x = L.v + n * 8;
    L.Sf = L.x + n * 8;
    L.rp = L.Sf + n * sw_ldf((int)n) * 4;
    L.Minv = L.rp + n8 * 4;
    L.yb = L.Minv + nblk * 2 * kSwMSize * 4;
    L.zs = L.yb + n8 * 4;
    L.Lc = L.zs + n8 * 4;
    L.bytes = L.Lc + (kSwThreads / 32) * n8 * kSwBlk * 4;
    return L;
}
__host__ __device__ inline size_t sw_smem_bytes(int nf) { return sw_layout(nf).bytes; }

// Rows per lane of the factor for n = 6 nf (2 up to n = 64, else 3).
__host__ __device__ inline int sw_rows(int nf) { return 6 * nf <= 64 ? 2 : 3; }

// a[u] for a warp-uniform u, without indexing a register array at run time.
template <int R>
__device__ __forceinline__ float sw_pick(const float (&a)[R], int u) {
    float r = a[0];
#pragma unroll
    for (int w = 1; w < R; ++w)
        if (u == w) r = a[w];
    return r;
}
template <int R>
__device__ __forceinline__ void sw_put(float (&a)[R], int u, float x) {
#pragma unroll
    for (int w = 0; w < R; ++w)
        if (u == w) a[w] = x;
}

// 8 consecutive floats from a 16-byte aligned address.
__device__ __forceinline__ void sw_ld8(const float *p, float (&o)[kSwBlk]) {
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void sw_st8(float *p, const float (&o)[kSwBlk]) {
    *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<float4 *>(p + 4) = make_float4(o[4], o[5], o[6], o[7]);
}

// Approximate reciprocal of a pivot (PTX rcp.approx: within an ulp; the FP32
// factor only preconditions the FP64 refinement).  Subnormal pivots flush to
// zero and give an infinite reciprocal, which fails the pivot test.
__device__ __forceinline__ float sw_rcp(float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return r;
}

// Rank-kSwBlk update of kw <= 4 consecutive columns k0.. (k0 a multiple of
// 4) of my rows: a_ik -= sum_q a_{i,J+q} l_{k,J+q}, the multipliers l_k of the
// trailing rows read from this warp's copy Lw (row k at Lw + kSwBlk k) as
// broadcast loads.  A full group moves a row's four entries as one 16-byte
// access; entries above the diagonal in it are updated too and never read.
template <int R>
__device__ __forceinline__ void sw_trail_group(float *Sf, int ldf, const float *Lw, int k0, int kw, int n,
                                               int lane, const float (&p)[R][kSwBlk]) {
    float lk[4][kSwBlk];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        if (kk < kw) {
            sw_ld8(Lw + (k0 + kk) * kSwBlk, lk[kk]);
        } else {
#pragma unroll
            for (int q = 0; q < kSwBlk; ++q) lk[kk][q] = 0.f;
        }
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int i = lane + 32 * u;
        if (i < k0 || i >= n) continue;
        float *row = Sf + i * ldf + k0;
        float a[4];
        if (kw == 4) {
            const float4 a4 = *reinterpret_cast<const float4 *>(row);
            a[0] = a4.x; a[1] = a4.y; a[2] = a4.z; a[3] = a4.w;
        } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) a[kk] = kk < kw ? row[kk] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < kSwBlk; ++q)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) a[kk] = fmaf(-p[u][q], lk[kk][q], a[kk]);
        if (kw == 4) {
            *reinterpret_cast<float4 *>(row) = make_float4(a[0], a[1], a[2], a[3]);
        } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                if (kk < kw) row[kk] = a[kk];
        }
    }
}

// Step 2, all kSwThreads threads.  Sf (row stride ldf; both triangles on
// entry, padding columns zero) receives the multipliers l_ij below the
// diagonal blocks; rp[j] = 1 / d_j; Minv holds, per diagonal block, its
// inverse M (row-major, stride kSwMLd) and then M^T.  Per panel: every warp
// factors the diagonal block and eliminates the rows below it (lane l: rows
// l, l + 32, l + 64), keeping the multipliers in a copy of its own (Lw); each
// warp then updates every fourth group of 4 trailing columns; one block
// barrier ends the panel.  Returns false, in every thread, for a failed pivot
// (the factor is then incomplete).
template <int R>
__device__ bool sw_factor(float *Sf, int ldf, float *rp, float *Minv, float *Lcopies, int n, int tid) {
    const int lane = tid & 31, warp = tid >> 5, n8 = (n + 7) & ~7;
    float *Lw = Lcopies + warp * n8 * kSwBlk;
    for (int J = 0; J < n; J += kSwBlk) {
        const int nb = min(kSwBlk, n - J);
        // the diagonal block in every lane (rows past n padded with the identity)
        float a[kSwBlk][kSwBlk], lb[kSwBlk][kSwBlk], rq[kSwBlk];
#pragma unroll
        for (int r = 0; r < kSwBlk; ++r) {
            if (r < nb) {
                sw_ld8(Sf + (J + r) * ldf + J, a[r]);
            } else {
#pragma unroll
                for (int q = 0; q < kSwBlk; ++q) a[r][q] = r == q ? 1.f : 0.f;
            }
        }
        bool ok = true;
#pragma unroll
        for (int q = 0; q < kSwBlk; ++q) {
            const float d = a[q][q], r = sw_rcp(d);
            ok = ok && d > 0.f && isfinite(r);
            rq[q] = r;
#pragma unroll
            for (int r2 = q + 1; r2 < kSwBlk; ++r2) lb[r2][q] = a[r2][q] * r;
#pragma unroll
            for (int r2 = q + 1; r2 < kSwBlk; ++r2)
#pragma unroll
                for (int q2 = q + 1; q2 <= r2; ++q2) a[r2][q2] = fmaf(-a[r2][q], lb[q2][q], a[r2][q2]);
        }
        if (!ok) return false;                   // the same decision in every thread
        // my rows below the block: eliminate the panel's columns; multipliers into Lw
        float p[R][kSwBlk], l[R][kSwBlk];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int i = lane + 32 * u;
            if (i >= J + kSwBlk && i < n) {      // rows below exist only under a full panel
                sw_ld8(Sf + i * ldf + J, p[u]);
#pragma unroll
                for (int q = 0; q < kSwBlk; ++q)
#pragma unroll
                    for (int q2 = q + 1; q2 < kSwBlk; ++q2) p[u][q2] = fmaf(-p[u][q], lb[q2][q], p[u][q2]);
#pragma unroll
                for (int q = 0; q < kSwBlk; ++q) l[u][q] = p[u][q] * rq[q];
                sw_st8(Lw + i * kSwBlk, l[u]);
            } else {
#pragma unroll
                for (int q = 0; q < kSwBlk; ++q) p[u][q] = l[u][q] = 0.f;
            }
        }
        if (warp == 0) {
            if (lane == 0) sw_st8(rp + J, rq);   // rp is padded to a whole panel
            if (lane < nb) {                     // column c = lane of the block's inverse
                const int c = lane;
                float m[kSwBlk];
#pragma unroll
                for (int r = 0; r < kSwBlk; ++r) {
                    float acc = r == c ? 1.f : 0.f;
#pragma unroll
                    for (int q = 0; q < r; ++q)
                        if (q >= c) acc = fmaf(-lb[r][q], m[q], acc);
                    m[r] = acc;
                }
                float *M = Minv + (J / kSwBlk) * 2 * kSwMSize;
#pragma unroll
                for (int r = 0; r < kSwBlk; ++r) M[r * kSwMLd + c] = m[r];
                sw_st8(M + kSwMSize + c * kSwMLd, m);   // row c of M^T
            }
        }
        __syncwarp();
        // rank-kSwBlk update of the trailing columns, groups of 4 dealt to the warps in turn
        for (int k0 = J + kSwBlk + 4 * warp; k0 < n; k0 += 16)
            sw_trail_group<R>(Sf, ldf, Lw, k0, min(4, n - k0), n, lane, p);
        __syncthreads();
        // the multipliers into the factor (every warp has read this panel's columns)
        if (warp == 0) {
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int i = lane + 32 * u;
                if (i >= J + kSwBlk && i < n) sw_st8(Sf + i * ldf + J, l[u]);
            }
        }
    }
    __syncwarp();
    return true;
}

// Step 3's solve, one warp: y <- S32^-1 y, y[u] the entry of row lane + 32 u.
// yb and zs are FP32 vectors in shared memory, padded to a whole panel.
template <int R>
__device__ void sw_solve(const float *Sf, int ldf, const float *rp, const float *Minv, float *yb, float *zs,
                         float (&y)[R], int n, int lane) {
    const int nblk = (n + kSwBlk - 1) / kSwBlk;
#pragma unroll
    for (int u = 0; u < R; ++u)
        if (lane + 32 * u < n) yb[lane + 32 * u] = y[u];
    __syncwarp();
    for (int blk = 0; blk < nblk; ++blk) {       // L z = y
        const int J = blk * kSwBlk, nb = min(kSwBlk, n - J), uJ = J >> 5, c = lane - (J & 31);
        float bJ[kSwBlk];
        sw_ld8(yb + J, bJ);
        if (c >= 0 && c < nb) {                  // z_c = sum_q M[c][q] b_q
            float m[kSwBlk];
            sw_ld8(Minv + blk * 2 * kSwMSize + c * kSwMLd, m);
            float z0 = 0.f, z1 = 0.f;
#pragma unroll
            for (int q = 0; q < kSwBlk; q += 2) {
                if (q < nb) z0 = fmaf(m[q], bJ[q], z0);
                if (q + 1 < nb) z1 = fmaf(m[q + 1], bJ[q + 1], z1);
            }
            const float z = z0 + z1;
            sw_put<R>(y, uJ, z);
            zs[J + c] = z;
        }
        __syncwarp();
        if (J + kSwBlk < n) {                    // rows below (full blocks only)
            sw_ld8(zs + J, bJ);
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int i = lane + 32 * u;
                if (i >= J + kSwBlk && i < n) {
                    float l[kSwBlk];
                    sw_ld8(Sf + i * ldf + J, l);
                    float a0 = y[u], a1 = 0.f;
#pragma unroll
                    for (int q = 0; q < kSwBlk; q += 2) {
                        a0 = fmaf(-l[q], bJ[q], a0);
                        a1 = fmaf(-l[q + 1], bJ[q + 1], a1);
                    }
                    y[u] = a0 + a1;
                    yb[i] = y[u];
                }
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {                // D^-1
        const int i = lane + 32 * u;
        if (i < n) {
            y[u] *= rp[i];
            yb[i] = y[u];
        }
    }
    __syncwarp();
    for (int blk = nblk - 1; blk >= 0; --blk) {  // L^T x = z
        const int J = blk * kSwBlk, nb = min(kSwBlk, n - J), uJ = J >> 5, c = lane - (J & 31);
        float wJ[kSwBlk];
        sw_ld8(yb + J, wJ);
        if (c >= 0 && c < nb) {                  // x_c = sum_q M^T[c][q] w_q
            float m[kSwBlk];
            sw_ld8(Minv + blk * 2 * kSwMSize + kSwMSize + c * kSwMLd, m);
            float x0 = 0.f, x1 = 0.f;
#pragma unroll
            for (int q = 0; q < kSwBlk; q += 2) {
                if (q < nb) x0 = fmaf(m[q], wJ[q], x0);
                if (q + 1 < nb) x1 = fmaf(m[q + 1], wJ[q + 1], x1);
            }
            const float x = x0 + x1;
            sw_put<R>(y, uJ, x);
            zs[J + c] = x;
        }
        __syncwarp();
        if (J > 0) {                             // rows above: y_r -= sum_q l_{J+q, r} x_{J+q}
            sw_ld8(zs + J, wJ);
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int r = lane + 32 * u;
                if (r < J) {
                    float a0 = y[u], a1 = 0.f;
#pragma unroll
                    for (int q = 0; q < kSwBlk; q += 2) {
                        if (q < nb) a0 = fmaf(-Sf[(J + q) * ldf + r], wJ[q], a0);
                        if (q + 1 < nb) a1 = fmaf(-Sf[(J + q + 1) * ldf + r], wJ[q + 1], a1);
                    }
                    y[u] = a0 + a1;
                    yb[r] = y[u];
                }
            }
            __syncwarp();
        }
    }
}

// Step 4's residual, all kSwThreads threads: yb = (float)(v' - S x), four
// threads per row (columns k = j mod 4), the four partial sums added pairwise.
__device__ inline void sw_residual(const double *S, int ld, const double *v, const double *x, float *yb, int n,
                                   int tid) {
    const int j = tid & 3;
    for (int i0 = 0; i0 < n; i0 += kSwThreads / 4) {
        const int i = i0 + (tid >> 2);
        double acc = 0.0;
        if (i < n) {
            const double *Srow = S + (size_t)i * ld;
            for (int k = j; k < n; k += 4) acc = fma(Srow[k], x[k], acc);
        }
        acc += __shfl_xor_sync(kSwFull, acc, 1);
        acc += __shfl_xor_sync(kSwFull, acc, 2);
        if (i < n && j == 0) yb[i] = (float)(v[i] - acc);
    }
}

// Step 5, one warp: right-looking FP64 elimination of the lower triangle of S
// (row stride ld) with v eliminated alongside, then back substitution; v ends
// as the solution.  Returns false for a pivot <= 0 or NaN.
__device__ inline bool sw_solve_f64(double *S, double *v, int n, int ld, int lane) {
    for (int j = 0; j < n; ++j) {
        const double d = S[j * ld + j];
        if (!(d > 0.0)) return false;
        const double r = 1.0 / d;
        for (int i = j + 1 + lane; i < n; i += 32) {
            const double f = S[i * ld + j] * r;
            for (int k = j + 1; k <= i; ++k) S[i * ld + k] = fma(-f, S[k * ld + j], S[i * ld + k]);
            v[i] = fma(-f, v[j], v[i]);
        }
        __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {          // x_j = v_j / d_j, then v_i -= a_ji x_j (i < j)
        const double xj = v[j] / S[j * ld + j];
        for (int i = lane; i < j; i += 32) v[i] = fma(-S[j * ld + i], xj, v[i]);
        __syncwarp();
        if (lane == 0) v[j] = xj;
        __syncwarp();
    }
    return true;
}

constexpr int kSwCluster = 8;          // CTAs summing the partials of a problem that has several
constexpr int kSwDirectParts = 4;      // partials per problem up to which one CTA sums them itself

// One CTA of kSwThreads per problem, which sums the problem's Schur partials
// itself, or, where some problem of the batch has more than kSwDirectParts
// partials, a cluster of csize = kSwCluster CTAs per problem: each sums a
// slice of the partials' entries into the shared memory of the cluster's
// first CTA, which then solves.  Both sum the parts in their order.
// R = sw_rows(nf) of the batch's largest problem.  Problems that keep the
// FP64 factor for the adjoint use solve_kernel.
template <int R>
__global__ void __launch_bounds__(kSwThreads) solve_warp_kernel(const Prob *__restrict__ probs, int t, int csize) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_state;                      // 1: refine again, 0: x final, 2: FP64 elimination
    __shared__ int s_status;
    const int b = blockIdx.x / csize, rank = blockIdx.x - b * csize;
    const Prob &pr = probs[b];
    const int tid = threadIdx.x, lane = tid & 31;
    if (t >= pr.iters) return;
    const int N = pr.N, t0 = pr.t0, nf = pr.nf, n = 6 * nf, ld = n + 1;
    const float *pose_cur = pr.pose_it + (size_t)t * N * 7;
    float *pose_next = pr.pose_it + (size_t)(t + 1) * N * 7;
    double *dxi = pr.dxi + (size_t)t * nf * 6;
    const SwLayout lay = sw_layout(nf);
    const int ldf = sw_ldf(n);
    double *S = reinterpret_cast<double *>(smem + lay.S);
    double *v = reinterpret_cast<double *>(smem + lay.v);
    double *x = reinterpret_cast<double *>(smem + lay.x);
    float *Sf = reinterpret_cast<float *>(smem + lay.Sf);
    float *rp = reinterpret_cast<float *>(smem + lay.rp);
    float *Minv = reinterpret_cast<float *>(smem + lay.Minv);
    float *yb = reinterpret_cast<float *>(smem + lay.yb);
    float *zs = reinterpret_cast<float *>(smem + lay.zs);
    float *Lc = reinterpret_cast<float *>(smem + lay.Lc);

    // -- 1. the summed partial (S: strips of 3 x 6 entries of block pair (a,
    // b), a <= b; then v'), a strip per thread, loaded while thread 0 reads
    // the status.  S gets both triangles, the FP32 copy too; the FP32 copy's
    // padding columns are zeroed.
    const int nbs = 2 * n_block_pairs(nf);
    float pin[7];                                // warp 0: pose `lane`, read now for the retraction
    if (tid < 32 && lane < N)
#pragma unroll
        for (int q = 0; q < 7; ++q) pin[q] = pose_cur[7 * lane + q];
    constexpr int kStrips = 2;                   // strips per thread with loads in flight together
    if (csize > 1) {
        // several partials: this CTA's slice of the entries, summed in the
        // parts' order, into the first CTA's S, FP32 copy and v'
        if (tid == 0) s_status = *pr.status;
        __syncthreads();
        if (s_status != 0 || nf == 0) {          // the same exit in every CTA of the cluster
            if (rank == 0) {
                for (int q = tid; q < N * 7; q += kSwThreads) pose_next[q] = pose_cur[q];
                for (int q = tid; q < nf * 6; q += kSwThreads) dxi[q] = 0.0;
            }
            return;
        }
        cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
        double *S0 = cl.map_shared_rank(S, 0), *v0 = cl.map_shared_rank(v, 0);
        float *Sf0 = cl.map_shared_rank(Sf, 0);
        const int Lp = pr.L, P = pr.n_parts, per = (Lp + csize - 1) / csize;
        const int q_lo = min(Lp, rank * per), q_hi = min(Lp, q_lo + per);
        constexpr int kE = 2, kG = 8;            // entries per thread, parts per group of loads
        for (int q0 = q_lo + tid; q0 < q_hi; q0 += kE * kSwThreads) {
            double acc[kE];
#pragma unroll
            for (int e = 0; e < kE; ++e) {
                const int q = q0 + e * kSwThreads;
                acc[e] = q < q_hi ? __ldg(pr.partial + q) : 0.0;
            }
            for (int part = 1; part < P; part += kG) {
                double xv[kE][kG];
#pragma unroll
                for (int e = 0; e < kE; ++e)
#pragma unroll
                    for (int u = 0; u < kG; ++u) {
                        const int q = q0 + e * kSwThreads;
                        xv[e][u] = q < q_hi && part + u < P ? __ldg(pr.partial + (size_t)(part + u) * Lp + q) : 0.0;
                    }
#pragma unroll
                for (int u = 0; u < kG; ++u)
#pragma unroll
                    for (int e = 0; e < kE; ++e)
                        if (part + u < P) acc[e] += xv[e][u];
            }
#pragma unroll
            for (int e = 0; e < kE; ++e) {
                const int q = q0 + e * kSwThreads;
                if (q >= q_hi) continue;
                if (q < 18 * nbs) {
                    const int st = q / 18, e18 = q - 18 * st;
                    int a, bb;
                    decode_pair(st >> 1, nf, a, bb);
                    const int row = 6 * a + 3 * (st & 1) + e18 / 6, col = 6 * bb + e18 % 6;
                    const float f = (float)acc[e];
                    S0[row * ld + col] = acc[e];
                    Sf0[row * ldf + col] = f;
                    if (a != bb) {
                        S0[col * ld + row] = acc[e];
                        Sf0[col * ldf + row] = f;
                    }
                } else {
                    v0[q - 18 * nbs] = acc[e];
                }
            }
        }
        if (rank == 0)
            for (int q = tid; q < n; q += kSwThreads)
                for (int c = n; c < ldf; ++c) Sf[q * ldf + c] = 0.f;
        cl.sync();
        if (rank != 0) return;
    }
    const int n_parts = csize == 1 ? pr.n_parts : 1;
    auto v_entry = [&](int q) {                  // entry q of v', summed over the parts
        double s = pr.partial[18 * nbs + q];
        for (int part = 1; part < n_parts; ++part) s += pr.partial[(size_t)part * pr.L + 18 * nbs + q];
        return s;
    };
    for (int st0 = 0; csize == 1 && st0 < max(nbs, 1); st0 += kStrips * kSwThreads) {
        double2 d2[kStrips][9];
#pragma unroll
        for (int h = 0; h < kStrips; ++h) {
            const int st = st0 + h * kSwThreads + tid;
            if (st < nbs) {
                const double2 *src = reinterpret_cast<const double2 *>(pr.partial + (size_t)st * 18);
#pragma unroll
                for (int e = 0; e < 9; ++e) d2[h][e] = src[e];
            }
        }
        for (int part = 1; part < n_parts; ++part) {
            double2 p2[kStrips][9];
#pragma unroll
            for (int h = 0; h < kStrips; ++h) {
                const int st = st0 + h * kSwThreads + tid;
                if (st < nbs) {
                    const double2 *src =
                        reinterpret_cast<const double2 *>(pr.partial + (size_t)part * pr.L + (size_t)st * 18);
#pragma unroll
                    for (int e = 0; e < 9; ++e) p2[h][e] = src[e];
                }
            }
#pragma unroll
            for (int h = 0; h < kStrips; ++h)
#pragma unroll
                for (int e = 0; e < 9; ++e) {
                    d2[h][e].x += p2[h][e].x;
                    d2[h][e].y += p2[h][e].y;
                }
        }
        double vq = 0.0;
        if (st0 == 0) {
            if (tid < n) vq = v_entry(tid);
            if (tid == 0) s_status = *pr.status;
            __syncthreads();
            if (s_status != 0 || nf == 0) {      // uniform: every thread passed the barrier
                for (int q = tid; q < N * 7; q += kSwThreads) pose_next[q] = pose_cur[q];
                for (int q = tid; q < nf * 6; q += kSwThreads) dxi[q] = 0.0;
                return;
            }
            for (int q = tid; q < n; q += kSwThreads) {
                v[q] = q == tid ? vq : v_entry(q);
                for (int c = n; c < ldf; ++c) Sf[q * ldf + c] = 0.f;
            }
        }
#pragma unroll
        for (int h = 0; h < kStrips; ++h) {
            const int st = st0 + h * kSwThreads + tid;
            if (st >= nbs) continue;
            int a, b;
            decode_pair(st >> 1, nf, a, b);
            const int row0 = 6 * a + 3 * (st & 1), col0 = 6 * b;
#pragma unroll
            for (int e = 0; e < 18; ++e) {
                const double val = (e & 1) ? d2[h][e >> 1].y : d2[h][e >> 1].x;
                const int row = row0 + e / 6, col = col0 + e % 6;
                const float f = (float)val;
                S[row * ld + col] = val;
                Sf[row * ldf + col] = f;
                if (a != b) {
                    S[col * ld + row] = val;
                    Sf[col * ldf + row] = f;
                }
            }
        }
    }
    __syncthreads();

    // -- 2. FP32 factor (all warps), 3. the first solve (warp 0)
    const bool factored = !pr.solve_f64 && sw_factor<R>(Sf, ldf, rp, Minv, Lc, n, tid);
    float y[R], xf[R];                           // warp 0: my rows' correction and FP32 view of x
    double prev = 0.0;
    if (tid < 32) {
        int state = 2;
        if (factored) {
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int i = lane + 32 * u;
                y[u] = i < n ? (float)v[i] : 0.f;
            }
            sw_solve<R>(Sf, ldf, rp, Minv, yb, zs, y, n, lane);
            float xm = 0.f;
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int i = lane + 32 * u;
                xf[u] = y[u];
                if (i < n) x[i] = (double)y[u];
                xm = fmaxf(xm, fabsf(y[u]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) xm = fmaxf(xm, __shfl_xor_sync(kSwFull, xm, o));
            state = xm <= 3e38f ? 1 : 2;         // NaN or overflow: FP64
            prev = xm;
        }
        if (lane == 0) s_state = state;
    }
    __syncthreads();

    // -- 4. refinement: residual by all warps, correction by warp 0
    for (int it = 1; s_state == 1; ++it) {
        sw_residual(S, ld, v, x, yb, n, tid);
        __syncthreads();
        if (tid < 32) {
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int i = lane + 32 * u;
                y[u] = i < n ? yb[i] : 0.f;
            }
            __syncwarp();
            sw_solve<R>(Sf, ldf, rp, Minv, yb, zs, y, n, lane);
            float dm = 0.f, xm = 0.f;
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int i = lane + 32 * u;
                if (i < n) x[i] += (double)y[u];
                xf[u] += y[u];
                dm = fmaxf(dm, fabsf(y[u]));
                xm = fmaxf(xm, fabsf(xf[u]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dm = fmaxf(dm, __shfl_xor_sync(kSwFull, dm, o));
                xm = fmaxf(xm, __shfl_xor_sync(kSwFull, xm, o));
            }
            int state = 1;
            if (!(dm <= 3e38f)) state = 2;
            else if (dm <= (float)kRefineTol * xm || (it == 1 && dm <= 1e-4f * xm)) state = 0;
            else if ((it > 1 && !(dm <= 0.5f * (float)prev)) || it == kMaxRefine) state = 2;
            prev = dm;
            __syncwarp();
            if (lane == 0) s_state = state;
        }
        __syncthreads();
    }
    if (tid >= 32) return;

    // -- 5. FP64 fallback on S, which the FP32 path left untouched
    int status = 0;
    if (s_state == 2) {
        if (!sw_solve_f64(S, v, n, ld, lane)) status = DPVO_BA_STATUS_NOT_SPD;
    } else {
        for (int q = lane; q < n; q += 32) v[q] = x[q];
    }
    __syncwarp();
    if (!status) {
        bool bad = false;
        for (int q = lane; q < n; q += 32) bad |= !isfinite(v[q]);
        if (__any_sync(kSwFull, bad)) status = DPVO_BA_STATUS_NONFINITE;
    }

    // -- 6. increments and retraction
    if (status) {
        if (lane == 0) *pr.status = status;
        for (int q = lane; q < N * 7; q += 32) pose_next[q] = pose_cur[q];
        for (int q = lane; q < nf * 6; q += 32) dxi[q] = 0.0;
        return;
    }
    for (int q = lane; q < n; q += 32) dxi[q] = v[q];
    for (int a = lane; a < N; a += 32) {
        if (a >= 32)
#pragma unroll
            for (int q = 0; q < 7; ++q) pin[q] = pose_cur[7 * a + q];
        if (a >= t0) {
            se3_left_update(v + 6 * (a - t0), pin, pose_next + 7 * a);
        } else {
#pragma unroll
            for (int q = 0; q < 7; ++q) pose_next[7 * a + q] = pin[q];
        }
    }
}

}  // namespace dpvo
