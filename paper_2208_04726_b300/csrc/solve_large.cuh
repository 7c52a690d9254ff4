// The reduced solve for more than 15 free poses (Sec. 3.1: the Schur complement
// system over the free poses, solved by Cholesky; n = 6 x free poses up to 192).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "ba_common.cuh"
#include "kernels.cuh"

namespace dpvo {

// ----------------------------------------------------------------------------
// solve_large_kernel: the reduced solve for more than kFusedMaxFree free poses
// (n = 6 nf up to 192), one CTA per problem.  S is packed, lower triangle by
// rows: (i, k), k <= i, at i (i + 1) / 2 + k.  The FP64 sum of the partials
// goes to the workspace (pr.sglob, read again by the FP64 residuals) and,
// equilibrated (Dg S Dg, Dg = diag(S)^-1/2) and rounded, to an FP32 copy in
// shared memory.  The copy is factored in place, S = U D^-1 U^T, by panels of
// 32 columns (the diagonal block by one warp, the rows below by one thread
// each, the trailing triangle by a rank-32 update in 4 x 4 register tiles);
// the diagonal blocks are then inverted, so the triangular solves are panel
// matrix-vector products.  The solution is refined in FP64 (each correction
// solves (Dg S Dg) y = Dg r and adds Dg y) until the correction is below
// kRefineTol of the solution.  Fallback (an FP32 pivot fails or the
// corrections stall): FP64 elimination of S loaded packed into shared memory.
// ----------------------------------------------------------------------------
__host__ __device__ inline int packed_index(int i, int k) { return i * (i + 1) / 2 + k; }
struct PackedIdx {
    __device__ __forceinline__ int operator()(int i, int k) const { return packed_index(i, k); }
};

constexpr int kDiagLd = 36;            // row stride (floats) of a staged diagonal block (16-byte rows)

// FP32 path of solve_large_kernel, in floats from the start of the packed
// copy: the copy (np) and the right-hand side (n), then the two panel buffers
// (kPanel rows of panel_ld(n) each, 16-byte aligned).
__host__ __device__ inline int panel_ld(int n) { return (n + 7) & ~3; }
__host__ __device__ inline int panel_off(int n) { return (n * (n + 1) / 2 + n + 3) & ~3; }

constexpr int kMaxRefineLarge = 10;

__host__ __device__ inline size_t solve_large_smem_bytes(int nf) {
    const size_t n = 6 * (size_t)nf, np = n * (n + 1) / 2;
    const size_t f32 = ((size_t)panel_off((int)n) + 2 * kPanel * (size_t)panel_ld((int)n)) * 4, f64 = np * 8;
    return (f32 > f64 ? f32 : f64) + 2 * n * 8 + 64;
}

__global__ void __launch_bounds__(kSolveThreads) solve_large_kernel(const Prob *__restrict__ probs, int t,
                                                                    double *S_out, double *v_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Prob &pr = probs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31;
    if (t >= pr.iters) return;
    const int N = pr.N, t0 = pr.t0, nf = pr.nf, n = 6 * nf, np = n * (n + 1) / 2;
    const float *pose_cur = pr.pose_it + (size_t)t * N * 7;
    float *pose_next = pr.pose_it + (size_t)(t + 1) * N * 7;
    double *dxi = pr.dxi + (size_t)t * nf * 6;
    __shared__ int s_flag, s_use64;
    __shared__ float s_rpf[6 * kMaxFree];
    __shared__ double s_rp[6 * kMaxFree];
    __shared__ double s_red[kSolveThreads / 32][2];
    __shared__ double s_dsc[6 * kMaxFree];              // equilibration diag(S)^-1/2
    if (tid == 0) s_flag = *pr.status;
    __syncthreads();
    if (s_flag != 0 || nf == 0) {
        if (S_out == nullptr) {
            for (int q = tid; q < N * 7; q += kSolveThreads) pose_next[q] = pose_cur[q];
            for (int q = tid; q < nf * 6; q += kSolveThreads) dxi[q] = 0.0;
        }
        return;
    }
    double *v = reinterpret_cast<double *>(smem);
    double *x = v + n;
    float *Sp = reinterpret_cast<float *>(x + n);      // FP32 packed copy
    float *bf = Sp + np;
    double *Sd = reinterpret_cast<double *>(x + n);    // FP64 packed (fallback), over the FP32 copy
    double *Sg = pr.sglob;

    // Block pair (a, b), a <= b, of each pair index, as a << 8 | b.
    __shared__ unsigned short s_pair[kMaxFree * (kMaxFree + 1) / 2];
    __shared__ __align__(16) float s_dR[kPanel * kDiagLd];   // factored diagonal block, by rows
    for (int a = tid; a < nf; a += kSolveThreads) {
        const int base = a * nf - a * (a - 1) / 2;
        for (int b = a; b < nf; ++b) s_pair[base + b - a] = (unsigned short)(a << 8 | b);
    }
    // FP64 sums of the partials, parts added in order.  First the diagonal,
    // for the equilibration Dg = diag(S)^-1/2.
    const int Lp = pr.L, nparts = pr.n_parts, nbs = 2 * n_block_pairs(nf);
    constexpr int kU = 4;                                  // parts with loads in flight together
    for (int i = tid; i < n; i += kSolveThreads) {
        const int a = i / 6, r = i - 6 * a, h = r / 3;
        const int q = 18 * (2 * (a * nf - a * (a - 1) / 2) + h) + 6 * (r - 3 * h) + r;
        double sii = 0.0;
        for (int p0 = 0; p0 < nparts; p0 += kU) {
            double xv[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) xv[u] = p0 + u < nparts ? pr.partial[(size_t)(p0 + u) * Lp + q] : 0.0;
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (p0 + u < nparts) sii += xv[u];
        }
        s_dsc[i] = sii > 0.0 ? 1.0 / sqrt(sii) : 1.0;
    }
    __syncthreads();
    // Then every entry, two at a time (a strip's entries (row, col), (row,
    // col + 1)): to the FP64 workspace copy and, equilibrated and rounded, to
    // the FP32 copy.
    {
        const double2 *P2 = reinterpret_cast<const double2 *>(pr.partial);
        const int L2 = Lp >> 1, nsp = 9 * nbs;
        constexpr int kQ = 4;
        auto put = [&](int i, int k, double val) {
            const int idx = packed_index(i, k);
            Sg[idx] = val;
            Sp[idx] = (float)(val * s_dsc[i] * s_dsc[k]);
        };
        for (int q0 = tid; q0 < L2; q0 += kQ * kSolveThreads) {
            double2 acc[kQ];
#pragma unroll
            for (int w = 0; w < kQ; ++w) acc[w] = make_double2(0.0, 0.0);
            for (int p0 = 0; p0 < nparts; p0 += kU) {
                double2 xv[kU][kQ];
#pragma unroll
                for (int u = 0; u < kU; ++u)
#pragma unroll
                    for (int w = 0; w < kQ; ++w) {
                        const int q = q0 + w * kSolveThreads;
                        xv[u][w] = p0 + u < nparts && q < L2 ? P2[(size_t)(p0 + u) * L2 + q] : make_double2(0.0, 0.0);
                    }
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (p0 + u < nparts)
#pragma unroll
                        for (int w = 0; w < kQ; ++w) {
                            acc[w].x += xv[u][w].x;
                            acc[w].y += xv[u][w].y;
                        }
            }
#pragma unroll
            for (int w = 0; w < kQ; ++w) {
                const int q = q0 + w * kSolveThreads;
                if (q >= L2) break;
                if (q < nsp) {
                    const int st = q / 9, e = 2 * (q - 9 * st);
                    const int pc = s_pair[st >> 1], a = pc >> 8, b = pc & 255;
                    const int row = 6 * a + 3 * (st & 1) + e / 6, col = 6 * b + e % 6;
                    if (a == b) {                          // diagonal block: its lower half only
                        if (col <= row) put(row, col, acc[w].x);
                        if (col + 1 <= row) put(row, col + 1, acc[w].y);
                    } else {                               // a < b: the mirror entries (col, row)
                        put(col, row, acc[w].x);
                        put(col + 1, row, acc[w].y);
                    }
                } else {
                    v[2 * (q - nsp)] = acc[w].x;
                    v[2 * (q - nsp) + 1] = acc[w].y;
                }
            }
        }
    }
    __syncthreads();
    if (S_out != nullptr) {
        for (int q = tid; q < n * n; q += kSolveThreads) {
            const int i = q / n, k = q - i * n;
            S_out[q] = Sg[k <= i ? packed_index(i, k) : packed_index(k, i)];
        }
        for (int q = tid; q < n; q += kSolveThreads) v_out[q] = v[q];
        return;
    }

    // FP32 factorisation Dg S Dg = U D^-1 U^T by panels of kPanel columns.
    // Per panel: (1) one warp factors the diagonal block (lane = row, the
    // eliminated column values by shuffle); (2) a thread per row below it
    // eliminates the panel's columns from its row, and records the eliminated
    // values a_ij and the multipliers a_ij / p_j; (3) the trailing triangle
    // takes the panel's rank-kPanel update, A_ik -= sum_j (a_ij / p_j) a_kj,
    // in 4 x 4 register tiles.
    const int ld = panel_ld(n);
    float *PuT = Sp + panel_off(n);                        // a_ij at [j * ld + i]
    float *PwT = PuT + kPanel * ld;                        // a_ij / p_j at [j * ld + i]
    const int ty = tid >> 4, tx = tid & 15;
    if (tid == 0) s_use64 = pr.solve_f64 || pr.store_factor;   // the adjoint keeps the FP64 factor
    for (int q = tid; q < n; q += kSolveThreads) {
        x[q] = 0.0;
        bf[q] = (float)(s_dsc[q] * v[q]);
    }
    for (int q = tid; q < kPanel * (ld - n); q += kSolveThreads) {   // tile columns past n read zeros
        const int j = q / (ld - n), c = n + q - j * (ld - n);
        PuT[j * ld + c] = 0.f;
        PwT[j * ld + c] = 0.f;
    }
    __syncthreads();
    for (int J = 0; J < n && !s_use64; J += kPanel) {
        const int nb = min(kPanel, n - J), Rb = J + nb, m = n - Rb;
        if (tid < 32) {                                    // (1)
            const int ri = packed_index(J + lane, J);
            float xr[kPanel];
#pragma unroll
            for (int c = 0; c < kPanel; ++c) xr[c] = lane < nb && c <= lane ? Sp[ri + c] : 0.f;
            bool bad = false;
#pragma unroll
            for (int j = 0; j < kPanel; ++j) {
                if (j < nb) {
                    const float pj = __shfl_sync(0xffffffffu, xr[j], j);
                    const float ip = pj > 0.f ? 1.0f / pj : -1.f;
                    bad |= !(ip > 0.f) || !isfinite(ip);
                    if (lane == 0) s_rpf[J + j] = ip;
                    // rows below the pivot only; the entries right of a row's
                    // diagonal (c > lane) take harmless updates and are never read
                    const float l = lane > j ? xr[j] * ip : 0.f;
#pragma unroll
                    for (int c = j + 1; c < kPanel; ++c) xr[c] = fmaf(-l, __shfl_sync(0xffffffffu, xr[j], c), xr[c]);
                }
            }
            if (lane < nb) {
#pragma unroll
                for (int c = 0; c < kPanel; ++c)
                    if (c <= lane) {
                        Sp[ri + c] = xr[c];
                        s_dR[lane * kDiagLd + c] = xr[c];
                    }
            }
            if (bad && lane == 0) s_use64 = 1;
        }
        __syncthreads();
        if (s_use64) break;
        if (m == 0) break;                                 // the last panel
        for (int i = Rb + tid; i < n; i += kSolveThreads) {   // (2); nb == kPanel here
            const int ri = packed_index(i, J);
            float l[kPanel];
#pragma unroll
            for (int c = 0; c < kPanel; ++c) {             // a_ic = A_ic - sum_j<c l_j a_cj, l_c = a_ic / p_c
                float a0 = Sp[ri + c], a1 = 0.f;
#pragma unroll
                for (int g = 0; g < (c + 3) / 4; ++g) {
                    const float4 d = *reinterpret_cast<const float4 *>(s_dR + c * kDiagLd + 4 * g);
                    if (4 * g + 0 < c) a0 = fmaf(-l[4 * g + 0], d.x, a0);
                    if (4 * g + 1 < c) a1 = fmaf(-l[4 * g + 1], d.y, a1);
                    if (4 * g + 2 < c) a0 = fmaf(-l[4 * g + 2], d.z, a0);
                    if (4 * g + 3 < c) a1 = fmaf(-l[4 * g + 3], d.w, a1);
                }
                const float a = a0 + a1;
                l[c] = a * s_rpf[J + c];
                Sp[ri + c] = a;
                PuT[c * ld + i] = a;
                PwT[c * ld + i] = l[c];
                asm volatile("" ::: "memory");             // keeps the s_dR loads per column (no spills)
            }
        }
        __syncthreads();
        const int mt = (m + 3) >> 2, ntile = mt * (mt + 1) / 2;
        for (int q = tid; q < ntile; q += kSolveThreads) {  // (3)
            int ti = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
            while (ti * (ti + 1) / 2 > q) --ti;
            while ((ti + 1) * (ti + 2) / 2 <= q) ++ti;
            const int tk = q - ti * (ti + 1) / 2;
            const int i0 = Rb + 4 * ti, k0 = Rb + 4 * tk;
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 8
            for (int j = 0; j < kPanel; ++j) {
                const float4 w = *reinterpret_cast<const float4 *>(PwT + j * ld + i0);
                const float4 u = *reinterpret_cast<const float4 *>(PuT + j * ld + k0);
                const float wv[4] = {w.x, w.y, w.z, w.w}, uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(wv[a], uv[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int i = i0 + a;
                if (i >= n) break;
                const int ri = packed_index(i, 0);
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (k0 + b <= i) Sp[ri + k0 + b] -= acc[a][b];
            }
        }
        __syncthreads();
    }
    __syncthreads();
    // inverted diagonal blocks over the panel buffers (free now): ceil(n / kPanel)
    // x kPanel x kLinvLd floats, within 2 kPanel panel_ld(n) for n >= 26 and, for
    // smaller n, within the FP32 region the launch sizes for more than 15 free poses
    if (!s_use64) invert_diag_blocks(Sp, PackedIdx{}, s_rpf, PuT, n, tid);
    __syncthreads();
    double prev = 0.0;
    for (int it = 0; it <= kMaxRefineLarge && !s_use64; ++it) {
        if (it > 0) {   // residual v - S x in FP64 from the packed workspace copy
            const int qk = tid & 3;
            for (int base = 0; base < n; base += kSolveThreads / 4) {
                const int i = base + (tid >> 2);
                double acc = 0.0;
                if (i < n) {
#pragma unroll 4
                    for (int k = qk; k < n; k += 4)
                        acc = fma(Sg[k <= i ? packed_index(i, k) : packed_index(k, i)], x[k], acc);
                }
                acc += shfl_double(acc, lane ^ 1);
                acc += shfl_double(acc, lane ^ 2);
                if (i < n && qk == 0) bf[i] = (float)(s_dsc[i] * (v[i] - acc));
            }
            __syncthreads();
        }
        solve_blocked_f32(Sp, PackedIdx{}, s_rpf, PuT, bf, n, tid);
        double dmax = 0.0, xmax = 0.0;
        for (int q = tid; q < n; q += kSolveThreads) {
            const double d = s_dsc[q] * (double)bf[q];
            const double xn = x[q] + d;
            x[q] = xn;
            dmax = fmax(dmax, fabs(d));
            xmax = fmax(xmax, fabs(xn));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dmax = fmax(dmax, shfl_double(dmax, lane ^ o));
            xmax = fmax(xmax, shfl_double(xmax, lane ^ o));
        }
        if (lane == 0) { s_red[tid >> 5][0] = dmax; s_red[tid >> 5][1] = xmax; }
        __syncthreads();
        dmax = 0.0; xmax = 0.0;
#pragma unroll
        for (int w = 0; w < kSolveThreads / 32; ++w) {
            dmax = fmax(dmax, s_red[w][0]);
            xmax = fmax(xmax, s_red[w][1]);
        }
        const bool done = it > 0 && dmax <= kRefineTol * xmax;
        const bool fail = !(dmax <= 1e300) || (!done && (it == kMaxRefineLarge || (it > 1 && !(dmax <= 0.5 * prev))));
        if (fail && tid == 0) s_use64 = 1;
        __syncthreads();
        if (done || fail) break;
        prev = dmax;
    }
    __syncthreads();
    if (!s_use64) {
        for (int q = tid; q < n; q += kSolveThreads) v[q] = x[q];
    } else {
        // FP64 elimination with the right-hand side eliminated alongside
        for (int q = tid; q < np; q += kSolveThreads) Sd[q] = Sg[q];
        if (tid == 0) {
            const double p0 = Sg[0];
            s_rp[0] = p0 > 0.0 ? 1.0 / p0 : -1.0;
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const double ip = s_rp[j];
            if (!(ip > 0.0)) {
                if (tid == 0) s_flag = DPVO_BA_STATUS_NOT_SPD;
                break;
            }
            const int jn = j + 1;
            if (tid == 0 && jn < n) {
                const double c = Sd[packed_index(jn, j)];
                const double pn = Sd[packed_index(jn, jn)] - (c * ip) * c;
                Sd[packed_index(jn, jn)] = pn;
                s_rp[jn] = pn > 0.0 ? 1.0 / pn : -1.0;
            }
            for (int i = jn + ty; i < n; i += 16) {
                const int ri = packed_index(i, 0);
                const double lij = Sd[ri + j] * ip;
                for (int k = jn + tx; k <= i; k += 16) {
                    if (k == jn && i == jn) continue;
                    Sd[ri + k] -= lij * Sd[packed_index(k, j)];
                }
            }
            if (tid < n - jn) {
                const int i = jn + tid;
                v[i] -= (Sd[packed_index(i, j)] * ip) * v[j];
            }
            __syncthreads();
        }
        __syncthreads();
        if (!s_flag && pr.store_factor) {                   // U for the adjoint solve (packed lower)
            double *u = pr.ufac + (size_t)t * np;
            for (int q = tid; q < np; q += kSolveThreads) u[q] = Sd[q];
        }
        if (!s_flag && tid < 32) {                          // U^T x = v'
            for (int j = n - 1; j >= 0; --j) {
                const double xj = v[j] * s_rp[j];
                for (int i = lane; i < j; i += 32) v[i] -= Sd[packed_index(j, i)] * xj;
                __syncwarp();
                if (lane == 0) v[j] = xj;
                __syncwarp();
            }
        }
    }
    __syncthreads();
    if (!s_flag && tid < 32) {
        bool bad = false;
        for (int q = lane; q < n; q += 32) bad |= !isfinite(v[q]);
        if (__any_sync(0xffffffffu, bad) && lane == 0) s_flag = DPVO_BA_STATUS_NONFINITE;
    }
    __syncthreads();
    if (s_flag) {
        if (tid == 0) *pr.status = s_flag;
        for (int q = tid; q < N * 7; q += kSolveThreads) pose_next[q] = pose_cur[q];
        for (int q = tid; q < nf * 6; q += kSolveThreads) dxi[q] = 0.0;
        return;
    }
    for (int q = tid; q < n; q += kSolveThreads) dxi[q] = v[q];
    for (int a = tid; a < N; a += kSolveThreads) {
        if (a >= t0) se3_left_update(v + 6 * (a - t0), pose_cur + 7 * a, pose_next + 7 * a);
        else
            for (int q = 0; q < 7; ++q) pose_next[7 * a + q] = pose_cur[7 * a + q];
    }
}

}  // namespace dpvo
