// Bundle-adjustment kernels (Deep Patch Visual Odometry, Sec. 3.1 Eq. 6).
//
//   plan_kernel       once per solve: validates indices and ordering, builds the
//                     patch -> edge offsets and the chunk table in one pass
//                     over the anchors and one over the edges, copies the
//                     initial state into iterate 0.
//   linearize_kernel  once per iteration (and once more at the end): for each
//                     chunk of patches that share a source frame,
//                       (a) back-substitutes the previous iteration's inverse-
//                           depth increments dd_k = (w_k - e_k^T dxi) / C_k
//                           from the patch's stored scaled Schur row,
//                       (b) linearises every edge at the new state (Eq. 2-3
//                           reprojection, residual, pose-j / inverse-depth
//                           Jacobians) and reduces the pose-pair blocks
//                           B_jj += J_j^T W J_j by frame,
//                       (c) accumulates the Schur complement
//                           S = B - sum_k E_k C_k^-1 E_k^T, v' = v - sum_k E_k C_k^-1 w_k
//                           over the free poses, with compensated sums, and
//                           stores each patch's row C_k^-1/2 (e_k, w_k, 1),
//                     and writes one FP64 partial of (S, v') per CTA.  The
//                     last launch only back-substitutes, per patch.
//   solve_kernel      once per iteration: sums the partials in FP64, factorises
//                     S = L L^T in FP64 (pivot check -> NOT_SPD), solves for the
//                     pose increments and retracts T <- Exp(dxi) T.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "ba_common.cuh"
#include "se3.cuh"
#include "tc.cuh"

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

// ----------------------------------------------------------------------------
// plan_kernel: grid (problems, edge slices), kPlanThreads per CTA.  Every CTA
// checks one slice of a problem's edges (valid indices, sorted by patch and
// then frame) and, at every change of patch, records where that patch's edges
// begin; the last CTA of the problem to finish (a ticket in its descriptor)
// then makes one pass over the anchors (where each frame's patches begin),
// copies the initial state into iterate 0, builds the chunk table and writes
// the status.  Coalesced passes, no searches.
// ----------------------------------------------------------------------------
constexpr int kPlanThreads = 1024;
constexpr int kPlanUnroll = 4;       // patches per thread with loads in flight together
constexpr int kPlanSliceEdges = 4 * kPlanThreads;   // edges of one slice at least (one load round)

__global__ void __launch_bounds__(kPlanThreads, 2) plan_kernel(const Prob *__restrict__ probs, int slices) {
    const Prob &pr = probs[blockIdx.x];
    Prob *mp = const_cast<Prob *>(probs) + blockIdx.x;   // the ticket and the bad flag
    const int tid = threadIdx.x, slice = blockIdx.y;
    const int N = pr.N, P = pr.P, E = pr.E;
    __shared__ int s_bad, s_last;
    __shared__ int s_fstart[DPVO_BA_MAX_FRAMES + 1];
    __shared__ int s_choff[DPVO_BA_MAX_FRAMES + 1];
    if (tid == 0) s_bad = 0;
    if (E == 0 && slice == 0)
        for (int k = tid; k <= P; k += kPlanThreads) pr.seg[k] = 0;
    __syncthreads();

    // Where kk and jj share their 16-byte phase the edges are read in groups
    // of four by 16-byte loads: a scalar head up to the 16-byte boundary and a
    // scalar tail (slice 0), and this slice's range of quads.
    const uintptr_t ka = (uintptr_t)pr.kk, ja = (uintptr_t)pr.jj;
    const bool vec = (ka & 3) == 0 && (ka & 15) == (ja & 15);
    const int head = vec ? min(E, (int)(((16 - (ka & 15)) & 15) >> 2)) : 0;
    const int Q = vec ? (E - head) >> 2 : 0;
    const int qs = (Q + slices - 1) / slices, q_lo = min(Q, slice * qs), q_hi = min(Q, q_lo + qs);
    const int4 *kk4 = reinterpret_cast<const int4 *>(pr.kk + head);
    const int4 *jj4 = reinterpret_cast<const int4 *>(pr.jj + head);
    int bad = 0;
    // edge e = (k, j) after (kp, jp): valid and ordered, and patches (kp, k] start at e
    auto edge = [&](int e, int k, int j, int kp, int jp) {
        if (k < 0 || k >= P || j < 0 || j >= N || kp > k || (kp == k && jp >= j)) {
            bad = 1;
            return;
        }
        for (int q = max(kp + 1, 0); q <= k; ++q) pr.seg[q] = e;
        if (e == E - 1)
            for (int q = k + 1; q <= P; ++q) pr.seg[q] = E;
    };
    auto edge_scalar = [&](int e) {   // one edge with its own loads
        edge(e, pr.kk[e], pr.jj[e], e > 0 ? pr.kk[e - 1] : -1, e > 0 ? pr.jj[e - 1] : -1);
    };
    const int lane = tid & 31, warp = tid >> 5;
    if (vec) {
        const int tail0 = head + 4 * Q;
        if (slice == 0) {
            if (tid < head) edge_scalar(tid);
            else if (tid >= 32 && tid - 32 < E - tail0) edge_scalar(tail0 + tid - 32);
        }
        // four edges per thread per step; the previous edge of a quad is the
        // neighbouring lane's last (a warp's first lane loads its own)
        for (int q = q_lo + tid; q - tid < q_hi; q += kPlanThreads) {
            int4 kv = make_int4(0, 0, 0, 0), jv = kv;
            int kq = -1, jq = -1;
            if (q < q_hi) {
                kv = kk4[q];
                jv = jj4[q];
                if (lane == 0 && head + 4 * q > 0) {
                    kq = pr.kk[head + 4 * q - 1];
                    jq = pr.jj[head + 4 * q - 1];
                }
            }
            const int ks = __shfl_up_sync(0xffffffffu, kv.w, 1);
            const int js = __shfl_up_sync(0xffffffffu, jv.w, 1);
            if (lane > 0) { kq = ks; jq = js; }
            if (q >= q_hi) continue;
            const int e = head + 4 * q;
            edge(e, kv.x, jv.x, kq, jq);
            edge(e + 1, kv.y, jv.y, kv.x, jv.x);
            edge(e + 2, kv.z, jv.z, kv.y, jv.y);
            edge(e + 3, kv.w, jv.w, kv.z, jv.z);
        }
    } else {
        const int es = (E + slices - 1) / slices, e_lo = min(E, slice * es), e_hi = min(E, e_lo + es);
        for (int e = e_lo + tid; e < e_hi; e += kPlanThreads) edge_scalar(e);
    }
    if (slices > 1) {                    // hand over to the last CTA of the problem
        if (bad) atomicOr(&mp->plan_bad, 1);
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = atomicAdd(&mp->plan_ticket, 1) == slices - 1;
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        bad = tid == 0 ? atomicOr(&mp->plan_bad, 0) : 0;
    }

    // the anchors (where each frame's patches begin) and the initial state
    if (P == 0)
        for (int i = tid; i <= N; i += kPlanThreads) s_fstart[i] = 0;
    for (int i = tid; i < N * 7; i += kPlanThreads) {
        const float v = pr.poses[i];
        pr.pose_it[i] = v;
        if (!isfinite(v)) bad = 1;
    }
    for (int base = 0; base < P; base += kPlanUnroll * kPlanThreads) {
        int av[kPlanUnroll], ap[kPlanUnroll];
        float dv[kPlanUnroll];
#pragma unroll
        for (int u = 0; u < kPlanUnroll; ++u) {   // loads of all unrolled patches first
            const int k = base + u * kPlanThreads + tid;
            av[u] = 0; ap[u] = -1; dv[u] = 0.f;
            if (k < P) {
                av[u] = pr.anchor[k];
                if (k > 0) ap[u] = pr.anchor[k - 1];
                dv[u] = pr.patches[3 * k + 2];
            }
        }
#pragma unroll
        for (int u = 0; u < kPlanUnroll; ++u) {
            const int k = base + u * kPlanThreads + tid;
            if (k >= P) continue;
            pr.depth_it[k] = dv[u];
            const int a = av[u];
            if (a < 0 || a >= N || ap[u] > a) {
                bad = 1;
            } else {
                for (int i = max(ap[u] + 1, 0); i <= a; ++i) s_fstart[i] = k;     // frames (ap, a] start at k
                if (k == P - 1)
                    for (int i = a + 1; i <= N; ++i) s_fstart[i] = P;
            }
        }
    }
    if (bad) atomicOr(&s_bad, 1);
    __syncthreads();
    if (s_bad) {
        if (tid == 0) { *pr.status = DPVO_BA_STATUS_BAD_INPUT; *pr.n_chunks = 0; }
        return;
    }
    if (warp == 0) {   // first chunk of each frame: exclusive scan of the frames' chunk counts
        int carry = 0;
        for (int i0 = 0; i0 < N; i0 += 32) {
            const int i = i0 + lane;
            const int cnt = i < N ? s_fstart[i + 1] - s_fstart[i] : 0;
            const int nc = (cnt + pr.chunk_cap - 1) / pr.chunk_cap;
            int incl = nc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (i < N) s_choff[i] = carry + incl - nc;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            s_choff[N] = carry;
            if (carry > pr.max_chunks) s_bad = 1;
        }
    }
    __syncthreads();
    for (int i = tid; i < N && !s_bad; i += kPlanThreads) {
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
            ch.e0 = __ldcg(pr.seg + k);
            ch.e1 = __ldcg(pr.seg + k + sz);
            ch.anchor = i;
            ch.jlo = i;          // window filled in below, one warp per chunk
            ch.jhi = i;
            ch.pad = 0;
            pr.chunks[s_choff[i] + c] = ch;
            k += sz;
        }
    }
    __syncthreads();
    // frame window [jlo, jhi] of each chunk: edges of a patch are sorted by
    // frame, so its first and last edges bound it
    const int n_built = s_bad ? 0 : s_choff[N];    // 0 if the chunk table overflowed
    for (int c = warp; c < n_built; c += kPlanThreads / 32) {
        const Chunk ch = pr.chunks[c];
        int jlo = ch.anchor, jhi = ch.anchor;
        for (int q = ch.k0 + lane; q < ch.k0 + ch.count; q += 32) {
            const int s0 = __ldcg(pr.seg + q), s1 = __ldcg(pr.seg + q + 1);
            if (s1 > s0) {
                jlo = min(jlo, (int)pr.jj[s0]);
                jhi = max(jhi, (int)pr.jj[s1 - 1]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            jlo = min(jlo, __shfl_xor_sync(0xffffffffu, jlo, o));
            jhi = max(jhi, __shfl_xor_sync(0xffffffffu, jhi, o));
        }
        if (lane == 0) {
            pr.chunks[c].jlo = jlo;
            pr.chunks[c].jhi = jhi;
            if (jhi - jlo + 1 > pr.win_cap) atomicOr(&s_bad, 1);
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_bad) { *pr.status = DPVO_BA_STATUS_BAD_INPUT; *pr.n_chunks = 0; }
        else { *pr.status = 0; *pr.n_chunks = s_choff[N]; }
    }
}

// ----------------------------------------------------------------------------
// linearize_kernel shared memory.  Sizes depend on the batch's frame-window
// cap W, chunk cap G and largest free-pose count.
// ----------------------------------------------------------------------------
struct LinSmem {
    int W, G, Gs, Gs1, ES, EC;  // window cap, chunk cap, slot strides (float4 / float arrays), E-row stride, edge capacity
    uint32_t sbo;          // tensor-core operand: bytes between 8-row groups
    size_t off_pose, off_rjj, off_rtg, off_rwt, off_rpx, off_rpy, off_rdep, off_rseg, off_idx, off_sc4, off_sc1,
        off_ec, off_op, off_mp, off_reln, off_adj, off_mc, off_aj, off_bp, off_bii, off_pd, off_ps, off_dx;
    size_t bytes;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Free poses up to which the Schur accumulation runs on the tensor cores:
// 6 nf + 2 rows (pose columns, then C^-1/2 w split in two) fit one 64-row operand.
constexpr int kTcMaxFree = 10;
constexpr int kTcRows = 64;                    // rows of each half (lo, hi) of the operand
constexpr int kTcXStride = 65;                 // row stride (floats) of the accumulator read-back
__host__ __device__ inline bool use_tensor_cores(int nf_max) { return nf_max <= kTcMaxFree; }

// tc: tensor-core variant.  It keeps no E_k rows (Ec); instead a K-major TF32
// operand of 2 x 64 rows (lo half, hi half) by G patches, and reads the TMEM
// accumulator back through a 128 x 65 float buffer that overlays the staging
// buffers, dead by then.
__host__ __device__ inline LinSmem lin_smem_layout(int W, int G, int nf_max, int n_max, bool tc) {
    LinSmem s;
    s.W = W;
    s.G = G;
    // slot (frame jl, patch p) at jl * Gs + p.  The per-patch sums read
    // frames sub, sub + 4, ... of 8 consecutive patches by 4 lanes each: with
    // Gs = 2 (mod 8) the 16-byte reads of a quarter warp, and with Gs1 = 8
    // (mod 16) the 4-byte reads of a warp, fall in distinct banks.
    s.Gs = G + ((2 - G) % 8 + 8) % 8;
    s.Gs1 = G + ((8 - G) % 16 + 16) % 16;
    // E_k row: frame f at floats 8f..8f+7 laid out [v0 v1 v2 _ v3 v4 v5 _],
    // then C_k^-1/2 w_k; the stride is an odd multiple of 4 floats
    const int es = 8 * nf_max + 4;
    s.ES = es;
    s.EC = W * G;
    const int kmax = (G + 7) & ~7;
    s.sbo = (uint32_t)(kmax / 4) * 144u;
    const size_t slots = (size_t)W * s.Gs, slots1 = (size_t)W * s.Gs1;
    // the per-slot sums share their buffer with the staged Schur rows of the
    // next chunk (read before the slots are written)
    const size_t rows = tc ? (size_t)kTcRows * kmax * 4 : (size_t)G * erow_smem_stride(nf_max) * 4;
    const size_t sc4 = slots * 16 > rows ? slots * 16 : rows;
    size_t o = 0;
    s.off_pose = o; o = align16(o + (size_t)n_max * 7 * 4);
    // edge staging, with room for the alignment slack of bulk copies
    s.off_rjj = o;  o = align16(o + (size_t)(s.EC + 8) * 4);
    s.off_rtg = o;  o = align16(o + (size_t)(s.EC + 2) * 8);
    s.off_rwt = o;  o = align16(o + (size_t)(s.EC + 2) * 8);
    s.off_rpx = o;  o = align16(o + (size_t)G * 4);
    s.off_rpy = o;  o = align16(o + (size_t)G * 4);
    s.off_rdep = o; o = align16(o + (size_t)G * 4);
    s.off_rseg = o; o = align16(o + (size_t)(G + 1) * 4);
    s.off_idx = o;  o = align16(o + slots * 2);
    s.off_sc4 = o;  o = align16(o + sc4);
    s.off_sc1 = o;  o = align16(o + slots1 * 4);
    if (tc) {
        s.off_ec = 0;
        s.off_op = o; o = align16(o + (size_t)2 * (kTcRows / 8) * s.sbo);
        const size_t xend = s.off_rjj + (size_t)2 * kTcRows * kTcXStride * 4;
        if (o < xend) o = align16(xend);
    } else {
        s.off_op = 0;
        s.off_ec = o; o = align16(o + (size_t)G * es * 4);
    }
    // the anchor-pair products (A_j, B_j) overlay the per-thread frame sums,
    // which are consumed before them
    s.off_mp = o;   o = align16(o + (size_t)kThreads * 27 * 4);
    s.off_aj = s.off_mp;
    s.off_bp = s.off_mp + align16((size_t)W * 42 * 4);
    s.off_reln = o; o = align16(o + (size_t)W * 12 * 4);
    s.off_adj = o;  o = align16(o + (size_t)W * 36 * 4);
    s.off_mc = o;   o = align16(o + (size_t)W * 27 * 4);
    s.off_bii = o;  o = align16(o + 42 * 4);
    s.off_pd = o;   o = align16(o + (size_t)G * 16);
    s.off_ps = o;   o = align16(o + (size_t)2 * G * 4);
    s.off_dx = o;   o = align16(o + (size_t)erow_len(kMaxFree) * 4);
    s.bytes = o;
    return s;
}

// Tensor-core variant: the stored Schur rows of chunk c form one block of
// kTcRows x Kmax floats (Kmax = chunk cap rounded up to 8) at c * kTcRows *
// Kmax, element (row r, patch p of the chunk) at (p / 4) * 256 + 4 r + p % 4:
// rows 0..6nf-1 hold C_k^-1/2 e_k, row 62 C_k^-1/2 w_k, row 63 C_k^-1/2, the
// rest zero.  The 8 x 4 (row, patch) tiles of the MMA operand map to 128
// contiguous bytes of it.
__host__ __device__ inline int tc_kmax(int G) { return (G + 7) & ~7; }
__host__ __device__ inline int tc_blk(int r, int p) { return (p >> 2) * (4 * kTcRows) + 4 * r + (p & 3); }

// Back-substitution dot products of one 4-patch group of a stored block
// (tensor-core variant): the 8 lanes rs = 0..7 of an aligned octet take rows
// rs, rs + 8, ... (< n6), each row one float4 of the 4 patches; the octet sum
// lands in every lane.  Returns the 4 dot products with dx (zero beyond n6).
__device__ __forceinline__ float4 group_dots(const float *grp, const float *dx, int n6, int rs) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r = rs; r < n6; r += 8) {
        const float4 v = *reinterpret_cast<const float4 *>(grp + 4 * r);
        const float x = dx[r];
        acc.x = fmaf(v.x, x, acc.x);
        acc.y = fmaf(v.y, x, acc.y);
        acc.z = fmaf(v.z, x, acc.z);
        acc.w = fmaf(v.w, x, acc.w);
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    }
    return acc;
}

// Compensated (Kahan) update of a running sum (s, c) with the block sum blk.
__device__ __forceinline__ void kahan_add(float &s, float &c, float blk) {
    const float y = blk - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Asynchronous global -> shared copies (completed by cp_async_wait_all + a barrier).
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// TMEM columns of the strip running sums per linearise CTA (FP32 fused
// variant): two warps per lane quarter, 36 columns each, rounded up to a
// power of two.  Two CTAs per SM take 256 of the 512.
constexpr uint32_t kSumsTmemCols = 128;

// Role rotation of the in-loop prefetch: its first roles (the bulk copies,
// the descriptor, the patch arrays) go to the last two warps, which hold no
// patch of the per-patch phase that follows for chunks of up to 48 patches.
constexpr int kPrefetchRot = 64;

// Start copying one chunk's inputs -- frames, targets and weights of its
// edges, its patches' centres and inverse depths, its patch -> edge offsets --
// into the staging buffers.  With an mbarrier (bar != 0) and 16-byte aligned
// edge arrays, the three edge ranges go by bulk asynchronous copies from one
// thread, each widened to 16-byte boundaries (but not past the array's last
// whole 16 bytes; the elements beyond go by per-thread copies) and completing
// on bar; the staged range then starts staged_offset() elements before e0.
// Otherwise every element goes by a per-thread copy at offset 0 (and bar, if
// given, gets a plain arrival so that it completes one phase per chunk).
__device__ __forceinline__ void staged_offsets(const Prob &pr, const Chunk &ch, bool bulk_path, int &o_jj,
                                               int &o_tw) {
    const bool bulk = bulk_path && pr.bulk_edges && ch.e1 > ch.e0;
    o_jj = bulk ? (ch.e0 & 3) : 0;
    o_tw = bulk ? (ch.e0 & 1) : 0;
}

__device__ __forceinline__ void prefetch_chunk(const Prob &pr, const Chunk &ch, const float *depth_src, int *rjj,
                                               float2 *rtg, float2 *rwt, float *rpx, float *rpy, float *rdep,
                                               int *rseg, const Chunk *desc_src, Chunk *desc_dst,
                                               uint32_t bar = 0, int rot = 0) {
    // vt: the thread's role, rotated by rot so that the single-thread and
    // low-index roles can fall on other warps than the first
    const int vt = ((int)threadIdx.x + rot) & (kThreads - 1);
    if (desc_src && vt < 8)   // the descriptor of the chunk after this one
        cp_async4(reinterpret_cast<int *>(desc_dst) + vt, reinterpret_cast<const int *>(desc_src) + vt);
    const float2 *tg = reinterpret_cast<const float2 *>(pr.target);
    const float2 *wt = reinterpret_cast<const float2 *>(pr.weight);
    const int e0 = ch.e0, e1 = ch.e1;
    if (bar != 0 && pr.bulk_edges && e1 > e0) {
        const int a0 = e0 & ~3, a1 = min((e1 + 3) & ~3, pr.E & ~3);   // jj: 4 per 16 bytes
        const int b0 = e0 & ~1, b1 = min((e1 + 1) & ~1, pr.E & ~1);   // target, weight: 2 per 16 bytes
        if (vt == 0) {
            const uint32_t bj = a1 > a0 ? (uint32_t)(a1 - a0) * 4u : 0u;
            const uint32_t bt = b1 > b0 ? (uint32_t)(b1 - b0) * 8u : 0u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bj + 2u * bt)
                         : "memory");
            if (bj) bulk_copy_g2s(rjj, pr.jj + a0, bj, bar);
            if (bt) {
                bulk_copy_g2s(rtg, tg + b0, bt, bar);
                bulk_copy_g2s(rwt, wt + b0, bt, bar);
            }
        }
        for (int e = max(e0, a1 > a0 ? a1 : e0) + vt; e < e1; e += kThreads)
            cp_async4(rjj + (e - a0), pr.jj + e);
        for (int e = max(e0, b1 > b0 ? b1 : e0) + vt; e < e1; e += kThreads) {
            cp_async8(rtg + (e - b0), tg + e);
            cp_async8(rwt + (e - b0), wt + e);
        }
    } else {
        if (bar != 0 && vt == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
        for (int q = vt; q < e1 - e0; q += kThreads) {
            const int e = e0 + q;
            cp_async4(rjj + q, pr.jj + e);
            cp_async8(rtg + q, tg + e);
            cp_async8(rwt + q, wt + e);
        }
    }
    for (int q = vt; q < ch.count; q += kThreads) {
        const int k = ch.k0 + q;
        cp_async4(rpx + q, pr.patches + 3 * k);
        cp_async4(rpy + q, pr.patches + 3 * k + 1);
        cp_async4(rdep + q, depth_src + k);
    }
    for (int q = vt; q <= ch.count; q += kThreads) cp_async4(rseg + q, pr.seg + ch.k0 + q);
    cp_async_commit();
}

// One thread: start one bulk copy of a chunk's stored Schur rows (rs floats
// each, contiguous) into shared memory, completing on the mbarrier.
__device__ __forceinline__ void prefetch_rows_bulk(const Prob &pr, const Chunk &ch, int rs, float *dst, uint32_t bar) {
    const uint32_t bytes = (uint32_t)(ch.count * rs * 4);
    fence_async_smem();                            // the buffer's earlier shared-memory reads come first
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
    if (bytes) bulk_copy_g2s(dst, pr.erow + (size_t)ch.k0 * rs, bytes, bar);
}

// Start copying chunk c's block of stored rows (its first ceil8(count) patches) to dst.
__device__ __forceinline__ void prefetch_block(const Prob &pr, int c, const Chunk &ch, int kmax, float *dst) {
    const int n16 = ((ch.count + 7) & ~7) * kTcRows / 4;
    const float4 *src = reinterpret_cast<const float4 *>(pr.erow + (size_t)c * kTcRows * kmax);
    for (int q = threadIdx.x; q < n16; q += kThreads) cp_async16(dst + 4 * q, src + q);
    cp_async_commit();
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float s) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
}

// Relative poses of the window frames w.r.t. the anchor (and their adjoints),
// by threads tid0 .. kThreads - 1.
__device__ __forceinline__ void window_poses(const float *poses, int anchor, int jlo, int W, float *rel,
                                             float *adj, int tid0 = 0) {
    for (int jl = (int)threadIdx.x - tid0; jl < W; jl += kThreads - tid0) {
        if (jl < 0) break;
        float *R = rel + jl * 12;
        relative_pose(poses + 7 * anchor, poses + 7 * (jlo + jl), R, R + 9);
        if (adj) adjoint6(R, R + 9, adj + jl * 36);
    }
}

// Sum over aligned groups of lp consecutive lanes (lp a power of two <= 32,
// the same in the whole warp; fixed order), broadcast to the group.
__device__ __forceinline__ float lane_group_sum(float v, int lp) {
    for (int o = 1; o < lp; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Lanes per patch for the per-patch phases of a chunk of cnt patches: 256 /
// (cnt rounded up to a power of two), at least 4, at most 32; log2 in *sh.
__device__ __forceinline__ int lanes_per_patch(int cnt, int *sh) {
    int p2 = 1;
    while (p2 < cnt) p2 <<= 1;
    int lp = kThreads / p2;
    lp = lp < 4 ? 4 : (lp > 32 ? 32 : lp);
    int l = 0;
    while ((1 << l) < lp) ++l;
    *sh = l;
    return lp;
}

// Sum of 4 consecutive lanes' values (fixed order), broadcast to all four.
__device__ __forceinline__ float quad_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// Last back-substitution of the depths (Eq. 6 with the final pose increment):
// dd_k = C_k^-1/2 (C_k^-1/2 w_k - (C_k^-1/2 e_k) . dxi), read from the stored
// Schur rows.  Row layout: patches [k_lo, k_hi), four lanes per patch, dxs the
// increment in the rows' padded frame layout.
constexpr int kBsLoads = 5;   // float4 loads of a stored row per lane in flight together

__device__ __forceinline__ void backsub_rows(const Prob &pr, const float *dxs, const float *depth_old,
                                             float *depth_new, int k_lo, int k_hi, int tid) {
    const int nf = pr.nf, RS = erow_len(nf);
    const float4 *dz4 = reinterpret_cast<const float4 *>(dxs);
    const int sub = tid & 3;
    for (int kb = k_lo; kb < k_hi; kb += kThreads / 4) {
        const int k = kb + (tid >> 2);
        float s = 0.f;
        const float *row = pr.erow + (size_t)k * RS;
        if (k < k_hi) {   // the lane's float4s q = sub + 4i, kBsLoads loads in flight at a time
            const float4 *row4 = reinterpret_cast<const float4 *>(row);
            for (int q0 = sub; q0 < RS / 4; q0 += 4 * kBsLoads) {
                float4 v[kBsLoads];
#pragma unroll
                for (int i = 0; i < kBsLoads; ++i)
                    v[i] = q0 + 4 * i < RS / 4 ? row4[q0 + 4 * i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int i = 0; i < kBsLoads; ++i)
                    if (q0 + 4 * i < RS / 4) s = dot4(v[i], dz4[q0 + 4 * i], s);
            }
        }
        s = quad_sum(s);
        if (k < k_hi && sub == 0) {
            const float dnew = depth_old[k] + row[8 * nf + 1] * (row[8 * nf] - s);
            depth_new[k] = dnew;
            if (!pr.no_writeback) pr.patches[3 * k + 2] = dnew;
        }
    }
}

// The same for chunk c in the tensor-core row layout (4-patch groups), one
// warp, one lane octet per group; dxs the increment zero-padded to kTcRows.
__device__ __forceinline__ void backsub_chunk_tc(const Prob &pr, int c, const float *dxs, const float *depth_old,
                                                 float *depth_new, int kmax, int lane) {
    const int n6 = 6 * pr.nf, rs = lane & 7, gw = lane >> 3;
    const Chunk ch = pr.chunks[c];
    const float *eb = pr.erow + (size_t)c * kTcRows * kmax;
    const int ng = (ch.count + 3) >> 2;
    for (int gb = 0; gb < ng; gb += 4) {      // warp-uniform trip count
        const int g = gb + gw;
        const float *grp = eb + (size_t)(g < ng ? g : 0) * (4 * kTcRows);
        const float4 dots = group_dots(grp, dxs, g < ng ? n6 : 0, rs);
        if (g < ng && rs < 4) {
            const int p = 4 * g + rs;
            if (p < ch.count) {
                const float dot = rs == 0 ? dots.x : rs == 1 ? dots.y : rs == 2 ? dots.z : dots.w;
                const int k = ch.k0 + p;
                const float dnew = depth_old[k] + grp[4 * (kTcRows - 1) + rs] * (grp[4 * (kTcRows - 2) + rs] - dot);
                depth_new[k] = dnew;
                if (!pr.no_writeback) pr.patches[3 * k + 2] = dnew;
            }
        }
    }
}

// Pose increment of iteration t - 1 as the back-substitution reads it: the
// tensor-core layout (zero-padded to kTcRows) or the rows' frame layout (frame
// f at 8f..8f+7 as [v 0 w 0], zero-padded to the row length).
template <bool TC>
__device__ __forceinline__ void stage_dxi(const Prob &pr, int t, float *dxs, int tid, int nthreads) {
    const int nf = pr.nf;
    const double *dx = pr.dxi + (size_t)(t - 1) * nf * 6;
    if constexpr (TC) {
        for (int q = tid; q < kTcRows; q += nthreads) dxs[q] = q < 6 * nf ? (float)dx[q] : 0.f;
    } else {
        const int RS = erow_len(nf);
        for (int q = tid; q < RS; q += nthreads) {
            const int f = q >> 3, m = q & 7;
            dxs[q] = (f < nf && (m & 3) != 3) ? (float)dx[6 * f + m - (m >> 2)] : 0.f;
        }
    }
}


// The pose-pair block entries a group of chunks adds to one strip of (S, v')
// (the same selection the fused path makes inline for its register strips):
// half-strip (a, b, sh) = rows 6a + 3sh .. +2, columns 6b .. 6b + 5 of the
// (free-pose) block (a, b), or the right-hand side of free pose a (vstrip).
// Blocks: B_jj = M_j for window frames, B_ii for the anchor, B_ij = -Ad^T M_j
// between anchor and frame.  Returns false if the group adds nothing there.
__device__ __forceinline__ bool strip_block_add(int sa, int sb, int sh, bool vstrip, int t0, int anc, int jlo, int W,
                                                const float *Mc, const float *Aj, const float *Bii, float *add) {
    const int fa = t0 + sa, fb = t0 + sb;
    const int ja = fa - jlo, jb = fb - jlo;
    const bool a_in = ja >= 0 && ja < W, b_in = jb >= 0 && jb < W;
    if (vstrip) {
        if (fa == anc) {
#pragma unroll
            for (int q = 0; q < 6; ++q) add[q] = Bii[36 + q];
        } else if (a_in) {
#pragma unroll
            for (int q = 0; q < 6; ++q) add[q] = Mc[ja * 27 + 21 + q];
        } else {
            return false;
        }
        return true;
    }
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
        } else {
            return false;
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
    } else {
        return false;
    }
    return true;
}

// ----------------------------------------------------------------------------
// linearize_kernel: one CTA per work item (a range of chunks of one problem).
// t = iteration.  For t < iters: back-substitute iteration t-1 (if t > 0), then
// linearise at iterate t and accumulate the Schur partial.  For t == iters:
// back-substitute the last iteration and write the caller's outputs.
// A chunk's inputs are copied into shared memory asynchronously while the
// previous chunk is still being reduced.  Consecutive chunks with the same
// anchor and frame window form a group that shares its window poses and its
// pose-pair blocks.
//
// TC (tensor-core variant, at most kTcMaxFree free poses): instead of FP32
// strips, sum_k E_k C_k^-1 E_k^T and sum_k E_k C_k^-1 w_k accumulate in TMEM
// through kind::tf32 MMAs with each operand value x split as hi = tf32(x),
// lo = tf32(x - hi) and the product taken as hi.hi + lo.hi + (lo.hi)^T (three
// TF32 terms, near-FP32 accuracy).  Per chunk, the operand holds lo (rows
// 0-63) and hi (rows 64-127) of C_k^-1/2 E_k^T by patch (K-major); rows 62 and
// 63 of the hi half carry hi and lo of C_k^-1/2 w_k.  One MMA per 8 patches
// with A = all 128 rows and B = the hi half gives D = [lo; hi] hi^T; the CTA
// reads D back once, after its last chunk.
// ----------------------------------------------------------------------------
template <bool TC, bool EXT>
__global__ void __launch_bounds__(kThreads, 2) linearize_kernel(const Prob *__restrict__ probs,
                                                             const Item *__restrict__ items, int t,
                                                             int W_cap, int G_cap, int nf_max, int n_max,
                                                             int adjoint_rhs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Item itm = items[blockIdx.x];
    const Prob &pr = probs[itm.prob];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (t > pr.iters) return;
    // adjoint_rhs: linearise at iterate t only and accumulate the pose part of
    // E C^-1 dbar (dbar = gradient w.r.t. the inverse depths) into the
    // right-hand-side strips, for the adjoint solve of iteration t
    const bool do_bs = t > 0 && !adjoint_rhs;
    const bool final_pass = t == pr.iters && !adjoint_rhs;
    {   // read once: every thread takes the same exit (the kernel has block barriers)
        __shared__ int s_st0;
        if (tid == 0) s_st0 = *pr.status;
        __syncthreads();
        const int st = s_st0;
        if (final_pass && itm.item == 0 && tid == 0 && pr.status_user) *pr.status_user = st;
        if (st != 0) return;
    }

    const LinSmem L = lin_smem_layout(W_cap, G_cap, nf_max, n_max, TC);
    float *spn = reinterpret_cast<float *>(smem + L.off_pose);        // poses of iterate t
    int *rjj_s = reinterpret_cast<int *>(smem + L.off_rjj);              // edge staging bases
    float2 *rtg_s = reinterpret_cast<float2 *>(smem + L.off_rtg);
    float2 *rwt_s = reinterpret_cast<float2 *>(smem + L.off_rwt);
    float *rpx = reinterpret_cast<float *>(smem + L.off_rpx);
    float *rpy = reinterpret_cast<float *>(smem + L.off_rpy);
    float *rdep = reinterpret_cast<float *>(smem + L.off_rdep);
    int *rseg = reinterpret_cast<int *>(smem + L.off_rseg);
    short *sidx = reinterpret_cast<short *>(smem + L.off_idx);
    float4 *sc4 = reinterpret_cast<float4 *>(smem + L.off_sc4);
    float *srow = reinterpret_cast<float *>(smem + L.off_sc4);        // staged Schur rows (aliases sc4)
    float *sc1 = reinterpret_cast<float *>(smem + L.off_sc1);
    float *Ec = reinterpret_cast<float *>(smem + L.off_ec);
    unsigned char *op = smem + L.off_op;                                // tensor-core operand
    const uint32_t sbo = L.sbo;
    float *Mp = reinterpret_cast<float *>(smem + L.off_mp);
    float *reln = reinterpret_cast<float *>(smem + L.off_reln);
    float *adj = reinterpret_cast<float *>(smem + L.off_adj);
    float *Mc = reinterpret_cast<float *>(smem + L.off_mc);
    float *Aj = reinterpret_cast<float *>(smem + L.off_aj);
    float *Bp = reinterpret_cast<float *>(smem + L.off_bp);
    float *Bii = reinterpret_cast<float *>(smem + L.off_bii);
    float4 *pd = reinterpret_cast<float4 *>(smem + L.off_pd);
    float *ps = reinterpret_cast<float *>(smem + L.off_ps);
    float *dxs = reinterpret_cast<float *>(smem + L.off_dx);
    const int Gs = L.Gs, Gs1 = L.Gs1, ES = L.ES;

    const int N = pr.N, t0 = pr.t0, nf = pr.nf;
    const int RS = erow_len(nf), RSS = erow_smem_stride(nf);
    const int kmax = tc_kmax(G_cap);
    const float fx = pr.fx, fy = pr.fy, cx = pr.cx, cy = pr.cy, z_min = pr.z_min, lam = pr.damping;
    const float ifx = 1.0f / fx, ify = 1.0f / fy;
    const float *pose_new = pr.pose_it + (size_t)t * N * 7;
    const float *depth_old = pr.depth_it + (size_t)(t > 0 ? t - 1 : 0) * pr.P;
    float *depth_new = pr.depth_it + (size_t)t * pr.P;
    const float *depth_src = do_bs ? depth_old : depth_new;

    const int nch = *pr.n_chunks;
    const int c_begin = (int)(((long long)itm.item * nch) / pr.n_items);
    const int c_end = (int)(((long long)(itm.item + 1) * nch) / pr.n_items);

    if (do_bs) stage_dxi<TC>(pr, t, dxs, tid, kThreads);   // the previous iteration's pose increments
    if (final_pass) {
        __syncthreads();
        if constexpr (TC) {
            for (int c = c_begin + warp; c < c_end; c += kThreads / 32)
                backsub_chunk_tc(pr, c, dxs, depth_old, depth_new, kmax, lane);
        } else if (c_begin < c_end) {
            const Chunk ca = pr.chunks[c_begin], cz = pr.chunks[c_end - 1];
            backsub_rows(pr, dxs, depth_old, depth_new, ca.k0, cz.k0 + cz.count, tid);
        }
        if (itm.item == 0 && !pr.no_writeback)
            for (int q = tid; q < N * 7; q += kThreads) pr.poses[q] = pose_new[q];
        return;
    }

    // strip ownership of the Schur accumulation
    const int nbp = n_block_pairs(nf);
    const int nbs = 2 * nbp;
    const int nst = nbs + nf;
    const int KS = pr.ks;
    // ext: more free poses than strips fit in registers; the patch products are
    // summed by the assembly kernel and the pose-pair blocks go to global memory
    constexpr bool ext = EXT;   // the host launches EXT exactly for batches with n_asm > 0
    const int my_strip = nst > 0 ? tid % nst : 0;
    const int my_ks = nst > 0 ? tid / nst : KS;
    const bool is_vstrip = my_strip >= nbs;
    const bool owns = !ext && nst > 0 && my_ks < KS && (is_vstrip || !adjoint_rhs);
    int sa = 0, sb = 0, sh = 0;
    if (owns) {
        if (!is_vstrip) {
            decode_pair(my_strip >> 1, nf, sa, sb);
            sh = my_strip & 1;
        } else {
            sa = sb = my_strip - nbs;
        }
    }
    // the strip's compensated running sums (s, c); in the FP32 fused variant
    // they wait in TMEM between the chunks' Schur phases, which leaves their
    // registers to the other phases
    constexpr bool kSumsInTmem = !TC && !EXT;
    float acc_s[18], acc_c[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) { acc_s[q] = 0.f; acc_c[q] = 0.f; }

    for (int q = tid; q < N * 7; q += kThreads) spn[q] = pose_new[q];
    if constexpr (EXT) {
        double *part = pr.partial + (size_t)itm.item * pr.L;
        for (int q = tid; q < pr.L; q += kThreads) part[q] = 0.0;
    }

    // tensor-core state: TMEM accumulator (64 columns), MMA-completion barrier
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_tc_bad;
    uint32_t tmem = 0;
    int n_commit = 0;          // MMA batches committed so far (the same in every thread)
    if constexpr (TC) {
        if (warp == 0) tmem_alloc(&s_tmem, 64);
        if (tid == 0) {
            mbar_init(smem_u32(&s_mbar), 1);
            s_tc_bad = 0;
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tmem = s_tmem;
    }

    // TMEM for the running sums: warp w uses lanes 32 (w % 4) .. + 31,
    // columns 36 (w / 4) .. + 35 (s, then c)
    __shared__ uint32_t s_sums_tmem;
    uint32_t tsums = 0;
    if constexpr (kSumsInTmem) {
        if (warp == 0) tmem_alloc(&s_sums_tmem, kSumsTmemCols);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tsums = s_sums_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(36 * (warp >> 2));
        tmem_st_sums36(tsums, acc_s, acc_c);                 // zeros
    }

    __shared__ __align__(16) Chunk s_ch[2];
    __shared__ __align__(8) uint64_t s_ldbar;    // edge staging: one phase per chunk
    __shared__ __align__(8) uint64_t s_rowbar;   // stored-row staging (back-substitution): one phase per chunk
    __shared__ int s_ld_bad;
    const uint32_t ldbar = smem_u32(&s_ldbar), rowbar = smem_u32(&s_rowbar);
    // Preparation of chunk pc (the pk-th of this CTA), from its staged inputs:
    // the slot -> edge table, the patch data (after the back-substitution of
    // the previous iteration from the staged rows), and, at the start of a
    // group, the window poses (parts: 1 the slot table and window poses, 2 the
    // patch data).  pc is read from shared memory (the descriptor slot stays
    // valid until the copies of the chunk after next start).  It runs during
    // the previous chunk's Schur products (and before the loop for the first
    // chunk): it writes only buffers that chunk no longer reads.  Thread
    // (p = tid mod PS, jl = tid / PS + (256 / PS) i) for the slots, PS = count
    // rounded up to a power of two (at least 8).
    auto prepare = [&](const Chunk &pc, int pk, bool new_group, int parts) {
        int o_jj, o_tw;                                    // alignment slack of the staged edge ranges
        staged_offsets(pr, pc, true, o_jj, o_tw);
        const int cnt = pc.count, e0 = pc.e0, k0 = pc.k0, jlo = pc.jlo;
        const int W = pc.jhi - jlo + 1;
        int lp_sh = 2;
        const int LP = EXT ? lanes_per_patch(cnt, &lp_sh) : 4;
        const int ps_sh = 8 - lp_sh, PSm = (1 << ps_sh) - 1;
        if (parts & 1) {
            const int p = tid & PSm;
            if (p < cnt) {
                const int a = rseg[p] - e0, b = rseg[p + 1] - e0;
                int jf = 0, jz = -1;
                bool contig = true;
                if (b > a) {
                    jf = rjj_s[o_jj + a];
                    jz = rjj_s[o_jj + b - 1];
                    contig = jz - jf + 1 == b - a;         // frames of this patch are contiguous
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
                    sidx[jl * Gs + p] = (short)(idx >= 0 ? idx + o_tw : -1);   // position in the staged target/weight
                }
            }
        }
        if (parts & 2) {   // patch data, after the back-substitution of the previous iteration
            // from the staged rows (four lanes per patch)
            if constexpr (TC) {
                // thread (group g = tid / 8, row slice tid % 8): 4 patches per group
                const int g = tid >> 3, rs = tid & 7, ng = (cnt + 3) >> 2;
                float4 dots = make_float4(0.f, 0.f, 0.f, 0.f);
                const float *grp = srow + (size_t)(g < ng ? g : 0) * (4 * kTcRows);
                if (do_bs) dots = group_dots(grp, dxs, g < ng ? 6 * nf : 0, rs);
                if (g < ng && rs < 4) {
                    const int p = 4 * g + rs;
                    if (p < cnt) {
                        float d = rdep[p];
                        if (do_bs) {
                            const float dot = rs == 0 ? dots.x : rs == 1 ? dots.y : rs == 2 ? dots.z : dots.w;
                            d += grp[4 * (kTcRows - 1) + rs] * (grp[4 * (kTcRows - 2) + rs] - dot);
                            depth_new[k0 + p] = d;
                        }
                        pd[p] = make_float4((rpx[p] - cx) * ifx, (rpy[p] - cy) * ify, d, 0.f);
                    }
                }
            } else {
                // the staged rows completed on rowbar (each reader waits)
                if (do_bs && !mbar_wait(rowbar, (uint32_t)pk & 1u)) atomicOr(&s_ld_bad, 1);
                const int p = tid >> lp_sh, sub = tid & (LP - 1);
                float s = 0.f;
                if (do_bs && p < cnt) {
                    const float4 *row = reinterpret_cast<const float4 *>(srow + p * RSS);
                    const float4 *dz4 = reinterpret_cast<const float4 *>(dxs);
#pragma unroll 4
                    for (int q = sub; q < RS / 4; q += LP) s = dot4(row[q], dz4[q], s);
                }
                s = lane_group_sum(s, LP);
                if (sub == 0 && p < cnt) {
                    float d = rdep[p];
                    if (do_bs) {
                        const float *row = srow + p * RSS;
                        d += row[8 * nf + 1] * (row[8 * nf] - s);
                        depth_new[k0 + p] = d;
                    }
                    pd[p] = make_float4((rpx[p] - cx) * ifx, (rpy[p] - cy) * ify, d, 0.f);
                }
            }
        }
        // (the last warp, which has the fewest patches in this phase)
        if ((parts & 1) && new_group) window_poses(spn, pc.anchor, jlo, W, reln, adj, kThreads - 32);
    };

    if (c_begin < c_end) {
        if (tid == 0) {
            s_ch[0] = pr.chunks[c_begin];
            mbar_init(ldbar, 1);
            mbar_init(rowbar, 1);
            s_ld_bad = 0;
        }
        __syncthreads();
        prefetch_chunk(pr, s_ch[0], depth_src, rjj_s, rtg_s, rwt_s, rpx, rpy, rdep, rseg,
                       c_begin + 1 < c_end ? pr.chunks + c_begin + 1 : nullptr, &s_ch[1], ldbar);
        if (do_bs) {
            if constexpr (TC) prefetch_block(pr, c_begin, s_ch[0], kmax, srow);
            else if (tid == 0) prefetch_rows_bulk(pr, s_ch[0], RS, srow, rowbar);
        }
        cp_async_wait_all();
        if (!mbar_wait(ldbar, 0u)) atomicOr(&s_ld_bad, 1);
        __syncthreads();                                   // the first chunk's inputs are in shared memory
        if (!s_ld_bad) prepare(s_ch[0], 0, true, 3);
        __syncthreads();
    }
    int cur = 0;
    bool group_open = false;   // the previous chunk continues into this one

    bool rows_pending = false;   // last warp: a bulk row store may still read Ec
    bool rows_issued = false;    // last warp: bulk row stores to complete before the exit
    for (int c = c_begin; c < c_end; ++c) {
        // chunk c is prepared (slot table, patch data, window poses) and its
        // edges are staged; the last barrier of the previous iteration (or
        // the prologue's) orders all of it
        if (s_ld_bad) break;                               // a bulk copy never landed: reported below
        const Chunk ch = s_ch[cur];
        const bool have_next = c + 1 < c_end;
        Chunk nx = ch;
        if (have_next) nx = s_ch[cur ^ 1];
        const bool group_next = have_next && nx.anchor == ch.anchor && nx.jlo == ch.jlo && nx.jhi == ch.jhi;
        const int k0 = ch.k0, cnt = ch.count, e0 = ch.e0;
        const int anc = ch.anchor, jlo = ch.jlo;
        const int W = ch.jhi - jlo + 1;
        const bool anc_free = anc >= t0;
        const int NG = kThreads / W;
        const int my_g = tid % NG, my_jl = tid / NG;       // consecutive lanes: consecutive patches of one frame
        const int my_j = jlo + my_jl;
        const bool edge_thread = my_jl < W;

        // lanes per patch of the per-patch phases (LP) and the slot layout
        // (PS = 256 >> lp_sh patches by 256 / PS frame rows)
        int lp_sh = 2;                                     // 4 lanes per patch in the fused variants
        const int LP = EXT ? lanes_per_patch(cnt, &lp_sh) : 4;
        const int ps_sh = 8 - lp_sh, PSm = (1 << ps_sh) - 1;
        if constexpr (TC) {
            // the previous chunk's MMAs read the operand: wait before rewriting it
            if (n_commit > 0 && !mbar_wait(smem_u32(&s_mbar), (uint32_t)(n_commit - 1) & 1u)) atomicOr(&s_tc_bad, 1);
        }
        {   // E columns of free frames outside the window are zero (the edge
            // threads write the others)
            const int p = tid & PSm;
            if (p < cnt)
                for (int f = tid >> ps_sh; f < nf; f += kThreads >> ps_sh) {
                    const int fr = t0 + f;
                    if (fr < jlo || fr > ch.jhi) {
                        if constexpr (TC) {
#pragma unroll
                            for (int m = 0; m < 6; ++m)
                                *reinterpret_cast<float *>(op + op_offset(kTcRows + 6 * f + m, p, sbo)) = 0.f;
                        } else {
                            float4 *e4 = reinterpret_cast<float4 *>(Ec + p * ES + 8 * f);
                            e4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                            e4[1] = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                }
        }


        // -- (b) linearise at the new state.  Each edge thread keeps its frame
        // sums (M_j, v_j) in its own Mp slot between the chunks of a group.
        if (edge_thread) {
            float M[21], V[6];
            {
                const float *mp = Mp + (size_t)tid * 27;
#pragma unroll
                for (int q = 0; q < 21; ++q) M[q] = group_open ? mp[q] : 0.f;
#pragma unroll
                for (int q = 0; q < 6; ++q) V[q] = group_open ? mp[21 + q] : 0.f;
            }
            float Rr[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) Rr[q] = reln[my_jl * 12 + q];
            const bool jfree = my_j >= t0 && my_j != anc;
            const int fj = jfree ? my_j - t0 : 0;
            for (int p = my_g; p < cnt; p += NG) {
                const int slot = my_jl * Gs + p;
                const int ei = sidx[slot];
                float Ce = 0.f, we = 0.f, Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
                float4 elo = make_float4(0.f, 0.f, 0.f, 0.f), ehi = elo;
                if (ei >= 0 && my_j != anc) {
                    const float2 tv = rtg_s[ei], wv = rwt_s[ei];
                    const float4 q = pd[p];
                    EdgeLin E;
                    if ((wv.x != 0.f || wv.y != 0.f) &&
                        edge_linearize(Rr, Rr + 9, q.x, q.y, q.z, tv.x, tv.y, fx, fy, cx, cy, z_min, E)) {
                        float wjd0, wjd1;
                        depth_terms(E, wv.x, wv.y, wjd0, wjd1, Ce, we);
                        anchor_terms(E, Rr, wjd0, wjd1, Y0, Y1, Y2);
                        float wj0[6], wj1[6];
#pragma unroll
                        for (int m = 0; m < 6; ++m) { wj0[m] = wv.x * E.j0[m]; wj1[m] = wv.y * E.j1[m]; }
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
                        elo = make_float4(wj0[0] * E.jd0, wj1[1] * E.jd1, fmaf(wj1[2], E.jd1, wj0[2] * E.jd0), 0.f);
                        ehi = make_float4(fmaf(wj1[3], E.jd1, wj0[3] * E.jd0), fmaf(wj1[4], E.jd1, wj0[4] * E.jd0),
                                          fmaf(wj1[5], E.jd1, wj0[5] * E.jd0), 0.f);
                    }
                }
                if (jfree) {   // e_jk = J_j^T W J_d (zero for a missing or inactive edge)
                    if constexpr (TC) {   // unscaled, FP32, in the hi half
                        const float ev[6] = {elo.x, elo.y, elo.z, ehi.x, ehi.y, ehi.z};
#pragma unroll
                        for (int m = 0; m < 6; ++m)
                            *reinterpret_cast<float *>(op + op_offset(kTcRows + 6 * fj + m, p, sbo)) = ev[m];
                    } else {
                        float4 *e4 = reinterpret_cast<float4 *>(Ec + p * ES + 8 * fj);
                        e4[0] = elo;
                        e4[1] = ehi;
                    }
                }
                sc4[slot] = make_float4(Ce, we, Y0, Y1);
                sc1[my_jl * Gs1 + p] = Y2;
            }
            float *mp = Mp + (size_t)tid * 27;
#pragma unroll
            for (int q = 0; q < 21; ++q) mp[q] = M[q];
#pragma unroll
            for (int q = 0; q < 6; ++q) mp[21 + q] = V[q];
        }
        __syncthreads();
        // the staging buffers are free: start the next chunk's copies
        if (have_next)
            prefetch_chunk(pr, nx, depth_src, rjj_s, rtg_s, rwt_s, rpx, rpy, rdep, rseg,
                           c + 2 < c_end ? pr.chunks + c + 2 : nullptr, &s_ch[cur], ldbar, kPrefetchRot);
        {   // per-patch sums over the window by LP lanes: C_k, w_k, Y; then
            // C_k^-1/2, C_k^-1/2 w_k and the anchor column e_ik = -[d Y; pbar x Y]
            const int p = tid >> lp_sh, sub = tid & (LP - 1);
            float C = sub == 0 ? lam : 0.f, w = 0.f, Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
            if (p < cnt)
#pragma unroll 4
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
            if constexpr (TC) {
                if (p < cnt) {
                    if (sub == 0) {
                        const float sq = sqrtf(1.0f / C);
                        ps[p] = sq;
                        ps[G_cap + p] = sq * (adjoint_rhs ? pr.dbar[k0 + p] : w);
                    } else if (anc_free && sub < 3) {
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
            } else {
                // the same lanes then scale the patch's row of E by C_k^-1/2 in
                // place; the chunk's rows go to global memory by one bulk copy
                // (below), for the next back-substitution
                const float sq = sqrtf(1.0f / C);
                float *e = Ec + p * ES;
                if (p < cnt) {
                    if (sub == 0) {
                        ps[p] = sq;
                        *reinterpret_cast<float4 *>(e + 8 * nf) =
                            make_float4(sq * (adjoint_rhs ? pr.dbar[k0 + p] : w), sq, 0.f, 0.f);
                    } else if (anc_free && sub < 3) {
                        const float4 qd = pd[p];
                        const float d = qd.z, px = qd.x, py = qd.y;
                        float4 *ei = reinterpret_cast<float4 *>(e + 8 * (anc - t0));
                        if (sub == 1) ei[0] = make_float4(-d * Y0, -d * Y1, -d * Y2, 0.f);
                        else          // -(pbar x Y), pbar = (px, py, 1)
                            ei[1] = make_float4(-(py * Y2 - Y1), -(Y0 - px * Y2), -(px * Y1 - py * Y0), 0.f);
                    }
                }
                __syncwarp();
                if (p < cnt) {
                    float4 *e4 = reinterpret_cast<float4 *>(e);
#pragma unroll 4
                    for (int m = sub; m < 2 * nf; m += LP) {
                        float4 v = e4[m];
                        v.x *= sq; v.y *= sq; v.z *= sq;
                        e4[m] = v;
                    }
                }
                fence_async_smem();                        // the rows are read by the bulk copy
            }
        }
        if (!group_next && !adjoint_rhs) {
            // combine the per-thread frame sums (M_j, v_j) over patch groups,
            // compensated; the entries start at the last two warps, which hold
            // no patch above for chunks of up to 48 patches
            for (int q = (tid + kPrefetchRot) & (kThreads - 1); q < W * 27; q += kThreads) {
                const int jl = q / 27, m = q - jl * 27;
                float s = 0.f, cc = 0.f;
#pragma unroll 4
                for (int g = 0; g < NG; ++g) kahan_add(s, cc, Mp[(size_t)(jl * NG + g) * 27 + m]);
                Mc[jl * 27 + m] = s - cc;
            }
        }
        if (!TC && have_next) {                            // the next chunk's inputs (copies started above)
            cp_async_wait_all();
            if (!mbar_wait(ldbar, (uint32_t)(c + 1 - c_begin) & 1u)) atomicOr(&s_ld_bad, 1);
        }
        __syncthreads();
        if constexpr (!TC) {
            // this chunk's scaled rows to global memory: one bulk copy when the
            // shared row stride is the problem's, else one per row (the last
            // warp, which owns the fewest Schur strips)
            // (beyond kFusedMaxFree the adjoint right-hand side is summed from
            // these rows too: they carry C_k^-1/2 dbar_k in place of C_k^-1/2 w_k)
            if (warp == kThreads / 32 - 1 && (EXT || !adjoint_rhs)) {
                if (ES == RS) {
                    if (lane == 0) bulk_copy_s2g(pr.erow + (size_t)k0 * RS, Ec, (uint32_t)(cnt * RS * 4));
                } else {
                    for (int p = lane; p < cnt; p += 32)
                        bulk_copy_s2g(pr.erow + (size_t)(k0 + p) * RS, Ec + p * ES, (uint32_t)(RS * 4));
                }
                bulk_commit();
                rows_pending = true;
                rows_issued = true;
            }
        }
        // the per-slot sums are consumed: start copying the next chunk's stored rows
        if (do_bs && have_next) {
            if constexpr (TC) prefetch_block(pr, c + 1, nx, kmax, srow);
            else if (tid == kThreads - 1) prefetch_rows_bulk(pr, nx, RS, srow, rowbar);
        }
        if constexpr (TC) {
            // Scale each pose column by C_k^-1/2, store the rows for the next
            // back-substitution and split the operand into TF32 hi and lo
            // halves.  A warp takes one 8 x 4 (row, patch) tile at a time,
            // lane = 4 (row % 8) + patch % 4: 128 contiguous bytes of the
            // operand and of the stored block.  Patches cnt..Kc-1 and unused
            // rows are zero.
            const int Kc = (cnt + 7) & ~7, n6 = 6 * nf;
            const int r8 = lane >> 2, k4 = lane & 3;
            float *eb = pr.erow + (size_t)c * kTcRows * kmax;
#pragma unroll 4
            for (int idx = warp; idx < 2 * Kc; idx += kThreads / 32) {   // 8 row groups x Kc / 4 patch groups
                const int rg = idx & 7, kg = idx >> 3;
                const int r = 8 * rg + r8, k = 4 * kg + k4;
                const uint32_t off = (uint32_t)rg * sbo + (uint32_t)kg * kLbo + (uint32_t)(16 * r8 + 4 * k4);
                uint32_t *lp = reinterpret_cast<uint32_t *>(op + off);
                uint32_t *hp = reinterpret_cast<uint32_t *>(op + off + (kTcRows / 8) * sbo);
                const bool in = k < cnt;
                float x = 0.f, e = 0.f;      // operand value, stored-row value
                if (in) {
                    if (r < n6) e = x = __uint_as_float(*hp) * ps[k];
                    else if (r == kTcRows - 2) e = x = ps[G_cap + k];
                    else if (r == kTcRows - 1) e = ps[k];
                }
                if (!adjoint_rhs) eb[kg * (4 * kTcRows) + 4 * r + k4] = e;
                if (r == kTcRows - 1) continue;  // its operand entries come with row 62
                const uint32_t h = to_tf32(x);
                const uint32_t lo = to_tf32(x - __uint_as_float(h));
                if (r == kTcRows - 2) {          // B rows 62, 63: hi and lo of C^-1/2 w
                    hp[0] = h;
                    hp[4] = lo;
                    lp[0] = 0u;
                    lp[4] = 0u;
                } else {
                    *hp = h;
                    *lp = r < n6 ? lo : 0u;
                }
            }
            // the next chunk's inputs and stored rows, for its preparation
            cp_async_wait_all();
            if (have_next && !mbar_wait(ldbar, (uint32_t)(c + 1 - c_begin) & 1u)) atomicOr(&s_ld_bad, 1);
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t base = smem_u32(op);
                constexpr uint32_t idesc = idesc_tf32(2 * kTcRows, kTcRows);
                for (int st = 0; st < (Kc >> 3); ++st) {
                    const uint64_t ad = smem_desc(base + st * 2 * kLbo, kLbo, sbo);
                    const uint64_t bd = smem_desc(base + (kTcRows / 8) * sbo + st * 2 * kLbo, kLbo, sbo);
                    mma_tf32(tmem, ad, bd, idesc, (n_commit > 0 || st > 0) ? 1 : 0);
                }
                mma_commit(smem_u32(&s_mbar));
            }
            ++n_commit;
        }
        if (!group_next && anc_free && !adjoint_rhs) {
            // pose-pair blocks involving the anchor, per window frame j:
            //   B_ij = -Ad_ij^T M_j,  B_ii += Ad_ij^T M_j Ad_ij,  v_i += -Ad_ij^T v_j
            for (int q = tid; q < W * 6; q += kThreads) {
                const int jl = q / 6, r = q - jl * 6;
                const float *Ad = adj + jl * 36;
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

        // the next chunk's slot table, window poses and (without stored rows
        // to wait for) patch data: none of them is read below (s_ld_bad was
        // last written before a barrier).  The tensor-core variant, whose
        // Schur products are not here, prepares after them instead.
        const bool prep_next = have_next && !s_ld_bad;
        if (!TC && prep_next) prepare(s_ch[cur ^ 1], c + 1 - c_begin, !group_next, do_bs ? 1 : 3);

        // -- (c) Schur accumulation over the chunk's patches, then the group's B blocks.
        // A strip with a frame outside the chunk's window would only add zeros
        // (those columns of E are zero): its owner skips the chunk's products.
        if constexpr (kSumsInTmem) tmem_ld_sums36(tsums, acc_s, acc_c);   // whole warps
        if (owns) {
            float blk[18];                                 // FP32 block sum of up to kFlushEvery patches
#pragma unroll
            for (int q = 0; q < 18; ++q) blk[q] = 0.f;
            int since = 0;
            const int fa_s = t0 + sa, fb_s = t0 + sb;
            const bool s_on = fa_s >= jlo && fa_s <= ch.jhi && fb_s >= jlo && fb_s <= ch.jhi;
            if (TC || !s_on) {
                // patch products on the tensor cores, or none in this chunk
            } else if (!is_vstrip) {
                // two patches per step: six 16-byte loads in flight before the FMAs
                const int oa = 8 * sa + 4 * sh, ob = 8 * sb;
                int p = my_ks;
                for (; p + KS < cnt; p += 2 * KS) {
                    const float *e = Ec + p * ES, *f = Ec + (p + KS) * ES;
                    const float4 a4 = *reinterpret_cast<const float4 *>(e + oa);
                    const float4 b0 = *reinterpret_cast<const float4 *>(e + ob);
                    const float4 b1 = *reinterpret_cast<const float4 *>(e + ob + 4);
                    const float4 c4 = *reinterpret_cast<const float4 *>(f + oa);
                    const float4 d0 = *reinterpret_cast<const float4 *>(f + ob);
                    const float4 d1 = *reinterpret_cast<const float4 *>(f + ob + 4);
                    const float ea[3] = {a4.x, a4.y, a4.z}, fa[3] = {c4.x, c4.y, c4.z};
                    const float eb[6] = {b0.x, b0.y, b0.z, b1.x, b1.y, b1.z};
                    const float fb[6] = {d0.x, d0.y, d0.z, d1.x, d1.y, d1.z};
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int cc = 0; cc < 6; ++cc)
                            blk[6 * r + cc] = fmaf(-fa[r], fb[cc], fmaf(-ea[r], eb[cc], blk[6 * r + cc]));
                    since += 2;
                    if (since >= kFlushEvery) {
#pragma unroll
                        for (int q = 0; q < 18; ++q) { kahan_add(acc_s[q], acc_c[q], blk[q]); blk[q] = 0.f; }
                        since = 0;
                    }
                }
                if (p < cnt) {
                    const float *e = Ec + p * ES;
                    const float4 a4 = *reinterpret_cast<const float4 *>(e + oa);
                    const float4 b0 = *reinterpret_cast<const float4 *>(e + ob);
                    const float4 b1 = *reinterpret_cast<const float4 *>(e + ob + 4);
                    const float ea[3] = {a4.x, a4.y, a4.z};
                    const float eb[6] = {b0.x, b0.y, b0.z, b1.x, b1.y, b1.z};
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int cc = 0; cc < 6; ++cc) blk[6 * r + cc] = fmaf(-ea[r], eb[cc], blk[6 * r + cc]);
                }
            } else {
                for (int p = my_ks; p < cnt; p += KS) {
                    const float *e = Ec + p * ES;
                    const float sw = e[8 * nf];
                    const float4 a0 = *reinterpret_cast<const float4 *>(e + 8 * sa);
                    const float4 a1 = *reinterpret_cast<const float4 *>(e + 8 * sa + 4);
                    const float ea[6] = {a0.x, a0.y, a0.z, a1.x, a1.y, a1.z};
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) blk[cc] = fmaf(-ea[cc], sw, blk[cc]);
                    if (++since == kFlushEvery) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) { kahan_add(acc_s[q], acc_c[q], blk[q]); blk[q] = 0.f; }
                        since = 0;
                    }
                }
            }
            if (s_on) {
#pragma unroll
                for (int q = 0; q < 18; ++q) { kahan_add(acc_s[q], acc_c[q], blk[q]); blk[q] = 0.f; }
            }
            if (my_ks == 0 && !group_next && !adjoint_rhs) {
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
        if constexpr (kSumsInTmem) tmem_st_sums36(tsums, acc_s, acc_c);   // whole warps
        if constexpr (EXT) if (!group_next && !adjoint_rhs) {
            // more strips than threads: each pose-pair block goes straight into
            // this CTA's FP64 partial (it owns the partial; groups are
            // sequential).  Only strips of a window frame or the anchor change:
            // per free pose f, its diagonal block (two strips), its v'-strip and
            // the block pairing it with the anchor (two strips).
            double *part = pr.partial + (size_t)itm.item * pr.L;
            const int fanc = anc - t0;
            for (int it5 = tid; it5 < 5 * nf; it5 += kThreads) {
                const int f = it5 / 5, kind = it5 - 5 * f, fr = t0 + f;
                const bool in_w = fr >= jlo && fr < jlo + W;
                int a2 = f, b2 = f, h2 = kind & 1;
                bool vs = false;
                if (kind < 3) {
                    if (!in_w && fr != anc) continue;
                    vs = kind == 2;
                    h2 = kind & 1;
                } else {
                    if (!anc_free || fr == anc || !in_w) continue;
                    a2 = min(f, fanc);
                    b2 = max(f, fanc);
                    h2 = kind - 3;
                }
                const int st = vs ? nbs + f : 2 * (a2 * nf - a2 * (a2 - 1) / 2 + (b2 - a2)) + h2;
                float add[18];
                if (!strip_block_add(a2, b2, h2, vs, t0, anc, jlo, W, Mc, Aj, Bii, add)) continue;
                if (vs) {
                    double *o = part + 18 * nbs + 6 * a2;
#pragma unroll
                    for (int q = 0; q < 6; ++q) o[q] += (double)add[q];
                } else {
                    double *o = part + 18 * st;
#pragma unroll
                    for (int q = 0; q < 18; ++q) o[q] += (double)add[q];
                }
            }
        }
        // with a back-substitution the next chunk's patch data come last, so
        // that its stored rows (started after the per-patch phase) have landed
        if (prep_next && (TC || do_bs)) prepare(s_ch[cur ^ 1], c + 1 - c_begin, !group_next, TC ? 3 : 2);
        if (rows_pending) {                                // Ec is rewritten after the barrier
            bulk_wait_read_all();
            rows_pending = false;
        }
        __syncthreads();
        group_open = group_next;
        cur ^= 1;
    }
    cp_async_wait_all();
    if (rows_issued) bulk_wait_all();                      // the stored rows are written
    if (c_begin < c_end && s_ld_bad) {
        // report, and give the copy that did not land one more bounded wait
        if (tid == 0) {
            atomicOr(pr.status, DPVO_BA_STATUS_TIMEOUT);
            mbar_wait(ldbar, 0u);
            mbar_wait(ldbar, 1u);
            if (!TC && do_bs) {
                mbar_wait(rowbar, 0u);
                mbar_wait(rowbar, 1u);
            }
        }
        __syncthreads();
    }

    if constexpr (TC) {
        // read the accumulator back (warps 0-3, one TMEM lane = one row each)
        // into a buffer over the dead staging area, then each strip owner
        // subtracts its entries: S -= hi.hi + lo.hi + (lo.hi)^T, v' -= the
        // w columns (rows 62, 63 of B)
        float *X = reinterpret_cast<float *>(smem + L.off_rjj);
        if (n_commit > 0 && !mbar_wait(smem_u32(&s_mbar), (uint32_t)(n_commit - 1) & 1u)) atomicOr(&s_tc_bad, 1);
        __syncthreads();
        const bool have = n_commit > 0 && s_tc_bad == 0;
        tc_fence_after();
        if (have && warp < 4) {
#pragma unroll 1
            for (int c4 = 0; c4 < kTcRows / 16; ++c4) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * c4, v);
                float *xr = X + (32 * warp + lane) * kTcXStride + 16 * c4;
#pragma unroll
                for (int q = 0; q < 16; ++q) xr[q] = v[q];
            }
        }
        tc_fence_before();
        __syncthreads();
        if (have && owns) {
            const float *XL = X, *XH = X + kTcRows * kTcXStride;
            if (!is_vstrip) {
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) {
                        const int m = 6 * sa + 3 * sh + r, n = 6 * sb + cc;
                        const float d = XH[m * kTcXStride + n] + XL[m * kTcXStride + n] + XL[n * kTcXStride + m];
                        kahan_add(acc_s[6 * r + cc], acc_c[6 * r + cc], -d);
                    }
            } else {
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) {
                    const int m = 6 * sa + cc;
                    const float d = XH[m * kTcXStride + kTcRows - 2] + XH[m * kTcXStride + kTcRows - 1] +
                                    XL[m * kTcXStride + kTcRows - 2];
                    kahan_add(acc_s[cc], acc_c[cc], -d);
                }
            }
        }
        if (s_tc_bad) {
            // an MMA batch did not complete in time: report it, give the
            // tensor core one more bounded wait, then release TMEM
            if (tid == 0) atomicOr(pr.status, DPVO_BA_STATUS_TIMEOUT);
            if (n_commit > 0) mbar_wait(smem_u32(&s_mbar), (uint32_t)(n_commit - 1) & 1u);
        }
        if (warp == 0) {
            tc_fence_after();
            tmem_dealloc(tmem, 64);
        }
    }

    // write this CTA's partial of (S, v'): with a patch-parity split (KS > 1,
    // at most 10 free poses) the KS parts of each strip are first summed in
    // FP64, in a fixed order, in the frame-sum buffer (dead here), so that the
    // reduced solve reads one partial per CTA
    if constexpr (kSumsInTmem) {
        tmem_ld_sums36(tsums, acc_s, acc_c);
        tc_fence_before();
        __syncthreads();
        if (warp == 0) {
            tc_fence_after();
            tmem_dealloc(s_sums_tmem, kSumsTmemCols);
        }
    }
    double *out = pr.partial + (size_t)itm.item * pr.L;
    if (KS == 1) {
        if (owns) {
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
    } else {
        double *buf = reinterpret_cast<double *>(smem + L.off_mp);
        __syncthreads();
        for (int q = tid; q < pr.L; q += kThreads) buf[q] = 0.0;
        __syncthreads();
        for (int r = 0; r < KS; ++r) {
            if (owns && my_ks == r) {
                if (!is_vstrip) {
                    double *o = buf + 18 * my_strip;
#pragma unroll
                    for (int q = 0; q < 18; ++q) o[q] += (double)acc_s[q] - (double)acc_c[q];
                } else {
                    double *o = buf + 18 * nbs + 6 * sa;
#pragma unroll
                    for (int q = 0; q < 6; ++q) o[q] += (double)acc_s[q] - (double)acc_c[q];
                }
            }
            __syncthreads();
        }
        for (int q = tid; q < pr.L; q += kThreads) out[q] = buf[q];
    }
}

// ----------------------------------------------------------------------------
// final_kernel: the last back-substitution of the depths, on its own.  Only
// reads the stored Schur rows, so it runs with a few hundred bytes of shared
// memory, many CTAs per SM and the problem's patches cut into slices of
// kFinalPatches (row layout) or kFinalChunks chunks (tensor-core layout):
// grid (problems, slices), y-stride over the slices.  Slice 0 also reports the
// status and writes the final poses back.  Problems whose last iteration is
// not t return at once (their final pass ran inside an earlier linearise
// launch).  Dynamic shared memory: the increment, max(kTcRows, erow_len(nf))
// floats.
// ----------------------------------------------------------------------------
constexpr int kFinalPatches = kThreads / 4;
constexpr int kFinalChunks = kThreads / 32;

template <bool TC>
__global__ void __launch_bounds__(kThreads, TC ? 5 : 6) final_kernel(const Prob *__restrict__ probs, int t, int G_cap) {
    extern __shared__ __align__(16) float dxf[];
    const Prob &pr = probs[blockIdx.x];
    const int tid = threadIdx.x;
    if (t != pr.iters) return;
    const int st = block_status(pr.status);
    if (blockIdx.y == 0 && tid == 0 && pr.status_user) *pr.status_user = st;
    if (st != 0) return;
    const int N = pr.N;
    if (blockIdx.y == 0 && !pr.no_writeback) {
        const float *pose_new = pr.pose_it + (size_t)t * N * 7;
        for (int q = tid; q < N * 7; q += kThreads) pr.poses[q] = pose_new[q];
    }
    const int n_units = TC ? *pr.n_chunks : pr.P;
    const int per = TC ? kFinalChunks : kFinalPatches;
    if ((int)blockIdx.y * per >= n_units) return;
    stage_dxi<TC>(pr, t, dxf, tid, kThreads);
    __syncthreads();
    const float *depth_old = pr.depth_it + (size_t)(t - 1) * pr.P;
    float *depth_new = pr.depth_it + (size_t)t * pr.P;
    for (int lo = blockIdx.y * per; lo < n_units; lo += gridDim.y * per) {
        if constexpr (TC) {
            const int c = lo + (tid >> 5);
            if (c < n_units) backsub_chunk_tc(pr, c, dxf, depth_old, depth_new, tc_kmax(G_cap), tid & 31);
        } else {
            backsub_rows(pr, dxf, depth_old, depth_new, lo, min(n_units, lo + per), tid);
        }
    }
}

// ----------------------------------------------------------------------------
// final_rows_kernel: the last back-substitution in the row layout, streamed.
// Grid (problems, CTAs per problem), one wave; each CTA takes the problem's
// 64-patch slices blockIdx.y, blockIdx.y + gridDim.y, ... and brings each
// slice's stored rows (64 consecutive rows, contiguous) into shared memory by
// one bulk copy, kFrStages slices ahead, so that enough bytes are in flight
// for the HBM rate; four lanes per patch then form the dot product from
// shared memory in the order backsub_rows uses.  Every wait is bounded: a copy
// that does not land marks TIMEOUT.  Dynamic shared memory: fr_smem_bytes.
// ----------------------------------------------------------------------------
constexpr int kFrPatches = kThreads / 4;   // patches per slice
constexpr int kFrStages = 2;               // slices in flight per CTA

__host__ __device__ inline size_t fr_smem_bytes(int rs_max) {
    return align16((size_t)rs_max * 4) + (size_t)kFrStages * kFrPatches * rs_max * 4;
}

__global__ void __launch_bounds__(kThreads) final_rows_kernel(const Prob *__restrict__ probs, int t, int rs_max) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ __align__(8) uint64_t s_full[kFrStages];
    __shared__ int s_bad;
    const Prob &pr = probs[blockIdx.x];
    const int tid = threadIdx.x;
    if (t != pr.iters) return;
    const int st = block_status(pr.status);
    if (blockIdx.y == 0 && tid == 0 && pr.status_user) *pr.status_user = st;
    if (st != 0) return;
    const int N = pr.N;
    if (blockIdx.y == 0 && !pr.no_writeback) {
        const float *pose_new = pr.pose_it + (size_t)t * N * 7;
        for (int q = tid; q < N * 7; q += kThreads) pr.poses[q] = pose_new[q];
    }
    const int P = pr.P, nf = pr.nf, RS = erow_len(nf);
    const int n_sl = (P + kFrPatches - 1) / kFrPatches;
    if ((int)blockIdx.y >= n_sl) return;
    const int n_mine = (n_sl - (int)blockIdx.y + (int)gridDim.y - 1) / (int)gridDim.y;
    float *dxf = reinterpret_cast<float *>(fsm);
    float *bufs = reinterpret_cast<float *>(fsm + align16((size_t)rs_max * 4));
    const size_t buf_floats = (size_t)kFrPatches * rs_max;
    if (tid == 0) {
        for (int b = 0; b < kFrStages; ++b) mbar_init(smem_u32(&s_full[b]), 1);
        s_bad = 0;
    }
    stage_dxi<false>(pr, t, dxf, tid, kThreads);
    __syncthreads();
    // thread 0: the i-th of this CTA's slices into buffer i % kFrStages
    auto issue = [&](int i) {
        const int k0 = ((int)blockIdx.y + i * (int)gridDim.y) * kFrPatches;
        const int cnt = min(kFrPatches, P - k0);
        const uint32_t bar = smem_u32(&s_full[i % kFrStages]);
        const uint32_t bytes = (uint32_t)(cnt * RS * 4);   // a multiple of 16: RS = 8 nf + 4
        fence_async_smem();                                // the buffer's earlier reads come first
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
        bulk_copy_g2s(bufs + (i % kFrStages) * buf_floats, pr.erow + (size_t)k0 * RS, bytes, bar);
    };
    if (tid == 0)
        for (int i = 0; i < min(kFrStages, n_mine); ++i) issue(i);
    const float *depth_old = pr.depth_it + (size_t)(t - 1) * P;
    float *depth_new = pr.depth_it + (size_t)t * P;
    const float4 *dz4 = reinterpret_cast<const float4 *>(dxf);
    const int p = tid >> 2, sub = tid & 3;
    for (int i = 0; i < n_mine; ++i) {
        const int k0 = ((int)blockIdx.y + i * (int)gridDim.y) * kFrPatches;
        const int cnt = min(kFrPatches, P - k0), k = k0 + p;
        const float d_old = p < cnt && sub == 0 ? depth_old[k] : 0.f;
        const bool landed = mbar_wait(smem_u32(&s_full[i % kFrStages]), (uint32_t)(i / kFrStages) & 1u);
        if (!landed) s_bad = 1;
        const float *row = bufs + (i % kFrStages) * buf_floats + (size_t)p * RS;
        float s = 0.f;
        if (landed && p < cnt) {
            const float4 *row4 = reinterpret_cast<const float4 *>(row);
#pragma unroll 4
            for (int q = sub; q < RS / 4; q += 4) s = dot4(row4[q], dz4[q], s);
        }
        s = quad_sum(s);
        if (landed && p < cnt && sub == 0) {
            const float dnew = d_old + row[8 * nf + 1] * (row[8 * nf] - s);
            depth_new[k] = dnew;
            if (!pr.no_writeback) pr.patches[3 * k + 2] = dnew;
        }
        __syncthreads();                                   // the buffer is read
        if (s_bad) break;                                  // read after the barrier: the same in every thread
        if (tid == 0 && i + kFrStages < n_mine) issue(i + kFrStages);
    }
    if (s_bad && tid == 0) {
        // report, and give the copies still in flight one more bounded wait
        atomicOr(pr.status, DPVO_BA_STATUS_TIMEOUT);
        for (int b = 0; b < kFrStages; ++b) {
            mbar_wait(smem_u32(&s_full[b]), 0u);
            mbar_wait(smem_u32(&s_full[b]), 1u);
        }
    }
}

// ----------------------------------------------------------------------------
// solve_kernel: one CTA of kSolveThreads per problem.  Sums the Schur partials
// in FP64 (fixed order), factors the reduced pose system by Cholesky in its
// square-root-free form S = U D^-1 U^T (U lower, D = diag U) with the right-
// hand side eliminated alongside, back-substitutes for the pose increments and
// retracts the free poses in FP64.  A pivot <= 0 or NaN marks the problem
// NOT_SPD.  If S_out is non-null, writes (S, v') there instead and changes
// nothing else.
// ----------------------------------------------------------------------------
constexpr int kSolveThreads = 256;
// elements of the largest trailing triangle of solve_kernel (at most kFusedMaxFree
// free poses), (6 nf - 1) 6 nf / 2, per thread
constexpr int kSolveOwn = ((6 * kFusedMaxFree - 1) * 6 * kFusedMaxFree / 2 + kSolveThreads - 1) / kSolveThreads;

__device__ __forceinline__ double shfl_double(double x, int src) {
    int lo = __double2loint(x), hi = __double2hiint(x);
    lo = __shfl_sync(0xffffffffu, lo, src);
    hi = __shfl_sync(0xffffffffu, hi, src);
    return __hiloint2double(hi, lo);
}

// ---- blocked triangular solves with inverted diagonal blocks (both reduced solves)
constexpr int kPanel = 32;             // panel width of the blocked factorisation and solves
constexpr int kLinvLd = kPanel + 1;     // row stride of an inverted diagonal block (conflict-free rows and columns)

// Warp w of the CTA, for panel J = kPanel w: the inverse of the panel's unit
// lower diagonal block, L_rj = a_rj / p_j (r > j), into Linv + w kPanel kLinvLd
// at [r kLinvLd + c].  Lane c computes column c by forward substitution.  The
// factor's element (i, k), k <= i, is Sp[idx(i, k)], each row's entries
// consecutive.
template <class Idx>
__device__ void invert_diag_blocks(const float *Sp, Idx idx, const float *rp, float *Linv, int n, int tid) {
    const int warp = tid >> 5, lane = tid & 31, J = kPanel * warp;
    if (J >= n) return;
    const int nb = min(kPanel, n - J);
    float z[kPanel];
#pragma unroll
    for (int r = 0; r < kPanel; ++r) {
        float acc = 0.f;
        if (r < nb) {
            const int rr = idx(J + r, J);
#pragma unroll
            for (int j = 0; j < r; ++j) acc = fmaf(Sp[rr + j] * rp[J + j], z[j], acc);
        }
        z[r] = r == lane ? 1.f : -acc;             // zero above the diagonal (z_j = 0 for j < lane)
    }
    float *L = Linv + warp * kPanel * kLinvLd;
    if (lane < nb) {
#pragma unroll
        for (int r = 0; r < kPanel; ++r)
            if (r < nb) L[r * kLinvLd + lane] = z[r];
    }
}

// All threads: solve S x = b in place in b (shared memory), S = U D^-1 U^T
// held as the eliminated values a_ij (j <= i) at Sp[idx(i, j)] with pivot
// reciprocals rp, by panels of kPanel: each panel's diagonal block by one warp
// as a product with its inverse (invert_diag_blocks), the rows outside it by
// one thread each.
template <class Idx>
__device__ void solve_blocked_f32(const float *Sp, Idx idx, const float *rp, const float *Linv, float *b, int n,
                                  int tid) {
    __shared__ float s_t[kPanel];                          // y_j / p_j of the current panel
    const int lane = tid & 31;
    for (int J = 0; J < n; J += kPanel) {                  // forward: y_J = L_JJ^-1 b_J, then the rows below
        const int nb = min(kPanel, n - J);
        if (tid < 32) {
            const float *L = Linv + (J / kPanel) * kPanel * kLinvLd + lane * kLinvLd;
            float y0 = 0.f, y1 = 0.f;
            if (lane < nb) {
#pragma unroll
                for (int c = 0; c < kPanel; c += 2) {
                    if (c <= lane && c < nb) y0 = fmaf(L[c], b[J + c], y0);
                    if (c + 1 <= lane && c + 1 < nb) y1 = fmaf(L[c + 1], b[J + c + 1], y1);
                }
            }
            __syncwarp();
            if (lane < nb) {
                const float y = y0 + y1;
                b[J + lane] = y;
                s_t[lane] = y * rp[J + lane];
            }
        }
        __syncthreads();
        for (int i = J + nb + tid; i < n; i += kSolveThreads) {   // nb == kPanel here
            const int ri = idx(i, J);
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < kPanel; ++j) acc = fmaf(Sp[ri + j], s_t[j], acc);
            b[i] -= acc;
        }
        __syncthreads();
    }
    for (int J = ((n - 1) / kPanel) * kPanel; J >= 0; J -= kPanel) {   // backward: x_J = L_JJ^-T D_J^-1 w_J
        const int nb = min(kPanel, n - J);
        if (tid < 32) {
            const float *L = Linv + (J / kPanel) * kPanel * kLinvLd + lane;
            float x0 = 0.f, x1 = 0.f;
            if (lane < nb) {
#pragma unroll
                for (int c = 0; c < kPanel; c += 2) {
                    if (c >= lane && c < nb) x0 = fmaf(L[c * kLinvLd], rp[J + c] * b[J + c], x0);
                    if (c + 1 >= lane && c + 1 < nb) x1 = fmaf(L[(c + 1) * kLinvLd], rp[J + c + 1] * b[J + c + 1], x1);
                }
            }
            __syncwarp();
            if (lane < nb) b[J + lane] = x0 + x1;
        }
        __syncthreads();
        for (int i = tid; i < J; i += kSolveThreads) {
            float acc = 0.f;
            for (int j = 0; j < nb; ++j) acc = fmaf(Sp[idx(J + j, i)], b[J + j], acc);
            b[i] -= acc;
        }
        __syncthreads();
    }
}

// Row-major storage with leading dimension ld.
struct RowMajorIdx {
    int ld;
    __device__ __forceinline__ int operator()(int i, int k) const { return i * ld + k; }
};

// ---- FP32 factorisation of the reduced system by panels (solve_kernel)
constexpr int kSolvePanel = 8;          // columns per panel: two block barriers per panel

// One warp: eliminate the nb x nb diagonal block at (J, J) of the FP32 copy Sf
// (row stride ldf) in the square-root-free form (pivots d_j on the diagonal,
// eliminated values a_ij below, a_ik -= a_ij a_kj / d_j), its pivot
// reciprocals into rp[J..J+nb).  A pivot <= 0 or not finite sets *bad.
__device__ __forceinline__ void factor_diag_block(float *Sf, int ldf, int J, int nb, float *rp, int lane,
                                                  int *bad) {
    for (int j = 0; j < nb; ++j) {
        const float d = Sf[(J + j) * ldf + J + j];
        const float r = 1.0f / d;
        if (lane == 0) {
            rp[J + j] = r;
            if (!(d > 0.f) || !isfinite(r)) *bad = 1;
        }
        // elements (i, k), j < k <= i < nb, one per lane (at most 28)
        const int m = nb - 1 - j;
        for (int e = lane; e < m * (m + 1) / 2; e += 32) {
            int c = 0, q = e;
            while (q >= m - c) { q -= m - c; ++c; }      // column c of the trailing block, row c + q
            const int k = J + j + 1 + c, i = k + q;
            Sf[i * ldf + k] = fmaf(-Sf[i * ldf + J + j] * r, Sf[k * ldf + J + j], Sf[i * ldf + k]);
        }
        __syncwarp();
    }
}

// One warp: solve (U D^-1 U^T) z = b for the factor above (l_ij = a_ij / d_j):
// forward L y = b, w = D^-1 y, backward L^T z = w.  b in shared memory (n
// entries), overwritten by z; each lane keeps rows lane, lane + 32, lane + 64.
__device__ __forceinline__ void solve_ldl_warp(const float *Sf, int ldf, const float *rp, float *b, int n,
                                               int lane) {
    float x[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) x[t] = lane + 32 * t < n ? b[lane + 32 * t] : 0.f;
    for (int j = 0; j < n; ++j) {                                   // forward
        const float y = __shfl_sync(0xffffffffu, x[j >> 5], j & 31) * rp[j];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int r = lane + 32 * t;
            if (r > j && r < n) x[t] = fmaf(-Sf[r * ldf + j], y, x[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t)
        if (lane + 32 * t < n) x[t] *= rp[lane + 32 * t];
    for (int j = n - 1; j > 0; --j) {                               // backward
        const float z = __shfl_sync(0xffffffffu, x[j >> 5], j & 31);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int r = lane + 32 * t;
            if (r < j) x[t] = fmaf(-Sf[j * ldf + r] * rp[r], z, x[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t)
        if (lane + 32 * t < n) b[lane + 32 * t] = x[t];
}

constexpr int kMaxRefine = 4;          // FP64 refinement steps of the FP32 solution at most
constexpr double kRefineTol = 1e-6;    // accept once the last correction is below this x max|x|

__global__ void __launch_bounds__(kSolveThreads) solve_kernel(const Prob *__restrict__ probs, int t,
                                                              double *S_out, double *v_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Prob &pr = probs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31;
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
            for (int q = tid; q < N * 7; q += kSolveThreads) pose_next[q] = pose_cur[q];
            for (int q = tid; q < nf * 6; q += kSolveThreads) dxi[q] = 0.0;
        }
        return;
    }
    const int ld = n + 1;
    double *S = reinterpret_cast<double *>(smem);
    double *v = S + (size_t)n * ld;
    __shared__ double s_rp[6 * kMaxFree];    // pivot reciprocals, reused by the back substitution

    // FP64 sum of the partials in a fixed order (deterministic)
    const int Lp = pr.L, nparts = pr.n_parts, nbs = 2 * n_block_pairs(nf);
    constexpr int kQ = 8;                       // entries per thread with loads in flight together
    for (int q0 = tid; q0 < Lp; q0 += kQ * kSolveThreads) {
        double accs[kQ];
#pragma unroll
        for (int u = 0; u < kQ; ++u) accs[u] = 0.0;
        for (int part = 0; part < nparts; ++part) {   // parts summed in order
            const double *src = pr.partial + (size_t)part * Lp;
            double x[kQ];
#pragma unroll
            for (int u = 0; u < kQ; ++u) {
                const int q = q0 + u * kSolveThreads;
                x[u] = q < Lp ? src[q] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kQ; ++u) accs[u] += x[u];
        }
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            const int q = q0 + u * kSolveThreads;
            if (q >= Lp) break;
            if (q < 18 * nbs) {
                const int st = q / 18, e = q - 18 * st;
                int a, b;
                decode_pair(st >> 1, nf, a, b);
                const int row = 6 * a + 3 * (st & 1) + e / 6, col = 6 * b + e % 6;
                S[row * ld + col] = accs[u];
                if (a != b) S[col * ld + row] = accs[u];
            } else {
                v[q - 18 * nbs] = accs[u];
            }
        }
    }
    __syncthreads();
    if (S_out != nullptr) {
        for (int q = tid; q < n * n; q += kSolveThreads) S_out[q] = S[(q / n) * ld + q % n];
        for (int q = tid; q < n; q += kSolveThreads) v_out[q] = v[q];
        return;
    }
    // right-looking elimination of the lower triangle.  The trailing triangle
    // of step j (rows i > j, columns j < k <= i) is enumerated in reversed
    // coordinates r = n-1-i <= c = n-1-k, column-major in c, so that the
    // elements of step j are exactly the first m (m + 1) / 2 of one fixed
    // sequence (m = n-1-j): thread tid owns elements tid + kSolveThreads u of
    // it for every step, and the warps stay full as the triangle shrinks.
    int own[kSolveOwn];
#pragma unroll
    for (int u = 0; u < kSolveOwn; ++u) {
        const int q = tid + kSolveThreads * u;
        int c = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
        while (c * (c + 1) / 2 > q) --c;                    // exact integer correction
        while ((c + 1) * (c + 2) / 2 <= q) ++c;
        const int r = q - c * (c + 1) / 2;
        own[u] = ((n - 1 - r) << 16) | (n - 1 - c);          // (i, k)
    }

    // Forward solves factor an FP32 copy of S (the same elimination, on the
    // FP32 pipes) and refine its solution against S in FP64: x += S32^-1 (v -
    // S x) until the correction is below kRefineTol of the solution.  A pivot
    // that fails in FP32, or corrections that do not shrink, hand the system
    // to the FP64 elimination below, which also serves the adjoint (it keeps
    // the FP64 factor).
    __shared__ int s_use64;
    __shared__ float s_rpf[6 * kMaxFree];
    __shared__ double s_red[kSolveThreads / 32][2];
    if (tid == 0) s_use64 = pr.store_factor ? 1 : 0;
    __syncthreads();
    if (!s_use64) {
        double *x = v + n;
        const int ldf = (n + 3) & ~3;
        float *Sf = reinterpret_cast<float *>(x + n);          // [n][ldf] FP32 copy, factored in place
        float *Lp = Sf + (size_t)n * ldf;                       // [n][kSolvePanel] a_im / d_m of the panel
        float *bf = Lp + (size_t)n * kSolvePanel;               // [n] right-hand side, then the correction
        __shared__ int s_next;                                  // 1: refine again, 0: done
        for (int q = tid; q < n * n; q += kSolveThreads) {
            const int i = q / n, k = q - i * n;
            if (k <= i) Sf[i * ldf + k] = (float)S[i * ld + k];
        }
        for (int q = tid; q < n * kSolvePanel; q += kSolveThreads) Lp[q] = 0.f;
        for (int q = tid; q < n; q += kSolveThreads) {
            x[q] = 0.0;
            bf[q] = (float)v[q];
        }
        __syncthreads();
        // Panels of kSolvePanel columns: (1) the diagonal block by warp 0
        // (the first one here, each next one at the end of (3)); (2) the
        // panel's rows below the block, by forward substitution with the
        // block's factor, one thread per row, with their scaled copies
        // l_im = a_im / d_m; (3) the trailing triangle's rank-kSolvePanel
        // update a_ik -= sum_m l_im a_km, every thread its own elements (the
        // next diagonal block's by warp 0, which then eliminates it).
        if (tid < 32) factor_diag_block(Sf, ldf, 0, min(kSolvePanel, n), s_rpf, lane, &s_use64);
        __syncthreads();
        for (int J = 0; J < n && !s_use64; J += kSolvePanel) {
            const int nb = min(kSolvePanel, n - J), J2 = J + nb;
            for (int i = J2 + tid; i < n; i += kSolveThreads) {
                float a[kSolvePanel];
                float *row = Sf + i * ldf + J;
#pragma unroll
                for (int j = 0; j < kSolvePanel; ++j) {
                    if (j >= nb) { a[j] = 0.f; continue; }
                    float t = row[j];
#pragma unroll
                    for (int m = 0; m < j; ++m) t = fmaf(-a[m] * s_rpf[J + m], Sf[(J + j) * ldf + J + m], t);
                    a[j] = t;
                }
#pragma unroll
                for (int j = 0; j < kSolvePanel; ++j) {
                    if (j < nb) row[j] = a[j];
                    Lp[i * kSolvePanel + j] = j < nb ? a[j] * s_rpf[J + j] : 0.f;
                }
            }
            __syncthreads();
            if (J2 < n) {
                const int m = n - J2, count = m * (m + 1) / 2;
                const int nb2 = min(kSolvePanel, n - J2), blk_end = J2 + nb2;
#pragma unroll
                for (int u = 0; u < kSolveOwn; ++u) {
                    const int q = tid + kSolveThreads * u;
                    if (q >= count) break;
                    const int i = own[u] >> 16, k = own[u] & 0xffff;
                    if (i < blk_end) continue;                  // the next diagonal block: warp 0 below
                    const float4 *li = reinterpret_cast<const float4 *>(Lp + i * kSolvePanel);
                    const float4 *ak = reinterpret_cast<const float4 *>(Sf + k * ldf + J);
                    const float4 l0 = li[0], l1 = li[1], a0 = ak[0], a1 = ak[1];
                    float t = Sf[i * ldf + k];
                    t = fmaf(-l0.x, a0.x, fmaf(-l0.y, a0.y, fmaf(-l0.z, a0.z, fmaf(-l0.w, a0.w, t))));
                    t = fmaf(-l1.x, a1.x, fmaf(-l1.y, a1.y, fmaf(-l1.z, a1.z, fmaf(-l1.w, a1.w, t))));
                    Sf[i * ldf + k] = t;
                }
                if (tid < 32) {
                    for (int e = lane; e < nb2 * (nb2 + 1) / 2; e += 32) {   // the next block's trailing update
                        int c = 0, q = e;
                        while (q >= nb2 - c) { q -= nb2 - c; ++c; }
                        const int k = J2 + c, i = k + q;
                        const float4 *li = reinterpret_cast<const float4 *>(Lp + i * kSolvePanel);
                        const float4 *ak = reinterpret_cast<const float4 *>(Sf + k * ldf + J);
                        const float4 l0 = li[0], l1 = li[1], a0 = ak[0], a1 = ak[1];
                        float t = Sf[i * ldf + k];
                        t = fmaf(-l0.x, a0.x, fmaf(-l0.y, a0.y, fmaf(-l0.z, a0.z, fmaf(-l0.w, a0.w, t))));
                        t = fmaf(-l1.x, a1.x, fmaf(-l1.y, a1.y, fmaf(-l1.z, a1.z, fmaf(-l1.w, a1.w, t))));
                        Sf[i * ldf + k] = t;
                    }
                    __syncwarp();
                    factor_diag_block(Sf, ldf, J2, nb2, s_rpf, lane, &s_use64);
                }
                __syncthreads();
            }
        }
        // Solve and refine: the FP32 solve by warp 0, the FP64 residual v - S x
        // by all threads.  Stop once a correction is below kRefineTol of the
        // solution, or once the first correction is below 1e-4 of it (the
        // refinement then contracts by about that ratio, so the next correction
        // would be below 1e-8 of it); a correction that does not shrink to half
        // the previous one, or kMaxRefine corrections, hand the system to FP64.
        if (tid == 0) s_next = s_use64 ? 0 : 1;
        __syncthreads();
        double prev = 0.0;
        for (int it = 0; it <= kMaxRefine && s_next; ++it) {
            if (it > 0) {
                const int qk = tid & 3;
                for (int base = 0; base < n; base += kSolveThreads / 4) {
                    const int i = base + (tid >> 2);
                    double acc = 0.0;
                    if (i < n)
                        for (int k = qk; k < n; k += 4) acc = fma(S[i * ld + k], x[k], acc);
                    acc += shfl_double(acc, lane ^ 1);
                    acc += shfl_double(acc, lane ^ 2);
                    if (i < n && qk == 0) bf[i] = (float)(v[i] - acc);
                }
                __syncthreads();
            }
            if (tid < 32) {
                solve_ldl_warp(Sf, ldf, s_rpf, bf, n, lane);
                __syncwarp();
                double dmax = 0.0, xmax = 0.0;
                for (int q = lane; q < n; q += 32) {
                    const double d = (double)bf[q];
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
                if (lane == 0) {
                    int next = 1;
                    if (!(dmax <= 1e300)) { s_use64 = 1; next = 0; }                    // non-finite
                    else if (it > 0 && (dmax <= kRefineTol * xmax || (it == 1 && dmax <= 1e-4 * xmax))) next = 0;
                    else if (it > 1 && !(dmax <= 0.5 * prev)) { s_use64 = 1; next = 0; }   // not contracting
                    else if (it == kMaxRefine) { s_use64 = 1; next = 0; }
                    s_next = next;
                }
                prev = dmax;
            }
            __syncthreads();
        }
        if (!s_use64)
            for (int q = tid; q < n; q += kSolveThreads) v[q] = x[q];
        __syncthreads();
    }

    if (s_use64) {
    // The reciprocal of each pivot is formed by the thread that updates the
    // pivot in the step before (it owns the last element of that step's
    // triangle), first in its list, so the division overlaps the step's
    // other updates; a pivot <= 0 or NaN is recorded as -1.
    if (tid == 0) {
        const double p0 = S[0];
        s_rp[0] = p0 > 0.0 ? 1.0 / p0 : -1.0;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        const double ip = s_rp[j];
        if (!(ip > 0.0)) {
            if (tid == 0) s_flag = DPVO_BA_STATUS_NOT_SPD;
            break;
        }
        const int m = n - 1 - j, count = m * (m + 1) / 2;
        const double *colj = S + j;
        const int last = count - 1;                          // element (j+1, j+1)
        if (count > 0 && tid == last % kSolveThreads) {
            const int jn = j + 1;
            const double pn = S[jn * ld + jn] - (colj[jn * ld] * ip) * colj[jn * ld];
            S[jn * ld + jn] = pn;
            s_rp[jn] = pn > 0.0 ? 1.0 / pn : -1.0;
        }
#pragma unroll
        for (int u = 0; u < kSolveOwn; ++u) {
            const int q = tid + kSolveThreads * u;
            if (q >= last) break;
            const int i = own[u] >> 16, k = own[u] & 0xffff;
            S[i * ld + k] -= (colj[i * ld] * ip) * colj[k * ld];
        }
        if (tid < m) {
            const int i = j + 1 + tid;
            v[i] -= (colj[i * ld] * ip) * v[j];
        }
        __syncthreads();
    }
    __syncthreads();
    if (!s_flag && pr.store_factor) {   // keep U for the adjoint solve
        double *u = pr.ufac + (size_t)t * (n * (n + 1) / 2);
        for (int q = tid; q < n * n; q += kSolveThreads) {
            const int i = q / n, k = q - i * n;
            if (k <= i) u[i * (i + 1) / 2 + k] = S[i * ld + k];
        }
    }
    if (!s_flag && tid < 32) {
        // U^T x = v' (back substitution, one warp): x_j = v_j / U_jj, v_i -= U_ji x_j,
        // with the reciprocals of the pivots kept from the factorisation
        for (int j = n - 1; j >= 0; --j) {
            const double xj = v[j] * s_rp[j];
            for (int i = lane; i < j; i += 32) v[i] -= S[j * ld + i] * xj;
            __syncwarp();
            if (lane == 0) v[j] = xj;
            __syncwarp();
        }
    }
    }   // FP64 elimination
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
