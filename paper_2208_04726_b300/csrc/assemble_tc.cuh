// Schur assembly on the tensor cores, for reduced systems with more free poses
// than the linearise kernel's strip owners hold (Sec. 3.1, the Schur
// complement over the inverse depths), in the opt-in TF32 Schur mode:
//     S  -= sum_k (C_k^-1/2 e_k)(C_k^-1/2 e_k)^T,   v' -= sum_k (C_k^-1/2 e_k)(C_k^-1/2 w_k).
// For a wide window this sum is a dense product X^T X over the patches, X the
// stored rows C_k^-1/2 (e_k, w_k): 16,384 patches by 192 pose columns on the
// 64-frame window.
//
// Operand: the n6 = 6 nf pose entries of each patch's row (the stored row's
// pads [v0 v1 v2 0 v3 v4 v5 0] dropped: operand row 6f + c is pose component c
// of free frame f) as a K-major TF32 operand of kAtcOpRows rows (zero beyond
// n6) over kAtcK patches, split into hi = tf32(x) and lo = tf32(x - hi)
// (rounded to nearest: |lo| <= 2^-11 |x|, and lo within 2^-11 |lo| of x - hi;
// truncating hi instead doubled the error of S and of late increments).
// Three TF32 products hi hi^T + lo hi^T + hi lo^T give the FP32-accurate
// product (the lo lo^T term is below FP32 rounding).  Per 8 patches: rows
// 0..127 against rows 0..n6-1 (M = 128, N = n6 rounded up to 16) into TMEM
// columns 0.., and, beyond 128 rows, rows a0..a0+127 (a0 = n6 rounded up to
// 8, less 128) against rows 120..n6-1 (from the first frame that reaches row
// 128, rounded down to 8) into columns 256..; every pose-pair block a <= b
// lies in one of the two.
// v' stays on the CUDA cores: it tends to zero as the iterations converge,
// so its terms cancel, and the two lanes that split row m (each half the
// patches of a stage) sum its products in FP32 per stage, with compensated
// adds across stages, as the CUDA-core assembly does; the halves meet in FP64.
//
// One CTA of kAtcThreads threads per (problem, work item): a range of at most
// kAtcMaxPatches patches (the FP32 accumulation length in TMEM).  A producer
// warp streams the stored rows through kAtcRawStages shared-memory stages by
// bulk copies and issues the MMAs of a stage once the split warps have
// arrived on its operands' mbarrier; the split warps fill one of two operand
// buffers while the MMAs of the previous stage run.  Every wait is bounded; on a
// timeout the CTA reports DPVO_BA_STATUS_TIMEOUT, waits (again bounded) for
// its copies and MMAs in flight and leaves.  The result goes to the CTA's FP64
// partial in the layout of schur_assembly_kernel (the 6 x 6 block of pair
// (a, b), a <= b, row-major at 36 x its pair index, then v').
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "assemble.cuh"
#include "ba_common.cuh"
#include "tc.cuh"

namespace dpvo {

constexpr int kAtcSplitWarps = 16;                            // warps that split the operands
constexpr int kAtcThreads = 32 * (kAtcSplitWarps + 1);         // + the producer warp (copies, MMAs)
constexpr int kAtcRowWarps = 14;                              // split warps with rows (7 row chunks x 2 halves)
constexpr int kAtcK = 32;                                      // patches per stage
constexpr int kAtcOpRows = 200;                                // operand rows: 6 x 32 pose entries, and the
                                                               // zero rows 192..199 the second product reads
constexpr int kAtcB0 = 120;                                    // first row of the second product's B operand
constexpr uint32_t kAtcSbo = (kAtcK / 4) * kLbo;               // bytes between 8-row groups
constexpr uint32_t kAtcOpBytes = (kAtcOpRows / 8) * kAtcSbo;   // one operand half (hi or lo)
constexpr int kAtcMaxPatches = 2048;                           // patches per CTA at most
constexpr int kAtcCols = 512;                                  // TMEM columns allocated (336 used at most)
constexpr int kAtcRawStages = 3;                               // row stages: copies two stages ahead

// Dynamic shared memory: two operand buffers (hi, lo), then the row stages.
__host__ __device__ inline size_t atc_smem_bytes(int rs_max) {
    return 4 * (size_t)kAtcOpBytes + kAtcRawStages * (size_t)kAtcK * rs_max * 4;
}

// x rounded to TF32 (10 mantissa bits), to nearest with ties away from zero,
// by integer operations on its bits: half a unit of the last kept place is
// added to the magnitude (a carry moves into the exponent as it should) and
// the 13 dropped bits are cleared.  For finite x.
__device__ __forceinline__ uint32_t tf32_rna(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

// Entry of the stored row that holds pose entry m = 6 f + c.
__device__ __forceinline__ int atc_src(int m) {
    const int f = m / 6, c = m - 6 * f;
    return 8 * f + (c < 3 ? c : c + 1);
}

__global__ void __launch_bounds__(kAtcThreads, 1) schur_assembly_tc_kernel(const Prob *__restrict__ probs,
                                                                           const Item *__restrict__ items, int t,
                                                                           int rs_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Item itm = items[blockIdx.x];
    const Prob &pr = probs[itm.prob];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (t >= pr.iters || block_status(pr.status) != 0) return;

    const int nf = pr.nf, RS = erow_len(nf), np = n_block_pairs(nf), n6 = 6 * nf;
    const int k_lo = (int)(((long long)itm.item * pr.P) / pr.n_asm);
    const int k_hi = (int)(((long long)(itm.item + 1) * pr.P) / pr.n_asm);
    const int n_st = (k_hi - k_lo + kAtcK - 1) / kAtcK;
    const bool two = n6 > 128;                                 // the second product
    const int N0 = (n6 + 15) & ~15, a0 = ((n6 + 7) & ~7) - 128, N1 = two ? (n6 - kAtcB0 + 15) & ~15 : 0;
    double *out = pr.partial + (size_t)(pr.n_items + itm.item) * pr.L;
    if (n_st == 0) {
        for (int q = tid; q < pr.L; q += kAtcThreads) out[q] = 0.0;
        return;
    }

    unsigned char *ops = smem;                                 // buffer b: hi at 2b kAtcOpBytes, lo after it
    float *raw0 = reinterpret_cast<float *>(smem + 4 * kAtcOpBytes);
    const size_t raw_len = (size_t)kAtcK * rs_max;
    __shared__ __align__(8) uint64_t s_full[kAtcRawStages], s_op[2], s_done[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_bad;
    if (warp == 0) tmem_alloc(&s_tmem, kAtcCols);
    if (tid == 0) {
        for (int r = 0; r < kAtcRawStages; ++r) mbar_init(smem_u32(&s_full[r]), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&s_op[b]), kAtcSplitWarps);
            mbar_init(smem_u32(&s_done[b]), 1);
        }
        s_bad = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int *bad = &s_bad;

    // the producer lane's bookkeeping: stages whose rows were requested, the last stage committed
    int n_issued = 0, last_commit = -1;
    float v_s = 0.f, v_c = 0.f;                                // v' of the lane's row, half the patches
    __shared__ double s_vh[kAtcOpRows];                        // the other half's v' (warps 7..13)
    if (warp == kAtcSplitWarps) {
        // producer: stored rows into the row stages, MMAs once a stage's operands are split
        if (lane == 0) {
            auto issue = [&](int s) {
                const int k0 = k_lo + s * kAtcK, rows = min(kAtcK, k_hi - k0);
                bulk_load(raw0 + (s % kAtcRawStages) * raw_len, pr.erow + (size_t)k0 * RS, (uint32_t)(rows * RS * 4),
                          smem_u32(&s_full[s % kAtcRawStages]));
                n_issued = s + 1;
            };
            for (int s = 0; s < kAtcRawStages && s < n_st; ++s) issue(s);
            const uint32_t oa = (uint32_t)(a0 >> 3) * kAtcSbo, ob = (uint32_t)(kAtcB0 >> 3) * kAtcSbo;
            const uint32_t id0 = idesc_tf32(128, N0), id1 = idesc_tf32(128, two ? N1 : 16);
            for (int s = 0; s < n_st && !*bad; ++s) {
                const int b = s & 1;
                if (!mbar_wait(smem_u32(&s_op[b]), (uint32_t)(s >> 1) & 1u)) {
                    *bad = 1;
                    break;
                }
                tc_fence_after();
                if (s + kAtcRawStages < n_st) issue(s + kAtcRawStages);   // row stage s is consumed
                const uint32_t hb = smem_u32(ops + 2 * b * kAtcOpBytes), lb = hb + kAtcOpBytes;
                for (int ks = 0; ks < kAtcK / 8; ++ks) {
                    const uint32_t o = ks * 2 * kLbo;
                    const int acc = (s > 0 || ks > 0) ? 1 : 0;
                    const uint64_t h0 = smem_desc(hb + o, kLbo, kAtcSbo), l0 = smem_desc(lb + o, kLbo, kAtcSbo);
                    mma_tf32(tmem, h0, h0, id0, acc);
                    mma_tf32(tmem, l0, h0, id0, 1);
                    mma_tf32(tmem, h0, l0, id0, 1);
                    if (two) {
                        const uint64_t ha = smem_desc(hb + oa + o, kLbo, kAtcSbo);
                        const uint64_t la = smem_desc(lb + oa + o, kLbo, kAtcSbo);
                        const uint64_t hbb = smem_desc(hb + ob + o, kLbo, kAtcSbo);
                        const uint64_t lbb = smem_desc(lb + ob + o, kLbo, kAtcSbo);
                        mma_tf32(tmem + 256, ha, hbb, id1, acc);
                        mma_tf32(tmem + 256, la, hbb, id1, 1);
                        mma_tf32(tmem + 256, ha, lbb, id1, 1);
                    }
                }
                mma_commit(smem_u32(&s_done[b]));
                last_commit = s;
            }
        }
    } else {
        // warp w < 14 splits rows 32 (w % 7) .. +31, one row per lane, and the
        // patch groups 4 (w / 7) .. +3 (4 patches each): a lane writes each of
        // its rows' core-matrix rows (4 patches, 16 bytes) of hi and of lo with
        // one store; warps 14 and 15 only arrive
        const int rc = warp % 7, kh = warp / 7, m = 32 * rc + lane;
        const bool row_ok = warp < kAtcRowWarps && m < kAtcOpRows, mv = row_ok && m < n6;
        const int src = mv ? atc_src(m) : 0;
        const uint32_t off_m = (uint32_t)(m >> 3) * kAtcSbo + (uint32_t)(m & 7) * 16u;
        for (int s = 0; s < n_st; ++s) {
            const int b = s & 1;
            bool ok = !*bad && mbar_wait(smem_u32(&s_full[s % kAtcRawStages]), (uint32_t)(s / kAtcRawStages) & 1u);
            if (ok && s >= 2) ok = mbar_wait(smem_u32(&s_done[b]), (uint32_t)((s - 2) >> 1) & 1u);   // buffer b read
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) *bad = 1;
                break;
            }
            const float *raw = raw0 + (s % kAtcRawStages) * raw_len;
            const int rows = min(kAtcK, k_hi - (k_lo + s * kAtcK));
            unsigned char *hi = ops + 2 * b * kAtcOpBytes, *lo = hi + kAtcOpBytes;
            if (row_ok) {
                // v' of row m: this lane's 16 patches in FP32, then a compensated add
                // across stages (the other half of the patches is summed by warp w + 7)
                float blk = 0.f;
#pragma unroll
                for (int kq = 0; kq < kAtcK / 8; ++kq) {
                    const int kg = (kAtcK / 8) * kh + kq;
                    uint32_t hv[4], lv[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int k = 4 * kg + j;
                        const bool in = mv && k < rows;
                        const float x = in ? raw[k * RS + src] : 0.f;
                        blk = fmaf(-(in ? raw[k * RS + 8 * nf] : 0.f), x, blk);
                        hv[j] = tf32_rna(x);
                        lv[j] = tf32_rna(x - __uint_as_float(hv[j]));
                    }
                    const uint32_t off = off_m + (uint32_t)kg * kLbo;
                    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                }
                kahan_add(v_s, v_c, blk);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&s_op[b]));
        }
    }
    if (warp >= 7 && warp < kAtcRowWarps && 32 * (warp - 7) + lane < n6)
        s_vh[32 * (warp - 7) + lane] = (double)v_s - (double)v_c;
    __syncthreads();
    if (!s_bad && !mbar_wait(smem_u32(&s_done[(n_st - 1) & 1]), (uint32_t)((n_st - 1) >> 1) & 1u))
        atomicOr(&s_bad, 1);
    __syncthreads();
    if (!s_bad) {
        if (warp < 7 && 32 * warp + lane < n6)
            out[36 * np + 32 * warp + lane] = (double)v_s - (double)v_c + s_vh[32 * warp + lane];
        // read-back: warp w reads TMEM lanes 32 (w % 4) .. +31 (m) and every
        // fourth 16-column chunk from chunk w / 4 of the N0 columns from 0
        // and the N1 columns from 256
        tc_fence_after();
        const int m = 32 * (warp & 3) + lane;
        const int n_ch0 = N0 / 16, n_ch = n_ch0 + N1 / 16;
        for (int j = warp >> 2; j < n_ch && warp < kAtcSplitWarps; j += kAtcSplitWarps / 4) {
            const bool r1 = j >= n_ch0;
            const int c0 = r1 ? 256 + 16 * (j - n_ch0) : 16 * j;
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + c0, v);
            const int R = r1 ? a0 + m : m;
            if (R >= n6 || (r1 && R < 128)) continue;
            const int fr = R / 6, ir = R - 6 * fr;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int C = r1 ? kAtcB0 + (c0 - 256) + q : c0 + q;
                const int fc = C / 6;
                if (C < n6 && fr <= fc)
                    out[36 * (fr * nf - fr * (fr - 1) / 2 + (fc - fr)) + 6 * ir + (C - 6 * fc)] = -(double)v[q];
            }
        }
    } else if (warp == kAtcSplitWarps && lane == 0) {
        // report, and give the copies and MMAs in flight a bounded wait before the TMEM is freed
        atomicOr(pr.status, DPVO_BA_STATUS_TIMEOUT);
        for (int u = n_issued > kAtcRawStages ? n_issued - kAtcRawStages : 0; u < n_issued; ++u)
            mbar_wait(smem_u32(&s_full[u % kAtcRawStages]), (uint32_t)(u / kAtcRawStages) & 1u);
        if (last_commit >= 0) mbar_wait(smem_u32(&s_done[last_commit & 1]), (uint32_t)(last_commit >> 1) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kAtcCols);
}

}  // namespace dpvo
