// Schur assembly for reduced systems with more free poses than the linearise
// kernel's strip owners hold in registers (Sec. 3.1, the Schur complement over
// the inverse depths):
//     S  -= sum_k (C_k^-1/2 e_k)(C_k^-1/2 e_k)^T,   v' -= sum_k (C_k^-1/2 e_k)(C_k^-1/2 w_k),
// read from the rows C_k^-1/2 (e_k, w_k, 1) the linearise kernel stores for the
// back-substitution, into FP64 partials in the strip layout of (S, v').
//
// One CTA per (problem, work item, strip slice): it takes a range of chunks
// and one thread per strip (a 3 x 6 half of a pose-pair block, or a pose's
// right-hand side).  A chunk's rows arrive in shared memory by one bulk
// asynchronous copy that completes on an mbarrier, double-buffered so the
// next chunk streams in while this one is summed.  A strip whose frames lie
// outside a chunk's frame window has zero rows there and skips the chunk.
// Sums: FP32 over blocks of kFlushEvery patches (across chunk boundaries),
// compensated across blocks, written once as FP64.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "ba_common.cuh"
#include "tc.cuh"

namespace dpvo {

constexpr int kAsmMaxThreads = 576;            // 2 slices of 544 strips at 32 free poses

// One thread: expect `bytes` on the mbarrier's current phase and bulk-copy
// them (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory; the phase completes when they have landed.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
    bulk_copy_g2s(dst, src, bytes, mbar);
}

// Strips: 2 per block pair (a <= b), then one per free pose.
__host__ __device__ inline int asm_slices(int nf) {
    const int nst = n_strips(nf);
    return nst <= 0 ? 1 : (nst + kAsmMaxThreads - 1) / kAsmMaxThreads;
}
__host__ __device__ inline int asm_threads(int nf) {
    const int nst = n_strips(nf), sl = asm_slices(nf);
    const int per = (nst + sl - 1) / sl;
    return per < 32 ? 32 : (per + 31) & ~31;
}

// Grid: x = assembly work items (Item{prob, item}), y = strip slices.  G_cap
// bounds the patches of a chunk, rs_max the row length; t = iteration.
__global__ void __launch_bounds__(kAsmMaxThreads) schur_assembly_kernel(const Prob *__restrict__ probs,
                                                                        const Item *__restrict__ items, int t,
                                                                        int G_cap, int rs_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Item itm = items[blockIdx.x];
    const Prob &pr = probs[itm.prob];
    const int tid = threadIdx.x;
    if (t >= pr.iters || *pr.status != 0) return;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int s_bad;

    const int nf = pr.nf, t0 = pr.t0, RS = erow_len(nf);
    const int nbs = 2 * n_block_pairs(nf), nst = nbs + nf;
    const int st = blockIdx.y * blockDim.x + tid;
    const bool active = st < nst, vs = st >= nbs;
    int sa = 0, sb = 0, sh = 0;
    if (active) {
        if (!vs) {
            decode_pair(st >> 1, nf, sa, sb);
            sh = st & 1;
        } else {
            sa = sb = st - nbs;
        }
    }
    const int fa = t0 + sa, fb = t0 + sb;
    const int oa = vs ? 8 * sa : 8 * sa + 4 * sh, ob = 8 * sb;

    const int nch = *pr.n_chunks;
    const int c_begin = (int)(((long long)itm.item * nch) / pr.n_asm);
    const int c_end = (int)(((long long)(itm.item + 1) * nch) / pr.n_asm);
    float *buf[2] = {reinterpret_cast<float *>(smem), reinterpret_cast<float *>(smem) + (size_t)G_cap * rs_max};
    const uint32_t bar[2] = {smem_u32(&s_bar[0]), smem_u32(&s_bar[1])};
    if (tid == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        s_bad = 0;
    }
    __syncthreads();
    if (tid == 0)
        for (int c = c_begin; c < c_end && c < c_begin + 2; ++c) {
            const Chunk ch = pr.chunks[c];
            bulk_load(buf[c - c_begin], pr.erow + (size_t)ch.k0 * RS, (uint32_t)(ch.count * RS * 4), bar[c - c_begin]);
        }

    float acc_s[18], acc_c[18], blk[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) { acc_s[q] = 0.f; acc_c[q] = 0.f; blk[q] = 0.f; }
    int issued = c_end - c_begin < 2 ? c_end - c_begin : 2;   // copies started (thread 0's count)
    int waited = 0, since = 0;
    for (int c = c_begin; c < c_end; ++c) {
        const int u = c - c_begin, bi = u & 1;
        if (!mbar_wait(bar[bi], (uint32_t)(u >> 1) & 1u)) atomicOr(&s_bad, 1);
        ++waited;
        __syncthreads();
        if (s_bad) break;                          // a copy never landed: stop, report below
        const Chunk ch = pr.chunks[c];
        const bool win_a = fa >= ch.jlo && fa <= ch.jhi, win_b = fb >= ch.jlo && fb <= ch.jhi;
        if (active && win_a && win_b) {
            const float *rows = buf[bi];
            if (!vs) {
                for (int p = 0; p < ch.count; ++p) {
                    const float *e = rows + (size_t)p * RS;
                    const float4 a4 = *reinterpret_cast<const float4 *>(e + oa);
                    const float4 b0 = *reinterpret_cast<const float4 *>(e + ob);
                    const float4 b1 = *reinterpret_cast<const float4 *>(e + ob + 4);
                    const float ea[3] = {a4.x, a4.y, a4.z};
                    const float eb[6] = {b0.x, b0.y, b0.z, b1.x, b1.y, b1.z};
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
                for (int p = 0; p < ch.count; ++p) {
                    const float *e = rows + (size_t)p * RS;
                    const float sw = e[8 * nf];
                    const float4 a0 = *reinterpret_cast<const float4 *>(e + oa);
                    const float4 a1 = *reinterpret_cast<const float4 *>(e + oa + 4);
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
        }
        __syncthreads();                           // buffer bi is free again
        if (tid == 0 && c + 2 < c_end) {
            const Chunk cn = pr.chunks[c + 2];
            bulk_load(buf[bi], pr.erow + (size_t)cn.k0 * RS, (uint32_t)(cn.count * RS * 4), bar[bi]);
            ++issued;
        }
    }
    if (s_bad) {
        // report, and give every copy this CTA started a bounded wait before it exits
        if (tid == 0) {
            atomicOr(pr.status, DPVO_BA_STATUS_TIMEOUT);
            for (int u = waited - 1; u < issued; ++u) mbar_wait(bar[u & 1], (uint32_t)(u >> 1) & 1u);
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < 18; ++q) kahan_add(acc_s[q], acc_c[q], blk[q]);
    if (active) {
        double *out = pr.partial + (size_t)(pr.n_items + itm.item) * pr.L;
        if (!vs) {
            double *o = out + 18 * st;
#pragma unroll
            for (int q = 0; q < 18; ++q) o[q] = (double)acc_s[q] - (double)acc_c[q];
        } else {
            double *o = out + 18 * nbs + 6 * sa;
#pragma unroll
            for (int q = 0; q < 6; ++q) o[q] = (double)acc_s[q] - (double)acc_c[q];
        }
    }
}

}  // namespace dpvo
