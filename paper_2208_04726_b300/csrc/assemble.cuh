// Schur assembly for reduced systems with more free poses than the linearise
// kernel's strip owners hold in registers (Sec. 3.1, the Schur complement over
// the inverse depths):
//     S  -= sum_k (C_k^-1/2 e_k)(C_k^-1/2 e_k)^T,   v' -= sum_k (C_k^-1/2 e_k)(C_k^-1/2 w_k),
// read from the rows C_k^-1/2 (e_k, w_k, 1) the linearise kernel stores for the
// back-substitution, into FP64 partials in the strip layout of (S, v').
//
// One CTA per (problem, work item, slice): it takes a range of chunks, and
// each compute thread one 6 x 6 pose-pair block (a, b), a <= b, in
// registers; a warp holds a 4 x 8 block of frame pairs (rows a, columns b),
// so that its operand loads from shared memory mostly coincide, and whole
// warps skip a chunk whose frame window misses their frames.  The right-hand
// side v' has warps of its own (a lane per free pose).
//
// Rows stream through kAsmStages shared-memory stages of up to
// kAsmStageRows patches (a chunk takes one or more stages).  One producer
// warp issues a bulk asynchronous copy per stage once every compute warp has
// released the stage (its "empty" mbarrier); a compute warp waits for the
// stage's copy (its "full" mbarrier), sums it or skips it, and releases it.
// No block-wide barrier inside the loop: each warp moves at the pace of its
// own work, up to kAsmStages stages ahead of the slowest.  Every wait is
// bounded; on a timeout the CTA reports DPVO_BA_STATUS_TIMEOUT, waits (again
// bounded) for its copies in flight and leaves.
//
// Sums: FP32 over blocks of kFlushEvery patches (a stage's last block may be
// shorter), compensated across blocks (the running sums in registers, their
// compensation terms in shared memory, thread-private), written once as FP64
// in the strip layout (the 6 x 6 block of pair (a, b) row-major at 36 x its
// pair index, then v').
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "ba_common.cuh"
#include "tc.cuh"

namespace dpvo {

constexpr int kAsmMaxWarps = 11;               // compute warps per CTA at most (6 x 6 register blocks)
constexpr int kAsmMaxThreads = 32 * (kAsmMaxWarps + 1);   // + the producer warp
constexpr int kAsmStages = 4;
constexpr int kAsmStageRows = 32;

// One thread: expect `bytes` on the mbarrier's current phase and bulk-copy
// them (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory; the phase completes when they have landed.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
    bulk_copy_g2s(dst, src, bytes, mbar);
}

// Warp blocks: for each column block B (frames 8B .. 8B+7), the row blocks
// of 4 frames that hold a pair a <= b; then ceil(nf / 32) warps for v'.
__host__ __device__ inline int asm_col_warps(int nf, int B) {
    const int last = 8 * B + 7 < nf - 1 ? 8 * B + 7 : nf - 1;
    return last / 4 + 1;
}
__host__ __device__ inline int asm_pair_warps(int nf) {
    int w = 0;
    for (int B = 0; 8 * B < nf; ++B) w += asm_col_warps(nf, B);
    return w;
}
__host__ __device__ inline int asm_warps(int nf) { return asm_pair_warps(nf) + (nf + 31) / 32; }
__host__ __device__ inline int asm_slices(int nf) {
    const int w = asm_warps(nf);
    return w <= 0 ? 1 : (w + kAsmMaxWarps - 1) / kAsmMaxWarps;
}
// Threads per CTA: the compute warps of a slice, then the producer warp.
__host__ __device__ inline int asm_threads(int nf) {
    const int w = asm_warps(nf), sl = asm_slices(nf);
    const int per = (w + sl - 1) / sl;
    return 32 * ((per < 1 ? 1 : per) + 1);
}

// Dynamic shared memory: the stages (kAsmStageRows x rs_max floats each),
// then 36 compensation terms per thread.
__host__ __device__ inline size_t asm_smem_bytes(int rs_max, int threads) {
    return ((size_t)kAsmStages * kAsmStageRows * rs_max + (size_t)36 * threads) * 4;
}

// Shared-memory accesses by 32-bit shared addresses (bytes).
__device__ __forceinline__ float4 lds4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}
__device__ __forceinline__ float lds1(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts4(uint32_t addr, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// Compensated add of a finished block: s += blk (Kahan), for NQ entries
// (a multiple of 4) whose compensation terms sit in shared memory as float4
// groups at c4 + g * gs (bytes); then blk = 0.  Three groups at a time: their
// loads in flight together, the updates independent.
template <int NQ>
__device__ __forceinline__ void flush_block(float *acc_s, float *blk, uint32_t c4, uint32_t gs) {
#pragma unroll
    for (int g0 = 0; g0 < NQ / 4; g0 += 3) {
        float4 cv[3];
#pragma unroll
        for (int g = 0; g < 3; ++g)
            if (g0 + g < NQ / 4) cv[g] = lds4(c4 + (g0 + g) * gs);
#pragma unroll
        for (int g = 0; g < 3; ++g)
            if (g0 + g < NQ / 4) {
                float *b = blk + 4 * (g0 + g), *a = acc_s + 4 * (g0 + g);
                kahan_add(a[0], cv[g].x, b[0]);
                kahan_add(a[1], cv[g].y, b[1]);
                kahan_add(a[2], cv[g].z, b[2]);
                kahan_add(a[3], cv[g].w, b[3]);
                b[0] = b[1] = b[2] = b[3] = 0.f;
            }
#pragma unroll
        for (int g = 0; g < 3; ++g)
            if (g0 + g < NQ / 4) sts4(c4 + (g0 + g) * gs, cv[g]);
    }
}

// One patch's product into a pair block: blk -= e_a e_b^T (6 x 6; ra, rb
// the shared addresses of the padded frame entries a and b of the row).
__device__ __forceinline__ void pair_patch(uint32_t ra, uint32_t rb, float *blk) {
    const float4 a0 = lds4(ra);
    const float4 a1 = lds4(ra + 16);
    const float4 b0 = lds4(rb);
    const float4 b1 = lds4(rb + 16);
    const float ea[6] = {a0.x, a0.y, a0.z, a1.x, a1.y, a1.z};
    const float eb[6] = {b0.x, b0.y, b0.z, b1.x, b1.y, b1.z};
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) blk[6 * r + cc] = fmaf(-ea[r], eb[cc], blk[6 * r + cc]);
}

// Grid: x = assembly work items (Item{prob, item}), y = slices (warp blocks
// dealt round robin).  rs_max bounds the row length; t = iteration.
__global__ void __launch_bounds__(kAsmMaxThreads, 1) schur_assembly_kernel(const Prob *__restrict__ probs,
                                                                           const Item *__restrict__ items, int t,
                                                                           int rs_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Item itm = items[blockIdx.x];
    const Prob &pr = probs[itm.prob];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (t >= pr.iters || block_status(pr.status) != 0) return;
    __shared__ __align__(8) uint64_t s_full[kAsmStages], s_empty[kAsmStages];
    __shared__ int s_bad, s_issued;
    const int n_comp = (int)(blockDim.x >> 5) - 1;         // compute warps; warp n_comp produces

    const int nf = pr.nf, t0 = pr.t0, RS = erow_len(nf);
    const int nbs = 2 * n_block_pairs(nf), npw = asm_pair_warps(nf);
    const int gw = warp * gridDim.y + blockIdx.y;
    int a = -1, b = -1;
    const bool vs = gw >= npw;                             // a right-hand-side warp
    if (warp < n_comp) {
        if (!vs) {
            int rem = gw, B = 0;
            while (rem >= asm_col_warps(nf, B)) rem -= asm_col_warps(nf, B++);
            a = 4 * rem + (lane >> 3);
            b = 8 * B + (lane & 7);
            if (a > b || b >= nf) a = b = -1;
        } else if (gw < npw + (nf + 31) / 32) {
            a = b = 32 * (gw - npw) + lane;
            if (a >= nf) a = b = -1;
        }
    }
    const bool active = a >= 0;
    const int fa = t0 + a, fb = t0 + b;
    const int oa = 8 * a, ob = vs ? 8 * nf : 8 * b;

    const int nch = *pr.n_chunks;
    const int c_begin = (int)(((long long)itm.item * nch) / pr.n_asm);
    const int c_end = (int)(((long long)(itm.item + 1) * nch) / pr.n_asm);
    float *stage0 = reinterpret_cast<float *>(smem);
    const size_t stage_len = (size_t)kAsmStageRows * rs_max;
    if (tid == 0) {
        for (int s = 0; s < kAsmStages; ++s) {
            mbar_init(smem_u32(&s_full[s]), 1);
            mbar_init(smem_u32(&s_empty[s]), n_comp);
        }
        s_bad = 0;
        s_issued = 0;
    }
    // compensation terms, float4 groups: the g-th (entries 4g .. 4g+3) of
    // this thread at acc_c + g * gs (bytes)
    const uint32_t acc_c = smem_u32(stage0 + kAsmStages * stage_len + 4 * tid), gs = 16 * blockDim.x;
#pragma unroll
    for (int g = 0; g < 9; ++g) sts4(acc_c + g * gs, make_float4(0.f, 0.f, 0.f, 0.f));
    __syncthreads();

    volatile int *bad = &s_bad;
    if (warp == n_comp) {
        // producer: one lane issues the stages in order
        if (lane == 0) {
            int u = 0;
            for (int c = c_begin; c < c_end && !*bad; ++c) {
                const Chunk ch = pr.chunks[c];
                for (int r0 = 0; r0 < ch.count; r0 += kAsmStageRows, ++u) {
                    const int s = u % kAsmStages;
                    if (u >= kAsmStages && !mbar_wait(smem_u32(&s_empty[s]), (uint32_t)(u / kAsmStages - 1) & 1u)) {
                        *bad = 1;
                        break;
                    }
                    const int rows = min(kAsmStageRows, ch.count - r0);
                    bulk_load(stage0 + s * stage_len, pr.erow + (size_t)(ch.k0 + r0) * RS, (uint32_t)(rows * RS * 4),
                              smem_u32(&s_full[s]));
                    s_issued = u + 1;
                }
            }
        }
    } else {
        float acc_s[36], blk[36];
#pragma unroll
        for (int q = 0; q < 36; ++q) { acc_s[q] = 0.f; blk[q] = 0.f; }
        int u = 0;
        for (int c = c_begin; c < c_end; ++c) {
            const Chunk ch = pr.chunks[c];
            const bool on = active && fa >= ch.jlo && fa <= ch.jhi && fb >= ch.jlo && fb <= ch.jhi;
            bool stop = false;
            for (int r0 = 0; r0 < ch.count; r0 += kAsmStageRows, ++u) {
                const int s = u % kAsmStages;
                if (*bad || !mbar_wait(smem_u32(&s_full[s]), (uint32_t)(u / kAsmStages) & 1u)) {
                    *bad = 1;
                    stop = true;
                    break;
                }
                const float *rows = stage0 + s * stage_len;
                const int nrow = min(kAsmStageRows, ch.count - r0);
                if (on) {
                    // blocks of kFlushEvery patches (the stage's last one may be shorter)
                    const uint32_t rs4 = 4 * RS;
                    for (int p0 = 0; p0 < nrow; p0 += kFlushEvery) {
                        const uint32_t rb0 = smem_u32(rows) + p0 * rs4;
                        const int m = min(kFlushEvery, nrow - p0);
                        if (!vs) {
                            const uint32_t ra = rb0 + 4 * oa, rb = rb0 + 4 * ob;
                            if (m == kFlushEvery) {
#pragma unroll
                                for (int k = 0; k < kFlushEvery; ++k) pair_patch(ra + k * rs4, rb + k * rs4, blk);
                            } else {
                                for (int k = 0; k < m; ++k) pair_patch(ra + k * rs4, rb + k * rs4, blk);
                            }
                            flush_block<36>(acc_s, blk, acc_c, gs);
                        } else {
                            for (int k = 0; k < m; ++k) {
                                const uint32_t re = rb0 + k * rs4;
                                const float sw = lds1(re + 4 * ob);
                                const float4 a0 = lds4(re + 4 * oa);
                                const float4 a1 = lds4(re + 4 * oa + 16);
                                const float ea[6] = {a0.x, a0.y, a0.z, a1.x, a1.y, a1.z};
#pragma unroll
                                for (int cc = 0; cc < 6; ++cc) blk[cc] = fmaf(-ea[cc], sw, blk[cc]);
                            }
                            flush_block<8>(acc_s, blk, acc_c, gs);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&s_empty[s]));
            }
            if (stop) break;
        }
        if (active && !*bad) {
            double *out = pr.partial + (size_t)(pr.n_items + itm.item) * pr.L;
            if (!vs) {
                double *o = out + 36 * (a * nf - a * (a - 1) / 2 + (b - a));
#pragma unroll
                for (int q = 0; q < 36; ++q) o[q] = (double)acc_s[q] - (double)lds1(acc_c + (q >> 2) * gs + 4 * (q & 3));
            } else {
                double *o = out + 18 * nbs + 6 * a;
#pragma unroll
                for (int q = 0; q < 6; ++q) o[q] = (double)acc_s[q] - (double)lds1(acc_c + (q >> 2) * gs + 4 * (q & 3));
            }
        }
    }
    __syncthreads();
    if (s_bad && tid == 0) {
        // report, and give every copy still in flight a bounded wait before the CTA exits
        atomicOr(pr.status, DPVO_BA_STATUS_TIMEOUT);
        const int iss = s_issued;
        for (int u = iss > kAsmStages ? iss - kAsmStages : 0; u < iss; ++u)
            mbar_wait(smem_u32(&s_full[u % kAsmStages]), (uint32_t)(u / kAsmStages) & 1u);
    }
}

}  // namespace dpvo
