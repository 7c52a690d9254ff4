// Correlation features of the update operator (Sec. 3.2 "Correlation", Eq. 4;
// Appendix "Correlation Operation").
//
// For an edge (k, j), a pixel q of patch k at level-l coordinates (x, y) has
// the 7 x 7 grid C[a][b] = <g_q, f(x + b - 3, y + a - 3)>, f bilinear.  With
// x0 = floor(x), wx = x - x0 (same for y), every sample has the weights of the
// grid's corner, so by linearity
//   C[a][b] = (1-wy)(1-wx) D[a][b] + (1-wy) wx D[a][b+1] + wy (1-wx) D[a+1][b] + wy wx D[a+1][b+1]
// with D[m][n] = <g_q, f[y0 - 3 + m][x0 - 3 + n]> on the 8 x 8 integer window.
// The 9 windows of a patch lie in one bounding box of footprint pixels; all
// footprint x patch-pixel products are one GEMM, M = footprint pixels (chunks of
// 128), N = 16 (9 patch pixels, zero-padded), K = 128 channels, BF16 operands
// staged in shared memory (zero outside the map) -- by TMA box loads for edges
// whose footprints fit the fixed boxes, else by 16-byte asynchronous copies --
// and multiplied by tcgen05.mma.kind::f16 into an FP32 accumulator in TMEM.  The epilogue reads the accumulator back, and forms the 49 outputs of
// each patch pixel and level from shared memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "dpvo_ba.h"
#include "tc.cuh"

namespace dpvo_corr {

using dpvo::kLbo;
using dpvo::smem_u32;

constexpr int kThreads = 128;                   // 4 warps: TMEM lanes 0..127
constexpr int kD = DPVO_BA_CORR_DIM;            // channels
constexpr int kQ = 9;                           // patch pixels (3 x 3)
constexpr int kChunk = 128;                     // footprint pixels per MMA (M)
constexpr int kN = 16;                          // patch pixels padded (N)
constexpr int kMaxChunks = 2;                   // general path: footprints up to 256 pixels on the tensor cores
constexpr uint32_t kSbo = (kD / 8) * kLbo + 16; // bytes between 8-row groups (16 core matrices of K, +16 so
                                                 // that the row groups a warp writes fall in distinct banks)
constexpr int kRows1 = 88;                      // level-1 fast footprints: at most 88 pixels (11 row groups)
constexpr uint32_t kAbytes = (kChunk / 8) * kSbo, kA1bytes = (kRows1 / 8) * kSbo, kBbytes = (kN / 8) * kSbo;
constexpr int kDld = kQ;                        // row stride (floats) of the accumulator copy
// Dynamic shared memory: A0 (128 rows), A1 (88 rows), B (16 rows), the accumulator copies
// (128 + 88 rows).  The level-1 GEMM reads 128 rows from A1: rows 88..127 fall on B and the
// copies (inside the allocation), and their results are never read.  3 CTAs per SM.
constexpr size_t kSmemBytes = kAbytes + kA1bytes + kBbytes + (size_t)(kChunk + kRows1) * kDld * 4;
static_assert(kA1bytes + kBbytes + (size_t)(kChunk + kRows1) * kDld * 4 >= kAbytes,
              "the level-1 GEMM's 128 operand rows stay inside the allocation");
// Fast edges load their footprints by TMA: one fixed box per level (level 0
// 11 x 11 pixels, level 1 9 x 9) per 64-channel half, with 128-byte swizzling:
// box-pixel rows of 128 bytes (row t = y * width + x), 16-byte pieces permuted
// within each 1024-byte group of 8 rows -- the canonical K-major operand with
// 128-byte swizzling, whose 8-row groups are 1024 bytes apart.  A level's two
// halves (channels 0-63, 64-127) are kHalf0 / kHalf1 bytes apart; an MMA's
// K = 16 slice starts 32 bytes further along the row.  The fast operands sit
// in the first kAbytes + kA1bytes of shared memory (A0f at 0, A1f at kA1f),
// which must then start on 1024 bytes.  Out-of-map pixels read as zero.
constexpr int kBoxW0 = 11, kBoxH0 = 11, kBoxW1 = 9, kBoxH1 = 9;
constexpr int kHalfC = 64;                                  // channels per box
constexpr uint32_t kHalf0 = kChunk * 128, kHalf1 = kRows1 * 128, kA1f = 2 * kHalf0;
constexpr uint32_t kTmaBytes = 2 * kHalfC * 2 * (kBoxW0 * kBoxH0 + kBoxW1 * kBoxH1);
static_assert(kBoxW0 * kBoxH0 <= kChunk && kBoxW1 * kBoxH1 <= kRows1, "boxes fit their operands");
static_assert(kHalf1 % 1024 == 0 && kA1f % 1024 == 0, "the swizzled halves start on 1024 bytes");
static_assert(kA1f + kHalf1 + kChunk * 128 <= kAbytes + kA1bytes,
              "the level-1 GEMM's 128 rows of either half stay inside A0 and A1");

// Shared-memory descriptor of a K-major operand with 128-byte swizzling:
// 8-row groups 1024 bytes apart (the leading offset is unused), version 1.
__device__ __forceinline__ uint64_t swz128_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kChunk >> 4) << 24);   // FP32 D, BF16 A and B, K-major, 128 x 16
constexpr float kCoordMax = 1e4f;

// Byte offset of (row r, channel c) in the K-major no-swizzle operand layout.
__device__ __forceinline__ uint32_t op_off(int r, int c) {
    return (uint32_t)(r >> 3) * kSbo + (uint32_t)(c >> 3) * kLbo + (uint32_t)(r & 7) * 16u + (uint32_t)(c & 7) * 2u;
}

// 16-byte asynchronous copy global -> shared; src_bytes 0 writes zeros.
__device__ __forceinline__ void cp16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ float bf16_to_f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

struct Args {
    CUtensorMap tm[2];                            // the two levels' feature maps ([N][H][W][128] bf16)
    const uint16_t *fmap[2], *gpatch;
    const int32_t *kk, *jj;
    const float *coords;
    float *corr;
    int32_t *status;
    int E, N, P, H[2], W[2];
    float scale1;
    int use_tma;                                  // tensor maps encoded: fast edges load by TMA
};

// Per-edge plan, double-buffered across the pipeline: patch, frame, the two
// levels' coordinates and footprint boxes, and the edge's mode.
enum Mode { kZero = 0, kFast = 1, kGeneral = 2, kBadIndex = 3 };
struct Plan {
    float xy[2][kQ][2];
    int box[2][4];                               // fx0, fy0, w, h per level
    int k, j, mode;
};

// Warp 0: plan edge e (coordinates, boxes, mode).
__device__ void plan_edge(const Args &A, int e, Plan &P, int lane, bool tma_ok) {
    const int k = A.kk[e], j = A.jj[e];
    const bool valid = k >= 0 && k < A.P && j >= 0 && j < A.N;
    bool finite = true;
    int npix[2] = {0, 0};
    for (int l = 0; l < 2; ++l) {
        const float s = l == 0 ? 1.f : A.scale1;
        float xs = 0.f, ys = 0.f;
        if (lane < kQ) {
            xs = A.coords[((size_t)e * kQ + lane) * 2] / s;
            ys = A.coords[((size_t)e * kQ + lane) * 2 + 1] / s;
            P.xy[l][lane][0] = xs;
            P.xy[l][lane][1] = ys;
        }
        const bool ok = lane >= kQ || (fabsf(xs) <= kCoordMax && fabsf(ys) <= kCoordMax);
        finite = finite && __all_sync(0xffffffffu, ok);
        const int xi = lane < kQ && ok ? (int)floorf(xs) : 0, yi = lane < kQ && ok ? (int)floorf(ys) : 0;
        const int x0 = __reduce_min_sync(0xffffffffu, lane < kQ ? xi : 0x7fffffff);
        const int x1 = __reduce_max_sync(0xffffffffu, lane < kQ ? xi : -0x7fffffff);
        const int y0 = __reduce_min_sync(0xffffffffu, lane < kQ ? yi : 0x7fffffff);
        const int y1 = __reduce_max_sync(0xffffffffu, lane < kQ ? yi : -0x7fffffff);
        if (lane == 0) {
            P.box[l][0] = x0 - 3;
            P.box[l][1] = y0 - 3;
            P.box[l][2] = x1 - x0 + 8;
            P.box[l][3] = y1 - y0 + 8;
        }
        npix[l] = (x1 - x0 + 8) * (y1 - y0 + 8);
    }
    if (lane == 0) {
        P.k = k;
        P.j = j;
        const bool fits = tma_ok && P.box[0][2] <= kBoxW0 && P.box[0][3] <= kBoxH0 && P.box[1][2] <= kBoxW1 &&
                          P.box[1][3] <= kBoxH1;
        P.mode = !valid ? kBadIndex : !finite ? kZero : fits ? kFast : kGeneral;
        if (P.mode == kFast) {   // the fixed boxes from the same corners
            P.box[0][2] = kBoxW0; P.box[0][3] = kBoxH0;
            P.box[1][2] = kBoxW1; P.box[1][3] = kBoxH1;
        }
    }
}

// All threads: stage rows t = t0 .. t0 + nrows - 1 of a footprint box of map
// fm into the operand at aOp (nrows rows of capacity), one row (pixel: 16
// copies of 8 channels) per thread; rows outside the box or the map are zero.
__device__ __forceinline__ void stage_footprint(uint32_t aOp, const uint16_t *fm, int H, int W, const int *box,
                                                int t0, int nrows, int tid) {
    const int w = box[2], npix = w * box[3];
    for (int r = tid; r < nrows; r += kThreads) {
        const int t = t0 + r;
        const int py = box[1] + t / w, px = box[0] + t % w;
        const bool in = t < npix && py >= 0 && py < H && px >= 0 && px < W;
        const uint16_t *src = in ? fm + ((size_t)py * W + px) * kD : fm;
        const uint32_t dst = aOp + (uint32_t)(r >> 3) * kSbo + (uint32_t)(r & 7) * 16u, nb = in ? 16u : 0u;
#pragma unroll
        for (int g = 0; g < kD / 8; ++g) cp16(dst + g * kLbo, src + (in ? 8 * g : 0), nb);
    }
}

__device__ __forceinline__ void stage_patch(uint32_t aB, const uint16_t *gpatch, int k, int tid) {
    for (int idx = tid; idx < kQ * (kD / 8); idx += kThreads) {
        const int r = idx / (kD / 8), g = idx % (kD / 8);
        cp16(aB + op_off(r, 8 * g), gpatch + ((size_t)k * kQ + r) * kD + 8 * g, 16u);
    }
}

// The 7 outputs b = 0..6 of grid row a, patch pixel q, level l, from an
// accumulator copy D (row t of the footprint at D[t * kDld + q]) or from
// per-pixel 8 x 8 windows (Dw[64 q + 8 m + n]), to out[0..6].
__device__ __forceinline__ void bilinear_row(const Plan &P, int l, int q, int a, const float *D, const float *Dw,
                                             float *out) {
    const float x = P.xy[l][q][0], y = P.xy[l][q][1];
    const float xf = floorf(x), yf = floorf(y), wx = x - xf, wy = y - yf;
    float r0[8], r1[8];                           // window rows a and a + 1, columns 0..7
    if (D) {
        const int w = P.box[l][2];
        const int t = ((int)yf - 3 + a - P.box[l][1]) * w + ((int)xf - 3 - P.box[l][0]);
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            r0[n] = D[(t + n) * kDld + q];
            r1[n] = D[(t + w + n) * kDld + q];
        }
    } else {
        const float *Dq = Dw + 64 * q + 8 * a;
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            r0[n] = Dq[n];
            r1[n] = Dq[8 + n];
        }
    }
#pragma unroll
    for (int b = 0; b < 7; ++b)
        out[b] = (1.f - wy) * ((1.f - wx) * r0[b] + wx * r0[b + 1]) + wy * ((1.f - wx) * r1[b] + wx * r1[b + 1]);
}

// One CTA of 4 warps takes edges blockIdx.x, + gridDim.x, ...  Fast edges
// (both levels' footprints within one 128-pixel chunk): both footprints and the
// patch are staged together, the two GEMMs run under one commit, and the next
// edge's copies are issued before this edge's epilogue.  Other edges: level by
// level, chunk by chunk, or on the CUDA cores when the footprint exceeds
// kMaxChunks chunks.
// One thread: one box of a level's tensor map into shared memory, counted on mbar.
__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap *tm, int c, int x, int y, int f,
                                        uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(c), "r"(x), "r"(y), "r"(f), "r"(mbar)
        : "memory");
}

__global__ void __launch_bounds__(kThreads) corr_kernel(const __grid_constant__ Args A) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *opA0 = smem, *opA1 = smem + kAbytes, *opB = smem + kAbytes + kA1bytes;
    float *Dfast = reinterpret_cast<float *>(smem + kAbytes + kA1bytes + kBbytes);   // rows 0..127 level 0, then level 1
    float *Dgen = reinterpret_cast<float *>(opA1);   // general path (up to kMaxChunks x 128 rows), over A1 .. copies
    __shared__ __align__(8) uint64_t s_mbar, s_tma;
    __shared__ uint32_t s_tmem;
    __shared__ Plan s_plan[2];
    __shared__ int s_bad, s_badin;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t aA0 = smem_u32(opA0), aA1 = smem_u32(opA1), aB = smem_u32(opB), mbar = smem_u32(&s_mbar);
    const uint32_t tbar = smem_u32(&s_tma);
    const bool tma_ok = A.use_tma && (aA0 & 1023u) == 0;   // the swizzled box destinations start on 1024 bytes
    if (warp == 0) dpvo::tmem_alloc(&s_tmem, 32);
    if (tid == 0) {
        dpvo::mbar_init(mbar, 1);
        dpvo::mbar_init(tbar, 1);
        s_bad = 0;
        s_badin = 0;
    }
    for (int idx = tid; idx < (kN - kQ) * (kD / 8); idx += kThreads) {   // rows 9..15 of B stay zero
        const int r = kQ + idx / (kD / 8), g = idx % (kD / 8);
        *reinterpret_cast<uint4 *>(opB + op_off(r, 8 * g)) = make_uint4(0u, 0u, 0u, 0u);
    }
    dpvo::tc_fence_before();
    __syncthreads();
    dpvo::tc_fence_after();
    const uint32_t tmem = s_tmem;
    int n_commit = 0, slot = 0, n_tma = 0, n_tma_done = 0;   // the same in every thread

    auto fmap_of = [&](int l, int j) { return A.fmap[l] + (size_t)j * A.H[l] * A.W[l] * kD; };
    auto issue_fast = [&](const Plan &P) {   // after a barrier that follows a proxy fence
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tbar), "r"(kTmaBytes)
                         : "memory");
            for (int h = 0; h < 2; ++h) {
                tma_box(aA0 + h * kHalf0, &A.tm[0], kHalfC * h, P.box[0][0], P.box[0][1], P.j, tbar);
                tma_box(aA0 + kA1f + h * kHalf1, &A.tm[1], kHalfC * h, P.box[1][0], P.box[1][1], P.j, tbar);
            }
        }
        ++n_tma;
        stage_patch(aB, A.gpatch, P.k, tid);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    int e = blockIdx.x;
    if (e < A.E) {
        if (warp == 0) plan_edge(A, e, s_plan[0], lane, tma_ok);
        __syncthreads();
        if (s_plan[0].mode == kFast) issue_fast(s_plan[0]);
    }
    for (; e < A.E; e += gridDim.x) {
        Plan &P = s_plan[slot];
        const int mode = P.mode;
        float *out = A.corr + (size_t)e * 2 * kQ * 49;
        // warp 0 plans the next edge now, while this edge's boxes land (its
        // plan slot was freed by the last barrier of the previous edge)
        const int en = e + gridDim.x;
        if (en < A.E && warp == 0) plan_edge(A, en, s_plan[slot ^ 1], lane, tma_ok);
        if (mode == kFast) {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            if (!dpvo::mbar_wait(tbar, (uint32_t)(n_tma - 1) & 1u)) atomicOr(&s_bad, 1);
            else n_tma_done = n_tma;
            dpvo::fence_async_smem();
            __syncthreads();
            if (s_bad == 0) {
                if (tid == 0) {
                    dpvo::tc_fence_after();
                    for (int ks = 0; ks < kD / 16; ++ks)   // K slice ks: half ks / 4, 32 bytes per slice
                        mma_bf16(tmem, swz128_desc(aA0 + (ks >> 2) * kHalf0 + (ks & 3) * 32),
                                 dpvo::smem_desc(aB + ks * 2 * kLbo, kLbo, kSbo), ks > 0 ? 1 : 0);
                    for (int ks = 0; ks < kD / 16; ++ks)
                        mma_bf16(tmem + kN, swz128_desc(aA0 + kA1f + (ks >> 2) * kHalf1 + (ks & 3) * 32),
                                 dpvo::smem_desc(aB + ks * 2 * kLbo, kLbo, kSbo), ks > 0 ? 1 : 0);
                    dpvo::mma_commit(mbar);
                }
                ++n_commit;
                if (!dpvo::mbar_wait(mbar, (uint32_t)(n_commit - 1) & 1u)) atomicOr(&s_bad, 1);
            }
            __syncthreads();
            if (s_bad == 0) {
                dpvo::tc_fence_after();
                float v[16];
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    dpvo::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + kN * l, v);
                    if (l == 0 || tid < kRows1) {
#pragma unroll
                        for (int q = 0; q < kQ; ++q) Dfast[(l * kChunk + tid) * kDld + q] = v[q];
                    }
                }
            }
            dpvo::tc_fence_before();
            __syncthreads();                             // operands free, accumulators copied
        } else if (mode == kGeneral && s_bad == 0) {
            for (int l = 0; l < 2; ++l) {
                const int H = A.H[l], W = A.W[l];
                const uint16_t *fm = fmap_of(l, P.j);
                const int npix = P.box[l][2] * P.box[l][3];
                const int nch = (npix + kChunk - 1) / kChunk;
                if (l == 0) stage_patch(aB, A.gpatch, P.k, tid);
                if (nch <= kMaxChunks) {
                    for (int c = 0; c < nch; ++c) {
                        stage_footprint(aA0, fm, H, W, P.box[l], kChunk * c, kChunk, tid);
                        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
                        dpvo::fence_async_smem();
                        __syncthreads();
                        if (tid == 0) {
                            dpvo::tc_fence_after();
                            for (int ks = 0; ks < kD / 16; ++ks)
                                mma_bf16(tmem, dpvo::smem_desc(aA0 + ks * 2 * kLbo, kLbo, kSbo),
                                         dpvo::smem_desc(aB + ks * 2 * kLbo, kLbo, kSbo), ks > 0 ? 1 : 0);
                            dpvo::mma_commit(mbar);
                        }
                        ++n_commit;
                        if (!dpvo::mbar_wait(mbar, (uint32_t)(n_commit - 1) & 1u)) atomicOr(&s_bad, 1);
                        __syncthreads();
                        if (s_bad) break;
                        dpvo::tc_fence_after();
                        float v[16];
                        dpvo::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16), v);
                        const int t = kChunk * c + tid;
                        if (t < npix) {
#pragma unroll
                            for (int q = 0; q < kQ; ++q) Dgen[t * kDld + q] = v[q];
                        }
                        dpvo::tc_fence_before();
                        __syncthreads();
                    }
                } else {
                    // windows too far apart: each patch pixel's 8 x 8 inner products on the CUDA cores
                    for (int idx = tid; idx < kQ * 64; idx += kThreads) {
                        const int q = idx >> 6, m = (idx >> 3) & 7, n = idx & 7;
                        const int py = (int)floorf(P.xy[l][q][1]) - 3 + m, px = (int)floorf(P.xy[l][q][0]) - 3 + n;
                        float acc = 0.f;
                        if (py >= 0 && py < H && px >= 0 && px < W) {
                            const uint16_t *f = fm + ((size_t)py * W + px) * kD;
                            const uint16_t *g = A.gpatch + ((size_t)P.k * kQ + q) * kD;
                            for (int c = 0; c < kD; ++c) acc = fmaf(bf16_to_f(g[c]), bf16_to_f(f[c]), acc);
                        }
                        Dgen[idx] = acc;
                    }
                    __syncthreads();
                }
                for (int task = tid; task < kQ * 7; task += kThreads) {
                    const int q = task / 7, a = task - 7 * q;
                    float *o = out + (l * kQ + q) * 49 + 7 * a;
                    if (s_bad) {
                        for (int b = 0; b < 7; ++b) o[b] = 0.f;
                    } else {
                        bilinear_row(P, l, q, a, nch <= kMaxChunks ? Dgen : nullptr, Dgen, o);
                    }
                }
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                __syncthreads();
            }
        }
        // start the next edge's copies (they fly during this epilogue)
        if (en < A.E) {
            dpvo::fence_async_smem();                    // this CTA's generic writes before the next copies
            __syncthreads();
            if (s_plan[slot ^ 1].mode == kFast && s_bad == 0) issue_fast(s_plan[slot ^ 1]);
        }
        if (mode == kFast) {
            for (int task = tid; task < 2 * kQ * 7; task += kThreads) {   // (level, pixel, grid row)
                const int l = task / (kQ * 7), r = task - l * kQ * 7, q = r / 7, a = r - 7 * q;
                float *o = out + (l * kQ + q) * 49 + 7 * a;
                if (s_bad) {
                    for (int b = 0; b < 7; ++b) o[b] = 0.f;
                } else {
                    bilinear_row(P, l, q, a, Dfast + l * kChunk * kDld, nullptr, o);
                }
            }
        } else if (mode == kZero || mode == kBadIndex || s_bad) {
            if (mode != kGeneral || s_bad)
                for (int o = tid; o < 2 * kQ * 49; o += kThreads) out[o] = 0.f;
            if (mode == kBadIndex && tid == 0) s_badin = 1;
        }
        __syncthreads();                                 // this edge's plan and accumulator copy are consumed
        slot ^= 1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        if (n_tma > n_tma_done) dpvo::mbar_wait(tbar, (uint32_t)(n_tma - 1) & 1u);   // a box load still in flight
        if (s_bad) {
            // report, and give the last commit one more bounded wait before the TMEM is freed
            atomicOr(A.status, DPVO_BA_STATUS_TIMEOUT);
            if (n_commit > 0) dpvo::mbar_wait(mbar, (uint32_t)(n_commit - 1) & 1u);
        }
        if (s_badin) atomicOr(A.status, DPVO_BA_STATUS_BAD_INPUT);
    }
    dpvo::tc_fence_before();
    __syncthreads();
    if (warp == 0) dpvo::tmem_dealloc(tmem, 32);
}

// Host: the tensor maps of both levels ([N][H][W][128] bfloat16, 16-byte
// aligned: checked by the entry point), boxes of 64 channels x the level's
// fixed box with 128-byte swizzling; false if the driver entry point is
// missing or rejects them.
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static bool encode_maps(Args &A) {
    static EncodeTiled encode = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<EncodeTiled>(fn);
        else
            cudaGetLastError();
    }
    if (!encode) return false;
    for (int l = 0; l < 2; ++l) {
        if (reinterpret_cast<uintptr_t>(A.fmap[l]) & 15) return false;
        const cuuint64_t W = (cuuint64_t)A.W[l], H = (cuuint64_t)A.H[l];
        const cuuint64_t dims[4] = {(cuuint64_t)kD, W, H, (cuuint64_t)A.N};
        const cuuint64_t strides[3] = {(cuuint64_t)kD * 2, W * kD * 2, H * W * kD * 2};
        const cuuint32_t box[4] = {(cuuint32_t)kHalfC, (cuuint32_t)(l == 0 ? kBoxW0 : kBoxW1),
                                   (cuuint32_t)(l == 0 ? kBoxH0 : kBoxH1), 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        if (encode(&A.tm[l], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(A.fmap[l]), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

}  // namespace dpvo_corr

extern "C" int dpvo_ba_correlation(const dpvo_ba_corr_dims *d, const void *fmap0, const void *fmap1,
                                   const void *gpatch, const int32_t *kk, const int32_t *jj, const float *coords,
                                   float *corr, int32_t *status, void *stream) {
    if (!d || d->n_frames < 1 || d->n_patches < 0 || d->n_edges < 0 || d->height < 1 || d->width < 1 ||
        d->height > 4096 || d->width > 4096 || d->level1_scale < 1 || !status)
        return DPVO_BA_EINVAL;
    if (d->n_edges > 0 && (!fmap0 || !fmap1 || !gpatch || !kk || !jj || !coords || !corr)) return DPVO_BA_EINVAL;
    if ((reinterpret_cast<uintptr_t>(fmap0) | reinterpret_cast<uintptr_t>(fmap1) | reinterpret_cast<uintptr_t>(gpatch)) & 15)
        return DPVO_BA_EINVAL;   // features are read in 16-byte pieces
    const int H1 = d->height / d->level1_scale, W1 = d->width / d->level1_scale;
    if (H1 < 1 || W1 < 1) return DPVO_BA_EINVAL;
    if (d->n_edges == 0) return 0;
    static int configured_device = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DPVO_BA_ECUDA;
    const size_t smem = dpvo_corr::kSmemBytes;
    if (configured_device != dev) {
        if (cudaFuncSetAttribute(dpvo_corr::corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return DPVO_BA_ECUDA;
        configured_device = dev;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    dpvo_corr::Args A;
    A.fmap[0] = static_cast<const uint16_t *>(fmap0);
    A.fmap[1] = static_cast<const uint16_t *>(fmap1);
    A.gpatch = static_cast<const uint16_t *>(gpatch);
    A.kk = kk;
    A.jj = jj;
    A.coords = coords;
    A.corr = corr;
    A.status = status;
    A.E = d->n_edges;
    A.N = d->n_frames;
    A.P = d->n_patches;
    A.H[0] = d->height;
    A.W[0] = d->width;
    A.H[1] = H1;
    A.W[1] = W1;
    A.scale1 = (float)d->level1_scale;
    A.use_tma = dpvo_corr::encode_maps(A) ? 1 : 0;   // else every edge takes the general path
    const int grid = d->n_edges < 3 * sms ? d->n_edges : 3 * sms;
    dpvo_corr::corr_kernel<<<grid, dpvo_corr::kThreads, smem, reinterpret_cast<cudaStream_t>(stream)>>>(A);
    return cudaGetLastError() == cudaSuccess ? 0 : DPVO_BA_ECUDA;
}
