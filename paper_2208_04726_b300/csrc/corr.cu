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
// staged in shared memory by 16-byte asynchronous copies (zero outside the
// map) and multiplied by tcgen05.mma.kind::f16 into an FP32 accumulator in
// TMEM.  The epilogue reads the accumulator back, and forms the 49 outputs of
// each patch pixel and level from shared memory.
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
constexpr int kMaxChunks = 4;
constexpr uint32_t kSbo = (kD / 8) * kLbo;      // bytes between 8-row groups (16 core matrices of K)
constexpr uint32_t kAbytes = (kChunk / 8) * kSbo, kBbytes = (kN / 8) * kSbo;
constexpr int kDld = 17;                        // row stride (floats) of the accumulator copy
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
    const uint16_t *fmap[2], *gpatch;
    const int32_t *kk, *jj;
    const float *coords;
    float *corr;
    int32_t *status;
    int E, N, P, H[2], W[2];
    float scale1;
};

__global__ void __launch_bounds__(kThreads) corr_kernel(Args A) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *opA = smem, *opB = smem + kAbytes;
    float *Dbuf = reinterpret_cast<float *>(smem + kAbytes + kBbytes);   // kMaxChunks * kChunk x kDld
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ float s_xy[kQ][2];
    __shared__ int s_box[6];                     // fx0, fy0, w, h, mode (0 zeros, 1 tensor, 2 CUDA cores), nchunk
    __shared__ int s_bad, s_badin;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t aA = smem_u32(opA), aB = smem_u32(opB), mbar = smem_u32(&s_mbar);
    if (warp == 0) dpvo::tmem_alloc(&s_tmem, 32);
    if (tid == 0) {
        dpvo::mbar_init(mbar, 1);
        s_bad = 0;
        s_badin = 0;
    }
    // rows 9..15 of the B operand stay zero
    for (int idx = tid; idx < (kN - kQ) * (kD / 8); idx += kThreads) {
        const int r = kQ + idx / (kD / 8), g = idx % (kD / 8);
        *reinterpret_cast<uint4 *>(opB + op_off(r, 8 * g)) = make_uint4(0u, 0u, 0u, 0u);
    }
    dpvo::tc_fence_before();
    __syncthreads();
    dpvo::tc_fence_after();
    const uint32_t tmem = s_tmem;
    int n_commit = 0;

    for (int e = blockIdx.x; e < A.E; e += gridDim.x) {
        const int k = A.kk[e], j = A.jj[e];
        const bool valid = k >= 0 && k < A.P && j >= 0 && j < A.N;   // the same in every thread
        if (!valid) {
            for (int o = tid; o < 2 * kQ * 49; o += kThreads) A.corr[(size_t)e * 2 * kQ * 49 + o] = 0.f;
            if (tid == 0) s_badin = 1;
            continue;
        }
        // the patch's features: B rows 0..8
        for (int idx = tid; idx < kQ * (kD / 8); idx += kThreads) {
            const int r = idx / (kD / 8), g = idx % (kD / 8);
            cp16(aB + op_off(r, 8 * g), A.gpatch + ((size_t)k * kQ + r) * kD + 8 * g, 16u);
        }
        for (int level = 0; level < 2; ++level) {
            const float s = level == 0 ? 1.f : A.scale1;
            const int H = A.H[level], W = A.W[level];
            const uint16_t *fm = A.fmap[level] + (size_t)j * H * W * kD;
            if (tid < kQ) {
                s_xy[tid][0] = A.coords[((size_t)e * kQ + tid) * 2] / s;
                s_xy[tid][1] = A.coords[((size_t)e * kQ + tid) * 2 + 1] / s;
            }
            __syncthreads();
            if (tid == 0) {
                bool ok = s_bad == 0;                // after a timed-out wait: no further MMAs
                int x0 = 1 << 30, x1 = -(1 << 30), y0 = 1 << 30, y1 = -(1 << 30);
                for (int q = 0; q < kQ; ++q) {
                    const float x = s_xy[q][0], y = s_xy[q][1];
                    if (!(fabsf(x) <= kCoordMax && fabsf(y) <= kCoordMax)) ok = false;
                    if (!ok) break;
                    const int xi = (int)floorf(x), yi = (int)floorf(y);
                    x0 = min(x0, xi); x1 = max(x1, xi);
                    y0 = min(y0, yi); y1 = max(y1, yi);
                }
                if (!ok) {
                    s_box[4] = 0;
                } else {
                    const int w = x1 - x0 + 8, h = y1 - y0 + 8;
                    const long long np = (long long)w * h;
                    s_box[0] = x0 - 3; s_box[1] = y0 - 3; s_box[2] = w; s_box[3] = h;
                    s_box[5] = (int)((np + kChunk - 1) / kChunk);
                    s_box[4] = np <= (long long)kMaxChunks * kChunk ? 1 : 2;
                }
            }
            __syncthreads();
            const int mode = s_box[4];
            if (mode == 1) {
                const int fx0 = s_box[0], fy0 = s_box[1], w = s_box[2], npix = w * s_box[3], nch = s_box[5];
                for (int c = 0; c < nch; ++c) {
                    for (int idx = tid; idx < kChunk * (kD / 8); idx += kThreads) {
                        const int r = idx / (kD / 8), g = idx % (kD / 8), t = kChunk * c + r;
                        const int py = fy0 + t / w, px = fx0 + t % w;
                        const bool in = t < npix && py >= 0 && py < H && px >= 0 && px < W;
                        const uint16_t *src = in ? fm + ((size_t)py * W + px) * kD + 8 * g : fm;
                        cp16(aA + op_off(r, 8 * g), src, in ? 16u : 0u);
                    }
                    cp_wait_all();
                    dpvo::fence_async_smem();
                    __syncthreads();
                    if (tid == 0) {
                        dpvo::tc_fence_after();
                        for (int ks = 0; ks < kD / 16; ++ks)
                            mma_bf16(tmem, dpvo::smem_desc(aA + ks * 2 * kLbo, kLbo, kSbo),
                                     dpvo::smem_desc(aB + ks * 2 * kLbo, kLbo, kSbo), ks > 0 ? 1 : 0);
                        dpvo::mma_commit(mbar);
                    }
                    ++n_commit;
                    if (!dpvo::mbar_wait(mbar, (uint32_t)(n_commit - 1) & 1u)) atomicOr(&s_bad, 1);
                    __syncthreads();
                    if (s_bad) break;                    // reported below; outputs of this edge stay zero
                    dpvo::tc_fence_after();
                    float v[16];
                    dpvo::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16), v);
                    const int t = kChunk * c + tid;
                    if (t < npix) {
#pragma unroll
                        for (int q = 0; q < kQ; ++q) Dbuf[t * kDld + q] = v[q];
                    }
                    dpvo::tc_fence_before();
                    __syncthreads();                     // the operand and the accumulator are reused
                }
            } else if (mode == 2) {
                // windows too far apart: each patch pixel's 8 x 8 inner products on the CUDA cores
                for (int idx = tid; idx < kQ * 64; idx += kThreads) {
                    const int q = idx >> 6, m = (idx >> 3) & 7, n = idx & 7;
                    const int py = (int)floorf(s_xy[q][1]) - 3 + m, px = (int)floorf(s_xy[q][0]) - 3 + n;
                    float acc = 0.f;
                    if (py >= 0 && py < H && px >= 0 && px < W) {
                        const uint16_t *f = fm + ((size_t)py * W + px) * kD, *g = A.gpatch + ((size_t)k * kQ + q) * kD;
                        for (int c = 0; c < kD; ++c) acc = fmaf(bf16_to_f(g[c]), bf16_to_f(f[c]), acc);
                    }
                    Dbuf[idx] = acc;
                }
                __syncthreads();
            }
            // epilogue: the 9 x 49 outputs of this level
            float *out = A.corr + ((size_t)e * 2 + level) * kQ * 49;
            for (int o = tid; o < kQ * 49; o += kThreads) {
                const int q = o / 49, ab = o - 49 * q, a = ab / 7, b = ab - 7 * a;
                float r = 0.f;
                if (mode != 0 && !s_bad) {
                    const float x = s_xy[q][0], y = s_xy[q][1];
                    const float xf = floorf(x), yf = floorf(y), wx = x - xf, wy = y - yf;
                    float d00, d01, d10, d11;
                    if (mode == 1) {
                        const int w = s_box[2];
                        const int t = ((int)yf - 3 + a - s_box[1]) * w + ((int)xf - 3 + b - s_box[0]);
                        d00 = Dbuf[t * kDld + q];
                        d01 = Dbuf[(t + 1) * kDld + q];
                        d10 = Dbuf[(t + w) * kDld + q];
                        d11 = Dbuf[(t + w + 1) * kDld + q];
                    } else {
                        const float *Dq = Dbuf + 64 * q + 8 * a + b;
                        d00 = Dq[0]; d01 = Dq[1]; d10 = Dq[8]; d11 = Dq[9];
                    }
                    r = (1.f - wy) * ((1.f - wx) * d00 + wx * d01) + wy * ((1.f - wx) * d10 + wx * d11);
                }
                out[o] = r;
            }
            __syncthreads();
        }
        cp_wait_all();                                   // this edge's copies are done before the next edge's
    }
    __syncthreads();
    if (tid == 0) {
        if (s_bad) {
            // report, and give the last commit one more bounded wait before the TMEM is freed
            atomicOr(A.status, DPVO_BA_STATUS_TIMEOUT);
            dpvo::mbar_wait(mbar, (uint32_t)(n_commit - 1) & 1u);
        }
        if (s_badin) atomicOr(A.status, DPVO_BA_STATUS_BAD_INPUT);
    }
    dpvo::tc_fence_before();
    __syncthreads();
    if (warp == 0) dpvo::tmem_dealloc(tmem, 32);
}

}  // namespace dpvo_corr

extern "C" int dpvo_ba_correlation(const dpvo_ba_corr_dims *d, const void *fmap0, const void *fmap1,
                                   const void *gpatch, const int32_t *kk, const int32_t *jj, const float *coords,
                                   float *corr, int32_t *status, void *stream) {
    if (!d || d->n_frames < 1 || d->n_patches < 0 || d->n_edges < 0 || d->height < 1 || d->width < 1 ||
        d->height > 4096 || d->width > 4096 || d->level1_scale < 1 || !status)
        return DPVO_BA_EINVAL;
    if (d->n_edges > 0 && (!fmap0 || !fmap1 || !gpatch || !kk || !jj || !coords || !corr)) return DPVO_BA_EINVAL;
    const int H1 = d->height / d->level1_scale, W1 = d->width / d->level1_scale;
    if (H1 < 1 || W1 < 1) return DPVO_BA_EINVAL;
    if (d->n_edges == 0) return 0;
    static int configured_device = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DPVO_BA_ECUDA;
    const size_t smem = dpvo_corr::kAbytes + dpvo_corr::kBbytes +
                        (size_t)dpvo_corr::kMaxChunks * dpvo_corr::kChunk * dpvo_corr::kDld * 4;
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
    const int grid = d->n_edges < 2 * sms ? d->n_edges : 2 * sms;
    dpvo_corr::corr_kernel<<<grid, dpvo_corr::kThreads, smem, reinterpret_cast<cudaStream_t>(stream)>>>(A);
    return cudaGetLastError() == cudaSuccess ? 0 : DPVO_BA_ECUDA;
}
