// Internal definitions shared by the bundle-adjustment kernels and the host API.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dpvo_ba.h"

namespace dpvo {

constexpr int kThreads = 256;          // block size of the linearise and solve kernels
constexpr int kMaxWindow = 64;         // frames the edges of one patch chunk may span
constexpr int kMaxFree = DPVO_BA_MAX_FREE;
// Free poses up to which the Schur complement accumulates inside the linearise
// kernel (each strip owner keeps its sums in registers) and the reduced system
// is factored from a full n x (n + 1) array in shared memory.  Beyond it a
// separate assembly kernel reads the stored Schur rows, and the solve keeps S
// packed (FP32 copy in shared memory, FP64 in the workspace).
constexpr int kFusedMaxFree = 15;
constexpr int kFlushEvery = 16;        // patches summed in FP32 before a compensated add
constexpr int kMaxKSplit = 8;          // patch-parity split of the Schur accumulation

// A run of consecutive patches that share one source frame (anchor).
struct Chunk {
    int k0, count;     // patches [k0, k0 + count)
    int e0, e1;        // their edges [e0, e1)
    int anchor;        // source frame of every patch in the chunk
    int jlo, jhi;      // frames touched by the chunk's edges lie in [jlo, jhi]
    int pad;
};

// Everything a kernel needs about one problem: caller arrays, sizes, workspace.
struct Prob {
    float *poses;            // [N][7] caller, IN/OUT
    float *patches;          // [P][3] caller, d IN/OUT
    const int32_t *anchor;   // [P]
    const int32_t *kk;       // [E]
    const int32_t *jj;       // [E]
    const float *target;     // [E][2]
    const float *weight;     // [E][2]
    int32_t *status_user;    // [1] or null

    int N, P, E, t0, iters, nf;
    float fx, fy, cx, cy;
    float damping, z_min;

    int32_t *seg;            // [P + 1] first edge of each patch
    Chunk *chunks;           // [max_chunks]
    int32_t *n_chunks;       // [1]
    int32_t *status;         // [1] DPVO_BA_STATUS_* bits
    float *pose_it;          // [iters + 1][N][7] iterates
    float *depth_it;         // [iters + 1][P]
    double *dxi;             // [iters][nf][6] pose increments
    double *partial;         // [n_parts][L] Schur partial sums (linearise CTAs, then assembly CTAs)
    double *sglob;           // [6nf (6nf + 1) / 2] FP64 reduced system, packed lower (more than kFusedMaxFree free poses)
    float *erow;             // [P][erow_len(nf)] scaled Schur row of each patch, last linearisation
    // backward (adjoint) state; null / zero for a plain solve
    int store_factor;        // keep the factored reduced system of every iteration
    int no_writeback;        // leave the caller's poses and patches untouched
    double *ufac;            // [iters][n (n + 1) / 2] factor U (lower, row-major) of each iteration
    const float *dL_dposes;  // [N][7] gradient of the loss w.r.t. the final poses
    const float *dL_ddepth;  // [P] gradient w.r.t. the final inverse depths
    float *dL_dtarget;       // [E][2] output
    float *dL_dweight;       // [E][2] output
    double *eps;             // [N][6] pose gradient (left-perturbation coordinates)
    double *dxibar;          // [nf][6] gradient w.r.t. the pose increment of the current iteration
    double *yxi;             // [nf][6] adjoint solution, pose part
    float *dbar;             // [P] gradient w.r.t. the inverse depths of the current state
    double *pgrad;           // [n_items][N][6] per-CTA pose-gradient partial sums

    int max_chunks;
    int n_items;             // linearise work items (CTAs) of this problem
    int n_asm;               // Schur-assembly work items (0: accumulated inside the linearise kernel)
    int n_parts;             // partials summed by the solve
    int bulk_edges;          // jj, target, weight 16-byte aligned: chunks staged by bulk copies
    int ks;                  // patch-parity split of the Schur accumulation
    int L;                   // doubles per partial
    int chunk_cap;           // patches per chunk at most
    int win_cap;             // frames per chunk window at most
    int solve_f64;           // reduced solve by FP64 elimination only (no FP32 factor)
    int plan_ticket;         // plan CTAs of this problem done with their edge slices (0 on upload)
    int plan_bad;            // an edge slice found invalid input (0 on upload)
};

// Stored Schur row of a patch, written when it is linearised and read by the
// back-substitution of that iteration: the pose columns C_k^-1/2 e_k, free
// frame f at floats 8f..8f+7 as [v0 v1 v2 0 v3 v4 v5 0] (the layout the
// linearisation keeps them in), then C_k^-1/2 w_k, C_k^-1/2, 0, 0.  Every row
// starts on a 16-byte boundary.
__host__ __device__ inline int erow_len(int nf) { return 8 * nf + 4; }
__host__ __device__ inline int erow_smem_stride(int nf) { return erow_len(nf); }

// One CTA of the linearise kernel: problem index and work-item index within it.
struct Item {
    int prob, item;
};

// Reduced-system layout.  The upper triangle of 6x6 pose blocks (a, b), a <= b,
// is split into half-blocks ("strips") of 3 rows x 6 columns; the right-hand
// side is one 6-entry strip per free pose.
__host__ __device__ inline int n_block_pairs(int nf) { return nf * (nf + 1) / 2; }
__host__ __device__ inline int n_strips(int nf) { return 2 * n_block_pairs(nf) + nf; }
__host__ __device__ inline int partial_len(int nf) { return 18 * 2 * n_block_pairs(nf) + 6 * nf; }
__host__ __device__ inline int k_split(int nf) {
    int s = n_strips(nf);
    if (s == 0) return 1;
    int k = kThreads / s;
    return k < 1 ? 1 : (k > kMaxKSplit ? kMaxKSplit : k);
}

// The problem's status bits as one thread of the block read them: every
// thread of a kernel with block barriers must take the same early exit, and
// another block may set a bit while this one starts.
__device__ inline int block_status(const int32_t *status) {
    __shared__ int s_status_once;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_status_once = *status;
    __syncthreads();
    return s_status_once;
}

// Decode the upper-triangle pair index of (a, b), a <= b.
__host__ __device__ inline void decode_pair(int idx, int nf, int &a, int &b) {
    a = 0;
    while (idx >= nf - a) {
        idx -= nf - a;
        ++a;
    }
    b = a + idx;
}

// Index into the 21 packed entries of a symmetric 6x6 matrix.
__host__ __device__ constexpr int sym6(int r, int c) {
    return r <= c ? r * 6 - r * (r - 1) / 2 + (c - r) : c * 6 - c * (c - 1) / 2 + (r - c);
}

}  // namespace dpvo
