// Host side of the C ABI declared in include/dpvo_ba.h: argument checks,
// workspace layout, descriptor upload and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <cstring>
#include <queue>
#include <vector>

#include "dpvo_ba.h"
#include "ba_common.cuh"
#include "kernels.cuh"
#include "solve_large.cuh"
#include "solve_warp.cuh"
#include "assemble_tc.cuh"
#include "assemble.cuh"
#include "backward.cuh"
#include "serve.cuh"
#include "window_host.h"

using namespace dpvo;

namespace {

constexpr size_t kLinSmemBudget = 112 * 1024;   // two CTAs per SM (228 KB, 1 KB reserved per CTA)

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// The edge arrays can be staged by bulk copies (16-byte aligned starts).
bool aligned16(const void *a, const void *b, const void *c) {
    return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15) == 0;
}

struct Layout {
    std::vector<Prob> probs;       // workspace pointers hold offsets until rebased
    std::vector<Item> items;       // linearise work items, then assembly work items
    size_t bytes = 0, off_probs = 0, off_items = 0;
    int W_cap = 1, G_cap = 64, nf_max = 0, iters_max = 0, n_max = 1;
    int max_parts = 1;             // Schur partials of the problem with the most
    int e_max = 0;                 // edges of the problem with the most
    bool tc = false;               // Schur accumulation on the tensor cores
    bool ext = false;              // more than kFusedMaxFree free poses: assembly kernel, packed solve
    bool tc_asm = false;           // ext with the TF32 Schur mode: the assembly on the tensor cores
    int n_lin_items = 0, n_asm_items = 0;
    int final_slices = 1;          // y extent of the last back-substitution's grid
    size_t lin_smem = 0, solve_smem = 0, asm_smem = 0;
    size_t sw_smem = 0;            // solve_warp_kernel (forward solves of at most kFusedMaxFree free poses)
};

// solve_kernel shared memory: S and its FP32 copy (n x (n+1)), v, x, the FP32 right-hand side,
// the inverted diagonal blocks of the factor.
static size_t solve_smem_bytes(int nf) {
    // S (FP64, n x (n+1)), v, x; the FP32 factor (rows padded to 4), the
    // panel's scaled columns, the right-hand side
    const size_t n = 6 * (size_t)nf, ldf = (n + 3) & ~(size_t)3;
    return n * (n + 1) * 8 + 2 * n * 8 + n * ldf * 4 + n * kSolvePanel * 4 + n * 4 + 64;
}

// Stored Schur rows: one row per patch, or in the tensor-core variant one
// block of kTcRows x Kmax floats per chunk.
static size_t erow_bytes(bool tc, const Prob &p, int G_cap) {
    if (tc) return (size_t)p.max_chunks * kTcRows * tc_kmax(G_cap) * 4 + 16;
    return (size_t)p.P * erow_len(p.nf) * 4 + 16;
}

// Assembly launch (ext batches): grid x = assembly items, y = strip slices.
static void launch_assembly(const Layout &L, cudaStream_t stream, const Prob *probs, const Item *asm_items, int t) {
    if (L.tc_asm) {
        schur_assembly_tc_kernel<<<L.n_asm_items, kAtcThreads, L.asm_smem, stream>>>(probs, asm_items, t,
                                                                                     erow_len(L.nf_max));
        return;
    }
    const dim3 grid(L.n_asm_items, asm_slices(L.nf_max));
    schur_assembly_kernel<<<grid, asm_threads(L.nf_max), L.asm_smem, stream>>>(probs, asm_items, t,
                                                                               erow_len(L.nf_max));
}

// The plan launch: one CTA per problem for batches of at least one problem
// per SM; smaller batches split each problem's edges into slices of at least
// kPlanSliceEdges, up to two CTAs per SM over the batch.
static void launch_plan(int n, int e_max, int num_sms, cudaStream_t stream, const Prob *probs) {
    int slices = 1;
    if (n < num_sms)
        slices = std::max(1, std::min((e_max + kPlanSliceEdges - 1) / kPlanSliceEdges, 2 * num_sms / n));
    plan_kernel<<<dim3(n, slices), kPlanThreads, 0, stream>>>(probs, slices);
}

// The forward reduced solve of at most kFusedMaxFree free poses: one CTA per
// problem, which sums the problem's Schur partials itself, or a cluster of
// kSwCluster CTAs per problem where some problem has more than kSwDirectParts
// partials (they sum them; a cluster grid of a large batch would take several
// waves); the rows per lane set by the largest problem.
static void launch_solve_warp(int nf_max, int max_parts, int n, cudaStream_t stream, const Prob *probs, int t,
                              size_t smem) {
    auto kernel = sw_rows(nf_max) == 2 ? solve_warp_kernel<2> : solve_warp_kernel<3>;
    if (max_parts <= kSwDirectParts || nf_max == 0) {
        kernel<<<n, kSwThreads, smem, stream>>>(probs, t, 1);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n * kSwCluster);
    cfg.blockDim = dim3(kSwThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kSwCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, probs, t, (int)kSwCluster);
}

// Reduced solve launch, in the batch's variant.
static void launch_solve(const Layout &L, int n, cudaStream_t stream, const Prob *probs, int t, double *S_out,
                         double *v_out) {
    if (L.ext) solve_large_kernel<<<n, kSolveThreads, L.solve_smem, stream>>>(probs, t, S_out, v_out);
    else if (S_out) solve_kernel<<<n, kSolveThreads, L.solve_smem, stream>>>(probs, t, S_out, v_out);
    else launch_solve_warp(L.nf_max, L.max_parts, n, stream, probs, t, L.sw_smem);
}

// The bounded mbarrier wait of the pipelined kernels, on a phase that completes
// only if `arrive` (one warp; lane 0 does the work).
__global__ void selftest_wait_kernel(int32_t *status, int arrive, int polls) {
    __shared__ __align__(8) uint64_t s_bar;
    if (threadIdx.x != 0) return;
    const uint32_t bar = smem_u32(&s_bar);
    mbar_init(bar, 1);
    if (arrive) mbar_arrive(bar);
    *status = mbar_wait(bar, 0u, polls) ? 0 : DPVO_BA_STATUS_TIMEOUT;
}

// Slices of one problem in the last back-substitution's grid: all of them, at
// most `cap` (the CTAs then stride over the rest, which spreads each CTA's
// start-up over several slices).
static int final_slices_of(bool tc, int n_patches, int max_chunks, int cap) {
    const int units = tc ? max_chunks : n_patches, per = tc ? kFinalChunks : kFinalPatches;
    return std::min(std::min(65535, cap), std::max(1, (units + per - 1) / per));
}

// The last back-substitution (iteration t = the batch's last): n problems.
// The row layout streams its stored rows through shared memory
// (final_rows_kernel); the tensor-core layout reads them in place.
static void launch_final(const Layout &L, int n, cudaStream_t stream, const Prob *probs, int t) {
    const dim3 grid(n, L.final_slices);
    if (L.tc) {
        const size_t smem = 4 * (size_t)std::max(kTcRows, erow_len(L.nf_max));
        final_kernel<true><<<grid, kThreads, smem, stream>>>(probs, t, L.G_cap);
    } else {
        const int rs = erow_len(L.nf_max);
        final_rows_kernel<<<grid, kThreads, fr_smem_bytes(rs), stream>>>(probs, t, rs);
    }
}

// CTAs of final_rows_kernel per problem that fill one wave of n problems.
static int final_rows_cap(int n, int nf_max, int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, final_rows_kernel, kThreads,
                                                      fr_smem_bytes(erow_len(nf_max))) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return std::max(1, per_sm * num_sms / n);
}

// One linearise launch, in the batch's variant.
static void launch_linearize(const Layout &L, int grid, cudaStream_t stream, const Prob *probs, const Item *items,
                             int t, int adjoint_rhs) {
    if (L.tc)
        linearize_kernel<true, false><<<grid, kThreads, L.lin_smem, stream>>>(probs, items, t, L.W_cap, L.G_cap,
                                                                          L.nf_max, L.n_max, adjoint_rhs);
    else if (L.ext)
        linearize_kernel<false, true><<<grid, kThreads, L.lin_smem, stream>>>(probs, items, t, L.W_cap, L.G_cap,
                                                                          L.nf_max, L.n_max, adjoint_rhs);
    else
        linearize_kernel<false, false><<<grid, kThreads, L.lin_smem, stream>>>(probs, items, t, L.W_cap, L.G_cap,
                                                                           L.nf_max, L.n_max, adjoint_rhs);
}

int check_dims(const dpvo_ba_dims &d) {
    if (d.n_frames < 1 || d.n_frames > DPVO_BA_MAX_FRAMES) return DPVO_BA_EINVAL;
    if (d.n_patches < 0 || d.n_edges < 0) return DPVO_BA_EINVAL;
    if (d.t0 < 0 || d.t0 > d.n_frames) return DPVO_BA_EINVAL;
    if (d.n_frames - d.t0 > DPVO_BA_MAX_FREE) return DPVO_BA_EINVAL;
    if (d.n_iters < 1 || d.n_iters > DPVO_BA_MAX_ITERS) return DPVO_BA_EINVAL;
    if (!(d.fx > 0.f) || !(d.fy > 0.f)) return DPVO_BA_EINVAL;
    return DPVO_BA_OK;
}

int check_problem(const dpvo_ba_dims &d, const dpvo_ba_problem &p) {
    if (!p.poses) return DPVO_BA_EINVAL;
    if (d.n_patches > 0 && (!p.patches || !p.anchor)) return DPVO_BA_EINVAL;
    if (d.n_edges > 0 && (!p.kk || !p.jj || !p.target || !p.weight)) return DPVO_BA_EINVAL;
    if (((uintptr_t)p.target & 7) || ((uintptr_t)p.weight & 7)) return DPVO_BA_EINVAL;
    return DPVO_BA_OK;
}

// Linearise work items per problem beyond kFusedMaxFree free poses (long
// passes over thousands of patches): the count, up to twice the one-wave
// count plus one, whose whole waves of two CTAs per SM are filled best.
static int ext_items(int n, int target_ctas) {
    const int k0 = std::max(1, target_ctas / n);
    int best = k0;
    double best_eff = 0.0;
    for (int k = k0; k <= 2 * k0 + 1; ++k) {
        const int ctas = n * k, waves = (ctas + target_ctas - 1) / target_ctas;
        const double eff = (double)ctas / ((double)waves * target_ctas);
        if (eff > best_eff + 1e-9) { best_eff = eff; best = k; }
    }
    return best;
}

Layout make_layout(const dpvo_ba_dims *dims, int n, int num_sms, const dpvo_ba_config &cfg, bool adjoint = false) {
    Layout L;
    int n_max = 1;
    for (int b = 0; b < n; ++b) {
        n_max = std::max(n_max, dims[b].n_frames);
        L.nf_max = std::max(L.nf_max, dims[b].n_frames - dims[b].t0);
        L.e_max = std::max(L.e_max, dims[b].n_edges);
        L.iters_max = std::max(L.iters_max, dims[b].n_iters);
    }
    L.n_max = n_max;
    L.tc = cfg.schur_tf32 == 1 && use_tensor_cores(L.nf_max);
    L.W_cap = std::min(n_max, kMaxWindow);
    L.G_cap = 64;
    while (L.G_cap > 8 && lin_smem_layout(L.W_cap, L.G_cap, L.nf_max, n_max, L.tc).bytes > kLinSmemBudget)
        L.G_cap -= 8;
    L.lin_smem = lin_smem_layout(L.W_cap, L.G_cap, L.nf_max, n_max, L.tc).bytes;
    L.ext = L.nf_max > kFusedMaxFree;
    L.tc_asm = L.ext && cfg.schur_tf32 != 2;   // beyond kFusedMaxFree: tensor cores unless FP32 is asked
    L.solve_smem = L.ext ? solve_large_smem_bytes(L.nf_max) : solve_smem_bytes(L.nf_max);
    L.sw_smem = L.ext ? 0 : sw_smem_bytes(L.nf_max);
    L.asm_smem = !L.ext ? 0
                 : L.tc_asm ? atc_smem_bytes(erow_len(L.nf_max))
                            : asm_smem_bytes(erow_len(L.nf_max), asm_threads(L.nf_max));
    const int asm_slices_max = L.ext && !L.tc_asm ? asm_slices(L.nf_max) : 1;

    const int target_ctas = 2 * num_sms;
    // one wave of the last back-substitution's CTAs
    const int final_cap = L.tc ? std::max(1, (6 * num_sms + n - 1) / n) : final_rows_cap(n, L.nf_max, num_sms);
    // a batch of unequal problems (serving mixes) deals the linearise CTAs of
    // one wave so that the most work (edges + patches) any CTA carries is
    // least: every problem starts with one CTA, and each further CTA goes to
    // the problem whose CTAs carry the most, up to its chunk count (and, in a
    // batch large enough that a cluster per problem would take several waves
    // of the reduced solve, up to the partials one solve CTA sums itself)
    double work_total = 0.0;
    bool uniform = true;
    for (int b = 0; b < n; ++b) {
        work_total += (double)dims[b].n_edges + dims[b].n_patches;
        uniform = uniform && dims[b].n_edges == dims[0].n_edges && dims[b].n_patches == dims[0].n_patches;
    }
    std::vector<int> items_of(n, 1);
    if (!L.ext && !uniform && work_total > 0.0 && n < target_ctas) {
        const int part_cap = n * kSwCluster > target_ctas ? kSwDirectParts : 1 << 30;
        std::priority_queue<std::pair<double, int>> heap;   // (work per CTA, problem)
        for (int b = 0; b < n; ++b) heap.push({(double)dims[b].n_edges + dims[b].n_patches, b});
        for (int left = target_ctas - n; left > 0 && !heap.empty();) {
            const int b = heap.top().second;
            heap.pop();
            const int cap = std::min(part_cap, (dims[b].n_patches + L.G_cap - 1) / L.G_cap + dims[b].n_frames);
            if (items_of[b] >= cap) continue;            // no further split of this one
            ++items_of[b];
            --left;
            heap.push({((double)dims[b].n_edges + dims[b].n_patches) / items_of[b], b});
        }
        // then no more CTAs than that largest share needs: a split that does
        // not lower it only adds a partial (e.g. some of many equal problems)
        double most = 0.0;
        for (int b = 0; b < n; ++b)
            most = std::max(most, ((double)dims[b].n_edges + dims[b].n_patches) / items_of[b]);
        for (int b = 0; b < n; ++b) {
            const double need = std::ceil(((double)dims[b].n_edges + dims[b].n_patches) / most * (1.0 - 1e-12));
            items_of[b] = std::max(1, std::min(items_of[b], (int)need));
        }
    }
    size_t off = 0;
    L.probs.resize(n);
    for (int b = 0; b < n; ++b) {
        const dpvo_ba_dims &d = dims[b];
        Prob &p = L.probs[b];
        std::memset(&p, 0, sizeof(Prob));
        p.N = d.n_frames; p.P = d.n_patches; p.E = d.n_edges; p.t0 = d.t0; p.iters = d.n_iters;
        p.nf = d.n_frames - d.t0;
        p.fx = d.fx; p.fy = d.fy; p.cx = d.cx; p.cy = d.cy;
        p.damping = cfg.damping; p.z_min = cfg.z_min;
        p.solve_f64 = cfg.reduced_solve_f64 ? 1 : 0;
        p.chunk_cap = L.G_cap;
        p.win_cap = L.W_cap;
        p.max_chunks = (d.n_patches + L.G_cap - 1) / L.G_cap + d.n_frames;
        p.ks = (L.tc || L.ext) ? 1 : k_split(p.nf);
        p.L = partial_len(p.nf);
        // work items: as many as fill one wave of the SMs (two linearise CTAs
        // per SM; one assembly CTA per SM), at least one per problem
        // at most one item per chunk: a frame's patches start a new chunk, so
        // there are up to ceil(P / G) + N of them
        int est_chunks = std::max(1, (d.n_patches + L.G_cap - 1) / L.G_cap);
        int items = std::max(1, target_ctas / n);
        if (L.ext) items = ext_items(n, target_ctas);
        else if (!uniform && work_total > 0.0)
            items = items_of[b];
        p.n_items = std::max(1, std::min(items, p.max_chunks));
        if (L.tc_asm) {   // ranges of at most kAtcMaxPatches patches, at least one CTA per SM over the batch
            const int need = (d.n_patches + kAtcMaxPatches - 1) / kAtcMaxPatches;
            const int stages = std::max(1, (d.n_patches + kAtcK - 1) / kAtcK);
            p.n_asm = std::max(1, std::min(stages, std::max(need, num_sms / n)));
        } else if (L.ext) {
            const int per = std::max(1, num_sms / (n * asm_slices_max));
            p.n_asm = std::max(1, std::min(per, est_chunks));
        }
        p.n_parts = L.ext ? p.n_items + p.n_asm : p.n_items;   // one partial per linearise CTA
        L.max_parts = std::max(L.max_parts, p.n_parts);
        // workspace offsets (rebased to device pointers later)
        auto take = [&](size_t bytes) { size_t o = off; off = al256(off + bytes); return o; };
        p.seg = (int32_t *)(uintptr_t)take((size_t)(d.n_patches + 1) * 4);
        p.chunks = (Chunk *)(uintptr_t)take((size_t)p.max_chunks * sizeof(Chunk));
        size_t ints = take(16);
        p.n_chunks = (int32_t *)(uintptr_t)ints;
        p.status = (int32_t *)(uintptr_t)(ints + 4);
        p.pose_it = (float *)(uintptr_t)take((size_t)(d.n_iters + 1) * d.n_frames * 7 * 4);
        p.depth_it = (float *)(uintptr_t)take((size_t)(d.n_iters + 1) * d.n_patches * 4);
        p.dxi = (double *)(uintptr_t)take((size_t)d.n_iters * p.nf * 6 * 8 + 8);
        p.partial = (double *)(uintptr_t)take((size_t)p.n_parts * p.L * 8 + 8);
        if (L.ext) {
            const size_t n6 = 6 * (size_t)p.nf;
            p.sglob = (double *)(uintptr_t)take(n6 * (n6 + 1) / 2 * 8 + 8);
        }
        p.erow = (float *)(uintptr_t)take(erow_bytes(L.tc, p, L.G_cap));
        if (adjoint) {
            const size_t n6 = 6 * (size_t)p.nf;
            p.store_factor = 1;
            p.no_writeback = 1;
            p.ufac = (double *)(uintptr_t)take((size_t)d.n_iters * (n6 * (n6 + 1) / 2) * 8 + 8);
            p.eps = (double *)(uintptr_t)take((size_t)d.n_frames * 6 * 8);
            p.dxibar = (double *)(uintptr_t)take(n6 * 8 + 8);
            p.yxi = (double *)(uintptr_t)take(n6 * 8 + 8);
            p.dbar = (float *)(uintptr_t)take((size_t)d.n_patches * 4 + 4);
            p.pgrad = (double *)(uintptr_t)take((size_t)p.n_items * d.n_frames * 6 * 8);
        }
        for (int w = 0; w < p.n_items; ++w) L.items.push_back(Item{b, w});
        L.final_slices = std::max(L.final_slices, final_slices_of(L.tc, d.n_patches, p.max_chunks, final_cap));
    }
    L.n_lin_items = (int)L.items.size();
    for (int b = 0; b < n; ++b)
        for (int w = 0; w < L.probs[b].n_asm; ++w) L.items.push_back(Item{b, w});
    L.n_asm_items = (int)L.items.size() - L.n_lin_items;
    L.off_probs = off;
    off = al256(off + sizeof(Prob) * n);
    L.off_items = off;
    off = al256(off + sizeof(Item) * L.items.size());
    L.bytes = off;
    return L;
}

template <typename T>
T *rebase(T *off, char *base) { return reinterpret_cast<T *>(base + (uintptr_t)off); }

}  // namespace

constexpr int kStageRing = 4;
constexpr int kHostSubBatches = 8;      // dpvo_ba_solve_host: sub-batches whose solves overlap the copies
constexpr int kHostSubBatchMin = 32;    // problems per sub-batch at least

struct dpvo_ba_handle {
    dpvo_ba_config cfg;
    int device = 0;
    int num_sms = 148;
    char *ws = nullptr;
    size_t ws_cap = 0;
    // page-locked host staging of the descriptors, a ring of buffers used in
    // turn: a call waits only for the copy out of the buffer it reuses, so
    // that the host can enqueue solves ahead of the device
    char *stage[kStageRing] = {};
    size_t stage_cap[kStageRing] = {};
    cudaEvent_t stage_done[kStageRing] = {};
    bool stage_pending[kStageRing] = {};
    int stage_next = 0;
    char *io = nullptr;             // device staging for dpvo_ba_solve_host
    cudaStream_t copy_stream = nullptr;              // dpvo_ba_solve_host: input copies of the sub-batches
    char *ws_sub[kHostSubBatches] = {};              // ... and each sub-batch's own workspace
    size_t ws_sub_cap[kHostSubBatches] = {};
    cudaEvent_t copy_ev[kHostSubBatches + 1] = {};   // a sub-batch's inputs landed; the caller's prior work
    size_t io_cap = 0;
    std::vector<Prob> last;         // descriptors of the last solve (for dpvo_ba_iterate)
    bool timing = false;            // record events around launches
    std::vector<cudaEvent_t> ev;    // event pool: (start, end) per timed launch
    std::vector<int> ev_kind;       // kernel of each timed launch
    int ev_used = 0;                // events recorded since the last read
    dpvo_serve::Server *srv = nullptr;   // serving runtime, if started
};

static int timed_event(dpvo_ba_handle *h, cudaStream_t s) {
    if (h->ev_used >= (int)h->ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return DPVO_BA_ECUDA;
        h->ev.push_back(e);
    }
    if (cudaEventRecord(h->ev[h->ev_used++], s) != cudaSuccess) return DPVO_BA_ECUDA;
    return DPVO_BA_OK;
}

static int grow_device(char **buf, size_t *cap, size_t need) {
    if (need <= *cap) return DPVO_BA_OK;
    if (*buf) {
        if (cudaDeviceSynchronize() != cudaSuccess) return DPVO_BA_ECUDA;
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    size_t sz = need + need / 4;
    if (cudaMalloc((void **)buf, sz) != cudaSuccess) {
        cudaGetLastError();
        return DPVO_BA_ENOMEM;
    }
    *cap = sz;
    return DPVO_BA_OK;
}

// The next staging buffer of the ring, at least `need` bytes, once the copy
// out of it (the call kStageRing calls ago) has completed.
static int take_stage(dpvo_ba_handle *h, size_t need, char **out) {
    const int i = h->stage_next;
    if (h->stage_pending[i]) {
        if (cudaEventSynchronize(h->stage_done[i]) != cudaSuccess) return DPVO_BA_ECUDA;
        h->stage_pending[i] = false;
    }
    if (need > h->stage_cap[i]) {
        if (h->stage[i]) cudaFreeHost(h->stage[i]);
        h->stage[i] = nullptr;
        h->stage_cap[i] = 0;
        if (cudaMallocHost((void **)&h->stage[i], need * 2) != cudaSuccess) {
            cudaGetLastError();
            return DPVO_BA_ENOMEM;
        }
        h->stage_cap[i] = need * 2;
    }
    *out = h->stage[i];
    return DPVO_BA_OK;
}

// After the copy out of the current staging buffer was enqueued on `stream`.
static int release_stage(dpvo_ba_handle *h, cudaStream_t stream) {
    const int i = h->stage_next;
    if (cudaEventRecord(h->stage_done[i], stream) != cudaSuccess) return DPVO_BA_ECUDA;
    h->stage_pending[i] = true;
    h->stage_next = (i + 1) % kStageRing;
    return DPVO_BA_OK;
}

// Kernel attributes belong to the current context, so they are set on every
// call that needs them (a handle's creation, each allocation-free solve) rather
// than cached per device: a context that is torn down and created again starts
// without them.  Setting them is a host-side call that allocates nothing.
static int set_kernel_attrs(int device) {
    (void)device;
    if (cudaFuncSetAttribute(linearize_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(linearize_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(linearize_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess)
        return DPVO_BA_ECUDA;
    if (cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
        cudaSuccess)
        return DPVO_BA_ECUDA;
    if (cudaFuncSetAttribute(solve_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
        cudaSuccess)
        return DPVO_BA_ECUDA;
    if (cudaFuncSetAttribute(solve_warp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sw_smem_bytes(kFusedMaxFree)) != cudaSuccess ||
        cudaFuncSetAttribute(solve_warp_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sw_smem_bytes(kFusedMaxFree)) != cudaSuccess)
        return DPVO_BA_ECUDA;
    if (cudaFuncSetAttribute(schur_assembly_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
        cudaSuccess)
        return DPVO_BA_ECUDA;
    if (cudaFuncSetAttribute(schur_assembly_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)atc_smem_bytes(erow_len(kMaxFree))) != cudaSuccess)
        return DPVO_BA_ECUDA;
    if (cudaFuncSetAttribute(bw_edge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
        cudaSuccess)
        return DPVO_BA_ECUDA;
    if (cudaFuncSetAttribute(final_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fr_smem_bytes(erow_len(kMaxFree))) != cudaSuccess)
        return DPVO_BA_ECUDA;
    return DPVO_BA_OK;
}

// Upload descriptors and run plan + iterations.  dims/probs host arrays.
// ws_slot >= 0 (dpvo_ba_solve_host's sub-batches): that sub-batch's own
// workspace, its descriptors uploaded on `upload` (the copy stream), then
// after_upload() (which enqueues the inputs there and orders `stream` after
// them) before the kernels go to `stream`.
static int run_solve(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *probs, int n,
                     cudaStream_t stream, double *S_out, double *v_out, int ws_slot = -1,
                     cudaStream_t upload = nullptr, const std::function<int()> &after_upload = {}) {
    Layout L = make_layout(dims, n, h->num_sms, h->cfg);
    char *&ws = ws_slot >= 0 ? h->ws_sub[ws_slot] : h->ws;
    size_t &ws_cap = ws_slot >= 0 ? h->ws_sub_cap[ws_slot] : h->ws_cap;
    if (!upload) upload = stream;
    int rc = grow_device(&ws, &ws_cap, L.bytes);
    if (rc) return rc;
    const size_t desc_bytes = L.bytes - L.off_probs;
    char *stage = nullptr;
    rc = take_stage(h, desc_bytes, &stage);
    if (rc) return rc;
    for (int b = 0; b < n; ++b) {
        Prob &p = L.probs[b];
        const dpvo_ba_problem &q = probs[b];
        p.poses = q.poses; p.patches = q.patches; p.anchor = q.anchor; p.kk = q.kk; p.jj = q.jj;
        p.target = q.target; p.weight = q.weight; p.status_user = q.status;
        p.bulk_edges = aligned16(q.jj, q.target, q.weight);
        p.seg = rebase(p.seg, ws);
        p.chunks = rebase(p.chunks, ws);
        p.n_chunks = rebase(p.n_chunks, ws);
        p.status = rebase(p.status, ws);
        p.pose_it = rebase(p.pose_it, ws);
        p.depth_it = rebase(p.depth_it, ws);
        p.dxi = rebase(p.dxi, ws);
        p.partial = rebase(p.partial, ws);
        p.erow = rebase(p.erow, ws);
        if (p.sglob) p.sglob = rebase(p.sglob, ws);
    }
    h->last = L.probs;
    std::memcpy(stage, L.probs.data(), sizeof(Prob) * n);
    std::memcpy(stage + (L.off_items - L.off_probs), L.items.data(), sizeof(Item) * L.items.size());
    if (cudaMemcpyAsync(ws + L.off_probs, stage, desc_bytes, cudaMemcpyHostToDevice, upload) != cudaSuccess)
        return DPVO_BA_ECUDA;
    if ((rc = release_stage(h, upload))) return rc;
    if (after_upload && (rc = after_upload())) return rc;

    const Prob *d_probs = reinterpret_cast<const Prob *>(ws + L.off_probs);
    const Item *d_items = reinterpret_cast<const Item *>(ws + L.off_items);
    const int n_items = L.n_lin_items;
    // with timing on, bracket each launch with a pair of events on `stream`
    auto timed = [&](int kind, auto &&launch) -> int {
        if (h->timing) {
            if (int r = timed_event(h, stream)) return r;
        }
        launch();
        if (h->timing) {
            if (int r = timed_event(h, stream)) return r;
            h->ev_kind.push_back(kind);
        }
        return DPVO_BA_OK;
    };
    if ((rc = timed(0, [&] { launch_plan(n, L.e_max, h->num_sms, stream, d_probs); }))) return rc;
    const Item *d_asm_items = d_items + L.n_lin_items;
    if (S_out) {
        launch_linearize(L, n_items, stream, d_probs, d_items, 0, 0);
        if (L.ext) launch_assembly(L, stream, d_probs, d_asm_items, 0);
        launch_solve(L, n, stream, d_probs, 0, S_out, v_out);
    } else {
        for (int t = 0; t <= L.iters_max; ++t) {
            if (t < L.iters_max) rc = timed(1, [&] { launch_linearize(L, n_items, stream, d_probs, d_items, t, 0); });
            else rc = timed(4, [&] { launch_final(L, n, stream, d_probs, t); });
            if (rc) return rc;
            if (t < L.iters_max) {
                if (L.ext) {
                    rc = timed(3, [&] { launch_assembly(L, stream, d_probs, d_asm_items, t); });
                    if (rc) return rc;
                }
                rc = timed(2, [&] { launch_solve(L, n, stream, d_probs, t, nullptr, nullptr); });
                if (rc) return rc;
            }
        }
    }
    if (cudaGetLastError() != cudaSuccess) return DPVO_BA_ECUDA;
    return DPVO_BA_OK;
}

static int serve_stop_impl(dpvo_ba_handle *h);

// Forward with the factors kept and the caller's state untouched, then the
// adjoint iterations from the last one back to the first.
static int run_backward(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *probs,
                        const dpvo_ba_grads *grads, int n, cudaStream_t stream) {
    Layout L = make_layout(dims, n, h->num_sms, h->cfg, true);
    int rc = grow_device(&h->ws, &h->ws_cap, L.bytes);
    if (rc) return rc;
    const size_t desc_bytes = L.bytes - L.off_probs;
    char *stage = nullptr;
    rc = take_stage(h, desc_bytes, &stage);
    if (rc) return rc;
    for (int b = 0; b < n; ++b) {
        Prob &p = L.probs[b];
        const dpvo_ba_problem &q = probs[b];
        p.poses = q.poses; p.patches = q.patches; p.anchor = q.anchor; p.kk = q.kk; p.jj = q.jj;
        p.target = q.target; p.weight = q.weight; p.status_user = q.status;
        p.bulk_edges = aligned16(q.jj, q.target, q.weight);
        p.dL_dposes = grads[b].dL_dposes;
        p.dL_ddepth = grads[b].dL_ddepth;
        p.dL_dtarget = grads[b].dL_dtarget;
        p.dL_dweight = grads[b].dL_dweight;
        p.seg = rebase(p.seg, h->ws);
        p.chunks = rebase(p.chunks, h->ws);
        p.n_chunks = rebase(p.n_chunks, h->ws);
        p.status = rebase(p.status, h->ws);
        p.pose_it = rebase(p.pose_it, h->ws);
        p.depth_it = rebase(p.depth_it, h->ws);
        p.dxi = rebase(p.dxi, h->ws);
        p.partial = rebase(p.partial, h->ws);
        p.erow = rebase(p.erow, h->ws);
        if (p.sglob) p.sglob = rebase(p.sglob, h->ws);
        p.ufac = rebase(p.ufac, h->ws);
        p.eps = rebase(p.eps, h->ws);
        p.dxibar = rebase(p.dxibar, h->ws);
        p.yxi = rebase(p.yxi, h->ws);
        p.dbar = rebase(p.dbar, h->ws);
        p.pgrad = rebase(p.pgrad, h->ws);
    }
    h->last = L.probs;
    std::memcpy(stage, L.probs.data(), sizeof(Prob) * n);
    std::memcpy(stage + (L.off_items - L.off_probs), L.items.data(), sizeof(Item) * L.items.size());
    if (cudaMemcpyAsync(h->ws + L.off_probs, stage, desc_bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return DPVO_BA_ECUDA;
    if ((rc = release_stage(h, stream))) return rc;
    const Prob *d_probs = reinterpret_cast<const Prob *>(h->ws + L.off_probs);
    const Item *d_items = reinterpret_cast<const Item *>(h->ws + L.off_items);
    const int n_items = L.n_lin_items;
    const size_t bw_smem = bw_smem_layout(L.W_cap, L.G_cap, L.n_max).bytes;
    const Item *d_asm_items = d_items + L.n_lin_items;
    launch_plan(n, L.e_max, h->num_sms, stream, d_probs);
    for (int t = 0; t < L.iters_max; ++t) {
        launch_linearize(L, n_items, stream, d_probs, d_items, t, 0);
        if (L.ext) {   // beyond kFusedMaxFree: the assembly, then the packed solve keeping its FP64 factor
            launch_assembly(L, stream, d_probs, d_asm_items, t);
            solve_large_kernel<<<n, kSolveThreads, L.solve_smem, stream>>>(d_probs, t, nullptr, nullptr);
        } else {
            solve_kernel<<<n, kSolveThreads, L.solve_smem, stream>>>(d_probs, t, nullptr, nullptr);
        }
    }
    launch_final(L, n, stream, d_probs, L.iters_max);
    bw_init_kernel<<<n, kThreads, 0, stream>>>(d_probs);
    for (int t = L.iters_max - 1; t >= 0; --t) {
        bw_retract_kernel<<<n, kSolveThreads, 0, stream>>>(d_probs, t);
        launch_linearize(L, n_items, stream, d_probs, d_items, t, 1);
        // beyond kFusedMaxFree the right-hand side sum_k E_k C_k^-1 dbar_k comes
        // from the assembly's v' part over the rows the adjoint pass stored
        if (L.ext) launch_assembly(L, stream, d_probs, d_asm_items, t);
        bw_solve_kernel<<<n, kSolveThreads, 0, stream>>>(d_probs, t);
        bw_edge_kernel<<<n_items, kThreads, bw_smem, stream>>>(d_probs, d_items, t, L.W_cap, L.G_cap, L.n_max);
    }
    if (cudaGetLastError() != cudaSuccess) return DPVO_BA_ECUDA;
    return DPVO_BA_OK;
}

extern "C" {

int dpvo_ba_backward(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *probs,
                     const dpvo_ba_grads *grads, int n_problems, void *stream) {
    if (!h || !dims || !probs || !grads || n_problems < 1) return DPVO_BA_EINVAL;
    for (int b = 0; b < n_problems; ++b) {
        if (int rc = check_dims(dims[b])) return rc;
        if (int rc = check_problem(dims[b], probs[b])) return rc;
        const dpvo_ba_grads &g = grads[b];
        if (!g.dL_dposes || (dims[b].n_patches > 0 && !g.dL_ddepth) ||
            (dims[b].n_edges > 0 && (!g.dL_dtarget || !g.dL_dweight)))
            return DPVO_BA_EINVAL;
    }
    return run_backward(h, dims, probs, grads, n_problems, (cudaStream_t)stream);
}

int dpvo_ba_create(const dpvo_ba_config *cfg, dpvo_ba_handle **out) {
    if (!out) return DPVO_BA_EINVAL;
    *out = nullptr;
    dpvo_ba_handle *h = new dpvo_ba_handle();
    h->cfg.damping = 1e-4f;
    h->cfg.z_min = 0.1f;
    h->cfg.mem_budget_bytes = (size_t)8 << 30;
    h->cfg.max_sessions = 256;
    h->cfg.schur_tf32 = 0;
    h->cfg.reduced_solve_f64 = 0;
    if (cfg) {
        h->cfg = *cfg;
        if (h->cfg.mem_budget_bytes == 0) h->cfg.mem_budget_bytes = (size_t)8 << 30;
        if (h->cfg.max_sessions <= 0) h->cfg.max_sessions = 256;
    }
    if (!(h->cfg.damping >= 0.f) || !(h->cfg.z_min == h->cfg.z_min)) { delete h; return DPVO_BA_EINVAL; }
    if (cudaGetDevice(&h->device) != cudaSuccess) { cudaGetLastError(); delete h; return DPVO_BA_ECUDA; }
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        cudaGetLastError(); delete h; return DPVO_BA_ECUDA;
    }
    for (int i = 0; i < kStageRing; ++i) {
        if (cudaEventCreateWithFlags(&h->stage_done[i], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (int k = 0; k < i; ++k) cudaEventDestroy(h->stage_done[k]);
            delete h;
            return DPVO_BA_ECUDA;
        }
    }
    if (set_kernel_attrs(h->device)) {
        for (int i = 0; i < kStageRing; ++i) cudaEventDestroy(h->stage_done[i]);
        delete h;
        return DPVO_BA_ECUDA;
    }
    *out = h;
    return DPVO_BA_OK;
}

int dpvo_ba_destroy(dpvo_ba_handle *h) {
    if (!h) return DPVO_BA_EINVAL;
    serve_stop_impl(h);
    cudaDeviceSynchronize();
    if (h->ws) cudaFree(h->ws);
    if (h->io) cudaFree(h->io);
    for (int i = 0; i < kStageRing; ++i) {
        if (h->stage[i]) cudaFreeHost(h->stage[i]);
        if (h->stage_done[i]) cudaEventDestroy(h->stage_done[i]);
    }
    for (cudaEvent_t e : h->copy_ev)
        if (e) cudaEventDestroy(e);
    for (char *w : h->ws_sub)
        if (w) cudaFree(w);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    delete h;
    return DPVO_BA_OK;
}

int dpvo_ba_reserve(dpvo_ba_handle *h, const dpvo_ba_dims *max_dims, int n_problems) {
    if (!h || !max_dims || n_problems < 1) return DPVO_BA_EINVAL;
    dpvo_ba_dims d = *max_dims;
    d.t0 = std::max(0, d.n_frames - DPVO_BA_MAX_FREE);
    if (int rc = check_dims(d)) return rc;
    std::vector<dpvo_ba_dims> all(n_problems, d);
    Layout L = make_layout(all.data(), n_problems, h->num_sms, h->cfg);
    if (int rc = grow_device(&h->ws, &h->ws_cap, L.bytes)) return rc;
    for (int i = 0; i < kStageRing; ++i) {   // every buffer of the ring, in turn
        char *stage = nullptr;
        if (int rc = take_stage(h, L.bytes - L.off_probs, &stage)) return rc;
        h->stage_next = (h->stage_next + 1) % kStageRing;
    }
    return DPVO_BA_OK;
}

int dpvo_ba_solve(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *probs, int n_problems,
                  void *stream) {
    if (!h || !dims || !probs || n_problems < 1) return DPVO_BA_EINVAL;
    for (int b = 0; b < n_problems; ++b) {
        if (int rc = check_dims(dims[b])) return rc;
        if (int rc = check_problem(dims[b], probs[b])) return rc;
    }
    return run_solve(h, dims, probs, n_problems, (cudaStream_t)stream, nullptr, nullptr);
}

int dpvo_ba_reduced_system(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *prob,
                           double *S_out, double *v_out, void *stream) {
    if (!h || !dims || !prob || !S_out || !v_out) return DPVO_BA_EINVAL;
    if (int rc = check_dims(*dims)) return rc;
    if (int rc = check_problem(*dims, *prob)) return rc;
    if (dims->n_frames == dims->t0) return DPVO_BA_EINVAL;
    dpvo_ba_dims d = *dims;
    d.n_iters = 1;
    return run_solve(h, &d, prob, 1, (cudaStream_t)stream, S_out, v_out);
}

// Copies for dpvo_ba_solve_host.  Device staging keeps each array kind of
// all problems back to back; runs of problems whose host arrays are also back
// to back move in one cudaMemcpyAsync.
namespace {
struct KindCopy {
    size_t dev_off;                 // start of this kind's region in h->io
    std::vector<size_t> pos;        // byte offset of problem b in the region
    std::vector<size_t> bytes;      // bytes of problem b
};

// Copies of problems [b0, b1) of one kind, merged where consecutive
// problems' host arrays are contiguous.
int copy_runs(char *dev_base, const KindCopy &k, const std::vector<char *> &host, cudaMemcpyKind dir,
              cudaStream_t s, size_t b0 = 0, size_t b1 = SIZE_MAX) {
    const size_t n = std::min(host.size(), b1);
    size_t b = b0;
    while (b < n) {
        size_t e = b + 1, len = k.bytes[b];
        while (e < n && host[e] == host[e - 1] + k.bytes[e - 1]) { len += k.bytes[e]; ++e; }
        if (len) {
            char *d = dev_base + k.dev_off + k.pos[b];
            cudaError_t r = dir == cudaMemcpyHostToDevice ? cudaMemcpyAsync(d, host[b], len, dir, s)
                                                          : cudaMemcpyAsync(host[b], d, len, dir, s);
            if (r != cudaSuccess) return DPVO_BA_ECUDA;
        }
        b = e;
    }
    return DPVO_BA_OK;
}
}  // namespace

int dpvo_ba_solve_host(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *hp, int n_problems,
                       void *stream_) {
    if (!h || !dims || !hp || n_problems < 1) return DPVO_BA_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    for (int b = 0; b < n_problems; ++b) {
        if (int rc = check_dims(dims[b])) return rc;
        if (int rc = check_problem(dims[b], hp[b])) return rc;
    }
    // kinds: 0 poses, 1 patches, 2 anchor, 3 kk, 4 jj, 5 target, 6 weight, 7 status
    const int NK = 8;
    KindCopy k[NK];
    size_t total = 0;
    for (int q = 0; q < NK; ++q) {
        k[q].dev_off = total;
        size_t pos = 0;
        for (int b = 0; b < n_problems; ++b) {
            const size_t N = dims[b].n_frames, P = dims[b].n_patches, E = dims[b].n_edges;
            const size_t sz[NK] = {N * 28, P * 12, P * 4, E * 4, E * 4, E * 8, E * 8, 4};
            k[q].pos.push_back(pos);
            k[q].bytes.push_back(sz[q]);
            pos += sz[q];
        }
        total = al256(total + pos);
    }
    if (int rc = grow_device(&h->io, &h->io_cap, total)) return rc;
    std::vector<dpvo_ba_problem> dp(n_problems);
    std::vector<char *> host[NK];
    for (int b = 0; b < n_problems; ++b) {
        auto dev = [&](int q) { return h->io + k[q].dev_off + k[q].pos[b]; };
        dp[b].poses = (float *)dev(0);
        dp[b].patches = (float *)dev(1);
        dp[b].anchor = (const int32_t *)dev(2);
        dp[b].kk = (const int32_t *)dev(3);
        dp[b].jj = (const int32_t *)dev(4);
        dp[b].target = (const float *)dev(5);
        dp[b].weight = (const float *)dev(6);
        dp[b].status = (int32_t *)dev(7);
        host[0].push_back((char *)hp[b].poses);
        host[1].push_back((char *)hp[b].patches);
        host[2].push_back((char *)hp[b].anchor);
        host[3].push_back((char *)hp[b].kk);
        host[4].push_back((char *)hp[b].jj);
        host[5].push_back((char *)hp[b].target);
        host[6].push_back((char *)hp[b].weight);
        host[7].push_back((char *)hp[b].status);
    }
    // Large calls go in up to kHostSubBatches sub-batches: the inputs of
    // every sub-batch are copied on the handle's copy stream, and each
    // sub-batch is solved on the caller's stream once its inputs have landed,
    // so that the solves run under the copies of the later sub-batches.
    const int subs = std::max(1, std::min(kHostSubBatches, n_problems / kHostSubBatchMin));
    cudaStream_t cs = stream;
    if (subs > 1) {
        if (!h->copy_stream) {
            if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return DPVO_BA_ECUDA;
            for (int s = 0; s <= kHostSubBatches; ++s)
                if (cudaEventCreateWithFlags(&h->copy_ev[s], cudaEventDisableTiming) != cudaSuccess)
                    return DPVO_BA_ECUDA;
        }
        cs = h->copy_stream;
        if (cudaEventRecord(h->copy_ev[kHostSubBatches], stream) != cudaSuccess ||   // after the caller's work
            cudaStreamWaitEvent(cs, h->copy_ev[kHostSubBatches], 0) != cudaSuccess)
            return DPVO_BA_ECUDA;
    }
    auto range = [&](int s, int &b0, int &b1) {
        b0 = (int)((long long)s * n_problems / subs);
        b1 = (int)((long long)(s + 1) * n_problems / subs);
    };
    // Enqueued sub-batch by sub-batch: a solve's own descriptor upload is a
    // host-to-device copy too, and it must not queue behind the later
    // sub-batches' inputs on the copy engine.
    for (int s = 0; s < subs; ++s) {
        int b0, b1;
        range(s, b0, b1);
        auto inputs = [&]() -> int {                      // the sub-batch's inputs, on cs
            for (int q = 0; q < 7; ++q)
                if (int r = copy_runs(h->io, k[q], host[q], cudaMemcpyHostToDevice, cs, b0, b1)) return r;
            if (subs > 1 && (cudaEventRecord(h->copy_ev[s], cs) != cudaSuccess ||
                             cudaStreamWaitEvent(stream, h->copy_ev[s], 0) != cudaSuccess))
                return DPVO_BA_ECUDA;
            return DPVO_BA_OK;
        };
        // with sub-batches: its descriptors (its own workspace) go on cs ahead
        // of its inputs, so that one copy queue holds them in order
        int rc = subs > 1 ? run_solve(h, dims + b0, dp.data() + b0, b1 - b0, stream, nullptr, nullptr, s, cs, inputs)
                          : (inputs() ? DPVO_BA_ECUDA
                                      : run_solve(h, dims + b0, dp.data() + b0, b1 - b0, stream, nullptr, nullptr));
        if (rc) return rc;
        for (int q : {0, 1})
            if (int rc = copy_runs(h->io, k[q], host[q], cudaMemcpyDeviceToHost, stream, b0, b1)) return rc;
        bool all_status = true;
        for (int b = b0; b < b1; ++b) all_status = all_status && hp[b].status;
        if (all_status) {
            if (int rc = copy_runs(h->io, k[7], host[7], cudaMemcpyDeviceToHost, stream, b0, b1)) return rc;
        } else {
            for (int b = b0; b < b1; ++b)
                if (hp[b].status && cudaMemcpyAsync(hp[b].status, dp[b].status, 4, cudaMemcpyDeviceToHost, stream))
                    return DPVO_BA_ECUDA;
        }
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) return DPVO_BA_ECUDA;
    return DPVO_BA_OK;
}

int dpvo_ba_iterate(dpvo_ba_handle *h, int index, int iter, float *poses_out, float *depth_out,
                    double *dxi_out) {
    if (!h || index < 0 || index >= (int)h->last.size()) return DPVO_BA_EINVAL;
    const Prob &p = h->last[index];
    if (iter < 0 || iter > p.iters) return DPVO_BA_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return DPVO_BA_ECUDA;
    if (poses_out &&
        cudaMemcpy(poses_out, p.pose_it + (size_t)iter * p.N * 7, (size_t)p.N * 7 * 4, cudaMemcpyDeviceToHost))
        return DPVO_BA_ECUDA;
    if (depth_out && p.P &&
        cudaMemcpy(depth_out, p.depth_it + (size_t)iter * p.P, (size_t)p.P * 4, cudaMemcpyDeviceToHost))
        return DPVO_BA_ECUDA;
    if (dxi_out && iter < p.iters && p.nf &&
        cudaMemcpy(dxi_out, p.dxi + (size_t)iter * p.nf * 6, (size_t)p.nf * 6 * 8, cudaMemcpyDeviceToHost))
        return DPVO_BA_ECUDA;
    return DPVO_BA_OK;
}

int dpvo_ba_selftest_bounded_wait(int32_t *status, int arrive, int polls, void *stream) {
    if (!status || polls < 1) return DPVO_BA_EINVAL;
    selftest_wait_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(status, arrive, polls);
    return cudaGetLastError() == cudaSuccess ? DPVO_BA_OK : DPVO_BA_ECUDA;
}

int dpvo_ba_set_timing(dpvo_ba_handle *h, int enable) {
    if (!h) return DPVO_BA_EINVAL;
    h->timing = enable != 0;
    h->ev_used = 0;
    h->ev_kind.clear();
    return DPVO_BA_OK;
}

int dpvo_ba_timing(dpvo_ba_handle *h, float *ms_out, int *kind_out, int cap) {
    if (!h || cap < 0) return DPVO_BA_EINVAL;
    const int launches = (int)h->ev_kind.size();
    if (launches == 0) return 0;
    if (cudaEventSynchronize(h->ev[h->ev_used - 1]) != cudaSuccess) return DPVO_BA_ECUDA;
    const int n = std::min(cap, launches);
    for (int i = 0; i < n; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) != cudaSuccess) return DPVO_BA_ECUDA;
        if (ms_out) ms_out[i] = ms;
        if (kind_out) kind_out[i] = h->ev_kind[i];
    }
    h->ev_used = 0;
    h->ev_kind.clear();
    return n;
}

const char *dpvo_ba_strerror(int code) {
    switch (code) {
        case DPVO_BA_OK: return "ok";
        case DPVO_BA_EINVAL: return "invalid argument";
        case DPVO_BA_ENOMEM: return "out of device memory or over the memory budget";
        case DPVO_BA_ECUDA: return "CUDA runtime error";
        case DPVO_BA_ETIMEOUT: return "timed out";
        case DPVO_BA_EBUSY: return "no serving slot free";
        case DPVO_BA_ENOTFOUND: return "unknown session or ticket";
        default: return "unknown error";
    }
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Serving runtime (see serve.cuh).
// ----------------------------------------------------------------------------
using dpvo_serve::Clock;
using dpvo_serve::Server;
using dpvo_serve::Session;
using dpvo_serve::Slot;
using dpvo_serve::Ticket;

static size_t session_bytes(const dpvo_ba_dims &d) {
    const size_t N = d.n_frames, P = d.n_patches, E = d.n_edges;
    return al256(N * 28) + al256(P * 12) + al256(P * 4) + 2 * al256(E * 4) + 2 * al256(E * 8) + 256;
}

// Factors of every request of a batch, read in place from page-locked host
// memory (jobs[b] for blockIdx.x = b, blocks strided over its edges).
__global__ void serve_gather_kernel(const dpvo_serve::GatherJob *__restrict__ jobs) {
    const dpvo_serve::GatherJob J = jobs[blockIdx.x];
    if (J.mode == 2) return;
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < J.n_edges; e += gridDim.y * blockDim.x) {
        const float2 t = J.src_t[e], w = J.src_w[e];
        if (J.mode == 0) {
            J.dst_t[e] = t;
        } else {
            float2 d = J.dst_t[e];
            d.x += t.x;
            d.y += t.y;
            J.dst_t[e] = d;
        }
        J.dst_w[e] = w;
    }
}

// Every request's status to its page-locked slot (one thread per request).
__global__ void serve_status_kernel(const dpvo_serve::GatherJob *__restrict__ jobs, int n) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) *jobs[b].status_host = *jobs[b].status_dev;
}

static void CUDART_CB serve_batch_done(void *arg) {
    Slot *slot = static_cast<Slot *>(arg);
    Server *srv = slot->srv;
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    for (uint64_t tk : slot->batch) {
        auto it = srv->tickets.find(tk);
        if (it == srv->tickets.end()) continue;
        Ticket &t = it->second;
        auto ss = srv->sessions.find(t.session);
        if (ss != srv->sessions.end()) {
            t.status = *ss->second->pinned_status;
            ss->second->busy = false;
        }
        t.done = true;
        t.done_at = now;
    }
    slot->batch.clear();
    slot->busy = false;
    srv->cv.notify_all();
}

// Launch one batch on a slot: the windows' appends, the factors, the solve, the
// statuses.  Called without the server lock; the batch's sessions are busy, so
// nothing else touches them.
static int serve_launch(Slot *slot, const std::vector<Session *> &ss, const std::vector<Ticket> &tks) {
    const int n = (int)ss.size();
    cudaStream_t st = slot->stream;
    std::vector<dpvo_ba_window *> wins;
    std::vector<const float *> xys;
    std::vector<int> nn;
    for (int b = 0; b < n; ++b)
        if (tks[b].kind == 1) {
            wins.push_back(ss[b]->win);
            xys.push_back(tks[b].src_xy);
            nn.push_back(tks[b].n_new);
        }
    if (!wins.empty()) {
        const int rc = dpvo_ba_window_append_batch(wins.data(), xys.data(), nn.data(), (int)wins.size(), st);
        if (rc) return rc;
    }
    std::vector<dpvo_ba_dims> dims(n);
    std::vector<dpvo_ba_problem> probs(n);
    int e_max = 0;
    for (int b = 0; b < n; ++b) {
        Session *s = ss[b];
        if (s->win) {
            if (dpvo_ba_window_problem(s->win, &dims[b], &probs[b])) return DPVO_BA_ECUDA;
        } else {
            dims[b] = s->dims;
            probs[b] = s->dev;
        }
        dpvo_serve::GatherJob &J = slot->jobs[b];
        J.src_t = reinterpret_cast<const float2 *>(tks[b].src_t);
        J.src_w = reinterpret_cast<const float2 *>(tks[b].src_w);
        J.dst_t = reinterpret_cast<float2 *>(const_cast<float *>(probs[b].target));
        J.dst_w = reinterpret_cast<float2 *>(const_cast<float *>(probs[b].weight));
        J.n_edges = dims[b].n_edges;
        J.mode = tks[b].kind == 0 ? 0 : (tks[b].src_t ? 1 : 2);
        J.status_dev = probs[b].status;
        J.status_host = s->pinned_status;
        e_max = std::max(e_max, J.n_edges);
    }
    const int ys = std::max(1, std::min(64, (e_max + 255) / 256));
    serve_gather_kernel<<<dim3(n, ys), 256, 0, st>>>(slot->jobs);
    int rc = run_solve(slot->h, dims.data(), probs.data(), n, st, nullptr, nullptr);
    if (rc) return rc;
    serve_status_kernel<<<(n + 127) / 128, 128, 0, st>>>(slot->jobs, n);
    if (cudaGetLastError() != cudaSuccess) return DPVO_BA_ECUDA;
    if (cudaLaunchHostFunc(st, serve_batch_done, slot) != cudaSuccess) return DPVO_BA_ECUDA;
    return DPVO_BA_OK;
}

static void serve_loop(Server *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (!srv->stop) {
        Slot *slot = nullptr;
        for (Slot *s : srv->slots)
            if (!s->busy) { slot = s; break; }
        if (!slot || srv->pending.empty()) {
            srv->cv.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        std::vector<uint64_t> batch;
        while (!srv->pending.empty() && (int)batch.size() < srv->max_batch) {
            batch.push_back(srv->pending.front());
            srv->pending.pop_front();
        }
        std::vector<Session *> ss;
        std::vector<Ticket> tks;
        for (uint64_t tk : batch) {
            const Ticket &t = srv->tickets[tk];
            ss.push_back(srv->sessions[t.session]);
            tks.push_back(t);
        }
        slot->busy = true;
        slot->batch = batch;
        lk.unlock();
        const int rc = serve_launch(slot, ss, tks);
        lk.lock();
        if (rc) {
            // could not launch: fail the batch's tickets on the host, free the slot
            srv->launch_error = rc;
            for (uint64_t tk : batch) {
                Ticket &t = srv->tickets[tk];
                t.done = true;
                t.done_at = Clock::now();
                t.status = DPVO_BA_STATUS_BAD_INPUT;
                auto it = srv->sessions.find(t.session);
                if (it != srv->sessions.end()) it->second->busy = false;
            }
            slot->batch.clear();
            slot->busy = false;
            srv->cv.notify_all();
        }
    }
}

static int serve_stop_impl(dpvo_ba_handle *h);

extern "C" int dpvo_ba_serve_start(dpvo_ba_handle *h, const dpvo_ba_dims *max_dims, int max_batch, int max_in_flight) {
    if (!h || !max_dims || max_batch < 1 || max_in_flight < 1 || max_in_flight > 8) return DPVO_BA_EINVAL;
    if (h->srv) return DPVO_BA_EBUSY;
    Server *srv = new Server();
    srv->owner = h;
    srv->device = h->device;
    srv->max_batch = max_batch;
    srv->budget = h->cfg.mem_budget_bytes;
    srv->max_dims = *max_dims;
    h->srv = srv;
    for (int i = 0; i < max_in_flight; ++i) {
        Slot *slot = new Slot();
        slot->srv = srv;
        srv->slots.push_back(slot);
        if (dpvo_ba_create(&h->cfg, &slot->h) != DPVO_BA_OK ||
            cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost((void **)&slot->jobs, sizeof(dpvo_serve::GatherJob) * (size_t)max_batch) != cudaSuccess ||
            dpvo_ba_reserve(slot->h, max_dims, max_batch) != DPVO_BA_OK) {
            cudaGetLastError();
            serve_stop_impl(h);
            return DPVO_BA_ENOMEM;
        }
    }
    srv->running = true;
    srv->thread = std::thread(serve_loop, srv);
    return DPVO_BA_OK;
}

static int serve_stop_impl(dpvo_ba_handle *h) {
    Server *srv = h->srv;
    if (!srv) return DPVO_BA_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv.notify_all();
    }
    if (srv->thread.joinable()) srv->thread.join();
    for (Slot *slot : srv->slots) {
        if (slot->stream) {
            cudaStreamSynchronize(slot->stream);
            cudaStreamDestroy(slot->stream);
        }
        if (slot->h) dpvo_ba_destroy(slot->h);
        if (slot->jobs) cudaFreeHost(slot->jobs);
        delete slot;
    }
    for (auto &kv : srv->sessions) {
        Session *s = kv.second;
        if (s->mem) cudaFree(s->mem);
        if (s->win) dpvo_ba_window_destroy(s->win);
        if (s->pinned_tw) cudaFreeHost(s->pinned_tw);
        delete s;
    }
    delete srv;
    h->srv = nullptr;
    return DPVO_BA_OK;
}

extern "C" int dpvo_ba_serve_stop(dpvo_ba_handle *h) {
    if (!h) return DPVO_BA_EINVAL;
    return serve_stop_impl(h);
}

extern "C" int dpvo_ba_session_open(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *hp,
                                    int64_t *session_id) {
    if (!h || !h->srv || !dims || !hp || !session_id) return DPVO_BA_EINVAL;
    if (int rc = check_dims(*dims)) return rc;
    if (int rc = check_problem(*dims, *hp)) return rc;
    Server *srv = h->srv;
    const size_t bytes = session_bytes(*dims);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->used_bytes + bytes > srv->budget) return DPVO_BA_EBUSY;   // not admitted: over the budget
        srv->used_bytes += bytes;
    }
    Session *s = new Session();
    s->dims = *dims;
    s->bytes = bytes;
    const size_t N = dims->n_frames, P = dims->n_patches, E = dims->n_edges;
    int rc = DPVO_BA_OK;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = DPVO_BA_ECUDA;
    if (!rc && cudaMallocAsync((void **)&s->mem, bytes, st) != cudaSuccess) rc = DPVO_BA_ENOMEM;
    if (!rc && cudaMallocHost((void **)&s->pinned_tw, E * 16 + 16) != cudaSuccess) rc = DPVO_BA_ENOMEM;
    if (!rc) {
        s->pinned_status = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(s->pinned_tw) + E * 16);
        s->max_edges = E;
        size_t o = 0;
        auto take = [&](size_t b) { char *p = s->mem + o; o += al256(b); return p; };
        s->dev.poses = (float *)take(N * 28);
        s->dev.patches = (float *)take(P * 12);
        s->dev.anchor = (const int32_t *)take(P * 4);
        s->dev.kk = (const int32_t *)take(E * 4);
        s->dev.jj = (const int32_t *)take(E * 4);
        s->dev.target = (const float *)take(E * 8);
        s->dev.weight = (const float *)take(E * 8);
        s->dev.status = (int32_t *)take(4);
        cudaMemcpyAsync(s->dev.poses, hp->poses, N * 28, cudaMemcpyHostToDevice, st);
        if (P) {
            cudaMemcpyAsync(s->dev.patches, hp->patches, P * 12, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync((void *)s->dev.anchor, hp->anchor, P * 4, cudaMemcpyHostToDevice, st);
        }
        if (E) {
            cudaMemcpyAsync((void *)s->dev.kk, hp->kk, E * 4, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync((void *)s->dev.jj, hp->jj, E * 4, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync((void *)s->dev.target, hp->target, E * 8, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync((void *)s->dev.weight, hp->weight, E * 8, cudaMemcpyHostToDevice, st);
        }
        cudaMemsetAsync(s->dev.status, 0, 4, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = DPVO_BA_ECUDA;
    }
    if (st) cudaStreamDestroy(st);
    std::lock_guard<std::mutex> lk(srv->mu);
    if (rc) {
        cudaGetLastError();
        if (s->mem) cudaFree(s->mem);
        if (s->pinned_tw) cudaFreeHost(s->pinned_tw);
        delete s;
        srv->used_bytes -= bytes;
        return rc;
    }
    s->id = srv->next_session++;
    srv->sessions[s->id] = s;
    *session_id = s->id;
    return DPVO_BA_OK;
}

static Session *find_idle_session(Server *srv, int64_t id, std::unique_lock<std::mutex> &lk, int timeout_ms,
                                  int *rc) {
    auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = srv->sessions.find(id);
        if (it == srv->sessions.end()) { *rc = DPVO_BA_ENOTFOUND; return nullptr; }
        if (!it->second->busy) { *rc = DPVO_BA_OK; return it->second; }
        if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout) { *rc = DPVO_BA_ETIMEOUT; return nullptr; }
    }
}

extern "C" int dpvo_ba_session_close(dpvo_ba_handle *h, int64_t session_id) {
    if (!h || !h->srv) return DPVO_BA_EINVAL;
    Server *srv = h->srv;
    std::unique_lock<std::mutex> lk(srv->mu);
    int rc;
    Session *s = find_idle_session(srv, session_id, lk, 10000, &rc);
    if (!s) return rc;
    srv->sessions.erase(session_id);
    srv->used_bytes -= s->bytes;
    lk.unlock();
    if (s->mem) cudaFree(s->mem);
    if (s->win) dpvo_ba_window_destroy(s->win);
    cudaFreeHost(s->pinned_tw);
    delete s;
    return DPVO_BA_OK;
}

extern "C" int dpvo_ba_session_read(dpvo_ba_handle *h, int64_t session_id, float *poses_out, float *patches_out) {
    if (!h || !h->srv) return DPVO_BA_EINVAL;
    Server *srv = h->srv;
    std::unique_lock<std::mutex> lk(srv->mu);
    int rc;
    Session *s = find_idle_session(srv, session_id, lk, 10000, &rc);
    if (!s) return rc;
    s->busy = true;        // hold it while copying
    lk.unlock();
    dpvo_ba_dims d = s->dims;
    dpvo_ba_problem p = s->dev;
    if (s->win && dpvo_ba_window_problem(s->win, &d, &p) != DPVO_BA_OK) d.n_frames = d.n_patches = 0;
    if (poses_out && d.n_frames && cudaMemcpy(poses_out, p.poses, (size_t)d.n_frames * 28, cudaMemcpyDeviceToHost))
        rc = DPVO_BA_ECUDA;
    if (patches_out && d.n_patches &&
        cudaMemcpy(patches_out, p.patches, (size_t)d.n_patches * 12, cudaMemcpyDeviceToHost))
        rc = DPVO_BA_ECUDA;
    lk.lock();
    s->busy = false;
    srv->cv.notify_all();
    return rc;
}

// Host memory the device can read in place (page-locked: cudaMallocHost,
// cudaHostAlloc or cudaHostRegister).
static bool page_locked(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

// Queue a ticket for an idle session marked busy by the caller.
static uint64_t enqueue(Server *srv, Ticket tk) {
    std::lock_guard<std::mutex> lk(srv->mu);
    const uint64_t t = srv->next_ticket++;
    tk.submitted = Clock::now();
    srv->tickets[t] = tk;
    srv->pending.push_back(t);
    srv->cv.notify_all();
    return t;
}

static Session *claim_session(Server *srv, int64_t id, bool window, int *rc) {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->sessions.find(id);
    if (it == srv->sessions.end()) { *rc = DPVO_BA_ENOTFOUND; return nullptr; }
    Session *s = it->second;
    if ((s->win != nullptr) != window) { *rc = DPVO_BA_EINVAL; return nullptr; }
    if (s->busy) { *rc = DPVO_BA_EBUSY; return nullptr; }   // one request per session at a time
    s->busy = true;
    *rc = DPVO_BA_OK;
    return s;
}

static void release_session(Server *srv, Session *s) {
    std::lock_guard<std::mutex> lk(srv->mu);
    s->busy = false;
    srv->cv.notify_all();
}

extern "C" int dpvo_ba_submit(dpvo_ba_handle *h, int64_t session_id, const float *target, const float *weight,
                              uint64_t *ticket) {
    if (!h || !h->srv || !ticket) return DPVO_BA_EINVAL;
    Server *srv = h->srv;
    int rc;
    Session *s = claim_session(srv, session_id, false, &rc);
    if (!s) return rc;
    const size_t E = s->dims.n_edges;
    if (E && (!target || !weight)) {
        release_session(srv, s);
        return DPVO_BA_EINVAL;
    }
    Ticket tk;
    tk.session = session_id;
    tk.kind = 0;
    tk.src_t = s->pinned_tw;
    tk.src_w = s->pinned_tw + 2 * E;
    if (E) {   // page-locked buffers are read in place; others are copied to the staging
        if (page_locked(target)) tk.src_t = target;
        else std::memcpy(s->pinned_tw, target, E * 8);
        if (page_locked(weight)) tk.src_w = weight;
        else std::memcpy(s->pinned_tw + 2 * E, weight, E * 8);
    }
    *ticket = enqueue(srv, tk);
    return DPVO_BA_OK;
}

extern "C" int dpvo_ba_session_open_window(dpvo_ba_handle *h, const dpvo_ba_window_params *params,
                                           int64_t *session_id) {
    if (!h || !h->srv || !params || !session_id) return DPVO_BA_EINVAL;
    Server *srv = h->srv;
    const dpvo_ba_dims &mx = srv->max_dims;
    const size_t max_p = (size_t)params->max_frames * (size_t)params->max_new_patches;
    const size_t max_e = dpvo_win_host::max_edges(*params);
    if (params->max_frames > mx.n_frames || max_p > (size_t)mx.n_patches || max_e > (size_t)mx.n_edges ||
        params->n_iters > mx.n_iters)
        return DPVO_BA_EINVAL;   // the slots' workspaces are reserved for max_dims
    const size_t bytes = dpvo_win_host::device_bytes(*params);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->used_bytes + bytes > srv->budget) return DPVO_BA_EBUSY;   // not admitted: over the budget
        srv->used_bytes += bytes;
    }
    Session *s = new Session();
    s->bytes = bytes;
    s->wprm = *params;
    s->max_edges = max_e;
    int rc = dpvo_ba_window_create(params, &s->win);
    if (!rc && cudaMallocHost((void **)&s->pinned_tw, max_e * 16 + (size_t)params->max_new_patches * 8 + 16) !=
                   cudaSuccess) {
        cudaGetLastError();
        rc = DPVO_BA_ENOMEM;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (rc) {
        if (s->win) dpvo_ba_window_destroy(s->win);
        if (s->pinned_tw) cudaFreeHost(s->pinned_tw);
        delete s;
        srv->used_bytes -= bytes;
        return rc;
    }
    s->pinned_xy = s->pinned_tw + 4 * max_e;
    s->pinned_status = reinterpret_cast<int32_t *>(s->pinned_xy + 2 * (size_t)params->max_new_patches);
    s->id = srv->next_session++;
    srv->sessions[s->id] = s;
    *session_id = s->id;
    return DPVO_BA_OK;
}

extern "C" int dpvo_ba_session_frame_edges(dpvo_ba_handle *h, int64_t session_id, int n_new, int32_t *n_edges) {
    if (!h || !h->srv || !n_edges) return DPVO_BA_EINVAL;
    Server *srv = h->srv;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->sessions.find(session_id);
    if (it == srv->sessions.end()) return DPVO_BA_ENOTFOUND;
    Session *s = it->second;
    if (!s->win || n_new < 0 || n_new > s->wprm.max_new_patches) return DPVO_BA_EINVAL;
    if (s->busy) return DPVO_BA_EBUSY;     // its frame count changes when the pending request runs
    *n_edges = dpvo_win_host::edges_after(s->win, n_new);
    return DPVO_BA_OK;
}

extern "C" int dpvo_ba_session_dims(dpvo_ba_handle *h, int64_t session_id, dpvo_ba_dims *dims) {
    if (!h || !h->srv || !dims) return DPVO_BA_EINVAL;
    Server *srv = h->srv;
    std::unique_lock<std::mutex> lk(srv->mu);
    int rc;
    Session *s = find_idle_session(srv, session_id, lk, 10000, &rc);
    if (!s) return rc;
    if (!s->win) {
        *dims = s->dims;
        return DPVO_BA_OK;
    }
    dpvo_ba_problem p;
    if (dpvo_ba_window_problem(s->win, dims, &p) != DPVO_BA_OK) {   // an empty window
        int N, P, E;
        dpvo_win_host::sizes(s->win, &N, &P, &E);
        *dims = dpvo_ba_dims{N, P, E, 0, s->wprm.n_iters, s->wprm.fx, s->wprm.fy, s->wprm.cx, s->wprm.cy};
    }
    return DPVO_BA_OK;
}

extern "C" int dpvo_ba_submit_frame(dpvo_ba_handle *h, int64_t session_id, const float *new_xy, int n_new,
                                    const float *delta, const float *weight, uint64_t *ticket) {
    if (!h || !h->srv || !ticket || (delta == nullptr) != (weight == nullptr)) return DPVO_BA_EINVAL;
    Server *srv = h->srv;
    int rc;
    Session *s = claim_session(srv, session_id, true, &rc);
    if (!s) return rc;
    if (n_new < 0 || n_new > s->wprm.max_new_patches || (n_new > 0 && !new_xy)) {
        release_session(srv, s);
        return DPVO_BA_EINVAL;
    }
    const size_t E = (size_t)dpvo_win_host::edges_after(s->win, n_new);   // the session is ours: mirror stable
    Ticket tk;
    tk.session = session_id;
    tk.kind = 1;
    tk.n_new = n_new;
    tk.src_xy = s->pinned_xy;
    if (n_new) {
        if (page_locked(new_xy)) tk.src_xy = new_xy;
        else std::memcpy(s->pinned_xy, new_xy, (size_t)n_new * 8);
    }
    if (delta) {
        tk.src_t = s->pinned_tw;
        tk.src_w = s->pinned_tw + 2 * E;
        if (E) {
            if (page_locked(delta)) tk.src_t = delta;
            else std::memcpy(s->pinned_tw, delta, E * 8);
            if (page_locked(weight)) tk.src_w = weight;
            else std::memcpy(s->pinned_tw + 2 * E, weight, E * 8);
        }
    }
    *ticket = enqueue(srv, tk);
    return DPVO_BA_OK;
}

static int collect(Server *srv, uint64_t ticket, int32_t *status, double *latency_ms) {
    auto it = srv->tickets.find(ticket);
    const Ticket &t = it->second;
    if (status) *status = t.status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(t.done_at - t.submitted).count();
    srv->tickets.erase(it);
    return DPVO_BA_OK;
}

extern "C" int dpvo_ba_poll(dpvo_ba_handle *h, uint64_t ticket, int32_t *status, double *latency_ms) {
    if (!h || !h->srv) return DPVO_BA_EINVAL;
    std::lock_guard<std::mutex> lk(h->srv->mu);
    auto it = h->srv->tickets.find(ticket);
    if (it == h->srv->tickets.end()) return DPVO_BA_ENOTFOUND;
    if (!it->second.done) return DPVO_BA_EBUSY;
    return collect(h->srv, ticket, status, latency_ms);
}

extern "C" int dpvo_ba_wait(dpvo_ba_handle *h, uint64_t ticket, int timeout_ms, int32_t *status,
                            double *latency_ms) {
    if (!h || !h->srv || timeout_ms < 0) return DPVO_BA_EINVAL;
    Server *srv = h->srv;
    std::unique_lock<std::mutex> lk(srv->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = srv->tickets.find(ticket);
        if (it == srv->tickets.end()) return DPVO_BA_ENOTFOUND;
        if (it->second.done) return collect(srv, ticket, status, latency_ms);
        if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = srv->tickets.find(ticket);
            if (it2 != srv->tickets.end() && it2->second.done) return collect(srv, ticket, status, latency_ms);
            return DPVO_BA_ETIMEOUT;
        }
    }
}

// ----------------------------------------------------------------------------
// Allocation-free single-problem solve.
//
// Some callers may not allocate device memory once they are running: a VO
// pipeline on an embedded GPU whose memory is fixed at start-up, a process
// whose device memory belongs to another allocator (a framework's caching
// allocator or a pre-sized pool), or a real-time frame loop that cannot take
// cudaMalloc's implicit device synchronisation.  dpvo_ba_solve_noalloc()
// serves them: its workspace lives in the fixed array below, which every GPU
// that loads this library holds until the process exits.  It makes no host or
// device allocation: the layout of its one problem is computed on the stack,
// and its descriptors reach the device as kernel arguments.
// ----------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;   // 8 MiB per device
}

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code g_noalloc_scratch names a host-side stand-in, not the device
// array: every call asks the runtime for the array's device address in the
// current context (cudaGetSymbolAddress) and passes that to the kernels.

__global__ void noalloc_descriptors_kernel(Prob p, int n_items, Prob *dst_prob, Item *dst_items) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *dst_prob = p;
    for (int w = threadIdx.x; w < n_items; w += blockDim.x) dst_items[w] = Item{0, w};
}

extern "C" int dpvo_ba_solve_noalloc(const dpvo_ba_config *cfg, const dpvo_ba_dims *dims,
                                     const dpvo_ba_problem *prob, void *stream_) {
    if (!dims || !prob) return DPVO_BA_EINVAL;
    if (int rc = check_dims(*dims)) return rc;
    if (int rc = check_problem(*dims, *prob)) return rc;
    if (dims->n_frames - dims->t0 > kFusedMaxFree) return DPVO_BA_EINVAL;   // no assembly kernel on this path
    cudaStream_t stream = (cudaStream_t)stream_;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return DPVO_BA_ECUDA; }
    cudaGetLastError();   // an error left pending by earlier, unrelated work is not this call's
    // Looked up on every call, with the caller's device current: the array's
    // address belongs to the current context and moves if that context is torn
    // down and created again; once the module is loaded the lookup allocates nothing.
    char *base = nullptr;
    {
        void *q = nullptr;
        if (cudaGetSymbolAddress(&q, g_noalloc_scratch) != cudaSuccess || !q) {
            cudaGetLastError();
            return DPVO_BA_ECUDA;
        }
        base = (char *)q;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return DPVO_BA_ECUDA;
    }
    if (set_kernel_attrs(dev)) return DPVO_BA_ECUDA;
    const float damping = cfg ? cfg->damping : 1e-4f;
    const float z_min = cfg ? cfg->z_min : 0.1f;
    if (!(damping >= 0.f) || !(z_min == z_min)) return DPVO_BA_EINVAL;

    // layout of one problem (same formulas as the handle path), on the stack
    const dpvo_ba_dims &d = *dims;
    const int nf = d.n_frames - d.t0;
    const int W_cap = std::min(d.n_frames, kMaxWindow);
    const bool tc = cfg && cfg->schur_tf32 == 1 && use_tensor_cores(nf);
    int G_cap = 64;
    while (G_cap > 8 && lin_smem_layout(W_cap, G_cap, nf, d.n_frames, tc).bytes > kLinSmemBudget) G_cap -= 8;
    const size_t lin_smem = lin_smem_layout(W_cap, G_cap, nf, d.n_frames, tc).bytes;
    const size_t solve_smem = sw_smem_bytes(nf);
    Prob p;
    std::memset(&p, 0, sizeof(Prob));
    p.poses = prob->poses; p.patches = prob->patches; p.anchor = prob->anchor; p.kk = prob->kk;
    p.jj = prob->jj; p.target = prob->target; p.weight = prob->weight; p.status_user = prob->status;
    p.bulk_edges = aligned16(prob->jj, prob->target, prob->weight);
    p.N = d.n_frames; p.P = d.n_patches; p.E = d.n_edges; p.t0 = d.t0; p.iters = d.n_iters; p.nf = nf;
    p.fx = d.fx; p.fy = d.fy; p.cx = d.cx; p.cy = d.cy;
    p.damping = damping; p.z_min = z_min;
    p.solve_f64 = cfg && cfg->reduced_solve_f64 ? 1 : 0;
    p.chunk_cap = G_cap;
    p.win_cap = W_cap;
    p.max_chunks = (d.n_patches + G_cap - 1) / G_cap + d.n_frames;
    p.ks = tc ? 1 : k_split(nf);
    p.L = partial_len(nf);
    p.n_items = std::max(1, std::min(2 * sms, p.max_chunks));   // at most one item per chunk
    p.n_parts = p.n_items;
    size_t off = 0;
    auto take = [&](size_t bytes) { char *q = base + off; off = al256(off + bytes); return q; };
    p.seg = (int32_t *)take((size_t)(d.n_patches + 1) * 4);
    p.chunks = (Chunk *)take((size_t)p.max_chunks * sizeof(Chunk));
    char *ints = take(16);
    p.n_chunks = (int32_t *)ints;
    p.status = (int32_t *)(ints + 4);
    p.pose_it = (float *)take((size_t)(d.n_iters + 1) * d.n_frames * 7 * 4);
    p.depth_it = (float *)take((size_t)(d.n_iters + 1) * d.n_patches * 4);
    p.dxi = (double *)take((size_t)d.n_iters * nf * 6 * 8 + 8);
    p.partial = (double *)take((size_t)p.n_items * p.L * 8 + 8);
    p.erow = (float *)take(erow_bytes(tc, p, G_cap));
    Prob *d_prob = (Prob *)take(sizeof(Prob));
    Item *d_items = (Item *)take(sizeof(Item) * p.n_items);
    if (off > kNoAllocScratchBytes) return DPVO_BA_EINVAL;   // problem too large for the fixed scratch

    Layout lay;   // launch shapes only (no workspace from it)
    lay.tc = tc;
    lay.W_cap = W_cap;
    lay.G_cap = G_cap;
    lay.nf_max = nf;
    lay.n_max = d.n_frames;
    lay.lin_smem = lin_smem;
    lay.final_slices = final_slices_of(tc, d.n_patches, p.max_chunks, 65535);
    noalloc_descriptors_kernel<<<1, kThreads, 0, stream>>>(p, p.n_items, d_prob, d_items);
    launch_plan(1, d.n_edges, sms, stream, d_prob);
    for (int t = 0; t < d.n_iters; ++t) {
        launch_linearize(lay, p.n_items, stream, d_prob, d_items, t, 0);
        launch_solve_warp(nf, p.n_parts, 1, stream, d_prob, t, solve_smem);
    }
    launch_final(lay, 1, stream, d_prob, d.n_iters);
    if (cudaGetLastError() != cudaSuccess) return DPVO_BA_ECUDA;
    return DPVO_BA_OK;
}
