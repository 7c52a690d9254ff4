// Window maintenance of the VO system (Sec. 3.3 "Expansion", "Optimization"):
// append a frame to a sliding optimisation window kept on the device.
//
// Layout: poses, patches and anchors live in two sets (the append reads one
// and writes the other, so dropping the oldest frame is a shifted copy); the
// edge arrays are regenerated in place.  The host keeps the per-frame patch
// counts, from which it computes every size and offset the kernel needs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "dpvo_ba.h"
#include "window_host.h"

namespace dpvo_win {

constexpr int kThreads = 256;

struct Args {
    const float *pose_in, *patch_in;
    const int32_t *anchor_in, *counts_in;
    float *pose_out, *patch_out;
    int32_t *anchor_out, *counts_out, *table, *kk, *jj;   // table: [f_first | e_first], N2 + 1 each
    float *target, *weight;
    const float *new_xy;
    int N, drop, c0, n_new, R, N2, P_keep, P2, med_lo, med_n;
    float fx, fy, cx, cy;
};
constexpr int kMaxBatch = 128;                  // windows per launch (kernel parameter space)
struct Batch {
    Args a[kMaxBatch];
};

// Hamilton product, quaternions x y z w, FP64.
__device__ inline void qmul(const double *a, const double *b, double *o) {
    o[0] = a[3] * b[0] + b[3] * a[0] + a[1] * b[2] - a[2] * b[1];
    o[1] = a[3] * b[1] + b[3] * a[1] + a[2] * b[0] - a[0] * b[2];
    o[2] = a[3] * b[2] + b[3] * a[2] + a[0] * b[1] - a[1] * b[0];
    o[3] = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
}
// v' = q v q^*
__device__ inline void qrot(const double *q, const double *v, double *o) {
    const double p[4] = {v[0], v[1], v[2], 0.0}, qc[4] = {-q[0], -q[1], -q[2], q[3]};
    double t[4], r[4];
    qmul(q, p, t);
    qmul(t, qc, r);
    o[0] = r[0]; o[1] = r[1]; o[2] = r[2];
}

// Phase A, one CTA per window: the median inverse depth, the new pose, the
// shifted copies, the new patches, the per-frame counts and offsets.
__global__ void __launch_bounds__(kThreads) append_state_kernel(Batch B) {
    const Args &A = B.a[blockIdx.x];
    extern __shared__ float s_d[];               // the median's candidates
    __shared__ float s_med;
    __shared__ float s_pose[7];
    const int tid = threadIdx.x;
    // median inverse depth of the patches of the previous 3 frames (lower median)
    if (tid == 0) s_med = 1.f;
    for (int q = tid; q < A.med_n; q += kThreads) s_d[q] = A.patch_in[3 * (A.med_lo + q) + 2];
    __syncthreads();
    if (A.med_n > 0) {
        const int r = (A.med_n - 1) / 2;
        for (int q = tid; q < A.med_n; q += kThreads) {
            const float v = s_d[q];
            int lt = 0, le = 0;
            for (int u = 0; u < A.med_n; ++u) {
                lt += s_d[u] < v;
                le += s_d[u] <= v;
            }
            if (lt <= r && r < le) s_med = v;     // every writer holds the same value
        }
    }
    // the new frame's pose: constant velocity
    if (tid == 0) {
        double q[4] = {0.0, 0.0, 0.0, 1.0}, t[3] = {0.0, 0.0, 0.0};
        if (A.N == 1) {
            for (int k = 0; k < 3; ++k) t[k] = A.pose_in[k];
            for (int k = 0; k < 4; ++k) q[k] = A.pose_in[3 + k];
        } else if (A.N >= 2) {
            const float *P1 = A.pose_in + 7 * (A.N - 1), *P2 = A.pose_in + 7 * (A.N - 2);
            const double q1[4] = {P1[3], P1[4], P1[5], P1[6]}, q2c[4] = {-P2[3], -P2[4], -P2[5], P2[6]};
            double m[4];
            qmul(q1, q2c, m);                     // R1 R2^T
            qmul(m, q1, q);                       // R1 R2^T R1
            const double d[3] = {(double)P1[0] - P2[0], (double)P1[1] - P2[1], (double)P1[2] - P2[2]};
            double rd[3];
            qrot(m, d, rd);                       // R1 R2^T (t1 - t2)
            for (int k = 0; k < 3; ++k) t[k] = P1[k] + rd[k];
        }
        const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int k = 0; k < 3; ++k) s_pose[k] = (float)t[k];
        for (int k = 0; k < 4; ++k) s_pose[3 + k] = (float)(q[k] / n);
    }
    __syncthreads();
    // shifted copies of the kept frames and patches, then the new frame and patches
    for (int q = tid; q < 7 * (A.N2 - 1); q += kThreads) A.pose_out[q] = A.pose_in[q + 7 * A.drop];
    if (tid < 7) A.pose_out[7 * (A.N2 - 1) + tid] = s_pose[tid];
    for (int k = tid; k < A.P_keep; k += kThreads) {
        const int ks = k + A.c0;
        A.patch_out[3 * k] = A.patch_in[3 * ks];
        A.patch_out[3 * k + 1] = A.patch_in[3 * ks + 1];
        A.patch_out[3 * k + 2] = A.patch_in[3 * ks + 2];
        A.anchor_out[k] = A.anchor_in[ks] - A.drop;
    }
    for (int m = tid; m < A.n_new; m += kThreads) {
        const int k = A.P_keep + m;
        A.patch_out[3 * k] = A.new_xy[2 * m];
        A.patch_out[3 * k + 1] = A.new_xy[2 * m + 1];
        A.patch_out[3 * k + 2] = s_med;
        A.anchor_out[k] = A.N2 - 1;
    }
    // per-frame patch counts, first patch and first edge of each frame
    for (int f = tid; f < A.N2; f += kThreads) A.counts_out[f] = f < A.N2 - 1 ? A.counts_in[f + A.drop] : A.n_new;
    __syncthreads();
    if (tid == 0) {
        int p = 0, e = 0;
        for (int f = 0; f < A.N2; ++f) {
            A.table[f] = p;
            A.table[A.N2 + 1 + f] = e;
            const int c = A.counts_out[f];
            p += c;
            e += c * (min(A.N2 - 1, f + A.R) - max(0, f - A.R) + 1);
        }
        A.table[A.N2] = p;
        A.table[2 * A.N2 + 1] = e;
    }
}

// Phase B, blockIdx.y slices of the patches: every edge of a patch (its frames
// within the radius, increasing) with the reprojection target (Eq. 2), FP32.
__global__ void __launch_bounds__(kThreads) append_edges_kernel(Batch B) {
    const Args &A = B.a[blockIdx.x];
    const int tid = threadIdx.x;
    const int k0 = blockIdx.y * kThreads;
    if (k0 >= A.P2) return;
    __shared__ float s_R[DPVO_BA_MAX_FRAMES][9], s_t[DPVO_BA_MAX_FRAMES][3];
    for (int f = tid; f < A.N2; f += kThreads) {
        const float *P = A.pose_out + 7 * f;
        const float x = P[3], y = P[4], z = P[5], w = P[6];
        float *R = s_R[f];
        R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
        R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
        R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
        s_t[f][0] = P[0];
        s_t[f][1] = P[1];
        s_t[f][2] = P[2];
    }
    __syncthreads();
    const int k = k0 + tid;
    if (k >= A.P2) return;
    const int a = A.anchor_out[k];
    const int jlo = max(0, a - A.R), jhi = min(A.N2 - 1, a + A.R);
    const int base = A.table[A.N2 + 1 + a] + (k - A.table[a]) * (jhi - jlo + 1);
    const float x = A.patch_out[3 * k], y = A.patch_out[3 * k + 1], d = A.patch_out[3 * k + 2];
    // the point in camera a is (xbar, ybar, 1) / d; in the world, scaled by d:
    // d X_w = R_a^T ((xbar, ybar, 1) - d t_a)
    const float *Ra = s_R[a];
    const float u0 = (x - A.cx) / A.fx - d * s_t[a][0], u1 = (y - A.cy) / A.fy - d * s_t[a][1],
                u2 = 1.f - d * s_t[a][2];
    const float w0 = Ra[0] * u0 + Ra[3] * u1 + Ra[6] * u2, w1 = Ra[1] * u0 + Ra[4] * u1 + Ra[7] * u2,
                w2 = Ra[2] * u0 + Ra[5] * u1 + Ra[8] * u2;
    for (int j = jlo; j <= jhi; ++j) {
        const int e = base + (j - jlo);
        A.kk[e] = k;
        A.jj[e] = j;
        float tx = x, ty = y;
        if (j != a) {
            const float *Rj = s_R[j];            // d X_j = R_j (d X_w) + d t_j
            const float c0 = Rj[0] * w0 + Rj[1] * w1 + Rj[2] * w2 + d * s_t[j][0];
            const float c1 = Rj[3] * w0 + Rj[4] * w1 + Rj[5] * w2 + d * s_t[j][1];
            const float c2 = Rj[6] * w0 + Rj[7] * w1 + Rj[8] * w2 + d * s_t[j][2];
            if (c2 > 1e-9f) {
                tx = A.fx * c0 / c2 + A.cx;
                ty = A.fy * c1 / c2 + A.cy;
            }
        }
        A.target[2 * e] = tx;
        A.target[2 * e + 1] = ty;
        A.weight[2 * e] = 1.f;
        A.weight[2 * e + 1] = 1.f;
    }
}

}  // namespace dpvo_win

struct dpvo_ba_window {
    dpvo_ba_window_params prm{};
    int N = 0, P = 0, E = 0, cur = 0;
    bool broken = false;                          // a launch failed after the mirror moved on: unusable
    std::vector<int> counts;                      // patches per frame, oldest first (host mirror)
    char *mem = nullptr;
    float *pose[2] = {nullptr, nullptr}, *patch[2] = {nullptr, nullptr};
    int32_t *anchor[2] = {nullptr, nullptr}, *dcounts[2] = {nullptr, nullptr};
    int32_t *table = nullptr, *kk = nullptr, *jj = nullptr, *status = nullptr;
    float *target = nullptr, *weight = nullptr;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// The median of a new frame's inverse depth ranks the patches of the previous
// 3 frames in shared memory (4 bytes each, at most 96 KiB).
constexpr int kMaxNewPatches = 96 * 1024 / 4 / 3;

static int edges_per_patch(int f, int N, int R) {
    const int lo = f - R < 0 ? 0 : f - R, hi = f + R > N - 1 ? N - 1 : f + R;
    return hi - lo + 1;
}

// Device layout of a window: offsets of its arrays (take() order) and total bytes.
struct WinLayout {
    size_t o_pose0, o_pose1, o_patch0, o_patch1, o_anc0, o_anc1, o_cnt0, o_cnt1, o_tab, o_kk, o_jj, o_tg, o_wt, o_st,
        bytes, edges;
};

static WinLayout win_layout(const dpvo_ba_window_params &p) {
    WinLayout L;
    const size_t F = (size_t)p.max_frames, Pc = F * (size_t)p.max_new_patches;
    const size_t span = (size_t)(2 * p.radius + 1) < F ? (size_t)(2 * p.radius + 1) : F;
    const size_t Ec = Pc * span;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = al256(off + b); return o; };
    L.o_pose0 = take(F * 28); L.o_pose1 = take(F * 28); L.o_patch0 = take(Pc * 12 + 4);
    L.o_patch1 = take(Pc * 12 + 4); L.o_anc0 = take(Pc * 4 + 4); L.o_anc1 = take(Pc * 4 + 4);
    L.o_cnt0 = take(F * 4); L.o_cnt1 = take(F * 4); L.o_tab = take((2 * F + 2) * 4);
    L.o_kk = take(Ec * 4 + 4); L.o_jj = take(Ec * 4 + 4); L.o_tg = take(Ec * 8 + 8); L.o_wt = take(Ec * 8 + 8);
    L.o_st = take(16);
    L.bytes = off;
    L.edges = Ec;
    return L;
}

namespace dpvo_win_host {
size_t device_bytes(const dpvo_ba_window_params &p) { return win_layout(p).bytes; }
size_t max_edges(const dpvo_ba_window_params &p) { return win_layout(p).edges; }
int edges_after(const dpvo_ba_window *w, int n_new) {
    const int drop = w->N == w->prm.max_frames ? 1 : 0;
    std::vector<int> cnt(w->counts.begin() + drop, w->counts.end());
    cnt.push_back(n_new);
    const int N2 = (int)cnt.size();
    int E2 = 0;
    for (int f = 0; f < N2; ++f) E2 += cnt[f] * edges_per_patch(f, N2, w->prm.radius);
    return E2;
}
void sizes(const dpvo_ba_window *w, int *n_frames, int *n_patches, int *n_edges) {
    *n_frames = w->N;
    *n_patches = w->P;
    *n_edges = w->E;
}
}  // namespace dpvo_win_host

extern "C" int dpvo_ba_window_create(const dpvo_ba_window_params *p, dpvo_ba_window **out) {
    if (!p || !out || p->max_frames < 1 || p->max_frames > DPVO_BA_MAX_FRAMES || p->max_new_patches < 0 ||
        p->max_new_patches > kMaxNewPatches || p->radius < 0 || p->free_poses < 0 || p->n_iters < 1 || p->n_iters > DPVO_BA_MAX_ITERS)
        return DPVO_BA_EINVAL;
    dpvo_ba_window *w = new (std::nothrow) dpvo_ba_window;
    if (!w) return DPVO_BA_ENOMEM;
    w->prm = *p;
    const WinLayout WL = win_layout(*p);
    const size_t off = WL.bytes;
    const size_t o_pose0 = WL.o_pose0, o_pose1 = WL.o_pose1, o_patch0 = WL.o_patch0, o_patch1 = WL.o_patch1,
                 o_anc0 = WL.o_anc0, o_anc1 = WL.o_anc1, o_cnt0 = WL.o_cnt0, o_cnt1 = WL.o_cnt1, o_tab = WL.o_tab,
                 o_kk = WL.o_kk, o_jj = WL.o_jj, o_tg = WL.o_tg, o_wt = WL.o_wt, o_st = WL.o_st;
    if (cudaMalloc(&w->mem, off) != cudaSuccess) {
        delete w;
        return DPVO_BA_ENOMEM;
    }
    w->pose[0] = (float *)(w->mem + o_pose0);
    w->pose[1] = (float *)(w->mem + o_pose1);
    w->patch[0] = (float *)(w->mem + o_patch0);
    w->patch[1] = (float *)(w->mem + o_patch1);
    w->anchor[0] = (int32_t *)(w->mem + o_anc0);
    w->anchor[1] = (int32_t *)(w->mem + o_anc1);
    w->dcounts[0] = (int32_t *)(w->mem + o_cnt0);
    w->dcounts[1] = (int32_t *)(w->mem + o_cnt1);
    w->table = (int32_t *)(w->mem + o_tab);
    w->kk = (int32_t *)(w->mem + o_kk);
    w->jj = (int32_t *)(w->mem + o_jj);
    w->target = (float *)(w->mem + o_tg);
    w->weight = (float *)(w->mem + o_wt);
    w->status = (int32_t *)(w->mem + o_st);
    if (cudaMemset(w->mem, 0, off) != cudaSuccess) {
        cudaFree(w->mem);
        delete w;
        return DPVO_BA_ECUDA;
    }
    *out = w;
    return 0;
}

extern "C" int dpvo_ba_window_destroy(dpvo_ba_window *w) {
    if (!w) return DPVO_BA_EINVAL;
    cudaDeviceSynchronize();
    cudaFree(w->mem);
    delete w;
    return 0;
}

// Host side of one window's append: the launch arguments, and the host mirror
// advanced to the new sizes.
static void plan_append(dpvo_ba_window *w, const float *new_xy, int n_new, dpvo_win::Args &A) {
    const int R = w->prm.radius;
    std::memset(&A, 0, sizeof(A));
    const int drop = w->N == w->prm.max_frames ? 1 : 0;
    const int c0 = drop ? w->counts[0] : 0;
    int med_lo = 0;                               // the previous 3 frames' patches: [med_lo, P)
    for (int f = 0; f < w->N - 3; ++f) med_lo += w->counts[f];
    std::vector<int> cnt(w->counts.begin() + drop, w->counts.end());
    cnt.push_back(n_new);
    const int N2 = (int)cnt.size();
    int P2 = 0, E2 = 0;
    for (int f = 0; f < N2; ++f) {
        P2 += cnt[f];
        E2 += cnt[f] * edges_per_patch(f, N2, R);
    }
    const int nx = w->cur ^ 1;
    A.pose_in = w->pose[w->cur];
    A.patch_in = w->patch[w->cur];
    A.anchor_in = w->anchor[w->cur];
    A.counts_in = w->dcounts[w->cur];
    A.pose_out = w->pose[nx];
    A.patch_out = w->patch[nx];
    A.anchor_out = w->anchor[nx];
    A.counts_out = w->dcounts[nx];
    A.table = w->table;
    A.kk = w->kk;
    A.jj = w->jj;
    A.target = w->target;
    A.weight = w->weight;
    A.new_xy = new_xy;
    A.N = w->N;
    A.drop = drop;
    A.c0 = c0;
    A.n_new = n_new;
    A.R = R;
    A.N2 = N2;
    A.P_keep = w->P - c0;
    A.P2 = P2;
    A.med_lo = med_lo;
    A.med_n = w->P - med_lo;
    A.fx = w->prm.fx;
    A.fy = w->prm.fy;
    A.cx = w->prm.cx;
    A.cy = w->prm.cy;
    w->counts.swap(cnt);
    w->N = N2;
    w->P = P2;
    w->E = E2;
    w->cur = nx;
}

extern "C" int dpvo_ba_window_append_batch(dpvo_ba_window *const *ws, const float *const *new_xy, const int *n_new,
                                          int n, void *stream) {
    if (n < 0 || (n > 0 && (!ws || !new_xy || !n_new))) return DPVO_BA_EINVAL;
    // every check comes before any window's host mirror moves on
    for (int b = 0; b < n; ++b) {
        const dpvo_ba_window *w = ws[b];
        if (!w || n_new[b] < 0 || n_new[b] > w->prm.max_new_patches || (n_new[b] > 0 && !new_xy[b]))
            return DPVO_BA_EINVAL;
        if (w->broken) return DPVO_BA_ECUDA;
        for (int c = 0; c < b; ++c)
            if (ws[c] == w) return DPVO_BA_EINVAL;   // one append per window per call
    }
    // the median candidates of any window fit in 96 KiB (max_new_patches is bounded at create)
    if (n > 0 && cudaFuncSetAttribute(dpvo_win::append_state_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      96 * 1024) != cudaSuccess) {
        cudaGetLastError();
        return DPVO_BA_ECUDA;
    }
    cudaGetLastError();                            // report only this call's launch errors
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int b0 = 0; b0 < n; b0 += dpvo_win::kMaxBatch) {
        const int nb = n - b0 < dpvo_win::kMaxBatch ? n - b0 : dpvo_win::kMaxBatch;
        dpvo_win::Batch B;
        int med_max = 0, p_max = 0;
        for (int b = 0; b < nb; ++b) {
            plan_append(ws[b0 + b], new_xy[b0 + b], n_new[b0 + b], B.a[b]);
            med_max = B.a[b].med_n > med_max ? B.a[b].med_n : med_max;
            p_max = B.a[b].P2 > p_max ? B.a[b].P2 : p_max;
        }
        const size_t smem = (size_t)med_max * 4;
        dpvo_win::append_state_kernel<<<nb, dpvo_win::kThreads, smem, st>>>(B);
        const int ys = p_max > 0 ? (p_max + dpvo_win::kThreads - 1) / dpvo_win::kThreads : 1;
        dpvo_win::append_edges_kernel<<<dim3(nb, ys), dpvo_win::kThreads, 0, st>>>(B);
        if (cudaGetLastError() != cudaSuccess) {
            // the mirrors of this sub-batch and of the ones before it have moved on
            // while the device may not have: mark every window of the call unusable
            for (int b = 0; b < n; ++b) ws[b]->broken = true;
            return DPVO_BA_ECUDA;
        }
    }
    return 0;
}

extern "C" int dpvo_ba_window_append(dpvo_ba_window *w, const float *new_xy, int n_new, void *stream) {
    return dpvo_ba_window_append_batch(&w, &new_xy, &n_new, 1, stream);
}

extern "C" int dpvo_ba_window_problem(const dpvo_ba_window *w, dpvo_ba_dims *dims, dpvo_ba_problem *prob) {
    if (!w || !dims || !prob || w->N == 0) return DPVO_BA_EINVAL;
    if (w->broken) return DPVO_BA_ECUDA;
    // the last free_poses poses are free, but at least the first two stay fixed (gauge and
    // monocular scale), all of them while the window has fewer than three frames
    int t0 = w->N - w->prm.free_poses;
    t0 = t0 < 2 ? 2 : t0;
    t0 = t0 > w->N ? w->N : t0;
    *dims = dpvo_ba_dims{w->N, w->P, w->E, t0, w->prm.n_iters, w->prm.fx, w->prm.fy, w->prm.cx, w->prm.cy};
    *prob = dpvo_ba_problem{w->pose[w->cur], w->patch[w->cur], w->anchor[w->cur], w->kk, w->jj, w->target,
                            w->weight, w->status};
    return 0;
}
