// Pose supervision loss of Sec. 3.4 (Eq. 7) and its gradient with respect to
// the predicted poses, for the backward pass of the bundle-adjustment layer.
//
// For an ordered pair (i, j), i != j: P = T_i^-1 T_j, Q = G_i^-1 G_j,
// E = Q^-1 P and xi = Log(E) = (rho, phi).  A left perturbation of T_j,
// T_j <- Exp(d) T_j, left-perturbs E by Ad(X) d with X = Q^-1 T_i^-1, so
// d xi = J_l^-1(xi) Ad(X) d; perturbing T_i gives the negative.  With
// g = xi / |xi|, pose j gains Ad(X)^T J_l^-T(xi) g and pose i loses it.
// J_l^-1(xi) = sum_n (B_n / n!) ad_xi^n (Bernoulli numbers; B_1 = -1/2, odd
// terms beyond vanish).  The tangent gradient e = (e_v, e_w) of a pose (t, q)
// maps to the layout of dpvo_ba_grads as t_bar = e_v and
// q_bar = 2 (0, e_w - t x e_v) (x) q.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "dpvo_ba.h"

namespace dpvo_pl {

constexpr int kThreads = 256;
constexpr int kMaxBatch = 128;                 // descriptors per launch (kernel parameter space)
constexpr float kKink = 1e-5f;                 // twists shorter than this: no gradient (FP32 rounding of the relative poses)

struct Desc {
    const float *T, *G;
    float *loss, *dT;
    int n;
    float s;
};
struct Batch {
    Desc d[kMaxBatch];
};

// B_2k / (2k)! for k = 1 .. 10
__constant__ float kBern[10] = {8.3333333333e-2f,  -1.3888888889e-3f, 3.3068783069e-5f,  -8.2671957672e-7f,
                                2.0876756988e-8f,  -5.2841901386e-10f, 1.3382536530e-11f, -3.3896802963e-13f,
                                8.5860620562e-15f, -2.1748686985e-16f};

struct Pose {
    float R[9];   // row-major
    float t[3];
    float q[4];   // x y z w
};

__device__ inline void quat_to_R(const float *q, float *R) {
    const float x = q[0], y = q[1], z = q[2], w = q[3];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ inline Pose load_pose(const float *p, float s) {
    Pose P;
    const float n = rsqrtf(p[3] * p[3] + p[4] * p[4] + p[5] * p[5] + p[6] * p[6]);
    for (int k = 0; k < 4; ++k) P.q[k] = p[3 + k] * n;
    for (int k = 0; k < 3; ++k) P.t[k] = s * p[k];
    quat_to_R(P.q, P.R);
    return P;
}

__device__ inline void matvec(const float *R, const float *v, float *o) {
    for (int r = 0; r < 3; ++r) o[r] = R[3 * r] * v[0] + R[3 * r + 1] * v[1] + R[3 * r + 2] * v[2];
}
__device__ inline void matTvec(const float *R, const float *v, float *o) {
    for (int r = 0; r < 3; ++r) o[r] = R[r] * v[0] + R[3 + r] * v[1] + R[6 + r] * v[2];
}
__device__ inline void cross(const float *a, const float *b, float *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
// a (x) b, quaternions x y z w
__device__ inline void qmul(const float *a, const float *b, float *o) {
    o[0] = a[3] * b[0] + b[3] * a[0] + a[1] * b[2] - a[2] * b[1];
    o[1] = a[3] * b[1] + b[3] * a[1] + a[2] * b[0] - a[0] * b[2];
    o[2] = a[3] * b[2] + b[3] * a[2] + a[0] * b[1] - a[1] * b[0];
    o[3] = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
}

// A^-1 B as (quaternion, translation): (q_A^* q_B, R_A^T (t_B - t_A)).
__device__ inline void rel(const Pose &A, const Pose &B, float *q, float *t) {
    const float qa[4] = {-A.q[0], -A.q[1], -A.q[2], A.q[3]};
    qmul(qa, B.q, q);
    const float d[3] = {B.t[0] - A.t[0], B.t[1] - A.t[1], B.t[2] - A.t[2]};
    matTvec(A.R, d, t);
}

// ad_xi^T w for xi = (rho, phi): (w_r x phi, w_r x rho + w_p x phi).
__device__ inline void adT(const float *xi, const float *w, float *o) {
    float a[3], b[3], c[3];
    cross(w, xi + 3, a);
    cross(w, xi, b);
    cross(w + 3, xi + 3, c);
    for (int k = 0; k < 3; ++k) {
        o[k] = a[k];
        o[3 + k] = b[k] + c[k];
    }
}

// Ordered pair (i, j): returns |xi| and c = Ad(X)^T J_l^-T(xi) xi / |xi|.
__device__ float pair_term(const Pose &Ti, const Pose &Tj, const Pose &Gi, const Pose &Gj, float *c) {
    float qP[4], tP[3], qQ[4], tQ[3];
    rel(Ti, Tj, qP, tP);
    rel(Gi, Gj, qQ, tQ);
    float RQ[9];
    quat_to_R(qQ, RQ);
    // E = Q^-1 P
    const float qQc[4] = {-qQ[0], -qQ[1], -qQ[2], qQ[3]};
    float qE[4], tE[3];
    qmul(qQc, qP, qE);
    const float d[3] = {tP[0] - tQ[0], tP[1] - tQ[1], tP[2] - tQ[2]};
    matTvec(RQ, d, tE);
    if (qE[3] < 0.f)
        for (int k = 0; k < 4; ++k) qE[k] = -qE[k];
    // phi = Log of the rotation
    const float vn = sqrtf(qE[0] * qE[0] + qE[1] * qE[1] + qE[2] * qE[2]);
    const float th = 2.f * atan2f(vn, qE[3]);
    const float kq = vn > 1e-7f ? th / vn : 2.f / qE[3];
    float xi[6];
    for (int k = 0; k < 3; ++k) xi[3 + k] = kq * qE[k];
    // rho = V^-1(phi) tE, V^-1 = I - phi^/2 + beta phi^^2
    // beta = (1 - (th / 2) cot(th / 2)) / th^2, its series below th = 0.5
    const float th2 = th * th;
    float beta;
    if (th < 0.5f) beta = 1.f / 12.f + th2 * (1.f / 720.f + th2 * (1.f / 30240.f + th2 * (1.f / 1209600.f)));
    else beta = (1.f - 0.5f * th * cosf(0.5f * th) / sinf(0.5f * th)) / th2;
    float p1[3], p2[3];
    cross(xi + 3, tE, p1);
    cross(xi + 3, p1, p2);
    for (int k = 0; k < 3; ++k) xi[k] = tE[k] - 0.5f * p1[k] + beta * p2[k];
    const float n = sqrtf(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] + xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5]);
    if (!(n > kKink)) {                            // the norm's kink: its direction is rounding noise
        for (int k = 0; k < 6; ++k) c[k] = 0.f;
        return n;
    }
    float g[6];
    for (int k = 0; k < 6; ++k) g[k] = xi[k] / n;
    // w = J_l^-T(xi) g: even part by Horner in (ad^T)^2, then - ad^T g / 2
    float h[6], u[6], v[6];
    for (int k = 0; k < 6; ++k) h[k] = kBern[9] * g[k];
    for (int m = 8; m >= -1; --m) {
        adT(xi, h, u);
        adT(xi, u, v);
        const float cm = m >= 0 ? kBern[m] : 1.f;
        for (int k = 0; k < 6; ++k) h[k] = cm * g[k] + v[k];
    }
    adT(xi, g, u);
    float w[6];
    for (int k = 0; k < 6; ++k) w[k] = h[k] - 0.5f * u[k];
    // X = Q^-1 Ti^-1 = (R_Q^T R_i^T, R_Q^T (-R_i^T t_i - t_Q))
    float RX[9], tX[3];
    {
        float a[3];
        matTvec(Ti.R, Ti.t, a);                    // R_i^T t_i
        const float mt[3] = {-a[0] - tQ[0], -a[1] - tQ[1], -a[2] - tQ[2]};
        matTvec(RQ, mt, tX);
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc)         // (R_Q^T R_i^T)[r][cc] = sum_m RQ[m][r] Ri[cc][m]
                RX[3 * r + cc] = RQ[r] * Ti.R[3 * cc] + RQ[3 + r] * Ti.R[3 * cc + 1] + RQ[6 + r] * Ti.R[3 * cc + 2];
    }
    // c = Ad(X)^T w = (R_X^T w_r, R_X^T (w_r x t_X + w_p))
    float e[3];
    cross(w, tX, e);
    for (int k = 0; k < 3; ++k) e[k] += w[3 + k];
    matTvec(RX, w, c);
    matTvec(RX, e, c + 3);
    return n;
}

__global__ void __launch_bounds__(kThreads) pose_loss_kernel(Batch b) {
    const Desc D = b.d[blockIdx.x];
    const int N = D.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ Pose sT[DPVO_BA_MAX_FRAMES], sG[DPVO_BA_MAX_FRAMES];
    __shared__ float red[kThreads / 32][7];
    for (int a = tid; a < N; a += kThreads) {
        sT[a] = load_pose(D.T + 7 * a, D.s);
        sG[a] = load_pose(D.G + 7 * a, 1.f);
    }
    __syncthreads();
    float loss = 0.f;
    const int M = 2 * (N - 1);
    for (int a = 0; a < N; ++a) {
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int u = tid; u < M; u += kThreads) {
            const int o = u / (N - 1), bp = u - o * (N - 1), bb = bp < a ? bp : bp + 1;
            float c[6];
            if (o == 0) {                              // pair (bb, a): pose a is j
                loss += pair_term(sT[bb], sT[a], sG[bb], sG[a], c);
                for (int k = 0; k < 6; ++k) acc[k] += c[k];
            } else {                                   // pair (a, bb): pose a is i
                pair_term(sT[a], sT[bb], sG[a], sG[bb], c);
                for (int k = 0; k < 6; ++k) acc[k] -= c[k];
            }
        }
        for (int k = 0; k < 6; ++k)
            for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
        if (lane == 0)
            for (int k = 0; k < 6; ++k) red[warp][k] = acc[k];
        __syncthreads();
        if (tid == 0) {
            float ev[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int w = 0; w < kThreads / 32; ++w)
                for (int k = 0; k < 6; ++k) ev[k] += red[w][k];
            // tangent gradient of the scaled pose -> (t, q) gradient of the input pose
            const Pose &P = sT[a];
            float txe[3], m[4];
            cross(P.t, ev, txe);
            for (int k = 0; k < 3; ++k) m[k] = 2.f * (ev[3 + k] - txe[k]);
            m[3] = 0.f;
            float qb[4];
            qmul(m, P.q, qb);
            float *o = D.dT + 7 * a;
            for (int k = 0; k < 3; ++k) o[k] = D.s * ev[k];
            for (int k = 0; k < 4; ++k) o[3 + k] = qb[k];
        }
        __syncthreads();
    }
    for (int off = 16; off > 0; off >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, off);
    if (lane == 0) red[warp][6] = loss;
    __syncthreads();
    if (tid == 0) {
        float L = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) L += red[w][6];
        *D.loss = L;
    }
}

}  // namespace dpvo_pl

extern "C" int dpvo_ba_pose_loss(const dpvo_ba_pose_loss_problem *probs, int n_problems, void *stream) {
    if (n_problems < 0 || (n_problems > 0 && probs == nullptr)) return DPVO_BA_EINVAL;
    for (int b = 0; b < n_problems; ++b) {
        const dpvo_ba_pose_loss_problem &p = probs[b];
        if (!p.poses || !p.gt_poses || !p.loss || !p.dL_dposes || p.n_frames < 1 || p.n_frames > DPVO_BA_MAX_FRAMES)
            return DPVO_BA_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int b0 = 0; b0 < n_problems; b0 += dpvo_pl::kMaxBatch) {
        dpvo_pl::Batch batch;
        const int nb = n_problems - b0 < dpvo_pl::kMaxBatch ? n_problems - b0 : dpvo_pl::kMaxBatch;
        for (int b = 0; b < nb; ++b) {
            const dpvo_ba_pose_loss_problem &p = probs[b0 + b];
            batch.d[b] = dpvo_pl::Desc{p.poses, p.gt_poses, p.loss, p.dL_dposes, p.n_frames, p.scale};
        }
        dpvo_pl::pose_loss_kernel<<<nb, dpvo_pl::kThreads, 0, st>>>(batch);
        if (cudaGetLastError() != cudaSuccess) return DPVO_BA_ECUDA;
    }
    return 0;
}
