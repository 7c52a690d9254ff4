// Device-side SE(3) helpers: quaternion -> rotation, relative poses, the
// group exponential in FP64 for the pose update.  Poses are world->camera,
// stored [tx ty tz qx qy qz qw]; increments are left twists (v, w).
#pragma once

#include <cuda_runtime.h>

namespace dpvo {

// Rotation matrix (row-major) of a quaternion, normalised on the way.
__device__ inline void quat_to_rot(const float *q, float *R) {
    float x = q[0], y = q[1], z = q[2], w = q[3];
    float s = rsqrtf(x * x + y * y + z * z + w * w);
    x *= s; y *= s; z *= s; w *= s;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - z * w);       R[2] = 2.f * (x * z + y * w);
    R[3] = 2.f * (x * y + z * w);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - x * w);
    R[6] = 2.f * (x * z - y * w);       R[7] = 2.f * (y * z + x * w);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// G_ij = T_j T_i^-1 (camera i -> camera j, Eq. 2): R_ij = R_j R_i^T,
// t_ij = t_j - R_ij t_i.
__device__ inline void relative_pose(const float *pose_i, const float *pose_j, float *Rij, float *tij) {
    float Ri[9], Rj[9];
    quat_to_rot(pose_i + 3, Ri);
    quat_to_rot(pose_j + 3, Rj);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Rij[3 * r + c] = Rj[3 * r + 0] * Ri[3 * c + 0] + Rj[3 * r + 1] * Ri[3 * c + 1] + Rj[3 * r + 2] * Ri[3 * c + 2];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        tij[r] = pose_j[r] - (Rij[3 * r + 0] * pose_i[0] + Rij[3 * r + 1] * pose_i[1] + Rij[3 * r + 2] * pose_i[2]);
}

// Adjoint of G for twists ordered (v, w): [[R, [t]x R], [0, R]], row-major 6x6.
__device__ inline void adjoint6(const float *R, const float *t, float *Ad) {
    float tx[9] = {0.f, -t[2], t[1], t[2], 0.f, -t[0], -t[1], t[0], 0.f};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Ad[6 * r + c] = R[3 * r + c];
            Ad[6 * r + 3 + c] = tx[3 * r + 0] * R[0 + c] + tx[3 * r + 1] * R[3 + c] + tx[3 * r + 2] * R[6 + c];
            Ad[6 * (r + 3) + c] = 0.f;
            Ad[6 * (r + 3) + 3 + c] = R[3 * r + c];
        }
}

// T <- Exp(xi) T in FP64 for xi = (v, w):
//   Exp(xi) = [[R(w), V(w) v], [0, 1]],  R(w) = exp([w]x),
//   V(w) = I + (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2,  th = |w|;
// quaternion of R(w) = (sin(th/2) w/th, cos(th/2)).
// The scalar coefficients come from FP32 (sincosf, or Taylor series below
// th = 0.1; (1 - cos th)/th^2 as 2 (sin(th/2)/th)^2, free of cancellation):
// their rounding enters the pose only multiplied by th or th^2, and the
// increment's quaternion is renormalised in FP64.  The composition is FP64.
__device__ inline void se3_left_update(const double *xi, const float *pose_in, float *pose_out) {
    const double v0 = xi[0], v1 = xi[1], v2 = xi[2];
    const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    const float th2f = (float)th2, tf = sqrtf(th2f);
    float hs, hc, bf;   // sin(th/2)/th, cos(th/2), (th - sin th)/th^3
    if (tf < 0.1f) {
        hs = 0.5f + th2f * (-1.f / 48.f + th2f * (1.f / 3840.f - th2f * (1.f / 645120.f)));
        hc = 1.f + th2f * (-1.f / 8.f + th2f * (1.f / 384.f - th2f * (1.f / 46080.f)));
        bf = 1.f / 6.f + th2f * (-1.f / 120.f + th2f * (1.f / 5040.f - th2f * (1.f / 362880.f)));
    } else {
        float s2, c2;
        sincosf(0.5f * tf, &s2, &c2);
        hs = s2 / tf;
        hc = c2;
        bf = (tf - 2.f * s2 * c2) / (th2f * tf);
    }
    const double half_s0 = hs, half_c0 = hc, B = bf;
    // renormalise (half_s0 w, half_c0): its squared norm is 1 to within FP32
    // rounding, where 1.5 - s/2 approximates s^-1/2 to (3/8)(s - 1)^2
    const double sn = half_s0 * half_s0 * th2 + half_c0 * half_c0;
    const double nrm = 1.5 - 0.5 * sn;
    const double half_s = half_s0 * nrm, half_c = half_c0 * nrm;
    const double A = 2.0 * half_s * half_s;   // (1 - cos th)/th^2
    // quaternion of the increment
    const double qx = half_s * w0, qy = half_s * w1, qz = half_s * w2, qw = half_c;
    // rotation matrix of the increment from its quaternion
    double R[9];
    R[0] = 1 - 2 * (qy * qy + qz * qz); R[1] = 2 * (qx * qy - qz * qw);     R[2] = 2 * (qx * qz + qy * qw);
    R[3] = 2 * (qx * qy + qz * qw);     R[4] = 1 - 2 * (qx * qx + qz * qz); R[5] = 2 * (qy * qz - qx * qw);
    R[6] = 2 * (qx * qz - qy * qw);     R[7] = 2 * (qy * qz + qx * qw);     R[8] = 1 - 2 * (qx * qx + qy * qy);
    // V v = v + A (w x v) + B (w x (w x v))
    const double c0 = w1 * v2 - w2 * v1, c1 = w2 * v0 - w0 * v2, c2 = w0 * v1 - w1 * v0;
    const double d0 = w1 * c2 - w2 * c1, d1 = w2 * c0 - w0 * c2, d2 = w0 * c1 - w1 * c0;
    const double tv0 = v0 + A * c0 + B * d0, tv1 = v1 + A * c1 + B * d1, tv2 = v2 + A * c2 + B * d2;
    const double t0 = pose_in[0], t1 = pose_in[1], t2 = pose_in[2];
    const double nt0 = R[0] * t0 + R[1] * t1 + R[2] * t2 + tv0;
    const double nt1 = R[3] * t0 + R[4] * t1 + R[5] * t2 + tv1;
    const double nt2 = R[6] * t0 + R[7] * t1 + R[8] * t2 + tv2;
    // q_new = q_inc (x) q_old  (Hamilton product, vector part first)
    const double bx = pose_in[3], by = pose_in[4], bz = pose_in[5], bw = pose_in[6];
    double nx = qw * bx + bw * qx + (qy * bz - qz * by);
    double ny = qw * by + bw * qy + (qz * bx - qx * bz);
    double nz = qw * bz + bw * qz + (qx * by - qy * bx);
    double nw = qw * bw - (qx * bx + qy * by + qz * bz);
    // the stored quaternion is unit to within FP32 rounding: one Newton step
    // from 1.5 - s/2; other norms take the exact root
    const double qs = nx * nx + ny * ny + nz * nz + nw * nw;
    double inv;
    if (fabs(qs - 1.0) < 1e-4) {
        const double y = 1.5 - 0.5 * qs;
        inv = y * (1.5 - 0.5 * qs * y * y);
    } else {
        inv = 1.0 / sqrt(qs);
    }
    pose_out[0] = (float)nt0; pose_out[1] = (float)nt1; pose_out[2] = (float)nt2;
    pose_out[3] = (float)(nx * inv); pose_out[4] = (float)(ny * inv);
    pose_out[5] = (float)(nz * inv); pose_out[6] = (float)(nw * inv);
}

}  // namespace dpvo
