// Device-side SE(3) helpers: quaternion -> rotation, relative poses, the
// group exponential for the pose update.  Poses are world->camera,
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

// T <- Exp(xi) T for xi = (v, w):
//   Exp(xi) = [[R(w), V(w) v], [0, 1]],  R(w) = exp([w]x),
//   V(w) = I + (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2,  th = |w|;
// quaternion of R(w) = q = (sin(th/2) w/th, cos(th/2)).
// FP32, in increment form: every output coordinate is the stored coordinate
// plus a correction that is small for a Gauss-Newton step and is formed with
// FP32 relative accuracy, so the result is rounded once, as if the
// composition were exact and then stored:
//   t' = t + [(R - I) t + V v],  R - I from q without the "1 -" cancellation;
//   q' = b + [(q - 1) (x) b - (eta/2) b],  q - 1 = (q_v, cos(th/2) - 1),
// where eta = |q (x) b|^2 - 1 (the stored quaternion's norm error) makes q'
// unit to first order.  The scalar coefficients are Taylor series below th =
// 0.1, else from sincosf (cos(th/2) - 1 as -sin^2(th/2) / (1 + cos(th/2)),
// free of cancellation).
__device__ inline void se3_left_update(const double *xi, const float *pose_in, float *pose_out) {
    const float v0 = (float)xi[0], v1 = (float)xi[1], v2 = (float)xi[2];
    const float w0 = (float)xi[3], w1 = (float)xi[4], w2 = (float)xi[5];
    const float th2 = w0 * w0 + w1 * w1 + w2 * w2, tf = sqrtf(th2);
    float hs, hcm1, B;   // sin(th/2)/th, cos(th/2) - 1, (th - sin th)/th^3
    if (tf < 0.1f) {
        hs = 0.5f + th2 * (-1.f / 48.f + th2 * (1.f / 3840.f - th2 * (1.f / 645120.f)));
        hcm1 = th2 * (-1.f / 8.f + th2 * (1.f / 384.f - th2 * (1.f / 46080.f)));
        B = 1.f / 6.f + th2 * (-1.f / 120.f + th2 * (1.f / 5040.f - th2 * (1.f / 362880.f)));
    } else {
        float s2, c2;
        sincosf(0.5f * tf, &s2, &c2);
        hs = s2 / tf;
        hcm1 = -s2 * s2 / (1.f + c2);
        B = (tf - 2.f * s2 * c2) / (th2 * tf);
    }
    const float A = 2.f * hs * hs;   // (1 - cos th)/th^2
    const float qx = hs * w0, qy = hs * w1, qz = hs * w2, qw = 1.f + hcm1;
    // R - I of the increment (unit quaternion form)
    const float E0 = -2.f * (qy * qy + qz * qz), E1 = 2.f * (qx * qy - qz * qw), E2 = 2.f * (qx * qz + qy * qw);
    const float E3 = 2.f * (qx * qy + qz * qw), E4 = -2.f * (qx * qx + qz * qz), E5 = 2.f * (qy * qz - qx * qw);
    const float E6 = 2.f * (qx * qz - qy * qw), E7 = 2.f * (qy * qz + qx * qw), E8 = -2.f * (qx * qx + qy * qy);
    // V v = v + A (w x v) + B (w x (w x v))
    const float c0 = w1 * v2 - w2 * v1, c1 = w2 * v0 - w0 * v2, c2 = w0 * v1 - w1 * v0;
    const float d0 = w1 * c2 - w2 * c1, d1 = w2 * c0 - w0 * c2, d2 = w0 * c1 - w1 * c0;
    const float t0 = pose_in[0], t1 = pose_in[1], t2 = pose_in[2];
    pose_out[0] = t0 + (E0 * t0 + E1 * t1 + E2 * t2 + (v0 + A * c0 + B * d0));
    pose_out[1] = t1 + (E3 * t0 + E4 * t1 + E5 * t2 + (v1 + A * c1 + B * d1));
    pose_out[2] = t2 + (E6 * t0 + E7 * t1 + E8 * t2 + (v2 + A * c2 + B * d2));
    // q' = q (x) b (Hamilton product, vector part first), as b + the correction
    const float bx = pose_in[3], by = pose_in[4], bz = pose_in[5], bw = pose_in[6];
    const float dx = hcm1 * bx + bw * qx + (qy * bz - qz * by);
    const float dy = hcm1 * by + bw * qy + (qz * bx - qx * bz);
    const float dz = hcm1 * bz + bw * qz + (qx * by - qy * bx);
    const float dw = hcm1 * bw - (qx * bx + qy * by + qz * bz);
    // eta = |b|^2 (1 + e) - 1, e = |q|^2 - 1 = th2 hs^2 + hcm1 (2 + hcm1)
    const float e = th2 * hs * hs + hcm1 * (2.f + hcm1);
    const float nb = fmaf(bx, bx, fmaf(by, by, fmaf(bz, bz, fmaf(bw, bw, -1.f))));
    const float h = 0.5f * (nb + e + nb * e);
    if (fabsf(h) < 1e-5f) {          // first order in eta: error below 3/8 eta^2
        pose_out[3] = bx + (dx - h * bx);
        pose_out[4] = by + (dy - h * by);
        pose_out[5] = bz + (dz - h * bz);
        pose_out[6] = bw + (dw - h * bw);
    } else {                         // a stored quaternion far from unit norm
        const float nx = bx + dx, ny = by + dy, nz = bz + dz, nw = bw + dw;
        const float inv = 1.f / sqrtf(nx * nx + ny * ny + nz * nz + nw * nw);
        pose_out[3] = nx * inv;
        pose_out[4] = ny * inv;
        pose_out[5] = nz * inv;
        pose_out[6] = nw * inv;
    }
}

}  // namespace dpvo
