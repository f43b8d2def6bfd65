// The predictor of Alg. 1 for one body, shared by the predictor kernel (k_step.cu) and the
// fused per-body prelude of ground-only scenes (k_collision.cu).
#pragma once
#include "pabd_internal.h"

namespace pabd {

__device__ __forceinline__ void quat_to_mat(float4 q, float* R) {
    float x = q.x, y = q.y, z = q.z, w = q.w;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - z * w);       R[2] = 2.f * (x * z + y * w);
    R[3] = 2.f * (x * y + z * w);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - x * w);
    R[6] = 2.f * (x * z - y * w);       R[7] = 2.f * (y * z + x * w);       R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ void store_q(float4* q, int b, const float* c, const float* A) {
    q[3 * b] = make_float4(c[0], c[1], c[2], A[0]);
    q[3 * b + 1] = make_float4(A[1], A[2], A[3], A[4]);
    q[3 * b + 2] = make_float4(A[5], A[6], A[7], A[8]);
}

// Predictor (Alg. 1): v* = v + h g; c* = c + h v*; Q* = normalise(Q + h/2 [w, 0] Q);
// A* = R(Q*); s = q^0 = (c*, A*).  Pinned bodies, and those of a group held this step, keep q^n.
__device__ __forceinline__ void predict_body(const Dev& d, int b) {
    if ((d.bflags[b] & BF_PINNED) || held(d, b)) {
        float4 a0 = d.qn[3 * b], a1 = d.qn[3 * b + 1], a2 = d.qn[3 * b + 2];
        d.sq[3 * b] = a0; d.sq[3 * b + 1] = a1; d.sq[3 * b + 2] = a2;
        d.qa[3 * b] = a0; d.qa[3 * b + 1] = a1; d.qa[3 * b + 2] = a2;
        d.qb[3 * b] = a0; d.qb[3 * b + 1] = a1; d.qb[3 * b + 2] = a2;
        d.qstar[b] = d.quat[b];
        return;
    }
    const float h = d.p.h;
    float4 v = d.vel[b], w = d.omg[b], Q = d.quat[b], c4 = d.qn[3 * b];
    float vs[3] = {v.x + h * d.p.g[0], v.y + h * d.p.g[1], v.z + h * d.p.g[2]};
    float cs[3] = {c4.x + h * vs[0], c4.y + h * vs[1], c4.z + h * vs[2]};
    float4 wq = make_float4(w.x * Q.w + (w.y * Q.z - w.z * Q.y), w.y * Q.w + (w.z * Q.x - w.x * Q.z),
                            w.z * Q.w + (w.x * Q.y - w.y * Q.x), -(w.x * Q.x + w.y * Q.y + w.z * Q.z));
    const float hh = 0.5f * h;
    float4 Qn = make_float4(Q.x + hh * wq.x, Q.y + hh * wq.y, Q.z + hh * wq.z, Q.w + hh * wq.w);
    float inv = rsqrtf(Qn.x * Qn.x + Qn.y * Qn.y + Qn.z * Qn.z + Qn.w * Qn.w);
    Qn.x *= inv; Qn.y *= inv; Qn.z *= inv; Qn.w *= inv;
    float A[9];
    quat_to_mat(Qn, A);
    store_q(d.sq, b, cs, A);
    store_q(d.qa, b, cs, A);
    d.qstar[b] = Qn;
}

}  // namespace pabd
