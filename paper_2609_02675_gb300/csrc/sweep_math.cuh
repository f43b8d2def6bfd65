// Device arithmetic shared by the sweep kernels (k_sweep.cu: bond + solve launches,
// k_persist.cu: the fused persistent sweep): bond split forces, the per-body 4x4 system
// and the rotation of the local solve.  One copy, so both paths compute identical bonds.
#pragma once
#include <type_traits>

#include "dfloat.cuh"
#include "pabd_internal.h"

namespace pabd {

__device__ __forceinline__ float shfl_xor(unsigned mask, float v, int o) { return __shfl_xor_sync(mask, v, o); }
__device__ __forceinline__ double shfl_xor(unsigned mask, double v, int o) { return __shfl_xor_sync(mask, v, o); }

__device__ __forceinline__ void ld_q(const float4* __restrict__ q, int b, float* c, float* A) {
    float4 a = q[3 * b], bb = q[3 * b + 1], cc = q[3 * b + 2];
    c[0] = a.x; c[1] = a.y; c[2] = a.z;
    A[0] = a.w; A[1] = bb.x; A[2] = bb.y; A[3] = bb.z; A[4] = bb.w;
    A[5] = cc.x; A[6] = cc.y; A[7] = cc.z; A[8] = cc.w;
}


// Split force of one bond from the iterate (Eq. 15-17): returns w = h^2 phi+(d)/d and the
// delta-form record f' of end i (end j gets -f'), see the file comment of k_sweep.cu.  Only
// the end-to-end vector r = y_j - y_i enters (bond_vec forms it without rounding at the
// scale of the bodies' positions).  Always single precision: a body on the extended path
// sums these same records in the extended type (sys_add_x).
__device__ __forceinline__ float bond_force(int type, float4 xi, float4 xj, float4 nm, const float* r, float* f) {
    float w = xi.w;
    if (type == K_CONTACT || type == K_GROUND) {
        const float dhat = xj.w;
        const float N[3] = {nm.x, nm.y, nm.z};
        const float rr[3] = {-r[0], -r[1], -r[2]};  // y_i - y_j
        float g = N[0] * rr[0] + N[1] * rr[1] + N[2] * rr[2];
        if (g < dhat) {
            float t[3] = {rr[0] - g * N[0], rr[1] - g * N[1], rr[2] - g * N[2]};
            float tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
            float tau = nm.w * (dhat - g);
            float keep = tn > tau ? 1.f - tau / tn : 0.f;  // t - t_c = keep * t
#pragma unroll
            for (int k = 0; k < 3; ++k) f[k] = w * ((dhat * N[k] + keep * t[k]) - rr[k]);
        } else {
            w = 0.f;
            f[0] = f[1] = f[2] = 0.f;
        }
        return w;
    }
    if (type == K_SPHERICAL || type == K_DRIVE) {
#pragma unroll
        for (int k = 0; k < 3; ++k) f[k] = w * r[k];
        return w;
    }
    float dd = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    float n[3];
    if (dd > 0.f) { float id = 1.f / dd; n[0] = r[0] * id; n[1] = r[1] * id; n[2] = r[2] * id; }
    else { n[0] = 0.f; n[1] = 1.f; n[2] = 0.f; }
    const float l = xj.w;
    float sc;
    if (type == K_SPRING) {
        sc = w * (dd - l);                      // h^2 phi(d)
    } else {                                    // nonlinear elastic, tangent split
        // h^2 phi(d) = (w / 3) (d^3 / l^2 - l) = (w / 3) (d - l) (d^2 + d l + l^2) / l^2: the
        // factored form has no cancellation near the rest length
        const float il2 = 1.f / (l * l);
        sc = (w * (1.f / 3.f)) * ((dd - l) * ((dd * dd + dd * l + l * l) * il2));
        w = w * dd * dd * il2;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = sc * n[k];
    return w;
}

// r = y_j - y_i for end points y = c + A x, formed as (c_j - c_i) + (A_j x_j - A_i x_i): the
// centres' difference rounds once at the scale of the bond, not of the positions, so a stiff
// short bond far from the origin keeps its length to single precision.  A world end j is
// the point x_j itself.
__device__ __forceinline__ void bond_vec(const float* ci, const float* Ai, float4 xi, const float* cj,
                                         const float* Aj, float4 xj, bool world_j, float* r) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ai = Ai[3 * k] * xi.x + Ai[3 * k + 1] * xi.y + Ai[3 * k + 2] * xi.z;
        if (world_j) {
            r[k] = ((&xj.x)[k] - ci[k]) - ai;
        } else {
            const float aj = Aj[3 * k] * xj.x + Aj[3 * k + 1] * xj.y + Aj[3 * k + 2] * xj.z;
            r[k] = (cj[k] - ci[k]) + (aj - ai);
        }
    }
}


// Augmented Lagrangian distance bond at sweep `it` (Eq. 27-29): for it >= 1 first the dual
// update from the constraint of this iterate (the primal result of sweep it - 1),
// lambda <- kappa C + lambda, kappa <- kappa + beta |C|, read from the parity-(it-1) buffer and
// stored by `writer` into the parity-it buffer; then the split force with those values:
// phi+ = kappa d + max(lambda - kappa l, 0), phi- = min(lambda - kappa l, 0); w = h^2 phi+/d
// (d kept above 1e-9), f' = w (y_j - y_i) + h^2 phi- n.  xi.w holds h^2, xj.w the rest length.
__device__ __forceinline__ float al_force(const Dev& d, int bond, int it, bool writer, float4 xi, float4 xj,
                                          const float* r, float* f) {
    float dd = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    float n[3];
    if (dd > 0.f) { float id = 1.f / dd; n[0] = r[0] * id; n[1] = r[1] * id; n[2] = r[2] * id; }
    else { n[0] = 0.f; n[1] = 1.f; n[2] = 0.f; }
    const float l = xj.w;
    float kap, lam;
    if (it == 0) {
        const float2 kl = d.al_st0[bond];
        kap = kl.x; lam = kl.y;
    } else {
        const float2 kl = ((it - 1) & 1) ? d.al_st1[bond] : d.al_st0[bond];
        const float c = dd - l;
        lam = kl.x * c + kl.y;
        kap = kl.x + d.al_par[bond].y * fabsf(c);
        if (writer) {
            float2* out = (it & 1) ? d.al_st1 : d.al_st0;
            out[bond] = make_float2(kap, lam);
        }
    }
    const float h2 = xi.w;
    const float cst = lam - kap * l;
    const float w = h2 * (kap + (cst > 0.f ? cst / (dd > 1e-9f ? dd : 1e-9f) : 0.f));
    const float sc = h2 * (cst < 0.f ? cst : 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = w * r[k] + sc * n[k];
    return w;
}

// The same vector for the FP32 path as accurately as if formed in twice the precision and
// rounded once (Ogita, Rump and Oishi's Dot2: TwoSum / TwoProduct of every term, the errors
// summed apart).  A stiff joint's gap is the small difference of the centres' offset and the
// lever arms; in plain FP32 its rounding (an ulp of the lever, independently at each end)
// reaches the forces as w times that ulp -- inconsistent between the two ends and far above
// the joint's own resolution -- and from there the body's softly held rotations.
__device__ __forceinline__ void bond_vec_dot2(const float* ci, const float* Ai, float4 xi, const float* cj,
                                              const float* Aj, float4 xj, bool world_j, float* r) {
    const float xiv[3] = {xi.x, xi.y, xi.z}, xjv[3] = {xj.x, xj.y, xj.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        df acc = two_sum(world_j ? xjv[k] : cj[k], -ci[k]);
        float err = acc.lo;
        float hi = acc.hi;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            df p = two_prod(-Ai[3 * k + l], xiv[l]);
            df t = two_sum(hi, p.hi);
            hi = t.hi;
            err = __fadd_rn(err, __fadd_rn(t.lo, p.lo));
            if (!world_j) {
                p = two_prod(Aj[3 * k + l], xjv[l]);
                t = two_sum(hi, p.hi);
                hi = t.hi;
                err = __fadd_rn(err, __fadd_rn(t.lo, p.lo));
            }
        }
        r[k] = __fadd_rn(hi, err);
    }
}

// Force of the bond seen from body `self`, given the other body's iterate (co, Ao; unused
// when the other end is the world): forms the bond vector (compensated for user bonds: stiff
// joints, elastic and AL bonds), evaluates the split force; returns w and writes the record
// of self's end.  `it` is the sweep index and `writer` whether this evaluation stores an
// augmented Lagrangian bond's updated state (exactly one evaluation per bond does).
__device__ __forceinline__ float end_force_q(const Dev& d, const float* co, const float* Ao, int self, const float* cs,
                                             const float* As, int4 m, float4 xa, float4 xb, int it, bool writer,
                                             float* f) {
    const bool side_j = (m.y == self);
    float r[3];
    if (m.z != K_CONTACT && m.z != K_GROUND) {
        if (side_j) bond_vec_dot2(co, Ao, xa, cs, As, xb, false, r);
        else bond_vec_dot2(cs, As, xa, co, Ao, xb, m.y < 0, r);
    } else if (side_j) {
        bond_vec(co, Ao, xa, cs, As, xb, false, r);
    } else {
        bond_vec(cs, As, xa, co, Ao, xb, m.y < 0, r);
    }
    float w;
    if (m.z == K_AL) {
        w = al_force(d, m.w, it, writer, xa, xb, r, f);
    } else {
        const float4 nm = (m.z == K_CONTACT || m.z == K_GROUND) ? d.bn[m.w] : make_float4(0.f, 0.f, 0.f, 0.f);
        w = bond_force(m.z, xa, xb, nm, r, f);
    }
    if (side_j) { f[0] = -f[0]; f[1] = -f[1]; f[2] = -f[2]; }
    return w;
}

// the other end's body of bond record m seen from `self` (-1 for the world)
__device__ __forceinline__ int other_body(int4 m, int self) { return m.y == self ? m.x : m.y; }

// q of body o, or zeros for the world (o < 0)
__device__ __forceinline__ void ld_q_or_zero(const float4* __restrict__ q, int o, float* c, float* A) {
    if (o >= 0) {
        ld_q(q, o, c, A);
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) c[k] = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) A[k] = 0.f;
    }
}

__device__ __forceinline__ float end_force(const Dev& d, const float4* __restrict__ q, int self, const float* cs,
                                           const float* As, int4 m, float4 xa, float4 xb, int it, bool writer,
                                           float* f) {
    float co[3], Ao[9];
    ld_q_or_zero(q, other_body(m, self), co, Ao);
    return end_force_q(d, co, Ao, self, cs, As, m, xa, xb, it, writer, f);
}

// ---- 4x4 SPD system with three right-hand sides ----
// G packed as g[10] = (00 01 02 03 11 12 13 22 23 33); R[4][3]
template <class T>
struct Sys {
    T g[10];
    T r[4][3];
};

// Compensated accumulator of the extended path (precision policy 1): the float running sum s
// and the float sum e of the rounding errors of every addition (TwoSum) and of every product
// (TwoProd) that entered it -- Ogita, Rump and Oishi's Sum2 / Dot2 ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005).  s + e is the sum as accurate as if it had been
// accumulated in twice the working precision and rounded, at about a third of the cost of
// double-float additions; the total is turned into a double-float (ca_to_df) for the
// factorisation.
struct ca {
    float s, e;
    ca() = default;
    __host__ __device__ constexpr ca(float v) : s(v), e(0.f) {}
    __host__ __device__ constexpr ca(float a, float b) : s(a), e(b) {}
};

__device__ __forceinline__ void ca_add(ca& a, float x) {
    const df t = two_sum(a.s, x);
    a.s = t.hi;
    a.e = __fadd_rn(a.e, t.lo);
}
// add hi + lo, where hi is the rounded value and lo a small correction (a product's error)
__device__ __forceinline__ void ca_add(ca& a, float hi, float lo) {
    const df t = two_sum(a.s, hi);
    a.s = t.hi;
    a.e = __fadd_rn(a.e, __fadd_rn(t.lo, lo));
}
__device__ __forceinline__ ca& operator+=(ca& a, ca b) {
    const df t = two_sum(a.s, b.s);
    a.s = t.hi;
    a.e = __fadd_rn(__fadd_rn(a.e, b.e), t.lo);
    return a;
}
__device__ __forceinline__ ca shfl_xor(unsigned mask, ca v, int o) {
    return ca{__shfl_xor_sync(mask, v.s, o), __shfl_xor_sync(mask, v.e, o)};
}
__device__ __forceinline__ ca ca_of(df v) { return ca{v.hi, v.lo}; }
// the accumulated value as a double-word for the factorisation, without renormalising: the
// error sum is far below the float sum (a few rounding errors of the partial sums), and the
// double-word operations that consume it carry both parts
__device__ __forceinline__ df ca_to_df(ca v) { return df(v.s, v.e, 0); }

// the extended system as it is factored: double-float from the compensated sums, FP64 as
// summed under policy 2
__device__ __forceinline__ Sys<df> ext_sys(const Sys<ca>& s) {
    Sys<df> t;
#pragma unroll
    for (int k = 0; k < 10; ++k) t.g[k] = ca_to_df(s.g[k]);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) t.r[r][k] = ca_to_df(s.r[r][k]);
    return t;
}
__device__ __forceinline__ const Sys<double>& ext_sys(const Sys<double>& s) { return s; }

// The system is assembled about a per-body expansion point x_s (Dev::xs; zero for most
// bodies): with z = x - x_s the unknowns are c' = c + A x_s and A, so G = diag(m, Pi) +
// sum w [1; x][1; x]^T becomes, exactly, T^-1 G T^-T = [m, -m x_s^T; -m x_s, Pi + m x_s x_s^T]
// + sum w [1; z][1; z]^T and the right-hand side [R_0; R_A - x_s R_0].  Placing x_s at the
// weighted centre of the body's stiff static bonds removes the cancellation between their
// c and A couplings (the Schur complement of G_00), which otherwise dominates the rounding of
// an FP32 factorisation of a stiffly jointed body; dc = dc' - dA x_s recovers the update.
template <class T>
__device__ __forceinline__ void sys_init(Sys<T>& s, float4 mass, const float* dc, const float* dA, const float* xs) {
    const T m = (T)mass.x;
    const T mx[3] = {m * (T)xs[0], m * (T)xs[1], m * (T)xs[2]};
    s.g[0] = m; s.g[1] = -mx[0]; s.g[2] = -mx[1]; s.g[3] = -mx[2];
    s.g[4] = (T)mass.y + mx[0] * (T)xs[0]; s.g[5] = mx[0] * (T)xs[1]; s.g[6] = mx[0] * (T)xs[2];
    s.g[7] = (T)mass.z + mx[1] * (T)xs[1]; s.g[8] = mx[1] * (T)xs[2];
    s.g[9] = (T)mass.w + mx[2] * (T)xs[2];
    const T pm[4] = {m, (T)mass.y, (T)mass.z, (T)mass.w};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s.r[0][k] = pm[0] * (T)dc[k];
#pragma unroll
        for (int l = 0; l < 3; ++l) s.r[1 + l][k] = pm[1 + l] * (T)dA[3 * k + l] - mx[l] * (T)dc[k];
    }
}

// the same initial system for the compensated accumulator: every product formed exactly by
// TwoProd (m x_s as a double-word), every sum by TwoSum, the errors kept in the accumulator
__device__ __forceinline__ void sys_init(Sys<ca>& s, float4 mass, const float* dc, const float* dA, const float* xs) {
    const float m = mass.x;
    const float pi[3] = {mass.y, mass.z, mass.w};
    df mx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) mx[a] = two_prod(m, xs[a]);
    s.g[0] = ca(m);
#pragma unroll
    for (int a = 0; a < 3; ++a) s.g[1 + a] = ca(-mx[a].hi, -mx[a].lo);
    int k = 4;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b, ++k) {
            const df p = two_prod(mx[a].hi, xs[b]);
            const float lo = __fmaf_rn(mx[a].lo, xs[b], p.lo);
            if (a == b) {
                const df t = two_sum(pi[a], p.hi);
                s.g[k] = ca(t.hi, __fadd_rn(t.lo, lo));
            } else {
                s.g[k] = ca(p.hi, lo);
            }
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const df r0 = two_prod(m, dc[c]);
        s.r[0][c] = ca(r0.hi, r0.lo);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const df p1 = two_prod(pi[a], dA[3 * c + a]);
            const df p2 = two_prod(mx[a].hi, dc[c]);
            const float lo2 = __fmaf_rn(mx[a].lo, dc[c], p2.lo);
            const df t = two_sum(p1.hi, -p2.hi);
            s.r[1 + a][c] = ca(t.hi, __fadd_rn(t.lo, __fsub_rn(p1.lo, lo2)));
        }
    }
}

// the exact difference a - b of two floats in the extended type
__device__ __forceinline__ df ext_diff(float a, float b, df*) { return two_sum(a, -b); }
__device__ __forceinline__ double ext_diff(float a, float b, double*) { return (double)a - (double)b; }

// One bond end's single-precision record (w, f') at material point x of the body, about the
// expansion point x_s, added to the body's system.  In FP32 as it stands; in the extended
// type X the offsets z = x - x_s are exact and every product w z_a z_b, z_a f'_k is formed
// and summed to X's precision, so the assembled G and R are those of the stored records
// without the single-precision rounding of the sums, whose cancellation (stiff joints, near
// singular G) is what the extended path exists to remove.
template <class T>
__device__ __forceinline__ void sys_add_t(Sys<T>& s, float w, const float* f, float4 x, const float* xs) {
    if constexpr (sizeof(T) == sizeof(float)) {
        const float z1 = x.x - xs[0], z2 = x.y - xs[1], z3 = x.z - xs[2];
        const float wz1 = w * z1, wz2 = w * z2, wz3 = w * z3;
        s.g[0] += w;   s.g[1] += wz1;      s.g[2] += wz2;      s.g[3] += wz3;
        s.g[4] += wz1 * z1; s.g[5] += wz1 * z2; s.g[6] += wz1 * z3;
        s.g[7] += wz2 * z2; s.g[8] += wz2 * z3;
        s.g[9] += wz3 * z3;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s.r[0][k] += f[k];
            s.r[1][k] += z1 * f[k];
            s.r[2][k] += z2 * f[k];
            s.r[3][k] += z3 * f[k];
        }
    } else if constexpr (std::is_same<T, ca>::value) {
        // compensated: z = x - x_s exact (TwoSum), w z_a as hi + lo to twice the precision,
        // every product's rounding error carried into the accumulator's error sum
        const df z[3] = {two_sum(x.x, -xs[0]), two_sum(x.y, -xs[1]), two_sum(x.z, -xs[2])};
        df wz[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const df p = two_prod(w, z[a].hi);
            wz[a] = df(p.hi, __fmaf_rn(w, z[a].lo, p.lo), 0);
        }
        ca_add(s.g[0], w);
#pragma unroll
        for (int a = 0; a < 3; ++a) ca_add(s.g[1 + a], wz[a].hi, wz[a].lo);
        int k = 4;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b, ++k) {
                const df p = two_prod(wz[a].hi, z[b].hi);
                ca_add(s.g[k], p.hi, __fmaf_rn(wz[a].hi, z[b].lo, __fmaf_rn(wz[a].lo, z[b].hi, p.lo)));
            }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ca_add(s.r[0][c], f[c]);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const df p = two_prod(z[a].hi, f[c]);
                ca_add(s.r[1 + a][c], p.hi, __fmaf_rn(z[a].lo, f[c], p.lo));
            }
        }
    } else {
        const T z1 = ext_diff(x.x, xs[0], (T*)nullptr), z2 = ext_diff(x.y, xs[1], (T*)nullptr),
                z3 = ext_diff(x.z, xs[2], (T*)nullptr);
        const T wz1 = w * z1, wz2 = w * z2, wz3 = w * z3;
        s.g[0] += w;   s.g[1] += wz1;      s.g[2] += wz2;      s.g[3] += wz3;
        s.g[4] += wz1 * z1; s.g[5] += wz1 * z2; s.g[6] += wz1 * z3;
        s.g[7] += wz2 * z2; s.g[8] += wz2 * z3;
        s.g[9] += wz3 * z3;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            s.r[0][k] += f[k];
            s.r[1][k] += z1 * f[k];
            s.r[2][k] += z2 * f[k];
            s.r[3][k] += z3 * f[k];
        }
    }
}

// a stored end record e = (w, f') of the two-launch sweep
template <class T>
__device__ __forceinline__ void sys_add(Sys<T>& s, float4 e, float4 x, const float* xs) {
    const float f[3] = {e.y, e.z, e.w};
    sys_add_t(s, e.x, f, x, xs);
}

// the update of c from the solution Y of the shifted system: dc = dc' - dA x_s
__device__ __forceinline__ void unshift(float (*X)[3], const float* xs) {
#pragma unroll
    for (int k = 0; k < 3; ++k) X[0][k] -= xs[0] * X[1][k] + xs[1] * X[2][k] + xs[2] * X[3][k];
}

// the expansion point of body b (zero unless the body is flagged BF_SHIFT)
__device__ __forceinline__ void ld_xs(const Dev& d, int b, int fl, float* xs) {
    if (fl & BF_SHIFT) {
        const float4 v = d.xs[b];
        xs[0] = v.x; xs[1] = v.y; xs[2] = v.z;
    } else {
        xs[0] = xs[1] = xs[2] = 0.f;
    }
}

// Cholesky G = L L^T and solve; returns 1 if every pivot is at least 1e-3 of its diagonal
// (the factorisation is trusted), -1 otherwise
__device__ __forceinline__ float inv_sqrt(float x) { return 1.f / sqrtf(x); }
__device__ __forceinline__ double inv_sqrt(double x) { return 1.0 / sqrt(x); }

template <class T>
__device__ __forceinline__ T sys_solve(const Sys<T>& s, T out[4][3]) {
    const T* g = s.g;
    // L = lower Cholesky factor, stored through its inverse diagonal i_k = 1 / L_kk
    T d0 = g[0];
    T i0 = inv_sqrt(d0);
    T l10 = g[1] * i0, l20 = g[2] * i0, l30 = g[3] * i0;
    T d1 = g[4] - l10 * l10;
    T i1 = inv_sqrt(d1);
    T l21 = (g[5] - l20 * l10) * i1, l31 = (g[6] - l30 * l10) * i1;
    T d2 = g[7] - l20 * l20 - l21 * l21;
    T i2 = inv_sqrt(d2);
    T l32 = (g[8] - l30 * l20 - l31 * l21) * i2;
    T d3 = g[9] - l30 * l30 - l31 * l31 - l32 * l32;
    T i3 = inv_sqrt(d3);
    // well conditioned iff every pivot keeps at least 1e-3 of its diagonal (no division): a
    // pivot ratio r costs about log10(1/r) digits of the FP32 solve
    const T lim = T(1e-3);
    const T ratio = (d0 > T(0) && d1 >= lim * g[4] && d2 >= lim * g[7] && d3 >= lim * g[9]) ? T(1) : T(-1);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T y0 = s.r[0][k] * i0;
        T y1 = (s.r[1][k] - l10 * y0) * i1;
        T y2 = (s.r[2][k] - l20 * y0 - l21 * y1) * i2;
        T y3 = (s.r[3][k] - l30 * y0 - l31 * y1 - l32 * y2) * i3;
        T x3 = y3 * i3;
        T x2 = (y2 - l32 * x3) * i2;
        T x1 = (y1 - l21 * x2 - l31 * x3) * i1;
        T x0 = (y0 - l10 * x1 - l20 * x2 - l30 * x3) * i0;
        out[0][k] = x0; out[1][k] = x1; out[2][k] = x2; out[3][k] = x3;
    }
    return ratio;
}

// The extended (double-float) system solved by an LDL^T factorisation: no square roots, the
// four pivots inverted once, every update a fused double-word multiply-add (fma_dd).  About
// half the work and half the code of the double-float Cholesky, at the same accuracy for these
// systems (errors of order 2^-48 of the entries, far below the single-precision result).
//   D0 = g00, L_k0 = g_0k / D0; D1 = g11 - L10 g01, u_k1 = g_1k - L_k0 g_0k (= L_k1 D1), ...
// The forward substitution y = L^-1 r stays in double-float: its last rows cancel (the soft
// directions of a stiffly jointed body's G), and the pivots' inverses then magnify what is
// left.  The rest, x = L^-T (D^-1 y), runs in single precision from the rounded y, D^-1 and L:
// a triangular solve's componentwise error is set by its unit factor L (the scaling by D^-1 is
// exact to rounding), which is well conditioned here, so x keeps single-precision accuracy
// relative to its own entries -- all that the single-precision update q + x can hold.
__device__ __forceinline__ void sys_solve_ldl(const Sys<df>& s, float out[4][3]) {
    const df* g = s.g;
    const df r0 = recip_dd(g[0]);
    const df l10 = g[1] * r0, l20 = g[2] * r0, l30 = g[3] * r0;
    const df m10 = -l10, m20 = -l20, m30 = -l30;
    const df d1 = fma_dd(m10, g[1], g[4]);
    const df u21 = fma_dd(m20, g[1], g[5]), u31 = fma_dd(m30, g[1], g[6]);
    const df r1 = recip_dd(d1);
    const df l21 = u21 * r1, l31 = u31 * r1;
    const df d2 = fma_dd(-l21, u21, fma_dd(m20, g[2], g[7]));
    const df u32 = fma_dd(-l31, u21, fma_dd(m30, g[2], g[8]));
    const df r2 = recip_dd(d2);
    const df l32 = u32 * r2;
    const df d3 = fma_dd(-l32, u32, fma_dd(-l31, u31, fma_dd(m30, g[3], g[9])));
    const df r3 = recip_dd(d3);
    const float f10 = (float)l10, f20 = (float)l20, f30 = (float)l30, f21 = (float)l21, f31 = (float)l31,
                f32 = (float)l32;
    const float i0 = (float)r0, i1 = (float)r1, i2 = (float)r2, i3 = (float)r3;
    // the three right-hand sides through one copy of the substitution code (a short
    // instruction footprint): each pass solves column 0 and rotates the columns left, the
    // solution entering as column 2 of the output, so after three passes both hold theirs in order
    df c0[4], c1[4], c2[4];
    float o0[4], o1[4], o2[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) { c0[r] = s.r[r][0]; c1[r] = s.r[r][1]; c2[r] = s.r[r][2]; o0[r] = o1[r] = o2[r] = 0.f; }
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        const df y0 = c0[0];
        const df y1 = fma_dd(m10, y0, c0[1]);
        const df y2 = fma_dd(-l21, y1, fma_dd(m20, y0, c0[2]));
        const df y3 = fma_dd(-l32, y2, fma_dd(-l31, y1, fma_dd(m30, y0, c0[3])));
        const float x3 = (float)y3 * i3;
        const float x2 = __fmaf_rn(-f32, x3, (float)y2 * i2);
        const float x1 = __fmaf_rn(-f31, x3, __fmaf_rn(-f21, x2, (float)y1 * i1));
        const float x0 = __fmaf_rn(-f30, x3, __fmaf_rn(-f20, x2, __fmaf_rn(-f10, x1, (float)y0 * i0)));
#pragma unroll
        for (int r = 0; r < 4; ++r) { c0[r] = c1[r]; c1[r] = c2[r]; o0[r] = o1[r]; o1[r] = o2[r]; }
        o2[0] = x0; o2[1] = x1; o2[2] = x2; o2[3] = x3;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) { out[r][0] = o0[r]; out[r][1] = o1[r]; out[r][2] = o2[r]; }
}

// the extended system's solve into the single-precision update: LDL^T in double-float,
// Cholesky in FP64
__device__ __forceinline__ void ext_solve(const Sys<df>& s, float out[4][3]) { sys_solve_ldl(s, out); }
__device__ __forceinline__ void ext_solve(const Sys<double>& s, float out[4][3]) {
    double x[4][3];
    sys_solve(s, x);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) out[r][k] = (float)x[r][k];
}

// ---- local solve: rotation of A ----

__device__ __forceinline__ void cofactor(const float* X, float* C) {
    C[0] = X[4] * X[8] - X[5] * X[7]; C[1] = X[5] * X[6] - X[3] * X[8]; C[2] = X[3] * X[7] - X[4] * X[6];
    C[3] = X[2] * X[7] - X[1] * X[8]; C[4] = X[0] * X[8] - X[2] * X[6]; C[5] = X[1] * X[6] - X[0] * X[7];
    C[6] = X[1] * X[5] - X[2] * X[4]; C[7] = X[2] * X[3] - X[0] * X[5]; C[8] = X[0] * X[4] - X[1] * X[3];
}

// Fallback: eigen-decomposition of S = A^T A by cyclic Jacobi rotations; R = U V^T with
// u1 = A v1 / |A v1|, u2 = normalised (A v2 - (u1 . A v2) u1), u3 = u1 x u2, det V = +1.
__device__ __noinline__ static void polar_eigen(float* X) {
    float S[9], V[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) S[3 * r + c] = X[r] * X[c] + X[3 + r] * X[3 + c] + X[6 + r] * X[6 + c];
    for (int sweep = 0; sweep < 12; ++sweep) {
        float off = fabsf(S[1]) + fabsf(S[2]) + fabsf(S[5]);
        float sc = fabsf(S[0]) + fabsf(S[4]) + fabsf(S[8]);
        if (off <= 1e-9f * sc) break;
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, qd = pq == 0 ? 1 : 2;
            float apq = S[3 * p + qd];
            if (fabsf(apq) <= 1e-30f) continue;
            float tau = (S[3 * qd + qd] - S[3 * p + p]) / (2.f * apq);
            float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            float cc = rsqrtf(1.f + t * t), ss = t * cc;
            for (int k = 0; k < 3; ++k) {  // S <- S J
                float skp = S[3 * k + p], skq = S[3 * k + qd];
                S[3 * k + p] = cc * skp - ss * skq;
                S[3 * k + qd] = ss * skp + cc * skq;
            }
            for (int k = 0; k < 3; ++k) {  // S <- J^T S
                float spk = S[3 * p + k], sqk = S[3 * qd + k];
                S[3 * p + k] = cc * spk - ss * sqk;
                S[3 * qd + k] = ss * spk + cc * sqk;
            }
            for (int k = 0; k < 3; ++k) {
                float vkp = V[3 * k + p], vkq = V[3 * k + qd];
                V[3 * k + p] = cc * vkp - ss * vkq;
                V[3 * k + qd] = ss * vkp + cc * vkq;
            }
        }
    }
    int o[3] = {0, 1, 2};
    float lam[3] = {S[0], S[4], S[8]};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (lam[o[b]] > lam[o[a]]) { int t = o[a]; o[a] = o[b]; o[b] = t; }
    float v[3][3], u[3][3];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) v[c][r] = V[3 * r + o[c]];
    // det V = +1
    float dv = v[0][0] * (v[1][1] * v[2][2] - v[1][2] * v[2][1]) - v[0][1] * (v[1][0] * v[2][2] - v[1][2] * v[2][0]) +
               v[0][2] * (v[1][0] * v[2][1] - v[1][1] * v[2][0]);
    if (dv < 0.f) for (int r = 0; r < 3; ++r) v[2][r] = -v[2][r];
    float av[3][3];
    for (int c = 0; c < 2; ++c)
        for (int r = 0; r < 3; ++r) av[c][r] = X[3 * r] * v[c][0] + X[3 * r + 1] * v[c][1] + X[3 * r + 2] * v[c][2];
    float n0 = sqrtf(av[0][0] * av[0][0] + av[0][1] * av[0][1] + av[0][2] * av[0][2]);
    if (n0 > 1e-20f) for (int r = 0; r < 3; ++r) u[0][r] = av[0][r] / n0;
    else { u[0][0] = v[0][0]; u[0][1] = v[0][1]; u[0][2] = v[0][2]; }
    float pr = u[0][0] * av[1][0] + u[0][1] * av[1][1] + u[0][2] * av[1][2];
    for (int r = 0; r < 3; ++r) u[1][r] = av[1][r] - pr * u[0][r];
    float n1 = sqrtf(u[1][0] * u[1][0] + u[1][1] * u[1][1] + u[1][2] * u[1][2]);
    if (n1 > 1e-20f) for (int r = 0; r < 3; ++r) u[1][r] /= n1;
    else {  // any unit vector orthogonal to u0
        int m = 0;
        for (int k = 1; k < 3; ++k) if (fabsf(u[0][k]) < fabsf(u[0][m])) m = k;
        float e[3] = {0.f, 0.f, 0.f};
        e[m] = 1.f;
        u[1][0] = u[0][1] * e[2] - u[0][2] * e[1];
        u[1][1] = u[0][2] * e[0] - u[0][0] * e[2];
        u[1][2] = u[0][0] * e[1] - u[0][1] * e[0];
        float nn = rsqrtf(u[1][0] * u[1][0] + u[1][1] * u[1][1] + u[1][2] * u[1][2]);
        for (int r = 0; r < 3; ++r) u[1][r] *= nn;
    }
    u[2][0] = u[0][1] * u[1][2] - u[0][2] * u[1][1];
    u[2][1] = u[0][2] * u[1][0] - u[0][0] * u[1][2];
    u[2][2] = u[0][0] * u[1][1] - u[0][1] * u[1][0];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) X[3 * r + c] = u[0][r] * v[0][c] + u[1][r] * v[1][c] + u[2][r] * v[2][c];
}

// The out-of-line eigen route works on a copy: were X's own address passed to it, X could not
// stay in registers on the common path.
__device__ __forceinline__ void polar_fallback(float* X) {
    float T[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) T[k] = X[k];
    polar_eigen(T);
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = T[k];
}

// Rotation of A^{k+1/2} (local solve), the orthogonal polar factor of X = A^{k+1/2}, in one
// inline loop for every body.  Each pass measures E = X^T X - I:
//   - ||E||_F^2 < 1e-13: done;
//   - ||E||_F^2 < 1/4: a Newton-Schulz step X <- X (3 I - X^T X) / 2 = X - X E / 2 (Higham
//     1986, Kovarik 1970): quadratic convergence from there, and a correction of X rather than
//     a recomputation, so it adds only the rounding of the correction;
//   - farther out (a stiffly jointed body's global update stretches A along its joints' lever
//     arms, past the Newton-Schulz region, for most jointed bodies of a batch of trees): a
//     step of Higham's scaled Newton iteration X <- (z X + X^-T / z) / 2, z = det(X)^(-1/3),
//     X^-T = cofactor(X) / det X, which converges from any nonsingular X.
// A det(X) that is not clearly positive (an inverted or degenerate A) goes to the
// eigen-decomposition route.
__device__ __forceinline__ void polar_rotation(float* X) {
    float C[9];
    cofactor(X, C);
    float det = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
    {
        const float nrm = X[0] * X[0] + X[1] * X[1] + X[2] * X[2] + X[3] * X[3] + X[4] * X[4] +
                          X[5] * X[5] + X[6] * X[6] + X[7] * X[7] + X[8] * X[8];
        if (!(det > 1e-6f * nrm * sqrtf(nrm))) { polar_fallback(X); return; }
    }
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
        float E[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = r; c < 3; ++c) {
                float t = X[r] * X[c] + X[3 + r] * X[3 + c] + X[6 + r] * X[6 + c];
                E[3 * r + c] = t - (r == c ? 1.f : 0.f);
                E[3 * c + r] = E[3 * r + c];
            }
        const float e2 = E[0] * E[0] + E[4] * E[4] + E[8] * E[8] + 2.f * (E[1] * E[1] + E[2] * E[2] + E[5] * E[5]);
        if (e2 < 1e-13f) break;
        if (e2 < 0.25f) {
            float Y[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    Y[3 * r + c] = X[3 * r + c] - 0.5f * (X[3 * r] * E[c] + X[3 * r + 1] * E[3 + c] + X[3 * r + 2] * E[6 + c]);
#pragma unroll
            for (int k = 0; k < 9; ++k) X[k] = Y[k];
        } else {
            if (it > 0) {
                cofactor(X, C);
                det = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
            }
            const float z = rcbrtf(det);
            const float iz = __frcp_rn(z * det);
#pragma unroll
            for (int k = 0; k < 9; ++k) X[k] = 0.5f * (z * X[k] + C[k] * iz);
        }
    }
}

template <class T>
__device__ __forceinline__ void sys_zero(Sys<T>& s) {
#pragma unroll
    for (int k = 0; k < 10; ++k) s.g[k] = T(0);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) s.r[r][k] = T(0);
}

// combine the L lanes' partial systems with a fixed xor butterfly (deterministic given L)
template <int L, class T>
__device__ __forceinline__ void sys_reduce(Sys<T>& s, unsigned mask) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 10; ++k) s.g[k] += shfl_xor(mask, s.g[k], o);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) s.r[r][k] += shfl_xor(mask, s.r[r][k], o);
    }
}

// The light bodies' slots 0..n-1, a warp's worth (32 / L slots) at a time, for the blocks from
// first_block on: each warp first takes the chunk of its own index, then the chunks past the
// grid's from the counter `next` until none are left, so the warps that finish early take more
// and a launch does not end on a few long blocks.  No counter traffic when the grid's warps
// cover every chunk.  f(slot) runs on the L lanes of each slot.
template <int L, class F>
__device__ __forceinline__ void for_light_slots(int* next, int n, int first_block, F&& f) {
    constexpr int PER_WARP = 32 / L;
    const int wpb = blockDim.x >> 5, wl = threadIdx.x & 31;
    const int warps = (gridDim.x - first_block) * wpb;
    const int chunks = (n + PER_WARP - 1) / PER_WARP;
    int chunk = (blockIdx.x - first_block) * wpb + (threadIdx.x >> 5);
    while (chunk < chunks) {
        const int slot = chunk * PER_WARP + wl / L;
        if (slot < n) f(slot);
        __syncwarp();
        if (warps >= chunks) break;
        int t = 0;
        if (wl == 0) t = atomicAdd(next, 1);
        chunk = warps + __shfl_sync(0xffffffffu, t, 0);
    }
    pdl_signal();  // nothing left for this warp
}

template <int L>
__device__ __forceinline__ unsigned lane_mask() {
    return (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1)));
}

__device__ __forceinline__ void finish_body(const Dev& d, int b, int lane, float4* __restrict__ qo, int last,
                                            const float* c, const float* A, const float (*Xs)[3]);


// Global + local solve of body b by L cooperating lanes (Eq. 19-24, Sec. 4.3):
// G dX = M (s - q^k) + sum_ends [1; x] f'^T, X^{k+1/2} = q^k + dX, A^{k+1} = rotation of
// A^{k+1/2}; lane 0 stores q^{k+1} and the body's squared update.  gather(sys, c, A, xs, e0,
// e1) adds this lane's share of the body's bond ends, about the expansion point xs: in FP32
// first; in the extended type X (double-float, or FP64) for flagged bodies (ill-conditioned or
// stiffly jointed, see the scene set-up) or when an FP32 Cholesky pivot falls below 1e-3 of
// its diagonal.
template <int L, class X, class Gather>
__device__ __forceinline__ void solve_body(const Dev& d, int b, int lane, unsigned mask,
                                           const float4* __restrict__ qi, float4* __restrict__ qo, int last,
                                           Gather&& gather, int max_ends = HEAVY_ENDS) {
    const int fl = d.bflags[b];
    if (fl & BF_PINNED) {
        if (lane == 0) {
            qo[3 * b] = d.qn[3 * b]; qo[3 * b + 1] = d.qn[3 * b + 1]; qo[3 * b + 2] = d.qn[3 * b + 2];
            if (last) d.resid_body[b] = 0.0;
        }
        return;
    }
    const int e0 = d.end_off[b], e1 = d.end_off[b + 1];
    if (e1 - e0 > max_ends) return;  // solved by the heavy role (heavy_role)
    if ((d.group_done && d.group_done[d.group[b]]) || held(d, b)) {  // stopped (residual threshold) or held
        if (lane == 0) { qo[3 * b] = qi[3 * b]; qo[3 * b + 1] = qi[3 * b + 1]; qo[3 * b + 2] = qi[3 * b + 2]; }
        return;
    }
    float c[3], A[9], sc[3], sA[9];
    ld_q(qi, b, c, A);
    ld_q(d.sq, b, sc, sA);
    float dc[3], dA[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) dc[k] = sc[k] - c[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) dA[k] = sA[k] - A[k];
    const float4 mass = d.mass[b];
    float xs[3];
    ld_xs(d, b, fl, xs);
    float Xs[4][3];
    bool ext = d.p.precision_policy == 3 || (d.p.precision_policy && (fl & BF_FP64));
    if (!ext) {
        Sys<float> s;
        if (lane == 0) sys_init(s, mass, dc, dA, xs);
        else sys_zero(s);
        gather(s, c, A, xs, e0, e1);
        sys_reduce<L>(s, mask);
        const float ratio = sys_solve(s, Xs);
        if (d.p.precision_policy && !(ratio >= 1e-3f)) {
            ext = true;
            if (last && lane == 0) atomicAdd(&d.ctr[C_FP64DYN], 1);
        }
    }
    if (ext) {
        Sys<X> s;
        if (lane == 0) sys_init(s, mass, dc, dA, xs);
        else sys_zero(s);
        gather(s, c, A, xs, e0, e1);
        sys_reduce<L>(s, mask);
        const auto se = ext_sys(s);
        ext_solve(se, Xs);
    }
    unshift(Xs, xs);
    finish_body(d, b, lane, qo, last, c, A, Xs);
}

// q^{k+1} from q^k and the solved update X: c + dc, rotation of A + dA; lane 0 stores it and,
// on the last sweep, the body's squared update and the finiteness check
__device__ __forceinline__ void finish_body(const Dev& d, int b, int lane, float4* __restrict__ qo, int last,
                                            const float* c, const float* A, const float (*Xs)[3]) {
    float cn[3], An[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cn[k] = c[k] + Xs[0][k];
#pragma unroll
        for (int l = 0; l < 3; ++l) An[3 * k + l] = A[3 * k + l] + Xs[1 + l][k];
    }
    if (d.p.project) polar_rotation(An);
    if (lane != 0) return;
    if (last) {  // residual and finiteness of the step's last sweep only
        double r2 = 0.0;
        bool finite = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) { double t = (double)cn[k] - (double)c[k]; r2 += t * t; finite &= isfinite(cn[k]); }
#pragma unroll
        for (int k = 0; k < 9; ++k) { double t = (double)An[k] - (double)A[k]; r2 += t * t; finite &= isfinite(An[k]); }
        if (!finite) atomicOr(&d.ctr[C_STATUS], ST_DIVERGED);
        d.resid_body[b] = r2;
    }
    qo[3 * b] = make_float4(cn[0], cn[1], cn[2], An[0]);
    qo[3 * b + 1] = make_float4(An[1], An[2], An[3], An[4]);
    qo[3 * b + 2] = make_float4(An[5], An[6], An[7], An[8]);
}

// an augmented Lagrangian bond's state is stored by end i, or by end j when i is pinned
__device__ __forceinline__ bool al_writer(const Dev& d, int4 m, int b) {
    return (m.z == K_AL) && (m.x == b || (d.bflags[m.x] & BF_PINNED));
}

// accumulate the ends lane, lane + L, ... of body b's CSR slice, in that order: each bond's
// force in single precision (end_force_q), summed into the system type T.  Two ends per round
// in FP32: both records and both other bodies' iterates are loaded before either force is
// evaluated, so a lane waits for two dependent loads per pair of ends.
template <int L, class T>
__device__ __forceinline__ void gather_ends(const Dev& d, const float4* __restrict__ q, int b, const float* cb,
                                            const float* Ab, const float* xs, int e0, int e1, int lane, int it,
                                            Sys<T>& s) {
    int p = e0 + lane;
    // (the extended type keeps one end per round: fewer live registers)
    if (sizeof(T) == 4) for (; p + L < e1; p += 2 * L) {
        const int4 m0 = d.rec_m[p], m1 = d.rec_m[p + L];
        const float4 a0 = d.rec_a[p], b0 = d.rec_b[p], a1 = d.rec_a[p + L], b1 = d.rec_b[p + L];
        float c0[3], A0[9], c1[3], A1[9];
        ld_q_or_zero(q, other_body(m0, b), c0, A0);
        ld_q_or_zero(q, other_body(m1, b), c1, A1);
        float f[3];
        float w = end_force_q(d, c0, A0, b, cb, Ab, m0, a0, b0, it, al_writer(d, m0, b), f);
        sys_add_t(s, w, f, (m0.y == b) ? b0 : a0, xs);
        w = end_force_q(d, c1, A1, b, cb, Ab, m1, a1, b1, it, al_writer(d, m1, b), f);
        sys_add_t(s, w, f, (m1.y == b) ? b1 : a1, xs);
    }
    for (; p < e1; p += L) {
        const int4 m = d.rec_m[p];
        const float4 xa = d.rec_a[p], xb = d.rec_b[p];
        float f[3];
        const float w = end_force(d, q, b, cb, Ab, m, xa, xb, it, al_writer(d, m, b), f);
        sys_add_t(s, w, f, (m.y == b) ? xb : xa, xs);
    }
}

// ---- bodies with many bond ends: one block of HEAVY_T threads per body ----

// Sum the block's partial systems: a xor butterfly inside each warp, then thread 0 adds the
// warps' sums in warp order (fixed, so the result depends only on HEAVY_T).  `buf` holds one
// system per warp (as doubles, wide enough for every T).  The total is valid in thread 0.
template <class T>
__device__ __forceinline__ void block_reduce(Sys<T>& s, Sys<T>* buf) {
    sys_reduce<32>(s, 0xffffffffu);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) buf[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < HEAVY_T / 32; ++k) {
#pragma unroll
            for (int i = 0; i < 10; ++i) s.g[i] += buf[k].g[i];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int i = 0; i < 3; ++i) s.r[r][i] += buf[k].r[r][i];
        }
    }
    __syncthreads();
}

// Global + local solve of body b (more than HEAVY_ENDS ends) by the whole block: thread t
// gathers ends t, t + HEAVY_T, ...; FP32 first, the extended type X where ill-conditioned
// (same rule as solve_body); thread 0 solves, projects and stores.  Every thread of the block
// must call it with the same b.
template <class X, class Gather>
__device__ __forceinline__ void solve_heavy(const Dev& d, int b, const float4* __restrict__ qi,
                                            float4* __restrict__ qo, int last, Gather&& gather) {
    __shared__ Sys<double> buf_raw[HEAVY_T / 32];
    __shared__ int s_ext;
    const int t = threadIdx.x;
    const int fl = d.bflags[b];
    if ((d.group_done && d.group_done[d.group[b]]) || held(d, b)) {  // stopped (residual threshold) or held
        if (t == 0) { qo[3 * b] = qi[3 * b]; qo[3 * b + 1] = qi[3 * b + 1]; qo[3 * b + 2] = qi[3 * b + 2]; }
        return;
    }
    const int e0 = d.end_off[b], e1 = d.end_off[b + 1];
    float c[3], A[9], sc[3], sA[9];
    ld_q(qi, b, c, A);
    ld_q(d.sq, b, sc, sA);
    float dc[3], dA[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) dc[k] = sc[k] - c[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) dA[k] = sA[k] - A[k];
    const float4 mass = d.mass[b];
    float xs[3];
    ld_xs(d, b, fl, xs);
    float Xs[4][3];
    if (t == 0) s_ext = d.p.precision_policy == 3 || (d.p.precision_policy && (fl & BF_FP64));
    __syncthreads();
    if (!s_ext) {
        Sys<float> s;
        if (t == 0) sys_init(s, mass, dc, dA, xs);
        else sys_zero(s);
        gather(s, c, A, xs, e0, e1);
        block_reduce(s, reinterpret_cast<Sys<float>*>(buf_raw));
        if (t == 0) {
            const float ratio = sys_solve(s, Xs);
            if (d.p.precision_policy && !(ratio >= 1e-3f)) {
                s_ext = 1;
                if (last) atomicAdd(&d.ctr[C_FP64DYN], 1);
            }
        }
        __syncthreads();
    }
    if (s_ext) {
        Sys<X> s;
        if (t == 0) sys_init(s, mass, dc, dA, xs);
        else sys_zero(s);
        gather(s, c, A, xs, e0, e1);
        block_reduce(s, reinterpret_cast<Sys<X>*>(buf_raw));
        if (t == 0) {
            const auto se = ext_sys(s);
            ext_solve(se, Xs);
        }
    }
    if (t == 0) {
        unshift(Xs, xs);
        finish_body(d, b, 0, qo, last, c, A, Xs);
    }
    __syncthreads();  // the shared buffers are reused by the block's next body
}

// The heavy role of a sweep launch's extra blocks (HEAVY_T threads each, block index hb of
// HEAVY_BLOCKS): the bodies on the heavy list with up to WIDE_ENDS ends, one warp each
// (32-lane butterfly, gather_w), then those with more, one block each (gather_b).  The
// summation order depends only on the body's end count, never on which block runs it.
template <class X, class GatherW, class GatherB>
__device__ __forceinline__ void heavy_role(const Dev& d, int hb, const float4* __restrict__ qi,
                                           float4* __restrict__ qo, int last, GatherW&& gather_w,
                                           GatherB&& gather_b) {
    const int nheavy = d.ctr[C_NHEAVY];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int h = hb * (HEAVY_T / 32) + warp; h < nheavy; h += HEAVY_BLOCKS * (HEAVY_T / 32)) {
        const int b = d.heavy[h];
        if (d.end_off[b + 1] - d.end_off[b] > WIDE_ENDS) continue;
        solve_body<32, X>(d, b, lane, 0xffffffffu, qi, qo, last,
                          [&](auto& s, const float* c, const float* A, const float* xs, int e0, int e1) {
                              gather_w(b, s, c, A, xs, e0, e1, lane);
                          },
                          WIDE_ENDS);
    }
    for (int h = hb; h < nheavy; h += HEAVY_BLOCKS) {
        const int b = d.heavy[h];
        if (d.end_off[b + 1] - d.end_off[b] <= WIDE_ENDS) continue;
        solve_heavy<X>(d, b, qi, qo, last, [&](auto& s, const float* c, const float* A, const float* xs, int e0, int e1) {
            gather_b(b, s, c, A, xs, e0, e1, (int)threadIdx.x);
        });
    }
}

}  // namespace pabd
