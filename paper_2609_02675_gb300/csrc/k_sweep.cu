// The semi-implicit successive-substitution sweep (Sec. 4.2-4.3), one launch pair per
// global/local iteration:
//
//   k_bond   one thread per bond: from q^k, the bond's split force (Eq. 15-17) as the two
//            ends' records (w, f'), w = h^2 phi+(d)/d and f' = f - w y_self, the right-hand
//            side term of Eq. 19 minus H's own-body term (the "delta" form) -- equal and
//            opposite f' on the two ends; each record is stored at the end's CSR slot.
//   k_solve  L lanes per body (the warp-cooperative gather): each lane adds its share of
//            the body's CSR slice and a fixed shuffle tree combines them; it forms, by the Kronecker
//            structure of H (Eq. 20, 23-24: H = P (G (x) I3) P^T with G the 4x4
//            diag(m, Pi) + sum w [1;x][1;x]^T), the 4x3 system G dX = M(s - q^k) + sum
//            [1;x] f'^T; factors G by Cholesky (the 12x12 Cholesky factor is L (x) I3),
//            solves the three right-hand sides, then takes the rotation of A^{k+1/2}
//            (the polar decomposition of sweep_math.cuh: Higham's scaled Newton
//            iteration, with an eigen-decomposition of A^T A as the fallback).
//            FP32, except bodies whose 4x4 factorisation is ill-conditioned (statically
//            flagged, or a Cholesky pivot below 1e-3 of its diagonal): those sum the same
//            single-precision records and factor in an extended type -- double-float on
//            the FP32 pipes (precision policy 1), or FP64 (policy 2).
#include "sweep_math.cuh"

namespace pabd {

constexpr int BOND_T = 256;
constexpr int SOLVE_T = 128;

// What a bond's records need that no sweep writes: its metadata and material points, the CSR
// slots of its ends and the ends' body flags (set at creation or by this step's front).
struct BondStatic {
    int4 m;
    float4 xi, xj;
    int p0, p1, fi, fj;
};

__device__ __forceinline__ BondStatic bond_static(const Dev& d, int b) {
    BondStatic s;
    s.m = d.bmeta[b];
    s.xi = d.bxi[b];
    s.xj = d.bxj[b];
    s.p0 = d.end_pos[2 * b];
    s.p1 = s.m.y >= 0 ? d.end_pos[2 * b + 1] : -1;
    s.fi = d.bflags[s.m.x];
    s.fj = s.m.y >= 0 ? d.bflags[s.m.y] : BF_PINNED;
    return s;
}

// one bond's end records from q^k
__device__ __forceinline__ void bond_one(const Dev& d, const float4* __restrict__ q, int it, int b,
                                         const BondStatic& s) {
    float c[3], A[9];
    ld_q(q, s.m.x, c, A);
    const int4 mm = make_int4(s.m.x, s.m.y, s.m.z, b);
    // a bond between two fixed ends is advanced by the final update alone (as in the sweep kernels)
    const bool writer = !(s.fi & BF_PINNED) || !(s.fj & BF_PINNED);
    float f[3];
    const float w = end_force(d, q, s.m.x, c, A, mm, s.xi, s.xj, it, writer, f);
    if (s.p0 >= 0) d.ends[s.p0] = make_float4(w, f[0], f[1], f[2]);
    if (s.p1 >= 0) d.ends[s.p1] = make_float4(w, -f[0], -f[1], -f[2]);
}

// (strides over this step's bonds with a grid capped at GS_BLOCKS blocks: the bond capacity
// holds room for every possible contact, far more than a step has).  Each thread loads its
// first bond's static part before it waits for the previous sweep (pdl_enter), so that the
// loads overlap that sweep's last blocks; q^k and the augmented Lagrangian state are read after.
__global__ void __launch_bounds__(BOND_T) k_bond(Dev d, const float4* __restrict__ q, int it) {
    const int nb = d.ctr[C_NBONDS];  // (set by the step's front, before the sweeps)
    const int b0 = blockIdx.x * blockDim.x + threadIdx.x;
    BondStatic s0;
    if (b0 < nb) s0 = bond_static(d, b0);
    pdl_enter();
    // the solve launch that follows hands out its light bodies from this counter (the previous
    // solve launch has finished: pdl_enter waited for it)
    if (blockIdx.x == 0 && threadIdx.x == 0) d.ctr[C_SOLVE_NEXT] = 0;
    if (b0 < nb) bond_one(d, q, it, b0, s0);
    for (int b = b0 + gridDim.x * blockDim.x; b < nb; b += gridDim.x * blockDim.x) bond_one(d, q, it, b, bond_static(d, b));
}

// add the records of ends p0, p0 + stride, ... < e1 in that order, each loaded one round
// ahead of its sum (the loads of the next end overlap the arithmetic of this one)
template <class T>
__device__ __forceinline__ void add_records(const Dev& d, Sys<T>& s, int p0, int e1, int stride, const float* xs) {
    if (p0 >= e1) return;
    float4 e = d.ends[p0], x = d.end_x[p0];
    for (int p = p0; p < e1; p += stride) {
        const float4 ec = e, xc = x;
        if (p + stride < e1) {
            e = d.ends[p + stride];
            x = d.end_x[p + stride];
        }
        sys_add(s, ec, xc, xs);
    }
}

// One body per group of L lanes; lane l adds the bond kernel's records of the body's ends
// l, l + L, ... -- in FP32, or in the extended type for a body on the extended path (the same
// records and order as the one-launch sweep, so the two modes agree bit for bit).  The first
// HEAVY_BLOCKS blocks take the heavy bodies (more than HEAVY_ENDS ends), a block each, and are
// dispatched first; the blocks after them stay resident and take the light bodies.
template <int L, class X>
__global__ void __launch_bounds__(SOLVE_T, 4) k_solve(Dev d, const float4* __restrict__ qi, float4* __restrict__ qo,
                                                   int it) {
    pdl_enter();
    const int last = it == d.p.n_iter - 1;
    if ((int)blockIdx.x < HEAVY_BLOCKS) {
        heavy_role<X>(d, blockIdx.x, qi, qo, last,
            [&](int b, auto& s, const float* c, const float* A, const float* xs, int e0, int e1, int ln) {
                add_records(d, s, e0 + ln, e1, 32, xs);
            },
            [&](int b, auto& s, const float* c, const float* A, const float* xs, int e0, int e1, int t) {
                add_records(d, s, e0 + t, e1, HEAVY_T, xs);
            });
        return;
    }
    // the light bodies in this step's (class, end count) order, or in body order (a body on
    // the heavy list then returns at once); either way the same arithmetic per body
    const int lane = threadIdx.x & (L - 1);
    for_light_slots<L>(&d.ctr[C_SOLVE_NEXT], d.light_sorted ? d.ctr[C_NLIGHT] : d.N, HEAVY_BLOCKS, [&](int slot) {
        const int b = d.light_sorted ? d.order[slot] : slot;
        solve_body<L, X>(d, b, lane, lane_mask<L>(), qi, qo, last,
                         [&](auto& s, const float* c, const float* A, const float* xs, int e0, int e1) {
            add_records(d, s, e0 + lane, e1, L, xs);
        });
    });
}

void launch_bond(const Dev& d, const float4* q, int it, cudaStream_t st, long long* launches) {
    launch_pdl(k_bond, dim3(stride_grid(d.cap_bonds > 0 ? d.cap_bonds : 1, BOND_T)), dim3(BOND_T), 0, st, d, q, it);
    *launches += 1;
}

void launch_solve(const Dev& d, const float4* q_in, float4* q_out, int it, int lanes, cudaStream_t st,
                  long long* launches) {
    static_assert(SOLVE_T == HEAVY_T, "the solve launch's blocks are the heavy bodies' blocks");
    // resident light blocks: as many as fit beside each other (4 per SM by the launch bounds),
    // fewer when the bodies do not need them
    const int slots = resident_slots(4);
    const long long n = (long long)(d.N > 0 ? d.N : 1) * lanes;
    const long long need = (n + SOLVE_T - 1) / SOLVE_T;
    const int light = (int)(need < slots ? need : slots);
    const int grid = HEAVY_BLOCKS + light;
    const bool f64 = d.p.precision_policy == 2;
    switch (lanes) {
        case 1: f64 ? launch_pdl(k_solve<1, double>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it)
                    : launch_pdl(k_solve<1, ca>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it); break;
        case 2: f64 ? launch_pdl(k_solve<2, double>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it)
                    : launch_pdl(k_solve<2, ca>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it); break;
        case 4: f64 ? launch_pdl(k_solve<4, double>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it)
                    : launch_pdl(k_solve<4, ca>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it); break;
        case 8: f64 ? launch_pdl(k_solve<8, double>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it)
                    : launch_pdl(k_solve<8, ca>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it); break;
        default: f64 ? launch_pdl(k_solve<16, double>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it)
                     : launch_pdl(k_solve<16, ca>, dim3(grid), dim3(SOLVE_T), 0, st, d, q_in, q_out, it); break;
    }
    *launches += 1;
}

}  // namespace pabd

namespace pabd {

// augmented Lagrangian warm start at the start of a step (Eq. 29), from the values the
// previous step ended with (parity n_iter): kappa <- max(gamma kappa, kappa_start),
// lambda <- alpha gamma lambda, into the parity-0 buffer read by the first sweep
__global__ void k_al_warm(Dev d) {
    pdl_enter();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.Nc || d.bmeta[b].z != K_AL) return;
    const float2 kl = (d.p.n_iter & 1) ? d.al_st1[b] : d.al_st0[b];
    const float4 pr = d.al_par[b];  // (kappa_start, beta, alpha, gamma)
    d.al_st0[b] = make_float2(fmaxf(pr.w * kl.x, pr.x), pr.z * pr.w * kl.y);
}

// the dual update from the step's final iterate (after the last sweep), into parity n_iter
__global__ void k_al_final(Dev d, const float4* __restrict__ q) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.Nc) return;
    const int4 m = d.bmeta[b];
    if (m.z != K_AL) return;
    const float4 xi = d.bxi[b], xj = d.bxj[b];
    float ci[3], Ai[9], cj[3], Aj[9], r[3];
    ld_q(q, m.x, ci, Ai);
    ld_q_or_zero(q, m.y, cj, Aj);
    bond_vec_dot2(ci, Ai, xi, cj, Aj, xj, m.y < 0, r);
    const float cc = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) - xj.w;
    const int it = d.p.n_iter;
    const float beta = d.al_par[b].y;
    float2* out = (it & 1) ? d.al_st1 : d.al_st0;
    const bool fixed_i = d.bflags[m.x] & BF_PINNED, fixed_j = m.y < 0 || (d.bflags[m.y] & BF_PINNED);
    if (fixed_i && fixed_j) {
        // no sweep evaluates a bond between two fixed ends; its constraint is the same at every
        // iterate, so all n_iter updates are taken here from the warm start
        float2 kl = d.al_st0[b];
        for (int k = 0; k < it; ++k) kl = make_float2(kl.x + beta * fabsf(cc), kl.x * cc + kl.y);
        out[b] = kl;
        return;
    }
    const float2 kl = ((it - 1) & 1) ? d.al_st1[b] : d.al_st0[b];
    out[b] = make_float2(kl.x + beta * fabsf(cc), kl.x * cc + kl.y);
}

void launch_al_warm(const Dev& d, cudaStream_t st, long long* launches) {
    if (d.Nal == 0) return;
    launch_pdl(k_al_warm, dim3((d.Nc + 255) / 256), dim3(256), 0, st, d);
    *launches += 1;
}

void launch_al_final(const Dev& d, const float4* q, cudaStream_t st, long long* launches) {
    if (d.Nal == 0) return;
    k_al_final<<<(d.Nc + 255) / 256, 256, 0, st>>>(d, q);
    *launches += 1;
}

}  // namespace pabd
