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
//            solves the three right-hand sides, then takes the rotation of A^{k+1/2} by
//            Higham's scaled Newton iteration for the polar decomposition
//            (X <- (z X + X^-T / z)/2, z = |det X|^(-1/3)); a near-singular or reflected
//            A falls back to an eigen-decomposition of A^T A with the proper-rotation
//            sign fix.  FP32, except bodies whose 4x4 factorisation is ill-conditioned
//            (statically flagged, or a Cholesky pivot below 1e-4 of its diagonal): those
//            re-gather and factor in FP64.
#include "sweep_math.cuh"

namespace pabd {

constexpr int BOND_T = 256;
constexpr int SOLVE_T = 128;

__global__ void __launch_bounds__(BOND_T) k_bond(Dev d, const float4* __restrict__ q, int it) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.ctr[C_NBONDS]) return;
    const int4 m = d.bmeta[b];
    const float4 xi = d.bxi[b], xj = d.bxj[b];
    float c[3], A[9];
    ld_q(q, m.x, c, A);
    const int4 mm = make_int4(m.x, m.y, m.z, b);
    const int fi = d.bflags[m.x], fj = m.y >= 0 ? d.bflags[m.y] : BF_PINNED;
    const bool dbl = d.p.precision_policy && ((fi | fj) & BF_FP64);
    // a bond between two fixed ends is advanced by the final update alone (as in the sweep kernels)
    const bool writer = !(fi & BF_PINNED) || !(fj & BF_PINNED);
    float w, f[3];
    if (dbl) {
        double fd[3];
        w = (float)end_force<double>(d, q, m.x, c, A, mm, xi, xj, it, writer, fd);
        f[0] = (float)fd[0]; f[1] = (float)fd[1]; f[2] = (float)fd[2];
    } else {
        w = end_force<float>(d, q, m.x, c, A, mm, xi, xj, it, writer, f);
    }
    const int p0 = d.end_pos[2 * b], p1 = (m.y >= 0) ? d.end_pos[2 * b + 1] : -1;
    if (p0 >= 0) d.ends[p0] = make_float4(w, f[0], f[1], f[2]);
    if (p1 >= 0) d.ends[p1] = make_float4(w, -f[0], -f[1], -f[2]);
}

// one body per group of L lanes; lane l adds the body's ends l, l + L, ... (float records)
template <int L>
__global__ void __launch_bounds__(SOLVE_T) k_solve(Dev d, const float4* __restrict__ qi, float4* __restrict__ qo,
                                                   int last) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = tid / L, lane = tid & (L - 1);
    if (b >= d.N) return;
    solve_body<L>(d, b, lane, lane_mask<L>(), qi, qo, last, [&](auto& s, const float*, const float*, int e0, int e1) {
        for (int p = e0 + lane; p < e1; p += L) sys_add(s, d.ends[p], d.end_x[p]);
    });
}

void launch_bond(const Dev& d, const float4* q, int it, cudaStream_t st, long long* launches) {
    const int n = d.cap_bonds > 0 ? d.cap_bonds : 1;
    k_bond<<<(n + BOND_T - 1) / BOND_T, BOND_T, 0, st>>>(d, q, it);
    *launches += 1;
}

void launch_solve(const Dev& d, const float4* q_in, float4* q_out, int last, int lanes, cudaStream_t st,
                  long long* launches) {
    const long long n = (long long)(d.N > 0 ? d.N : 1) * lanes;
    const int grid = (int)((n + SOLVE_T - 1) / SOLVE_T);
    if (last) cudaMemsetAsync(d.ctr + C_FP64DYN, 0, sizeof(int), st);
    switch (lanes) {
        case 1: k_solve<1><<<grid, SOLVE_T, 0, st>>>(d, q_in, q_out, last); break;
        case 2: k_solve<2><<<grid, SOLVE_T, 0, st>>>(d, q_in, q_out, last); break;
        case 4: k_solve<4><<<grid, SOLVE_T, 0, st>>>(d, q_in, q_out, last); break;
        case 8: k_solve<8><<<grid, SOLVE_T, 0, st>>>(d, q_in, q_out, last); break;
        default: k_solve<16><<<grid, SOLVE_T, 0, st>>>(d, q_in, q_out, last); break;
    }
    *launches += 1;
}

}  // namespace pabd

namespace pabd {

// augmented Lagrangian warm start at the start of a step (Eq. 29), from the values the
// previous step ended with (parity n_iter): kappa <- max(gamma kappa, kappa_start),
// lambda <- alpha gamma lambda, into the parity-0 buffer read by the first sweep
__global__ void k_al_warm(Dev d) {
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
    float c[3], A[9], yi[3], yj[3];
    ld_q(q, m.x, c, A);
    world_pt_t(c, A, xi, yi);
    if (m.y >= 0) { ld_q(q, m.y, c, A); world_pt_t(c, A, xj, yj); }
    else { yj[0] = xj.x; yj[1] = xj.y; yj[2] = xj.z; }
    const float r0 = yj[0] - yi[0], r1 = yj[1] - yi[1], r2 = yj[2] - yi[2];
    const float cc = sqrtf(r0 * r0 + r1 * r1 + r2 * r2) - xj.w;
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
    k_al_warm<<<(d.Nc + 255) / 256, 256, 0, st>>>(d);
    *launches += 1;
}

void launch_al_final(const Dev& d, const float4* q, cudaStream_t st, long long* launches) {
    if (d.Nal == 0) return;
    k_al_final<<<(d.Nc + 255) / 256, 256, 0, st>>>(d, q);
    *launches += 1;
}

}  // namespace pabd
