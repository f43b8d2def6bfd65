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

__global__ void __launch_bounds__(BOND_T) k_bond(Dev d, const float4* __restrict__ q) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.ctr[C_NBONDS]) return;
    const int4 m = d.bmeta[b];
    const float4 xi = d.bxi[b], xj = d.bxj[b];
    float c[3], A[9];
    ld_q(q, m.x, c, A);
    const int4 mm = make_int4(m.x, m.y, m.z, b);
    const bool dbl = d.p.precision_policy &&
                     ((d.bflags[m.x] | (m.y >= 0 ? d.bflags[m.y] : 0)) & BF_FP64);
    float w, f[3];
    if (dbl) {
        double fd[3];
        w = (float)end_force<double>(q, d.bn, m.x, c, A, mm, xi, xj, fd);
        f[0] = (float)fd[0]; f[1] = (float)fd[1]; f[2] = (float)fd[2];
    } else {
        w = end_force<float>(q, d.bn, m.x, c, A, mm, xi, xj, f);
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

void launch_bond(const Dev& d, const float4* q, cudaStream_t st, long long* launches) {
    const int n = d.cap_bonds > 0 ? d.cap_bonds : 1;
    k_bond<<<(n + BOND_T - 1) / BOND_T, BOND_T, 0, st>>>(d, q);
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
