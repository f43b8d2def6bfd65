// The semi-implicit successive-substitution sweep (Sec. 4.2-4.3), one launch pair per
// global/local iteration:
//
//   k_bond   one thread per bond: from q^k, the bond's split force (Eq. 15-17) as the two
//            ends' records (w, f'), w = h^2 phi+(d)/d and f' = f - w y_self, the right-hand
//            side term of Eq. 19 minus H's own-body term (the "delta" form) -- equal and
//            opposite f' on the two ends; each record is stored at the end's CSR slot.
//   k_solve  one thread per body: gathers its CSR slice and forms, by the Kronecker
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
    float c[3], A[9], yi[3], yj[3];
    ld_q(q, m.x, c, A);
    world_pt(c, A, xi, yi);
    if (m.y >= 0) {
        ld_q(q, m.y, c, A);
        world_pt(c, A, xj, yj);
    } else {
        yj[0] = xj.x; yj[1] = xj.y; yj[2] = xj.z;
    }
    const float4 nm = (m.z == K_CONTACT || m.z == K_GROUND) ? d.bn[b] : make_float4(0.f, 0.f, 0.f, 0.f);
    float f[3];
    const float w = bond_force(m.z, xi, xj, nm, yi, yj, f);
    const int p0 = d.end_pos[2 * b], p1 = (m.y >= 0) ? d.end_pos[2 * b + 1] : -1;
    if (p0 >= 0) d.ends[p0] = make_float4(w, f[0], f[1], f[2]);
    if (p1 >= 0) d.ends[p1] = make_float4(w, -f[0], -f[1], -f[2]);
}

template <class T>
__device__ __forceinline__ T gather_solve(const Dev& d, int b, float4 mass, const float* dc, const float* dA,
                                          T out[4][3]) {
    Sys<T> s;
    sys_init(s, mass, dc, dA);
    const int e0 = d.end_off[b], e1 = d.end_off[b + 1];
    for (int p = e0; p < e1; ++p) sys_add(s, d.ends[p], d.end_x[p]);
    return sys_solve(s, out);
}

__global__ void __launch_bounds__(SOLVE_T) k_solve(Dev d, const float4* __restrict__ qi, float4* __restrict__ qo,
                                                   int last) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.N) return;
    const int fl = d.bflags[b];
    if (fl & BF_PINNED) {
        qo[3 * b] = d.qn[3 * b]; qo[3 * b + 1] = d.qn[3 * b + 1]; qo[3 * b + 2] = d.qn[3 * b + 2];
        d.resid_body[b] = 0.0;
        return;
    }
    float c[3], A[9], sc[3], sA[9];
    ld_q(qi, b, c, A);
    ld_q(d.sq, b, sc, sA);
    float dc[3], dA[9];
    for (int k = 0; k < 3; ++k) dc[k] = sc[k] - c[k];
    for (int k = 0; k < 9; ++k) dA[k] = sA[k] - A[k];
    const float4 mass = d.mass[b];
    float X[4][3];
    bool use64 = d.p.precision_policy && (fl & BF_FP64);
    if (!use64) {
        float ratio = gather_solve<float>(d, b, mass, dc, dA, X);
        if (!(ratio >= 1e-4f)) {
            if (d.p.precision_policy) {
                use64 = true;
                if (last) atomicAdd(&d.ctr[C_FP64DYN], 1);
            }
        }
    }
    if (use64) {
        double Xd[4][3];
        gather_solve<double>(d, b, mass, dc, dA, Xd);
        for (int r = 0; r < 4; ++r)
            for (int k = 0; k < 3; ++k) X[r][k] = (float)Xd[r][k];
    }
    float cn[3], An[9];
    for (int k = 0; k < 3; ++k) {
        cn[k] = c[k] + X[0][k];
        for (int l = 0; l < 3; ++l) An[3 * k + l] = A[3 * k + l] + X[1 + l][k];
    }
    if (d.p.project) polar_rotation(An);
    double r2 = 0.0;
    bool finite = true;
    for (int k = 0; k < 3; ++k) { double t = (double)cn[k] - (double)c[k]; r2 += t * t; finite &= isfinite(cn[k]); }
    for (int k = 0; k < 9; ++k) { double t = (double)An[k] - (double)A[k]; r2 += t * t; finite &= isfinite(An[k]); }
    if (!finite) atomicOr(&d.ctr[C_STATUS], ST_DIVERGED);
    d.resid_body[b] = r2;
    qo[3 * b] = make_float4(cn[0], cn[1], cn[2], An[0]);
    qo[3 * b + 1] = make_float4(An[1], An[2], An[3], An[4]);
    qo[3 * b + 2] = make_float4(An[5], An[6], An[7], An[8]);
}

void launch_bond(const Dev& d, const float4* q, cudaStream_t st, long long* launches) {
    const int n = d.cap_bonds > 0 ? d.cap_bonds : 1;
    k_bond<<<(n + BOND_T - 1) / BOND_T, BOND_T, 0, st>>>(d, q);
    *launches += 1;
}

void launch_solve(const Dev& d, const float4* q_in, float4* q_out, int last, cudaStream_t st, long long* launches) {
    const int n = d.N > 0 ? d.N : 1;
    if (last) cudaMemsetAsync(d.ctr + C_FP64DYN, 0, sizeof(int), st);
    k_solve<<<(n + SOLVE_T - 1) / SOLVE_T, SOLVE_T, 0, st>>>(d, q_in, q_out, last);
    *launches += 1;
}

}  // namespace pabd
