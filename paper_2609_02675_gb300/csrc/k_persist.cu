// Fused, persistent sweep: all n_iter global/local iterations of one step in one
// cooperative launch (a grid barrier between iterations), Jacobi double buffering.
//
// Each body is handled by a group of L lanes (L = 1..16, a power of two).  The lanes walk the
// body's CSR slice of bond-end records (copied in CSR order once per step, so the walk is a
// contiguous read), evaluate each bond's split force from q^k directly -- the same
// arithmetic as the bond kernel of the two-launch path -- and accumulate their share of the
// 4x4 system G dX = R; the shares are combined by a fixed butterfly of warp shuffles, so the
// result depends only on L, never on scheduling.  Every lane then solves, projects, and
// lane 0 stores q^{k+1}.  Bodies whose factorisation is ill-conditioned redo the
// accumulation and the solve in FP64 (same rule as the two-launch path).
//
// The grid barrier is a counter + generation word in device memory; every wait is bounded
// (about a second), after which the block records PABD_ERR_TIMEOUT and leaves the kernel.
// The launch is cooperative, so all blocks are co-resident.
#include "sweep_math.cuh"

namespace pabd {

__device__ __forceinline__ bool grid_sync(unsigned* bar, int* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned prev = atomicAdd(bar, 1u);
        int ok = 1;
        if (prev == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned spins = 0;
            while (*vgen == gen) {  // poll without sleeping first, then back off
                if (++spins > (1u << 24)) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (spins > 4096) __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T, int L>
__device__ __forceinline__ void sys_reduce(Sys<T>& s, unsigned mask) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 10; ++k) s.g[k] += __shfl_xor_sync(mask, s.g[k], o);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) s.r[r][k] += __shfl_xor_sync(mask, s.r[r][k], o);
    }
}

// accumulate the ends lane, lane + L, ... of body b's CSR slice
template <class T, int L>
__device__ __forceinline__ void gather_ends(const Dev& d, const float4* __restrict__ q, int b, const float* cb,
                                            const float* Ab, int e0, int e1, int lane, Sys<T>& s) {
    for (int p = e0 + lane; p < e1; p += L) {
        const int4 m = d.rec_m[p];
        const float4 xa = d.rec_a[p], xb = d.rec_b[p];
        const bool side_j = (m.y == b);
        float c[3], A[9], yi[3], yj[3];
        if (side_j) {
            ld_q(q, m.x, c, A);
            world_pt(c, A, xa, yi);
            world_pt(cb, Ab, xb, yj);
        } else {
            world_pt(cb, Ab, xa, yi);
            if (m.y >= 0) {
                ld_q(q, m.y, c, A);
                world_pt(c, A, xb, yj);
            } else {
                yj[0] = xb.x; yj[1] = xb.y; yj[2] = xb.z;
            }
        }
        const float4 nm = (m.z == K_CONTACT || m.z == K_GROUND) ? d.bn[m.w] : make_float4(0.f, 0.f, 0.f, 0.f);
        float f[3];
        const float w = bond_force(m.z, xa, xb, nm, yi, yj, f);
        const float sg = side_j ? -1.f : 1.f;
        sys_add(s, make_float4(w, sg * f[0], sg * f[1], sg * f[2]), side_j ? xb : xa);
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

template <int L>
__device__ __forceinline__ void body_update(const Dev& d, int b, int lane, unsigned mask,
                                            const float4* __restrict__ qi, float4* __restrict__ qo, int last) {
    const int fl = d.bflags[b];
    if (fl & BF_PINNED) {
        if (lane == 0) {
            qo[3 * b] = d.qn[3 * b]; qo[3 * b + 1] = d.qn[3 * b + 1]; qo[3 * b + 2] = d.qn[3 * b + 2];
            d.resid_body[b] = 0.0;
        }
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
    const int e0 = d.end_off[b], e1 = d.end_off[b + 1];
    float X[4][3];
    bool use64 = d.p.precision_policy && (fl & BF_FP64);
    if (!use64) {
        Sys<float> s;
        if (lane == 0) sys_init(s, mass, dc, dA);
        else sys_zero(s);
        gather_ends<float, L>(d, qi, b, c, A, e0, e1, lane, s);
        sys_reduce<float, L>(s, mask);
        const float ratio = sys_solve(s, X);
        if (!(ratio >= 1e-4f) && d.p.precision_policy) {
            use64 = true;
            if (last && lane == 0) atomicAdd(&d.ctr[C_FP64DYN], 1);
        }
    }
    if (use64) {
        Sys<double> s;
        if (lane == 0) sys_init(s, mass, dc, dA);
        else sys_zero(s);
        gather_ends<double, L>(d, qi, b, c, A, e0, e1, lane, s);
        sys_reduce<double, L>(s, mask);
        double Xd[4][3];
        sys_solve(s, Xd);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) X[r][k] = (float)Xd[r][k];
    }
    float cn[3], An[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cn[k] = c[k] + X[0][k];
#pragma unroll
        for (int l = 0; l < 3; ++l) An[3 * k + l] = A[3 * k + l] + X[1 + l][k];
    }
    if (d.p.project) polar_rotation(An);
    if (lane != 0) return;
    double r2 = 0.0;
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) { double t = (double)cn[k] - (double)c[k]; r2 += t * t; finite &= isfinite(cn[k]); }
#pragma unroll
    for (int k = 0; k < 9; ++k) { double t = (double)An[k] - (double)A[k]; r2 += t * t; finite &= isfinite(An[k]); }
    if (!finite) atomicOr(&d.ctr[C_STATUS], ST_DIVERGED);
    d.resid_body[b] = r2;
    qo[3 * b] = make_float4(cn[0], cn[1], cn[2], An[0]);
    qo[3 * b + 1] = make_float4(An[1], An[2], An[3], An[4]);
    qo[3 * b + 2] = make_float4(An[5], An[6], An[7], An[8]);
}

template <int L>
__global__ void k_sweep_fused(Dev d) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & (L - 1);
    const int grp = tid / L;
    const int ngrp = (gridDim.x * blockDim.x) / L;
    const unsigned mask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1)));
    for (int it = 0; it < d.p.n_iter; ++it) {
        const float4* qi = (it & 1) ? d.qb : d.qa;
        float4* qo = (it & 1) ? d.qa : d.qb;
        const int last = it == d.p.n_iter - 1;
        for (int b = grp; b < d.N; b += ngrp) body_update<L>(d, b, lane, mask, qi, qo, last);
        if (it + 1 < d.p.n_iter && !grid_sync(d.gbar, &d.ctr[C_STATUS])) return;
    }
}

// copy of every bond end's record into CSR order (once per step, after the CSR sort)
__global__ void k_end_records(Dev d) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d.end_off[d.N]) return;
    const int bond = d.end_id[p] >> 1;
    const int4 m = d.bmeta[bond];
    d.rec_m[p] = make_int4(m.x, m.y, m.z, bond);
    d.rec_a[p] = d.bxi[bond];
    d.rec_b[p] = d.bxj[bond];
}

using FusedFn = void (*)(Dev);

static FusedFn fused_fn(int L) {
    switch (L) {
        case 1: return k_sweep_fused<1>;
        case 2: return k_sweep_fused<2>;
        case 4: return k_sweep_fused<4>;
        case 8: return k_sweep_fused<8>;
        default: return k_sweep_fused<16>;
    }
}

int fused_max_blocks(int L, int block) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_fn(L), block, 0);
    return per_sm * sms;
}

cudaError_t launch_fused_sweep(const Dev& d, int L, int block, int grid, cudaStream_t st, long long* launches) {
    const int nrec = d.cap_ends > 0 ? d.cap_ends : 1;
    k_end_records<<<(nrec + 255) / 256, 256, 0, st>>>(d);
    Dev dd = d;
    void* args[] = {&dd};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)fused_fn(L), dim3(grid), dim3(block), args, 0, st);
    *launches += 2;
    return e;
}

}  // namespace pabd
