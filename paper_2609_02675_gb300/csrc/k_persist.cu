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

// accumulate the ends lane, lane + L, ... of body b's CSR slice (bond forces in T)
template <int L, class T>
__device__ __forceinline__ void gather_ends(const Dev& d, const float4* __restrict__ q, int b, const float* cb,
                                            const float* Ab, int e0, int e1, int lane, int it, Sys<T>& s) {
    for (int p = e0 + lane; p < e1; p += L) {
        const int4 m = d.rec_m[p];
        const float4 xa = d.rec_a[p], xb = d.rec_b[p];
        // an augmented Lagrangian bond's state is stored by end i, or by end j when i is pinned
        const bool writer = (m.z == K_AL) && (m.x == b || (d.bflags[m.x] & BF_PINNED));
        T f[3];
        const T w = end_force<T>(d, q, b, cb, Ab, m, xa, xb, it, writer, f);
        sys_add_t(s, w, f, (m.y == b) ? xb : xa);
    }
}

template <int L>
__global__ void k_sweep_fused(Dev d) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & (L - 1);
    const int grp = tid / L;
    const int ngrp = (gridDim.x * blockDim.x) / L;
    const unsigned mask = lane_mask<L>();
    for (int it = 0; it < d.p.n_iter; ++it) {
        const float4* qi = (it & 1) ? d.qb : d.qa;
        float4* qo = (it & 1) ? d.qa : d.qb;
        const int last = it == d.p.n_iter - 1;
        for (int b = grp; b < d.N; b += ngrp)
            solve_body<L>(d, b, lane, mask, qi, qo, last, [&](auto& s, const float* c, const float* A, int e0, int e1) {
                gather_ends<L>(d, qi, b, c, A, e0, e1, lane, it, s);
            });
        if (it + 1 < d.p.n_iter && !grid_sync(d.gbar, &d.ctr[C_STATUS])) return;
    }
}

// One sweep per launch: the same per-body work as the fused kernel, with the launch boundary
// (a graph edge) in place of the grid barrier.
template <int L>
__global__ void __launch_bounds__(128) k_sweep_one(Dev d, const float4* __restrict__ qi, float4* __restrict__ qo,
                                                   int it) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = tid / L, lane = tid & (L - 1);
    if (b >= d.N) return;
    const int last = it == d.p.n_iter - 1;
    solve_body<L>(d, b, lane, lane_mask<L>(), qi, qo, last, [&](auto& s, const float* c, const float* A, int e0, int e1) {
        gather_ends<L>(d, qi, b, c, A, e0, e1, lane, it, s);
    });
}

void launch_end_records(const Dev& d, cudaStream_t st, long long* launches);

void launch_sweep_one(const Dev& d, const float4* qi, float4* qo, int it, int L, cudaStream_t st,
                      long long* launches) {
    const long long n = (long long)(d.N > 0 ? d.N : 1) * L;
    const int grid = (int)((n + 127) / 128);
    if (it == d.p.n_iter - 1) cudaMemsetAsync(d.ctr + C_FP64DYN, 0, sizeof(int), st);
    switch (L) {
        case 1: k_sweep_one<1><<<grid, 128, 0, st>>>(d, qi, qo, it); break;
        case 2: k_sweep_one<2><<<grid, 128, 0, st>>>(d, qi, qo, it); break;
        case 4: k_sweep_one<4><<<grid, 128, 0, st>>>(d, qi, qo, it); break;
        case 8: k_sweep_one<8><<<grid, 128, 0, st>>>(d, qi, qo, it); break;
        default: k_sweep_one<16><<<grid, 128, 0, st>>>(d, qi, qo, it); break;
    }
    *launches += 1;
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

void launch_end_records(const Dev& d, cudaStream_t st, long long* launches) {
    const int nrec = d.cap_ends > 0 ? d.cap_ends : 1;
    k_end_records<<<(nrec + 255) / 256, 256, 0, st>>>(d);
    *launches += 1;
}

cudaError_t launch_fused_sweep(const Dev& d, int L, int block, int grid, cudaStream_t st, long long* launches) {
    launch_end_records(d, st, launches);
    Dev dd = d;
    void* args[] = {&dd};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)fused_fn(L), dim3(grid), dim3(block), args, 0, st);
    *launches += 1;
    return e;
}

}  // namespace pabd
