// Fused, persistent sweep: all n_iter global/local iterations of one step in one
// cooperative launch (a grid barrier between iterations), Jacobi double buffering.
//
// Each body is handled by a group of L lanes (L = 1..16, a power of two).  The lanes walk the
// body's CSR slice of bond-end records (copied in CSR order once per step, so the walk is a
// contiguous read), evaluate each bond's split force from q^k directly -- the same
// arithmetic as the bond kernel of the two-launch path -- and accumulate their share of the
// 4x4 system G dX = R; the shares are combined by a fixed butterfly of warp shuffles, so the
// result depends only on L, never on scheduling.  Every lane then solves, projects, and
// lane 0 stores q^{k+1}.  Bodies whose factorisation is ill-conditioned accumulate the same
// single-precision forces and solve in the extended type (same rule as the two-launch path).
//
// The grid barrier is a counter + generation word in device memory, cleared before every
// launch; every wait is bounded (by default 2^24 polls, about a second; pabd_set_wait_limit
// changes it), after which the block records PABD_ERR_TIMEOUT and leaves the kernel, and so
// do the blocks still running when they reach the next barrier, which can no longer fill.
// The launch is cooperative, so all blocks are co-resident.
#include "sweep_math.cuh"

namespace pabd {

__device__ __forceinline__ bool grid_sync(unsigned* bar, int* status, unsigned limit) {
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
                if (++spins > limit) {
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

template <int L, class X>
__global__ void __launch_bounds__(HEAVY_T, 4) k_sweep_fused(Dev d) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & (L - 1);
    const int grp = tid / L;
    const int ngrp = (gridDim.x * blockDim.x) / L;
    const unsigned mask = lane_mask<L>();
    const int nheavy = d.ctr[C_NHEAVY];
    const unsigned limit = *d.wait_limit;
    for (int it = 0; it < d.p.n_iter; ++it) {
        const float4* qi = (it & 1) ? d.qb : d.qa;
        float4* qo = (it & 1) ? d.qa : d.qb;
        const int last = it == d.p.n_iter - 1;
        // bodies with many ends first: the first HEAVY_BLOCKS blocks take the heavy role (the
        // launch uses HEAVY_T threads per block and at least HEAVY_BLOCKS blocks)
        if ((int)blockIdx.x < HEAVY_BLOCKS && nheavy > 0)
            heavy_role<X>(d, blockIdx.x, qi, qo, last,
                [&](int b, auto& s, const float* c, const float* A, const float* xs, int e0, int e1, int ln) {
                    gather_ends<32>(d, qi, b, c, A, xs, e0, e1, ln, it, s);
                },
                [&](int b, auto& s, const float* c, const float* A, const float* xs, int e0, int e1, int t) {
                    gather_ends<HEAVY_T>(d, qi, b, c, A, xs, e0, e1, t, it, s);
                });
        for (int b = grp; b < d.N; b += ngrp)
            solve_body<L, X>(d, b, lane, mask, qi, qo, last, [&](auto& s, const float* c, const float* A, const float* xs, int e0, int e1) {
                gather_ends<L>(d, qi, b, c, A, xs, e0, e1, lane, it, s);
            });
        if (it + 1 < d.p.n_iter && !grid_sync(d.gbar, &d.ctr[C_STATUS], limit)) return;
    }
}

// copy of every bond end's record into CSR order (once per step, after the CSR sort)
__global__ void k_end_records(Dev d) {
    pdl_enter();
    const int ne = d.end_off[d.N];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < ne; p += gridDim.x * blockDim.x) {
        const int bond = d.end_id[p] >> 1;
        const int4 m = d.bmeta[bond];
        d.rec_m[p] = make_int4(m.x, m.y, m.z, bond);
        d.rec_a[p] = d.bxi[bond];
        d.rec_b[p] = d.bxj[bond];
    }
}

using FusedFn = void (*)(Dev);

static FusedFn fused_fn(int L, bool fp64) {
    if (fp64) {
        switch (L) {
            case 1: return k_sweep_fused<1, double>;
            case 2: return k_sweep_fused<2, double>;
            case 4: return k_sweep_fused<4, double>;
            case 8: return k_sweep_fused<8, double>;
            default: return k_sweep_fused<16, double>;
        }
    }
    switch (L) {
        case 1: return k_sweep_fused<1, ca>;
        case 2: return k_sweep_fused<2, ca>;
        case 4: return k_sweep_fused<4, ca>;
        case 8: return k_sweep_fused<8, ca>;
        default: return k_sweep_fused<16, ca>;
    }
}

int fused_max_blocks(int L, int block, bool fp64) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_fn(L, fp64), block, 0);
    return per_sm * sms;
}

void launch_end_records(const Dev& d, cudaStream_t st, long long* launches) {
    const int nrec = d.cap_ends > 0 ? d.cap_ends : 1;
    launch_pdl(k_end_records, dim3(stride_grid(nrec, 256)), dim3(256), 0, st, d);
    *launches += 1;
}

cudaError_t launch_fused_sweep(const Dev& d, int L, int block, int grid, cudaStream_t st, long long* launches) {
    launch_end_records(d, st, launches);
    // a barrier that gave up in an earlier launch leaves its arrivals counted: start clean
    cudaMemsetAsync(d.gbar, 0, 2 * sizeof(unsigned), st);
    Dev dd = d;
    void* args[] = {&dd};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)fused_fn(L, d.p.precision_policy == 2), dim3(grid),
                                                dim3(block), args, 0, st);
    *launches += 1;
    return e;
}

}  // namespace pabd
