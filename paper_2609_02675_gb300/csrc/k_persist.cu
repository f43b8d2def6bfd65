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

// an augmented Lagrangian bond's state is stored by end i, or by end j when i is pinned
__device__ __forceinline__ bool al_writer(const Dev& d, int4 m, int b) {
    return (m.z == K_AL) && (m.x == b || (d.bflags[m.x] & BF_PINNED));
}

// accumulate the ends lane, lane + L, ... of body b's CSR slice (bond forces in T), in that
// order.  Two ends per round in FP32: both records and both other bodies' iterates are loaded
// before either force is evaluated, so a lane waits for two dependent loads per pair of ends.
template <int L, class T>
__device__ __forceinline__ void gather_ends(const Dev& d, const float4* __restrict__ q, int b, const float* cb,
                                            const float* Ab, const float* xs, int e0, int e1, int lane, int it,
                                            Sys<T>& s) {
    int p = e0 + lane;
    // (the FP64 redo, rare, keeps one end per round: fewer live registers)
    if (sizeof(T) == 4) for (; p + L < e1; p += 2 * L) {
        const int4 m0 = d.rec_m[p], m1 = d.rec_m[p + L];
        const float4 a0 = d.rec_a[p], b0 = d.rec_b[p], a1 = d.rec_a[p + L], b1 = d.rec_b[p + L];
        float c0[3], A0[9], c1[3], A1[9];
        ld_q_or_zero(q, other_body(m0, b), c0, A0);
        ld_q_or_zero(q, other_body(m1, b), c1, A1);
        T f[3];
        T w = end_force_q<T>(d, c0, A0, b, cb, Ab, m0, a0, b0, it, al_writer(d, m0, b), f);
        sys_add_t(s, w, f, (m0.y == b) ? b0 : a0, xs);
        w = end_force_q<T>(d, c1, A1, b, cb, Ab, m1, a1, b1, it, al_writer(d, m1, b), f);
        sys_add_t(s, w, f, (m1.y == b) ? b1 : a1, xs);
    }
    for (; p < e1; p += L) {
        const int4 m = d.rec_m[p];
        const float4 xa = d.rec_a[p], xb = d.rec_b[p];
        T f[3];
        const T w = end_force<T>(d, q, b, cb, Ab, m, xa, xb, it, al_writer(d, m, b), f);
        sys_add_t(s, w, f, (m.y == b) ? xb : xa, xs);
    }
}

template <int L, class X>
__global__ void __launch_bounds__(HEAVY_T, 4) k_sweep_fused(Dev d) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & (L - 1);
    const int grp = tid / L;
    const int ngrp = (gridDim.x * blockDim.x) / L;
    const unsigned mask = lane_mask<L>();
    const int nheavy = d.ctr[C_NHEAVY];
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
        if (it + 1 < d.p.n_iter && !grid_sync(d.gbar, &d.ctr[C_STATUS])) return;
    }
}

// One sweep per launch: the same per-body work as the fused kernel, with the launch boundary
// (a graph edge) in place of the grid barrier.  Capped at 128 registers (4 blocks per SM):
// the heavy role and the extended-precision paths, which alone need more, spill a little.  The first `light` blocks take the bodies with
// at most HEAVY_ENDS ends (L lanes each); the HEAVY_BLOCKS blocks after them take the heavy
// bodies, a block each.
template <int L, class X>
__global__ void __launch_bounds__(128, 4) k_sweep_one(Dev d, const float4* __restrict__ qi, float4* __restrict__ qo,
                                                   int it, int light) {
    const int last = it == d.p.n_iter - 1;
    if ((int)blockIdx.x >= light) {
        heavy_role<X>(d, blockIdx.x - light, qi, qo, last,
            [&](int b, auto& s, const float* c, const float* A, const float* xs, int e0, int e1, int ln) {
                gather_ends<32>(d, qi, b, c, A, xs, e0, e1, ln, it, s);
            },
            [&](int b, auto& s, const float* c, const float* A, const float* xs, int e0, int e1, int t) {
                gather_ends<HEAVY_T>(d, qi, b, c, A, xs, e0, e1, t, it, s);
            });
        return;
    }
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = tid / L, lane = tid & (L - 1);
    if (b >= d.N) return;
    solve_body<L, X>(d, b, lane, lane_mask<L>(), qi, qo, last, [&](auto& s, const float* c, const float* A, const float* xs, int e0, int e1) {
        gather_ends<L>(d, qi, b, c, A, xs, e0, e1, lane, it, s);
    });
}

void launch_end_records(const Dev& d, cudaStream_t st, long long* launches);

void launch_sweep_one(const Dev& d, const float4* qi, float4* qo, int it, int L, cudaStream_t st,
                      long long* launches) {
    static_assert(HEAVY_T == 128, "the sweep launch's blocks are the heavy bodies' blocks");
    const long long n = (long long)(d.N > 0 ? d.N : 1) * L;
    const int light = (int)((n + 127) / 128);
    const int grid = light + HEAVY_BLOCKS;
    // the extended type of ill-conditioned bodies: FP64 under policy 2, double-float otherwise
    if (d.p.precision_policy == 2) {
        switch (L) {
            case 1: k_sweep_one<1, double><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
            case 2: k_sweep_one<2, double><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
            case 4: k_sweep_one<4, double><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
            case 8: k_sweep_one<8, double><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
            default: k_sweep_one<16, double><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
        }
    } else {
        switch (L) {
            case 1: k_sweep_one<1, df><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
            case 2: k_sweep_one<2, df><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
            case 4: k_sweep_one<4, df><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
            case 8: k_sweep_one<8, df><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
            default: k_sweep_one<16, df><<<grid, 128, 0, st>>>(d, qi, qo, it, light); break;
        }
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
        case 1: return k_sweep_fused<1, df>;
        case 2: return k_sweep_fused<2, df>;
        case 4: return k_sweep_fused<4, df>;
        case 8: return k_sweep_fused<8, df>;
        default: return k_sweep_fused<16, df>;
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
    k_end_records<<<(nrec + 255) / 256, 256, 0, st>>>(d);
    *launches += 1;
}

cudaError_t launch_fused_sweep(const Dev& d, int L, int block, int grid, cudaStream_t st, long long* launches) {
    launch_end_records(d, st, launches);
    Dev dd = d;
    void* args[] = {&dd};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)fused_fn(L, d.p.precision_policy == 2), dim3(grid),
                                                dim3(block), args, 0, st);
    *launches += 1;
    return e;
}

}  // namespace pabd
