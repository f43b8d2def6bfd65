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
// (a graph edge) in place of the grid barrier.  Capped at 128 registers (4 blocks per SM),
// without spills (the fused kernel, which loops over the sweeps, spills a few bytes).  The
// first `light` blocks take the bodies with at most HEAVY_ENDS ends (L lanes each); the
// HEAVY_BLOCKS blocks after them take the heavy bodies.
template <int L, class X>
__global__ void __launch_bounds__(128, 4) k_sweep_one(Dev d, const float4* __restrict__ qi, float4* __restrict__ qo,
                                                   int it, int light) {
    // Programmatic dependent launch: wait until the previous sweep has completed and its writes
    // are visible (a no-op when launched without the attribute); no early signal to the next
    // sweep, whose waiting blocks would take SM slots (measured slower)
    pdl_enter();
    int last = it == d.p.n_iter - 1;
    if (it < 0) {
        // under a residual threshold: the sweep index and buffers from the device, the
        // per-body residual every sweep; nothing once the loop has ended (eager launches)
        if (!d.sweep_ctl[2]) return;
        it = d.sweep_ctl[0];
        qi = (it & 1) ? d.qb : d.qa;
        qo = (it & 1) ? d.qa : d.qb;
        last = 1;
    }
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

template <int L, class X>
static void sweep_one_ex(const Dev& d, const float4* qi, float4* qo, int it, int light, int grid, bool pdl,
                         cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k_sweep_one<L, X>, d, qi, qo, it, light);
}

template <class X>
static void sweep_one_l(const Dev& d, const float4* qi, float4* qo, int it, int L, int light, int grid, bool pdl,
                        cudaStream_t st) {
    switch (L) {
        case 1: sweep_one_ex<1, X>(d, qi, qo, it, light, grid, pdl, st); break;
        case 2: sweep_one_ex<2, X>(d, qi, qo, it, light, grid, pdl, st); break;
        case 4: sweep_one_ex<4, X>(d, qi, qo, it, light, grid, pdl, st); break;
        case 8: sweep_one_ex<8, X>(d, qi, qo, it, light, grid, pdl, st); break;
        default: sweep_one_ex<16, X>(d, qi, qo, it, light, grid, pdl, st); break;
    }
}

// `pdl`: launched as a programmatic dependent of the previous kernel on the stream (the
// previous sweep), so that its launch overlaps that sweep's tail
void launch_sweep_one(const Dev& d, const float4* qi, float4* qo, int it, int L, cudaStream_t st,
                      long long* launches, bool pdl) {
    static_assert(HEAVY_T == 128, "the sweep launch's blocks are the heavy bodies' blocks");
    const long long n = (long long)(d.N > 0 ? d.N : 1) * L;
    const int light = (int)((n + 127) / 128);
    const int grid = light + HEAVY_BLOCKS;
    // the extended type of ill-conditioned bodies: FP64 under policy 2, double-float otherwise
    if (d.p.precision_policy == 2) sweep_one_l<double>(d, qi, qo, it, L, light, grid, pdl, st);
    else sweep_one_l<df>(d, qi, qo, it, L, light, grid, pdl, st);
    *launches += 1;
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
    launch_pdl(k_end_records, dim3(stride_grid(nrec, 256)), dim3(256), 0, st, d);
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
