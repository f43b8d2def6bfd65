// One launch per sweep (sweep mode 2): every body gathers its bond ends from the CSR-ordered
// end records, evaluates each bond's split force from q^k (Eq. 15-17) and solves its 4x4
// system and local rotation (Eq. 19-24, Sec. 4.3); the launch boundary orders the sweeps.
#include "sweep_math.cuh"

namespace pabd {

// One sweep per launch: the same per-body work as the fused kernel, with the launch boundary
// (a graph edge) in place of the grid barrier.  Capped at 128 registers (4 blocks per SM),
// without spills (the fused kernel, which loops over the sweeps, spills a few bytes).  The
// first HEAVY_BLOCKS blocks take the heavy bodies (more than HEAVY_ENDS ends) and are
// dispatched first; the blocks after them stay resident and take the light bodies (L lanes
// each, in the step's light order), a warp's worth at a time (for_light_slots).
template <int L, class X>
__global__ void __launch_bounds__(128, 4) k_sweep_one(Dev d, const float4* __restrict__ qi, float4* __restrict__ qo,
                                                   int it) {
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
    // this sweep's counter of light chunks, and the next sweep's zeroed (the previous sweep,
    // which used it, has finished)
    int* next = &d.ctr[C_SWEEP_NEXT + (it & 1)];
    if (blockIdx.x == 0 && threadIdx.x == 0) d.ctr[C_SWEEP_NEXT + ((it + 1) & 1)] = 0;
    if ((int)blockIdx.x < HEAVY_BLOCKS) {
        heavy_role<X>(d, blockIdx.x, qi, qo, last,
            [&](int b, auto& s, const float* c, const float* A, const float* xs, int e0, int e1, int ln) {
                gather_ends<32>(d, qi, b, c, A, xs, e0, e1, ln, it, s);
            },
            [&](int b, auto& s, const float* c, const float* A, const float* xs, int e0, int e1, int t) {
                gather_ends<HEAVY_T>(d, qi, b, c, A, xs, e0, e1, t, it, s);
            });
        return;
    }
    // the light bodies in this step's (class, end count) order, or in body order (a body on
    // the heavy list then returns at once); either way the same arithmetic per body
    const int lane = threadIdx.x & (L - 1);
    for_light_slots<L>(next, d.light_sorted ? d.ctr[C_NLIGHT] : d.N, HEAVY_BLOCKS, [&](int slot) {
        const int b = d.light_sorted ? d.order[slot] : slot;
        solve_body<L, X>(d, b, lane, lane_mask<L>(), qi, qo, last,
                         [&](auto& s, const float* c, const float* A, const float* xs, int e0, int e1) {
            gather_ends<L>(d, qi, b, c, A, xs, e0, e1, lane, it, s);
        });
    });
}

template <int L, class X>
static void sweep_one_ex(const Dev& d, const float4* qi, float4* qo, int it, int grid, bool pdl,
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
    cudaLaunchKernelEx(&cfg, k_sweep_one<L, X>, d, qi, qo, it);
}

template <class X>
static void sweep_one_l(const Dev& d, const float4* qi, float4* qo, int it, int L, int grid, bool pdl,
                        cudaStream_t st) {
    switch (L) {
        case 1: sweep_one_ex<1, X>(d, qi, qo, it, grid, pdl, st); break;
        case 2: sweep_one_ex<2, X>(d, qi, qo, it, grid, pdl, st); break;
        case 4: sweep_one_ex<4, X>(d, qi, qo, it, grid, pdl, st); break;
        case 8: sweep_one_ex<8, X>(d, qi, qo, it, grid, pdl, st); break;
        default: sweep_one_ex<16, X>(d, qi, qo, it, grid, pdl, st); break;
    }
}

// `pdl`: launched as a programmatic dependent of the previous kernel on the stream (the
// previous sweep), so that its launch overlaps that sweep's tail
void launch_sweep_one(const Dev& d, const float4* qi, float4* qo, int it, int L, cudaStream_t st,
                      long long* launches, bool pdl) {
    static_assert(HEAVY_T == 128, "the sweep launch's blocks are the heavy bodies' blocks");
    const long long n = (long long)(d.N > 0 ? d.N : 1) * L;
    const long long need = (n + 127) / 128;
    const int slots = resident_slots(4);
    const int grid = HEAVY_BLOCKS + (int)(need < slots ? need : slots);
    // the extended type of ill-conditioned bodies: FP64 under policy 2, double-float otherwise
    if (d.p.precision_policy == 2) sweep_one_l<double>(d, qi, qo, it, L, grid, pdl, st);
    else sweep_one_l<ca>(d, qi, qo, it, L, grid, pdl, st);
    *launches += 1;
}

}  // namespace pabd
