// Internal layout of a scene on the device and the launchers of every kernel.
//
// Memory layout (structure of arrays; one slot per body / bond / bond end):
//   q (12 floats per body) as 3 float4: (c0 c1 c2 A00) (A01 A02 A10 A11) (A12 A20 A21 A22),
//   i.e. the generalised coordinates q = (c, a1, a2, a3) of Eq. 1 in order, 48 contiguous
//   bytes per body so a gather of one body is three 16-byte loads of one 64-byte segment.
//   Bonds: meta int4 (i, j, type, aux), xi float4 (x_i, w0), xj float4 (x_j, p1),
//   bn float4 (N, mu) -- static bonds first, then this step's contact bonds.
//   Bond ends: a CSR over bodies sorted by (body, 2*bond + side); per end the bond kernel
//   writes one float4 (w, f') at its CSR slot and the solve reads its body's slice.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pabd {

enum BondKind { K_SPHERICAL = 0, K_SPRING = 1, K_ELASTIC_NL = 2, K_DRIVE = 4, K_CONTACT = 5, K_GROUND = 6, K_AL = 7 };

enum StatusBits { ST_CAPACITY = 1, ST_DIVERGED = 2, ST_TIMEOUT = 4 };

// BF_SHIFT: the body's system is assembled about a nonzero expansion point Dev::xs.
// BF_STIFF: its static bonds' weights sum to more than 10 times its mass (stiff joints).
enum BodyFlags { BF_PINNED = 1, BF_FP64 = 2, BF_LARGE = 4, BF_SHIFT = 8, BF_STIFF = 16 };

// device counters (ints) -- one small array so that one memset resets them
enum Counter {
    C_NPAIRS = 0,      // broad-phase pairs (clamped to capacity)
    C_NPC,             // body-body contacts
    C_NGC,             // ground contacts
    C_NBONDS,          // static + contact bonds this step
    C_STATUS,          // latched StatusBits (never reset by a step)
    C_CELLBITS,        // float bits of the grid cell size
    C_FP64DYN,         // bodies that switched to FP64 by the pivot test (last sweep)
    C_NHEAVY,          // bodies with more than HEAVY_ENDS bond ends this step (list in Dev::heavy)
    C_NLARGE,          // bodies off the grid this step (list in Dev::large_ids)
    C_NPHEAVY,         // bodies with more than 64 partners this step (list in Dev::pair_heavy)
    C_CELLBITS1,       // float bits of the widest box of grid level 1 (multilevel grid)
    C_CELLBITS2,       // ... of grid level 2
    C_NLIGHT,          // bodies on this step's light list (Dev::order)
    C_SOLVE_NEXT,      // next chunk of light bodies for the solve launch's warps (reset by k_bond)
    C_SWEEP_NEXT,      // the same for the one-launch sweeps, one counter per sweep parity: sweep k
    C_SWEEP_NEXT1,     // takes counter k & 1 and zeroes the other one for sweep k + 1
    C_COUNT
};

struct Params {
    float h, h2, inv_h;
    float g[3];
    float gn[3], gd;
    float mu, c_kappa, d_hat_rel, margin;
    float cell;                 // cap of the grid cell size (0: none); wider boxes leave the grid
    double resid_tol;           // per-scene residual threshold of the sweeps (0: fixed n_iter)
    int broadphase;             // 0: uniform grid hash, 1: linear BVH
    int n_iter, has_ground, project, body_contacts, precision_policy;
    double h_d;
};

// A body with more than HEAVY_ENDS bond ends (a large body under a pile or a bed of grains)
// is gathered and solved by a whole block of HEAVY_T threads instead of L lanes (the last
// HEAVY_BLOCKS blocks of every sweep launch take the heavy bodies), and its CSR slice is
// sorted by a block.
constexpr int HEAVY_ENDS = 64;
constexpr int HEAVY_T = 128;
// of those, bodies with up to WIDE_ENDS ends are summed by one warp (32 lanes), more by the block
constexpr int WIDE_ENDS = 256;
// blocks of each sweep launch for the heavy bodies (they loop over the heavy list)
constexpr int HEAVY_BLOCKS = 152;
// The light bodies (at most HEAVY_ENDS ends) are ordered every step by (class, end count):
// the bodies on the extended path first, then the rest, each class from the most ends to the
// fewest, so that the lanes of one warp walk slices of the same length down the same path and
// the longest warps start first (the launch does not end on them).  2 * END_BINS bins; which
// lanes take a body never changes its arithmetic.
constexpr int END_BINS = HEAVY_ENDS + 1;
constexpr int RES_CHUNK = 4096;
constexpr int PAIR_STASH = 4;
constexpr int STASH_DELIVER = 0x40000000;

struct Dev {
    Params p;
    int N, Nc, Ndrive, G, Nlarge;
    int cap_pairs, cap_contacts, cap_bonds, cap_ends;
    int table_bits;             // grid hash table has 1 << table_bits buckets
    int multilevel;             // grid of NLEV levels (k_collision.cu); off-grid pairs by k_offgrid_pairs
    // bodies
    float4 *qn, *qa, *qb, *sq;  // 3 float4 per body each
    float4 *vel, *omg, *quat, *qstar;
    float4 *mass;               // (m, Pi_xx, Pi_yy, Pi_zz)
    float4 *he;                 // (hx, hy, hz, dhat)
    float4 *xs;                 // expansion point of the per-body system (x, y, z, 0), see sys_init
    int *bflags, *group, *group_off;
    int small_groups;           // every group has at most 128 bodies: one warp per group finalizes it
    // a group of more than RES_CHUNK bodies: its residual summed by chunks (k_resid_chunks),
    // (start, end) of each chunk, each group's first chunk, the chunks' sums; null otherwise
    int2 *res_chunk;
    int *res_coff;
    double *res_part;
    int n_res_chunks;
    int *large_ids;             // this step's bodies off the grid (C_NLARGE of them), or null
    int *adj_off, *adj_nbr;     // sorted partners joined by user bonds (no contact), or null
    double *resid_body, *resid_group;
    // bonds
    int4 *bmeta;
    float4 *bxi, *bxj, *bn;
    // augmented Lagrangian bonds: (kappa, lambda) for the sweep of parity k in al_st[k & 1],
    // parameters (kappa_start, beta, alpha, gamma); indexed by static bond id
    float2 *al_st0, *al_st1;
    float4 *al_par;
    int Nal;
    float4 *drv;                // 3 float4 per drive: (x_i0, arm) (r, amp) (u x r, 0); period/phase in drv_t
    float2 *drv_t;              // (period, phase)
    int *drv_bond;              // bond index of each drive
    // CSR of bond ends
    int *end_cnt, *end_cur, *end_off, *end_id, *end_pos;
    float4 *ends, *end_x;
    int *heavy;                 // ids of the bodies with more than HEAVY_ENDS ends (C_NHEAVY of them)
    // scenes whose only contacts are with the ground: each body's live static bond ends, sorted
    // by end id (2 bond + side), fixed at creation -- the CSR is these plus the step's ground
    // contacts (k_csr_ground); null otherwise
    int *sta_off, *sta_id;
    int *sta_body;              // the body of each entry of sta_id
    // ground contacts of the bodies before b in the fused front of a ground-only scene: the
    // prefix inside b's block of 256 bodies, the blocks' totals and their exclusive scan
    int *gnd_loc, *gnd_blk, *gnd_bof;
    int light_sorted;           // 1: the sweeps take the light bodies in Dev::order; 0: in body order
    int *order;                 // this step's light bodies by (class, end count), C_NLIGHT of them
    int *bin_cnt, *bin_cur;     // per bin of the light order: bodies, and the blocks' reservations
    // bond-end records in CSR order for the fused sweep: (i, j, type, bond), x_i (+w0), x_j (+p1)
    int4 *rec_m;
    float4 *rec_a, *rec_b;
    unsigned *gbar;             // grid barrier: arrival counter, generation
    unsigned *wait_limit;       // polls before a device-side wait gives up (PABD_ERR_TIMEOUT)
    // collision
    float4 *lo, *hi;            // inflated AABB; lo.w = inflation
    int4 *cell;                 // cell coords (.w = bucket)
    int *bucket_cnt, *bucket_cur, *bucket_off, *bucket_items;
    float4 *brec_lo, *brec_hi;  // per bucket slot: (lo, body id bits), (hi, group bits)
    int4 *brec_cell;            // per bucket slot: (cell x, y, z, flags)
    int *lane_cnt;              // per body x 32 lanes: partners found by each lane
    // per body x 32 lanes: the first PAIR_STASH partners each lane found while counting (a
    // partner delivered to a smaller id tagged by STASH_DELIVER), and the lane's number of
    // entries, so that writing the pairs replays them instead of scanning the cells again (a
    // lane with more rescans); null where the pair kernels run without them
    int *pair_stash, *lane_tot;
    int *pair_cnt, *pair_off;
    int2 *pairs;
    int *npc, *npc_off, *gnd_cnt, *gnd_off;
    // linear BVH broad phase (Params::broadphase == 1)
    unsigned *bvh_key, *bvh_key2;   // Morton codes (radix sort ping-pong)
    int *bvh_id, *bvh_id2;          // body ids in Morton order
    int *rx_cnt, *rx_off;           // radix sort: counts per (digit, tile) and their prefix sums
    int2 *bvh_kids;                 // children of the internal nodes (leaf k is node N - 1 + k)
    int *bvh_parent;                // parent of every node (-1 at the root)
    float4 *bvh_lo, *bvh_hi;        // boxes of the internal nodes
    int *bvh_visit;                 // refit arrivals per internal node
    int *bvh_bounds;                // box of the centres (order-preserving int bits: min xyz, max xyz)
    int *pair_j, *pair_tmp;         // partner slices while they are sorted
    int *pair_heavy;                // bodies with more than 64 partners
    // multilevel grid (Dev::multilevel)
    int *blevel;                    // grid level of each body this step (-1: off the grid)
    int *pair_own, *pair_cur;       // partners a body finds itself; cursor of those delivered to it
    // misc
    int *ctr;                   // Counter array
    // sweeps under a residual threshold: (sweeps done, scenes still active, loop on, -) and
    // the scenes that have stopped
    int *sweep_ctl;
    unsigned char *group_done;
    // groups held still by the host this step (pabd_set_group_hold): their bodies keep q, v, omega
    // and Q, as if pinned for the step
    unsigned char *group_hold;
    long long *step_index;
    int *scan_scratch;          // block sums of the scans
};

// body b's group is held still this step (pabd_set_group_hold)
__device__ __forceinline__ bool held(const Dev& d, int b) { return d.group_hold[d.group[b]] != 0; }

// ---- programmatic dependent launch ----
// A kernel launched by launch_pdl may be launched while its predecessor on the stream is still
// finishing: every kernel of the step calls pdl_enter(), which waits until its predecessor
// has completed and its writes are visible (a no-op for a launch without the attribute), before
// it reads anything that the predecessor may write.  Only the light loop of the sweep launches
// signals its successor before it exits (pdl_signal, once a warp has no work left): a signal
// at a kernel's start let waiting blocks of the successor take SM slots and made the step
// slower.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
// The calling thread has no work left that the successor's blocks could delay: once every
// thread of every block has signalled (or exited), the successor's grid may be launched.  Its
// blocks then take the SM slots this grid frees and load what does not depend on this grid
// (the bond launch's static part) while its last blocks finish; they still wait in pdl_enter
// for its completion before reading its results.
__device__ __forceinline__ void pdl_signal() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Grid of a kernel that strides over a device-counted range sized for `cap` items: one
// block per BLOCK items, at most GS_BLOCKS blocks (enough to fill every SM), so that a large
// capacity with few live items does not dispatch thousands of idle blocks.
constexpr int GS_BLOCKS = 152 * 8;
inline int stride_grid(long long cap, int block) {
    const long long b = (cap + block - 1) / block;
    return (int)(b < 1 ? 1 : (b > GS_BLOCKS ? GS_BLOCKS : b));
}

// blocks of a kernel with `per_sm` resident blocks per SM that fit on the current device at once
inline int resident_slots(int per_sm) {
    static const int sms = [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
        return n;
    }();
    return per_sm * sms;
}

template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
}

// ---- launchers (all asynchronous on `st`) ----
// scan: out[0..n] exclusive prefix sums of in[0..n-1], n read from *n_dev (or n_cap if
// n_dev is null), out[n] = total; grid sized for n_cap.
void scan_exclusive(const int* in, int* out, const int* n_dev, int n_cap, int* scratch, cudaStream_t st,
                    long long* launches);
int scan_scratch_ints(int n_cap);

// zeroes the step's counters and accumulation scratch; precedes launch_collision / launch_csr
void launch_step_reset(const Dev& d, cudaStream_t st, long long* launches);
void launch_collision(const Dev& d, cudaStream_t st, long long* launches);
// the front of a step in a ground-only scene: collision, CSR and predictor (k_collision.cu)
void launch_ground_front(const Dev& d, cudaStream_t st, long long* launches);
// LBVH pairs from this step's boxes (after k_aabb): the same output as the grid's pair stage
void launch_lbvh_pairs(const Dev& d, cudaStream_t st, long long* launches);
cudaError_t setup_pair_sort();
// each body's partner slice of Dev::pair_j sorted ascending into Dev::pairs
void launch_pair_sort(const Dev& d, cudaStream_t st, long long* launches);
void launch_broadphase(const Dev& d, cudaStream_t st, long long* launches);
void launch_csr(const Dev& d, cudaStream_t st, long long* launches);
// the light bodies ordered by (class, end count) into Dev::order (after launch_csr)
void launch_light_order(const Dev& d, cudaStream_t st, long long* launches);
// opt the CSR block sort into its 128 KB of dynamic shared memory (once per process and device)
cudaError_t setup_csr_kernels();
void launch_predict(const Dev& d, cudaStream_t st, long long* launches);
void launch_bond(const Dev& d, const float4* q, int it, cudaStream_t st, long long* launches);
// augmented Lagrangian: warm start (before the sweeps) and the update after the last sweep
void launch_al_warm(const Dev& d, cudaStream_t st, long long* launches);
void launch_al_final(const Dev& d, const float4* q, cudaStream_t st, long long* launches);
void launch_solve(const Dev& d, const float4* q_in, float4* q_out, int it, int lanes, cudaStream_t st,
                  long long* launches);
void launch_finalize(const Dev& d, const float4* q_fin, cudaStream_t st, long long* launches);
// sweeps under a residual threshold (Dev::sweep_ctl): the loop's start, one sweep's residual
// check and loop control (sets the conditional node's value when `handle` is non-zero), and
// the finalize that reads the last iterate from the buffer of the sweep count's parity
void launch_sweep_ctl_init(const Dev& d, cudaStream_t st, long long* launches);
void launch_sweep_check(const Dev& d, unsigned long long handle, cudaStream_t st, long long* launches);
void launch_finalize_dynamic(const Dev& d, cudaStream_t st, long long* launches);
void launch_drive_update(const Dev& d, cudaStream_t st, long long* launches);
// fused persistent sweep (all n_iter iterations, cooperative launch); L lanes per body
cudaError_t launch_fused_sweep(const Dev& d, int L, int block, int grid, cudaStream_t st, long long* launches);
int fused_max_blocks(int L, int block, bool fp64);
// one launch per sweep (bonds evaluated by the solve from CSR-ordered end records)
void launch_end_records(const Dev& d, cudaStream_t st, long long* launches);
void launch_sweep_one(const Dev& d, const float4* qi, float4* qo, int it, int L, cudaStream_t st,
                      long long* launches, bool pdl = false);


}  // namespace pabd
