// Collision detection (Alg. 1, first line) on the device.
//
// Broad phase: uniform grid hash.  Every body's inflated AABB is computed in IEEE single
// precision with a fixed operation order.  The cell size is the widest grid box of the step
// (times 1.01), so two overlapping grid boxes always sit in the same or in adjacent cells.
// A scene caps it at creation (grid_cell_cap: the widest box at rest, or below it when a few
// much wider boxes make that cheaper): a body whose inflated box is wider than the cap this
// step -- one flagged larger than the scene's `large_he`, or one moving fast -- goes off the
// grid and is tested against all bodies instead of widening every cell.  Scenes with such
// bodies by design use a multilevel grid instead (below), where a fast body moves up a level
// rather than off the grid.  Bodies are counting-sorted into hash buckets; each body scans
// the 27 cells around its own and keeps the neighbours j > i whose boxes overlap, whose cell
// really is the visited one (so hash collisions never duplicate a pair), that share its group
// and are not joined to it by a user bond.  Each body's partner list is sorted, so the final
// list is the sorted set of overlapping pairs -- independent of bucket order.
//
// Narrow phase: box-box contact manifold (reference face by separating axis over the six
// face normals, incident face clipped against the reference face's side planes) and
// corner-vs-ground-plane contacts, all in single precision with the same fixed operation
// order as the specification in the tests' oracle; contacts are written in pair order
// (then ground, in body order) through prefix sums, so the contact list is deterministic.
//
// All arithmetic here that decides an integer (overlap, inside, face) uses __fmul_rn /
// __fadd_rn / __fsub_rn so that no multiply-add is contracted into an FMA.
#include "pair_filter.cuh"
#include "sort_slices.cuh"
#include "predict.cuh"

namespace pabd {

#define FM(a, b) __fmul_rn((a), (b))
#define FA(a, b) __fadd_rn((a), (b))
#define FS(a, b) __fsub_rn((a), (b))

constexpr int CT = 256;  // threads per block for per-body / per-pair kernels
constexpr int NLEV = 3;           // levels of the multilevel grid
constexpr float LEV_RATIO = 4.f;  // cap ratio of consecutive levels

struct FBox {
    float c[3], A[9], he[3], infl;
};

__device__ __forceinline__ void load_q(const float4* q, int b, float* c, float* A) {
    float4 a = q[3 * b], bb = q[3 * b + 1], cc = q[3 * b + 2];
    c[0] = a.x; c[1] = a.y; c[2] = a.z;
    A[0] = a.w; A[1] = bb.x; A[2] = bb.y; A[3] = bb.z; A[4] = bb.w;
    A[5] = cc.x; A[6] = cc.y; A[7] = cc.z; A[8] = cc.w;
}

__device__ __forceinline__ void load_box(const Dev& d, int b, FBox& f) {
    load_q(d.qn, b, f.c, f.A);
    float4 h = d.he[b];
    f.he[0] = h.x; f.he[1] = h.y; f.he[2] = h.z;
    f.infl = d.lo[b].w;
}

// inflation of one body: (dhat + h*|v|) + margin, dhat = d_hat_rel * (2 * min he)
__device__ __forceinline__ float body_infl(const Dev& d, int b) {
    float4 h = d.he[b];
    float4 v = d.vel[b];
    float dh = FM(d.p.d_hat_rel, FM(2.0f, fminf(fminf(h.x, h.y), h.z)));
    float sp = __fsqrt_rn(FA(FA(FM(v.x, v.x), FM(v.y, v.y)), FM(v.z, v.z)));
    return FA(FA(dh, FM(d.p.h, sp)), d.p.margin);
}

// One body's AABB, inflation and grid level (one thread per body, b = the thread's global
// index, the threads at and above N already returned: the per-warp maximum below relies on it).
__device__ __forceinline__ void aabb_body(const Dev& d, int b) {
    float c[3], A[9];
    load_q(d.qn, b, c, A);
    float4 h = d.he[b];
    float infl = body_infl(d, b);
    float lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float e = FA(FA(FA(FM(fabsf(A[3 * k]), h.x), FM(fabsf(A[3 * k + 1]), h.y)), FM(fabsf(A[3 * k + 2]), h.z)), infl);
        lo[k] = FS(c[k], e);
        hi[k] = FA(c[k], e);
    }
    d.lo[b] = make_float4(lo[0], lo[1], lo[2], infl);
    d.hi[b] = make_float4(hi[0], hi[1], hi[2], 0.f);
    // off the grid: flagged large, or (with a fixed cell size) a box wider than a cell -- a fast
    // body whose inflation grew its box -- or a box that is not finite
    // The cell is the widest grid box of this step (times 1.01); with a scene cap p.cell, a box
    // wider than the cap leaves the grid instead of widening every cell.
    const float w = fmaxf(fmaxf(FS(hi[0], lo[0]), FS(hi[1], lo[1])), FS(hi[2], lo[2]));
    bool large = d.bflags[b] & BF_LARGE;
    int lv = 0;
    if (d.p.cell > 0.f) {
        if (d.multilevel) {  // the first level whose cap (cell cap x 4^level) holds the box
            float cap = d.p.cell;
            while (lv < NLEV - 1 && !(w <= cap)) { cap *= LEV_RATIO; ++lv; }
            large = large || !(w <= cap);
        } else {
            large = large || !(w <= d.p.cell);
        }
    }
    // the widest box of each level (positive floats order as ints): a warp's maximum first, then
    // one atomic per warp and level -- one per body on a single word serialises in L2
    const float wc = w * 1.01f + 1e-6f;
    const int bits = (!large && wc < 1e30f) ? __float_as_int(wc) : 0;
    const int wbase = b - (int)(threadIdx.x & 31);  // the warp's lanes below N (those above returned)
    const unsigned act = d.N - wbase >= 32 ? 0xffffffffu : ((1u << (d.N - wbase)) - 1u);
    const bool leader = (threadIdx.x & 31) == 0;
    for (int l = 0; l < (d.multilevel ? NLEV : 1); ++l) {
        const int m = __reduce_max_sync(act, lv == l ? bits : 0);
        if (leader && m > 0) atomicMax(&d.ctr[l == 0 ? C_CELLBITS : C_CELLBITS1 + l - 1], m);
    }
    d.cell[b] = make_int4(0, 0, 0, large ? -1 : 0);
    if (d.blevel) d.blevel[b] = large ? -1 : lv;
    if (large && d.large_ids) d.large_ids[atomicAdd(&d.ctr[C_NLARGE], 1)] = b;
}

__global__ void k_aabb(Dev d) {
    pdl_enter();
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.N) return;
    aabb_body(d, b);
}

__device__ __forceinline__ int cell_coord(float x, float inv_cs) {
    float t = floorf(x * inv_cs);
    t = fminf(fmaxf(t, -1048576.f), 1048576.f);
    return (int)t;
}

__device__ __forceinline__ int cell_hash(int x, int y, int z, int bits) {
    unsigned h = (unsigned)x * 73856093u ^ (unsigned)y * 19349663u ^ (unsigned)z * 83492791u;
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    return (int)(h & ((1u << bits) - 1u));
}

// Cell size of grid level lv: the widest box of that level or any finer one (times 1.01), so
// that a box of one level and a box of a coarser level that overlap sit in the same or in
// adjacent cells of the coarser level.
__device__ __forceinline__ float level_cell(const Dev& d, int lv) {
    float cs = __int_as_float(d.ctr[C_CELLBITS]);
    if (lv >= 1) cs = fmaxf(cs, __int_as_float(d.ctr[C_CELLBITS1]));
    if (lv >= 2) cs = fmaxf(cs, __int_as_float(d.ctr[C_CELLBITS2]));
    return cs;
}

// bucket of cell (x, y, z) of level lv (levels apart: coordinates stay within +-2^20)
__device__ __forceinline__ int level_hash(int x, int y, int z, int lv, int bits) {
    return cell_hash(x + (lv << 22), y, z, bits);
}

__global__ void k_cells(Dev d) {
    pdl_enter();
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.N) return;
    if (d.cell[b].w < 0) return;  // off the grid (k_aabb)
    const int lv = d.blevel ? d.blevel[b] : 0;
    const float cs = level_cell(d, lv);
    float inv = 1.0f / cs;
    float4 a = d.qn[3 * b];
    int x = cell_coord(a.x, inv), y = cell_coord(a.y, inv), z = cell_coord(a.z, inv);
    int hb = level_hash(x, y, z, lv, d.table_bits);
    d.cell[b] = make_int4(x, y, z, hb);
    atomicAdd(&d.bucket_cnt[hb], 1);
}

// Bodies into their buckets, with a compact copy of what the pair test reads (box, id, group,
// flags, cell) so that a candidate costs one contiguous record read.
__global__ void k_bucket_fill(Dev d) {
    pdl_enter();
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.N) return;
    const int4 c = d.cell[b];
    if (c.w < 0) return;
    const int pos = d.bucket_off[c.w] + atomicAdd(&d.bucket_cur[c.w], 1);
    d.bucket_items[pos] = b;
    if (d.brec_lo) {
        const float4 lo = d.lo[b], hi = d.hi[b];
        d.brec_lo[pos] = make_float4(lo.x, lo.y, lo.z, __int_as_float(b));
        d.brec_hi[pos] = make_float4(hi.x, hi.y, hi.z, __int_as_float(d.group[b]));
        d.brec_cell[pos] = make_int4(c.x, c.y, c.z, d.bflags[b] | ((d.blevel ? d.blevel[b] : 0) << 8));
    }
}

// Pair finding, one warp per body i.  A grid body: lane c < 27 scans neighbour cell c
// (dx, dy, dz = c % 3 - 1, c / 3 % 3 - 1, c / 9 - 1), then the lanes stride over the large
// bodies; the partners are written at per-lane offsets and the body's slice is sorted.  A
// large body: the warp sweeps j = i+1 .. N-1 in chunks of 32 and compacts with a ballot,
// which keeps j ascending.  Accepted partners: j > i, same group, not both pinned, inflated
// boxes overlap, not joined by a user bond.
template <class F>
__device__ __forceinline__ int lane_partners(const Dev& d, int i, int lane, F&& f) {
    const int gi = d.group[i], fi = d.bflags[i];
    int n = 0;
    if (lane < 27) {
        const int4 ci = d.cell[i];
        const int x = ci.x + lane % 3 - 1, y = ci.y + (lane / 3) % 3 - 1, z = ci.z + lane / 9 - 1;
        const int hb = cell_hash(x, y, z, d.table_bits);
        const int s = d.bucket_off[hb], e = d.bucket_off[hb + 1];
        if (d.brec_lo) {
            const float4 li = d.lo[i], hi_ = d.hi[i];
            for (int k = s; k < e; ++k) {
                const int4 cj = d.brec_cell[k];
                const float4 lj = d.brec_lo[k], hj = d.brec_hi[k];
                const int j = __float_as_int(lj.w);
                if (j <= i || cj.x != x || cj.y != y || cj.z != z) continue;
                if (__float_as_int(hj.w) != gi || ((fi & BF_PINNED) && (cj.w & BF_PINNED))) continue;
                if (!overlap(li, hi_, lj, hj)) continue;
                if (adj_has(d, i, j)) continue;
                f(j, n);
                ++n;
            }
        } else {
            for (int k = s; k < e; ++k) {
                const int j = d.bucket_items[k];
                if (j <= i) continue;
                const int4 cj = d.cell[j];
                if (cj.x != x || cj.y != y || cj.z != z) continue;
                if (pair_ok(d, i, j, gi, fi)) { f(j, n); ++n; }
            }
        }
    }
    const int nl = d.large_ids ? d.ctr[C_NLARGE] : 0;
    if (nl > 0) {
        const float4 li = d.lo[i], hi_ = d.hi[i];
        for (int k = lane; k < nl; k += 32) {
            const int j = d.large_ids[k];
            if (j > i && pair_ok(d, i, j, gi, fi, li, hi_)) { f(j, n); ++n; }
        }
    }
    return n;
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_excl(int v, int lane) {
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    return inc - v;
}

__global__ void k_pair_count(Dev d) {
    pdl_enter();
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= d.N) return;
    int n = 0;
    if (d.p.body_contacts) {
        const int gi = d.group[i], fi = d.bflags[i];
        if (d.cell[i].w < 0) {
            const float4 li = d.lo[i], hi_ = d.hi[i];
            for (int j0 = i + 1; j0 < d.N; j0 += 32) {
                const int j = j0 + lane;
                n += (j < d.N && pair_ok(d, i, j, gi, fi, li, hi_)) ? 1 : 0;
            }
        } else {
            int* st = d.pair_stash ? d.pair_stash + (size_t)(32 * i + lane) * PAIR_STASH : nullptr;
            n = lane_partners(d, i, lane, [&](int j, int k) { if (st && k < PAIR_STASH) st[k] = j; });
        }
    }
    if (d.lane_cnt) d.lane_cnt[32 * i + lane] = n;
    n = warp_sum(n);
    if (lane == 0) d.pair_cnt[i] = n;
}

__global__ void k_pair_write(Dev d) {
    pdl_enter();
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= d.N) return;
    const int s = d.pair_off[i];
    const int cap = d.cap_pairs;
    if (d.p.body_contacts) {
        const int gi = d.group[i], fi = d.bflags[i];
        if (d.cell[i].w < 0) {
            int pos = s;
            const float4 li = d.lo[i], hi_ = d.hi[i];
            for (int j0 = i + 1; j0 < d.N; j0 += 32) {
                const int j = j0 + lane;
                const bool ok = j < d.N && pair_ok(d, i, j, gi, fi, li, hi_);
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                const int at = pos + __popc(bal & ((1u << lane) - 1u));
                if (ok && at < cap) d.pairs[at] = make_int2(i, j);
                pos += __popc(bal);
            }
        } else {
            const int mine = d.lane_cnt ? d.lane_cnt[32 * i + lane] : lane_partners(d, i, lane, [](int, int) {});
            const int base = s + warp_excl(mine, lane);
            if (d.pair_stash && d.lane_cnt && mine <= PAIR_STASH) {  // the partners found while counting
                const int* st = d.pair_stash + (size_t)(32 * i + lane) * PAIR_STASH;
                for (int k = 0; k < mine; ++k)
                    if (base + k < cap) d.pairs[base + k] = make_int2(i, st[k]);
            } else {
                lane_partners(d, i, lane, [&](int j, int k) {
                    if (base + k < cap) d.pairs[base + k] = make_int2(i, j);
                });
            }
            __syncwarp();
            const int e = min(d.pair_off[i + 1], cap);
            if (e - s <= 32) {  // the slice sorted by j: each partner's rank among the slice
                const int n = e - s;
                const int j = lane < n ? d.pairs[s + lane].y : 0x7fffffff;
                const int r = warp_rank32(j, n, lane);
                __syncwarp();
                if (r >= 0) d.pairs[s + r] = make_int2(i, j);
            } else if (e - s <= 64) {  // by the bitonic network in registers
                const int n = e - s;
                int v0 = (2 * lane < n) ? d.pairs[s + 2 * lane].y : 0x7fffffff;
                int v1 = (2 * lane + 1 < n) ? d.pairs[s + 2 * lane + 1].y : 0x7fffffff;
                warp_sort64(v0, v1, lane);
                if (2 * lane < n) d.pairs[s + 2 * lane] = make_int2(i, v0);
                if (2 * lane + 1 < n) d.pairs[s + 2 * lane + 1] = make_int2(i, v1);
            } else if (lane == 0) {
                for (int a = s + 1; a < e; ++a) {  // insertion sort of the slice by j
                    int2 v = d.pairs[a];
                    int b = a - 1;
                    while (b >= s && d.pairs[b].y > v.y) { d.pairs[b + 1] = d.pairs[b]; --b; }
                    d.pairs[b + 1] = v;
                }
            }
        }
    }
    if (i == d.N - 1 && lane == 0) {
        int tot = d.pair_off[d.N];
        if (tot > cap) atomicOr(&d.ctr[C_STATUS], ST_CAPACITY);
        d.ctr[C_NPAIRS] = min(tot, cap);
    }
}

// ---- multilevel grid (Dev::multilevel: scenes with bodies of very different widths) ----
//
// A grid body sits at the first level l whose cap, cell cap x 4^l, holds its box (NLEV
// levels); a wider one, or one flagged large, goes off the grid.  Level l's cell is the widest
// box of that level or a finer one, so a body meets every overlapping body of its own or a
// coarser level in the 27 cells around its centre at that level.  Each body therefore scans
// its own level (keeping partners j > i, as the single-level grid does) and every non-empty
// coarser level (keeping all partners): a partner j > i joins i's slice, a partner j < i is
// delivered to j's slice (counted, then placed, with atomics).  The off-grid bodies take all
// j > i by a block-parallel sweep (k_offgrid_pairs) and the grid bodies test the off-grid
// list for j > i.  Every slice is then sorted (launch_pair_sort), so the list is again the
// sorted set of overlapping pairs whatever the order of the atomics.

template <class Own, class Deliver>
__device__ __forceinline__ int lane_partners_ml(const Dev& d, int i, int lane, Own&& own, Deliver&& deliver) {
    const int gi = d.group[i], fi = d.bflags[i];
    const int lvi = d.blevel[i];
    const float4 li = d.lo[i], hi_ = d.hi[i];
    const int4 ci = d.cell[i];
    const float4 pos = d.qn[3 * i];
    // the levels to scan: its own, then each coarser one that holds any body
    unsigned lvmask = 1u << lvi;
    for (int l = lvi + 1; l < NLEV; ++l)
        if (d.ctr[C_CELLBITS1 + l - 1] != 0) lvmask |= 1u << l;
    const int nscan = 27 * __popc(lvmask);
    int n = 0;
    for (int t = lane; t < nscan; t += 32) {
        int rank = t / 27, l = 0;
        for (unsigned m = lvmask;; m &= m - 1) {  // the rank-th set bit
            if (rank-- == 0) { l = __ffs(m) - 1; break; }
        }
        int bx = ci.x, by = ci.y, bz = ci.z;
        if (l != lvi) {
            const float inv = 1.0f / level_cell(d, l);
            bx = cell_coord(pos.x, inv); by = cell_coord(pos.y, inv); bz = cell_coord(pos.z, inv);
        }
        const int c = t % 27;
        const int x = bx + c % 3 - 1, y = by + (c / 3) % 3 - 1, z = bz + c / 9 - 1;
        const int hb = level_hash(x, y, z, l, d.table_bits);
        const int s = d.bucket_off[hb], e = d.bucket_off[hb + 1];
        for (int k = s; k < e; ++k) {
            const int4 cj = d.brec_cell[k];
            const float4 lj = d.brec_lo[k], hj = d.brec_hi[k];
            const int j = __float_as_int(lj.w);
            if (cj.x != x || cj.y != y || cj.z != z || (cj.w >> 8) != l || j == i) continue;
            if (l == lvi && j < i) continue;  // same level: found by the smaller id
            if (__float_as_int(hj.w) != gi || ((fi & BF_PINNED) && (cj.w & BF_PINNED))) continue;
            if (!overlap(li, hi_, lj, hj)) continue;
            if (adj_has(d, i, j)) continue;
            if (j > i) { own(j, n); ++n; }
            else deliver(j);
        }
    }
    const int nl = d.ctr[C_NLARGE];
    for (int k = lane; k < nl; k += 32) {
        const int j = d.large_ids[k];
        if (j > i && pair_ok(d, i, j, gi, fi, li, hi_)) { own(j, n); ++n; }
    }
    return n;
}

// counts: pair_cnt (zeroed before) gains each body's own partners and the deliveries to it
__global__ void k_ml_pair_count(Dev d) {
    pdl_enter();
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= d.N || !d.p.body_contacts || d.cell[i].w < 0) return;
    int* st = d.pair_stash ? d.pair_stash + (size_t)(32 * i + lane) * PAIR_STASH : nullptr;
    int tot = 0;  // entries: own partners and deliveries, in the order found
    int n = lane_partners_ml(d, i, lane,
        [&](int j, int) { if (st && tot < PAIR_STASH) st[tot] = j; ++tot; },
        [&](int j) {
            atomicAdd(&d.pair_cnt[j], 1);
            if (st && tot < PAIR_STASH) st[tot] = j | STASH_DELIVER;
            ++tot;
        });
    d.lane_cnt[32 * i + lane] = n;
    if (d.lane_tot) d.lane_tot[32 * i + lane] = tot;
    n = warp_sum(n);
    if (lane == 0) {
        d.pair_own[i] = n;
        atomicAdd(&d.pair_cnt[i], n);
    }
}

// partner ids into pair_j: own partners at per-lane offsets, deliveries after the receiver's
// own ones through its cursor (pair_cur, zeroed before)
__global__ void k_ml_pair_write(Dev d) {
    pdl_enter();
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= d.N) return;
    const int cap = d.cap_pairs;
    if (d.p.body_contacts && d.cell[i].w >= 0) {
        const int base = d.pair_off[i] + warp_excl(d.lane_cnt[32 * i + lane], lane);
        auto own = [&](int j, int k) { if (base + k < cap) d.pair_j[base + k] = j; };
        auto deliver = [&](int j) {
            const int at = d.pair_off[j] + d.pair_own[j] + atomicAdd(&d.pair_cur[j], 1);
            if (at < cap) d.pair_j[at] = i;
        };
        const int tot = d.pair_stash && d.lane_tot ? d.lane_tot[32 * i + lane] : PAIR_STASH + 1;
        if (tot <= PAIR_STASH) {  // the entries found while counting
            const int* st = d.pair_stash + (size_t)(32 * i + lane) * PAIR_STASH;
            int k = 0;
            for (int t = 0; t < tot; ++t) {
                const int v = st[t];
                if (v & STASH_DELIVER) deliver(v & ~STASH_DELIVER);
                else own(v, k++);
            }
        } else {
            lane_partners_ml(d, i, lane, own, deliver);
        }
    }
    if (i == d.N - 1 && lane == 0) {
        const int tot = d.pair_off[d.N];
        if (tot > cap) atomicOr(&d.ctr[C_STATUS], ST_CAPACITY);
        d.ctr[C_NPAIRS] = min(tot, cap);
    }
}

// Pairs of the off-grid bodies: body i of the off-grid list against every j > i, one block of
// OFF_T threads per body.  Warp w takes the w-th of 32 contiguous runs of (i, N), so the warps'
// hits concatenated in warp order keep the slice sorted by j; the runs' loads are
// independent, so a body's sweep costs about N / OFF_T dependent rounds instead of N / 32.
// WRITE = false counts (into pair_cnt[i], and each warp's count in lane_cnt[32 i + w]); true
// stores the partners into pair_j.
constexpr int OFF_T = 1024;
constexpr int OFF_BLOCKS = 152;

template <bool WRITE>
__global__ void __launch_bounds__(OFF_T) k_offgrid_pairs(Dev d) {
    pdl_enter();
    __shared__ int s_cnt[OFF_T / 32];
    if (!d.p.body_contacts) return;
    const int nl = d.ctr[C_NLARGE];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cap = d.cap_pairs;
    for (int h = blockIdx.x; h < nl; h += gridDim.x) {
        const int i = d.large_ids[h];
        const int gi = d.group[i], fi = d.bflags[i];
        const float4 li = d.lo[i], hi_ = d.hi[i];
        const int len = (((d.N - i - 1) + 31) / 32 + 31) & ~31;  // per warp, a multiple of 32
        const int j_beg = i + 1 + w * len, j_end = min(d.N, j_beg + len);
        if (!WRITE) {
            int n = 0;
            for (int j0 = j_beg; j0 < j_end; j0 += 32) {
                const int j = j0 + lane;
                n += (j < j_end && pair_ok(d, i, j, gi, fi, li, hi_)) ? 1 : 0;
            }
            n = warp_sum(n);
            if (lane == 0) { d.lane_cnt[32 * i + w] = n; s_cnt[w] = n; }
            __syncthreads();
            if (threadIdx.x == 0) {
                int t = 0;
                for (int k = 0; k < OFF_T / 32; ++k) t += s_cnt[k];
                atomicAdd(&d.pair_cnt[i], t);
            }
            __syncthreads();
        } else {
            int pos = d.pair_off[i];
            for (int k = 0; k < w; ++k) pos += d.lane_cnt[32 * i + k];
            for (int j0 = j_beg; j0 < j_end; j0 += 32) {
                const int j = j0 + lane;
                const bool ok = j < j_end && pair_ok(d, i, j, gi, fi, li, hi_);
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                const int at = pos + __popc(bal & ((1u << lane) - 1u));
                if (ok && at < cap) d.pair_j[at] = j;
                pos += __popc(bal);
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// narrow phase
// ------------------------------------------------------------------------------------

struct CPt {
    float u[3], x[3];
};

__device__ __forceinline__ float dot_col(const float* A, int l, const float* r) {
    return FA(FA(FM(A[l], r[0]), FM(A[3 + l], r[1])), FM(A[6 + l], r[2]));
}

// Manifold of the pair (a, b); calls emit(i, j, x_i, x_j, N) for each contact, returns count.
template <class Emit>
__device__ int box_box(const FBox& fa, const FBox& fb, int a, int b, Emit&& emit) {
    const float delta = FA(fa.infl, fb.infl);
    float dv[3], dab[3], dba[3], R[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) dv[k] = FS(fa.c[k], fb.c[k]);
#pragma unroll
    for (int l = 0; l < 3; ++l) dab[l] = dot_col(fb.A, l, dv);
    float dn[3] = {-dv[0], -dv[1], -dv[2]};
#pragma unroll
    for (int k = 0; k < 3; ++k) dba[k] = dot_col(fa.A, k, dn);
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            R[3 * l + k] = FA(FA(FM(fb.A[l], fa.A[k]), FM(fb.A[3 + l], fa.A[3 + k])), FM(fb.A[6 + l], fa.A[6 + k]));
    float best = 0.f;
    int ref_b = 1, l = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float ext = FA(FA(FM(fabsf(R[3 * ax]), fa.he[0]), FM(fabsf(R[3 * ax + 1]), fa.he[1])), FM(fabsf(R[3 * ax + 2]), fa.he[2]));
        float sep = FS(fabsf(dab[ax]), FA(fb.he[ax], ext));
        if (ax == 0 || sep > best) { best = sep; ref_b = 1; l = ax; }
    }
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float ext = FA(FA(FM(fabsf(R[ax]), fb.he[0]), FM(fabsf(R[3 + ax]), fb.he[1])), FM(fabsf(R[6 + ax]), fb.he[2]));
        float sep = FS(fabsf(dba[ax]), FA(fa.he[ax], ext));
        if (sep > best) { best = sep; ref_b = 0; l = ax; }
    }
    if (!(best <= delta)) return 0;
    const FBox& fr = ref_b ? fb : fa;
    const FBox& fi = ref_b ? fa : fb;
    const int ir = ref_b ? b : a, ii = ref_b ? a : b;
    const float sg = ref_b ? (dab[l] >= 0.f ? 1.f : -1.f) : (dba[l] >= 0.f ? 1.f : -1.f);
    float N[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) N[k] = FM(sg, fr.A[3 * k + l]);
    int ki = 0;
    float bestd = 0.f, dsel = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float dk = dot_col(fi.A, k, N);
        if (k == 0 || fabsf(dk) > bestd) { bestd = fabsf(dk); ki = k; dsel = dk; }
    }
    const float si = dsel > 0.f ? -1.f : 1.f;
    const int k1 = (ki + 1) % 3, k2 = (ki + 2) % 3;
    const float sgn1[4] = {1.f, -1.f, -1.f, 1.f}, sgn2[4] = {1.f, 1.f, -1.f, -1.f};
    CPt poly[8], tmp[8];
    int np = 4;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        float x[3], y[3], r[3];
        x[ki] = FM(si, fi.he[ki]);
        x[k1] = FM(sgn1[v], fi.he[k1]);
        x[k2] = FM(sgn2[v], fi.he[k2]);
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
            y[dd] = FA(FA(FA(fi.c[dd], FM(fi.A[3 * dd], x[0])), FM(fi.A[3 * dd + 1], x[1])), FM(fi.A[3 * dd + 2], x[2]));
            r[dd] = FS(y[dd], fr.c[dd]);
        }
#pragma unroll
        for (int m = 0; m < 3; ++m) { poly[v].u[m] = dot_col(fr.A, m, r); poly[v].x[m] = x[m]; }
    }
    const int m1 = (l + 1) % 3, m2 = (l + 2) % 3;
    for (int pl = 0; pl < 4 && np > 0; ++pl) {
        const int m = pl < 2 ? m1 : m2;
        const float ps = (pl & 1) ? -1.f : 1.f, lim = fr.he[m];
        int nt = 0;
        for (int v = 0; v < np; ++v) {
            const CPt& P = poly[v];
            const CPt& Q = poly[(v + 1) % np];
            float dp = FS(FM(ps, P.u[m]), lim), dq = FS(FM(ps, Q.u[m]), lim);
            bool pin = dp <= 0.f, qin = dq <= 0.f;
            if (pin) tmp[nt++] = P;
            if (pin != qin) {
                float t = __fdiv_rn(dp, FS(dp, dq));
                CPt X;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    X.u[c] = FA(P.u[c], FM(t, FS(Q.u[c], P.u[c])));
                    X.x[c] = FA(P.x[c], FM(t, FS(Q.x[c], P.x[c])));
                }
                tmp[nt++] = X;
            }
        }
        np = nt;
        for (int v = 0; v < nt; ++v) poly[v] = tmp[v];
    }
    int cnt = 0;
    for (int v = 0; v < np; ++v) {
        float hgt = FS(FM(sg, poly[v].u[l]), fr.he[l]);
        if (!(hgt < delta)) continue;
        float xj[3] = {poly[v].u[0], poly[v].u[1], poly[v].u[2]};
        xj[l] = FM(sg, fr.he[l]);
        emit(ii, ir, poly[v].x, xj, N, cnt);
        ++cnt;
    }
    return cnt;
}

template <class Emit>
__device__ int ground_corners(const Dev& d, const FBox& fa, int a, Emit&& emit) {
    int cnt = 0;
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        float x[3] = {(k & 1) ? fa.he[0] : -fa.he[0], (k & 2) ? fa.he[1] : -fa.he[1], (k & 4) ? fa.he[2] : -fa.he[2]};
        float y[3];
#pragma unroll
        for (int dd = 0; dd < 3; ++dd)
            y[dd] = FA(FA(FA(fa.c[dd], FM(fa.A[3 * dd], x[0])), FM(fa.A[3 * dd + 1], x[1])), FM(fa.A[3 * dd + 2], x[2]));
        float g = FS(FA(FA(FM(d.p.gn[0], y[0]), FM(d.p.gn[1], y[1])), FM(d.p.gn[2], y[2])), d.p.gd);
        if (!(g < fa.infl)) continue;
        float anc[3] = {FS(y[0], FM(g, d.p.gn[0])), FS(y[1], FM(g, d.p.gn[1])), FS(y[2], FM(g, d.p.gn[2]))};
        emit(a, -1, x, anc, d.p.gn, cnt);
        ++cnt;
    }
    return cnt;
}

// Items [0, np) are this step's pairs, items np + b the ground corners of body b (apart, so
// that no item runs both manifolds in series); the threads stride over them.
__global__ void k_narrow_count(Dev d) {
    pdl_enter();
    const int np = d.ctr[C_NPAIRS];
    const int items = np + d.N;
    for (int tt = blockIdx.x * blockDim.x + threadIdx.x; tt < items; tt += gridDim.x * blockDim.x) {
        if (tt < np) {
            int2 pr = d.pairs[tt];
            FBox fa, fb;
            load_box(d, pr.x, fa);
            load_box(d, pr.y, fb);
            d.npc[tt] = box_box(fa, fb, pr.x, pr.y, [](int, int, const float*, const float*, const float*, int) {});
        } else {
            const int t = tt - np;
            int n = 0;
            if (d.p.has_ground && !(d.bflags[t] & BF_PINNED)) {
                FBox fa;
                load_box(d, t, fa);
                n = ground_corners(d, fa, t, [](int, int, const float*, const float*, const float*, int) {});
            }
            d.gnd_cnt[t] = n;
        }
    }
}

__device__ __forceinline__ float pair_dhat(const Dev& d, int i, int j) {
    float di = d.he[i].w;
    return j < 0 ? di : fminf(di, d.he[j].w);
}

__device__ __forceinline__ void write_contact(const Dev& d, int slot, int type, int i, int j, const float* xi,
                                              const float* xj, const float* N) {
    if (slot >= d.cap_contacts) return;
    const int b = d.Nc + slot;
    float mi = d.mass[i].x;
    float mm;
    if (j < 0) mm = mi;
    else {
        float mj = d.mass[j].x;
        bool pi = d.bflags[i] & BF_PINNED, pj = d.bflags[j] & BF_PINNED;
        mm = pj ? mi : (pi ? mj : fminf(mi, mj));
    }
    d.bmeta[b] = make_int4(i, j, type, 0);
    d.bxi[b] = make_float4(xi[0], xi[1], xi[2], d.p.c_kappa * mm);
    d.bxj[b] = make_float4(xj[0], xj[1], xj[2], pair_dhat(d, i, j));
    d.bn[b] = make_float4(N[0], N[1], N[2], d.p.mu);
}

// (the items as in k_narrow_count)
__global__ void k_narrow_write(Dev d) {
    pdl_enter();
    const int np = d.ctr[C_NPAIRS];
    const int npc = d.npc_off[np];
    const int items = np + d.N;
    for (int tt = blockIdx.x * blockDim.x + threadIdx.x; tt < items; tt += gridDim.x * blockDim.x) {
        if (tt < np) {
            int2 pr = d.pairs[tt];
            FBox fa, fb;
            load_box(d, pr.x, fa);
            load_box(d, pr.y, fb);
            const int base = d.npc_off[tt];
            box_box(fa, fb, pr.x, pr.y, [&](int i, int j, const float* xi, const float* xj, const float* N, int k) {
                write_contact(d, base + k, K_CONTACT, i, j, xi, xj, N);
            });
        } else {
            const int t = tt - np;
            if (d.gnd_cnt[t] > 0) {
                FBox fa;
                load_box(d, t, fa);
                const int base = npc + d.gnd_off[t];
                ground_corners(d, fa, t, [&](int i, int j, const float* xi, const float* xj, const float* N, int k) {
                    write_contact(d, base + k, K_GROUND, i, j, xi, xj, N);
                });
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int nk = npc + d.gnd_off[d.N];
        if (nk > d.cap_contacts) { atomicOr(&d.ctr[C_STATUS], ST_CAPACITY); nk = d.cap_contacts; }
        d.ctr[C_NPC] = min(npc, d.cap_contacts);
        d.ctr[C_NGC] = nk - min(npc, d.cap_contacts);
        d.ctr[C_NBONDS] = d.Nc + nk;
    }
}

static inline int nblk(int n) { return (n + CT - 1) / CT > 0 ? (n + CT - 1) / CT : 1; }

// ---- the front of a step in scenes whose only contacts are with the ground ----
//
// Three launches in place of the AABB, ground-count, scan, contact-write, CSR and predictor
// kernels (the same arithmetic, fewer launch boundaries): k_ground_prelude per body, the scan of
// its blocks' totals, k_ground_bonds_csr per static end and per body.

// per body: AABB and inflation, ground contacts counted, predictor; per block of CT bodies, the
// exclusive prefix of the counts inside the block (Dev::gnd_loc) and their total (Dev::gnd_blk)
__global__ void __launch_bounds__(CT) k_ground_prelude(Dev d) {
    pdl_enter();
    __shared__ int wsum[CT / 32];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    int n = 0;
    if (b < d.N) {
        aabb_body(d, b);
        if (d.p.has_ground && !(d.bflags[b] & BF_PINNED)) {
            FBox fa;
            load_box(d, b, fa);
            n = ground_corners(d, fa, b, [](int, int, const float*, const float*, const float*, int) {});
        }
        d.gnd_cnt[b] = n;
        predict_body(d, b);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < CT / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < CT / 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < CT / 32) wsum[lane] = w;
    }
    __syncthreads();
    if (b < d.N) d.gnd_loc[b] = (warp ? wsum[warp - 1] : 0) + inc - n;
    if (threadIdx.x == 0) d.gnd_blk[blockIdx.x] = wsum[CT / 32 - 1];
}

// ground contacts of the bodies before b (b <= N), from the prelude's block prefixes and the
// scan of its block totals (Dev::gnd_bof, whose last entry is the total)
__device__ __forceinline__ int gnd_prefix(const Dev& d, int b) {
    return b < d.N ? d.gnd_bof[b / CT] + d.gnd_loc[b] : d.gnd_bof[(d.N + CT - 1) / CT];
}

// After the scan: items [0, Ns) are the static ends in Dev::sta_id order -- end e of body b
// takes slot e + g0(b), g0(b) = the ground contacts of the bodies before b (at most the
// contact capacity); items Ns + b, b <= N, the bodies -- slice start sta_off[b] + g0(b), the
// body's ground contacts written as bonds Nc + g0(b) + k and given slots after its static ends,
// and the heavy list.  The same CSR, in the same order, as counting, filling and sorting it.
__global__ void k_ground_bonds_csr(Dev d) {
    pdl_enter();
    const int nb = d.N, Ns = d.sta_off[nb], cap = d.cap_contacts;
    const int items = Ns + nb + 1;
    for (int tt = blockIdx.x * blockDim.x + threadIdx.x; tt < items; tt += gridDim.x * blockDim.x) {
        if (tt < Ns) {
            const int b = d.sta_body[tt];
            const int slot = tt + min(gnd_prefix(d, b), cap);
            const int id = d.sta_id[tt], bond = id >> 1;
            d.end_id[slot] = id;
            d.end_pos[id] = slot;
            const float4 x = (id & 1) ? d.bxj[bond] : d.bxi[bond];
            d.end_x[slot] = make_float4(x.x, x.y, x.z, 0.f);
            continue;
        }
        const int b = tt - Ns;
        const int gb = gnd_prefix(d, b), g0 = min(gb, cap);
        d.gnd_off[b] = gb;
        d.end_off[b] = d.sta_off[b] + g0;
        if (b == nb) continue;
        const int gn = min(gnd_prefix(d, b + 1), cap) - g0;
        if (gn > 0) {
            FBox fa;
            load_box(d, b, fa);
            const int p0 = d.sta_off[b + 1] + g0;
            ground_corners(d, fa, b, [&](int i, int j, const float* xi, const float* xj, const float* N, int k) {
                if (k >= gn) return;  // past the contact capacity (latched below)
                write_contact(d, g0 + k, K_GROUND, i, j, xi, xj, N);
                const int bond = d.Nc + g0 + k, p = p0 + k;
                d.end_id[p] = 2 * bond;
                d.end_pos[2 * bond] = p;
                d.end_x[p] = make_float4(xi[0], xi[1], xi[2], 0.f);
            });
        }
        if (d.sta_off[b + 1] - d.sta_off[b] + gn > HEAVY_ENDS) d.heavy[atomicAdd(&d.ctr[C_NHEAVY], 1)] = b;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int nk = gnd_prefix(d, nb);
        if (nk > cap) { atomicOr(&d.ctr[C_STATUS], ST_CAPACITY); nk = cap; }
        d.ctr[C_NPC] = 0;
        d.ctr[C_NGC] = nk;
        d.ctr[C_NBONDS] = d.Nc + nk;
    }
}

void launch_ground_front(const Dev& d, cudaStream_t st, long long* launches) {
    launch_pdl(k_ground_prelude, dim3(nblk(d.N)), dim3(CT), 0, st, d);
    scan_exclusive(d.gnd_blk, d.gnd_bof, nullptr, nblk(d.N), d.scan_scratch, st, launches);
    launch_pdl(k_ground_bonds_csr, dim3(stride_grid((long long)d.cap_ends + d.N + 1, CT)), dim3(CT), 0, st, d);
    *launches += 2;
}

// The broad phase alone (bucket / counter resets, AABBs, grid, sorted pair list), on whatever
// buffers `d` points at; used by the allocation-free entry point.
void launch_broadphase(const Dev& d, cudaStream_t st, long long* launches) {
    const int T = 1 << d.table_bits;
    cudaMemsetAsync(d.bucket_cnt, 0, sizeof(int) * T, st);
    cudaMemsetAsync(d.bucket_cur, 0, sizeof(int) * T, st);
    cudaMemsetAsync(d.ctr, 0, sizeof(int) * C_COUNT, st);
    launch_pdl(k_aabb, dim3(nblk(d.N)), dim3(CT), 0, st, d);
    launch_pdl(k_cells, dim3(nblk(d.N)), dim3(CT), 0, st, d);
    scan_exclusive(d.bucket_cnt, d.bucket_off, nullptr, T, d.scan_scratch, st, launches);
    launch_pdl(k_bucket_fill, dim3(nblk(d.N)), dim3(CT), 0, st, d);
    const int wblk = (d.N * 32 + CT - 1) / CT > 0 ? (d.N * 32 + CT - 1) / CT : 1;
    launch_pdl(k_pair_count, dim3(wblk), dim3(CT), 0, st, d);
    scan_exclusive(d.pair_cnt, d.pair_off, nullptr, d.N, d.scan_scratch, st, launches);
    launch_pdl(k_pair_write, dim3(wblk), dim3(CT), 0, st, d);
    *launches += 5;
}

// (the counters and buckets it accumulates into are zeroed by launch_step_reset)
void launch_collision(const Dev& d, cudaStream_t st, long long* launches) {
    launch_pdl(k_aabb, dim3(nblk(d.N)), dim3(CT), 0, st, d);
    *launches += 1;
    if (!d.p.body_contacts) {
        // ground contacts only: no broad phase (the pair count stays at the zero the step's
        // reset wrote, and the pair contacts' prefix at the zero written at creation)
        launch_pdl(k_narrow_count, dim3(stride_grid(d.N, CT)), dim3(CT), 0, st, d);
        scan_exclusive(d.gnd_cnt, d.gnd_off, nullptr, d.N, d.scan_scratch, st, launches);
        launch_pdl(k_narrow_write, dim3(stride_grid(d.N, CT)), dim3(CT), 0, st, d);
        *launches += 2;
        return;
    }
    if (d.p.broadphase == 1) {
        launch_lbvh_pairs(d, st, launches);
    } else {
        const int T = 1 << d.table_bits;
        launch_pdl(k_cells, dim3(nblk(d.N)), dim3(CT), 0, st, d);
        scan_exclusive(d.bucket_cnt, d.bucket_off, nullptr, T, d.scan_scratch, st, launches);
        launch_pdl(k_bucket_fill, dim3(nblk(d.N)), dim3(CT), 0, st, d);
        const int wblk = (d.N * 32 + CT - 1) / CT > 0 ? (d.N * 32 + CT - 1) / CT : 1;  // one warp per body
        if (d.multilevel) {
            launch_pdl(k_ml_pair_count, dim3(wblk), dim3(CT), 0, st, d);
            launch_pdl(k_offgrid_pairs<false>, dim3(OFF_BLOCKS), dim3(OFF_T), 0, st, d);
            scan_exclusive(d.pair_cnt, d.pair_off, nullptr, d.N, d.scan_scratch, st, launches);
            launch_pdl(k_ml_pair_write, dim3(wblk), dim3(CT), 0, st, d);
            launch_pdl(k_offgrid_pairs<true>, dim3(OFF_BLOCKS), dim3(OFF_T), 0, st, d);
            *launches += 6;
            launch_pair_sort(d, st, launches);
        } else {
            launch_pdl(k_pair_count, dim3(wblk), dim3(CT), 0, st, d);
            scan_exclusive(d.pair_cnt, d.pair_off, nullptr, d.N, d.scan_scratch, st, launches);
            launch_pdl(k_pair_write, dim3(wblk), dim3(CT), 0, st, d);
            *launches += 4;
        }
    }
    const long long nt = (long long)d.cap_pairs + d.N;
    launch_pdl(k_narrow_count, dim3(stride_grid(nt, CT)), dim3(CT), 0, st, d);
    scan_exclusive(d.npc, d.npc_off, d.ctr + C_NPAIRS, d.cap_pairs, d.scan_scratch, st, launches);
    scan_exclusive(d.gnd_cnt, d.gnd_off, nullptr, d.N, d.scan_scratch, st, launches);
    launch_pdl(k_narrow_write, dim3(stride_grid(nt, CT)), dim3(CT), 0, st, d);
    *launches += 2;
}

}  // namespace pabd
