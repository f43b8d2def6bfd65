// Linear BVH broad phase (the paper's choice for collision detection, Sec. 5), beside the
// grid hash: it needs no cell size, so boxes of any mix of sizes and speeds cost the same.
//
//   1. scene box of the bodies' box centres (min / max over order-preserving int bits: exact
//      and order-independent);
//   2. 30-bit Morton code of every centre (10 bits per axis over the scene box);
//   3. stable LSD radix sort of (code, body) -- 8-bit digits, tiles of 1024 keys per warp,
//      per-(digit, tile) counts, their prefix sums, and a stable scatter that ranks equal
//      digits within a tile with warp match masks, so the order is deterministic;
//   4. the binary radix tree over the sorted codes by Karras' construction ("Maximizing
//      parallelism in the construction of BVHs, octrees, and k-d trees", HPG 2012): each
//      internal node finds its range and split from the longest common prefixes (equal codes
//      broken by leaf index);
//   5. bottom-up refit of the internal nodes' boxes (the second child to arrive merges);
//   6. every body i walks the tree for the leaves j > i its box overlaps that the pair filter
//      accepts: a counting walk, prefix sums, a writing walk, then each body's partner slice
//      sorted (warp or block).  The list is the sorted set of overlapping pairs: the same
//      pairs, bit for bit, as the grid hash's.
#include "pair_filter.cuh"
#include "sort_slices.cuh"

namespace pabd {

constexpr int BT = 256;        // threads per block for per-body / per-node kernels
constexpr int RX_TILE = 1024;  // keys per radix tile (one warp)

static inline int bblk(long long n) { return (int)((n + BT - 1) / BT > 0 ? (n + BT - 1) / BT : 1); }

__device__ __forceinline__ int f2o(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_bvh_init(Dev d) {
    if (threadIdx.x < 3) {
        d.bvh_bounds[threadIdx.x] = 0x7fffffff;
        d.bvh_bounds[3 + threadIdx.x] = (int)0x80000000;
    }
    if (threadIdx.x == 0) {
        d.bvh_parent[0] = -1;
        d.ctr[C_NPHEAVY] = 0;
    }
}

__global__ void k_bvh_bounds(Dev d) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.N) return;
    const float4 lo = d.lo[b], hi = d.hi[b];
    const float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (!isfinite(c[k])) continue;
        atomicMin(&d.bvh_bounds[k], f2o(c[k]));
        atomicMax(&d.bvh_bounds[3 + k], f2o(c[k]));
    }
}

// spread the low 10 bits of v to every third bit
__device__ __forceinline__ unsigned spread3(unsigned v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_bvh_morton(Dev d) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.N) return;
    const float4 lo = d.lo[b], hi = d.hi[b];
    const float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
    unsigned q[3];
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float b0 = o2f(d.bvh_bounds[k]), b1 = o2f(d.bvh_bounds[3 + k]);
        const float ext = b1 - b0;
        float u = ext > 0.f ? (c[k] - b0) / ext : 0.f;
        finite = finite && isfinite(u);
        u = fminf(fmaxf(u, 0.f), 1.f);
        q[k] = min((unsigned)(u * 1024.f), 1023u);
    }
    d.bvh_key[b] = finite ? (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]) : 0xffffffffu;
    d.bvh_id[b] = b;
}

// ---- stable radix sort of (key, id), 8 bits per pass ----

__global__ void k_rx_count(const unsigned* __restrict__ key, int n, int shift, int ntile, int* __restrict__ cnt) {
    __shared__ int c[256];
    const int tile = blockIdx.x, lane = threadIdx.x;
    for (int k = lane; k < 256; k += 32) c[k] = 0;
    __syncwarp();
    for (int step = 0; step < RX_TILE / 32; ++step) {
        const int idx = tile * RX_TILE + step * 32 + lane;
        if (idx < n) atomicAdd(&c[(key[idx] >> shift) & 255u], 1);
    }
    __syncwarp();
    for (int k = lane; k < 256; k += 32) cnt[k * ntile + tile] = c[k];
}

__global__ void k_rx_scatter(const unsigned* __restrict__ key_in, const int* __restrict__ id_in,
                             unsigned* __restrict__ key_out, int* __restrict__ id_out, int n, int shift,
                             int ntile, const int* __restrict__ off) {
    __shared__ int base[256];
    const int tile = blockIdx.x, lane = threadIdx.x;
    for (int k = lane; k < 256; k += 32) base[k] = off[k * ntile + tile];
    __syncwarp();
    const unsigned below = (1u << lane) - 1u;
    for (int step = 0; step < RX_TILE / 32; ++step) {
        const int idx = tile * RX_TILE + step * 32 + lane;
        const bool valid = idx < n;
        const unsigned k = valid ? key_in[idx] : 0u;
        const int digit = valid ? (int)((k >> shift) & 255u) : 256 + lane;  // unmatched if invalid
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        if (valid) {
            const int dst = base[digit] + __popc(peers & below);
            key_out[dst] = k;
            id_out[dst] = id_in[idx];
        }
        __syncwarp();
        if (valid && (peers & below) == 0) base[digit] += __popc(peers);  // the group's first lane
        __syncwarp();
    }
}

// ---- Karras radix tree ----

__device__ __forceinline__ int prefix(const unsigned* __restrict__ key, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const unsigned a = key[i], b = key[j];
    return a == b ? 32 + __clz(i ^ j) : __clz(a ^ b);
}

__global__ void k_bvh_build(Dev d) {
    const int n = d.N;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const unsigned* key = d.bvh_key;
    const int dir = prefix(key, n, i, i + 1) - prefix(key, n, i, i - 1) > 0 ? 1 : -1;
    const int dmin = prefix(key, n, i, i - dir);
    int lmax = 2;
    while (prefix(key, n, i, i + lmax * dir) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (prefix(key, n, i, i + (l + t) * dir) > dmin) l += t;
    const int j = i + l * dir;
    const int dnode = prefix(key, n, i, j);
    int s = 0;
    for (int div = 2;; div <<= 1) {
        const int t = (l + div - 1) / div;
        if (prefix(key, n, i, i + (s + t) * dir) > dnode) s += t;
        if (t <= 1) break;
    }
    const int gamma = i + s * dir + min(dir, 0);
    const int left = min(i, j) == gamma ? (n - 1) + gamma : gamma;
    const int right = max(i, j) == gamma + 1 ? (n - 1) + gamma + 1 : gamma + 1;
    d.bvh_kids[i] = make_int2(left, right);
    d.bvh_parent[left] = i;
    d.bvh_parent[right] = i;
}

// the box of node c (a leaf: its body's inflated box)
__device__ __forceinline__ void node_box(const Dev& d, int c, float4& lo, float4& hi) {
    const int n = d.N;
    if (c >= n - 1) {
        const int b = d.bvh_id[c - (n - 1)];
        lo = d.lo[b];
        hi = d.hi[b];
    } else {
        lo = __ldcg(&d.bvh_lo[c]);
        hi = __ldcg(&d.bvh_hi[c]);
    }
}

__global__ void k_bvh_refit(Dev d) {
    const int n = d.N;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || n < 2) return;
    int node = d.bvh_parent[(n - 1) + k];
    while (node >= 0) {
        __threadfence();
        if (atomicAdd(&d.bvh_visit[node], 1) == 0) return;  // the sibling's walk is not here yet
        __threadfence();
        const int2 ch = d.bvh_kids[node];
        float4 al, ah, bl, bh;
        node_box(d, ch.x, al, ah);
        node_box(d, ch.y, bl, bh);
        __stcg(&d.bvh_lo[node], make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.f));
        __stcg(&d.bvh_hi[node], make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.f));
        node = d.bvh_parent[node];
    }
}

// every accepted partner j > i of body i, in tree order
template <class F>
__device__ __forceinline__ int bvh_partners(const Dev& d, int i, F&& f) {
    const int n = d.N;
    if (n < 2 || !d.p.body_contacts) return 0;
    const float4 li = d.lo[i], hi = d.hi[i];
    const int gi = d.group[i], fi = d.bflags[i];
    int stack[64];
    int sp = 0, cnt = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const int node = stack[--sp];
        const int2 ch = d.bvh_kids[node];
        const int kid[2] = {ch.x, ch.y};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (kid[c] >= n - 1) {
                const int j = d.bvh_id[kid[c] - (n - 1)];
                if (j > i && pair_ok(d, i, j, gi, fi)) { f(j, cnt); ++cnt; }
            } else if (overlap(li, hi, d.bvh_lo[kid[c]], d.bvh_hi[kid[c]])) {
                if (sp < 64) stack[sp++] = kid[c];
                else atomicOr(&d.ctr[C_STATUS], ST_CAPACITY);  // deeper than any tree of 30-bit codes
            }
        }
    }
    return cnt;
}

__global__ void k_bvh_pair_count(Dev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    d.pair_cnt[i] = bvh_partners(d, i, [](int, int) {});
}

__global__ void k_bvh_pair_write(Dev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int s = d.pair_off[i], cap = d.cap_pairs;
    bvh_partners(d, i, [&](int j, int k) {
        if (s + k < cap) d.pair_j[s + k] = j;
    });
    if (i == d.N - 1) {
        const int tot = d.pair_off[d.N];
        if (tot > cap) atomicOr(&d.ctr[C_STATUS], ST_CAPACITY);
        d.ctr[C_NPAIRS] = min(tot, cap);
    }
}

// each body's partners ascending (a warp each; longer than 64: the block sort below); shared
// by the LBVH and the multilevel grid
__global__ void k_pair_sort(Dev d) {
    pdl_enter();
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= d.N) return;
    const int cap = d.cap_pairs;
    const int s = min(d.pair_off[i], cap), e = min(d.pair_off[i + 1], cap), n = e - s;
    if (n > 64) {
        if (lane == 0) d.pair_heavy[atomicAdd(&d.ctr[C_NPHEAVY], 1)] = i;
        return;
    }
    warp_sort_slice64(d.pair_j + s, n, lane);
    __syncwarp();
    for (int p = s + lane; p < e; p += 32) d.pairs[p] = make_int2(i, d.pair_j[p]);
}

__global__ void __launch_bounds__(LONG_T) k_pair_sort_long(Dev d) {
    pdl_enter();
    extern __shared__ int key[];
    const int nh = d.ctr[C_NPHEAVY], cap = d.cap_pairs;
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        const int i = d.pair_heavy[h];
        const int s = min(d.pair_off[i], cap), e = min(d.pair_off[i + 1], cap);
        block_sort_slice(d.pair_j + s, e - s, d.pair_tmp + s, key);
        for (int p = s + threadIdx.x; p < e; p += LONG_T) d.pairs[p] = make_int2(i, d.pair_j[p]);
        __syncthreads();
    }
}

cudaError_t setup_pair_sort() {
    return cudaFuncSetAttribute(k_pair_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                LONG_SMEM * (int)sizeof(int));
}

void launch_pair_sort(const Dev& d, cudaStream_t st, long long* launches) {
    launch_pdl(k_pair_sort, dim3(bblk((long long)d.N * 32)), dim3(BT), 0, st, d);
    launch_pdl(k_pair_sort_long, dim3(152), dim3(LONG_T), LONG_SMEM * sizeof(int), st, d);
    *launches += 2;
}

void launch_lbvh_pairs(const Dev& d, cudaStream_t st, long long* launches) {
    const int n = d.N;
    k_bvh_init<<<1, 32, 0, st>>>(d);
    k_bvh_bounds<<<bblk(n), BT, 0, st>>>(d);
    k_bvh_morton<<<bblk(n), BT, 0, st>>>(d);
    *launches += 3;
    const int ntile = (n + RX_TILE - 1) / RX_TILE > 0 ? (n + RX_TILE - 1) / RX_TILE : 1;
    unsigned* ka = d.bvh_key;
    unsigned* kb = d.bvh_key2;
    int* ia = d.bvh_id;
    int* ib = d.bvh_id2;
    for (int shift = 0; shift < 32; shift += 8) {
        k_rx_count<<<ntile, 32, 0, st>>>(ka, n, shift, ntile, d.rx_cnt);
        scan_exclusive(d.rx_cnt, d.rx_off, nullptr, 256 * ntile, d.scan_scratch, st, launches);
        k_rx_scatter<<<ntile, 32, 0, st>>>(ka, ia, kb, ib, n, shift, ntile, d.rx_off);
        *launches += 2;
        unsigned* tk = ka; ka = kb; kb = tk;
        int* ti = ia; ia = ib; ib = ti;
    }
    // four passes: the sorted keys and ids are back in bvh_key / bvh_id
    cudaMemsetAsync(d.bvh_visit, 0, sizeof(int) * (n > 1 ? n - 1 : 1), st);
    k_bvh_build<<<bblk(n - 1), BT, 0, st>>>(d);
    k_bvh_refit<<<bblk(n), BT, 0, st>>>(d);
    k_bvh_pair_count<<<bblk(n), BT, 0, st>>>(d);
    scan_exclusive(d.pair_cnt, d.pair_off, nullptr, n, d.scan_scratch, st, launches);
    k_bvh_pair_write<<<bblk(n), BT, 0, st>>>(d);
    *launches += 4;
    launch_pair_sort(d, st, launches);
}

}  // namespace pabd
