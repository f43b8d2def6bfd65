// Sorting of short integer slices in place (ascending, keys unique within a slice): a warp's
// ranking for up to 32 keys, its bitonic network in registers for up to 64, and a block's for
// longer slices -- runs of up
// to LONG_SMEM keys in shared memory, then merge passes through a scratch slice.  Used for
// the CSR of bond ends (k_step.cu) and for the pair lists of both broad phases (k_collision.cu,
// k_lbvh.cu).
#pragma once
#include "pabd_internal.h"

namespace pabd {

constexpr int LONG_T = 1024;
constexpr int LONG_SMEM = 4096;  // ints of dynamic shared memory (16 KB: several blocks per SM, no carve-out change)

// 64 keys held two per lane (key k in lane k / 2, slot k % 2) sorted ascending by the 32
// lanes of a warp: a bitonic network of shuffles
__device__ __forceinline__ void warp_sort64(int& v0, int& v1, int lane) {
    for (int size = 2; size <= 64; size <<= 1) {
        const bool up = ((2 * lane) & size) == 0;       // ascending block (same for both slots)
        for (int stride = size >> 1; stride > 1; stride >>= 1) {
            const bool lower = ((2 * lane) & stride) == 0; // partner k ^ stride is in lane ^ stride/2
            const int o0 = __shfl_xor_sync(0xffffffffu, v0, stride >> 1);
            const int o1 = __shfl_xor_sync(0xffffffffu, v1, stride >> 1);
            v0 = (lower == up) ? min(v0, o0) : max(v0, o0);
            v1 = (lower == up) ? min(v1, o1) : max(v1, o1);
        }
        const int mn = min(v0, v1), mx = max(v0, v1);  // stride 1: the lane's own pair
        v0 = up ? mn : mx;
        v1 = up ? mx : mn;
    }
}

// up to 32 unique keys, one per lane (lanes >= n hold nothing): each key's rank among the n,
// counted through n broadcasts -- independent shuffles, no dependent network
__device__ __forceinline__ int warp_rank32(int v, int n, int lane) {
    int r = 0;
    for (int k = 0; k < n; ++k) {
        const int o = __shfl_sync(0xffffffffu, v, k);
        r += (o < v) ? 1 : 0;
    }
    return lane < n ? r : -1;
}

// slice v[0..n), n <= 64, by the 32 lanes of a warp: by rank up to 32 keys, else the bitonic
// network (padding INT_MAX)
__device__ __forceinline__ void warp_sort_slice64(int* v, int n, int lane) {
    if (n <= 32) {
        const int x = lane < n ? v[lane] : 0x7fffffff;
        const int r = warp_rank32(x, n, lane);
        __syncwarp();
        if (r >= 0) v[r] = x;
        return;
    }
    int v0 = (2 * lane < n) ? v[2 * lane] : 0x7fffffff;
    int v1 = (2 * lane + 1 < n) ? v[2 * lane + 1] : 0x7fffffff;
    warp_sort64(v0, v1, lane);
    if (2 * lane < n) v[2 * lane] = v0;
    if (2 * lane + 1 < n) v[2 * lane + 1] = v1;
}

// slice v[0..n) by a whole block of LONG_T threads with `key` LONG_SMEM ints of shared memory
// and tmp[0..n) scratch: runs of up to LONG_SMEM keys by a bitonic network in shared memory,
// then runs merged pairwise (run length doubling), each key placed at its index in its run
// plus its rank in the partner run (a binary search), ping-ponging between v and tmp.  Every
// thread of the block calls it with the same slice.
__device__ __forceinline__ void block_sort_slice(int* v, int n, int* tmp, int* key) {
    for (int r0 = 0; r0 < n; r0 += LONG_SMEM) {
        const int rn = min(LONG_SMEM, n - r0);
        int m = 2;
        while (m < rn) m <<= 1;
        for (int k = threadIdx.x; k < m; k += LONG_T) key[k] = k < rn ? v[r0 + k] : 0x7fffffff;
        __syncthreads();
        for (int size = 2; size <= m; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int k = threadIdx.x; k < m; k += LONG_T) {
                    const int l = k ^ stride;
                    if (l > k) {
                        const bool up = (k & size) == 0;
                        const int a = key[k], b = key[l];
                        if ((a > b) == up) { key[k] = b; key[l] = a; }
                    }
                }
                __syncthreads();
            }
        }
        for (int k = threadIdx.x; k < rn; k += LONG_T) v[r0 + k] = key[k];
        __syncthreads();
    }
    int* src = v;
    int* dst = tmp;
    for (int R = LONG_SMEM; R < n; R <<= 1) {
        for (int k = threadIdx.x; k < n; k += LONG_T) {
            const int run = k / R, start = run * R, pstart = (run ^ 1) * R;
            const int plen = max(0, min(R, n - pstart));
            const int x = src[k];
            int lo = 0, hi = plen;  // keys of the partner run below x
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (src[pstart + mid] < x) lo = mid + 1; else hi = mid;
            }
            dst[min(start, pstart) + (k - start) + lo] = x;
        }
        __syncthreads();
        int* t = src; src = dst; dst = t;
    }
    if (src != v) {
        for (int k = threadIdx.x; k < n; k += LONG_T) v[k] = src[k];
        __syncthreads();
    }
}

}  // namespace pabd
