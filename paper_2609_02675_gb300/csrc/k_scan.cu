// Exclusive prefix sums of int arrays whose length lives in device memory, so that the
// launches can be captured once in a CUDA graph and replayed while the lengths change.
// Chunks of 4096 values (1024 threads x 4) are scanned per block; block totals go to a
// scratch array that one block scans; a third pass adds the block offsets.  Up to 16 chunks
// are scanned by a single block in one launch.
#include "pabd_internal.h"

namespace pabd {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// inclusive block scan of one value per thread; returns the inclusive prefix, block total in *total
__device__ __forceinline__ int block_incl_scan(int v, int* smem, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < (blockDim.x >> 5)) ? smem[lane] : 0;
        int wi = warp_incl_scan(w);
        smem[lane] = wi;  // inclusive over warps
    }
    __syncthreads();
    int base = warp ? smem[warp - 1] : 0;
    *total = smem[(blockDim.x >> 5) - 1];
    return base + inc;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_chunks(const int* __restrict__ in, int* __restrict__ out,
                                                              const int* n_dev, int n_cap, int* block_sums,
                                                              int single) {
    pdl_enter();
    __shared__ int smem[32];
    const int n = n_dev ? min(*n_dev, n_cap) : n_cap;
    const int base = blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int incl = block_incl_scan(s, smem, &total);
    int run = incl - s;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) {
        if (single) out[n] = total;
        else block_sums[blockIdx.x] = total;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_totals(int* block_sums, int nb, int* out, const int* n_dev,
                                                              int n_cap) {
    pdl_enter();
    __shared__ int smem[32];
    const int n = n_dev ? min(*n_dev, n_cap) : n_cap;
    const int base = threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < nb) ? block_sums[base + k] : 0;
        s += v[k];
    }
    int total;
    int incl = block_incl_scan(s, smem, &total);
    int run = incl - s;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < nb) block_sums[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) out[n] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_add(int* out, const int* n_dev, int n_cap,
                                                           const int* block_sums) {
    pdl_enter();
    const int n = n_dev ? min(*n_dev, n_cap) : n_cap;
    if (blockIdx.x == 0) return;
    const int add = block_sums[blockIdx.x];
    const int base = blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) out[base + k] += add;
}

// one block over up to SCAN_LOOP_MAX values: chunk after chunk, carrying the running total
// (one launch instead of three for the small arrays of a small scene)
constexpr int SCAN_LOOP_MAX = 16 * SCAN_CHUNK;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_loop(const int* __restrict__ in, int* __restrict__ out,
                                                            const int* n_dev, int n_cap) {
    pdl_enter();
    __shared__ int smem[32];
    const int n = n_dev ? min(*n_dev, n_cap) : n_cap;
    int carry = 0;
    for (int c0 = 0; c0 < n; c0 += SCAN_CHUNK) {
        const int base = c0 + threadIdx.x * SCAN_ITEMS;
        int v[SCAN_ITEMS];
        int s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            v[k] = (base + k < n) ? in[base + k] : 0;
            s += v[k];
        }
        int total;
        const int incl = block_incl_scan(s, smem, &total);
        int run = carry + incl - s;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            if (base + k < n) out[base + k] = run;
            run += v[k];
        }
        carry += total;
        __syncthreads();  // smem is rewritten by the next chunk's scan
    }
    if (threadIdx.x == 0) out[n] = carry;
}

int scan_scratch_ints(int n_cap) { return (n_cap + SCAN_CHUNK - 1) / SCAN_CHUNK + 1; }

void scan_exclusive(const int* in, int* out, const int* n_dev, int n_cap, int* scratch, cudaStream_t st,
                    long long* launches) {
    const int nb = n_cap > 0 ? (n_cap + SCAN_CHUNK - 1) / SCAN_CHUNK : 1;
    if (nb == 1) {
        launch_pdl(k_scan_chunks, dim3(1), dim3(SCAN_THREADS), 0, st, in, out, n_dev, n_cap, scratch, 1);
        *launches += 1;
        return;
    }
    if (n_cap <= SCAN_LOOP_MAX) {
        launch_pdl(k_scan_loop, dim3(1), dim3(SCAN_THREADS), 0, st, in, out, n_dev, n_cap);
        *launches += 1;
        return;
    }
    // the level-2 scan handles up to SCAN_CHUNK block totals (n_cap <= 16.7 M)
    launch_pdl(k_scan_chunks, dim3(nb), dim3(SCAN_THREADS), 0, st, in, out, n_dev, n_cap, scratch, 0);
    launch_pdl(k_scan_totals, dim3(1), dim3(SCAN_THREADS), 0, st, scratch, nb, out, n_dev, n_cap);
    launch_pdl(k_scan_add, dim3(nb), dim3(SCAN_THREADS), 0, st, out, n_dev, n_cap, scratch);
    *launches += 3;
}

}  // namespace pabd
