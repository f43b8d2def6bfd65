// Per-step kernels around the sweep: the predictor and the velocity recovery of Alg. 1,
// the time-dependent drive anchors, the CSR of bond ends and the per-group residual.
#include "pabd_internal.h"
#include "predict.cuh"
#include "sort_slices.cuh"

namespace pabd {

constexpr int ST_T = 256;
static inline int nblk(int n) { return n > 0 ? (n + ST_T - 1) / ST_T : 1; }

// the predictor of every body (predict_body)
__global__ void k_predict(Dev d) {
    pdl_enter();
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.N) return;
    predict_body(d, b);
}

// Rotation matrix -> unit quaternion (Shepperd's method: divide by the largest of
// 4w^2, 4x^2, 4y^2, 4z^2).
__device__ __forceinline__ float4 mat_to_quat(const float* R) {
    float tr = R[0] + R[4] + R[8];
    float x, y, z, w;
    if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
        float s = sqrtf(1.f + tr) * 2.f;
        w = 0.25f * s; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
    } else if (R[0] >= R[4] && R[0] >= R[8]) {
        float s = sqrtf(1.f + R[0] - R[4] - R[8]) * 2.f;
        x = 0.25f * s; w = (R[7] - R[5]) / s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
    } else if (R[4] >= R[8]) {
        float s = sqrtf(1.f + R[4] - R[0] - R[8]) * 2.f;
        y = 0.25f * s; w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; z = (R[5] + R[7]) / s;
    } else {
        float s = sqrtf(1.f + R[8] - R[0] - R[4]) * 2.f;
        z = 0.25f * s; w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s;
    }
    float n = rsqrtf(x * x + y * y + z * z + w * w);
    return make_float4(x * n, y * n, z * n, w * n);
}

// Velocity recovery (Alg. 1, Sec. 4.4): v = (c^{n+1} - c^n)/h;
// [w]x = skew part of (A^{n+1} - A^n)(A^n)^T / h; Q^{n+1} = quat(A^{n+1}), sign-continuous.
__device__ __forceinline__ void finalize_body(const Dev& d, int b, const float4* __restrict__ qf) {
    if ((d.bflags[b] & BF_PINNED) || held(d, b)) return;  // (a held group keeps its state)
    float4 n0 = d.qn[3 * b], n1 = d.qn[3 * b + 1], n2 = d.qn[3 * b + 2];
    float4 f0 = qf[3 * b], f1 = qf[3 * b + 1], f2 = qf[3 * b + 2];
    const float c0[3] = {n0.x, n0.y, n0.z}, c1[3] = {f0.x, f0.y, f0.z};
    const float A0[9] = {n0.w, n1.x, n1.y, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w};
    const float A1[9] = {f0.w, f1.x, f1.y, f1.z, f1.w, f2.x, f2.y, f2.z, f2.w};
    const float ih = d.p.inv_h;
    bool finite = true;
    float v[3];
    for (int k = 0; k < 3; ++k) { v[k] = (c1[k] - c0[k]) * ih; finite &= isfinite(c1[k]); }
    float W[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            float s = 0.f;
            for (int k = 0; k < 3; ++k) s += (A1[3 * r + k] - A0[3 * r + k]) * A0[3 * c + k];
            W[3 * r + c] = s * ih;
        }
    for (int k = 0; k < 9; ++k) finite &= isfinite(A1[k]);
    if (!finite) atomicOr(&d.ctr[C_STATUS], ST_DIVERGED);
    d.vel[b] = make_float4(v[0], v[1], v[2], 0.f);
    d.omg[b] = make_float4(0.5f * (W[7] - W[5]), 0.5f * (W[2] - W[6]), 0.5f * (W[3] - W[1]), 0.f);
    float4 Q;
    if (d.p.project) {
        Q = mat_to_quat(A1);
        float4 Qo = d.quat[b];
        if (Q.x * Qo.x + Q.y * Qo.y + Q.z * Qo.z + Q.w * Qo.w < 0.f) Q = make_float4(-Q.x, -Q.y, -Q.z, -Q.w);
    } else {
        Q = d.qstar[b];
    }
    d.quat[b] = Q;
    d.qn[3 * b] = f0; d.qn[3 * b + 1] = f1; d.qn[3 * b + 2] = f2;
}

__global__ void k_finalize(Dev d, const float4* __restrict__ qf, int dyn) {
    pdl_enter();
    // under a residual threshold the last iterate sits in the buffer of the sweep count's parity
    if (dyn) qf = (d.sweep_ctl[0] & 1) ? d.qb : d.qa;
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) atomicAdd((unsigned long long*)d.step_index, 1ull);
    if (b >= d.N) return;
    finalize_body(d, b, qf);
}

// Drive anchors at t = (step + 1) h: x_i = x_i0 + arm (cos th r + sin th (u x r)),
// th = amp sin(2 pi t / period + phase).
__global__ void k_drive_update(Dev d) {
    pdl_enter();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.Ndrive) return;
    const double t = (double)(*d.step_index + 1) * d.p.h_d;
    float4 a = d.drv[3 * k], r = d.drv[3 * k + 1], ur = d.drv[3 * k + 2];
    float2 pp = d.drv_t[k];
    const float th = r.w * sinf((float)(6.283185307179586 * t / (double)pp.x) + pp.y);
    float cs, sn;
    sincosf(th, &sn, &cs);
    const int bi = d.drv_bond[k];
    float4 cur = d.bxi[bi];
    d.bxi[bi] = make_float4(a.x + a.w * (cs * r.x + sn * ur.x), a.y + a.w * (cs * r.y + sn * ur.y),
                            a.z + a.w * (cs * r.z + sn * ur.z), cur.w);
}

// ---- CSR of bond ends: ends of dynamic bodies, sorted by (body, 2 * bond + side) ----

__device__ __forceinline__ bool end_live(const Dev& d, int body) {
    return body >= 0 && !(d.bflags[body] & BF_PINNED);
}

// (both stride over this step's bonds, C_NBONDS of them)
__global__ void k_csr_count(Dev d) {
    pdl_enter();
    const int nb = d.ctr[C_NBONDS];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        int4 m = d.bmeta[b];
        if (end_live(d, m.x)) atomicAdd(&d.end_cnt[m.x], 1);
        if (end_live(d, m.y)) atomicAdd(&d.end_cnt[m.y], 1);
    }
}

__global__ void k_csr_fill(Dev d) {
    pdl_enter();
    const int nb = d.ctr[C_NBONDS];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        int4 m = d.bmeta[b];
        if (end_live(d, m.x)) d.end_id[d.end_off[m.x] + atomicAdd(&d.end_cur[m.x], 1)] = 2 * b;
        else d.end_pos[2 * b] = -1;
        if (end_live(d, m.y)) d.end_id[d.end_off[m.y] + atomicAdd(&d.end_cur[m.y], 1)] = 2 * b + 1;
        else d.end_pos[2 * b + 1] = -1;
    }
}

// Sort each body's slice of end ids (one warp per body), then record every end's slot and
// material point.  Slices of up to HEAVY_ENDS (64) ends are sorted in registers by a bitonic
// network (element k sits in lane k / 2, slot k % 2; padding is INT_MAX); a longer slice's
// body goes on the heavy list, whose slices k_csr_sort_long sorts.  Either way the slice ends
// up in ascending end id.
__global__ void k_csr_sort(Dev d) {
    pdl_enter();
    const int body = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (body >= d.N) return;
    const int s = d.end_off[body], e = d.end_off[body + 1], n = e - s;
    if (n > HEAVY_ENDS) {
        if (lane == 0) d.heavy[atomicAdd(&d.ctr[C_NHEAVY], 1)] = body;
        return;
    }
    warp_sort_slice64(d.end_id + s, n, lane);
    __syncwarp();
    for (int p = s + lane; p < e; p += 32) {
        const int id = d.end_id[p];
        const int bond = id >> 1;
        d.end_pos[id] = p;
        const float4 x = (id & 1) ? d.bxj[bond] : d.bxi[bond];
        d.end_x[p] = make_float4(x.x, x.y, x.z, 0.f);
    }
}

// CSR of a scene whose only contacts are with the ground.  Contact bonds follow the static
// ones and the ground contacts are numbered in body order (k_narrow_write), so in (body,
// 2 bond + side) order body b's slice is its static ends (fixed at creation) followed by its
// ground contacts, and starts at sta_off[b] + gnd_off[b] -- the sum of two prefix sums: no
// count, atomics or sort.  Ground contacts past the contact capacity were not written (the
// narrow phase latched PABD_ERR_CAPACITY); the slices skip them.
__global__ void k_csr_ground(Dev d) {
    pdl_enter();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > d.N) return;
    const int cap = d.cap_contacts;
    const int g0 = min(d.gnd_off[b], cap);
    const int off = d.sta_off[b] + g0;
    d.end_off[b] = off;
    if (b == d.N) return;
    const int s0 = d.sta_off[b], sn = d.sta_off[b + 1] - s0;
    const int gn = min(d.gnd_off[b + 1], cap) - g0;
    for (int k = 0; k < sn; ++k) {
        const int id = d.sta_id[s0 + k];
        const int bond = id >> 1;
        d.end_id[off + k] = id;
        d.end_pos[id] = off + k;
        const float4 x = (id & 1) ? d.bxj[bond] : d.bxi[bond];
        d.end_x[off + k] = make_float4(x.x, x.y, x.z, 0.f);
    }
    for (int k = 0; k < gn; ++k) {
        const int bond = d.Nc + g0 + k;
        const int p = off + sn + k;
        d.end_id[p] = 2 * bond;
        d.end_pos[2 * bond] = p;
        const float4 x = d.bxi[bond];
        d.end_x[p] = make_float4(x.x, x.y, x.z, 0.f);
    }
    if (sn + gn > HEAVY_ENDS) d.heavy[atomicAdd(&d.ctr[C_NHEAVY], 1)] = b;
}

// The heavy bodies' slices, one block per body (block_sort_slice), the end-record buffer
// (unused at this stage) as scratch.
__global__ void __launch_bounds__(LONG_T) k_csr_sort_long(Dev d) {
    pdl_enter();
    extern __shared__ int key[];
    const int nheavy = d.ctr[C_NHEAVY];
    for (int h = blockIdx.x; h < nheavy; h += gridDim.x) {
        const int body = d.heavy[h];
        const int s = d.end_off[body], e = d.end_off[body + 1], n = e - s;
        block_sort_slice(d.end_id + s, n, reinterpret_cast<int*>(d.ends) + s, key);
        for (int p = s + threadIdx.x; p < e; p += LONG_T) {
            const int id = d.end_id[p];
            const int bond = id >> 1;
            d.end_pos[id] = p;
            const float4 x = (id & 1) ? d.bxj[bond] : d.bxi[bond];
            d.end_x[p] = make_float4(x.x, x.y, x.z, 0.f);
        }
        __syncthreads();
    }
}

// ---- light bodies ordered by (class, end count) ----

constexpr int BIN_T = 256;

// bin of body b in the light order, or -1 for a body on the heavy list: the bodies on the
// extended path (statically flagged) in bins 0..HEAVY_ENDS by descending end count, the others
// after them in the same way
__device__ __forceinline__ int light_bin(const Dev& d, int b) {
    const int fl = d.bflags[b];
    const int n = d.end_off[b + 1] - d.end_off[b];
    if (fl & BF_PINNED) return END_BINS;
    if (n > HEAVY_ENDS) return -1;
    const bool ext = d.p.precision_policy == 3 || (d.p.precision_policy && (fl & BF_FP64));
    return (ext ? 0 : END_BINS) + (HEAVY_ENDS - n);
}

// bodies per bin: a block histogram in shared memory, one global atomic per bin and block
__global__ void __launch_bounds__(BIN_T) k_bin_count(Dev d) {
    pdl_enter();
    __shared__ int h[2 * END_BINS];
    for (int k = threadIdx.x; k < 2 * END_BINS; k += BIN_T) h[k] = 0;
    __syncthreads();
    const int b = blockIdx.x * BIN_T + threadIdx.x;
    if (b < d.N) {
        const int k = light_bin(d, b);
        if (k >= 0) atomicAdd(&h[k], 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * END_BINS; k += BIN_T)
        if (h[k]) atomicAdd(&d.bin_cnt[k], h[k]);
}

// Each body's slot: the bin's start (prefix of the bin counts), plus the range this block
// reserved inside the bin, plus the body's rank among the block's bodies of that bin (warps
// in order, lanes in order: a block's bodies keep their body order inside its range).
__global__ void __launch_bounds__(BIN_T) k_bin_scatter(Dev d) {
    pdl_enter();
    constexpr int NW = BIN_T / 32, NB = 2 * END_BINS;
    static_assert(NB <= BIN_T, "one thread per bin");
    __shared__ int cnt[NW][NB];
    __shared__ int start[NB];
    __shared__ int incl[NB];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    for (int k = t; k < NW * NB; k += BIN_T) (&cnt[0][0])[k] = 0;
    const int b = blockIdx.x * BIN_T + t;
    const int key = b < d.N ? light_bin(d, b) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int gc = t < NB ? d.bin_cnt[t] : 0;
    if (t < NB) incl[t] = gc;
    __syncthreads();
    if (key >= 0 && rank == 0) cnt[w][key] = __popc(peers);
    // inclusive prefix of the bin counts (Hillis-Steele in shared memory)
    for (int o = 1; o < NB; o <<= 1) {
        const int v = (t < NB && t >= o) ? incl[t - o] : 0;
        __syncthreads();
        if (t < NB) incl[t] += v;
        __syncthreads();
    }
    if (t < NB) {
        int run = 0;
        for (int k = 0; k < NW; ++k) {
            const int c = cnt[k][t];
            cnt[k][t] = run;
            run += c;
        }
        start[t] = (incl[t] - gc) + (run ? atomicAdd(&d.bin_cur[t], run) : 0);
    }
    if (blockIdx.x == 0 && t == 0) d.ctr[C_NLIGHT] = incl[NB - 1];
    __syncthreads();
    if (key >= 0) d.order[start[key] + cnt[w][key] + rank] = b;
}

void launch_light_order(const Dev& d, cudaStream_t st, long long* launches) {
    const int g = d.N > 0 ? (d.N + BIN_T - 1) / BIN_T : 1;
    launch_pdl(k_bin_count, dim3(g), dim3(BIN_T), 0, st, d);
    launch_pdl(k_bin_scatter, dim3(g), dim3(BIN_T), 0, st, d);
    *launches += 2;
}

cudaError_t setup_csr_kernels() {
    return cudaFuncSetAttribute(k_csr_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                LONG_SMEM * (int)sizeof(int));
}

// per-group residual sqrt(sum over the group's bodies of |q^{k+1} - q^k|^2): one block of
// RES_T threads per group, fixed per-thread strides, warp shuffle tree, warps summed in
// order by thread 0 (deterministic)
constexpr int RES_T = 128;

// the sum of resid_body over [s, e) in the fixed order: RES_T-strided per thread, a warp xor
// tree, the warps in order (thread 0 returns it)
__device__ __forceinline__ double block_resid_sum(const Dev& d, int s, int e, double* part) {
    double acc = 0.0;
    for (int b = s + threadIdx.x; b < e; b += RES_T) acc += d.resid_body[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < RES_T / 32; ++w) t += part[w];
    return t;
}

// Scenes with a group of more than RES_CHUNK bodies: a block per chunk of at most RES_CHUNK
// bodies of one group (Dev::res_chunk, the chunks of each group in order) sums it as
// k_group_resid sums a group, then each group adds its chunks' sums in order.  A group of one
// chunk gets k_group_resid's value bit for bit; a larger group is summed by as many blocks as it
// has chunks instead of by one.
__global__ void __launch_bounds__(RES_T) k_resid_chunks(Dev d) {
    pdl_enter();
    __shared__ double part[RES_T / 32];
    const int2 c = d.res_chunk[blockIdx.x];
    const double t = block_resid_sum(d, c.x, c.y, part);
    if (threadIdx.x == 0) d.res_part[blockIdx.x] = t;
}

__global__ void k_resid_groups(Dev d) {
    pdl_enter();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.G) return;
    double t = 0.0;
    for (int c = d.res_coff[g]; c < d.res_coff[g + 1]; ++c) t += d.res_part[c];
    d.resid_group[g] = sqrt(t);
}

__global__ void __launch_bounds__(RES_T) k_group_resid(Dev d) {
    pdl_enter();
    __shared__ double part[RES_T / 32];
    const int g = blockIdx.x;
    if (g >= d.G) return;
    const double t = block_resid_sum(d, d.group_off[g], d.group_off[g + 1], part);
    if (threadIdx.x == 0) d.resid_group[g] = sqrt(t);
}

void launch_predict(const Dev& d, cudaStream_t st, long long* launches) {
    launch_pdl(k_predict, dim3(nblk(d.N)), dim3(ST_T), 0, st, d);
    *launches += 1;
}

void launch_drive_update(const Dev& d, cudaStream_t st, long long* launches) {
    if (d.Ndrive == 0) return;
    launch_pdl(k_drive_update, dim3(nblk(d.Ndrive)), dim3(ST_T), 0, st, d);
    *launches += 1;
}

// The per-step counters and scratch that the collision and CSR stages accumulate into, zeroed
// by one kernel at the head of the step: no memset nodes between the step's kernels, so each
// of them may launch while its predecessor runs.
__global__ void k_step_reset(Dev d) {
    pdl_enter();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        d.ctr[C_NPAIRS] = 0;
        d.ctr[C_CELLBITS] = 0;
        d.ctr[C_NLARGE] = 0;
        d.ctr[C_NHEAVY] = 0;
        d.ctr[C_FP64DYN] = 0;
        for (int k = C_NPHEAVY; k < C_COUNT; ++k) d.ctr[k] = 0;
    }
    if (d.p.broadphase == 0 && t < (1 << d.table_bits)) {
        d.bucket_cnt[t] = 0;
        d.bucket_cur[t] = 0;
    }
    if (t < 2 * END_BINS) {
        d.bin_cnt[t] = 0;
        d.bin_cur[t] = 0;
    }
    if (t < d.N) {
        d.end_cnt[t] = 0;
        d.end_cur[t] = 0;
        if (d.multilevel) {
            d.pair_cnt[t] = 0;
            d.pair_cur[t] = 0;
        }
    }
}

void launch_step_reset(const Dev& d, cudaStream_t st, long long* launches) {
    const long long n = std::max<long long>(1ll << d.table_bits, d.N);
    launch_pdl(k_step_reset, dim3((unsigned)((n + ST_T - 1) / ST_T)), dim3(ST_T), 0, st, d);
    *launches += 1;
}

void launch_csr(const Dev& d, cudaStream_t st, long long* launches) {
    if (d.sta_off) {
        launch_pdl(k_csr_ground, dim3(nblk(d.N + 1)), dim3(ST_T), 0, st, d);
        *launches += 1;
        return;
    }
    launch_pdl(k_csr_count, dim3(stride_grid(d.cap_bonds, ST_T)), dim3(ST_T), 0, st, d);
    scan_exclusive(d.end_cnt, d.end_off, nullptr, d.N, d.scan_scratch, st, launches);
    launch_pdl(k_csr_fill, dim3(stride_grid(d.cap_bonds, ST_T)), dim3(ST_T), 0, st, d);
    launch_pdl(k_csr_sort, dim3(nblk(d.N * 32)), dim3(ST_T), 0, st, d);
    launch_pdl(k_csr_sort_long, dim3(152), dim3(LONG_T), LONG_SMEM * sizeof(int), st, d);
    *launches += 4;
}

// Scenes whose groups have at most 128 bodies (a block per group would leave most of its threads
// idle and take one block slot per group; a larger group is better spread over the per-body
// kernel): one warp per group recovers its bodies' velocities (finalize_body) and sums
// their residuals.  Lane l plays the residual block's threads l, l + 32, ... (its RES_T / 32
// accumulators), each accumulator is combined by the same xor tree and the results added in the
// same order -- the block's value bit for bit.
__global__ void k_finalize_groups(Dev d, const float4* __restrict__ qf) {
    pdl_enter();
    const int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (g == 0 && lane == 0) atomicAdd((unsigned long long*)d.step_index, 1ull);
    if (g >= d.G) return;
    const int s = d.group_off[g], e = d.group_off[g + 1];
    for (int b = s + lane; b < e; b += 32) finalize_body(d, b, qf);
    double acc[RES_T / 32];
#pragma unroll
    for (int w = 0; w < RES_T / 32; ++w) {
        acc[w] = 0.0;
        for (int b = s + 32 * w + lane; b < e; b += RES_T) acc[w] += d.resid_body[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[w] += __shfl_xor_sync(0xffffffffu, acc[w], o);
    }
    if (lane == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < RES_T / 32; ++w) t += acc[w];
        d.resid_group[g] = sqrt(t);
    }
}

void launch_finalize(const Dev& d, const float4* q_fin, cudaStream_t st, long long* launches) {
    if (d.small_groups) {
        launch_pdl(k_finalize_groups, dim3(nblk(32 * (d.G > 0 ? d.G : 1))), dim3(ST_T), 0, st, d, q_fin);
        *launches += 1;
        return;
    }
    launch_pdl(k_finalize, dim3(nblk(d.N)), dim3(ST_T), 0, st, d, q_fin, 0);
    if (d.res_chunk) {
        launch_pdl(k_resid_chunks, dim3(d.n_res_chunks), dim3(RES_T), 0, st, d);
        launch_pdl(k_resid_groups, dim3(nblk(d.G)), dim3(ST_T), 0, st, d);
        *launches += 3;
        return;
    }
    launch_pdl(k_group_resid, dim3(d.G > 0 ? d.G : 1), dim3(RES_T), 0, st, d);
    *launches += 2;
}

// ---- sweeps under a residual threshold (Sec. 4.2 stopping rule, per scene) ----

__global__ void k_sweep_ctl_init(Dev d) {
    d.sweep_ctl[0] = 0;  // sweeps done
    d.sweep_ctl[1] = 0;  // scenes still active after this sweep
    d.sweep_ctl[2] = 1;  // loop on
    d.sweep_ctl[3] = 0;
}

// After a sweep: one block per scene still running computes that sweep's residual (the same
// fixed reduction as k_group_resid); at most resid_tol stops the scene, else it counts as
// active.  The last block to finish (a ticket counter) runs the loop control: one more sweep
// done, go on while a scene is active and fewer than n_iter sweeps ran; in a graph it also
// sets the conditional node's value.  The decision depends only on integer counts.
__global__ void __launch_bounds__(RES_T) k_sweep_check(Dev d, cudaGraphConditionalHandle h, int use_handle) {
    __shared__ double part[RES_T / 32];
    __shared__ int s_last;
    const int g = blockIdx.x;
    const bool on = d.sweep_ctl[2] != 0;
    if (on && g < d.G && !d.group_done[g]) {
        const int s = d.group_off[g], e = d.group_off[g + 1];
        double acc = 0.0;
        for (int b = s + threadIdx.x; b < e; b += RES_T) acc += d.resid_body[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < RES_T / 32; ++w) t += part[w];
            const double r = sqrt(t);
            d.resid_group[g] = r;
            if (r <= d.p.resid_tol) d.group_done[g] = 1;
            else atomicAdd(&d.sweep_ctl[1], 1);
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&d.sweep_ctl[3], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    d.sweep_ctl[3] = 0;
    int go = 0;
    if (on) {
        const int it = d.sweep_ctl[0] + 1;
        d.sweep_ctl[0] = it;
        go = atomicAdd(&d.sweep_ctl[1], 0) > 0 && it < d.p.n_iter;
        d.sweep_ctl[1] = 0;
        d.sweep_ctl[2] = go;
    }
    if (use_handle) cudaGraphSetConditional(h, go);
}

void launch_sweep_ctl_init(const Dev& d, cudaStream_t st, long long* launches) {
    k_sweep_ctl_init<<<1, 1, 0, st>>>(d);
    cudaMemsetAsync(d.group_done, 0, d.G > 0 ? d.G : 1, st);
    *launches += 1;
}

void launch_sweep_check(const Dev& d, unsigned long long handle, cudaStream_t st, long long* launches) {
    k_sweep_check<<<d.G > 0 ? d.G : 1, RES_T, 0, st>>>(d, (cudaGraphConditionalHandle)handle, handle != 0);
    *launches += 1;
}

void launch_finalize_dynamic(const Dev& d, cudaStream_t st, long long* launches) {
    launch_pdl(k_finalize, dim3(nblk(d.N)), dim3(ST_T), 0, st, d, nullptr, 1);
    *launches += 1;
}

}  // namespace pabd
