// Allocation-free broad phase (pabd_broadphase_noalloc): the same kernels as a scene's
// broad phase, run on caller-provided inputs and outputs with their scratch in a static
// device array of fixed size instead of memory allocated at scene creation.
#include <mutex>

#include "../../include/pabd.h"
#include "pabd_internal.h"

using namespace pabd;

namespace {

constexpr int NA_MAX = PABD_NOALLOC_MAX_BODIES;
constexpr int NA_TABLE = 2 * NA_MAX;  // largest hash table (buckets >= 2 x bodies)
constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_LO = 0;
constexpr size_t OFF_HI = OFF_LO + al(sizeof(float4) * NA_MAX);
constexpr size_t OFF_CELL = OFF_HI + al(sizeof(float4) * NA_MAX);
constexpr size_t OFF_BCNT = OFF_CELL + al(sizeof(int4) * NA_MAX);
constexpr size_t OFF_BCUR = OFF_BCNT + al(sizeof(int) * NA_TABLE);
constexpr size_t OFF_BOFF = OFF_BCUR + al(sizeof(int) * NA_TABLE);
constexpr size_t OFF_ITEMS = OFF_BOFF + al(sizeof(int) * (NA_TABLE + 1));
constexpr size_t OFF_PCNT = OFF_ITEMS + al(sizeof(int) * NA_MAX);
constexpr size_t OFF_POFF = OFF_PCNT + al(sizeof(int) * NA_MAX);
constexpr size_t OFF_LARGE = OFF_POFF + al(sizeof(int) * (NA_MAX + 1));
constexpr size_t OFF_CTR = OFF_LARGE + al(sizeof(int) * NA_MAX);
constexpr size_t OFF_SCAN = OFF_CTR + al(sizeof(int) * C_COUNT);
constexpr size_t SCAN_INTS = NA_TABLE / 4096 + 2;  // block totals of the largest scan
constexpr size_t NA_BYTES = OFF_SCAN + al(sizeof(int) * SCAN_INTS);

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_addr[MAX_DEVICES] = {nullptr};

}  // namespace

// the scratch (about 1.5 MB); device code could name it directly, host code needs its address
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

extern "C" pabd_status pabd_broadphase_noalloc(const float* q, const float* vel, const float* he,
                                               const int32_t* group, const int32_t* flags, int32_t n_bodies,
                                               double h, double margin, double d_hat_rel, int32_t* pairs_out,
                                               int32_t max_pairs, int32_t* n_pairs_out, void* stream) {
    if (n_bodies < 0 || n_bodies > NA_MAX || max_pairs < 0) return PABD_ERR_ARG;
    if (n_bodies > 0 && (!q || !vel || !he || !group || !flags)) return PABD_ERR_ARG;
    if (!n_pairs_out || (max_pairs > 0 && !pairs_out)) return PABD_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return PABD_ERR_CUDA;
    unsigned char* base = nullptr;
    {
        // once per device, with that device current: the device address of the static array
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return PABD_ERR_CUDA;
            g_addr[dev] = static_cast<unsigned char*>(ptr);
        }
        base = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    Dev d{};
    d.N = n_bodies;
    d.p.h = (float)h;
    d.p.margin = (float)margin;
    d.p.d_hat_rel = (float)d_hat_rel;
    d.p.body_contacts = 1;
    int bits = 6;
    while ((1 << bits) < 2 * n_bodies) ++bits;
    d.table_bits = bits;
    d.cap_pairs = max_pairs;
    d.qn = (float4*)q;
    d.vel = (float4*)vel;
    d.he = (float4*)he;
    d.group = (int*)group;
    d.bflags = (int*)flags;
    d.lo = (float4*)(base + OFF_LO);
    d.hi = (float4*)(base + OFF_HI);
    d.cell = (int4*)(base + OFF_CELL);
    d.bucket_cnt = (int*)(base + OFF_BCNT);
    d.bucket_cur = (int*)(base + OFF_BCUR);
    d.bucket_off = (int*)(base + OFF_BOFF);
    d.bucket_items = (int*)(base + OFF_ITEMS);
    d.pair_cnt = (int*)(base + OFF_PCNT);
    d.pair_off = (int*)(base + OFF_POFF);
    d.ctr = (int*)(base + OFF_CTR);
    d.large_ids = (int*)(base + OFF_LARGE);
    d.scan_scratch = (int*)(base + OFF_SCAN);
    d.pairs = (int2*)pairs_out;
    long long launches = 0;
    if (n_bodies == 0) {
        if (cudaMemsetAsync(n_pairs_out, 0, sizeof(int32_t), st) != cudaSuccess) return PABD_ERR_CUDA;
        return PABD_OK;
    }
    launch_broadphase(d, st, &launches);
    // the number found (before any cut to max_pairs) is the last prefix sum
    if (cudaMemcpyAsync(n_pairs_out, d.pair_off + n_bodies, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
        return PABD_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return PABD_ERR_CUDA;
    return PABD_OK;
}
