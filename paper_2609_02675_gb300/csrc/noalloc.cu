// Allocation-free broad phase (pabd_broadphase_noalloc): the same kernels as a scene's
// broad phase, run on caller-provided inputs and outputs with their scratch in a static
// device array of fixed size instead of memory allocated at scene creation.
#include <cuda.h>

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

// Device addresses of the static array, one per CUDA context that has called: the address
// belongs to the context that looked it up (a device reset or another context on the same
// device makes it stale), so the cache is keyed by the current context's unique id.
struct AddrEntry {
    int dev;
    unsigned long long ctx;
    unsigned char* addr;
};
constexpr int MAX_ENTRIES = 64;
std::mutex g_mu;
AddrEntry g_addr[MAX_ENTRIES];
int g_n_addr = 0;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// unique id of the current context (driver entry points looked up through the runtime, so
// the library needs no link to the driver library)
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_cur || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || !f1)
            return false;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess || !f2)
            return false;
        get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

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
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return PABD_ERR_CUDA;
    unsigned char* base = nullptr;
    {
        // once per device and context, with that device current: the device address of the
        // static array
        std::lock_guard<std::mutex> lk(g_mu);
        unsigned long long ctx = 0;
        const bool have_ctx = current_context_id(&ctx);  // false before the runtime made one current
        for (int k = 0; have_ctx && k < g_n_addr && !base; ++k)
            if (g_addr[k].dev == dev && g_addr[k].ctx == ctx) base = g_addr[k].addr;
        if (!base) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return PABD_ERR_CUDA;
            base = static_cast<unsigned char*>(ptr);
            if ((have_ctx || current_context_id(&ctx)) && g_n_addr < MAX_ENTRIES) g_addr[g_n_addr++] = AddrEntry{dev, ctx, base};
        }
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
