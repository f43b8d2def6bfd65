// Host side of the C-ABI: scene construction, upload to the device, the step sequence of
// Alg. 1 (captured once as a CUDA graph and replayed per step), state exchange and errors.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/pabd.h"
#include "pabd_internal.h"

namespace {

// Cap of the grid cell.  Every grid body tests the bodies of the 27 cells around its own, so
// the cell should be about as wide as the common box rather than the widest one: a few much
// wider boxes are cheaper off the grid, where each is tested against all N bodies.  The
// candidates are 1.25 x the widest grid box at rest (inflated by dhat and the margin) and
// 1.25 x the width that leaves the widest 8, 32, 128 or 512 boxes off the grid.  Each is
// scored by the pair tests it would take at the positions of creation: the bodies in the 27
// cells around each body (counted on a strided sample of at most 2^18 bodies, scaled back),
// plus 1.5 N per body off the grid; the cheapest wins.  With a single candidate (boxes of
// similar size) nothing is counted.
double grid_cell_cap(const std::vector<pabd_body_desc>& bodies, const std::vector<int>& flags,
                     const pabd_scene_desc& ds, bool* below_widest) {
    *below_widest = false;
    const int N = (int)bodies.size();
    std::vector<double> w;
    std::vector<int> ids;
    for (int b = 0; b < N; ++b) {
        if (flags[b] & pabd::BF_LARGE) continue;
        const double* he = bodies[b].he;
        const double hn = std::sqrt(he[0] * he[0] + he[1] * he[1] + he[2] * he[2]);
        const double dh = ds.d_hat_rel * 2.0 * std::min(std::min(he[0], he[1]), he[2]);
        w.push_back(2.0 * hn + 2.0 * (dh + ds.margin));
        ids.push_back(b);
    }
    if (w.empty()) return 0.0;
    std::vector<double> sorted = w;
    std::sort(sorted.begin(), sorted.end(), [](double a, double b) { return a > b; });
    std::vector<double> caps = {1.25 * sorted[0]};
    if (ds.body_contacts) {
        for (int k : {8, 32, 128, 512}) {
            if (k >= (int)sorted.size() / 4) break;
            const double c = 1.25 * sorted[k];
            if (c < 0.8 * caps.back()) caps.push_back(c);
        }
    }
    if (caps.size() == 1) return caps[0];
    const int n = (int)w.size();
    const int stride = std::max(1, n / (1 << 18));
    double best = caps[0], best_cost = -1.0;
    for (const double cap : caps) {
        double cell = 0.0;
        long long off = 0;
        for (int i = 0; i < n; ++i) {
            if (w[i] > cap) ++off;
            else cell = std::max(cell, w[i]);
        }
        cell *= 1.01;
        auto key = [&](long long x, long long y, long long z) {
            return (uint64_t)((x & 0x1fffff) | ((y & 0x1fffff) << 21) | ((z & 0x1fffff) << 42));
        };
        // the sampled grid bodies' cells (bodies i = 0, stride, 2 stride, ...)
        std::vector<long long> cxyz;
        std::unordered_map<uint64_t, int> cnt;
        for (int i = 0; i < n; i += stride) {
            if (w[i] > cap) continue;
            const double* c = bodies[ids[i]].c;
            const long long x = (long long)std::floor(c[0] / cell), y = (long long)std::floor(c[1] / cell),
                            z = (long long)std::floor(c[2] / cell);
            cxyz.insert(cxyz.end(), {x, y, z});
            ++cnt[key(x, y, z)];
        }
        double tests = 0.0;
        for (size_t k = 0; k < cxyz.size(); k += 3) {
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        auto it = cnt.find(key(cxyz[k] + dx, cxyz[k + 1] + dy, cxyz[k + 2] + dz));
                        if (it != cnt.end()) tests += it->second;
                    }
        }
        tests *= (double)stride * stride;
        const double cost = tests + 1.5 * (double)N * (double)off;
        if (best_cost < 0.0 || cost < best_cost) { best_cost = cost; best = cap; }
    }
    *below_widest = best < caps[0];
    return best;
}

}  // namespace

using namespace pabd;

namespace {

thread_local char g_cuda_err[256] = "";

bool cuda_ok(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", what, cudaGetErrorString(e));
    return false;
}

#define CK(call)                                              \
    do {                                                      \
        if (!cuda_ok((call), #call)) return PABD_ERR_CUDA;    \
    } while (0)

struct HostBond {
    int type;  // BondKind
    int i, j;
    double xi[3], xj[3];
    double w, p1;  // w = h^2 kappa; p1 = rest length
    // drive
    double ui[3], ri[3], arm, amp, period, phase;
    // augmented Lagrangian distance bond: kappa_start, growth, dual decay, stiffness decay
    double kappa, al_beta, al_alpha, al_gamma;
};

void quat_to_mat_d(const double* q, double* R) {
    double x = q[0], y = q[1], z = q[2], w = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
    R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
    R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

void normalize_quat(const double* q, double* o) {
    double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) o[k] = q[k] / n;
}

}  // namespace

struct pabd_scene {
    pabd_scene_desc desc;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<pabd_body_desc> bodies;
    std::vector<HostBond> bonds;
    std::vector<int> drive_ids;
    bool ready = false;
    Dev d{};
    std::vector<void*> allocs;
    size_t bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t graph_nodes = 0;
    long long launches = 0;
    long long launches_per_step = 0;
    int* h_status = nullptr;  // pinned
    cudaEvent_t ev_status = nullptr;
    bool status_pending = false;
    int fp64_bodies = 0;
    int latched = 0;
    // stage timing: events recorded between the stages of a step, captured in a second graph
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;
    cudaGraph_t prof_graph = nullptr;
    cudaGraphExec_t prof_exec = nullptr;
    double prof_acc[PABD_PROFILE_SLOTS] = {0};
    // fused sweep launch shape
    int fused = 0, mode = 1, lanes = 8, sw_block = 128, sw_grid = 1;
    // the default path's autotuner: whether it chose the mode and light order, and the mean
    // sweep time it measured for each candidate (mode 2 ordered, mode 2 in body order, mode 1
    // ordered, mode 1 in body order), nanoseconds
    int tuned = 0;
    long long tune_ns[4] = {0, 0, 0, 0};
    long long coop_fallbacks = 0;
    // augmented Lagrangian bonds: (kappa_start, 0) per static bond, the state before the first step
    std::vector<float2> al_init;
    // stream on which the body of the residual-threshold loop is captured into its graph node
    cudaStream_t body_st = nullptr;
    // polls before a device-side wait gives up (PABD_ERR_TIMEOUT); about a second by default
    unsigned wait_polls = 1u << 24;
    // pinned staging of the group hold masks: HOLD_SLOTS slots of G bytes used in turn, each
    // reused only after its previous copy to the device has completed
    static constexpr int HOLD_SLOTS = 8;
    unsigned char* hold_pinned = nullptr;
    cudaEvent_t hold_ev[HOLD_SLOTS] = {};
    int hold_next = 0;

    void* dalloc(size_t n) {
        if (n == 0) n = 16;
        n = (n + 255) & ~size_t(255);
        void* p = nullptr;
        if (desc.alloc) p = desc.alloc(n, desc.alloc_ctx);
        else if (cudaMalloc(&p, n) != cudaSuccess) p = nullptr;
        if (p) { allocs.push_back(p); bytes += n; }
        return p;
    }
};

namespace {

pabd_status status_from_bits(int bits) {
    if (bits & ST_DIVERGED) return PABD_ERR_DIVERGED;
    if (bits & ST_TIMEOUT) return PABD_ERR_TIMEOUT;
    if (bits & ST_CAPACITY) return PABD_ERR_CAPACITY;
    return PABD_OK;
}

template <class T>
bool alloc_arr(pabd_scene* s, T*& p, size_t n) {
    p = static_cast<T*>(s->dalloc(sizeof(T) * (n ? n : 1)));
    return p != nullptr;
}

// enqueue one time step of Alg. 1 on the scene's stream; with `ev` (PROF_EVENTS events) an
// event is recorded at every stage boundary: [0] start, [1] after drives + collision
// detection, [2] CSR, [3] predictor, [4] all n_iter sweeps, [5] finalize + residual
constexpr int PROF_EVENTS = 6;

void enqueue_step(pabd_scene* s, long long* launches, const cudaEvent_t* ev = nullptr) {
    const Dev& d = s->d;
    int e = 0;
    auto mark = [&]() {
        if (ev) cudaEventRecordWithFlags(ev[e++], s->st, cudaEventRecordExternal);
    };
    mark();
    launch_step_reset(d, s->st, launches);
    launch_drive_update(d, s->st, launches);
    if (d.sta_off) {
        // ground-only scene: collision, CSR and predictor in one fused front (the predictor's
        // stage is then empty in the profiling graph's split)
        launch_ground_front(d, s->st, launches);
        mark();
        if (d.light_sorted) launch_light_order(d, s->st, launches);
        mark();
    } else {
        launch_collision(d, s->st, launches);
        mark();
        launch_csr(d, s->st, launches);
        if (d.light_sorted) launch_light_order(d, s->st, launches);
        mark();
        launch_predict(d, s->st, launches);
    }
    launch_al_warm(d, s->st, launches);
    mark();
    float4* cur = d.qa;
    float4* nxt = d.qb;
    auto two_launch = [&]() {
        for (int it = 0; it < d.p.n_iter; ++it) {
            // (the counter of run-time extended-precision redos, which counts the last sweep's,
            // was reset at the head of the step; the launches follow each other as
            // programmatic dependents)
            launch_bond(d, cur, it, s->st, launches);
            launch_solve(d, cur, nxt, it, s->lanes, s->st, launches);
            float4* t = cur; cur = nxt; nxt = t;
        }
    };
    if (s->fused) {
        cudaMemsetAsync(d.ctr + C_FP64DYN, 0, sizeof(int), s->st);
        if (launch_fused_sweep(d, s->lanes, s->sw_block, s->sw_grid, s->st, launches) != cudaSuccess) {
            // the cooperative launch was refused (e.g. co-residency not available): run the
            // same sweeps as two launches each and count the fallback
            cudaGetLastError();
            s->coop_fallbacks++;
            two_launch();
        } else {
            if (d.p.n_iter & 1) { float4* t = cur; cur = nxt; nxt = t; }
        }
    } else if (s->mode == 2 && d.p.resid_tol > 0) {
        // Sec. 4.2 stopping rule: the sweeps loop on the device until every scene's residual
        // is at most resid_tol (or n_iter sweeps).  In a graph the loop is a conditional WHILE
        // node whose body is one sweep; launched eagerly, n_iter sweeps are enqueued and those
        // after the loop has ended return at once.
        launch_end_records(d, s->st, launches);
        launch_sweep_ctl_init(d, s->st, launches);
        auto one_sweep = [&](cudaStream_t st, unsigned long long handle) {
            cudaMemsetAsync(d.ctr + C_FP64DYN, 0, sizeof(int), st);
            launch_sweep_one(d, nullptr, nullptr, -1, s->lanes, st, launches);
            launch_sweep_check(d, handle, st, launches);
        };
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s->st, &cs);
        if (cs == cudaStreamCaptureStatusActive) {
            cudaGraph_t g = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            cudaStreamGetCaptureInfo(s->st, &cs, nullptr, &g, &deps, nullptr, &nd);
            cudaGraphConditionalHandle h = 0;
            cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node = nullptr;
            cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            // four sweeps (each followed by its check) per pass of the loop: the sweeps after the
            // loop has ended return at once, and a pass of the conditional node costs more than
            // a launch
            cudaStreamBeginCaptureToGraph(s->body_st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            for (int u = 0; u < 4; ++u) one_sweep(s->body_st, (unsigned long long)h);
            cudaStreamEndCapture(s->body_st, &body);
            cudaStreamUpdateCaptureDependencies(s->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        } else {
            for (int it = 0; it < d.p.n_iter; ++it) one_sweep(s->st, 0);
        }
        cur = nullptr;  // the last iterate's buffer is known on the device only
    } else if (s->mode == 2) {
        launch_end_records(d, s->st, launches);
        // (the counter of run-time extended-precision redos, which counts the last sweep's, was
        // reset at the head of the step): the sweeps follow each other as programmatic dependents
        for (int it = 0; it < d.p.n_iter; ++it) {
            launch_sweep_one(d, cur, nxt, it, s->lanes, s->st, launches, true);
            float4* t = cur; cur = nxt; nxt = t;
        }
    } else {
        two_launch();  // (the bond kernel reads the bonds, the solve their stored end records)
    }
    if (cur) launch_al_final(d, cur, s->st, launches);
    mark();
    if (cur) launch_finalize(d, cur, s->st, launches);
    else launch_finalize_dynamic(d, s->st, launches);
    mark();
}

// Launch-shape autotuner for the fused sweep: with the scene's step-0 collision, CSR and
// predictor in place (none of them changes q^n), time the sweep for each candidate grid of
// HEAVY_T-thread blocks; keep the fastest.  The shape never changes the results (each body's
// arithmetic does not depend on which block runs it).
pabd_status autotune_sweep(pabd_scene* s) {
    Dev& d = s->d;
    long long lc = 0;
    launch_step_reset(d, s->st, &lc);
    launch_drive_update(d, s->st, &lc);
    launch_collision(d, s->st, &lc);
    launch_csr(d, s->st, &lc);
    launch_predict(d, s->st, &lc);
    CK(cudaGetLastError());
    // blocks of HEAVY_T threads (a heavy body takes a whole block); the grid is tuned: all
    // co-resident blocks, or the blocks the light bodies fill, or half or a quarter of those,
    // never fewer than the HEAVY_BLOCKS blocks of the heavy role
    const int bs = HEAVY_T;
    const int maxg = fused_max_blocks(s->lanes, bs, d.p.precision_policy == 2);
    const long long need = std::max<long long>(1, ((long long)d.N * s->lanes + bs - 1) / bs);
    std::vector<int> grids;
    for (long long g : {(long long)maxg, std::min<long long>(need, maxg), (long long)maxg / 2, (long long)maxg / 4}) {
        g = std::max<long long>(g, HEAVY_BLOCKS);
        if (g <= maxg && std::find(grids.begin(), grids.end(), (int)g) == grids.end()) grids.push_back((int)g);
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int grid : grids) {
        float tot = 0.f;
        bool ok = true;
        for (int r = 0; r < 4 && ok; ++r) {
            CK(cudaEventRecord(e0, s->st));
            ok = launch_fused_sweep(d, s->lanes, bs, grid, s->st, &lc) == cudaSuccess;
            CK(cudaEventRecord(e1, s->st));
            CK(cudaEventSynchronize(e1));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, e0, e1));
            if (r > 0) tot += t;  // first launch warms caches
        }
        if (ok && tot < best) { best = tot; s->sw_block = bs; s->sw_grid = grid; }
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best >= 1e30f) { s->fused = 0; s->mode = 1; }
    // leave the counters as a fresh scene has them
    CK(cudaMemsetAsync(d.ctr, 0, sizeof(int) * C_COUNT, s->st));
    int nb0 = d.Nc;
    CK(cudaMemcpyAsync(d.ctr + C_NBONDS, &nb0, sizeof(int), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    return PABD_OK;
}

// The default path's autotuner (sweep_mode 0).  With the current state's collision, CSR,
// light order, predictor and end records in place (none of them changes the scene's state),
// time the n_iter sweeps of each candidate launch shape: one launch per sweep or a bond and a
// solve launch per sweep, each with the light bodies in (class, end count) order or in body
// order.  Every candidate gives the same results bit for bit (each body's arithmetic depends
// on its end count and the lane count only), so the fastest is kept.  Scenes with augmented
// Lagrangian bonds, whose sweeps update the bonds' state, keep one launch per sweep, ordered.
pabd_status autotune_default(pabd_scene* s) {
    Dev& d = s->d;
    const bool tune_mode = s->desc.sweep_mode == 0, tune_order = s->desc.light_order == 0;
    if (tune_mode) s->mode = 2;
    if (tune_order) d.light_sorted = 1;
    if (d.N == 0 || d.Nal > 0 || (!tune_mode && !tune_order)) return PABD_OK;
    long long lc = 0;
    Dev dd = d;
    launch_step_reset(dd, s->st, &lc);
    launch_drive_update(dd, s->st, &lc);
    if (dd.sta_off) {
        launch_ground_front(dd, s->st, &lc);
    } else {
        launch_collision(dd, s->st, &lc);
        launch_csr(dd, s->st, &lc);
        launch_predict(dd, s->st, &lc);
    }
    launch_light_order(dd, s->st, &lc);
    launch_end_records(dd, s->st, &lc);
    CK(cudaGetLastError());
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int n_it = d.p.n_iter;
    float best = 1e30f;
    for (int c = 0; c < 4; ++c) {
        const int mode = c < 2 ? 2 : 1;
        dd.light_sorted = (c & 1) ? 0 : 1;
        if ((!tune_mode && mode != s->mode) || (!tune_order && dd.light_sorted != d.light_sorted)) continue;
        float tot = 1e30f;
        for (int r = 0; r < 5; ++r) {
            // the one-launch sweeps' chunk counters, as the step's reset leaves them (each
            // sweep zeroes the next sweep's counter, so a pass must start from clean ones)
            CK(cudaMemsetAsync(dd.ctr + C_SWEEP_NEXT, 0, 2 * sizeof(int), s->st));
            CK(cudaEventRecord(e0, s->st));
            float4* cur = dd.qa;
            float4* nxt = dd.qb;
            for (int it = 0; it < n_it; ++it) {
                if (mode == 2) {
                    launch_sweep_one(dd, cur, nxt, it, s->lanes, s->st, &lc, true);
                } else {
                    launch_bond(dd, cur, it, s->st, &lc);
                    launch_solve(dd, cur, nxt, it, s->lanes, s->st, &lc);
                }
                float4* t = cur; cur = nxt; nxt = t;
            }
            CK(cudaEventRecord(e1, s->st));
            CK(cudaEventSynchronize(e1));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, e0, e1));
            if (r > 0) tot = std::min(tot, t);  // the first pass warms the caches; the fastest
                                                // of the others (least disturbed) is the figure
        }
        CK(cudaGetLastError());
        s->tune_ns[c] = (long long)(1e6 * tot / (double)n_it);
        if (tot < best) { best = tot; s->mode = mode; d.light_sorted = dd.light_sorted; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->tuned = 1;
    return PABD_OK;
}

// Capture one step as the scene's graph (if the cooperative sweep cannot be captured, capture
// the two-launch sweep instead).
pabd_status capture_step(pabd_scene* s) {
    cudaStream_t st = s->st;
    long long lc = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        lc = 0;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        enqueue_step(s, &lc);
        cudaError_t ce = cudaStreamEndCapture(st, &s->graph);
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&s->exec, s->graph, 0);
        if (ce == cudaSuccess) break;
        cudaGetLastError();
        if (s->graph) { cudaGraphDestroy(s->graph); s->graph = nullptr; }
        if (!s->fused || attempt == 1) { cuda_ok(ce, "capture of the step graph"); return PABD_ERR_CUDA; }
        s->fused = 0;
        s->mode = 1;
        s->d.light_sorted = 0;
        s->coop_fallbacks = 0;
    }
    CK(cudaGraphGetNodes(s->graph, nullptr, &s->graph_nodes));
    s->launches_per_step = lc;
    return PABD_OK;
}

pabd_status finalize_scene(pabd_scene* s) {
    if (s->ready) return PABD_OK;
    const pabd_scene_desc& ds = s->desc;
    const int N = (int)s->bodies.size();
    const int Nc = (int)s->bonds.size();
    Dev& d = s->d;
    d = Dev{};
    d.N = N;
    d.Nc = Nc;
    d.Ndrive = (int)s->drive_ids.size();
    d.G = N ? s->bodies.back().group + 1 : 0;
    // parameters
    Params& p = d.p;
    p.h = (float)ds.h; p.h2 = (float)(ds.h * ds.h); p.inv_h = (float)(1.0 / ds.h); p.h_d = ds.h;
    for (int k = 0; k < 3; ++k) p.g[k] = (float)ds.gravity[k];
    double gl = std::sqrt(ds.ground_n[0] * ds.ground_n[0] + ds.ground_n[1] * ds.ground_n[1] + ds.ground_n[2] * ds.ground_n[2]);
    for (int k = 0; k < 3; ++k) p.gn[k] = (float)(gl > 0 ? ds.ground_n[k] / gl : 0.0);
    p.gd = (float)ds.ground_d;
    p.mu = (float)ds.mu; p.c_kappa = (float)ds.c_kappa; p.d_hat_rel = (float)ds.d_hat_rel; p.margin = (float)ds.margin;
    p.n_iter = ds.n_iter; p.has_ground = ds.has_ground; p.project = ds.project; p.body_contacts = ds.body_contacts;
    if (ds.precision_policy < 0 || ds.precision_policy > 3) return PABD_ERR_ARG;
    p.precision_policy = ds.precision_policy;
    if (!(ds.resid_tol >= 0) || !std::isfinite(ds.resid_tol)) return PABD_ERR_ARG;
    p.resid_tol = ds.resid_tol;
    if (ds.broadphase < 0 || ds.broadphase > 1) return PABD_ERR_ARG;
    p.broadphase = ds.broadphase;
    // capacities
    // the two-level scans cover 4096 x 4096 values; bond ends are counted in int.  Defaults:
    // 16 pairs and 32 contacts per body (a dense granular bed reaches about 24), clamped to
    // those limits; an explicit capacity beyond them is an error
    const size_t PAIR_LIMIT = 16000000, CONTACT_LIMIT = 60000000;
    const size_t nb64 = (size_t)(N > 64 ? N : 64);
    const size_t want_pairs = ds.max_pairs ? ds.max_pairs : std::min(16 * nb64, PAIR_LIMIT);
    const size_t want_contacts = ds.max_contacts ? ds.max_contacts : std::min(32 * nb64, CONTACT_LIMIT);
    if (want_pairs > PAIR_LIMIT || want_contacts > CONTACT_LIMIT || (size_t)N > 8000000) return PABD_ERR_ARG;
    d.cap_pairs = (int)want_pairs;
    d.cap_contacts = (int)want_contacts;
    d.cap_bonds = Nc + d.cap_contacts;
    d.cap_ends = 2 * d.cap_bonds;
    int bits = 6;
    while ((1 << bits) < 2 * N) ++bits;
    d.table_bits = bits;
    const int T = 1 << bits;
    if (T > 16777216 || (long long)d.cap_bonds * 2 > 2000000000LL) return PABD_ERR_ARG;

    // host staging
    std::vector<float4> qn(3 * N), vel(N), omg(N), quat(N), mass(N), he(N);
    std::vector<int> flags(N), group(N), group_off(d.G + 1, 0), large;
    const float dr = (float)ds.d_hat_rel;
    for (int b = 0; b < N; ++b) {
        const pabd_body_desc& bd = s->bodies[b];
        double Q[4], R[9];
        normalize_quat(bd.quat, Q);
        quat_to_mat_d(Q, R);
        qn[3 * b] = make_float4((float)bd.c[0], (float)bd.c[1], (float)bd.c[2], (float)R[0]);
        qn[3 * b + 1] = make_float4((float)R[1], (float)R[2], (float)R[3], (float)R[4]);
        qn[3 * b + 2] = make_float4((float)R[5], (float)R[6], (float)R[7], (float)R[8]);
        bool pin = bd.pinned != 0;
        vel[b] = pin ? make_float4(0, 0, 0, 0) : make_float4((float)bd.v[0], (float)bd.v[1], (float)bd.v[2], 0);
        omg[b] = pin ? make_float4(0, 0, 0, 0) : make_float4((float)bd.omega[0], (float)bd.omega[1], (float)bd.omega[2], 0);
        quat[b] = make_float4((float)Q[0], (float)Q[1], (float)Q[2], (float)Q[3]);
        // Thm 4.1 for a uniform box about its centre of mass: Pi_0 = m diag(he^2) / 3
        double m = bd.mass;
        mass[b] = make_float4((float)m, (float)(m * bd.he[0] * bd.he[0] / 3.0), (float)(m * bd.he[1] * bd.he[1] / 3.0),
                              (float)(m * bd.he[2] * bd.he[2] / 3.0));
        float hx = (float)bd.he[0], hy = (float)bd.he[1], hz = (float)bd.he[2];
        float mn = std::fmin(std::fmin(hx, hy), hz);
        he[b] = make_float4(hx, hy, hz, dr * (2.0f * mn));
        int f = pin ? BF_PINNED : 0;
        double hmax = std::fmax(std::fmax(bd.he[0], bd.he[1]), bd.he[2]);
        if (hmax > ds.large_he) { f |= BF_LARGE; large.push_back(b); }
        flags[b] = f;
        group[b] = bd.group;
        group_off[bd.group + 1] = b + 1;
    }
    for (int g = 1; g <= d.G; ++g) if (group_off[g] < group_off[g - 1]) group_off[g] = group_off[g - 1];
    d.small_groups = 1;
    bool big_group = false;
    for (int g = 0; g < d.G; ++g) {
        if (group_off[g + 1] - group_off[g] > 128) d.small_groups = 0;
        if (group_off[g + 1] - group_off[g] > RES_CHUNK) big_group = true;
    }
    std::vector<int2> res_chunk;
    std::vector<int> res_coff;
    if (big_group) {
        res_coff.assign(d.G + 1, 0);
        for (int g = 0; g < d.G; ++g) {
            for (int b = group_off[g]; b < group_off[g + 1]; b += RES_CHUNK)
                res_chunk.push_back(make_int2(b, std::min(b + RES_CHUNK, group_off[g + 1])));
            if (group_off[g + 1] == group_off[g]) res_chunk.push_back(make_int2(group_off[g], group_off[g]));
            res_coff[g + 1] = (int)res_chunk.size();
        }
        d.n_res_chunks = (int)res_chunk.size();
    }
    d.Nlarge = (int)large.size();
    bool cap_below_widest = false;
    p.cell = (float)grid_cell_cap(s->bodies, flags, ds, &cap_below_widest);
    // scenes with bodies of very different widths (some flagged large, or a cell cap below the
    // widest box) use the multilevel grid (k_collision.cu)
    d.multilevel = ds.body_contacts && ds.broadphase == 0 && (d.Nlarge > 0 || cap_below_widest);
    // Expansion point of each body's system (sys_init): x_s = sum w x / (m + sum w) over the
    // ends of its static bonds (w = h^2 kappa; a drive's moving anchor at its rest angle).
    // Static extended-precision flag (reading R18): the FP64 Cholesky of the diagonally scaled
    // static-only system about x_s has a pivot below 1e-2 of its diagonal (ten times the
    // dynamic test's margin, since contacts add to the system at run time), or the static
    // bonds' weights sum to more than 10 times the mass (BF_STIFF).
    std::vector<double> sw(N, 0.0), swx(3 * (size_t)N, 0.0);
    for (const HostBond& hb : s->bonds) {
        if (hb.i >= 0) { sw[hb.i] += hb.w; for (int k = 0; k < 3; ++k) swx[3 * hb.i + k] += hb.w * hb.xi[k]; }
        if (hb.j >= 0) { sw[hb.j] += hb.w; for (int k = 0; k < 3; ++k) swx[3 * hb.j + k] += hb.w * hb.xj[k]; }
    }
    std::vector<float4> xs(N, make_float4(0, 0, 0, 0));
    std::vector<double> xsd(3 * (size_t)N, 0.0);
    for (int b = 0; b < N; ++b) {
        if (flags[b] & BF_PINNED) continue;
        const double m = s->bodies[b].mass;
        for (int k = 0; k < 3; ++k) xsd[3 * b + k] = swx[3 * b + k] / (m + sw[b]);
        xs[b] = make_float4((float)xsd[3 * b], (float)xsd[3 * b + 1], (float)xsd[3 * b + 2], 0.f);
        if (xs[b].x != 0.f || xs[b].y != 0.f || xs[b].z != 0.f) flags[b] |= BF_SHIFT;
        if (sw[b] > 10.0 * m) flags[b] |= BF_STIFF;
        // the shifted expansion point as the device uses it (rounded to FP32)
        for (int k = 0; k < 3; ++k) xsd[3 * b + k] = k == 0 ? xs[b].x : (k == 1 ? xs[b].y : xs[b].z);
    }
    std::vector<double> G(10 * (size_t)N, 0.0);
    for (int b = 0; b < N; ++b) {
        const pabd_body_desc& bd = s->bodies[b];
        const double m = bd.mass, *x = &xsd[3 * b];
        double* g = &G[10 * (size_t)b];
        g[0] = m; g[1] = -m * x[0]; g[2] = -m * x[1]; g[3] = -m * x[2];
        g[4] = m * bd.he[0] * bd.he[0] / 3.0 + m * x[0] * x[0]; g[5] = m * x[0] * x[1]; g[6] = m * x[0] * x[2];
        g[7] = m * bd.he[1] * bd.he[1] / 3.0 + m * x[1] * x[1]; g[8] = m * x[1] * x[2];
        g[9] = m * bd.he[2] * bd.he[2] / 3.0 + m * x[2] * x[2];
    }
    auto add_end = [&](int b, double w, const double* p) {
        if (b < 0) return;
        const double z[4] = {1.0, p[0] - xsd[3 * b], p[1] - xsd[3 * b + 1], p[2] - xsd[3 * b + 2]};
        double* g = &G[10 * (size_t)b];
        int k = 0;
        for (int r = 0; r < 4; ++r)
            for (int c = r; c < 4; ++c) g[k++] += w * z[r] * z[c];
    };
    for (const HostBond& hb : s->bonds) { add_end(hb.i, hb.w, hb.xi); add_end(hb.j, hb.w, hb.xj); }
    s->fp64_bodies = 0;
    for (int b = 0; b < N; ++b) {
        if (flags[b] & BF_PINNED) continue;
        const double* g = &G[10 * (size_t)b];
        const double M[4][4] = {{g[0], g[1], g[2], g[3]}, {g[1], g[4], g[5], g[6]},
                                {g[2], g[5], g[7], g[8]}, {g[3], g[6], g[8], g[9]}};
        double Lm[4][4] = {{0}};
        double worst = 1.0;
        for (int i = 0; i < 4; ++i) {
            for (int j = 0; j <= i; ++j) {
                double t = M[i][j];
                for (int k = 0; k < j; ++k) t -= Lm[i][k] * Lm[j][k];
                if (i == j) {
                    const double ratio = t / M[i][i];
                    worst = std::min(worst, ratio);
                    Lm[i][i] = std::sqrt(std::max(t, 1e-300));
                } else {
                    Lm[i][j] = t / Lm[j][j];
                }
            }
        }
        // stiffly jointed bodies too: their FP32 system resolves a joint correction only to
        // about 1e-4 (joint weights many times the mass against a rotational inertia that is
        // not -- the cancellation lands on the rotation), errors that the joints pass on to
        // their neighbours; taking them straight to the extended type costs less than a
        // test-and-redo
        if (!(worst >= 1e-2) || (flags[b] & BF_STIFF)) { flags[b] |= BF_FP64; s->fp64_bodies++; }
    }
    // static bonds
    std::vector<int4> bmeta(Nc);
    std::vector<float4> bxi(Nc), bxj(Nc), bn(Nc);
    std::vector<float4> drv(3 * d.Ndrive);
    std::vector<float2> drv_t(d.Ndrive);
    std::vector<int> drv_bond(d.Ndrive);
    std::vector<std::vector<int>> adj(N);
    for (int k = 0; k < Nc; ++k) {
        const HostBond& hb = s->bonds[k];
        bmeta[k] = make_int4(hb.i, hb.j, hb.type, 0);
        // an augmented Lagrangian bond carries h^2 here; its kappa lives in the per-bond state
        const double xw = hb.type == K_AL ? ds.h * ds.h : hb.w;
        bxi[k] = make_float4((float)hb.xi[0], (float)hb.xi[1], (float)hb.xi[2], (float)xw);
        bxj[k] = make_float4((float)hb.xj[0], (float)hb.xj[1], (float)hb.xj[2], (float)hb.p1);
        bn[k] = make_float4(0, 0, 0, 0);
        if (hb.i >= 0 && hb.j >= 0) { adj[hb.i].push_back(hb.j); adj[hb.j].push_back(hb.i); }
    }
    for (int k = 0; k < d.Ndrive; ++k) {
        const HostBond& hb = s->bonds[s->drive_ids[k]];
        double ur[3] = {hb.ui[1] * hb.ri[2] - hb.ui[2] * hb.ri[1], hb.ui[2] * hb.ri[0] - hb.ui[0] * hb.ri[2],
                        hb.ui[0] * hb.ri[1] - hb.ui[1] * hb.ri[0]};
        drv[3 * k] = make_float4((float)hb.xi[0], (float)hb.xi[1], (float)hb.xi[2], (float)hb.arm);
        drv[3 * k + 1] = make_float4((float)hb.ri[0], (float)hb.ri[1], (float)hb.ri[2], (float)hb.amp);
        drv[3 * k + 2] = make_float4((float)ur[0], (float)ur[1], (float)ur[2], 0.f);
        drv_t[k] = make_float2((float)hb.period, (float)hb.phase);
        drv_bond[k] = s->drive_ids[k];
        bmeta[s->drive_ids[k]].w = k;
    }
    // augmented Lagrangian bonds: parameters and the state a fresh scene starts from
    std::vector<float4> al_par;
    for (const HostBond& hb : s->bonds) d.Nal += hb.type == K_AL;
    if (d.Nal) {
        al_par.assign(Nc, make_float4(0, 0, 0, 0));
        s->al_init.assign(Nc, make_float2(0, 0));
        for (int k = 0; k < Nc; ++k) {
            const HostBond& hb = s->bonds[k];
            if (hb.type != K_AL) continue;
            al_par[k] = make_float4((float)hb.kappa, (float)hb.al_beta, (float)hb.al_alpha, (float)hb.al_gamma);
            s->al_init[k] = make_float2((float)hb.kappa, 0.f);
        }
    }
    // scenes whose only contacts are with the ground: each body's live static ends, sorted
    std::vector<int> sta_off, sta_id, sta_body;
    if (!ds.body_contacts) {
        std::vector<int> cnt(N + 1, 0);
        for (int k = 0; k < Nc; ++k) {
            const HostBond& hb = s->bonds[k];
            if (hb.i >= 0 && !(flags[hb.i] & BF_PINNED)) ++cnt[hb.i];
            if (hb.j >= 0 && !(flags[hb.j] & BF_PINNED)) ++cnt[hb.j];
        }
        sta_off.assign(N + 1, 0);
        for (int b = 0; b < N; ++b) sta_off[b + 1] = sta_off[b] + cnt[b];
        sta_id.assign(sta_off[N] > 0 ? sta_off[N] : 1, 0);
        sta_body.assign(sta_id.size(), 0);
        for (int b = 0; b < N; ++b)
            for (int e = sta_off[b]; e < sta_off[b + 1]; ++e) sta_body[e] = b;
        std::vector<int> cur(sta_off.begin(), sta_off.end() - 1);
        for (int k = 0; k < Nc; ++k) {  // bond order: each body's ends come out sorted
            const HostBond& hb = s->bonds[k];
            if (hb.i >= 0 && !(flags[hb.i] & BF_PINNED)) sta_id[cur[hb.i]++] = 2 * k;
            if (hb.j >= 0 && !(flags[hb.j] & BF_PINNED)) sta_id[cur[hb.j]++] = 2 * k + 1;
        }
    }
    std::vector<int> adj_off(N + 1, 0), adj_nbr;
    for (int b = 0; b < N; ++b) {
        std::vector<int>& v = adj[b];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        adj_off[b + 1] = adj_off[b] + (int)v.size();
        adj_nbr.insert(adj_nbr.end(), v.begin(), v.end());
    }

    // device allocations
    bool ok = true;
    ok &= alloc_arr(s, d.qn, 3 * N) && alloc_arr(s, d.qa, 3 * N) && alloc_arr(s, d.qb, 3 * N) && alloc_arr(s, d.sq, 3 * N);
    ok &= alloc_arr(s, d.vel, N) && alloc_arr(s, d.omg, N) && alloc_arr(s, d.quat, N) && alloc_arr(s, d.qstar, N);
    ok &= alloc_arr(s, d.mass, N) && alloc_arr(s, d.he, N) && alloc_arr(s, d.xs, N);
    ok &= alloc_arr(s, d.bflags, N) && alloc_arr(s, d.group, N) && alloc_arr(s, d.group_off, d.G + 1);
    ok &= alloc_arr(s, d.group_hold, d.G);
    ok &= alloc_arr(s, d.large_ids, N);
    ok &= alloc_arr(s, d.resid_body, N) && alloc_arr(s, d.resid_group, d.G);
    if (!res_chunk.empty())
        ok &= alloc_arr(s, d.res_chunk, res_chunk.size()) && alloc_arr(s, d.res_coff, d.G + 1) &&
              alloc_arr(s, d.res_part, res_chunk.size());
    ok &= alloc_arr(s, d.bmeta, d.cap_bonds) && alloc_arr(s, d.bxi, d.cap_bonds) && alloc_arr(s, d.bxj, d.cap_bonds) &&
          alloc_arr(s, d.bn, d.cap_bonds);
    ok &= alloc_arr(s, d.drv, 3 * d.Ndrive) && alloc_arr(s, d.drv_t, d.Ndrive) && alloc_arr(s, d.drv_bond, d.Ndrive);
    ok &= alloc_arr(s, d.end_cnt, N) && alloc_arr(s, d.end_cur, N) && alloc_arr(s, d.end_off, N + 1);
    ok &= alloc_arr(s, d.end_id, d.cap_ends) && alloc_arr(s, d.end_pos, d.cap_ends) && alloc_arr(s, d.heavy, N);
    ok &= alloc_arr(s, d.order, N) && alloc_arr(s, d.bin_cnt, 2 * END_BINS) && alloc_arr(s, d.bin_cur, 2 * END_BINS);
    ok &= alloc_arr(s, d.ends, d.cap_ends) && alloc_arr(s, d.end_x, d.cap_ends);
    ok &= alloc_arr(s, d.rec_m, d.cap_ends) && alloc_arr(s, d.rec_a, d.cap_ends) && alloc_arr(s, d.rec_b, d.cap_ends);
    ok &= alloc_arr(s, d.gbar, 2) && alloc_arr(s, d.wait_limit, 1);
    ok &= alloc_arr(s, d.lo, N) && alloc_arr(s, d.hi, N) && alloc_arr(s, d.cell, N);
    ok &= alloc_arr(s, d.bucket_cnt, T) && alloc_arr(s, d.bucket_cur, T) && alloc_arr(s, d.bucket_off, T + 1) &&
          alloc_arr(s, d.bucket_items, N);
    ok &= alloc_arr(s, d.pair_cnt, N) && alloc_arr(s, d.pair_off, N + 1) && alloc_arr(s, d.pairs, d.cap_pairs);
    ok &= alloc_arr(s, d.brec_lo, N) && alloc_arr(s, d.brec_hi, N) && alloc_arr(s, d.brec_cell, N);
    ok &= alloc_arr(s, d.lane_cnt, (size_t)32 * N);
    if (ds.body_contacts && p.broadphase == 0)
        ok &= alloc_arr(s, d.pair_stash, (size_t)32 * PAIR_STASH * N) && alloc_arr(s, d.lane_tot, (size_t)32 * N);
    ok &= alloc_arr(s, d.npc, d.cap_pairs) && alloc_arr(s, d.npc_off, d.cap_pairs + 1);
    ok &= alloc_arr(s, d.gnd_cnt, N) && alloc_arr(s, d.gnd_off, N + 1);
    ok &= alloc_arr(s, d.ctr, C_COUNT) && alloc_arr(s, d.step_index, 1);
    int ns = scan_scratch_ints(T);
    ns = std::max(ns, scan_scratch_ints(256 * (N / 1024 + 1)));
    ns = std::max(ns, scan_scratch_ints(N + 1));
    ns = std::max(ns, scan_scratch_ints(d.cap_pairs));
    ok &= alloc_arr(s, d.scan_scratch, ns);
    if (!adj_nbr.empty()) {
        ok &= alloc_arr(s, d.adj_off, N + 1) && alloc_arr(s, d.adj_nbr, adj_nbr.size());
    }
    if (d.Nal) ok &= alloc_arr(s, d.al_st0, Nc) && alloc_arr(s, d.al_st1, Nc) && alloc_arr(s, d.al_par, Nc);
    if (!sta_off.empty())
        ok &= alloc_arr(s, d.sta_off, N + 1) && alloc_arr(s, d.sta_id, sta_id.size()) &&
              alloc_arr(s, d.sta_body, sta_body.size()) && alloc_arr(s, d.gnd_loc, N) &&
              alloc_arr(s, d.gnd_blk, (N + 255) / 256 + 1) && alloc_arr(s, d.gnd_bof, (N + 255) / 256 + 1);
    if (p.resid_tol > 0) ok &= alloc_arr(s, d.sweep_ctl, 4) && alloc_arr(s, d.group_done, d.G);
    if (p.broadphase == 1) {
        const size_t ntile = ((size_t)N + 1023) / 1024 + 1;
        ok &= alloc_arr(s, d.bvh_key, N) && alloc_arr(s, d.bvh_key2, N) && alloc_arr(s, d.bvh_id, N) &&
              alloc_arr(s, d.bvh_id2, N) && alloc_arr(s, d.rx_cnt, 256 * ntile) && alloc_arr(s, d.rx_off, 256 * ntile + 1);
        ok &= alloc_arr(s, d.bvh_kids, N) && alloc_arr(s, d.bvh_parent, 2 * (size_t)N) && alloc_arr(s, d.bvh_lo, N) &&
              alloc_arr(s, d.bvh_hi, N) && alloc_arr(s, d.bvh_visit, N) && alloc_arr(s, d.bvh_bounds, 6);
    }
    if (p.broadphase == 1 || d.multilevel) {
        ok &= alloc_arr(s, d.pair_j, d.cap_pairs) && alloc_arr(s, d.pair_tmp, d.cap_pairs) &&
              alloc_arr(s, d.pair_heavy, N);
    }
    if (d.multilevel) {
        ok &= alloc_arr(s, d.blevel, N) && alloc_arr(s, d.pair_own, N) && alloc_arr(s, d.pair_cur, N);
    }
    if (!ok) return PABD_ERR_OOM;

    cudaStream_t st = s->st;
    auto up = [&](void* dst, const void* src, size_t n) { return n ? cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st) : cudaSuccess; };
    CK(up(d.qn, qn.data(), sizeof(float4) * 3 * N));
    CK(up(d.vel, vel.data(), sizeof(float4) * N));
    CK(up(d.omg, omg.data(), sizeof(float4) * N));
    CK(up(d.quat, quat.data(), sizeof(float4) * N));
    CK(up(d.mass, mass.data(), sizeof(float4) * N));
    CK(up(d.he, he.data(), sizeof(float4) * N));
    CK(up(d.xs, xs.data(), sizeof(float4) * N));
    CK(up(d.bflags, flags.data(), sizeof(int) * N));
    CK(up(d.group, group.data(), sizeof(int) * N));
    CK(up(d.group_off, group_off.data(), sizeof(int) * (d.G + 1)));
    if (d.res_chunk) {
        CK(up(d.res_chunk, res_chunk.data(), sizeof(int2) * res_chunk.size()));
        CK(up(d.res_coff, res_coff.data(), sizeof(int) * (d.G + 1)));
    }
    CK(up(d.bmeta, bmeta.data(), sizeof(int4) * Nc));
    CK(up(d.bxi, bxi.data(), sizeof(float4) * Nc));
    CK(up(d.bxj, bxj.data(), sizeof(float4) * Nc));
    CK(up(d.bn, bn.data(), sizeof(float4) * Nc));
    CK(up(d.drv, drv.data(), sizeof(float4) * 3 * d.Ndrive));
    CK(up(d.drv_t, drv_t.data(), sizeof(float2) * d.Ndrive));
    CK(up(d.drv_bond, drv_bond.data(), sizeof(int) * d.Ndrive));
    if (d.adj_off) {
        CK(up(d.adj_off, adj_off.data(), sizeof(int) * (N + 1)));
        CK(up(d.adj_nbr, adj_nbr.data(), sizeof(int) * adj_nbr.size()));
    }
    if (d.Nal) CK(up(d.al_par, al_par.data(), sizeof(float4) * Nc));
    if (d.sta_off) {
        CK(up(d.sta_off, sta_off.data(), sizeof(int) * (N + 1)));
        CK(up(d.sta_id, sta_id.data(), sizeof(int) * sta_id.size()));
        CK(up(d.sta_body, sta_body.data(), sizeof(int) * sta_body.size()));
    }
    CK(cudaMemsetAsync(d.ctr, 0, sizeof(int) * C_COUNT, st));
    CK(cudaMemsetAsync(d.step_index, 0, sizeof(long long), st));
    CK(cudaMemsetAsync(d.resid_body, 0, sizeof(double) * (N ? N : 1), st));
    CK(cudaMemsetAsync(d.resid_group, 0, sizeof(double) * (d.G ? d.G : 1), st));
    CK(cudaMemsetAsync(d.group_hold, 0, d.G ? d.G : 1, st));
    CK(cudaMemsetAsync(d.npc_off, 0, sizeof(int), st));  // no pair contacts before the first step
    CK(cudaMemsetAsync(d.end_pos, 0xff, sizeof(int) * d.cap_ends, st));
    CK(cudaMemsetAsync(d.gbar, 0, 2 * sizeof(unsigned), st));
    const unsigned wait_polls = s->wait_polls;
    CK(cudaMemcpyAsync(d.wait_limit, &wait_polls, sizeof(unsigned), cudaMemcpyHostToDevice, st));
    // bonds beyond Nc start counted as zero until the first detection
    int nb0 = Nc;
    CK(cudaMemcpyAsync(d.ctr + C_NBONDS, &nb0, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));

    // lanes per body from the descriptor; fused sweep block / grid from a timing sweep
    CK(setup_csr_kernels());
    if (p.broadphase == 1 || d.multilevel) CK(setup_pair_sort());

    // lanes per body: given, or from the body count -- the largest of 16, 8, 4, 2, 1 lanes
    // with lanes * N <= 2^17, but two rather than one for up to 2^18 bodies whose solves are
    // mostly single precision (measured: the 262 k-body pile sweeps 6% faster on two lanes than
    // on one, the 140 k-body trees, whose double-float sums every lane of a body repeats, 50%
    // slower).  A function of the scene only, so its results never depend on timing.
    int L = ds.sweep_lanes;
    if (L == 0) {
        L = 16;
        while (L > 1 && (long long)L * N > 131072) L >>= 1;
        if (L == 1 && N <= 262144 && 2 * s->fp64_bodies < N) L = 2;
    }
    if (L != 1 && L != 2 && L != 4 && L != 8 && L != 16) return PABD_ERR_ARG;
    s->lanes = L;
    // sweep mode: 1 two launches per sweep, 2 one launch per sweep, 3 fused persistent;
    // 0 = one launch per sweep (the fastest on the measured scenes).  A residual threshold
    // runs one launch per sweep.
    if (ds.sweep_mode < 0 || ds.sweep_mode > 3) return PABD_ERR_ARG;
    s->mode = ds.sweep_mode == 0 ? 2 : ds.sweep_mode;
    if (ds.light_order < 0 || ds.light_order > 2) return PABD_ERR_ARG;
    d.light_sorted = s->mode != 3 && ds.light_order != 2;
    if (p.resid_tol > 0) {
        if (d.Nal) return PABD_ERR_ARG;
        s->mode = 2;
        CK(cudaStreamCreateWithFlags(&s->body_st, cudaStreamNonBlocking));
    }
    s->fused = (s->mode == 3) && N > 0;
    if (s->fused) {
        int coop = 0, dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        if (!coop) s->fused = 0;
    }
    if (s->fused) {
        s->lanes = L;
        pabd_status tr = autotune_sweep(s);
        if (tr != PABD_OK) return tr;
    } else if ((ds.sweep_mode == 0 || ds.light_order == 0) && p.resid_tol <= 0) {
        pabd_status tr = autotune_default(s);
        if (tr != PABD_OK) return tr;
        // leave the counters as a fresh scene has them
        CK(cudaMemsetAsync(d.ctr, 0, sizeof(int) * C_COUNT, st));
        CK(cudaMemcpyAsync(d.ctr + C_NBONDS, &nb0, sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    // the state the first step's warm start reads (the trial sweeps above may have written it)
    if (d.Nal) {
        CK(up((d.p.n_iter & 1) ? d.al_st1 : d.al_st0, s->al_init.data(), sizeof(float2) * Nc));
        CK(cudaStreamSynchronize(st));
    }

    pabd_status cr = capture_step(s);
    if (cr != PABD_OK) return cr;
    CK(cudaMallocHost(&s->h_status, sizeof(int)));
    *s->h_status = 0;
    CK(cudaEventCreateWithFlags(&s->ev_status, cudaEventDisableTiming));
    s->ready = true;
    return PABD_OK;
}

pabd_status poll_status(pabd_scene* s, bool wait) {
    if (!s->status_pending) return status_from_bits(s->latched);
    cudaError_t q = wait ? cudaEventSynchronize(s->ev_status) : cudaEventQuery(s->ev_status);
    if (q == cudaErrorNotReady) return PABD_OK;
    CK(q);
    s->status_pending = false;
    s->latched |= *s->h_status;
    return status_from_bits(s->latched);
}

pabd_status enqueue_status(pabd_scene* s) {
    CK(cudaMemcpyAsync(s->h_status, s->d.ctr + C_STATUS, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    CK(cudaEventRecord(s->ev_status, s->st));
    s->status_pending = true;
    return PABD_OK;
}

}  // namespace

extern "C" {

const char* pabd_status_str(pabd_status st) {
    switch (st) {
        case PABD_OK: return "ok";
        case PABD_ERR_ARG: return "invalid argument";
        case PABD_ERR_OOM: return "device allocation failed";
        case PABD_ERR_CAPACITY: return "pair or contact capacity exceeded";
        case PABD_ERR_DIVERGED: return "state became non-finite";
        case PABD_ERR_TIMEOUT: return "device-side wait timed out";
        case PABD_ERR_CUDA: return "CUDA runtime error";
        case PABD_ERR_STATE: return "call not legal in this state";
    }
    return "unknown status";
}

const char* pabd_last_cuda_error(void) { return g_cuda_err; }

pabd_status pabd_create_scene(const pabd_scene_desc* desc, pabd_scene** out) {
    if (!desc || !out) return PABD_ERR_ARG;
    if (!(desc->h > 0) || desc->n_iter < 1 || desc->n_iter > 100000) return PABD_ERR_ARG;
    if ((desc->alloc == nullptr) != (desc->free == nullptr)) return PABD_ERR_ARG;
    pabd_scene* s = new (std::nothrow) pabd_scene();
    if (!s) return PABD_ERR_OOM;
    s->desc = *desc;
    if (desc->stream) {
        s->st = (cudaStream_t)desc->stream;
    } else {
        if (!cuda_ok(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking), "cudaStreamCreate")) {
            delete s;
            return PABD_ERR_CUDA;
        }
        s->own_stream = true;
    }
    *out = s;
    return PABD_OK;
}

pabd_status pabd_add_body(pabd_scene* s, const pabd_body_desc* b, uint32_t* out_id) {
    if (!s || !b) return PABD_ERR_ARG;
    if (s->ready) return PABD_ERR_STATE;
    for (int k = 0; k < 3; ++k) if (!(b->he[k] > 0) || !std::isfinite(b->he[k])) return PABD_ERR_ARG;
    if (!(b->mass > 0) || !std::isfinite(b->mass)) return PABD_ERR_ARG;
    double qn = b->quat[0] * b->quat[0] + b->quat[1] * b->quat[1] + b->quat[2] * b->quat[2] + b->quat[3] * b->quat[3];
    if (!(qn > 0) || !std::isfinite(qn)) return PABD_ERR_ARG;
    int last_g = s->bodies.empty() ? 0 : s->bodies.back().group;
    if (b->group < last_g || b->group < 0 || (s->bodies.empty() && b->group != 0) || b->group > last_g + 1)
        return PABD_ERR_ARG;
    if (s->bodies.size() >= 0x7fffffffu / 4) return PABD_ERR_ARG;
    if (out_id) *out_id = (uint32_t)s->bodies.size();
    s->bodies.push_back(*b);
    return PABD_OK;
}

pabd_status pabd_add_bond(pabd_scene* s, const pabd_bond_desc* b, uint32_t* out_ids, int* n_out) {
    if (!s || !b) return PABD_ERR_ARG;
    if (s->ready) return PABD_ERR_STATE;
    const long nbod = (long)s->bodies.size();
    if (b->body_i >= (uint32_t)nbod) return PABD_ERR_ARG;
    if (b->body_j != PABD_WORLD && b->body_j >= (uint32_t)nbod) return PABD_ERR_ARG;
    if (b->body_j == b->body_i) return PABD_ERR_ARG;
    if (!(b->kappa >= 0) || !std::isfinite(b->kappa)) return PABD_ERR_ARG;
    if (b->type == PABD_ELASTIC_NL && !(b->rest_len > 0)) return PABD_ERR_ARG;
    if (b->type == PABD_SPRING && !(b->rest_len >= 0)) return PABD_ERR_ARG;
    const int i = (int)b->body_i, j = b->body_j == PABD_WORLD ? -1 : (int)b->body_j;
    const double h2 = s->desc.h * s->desc.h;
    HostBond hb{};
    hb.i = i; hb.j = j;
    hb.w = h2 * b->kappa;
    hb.p1 = b->rest_len;
    for (int k = 0; k < 3; ++k) { hb.xi[k] = b->x_i[k]; hb.xj[k] = b->x_j[k]; }
    const uint32_t first = (uint32_t)s->bonds.size();
    if (b->type == PABD_SPHERICAL || b->type == PABD_SPRING || b->type == PABD_ELASTIC_NL) {
        hb.type = b->type;
        s->bonds.push_back(hb);
        if (out_ids) out_ids[0] = first;
        if (n_out) *n_out = 1;
        return PABD_OK;
    }
    if (b->type == PABD_AL_DISTANCE) {
        if (!(b->rest_len >= 0) || !std::isfinite(b->rest_len)) return PABD_ERR_ARG;
        if (!(b->al_beta >= 0) || !std::isfinite(b->al_beta) || !std::isfinite(b->al_alpha) ||
            !std::isfinite(b->al_gamma))
            return PABD_ERR_ARG;
        hb.type = K_AL;
        hb.kappa = b->kappa;
        hb.al_beta = b->al_beta; hb.al_alpha = b->al_alpha; hb.al_gamma = b->al_gamma;
        s->bonds.push_back(hb);
        if (out_ids) out_ids[0] = first;
        if (n_out) *n_out = 1;
        return PABD_OK;
    }
    if (b->type != PABD_REVOLUTE && b->type != PABD_DRIVE) return PABD_ERR_ARG;
    double an = std::sqrt(b->axis[0] * b->axis[0] + b->axis[1] * b->axis[1] + b->axis[2] * b->axis[2]);
    if (!(an > 0)) return PABD_ERR_ARG;
    double ui[3] = {b->axis[0] / an, b->axis[1] / an, b->axis[2] / an};
    // carry directions from body i's frame into body j's frame (world for PABD_WORLD)
    double Qi[4], Ri[9], Rj[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    normalize_quat(s->bodies[i].quat, Qi);
    quat_to_mat_d(Qi, Ri);
    if (j >= 0) { double Qj[4]; normalize_quat(s->bodies[j].quat, Qj); quat_to_mat_d(Qj, Rj); }
    auto carry = [&](const double* di, double* dj) {
        double wv[3];
        for (int r = 0; r < 3; ++r) wv[r] = Ri[3 * r] * di[0] + Ri[3 * r + 1] * di[1] + Ri[3 * r + 2] * di[2];
        for (int c = 0; c < 3; ++c) dj[c] = Rj[c] * wv[0] + Rj[3 + c] * wv[1] + Rj[6 + c] * wv[2];
    };
    double uj[3];
    carry(ui, uj);
    if (b->type == PABD_REVOLUTE) {
        for (int sg = 1; sg >= -1; sg -= 2) {
            HostBond h = hb;
            h.type = K_SPHERICAL;
            for (int k = 0; k < 3; ++k) {
                h.xi[k] = b->x_i[k] + sg * b->arm * ui[k];
                h.xj[k] = b->x_j[k] + sg * b->arm * uj[k];
            }
            s->bonds.push_back(h);
        }
        if (out_ids) { out_ids[0] = first; out_ids[1] = first + 1; }
        if (n_out) *n_out = 2;
        return PABD_OK;
    }
    // drive: lever r_i orthogonal to u_i (u_i x e_m, e_m the axis least aligned with u_i)
    if (!(b->drive_period > 0)) return PABD_ERR_ARG;
    int m = 0;
    for (int k = 1; k < 3; ++k) if (std::fabs(ui[k]) < std::fabs(ui[m])) m = k;
    double e[3] = {0, 0, 0};
    e[m] = 1.0;
    double ri[3] = {ui[1] * e[2] - ui[2] * e[1], ui[2] * e[0] - ui[0] * e[2], ui[0] * e[1] - ui[1] * e[0]};
    double rn = std::sqrt(ri[0] * ri[0] + ri[1] * ri[1] + ri[2] * ri[2]);
    for (int k = 0; k < 3; ++k) ri[k] /= rn;
    double rj[3];
    carry(ri, rj);
    hb.type = K_DRIVE;
    for (int k = 0; k < 3; ++k) { hb.ui[k] = ui[k]; hb.ri[k] = ri[k]; hb.xj[k] = b->x_j[k] + b->arm * rj[k]; }
    hb.arm = b->arm; hb.amp = b->drive_amp; hb.period = b->drive_period; hb.phase = b->drive_phase;
    s->drive_ids.push_back((int)first);
    s->bonds.push_back(hb);
    if (out_ids) out_ids[0] = first;
    if (n_out) *n_out = 1;
    return PABD_OK;
}

pabd_status pabd_add_bodies(pabd_scene* s, const pabd_body_desc* b, size_t n, uint32_t* out_ids, size_t* n_done) {
    if (!s || (n && !b)) return PABD_ERR_ARG;
    if (n_done) *n_done = 0;
    s->bodies.reserve(s->bodies.size() + n);
    for (size_t k = 0; k < n; ++k) {
        pabd_status r = pabd_add_body(s, b + k, out_ids ? out_ids + k : nullptr);
        if (r != PABD_OK) return r;
        if (n_done) *n_done = k + 1;
    }
    return PABD_OK;
}

pabd_status pabd_add_bonds(pabd_scene* s, const pabd_bond_desc* b, size_t n, size_t* n_done) {
    if (!s || (n && !b)) return PABD_ERR_ARG;
    if (n_done) *n_done = 0;
    for (size_t k = 0; k < n; ++k) {
        pabd_status r = pabd_add_bond(s, b + k, nullptr, nullptr);
        if (r != PABD_OK) return r;
        if (n_done) *n_done = k + 1;
    }
    return PABD_OK;
}

pabd_status pabd_set_profiling(pabd_scene* s, int on) {
    if (!s) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    if (on && !s->prof_exec) {
        const int ne = PROF_EVENTS;
        s->prof_ev.resize(ne);
        for (int k = 0; k < ne; ++k) CK(cudaEventCreate(&s->prof_ev[k]));
        long long lc = 0;
        CK(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
        enqueue_step(s, &lc, s->prof_ev.data());
        CK(cudaStreamEndCapture(s->st, &s->prof_graph));
        CK(cudaGraphInstantiate(&s->prof_exec, s->prof_graph, 0));
    }
    s->profiling = on != 0;
    return PABD_OK;
}

pabd_status pabd_read_profile(pabd_scene* s, double* out, size_t n, int reset) {
    if (!s || !out || n > PABD_PROFILE_SLOTS) return PABD_ERR_ARG;
    for (size_t k = 0; k < n; ++k) out[k] = s->prof_acc[k];
    if (reset) for (double& v : s->prof_acc) v = 0.0;
    return PABD_OK;
}

namespace {
// one profiled step: launch the graph with event nodes, wait, accumulate stage times
pabd_status profiled_step(pabd_scene* s) {
    CK(cudaGraphLaunch(s->prof_exec, s->st));
    s->launches += s->launches_per_step;
    const std::vector<cudaEvent_t>& e = s->prof_ev;
    CK(cudaEventSynchronize(e.back()));
    auto ms = [&](int a, int b) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e[a], e[b]);
        return (double)t;
    };
    const int n_it = s->d.p.n_iter;
    double* acc = s->prof_acc;
    acc[0] += 1.0;
    acc[1] += ms(0, 1);
    acc[2] += ms(1, 2);
    acc[3] += ms(2, 3);
    acc[4] += ms(3, 4);                 // all sweeps of the step
    acc[5] += 0.0;
    acc[6] += ms(4, 5);
    acc[7] += s->fused ? 1 : (s->mode == 1 ? 2 * n_it : n_it);  // sweep-kernel launches
    acc[8] += n_it;
    acc[9] += ms(0, 5);
    int nb = 0;
    CK(cudaMemcpy(&nb, s->d.ctr + C_NBONDS, sizeof(int), cudaMemcpyDeviceToHost));
    acc[10] += nb;
    return PABD_OK;
}
}  // namespace

pabd_status pabd_step(pabd_scene* s, int nsteps) {
    if (!s || nsteps < 0) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    r = poll_status(s, false);
    if (r != PABD_OK) return r;
    for (int k = 0; k < nsteps; ++k) {
        if (s->profiling) {
            r = profiled_step(s);
            if (r != PABD_OK) return r;
            continue;
        }
        CK(cudaGraphLaunch(s->exec, s->st));
        s->launches += s->launches_per_step;
    }
    return enqueue_status(s);
}

pabd_status pabd_tune(pabd_scene* s) {
    if (!s) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    if ((s->desc.sweep_mode != 0 && s->desc.light_order != 0) || s->d.p.resid_tol > 0 || s->fused) return PABD_OK;
    r = poll_status(s, true);
    if (r != PABD_OK) return r;
    CK(cudaStreamSynchronize(s->st));
    const int mode0 = s->mode, sorted0 = s->d.light_sorted;
    r = autotune_default(s);
    if (r != PABD_OK) return r;
    CK(cudaStreamSynchronize(s->st));
    if (s->mode == mode0 && s->d.light_sorted == sorted0) return PABD_OK;
    // the step graphs were captured with the old shape: capture them again
    cudaGraphExecDestroy(s->exec);
    cudaGraphDestroy(s->graph);
    s->exec = nullptr;
    s->graph = nullptr;
    r = capture_step(s);
    if (r != PABD_OK) return r;
    if (s->prof_exec) {
        cudaGraphExecDestroy(s->prof_exec);
        cudaGraphDestroy(s->prof_graph);
        s->prof_exec = nullptr;
        s->prof_graph = nullptr;
        const bool on = s->profiling;
        r = pabd_set_profiling(s, 1);
        s->profiling = on;
        if (r != PABD_OK) return r;
    }
    return PABD_OK;
}

pabd_status pabd_step_many(pabd_scene* const* scenes, int n, const int* nsteps) {
    if (n < 0 || (n > 0 && (!scenes || !nsteps))) return PABD_ERR_ARG;
    for (int k = 0; k < n; ++k)
        if (!scenes[k] || nsteps[k] < 0) return PABD_ERR_ARG;
    // every scene enqueues on its own stream, so the scenes' steps overlap on the device; the
    // first error stops the loop (the scenes before it have been enqueued)
    for (int k = 0; k < n; ++k) {
        pabd_status r = pabd_step(scenes[k], nsteps[k]);
        if (r != PABD_OK) return r;
    }
    return PABD_OK;
}

pabd_status pabd_set_group_hold(pabd_scene* s, const uint8_t* hold, size_t n_groups) {
    if (!s) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    Dev& d = s->d;
    if (n_groups != (size_t)d.G) return PABD_ERR_ARG;
    // a held group must keep every part of its state: no drive anchors moving with the step
    // index, no augmented Lagrangian warm start
    if (d.Ndrive > 0 || d.Nal > 0) return PABD_ERR_ARG;
    if (d.G == 0) return PABD_OK;
    if (!hold) {
        CK(cudaMemsetAsync(d.group_hold, 0, d.G, s->st));
        return PABD_OK;
    }
    if (!s->hold_pinned) {
        CK(cudaMallocHost(&s->hold_pinned, (size_t)pabd_scene::HOLD_SLOTS * d.G));
        for (cudaEvent_t& e : s->hold_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const int k = s->hold_next;
    s->hold_next = (k + 1) % pabd_scene::HOLD_SLOTS;
    CK(cudaEventSynchronize(s->hold_ev[k]));  // this slot's previous copy has left the host
    unsigned char* slot = s->hold_pinned + (size_t)k * d.G;
    for (int g = 0; g < d.G; ++g) slot[g] = hold[g] ? 1 : 0;
    CK(cudaMemcpyAsync(d.group_hold, slot, d.G, cudaMemcpyHostToDevice, s->st));
    CK(cudaEventRecord(s->hold_ev[k], s->st));
    return PABD_OK;
}

pabd_status pabd_set_wait_limit(pabd_scene* s, uint32_t polls) {
    if (!s || polls == 0) return PABD_ERR_ARG;
    s->wait_polls = polls;
    if (!s->ready) return PABD_OK;  // written at finalisation
    CK(cudaMemcpyAsync(s->d.wait_limit, &s->wait_polls, sizeof(unsigned), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    return PABD_OK;
}

pabd_status pabd_step_eager(pabd_scene* s, int nsteps) {
    if (!s || nsteps < 0) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    r = poll_status(s, false);
    if (r != PABD_OK) return r;
    for (int k = 0; k < nsteps; ++k) enqueue_step(s, &s->launches);
    CK(cudaGetLastError());
    return enqueue_status(s);
}

pabd_status pabd_detect(pabd_scene* s) {
    if (!s) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    launch_step_reset(s->d, s->st, &s->launches);
    launch_drive_update(s->d, s->st, &s->launches);
    launch_collision(s->d, s->st, &s->launches);
    CK(cudaGetLastError());
    return enqueue_status(s);
}

pabd_status pabd_sync(pabd_scene* s) {
    if (!s) return PABD_ERR_ARG;
    CK(cudaStreamSynchronize(s->st));
    if (!s->ready) return PABD_OK;
    pabd_status r = poll_status(s, true);
    if (r != PABD_OK) return r;
    int bits = 0;
    CK(cudaMemcpy(&bits, s->d.ctr + C_STATUS, sizeof(int), cudaMemcpyDeviceToHost));
    s->latched |= bits;
    return status_from_bits(s->latched);
}

pabd_status pabd_read_state(pabd_scene* s, double* rows, size_t n) {
    if (!s || !rows) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    const int N = s->d.N;
    if (n != (size_t)N) return PABD_ERR_ARG;
    std::vector<float4> q(3 * N), v(N), w(N), Q(N);
    CK(cudaMemcpyAsync(q.data(), s->d.qn, sizeof(float4) * 3 * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(v.data(), s->d.vel, sizeof(float4) * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(w.data(), s->d.omg, sizeof(float4) * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(Q.data(), s->d.quat, sizeof(float4) * N, cudaMemcpyDeviceToHost, s->st));
    r = pabd_sync(s);
    for (int b = 0; b < N; ++b) {
        double* o = rows + (size_t)PABD_STATE_COLS * b;
        const float* qf = reinterpret_cast<const float*>(&q[3 * b]);
        for (int k = 0; k < 12; ++k) o[k] = qf[k];
        o[12] = Q[b].x; o[13] = Q[b].y; o[14] = Q[b].z; o[15] = Q[b].w;
        o[16] = v[b].x; o[17] = v[b].y; o[18] = v[b].z;
        o[19] = w[b].x; o[20] = w[b].y; o[21] = w[b].z;
    }
    return r;
}

pabd_status pabd_write_state(pabd_scene* s, const double* rows, size_t n) {
    if (!s || !rows) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    const int N = s->d.N;
    if (n != (size_t)N) return PABD_ERR_ARG;
    std::vector<float4> q(3 * N), v(N), w(N), Q(N);
    for (int b = 0; b < N; ++b) {
        const double* o = rows + (size_t)PABD_STATE_COLS * b;
        for (int k = 0; k < PABD_STATE_COLS; ++k) if (!std::isfinite(o[k])) return PABD_ERR_ARG;
        float* qf = reinterpret_cast<float*>(&q[3 * b]);
        for (int k = 0; k < 12; ++k) qf[k] = (float)o[k];
        Q[b] = make_float4((float)o[12], (float)o[13], (float)o[14], (float)o[15]);
        bool pin = s->bodies[b].pinned != 0;
        v[b] = pin ? make_float4(0, 0, 0, 0) : make_float4((float)o[16], (float)o[17], (float)o[18], 0.f);
        w[b] = pin ? make_float4(0, 0, 0, 0) : make_float4((float)o[19], (float)o[20], (float)o[21], 0.f);
    }
    CK(cudaMemcpyAsync(s->d.qn, q.data(), sizeof(float4) * 3 * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->d.vel, v.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->d.omg, w.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->d.quat, Q.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));  // the staging vectors go out of scope
    return PABD_OK;
}

pabd_status pabd_read_state_f32(pabd_scene* s, float* host, size_t n) {
    if (!s || !host) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    const int N = s->d.N;
    if (n != (size_t)N) return PABD_ERR_ARG;
    float* o = host;
    CK(cudaMemcpyAsync(o, s->d.qn, sizeof(float4) * 3 * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(o + 12 * (size_t)N, s->d.quat, sizeof(float4) * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(o + 16 * (size_t)N, s->d.vel, sizeof(float4) * N, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(o + 20 * (size_t)N, s->d.omg, sizeof(float4) * N, cudaMemcpyDeviceToHost, s->st));
    return PABD_OK;
}

pabd_status pabd_write_state_f32(pabd_scene* s, const float* host, size_t n) {
    if (!s || !host) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    const int N = s->d.N;
    if (n != (size_t)N) return PABD_ERR_ARG;
    const float* o = host;
    CK(cudaMemcpyAsync(s->d.qn, o, sizeof(float4) * 3 * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->d.quat, o + 12 * (size_t)N, sizeof(float4) * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->d.vel, o + 16 * (size_t)N, sizeof(float4) * N, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->d.omg, o + 20 * (size_t)N, sizeof(float4) * N, cudaMemcpyHostToDevice, s->st));
    return PABD_OK;
}

pabd_status pabd_read_bond_state(pabd_scene* s, double* host_out, size_t n_bonds) {
    if (!s || (n_bonds && !host_out)) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    const Dev& d = s->d;
    if (n_bonds != (size_t)d.Nc) return PABD_ERR_ARG;
    std::vector<float2> kl(d.Nc, make_float2(0, 0));
    if (d.Nal) {
        // the state a step ends with sits in the buffer of parity n_iter
        CK(cudaMemcpyAsync(kl.data(), (d.p.n_iter & 1) ? d.al_st1 : d.al_st0, sizeof(float2) * d.Nc,
                           cudaMemcpyDeviceToHost, s->st));
    }
    r = pabd_sync(s);
    for (int k = 0; k < d.Nc; ++k) {
        const bool al = s->bonds[k].type == K_AL;
        host_out[2 * k] = al ? kl[k].x : 0.0;
        host_out[2 * k + 1] = al ? kl[k].y : 0.0;
    }
    return r;
}

pabd_status pabd_write_bond_state(pabd_scene* s, const double* host_in, size_t n_bonds) {
    if (!s || (n_bonds && !host_in)) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    const Dev& d = s->d;
    if (n_bonds != (size_t)d.Nc) return PABD_ERR_ARG;
    if (!d.Nal) return PABD_OK;
    std::vector<float2> kl(d.Nc, make_float2(0, 0));
    for (int k = 0; k < d.Nc; ++k) {
        if (s->bonds[k].type != K_AL) continue;
        if (!std::isfinite(host_in[2 * k]) || !std::isfinite(host_in[2 * k + 1])) return PABD_ERR_ARG;
        kl[k] = make_float2((float)host_in[2 * k], (float)host_in[2 * k + 1]);
    }
    CK(cudaMemcpyAsync((d.p.n_iter & 1) ? d.al_st1 : d.al_st0, kl.data(), sizeof(float2) * d.Nc,
                       cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));  // the staging vector goes out of scope
    return PABD_OK;
}

pabd_status pabd_set_step_index(pabd_scene* s, int64_t step_index) {
    if (!s || step_index < 0) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    long long v = step_index;
    CK(cudaMemcpyAsync(s->d.step_index, &v, sizeof v, cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    return PABD_OK;
}

pabd_status pabd_read_pairs(pabd_scene* s, int32_t* out, size_t cap, size_t* n) {
    if (!s || !n) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    int np = 0;
    CK(cudaMemcpyAsync(&np, s->d.ctr + C_NPAIRS, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    r = pabd_sync(s);
    *n = (size_t)np;
    size_t m = (size_t)np < cap ? (size_t)np : cap;
    if (m && out) {
        CK(cudaMemcpy(out, s->d.pairs, sizeof(int2) * m, cudaMemcpyDeviceToHost));
    }
    return r;
}

pabd_status pabd_read_contacts(pabd_scene* s, int32_t* meta, float* data, size_t cap, size_t* n) {
    if (!s || !n) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    int c[C_COUNT];
    CK(cudaMemcpyAsync(c, s->d.ctr, sizeof c, cudaMemcpyDeviceToHost, s->st));
    r = pabd_sync(s);
    const int nk = c[C_NPC] + c[C_NGC];
    *n = (size_t)nk;
    size_t m = (size_t)nk < cap ? (size_t)nk : cap;
    if (!m || !meta || !data) return r;
    std::vector<int4> bm(m);
    std::vector<float4> xi(m), xj(m), bn(m);
    const int o = s->d.Nc;
    CK(cudaMemcpy(bm.data(), s->d.bmeta + o, sizeof(int4) * m, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(xi.data(), s->d.bxi + o, sizeof(float4) * m, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(xj.data(), s->d.bxj + o, sizeof(float4) * m, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(bn.data(), s->d.bn + o, sizeof(float4) * m, cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < m; ++k) {
        meta[3 * k] = bm[k].z; meta[3 * k + 1] = bm[k].x; meta[3 * k + 2] = bm[k].y;
        float* dd = data + 11 * k;
        dd[0] = xi[k].x; dd[1] = xi[k].y; dd[2] = xi[k].z;
        dd[3] = xj[k].x; dd[4] = xj[k].y; dd[5] = xj[k].z;
        dd[6] = bn[k].x; dd[7] = bn[k].y; dd[8] = bn[k].z;
        dd[9] = xj[k].w; dd[10] = xi[k].w;
    }
    return r;
}

pabd_status pabd_read_residual(pabd_scene* s, double* out, size_t n_groups) {
    if (!s || !out) return PABD_ERR_ARG;
    pabd_status r = finalize_scene(s);
    if (r != PABD_OK) return r;
    if (n_groups != (size_t)s->d.G) return PABD_ERR_ARG;
    r = pabd_sync(s);
    if (n_groups) CK(cudaMemcpy(out, s->d.resid_group, sizeof(double) * n_groups, cudaMemcpyDeviceToHost));
    return r;
}

pabd_status pabd_get_info(pabd_scene* s, pabd_info* info) {
    if (!s || !info) return PABD_ERR_ARG;
    pabd_status fr = finalize_scene(s);
    if (fr != PABD_OK) return fr;
    std::memset(info, 0, sizeof *info);
    info->n_bodies = (int64_t)s->bodies.size();
    info->n_groups = s->bodies.empty() ? 0 : s->bodies.back().group + 1;
    info->n_static_bonds = (int64_t)s->bonds.size();
    info->launches = s->launches;
    if (!s->ready) return PABD_OK;
    int c[C_COUNT];
    long long step = 0;
    CK(cudaMemcpyAsync(c, s->d.ctr, sizeof c, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(&step, s->d.step_index, sizeof step, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    info->n_bonds = c[C_NBONDS];
    info->n_pairs = c[C_NPAIRS];
    info->n_contacts = c[C_NPC] + c[C_NGC];
    info->step_index = step;
    info->max_pairs = s->d.cap_pairs;
    info->max_contacts = s->d.cap_contacts;
    info->graph_nodes = (int64_t)s->graph_nodes;
    info->fp64_bodies = s->fp64_bodies;
    info->device_bytes = (int64_t)s->bytes;
    info->sweep_mode = s->fused ? 3 : s->mode;
    info->sweep_lanes = s->lanes;
    info->sweep_block = s->sw_block;
    info->sweep_grid = s->sw_grid;
    info->coop_fallbacks = s->coop_fallbacks;
    info->heavy_bodies = c[C_NHEAVY];
    info->fp64_dynamic = c[C_FP64DYN];
    info->offgrid_bodies = c[C_NLARGE];
    info->light_order = s->d.light_sorted;
    info->tuned = s->tuned;
    for (int k = 0; k < 4; ++k) info->tune_sweep_ns[k] = s->tune_ns[k];
    info->last_sweeps = s->d.p.n_iter;
    if (s->d.sweep_ctl) {
        int ctl[4] = {0, 0, 0, 0};
        CK(cudaMemcpy(ctl, s->d.sweep_ctl, sizeof ctl, cudaMemcpyDeviceToHost));
        info->last_sweeps = ctl[0];
    }
    return PABD_OK;
}

pabd_status pabd_destroy_scene(pabd_scene* s) {
    if (!s) return PABD_ERR_ARG;
    cudaStreamSynchronize(s->st);
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->prof_exec) cudaGraphExecDestroy(s->prof_exec);
    if (s->prof_graph) cudaGraphDestroy(s->prof_graph);
    for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->ev_status) cudaEventDestroy(s->ev_status);
    if (s->h_status) cudaFreeHost(s->h_status);
    for (void* p : s->allocs) {
        if (s->desc.free) s->desc.free(p, s->desc.alloc_ctx);
        else cudaFree(p);
    }
    if (s->body_st) cudaStreamDestroy(s->body_st);
    if (s->hold_pinned) cudaFreeHost(s->hold_pinned);
    for (cudaEvent_t e : s->hold_ev) if (e) cudaEventDestroy(e);
    if (s->own_stream) cudaStreamDestroy(s->st);
    delete s;
    return PABD_OK;
}

}  // extern "C"
