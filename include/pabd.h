/*
 * pabd.h -- C-ABI of the GB300 (sm_103a) Projective Affine Body Dynamics library.
 *
 * One time step is Algorithm 1 of "Projective Affine Body Dynamics for Multibody Systems":
 * collision detection, the quaternion predictor, n_iter sweeps of the global solve
 * (Eq. 19, one 12x12 system per affine body, no global Hessian) and the local solve
 * (polar rotation, Sec. 4.3), then the velocity recovery of Sec. 4.4.  Every stage runs
 * in CUDA kernels on the caller's stream; the host only enqueues work.
 *
 * Conventions shared by every call:
 *   - All descriptors passed in are copied; the caller keeps ownership of its memory.
 *     Host output buffers are caller-owned and must hold the documented number of values.
 *   - Body and bond ids are dense and follow insertion order; they fix the deterministic
 *     summation order of the per-body gathers, so results are identical run to run.
 *   - Bodies of one group (an independent scene inside a batch) must be added
 *     contiguously, with non-decreasing group ids starting at 0.
 *   - pabd_add_* is legal only before the first pabd_step / pabd_detect; afterwards it
 *     returns PABD_ERR_STATE.
 *   - Kernels run asynchronously on desc.stream.  A device-side error (capacity overflow,
 *     non-finite state) is latched on the device and returned by the next call that
 *     synchronises (pabd_sync, pabd_read_*), or by pabd_step once the earlier work is done.
 *   - Every function returns PABD_ERR_ARG for NULL handles or out-of-range arguments and
 *     PABD_ERR_CUDA when a CUDA runtime call fails (see pabd_last_cuda_error).
 */
#ifndef PABD_H
#define PABD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PABD_OK = 0,
    PABD_ERR_ARG = 1,       /* invalid argument */
    PABD_ERR_OOM = 2,       /* device allocation failed */
    PABD_ERR_CAPACITY = 3,  /* more pairs / contacts than the scene's capacity (truncated) */
    PABD_ERR_DIVERGED = 4,  /* a body's state became non-finite */
    PABD_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    PABD_ERR_CUDA = 6,      /* a CUDA runtime call failed */
    PABD_ERR_STATE = 7      /* call not legal in the scene's current state */
} pabd_status;

#define PABD_WORLD 0xFFFFFFFFu

/* Bond types.  Energies Psi(d) of the distance d between the two material points
 * (Eq. 10-11, 15-17), split phi = phi+ + phi- for the semi-implicit sweep:
 *   SPHERICAL   zero-length bond, Psi = kappa d^2 / 2 (spherical joint)
 *   SPRING      Psi = kappa (d - rest_len)^2 / 2 (Eq. 26); phi+ = kappa d, phi- = -kappa l
 *   ELASTIC_NL  phi = (kappa/3)(d^3/l^2 - l): strain-stiffening, small-strain stiffness kappa;
 *               phi+ = phi'(d) d, phi- = phi(d) - phi'(d) d
 *   REVOLUTE    hinge about `axis` (body_i frame) through the pivot: two zero-length bonds
 *               at pivot +- arm * axis in both bodies' frames (creates 2 bond ids)
 *   DRIVE       zero-length bond pulling the child point pivot_j + arm * r_j to the parent
 *               point pivot_i + arm * Rot(axis, theta(t)) r_i, theta(t) = drive_amp *
 *               sin(2 pi t / drive_period + drive_phase), t the end time of the step;
 *               r_i is a fixed unit vector orthogonal to the axis.
 *   AL_DISTANCE augmented Lagrangian distance constraint (Eq. 27-29): Psi = kappa C^2/2 +
 *               lambda C, C = d - rest_len; phi+ = kappa d + max(lambda - kappa l, 0),
 *               phi- = min(lambda - kappa l, 0).  After every sweep, from the new iterate:
 *               lambda <- kappa C + lambda, kappa <- kappa + al_beta |C|; at the start of every
 *               step kappa <- max(al_gamma kappa, kappa_start), lambda <- al_alpha al_gamma
 *               lambda.  `kappa` is kappa_start; kappa starts there and lambda at 0.
 * Directions given in body_i's frame are carried into body_j's frame through the bodies'
 * orientations at the time the bond is added. */
typedef enum {
    PABD_SPHERICAL = 0,
    PABD_SPRING = 1,
    PABD_ELASTIC_NL = 2,
    PABD_REVOLUTE = 3,
    PABD_DRIVE = 4,
    PABD_AL_DISTANCE = 5
} pabd_bond_type;

typedef struct pabd_scene pabd_scene; /* opaque, owned by the library */

/* Scene parameters.  Ground and contacts are scene-level (Alg. 1 "collision detection");
 * contact bonds are rebuilt every step and are never added by the user. */
typedef struct {
    double h;                 /* time step */
    double gravity[3];
    int n_iter;               /* fixed number of global/local sweeps per step (>= 1) */
    int has_ground;           /* ground plane ground_n . y = ground_d */
    double ground_n[3];
    double ground_d;
    double mu;                /* Coulomb friction coefficient of every contact */
    double c_kappa;           /* contact stiffness kappa_c = c_kappa * min(m_i, m_j) / h^2 */
    double d_hat_rel;         /* contact distance dhat = d_hat_rel * smallest edge of the body */
    double margin;            /* absolute extra inflation of every body's contact box */
    int project;              /* 1: local solve (polar rotation); 0: affine bodies */
    int body_contacts;        /* 0: only ground contacts */
    double large_he;          /* bodies with a half extent above this skip the grid */
    int precision_policy;     /* per-body solves in FP32 (each body's 4x4 system assembled about
                                 the weighted centre of its static bonds, which removes the
                                 cancellation of stiff joints), and where still ill-conditioned
                                 (static flag: the scaled static-only system has a Cholesky pivot
                                 below 1e-2 of its diagonal; or at run time an FP32 pivot below
                                 1e-3 of its diagonal) the
                                 body's bond gather and factorisation redone in 1: double-float
                                 (two floats, ~48-bit significand, FP32 pipes; the default),
                                 2: FP64; 3: every body in double-float; 0: never (FP32 only).
                                 Other values: PABD_ERR_ARG. */
    int sweep_mode;           /* 1: a bond launch + a solve launch per sweep; 2: one launch per
                                 sweep (the solve evaluates its bonds); 3: one cooperative launch
                                 runs all n_iter sweeps; 0: the library's choice -- an autotuner
                                 times modes 1 and 2, each with the light bodies ordered by end
                                 count or not, on the state at creation (pabd_tune repeats it on
                                 a later state) and keeps the fastest.  All modes and orders give
                                 the same results for the same sweep_lanes */
    int sweep_lanes;          /* lanes per body in the per-body solve: 1, 2, 4, 8 or 16; 0 = from
                                 the scene: the largest of 16, 8, 4, 2, 1 with lanes * N <= 2^17,
                                 but 2 instead of 1 when N <= 2^18 and fewer than half the bodies
                                 are flagged for the extended solve.  Fixes the summation order
                                 (results depend on it, not on the block / grid sizes, which the
                                 library autotunes).  A body with more than 64 bond ends is
                                 summed by a warp (up to 256 ends) or a block of 128 threads in
                                 every mode. */
    size_t max_pairs;         /* capacities: at most 16 M pairs, 0 = 16 per body (clamped to 16 M) */
    size_t max_contacts;      /* at most 60 M, 0 = 32 per body (clamped to 60 M); at most 8 M bodies.
                                 Exceeding one in a step latches PABD_ERR_CAPACITY. */
    double resid_tol;         /* Sec. 4.2 stopping rule.  0: every step runs n_iter sweeps.  > 0:
                                 each scene (group) stops after the first sweep whose residual
                                 sqrt(sum |q^{k+1} - q^k|^2) is at most resid_tol (at most n_iter
                                 sweeps); the loop ends on the device (a conditional graph node)
                                 once every scene has stopped.  Runs the one-launch-per-sweep
                                 mode; not with AL_DISTANCE bonds (PABD_ERR_ARG). */
    int broadphase;           /* 0: uniform grid hash (cell = widest grid box of the step under a
                                 cap chosen at creation; in scenes of very different widths, three
                                 grid levels with caps 1, 4 and 16 times it, and wider boxes tested
                                 against all bodies); 1: linear BVH over the boxes' Morton codes
                                 (Sec. 5).  Both give the same pair list. */
    int light_order;          /* bodies with at most 64 bond ends, in each sweep: 1 ordered every
                                 step by (extended path or not, end count, most ends first), so a
                                 warp's lanes walk slices of one length down one path and the
                                 longest warps start first; 2 in body order; 0 the
                                 library's choice (timed with sweep_mode 0, else ordered).  Other
                                 values: PABD_ERR_ARG.  Results do not depend on it. */
    void* stream;             /* cudaStream_t on which all work is enqueued (NULL: default) */
    /* optional device allocator (e.g. a framework's caching allocator); NULL: cudaMalloc */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* alloc_ctx;
} pabd_scene_desc;

/* A box body: half extents he, material origin at the centre of mass (so the generalised
 * mass of Thm 4.1 is block diagonal with Pi_0 = m diag(he^2)/3).  quat is (x, y, z, w). */
typedef struct {
    double he[3];
    double mass;
    double c[3];
    double quat[4];
    double v[3];
    double omega[3];          /* world frame */
    int pinned;               /* kinematic: never moves, infinite mass */
    int group;                /* independent scene id (no contacts across groups) */
} pabd_body_desc;

typedef struct {
    int type;                 /* pabd_bond_type */
    uint32_t body_i, body_j;  /* body_j may be PABD_WORLD (then x_j is a world point) */
    double x_i[3], x_j[3];    /* material points (pivots for REVOLUTE / DRIVE) */
    double axis[3];           /* REVOLUTE / DRIVE axis in body_i's frame */
    double kappa, rest_len, arm;
    double drive_amp, drive_period, drive_phase;
    double al_beta, al_alpha, al_gamma;  /* AL_DISTANCE parameters */
} pabd_bond_desc;

/* State rows exchanged with the host: 22 doubles per body,
 * c[3], A[9] (row-major, rows a_k of Eq. 1), quat[4] (x, y, z, w), v[3], omega[3]. */
#define PABD_STATE_COLS 22

typedef struct {
    int64_t n_bodies, n_groups, n_static_bonds, n_bonds, n_pairs, n_contacts;
    int64_t step_index;
    int64_t max_pairs, max_contacts;
    int64_t graph_nodes;      /* kernel + memset nodes of one captured step */
    int64_t launches;         /* kernels launched by this scene so far */
    int64_t fp64_bodies;      /* bodies whose solve is statically flagged for the extended type */
    int64_t device_bytes;     /* device memory held by the scene */
    int64_t sweep_mode, sweep_lanes, sweep_block, sweep_grid;  /* sweep mode (1, 2, 3) and the
                                 fused sweep's launch shape */
    int64_t coop_fallbacks;   /* steps whose cooperative sweep launch was refused and ran as
                                 two launches per sweep instead */
    int64_t heavy_bodies;     /* bodies of the last step with more than 64 bond ends, each
                                 gathered and solved by a warp (up to 256 ends) or a block of
                                 128 threads */
    int64_t fp64_dynamic;     /* bodies that took the extended-precision redo in the last sweep
                                 of the last step because of a small FP32 pivot */
    int64_t last_sweeps;      /* sweeps the last step ran (n_iter unless resid_tol ended it) */
    int64_t offgrid_bodies;   /* bodies the last step's grid broad phase took off the grid
                                 (flagged large, or a box wider than the cell cap) */
    int64_t light_order;      /* 1: each sweep takes the light bodies ordered by (path, end
                                 count), rebuilt every step; 0: in body order */
    int64_t tuned;            /* 1 if sweep_mode and light_order were chosen by timing (sweep_mode
                                 0 in the descriptor, no resid_tol, no AL_DISTANCE bonds) */
    int64_t tune_sweep_ns[4]; /* the autotuner's time per sweep for each candidate (the fastest of
                                 four timed passes over n_iter sweeps), nanoseconds: one
                                 launch per sweep ordered / in body order, a bond and a solve
                                 launch per sweep ordered / in body order (0: not tuned) */
} pabd_info;

/* Create an empty scene on the current CUDA device.  *out receives the handle. */
pabd_status pabd_create_scene(const pabd_scene_desc* desc, pabd_scene** out);

/* Append one body; *out_id (may be NULL) receives its id. */
pabd_status pabd_add_body(pabd_scene* s, const pabd_body_desc* b, uint32_t* out_id);

/* Append one user bond. out_ids (capacity >= 2, may be NULL) receives the internal bond
 * ids it expands to; *n_out (may be NULL) their number (REVOLUTE: 2, others: 1). */
pabd_status pabd_add_bond(pabd_scene* s, const pabd_bond_desc* b, uint32_t* out_ids, int* n_out);

/* Bulk forms of pabd_add_body / pabd_add_bond for n descriptors in an array; out_ids (may be
 * NULL) receives the n body ids, or the internal bond ids (2 per REVOLUTE) up to out_cap.
 * Stops at the first invalid descriptor and returns its error; *n_done (may be NULL) is the
 * number of descriptors added before it. */
pabd_status pabd_add_bodies(pabd_scene* s, const pabd_body_desc* b, size_t n, uint32_t* out_ids, size_t* n_done);
pabd_status pabd_add_bonds(pabd_scene* s, const pabd_bond_desc* b, size_t n, size_t* n_done);

/* Advance nsteps time steps (asynchronous on desc.stream; one CUDA graph launch each). */
pabd_status pabd_step(pabd_scene* s, int nsteps);

/* Same work launched kernel by kernel without the CUDA graph (the plain path). */
pabd_status pabd_step_eager(pabd_scene* s, int nsteps);

/* Re-run the sweep autotuner of a scene created with sweep_mode 0 on its current state (for
 * instance once a pile has landed, when its contacts are in place) and re-capture its step
 * graph if the choice changed.  Synchronises the scene's stream.  The trial sweeps change no
 * state; the pair and contact lists afterwards are those of the current state.  Returns
 * PABD_OK without tuning for scenes whose shape is fixed (sweep_mode 1-3, resid_tol > 0,
 * AL_DISTANCE bonds); a latched device error is returned first. */
pabd_status pabd_tune(pabd_scene* s);

/* Batched form of pabd_step over n scenes: scene k advances nsteps[k] steps (0 allowed).
 * Every scene enqueues on its own stream, so their steps overlap on the device.  The call
 * checks every handle and count first (PABD_ERR_ARG, nothing enqueued); after that the first
 * scene whose pabd_step fails stops the loop and its status is returned (the scenes before it
 * have been enqueued).  Independent scenes that share one launch per sweep are the groups of
 * one scene (pabd_body_desc.group); this call serves scenes that must stay separate (their
 * own streams, capacities or parameters). */
pabd_status pabd_step_many(pabd_scene* const* scenes, int n, const int* nsteps);

/* Hold groups still: from the next step on (ordered on the scene's stream), every body of a
 * group g with hold[g] != 0 keeps its state (q, v, omega, Q) through each step, as if pinned
 * for the step, while the other groups step; a held group's bodies still take part in
 * collision detection, whose contacts stay within the group.  hold has n_groups bytes
 * (n_groups must equal pabd_info.n_groups); NULL releases every group.  A group's step
 * depends only on its own bodies and bonds, so a group stepped k times among held groups ends
 * where it ends stepped k times alone with the same sweep_lanes.  The mask is copied through
 * the library's pinned staging, so the caller may reuse its buffer at once.  Scenes with
 * DRIVE or AL_DISTANCE bonds (whose state moves with the step) return PABD_ERR_ARG.  This is
 * how a server steps only the resident scenes that have work, packed as groups of one scene. */
pabd_status pabd_set_group_hold(pabd_scene* s, const uint8_t* hold, size_t n_groups);

/* Bound of the device-side waits of the scene (the grid barrier between the sweeps of the
 * fused persistent sweep, sweep_mode 3): a wait gives up after `polls` polls (default 2^24,
 * about a second), latches PABD_ERR_TIMEOUT and ends its kernel, which the next
 * synchronising call returns; the scene's later steps are not trustworthy.  Tests shorten the
 * bound to check that a wait that runs out is reported.  polls == 0 is PABD_ERR_ARG. */
pabd_status pabd_set_wait_limit(pabd_scene* s, uint32_t polls);

/* Stage timing.  With profiling on, pabd_step launches a second captured graph that also
 * records CUDA events at the stage boundaries, waits for each step and accumulates the
 * times (milliseconds) read back by pabd_read_profile into PABD_PROFILE_SLOTS doubles:
 *   [0] steps, [1] drives + collision detection, [2] CSR build, [3] predictor,
 *   [4] all sweeps (bond + solve of every iteration), [5] unused (0), [6] finalize +
 *   residual, [7] sweep-kernel launches, [8] sweeps, [9] whole steps, [10] sum over steps
 *   of the bond count.
 * reset != 0 clears the accumulators after reading. */
#define PABD_PROFILE_SLOTS 11
pabd_status pabd_set_profiling(pabd_scene* s, int on);
pabd_status pabd_read_profile(pabd_scene* s, double* out, size_t n, int reset);

/* Collision detection only, on the current state (fills pairs and contacts). */
pabd_status pabd_detect(pabd_scene* s);

/* Wait for the scene's stream; returns the first latched device error, if any. */
pabd_status pabd_sync(pabd_scene* s);

/* Copy the state of all bodies to / from host rows (n_bodies x PABD_STATE_COLS doubles).
 * Reads synchronise; writes are ordered on the stream before later steps. */
pabd_status pabd_read_state(pabd_scene* s, double* host_rows, size_t n_bodies);
pabd_status pabd_write_state(pabd_scene* s, const double* host_rows, size_t n_bodies);

/* The same state in the device's own single-precision layout, for callers that move it every
 * step (no conversion, no validation, asynchronous): host holds 24 * n_bodies floats, the four
 * device arrays one after the other -- q (12 floats per body: c, then A row-major), then the
 * quaternion (x, y, z, w), then v (x, y, z, unused), then omega (x, y, z, unused), each
 * n_bodies rows.  Both calls only enqueue copies on the scene's stream and return: the host
 * buffer must stay untouched until the stream has passed them (pabd_sync), and should be
 * page-locked for the copies to run at full speed.  v and omega of pinned bodies are ignored
 * by the step; a non-finite value written surfaces as PABD_ERR_DIVERGED after the next step.
 * n_bodies must equal the scene's body count (else PABD_ERR_ARG). */
pabd_status pabd_read_state_f32(pabd_scene* s, float* host, size_t n_bodies);
pabd_status pabd_write_state_f32(pabd_scene* s, const float* host, size_t n_bodies);

/* Set the index n of the next step (its end time is (n + 1) h, used by DRIVE bonds);
 * ordered on the stream like a state write. */
pabd_status pabd_set_step_index(pabd_scene* s, int64_t step_index);

/* Augmented Lagrangian state of the static bonds (internal ids, as pabd_add_bond returns
 * them; n_bonds must equal pabd_info.n_static_bonds, else PABD_ERR_ARG): (kappa, lambda) per
 * bond, 2 doubles each, zeros for other bond types -- the values the last step ended with,
 * which the next step warm-starts from (Eq. 29).  Held on the device in FP32.  Both calls
 * finalize the scene if needed and synchronise its stream; a write ignores the entries of
 * other bond types and rejects non-finite values (PABD_ERR_ARG, nothing written). */
pabd_status pabd_read_bond_state(pabd_scene* s, double* host_out, size_t n_bonds);
pabd_status pabd_write_bond_state(pabd_scene* s, const double* host_in, size_t n_bonds);

/* Broad-phase pairs of the last detection: *n receives the count; up to cap (i, j)
 * int32 pairs (i < j, sorted) are written to host_pairs. */
pabd_status pabd_read_pairs(pabd_scene* s, int32_t* host_pairs, size_t cap, size_t* n);

/* Contact bonds of the last detection, in bond order: meta (type 5 = body-body, 6 =
 * ground; i; j or -1) as 3 int32 per contact, data as 11 float per contact:
 * x_i[3], x_j[3] (material point of j, or world anchor), N[3], dhat, w = h^2 kappa_c. */
pabd_status pabd_read_contacts(pabd_scene* s, int32_t* host_meta, float* host_data, size_t cap, size_t* n);

/* Per-group residual sqrt(sum_i |q_i^{k+1} - q_i^k|^2) of the last sweep of the last step. */
pabd_status pabd_read_residual(pabd_scene* s, double* host_out, size_t n_groups);

pabd_status pabd_get_info(pabd_scene* s, pabd_info* info);

/* Release all device memory of the scene (synchronises its stream). */
pabd_status pabd_destroy_scene(pabd_scene* s);

/* Broad phase for callers that cannot allocate device memory.  Some callers must not call
 * cudaMalloc or cudaFree: real-time loops that may not block on the allocator (both calls can
 * synchronise the device), applications whose device memory is owned and handed out by
 * another runtime or memory pool, and plug-ins embedded in a host program that holds the
 * GPU's memory budget.  This call allocates nothing: its scratch (hash buckets, per-body
 * counts and offsets, the scan's block sums) is a static device array inside the library,
 * sized for PABD_NOALLOC_MAX_BODIES bodies (about 1.5 MB) and held by every GPU that loads
 * the library until the process exits.  The paper has no counterpart of this entry point; it
 * returns the same sorted pair list as pabd_detect / pabd_read_pairs for a scene with these
 * bodies and no user bonds.
 *
 * Inputs (device pointers, n_bodies rows each): q 12 floats per body (c, then A row-major),
 * vel 4 floats per body (v, unused), he 4 floats per body (half extents, unused), group and
 * flags one int32 per body (flags bit 0 = pinned; no other bit may be set).  h, margin and
 * d_hat_rel are the scene parameters of pabd_scene_desc.  Outputs (device): *n_pairs_out the
 * number of overlapping pairs found; pairs_out receives min(found, max_pairs) (i, j) int32
 * pairs, i < j, sorted.  When more than max_pairs are found the list is cut: the pairs written
 * are max_pairs of the found ones, sorted, but not necessarily the first max_pairs of the
 * full sorted list.
 * Asynchronous on `stream` (NULL: the legacy default stream).  Returns PABD_ERR_ARG for
 * null pointers, n_bodies < 0 or n_bodies > PABD_NOALLOC_MAX_BODIES.  The first call in a
 * CUDA context looks up the device address of the static array (with that context's device
 * current) and should come before any stream capture; later calls in the same context only
 * enqueue memsets and kernels.  Every call reuses the same array and keeps nothing from the
 * previous call: it clears the buckets and counters it needs first.  Calls that overlap on the
 * GPU (on different streams, or from several threads) race on that array and must be
 * serialised by the caller. */
#define PABD_NOALLOC_MAX_BODIES 16384
pabd_status pabd_broadphase_noalloc(const float* q, const float* vel, const float* he, const int32_t* group,
                                    const int32_t* flags, int32_t n_bodies, double h, double margin,
                                    double d_hat_rel, int32_t* pairs_out, int32_t max_pairs,
                                    int32_t* n_pairs_out, void* stream);

const char* pabd_status_str(pabd_status st);

/* Text of the last CUDA runtime error seen by the library in this thread. */
const char* pabd_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PABD_H */
