/*
 * klb.h -- C ABI of the GB300 (sm_103a) finite-difference lattice Boltzmann
 * time step of Gan, Xu, Zhang & Li, "Lattice Boltzmann study on
 * Kelvin-Helmholtz instability: the roles of velocity and density gradients"
 * (arXiv:1010.4124).
 *
 * The method (Secs. II-III of the paper): 19 discrete velocities (a rest
 * velocity plus three rings of six directions, Eq. 5); the truncated
 * equilibrium f^(0) from the moments rho, u, T through the closed-form global
 * coefficients F_k(T) (Eqs. 10, 28, 44-46); the convection term v . grad f by
 * fifth-order WENO finite differences of F = v_alpha f, upwinded by the sign of
 * each velocity component (Eqs. 48-55 and the mirror procedure that follows
 * them); BGK relaxation and forward-Euler time integration (Eq. 47); ghost-node
 * boundaries: periodic, outflow by zeroth-order extrapolation (Eqs. 63-64) and
 * fixed equilibrium (Eqs. 57-58).
 *
 * Conventions of every entry point:
 *  - Return value: KLB_OK (0) or a negative KLB_E_* code; klb_last_error()
 *    gives a one-line message for the handle's last failure.
 *  - Host-facing arrays are always double, C order, owned by the caller.
 *    Macroscopic fields are [ny][nx] (x fastest); a distribution array is
 *    [19][ny][nx].  `on_device` = 1 means the pointer is a CUDA device pointer
 *    (e.g. from torch), 0 means host memory (pinned memory gives the fastest
 *    copies).
 *  - The library owns all device memory of a handle (two copies of f plus
 *    small buffers), allocated in klb_create and freed in klb_destroy.
 *  - Work is enqueued on the handle's stream; calls that return data to the
 *    caller synchronise that stream.  Errors raised by kernels (a bounded wait
 *    that ran out, a non-finite state) surface at the next synchronising call.
 *  - A handle is not thread-safe; separate handles are independent.
 *
 * Velocity index q: 0 is the rest velocity; q = 1 + 6(k-1) + (i-1) is ring
 * k = 1..3 (speed v[k-1]) in direction i = 1..6 at angle 60 i degrees.
 */
#ifndef KLB_H
#define KLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KLB_OK 0
#define KLB_E_INVAL (-1)          /* an argument is out of range */
#define KLB_E_NOMEM (-2)          /* device or host allocation failed */
#define KLB_E_CUDA (-3)           /* a CUDA runtime call failed */
#define KLB_E_NONFINITE (-4)      /* a sampled state had rho or T non-finite or <= 0 */
#define KLB_E_DEVICE_TIMEOUT (-5) /* a bounded device-side wait ran out */
#define KLB_E_STATE (-6)          /* call out of order (e.g. step before init) */
#define KLB_E_IO (-7)             /* file I/O failed (save / load) */
#define KLB_E_BOUNDS (-8)         /* bounds-checked build (libklb_checked.so) only: a kernel formed
                                   * an index outside its buffer; the access was skipped */

/* Boundary kinds of Sec. III.B and IV: periodic wrap, outflow (zeroth-order
 * extrapolation, Eqs. 63-64), fixed equilibrium ghosts (Eq. 57).  KLB_BC_HALO
 * (y sides only) marks a side whose three ghost rows another grid supplies:
 * the step neither writes nor reads anything else there; the slab engine
 * (klb_slabs_*) fills them from the neighbouring slab before every step. */
typedef enum { KLB_BC_PERIODIC = 0, KLB_BC_OUTFLOW = 1, KLB_BC_FIXED_EQ = 2, KLB_BC_HALO = 3 } klb_bc;
typedef enum { KLB_FP32 = 0, KLB_FP64 = 1 } klb_prec;

/* Convection scheme of the face fluxes h (Eq. 47).  The paper's method is
 * WENO5 (Sec. III.A, Eqs. 48-55); it compares it near the Sod shock with three
 * lower-order schemes (Sec. III.B, Fig. 2), which it names without formulas:
 * with c the upwind node's value F_I, b = F_{I-1}, d = F_{I+1} (mirrored for a
 * negative velocity component):
 *   KLB_UPWIND1  h = c                                  (first-order upwind)
 *   KLB_UPWIND2  h = c + (c - b) / 2                    (second-order upwind)
 *   KLB_TVD2     h = c + minmod(c - b, d - c) / 2       (second-order TVD) */
typedef enum { KLB_WENO5 = 0, KLB_UPWIND1 = 1, KLB_UPWIND2 = 2, KLB_TVD2 = 3 } klb_scheme;

/* Problem statement of one run (Sec. III.B, Sec. IV of the paper). */
typedef struct {
    int32_t nx, ny;           /* interior nodes in x (fastest) and y; >= 1 each */
    double dx, dy;            /* node spacing, > 0 */
    double dt;                /* time step, > 0 */
    double tau;               /* BGK relaxation time, > 0 */
    double v[3];              /* ring speeds v_1, v_2, v_3: distinct, > 0; the paper uses 1, 2, 3 */
    int32_t bc_x_lo, bc_x_hi; /* klb_bc of the x = 0 and x = nx-1 sides; periodic must pair */
    int32_t bc_y_lo, bc_y_hi; /* same for y */
    int32_t precision;        /* klb_prec: storage and arithmetic type of f on the device */
    int32_t sample_every;     /* diagnostics every n steps (0 = off); see klb_diagnostics */
    int32_t diag_capacity;    /* samples kept on the device (0 = 4096); older samples are dropped */
    double eps;               /* WENO epsilon of Eq. 52; 0 selects the paper's 1e-6.  FP32
                               * WENO5 needs 3/4 eps / max(v)^2 >= 2e-19 (the squared
                               * reciprocals of the smoothness indicators stay normal
                               * FP32 numbers) and keeps
                               * its weights exact while the smallest indicator of a face
                               * is below 9e18 (differences of f up to about 1e9) */
    void* stream;             /* cudaStream_t to enqueue on; NULL = a stream owned by the handle */
    int32_t scheme;           /* klb_scheme: convection scheme of the x and y fluxes (default WENO5) */
} klb_params;

typedef struct klb klb_t;

/* Fill `p` with the defaults: v = {1,2,3}, all sides periodic, FP32,
 * sample_every 0, eps 1e-6, NULL stream, WENO5.  nx, ny, dx, dy, dt, tau stay 0 and
 * must be set by the caller. */
void klb_params_default(klb_params* p);

/* Validate `p`, allocate the device state on the current CUDA device and
 * return a handle in *out.  Ownership: the caller destroys it with
 * klb_destroy.  Logs (stderr) a warning when dt/tau > 2 or the convective CFL
 * number max(v) dt / min(dx, dy) > 0.03 (forward Euler with WENO5 then grows
 * linearly unstable modes).  Errors: KLB_E_INVAL (also for an FP32 grid of
 * 2^24 tiles or more, about 2^32 nodes, and for an FP32 WENO5 eps below the
 * range given at klb_params.eps), KLB_E_NOMEM, KLB_E_CUDA. */
int klb_create(const klb_params* p, klb_t** out);

/* Free every resource of the handle.  NULL-safe. */
void klb_destroy(klb_t* h);

/* Initial state (Sec. III.B Eq. 56, Sec. IV Eqs. 59-62): f := f^(0)(rho, u, T)
 * at every node, ghost nodes filled, and the fixed-equilibrium ghost values of
 * Eq. 57 taken from the edge nodes of these fields.  Fields are [ny][nx]
 * doubles; T > 0 and rho > 0.  Resets the step counter and the diagnostics
 * series (the state at step 0 is sampled when sample_every > 0).  Enqueued
 * on the handle's stream: host fields in pinned (page-locked, mapped) memory
 * are read by the kernel directly across the host link, other host fields
 * are first copied to device staging; either way the host arrays must stay
 * unchanged until the stream has passed the call (klb_sync).  Errors:
 * KLB_E_INVAL (NULL pointer), KLB_E_CUDA. */
int klb_init_fields(klb_t* h, const double* rho, const double* ux, const double* uy,
                    const double* T, int on_device);

/* Overwrite the interior distribution with f[19][ny][nx] (doubles, converted
 * to the handle's precision) and refresh the periodic / outflow ghost nodes.
 * Fixed-equilibrium ghosts keep the values set by klb_init_fields.  Requires a
 * prior klb_init_fields (KLB_E_STATE otherwise). */
int klb_set_f(klb_t* h, const double* f, int on_device);

/* Copy the interior distribution to f[19][ny][nx] (doubles).  Synchronises. */
int klb_get_f(klb_t* h, double* f, int on_device);

/* Enqueue n time steps (Eq. 47) on the handle's stream and return without
 * waiting.  Each step is one launch of the fused step kernel (ghost images of
 * the new state are written by the same launch).  FP32 WENO5 handles replay
 * runs of steps (at least 64, whole sampling periods, starting at a sampling
 * point) from CUDA graphs captured on first use, one per buffer parity and
 * sampling state; the results are bitwise those of one launch per step.
 * n >= 0.  Errors: KLB_E_STATE (no klb_init_fields yet), KLB_E_INVAL,
 * KLB_E_CUDA. */
int klb_step(klb_t* h, int64_t n);

/* Wait for the handle's stream; report device-side errors recorded since the
 * last synchronising call (KLB_E_DEVICE_TIMEOUT, KLB_E_NONFINITE; KLB_E_BOUNDS
 * in the bounds-checked build). */
int klb_sync(klb_t* h);

/* Macroscopic fields (Eq. 10) of the current state into caller-owned [ny][nx]
 * double arrays: rho, u_x, u_y and T (P = rho T).  Any pointer may be NULL to
 * skip that field.  Host arrays in pinned memory are written by the kernel
 * directly, others through device staging.  Synchronises. */
int klb_moments(klb_t* h, double* rho, double* ux, double* uy, double* T, int on_device);

/* Averaged density profile of the mixing layer (Sec. IV.A, Fig. 4): the
 * density averaged along the interface, which in this library lies along x
 * (the periodic axis of the Kelvin-Helmholtz set-up):
 *   out[j] = (1/nx) sum_i rho(x_i, y_j),  j = 0 .. ny-1,  rho = sum_q f_q,
 * summed in FP64 in a fixed order.  out is caller-owned, ny doubles, on the
 * host (on_device = 0) or the device (on_device = 1).  Synchronises.  Errors:
 * KLB_E_INVAL, KLB_E_STATE (before klb_init_fields), KLB_E_CUDA. */
int klb_mean_density(klb_t* h, double* out, int on_device);

/* Diagnostics series (Sec. IV): one record of 7 doubles per sample, taken on
 * the states after 0, s, 2s, ... steps (s = sample_every):
 *   [0] sum rho, [1] sum rho u_x, [2] sum rho u_y, [3] sum rho (T + |u|^2/2),
 *   [4] max |u_y|, [5] max rho u_y^2 / 2, [6] sum rho u_y^2 / 2,
 * sums over interior nodes (unweighted), accumulated in FP64 in a fixed order
 * (deterministic); an FP32 grid forms each node's values in FP32 and sums
 * them per thread as compensated FP32 pairs before the FP64 reduction.  Copies min(cap, available) records, oldest first, into
 * out[cap][7] (host) and the number copied into *count.  Synchronises; returns
 * KLB_E_NONFINITE if any sampled state had rho or T non-finite or <= 0. */
int klb_diagnostics(klb_t* h, double* out, int64_t cap, int64_t* count);

/* Number of steps taken since klb_init_fields. */
int64_t klb_step_count(const klb_t* h);

/* Checkpoint / resume: write (or read) the parameters, the step counter, the
 * diagnostics series and both the interior and ghost nodes of f in the
 * handle's precision, so that a resumed run continues bitwise identically.
 * klb_load requires a handle created with the same nx, ny and precision.
 * Errors: KLB_E_IO, KLB_E_INVAL (mismatch), KLB_E_CUDA. */
int klb_save(klb_t* h, const char* path);
int klb_load(klb_t* h, const char* path);

/* Message of the handle's last error ("" if none); with h == NULL, the last
 * error of a failed klb_create on this thread. */
const char* klb_last_error(const klb_t* h);

/* Device layout of f, for profilers and tests: base pointer of the current
 * state, row pitch and plane stride in elements, and the offsets (gx, gy) of
 * interior node (0,0) inside a plane.  Element (q, j, i) of the interior is
 * at base[q*plane + (j+gy)*pitch + (i+gx)]. */
int klb_layout(const klb_t* h, const void** base, int64_t* pitch, int64_t* plane,
               int32_t* gx, int32_t* gy);

/* Kernel launches enqueued by this handle since klb_create (every kernel the
 * library launched on its stream). */
int64_t klb_launch_count(const klb_t* h);

/* Kernel variant (tile shape) of the FP32 step: 0 = tiles of 32 x 16 nodes,
 * one CTA of 16 warps per SM; 1 = tiles of 32 x 8 nodes, two CTAs of 8 warps
 * per SM.  Every node is computed by the same arithmetic in both, so the
 * states are bitwise identical; only the speed differs (the diagnostics sums
 * may differ in the last bits, being reduced in another order).  A new FP32
 * handle starts with the shape measured faster for its size: 1 up to 40
 * sixteen-row tiles per SM (about 2048 x 1024 nodes on 152 SMs), 0 beyond.
 * The FP64 step has variant 0 only.  Synchronises the handle's stream.
 * Errors: KLB_E_INVAL or KLB_E_CUDA, after which the handle keeps its tile
 * shape; KLB_E_STATE when putting the old shape back failed as well: the
 * handle then refuses klb_step (and batches holding it refuse to step) and
 * should be destroyed. */
int klb_set_variant(klb_t* h, int variant);
int klb_get_variant(const klb_t* h);

/* Self-test of the bounds-checked debug build (libklb_checked.so, compiled
 * with -DKLB_CHECK_BOUNDS, in which every kernel compares each global index it
 * forms with the extent of its buffer, skips an access out of range and
 * raises a flag that klb_sync reports as KLB_E_BOUNDS; nothing traps):
 * enqueues one guarded store one element past the end of the handle's FP32
 * state buffer, which the guard skips and flags, so that the next klb_sync
 * returns KLB_E_BOUNDS (and clears the flag).  The ordinary library has no
 * guards and refuses the call (KLB_E_INVAL) without launching anything.
 * This is a debugging aid with no counterpart in the paper. */
int klb_debug_bounds_probe(klb_t* h);

/* ---------------------------------------------------------------------------
 * Slab decomposition (the domain decomposition of Eq. 47 over the grid of
 * Sec. III.B that a step spread over several devices would use; here all
 * slabs live on the current device).  The grid of `p` is cut in y into n
 * slabs of contiguous rows; each slab is a grid of its own (klb_t with its
 * own buffers) whose sides between slabs are KLB_BC_HALO.  Every step first
 * copies, in one kernel, the three rows next to each cut (19 planes, interior
 * columns) into the neighbouring slab's ghost rows (with a periodic y, across
 * the domain's ends too), then steps every slab: the result is bitwise that
 * of the whole grid.  Slabs hold at least 3 rows (the depth of the ghost
 * layer).  Errors as for klb_create / klb_step; the message of a failed call
 * is in klb_slabs_last_error.
 * ------------------------------------------------------------------------- */
typedef struct klb_slabs klb_slabs_t;

/* Host only (no device work): the rows of slab k of n over ny rows, as
 * balanced as possible (the first ny % n slabs one row more): row0[k] and
 * rows[k], arrays of n entries owned by the caller.  KLB_E_INVAL when n < 1
 * or a slab would hold fewer than 3 rows. */
int klb_slab_partition(int32_t ny, int32_t n, int32_t* row0, int32_t* rows);

/* Host only: the slabs whose rows fill the ghost rows of slab k -- *below
 * supplies rows -3..-1, *above rows rows[k]..rows[k]+2 -- or -1 where the
 * side is the domain's own (outflow, fixed-equilibrium) side.  With a
 * periodic y the neighbours wrap (n = 1: the slab is its own neighbour and
 * keeps the periodic sides). */
int klb_slab_neighbors(const klb_params* p, int32_t n, int32_t k, int32_t* below, int32_t* above);

/* n slabs of the grid of p (p->bc_y_* are the domain's y sides). */
int klb_slabs_create(const klb_params* p, int32_t n, klb_slabs_t** out);
void klb_slabs_destroy(klb_slabs_t* s);
/* The whole grid's initial fields [ny][nx] (host or device): each slab takes
 * its rows. */
int klb_slabs_init_fields(klb_slabs_t* s, const double* rho, const double* ux, const double* uy, const double* T,
                          int on_device);
/* n steps of every slab (asynchronous, on the slabs' shared stream). */
int klb_slabs_step(klb_slabs_t* s, int64_t n);
/* The whole grid's distribution [19][ny][nx] assembled from the slabs
 * (synchronises). */
int klb_slabs_get_f(klb_slabs_t* s, double* f, int on_device);
/* Slab k's handle (owned by the slab set) or NULL. */
klb_t* klb_slabs_member(klb_slabs_t* s, int32_t k);
const char* klb_slabs_last_error(const klb_slabs_t* s);

/* ---------------------------------------------------------------------------
 * Batched engine (the D_v x D_rho sweeps of Sec. IV).  A batch holds n FP32
 * grids that share the step constants (dx, dy, dt, tau, v, eps) but may differ
 * in size, boundaries, initial fields and diagnostics cadence.  One launch of
 * the persistent step kernel advances every grid by one step (the grids' tiles
 * form one work list, so uneven sizes balance over the GPU); klb_batch_step
 * replays the step loop from a CUDA graph of whole sampling periods.
 * ------------------------------------------------------------------------- */
typedef struct klb_batch klb_batch_t;

/* Create a batch of n grids (params p[0..n-1]; precision must be FP32; the
 * stream of p[0], or a stream owned by the batch when NULL, serves all of
 * them).  Errors: KLB_E_INVAL (n < 1 or n > 256, differing constants),
 * KLB_E_NOMEM, KLB_E_CUDA; the message is klb_batch_last_error(NULL). */
int klb_batch_create(const klb_params* p, int n, klb_batch_t** out);
void klb_batch_destroy(klb_batch_t* b); /* NULL-safe; destroys the members */
int klb_batch_size(const klb_batch_t* b);

/* Borrowed handle of member i (0 <= i < n), owned by the batch: use it for
 * klb_init_fields, klb_set_f, klb_get_f, klb_moments, klb_diagnostics,
 * klb_save.  Do not destroy it and do not step it alone (klb_batch_step
 * requires all members at the same step).  NULL if i is out of range. */
klb_t* klb_batch_member(klb_batch_t* b, int i);

/* Enqueue n steps of every member and return without waiting.  Diagnostics
 * of each member are sampled on its own cadence, as klb_step does.  Errors:
 * KLB_E_STATE (a member not initialised, or members at different steps),
 * KLB_E_INVAL, KLB_E_CUDA. */
int klb_batch_step(klb_batch_t* b, int64_t n);

/* Wait for the batch's stream; report device-side errors of the batched step
 * (KLB_E_DEVICE_TIMEOUT) and of the members (as klb_sync). */
int klb_batch_sync(klb_batch_t* b);

/* Tile shape of the batched FP32 kernel (as klb_set_variant) for all members. */
int klb_batch_set_variant(klb_batch_t* b, int variant);
int klb_batch_get_variant(const klb_batch_t* b);

/* Autotuner: times `steps` batched launches of each tile shape on the
 * members' current state, keeps the fastest (returned in *variant when not
 * NULL) and restores the state, so the run continues exactly as if it had not
 * been called.  Synchronises.  Needs temporary device memory for one copy of
 * every member's state (KLB_E_NOMEM otherwise). */
int klb_batch_autotune(klb_batch_t* b, int steps, int* variant);

/* Graph replay on (1, default) or off (0; one launch sequence per call). */
int klb_batch_use_graph(klb_batch_t* b, int on);

/* Kernel launches enqueued by the batch (graph replays count their kernels);
 * tiles of one batched launch. */
int64_t klb_batch_launch_count(const klb_batch_t* b);
int64_t klb_batch_tiles(const klb_batch_t* b);
const char* klb_batch_last_error(const klb_batch_t* b);

/* ---------------------------------------------------------------------------
 * Adjoint run (reverse-mode sensitivities of the whole time integration).
 * Objective, from the quantities Sec. IV measures the instability with
 * (E_x = rho u_y^2 / 2 and its growth coefficient):
 *   KE    = dx dy sum_nodes rho u_y^2 / 2 after the last step,
 *   gamma = 1/2 x the least-squares slope of ln K_s against t over the last
 *           75% of the samples, K_s = sum_nodes rho u_y^2 / 2 of sample s
 *           (samples every sample_every steps from t = 0),
 *   L = g_KE KE + g_gamma gamma.
 * The reverse sweep applies the hand-written transpose of the step's Jacobian
 * (WENO5 including its nonlinear weights, f^(0) through the moments, BGK),
 * segment by segment from checkpoints taken every checkpoint_every steps
 * (the segment's states are recomputed), and ends with the sensitivities of
 * the initial fields (f^0 = f^(0)(rho, u, T)).  In FP32 the forward run and
 * the reverse sweep are captured into CUDA graphs on their first call and
 * replayed (the objective's weights are data, not launch parameters); a
 * change of the grid's tile shape or wait budget recaptures them.
 * ------------------------------------------------------------------------- */
typedef struct klb_adj klb_adj_t;

/* A forward grid with params p (FP32 or FP64; periodic or outflow sides only;
 * sample_every >= 1 dividing nsteps) and room for ceil(nsteps /
 * checkpoint_every) checkpoints plus one segment of states.
 * checkpoint_every = 1 stores every state (no recomputation).  Errors:
 * KLB_E_INVAL, KLB_E_NOMEM, KLB_E_CUDA (message: klb_adjoint_last_error(NULL)). */
int klb_adjoint_create(const klb_params* p, int64_t nsteps, int32_t checkpoint_every, klb_adj_t** out);
void klb_adjoint_destroy(klb_adj_t* a); /* NULL-safe */

/* The forward run from the initial fields ([ny][nx] doubles): checkpoints,
 * samples, and the objective parts *ke and *gamma (either may be NULL).
 * Synchronises. */
int klb_adjoint_forward(klb_adj_t* a, const double* rho, const double* ux, const double* uy, const double* T,
                        int on_device, double* ke, double* gamma);

/* dL/d(rho, u_x, u_y, T) of the initial fields ([ny][nx] doubles, caller
 * owned) for L = g_ke KE + g_gamma gamma of the last forward run.  Requires a
 * preceding klb_adjoint_forward (KLB_E_STATE otherwise; the reverse sweep
 * reuses the forward grid's buffers, so each backward needs its own forward).
 * Synchronises. */
int klb_adjoint_backward(klb_adj_t* a, double g_ke, double g_gamma, double* d_rho, double* d_ux, double* d_uy,
                         double* d_T, int on_device);

/* The bare vector-Jacobian product of the nsteps-step map of the last forward
 * run: lam_0 = (d f^N / d f^0)^T lam_N, both [19][ny][nx] doubles over the
 * interior nodes (dependences through ghost nodes folded in).  Requires a
 * preceding klb_adjoint_forward.  Synchronises. */
int klb_adjoint_vjp(klb_adj_t* a, const double* lam_N, double* lam_0, int on_device);

/* K_s of the last forward run (up to cap values into out; count in *count). */
int klb_adjoint_samples(klb_adj_t* a, double* out, int64_t cap, int64_t* count);

/* The forward grid (borrowed; for klb_get_f / klb_moments after a forward,
 * or klb_set_variant to choose its FP32 tile shape). */
klb_t* klb_adjoint_grid(klb_adj_t* a);
const char* klb_adjoint_last_error(const klb_adj_t* a);

/* Diagnostics of a state without any device allocation (the paper has no
 * counterpart; this serves callers that cannot allocate device memory while
 * they run: a host application whose memory manager owns every device
 * allocation; a service that must not grow its device footprint after
 * start-up; a latency-bound loop that cannot afford the device-wide
 * synchronisation a cudaMalloc/cudaFree pair may bring).
 *
 * Computes the 7 diagnostics of klb_diagnostics -- sum rho, sum rho u_x,
 * sum rho u_y, sum rho (T + |u|^2/2), max |u_y|, max rho u_y^2 / 2,
 * sum rho u_y^2 / 2 over the interior nodes, in FP64 -- of the state f and
 * writes them to out[0..6], a DEVICE pointer owned by the caller.  f is a
 * device pointer to plane 0 of a distribution array in the library's layout
 * (as klb_layout reports it: element (q, j, i) of the interior at
 * f[q*plane + (j+gy)*pitch + (i+gx)], gx = 4, gy = 3, in the precision given, KLB_FP32 or
 * KLB_FP64); v are the ring speeds.  The work is enqueued on `stream` (NULL =
 * the default stream) and the call returns without waiting; it calls no
 * cudaMalloc, cudaFree or allocating library routine.  The sums are reduced
 * in the same order as the handle-based path with kernel variant 0 (the
 * default), so both agree to the last bit; with variant 1, to rounding.
 *
 * Scratch: the per-CTA partial records live in a fixed device array of this
 * library, 4096 records (256 KiB), held by every GPU that loads the library
 * until the process exits; FP32 states need one record per CTA (at most two
 * per SM), FP64 states one per tile of 32 x 8 nodes, so FP64 grids above 4096
 * tiles are rejected with KLB_E_INVAL and a message.  All calls on a device
 * share that array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU (on different streams, or from different threads) race
 * and must be ordered by the caller.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  A non-finite state shows as
 * NaN sums.  Errors: KLB_E_INVAL, KLB_E_CUDA; message:
 * klb_diagnostics_static_error(). */
int klb_diagnostics_static(const void* f, int32_t precision, int32_t nx, int32_t ny, int64_t pitch, int64_t plane,
                           const double v[3], double* out, void* stream);
const char* klb_diagnostics_static_error(void);

/* Fault injection for tests.  With polls > 0, every later step launch also
 * waits, with a budget of `polls` polls, on a device barrier that nothing
 * arrives on (a flag that nothing sets): the wait runs out, each CTA records
 * KLB_E_DEVICE_TIMEOUT (reported by the next synchronising call), lets its
 * tile copy in flight land and exits without computing, and the CUDA context
 * stays usable.  polls = 0 switches the injection off.  The state of a step
 * that ran under injection is undefined. */
int klb_debug_inject_wait_timeout(klb_t* h, int64_t polls);

#ifdef __cplusplus
}
#endif
#endif /* KLB_H */
