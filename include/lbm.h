/*
 * lbm.h -- C ABI of the GB300 (sm_103a) free-surface lattice Boltzmann library for
 * liquid-gas-solid flow (Bogner, Harting, Ruede, "Direct simulation of liquid-gas-solid
 * flow with a free surface lattice Boltzmann method").
 *
 * One time step (lbm_step) is the paper's per-step hot path, on the GPU:
 *   - D3Q19 pull streaming (Sec. 2.1, Eq. LBE1) with halfway bounce-back at no-slip walls
 *     or periodic wrap per axis;
 *   - moving-wall bounce-back on sphere links (Sec. 2.3, Eq. bbrule) with the
 *     momentum-exchange force and torque (Eqs. netforce, torque, momentum_transfer);
 *   - gas-side PDF reconstruction from each bubble's gas pressure (Sec. 2.2, Eq. fsk, with
 *     p_w = p_g + 2 sigma kappa when sigma > 0);
 *   - fill-level-weighted mass exchange of interface cells (Eqs. massExchange,
 *     massExchangeb);
 *   - TRT collision with the magic parameter 3/16 (Eq. LBE2, Eq. latticeViscosity and the
 *     relation below it) and a Guo gravity force;
 *   - interface / liquid / gas conversions with layer closure, equilibrium initialisation
 *     of new interface cells and excess-mass redistribution (Sec. 2.2, Fig.
 *     cellConversions);
 *   - the bubble model (per-bubble volume -> gas density; touching bubbles merge, and with
 *     lbm_params.split_every > 0 a bubble whose region breaks apart splits, Sec. 2.2);
 *   - sphere update: lubrication correction (Eq. lubrication) and Newton-Euler sub-steps
 *     (Sec. 2.3), then cells covered / uncovered by the moved spheres and PDF refill.
 *
 * Conventions for every call:
 *   - lattice units (dx = dt = 1); cell (x,y,z) is centred at integer coordinates and has
 *     linear index i = x + nx*(y + ny*z); N = nx*ny*nz;
 *   - the library never allocates device memory: all device state lives in one caller-owned
 *     arena (lbm_arena_bytes / lbm_init); the library never frees it;
 *   - work is enqueued on the caller's CUDA stream and is asynchronous, except where a call
 *     says it synchronises;
 *   - every call returns LBM_OK (0) or a negative LBM_E* code; no exception crosses the ABI;
 *   - a pointer documented as "device" must point to device memory of the current device,
 *     "host" to host memory; sizes are counts of elements unless stated otherwise.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define LBM_OK 0
#define LBM_EINVAL (-1)      /* bad argument */
#define LBM_ESTATE (-2)      /* call not allowed in the current state */
#define LBM_ECUDA (-3)       /* a CUDA runtime call failed */
#define LBM_EUNSTABLE (-4)   /* a cell's density became non-positive or NaN */
#define LBM_EOVERFLOW (-5)   /* a conversion worklist or a sphere bin overflowed */
#define LBM_EMERGE (-6)      /* more distinct pairs of bubbles met in one step than the merge
                                table holds (1024); the pairs beyond it were not merged */
#define LBM_ESPLIT (-7)      /* a bubble could not be split: no free row in the bubble table, or
                                more connected parts at a split step than the part table holds
                                (4096); the parts stayed one bubble */

/* per-axis boundary kind */
#define LBM_BC_WALL 0        /* no-slip wall halfway beyond the outermost cells */
#define LBM_BC_PERIODIC 1
#define LBM_BC_FREESLIP 2    /* free-slip wall halfway beyond the outermost cells (specular
                                reflection: a population leaving toward the wall comes back
                                with its normal component reversed, one cell further along its
                                tangential components; Fig. bubbleSetup's side walls) */

/* PDF storage between steps (collisions always run in FP32) */
#define LBM_STORE_F32 0      /* f stored as FP32 */
#define LBM_STORE_F16DEV 1   /* f - w_q stored as IEEE half */
#define LBM_STORE_BF16DEV 2  /* f - w_q stored as bfloat16 */

/* sphere motion */
#define LBM_SPHERES_FIXED 0       /* x, u, w held; u, w still act as surface velocity */
#define LBM_SPHERES_FREE 1        /* Newton-Euler with lubrication and sub-steps (Sec. 2.3) */
#define LBM_SPHERES_PRESCRIBED 2  /* x advances by u every step, u and w held */

/* cell types reported by lbm_fields / lbm_export_state */
#define LBM_CELL_LIQUID 1
#define LBM_CELL_INTERFACE 2
#define LBM_CELL_GAS 4
#define LBM_CELL_OBSTACLE 8

/* status bits (lbm_status) */
#define LBM_S_UNSTABLE 1u        /* density <= 0 or NaN in some cell */
#define LBM_S_OVERFLOW 2u        /* a conversion / covering worklist overflowed */
#define LBM_S_BUBBLE_GONE 4u     /* a bubble's volume reached zero */
#define LBM_S_BIN_OVERFLOW 8u    /* more spheres in a neighbour-search bin than it holds */
#define LBM_S_MERGE 64u          /* the merge table overflowed (see LBM_EMERGE) */
#define LBM_S_SPLIT 128u         /* a bubble could not be split (see LBM_ESPLIT) */
#define LBM_S_FAST_SPHERE 32u    /* a sphere moved more than a quarter cell in one step (the
                                    per-step partner searches assume less) */

typedef struct lbm_params {
    int32_t nx, ny, nz;        /* grid size, each >= 3 */
    int32_t bc[3];             /* LBM_BC_* per axis */
    int32_t storage;           /* LBM_STORE_* */
    int32_t n_substeps;        /* sphere sub-steps per LBM step, 1..64 (the paper: up to 10) */
    int32_t sphere_mode;       /* LBM_SPHERES_* */
    int32_t max_bubbles;       /* capacity of the bubble table, >= 1 */
    int32_t max_spheres;       /* capacity of the sphere table, >= 1 */
    int32_t worklist_cap;      /* entries per conversion worklist; 0 = N/50 + 4096 */
    double tau;                /* relaxation time, lambda_+ = -1/tau, tau > 1/2 */
    double g[3];               /* body force per unit mass (gravity) */
    double sigma;              /* surface tension (0: no curvature term) */
    double rho_gas0;           /* initial gas density of every bubble (1 = liquid reference) */
    double eps;                /* conversion band: fill >= 1+eps fills, fill <= -eps empties */
    int32_t open_top;          /* 1: the +z face is an open boundary at the reference pressure
                                  (Fig. bubbleSetup's top) instead of bc[2]'s wall: a link
                                  from beyond it gets -f*_qb + 2 e+_q(1, u), u the cell's own
                                  velocity (Eq. fsk with rho_w = 1); the mass it lets in or out
                                  is reported by lbm_mass_budget.  bc[2] must not be periodic. */
    int32_t hydrostatic;       /* 1 (with open_top): the liquid starts in hydrostatic equilibrium,
                                  rho = exp(3 g[2] (z - z_top)) with rho = 1 on the open face's
                                  plane z_top = nz - 1/2 (dp/dz = rho g[2], p = rho/3), and each
                                  bubble's gas at the liquid's pressure at its centre plus the
                                  Laplace jump 2 sigma / r (rho_gas0 is then unused); 0: rho = 1
                                  and the gas at rho_gas0 */
    int32_t split_every;       /* > 0: every split_every steps, at the end of the step, bubbles
                                  split into their connected parts (a bubble is a connected gas
                                  region, Sec. 2.2): every gas / interface cell first takes its
                                  bubble's root id (ids left without cells become free rows);
                                  a bubble whose cells form several D3Q19-connected parts keeps
                                  its largest part (equal volumes to within 1e-9: the part with
                                  the lowest cell index) and every other part of non-zero volume,
                                  in the order of the parts' lowest cell indices, becomes a
                                  bubble with the lowest free id, gas mass and reference volume
                                  divided in proportion to the parts' volumes (the gas density
                                  carries over).  Bubble ids then range over the whole table
                                  (max_bubbles rows).  0: bubbles never split. */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Size in bytes of the device arena a simulation with these parameters needs (all PDF
 * grids, per-cell fields, tables, worklists and scratch).  p: host.  Returns LBM_EINVAL for
 * invalid parameters. */
int lbm_arena_bytes(const lbm_params* p, size_t* bytes);

/* Create a simulation over a caller-owned device arena of at least lbm_arena_bytes(p)
 * bytes, 256-byte aligned.  The arena must stay alive and untouched by the caller until
 * lbm_destroy.  cuda_stream: the cudaStream_t all work goes to (NULL = legacy default
 * stream).  *out receives a host-side handle.  Nothing is written to the device until the
 * first lbm_step. */
int lbm_init(const lbm_params* p, void* arena, size_t arena_bytes, void* cuda_stream, lbm_ctx** out);

/* Switch the stream subsequent calls enqueue on. */
int lbm_set_stream(lbm_ctx* ctx, void* cuda_stream);

/* Add a spherical gas bubble of centre c[3] (host) and radius r (> 0).  Only before the
 * first lbm_step (else LBM_ESTATE).  *id (host, may be NULL) receives its index.
 * Initial fill level (Sec. 3.2 / 4: a spherical bubble in quiescent liquid):
 * phi = prod_b clamp(|x - c_b| - (r_b - 1/2), 0, 1). */
int lbm_add_bubble(lbm_ctx* ctx, const double c[3], double r, int* id);

/* Add a sphere (Sec. 2.3): centre c[3], radius r, density rho_p, velocity u[3], angular
 * velocity w[3] (all host).  Only before the first lbm_step.  Cells with
 * |x - c|^2 <= r^2 become its obstacle cells (the lowest sphere id wins where spheres
 * overlap). */
int lbm_add_sphere(lbm_ctx* ctx, const double c[3], double r, double rho_p, const double u[3],
                   const double w[3], int* id);

/* The same for n spheres at once, from host arrays: centres c[n][3], radii r[n], densities
 * rho_p[n], velocities u[n][3] and angular velocities w[n][3] (u, w may be NULL: at rest).
 * They get ids first_id .. first_id + n - 1 (*first_id, host, may be NULL).  Every sphere is
 * checked before any is added: LBM_EINVAL (nothing added) if one has r <= 0 or rho_p <= 0 or
 * they do not fit the table (max_spheres); LBM_ESTATE after the first lbm_step. */
int lbm_add_spheres(lbm_ctx* ctx, int n, const double* c, const double* r, const double* rho_p, const double* u,
                    const double* w, int* first_id);

/* Advance nsteps >= 0 time steps.  The first call initialises the fields on the device
 * (liquid at rest, bubbles, layer closure, spheres).  Asynchronous: problems found on the
 * device are latched in the status word and reported by lbm_status / lbm_forces.
 * The end-of-step kernels of the last step (conversions, sphere motion, cover/uncover,
 * bubble model) are left pending: the next lbm_step runs them concurrently with its bulk
 * sweep, and every call that reads the state (lbm_forces, lbm_spheres, lbm_bubbles,
 * lbm_fields, lbm_export_state, lbm_mass_budget, lbm_status and the window calls below)
 * enqueues them first, so what a caller sees is always the complete step. */
int lbm_step(lbm_ctx* ctx, int nsteps);

/* Momentum-exchange force F[n][3] and torque T[n][3] (host, FP64) of the last step, for
 * the first n spheres (hydrodynamic part only: no lubrication, no gravity).  Synchronises
 * the stream.  Returns the status as an error code if the status word is set. */
int lbm_forces(lbm_ctx* ctx, double* F, double* T, int n);

/* Sphere state x[n][3], u[n][3], w[n][3] (host, FP64; any may be NULL).  Synchronises. */
int lbm_spheres(lbm_ctx* ctx, double* x, double* u, double* w, int n);

/* Lubrication force Fl[n][3] (host, FP64) of the first n spheres in the last sub-step of the
 * last step (Sec. 2.3, Eq. lubrication: pairs closer than 2/3 of a cell, the gap floored at
 * 0.2 x 2/3, mu = (tau - 1/2)/3, +F on one sphere and -F on the other); zero for spheres with
 * no partner that close.  Synchronises. */
int lbm_lubrication(lbm_ctx* ctx, double* Fl, int n);

/* Bubble table (host, FP64; any may be NULL): reference volume V0[n], volume V[n], gas
 * density rho_g[n] for bubble ids 0..n-1.  An id that has merged into a larger bubble
 * reports the merged bubble's values.  Synchronises.
 *
 * Bubble merging (Sec. 2.2: a bubble is a connected gas region).  When a gas or interface
 * cell of one bubble lies next to one of another (D3Q19 neighbourhood), the two are one bubble
 * from the end of that step on: the larger root id joins the smaller, the gas masses add
 * (rho_g0 V0 each, so the V0 add), V is the sum over all ids of the bubble and every id gets
 * rho_g = rho_g0 V0 / V.  Cells keep the id they were created with.  Bubbles that touch
 * from the start are merged at lbm_step(ctx, 0).  With splitting on
 * (lbm_params.split_every > 0) n may be up to max_bubbles: at each split step every cell takes
 * its bubble's root id, rows left without cells are reset (V0 = V = 0, rho_g = rho_gas0) and
 * reused for the parts split off (lbm_bubble_splits). */
int lbm_bubbles(lbm_ctx* ctx, double* V0, double* V, double* rho_g, int n);

/* Root id root[n] (host; NULL allowed) of bubble ids 0..n-1 -- the smallest id of the bubble
 * each belongs to, itself if it never merged -- and the number of merges so far (*n_merges,
 * NULL allowed).  Synchronises. */
int lbm_bubble_roots(lbm_ctx* ctx, int32_t* root, int n, int* n_merges);

/* With splitting on (lbm_params.split_every > 0): *n_ids (NULL allowed) one past the highest
 * bubble id that ever carried cells -- lbm_bubbles and lbm_bubble_roots take n up to
 * max_bubbles -- and *n_splits (NULL allowed) the parts split off so far.  Without splitting
 * *n_ids is the number of bubbles added and *n_splits 0.  Synchronises. */
int lbm_bubble_splits(lbm_ctx* ctx, int* n_ids, int* n_splits);

/* Macroscopic fields into caller device buffers (any may be NULL): rho[N] and u[3][N]
 * (post-collision moments, u = (sum c f* - rho g / 2) / rho, the velocity the collision
 * used; 0 in inactive cells), phi[N] (fill level: 1 liquid, 0 gas, phi interface, 1
 * obstacle), flags[N] (LBM_CELL_*).  Asynchronous. */
int lbm_fields(lbm_ctx* ctx, float* rho, float* u, float* phi, uint8_t* flags);

/* Full state into caller device buffers (any may be NULL): f[19][N] post-collision PDFs as
 * FP32 deviations f*_q - w_q from the lattice weights (w_0 = 1/3, w_1..6 = 1/18,
 * w_7..18 = 1/36; whatever the storage; undefined in inactive cells), flags[N]
 * (LBM_CELL_*), mass[N] (interface mass), phi[N], owner[N] (bubble id of gas / interface
 * cells, sphere id of obstacle cells, -1 otherwise), kappa[N] (curvature; 0 if sigma = 0).
 * D3Q19 order: q = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (+1,+1,0),(-1,-1,0),(+1,-1,0),
 * (-1,+1,0),(+1,0,+1),(-1,0,-1),(+1,0,-1),(-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1).
 * Asynchronous. */
int lbm_export_state(lbm_ctx* ctx, float* f, uint8_t* flags, float* mass, float* phi, int32_t* owner, float* kappa);

/* Mass budget (host out[5], FP64): total liquid mass M = sum_liquid rho + sum_interface m +
 * pool, boundary source S_bb (moving-wall bounce-back links and, with open_top, the open
 * face's links), mass removed by covering S_cover, mass added by
 * refill S_uncover, undistributed excess pool.  M - M(0) - S_bb - S_uncover + S_cover is
 * the drift.  Synchronises. */
int lbm_mass_budget(lbm_ctx* ctx, double out[5]);

/* Latched status bits (LBM_S_*) into *status (host).  Synchronises. */
int lbm_status(lbm_ctx* ctx, uint32_t* status);

/* ---- differentiation over a window with frozen cell types ------------------------------
 * The window is liquid only (no bubbles), the spheres fixed (LBM_SPHERES_FIXED; their u and w
 * still act as surface velocities), the faces no-slip or periodic and the PDFs stored in FP32,
 * so no cell changes type; else these calls return LBM_ESTATE.  States are post-collision PDFs as FP32 deviations
 * f*_q - w_q, [19][N], device, in the D3Q19 order of lbm_export_state.  The objective is
 * J = sum over the window's steps t of jdir . (sum over spheres of the momentum-exchange
 * force F_P(t), Eqs. netforce and momentum_transfer). */

/* Set the relaxation time tau (> 1/2; lambda_+ = -1/tau, lambda_- from the magic relation,
 * Sec. 2.1) and the body force g[3] (host) of the steps that follow, so that a window can be
 * evaluated at other parameters.  Between steps only: the last step's end-of-step kernels are
 * run first with the parameters it had.  Synchronises.  LBM_EINVAL for tau <= 1/2 or a
 * non-finite g. */
int lbm_set_params(lbm_ctx* ctx, double tau, const double g[3]);

/* Replace the current post-collision PDFs by f[19][N] (device, FP32 deviations f*_q - w_q in
 * the layout lbm_export_state writes): the start state of a window.  The cell types, masses and
 * spheres stay.  Window conditions as below (else LBM_ESTATE).  Asynchronous. */
int lbm_import_state(lbm_ctx* ctx, const float* f);

/* The objective of a window accumulated on the device: from this call on, every step adds
 * jdir . (sum over spheres of the momentum-exchange force F_P of the step, Eqs. netforce and
 * momentum_transfer) to an FP64 scalar, which this call resets to 0 (jdir[3]: host; NULL stops
 * the accumulation).  The last step's force is not counted.  Synchronises. */
int lbm_objective(lbm_ctx* ctx, const double jdir[3]);

/* The objective accumulated since lbm_objective, including the last step's force, into *J
 * (host).  Synchronises. */
int lbm_objective_read(lbm_ctx* ctx, double* J);

/* One forward step of the window from f_in to f_out (device, distinct): streaming with
 * bounce-back at walls and spheres, then the TRT/Guo collision (Eqs. LBE1, bbrule, LBE2), the
 * same arithmetic as lbm_step.  Used to recompute states between checkpoints.  Asynchronous. */
int lbm_forward_frozen(lbm_ctx* ctx, const float* f_in, float* f_out);

/* One reverse step: given the forward state f_fwd = f*(t) and adj_in = dJ/df*(t+1), writes
 * adj_out = dJ/df*(t) (device [19][N], distinct from adj_in; only liquid cells' entries are
 * defined) = (d f*(t+1) / d f*(t))^T adj_in + d(jdir . F(t+1)) / d f*(t), and adds
 * adj_in . d f*(t+1)/d theta, theta = (g, tau), to FP64 accumulators on the device, which it
 * clears first unless accumulate != 0 (lambda_- follows tau through the magic relation).
 * jdir[3]: host.  With dJdg and dJdtau NULL the call is asynchronous; with both non-NULL
 * (host) it synchronises the stream and returns there the accumulated d/dg[3] and d/dtau.
 * LBM_EINVAL for NULL device pointers, adj_in == adj_out or only one of dJdg, dJdtau NULL. */
int lbm_adjoint_step(lbm_ctx* ctx, const float* f_fwd, const float* adj_in, float* adj_out, const double jdir[3],
                     int accumulate, double dJdg[3], double* dJdtau);

/* Timing of the sweep: while on != 0, lbm_step launches steps one by one (no CUDA graph)
 * and records CUDA event pairs on the library's stream around the bulk sweep kernel (the
 * dominant one; it runs concurrently with the previous step's end-of-step kernels) and
 * around the rest of the sweep (fix pass and boundary kernel, after those kernels). */
int lbm_profile(lbm_ctx* ctx, int on);

/* Sums of the recorded durations in milliseconds since the last read (host ms[0]: bulk
 * sweep kernel, ms[1]: rest of the sweep) and their number (host *sweeps); waits for the
 * recorded events.  Resets them. */
int lbm_profile_read(lbm_ctx* ctx, double ms[2], uint64_t* sweeps);

/* Bytes the library itself has copied host -> device (*h2d) and device -> host (*d2h)
 * so far (table uploads, copy-out calls), both host pointers. */
int lbm_copy_bytes(lbm_ctx* ctx, uint64_t* h2d, uint64_t* d2h);

/* Kernel launches enqueued so far (each node of a replayed CUDA graph counts). */
int lbm_launch_count(lbm_ctx* ctx, uint64_t* launches);

/* Bubble volumes for callers that cannot allocate device memory.  Some callers cannot call
 * cudaMalloc at all (code inside an allocator hook or a host callback, real-time sections,
 * programs whose device memory is fully handed out before they start); this entry point
 * allocates nothing, neither directly nor through any library, once its set-up on a device is
 * done (below).  The paper has no counterpart: it offers the two per-id sums of lbm_step's
 * bubble model on their own, V_id = number of gas cells carrying bubble id `id` + sum over the
 * interface cells carrying `id` of (1 - phi), FP64.  Cells keep the id they were created with,
 * so after bubbles merge these are per-id parts: the merged bubble's V (what lbm_bubbles
 * reports for each of its ids) is the sum of volumes[id] over the ids with the same root
 * (lbm_bubble_roots).
 *   flags[n_cells], owner[n_cells], phi[n_cells]: device, in the layout lbm_export_state
 *     writes (LBM_CELL_* types, bubble id or -1, fill level);
 *   volumes[n_bubbles]: device, FP64 output, one entry per id 0..n_bubbles-1;
 *   n_bubbles: 1..1024, else LBM_EINVAL (nothing is enqueued);
 *   cuda_stream: the cudaStream_t the work goes to (asynchronous).
 * Its scratch is a 16 KB static device array that every device using the library holds
 * until the process exits, shared by all calls: calls whose work overlaps on the GPU (e.g.
 * on two streams) race and must be ordered by the caller.  Each call clears the part it uses.
 * The first call on a device is its set-up: it looks up that array's device address and the
 * device's multiprocessor count and loads the call's two kernels (under CUDA's lazy loading a
 * kernel's code is loaded on first use, which takes device memory).  Make that first call
 * outside any section where allocation is forbidden, and before any stream capture.
 * LBM_ECUDA if the set-up or a launch fails. */
int lbm_bubble_volumes_noalloc(const uint8_t* flags, const int32_t* owner, const float* phi, size_t n_cells,
                               int n_bubbles, double* volumes, void* cuda_stream);

/* Release the host-side handle (the arena stays the caller's). */
int lbm_destroy(lbm_ctx* ctx);

/* Static text for a return code. */
const char* lbm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
