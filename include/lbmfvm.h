/*
 * lbmfvm — GB300 (sm_103a) coupled lattice-Boltzmann / finite-volume solver
 * for natural convection: the hybrid LBM(velocity) + FVM(temperature) method
 * of Li, Yang & Zhang, arXiv 1908.08386, Section 5.
 *
 * One time step of a handle is one launch of a fused CUDA kernel that, per
 * node,
 *   - pulls the post-collision D2Q9 populations of the previous step from the
 *     neighbours (Eq. 5, velocity set of Eq. 4, weights of Eq. 9);
 *   - rebuilds wall nodes by non-equilibrium extrapolation from their inner
 *     partner node x_f with rho_b = rho(x_f) (Eqs. 60, 94, 96);
 *   - takes the moments rho, u (Eqs. 16-17);
 *   - advances T by an explicit finite-volume energy balance over the
 *     node-centred control volume (grid setting 1 of Section 5.1, energy
 *     equation Eq. 76), with face velocities interpolated from the new u;
 *   - relaxes toward the equilibrium of Eq. 8 with the Boussinesq buoyancy
 *     force of Eqs. 18 and 81 evaluated with the new T, and stores the result.
 * Two options of the energy update (lbmfvm_opts_t.fv_scheme, fv_substeps):
 * QUICK face temperatures stay in the fused launch; m > 1 explicit sub-steps
 * per lattice step take m + 2 launches per step (the new velocity into two
 * planes, m sub-steps with it held, then the collision with the final T).
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: LBMFVM_OK (0) or a negative
 *     LBMFVM_ERR_* code.  Nothing throws or exits across this boundary.
 *     lbmfvm_last_error() gives a one-line message for the last failure.
 *   - Fields are row-major [ny][nx], x fastest, j = 0 the bottom row.
 *     Lengths are in lattice units (node spacing 1, time step 1); the cavity
 *     height is H = ny - 1 (N nodes per side span N - 1 spacings).
 *   - Input and output pointers may be host or device memory (the library
 *     copies with cudaMemcpyDefault).  The caller keeps ownership of all of
 *     them; nothing is retained after the call returns.
 *   - Work is ordered after all work previously enqueued on the handle's
 *     stream (lbmfvm_opts_t.cuda_stream), and later work on that stream is
 *     ordered after it.  Calls that return values to the caller synchronise.
 *   - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef LBMFVM_H
#define LBMFVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define LBMFVM_OK 0
#define LBMFVM_ERR_ARG (-1)      /* invalid argument, size or null handle */
#define LBMFVM_ERR_UNSTABLE (-2) /* parameters outside the scheme's stability limits */
#define LBMFVM_ERR_CUDA (-3)     /* a CUDA runtime call or kernel failed */
#define LBMFVM_ERR_DIVERGED (-4) /* a reduction met a non-finite value */
#define LBMFVM_ERR_TIMEOUT (-5)  /* a bounded device-side wait ran out */
#define LBMFVM_ERR_NOMEM (-6)    /* device allocation failed or workspace too small */
#define LBMFVM_ERR_IO (-7)       /* a checkpoint file could not be written or read, or is corrupt */

/* Sides of the rectangle, index into lbmfvm_grid_t.bc / t_wall. */
#define LBMFVM_SIDE_W 0
#define LBMFVM_SIDE_E 1
#define LBMFVM_SIDE_S 2
#define LBMFVM_SIDE_N 3

/* Boundary kinds.  Walls are no-slip nodes rebuilt by non-equilibrium
 * extrapolation (Eqs. 94, 96).  DIRICHLET holds T at t_wall (Eqs. 77-78);
 * ADIABATIC has zero heat flux through the wall (Eqs. 79-80); MOVING is an
 * adiabatic wall sliding tangentially at u_lid (lid-driven flow, Section 3);
 * PERIODIC must be set on both opposite sides. */
#define LBMFVM_BC_DIRICHLET 0
#define LBMFVM_BC_ADIABATIC 1
#define LBMFVM_BC_PERIODIC 2
#define LBMFVM_BC_MOVING 3

/* Step kernel selection; both compute the same arithmetic.
 *   TMA      persistent, one block per SM: each tile's populations,
 *            temperature, node codes and face flags are staged in shared
 *            memory by TMA through a multi-stage mbarrier pipeline and the
 *            results leave by TMA bulk stores (walls on every side; every
 *            storage type);
 *   GENERIC  one block per tile, gathers straight from global memory (any
 *            boundary, every storage type).
 * AUTO takes TMA where it applies and GENERIC otherwise. */
#define LBMFVM_KERNEL_AUTO 0
#define LBMFVM_KERNEL_GENERIC 1
#define LBMFVM_KERNEL_TMA 2
#define LBMFVM_TMA_AUTOTUNE (-1)
#define LBMFVM_TMA_DEFAULT (-2)

/* Face temperatures of the explicit energy update (lbmfvm_opts_t.fv_scheme)
 * and automatic sub-steps (lbmfvm_opts_t.fv_substeps). */
#define LBMFVM_FV_CENTRAL 0
#define LBMFVM_FV_QUICK 1
#define LBMFVM_FV_SUBSTEPS_AUTO 0

/* Energy solver (lbmfvm_opts_t.energy).
 *   FV        the explicit finite-volume energy balance of Section 5 (the
 *             hybrid method; default);
 *   LBM_D2Q5  the D2Q5 thermal lattice-Boltzmann model of Section 2.4 (the
 *             paper's pure-LBM comparison, Tables 1-2): energy populations
 *             g_i relax toward g_eq = T w_i (1 + e_i.u / c_s^2) (Eqs. 19, 21,
 *             22) with tau_T = alpha / c_s^2 + 1/2 (Eq. 20), stream like f
 *             and give T = sum g (Eq. 23); walls rebuild g by
 *             non-equilibrium extrapolation (Eq. 95) with the wall
 *             temperature on Dirichlet sides and the partner's temperature on
 *             adiabatic sides and obstacle surfaces.  One step is one launch
 *             of its own kernel (one node per thread, pulls from global
 *             memory).  F64, F32 or F32X2 storage; single cavities only; no
 *             energy-update options. */
#define LBMFVM_ENERGY_FV 0
#define LBMFVM_ENERGY_LBM_D2Q5 1

/* Box-wall treatment of the populations (lbmfvm_opts_t.wall_bc).
 *   NEE  non-equilibrium extrapolation, f_b = f_eq(rho_f, u_w) + f(x_f)
 *        - f_eq(rho_f, u_f) (Eqs. 94, 96; default);
 *   FD   the finite-difference velocity-gradient scheme of Section 3
 *        (hybrid method 2, Eqs. 61-72): f_b = f_eq(rho_f, u_w) - (tau w_i /
 *        c_s^2) rho_f Q_i : S with Q_i = e_i e_i - c_s^2 I (Eqs. 67, 69-71),
 *        the strain rate S from finite differences of the new velocity field
 *        (centred along the wall, second-order one-sided into the fluid) and
 *        the normal strain from continuity (Eq. 72) off the corners.
 *        Obstacle surfaces keep the extrapolation.  Runs on the GENERIC
 *        kernel (the one-sided differences reach two nodes into the fluid);
 *        single cavities with the finite-volume energy update only. */
#define LBMFVM_WALL_NEE 0
#define LBMFVM_WALL_FD 1

/* Storage precision of the distributions.  F32/F16/BF16 store f - w_i and
 * compute in FP32 with FP32 temperature; F64 stores and computes in FP64.
 * F32X2 ("double-single") stores f - w_i and T as pairs of FP32 numbers
 * (hi + lo, about 48 significant bits, 8 bytes) and computes with them on the
 * FP32 units, so it reaches FP64-level residuals (FP32 storage floors near
 * 2e-7) at several times the speed of FP64 arithmetic on this GPU. */
#define LBMFVM_F64 0
#define LBMFVM_F32 1
#define LBMFVM_F16 2
#define LBMFVM_BF16 3
#define LBMFVM_F32X2 4

typedef struct lbmfvm lbmfvm_t;

/* Geometry and boundary conditions of one cavity. */
typedef struct {
    int32_t nx, ny;    /* nodes along x and y, each >= 3 */
    int32_t bc[4];     /* LBMFVM_BC_* per side W, E, S, N */
    double t_wall[4];  /* wall temperature of DIRICHLET sides (W = hot, E = cold) */
    double u_lid;      /* tangential speed of MOVING sides */
    double t_init;     /* uniform initial temperature of the default state */
} lbmfvm_grid_t;

/* Options; fill with lbmfvm_opts_default() first. */
typedef struct {
    int32_t store;          /* LBMFVM_F64/F32/F16/BF16/F32X2; default LBMFVM_F32 */
    int32_t tile_y;         /* rows per thread block of the generic step kernel:
                               0 = default, else one of 4, 8, 16 */
    int32_t kernel;         /* LBMFVM_KERNEL_*; default AUTO */
    int32_t tma_config;     /* tile shape of the TMA kernel, 0..5,
                               LBMFVM_TMA_DEFAULT (the default) or
                               LBMFVM_TMA_AUTOTUNE.  32- and 16-bit storage
                               (width x height, threads, input stages at 32 / 16
                               bit, population halo rows): 64x16, 1024, 3/3, 3;
                               64x16, 512, 3/3, 3; 64x8, 512, 2/3, 3 (two blocks
                               per SM); 128x8, 1024, 2/3, 3; 64x16, 512 + 128 ring
                               threads (four warps that take the one-node ring's
                               moments and issue the copies), 3/3, 2; the same
                               with 3 halo rows.  64-bit storage: 64x8, 256, 2;
                               32x8, 256, 3; 32x16, 512, 2; 32x8, 256, 2 (two
                               blocks per SM); 32x8, 256 + 64 ring threads, 3;
                               the same with 3 halo rows (64-bit shapes 0-4 take 2).
                               LBMFVM_TMA_DEFAULT: for a grid with fewer tiles
                               than the GPU has SMs, 2 (32- and 16-bit storage)
                               or 4 (64-bit), which spread it over more SMs;
                               otherwise 4 when both population buffers and
                               temperature planes fit in the L2, 5 if not (32-
                               and 16-bit), 3 for 64-bit storage: the fastest
                               measured on 64^2 to 4096^2 cavities.
                               LBMFVM_TMA_AUTOTUNE times every shape (a
                               captured graph of 32 launches, replayed twice)
                               on the handle's own grid at create and keeps
                               the fastest (remembered per storage precision and
                               power-of-two size class for the process); shapes
                               never change results. */
    double t_ref;           /* reference temperature of the buoyancy term; NaN (the
                               default) selects T_l = t_wall[E] as in Eq. 81 */
    void *cuda_stream;      /* cudaStream_t the handle orders its work on; NULL =
                               the legacy default stream */
    void *workspace;        /* device memory of at least lbmfvm_workspace_bytes(),
                               256-byte aligned, owned by the caller and kept alive
                               until lbmfvm_destroy; NULL = the library allocates */
    size_t workspace_bytes; /* size of workspace */
    int32_t fv_scheme;      /* face temperatures of the energy update:
                               LBMFVM_FV_CENTRAL (default; the mean of the two
                               nodes) or LBMFVM_FV_QUICK (quadratic upstream
                               interpolation, the scheme Section 3.1 names for
                               its finite-volume solver; the face keeps the
                               central value where the far upstream node takes
                               no part in the energy balance) */
    int32_t fv_substeps;    /* explicit energy-update sub-steps m per lattice
                               step, each of dt = 1/m with the velocity u^{n+1}
                               held (Section 5.1's energy update taken in m
                               explicit steps): 1 (default), m >= 2, or
                               LBMFVM_FV_SUBSTEPS_AUTO = 0, the fewest with
                               alpha/m <= 0.2 and U0^2/m <= 1.8 alpha (U0 from
                               Ma; lbmfvm_create_lattice uses alpha only).  The
                               stability limits become alpha/m <= 1/4 and
                               U0^2/m <= 2 alpha.  QUICK and m != 1 need the TMA
                               kernel (walls on every side); they fix its tile
                               shape to 1 (no autotuning). */
    int32_t energy;         /* LBMFVM_ENERGY_FV (default) or LBMFVM_ENERGY_LBM_D2Q5 */
    int32_t wall_bc;        /* LBMFVM_WALL_NEE (default) or LBMFVM_WALL_FD */
    int32_t fv_grid;        /* 1 (default): the energy balance on the lattice's own
                               node-centred volumes (grid setting 1, Fig. 29);
                               2: grid setting 2 (Section 5.1, Fig. 30), NX x NY
                               control volumes of 2 x 2 lattice spacings whose
                               faces pass through lattice nodes (face velocities
                               are lattice velocities), centres at the odd-odd
                               nodes, node temperatures interpolated from the
                               volumes (the centre's value, the mean of two or
                               four centres, the nearest volume on a wall without
                               heat flux, the wall value on a Dirichlet wall).
                               Grid setting 2 needs an even number of spacings
                               along each axis, no obstacle, walls on every side,
                               the central update without sub-steps, single
                               cavities; it takes four more launches on a coarse
                               step and the collision with the node temperatures
                               every step; no checkpoints. */
    int32_t fv_every;       /* grid setting 2: lattice steps per coarse explicit
                               energy step, each of time step fv_every (default
                               1; alpha * fv_every <= 0.8, the coarse explicit
                               limit beside a Dirichlet wall).  A captured graph
                               of steps is used when fv_every divides 64. */
} lbmfvm_opts_t;

/* Fill *opts with the defaults listed above. */
void lbmfvm_opts_default(lbmfvm_opts_t *opts);

/* Device bytes one handle of this grid and options needs (the distributions,
 * two temperature planes, node codes and face flags, a velocity snapshot,
 * the tile list and reduction scratch).  Returns LBMFVM_ERR_ARG for an invalid grid. */
int lbmfvm_workspace_bytes(const lbmfvm_grid_t *grid, const lbmfvm_opts_t *opts, size_t *bytes);

/* Create a cavity from the nondimensional groups (Eqs. 83-89):
 *   U0 = Ma/sqrt(3) (Eq. 84, u_c = sqrt(g beta dT H), c_s = 1/sqrt(3)),
 *   nu = U0 H sqrt(Pr/Ra), alpha = U0 H / sqrt(Ra Pr), g beta dT = U0^2/H,
 *   tau = 3 nu + 1/2 (Eq. 15), dT = t_wall[W] - t_wall[E] (must be non-zero).
 * mask: ny*nx bytes, 1 = solid obstacle node, may be NULL; copied at create.
 * The state starts at rest, f = w_i, T = grid->t_init, Dirichlet nodes at
 * their wall value.  opts may be NULL (defaults).
 * Returns LBMFVM_ERR_UNSTABLE if tau < 0.51, alpha > 0.25 (explicit diffusion
 * limit), U0^2 > 2 alpha (explicit central advection limit) or Ma > 0.3. */
int lbmfvm_create(const lbmfvm_grid_t *grid, const uint8_t *mask, double Ra, double Pr, double Ma,
                  const lbmfvm_opts_t *opts, lbmfvm_t **out);

/* Create from lattice parameters: kinematic viscosity nu (tau = 3 nu + 1/2),
 * thermal diffusivity alpha, buoyancy coefficient gbeta and an extra uniform
 * body force (force[0], force[1]) (may be NULL), so that the body force per
 * unit mass is G = (force[0], force[1] + gbeta (T - t_ref)) (Eq. 81 with
 * gravity along -y).  Returns LBMFVM_ERR_UNSTABLE if tau < 0.51 or
 * alpha > 0.25. */
int lbmfvm_create_lattice(const lbmfvm_grid_t *grid, const uint8_t *mask, double nu, double alpha,
                          double gbeta, const double *force, const lbmfvm_opts_t *opts,
                          lbmfvm_t **out);

/* Reset the state: f = f_eq(1, (u, v)) (Eq. 8), T as given (Dirichlet nodes
 * are reset to their wall value), step count 0, and the residual snapshot set
 * to this velocity.  u, v, T: ny*nx floats each, host or device; any may be
 * NULL (zero velocity, grid->t_init). */
int lbmfvm_set_state(lbmfvm_t *h, const float *u, const float *v, const float *T);

/* Enqueue n coupled time steps (n >= 0) on the handle's stream and return. */
int lbmfvm_step(lbmfvm_t *h, int64_t n);

/* Fault-injection hook for testing the bounded device-side waits: the next
 * single step launched by lbmfvm_step makes block 0 of the TMA kernel wait for
 * a staged load that is never issued.  That wait gives up after about one
 * second, the kernel records the failure in the handle's device status word
 * and the block returns; the next synchronising call (fields, Nusselt,
 * residual) returns LBMFVM_ERR_TIMEOUT and clears the word.  The state of that
 * step is then incomplete: call lbmfvm_set_state before trusting it again.
 * Nothing faults and the CUDA context stays usable.  Returns LBMFVM_ERR_ARG if
 * the handle runs the generic kernel, which has no such waits. */
int lbmfvm_inject_stall(lbmfvm_t *h);

/* Number of time steps taken since the last set_state. */
int lbmfvm_step_count(const lbmfvm_t *h, int64_t *steps);

/* Macroscopic fields of the current state: density, velocity (lattice units;
 * divide by U0 for the nondimensional U, V of Eq. 85) and temperature.
 * Each pointer may be NULL; otherwise ny*nx values, host or device.  Inert
 * solid nodes report rho = u = v = 0.  Synchronises. */
int lbmfvm_fields(lbmfvm_t *h, double *rho, double *u, double *v, double *T);
int lbmfvm_fields_f32(lbmfvm_t *h, float *rho, float *u, float *v, float *T);

/* Nusselt number of Eq. 90, Nu = -d theta/dX, at the hot west wall from the
 * second-order one-sided difference (-3 T0 + 4 T1 - T2)/2 along each node row,
 * theta = (T - t_wall[E])/(t_wall[W] - t_wall[E]), X = x/H; the mean is the
 * trapezoid integral over Y in [0, 1].  The cold east wall uses the mirrored
 * stencil.  Accumulated in FP64.  local_hot may be NULL, else ny doubles
 * (host or device); either mean pointer may be NULL.  Synchronises. */
int lbmfvm_nusselt(lbmfvm_t *h, double *mean_hot, double *local_hot, double *mean_cold);

/* Steady-state residual ||u^n - u^s||_2 / ||u^n||_2 over fluid nodes in FP64,
 * where u^s is the snapshot taken by the previous call (or by set_state); the
 * current velocity becomes the new snapshot.  Returns LBMFVM_ERR_DIVERGED
 * (with *r set to NaN) if a non-finite velocity was met.  Synchronises. */
int lbmfvm_residual(lbmfvm_t *h, double *r);

/* Step in chunks of check_every, computing the residual after each chunk,
 * until it falls below tol or max_steps steps were taken.  After each check
 * that does not stop the run, the populations are rescaled so that the fluid
 * nodes average rho = 1 (this changes neither u nor T; see the batch notes
 * below).  steps_done and r_final may be NULL. */
int lbmfvm_run_to_steady(lbmfvm_t *h, double tol, int64_t check_every, int64_t max_steps,
                         int64_t *steps_done, double *r_final);

/* Copy the state of src into dst, converting the storage precision: the
 * populations (stored as f - w_i in every precision, Eq. 9 weights), the
 * temperature, the step count and the residual snapshot.  dst keeps its own
 * lattice parameters and mask; the grids must have the same nx and ny
 * (LBMFVM_ERR_ARG otherwise) and the caller keeps the masks equal.  The
 * reduced-precision forms use it to finish a run in FP32 storage once their
 * residual reaches their storage's floor: the iteration then continues
 * exactly as an FP32 run from the converted state.  Runs on dst's stream
 * after src's queued work. */
int lbmfvm_copy_state(lbmfvm_t *dst, lbmfvm_t *src);

/* Number of step-kernel launches lbmfvm_step has issued on this handle (one
 * per coupled step; a CUDA-graph replay counts the launches it holds). */
int lbmfvm_launch_count(const lbmfvm_t *h, int64_t *launches);

/* Step kernel in use (LBMFVM_KERNEL_TMA or LBMFVM_KERNEL_GENERIC) and the TMA
 * tile shape (-1 for the generic kernel); either pointer may be NULL. */
int lbmfvm_kernel_info(const lbmfvm_t *h, int32_t *kernel, int32_t *tma_config);

/* Energy update of the handle: LBMFVM_FV_CENTRAL or LBMFVM_FV_QUICK, and the
 * sub-steps per lattice step (lbmfvm_opts_t.fv_substeps resolved); either
 * pointer may be NULL. */
int lbmfvm_fv_info(const lbmfvm_t *h, int32_t *scheme, int32_t *substeps);

/* Derived lattice parameters: nu, alpha, gbeta, tau (any may be NULL). */
int lbmfvm_params(const lbmfvm_t *h, double *nu, double *alpha, double *gbeta, double *tau);

/* The residual of lbmfvm_residual computed on caller arrays without any
 * device allocation (the paper has no counterpart; this is a service for
 * callers that cannot allocate: code whose device memory belongs to another
 * allocator, such as a framework's caching allocator or a fixed arena, and
 * loops that cannot pay for cudaMalloc's implicit synchronisation).
 *   r = ||(u, v) - (u_prev, v_prev)||_2 / ||(u, v)||_2 in FP64 over the nodes
 *   with select[i] != 0 (all n nodes if select is NULL).
 * u, v, u_prev, v_prev: device arrays of n doubles; select: device array of n
 * bytes or NULL; stream: cudaStream_t to run on (NULL = legacy stream); r: host
 * pointer, written after the stream has been synchronised.
 * Its scratch is a file-scope __device__ array of 8 KB (512 blocks x 2
 * partial sums + 2 totals) that every GPU loading the library keeps until the
 * process exits; n is limited to [1, 2^30] (LBMFVM_ERR_ARG beyond).  The first
 * call on a device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current); make that first call
 * before any stream capture begins.  The call synchronises `stream` and copies
 * the two totals to the host before it returns.  Every call shares the array: calls that overlap
 * on the GPU (on different streams, or from several host threads) race and
 * must be serialised by the caller.  Calls no cudaMalloc, cudaFree or other
 * allocating routine.  Returns LBMFVM_ERR_DIVERGED if a sum is not finite. */
int lbmfvm_residual_noalloc(const double *u, const double *v, const double *u_prev, const double *v_prev,
                            const uint8_t *select, int64_t n, void *stream, double *r);

/* ---- Batches: many cavities advanced by one persistent launch per step ----
 * The cavities (each with its own size, obstacle mask, Ra, Pr and Ma) are
 * packed into one grid, each in its own slot; every step is one launch of the
 * TMA kernel over the tiles of the cavities still active, each tile with its
 * cavity's lattice parameters.  Cavities converge independently: once a
 * cavity's residual drops below the tolerance of lbmfvm_batch_run it leaves
 * the launch and keeps its state.  F32, F16 or BF16 storage, walls on every
 * side; the library allocates the memory (opts->workspace must be NULL); the
 * other options apply to the whole batch.
 * Precision ladder: the rounding of the stored populations puts a floor under
 * the residual, about 1e-3 for F16, 4e-3 for BF16 and 2e-7 to 2e-6 for F32.
 * Above its storage precision a batch keeps packed grids in the wider
 * precisions (F32, then F32X2), created when first needed.  During
 * lbmfvm_batch_run a cavity moves one level up (lbmfvm_copy_state's
 * conversion) when its residual falls below its level's switch value, or when
 * it is within a factor 100 of that value and has not halved for a number of
 * checks (lbmfvm_batch_set_polish; defaults: F16 2e-3, BF16 1e-2, 16 checks;
 * F32 1e-6, 32 checks), and is stepped there until it meets the run's
 * tolerance.  Each step is one launch per level with active cavities.
 * lbmfvm_batch_run also rescales the populations of every active cavity after
 * each residual check so that its fluid nodes average rho = 1: the step is
 * homogeneous of degree one in f (Eq. 18 with the pressure rho0 cs^2,
 * non-equilibrium extrapolation walls Eqs. 94, 96), so this changes neither u
 * nor T, and it undoes the walls' steady mass loss, which would otherwise
 * inflate the stored f - w_i and the rounding of u with it.
 * lbmfvm_run_to_steady does the same for a single handle. */
typedef struct lbmfvm_batch lbmfvm_batch_t;

/* n cavities: grids[i], masks[i] (ny*nx bytes, 1 = solid; masks or masks[i]
 * may be NULL), Ra[i], Pr[i], Ma[i] with the parameter rules and limits of
 * lbmfvm_create.  Every cavity starts at rest with T = grids[i].t_init. */
int lbmfvm_batch_create(int32_t n, const lbmfvm_grid_t *grids, const uint8_t *const *masks, const double *Ra,
                        const double *Pr, const double *Ma, const lbmfvm_opts_t *opts, lbmfvm_batch_t **out);
/* lbmfvm_set_state for cavity i (which becomes active again). */
int lbmfvm_batch_set_state(lbmfvm_batch_t *b, int32_t i, const float *u, const float *v, const float *T);
/* n steps of every active cavity. */
int lbmfvm_batch_step(lbmfvm_batch_t *b, int64_t n);
/* Residual of lbmfvm_residual for every active cavity (snapshots advance);
 * inactive cavities report their last value.  r: n doubles, host. */
int lbmfvm_batch_residuals(lbmfvm_batch_t *b, double *r);
/* Step in chunks of check_every until every cavity's residual is below tol
 * (converged cavities leave the launch) or max_steps steps were taken.
 * steps_out, r_out: n entries each (host, may be NULL): steps taken by each
 * cavity since its set_state and its last residual. */
int lbmfvm_batch_run(lbmfvm_batch_t *b, double tol, int64_t check_every, int64_t max_steps, int64_t *steps_out,
                     double *r_out);
/* lbmfvm_fields and lbmfvm_nusselt for cavity i. */
int lbmfvm_batch_fields(lbmfvm_batch_t *b, int32_t i, double *rho, double *u, double *v, double *T);
int lbmfvm_batch_nusselt(lbmfvm_batch_t *b, int32_t i, double *mean_hot, double *local_hot, double *mean_cold);
/* Steps since set_state, whether cavity i is still stepped, and its lattice
 * parameters nu, alpha, gbeta, tau (params: 4 doubles or NULL). */
int lbmfvm_batch_info(const lbmfvm_batch_t *b, int32_t i, int64_t *steps, int32_t *active, double *params);
/* Energy-update sub-steps per lattice step of cavity i (lbmfvm_opts_t.fv_substeps
 * resolved for that cavity). */
int lbmfvm_batch_substeps(const lbmfvm_batch_t *b, int32_t i, int32_t *substeps);
/* Ladder switch for cavities stepped in precision prec (a level below the
 * top of this batch's ladder, LBMFVM_ERR_ARG otherwise): the residual below
 * which lbmfvm_batch_run moves them one level up, and the number of checks
 * without halving the residual that also moves them (within a factor 100 of
 * r_switch).  r_switch <= 0 keeps them at prec; stall_checks <= 0 turns the
 * second rule off. */
int lbmfvm_batch_set_polish(lbmfvm_batch_t *b, int32_t prec, double r_switch, int32_t stall_checks);
/* TMA tile shape of the batch's packed grid in precision prec (-1 while that
 * level of the ladder has not been created).  Unless opts.tma_config pinned a
 * shape, a level changes its shape with its active set: once cavities have
 * left it and the rest fill fewer tiles than the GPU has SMs, it takes the
 * small-grid shape of LBMFVM_TMA_DEFAULT, and its first shape again when the
 * set grows (shapes never change results). */
int lbmfvm_batch_kernel_info(const lbmfvm_batch_t *b, int32_t prec, int32_t *tma_config);
/* Storage precision cavity i is currently stepped in (lbmfvm_prec). */
int lbmfvm_batch_precision(const lbmfvm_batch_t *b, int32_t i, int32_t *prec);
void lbmfvm_batch_destroy(lbmfvm_batch_t *b);
const char *lbmfvm_batch_last_error(const lbmfvm_batch_t *b);

/* Checkpoints.  The paper runs every case from rest to a steady state and
 * defines no restart; these calls let a long run stop and resume.  A file
 * holds one handle's state: the 256-byte header below (little-endian, the
 * struct's layout has no implicit padding), then the payload:
 *   the nine planes f_i - w_i (f_i for F64) of the current post-collision
 *   state f*^n, [9][ny][nx] in the storage type (2, 4 or 8 bytes; F32X2 as
 *   the (hi, lo) FP32 pairs), then the same for the previous step's f*^(n-1)
 *   (at step 0 the unrelaxed f^0), from which the fields at step n are read;
 *   the temperature T^n, [ny][nx], FP32 (8 bytes for F64 and F32X2);
 *   the residual snapshot u, v of the last residual check, [2][ny][nx] FP64.
 * The CRCs are CRC-32 of the ISO-HDLC polynomial (reflected 0xEDB88320, the
 * one zlib's crc32 computes). */
typedef struct {
    char magic[8];              /* "LBMFVMC1" */
    uint32_t version;           /* 1 */
    uint32_t header_bytes;      /* 256 */
    int32_t nx, ny, store, reserved;
    int64_t steps;              /* steps since set_state */
    int32_t bc[4];              /* lbmfvm_grid_t.bc */
    double t_wall[4], u_lid;    /* lbmfvm_grid_t.t_wall, u_lid */
    double tau, alpha, gbeta, t_ref, force[2]; /* lattice parameters */
    uint64_t payload_bytes;
    uint32_t code_crc;          /* CRC-32 of the handle's node codes (geometry, mask) */
    uint32_t payload_crc;       /* CRC-32 of the payload */
    int32_t fv_scheme;          /* LBMFVM_FV_* of the energy update */
    int32_t fv_substeps;        /* its sub-steps per lattice step (0 is read as 1) */
    int32_t energy;             /* LBMFVM_ENERGY_*; with LBM_D2Q5 the payload ends
                                   with both energy-population buffers, [5][ny][nx]
                                   each in the storage type, stored as g_i - w_i T_0
                                   (T_0 = (t_wall[W] + t_wall[E]) / 2), current
                                   state first */
    int32_t wall_bc;            /* LBMFVM_WALL_* */
    uint8_t pad[76];            /* zero */
    uint32_t header_crc;        /* CRC-32 of the 252 bytes before it */
} lbmfvm_checkpoint_header_t;

/* Write the state of h (after all work enqueued on its stream) to the file
 * at path.  Single-cavity handles only.  Synchronises.  The file is written
 * as path.tmp, flushed to the disk and then renamed over path, so a save that
 * fails part-way leaves any earlier checkpoint at path intact.  LBMFVM_ERR_IO
 * if the file cannot be written; LBMFVM_ERR_TIMEOUT if an earlier step
 * reported a wait that ran out (the state is then not written). */
int lbmfvm_save(lbmfvm_t *h, const char *path);

/* Replace the state of h by the one saved at path: populations,
 * temperature, residual snapshot and step count.  The handle must have the
 * grid, node codes, storage type and lattice parameters the file was saved
 * with (LBMFVM_ERR_ARG otherwise); the file must be complete with matching
 * CRCs (LBMFVM_ERR_IO otherwise).  Nothing on the device changes on an
 * error.  Continuing from a loaded state gives bit for bit the results of
 * the run that saved it.  Synchronises. */
int lbmfvm_load(lbmfvm_t *h, const char *path);

/* Read and verify the checkpoint at path without a GPU: fills *header after
 * checking the magic, version, sizes and all three CRCs (LBMFVM_ERR_IO on
 * any mismatch, a short file or a read error; LBMFVM_ERR_ARG for NULL
 * arguments). */
int lbmfvm_checkpoint_info(const char *path, lbmfvm_checkpoint_header_t *header);

/* Release the handle and any memory the library allocated.  NULL is a no-op. */
void lbmfvm_destroy(lbmfvm_t *h);

/* Message of the last failed call on h (or, for h == NULL, of the last failed
 * create or argument check on this thread).  Never NULL. */
const char *lbmfvm_last_error(const lbmfvm_t *h);

#ifdef __cplusplus
}
#endif

#endif /* LBMFVM_H */
