/*
 * sph.h -- C ABI of the GB300 (sm_103a) implementation of one weakly-
 * compressible SPH time step with the generalised wall boundary treatment of
 * Rezavand, Zhang & Hu, "Generalised and efficient wall boundary condition
 * treatment in GPU-accelerated smoothed particle hydrodynamics" (arXiv
 * 2110.02621).
 *
 * The problem statement follows Sec. 2 and Sec. 3 of the paper: a set of
 * fluid particles (one or two phases) and a fixed set of wall dummy
 * particles, a smoothing length h with support radius 2h, an equation of
 * state per phase, and a one-time upload of the particle data after which
 * every step runs on the device ("copy the simulation data once at the
 * beginning ... and vice versa when we need to save the computational
 * results", Sec. 3).
 *
 * Conventions for every call:
 *   - Every call returns sph_status; nothing is thrown across the ABI.
 *   - Host arrays passed in are copied before the call returns; the caller
 *     keeps ownership.  The library owns all device memory it allocates.
 *   - Positions and velocities are arrays of n*3 doubles (x, y, z of
 *     particle 0, then particle 1, ...), in absolute coordinates.
 *   - Particle identities are the indices of the input arrays ("original
 *     order"); every output is returned in that order unless stated.
 *   - All work is enqueued on the CUDA stream given to sph_create (NULL =
 *     legacy default stream).
 *   - SPH_ERR_CUDA and SPH_ERR_NONFINITE are sticky: afterwards every call
 *     on the context returns SPH_ERR_STATE, except sph_last_error and
 *     sph_destroy.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPH_OK = 0,
    SPH_ERR_ARG = 1,       /* invalid argument: NULL, size, parameter range  */
    SPH_ERR_CUDA = 2,      /* a CUDA runtime call failed (sticky)            */
    SPH_ERR_OOM = 3,       /* device allocation failed                       */
    SPH_ERR_DOMAIN = 4,    /* fluid particles are outside the grid [lo, hi)  */
    SPH_ERR_NONFINITE = 5, /* a non-finite acceleration appeared (sticky)    */
    SPH_ERR_STATE = 6,     /* context unusable after a sticky error          */
    SPH_ERR_UNSUPPORTED = 7, /* the call does not cover this configuration    */
    SPH_ERR_CAPACITY = 8   /* input larger than a fixed-size scratch allows   */
} sph_status;

enum { SPH_EOS_LINEAR = 0, SPH_EOS_TAIT = 1 };
enum { SPH_DENSITY_CONTINUITY = 0, SPH_DENSITY_SUMMATION = 1 };
enum { SPH_REINIT_NONE = 0, SPH_REINIT_FREE_SURFACE = 1, SPH_REINIT_INTERNAL = 2 };
enum { SPH_FP32 = 0, SPH_FP64_PLAIN = 1 };
enum { SPH_HOST = 0, SPH_DEVICE = 1 };

/* One fluid phase (Sec. 2.1: heavy and light phases of a multi-phase flow). */
typedef struct {
    double rho0;     /* reference density rho^0 [kg/m^3], > 0                */
    double mu;       /* dynamic viscosity [Pa s], >= 0 (0: inviscid, as in    *
                      * the paper); laminar form of Morris et al. (1997)     */
    double z_top;    /* top of the phase's column; used only for the          *
                      * hydrostatic start (sph_fluid.rho == NULL)            */
    int32_t eos;     /* SPH_EOS_LINEAR: Eq. (EoS) p = c^2 (rho - rho0);       *
                      * SPH_EOS_TAIT:   p = rho0 c^2/gamma ((rho/rho0)^gamma - 1) */
    int32_t density; /* SPH_DENSITY_CONTINUITY: Eq. (SPH_star_massConservation)
                      * SPH_DENSITY_SUMMATION:  Eq. (densitySummation)       */
    int32_t reinit;  /* SPH_REINIT_FREE_SURFACE: Eq. (eqrhosum);              *
                      * SPH_REINIT_INTERNAL: Eq. (eqrhosumnosurface)         */
    int32_t penalty; /* 1: penalty force F_p, Eq. (SPH_penaltyMethodTerm),   *
                      * on this phase's wall interactions; delta of Eq.      *
                      * (deltaForPenalty) is the signed distance 2 (r_i -   *
                      * r_w).n_w / dx (a barrier behind the wall particle's *
                      * plane), through wall particles that have fluid      *
                      * within 2h on their normal's side in the step        */
} sph_phase;

typedef struct {
    double dp;          /* initial particle spacing dx [m], > 0              */
    double h;           /* smoothing length [m]; support radius 2h; grid cells*
                         * are cubes of side 2h                               */
    double c0;          /* artificial speed of sound, one value for all       *
                         * phases (Sec. 2.6), > 0                             */
    double gamma_tait;  /* Tait exponent (7)                                  */
    double gamma_p;     /* penalty strength gamma_p (1 in the paper)          */
    double cfl;         /* time-step coefficient (0.25, Sec. 2.6)             */
    double g[3];        /* body force [m/s^2]                                 */
    double lo[3];       /* grid origin; particles must stay in [lo, hi)       *
                         * (along non-periodic axes)                         */
    double hi[3];
    int32_t n_phases;   /* 1 or 2                                             */
    int32_t reinit_every; /* density reinitialisation at the start of steps   *
                         * n with n % reinit_every == 0 (the paper: every     *
                         * step, i.e. 1); 0 = only on sph_reinit_density      */
    sph_phase phase[2];
    int32_t precision;  /* SPH_FP32: FP32 pair arithmetic, positions as cell  *
                         * index + FP32 offset with Kahan-compensated drift;  *
                         * SPH_FP64_PLAIN: the same kernels in FP64           */
    int32_t dim;        /* 3 (or 0): 3-D.  2: the 2-D form (Sec. 4.1): every  *
                         * fluid and wall particle in one plane y = const    *
                         * (checked), Wendland C2 with 7/(4 pi h^2), masses  *
                         * rho0 dx^2 per unit depth                          */
    int32_t periodic;   /* bit d (1 = x, 2 = y, 4 = z) set: axis d is         *
                         * periodic with period hi - lo, which must be a      *
                         * whole number >= 3 of 2h cells (to 1e-9); particles *
                         * are wrapped into [lo, hi) at create and after each *
                         * drift, pairs use the nearest image.  Not in the    *
                         * paper (a periodic fluid-only box conserves total   *
                         * momentum by pair antisymmetry).  0 = none; y may   *
                         * not be periodic in 2-D                            */
} sph_params;

/* Fluid particles.  rho may be NULL: each particle then starts from the
 * hydrostatic pressure of the stacked phase columns (phase k spans
 * (z_top[k-1], z_top[k]], gravity along -z) converted by the inverse EOS.
 * phase may be NULL (all phase 0). */
typedef struct {
    int64_t n;
    const double* pos;    /* [n*3] */
    const double* vel;    /* [n*3], may be NULL (at rest) */
    const double* rho;    /* [n] or NULL */
    const int32_t* phase; /* [n] or NULL */
} sph_fluid;

/* Wall dummy particles: fixed for the whole run (Sec. 2.3). */
typedef struct {
    int64_t n;
    const double* pos;    /* [n*3] */
} sph_wall;

/* Output buffers of sph_get_state.  Any pointer may be NULL (skipped).  With
 * where = SPH_HOST they are host memory, with SPH_DEVICE device memory on the
 * context's device.  Fluid arrays are in original order. */
typedef struct {
    double* pos;      /* [n_fluid*3] absolute position                         */
    double* vel;      /* [n_fluid*3]                                           */
    double* rho;      /* [n_fluid] density                                     */
    double* p;        /* [n_fluid] pressure                                    */
    double* acc;      /* [n_fluid*3] dv/dt at the current state                */
    double* drho_dt;  /* [n_fluid] d rho/dt of the last continuity update      */
    double* sigma;    /* [n_fluid] number density sum_j W_ij (self included)   */
    double* pw;       /* [n_wall] wall dummy pressure p_w, Eq. (wallPressure)  */
    double* rhow;     /* [n_wall*2] wall density per fluid phase (EOS^-1 p_w)  */
    double* normal;   /* [n_wall*3] wall normal n_w, Eq. (normalVectors)       */
} sph_state_out;

typedef struct sph_ctx sph_ctx;

/* Create a simulation (Sec. 3: one upload, then device-resident state).
 * Validates the arguments, bins and sorts walls (once) and fluid into the
 * cell grid, computes wall normals (Eq. normalVectors), the initial density
 * and pressure, the wall pressure (Eq. wallPressure) and the initial
 * acceleration (Eq. SPH_star_momentumConservation).  cuda_stream is a
 * cudaStream_t (or NULL).  On success *out owns all device memory until
 * sph_destroy.  Errors: SPH_ERR_ARG, SPH_ERR_OOM, SPH_ERR_CUDA,
 * SPH_ERR_DOMAIN (a particle outside [lo, hi)). */
sph_status sph_create(const sph_params* params, const sph_fluid* fluid,
                      const sph_wall* wall, void* cuda_stream, sph_ctx** out);

/* sph_create with the fluid arrays (pos, vel, rho, phase of *fluid) in
 * device memory of the current device, e.g. tensors a framework already
 * holds there: they are copied on the stream (device to device), so the
 * state never passes through the host (Sec. 3: device-resident state).
 * The struct itself and the walls stay host memory.  The per-particle
 * checks of sph_create (finite positions and velocities, rho > 0, phase in
 * range, one y in 2-D) run as a kernel before any other use, with one
 * synchronisation; a failure returns SPH_ERR_ARG.  The caller keeps its
 * arrays.  Other errors as sph_create. */
sph_status sph_create_device(const sph_params* params, const sph_fluid* fluid,
                             const sph_wall* wall, void* cuda_stream, sph_ctx** out);

/* Advance nsteps kick-drift-kick steps (Sec. 2.6): reinitialise density if
 * due (Eqs. eqrhosum / eqrhosumnosurface), half kick and drift, re-bin and
 * sort, continuity or summation density and EOS, wall pressure, momentum
 * with penalty, viscosity and gravity, final kick.  dt > 0 fixes the step;
 * dt <= 0 takes dt = cfl min(h/(c0 + U_max), sqrt(h/|g|)) on the device.
 * dt_out (may be NULL) receives the last step's dt.  Synchronises the
 * stream once at the end to read the error word.  Errors: SPH_ERR_ARG
 * (nsteps < 0), SPH_ERR_DOMAIN (particles left the grid; they are excluded
 * from all interactions and the count is in sph_last_error),
 * SPH_ERR_NONFINITE, SPH_ERR_CUDA, SPH_ERR_STATE. */
sph_status sph_step(sph_ctx* ctx, int32_t nsteps, double dt, double* dt_out);

/* Enqueue nsteps steps like sph_step and return without waiting for them:
 * the host can queue further work (an L2 flush, events, more steps) while
 * the GPU runs.  Errors of the enqueued steps (SPH_ERR_DOMAIN,
 * SPH_ERR_NONFINITE) are reported by the next sph_sync or sph_step.  A dt
 * different from the previous call's waits for the stream first (the value
 * travels through one pinned word).  Errors: SPH_ERR_ARG, SPH_ERR_CUDA,
 * SPH_ERR_STATE. */
sph_status sph_step_async(sph_ctx* ctx, int32_t nsteps, double dt);

/* Wait for the enqueued steps and report their status as sph_step does;
 * *dt_out (may be NULL) receives the last step's dt. */
sph_status sph_sync(sph_ctx* ctx, double* dt_out);

/* Reinitialise the fluid density now with the number density of the current
 * positions (Eqs. eqrhosum / eqrhosumnosurface per phase mode), and update
 * the pressure.  Errors: SPH_ERR_CUDA, SPH_ERR_STATE. */
sph_status sph_reinit_density(sph_ctx* ctx);

/* Copy the current state into caller buffers (Sec. 3, "save the
 * computational results"), converted to FP64 and original order.  where =
 * SPH_HOST or SPH_DEVICE says where the buffers live; the call synchronises
 * the stream before returning.  Errors: SPH_ERR_ARG, SPH_ERR_CUDA,
 * SPH_ERR_STATE. */
sph_status sph_get_state(sph_ctx* ctx, const sph_state_out* out, int32_t where);

/* Neighbour grid of the context: dims[3] cells per axis, n_cells, cell side
 * (2h).  Any pointer may be NULL. */
sph_status sph_grid_info(const sph_ctx* ctx, int32_t dims[3], int64_t* n_cells,
                         double* cell_size);

/* The cell-linked list (Sec. 3, neighbour search) as host arrays:
 *   key_fluid[id]  cell key (cz*ny + cy)*nx + cx of fluid particle id,
 *                  0xFFFFFFFF outside the grid;
 *   order_fluid[k] id of the particle in sorted slot k (sorted by key, id);
 *   start_fluid[c] first sorted slot of cell c, c in [0, n_cells];
 *                  start_fluid[n_cells] = number of in-grid particles;
 * and the same for the walls.  Any pointer may be NULL.  Synchronises. */
sph_status sph_get_cells(sph_ctx* ctx, uint32_t* key_fluid, int32_t* order_fluid,
                         int32_t* start_fluid, uint32_t* key_wall,
                         int32_t* order_wall, int32_t* start_wall);

/* The neighbour sets of the last neighbour build (Sec. 3: the particles
 * within the support 2h of each fluid particle, found through the 27 cells
 * around its own), as the continuity and momentum sweeps of the last step
 * visited them: for fluid particle i (original id), the original ids of the
 * fluid particles j with 0 < |r_ij| < 2h and of the wall particles w with
 * 0 < |r_iw| < 2h, where |r|^2 is evaluated in the context's precision from
 * the cell-relative positions (the sweeps' own test).  A particle whose
 * list overflowed the fixed list capacity is reported with the set its
 * sweeps scanned from the cells instead.  Particles outside the grid have
 * none.  Host arrays:
 *   fluid_offsets[n_fluid + 1], wall_offsets[n_fluid + 1] (int64): the
 *     neighbours of i are fluid_ids[fluid_offsets[i] .. fluid_offsets[i+1])
 *     and wall_ids[wall_offsets[i] .. wall_offsets[i+1]), ascending;
 *   fluid_ids[fluid_cap], wall_ids[wall_cap] (int32);
 *   overflow[2]: the number of fluid particles whose fluid / wall list
 *     overflowed (and were scanned).
 * Any pointer may be NULL.  Call once with NULL id arrays to learn the
 * totals (fluid_offsets[n_fluid], wall_offsets[n_fluid]); a capacity below
 * the total gives SPH_ERR_ARG with the offsets written.  When the lists no
 * longer hold the build of the current state (after sph_tape kept them with
 * its products, or after sph_backward), the builder runs again on the
 * current state, which reproduces them.  An inspection call, not part of
 * the step: it allocates device memory on the stream and synchronises.
 * Errors: SPH_ERR_ARG, SPH_ERR_CUDA, SPH_ERR_STATE. */
sph_status sph_get_neighbors(sph_ctx* ctx, int64_t* fluid_offsets, int32_t* fluid_ids,
                             int64_t fluid_cap, int64_t* wall_offsets, int32_t* wall_ids,
                             int64_t wall_cap, int64_t overflow[2]);

/* FP64 device reductions of the fluid state: out[8] = {total mass,
 * momentum x, y, z, kinetic energy, potential energy -sum m g.r, U_max,
 * number of particles outside the grid}.  Synchronises. */
sph_status sph_diagnostics(sph_ctx* ctx, double out[8]);

/* The same reductions enqueued on the stream without waiting: the 8 values
 * are copied to out when the stream reaches them (valid after sph_sync or
 * any synchronising call).  where = SPH_DEVICE: out is device memory;
 * SPH_HOST: out must be page-locked host memory (SPH_ERR_ARG otherwise), so
 * that the copy does not block the host.  Successive calls may target
 * different buffers (a ring of per-step results).  Errors: SPH_ERR_ARG,
 * SPH_ERR_CUDA, SPH_ERR_STATE. */
sph_status sph_diagnostics_async(sph_ctx* ctx, double* out, int32_t where);

/* Rigid sinusoidal motion of the tank (all wall particles), x_w(t) = x_w(0) +
 * amp sin(2 pi freq t), t counted from sph_create -- the excitation of the
 * sloshing case of Sec. 4.2.  The run proceeds in the tank's frame, where the
 * walls stay fixed and the body force becomes g - d2x/dt2 = g + amp (2 pi
 * freq)^2 sin(2 pi freq t), evaluated at t^{n+1} in the momentum equation and
 * in the (g - a_w) term of Eq. (wallPressure); fluid velocities relative to
 * the walls enter the Riemann states unchanged.  Positions and velocities are
 * reported in the tank frame (add amp sin(2 pi freq t), amp 2 pi freq
 * cos(2 pi freq t) for the laboratory frame).  amp = 0 or freq = 0 stops the
 * motion.  Synchronises.  Errors: SPH_ERR_ARG, SPH_ERR_CUDA, SPH_ERR_STATE. */
sph_status sph_set_excitation(sph_ctx* ctx, const double amp[3], double freq);

/* Simulated time since sph_create (the sum of the steps' dt).  Synchronises. */
sph_status sph_time(sph_ctx* ctx, double* t);

/* Pressure sensors (the sensors P_i of Sec. 4.3).  The paper defers the
 * sampling to the work it cites; the operation here is the kernel-weighted,
 * Shepard-normalised interpolation over fluid particles: for each point r_k
 * (pts[3k..3k+2], absolute coordinates)
 *   w_k = sum_j V_j W(|r_k - r_j|),  V_j = m_j / rho_j,
 *   p_k = sum_j p_j V_j W(|r_k - r_j|) / w_k   (p_k = 0 where w_k = 0),
 * j over every fluid particle of every phase inside the grid with
 * |r_k - r_j| < 2h (r = r_j included), W the Wendland C2 kernel of the run's
 * dimension; evaluated from the current state between steps, pair terms in
 * the run's precision, sums in FP64.  w_k is
 * the fluid's volume fraction at r_k (about 1 inside the fluid, 1/2 on a flat
 * free surface or a wall face).  Points may lie anywhere, outside the grid
 * included.  p and w (n doubles each; either may be NULL) receive the results.
 * where = SPH_HOST: pts, p and w are host memory and the call synchronises;
 * SPH_DEVICE: device memory, the work is enqueued on the stream and the call
 * returns without waiting (results valid after sph_sync or any synchronising
 * call), so that a sensor time series can be recorded between
 * sph_step_async calls.  Errors: SPH_ERR_ARG (n < 0, pts NULL with n > 0, a
 * non-finite host point), SPH_ERR_CUDA, SPH_ERR_STATE. */
sph_status sph_probe_pressure(sph_ctx* ctx, const double* pts, int32_t n,
                              double* p, double* w, int32_t where);

enum { SPH_GAUGE_MAX_SAMPLES = 65536, SPH_GAUGE_MAX_LINES = 65535 };

/* Wave-height gauges (the gauges H_i of Sec. 4.3).  For each vertical line
 * gauges[4k..4k+3] = (x, y, z_lo, z_hi) (z along -g; in 2-D y is the plane's
 * y), the liquid volume fraction phi(z) = sum_{j in phase 0} V_j
 * W(|(x, y, z) - r_j|) is sampled at z_i = z_lo + i dz, i = 0..K,
 * K = floor((z_hi - z_lo)/dz); the height is the highest sample with
 * phi >= 1/2, moved to the linear interpolate of the crossing with the sample
 * above: H = z_i + dz (phi_i - 1/2)/(phi_i - phi_{i+1}); H = z_lo when no
 * sample reaches 1/2 (a dry line) and z_K when the top one does.  1/2 is the
 * value of phi on the face of a half-space of particles, so H reads the free
 * surface of the first phase (the liquid of a two-phase run); isolated drops
 * (phi below 1/2) are not counted.  Evaluated between steps.  H
 * receives n doubles.  where as for sph_probe_pressure; with SPH_DEVICE a
 * line that is not finite, has z_hi < z_lo or K >= SPH_GAUGE_MAX_SAMPLES
 * yields NaN.  Pair terms are evaluated in the run's precision and summed
 * in FP64 (sph_probe_pressure alike).  Errors: SPH_ERR_ARG (n < 0 or above
 * SPH_GAUGE_MAX_LINES, NULL arrays with n > 0, dz not finite and > 0, such a
 * line in host memory), SPH_ERR_CUDA, SPH_ERR_STATE. */
sph_status sph_gauge_height(sph_ctx* ctx, const double* gauges, int32_t n,
                            double dz, double* H, int32_t where);

/* Counters since creation: steps taken and the summed number of wall
 * particles that had fluid support in each step's wall-pressure sweep.
 * Either pointer may be NULL.  Synchronises. */
sph_status sph_counters(sph_ctx* ctx, int64_t* steps, int64_t* active_wall_steps);

/* Kernel classes of one step, in launch order (cf. the paper's Table 1:
 * mass conservation, momentum conservation, BC pressure, density update,
 * neighbour search including sorting, time integration). */
enum {
    SPH_K_BEGIN_STEP = 0,   /* time step from U_max, clear cell counters      */
    SPH_K_PREDICT = 1,      /* half kick, drift, new cell, cell counts        */
    SPH_K_SCAN = 2,         /* exclusive scan of cell counts (1-3 launches)   */
    SPH_K_SCATTER = 3,      /* first placement by arrival rank                */
    SPH_K_GATHER = 4,       /* (key, id) order, reinitialisation, EOS         */
    SPH_K_NEIGHBORS = 5,    /* per-particle neighbour lists (r < 2h)          */
    SPH_K_CONTINUITY = 6,   /* Riemann continuity / summation density, EOS    */
    SPH_K_WALL_PRESSURE = 7,/* wall dummy pressure, Eq. (wallPressure)        */
    SPH_K_MOMENTUM = 8,     /* momentum, penalty, viscosity, gravity, kick    */
    SPH_K_OTHER = 9,        /* create, export, diagnostics                    */
    SPH_K_ADJ_MOMENTUM = 10,   /* backward of momentum and wall pressure      */
    SPH_K_ADJ_CONTINUITY = 11, /* backward of continuity, kicks, reinit       */
    SPH_K_ADJ_WALL = 12,       /* per-wall adjoints (2 launches per step)     */
    SPH_K_ADJ_OTHER = 13,      /* seeds, permutation, prep, export, restores  */
    SPH_NK = 14
};

/* Per-kernel timing with CUDA events recorded on the context's stream around
 * every launch of the kinds whose bit is set in kind_mask (0 = off).  Resets
 * the accumulated times.  Launch counts are always kept.  Errors:
 * SPH_ERR_CUDA, SPH_ERR_STATE. */
sph_status sph_profile(sph_ctx* ctx, uint32_t kind_mask);

/* Read the profile (synchronises): ms[k] = summed event time of the timed
 * launches of kind k since the last sph_profile call, timed[k] = their
 * number, launches[k] = all launches of kind k since creation.  Each pointer
 * may be NULL; arrays have SPH_NK entries. */
sph_status sph_profile_read(sph_ctx* ctx, double* ms, int64_t* timed, int64_t* launches);

/* ------------------------------------------------------------ adjoint
 * Reverse-mode differentiation of a run of kick-drift-kick steps (Sec. 2.6)
 * through the continuity and momentum equations with the Riemann solver
 * (Eqs. (RSsolution), (SPH_star_massConservation),
 * (SPH_star_momentumConservation)), the wall pressure extrapolation
 * (Eq. (wallPressure)), the wall Riemann pressure (Eq. (RSatWall)), the
 * penalty force (Eq. (SPH_penaltyMethodTerm)), the viscosity and the
 * density reinitialisation (Eq. (eqrhosum)), with each step's neighbour
 * sets frozen and each step's dt a constant.  The differentiated map is
 * (x^0, v^0, rho^0; c0, gamma_p, mu) -> state after the taped steps, where
 * x^0, v^0, rho^0 are the fluid state given to sph_create (when
 * sph_fluid.rho was NULL, rho^0 is the hydrostatic density, whose own
 * dependence on c0 is not differentiated).  One phase with continuity
 * density only (SPH_ERR_UNSUPPORTED otherwise). */

/* Adjoint seed: dL/d(final state), arrays in original particle order, FP64,
 * host or device memory as the `where` argument of sph_backward says.  Any
 * pointer may be NULL (zero). */
typedef struct {
    const double* x;    /* [n_fluid*3] dL/dx of the final positions          */
    const double* v;    /* [n_fluid*3] dL/dv of the final velocities         */
    const double* rho;  /* [n_fluid]   dL/drho of the final densities        */
    const double* pw;   /* [n_wall]    dL/dp_w of the last step's wall
                           pressures (in the order sph_create received)     */
} sph_adjoint_seed;

/* Gradients of L: arrays in original particle order (FP64, caller-owned,
 * host or device memory as `where` says, NULL = not wanted), and the
 * parameter gradients {dL/dc0, dL/dgamma_p, dL/dmu} (host). */
typedef struct {
    double* x;          /* [n_fluid*3] dL/dx^0   */
    double* v;          /* [n_fluid*3] dL/dv^0   */
    double* rho;        /* [n_fluid]   dL/drho^0 */
    double params[3];
} sph_adjoint_grad;

/* Advance nsteps steps like sph_step, recording a checkpoint of the state
 * before each step (about 96 bytes per fluid and 24 per wall particle in the
 * FP32 form, twice that in FP64) and the dt used.  Within the budget set by
 * sph_tape_budget each step also keeps the products its backward reads:
 * its neighbour lists and the state after its sweeps (about 1 KB per fluid
 * and 32 bytes per wall particle in the FP32 form), so that the backward
 * need not recompute it.  Taping must start right after sph_create and
 * continue without untaped steps in between (SPH_ERR_STATE otherwise);
 * nsteps = 0 only records the created state.  Checkpoints and products live
 * until sph_destroy.  Errors: those of sph_step, SPH_ERR_UNSUPPORTED,
 * SPH_ERR_STATE, SPH_ERR_OOM. */
sph_status sph_tape(sph_ctx* ctx, int32_t nsteps, double dt, double* dt_out);

/* Device memory that sph_tape may spend on keeping step products, in bytes:
 * -1 (the default) = half the device memory free when the first product is
 * kept; 0 = keep none (every step is recomputed by the backward).  Steps
 * beyond the budget are recomputed; the gradients are the same bit for bit
 * either way.  Takes effect for steps taped afterwards.  Errors: SPH_ERR_ARG
 * (bytes < -1), SPH_ERR_STATE. */
sph_status sph_tape_budget(sph_ctx* ctx, int64_t bytes);

/* Backward sweep over all taped steps, newest first: each step's products
 * are taken from the tape, or the step is recomputed from its checkpoint
 * (bit-identical, so the neighbour lists are the forward's); then the
 * adjoint kernels run; finally the sweeps of sph_create at r^0 are
 * differentiated.  The context's state is restored afterwards.  The state
 * must still be the taped run's end (SPH_ERR_STATE after untaped steps).
 * Synchronises the stream.  Errors: SPH_ERR_ARG, SPH_ERR_STATE,
 * SPH_ERR_OOM, SPH_ERR_CUDA. */
sph_status sph_backward(sph_ctx* ctx, const sph_adjoint_seed* seed, sph_adjoint_grad* grad,
                        int32_t where);

/* Message of the last error on ctx (or of the last failed sph_create when
 * ctx is NULL).  The string lives until the next call on the context. */
const char* sph_last_error(const sph_ctx* ctx);

/* Free all device memory of the context.  NULL is ignored. */
void sph_destroy(sph_ctx* ctx);

/* Stand-alone neighbour binning (Sec. 3, neighbour search including
 * sorting): for n positions (device array [n*3], FP64) compute each
 * particle's cell key on the grid of cells of side 2h starting at lo with
 * dims[3] cells, the particle order sorted by (key, id) and the first
 * sorted slot of each cell.  Outputs are device arrays: key[n] (per id),
 * order[n], start[n_cells + 1] with n_cells = dims[0]*dims[1]*dims[2].
 * Particles outside the grid get key 0xFFFFFFFF and come last in order.
 * Scratch memory is allocated and freed on the stream inside the call.
 * Limits: every extent >= 1 and n_cells <= 2^24 - 2 (checked factor by
 * factor, before any launch: SPH_ERR_ARG); n <= 2e9.  Cost: each particle
 * finds its rank inside its cell by counting the smaller ids of that cell,
 * so a cell holding k particles costs k^2 reads.  This suits SPH grids
 * (cells of side 2h hold about 20 particles) but not coarse grids over
 * clustered points: a cell of 10^5 points costs 10^10 reads.
 * Errors: SPH_ERR_ARG, SPH_ERR_OOM, SPH_ERR_CUDA. */
sph_status sph_bin_sort(const double* pos, int64_t n, const double lo[3],
                        double h, const int32_t dims[3], uint32_t* key,
                        int32_t* order, int32_t* start, void* cuda_stream);

/* The same binning as sph_bin_sort, for callers that cannot allocate device
 * memory while they run: code whose device memory is all owned by another
 * framework's pool, loops that must not risk an out-of-memory failure or the
 * synchronisation an allocation can cause part-way through, and callers that
 * must not grow the process's device footprint.  The paper has no
 * counterpart; it is a service of this library.
 *
 * Arguments, layout and results are those of sph_bin_sort (device arrays,
 * outputs identical bit for bit).  Its scratch is one fixed array of
 * SPH_BIN_SORT_NOALLOC_SCRATCH bytes inside the library, which every GPU that
 * loads the library keeps until the process exits; the call itself allocates
 * and frees nothing.  The scratch needs 32 bytes per particle, 8 bytes per
 * grid cell and 4 bytes per 1024 cells, each of its 8 parts rounded up to 256
 * bytes (about 1 M particles with 0.2 M cells, or 0.5 M particles with 2 M
 * cells); larger inputs are refused with SPH_ERR_CAPACITY before any work is
 * queued.
 * The first call on each device looks up the array's device address (with
 * that device current), so make that first call outside any CUDA stream
 * capture.  All calls share the one array: calls whose work overlaps on the
 * GPU (two streams, or two host threads) race on it and must be serialised
 * by the caller.  The parts that must start at zero are cleared by each call.
 * Errors: SPH_ERR_ARG, SPH_ERR_CAPACITY, SPH_ERR_CUDA. */
#define SPH_BIN_SORT_NOALLOC_SCRATCH (32u << 20)
sph_status sph_bin_sort_noalloc(const double* pos, int64_t n, const double lo[3],
                                double h, const int32_t dims[3], uint32_t* key,
                                int32_t* order, int32_t* start, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SPH_GB300_H */
