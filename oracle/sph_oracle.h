/*
 * Plain FP64 CPU oracle of one weakly-compressible SPH time step with the
 * generalised wall boundary treatment of Rezavand, Zhang & Hu (arXiv
 * 2110.02621).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library.  It
 * shares no source with it, and only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It is deliberately slow and
 * literal: every function follows one equation or step of the paper, in the
 * paper's notation, with no blocking, fusion or reordering.
 *
 * Conventions (state is kept in the caller's original particle order):
 *   positions, velocities: [n*3] interleaved x,y,z, absolute coordinates;
 *   phases: int32 index into params.phase[];
 *   the neighbour grid has cubic cells of side 2h starting at params.lo;
 *   the cell key is (cz*ny + cy)*nx + cx, 0xFFFFFFFF outside the grid.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_EOS_LINEAR = 0, ORC_EOS_TAIT = 1 };
enum { ORC_DENSITY_CONTINUITY = 0, ORC_DENSITY_SUMMATION = 1 };
enum { ORC_REINIT_NONE = 0, ORC_REINIT_FREE_SURFACE = 1, ORC_REINIT_INTERNAL = 2 };

typedef struct {
    double rho0;     /* reference density rho^0 of the phase */
    double mu;       /* dynamic viscosity (0: inviscid, the paper's setting) */
    double z_top;    /* top of the phase's column, for hydrostatic start */
    int32_t eos;     /* ORC_EOS_* */
    int32_t density; /* ORC_DENSITY_* */
    int32_t reinit;  /* ORC_REINIT_* */
    int32_t penalty; /* 1: penalty force F_p on this phase's wall pairs */
} orc_phase;

typedef struct {
    double dp;         /* initial particle spacing dx */
    double h;          /* smoothing length; support radius 2h */
    double c0;         /* artificial speed of sound, shared by all phases */
    double gamma_tait; /* Tait exponent */
    double gamma_p;    /* penalty strength */
    double cfl;        /* time-step coefficient (0.25 in the paper) */
    double g[3];       /* body force */
    double lo[3], hi[3];
    int32_t n_phases;
    int32_t reinit_every; /* reinitialise at steps n with n % k == 0; 0 = never */
    orc_phase phase[2];
    int32_t dim;          /* 3, or 2: particles in one x-z plane (all y equal) */
    int32_t periodic;     /* bit d set: axis d is periodic with period hi - lo, an
                           * integer number (>= 3) of cells of side 2h */
} orc_params;

typedef struct orc_sim orc_sim;

/* kernel and equation of state, exposed for the pins (orc_W, orc_dWdr and
 * orc_lattice_sigma0: 3-D; the _dim forms take dim = 2 or 3) */
double orc_W(double r, double h);
double orc_dWdr(double r, double h);
double orc_W_dim(double r, double h, int32_t dim);
double orc_dWdr_dim(double r, double h, int32_t dim);
double orc_lattice_sigma0_dim(double dp, double h, int32_t dim);
double orc_eos_p(double rho, const orc_phase* ph, double c0, double gamma_tait);
double orc_eos_rho(double p, const orc_phase* ph, double c0, double gamma_tait);
void orc_riemann(double rhoL, double UL, double pL, double rhoR, double UR,
                 double pR, double c, int32_t limiter, double out[4]);
double orc_lattice_sigma0(double dp, double h);

/* rho may be NULL: hydrostatic density from phase z_top and g; returns NULL
 * when a periodic axis is not a whole number (>= 3) of cells */
orc_sim* orc_create(const orc_params* P, int64_t nf, const double* x,
                    const double* v, const double* rho, const int32_t* phase,
                    int64_t nw, const double* xw);
void orc_destroy(orc_sim* s);
/* advance nsteps; dt > 0 fixes the step, otherwise CFL; returns last dt */
double orc_step(orc_sim* s, int32_t nsteps, double dt);
void orc_reinit_density(orc_sim* s);
/* rigid sinusoidal tank motion x = amp sin(2 pi freq t) from now on (t counts
 * from creation), simulated in the tank frame (Sec. 4.2 excitation) */
void orc_set_excitation(orc_sim* s, const double amp[3], double freq);
double orc_time(const orc_sim* s);
/* rates at the current state without advancing */
void orc_rates(orc_sim* s, double* drho_dt, double* a);

/* state access (NULL pointers are skipped) */
void orc_get_fluid(const orc_sim* s, double* x, double* v, double* rho,
                   double* p, double* a, double* drho_dt, double* sigma);
void orc_get_wall(const orc_sim* s, double* pw, double* rhow, double* nw);
int64_t orc_n_cells(const orc_sim* s, int32_t dims[3]);
void orc_get_cells(const orc_sim* s, uint32_t* key_f, int64_t* order_f,
                   int64_t* start_f, uint32_t* key_w, int64_t* order_w,
                   int64_t* start_w);
/* neighbour list of fluid particle i (fluid then wall ids); returns count */
int64_t orc_neighbors(const orc_sim* s, int64_t i, int64_t* fluid_ids,
                      int64_t max_f, int64_t* n_f, int64_t* wall_ids,
                      int64_t max_w, int64_t* n_w);
/* [mass, mom_x, mom_y, mom_z, E_kin, E_pot, U_max, n_escaped] */
void orc_diagnostics(const orc_sim* s, double out[8]);
double orc_sigma0(const orc_sim* s);
int64_t orc_step_count(const orc_sim* s);
int32_t orc_threads(void);
void orc_set_threads(int32_t n); /* OpenMP threads of the following calls */
/* sensors (Sec. 4.3): Shepard-interpolated pressure p_bar and kernel sum w at
 * n points pts[3k..3k+2]; either output may be NULL */
void orc_probe_pressure(const orc_sim* s, const double* pts, int64_t n,
                        double* p_out, double* w_out);
/* wave-height gauges g[4k..4k+3] = (x, y, z_lo, z_hi), samples dz apart */
void orc_gauge_height(const orc_sim* s, const double* g, int64_t n, double dz, double* H);

#ifdef __cplusplus
}
#endif
#endif
