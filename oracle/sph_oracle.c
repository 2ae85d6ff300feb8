/*
 * Plain FP64 CPU oracle of the WCSPH step with the generalised wall boundary
 * treatment of Rezavand, Zhang & Hu, "Generalised and efficient wall
 * boundary condition treatment in GPU-accelerated smoothed particle
 * hydrodynamics" (arXiv 2110.02621).
 *
 * TEST INFRASTRUCTURE ONLY: this file checks the CUDA library and is never
 * part of it.  It shares no code with it.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.
 *
 * Every routine follows one numbered part of the paper (Sec. 2 equations,
 * Sec. 2.6 time integration) in the paper's notation.  Where the paper is
 * silent or garbled, the reading taken is stated beside the code:
 *   - wall pressure (Eq. wallPressure): the (g - a_w) term is weighted by
 *     rho_f, which makes the printed expression dimensionally consistent;
 *     multi-phase weights are W/rho_f (the "divided by rho_f" of Sec. 2.3);
 *   - wall mass m_w = rho^0 dx^3 of the interacting fluid particle's phase,
 *     wall density rho_w from the inverse equation of state of that phase,
 *     kept at or above rho^0/2 (below EOS(rho^0/2) the Tait inverse nears
 *     the edge of its domain p > -rho^0 c^2/gamma, and extrapolations that
 *     average fluid torn to half its density pass it);
 *     walls have zero velocity;
 *   - penalty (Eq. penaltyMethodTerm): delta = 2 (r_i - r_w).n_w / dx, the
 *     signed distance of i from the wall particle's tangent plane in units of
 *     dx/2, positive on the side n_w points to (e_iw of Eq. deltaForPenalty
 *     taken from w to i; with e_iw from i to w, delta < 0 on the fluid side
 *     and lambda would grow with the distance from the wall).  lambda then
 *     rises from 0 at dx/2 in front of the plane and keeps rising behind it:
 *     a barrier.  The penalty acts through a wall particle only while fluid
 *     lies within 2h on the side its normal points to (the fluid-facing
 *     particles): Eq. (normalVectors), a sum over walls alone, turns the
 *     normals of the outer wall layers away from the fluid, and a signed
 *     delta would switch the penalty on at rest through them.  The printed
 *     factors lambda = (1 - delta)^2 / dx and |r_iw|^-2 leave F_p with
 *     three surplus inverse lengths, which the factor dx^3 restores;
 *   - density reinitialisation: free-surface form for continuity-density
 *     phases, internal form for summation-density phases; sigma sums over
 *     the particle's own phase and walls (continuity phases) or over all
 *     particles (summation phases), self included; sigma^0 is the number
 *     density of a full cubic lattice of spacing dx;
 *   - summation density (Eq. densitySummation) sums over all particles and
 *     walls, self included;
 *   - viscosity (absent from the paper, which is inviscid): the laminar form
 *     of Morris et al. (1997); mu = 0 reproduces the paper;
 *   - Tait equation of state p = rho0 c^2/gamma ((rho/rho0)^gamma - 1) is
 *     offered beside the paper's linear Eq. (EoS);
 *   - the wall pressure is evaluated after the density update of a step and
 *     before the momentum equation; the next step's continuity equation uses
 *     that same wall pressure;
 *   - periodic axes (not in the paper; for the momentum-conservation check of
 *     a periodic fluid-only box): positions are wrapped into [lo, hi) after
 *     every drift, neighbour cells wrap around, and pair vectors take the
 *     nearest image.
 */
#include "sph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846
#define KEY_NONE 0xFFFFFFFFu

struct orc_sim {
    orc_params P;
    int64_t nf, nw;
    double *x, *v, *rho, *p, *a, *drho_dt, *sigma;
    int32_t* phase;
    double *xw, *pw, *rhow, *nwall; /* rhow: [nw*2] per fluid phase */
    int* wfront;                    /* 1: fluid within 2h on the normal's side (penalty) */
    /* cell-linked list */
    int32_t nc[3];
    double cs;
    int64_t n_cells;
    uint32_t *key_f, *key_w;
    int64_t *order_f, *order_w;
    int64_t *start_f, *start_w; /* [n_cells + 1] */
    double sigma0;
    int64_t step;
    double last_dt;
    /* rigid sinusoidal tank motion x_w = amp sin(2 pi f t) (Sec. 4.2),
     * simulated in the tank's frame: the body force there is
     * g_eff = g - d2x/dt2 = g + amp (2 pi f)^2 sin(2 pi f t) */
    double t, ex_amp[3], ex_freq, geff[3];
};

static void body_force(orc_sim* s, double t)
{
    double w = 2.0 * PI * s->ex_freq, sw = sin(w * t);
    for (int d = 0; d < 3; d++) s->geff[d] = s->P.g[d] + s->ex_amp[d] * w * w * sw;
}

/* ---------------------------------------------------------------------- */
/* Wendland C2 kernel, support kappa*h with kappa = 2 (Sec. 2.3, Sec. 4:
 * h = 1.3 dx, support radius 2.6 dx).
 *   W(q) = alpha (1 - q/2)^4 (2q + 1),  q = r/h < 2,
 *   alpha = 21/(16 pi h^3) in 3-D, 7/(4 pi h^2) in 2-D (the 2-D tank of
 *   Sec. 4.1).                                                            */
static double wendland_alpha(double h, int32_t dim)
{
    return dim == 2 ? 7.0 / (4.0 * PI * h * h) : 21.0 / (16.0 * PI * h * h * h);
}

double orc_W_dim(double r, double h, int32_t dim)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return wendland_alpha(h, dim) * t * t * t * t * (2.0 * q + 1.0);
}

/* dW/dr of the same kernel: -5 alpha q (1 - q/2)^3 / h. */
double orc_dWdr_dim(double r, double h, int32_t dim)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return -5.0 * wendland_alpha(h, dim) * q * t * t * t / h;
}

double orc_W(double r, double h) { return orc_W_dim(r, h, 3); }
double orc_dWdr(double r, double h) { return orc_dWdr_dim(r, h, 3); }

/* grad_i W_ij = dW/dr * r_ij / |r_ij|  (Eq. SPH_massConservation notation) */
static void grad_W(const double rij[3], double r, double h, int32_t dim, double out[3])
{
    double f = orc_dWdr_dim(r, h, dim) / r;
    out[0] = f * rij[0];
    out[1] = f * rij[1];
    out[2] = f * rij[2];
}

/* ---------------------------------------------------------------------- */
/* Equation of state.  Linear: Eq. (EoS) p = c^2 (rho - rho0).
 * Tait: p = rho0 c^2 / gamma ((rho/rho0)^gamma - 1).                     */
double orc_eos_p(double rho, const orc_phase* ph, double c0, double gamma_tait)
{
    if (ph->eos == ORC_EOS_TAIT)
        return ph->rho0 * c0 * c0 / gamma_tait * (pow(rho / ph->rho0, gamma_tait) - 1.0);
    return c0 * c0 * (rho - ph->rho0);
}

/* inverse of the above: density from pressure (used for wall particles,
 * Sec. 2.3, and for the hydrostatic start). */
double orc_eos_rho(double p, const orc_phase* ph, double c0, double gamma_tait)
{
    if (ph->eos == ORC_EOS_TAIT)
        return ph->rho0 * pow(1.0 + gamma_tait * p / (ph->rho0 * c0 * c0), 1.0 / gamma_tait);
    return ph->rho0 + p / (c0 * c0);
}

/* ---------------------------------------------------------------------- */
/* Inter-particle Riemann problem, Eqs. (LRstates) and (RSsolution):
 *   rho_bar = (rho_L + rho_R)/2
 *   U_bar   = (rho_L U_L + rho_R U_R)/(rho_L + rho_R)
 *   P_bar   = (rho_L p_R + rho_R p_L)/(rho_L + rho_R)
 *   U*      = U_bar + (p_L - p_R) / (2 c rho_bar)
 *   p*      = P_bar + rho_L rho_R beta (U_L - U_R)/(rho_L + rho_R)
 *   beta    = min(3 max(U_L - U_R, 0), c)           (limiter, Sec. 2.2)
 * With limiter = 0 the dissipation term is dropped, which is Eq. (RSatWall)
 * for the fluid-wall pair.  out = {U*, p*, U_bar, P_bar}.                 */
void orc_riemann(double rhoL, double UL, double pL, double rhoR, double UR,
                 double pR, double c, int32_t limiter, double out[4])
{
    double rho_bar = 0.5 * (rhoL + rhoR);
    double U_bar = (rhoL * UL + rhoR * UR) / (rhoL + rhoR);
    double P_bar = (rhoL * pR + rhoR * pL) / (rhoL + rhoR);
    double Ustar = U_bar + 0.5 * (pL - pR) / (c * rho_bar);
    double pstar = P_bar;
    if (limiter) {
        double beta = fmin(3.0 * fmax(UL - UR, 0.0), c);
        pstar += rhoL * rhoR * beta * (UL - UR) / (rhoL + rhoR);
    }
    out[0] = Ustar;
    out[1] = pstar;
    out[2] = U_bar;
    out[3] = P_bar;
}

/* sigma^0: number density sum_j W of a full cubic lattice of spacing dp,
 * self included (the "initial reference" of Eq. eqrhosum). */
double orc_lattice_sigma0_dim(double dp, double h, int32_t dim)
{
    int K = (int)ceil(2.0 * h / dp) + 1;
    int KY = dim == 2 ? 0 : K; /* 2-D: the x-z plane of the lattice */
    double s = 0.0;
    for (int i = -K; i <= K; i++)
        for (int j = -KY; j <= KY; j++)
            for (int k = -K; k <= K; k++) {
                double r = dp * sqrt((double)(i * i + j * j + k * k));
                s += orc_W_dim(r, h, dim);
            }
    return s;
}

double orc_lattice_sigma0(double dp, double h) { return orc_lattice_sigma0_dim(dp, h, 3); }

/* ---------------------------------------------------------------------- */
/* neighbour search: cell-linked list with cells of side 2h (Sec. 3, item d) */

static int is_periodic(const orc_sim* s, int d);
static void nearest_image(const orc_sim* s, double r[3]);

static uint32_t cell_key(const orc_sim* s, const double x[3], int32_t c[3])
{
    int inside = 1;
    for (int d = 0; d < 3; d++) {
        c[d] = (int32_t)floor((x[d] - s->P.lo[d]) / s->cs);
        if (is_periodic(s, d)) { /* x is wrapped; rounding may leave it one cell off */
            if (c[d] >= s->nc[d]) c[d] -= s->nc[d];
            if (c[d] < 0) c[d] += s->nc[d];
        }
        if (c[d] < 0 || c[d] >= s->nc[d]) inside = 0;
    }
    if (!inside) return KEY_NONE;
    return (uint32_t)(((int64_t)c[2] * s->nc[1] + c[1]) * s->nc[0] + c[0]);
}

typedef struct { uint32_t key; int64_t id; } key_id;

static int cmp_key_id(const void* a, const void* b)
{
    const key_id* p = (const key_id*)a;
    const key_id* q = (const key_id*)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return (p->id > q->id) - (p->id < q->id);
}

/* keys of all particles; order = ids sorted by (key, id); start[c] = first
 * sorted slot of cell c, start[n_cells] = number of in-grid particles. */
static void build_cells(orc_sim* s, int64_t n, const double* x, uint32_t* key,
                        int64_t* order, int64_t* start)
{
    key_id* tmp = (key_id*)malloc(sizeof(key_id) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        int32_t c[3];
        key[i] = cell_key(s, x + 3 * i, c);
        tmp[i].key = key[i];
        tmp[i].id = i;
    }
    qsort(tmp, (size_t)n, sizeof(key_id), cmp_key_id);
    int64_t k = 0;
    for (int64_t c = 0; c <= s->n_cells; c++) {
        while (k < n && tmp[k].key < (uint32_t)c) k++;
        start[c] = k;
    }
    for (int64_t i = 0; i < n; i++) order[i] = tmp[i].id;
    free(tmp);
}

/* visit the particles of the 27 cells around position x, calling fn for
 * each candidate j with r_ij = x - x_j and r = |r_ij| when 0 < r < 2h. */
typedef void (*visit_fn)(void* ctx, int64_t j, const double rij[3], double r);

static void for_neighbors(const orc_sim* s, const double* xi, const double* xs,
                          const int64_t* order, const int64_t* start,
                          visit_fn fn, void* ctx)
{
    int32_t c[3];
    if (cell_key(s, xi, c) == KEY_NONE) return;
    double rc2 = 4.0 * s->P.h * s->P.h;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int32_t q[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
                for (int d = 0; d < 3; d++)
                    if (is_periodic(s, d)) q[d] = (q[d] + s->nc[d]) % s->nc[d];
                if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= s->nc[0] ||
                    q[1] >= s->nc[1] || q[2] >= s->nc[2])
                    continue;
                int64_t cc = ((int64_t)q[2] * s->nc[1] + q[1]) * s->nc[0] + q[0];
                for (int64_t k = start[cc]; k < start[cc + 1]; k++) {
                    int64_t j = order[k];
                    double rij[3] = {xi[0] - xs[3 * j], xi[1] - xs[3 * j + 1],
                                     xi[2] - xs[3 * j + 2]};
                    if (s->P.periodic) nearest_image(s, rij);
                    double r2 = rij[0] * rij[0] + rij[1] * rij[1] + rij[2] * rij[2];
                    if (r2 >= rc2 || r2 == 0.0) continue; /* self and r = 0 skipped */
                    fn(ctx, j, rij, sqrt(r2));
                }
            }
}

static int in_grid(const orc_sim* s, int64_t i)
{
    return s->key_f[i] != KEY_NONE;
}

static int is_periodic(const orc_sim* s, int d) { return (s->P.periodic >> d) & 1; }

/* the nearest periodic image of a pair vector */
static void nearest_image(const orc_sim* s, double r[3])
{
    for (int d = 0; d < 3; d++)
        if (is_periodic(s, d)) {
            double L = s->P.hi[d] - s->P.lo[d];
            r[d] -= L * floor(r[d] / L + 0.5);
        }
}

/* a position wrapped into [lo, hi) along the periodic axes */
static void wrap_position(const orc_sim* s, double x[3])
{
    for (int d = 0; d < 3; d++)
        if (is_periodic(s, d)) {
            double L = s->P.hi[d] - s->P.lo[d];
            double u = fmod(x[d] - s->P.lo[d], L);
            if (u < 0.0) u += L;
            x[d] = s->P.lo[d] + u;
        }
}

/* dx^3, or dx^2 in 2-D: the volume of a particle (per unit depth in 2-D);
 * m = rho^0 dx^dim (reading R20) */
static double volume(const orc_sim* s)
{
    double d = s->P.dp;
    return s->P.dim == 2 ? d * d : d * d * d;
}

static double W_of(const orc_sim* s, double r) { return orc_W_dim(r, s->P.h, s->P.dim); }

/* ---------------------------------------------------------------------- */
/* wall unit normals, Eq. (normalVectors): n_w = Psi/|Psi| with
 * Psi = - sum_{j in wall} (m_j/rho_j) grad_w W_wj, m_j/rho_j = dx^3.
 * |Psi| below 1e-6/dx (a wall particle with symmetric wall support) gives
 * n_w = 0. */
typedef struct { const orc_sim* s; double psi[3]; } normal_ctx;

static void normal_visit(void* vctx, int64_t j, const double rij[3], double r)
{
    (void)j;
    normal_ctx* c = (normal_ctx*)vctx;
    double g[3], V = volume(c->s);
    grad_W(rij, r, c->s->P.h, c->s->P.dim, g);
    for (int d = 0; d < 3; d++) c->psi[d] -= V * g[d];
}

static void wall_normals(orc_sim* s)
{
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < s->nw; w++) {
        normal_ctx c = {s, {0.0, 0.0, 0.0}};
        for_neighbors(s, s->xw + 3 * w, s->xw, s->order_w, s->start_w, normal_visit, &c);
        double m = sqrt(c.psi[0] * c.psi[0] + c.psi[1] * c.psi[1] + c.psi[2] * c.psi[2]);
        for (int d = 0; d < 3; d++)
            s->nwall[3 * w + d] = (m >= 1e-6 / s->P.dp) ? c.psi[d] / m : 0.0;
    }
}

/* ---------------------------------------------------------------------- */
/* wall dummy pressure, Eq. (wallPressure) with a_w = 0 (fixed walls):
 *   p_w = sum_f (p_f + rho_f (g - a_w).r_wf) w_wf / sum_f w_wf,
 *   r_wf = r_w - r_f,  w_wf = W_wf (one phase) or W_wf / rho_f (several).
 * Empty support: p_w = 0.  Wall density rho_w = EOS^-1(p_w) per phase.
 * The same pass marks the fluid-facing wall particles of the penalty: some
 * fluid f of the support with (r_f - r_w).n_w > 0. */
typedef struct { const orc_sim* s; int64_t w; double num, den; int front; } wallp_ctx;

static void wallp_visit(void* vctx, int64_t f, const double rwf[3], double r)
{
    wallp_ctx* c = (wallp_ctx*)vctx;
    const orc_sim* s = c->s;
    if (!in_grid(s, f)) return;
    double W = W_of(s, r);
    double w = (s->P.n_phases > 1) ? W / s->rho[f] : W;
    double gr = s->geff[0] * rwf[0] + s->geff[1] * rwf[1] + s->geff[2] * rwf[2];
    c->num += (s->p[f] + s->rho[f] * gr) * w;
    c->den += w;
    const double* n = s->nwall + 3 * c->w;
    if (rwf[0] * n[0] + rwf[1] * n[1] + rwf[2] * n[2] < 0.0) c->front = 1;
}

static void wall_pressure(orc_sim* s)
{
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < s->nw; w++) {
        wallp_ctx c = {s, w, 0.0, 0.0, 0};
        for_neighbors(s, s->xw + 3 * w, s->x, s->order_f, s->start_f, wallp_visit, &c);
        double pw = (c.den > 0.0) ? c.num / c.den : 0.0;
        s->pw[w] = pw;
        s->wfront[w] = c.front;
        for (int k = 0; k < 2; k++) {
            int kk = k < s->P.n_phases ? k : 0;
            const orc_phase* ph = &s->P.phase[kk];
            /* rho_w = EOS^-1(p_w), kept at or above rho0/2 */
            double p_half = orc_eos_p(0.5 * ph->rho0, ph, s->P.c0, s->P.gamma_tait);
            s->rhow[2 * w + k] = pw < p_half ? 0.5 * ph->rho0
                                             : orc_eos_rho(pw, ph, s->P.c0, s->P.gamma_tait);
        }
    }
}

/* ---------------------------------------------------------------------- */
/* number density sigma_i = sum_j W_ij (self included), Sec. 2.5.  The set
 * of j: own phase and walls for continuity-density phases, everything for
 * summation-density phases. */
typedef struct { const orc_sim* s; int64_t i; int all; double sum; } sigma_ctx;

static void sigma_visit_f(void* vctx, int64_t j, const double rij[3], double r)
{
    (void)rij;
    sigma_ctx* c = (sigma_ctx*)vctx;
    if (!in_grid(c->s, j)) return;
    if (!c->all && c->s->phase[j] != c->s->phase[c->i]) return;
    c->sum += W_of(c->s, r);
}

static void sigma_visit_w(void* vctx, int64_t w, const double rij[3], double r)
{
    (void)w; (void)rij;
    sigma_ctx* c = (sigma_ctx*)vctx;
    c->sum += W_of(c->s, r);
}

static double number_density(const orc_sim* s, int64_t i)
{
    const orc_phase* ph = &s->P.phase[s->phase[i]];
    sigma_ctx c = {s, i, ph->density == ORC_DENSITY_SUMMATION, W_of(s, 0.0)};
    for_neighbors(s, s->x + 3 * i, s->x, s->order_f, s->start_f, sigma_visit_f, &c);
    for_neighbors(s, s->x + 3 * i, s->xw, s->order_w, s->start_w, sigma_visit_w, &c);
    return c.sum;
}

static void compute_sigma(orc_sim* s)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s->nf; i++)
        s->sigma[i] = in_grid(s, i) ? number_density(s, i) : 0.0;
}

/* density reinitialisation, Eqs. (eqrhosum) and (eqrhosumnosurface):
 *   free surface: rho = rho0 s/s0 + max(0, rho* - rho0 s/s0) rho0/rho*
 *   internal:     rho = rho0 s/s0                                          */
static void reinit_density(orc_sim* s)
{
    compute_sigma(s);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s->nf; i++) {
        if (!in_grid(s, i)) continue;
        const orc_phase* ph = &s->P.phase[s->phase[i]];
        double rho_num = ph->rho0 * s->sigma[i] / s->sigma0;
        double rho_star = s->rho[i];
        if (ph->reinit == ORC_REINIT_FREE_SURFACE)
            s->rho[i] = rho_num + fmax(0.0, rho_star - rho_num) * ph->rho0 / rho_star;
        else if (ph->reinit == ORC_REINIT_INTERNAL)
            s->rho[i] = rho_num;
        s->p[i] = orc_eos_p(s->rho[i], ph, s->P.c0, s->P.gamma_tait);
    }
}

/* ---------------------------------------------------------------------- */
/* continuity with the Riemann solution, Eq. (SPH_star_massConservation):
 *   d rho_i/dt = 2 rho_i sum_j (m_j/rho_j) (v_i - v*) . grad_i W_ij
 *   v* = U* e_ij + ((rho_i v_i + rho_j v_j)/(rho_i + rho_j) - U_bar e_ij)
 *   e_ij = -r_ij/|r_ij|, states from Eq. (LRstates).
 * Walls enter with v_w = 0, (rho_w, p_w), m_w = rho0_i dx^3; U* still comes
 * from Eq. (RSsolution) (Sec. 2.3). */
typedef struct { const orc_sim* s; int64_t i; const double* vel; double sum; } cont_ctx;

static void cont_term(cont_ctx* c, const double rij[3], double r, double rho_j,
                      double p_j, const double v_j[3], double m_j)
{
    const orc_sim* s = c->s;
    int64_t i = c->i;
    const double* v_i = c->vel + 3 * i;
    double rho_i = s->rho[i], p_i = s->p[i];
    double e[3] = {-rij[0] / r, -rij[1] / r, -rij[2] / r};
    double UL = v_i[0] * e[0] + v_i[1] * e[1] + v_i[2] * e[2];
    double UR = v_j[0] * e[0] + v_j[1] * e[1] + v_j[2] * e[2];
    double rs[4];
    orc_riemann(rho_i, UL, p_i, rho_j, UR, p_j, s->P.c0, 1, rs);
    double Ustar = rs[0], U_bar = rs[2];
    double gw[3];
    grad_W(rij, r, s->P.h, s->P.dim, gw);
    double dot = 0.0;
    for (int d = 0; d < 3; d++) {
        double vmix = (rho_i * v_i[d] + rho_j * v_j[d]) / (rho_i + rho_j);
        double vstar = Ustar * e[d] + (vmix - U_bar * e[d]);
        dot += (v_i[d] - vstar) * gw[d];
    }
    c->sum += 2.0 * rho_i * (m_j / rho_j) * dot;
}

static void cont_visit_f(void* vctx, int64_t j, const double rij[3], double r)
{
    cont_ctx* c = (cont_ctx*)vctx;
    const orc_sim* s = c->s;
    if (!in_grid(s, j)) return;
    double m_j = s->P.phase[s->phase[j]].rho0 * volume(s);
    cont_term(c, rij, r, s->rho[j], s->p[j], c->vel + 3 * j, m_j);
}

static void cont_visit_w(void* vctx, int64_t w, const double rij[3], double r)
{
    cont_ctx* c = (cont_ctx*)vctx;
    const orc_sim* s = c->s;
    int ph = s->phase[c->i];
    double m_w = s->P.phase[ph].rho0 * volume(s);
    double zero[3] = {0.0, 0.0, 0.0};
    cont_term(c, rij, r, s->rhow[2 * w + ph], s->pw[w], zero, m_w);
}

static double continuity_rate(const orc_sim* s, int64_t i, const double* vel)
{
    cont_ctx c = {s, i, vel, 0.0};
    for_neighbors(s, s->x + 3 * i, s->x, s->order_f, s->start_f, cont_visit_f, &c);
    for_neighbors(s, s->x + 3 * i, s->xw, s->order_w, s->start_w, cont_visit_w, &c);
    return c.sum;
}

/* summation density, Eq. (densitySummation): rho_i = m_i sum_j W_ij over all
 * particles and walls, self included. */
typedef struct { const orc_sim* s; double sum; } sum_ctx;

static void sum_visit_f(void* vctx, int64_t j, const double rij[3], double r)
{
    (void)rij;
    sum_ctx* c = (sum_ctx*)vctx;
    if (!in_grid(c->s, j)) return;
    c->sum += W_of(c->s, r);
}

static void sum_visit_w(void* vctx, int64_t w, const double rij[3], double r)
{
    (void)w; (void)rij;
    sum_ctx* c = (sum_ctx*)vctx;
    c->sum += W_of(c->s, r);
}

static double summation_density(const orc_sim* s, int64_t i)
{
    const orc_phase* ph = &s->P.phase[s->phase[i]];
    double m_i = ph->rho0 * volume(s);
    sum_ctx c = {s, W_of(s, 0.0)};
    for_neighbors(s, s->x + 3 * i, s->x, s->order_f, s->start_f, sum_visit_f, &c);
    for_neighbors(s, s->x + 3 * i, s->xw, s->order_w, s->start_w, sum_visit_w, &c);
    return m_i * c.sum;
}

/* ---------------------------------------------------------------------- */
/* momentum, Eq. (momentumGeneral) discretised as
 * Eq. (SPH_star_momentumConservation):
 *   dv_i/dt = -2 sum_j m_j p* / (rho_i rho_j) grad_i W_ij + g + F_p (+ visc)
 * fluid-fluid p* from Eq. (RSsolution) with the limiter; fluid-wall p* from
 * Eq. (RSatWall).  Penalty F_p, Eqs. (SPH_penaltyMethodTerm), (symbc),
 * (deltaForPenalty), for phases with the penalty flag:
 *   F_p = -2 sum_w m_w/(rho_i rho_w) P n_w dx^3 |r_iw|^-2 dW/dr,
 *   P = gamma_p lambda |p_i e_iw.n_w|, lambda = (1-delta)^2/dx if delta < 1,
 *   delta = 2 r_iw . n_w / dx (signed), r_iw = r_i - r_w,
 * through fluid-facing wall particles only (wfront).
 * Viscosity (Morris et al. 1997):
 *   sum_j m_j (mu_i + mu_j) (r_ij . grad_i W_ij) v_ij / (rho_i rho_j (r^2 + 0.01 h^2)). */
typedef struct { const orc_sim* s; int64_t i; const double* vel; double a[3]; } mom_ctx;

static void viscous_term(mom_ctx* c, const double rij[3], double r, double rho_j,
                         double mu_j, const double v_j[3], double m_j)
{
    const orc_sim* s = c->s;
    int64_t i = c->i;
    double mu_i = s->P.phase[s->phase[i]].mu;
    if (mu_i + mu_j == 0.0) return;
    double gw[3];
    grad_W(rij, r, s->P.h, s->P.dim, gw);
    double rg = rij[0] * gw[0] + rij[1] * gw[1] + rij[2] * gw[2];
    double k = m_j * (mu_i + mu_j) * rg /
               (s->rho[i] * rho_j * (r * r + 0.01 * s->P.h * s->P.h));
    for (int d = 0; d < 3; d++) c->a[d] += k * (c->vel[3 * i + d] - v_j[d]);
}

static void mom_visit_f(void* vctx, int64_t j, const double rij[3], double r)
{
    mom_ctx* c = (mom_ctx*)vctx;
    const orc_sim* s = c->s;
    if (!in_grid(s, j)) return;
    int64_t i = c->i;
    const double *v_i = c->vel + 3 * i, *v_j = c->vel + 3 * j;
    double e[3] = {-rij[0] / r, -rij[1] / r, -rij[2] / r};
    double UL = v_i[0] * e[0] + v_i[1] * e[1] + v_i[2] * e[2];
    double UR = v_j[0] * e[0] + v_j[1] * e[1] + v_j[2] * e[2];
    double rs[4];
    orc_riemann(s->rho[i], UL, s->p[i], s->rho[j], UR, s->p[j], s->P.c0, 1, rs);
    double pstar = rs[1];
    const orc_phase* phj = &s->P.phase[s->phase[j]];
    double m_j = phj->rho0 * volume(s);
    double gw[3];
    grad_W(rij, r, s->P.h, s->P.dim, gw);
    for (int d = 0; d < 3; d++) c->a[d] += -2.0 * m_j * pstar / (s->rho[i] * s->rho[j]) * gw[d];
    viscous_term(c, rij, r, s->rho[j], phj->mu, v_j, m_j);
}

static void mom_visit_w(void* vctx, int64_t w, const double rij[3], double r)
{
    mom_ctx* c = (mom_ctx*)vctx;
    const orc_sim* s = c->s;
    int64_t i = c->i;
    int ph = s->phase[i];
    const orc_phase* phi = &s->P.phase[ph];
    double rho_i = s->rho[i], p_i = s->p[i];
    double rho_w = s->rhow[2 * w + ph], p_w = s->pw[w];
    double m_w = phi->rho0 * volume(s);
    /* Eq. (RSatWall) */
    double pstar = (rho_i * p_w + rho_w * p_i) / (rho_i + rho_w);
    double gw[3];
    grad_W(rij, r, s->P.h, s->P.dim, gw);
    for (int d = 0; d < 3; d++) c->a[d] += -2.0 * m_w * pstar / (rho_i * rho_w) * gw[d];
    double zero[3] = {0.0, 0.0, 0.0};
    viscous_term(c, rij, r, rho_w, phi->mu, zero, m_w);
    if (phi->penalty && s->wfront[w] && r > 1e-6 * s->P.dp) {
        const double* n_w = s->nwall + 3 * w;
        double e[3] = {-rij[0] / r, -rij[1] / r, -rij[2] / r}; /* e_iw */
        double en = e[0] * n_w[0] + e[1] * n_w[1] + e[2] * n_w[2];
        double dx = s->P.dp;
        double delta = -2.0 * r / dx * en; /* = 2 r_iw . n_w / dx, signed */
        double lambda = (delta < 1.0) ? (1.0 - delta) * (1.0 - delta) / dx : 0.0;
        double Ppen = s->P.gamma_p * lambda * fabs(p_i * en);
        double k = -2.0 * m_w / (rho_i * rho_w) * Ppen * (dx * dx * dx) / (r * r) *
                   orc_dWdr_dim(r, s->P.h, s->P.dim);
        for (int d = 0; d < 3; d++) c->a[d] += k * n_w[d];
    }
}

static void acceleration(const orc_sim* s, int64_t i, const double* vel, double out[3])
{
    mom_ctx c = {s, i, vel, {0.0, 0.0, 0.0}};
    for_neighbors(s, s->x + 3 * i, s->x, s->order_f, s->start_f, mom_visit_f, &c);
    for_neighbors(s, s->x + 3 * i, s->xw, s->order_w, s->start_w, mom_visit_w, &c);
    for (int d = 0; d < 3; d++) out[d] = c.a[d] + s->geff[d];
}

static void momentum(orc_sim* s, const double* vel)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s->nf; i++) {
        if (!in_grid(s, i)) {
            s->a[3 * i] = s->a[3 * i + 1] = s->a[3 * i + 2] = 0.0;
            continue;
        }
        acceleration(s, i, vel, s->a + 3 * i);
    }
}

/* ---------------------------------------------------------------------- */
/* time step limits (Sec. 2.6): dt <= 0.25 h/(c + U_max), dt <= 0.25 sqrt(h/|g|),
 * with the coefficient taken from params.cfl. */
static double max_speed(const orc_sim* s)
{
    double u = 0.0;
    for (int64_t i = 0; i < s->nf; i++) {
        if (!in_grid(s, i)) continue;
        const double* v = s->v + 3 * i;
        u = fmax(u, sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    }
    return u;
}

static double time_step(const orc_sim* s)
{
    double dt = s->P.cfl * s->P.h / (s->P.c0 + max_speed(s));
    /* body-force limit with the largest |g_eff| of the motion, |g| + |amp| w^2 */
    double gn = sqrt(s->P.g[0] * s->P.g[0] + s->P.g[1] * s->P.g[1] + s->P.g[2] * s->P.g[2]);
    double w = 2.0 * PI * s->ex_freq;
    gn += sqrt(s->ex_amp[0] * s->ex_amp[0] + s->ex_amp[1] * s->ex_amp[1] + s->ex_amp[2] * s->ex_amp[2]) * w * w;
    if (gn > 0.0) dt = fmin(dt, s->P.cfl * sqrt(s->P.h / gn));
    return dt;
}

/* one kick-drift-kick step (Sec. 2.6). */
static double one_step(orc_sim* s, double dt_in)
{
    int64_t nf = s->nf;
    /* density reinitialisation at the beginning of the step */
    if (s->P.reinit_every > 0 && s->step % s->P.reinit_every == 0) reinit_density(s);
    double dt = dt_in > 0.0 ? dt_in : time_step(s);
    /* v^{n+1/2} = v^n + dt/2 a^n;  r^{n+1} = r^n + dt v^{n+1/2} */
    for (int64_t i = 0; i < nf; i++) {
        for (int d = 0; d < 3; d++) {
            s->v[3 * i + d] += 0.5 * dt * s->a[3 * i + d];
            s->x[3 * i + d] += dt * s->v[3 * i + d];
        }
        wrap_position(s, s->x + 3 * i);
    }
    build_cells(s, nf, s->x, s->key_f, s->order_f, s->start_f);
    /* density: continuity (heavy phases) or summation (light phases) */
    double* rho_new = (double*)malloc(sizeof(double) * (size_t)(nf > 0 ? nf : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nf; i++) {
        s->drho_dt[i] = 0.0;
        rho_new[i] = s->rho[i];
        if (!in_grid(s, i)) continue;
        const orc_phase* ph = &s->P.phase[s->phase[i]];
        if (ph->density == ORC_DENSITY_SUMMATION) {
            rho_new[i] = summation_density(s, i);
        } else {
            s->drho_dt[i] = continuity_rate(s, i, s->v);
            rho_new[i] = s->rho[i] + dt * s->drho_dt[i];
        }
    }
    for (int64_t i = 0; i < nf; i++) {
        s->rho[i] = rho_new[i];
        s->p[i] = orc_eos_p(s->rho[i], &s->P.phase[s->phase[i]], s->P.c0, s->P.gamma_tait);
    }
    free(rho_new);
    /* the body force of t^{n+1}, then wall pressure from the updated fluid
     * and momentum at n+1 */
    s->t += dt;
    body_force(s, s->t);
    wall_pressure(s);
    momentum(s, s->v);
    /* v^{n+1} = v^{n+1/2} + dt/2 a^{n+1} */
    for (int64_t i = 0; i < nf; i++)
        for (int d = 0; d < 3; d++) s->v[3 * i + d] += 0.5 * dt * s->a[3 * i + d];
    s->step++;
    s->last_dt = dt;
    return dt;
}

/* ---------------------------------------------------------------------- */

static void* dup(const void* p, size_t bytes)
{
    void* q = malloc(bytes > 0 ? bytes : 1);
    if (p && bytes) memcpy(q, p, bytes);
    else memset(q, 0, bytes > 0 ? bytes : 1);
    return q;
}

/* hydrostatic pressure of a column of stacked phases (phase k between the
 * tops of phases k-1 and k), the analytic still-water state of Sec. 4.1. */
static double hydrostatic_p(const orc_params* P, int k, double z)
{
    double gz = -P->g[2];
    double p = P->phase[k].rho0 * gz * (P->phase[k].z_top - z);
    for (int m = k + 1; m < P->n_phases; m++)
        p += P->phase[m].rho0 * gz * (P->phase[m].z_top - P->phase[m - 1].z_top);
    return p;
}

orc_sim* orc_create(const orc_params* P, int64_t nf, const double* x,
                    const double* v, const double* rho, const int32_t* phase,
                    int64_t nw, const double* xw)
{
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->P = *P;
    if (s->P.dim != 2) s->P.dim = 3;
    body_force(s, 0.0); /* no motion until orc_set_excitation: g_eff = g */
    s->nf = nf;
    s->nw = nw;
    s->cs = 2.0 * P->h;
    s->n_cells = 1;
    for (int d = 0; d < 3; d++) {
        double u = (P->hi[d] - P->lo[d]) / s->cs;
        if ((P->periodic >> d) & 1) {
            s->nc[d] = (int32_t)floor(u + 0.5);
            if (s->nc[d] < 3 || fabs(u - s->nc[d]) > 1e-9 * (double)s->nc[d]) {
                free(s);
                return NULL;
            }
        } else {
            s->nc[d] = (int32_t)ceil(u);
            if (s->nc[d] < 1) s->nc[d] = 1;
        }
        s->n_cells *= s->nc[d];
    }
    size_t f3 = sizeof(double) * 3 * (size_t)nf, f1 = sizeof(double) * (size_t)nf;
    s->x = (double*)dup(x, f3);
    s->v = (double*)dup(v, f3);
    s->rho = (double*)dup(NULL, f1);
    s->p = (double*)dup(NULL, f1);
    s->a = (double*)dup(NULL, f3);
    s->drho_dt = (double*)dup(NULL, f1);
    s->sigma = (double*)dup(NULL, f1);
    s->phase = (int32_t*)dup(phase, sizeof(int32_t) * (size_t)nf);
    s->xw = (double*)dup(xw, sizeof(double) * 3 * (size_t)nw);
    s->pw = (double*)dup(NULL, sizeof(double) * (size_t)nw);
    s->rhow = (double*)dup(NULL, sizeof(double) * 2 * (size_t)nw);
    s->nwall = (double*)dup(NULL, sizeof(double) * 3 * (size_t)nw);
    s->wfront = (int*)calloc((size_t)(nw > 0 ? nw : 1), sizeof(int));
    s->key_f = (uint32_t*)dup(NULL, sizeof(uint32_t) * (size_t)nf);
    s->order_f = (int64_t*)dup(NULL, sizeof(int64_t) * (size_t)nf);
    s->start_f = (int64_t*)dup(NULL, sizeof(int64_t) * (size_t)(s->n_cells + 1));
    s->key_w = (uint32_t*)dup(NULL, sizeof(uint32_t) * (size_t)nw);
    s->order_w = (int64_t*)dup(NULL, sizeof(int64_t) * (size_t)nw);
    s->start_w = (int64_t*)dup(NULL, sizeof(int64_t) * (size_t)(s->n_cells + 1));
    if (!phase)
        for (int64_t i = 0; i < nf; i++) s->phase[i] = 0;
    for (int64_t i = 0; i < nf; i++) wrap_position(s, s->x + 3 * i);

    build_cells(s, nw, s->xw, s->key_w, s->order_w, s->start_w);
    build_cells(s, nf, s->x, s->key_f, s->order_f, s->start_f);
    wall_normals(s);
    for (int64_t i = 0; i < nf; i++) {
        const orc_phase* ph = &P->phase[s->phase[i]];
        if (rho) s->rho[i] = rho[i];
        else s->rho[i] = orc_eos_rho(hydrostatic_p(P, s->phase[i], s->x[3 * i + 2]), ph,
                                     P->c0, P->gamma_tait);
        s->p[i] = orc_eos_p(s->rho[i], ph, P->c0, P->gamma_tait);
    }
    s->sigma0 = orc_lattice_sigma0_dim(P->dp, P->h, s->P.dim);
    wall_pressure(s);
    momentum(s, s->v);
    compute_sigma(s);
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    free(s->x); free(s->v); free(s->rho); free(s->p); free(s->a);
    free(s->drho_dt); free(s->sigma); free(s->phase);
    free(s->xw); free(s->pw); free(s->rhow); free(s->nwall); free(s->wfront);
    free(s->key_f); free(s->order_f); free(s->start_f);
    free(s->key_w); free(s->order_w); free(s->start_w);
    free(s);
}

double orc_step(orc_sim* s, int32_t nsteps, double dt)
{
    double last = 0.0;
    for (int32_t k = 0; k < nsteps; k++) last = one_step(s, dt);
    compute_sigma(s);
    return last;
}

void orc_reinit_density(orc_sim* s)
{
    reinit_density(s);
}

void orc_rates(orc_sim* s, double* drho_dt, double* a)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s->nf; i++) {
        if (drho_dt) drho_dt[i] = in_grid(s, i) ? continuity_rate(s, i, s->v) : 0.0;
        if (a) {
            if (in_grid(s, i)) acceleration(s, i, s->v, a + 3 * i);
            else a[3 * i] = a[3 * i + 1] = a[3 * i + 2] = 0.0;
        }
    }
}

void orc_get_fluid(const orc_sim* s, double* x, double* v, double* rho,
                   double* p, double* a, double* drho_dt, double* sigma)
{
    size_t f3 = sizeof(double) * 3 * (size_t)s->nf, f1 = sizeof(double) * (size_t)s->nf;
    if (x) memcpy(x, s->x, f3);
    if (v) memcpy(v, s->v, f3);
    if (rho) memcpy(rho, s->rho, f1);
    if (p) memcpy(p, s->p, f1);
    if (a) memcpy(a, s->a, f3);
    if (drho_dt) memcpy(drho_dt, s->drho_dt, f1);
    if (sigma) memcpy(sigma, s->sigma, f1);
}

void orc_get_wall(const orc_sim* s, double* pw, double* rhow, double* nw)
{
    if (pw) memcpy(pw, s->pw, sizeof(double) * (size_t)s->nw);
    if (rhow) memcpy(rhow, s->rhow, sizeof(double) * 2 * (size_t)s->nw);
    if (nw) memcpy(nw, s->nwall, sizeof(double) * 3 * (size_t)s->nw);
}

int64_t orc_n_cells(const orc_sim* s, int32_t dims[3])
{
    if (dims) for (int d = 0; d < 3; d++) dims[d] = s->nc[d];
    return s->n_cells;
}

void orc_get_cells(const orc_sim* s, uint32_t* key_f, int64_t* order_f,
                   int64_t* start_f, uint32_t* key_w, int64_t* order_w,
                   int64_t* start_w)
{
    size_t nc1 = sizeof(int64_t) * (size_t)(s->n_cells + 1);
    if (key_f) memcpy(key_f, s->key_f, sizeof(uint32_t) * (size_t)s->nf);
    if (order_f) memcpy(order_f, s->order_f, sizeof(int64_t) * (size_t)s->nf);
    if (start_f) memcpy(start_f, s->start_f, nc1);
    if (key_w) memcpy(key_w, s->key_w, sizeof(uint32_t) * (size_t)s->nw);
    if (order_w) memcpy(order_w, s->order_w, sizeof(int64_t) * (size_t)s->nw);
    if (start_w) memcpy(start_w, s->start_w, nc1);
}

typedef struct { int64_t* ids; int64_t max, n; } collect_ctx;

static void collect_visit(void* vctx, int64_t j, const double rij[3], double r)
{
    (void)rij; (void)r;
    collect_ctx* c = (collect_ctx*)vctx;
    if (c->n < c->max) c->ids[c->n] = j;
    c->n++;
}

int64_t orc_neighbors(const orc_sim* s, int64_t i, int64_t* fluid_ids,
                      int64_t max_f, int64_t* n_f, int64_t* wall_ids,
                      int64_t max_w, int64_t* n_w)
{
    collect_ctx cf = {fluid_ids, max_f, 0}, cw = {wall_ids, max_w, 0};
    for_neighbors(s, s->x + 3 * i, s->x, s->order_f, s->start_f, collect_visit, &cf);
    for_neighbors(s, s->x + 3 * i, s->xw, s->order_w, s->start_w, collect_visit, &cw);
    *n_f = cf.n;
    *n_w = cw.n;
    return cf.n + cw.n;
}

void orc_diagnostics(const orc_sim* s, double out[8])
{
    double m_tot = 0, px = 0, py = 0, pz = 0, ek = 0, ep = 0;
    int64_t esc = 0;
    double vol = volume(s);
    for (int64_t i = 0; i < s->nf; i++) {
        double m = s->P.phase[s->phase[i]].rho0 * vol;
        const double *v = s->v + 3 * i, *x = s->x + 3 * i;
        m_tot += m;
        px += m * v[0];
        py += m * v[1];
        pz += m * v[2];
        ek += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        ep -= m * (s->P.g[0] * x[0] + s->P.g[1] * x[1] + s->P.g[2] * x[2]);
        if (!in_grid(s, i)) esc++;
    }
    out[0] = m_tot; out[1] = px; out[2] = py; out[3] = pz;
    out[4] = ek; out[5] = ep; out[6] = max_speed(s); out[7] = (double)esc;
}

double orc_sigma0(const orc_sim* s) { return s->sigma0; }
int64_t orc_step_count(const orc_sim* s) { return s->step; }

int32_t orc_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads((int)n);
#else
    (void)n;
#endif
}

void orc_set_excitation(orc_sim* s, const double amp[3], double freq)
{
    for (int d = 0; d < 3; d++) s->ex_amp[d] = amp[d];
    s->ex_freq = freq;
    body_force(s, s->t);
}

double orc_time(const orc_sim* s) { return s->t; }

/* ---------------------------------------------------------------------- */
/* Pressure sensors and wave-height gauges (Sec. 4.3: the sensors P_i and the
 * gauges H_i of the dam break with an obstacle).  The paper leaves the
 * sampling to the work it cites; the reading taken here is the kernel-
 * weighted (Shepard-normalised) interpolation over fluid particles:
 *   w(r)    = sum_j V_j W(|r - r_j|),        V_j = m_j / rho_j,
 *   p_bar(r) = sum_j p_j V_j W(|r - r_j|) / w(r)   (0 where w = 0),
 * where j runs over every fluid particle inside the grid (all phases) with
 * |r - r_j| < 2h, r = r_j included.  Plain brute force over all particles. */
void orc_probe_pressure(const orc_sim* s, const double* pts, int64_t n,
                        double* p_out, double* w_out)
{
    const double h = s->P.h, rc2 = 4.0 * h * h, V0 = volume(s);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n; k++) {
        const double* r = pts + 3 * k;
        double sw = 0.0, spw = 0.0;
        for (int64_t j = 0; j < s->nf; j++) {
            if (!in_grid(s, j)) continue;
            const double* xj = s->x + 3 * j;
            double dd[3] = {r[0] - xj[0], r[1] - xj[1], r[2] - xj[2]};
            nearest_image(s, dd);
            double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
            if (r2 >= rc2) continue;
            const orc_phase* ph = &s->P.phase[s->phase[j]];
            double Vj = ph->rho0 * V0 / s->rho[j];
            double wj = Vj * W_of(s, sqrt(r2));
            sw += wj;
            spw += s->p[j] * wj;
        }
        if (w_out) w_out[k] = sw;
        if (p_out) p_out[k] = sw > 0.0 ? spw / sw : 0.0;
    }
}

/* liquid volume fraction phi(r) = sum_{j in phase 0} V_j W(|r - r_j|) over
 * the candidate list cand[0..nc) */
static double liquid_fraction(const orc_sim* s, const int64_t* cand, int64_t nc,
                              const double r[3])
{
    const double rc2 = 4.0 * s->P.h * s->P.h, V0 = volume(s);
    double phi = 0.0;
    for (int64_t c = 0; c < nc; c++) {
        int64_t j = cand[c];
        const double* xj = s->x + 3 * j;
        double dd[3] = {r[0] - xj[0], r[1] - xj[1], r[2] - xj[2]};
        nearest_image(s, dd);
        double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
        if (r2 >= rc2) continue;
        phi += s->P.phase[0].rho0 * V0 / s->rho[j] * W_of(s, sqrt(r2));
    }
    return phi;
}

/* Wave-height gauge on the vertical line through (x, y) between z_lo and z_hi
 * (g[4k..4k+3] = x, y, z_lo, z_hi).  Reading: the free surface is where the
 * liquid (phase 0) volume fraction phi falls through 1/2 -- the value on the
 * face of a half-space of uniform particles.  phi is sampled at
 * z_k = z_lo + k dz, k = 0..K, K = floor((z_hi - z_lo)/dz); H is the highest
 * sample k with phi_k >= 1/2, moved up to the linear interpolate of the
 * crossing between k and k + 1: H = z_k + dz (phi_k - 1/2)/(phi_k - phi_{k+1}).
 * H = z_lo when no sample reaches 1/2 (a dry line), z_K when the top sample
 * does.  Only particles within 2h of the line horizontally can contribute;
 * they are collected first. */
void orc_gauge_height(const orc_sim* s, const double* g, int64_t n, double dz, double* H)
{
    const double rc2 = 4.0 * s->P.h * s->P.h;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n; k++) {
        const double x = g[4 * k], y = g[4 * k + 1], zlo = g[4 * k + 2], zhi = g[4 * k + 3];
        int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->nf > 0 ? s->nf : 1));
        int64_t nc = 0;
        for (int64_t j = 0; j < s->nf; j++) {
            if (!in_grid(s, j) || s->phase[j] != 0) continue;
            double dd[3] = {x - s->x[3 * j], y - s->x[3 * j + 1], 0.0};
            nearest_image(s, dd);
            if (dd[0] * dd[0] + dd[1] * dd[1] < rc2) cand[nc++] = j;
        }
        int64_t K = (int64_t)floor((zhi - zlo) / dz);
        double out = zlo;
        double phi_above = 0.0;
        for (int64_t i = K; i >= 0; i--) {
            double r[3] = {x, y, zlo + (double)i * dz};
            double phi = liquid_fraction(s, cand, nc, r);
            if (phi >= 0.5) {
                out = i == K ? r[2] : r[2] + dz * (phi - 0.5) / (phi - phi_above);
                break;
            }
            phi_above = phi;
        }
        H[k] = out;
        free(cand);
    }
}
