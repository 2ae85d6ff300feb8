// C ABI of the library (declared in include/sph.h): argument validation,
// context lifetime and error reporting around the two compiled forms.
#include <cmath>
#include <cstdio>
#include <new>
#include <string>

#include "sph_internal.h"

struct sph_ctx {
    sph::SimBase* sim = nullptr;
};

namespace {

thread_local std::string g_create_error;

bool finite3(const double* v)
{
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

sph_status bad(std::string* where, const std::string& msg)
{
    *where = msg;
    return SPH_ERR_ARG;
}

// fluid_host: the fluid arrays are host memory and are checked here; device
// arrays are checked by a kernel at create.
sph_status validate(const sph_params* P, const sph_fluid* F, const sph_wall* W, std::string* msg,
                    bool fluid_host = true)
{
    if (!P || !F) return bad(msg, "params and fluid must not be NULL");
    if (!(P->dp > 0) || !(P->h > 0) || !(P->c0 > 0) || !(P->cfl > 0) || !(P->gamma_tait > 0) ||
        !(P->gamma_p >= 0) || !std::isfinite(P->dp + P->h + P->c0 + P->cfl + P->gamma_tait + P->gamma_p))
        return bad(msg, "dp, h, c0, cfl, gamma_tait must be finite and > 0, gamma_p >= 0");
    if (!finite3(P->g) || !finite3(P->lo) || !finite3(P->hi)) return bad(msg, "g, lo, hi must be finite");
    for (int d = 0; d < 3; ++d)
        if (!(P->hi[d] > P->lo[d])) return bad(msg, "hi must exceed lo on every axis");
    if (P->n_phases < 1 || P->n_phases > 2) return bad(msg, "n_phases must be 1 or 2");
    if (P->reinit_every < 0) return bad(msg, "reinit_every must be >= 0");
    if (P->precision != SPH_FP32 && P->precision != SPH_FP64_PLAIN) return bad(msg, "unknown precision");
    if (P->dim != 0 && P->dim != 2 && P->dim != 3) return bad(msg, "dim must be 0, 2 or 3");
    for (int k = 0; k < P->n_phases; ++k) {
        const sph_phase& ph = P->phase[k];
        if (!(ph.rho0 > 0) || !(ph.mu >= 0) || !std::isfinite(ph.rho0 + ph.mu + ph.z_top))
            return bad(msg, "phase rho0 must be > 0, mu >= 0, all finite");
        if (ph.eos < 0 || ph.eos > 1 || ph.density < 0 || ph.density > 1 || ph.reinit < 0 || ph.reinit > 2 ||
            ph.penalty < 0 || ph.penalty > 1)
            return bad(msg, "phase eos/density/reinit/penalty out of range");
    }
    double cs = 2.0 * P->h;
    if (P->periodic & ~7) return bad(msg, "periodic is a mask of bits 1 (x), 2 (y), 4 (z)");
    if (P->dim == 2 && (P->periodic & 2)) return bad(msg, "dim = 2: y cannot be periodic");
    for (int d = 0; d < 3; ++d)
        if ((P->periodic >> d) & 1) {
            const double u = (P->hi[d] - P->lo[d]) / cs, n = std::floor(u + 0.5);
            if (n < 3.0 || std::fabs(u - n) > 1e-9 * n)
                return bad(msg, "a periodic axis must span a whole number (>= 3) of 2h cells");
        }
    double cells = 1.0;
    for (int d = 0; d < 3; ++d) cells *= std::ceil((P->hi[d] - P->lo[d]) / cs);
    if (cells > (double)(sph::scan_max_len() - 2) || cells > 2.0e9)
        return bad(msg, "grid has too many cells (enlarge h or shrink [lo, hi))");
    // neighbour-list entries address 2^26 particles per set
    if (F->n < 0 || F->n >= (1 << 26)) return bad(msg, "fluid.n must be in [0, 2^26)");
    if (F->n > 0 && !F->pos) return bad(msg, "fluid.pos must not be NULL");
    int64_t nw = W ? W->n : 0;
    if (nw < 0 || nw >= (1 << 26)) return bad(msg, "wall.n must be in [0, 2^26)");
    if (nw > 0 && !W->pos) return bad(msg, "wall.pos must not be NULL");
    for (int64_t i = 0; fluid_host && i < F->n; ++i) {
        if (!finite3(F->pos + 3 * i)) return bad(msg, "non-finite fluid position");
        if (F->vel && !finite3(F->vel + 3 * i)) return bad(msg, "non-finite fluid velocity");
        if (F->rho && !(F->rho[i] > 0 && std::isfinite(F->rho[i]))) return bad(msg, "fluid rho must be > 0");
        if (F->phase && (F->phase[i] < 0 || F->phase[i] >= P->n_phases)) return bad(msg, "fluid phase out of range");
    }
    for (int64_t i = 0; i < nw; ++i)
        if (!finite3(W->pos + 3 * i)) return bad(msg, "non-finite wall position");
    if (P->dim == 2) {
        // one plane: every y equal (pairs then have r_y = 0 exactly)
        const double y0 = F->n > 0 && fluid_host ? F->pos[1] : (nw > 0 ? W->pos[1] : 0.0);
        for (int64_t i = 0; fluid_host && i < F->n; ++i)
            if (F->pos[3 * i + 1] != y0 || (F->vel && F->vel[3 * i + 1] != 0.0))
                return bad(msg, "dim = 2: every particle needs the same y and zero y velocity");
        for (int64_t i = 0; i < nw; ++i)
            if (W->pos[3 * i + 1] != y0) return bad(msg, "dim = 2: every particle needs the same y");
        if (P->g[1] != 0.0) return bad(msg, "dim = 2: g must lie in the x-z plane");
    }
    return SPH_OK;
}

sph_status usable(const sph_ctx* ctx)
{
    if (!ctx || !ctx->sim) return SPH_ERR_ARG;
    if (ctx->sim->dead) return SPH_ERR_STATE;
    return SPH_OK;
}

}  // namespace

extern "C" {

sph_status sph_create(const sph_params* params, const sph_fluid* fluid, const sph_wall* wall,
                      void* cuda_stream, sph_ctx** out)
{
    g_create_error.clear();
    if (!out) {
        g_create_error = "out must not be NULL";
        return SPH_ERR_ARG;
    }
    *out = nullptr;
    sph_status s = validate(params, fluid, wall, &g_create_error);
    if (s != SPH_OK) return s;
    sph_wall empty{0, nullptr};
    cudaStream_t st = (cudaStream_t)cuda_stream;
    sph_ctx* ctx = new (std::nothrow) sph_ctx;
    if (!ctx) return SPH_ERR_OOM;
    ctx->sim = params->precision == SPH_FP64_PLAIN ? sph::make_sim_f64(st) : sph::make_sim_f32(st);
    s = ctx->sim->create(*params, *fluid, wall ? *wall : empty, false);
    if (s != SPH_OK) {
        g_create_error = ctx->sim->err;
        delete ctx->sim;
        delete ctx;
        return s;
    }
    *out = ctx;
    return SPH_OK;
}

sph_status sph_create_device(const sph_params* params, const sph_fluid* fluid, const sph_wall* wall,
                             void* cuda_stream, sph_ctx** out)
{
    g_create_error.clear();
    if (!out) {
        g_create_error = "out must not be NULL";
        return SPH_ERR_ARG;
    }
    *out = nullptr;
    sph_status s = validate(params, fluid, wall, &g_create_error, false);
    if (s != SPH_OK) return s;
    sph_wall empty{0, nullptr};
    cudaStream_t st = (cudaStream_t)cuda_stream;
    sph_ctx* ctx = new (std::nothrow) sph_ctx;
    if (!ctx) return SPH_ERR_OOM;
    ctx->sim = params->precision == SPH_FP64_PLAIN ? sph::make_sim_f64(st) : sph::make_sim_f32(st);
    s = ctx->sim->create(*params, *fluid, wall ? *wall : empty, true);
    if (s != SPH_OK) {
        g_create_error = ctx->sim->err;
        delete ctx->sim;
        delete ctx;
        return s;
    }
    *out = ctx;
    return SPH_OK;
}

sph_status sph_step(sph_ctx* ctx, int32_t nsteps, double dt, double* dt_out)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (nsteps < 0 || !std::isfinite(dt)) {
        ctx->sim->err = "nsteps must be >= 0 and dt finite";
        return SPH_ERR_ARG;
    }
    return ctx->sim->step(nsteps, dt, dt_out);
}

sph_status sph_step_async(sph_ctx* ctx, int32_t nsteps, double dt)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (nsteps < 0 || !std::isfinite(dt)) {
        ctx->sim->err = "nsteps must be >= 0 and dt finite";
        return SPH_ERR_ARG;
    }
    return ctx->sim->step_async(nsteps, dt);
}

sph_status sph_sync(sph_ctx* ctx, double* dt_out)
{
    sph_status s = usable(ctx);
    return s != SPH_OK ? s : ctx->sim->sync(dt_out);
}

sph_status sph_reinit_density(sph_ctx* ctx)
{
    sph_status s = usable(ctx);
    return s != SPH_OK ? s : ctx->sim->reinit();
}

sph_status sph_get_state(sph_ctx* ctx, const sph_state_out* out, int32_t where)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (!out || (where != SPH_HOST && where != SPH_DEVICE)) {
        ctx->sim->err = "out must not be NULL; where must be SPH_HOST or SPH_DEVICE";
        return SPH_ERR_ARG;
    }
    return ctx->sim->get_state(*out, where);
}

sph_status sph_grid_info(const sph_ctx* ctx, int32_t dims[3], int64_t* n_cells, double* cell_size)
{
    if (!ctx || !ctx->sim) return SPH_ERR_ARG;
    ctx->sim->grid(dims, n_cells, cell_size);
    return SPH_OK;
}

sph_status sph_get_cells(sph_ctx* ctx, uint32_t* key_fluid, int32_t* order_fluid, int32_t* start_fluid,
                         uint32_t* key_wall, int32_t* order_wall, int32_t* start_wall)
{
    sph_status s = usable(ctx);
    return s != SPH_OK ? s : ctx->sim->get_cells(key_fluid, order_fluid, start_fluid, key_wall, order_wall,
                                                 start_wall);
}

sph_status sph_get_neighbors(sph_ctx* ctx, int64_t* fluid_offsets, int32_t* fluid_ids, int64_t fluid_cap,
                             int64_t* wall_offsets, int32_t* wall_ids, int64_t wall_cap, int64_t overflow[2])
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (fluid_cap < 0 || wall_cap < 0) {
        ctx->sim->err = "capacities must be >= 0";
        return SPH_ERR_ARG;
    }
    return ctx->sim->get_neighbors(fluid_offsets, fluid_ids, fluid_cap, wall_offsets, wall_ids, wall_cap,
                                   overflow);
}

sph_status sph_diagnostics(sph_ctx* ctx, double out[8])
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (!out) return SPH_ERR_ARG;
    return ctx->sim->diagnostics(out);
}

sph_status sph_diagnostics_async(sph_ctx* ctx, double* out, int32_t where)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (!out || (where != SPH_HOST && where != SPH_DEVICE)) {
        ctx->sim->err = "out must not be NULL; where must be SPH_HOST or SPH_DEVICE";
        return SPH_ERR_ARG;
    }
    if (where == SPH_HOST) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, out) != cudaSuccess || a.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            ctx->sim->err = "out must be page-locked host memory (cudaHostAlloc / pinned)";
            return SPH_ERR_ARG;
        }
    }
    return ctx->sim->diagnostics_async(out, where);
}

sph_status sph_set_excitation(sph_ctx* ctx, const double amp[3], double freq)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (!amp || !finite3(amp) || !(freq >= 0.0) || !std::isfinite(freq)) {
        ctx->sim->err = "amp must be finite and freq finite and >= 0";
        return SPH_ERR_ARG;
    }
    return ctx->sim->set_excitation(amp, freq);
}

sph_status sph_time(sph_ctx* ctx, double* t)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (!t) return SPH_ERR_ARG;
    return ctx->sim->time(t);
}

sph_status sph_tape_budget(sph_ctx* ctx, int64_t bytes)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (bytes < -1) {
        ctx->sim->err = "bytes must be -1 (half the free memory), 0 (keep none) or a positive budget";
        return SPH_ERR_ARG;
    }
    return ctx->sim->tape_budget(bytes);
}

sph_status sph_probe_pressure(sph_ctx* ctx, const double* pts, int32_t n, double* p, double* w, int32_t where)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (n < 0 || (n > 0 && !pts) || (where != SPH_HOST && where != SPH_DEVICE)) {
        ctx->sim->err = "n must be >= 0, pts non-NULL when n > 0; where must be SPH_HOST or SPH_DEVICE";
        return SPH_ERR_ARG;
    }
    if (where == SPH_HOST)
        for (int32_t k = 0; k < n; ++k)
            if (!finite3(pts + 3 * (size_t)k)) {
                ctx->sim->err = "non-finite sensor position";
                return SPH_ERR_ARG;
            }
    return ctx->sim->probe_pressure(pts, n, p, w, where);
}

sph_status sph_gauge_height(sph_ctx* ctx, const double* gauges, int32_t n, double dz, double* H, int32_t where)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (n < 0 || n > SPH_GAUGE_MAX_LINES || (n > 0 && (!gauges || !H)) || !(dz > 0.0) || !std::isfinite(dz) ||
        (where != SPH_HOST && where != SPH_DEVICE)) {
        ctx->sim->err = "n must be in [0, SPH_GAUGE_MAX_LINES], gauges and H non-NULL when n > 0, dz finite and "
                        "> 0; where must be SPH_HOST or SPH_DEVICE";
        return SPH_ERR_ARG;
    }
    if (where == SPH_HOST)
        for (int32_t k = 0; k < n; ++k) {
            const double* g = gauges + 4 * (size_t)k;
            const bool fin = std::isfinite(g[0]) && std::isfinite(g[1]) && std::isfinite(g[2]) && std::isfinite(g[3]);
            if (!fin || !(g[3] >= g[2]) || !(std::floor((g[3] - g[2]) / dz) < (double)SPH_GAUGE_MAX_SAMPLES)) {
                ctx->sim->err = "gauge lines must be finite with z_lo <= z_hi and fewer than "
                                "SPH_GAUGE_MAX_SAMPLES samples";
                return SPH_ERR_ARG;
            }
        }
    return ctx->sim->gauge_height(gauges, n, dz, H, where);
}

sph_status sph_counters(sph_ctx* ctx, int64_t* steps, int64_t* active_wall_steps)
{
    sph_status s = usable(ctx);
    return s != SPH_OK ? s : ctx->sim->counters(steps, active_wall_steps);
}

sph_status sph_profile(sph_ctx* ctx, uint32_t kind_mask)
{
    sph_status s = usable(ctx);
    return s != SPH_OK ? s : ctx->sim->profile(kind_mask);
}

sph_status sph_profile_read(sph_ctx* ctx, double* ms, int64_t* timed, int64_t* launches)
{
    sph_status s = usable(ctx);
    return s != SPH_OK ? s : ctx->sim->profile_read(ms, timed, launches);
}

sph_status sph_tape(sph_ctx* ctx, int32_t nsteps, double dt, double* dt_out)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (nsteps < 0 || !std::isfinite(dt)) {
        ctx->sim->err = "nsteps must be >= 0 and dt finite";
        return SPH_ERR_ARG;
    }
    return ctx->sim->tape(nsteps, dt, dt_out);
}

sph_status sph_backward(sph_ctx* ctx, const sph_adjoint_seed* seed, sph_adjoint_grad* grad, int32_t where)
{
    sph_status s = usable(ctx);
    if (s != SPH_OK) return s;
    if (!seed || !grad || (where != SPH_HOST && where != SPH_DEVICE)) {
        ctx->sim->err = "seed and grad must not be NULL; where must be SPH_HOST or SPH_DEVICE";
        return SPH_ERR_ARG;
    }
    return ctx->sim->backward(*seed, *grad, where);
}

const char* sph_last_error(const sph_ctx* ctx)
{
    if (!ctx || !ctx->sim) return g_create_error.c_str();
    return ctx->sim->err.c_str();
}

void sph_destroy(sph_ctx* ctx)
{
    if (!ctx) return;
    delete ctx->sim;
    delete ctx;
}

sph_status sph_bin_sort(const double* pos, int64_t n, const double lo[3], double h, const int32_t dims[3],
                        uint32_t* key, int32_t* order, int32_t* start, void* cuda_stream)
{
    if (n < 0 || n > 2000000000 || !lo || !dims || !(h > 0) || !start || (n > 0 && (!pos || !key || !order)))
        return SPH_ERR_ARG;
    const int64_t n_cells = sph::grid_cell_count(dims);
    if (n_cells < 0) return SPH_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    sph::BinSortScratch L = sph::bin_sort_scratch_layout(n, n_cells);
    char* scratch = nullptr;
    if (cudaMallocAsync((void**)&scratch, L.bytes, st) != cudaSuccess) return SPH_ERR_OOM;
    cudaError_t e = sph::bin_sort_run(pos, (int32_t)n, lo, 2.0 * h, dims, key, order, start, scratch, st);
    cudaError_t f = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess || f != cudaSuccess) return SPH_ERR_CUDA;
    return SPH_OK;
}

}  // extern "C"
