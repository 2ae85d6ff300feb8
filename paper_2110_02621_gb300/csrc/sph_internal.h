// Internal interface between the C ABI (sph_api.cu) and the two compiled
// forms of the simulation (FP32 in sim_f32.cu, plain FP64 in sim_f64.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "sph.h"

namespace sph {

int32_t scan_blocks(int64_t n);
int64_t scan_max_len();
// Cell count of a dims[0] x dims[1] x dims[2] grid, or -1 when an extent is
// below 1 or the grid holds more cells than the scan takes (scan_max_len() - 2).
// Each extent is checked before it is multiplied in, so no product overflows.
int64_t grid_cell_count(const int32_t dims[3]);
// out[0..n] = exclusive prefix sums of in[0..n-1] (out[n] = total);
// sums needs scan_blocks(n) entries; clear (NULL or in) is zeroed behind the
// scan.  Returns the number of kernels launched.
int scan_exclusive(const int32_t* in, int32_t n, int32_t* out, int32_t* sums, cudaStream_t st,
                   int32_t* clear);

struct BinSortScratch {
    size_t cell, id, rank, tmp_src, tmp_id, counts, start, sums, bytes;
};
BinSortScratch bin_sort_scratch_layout(int64_t n, int64_t n_cells);
cudaError_t bin_sort_run(const double* pos, int32_t n, const double lo[3], double cs,
                         const int32_t dims[3], uint32_t* key, int32_t* order, int32_t* start,
                         char* scratch, cudaStream_t st);

struct SimBase {
    virtual ~SimBase() {}
    // fluid_dev: F's arrays are device memory (checked by a kernel), else host
    virtual sph_status create(const sph_params& P, const sph_fluid& F, const sph_wall& W, bool fluid_dev) = 0;
    virtual sph_status step(int32_t nsteps, double dt, double* dt_out) = 0;
    virtual sph_status step_async(int32_t nsteps, double dt) = 0;
    virtual sph_status sync(double* dt_out) = 0;
    virtual sph_status reinit() = 0;
    virtual sph_status get_state(const sph_state_out& o, int32_t where) = 0;
    virtual sph_status get_cells(uint32_t* kf, int32_t* of, int32_t* sf, uint32_t* kw, int32_t* ow,
                                 int32_t* sw) = 0;
    virtual sph_status get_neighbors(int64_t* f_off, int32_t* f_ids, int64_t f_cap, int64_t* w_off,
                                     int32_t* w_ids, int64_t w_cap, int64_t overflow[2]) = 0;
    virtual sph_status diagnostics(double out[8]) = 0;
    virtual sph_status diagnostics_async(double* out, int32_t where) = 0;
    virtual sph_status counters(int64_t* steps, int64_t* active) = 0;
    virtual void grid(int32_t dims[3], int64_t* n_cells, double* cs) const = 0;
    virtual sph_status profile(uint32_t mask) = 0;
    virtual sph_status profile_read(double* ms, int64_t* timed, int64_t* launches) = 0;
    virtual sph_status tape(int32_t nsteps, double dt, double* dt_out) = 0;
    virtual sph_status tape_budget(int64_t bytes) = 0;
    virtual sph_status set_excitation(const double amp[3], double freq) = 0;
    virtual sph_status time(double* t) = 0;
    virtual sph_status probe_pressure(const double* pts, int32_t n, double* p, double* w, int32_t where) = 0;
    virtual sph_status gauge_height(const double* g, int32_t n, double dz, double* H, int32_t where) = 0;
    virtual sph_status backward(const sph_adjoint_seed& seed, sph_adjoint_grad& grad, int32_t where) = 0;

    std::string err;
    cudaStream_t stream = nullptr;
    bool dead = false;  // a sticky error happened
};

SimBase* make_sim_f32(cudaStream_t st);
SimBase* make_sim_f64(cudaStream_t st);

}  // namespace sph
