// Host-side orchestration of one simulation context: device buffers, the
// create sequence and the kernel sequence of one step (Sec. 2.6, Sec. 3).
// Included once per precision (sim_f32.cu, sim_f64.cu).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <utility>
#include <vector>

#include "sph_internal.h"
#include "sph_adjoint.cuh"
#include "sph_probes.cuh"
#include "sph_setup.cuh"

namespace sph {

#define SPH_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return fail_cuda(e_, #call, __LINE__);                      \
    } while (0)
#define SPH_LAUNCH()                                                                       \
    do {                                                                                   \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess) return fail_cuda(e_, "kernel launch", __LINE__);            \
    } while (0)

// Launch one kernel (or a fixed group of nlaunch kernels) of a kind: counts
// the launches and, when that kind is being profiled, brackets it with CUDA
// events on the context's stream.
#define SPH_KERNEL(kind, nlaunch, ...)                                                     \
    do {                                                                                   \
        sph_status ks_ = prof_begin(kind);                                                 \
        if (ks_ != SPH_OK) return ks_;                                                     \
        __VA_ARGS__;                                                                       \
        SPH_LAUNCH();                                                                      \
        launches_[kind] += (nlaunch);                                                      \
        ks_ = prof_end(kind);                                                              \
        if (ks_ != SPH_OK) return ks_;                                                     \
    } while (0)

inline int grid_for(int64_t n) { return (int)((n + BLOCK - 1) / BLOCK); }


// Wendland C2 normalisation: 21/(16 pi h^3) in 3-D, 7/(4 pi h^2) in 2-D
inline double wendland_alpha(double h, int dim)
{
    const double pi = 3.14159265358979323846;
    return dim == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
}

// number density of a full lattice of spacing dp (cubic, or square in the
// x-z plane in 2-D), self included
inline double lattice_sigma0(double dp, double h, int dim)
{
    int K = (int)std::ceil(2.0 * h / dp) + 1;
    const int KY = dim == 2 ? 0 : K;
    double alpha = wendland_alpha(h, dim), s = 0.0;
    for (int i = -K; i <= K; ++i)
        for (int j = -KY; j <= KY; ++j)
            for (int k = -K; k <= K; ++k) {
                double q = dp * std::sqrt((double)(i * i + j * j + k * k)) / h;
                if (q < 2.0) {
                    double t = 1.0 - 0.5 * q;
                    s += alpha * t * t * t * t * (2.0 * q + 1.0);
                }
            }
    return s;
}

// body-force limit of the time step (Sec. 2.6), with the largest body force
// of the tank motion, |g| + |amp| w^2
template <class T>
void set_body_dt(Cfg<T>& C, double cfl, double h)
{
    double gn = std::sqrt(C.g64[0] * C.g64[0] + C.g64[1] * C.g64[1] + C.g64[2] * C.g64[2]);
    gn += std::sqrt(C.ex_amp[0] * C.ex_amp[0] + C.ex_amp[1] * C.ex_amp[1] + C.ex_amp[2] * C.ex_amp[2]) * C.ex_w *
          C.ex_w;
    C.body_dt = gn > 0.0 ? (T)(cfl * std::sqrt(h / gn)) : T(0);
}

template <class T>
Cfg<T> make_cfg(const sph_params& P, const int32_t dims[3])
{
    Cfg<T> C;
    double h = P.h, cs = 2.0 * h;
    const int dim = P.dim == 2 ? 2 : 3;
    const double vol = dim == 2 ? P.dp * P.dp : P.dp * P.dp * P.dp;  // particle volume dx^dim
    double alpha = wendland_alpha(h, dim);
    C.h = (T)h;
    C.rc2 = (T)(cs * cs);
    C.nf = C.nw = 0;
    C.cs = (T)cs;
    C.alpha = (T)alpha;
    C.fcoef = (T)(-5.0 * alpha / (h * h));
    C.W0 = (T)alpha;
    C.inv_h = (T)(1.0 / h);
    C.c0 = (T)P.c0;
    C.inv_c0 = (T)(1.0 / P.c0);
    C.gamma = (T)P.gamma_tait;
    C.inv_gamma = (T)(1.0 / P.gamma_tait);
    C.gamma_p = (T)P.gamma_p;
    C.dp = (T)P.dp;
    C.dp3 = (T)(P.dp * P.dp * P.dp);  // the penalty's dx^3 (in 2-D as well)
    C.vol = (T)vol;
    C.inv_dp = (T)(1.0 / P.dp);
    C.eta2 = (T)(0.01 * h * h);
    C.pen_rmin = (T)(1e-6 * P.dp);
    C.gx = (T)P.g[0];
    C.gy = (T)P.g[1];
    C.gz = (T)P.g[2];
    const double sigma0 = lattice_sigma0(P.dp, h, dim), inv_vol = 1.0 / vol;
    C.inv_sigma0 = (T)(1.0 / sigma0);
    C.sigma0_hi = (T)sigma0;
    C.sigma0_lo = (T)(sigma0 - (double)C.sigma0_hi);
    C.inv_vol_hi = (T)inv_vol;
    C.inv_vol_lo = (T)(inv_vol - (double)C.inv_vol_hi);
    C.cfl = (T)P.cfl;
    for (int d = 0; d < 3; ++d) {
        C.g64[d] = P.g[d];
        C.ex_amp[d] = 0.0;
    }
    C.ex_w = 0.0;
    set_body_dt(C, P.cfl, h);
    C.nx = dims[0];
    C.ny = dims[1];
    C.nz = dims[2];
    C.n_cells = dims[0] * dims[1] * dims[2];
    C.periodic = P.periodic;
    C.n_phases = P.n_phases;
    for (int k = 0; k < 2; ++k) {
        const sph_phase& ph = P.phase[k < P.n_phases ? k : 0];
        PhaseK<T>& q = C.ph[k];
        q.rho0 = (T)ph.rho0;
        q.inv_rho0 = (T)(1.0 / ph.rho0);
        q.mu = (T)ph.mu;
        q.m = (T)(ph.rho0 * vol);
        q.eos_k = ph.eos == SPH_EOS_TAIT ? (T)(ph.rho0 * P.c0 * P.c0 / P.gamma_tait) : (T)(P.c0 * P.c0);
        q.p_half = ph.eos == SPH_EOS_TAIT
                       ? (T)(ph.rho0 * P.c0 * P.c0 / P.gamma_tait * (std::pow(0.5, P.gamma_tait) - 1.0))
                       : (T)(-0.5 * ph.rho0 * P.c0 * P.c0);
        q.eos = ph.eos;
        q.density = ph.density;
        q.reinit = ph.reinit;
        q.penalty = ph.penalty;
    }
    return C;
}

template <class T>
class Sim final : public SimBase {
    static constexpr bool KAHAN = std::is_same<T, float>::value;

  public:
    explicit Sim(cudaStream_t st) { stream = st; }
    ~Sim() override
    {
        for (cudaGraphExec_t& g : gexec_)
            if (g) cudaGraphExecDestroy(g);
        if (cap_stream_) cudaStreamDestroy(cap_stream_);
        if (adj_side_) cudaStreamDestroy(adj_side_);
        for (cudaEvent_t& e : adj_ev_)
            if (e) cudaEventDestroy(e);
        for (void* p : allocs_) cudaFree(p);
        for (EvPair& e : ev_) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
        if (host_status_) cudaFreeHost(host_status_);
    }

    sph_status create(const sph_params& P, const sph_fluid& F, const sph_wall& Wl, bool fluid_dev) override
    {
        P_ = P;
        cs_ = 2.0 * P.h;
        n_cells_ = 1;
        for (int d = 0; d < 3; ++d) {
            const double u = (P.hi[d] - P.lo[d]) / cs_;
            // a periodic axis is a whole number of cells (checked by the ABI)
            dims_[d] = (P.periodic >> d) & 1 ? (int32_t)std::floor(u + 0.5) : (int32_t)std::ceil(u);
            if (dims_[d] < 1) dims_[d] = 1;
            n_cells_ *= dims_[d];
        }
        C_ = make_cfg<T>(P, dims_);
        D_ = make_cfg<double>(P, dims_);
        C_.nf = D_.nf = (int32_t)F.n;
        C_.nw = D_.nw = (int32_t)Wl.n;
        for (int d = 0; d < 3; ++d) I_.lo[d] = P.lo[d];
        I_.cs = cs_;
        I_.gz = P.g[2];
        I_.c0 = P.c0;
        I_.gamma = P.gamma_tait;
        I_.n_phases = P.n_phases;
        I_.has_rho = F.rho != nullptr;
        I_.sigma0 = lattice_sigma0(P.dp, P.h, P.dim == 2 ? 2 : 3);
        for (int k = 0; k < 2; ++k) {
            const sph_phase& ph = P.phase[k < P.n_phases ? k : 0];
            I_.rho0[k] = ph.rho0;
            I_.z_top[k] = ph.z_top;
            I_.eos[k] = ph.eos;
        }
        nf_ = (int32_t)F.n;
        nw_ = (int32_t)Wl.n;
        sph_status s = allocate();
        if (s != SPH_OK) return s;
        SPH_CUDA(cudaMallocHost(&host_status_, sizeof(HostStatus)));

        // ---- walls: bin, sort once, normals (Eq. normalVectors)
        double* xw_in = nullptr;
        double* xw_sorted = nullptr;
        if (nw_ > 0) {
            SPH_CUDA(cudaMallocAsync(&xw_in, sizeof(double) * 3 * (size_t)nw_, stream));
            SPH_CUDA(cudaMallocAsync(&xw_sorted, sizeof(double) * 3 * (size_t)nw_, stream));
            SPH_CUDA(cudaMemcpyAsync(xw_in, Wl.pos, sizeof(double) * 3 * (size_t)nw_,
                                     cudaMemcpyHostToDevice, stream));
        }
        SPH_CUDA(cudaMemsetAsync(counts_, 0, sizeof(int32_t) * (size_t)(n_cells_ + 1), stream));
        if (nw_ > 0) {
            k_init_wall<T><<<grid_for(nw_), BLOCK, 0, stream>>>(C_, I_, nw_, xw_in, wpos_tmp_, wcell_tmp_,
                                                                wid_tmp_, rank_, counts_);
            SPH_LAUNCH();
        }
        scan_exclusive(counts_, n_cells_ + 1, wstart_, sums_, stream, counts_);
        SPH_LAUNCH();
        if (nw_ > 0) {
            k_scatter<<<grid_for(nw_), BLOCK, 0, stream>>>(nw_, n_cells_, wcell_tmp_, rank_, wstart_,
                                                           wid_tmp_, tmp_src_, tmp_id_, nullptr);
            k_gather_wall<T><<<grid_for(nw_), BLOCK, 0, stream>>>(nw_, n_cells_, wstart_, tmp_src_, tmp_id_,
                                                                  wpos_tmp_, wcell_tmp_, xw_in, wpos_, wcell_,
                                                                  wid_, xw_sorted);
            k_wall_normals<T><<<grid_for(nw_), BLOCK, 0, stream>>>(D_, nw_, wstart_, wcell_, xw_sorted, wnrm_);
            SPH_LAUNCH();
            if (P_.periodic)
                k_wall_rows<true, T><<<grid_for(n_cells_), BLOCK, 0, stream>>>(C_, n_cells_, wstart_, wrows_);
            else
                k_wall_rows<false, T><<<grid_for(n_cells_), BLOCK, 0, stream>>>(C_, n_cells_, wstart_, wrows_);
            SPH_LAUNCH();
            SPH_CUDA(cudaFreeAsync(xw_in, stream));
            SPH_CUDA(cudaFreeAsync(xw_sorted, stream));
        } else {
            SPH_CUDA(cudaMemsetAsync(wrows_, 0, sizeof(uint16_t) * (size_t)n_cells_, stream));
        }

        // ---- fluid: upload, initial density, first sort
        double *x_in = nullptr, *v_in = nullptr, *r_in = nullptr;
        int32_t* ph_in = nullptr;
        if (nf_ > 0) {
            // device inputs are copied too: the caller keeps its arrays
            const cudaMemcpyKind kind = fluid_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            size_t b3 = sizeof(double) * 3 * (size_t)nf_;
            SPH_CUDA(cudaMallocAsync(&x_in, b3, stream));
            SPH_CUDA(cudaMemcpyAsync(x_in, F.pos, b3, kind, stream));
            if (F.vel) {
                SPH_CUDA(cudaMallocAsync(&v_in, b3, stream));
                SPH_CUDA(cudaMemcpyAsync(v_in, F.vel, b3, kind, stream));
            }
            if (F.rho) {
                SPH_CUDA(cudaMallocAsync(&r_in, sizeof(double) * (size_t)nf_, stream));
                SPH_CUDA(cudaMemcpyAsync(r_in, F.rho, sizeof(double) * (size_t)nf_, kind, stream));
            }
            if (F.phase) {
                SPH_CUDA(cudaMallocAsync(&ph_in, sizeof(int32_t) * (size_t)nf_, stream));
                SPH_CUDA(cudaMemcpyAsync(ph_in, F.phase, sizeof(int32_t) * (size_t)nf_, kind, stream));
            }
            if (fluid_dev) {
                // the host checks of sph_create, on the device, before any use
                SPH_CUDA(cudaMemsetAsync(d_flags_, 0, sizeof(int32_t), stream));
                k_check_fluid<<<grid_for(nf_), BLOCK, 0, stream>>>(
                    nf_, x_in, v_in, r_in, ph_in, P.n_phases, P.dim == 2 ? 1 : 0, nw_ > 0 ? Wl.pos[1] : 0.0,
                    nw_ > 0 ? 0 : 1, d_flags_);
                SPH_LAUNCH();
                SPH_CUDA(cudaMemcpyAsync(&host_status_->flags, d_flags_, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                         stream));
                SPH_CUDA(cudaStreamSynchronize(stream));
                if (host_status_->flags) {
                    for (void* p : {(void*)x_in, (void*)v_in, (void*)r_in, (void*)ph_in})
                        if (p) SPH_CUDA(cudaFreeAsync(p, stream));
                    SPH_CUDA(cudaStreamSynchronize(stream));
                    err = P.dim == 2 ? "fluid inputs: non-finite position or velocity, rho <= 0, phase out of range, "
                                       "or (2-D) a y or y velocity that differs"
                                     : "fluid inputs: non-finite position or velocity, rho <= 0 or phase out of range";
                    return SPH_ERR_ARG;
                }
            }
        }
        SPH_CUDA(cudaMemsetAsync(counts_, 0, sizeof(int32_t) * (size_t)(n_cells_ + 1), stream));
        SPH_CUDA(cudaMemsetAsync(d_dt_, 0, sizeof(T), stream));
        SPH_CUDA(cudaMemsetAsync(d_dt_fixed_, 0, sizeof(T), stream));
        SPH_CUDA(cudaMemsetAsync(d_vmax_, 0, sizeof(unsigned long long), stream));
        {
            // t = 0, body force g
            const V4<T> g0{C_.gx, C_.gy, C_.gz, T(0)};
            const double t0 = 0.0;
            SPH_CUDA(cudaMemcpyAsync(d_geff_, &g0, sizeof g0, cudaMemcpyHostToDevice, stream));
            SPH_CUDA(cudaMemcpyAsync(d_time_, &t0, sizeof t0, cudaMemcpyHostToDevice, stream));
            SPH_CUDA(cudaStreamSynchronize(stream));
        }
        SPH_CUDA(cudaMemsetAsync(d_flags_, 0, sizeof(int32_t), stream));
        SPH_CUDA(cudaMemsetAsync(d_active_, 0, sizeof(unsigned long long), stream));
        SPH_CUDA(cudaMemsetAsync(d_tag_, 0, sizeof(int32_t), stream));
        SPH_CUDA(cudaMemsetAsync(wtag_, 0xff, sizeof(int32_t) * (size_t)(nw_ > 0 ? nw_ : 1), stream));
        SPH_CUDA(cudaMemsetAsync(wfront_, 0, sizeof(int32_t) * (size_t)(nw_ > 0 ? nw_ : 1), stream));
        par_ = 0;
        if (nf_ > 0) {
            k_init_fluid<T><<<grid_for(nf_), BLOCK, 0, stream>>>(
                C_, I_, nf_, x_in, v_in, r_in, ph_in, pos_[0], vel_[0], drho_[0], acc_, comp_[0], newcell_,
                id_[0], phase_[0], rank_, counts_);
            SPH_LAUNCH();
        }
        scan_exclusive(counts_, n_cells_ + 1, fstart_, sums_, stream, counts_);
        SPH_LAUNCH();
        if (nf_ > 0) {
            k_scatter<<<grid_for(nf_), BLOCK, 0, stream>>>(nf_, n_cells_, newcell_, rank_, fstart_, id_[0],
                                                           tmp_src_, tmp_id_, nullptr);
            // dt = 0 and no reinitialisation: a pure permutation into (key, id) order
            k_gather<T, KAHAN><<<grid_for(nf_), BLOCK, 0, stream>>>(
                C_, nf_, fstart_, tmp_src_, tmp_id_, newcell_, d_dt_, 0, pos_[0], vel_[0], drho_[0], acc_,
                comp_[0], sigma_, newcell_, phase_[0], pos_[1], vel_[1], drho_[1], comp_[1], cell_[1], id_[1],
                phase_[1]);
            SPH_LAUNCH();
            for (void* p : {(void*)x_in, (void*)v_in, (void*)r_in, (void*)ph_in})
                if (p) SPH_CUDA(cudaFreeAsync(p, stream));
        }
        // the sorted state is in the [1] buffers; make it current
        std::swap(pos_[0], pos_[1]);
        std::swap(drho_[0], drho_[1]);
        par_ = 1;

        // ---- wall pressure of the initial state, then a^0, sigma^0, U_max
        s = neighbors(pos_[0], cell_[1]);
        if (s != SPH_OK) return s;
        s = wall_pressure(vel_[1]);
        if (s != SPH_OK) return s;
        s = momentum(vel_[1], vel_[0], cell_[1], phase_[1]);  // dt = 0: writes v + 0*a
        if (s != SPH_OK) return s;
        std::swap(vel_[0], vel_[1]);

        SPH_CUDA(cudaMemcpyAsync(&host_status_->n_in, fstart_ + n_cells_, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaMemcpyAsync(&host_status_->w_in, wstart_ + n_cells_, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaStreamSynchronize(stream));
        if (sph_status sc = index_check(); sc != SPH_OK) return sc;
        if (host_status_->n_in != nf_ || host_status_->w_in != nw_) {
            char buf[160];
            snprintf(buf, sizeof buf, "%d fluid and %d wall particles lie outside the grid [lo, hi)",
                     nf_ - host_status_->n_in, nw_ - host_status_->w_in);
            err = buf;
            return SPH_ERR_DOMAIN;
        }
        return SPH_OK;
    }

    sph_status step(int32_t nsteps, double dt, double* dt_out) override
    {
        sph_status s = enqueue_steps(nsteps, dt);
        if (s != SPH_OK) return s;
        return finish_steps(dt_out);
    }

    sph_status step_async(int32_t nsteps, double dt) override { return enqueue_steps(nsteps, dt); }

    sph_status sync(double* dt_out) override { return finish_steps(dt_out); }

    // The fixed dt reaches the device through a pinned word.  A copy from it
    // may still be pending after an asynchronous call, so a new value first
    // waits for the stream; an unchanged value is not copied again.
    sph_status set_dt_fixed(double dt)
    {
        const T want = (T)(dt > 0.0 ? dt : 0.0);
        if (dt_valid_ && want == host_status_->dt_fixed) return SPH_OK;
        SPH_CUDA(cudaStreamSynchronize(stream));
        host_status_->dt_fixed = want;
        SPH_CUDA(cudaMemcpyAsync(d_dt_fixed_, &host_status_->dt_fixed, sizeof(T), cudaMemcpyHostToDevice,
                                 stream));
        dt_valid_ = true;
        return SPH_OK;
    }

    sph_status enqueue_steps(int32_t nsteps, double dt)
    {
        sph_status s0 = set_dt_fixed(dt);
        if (s0 != SPH_OK) return s0;
        for (int32_t k = 0; k < nsteps; ++k) {
            bool reinit = P_.reinit_every > 0 && (steps_ % P_.reinit_every) == 0;
            const bool sig = sigma_next();
            // the kernel sequence of a step as one CUDA graph launch, unless
            // kernels are being timed one by one
            sph_status s = prof_mask_ ? one_step(reinit, true, sig) : graph_step(reinit, true, sig);
            if (s != SPH_OK) return s;
            ++steps_;
        }
        return SPH_OK;
    }

    // Whether the step about to run must leave sigma(r^{n+1}) for the next
    // one: only when that step reinitialises (the other readers, the state
    // export and sph_reinit_density, call ensure_sigma).
    bool sigma_next() const
    {
        return P_.reinit_every > 0 && ((steps_ + 1) % P_.reinit_every) == 0;
    }

    // sigma - sigma^0 at the current positions, when the last momentum sweep
    // left it out (k_sigma: the same bits the sweep would have written).
    sph_status ensure_sigma()
    {
        if (sigma_valid_ || nf_ == 0) return SPH_OK;
        if (!lists_current_) {
            sph_status s = neighbors(pos_[0], cell_[par_]);
            if (s != SPH_OK) return s;
        }
        auto launch = [&](auto kernel) {
            kernel<<<grid_for((int64_t)nf_ * LP), BLOCK, 0, stream>>>(C_, nf_, fstart_, wstart_, nbf_, nbw_, ncnt_,
                                                                      pos_[0], cell_[par_], phase_[par_], wpos_,
                                                                      sigma_);
        };
        SPH_KERNEL(SPH_K_OTHER, 1, P_.periodic ? launch(k_sigma<T, true>) : launch(k_sigma<T, false>));
        sigma_valid_ = true;
        return SPH_OK;
    }

    // The check word of the index-checking build (-DSPH_CHECK): a set bit
    // names the kind of index found out of range since the last call.
    sph_status index_check()
    {
#ifdef SPH_CHECK
        unsigned w = 0;
        const unsigned zero = 0;
        SPH_CUDA(cudaMemcpyFromSymbolAsync(&w, g_sph_check, sizeof w, 0, cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaMemcpyToSymbolAsync(g_sph_check, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, stream));
        SPH_CUDA(cudaStreamSynchronize(stream));
        if (w) {
            char buf[160];
            snprintf(buf, sizeof buf,
                     "index check: out of range (bits 0x%x: 1 fluid list, 2 wall list, 4 cell, 8 range, 16 slot)", w);
            err = buf;
            dead = true;
            return SPH_ERR_CUDA;
        }
#endif
        return SPH_OK;
    }

    // read the error word, the in-grid count and the last dt after a run of
    // steps (one synchronisation)
    sph_status finish_steps(double* dt_out)
    {
        SPH_CUDA(cudaMemcpyAsync(&host_status_->flags, d_flags_, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 stream));
        SPH_CUDA(cudaMemcpyAsync(&host_status_->n_in, fstart_ + n_cells_, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaMemcpyAsync(&host_status_->dt, d_dt_, sizeof(T), cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaStreamSynchronize(stream));
        if (dt_out) *dt_out = (double)host_status_->dt;
        if (sph_status sc = index_check(); sc != SPH_OK) return sc;
        if (host_status_->flags & 1) {
            err = "non-finite acceleration";
            dead = true;
            return SPH_ERR_NONFINITE;
        }
        if (host_status_->n_in != nf_) {
            char buf[96];
            snprintf(buf, sizeof buf, "%d fluid particles outside the grid", nf_ - host_status_->n_in);
            err = buf;
            return SPH_ERR_DOMAIN;
        }
        return SPH_OK;
    }

    sph_status reinit() override
    {
        if (sph_status s = ensure_sigma(); s != SPH_OK) return s;
        if (nf_ > 0)
            SPH_KERNEL(SPH_K_OTHER, 1,
                       k_reinit<T><<<grid_for(nf_), BLOCK, 0, stream>>>(C_, nf_, sigma_, cell_[par_], phase_[par_],
                                                                        pos_[0], vel_[par_], drho_[0]));
        SPH_CUDA(cudaStreamSynchronize(stream));
        return SPH_OK;
    }

    // Rigid sinusoidal tank motion from now on (Sec. 4.2 excitation): the
    // body force of later steps follows amp w^2 sin(w t); the captured step
    // graphs hold the old constants and are dropped.
    sph_status set_excitation(const double amp[3], double freq) override
    {
        if (P_.dim == 2 && amp[1] != 0.0) {
            err = "dim = 2: the motion must lie in the x-z plane";
            return SPH_ERR_ARG;
        }
        for (int d = 0; d < 3; ++d) C_.ex_amp[d] = D_.ex_amp[d] = amp[d];
        C_.ex_w = D_.ex_w = 2.0 * 3.14159265358979323846 * freq;
        set_body_dt(C_, P_.cfl, P_.h);
        set_body_dt(D_, P_.cfl, P_.h);
        SPH_CUDA(cudaStreamSynchronize(stream));
        for (cudaGraphExec_t& g : gexec_)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
        return SPH_OK;
    }

    sph_status time(double* t) override
    {
        SPH_CUDA(cudaMemcpyAsync(&host_status_->time, d_time_, sizeof(double), cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaStreamSynchronize(stream));
        *t = host_status_->time;
        return SPH_OK;
    }

    // ------------------------------------------------------------ adjoint
    sph_status tape(int32_t nsteps, double dt, double* dt_out) override
    {
        if (P_.n_phases != 1 || P_.phase[0].density != SPH_DENSITY_CONTINUITY) {
            err = "the adjoint covers one phase with continuity density";
            return SPH_ERR_UNSUPPORTED;
        }
        if (ck_.empty()) {
            if (steps_ != 0) {
                err = "taping must start right after sph_create";
                return SPH_ERR_STATE;
            }
            ck_.emplace_back();
            sph_status s = save(ck_.back());
            if (s != SPH_OK) return s;
            tape_end_ = 0;
        } else if (steps_ != tape_end_) {
            err = "untaped steps were taken since the last sph_tape";
            return SPH_ERR_STATE;
        }
        sph_status s0 = set_dt_fixed(dt);
        if (s0 != SPH_OK) return s0;
        const int64_t first = ntaped_;
        for (int32_t k = 0; k < nsteps; ++k) {
            // ck_[k] is the state before taped step k (copies ordered on the stream)
            if ((size_t)ntaped_ == ck_.size()) {
                ck_.emplace_back();
                sph_status s = save(ck_.back());
                if (s != SPH_OK) return s;
            }
            Ckpt& c = ck_[(size_t)ntaped_];
            c.reinit = P_.reinit_every > 0 && (steps_ % P_.reinit_every) == 0;
            Fwd* f = nullptr;
            sph_status s = fwd_slot((size_t)ntaped_, f);
            if (s != SPH_OK) return s;
            if (f) {
                // the step writes its neighbour lists straight into the
                // products (kernel by kernel: a graph holds the live lists)
                int32_t *lf = nbf_, *lw = nbw_, *lc = ncnt_;
                nbf_ = f->nbf;
                nbw_ = f->nbw;
                ncnt_ = f->ncnt;
                s = one_step(c.reinit, true, sigma_next());
                nbf_ = lf;
                nbw_ = lw;
                ncnt_ = lc;
                if (s == SPH_OK) s = keep_products(*f, c.par);
            } else {
                s = prof_mask_ ? one_step(c.reinit, true, sigma_next()) : graph_step(c.reinit, true, sigma_next());
            }
            if (s != SPH_OK) return s;
            // the dt the step used, kept on the device for the recompute
            SPH_CUDA(cudaMemcpyAsync(c.dtd, d_dt_, sizeof(T), cudaMemcpyDeviceToDevice, stream));
            ++steps_;
            ++ntaped_;
            tape_end_ = steps_;
        }
        for (int64_t k = first; k < ntaped_; ++k)
            SPH_CUDA(cudaMemcpyAsync(&ck_[(size_t)k].dt, ck_[(size_t)k].dtd, sizeof(T), cudaMemcpyDeviceToHost,
                                     stream));
        return finish_steps(dt_out);
    }

    sph_status tape_budget(int64_t bytes) override
    {
        fwd_limit_ = bytes;
        fwd_budget_ = bytes >= 0 ? (size_t)bytes : 0;
        return SPH_OK;
    }

    sph_status backward(const sph_adjoint_seed& seed, sph_adjoint_grad& grad, int32_t where) override
    {
        // the periodic forms of the adjoint kernels only where an axis wraps
        return P_.periodic ? backward_impl<true>(seed, grad, where) : backward_impl<false>(seed, grad, where);
    }

    template <bool PER>
    sph_status backward_impl(const sph_adjoint_seed& seed, sph_adjoint_grad& grad, int32_t where)
    {
        if (ck_.empty()) {
            err = "nothing was taped";
            return SPH_ERR_STATE;
        }
        if (steps_ != tape_end_) {
            err = "untaped steps were taken since the last sph_tape";
            return SPH_ERR_STATE;
        }
        sph_status s = adj_allocate();
        if (s != SPH_OK) return s;
        const size_t nf = (size_t)nf_, nw = (size_t)nw_;
        // seeds and outputs on the device (FP64, original order)
        const double *sx = seed.x, *sv = seed.v, *srho = seed.rho, *spw = seed.pw;
        double *ox = grad.x, *ov = grad.v, *orho = grad.rho;
        if (where == SPH_HOST) {
            double* b = adj_io_;
            auto up = [&](const double*& p, size_t cnt, double* dst) -> sph_status {
                if (!p) return SPH_OK;
                SPH_CUDA(cudaMemcpyAsync(dst, p, sizeof(double) * cnt, cudaMemcpyHostToDevice, stream));
                p = dst;
                return SPH_OK;
            };
            if ((s = up(sx, 3 * nf, b)) != SPH_OK) return s;
            if ((s = up(sv, 3 * nf, b + 3 * nf)) != SPH_OK) return s;
            if ((s = up(srho, nf, b + 6 * nf)) != SPH_OK) return s;
            if ((s = up(spw, nw, b + 7 * nf)) != SPH_OK) return s;
            ox = grad.x ? b + 7 * nf + nw : nullptr;
            ov = grad.v ? b + 10 * nf + nw : nullptr;
            orho = grad.rho ? b + 13 * nf + nw : nullptr;
        }
        if ((s = save(snap_)) != SPH_OK) return s;
        SPH_CUDA(cudaMemsetAsync(adj_param_, 0, 3 * sizeof(double), stream));
        int cur = 0;  // adjoint state buffers in use
        if (nf_ > 0)
            SPH_KERNEL(SPH_K_ADJ_OTHER, 1,
                       k_adj_seed<T><<<grid_for(nf_), BLOCK, 0, stream>>>(nf_, id_[par_], sx, sv, srho, gx_[0],
                                                                         gv_[0], ga_[0]));
        if (nw_ > 0)
            SPH_KERNEL(SPH_K_ADJ_OTHER, 1,
                       k_adj_seed_wall<T><<<grid_for(nw_), BLOCK, 0, stream>>>(nw_, wid_, spw, gpw_[0]));

        for (int64_t k = ntaped_ - 1; k >= 0; --k) {
            const Ckpt& c = ck_[(size_t)k];
            const Fwd* f = (size_t)k < fwd_.size() && fwd_[(size_t)k].buf ? &fwd_[(size_t)k] : nullptr;
            const int p = c.par, q = p ^ 1;
            if (!f) {
                if ((s = restore(c)) != SPH_OK) return s;
                // recompute the step bit-identically (same dt, same reinit)
                SPH_CUDA(cudaMemcpyAsync(d_dt_fixed_, c.dtd, sizeof(T), cudaMemcpyDeviceToDevice, stream));
                // (momentum's outputs a', v', sigma' are not read by the backward)
                s = prof_mask_ ? one_step(c.reinit, false) : graph_step(c.reinit, false);
                if (s != SPH_OK) return s;
            }
            // the step's products: kept from the tape, or just recomputed
            const int32_t* fs = f ? f->fstart : fstart_;
            const int32_t *lf = f ? f->nbf : nbf_, *lw = f ? f->nbw : nbw_, *lc = f ? f->ncnt : ncnt_;
            const V4<T>* P0 = f ? f->pos0 : pos_[0];
            const V4<T>* P1 = f ? f->pos1 : pos_[1];
            const V4<T>* VP = f ? f->velp : vel_[p];
            const T* R0 = f ? f->drho0 : drho_[0];
            const T* R1 = f ? f->drho1 : drho_[1];
            const int4* CQ = f ? f->cellq : cell_[q];
            const int32_t* IQ = f ? f->idq : id_[q];
            const V4<T>* WP = f ? f->wpos : wpos_;
            const V2<T>* WR = f ? f->wrho : wrho_;
            const int32_t* WT = f ? f->wtag : wtag_;
            const int32_t* TG = f ? f->tag : d_tag_;
            const V4<T>* GE = f ? f->geff : d_geff_;
            const int nxt = cur ^ 1;
            const T dt = c.dt;
            if (nf_ > 0) {
                SPH_KERNEL(SPH_K_ADJ_OTHER, 1,
                           k_adj_inverse<<<grid_for(nf_), BLOCK, 0, stream>>>(nf_, c.id, adj_inv_));
                SPH_KERNEL(SPH_K_ADJ_OTHER, 1,
                           k_adj_prep<T><<<grid_for(nf_), BLOCK, 0, stream>>>(nf_, T(0.5) * dt, gv_[cur], ga_[cur],
                                                                              tA_));
            }
            if (nw_ > 0)
                SPH_KERNEL(SPH_K_ADJ_WALL, 1,
                           k_adj_wall_momentum<T, PER><<<grid_for((int64_t)nw_ * AWLP), BLOCK, 0, stream>>>(
                               C_, nw_, fs, WP, WR, wnrm_, wcell_, WT, TG, P0, VP, tA_, gpw_[cur], wc_, adj_param_,
                               wfront_));
            // The wall continuity adjoint reads only tX of the momentum
            // adjoint and writes only gpw and the parameter sums, so it runs
            // beside the fluid continuity adjoint on a side stream (not while
            // kernels are timed one by one).
            const bool overlap = adj_side_ && !prof_mask_ && nf_ > 0 && nw_ > 0;
            if (nf_ > 0) {
                SPH_KERNEL(SPH_K_ADJ_MOMENTUM, 1,
                           k_adj_momentum<T, PER><<<grid_for((int64_t)nf_ * LP), BLOCK, 0, stream>>>(
                               C_, nf_, dt, 0, fs, wstart_, lf, lw, lc, P0, VP, R0, CQ, WP, WR, wnrm_, wc_, tA_,
                               gx_[cur], gv_[cur], GE, tX_, tV_, adj_param_, wfront_));
                if (overlap) {
                    SPH_CUDA(cudaEventRecord(adj_ev_[0], stream));
                    SPH_CUDA(cudaStreamWaitEvent(adj_side_, adj_ev_[0], 0));
                    k_adj_wall_continuity<T, PER><<<grid_for((int64_t)nw_ * AWLP), BLOCK, 0, adj_side_>>>(
                        C_, nw_, fs, c.wpos, c.wrho, wcell_, WT, TG, P1, VP, R1, tX_, gpw_[nxt], adj_param_);
                    SPH_LAUNCH();
                    launches_[SPH_K_ADJ_WALL] += 1;
                    SPH_CUDA(cudaEventRecord(adj_ev_[1], adj_side_));
                }
                SPH_KERNEL(SPH_K_ADJ_CONTINUITY, 1,
                           k_adj_continuity<T, PER><<<grid_for((int64_t)nf_ * LP), BLOCK, 0, stream>>>(
                               C_, nf_, dt, c.reinit ? 1 : 0, fs, wstart_, lf, lw, lc, P1, VP, R1, CQ, c.wpos,
                               c.wrho, tX_, tV_, gx_[cur], IQ, adj_inv_, c.drho, c.sigma, gx_[nxt], gv_[nxt],
                               ga_[nxt], adj_param_));
                if (overlap) SPH_CUDA(cudaStreamWaitEvent(stream, adj_ev_[1], 0));
            }
            if (nw_ > 0 && !overlap)
                SPH_KERNEL(SPH_K_ADJ_WALL, 1,
                           k_adj_wall_continuity<T, PER><<<grid_for((int64_t)nw_ * AWLP), BLOCK, 0, stream>>>(
                               C_, nw_, fs, c.wpos, c.wrho, wcell_, WT, TG, P1, VP, R1, tX_, gpw_[nxt], adj_param_));
            cur = nxt;
        }

        // the sweeps of sph_create at r^0: wall pressure, a^0, sigma^0
        if ((s = restore(ck_[0])) != SPH_OK) return s;
        SPH_KERNEL(SPH_K_ADJ_OTHER, 1, k_bump_tag<<<1, 32, 0, stream>>>(d_tag_));
        if ((s = neighbors(pos_[0], cell_[par_])) != SPH_OK) return s;
        const int p0 = par_;
        if (nf_ > 0)
            SPH_KERNEL(SPH_K_ADJ_OTHER, 1,
                       k_adj_prep<T><<<grid_for(nf_), BLOCK, 0, stream>>>(nf_, T(0), gv_[cur], ga_[cur], tA_));
        if (nw_ > 0)
            SPH_KERNEL(SPH_K_ADJ_WALL, 1,
                       k_adj_wall_momentum<T, PER><<<grid_for((int64_t)nw_ * AWLP), BLOCK, 0, stream>>>(
                           C_, nw_, fstart_, wpos_, wrho_, wnrm_, wcell_, wtag_, d_tag_, pos_[0], vel_[p0], tA_,
                           gpw_[cur], wc_, adj_param_, wfront_));
        if (nf_ > 0) {
            SPH_KERNEL(SPH_K_ADJ_MOMENTUM, 1,
                       k_adj_momentum<T, PER><<<grid_for((int64_t)nf_ * LP), BLOCK, 0, stream>>>(
                           C_, nf_, T(0), 1, fstart_, wstart_, nbf_, nbw_, ncnt_, pos_[0], vel_[p0], drho_[0],
                           cell_[p0], wpos_, wrho_, wnrm_, wc_, tA_, gx_[cur], gv_[cur], d_geff_, tX_, tV_,
                           adj_param_, wfront_));
            SPH_KERNEL(SPH_K_ADJ_OTHER, 1,
                       k_adj_export<T><<<grid_for(nf_), BLOCK, 0, stream>>>(nf_, id_[p0], tX_, tV_, ox, ov, orho));
        }
        SPH_CUDA(cudaMemcpyAsync(grad.params, adj_param_, 3 * sizeof(double), cudaMemcpyDeviceToHost, stream));
        if ((s = restore(snap_)) != SPH_OK) return s;
        dt_valid_ = false;  // the recompute rewrote the device dt word
        if (where == SPH_HOST) {
            if (grad.x) SPH_CUDA(cudaMemcpyAsync(grad.x, ox, sizeof(double) * 3 * nf, cudaMemcpyDeviceToHost, stream));
            if (grad.v) SPH_CUDA(cudaMemcpyAsync(grad.v, ov, sizeof(double) * 3 * nf, cudaMemcpyDeviceToHost, stream));
            if (grad.rho)
                SPH_CUDA(cudaMemcpyAsync(grad.rho, orho, sizeof(double) * nf, cudaMemcpyDeviceToHost, stream));
        }
        SPH_CUDA(cudaStreamSynchronize(stream));
        return index_check();
    }

    sph_status profile(uint32_t mask) override
    {
        SPH_CUDA(cudaStreamSynchronize(stream));
        prof_mask_ = mask;
        ev_used_ = 0;
        return SPH_OK;
    }

    sph_status profile_read(double* ms, int64_t* timed, int64_t* launches) override
    {
        SPH_CUDA(cudaStreamSynchronize(stream));
        double acc_ms[SPH_NK] = {0};
        int64_t cnt[SPH_NK] = {0};
        for (size_t k = 0; k < ev_used_; ++k) {
            float t = 0.f;
            SPH_CUDA(cudaEventElapsedTime(&t, ev_[k].a, ev_[k].b));
            acc_ms[ev_[k].kind] += t;
            cnt[ev_[k].kind] += 1;
        }
        for (int k = 0; k < SPH_NK; ++k) {
            if (ms) ms[k] = acc_ms[k];
            if (timed) timed[k] = cnt[k];
            if (launches) launches[k] = launches_[k];
        }
        return SPH_OK;
    }

    sph_status get_state(const sph_state_out& o, int32_t where) override
    {
        if (o.sigma)
            if (sph_status s = ensure_sigma(); s != SPH_OK) return s;
        const bool host = where == SPH_HOST;
        const size_t n1 = sizeof(double) * (size_t)nf_, n3 = 3 * n1;
        const size_t w1 = sizeof(double) * (size_t)nw_;
        struct Req {
            double* user;
            size_t bytes;
            double* dev;
        };
        Req req[10] = {{o.pos, n3, nullptr},    {o.vel, n3, nullptr},     {o.rho, n1, nullptr},
                       {o.p, n1, nullptr},      {o.acc, n3, nullptr},     {o.drho_dt, n1, nullptr},
                       {o.sigma, n1, nullptr},  {o.pw, w1, nullptr},      {o.rhow, 2 * w1, nullptr},
                       {o.normal, 3 * w1, nullptr}};
        for (Req& r : req) {
            if (!r.user || r.bytes == 0) continue;
            if (host)
                SPH_CUDA(cudaMallocAsync(&r.dev, r.bytes, stream));
            else
                r.dev = r.user;
        }
        if (nf_ > 0) {
            ExportOut eo{req[0].dev, req[1].dev, req[2].dev, req[3].dev, req[4].dev, req[5].dev, req[6].dev};
            k_export_fluid<T><<<grid_for(nf_), BLOCK, 0, stream>>>(C_, I_, nf_, pos_[0], vel_[par_], drho_[0], acc_,
                                                                 sigma_, cell_[par_], id_[par_], phase_[par_],
                                                                 eo);
            SPH_LAUNCH();
        }
        if (nw_ > 0) {
            k_export_wall<T><<<grid_for(nw_), BLOCK, 0, stream>>>(nw_, wpos_, wrho_, wnrm_, wid_, req[7].dev,
                                                                req[8].dev, req[9].dev);
            SPH_LAUNCH();
        }
        if (host) {
            for (Req& r : req) {
                if (!r.dev) continue;
                SPH_CUDA(cudaMemcpyAsync(r.user, r.dev, r.bytes, cudaMemcpyDeviceToHost, stream));
                SPH_CUDA(cudaFreeAsync(r.dev, stream));
            }
        }
        SPH_CUDA(cudaStreamSynchronize(stream));
        return SPH_OK;
    }

    // The neighbour sets the last sweeps visited (sph_get_neighbors), in
    // original ids, each particle's ids ascending.  When the context's lists
    // do not hold the build of the current state (after a taped step that
    // wrote its lists elsewhere, or a backward sweep), the builder runs again
    // on the current state first: it is deterministic, so the lists are
    // those of the last step.
    sph_status get_neighbors(int64_t* f_off, int32_t* f_ids, int64_t f_cap, int64_t* w_off, int32_t* w_ids,
                             int64_t w_cap, int64_t overflow[2])
    {
        const size_t lanes = (size_t)LP * (size_t)nf_;
        if (nf_ == 0) {
            if (f_off) f_off[0] = 0;
            if (w_off) w_off[0] = 0;
            if (overflow) overflow[0] = overflow[1] = 0;
            return SPH_OK;
        }
        if (!lists_current_) {
            sph_status s = neighbors(pos_[0], cell_[par_]);
            if (s != SPH_OK) return s;
        }
        int32_t* lc = nullptr;
        unsigned long long* dof = nullptr;
        SPH_CUDA(cudaMallocAsync(&lc, sizeof(int32_t) * 2 * lanes, stream));
        SPH_CUDA(cudaMallocAsync(&dof, sizeof(unsigned long long) * 2, stream));
        SPH_CUDA(cudaMemsetAsync(dof, 0, sizeof(unsigned long long) * 2, stream));
        const unsigned nb = (unsigned)((lanes + LBLOCK - 1) / LBLOCK);
        if (P_.periodic)
            k_nb_count<T, true><<<nb, LBLOCK, 0, stream>>>(C_, nf_, fstart_, wstart_, nbf_, nbw_, ncnt_, pos_[0],
                                                           wpos_, cell_[par_], lc, dof);
        else
            k_nb_count<T, false><<<nb, LBLOCK, 0, stream>>>(C_, nf_, fstart_, wstart_, nbf_, nbw_, ncnt_, pos_[0],
                                                            wpos_, cell_[par_], lc, dof);
        SPH_LAUNCH();
        std::vector<int32_t> hc(2 * lanes), hid((size_t)nf_);
        unsigned long long hof[2] = {0, 0};
        SPH_CUDA(cudaMemcpyAsync(hc.data(), lc, sizeof(int32_t) * 2 * lanes, cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaMemcpyAsync(hof, dof, sizeof hof, cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaMemcpyAsync(hid.data(), id_[par_], sizeof(int32_t) * (size_t)nf_, cudaMemcpyDeviceToHost,
                                 stream));
        SPH_CUDA(cudaStreamSynchronize(stream));
        SPH_CUDA(cudaFreeAsync(lc, stream));
        SPH_CUDA(cudaFreeAsync(dof, stream));
        if (sph_status sc = index_check(); sc != SPH_OK) return sc;
        if (overflow) {
            overflow[0] = (int64_t)hof[0];
            overflow[1] = (int64_t)hof[1];
        }
        // lane offsets in sorted order (fluid lanes, then wall lanes), and
        // per-particle counts in original order
        std::vector<int64_t> loff(2 * lanes + 2);
        std::vector<int64_t> cf((size_t)nf_ + 1, 0), cw((size_t)nf_ + 1, 0);
        int64_t tf = 0, tw = 0;
        for (size_t t = 0; t < lanes; ++t) {
            loff[t] = tf;
            tf += hc[t];
            cf[(size_t)hid[t / LP]] += hc[t];
        }
        for (size_t t = 0; t < lanes; ++t) {
            loff[lanes + t] = tw;
            tw += hc[lanes + t];
            cw[(size_t)hid[t / LP]] += hc[lanes + t];
        }
        auto to_offsets = [&](std::vector<int64_t>& c, int64_t* out) {
            int64_t acc = 0;
            for (size_t i = 0; i <= (size_t)nf_; ++i) {
                const int64_t v = i < (size_t)nf_ ? c[i] : 0;
                c[i] = acc;
                acc += v;
            }
            if (out) memcpy(out, c.data(), sizeof(int64_t) * ((size_t)nf_ + 1));
        };
        to_offsets(cf, f_off);
        to_offsets(cw, w_off);
        if ((f_ids && f_cap < tf) || (w_ids && w_cap < tw)) {
            char buf[160];
            snprintf(buf, sizeof buf, "id buffers too small: %lld fluid and %lld wall entries needed",
                     (long long)tf, (long long)tw);
            err = buf;
            return SPH_ERR_ARG;
        }
        if (!f_ids && !w_ids) return SPH_OK;
        int64_t* doff = nullptr;
        int32_t *dout_f = nullptr, *dout_w = nullptr;
        SPH_CUDA(cudaMallocAsync(&doff, sizeof(int64_t) * 2 * lanes, stream));
        SPH_CUDA(cudaMallocAsync(&dout_f, sizeof(int32_t) * (size_t)(tf > 0 ? tf : 1), stream));
        SPH_CUDA(cudaMallocAsync(&dout_w, sizeof(int32_t) * (size_t)(tw > 0 ? tw : 1), stream));
        SPH_CUDA(cudaMemcpyAsync(doff, loff.data(), sizeof(int64_t) * 2 * lanes, cudaMemcpyHostToDevice, stream));
        if (P_.periodic)
            k_nb_fill<T, true><<<nb, LBLOCK, 0, stream>>>(C_, nf_, fstart_, wstart_, nbf_, nbw_, ncnt_, pos_[0],
                                                          wpos_, cell_[par_], id_[par_], wid_, doff, dout_f, dout_w);
        else
            k_nb_fill<T, false><<<nb, LBLOCK, 0, stream>>>(C_, nf_, fstart_, wstart_, nbf_, nbw_, ncnt_, pos_[0],
                                                           wpos_, cell_[par_], id_[par_], wid_, doff, dout_f,
                                                           dout_w);
        SPH_LAUNCH();
        std::vector<int32_t> hf((size_t)tf), hw((size_t)tw);
        if (tf > 0)
            SPH_CUDA(cudaMemcpyAsync(hf.data(), dout_f, sizeof(int32_t) * (size_t)tf, cudaMemcpyDeviceToHost, stream));
        if (tw > 0)
            SPH_CUDA(cudaMemcpyAsync(hw.data(), dout_w, sizeof(int32_t) * (size_t)tw, cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaStreamSynchronize(stream));
        SPH_CUDA(cudaFreeAsync(doff, stream));
        SPH_CUDA(cudaFreeAsync(dout_f, stream));
        SPH_CUDA(cudaFreeAsync(dout_w, stream));
        // each particle's lanes are consecutive: move its entries to its
        // original id's range and sort them
        auto place = [&](const std::vector<int32_t>& src, const std::vector<int64_t>& start, size_t base,
                         int32_t* out) {
            for (size_t i = 0; i < (size_t)nf_; ++i) {
                const int64_t b = loff[base + LP * i];
                const int64_t e = i + 1 < (size_t)nf_ ? loff[base + LP * (i + 1)] : (base ? tw : tf);
                int32_t* dst = out + start[(size_t)hid[i]];
                std::copy(src.begin() + b, src.begin() + e, dst);
                std::sort(dst, dst + (e - b));
            }
        };
        if (f_ids) place(hf, cf, 0, f_ids);
        if (w_ids) place(hw, cw, lanes, w_ids);
        SPH_CUDA(cudaStreamSynchronize(stream));
        return SPH_OK;
    }

    sph_status get_cells(uint32_t* kf, int32_t* of, int32_t* sf, uint32_t* kw, int32_t* ow,
                         int32_t* sw) override
    {
        uint32_t* dk = nullptr;
        int32_t* dord = nullptr;
        size_t nmax = (size_t)(nf_ > nw_ ? nf_ : nw_);
        if (nmax > 0) {
            SPH_CUDA(cudaMallocAsync(&dk, sizeof(uint32_t) * nmax, stream));
            SPH_CUDA(cudaMallocAsync(&dord, sizeof(int32_t) * nmax, stream));
        }
        if ((kf || of) && nf_ > 0) {
            k_export_cells<<<grid_for(nf_), BLOCK, 0, stream>>>(nf_, cell_[par_], id_[par_], dk, dord);
            SPH_LAUNCH();
            if (kf) SPH_CUDA(cudaMemcpyAsync(kf, dk, sizeof(uint32_t) * nf_, cudaMemcpyDeviceToHost, stream));
            if (of) SPH_CUDA(cudaMemcpyAsync(of, dord, sizeof(int32_t) * nf_, cudaMemcpyDeviceToHost, stream));
            SPH_CUDA(cudaStreamSynchronize(stream));
        }
        if (sf)
            SPH_CUDA(cudaMemcpyAsync(sf, fstart_, sizeof(int32_t) * (size_t)(n_cells_ + 1),
                                     cudaMemcpyDeviceToHost, stream));
        if ((kw || ow) && nw_ > 0) {
            k_export_cells<<<grid_for(nw_), BLOCK, 0, stream>>>(nw_, wcell_, wid_, dk, dord);
            SPH_LAUNCH();
            if (kw) SPH_CUDA(cudaMemcpyAsync(kw, dk, sizeof(uint32_t) * nw_, cudaMemcpyDeviceToHost, stream));
            if (ow) SPH_CUDA(cudaMemcpyAsync(ow, dord, sizeof(int32_t) * nw_, cudaMemcpyDeviceToHost, stream));
        }
        if (sw)
            SPH_CUDA(cudaMemcpyAsync(sw, wstart_, sizeof(int32_t) * (size_t)(n_cells_ + 1),
                                     cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaStreamSynchronize(stream));
        if (dk) SPH_CUDA(cudaFreeAsync(dk, stream));
        if (dord) SPH_CUDA(cudaFreeAsync(dord, stream));
        SPH_CUDA(cudaStreamSynchronize(stream));
        return SPH_OK;
    }

    sph_status diagnostics(double out[8]) override
    {
        sph_status s = diagnostics_async(host_status_->diag, SPH_HOST);
        if (s != SPH_OK) return s;
        SPH_CUDA(cudaStreamSynchronize(stream));
        memcpy(out, host_status_->diag, sizeof(double) * 8);
        return SPH_OK;
    }

    // the reductions and the copy of their 8 results to out (device memory,
    // or page-locked host memory), enqueued on the stream
    sph_status diagnostics_async(double* out, int32_t where) override
    {
        int nb = grid_for(nf_ > 0 ? nf_ : 1);
        if (nb > DIAG_MAX_BLOCKS) nb = DIAG_MAX_BLOCKS;
        SPH_KERNEL(SPH_K_OTHER, 1,
                   k_diag_partial<T><<<nb, BLOCK, 0, stream>>>(C_, I_, nf_, pos_[0], vel_[par_], cell_[par_],
                                                               phase_[par_], diag_partial_));
        SPH_KERNEL(SPH_K_OTHER, 1, k_diag_final<<<1, DIAG_THREADS, 0, stream>>>(nb, diag_partial_, diag_out_));
        SPH_CUDA(cudaMemcpyAsync(out, diag_out_, sizeof(double) * 8,
                                 where == SPH_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, stream));
        return SPH_OK;
    }

    // Sensors (Sec. 4.3) at n points; HOST: pts and outputs are host memory
    // and the call synchronises; DEVICE: device memory, enqueued only.
    sph_status probe_pressure(const double* pts, int32_t n, double* p, double* w, int32_t where) override
    {
        if (n == 0) return SPH_OK;
        const bool host = where == SPH_HOST;
        const size_t b1 = sizeof(double) * (size_t)n;
        const double* dpts = pts;
        double *dp = p, *dw = w, *scratch = nullptr;
        if (host) {
            SPH_CUDA(cudaMallocAsync(&scratch, 5 * b1, stream));
            SPH_CUDA(cudaMemcpyAsync(scratch, pts, 3 * b1, cudaMemcpyHostToDevice, stream));
            dpts = scratch;
            dp = p ? scratch + 3 * (size_t)n : nullptr;
            dw = w ? scratch + 4 * (size_t)n : nullptr;
        }
        const int64_t threads = (int64_t)n * 32;
        SPH_KERNEL(SPH_K_OTHER, 1,
                   k_probe_pressure<T><<<(unsigned)((threads + BLOCK - 1) / BLOCK), BLOCK, 0, stream>>>(
                       C_, D_, I_, n, dpts, fstart_, pos_[0], drho_[0], phase_[par_], dp, dw));
        if (host) {
            if (p) SPH_CUDA(cudaMemcpyAsync(p, dp, b1, cudaMemcpyDeviceToHost, stream));
            if (w) SPH_CUDA(cudaMemcpyAsync(w, dw, b1, cudaMemcpyDeviceToHost, stream));
            SPH_CUDA(cudaFreeAsync(scratch, stream));
            SPH_CUDA(cudaStreamSynchronize(stream));
        }
        return SPH_OK;
    }

    // Wave-height gauges (Sec. 4.3) on n vertical lines (x, y, z_lo, z_hi).
    sph_status gauge_height(const double* g, int32_t n, double dz, double* H, int32_t where) override
    {
        if (n == 0) return SPH_OK;
        const bool host = where == SPH_HOST;
        const size_t b1 = sizeof(double) * (size_t)n;
        const double* dg = g;
        double* dH = H;
        char* scratch = nullptr;  // [the lines, H (host path)], the best sample per line
        const size_t lines_b = host ? 5 * b1 : 0;
        SPH_CUDA(cudaMallocAsync(&scratch, lines_b + sizeof(int32_t) * (size_t)n, stream));
        if (host) {
            SPH_CUDA(cudaMemcpyAsync(scratch, g, 4 * b1, cudaMemcpyHostToDevice, stream));
            dg = (const double*)scratch;
            dH = (double*)scratch + 4 * (size_t)n;
        }
        int32_t* best = (int32_t*)(scratch + lines_b);
        SPH_CUDA(cudaMemsetAsync(best, 0xff, sizeof(int32_t) * (size_t)n, stream));  // -1: no wet sample yet
        SPH_KERNEL(SPH_K_OTHER, 1,
                   k_gauge_crossing<T><<<dim3(GAUGE_BLOCKS_PER_LINE, (unsigned)n), GAUGE_BLOCK, 0, stream>>>(
                       C_, D_, I_, n, dg, dz, fstart_, pos_[0], drho_[0], phase_[par_], best));
        const int64_t threads = (int64_t)n * 32;
        SPH_KERNEL(SPH_K_OTHER, 1,
                   k_gauge_finish<T><<<(unsigned)((threads + BLOCK - 1) / BLOCK), BLOCK, 0, stream>>>(
                       C_, D_, I_, n, dg, dz, fstart_, pos_[0], drho_[0], phase_[par_], best, dH));
        if (host) SPH_CUDA(cudaMemcpyAsync(H, dH, b1, cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaFreeAsync(scratch, stream));
        if (host) SPH_CUDA(cudaStreamSynchronize(stream));
        return SPH_OK;
    }

    sph_status counters(int64_t* steps, int64_t* active) override
    {
        SPH_CUDA(cudaMemcpyAsync(&host_status_->active, d_active_, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, stream));
        SPH_CUDA(cudaStreamSynchronize(stream));
        if (steps) *steps = steps_;
        if (active) *active = (int64_t)host_status_->active;
        return SPH_OK;
    }

    void grid(int32_t dims[3], int64_t* n_cells, double* cs) const override
    {
        if (dims)
            for (int d = 0; d < 3; ++d) dims[d] = dims_[d];
        if (n_cells) *n_cells = n_cells_;
        if (cs) *cs = cs_;
    }

  private:
    struct HostStatus {
        int32_t flags, n_in, w_in, pad;
        T dt, dt_fixed;
        unsigned long long active;
        double diag[8];
        double time;
    };
    struct EvPair {
        cudaEvent_t a, b;
        int kind;
    };
    static constexpr size_t kMaxEvents = 1u << 18;

    sph_status fail_cuda(cudaError_t e, const char* what, int line)
    {
        char buf[256];
        snprintf(buf, sizeof buf, "CUDA error %s (%s) at %s [sph_sim.cuh:%d]", cudaGetErrorName(e),
                 cudaGetErrorString(e), what, line);
        err = buf;
        dead = true;
        return e == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA;
    }

    template <class U>
    sph_status alloc(U*& p, size_t count)
    {
        p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void**)&p, sizeof(U) * count);
        if (e != cudaSuccess) return fail_cuda(e, "cudaMalloc", __LINE__);
        allocs_.push_back((void*)p);
        return SPH_OK;
    }

    sph_status allocate()
    {
        size_t nf = (size_t)nf_, nw = (size_t)nw_, nc = (size_t)n_cells_;
        size_t nmax = nf > nw ? nf : nw;
        sph_status s = SPH_OK;
        for (int b = 0; b < 2 && s == SPH_OK; ++b) {
            if ((s = alloc(pos_[b], nf)) != SPH_OK) return s;
            if ((s = alloc(vel_[b], nf)) != SPH_OK) return s;
            if ((s = alloc(drho_[b], nf)) != SPH_OK) return s;
            if ((s = alloc(comp_[b], nf)) != SPH_OK) return s;
            if ((s = alloc(cell_[b], nf)) != SPH_OK) return s;
            if ((s = alloc(id_[b], nf)) != SPH_OK) return s;
            if ((s = alloc(phase_[b], nf)) != SPH_OK) return s;
        }
        if ((s = alloc(acc_, nf)) != SPH_OK) return s;
        if ((s = alloc(sigma_, nf)) != SPH_OK) return s;
        if ((s = alloc(nbf_, (size_t)SUBF * LP * nf)) != SPH_OK) return s;
        if ((s = alloc(nbw_, (size_t)SUBW * LP * nf)) != SPH_OK) return s;
        if ((s = alloc(ncnt_, (size_t)LP * nf)) != SPH_OK) return s;
        nbf_live_ = nbf_;
        if ((s = alloc(wtag_, nw)) != SPH_OK) return s;
        if ((s = alloc(wfront_, nw)) != SPH_OK) return s;
        if ((s = alloc(d_tag_, 1)) != SPH_OK) return s;
        if ((s = alloc(newcell_, nmax)) != SPH_OK) return s;
        if ((s = alloc(rank_, nmax)) != SPH_OK) return s;
        if ((s = alloc(tmp_src_, nmax)) != SPH_OK) return s;
        if ((s = alloc(tmp_id_, nmax)) != SPH_OK) return s;
        if ((s = alloc(counts_, nc + 1)) != SPH_OK) return s;
        if ((s = alloc(fstart_, nc + 2)) != SPH_OK) return s;
        if ((s = alloc(wstart_, nc + 2)) != SPH_OK) return s;
        if ((s = alloc(wrows_, nc)) != SPH_OK) return s;
        if ((s = alloc(sums_, (size_t)scan_blocks(n_cells_ + 1))) != SPH_OK) return s;
        if ((s = alloc(wpos_, nw)) != SPH_OK) return s;
        if ((s = alloc(wpos_tmp_, nw)) != SPH_OK) return s;
        if ((s = alloc(wrho_, nw)) != SPH_OK) return s;
        if ((s = alloc(wnrm_, nw)) != SPH_OK) return s;
        if ((s = alloc(wcell_, nw)) != SPH_OK) return s;
        if ((s = alloc(wcell_tmp_, nw)) != SPH_OK) return s;
        if ((s = alloc(wid_, nw)) != SPH_OK) return s;
        if ((s = alloc(wid_tmp_, nw)) != SPH_OK) return s;
        if ((s = alloc(d_dt_, 1)) != SPH_OK) return s;
        if ((s = alloc(d_dt_fixed_, 1)) != SPH_OK) return s;
        if ((s = alloc(d_vmax_, 1)) != SPH_OK) return s;
        if ((s = alloc(d_time_, 1)) != SPH_OK) return s;
        if ((s = alloc(d_geff_, 1)) != SPH_OK) return s;
        if ((s = alloc(d_flags_, 1)) != SPH_OK) return s;
        if ((s = alloc(d_active_, 1)) != SPH_OK) return s;
        if ((s = alloc(diag_partial_, 8 * (size_t)grid_for(nf_ > 0 ? nf_ : 1))) != SPH_OK) return s;
        if ((s = alloc(diag_out_, 8)) != SPH_OK) return s;
        return SPH_OK;
    }

    // neighbour lists of the sorted fluid at positions pts / cells cell
    sph_status neighbors(const V4<T>* pts, const int4* cell)
    {
        lists_current_ = nbf_ == nbf_live_;
        if (nf_ == 0) return SPH_OK;
        {
            // the periodic form only where an axis wraps: the others compile its code out
            auto launch = [&](auto kernel) {
                kernel<<<grid_for((int64_t)nf_ * LP), BLOCK, 0, stream>>>(
                    C_, nf_, fstart_, wstart_, wrows_, pts, wpos_, cell, nbf_, nbw_, ncnt_, wtag_, d_tag_);
            };
            SPH_KERNEL(SPH_K_NEIGHBORS, 1,
                       P_.periodic ? launch(k_neighbors<T, true>) : launch(k_neighbors<T, false>));
        }
        return SPH_OK;
    }

    // Eq. (wallPressure) from the fluid state pos[0] / vel_cur
    sph_status wall_pressure(const V4<T>* vel_cur)
    {
        if (nw_ == 0) return SPH_OK;
        {
            // the periodic form only where an axis wraps: the others compile its code out
            // WLP lanes per wall particle, WLP_LARGE for large wall sets
            const bool large = nw_ >= WLP_LARGE_MIN;
            const int lanes = large ? WLP_LARGE : WLP;
            auto launch = [&](auto kernel) {
                kernel<<<grid_for((int64_t)nw_ * lanes), BLOCK, 0, stream>>>(
                    C_, nw_, fstart_, wpos_, wcell_, pos_[0], vel_cur, wrho_, wtag_, d_tag_, d_geff_, d_active_, wnrm_);
            };
            if (large)
                SPH_KERNEL(SPH_K_WALL_PRESSURE, 1,
                           P_.periodic ? launch(k_wall_pressure<T, true, WLP_LARGE>)
                                       : launch(k_wall_pressure<T, false, WLP_LARGE>));
            else
                SPH_KERNEL(SPH_K_WALL_PRESSURE, 1,
                           P_.periodic ? launch(k_wall_pressure<T, true>) : launch(k_wall_pressure<T, false>));
        }
        return SPH_OK;
    }

    // momentum from pos[0] / vel_cur; writes acc, vel_out (final kick),
    // sigma - sigma^0 and U_max
    sph_status momentum(const V4<T>* vel_cur, V4<T>* vel_out, const int4* cell, const int32_t* phase,
                        bool sigma = true)
    {
        if (nf_ == 0) return SPH_OK;
        {
            // the periodic form only where an axis wraps: the others compile its code out
            auto launch = [&](auto kernel) {
                kernel<<<grid_for((int64_t)nf_ * LP), BLOCK, 0, stream>>>(
                    C_, nf_, fstart_, wstart_, nbf_, nbw_, ncnt_, pos_[0], vel_cur, cell, phase, wpos_, wrho_, wnrm_,
                    d_dt_, d_geff_, acc_, vel_out, sigma_, d_vmax_, d_flags_);
            };
            if (sigma)
                SPH_KERNEL(SPH_K_MOMENTUM, 1,
                           P_.periodic ? launch(k_momentum<T, true, true>) : launch(k_momentum<T, false, true>));
            else
                SPH_KERNEL(SPH_K_MOMENTUM, 1,
                           P_.periodic ? launch(k_momentum<T, true, false>) : launch(k_momentum<T, false, false>));
            sigma_valid_ = sigma;
        }
        return SPH_OK;
    }

    // One kick-drift-kick step (Sec. 2.6).  Buffer roles with p = par_, q = p^1:
    //   gather    : pos[0], vel[p], drho[0], comp/cell/id/phase[p] (old order)
    //               -> pos[1], vel[q], drho[1], comp/cell/id/phase[q] (new order)
    //   continuity: pos[1], vel[q], drho[1] -> pos[0], vel[p], drho[0], acc.w
    //   wall pressure, momentum read pos[0], vel[p]; momentum writes vel[q]
    // so pos and drho stay in [0] while vel, comp, cell, id, phase alternate.
    sph_status one_step(bool reinit, bool with_momentum = true, bool sigma = true)
    {
        const int p = par_, q = par_ ^ 1;
        // the step's dt and wall tag come from k_predict, the U_max reset from
        // k_scatter, and the scan leaves the cell counters cleared; without
        // fluid a small kernel does all of it
        if (nf_ > 0)
            SPH_KERNEL(SPH_K_PREDICT, 1,
                       k_predict<T, KAHAN><<<grid_for(nf_), BLOCK, 0, stream>>>(
                           C_, nf_, pos_[0], vel_[p], acc_, comp_[p], cell_[p], d_dt_fixed_, d_vmax_, d_dt_, d_tag_,
                           d_time_, d_geff_, newcell_, rank_, counts_));
        else
            SPH_KERNEL(SPH_K_BEGIN_STEP, 1,
                       k_begin_step<T><<<grid_for(n_cells_ + 1), BLOCK, 0, stream>>>(
                           C_, d_dt_fixed_, d_vmax_, d_dt_, counts_, n_cells_ + 1, d_tag_, d_time_, d_geff_));
        int nscan = 0;
        SPH_KERNEL(SPH_K_SCAN, nscan, nscan = scan_exclusive(counts_, n_cells_ + 1, fstart_, sums_, stream, counts_));
        if (nf_ > 0) {
            SPH_KERNEL(SPH_K_SCATTER, 1,
                       k_scatter<<<grid_for(nf_), BLOCK, 0, stream>>>(nf_, n_cells_, newcell_, rank_, fstart_,
                                                                      id_[p], tmp_src_, tmp_id_, d_vmax_));
            SPH_KERNEL(SPH_K_GATHER, 1,
                       k_gather<T, KAHAN><<<grid_for(nf_), BLOCK, 0, stream>>>(
                           C_, nf_, fstart_, tmp_src_, tmp_id_, newcell_, d_dt_, reinit ? 1 : 0, pos_[0], vel_[p],
                           drho_[0], acc_, comp_[p], sigma_, cell_[p], phase_[p], pos_[1], vel_[q], drho_[1],
                           comp_[q], cell_[q], id_[q], phase_[q]));
            sph_status sn = neighbors(pos_[1], cell_[q]);
            if (sn != SPH_OK) return sn;
            {
                // the periodic form only where an axis wraps: the others compile its code out
                auto launch = [&](auto kernel) {
                    kernel<<<grid_for((int64_t)nf_ * LP), BLOCK, 0, stream>>>(
                        C_, nf_, fstart_, wstart_, nbf_, nbw_, ncnt_, pos_[1], vel_[q], drho_[1], cell_[q], phase_[q],
                        wpos_, wrho_, d_dt_, pos_[0], vel_[p], drho_[0], acc_, sigma_);
                };
                SPH_KERNEL(SPH_K_CONTINUITY, 1,
                           P_.periodic ? launch(k_continuity<T, true>) : launch(k_continuity<T, false>));
            }
        }
        sph_status s = wall_pressure(vel_[p]);
        if (s != SPH_OK) return s;
        if (with_momentum) {
            s = momentum(vel_[p], vel_[q], cell_[q], phase_[q], sigma);
            if (s != SPH_OK) return s;
        }
        par_ = q;
        return SPH_OK;
    }

    // One step through a CUDA graph of its kernel sequence.  The buffer roles
    // alternate between steps and the reinitialisation flag changes one
    // kernel argument, so up to four graphs exist, captured on first use on
    // an internal stream (the caller's may be the legacy default stream,
    // which cannot be captured) and launched on the caller's stream.
    sph_status graph_step(bool reinit, bool with_momentum = true, bool sigma = true)
    {
        const int key = (sigma ? 8 : 0) | (with_momentum ? 0 : 4) | (par_ << 1) | (reinit ? 1 : 0);
        if (!gexec_[key]) {
            if (!cap_stream_) SPH_CUDA(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
            cudaStream_t user = stream;
            const int par0 = par_;
            int64_t before[SPH_NK];
            memcpy(before, launches_, sizeof before);
            stream = cap_stream_;
            cudaError_t e = cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal);
            sph_status s = e == cudaSuccess ? one_step(reinit, with_momentum, sigma) : SPH_OK;
            cudaGraph_t g = nullptr;
            cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cap_stream_, &g) : e;
            stream = user;
            par_ = par0;
            for (int k = 0; k < SPH_NK; ++k) {
                glaunch_[key][k] = launches_[k] - before[k];
                launches_[k] = before[k];
            }
            if (s != SPH_OK) {
                if (g) cudaGraphDestroy(g);
                return s;
            }
            SPH_CUDA(e2);
            e = cudaGraphInstantiate(&gexec_[key], g, 0);
            cudaGraphDestroy(g);
            SPH_CUDA(e);
        }
        SPH_CUDA(cudaGraphLaunch(gexec_[key], stream));
        if (with_momentum) sigma_valid_ = sigma;
        for (int k = 0; k < SPH_NK; ++k) launches_[k] += glaunch_[key][k];
        par_ ^= 1;
        return SPH_OK;
    }

    // Checkpoint of the mutable state (the buffers of the current parity).
    struct Ckpt {
        char* buf = nullptr;
        V4<T>*pos = nullptr, *vel = nullptr, *acc = nullptr, *comp = nullptr, *wpos = nullptr;
        T *drho = nullptr, *sigma = nullptr, *dtd = nullptr;  // dtd: the step's dt (device)
        int4* cell = nullptr;
        int32_t *id = nullptr, *phase = nullptr, *fstart = nullptr;
        V2<T>* wrho = nullptr;
        unsigned long long *vmax = nullptr, *active = nullptr;
        double* time = nullptr;
        V4<T>* geff = nullptr;
        int par = 0;
        int64_t steps = 0;
        T dt = T(0);
        bool reinit = false;
        bool sigma_valid = false;
    };

    sph_status save(Ckpt& c)
    {
        const size_t nf = (size_t)nf_, nw = (size_t)nw_;
        if (!c.buf) {
            size_t off = 0;
            auto take = [&](size_t bytes) {
                size_t at = off;
                off += (bytes + 255) & ~(size_t)255;
                return at;
            };
            const size_t o_pos = take(nf * sizeof(V4<T>)), o_vel = take(nf * sizeof(V4<T>)),
                         o_acc = take(nf * sizeof(V4<T>)), o_comp = take(nf * sizeof(V4<T>)),
                         o_drho = take(nf * sizeof(T)), o_sig = take(nf * sizeof(T)),
                         o_cell = take(nf * sizeof(int4)), o_id = take(nf * sizeof(int32_t)),
                         o_ph = take(nf * sizeof(int32_t)), o_wpos = take(nw * sizeof(V4<T>)),
                         o_wrho = take(nw * sizeof(V2<T>)), o_vm = take(sizeof(unsigned long long)),
                         o_ac = take(sizeof(unsigned long long)),
                         o_fs = take(((size_t)n_cells_ + 2) * sizeof(int32_t)), o_dt = take(sizeof(T)),
                         o_tm = take(sizeof(double)), o_ge = take(sizeof(V4<T>));
            sph_status s = alloc(c.buf, off);
            if (s != SPH_OK) return s;
            c.pos = (V4<T>*)(c.buf + o_pos);
            c.vel = (V4<T>*)(c.buf + o_vel);
            c.acc = (V4<T>*)(c.buf + o_acc);
            c.comp = (V4<T>*)(c.buf + o_comp);
            c.drho = (T*)(c.buf + o_drho);
            c.sigma = (T*)(c.buf + o_sig);
            c.cell = (int4*)(c.buf + o_cell);
            c.id = (int32_t*)(c.buf + o_id);
            c.phase = (int32_t*)(c.buf + o_ph);
            c.wpos = (V4<T>*)(c.buf + o_wpos);
            c.wrho = (V2<T>*)(c.buf + o_wrho);
            c.vmax = (unsigned long long*)(c.buf + o_vm);
            c.active = (unsigned long long*)(c.buf + o_ac);
            c.fstart = (int32_t*)(c.buf + o_fs);
            c.dtd = (T*)(c.buf + o_dt);
            c.time = (double*)(c.buf + o_tm);
            c.geff = (V4<T>*)(c.buf + o_ge);
        }
        c.par = par_;
        c.steps = steps_;
        c.sigma_valid = sigma_valid_;
        return copy_ckpt(c, true);
    }

    // One launch copying every array of a checkpoint (to it when save, from
    // it otherwise).  The cell ranges are included: a step recomputes them,
    // but the create-time sweeps and sph_get_cells read them.
    sph_status copy_ckpt(const Ckpt& c, bool save)
    {
        const size_t nf = (size_t)nf_, nw = (size_t)nw_;
        const int p = c.par;
        CopyList L{};
        auto add = [&](void* state, void* ck, size_t bytes) {
            CopySeg& g = L.seg[L.n++];
            g.dst = save ? ck : state;
            g.src = save ? state : ck;
            g.words = bytes / 4;
            L.total += g.words;
        };
        add(pos_[0], c.pos, nf * sizeof(V4<T>));
        add(vel_[p], c.vel, nf * sizeof(V4<T>));
        add(acc_, c.acc, nf * sizeof(V4<T>));
        add(comp_[p], c.comp, nf * sizeof(V4<T>));
        add(drho_[0], c.drho, nf * sizeof(T));
        add(sigma_, c.sigma, nf * sizeof(T));
        add(cell_[p], c.cell, nf * sizeof(int4));
        add(id_[p], c.id, nf * sizeof(int32_t));
        add(phase_[p], c.phase, nf * sizeof(int32_t));
        add(wpos_, c.wpos, nw * sizeof(V4<T>));
        add(wrho_, c.wrho, nw * sizeof(V2<T>));
        add(d_vmax_, c.vmax, sizeof(unsigned long long));
        add(d_active_, c.active, sizeof(unsigned long long));
        add(fstart_, c.fstart, ((size_t)n_cells_ + 2) * sizeof(int32_t));
        add(d_time_, c.time, sizeof(double));
        add(d_geff_, c.geff, sizeof(V4<T>));
        const int64_t want = (int64_t)((L.total / 4 + 255) / 256);
        const int nb = (int)(want < 1 ? 1 : (want > 152 * 8 ? 152 * 8 : want));
        SPH_KERNEL(SPH_K_ADJ_OTHER, 1, k_copy_segments<<<nb, 256, 0, stream>>>(L));
        return SPH_OK;
    }

    // Products of a taped step that its backward reads, kept on the device
    // while memory allows, so that the reverse sweep need not recompute the
    // step: the neighbour lists (the step writes them there directly), the
    // sorted fluid after the continuity sweep (r^{n+1} with p^{n+1}) and as
    // gathered (r^{n+1} with p^n), v^{n+1/2}, both density excesses, cells and
    // ids of the new order, the cell ranges, the wall pressures and densities,
    // the wall support tags with the step's tag, and the body force.
    struct Fwd {
        char* buf = nullptr;
        int32_t *nbf = nullptr, *nbw = nullptr, *ncnt = nullptr;
        V4<T>*pos0 = nullptr, *pos1 = nullptr, *velp = nullptr, *wpos = nullptr, *geff = nullptr;
        T *drho0 = nullptr, *drho1 = nullptr;
        int4* cellq = nullptr;
        int32_t *idq = nullptr, *fstart = nullptr, *wtag = nullptr, *tag = nullptr;
        V2<T>* wrho = nullptr;
    };

    // The products of taped step k: f = &fwd_[k] with its buffer allocated,
    // or nullptr once the products of the run would pass the budget (by
    // default half the device memory free when the first one is kept); those
    // steps are recomputed by the backward.
    sph_status fwd_slot(size_t k, Fwd*& f)
    {
        f = nullptr;
        if (fwd_.size() <= k) fwd_.resize(k + 1);
        Fwd& g = fwd_[k];
        if (g.buf) {
            f = &g;
            return SPH_OK;
        }
        const size_t nf = (size_t)nf_, nw = (size_t)nw_;
        size_t off = 0;
        auto take = [&](size_t bytes) {
            size_t at = off;
            off += (bytes + 255) & ~(size_t)255;
            return at;
        };
        const size_t o_nbf = take((size_t)SUBF * LP * nf * sizeof(int32_t)),
                     o_nbw = take((size_t)SUBW * LP * nf * sizeof(int32_t)),
                     o_cnt = take((size_t)LP * nf * sizeof(int32_t)), o_p0 = take(nf * sizeof(V4<T>)),
                     o_p1 = take(nf * sizeof(V4<T>)), o_v = take(nf * sizeof(V4<T>)), o_r0 = take(nf * sizeof(T)),
                     o_r1 = take(nf * sizeof(T)), o_c = take(nf * sizeof(int4)), o_id = take(nf * sizeof(int32_t)),
                     o_fs = take(((size_t)n_cells_ + 2) * sizeof(int32_t)), o_wp = take(nw * sizeof(V4<T>)),
                     o_wr = take(nw * sizeof(V2<T>)), o_wt = take(nw * sizeof(int32_t)),
                     o_tg = take(sizeof(int32_t)), o_ge = take(sizeof(V4<T>));
        if (fwd_limit_ < 0 && fwd_budget_ == 0) {
            size_t fr = 0, tot = 0;
            SPH_CUDA(cudaMemGetInfo(&fr, &tot));
            fwd_budget_ = fr / 2 > 1 ? fr / 2 : 1;
        }
        if (fwd_bytes_ + off > fwd_budget_) return SPH_OK;
        sph_status s = alloc(g.buf, off);
        if (s != SPH_OK) return s;
        fwd_bytes_ += off;
        g.nbf = (int32_t*)(g.buf + o_nbf);
        g.nbw = (int32_t*)(g.buf + o_nbw);
        g.ncnt = (int32_t*)(g.buf + o_cnt);
        g.pos0 = (V4<T>*)(g.buf + o_p0);
        g.pos1 = (V4<T>*)(g.buf + o_p1);
        g.velp = (V4<T>*)(g.buf + o_v);
        g.drho0 = (T*)(g.buf + o_r0);
        g.drho1 = (T*)(g.buf + o_r1);
        g.cellq = (int4*)(g.buf + o_c);
        g.idq = (int32_t*)(g.buf + o_id);
        g.fstart = (int32_t*)(g.buf + o_fs);
        g.wpos = (V4<T>*)(g.buf + o_wp);
        g.wrho = (V2<T>*)(g.buf + o_wr);
        g.wtag = (int32_t*)(g.buf + o_wt);
        g.tag = (int32_t*)(g.buf + o_tg);
        g.geff = (V4<T>*)(g.buf + o_ge);
        f = &g;
        return SPH_OK;
    }

    // Copy the products of the step just taken (it started with parity p)
    // next to its lists, in one launch.
    sph_status keep_products(Fwd& f, int p)
    {
        const size_t nf = (size_t)nf_, nw = (size_t)nw_;
        const int q = p ^ 1;
        CopyList L{};
        auto add = [&](const void* src, void* dst, size_t bytes) {
            CopySeg& g = L.seg[L.n++];
            g.dst = dst;
            g.src = const_cast<void*>(src);
            g.words = bytes / 4;
            L.total += g.words;
        };
        add(pos_[0], f.pos0, nf * sizeof(V4<T>));
        add(pos_[1], f.pos1, nf * sizeof(V4<T>));
        add(vel_[p], f.velp, nf * sizeof(V4<T>));
        add(drho_[0], f.drho0, nf * sizeof(T));
        add(drho_[1], f.drho1, nf * sizeof(T));
        add(cell_[q], f.cellq, nf * sizeof(int4));
        add(id_[q], f.idq, nf * sizeof(int32_t));
        add(fstart_, f.fstart, ((size_t)n_cells_ + 2) * sizeof(int32_t));
        add(wpos_, f.wpos, nw * sizeof(V4<T>));
        add(wrho_, f.wrho, nw * sizeof(V2<T>));
        add(wtag_, f.wtag, nw * sizeof(int32_t));
        add(d_tag_, f.tag, sizeof(int32_t));
        add(d_geff_, f.geff, sizeof(V4<T>));
        const int64_t want = (int64_t)((L.total / 4 + 255) / 256);
        const int nb = (int)(want < 1 ? 1 : (want > 152 * 8 ? 152 * 8 : want));
        SPH_KERNEL(SPH_K_ADJ_OTHER, 1, k_copy_segments<<<nb, 256, 0, stream>>>(L));
        return SPH_OK;
    }

    sph_status restore(const Ckpt& c)
    {
        lists_current_ = false;  // the lists belong to a later state
        sph_status s = copy_ckpt(c, false);
        if (s != SPH_OK) return s;
        par_ = c.par;
        steps_ = c.steps;
        sigma_valid_ = c.sigma_valid;
        return SPH_OK;
    }

    // adjoint work buffers, allocated on the first backward sweep
    sph_status adj_allocate()
    {
        if (adj_param_) return SPH_OK;
        const size_t nf = (size_t)nf_, nw = (size_t)nw_;
        sph_status s;
        for (int b = 0; b < 2; ++b) {
            if ((s = alloc(gx_[b], nf)) != SPH_OK) return s;
            if ((s = alloc(gv_[b], nf)) != SPH_OK) return s;
            if ((s = alloc(ga_[b], nf)) != SPH_OK) return s;
            if ((s = alloc(gpw_[b], nw)) != SPH_OK) return s;
        }
        if ((s = alloc(tA_, nf)) != SPH_OK) return s;
        if ((s = alloc(tX_, nf)) != SPH_OK) return s;
        if ((s = alloc(tV_, nf)) != SPH_OK) return s;
        if ((s = alloc(adj_inv_, nf)) != SPH_OK) return s;
        if ((s = alloc(wc_, nw)) != SPH_OK) return s;
        if ((s = alloc(adj_io_, 14 * nf + nw)) != SPH_OK) return s;
        SPH_CUDA(cudaStreamCreateWithFlags(&adj_side_, cudaStreamNonBlocking));
        for (cudaEvent_t& e : adj_ev_) SPH_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return alloc(adj_param_, 3);
    }

    sph_status prof_begin(int kind)
    {
        if (!((prof_mask_ >> kind) & 1u) || ev_used_ >= kMaxEvents) return SPH_OK;
        if (ev_used_ == ev_.size()) {
            EvPair e{nullptr, nullptr, 0};
            SPH_CUDA(cudaEventCreate(&e.a));
            SPH_CUDA(cudaEventCreate(&e.b));
            ev_.push_back(e);
        }
        ev_[ev_used_].kind = kind;
        SPH_CUDA(cudaEventRecord(ev_[ev_used_].a, stream));
        prof_open_ = true;
        return SPH_OK;
    }

    sph_status prof_end(int kind)
    {
        (void)kind;
        if (!prof_open_) return SPH_OK;
        SPH_CUDA(cudaEventRecord(ev_[ev_used_].b, stream));
        ++ev_used_;
        prof_open_ = false;
        return SPH_OK;
    }

    sph_params P_{};
    Cfg<T> C_{};
    Cfg<double> D_{};
    InitCfg I_{};
    int32_t nf_ = 0, nw_ = 0, n_cells_ = 0, dims_[3] = {1, 1, 1};
    double cs_ = 0.0;
    int par_ = 0;
    int64_t steps_ = 0;

    V4<T>* pos_[2] = {nullptr, nullptr};
    V4<T>* vel_[2] = {nullptr, nullptr};
    T* drho_[2] = {nullptr, nullptr};
    V4<T>* comp_[2] = {nullptr, nullptr};
    int4* cell_[2] = {nullptr, nullptr};
    int32_t* id_[2] = {nullptr, nullptr};
    int32_t* phase_[2] = {nullptr, nullptr};
    V4<T>* acc_ = nullptr;
    T* sigma_ = nullptr;  // sigma - sigma^0
    int32_t *nbf_ = nullptr, *nbw_ = nullptr;  // neighbour sub-lists (fluid, wall)
    int32_t* nbf_live_ = nullptr;  // the context's own list buffer (the tape may swap in others)
    bool lists_current_ = false;   // the own lists hold the build of the current state
    int32_t* ncnt_ = nullptr;                  // per-lane entry counts
    int32_t *wtag_ = nullptr, *d_tag_ = nullptr;  // wall support tags, current tag
    int32_t* wfront_ = nullptr;  // the adjoint's fluid-facing flags of the step it reverses
    cudaStream_t cap_stream_ = nullptr;
    // graphs keyed by (recompute without momentum, parity, reinit)
    cudaGraphExec_t gexec_[16] = {};
    int64_t glaunch_[16][SPH_NK] = {};
    bool sigma_valid_ = false;  // sigma_ holds sigma - sigma^0 of the current positions
    int4* newcell_ = nullptr;
    int32_t *rank_ = nullptr, *tmp_src_ = nullptr, *tmp_id_ = nullptr;
    int32_t *counts_ = nullptr, *fstart_ = nullptr, *wstart_ = nullptr, *sums_ = nullptr;
    uint16_t* wrows_ = nullptr;  // per cell: the stencil rows that hold wall particles
    V4<T>* wpos_ = nullptr;
    V4<T>* wpos_tmp_ = nullptr;
    V2<T>* wrho_ = nullptr;
    V4<T>* wnrm_ = nullptr;
    int4 *wcell_ = nullptr, *wcell_tmp_ = nullptr;
    int32_t *wid_ = nullptr, *wid_tmp_ = nullptr;
    T* d_dt_ = nullptr;
    T* d_dt_fixed_ = nullptr;
    unsigned long long* d_vmax_ = nullptr;
    double* d_time_ = nullptr;  // simulated time since create
    V4<T>* d_geff_ = nullptr;   // body force of the current step (g, or g + amp w^2 sin(w t))
    int32_t* d_flags_ = nullptr;
    unsigned long long* d_active_ = nullptr;
    double* diag_partial_ = nullptr;
    double* diag_out_ = nullptr;
    // adjoint: checkpoints (ck_[k] = state before taped step k), snapshot,
    // adjoint state (x, d), (v, sigma), a, p_w in two parities, step temporaries
    std::vector<Ckpt> ck_;
    std::vector<Fwd> fwd_;  // fwd_[k]: the products of taped step k (buf NULL: recomputed)
    cudaStream_t adj_side_ = nullptr;  // the backward's second stream and its fork/join events
    cudaEvent_t adj_ev_[2] = {nullptr, nullptr};
    size_t fwd_bytes_ = 0, fwd_budget_ = 0;  // bytes kept, and the budget (0: not yet set)
    int64_t fwd_limit_ = -1;                 // sph_tape_budget: -1 = half the free memory
    Ckpt snap_;
    int64_t ntaped_ = 0, tape_end_ = -1;
    V4<T>*gx_[2] = {nullptr, nullptr}, *gv_[2] = {nullptr, nullptr}, *ga_[2] = {nullptr, nullptr};
    T* gpw_[2] = {nullptr, nullptr};
    V4<T>*tA_ = nullptr, *tX_ = nullptr, *tV_ = nullptr;
    int32_t* adj_inv_ = nullptr;
    T* wc_ = nullptr;
    double* adj_io_ = nullptr;
    double* adj_param_ = nullptr;
    HostStatus* host_status_ = nullptr;
    bool dt_valid_ = false;  // d_dt_fixed_ holds host_status_->dt_fixed
    std::vector<void*> allocs_;
    uint32_t prof_mask_ = 0;
    bool prof_open_ = false;
    int64_t launches_[SPH_NK] = {0};
    std::vector<EvPair> ev_;
    size_t ev_used_ = 0;
};

}  // namespace sph
