// Kernels of one kick-drift-kick WCSPH step with the generalised wall
// boundary treatment (arXiv 2110.02621, Sec. 2 and Sec. 3).  Templated on the
// arithmetic type T (float: the production form, positions as cell index plus
// FP32 offset with Kahan-compensated drift; double: the plain FP64 form).
//
// Data layout (structure of arrays, fluid sorted by (cell key, id) each step):
//   pos  V4<T>  (ox, oy, oz, p)   offset inside the cell, pressure
//   vel  V4<T>  (vx, vy, vz, rho) velocity, density
//   drho T      rho - rho0        master copy of the density
//   acc  V4<T>  (ax, ay, az, drho/dt)
//   comp V4<T>  Kahan compensation of the drift (FP32 form only)
//   cell int4   (cx, cy, cz, key) key = (cz*ny + cy)*nx + cx or -1 outside
//   id, phase   int32
// Walls (static, sorted once): wpos (ox, oy, oz, p_w), wrho (rho_w per phase),
// wnrm (n_w, 0), wcell int4, wid int32.
#pragma once

#include "sph_device.cuh"

namespace sph {

template <class T>
__device__ __forceinline__ T bits_to(unsigned long long b);
template <>
__device__ __forceinline__ float bits_to<float>(unsigned long long b) { return __uint_as_float((unsigned)b); }
template <>
__device__ __forceinline__ double bits_to<double>(unsigned long long b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ unsigned long long to_bits(float x) { return (unsigned long long)__float_as_uint(x); }
__device__ __forceinline__ unsigned long long to_bits(double x) { return (unsigned long long)__double_as_longlong(x); }

template <class T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <class T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <class T>
__device__ __forceinline__ T tabs(T a) { return a < T(0) ? -a : a; }

// dt of the coming step (Sec. 2.6): the caller's fixed dt, or
// cfl min(h/(c0 + U_max), sqrt(h/|g|)) from the previous momentum sweep's U_max
template <class T>
__device__ __forceinline__ T step_dt(const Cfg<T>& C, const T* dt_fixed, const unsigned long long* vmax_bits)
{
    T dt = *dt_fixed;
    if (!(dt > T(0))) {
        const T umax = bits_to<T>(*vmax_bits);
        dt = C.cfl * C.h / (C.c0 + umax);
        if (C.body_dt > T(0)) dt = tmin(dt, C.body_dt);
    }
    return dt;
}

// --------------------------------------------------------------- step start
// Step start for a context without fluid (with fluid, k_predict and k_scatter
// do this): the step's dt, the wall-support tag, U_max and the per-cell
// counters of the coming re-binning.
template <class T>
__global__ void k_begin_step(Cfg<T> C, const T* __restrict__ dt_fixed, unsigned long long* vmax_bits,
                             T* d_dt, int32_t* counts, int32_t n_counts, int32_t* d_tag, double* d_time,
                             V4<T>* d_geff)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        *d_tag += 1;  // new wall-support tag for this step's neighbour build
        const T dt = step_dt(C, dt_fixed, vmax_bits);
        *d_dt = dt;
        *vmax_bits = 0ull;
        advance_time(C, dt, d_time, d_geff);
    }
    for (int k = t; k < n_counts; k += gridDim.x * blockDim.x) counts[k] = 0;
}

// Advance the simulated time by the step's dt and set the body force of
// t^{n+1} for the sweeps: in the frame of a tank moving as x = amp sin(w t)
// it is g - d2x/dt2 = g + amp w^2 sin(w t) (Sec. 4.2); g without motion.
template <class T>
__device__ __forceinline__ void advance_time(const Cfg<T>& C, T dt, double* d_time, V4<T>* d_geff)
{
    const double t = *d_time + (double)dt;
    *d_time = t;
    const double k = C.ex_w * C.ex_w * sin(C.ex_w * t);
    *d_geff = V4<T>{(T)(C.g64[0] + C.ex_amp[0] * k), (T)(C.g64[1] + C.ex_amp[1] * k),
                    (T)(C.g64[2] + C.ex_amp[2] * k), T(0)};
}

// half kick and drift of one particle, then move the offset back into its
// cell; shared by the counting and the moving kernels so both agree bitwise.
template <class T, bool KAHAN>
__device__ __forceinline__ void kick_drift(const Cfg<T>& C, T dt, V4<T>& p, V4<T>& v, const V4<T>& a,
                                           V4<T>& cm, int4& c)
{
    T hdt = T(0.5) * dt;
    v.x = fma_rn(hdt, a.x, v.x);
    v.y = fma_rn(hdt, a.y, v.y);
    v.z = fma_rn(hdt, a.z, v.z);
    drift1<T, KAHAN>(p.x, cm.x, dt, v.x);
    drift1<T, KAHAN>(p.y, cm.y, dt, v.y);
    drift1<T, KAHAN>(p.z, cm.z, dt, v.z);
    rebin1(p.x, c.x, C.cs);
    rebin1(p.y, c.y, C.cs);
    rebin1(p.z, c.z, C.cs);
    if (C.periodic) {  // a step moves a particle by less than one cell
        if (C.periodic & 1) c.x = wrap_cell(c.x, C.nx);
        if (C.periodic & 2) c.y = wrap_cell(c.y, C.ny);
        if (C.periodic & 4) c.z = wrap_cell(c.z, C.nz);
    }
}

// v^{n+1/2} = v^n + dt/2 a^n, r^{n+1} = r^n + dt v^{n+1/2} (Sec. 2.6), new cell
// and its occupancy count; bucket n_cells collects particles outside the grid.
// Every thread evaluates the step's dt; thread 0 publishes it for the later
// kernels, opens the step's wall-support tag and advances the time and the
// body force.  (U_max is cleared by the
// scatter that follows, once every thread here has read it.)
template <class T, bool KAHAN>
__global__ void k_predict(Cfg<T> C, int32_t n, const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel,
                          const V4<T>* __restrict__ acc, const V4<T>* __restrict__ comp,
                          const int4* __restrict__ cell, const T* __restrict__ dt_fixed,
                          const unsigned long long* __restrict__ vmax_bits, T* __restrict__ d_dt,
                          int32_t* __restrict__ d_tag, double* __restrict__ d_time, V4<T>* __restrict__ d_geff,
                          int4* __restrict__ newcell, int32_t* __restrict__ rank, int32_t* counts)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const T dt = step_dt(C, dt_fixed, vmax_bits);
    if (s == 0) {
        *d_dt = dt;
        *d_tag += 1;
        advance_time(C, dt, d_time, d_geff);
    }
    V4<T> p = pos[s], v = vel[s], a = acc[s], cm = comp[s];
    int4 c = cell[s];
    kick_drift<T, KAHAN>(C, dt, p, v, a, cm, c);
    uint32_t key = cell_key(C, c.x, c.y, c.z);
    int bucket = key == KEY_NONE ? C.n_cells : (int)key;
    // Consecutive particles mostly share a cell: the lanes of a warp with the
    // same bucket take one atomic (their leader adds their number) and each
    // its rank among them.  The arrival order is irrelevant: the gather
    // orders every cell by id.
    const unsigned peers = __match_any_sync(__activemask(), bucket);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counts + bucket, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    rank[s] = base + __popc(peers & ((1u << lane) - 1u));
    c.w = (int)key;
    newcell[s] = c;
}

// first placement: slot = start of the bucket + arrival rank.  In a step,
// thread 0 also clears U_max for the coming momentum sweep (vmax_reset).
static __global__ void k_scatter(int32_t n, int32_t n_cells, const int4* __restrict__ newcell,
                                 const int32_t* __restrict__ rank, const int32_t* __restrict__ start,
                                 const int32_t* __restrict__ id, int32_t* __restrict__ tmp_src,
                                 int32_t* __restrict__ tmp_id, unsigned long long* vmax_reset)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    if (s == 0 && vmax_reset) *vmax_reset = 0ull;
    int key = newcell[s].w;
    int t = SPH_CK(start[key < 0 ? n_cells : SPH_CK(key, n_cells, CK_CELL)] + rank[s], n, CK_SLOT);
    tmp_src[t] = s;
    tmp_id[t] = id[s];
}

// final slot inside the cell: rank of the particle's id among the ids of its
// cell, so the order is (key, id) whatever the arrival order was.
__device__ __forceinline__ int32_t sorted_slot(int32_t t, int32_t key, int32_t n_cells,
                                               const int32_t* __restrict__ start,
                                               const int32_t* __restrict__ tmp_id)
{
    if (key < 0) return t;  // outside the grid: order inside the bucket unspecified
    key = SPH_CK(key, n_cells, CK_CELL);
    int b = start[key], e = start[key + 1];
    int my = tmp_id[t], r = 0;
    for (int u = b; u < e; ++u) r += (tmp_id[u] < my);
    return b + r;
}

// Density reinitialisation, Eqs. (eqrhosum) / (eqrhosumnosurface), on the
// density excess d = rho* - rho0, given dsig = sigma - sigma^0:
//   rho_num - rho0 = rho0 dsig / sigma^0 =: dnum
//   free surface: rho = rho_num + max(0, rho* - rho_num) rho0/rho*, i.e.
//     d' = d - (d - dnum) d/rho*   if d > dnum,  d' = dnum otherwise
//     (the same value written without the cancellation of the printed form)
//   internal:     d' = dnum
template <class T>
__device__ __forceinline__ T reinit_drho(const PhaseK<T>& P, const Cfg<T>& C, T d, T dsig)
{
    const T dnum = P.rho0 * dsig * C.inv_sigma0;
    if (P.reinit == 1) return d > dnum ? d - (d - dnum) * (d / (P.rho0 + d)) : dnum;
    if (P.reinit == 2) return dnum;
    return d;
}

// Move every particle into its sorted slot, applying the half kick and drift
// (recomputed bitwise-identically) and, when due, the density
// reinitialisation with the number density of r^n (stored as
// sigma - sigma^0), followed by the EOS.
template <class T, bool KAHAN>
__global__ void k_gather(Cfg<T> C, int32_t n, const int32_t* __restrict__ start,
                         const int32_t* __restrict__ tmp_src, const int32_t* __restrict__ tmp_id,
                         const int4* __restrict__ newcell, const T* __restrict__ d_dt, int32_t reinit,
                         const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel,
                         const T* __restrict__ drho, const V4<T>* __restrict__ acc,
                         const V4<T>* __restrict__ comp, const T* __restrict__ sigma,
                         const int4* __restrict__ cell, const int32_t* __restrict__ phase,
                         V4<T>* __restrict__ pos_o, V4<T>* __restrict__ vel_o, T* __restrict__ drho_o,
                         V4<T>* __restrict__ comp_o, int4* __restrict__ cell_o,
                         int32_t* __restrict__ id_o, int32_t* __restrict__ phase_o)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int s = SPH_CK(tmp_src[t], n, CK_SLOT);
    int4 c = newcell[s];
    int dst = SPH_CK(sorted_slot(t, c.w, C.n_cells, start, tmp_id), n, CK_SLOT);
    T dt = *d_dt;
    V4<T> p = pos[s], v = vel[s], a = acc[s], cm = comp[s];
    int4 c_old = cell[s];
    int4 c_new = c_old;
    kick_drift<T, KAHAN>(C, dt, p, v, a, cm, c_new);
    int ph = phase[s];
    const PhaseK<T>& P = C.ph[ph];
    T d = drho[s];
    if (reinit && c_old.w >= 0) d = reinit_drho(P, C, d, sigma[s]);
    p.w = eos_p(P, C, d);
    v.w = P.rho0 + d;
    pos_o[dst] = p;
    vel_o[dst] = v;
    drho_o[dst] = d;
    comp_o[dst] = cm;
    cell_o[dst] = c;
    id_o[dst] = tmp_id[t];
    phase_o[dst] = ph;
}

// Density reinitialisation in place on the current (sorted) state, for the
// explicit sph_reinit_density call: same arithmetic as in k_gather.
template <class T>
__global__ void k_reinit(Cfg<T> C, int32_t n, const T* __restrict__ sigma, const int4* __restrict__ cell,
                         const int32_t* __restrict__ phase, V4<T>* __restrict__ pos,
                         V4<T>* __restrict__ vel, T* __restrict__ drho)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const PhaseK<T>& P = C.ph[phase[i]];
    if (cell[i].w < 0 || P.reinit == 0) return;
    const T d = reinit_drho(P, C, drho[i], sigma[i]);
    drho[i] = d;
    reinterpret_cast<T*>(pos + i)[3] = eos_p(P, C, d);
    reinterpret_cast<T*>(vel + i)[3] = P.rho0 + d;
}

}  // namespace sph
