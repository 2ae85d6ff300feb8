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

// --------------------------------------------------------------- step start
// Time step (Sec. 2.6): dt = cfl min(h/(c0 + U_max), sqrt(h/|g|)) from the
// U_max of the previous momentum sweep, unless a fixed dt > 0 is given.
// Also clears the per-cell counters of the coming re-binning.
template <class T>
__global__ void k_begin_step(Cfg<T> C, const T* __restrict__ dt_fixed, unsigned long long* vmax_bits,
                             T* d_dt, int32_t* counts, int32_t n_counts)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        T dt = *dt_fixed;
        if (!(dt > T(0))) {
            T umax = bits_to<T>(*vmax_bits);
            dt = C.cfl * C.h / (C.c0 + umax);
            if (C.body_dt > T(0)) dt = tmin(dt, C.body_dt);
        }
        *d_dt = dt;
        *vmax_bits = 0ull;
    }
    for (int k = t; k < n_counts; k += gridDim.x * blockDim.x) counts[k] = 0;
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
}

// v^{n+1/2} = v^n + dt/2 a^n, r^{n+1} = r^n + dt v^{n+1/2} (Sec. 2.6), new cell
// and its occupancy count; bucket n_cells collects particles outside the grid.
template <class T, bool KAHAN>
__global__ void k_predict(Cfg<T> C, int32_t n, const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel,
                          const V4<T>* __restrict__ acc, const V4<T>* __restrict__ comp,
                          const int4* __restrict__ cell, const T* __restrict__ d_dt,
                          int4* __restrict__ newcell, int32_t* __restrict__ rank, int32_t* counts)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    T dt = *d_dt;
    V4<T> p = pos[s], v = vel[s], a = acc[s], cm = comp[s];
    int4 c = cell[s];
    kick_drift<T, KAHAN>(C, dt, p, v, a, cm, c);
    uint32_t key = cell_key(C, c.x, c.y, c.z);
    int bucket = key == KEY_NONE ? C.n_cells : (int)key;
    rank[s] = atomicAdd(counts + bucket, 1);
    c.w = (int)key;
    newcell[s] = c;
}

// first placement: slot = start of the bucket + arrival rank.
static __global__ void k_scatter(int32_t n, int32_t n_cells, const int4* __restrict__ newcell,
                                 const int32_t* __restrict__ rank, const int32_t* __restrict__ start,
                                 const int32_t* __restrict__ id, int32_t* __restrict__ tmp_src,
                                 int32_t* __restrict__ tmp_id)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int key = newcell[s].w;
    int t = start[key < 0 ? n_cells : key] + rank[s];
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
    int b = start[key], e = start[key + 1];
    int my = tmp_id[t], r = 0;
    for (int u = b; u < e; ++u) r += (tmp_id[u] < my);
    return b + r;
}

// Move every particle into its sorted slot, applying the half kick and drift
// (recomputed bitwise-identically) and, when due, the density
// reinitialisation of Eqs. (eqrhosum) / (eqrhosumnosurface) with the number
// density sigma of r^n, followed by the EOS.
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
    int s = tmp_src[t];
    int4 c = newcell[s];
    int dst = sorted_slot(t, c.w, C.n_cells, start, tmp_id);
    T dt = *d_dt;
    V4<T> p = pos[s], v = vel[s], a = acc[s], cm = comp[s];
    int4 c_old = cell[s];
    int4 c_new = c_old;
    kick_drift<T, KAHAN>(C, dt, p, v, a, cm, c_new);
    int ph = phase[s];
    const PhaseK<T>& P = C.ph[ph];
    T d = drho[s];
    if (reinit && c_old.w >= 0 && P.reinit != 0) {
        T dnum = P.rho0 * (sigma[s] * C.inv_sigma0 - T(1));   // rho0 sigma/sigma0 - rho0
        if (P.reinit == 1) {
            T rho_star = P.rho0 + d;
            d = dnum + tmax(T(0), d - dnum) * P.rho0 / rho_star;
        } else {
            d = dnum;
        }
    }
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
    T d = drho[i];
    T dnum = P.rho0 * (sigma[i] * C.inv_sigma0 - T(1));
    if (P.reinit == 1) {
        T rho_star = P.rho0 + d;
        d = dnum + tmax(T(0), d - dnum) * P.rho0 / rho_star;
    } else {
        d = dnum;
    }
    drho[i] = d;
    reinterpret_cast<T*>(pos + i)[3] = eos_p(P, C, d);
    reinterpret_cast<T*>(vel + i)[3] = P.rho0 + d;
}

// ------------------------------------------------------------- continuity
// Heavy (continuity) phases: Eq. (SPH_star_massConservation) with the
// Riemann solution of Eq. (RSsolution).  Substituting v* gives, per pair,
//   (v_i - v*).grad_i W_ij (m_j/rho_j) = m_j F [v_ij.r_ij + (p_i - p_j) r/(c rho_j)]/(rho_i + rho_j)
// with grad_i W_ij = F r_ij; walls enter with v_w = 0, (rho_w, p_w), m_w = m_i.
// Then rho^{n+1} = rho^n + dt d rho/dt (Sec. 2.6).
// Light (summation) phases: Eq. (densitySummation), rho = m sum_j W_ij over all
// particles and walls, self included.  The EOS gives p^{n+1}.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_continuity(
    Cfg<T> C, int32_t n, const int32_t* __restrict__ fstart, const int32_t* __restrict__ wstart,
    const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel, const T* __restrict__ drho,
    const int4* __restrict__ cell, const int32_t* __restrict__ phase,
    const V4<T>* __restrict__ wpos, const V2<T>* __restrict__ wrho, const T* __restrict__ d_dt,
    V4<T>* __restrict__ pos_o, V4<T>* __restrict__ vel_o, T* __restrict__ drho_o,
    V4<T>* __restrict__ acc_o)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V4<T> pi = pos[i], vi = vel[i];
    int4 c = cell[i];
    T d = drho[i];
    if (c.w < 0) {
        pos_o[i] = pi;
        vel_o[i] = vi;
        drho_o[i] = d;
        acc_o[i] = V4<T>{T(0), T(0), T(0), T(0)};
        return;
    }
    const int ph = phase[i];
    const PhaseK<T>& P = C.ph[ph];
    const T rho_i = vi.w, p_i = pi.w;
    T drdt = T(0);
    if (P.density == 1) {
        T sig = C.W0;
        for_cells27(C, c.x, c.y, c.z, fstart, [&](int j, T sx, T sy, T sz) {
            V4<T> pj = pos[j];
            T rx = pi.x - pj.x - sx, ry = pi.y - pj.y - sy, rz = pi.z - pj.z - sz;
            T r2 = rx * rx + ry * ry + rz * rz;
            if (r2 >= C.rc2 || r2 == T(0)) return;
            sig += kernel_W(C, f_sqrt(r2));
        });
        for_cells27(C, c.x, c.y, c.z, wstart, [&](int w, T sx, T sy, T sz) {
            V4<T> pw = wpos[w];
            T rx = pi.x - pw.x - sx, ry = pi.y - pw.y - sy, rz = pi.z - pw.z - sz;
            T r2 = rx * rx + ry * ry + rz * rz;
            if (r2 >= C.rc2 || r2 == T(0)) return;
            sig += kernel_W(C, f_sqrt(r2));
        });
        d = P.rho0 * (C.dp3 * sig - T(1));
    } else {
        T s = T(0);
        const bool multi = C.n_phases > 1;
        for_cells27(C, c.x, c.y, c.z, fstart, [&](int j, T sx, T sy, T sz) {
            V4<T> pj = pos[j];
            T rx = pi.x - pj.x - sx, ry = pi.y - pj.y - sy, rz = pi.z - pj.z - sz;
            T r2 = rx * rx + ry * ry + rz * rz;
            if (r2 >= C.rc2 || r2 == T(0)) return;
            V4<T> vj = vel[j];
            T r = f_sqrt(r2);
            T F = kernel_F(C, r);
            T m_j = multi ? C.ph[phase[j]].m : P.m;
            T rv = rx * (vi.x - vj.x) + ry * (vi.y - vj.y) + rz * (vi.z - vj.z);
            s += m_j * F * (rv + (p_i - pj.w) * r * C.inv_c0 / vj.w) / (rho_i + vj.w);
        });
        for_cells27(C, c.x, c.y, c.z, wstart, [&](int w, T sx, T sy, T sz) {
            V4<T> pw = wpos[w];
            T rx = pi.x - pw.x - sx, ry = pi.y - pw.y - sy, rz = pi.z - pw.z - sz;
            T r2 = rx * rx + ry * ry + rz * rz;
            if (r2 >= C.rc2 || r2 == T(0)) return;
            T r = f_sqrt(r2);
            T F = kernel_F(C, r);
            V2<T> rw = wrho[w];
            T rho_w = ph == 0 ? rw.x : rw.y;
            T rv = rx * vi.x + ry * vi.y + rz * vi.z;
            s += P.m * F * (rv + (p_i - pw.w) * r * C.inv_c0 / rho_w) / (rho_i + rho_w);
        });
        drdt = T(2) * rho_i * s;
        d = d + (*d_dt) * drdt;
    }
    pos_o[i] = V4<T>{pi.x, pi.y, pi.z, eos_p(P, C, d)};
    vel_o[i] = V4<T>{vi.x, vi.y, vi.z, P.rho0 + d};
    drho_o[i] = d;
    acc_o[i] = V4<T>{T(0), T(0), T(0), drdt};
}

// ----------------------------------------------------------- wall pressure
// Eq. (wallPressure) with fixed walls (a_w = 0), reading the (g - a_w) term
// with the fluid density (dimensionally consistent form):
//   p_w = sum_f (p_f + rho_f g.r_wf) w_wf / sum_f w_wf,  r_wf = r_w - r_f,
// w = W (one phase) or W/rho_f (several phases, Sec. 2.3).  Walls without
// fluid support get p_w = 0.  rho_w = rho0 + EOS^-1(p_w) per phase.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_wall_pressure(
    Cfg<T> C, int32_t nw, const int32_t* __restrict__ fstart, V4<T>* __restrict__ wpos,
    const int4* __restrict__ wcell, const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel,
    V2<T>* __restrict__ wrho, unsigned long long* active)
{
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    int has = 0;
    if (w < nw) {
        int4 c = wcell[w];
        V4<T> pw = wpos[w];
        T num = T(0), den = T(0);
        const bool multi = C.n_phases > 1;
        if (c.w >= 0) {
            for_cells27(C, c.x, c.y, c.z, fstart, [&](int j, T sx, T sy, T sz) {
                V4<T> pf = pos[j];
                T rx = pw.x - pf.x - sx, ry = pw.y - pf.y - sy, rz = pw.z - pf.z - sz;
                T r2 = rx * rx + ry * ry + rz * rz;
                if (r2 >= C.rc2 || r2 == T(0)) return;
                T W = kernel_W(C, f_sqrt(r2));
                T rho_f = vel[j].w;
                T om = multi ? W / rho_f : W;
                num += (pf.w + rho_f * (C.gx * rx + C.gy * ry + C.gz * rz)) * om;
                den += om;
            });
        }
        T p_w = den > T(0) ? num / den : T(0);
        has = den > T(0);
        reinterpret_cast<T*>(wpos + w)[3] = p_w;
        T r0 = C.ph[0].rho0 + eos_drho(C.ph[0], C, p_w);
        T r1 = multi ? C.ph[1].rho0 + eos_drho(C.ph[1], C, p_w) : r0;
        wrho[w] = V2<T>{r0, r1};
    }
    int cnt = __syncthreads_count(has);
    if (threadIdx.x == 0 && cnt) atomicAdd(active, (unsigned long long)cnt);
}

// --------------------------------------------------------------- momentum
// Eq. (SPH_star_momentumConservation) with p* from Eq. (RSsolution) (fluid)
// or Eq. (RSatWall) (wall); per pair -2 m_j p*/(rho_i rho_j) F r_ij, where
//   p*/(rho_i rho_j) = (p_i/rho_i + p_j/rho_j + beta dU)/(rho_i + rho_j),
//   dU = U_L - U_R = -v_ij.r_ij/r, beta = min(3 max(dU, 0), c).
// Plus gravity, the Morris viscous term, and the penalty force of
// Eq. (SPH_penaltyMethodTerm) with delta = 2|r_iw.n_w|/dx, lambda from
// Eq. (symbc) and dx^3 restoring its units.  Then the final kick
// v^{n+1} = v^{n+1/2} + dt/2 a^{n+1}, the number density sigma(r^{n+1})
// for the next reinitialisation, and U_max for the next dt.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_momentum(
    Cfg<T> C, int32_t n, const int32_t* __restrict__ fstart, const int32_t* __restrict__ wstart,
    const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel, const int4* __restrict__ cell,
    const int32_t* __restrict__ phase, const V4<T>* __restrict__ wpos, const V2<T>* __restrict__ wrho,
    const V4<T>* __restrict__ wnrm, const T* __restrict__ d_dt, V4<T>* __restrict__ acc,
    V4<T>* __restrict__ vel_o, T* __restrict__ sigma_o, unsigned long long* vmax_bits, int32_t* flags)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    T speed = T(0);
    bool bad = false;
    if (i < n) {
        V4<T> pi = pos[i], vi = vel[i];
        int4 c = cell[i];
        T drdt = acc[i].w;
        T hdt = T(0.5) * (*d_dt);
        if (c.w < 0) {
            acc[i] = V4<T>{T(0), T(0), T(0), drdt};
            vel_o[i] = vi;
            sigma_o[i] = T(0);
        } else {
            const int ph = phase[i];
            const PhaseK<T>& P = C.ph[ph];
            const bool multi = C.n_phases > 1;
            const bool sig_all = P.density == 1;
            const T rho_i = vi.w, p_i = pi.w, pr_i = p_i / rho_i, mu_i = P.mu;
            T ax = T(0), ay = T(0), az = T(0), sig = C.W0;
            for_cells27(C, c.x, c.y, c.z, fstart, [&](int j, T sx, T sy, T sz) {
                V4<T> pj = pos[j];
                T rx = pi.x - pj.x - sx, ry = pi.y - pj.y - sy, rz = pi.z - pj.z - sz;
                T r2 = rx * rx + ry * ry + rz * rz;
                if (r2 >= C.rc2 || r2 == T(0)) return;
                V4<T> vj = vel[j];
                T r = f_sqrt(r2), W, F;
                kernel_WF(C, r, W, F);
                int phj = multi ? phase[j] : 0;
                const PhaseK<T>& Pj = C.ph[phj];
                T vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                T dU = -(rx * vx + ry * vy + rz * vz) / r;
                T beta = tmin(T(3) * tmax(dU, T(0)), C.c0);
                T coef = (pr_i + pj.w / vj.w + beta * dU) / (rho_i + vj.w);
                T k = T(-2) * Pj.m * F * coef;
                T mu = mu_i + Pj.mu;
                if (mu > T(0)) {
                    T kv = Pj.m * mu * r2 * F / (rho_i * vj.w * (r2 + C.eta2));
                    ax += kv * vx; ay += kv * vy; az += kv * vz;
                }
                ax += k * rx; ay += k * ry; az += k * rz;
                if (sig_all || phj == ph) sig += W;
            });
            for_cells27(C, c.x, c.y, c.z, wstart, [&](int w, T sx, T sy, T sz) {
                V4<T> pw = wpos[w];
                T rx = pi.x - pw.x - sx, ry = pi.y - pw.y - sy, rz = pi.z - pw.z - sz;
                T r2 = rx * rx + ry * ry + rz * rz;
                if (r2 >= C.rc2 || r2 == T(0)) return;
                T r = f_sqrt(r2), W, F;
                kernel_WF(C, r, W, F);
                V2<T> rw = wrho[w];
                T rho_w = ph == 0 ? rw.x : rw.y;
                T coef = (pr_i + pw.w / rho_w) / (rho_i + rho_w);
                T k = T(-2) * P.m * F * coef;
                ax += k * rx; ay += k * ry; az += k * rz;
                if (mu_i > T(0)) {
                    T kv = P.m * (T(2) * mu_i) * r2 * F / (rho_i * rho_w * (r2 + C.eta2));
                    ax += kv * vi.x; ay += kv * vi.y; az += kv * vi.z;
                }
                if (P.penalty && r > C.pen_rmin) {
                    V4<T> nw = wnrm[w];
                    T rn = rx * nw.x + ry * nw.y + rz * nw.z;   // r_iw . n_w
                    T delta = T(2) * tabs(rn) * C.inv_dp;
                    if (delta < T(1)) {
                        T en = -rn / r;                          // e_iw . n_w
                        T lam = (T(1) - delta) * (T(1) - delta) * C.inv_dp;
                        T Ppen = C.gamma_p * lam * tabs(p_i * en);
                        T kp = T(-2) * P.m / (rho_i * rho_w) * Ppen * C.dp3 * F / r;
                        ax += kp * nw.x; ay += kp * nw.y; az += kp * nw.z;
                    }
                }
                sig += W;
            });
            ax += C.gx; ay += C.gy; az += C.gz;
            V4<T> vo{fma_rn(hdt, ax, vi.x), fma_rn(hdt, ay, vi.y), fma_rn(hdt, az, vi.z), rho_i};
            bad = !(f_finite(ax) && f_finite(ay) && f_finite(az));
            acc[i] = V4<T>{ax, ay, az, drdt};
            vel_o[i] = vo;
            sigma_o[i] = sig;
            speed = f_sqrt(vo.x * vo.x + vo.y * vo.y + vo.z * vo.z);
        }
    }
    // block maximum of |v| (non-negative: integer order of the bits is the
    // order of the values), one atomic per block
    __shared__ unsigned long long smax[BLOCK / 32];
    unsigned long long b = to_bits(speed);
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long q = __shfl_xor_sync(0xffffffffu, b, o);
        b = q > b ? q : b;
    }
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = b;
    int nbad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int k = 0; k < BLOCK / 32; ++k) m = smax[k] > m ? smax[k] : m;
        atomicMax(vmax_bits, m);
        if (nbad) atomicOr(flags, 1);
    }
}

}  // namespace sph
