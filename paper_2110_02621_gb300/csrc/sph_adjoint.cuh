// Backward (vector-Jacobian product) of one kick-drift-kick step, with the
// neighbour sets of the forward step frozen and the time step a constant of
// the run.  One phase with continuity density (Sec. 2.2), fixed walls with the
// extrapolated pressure of Eq. (wallPressure), the wall Riemann pressure of
// Eq. (RSatWall), the penalty force of Eq. (SPH_penaltyMethodTerm) and the
// Morris viscosity; the free-surface reinitialisation of Eq. (eqrhosum).
//
// Forward step n in the notation used below (new sorted order after the
// re-binning; d = rho - rho0 is the density state, p = EOS(d)):
//   d~  = R(d, sigma - sigma0) if reinitialised, else d;  p~ = EOS(d~)
//   v'' = v + dt/2 a;  x' = x + dt v''
//   D_i = sum_j e_ij(x', v'', d~, p~) + sum_w e_iw(x', v'', d~, p~; p_w^n, rho_w^n)
//   d'  = d~ + dt D;   p' = EOS(d')
//   p_w' = sum_f (p'_f + rho'_f g.r_wf) W_wf / sum_f W_wf,  rho_w' = rho0 + EOS^-1(p_w')
//   a'  = sum_j T_ij + sum_w T_iw + g   (pressure, limiter, viscosity, penalty)
//   v'  = v'' + dt/2 a';  sigma' = W(0) + sum_j W_ij + sum_w W_iw
// The adjoint state carried between steps is (x, d), (v, sigma), a per fluid
// particle and p_w per wall, in the sorted order of the state it belongs to.
//
// Kernels of one backward step (after the forward step is recomputed from its
// checkpoint):
//   k_adj_inverse       old sorted slot of every particle id
//   k_adj_prep          A_i = a_bar'_i + dt/2 v_bar'_i  (adjoint of a' in total)
//   k_adj_wall_momentum per wall: p_w' and rho_w' adjoints of the momentum
//                       pairs, plus the incoming adjoint, divided by sum W
//   k_adj_momentum      per fluid: momentum, sigma' and wall-pressure
//                       extrapolation adjoints; the adjoint of d' and D
//   k_adj_continuity    per fluid: continuity adjoints (each pair term e_ij
//                       and e_ji seen from i), the kicks, drift and
//                       reinitialisation, written in the old order
//   k_adj_wall_continuity per wall: adjoint of the previous wall pressure
// Every kernel gathers (no atomics on state); the FP64 parameter gradients
// (c0, gamma_p, mu) are block sums added atomically.  Pair terms of a
// fluid-fluid pair are visited by both of its particles, so their parameter
// derivatives are halved.
#pragma once

#include "sph_sweeps.cuh"

namespace sph {

// dF/dr of the Wendland C2 kernel: 15 alpha (1 - q/2)^2 / (2 h^3)
template <class T>
__device__ __forceinline__ T kernel_dF(const Cfg<T>& C, T r)
{
    const T t = T(1) - T(0.5) * (r * C.inv_h);
    return T(-1.5) * C.fcoef * t * t * C.inv_h;
}

// dp/dd of the equation of state at (d, p = EOS(d)); dp/dc0 = 2 p / c0
template <class T>
__device__ __forceinline__ T eos_dp_dd(const PhaseK<T>& P, const Cfg<T>& C, T d, T p)
{
    const T c2 = C.c0 * C.c0;
    if (P.eos == 1) return c2 * (T(1) + p / P.eos_k) / (T(1) + d * P.inv_rho0);
    return c2;
}

template <class T>
__device__ __forceinline__ T sgn(T x) { return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0)); }

// block sum of three FP64 values added to out[0..2]; every thread of the
// block calls it
__device__ __forceinline__ void block_add3(double* out, double a, double b, double c)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    __shared__ double sm[3][LBLOCK / 32];
    if ((threadIdx.x & 31) == 0) {
        sm[0][threadIdx.x >> 5] = a;
        sm[1][threadIdx.x >> 5] = b;
        sm[2][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            s0 += sm[0][k];
            s1 += sm[1][k];
            s2 += sm[2][k];
        }
        if (s0 != 0.0) atomicAdd(out, s0);
        if (s1 != 0.0) atomicAdd(out + 1, s1);
        if (s2 != 0.0) atomicAdd(out + 2, s2);
    }
}

// ------------------------------------------------------------ pair adjoints
// Fluid-wall momentum pair i-w, a_i += T_iw with
//   T_iw = K r + V v_i + kp n_w,  K = -2 m F (pi_i + pi_w)/(rho_i + rho_w),
//   V = 2 mu_i m r^2 F / (rho_i rho_w (r^2 + eta^2)),
//   kp = -2 m dx^3 / (rho_i rho_w) P F / r,  P = gamma_p lambda |p_i e.n|
// (Eq. (RSatWall), Eq. (SPH_penaltyMethodTerm); delta = 2 r.n_w/dx signed,
// the penalty only through a fluid-facing wall particle, facing), plus
// sigma' += W.
// Given g = adjoint of a_i and sb = adjoint of sigma'_i, returns the
// adjoints of r = x_i - x_w, v_i, p_i, rho_i, p_w, rho_w, mu and gamma_p.
template <class T>
struct WallMomAdj {
    T rx, ry, rz, vx, vy, vz, p_i, rho_i, p_w, rho_w, mu, gp;
};

template <class T>
__device__ __forceinline__ void wall_momentum_adj(const Cfg<T>& C, const PhaseK<T>& P, T rx, T ry, T rz, T r2,
                                                  T vx, T vy, T vz, T rho_i, T p_i, T rho_w, T p_w,
                                                  const V4<T>& nw, bool facing, T gx, T gy, T gz, T sb,
                                                  WallMomAdj<T>& o)
{
    const T rinv = p_rsqrt(r2);
    const T R = r2 * rinv;
    T W, F;
    kernel_WF(C, R, W, F);
    const T Fp = kernel_dF(C, R);
    const T m = P.m;
    const T rs = rho_i + rho_w;
    const T pi_i = p_div(p_i, rho_i), pi_w = p_div(p_w, rho_w);
    const T Cc = p_div(pi_i + pi_w, rs);
    const T K = T(-2) * m * F * Cc;
    const T e2 = r2 + C.eta2;
    const T Q = p_div(r2 * F, e2);
    const T dQ = p_div(T(2) * R * F * C.eta2 + r2 * Fp * e2, e2 * e2);
    const T mv = p_div(m, rho_i * rho_w);
    const T mu2 = T(2) * P.mu;
    const T V = mu2 * mv * Q;
    const T Kb = gx * rx + gy * ry + gz * rz;
    const T Vb = gx * vx + gy * vy + gz * vz;
    T Fb = Kb * (T(-2) * m * Cc);
    const T Cb = Kb * (T(-2) * m * F);
    const T pib = p_div(Cb, rs);
    const T rsb = -pib * Cc;
    T Rb = Vb * mu2 * mv * dQ + sb * F * R;
    o.rx = K * gx;
    o.ry = K * gy;
    o.rz = K * gz;
    o.vx = V * gx;
    o.vy = V * gy;
    o.vz = V * gz;
    o.p_i = p_div(pib, rho_i);
    o.rho_i = -pib * p_div(pi_i, rho_i) + rsb - p_div(Vb * V, rho_i);
    o.p_w = p_div(pib, rho_w);
    o.rho_w = -pib * p_div(pi_w, rho_w) + rsb - p_div(Vb * V, rho_w);
    o.mu = Vb * T(2) * mv * Q;
    o.gp = T(0);
    if (P.penalty && R > C.pen_rmin && facing) {
        const T rn = rx * nw.x + ry * nw.y + rz * nw.z;
        const T delta = T(2) * rn * C.inv_dp;
        if (delta < T(1)) {
            const T en = -rn * rinv;
            const T om = T(1) - delta;
            const T lam = om * om * C.inv_dp;
            const T ape = tabs(p_i * en);
            const T Ppen = C.gamma_p * lam * ape;
            const T Ap = T(-2) * mv * C.dp3;
            const T kp = Ap * Ppen * F * rinv;
            const T kb = gx * nw.x + gy * nw.y + gz * nw.z;
            Fb += kb * Ap * Ppen * rinv;
            Rb -= kb * Ap * Ppen * F * rinv * rinv;
            const T Pb = kb * Ap * F * rinv;
            o.gp = Pb * lam * ape;
            const T s = sgn(p_i * en);
            o.p_i += Pb * C.gamma_p * lam * s * en;
            const T enb = Pb * C.gamma_p * lam * s * p_i;
            const T lamb = Pb * C.gamma_p * ape;
            const T deltab = lamb * (T(-2) * om * C.inv_dp);
            const T rnb = deltab * T(2) * C.inv_dp - enb * rinv;
            Rb += enb * rn * rinv * rinv;
            o.rx += rnb * nw.x;
            o.ry += rnb * nw.y;
            o.rz += rnb * nw.z;
            o.rho_i -= p_div(kb * kp, rho_i);
            o.rho_w -= p_div(kb * kp, rho_w);
        }
    }
    Rb += Fb * Fp;
    o.rx += Rb * rx * rinv;
    o.ry += Rb * ry * rinv;
    o.rz += Rb * rz * rinv;
}

// Continuity pair term of a wall, e_iw = 2 m F rho_i B / (rho_i + rho_w),
// B = r.v_i + (p_i - p_w) r / (c0 rho_w)  (Eq. (SPH_star_massConservation)
// with the Riemann solution, v_w = 0), times Db = adjoint of D_i: adjoints of
// r = x_i - x_w, v_i, p_i, rho_i, p_w, rho_w and c0.
template <class T>
struct WallContAdj {
    T rx, ry, rz, vx, vy, vz, p_i, rho_i, p_w, rho_w, c0;
};

template <class T>
__device__ __forceinline__ void wall_continuity_adj(const Cfg<T>& C, const PhaseK<T>& P, T rx, T ry, T rz, T r2,
                                                    T vx, T vy, T vz, T rho_i, T p_i, T rho_w, T p_w, T Db,
                                                    WallContAdj<T>& o)
{
    const T rinv = p_rsqrt(r2);
    const T R = r2 * rinv;
    const T F = kernel_F(C, R);
    const T Fp = kernel_dF(C, R);
    const T k = C.inv_c0;
    const T rs = rho_i + rho_w;
    const T A = p_div(T(2) * P.m, rs);
    const T dpw = p_i - p_w;
    const T S = rx * vx + ry * vy + rz * vz;
    const T B = S + p_div(dpw * R * k, rho_w);
    const T e = A * F * rho_i * B;
    const T DA = Db * A * rho_i;
    const T cr = Fp * B * rinv + F * p_div(dpw * k, rho_w) * rinv;
    o.rx = DA * (cr * rx + F * vx);
    o.ry = DA * (cr * ry + F * vy);
    o.rz = DA * (cr * rz + F * vz);
    o.vx = DA * F * rx;
    o.vy = DA * F * ry;
    o.vz = DA * F * rz;
    o.p_i = DA * F * p_div(R * k, rho_w);
    o.rho_i = Db * (A * F * B - p_div(e, rs));
    o.p_w = -o.p_i;
    o.rho_w = Db * (-A * F * rho_i * p_div(dpw * R * k, rho_w * rho_w) - p_div(e, rs));
    o.c0 = -DA * F * p_div(dpw * R * k * k, rho_w);
}

// ------------------------------------------------------------ kernels
// old sorted slot of every particle id (ids are 0..n-1)
static __global__ void k_adj_inverse(int32_t n, const int32_t* __restrict__ id_old, int32_t* __restrict__ inv)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) inv[SPH_CK(id_old[s], n, CK_SLOT)] = s;
}

// A = adjoint of a' in total (a' enters a'-state and the final kick)
template <class T>
__global__ void k_adj_prep(int32_t n, T hdt, const V4<T>* __restrict__ gv, const V4<T>* __restrict__ ga,
                           V4<T>* __restrict__ tA)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const V4<T> v = gv[i], a = ga[i];
    tA[i] = V4<T>{a.x + hdt * v.x, a.y + hdt * v.y, a.z + hdt * v.z, v.w};
}

// Per wall with fluid support in this step: the adjoints of p_w' and
// rho_w' from the fluid's momentum pairs, folded with rho_w' = rho0 +
// EOS^-1(p_w') and the incoming adjoint of p_w', then divided by sum_f W_wf
// for the extrapolation's backward.  wc = 0 for walls without support
// (their p_w' = 0 is a constant).
template <class T, bool PER>
__global__ void __launch_bounds__(LBLOCK) k_adj_wall_momentum(
    Cfg<T> C, int32_t nw, const int32_t* __restrict__ fstart, const V4<T>* __restrict__ wpos,
    const V2<T>* __restrict__ wrho, const V4<T>* __restrict__ wnrm, const int4* __restrict__ wcell,
    const int32_t* __restrict__ wtag, const int32_t* __restrict__ d_tag, const V4<T>* __restrict__ pos,
    const V4<T>* __restrict__ vel, const V4<T>* __restrict__ tA, const T* __restrict__ gpw_in,
    T* __restrict__ wc, double* gparam, int32_t* __restrict__ wfront)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = t / AWLP;
    double gc0 = 0.0;
    if (w < nw) {
        const PhaseK<T>& P = C.ph[0];
        T Gp = T(0), Gr = T(0), den = T(0);
        const bool live = wtag[w] == *d_tag;
        const V4<T> pw = wpos[w];
        const T rho_w = wrho[w].x;
        bool facing = false;
        if (live) {
            const V4<T> nn = wnrm[w];
            const int4 c = wcell[w];
            // the forward's fluid-facing flag, from the same scan of the same
            // positions (k_wall_pressure), for this kernel and for the fluid side
            scan_compact<PER, AWLP>(C, c, pw, fstart, pos, t % AWLP, [&](int, T rx, T ry, T rz, T, int) {
                facing |= rx * nn.x + ry * nn.y + rz * nn.z < T(0);
            });
            facing = (__ballot_sync(group_mask<AWLP>(), facing) & group_mask<AWLP>()) != 0u;
            scan_compact<PER, AWLP>(C, c, pw, fstart, pos, t % AWLP, [&](int j, T rx, T ry, T rz, T r2, int) {
                // scan vector is x_w - x_f; the pair vector of the fluid is x_f - x_w
                const V4<T> pf = pos[j], vf = vel[j], Aj = tA[j];
                WallMomAdj<T> o;
                wall_momentum_adj(C, P, -rx, -ry, -rz, r2, vf.x, vf.y, vf.z, vf.w, pf.w, rho_w, pw.w, nn, facing,
                                  Aj.x, Aj.y, Aj.z, T(0), o);
                Gp += o.p_w;
                Gr += o.rho_w;
                den += kernel_W(C, r2 * p_rsqrt(r2));
            });
            Gp = group_sum<AWLP>(Gp);
            Gr = group_sum<AWLP>(Gr);
            den = group_sum<AWLP>(den);
        }
        if (t % AWLP == 0) {
            T out = T(0);
            if (live && den > T(0)) {
                const T dw = rho_w - P.rho0;
                // rho_w held at rho0/2 below p_half does not move with p_w or c0
                const T dd_dp = pw.w < P.p_half ? T(0) : T(1) / eos_dp_dd(P, C, dw, pw.w);
                const T pbar = gpw_in[w] + Gp + Gr * dd_dp;
                gc0 = (double)(Gr * (T(-2) * pw.w * C.inv_c0 * dd_dp));
                out = pbar / den;
            }
            wc[w] = out;
            wfront[w] = facing;
        }
    }
    block_add3(gparam, gc0, 0.0, 0.0);
}

// Per fluid particle: backward of the momentum sweep (fluid and wall pairs,
// sigma'), of the wall-pressure extrapolation (through wc) and of
// p' = EOS(d'), rho' = rho0 + d'.  Regular mode writes the partial adjoint of
// x' and D = dt * (adjoint of d') into tX, the partial adjoint of v'' (v_bar'
// included) and the adjoint of d' into tV.  Create mode (the sweeps of
// sph_create at r^0, no kick) writes the final adjoints of x^0 and d^0 into
// tX and of v^0 into tV.
// FP32: seven blocks per SM (at most 72 registers; the compiler's free choice
// is 96, five blocks): a small spill costs less than the latency the extra
// warps hide (185 against 209 us per step at 189 k fluid particles, one
// GB300).  The FP64 form keeps the 166 registers it takes unbounded (capped,
// it would spill kilobytes).
template <class T, bool PER>
__global__ void __launch_bounds__(LBLOCK, sizeof(T) == 4 ? 7 : 3) k_adj_momentum(
    Cfg<T> C, int32_t n, T dt, int32_t create, const int32_t* __restrict__ fstart,
    const int32_t* __restrict__ wstart, const int32_t* __restrict__ nbf, const int32_t* __restrict__ nbw,
    const int32_t* __restrict__ cnt, const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel,
    const T* __restrict__ drho, const int4* __restrict__ cell, const V4<T>* __restrict__ wpos,
    const V2<T>* __restrict__ wrho, const V4<T>* __restrict__ wnrm, const T* __restrict__ wc,
    const V4<T>* __restrict__ tA, const V4<T>* __restrict__ gx_in, const V4<T>* __restrict__ gv_in,
    const V4<T>* __restrict__ geff, V4<T>* __restrict__ tX, V4<T>* __restrict__ tV, double* gparam,
    const int32_t* __restrict__ wfront)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / LP;
    const bool lead = (t % LP) == 0;
    double gc0 = 0.0, ggp = 0.0, gmu = 0.0;
    if (i < n) {
        const PhaseK<T>& P = C.ph[0];
        const V4<T> pi = pos[i], vi = vel[i], Ai = tA[i], ge = *geff;
        const int4 c = cell[i];
        const T rho_i = vi.w, p_i = pi.w, m = P.m;
        const T inv_rho_i = T(1) / rho_i;
        const T pi_i = p_i * inv_rho_i;
        const T mu2 = T(2) * P.mu;
        const bool visc = P.mu > T(0);
        // pair sums of the adjoint of pi_i (sp), of pi_i's share of 1/(rho_i +
        // rho_j) (spc) and of V's dependence on rho_i (svv), divided by rho_i
        // once at the end
        T xx = T(0), xy = T(0), xz = T(0), ux = T(0), uy = T(0), uz = T(0), pb = T(0), rb = T(0);
        T sp = T(0), spc = T(0), svv = T(0);
        T c0h = T(0), muh = T(0), muf = T(0), gpf = T(0);
        for_neighbors<PER>(
            C, n, t, pi, c, nbf, nbw, cnt[t], fstart, wstart, pos, wpos,
            [&](int j, const V4<T>& pj, T rx, T ry, T rz, T r2) {
                const V4<T> vj = vel[j], Aj = tA[j];
                const T rinv = p_rsqrt(r2);
                const T R = r2 * rinv;
                const T F = kernel_F(C, R), Fp = kernel_dF(C, R);
                const T inv_rho_j = p_div(T(1), vj.w);
                const T pi_j = pj.w * inv_rho_j;
                const T inv_rs = p_div(T(1), rho_i + vj.w);
                const T vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                const T dU = -(rx * vx + ry * vy + rz * vz) * rinv;
                T phi = T(0), dphi = T(0), dphic = T(0);
                if (dU > T(0)) {
                    if (T(3) * dU < C.c0) {
                        phi = T(3) * dU * dU;
                        dphi = T(6) * dU;
                    } else {
                        phi = C.c0 * dU;
                        dphi = C.c0;
                        dphic = dU;
                    }
                }
                const T Cc = (pi_i + pi_j + phi) * inv_rs;
                const T K = T(-2) * m * F * Cc;
                const T inv_e2 = p_div(T(1), r2 + C.eta2);
                const T Q = r2 * F * inv_e2;
                const T mv = m * inv_rho_i * inv_rho_j;
                const T gx = Ai.x - Aj.x, gy = Ai.y - Aj.y, gz = Ai.z - Aj.z;
                const T Kb = gx * rx + gy * ry + gz * rz;
                const T Vb = gx * vx + gy * vy + gz * vz;
                const T Fb = Kb * (T(-2) * m * Cc);
                const T pib = Kb * (T(-2) * m * F) * inv_rs;
                const T Ub = pib * dphi;
                T Rb = Fb * Fp + (Ai.w + Aj.w) * F * R;
                T V = T(0);
                if (visc) {
                    const T dQ = (T(2) * R * F * C.eta2 * inv_e2 + r2 * Fp) * inv_e2;
                    V = mu2 * mv * Q;
                    Rb += Vb * mu2 * mv * dQ;
                    svv += Vb * V;
                }
                const T cr = Rb * rinv - Ub * dU * rinv * rinv;
                const T cv = -Ub * rinv;
                xx += K * gx + cr * rx + cv * vx;
                xy += K * gy + cr * ry + cv * vy;
                xz += K * gz + cr * rz + cv * vz;
                ux += V * gx + cv * rx;
                uy += V * gy + cv * ry;
                uz += V * gz + cv * rz;
                sp += pib;
                spc += pib * Cc;
                c0h += pib * dphic;
                muh += Vb * T(2) * mv * Q;
            },
            [&](int w, const V4<T>& pw, T rx, T ry, T rz, T r2) {
                WallMomAdj<T> o;
                wall_momentum_adj(C, P, rx, ry, rz, r2, vi.x, vi.y, vi.z, rho_i, p_i, wrho[w].x, pw.w, wnrm[w],
                                  wfront[w] != 0, Ai.x, Ai.y, Ai.z, Ai.w, o);
                xx += o.rx;
                xy += o.ry;
                xz += o.rz;
                ux += o.vx;
                uy += o.vy;
                uz += o.vz;
                pb += o.p_i;
                rb += o.rho_i;
                muf += o.mu;
                gpf += o.gp;
                // extrapolation p_w' = sum_f (p_f + rho_f g.r_wf) W_wf / sum W, r_wf = -r
                const T cw = wc[w];
                if (cw != T(0)) {
                    const T rinv = p_rsqrt(r2);
                    const T R = r2 * rinv;
                    T W, F;
                    kernel_WF(C, R, W, F);
                    const T gr = ge.x * rx + ge.y * ry + ge.z * rz;
                    pb += cw * W;
                    rb -= cw * gr * W;
                    const T k = cw * (p_i - rho_i * gr - pw.w) * F;
                    const T kg = -cw * rho_i * W;
                    xx += kg * ge.x + k * rx;
                    xy += kg * ge.y + k * ry;
                    xz += kg * ge.z + k * rz;
                }
            });
        pb += sp * inv_rho_i;
        rb -= sp * pi_i * inv_rho_i + spc + svv * inv_rho_i;
        xx = group_sum(xx);
        xy = group_sum(xy);
        xz = group_sum(xz);
        ux = group_sum(ux);
        uy = group_sum(uy);
        uz = group_sum(uz);
        pb = group_sum(pb);
        rb = group_sum(rb);
        gc0 = 0.5 * (double)c0h;
        gmu = 0.5 * (double)muh + (double)muf;
        ggp = (double)gpf;
        if (lead) {
            const T d = drho[i];
            const V4<T> gx = gx_in[i], gv = gv_in[i];
            const T dbar = gx.w + rb + pb * eos_dp_dd(P, C, d, p_i);
            gc0 += (double)(pb * T(2) * p_i * C.inv_c0);
            if (create) {
                tX[i] = V4<T>{gx.x + xx, gx.y + xy, gx.z + xz, dbar};
                tV[i] = V4<T>{gv.x + ux, gv.y + uy, gv.z + uz, T(0)};
            } else {
                tX[i] = V4<T>{xx, xy, xz, dt * dbar};
                tV[i] = V4<T>{gv.x + ux, gv.y + uy, gv.z + uz, dbar};
            }
        }
    }
    block_add3(gparam, gc0, ggp, gmu);
}

// Per fluid particle: backward of the continuity sweep (D_i and, for each
// neighbour j, the term e_ji of D_j that depends on particle i), of
// p~ = EOS(d~), the drift, both kicks and the reinitialisation.  Writes the
// adjoint state of the step's input in its own (old) sorted order.
// FP32: eight blocks per SM (at most 64 registers, against 72 unbounded): 125
// against 134 us per step at 189 k fluid particles.  FP64: its unbounded 128.
template <class T, bool PER>
__global__ void __launch_bounds__(LBLOCK, sizeof(T) == 4 ? 8 : 4) k_adj_continuity(
    Cfg<T> C, int32_t n, T dt, int32_t reinit, const int32_t* __restrict__ fstart,
    const int32_t* __restrict__ wstart, const int32_t* __restrict__ nbf, const int32_t* __restrict__ nbw,
    const int32_t* __restrict__ cnt, const V4<T>* __restrict__ pos1, const V4<T>* __restrict__ vel,
    const T* __restrict__ drho1, const int4* __restrict__ cell, const V4<T>* __restrict__ wpos_prev,
    const V2<T>* __restrict__ wrho_prev, const V4<T>* __restrict__ tX, const V4<T>* __restrict__ tV,
    const V4<T>* __restrict__ gx_in, const int32_t* __restrict__ id_new, const int32_t* __restrict__ inv_old,
    const T* __restrict__ drho_old, const T* __restrict__ dsig_old, V4<T>* __restrict__ gx_out,
    V4<T>* __restrict__ gv_out, V4<T>* __restrict__ ga_out, double* gparam)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / LP;
    const bool lead = (t % LP) == 0;
    double gc0 = 0.0;
    if (i < n) {
        const PhaseK<T>& P = C.ph[0];
        const V4<T> pi = pos1[i], vi = vel[i];
        const int4 c = cell[i];
        const T d_i = drho1[i];
        const T rho_i = P.rho0 + d_i, p_i = pi.w;
        const T inv_rho_i = T(1) / rho_i;
        const T Di = tX[i].w;
        const T k = C.inv_c0, m2 = T(2) * P.m;
        T xx = T(0), xy = T(0), xz = T(0), ux = T(0), uy = T(0), uz = T(0), pb = T(0), rb = T(0), cb = T(0);
        for_neighbors<PER>(
            C, n, t, pi, c, nbf, nbw, cnt[t], fstart, wstart, pos1, wpos_prev,
            [&](int j, const V4<T>& pj, T rx, T ry, T rz, T r2) {
                const V4<T> vj = vel[j];
                const T rho_j = P.rho0 + drho1[j], p_j = pj.w;
                const T Dj = tX[j].w;
                const T rinv = p_rsqrt(r2);
                const T R = r2 * rinv;
                const T F = kernel_F(C, R), Fp = kernel_dF(C, R);
                const T inv_rs = p_div(T(1), rho_i + rho_j);
                const T inv_rho_j = p_div(T(1), rho_j);
                const T A = m2 * inv_rs;
                const T vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                const T S = rx * vx + ry * vy + rz * vz;
                const T dpk = (p_i - p_j) * k;
                const T qj = dpk * inv_rho_j, qi = dpk * inv_rho_i;
                const T Bij = S + qj * R, Bji = S - qi * R;
                const T a = Di * rho_i, b = Dj * rho_j;
                const T U = a * Bij + b * Bji;
                const T AF = A * F;
                const T cr = A * (Fp * U + F * (a * qj - b * qi)) * rinv;
                const T cv = AF * (a + b);
                xx += cr * rx + cv * vx;
                xy += cr * ry + cv * vy;
                xz += cr * rz + cv * vz;
                ux += cv * rx;
                uy += cv * ry;
                uz += cv * rz;
                pb += AF * R * k * (a * inv_rho_j - b * inv_rho_i);
                rb += AF * (Di * Bij + b * qi * R * inv_rho_i - U * inv_rs);
                cb -= a * AF * qj * R * k;
            },
            [&](int w, const V4<T>& pw, T rx, T ry, T rz, T r2) {
                WallContAdj<T> o;
                wall_continuity_adj(C, P, rx, ry, rz, r2, vi.x, vi.y, vi.z, rho_i, p_i, wrho_prev[w].x, pw.w, Di,
                                    o);
                xx += o.rx;
                xy += o.ry;
                xz += o.rz;
                ux += o.vx;
                uy += o.vy;
                uz += o.vz;
                pb += o.p_i;
                rb += o.rho_i;
                cb += o.c0;
            });
        xx = group_sum(xx);
        xy = group_sum(xy);
        xz = group_sum(xz);
        ux = group_sum(ux);
        uy = group_sum(uy);
        uz = group_sum(uz);
        pb = group_sum(pb);
        rb = group_sum(rb);
        gc0 = (double)cb;
        if (lead) {
            const V4<T> gx = gx_in[i], tx = tX[i], tv = tV[i];
            // x' = x + dt v'': adjoint of x' in total, then of v''
            const T Xx = gx.x + tx.x + xx, Xy = gx.y + tx.y + xy, Xz = gx.z + tx.z + xz;
            const T Ux = tv.x + ux + dt * Xx, Uy = tv.y + uy + dt * Xy, Uz = tv.z + uz + dt * Xz;
            // d' = d~ + dt D, p~ = EOS(d~), rho~ = rho0 + d~
            const T dt_bar = tv.w + rb + pb * eos_dp_dd(P, C, d_i, p_i);
            gc0 += (double)(pb * T(2) * p_i * C.inv_c0);
            const int s = SPH_CK(inv_old[SPH_CK(id_new[i], n, CK_SLOT)], n, CK_SLOT);
            T dbar = dt_bar, sbar = T(0);
            if (reinit) {
                // d~ = R(d, dsig), Eq. (eqrhosum) written on d = rho - rho0
                const T d = drho_old[s];
                const T dnum = P.rho0 * dsig_old[s] * C.inv_sigma0;
                T dd = T(1), dn = T(0);
                if (P.reinit == 1) {
                    if (d > dnum) {
                        const T rst = P.rho0 + d;
                        dd = T(1) - d / rst - (d - dnum) * P.rho0 / (rst * rst);
                        dn = d / rst;
                    } else {
                        dd = T(0);
                        dn = T(1);
                    }
                } else if (P.reinit == 2) {
                    dd = T(0);
                    dn = T(1);
                }
                dbar = dt_bar * dd;
                sbar = dt_bar * dn * P.rho0 * C.inv_sigma0;
            }
            const T hdt = T(0.5) * dt;
            gx_out[s] = V4<T>{Xx, Xy, Xz, dbar};
            gv_out[s] = V4<T>{Ux, Uy, Uz, sbar};
            ga_out[s] = V4<T>{hdt * Ux, hdt * Uy, hdt * Uz, T(0)};
        }
    }
    block_add3(gparam, gc0, 0.0, 0.0);
}

// Per wall: adjoint of the previous wall pressure p_w^n through the
// continuity pairs (and rho_w^n = rho0 + EOS^-1(p_w^n)).
template <class T, bool PER>
__global__ void __launch_bounds__(LBLOCK) k_adj_wall_continuity(
    Cfg<T> C, int32_t nw, const int32_t* __restrict__ fstart, const V4<T>* __restrict__ wpos_prev,
    const V2<T>* __restrict__ wrho_prev, const int4* __restrict__ wcell, const int32_t* __restrict__ wtag,
    const int32_t* __restrict__ d_tag, const V4<T>* __restrict__ pos1, const V4<T>* __restrict__ vel,
    const T* __restrict__ drho1, const V4<T>* __restrict__ tX, T* __restrict__ gpw_out, double* gparam)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = t / AWLP;
    double gc0 = 0.0;
    if (w < nw) {
        const PhaseK<T>& P = C.ph[0];
        const bool live = wtag[w] == *d_tag;
        const V4<T> pw = wpos_prev[w];
        const T rho_w = wrho_prev[w].x;
        T Gp = T(0), Gr = T(0), Gc = T(0);
        if (live) {
            const int4 c = wcell[w];
            scan_compact<PER, AWLP>(C, c, pw, fstart, pos1, t % AWLP, [&](int j, T rx, T ry, T rz, T r2, int) {
                const V4<T> pf = pos1[j], vf = vel[j];
                WallContAdj<T> o;
                wall_continuity_adj(C, P, -rx, -ry, -rz, r2, vf.x, vf.y, vf.z, P.rho0 + drho1[j], pf.w, rho_w,
                                    pw.w, tX[j].w, o);
                Gp += o.p_w;
                Gr += o.rho_w;
            });
            Gp = group_sum<AWLP>(Gp);
            Gr = group_sum<AWLP>(Gr);
        }
        if (t % AWLP == 0) {
            T out = T(0);
            if (live) {
                const T dd_dp = pw.w < P.p_half ? T(0) : T(1) / eos_dp_dd(P, C, rho_w - P.rho0, pw.w);
                out = Gp + Gr * dd_dp;
                Gc = Gr * (T(-2) * pw.w * C.inv_c0 * dd_dp);
            }
            gpw_out[w] = out;
            gc0 = (double)Gc;
        }
    }
    block_add3(gparam, gc0, 0.0, 0.0);
}

// seeds in original particle order (FP64, NULL = 0) -> adjoint state in the
// current sorted order
template <class T>
__global__ void k_adj_seed(int32_t n, const int32_t* __restrict__ id, const double* __restrict__ sx,
                           const double* __restrict__ sv, const double* __restrict__ srho, V4<T>* __restrict__ gx,
                           V4<T>* __restrict__ gv, V4<T>* __restrict__ ga)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = id[i];
    V4<T> x{T(0), T(0), T(0), T(0)}, v{T(0), T(0), T(0), T(0)};
    if (sx) x = V4<T>{(T)sx[3 * k], (T)sx[3 * k + 1], (T)sx[3 * k + 2], T(0)};
    if (srho) x.w = (T)srho[k];
    if (sv) v = V4<T>{(T)sv[3 * k], (T)sv[3 * k + 1], (T)sv[3 * k + 2], T(0)};
    gx[i] = x;
    gv[i] = v;
    ga[i] = V4<T>{T(0), T(0), T(0), T(0)};
}

template <class T>
__global__ void k_adj_seed_wall(int32_t nw, const int32_t* __restrict__ wid, const double* __restrict__ spw,
                                T* __restrict__ gpw)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    gpw[w] = spw ? (T)spw[wid[w]] : T(0);
}

// final adjoints (create order) -> original particle order, FP64
template <class T>
__global__ void k_adj_export(int32_t n, const int32_t* __restrict__ id, const V4<T>* __restrict__ tX,
                             const V4<T>* __restrict__ tV, double* __restrict__ ox, double* __restrict__ ov,
                             double* __restrict__ orho)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = id[i];
    const V4<T> x = tX[i], v = tV[i];
    if (ox) {
        ox[3 * k] = (double)x.x;
        ox[3 * k + 1] = (double)x.y;
        ox[3 * k + 2] = (double)x.z;
    }
    if (ov) {
        ov[3 * k] = (double)v.x;
        ov[3 * k + 1] = (double)v.y;
        ov[3 * k + 2] = (double)v.z;
    }
    if (orho) orho[k] = (double)x.w;
}

// Copy of up to 16 device arrays in one launch (checkpoint save / restore).
// Sizes are in 4-byte words; every array starts 16-byte aligned (cudaMalloc
// bases, 256-byte checkpoint slots), so whole 16-byte chunks move as uint4.
struct CopySeg {
    void* dst;
    const void* src;
    size_t words;
};
struct CopyList {
    CopySeg seg[16];
    int n;
    size_t total;
};

static __global__ void k_copy_segments(CopyList L)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int s = 0; s < L.n; ++s) {
        uint32_t* d = (uint32_t*)L.seg[s].dst;
        const uint32_t* q = (const uint32_t*)L.seg[s].src;
        const size_t n = L.seg[s].words, n4 = n / 4;
        uint4* d4 = (uint4*)d;
        const uint4* q4 = (const uint4*)q;
        for (size_t k = t0; k < n4; k += stride) d4[k] = q4[k];
        for (size_t k = 4 * n4 + t0; k < n; k += stride) d[k] = q[k];
    }
}

static __global__ void k_bump_tag(int32_t* d_tag)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *d_tag += 1;
}

}  // namespace sph
