// Create-time kernels (binning from FP64 input, hydrostatic start, wall
// normals), the FP64 state export and the FP64 diagnostics reductions.
#pragma once

#include "sph_sweeps.cuh"

namespace sph {

// FP64 per-phase numbers used only at create time.
struct InitCfg {
    double lo[3];
    double cs;
    double gz;          // g_z (hydrostatic column along -z)
    double c0, gamma;
    int32_t n_phases;
    int32_t has_rho;
    double rho0[2], z_top[2];
    int32_t eos[2];
    double sigma0;      // lattice number density (the stored sigma is sigma - sigma0)
};

// cell of an FP64 position: c = floor((x - lo)/cs) in FP64, offset x - lo - c cs
// clamped into [0, cs] before rounding to T; along a periodic axis x - lo is
// first wrapped into [0, period).
template <class T>
__device__ __forceinline__ void bin_fp64(const Cfg<T>& C, const InitCfg& I, const double* x,
                                         int4& c, V4<T>& o)
{
    int32_t cc[3];
    T oo[3];
    const int32_t nd[3] = {C.nx, C.ny, C.nz};
    for (int d = 0; d < 3; ++d) {
        double u = x[d] - I.lo[d];
        if ((C.periodic >> d) & 1) {  // into [0, n cs): the period is n whole cells
            const double L = (double)nd[d] * I.cs;
            u = fmod(u, L);
            if (u < 0.0) u += L;
        }
        double f = floor(u / I.cs);
        if (((C.periodic >> d) & 1) && f > (double)(nd[d] - 1)) f = (double)(nd[d] - 1);
        cc[d] = (f < -1e9) ? -1000000000 : (f > 1e9 ? 1000000000 : (int32_t)f);
        double r = u - f * I.cs;
        r = r < 0.0 ? 0.0 : (r > I.cs ? I.cs : r);
        T rt = (T)r;
        oo[d] = rt > C.cs ? C.cs : rt;
    }
    c = int4{cc[0], cc[1], cc[2], (int)cell_key(C, cc[0], cc[1], cc[2])};
    o = V4<T>{oo[0], oo[1], oo[2], T(0)};
}

// hydrostatic pressure of stacked phase columns (phase k spans
// (z_top[k-1], z_top[k]]), FP64
__device__ __forceinline__ double hydro_p(const InitCfg& I, int k, double z)
{
    double g = -I.gz;
    double p = I.rho0[k] * g * (I.z_top[k] - z);
    for (int m = k + 1; m < I.n_phases; ++m) p += I.rho0[m] * g * (I.z_top[m] - I.z_top[m - 1]);
    return p;
}

// Checks of fluid inputs that are device memory (sph_create_device), the
// same as sph_create makes on the host: finite positions and velocities,
// finite rho > 0, phase in [0, n_phases), and in 2-D one y for every
// particle (y0, or the first particle's y) with zero y velocity.  Any failure
// sets bit 0 of *bad.
static __global__ void k_check_fluid(int32_t n, const double* __restrict__ x, const double* __restrict__ v,
                                     const double* __restrict__ rho, const int32_t* __restrict__ phase,
                                     int32_t n_phases, int32_t dim2, double y0, int32_t y0_first, int32_t* bad)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = isfinite(x[3 * i]) && isfinite(x[3 * i + 1]) && isfinite(x[3 * i + 2]);
    if (v) ok = ok && isfinite(v[3 * i]) && isfinite(v[3 * i + 1]) && isfinite(v[3 * i + 2]);
    if (rho) ok = ok && rho[i] > 0.0 && isfinite(rho[i]);
    if (phase) ok = ok && phase[i] >= 0 && phase[i] < n_phases;
    if (dim2) {
        const double yr = y0_first ? x[1] : y0;
        ok = ok && x[3 * i + 1] == yr && (!v || v[3 * i + 1] == 0.0);
    }
    if (!ok) atomicOr(bad, 1);
}

// Fluid in input order: cell, offset, velocity, density excess and pressure;
// counts the cell occupancy for the first sort.
template <class T>
__global__ void k_init_fluid(Cfg<T> C, InitCfg I, int32_t n, const double* __restrict__ x,
                             const double* __restrict__ v, const double* __restrict__ rho,
                             const int32_t* __restrict__ phase_in, V4<T>* __restrict__ pos,
                             V4<T>* __restrict__ vel, T* __restrict__ drho, V4<T>* __restrict__ acc,
                             V4<T>* __restrict__ comp, int4* __restrict__ newcell,
                             int32_t* __restrict__ id, int32_t* __restrict__ phase,
                             int32_t* __restrict__ rank, int32_t* counts)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 c;
    V4<T> o;
    bin_fp64(C, I, x + 3 * i, c, o);
    int ph = phase_in ? phase_in[i] : 0;
    double d;
    if (I.has_rho) {
        d = rho[i] - I.rho0[ph];
    } else {
        double p = hydro_p(I, ph, x[3 * i + 2]);
        if (I.eos[ph] == 1)
            d = I.rho0[ph] * expm1(log1p(I.gamma * p / (I.rho0[ph] * I.c0 * I.c0)) / I.gamma);
        else
            d = p / (I.c0 * I.c0);
    }
    T dt = (T)d;
    o.w = eos_p(C.ph[ph], C, dt);
    pos[i] = o;
    if (v)
        vel[i] = V4<T>{(T)v[3 * i], (T)v[3 * i + 1], (T)v[3 * i + 2], C.ph[ph].rho0 + dt};
    else
        vel[i] = V4<T>{T(0), T(0), T(0), C.ph[ph].rho0 + dt};
    drho[i] = dt;
    acc[i] = V4<T>{T(0), T(0), T(0), T(0)};
    comp[i] = V4<T>{T(0), T(0), T(0), T(0)};
    newcell[i] = c;
    id[i] = i;
    phase[i] = ph;
    int bucket = c.w < 0 ? C.n_cells : c.w;
    rank[i] = atomicAdd(counts + bucket, 1);
}

// Walls in input order: cell, offset, counts.
template <class T>
__global__ void k_init_wall(Cfg<T> C, InitCfg I, int32_t n, const double* __restrict__ x,
                            V4<T>* __restrict__ wpos, int4* __restrict__ wcell,
                            int32_t* __restrict__ wid, int32_t* __restrict__ rank, int32_t* counts)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 c;
    V4<T> o;
    bin_fp64(C, I, x + 3 * i, c, o);
    wpos[i] = o;
    wcell[i] = c;
    wid[i] = i;
    int bucket = c.w < 0 ? C.n_cells : c.w;
    rank[i] = atomicAdd(counts + bucket, 1);
}

// Walls into (key, id) order, with their FP64 positions for the normals.
template <class T>
__global__ void k_gather_wall(int32_t n, int32_t n_cells, const int32_t* __restrict__ start,
                              const int32_t* __restrict__ tmp_src, const int32_t* __restrict__ tmp_id,
                              const V4<T>* __restrict__ wpos, const int4* __restrict__ wcell,
                              const double* __restrict__ x, V4<T>* __restrict__ wpos_o,
                              int4* __restrict__ wcell_o, int32_t* __restrict__ wid_o,
                              double* __restrict__ x_o)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int s = tmp_src[t];
    int4 c = wcell[s];
    int dst = sorted_slot(t, c.w, n_cells, start, tmp_id);
    wpos_o[dst] = wpos[s];
    wcell_o[dst] = c;
    wid_o[dst] = tmp_id[t];
    int id = tmp_id[t];
    x_o[3 * dst] = x[3 * id];
    x_o[3 * dst + 1] = x[3 * id + 1];
    x_o[3 * dst + 2] = x[3 * id + 2];
}

// Wall unit normals, Eq. (normalVectors): n_w = Psi/|Psi|,
// Psi = -sum_{j in wall} dx^3 grad_w W_wj, in FP64 from the FP64 positions
// (exact lattice symmetry); |Psi| < 1e-6/dx gives n_w = 0.
template <class T>
__global__ void k_wall_normals(Cfg<double> D, int32_t n, const int32_t* __restrict__ wstart,
                               const int4* __restrict__ wcell, const double* __restrict__ x,
                               V4<T>* __restrict__ wnrm)
{
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n) return;
    int4 c = wcell[w];
    double px = 0.0, py = 0.0, pz = 0.0;
    const double xw = x[3 * w], yw = x[3 * w + 1], zw = x[3 * w + 2];
    if (c.w >= 0) {
        for_cells27(D, c.x, c.y, c.z, wstart, [&](int j, double, double, double) {
            double rx = xw - x[3 * j], ry = yw - x[3 * j + 1], rz = zw - x[3 * j + 2];
            if (D.periodic) {  // nearest image along the periodic axes
                if (D.periodic & 1) rx -= D.nx * D.cs * rint(rx / (D.nx * D.cs));
                if (D.periodic & 2) ry -= D.ny * D.cs * rint(ry / (D.ny * D.cs));
                if (D.periodic & 4) rz -= D.nz * D.cs * rint(rz / (D.nz * D.cs));
            }
            double r2 = rx * rx + ry * ry + rz * rz;
            if (r2 >= D.rc2 || r2 == 0.0) return;
            double F = kernel_F(D, sqrt(r2));
            px -= D.vol * F * rx;
            py -= D.vol * F * ry;
            pz -= D.vol * F * rz;
        });
    }
    double m = sqrt(px * px + py * py + pz * pz);
    if (m >= 1e-6 * D.inv_dp)
        wnrm[w] = V4<T>{(T)(px / m), (T)(py / m), (T)(pz / m), T(0)};
    else
        wnrm[w] = V4<T>{T(0), T(0), T(0), T(0)};
}

// ------------------------------------------------------------------ export
struct ExportOut {
    double *pos, *vel, *rho, *p, *acc, *drho_dt, *sigma;
};

template <class T>
__global__ void k_export_fluid(Cfg<T> C, InitCfg I, int32_t n, const V4<T>* __restrict__ pos,
                               const V4<T>* __restrict__ vel, const T* __restrict__ drho,
                               const V4<T>* __restrict__ acc, const T* __restrict__ sigma,
                               const int4* __restrict__ cell, const int32_t* __restrict__ id,
                               const int32_t* __restrict__ phase, ExportOut o)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = id[k];
    V4<T> p = pos[k], v = vel[k], a = acc[k];
    int4 c = cell[k];
    if (o.pos) {
        o.pos[3 * i] = I.lo[0] + (double)c.x * I.cs + (double)p.x;
        o.pos[3 * i + 1] = I.lo[1] + (double)c.y * I.cs + (double)p.y;
        o.pos[3 * i + 2] = I.lo[2] + (double)c.z * I.cs + (double)p.z;
    }
    if (o.vel) {
        o.vel[3 * i] = v.x;
        o.vel[3 * i + 1] = v.y;
        o.vel[3 * i + 2] = v.z;
    }
    if (o.rho) o.rho[i] = I.rho0[phase[k]] + (double)drho[k];
    if (o.p) o.p[i] = p.w;
    if (o.acc) {
        o.acc[3 * i] = a.x;
        o.acc[3 * i + 1] = a.y;
        o.acc[3 * i + 2] = a.z;
    }
    if (o.drho_dt) o.drho_dt[i] = a.w;
    if (o.sigma) o.sigma[i] = I.sigma0 + (double)sigma[k];
}

template <class T>
__global__ void k_export_wall(int32_t n, const V4<T>* __restrict__ wpos, const V2<T>* __restrict__ wrho,
                              const V4<T>* __restrict__ wnrm, const int32_t* __restrict__ wid,
                              double* pw, double* rhow, double* nrm)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = wid[k];
    if (pw) pw[i] = wpos[k].w;
    if (rhow) {
        V2<T> r = wrho[k];
        rhow[2 * i] = r.x;
        rhow[2 * i + 1] = r.y;
    }
    if (nrm) {
        V4<T> q = wnrm[k];
        nrm[3 * i] = q.x;
        nrm[3 * i + 1] = q.y;
        nrm[3 * i + 2] = q.z;
    }
}

// key per id and the sorted order, as the cell-list API returns them
static __global__ void k_export_cells(int32_t n, const int4* __restrict__ cell,
                                      const int32_t* __restrict__ id, uint32_t* __restrict__ key_by_id,
                                      int32_t* __restrict__ order)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = id[k];
    if (key_by_id) key_by_id[i] = (uint32_t)cell[k].w;
    if (order) order[k] = i;
}

// ------------------------------------------------------------- diagnostics
// FP64 sums of {mass, momentum x/y/z, E_kin, E_pot, -, escaped} and the
// maximum of |v|^2 (field 6; its square root is taken at the end, which gives
// the same bits as the maximum of the roots), in a fixed order
// (deterministic): each thread accumulates a fixed grid-stride share of the
// particles, warps and blocks reduce with fixed trees, one block combines the
// block partials.
constexpr int DIAG_MAX_BLOCKS = 1216;  // 8 blocks of 128 threads on each of the 152 SMs

// The warp totals of the 8 fields of q (field 6 included as a sum; callers
// reduce it separately with max): a transposing butterfly in which, at each
// of the first three xor levels, a lane keeps half of its values and adds the
// partner's copy of that half, so that 9 additions and 9 shuffles replace 40.
// Lanes 4f..4f+3 end up holding the total of field f = (lane >> 2) & 7.
__device__ __forceinline__ double warp_sum8(const double (&q)[8], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    double r[4], s[2];
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // r[j] is field j + 4 b4
        const double send = b4 ? q[j] : q[j + 4];
        r[j] = (b4 ? q[j + 4] : q[j]) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {  // s[j] is field j + 2 b3 + 4 b4
        const double send = b3 ? r[j] : r[j + 2];
        s[j] = (b3 ? r[j + 2] : r[j]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    double u = (b2 ? s[1] : s[0]) + __shfl_xor_sync(0xffffffffu, b2 ? s[0] : s[1], 4);
    u += __shfl_xor_sync(0xffffffffu, u, 2);
    u += __shfl_xor_sync(0xffffffffu, u, 1);
    return u;
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block stage shared by both kernels: the warps' 8 results, then thread f < 8
// combines field f over the warps in order.
template <int THREADS>
__device__ __forceinline__ double block_reduce8(const double (&q)[8], double vmax2, double (&sh)[8][THREADS / 32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double u = warp_sum8(q, lane);
    const double m = warp_max(vmax2);
    const int f = (lane >> 2) & 7;
    if ((lane & 3) == 0 && f != 6) sh[f][warp] = u;
    if (lane == 0) sh[6][warp] = m;
    __syncthreads();
    double a = 0.0;
    if (threadIdx.x < 8) {
        const int g = threadIdx.x;
        a = sh[g][0];
        for (int w = 1; w < THREADS / 32; ++w) a = g == 6 ? fmax(a, sh[g][w]) : a + sh[g][w];
    }
    return a;
}

template <class T>
__global__ void __launch_bounds__(BLOCK) k_diag_partial(Cfg<T> C, InitCfg I, int32_t n,
                                                        const V4<T>* __restrict__ pos,
                                                        const V4<T>* __restrict__ vel,
                                                        const int4* __restrict__ cell,
                                                        const int32_t* __restrict__ phase,
                                                        double* __restrict__ partial)
{
    __shared__ double sh[8][BLOCK / 32];
    double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double vmax2 = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const V4<T> p = pos[k], v = vel[k];
        const int4 c = cell[k];
        // the phase picked by value: an indexed kernel parameter would go
        // through local memory
        const double m = (double)(phase[k] == 0 ? C.ph[0].m : C.ph[1].m);
        const double vx = v.x, vy = v.y, vz = v.z;
        const double x = I.lo[0] + (double)c.x * I.cs + (double)p.x;
        const double y = I.lo[1] + (double)c.y * I.cs + (double)p.y;
        const double z = I.lo[2] + (double)c.z * I.cs + (double)p.z;
        const double v2 = vx * vx + vy * vy + vz * vz;
        q[0] += m;
        q[1] += m * vx;
        q[2] += m * vy;
        q[3] += m * vz;
        q[4] += 0.5 * m * v2;
        q[5] += -m * ((double)C.gx * x + (double)C.gy * y + (double)C.gz * z);
        if (c.w >= 0)
            vmax2 = fmax(vmax2, v2);
        else
            q[7] += 1.0;
    }
    const double a = block_reduce8<BLOCK>(q, vmax2, sh);
    if (threadIdx.x < 8) partial[blockIdx.x * 8 + threadIdx.x] = a;
}

// The 8 results over the blocks' partials: DIAG_THREADS threads stride over
// the blocks for each quantity, then the fixed trees combine them.
constexpr int DIAG_THREADS = 256;

static __global__ void __launch_bounds__(DIAG_THREADS) k_diag_final(int32_t nblocks,
                                                                    const double* __restrict__ partial,
                                                                    double* __restrict__ out)
{
    __shared__ double sh[8][DIAG_THREADS / 32];
    double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double vmax2 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += DIAG_THREADS) {
        for (int f = 0; f < 8; ++f)
            if (f != 6) q[f] += partial[b * 8 + f];
        vmax2 = fmax(vmax2, partial[b * 8 + 6]);
    }
    const double a = block_reduce8<DIAG_THREADS>(q, vmax2, sh);
    if (threadIdx.x < 8) out[threadIdx.x] = threadIdx.x == 6 ? sqrt(a) : a;
}

}  // namespace sph
