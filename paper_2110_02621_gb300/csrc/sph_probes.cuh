// Pressure sensors and wave-height gauges (arXiv 2110.02621, Sec. 4.3: the
// sensors P_i and the gauges H_i of the dam break with an obstacle).  Both
// read the sorted fluid state between steps; pair terms are evaluated in the
// state's precision (as the sweeps do) and summed in FP64:
//   sensors: w(r) = sum_j V_j W(|r - r_j|), V_j = m_j/rho_j, and the Shepard
//            average p_bar(r) = sum_j p_j V_j W(|r - r_j|) / w(r) (0 if w = 0),
//            over every in-grid fluid particle with |r - r_j| < 2h;
//   gauges:  the highest crossing of the liquid (phase 0) volume fraction
//            phi = 1/2 along a vertical line, sampled dz apart from z_lo,
//            linearly interpolated between the bracketing samples.
// Positions are taken relative to the cell being walked (point minus cell
// corner in FP64, then the particle's offset), the geometry the export uses.
#pragma once

#include "sph.h"
#include "sph_device.cuh"
#include "sph_setup.cuh"
#include "sph_sweeps.cuh"

namespace sph {

constexpr int GAUGE_BLOCK = 128;  // threads per block of the gauge sweep (4 samples at a time)
constexpr int64_t GAUGE_MAX_SAMPLES = SPH_GAUGE_MAX_SAMPLES;  // samples per gauge line

// Cell index of coordinate u = x - lo along one axis, clamped to [-2, n + 1]
// so that a point far outside the grid (or a NaN) walks no cell and the
// conversion never overflows.
__device__ __forceinline__ int32_t probe_cell(double u, double cs, int32_t n)
{
    double f = floor(u / cs);
    f = f >= -2.0 ? f : -2.0;
    f = f <= (double)(n + 1) ? f : (double)(n + 1);
    return (int32_t)f;
}

// Calls fn(j, r2) for every sorted fluid particle j of the 27 cells around
// point (px, py, pz) whose squared distance r2 = |x - r_j|^2 (in T) is below
// (2h)^2, r = 0 included.  A whole warp walks the cells: lane l < 27 first
// fetches the particle range of cell l (so the 27 range loads overlap instead
// of forming a chain), then every cell's range is broadcast and split over
// the 32 lanes.
template <class T, class Fn>
__device__ __forceinline__ void for_fluid_near(const Cfg<T>& C, const Cfg<double>& D, const InitCfg& I, double px,
                                               double py, double pz, const int32_t* __restrict__ start,
                                               const V4<T>* __restrict__ pos, int lane, Fn&& fn)
{
    // along a periodic axis the point is first wrapped into [0, period)
    auto wrapped = [&](double u, int32_t n, int bit) {
        if (!(D.periodic & bit)) return u;
        const double L = (double)n * I.cs;
        u = fmod(u, L);
        return u < 0.0 ? u + L : u;
    };
    const double ux = wrapped(px - I.lo[0], D.nx, 1), uy = wrapped(py - I.lo[1], D.ny, 2),
                 uz = wrapped(pz - I.lo[2], D.nz, 4);
    const int32_t cx = probe_cell(ux, I.cs, D.nx), cy = probe_cell(uy, I.cs, D.ny),
                  cz = probe_cell(uz, I.cs, D.nz);
    // lane l < 27 owns cell (dx, dy, dz) = (l % 3, l / 3 % 3, l / 9) - 1: its
    // geometric position (the shift) and, where it exists, its stored range
    int b = 0, e = 0;
    T bx = T(0), by = T(0), bz = T(0);
    if (lane < 27) {
        const int x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
        int xm = x, ym = y, zm = z;
        if (row_axis(xm, D.nx, D.periodic & 1) && row_axis(ym, D.ny, D.periodic & 2) &&
            row_axis(zm, D.nz, D.periodic & 4)) {
            const int c = (zm * D.ny + ym) * D.nx + xm;
            b = __ldg(start + c);
            e = __ldg(start + c + 1);
        }
        bx = (T)(ux - (double)x * I.cs);
        by = (T)(uy - (double)y * I.cs);
        bz = (T)(uz - (double)z * I.cs);
    }
#pragma unroll 3
    for (int k = 0; k < 27; ++k) {
        const int cb = __shfl_sync(0xffffffffu, b, k), ce = __shfl_sync(0xffffffffu, e, k);
        const T sx = __shfl_sync(0xffffffffu, bx, k), sy = __shfl_sync(0xffffffffu, by, k),
                sz = __shfl_sync(0xffffffffu, bz, k);
        for (int j = cb + lane; j < ce; j += 32) {
            const V4<T> o = pos[j];
            const T rx = sx - o.x, ry = sy - o.y, rz = sz - o.z;
            const T r2 = dist2(rx, ry, rz);
            if (r2 < C.rc2) fn(j, r2);
        }
    }
}

// V_j W(r): the volume m/rho of a particle of the phase times the kernel
template <class T>
__device__ __forceinline__ T volume_W(const Cfg<T>& C, T m, T rho, T r2)
{
    return p_div(m, rho) * kernel_W(C, r2 * p_rsqrt(r2));
}

// One warp per sensor point.
template <class T>
__global__ void k_probe_pressure(Cfg<T> C, Cfg<double> D, InitCfg I, int32_t n, const double* __restrict__ pts,
                                 const int32_t* __restrict__ start, const V4<T>* __restrict__ pos,
                                 const T* __restrict__ drho, const int32_t* __restrict__ phase,
                                 double* __restrict__ p_out, double* __restrict__ w_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= n) return;
    double sw = 0.0, spw = 0.0;
    for_fluid_near(C, D, I, pts[3 * k], pts[3 * k + 1], pts[3 * k + 2], start, pos, lane, [&](int j, T r2) {
        // phase selected by value: an indexed kernel parameter would be
        // copied to local memory
        const bool p0 = phase[j] == 0;
        const T wj = volume_W(C, p0 ? C.ph[0].m : C.ph[1].m, (p0 ? C.ph[0].rho0 : C.ph[1].rho0) + drho[j], r2);
        sw += (double)wj;
        spw += (double)pos[j].w * (double)wj;
    });
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        spw += __shfl_xor_sync(0xffffffffu, spw, o);
    }
    if (lane == 0) {
        if (w_out) w_out[k] = sw;
        if (p_out) p_out[k] = sw > 0.0 ? spw / sw : 0.0;
    }
}

// Samples K of a gauge line: z_i = z_lo + i dz for i = 0..K; -1 for a line
// that is not finite, has z_hi < z_lo or more than GAUGE_MAX_SAMPLES samples.
__device__ __forceinline__ int64_t gauge_top(const double* g, double dz)
{
    const double Kd = floor((g[3] - g[2]) / dz);
    if (!(Kd >= 0.0 && Kd < (double)GAUGE_MAX_SAMPLES) || !isfinite(g[0]) || !isfinite(g[1]) || !isfinite(g[2]))
        return -1;
    return (int64_t)Kd;
}

// The liquid (phase 0) volume fraction at sample i of line g, one warp
// (lanes over each cell's particles, a fixed shuffle tree: the same value
// whichever warp computes it).
template <class T>
__device__ __forceinline__ double gauge_phi(const Cfg<T>& C, const Cfg<double>& D, const InitCfg& I,
                                            const double* g, double dz, int64_t i,
                                            const int32_t* __restrict__ start, const V4<T>* __restrict__ pos,
                                            const T* __restrict__ drho, const int32_t* __restrict__ phase, int lane)
{
    double phi = 0.0;
    const T m0 = C.ph[0].m, rho00 = C.ph[0].rho0;
    for_fluid_near(C, D, I, g[0], g[1], g[2] + (double)i * dz, start, pos, lane, [&](int j, T r2) {
        if (phase[j] != 0) return;
        phi += (double)volume_W(C, m0, rho00 + drho[j], r2);
    });
    for (int o = 16; o > 0; o >>= 1) phi += __shfl_xor_sync(0xffffffffu, phi, o);
    return phi;
}

constexpr int GAUGE_BLOCKS_PER_LINE = 128;

// Every sample of every line in parallel (a warp per sample, grid-stride over
// the line's samples): best[k] = the highest sample index with phi >= 1/2
// (best[] starts at -1; the maximum of an index is independent of order).
template <class T>
__global__ void __launch_bounds__(GAUGE_BLOCK) k_gauge_crossing(Cfg<T> C, Cfg<double> D, InitCfg I, int32_t n,
                                                                const double* __restrict__ g, double dz,
                                                                const int32_t* __restrict__ start,
                                                                const V4<T>* __restrict__ pos,
                                                                const T* __restrict__ drho,
                                                                const int32_t* __restrict__ phase,
                                                                int32_t* __restrict__ best)
{
    const int k = blockIdx.y;
    if (k >= n) return;
    const int64_t K = gauge_top(g + 4 * k, dz);
    const int lane = threadIdx.x & 31, warps = GAUGE_BLOCK / 32;
    for (int64_t i = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); i <= K; i += (int64_t)gridDim.x * warps) {
        const double phi = gauge_phi(C, D, I, g + 4 * k, dz, i, start, pos, drho, phase, lane);
        if (lane == 0 && phi >= 0.5) atomicMax(best + k, (int32_t)i);
    }
}

// One warp per line: H from the highest wet sample and the one above it.
template <class T>
__global__ void k_gauge_finish(Cfg<T> C, Cfg<double> D, InitCfg I, int32_t n, const double* __restrict__ g,
                               double dz, const int32_t* __restrict__ start, const V4<T>* __restrict__ pos,
                               const T* __restrict__ drho, const int32_t* __restrict__ phase,
                               const int32_t* __restrict__ best, double* __restrict__ H)
{
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= n) return;
    const double* gk = g + 4 * k;
    const int64_t K = gauge_top(gk, dz);
    double out;
    if (K < 0) {
        out = __longlong_as_double(0x7ff8000000000000ll);
    } else {
        const int64_t b = best[k];
        if (b < 0) {
            out = gk[2];  // dry line
        } else {
            const double zb = gk[2] + (double)b * dz;
            if (b == K) {
                out = zb;  // wet to the top sample
            } else {
                const double pb = gauge_phi(C, D, I, gk, dz, b, start, pos, drho, phase, lane);
                const double pa = gauge_phi(C, D, I, gk, dz, b + 1, start, pos, drho, phase, lane);
                out = zb + dz * (pb - 0.5) / (pb - pa);
            }
        }
    }
    if (lane == 0) H[k] = out;
}

}  // namespace sph
