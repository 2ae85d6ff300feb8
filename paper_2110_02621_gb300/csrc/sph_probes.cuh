// Pressure sensors and wave-height gauges (arXiv 2110.02621, Sec. 4.3: the
// sensors P_i and the gauges H_i of the dam break with an obstacle).  Both
// read the sorted fluid state between steps and evaluate in FP64 whatever the
// precision of the state:
//   sensors: w(r) = sum_j V_j W(|r - r_j|), V_j = m_j/rho_j, and the Shepard
//            average p_bar(r) = sum_j p_j V_j W(|r - r_j|) / w(r) (0 if w = 0),
//            over every in-grid fluid particle with |r - r_j| < 2h;
//   gauges:  the highest crossing of the liquid (phase 0) volume fraction
//            phi = 1/2 along a vertical line, sampled dz apart from z_lo,
//            linearly interpolated between the bracketing samples.
// Positions are rebuilt as lo + cell cs + offset from the cell being walked,
// exactly as the FP64 export rebuilds them.
#pragma once

#include "sph.h"
#include "sph_device.cuh"
#include "sph_setup.cuh"
#include "sph_sweeps.cuh"

namespace sph {

constexpr int GAUGE_BLOCK = 128;
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
// point (px, py, pz) whose squared distance r2 = |x - r_j|^2 is below (2h)^2, r = 0
// included;
// the walk over each cell's range is strided by (lane, nlanes).
template <class T, class Fn>
__device__ __forceinline__ void for_fluid_near(const Cfg<double>& D, const InitCfg& I, double px, double py,
                                               double pz, const int32_t* __restrict__ start,
                                               const V4<T>* __restrict__ pos, int lane, int nlanes, Fn&& fn)
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
    const double rc2 = D.rc2;
    // z, y, xx: the geometric cells (their shift); zm, ym, xm: where they are stored
    for (int z = cz - 1; z <= cz + 1; ++z) {
        int zm = z;
        if (!row_axis(zm, D.nz, D.periodic & 4)) continue;
        const double bz = uz - (double)z * I.cs;
        for (int y = cy - 1; y <= cy + 1; ++y) {
            int ym = y;
            if (!row_axis(ym, D.ny, D.periodic & 2)) continue;
            const double by = uy - (double)y * I.cs;
            const int row = (zm * D.ny + ym) * D.nx;
            for (int xx = cx - 1; xx <= cx + 1; ++xx) {
                int xm = xx;
                if (!row_axis(xm, D.nx, D.periodic & 1)) continue;
                const double bx = ux - (double)xx * I.cs;
                const int c = row + xm;
                const int b = __ldg(start + c), e = __ldg(start + c + 1);
                for (int j = b + lane; j < e; j += nlanes) {
                    const V4<T> o = pos[j];
                    const double rx = bx - (double)o.x, ry = by - (double)o.y, rz = bz - (double)o.z;
                    const double r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 < rc2) fn(j, r2);
                }
            }
        }
    }
}

__device__ __forceinline__ double wendland_W64(const Cfg<double>& D, double r2)
{
    return kernel_W(D, sqrt(r2));
}

// One warp per sensor point.
template <class T>
__global__ void k_probe_pressure(Cfg<double> D, InitCfg I, int32_t n, const double* __restrict__ pts,
                                 const int32_t* __restrict__ start, const V4<T>* __restrict__ pos,
                                 const T* __restrict__ drho, const int32_t* __restrict__ phase,
                                 double* __restrict__ p_out, double* __restrict__ w_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= n) return;
    double sw = 0.0, spw = 0.0;
    for_fluid_near(D, I, pts[3 * k], pts[3 * k + 1], pts[3 * k + 2], start, pos, lane, 32, [&](int j, double r2) {
        // phase selected by value: an indexed kernel parameter would be
        // copied to local memory
        const bool p0 = phase[j] == 0;
        const double Vj = (p0 ? D.ph[0].m : D.ph[1].m) / ((p0 ? I.rho0[0] : I.rho0[1]) + (double)drho[j]);
        const double wj = Vj * wendland_W64(D, r2);
        sw += wj;
        spw += (double)pos[j].w * wj;
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

// One block per gauge: chunks of GAUGE_BLOCK samples from the top down, one
// sample per thread; the first chunk holding a sample with phi >= 1/2 gives
// the highest such sample, whose upper neighbour is in the same chunk or is
// the lowest sample of the chunk before.  A line that is not finite, has
// z_hi < z_lo or more than GAUGE_MAX_SAMPLES samples gives NaN (the host
// entry point rejects such lines before launching).
template <class T>
__global__ void k_gauge_height(Cfg<double> D, InitCfg I, int32_t n, const double* __restrict__ g, double dz,
                               const int32_t* __restrict__ start, const V4<T>* __restrict__ pos,
                               const T* __restrict__ drho, const int32_t* __restrict__ phase,
                               double* __restrict__ H)
{
    __shared__ double phi_s[GAUGE_BLOCK];
    __shared__ int best;
    const int k = blockIdx.x;
    if (k >= n) return;
    const double gx = g[4 * k], gy = g[4 * k + 1], zlo = g[4 * k + 2], zhi = g[4 * k + 3];
    const double Kd = floor((zhi - zlo) / dz);
    if (!(Kd >= 0.0 && Kd < (double)GAUGE_MAX_SAMPLES) || !isfinite(gx) || !isfinite(gy) || !isfinite(zlo)) {
        if (threadIdx.x == 0) H[k] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int64_t K = (int64_t)Kd;
    const double m0 = D.ph[0].m, rho00 = I.rho0[0];
    double phi_above = 0.0;  // phi of the sample above the current chunk
    double out = zlo;
    for (int64_t top = K; top >= 0; top -= GAUGE_BLOCK) {
        const int64_t i = top - threadIdx.x;
        double phi = 0.0;
        if (i >= 0) {
            for_fluid_near(D, I, gx, gy, zlo + (double)i * dz, start, pos, 0, 1, [&](int j, double r2) {
                if (phase[j] != 0) return;
                phi += m0 / (rho00 + (double)drho[j]) * wendland_W64(D, r2);
            });
        }
        phi_s[threadIdx.x] = phi;
        if (threadIdx.x == 0) best = GAUGE_BLOCK;
        __syncthreads();
        if (i >= 0 && phi >= 0.5) atomicMin(&best, (int)threadIdx.x);
        __syncthreads();
        const int b = best;
        if (b < GAUGE_BLOCK) {
            if (threadIdx.x == 0) {
                const int64_t ib = top - b;
                const double zb = zlo + (double)ib * dz, pb = phi_s[b];
                const double pa = b > 0 ? phi_s[b - 1] : phi_above;
                out = ib == K ? zb : zb + dz * (pb - 0.5) / (pb - pa);
            }
            break;
        }
        phi_above = phi_s[GAUGE_BLOCK - 1];
        __syncthreads();  // phi_s and best are rewritten by the next chunk
    }
    if (threadIdx.x == 0) H[k] = out;
}

}  // namespace sph
