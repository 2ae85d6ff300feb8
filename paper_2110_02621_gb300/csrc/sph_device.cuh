// Device building blocks of the WCSPH step (arXiv 2110.02621, Sec. 2):
// typed per-run constants, the Wendland C2 kernel, the equations of state,
// rounding-exact drift/rebin helpers and the 27-cell neighbour walk.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sph {

constexpr uint32_t KEY_NONE = 0xFFFFFFFFu;
constexpr int BLOCK = 128;

// 4-vector of T with natural 4*sizeof(T) alignment (float4-like for both
// precisions; CUDA 13 deprecates the plain double4).
template <class T>
struct alignas(4 * sizeof(T)) V4 {
    T x, y, z, w;
};
template <class T>
struct alignas(2 * sizeof(T)) V2 {
    T x, y;
};

template <class T>
struct PhaseK {
    T rho0, inv_rho0;   // reference density and its inverse
    T mu;               // dynamic viscosity
    T m;                // particle mass rho0 dx^3 (also the wall mass seen by this phase)
    T eos_k;            // Tait: rho0 c^2 / gamma; linear: c^2
    T p_half;           // EOS(rho0 / 2): wall densities are kept at or above rho0 / 2
    int32_t eos, density, reinit, penalty;
};

// Per-run constants, passed by value to every kernel (constant bank).
template <class T>
struct Cfg {
    T h, rc2, cs;           // smoothing length, (2h)^2, cell side 2h
    T alpha, fcoef, W0;     // 21/(16 pi h^3), -5 alpha / h^2 (=F(r)/(1-q/2)^3), W(0)
    T inv_h;
    T c0, inv_c0, gamma, inv_gamma, gamma_p;
    T dp, dp3, inv_dp, eta2, pen_rmin;  // dx, dx^3, 1/dx, 0.01 h^2, 1e-6 dx
    T vol;                  // particle volume dx^3 (3-D) or dx^2 (2-D, per unit depth)
    T gx, gy, gz;
    T inv_sigma0;           // 1 / (lattice number density)
    T sigma0_hi, sigma0_lo; // lattice number density sigma^0 as an unevaluated sum
    T inv_vol_hi, inv_vol_lo;  // 1/vol likewise (summation-density reference)
    T cfl, body_dt;         // cfl, cfl*sqrt(h/(|g| + |amp| w^2)) (0 if both vanish)
    double g64[3];          // g in FP64 (for the body force of a moving tank)
    double ex_amp[3], ex_w; // rigid tank motion x = amp sin(w t), w = 2 pi f (Sec. 4.2)
    int32_t nx, ny, nz, n_cells;
    int32_t nf, nw;         // fluid and wall particle counts (index checks)
    int32_t periodic;       // bit d: axis d wraps (n_d cells of side cs make the period)
    int32_t n_phases;
    PhaseK<T> ph[2];
};

// ------------------------------------------------------------ index checks
// Debug build (-DSPH_CHECK): an index read from memory (a list entry, a cell
// key, a cell range, a sort slot) is checked before it addresses anything.
// One out of range sets a bit of the translation unit's check word and is
// replaced by 0, so the kernel carries on without a wild access; the host
// reads the word after each synchronising call and reports SPH_ERR_CUDA.
// Without the flag SPH_CK(i, n, bit) is i.
constexpr unsigned CK_FLIST = 1, CK_WLIST = 2, CK_CELL = 4, CK_RANGE = 8, CK_SLOT = 16;
#ifdef SPH_CHECK
static __device__ unsigned int g_sph_check;
__device__ __forceinline__ int32_t sph_ck(int32_t i, int32_t n, unsigned bit)
{
    if ((uint32_t)i < (uint32_t)n) return i;
    atomicOr(&g_sph_check, bit);
    return 0;
}
#define SPH_CK(i, n, bit) ::sph::sph_ck((i), (n), (bit))
#else
#define SPH_CK(i, n, bit) (i)
#endif

// ---------------------------------------------------------------- rounding
// The drift is evaluated twice (when counting cells and when moving the
// particle): explicit round-to-nearest intrinsics keep the two bit-identical.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ float f_floor(float x) { return floorf(x); }
__device__ __forceinline__ double f_floor(double x) { return floor(x); }
__device__ __forceinline__ float f_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double f_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float f_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double f_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float f_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double f_log1p(double x) { return log1p(x); }
__device__ __forceinline__ bool f_finite(float x) { return isfinite(x); }
__device__ __forceinline__ bool f_finite(double x) { return isfinite(x); }

// Pair-loop division and distance.  FP32: the hardware reciprocal-based
// quotient (__fdividef, at most 2 ulp for divisors in the normal range) and
// r = r^2 rsqrt(r^2) (rsqrt at most 2 ulp): relative errors of ~2.4e-7, far
// inside the 2e-5 tolerance of the sums, at a fraction of the instruction
// count of the IEEE sequences.  FP64: IEEE division and square root.
__device__ __forceinline__ float p_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double p_div(double a, double b) { return a / b; }
__device__ __forceinline__ float p_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double p_rsqrt(double x) { return 1.0 / sqrt(x); }

// Kahan-compensated drift of one coordinate, o += dt v (FP32 form).  In the
// FP64 form the compensation is not needed and stays zero.
template <class T, bool KAHAN>
__device__ __forceinline__ void drift1(T& o, T& comp, T dt, T v)
{
    if (KAHAN) {
        T y = fma_rn(dt, v, -comp);
        T t = add_rn(o, y);
        comp = sub_rn(sub_rn(t, o), y);
        o = t;
    } else {
        o = fma_rn(dt, v, o);
    }
}

// Move an offset back into [0, cs] and shift the cell index accordingly.
// Offsets already in the closed interval stay where they are: an offset of
// exactly cs (a particle on the upper face, as the FP64 binning at create
// can leave it) still has every pair within 2h inside its 27-cell stencil,
// while a negative offset would not.
template <class T>
__device__ __forceinline__ void rebin1(T& o, int32_t& c, T cs)
{
    if (o >= T(0) && o <= cs) return;
    T k = f_floor(o / cs);
    o = fma_rn(-k, cs, o);
    c += (int32_t)k;
    if (o < T(0)) { o = add_rn(o, cs); c -= 1; }
    if (o > cs) { o = sub_rn(o, cs); c += 1; }
}

// A cell index one step outside [0, n) along a periodic axis wraps around.
__device__ __forceinline__ int32_t wrap_cell(int32_t c, int32_t n)
{
    return c < 0 ? c + n : (c >= n ? c - n : c);
}

template <class T>
__device__ __forceinline__ uint32_t cell_key(const Cfg<T>& C, int32_t cx, int32_t cy, int32_t cz)
{
    if (cx < 0 || cy < 0 || cz < 0 || cx >= C.nx || cy >= C.ny || cz >= C.nz) return KEY_NONE;
    return (uint32_t)((cz * C.ny + cy) * C.nx + cx);
}

// ------------------------------------------------------- Wendland C2, 3-D
// W = alpha (1 - q/2)^4 (2q + 1), q = r/h; F = (dW/dr)/r = -5 alpha (1-q/2)^3/h^2.
template <class T>
__device__ __forceinline__ void kernel_WF(const Cfg<T>& C, T r, T& W, T& F)
{
    T q = r * C.inv_h;
    T t = T(1) - T(0.5) * q;
    T t3 = t * t * t;
    F = C.fcoef * t3;
    W = C.alpha * t3 * t * (T(2) * q + T(1));
}
template <class T>
__device__ __forceinline__ T kernel_F(const Cfg<T>& C, T r)
{
    T t = T(1) - T(0.5) * (r * C.inv_h);
    return C.fcoef * t * t * t;
}
template <class T>
__device__ __forceinline__ T kernel_W(const Cfg<T>& C, T r)
{
    T q = r * C.inv_h;
    T t = T(1) - T(0.5) * q;
    T t2 = t * t;
    return C.alpha * t2 * t2 * (T(2) * q + T(1));
}

// ------------------------------------------------------- equation of state
// Pressure from the density excess drho = rho - rho0 (kept instead of rho to
// avoid cancellation in FP32).  Linear: Eq. (EoS); Tait written as
// rho0 c^2/gamma * expm1(gamma log1p(drho/rho0)).
template <class T>
__device__ __forceinline__ T eos_p(const PhaseK<T>& P, const Cfg<T>& C, T drho)
{
    if (P.eos == 1) return P.eos_k * f_expm1(C.gamma * f_log1p(drho * P.inv_rho0));
    return P.eos_k * drho;
}
// density excess from pressure (inverse EOS), for wall dummy particles
template <class T>
__device__ __forceinline__ T eos_drho(const PhaseK<T>& P, const Cfg<T>& C, T p)
{
    if (P.eos == 1) return P.rho0 * f_expm1(C.inv_gamma * f_log1p(p / P.eos_k));
    return p / P.eos_k;
}

// ------------------------------------------------------- neighbour walk
// Visits every particle of the (up to) 27 cells around cell (cx, cy, cz) of
// a sorted set with cell ranges start[], passing its sorted index j and the
// shift d*cs such that r_ij = o_i - o_j - shift (cells wrap along periodic
// axes; the shift is the geometric one, so r_ij is the nearest image).
template <class T, class Fn>
__device__ __forceinline__ void for_cells27(const Cfg<T>& C, int32_t cx, int32_t cy, int32_t cz,
                                            const int32_t* __restrict__ start, Fn&& fn)
{
    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        if (z < 0 || z >= C.nz) {
            if (!(C.periodic & 4)) continue;
            z = wrap_cell(z, C.nz);
        }
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            if (y < 0 || y >= C.ny) {
                if (!(C.periodic & 2)) continue;
                y = wrap_cell(y, C.ny);
            }
            int row = (z * C.ny + y) * C.nx;
            for (int dx = -1; dx <= 1; ++dx) {
                int x = cx + dx;
                if (x < 0 || x >= C.nx) {
                    if (!(C.periodic & 1)) continue;
                    x = wrap_cell(x, C.nx);
                }
                int c = row + x;
                int b = __ldg(start + c), e = __ldg(start + c + 1);
                T sx = T(dx) * C.cs, sy = T(dy) * C.cs, sz = T(dz) * C.cs;
                for (int j = b; j < e; ++j) fn(j, sx, sy, sz);
            }
        }
    }
}

}  // namespace sph
