// Pair sweeps of the step (Sec. 3, compartments a-c) over per-particle
// neighbour lists, with LP consecutive lanes per target particle.
//
// k_neighbors builds, once per step (after the re-binning, at the positions
// r^{n+1} that continuity and momentum share), each fluid particle's lists of
// fluid and wall neighbours with 0 < |r_ij| < 2h.  The 27 cells around a cell
// are 9 rows of 3 x-consecutive cells, each row one contiguous range of the
// sorted arrays.  The LP lanes of a particle split every row (lane l takes
// every LP-th candidate) and each keeps its own sub-list; neighbouring lane
// groups are consecutive sorted particles, mostly of the same cell, so their
// candidate loads are shared.  An entry is (j << 6) | (dx+1) | (dy+1) << 2 |
// (dz+1) << 4 with (dx, dy, dz) the cell of j relative to the cell of i (so
// j < 2^26); entry k of lane t = LP i + l is stored at k (LP n) + t
// (coalesced).  Builder and sweeps evaluate r_ij = (o_i - d cs) - o_j and its
// square with the same rounded operations, so they agree bit for bit on
// which pairs are within 2h.  The build also tags every wall particle with
// fluid support in this step (the pair test is symmetric).
//
// The continuity and momentum kernels run the same lane groups over the
// sub-lists and combine the LP partial sums with a fixed xor-shuffle tree
// (deterministic).  A lane whose sub-list overflowed scans its share of the
// 27 cells directly instead.
//
// The kernels and scans take PER = true for runs with periodic axes, so that
// the wrap-around code is compiled out of the others.
#pragma once

#include "sph_kernels.cuh"

namespace sph {

constexpr int LP = 4;        // lanes per target particle
constexpr int SUBF = 40;     // fluid entries per lane sub-list (about 80/LP used)
constexpr int SUBW = 24;     // wall entries per lane sub-list: a particle at a tank edge has up to
                             // ~60 wall neighbours, and one lane past its capacity sends the particle's
                             // sweeps to the cell scan (with 16, 4-6 particles of the 80 k dam break
                             // did, and their warps set the sweeps' length: 190.7 against 174.4 us)
constexpr int WLP = 8;       // lanes per wall particle in the wall-pressure sweep (WLP_LARGE from
constexpr int WLP_LARGE = 4; // WLP_LARGE_MIN wall particles on: measured faster at 0.36 M and 2.2 M walls,
constexpr int WLP_LARGE_MIN = 250000;  // slower at 0.12 M, where 4 lanes leave too few threads in flight
constexpr int AWLP = 4;      // lanes per wall particle in the adjoint's wall sweeps
constexpr int LBLOCK = 128;  // threads per block

__device__ __forceinline__ int code_of(int dx, int dy, int dz) { return (dx + 1) | (dy + 1) << 2 | (dz + 1) << 4; }

template <class T>
__device__ __forceinline__ void shift_of(const Cfg<T>& C, int e, T& sx, T& sy, T& sz)
{
    sx = T((e & 3) - 1) * C.cs;
    sy = T(((e >> 2) & 3) - 1) * C.cs;
    sz = T(((e >> 4) & 3) - 1) * C.cs;
}

// |r|^2 with a fixed rounding sequence (shared by builder and sweeps)
template <class T>
__device__ __forceinline__ T dist2(T x, T y, T z)
{
    return fma_rn(z, z, fma_rn(y, y, mul_rn(x, x)));
}

// Kahan-compensated accumulation; the sum is s - c.  Used for number
// densities, whose deviation from the lattice value is the signal.
// Every operation rounds on its own (the _rn intrinsics are never fused with
// the product that made x), so the sum has the same bits in every kernel that
// adds the same terms in the same order.
template <class T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T x)
{
    const T y = sub_rn(x, c);
    const T t = add_rn(s, y);
    c = sub_rn(sub_rn(t, s), y);
    s = t;
}

// (s - c) - (ref_hi + ref_lo) without cancellation: s - ref_hi is exact for
// s within a factor 2 of ref_hi (Sterbenz).
template <class T>
__device__ __forceinline__ T minus_ref(T s, T c, T ref_hi, T ref_lo)
{
    return (s - ref_hi) - (c + ref_lo);
}

// The G lanes of a particle (G = LP, WLP, WLP_LARGE or AWLP for wall particles)
// always take the same path (everything they branch on is per particle),
// while different groups of a warp may not: the group shuffles therefore
// name only the group's own lanes.
template <int G = LP>
__device__ __forceinline__ unsigned group_mask()
{
    return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
}

// sum over the G lanes of a group (fixed tree: deterministic)
template <int G = LP, class T>
__device__ __forceinline__ T group_sum(T v)
{
    const unsigned m = group_mask<G>();
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o, G);
    return v;
}

// merge the compensated sums (s - c) of the G lanes (TwoSum of the s parts)
template <int G = LP, class T>
__device__ __forceinline__ void group_kahan(T& s, T& c)
{
    const unsigned m = group_mask<G>();
    for (int o = G / 2; o > 0; o >>= 1) {
        const T s2 = __shfl_xor_sync(m, s, o, G);
        const T c2 = __shfl_xor_sync(m, c, o, G);
        const T t = s + s2;
        const T bp = t - s;
        const T err = (s - (t - bp)) + (s2 - bp);  // s + s2 = t + err exactly
        s = t;
        c = (c + c2) - err;
    }
}

// The y or z cell of a stencil row, wrapped along a periodic axis; false when
// it lies outside a non-periodic grid.
__device__ __forceinline__ bool row_axis(int32_t& v, int32_t n, bool periodic)
{
    if (v >= 0 && v < n) return true;
    if (!periodic) return false;
    v = wrap_cell(v, n);
    return true;
}

// One stencil row whose x-neighbour cells wrap around a periodic x (the
// target's cell is the first or last along x): its three cells are not one
// contiguous range, so each is scanned in turn; lane l of NL takes the
// candidates at positions l, l + NL, ... of the three cells' concatenation.
template <int NL, class T, class Fn>
__device__ __forceinline__ void scan_row_wrapped(const Cfg<T>& C, int row, int cx, const int32_t* __restrict__ start,
                                                 const V4<T>* __restrict__ pts, int l, T xl, T x0, T xr, T ys,
                                                 T zs, int cyz, Fn&& fn)
{
    const int cells[3] = {wrap_cell(cx - 1, C.nx), cx, wrap_cell(cx + 1, C.nx)};
    const T xs[3] = {xl, x0, xr};
    int v = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int e = __ldg(start + SPH_CK(row + cells[k] + 1, C.n_cells + 1, CK_CELL));
        const int b = SPH_CK(__ldg(start + row + cells[k]), e + 1, CK_RANGE);
#pragma unroll 1
        for (int j = b + ((l - v) % NL + NL) % NL; j < e; j += NL) {
            const V4<T> pj = pts[j];
            const T rx = xs[k] - pj.x, ry = ys - pj.y, rz = zs - pj.z;
            const T r2 = dist2(rx, ry, rz);
            if (r2 < C.rc2 && r2 > T(0)) fn(j, rx, ry, rz, r2, cyz | k);
        }
        v += e - b;
    }
}

// Lane l's share (every LP-th candidate) of the 27 cells around cell c of a
// sorted set with cell ranges start[]: fn(j, rx, ry, rz, r2, code) for every
// candidate with 0 < r^2 < (2h)^2, o = the target's offset, code = the
// 6-bit cell shift of j.
template <bool PER, class T, class Fn>
__device__ __forceinline__ void scan_share(const Cfg<T>& C, const int4& c, const V4<T>& o,
                                           const int32_t* __restrict__ start, const V4<T>* __restrict__ pts,
                                           int l, Fn&& fn)
{
    const int xa = c.x > 0 ? c.x - 1 : 0;
    const int xb = c.x + 1 < C.nx ? c.x + 1 : C.nx - 1;
    const T xl = o.x + C.cs, xr = o.x - C.cs;  // o_x - dx cs for dx = -1, +1
    // along a periodic x the first and last cells' rows wrap (not contiguous)
    const bool wrap_x = PER && (C.periodic & 1) && (c.x == 0 || c.x == C.nx - 1);
    for (int dz = -1; dz <= 1; ++dz) {
        int z = c.z + dz;
        if (!row_axis(z, C.nz, PER && (C.periodic & 4))) continue;
        const T zs = o.z - T(dz) * C.cs;
        for (int dy = -1; dy <= 1; ++dy) {
            int y = c.y + dy;
            if (!row_axis(y, C.ny, PER && (C.periodic & 2))) continue;
            const T ys = o.y - T(dy) * C.cs;
            const int row = (z * C.ny + y) * C.nx;
            const int cyz = (dy + 1) << 2 | (dz + 1) << 4;
            if (wrap_x) {
                scan_row_wrapped<LP>(C, row, c.x, start, pts, l, xl, o.x, xr, ys, zs, cyz, fn);
                continue;
            }
            const int rb = SPH_CK(row + xa, C.n_cells, CK_CELL), re = SPH_CK(row + xb + 1, C.n_cells + 1, CK_CELL);
            const int e = __ldg(start + re), b = SPH_CK(__ldg(start + rb), e + 1, CK_RANGE);
            const int b1 = __ldg(start + row + c.x), b2 = __ldg(start + row + c.x + 1);
#pragma unroll 4
            for (int j = b + l; j < e; j += LP) {
                const V4<T> pj = pts[j];
                const int dxc = j < b1 ? 0 : (j < b2 ? 1 : 2);  // dx + 1
                const T rx = (dxc == 0 ? xl : (dxc == 1 ? o.x : xr)) - pj.x;
                const T ry = ys - pj.y, rz = zs - pj.z;
                const T r2 = dist2(rx, ry, rz);
                if (r2 < C.rc2 && r2 > T(0)) fn(j, rx, ry, rz, r2, cyz | dxc);
            }
        }
    }
}

// scan_share for the list builder: each row's three cells in turn with a
// constant x shift (fewer instructions per candidate; larger code).
// Lane l's share (every LP-th candidate) of the 27 cells around cell c of a
// sorted set with cell ranges start[]: fn(j, code, hit) for every
// candidate, hit = (0 < r^2 < (2h)^2), o = the target's offset, code = the
// 6-bit cell shift of j.  The callback runs for every candidate, so that the
// builder records hits with predicated instructions instead of a branch.
// Only the rows whose bit (dz + 1) 3 + (dy + 1) is set in rows are walked.
template <bool PER, class T, class Fn>
__device__ __forceinline__ void scan_rows(const Cfg<T>& C, const int4& c, const V4<T>& o,
                                           const int32_t* __restrict__ start, const V4<T>* __restrict__ pts,
                                           int l, Fn&& fn, unsigned rows = 0x1ffu)
{
    const int xa = c.x > 0 ? c.x - 1 : 0;
    const int xb = c.x + 1 < C.nx ? c.x + 1 : C.nx - 1;
    const T xl = o.x + C.cs, xr = o.x - C.cs;  // o_x - dx cs for dx = -1, +1
    // along a periodic x the first and last cells' rows wrap (not contiguous)
    const bool wrap_x = PER && (C.periodic & 1) && (c.x == 0 || c.x == C.nx - 1);
    for (int dz = -1; dz <= 1; ++dz) {
        int z = c.z + dz;
        if (!row_axis(z, C.nz, PER && (C.periodic & 4))) continue;
        const T zs = o.z - T(dz) * C.cs;
        for (int dy = -1; dy <= 1; ++dy) {
            if (!((rows >> ((dz + 1) * 3 + dy + 1)) & 1u)) continue;
            int y = c.y + dy;
            if (!row_axis(y, C.ny, PER && (C.periodic & 2))) continue;
            const T ys = o.y - T(dy) * C.cs;
            const int row = (z * C.ny + y) * C.nx;
            const int cyz = (dy + 1) << 2 | (dz + 1) << 4;
            if (wrap_x) {
                scan_row_wrapped<LP>(C, row, c.x, start, pts, l, xl, o.x, xr, ys, zs, cyz,
                                     [&](int j, T, T, T, T, int code) { fn(j, code, true); });
                continue;
            }
            const int rb = SPH_CK(row + xa, C.n_cells, CK_CELL), re = SPH_CK(row + xb + 1, C.n_cells + 1, CK_CELL);
            const int e = __ldg(start + re), b = SPH_CK(__ldg(start + rb), e + 1, CK_RANGE);
            const int b1 = __ldg(start + row + c.x), b2 = __ldg(start + row + c.x + 1);
            // the row's three cells in turn, each with its constant x shift;
            // j runs on across them, so the lanes' shares stay interleaved
            int j = b + l;
            auto segment = [&](int end, T xs, int code) {
#pragma unroll 4
                for (; j < end; j += LP) {
                    const V4<T> pj = pts[j];
                    const T rx = xs - pj.x, ry = ys - pj.y, rz = zs - pj.z;
                    const T r2 = dist2(rx, ry, rz);
                    fn(j, code, r2 < C.rc2 && r2 > T(0));
                }
            };
            segment(b1, xl, cyz);
            segment(b2, o.x, cyz | 1);
            segment(e, xr, cyz | 2);
        }
    }
}

// The same candidates as scan_share in a compact loop (one loop per row, the
// x shift chosen per candidate, no unrolling), lane l of NL taking every NL-th
// candidate: for the rare fall-back scans of over-full sub-lists and for the
// per-wall kernels, where code size and registers matter more than the last
// instruction per candidate.
template <bool PER, int NL = LP, class T, class Fn>
__device__ __forceinline__ void scan_compact(const Cfg<T>& C, const int4& c, const V4<T>& o,
                                             const int32_t* __restrict__ start, const V4<T>* __restrict__ pts,
                                             int l, Fn&& fn)
{
    const int xa = c.x > 0 ? c.x - 1 : 0;
    const int xb = c.x + 1 < C.nx ? c.x + 1 : C.nx - 1;
    const T xl = o.x + C.cs, xr = o.x - C.cs;
    // along a periodic x the first and last cells' rows wrap (not contiguous)
    const bool wrap_x = PER && (C.periodic & 1) && (c.x == 0 || c.x == C.nx - 1);
    for (int dz = -1; dz <= 1; ++dz) {
        int z = c.z + dz;
        if (!row_axis(z, C.nz, PER && (C.periodic & 4))) continue;
        const T zs = o.z - T(dz) * C.cs;
        for (int dy = -1; dy <= 1; ++dy) {
            int y = c.y + dy;
            if (!row_axis(y, C.ny, PER && (C.periodic & 2))) continue;
            const T ys = o.y - T(dy) * C.cs;
            const int row = (z * C.ny + y) * C.nx;
            const int cyz = (dy + 1) << 2 | (dz + 1) << 4;
            if (wrap_x) {
                scan_row_wrapped<NL>(C, row, c.x, start, pts, l, xl, o.x, xr, ys, zs, cyz, fn);
                continue;
            }
            const int rb = SPH_CK(row + xa, C.n_cells, CK_CELL), re = SPH_CK(row + xb + 1, C.n_cells + 1, CK_CELL);
            const int e = __ldg(start + re), b = SPH_CK(__ldg(start + rb), e + 1, CK_RANGE);
            const int b1 = __ldg(start + row + c.x), b2 = __ldg(start + row + c.x + 1);
#pragma unroll 1
            for (int j = b + l; j < e; j += NL) {
                const V4<T> pj = pts[j];
                const int dxc = j < b1 ? 0 : (j < b2 ? 1 : 2);  // dx + 1
                const T rx = (dxc == 0 ? xl : (dxc == 1 ? o.x : xr)) - pj.x;
                const T ry = ys - pj.y, rz = zs - pj.z;
                const T r2 = dist2(rx, ry, rz);
                if (r2 < C.rc2 && r2 > T(0)) fn(j, rx, ry, rz, r2, cyz | dxc);
            }
        }
    }
}

// Which of the 9 stencil rows around each cell hold wall particles: bit
// (dz + 1) 3 + (dy + 1) of rows[k] is set when the cells of that row that
// scan_rows walks (clamped to the grid, or wrapped along periodic axes) hold
// any.  The walls are fixed, so this runs once, after they are binned; the
// neighbour build then skips the empty wall rows, which are all nine for a
// cell inside the fluid.
template <bool PER, class T>
__global__ void k_wall_rows(Cfg<T> C, int32_t n_cells, const int32_t* __restrict__ wstart,
                            uint16_t* __restrict__ rows)
{
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_cells) return;
    const int32_t cx = k % C.nx, cy = (k / C.nx) % C.ny, cz = k / C.nx / C.ny;
    const int xa = cx > 0 ? cx - 1 : 0;
    const int xb = cx + 1 < C.nx ? cx + 1 : C.nx - 1;
    const bool wrap_x = PER && (C.periodic & 1) && (cx == 0 || cx == C.nx - 1);
    unsigned m = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        if (!row_axis(z, C.nz, PER && (C.periodic & 4))) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            if (!row_axis(y, C.ny, PER && (C.periodic & 2))) continue;
            const int row = (z * C.ny + y) * C.nx;
            bool any = false;
            if (wrap_x) {
                for (int dx = -1; dx <= 1; ++dx) {
                    const int x = wrap_cell(cx + dx, C.nx);
                    any |= wstart[row + x + 1] > wstart[row + x];
                }
            } else {
                any = wstart[row + xb + 1] > wstart[row + xa];
            }
            if (any) m |= 1u << ((dz + 1) * 3 + dy + 1);
        }
    }
    rows[k] = (uint16_t)m;
}

// --------------------------------------------------------- neighbour lists
// Evens out the LP sub-lists of one particle.  The build gives lane l every
// LP-th candidate, so the lanes' hit counts c_l scatter around N/LP, and a
// sweep's warp walks as many entries as its longest sub-list.  Here lane l
// keeps q_l = (N + LP - 1 - l) / LP entries: each lane with c_l > q_l moves
// its last c_l - q_l entries to the ends of the short sub-lists (excess and
// room both ranked in lane order, so the moves are fixed).  Entries stay
// what they were, only their lane changes.  A particle whose sub-list
// overflowed (some c_l > CAP, entries missing) keeps its counts: its sweeps
// fall back to the cell scan, whose lane shares are the build's.  col points
// at lane 0's column of the particle (entry k of lane l at k stride + l).
// Called by all LP lanes of the group; returns lane l's count.
template <int CAP>
__device__ __forceinline__ int balance_lists(int32_t* __restrict__ col, uint32_t stride, int l, int cnt)
{
    const unsigned m = group_mask<LP>();
    int c[LP], q[LP];
    int N = 0;
    bool over = false;
#pragma unroll
    for (int k = 0; k < LP; ++k) {
        c[k] = __shfl_sync(m, cnt, k, LP);
        N += c[k];
        over |= c[k] > CAP;
    }
    if (over) return cnt;
    int before = 0;  // excess of the lanes before l
#pragma unroll
    for (int k = 0; k < LP; ++k) {
        q[k] = (N + LP - 1 - k) / LP;
        if (k < l) before += c[k] > q[k] ? c[k] - q[k] : 0;
    }
    const int ql = (N + LP - 1 - l) / LP;  // q[l], c[l] = cnt (no indexed access)
    // four entries at a time: their loads are issued before any store
    constexpr int CH = 4;
    for (int r0 = 0; r0 < cnt - ql; r0 += CH) {
        int32_t e[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if (r0 + u < cnt - ql) e[u] = col[(size_t)(uint32_t)(ql + r0 + u) * stride + l];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            if (r0 + u >= cnt - ql) break;
            const int g = before + r0 + u;  // rank of this entry among all moved ones
            int acc = 0;
#pragma unroll
            for (int d = 0; d < LP; ++d) {
                const int room = q[d] > c[d] ? q[d] - c[d] : 0;
                if (g >= acc && g < acc + room) col[(size_t)(uint32_t)(c[d] + g - acc) * stride + d] = e[u];
                acc += room;
            }
        }
    }
    return ql;
}

// Ten blocks per SM (48 registers): measured 64.3 against 65.7 us at 80 k
// particles and 5.33 against 5.66 ms at 10.35 M without the bound.
template <class T, bool PER>
__global__ void __launch_bounds__(LBLOCK, 10) k_neighbors(
    Cfg<T> C, int32_t n, const int32_t* __restrict__ fstart, const int32_t* __restrict__ wstart,
    const uint16_t* __restrict__ wrows, const V4<T>* __restrict__ pos, const V4<T>* __restrict__ wpos,
    const int4* __restrict__ cell, int32_t* __restrict__ nbf, int32_t* __restrict__ nbw,
    int32_t* __restrict__ cnt, int32_t* __restrict__ wtag, const int32_t* __restrict__ d_tag)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / LP, l = t % LP;
    if (i >= n) return;
    const int4 c = cell[i];
    int nf = 0, nw = 0;
    if (c.w >= 0) {
        const V4<T> o = pos[i];
        const int tag = *d_tag;
        const uint32_t stride = (uint32_t)n * LP;
        // entry k of this lane's sub-list sits at k stride (one wide
        // multiply-add per store)
        int32_t* const qf = nbf + t;
        int32_t* const qw = nbw + t;
        scan_rows<PER>(C, c, o, fstart, pos, l, [&](int j, int code, bool hit) {
            if (hit && nf < SUBF) qf[(size_t)(uint32_t)nf * stride] = (j << 6) | code;
            nf += hit;
        });
        const unsigned wr = __ldg(wrows + SPH_CK(c.w, C.n_cells, CK_CELL));
        if (wr)
            scan_rows<PER>(
                C, c, o, wstart, wpos, l,
                [&](int w, int code, bool hit) {
                    if (hit && nw < SUBW) qw[(size_t)(uint32_t)nw * stride] = (w << 6) | code;
                    if (hit) wtag[w] = tag;
                    nw += hit;
                },
                wr);
        nf = balance_lists<SUBF>(nbf + (size_t)LP * i, stride, l, nf);
        nw = balance_lists<SUBW>(nbw + (size_t)LP * i, stride, l, nw);
    }
    cnt[t] = nf | (nw << 16);
}

// Visits lane l's neighbours of particle i: its sub-list entries, or, for an
// over-full sub-list, its share of the 27 cells.
// ff(j, p_j, rx, ry, rz, r2) for fluid, fw(w, p_w, rx, ry, rz, r2) for walls.
template <bool PER, class T, class FF, class FW>
__device__ __forceinline__ void for_neighbors(const Cfg<T>& C, int32_t n, int t, const V4<T>& pi, const int4& c,
                                              const int32_t* __restrict__ nbf, const int32_t* __restrict__ nbw,
                                              int32_t count, const int32_t* __restrict__ fstart,
                                              const int32_t* __restrict__ wstart, const V4<T>* __restrict__ pos,
                                              const V4<T>* __restrict__ wpos, FF&& ff, FW&& fw)
{
    const int nf = count & 0xffff, nw = count >> 16;
    const size_t stride = (size_t)n * LP;
    if (nf <= SUBF) {
        size_t at = t;
#pragma unroll 4
        for (int k = 0; k < nf; ++k, at += stride) {
            const int e = __ldg(nbf + at);
            T sx, sy, sz;
            shift_of(C, e, sx, sy, sz);
            const int j = SPH_CK(e >> 6, C.nf, CK_FLIST);
            const V4<T> pj = pos[j];
            const T rx = (pi.x - sx) - pj.x, ry = (pi.y - sy) - pj.y, rz = (pi.z - sz) - pj.z;
            ff(j, pj, rx, ry, rz, dist2(rx, ry, rz));
        }
    } else {
        scan_share<PER>(C, c, pi, fstart, pos, t % LP,
                   [&](int j, T rx, T ry, T rz, T r2, int) { ff(j, pos[j], rx, ry, rz, r2); });
    }
    if (nw <= SUBW) {
        size_t at = t;
#pragma unroll 2
        for (int k = 0; k < nw; ++k, at += stride) {
            const int e = __ldg(nbw + at);
            T sx, sy, sz;
            shift_of(C, e, sx, sy, sz);
            const int w = SPH_CK(e >> 6, C.nw, CK_WLIST);
            const V4<T> pw = wpos[w];
            const T rx = (pi.x - sx) - pw.x, ry = (pi.y - sy) - pw.y, rz = (pi.z - sz) - pw.z;
            fw(w, pw, rx, ry, rz, dist2(rx, ry, rz));
        }
    } else {
        scan_share<PER>(C, c, pi, wstart, wpos, t % LP,
                   [&](int w, T rx, T ry, T rz, T r2, int) { fw(w, wpos[w], rx, ry, rz, r2); });
    }
}

// ------------------------------------------------- neighbour-set export
// The neighbour sets the continuity and momentum sweeps visit, for the
// inspection call sph_get_neighbors: each lane walks its share through
// for_neighbors, the sweeps' own iterator (its sub-list, or its share of the
// 27 cells after an overflow).  k_nb_count writes lane t's fluid and wall
// counts to lc[t] and lc[LP n + t] and counts the particles whose fluid or
// wall lists overflowed (lane 0 of each particle checks its group);
// k_nb_fill then writes the neighbours' original ids from the lanes'
// offsets (an exclusive scan of the counts, in sorted lane order).
template <class T, bool PER>
__global__ void __launch_bounds__(LBLOCK) k_nb_count(
    Cfg<T> C, int32_t n, const int32_t* __restrict__ fstart, const int32_t* __restrict__ wstart,
    const int32_t* __restrict__ nbf, const int32_t* __restrict__ nbw, const int32_t* __restrict__ cnt,
    const V4<T>* __restrict__ pos, const V4<T>* __restrict__ wpos, const int4* __restrict__ cell,
    int32_t* __restrict__ lc, unsigned long long* overflow)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / LP;
    if (i >= n) return;
    const int4 c = cell[i];
    int nf = 0, nw = 0;
    if (c.w >= 0) {
        const int32_t k = cnt[t];
        for_neighbors<PER>(C, n, t, pos[i], c, nbf, nbw, k, fstart, wstart, pos, wpos,
                           [&](int, const V4<T>&, T, T, T, T) { ++nf; },
                           [&](int, const V4<T>&, T, T, T, T) { ++nw; });
        if (t % LP == 0) {
            bool of = false, ow = false;
            for (int l = 0; l < LP; ++l) {
                of |= (cnt[t + l] & 0xffff) > SUBF;
                ow |= (cnt[t + l] >> 16) > SUBW;
            }
            if (of) atomicAdd(overflow, 1ull);
            if (ow) atomicAdd(overflow + 1, 1ull);
        }
    }
    lc[t] = nf;
    lc[(size_t)LP * n + t] = nw;
}

template <class T, bool PER>
__global__ void __launch_bounds__(LBLOCK) k_nb_fill(
    Cfg<T> C, int32_t n, const int32_t* __restrict__ fstart, const int32_t* __restrict__ wstart,
    const int32_t* __restrict__ nbf, const int32_t* __restrict__ nbw, const int32_t* __restrict__ cnt,
    const V4<T>* __restrict__ pos, const V4<T>* __restrict__ wpos, const int4* __restrict__ cell,
    const int32_t* __restrict__ id, const int32_t* __restrict__ wid, const int64_t* __restrict__ off,
    int32_t* __restrict__ out_f, int32_t* __restrict__ out_w)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / LP;
    if (i >= n) return;
    const int4 c = cell[i];
    if (c.w < 0) return;
    int64_t af = off[t], aw = off[(size_t)LP * n + t];
    for_neighbors<PER>(C, n, t, pos[i], c, nbf, nbw, cnt[t], fstart, wstart, pos, wpos,
                       [&](int j, const V4<T>&, T, T, T, T) { out_f[af++] = id[j]; },
                       [&](int w, const V4<T>&, T, T, T, T) { out_w[aw++] = wid[w]; });
}

// ------------------------------------------------------------- continuity
// Heavy (continuity) phases: Eq. (SPH_star_massConservation) with the
// Riemann solution of Eq. (RSsolution).  Substituting v* gives, per pair,
//   (m_j/rho_j)(v_i - v*).grad_i W_ij
//      = m_j F [v_ij.r_ij + (p_i - p_j) r/(c rho_j)] / (rho_i + rho_j)
// with grad_i W_ij = F r_ij, F = (dW/dr)/r; walls enter with v_w = 0,
// (rho_w, p_w) and m_w = m_i.  Then rho^{n+1} = rho^n + dt d rho/dt (Sec. 2.6).
// Light (summation) phases: Eq. (densitySummation), rho = m sum_j W_ij over
// all particles and walls, self included, evaluated as
// rho - rho0 = rho0 vol (sum_j W_ij - 1/vol), vol = dx^3 (dx^2 in 2-D), with a
// compensated sum.  The
// EOS then gives p^{n+1}.  Particles outside the grid keep their state and
// get a = 0 (their momentum outputs are written here: nobody reads them).
template <class T, bool PER>
__global__ void __launch_bounds__(LBLOCK) k_continuity(
    Cfg<T> C, int32_t n, const int32_t* __restrict__ fstart, const int32_t* __restrict__ wstart,
    const int32_t* __restrict__ nbf, const int32_t* __restrict__ nbw, const int32_t* __restrict__ cnt,
    const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel, const T* __restrict__ drho,
    const int4* __restrict__ cell, const int32_t* __restrict__ phase,
    const V4<T>* __restrict__ wpos, const V2<T>* __restrict__ wrho, const T* __restrict__ d_dt,
    V4<T>* __restrict__ pos_o, V4<T>* __restrict__ vel_o, T* __restrict__ drho_o,
    V4<T>* __restrict__ acc_o, T* __restrict__ dsig_o)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / LP;
    const bool lead = (t % LP) == 0;
    if (i >= n) return;  // whole lane groups: n * LP threads are live
    const V4<T> pi = pos[i], vi = vel[i];
    const int4 c = cell[i];
    T d = drho[i];
    if (c.w < 0) {
        if (lead) {
            pos_o[i] = pi;
            vel_o[i] = vi;
            drho_o[i] = d;
            acc_o[i] = V4<T>{T(0), T(0), T(0), T(0)};
            dsig_o[i] = T(0);
        }
        return;
    }
    const int ph = phase[i];
    const PhaseK<T>& P = C.ph[ph];
    const T rho_i = vi.w, p_i = pi.w;
    const bool multi = C.n_phases > 1;
    T drdt = T(0);
    if (P.density == 1) {
        T s = lead ? C.W0 : T(0), e = T(0);
        for_neighbors<PER>(C, n, t, pi, c, nbf, nbw, cnt[t], fstart, wstart, pos, wpos,
                      [&](int, const V4<T>&, T, T, T, T r2) { kahan_add(s, e, kernel_W(C, r2 * p_rsqrt(r2))); },
                      [&](int, const V4<T>&, T, T, T, T r2) { kahan_add(s, e, kernel_W(C, r2 * p_rsqrt(r2))); });
        group_kahan(s, e);
        d = P.rho0 * C.vol * minus_ref(s, e, C.inv_vol_hi, C.inv_vol_lo);
    } else {
        T s = T(0);
        const T kc = C.inv_c0;
        for_neighbors<PER>(
            C, n, t, pi, c, nbf, nbw, cnt[t], fstart, wstart, pos, wpos,
            [&](int j, const V4<T>& pj, T rx, T ry, T rz, T r2) {
                const V4<T> vj = vel[j];
                const T r = r2 * p_rsqrt(r2);
                const T F = kernel_F(C, r);
                const T m_j = multi ? C.ph[phase[j]].m : P.m;
                const T rv = rx * (vi.x - vj.x) + ry * (vi.y - vj.y) + rz * (vi.z - vj.z);
                s += m_j * F * p_div(rv + p_div((p_i - pj.w) * r * kc, vj.w), rho_i + vj.w);
            },
            [&](int w, const V4<T>& pw, T rx, T ry, T rz, T r2) {
                const V2<T> rw = wrho[w];
                const T rho_w = ph == 0 ? rw.x : rw.y;
                const T r = r2 * p_rsqrt(r2);
                const T F = kernel_F(C, r);
                const T rv = rx * vi.x + ry * vi.y + rz * vi.z;
                s += P.m * F * p_div(rv + p_div((p_i - pw.w) * r * kc, rho_w), rho_i + rho_w);
            });
        drdt = T(2) * rho_i * group_sum(s);
        d = d + (*d_dt) * drdt;
    }
    if (lead) {
        pos_o[i] = V4<T>{pi.x, pi.y, pi.z, eos_p(P, C, d)};
        vel_o[i] = V4<T>{vi.x, vi.y, vi.z, P.rho0 + d};
        drho_o[i] = d;
        acc_o[i] = V4<T>{T(0), T(0), T(0), drdt};
    }
}

// ----------------------------------------------------------- wall pressure
// Wall dummy density of a phase from the wall pressure, rho_w = EOS^-1(p_w)
// (Sec. 2.3), kept at or above rho0/2: below EOS(rho0/2) -- reached only
// where the extrapolation averages fluid torn to half its density -- the
// inverse would approach (Tait: leave) the edge of its domain, p > -rho0 c^2/gamma.
template <class T>
__device__ __forceinline__ T wall_density(const PhaseK<T>& P, const Cfg<T>& C, T p_w)
{
    return p_w < P.p_half ? T(0.5) * P.rho0 : P.rho0 + eos_drho(P, C, p_w);
}

// Eq. (wallPressure) with fixed walls (a_w = 0), reading the (g - a_w) term
// with the fluid density (dimensionally consistent form):
//   p_w = sum_f (p_f + rho_f g.r_wf) w_wf / sum_f w_wf,  r_wf = r_w - r_f,
// w = W (one phase) or W/rho_f (several phases, Sec. 2.3).  Walls without
// fluid support (not tagged by this step's neighbour build) get p_w = 0 and
// rho_w = rho0 at once; the others split the fluid of their 27 cells over G
// lanes.  rho_w = rho0 + EOS^-1(p_w) per phase, at least rho0/2.
// The same scan marks the wall particles through which the penalty acts
// (wnrm.w = 1, else 0): some fluid of the support lies on the side n_w
// points to.
template <class T, bool PER, int G = WLP>
__global__ void __launch_bounds__(LBLOCK) k_wall_pressure(
    Cfg<T> C, int32_t nw, const int32_t* __restrict__ fstart, V4<T>* __restrict__ wpos,
    const int4* __restrict__ wcell, const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel,
    V2<T>* __restrict__ wrho, const int32_t* __restrict__ wtag, const int32_t* __restrict__ d_tag,
    const V4<T>* __restrict__ geff, unsigned long long* active, V4<T>* __restrict__ wnrm)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = t / G;
    int has = 0;
    if (w < nw) {
        const bool multi = C.n_phases > 1;
        T num = T(0), den = T(0);
        bool front = false;
        if (wtag[w] == *d_tag) {
            const V4<T> ge = *geff;
            const int4 c = wcell[w];
            const V4<T> pw = wpos[w];
            const V4<T> nn = wnrm[w];
            scan_compact<PER, G>(C, c, pw, fstart, pos, t % G, [&](int j, T rx, T ry, T rz, T r2, int) {
                const T W = kernel_W(C, r2 * p_rsqrt(r2));
                const T p_f = reinterpret_cast<const T*>(pos + j)[3];
                const T rho_f = vel[j].w;
                const T om = multi ? p_div(W, rho_f) : W;
                num += (p_f + rho_f * (ge.x * rx + ge.y * ry + ge.z * rz)) * om;
                den += om;
                front |= rx * nn.x + ry * nn.y + rz * nn.z < T(0);  // (r_f - r_w).n_w > 0
            });
            num = group_sum<G>(num);
            den = group_sum<G>(den);
            front = (__ballot_sync(group_mask<G>(), front) & group_mask<G>()) != 0u;
        }
        if (t % G == 0) {
            const T p_w = den > T(0) ? num / den : T(0);
            has = den > T(0);
            reinterpret_cast<T*>(wpos + w)[3] = p_w;
            reinterpret_cast<T*>(wnrm + w)[3] = front ? T(1) : T(0);
            const T r0 = wall_density(C.ph[0], C, p_w);
            const T r1 = multi ? wall_density(C.ph[1], C, p_w) : r0;
            wrho[w] = V2<T>{r0, r1};
        }
    }
    // walls with support, counted per warp (no block barrier: a warp whose
    // walls had no support leaves at once)
    const unsigned bal = __ballot_sync(0xffffffffu, has);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(active, (unsigned long long)__popc(bal));
}

// --------------------------------------------------------------- momentum
// Eq. (SPH_star_momentumConservation) with p* from Eq. (RSsolution) (fluid)
// or Eq. (RSatWall) (wall); per pair -2 m_j p*/(rho_i rho_j) F r_ij, where
//   p*/(rho_i rho_j) = (p_i/rho_i + p_j/rho_j + beta dU)/(rho_i + rho_j),
//   dU = U_L - U_R = -v_ij.r_ij/r, beta = min(3 max(dU, 0), c).
// Plus the body force (g, or g + amp w^2 sin(w t) in a moving tank's frame),
// the Morris viscous term, and the penalty force of
// Eq. (SPH_penaltyMethodTerm) with the signed delta = 2 r_iw.n_w/dx (a
// barrier that keeps rising behind the wall particle's plane), lambda from
// Eq. (symbc) and dx^3 restoring its units, through the wall particles with
// fluid on their normal's side (wnrm.w, set by k_wall_pressure).  Then the final kick
// v^{n+1} = v^{n+1/2} + dt/2 a^{n+1}, the number density sigma(r^{n+1}) for
// the next reinitialisation (own phase and walls for continuity phases,
// everything for summation phases; stored as sigma - sigma^0 from a
// compensated sum) and U_max for the next dt.
// SIG = false leaves sigma out (and dsig_o untouched): the number density is
// read only by the next step's reinitialisation, so steps before a step
// without one skip it (k_sigma gives it on demand, bit for bit the same).
template <class T, bool PER, bool SIG = true>
__global__ void __launch_bounds__(LBLOCK) k_momentum(
    Cfg<T> C, int32_t n, const int32_t* __restrict__ fstart, const int32_t* __restrict__ wstart,
    const int32_t* __restrict__ nbf, const int32_t* __restrict__ nbw, const int32_t* __restrict__ cnt,
    const V4<T>* __restrict__ pos, const V4<T>* __restrict__ vel, const int4* __restrict__ cell,
    const int32_t* __restrict__ phase, const V4<T>* __restrict__ wpos, const V2<T>* __restrict__ wrho,
    const V4<T>* __restrict__ wnrm, const T* __restrict__ d_dt, const V4<T>* __restrict__ geff,
    V4<T>* __restrict__ acc, V4<T>* __restrict__ vel_o, T* __restrict__ dsig_o, unsigned long long* vmax_bits,
    int32_t* flags)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / LP;
    const bool lead = (t % LP) == 0;
    T speed = T(0);
    bool bad = false;
    if (i < n) {
        const V4<T> pi = pos[i], vi = vel[i];
        const int4 c = cell[i];
        if (c.w >= 0) {  // particles outside the grid were finished by k_continuity
            const T hdt = T(0.5) * (*d_dt);
            const int ph = phase[i];
            const PhaseK<T>& P = C.ph[ph];
            const bool multi = C.n_phases > 1;
            const bool sig_all = P.density == 1;
            const T rho_i = vi.w, p_i = pi.w, pr_i = p_div(p_i, rho_i), mu_i = P.mu;
            T ax = T(0), ay = T(0), az = T(0), sg = lead ? C.W0 : T(0), se = T(0);
            auto fluid_pair = [&](int j, const V4<T>& pj, T rx, T ry, T rz, T r2) {
                    const V4<T> vj = vel[j];
                    const T rinv = p_rsqrt(r2);
                    const T r = r2 * rinv;
                    T W, F;
                    kernel_WF(C, r, W, F);
                    const int phj = multi ? phase[j] : 0;
                    const PhaseK<T>& Pj = C.ph[phj];
                    const T vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                    const T dU = -(rx * vx + ry * vy + rz * vz) * rinv;
                    const T beta = tmin(T(3) * tmax(dU, T(0)), C.c0);
                    const T coef = p_div(pr_i + p_div(pj.w, vj.w) + beta * dU, rho_i + vj.w);
                    const T k = T(-2) * Pj.m * F * coef;
                    const T mu = mu_i + Pj.mu;
                    if (mu > T(0)) {
                        const T kv = p_div(Pj.m * mu * r2 * F, rho_i * vj.w * (r2 + C.eta2));
                        ax += kv * vx;
                        ay += kv * vy;
                        az += kv * vz;
                    }
                    ax += k * rx;
                    ay += k * ry;
                    az += k * rz;
                    if (SIG && (sig_all || phj == ph)) kahan_add(sg, se, W);
                };
            auto wall_pair = [&](int w, const V4<T>& pw, T rx, T ry, T rz, T r2) {
                    const V2<T> rw = wrho[w];
                    const T rho_w = ph == 0 ? rw.x : rw.y;
                    const T rinv = p_rsqrt(r2);
                    const T r = r2 * rinv;
                    T W, F;
                    kernel_WF(C, r, W, F);
                    const T coef = p_div(pr_i + p_div(pw.w, rho_w), rho_i + rho_w);
                    const T k = T(-2) * P.m * F * coef;
                    ax += k * rx;
                    ay += k * ry;
                    az += k * rz;
                    if (mu_i > T(0)) {
                        const T kv = p_div(P.m * (T(2) * mu_i) * r2 * F, rho_i * rho_w * (r2 + C.eta2));
                        ax += kv * vi.x;
                        ay += kv * vi.y;
                        az += kv * vi.z;
                    }
                    if (P.penalty && r > C.pen_rmin) {
                        const V4<T> nw = wnrm[w];
                        const T rn = rx * nw.x + ry * nw.y + rz * nw.z;   // r_iw . n_w
                        const T delta = T(2) * rn * C.inv_dp;              // signed
                        if (delta < T(1) && nw.w != T(0)) {
                            const T en = -rn * rinv;                      // e_iw . n_w
                            const T lam = (T(1) - delta) * (T(1) - delta) * C.inv_dp;
                            const T Ppen = C.gamma_p * lam * tabs(p_i * en);
                            const T kp = T(-2) * p_div(P.m, rho_i * rho_w) * Ppen * C.dp3 * F * rinv;
                            ax += kp * nw.x;
                            ay += kp * nw.y;
                            az += kp * nw.z;
                        }
                    }
                    if (SIG) kahan_add(sg, se, W);
                };
            for_neighbors<PER>(C, n, t, pi, c, nbf, nbw, cnt[t], fstart, wstart, pos, wpos, fluid_pair, wall_pair);
            const V4<T> ge = *geff;
            ax = group_sum(ax) + ge.x;
            ay = group_sum(ay) + ge.y;
            az = group_sum(az) + ge.z;
            if (SIG) group_kahan(sg, se);
            const V4<T> vo{fma_rn(hdt, ax, vi.x), fma_rn(hdt, ay, vi.y), fma_rn(hdt, az, vi.z), rho_i};
            bad = !(f_finite(ax) && f_finite(ay) && f_finite(az));
            speed = f_sqrt(vo.x * vo.x + vo.y * vo.y + vo.z * vo.z);
            if (lead) {
                acc[i] = V4<T>{ax, ay, az, acc[i].w};
                vel_o[i] = vo;
                if (SIG) dsig_o[i] = minus_ref(sg, se, C.sigma0_hi, C.sigma0_lo);
            }
        }
    }
    // block maximum of |v| (non-negative: the integer order of the bits is
    // the order of the values) and the non-finite flag, one atomic per block
    __shared__ unsigned long long smax[LBLOCK / 32];
    unsigned long long b = to_bits(speed);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, b, o);
        b = q > b ? q : b;
    }
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = b;
    const int nbad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int k = 0; k < LBLOCK / 32; ++k) m = smax[k] > m ? smax[k] : m;
        if (m) atomicMax(vmax_bits, m);
        if (nbad) atomicOr(flags, 1);
    }
}

// sigma - sigma^0 of every particle at the positions of the current lists,
// for steps whose momentum sweep left it out: the same lanes, list walk,
// kernel values (kernel_WF), compensated sums and shuffle tree as
// k_momentum with SIG, so the result is the same bits.  Particles outside
// the grid get 0, as from k_continuity.
template <class T, bool PER>
__global__ void __launch_bounds__(LBLOCK) k_sigma(
    Cfg<T> C, int32_t n, const int32_t* __restrict__ fstart, const int32_t* __restrict__ wstart,
    const int32_t* __restrict__ nbf, const int32_t* __restrict__ nbw, const int32_t* __restrict__ cnt,
    const V4<T>* __restrict__ pos, const int4* __restrict__ cell, const int32_t* __restrict__ phase,
    const V4<T>* __restrict__ wpos, T* __restrict__ dsig_o)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / LP;
    const bool lead = (t % LP) == 0;
    if (i >= n) return;
    const int4 c = cell[i];
    if (c.w < 0) {
        if (lead) dsig_o[i] = T(0);
        return;
    }
    const int ph = phase[i];
    const bool multi = C.n_phases > 1;
    const bool sig_all = C.ph[ph].density == 1;
    T sg = lead ? C.W0 : T(0), se = T(0);
    for_neighbors<PER>(
        C, n, t, pos[i], c, nbf, nbw, cnt[t], fstart, wstart, pos, wpos,
        [&](int j, const V4<T>&, T, T, T, T r2) {
            const T r = r2 * p_rsqrt(r2);
            T W, F;
            kernel_WF(C, r, W, F);
            const int phj = multi ? phase[j] : 0;
            if (sig_all || phj == ph) kahan_add(sg, se, W);
        },
        [&](int, const V4<T>&, T, T, T, T r2) {
            const T r = r2 * p_rsqrt(r2);
            T W, F;
            kernel_WF(C, r, W, F);
            kahan_add(sg, se, W);
        });
    group_kahan(sg, se);
    if (lead) dsig_o[i] = minus_ref(sg, se, C.sigma0_hi, C.sigma0_lo);
}

}  // namespace sph
