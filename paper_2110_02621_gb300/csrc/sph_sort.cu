// Counting sort of particles by cell key (Sec. 3, "neighbour search
// including sorting"): exclusive scan of the per-cell counts, first
// placement by arrival rank, then the in-cell rank by particle id makes the
// final order (key, id) independent of atomic arrival order.  The scan is one
// block for short inputs, else a reduce / down-sweep pair of kernels in which
// each down-sweep block adds up the sums of the blocks before it, and for
// long inputs (more than SCAN_DIRECT blocks) a reduce / scan-of-sums /
// down-sweep; none has inter-block waits.  It can clear its input behind
// itself, so the step's cell counters are zero for the next step.
#include <cstdint>
#include <cstdio>

#include "sph_internal.h"
#include "sph_setup.cuh"

namespace sph {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 1024 values per block
constexpr int SCAN_DIRECT = 512;  // block counts up to which each down-sweep block sums its predecessors
constexpr int64_t SCAN_MAX = (int64_t)1 << 24;  // longest input

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* total)
{
    __shared__ int32_t warp_sums[SCAN_THREADS / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    int32_t before = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int32_t* __restrict__ in, int32_t n,
                                                              int32_t* __restrict__ sums)
{
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int32_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) s += in[base + k];
    int32_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one block: exclusive scan of the nb block sums, SCAN_TILE of them at a
// time with a running carry
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(int32_t* sums, int32_t nb)
{
    int32_t carry = 0;
    for (int c0 = 0; c0 < nb; c0 += SCAN_TILE) {
        const int base = c0 + threadIdx.x * SCAN_ITEMS;
        int32_t v[SCAN_ITEMS], s = 0;
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            v[k] = base + k < nb ? sums[base + k] : 0;
            s += v[k];
        }
        int32_t total;
        int32_t off = block_exclusive_scan(s, &total) + carry;
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            if (base + k < nb) sums[base + k] = off;
            off += v[k];
        }
        carry += total;
    }
}

// scanned: sums[] holds the blocks' exclusive offsets (k_scan_sums ran);
// else it holds their totals and each block adds up those before it.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const int32_t* in, int32_t n,
                                                            const int32_t* __restrict__ sums, int32_t scanned,
                                                            int32_t* __restrict__ out, int32_t* clear)
{
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS], s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    if (clear)
        for (int k = 0; k < SCAN_ITEMS; ++k)
            if (base + k < n) clear[base + k] = 0;
    int32_t offset;
    if (scanned) {
        offset = sums[blockIdx.x];
    } else {
        // integer sums: the order of the additions does not matter
        int32_t before = 0;
        for (int k = threadIdx.x; k < (int)blockIdx.x; k += SCAN_THREADS) before += sums[k];
        block_exclusive_scan(before, &offset);
    }
    int32_t total;
    int32_t off = block_exclusive_scan(s, &total) + offset;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = off;
        off += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = off;
}

// Whole scan in one block for short inputs: thread t owns a contiguous chunk
// of ceil(n / SCAN_THREADS) values, sums it, takes its offset from a block
// scan of the chunk sums, then writes its chunk's prefix sums.
constexpr int SCAN_SMALL = SCAN_THREADS * 64;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_single(const int32_t* in, int32_t n,
                                                              int32_t* __restrict__ out, int32_t* clear)
{
    const int per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    const int b = threadIdx.x * per;
    const int e = b + per < n ? b + per : n;
    int32_t s = 0;
    for (int k = b; k < e; ++k) s += in[k];
    int32_t total;
    int32_t off = block_exclusive_scan(s, &total);
    for (int k = b; k < e; ++k) {
        const int32_t v = in[k];
        out[k] = off;
        off += v;
        if (clear) clear[k] = 0;
    }
    if (threadIdx.x == 0) out[n] = total;
}

int32_t scan_blocks(int64_t n) { return (int32_t)((n + SCAN_TILE - 1) / SCAN_TILE); }
int64_t scan_max_len() { return SCAN_MAX; }

int64_t grid_cell_count(const int32_t dims[3])
{
    int64_t n = 1;
    for (int d = 0; d < 3; ++d) {
        if (dims[d] < 1 || dims[d] > SCAN_MAX) return -1;
        n *= dims[d];  // <= 2^24 * 2^24: no overflow
        if (n > SCAN_MAX - 2) return -1;
    }
    return n;
}

int scan_exclusive(const int32_t* in, int32_t n, int32_t* out, int32_t* sums, cudaStream_t st, int32_t* clear)
{
    if (n <= SCAN_SMALL) {
        k_scan_single<<<1, SCAN_THREADS, 0, st>>>(in, n, out, clear);
        return 1;
    }
    int nb = scan_blocks(n);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(in, n, sums);
    const bool direct = nb <= SCAN_DIRECT;
    if (!direct) k_scan_sums<<<1, SCAN_THREADS, 0, st>>>(sums, nb);
    k_scan_down<<<nb, SCAN_THREADS, 0, st>>>(in, n, sums, direct ? 0 : 1, out, clear);
    return direct ? 2 : 3;
}

// ------------------------------------------------- stand-alone binning API
__global__ void k_bin_keys(int32_t n, const double* __restrict__ x, double lo0, double lo1, double lo2,
                           double cs, int32_t nx, int32_t ny, int32_t nz, int4* __restrict__ cell,
                           int32_t* __restrict__ id, int32_t* __restrict__ rank, int32_t* counts,
                           int32_t n_cells)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo[3] = {lo0, lo1, lo2};
    int32_t dims[3] = {nx, ny, nz}, c[3];
    bool inside = true;
    for (int d = 0; d < 3; ++d) {
        double f = floor((x[3 * i + d] - lo[d]) / cs);
        c[d] = (f < -1e9) ? -1000000000 : (f > 1e9 ? 1000000000 : (int32_t)f);
        inside = inside && c[d] >= 0 && c[d] < dims[d];
    }
    int key = inside ? (c[2] * ny + c[1]) * nx + c[0] : -1;
    cell[i] = int4{c[0], c[1], c[2], key};
    id[i] = i;
    rank[i] = atomicAdd(counts + (key < 0 ? n_cells : key), 1);
}

__global__ void k_bin_order(int32_t n, int32_t n_cells, const int32_t* __restrict__ start,
                            const int32_t* __restrict__ tmp_src, const int32_t* __restrict__ tmp_id,
                            const int4* __restrict__ cell, uint32_t* __restrict__ key_by_id,
                            int32_t* __restrict__ order)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int s = tmp_src[t];
    int key = cell[s].w;
    int dst = sorted_slot(t, key, n_cells, start, tmp_id);
    order[dst] = tmp_id[t];
    key_by_id[tmp_id[t]] = (uint32_t)key;
}

BinSortScratch bin_sort_scratch_layout(int64_t n, int64_t n_cells)
{
    BinSortScratch L;
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t off = 0;
    L.cell = off; off += up(sizeof(int4) * (size_t)n);
    L.id = off; off += up(sizeof(int32_t) * (size_t)n);
    L.rank = off; off += up(sizeof(int32_t) * (size_t)n);
    L.tmp_src = off; off += up(sizeof(int32_t) * (size_t)n);
    L.tmp_id = off; off += up(sizeof(int32_t) * (size_t)n);
    L.counts = off; off += up(sizeof(int32_t) * (size_t)(n_cells + 1));
    L.start = off; off += up(sizeof(int32_t) * (size_t)(n_cells + 2));
    L.sums = off; off += up(sizeof(int32_t) * (size_t)scan_blocks(n_cells + 1));
    L.bytes = off;
    return L;
}

cudaError_t bin_sort_run(const double* pos, int32_t n, const double lo[3], double cs,
                         const int32_t dims[3], uint32_t* key, int32_t* order, int32_t* start,
                         char* scratch, cudaStream_t st)
{
    int32_t n_cells = dims[0] * dims[1] * dims[2];
    BinSortScratch L = bin_sort_scratch_layout(n, n_cells);
    int4* cell = (int4*)(scratch + L.cell);
    int32_t* id = (int32_t*)(scratch + L.id);
    int32_t* rank = (int32_t*)(scratch + L.rank);
    int32_t* tmp_src = (int32_t*)(scratch + L.tmp_src);
    int32_t* tmp_id = (int32_t*)(scratch + L.tmp_id);
    int32_t* counts = (int32_t*)(scratch + L.counts);
    int32_t* fullstart = (int32_t*)(scratch + L.start);
    int32_t* sums = (int32_t*)(scratch + L.sums);
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)(n_cells + 1), st);
    if (e != cudaSuccess) return e;
    int nb = (n + BLOCK - 1) / BLOCK;
    if (n > 0)
        k_bin_keys<<<nb, BLOCK, 0, st>>>(n, pos, lo[0], lo[1], lo[2], cs, dims[0], dims[1], dims[2],
                                         cell, id, rank, counts, n_cells);
    scan_exclusive(counts, n_cells + 1, fullstart, sums, st, nullptr);
    if (n > 0) {
        k_scatter<<<nb, BLOCK, 0, st>>>(n, n_cells, cell, rank, fullstart, id, tmp_src, tmp_id, nullptr);
        k_bin_order<<<nb, BLOCK, 0, st>>>(n, n_cells, fullstart, tmp_src, tmp_id, cell, key, order);
    }
    e = cudaMemcpyAsync(start, fullstart, sizeof(int32_t) * (size_t)(n_cells + 1),
                        cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace sph
