// Allocation-free variant of the stand-alone binning (sph_bin_sort_noalloc):
// the same kernels as sph_bin_sort, with their scratch in one fixed array in
// device memory instead of memory allocated per call.  For callers that must
// not allocate while they run (see include/sph.h).
#include <cstdint>
#include <mutex>

#include "sph_internal.h"

namespace {

constexpr size_t kScratchBytes = SPH_BIN_SORT_NOALLOC_SCRATCH;
constexpr int kMaxDevices = 64;

// The scratch: every GPU that loads the library holds it until exit.  Host
// code must not take its address directly (that is a host-side stand-in);
// the device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) char g_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device, looked up once per
// device (the first call must therefore not happen inside a stream capture).
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sph_status sph_bin_sort_noalloc(const double* pos, int64_t n, const double lo[3], double h,
                                           const int32_t dims[3], uint32_t* key, int32_t* order,
                                           int32_t* start, void* cuda_stream)
{
    if (n < 0 || n > 2000000000 || !lo || !dims || !(h > 0) || !start || (n > 0 && (!pos || !key || !order)))
        return SPH_ERR_ARG;
    const int64_t n_cells = sph::grid_cell_count(dims);
    if (n_cells < 0) return SPH_ERR_ARG;
    const sph::BinSortScratch L = sph::bin_sort_scratch_layout(n, n_cells);
    if (L.bytes > kScratchBytes) return SPH_ERR_CAPACITY;
    void* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return SPH_ERR_CUDA;
    // bin_sort_run clears the per-cell counters itself before counting
    const cudaError_t e = sph::bin_sort_run(pos, (int32_t)n, lo, 2.0 * h, dims, key, order, start,
                                            static_cast<char*>(scratch), (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
