// Plain FP64 form of the step: the same kernels instantiated in double.
#include "sph_sim.cuh"

namespace sph {
SimBase* make_sim_f64(cudaStream_t st) { return new Sim<double>(st); }
}  // namespace sph
