// FP32 form of the step: FP32 pair arithmetic and accumulation, positions as
// cell index + FP32 offset with a Kahan-compensated drift.
#include "sph_sim.cuh"

namespace sph {
SimBase* make_sim_f32(cudaStream_t st) { return new Sim<float>(st); }
}  // namespace sph
