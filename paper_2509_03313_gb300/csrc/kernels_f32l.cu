// FP32-local-mode kernels: positions as FP32 offsets from their hash cell's origin,
// FP32 normals and distances; clock, schedule, reaction probabilities and tallies FP64.
#include "kernels.cuh"

namespace chem {

cudaError_t enqueue_step_f32l(const Dev& d, const LaunchCfg& lc, cudaStream_t s, cudaEvent_t* ev, bool first,
                              bool last) {
  return enqueue_phases<true>(d, lc, s, ev, first, last);
}

cudaError_t enqueue_persistent_f32l(const Dev& d, const LaunchCfg& lc, int n_steps, cudaStream_t s) {
  return enqueue_persistent<true>(d, lc, n_steps, s);
}

cudaError_t persistent_occupancy_f32l(int* blocks_per_sm) { return persistent_occupancy<true>(blocks_per_sm); }

cudaError_t enqueue_check_accept_f32l(const Dev& d, uint32_t n, uint32_t step, double dt, const double* d0sq,
                                     const double* d1sq, const int32_t* rxn, const uint32_t* id_lo,
                                     const uint32_t* id_hi, uint8_t* out, cudaStream_t s) {
  return enqueue_check_accept<true>(d, n, step, dt, d0sq, d1sq, rxn, id_lo, id_hi, out, s);
}

}  // namespace chem
