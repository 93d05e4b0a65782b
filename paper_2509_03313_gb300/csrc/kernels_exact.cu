// FP64-mode kernels and the precision-independent ones (step begin, sort passes).
// Built with --fmad=false: together with the explicit _rn intrinsics in phases.cuh
// this keeps the FP64 mode's rounding identical to the FP64 reference's.
#include "kernels.cuh"

namespace chem {

__global__ void __launch_bounds__(256) k_begin(const __grid_constant__ Dev d) {
  __shared__ BeginSmem sb;
  phase_begin(d, sb);
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_pass(const __grid_constant__ Dev d, int pass) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  phase_sort_pass(d, pass, *reinterpret_cast<SortSmem*>(smem_raw));
}

__global__ void __launch_bounds__(256) k_match_fast(const __grid_constant__ Dev d) {
  phase_match_fast(d);
}

constexpr size_t REACT_SERIAL_DYN_SMEM = (4 * EV_SMEM_CAP * sizeof(uint32_t) > RC_SMEM_BYTES)
                                           ? 4 * EV_SMEM_CAP * sizeof(uint32_t) : RC_SMEM_BYTES;

__global__ void __launch_bounds__(REACT_THREADS) k_react_serial(const __grid_constant__ Dev d) {
  __shared__ SerialSmem sm;
  extern __shared__ __align__(16) uint32_t sbuf[];
  phase_react_serial(d, sm, sbuf);
}

__global__ void __launch_bounds__(256) k_end_step(const __grid_constant__ Dev d) {
  __shared__ EndSmem sm;
  phase_end_step(d, sm);
}

cudaError_t enqueue_react_head(const Dev& d, const LaunchCfg& lc, cudaStream_t s) {
  k_match_fast<<<lc.stream_blocks, 256, 0, s>>>(d);
  k_react_serial<<<1, REACT_THREADS, REACT_SERIAL_DYN_SMEM, s>>>(d);
  return cudaGetLastError();
}

cudaError_t enqueue_end_step(const Dev& d, cudaStream_t s) {
  k_end_step<<<1, 256, 0, s>>>(d);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_end_begin(const __grid_constant__ Dev d) {
  __shared__ EndSmem se;
  __shared__ BeginSmem sb;
  phase_end_step(d, se);
  phase_begin(d, sb);
}

cudaError_t enqueue_end_begin(const Dev& d, cudaStream_t s) {
  k_end_begin<<<1, 256, 0, s>>>(d);
  return cudaGetLastError();
}

__global__ void k_set_t_end(const __grid_constant__ Dev d, const double* t_end) {
  for (uint32_t b = threadIdx.x; b < d.n_trains; b += blockDim.x) d.trains[b].t_end = t_end[b];
}

cudaError_t enqueue_begin(const Dev& d, cudaStream_t s) {
  k_begin<<<1, 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t enqueue_sort_pass(const Dev& d, int pass, int blocks, cudaStream_t s) {
  k_sort_pass<<<blocks, SORT_THREADS, sizeof(SortSmem), s>>>(d, pass);
  return cudaGetLastError();
}

cudaError_t sort_pass_occupancy(int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sizeof(SortSmem)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_react_serial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(REACT_SERIAL_DYN_SMEM));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_sort_pass, SORT_THREADS,
                                                       sizeof(SortSmem));
}

// One thread waits for a word that nothing writes (Global::never_set), polling it until
// limit_ns of the global timer have passed, then raises CHEM_ETIMEOUT: the error path of
// every bounded device wait of the library, without a fault.
__global__ void k_bounded_wait(const __grid_constant__ Dev d, unsigned long long limit_ns) {
  if (threadIdx.x != 0) return;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  const volatile uint32_t* flag = &d.g->never_set;
  for (;;) {
    if (*flag != 0u) return;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) {
      raise_status(d.g, CHEM_ETIMEOUT);
      return;
    }
    __nanosleep(1000);
  }
}

cudaError_t enqueue_bounded_wait(const Dev& d, double limit_s, cudaStream_t s) {
  k_bounded_wait<<<1, 32, 0, s>>>(d, static_cast<unsigned long long>(limit_s * 1e9));
  return cudaGetLastError();
}

cudaError_t enqueue_set_t_end(const Dev& d, const double* t_end_dev, cudaStream_t s) {
  k_set_t_end<<<1, 256, 0, s>>>(d, t_end_dev);
  return cudaGetLastError();
}

cudaError_t enqueue_step_f64(const Dev& d, const LaunchCfg& lc, cudaStream_t s, cudaEvent_t* ev, bool first,
                             bool last) {
  return enqueue_phases<false>(d, lc, s, ev, first, last);
}

cudaError_t enqueue_persistent_f64(const Dev& d, const LaunchCfg& lc, int n_steps, cudaStream_t s) {
  return enqueue_persistent<false>(d, lc, n_steps, s);
}

cudaError_t persistent_occupancy_f64(int* blocks_per_sm) { return persistent_occupancy<false>(blocks_per_sm); }

cudaError_t enqueue_check_accept_f64(const Dev& d, uint32_t n, uint32_t step, double dt, const double* d0sq,
                                     const double* d1sq, const int32_t* rxn, const uint32_t* id_lo,
                                     const uint32_t* id_hi, uint8_t* out, cudaStream_t s) {
  return enqueue_check_accept<false>(d, n, step, dt, d0sq, d1sq, rxn, id_lo, id_hi, out, s);
}

}  // namespace chem
