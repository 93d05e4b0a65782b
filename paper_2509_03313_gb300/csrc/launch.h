// Host-side entry points of the kernel translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace chem {

struct Dev;

// Phase indices of chem_stats.phase_ms.
enum Phase { PH_BEGIN = 0, PH_RELEASE, PH_DIFFUSE, PH_SORT, PH_GATHER, PH_SEARCH, PH_REACT,
             PH_PERSISTENT, N_PHASES };

struct LaunchCfg {
  int stream_blocks;      // grid of the grid-stride phases (release, diffuse, gather)
  int search_blocks;      // grid of the pair search
  int sort_blocks;        // resident CTAs of a sort pass
  int persistent_blocks;  // resident CTAs of the persistent step kernel
  int search_tps;         // pair search: 1 one thread per home species, 0 cell tiles,
                          // 2 both launched, the step's choice runs (adaptive)
};

// kernels_exact.cu (FP64 arithmetic without contraction)
cudaError_t enqueue_begin(const Dev& d, cudaStream_t s);
cudaError_t enqueue_sort_pass(const Dev& d, int pass, int blocks, cudaStream_t s);
// matching (fast path + conflict rounds), event ordering, product prefix
cudaError_t enqueue_react_head(const Dev& d, const LaunchCfg& lc, cudaStream_t s);
cudaError_t enqueue_end_step(const Dev& d, cudaStream_t s);
// end of one step and begin of the next in one one-CTA kernel
cudaError_t enqueue_end_begin(const Dev& d, cudaStream_t s);
cudaError_t sort_pass_occupancy(int* blocks_per_sm);
// One SBS step. `first`: the step begins with its own begin kernel (else the previous
// step's end kernel began it); `last`: it ends with a plain end kernel (else its end
// kernel also begins the next step).
cudaError_t enqueue_step_f64(const Dev& d, const LaunchCfg& lc, cudaStream_t s, cudaEvent_t* ev, bool first,
                             bool last);
cudaError_t enqueue_persistent_f64(const Dev& d, const LaunchCfg& lc, int n_steps, cudaStream_t s);
cudaError_t persistent_occupancy_f64(int* blocks_per_sm);
cudaError_t enqueue_set_t_end(const Dev& d, const double* t_end_dev, cudaStream_t s);
// one device thread waits, up to limit_s, for a word nothing writes (then CHEM_ETIMEOUT)
cudaError_t enqueue_bounded_wait(const Dev& d, double limit_s, cudaStream_t s);

// the pair acceptance test on given squared separations (diagnostic; one per precision)
cudaError_t enqueue_check_accept_f64(const Dev& d, uint32_t n, uint32_t step, double dt, const double* d0sq,
                                     const double* d1sq, const int32_t* rxn, const uint32_t* id_lo,
                                     const uint32_t* id_hi, uint8_t* out, cudaStream_t s);
cudaError_t enqueue_check_accept_f32l(const Dev& d, uint32_t n, uint32_t step, double dt, const double* d0sq,
                                      const double* d1sq, const int32_t* rxn, const uint32_t* id_lo,
                                      const uint32_t* id_hi, uint8_t* out, cudaStream_t s);

// homog.cu: homogeneous (beam-off) stage of the trains with Train::hx_sel set
cudaError_t enqueue_homogeneous(const Dev& d, int blocks, cudaStream_t s);

// kernels_f32l.cu (FP32-local mode)
cudaError_t enqueue_step_f32l(const Dev& d, const LaunchCfg& lc, cudaStream_t s, cudaEvent_t* ev, bool first,
                              bool last);
cudaError_t enqueue_persistent_f32l(const Dev& d, const LaunchCfg& lc, int n_steps, cudaStream_t s);
cudaError_t persistent_occupancy_f32l(int* blocks_per_sm);

}  // namespace chem
