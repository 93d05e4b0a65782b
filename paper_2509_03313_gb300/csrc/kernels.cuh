// Kernels of one SBS step: one kernel per phase (captured into a CUDA graph of several
// steps), and a persistent cooperative kernel that runs the same phases for several
// steps of every train with grid barriers in between.
#pragma once
#include "launch.h"
#include "phases.cuh"
#include "search_cells.cuh"

namespace chem {

union PhaseSmem {
  BeginSmem begin;
  SerialSmem serial;
  ProductsSmem products;
  EndSmem end;
  ScSmem<8> cells;
  TpsSmem<true, 8> tps32;
  TpsSmem<false, 8> tps64;
  uint32_t hist[MAX_PASSES][RADIX];
  SortSmemP sort;
};

// Grid-wide barrier of the persistent kernel. The wait is bounded: past the limit the
// kernel raises CHEM_ETIMEOUT, and once any error is raised the barrier stops waiting
// (every phase then skips its work), so a launch always ends.
__device__ __forceinline__ void grid_sync(const Dev& d) {
  __syncthreads();
  if (threadIdx.x == 0) {
    Global* g = d.g;
    const uint32_t gen = ld_acquire_u32(&g->bar_gen);
    __threadfence();
    const uint32_t arrived = atomicAdd(&g->bar_count, 1u) + 1u;
    if (arrived == gridDim.x) {
      g->bar_count = 0;
      __threadfence();
      atomicAdd(&g->bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_u32(&g->bar_gen) == gen) {
        if (*reinterpret_cast<volatile int*>(&g->status) != 0) break;
        if (clock64() - t0 > SPIN_LIMIT_CYCLES) {
          raise_status(g, CHEM_ETIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

template <bool F32L>
__global__ void __launch_bounds__(256) k_diffuse(const __grid_constant__ Dev d) {
  __shared__ uint32_t hist[MAX_PASSES][RADIX];
  phase_diffuse<F32L>(d, hist);
}

template <bool F32L>
__global__ void __launch_bounds__(256) k_gather(const __grid_constant__ Dev d) {
  phase_gather<F32L>(d);
}

template <bool F32L>
__global__ void __launch_bounds__(256, 4) k_search(const __grid_constant__ Dev d) {
  __shared__ ScSmem<8> sm;
  phase_search_cells<F32L, 8>(d, sm);
}

constexpr int TPS_WARPS = 4;  // warps per CTA of the one-thread-per-species search

template <bool F32L>
__global__ void __launch_bounds__(32 * TPS_WARPS, F32L ? 6 : 5) k_search_tps(const __grid_constant__ Dev d) {
  __shared__ TpsSmem<F32L, TPS_WARPS> sm;
  phase_search_tps<F32L, TPS_WARPS>(d, sm);
}

template <bool F32L>
__global__ void __launch_bounds__(256) k_products(const __grid_constant__ Dev d) {
  __shared__ ProductsSmem sm;
  phase_products<F32L>(d, sm);
}

template <bool F32L>
__global__ void __launch_bounds__(PERSIST_THREADS) k_persistent(const __grid_constant__ Dev d, int n_steps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PhaseSmem& sm = *reinterpret_cast<PhaseSmem*>(smem_raw);
  if (blockIdx.x == 0) phase_begin(d, sm.begin);
  grid_sync(d);
  for (int step = 0; step < n_steps; ++step) {
    phase_diffuse<F32L>(d, sm.hist);  // includes the release
    grid_sync(d);
    for (int p = 0; p < d.passes; ++p) {
      phase_sort_pass(d, p, sm.sort);
      grid_sync(d);
    }
    phase_gather<F32L>(d);
    grid_sync(d);
    if (d.g->search_cells_now) {
      phase_search_cells<F32L, 8>(d, sm.cells);
    } else {
      if constexpr (F32L) phase_search_tps<true, 8>(d, sm.tps32);
      else phase_search_tps<false, 8>(d, sm.tps64);
    }
    grid_sync(d);
    phase_match_fast(d);
    grid_sync(d);
    if (blockIdx.x == 0) phase_react_serial(d, sm.serial, nullptr);
    grid_sync(d);
    phase_products<F32L>(d, sm.products);
    grid_sync(d);
    if (blockIdx.x == 0) {
      phase_end_step(d, sm.end);
      if (step + 1 < n_steps) phase_begin(d, sm.begin);  // the next step's begin
    }
    grid_sync(d);
  }
}

// One step as one kernel per phase. With ev != nullptr, CUDA events are recorded
// before and after each phase (ev[2 * phase], ev[2 * phase + 1]); a step that is not the
// first of a graph was begun by the previous step's end kernel (its time falls in the
// previous step's react phase).
template <bool F32L>
cudaError_t enqueue_phases(const Dev& d, const LaunchCfg& lc, cudaStream_t s, cudaEvent_t* ev, bool first,
                           bool last) {
  auto mark = [&](int i) { if (ev) cudaEventRecordWithFlags(ev[i], s, cudaEventRecordExternal); };
  cudaError_t e = cudaSuccess;
  mark(2 * PH_BEGIN);
  if (first) {
    e = enqueue_begin(d, s);
    if (e != cudaSuccess) return e;
  }
  mark(2 * PH_BEGIN + 1);
  mark(2 * PH_RELEASE);  // the release runs inside the diffusion kernel
  mark(2 * PH_RELEASE + 1);
  mark(2 * PH_DIFFUSE);
  k_diffuse<F32L><<<lc.stream_blocks, 256, 0, s>>>(d);
  mark(2 * PH_DIFFUSE + 1);
  mark(2 * PH_SORT);
  for (int p = 0; p < d.passes; ++p) {
    e = enqueue_sort_pass(d, p, lc.sort_blocks, s);
    if (e != cudaSuccess) return e;
  }
  mark(2 * PH_SORT + 1);
  mark(2 * PH_GATHER);
  k_gather<F32L><<<lc.stream_blocks, 256, 0, s>>>(d);
  mark(2 * PH_GATHER + 1);
  mark(2 * PH_SEARCH);
  // one mapping, or both with the one not chosen for the step returning at once
  if (lc.search_tps != 0) k_search_tps<F32L><<<2 * lc.search_blocks, 32 * TPS_WARPS, 0, s>>>(d);
  if (lc.search_tps != 1) k_search<F32L><<<lc.search_blocks, 256, 0, s>>>(d);
  mark(2 * PH_SEARCH + 1);
  mark(2 * PH_REACT);
  e = enqueue_react_head(d, lc, s);
  if (e != cudaSuccess) return e;
  k_products<F32L><<<lc.stream_blocks, 256, 0, s>>>(d);
  e = last ? enqueue_end_step(d, s) : enqueue_end_begin(d, s);
  if (e != cudaSuccess) return e;
  mark(2 * PH_REACT + 1);
  return cudaGetLastError();
}

// Diagnostic: the pair search's acceptance test on given squared separations d0^2 and
// d1^2 of reaction rxn[i] for the pair (id_lo[i], id_hi[i]) at `step`, with the constants
// the begin phase derives from dt. out[i] bit 0: the tiered test of the search (FP32
// estimate, FP64 where undecided); bit 1: the FP64 test u < p itself on the same inputs
// (in FP32-local mode, on the FP32 roundings of the squared separations).
template <bool F32L>
__global__ void __launch_bounds__(256) k_check_accept(const __grid_constant__ Dev d, uint32_t n, uint32_t step,
                                                      double dt, const double* d0sq, const double* d1sq,
                                                      const int32_t* rxn, const uint32_t* id_lo,
                                                      const uint32_t* id_hi, uint8_t* out) {
  __shared__ Train tr;
  const Tables& tb = *d.tables;
  if (threadIdx.x == 0) {
    tr = d.trains[0];
    tr.step = step;
    for (int r = 0; r < tb.n_rxn; ++r) set_pair_constants(tr, tb, r, dt);
  }
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int r = rxn[i];
    const uint32_t lo = id_lo[i], hi = id_hi[i];
    const double u = pair_uniform(lo, hi, step, tr.key0, tr.key1);
    bool tiered, exact;
    if constexpr (F32L) {
      const float a = static_cast<float>(d0sq[i]), b = static_cast<float>(d1sq[i]);
      tiered = accept_f32(a, b, r, tb, tr, lo, hi);
      exact = u < bridge_p(sqrt(static_cast<double>(a)), sqrt(static_cast<double>(b)), tb.R[r], tr.ddt[r]);
    } else {
      tiered = accept_f64(d0sq[i], d1sq[i], r, tb, tr, lo, hi);
      exact = u < bridge_p(sqrt(d0sq[i]), sqrt(d1sq[i]), tb.R[r], tr.ddt[r]);
    }
    out[i] = static_cast<uint8_t>((tiered ? 1 : 0) | (exact ? 2 : 0));
  }
}

template <bool F32L>
cudaError_t enqueue_check_accept(const Dev& d, uint32_t n, uint32_t step, double dt, const double* d0sq,
                                 const double* d1sq, const int32_t* rxn, const uint32_t* id_lo,
                                 const uint32_t* id_hi, uint8_t* out, cudaStream_t s) {
  const uint32_t blocks = n ? (n + 255u) / 256u : 1u;
  k_check_accept<F32L><<<blocks < 1024u ? blocks : 1024u, 256, 0, s>>>(d, n, step, dt, d0sq, d1sq, rxn, id_lo,
                                                                       id_hi, out);
  return cudaGetLastError();
}

template <bool F32L>
cudaError_t enqueue_persistent(const Dev& d, const LaunchCfg& lc, int n_steps, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(lc.persistent_blocks);
  cfg.blockDim = dim3(PERSIST_THREADS);
  cfg.dynamicSmemBytes = sizeof(PhaseSmem);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_persistent<F32L>, d, n_steps);
}

template <bool F32L>
cudaError_t persistent_occupancy(int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_persistent<F32L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sizeof(PhaseSmem)));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_persistent<F32L>, PERSIST_THREADS,
                                                       sizeof(PhaseSmem));
}

}  // namespace chem
