// Onesweep LSD radix sort pass (Adinets & Merrill 2022, "Onesweep: a faster least
// significant digit radix sort for GPUs"), written for sm_103a.
//
// One pass sorts (key, value) pairs stably by one 8-bit digit:
//  * the digit histogram of the whole input comes precomputed (it is accumulated for
//    every pass at once while the keys are produced), so each CTA derives the global
//    digit bases with a 256-wide exclusive scan;
//  * tiles of 3840 keys are claimed in order through an atomic counter; inside a tile
//    each warp ranks its keys with __match_any_sync (warp-private digit counters keep
//    the pass stable; the keys of a tile are nearly sorted, so few digits are distinct),
//    warps are combined through shared memory;
//  * decoupled look-back (Merrill & Garland 2016) chains the per-digit tile counts:
//    a tile publishes its local count (AGGREGATE) at once, then walks back over its
//    predecessors until it meets an INCLUSIVE prefix, and publishes its own inclusive
//    prefix. Status words carry a pass epoch so they never need clearing. Every wait
//    is bounded by a clock64 limit; on expiry the kernel raises CHEM_ETIMEOUT,
//    publishes what it has so no successor waits forever, and finishes the tile.
//  * keys are reordered by digit in shared memory and written out in runs.
#pragma once
#include "sbs_device.cuh"

namespace chem {

// NT threads per CTA, tiles of NT * SORT_ITEMS keys.
template <int NT>
struct SortSmemT {
  static constexpr int TILE = NT * SORT_ITEMS;
  uint32_t wcnt[NT / 32][RADIX];
  uint32_t gbase[RADIX];      // global exclusive digit base
  uint32_t tile_cnt[RADIX];
  uint32_t tile_off[RADIX];   // exclusive digit offsets inside the tile
  uint32_t tile_out[RADIX];   // gbase + look-back prefix
  uint32_t k[TILE];
  uint32_t v[TILE];
  uint32_t tile;
  uint32_t warp_tot[NT / 32];
};
using SortSmem = SortSmemT<SORT_THREADS>;      // the per-pass kernel
using SortSmemP = SortSmemT<PERSIST_THREADS>;  // the persistent kernel

constexpr unsigned long long LB_AGG = 1ull, LB_INC = 2ull;

__device__ __forceinline__ unsigned long long lb_pack(uint32_t epoch, unsigned long long flag,
                                                      uint32_t count) {
  return (static_cast<unsigned long long>(epoch & 0x3FFFFFFFu) << 34) | (flag << 32) | count;
}

// Exclusive scan of 256 values held one per thread (threads 0..255) through smem.
__device__ __forceinline__ uint32_t block_exclusive_scan256(uint32_t v, uint32_t* warp_tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  uint32_t add = 0;
  for (int i = 0; i < w; ++i) add += warp_tot[i];
  __syncthreads();
  return x - v + add;
}

// One pass over n keys by digit (key >> shift) & 255. ghist = this digit's histogram
// over all n keys; vin == nullptr means value = input index. Must be called by all NT
// threads of every CTA.
template <int NT>
__device__ void onesweep_pass(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                              uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n,
                              int shift, const uint32_t* ghist, uint32_t* tile_ctr,
                              unsigned long long* lookback, uint32_t epoch, Global* g,
                              SortSmemT<NT>& sm) {
  constexpr int SORT_TILE = SortSmemT<NT>::TILE;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  {
    uint32_t c = (tid < RADIX) ? ghist[tid] : 0u;
    uint32_t e = block_exclusive_scan256(c, sm.warp_tot);
    if (tid < RADIX) sm.gbase[tid] = e;
  }
  const uint32_t n_tiles = (n + SORT_TILE - 1) / SORT_TILE;
  for (;;) {
    if (tid == 0) sm.tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const uint32_t tile = sm.tile;
    if (tile >= n_tiles) break;
    const uint32_t tile_base = tile * SORT_TILE;
    const uint32_t tile_n = min(static_cast<uint32_t>(SORT_TILE), n - tile_base);
    // clear this warp's digit counters
#pragma unroll
    for (int i = lane; i < RADIX; i += 32) sm.wcnt[w][i] = 0u;
    __syncwarp();
    uint32_t key[SORT_ITEMS], val[SORT_ITEMS], rank[SORT_ITEMS];
    const uint32_t wbase = tile_base + w * (32 * SORT_ITEMS);
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
      const uint32_t idx = wbase + r * 32 + lane;
      const bool valid = idx < n;
      key[r] = valid ? kin[idx] : 0xFFFFFFFFu;
      val[r] = valid ? (vin ? vin[idx] : idx) : 0u;
    }
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
      const uint32_t idx = wbase + r * 32 + lane;
      const bool valid = idx < n;
      const uint32_t d = (key[r] >> shift) & 255u;
      const uint32_t mask = __ballot_sync(0xffffffffu, valid);
      uint32_t peers = 0, pre = 0;
      if (valid) {
        peers = __match_any_sync(mask, d);
        pre = sm.wcnt[w][d];
        rank[r] = pre + __popc(peers & lanemask_lt);
      }
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) sm.wcnt[w][d] = pre + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // combine warps: exclusive over warps per digit, tile totals
    if (tid < RADIX) {
      uint32_t s = 0;
#pragma unroll
      for (int ww = 0; ww < NT / 32; ++ww) {
        const uint32_t c = sm.wcnt[ww][tid];
        sm.wcnt[ww][tid] = s;
        s += c;
      }
      sm.tile_cnt[tid] = s;
      // publish the aggregate at once so successors can proceed
      unsigned long long* slot = lookback + static_cast<size_t>(tile) * RADIX + tid;
      st_relaxed_u64(slot, lb_pack(epoch, tile == 0 ? LB_INC : LB_AGG, s));
    }
    {
      uint32_t c = (tid < RADIX) ? sm.tile_cnt[tid] : 0u;
      uint32_t e = block_exclusive_scan256(c, sm.warp_tot);
      if (tid < RADIX) sm.tile_off[tid] = e;
    }
    // decoupled look-back, one thread per digit; the status words of LB_BATCH
    // predecessors are read together, then consumed newest first until an inclusive
    // prefix (done) or a word not yet published (read again from there)
    if (tid < RADIX) {
      uint32_t excl = 0;
      if (tile > 0) {
        long long t0 = clock64();
        int32_t t = static_cast<int32_t>(tile) - 1;
        bool timed_out = false;
        while (t >= 0) {
          constexpr int LB_BATCH = 8;
          unsigned long long wv[LB_BATCH];
#pragma unroll
          for (int q = 0; q < LB_BATCH; ++q)
            wv[q] = (q <= t) ? ld_relaxed_u64(lookback + static_cast<size_t>(t - q) * RADIX + tid) : 0ull;
          int used = 0;
          bool done = false;
#pragma unroll
          for (int q = 0; q < LB_BATCH; ++q) {
            if (done || used < q || q > t) continue;  // stop at the first gap
            const uint32_t ep = static_cast<uint32_t>(wv[q] >> 34);
            const unsigned long long fl = (wv[q] >> 32) & 3ull;
            if (ep != (epoch & 0x3FFFFFFFu) || fl == 0ull) continue;
            excl += static_cast<uint32_t>(wv[q]);
            used = q + 1;
            if (fl == LB_INC) done = true;
          }
          if (done) break;
          t -= used;
          if (used == 0 && clock64() - t0 > SPIN_LIMIT_CYCLES) { timed_out = true; break; }
        }
        if (timed_out) raise_status(g, CHEM_ETIMEOUT);
        st_relaxed_u64(lookback + static_cast<size_t>(tile) * RADIX + tid,
                       lb_pack(epoch, LB_INC, excl + sm.tile_cnt[tid]));
      }
      sm.tile_out[tid] = sm.gbase[tid] + excl;
    }
    __syncthreads();
    // scatter into shared memory in digit order
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
      const uint32_t idx = wbase + r * 32 + lane;
      if (idx < n) {
        const uint32_t d = (key[r] >> shift) & 255u;
        const uint32_t p = sm.tile_off[d] + sm.wcnt[w][d] + rank[r];
        sm.k[p] = key[r];
        sm.v[p] = val[r];
      }
    }
    __syncthreads();
    for (uint32_t p = tid; p < tile_n; p += NT) {
      const uint32_t k = sm.k[p];
      const uint32_t d = (k >> shift) & 255u;
      const uint32_t o = sm.tile_out[d] + (p - sm.tile_off[d]);
      if (o < n) {  // always true unless a look-back wait timed out
        kout[o] = k;
        vout[o] = sm.v[p];
      }
    }
    __syncthreads();
  }
}

}  // namespace chem
