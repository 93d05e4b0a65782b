// Device-side data layout and helpers of the SBS chemistry library (sm_103a).
//
// Layout in HBM (one context = B >= 1 independent pulse trains):
//  * species state S, sorted by global hash cell (cell_base[train] + local cell):
//      FP64 mode        SoA  double x[cap], y[cap], z[cap]; uint32 tid[cap]
//      FP32-local mode  AoS  float4 {off_x, off_y, off_z, bits(tid)} per slot; the
//                       offsets are relative to the origin of the slot's hash cell
//    tid = (id << 3) | type. A scratch copy T of the same layout receives the diffused
//    species in S order before the sort.
//  * cell_sorted[cap]: global cell of every slot of S (train = cell -> train lookup)
//  * radix scratch keys[2][cap], vals[2][cap] (reused as the matching arrays)
//  * cell_info[total_cells]: int4 {first slot, end slot, epoch stamp, 0}. An entry is
//    valid only when its stamp equals the current step epoch, so the table (large at
//    fine grids) is never cleared.
//  * occ[total_cells / 32]: occupancy bitmap (one bit per cell, L2-resident in use),
//    rebuilt every step (the diffusion clears the words of the last step's cells); the
//    pair search tests it before reading an entry. A stale bit only costs a lookup:
//    the entry's epoch stamp still decides.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/chem.h"

namespace chem {

constexpr int MAXT = CHEM_MAX_TYPES;
constexpr int MAXR = CHEM_MAX_RXN;
constexpr int MAX_TRAINS = 256;
constexpr int RADIX = 256;
constexpr int MAX_PASSES = 4;
constexpr int SORT_THREADS = 512;    // threads of the per-pass sort kernel
constexpr int PERSIST_THREADS = 256; // threads of the persistent step kernel
constexpr int SORT_ITEMS = 15;
constexpr int GATHER_BATCH = 4;   // slots per thread and iteration of the gather
// the smallest sort tile (persistent kernel): sizes the look-back buffer
constexpr int SORT_TILE_MIN = PERSIST_THREADS * SORT_ITEMS;
constexpr int REACT_THREADS = 1024;
constexpr int ITEM_HOME = 32;   // most home species per pair-search work item (one cell)
constexpr int N_FWD = 14;       // own cell + 13 forward neighbour cells (half shell)
constexpr double END_SLACK = 1.0 + 1e-6;    // last-step trim slack (relative)
constexpr float CELL_SLACK_F = 1.0001f;    // hash cell >= cutoff * CELL_SLACK_F
constexpr long long SPIN_LIMIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// Chemistry shared by all trains of a context (Table 1, Table S2).
struct Tables {
  int n_types, n_rxn;
  double D[MAXT];
  float Df[MAXT];
  int8_t pair_rxn[MAXT][MAXT];  // reaction index of a type pair, -1 if none
  uint32_t reactive_mask[MAXT]; // bit j set when types (i, j) react
  double R[MAXR], D_AB[MAXR];   // radius (nm) and D_A + D_B
  float Rf[MAXR], D_ABf[MAXR];
  int n_prod[MAXR];
  int prod[MAXR][3];
  int water[MAXR];
  int rxn_a[MAXR], rxn_b[MAXR]; // reactant types of each reaction
  double k_tab[MAXR];           // rate constant as tabulated (L mol^-1 s^-1; self: 2k)
};

// Per-train state. Constants are written at init; the clock and tallies live here on
// the device in FP64 / int64 and are read back by the host only on request.
struct Train {
  // constants
  double L, halfL, dt_min, dt_max, dt_growth, dt_L, c, horizon;
  uint32_t key0, key1;
  int reset_on_release;
  int n_max;               // cells per axis limit used at run time (<= n_alloc)
  int n_alloc;             // cells per axis the hash table is allocated for
  int cb_alloc;            // bits per axis of the allocated hash (n_alloc <= 2^cb_alloc)
  int cb;                  // bits per axis of this step's cell index (n < 2^cb <= 2^cb_alloc,
                           // so the all-ones index is no cell): fewer key bits, fewer radix
                           // passes on coarse grids
  int cb_ref;              // the same for the grid that cell_sorted refers to
  double inv_L;
  uint32_t cell_base;      // first global cell of this train
  uint32_t pend_base;      // first pending slot of this train
  uint32_t pend_cap;
  uint32_t id_limit;       // ids must stay below this
  // clock and tallies
  double t, t_end, dt_cur, t_last_release;
  uint32_t step, next_id;
  uint32_t p_head, p_tail; // pending queue [p_head, p_tail) relative to pend_base
  long long species_steps, water;
  long long counts[MAXT];
  long long events[MAXR];
  // grid that cell_sorted of this train refers to (FP32-local offsets too)
  int n_ref;
  double h_ref;
  // per step, written by the begin phase
  int active, free_jump;
  double dt, t_next, t_start;
  int n;                   // cells per axis this step
  double h, inv_h;
  float hf, inv_hf;
  double rc2[MAXR];
  float rc2f[MAXR];
  double rc2_tt[MAXT * MAXT];  // squared cutoff of each type pair (-1: no reaction)
  float rc2f_tt[MAXT * MAXT];
  float rc2w_tt[MAXT * MAXT];  // FP32 bound above rc2_tt by more than any FP32-offset error
  double sig[MAXT];        // sqrt(2 D dt) per type
  float sigf[MAXT];
  double ddt[MAXR];        // D_AB dt per reaction (bridge denominator)
  float inv_ddt_f[MAXR];   // 1 / (D_AB dt) in FP32 (first tier of the acceptance test)
  uint32_t rel_n, rel_off, rel_id0, rel_p0;
  uint32_t pref0;          // product prefix of this train's first event (this step)
  uint32_t prods_step;     // products created by this train this step
  long long n_live_step;
  uint32_t n_events_step;
  uint32_t pad_;
  // homogeneous (beam-off) stage: set by the host for the stage being launched, then
  // its results; the survivors wait in mat_n until the next release re-creates them
  int hx_sel;
  uint32_t hx_stage;       // stages taken so far (Philox counter of the rounding)
  uint32_t mat_n;          // survivors to re-create at the next release
  uint32_t rel_mat;        // of this step's releases, the re-created survivors (first)
  uint32_t mat_cum[MAXT];  // survivors of types <= t (inclusive prefix)
  // parking (batched contexts): the species of a train that does not advance are moved
  // out of the stepped slots, so that idle trains cost no diffusion, sort or gather, and
  // come back as the first releases of the train's next step
  uint32_t park_base;      // first slot of this train in the parking buffers
  uint32_t park_cap;       // slots there (the train's species capacity)
  uint32_t park_n;         // species parked
  uint32_t park_now;       // this step moves the train's species to the parking buffers
  uint32_t rel_park;       // of this step's releases, the unparked species (first)
  double hx_t_end;
  double hx_e[MAXR];       // real extents of the last stage (events)
  long long hx_E[MAXR];    // whole events of the last stage
  long long hx_steps;      // accepted integrator steps of the last stage
};

// Context-wide counters.
struct Global {
  uint32_t n_total;      // slots in use: sorted live + appended products/releases
  uint32_t n_dead;       // dead marks among them (removed by the next sort)
  uint32_t n_live;       // after the gather: live slots [0, n_live)
  uint32_t n_released;
  uint32_t n_cand, n_events, n_products;
  uint32_t epoch;        // per-step stamp, also the look-back epoch base
  int status;            // chem_status raised on the device
  uint32_t any_active;
  uint32_t ev_log_n, step_log_n;
  uint32_t hist[MAX_PASSES][RADIX];
  uint32_t tile_ctr[MAX_PASSES];
  uint32_t bar_count, bar_gen;  // grid barrier of the persistent launch
  uint32_t err_where;
  uint32_t steps_active;  // steps in which at least one train advanced
  uint32_t n_items;       // pair-search work items emitted by the gather
  uint32_t item_home;     // home species per cell-tile work item (<= ITEM_HOME; 0: no tiles)
  uint32_t search_adaptive;   // choose the search mapping per step (below)
  uint32_t search_cells_now;  // this step's mapping: 1 cell tiles, 0 one thread per species
  uint32_t n_conflict;    // accepted pairs sharing a species with another accepted pair
  uint32_t item_ctr;      // next pair-search work item (work stealing)
  uint32_t sort_parity;   // number of non-trivial passes of this step's cell sort, mod 2
  uint32_t sort_any;      // at least one pass executed (else the order is unchanged)
  uint32_t ev_parity;     // event order in ev_v1 (1) or ev_v0 (0), prefix in the other key buffer
  uint32_t never_set;     // stays 0: the word chem_check_bounded_wait waits for
  // which branches reaction resolution took (cumulative since the last reset)
  uint32_t react_rounds_global;  // steps whose conflict rounds ran in global memory
  uint32_t react_order_global;   // steps whose event order ran in global memory
  uint32_t react_order_radix;    // steps whose shared-memory event order needed the radix sort
  uint32_t max_conflict;         // most conflicting accepted pairs in one step
  uint32_t max_events;           // most events in one step
  // pair-search work (cumulative since the last reset)
  unsigned long long pairs_tested;     // neighbour pairs whose separation was tested
  unsigned long long pairs_in_cutoff;  // of them, reacting type pairs inside the cutoff
  unsigned long long pairs_accepted;   // of them, accepted (the steps' reactive pairs)
  unsigned long long incut_mark;       // pairs_in_cutoff when the last step began
  uint32_t cells_steps;                // steps searched with cell tiles (cumulative)
  uint32_t sentinel_step;              // key of removed species this step: above every cell
                                       // key of the step (one train: the unused all-ones cell)
};

// Accepted reactive pair.
struct Cand {
  uint32_t s_lo, s_hi;   // slots in S (lo = lower id)
  uint32_t id_lo, id_hi;
  uint32_t rxn_train;    // rxn | train << 8
  uint32_t pad;
  double d1sq;           // squared end-of-step separation (FP64 mode: exact FP64)
};

// Everything a kernel needs, passed by value.
struct Dev {
  uint32_t cap, cap_cand, cap_ev_log, cap_step_log, cap_pend;
  uint32_t n_trains, total_cells, sentinel;
  int passes, precision;
  int train_bits;        // bits of (n_trains - 1): event key = train << (32 - bits) | id_lo
  double* sx; double* sy; double* sz; uint32_t* stid;
  double* tx; double* ty; double* tz; uint32_t* ttid;
  float4* s4; float4* t4;
  double* tdx; double* tdy; double* tdz;  // FP64 displacement of this step, pre-sort order
  float4* td4;                            // FP32-local displacement of this step, pre-sort order
  float4* sd4;                            // the same in sorted order (gathered with the state)
  // parking buffers (batched contexts; nullptr otherwise): the state and cell key of
  // species of idle trains, per train from Train::park_base
  float4* pk4; uint32_t* pk_cell;
  double* pkx; double* pky; double* pkz; uint32_t* pk_tid;
  uint2* items;                           // pair-search work items {first home slot, cell}
  uint32_t cap_items;
  uint32_t* cell_sorted;
  uint32_t* keys0; uint32_t* keys1; uint32_t* vals0; uint32_t* vals1;
  uint8_t* dead;
  uint32_t* touch;       // accepted pairs per slot this step (zero between steps)
  int4* cell_info;
  uint32_t* occ;         // occupancy bitmap, one bit per cell, rebuilt every step
  uint32_t occ_vec4;     // its size in 16-byte words
  unsigned long long* lookback;
  uint32_t max_tiles;
  Cand* cand;
  uint32_t* ev_list;     // committed candidate indices (cap_cand)
  uint32_t* alive0; uint32_t* alive1;
  uint32_t* ev_k0; uint32_t* ev_k1; uint32_t* ev_v0; uint32_t* ev_v1;
  chem_event* ev_log;
  chem_step_record* step_log;
  int32_t* p_type; double* px; double* py; double* pz; double* pt;
  Train* trains;
  const Tables* tables;
  Global* g;
};

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ void raise_status(Global* g, int code) {
  atomicCAS(&g->status, 0, code);
}

__device__ __forceinline__ uint32_t tid_type(uint32_t tid) { return tid & 7u; }
__device__ __forceinline__ uint32_t tid_id(uint32_t tid) { return tid >> 3; }

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Local cell index with power-of-two strides: ix | iy << cb | iz << 2 cb.
__device__ __forceinline__ uint32_t cell_encode(int ix, int iy, int iz, int cb) {
  return static_cast<uint32_t>(ix) | (static_cast<uint32_t>(iy) << cb) |
         (static_cast<uint32_t>(iz) << (2 * cb));
}
__device__ __forceinline__ void cell_decode(uint32_t loc, int cb, int& ix, int& iy, int& iz) {
  const uint32_t m = (1u << cb) - 1u;
  ix = static_cast<int>(loc & m);
  iy = static_cast<int>((loc >> cb) & m);
  iz = static_cast<int>(loc >> (2 * cb));
}
// i + d wrapped into [0, n) for |d| <= n.
__device__ __forceinline__ int step_cell(int i, int d, int n) {
  i += d;
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Train owning a global cell: largest b with cell_base[b] <= cell (bases ascending).
__device__ __forceinline__ int train_of_cell(const Train* tr, int n_trains, uint32_t cell) {
  int lo = 0, hi = n_trains - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tr[mid].cell_base <= cell) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: 10 rounds of two 32x32->64 multiplies; the high
// halves are XORed with the other words and the round key, the key is bumped by the
// Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Lanes of the warp whose 8-bit digit equals this lane's, among the lanes in `active`:
// eight ballots, a fixed cost whatever the number of distinct digits. Every lane of the
// warp must call it.
__device__ __forceinline__ uint32_t match_digit8(uint32_t digit, uint32_t active) {
  uint32_t peers = active;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const uint32_t bit = (digit >> b) & 1u;
    const uint32_t m = __ballot_sync(0xffffffffu, bit != 0u);
    peers &= bit ? m : ~m;
  }
  return peers;
}

__device__ __forceinline__ unsigned long long u53(uint32_t hi, uint32_t lo) {
  return ((static_cast<unsigned long long>(hi) << 32) | lo) >> 11;
}

}  // namespace chem
