// chem_step_noalloc: one FP64 SBS step of a small pulse train whose species live in the
// caller's device buffers, for callers that cannot allocate device memory themselves or
// let a library do it: code that runs under another framework's memory pool (which owns
// the whole device and forbids cudaMalloc), allocation-free real-time loops, or hosts
// whose allocator must not be re-entered from a library. All working memory of the
// step's kernels (sorted state, hash cells, radix buffers, candidate and event lists,
// per-train and global counters) lives in the file-scope array `g_noalloc_scratch`
// below: a fixed NOALLOC_SCRATCH_BYTES that every GPU that loads this library keeps
// until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>

#include "launch.h"
#include "sbs_device.cuh"

using namespace chem;

namespace {

constexpr uint32_t NA_MAX_SPECIES = CHEM_NOALLOC_MAX_SPECIES;
constexpr uint32_t NA_MAX_CAND = CHEM_NOALLOC_MAX_SPECIES;
constexpr uint32_t NA_MAX_EVENTS = CHEM_NOALLOC_MAX_SPECIES / 2;
constexpr int NA_CELLS_AXIS = 32;
constexpr uint32_t NA_CELLS = NA_CELLS_AXIS * NA_CELLS_AXIS * NA_CELLS_AXIS;
constexpr uint32_t NA_TILES = NA_MAX_SPECIES / SORT_TILE_MIN + 2;

constexpr size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Byte layout of the scratch array.
struct Layout {
  size_t sx, sy, sz, stid, tx, ty, tz, ttid, tdx, tdy, tdz, s4, t4, items, touch, cell_sorted, sortbuf, dead, cell_info, occ, lookback, cand,
      ev_list, alive0, alive1, ev_k0, ev_k1, ev_v0, ev_v1, ev_log, step_log, pend, trains, tables,
      global, total;
};

constexpr Layout make_layout() {
  Layout L{};
  size_t o = 0;
  auto take = [&o](size_t bytes) { size_t at = o; o += align256(bytes); return at; };
  const size_t M = NA_MAX_SPECIES, C = NA_MAX_CAND;
  L.sx = take(M * 8); L.sy = take(M * 8); L.sz = take(M * 8); L.stid = take(M * 4);
  L.tx = take(M * 8); L.ty = take(M * 8); L.tz = take(M * 8); L.ttid = take(M * 4);
  L.tdx = take(M * 8); L.tdy = take(M * 8); L.tdz = take(M * 8);
  L.s4 = take(M * 16); L.t4 = take(M * 16);  // FP32 cell offsets (the search's prefilter)
  L.items = take((M + M / ITEM_HOME + 64) * 8);
  L.touch = take(M * 4);
  L.cell_sorted = take(M * 4);
  L.sortbuf = take(M * 16);
  L.dead = take(M);
  L.cell_info = take((NA_CELLS + 1) * 16);
  L.occ = take((NA_CELLS + 127) / 128 * 16);
  L.lookback = take(static_cast<size_t>(NA_TILES) * RADIX * 8);
  L.cand = take(C * sizeof(Cand));
  L.ev_list = take(C * 4); L.alive0 = take(C * 4); L.alive1 = take(C * 4);
  L.ev_k0 = take(C * 4); L.ev_k1 = take(C * 4); L.ev_v0 = take(C * 4); L.ev_v1 = take(C * 4);
  L.ev_log = take(NA_MAX_EVENTS * sizeof(chem_event));
  L.step_log = take(sizeof(chem_step_record));
  L.pend = take(64);
  L.trains = take(sizeof(Train));
  L.tables = take(sizeof(Tables));
  L.global = take(sizeof(Global));
  L.total = o;
  return L;
}

constexpr Layout LAYOUT = make_layout();
constexpr size_t NOALLOC_SCRATCH_BYTES = LAYOUT.total;

}  // namespace

// The shared working memory of chem_step_noalloc (about 4.2 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch per device, looked up once per device.
std::mutex g_addr_mu;
void* g_addr[64] = {};

__global__ void k_noalloc_setup(Dev d, Tables tb, Train tr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *const_cast<Tables*>(d.tables) = tb;
    *d.trains = tr;
    Global g;
    std::memset(&g, 0, sizeof(g));
    g.item_home = ITEM_HOME;
    *d.g = g;
  }
}

// Copy the caller's species into the scratch state. The inputs live on the device, so
// they are checked here: a type outside [0, n_types), an id at or above the id limit (it
// would overlap the type bits) or a position that is not finite and inside [-L/2, L/2)^3
// raises CHEM_EINVAL and is not written; every later phase then does nothing and the
// store kernel reports no species and no events.
__global__ void k_noalloc_load(Dev d, int32_t n, const uint32_t* id, const int32_t* type,
                               const double* xyz) {
  const Train& tr = d.trains[0];
  const int n_types = d.tables->n_types;
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int32_t ty = type[s];
    const uint32_t ids = id[s];
    const double x = xyz[3 * s], y = xyz[3 * s + 1], z = xyz[3 * s + 2];
    // written so that NaN fails every comparison
    const bool in_box = x >= -tr.halfL && x < tr.halfL && y >= -tr.halfL && y < tr.halfL &&
                        z >= -tr.halfL && z < tr.halfL;
    if (ty < 0 || ty >= n_types || ids >= tr.id_limit || !in_box) {
      raise_status(d.g, CHEM_EINVAL);
      continue;
    }
    d.sx[s] = x;
    d.sy[s] = y;
    d.sz[s] = z;
    d.stid[s] = (ids << 3) | static_cast<uint32_t>(ty);
    d.cell_sorted[s] = 0;
    d.dead[s] = 0;
    atomicAdd(reinterpret_cast<unsigned long long*>(&d.trains[0].counts[ty]), 1ull);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) d.g->n_total = static_cast<uint32_t>(n);
}

// Copy the live species (slot order) and this step's events to the caller's buffers.
__global__ void k_noalloc_store(Dev d, uint32_t* id_out, int32_t* type_out, double* xyz_out,
                                int32_t* n_out, uint32_t* next_id_out, chem_event* ev_out,
                                int32_t* n_ev_out) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  const uint32_t n = d.g->status == 0 ? d.g->n_total : 0u;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t s = base + threadIdx.x;
    const uint32_t live = (s < n && !d.dead[s]) ? 1u : 0u;
    uint32_t x = live;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    uint32_t add = 0, tot = 0;
    for (int i = 0; i < nw; ++i) {
      if (i < w) add += warp_tot[i];
      tot += warp_tot[i];
    }
    if (live) {
      const uint32_t k = carry + add + x - 1;
      const uint32_t t = d.stid[s];
      id_out[k] = t >> 3;
      type_out[k] = static_cast<int32_t>(t & 7u);
      xyz_out[3 * k] = d.sx[s];
      xyz_out[3 * k + 1] = d.sy[s];
      xyz_out[3 * k + 2] = d.sz[s];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  const uint32_t ne = d.g->status == 0 ? min(d.g->ev_log_n, d.cap_ev_log) : 0u;
  for (uint32_t e = threadIdx.x; e < ne; e += blockDim.x) ev_out[e] = d.ev_log[e];
  if (threadIdx.x == 0) {
    *n_out = static_cast<int32_t>(carry);
    *next_id_out = d.trains[0].next_id;
    *n_ev_out = static_cast<int32_t>(ne);
  }
}

chem_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return CHEM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CHEM_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return CHEM_OK;
}

}  // namespace

extern "C" chem_status chem_step_noalloc(const chem_config* cfg, uint32_t step, double t_s, double dt_s,
                                         uint32_t next_id, int32_t n, const uint32_t* id,
                                         const int32_t* type, const double* xyz, uint32_t* id_out,
                                         int32_t* type_out, double* xyz_out, int32_t* n_out,
                                         uint32_t* next_id_out, chem_event* events_out,
                                         int32_t* n_events_out) {
  if (!cfg || n < 0 || !n_out || !next_id_out || !n_events_out) return CHEM_EINVAL;
  if (n > static_cast<int32_t>(NA_MAX_SPECIES)) return CHEM_ECAPACITY;
  if (n > 0 && (!id || !type || !xyz || !id_out || !type_out || !xyz_out)) return CHEM_EINVAL;
  if (!events_out) return CHEM_EINVAL;
  if (cfg->precision != CHEM_FP64) return CHEM_EINVAL;
  if (cfg->n_types < 1 || cfg->n_types > CHEM_MAX_TYPES || !cfg->D_nm2_s) return CHEM_EINVAL;
  if (cfg->n_rxn < 0 || cfg->n_rxn > CHEM_MAX_RXN || (cfg->n_rxn > 0 && !cfg->rxn)) return CHEM_EINVAL;
  if (!(cfg->L_nm > 0.0) || !std::isfinite(cfg->L_nm) || !(dt_s > 0.0) || !std::isfinite(t_s))
    return CHEM_EINVAL;
  if (!(cfg->cutoff_c >= 0.0) || next_id + static_cast<uint64_t>(n) * 3 >= (1u << 29)) return CHEM_EINVAL;

  // chemistry tables (Table 1, Table S2; R from Eq. kdiff1 with k_tab = 2k for self reactions)
  Tables tb;
  std::memset(&tb, 0, sizeof(tb));
  tb.n_types = cfg->n_types;
  tb.n_rxn = cfg->n_rxn;
  for (int t = 0; t < tb.n_types; ++t) {
    if (!(cfg->D_nm2_s[t] > 0.0)) return CHEM_EINVAL;
    tb.D[t] = cfg->D_nm2_s[t];
    tb.Df[t] = static_cast<float>(tb.D[t]);
  }
  std::memset(tb.pair_rxn, -1, sizeof(tb.pair_rxn));
  double dt_L = std::numeric_limits<double>::infinity();
  for (int r = 0; r < tb.n_rxn; ++r) {
    const chem_reaction& x = cfg->rxn[r];
    if (x.a < 0 || x.a >= tb.n_types || x.b < 0 || x.b >= tb.n_types || !(x.k_tab > 0.0) ||
        x.n_prod < 0 || x.n_prod > 3 || tb.pair_rxn[x.a][x.b] >= 0)
      return CHEM_EINVAL;
    for (int q = 0; q < x.n_prod; ++q)
      if (x.prod[q] < 0 || x.prod[q] >= tb.n_types) return CHEM_EINVAL;
    tb.pair_rxn[x.a][x.b] = tb.pair_rxn[x.b][x.a] = static_cast<int8_t>(r);
    tb.reactive_mask[x.a] |= 1u << x.b;
    tb.reactive_mask[x.b] |= 1u << x.a;
    tb.D_AB[r] = tb.D[x.a] + tb.D[x.b];
    tb.R[r] = (x.k_tab * 1e24 / 6.02214076e23) / (4.0 * 3.141592653589793 * tb.D_AB[r]);
    tb.Rf[r] = static_cast<float>(tb.R[r]);
    tb.D_ABf[r] = static_cast<float>(tb.D_AB[r]);
    tb.n_prod[r] = x.n_prod;
    for (int q = 0; q < 3; ++q) tb.prod[r][q] = q < x.n_prod ? x.prod[q] : 0;
    tb.water[r] = x.water_delta;
    const double room = cfg->L_nm / 3.0 - tb.R[r];
    if (!(room > 0.0)) return CHEM_EINVAL;
    if (cfg->cutoff_c > 0.0) {
      const double q = room / cfg->cutoff_c;
      dt_L = std::min(dt_L, q * q / (2.0 * tb.D_AB[r]));
    }
  }
  if (dt_s > dt_L) return CHEM_EINVAL;  // the step would be shortened

  Train tr;
  std::memset(&tr, 0, sizeof(tr));
  tr.L = cfg->L_nm;
  tr.halfL = 0.5 * cfg->L_nm;
  tr.dt_min = tr.dt_max = tr.dt_cur = dt_s;
  tr.dt_growth = 1.0;
  tr.dt_L = dt_L;
  tr.c = cfg->cutoff_c;
  tr.key0 = static_cast<uint32_t>(cfg->seed & 0xFFFFFFFFull);
  tr.key1 = static_cast<uint32_t>(cfg->seed >> 32) ^ cfg->train_id;
  tr.n_max = NA_CELLS_AXIS;
  tr.n_alloc = NA_CELLS_AXIS;
  tr.cb = tr.cb_ref = tr.cb_alloc = 5;  // 32 = 2^5 cells per axis
  tr.inv_L = 1.0 / cfg->L_nm;
  tr.id_limit = (1u << 29) - 1u;
  tr.t = t_s;
  tr.t_end = std::numeric_limits<double>::infinity();
  tr.t_last_release = t_s;
  tr.step = step;
  tr.next_id = next_id;
  tr.n_ref = NA_CELLS_AXIS;
  tr.h_ref = cfg->L_nm / NA_CELLS_AXIS;

  void* base = nullptr;
  if (scratch_address(&base) != CHEM_OK) return CHEM_ECUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  Dev d;
  std::memset(&d, 0, sizeof(d));
  d.cap = NA_MAX_SPECIES;
  d.cap_cand = NA_MAX_CAND;
  d.cap_ev_log = NA_MAX_EVENTS;
  d.cap_step_log = 0;
  d.cap_pend = 1;
  d.n_trains = 1;
  d.total_cells = NA_CELLS;
  d.sentinel = NA_CELLS;
  d.passes = 2;  // keys < 2^16
  d.precision = CHEM_FP64;
  d.sx = reinterpret_cast<double*>(b + LAYOUT.sx);
  d.sy = reinterpret_cast<double*>(b + LAYOUT.sy);
  d.sz = reinterpret_cast<double*>(b + LAYOUT.sz);
  d.stid = reinterpret_cast<uint32_t*>(b + LAYOUT.stid);
  d.tx = reinterpret_cast<double*>(b + LAYOUT.tx);
  d.ty = reinterpret_cast<double*>(b + LAYOUT.ty);
  d.tz = reinterpret_cast<double*>(b + LAYOUT.tz);
  d.ttid = reinterpret_cast<uint32_t*>(b + LAYOUT.ttid);
  d.tdx = reinterpret_cast<double*>(b + LAYOUT.tdx);
  d.tdy = reinterpret_cast<double*>(b + LAYOUT.tdy);
  d.tdz = reinterpret_cast<double*>(b + LAYOUT.tdz);
  d.s4 = reinterpret_cast<float4*>(b + LAYOUT.s4);
  d.t4 = reinterpret_cast<float4*>(b + LAYOUT.t4);
  d.items = reinterpret_cast<uint2*>(b + LAYOUT.items);
  d.touch = reinterpret_cast<uint32_t*>(b + LAYOUT.touch);
  d.cap_items = NA_MAX_SPECIES + NA_MAX_SPECIES / ITEM_HOME + 64;
  d.cell_sorted = reinterpret_cast<uint32_t*>(b + LAYOUT.cell_sorted);
  uint32_t* sortbuf = reinterpret_cast<uint32_t*>(b + LAYOUT.sortbuf);
  d.keys0 = sortbuf;
  d.keys1 = sortbuf + NA_MAX_SPECIES;
  d.vals0 = sortbuf + 2 * NA_MAX_SPECIES;
  d.vals1 = sortbuf + 3 * NA_MAX_SPECIES;
  d.dead = b + LAYOUT.dead;
  d.cell_info = reinterpret_cast<int4*>(b + LAYOUT.cell_info);
  d.occ = reinterpret_cast<uint32_t*>(b + LAYOUT.occ);
  d.occ_vec4 = (NA_CELLS + 127) / 128;
  d.lookback = reinterpret_cast<unsigned long long*>(b + LAYOUT.lookback);
  d.max_tiles = NA_TILES;
  d.cand = reinterpret_cast<Cand*>(b + LAYOUT.cand);
  d.ev_list = reinterpret_cast<uint32_t*>(b + LAYOUT.ev_list);
  d.alive0 = reinterpret_cast<uint32_t*>(b + LAYOUT.alive0);
  d.alive1 = reinterpret_cast<uint32_t*>(b + LAYOUT.alive1);
  d.ev_k0 = reinterpret_cast<uint32_t*>(b + LAYOUT.ev_k0);
  d.ev_k1 = reinterpret_cast<uint32_t*>(b + LAYOUT.ev_k1);
  d.ev_v0 = reinterpret_cast<uint32_t*>(b + LAYOUT.ev_v0);
  d.ev_v1 = reinterpret_cast<uint32_t*>(b + LAYOUT.ev_v1);
  d.ev_log = reinterpret_cast<chem_event*>(b + LAYOUT.ev_log);
  d.step_log = reinterpret_cast<chem_step_record*>(b + LAYOUT.step_log);
  d.p_type = reinterpret_cast<int32_t*>(b + LAYOUT.pend);
  d.px = d.py = d.pz = d.pt = reinterpret_cast<double*>(b + LAYOUT.pend + 16);
  d.trains = reinterpret_cast<Train*>(b + LAYOUT.trains);
  d.tables = reinterpret_cast<const Tables*>(b + LAYOUT.tables);
  d.g = reinterpret_cast<Global*>(b + LAYOUT.global);

  int dev = 0, sms = 0, sort_occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sort_pass_occupancy(&sort_occ) != cudaSuccess || sms < 1 || sort_occ < 1) {
    cudaGetLastError();
    return CHEM_ECUDA;
  }
  LaunchCfg lc;
  lc.stream_blocks = std::max(1, std::min(sms * 2, (n + 255) / 256 + 1));
  lc.search_blocks = lc.stream_blocks;
  lc.sort_blocks = std::min(sms * sort_occ, static_cast<int>(NA_TILES));
  lc.persistent_blocks = 1;
  lc.search_tps = 0;
  cudaStream_t s = static_cast<cudaStream_t>(cfg->cuda_stream);
  // leftovers of the previous call: stale hash cells and look-back words must not match
  bool ok = cudaMemsetAsync(d.cell_info, 0xFF, (NA_CELLS + 1) * 16, s) == cudaSuccess &&
            cudaMemsetAsync(d.occ, 0, (NA_CELLS + 127) / 128 * 16, s) == cudaSuccess &&
            cudaMemsetAsync(d.touch, 0, NA_MAX_SPECIES * 4, s) == cudaSuccess &&
            cudaMemsetAsync(d.lookback, 0, static_cast<size_t>(NA_TILES) * RADIX * 8, s) == cudaSuccess;
  if (ok) {
    k_noalloc_setup<<<1, 1, 0, s>>>(d, tb, tr);
    k_noalloc_load<<<lc.stream_blocks, 256, 0, s>>>(d, n, id, type, xyz);
    ok = cudaGetLastError() == cudaSuccess && enqueue_step_f64(d, lc, s, nullptr, true, true) == cudaSuccess;
  }
  if (ok) {
    k_noalloc_store<<<1, 1024, 0, s>>>(d, id_out, type_out, xyz_out, n_out, next_id_out, events_out,
                                       n_events_out);
    ok = cudaGetLastError() == cudaSuccess;
  }
  int status = 0;
  if (ok) ok = cudaMemcpyAsync(&status, &d.g->status, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (ok) ok = cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return CHEM_ECUDA;
  }
  return static_cast<chem_status>(status);
}
