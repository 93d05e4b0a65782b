// Host side of the C ABI declared in include/chem.h: validation, device allocation,
// the pending-species queue, CUDA-graph capture of the step kernels and the run loop.
// The host never computes a step: it only queues kernels and copies data.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <limits>
#include <string>
#include <thread>
#include <vector>

#include "launch.h"
#include "sbs_device.cuh"

using namespace chem;

namespace {

constexpr double N_AVOGADRO = 6.02214076e23;
constexpr double PI = 3.141592653589793;

// One train's pending species on the host (arrival, position, type), in page-locked
// memory so that the copy to the device queue runs at full link speed.
struct PendingBuf {
  size_t cap = 0;
  double* t = nullptr;   // one block: t, x, y, z (cap each), then type
  double* x = nullptr;
  double* y = nullptr;
  double* z = nullptr;
  int32_t* type = nullptr;
  bool reserve(size_t want) {
    if (want <= cap) return true;
    release();
    void* p = nullptr;
    if (cudaHostAlloc(&p, want * (4 * sizeof(double) + sizeof(int32_t)), cudaHostAllocDefault) != cudaSuccess)
      return false;
    t = static_cast<double*>(p);
    x = t + want; y = x + want; z = y + want;
    type = reinterpret_cast<int32_t*>(z + want);
    cap = want;
    return true;
  }
  void release() {
    if (t) cudaFreeHost(t);
    t = x = y = z = nullptr;
    type = nullptr;
    cap = 0;
  }
};

// Mirror of the device queue [0, p_tail) of one train; the merge of a new injection
// writes the spare buffer, which then becomes the current one.
struct PendingHost {
  PendingBuf buf[2];
  int cur = 0;
  size_t n = 0;
  size_t size() const { return n; }
  void clear() { n = 0; }
  void release() { buf[0].release(); buf[1].release(); n = 0; }
};

struct TrainHost {
  chem_config cfg;
  double E_dep = 0.0;
  PendingHost pend;   // mirror of the device queue [0, p_tail)
};

}  // namespace

struct chem_ctx {
  int B = 0;
  int precision = CHEM_FP64;
  std::vector<TrainHost> th;
  Tables tables{};
  Dev d{};
  LaunchCfg lc{};
  int sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  chem_alloc_fn alloc = nullptr;
  chem_free_fn dfree = nullptr;
  void* alloc_user = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  bool graph_events = false;  // the captured graph records the phase events
  int steps_per_launch = 16;
  bool persistent = false;
  int cell_factor_x100 = 1600;  // hash cells per species (x100) of the runtime grid limit
  // radix passes of the cell sort: with one train only as many as the runtime grid limit
  // needs (pass_nmax cells per axis at most, and pass_cbref bits per axis for the cells
  // the species were last sorted in); with several trains all of the allocated key bits
  int passes_alloc = 1;
  int cb_alloc0 = 0;
  int pass_nmax = 3;
  int pass_cbref = 0;
  int item_home = -1;            // pair search: 0 = one thread per home species, 1..32 =
                                 // cell tiles of that many homes, -1 = chosen per step
  Global* g_pinned = nullptr;  // host copy of the global counters
  double* t_end_pinned = nullptr;
  double* t_end_dev = nullptr;
  bool profiling = false;
  std::vector<cudaEvent_t> events;  // 2 * N_PHASES per captured step when profiling
  chem_stats stats{};
  uint32_t seen_rounds_global = 0, seen_order_global = 0, seen_order_radix = 0;  // device counters seen
  unsigned long long seen_tested = 0, seen_in_cut = 0, seen_accepted = 0;
  uint32_t seen_steps = 0, seen_cells_steps = 0;
  std::string err;
  chem_status status = CHEM_OK;
};

namespace {

chem_status fail(chem_ctx* c, chem_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) {
    if (c->status == CHEM_OK) {
      c->status = s;
      c->err = buf;
    }
  }
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, CHEM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

void* dev_alloc(chem_ctx* ctx, size_t bytes) {
  bytes = (bytes + 255) & ~static_cast<size_t>(255);
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (ctx->alloc) {
    p = ctx->alloc(bytes, ctx->alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) ctx->allocs.emplace_back(p, bytes);
  return p;
}

void release_all(chem_ctx* ctx) {
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  ctx->graph = nullptr;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& a : ctx->allocs) {
    if (ctx->dfree) ctx->dfree(a.first, a.second, ctx->alloc_user);
    else cudaFree(a.first);
  }
  ctx->allocs.clear();
  for (TrainHost& h : ctx->th) h.pend.release();
  if (ctx->g_pinned) cudaFreeHost(ctx->g_pinned);
  if (ctx->t_end_pinned) cudaFreeHost(ctx->t_end_pinned);
  ctx->g_pinned = nullptr;
  ctx->t_end_pinned = nullptr;
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  ctx->events.clear();
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  ctx->stream = nullptr;
}

int bits_for(uint64_t v) {
  int b = 0;
  while ((1ull << b) <= v) ++b;
  return b;
}

chem_status validate(const chem_config* cfgs, int B) {
  if (!cfgs || B < 1 || B > MAX_TRAINS) return CHEM_EINVAL;
  const chem_config& c0 = cfgs[0];
  for (int b = 0; b < B; ++b) {
    const chem_config& c = cfgs[b];
    if (c.n_types < 1 || c.n_types > CHEM_MAX_TYPES || !c.D_nm2_s) return CHEM_EINVAL;
    if (c.n_rxn < 0 || c.n_rxn > CHEM_MAX_RXN || (c.n_rxn > 0 && !c.rxn)) return CHEM_EINVAL;
    if (c.precision != CHEM_FP64 && c.precision != CHEM_FP32_LOCAL) return CHEM_EINVAL;
    if (!(c.L_nm > 0.0) || !std::isfinite(c.L_nm)) return CHEM_EINVAL;
    if (!(c.dt_min_s > 0.0) || !(c.dt_max_s >= c.dt_min_s) || !(c.dt_growth >= 1.0)) return CHEM_EINVAL;
    if (!(c.cutoff_c >= 0.0) || !(c.sbs_horizon_s >= 0.0)) return CHEM_EINVAL;
    if (c.capacity_species < 1 || c.capacity_species > (1ll << 30)) return CHEM_EINVAL;
    if (c.capacity_pending < 0 || c.capacity_candidates < 0) return CHEM_EINVAL;
    if (c.capacity_event_log < 0 || c.capacity_step_log < 0) return CHEM_EINVAL;
    if (c.n_types != c0.n_types || c.n_rxn != c0.n_rxn || c.precision != c0.precision) return CHEM_EINVAL;
    for (int t = 0; t < c.n_types; ++t) {
      if (!(c.D_nm2_s[t] > 0.0) || c.D_nm2_s[t] != c0.D_nm2_s[t]) return CHEM_EINVAL;
    }
    for (int r = 0; r < c.n_rxn; ++r) {
      const chem_reaction& x = c.rxn[r];
      if (x.a < 0 || x.a >= c.n_types || x.b < 0 || x.b >= c.n_types) return CHEM_EINVAL;
      if (!(x.k_tab > 0.0) || x.n_prod < 0 || x.n_prod > 3) return CHEM_EINVAL;
      for (int q = 0; q < x.n_prod; ++q)
        if (x.prod[q] < 0 || x.prod[q] >= c.n_types) return CHEM_EINVAL;
      if (std::memcmp(&x, &c0.rxn[r], sizeof(chem_reaction)) != 0) return CHEM_EINVAL;
    }
  }
  return CHEM_OK;
}

// Reaction radius from Eq. kdiff1 at steady state: k = 4 pi R D_AB N_A, k in L/mol/s
// (1 L = 1e24 nm^3); for self reactions k_tab is the printed 2k (Eq. kdiff2).
double reaction_radius(double k_tab, double D_AB) {
  const double k_nm3_per_s = k_tab * 1e24 / N_AVOGADRO;
  return k_nm3_per_s / (4.0 * PI * D_AB);
}

chem_status upload_trains(chem_ctx* ctx, const std::vector<Train>& h) {
  ctx->stats.bytes_h2d += static_cast<int64_t>(sizeof(Train) * h.size());
  CK(cudaMemcpyAsync(ctx->d.trains, h.data(), sizeof(Train) * h.size(), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHEM_OK;
}

chem_status download_trains(chem_ctx* ctx, std::vector<Train>& h) {
  h.resize(ctx->B);
  ctx->stats.bytes_d2h += static_cast<int64_t>(sizeof(Train) * ctx->B);
  CK(cudaMemcpyAsync(h.data(), ctx->d.trains, sizeof(Train) * ctx->B, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHEM_OK;
}

// The Global fields that select the pair-search mapping for a tuning value ih (-1
// adaptive, 0 one thread per species, 1..32 cell tiles of that many homes).
void set_mapping(Global& g, int ih) {
  g.item_home = ih < 0 ? static_cast<uint32_t>(ITEM_HOME) : static_cast<uint32_t>(ih);
  g.search_adaptive = ih < 0 ? 1u : 0u;
}

chem_status upload_mapping(chem_ctx* ctx, int ih) {
  Global g{};
  set_mapping(g, ih);
  static_assert(offsetof(Global, search_adaptive) == offsetof(Global, item_home) + 4, "adjacent fields");
  CK(cudaMemcpyAsync(&ctx->d.g->item_home, &g.item_home, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHEM_OK;
}

chem_status init_global(chem_ctx* ctx) {
  ctx->seen_rounds_global = ctx->seen_order_global = ctx->seen_order_radix = 0;
  ctx->seen_tested = ctx->seen_in_cut = ctx->seen_accepted = 0;
  ctx->seen_steps = 0;
  ctx->seen_cells_steps = 0;
  CK(cudaMemsetAsync(ctx->d.g, 0, sizeof(Global), ctx->stream));
  return upload_mapping(ctx, ctx->item_home);
}

// Fold the device's counters (reaction-resolution branches, pair-search work, steps;
// cumulative since the last reset) into the context's statistics.
void note_device_counters(chem_ctx* ctx, const Global& g) {
  chem_stats& st = ctx->stats;
  st.react_rounds_global += g.react_rounds_global - ctx->seen_rounds_global;
  st.react_order_global += g.react_order_global - ctx->seen_order_global;
  st.react_order_radix += g.react_order_radix - ctx->seen_order_radix;
  ctx->seen_rounds_global = g.react_rounds_global;
  ctx->seen_order_global = g.react_order_global;
  ctx->seen_order_radix = g.react_order_radix;
  st.max_conflict_pairs = std::max<int64_t>(st.max_conflict_pairs, g.max_conflict);
  st.max_step_events = std::max<int64_t>(st.max_step_events, g.max_events);
  st.pairs_tested += static_cast<int64_t>(g.pairs_tested - ctx->seen_tested);
  st.pairs_in_cutoff += static_cast<int64_t>(g.pairs_in_cutoff - ctx->seen_in_cut);
  st.pairs_accepted += static_cast<int64_t>(g.pairs_accepted - ctx->seen_accepted);
  st.steps_advanced += g.steps_active - ctx->seen_steps;
  ctx->seen_steps = g.steps_active;
  st.steps_cell_tiles += g.cells_steps - ctx->seen_cells_steps;
  ctx->seen_cells_steps = g.cells_steps;
  ctx->seen_tested = g.pairs_tested;
  ctx->seen_in_cut = g.pairs_in_cutoff;
  ctx->seen_accepted = g.pairs_accepted;
}

chem_status download_global(chem_ctx* ctx) {
  ctx->stats.bytes_d2h += sizeof(Global);
  CK(cudaMemcpyAsync(ctx->g_pinned, ctx->d.g, sizeof(Global), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  note_device_counters(ctx, *ctx->g_pinned);
  return CHEM_OK;
}

void init_train_dynamic(Train& t, const chem_config& c, int n_max) {
  t.t = 0.0;
  t.t_end = 0.0;
  t.dt_cur = c.dt_min_s;
  t.t_last_release = 0.0;
  t.step = 0;
  t.next_id = 0;
  t.p_head = 0;
  t.p_tail = 0;
  t.species_steps = 0;
  t.water = 0;
  for (int i = 0; i < MAXT; ++i) t.counts[i] = 0;
  for (int i = 0; i < MAXR; ++i) t.events[i] = 0;
  (void)n_max;
  t.n_ref = 0;  // chosen by the first step
  t.h_ref = 0.0;
  t.hx_sel = 0;
  t.hx_stage = 0;
  t.mat_n = 0;
  t.park_n = 0;
  t.park_now = 0;
  t.rel_park = 0;
  t.rel_mat = 0;
  t.hx_t_end = 0.0;
  t.hx_steps = 0;
  for (int i = 0; i < MAXT; ++i) t.mat_cum[i] = 0;
  for (int i = 0; i < MAXR; ++i) {
    t.hx_e[i] = 0.0;
    t.hx_E[i] = 0;
  }
  t.active = 0;
  t.free_jump = 0;
  t.key0 = static_cast<uint32_t>(c.seed & 0xFFFFFFFFull);
  t.key1 = static_cast<uint32_t>(c.seed >> 32) ^ c.train_id;
}

// Kernels of one captured step: diffusion, the sort passes, gather, the search (one or
// both mappings), fast matching, the one-CTA reaction kernel, products, and the end (or
// end-and-next-begin) kernel.
int kernels_per_step(const chem_ctx* ctx) {
  return ctx->persistent ? 0 : 6 + ctx->d.passes + (ctx->lc.search_tps == 2 ? 2 : 1);
}

// Radix passes for the captured graph (see chem_ctx::passes_alloc).
int sort_passes(const chem_ctx* ctx) {
  if (ctx->B != 1) return ctx->passes_alloc;
  const int nm = std::min(ctx->pass_nmax, (1 << ctx->cb_alloc0) - 1);
  const int cb = std::min(ctx->cb_alloc0, std::max(bits_for(static_cast<uint64_t>(nm)), ctx->pass_cbref));
  return std::max(1, std::min(ctx->passes_alloc, (3 * cb + 7) / 8));
}

chem_status capture_graph(chem_ctx* ctx) {
  ctx->lc.search_tps = ctx->item_home == 0 ? 1 : (ctx->item_home > 0 ? 0 : 2);
  ctx->d.passes = sort_passes(ctx);
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  ctx->graph_events = false;
  const size_t n_ev = (ctx->profiling && !ctx->persistent)
                          ? static_cast<size_t>(ctx->steps_per_launch) * 2 * N_PHASES : 0;
  while (ctx->events.size() < n_ev) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    ctx->events.push_back(e);
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  if (ctx->persistent) {
    e = ctx->precision == CHEM_FP64
            ? enqueue_persistent_f64(ctx->d, ctx->lc, ctx->steps_per_launch, ctx->stream)
            : enqueue_persistent_f32l(ctx->d, ctx->lc, ctx->steps_per_launch, ctx->stream);
  } else {
    for (int s = 0; s < ctx->steps_per_launch && e == cudaSuccess; ++s) {
      cudaEvent_t* ev = n_ev ? &ctx->events[static_cast<size_t>(s) * 2 * N_PHASES] : nullptr;
      const bool first = s == 0, last = s + 1 == ctx->steps_per_launch;
      e = ctx->precision == CHEM_FP64 ? enqueue_step_f64(ctx->d, ctx->lc, ctx->stream, ev, first, last)
                                      : enqueue_step_f32l(ctx->d, ctx->lc, ctx->stream, ev, first, last);
    }
  }
  cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(ctx, CHEM_ECUDA, "kernel launch during capture failed: %s", cudaGetErrorString(e));
  }
  CK(e2);
  e = cudaGraphInstantiate(&ctx->graph, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  ctx->graph_steps = ctx->steps_per_launch;
  ctx->graph_events = n_ev > 0;
  return CHEM_OK;
}

chem_status check_ctx(chem_ctx* ctx) {
  if (!ctx) return CHEM_EINVAL;
  return ctx->status;
}

chem_status run_loop(chem_ctx* ctx) {
  if (!ctx->graph) {
    chem_status s = capture_graph(ctx);
    if (s) return s;
  }
  {
    chem_status s0 = download_global(ctx);
    if (s0) return s0;
  }
  uint32_t active_before = ctx->g_pinned->steps_active;
  for (long long it = 0;; ++it) {
    CK(cudaGraphLaunch(ctx->graph, ctx->stream));
    CK(cudaMemcpyAsync(ctx->g_pinned, ctx->d.g, sizeof(Global), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const Global& g = *ctx->g_pinned;
    note_device_counters(ctx, g);
    ctx->stats.graph_replays += 1;
    ctx->stats.steps_launched += ctx->graph_steps;
    // per replay: one begin kernel, then every step's kernels (the end kernel of each step
    // but the last also begins the next)
    ctx->stats.kernel_launches += ctx->persistent ? 1 : 1 + static_cast<int64_t>(ctx->graph_steps) * kernels_per_step(ctx);
    ctx->stats.bytes_d2h += sizeof(Global);
    const uint32_t stepped = g.steps_active - active_before;
    active_before = g.steps_active;
    if (ctx->persistent) {
      ctx->stats.phase_launches[PH_PERSISTENT] += 1;
    } else if (ctx->graph_events) {
      for (uint32_t st = 0; st < stepped && st < static_cast<uint32_t>(ctx->graph_steps); ++st) {
        for (int ph = 0; ph < PH_PERSISTENT; ++ph) {
          float ms = 0.f;
          cudaEvent_t* ev = &ctx->events[static_cast<size_t>(st) * 2 * N_PHASES];
          if (cudaEventElapsedTime(&ms, ev[2 * ph], ev[2 * ph + 1]) == cudaSuccess) {
            ctx->stats.phase_ms[ph] += ms;
            ctx->stats.phase_launches[ph] += ph == PH_SORT ? ctx->d.passes : (ph == PH_RELEASE ? 0 : 1);
          } else {
            cudaGetLastError();  // a phase not timed: no error is left for the next launch check
          }
        }
      }
    }
    if (g.status != 0) {
      const char* what = g.status == CHEM_ECAPACITY ? "a device capacity was exceeded"
                         : g.status == CHEM_ETIMEOUT ? "a bounded device wait timed out"
                                                     : "device error";
      return fail(ctx, static_cast<chem_status>(g.status), "%s (status %d)", what, g.status);
    }
    if (!g.any_active) break;
    if (it > (1ll << 40)) return fail(ctx, CHEM_ESTATE, "run loop made no progress");
  }
  return CHEM_OK;
}

// fn(lo, hi) over [0, n), split between up to 16 host threads when n is large.
template <class F>
void parallel_ranges(size_t n, F fn) {
  const size_t min_chunk = size_t(1) << 16;
  const size_t hw = std::max<size_t>(1, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>({hw, 16, (n + min_chunk - 1) / min_chunk});
  if (nt <= 1) {
    fn(size_t(0), n);
    return;
  }
  const size_t step = (n + nt - 1) / nt;
  std::vector<std::thread> th;
  for (size_t k = 1; k < nt; ++k) {
    const size_t lo = k * step, hi = std::min(n, lo + step);
    if (lo < hi) th.emplace_back(fn, lo, hi);
  }
  fn(size_t(0), std::min(n, step));
  for (auto& x : th) x.join();
}

// Homogeneous stage (Sec. 2.3) of every train b with t_end[b] > its clock. Pending
// species already due join the stage; one arriving inside it is an error (EINVAL, nothing
// changed).
chem_status homogeneous_run(chem_ctx* ctx, const double* t_end) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  if (!t_end) return CHEM_EINVAL;
  for (int b = 0; b < ctx->B; ++b)
    if (!std::isfinite(t_end[b])) return CHEM_EINVAL;
  std::vector<Train> tr;
  s = download_trains(ctx, tr);
  if (s) return s;
  std::vector<size_t> due_end(ctx->B, 0);
  bool any = false;
  for (int b = 0; b < ctx->B; ++b) {
    const Train& t = tr[b];
    if (!(t_end[b] > t.t)) continue;
    const PendingHost& p = ctx->th[b].pend;
    const PendingBuf& buf = p.buf[p.cur];
    const double* first = buf.t ? buf.t + t.p_head : nullptr;
    const double* last = buf.t ? buf.t + p.size() : nullptr;
    const size_t i = t.p_head + static_cast<size_t>(first ? std::upper_bound(first, last, t.t) - first : 0);
    if (i < p.size() && buf.t[i] < t_end[b]) {
      ctx->err = "species arrive during the homogeneous stage";
      return CHEM_EINVAL;
    }
    due_end[b] = i;
    any = true;
  }
  if (!any) return CHEM_OK;
  for (int b = 0; b < ctx->B; ++b) {
    Train& t = tr[b];
    t.hx_sel = 0;
    if (!(t_end[b] > t.t)) continue;
    const PendingHost& p = ctx->th[b].pend;
    const PendingBuf& buf = p.buf[p.cur];
    for (size_t i = t.p_head; i < due_end[b]; ++i) t.counts[buf.type[i]] += 1;
    t.p_head = static_cast<uint32_t>(due_end[b]);
    t.hx_sel = 1;
    t.park_n = 0;  // parked particles are removed with the others (their counts stay)
    t.hx_t_end = t_end[b];
  }
  s = upload_trains(ctx, tr);
  if (s) return s;
  CK(enqueue_homogeneous(ctx->d, ctx->lc.stream_blocks, ctx->stream));
  ctx->stats.kernel_launches += 2;
  s = download_global(ctx);
  if (s) return s;
  const Global& g = *ctx->g_pinned;
  if (g.status != 0) {
    return fail(ctx, static_cast<chem_status>(g.status), "homogeneous stage: %s (status %d)",
                g.err_where == 0x4858u ? "rate-equation integrator step limit" : "device error", g.status);
  }
  return CHEM_OK;
}

chem_status homogeneous_report(chem_ctx* ctx, int b, double* extents, int64_t* events, int64_t* steps) {
  if (!ctx) return CHEM_EINVAL;
  if (b < 0 || b >= ctx->B) return CHEM_EINVAL;
  std::vector<Train> tr;
  chem_status s = download_trains(ctx, tr);
  if (s) return s;
  for (int r = 0; r < ctx->tables.n_rxn; ++r) {
    if (extents) extents[r] = tr[b].hx_e[r];
    if (events) events[r] = tr[b].hx_E[r];
  }
  if (steps) *steps = tr[b].hx_steps;
  return ctx->status;
}

chem_status inject_one(chem_ctx* ctx, int b, int64_t n, const int32_t* type, const double* xyz,
                       const double* t_arr, double energy_eV) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  if (b < 0 || b >= ctx->B) return CHEM_EINVAL;
  if (n < 0 || (n > 0 && (!type || !xyz || !t_arr))) return CHEM_EINVAL;
  std::vector<Train> tr;
  s = download_trains(ctx, tr);
  if (s) return s;
  Train& t = tr[b];
  TrainHost& h = ctx->th[b];
  const double halfL = t.halfL, t_now = t.t;
  const int n_types = ctx->tables.n_types;
  std::atomic<bool> bad(false);
  parallel_ranges(static_cast<size_t>(n), [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi && !bad.load(std::memory_order_relaxed); ++i) {
      bool ok = type[i] >= 0 && type[i] < n_types && t_arr[i] >= t_now && std::isfinite(t_arr[i]);
      for (int a = 0; a < 3; ++a) {
        const double v = xyz[3 * i + a];
        ok = ok && v >= -halfL && v < halfL;
      }
      if (!ok) bad.store(true, std::memory_order_relaxed);
    }
  });
  if (bad.load()) return CHEM_EINVAL;
  // drop what the device already released, merge the new species stably by arrival
  // (still-pending species first on equal arrival, new ones in call order)
  PendingHost& p = h.pend;
  const size_t head = t.p_head;
  const size_t keep = p.size() - head;
  const size_t tot = keep + static_cast<size_t>(n);
  if (tot > t.pend_cap) return fail(ctx, CHEM_ECAPACITY, "pending queue of train %d would hold %zu > %u",
                                    b, tot, t.pend_cap);
  PendingBuf& src = p.buf[p.cur];
  PendingBuf& dst = p.buf[1 - p.cur];
  if (!dst.reserve(static_cast<size_t>(t.pend_cap))) return fail(ctx, CHEM_ENOMEM, "page-locked pending buffer");
  // the new species in arrival order: the identity when already sorted (a pulse in
  // arrival order, or all at one time), else a stable sort of (arrival, index)
  std::vector<std::pair<double, uint32_t>> by_t;
  const bool sorted_new = std::is_sorted(t_arr, t_arr + n);
  if (!sorted_new) {
    by_t.resize(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) by_t[static_cast<size_t>(i)] = {t_arr[i], static_cast<uint32_t>(i)};
    std::stable_sort(by_t.begin(), by_t.end(),
                     [](const std::pair<double, uint32_t>& a, const std::pair<double, uint32_t>& c) {
                       return a.first < c.first;
                     });
  }
  const size_t nn = static_cast<size_t>(n);
  if (sorted_new && (keep == 0 || nn == 0 || src.t[head + keep - 1] <= t_arr[0])) {
    // every kept species arrives no later than the first new one: an append
    parallel_ranges(keep, [&](size_t lo, size_t hi) {
      std::memcpy(dst.t + lo, src.t + head + lo, (hi - lo) * sizeof(double));
      std::memcpy(dst.x + lo, src.x + head + lo, (hi - lo) * sizeof(double));
      std::memcpy(dst.y + lo, src.y + head + lo, (hi - lo) * sizeof(double));
      std::memcpy(dst.z + lo, src.z + head + lo, (hi - lo) * sizeof(double));
      std::memcpy(dst.type + lo, src.type + head + lo, (hi - lo) * sizeof(int32_t));
    });
    parallel_ranges(nn, [&](size_t lo, size_t hi) {
      for (size_t q = lo; q < hi; ++q) {
        const size_t k = keep + q;
        dst.t[k] = t_arr[q];
        dst.x[k] = xyz[3 * q]; dst.y[k] = xyz[3 * q + 1]; dst.z[k] = xyz[3 * q + 2];
        dst.type[k] = type[q];
      }
    });
  } else {
    size_t i = 0, j = 0;
    for (size_t k = 0; k < tot; ++k) {
      const size_t jn = j < static_cast<size_t>(n) ? (sorted_new ? j : by_t[j].second) : 0;
      const bool take_old = i < keep && (j >= static_cast<size_t>(n) || src.t[head + i] <= t_arr[jn]);
      if (take_old) {
        const size_t q = head + i++;
        dst.t[k] = src.t[q]; dst.x[k] = src.x[q]; dst.y[k] = src.y[q]; dst.z[k] = src.z[q];
        dst.type[k] = src.type[q];
      } else {
        dst.t[k] = t_arr[jn];
        dst.x[k] = xyz[3 * jn]; dst.y[k] = xyz[3 * jn + 1]; dst.z[k] = xyz[3 * jn + 2];
        dst.type[k] = type[jn];
        ++j;
      }
    }
  }
  p.cur = 1 - p.cur;
  p.n = tot;
  if (tot) {
    ctx->stats.bytes_h2d += static_cast<int64_t>(tot * (4 * sizeof(double) + sizeof(int32_t)));
    const size_t off = t.pend_base;
    CK(cudaMemcpyAsync(ctx->d.pt + off, dst.t, tot * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d.px + off, dst.x, tot * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d.py + off, dst.y, tot * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d.pz + off, dst.z, tot * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d.p_type + off, dst.type, tot * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  }
  t.p_head = 0;
  t.p_tail = static_cast<uint32_t>(tot);
  h.E_dep += energy_eV;
  return upload_trains(ctx, tr);
}

chem_status tally_one(chem_ctx* ctx, int b, int64_t* counts, double* G, int64_t* events,
                      double* t_now, int64_t* species_steps) {
  if (!ctx) return CHEM_EINVAL;
  if (b < 0 || b >= ctx->B) return CHEM_EINVAL;
  std::vector<Train> tr;
  chem_status s = download_trains(ctx, tr);
  if (s) return s;
  const Train& t = tr[b];
  const double E = ctx->th[b].E_dep;
  for (int i = 0; i < ctx->tables.n_types; ++i) {
    if (counts) counts[i] = t.counts[i];
    if (G) G[i] = E > 0.0 ? static_cast<double>(t.counts[i]) * 100.0 / E : 0.0;
  }
  for (int r = 0; r < ctx->tables.n_rxn; ++r)
    if (events) events[r] = t.events[r];
  if (t_now) *t_now = t.t;
  if (species_steps) *species_steps = t.species_steps;
  return ctx->status;
}

chem_status state_one(chem_ctx* ctx, int b, int64_t cap, int32_t* type, uint32_t* id, double* xyz,
                      int64_t* n_out) {
  if (!ctx) return CHEM_EINVAL;
  if (b < 0 || b >= ctx->B || cap < 0) return CHEM_EINVAL;
  chem_status s = download_global(ctx);
  if (s) return s;
  std::vector<Train> tr;
  s = download_trains(ctx, tr);
  if (s) return s;
  const uint32_t n_slots = ctx->g_pinned->n_total;
  // the stepped slots, then the train's parked species (idle trains of a batch)
  const uint32_t np = ctx->d.pk_cell ? tr[b].park_n : 0u, pb = tr[b].park_base;
  const uint32_t n = n_slots + np;
  std::vector<uint8_t> dead(n, 0);
  std::vector<uint32_t> cell(n), tid(n);
  std::vector<double> x(n), y(n), z(n);
  std::vector<float4> v4;
  if (ctx->precision != CHEM_FP64) v4.resize(n);
  if (n_slots) {
    CK(cudaMemcpy(dead.data(), ctx->d.dead, n_slots, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cell.data(), ctx->d.cell_sorted, n_slots * 4, cudaMemcpyDeviceToHost));
    if (ctx->precision == CHEM_FP64) {
      CK(cudaMemcpy(tid.data(), ctx->d.stid, n_slots * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(x.data(), ctx->d.sx, n_slots * 8, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(y.data(), ctx->d.sy, n_slots * 8, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(z.data(), ctx->d.sz, n_slots * 8, cudaMemcpyDeviceToHost));
    } else {
      CK(cudaMemcpy(v4.data(), ctx->d.s4, n_slots * 16, cudaMemcpyDeviceToHost));
    }
  }
  if (np) {
    CK(cudaMemcpy(cell.data() + n_slots, ctx->d.pk_cell + pb, np * 4, cudaMemcpyDeviceToHost));
    if (ctx->precision == CHEM_FP64) {
      CK(cudaMemcpy(tid.data() + n_slots, ctx->d.pk_tid + pb, np * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(x.data() + n_slots, ctx->d.pkx + pb, np * 8, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(y.data() + n_slots, ctx->d.pky + pb, np * 8, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(z.data() + n_slots, ctx->d.pkz + pb, np * 8, cudaMemcpyDeviceToHost));
    } else {
      CK(cudaMemcpy(v4.data() + n_slots, ctx->d.pk4 + pb, np * 16, cudaMemcpyDeviceToHost));
    }
  }
  int64_t k = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (dead[i]) continue;
    // train of the slot from its cell
    int tb = 0;
    for (int q = ctx->B - 1; q >= 0; --q)
      if (tr[q].cell_base <= cell[i]) { tb = q; break; }
    if (tb != b) continue;
    const Train& t = tr[b];
    uint32_t tt;
    double px, py, pz;
    if (ctx->precision == CHEM_FP64) {
      tt = tid[i]; px = x[i]; py = y[i]; pz = z[i];
    } else {
      std::memcpy(&tt, &v4[i].w, 4);
      const uint32_t loc = cell[i] - t.cell_base;
      const uint32_t m = (1u << t.cb_ref) - 1u;  // the grid of the last step
      const double h = t.h_ref;
      const int ix = static_cast<int>(loc & m), iy = static_cast<int>((loc >> t.cb_ref) & m),
                iz = static_cast<int>(loc >> (2 * t.cb_ref));
      auto wrapb = [&](double q) {
        q -= t.L * std::floor((q + t.halfL) / t.L);
        if (q >= t.halfL) q -= t.L;
        if (q < -t.halfL) q += t.L;
        return q;
      };
      px = wrapb(ix * h - t.halfL + v4[i].x);
      py = wrapb(iy * h - t.halfL + v4[i].y);
      pz = wrapb(iz * h - t.halfL + v4[i].z);
    }
    if (k < cap) {
      if (type) type[k] = static_cast<int32_t>(tt & 7u);
      if (id) id[k] = tt >> 3;
      if (xyz) { xyz[3 * k] = px; xyz[3 * k + 1] = py; xyz[3 * k + 2] = pz; }
    }
    ++k;
  }
  if (n_out) *n_out = k;
  if (k > cap) return CHEM_EINVAL;
  return ctx->status;
}

}  // namespace

extern "C" {

const char* chem_version(void) { return "chemgb 0.1 (sm_103a)"; }

const char* chem_last_error(const chem_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.empty() ? "" : ctx->err.c_str();
}

void chem_destroy(chem_ctx* ctx) {
  if (!ctx) return;
  release_all(ctx);
  delete ctx;
}

chem_status chem_batch_init(const chem_config* cfgs, int32_t n_trains, chem_ctx** out) {
  if (!out) return CHEM_EINVAL;
  *out = nullptr;
  chem_status vs = validate(cfgs, n_trains);
  if (vs) return vs;
  chem_ctx* ctx = new chem_ctx();
  const chem_config& c0 = cfgs[0];
  ctx->B = n_trains;
  ctx->precision = c0.precision;
  ctx->alloc = c0.dev_alloc;
  ctx->dfree = c0.dev_free;
  ctx->alloc_user = c0.alloc_user;
  if ((ctx->alloc == nullptr) != (ctx->dfree == nullptr)) {
    delete ctx;
    return CHEM_EINVAL;
  }
  ctx->th.resize(n_trains);
  for (int b = 0; b < n_trains; ++b) ctx->th[b].cfg = cfgs[b];
  if (c0.steps_per_launch > 0) ctx->steps_per_launch = c0.steps_per_launch;
  if (c0.launch_mode < CHEM_LAUNCH_AUTO || c0.launch_mode > CHEM_LAUNCH_PERSISTENT) {
    delete ctx;
    return CHEM_EINVAL;
  }
  ctx->persistent = c0.launch_mode == CHEM_LAUNCH_PERSISTENT ||
                    (c0.launch_mode == CHEM_LAUNCH_AUTO && n_trains > 1);

  // ---- chemistry tables
  Tables& T = ctx->tables;
  std::memset(&T, 0, sizeof(T));
  T.n_types = c0.n_types;
  T.n_rxn = c0.n_rxn;
  for (int t = 0; t < T.n_types; ++t) {
    T.D[t] = c0.D_nm2_s[t];
    T.Df[t] = static_cast<float>(c0.D_nm2_s[t]);
  }
  std::memset(T.pair_rxn, -1, sizeof(T.pair_rxn));
  for (int r = 0; r < T.n_rxn; ++r) {
    const chem_reaction& x = c0.rxn[r];
    if (T.pair_rxn[x.a][x.b] >= 0) {
      delete ctx;
      return CHEM_EINVAL;  // two reactions for one type pair
    }
    T.pair_rxn[x.a][x.b] = T.pair_rxn[x.b][x.a] = static_cast<int8_t>(r);
    T.reactive_mask[x.a] |= 1u << x.b;
    T.reactive_mask[x.b] |= 1u << x.a;
    T.D_AB[r] = T.D[x.a] + T.D[x.b];
    T.R[r] = reaction_radius(x.k_tab, T.D_AB[r]);
    T.Rf[r] = static_cast<float>(T.R[r]);
    T.D_ABf[r] = static_cast<float>(T.D_AB[r]);
    T.n_prod[r] = x.n_prod;
    for (int q = 0; q < 3; ++q) T.prod[r][q] = q < x.n_prod ? x.prod[q] : 0;
    T.water[r] = x.water_delta;
    T.rxn_a[r] = x.a;
    T.rxn_b[r] = x.b;
    T.k_tab[r] = x.k_tab;
  }

  // ---- per-train constants and global sizes
  std::vector<Train> tr(n_trains);
  uint64_t cap = 0, pend = 0, cells = 0, cand = 0, evlog = 0, steplog = 0;
  int tbits = bits_for(static_cast<uint64_t>(n_trains - 1));
  for (int b = 0; b < n_trains; ++b) {
    const chem_config& c = cfgs[b];
    Train& t = tr[b];
    std::memset(&t, 0, sizeof(Train));
    t.L = c.L_nm;
    t.halfL = 0.5 * c.L_nm;
    t.dt_min = c.dt_min_s;
    t.dt_max = c.dt_max_s;
    t.dt_growth = c.dt_growth;
    t.c = c.cutoff_c;
    t.horizon = c.sbs_horizon_s;
    t.reset_on_release = c.dt_reset_on_release ? 1 : 0;
    // dt cap: every cutoff R + c sqrt(2 D_AB dt) stays <= L/3
    double dt_L = std::numeric_limits<double>::infinity();
    for (int r = 0; r < T.n_rxn; ++r) {
      const double room = c.L_nm / 3.0 - T.R[r];
      if (!(room > 0.0)) {
        delete ctx;
        return CHEM_EINVAL;
      }
      if (c.cutoff_c > 0.0) {
        const double q = room / c.cutoff_c;
        dt_L = std::min(dt_L, q * q / (2.0 * T.D_AB[r]));
      }
    }
    t.dt_L = dt_L;
    // hash resolution: the table is allocated for n_alloc cells per axis; the runtime
    // limit n_max (<= n_alloc) is what the autotuner varies
    int n_alloc = c.cells_per_axis_max, n_max = c.cells_per_axis_max;
    if (n_alloc <= 0) {
      const double cap_sp = static_cast<double>(c.capacity_species);
      n_alloc = static_cast<int>(std::floor(std::cbrt(cap_sp * 128.0)));
      n_alloc = std::max(3, std::min(n_alloc, 512));
      n_max = static_cast<int>(std::floor(std::cbrt(cap_sp * ctx->cell_factor_x100 / 100.0)));
      n_max = std::max(3, std::min(n_max, n_alloc));
    }
    if (n_alloc < 3 || n_alloc > 1024) {
      delete ctx;
      return CHEM_EINVAL;
    }
    t.n_max = n_max;
    t.n_alloc = n_alloc;
    t.cb_alloc = bits_for(static_cast<uint64_t>(n_alloc - 1));
    t.cb = t.cb_ref = t.cb_alloc;
    if (b == 0) {
      ctx->cb_alloc0 = t.cb_alloc;
      ctx->pass_nmax = n_max;
      ctx->pass_cbref = 0;  // no species sorted yet: the first step picks the grid
    }
    t.inv_L = 1.0 / c.L_nm;
    t.cell_base = static_cast<uint32_t>(cells);
    cells += 1ull << (3 * t.cb_alloc);
    t.pend_base = static_cast<uint32_t>(pend);
    t.pend_cap = static_cast<uint32_t>(c.capacity_pending);
    pend += static_cast<uint64_t>(c.capacity_pending);
    t.id_limit = (tbits + 29 <= 32) ? (1u << 29) - 1u : (1u << (32 - tbits)) - 1u;
    init_train_dynamic(t, c, n_alloc);
    t.park_base = static_cast<uint32_t>(cap);
    t.park_cap = static_cast<uint32_t>(c.capacity_species);
    cap += static_cast<uint64_t>(c.capacity_species);
    cand += static_cast<uint64_t>(c.capacity_candidates);
    evlog += static_cast<uint64_t>(c.capacity_event_log);
    steplog += static_cast<uint64_t>(c.capacity_step_log);
  }
  if (cap >= (1ull << 31) || cells >= (1ull << 32) - 2 || pend >= (1ull << 31) || cand >= (1ull << 24)) {
    delete ctx;
    return CHEM_EINVAL;
  }
  if (cand == 0) cand = 1;

  // ---- stream, device properties, launch shapes
  if (c0.cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(c0.cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      chem_status s = fail(ctx, CHEM_ECUDA, "no usable CUDA device");
      *out = ctx;
      return s;
    }
    ctx->own_stream = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
  if (ctx->sms <= 0) {
    *out = ctx;
    return fail(ctx, CHEM_ECUDA, "no usable CUDA device");
  }
  int sort_occ = 0, pers_occ = 0;
  if (sort_pass_occupancy(&sort_occ) != cudaSuccess || sort_occ < 1) {
    *out = ctx;
    return fail(ctx, CHEM_ECUDA, "sort kernel not loadable: %s", cudaGetErrorString(cudaGetLastError()));
  }
  cudaError_t pe = ctx->precision == CHEM_FP64 ? persistent_occupancy_f64(&pers_occ)
                                               : persistent_occupancy_f32l(&pers_occ);
  if (pe != cudaSuccess || pers_occ < 1) {
    *out = ctx;
    return fail(ctx, CHEM_ECUDA, "step kernel not loadable: %s", cudaGetErrorString(pe));
  }
  ctx->lc.stream_blocks = ctx->sms * 4;
  ctx->lc.search_blocks = ctx->sms * 4;  // resident CTAs (launch bounds 256 x 4); items are stolen
  ctx->lc.sort_blocks = ctx->sms * sort_occ;
  ctx->lc.persistent_blocks = ctx->sms * pers_occ;

  // ---- device allocations
  Dev& d = ctx->d;
  d.cap = static_cast<uint32_t>(cap);
  d.cap_cand = static_cast<uint32_t>(cand);
  d.cap_ev_log = static_cast<uint32_t>(evlog);
  d.cap_step_log = static_cast<uint32_t>(steplog);
  d.cap_pend = static_cast<uint32_t>(pend);
  d.n_trains = static_cast<uint32_t>(n_trains);
  d.total_cells = static_cast<uint32_t>(cells);
  d.sentinel = static_cast<uint32_t>(cells);
  d.train_bits = bits_for(static_cast<uint64_t>(n_trains - 1));
  d.passes = (bits_for(cells) + 7) / 8;
  if (d.passes < 1) d.passes = 1;
  if (d.passes > MAX_PASSES) {
    *out = ctx;
    return fail(ctx, CHEM_EINVAL, "too many hash cells");
  }
  ctx->passes_alloc = d.passes;
  d.precision = ctx->precision;
  d.max_tiles = static_cast<uint32_t>(cap / SORT_TILE_MIN + 2);
  bool ok = true;
  auto A = [&](size_t bytes) {
    void* p = dev_alloc(ctx, bytes);
    if (!p) ok = false;
    return p;
  };
  if (ctx->precision == CHEM_FP64) {
    d.sx = static_cast<double*>(A(cap * 8)); d.sy = static_cast<double*>(A(cap * 8));
    d.sz = static_cast<double*>(A(cap * 8)); d.stid = static_cast<uint32_t*>(A(cap * 4));
    d.tx = static_cast<double*>(A(cap * 8)); d.ty = static_cast<double*>(A(cap * 8));
    d.tz = static_cast<double*>(A(cap * 8)); d.ttid = static_cast<uint32_t*>(A(cap * 4));
    d.tdx = static_cast<double*>(A(cap * 8)); d.tdy = static_cast<double*>(A(cap * 8));
    d.tdz = static_cast<double*>(A(cap * 8));
    // FP32 cell offsets of the same species for the pair search's prefilter
    d.s4 = static_cast<float4*>(A(cap * 16));
    d.t4 = static_cast<float4*>(A(cap * 16));
  } else {
    d.s4 = static_cast<float4*>(A(cap * 16));
    d.t4 = static_cast<float4*>(A(cap * 16));
    d.td4 = static_cast<float4*>(A(cap * 16));
    d.sd4 = static_cast<float4*>(A(cap * 16));
  }
  if (n_trains > 1) {  // parking buffers of idle trains
    d.pk_cell = static_cast<uint32_t*>(A(cap * 4));
    if (ctx->precision == CHEM_FP64) {
      d.pkx = static_cast<double*>(A(cap * 8)); d.pky = static_cast<double*>(A(cap * 8));
      d.pkz = static_cast<double*>(A(cap * 8)); d.pk_tid = static_cast<uint32_t*>(A(cap * 4));
    } else {
      d.pk4 = static_cast<float4*>(A(cap * 16));
    }
  }
  d.cap_items = static_cast<uint32_t>(cap + cap / ITEM_HOME + 64);
  d.items = static_cast<uint2*>(A(static_cast<size_t>(d.cap_items) * 8));
  d.cell_sorted = static_cast<uint32_t*>(A(cap * 4));
  {
    uint32_t* sortbuf = static_cast<uint32_t*>(A(cap * 16));  // keys0|keys1|vals0|vals1
    d.keys0 = sortbuf;
    d.keys1 = sortbuf + cap;
    d.vals0 = sortbuf + 2 * cap;
    d.vals1 = sortbuf + 3 * cap;
  }
  d.dead = static_cast<uint8_t*>(A(cap));
  d.touch = static_cast<uint32_t*>(A(cap * 4));
  d.cell_info = static_cast<int4*>(A((cells + 1) * 16));
  d.occ_vec4 = static_cast<uint32_t>((cells + 127) / 128);
  d.occ = static_cast<uint32_t*>(A(static_cast<size_t>(d.occ_vec4) * 16));
  d.lookback = static_cast<unsigned long long*>(A(static_cast<size_t>(d.max_tiles) * RADIX * 8));
  d.cand = static_cast<Cand*>(A(cand * sizeof(Cand)));
  const uint64_t evn = std::max<uint64_t>(cand, RADIX);
  d.ev_list = static_cast<uint32_t*>(A(evn * 4));
  d.alive0 = static_cast<uint32_t*>(A(evn * 4));
  d.alive1 = static_cast<uint32_t*>(A(evn * 4));
  d.ev_k0 = static_cast<uint32_t*>(A(evn * 4));
  d.ev_k1 = static_cast<uint32_t*>(A(evn * 4));
  d.ev_v0 = static_cast<uint32_t*>(A(evn * 4));
  d.ev_v1 = static_cast<uint32_t*>(A(evn * 4));
  d.ev_log = static_cast<chem_event*>(A(std::max<uint64_t>(evlog, 1) * sizeof(chem_event)));
  d.step_log = static_cast<chem_step_record*>(A(std::max<uint64_t>(steplog, 1) * sizeof(chem_step_record)));
  const uint64_t pn = std::max<uint64_t>(pend, 1);
  d.p_type = static_cast<int32_t*>(A(pn * 4));
  d.px = static_cast<double*>(A(pn * 8)); d.py = static_cast<double*>(A(pn * 8));
  d.pz = static_cast<double*>(A(pn * 8)); d.pt = static_cast<double*>(A(pn * 8));
  d.trains = static_cast<Train*>(A(sizeof(Train) * n_trains));
  Tables* tables_dev = static_cast<Tables*>(A(sizeof(Tables)));
  d.tables = tables_dev;
  d.g = static_cast<Global*>(A(sizeof(Global)));
  *out = ctx;
  if (!ok) return fail(ctx, CHEM_ENOMEM, "device allocation failed");
  if (cudaMallocHost(&ctx->g_pinned, sizeof(Global)) != cudaSuccess ||
      cudaMallocHost(&ctx->t_end_pinned, sizeof(double) * n_trains) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, CHEM_ENOMEM, "pinned host allocation failed");
  }
  ctx->t_end_dev = static_cast<double*>(A(sizeof(double) * n_trains));
  if (!ok) return fail(ctx, CHEM_ENOMEM, "device allocation failed");
  CK(cudaMemsetAsync(d.dead, 0, cap, ctx->stream));
  CK(cudaMemsetAsync(d.touch, 0, cap * 4, ctx->stream));
  CK(cudaMemsetAsync(d.cell_info, 0xFF, (cells + 1) * 16, ctx->stream));
  CK(cudaMemsetAsync(d.occ, 0, static_cast<size_t>(d.occ_vec4) * 16, ctx->stream));
  CK(cudaMemsetAsync(d.lookback, 0, static_cast<size_t>(d.max_tiles) * RADIX * 8, ctx->stream));
  CK(cudaMemcpyAsync(tables_dev, &T, sizeof(Tables), cudaMemcpyHostToDevice, ctx->stream));
  chem_status gs = init_global(ctx);
  if (gs) return gs;
  return upload_trains(ctx, tr);
}

chem_status chem_init(const chem_config* cfg, chem_ctx** out) { return chem_batch_init(cfg, 1, out); }

chem_status chem_batch_inject(chem_ctx* ctx, int32_t train, int64_t n, const int32_t* type,
                              const double* xyz, const double* t_arrival, double energy_eV) {
  return inject_one(ctx, train, n, type, xyz, t_arrival, energy_eV);
}

chem_status chem_inject_pulse(chem_ctx* ctx, int64_t n, const int32_t* type, const double* xyz,
                              const double* t_arrival, double energy_eV) {
  return inject_one(ctx, 0, n, type, xyz, t_arrival, energy_eV);
}

chem_status chem_batch_run_until(chem_ctx* ctx, const double* t_end_s) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  if (!t_end_s) return CHEM_EINVAL;
  for (int b = 0; b < ctx->B; ++b) {
    if (!std::isfinite(t_end_s[b])) return CHEM_EINVAL;
    ctx->t_end_pinned[b] = t_end_s[b];
  }
  CK(cudaMemcpyAsync(ctx->t_end_dev, ctx->t_end_pinned, sizeof(double) * ctx->B, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(enqueue_set_t_end(ctx->d, ctx->t_end_dev, ctx->stream));
  ctx->stats.bytes_h2d += static_cast<int64_t>(sizeof(double) * ctx->B);
  ctx->stats.kernel_launches += 1;
  return run_loop(ctx);
}

chem_status chem_run_until(chem_ctx* ctx, double t_end_s) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  std::vector<double> t(ctx->B, t_end_s);
  return chem_batch_run_until(ctx, t.data());
}

chem_status chem_check_bounded_wait(chem_ctx* ctx, double limit_s) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  if (!(limit_s > 0.0) || !(limit_s <= 10.0)) return CHEM_EINVAL;
  CK(enqueue_bounded_wait(ctx->d, limit_s, ctx->stream));
  ctx->stats.kernel_launches += 1;
  s = download_global(ctx);
  if (s) return s;
  const int st = ctx->g_pinned->status;
  if (st != 0)
    return fail(ctx, static_cast<chem_status>(st), "a bounded device wait ran out after %.3g s (status %d)",
                limit_s, st);
  return CHEM_OK;
}

chem_status chem_check_acceptance(chem_ctx* ctx, int32_t precision, uint32_t step, double dt_s, int64_t n,
                                  const double* d0sq, const double* d1sq, const int32_t* rxn,
                                  const uint32_t* id_lo, const uint32_t* id_hi, uint8_t* accept) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  if (precision != CHEM_FP64 && precision != CHEM_FP32_LOCAL) return CHEM_EINVAL;
  if (!(dt_s > 0.0) || !std::isfinite(dt_s) || n < 0 || n > (1ll << 24)) return CHEM_EINVAL;
  if (n == 0) return CHEM_OK;
  if (!d0sq || !d1sq || !rxn || !id_lo || !id_hi || !accept) return CHEM_EINVAL;
  for (int64_t i = 0; i < n; ++i) {
    if (rxn[i] < 0 || rxn[i] >= ctx->tables.n_rxn) return CHEM_EINVAL;
    if (!(d0sq[i] >= 0.0) || !(d1sq[i] >= 0.0) || !std::isfinite(d0sq[i]) || !std::isfinite(d1sq[i]))
      return CHEM_EINVAL;
  }
  const size_t un = static_cast<size_t>(n);
  const size_t bytes = un * (8 + 8 + 4 + 4 + 4 + 1);
  void* buf = nullptr;  // one temporary block, released before returning
  if (ctx->alloc) buf = ctx->alloc((bytes + 255) & ~static_cast<size_t>(255), ctx->alloc_user);
  else if (cudaMalloc(&buf, bytes) != cudaSuccess) { cudaGetLastError(); buf = nullptr; }
  if (!buf) return CHEM_ENOMEM;
  char* b = static_cast<char*>(buf);
  double* dd0 = reinterpret_cast<double*>(b);
  double* dd1 = dd0 + un;
  int32_t* dr = reinterpret_cast<int32_t*>(dd1 + un);
  uint32_t* dlo = reinterpret_cast<uint32_t*>(dr + un);
  uint32_t* dhi = dlo + un;
  uint8_t* dout = reinterpret_cast<uint8_t*>(dhi + un);
  cudaError_t e = cudaMemcpyAsync(dd0, d0sq, un * 8, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dd1, d1sq, un * 8, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dr, rxn, un * 4, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dlo, id_lo, un * 4, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dhi, id_hi, un * 4, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = precision == CHEM_FP64
            ? enqueue_check_accept_f64(ctx->d, static_cast<uint32_t>(n), step, dt_s, dd0, dd1, dr, dlo, dhi, dout,
                                       ctx->stream)
            : enqueue_check_accept_f32l(ctx->d, static_cast<uint32_t>(n), step, dt_s, dd0, dd1, dr, dlo, dhi,
                                        dout, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(accept, dout, un, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (ctx->dfree) ctx->dfree(buf, (bytes + 255) & ~static_cast<size_t>(255), ctx->alloc_user);
  else cudaFree(buf);
  if (e != cudaSuccess) return fail(ctx, CHEM_ECUDA, "acceptance check: %s", cudaGetErrorString(e));
  ctx->stats.kernel_launches += 1;
  return CHEM_OK;
}

chem_status chem_batch_run_homogeneous(chem_ctx* ctx, const double* t_end_s) {
  return homogeneous_run(ctx, t_end_s);
}

chem_status chem_run_homogeneous(chem_ctx* ctx, double t_end_s) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  std::vector<double> t(ctx->B, t_end_s);
  return homogeneous_run(ctx, t.data());
}

chem_status chem_batch_homogeneous_report(chem_ctx* ctx, int32_t train, double* extents, int64_t* events,
                                          int64_t* integrator_steps) {
  return homogeneous_report(ctx, train, extents, events, integrator_steps);
}

chem_status chem_batch_tally(chem_ctx* ctx, int32_t train, int64_t* counts, double* G, int64_t* events,
                             double* t_now, int64_t* species_steps) {
  return tally_one(ctx, train, counts, G, events, t_now, species_steps);
}

chem_status chem_tally(chem_ctx* ctx, int64_t* counts, double* G, int64_t* events, double* t_now,
                       int64_t* species_steps) {
  return tally_one(ctx, 0, counts, G, events, t_now, species_steps);
}

chem_status chem_batch_get_state(chem_ctx* ctx, int32_t train, int64_t cap, int32_t* type, uint32_t* id,
                                 double* xyz, int64_t* n) {
  return state_one(ctx, train, cap, type, id, xyz, n);
}

chem_status chem_get_state(chem_ctx* ctx, int64_t cap, int32_t* type, uint32_t* id, double* xyz,
                           int64_t* n) {
  return state_one(ctx, 0, cap, type, id, xyz, n);
}

chem_status chem_get_events(chem_ctx* ctx, int64_t cap, chem_event* ev, int64_t* n) {
  if (!ctx || cap < 0) return CHEM_EINVAL;
  chem_status s = download_global(ctx);
  if (s) return s;
  const uint64_t have = std::min<uint64_t>(ctx->g_pinned->ev_log_n, ctx->d.cap_ev_log);
  const uint64_t k = std::min<uint64_t>(have, static_cast<uint64_t>(cap));
  if (k && ev) CK(cudaMemcpy(ev, ctx->d.ev_log, k * sizeof(chem_event), cudaMemcpyDeviceToHost));
  if (n) *n = static_cast<int64_t>(have);
  return ctx->status;
}

chem_status chem_get_step_log(chem_ctx* ctx, int64_t cap, chem_step_record* rec, int64_t* n) {
  if (!ctx || cap < 0) return CHEM_EINVAL;
  chem_status s = download_global(ctx);
  if (s) return s;
  const uint64_t have = std::min<uint64_t>(ctx->g_pinned->step_log_n, ctx->d.cap_step_log);
  const uint64_t k = std::min<uint64_t>(have, static_cast<uint64_t>(cap));
  if (k && rec) CK(cudaMemcpy(rec, ctx->d.step_log, k * sizeof(chem_step_record), cudaMemcpyDeviceToHost));
  if (n) *n = static_cast<int64_t>(have);
  return ctx->status;
}

chem_status chem_batch_reset(chem_ctx* ctx, const uint64_t* seeds) {
  if (!ctx) return CHEM_EINVAL;
  if (ctx->status == CHEM_ECUDA) return ctx->status;
  std::vector<Train> tr;
  chem_status s = download_trains(ctx, tr);
  if (s) return s;
  for (int b = 0; b < ctx->B; ++b) {
    TrainHost& h = ctx->th[b];
    if (seeds) h.cfg.seed = seeds[b];
    h.E_dep = 0.0;
    h.pend.clear();
    init_train_dynamic(tr[b], h.cfg, tr[b].n_alloc);
  }
  s = init_global(ctx);
  if (s) return s;
  CK(cudaMemsetAsync(ctx->d.dead, 0, ctx->d.cap, ctx->stream));
  CK(cudaMemsetAsync(ctx->d.touch, 0, static_cast<size_t>(ctx->d.cap) * 4, ctx->stream));
  CK(cudaMemsetAsync(ctx->d.cell_info, 0xFF, (static_cast<size_t>(ctx->d.total_cells) + 1) * 16, ctx->stream));
  CK(cudaMemsetAsync(ctx->d.occ, 0, static_cast<size_t>(ctx->d.occ_vec4) * 16, ctx->stream));
  CK(cudaMemsetAsync(ctx->d.lookback, 0, static_cast<size_t>(ctx->d.max_tiles) * RADIX * 8, ctx->stream));
  s = upload_trains(ctx, tr);
  if (s) return s;
  ctx->status = CHEM_OK;
  ctx->err.clear();
  return CHEM_OK;
}

chem_status chem_reset(chem_ctx* ctx, uint64_t seed) {
  if (!ctx) return CHEM_EINVAL;
  std::vector<uint64_t> seeds(ctx->B);
  for (int b = 0; b < ctx->B; ++b) seeds[b] = seed + static_cast<uint64_t>(b);
  return chem_batch_reset(ctx, seeds.data());
}

int32_t chem_batch_size(const chem_ctx* ctx) { return ctx ? ctx->B : 0; }

chem_status chem_get_stats(const chem_ctx* ctx, chem_stats* out) {
  if (!ctx || !out) return CHEM_EINVAL;
  *out = ctx->stats;
  return ctx->status;
}

chem_status chem_set_profiling(chem_ctx* ctx, int32_t on) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  ctx->profiling = on != 0;
  for (int i = 0; i < 8; ++i) {
    ctx->stats.phase_ms[i] = 0.0;
    ctx->stats.phase_launches[i] = 0;
  }
  return capture_graph(ctx);
}

chem_status chem_autotune(chem_ctx* ctx, double budget_ms, int32_t* chosen) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  if (!(budget_ms > 0.0)) return CHEM_EINVAL;
  // ---- snapshot of everything a step changes (pending data and tables do not change)
  s = download_global(ctx);
  if (s) return s;
  const uint32_t n = ctx->g_pinned->n_total;
  Dev& d = ctx->d;
  const bool f64 = ctx->precision == CHEM_FP64;
  const size_t state_b = f64 ? 28 : 16;
  const size_t snap_bytes = static_cast<size_t>(n) * (state_b + 4 + 1) + sizeof(Train) * ctx->B + sizeof(Global) + 256;
  unsigned char* snap = static_cast<unsigned char*>(dev_alloc(ctx, snap_bytes));
  if (!snap) return fail(ctx, CHEM_ENOMEM, "autotune snapshot allocation failed");
  auto copies = [&](bool save) -> cudaError_t {
    size_t o = 0;
    auto cp = [&](void* dev, size_t bytes) {
      cudaError_t e = save ? cudaMemcpyAsync(snap + o, dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream)
                           : cudaMemcpyAsync(dev, snap + o, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
      o += bytes;
      return e;
    };
    cudaError_t e = cudaSuccess;
    if (n) {
      if (f64) {
        e = cp(d.sx, n * 8ull); if (e) return e;
        e = cp(d.sy, n * 8ull); if (e) return e;
        e = cp(d.sz, n * 8ull); if (e) return e;
        e = cp(d.stid, n * 4ull); if (e) return e;
      } else {
        e = cp(d.s4, n * 16ull); if (e) return e;
      }
      e = cp(d.cell_sorted, n * 4ull); if (e) return e;
      e = cp(d.dead, n); if (e) return e;
    }
    return cp(d.trains, sizeof(Train) * ctx->B);
  };
  const size_t global_off = static_cast<size_t>(n) * (state_b + 4 + 1) + sizeof(Train) * ctx->B;
  CK(copies(true));
  CK(cudaMemcpyAsync(snap + global_off, d.g, sizeof(Global), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<Train> tr0;
  s = download_trains(ctx, tr0);
  if (s) return s;
  // ---- candidates: runtime hash limit, steps per replay, launch form. The search
  // mapping is not a candidate: trials time the next few steps only, while the mapping's
  // payoff changes along a trajectory; it stays the context's (by default chosen per
  // step from the pairs inside the cutoffs, see phase_begin).
  const int n_alloc = tr0[0].n_alloc;
  std::vector<int> n_cands;
  // (half the allocated resolution minus one keeps one bit per axis less: one radix pass less)
  for (int nm : {n_alloc, (3 * n_alloc) / 4, n_alloc / 2 - 1, (2 * n_alloc) / 5}) n_cands.push_back(std::max(3, nm));
  const int ih_cands[1] = {ctx->item_home};
  const int spl_cands[2] = {8, 32};
  const bool mode_cands[2] = {false, true};  // per-phase graph, persistent launch
  const bool saved_persistent = ctx->persistent;
  bool best_persistent = saved_persistent;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const auto t_start = std::chrono::steady_clock::now();
  double best_rate = -1.0;
  int best_n = tr0[0].n_max, best_ih = ctx->item_home, best_spl = ctx->steps_per_launch;
  const int saved_spl = ctx->steps_per_launch;
  const bool saved_prof = ctx->profiling;
  ctx->profiling = false;
  // each trial's graph sorts the key bits its grid limit needs
  ctx->pass_cbref = tr0[0].n_ref != 0 ? tr0[0].cb_ref : 0;
  for (int combo = 0; combo < 4; ++combo) {
    const bool pers = mode_cands[combo / 2];
    const int spl = spl_cands[combo % 2];
    const int ih = ih_cands[0];
    ctx->persistent = pers;
    ctx->steps_per_launch = spl;
    ctx->item_home = ih;  // selects the search kernel of the captured graph
    {
      for (int nm : n_cands) {
        const double spent = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        if (spent > budget_ms && best_rate > 0.0) break;
        // restore the state, then set this trial's parameters and an open end time
        CK(copies(false));
        const uint32_t epoch_now = ctx->g_pinned->epoch;
        CK(cudaMemcpyAsync(d.g, snap + global_off, sizeof(Global), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        std::vector<Train> tr = tr0;
        for (auto& t : tr) { t.n_max = std::min(nm, t.n_alloc); t.t_end = std::numeric_limits<double>::infinity(); }
        s = upload_trains(ctx, tr);
        if (s) break;
        ctx->pass_nmax = tr[0].n_max;
        s = capture_graph(ctx);
        if (s) break;
        Global& gfix = *ctx->g_pinned;
        CK(cudaMemcpyAsync(&gfix, d.g, sizeof(Global), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        gfix.epoch = std::max(gfix.epoch, epoch_now) + 1;  // stale hash stamps never match
        set_mapping(gfix, ih);
        CK(cudaMemcpyAsync(d.g, &gfix, sizeof(Global), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        const int reps = std::max(1, 24 / spl);
        CK(cudaGraphLaunch(ctx->graph, ctx->stream));  // settle
        CK(cudaEventRecord(e0, ctx->stream));
        for (int r = 0; r < reps; ++r) CK(cudaGraphLaunch(ctx->graph, ctx->stream));
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaMemcpyAsync(ctx->g_pinned, d.g, sizeof(Global), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        std::vector<Train> after;
        s = download_trains(ctx, after);
        if (s) break;
        if (ctx->g_pinned->status != 0) {
          // a trial ran out of a capacity (e.g. candidates on a coarse grid): skip it
          CK(cudaMemsetAsync(&d.g->status, 0, sizeof(int), ctx->stream));
          continue;
        }
        long long ss = 0;
        for (int b = 0; b < ctx->B; ++b) ss += after[b].species_steps;
        // steps of the settle replay are included in ss; subtract them with the rate of
        // the timed part by counting the timed replays' share
        const double timed_frac = static_cast<double>(reps) / (reps + 1);
        const double rate = ms > 0.f ? (static_cast<double>(ss - [&] { long long z = 0; for (int b = 0; b < ctx->B; ++b) z += tr0[b].species_steps; return z; }()) * timed_frac) / (ms * 1e-3) : 0.0;
        if (rate > best_rate) { best_rate = rate; best_n = nm; best_ih = ih; best_spl = spl; best_persistent = pers; }
      }
    }
    if (s) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // ---- restore the state and apply the best parameters (the trials' occupancy bits
  // are cleared; stale ones would only cost lookups)
  CK(copies(false));
  CK(cudaMemsetAsync(d.occ, 0, static_cast<size_t>(d.occ_vec4) * 16, ctx->stream));
  {
    const uint32_t epoch_now = ctx->g_pinned->epoch;
    Global& gfix = *ctx->g_pinned;
    CK(cudaMemcpyAsync(&gfix, snap + global_off, sizeof(Global), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    gfix.epoch = std::max(gfix.epoch, epoch_now) + 1;
    set_mapping(gfix, best_ih);
    CK(cudaMemcpyAsync(d.g, &gfix, sizeof(Global), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  for (auto& t : tr0) t.n_max = std::min(best_n, t.n_alloc);
  chem_status s2 = upload_trains(ctx, tr0);
  ctx->pass_nmax = tr0[0].n_max;
  // release the snapshot
  for (size_t i = 0; i < ctx->allocs.size(); ++i) {
    if (ctx->allocs[i].first == snap) {
      if (ctx->dfree) ctx->dfree(snap, ctx->allocs[i].second, ctx->alloc_user);
      else cudaFree(snap);
      ctx->allocs.erase(ctx->allocs.begin() + static_cast<long>(i));
      break;
    }
  }
  if (s) return s;
  if (s2) return s2;
  ctx->item_home = best_ih;
  ctx->steps_per_launch = best_rate > 0.0 ? best_spl : saved_spl;
  ctx->persistent = best_rate > 0.0 ? best_persistent : saved_persistent;
  ctx->profiling = saved_prof;
  s = capture_graph(ctx);
  if (s) return s;
  if (chosen) {
    chosen[0] = ctx->steps_per_launch;
    chosen[1] = best_n;
    chosen[2] = best_ih;
    chosen[3] = ctx->persistent ? CHEM_LAUNCH_PERSISTENT : CHEM_LAUNCH_PHASES;
  }
  return ctx->status;
}

chem_status chem_set_tuning(chem_ctx* ctx, const int32_t* tuning) {
  chem_status s = check_ctx(ctx);
  if (s) return s;
  if (!tuning) return CHEM_EINVAL;
  const int spl = tuning[0], n_lim = tuning[1], ih = tuning[2], mode = tuning[3];
  if (spl < 1 || spl > 1024 || n_lim < 3 || ih < -1 || ih > ITEM_HOME ||
      (mode != CHEM_LAUNCH_PHASES && mode != CHEM_LAUNCH_PERSISTENT))
    return CHEM_EINVAL;
  std::vector<Train> tr;
  s = download_trains(ctx, tr);
  if (s) return s;
  for (auto& t : tr) t.n_max = std::min(n_lim, t.n_alloc);
  s = upload_trains(ctx, tr);
  if (s) return s;
  ctx->pass_nmax = tr[0].n_max;
  ctx->pass_cbref = tr[0].n_ref != 0 ? tr[0].cb_ref : 0;
  s = upload_mapping(ctx, ih);
  if (s) return s;
  ctx->item_home = ih;
  ctx->steps_per_launch = spl;
  ctx->persistent = mode == CHEM_LAUNCH_PERSISTENT;
  s = capture_graph(ctx);
  if (s) return s;
  return ctx->status;
}

}  // extern "C"
