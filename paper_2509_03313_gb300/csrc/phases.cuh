// The phases of one SBS step, as device functions usable both from one-kernel-per-phase
// launches and from the persistent batched launch. Every phase is grid-stride over its
// work and reads the device status word first: once a phase has raised an error the
// remaining phases of the step do nothing.
//
// Arithmetic that the FP64 mode shares with the FP64 reference is written with explicit
// round-to-nearest intrinsics (__dmul_rn, __dadd_rn, ...) so that no multiply-add is ever
// contracted, whatever the compilation flags: in FP64 mode the library reproduces the
// reference's positions to rounding and its decisions exactly.
#pragma once
#include <cfloat>
#include <type_traits>
#include <math_constants.h>

#include "onesweep.cuh"
#include "sbs_device.cuh"

namespace chem {

constexpr double TWO_PI = 6.283185307179586;  // 2 * pi rounded to double
constexpr double TWO_POW_M53 = 1.1102230246251565e-16;
constexpr float TWO_POW_M24F = 5.9604644775390625e-08f;

__device__ __forceinline__ int status_of(const Dev& d) {
  return *reinterpret_cast<volatile int*>(&d.g->status);
}

// Eq. 1 applied as often as needed: x shifted by whole box lengths into [-L/2, L/2).
__device__ __forceinline__ double wrap_box(double x, double L, double halfL) {
  const double k = floor(__ddiv_rn(__dadd_rn(x, halfL), L));
  x = __dsub_rn(x, __dmul_rn(k, L));
  if (x >= halfL) x = __dsub_rn(x, L);
  if (x < -halfL) x = __dadd_rn(x, L);
  return x;
}

// The same shift computed with 1/L instead of a division (FP32-local regrid only; the
// FP64 mode keeps wrap_box, whose rounding is the reference's).
__device__ __forceinline__ double wrap_box_fast(double x, double L, double halfL, double inv_L) {
  const double k = floor((x + halfL) * inv_L);
  x -= k * L;
  if (x >= halfL) x -= L;
  if (x < -halfL) x += L;
  return x;
}

// A coordinate measured from the box corner folded into [0, L) (FP32-local regrid).
__device__ __forceinline__ double rebase_corner(double a, double L, double inv_L) {
  if (a >= L || a < 0.0) a -= L * floor(a * inv_L);
  if (a >= L) a -= L;
  if (a < 0.0) a += L;
  return a;
}

// Eq. 2 (minimum image) for the separation of two in-box points.
__device__ __forceinline__ double min_image(double dx, double L, double halfL) {
  if (dx >= halfL) return __dsub_rn(dx, L);
  if (dx < -halfL) return __dadd_rn(dx, L);
  return dx;
}

__device__ __forceinline__ double sq3(double x, double y, double z) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}

// Three standard normals for species `id` at step `step` (FP64 mode): two Philox blocks,
// 53-bit uniforms u1 in (0,1], u2 in [0,1), Box-Muller.
__device__ __forceinline__ void gauss3_f64(uint32_t id, uint32_t step, uint32_t k0, uint32_t k1,
                                           double& g0, double& g1, double& g2) {
  const uint4 a = philox4x32_10(make_uint4(id, step, 0u, 0u), k0, k1);
  const uint4 b = philox4x32_10(make_uint4(id, step, 0u, 1u), k0, k1);
  const double u1 = __dmul_rn(__dadd_rn(static_cast<double>(u53(a.x, a.y)), 1.0), TWO_POW_M53);
  const double u2 = __dmul_rn(static_cast<double>(u53(a.z, a.w)), TWO_POW_M53);
  const double u3 = __dmul_rn(__dadd_rn(static_cast<double>(u53(b.x, b.y)), 1.0), TWO_POW_M53);
  const double u4 = __dmul_rn(static_cast<double>(u53(b.z, b.w)), TWO_POW_M53);
  const double r = sqrt(__dmul_rn(-2.0, log(u1)));
  const double th = __dmul_rn(TWO_PI, u2);
  double s, c;
  sincos(th, &s, &c);
  g0 = __dmul_rn(r, c);
  g1 = __dmul_rn(r, s);
  const double r2 = sqrt(__dmul_rn(-2.0, log(u3)));
  g2 = __dmul_rn(r2, cos(__dmul_rn(TWO_PI, u4)));
}

// Three standard normals (FP32-local mode): one Philox block, 24-bit uniforms.
__device__ __forceinline__ void gauss3_f32(uint32_t id, uint32_t step, uint32_t k0, uint32_t k1,
                                           float& g0, float& g1, float& g2) {
  const uint4 a = philox4x32_10(make_uint4(id, step, 0u, 0u), k0, k1);
  const float u1 = static_cast<float>((a.x >> 8) + 1u) * TWO_POW_M24F;
  const float u2 = static_cast<float>(a.y >> 8) * TWO_POW_M24F;
  const float u3 = static_cast<float>((a.z >> 8) + 1u) * TWO_POW_M24F;
  const float u4 = static_cast<float>(a.w >> 8) * TWO_POW_M24F;
  // hardware approximations (a few ulp): the FP32-local normals need no more
  const float r = sqrtf(-2.0f * __logf(u1));
  float s, c;
  __sincosf(6.2831853f * u2, &s, &c);
  g0 = r * c;
  g1 = r * s;
  g2 = sqrtf(-2.0f * __logf(u3)) * __cosf(6.2831853f * u4);
}

// Uniform in [0, 1) for the pair (id_lo, id_hi) at `step` (counter tag 2).
__device__ __forceinline__ double pair_uniform(uint32_t id_lo, uint32_t id_hi, uint32_t step,
                                               uint32_t k0, uint32_t k1) {
  const uint4 c = philox4x32_10(make_uint4(id_lo, step, id_hi, 2u), k0, k1);
  return __dmul_rn(static_cast<double>(u53(c.x, c.y)), TWO_POW_M53);
}

// Probability that the pair's relative Brownian path touched the reaction sphere during
// the step, given its start and end separations d0, d1 (p = 1 when either is inside R):
// 1 - G_abs / G_free for the angle-averaged relative motion (image solutions of r times
// the density, outside a fully absorbing sphere and free), i.e.
// (exp(-a) - exp(-b)) / (1 - exp(-b)) with a = (d0 - R)(d1 - R) / (D_AB dt) and
// b = d0 d1 / (D_AB dt), evaluated as exp(-a) expm1(-c) / expm1(-b), c = b - a =
// R (d0 + d1 - R) / (D_AB dt). Its expectation is the absorbing-sphere rate behind
// Eq. kdiff1 at any dt; for R >> sqrt(D_AB dt) it is the planar bridge exp(-a).
__device__ __forceinline__ double bridge_p(double d0, double d1, double R, double DABdt) {
  if (d1 <= R || d0 <= R) return 1.0;
  const double a = __ddiv_rn(__dmul_rn(__dsub_rn(d0, R), __dsub_rn(d1, R)), DABdt);
  const double b = __ddiv_rn(__dmul_rn(d0, d1), DABdt);
  const double c = __ddiv_rn(__dmul_rn(R, __dsub_rn(__dadd_rn(d0, d1), R)), DABdt);
  return __dmul_rn(exp(-a), __ddiv_rn(expm1(-c), expm1(-b)));
}

__device__ __forceinline__ int cell_index(double x, double halfL, double inv_h, int n) {
  int i = static_cast<int>(floor(__dmul_rn(__dadd_rn(x, halfL), inv_h)));
  return min(max(i, 0), n - 1);
}

// Bits per axis of the cell index of a grid of n cells per axis: enough for the values
// 0..n, so the all-ones index (>= n) is never a cell.
__device__ __forceinline__ int axis_bits(int n) { return 32 - __clz(n); }

__device__ __forceinline__ int wrap_cell(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Per-reaction constants of the acceptance test for a step of length dt: D_AB dt (the
// exponents' denominator) in FP64 and its reciprocal in FP32 (the first tier).
__device__ __forceinline__ void set_pair_constants(Train& tr, const Tables& tb, int r, double dt) {
  tr.ddt[r] = __dmul_rn(tb.D_AB[r], dt);
  tr.inv_ddt_f[r] = 1.0f / static_cast<float>(tr.ddt[r]);
}

// ======================================================================== begin
struct BeginSmem {
  Tables tb;                              // the reaction tables, read once per step
  uint32_t rel[MAX_TRAINS];
  double dt[MAX_TRAINS];
  unsigned long long rcmax_bits[MAX_TRAINS];
  float hf[MAX_TRAINS];                   // this step's cell side
  int cb0;                                // train 0: key bits per axis of its cells
  uint32_t base0;                         // train 0: first global cell
  uint32_t any;
};

// One CTA. (1) per train: release count, clock step and free-jump decision; (2) per
// (train, reaction) cutoff and bridge constants and per (train, type) step sigma, spread
// over the threads because FP64 square roots and divisions are long on this part;
// (3) per train: hash grid of the step; (4) per (train, type pair) cutoff tables; (5) slot
// offsets of the releases and the step counters. The step is one short chain of
// dependent loads: the tables, the status and the global counters are read together at
// the start, and later stages read what earlier ones wrote from shared memory.
static __device__ void phase_begin(const Dev& d, BeginSmem& sb) {
  const int tid = threadIdx.x, nt = blockDim.x;
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(d.tables);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sb.tb);
    for (int i = tid; i < static_cast<int>(sizeof(Tables) / 4); i += nt) dst[i] = src[i];
  }
  for (int i = tid; i < MAX_PASSES * RADIX; i += nt) (&d.g->hist[0][0])[i] = 0u;
  const int st = status_of(d);
  // the counters thread 0 updates below, read with the tables
  Global* g = d.g;
  uint32_t g_total = 0, g_live = 0, g_adaptive = 0, g_home = 0, g_epoch = 0, g_cells = 0;
  unsigned long long g_incut = 0, g_mark = 0;
  if (tid == 0) {
    g_total = g->n_total; g_live = g->n_live; g_adaptive = g->search_adaptive; g_home = g->item_home;
    g_epoch = g->epoch; g_cells = g->cells_steps; g_incut = g->pairs_in_cutoff; g_mark = g->incut_mark;
    sb.any = 0;
  }
  __syncthreads();
  const Tables& tb = sb.tb;
  for (uint32_t b = tid; b < d.n_trains; b += nt) {
    Train& tr = d.trains[b];
    // independent loads first: the per-train work below is one short dependency chain
    const double t = tr.t, t_end = tr.t_end, t_lr = tr.t_last_release, horizon = tr.horizon;
    const double dt_min = tr.dt_min, dt_L = tr.dt_L;
    double dt_cur = tr.dt_cur;
    const uint32_t p_head = tr.p_head, p_tail = tr.p_tail, pend_base = tr.pend_base;
    const uint32_t next_id = tr.next_id, id_limit = tr.id_limit;
    const uint32_t mat = tr.mat_n;  // survivors of a homogeneous stage (already counted)
    const uint32_t parked = tr.park_n;  // species parked while the train was idle (counted)
    const int reset = tr.reset_on_release;
    long long live = 0;
    for (int ty = 0; ty < MAXT; ++ty) live += (ty < tb.n_types) ? tr.counts[ty] : 0;
    const bool act = (st == 0) && (t < t_end);
    // an idle train with species among the stepped slots parks them this step
    tr.park_now = (!act && d.pk_cell != nullptr && live > static_cast<long long>(parked) + mat) ? 1u : 0u;
    uint32_t rel = 0;
    int free_jump = 0;
    double dt = 0.0;
    sb.rcmax_bits[b] = 0ull;
    if (act) {
      // pending arrivals are sorted; release those with arrival <= t
      uint32_t lo = p_head, hi = p_tail;
      const double* pt = d.pt + pend_base;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pt[mid] <= t) lo = mid + 1; else hi = mid;
      }
      rel = lo - p_head;
      double t_last = t_lr;
      if (rel + mat > 0) {
        t_last = t;
        tr.t_last_release = t;
        if (reset) dt_cur = dt_min;
      }
      const double next_arr = (lo < p_tail) ? pt[lo] : CUDART_INF;
      double t_next;
      if (horizon > 0.0 && __dsub_rn(t, t_last) >= horizon && next_arr > t) {
        free_jump = 1;
        t_next = fmin(t_end, next_arr);
        dt = __dsub_rn(t_next, t);
      } else {
        dt = fmin(dt_cur, dt_L);
        if (__dsub_rn(t_end, t) <= __dmul_rn(dt, END_SLACK)) {
          dt = __dsub_rn(t_end, t);
          t_next = t_end;
        } else {
          t_next = __dadd_rn(t, dt);
        }
      }
      tr.dt_cur = dt_cur;
      tr.dt = dt;
      tr.t_next = t_next;
      tr.t_start = t;
      // releases: the unparked species first (they keep their ids), then the re-created
      // survivors, then the arrived species
      tr.rel_n = parked + rel + mat;
      tr.rel_park = parked;
      tr.park_n = 0;
      tr.rel_mat = mat;
      tr.mat_n = 0;
      tr.rel_id0 = next_id;
      tr.rel_p0 = p_head;
      tr.p_head = p_head + rel;
      tr.next_id = next_id + rel + mat;
      tr.n_live_step = live + rel;
      tr.n_events_step = 0;
      if (static_cast<unsigned long long>(next_id) + rel + mat > id_limit) raise_status(d.g, CHEM_ECAPACITY);
      atomicOr(&sb.any, 1u);
    } else {
      tr.rel_n = 0;
      tr.rel_mat = 0;
      tr.rel_park = 0;
    }
    tr.active = act ? 1 : 0;
    tr.free_jump = free_jump;
    sb.rel[b] = act ? parked + rel + mat : 0u;
    sb.dt[b] = act ? dt : 0.0;
  }
  __syncthreads();
  // cutoffs R + c sqrt(2 D_AB dt), bridge constants, and sigma = sqrt(2 D dt)
  const int per = MAXR + MAXT;
  for (uint32_t w = tid; w < d.n_trains * per; w += nt) {
    const uint32_t b = w / per;
    const int q = static_cast<int>(w % per);
    const double dt = sb.dt[b];
    if (dt <= 0.0) continue;  // train not advancing this step
    Train& tr = d.trains[b];
    if (q < MAXR) {
      if (q >= tb.n_rxn) continue;
      const double rc = __dadd_rn(tb.R[q], __dmul_rn(tr.c, sqrt(__dmul_rn(__dmul_rn(2.0, tb.D_AB[q]), dt))));
      tr.rc2[q] = __dmul_rn(rc, rc);
      tr.rc2f[q] = static_cast<float>(tr.rc2[q]);
      set_pair_constants(tr, tb, q, dt);
      atomicMax(&sb.rcmax_bits[b], static_cast<unsigned long long>(__double_as_longlong(rc)));
    } else {
      const int ty = q - MAXR;
      if (ty >= tb.n_types) continue;
      tr.sig[ty] = sqrt(__dmul_rn(__dmul_rn(2.0, tb.D[ty]), dt));
      tr.sigf[ty] = static_cast<float>(tr.sig[ty]);
    }
  }
  __syncthreads();
  for (uint32_t b = tid; b < d.n_trains; b += nt) {
    Train& tr = d.trains[b];
    if (b == 0) {  // the removed species' key below needs train 0's grid, idle or not
      sb.cb0 = tr.cb;
      sb.base0 = tr.cell_base;
    }
    if (sb.dt[b] <= 0.0) continue;
    const double L = tr.L, inv_L = tr.inv_L;
    const int n_max = min(tr.n_max, (1 << tr.cb_alloc) - 1), fj = tr.free_jump;
    int n_ref = tr.n_ref;
    const double rcmax = __longlong_as_double(static_cast<long long>(sb.rcmax_bits[b]));
    // finest admissible grid: cells at least the largest cutoff (with slack), at least 3
    // per axis (no cell met twice among a cell's neighbours)
    int n_target = n_max;
    if (rcmax > 0.0) {
      const float cut = static_cast<float>(rcmax) * CELL_SLACK_F;
      const float nf1 = floorf(static_cast<float>(L) / cut);
      n_target = max(3, min(n_max, static_cast<int>(fminf(nf1, 1048576.f))));
    }
    if (n_ref == 0) {  // first step after init or reset
      n_ref = n_target;
      tr.n_ref = n_target;
      tr.h_ref = __ddiv_rn(L, static_cast<double>(n_target));
      tr.cb_ref = axis_bits(n_target);
    }
    // keep the current grid while it is valid and at most 2x too coarse; when the
    // cutoff outgrows it, move to cells 1.2x larger than needed (fewer regrids)
    int n = n_ref;
    if (!fj) {
      if (n > n_target) n = max(3, (5 * n_target) / 6);
      else if (2 * n < n_target) n = n_target;
    }
    // the search looks one cell out: a cell must cover the largest cutoff
    if (!fj && rcmax > 0.0) {
      const double cut = rcmax * static_cast<double>(CELL_SLACK_F);
      if (L / static_cast<double>(n) < cut) n = n_target;
    }
    const double h = __ddiv_rn(L, static_cast<double>(n));
    const double inv_h = __dmul_rn(static_cast<double>(n), inv_L);
    tr.n = n;
    tr.cb = axis_bits(n);
    tr.h = h;
    tr.inv_h = inv_h;
    tr.hf = static_cast<float>(h);
    tr.inv_hf = static_cast<float>(inv_h);
    sb.hf[b] = static_cast<float>(h);
    if (b == 0) sb.cb0 = axis_bits(n);
  }
  __syncthreads();
  // per type pair (the pair search's lookup tables): the squared cutoff, in FP64 and
  // FP32, and the FP32 one widened past any error of FP32 cell offsets (a few 1e-7 of a
  // cell per component), so that a pair the FP32 test rejects is outside the FP64 cutoff
  for (uint32_t w = tid; w < d.n_trains * (MAXT * MAXT); w += nt) {
    const uint32_t b = w / (MAXT * MAXT);
    const int q = static_cast<int>(w % (MAXT * MAXT));
    if (sb.dt[b] <= 0.0) continue;
    Train& tr = d.trains[b];
    const int r = tb.pair_rxn[q / MAXT][q % MAXT];
    const double c2 = r >= 0 ? tr.rc2[r] : -1.0;
    const float c2f = r >= 0 ? static_cast<float>(c2) : -1.f;
    tr.rc2_tt[q] = c2;
    tr.rc2f_tt[q] = c2f;
    const float rc = c2f >= 0.f ? sqrtf(c2f) : -1.f;
    const float rw = rc * 1.00001f + 2e-6f * sb.hf[b];
    tr.rc2w_tt[q] = rc >= 0.f ? rw * rw * 1.00001f : -1.f;
  }
  if (tid == 0) {
    uint32_t off = g_total;
    const uint32_t before = off;
    unsigned long long total = off;
    for (uint32_t b = 0; b < d.n_trains; ++b) {
      d.trains[b].rel_off = off;
      total += sb.rel[b];
      off += sb.rel[b];
    }
    if (total > d.cap) {
      raise_status(g, CHEM_ECAPACITY);
      g->n_released = 0;
    } else {
      g->n_released = off - before;
      g->n_total = off;
    }
    for (int p = 0; p < MAX_PASSES; ++p) g->tile_ctr[p] = 0;
    g->n_cand = 0;
    g->n_conflict = 0;
    g->n_items = 0;
    g->item_ctr = 0;
    g->n_events = 0;
    g->n_products = 0;
    g->n_dead = 0;
    g->epoch = g_epoch + 1u;
    g->any_active = sb.any;
    // Search mapping of this step. Cell tiles amortise the neighbour-cell lookups over
    // the homes of a cell and test a pair only when the types react; one thread per
    // species has the shorter per-item latency chain. Adaptive: cell tiles when the last
    // step found more than 3 pairs inside the cutoffs per live species (the measured
    // crossover on track workloads); results do not depend on the mapping.
    uint32_t cells_now;
    if (g_adaptive) {
      const unsigned long long inc = g_incut - g_mark;
      cells_now = inc > 3ull * static_cast<unsigned long long>(g_live) ? 1u : 0u;
    } else {
      cells_now = g_home != 0u ? 1u : 0u;
    }
    g->search_cells_now = cells_now;
    g->incut_mark = g_incut;
    if (cells_now && sb.any) g->cells_steps = g_cells + 1u;
    // removed species sort after every live one: with one train the all-ones cell index
    // of the grid's width (this step's grid, or the last one when the train is idle; no
    // cell has it, and it stays within the bits the launched passes sort), so the top
    // key bits stay zero and their radix pass is skipped; with several trains, past the
    // last train's cells
    const int kb = min(3 * sb.cb0, 8 * d.passes);
    g->sentinel_step = d.n_trains == 1 ? sb.base0 + (kb >= 32 ? 0xFFFFFFFFu : (1u << kb) - 1u) : d.sentinel;
  }
  __syncthreads();
}

// Train whose release block holds `slot` (release offsets ascend with b).
__device__ __forceinline__ int train_of_release(const Dev& d, uint32_t slot) {
  int lo = 0, hi = static_cast<int>(d.n_trains) - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d.trains[mid].rel_off <= slot) lo = mid; else hi = mid - 1;
  }
  // skip empty blocks sharing the same offset
  while (lo > 0 && d.trains[lo].rel_n == 0) --lo;
  return lo;
}

// Warp-aggregated increment of counts[train][type].
__device__ __forceinline__ void count_add(const Dev& d, uint32_t b, uint32_t type, long long v,
                                          bool valid) {
  const uint32_t mask = __ballot_sync(0xffffffffu, valid);
  if (!valid) return;
  const uint32_t key = (b << 3) | type;
  const uint32_t peers = __match_any_sync(mask, key);
  const int lane = threadIdx.x & 31;
  if (lane == __ffs(peers) - 1)
    atomicAdd(reinterpret_cast<unsigned long long*>(&d.trains[b].counts[type]),
              static_cast<unsigned long long>(v * __popc(peers)));
}

// ======================================================================== release
// Position of a survivor of a homogeneous stage re-created with id `id`: uniform in the
// box, -L/2 + L u per axis with u from counter (id, 0, 0, 3) words (0,1) -> x, (2,3) -> y
// and counter (id, 1, 0, 3) words (0,1) -> z, then Eq. 1.
__device__ __forceinline__ void recreated_position(const Train& tr, uint32_t id, double& x, double& y,
                                                   double& z) {
  const uint4 a = philox4x32_10(make_uint4(id, 0u, 0u, 3u), tr.key0, tr.key1);
  const uint4 c = philox4x32_10(make_uint4(id, 1u, 0u, 3u), tr.key0, tr.key1);
  const double ux = __dmul_rn(static_cast<double>(u53(a.x, a.y)), TWO_POW_M53);
  const double uy = __dmul_rn(static_cast<double>(u53(a.z, a.w)), TWO_POW_M53);
  const double uz = __dmul_rn(static_cast<double>(u53(c.x, c.y)), TWO_POW_M53);
  x = wrap_box(__dadd_rn(-tr.halfL, __dmul_rn(tr.L, ux)), tr.L, tr.halfL);
  y = wrap_box(__dadd_rn(-tr.halfL, __dmul_rn(tr.L, uy)), tr.L, tr.halfL);
  z = wrap_box(__dadd_rn(-tr.halfL, __dmul_rn(tr.L, uz)), tr.L, tr.halfL);
}

// Type of the k-th re-created survivor (ascending type order).
__device__ __forceinline__ uint32_t recreated_type(const Train& tr, uint32_t k) {
  uint32_t ty = 0;
  while (ty + 1 < static_cast<uint32_t>(MAXT) && k >= tr.mat_cum[ty]) ++ty;
  return ty;
}

// ======================================================================== diffuse
// Displace every species of an active train (Sec. 2.1 SBS step) with periodic wrap
// (Eq. 1), compute its hash key, and accumulate the radix histograms of every pass.
// Species marked dead by the last step's reactions get the sentinel key. Species
// released this step (slots [n_total - n_released, n_total)) are first built from the
// pending queue (the release of Sec. 2.1) by the thread that then diffuses them.
template <bool F32L>
__device__ void phase_diffuse(const Dev& d, uint32_t (*hist)[RADIX]) {
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&hist[0][0])[i] = 0u;
  __syncthreads();
  // the trip count below must be the same for a whole warp (count_add votes)
  const bool ok = __shfl_sync(0xffffffffu, status_of(d) == 0 ? 1 : 0, 0) != 0;
  const uint32_t n_total = d.g->n_total;
  const uint32_t rel_base = n_total - d.g->n_released;
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t n_iter = ok ? (n_total + stride - 1) / stride : 0u;
  uint32_t n_dead_local = 0;
  // the next iteration's state of a stepped slot is loaded while this one is worked on
  // (released slots read their own sources below)
  uint32_t pf_cell = 0, pf_prev = 0, pf_tid = 0;
  bool pf_dead = false;
  float4 pf_v = make_float4(0.f, 0.f, 0.f, 0.f);
  double pf_x = 0, pf_y = 0, pf_z = 0;
  auto prefetch = [&](uint32_t s) {
    if (s < rel_base) {
      pf_cell = d.cell_sorted[s];
      pf_prev = s > 0 ? d.cell_sorted[s - 1] : 0u;
      pf_dead = d.dead[s] != 0;
      if (F32L) {
        pf_v = d.s4[s];
      } else {
        pf_x = d.sx[s]; pf_y = d.sy[s]; pf_z = d.sz[s]; pf_tid = d.stid[s];
      }
    }
  };
  if (n_iter > 0) prefetch(blockIdx.x * blockDim.x + threadIdx.x);
  for (uint32_t it = 0; it < n_iter; ++it) {
    const uint32_t s = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t c_cell = pf_cell, c_prev = pf_prev, c_tid = pf_tid;
    const bool c_dead = pf_dead;
    const float4 c_v = pf_v;
    const double c_x = pf_x, c_y = pf_y, c_z = pf_z;
    if (it + 1 < n_iter) prefetch(s + stride);
    const bool valid = s < n_total;
    const bool rel = valid && s >= rel_base;
    uint32_t rel_b = 0, rel_type = 0;
    bool rel_new = false;  // a released species not yet in the train's counts
    if (valid) {
      uint32_t key;
      uint32_t cell;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      double px = 0, py = 0, pz = 0;
      uint32_t tid = 0;
      bool dead = false;
      if (rel) {
        // release: re-created survivors of a homogeneous stage first, then the pending
        // queue; ids in that order (arrival, call order within the queue)
        rel_b = train_of_release(d, s);
        const Train& tr = d.trains[rel_b];
        const uint32_t kp = s - tr.rel_off;
        if (kp < tr.rel_park) {
          // an unparked species: its state and cell key as they were parked (the train's
          // grid has not changed since); it then takes the step like any other
          const uint32_t q = tr.park_base + kp;
          cell = d.pk_cell[q];
          if (F32L) {
            v = d.pk4[q];
            d.s4[s] = v;
          } else {
            px = d.pkx[q]; py = d.pky[q]; pz = d.pkz[q]; tid = d.pk_tid[q];
            d.sx[s] = px; d.sy[s] = py; d.sz[s] = pz; d.stid[s] = tid;
          }
          d.cell_sorted[s] = cell;
          d.dead[s] = 0;
        } else {
        const uint32_t k = kp - tr.rel_park;
        if (k < tr.rel_mat) {
          rel_type = recreated_type(tr, k);
          recreated_position(tr, tr.rel_id0 + k, px, py, pz);
        } else {
          const uint32_t p = tr.pend_base + tr.rel_p0 + (k - tr.rel_mat);
          rel_type = static_cast<uint32_t>(d.p_type[p]);
          px = d.px[p]; py = d.py[p]; pz = d.pz[p];
          rel_new = true;
        }
        tid = ((tr.rel_id0 + k) << 3) | rel_type;
        if (F32L) {
          const int n = tr.n_ref;
          const double h = tr.h_ref, inv_h = static_cast<double>(n) * tr.inv_L;
          const int ix = cell_index(px, tr.halfL, inv_h, n);
          const int iy = cell_index(py, tr.halfL, inv_h, n);
          const int iz = cell_index(pz, tr.halfL, inv_h, n);
          v = make_float4(static_cast<float>(__dsub_rn(__dadd_rn(px, tr.halfL), __dmul_rn(ix, h))),
                          static_cast<float>(__dsub_rn(__dadd_rn(py, tr.halfL), __dmul_rn(iy, h))),
                          static_cast<float>(__dsub_rn(__dadd_rn(pz, tr.halfL), __dmul_rn(iz, h))),
                          __uint_as_float(tid));
          cell = tr.cell_base + cell_encode(ix, iy, iz, tr.cb_ref);
          d.s4[s] = v;
        } else {
          cell = tr.cell_base;  // FP64 mode recomputes cells from positions
          d.sx[s] = px; d.sy[s] = py; d.sz[s] = pz; d.stid[s] = tid;
        }
        d.cell_sorted[s] = cell;
        d.dead[s] = 0;
        }  // unparked or new
      } else {
        cell = c_cell;
        // the occupancy bitmap is rebuilt by this step's gather: clear the words holding
        // the last step's cells (the first slot of each run of equal cells clears its
        // word; the last step's search has finished reading them)
        if (s == 0 || c_prev != cell) d.occ[cell >> 5] = 0u;
        dead = c_dead;
        if (dead) {
          d.dead[s] = 0;
        } else if (F32L) {
          v = c_v;
        } else {
          px = c_x; py = c_y; pz = c_z; tid = c_tid;
        }
      }
      if (dead) {
        key = d.g->sentinel_step;
        ++n_dead_local;
      } else {
        const int b = (d.n_trains == 1) ? 0 : train_of_cell(d.trains, d.n_trains, cell);
        const Train& tr = d.trains[b];
        if (!tr.active && tr.park_now) {
          // park: the species moves to its train's parking buffers and leaves the
          // stepped slots (sorted out with the removed ones)
          const uint32_t am = __activemask();
          const uint32_t peers = __match_any_sync(am, static_cast<uint32_t>(b));
          const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
          uint32_t base = 0;
          if (lane == leader) base = atomicAdd(&d.trains[b].park_n, static_cast<uint32_t>(__popc(peers)));
          base = __shfl_sync(peers, base, leader);
          const uint32_t k = base + __popc(peers & ((1u << lane) - 1u));
          if (k < tr.park_cap) {
            const uint32_t q = tr.park_base + k;
            d.pk_cell[q] = cell;
            if (F32L) d.pk4[q] = v;
            else { d.pkx[q] = px; d.pky[q] = py; d.pkz[q] = pz; d.pk_tid[q] = tid; }
          } else {
            raise_status(d.g, CHEM_ECAPACITY);
          }
          key = d.g->sentinel_step;
          ++n_dead_local;
        } else if (!tr.active) {
          if (F32L) d.t4[s] = v;
          else { d.tx[s] = px; d.ty[s] = py; d.tz[s] = pz; d.ttid[s] = tid; }
          key = cell;
        } else if (!F32L) {
          const uint32_t ty = tid_type(tid);
          double g0, g1, g2;
          gauss3_f64(tid_id(tid), tr.step, tr.key0, tr.key1, g0, g1, g2);
          const double sig = tr.sig[ty];
          const double ex = __dmul_rn(sig, g0), ey = __dmul_rn(sig, g1), ez = __dmul_rn(sig, g2);
          const double x = wrap_box(__dadd_rn(px, ex), tr.L, tr.halfL);
          const double y = wrap_box(__dadd_rn(py, ey), tr.L, tr.halfL);
          const double z = wrap_box(__dadd_rn(pz, ez), tr.L, tr.halfL);
          d.tx[s] = x; d.ty[s] = y; d.tz[s] = z; d.ttid[s] = tid;
          d.tdx[s] = ex; d.tdy[s] = ey; d.tdz[s] = ez;
          const int n = tr.n;
          const int ix = cell_index(x, tr.halfL, tr.inv_h, n);
          const int iy = cell_index(y, tr.halfL, tr.inv_h, n);
          const int iz = cell_index(z, tr.halfL, tr.inv_h, n);
          key = tr.cell_base + cell_encode(ix, iy, iz, tr.cb);
          if (d.t4) {  // FP32 offsets from the cell's corner for the pair search's prefilter
            d.t4[s] = make_float4(
                static_cast<float>(__dsub_rn(__dadd_rn(x, tr.halfL), __dmul_rn(static_cast<double>(ix), tr.h))),
                static_cast<float>(__dsub_rn(__dadd_rn(y, tr.halfL), __dmul_rn(static_cast<double>(iy), tr.h))),
                static_cast<float>(__dsub_rn(__dadd_rn(z, tr.halfL), __dmul_rn(static_cast<double>(iz), tr.h))),
                __uint_as_float(tid));
          }
        } else {
          const uint32_t ftid = __float_as_uint(v.w);
          const uint32_t ty = tid_type(ftid);
          float g0, g1, g2;
          gauss3_f32(tid_id(ftid), tr.step, tr.key0, tr.key1, g0, g1, g2);
          const float sig = tr.sigf[ty];
          const int nr = tr.n_ref;
          int ix, iy, iz;
          cell_decode(cell - tr.cell_base, tr.cb_ref, ix, iy, iz);
          const int n = tr.n;
          const float ex = sig * g0, ey = sig * g1, ez = sig * g2;
          d.td4[s] = make_float4(ex, ey, ez, 0.f);
          float ox, oy, oz;
          if (nr == n) {
            ox = v.x + ex; oy = v.y + ey; oz = v.z + ez;
            const float fx = floorf(ox * tr.inv_hf), fy = floorf(oy * tr.inv_hf), fz = floorf(oz * tr.inv_hf);
            ox -= fx * tr.hf; oy -= fy * tr.hf; oz -= fz * tr.hf;
            const int jx = static_cast<int>(fx), jy = static_cast<int>(fy), jz = static_cast<int>(fz);
            ix = (jx >= -1 && jx <= 1) ? step_cell(ix, jx, n) : wrap_cell(ix + jx, n);
            iy = (jy >= -1 && jy <= 1) ? step_cell(iy, jy, n) : wrap_cell(iy + jy, n);
            iz = (jz >= -1 && jz <= 1) ? step_cell(iz, jz, n) : wrap_cell(iz + jz, n);
          } else {
            // the hash grid changed this step: FP64 position from the box corner, then
            // the new cell and offset (no division)
            const double hr = tr.h_ref;
            const double ax = rebase_corner(ix * hr + static_cast<double>(v.x + ex), tr.L, tr.inv_L);
            const double ay = rebase_corner(iy * hr + static_cast<double>(v.y + ey), tr.L, tr.inv_L);
            const double az = rebase_corner(iz * hr + static_cast<double>(v.z + ez), tr.L, tr.inv_L);
            ix = min(static_cast<int>(ax * tr.inv_h), n - 1);
            iy = min(static_cast<int>(ay * tr.inv_h), n - 1);
            iz = min(static_cast<int>(az * tr.inv_h), n - 1);
            ox = static_cast<float>(ax - ix * tr.h);
            oy = static_cast<float>(ay - iy * tr.h);
            oz = static_cast<float>(az - iz * tr.h);
          }
          d.t4[s] = make_float4(ox, oy, oz, v.w);
          key = tr.cell_base + cell_encode(ix, iy, iz, tr.cb);
        }
      }
      d.keys0[s] = key;  // the first radix pass takes the slot itself as the value
      for (int p = 0; p < d.passes; ++p) atomicAdd(&hist[p][(key >> (8 * p)) & 255u], 1u);
    }
    count_add(d, rel_b, rel_type, 1, rel_new);
  }
  // warp-aggregate the dead count
  for (int o = 16; o > 0; o >>= 1) n_dead_local += __shfl_xor_sync(0xffffffffu, n_dead_local, o);
  if ((threadIdx.x & 31) == 0 && n_dead_local) atomicAdd(&d.g->n_dead, n_dead_local);
  __syncthreads();
  if (ok) {
    for (int i = threadIdx.x; i < d.passes * RADIX; i += blockDim.x) {
      const uint32_t c = (&hist[0][0])[i];
      if (c) atomicAdd(&d.g->hist[0][0] + i, c);
    }
  }
}

// ======================================================================== sort pass
// A pass whose digit is the same for every key is the identity and is skipped; the
// ping-pong buffers of the remaining passes follow from the histograms, which every CTA
// reads identically. Returns the number of executed passes before `pass` in *before.
__device__ __forceinline__ bool pass_active(const uint32_t (*hist)[RADIX], int pass, uint32_t n,
                                            int* before) {
  int cnt = 0;
  bool act = false;
  for (int q = 0; q <= pass; ++q) {
    const int trivial = __syncthreads_or(static_cast<int>(hist[q][threadIdx.x & (RADIX - 1)] == n));
    if (q < pass) cnt += trivial ? 0 : 1;
    else act = !trivial;
  }
  *before = cnt;
  return act;
}

// Status read once per CTA so that every thread takes the same branch before barriers.
__device__ __forceinline__ bool block_status_ok(const Dev& d) {
  return __syncthreads_and(threadIdx.x == 0 ? (status_of(d) == 0) : 1) != 0;
}

template <int NT>
__device__ void phase_sort_pass(const Dev& d, int pass, SortSmemT<NT>& sm) {
  if (!block_status_ok(d)) return;
  const uint32_t n = d.g->n_total;
  int before = 0;
  const bool act = pass_active(d.g->hist, pass, n, &before);
  if (pass == d.passes - 1 && blockIdx.x == 0 && threadIdx.x == 0) {
    d.g->sort_parity = static_cast<uint32_t>((before + (act ? 1 : 0)) & 1);
    d.g->sort_any = (before + (act ? 1 : 0)) > 0 ? 1u : 0u;
  }
  if (!act) return;
  const bool odd = before & 1;
  const uint32_t* kin = odd ? d.keys1 : d.keys0;
  const uint32_t* vin = before == 0 ? nullptr : (odd ? d.vals1 : d.vals0);  // nullptr: value = index
  uint32_t* kout = odd ? d.keys0 : d.keys1;
  uint32_t* vout = odd ? d.vals0 : d.vals1;
  onesweep_pass(kin, vin, kout, vout, n, 8 * pass, d.g->hist[pass], &d.g->tile_ctr[pass],
                d.lookback, d.g->epoch * 2 * MAX_PASSES + pass, d.g, sm);
}

// ======================================================================== gather
// Reorder the diffused species into cell order, record each cell's slot range (stamped
// with this step's epoch) and drop the dead (sentinel keys sort last).
template <bool F32L>
__device__ void phase_gather(const Dev& d) {
  if (status_of(d)) return;
  const uint32_t* kf = d.g->sort_parity ? d.keys1 : d.keys0;
  const uint32_t* vf = d.g->sort_any ? (d.g->sort_parity ? d.vals1 : d.vals0) : nullptr;
  const uint32_t n_total = d.g->n_total;
  const uint32_t n_live = n_total - d.g->n_dead;
  const uint32_t epoch = d.g->epoch;
  const uint32_t sentinel = d.g->sentinel_step;
  const uint32_t item_home = d.g->item_home;
  const bool items_now = item_home != 0 && d.g->search_cells_now;
  const uint32_t stride = gridDim.x * blockDim.x;
  // GATHER_BATCH slots per thread and iteration, their loads in flight together: the
  // permutation and neighbouring keys first, then the gathered state
  for (uint32_t s0 = blockIdx.x * blockDim.x + threadIdx.x; s0 < n_live; s0 += stride * GATHER_BATCH) {
    uint32_t key[GATHER_BATCH], idx[GATHER_BATCH], prv[GATHER_BATCH], nxt[GATHER_BATCH];
    bool ok[GATHER_BATCH];
#pragma unroll
    for (int g = 0; g < GATHER_BATCH; ++g) {
      const uint32_t s = s0 + static_cast<uint32_t>(g) * stride;
      ok[g] = s < n_live;
      key[g] = 0u; idx[g] = 0u; prv[g] = 0u; nxt[g] = 0u;
      if (ok[g]) {
        key[g] = kf[s];
        idx[g] = vf ? vf[s] : s;
        prv[g] = s > 0 ? kf[s - 1] : 0u;
        nxt[g] = s + 1 < n_live ? kf[s + 1] : 0u;
      }
    }
#pragma unroll
    for (int g = 0; g < GATHER_BATCH; ++g) {
      if (ok[g] && (key[g] >= sentinel || idx[g] >= n_total)) {  // only after a timed-out sort
        raise_status(d.g, CHEM_ETIMEOUT);
        ok[g] = false;
      }
    }
    if (F32L) {
      float4 a[GATHER_BATCH], b[GATHER_BATCH];
#pragma unroll
      for (int g = 0; g < GATHER_BATCH; ++g) {
        if (ok[g]) {
          a[g] = d.t4[idx[g]];
          if (d.sd4) b[g] = d.td4[idx[g]];
        }
      }
#pragma unroll
      for (int g = 0; g < GATHER_BATCH; ++g) {
        if (ok[g]) {
          const uint32_t s = s0 + static_cast<uint32_t>(g) * stride;
          d.s4[s] = a[g];
          if (d.sd4) d.sd4[s] = b[g];
        }
      }
    } else {
#pragma unroll
      for (int g = 0; g < GATHER_BATCH; ++g) {
        if (ok[g]) {
          const uint32_t s = s0 + static_cast<uint32_t>(g) * stride, i = idx[g];
          d.sx[s] = d.tx[i]; d.sy[s] = d.ty[i]; d.sz[s] = d.tz[i]; d.stid[s] = d.ttid[i];
          if (d.s4) d.s4[s] = d.t4[i];
        }
      }
    }
#pragma unroll
    for (int g = 0; g < GATHER_BATCH; ++g) {
      if (!ok[g]) continue;
      const uint32_t s = s0 + static_cast<uint32_t>(g) * stride, k = key[g];
      d.cell_sorted[s] = k;
      int* ci = reinterpret_cast<int*>(&d.cell_info[k]);
      const bool first = (s == 0 || prv[g] != k);
      if (first) {
        ci[0] = static_cast<int>(s);
        ci[2] = static_cast<int>(epoch);
        atomicOr(&d.occ[k >> 5], 1u << (k & 31u));
      }
      if (s + 1 == n_live || nxt[g] != k) ci[1] = static_cast<int>(s + 1);
      // pair-search work item: a cell's first slot and every item_home-th slot (none when
      // the search runs one thread per species)
      if (items_now && (first || (s % item_home) == 0)) {
        const int b = (d.n_trains == 1) ? 0 : train_of_cell(d.trains, d.n_trains, k);
        if (d.trains[b].active && !d.trains[b].free_jump) {
          const uint32_t it = atomicAdd(&d.g->n_items, 1u);
          if (it < d.cap_items) d.items[it] = make_uint2(s, k);
          else raise_status(d.g, CHEM_ECAPACITY);
        }
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) d.g->n_live = n_live;
}

// ======================================================================== search
// For every unordered pair of live species whose types react (Table 1), separated by
// less than the reaction's cutoff under the minimum image (Eq. 2), evaluate the
// encounter probability and keep the pair if its uniform falls below it. Two mappings
// visit the same pairs: one thread per home species (below) and cell tiles
// (search_cells.cuh). With at least 3 cells per axis each unordered pair is visited
// once: the own cell's later slots and the forward half of the surrounding cells.

// Half-shell offsets: entry 0 is the own cell, 1..13 the cells one away in fwd_offset's
// order; each keeps the offsets (dz, dy, dx) that are lexicographically positive, so
// every unordered pair of cells is met once.
struct FwdOffsets {
  signed char x[N_FWD], y[N_FWD], z[N_FWD];
  int count;
};
constexpr FwdOffsets make_fwd_offsets() {
  FwdOffsets t{};
  int k = 1;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) { t.x[k] = static_cast<signed char>(dx); t.y[k] = static_cast<signed char>(dy); t.z[k] = 1; ++k; }
  for (int dx = -1; dx <= 1; ++dx) { t.x[k] = static_cast<signed char>(dx); t.y[k] = 1; t.z[k] = 0; ++k; }
  t.x[k] = 1; t.y[k] = 0; t.z[k] = 0; ++k;
  t.count = k;
  return t;
}
static_assert(make_fwd_offsets().count == N_FWD, "13 forward cells");
static __constant__ FwdOffsets c_fwd = make_fwd_offsets();

// The half-shell offsets in shared memory: looked up with a different offset number in
// each lane, the constant-memory table would serialise a warp's access per distinct
// address. Filled by every thread of the CTA (fwd_smem_fill), then a CTA barrier.
struct FwdSmem {
  float f[3][N_FWD];       // as FP32 factors of the cell side
  int8_t i[3][N_FWD + 2];  // as cell steps
};

__device__ __forceinline__ void fwd_smem_fill(FwdSmem& fo) {
  for (int k = threadIdx.x; k < N_FWD; k += blockDim.x) {
    fo.f[0][k] = c_fwd.x[k]; fo.f[1][k] = c_fwd.y[k]; fo.f[2][k] = c_fwd.z[k];
    fo.i[0][k] = c_fwd.x[k]; fo.i[1][k] = c_fwd.y[k]; fo.i[2][k] = c_fwd.z[k];
  }
}

// Half-shell offsets: 0 = own cell, 1..9 dz = +1, 10..12 (dz, dy) = (0, +1), 13 (0, 0, +1).
__device__ __forceinline__ void fwd_offset(int k, int& dx, int& dy, int& dz) {
  if (k == 0) { dx = dy = dz = 0; return; }
  if (k <= 9) { const int q = k - 1; dz = 1; dy = q / 3 - 1; dx = q % 3 - 1; return; }
  if (k <= 12) { dz = 0; dy = 1; dx = k - 11; return; }
  dz = 0; dy = 0; dx = 1;
}

// FP32 separation x_j - x_i of two species held as offsets from their cells' corners,
// the neighbour's cell lying (cfx, cfy, cfz) cells away (cell side hf), and its square.
// Written with explicit roundings (no contraction left to the compiler) so that every
// kernel that forms it, both search mappings and the acceptance, gets the same bits.
__device__ __forceinline__ float sep_f32(float cfx, float cfy, float cfz, float hf, const float4& vj,
                                         const float4& vi, float& fx, float& fy, float& fz) {
  fx = __fsub_rn(__fmaf_rn(cfx, hf, vj.x), vi.x);
  fy = __fsub_rn(__fmaf_rn(cfy, hf, vj.y), vi.y);
  fz = __fsub_rn(__fmaf_rn(cfz, hf, vj.z), vi.z);
  return __fmaf_rn(fz, fz, __fmaf_rn(fy, fy, __fmul_rn(fx, fx)));
}

// Warp-reduced pair-search counters, added once per warp to the context's totals.
__device__ __forceinline__ void add_pair_counts(const Dev& d, uint32_t tested, uint32_t in_cut) {
  unsigned long long t = tested, c = in_cut;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (t) atomicAdd(&d.g->pairs_tested, t);
    if (c) atomicAdd(&d.g->pairs_in_cutoff, c);
  }
}

__device__ __forceinline__ void emit_candidate(const Dev& d, uint32_t s_lo, uint32_t s_hi, uint32_t id_lo,
                                               uint32_t id_hi, int r, int b, double d1sq) {
  const uint32_t c = atomicAdd(&d.g->n_cand, 1u);
  if (c >= d.cap_cand) { raise_status(d.g, CHEM_ECAPACITY); return; }
  atomicAdd(&d.touch[s_lo], 1u);
  atomicAdd(&d.touch[s_hi], 1u);
  Cand cd;
  cd.s_lo = s_lo; cd.s_hi = s_hi; cd.id_lo = id_lo; cd.id_hi = id_hi;
  cd.rxn_train = static_cast<uint32_t>(r) | (static_cast<uint32_t>(b) << 8);
  cd.pad = 0;
  cd.d1sq = d1sq;
  d.cand[c] = cd;
}

// Accept iff u < p with p = bridge_p evaluated in FP64 from the FP32 squared distances.
// The uniform u = (w0:w1 >> 11) 2^-53 of the pair's Philox block lies in
// [k 2^-24, (k + 1) 2^-24) with k = w0 >> 8, bounds that are exact in FP32. An FP32
// estimate of p decides whenever those bounds clear it by twice its error bound (FP32
// rounding of d0, d1, R and of the products, cancellation in d - R, the documented
// __expf error, and a few ulp for the two expm1f and their quotient, whose arguments
// suffer no cancellation since d0 + d1 - R > R); since p <= exp(-a), a uniform above the
// bound of exp(-a) alone rejects before the expm1f. Otherwise u and p are formed in FP64,
// so the outcome is always that of the FP64 test. The fast path uses no FP64
// arithmetic (a slow pipe on this part).
__device__ __forceinline__ bool accept_f32(float d0sq, float d1sq, int r, const Tables& tb, const Train& tr,
                                          uint32_t id_lo, uint32_t id_hi) {
  const float d1f = sqrtf(d1sq), d0f = sqrtf(d0sq);
  const float Rf = tb.Rf[r];
  if (d1f < Rf * 0.999f || d0f < Rf * 0.999f) return true;  // p = 1 > u
  const uint4 w = philox4x32_10(make_uint4(id_lo, tr.step, id_hi, 2u), tr.key0, tr.key1);
  if (d1f > Rf * 1.001f && d0f > Rf * 1.001f) {
    const float a = d0f - Rf, b = d1f - Rf, inv = tr.inv_ddt_f[r];
    const float x = a * b * inv;
    if (x > 60.f) {
      if ((w.x | (w.y >> 11)) != 0u) return false;  // p <= exp(-a) < 1e-26 < 2^-53 <= u
    } else {
      const float ea = __expf(-x);
      const float ulo = static_cast<float>(w.x >> 8) * 5.9604645e-8f;  // k 2^-24 <= u
      const float err = 1.2e-7f * inv * (b * (d0f + Rf) + a * (d1f + Rf)) + 1e-6f * (1.f + x) + 3e-6f;
      // p <= exp(-a): most pairs are rejected on that bound alone
      if (ulo >= ea * (1.f + 2.f * err)) return false;
      const float cb = d0f * d1f * inv, cc = Rf * (d0f + d1f - Rf) * inv;
      const float p = ea * (expm1f(-cc) / expm1f(-cb));
      const float band = 2.f * err * p;
      if (ulo >= p + band) return false;
      if (ulo + 5.9604645e-8f <= p - band) return true;               // u < (k + 1) 2^-24
    }
  }
  const double u = __dmul_rn(static_cast<double>(u53(w.x, w.y)), TWO_POW_M53);
  const double d0 = sqrt(static_cast<double>(d0sq)), d1 = sqrt(static_cast<double>(d1sq));
  return u < bridge_p(d0, d1, tb.R[r], tr.ddt[r]);
}

// The same test for FP64 squared distances: the FP32 estimate starts from their FP32
// roundings (one more rounding, covered by a doubled distance term in the error
// bound), and the exact fallback is the FP64 reference's own arithmetic.
__device__ __forceinline__ bool accept_f64(double d0sq, double d1sq, int r, const Tables& tb, const Train& tr,
                                          uint32_t id_lo, uint32_t id_hi) {
  const float d1f = sqrtf(static_cast<float>(d1sq)), d0f = sqrtf(static_cast<float>(d0sq));
  const float Rf = tb.Rf[r];
  if (d1f < Rf * 0.999f || d0f < Rf * 0.999f) return true;  // p = 1 > u
  const uint4 w = philox4x32_10(make_uint4(id_lo, tr.step, id_hi, 2u), tr.key0, tr.key1);
  if (d1f > Rf * 1.001f && d0f > Rf * 1.001f) {
    const float a = d0f - Rf, b = d1f - Rf, inv = tr.inv_ddt_f[r];
    const float x = a * b * inv;
    if (x > 60.f) {
      if ((w.x | (w.y >> 11)) != 0u) return false;
    } else {
      const float ea = __expf(-x);
      const float ulo = static_cast<float>(w.x >> 8) * 5.9604645e-8f;
      const float err = 2.4e-7f * inv * (b * (d0f + Rf) + a * (d1f + Rf)) + 1e-6f * (1.f + x) + 4e-6f;
      if (ulo >= ea * (1.f + 2.f * err)) return false;  // p <= exp(-a)
      const float cb = d0f * d1f * inv, cc = Rf * (d0f + d1f - Rf) * inv;
      const float p = ea * (expm1f(-cc) / expm1f(-cb));
      const float band = 2.f * err * p;
      if (ulo >= p + band) return false;
      if (ulo + 5.9604645e-8f <= p - band) return true;
    }
  }
  const double u = __dmul_rn(static_cast<double>(u53(w.x, w.y)), TWO_POW_M53);
  return u < bridge_p(sqrt(d0sq), sqrt(d1sq), tb.R[r], tr.ddt[r]);
}

// Neighbours whose loads one iteration of the per-species walk keeps in flight together.
constexpr int TPS_UNROLL = 4;

// ---- one thread per home species
// Each lane takes one home species (warps take 32 consecutive sorted slots by work
// stealing), keeps the forward cells its largest cutoff can reach (a 13-bit mask from
// per-axis face gaps), collects their non-empty ranges after its own cell's later slots,
// and walks them one range at a time, TPS_UNROLL neighbours per iteration. Lanes of one
// cell walk the same ranges in step, so their neighbour loads are broadcasts; the loops
// are warp-uniform (trip count = the longest walk among the lanes) and pairs inside the
// cutoff go to the warp's pair queue.

template <bool F32L>
struct TpsQueue;

template <>
struct TpsQueue<true> {
  static constexpr int CAP = 64;
  uint32_t si[CAP], j[CAP], tid_i[CAP], b[CAP];
  float fx[CAP], fy[CAP], fz[CAP], f2[CAP];
  uint32_t n;
};

template <>
struct TpsQueue<false> {
  static constexpr int CAP = 64;
  uint32_t si[CAP], j[CAP], tid_i[CAP], b[CAP];
  double rx[CAP], ry[CAP], rz[CAP], d2[CAP];
  uint32_t n;
};

template <bool F32L, int W>
struct TpsSmem {
  using T = float;            // FP32 cutoffs (FP64 mode: widened, for its FP32 prefilter)
  T ct[W][MAXT * MAXT];       // per warp: squared cutoffs of one train (-1: no reaction) ...
  int ct_b[W];                // ... that train
  uint32_t rs[W][N_FWD][32];  // per lane: its non-empty neighbour ranges [rs, re) ...
  uint32_t re[W][N_FWD][32];
  uint8_t rk[W][N_FWD][32];   // ... and their half-shell offsets
  TpsQueue<F32L> q[W];
  FwdSmem fo;                 // half-shell offsets
};

// Acceptance of one queued pair (home species given by slot and packed id/type).
template <bool F32L>
__device__ __forceinline__ void tps_accept(const Dev& d, const Tables& tb, const Train& tr, int b, uint32_t si,
                                           uint32_t tid_i, uint32_t j, uint32_t tid_j, float fx, float fy,
                                           float fz, float f2, double d1sq, double rx1, double ry1, double rz1,
                                           const uint32_t* vf) {
  const uint32_t ti = tid_type(tid_i), tj = tid_type(tid_j);
  const int r = tb.pair_rxn[ti][tj];
  const uint32_t id_i = tid_id(tid_i), id_j = tid_id(tid_j);
  const bool i_lo = id_i < id_j;
  const uint32_t id_lo = i_lo ? id_i : id_j, id_hi = i_lo ? id_j : id_i;
  if constexpr (F32L) {
    if (!i_lo) { fx = -fx; fy = -fy; fz = -fz; }
    const float4 di = d.td4[vf ? vf[si] : si];
    const float4 dj = d.td4[vf ? vf[j] : j];
    const float4 dlo = i_lo ? di : dj, dhi = i_lo ? dj : di;
    const float r0x = fx - (dhi.x - dlo.x), r0y = fy - (dhi.y - dlo.y), r0z = fz - (dhi.z - dlo.z);
    const float d0sq = r0x * r0x + r0y * r0y + r0z * r0z;
    if (!accept_f32(d0sq, f2, r, tb, tr, id_lo, id_hi)) return;
    emit_candidate(d, i_lo ? si : j, i_lo ? j : si, id_lo, id_hi, r, b, static_cast<double>(f2));
  } else {
    if (!i_lo) { rx1 = -rx1; ry1 = -ry1; rz1 = -rz1; }
    const uint32_t tj_idx = vf ? vf[j] : j, ti_idx = vf ? vf[si] : si;
    const double ejx = d.tdx[tj_idx], ejy = d.tdy[tj_idx], ejz = d.tdz[tj_idx];
    const double eix = d.tdx[ti_idx], eiy = d.tdy[ti_idx], eiz = d.tdz[ti_idx];
    const double elx = i_lo ? eix : ejx, ely = i_lo ? eiy : ejy, elz = i_lo ? eiz : ejz;
    const double ehx = i_lo ? ejx : eix, ehy = i_lo ? ejy : eiy, ehz = i_lo ? ejz : eiz;
    const double r0x = __dsub_rn(rx1, __dsub_rn(ehx, elx));
    const double r0y = __dsub_rn(ry1, __dsub_rn(ehy, ely));
    const double r0z = __dsub_rn(rz1, __dsub_rn(ehz, elz));
    if (!accept_f64(sq3(r0x, r0y, r0z), d1sq, r, tb, tr, id_lo, id_hi)) return;
    emit_candidate(d, i_lo ? si : j, i_lo ? j : si, id_lo, id_hi, r, b, d1sq);
  }
}

template <bool F32L>
__device__ __forceinline__ void tps_flush(const Dev& d, const Tables& tb, TpsQueue<F32L>& q, const uint32_t* vf,
                                          int lane) {
  const uint32_t nq = q.n;
  for (uint32_t e = lane; e < nq; e += 32) {
    const uint32_t j = q.j[e];
    const int b = static_cast<int>(q.b[e]);
    const Train& tr = d.trains[b];
    if constexpr (F32L)
      tps_accept<true>(d, tb, tr, b, q.si[e], q.tid_i[e], j, __float_as_uint(d.s4[j].w), q.fx[e], q.fy[e],
                       q.fz[e], q.f2[e], 0.0, 0.0, 0.0, 0.0, vf);
    else
      tps_accept<false>(d, tb, tr, b, q.si[e], q.tid_i[e], j, d.stid[j], 0.f, 0.f, 0.f, 0.f, q.d2[e], q.rx[e],
                        q.ry[e], q.rz[e], vf);
  }
  __syncwarp();
  if (lane == 0) q.n = 0;
  __syncwarp();
}

template <bool F32L, int W>
__device__ void phase_search_tps(const Dev& d, TpsSmem<F32L, W>& sm) {
  using T = typename TpsSmem<F32L, W>::T;
  if (d.g->search_cells_now) return;  // this step runs the cell tiles (grid-uniform)
  const uint32_t n_live = d.g->n_total - d.g->n_dead;
  const uint32_t epoch = d.g->epoch;
  const uint32_t* vf = d.g->sort_any ? (d.g->sort_parity ? d.vals1 : d.vals0) : nullptr;
  const Tables& tb = *d.tables;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  TpsQueue<F32L>& q = sm.q[wib];
  fwd_smem_fill(sm.fo);
  if (lane == 0) { q.n = 0; sm.ct_b[wib] = -1; }
  // one status for the whole CTA (a barrier, which also publishes the offsets)
  if (!block_status_ok(d)) return;
  const FwdSmem& fo = sm.fo;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  const uint32_t n_chunks = (n_live + 31u) / 32u;
  uint32_t n_tested = 0, n_in_cut = 0;  // pair-search counters of this lane
  uint32_t c_next = 0;
  if (lane == 0) c_next = atomicAdd(&d.g->item_ctr, 1u);
  c_next = __shfl_sync(0xffffffffu, c_next, 0);
  while (c_next < n_chunks) {
    const uint32_t c = c_next;
    if (lane == 0) c_next = atomicAdd(&d.g->item_ctr, 1u);  // the next chunk, used at the end
    const uint32_t s = c * 32u + static_cast<uint32_t>(lane);
    bool home = s < n_live;
    uint32_t tid_i = 0, cell = 0;
    float4 vi = make_float4(0.f, 0.f, 0.f, 0.f);
    double xi = 0, yi = 0, zi = 0;
    // FP64 mode tests pairs first on FP32 cell offsets against widened cutoffs (when the
    // context keeps them), then exactly in FP64
    const bool pref = F32L || d.s4 != nullptr;
    if (home) {
      cell = d.cell_sorted[s];
      if constexpr (F32L) { vi = d.s4[s]; tid_i = __float_as_uint(vi.w); }
      else {
        xi = d.sx[s]; yi = d.sy[s]; zi = d.sz[s]; tid_i = d.stid[s];
        if (pref) vi = d.s4[s];
      }
    }
    const int b = (d.n_trains == 1 || !home) ? 0 : train_of_cell(d.trains, d.n_trains, cell);
    const Train& tr = d.trains[b];
    const uint32_t ti = tid_type(tid_i);
    home = home && tr.active && !tr.free_jump && tb.reactive_mask[ti] != 0u;
    // cutoff row of this lane's type: from the warp's table of its train when every
    // lane of the chunk is in one train (refilled only when the train changes), else
    // from a per-lane row
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    const T* rc2;
    if (__all_sync(0xffffffffu, b == b0)) {
      if (sm.ct_b[wib] != b0) {
        const Train& t0 = d.trains[b0];
        for (int qq = lane; qq < MAXT * MAXT; qq += 32) {
          if constexpr (F32L) sm.ct[wib][qq] = t0.rc2f_tt[qq];
          else sm.ct[wib][qq] = t0.rc2w_tt[qq];
        }
        __syncwarp();
        if (lane == 0) sm.ct_b[wib] = b0;
        __syncwarp();
      }
      rc2 = &sm.ct[wib][ti * MAXT];
    } else {  // the rare chunk spanning several trains reads its rows from global memory
      if constexpr (F32L) rc2 = &tr.rc2f_tt[ti * MAXT];
      else rc2 = &tr.rc2w_tt[ti * MAXT];
    }
    if (__any_sync(0xffffffffu, home)) {
      // this lane's non-empty ranges: the own cell's later slots, then the forward cells
      // within reach that are occupied (bit test in the L2-resident bitmap, then their
      // 16-byte entries), collected (at most N_FWD ranges) and walked
      uint32_t* rs_l = &sm.rs[wib][0][lane];
      uint32_t* re_l = &sm.re[wib][0][lane];
      uint8_t* rk_l = &sm.rk[wib][0][lane];
      // bit 0: the own cell's later slots; bits 1..13: forward cells within reach
      uint32_t kmask = 0u;
      if (home) {
        int ix, iy, iz;
        cell_decode(cell - tr.cell_base, tr.cb, ix, iy, iz);
        if (s + 1u < static_cast<uint32_t>(d.cell_info[cell].y)) kmask = 1u;
        // a forward cell whose nearest point is farther from the home than the largest
        // cutoff of the home's type holds no partner and is not looked up (the gaps are
        // taken 1e-5 of a cell short, which covers every rounding of the offsets)
        const float hcell = tr.hf, eps = 1e-5f * tr.hf;
        float ofx, ofy, ofz;
        if constexpr (F32L) {
          ofx = vi.x; ofy = vi.y; ofz = vi.z;
        } else {
          ofx = static_cast<float>(__dsub_rn(__dadd_rn(xi, tr.halfL), __dmul_rn(static_cast<double>(ix), tr.h)));
          ofy = static_cast<float>(__dsub_rn(__dadd_rn(yi, tr.halfL), __dmul_rn(static_cast<double>(iy), tr.h)));
          ofz = static_cast<float>(__dsub_rn(__dadd_rn(zi, tr.halfL), __dmul_rn(static_cast<double>(iz), tr.h)));
        }
        float rcmax2 = -1.f;
#pragma unroll
        for (int t = 0; t < MAXT; ++t) rcmax2 = fmaxf(rcmax2, static_cast<float>(rc2[t]));
        rcmax2 *= 1.0001f;
        auto gap = [&](int o, float of) {
          const float g = o > 0 ? static_cast<float>(o) * hcell - of
                                : (o < 0 ? of + static_cast<float>(-o - 1) * hcell : 0.f);
          return fmaxf(g - eps, 0.f);
        };
        // per axis the gap is 0 (same layer), the distance to the lower face (offset -1)
        // or to the upper face (offset +1); the 13 offsets unrolled
        const float xm = gap(-1, ofx), xp = gap(1, ofx), ym = gap(-1, ofy), yp = gap(1, ofy);
        const float zp = gap(1, ofz);
        const float xm2 = xm * xm, xp2 = xp * xp, ym2 = ym * ym, yp2 = yp * yp, zp2 = zp * zp;
#pragma unroll
        for (int k = 1; k < N_FWD; ++k) {
          int dx, dy, dz;
          fwd_offset(k, dx, dy, dz);
          const float sx = dx < 0 ? xm2 : (dx > 0 ? xp2 : 0.f);
          const float sy = dy < 0 ? ym2 : (dy > 0 ? yp2 : 0.f);
          const float sz = dz > 0 ? zp2 : 0.f;
          if ((sx + sy) + sz <= rcmax2) kmask |= 1u << k;
        }
      }
      // the lane's home for the walk (ranges are not moved between lanes: on clustered
      // tracks, taking over half of a busy lane's range cost more issue slots than the
      // idle lanes it saved; dense cells go to the cell-tile mapping instead)
      const uint32_t hs = s, htid = tid_i;
      const int hb = b;
      const float4 hv = vi;
      const double hx = xi, hy = yi, hz = zi;
      const T* hrow = rc2;
      const Train* htr = &tr;
      // enqueue the pairs inside the cutoff (queue pushes are warp-wide)
      auto push = [&](bool pass, uint32_t jj, float fx, float fy, float fz, float f2, double rx1, double ry1,
                      double rz1, double d1sq) {
        const uint32_t bal = __ballot_sync(0xffffffffu, pass);
        if (bal) {
          const uint32_t base = q.n;
          if (pass) {
            const uint32_t pos = base + __popc(bal & lanemask_lt);
            q.si[pos] = hs; q.j[pos] = jj; q.tid_i[pos] = htid; q.b[pos] = static_cast<uint32_t>(hb);
            if constexpr (F32L) { q.fx[pos] = fx; q.fy[pos] = fy; q.fz[pos] = fz; q.f2[pos] = f2; }
            else { q.rx[pos] = rx1; q.ry[pos] = ry1; q.rz[pos] = rz1; q.d2[pos] = d1sq; }
          }
          __syncwarp();
          if (lane == 0) q.n = base + __popc(bal);
          __syncwarp();
          if (q.n > static_cast<uint32_t>(TpsQueue<F32L>::CAP) - 32u) tps_flush<F32L>(d, tb, q, vf, lane);
        }
      };
      int nr = 0;
      // look up only the cells within reach (warp-uniform loop over each lane's set bits:
      // at most N_FWD of them, so one pass collects them all)
      {
      // two cells per iteration, their bitmap words and then their entries loaded together
      while (__any_sync(0xffffffffu, kmask != 0u)) {
        int kk[2] = {-1, -1};
        if (kmask != 0u) {
          kk[0] = __ffs(kmask) - 1;
          kmask &= kmask - 1u;
        }
        if (kmask != 0u) {
          kk[1] = __ffs(kmask) - 1;
          kmask &= kmask - 1u;
        }
        uint32_t nc[2] = {0u, 0u}, word[2] = {0u, 0u};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (kk[q] > 0) {
            const int k = kk[q], n = tr.n;
            int ix, iy, iz;
            cell_decode(cell - tr.cell_base, tr.cb, ix, iy, iz);
            nc[q] = tr.cell_base + cell_encode(step_cell(ix, fo.i[0][k], n), step_cell(iy, fo.i[1][k], n),
                                               step_cell(iz, fo.i[2][k], n), tr.cb);
            word[q] = d.occ[nc[q] >> 5];
          }
        }
        int4 ci[2];
        bool occ[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          occ[q] = kk[q] > 0 && ((word[q] >> (nc[q] & 31u)) & 1u);
          ci[q] = occ[q] ? d.cell_info[nc[q]] : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (kk[q] == 0) {
            rs_l[0] = s + 1u;
            re_l[0] = static_cast<uint32_t>(d.cell_info[cell].y);
            rk_l[0] = 0;
            nr = 1;
          } else if (occ[q] && static_cast<uint32_t>(ci[q].z) == epoch && ci[q].y > ci[q].x) {
            rs_l[32 * nr] = static_cast<uint32_t>(ci[q].x);
            re_l[32 * nr] = static_cast<uint32_t>(ci[q].y);
            rk_l[32 * nr] = static_cast<uint8_t>(kk[q]);
            ++nr;
          }
        }
      }
      }
      // walk the ranges one after the other, TPS_UNROLL neighbours per iteration whose loads
      // are in flight together; lanes of one cell stay in step (broadcast loads)
      int ri = 0;
      uint32_t j = 0, je = 0;
      float cx = 0.f, cy = 0.f, cz = 0.f;
      auto open = [&](int r) {
        j = rs_l[32 * r];
        je = re_l[32 * r];
        const int k = rk_l[32 * r];
        cx = fo.f[0][k]; cy = fo.f[1][k]; cz = fo.f[2][k];  // in cells
      };
      if (nr > 0) open(0);
      while (__any_sync(0xffffffffu, ri < nr)) {
        // the next TPS_UNROLL neighbours of the lane's current range (one cell offset for
        // the batch; a range's last batch may be partly empty)
        uint32_t ju[TPS_UNROLL];
        bool vu[TPS_UNROLL];
        const bool act = ri < nr;
#pragma unroll
        for (int u = 0; u < TPS_UNROLL; ++u) {
          ju[u] = j + static_cast<uint32_t>(u);
          vu[u] = act && ju[u] < je;
        }
        const float bx = cx, by = cy, bz = cz;
        if (act) {
          j += TPS_UNROLL;
          if (j >= je && ++ri < nr) open(ri);
        }
        float4 vj[TPS_UNROLL];
        uint32_t tj[TPS_UNROLL];
#pragma unroll
        for (int u = 0; u < TPS_UNROLL; ++u) {
          vj[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          tj[u] = 0u;
          if (vu[u]) {
            if (pref) {
              vj[u] = d.s4[ju[u]];
              tj[u] = __float_as_uint(vj[u].w);
            } else {
              tj[u] = d.stid[ju[u]];
            }
          }
        }
        if constexpr (F32L) {
          // the cutoff test for the four neighbours first; the separation is formed again,
          // identically, for the rare pairs inside the cutoff
          auto sep = [&](int u, float& fx, float& fy, float& fz) {
            return sep_f32(bx, by, bz, htr->hf, vj[u], hv, fx, fy, fz);
          };
          bool pass[TPS_UNROLL];
          bool any = false;
#pragma unroll
          for (int u = 0; u < TPS_UNROLL; ++u) {
            float fx, fy, fz;
            const float rc2u = hrow[__float_as_uint(vj[u].w) & 7u];  // -1 when the types do not react
            pass[u] = vu[u] && sep(u, fx, fy, fz) < rc2u;
            any = any || pass[u];
            n_tested += (vu[u] && rc2u >= 0.f) ? 1u : 0u;  // reacting type pairs only
            n_in_cut += pass[u] ? 1u : 0u;
          }
          if (__any_sync(0xffffffffu, any)) {
#pragma unroll
            for (int u = 0; u < TPS_UNROLL; ++u) {
              float fx = 0.f, fy = 0.f, fz = 0.f, f2 = 0.f;
              if (pass[u]) f2 = sep(u, fx, fy, fz);
              push(pass[u], ju[u], fx, fy, fz, f2, 0.0, 0.0, 0.0, 0.0);
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < TPS_UNROLL; ++u) {
            const uint32_t jj = ju[u];
            bool pass = false;
            double rx1 = 0, ry1 = 0, rz1 = 0, d1sq = 0;
            if (vu[u]) {
              const uint32_t tjj = tj[u] & 7u;
              const float cw = hrow[tjj];  // widened FP32 bound, -1 when the types do not react
              bool near = cw >= 0.f;
              if (near && pref) {
                float fx, fy, fz;
                near = sep_f32(bx, by, bz, htr->hf, vj[u], hv, fx, fy, fz) < cw;
              }
              if (near) {
                const double c2 = htr->rc2_tt[tid_type(htid) * MAXT + tjj];
                // minimum image of x_j - x_i (Eq. 2); negated later into the reference's
                // x_hi - x_lo orientation, which is exact for pairs inside the cutoff
                rx1 = min_image(__dsub_rn(d.sx[jj], hx), htr->L, htr->halfL);
                ry1 = min_image(__dsub_rn(d.sy[jj], hy), htr->L, htr->halfL);
                rz1 = min_image(__dsub_rn(d.sz[jj], hz), htr->L, htr->halfL);
                d1sq = sq3(rx1, ry1, rz1);
                pass = d1sq < c2;
              }
            }
            n_tested += (vu[u] && hrow[tj[u] & 7u] >= 0.f) ? 1u : 0u;  // reacting type pairs only
            n_in_cut += pass ? 1u : 0u;
            push(pass, jj, 0.f, 0.f, 0.f, 0.f, rx1, ry1, rz1, d1sq);
          }
        }
      }
    }
    c_next = __shfl_sync(0xffffffffu, c_next, 0);
  }
  tps_flush<F32L>(d, tb, q, vf, lane);
  add_pair_counts(d, n_tested, n_in_cut);
}

// ======================================================================== react
// One reaction per species (Sec. 2.4: diffusion-controlled reactions, reactants react
// on encounter):
//  1. phase_match_fast (all CTAs): an accepted pair whose two species are in no other
//     accepted pair is committed at once; the others go to a conflict list.
//  2. phase_match_rounds (one CTA): rounds of locally-dominant selection over the
//     conflict list; a pair is committed when it is the smallest (d1^2, id_lo, id_hi)
//     remaining pair of both its species. Together with 1 this equals the greedy walk
//     over all accepted pairs sorted by that key (closest first, lower ids first).
//  3. phase_react_serial runs 2 and then, in the same CTA, orders the events by
//     (train, id_lo) with a block radix sort (in shared memory when they fit) and forms
//     the product-count prefix in that order;
//  4. phase_products (all CTAs): product ids and positions at the diffusion-weighted
//     encounter point (Table 1 right-hand sides), tallies summed per CTA, event log;
//  5. phase_end_step (one CTA): FP64 clock, step counter, dt growth, step records.
struct MatchSmem {
  uint32_t n_alive, n_next;
  uint32_t n_won, won_base;
};

// Events ordered in shared memory by the one-CTA react kernel (4 arrays of this size).
constexpr int EV_SMEM_CAP = 8192;

struct BlockSortSmem {
  uint32_t whist[REACT_THREADS / 32][RADIX];  // per warp: digit counts, then offsets
  uint32_t dtot[RADIX];                       // digit totals, then digit starts
  uint32_t trivial[4];                        // pass p has one digit for every key
};

struct ScanSmem {
  uint32_t carry;
  uint32_t warp_tot[REACT_THREADS / 32];
  uint32_t total;
  uint32_t first_pref[MAX_TRAINS];  // product prefix at the train's first event ...
  uint32_t first_k[MAX_TRAINS];     // ... and that event's position
  uint32_t prods_tr[MAX_TRAINS];
  uint32_t evs_tr[MAX_TRAINS];
};

struct ProductsSmem {
  int dcount[MAX_TRAINS][MAXT];
  int devents[MAX_TRAINS][MAXR];
  int dwater[MAX_TRAINS];
};

struct EndSmem {
  uint32_t any;
};

// Exclusive block-wide prefix of v (one value per thread); `total` gets the block sum.
// Warp totals are scanned once by warp 0.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_tot, uint32_t* total_s,
                                                    uint32_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    const uint32_t t = lane < nw ? warp_tot[lane] : 0u;
    uint32_t y = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    if (lane < nw) warp_tot[lane] = y - t;
    if (lane == 31) *total_s = y;
  }
  __syncthreads();
  total = *total_s;
  const uint32_t r = x - v + warp_tot[w];
  __syncthreads();
  return r;
}

__device__ __forceinline__ uint32_t event_key(const Dev& d, const Cand& cd) {
  const uint32_t b = cd.rxn_train >> 8;
  return d.train_bits ? ((b << (32 - d.train_bits)) | cd.id_lo) : cd.id_lo;
}

// Event value: candidate index (< 2^24) with the reaction's product count in bits 24-25.
constexpr uint32_t EV_CAND_MASK = 0xFFFFFFu;

// Consecutive indices from *counter for the lanes with `pred` set, one atomic per warp.
// Every lane of the warp must call it.
__device__ __forceinline__ uint32_t warp_reserve(uint32_t* counter, bool pred) {
  const uint32_t m = __ballot_sync(0xffffffffu, pred);
  const int lane = threadIdx.x & 31;
  const int leader = m ? __ffs(m) - 1 : 0;
  uint32_t base = 0;
  if (m && lane == leader) base = atomicAdd(counter, static_cast<uint32_t>(__popc(m)));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + static_cast<uint32_t>(__popc(m & ((1u << lane) - 1u)));
}

// Record accepted pair c as event number e (reserved by the caller).
__device__ __forceinline__ void commit_event(const Dev& d, uint32_t c, const Cand& cd, uint32_t e) {
  d.dead[cd.s_lo] = 1;
  d.dead[cd.s_hi] = 1;
  d.ev_k0[e] = event_key(d, cd);
  d.ev_v0[e] = c | (static_cast<uint32_t>(d.tables->n_prod[cd.rxn_train & 255u]) << 24);
}

static __device__ void phase_match_fast(const Dev& d) {
  const bool ok = block_status_ok(d);  // includes a barrier
  const uint32_t n_c = ok ? min(d.g->n_cand, d.cap_cand) : 0u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t c0 = blockIdx.x * blockDim.x; c0 < n_c; c0 += stride) {  // uniform per block
    const uint32_t c = c0 + threadIdx.x;
    const bool valid = c < n_c;
    Cand cd{};
    bool lone = false;
    if (valid) {
      cd = d.cand[c];
      lone = d.touch[cd.s_lo] == 1u && d.touch[cd.s_hi] == 1u;
    }
    const uint32_t e = warp_reserve(&d.g->n_events, valid && lone);
    const uint32_t a = warp_reserve(&d.g->n_conflict, valid && !lone);
    if (valid && lone) {
      commit_event(d, c, cd, e);
      d.touch[cd.s_lo] = 0u;
      d.touch[cd.s_hi] = 0u;
    } else if (valid) {
      d.alive0[a] = c;
    }
  }
}

static __device__ void phase_match_rounds(const Dev& d, MatchSmem& sm) {
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  const bool ok = block_status_ok(d);
  unsigned long long* bd = reinterpret_cast<unsigned long long*>(d.keys0);
  unsigned long long* bp = bd + d.cap;
  const uint32_t n_c = ok ? d.g->n_conflict : 0u;
  if (tid == 0) sm.n_alive = n_c;
  // the rounds do not use the accepted-pair counts: reset them for the next step now
  for (uint32_t i = tid; i < n_c; i += nt) {
    const Cand cd = d.cand[d.alive0[i]];
    d.touch[cd.s_lo] = 0u;
    d.touch[cd.s_hi] = 0u;
  }
  __syncthreads();
  uint32_t* alive = d.alive0;
  uint32_t* nxt = d.alive1;
  for (uint32_t round = 0; sm.n_alive > 0; ++round) {
    if (round > n_c) {
      if (tid == 0) raise_status(d.g, CHEM_ESTATE);
      break;
    }
    const uint32_t na = sm.n_alive;
    for (uint32_t i = tid; i < na; i += nt) {
      const Cand cd = d.cand[alive[i]];
      bd[cd.s_lo] = ~0ull; bd[cd.s_hi] = ~0ull;
      bp[cd.s_lo] = ~0ull; bp[cd.s_hi] = ~0ull;
    }
    __syncthreads();
    for (uint32_t i = tid; i < na; i += nt) {
      const Cand cd = d.cand[alive[i]];
      const unsigned long long kd = __double_as_longlong(cd.d1sq);
      atomicMin(&bd[cd.s_lo], kd);
      atomicMin(&bd[cd.s_hi], kd);
    }
    __syncthreads();
    for (uint32_t i = tid; i < na; i += nt) {
      const Cand cd = d.cand[alive[i]];
      const unsigned long long kd = __double_as_longlong(cd.d1sq);
      const unsigned long long kp = (static_cast<unsigned long long>(cd.id_lo) << 32) | cd.id_hi;
      if (bd[cd.s_lo] == kd) atomicMin(&bp[cd.s_lo], kp);
      if (bd[cd.s_hi] == kd) atomicMin(&bp[cd.s_hi], kp);
    }
    __syncthreads();
    for (uint32_t i0 = 0; i0 < na; i0 += nt) {  // uniform trip count (warp_reserve)
      const uint32_t i = i0 + tid;
      bool win = false;
      uint32_t c = 0;
      Cand cd{};
      if (i < na) {
        c = alive[i];
        cd = d.cand[c];
        const unsigned long long kd = __double_as_longlong(cd.d1sq);
        const unsigned long long kp = (static_cast<unsigned long long>(cd.id_lo) << 32) | cd.id_hi;
        win = bd[cd.s_lo] == kd && bp[cd.s_lo] == kp && bd[cd.s_hi] == kd && bp[cd.s_hi] == kp;
      }
      const uint32_t e = warp_reserve(&d.g->n_events, win);
      if (win) commit_event(d, c, cd, e);
    }
    if (tid == 0) sm.n_next = 0;
    __syncthreads();
    for (uint32_t i0 = 0; i0 < na; i0 += nt) {
      const uint32_t i = i0 + tid;
      bool keep = false;
      uint32_t c = 0;
      if (i < na) {
        c = alive[i];
        const Cand cd = d.cand[c];
        keep = !d.dead[cd.s_lo] && !d.dead[cd.s_hi];
      }
      const uint32_t a = warp_reserve(&sm.n_next, keep);
      if (keep) nxt[a] = c;
    }
    __syncthreads();
    if (tid == 0) sm.n_alive = sm.n_next;
    uint32_t* tmp = alive; alive = nxt; nxt = tmp;
    __syncthreads();
  }
  __syncthreads();
}

// The conflict rounds of phase_match_rounds with everything in shared memory: the
// conflict pairs, a hash of their slots to local indices, and per local slot the
// smallest (d1^2) and then smallest (id_lo, id_hi) key of its remaining pairs. Returns
// false (nothing done) when the conflict list does not fit; the caller then runs the
// global-memory version. `sbuf` holds RC_SMEM_BYTES.
constexpr int RC_CAP = 1536;                 // conflict pairs
constexpr int RC_SLOTS = 2 * RC_CAP;         // distinct slots at most
constexpr int RC_HASH = 8192;                // >= 2 RC_SLOTS, power of two
constexpr size_t RC_SMEM_BYTES = static_cast<size_t>(RC_CAP) * (4 + 4 + 4 + 8 + 8) +
                                 static_cast<size_t>(RC_HASH) * 8 + static_cast<size_t>(RC_SLOTS) * (8 + 8 + 4) +
                                 static_cast<size_t>(RC_CAP) * 8;

static __device__ bool phase_match_rounds_smem(const Dev& d, MatchSmem& sm, uint32_t* sbuf) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool ok = block_status_ok(d);
  const uint32_t n_c = ok ? d.g->n_conflict : 0u;
  if (n_c > static_cast<uint32_t>(RC_CAP)) return false;  // uniform
  // carve the buffer (8-byte arrays first)
  unsigned long long* kd = reinterpret_cast<unsigned long long*>(sbuf);
  unsigned long long* kp = kd + RC_CAP;
  unsigned long long* bd = kp + RC_CAP;
  unsigned long long* bp = bd + RC_SLOTS;
  uint32_t* hkey = reinterpret_cast<uint32_t*>(bp + RC_SLOTS);
  uint32_t* hval = hkey + RC_HASH;
  uint32_t* lo = hval + RC_HASH;
  uint32_t* hi = lo + RC_CAP;
  uint32_t* cix = hi + RC_CAP;
  uint32_t* alive = cix + RC_CAP;
  uint32_t* nxt = alive + RC_CAP;
  uint32_t* ldead = nxt + RC_CAP;
  for (int i = tid; i < RC_HASH; i += nt) hkey[i] = 0xFFFFFFFFu;
  for (int i = tid; i < RC_SLOTS; i += nt) ldead[i] = 0u;
  if (tid == 0) { sm.n_alive = n_c; sm.n_next = 0; }
  __syncthreads();
  // load the pairs, reset the accepted-pair counts for the next step, insert the slots
  for (uint32_t i = tid; i < n_c; i += nt) {
    const uint32_t c = d.alive0[i];
    const Cand cd = d.cand[c];
    d.touch[cd.s_lo] = 0u;
    d.touch[cd.s_hi] = 0u;
    cix[i] = c;
    kd[i] = static_cast<unsigned long long>(__double_as_longlong(cd.d1sq));
    kp[i] = (static_cast<unsigned long long>(cd.id_lo) << 32) | cd.id_hi;
    lo[i] = cd.s_lo;
    hi[i] = cd.s_hi;
    alive[i] = i;
  }
  __syncthreads();
  // slot -> local index: open addressing; the thread whose CAS claims a bucket numbers it
  for (uint32_t e = tid; e < 2 * n_c; e += nt) {
    const uint32_t slot = (e & 1u) ? hi[e >> 1] : lo[e >> 1];
    uint32_t h = (slot * 2654435761u) & (RC_HASH - 1);
    for (int probe = 0; probe < RC_HASH; ++probe) {
      const uint32_t prev = atomicCAS(&hkey[h], 0xFFFFFFFFu, slot);
      if (prev == 0xFFFFFFFFu) { hval[h] = atomicAdd(&sm.n_next, 1u); break; }
      if (prev == slot) break;
      h = (h + 1u) & (RC_HASH - 1);
    }
  }
  __syncthreads();
  for (uint32_t e = tid; e < 2 * n_c; e += nt) {
    const uint32_t slot = (e & 1u) ? hi[e >> 1] : lo[e >> 1];
    uint32_t h = (slot * 2654435761u) & (RC_HASH - 1);
    for (int probe = 0; probe < RC_HASH && hkey[h] != slot; ++probe) h = (h + 1u) & (RC_HASH - 1);
    if (e & 1u) hi[e >> 1] = hval[h]; else lo[e >> 1] = hval[h];
  }
  __syncthreads();
  // winners are listed in shared memory (the hash values are no longer needed) and
  // recorded as events after the last round with one reservation
  uint32_t* won = hval;
  if (tid == 0) sm.n_won = 0;
  for (uint32_t a = tid; a < n_c; a += nt) {
    const uint32_t i = alive[a];
    bd[lo[i]] = ~0ull; bd[hi[i]] = ~0ull;
    bp[lo[i]] = ~0ull; bp[hi[i]] = ~0ull;
  }
  __syncthreads();
  for (uint32_t round = 0; sm.n_alive > 0; ++round) {
    if (round > n_c) {
      if (tid == 0) raise_status(d.g, CHEM_ESTATE);
      break;
    }
    const uint32_t na = sm.n_alive;
    for (uint32_t a = tid; a < na; a += nt) {
      const uint32_t i = alive[a];
      atomicMin(&bd[lo[i]], kd[i]);
      atomicMin(&bd[hi[i]], kd[i]);
    }
    __syncthreads();
    for (uint32_t a = tid; a < na; a += nt) {
      const uint32_t i = alive[a];
      if (bd[lo[i]] == kd[i]) atomicMin(&bp[lo[i]], kp[i]);
      if (bd[hi[i]] == kd[i]) atomicMin(&bp[hi[i]], kp[i]);
    }
    __syncthreads();
    for (uint32_t a0 = 0; a0 < na; a0 += nt) {  // uniform trip count (warp_reserve)
      const uint32_t a = a0 + tid;
      bool win = false;
      uint32_t i = 0;
      if (a < na) {
        i = alive[a];
        win = bd[lo[i]] == kd[i] && bp[lo[i]] == kp[i] && bd[hi[i]] == kd[i] && bp[hi[i]] == kp[i];
      }
      const uint32_t q = warp_reserve(&sm.n_won, win);
      if (win) {
        ldead[lo[i]] = 1u;
        ldead[hi[i]] = 1u;
        won[q] = i;
      }
    }
    if (tid == 0) sm.n_next = 0;
    __syncthreads();
    // survivors (both species still free) move to the next round with their slots'
    // minima reset; nothing reads the minima in this pass
    for (uint32_t a0 = 0; a0 < na; a0 += nt) {
      const uint32_t a = a0 + tid;
      bool keep = false;
      uint32_t i = 0;
      if (a < na) {
        i = alive[a];
        keep = !ldead[lo[i]] && !ldead[hi[i]];
      }
      const uint32_t q = warp_reserve(&sm.n_next, keep);
      if (keep) {
        nxt[q] = i;
        bd[lo[i]] = ~0ull; bd[hi[i]] = ~0ull;
        bp[lo[i]] = ~0ull; bp[hi[i]] = ~0ull;
      }
    }
    __syncthreads();
    if (tid == 0) sm.n_alive = sm.n_next;
    uint32_t* t = alive; alive = nxt; nxt = t;
    __syncthreads();
  }
  if (tid == 0) sm.won_base = atomicAdd(&d.g->n_events, sm.n_won);
  __syncthreads();
  for (uint32_t q = tid; q < sm.n_won; q += nt) {
    const uint32_t c = cix[won[q]];
    commit_event(d, c, d.cand[c], sm.won_base + q);
  }
  __syncthreads();
  return true;
}

// Sort of n (key, value) pairs by the whole CTA, in shared memory (keys are distinct
// here; equal keys would be ordered by value): one counting pass over 2048 buckets of
// the key range (bucket = (key - min) >> shift), then each key's rank inside its bucket
// by comparison with the bucket's other keys (buckets hold a handful of keys for the
// id-like keys sorted here). The result is in (k0, v0); (k1, v1) is scratch. Returns
// false, with nothing changed, when a bucket holds more than 64 keys (clustered keys)
// or the CTA is not 1024 threads; the caller then uses block_sort_pairs.
constexpr int BUCKETS = 2048;
static __device__ bool block_bucket_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t n,
                                         BlockSortSmem& sm, ScanSmem& ss) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5;
  if (2 * nt != BUCKETS) return false;     // two buckets per thread in the scan below
  uint32_t* cnt = &sm.whist[0][0];         // BUCKETS counts, then exclusive starts
  uint32_t* cur = cnt + BUCKETS;           // scatter cursors, then bucket ends
  uint32_t* red = cnt + 2 * BUCKETS;       // per-warp min / max / largest bucket
  // key range
  uint32_t mn = 0xFFFFFFFFu, mx = 0u;
  for (uint32_t i = tid; i < n; i += nt) { mn = min(mn, k0[i]); mx = max(mx, k0[i]); }
  mn = __reduce_min_sync(0xffffffffu, mn);
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) { red[w] = mn; red[32 + w] = mx; }
  for (int i = tid; i < BUCKETS; i += nt) cnt[i] = 0u;
  __syncthreads();
  mn = 0xFFFFFFFFu; mx = 0u;
  for (int q = 0; q < (nt >> 5); ++q) { mn = min(mn, red[q]); mx = max(mx, red[32 + q]); }
  const uint32_t range = n ? mx - mn : 0u;
  const int bits = range ? 32 - __clz(range) : 0;
  const int shift = bits > 11 ? bits - 11 : 0;
  for (uint32_t i = tid; i < n; i += nt) atomicAdd(&cnt[(k0[i] - mn) >> shift], 1u);
  __syncthreads();
  // largest bucket (clustered keys would make the in-bucket ranks quadratic)
  uint32_t big = 0u;
  for (int i = tid; i < BUCKETS; i += nt) big = max(big, cnt[i]);
  big = __reduce_max_sync(0xffffffffu, big);
  if (lane == 0) red[64 + w] = big;
  // exclusive starts: each thread scans two consecutive buckets
  const uint32_t c0 = cnt[2 * tid], c1 = cnt[2 * tid + 1];
  uint32_t tot;
  const uint32_t ex = block_excl_scan(c0 + c1, ss.warp_tot, &ss.total, tot);
  big = 0u;
  for (int q = 0; q < (nt >> 5); ++q) big = max(big, red[64 + q]);
  if (big > 64u) return false;  // uniform: every thread read the same values
  cnt[2 * tid] = ex; cnt[2 * tid + 1] = ex + c0;
  cur[2 * tid] = ex; cur[2 * tid + 1] = ex + c0;
  __syncthreads();
  for (uint32_t i = tid; i < n; i += nt) {
    const uint32_t b = (k0[i] - mn) >> shift;
    const uint32_t p = atomicAdd(&cur[b], 1u);
    k1[p] = k0[i];
    v1[p] = v0[i];
  }
  __syncthreads();
  for (uint32_t p = tid; p < n; p += nt) {
    const uint32_t k = k1[p], v = v1[p];
    const uint32_t b = (k - mn) >> shift;
    const uint32_t lo = cnt[b], hi = cur[b];
    uint32_t r = 0;
    for (uint32_t q = lo; q < hi; ++q) r += (k1[q] < k || (k1[q] == k && v1[q] < v)) ? 1u : 0u;
    k0[lo + r] = k;
    v0[lo + r] = v;
  }
  __syncthreads();
  return true;
}

// Stable LSD radix sort of n (key, value) pairs by the whole CTA, 8-bit digits over the
// 32 key bits. Each warp owns one contiguous chunk of the input and scatters it in order
// (ranks among equal digits from match_digit8), so equal digits keep their order.
// A pass whose digit is the same for every key is skipped. The arrays may live in shared
// or global memory. Returns 0 when the result is in (k0, v0), 1 when in (k1, v1).
static __device__ int block_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t n,
                                BlockSortSmem& sm) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  const uint32_t chunk = (n + static_cast<uint32_t>(nw) - 1u) / static_cast<uint32_t>(nw);
  const uint32_t lo = min(n, static_cast<uint32_t>(w) * chunk), hi = min(n, lo + chunk);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t *kin = k0, *vin = v0, *kout = k1, *vout = v1;
  int parity = 0;
  if (tid < 4) sm.trivial[tid] = 0u;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 8 * pass;
    for (int i = tid; i < nw * RADIX; i += nt) (&sm.whist[0][0])[i] = 0u;
    __syncthreads();
    for (uint32_t i = lo + lane; i < hi; i += 32) atomicAdd(&sm.whist[w][(kin[i] >> shift) & 255u], 1u);
    __syncthreads();
    for (int dg = tid; dg < RADIX; dg += nt) {
      uint32_t run = 0;
      for (int q = 0; q < nw; ++q) {
        const uint32_t c = sm.whist[q][dg];
        sm.whist[q][dg] = run;
        run += c;
      }
      sm.dtot[dg] = run;
      if (run == n) sm.trivial[pass] = 1u;
    }
    __syncthreads();
    if (sm.trivial[pass]) continue;  // the same value for every thread
    if (w == 0) {
      uint32_t carry = 0;
      for (int base = 0; base < RADIX; base += 32) {
        const uint32_t v = sm.dtot[base + lane];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        sm.dtot[base + lane] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
      }
    }
    __syncthreads();
    for (uint32_t b0 = lo; b0 < hi; b0 += 32) {
      const uint32_t i = b0 + lane;
      const bool act = i < hi;
      uint32_t key = 0, val = 0, dg = RADIX;  // inactive lanes form their own group
      if (act) {
        key = kin[i];
        val = vin[i];
        dg = (key >> shift) & 255u;
      }
      const uint32_t peers = match_digit8(dg, __ballot_sync(0xffffffffu, act));
      if (act) {
        const uint32_t dst = sm.dtot[dg] + sm.whist[w][dg] + __popc(peers & lt);
        kout[dst] = key;
        vout[dst] = val;
      }
      __syncwarp();
      if (act && (peers & lt) == 0u) sm.whist[w][dg] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    uint32_t* t = kin; kin = kout; kout = t;
    t = vin; vin = vout; vout = t;
    parity ^= 1;
  }
  return parity;
}

// Product-count prefix over the ordered events (`order`, optionally copied to
// `order_out`), written to `pref`, plus each train's first prefix, event and product
// counts.
static __device__ void products_prefix(const Dev& d, ScanSmem& sm, const uint32_t* okeys, const uint32_t* order,
                                       uint32_t* order_out, uint32_t* pref, uint32_t E, bool ok) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tshift = 32 - static_cast<int>(d.train_bits);
  for (uint32_t b = tid; b < d.n_trains; b += nt) {
    sm.first_pref[b] = 0; sm.first_k[b] = 0; sm.prods_tr[b] = 0; sm.evs_tr[b] = 0;
  }
  // each thread takes one contiguous segment of the ordered events: its product count,
  // one block-wide scan of the segment sums, then the per-event prefixes in the segment
  const uint32_t seg = (E + static_cast<uint32_t>(nt) - 1u) / static_cast<uint32_t>(nt);
  const uint32_t k0 = min(E, static_cast<uint32_t>(tid) * seg), k1 = min(E, k0 + seg);
  uint32_t local = 0;
  for (uint32_t k = k0; k < k1; ++k) local += order[k] >> 24;
  uint32_t total;
  uint32_t ex = block_excl_scan(local, sm.warp_tot, &sm.total, total);  // includes barriers
  // train boundaries: a train's counts are differences at its last event (events are in
  // train order)
  for (uint32_t k = k0; k < k1; ++k) {
    const uint32_t v = order[k];
    pref[k] = ex;
    if (order_out) order_out[k] = v;
    const uint32_t b = d.train_bits ? okeys[k] >> tshift : 0u;
    if (k == 0 || (d.train_bits && (okeys[k - 1] >> tshift) != b)) { sm.first_pref[b] = ex; sm.first_k[b] = k; }
    ex += v >> 24;
  }
  __syncthreads();
  for (uint32_t k = k0; k < k1; ++k) {
    const uint32_t b = d.train_bits ? okeys[k] >> tshift : 0u;
    if (k + 1 == E || (d.train_bits && (okeys[k + 1] >> tshift) != b)) {
      sm.prods_tr[b] = pref[k] + (order[k] >> 24) - sm.first_pref[b];
      sm.evs_tr[b] = k + 1 - sm.first_k[b];
    }
  }
  __syncthreads();
  for (uint32_t b = tid; b < d.n_trains; b += nt) {
    Train& tr = d.trains[b];
    tr.pref0 = sm.first_pref[b];
    tr.prods_step = sm.prods_tr[b];
    tr.n_events_step = sm.evs_tr[b];
  }
  if (tid == 0 && ok) d.g->n_products = total;
  __syncthreads();
}

struct SerialSmem {
  MatchSmem match;
  BlockSortSmem sort;
  ScanSmem scan;
};

// The one-CTA part of the react phase: conflict rounds, event order, product prefix.
// With `sbuf` (4 * EV_SMEM_CAP words of shared memory) and at most EV_SMEM_CAP events
// the sort runs in shared memory; otherwise in the global event buffers.
static __device__ void phase_react_serial(const Dev& d, SerialSmem& sm, uint32_t* sbuf) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint32_t n_conflict = d.g->n_conflict;  // read before the rounds (all threads, uniform)
  const bool rounds_smem = sbuf != nullptr && phase_match_rounds_smem(d, sm.match, sbuf);
  if (!rounds_smem) phase_match_rounds(d, sm.match);
  const bool ok = block_status_ok(d);
  const uint32_t E = ok ? min(d.g->n_events, d.cap_cand) : 0u;
  const uint32_t* okeys;
  const uint32_t* order;
  uint32_t* order_out = nullptr;
  uint32_t* pref;
  if (tid == 0 && ok) {  // branch record (read by chem_get_stats)
    Global* g = d.g;
    if (!rounds_smem && n_conflict > 0) g->react_rounds_global += 1;
    if (n_conflict > g->max_conflict) g->max_conflict = n_conflict;
    g->pairs_accepted += min(g->n_cand, d.cap_cand);
    if (E > g->max_events) g->max_events = E;
    if (E > 0 && (sbuf == nullptr || E > static_cast<uint32_t>(EV_SMEM_CAP))) g->react_order_global += 1;
  }
  if (sbuf != nullptr && E <= static_cast<uint32_t>(EV_SMEM_CAP)) {
    uint32_t* k0 = sbuf;
    uint32_t* v0 = sbuf + EV_SMEM_CAP;
    uint32_t* k1 = sbuf + 2 * EV_SMEM_CAP;
    uint32_t* v1 = sbuf + 3 * EV_SMEM_CAP;
    for (uint32_t i = tid; i < E; i += nt) { k0[i] = d.ev_k0[i]; v0[i] = d.ev_v0[i]; }
    __syncthreads();
    const bool bucketed = block_bucket_sort(k0, v0, k1, v1, E, sm.sort, sm.scan);
    if (!bucketed && tid == 0 && E > 0) d.g->react_order_radix += 1;
    const int p = bucketed ? 0 : block_sort_pairs(k0, v0, k1, v1, E, sm.sort);
    okeys = p ? k1 : k0;
    order = p ? v1 : v0;
    order_out = d.ev_v0;
    pref = d.ev_k1;
    if (tid == 0) d.g->ev_parity = 0u;
  } else {
    const int p = block_sort_pairs(d.ev_k0, d.ev_v0, d.ev_k1, d.ev_v1, E, sm.sort);
    okeys = p ? d.ev_k1 : d.ev_k0;
    order = p ? d.ev_v1 : d.ev_v0;
    pref = p ? d.ev_k0 : d.ev_k1;
    if (tid == 0) d.g->ev_parity = static_cast<uint32_t>(p);
  }
  products_prefix(d, sm.scan, okeys, order, order_out, pref, E, ok);
}

template <bool F32L>
__device__ void phase_products(const Dev& d, ProductsSmem& sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const Tables& tb = *d.tables;
  for (uint32_t b = tid; b < d.n_trains; b += nt) {
    sm.dwater[b] = 0;
    for (int q = 0; q < MAXT; ++q) sm.dcount[b][q] = 0;
    for (int q = 0; q < MAXR; ++q) sm.devents[b][q] = 0;
  }
  const bool ok = block_status_ok(d);
  const uint32_t E = ok ? d.g->n_events : 0u;
  const uint32_t* order = d.g->ev_parity ? d.ev_v1 : d.ev_v0;
  const uint32_t* pref = d.g->ev_parity ? d.ev_k0 : d.ev_k1;
  const uint32_t n_live = d.g->n_total - d.g->n_dead;
  for (uint32_t k = blockIdx.x * nt + tid; k < E; k += gridDim.x * nt) {
    const Cand cd = d.cand[order[k] & EV_CAND_MASK];
    const uint32_t r = cd.rxn_train & 255u, b = cd.rxn_train >> 8;
    const uint32_t np = static_cast<uint32_t>(tb.n_prod[r]);
    Train& tr = d.trains[b];
    const uint32_t ex = pref[k];
    const uint32_t id0 = tr.next_id + (ex - tr.pref0);
    const uint32_t slot0 = n_live + ex;
    if (slot0 + np > d.cap) {
      raise_status(d.g, CHEM_ECAPACITY);
      continue;
    }
    const uint32_t tlo = tid_type(F32L ? __float_as_uint(d.s4[cd.s_lo].w) : d.stid[cd.s_lo]);
    const uint32_t thi = tid_type(F32L ? __float_as_uint(d.s4[cd.s_hi].w) : d.stid[cd.s_hi]);
    if (F32L) {
      const float4 a = d.s4[cd.s_lo], c = d.s4[cd.s_hi];
      const uint32_t ca = d.cell_sorted[cd.s_lo], cc = d.cell_sorted[cd.s_hi];
      const int n = tr.n;
      int ax_, ay_, az_, cx_, cy_, cz_;
      cell_decode(ca - tr.cell_base, tr.cb, ax_, ay_, az_);
      cell_decode(cc - tr.cell_base, tr.cb, cx_, cy_, cz_);
      int dx = cx_ - ax_, dy = cy_ - ay_, dz = cz_ - az_;
      // the cells of a reacting pair are at most one apart per axis (n >= 3)
      dx = dx > 1 ? dx - n : (dx < -1 ? dx + n : dx);
      dy = dy > 1 ? dy - n : (dy < -1 ? dy + n : dy);
      dz = dz > 1 ? dz - n : (dz < -1 ? dz + n : dz);
      const float w = tb.Df[tlo] / (tb.Df[tlo] + tb.Df[thi]);
      const float px = a.x + w * (dx * tr.hf + (c.x - a.x));
      const float py = a.y + w * (dy * tr.hf + (c.y - a.y));
      const float pz = a.z + w * (dz * tr.hf + (c.z - a.z));
      for (uint32_t q = 0; q < np; ++q) {
        const uint32_t pt = static_cast<uint32_t>(tb.prod[r][q]);
        d.s4[slot0 + q] = make_float4(px, py, pz, __uint_as_float(((id0 + q) << 3) | pt));
        d.cell_sorted[slot0 + q] = ca;
        d.dead[slot0 + q] = 0;
      }
    } else {
      const double xa = d.sx[cd.s_lo], ya = d.sy[cd.s_lo], za = d.sz[cd.s_lo];
      const double rx = min_image(__dsub_rn(d.sx[cd.s_hi], xa), tr.L, tr.halfL);
      const double ry = min_image(__dsub_rn(d.sy[cd.s_hi], ya), tr.L, tr.halfL);
      const double rz = min_image(__dsub_rn(d.sz[cd.s_hi], za), tr.L, tr.halfL);
      const double w = __ddiv_rn(tb.D[tlo], __dadd_rn(tb.D[tlo], tb.D[thi]));
      const double px = wrap_box(__dadd_rn(xa, __dmul_rn(w, rx)), tr.L, tr.halfL);
      const double py = wrap_box(__dadd_rn(ya, __dmul_rn(w, ry)), tr.L, tr.halfL);
      const double pz = wrap_box(__dadd_rn(za, __dmul_rn(w, rz)), tr.L, tr.halfL);
      for (uint32_t q = 0; q < np; ++q) {
        const uint32_t pt = static_cast<uint32_t>(tb.prod[r][q]);
        d.sx[slot0 + q] = px; d.sy[slot0 + q] = py; d.sz[slot0 + q] = pz;
        d.stid[slot0 + q] = ((id0 + q) << 3) | pt;
        d.cell_sorted[slot0 + q] = tr.cell_base;
        d.dead[slot0 + q] = 0;
      }
    }
    atomicSub(&sm.dcount[b][tlo], 1);
    atomicSub(&sm.dcount[b][thi], 1);
    for (uint32_t q = 0; q < np; ++q) atomicAdd(&sm.dcount[b][tb.prod[r][q]], 1);
    atomicAdd(&sm.devents[b][r], 1);
    if (tb.water[r]) atomicAdd(&sm.dwater[b], tb.water[r]);
    if (d.cap_ev_log) {
      const uint32_t e = d.g->ev_log_n + k;
      if (e < d.cap_ev_log) {
        chem_event ev;
        ev.step = tr.step; ev.rxn = static_cast<int32_t>(r); ev.id_lo = cd.id_lo; ev.id_hi = cd.id_hi;
        ev.prod_id0 = id0; ev.n_prod = static_cast<int32_t>(np); ev.train = b; ev.reserved = 0;
        d.ev_log[e] = ev;
      } else {
        raise_status(d.g, CHEM_ECAPACITY);
      }
    }
  }
  __syncthreads();
  for (uint32_t b = 0; b < d.n_trains; ++b) {
    Train& tr = d.trains[b];
    for (int q = tid; q < MAXT + MAXR + 1; q += nt) {
      if (q < MAXT) {
        const int v = sm.dcount[b][q];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&tr.counts[q]),
                         static_cast<unsigned long long>(static_cast<long long>(v)));
      } else if (q < MAXT + MAXR) {
        const int v = sm.devents[b][q - MAXT];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&tr.events[q - MAXT]),
                         static_cast<unsigned long long>(static_cast<long long>(v)));
      } else {
        const int v = sm.dwater[b];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&tr.water),
                         static_cast<unsigned long long>(static_cast<long long>(v)));
      }
    }
  }
}

static __device__ void phase_end_step(const Dev& d, EndSmem& sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) sm.any = 0;
  const bool ok = block_status_ok(d);
  const Tables& tb = *d.tables;
  for (uint32_t b = tid; b < d.n_trains; b += nt) {
    Train& tr = d.trains[b];
    if (tr.active && ok) {
      tr.next_id += tr.prods_step;
      tr.species_steps += tr.n_live_step;
      if (d.cap_step_log) {
        const uint32_t e = atomicAdd(&d.g->step_log_n, 1u);
        if (e < d.cap_step_log) {
          chem_step_record rec;
          rec.step = tr.step; rec.train = b; rec.t_start_s = tr.t_start; rec.dt_s = tr.dt;
          rec.n_live = tr.n_live_step; rec.n_events = tr.n_events_step;
          for (int q = 0; q < 8; ++q) rec.counts[q] = q < tb.n_types ? tr.counts[q] : 0;
          d.step_log[e] = rec;
        } else {
          raise_status(d.g, CHEM_ECAPACITY);
        }
      }
      tr.t = tr.t_next;
      tr.step += 1;
      tr.dt_cur = fmin(__dmul_rn(tr.dt_cur, tr.dt_growth), tr.dt_max);
      tr.n_ref = tr.n;
      tr.h_ref = tr.h;
      tr.cb_ref = tr.cb;
    }
    if (tr.t < tr.t_end) atomicOr(&sm.any, 1u);
  }
  __syncthreads();
  if (tid == 0) {
    bool stepped = false;
    for (uint32_t b = 0; b < d.n_trains; ++b) stepped |= d.trains[b].active != 0;
    if (ok && stepped) d.g->steps_active += 1;
    if (ok) {
      const uint32_t n_live = d.g->n_total - d.g->n_dead;
      d.g->n_total = n_live + d.g->n_products;
      if (d.cap_ev_log) d.g->ev_log_n += d.g->n_events;
    }
    d.g->any_active = sm.any;
  }
  __syncthreads();
}

}  // namespace chem
