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
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  g0 = r * c;
  g1 = r * s;
  g2 = sqrtf(-2.0f * logf(u3)) * cospif(2.0f * u4);
}

// Uniform in [0, 1) for the pair (id_lo, id_hi) at `step` (counter tag 2).
__device__ __forceinline__ double pair_uniform(uint32_t id_lo, uint32_t id_hi, uint32_t step,
                                               uint32_t k0, uint32_t k1) {
  const uint4 c = philox4x32_10(make_uint4(id_lo, step, id_hi, 2u), k0, k1);
  return __dmul_rn(static_cast<double>(u53(c.x, c.y)), TWO_POW_M53);
}

// Brownian-bridge encounter probability (p = 1 when either end is inside R).
__device__ __forceinline__ double bridge_p(double d0, double d1, double R, double DABdt) {
  if (d1 <= R || d0 <= R) return 1.0;
  return exp(__ddiv_rn(-__dmul_rn(__dsub_rn(d0, R), __dsub_rn(d1, R)), DABdt));
}

__device__ __forceinline__ int cell_index(double x, double halfL, double inv_h, int n) {
  int i = static_cast<int>(floor(__dmul_rn(__dadd_rn(x, halfL), inv_h)));
  return min(max(i, 0), n - 1);
}

__device__ __forceinline__ int wrap_cell(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// ======================================================================== begin
// One CTA. Per train: release count, clock step, free-jump decision, hash grid and
// cutoffs of this step; then the slot offsets of the releases and the step counters.
struct BeginSmem {
  uint32_t rel[MAX_TRAINS];
  uint32_t any;
};

static __device__ void phase_begin(const Dev& d, BeginSmem& sb) {
  uint32_t* s_rel = sb.rel;
  uint32_t& s_any = sb.any;
  const int st = status_of(d);
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  const Tables& tb = *d.tables;
  for (uint32_t b = threadIdx.x; b < d.n_trains; b += blockDim.x) {
    Train& tr = d.trains[b];
    const bool act = (st == 0) && (tr.t < tr.t_end);
    uint32_t rel = 0;
    int free_jump = 0;
    if (act) {
      // pending arrivals are sorted; release those with arrival <= t
      uint32_t lo = tr.p_head, hi = tr.p_tail;
      const double* pt = d.pt + tr.pend_base;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pt[mid] <= tr.t) lo = mid + 1; else hi = mid;
      }
      rel = lo - tr.p_head;
      if (rel > 0) {
        tr.t_last_release = tr.t;
        if (tr.reset_on_release) tr.dt_cur = tr.dt_min;
      }
      const double next_arr = (lo < tr.p_tail) ? pt[lo] : CUDART_INF;
      double dt, t_next;
      if (tr.horizon > 0.0 && __dsub_rn(tr.t, tr.t_last_release) >= tr.horizon && next_arr > tr.t) {
        free_jump = 1;
        t_next = fmin(tr.t_end, next_arr);
        dt = __dsub_rn(t_next, tr.t);
      } else {
        dt = fmin(tr.dt_cur, tr.dt_L);
        if (__dsub_rn(tr.t_end, tr.t) <= __dmul_rn(dt, END_SLACK)) {
          dt = __dsub_rn(tr.t_end, tr.t);
          t_next = tr.t_end;
        } else {
          t_next = __dadd_rn(tr.t, dt);
        }
      }
      tr.dt = dt;
      tr.t_next = t_next;
      tr.t_start = tr.t;
      // cutoffs R + c sqrt(2 D_AB dt) and the hash grid (cell >= largest cutoff)
      double rcmax = 0.0;
      for (int r = 0; r < tb.n_rxn; ++r) {
        const double rc = __dadd_rn(tb.R[r], __dmul_rn(tr.c, sqrt(__dmul_rn(__dmul_rn(2.0, tb.D_AB[r]), dt))));
        tr.rc2[r] = __dmul_rn(rc, rc);
        tr.rc2f[r] = static_cast<float>(tr.rc2[r]);
        tr.ddt[r] = __dmul_rn(tb.D_AB[r], dt);
        tr.inv_ddt_f[r] = static_cast<float>(__ddiv_rn(1.0, tr.ddt[r]));
        rcmax = fmax(rcmax, rc);
      }
      for (int ty = 0; ty < tb.n_types; ++ty) {
        tr.sig[ty] = sqrt(__dmul_rn(__dmul_rn(2.0, tb.D[ty]), dt));
        tr.sigf[ty] = static_cast<float>(tr.sig[ty]);
      }
      int n = tr.n_max;
      if (free_jump) {
        n = tr.n_ref;  // no pair search: keep the hash grid
      } else if (rcmax > 0.0) {
        const double nf = floor(__ddiv_rn(tr.L, __dmul_rn(rcmax, CELL_SLACK)));
        n = static_cast<int>(fmin(nf, static_cast<double>(tr.n_max)));
        n = max(n, 3);
      }
      tr.n = n;
      tr.h = __ddiv_rn(tr.L, static_cast<double>(n));
      tr.inv_h = __ddiv_rn(static_cast<double>(n), tr.L);
      tr.hf = static_cast<float>(tr.h);
      tr.inv_hf = static_cast<float>(tr.inv_h);
      tr.rel_n = rel;
      tr.rel_id0 = tr.next_id;
      tr.rel_p0 = tr.p_head;
      tr.p_head += rel;
      tr.next_id += rel;
      long long live = rel;
      for (int ty = 0; ty < tb.n_types; ++ty) live += tr.counts[ty];
      tr.n_live_step = live;
      tr.n_events_step = 0;
      if (tr.next_id > tr.id_limit) raise_status(d.g, CHEM_ECAPACITY);
      atomicOr(&s_any, 1u);
    } else {
      tr.rel_n = 0;
    }
    tr.active = act ? 1 : 0;
    tr.free_jump = free_jump;
    s_rel[b] = rel;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Global* g = d.g;
    uint32_t off = g->n_total;
    const uint32_t before = off;
    unsigned long long total = off;
    for (uint32_t b = 0; b < d.n_trains; ++b) {
      d.trains[b].rel_off = off;
      total += s_rel[b];
      off += s_rel[b];
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
    g->n_items = 0;
    g->n_events = 0;
    g->n_products = 0;
    g->n_dead = 0;
    g->epoch += 1;
    g->any_active = s_any;
  }
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) {
    (&d.g->hist[0][0])[i] = 0u;
    (&d.g->ev_hist[0][0])[i] = 0u;
  }
  if (threadIdx.x < MAX_PASSES) d.g->ev_tile_ctr[threadIdx.x] = 0u;
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
template <bool F32L>
__device__ void phase_release(const Dev& d) {
  if (status_of(d)) return;
  const uint32_t n_rel = d.g->n_released;
  const uint32_t base = d.g->n_total - n_rel;
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t n_iter = (n_rel + stride - 1) / stride;
  for (uint32_t it = 0; it < n_iter; ++it) {
    const uint32_t i = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n_rel;
    uint32_t b = 0, type = 0;
    if (valid) {
      const uint32_t slot = base + i;
      b = train_of_release(d, slot);
      const Train& tr = d.trains[b];
      const uint32_t k = slot - tr.rel_off;
      const uint32_t p = tr.pend_base + tr.rel_p0 + k;
      type = static_cast<uint32_t>(d.p_type[p]);
      const uint32_t id = tr.rel_id0 + k;
      const uint32_t tid = (id << 3) | type;
      const double x = d.px[p], y = d.py[p], z = d.pz[p];
      if (F32L) {
        const int n = tr.n_ref;
        const double h = tr.h_ref, inv_h = __ddiv_rn(1.0, h);
        const int ix = cell_index(x, tr.halfL, inv_h, n);
        const int iy = cell_index(y, tr.halfL, inv_h, n);
        const int iz = cell_index(z, tr.halfL, inv_h, n);
        const float ox = static_cast<float>(__dsub_rn(__dadd_rn(x, tr.halfL), __dmul_rn(ix, h)));
        const float oy = static_cast<float>(__dsub_rn(__dadd_rn(y, tr.halfL), __dmul_rn(iy, h)));
        const float oz = static_cast<float>(__dsub_rn(__dadd_rn(z, tr.halfL), __dmul_rn(iz, h)));
        d.s4[slot] = make_float4(ox, oy, oz, __uint_as_float(tid));
        d.cell_sorted[slot] = tr.cell_base + static_cast<uint32_t>((iz * n + iy) * n + ix);
      } else {
        d.sx[slot] = x;
        d.sy[slot] = y;
        d.sz[slot] = z;
        d.stid[slot] = tid;
        d.cell_sorted[slot] = tr.cell_base;  // FP64 mode recomputes cells from positions
      }
      d.dead[slot] = 0;
    }
    count_add(d, b, type, 1, valid);
  }
}

// ======================================================================== diffuse
// Displace every species of an active train (Sec. 2.1 SBS step) with periodic wrap
// (Eq. 1), compute its hash key, and accumulate the radix histograms of every pass.
// Species marked dead by the last step's reactions get the sentinel key.
template <bool F32L>
__device__ void phase_diffuse(const Dev& d, uint32_t (*hist)[RADIX]) {
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&hist[0][0])[i] = 0u;
  __syncthreads();
  const bool ok = status_of(d) == 0;
  const uint32_t n_total = d.g->n_total;
  const uint32_t stride = gridDim.x * blockDim.x;
  const Tables& tb = *d.tables;
  uint32_t n_dead_local = 0;
  if (ok) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_total; s += stride) {
      uint32_t key;
      if (d.dead[s]) {
        d.dead[s] = 0;
        key = d.sentinel;
        ++n_dead_local;
      } else {
        const uint32_t cell = d.cell_sorted[s];
        const int b = (d.n_trains == 1) ? 0 : train_of_cell(d.trains, d.n_trains, cell);
        const Train& tr = d.trains[b];
        if (!tr.active) {
          if (F32L) d.t4[s] = d.s4[s];
          else { d.tx[s] = d.sx[s]; d.ty[s] = d.sy[s]; d.tz[s] = d.sz[s]; d.ttid[s] = d.stid[s]; }
          key = cell;
        } else if (!F32L) {
          const uint32_t tid = d.stid[s];
          const uint32_t ty = tid_type(tid);
          double g0, g1, g2;
          gauss3_f64(tid_id(tid), tr.step, tr.key0, tr.key1, g0, g1, g2);
          const double sig = tr.sig[ty];
          const double ex = __dmul_rn(sig, g0), ey = __dmul_rn(sig, g1), ez = __dmul_rn(sig, g2);
          const double x = wrap_box(__dadd_rn(d.sx[s], ex), tr.L, tr.halfL);
          const double y = wrap_box(__dadd_rn(d.sy[s], ey), tr.L, tr.halfL);
          const double z = wrap_box(__dadd_rn(d.sz[s], ez), tr.L, tr.halfL);
          d.tx[s] = x; d.ty[s] = y; d.tz[s] = z; d.ttid[s] = tid;
          d.tdx[s] = ex; d.tdy[s] = ey; d.tdz[s] = ez;
          const int n = tr.n;
          const int ix = cell_index(x, tr.halfL, tr.inv_h, n);
          const int iy = cell_index(y, tr.halfL, tr.inv_h, n);
          const int iz = cell_index(z, tr.halfL, tr.inv_h, n);
          key = tr.cell_base + static_cast<uint32_t>((iz * n + iy) * n + ix);
        } else {
          const float4 v = d.s4[s];
          const uint32_t tid = __float_as_uint(v.w);
          const uint32_t ty = tid_type(tid);
          float g0, g1, g2;
          gauss3_f32(tid_id(tid), tr.step, tr.key0, tr.key1, g0, g1, g2);
          const float sig = tr.sigf[ty];
          const int nr = tr.n_ref;
          const uint32_t loc = cell - tr.cell_base;
          int ix = static_cast<int>(loc % nr), iy = static_cast<int>((loc / nr) % nr),
              iz = static_cast<int>(loc / (static_cast<uint32_t>(nr) * nr));
          const int n = tr.n;
          const float ex = sig * g0, ey = sig * g1, ez = sig * g2;
          d.td4[s] = make_float4(ex, ey, ez, 0.f);
          float ox, oy, oz;
          if (nr == n) {
            ox = v.x + ex; oy = v.y + ey; oz = v.z + ez;
            const float fx = floorf(ox * tr.inv_hf), fy = floorf(oy * tr.inv_hf), fz = floorf(oz * tr.inv_hf);
            ox -= fx * tr.hf; oy -= fy * tr.hf; oz -= fz * tr.hf;
            ix = wrap_cell(ix + static_cast<int>(fx), n);
            iy = wrap_cell(iy + static_cast<int>(fy), n);
            iz = wrap_cell(iz + static_cast<int>(fz), n);
          } else {
            // the hash grid changed this step: go through FP64 absolute positions
            const double hr = tr.h_ref;
            double ax = wrap_box((ix * hr - tr.halfL) + v.x + static_cast<double>(ex), tr.L, tr.halfL);
            double ay = wrap_box((iy * hr - tr.halfL) + v.y + static_cast<double>(ey), tr.L, tr.halfL);
            double az = wrap_box((iz * hr - tr.halfL) + v.z + static_cast<double>(ez), tr.L, tr.halfL);
            ix = cell_index(ax, tr.halfL, tr.inv_h, n);
            iy = cell_index(ay, tr.halfL, tr.inv_h, n);
            iz = cell_index(az, tr.halfL, tr.inv_h, n);
            ox = static_cast<float>((ax + tr.halfL) - ix * tr.h);
            oy = static_cast<float>((ay + tr.halfL) - iy * tr.h);
            oz = static_cast<float>((az + tr.halfL) - iz * tr.h);
          }
          d.t4[s] = make_float4(ox, oy, oz, v.w);
          key = tr.cell_base + static_cast<uint32_t>((iz * n + iy) * n + ix);
        }
      }
      d.keys0[s] = key;
      d.vals0[s] = s;
      for (int p = 0; p < d.passes; ++p) atomicAdd(&hist[p][(key >> (8 * p)) & 255u], 1u);
    }
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
static __device__ void phase_sort_pass(const Dev& d, int pass, SortSmem& sm) {
  if (status_of(d)) return;
  const uint32_t* kin = (pass & 1) ? d.keys1 : d.keys0;
  const uint32_t* vin = (pass & 1) ? d.vals1 : d.vals0;
  uint32_t* kout = (pass & 1) ? d.keys0 : d.keys1;
  uint32_t* vout = (pass & 1) ? d.vals0 : d.vals1;
  onesweep_pass(kin, vin, kout, vout, d.g->n_total, 8 * pass, d.g->hist[pass], &d.g->tile_ctr[pass],
                d.lookback, d.g->epoch * 2 * MAX_PASSES + pass, d.g, sm);
}

// ======================================================================== gather
// Reorder the diffused species into cell order, record each cell's slot range (stamped
// with this step's epoch) and drop the dead (sentinel keys sort last).
template <bool F32L>
__device__ void phase_gather(const Dev& d) {
  if (status_of(d)) return;
  const uint32_t* kf = (d.passes & 1) ? d.keys1 : d.keys0;
  const uint32_t* vf = (d.passes & 1) ? d.vals1 : d.vals0;
  const uint32_t n_live = d.g->n_total - d.g->n_dead;
  const uint32_t epoch = d.g->epoch;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_live; s += stride) {
    const uint32_t key = kf[s];
    const uint32_t i = vf[s];
    if (key >= d.sentinel || i >= d.g->n_total) {  // only after a timed-out sort
      raise_status(d.g, CHEM_ETIMEOUT);
      continue;
    }
    if (F32L) {
      d.s4[s] = d.t4[i];
    } else {
      d.sx[s] = d.tx[i]; d.sy[s] = d.ty[i]; d.sz[s] = d.tz[i]; d.stid[s] = d.ttid[i];
    }
    d.cell_sorted[s] = key;
    int* ci = reinterpret_cast<int*>(&d.cell_info[key]);
    const bool first = (s == 0 || kf[s - 1] != key);
    if (first) { ci[0] = static_cast<int>(s); ci[2] = static_cast<int>(epoch); }
    if (s + 1 == n_live || kf[s + 1] != key) ci[1] = static_cast<int>(s + 1);
    // pair-search work item: a cell's first slot and every ITEM_HOME-th slot
    if (first || (s % ITEM_HOME) == 0) {
      const int b = (d.n_trains == 1) ? 0 : train_of_cell(d.trains, d.n_trains, key);
      if (d.trains[b].active && !d.trains[b].free_jump) {
        const uint32_t it = atomicAdd(&d.g->n_items, 1u);
        if (it < d.cap_items) d.items[it] = s;
        else raise_status(d.g, CHEM_ECAPACITY);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) d.g->n_live = n_live;
}

// ======================================================================== search
// For every unordered pair of live species whose types react (Table 1), separated by
// less than the reaction's cutoff under the minimum image (Eq. 2), evaluate the
// encounter probability and keep the pair if its uniform falls below it.
//
// One warp per work item: up to ITEM_HOME home species of one cell, staged in shared
// memory. The own cell (slots after the item's first slot) and the 13 forward cells of
// the half shell are flattened into one neighbour list; lanes stride over it (coalesced
// loads) and each lane tests its neighbour against every home species (shared-memory
// broadcast). With at least 3 cells per axis each unordered pair is visited once.

// Half-shell offsets: 0 = own cell, 1..9 dz = +1, 10..12 (dz, dy) = (0, +1), 13 (0, 0, +1).
__device__ __forceinline__ void fwd_offset(int k, int& dx, int& dy, int& dz) {
  if (k == 0) { dx = dy = dz = 0; return; }
  if (k <= 9) { const int q = k - 1; dz = 1; dy = q / 3 - 1; dx = q % 3 - 1; return; }
  if (k <= 12) { dz = 0; dy = 1; dx = k - 11; return; }
  dz = 0; dy = 0; dx = 1;
}

template <bool F32L>
struct SearchWarpSmem;

template <>
struct SearchWarpSmem<true> {
  float4 pos[ITEM_HOME];   // offsets + tid bits
  float4 dl[ITEM_HOME];    // this step's displacement
};

template <>
struct SearchWarpSmem<false> {
  double x[ITEM_HOME], y[ITEM_HOME], z[ITEM_HOME];
  double ex[ITEM_HOME], ey[ITEM_HOME], ez[ITEM_HOME];
  uint32_t tid[ITEM_HOME];
};

template <bool F32L>
struct SearchSmem {
  SearchWarpSmem<F32L> w[8];
};

__device__ __forceinline__ void emit_candidate(const Dev& d, uint32_t s_lo, uint32_t s_hi, uint32_t id_lo,
                                               uint32_t id_hi, int r, int b, double d1sq) {
  const uint32_t c = atomicAdd(&d.g->n_cand, 1u);
  if (c >= d.cap_cand) { raise_status(d.g, CHEM_ECAPACITY); return; }
  Cand cd;
  cd.s_lo = s_lo; cd.s_hi = s_hi; cd.id_lo = id_lo; cd.id_hi = id_hi;
  cd.rxn_train = static_cast<uint32_t>(r) | (static_cast<uint32_t>(b) << 8);
  cd.pad = 0;
  cd.d1sq = d1sq;
  d.cand[c] = cd;
}

// Accept iff u < p with p evaluated in FP64 from the FP32 squared distances:
// p = 1 when d0 <= R or d1 <= R, else exp(-(d0 - R)(d1 - R) / (D_AB dt)). An FP32
// estimate decides whenever it lies farther from u than twice its error bound (FP32
// rounding of d0, d1, R and of the products, cancellation in d - R, and __expf);
// otherwise the FP64 value decides, so the outcome is always that of the FP64 test.
__device__ __forceinline__ bool accept_f32(float d0sq, float d1sq, int r, const Tables& tb, const Train& tr,
                                          uint32_t id_lo, uint32_t id_hi) {
  const float d1f = sqrtf(d1sq), d0f = sqrtf(d0sq);
  const float Rf = tb.Rf[r];
  const double u = pair_uniform(id_lo, id_hi, tr.step, tr.key0, tr.key1);
  if (d1f < Rf * 0.999f || d0f < Rf * 0.999f) return true;  // p = 1 > u
  if (d1f > Rf * 1.001f && d0f > Rf * 1.001f) {
    const float a = d0f - Rf, b = d1f - Rf, inv = tr.inv_ddt_f[r];
    const float x = a * b * inv;
    if (x > 60.f) {
      if (u != 0.0) return false;  // p < 1e-26 < 2^-53 <= u
    } else {
      const float p = __expf(-x);
      const float err = 1.2e-7f * inv * (b * (d0f + Rf) + a * (d1f + Rf)) + 1e-6f * (1.f + x);
      const double band = 2.0 * static_cast<double>(err) * p + 1e-300;
      if (u > static_cast<double>(p) + band) return false;
      if (u < static_cast<double>(p) - band) return true;
    }
  }
  const double d0 = sqrt(static_cast<double>(d0sq)), d1 = sqrt(static_cast<double>(d1sq));
  return u < bridge_p(d0, d1, tb.R[r], tr.ddt[r]);
}

template <bool F32L>
__device__ void phase_search(const Dev& d, SearchSmem<F32L>& sm) {
  if (status_of(d)) return;
  const uint32_t n_items = min(d.g->n_items, d.cap_items);
  const uint32_t epoch = d.g->epoch;
  const uint32_t* vf = (d.passes & 1) ? d.vals1 : d.vals0;
  const Tables& tb = *d.tables;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t warps_total = gridDim.x * (blockDim.x >> 5);
  SearchWarpSmem<F32L>& hs = sm.w[wib];
  for (uint32_t it = blockIdx.x * (blockDim.x >> 5) + wib; it < n_items; it += warps_total) {
    const uint32_t s0 = d.items[it];
    const uint32_t cell = d.cell_sorted[s0];
    const int b = (d.n_trains == 1) ? 0 : train_of_cell(d.trains, d.n_trains, cell);
    const Train& tr = d.trains[b];
    const int4 ci = d.cell_info[cell];
    const uint32_t s_end = min(static_cast<uint32_t>(ci.y), (s0 / ITEM_HOME + 1) * ITEM_HOME);
    const uint32_t nh = s_end - s0;
    // stage the home species; OR of the types they react with
    uint32_t want = 0;
    for (uint32_t h = lane; h < nh; h += 32) {
      const uint32_t s = s0 + h;
      const uint32_t ti = vf[s];
      uint32_t t;
      if (F32L) {
        const float4 v = d.s4[s];
        reinterpret_cast<SearchWarpSmem<true>&>(hs).pos[h] = v;
        reinterpret_cast<SearchWarpSmem<true>&>(hs).dl[h] = d.td4[ti];
        t = __float_as_uint(v.w);
      } else {
        auto& hd = reinterpret_cast<SearchWarpSmem<false>&>(hs);
        hd.x[h] = d.sx[s]; hd.y[h] = d.sy[s]; hd.z[h] = d.sz[s];
        hd.ex[h] = d.tdx[ti]; hd.ey[h] = d.tdy[ti]; hd.ez[h] = d.tdz[ti];
        t = d.stid[s];
        hd.tid[h] = t;
      }
      want |= tb.reactive_mask[tid_type(t)];
    }
    want = __reduce_or_sync(0xffffffffu, want);
    __syncwarp();
    if (!want) continue;
    // neighbour ranges of the half shell
    const int n = tr.n;
    const uint32_t loc = cell - tr.cell_base;
    const int ix = static_cast<int>(loc % n), iy = static_cast<int>((loc / n) % n),
              iz = static_cast<int>(loc / (static_cast<uint32_t>(n) * n));
    uint32_t rs = 0, rl = 0;
    if (lane < N_FWD) {
      if (lane == 0) {
        rs = s0 + 1;
        rl = static_cast<uint32_t>(ci.y) - rs;
      } else {
        int ox, oy, oz;
        fwd_offset(lane, ox, oy, oz);
        const uint32_t nc = tr.cell_base + static_cast<uint32_t>(
            (wrap_cell(iz + oz, n) * n + wrap_cell(iy + oy, n)) * n + wrap_cell(ix + ox, n));
        const int4 nci = d.cell_info[nc];
        if (static_cast<uint32_t>(nci.z) == epoch) {
          rs = static_cast<uint32_t>(nci.x);
          rl = static_cast<uint32_t>(nci.y - nci.x);
        }
      }
    }
    uint32_t incl = rl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - rl;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, N_FWD - 1);
    uint32_t ex_k[N_FWD];
#pragma unroll
    for (int q = 0; q < N_FWD; ++q) ex_k[q] = __shfl_sync(0xffffffffu, excl, q);
    for (uint32_t f0 = 0; f0 < total; f0 += 32) {
      const uint32_t f = f0 + lane;
      const bool valid = f < total;
      int k = 0;
#pragma unroll
      for (int q = 1; q < N_FWD; ++q) k += (ex_k[q] <= f) ? 1 : 0;
      const uint32_t j_start = __shfl_sync(0xffffffffu, rs, k);
      const uint32_t j_off = __shfl_sync(0xffffffffu, excl, k);
      if (!valid) continue;
      const uint32_t j = j_start + (f - j_off);
      int odx, ody, odz;
      fwd_offset(k, odx, ody, odz);
      uint32_t tid_j;
      float4 vj = make_float4(0.f, 0.f, 0.f, 0.f);
      double xj = 0, yj = 0, zj = 0;
      if (F32L) { vj = d.s4[j]; tid_j = __float_as_uint(vj.w); }
      else { tid_j = d.stid[j]; }
      const uint32_t tj = tid_type(tid_j);
      if (!((want >> tj) & 1u)) continue;
      if (!F32L) { xj = d.sx[j]; yj = d.sy[j]; zj = d.sz[j]; }
      const uint32_t id_j = tid_id(tid_j);
      const uint32_t jmask = tb.reactive_mask[tj];
      const float cx = odx * tr.hf, cy = ody * tr.hf, cz = odz * tr.hf;
      for (uint32_t h = 0; h < nh; ++h) {
        if (k == 0 && j <= s0 + h) break;  // own cell: only later slots (slots ascend with h)
        uint32_t tid_i;
        if (F32L) tid_i = __float_as_uint(reinterpret_cast<SearchWarpSmem<true>&>(hs).pos[h].w);
        else tid_i = reinterpret_cast<SearchWarpSmem<false>&>(hs).tid[h];
        const uint32_t ti = tid_type(tid_i);
        if (!((jmask >> ti) & 1u)) continue;
        const int r = tb.pair_rxn[ti][tj];
        const uint32_t id_i = tid_id(tid_i);
        const bool i_lo = id_i < id_j;
        if (F32L) {
          const SearchWarpSmem<true>& hf = reinterpret_cast<const SearchWarpSmem<true>&>(hs);
          const float4 vi = hf.pos[h];
          float fx = cx + (vj.x - vi.x), fy = cy + (vj.y - vi.y), fz = cz + (vj.z - vi.z);
          const float f2 = fx * fx + fy * fy + fz * fz;
          if (!(f2 < tr.rc2f[r])) continue;
          if (!i_lo) { fx = -fx; fy = -fy; fz = -fz; }
          const float4 di = hf.dl[h];
          const float4 dj = d.td4[vf[j]];
          const float4 dlo = i_lo ? di : dj, dhi = i_lo ? dj : di;
          const float r0x = fx - (dhi.x - dlo.x), r0y = fy - (dhi.y - dlo.y), r0z = fz - (dhi.z - dlo.z);
          const float d0sq = r0x * r0x + r0y * r0y + r0z * r0z;
          const uint32_t id_lo = i_lo ? id_i : id_j, id_hi = i_lo ? id_j : id_i;
          if (!accept_f32(d0sq, f2, r, tb, tr, id_lo, id_hi)) continue;
          const uint32_t si = s0 + h;
          emit_candidate(d, i_lo ? si : j, i_lo ? j : si, id_lo, id_hi, r, b, static_cast<double>(f2));
        } else {
          const SearchWarpSmem<false>& hd = reinterpret_cast<const SearchWarpSmem<false>&>(hs);
          const double xi = hd.x[h], yi = hd.y[h], zi = hd.z[h];
          double rx1, ry1, rz1;
          if (i_lo) {
            rx1 = min_image(__dsub_rn(xj, xi), tr.L, tr.halfL);
            ry1 = min_image(__dsub_rn(yj, yi), tr.L, tr.halfL);
            rz1 = min_image(__dsub_rn(zj, zi), tr.L, tr.halfL);
          } else {
            rx1 = min_image(__dsub_rn(xi, xj), tr.L, tr.halfL);
            ry1 = min_image(__dsub_rn(yi, yj), tr.L, tr.halfL);
            rz1 = min_image(__dsub_rn(zi, zj), tr.L, tr.halfL);
          }
          const double d1sq = sq3(rx1, ry1, rz1);
          if (!(d1sq < tr.rc2[r])) continue;
          const uint32_t tj_idx = vf[j];
          const double ejx = d.tdx[tj_idx], ejy = d.tdy[tj_idx], ejz = d.tdz[tj_idx];
          const double elx = i_lo ? hd.ex[h] : ejx, ely = i_lo ? hd.ey[h] : ejy, elz = i_lo ? hd.ez[h] : ejz;
          const double ehx = i_lo ? ejx : hd.ex[h], ehy = i_lo ? ejy : hd.ey[h], ehz = i_lo ? ejz : hd.ez[h];
          const double r0x = __dsub_rn(rx1, __dsub_rn(ehx, elx));
          const double r0y = __dsub_rn(ry1, __dsub_rn(ehy, ely));
          const double r0z = __dsub_rn(rz1, __dsub_rn(ehz, elz));
          const double d1 = sqrt(d1sq);
          const double d0 = sqrt(sq3(r0x, r0y, r0z));
          const uint32_t id_lo = i_lo ? id_i : id_j, id_hi = i_lo ? id_j : id_i;
          const double p = bridge_p(d0, d1, tb.R[r], tr.ddt[r]);
          const double u = pair_uniform(id_lo, id_hi, tr.step, tr.key0, tr.key1);
          if (!(u < p)) continue;
          const uint32_t si = s0 + h;
          emit_candidate(d, i_lo ? si : j, i_lo ? j : si, id_lo, id_hi, r, b, d1sq);
        }
      }
    }
    __syncwarp();
  }
}

// ======================================================================== react
// One reaction per species (Sec. 2.3: reactants react on encounter), in three phases:
//  1. phase_match (one CTA): rounds of locally-dominant selection; a pair is committed
//     when it is the smallest (d1^2, id_lo, id_hi) remaining pair of both its species,
//     which equals the greedy walk over pairs sorted by that key (closest first, lower
//     ids first). Emits every event with its key (train, id_lo) and digit histograms.
//  2. the event keys are ordered by the Onesweep passes (all CTAs);
//  3. phase_products (one CTA): product ids in (train, id_lo) order, products at the
//     diffusion-weighted encounter point (Table 1 right-hand sides), tallies summed in
//     shared memory, logs, and the end of the step (FP64 clock, step counter, dt growth).
struct MatchSmem {
  uint32_t n_alive, n_next, n_ev;
  uint32_t hist[MAX_PASSES][RADIX];
};

struct ProductsSmem {
  uint32_t carry, any;
  uint32_t warp_tot[REACT_THREADS / 32];
  uint32_t first_pref[MAX_TRAINS];
  uint32_t prods_tr[MAX_TRAINS];
  uint32_t evs_tr[MAX_TRAINS];
  int dcount[MAX_TRAINS][MAXT];
  int devents[MAX_TRAINS][MAXR];
  int dwater[MAX_TRAINS];
};

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_tot,
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
  uint32_t add = 0, tot = 0;
  for (int i = 0; i < nw; ++i) {
    if (i < w) add += warp_tot[i];
    tot += warp_tot[i];
  }
  __syncthreads();
  total = tot;
  return x - v + add;
}

__device__ __forceinline__ uint32_t event_key(const Dev& d, const Cand& cd) {
  const uint32_t b = cd.rxn_train >> 8;
  return d.train_bits ? ((b << (32 - d.train_bits)) | cd.id_lo) : cd.id_lo;
}

static __device__ void phase_match(const Dev& d, MatchSmem& sm) {
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  const bool ok = status_of(d) == 0;
  unsigned long long* bd = reinterpret_cast<unsigned long long*>(d.keys0);
  unsigned long long* bp = bd + d.cap;
  uint32_t n_c = min(d.g->n_cand, d.cap_cand);
  if (!ok) n_c = 0;
  if (tid == 0) { sm.n_alive = n_c; sm.n_ev = 0; }
  for (int i = tid; i < MAX_PASSES * RADIX; i += nt) (&sm.hist[0][0])[i] = 0u;
  for (uint32_t i = tid; i < n_c; i += nt) d.alive0[i] = i;
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
    for (uint32_t i = tid; i < na; i += nt) {
      const uint32_t c = alive[i];
      const Cand cd = d.cand[c];
      const unsigned long long kd = __double_as_longlong(cd.d1sq);
      const unsigned long long kp = (static_cast<unsigned long long>(cd.id_lo) << 32) | cd.id_hi;
      if (bd[cd.s_lo] == kd && bp[cd.s_lo] == kp && bd[cd.s_hi] == kd && bp[cd.s_hi] == kp) {
        d.dead[cd.s_lo] = 1;
        d.dead[cd.s_hi] = 1;
        const uint32_t e = atomicAdd(&sm.n_ev, 1u);
        const uint32_t key = event_key(d, cd);
        d.ev_k0[e] = key;
        d.ev_v0[e] = c;
#pragma unroll
        for (int p = 0; p < MAX_PASSES; ++p) atomicAdd(&sm.hist[p][(key >> (8 * p)) & 255u], 1u);
      }
    }
    if (tid == 0) sm.n_next = 0;
    __syncthreads();
    for (uint32_t i = tid; i < na; i += nt) {
      const uint32_t c = alive[i];
      const Cand cd = d.cand[c];
      if (!d.dead[cd.s_lo] && !d.dead[cd.s_hi]) nxt[atomicAdd(&sm.n_next, 1u)] = c;
    }
    __syncthreads();
    if (tid == 0) sm.n_alive = sm.n_next;
    uint32_t* tmp = alive; alive = nxt; nxt = tmp;
    __syncthreads();
  }
  for (int i = tid; i < MAX_PASSES * RADIX; i += nt) (&d.g->ev_hist[0][0])[i] = (&sm.hist[0][0])[i];
  if (tid == 0) d.g->n_events = sm.n_ev;
  __syncthreads();
}

// One Onesweep pass over the event keys (ev_k0/ev_v0 -> ev_k1/ev_v1 and back).
static __device__ void phase_event_sort_pass(const Dev& d, int pass, SortSmem& sm) {
  if (status_of(d)) return;
  const uint32_t* kin = (pass & 1) ? d.ev_k1 : d.ev_k0;
  const uint32_t* vin = (pass & 1) ? d.ev_v1 : d.ev_v0;
  uint32_t* kout = (pass & 1) ? d.ev_k0 : d.ev_k1;
  uint32_t* vout = (pass & 1) ? d.ev_v0 : d.ev_v1;
  onesweep_pass(kin, vin, kout, vout, d.g->n_events, 8 * pass, d.g->ev_hist[pass],
                &d.g->ev_tile_ctr[pass], d.lookback, d.g->epoch * 2 * MAX_PASSES + MAX_PASSES + pass,
                d.g, sm);
}

template <bool F32L>
__device__ void phase_products(const Dev& d, ProductsSmem& sm) {
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  const bool ok = status_of(d) == 0;
  const Tables& tb = *d.tables;
  const uint32_t E = ok ? d.g->n_events : 0u;
  const uint32_t* order = d.ev_v0;  // after an even number of passes
  for (uint32_t b = tid; b < d.n_trains; b += nt) {
    sm.first_pref[b] = 0xFFFFFFFFu; sm.prods_tr[b] = 0; sm.evs_tr[b] = 0; sm.dwater[b] = 0;
    for (int q = 0; q < MAXT; ++q) sm.dcount[b][q] = 0;
    for (int q = 0; q < MAXR; ++q) sm.devents[b][q] = 0;
  }
  if (tid == 0) { sm.carry = 0; sm.any = 0; }
  __syncthreads();
  const uint32_t n_live = d.g->n_total - d.g->n_dead;
  for (uint32_t t0 = 0; t0 < E; t0 += nt) {
    const uint32_t k = t0 + tid;
    const bool valid = k < E;
    Cand cd;
    uint32_t r = 0, b = 0, np = 0;
    if (valid) {
      cd = d.cand[order[k]];
      r = cd.rxn_train & 255u;
      b = cd.rxn_train >> 8;
      np = static_cast<uint32_t>(tb.n_prod[r]);
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan(np, sm.warp_tot, tot) + sm.carry;
    if (valid) {
      bool first = (k == 0);
      if (!first) first = ((d.cand[order[k - 1]].rxn_train >> 8) != b);
      if (first) sm.first_pref[b] = ex;
    }
    __syncthreads();
    if (valid) {
      Train& tr = d.trains[b];
      const uint32_t id0 = tr.next_id + (ex - sm.first_pref[b]);
      const uint32_t slot0 = n_live + ex;
      if (slot0 + np > d.cap) {
        raise_status(d.g, CHEM_ECAPACITY);
      } else {
        const uint32_t tlo = tid_type(F32L ? __float_as_uint(d.s4[cd.s_lo].w) : d.stid[cd.s_lo]);
        const uint32_t thi = tid_type(F32L ? __float_as_uint(d.s4[cd.s_hi].w) : d.stid[cd.s_hi]);
        if (F32L) {
          const float4 a = d.s4[cd.s_lo], c = d.s4[cd.s_hi];
          const uint32_t ca = d.cell_sorted[cd.s_lo], cc = d.cell_sorted[cd.s_hi];
          const int n = tr.n;
          const uint32_t la = ca - tr.cell_base, lc = cc - tr.cell_base;
          int dx = static_cast<int>(lc % n) - static_cast<int>(la % n);
          int dy = static_cast<int>((lc / n) % n) - static_cast<int>((la / n) % n);
          int dz = static_cast<int>(lc / (n * n)) - static_cast<int>(la / (n * n));
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
        atomicAdd(&sm.prods_tr[b], np);
        atomicAdd(&sm.evs_tr[b], 1u);
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
    }
    __syncthreads();
    if (tid == 0) sm.carry += tot;
    __syncthreads();
  }
  // end of step
  for (uint32_t b = tid; b < d.n_trains; b += nt) {
    Train& tr = d.trains[b];
    if (tr.active && ok) {
      for (int q = 0; q < tb.n_types; ++q) tr.counts[q] += sm.dcount[b][q];
      for (int q = 0; q < tb.n_rxn; ++q) tr.events[q] += sm.devents[b][q];
      tr.water += sm.dwater[b];
      tr.next_id += sm.prods_tr[b];
      tr.n_events_step = sm.evs_tr[b];
      tr.species_steps += tr.n_live_step;
      if (d.cap_step_log) {
        const uint32_t e = atomicAdd(&d.g->step_log_n, 1u);
        if (e < d.cap_step_log) {
          chem_step_record rec;
          rec.step = tr.step; rec.train = b; rec.t_start_s = tr.t_start; rec.dt_s = tr.dt;
          rec.n_live = tr.n_live_step; rec.n_events = sm.evs_tr[b];
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
    }
    if (tr.t < tr.t_end) atomicOr(&sm.any, 1u);
  }
  __syncthreads();
  if (tid == 0) {
    bool stepped = false;
    for (uint32_t b = 0; b < d.n_trains; ++b) stepped |= d.trains[b].active != 0;
    if (ok && stepped) d.g->steps_active += 1;
    if (ok) {
      d.g->n_products = sm.carry;
      d.g->n_total = n_live + sm.carry;
      if (d.cap_ev_log) d.g->ev_log_n += E;
    }
    d.g->any_active = sm.any;
  }
  __syncthreads();
}

}  // namespace chem
