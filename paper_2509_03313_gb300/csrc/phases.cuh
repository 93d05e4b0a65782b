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
    g->n_events = 0;
    g->n_products = 0;
    g->n_dead = 0;
    g->epoch += 1;
    g->any_active = s_any;
  }
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) (&d.g->hist[0][0])[i] = 0u;
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
          const double x = wrap_box(__dadd_rn(d.sx[s], __dmul_rn(sig, g0)), tr.L, tr.halfL);
          const double y = wrap_box(__dadd_rn(d.sy[s], __dmul_rn(sig, g1)), tr.L, tr.halfL);
          const double z = wrap_box(__dadd_rn(d.sz[s], __dmul_rn(sig, g2)), tr.L, tr.halfL);
          d.tx[s] = x; d.ty[s] = y; d.tz[s] = z; d.ttid[s] = tid;
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
          float ox, oy, oz;
          if (nr == n) {
            ox = v.x + sig * g0; oy = v.y + sig * g1; oz = v.z + sig * g2;
            const float fx = floorf(ox * tr.inv_hf), fy = floorf(oy * tr.inv_hf), fz = floorf(oz * tr.inv_hf);
            ox -= fx * tr.hf; oy -= fy * tr.hf; oz -= fz * tr.hf;
            ix = wrap_cell(ix + static_cast<int>(fx), n);
            iy = wrap_cell(iy + static_cast<int>(fy), n);
            iz = wrap_cell(iz + static_cast<int>(fz), n);
          } else {
            // the hash grid changed this step: go through FP64 absolute positions
            const double hr = tr.h_ref;
            double ax = wrap_box((ix * hr - tr.halfL) + v.x + static_cast<double>(sig * g0), tr.L, tr.halfL);
            double ay = wrap_box((iy * hr - tr.halfL) + v.y + static_cast<double>(sig * g1), tr.L, tr.halfL);
            double az = wrap_box((iz * hr - tr.halfL) + v.z + static_cast<double>(sig * g2), tr.L, tr.halfL);
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
                d.lookback, d.g->epoch * MAX_PASSES + pass, d.g, sm);
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
    if (s == 0 || kf[s - 1] != key) { ci[0] = static_cast<int>(s); ci[2] = static_cast<int>(epoch); }
    if (s + 1 == n_live || kf[s + 1] != key) ci[1] = static_cast<int>(s + 1);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) d.g->n_live = n_live;
}

// ======================================================================== search
// For every unordered pair of live species whose types react (Table 1), separated by
// less than the reaction's cutoff under the minimum image (Eq. 2), evaluate the
// encounter probability and keep the pair if its uniform falls below it.
template <bool F32L>
__device__ void phase_search(const Dev& d) {
  if (status_of(d)) return;
  const uint32_t n_live = d.g->n_total - d.g->n_dead;
  const uint32_t epoch = d.g->epoch;
  const Tables& tb = *d.tables;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_live; s += stride) {
    const uint32_t cell = d.cell_sorted[s];
    const int b = (d.n_trains == 1) ? 0 : train_of_cell(d.trains, d.n_trains, cell);
    const Train& tr = d.trains[b];
    if (!tr.active || tr.free_jump) continue;
    uint32_t tid_i;
    double xi = 0, yi = 0, zi = 0;
    float4 vi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (F32L) { vi = d.s4[s]; tid_i = __float_as_uint(vi.w); }
    else { xi = d.sx[s]; yi = d.sy[s]; zi = d.sz[s]; tid_i = d.stid[s]; }
    const uint32_t ti = tid_type(tid_i);
    const uint32_t rmask = tb.reactive_mask[ti];
    if (!rmask) continue;
    const uint32_t id_i = tid_id(tid_i);
    const int n = tr.n;
    const uint32_t loc = cell - tr.cell_base;
    const int ix = static_cast<int>(loc % n), iy = static_cast<int>((loc / n) % n),
              iz = static_cast<int>(loc / (static_cast<uint32_t>(n) * n));
    for (int dz = -1; dz <= 1; ++dz) {
      const int cz = wrap_cell(iz + dz, n);
      for (int dy = -1; dy <= 1; ++dy) {
        const int cy = wrap_cell(iy + dy, n);
        for (int dx = -1; dx <= 1; ++dx) {
          const int cx = wrap_cell(ix + dx, n);
          const uint32_t nc = tr.cell_base + static_cast<uint32_t>((cz * n + cy) * n + cx);
          const int4 ci = d.cell_info[nc];
          if (static_cast<uint32_t>(ci.z) != epoch) continue;
          const uint32_t j0 = max(static_cast<uint32_t>(ci.x), s + 1);
          for (uint32_t j = j0; j < static_cast<uint32_t>(ci.y); ++j) {
            uint32_t tid_j;
            double xj = 0, yj = 0, zj = 0;
            float4 vj;
            if (F32L) { vj = d.s4[j]; tid_j = __float_as_uint(vj.w); }
            else { tid_j = d.stid[j]; }
            const uint32_t tj = tid_type(tid_j);
            if (!((rmask >> tj) & 1u)) continue;
            const int r = tb.pair_rxn[ti][tj];
            const uint32_t id_j = tid_id(tid_j);
            const bool i_lo = id_i < id_j;
            double d1sq, rx1, ry1, rz1;
            if (F32L) {
              float fx = dx * tr.hf + (vj.x - vi.x);
              float fy = dy * tr.hf + (vj.y - vi.y);
              float fz = dz * tr.hf + (vj.z - vi.z);
              if (!i_lo) { fx = -fx; fy = -fy; fz = -fz; }
              const float f2 = fx * fx + fy * fy + fz * fz;
              if (!(f2 < tr.rc2f[r])) continue;
              d1sq = f2; rx1 = fx; ry1 = fy; rz1 = fz;
            } else {
              xj = d.sx[j]; yj = d.sy[j]; zj = d.sz[j];
              if (i_lo) {
                rx1 = min_image(__dsub_rn(xj, xi), tr.L, tr.halfL);
                ry1 = min_image(__dsub_rn(yj, yi), tr.L, tr.halfL);
                rz1 = min_image(__dsub_rn(zj, zi), tr.L, tr.halfL);
              } else {
                rx1 = min_image(__dsub_rn(xi, xj), tr.L, tr.halfL);
                ry1 = min_image(__dsub_rn(yi, yj), tr.L, tr.halfL);
                rz1 = min_image(__dsub_rn(zi, zj), tr.L, tr.halfL);
              }
              d1sq = sq3(rx1, ry1, rz1);
              if (!(d1sq < tr.rc2[r])) continue;
            }
            const uint32_t id_lo = i_lo ? id_i : id_j, id_hi = i_lo ? id_j : id_i;
            const uint32_t t_lo = i_lo ? ti : tj, t_hi = i_lo ? tj : ti;
            // this step's displacements, regenerated from the counter-based stream
            double r0x, r0y, r0z;
            if (F32L) {
              float a0, a1, a2, c0, c1, c2;
              gauss3_f32(id_lo, tr.step, tr.key0, tr.key1, a0, a1, a2);
              gauss3_f32(id_hi, tr.step, tr.key0, tr.key1, c0, c1, c2);
              const float sl = tr.sigf[t_lo];
              const float sh = tr.sigf[t_hi];
              r0x = static_cast<float>(rx1) - (sh * c0 - sl * a0);
              r0y = static_cast<float>(ry1) - (sh * c1 - sl * a1);
              r0z = static_cast<float>(rz1) - (sh * c2 - sl * a2);
            } else {
              double a0, a1, a2, c0, c1, c2;
              gauss3_f64(id_lo, tr.step, tr.key0, tr.key1, a0, a1, a2);
              gauss3_f64(id_hi, tr.step, tr.key0, tr.key1, c0, c1, c2);
              const double sl = tr.sig[t_lo];
              const double sh = tr.sig[t_hi];
              r0x = __dsub_rn(rx1, __dsub_rn(__dmul_rn(sh, c0), __dmul_rn(sl, a0)));
              r0y = __dsub_rn(ry1, __dsub_rn(__dmul_rn(sh, c1), __dmul_rn(sl, a1)));
              r0z = __dsub_rn(rz1, __dsub_rn(__dmul_rn(sh, c2), __dmul_rn(sl, a2)));
            }
            const double d1 = sqrt(d1sq);
            const double d0 = sqrt(sq3(r0x, r0y, r0z));
            const double p = bridge_p(d0, d1, tb.R[r], __dmul_rn(tb.D_AB[r], tr.dt));
            const double u = pair_uniform(id_lo, id_hi, tr.step, tr.key0, tr.key1);
            if (!(u < p)) continue;
            const uint32_t c = atomicAdd(&d.g->n_cand, 1u);
            if (c >= d.cap_cand) { raise_status(d.g, CHEM_ECAPACITY); continue; }
            Cand cd;
            cd.s_lo = i_lo ? s : j;
            cd.s_hi = i_lo ? j : s;
            cd.id_lo = id_lo;
            cd.id_hi = id_hi;
            cd.rxn_train = static_cast<uint32_t>(r) | (static_cast<uint32_t>(b) << 8);
            cd.pad = 0;
            cd.d1sq = d1sq;
            d.cand[c] = cd;
          }
        }
      }
    }
  }
}

// ======================================================================== react
// One CTA of REACT_THREADS threads.
//  1. matching: rounds of locally-dominant selection; a pair is committed when it is the
//     smallest (d1^2, id_lo, id_hi) remaining pair of both its species. This equals the
//     greedy walk over pairs sorted by that key (closest first, lower ids first).
//  2. events ordered by (train, id_lo); product ids assigned in that order.
//  3. products written at the diffusion-weighted encounter point; tallies; logs.
//  4. end of step per train: FP64 clock, step counter, dt growth, step record.
struct ReactSmem {
  uint32_t n_alive, n_next, n_ev, carry;
  uint32_t first_pref[MAX_TRAINS];
  uint32_t prods_tr[MAX_TRAINS];
  uint32_t evs_tr[MAX_TRAINS];
  uint32_t warp_tot[REACT_THREADS / 32];
  unsigned long long small_keys[REACT_THREADS];
  uint32_t any;
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

__device__ __forceinline__ unsigned long long ev_key(const Dev& d, uint32_t c) {
  const Cand& cd = d.cand[c];
  return (static_cast<unsigned long long>(cd.rxn_train >> 8) << 32) | cd.id_lo;
}

template <bool F32L>
__device__ void phase_react(const Dev& d, ReactSmem& sm) {
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  const bool ok = status_of(d) == 0;
  const Tables& tb = *d.tables;
  unsigned long long* bd = reinterpret_cast<unsigned long long*>(d.keys0);
  unsigned long long* bp = bd + d.cap;
  uint32_t n_c = min(d.g->n_cand, d.cap_cand);
  if (!ok) n_c = 0;
  if (tid == 0) { sm.n_alive = n_c; sm.n_ev = 0; sm.any = 0; }
  for (uint32_t i = tid; i < n_c; i += nt) d.alive0[i] = i;
  __syncthreads();
  uint32_t* alive = d.alive0;
  uint32_t* nxt = d.alive1;
  // ---- 1. matching rounds (each round commits at least the smallest remaining pair)
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
        d.ev_list[atomicAdd(&sm.n_ev, 1u)] = c;
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
  // ---- 2. order events by (train, id_lo); keys are unique
  const uint32_t E = sm.n_ev;
  uint32_t* order;  // order[k] = candidate index of the k-th event
  if (E <= static_cast<uint32_t>(nt)) {
    if (static_cast<uint32_t>(tid) < E) sm.small_keys[tid] = ev_key(d, d.ev_list[tid]);
    __syncthreads();
    uint32_t rank = 0;
    if (static_cast<uint32_t>(tid) < E) {
      const unsigned long long k = sm.small_keys[tid];
      for (uint32_t q = 0; q < E; ++q) rank += (sm.small_keys[q] < k);
    }
    __syncthreads();
    if (static_cast<uint32_t>(tid) < E) d.ev_v1[rank] = d.ev_list[tid];
    order = d.ev_v1;
  } else {
    // LSD radix over the 64-bit key (train | id_lo), 8 bits per pass, stable per pass:
    // each pass walks the events in tiles of blockDim, ranking within a tile by
    // counting equal digits at lower positions, with running digit offsets.
    uint32_t* ord_in = d.ev_v0;
    uint32_t* ord_out = d.ev_v1;
    for (uint32_t i = tid; i < E; i += nt) ord_in[i] = d.ev_list[i];
    __syncthreads();
    uint32_t* digit_base = d.ev_k0;  // [256] scratch
    uint32_t* digit_run = d.ev_k1;   // [256]
    int top_bit = 32 + 8;            // trains < 256
    for (int shift = 0; shift < top_bit; shift += 8) {
      for (int i = tid; i < RADIX; i += nt) digit_base[i] = 0;
      __syncthreads();
      for (uint32_t i = tid; i < E; i += nt)
        atomicAdd(&digit_base[(ev_key(d, ord_in[i]) >> shift) & 255u], 1u);
      __syncthreads();
      if (tid == 0) {
        uint32_t s = 0;
        for (int q = 0; q < RADIX; ++q) { const uint32_t c = digit_base[q]; digit_run[q] = s; s += c; }
      }
      __syncthreads();
      for (uint32_t t0 = 0; t0 < E; t0 += nt) {
        const uint32_t i = t0 + tid;
        const bool valid = i < E;
        const uint32_t dg = valid ? static_cast<uint32_t>((ev_key(d, ord_in[i]) >> shift) & 255u) : 0u;
        if (valid) sm.small_keys[tid] = dg;
        __syncthreads();
        uint32_t rk = 0;
        if (valid) for (int q = 0; q < tid; ++q) rk += (sm.small_keys[q] == dg);
        if (valid) ord_out[digit_run[dg] + rk] = ord_in[i];
        __syncthreads();
        if (valid) atomicAdd(&digit_run[dg], 1u);
        __syncthreads();
      }
      uint32_t* t = ord_in; ord_in = ord_out; ord_out = t;
      __syncthreads();
    }
    order = ord_in;
  }
  __syncthreads();
  // ---- 3. products: exclusive prefix of product counts in event order
  for (uint32_t b = tid; b < d.n_trains; b += nt) { sm.first_pref[b] = 0xFFFFFFFFu; sm.prods_tr[b] = 0; sm.evs_tr[b] = 0; }
  if (tid == 0) sm.carry = 0;
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
        atomicAdd(reinterpret_cast<unsigned long long*>(&tr.counts[tlo]), static_cast<unsigned long long>(-1ll));
        atomicAdd(reinterpret_cast<unsigned long long*>(&tr.counts[thi]), static_cast<unsigned long long>(-1ll));
        for (uint32_t q = 0; q < np; ++q)
          atomicAdd(reinterpret_cast<unsigned long long*>(&tr.counts[tb.prod[r][q]]), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(&tr.events[r]), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(&tr.water), static_cast<unsigned long long>(static_cast<long long>(tb.water[r])));
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
  // ---- 4. end of step
  for (uint32_t b = tid; b < d.n_trains; b += nt) {
    Train& tr = d.trains[b];
    if (tr.active && ok) {
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
      d.g->n_events = E;
      if (d.cap_ev_log) d.g->ev_log_n += E;
    }
    d.g->any_active = sm.any;
  }
  __syncthreads();
}

}  // namespace chem
