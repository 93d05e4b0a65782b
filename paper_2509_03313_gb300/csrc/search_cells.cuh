// Pair search by cell tiles (the "species_per_item > 0" mapping).
//
// For every unordered pair of live species whose types react (Table 1), separated by
// less than the reaction's cutoff under the minimum image (Eq. 2), the search evaluates
// the encounter probability and keeps the pair if its uniform falls below it.
//
// One warp per work item: up to SC_HOMES consecutive sorted species ("homes") of one
// hash cell, one home per bit of a 32-bit mask.
//  1. Each home lane loads its state and decides, with the box-gap test against the
//     largest cutoff of its type, which cells of the half shell (the 13 forward cells) it
//     can reach; a bit mask per home. Bit 0 is the own cell's later slots.
//  2. The warp looks up the union of those cells (occupancy bit, then the epoch-stamped
//     range) and lays the non-empty ranges end to end as one list.
//  3. Lanes take 32 list entries at a time (coalesced 16-byte loads). For its neighbour
//     a lane forms the set of homes to test: those that reach the neighbour's cell, whose
//     type reacts with the neighbour's, and (own cell) that precede it. It tests them
//     one by one (home data is a shared-memory broadcast) and sets one bit per pair
//     inside the cutoff.
//  4. The set bits go to the warp's pair queue through one warp-wide prefix sum; the
//     queue is resolved one pair per lane (orientation, start separation from the
//     step's displacements, Philox uniform, touch probability) whenever it fills.
// In FP64 mode the walk tests the FP32 cell offsets against cutoffs widened past any
// FP32 rounding and the queue resolution repeats the test exactly in FP64, so the
// candidate set is the FP64 reference's.
#pragma once
#include "phases.cuh"

namespace chem {

constexpr int SC_HOMES = 32;    // home species per work item (one bit each)
constexpr int SC_QCAP = 128;    // queued pairs per warp
constexpr int SC_RANGES = N_FWD;  // own cell + 13 forward cells

struct ScWarp {
  float4 hv[SC_HOMES];             // homes: FP32 cell offsets and id/type bits
  uint32_t reach[SC_RANGES];       // per half-shell cell: homes that reach it
  uint32_t hm_type[MAXT];          // per neighbour type: homes whose type reacts with it
  uint32_t rs[SC_RANGES];          // non-empty neighbour ranges: first slot,
  uint32_t rlen[SC_RANGES + 1];    // length,
  uint32_t roff[SC_RANGES + 1];    // offset in the flattened list (roff[nr] = total),
  uint8_t rk[SC_RANGES + 1];       // and half-shell index
  float ct[MAXT * MAXT];           // squared cutoffs of the item's train (FP64 mode: widened)
  uint32_t qi[SC_QCAP];            // queued pairs: home slot,
  uint32_t qj[SC_QCAP];            // neighbour slot,
  uint32_t qk[SC_QCAP];            // half-shell index | train << 8
  uint32_t qn;
  int ct_b;
};

template <int W>
struct ScSmem {
  FwdSmem fo;  // half-shell offsets
  ScWarp w[W];
};

// Acceptance of one queued pair (home slot si, neighbour slot j in the forward cell k of
// the home's cell) and, when accepted, its candidate record.
template <bool F32L>
__device__ __forceinline__ void sc_resolve(const Dev& d, const Tables& tb, const FwdSmem& fo, uint32_t si,
                                           uint32_t j, uint32_t kb, const uint32_t* vf, uint32_t& n_in_cut) {
  const int k = static_cast<int>(kb & 255u), b = static_cast<int>(kb >> 8);
  const Train& tr = d.trains[b];
  if constexpr (F32L) {
    const float4 hv = d.s4[si], vj = d.s4[j];
    // the walk's separation, formed the same way
    float fx, fy, fz;
    const float f2 = sep_f32(fo.f[0][k], fo.f[1][k], fo.f[2][k], tr.hf, vj, hv, fx, fy, fz);
    const uint32_t tid_i = __float_as_uint(hv.w), tid_j = __float_as_uint(vj.w);
    const int r = tb.pair_rxn[tid_type(tid_i)][tid_type(tid_j)];
    const uint32_t id_i = tid_id(tid_i), id_j = tid_id(tid_j);
    const bool i_lo = id_i < id_j;
    const uint32_t id_lo = i_lo ? id_i : id_j, id_hi = i_lo ? id_j : id_i;
    if (!i_lo) { fx = -fx; fy = -fy; fz = -fz; }
    // this step's displacements, gathered into sorted order
    const float4 di = d.sd4[si], dj = d.sd4[j];
    const float4 dlo = i_lo ? di : dj, dhi = i_lo ? dj : di;
    const float r0x = fx - (dhi.x - dlo.x), r0y = fy - (dhi.y - dlo.y), r0z = fz - (dhi.z - dlo.z);
    const float d0sq = r0x * r0x + r0y * r0y + r0z * r0z;
    if (!accept_f32(d0sq, f2, r, tb, tr, id_lo, id_hi)) return;
    emit_candidate(d, i_lo ? si : j, i_lo ? j : si, id_lo, id_hi, r, b, static_cast<double>(f2));
  } else {
    const uint32_t tid_i = d.stid[si], tid_j = d.stid[j];
    const uint32_t ti = tid_type(tid_i), tj = tid_type(tid_j);
    // minimum image of x_j - x_i (Eq. 2), exactly as the reference forms it up to the
    // orientation, which is negated below without rounding
    double rx1 = min_image(__dsub_rn(d.sx[j], d.sx[si]), tr.L, tr.halfL);
    double ry1 = min_image(__dsub_rn(d.sy[j], d.sy[si]), tr.L, tr.halfL);
    double rz1 = min_image(__dsub_rn(d.sz[j], d.sz[si]), tr.L, tr.halfL);
    const double d1sq = sq3(rx1, ry1, rz1);
    if (!(d1sq < tr.rc2_tt[ti * MAXT + tj])) return;
    ++n_in_cut;
    const int r = tb.pair_rxn[ti][tj];
    const uint32_t id_i = tid_id(tid_i), id_j = tid_id(tid_j);
    const bool i_lo = id_i < id_j;
    const uint32_t id_lo = i_lo ? id_i : id_j, id_hi = i_lo ? id_j : id_i;
    if (!i_lo) { rx1 = -rx1; ry1 = -ry1; rz1 = -rz1; }
    const uint32_t ti_idx = vf ? vf[si] : si, tj_idx = vf ? vf[j] : j;
    const double eix = d.tdx[ti_idx], eiy = d.tdy[ti_idx], eiz = d.tdz[ti_idx];
    const double ejx = d.tdx[tj_idx], ejy = d.tdy[tj_idx], ejz = d.tdz[tj_idx];
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
__device__ __forceinline__ void sc_flush(const Dev& d, const Tables& tb, const FwdSmem& fo, ScWarp& w,
                                         const uint32_t* vf, int lane, uint32_t& n_in_cut) {
  const uint32_t nq = w.qn;
  for (uint32_t e = lane; e < nq; e += 32) sc_resolve<F32L>(d, tb, fo, w.qi[e], w.qj[e], w.qk[e], vf, n_in_cut);
  __syncwarp();
  if (lane == 0) w.qn = 0;
  __syncwarp();
}

template <bool F32L, int W>
__device__ void phase_search_cells(const Dev& d, ScSmem<W>& sm) {
  if (!d.g->search_cells_now) return;  // this step runs one thread per species (grid-uniform)
  constexpr uint32_t FULL = 0xffffffffu;
  const uint32_t n_items = min(d.g->n_items, d.cap_items);
  const uint32_t epoch = d.g->epoch;
  // pre-sort slot of each sorted slot (FP64 displacements); nullptr when nothing moved
  const uint32_t* vf = d.g->sort_any ? (d.g->sort_parity ? d.vals1 : d.vals0) : nullptr;
  const Tables& tb = *d.tables;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  ScWarp& w = sm.w[wib];
  const FwdSmem& fo = sm.fo;
  fwd_smem_fill(sm.fo);
  if (lane == 0) { w.qn = 0; w.ct_b = -1; }
  // one status for the whole CTA (a barrier, which also publishes the offsets)
  if (!block_status_ok(d)) return;
  uint32_t n_tested = 0, n_in_cut = 0;  // pair-search counters of this lane
  const uint32_t item_home = min(max(d.g->item_home, 1u), static_cast<uint32_t>(SC_HOMES));
  const uint32_t n_live = d.g->n_total - d.g->n_dead;
  // work stealing two items ahead: while an item is processed, lane 0 holds the claim of
  // the item after next and the record of the next one, both in flight
  uint32_t it = 0, it_n1 = 0;
  if (lane == 0) {
    it = atomicAdd(&d.g->item_ctr, 1u);
    it_n1 = atomicAdd(&d.g->item_ctr, 1u);
  }
  it = __shfl_sync(FULL, it, 0);
  it_n1 = __shfl_sync(FULL, it_n1, 0);
  uint2 rec = it < n_items ? d.items[it] : make_uint2(0u, 0u);
  while (it < n_items) {
    uint32_t it_n2 = 0;
    uint2 rec_n1 = make_uint2(0u, 0u);
    if (lane == 0) {
      it_n2 = atomicAdd(&d.g->item_ctr, 1u);
      if (it_n1 < n_items) rec_n1 = d.items[it_n1];
    }
    const uint32_t s0 = rec.x, cell = rec.y;
    const int b = (d.n_trains == 1) ? 0 : train_of_cell(d.trains, d.n_trains, cell);
    const Train& tr = d.trains[b];
    if (w.ct_b != b) {  // cutoff table of this train (warp-uniform)
      for (int q = lane; q < MAXT * MAXT; q += 32) w.ct[q] = F32L ? tr.rc2f_tt[q] : tr.rc2w_tt[q];
      __syncwarp();
      if (lane == 0) w.ct_b = b;
      __syncwarp();
    }
    const float hf = tr.hf;
    int cx, cy, cz;
    cell_decode(cell - tr.cell_base, tr.cb, cx, cy, cz);
    // independent loads issued together: this lane's home (speculatively, up to the item
    // size), the own cell's end, and the occupancy bit of the half-shell cell k = lane
    const uint32_t s_home = s0 + static_cast<uint32_t>(lane);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (static_cast<uint32_t>(lane) < item_home && s_home < n_live) v = d.s4[s_home];
    const uint32_t own_end = static_cast<uint32_t>(d.cell_info[cell].y);
    uint32_t nc0 = 0;
    bool occ0 = false;
    if (lane >= 1 && lane < N_FWD) {
      const int n = tr.n;
      nc0 = tr.cell_base + cell_encode(step_cell(cx, fo.i[0][lane], n), step_cell(cy, fo.i[1][lane], n),
                                       step_cell(cz, fo.i[2][lane], n), tr.cb);
      occ0 = (d.occ[nc0 >> 5] >> (nc0 & 31u)) & 1u;
    }
    // homes: from s0 to the cell's end or the next multiple of the item size, where the
    // gather starts the next item
    const uint32_t item_end = min(own_end, (s0 / item_home + 1u) * item_home);
    const uint32_t nh = item_end - s0;  // 1..32 homes
    // cells worth looking at: the own cell, and forward cells with their occupancy bit set
    const uint32_t occ_mask = 1u | __ballot_sync(FULL, occ0);
    // 1. homes and the cells each can reach
    uint32_t km = 0u;
    uint32_t rmask = 0u;  // partner types of this lane's home
    if (static_cast<uint32_t>(lane) < nh) {
      w.hv[lane] = v;
      const uint32_t t = tid_type(__float_as_uint(v.w));
      rmask = tb.reactive_mask[t];
      if (rmask != 0u) {
        if (s_home + 1u < own_end) km = 1u;
        float rcmax2 = -1.f;
#pragma unroll
        for (int u = 0; u < MAXT; ++u) rcmax2 = fmaxf(rcmax2, w.ct[t * MAXT + u]);
        rcmax2 *= 1.0001f;
        // a forward cell whose nearest point is farther from the home than its largest
        // cutoff holds no partner (gaps taken 1e-5 of a cell short: no rounding drops one)
        const float eps = 1e-5f * hf;
        auto gap = [&](int o, float of) {
          const float g = o > 0 ? static_cast<float>(o) * hf - of : (o < 0 ? of + static_cast<float>(-o - 1) * hf : 0.f);
          return fmaxf(g - eps, 0.f);
        };
        // per axis the gap is 0 (same layer), the distance to the lower face (offset -1)
        // or to the upper face (offset +1); the 13 offsets unrolled
        const float xm = gap(-1, v.x), xp = gap(1, v.x), ym = gap(-1, v.y), yp = gap(1, v.y);
        const float zp = gap(1, v.z);
        const float xm2 = xm * xm, xp2 = xp * xp, ym2 = ym * ym, yp2 = yp * yp, zp2 = zp * zp;
        uint32_t kr = 0u;
#pragma unroll
        for (int k = 1; k < N_FWD; ++k) {
          int dx, dy, dz;
          fwd_offset(k, dx, dy, dz);
          const float sx = dx < 0 ? xm2 : (dx > 0 ? xp2 : 0.f);
          const float sy = dy < 0 ? ym2 : (dy > 0 ? yp2 : 0.f);
          const float sz = dz > 0 ? zp2 : 0.f;
          if ((sx + sy) + sz <= rcmax2) kr |= 1u << k;
        }
        km |= kr & occ_mask;
      }
    }
    // a 32 x 32 bit transpose of (lane = home; bits 0..13 the half-shell cells it
    // reaches, bits 16..23 the types it reacts with) leaves in lane k the homes that
    // reach cell k and in lane 16 + u the homes that react with type u
    static_assert(N_FWD <= 16 && MAXT <= 16, "reach and partner-type bits share one word");
    uint32_t x = km | (rmask << 16);
    auto stage = [&](int sh, uint32_t msk) {
      const uint32_t y = __shfl_xor_sync(FULL, x, sh);
      x = (lane & sh) ? ((x & ~msk) | ((y >> sh) & msk)) : ((x & msk) | ((y & msk) << sh));
    };
    stage(16, 0x0000FFFFu);
    stage(8, 0x00FF00FFu);
    stage(4, 0x0F0F0F0Fu);
    stage(2, 0x33333333u);
    stage(1, 0x55555555u);
    if (lane < N_FWD) w.reach[lane] = x;
    if (lane >= 16 && lane < 16 + MAXT) w.hm_type[lane - 16] = x;
    // 2. the reachable cells' ranges (lane k: half-shell cell k), non-empty ones laid end
    // to end in half-shell order
    uint32_t st = 0, len = 0;
    if (lane < N_FWD && x != 0u) {
      if (lane == 0) {
        st = s0 + 1u;
        len = own_end - st;
      } else {
        // occupied (the bit was tested above); the epoch-stamped entry confirms
        const int4 ci = d.cell_info[nc0];
        if (static_cast<uint32_t>(ci.z) == epoch && ci.y > ci.x) {
          st = static_cast<uint32_t>(ci.x);
          len = static_cast<uint32_t>(ci.y - ci.x);
        }
      }
    }
    const uint32_t bal = __ballot_sync(FULL, len > 0u);
    const uint32_t nr = __popc(bal);
    if (len > 0u) {
      const uint32_t pos = __popc(bal & lanemask_lt);
      w.rs[pos] = st;
      w.rlen[pos] = len;
      w.rk[pos] = static_cast<uint8_t>(lane);
    }
    __syncwarp();
    {  // exclusive offsets of the ranges (at most N_FWD <= 16: lanes 0..15)
      const uint32_t x0 = static_cast<uint32_t>(lane) < nr ? w.rlen[lane] : 0u;
      uint32_t a = x0;
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
        const uint32_t ya = __shfl_up_sync(FULL, a, o);
        if (lane >= o) a += ya;
      }
      if (static_cast<uint32_t>(lane) < nr) w.roff[lane] = a - x0;
      if (lane == 15) w.roff[nr] = a;
    }
    __syncwarp();
    const uint32_t total = w.roff[nr];
    const uint32_t home_bits = nh >= 32u ? FULL : ((1u << nh) - 1u);
    // 3. lanes over the flattened neighbour list, each against its set of homes
    for (uint32_t f0 = 0; f0 < total; f0 += 32) {
      const uint32_t f = f0 + static_cast<uint32_t>(lane);
      uint32_t pass = 0u, j = 0u, k = 0u;
      if (f < total) {
        int lo = 0, hi = static_cast<int>(nr) - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (w.roff[mid] <= f) lo = mid; else hi = mid - 1;
        }
        j = w.rs[lo] + (f - w.roff[lo]);
        k = w.rk[lo];
        const float4 vj = d.s4[j];
        const uint32_t tj = tid_type(__float_as_uint(vj.w));
        // the neighbour in the home cell's frame; the separation below is sep_f32's
        const float bx = __fmaf_rn(fo.f[0][k], hf, vj.x), by = __fmaf_rn(fo.f[1][k], hf, vj.y),
                    bz = __fmaf_rn(fo.f[2][k], hf, vj.z);
        uint32_t m = w.reach[k] & w.hm_type[tj] & home_bits;
        if (k == 0u) {  // own cell: only the homes before this slot
          const uint32_t lim = j - s0;
          m &= lim >= 32u ? FULL : ((1u << lim) - 1u);
        }
        n_tested += __popc(m);
        while (m != 0u) {
          const int h = __ffs(m) - 1;
          m &= m - 1u;
          const float4 hv = w.hv[h];
          const float dx = __fsub_rn(bx, hv.x), dy = __fsub_rn(by, hv.y), dz = __fsub_rn(bz, hv.z);
          const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
          if (d2 < w.ct[(tid_type(__float_as_uint(hv.w)) << 3) | tj]) pass |= 1u << h;
        }
        if constexpr (F32L) n_in_cut += __popc(pass);
      }
      // 4. queue the passing pairs (one warp-wide prefix sum), resolving when full
      const uint32_t kb = k | (static_cast<uint32_t>(b) << 8);
      while (__any_sync(FULL, pass != 0u)) {
        const uint32_t cnt = __popc(pass);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += y;
        }
        const uint32_t base = w.qn;
        const uint32_t want = __shfl_sync(FULL, incl, 31);
        uint32_t pos = base + incl - cnt;
        while (pass != 0u && pos < static_cast<uint32_t>(SC_QCAP)) {
          const int h = __ffs(pass) - 1;
          pass &= pass - 1u;
          w.qi[pos] = s0 + static_cast<uint32_t>(h);
          w.qj[pos] = j;
          w.qk[pos] = kb;
          ++pos;
        }
        __syncwarp();
        if (lane == 0) w.qn = min(static_cast<uint32_t>(SC_QCAP), base + want);
        __syncwarp();
        if (w.qn > static_cast<uint32_t>(SC_QCAP) - 32u) sc_flush<F32L>(d, tb, fo, w, vf, lane, n_in_cut);
      }
    }
    it = it_n1;
    rec = make_uint2(__shfl_sync(FULL, rec_n1.x, 0), __shfl_sync(FULL, rec_n1.y, 0));
    it_n1 = __shfl_sync(FULL, it_n2, 0);
  }
  sc_flush<F32L>(d, tb, fo, w, vf, lane, n_in_cut);
  add_pair_counts(d, n_tested, n_in_cut);
}

}  // namespace chem
