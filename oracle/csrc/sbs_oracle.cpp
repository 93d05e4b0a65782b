// Plain FP64 C++ reference ("oracle") of the step-by-step (SBS) chemical stage.
//
// TEST INFRASTRUCTURE ONLY: only the tests and the CPU-baseline legs of bench.py load it;
// the library never does. It shares no code with the CUDA path (no header, helper or
// table) and computes, single-threaded and step by step, what oracle/sbs.py computes, from
// the paper's definitions and the same readings where the paper is silent:
//
//  * Sec. 2.1 workflow: species enter at their arrival (rounded up to the next step
//    boundary), ids in (arrival, call order) order, and are carried from step to step;
//  * Eq. 1 (periodic boundary condition 1) after every displacement, applied as often as
//    needed; Eq. 2 (minimum image) for every pair separation;
//  * Sec. 2.4 with Table 1 and Eq. kdiff1/kdiff2: R = k_tab / (4 pi D_AB N_A) with
//    D_AB = D_A + D_B, the printed 2k used as is for the self reactions;
//  * Brownian steps: Philox4x32-10 (Salmon et al., SC'11) keyed by (seed low word, seed
//    high word XOR train id), counters (id, step, 0, tag) for tags 0 and 1, 53-bit
//    uniforms, Box-Muller;
//  * reactions (Sec. 2.2 Fig. PBClattice, Sec. 2.4): a reacting type pair closer than
//    R + c sqrt(2 D_AB dt) at the end of a step is accepted with the probability that its
//    relative path touched the reaction sphere during the step given both separations,
//    (exp(-a) - exp(-b)) / (1 - exp(-b)), a = (d0 - R)(d1 - R) / (D_AB dt),
//    b = d0 d1 / (D_AB dt), 1 when d0 or d1 <= R, against a uniform from counter
//    (id_lo, step, id_hi, 2); one reaction per species, closest pair first, lower ids
//    breaking ties; products at the diffusion-weighted encounter point, ids in id_lo
//    order and table order;
//  * time step: dt_min, growing by dt_growth up to dt_max, restarting at dt_min after a
//    release, capped so that every cutoff stays <= L/3, the last step of a run trimmed to
//    land on its end time (1e-6 relative slack); optional free-diffusion jump once
//    sbs_horizon has passed since the last release.
// Pairs are found with a periodic cell list (sorted cell keys, cells at least as wide as
// the largest cutoff; all pairs when the box holds fewer than 3 cells per axis). The
// beam-off (homogeneous) stage of Sec. 2.3 is not part of this program.
//
// Build: g++ -O2 -ffp-contract=off -shared -fPIC (no fused multiply-add anywhere).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <numeric>
#include <unordered_set>
#include <utility>
#include <vector>

namespace {

constexpr double kNA = 6.02214076e23;  // 1/mol, exact SI
constexpr double kPi = 3.141592653589793;
constexpr double kTwoPi = 2.0 * kPi;
constexpr double kTwoPowM53 = 1.0 / 9007199254740992.0;
constexpr double kEndSlack = 1.0 + 1e-6;

// Philox4x32 with 10 rounds (the published algorithm: two 32x32 -> 64 multiplications per
// round, high halves XORed with the other words and the round key, Weyl key schedule).
struct Block { uint32_t w[4]; };
Block philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c0;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c2;
    const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
    const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return Block{{c0, c1, c2, c3}};
}

uint64_t top53(uint32_t hi, uint32_t lo) { return ((static_cast<uint64_t>(hi) << 32) | lo) >> 11; }
// (0, 1]: (m + 1) 2^-53 and [0, 1): m 2^-53 for the top 53 bits m of (hi:lo).
double uniform_open0(uint32_t hi, uint32_t lo) { return (static_cast<double>(top53(hi, lo)) + 1.0) * kTwoPowM53; }
double uniform_closed0(uint32_t hi, uint32_t lo) { return static_cast<double>(top53(hi, lo)) * kTwoPowM53; }

// Three standard normals of one species at one step (Box-Muller on the blocks of tags 0
// and 1; the fourth normal is unused).
void gaussians(uint32_t id, uint32_t step, uint32_t k0, uint32_t k1, double g[3]) {
  const Block a = philox(id, step, 0u, 0u, k0, k1);
  const Block b = philox(id, step, 0u, 1u, k0, k1);
  const double u1 = uniform_open0(a.w[0], a.w[1]), u2 = uniform_closed0(a.w[2], a.w[3]);
  const double u3 = uniform_open0(b.w[0], b.w[1]), u4 = uniform_closed0(b.w[2], b.w[3]);
  const double r = std::sqrt(-2.0 * std::log(u1)), th = kTwoPi * u2;
  const double r2 = std::sqrt(-2.0 * std::log(u3)), th2 = kTwoPi * u4;
  g[0] = r * std::cos(th);
  g[1] = r * std::sin(th);
  g[2] = r2 * std::cos(th2);
}

double acceptance_uniform(uint32_t id_lo, uint32_t id_hi, uint32_t step, uint32_t k0, uint32_t k1) {
  const Block w = philox(id_lo, step, id_hi, 2u, k0, k1);
  return uniform_closed0(w.w[0], w.w[1]);
}

// Eq. 1: shift x by whole box lengths into [-L/2, L/2).
double wrap(double x, double L) {
  const double k = std::floor((x + 0.5 * L) / L);
  x = x - k * L;
  if (x >= 0.5 * L) x = x - L;
  if (x < -0.5 * L) x = x + L;
  return x;
}

// Eq. 2 for the separation of two in-box points.
double min_image(double dx, double L) {
  if (dx >= 0.5 * L) return dx - L;
  if (dx < -0.5 * L) return dx + L;
  return dx;
}

double sq_norm(double x, double y, double z) { return (x * x + y * y) + z * z; }

// (exp(-a) - exp(-b)) / (1 - exp(-b)) written as exp(-a) expm1(-c) / expm1(-b), c = b - a.
double touch_probability(double d0, double d1, double R, double ddt) {
  if (d1 <= R || d0 <= R) return 1.0;
  const double a = ((d0 - R) * (d1 - R)) / ddt;
  const double b = (d0 * d1) / ddt;
  const double c = (R * ((d0 + d1) - R)) / ddt;
  return std::exp(-a) * (std::expm1(-c) / std::expm1(-b));
}

// Eq. kdiff1 at steady state solved for R (nm): k in L/mol/s, D_AB in nm^2/s, 1 L = 1e24 nm^3.
double reaction_radius(double k_tab, double D_AB) { return (k_tab * 1e24 / kNA) / (4.0 * kPi * D_AB); }

// Calls f(i, j) once for every unordered pair of points in the same or neighbouring cells
// of a periodic cell list whose cells are at least r wide: a superset of the pairs closer
// than r (minimum image). All pairs when fewer than 3 cells fit along the box.
template <class F>
void near_pairs(const std::vector<double>& pos, double L, double r, F&& f) {
  const size_t n = pos.size() / 3;
  const double ncd = r > 0.0 ? std::floor(L / r) : 1.0;
  const int64_t nc = static_cast<int64_t>(std::min(ncd, 1048576.0));
  if (nc < 3) {
    for (size_t i = 0; i < n; ++i)
      for (size_t j = i + 1; j < n; ++j) f(i, j);
    return;
  }
  const double h = L / static_cast<double>(nc);
  auto key_of = [&](int64_t qx, int64_t qy, int64_t qz) { return (qz * nc + qy) * nc + qx; };
  std::vector<std::pair<int64_t, size_t>> keyed(n);
  for (size_t i = 0; i < n; ++i) {
    int64_t q[3];
    for (int a = 0; a < 3; ++a) {
      const int64_t v = static_cast<int64_t>(std::floor((pos[3 * i + a] + 0.5 * L) / h));
      q[a] = std::min<int64_t>(std::max<int64_t>(v, 0), nc - 1);
    }
    keyed[i] = {key_of(q[0], q[1], q[2]), i};
  }
  std::sort(keyed.begin(), keyed.end());
  // occupied cells: key and [begin, end) into keyed
  std::vector<int64_t> ckey;
  std::vector<size_t> cbeg;
  for (size_t k = 0; k < n; ++k)
    if (k == 0 || keyed[k].first != keyed[k - 1].first) {
      ckey.push_back(keyed[k].first);
      cbeg.push_back(k);
    }
  cbeg.push_back(n);
  for (size_t c = 0; c < ckey.size(); ++c) {
    const int64_t qx = ckey[c] % nc, qy = (ckey[c] / nc) % nc, qz = ckey[c] / (nc * nc);
    for (size_t a = cbeg[c]; a < cbeg[c + 1]; ++a)
      for (size_t b = a + 1; b < cbeg[c + 1]; ++b) f(keyed[a].second, keyed[b].second);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          // the 13 neighbours with (dz, dy, dx) lexicographically after (0, 0, 0)
          if (!(dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0))))) continue;
          const int64_t k1 = key_of(((qx + dx) % nc + nc) % nc, ((qy + dy) % nc + nc) % nc, ((qz + dz) % nc + nc) % nc);
          const auto it = std::lower_bound(ckey.begin(), ckey.end(), k1);
          if (it == ckey.end() || *it != k1) continue;
          const size_t c1 = static_cast<size_t>(it - ckey.begin());
          for (size_t a = cbeg[c]; a < cbeg[c + 1]; ++a)
            for (size_t b = cbeg[c1]; b < cbeg[c1 + 1]; ++b) f(keyed[a].second, keyed[b].second);
        }
  }
}

// One reaction per species: the pairs by increasing (d1^2, id_lo, id_hi), each kept when
// neither species is taken yet. Returns the kept indices in that order.
std::vector<size_t> greedy_matching(const std::vector<int64_t>& id_lo, const std::vector<int64_t>& id_hi,
                                    const std::vector<double>& d1sq) {
  std::vector<size_t> order(d1sq.size());
  std::iota(order.begin(), order.end(), size_t(0));
  std::sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    if (d1sq[x] != d1sq[y]) return d1sq[x] < d1sq[y];
    if (id_lo[x] != id_lo[y]) return id_lo[x] < id_lo[y];
    return id_hi[x] < id_hi[y];
  });
  std::unordered_set<int64_t> taken;
  std::vector<size_t> kept;
  for (size_t c : order) {
    if (taken.count(id_lo[c]) || taken.count(id_hi[c])) continue;
    taken.insert(id_lo[c]);
    taken.insert(id_hi[c]);
    kept.push_back(c);
  }
  return kept;
}

struct Rxn {
  int a, b;
  double k_tab, D_AB, R;
  int n_prod, prod[3], water;
};

struct Oracle {
  int n_types = 0;
  std::vector<double> D;
  std::vector<Rxn> rx;
  std::vector<int> pair_rxn;  // n_types^2, -1 when the types do not react
  double L = 0, dt_min = 0, dt_max = 0, dt_growth = 1, c = 3, horizon = 0, dt_L = 0;
  bool reset_on_release = true, record = true;
  uint32_t k0 = 0, k1 = 0;
  std::vector<int64_t> ids;  // live species
  std::vector<int> types;
  std::vector<double> pos;   // 3 per species
  std::vector<double> p_t, p_pos;  // pending species in (arrival, call order) order
  std::vector<int> p_types;
  double t = 0, dt_cur = 0, t_last_release = 0, E_dep = 0;
  int64_t step = 0, next_id = 0, water = 0, species_steps = 0;
  std::vector<int64_t> events_total;
  std::vector<int64_t> event_log;   // (step, rxn, id_lo, id_hi, first product id, n_prod)
  std::vector<int64_t> step_log;    // (step, n_live, n_events, counts per type)
  std::vector<double> step_times;   // (t_start, dt)
};

void release(Oracle& o) {
  const size_t n = static_cast<size_t>(std::upper_bound(o.p_t.begin(), o.p_t.end(), o.t) - o.p_t.begin());
  if (n == 0) return;
  for (size_t i = 0; i < n; ++i) {
    o.ids.push_back(o.next_id++);
    o.types.push_back(o.p_types[i]);
    for (int a = 0; a < 3; ++a) o.pos.push_back(o.p_pos[3 * i + a]);
  }
  o.p_t.erase(o.p_t.begin(), o.p_t.begin() + static_cast<std::ptrdiff_t>(n));
  o.p_types.erase(o.p_types.begin(), o.p_types.begin() + static_cast<std::ptrdiff_t>(n));
  o.p_pos.erase(o.p_pos.begin(), o.p_pos.begin() + static_cast<std::ptrdiff_t>(3 * n));
  o.t_last_release = o.t;
  if (o.reset_on_release) o.dt_cur = o.dt_min;
}

struct Cand {
  size_t lo, hi;  // indices into the live arrays, ids[lo] < ids[hi]
  int r;
  double d1sq, r1[3];
};

void step_once(Oracle& o, double t_end) {
  release(o);
  const double next_arrival = o.p_t.empty() ? std::numeric_limits<double>::infinity() : o.p_t.front();
  const bool free_jump = o.horizon > 0.0 && (o.t - o.t_last_release) >= o.horizon && next_arrival > o.t;
  double dt, t_next;
  if (free_jump) {
    t_next = std::min(t_end, next_arrival);
    dt = t_next - o.t;
  } else {
    dt = std::min(o.dt_cur, o.dt_L);
    if (t_end - o.t <= dt * kEndSlack) {
      dt = t_end - o.t;
      t_next = t_end;
    } else {
      t_next = o.t + dt;
    }
  }
  const size_t n_live = o.ids.size();
  o.species_steps += static_cast<int64_t>(n_live);
  const uint32_t st = static_cast<uint32_t>(o.step);
  // Brownian displacement and Eq. 1
  std::vector<double> delta(3 * n_live);
  for (size_t i = 0; i < n_live; ++i) {
    double g[3];
    gaussians(static_cast<uint32_t>(o.ids[i]), st, o.k0, o.k1, g);
    const double s = std::sqrt(2.0 * o.D[o.types[i]] * dt);
    for (int k = 0; k < 3; ++k) {
      delta[3 * i + k] = s * g[k];
      o.pos[3 * i + k] = wrap(o.pos[3 * i + k] + delta[3 * i + k], o.L);
    }
  }
  int64_t n_events = 0;
  if (!free_jump && n_live >= 2 && !o.rx.empty()) {
    std::vector<double> rc2(o.rx.size()), ddt(o.rx.size());
    double rmax = 0.0;
    for (size_t q = 0; q < o.rx.size(); ++q) {
      const double rc = o.rx[q].R + o.c * std::sqrt(2.0 * o.rx[q].D_AB * dt);
      rc2[q] = rc * rc;
      ddt[q] = o.rx[q].D_AB * dt;
      rmax = std::max(rmax, rc);
    }
    // candidates: reacting type pairs closer than their cutoff, accepted against the
    // pair's uniform
    std::vector<Cand> acc;
    near_pairs(o.pos, o.L, rmax * (1.0 + 1e-9) + 1e-9, [&](size_t i, size_t j) {
      const int r = o.pair_rxn[o.types[i] * o.n_types + o.types[j]];
      if (r < 0) return;
      const size_t lo = o.ids[i] < o.ids[j] ? i : j, hi = o.ids[i] < o.ids[j] ? j : i;
      Cand cd{lo, hi, r, 0.0, {0.0, 0.0, 0.0}};
      for (int a = 0; a < 3; ++a) cd.r1[a] = min_image(o.pos[3 * hi + a] - o.pos[3 * lo + a], o.L);
      cd.d1sq = sq_norm(cd.r1[0], cd.r1[1], cd.r1[2]);
      if (!(cd.d1sq < rc2[r])) return;
      double r0[3];
      for (int a = 0; a < 3; ++a) r0[a] = cd.r1[a] - (delta[3 * hi + a] - delta[3 * lo + a]);
      const double d0 = std::sqrt(sq_norm(r0[0], r0[1], r0[2]));
      const double p = touch_probability(d0, std::sqrt(cd.d1sq), o.rx[r].R, ddt[r]);
      const double u = acceptance_uniform(static_cast<uint32_t>(o.ids[lo]), static_cast<uint32_t>(o.ids[hi]), st,
                                          o.k0, o.k1);
      if (u < p) acc.push_back(cd);
    });
    std::vector<int64_t> a_lo(acc.size()), a_hi(acc.size());
    std::vector<double> a_d(acc.size());
    for (size_t k = 0; k < acc.size(); ++k) {
      a_lo[k] = o.ids[acc[k].lo];
      a_hi[k] = o.ids[acc[k].hi];
      a_d[k] = acc[k].d1sq;
    }
    std::vector<size_t> kept = greedy_matching(a_lo, a_hi, a_d);
    std::sort(kept.begin(), kept.end(), [&](size_t x, size_t y) { return a_lo[x] < a_lo[y]; });
    std::vector<char> taken(n_live, 0);
    std::vector<int64_t> new_ids;
    std::vector<int> new_types;
    std::vector<double> new_pos;
    for (size_t k : kept) {
      const Cand& cd = acc[k];
      const Rxn& x = o.rx[cd.r];
      taken[cd.lo] = taken[cd.hi] = 1;
      const int ta = o.types[cd.lo], tb = o.types[cd.hi];
      const double w = o.D[ta] / (o.D[ta] + o.D[tb]);
      double P[3];
      for (int a = 0; a < 3; ++a) P[a] = wrap(o.pos[3 * cd.lo + a] + w * cd.r1[a], o.L);
      const int64_t first = o.next_id;
      for (int q = 0; q < x.n_prod; ++q) {
        new_ids.push_back(o.next_id++);
        new_types.push_back(x.prod[q]);
        for (int a = 0; a < 3; ++a) new_pos.push_back(P[a]);
      }
      o.water += x.water;
      o.events_total[cd.r] += 1;
      if (o.record) {
        const int64_t ev[6] = {o.step, cd.r, o.ids[cd.lo], o.ids[cd.hi], first, x.n_prod};
        o.event_log.insert(o.event_log.end(), ev, ev + 6);
      }
    }
    n_events = static_cast<int64_t>(kept.size());
    if (n_events) {
      std::vector<int64_t> ids2;
      std::vector<int> types2;
      std::vector<double> pos2;
      for (size_t i = 0; i < n_live; ++i) {
        if (taken[i]) continue;
        ids2.push_back(o.ids[i]);
        types2.push_back(o.types[i]);
        for (int a = 0; a < 3; ++a) pos2.push_back(o.pos[3 * i + a]);
      }
      ids2.insert(ids2.end(), new_ids.begin(), new_ids.end());
      types2.insert(types2.end(), new_types.begin(), new_types.end());
      pos2.insert(pos2.end(), new_pos.begin(), new_pos.end());
      o.ids.swap(ids2);
      o.types.swap(types2);
      o.pos.swap(pos2);
    }
  }
  if (o.record) {
    o.step_log.push_back(o.step);
    o.step_log.push_back(static_cast<int64_t>(n_live));
    o.step_log.push_back(n_events);
    std::vector<int64_t> cnt(o.n_types, 0);
    for (int ty : o.types) ++cnt[ty];
    o.step_log.insert(o.step_log.end(), cnt.begin(), cnt.end());
    o.step_times.push_back(o.t);
    o.step_times.push_back(dt);
  }
  o.t = t_next;
  o.step += 1;
  o.dt_cur = std::min(o.dt_cur * o.dt_growth, o.dt_max);
}

}  // namespace

extern "C" {

struct OracleReaction {
  int32_t a, b;
  double k_tab;
  int32_t n_prod;
  int32_t prod[3];
  int32_t water_delta;
};

// A new train, or null when a reaction is malformed (bad type, a second reaction for one
// type pair, more than 3 products) or a radius does not fit the box (R >= L/3).
void* oracle_new(int32_t n_types, const double* D, int32_t n_rxn, const OracleReaction* rx, double L, uint64_t seed,
                 uint32_t train_id, double dt_min, double dt_max, double dt_growth, int32_t reset_on_release,
                 double cutoff_c, double sbs_horizon, int32_t record) {
  Oracle* o = new Oracle();
  o->n_types = n_types;
  o->D.assign(D, D + n_types);
  o->pair_rxn.assign(static_cast<size_t>(n_types) * n_types, -1);
  o->L = L;
  o->dt_min = dt_min;
  o->dt_max = dt_max;
  o->dt_growth = dt_growth;
  o->reset_on_release = reset_on_release != 0;
  o->record = record != 0;
  o->c = cutoff_c;
  o->horizon = sbs_horizon;
  o->k0 = static_cast<uint32_t>(seed & 0xFFFFFFFFull);
  o->k1 = static_cast<uint32_t>(seed >> 32) ^ train_id;
  o->dt_L = std::numeric_limits<double>::infinity();
  for (int r = 0; r < n_rxn; ++r) {
    Rxn x;
    x.a = rx[r].a;
    x.b = rx[r].b;
    x.k_tab = rx[r].k_tab;
    x.n_prod = rx[r].n_prod;
    x.water = rx[r].water_delta;
    bool ok = x.a >= 0 && x.a < n_types && x.b >= 0 && x.b < n_types && x.n_prod >= 0 && x.n_prod <= 3;
    for (int q = 0; ok && q < x.n_prod; ++q) ok = rx[r].prod[q] >= 0 && rx[r].prod[q] < n_types;
    if (ok) ok = o->pair_rxn[x.a * n_types + x.b] < 0;
    if (!ok) {
      delete o;
      return nullptr;
    }
    for (int q = 0; q < 3; ++q) x.prod[q] = q < x.n_prod ? rx[r].prod[q] : -1;
    x.D_AB = o->D[x.a] + o->D[x.b];
    x.R = reaction_radius(x.k_tab, x.D_AB);
    o->pair_rxn[x.a * n_types + x.b] = o->pair_rxn[x.b * n_types + x.a] = r;
    // largest dt whose cutoff R + c sqrt(2 D_AB dt) stays <= L/3 (Eq. 2 stays unambiguous)
    const double room = L / 3.0 - x.R;
    if (room <= 0.0) {
      delete o;
      return nullptr;
    }
    if (cutoff_c > 0.0) o->dt_L = std::min(o->dt_L, (room / cutoff_c) * (room / cutoff_c) / (2.0 * x.D_AB));
    o->rx.push_back(x);
  }
  o->dt_cur = dt_min;
  o->events_total.assign(o->rx.size(), 0);
  return o;
}

void oracle_free(void* h) { delete static_cast<Oracle*>(h); }

// Queue species, merged stably by arrival after those already pending. Returns 0, or -1
// (nothing queued) for an arrival before the current time or not a number, a bad type or
// a position outside [-L/2, L/2).
int32_t oracle_inject(void* h, int64_t n, const int32_t* type, const double* xyz, const double* t_arr,
                      double energy_eV) {
  Oracle& o = *static_cast<Oracle*>(h);
  for (int64_t i = 0; i < n; ++i) {
    if (!(t_arr[i] >= o.t) || type[i] < 0 || type[i] >= o.n_types) return -1;  // NaN too
    for (int a = 0; a < 3; ++a)
      if (!(xyz[3 * i + a] >= -0.5 * o.L && xyz[3 * i + a] < 0.5 * o.L)) return -1;
  }
  o.E_dep += energy_eV;
  const size_t m = o.p_t.size();
  std::vector<double> t_all(o.p_t);
  t_all.insert(t_all.end(), t_arr, t_arr + n);
  std::vector<size_t> order(t_all.size());
  std::iota(order.begin(), order.end(), size_t(0));
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return t_all[a] < t_all[b]; });
  std::vector<double> nt, np;
  std::vector<int> ny;
  for (size_t k : order) {
    nt.push_back(t_all[k]);
    ny.push_back(k < m ? o.p_types[k] : type[k - m]);
    for (int a = 0; a < 3; ++a) np.push_back(k < m ? o.p_pos[3 * k + a] : xyz[3 * (k - m) + a]);
  }
  o.p_t.swap(nt);
  o.p_types.swap(ny);
  o.p_pos.swap(np);
  return 0;
}

void oracle_step_once(void* h, double t_end) { step_once(*static_cast<Oracle*>(h), t_end); }

// Steps until t_end (at most max_steps when max_steps >= 0); returns the steps taken.
int64_t oracle_run_until(void* h, double t_end, int64_t max_steps) {
  Oracle& o = *static_cast<Oracle*>(h);
  int64_t n = 0;
  while (o.t < t_end && (max_steps < 0 || n < max_steps)) {
    step_once(o, t_end);
    ++n;
  }
  return n;
}

double oracle_time(void* h) { return static_cast<Oracle*>(h)->t; }
double oracle_energy(void* h) { return static_cast<Oracle*>(h)->E_dep; }
int64_t oracle_step_index(void* h) { return static_cast<Oracle*>(h)->step; }
int64_t oracle_species_steps(void* h) { return static_cast<Oracle*>(h)->species_steps; }
int64_t oracle_water(void* h) { return static_cast<Oracle*>(h)->water; }
int64_t oracle_n_live(void* h) { return static_cast<int64_t>(static_cast<Oracle*>(h)->ids.size()); }
int64_t oracle_n_pending(void* h) { return static_cast<int64_t>(static_cast<Oracle*>(h)->p_t.size()); }
int64_t oracle_n_events(void* h) { return static_cast<int64_t>(static_cast<Oracle*>(h)->event_log.size() / 6); }
int64_t oracle_n_steps(void* h) { return static_cast<int64_t>(static_cast<Oracle*>(h)->step_times.size() / 2); }

void oracle_counts(void* h, int64_t* counts) {
  const Oracle& o = *static_cast<Oracle*>(h);
  std::fill(counts, counts + o.n_types, int64_t(0));
  for (int ty : o.types) ++counts[ty];
}

void oracle_events_total(void* h, int64_t* out) {
  const Oracle& o = *static_cast<Oracle*>(h);
  std::copy(o.events_total.begin(), o.events_total.end(), out);
}

void oracle_events(void* h, int64_t* out) {
  const Oracle& o = *static_cast<Oracle*>(h);
  std::copy(o.event_log.begin(), o.event_log.end(), out);
}

void oracle_steps(void* h, int64_t* out, double* times) {
  const Oracle& o = *static_cast<Oracle*>(h);
  std::copy(o.step_log.begin(), o.step_log.end(), out);
  std::copy(o.step_times.begin(), o.step_times.end(), times);
}

void oracle_pending_types(void* h, int32_t* out) {
  const Oracle& o = *static_cast<Oracle*>(h);
  std::copy(o.p_types.begin(), o.p_types.end(), out);
}

// Live species sorted by id.
void oracle_state(void* h, int64_t* ids, int32_t* types, double* xyz) {
  const Oracle& o = *static_cast<Oracle*>(h);
  std::vector<size_t> order(o.ids.size());
  std::iota(order.begin(), order.end(), size_t(0));
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return o.ids[a] < o.ids[b]; });
  for (size_t k = 0; k < order.size(); ++k) {
    ids[k] = o.ids[order[k]];
    types[k] = o.types[order[k]];
    for (int a = 0; a < 3; ++a) xyz[3 * k + a] = o.pos[3 * order[k] + a];
  }
}

// ---- the building blocks, elementwise (for the pins)
void oracle_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  const Block w = philox(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
  std::memcpy(out, w.w, sizeof(w.w));
}

void oracle_uniforms(int64_t n, const uint32_t* hi, const uint32_t* lo, double* open0, double* closed0) {
  for (int64_t i = 0; i < n; ++i) {
    open0[i] = uniform_open0(hi[i], lo[i]);
    closed0[i] = uniform_closed0(hi[i], lo[i]);
  }
}

void oracle_gaussians(int64_t n, const int64_t* ids, int64_t step, uint32_t k0, uint32_t k1, double* out) {
  for (int64_t i = 0; i < n; ++i)
    gaussians(static_cast<uint32_t>(ids[i]), static_cast<uint32_t>(step), k0, k1, out + 3 * i);
}

void oracle_acceptance_uniform(int64_t n, const int64_t* id_lo, const int64_t* id_hi, int64_t step, uint32_t k0,
                               uint32_t k1, double* out) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = acceptance_uniform(static_cast<uint32_t>(id_lo[i]), static_cast<uint32_t>(id_hi[i]),
                                static_cast<uint32_t>(step), k0, k1);
}

void oracle_wrap(int64_t n, const double* x, double L, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = wrap(x[i], L);
}

void oracle_min_image(int64_t n, const double* dx, double L, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = min_image(dx[i], L);
}

void oracle_touch_probability(int64_t n, const double* d0, const double* d1, const double* R, double ddt,
                              double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = touch_probability(d0[i], d1[i], R[i], ddt);
}

double oracle_reaction_radius(double k_tab, double D_AB) { return reaction_radius(k_tab, D_AB); }

// Index pairs (i < j) of points at most r apart (minimum image); writes at most cap pairs
// and returns how many there are.
int64_t oracle_pairs_within(int64_t n, const double* xyz, double L, double r, int64_t* out, int64_t cap) {
  const std::vector<double> pos(xyz, xyz + 3 * n);
  int64_t m = 0;
  near_pairs(pos, L, r * (1.0 + 1e-9) + 1e-12, [&](size_t i, size_t j) {
    const double d2 = sq_norm(min_image(pos[3 * j] - pos[3 * i], L), min_image(pos[3 * j + 1] - pos[3 * i + 1], L),
                              min_image(pos[3 * j + 2] - pos[3 * i + 2], L));
    if (d2 > r * r) return;
    if (m < cap) {
      out[2 * m] = static_cast<int64_t>(std::min(i, j));
      out[2 * m + 1] = static_cast<int64_t>(std::max(i, j));
    }
    ++m;
  });
  return m;
}

// Indices of the pairs the greedy matching keeps, in matching order; returns their number.
int64_t oracle_greedy_matching(int64_t n, const int64_t* id_lo, const int64_t* id_hi, const double* d1sq,
                               int64_t* kept) {
  const std::vector<size_t> k =
      greedy_matching(std::vector<int64_t>(id_lo, id_lo + n), std::vector<int64_t>(id_hi, id_hi + n),
                      std::vector<double>(d1sq, d1sq + n));
  for (size_t i = 0; i < k.size(); ++i) kept[i] = static_cast<int64_t>(k[i]);
  return static_cast<int64_t>(k.size());
}

}  // extern "C"
