// Homogeneous (beam-off) stage of a pulse train, Sec. 2.3 of arxiv 2509.03313: between
// pulses, and after the last one, the species are followed as a well-mixed system by
// the rate equations of Table 1 (Eq. 3, Eq. 4) instead of particle by particle.
//
// For every train the host selected (Train::hx_sel):
//  1. k_hx_remove marks every particle of the train removed (the next sort drops it);
//  2. k_hx_integrate, one warp per train, takes the train's species counts n0 as
//     molecule numbers in the box volume V and integrates the reaction extents e_r
//     (events): n(e) = n0 + nu e, de_r/dt = kappa_r n_a n_b, kappa_r = k_r / (N_A V), and
//     (k_tab / 2) / (N_A V) for a self reaction whose tabulated value is 2k. This is Eq. 3
//     multiplied through by N_A V. The integrator is the extrapolated linearly implicit
//     Euler method (Deuflhard 1985; Hairer and Wanner, Solving ODEs II, Sec. IV.9) with
//     the harmonic substep sequence 1..6 (one lane per column) and an analytic
//     Jacobian: stiff rate equations
//     (R9 at 1.1e11 L/mol/s) over 10 s take a few hundred steps;
//  3. the extents are rounded to whole events without bias, E_r = floor(e_r) +
//     [u_r < frac(e_r)], u_r from Philox4x32-10 at counter (stage, r, 0, 4); while a
//     species count would be negative, the lowest-index reaction consuming the lowest
//     negative species gives back one event; counts, event tallies and the water balance
//     take the whole events, so charge and atoms stay exactly conserved;
//  4. the survivors wait in Train::mat_n / mat_cum until the train's next step, whose
//     release re-creates them at uniform positions (phase_diffuse).
#include "launch.h"
#include "sbs_device.cuh"

namespace chem {
namespace {

constexpr double HX_N_AVOGADRO = 6.02214076e23;
constexpr double HX_TWO_POW_M53 = 1.1102230246251565e-16;
constexpr int HX_K = 6;              // extrapolation columns, substep counts 1..HX_K
constexpr double HX_RTOL = 1e-12;    // per step, relative to the extent
constexpr double HX_ATOL = 1e-8;     // per step, events
constexpr int HX_MAX_STEPS = 200000;

__device__ __forceinline__ int status_of_hx(const Dev& d) {
  return *reinterpret_cast<volatile int*>(&d.g->status);
}

// Kinetics of one train in molecule numbers.
struct Kin {
  int nt, nr;
  int a[MAXR], b[MAXR];
  double kappa[MAXR];
  double nu[MAXT][MAXR];
  double n0[MAXT];
};

__device__ void hx_numbers(const Kin& k, const double* e, double* n) {
  for (int x = 0; x < k.nt; ++x) {
    double v = k.n0[x];
    for (int r = 0; r < k.nr; ++r) v += k.nu[x][r] * e[r];
    n[x] = v;
  }
}

__device__ void hx_rates(const Kin& k, const double* e, double* out) {
  double n[MAXT];
  hx_numbers(k, e, n);
  for (int r = 0; r < k.nr; ++r) out[r] = k.kappa[r] * n[k.a[r]] * n[k.b[r]];
}

// d rate_r / d e_s = kappa_r (n_b nu[a][s] + n_a nu[b][s]) (both terms for a self reaction)
__device__ void hx_jacobian(const Kin& k, const double* e, double (*J)[MAXR]) {
  double n[MAXT];
  hx_numbers(k, e, n);
  for (int r = 0; r < k.nr; ++r) {
    const int a = k.a[r], b = k.b[r];
    for (int s = 0; s < k.nr; ++s) J[r][s] = k.kappa[r] * (n[b] * k.nu[a][s] + n[a] * k.nu[b][s]);
  }
}

// In-place LU with partial pivoting of the nr x nr matrix M. False when singular.
__device__ bool hx_lu(double (*M)[MAXR], int* piv, int nr) {
  for (int c = 0; c < nr; ++c) {
    int p = c;
    double best = fabs(M[c][c]);
    for (int r = c + 1; r < nr; ++r) {
      if (fabs(M[r][c]) > best) { best = fabs(M[r][c]); p = r; }
    }
    if (!(best > 0.0)) return false;
    piv[c] = p;
    if (p != c) {
      for (int q = 0; q < nr; ++q) { const double t = M[c][q]; M[c][q] = M[p][q]; M[p][q] = t; }
    }
    const double inv = 1.0 / M[c][c];
    for (int r = c + 1; r < nr; ++r) {
      const double f = M[r][c] * inv;
      M[r][c] = f;
      for (int q = c + 1; q < nr; ++q) M[r][q] -= f * M[c][q];
    }
  }
  return true;
}

__device__ void hx_solve(const double (*M)[MAXR], const int* piv, int nr, double* x) {
  for (int c = 0; c < nr; ++c) {
    const int p = piv[c];
    if (p != c) { const double t = x[c]; x[c] = x[p]; x[p] = t; }
  }
  for (int r = 1; r < nr; ++r) {
    double v = x[r];
    for (int q = 0; q < r; ++q) v -= M[r][q] * x[q];
    x[r] = v;
  }
  for (int r = nr - 1; r >= 0; --r) {
    double v = x[r];
    for (int q = r + 1; q < nr; ++q) v -= M[r][q] * x[q];
    x[r] = v / M[r][r];
  }
}

// Per-warp shared memory of the integrator: the columns' end values and the step's result.
struct HxWarpSmem {
  double col[HX_K][MAXR];
  double y1[MAXR];
};

// One extrapolated step of length H from y0, taken by one warp (every lane calls it with
// the same y0 and H): lane j - 1 integrates H with j linearly implicit Euler substeps,
// (I - hJ) d = h f(y), y += d, with the Jacobian J of y0 (columns are independent, so the
// six run side by side); lane 0 then applies the Aitken-Neville table, which removes the
// error terms in h, h^2, ... (the method's expansion is in powers of h). Returns false
// (on every lane) when a column is singular or the result is not finite; else y1 and
// the scaled error estimate on every lane.
__device__ bool hx_step(const Kin& k, const double* y0, double H, double* y1, double* err, HxWarpSmem& sm,
                        int lane) {
  const int nr = k.nr;
  bool ok = true;
  if (lane < HX_K) {
    const int j = lane + 1;
    double J[MAXR][MAXR], M[MAXR][MAXR];
    double y[MAXR], f[MAXR];
    int piv[MAXR];
    hx_jacobian(k, y0, J);
    const double h = H / j;
    for (int r = 0; r < nr; ++r)
      for (int s = 0; s < nr; ++s) M[r][s] = (r == s ? 1.0 : 0.0) - h * J[r][s];
    ok = hx_lu(M, piv, nr);
    if (ok) {
      for (int r = 0; r < nr; ++r) y[r] = y0[r];
      for (int i = 0; i < j; ++i) {
        hx_rates(k, y, f);
        for (int r = 0; r < nr; ++r) f[r] *= h;
        hx_solve(M, piv, nr, f);
        for (int r = 0; r < nr; ++r) y[r] += f[r];
      }
      for (int r = 0; r < nr; ++r) sm.col[lane][r] = y[r];
    }
  }
  ok = __all_sync(0xffffffffu, ok);
  __syncwarp();
  if (!ok) return false;
  double e = 0.0;
  bool fin = true;
  if (lane == 0) {
    double prev[HX_K][MAXR], cur[HX_K][MAXR];
    for (int jj = 1; jj <= HX_K; ++jj) {
      for (int r = 0; r < nr; ++r) cur[0][r] = sm.col[jj - 1][r];
      for (int l = 0; l + 1 < jj; ++l) {
        const double den = static_cast<double>(jj) / static_cast<double>(jj - l - 1) - 1.0;
        for (int r = 0; r < nr; ++r) cur[l + 1][r] = cur[l][r] + (cur[l][r] - prev[l][r]) / den;
      }
      for (int l = 0; l < jj; ++l)
        for (int r = 0; r < nr; ++r) prev[l][r] = cur[l][r];
    }
    for (int r = 0; r < nr; ++r) {
      const double v = cur[HX_K - 1][r];
      fin = fin && isfinite(v);
      sm.y1[r] = v;
      const double sc = HX_ATOL + HX_RTOL * fmax(fabs(y0[r]), fabs(v));
      e = fmax(e, fabs(v - cur[HX_K - 2][r]) / sc);
    }
  }
  fin = __shfl_sync(0xffffffffu, fin, 0);
  e = __shfl_sync(0xffffffffu, e, 0);
  __syncwarp();
  if (!fin) return false;
  for (int r = 0; r < nr; ++r) y1[r] = sm.y1[r];
  __syncwarp();
  *err = e;
  return true;
}

// Extents after T seconds from e = 0, by one warp (identical control flow on every lane).
// Returns the accepted steps, or -1 on failure.
__device__ long long hx_integrate(const Kin& k, double T, double* e, HxWarpSmem& sm, int lane) {
  for (int r = 0; r < k.nr; ++r) e[r] = 0.0;
  if (k.nr == 0 || !(T > 0.0)) return 0;
  double t = 0.0, H = fmin(T, 1e-9);
  long long accepted = 0;
  double y1[MAXR];
  for (int it = 0; it < HX_MAX_STEPS; ++it) {
    if (t >= T) return accepted;
    const bool last = H >= T - t;
    const double Hs = last ? T - t : H;
    double err = 0.0;
    const bool ok = hx_step(k, e, Hs, y1, &err, sm, lane);
    if (ok && err <= 1.0) {
      for (int r = 0; r < k.nr; ++r) e[r] = y1[r];
      t = last ? T : t + Hs;
      ++accepted;
      const double fac = err > 0.0 ? 0.9 * pow(err, -1.0 / HX_K) : 4.0;
      H = Hs * fmin(4.0, fmax(0.2, fac));
    } else {
      const double fac = ok ? 0.9 * pow(err, -1.0 / HX_K) : 0.2;
      H = Hs * fmin(0.5, fmax(0.2, fac));
    }
  }
  return -1;
}

__global__ void k_hx_remove(Dev d) {
  if (status_of_hx(d)) return;
  const uint32_t n = d.g->n_total;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    if (d.dead[s]) continue;
    const int b = d.n_trains == 1 ? 0 : train_of_cell(d.trains, d.n_trains, d.cell_sorted[s]);
    if (d.trains[b].hx_sel) d.dead[s] = 1;
  }
}

constexpr int HX_WARPS = 2;  // trains per CTA, one warp each

__global__ void __launch_bounds__(32 * HX_WARPS) k_hx_integrate(Dev d) {
  __shared__ HxWarpSmem smem[HX_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t b = blockIdx.x * HX_WARPS + static_cast<uint32_t>(w);
  if (b >= d.n_trains || status_of_hx(d)) return;  // warp-uniform
  Train& tr = d.trains[b];
  if (!tr.hx_sel) return;
  const Tables& tb = *d.tables;
  Kin k;
  k.nt = tb.n_types;
  k.nr = tb.n_rxn;
  const double NV = HX_N_AVOGADRO * (tr.L * tr.L * tr.L * 1e-24);
  for (int x = 0; x < MAXT; ++x) {
    k.n0[x] = x < k.nt ? static_cast<double>(tr.counts[x]) : 0.0;
    for (int r = 0; r < MAXR; ++r) k.nu[x][r] = 0.0;
  }
  for (int r = 0; r < k.nr; ++r) {
    const int a = tb.rxn_a[r], c = tb.rxn_b[r];
    k.a[r] = a;
    k.b[r] = c;
    k.kappa[r] = (a == c ? 0.5 * tb.k_tab[r] : tb.k_tab[r]) / NV;
    k.nu[a][r] -= 1.0;
    k.nu[c][r] -= 1.0;
    for (int q = 0; q < tb.n_prod[r]; ++q) k.nu[tb.prod[r][q]][r] += 1.0;
  }
  double e[MAXR];
  const long long steps = hx_integrate(k, tr.hx_t_end - tr.t, e, smem[w], lane);
  if (lane != 0) return;  // the rounding and the train's record: one lane
  if (steps < 0) {
    raise_status(d.g, CHEM_ECAPACITY);
    d.g->err_where = 0x4858u;  // integrator step limit of the homogeneous stage
    tr.hx_sel = 0;
    return;
  }
  // whole events: unbiased rounding, then take-backs while a count is negative
  long long E[MAXR], n[MAXT];
  for (int r = 0; r < k.nr; ++r) {
    const uint4 w = philox4x32_10(make_uint4(tr.hx_stage, static_cast<uint32_t>(r), 0u, 4u), tr.key0, tr.key1);
    const double u = static_cast<double>(u53(w.x, w.y)) * HX_TWO_POW_M53;
    const double x = fmax(e[r], 0.0);
    const double fl = floor(x);
    E[r] = static_cast<long long>(fl) + (u < x - fl ? 1 : 0);
  }
  for (int x = 0; x < k.nt; ++x) {
    long long v = tr.counts[x];
    for (int r = 0; r < k.nr; ++r) v += static_cast<long long>(k.nu[x][r]) * E[r];
    n[x] = v;
  }
  for (;;) {
    int neg = -1;
    for (int x = 0; x < k.nt && neg < 0; ++x)
      if (n[x] < 0) neg = x;
    if (neg < 0) break;
    int rr = -1;
    for (int r = 0; r < k.nr && rr < 0; ++r)
      if (k.nu[neg][r] < 0.0 && E[r] > 0) rr = r;
    if (rr < 0) {  // cannot happen: a negative count always has a consuming event
      raise_status(d.g, CHEM_ECAPACITY);
      tr.hx_sel = 0;
      return;
    }
    E[rr] -= 1;
    for (int x = 0; x < k.nt; ++x) n[x] -= static_cast<long long>(k.nu[x][rr]);
  }
  long long water = 0;
  uint32_t cum = 0;
  for (int r = 0; r < MAXR; ++r) {
    tr.hx_e[r] = r < k.nr ? e[r] : 0.0;
    tr.hx_E[r] = r < k.nr ? E[r] : 0;
    if (r < k.nr) {
      tr.events[r] += E[r];
      water += E[r] * tb.water[r];
    }
  }
  for (int x = 0; x < MAXT; ++x) {
    const long long v = x < k.nt ? n[x] : 0;
    tr.counts[x] = v;
    cum += static_cast<uint32_t>(v);
    tr.mat_cum[x] = cum;
  }
  tr.water += water;
  tr.mat_n = cum;
  tr.hx_steps = steps;
  tr.hx_stage += 1;
  tr.t = tr.hx_t_end;
  tr.hx_sel = 0;
}

}  // namespace

cudaError_t enqueue_homogeneous(const Dev& d, int blocks, cudaStream_t s) {
  k_hx_remove<<<blocks, 256, 0, s>>>(d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_hx_integrate<<<(static_cast<int>(d.n_trains) + HX_WARPS - 1) / HX_WARPS, 32 * HX_WARPS, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace chem
