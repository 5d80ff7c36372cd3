// pdd_fit.cu -- fast fit of nodal constants (Bernal & Acebron, Sec. 5 H5 and
// Algorithm 3): all (node, h) pairs of an h-cloud run as levels of the
// persistent path kernel; the per-node fits are small host-side regressions.
//   first moments: E[eta_h] = E[eta_0] + B h^delta, normal noise and identity
//     link, i.e. ordinary least squares in x = h^delta;
//   variances: E[V[eta_h]] = V[eta_0] + B h^delta, gamma noise and identity
//     link, i.e. iteratively reweighted least squares with weights 1/mu^2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/pdd.h"
#include "pdd_internal.h"

namespace pdd {
void set_error(const char* fmt, ...);
}

using namespace pdd;

namespace {

// y = a + b x by ordinary least squares.
void ols(const std::vector<double>& x, const std::vector<double>& y, double* a, double* b) {
  const size_t m = x.size();
  double mx = 0, my = 0;
  for (size_t j = 0; j < m; ++j) {
    mx += x[j];
    my += y[j];
  }
  mx /= (double)m;
  my /= (double)m;
  double sxy = 0, sxx = 0;
  for (size_t j = 0; j < m; ++j) {
    sxy += (x[j] - mx) * (y[j] - my);
    sxx += (x[j] - mx) * (x[j] - mx);
  }
  *b = sxx > 0 ? sxy / sxx : 0.0;
  *a = my - *b * mx;
}

// mu = a + b x for gamma-distributed y (variance proportional to mu^2), identity
// link: weighted least squares with weights 1/mu^2 from the previous fit until
// the coefficients settle (Fisher scoring for this model).
void gamma_identity(const std::vector<double>& x, const std::vector<double>& y, double* a,
                    double* b) {
  ols(x, y, a, b);
  const size_t m = x.size();
  double ymin = 1e300;
  for (double v : y) ymin = std::min(ymin, std::fabs(v));
  const double floor_mu = std::max(ymin * 1e-6, 1e-300);
  for (int it = 0; it < 200; ++it) {
    double sw = 0, swx = 0, swy = 0, swxx = 0, swxy = 0;
    for (size_t j = 0; j < m; ++j) {
      const double mu = std::max(*a + *b * x[j], floor_mu);
      const double w = 1.0 / (mu * mu);
      sw += w;
      swx += w * x[j];
      swy += w * y[j];
      swxx += w * x[j] * x[j];
      swxy += w * x[j] * y[j];
    }
    const double det = sw * swxx - swx * swx;
    if (!(det > 0)) break;
    const double nb = (sw * swxy - swx * swy) / det;
    const double na = (swy - nb * swx) / sw;
    const double change = std::fabs(na - *a) + std::fabs(nb - *b);
    *a = na;
    *b = nb;
    if (change <= 1e-14 * (std::fabs(na) + std::fabs(nb) + 1e-300)) break;
  }
}

}  // namespace

extern "C" int pdd_fit_constants(pdd_problem* p, const pdd_fit_args* a, pdd_fit_out* out) {
  ProblemView pv;
  if (!p || !a || !out || !problem_view(p, &pv)) {
    set_error("pdd_fit_constants: NULL argument");
    return PDD_ERR_INVALID;
  }
  if (a->n_nodes < 1 || a->n_nodes >= ((int64_t)1 << 31) || a->n_h < 2 || a->n_h > 4096 ||
      !(a->h_min > 0) || !(a->h_max > a->h_min) || !std::isfinite(a->h_max) || a->n_paths < 2 ||
      !(a->delta > 0) || !(a->q > 0)) {
    set_error("pdd_fit_constants: bad arguments (need n_nodes >= 1, 2 <= n_h <= 4096, "
              "0 < h_min < h_max, n_paths >= 2, delta > 0, q > 0)");
    return PDD_ERR_INVALID;
  }
  for (int j = 0; j < pv.dim; ++j)
    if (!a->coords[j]) {
      set_error("pdd_fit_constants: coords[%d] is NULL", j);
      return PDD_ERR_INVALID;
    }
  const bool with_psi = a->grid_id != PDD_CV_NONE;
  const size_t n = (size_t)a->n_nodes, M = (size_t)a->n_h;
  // per (h, field, node) device statistics: mean_phi, var_phi, mean_steps, cov, var_xi
  const int kF = 5;
  DeviceGuard guard(pv.device);  // restores the caller's device on return
  if (!guard.ok) {
    set_error("pdd_fit_constants: cannot select device %d", pv.device);
    return PDD_ERR_CUDA;
  }
  double* dstat = nullptr;
  cudaError_t e = cudaMalloc(&dstat, M * kF * n * sizeof(double));
  if (e != cudaSuccess) {
    set_error("pdd_fit_constants: cudaMalloc: %s", cudaGetErrorString(e));
    return PDD_ERR_NOMEM;
  }
  std::vector<double> hs(M);
  for (size_t j = 0; j < M; ++j)
    hs[j] = a->h_max - (a->h_max - a->h_min) * (double)j / (double)(M - 1);
  int rc = PDD_OK;
  for (size_t j0 = 0; j0 < M && rc >= 0; j0 += PDD_MAX_LEVELS) {
    const size_t nl = std::min<size_t>(PDD_MAX_LEVELS, M - j0);
    std::vector<pdd_estimate_args> lv(nl);
    std::vector<pdd_node_stats> os(nl);
    for (size_t l = 0; l < nl; ++l) {
      const size_t j = j0 + l;
      pdd_estimate_args& x = lv[l];
      x = pdd_estimate_args{};
      x.n_nodes = a->n_nodes;
      for (int d = 0; d < 3; ++d) x.coords[d] = a->coords[d];
      x.coords_on_device = 1;
      x.grid_id = a->grid_id;
      x.n_paths = a->n_paths;
      x.dt = hs[j];
      x.kappa = 1.0;
      x.seed = a->seed;
      x.stream_tag = a->stream_tag_base + (uint32_t)j;
      pdd_node_stats& o = os[l];
      o = pdd_node_stats{};
      o.on_device = 1;
      double* base = dstat + j * kF * n;
      o.mean_phi = base;
      o.var_phi = base + n;
      o.mean_steps = base + 2 * n;
      o.cov_phi_xi = base + 3 * n;
      o.var_xi = base + 4 * n;
    }
    rc = pdd_estimate_levels(p, (int)nl, lv.data(), os.data(), 0);
  }
  std::vector<double> hstat(M * kF * n);
  if (rc >= 0) {
    e = cudaMemcpy(hstat.data(), dstat, hstat.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      set_error("pdd_fit_constants: cudaMemcpy: %s", cudaGetErrorString(e));
      rc = PDD_ERR_CUDA;
    }
  }
  cudaFree(dstat);
  if (rc < 0) return rc;
  std::vector<double> x(M), y(M);
  for (size_t j = 0; j < M; ++j) x[j] = std::pow(hs[j], a->delta);
  auto stat = [&](size_t j, int f, size_t i) { return hstat[(j * kF + f) * n + i]; };
  for (size_t i = 0; i < n; ++i) {
    // A node whose paths all leave at k = 0 at some time step of the cloud
    // (mean exit index exactly 0, so phi is deterministic there: the node lies
    // inside the shrinkage layer c0 sqrt(h) of the boundary) is outside the
    // model E[eta_h] = E[eta_0] + B h^delta the fits assume: its constants are
    // NaN and the schedule leaves it out.
    bool degenerate = false;
    for (size_t j = 0; j < M; ++j) degenerate |= !(stat(j, 2, i) > 0.0);
    if (degenerate) {
      double* const outs[9] = {out->E_phi, out->beta, out->V_phi, out->alpha, out->E_tau,
                               out->K, out->cov_phi_psi, out->V_psi, out->rho_phi_psi};
      for (double* o : outs)
        if (o) o[i] = NAN;
    }
    double e_phi, beta, v_phi, alpha, e_tau, slope, cov0 = NAN, v_psi = NAN;
    for (size_t j = 0; j < M; ++j) y[j] = stat(j, 0, i);
    ols(x, y, &e_phi, &beta);
    for (size_t j = 0; j < M; ++j) y[j] = stat(j, 2, i) * hs[j];  // tau_h = k h
    ols(x, y, &e_tau, &slope);
    for (size_t j = 0; j < M; ++j) y[j] = stat(j, 1, i);
    gamma_identity(x, y, &v_phi, &alpha);
    if (with_psi) {
      for (size_t j = 0; j < M; ++j) y[j] = stat(j, 3, i);  // E[psi phi] = Cov (E psi = 0)
      ols(x, y, &cov0, &slope);
      for (size_t j = 0; j < M; ++j) y[j] = stat(j, 4, i);
      gamma_identity(x, y, &v_psi, &slope);
    }
    const double K = 4.0 * a->q * a->q * e_tau * std::pow(2.0 * std::fabs(beta), 1.0 / a->delta);
    if (!degenerate) {
      if (out->E_phi) out->E_phi[i] = e_phi;
      if (out->beta) out->beta[i] = beta;
      if (out->V_phi) out->V_phi[i] = v_phi;
      if (out->alpha) out->alpha[i] = alpha;
      if (out->E_tau) out->E_tau[i] = e_tau;
      if (out->K) out->K[i] = K;
      if (out->cov_phi_psi) out->cov_phi_psi[i] = cov0;
      if (out->V_psi) out->V_psi[i] = v_psi;
      if (out->rho_phi_psi) out->rho_phi_psi[i] = cov0 / std::sqrt(v_phi * v_psi);
    }
    if (out->cloud)
      for (size_t j = 0; j < M; ++j) {
        double* c = out->cloud + (i * M + j) * 6;
        c[0] = hs[j];
        c[1] = stat(j, 0, i);
        c[2] = stat(j, 1, i);
        c[3] = stat(j, 2, i) * hs[j];
        c[4] = stat(j, 3, i);
        c[5] = stat(j, 4, i);
      }
  }
  return rc;
}

// ---------------------------------------------------------------------------
// Algorithm 4: scheduling of the tolerance sequence a_J > ... > a_1 > a_0.
// ---------------------------------------------------------------------------
namespace {

struct SchedData {
  const pdd_schedule_args* a;
  double p;  // 2 + 1/delta
};

// Nodes the schedule uses: finite fitted constants, V[phi] > 0 and beta != 0
// (a node Algorithm 3 could not fit has NaN constants and is left out).
bool usable(const pdd_schedule_args& s, int64_t i) {
  return std::isfinite(s.K[i]) && std::isfinite(s.beta[i]) && std::isfinite(s.alpha[i]) &&
         std::isfinite(s.V_phi[i]) && std::isfinite(s.V_psi[i]) &&
         std::isfinite(s.rho_phi_psi[i]) && s.V_phi[i] > 0.0 && s.beta[i] != 0.0;
}

// Predicted cost of the level with tolerance aj using the control variate of
// the coarser level with tolerance a (the minimised objective of Algorithm 4).
double sched_cost(const SchedData& d, double a, double aj) {
  const pdd_schedule_args& s = *d.a;
  double tot = 0.0;
  for (int64_t i = 0; i < s.n_nodes; ++i) {
    if (!usable(s, i)) continue;
    double r2 = 1.0 - s.V_psi[i] * a * a * (1.0 - s.rho_phi_psi[i] * s.rho_phi_psi[i]) /
                          (4.0 * s.V_phi[i]);
    if (r2 < 0.0) r2 = 0.0;
    const double r = std::sqrt(r2);
    const double vr = 1.0 - r2 + std::fabs(s.alpha[i] * r / s.beta[i]) * aj;
    tot += s.K[i] * s.V_phi[i] * (s.kappa * vr + std::pow(aj / a, d.p));
  }
  return tot;
}

}  // namespace

extern "C" int pdd_schedule(const pdd_schedule_args* s, double* a, double* speedup,
                            int max_levels, int* n_levels) {
  if (!s || !a || !n_levels || max_levels < 1 || s->n_nodes < 1 || !s->K || !s->beta ||
      !s->alpha || !s->V_phi || !s->V_psi || !s->rho_phi_psi || !(s->delta > 0) ||
      !(s->kappa > 0) || !(s->a0 > 0)) {
    set_error("pdd_schedule: bad arguments");
    return PDD_ERR_INVALID;
  }
  SchedData d{s, 2.0 + 1.0 / s->delta};
  double plain = 0.0, amax = 0.0;
  int64_t n_usable = 0;
  for (int64_t i = 0; i < s->n_nodes; ++i) {
    if (!usable(*s, i)) continue;
    ++n_usable;
    plain += s->K[i] * s->V_phi[i];
    const double c = s->V_psi[i] * (1.0 - s->rho_phi_psi[i] * s->rho_phi_psi[i]) /
                     (4.0 * s->V_phi[i]);
    if (c > 0) amax = std::max(amax, 1.0 / std::sqrt(c));
  }
  if (n_usable == 0) {
    set_error("pdd_schedule: no node has usable fitted constants");
    return PDD_ERR_INVALID;
  }
  const double min_s = s->min_speedup > 0 ? s->min_speedup : 1.5;
  a[0] = s->a0;
  int J = 0;
  double aj = s->a0;
  if (speedup)
    for (int k = 0; k <= max_levels; ++k) speedup[k] = NAN;  // steps not taken
  while (J < max_levels && aj < amax) {
    // log-spaced scan of (aj, amax], then golden-section refinement
    const int kScan = 2000;
    const double l0 = std::log(aj), l1 = std::log(amax);
    int best = 1;
    double bestv = 1e300;
    for (int k = 1; k <= kScan; ++k) {
      const double v = sched_cost(d, std::exp(l0 + (l1 - l0) * k / kScan), aj);
      if (v < bestv) {
        bestv = v;
        best = k;
      }
    }
    double lo = l0 + (l1 - l0) * (best - 1) / kScan, hi = l0 + (l1 - l0) * std::min(best + 1, kScan) / kScan;
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    double f1 = sched_cost(d, std::exp(x1), aj), f2 = sched_cost(d, std::exp(x2), aj);
    for (int it = 0; it < 200 && hi - lo > 1e-14; ++it) {
      if (f1 < f2) {
        hi = x2;
        x2 = x1;
        f2 = f1;
        x1 = hi - g * (hi - lo);
        f1 = sched_cost(d, std::exp(x1), aj);
      } else {
        lo = x1;
        x1 = x2;
        f1 = f2;
        x2 = lo + g * (hi - lo);
        f2 = sched_cost(d, std::exp(x2), aj);
      }
    }
    const double xbest = f1 < f2 ? x1 : x2;
    const double fbest = std::min(f1, f2);
    const double S = plain / std::min(fbest, bestv);
    const double anext = fbest <= bestv ? std::exp(xbest) : std::exp(l0 + (l1 - l0) * best / kScan);
    if (speedup) speedup[J] = S;
    if (S < min_s) break;
    a[++J] = anext;
    aj = anext;
  }
  *n_levels = J;
  return PDD_OK;
}

// ---------------------------------------------------------------------------
// Balanced simulation per node (Definition "Balanced MC simulation",
// eq. F:N_y_h) and the scheduling model's per-level prediction (Algorithm 4,
// eq. F:Sensitivity_formula), used to run the levels Algorithm 4 schedules
// (Algorithm 5: "for node x_i and a_j, determine h and N").
// ---------------------------------------------------------------------------
extern "C" int pdd_balanced_plan(int64_t n_nodes, double a, double q, double delta,
                                 const double* beta, const double* var, double h_min,
                                 double h_max, int64_t n_min, int64_t n_max, double* h,
                                 int64_t* n_paths) {
  if (n_nodes < 0 || !(a > 0) || !std::isfinite(a) || !(q > 0) || !(delta > 0) ||
      !(h_min > 0) || !(h_max >= h_min) || !std::isfinite(h_max) || n_min < 1 ||
      n_max < n_min || (n_nodes > 0 && (!beta || !var || !h || !n_paths))) {
    set_error("pdd_balanced_plan: bad arguments (need a, q, delta > 0, 0 < h_min <= h_max, "
              "1 <= n_min <= n_max, non-NULL arrays)");
    return PDD_ERR_INVALID;
  }
  for (int64_t i = 0; i < n_nodes; ++i) {
    // bias |beta| h^delta = a / 2 and statistical error q sqrt(V / N) = a / 2
    const double b = std::fabs(beta[i]);
    double hi = b > 0 ? std::pow(a / (2.0 * b), 1.0 / delta) : h_max;
    if (!(hi >= h_min)) hi = h_min;  // also catches NaN
    if (hi > h_max) hi = h_max;
    h[i] = hi;
    const double v = var[i] > 0 ? var[i] : 0.0;
    const double nn = std::ceil(4.0 * q * q * v / (a * a));
    int64_t ni = nn >= (double)n_max || !std::isfinite(nn) ? n_max : (int64_t)nn;
    if (ni < n_min) ni = n_min;
    n_paths[i] = ni;
  }
  return PDD_OK;
}

extern "C" int pdd_schedule_predict(const pdd_schedule_args* s, double a, double aj, double* rho2,
                                    double* cost) {
  if (!s || s->n_nodes < 1 || !s->K || !s->beta || !s->alpha || !s->V_phi || !s->V_psi ||
      !s->rho_phi_psi || !(s->delta > 0) || !(aj > 0) || !rho2 || !cost) {
    set_error("pdd_schedule_predict: bad arguments");
    return PDD_ERR_INVALID;
  }
  const double p = 2.0 + 1.0 / s->delta;
  const double scale = std::pow(aj, -p);
  for (int64_t i = 0; i < s->n_nodes; ++i) {
    const double base = s->K[i] * s->V_phi[i] * scale;  // plain cost at aj (eq. F:Pointwise_cost)
    if (!(a > 0)) {
      rho2[i] = 0.0;
      cost[i] = base;
      continue;
    }
    double r2 = 1.0 - s->V_psi[i] * a * a * (1.0 - s->rho_phi_psi[i] * s->rho_phi_psi[i]) /
                          (4.0 * s->V_phi[i]);
    if (r2 < 0.0) r2 = 0.0;
    const double r = std::sqrt(r2);
    const double loss = std::fabs(s->alpha[i] * r / s->beta[i]) * aj;
    rho2[i] = std::max(r2 - loss, 0.0);
    cost[i] = base * (1.0 - r2 + loss);
  }
  return PDD_OK;
}
