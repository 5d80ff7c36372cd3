// pdd_mlmc.cu -- multilevel Monte Carlo driver (host) over the path kernels.
//
// The paper names the multilevel variant of its Monte Carlo stage as future
// work (Sec. 1, Sec. 7).  Level 0 is Algorithm 1 at h_0; level l >= 1 is the
// difference of a fine path at h_l = h_0 / 2^l and a coarse path at h_(l-1)
// driven by the same Brownian increments (pdd_accumulate_coupled).  The
// sample counts follow the standard level-adaptive rule of multilevel Monte
// Carlo: the counts that minimise the total cost sum_l N_l C_l subject to
// sum_l V_l / N_l = eps^2 / 2 (Lagrange multipliers give
// N_l proportional to sqrt(V_l / C_l)), and levels are added until the
// finest correction, scaled by the weak order, is below eps / sqrt(2).  The
// finest pair also gives the Talay-Tubaro (Richardson) extrapolation.
//
// Every level accumulates exact integer node records, and extra paths of a
// level continue its path indices, so the result is the same function of
// the final counts N_l whatever the rounds that produced them.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

#include <vector>

#include "../../include/pdd.h"
#include "pdd_internal.h"

namespace pdd {
void set_error(const char* fmt, ...);
}

using namespace pdd;

namespace {

constexpr int kMaxRounds = 64;
constexpr int64_t kMaxPaths = 0xFFFFFFFFll;  // path indices stay below 2^32

struct DeviceSelect {
  int old = -1;
  explicit DeviceSelect(int d) {
    if (cudaGetDevice(&old) != cudaSuccess) old = -1;
    cudaSetDevice(d);
  }
  ~DeviceSelect() {
    if (old >= 0) cudaSetDevice(old);
  }
};

// Device allocations of one pdd_mlmc call, released on every exit.
struct Buffers {
  std::vector<void*> ptrs;
  ~Buffers() {
    for (void* q : ptrs) cudaFree(q);
  }
  template <class T>
  cudaError_t alloc(T** out, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e == cudaSuccess) ptrs.push_back(q);
    *out = (T*)q;
    return e;
  }
};

}  // namespace

extern "C" {

int pdd_mlmc_allocate(int n_levels, const double* V, const double* C, double eps, int64_t* N) {
  if (n_levels < 1 || n_levels > PDD_MLMC_MAX_LEVELS || !V || !C || !N) {
    set_error("pdd_mlmc_allocate: n_levels = %d outside [1, %d] or NULL array", n_levels,
              PDD_MLMC_MAX_LEVELS);
    return PDD_ERR_INVALID;
  }
  if (!(eps > 0.0) || !isfinite(eps)) {
    set_error("pdd_mlmc_allocate: target_rmse must be finite and > 0");
    return PDD_ERR_INVALID;
  }
  double s = 0.0;
  for (int l = 0; l < n_levels; ++l) {
    if (!(V[l] >= 0.0) || !isfinite(V[l]) || !(C[l] > 0.0) || !isfinite(C[l])) {
      set_error("pdd_mlmc_allocate: level %d needs V >= 0 and C > 0 (finite)", l);
      return PDD_ERR_INVALID;
    }
    s += sqrt(V[l] * C[l]);
  }
  int rc = PDD_OK;
  for (int l = 0; l < n_levels; ++l) {
    double x = ceil(2.0 / (eps * eps) * sqrt(V[l] / C[l]) * s);
    if (x < 1.0) x = 1.0;
    if (x > (double)kMaxPaths) {
      x = (double)kMaxPaths;
      rc = PDD_WARN_NOT_CONVERGED;
    }
    N[l] = (int64_t)x;
  }
  if (rc != PDD_OK) set_error("pdd_mlmc_allocate: counts clamped to 2^32 - 1 paths");
  return rc;
}

int pdd_mlmc(pdd_problem* p, const pdd_mlmc_args* a, pdd_mlmc_out* out) {
  const char* who = "pdd_mlmc";
  if (!p || !a || !out) {
    set_error("%s: NULL argument", who);
    return PDD_ERR_INVALID;
  }
  ProblemView pv;
  if (!problem_view(p, &pv)) {
    set_error("%s: bad problem", who);
    return PDD_ERR_INVALID;
  }
  const int64_t n = a->n_nodes;
  if (n < 1 || n >= ((int64_t)1 << 32)) {
    set_error("%s: n_nodes = %lld outside [1, 2^32)", who, (long long)n);
    return PDD_ERR_INVALID;
  }
  for (int j = 0; j < pv.dim; ++j)
    if (!a->coords[j]) {
      set_error("%s: coords[%d] is NULL", who, j);
      return PDD_ERR_INVALID;
    }
  if (a->min_levels < 2 || a->max_levels < a->min_levels ||
      a->max_levels > PDD_MLMC_MAX_LEVELS) {
    set_error("%s: need 2 <= min_levels (%d) <= max_levels (%d) <= %d", who, a->min_levels,
              a->max_levels, PDD_MLMC_MAX_LEVELS);
    return PDD_ERR_INVALID;
  }
  if (!(a->dt0 > 0.0) || !isfinite(a->dt0) || !(a->target_rmse > 0.0) ||
      !isfinite(a->target_rmse) || !(a->alpha > 0.0) || !isfinite(a->alpha)) {
    set_error("%s: dt0, target_rmse and alpha must be finite and > 0", who);
    return PDD_ERR_INVALID;
  }
  if (a->n_pilot < 2 || a->n_pilot > kMaxPaths) {
    set_error("%s: n_pilot = %lld outside [2, 2^32)", who, (long long)a->n_pilot);
    return PDD_ERR_INVALID;
  }
  const int max_l = a->max_levels;
  const bool controlled = a->grid_id != PDD_CV_NONE;
  const double eps = a->target_rmse, r2 = pow(2.0, a->alpha);
  DeviceSelect dsel(pv.device);
  (void)cudaGetLastError();
  const size_t rec_bytes = (size_t)n * kAccWords * 8;
  Buffers buf;
  std::vector<unsigned long long*> fine(max_l, nullptr), diff(max_l, nullptr);
  double* scratch = nullptr;  // mean, var, steps of one record array
  if (buf.alloc(&scratch, 3 * (size_t)n * sizeof(double)) != cudaSuccess) {
    set_error("%s: device allocation failed", who);
    return PDD_ERR_NOMEM;
  }
  auto add_level = [&](int l) -> int {
    if (buf.alloc(&fine[l], rec_bytes) != cudaSuccess ||
        (l > 0 && buf.alloc(&diff[l], rec_bytes) != cudaSuccess)) {
      set_error("%s: device allocation failed (level %d)", who, l);
      return PDD_ERR_NOMEM;
    }
    cudaError_t e = cudaMemsetAsync(fine[l], 0, rec_bytes, pv.stream);
    if (e == cudaSuccess && l > 0) e = cudaMemsetAsync(diff[l], 0, rec_bytes, pv.stream);
    if (e != cudaSuccess) {
      set_error("%s: %s", who, cudaGetErrorString(e));
      return PDD_ERR_CUDA;
    }
    return PDD_OK;
  };
  // mean and variance of the level's score and the mean exit index of one
  // record array, on the host
  std::vector<double> hm(n), hv(n), hs(n);
  auto moments = [&](const unsigned long long* rec) -> int {
    StatPtrs sp{};
    if (controlled) {
      sp.mean_cv = scratch;
      sp.var_cv = scratch + n;
    } else {
      sp.mean_phi = scratch;
      sp.var_phi = scratch + n;
    }
    sp.mean_steps = scratch + 2 * n;
    cudaError_t e = launch_finalize(rec, (uint32_t)n, 1.0, sp, pv.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hm.data(), scratch, n * sizeof(double), cudaMemcpyDeviceToHost,
                          pv.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hv.data(), scratch + n, n * sizeof(double), cudaMemcpyDeviceToHost,
                          pv.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hs.data(), scratch + 2 * n, n * sizeof(double),
                          cudaMemcpyDeviceToHost, pv.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pv.stream);
    if (e != cudaSuccess) {
      set_error("%s: %s", who, cudaGetErrorString(e));
      return PDD_ERR_CUDA;
    }
    return PDD_OK;
  };

  std::vector<int64_t> N(max_l, 0), dN(max_l, 0), Ns(max_l, 0);
  std::vector<std::vector<double>> m(max_l), v(max_l);
  std::vector<double> Vb(max_l, 0.0), Cb(max_l, 0.0), Rl(max_l, 0.0), steps(max_l, 0.0);
  int L = a->min_levels - 1;
  for (int l = 0; l <= L; ++l) {
    int rc = add_level(l);
    if (rc != PDD_OK) return rc;
    dN[l] = a->n_pilot;
  }
  bool converged = false, truncated = false, clamped = false;
  double bias = NAN;
  int rounds = 0;
  while (rounds < kMaxRounds) {
    ++rounds;
    // 1. the missing paths of every level
    for (int l = 0; l <= L; ++l) {
      if (dN[l] == 0) continue;
      pdd_estimate_args e{};
      e.n_nodes = n;
      for (int j = 0; j < 3; ++j) e.coords[j] = a->coords[j];
      e.coords_on_device = 1;
      e.grid_id = a->grid_id;
      e.n_paths = dN[l];
      e.dt = l == 0 ? a->dt0 : a->dt0 / ldexp(1.0, l - 1);
      e.kappa = 1.0;
      e.seed = a->seed;
      e.stream_tag = a->stream_tag_base + (uint32_t)l;
      const int rc = l == 0 ? pdd_accumulate(p, &e, (uint64_t)N[l], (uint64_t*)fine[0])
                            : pdd_accumulate_coupled(p, &e, (uint64_t)N[l], (uint64_t*)fine[l],
                                                     (uint64_t*)diff[l]);
      if (rc == PDD_WARN_TRUNCATED) truncated = true;
      else if (rc != PDD_OK) return rc;
      N[l] += dN[l];
      dN[l] = 0;
    }
    // 2. per-node level means, variances and costs from the records
    for (int l = 0; l <= L; ++l) {
      int rc = moments(l == 0 ? fine[0] : diff[l]);
      if (rc != PDD_OK) return rc;
      m[l] = hm;
      v[l] = hv;
      std::vector<double> cost = hs;  // level 0: its steps; l >= 1: coarse steps
      if (l > 0) {
        rc = moments(fine[l]);
        if (rc != PDD_OK) return rc;
        for (int64_t i = 0; i < n; ++i) cost[i] += hs[i];
      }
      double sv = 0, sc = 0, sm2 = 0;
      for (int64_t i = 0; i < n; ++i) {
        sv += v[l][i];
        sc += cost[i];
        sm2 += m[l][i] * m[l][i];
      }
      Vb[l] = sv / (double)n;
      steps[l] = sc;
      Cb[l] = fmax(sc / (double)n, 1.0);  // a path costs at least its start
      Rl[l] = sqrt(fmax(0.0, sm2 / (double)n - Vb[l] / (double)N[l]));
    }
    // 3. counts for a node-mean variance eps^2 / 2
    const int arc = pdd_mlmc_allocate(L + 1, Vb.data(), Cb.data(), eps, Ns.data());
    if (arc < 0) return arc;
    if (arc == PDD_WARN_NOT_CONVERGED) clamped = true;
    bool more = false;
    for (int l = 0; l <= L; ++l)
      if (Ns[l] > N[l]) {
        dN[l] = Ns[l] - N[l];
        more = true;
      }
    if (more) continue;
    // 4. bias test on the finest corrections; add a level if it fails (with
    // min_levels == max_levels the levels are fixed and the test only reported)
    bias = fmax(Rl[L], Rl[L - 1] / r2) / (r2 - 1.0);
    if (bias <= eps / sqrt(2.0) || a->min_levels == a->max_levels) {
      converged = !clamped;
      break;
    }
    if (L + 1 >= max_l) break;
    L += 1;
    int rc = add_level(L);
    if (rc != PDD_OK) return rc;
    dN[L] = a->n_pilot;
    // the new level's statistics enter at the next round
  }
  // a new level added in the last allowed round has no paths yet: leave it out
  while (L > 0 && N[L] == 0) L -= 1;

  const double f_ext = 1.0 / (r2 - 1.0), g_ext = r2 / (r2 - 1.0);
  for (int64_t i = 0; i < n; ++i) {
    double est = 0.0, var = 0.0;
    for (int l = 0; l <= L; ++l) {
      est += m[l][i];
      var += v[l][i] / (double)N[l];
    }
    if (out->estimate) out->estimate[i] = est;
    if (out->variance) out->variance[i] = var;
    if (out->extrapolated) out->extrapolated[i] = est + f_ext * m[L][i];
    if (out->extrap_variance)
      out->extrap_variance[i] = var - v[L][i] / (double)N[L] + g_ext * g_ext * v[L][i] / (double)N[L];
  }
  out->n_levels = L + 1;
  out->rounds = rounds;
  double total = 0.0;
  for (int l = 0; l < PDD_MLMC_MAX_LEVELS; ++l) {
    const bool used = l <= L;
    out->n_paths[l] = used ? N[l] : 0;
    out->var_mean[l] = used ? Vb[l] : 0.0;
    out->cost_mean[l] = used ? Cb[l] : 0.0;
    out->corr_rms[l] = used ? Rl[l] : 0.0;
    if (used) total += steps[l] * (double)N[l];
  }
  out->bias_estimate = bias;
  out->path_steps = (int64_t)llround(total);
  if (!converged) {
    set_error("%s: stopping test not met (bias estimate %.3g, %d levels, %d rounds%s)", who, bias,
              L + 1, rounds, clamped ? ", counts clamped at 2^32 - 1" : "");
    return PDD_WARN_NOT_CONVERGED;
  }
  if (truncated) {
    set_error("%s: some paths hit max_steps", who);
    return PDD_WARN_TRUNCATED;
  }
  return PDD_OK;
}

}  // extern "C"
