// pdd_api.cu -- host runtime and C ABI of libpdd.so (declared in
// include/pdd.h): contexts, problems, control grids and the synchronous /
// stream-ordered estimate of the Monte Carlo nodal stage (Bernal & Acebron,
// Algorithm 1 and Sec. 2.2-3.1).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pdd.h"
#include "pdd_internal.h"

namespace pdd {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

// Makes `dev` current for the lifetime of the guard.  cudaSetDevice is called
// even when `dev` is already the current device: it (re)binds the device's
// primary context to the calling thread, which other libraries in the process
// may have changed.  A stale error left by an unchecked earlier call is
// cleared so that it cannot be reported against this call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
    (void)cudaGetLastError();
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

static int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: CUDA error %d (%s)", what, (int)e, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PDD_ERR_NOMEM : PDD_ERR_CUDA;
}

#define PDD_CUDA(call, what)                 \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace pdd

using namespace pdd;

struct pdd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  int num_sms = 0;
  void* ws = nullptr;  // workspace: header | node records | coords | staged outputs
  size_t ws_size = 0;
  std::mutex mu;
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  int64_t launches = 0;
};

struct GridSlot {
  int n = 0;
  void* table = nullptr;  // float2 / float4 gradient table
};

struct pdd_problem {
  pdd_ctx* ctx = nullptr;
  pdd_problem_desc desc{};
  int dim = 2;
  GridSlot grids[PDD_MAX_GRIDS];
};

// Workspace header (first 256 bytes).
struct WsHeader {
  unsigned long long cursor;
  unsigned err;
  unsigned pad;
  unsigned long long trunc_total;
};

namespace pdd {
// Read-only view of a problem and its context for other translation units of
// the library (the allocation-free entry point).
bool problem_view(pdd_problem* p, ProblemView* v) {
  if (!p || !p->ctx || !v) return false;
  v->device = p->ctx->device;
  v->stream = p->ctx->stream;
  v->num_sms = p->ctx->num_sms;
  v->kind = p->desc.kind;
  v->precision = p->desc.precision;
  v->exit_rule = p->desc.exit_rule;
  v->y_rule = p->desc.y_rule;
  v->max_steps = p->desc.max_steps;
  v->dim = p->dim;
  for (int i = 0; i < PDD_MAX_GRIDS; ++i) {
    v->grid_table[i] = p->grids[i].table;
    v->grid_n[i] = p->grids[i].n;
  }
  v->mu = &p->ctx->mu;
  v->launches = &p->ctx->launches;
  return true;
}
}  // namespace pdd

static int ensure_workspace(pdd_ctx* c, size_t bytes) {
  if (c->ws_size >= bytes) return PDD_OK;
  if (c->budget != 0 && bytes > c->budget) {
    set_error("workspace of %zu bytes exceeds the context budget of %zu bytes", bytes, c->budget);
    return PDD_ERR_NOMEM;
  }
  PDD_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (c->ws) {
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_size = 0;
  }
  size_t want = bytes + bytes / 2;
  if (c->budget != 0 && want > c->budget) want = c->budget;
  PDD_CUDA(cudaMalloc(&c->ws, want), "cudaMalloc(workspace)");
  c->ws_size = want;
  return PDD_OK;
}

extern "C" {

int pdd_abi_version(void) { return PDD_ABI_VERSION; }

const char* pdd_last_error(void) { return g_last_error.c_str(); }

int pdd_ctx_create(int device, void* cuda_stream, size_t mem_budget, pdd_ctx** out) {
  if (!out) {
    set_error("pdd_ctx_create: out is NULL");
    return PDD_ERR_INVALID;
  }
  *out = nullptr;
  int ndev = 0;
  PDD_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) {
    set_error("pdd_ctx_create: device %d out of range (%d devices)", device, ndev);
    return PDD_ERR_INVALID;
  }
  DeviceGuard g(device);
  if (!g.ok) {
    set_error("pdd_ctx_create: cannot select device %d", device);
    return PDD_ERR_CUDA;
  }
  int sms = 0;
  PDD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device),
           "cudaDeviceGetAttribute");
  pdd_ctx* c = new pdd_ctx();
  c->device = device;
  c->budget = mem_budget;
  c->num_sms = sms;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "cudaStreamCreate");
    }
    c->own_stream = true;
  }
  *out = c;
  return PDD_OK;
}

void pdd_ctx_destroy(pdd_ctx* c) {
  if (!c) return;
  {
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& ev : c->events) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
    if (c->ws) cudaFree(c->ws);
    if (c->own_stream) cudaStreamDestroy(c->stream);
  }
  delete c;
}

int pdd_ctx_set_stream(pdd_ctx* c, void* cuda_stream) {
  if (!c) {
    set_error("pdd_ctx_set_stream: NULL context");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  PDD_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (c->own_stream) {
    cudaStreamDestroy(c->stream);
    c->own_stream = false;
  }
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    PDD_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    c->own_stream = true;
  }
  return PDD_OK;
}

int pdd_ctx_set_timing(pdd_ctx* c, int enable) {
  if (!c) {
    set_error("pdd_ctx_set_timing: NULL context");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->timing = enable != 0;
  return PDD_OK;
}

int pdd_ctx_kernel_time(pdd_ctx* c, double* total_ms, int64_t* launches, double* per_launch_ms,
                        int64_t capacity) {
  if (!c || !total_ms) {
    set_error("pdd_ctx_kernel_time: NULL argument");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  double tot = 0.0;
  int64_t n = 0;
  int rc = PDD_OK;
  for (auto& ev : c->events) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(ev.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.first, ev.second);
    if (e != cudaSuccess && rc == PDD_OK) rc = cuda_fail(e, "cudaEventElapsedTime");
    tot += ms;
    if (per_launch_ms && n < capacity) per_launch_ms[n] = ms;
    ++n;
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  c->events.clear();
  *total_ms = tot;
  if (launches) *launches = n;
  return rc;
}

int pdd_ctx_launch_count(pdd_ctx* c, int64_t* launches) {
  if (!c || !launches) {
    set_error("pdd_ctx_launch_count: NULL argument");
    return PDD_ERR_INVALID;
  }
  *launches = c->launches;
  return PDD_OK;
}

int pdd_create_problem(pdd_ctx* c, const pdd_problem_desc* d, pdd_problem** out) {
  if (!c || !d || !out) {
    set_error("pdd_create_problem: NULL argument");
    return PDD_ERR_INVALID;
  }
  *out = nullptr;
  if (d->kind < PDD_PROBLEM_CFG0_2D || d->kind > PDD_PROBLEM_HARMONIC_2D) {
    set_error("pdd_create_problem: unknown problem kind %d", d->kind);
    return PDD_ERR_INVALID;
  }
  if (d->exit_rule != PDD_EXIT_GOBET_MENOZZI && d->exit_rule != PDD_EXIT_NAIVE) {
    set_error("pdd_create_problem: unknown exit rule %d", d->exit_rule);
    return PDD_ERR_INVALID;
  }
  if (d->y_rule != PDD_Y_EULER && d->y_rule != PDD_Y_EXP) {
    set_error("pdd_create_problem: unknown Y rule %d", d->y_rule);
    return PDD_ERR_INVALID;
  }
  if (d->precision != PDD_PATH_FP32 && d->precision != PDD_PATH_FP64) {
    set_error("pdd_create_problem: unknown precision %d", d->precision);
    return PDD_ERR_INVALID;
  }
  pdd_problem* p = new pdd_problem();
  p->ctx = c;
  p->desc = *d;
  p->dim = d->kind == PDD_PROBLEM_CUBE_3D ? 3 : 2;
  *out = p;
  return PDD_OK;
}

int pdd_destroy_problem(pdd_problem* p) {
  if (!p) return PDD_OK;
  pdd_ctx* c = p->ctx;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& s : p->grids)
      if (s.table) cudaFree(s.table);
  }
  delete p;
  return PDD_OK;
}

int pdd_set_control_grid(pdd_problem* p, int grid_id, const pdd_grid_desc* d) {
  if (!p || !d || !d->data) {
    set_error("pdd_set_control_grid: NULL argument");
    return PDD_ERR_INVALID;
  }
  if (grid_id < 0 || grid_id >= PDD_MAX_GRIDS) {
    set_error("pdd_set_control_grid: grid_id %d outside [0, %d)", grid_id, PDD_MAX_GRIDS);
    return PDD_ERR_INVALID;
  }
  const int dim = p->dim;
  const int nmax = dim == 2 ? 4097 : 513;
  if (d->n < 3 || d->n > nmax) {
    set_error("pdd_set_control_grid: n = %d outside [3, %d]", d->n, nmax);
    return PDD_ERR_INVALID;
  }
  if ((d->kind != PDD_GRID_VALUES && d->kind != PDD_GRID_GRADIENT) ||
      (d->dtype != PDD_DTYPE_F32 && d->dtype != PDD_DTYPE_F64)) {
    set_error("pdd_set_control_grid: bad kind %d or dtype %d", d->kind, d->dtype);
    return PDD_ERR_INVALID;
  }
  pdd_ctx* c = p->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  const size_t npts = dim == 2 ? (size_t)d->n * d->n : (size_t)d->n * d->n * d->n;
  const size_t comps = d->kind == PDD_GRID_VALUES ? 1 : (size_t)dim;
  const size_t count = npts * comps;
  const size_t elt = d->dtype == PDD_DTYPE_F32 ? 4 : 8;
  // stage the input as FP64 on the device
  double* staged = nullptr;
  PDD_CUDA(cudaMalloc(&staged, count * sizeof(double)), "cudaMalloc(grid staging)");
  cudaError_t e = cudaSuccess;
  if (d->dtype == PDD_DTYPE_F64) {
    e = cudaMemcpyAsync(staged, d->data, count * elt,
                        d->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->stream);
  } else if (d->on_device) {
    e = launch_f32_to_f64((const float*)d->data, staged, count, c->stream);
    c->launches += 1;
  } else {
    std::vector<double> tmp(count);
    const float* src = (const float*)d->data;
    for (size_t i = 0; i < count; ++i) tmp[i] = (double)src[i];
    e = cudaMemcpyAsync(staged, tmp.data(), count * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  void* table = nullptr;
  const size_t tbytes = npts * (dim == 2 ? sizeof(float2) : sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&table, tbytes);
  if (e == cudaSuccess) {
    e = d->kind == PDD_GRID_VALUES ? launch_grid_gradient(staged, d->n, dim, table, c->stream)
                                   : launch_grid_pack(staged, d->n, dim, table, c->stream);
    c->launches += 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(staged);
  if (e != cudaSuccess) {
    if (table) cudaFree(table);
    return cuda_fail(e, "pdd_set_control_grid");
  }
  GridSlot& s = p->grids[grid_id];
  if (s.table) cudaFree(s.table);  // the stream was drained above
  s.table = table;
  s.n = d->n;
  return PDD_OK;
}

int pdd_estimate_nodes(pdd_problem* p, const pdd_estimate_args* a, pdd_node_stats* out) {
  if (!p || !a || !out) {
    set_error("pdd_estimate_nodes: NULL argument");
    return PDD_ERR_INVALID;
  }
  const int dim = p->dim;
  if (a->n_nodes < 0 || a->n_nodes >= (int64_t)1 << 32) {
    set_error("pdd_estimate_nodes: n_nodes = %lld outside [0, 2^32)", (long long)a->n_nodes);
    return PDD_ERR_INVALID;
  }
  if (a->n_paths < 1 || a->n_paths >= (int64_t)1 << 32) {
    set_error("pdd_estimate_nodes: n_paths = %lld outside [1, 2^32)", (long long)a->n_paths);
    return PDD_ERR_INVALID;
  }
  if (!(a->dt > 0.0) || !std::isfinite(a->dt)) {
    set_error("pdd_estimate_nodes: dt must be finite and > 0");
    return PDD_ERR_INVALID;
  }
  if ((unsigned long long)a->n_nodes * (unsigned long long)a->n_paths >= (1ull << 62)) {
    set_error("pdd_estimate_nodes: n_nodes * n_paths too large");
    return PDD_ERR_INVALID;
  }
  const bool emit = (a->flags & PDD_FLAG_EMIT_PATHS) != 0;
  const bool async = (a->flags & PDD_FLAG_ASYNC) != 0;
  if (a->flags & ~(PDD_FLAG_EMIT_PATHS | PDD_FLAG_ASYNC)) {
    set_error("pdd_estimate_nodes: unknown flags 0x%x", a->flags);
    return PDD_ERR_INVALID;
  }
  if (emit && (!a->path_phi || !a->path_xi || !a->path_steps)) {
    set_error("pdd_estimate_nodes: EMIT_PATHS needs path_phi, path_xi and path_steps");
    return PDD_ERR_INVALID;
  }
  if (async && (!a->coords_on_device || !out->on_device)) {
    set_error("pdd_estimate_nodes: PDD_FLAG_ASYNC needs device coordinates and outputs");
    return PDD_ERR_INVALID;
  }
  int cv = 0;  // kernel CV mode: 0 none, 1 grid, 2 exact
  const void* table = nullptr;
  int grid_n = 0;
  if (a->grid_id == PDD_CV_NONE) {
    cv = 0;
  } else if (a->grid_id == PDD_CV_EXACT) {
    cv = 2;
  } else if (a->grid_id >= 0 && a->grid_id < PDD_MAX_GRIDS && p->grids[a->grid_id].table) {
    cv = 1;
    table = p->grids[a->grid_id].table;
    grid_n = p->grids[a->grid_id].n;
  } else {
    set_error("pdd_estimate_nodes: grid_id %d is not a loaded grid", a->grid_id);
    return PDD_ERR_INVALID;
  }
  if (a->n_nodes == 0) return PDD_OK;
  for (int j = 0; j < dim; ++j)
    if (!a->coords[j]) {
      set_error("pdd_estimate_nodes: coords[%d] is NULL", j);
      return PDD_ERR_INVALID;
    }
  int64_t max_steps = p->desc.max_steps;
  if (max_steps <= 0) {
    const double ms = std::ceil(100.0 / a->dt);
    max_steps = ms > 2.0e9 ? 2000000000ll : (int64_t)ms;
  }
  if (max_steps > 2000000000ll) max_steps = 2000000000ll;

  pdd_ctx* c = p->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  if (!g.ok) {
    set_error("pdd_estimate_nodes: cannot select device %d", c->device);
    return PDD_ERR_CUDA;
  }
  const size_t n = (size_t)a->n_nodes;
  // workspace layout
  const size_t off_acc = 256;
  const size_t off_coords = align_up(off_acc + n * kAccWords * 8, 256);
  const size_t coords_bytes = a->coords_on_device ? 0 : align_up(n * 4, 256) * dim;
  const size_t off_out = off_coords + coords_bytes;
  const size_t out_bytes = out->on_device ? 0 : 14 * align_up(n * 8, 256);
  int rc = ensure_workspace(c, off_out + out_bytes);
  if (rc != PDD_OK) return rc;
  char* ws = (char*)c->ws;
  WsHeader* hdr = (WsHeader*)ws;
  unsigned long long* acc = (unsigned long long*)(ws + off_acc);
  PDD_CUDA(cudaMemsetAsync(ws, 0, off_acc + n * kAccWords * 8, c->stream), "cudaMemsetAsync");
  const float* coords[3] = {a->coords[0], a->coords[1], dim == 3 ? a->coords[2] : nullptr};
  if (!a->coords_on_device) {
    for (int j = 0; j < dim; ++j) {
      float* dst = (float*)(ws + off_coords + j * align_up(n * 4, 256));
      PDD_CUDA(cudaMemcpyAsync(dst, a->coords[j], n * 4, cudaMemcpyHostToDevice, c->stream),
               "cudaMemcpyAsync(coords)");
      coords[j] = dst;
    }
  }
  PathArgs pa{};
  pa.cx = coords[0];
  pa.cy = coords[1];
  pa.cz = coords[2] ? coords[2] : coords[0];
  pa.total = (unsigned long long)n * (unsigned long long)a->n_paths;
  pa.n_paths = (unsigned long long)a->n_paths;
  pa.cursor = &hdr->cursor;
  pa.acc = acc;
  pa.err = &hdr->err;
  pa.trunc_total = &hdr->trunc_total;
  pa.emit_phi = emit ? a->path_phi : nullptr;
  pa.emit_xi = emit ? a->path_xi : nullptr;
  pa.emit_steps = emit ? a->path_steps : nullptr;
  pa.grad = table;
  pa.grid_n = grid_n;
  pa.max_steps = (int)max_steps;
  pa.y_exp = p->desc.y_rule == PDD_Y_EXP;
  pa.max_blocks = 0;
  pa.h = a->dt;
  pa.sqrt_h = std::sqrt(a->dt);
  const double c0 = p->desc.exit_rule == PDD_EXIT_GOBET_MENOZZI ? 0.5826 : 0.0;
  pa.thr0 = c0 * pa.sqrt_h;
  pa.key0 = (uint32_t)a->seed;
  pa.key1 = a->stream_tag;
  pa.seed_hi = (uint32_t)(a->seed >> 32);

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (c->timing) {
    PDD_CUDA(cudaEventCreate(&ev0), "cudaEventCreate");
    PDD_CUDA(cudaEventCreate(&ev1), "cudaEventCreate");
    PDD_CUDA(cudaEventRecord(ev0, c->stream), "cudaEventRecord");
  }
  int blocks = 0;
  PDD_CUDA(launch_paths(p->desc.kind, p->desc.precision, cv, pa, c->num_sms, c->stream, &blocks),
           "path kernel launch");
  c->launches += 1;
  if (c->timing) {
    PDD_CUDA(cudaEventRecord(ev1, c->stream), "cudaEventRecord");
    c->events.emplace_back(ev0, ev1);
  }
  StatPtrs sp{};
  double* dptr[12];
  unsigned long long* uptr[2];
  double* const* user_d[12] = {&out->mean_phi, &out->var_phi, &out->mean_cv, &out->var_cv,
                               &out->cov_phi_xi, &out->var_xi, &out->rho, &out->se_phi,
                               &out->se_cv, &out->vr, &out->pred_speedup, &out->mean_steps};
  uint64_t* const* user_u[2] = {&out->n_paths, &out->n_truncated};
  for (int i = 0; i < 12; ++i) {
    dptr[i] = *user_d[i];
    if (!out->on_device && dptr[i]) dptr[i] = (double*)(ws + off_out + i * align_up(n * 8, 256));
  }
  for (int i = 0; i < 2; ++i) {
    uptr[i] = (unsigned long long*)*user_u[i];
    if (!out->on_device && uptr[i])
      uptr[i] = (unsigned long long*)(ws + off_out + (12 + i) * align_up(n * 8, 256));
  }
  sp.mean_phi = dptr[0];
  sp.var_phi = dptr[1];
  sp.mean_cv = dptr[2];
  sp.var_cv = dptr[3];
  sp.cov_phi_xi = dptr[4];
  sp.var_xi = dptr[5];
  sp.rho = dptr[6];
  sp.se_phi = dptr[7];
  sp.se_cv = dptr[8];
  sp.vr = dptr[9];
  sp.pred_speedup = dptr[10];
  sp.mean_steps = dptr[11];
  sp.n_paths = uptr[0];
  sp.n_truncated = uptr[1];
  const double kappa = a->kappa > 0.0 ? a->kappa : 1.0;
  PDD_CUDA(launch_finalize(acc, (uint32_t)n, kappa, sp, c->stream), "finalize launch");
  c->launches += 1;
  if (!out->on_device) {
    for (int i = 0; i < 12; ++i)
      if (*user_d[i])
        PDD_CUDA(cudaMemcpyAsync(*user_d[i], dptr[i], n * 8, cudaMemcpyDeviceToHost, c->stream),
                 "cudaMemcpyAsync(outputs)");
    for (int i = 0; i < 2; ++i)
      if (*user_u[i])
        PDD_CUDA(cudaMemcpyAsync(*user_u[i], uptr[i], n * 8, cudaMemcpyDeviceToHost, c->stream),
                 "cudaMemcpyAsync(outputs)");
  }
  if (async) return PDD_OK;
  WsHeader h{};
  PDD_CUDA(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, c->stream),
           "cudaMemcpyAsync(header)");
  PDD_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (h.err & kErrOverflow) {
    set_error("pdd_estimate_nodes: a score left the fixed-point range |score| < 32768");
    return PDD_ERR_OVERFLOW;
  }
  if (h.cursor < pa.total) {
    set_error("pdd_estimate_nodes: internal error, %llu of %llu paths scheduled", h.cursor,
              pa.total);
    return PDD_ERR_CUDA;
  }
  if (h.trunc_total > 0) {
    set_error("pdd_estimate_nodes: %llu paths hit max_steps = %lld", h.trunc_total,
              (long long)max_steps);
    return PDD_WARN_TRUNCATED;
  }
  return PDD_OK;
}

}  // extern "C"
