// pdd_api.cu -- host runtime and C ABI of libpdd.so (declared in
// include/pdd.h): contexts, problems, control grids and the synchronous /
// stream-ordered estimate of the Monte Carlo nodal stage (Bernal & Acebron,
// Algorithm 1 and Sec. 2.2-3.1).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pdd.h"
#include "pdd_device.cuh"
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

int error_word_status(unsigned err, const char* who) {
  if (err & kErrBoundsAll) {
    set_error("%s: bounds check failed (error bits 0x%x:%s%s%s%s%s)", who, err,
              (err & kErrBoundsGrid) ? " grid cell" : "",
              (err & kErrBoundsIndex) ? " path index" : "",
              (err & kErrBoundsRecord) ? " node record" : "",
              (err & kErrBoundsRing) ? " exit ring" : "",
              (err & kErrBoundsEmit) ? " per-path output" : "");
    return PDD_ERR_BOUNDS;
  }
  if (err & kErrOverflow) {
    set_error("%s: a score left the fixed-point range |score| < 32768", who);
    return PDD_ERR_OVERFLOW;
  }
  return PDD_OK;
}

static int aborted_status(const char* who) {
  set_error("%s: aborted by pdd_ctx_abort; the results hold the paths that ran (n_paths per "
            "node)", who);
  return PDD_ERR_CANCELLED;
}

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
  int block_threads = 0;  // launch shape (0: defaults), set by pdd_ctx_set_launch / pdd_autotune
  int max_blocks = 0;
  int iter_mode = PDD_ITER_AUTO;  // steps per iteration (pdd_ctx_set_iteration / pdd_autotune)
  int claim = 0;  // paths per lane per cursor claim, 0 = automatic (pdd_ctx_set_claim)
  cudaGraphExec_t gexec = nullptr;  // cached graph of the last PDD_FLAG_GRAPH call
  uint64_t gkey = 0;
  int64_t graph_captures = 0;
  // pdd_ctx_abort: copies into the workspace header on a stream of its own
  // (created at the first abort), ordered before the next call's header reset
  std::mutex abort_mu;  // held while the workspace is replaced and while an abort is enqueued
  cudaStream_t abort_stream = nullptr;
  cudaEvent_t abort_ev = nullptr;
  unsigned long long* abort_src = nullptr;  // page-locked: {cursor past any launch, flag}
  std::atomic<bool> abort_pending{false};
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

// Workspace header (first 256 bytes).  pdd_ctx_abort writes a cursor past
// any launch's paths (so no warp takes another batch) and sets `aborted`.
struct WsHeader {
  unsigned long long cursor;
  unsigned err;
  unsigned aborted;
  unsigned long long trunc_total;
};
static_assert(offsetof(WsHeader, aborted) == 12, "abort flag offset");

// Orders the context stream after an abort enqueued since its last call, so
// that the abort's copies land before this call resets the header.
static void wait_abort(pdd_ctx* c) {
  if (c->abort_pending.exchange(false)) cudaStreamWaitEvent(c->stream, c->abort_ev, 0);
}

namespace pdd {
// Device, SM count and launch shape of a context, for the serving runtime.
bool ctx_view(pdd_ctx* c, int* device, int* num_sms, int* block_threads, int* max_blocks) {
  if (!c) return false;
  *device = c->device;
  *num_sms = c->num_sms;
  *block_threads = c->block_threads;
  *max_blocks = c->max_blocks;
  return true;
}
pdd_ctx* problem_ctx(pdd_problem* p) { return p ? p->ctx : nullptr; }
int ctx_iter_mode(pdd_ctx* c) { return c ? c->iter_mode : PDD_ITER_AUTO; }
int ctx_claim(pdd_ctx* c) { return c ? c->claim : 0; }
}  // namespace pdd

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
  // no abort copy may still target the buffer about to be freed
  std::lock_guard<std::mutex> ak(c->abort_mu);
  if (c->abort_stream) PDD_CUDA(cudaStreamSynchronize(c->abort_stream), "cudaStreamSynchronize");
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


// ---------------------------------------------------------------------------
// Estimation of one or several levels in one persistent launch.
// ---------------------------------------------------------------------------
namespace {

struct LevelPlan {
  int cv;              // 0 none, 1 grid, 2 exact
  const void* table;
  int grid_n;
  int64_t max_steps;
};

int check_level(const pdd_problem* p, const pdd_estimate_args* a, const pdd_node_stats* out,
                const char* who, int l, LevelPlan* lp) {
  const int dim = p->dim;
  if (a->n_nodes < 0 || a->n_nodes >= (int64_t)1 << 32) {
    set_error("%s: level %d: n_nodes = %lld outside [0, 2^32)", who, l, (long long)a->n_nodes);
    return PDD_ERR_INVALID;
  }
  if (a->n_paths < 1 || a->n_paths >= (int64_t)1 << 32) {
    set_error("%s: level %d: n_paths = %lld outside [1, 2^32)", who, l, (long long)a->n_paths);
    return PDD_ERR_INVALID;
  }
  if (!(a->dt > 0.0) || !std::isfinite(a->dt)) {
    set_error("%s: level %d: dt must be finite and > 0", who, l);
    return PDD_ERR_INVALID;
  }
  if ((unsigned long long)a->n_nodes * (unsigned long long)a->n_paths >= (1ull << 62)) {
    set_error("%s: level %d: n_nodes * n_paths too large", who, l);
    return PDD_ERR_INVALID;
  }
  if (a->flags & ~(PDD_FLAG_EMIT_PATHS | PDD_FLAG_ASYNC)) {
    set_error("%s: level %d: unknown flags 0x%x", who, l, a->flags);
    return PDD_ERR_INVALID;
  }
  if ((a->flags & PDD_FLAG_EMIT_PATHS) && (!a->path_phi || !a->path_xi || !a->path_steps)) {
    set_error("%s: level %d: EMIT_PATHS needs path_phi, path_xi and path_steps", who, l);
    return PDD_ERR_INVALID;
  }
  if (a->grid_id == PDD_CV_NONE) {
    lp->cv = 0;
    lp->table = nullptr;
    lp->grid_n = 0;
  } else if (a->grid_id == PDD_CV_EXACT) {
    lp->cv = 2;
    lp->table = nullptr;
    lp->grid_n = 0;
  } else if (a->grid_id >= 0 && a->grid_id < PDD_MAX_GRIDS && p->grids[a->grid_id].table) {
    lp->cv = 1;
    lp->table = p->grids[a->grid_id].table;
    lp->grid_n = p->grids[a->grid_id].n;
  } else {
    set_error("%s: level %d: grid_id %d is not a loaded grid", who, l, a->grid_id);
    return PDD_ERR_INVALID;
  }
  if (a->n_nodes > 0)
    for (int j = 0; j < dim; ++j)
      if (!a->coords[j]) {
        set_error("%s: level %d: coords[%d] is NULL", who, l, j);
        return PDD_ERR_INVALID;
      }
  (void)out;
  int64_t max_steps = p->desc.max_steps;
  if (max_steps <= 0) {
    const double ms = std::ceil(100.0 / a->dt);
    max_steps = ms > 2.0e9 ? 2000000000ll : (int64_t)ms;
  }
  if (max_steps > 2000000000ll) max_steps = 2000000000ll;
  lp->max_steps = max_steps;
  return PDD_OK;
}

uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* b = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

static int query_occupancy(pdd_problem* p, int grid_id, int threads, int* occ) {
  const int cv = grid_id == PDD_CV_NONE ? 0 : (grid_id == PDD_CV_EXACT ? 2 : 1);
  *occ = 0;
  cudaError_t e = occupancy_paths(p->desc.kind, p->desc.precision, cv, false, threads, occ);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  return PDD_OK;
}

static int estimate_impl(pdd_problem* p, int n_levels, const pdd_estimate_args* levels,
                         pdd_node_stats* outs, uint32_t call_flags, const char* who) {
  const int dim = p->dim;
  const bool async = (call_flags & PDD_FLAG_ASYNC) != 0;
  const bool graph = (call_flags & PDD_FLAG_GRAPH) != 0;
  LevelPlan plan[PDD_MAX_LEVELS];
  int cv_all = -1;
  bool any_grid = false;
  size_t total_nodes = 0;
  for (int l = 0; l < n_levels; ++l) {
    int rc = check_level(p, &levels[l], &outs[l], who, l, &plan[l]);
    if (rc != PDD_OK) return rc;
    const bool host_io = !levels[l].coords_on_device || !outs[l].on_device;
    if ((async || graph) && host_io) {
      set_error("%s: PDD_FLAG_ASYNC / PDD_FLAG_GRAPH need device coordinates and outputs", who);
      return PDD_ERR_INVALID;
    }
    if (plan[l].cv == 1) any_grid = true;
    // one launch shares one control-variate mode: grids may mix with plain
    // levels (no grid), the analytic gradient may not mix with either
    const int cls = plan[l].cv == 2 ? 2 : 0;
    if (cv_all < 0) cv_all = cls;
    if (cv_all != cls) {
      set_error("%s: levels mix the exact-gradient control variate with grids or plain levels",
                who);
      return PDD_ERR_INVALID;
    }
    total_nodes += (size_t)levels[l].n_nodes;
  }
  if (total_nodes >= (size_t)1 << 32) {
    set_error("%s: more than 2^32 nodes in one call", who);
    return PDD_ERR_INVALID;
  }
  const int cv = cv_all == 2 ? 2 : (any_grid ? 1 : 0);
  if (total_nodes == 0) return PDD_OK;

  pdd_ctx* c = p->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  if (!g.ok) {
    set_error("%s: cannot select device %d", who, c->device);
    return PDD_ERR_CUDA;
  }
  // workspace: header | records | staged coordinates | staged outputs
  const size_t off_acc = 256;
  size_t off = align_up(off_acc + total_nodes * kAccWords * 8, 256);
  size_t coord_off[PDD_MAX_LEVELS], out_off[PDD_MAX_LEVELS];
  for (int l = 0; l < n_levels; ++l) {
    coord_off[l] = off;
    if (!levels[l].coords_on_device) off += align_up((size_t)levels[l].n_nodes * 4, 256) * dim;
  }
  for (int l = 0; l < n_levels; ++l) {
    out_off[l] = off;
    if (!outs[l].on_device) off += 14 * align_up((size_t)levels[l].n_nodes * 8, 256);
  }
  int rc = ensure_workspace(c, off);
  if (rc != PDD_OK) return rc;
  char* ws = (char*)c->ws;
  WsHeader* hdr = (WsHeader*)ws;
  unsigned long long* acc = (unsigned long long*)(ws + off_acc);

  // segments: levels with the smallest time step (the longest paths) first
  int order[PDD_MAX_LEVELS];
  for (int l = 0; l < n_levels; ++l) order[l] = l;
  std::stable_sort(order, order + n_levels,
                   [&](int x, int y) { return levels[x].dt < levels[y].dt; });
  PathArgs pa{};
  pa.cursor = &hdr->cursor;
  pa.err = &hdr->err;
  pa.trunc_total = &hdr->trunc_total;
  pa.y_exp = p->desc.y_rule == PDD_Y_EXP;
  pa.max_blocks = c->max_blocks;
  pa.block_threads = c->block_threads;
  pa.iter_mode = c->iter_mode;
  pa.claim = c->claim;
  const double c0 = p->desc.exit_rule == PDD_EXIT_GOBET_MENOZZI ? 0.5826 : 0.0;
  uint32_t rec_base[PDD_MAX_LEVELS];
  {
    uint32_t rb = 0;
    for (int l = 0; l < n_levels; ++l) {
      rec_base[l] = rb;
      rb += (uint32_t)levels[l].n_nodes;
    }
  }
  unsigned long long begin = 0;
  int ns = 0;
  for (int oi = 0; oi < n_levels; ++oi) {
    const int l = order[oi];
    const pdd_estimate_args& a = levels[l];
    if (a.n_nodes == 0) continue;
    SegArgs& sg = pa.seg[ns++];
    sg.cx = a.coords[0];
    sg.cy = a.coords[1];
    sg.cz = dim == 3 ? a.coords[2] : a.coords[0];
    if (!a.coords_on_device) {
      const float* dev[3];
      for (int j = 0; j < dim; ++j)
        dev[j] = (const float*)(ws + coord_off[l] + j * align_up((size_t)a.n_nodes * 4, 256));
      sg.cx = dev[0];
      sg.cy = dev[1];
      sg.cz = dim == 3 ? dev[2] : dev[0];
    }
    sg.begin = begin;
    sg.total = (unsigned long long)a.n_nodes * (unsigned long long)a.n_paths;
    sg.n_paths = (unsigned long long)a.n_paths;
    sg.n_nodes = (unsigned long long)a.n_nodes;
    sg.acc = acc + (size_t)rec_base[l] * kAccWords;
    sg.path_off = 0;
    sg.emit_stride = (unsigned long long)a.n_paths;
    sg.grad = plan[l].table;
    const bool emit = (a.flags & PDD_FLAG_EMIT_PATHS) != 0;
    sg.emit_phi = emit ? a.path_phi : nullptr;
    sg.emit_xi = emit ? a.path_xi : nullptr;
    sg.emit_steps = emit ? a.path_steps : nullptr;
    sg.h = a.dt;
    sg.sqrt_h = std::sqrt(a.dt);
    sg.thr0 = c0 * sg.sqrt_h;
    sg.key0 = (uint32_t)a.seed;
    sg.key1 = a.stream_tag;
    sg.seed_hi = (uint32_t)(a.seed >> 32);
    sg.grid_n = plan[l].grid_n;
    sg.max_steps = (int)plan[l].max_steps;
    begin += sg.total;
  }
  pa.n_segs = ns;
  pa.total = begin;

  StatPtrs sp[PDD_MAX_LEVELS];
  uint32_t lvl_nodes[PDD_MAX_LEVELS];
  double lvl_kappa[PDD_MAX_LEVELS];
  for (int l = 0; l < n_levels; ++l) {
    lvl_nodes[l] = (uint32_t)levels[l].n_nodes;
    lvl_kappa[l] = levels[l].kappa > 0.0 ? levels[l].kappa : 1.0;
  }
  for (int l = 0; l < n_levels; ++l) {
    const pdd_node_stats& o = outs[l];
    double* const user_d[12] = {o.mean_phi, o.var_phi, o.mean_cv, o.var_cv, o.cov_phi_xi,
                                o.var_xi, o.rho, o.se_phi, o.se_cv, o.vr, o.pred_speedup,
                                o.mean_steps};
    uint64_t* const user_u[2] = {o.n_paths, o.n_truncated};
    double* d[12];
    unsigned long long* u[2];
    const size_t n8 = align_up((size_t)levels[l].n_nodes * 8, 256);
    for (int i = 0; i < 12; ++i)
      d[i] = (!o.on_device && user_d[i]) ? (double*)(ws + out_off[l] + i * n8) : user_d[i];
    for (int i = 0; i < 2; ++i)
      u[i] = (!o.on_device && user_u[i]) ? (unsigned long long*)(ws + out_off[l] + (12 + i) * n8)
                                         : (unsigned long long*)user_u[i];
    sp[l] = StatPtrs{d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], d[8], d[9], d[10], d[11],
                     u[0], u[1]};
  }

  // The launch sequence: clear the header and records, run every path, finalise
  // every level.  With PDD_FLAG_GRAPH it is captured once into a CUDA graph and
  // replayed while the arguments stay the same.
  auto enqueue = [&](cudaStream_t st) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(ws, 0, off_acc + total_nodes * kAccWords * 8, st);
    if (e != cudaSuccess) return e;
    int blocks = 0;
    e = launch_paths(p->desc.kind, p->desc.precision, cv, pa, c->num_sms, st, &blocks);
    if (e != cudaSuccess) return e;
    return launch_finalize_levels(acc, n_levels, rec_base, lvl_nodes, lvl_kappa, sp, st);
  };
  const int n_launch = 2;  // the path kernel and one finalisation for every level

  // host inputs
  for (int l = 0; l < n_levels; ++l) {
    const pdd_estimate_args& a = levels[l];
    if (a.coords_on_device || a.n_nodes == 0) continue;
    for (int j = 0; j < dim; ++j) {
      float* dst = (float*)(ws + coord_off[l] + j * align_up((size_t)a.n_nodes * 4, 256));
      PDD_CUDA(cudaMemcpyAsync(dst, a.coords[j], (size_t)a.n_nodes * 4, cudaMemcpyHostToDevice,
                               c->stream),
               "cudaMemcpyAsync(coords)");
    }
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (c->timing) {
    PDD_CUDA(cudaEventCreate(&ev0), "cudaEventCreate");
    PDD_CUDA(cudaEventCreate(&ev1), "cudaEventCreate");
  }
  if (graph) {
    uint64_t key = 1469598103934665603ull;
    key = fnv1a(key, &p, sizeof(p));
    key = fnv1a(key, &pa, sizeof(pa));
    key = fnv1a(key, &n_levels, sizeof(n_levels));
    key = fnv1a(key, sp, sizeof(StatPtrs) * n_levels);
    for (int l = 0; l < n_levels; ++l) key = fnv1a(key, &levels[l].kappa, sizeof(double));
    key = fnv1a(key, &c->ws, sizeof(c->ws));
    if (!c->gexec || c->gkey != key) {
      if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
      }
      cudaGraph_t gr = nullptr;
      PDD_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal),
               "cudaStreamBeginCapture");
      cudaError_t e = enqueue(c->stream);
      cudaError_t e2 = cudaStreamEndCapture(c->stream, &gr);
      if (e != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return cuda_fail(e, "graph capture");
      }
      if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&c->gexec, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
      }
      c->gkey = key;
      c->graph_captures += 1;
    }
    wait_abort(c);
    if (c->timing) PDD_CUDA(cudaEventRecord(ev0, c->stream), "cudaEventRecord");
    PDD_CUDA(cudaGraphLaunch(c->gexec, c->stream), "cudaGraphLaunch");
    if (c->timing) PDD_CUDA(cudaEventRecord(ev1, c->stream), "cudaEventRecord");
  } else {
    wait_abort(c);
    PDD_CUDA(cudaMemsetAsync(ws, 0, off_acc + total_nodes * kAccWords * 8, c->stream),
             "cudaMemsetAsync");
    if (c->timing) PDD_CUDA(cudaEventRecord(ev0, c->stream), "cudaEventRecord");
    int blocks = 0;
    PDD_CUDA(launch_paths(p->desc.kind, p->desc.precision, cv, pa, c->num_sms, c->stream, &blocks),
             "path kernel launch");
    if (c->timing) PDD_CUDA(cudaEventRecord(ev1, c->stream), "cudaEventRecord");
    PDD_CUDA(launch_finalize_levels(acc, n_levels, rec_base, lvl_nodes, lvl_kappa, sp, c->stream),
             "finalize launch");
  }
  if (c->timing) c->events.emplace_back(ev0, ev1);
  c->launches += n_launch;
  // host outputs
  for (int l = 0; l < n_levels; ++l) {
    const pdd_node_stats& o = outs[l];
    if (o.on_device || levels[l].n_nodes == 0) continue;
    const size_t nb = (size_t)levels[l].n_nodes * 8;
    double* const user_d[12] = {o.mean_phi, o.var_phi, o.mean_cv, o.var_cv, o.cov_phi_xi,
                                o.var_xi, o.rho, o.se_phi, o.se_cv, o.vr, o.pred_speedup,
                                o.mean_steps};
    uint64_t* const user_u[2] = {o.n_paths, o.n_truncated};
    double* const dd[12] = {sp[l].mean_phi, sp[l].var_phi, sp[l].mean_cv, sp[l].var_cv,
                            sp[l].cov_phi_xi, sp[l].var_xi, sp[l].rho, sp[l].se_phi,
                            sp[l].se_cv, sp[l].vr, sp[l].pred_speedup, sp[l].mean_steps};
    unsigned long long* const du[2] = {sp[l].n_paths, sp[l].n_truncated};
    for (int i = 0; i < 12; ++i)
      if (user_d[i])
        PDD_CUDA(cudaMemcpyAsync(user_d[i], dd[i], nb, cudaMemcpyDeviceToHost, c->stream),
                 "cudaMemcpyAsync(outputs)");
    for (int i = 0; i < 2; ++i)
      if (user_u[i])
        PDD_CUDA(cudaMemcpyAsync(user_u[i], du[i], nb, cudaMemcpyDeviceToHost, c->stream),
                 "cudaMemcpyAsync(outputs)");
  }
  if (async) return PDD_OK;
  WsHeader h{};
  PDD_CUDA(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, c->stream),
           "cudaMemcpyAsync(header)");
  PDD_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (h.aborted) return aborted_status(who);
  if (h.err != 0u) return error_word_status(h.err, who);
  if (h.cursor < pa.total) {
    set_error("%s: internal error, %llu of %llu paths scheduled", who, h.cursor, pa.total);
    return PDD_ERR_CUDA;
  }
  if (h.trunc_total > 0) {
    set_error("%s: %llu paths hit max_steps", who, h.trunc_total);
    return PDD_WARN_TRUNCATED;
  }
  (void)enqueue;
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
  // what pdd_ctx_abort uses, made now so that an abort allocates nothing (page-locked
  // allocation can wait for the device)
  cudaError_t ea = cudaStreamCreateWithFlags(&c->abort_stream, cudaStreamNonBlocking);
  if (ea == cudaSuccess) ea = cudaEventCreateWithFlags(&c->abort_ev, cudaEventDisableTiming);
  if (ea == cudaSuccess)
    ea = cudaMallocHost((void**)&c->abort_src, 2 * sizeof(unsigned long long));
  if (ea != cudaSuccess) {
    if (c->abort_ev) cudaEventDestroy(c->abort_ev);
    if (c->abort_stream) cudaStreamDestroy(c->abort_stream);
    delete c;
    return cuda_fail(ea, "pdd_ctx_create: abort resources");
  }
  c->abort_src[0] = 1ull << 62;  // past the index space of any launch (< 2^62 paths)
  c->abort_src[1] = 1ull;        // low word: the header's `aborted`
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
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->abort_stream) {
      cudaStreamSynchronize(c->abort_stream);
      cudaStreamDestroy(c->abort_stream);
      cudaEventDestroy(c->abort_ev);
      cudaFreeHost(c->abort_src);
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

int pdd_ctx_graph_count(pdd_ctx* c, int64_t* captures) {
  if (!c || !captures) {
    set_error("pdd_ctx_graph_count: NULL argument");
    return PDD_ERR_INVALID;
  }
  *captures = c->graph_captures;
  return PDD_OK;
}

int pdd_ctx_launch_count(pdd_ctx* c, int64_t* launches) {
  if (!c || !launches) {
    set_error("pdd_ctx_launch_count: NULL argument");
    return PDD_ERR_INVALID;
  }
  *launches = c->launches;
  return PDD_OK;
}

int pdd_ctx_abort(pdd_ctx* c) {
  if (!c) {
    set_error("pdd_ctx_abort: NULL context");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->abort_mu);
  DeviceGuard g(c->device);
  if (!c->ws) return PDD_OK;  // nothing has run on this context yet
  PDD_CUDA(cudaMemcpyAsync((char*)c->ws + offsetof(WsHeader, aborted), &c->abort_src[1], 4,
                           cudaMemcpyHostToDevice, c->abort_stream),
           "cudaMemcpyAsync(abort flag)");
  PDD_CUDA(cudaMemcpyAsync(c->ws, &c->abort_src[0], 8, cudaMemcpyHostToDevice, c->abort_stream),
           "cudaMemcpyAsync(abort cursor)");
  PDD_CUDA(cudaEventRecord(c->abort_ev, c->abort_stream), "cudaEventRecord");
  c->abort_pending = true;
  return PDD_OK;
}

int pdd_create_problem(pdd_ctx* c, const pdd_problem_desc* d, pdd_problem** out) {
  if (!c || !d || !out) {
    set_error("pdd_create_problem: NULL argument");
    return PDD_ERR_INVALID;
  }
  *out = nullptr;
  if (d->kind < PDD_PROBLEM_CFG0_2D || d->kind > PDD_PROBLEM_PAPER_EX_2D) {
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
  // stage the input as FP64 on the device (plus a flag word for the cell table)
  double* staged = nullptr;
  PDD_CUDA(cudaMalloc(&staged, count * sizeof(double) + 16), "cudaMalloc(grid staging)");
  unsigned* overflow = (unsigned*)(staged + count);
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
  // one allocation: the nodal gradient table, then the per-cell coefficients
  void* table = nullptr;
  const size_t m = (size_t)d->n - 1;
  const size_t ncell = dim == 2 ? m * m : m * m * m;
  const size_t tbytes = cell_table_offset(d->n, dim) + ncell * (dim == 2 ? 32 : 64);
  if (e == cudaSuccess) e = cudaMalloc(&table, tbytes);
  // cell records are read with 32-byte vector loads: the table must start on a
  // 32-byte boundary (cudaMalloc gives 256; the offset is a multiple of 256)
  if (e == cudaSuccess && (((uintptr_t)table | cell_table_offset(d->n, dim)) & 31u) != 0) {
    cudaFree(table);
    cudaFree(staged);
    set_error("pdd_set_control_grid: misaligned table");
    return PDD_ERR_CUDA;
  }
  if (e == cudaSuccess) {
    e = d->kind == PDD_GRID_VALUES ? launch_grid_gradient(staged, d->n, dim, table, c->stream)
                                   : launch_grid_pack(staged, d->n, dim, table, c->stream);
    c->launches += 1;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(overflow, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess) {
    e = launch_grid_cells(table, d->n, dim, (char*)table + cell_table_offset(d->n, dim),
                          overflow, c->stream);
    c->launches += 1;
  }
  unsigned ovf = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&ovf, overflow, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(staged);
  if (e != cudaSuccess) {
    if (table) cudaFree(table);
    return cuda_fail(e, "pdd_set_control_grid");
  }
  // FP32 3D paths read binary16 differences: a grid beyond that range would
  // give them a wrong gradient (such gradients would overflow the scores'
  // fixed-point range within a few steps anyway)
  if (ovf != 0 && dim == 3 && p->desc.precision == PDD_PATH_FP32) {
    cudaFree(table);
    set_error("pdd_set_control_grid: gradient differences between neighbouring grid points "
              "exceed 65504 (the binary16 range of the 3D cell table)");
    return PDD_ERR_INVALID;
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
  return estimate_impl(p, 1, a, out, a->flags & PDD_FLAG_ASYNC, "pdd_estimate_nodes");
}

int pdd_estimate_levels(pdd_problem* p, int n_levels, const pdd_estimate_args* levels,
                        pdd_node_stats* outs, uint32_t flags) {
  if (!p || !levels || !outs) {
    set_error("pdd_estimate_levels: NULL argument");
    return PDD_ERR_INVALID;
  }
  if (n_levels < 1 || n_levels > PDD_MAX_LEVELS) {
    set_error("pdd_estimate_levels: n_levels = %d outside [1, %d]", n_levels, PDD_MAX_LEVELS);
    return PDD_ERR_INVALID;
  }
  if (flags & ~(PDD_FLAG_ASYNC | PDD_FLAG_GRAPH)) {
    set_error("pdd_estimate_levels: unknown call flags 0x%x", flags);
    return PDD_ERR_INVALID;
  }
  for (int l = 0; l < n_levels; ++l)
    if (levels[l].flags & PDD_FLAG_ASYNC) {
      set_error("pdd_estimate_levels: PDD_FLAG_ASYNC belongs to the call flags, not to level %d",
                l);
      return PDD_ERR_INVALID;
    }
  return estimate_impl(p, n_levels, levels, outs, flags, "pdd_estimate_levels");
}

int pdd_accumulate(pdd_problem* p, const pdd_estimate_args* a, uint64_t path_offset,
                   uint64_t* records) {
  if (!p || !a || !records) {
    set_error("pdd_accumulate: NULL argument");
    return PDD_ERR_INVALID;
  }
  LevelPlan lp;
  pdd_node_stats dummy{};
  int rc = check_level(p, a, &dummy, "pdd_accumulate", 0, &lp);
  if (rc != PDD_OK) return rc;
  if (a->flags & PDD_FLAG_EMIT_PATHS) {
    set_error("pdd_accumulate: per-path output is not available here");
    return PDD_ERR_INVALID;
  }
  if (!a->coords_on_device) {
    set_error("pdd_accumulate: coordinates must be device pointers");
    return PDD_ERR_INVALID;
  }
  if (path_offset + (uint64_t)a->n_paths > (1ull << 32)) {
    set_error("pdd_accumulate: path indices beyond 2^32");
    return PDD_ERR_INVALID;
  }
  if (a->n_nodes == 0) return PDD_OK;
  pdd_ctx* c = p->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  rc = ensure_workspace(c, 256);
  if (rc != PDD_OK) return rc;
  WsHeader* hdr = (WsHeader*)c->ws;
  PathArgs pa{};
  pa.cursor = &hdr->cursor;
  pa.err = &hdr->err;
  pa.trunc_total = &hdr->trunc_total;
  pa.y_exp = p->desc.y_rule == PDD_Y_EXP;
  pa.max_blocks = c->max_blocks;
  pa.block_threads = c->block_threads;
  pa.iter_mode = c->iter_mode;
  pa.claim = c->claim;
  pa.n_segs = 1;
  SegArgs& sg = pa.seg[0];
  const int dim = p->dim;
  sg.cx = a->coords[0];
  sg.cy = a->coords[1];
  sg.cz = dim == 3 ? a->coords[2] : a->coords[0];
  sg.begin = 0;
  sg.total = (unsigned long long)a->n_nodes * (unsigned long long)a->n_paths;
  sg.n_paths = (unsigned long long)a->n_paths;
  sg.n_nodes = (unsigned long long)a->n_nodes;
  sg.acc = (unsigned long long*)records;
  sg.grad = lp.table;
  sg.emit_stride = 0;
  sg.h = a->dt;
  sg.sqrt_h = std::sqrt(a->dt);
  const double c0 = p->desc.exit_rule == PDD_EXIT_GOBET_MENOZZI ? 0.5826 : 0.0;
  sg.thr0 = c0 * sg.sqrt_h;
  sg.path_off = (uint32_t)path_offset;
  sg.key0 = (uint32_t)a->seed;
  sg.key1 = a->stream_tag;
  sg.seed_hi = (uint32_t)(a->seed >> 32);
  sg.grid_n = lp.grid_n;
  sg.max_steps = (int)lp.max_steps;
  pa.total = sg.total;
  wait_abort(c);
  PDD_CUDA(cudaMemsetAsync(hdr, 0, 256, c->stream), "cudaMemsetAsync");
  int blocks = 0;
  PDD_CUDA(launch_paths(p->desc.kind, p->desc.precision, lp.cv, pa, c->num_sms, c->stream, &blocks),
           "path kernel launch");
  c->launches += 1;
  if (a->flags & PDD_FLAG_ASYNC) return PDD_OK;
  WsHeader h{};
  PDD_CUDA(cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, c->stream),
           "cudaMemcpyAsync(header)");
  PDD_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (h.aborted) return aborted_status("pdd_accumulate");
  if (h.err != 0u) return error_word_status(h.err, "pdd_accumulate");
  if (h.trunc_total > 0) {
    set_error("pdd_accumulate: %llu paths hit max_steps", h.trunc_total);
    return PDD_WARN_TRUNCATED;
  }
  return PDD_OK;
}

int pdd_finalize_records(pdd_ctx* c, const uint64_t* records, int64_t n_nodes, double kappa,
                         pdd_node_stats* out) {
  if (!c || !records || !out || n_nodes < 0 || n_nodes >= ((int64_t)1 << 32)) {
    set_error("pdd_finalize_records: bad arguments");
    return PDD_ERR_INVALID;
  }
  if (n_nodes == 0) return PDD_OK;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  const size_t n = (size_t)n_nodes, n8 = align_up(n * 8, 256);
  if (!out->on_device) {
    int rc = ensure_workspace(c, 256 + 14 * n8);
    if (rc != PDD_OK) return rc;
  }
  char* stage = (char*)c->ws + 256;
  double* const user_d[12] = {out->mean_phi, out->var_phi, out->mean_cv, out->var_cv,
                              out->cov_phi_xi, out->var_xi, out->rho, out->se_phi, out->se_cv,
                              out->vr, out->pred_speedup, out->mean_steps};
  uint64_t* const user_u[2] = {out->n_paths, out->n_truncated};
  double* d[12];
  unsigned long long* u[2];
  for (int i = 0; i < 12; ++i)
    d[i] = (!out->on_device && user_d[i]) ? (double*)(stage + i * n8) : user_d[i];
  for (int i = 0; i < 2; ++i)
    u[i] = (!out->on_device && user_u[i]) ? (unsigned long long*)(stage + (12 + i) * n8)
                                          : (unsigned long long*)user_u[i];
  const StatPtrs sp{d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], d[8], d[9], d[10], d[11],
                    u[0], u[1]};
  PDD_CUDA(launch_finalize((const unsigned long long*)records, (uint32_t)n,
                           kappa > 0.0 ? kappa : 1.0, sp, c->stream),
           "finalize launch");
  c->launches += 1;
  if (!out->on_device) {
    for (int i = 0; i < 14; ++i) {
      void* dst = i < 12 ? (void*)user_d[i] : (void*)user_u[i - 12];
      const void* src = i < 12 ? (const void*)d[i] : (const void*)u[i - 12];
      if (dst)
        PDD_CUDA(cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToHost, c->stream),
                 "cudaMemcpyAsync(outputs)");
    }
  }
  PDD_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  return PDD_OK;
}

int pdd_records_merge(uint64_t* dst, const uint64_t* src, int64_t n_nodes) {
  if ((!dst || !src) && n_nodes > 0) {
    set_error("pdd_records_merge: NULL argument");
    return PDD_ERR_INVALID;
  }
  for (int64_t i = 0; i < n_nodes; ++i) {
    uint64_t* a = dst + i * PDD_RECORD_WORDS;
    const uint64_t* b = src + i * PDD_RECORD_WORDS;
    for (int w = 0; w < 14; w += 2) {  // seven 128-bit sums
      const uint64_t lo = a[w] + b[w];
      a[w + 1] += b[w + 1] + (lo < a[w] ? 1u : 0u);
      a[w] = lo;
    }
    a[14] += b[14];
    a[15] += b[15];
  }
  return PDD_OK;
}

// One launch of the coupled kernel over pairs path_offset .. path_offset +
// n_paths - 1 of every node, adding into the fine / difference records rf, rd
// (device).  The caller holds the context lock and has checked the level.
static int coupled_launch(pdd_problem* p, const pdd_estimate_args* a, const LevelPlan& lp,
                          uint64_t path_offset, unsigned long long* rf, unsigned long long* rd,
                          const char* who) {
  pdd_ctx* c = p->ctx;
  const double hf = 0.5 * a->dt, hc = a->dt;
  auto steps_cap = [&](double h) -> int {
    int64_t ms = p->desc.max_steps;
    if (ms <= 0) ms = (int64_t)std::min(2.0e9, std::ceil(100.0 / h));
    return (int)std::min<int64_t>(ms, 2000000000ll);
  };
  const size_t n = (size_t)a->n_nodes;
  int rc = ensure_workspace(c, 256);
  if (rc != PDD_OK) return rc;
  WsHeader* hdr = (WsHeader*)c->ws;
  PathArgs pa{};
  pa.cursor = &hdr->cursor;
  pa.err = &hdr->err;
  pa.trunc_total = &hdr->trunc_total;
  pa.y_exp = p->desc.y_rule == PDD_Y_EXP;
  pa.max_blocks = c->max_blocks;
  pa.block_threads = c->block_threads;
  pa.iter_mode = c->iter_mode;
  pa.claim = c->claim;
  pa.n_segs = 2;
  pa.total = (unsigned long long)n * (unsigned long long)a->n_paths;
  const double c0 = p->desc.exit_rule == PDD_EXIT_GOBET_MENOZZI ? 0.5826 : 0.0;
  const bool emit = (a->flags & PDD_FLAG_EMIT_PATHS) != 0;
  for (int l = 0; l < 2; ++l) {
    SegArgs& sg = pa.seg[l];
    const double h = l == 0 ? hf : hc;
    sg.cx = a->coords[0];
    sg.cy = a->coords[1];
    sg.cz = p->dim == 3 ? a->coords[2] : a->coords[0];
    sg.begin = 0;
    sg.total = pa.total;
    sg.n_paths = (unsigned long long)a->n_paths;
    sg.n_nodes = (unsigned long long)n;
    sg.acc = l == 0 ? rf : rd;
    sg.grad = lp.table;
    const size_t off = l == 0 ? 0 : n * (size_t)a->n_paths;
    sg.emit_phi = emit ? a->path_phi + off : nullptr;
    sg.emit_xi = emit ? a->path_xi + off : nullptr;
    sg.emit_steps = emit ? a->path_steps + off : nullptr;
    sg.emit_stride = (unsigned long long)a->n_paths;
    sg.h = h;
    sg.sqrt_h = std::sqrt(h);
    sg.thr0 = c0 * sg.sqrt_h;
    sg.path_off = (uint32_t)path_offset;
    sg.key0 = (uint32_t)a->seed;
    sg.key1 = a->stream_tag;
    sg.seed_hi = (uint32_t)(a->seed >> 32);
    sg.grid_n = lp.grid_n;
    sg.max_steps = steps_cap(h);
  }
  wait_abort(c);
  PDD_CUDA(cudaMemsetAsync(hdr, 0, 256, c->stream), "cudaMemsetAsync");
  int blocks = 0;
  char what[96];
  snprintf(what, sizeof(what), "%s: coupled kernel launch", who);
  PDD_CUDA(launch_coupled(p->desc.kind, lp.cv, pa, c->num_sms, c->stream, &blocks), what);
  c->launches += 1;
  return PDD_OK;
}

// Read the launch header (synchronising the context stream) and turn its
// error bits into a status.
static int coupled_status(pdd_ctx* c, const char* who) {
  WsHeader h{};
  PDD_CUDA(cudaMemcpyAsync(&h, c->ws, sizeof(h), cudaMemcpyDeviceToHost, c->stream),
           "cudaMemcpyAsync(header)");
  PDD_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (h.aborted) return aborted_status(who);
  if (h.err != 0u) return error_word_status(h.err, who);
  if (h.trunc_total > 0) {
    set_error("%s: %llu paths hit max_steps", who, h.trunc_total);
    return PDD_WARN_TRUNCATED;
  }
  return PDD_OK;
}

static int coupled_check(pdd_problem* p, const pdd_estimate_args* a, LevelPlan* lp,
                         const char* who) {
  if (p->desc.precision != PDD_PATH_FP32) {
    set_error("%s: provided for FP32 paths", who);
    return PDD_ERR_INVALID;
  }
  pdd_node_stats dummy{};
  dummy.on_device = 1;
  int rc = check_level(p, a, &dummy, who, 0, lp);
  if (rc != PDD_OK) return rc;
  if (!a->coords_on_device) {
    set_error("%s: coordinates must be device pointers", who);
    return PDD_ERR_INVALID;
  }
  return PDD_OK;
}

int pdd_estimate_coupled(pdd_problem* p, const pdd_estimate_args* a, pdd_node_stats* out_fine,
                         pdd_node_stats* out_diff) {
  const char* who = "pdd_estimate_coupled";
  if (!p || !a || !out_fine || !out_diff) {
    set_error("%s: NULL argument", who);
    return PDD_ERR_INVALID;
  }
  LevelPlan lp;
  int rc = coupled_check(p, a, &lp, who);
  if (rc != PDD_OK) return rc;
  if (!out_fine->on_device || !out_diff->on_device) {
    set_error("%s: outputs must be device pointers", who);
    return PDD_ERR_INVALID;
  }
  if (a->n_nodes == 0) return PDD_OK;
  pdd_ctx* c = p->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  const size_t n = (size_t)a->n_nodes;
  const size_t rec_bytes = align_up(n * kAccWords * 8, 256);
  rc = ensure_workspace(c, 256 + 2 * rec_bytes);
  if (rc != PDD_OK) return rc;
  char* ws = (char*)c->ws;
  unsigned long long* rf = (unsigned long long*)(ws + 256);
  unsigned long long* rd = (unsigned long long*)(ws + 256 + rec_bytes);
  PDD_CUDA(cudaMemsetAsync(ws + 256, 0, 2 * rec_bytes, c->stream), "cudaMemsetAsync");
  rc = coupled_launch(p, a, lp, 0, rf, rd, who);
  if (rc != PDD_OK) return rc;
  const double kappa = a->kappa > 0.0 ? a->kappa : 1.0;
  pdd_node_stats* outs[2] = {out_fine, out_diff};
  unsigned long long* recs[2] = {rf, rd};
  for (int l = 0; l < 2; ++l) {
    const pdd_node_stats& o = *outs[l];
    const StatPtrs sp{o.mean_phi, o.var_phi, o.mean_cv, o.var_cv, o.cov_phi_xi, o.var_xi, o.rho,
                      o.se_phi, o.se_cv, o.vr, o.pred_speedup, o.mean_steps,
                      (unsigned long long*)o.n_paths, (unsigned long long*)o.n_truncated};
    PDD_CUDA(launch_finalize(recs[l], (uint32_t)n, kappa, sp, c->stream), "finalize launch");
  }
  c->launches += 2;
  if (a->flags & PDD_FLAG_ASYNC) return PDD_OK;
  return coupled_status(c, who);
}

int pdd_accumulate_coupled(pdd_problem* p, const pdd_estimate_args* a, uint64_t path_offset,
                           uint64_t* rec_fine, uint64_t* rec_diff) {
  const char* who = "pdd_accumulate_coupled";
  if (!p || !a || !rec_fine || !rec_diff) {
    set_error("%s: NULL argument", who);
    return PDD_ERR_INVALID;
  }
  LevelPlan lp;
  int rc = coupled_check(p, a, &lp, who);
  if (rc != PDD_OK) return rc;
  if (a->flags & PDD_FLAG_EMIT_PATHS) {
    set_error("%s: per-path output is not available here", who);
    return PDD_ERR_INVALID;
  }
  if (path_offset + (uint64_t)a->n_paths > (1ull << 32)) {
    set_error("%s: path indices beyond 2^32", who);
    return PDD_ERR_INVALID;
  }
  if (a->n_nodes == 0) return PDD_OK;
  pdd_ctx* c = p->ctx;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  rc = coupled_launch(p, a, lp, path_offset, (unsigned long long*)rec_fine,
                      (unsigned long long*)rec_diff, who);
  if (rc != PDD_OK) return rc;
  if (a->flags & PDD_FLAG_ASYNC) return PDD_OK;
  return coupled_status(c, who);
}

int pdd_ctx_set_launch(pdd_ctx* c, int block_threads, int max_blocks) {
  if (!c) {
    set_error("pdd_ctx_set_launch: NULL context");
    return PDD_ERR_INVALID;
  }
  if (block_threads != 0 && (block_threads < 32 || block_threads > 512 || block_threads % 32)) {
    set_error("pdd_ctx_set_launch: block_threads = %d must be 0 or a multiple of 32 in [32, 512]",
              block_threads);
    return PDD_ERR_INVALID;
  }
  if (max_blocks < 0) {
    set_error("pdd_ctx_set_launch: max_blocks = %d must be >= 0", max_blocks);
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->block_threads = block_threads;
  c->max_blocks = max_blocks;
  return PDD_OK;
}

int pdd_ctx_set_iteration(pdd_ctx* c, int mode) {
  if (!c || (mode != PDD_ITER_AUTO && mode != PDD_ITER_SHORT && mode != PDD_ITER_LONG)) {
    set_error("pdd_ctx_set_iteration: NULL context or mode not PDD_ITER_AUTO/SHORT/LONG");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->iter_mode = mode;
  return PDD_OK;
}

int pdd_ctx_set_claim(pdd_ctx* c, int paths_per_lane) {
  if (!c || paths_per_lane < 0 || paths_per_lane > 64 ||
      (paths_per_lane & (paths_per_lane - 1)) != 0) {
    set_error("pdd_ctx_set_claim: NULL context or paths_per_lane not 0 or a power of two <= 64");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->claim = paths_per_lane;
  return PDD_OK;
}

int pdd_ctx_get_claim(pdd_ctx* c, int* paths_per_lane) {
  if (!c || !paths_per_lane) {
    set_error("pdd_ctx_get_claim: NULL argument");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  *paths_per_lane = c->claim;
  return PDD_OK;
}

int pdd_ctx_get_launch(pdd_ctx* c, int* block_threads, int* max_blocks, int* iteration) {
  if (!c) {
    set_error("pdd_ctx_get_launch: NULL context");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  if (block_threads) *block_threads = c->block_threads;
  if (max_blocks) *max_blocks = c->max_blocks;
  if (iteration) *iteration = c->iter_mode;
  return PDD_OK;
}

int pdd_autotune(pdd_problem* p, const pdd_estimate_args* sample, int* best_threads,
                 int* best_max_blocks, double* best_ms) {
  if (!p || !sample) {
    set_error("pdd_autotune: NULL argument");
    return PDD_ERR_INVALID;
  }
  if (!sample->coords_on_device) {
    set_error("pdd_autotune: the sample must use device coordinates");
    return PDD_ERR_INVALID;
  }
  pdd_ctx* c = p->ctx;
  const int old_threads = c->block_threads, old_blocks = c->max_blocks;
  const size_t n = (size_t)sample->n_nodes;
  if (n == 0) {
    set_error("pdd_autotune: empty sample");
    return PDD_ERR_INVALID;
  }
  // device outputs: the means only (the other statistics are not needed here)
  double* dmean = nullptr;
  {
    DeviceGuard g(c->device);
    PDD_CUDA(cudaMalloc(&dmean, n * sizeof(double)), "cudaMalloc(autotune)");
  }
  pdd_node_stats out{};
  out.on_device = 1;
  out.mean_phi = dmean;
  pdd_estimate_args a = *sample;
  a.flags &= ~(PDD_FLAG_EMIT_PATHS | PDD_FLAG_ASYNC);
  const int old_iter = c->iter_mode, old_claim = c->claim;
  int rc = PDD_OK;
  // CUDA-event time of the sample under the context's current settings (the
  // first of two runs warms up)
  auto time_one = [&]() -> double {
    double ms = 0.0;
    for (int rep = 0; rep < 2 && rc >= 0; ++rep) {
      cudaEvent_t e0, e1;
      {
        DeviceGuard g(c->device);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, c->stream);
      }
      rc = pdd_estimate_nodes(p, &a, &out);
      {
        DeviceGuard g(c->device);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        ms = f;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
      }
    }
    return ms;
  };
  const int threads_c[3] = {128, 256, 512};
  int bt = 0, bb = 0, bi = PDD_ITER_AUTO;
  double bms = 1e300;
  pdd_ctx_set_iteration(c, PDD_ITER_AUTO);
  pdd_ctx_set_claim(c, 0);
  for (int ti = 0; ti < 3 && rc >= 0; ++ti) {
    // full occupancy, and half of it (fewer resident warps, less L1 pressure)
    for (int frac = 0; frac < 2 && rc >= 0; ++frac) {
      int max_blocks = 0;
      if (frac == 1) {
        int occ = 0;
        rc = query_occupancy(p, a.grid_id, threads_c[ti], &occ);
        if (rc < 0) break;
        max_blocks = (occ / 2 > 0 ? occ / 2 : 1) * c->num_sms;
      }
      pdd_ctx_set_launch(c, threads_c[ti], max_blocks);
      const double ms = time_one();
      if (rc >= 0 && ms < bms) {
        bms = ms;
        bt = threads_c[ti];
        bb = max_blocks;
      }
    }
  }
  // the scheduling quantum (steps per iteration) at the fastest shape
  if (rc >= 0 && p->desc.precision == PDD_PATH_FP32) {
    pdd_ctx_set_launch(c, bt, bb);
    for (int mode : {PDD_ITER_SHORT, PDD_ITER_LONG}) {
      pdd_ctx_set_iteration(c, mode);
      const double ms = time_one();
      if (rc >= 0 && ms < bms) {
        bms = ms;
        bi = mode;
      }
    }
  }
  // paths per lane per cursor claim (the automatic choice was timed above)
  int bc = 0;
  if (rc >= 0) {
    pdd_ctx_set_launch(c, bt, bb);
    pdd_ctx_set_iteration(c, bi);
    for (int claim : {1, 4, 16}) {
      pdd_ctx_set_claim(c, claim);
      const double ms = time_one();
      if (rc >= 0 && ms < bms) {
        bms = ms;
        bc = claim;
      }
    }
  }
  {
    DeviceGuard g(c->device);
    cudaFree(dmean);
  }
  if (rc < 0) {
    pdd_ctx_set_launch(c, old_threads, old_blocks);
    pdd_ctx_set_iteration(c, old_iter);
    pdd_ctx_set_claim(c, old_claim);
    return rc;
  }
  pdd_ctx_set_launch(c, bt, bb);
  pdd_ctx_set_iteration(c, bi);
  pdd_ctx_set_claim(c, bc);
  if (best_threads) *best_threads = bt;
  if (best_max_blocks) *best_max_blocks = bb;
  if (best_ms) *best_ms = bms;
  return PDD_OK;
}

}  // extern "C"
