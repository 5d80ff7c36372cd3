// pdd_noalloc.cu -- pdd_estimate_nodes_noalloc: the estimate of
// pdd_estimate_nodes for callers that cannot let the library allocate device
// memory.  Its scratch (the path cursor, error bits and the per-node exact
// sums) lives in a fixed, file-scope device array instead of the context's
// workspace, so a call performs no cudaMalloc, cudaFree or other allocating
// call.  The kernels are the same path and finalisation kernels; only the
// scratch pointers they receive differ.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/pdd.h"
#include "pdd_internal.h"

namespace pdd {
void set_error(const char* fmt, ...);
}

using namespace pdd;

namespace {

constexpr size_t kHeaderBytes = 256;
constexpr size_t kScratchBytes = kHeaderBytes + (size_t)PDD_NOALLOC_MAX_NODES * kAccWords * 8;

// Shared by every call on a device; each device that loads the library holds
// its own copy (about 512 KiB) until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct ScratchHeader {
  unsigned long long cursor;
  unsigned err;
  unsigned pad;
  unsigned long long trunc_total;
};

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `device` (which must be current).
// The host-side name of the array is only a stand-in, so the address is
// looked up once per device and cached.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("pdd_estimate_nodes_noalloc: device %d not supported", device);
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      set_error("pdd_estimate_nodes_noalloc: cudaGetSymbolAddress failed: %s",
                cudaGetErrorString(e));
      return PDD_ERR_CUDA;
    }
    g_scratch_ptr[device] = ptr;
  }
  *out = g_scratch_ptr[device];
  return PDD_OK;
}

int fail(cudaError_t e, const char* what) {
  set_error("pdd_estimate_nodes_noalloc: %s: %s", what, cudaGetErrorString(e));
  return PDD_ERR_CUDA;
}

}  // namespace

extern "C" int pdd_estimate_nodes_noalloc(pdd_problem* problem, const pdd_estimate_args* a,
                                          pdd_node_stats* out) {
  ProblemView pv;
  if (!problem || !a || !out || !problem_view(problem, &pv)) {
    set_error("pdd_estimate_nodes_noalloc: NULL argument");
    return PDD_ERR_INVALID;
  }
  if (a->n_nodes < 0 || a->n_nodes > PDD_NOALLOC_MAX_NODES) {
    set_error("pdd_estimate_nodes_noalloc: n_nodes = %lld outside [0, %d] (the fixed scratch "
              "holds PDD_NOALLOC_MAX_NODES nodes; use pdd_estimate_nodes for more)",
              (long long)a->n_nodes, PDD_NOALLOC_MAX_NODES);
    return PDD_ERR_INVALID;
  }
  if (a->n_paths < 1 || a->n_paths >= (int64_t)1 << 32) {
    set_error("pdd_estimate_nodes_noalloc: n_paths = %lld outside [1, 2^32)",
              (long long)a->n_paths);
    return PDD_ERR_INVALID;
  }
  if (!(a->dt > 0.0) || !std::isfinite(a->dt)) {
    set_error("pdd_estimate_nodes_noalloc: dt must be finite and > 0");
    return PDD_ERR_INVALID;
  }
  if (a->flags & ~(PDD_FLAG_EMIT_PATHS | PDD_FLAG_ASYNC)) {
    set_error("pdd_estimate_nodes_noalloc: unknown flags 0x%x", a->flags);
    return PDD_ERR_INVALID;
  }
  const bool emit = (a->flags & PDD_FLAG_EMIT_PATHS) != 0;
  if (emit && (!a->path_phi || !a->path_xi || !a->path_steps)) {
    set_error("pdd_estimate_nodes_noalloc: EMIT_PATHS needs path_phi, path_xi and path_steps");
    return PDD_ERR_INVALID;
  }
  if (!a->coords_on_device || !out->on_device) {
    set_error("pdd_estimate_nodes_noalloc: coordinates and outputs must be device pointers "
              "(staging host buffers would need device memory)");
    return PDD_ERR_INVALID;
  }
  int cv = 0;
  const void* table = nullptr;
  int grid_n = 0;
  if (a->grid_id == PDD_CV_NONE) {
    cv = 0;
  } else if (a->grid_id == PDD_CV_EXACT) {
    cv = 2;
  } else if (a->grid_id >= 0 && a->grid_id < PDD_MAX_GRIDS && pv.grid_table[a->grid_id]) {
    cv = 1;
    table = pv.grid_table[a->grid_id];
    grid_n = pv.grid_n[a->grid_id];
  } else {
    set_error("pdd_estimate_nodes_noalloc: grid_id %d is not a loaded grid", a->grid_id);
    return PDD_ERR_INVALID;
  }
  if (a->n_nodes == 0) return PDD_OK;
  for (int j = 0; j < pv.dim; ++j)
    if (!a->coords[j]) {
      set_error("pdd_estimate_nodes_noalloc: coords[%d] is NULL", j);
      return PDD_ERR_INVALID;
    }
  int64_t max_steps = pv.max_steps;
  if (max_steps <= 0) {
    const double ms = std::ceil(100.0 / a->dt);
    max_steps = ms > 2.0e9 ? 2000000000ll : (int64_t)ms;
  }
  if (max_steps > 2000000000ll) max_steps = 2000000000ll;

  std::lock_guard<std::mutex> lk(*pv.mu);
  // the caller's current device is restored on every return
  DeviceGuard guard(pv.device);
  if (!guard.ok) {
    set_error("pdd_estimate_nodes_noalloc: cannot select device %d", pv.device);
    return PDD_ERR_CUDA;
  }
  // the launch shape of the context (pdd_ctx_set_launch / pdd_autotune), as
  // pdd_estimate_nodes uses it
  int ctx_dev = 0, ctx_sms = 0, block_threads = 0, max_blocks = 0;
  ctx_view(problem_ctx(problem), &ctx_dev, &ctx_sms, &block_threads, &max_blocks);
  void* scratch = nullptr;
  int rc = scratch_address(pv.device, &scratch);
  if (rc != PDD_OK) return rc;
  const size_t n = (size_t)a->n_nodes;
  char* base = (char*)scratch;
  ScratchHeader* hdr = (ScratchHeader*)base;
  unsigned long long* acc = (unsigned long long*)(base + kHeaderBytes);
  // The array keeps the previous call's contents: clear the header and the
  // records this call uses.
  cudaError_t e = cudaMemsetAsync(base, 0, kHeaderBytes + n * kAccWords * 8, pv.stream);
  if (e != cudaSuccess) return fail(e, "cudaMemsetAsync");

  PathArgs pa{};
  pa.total = (unsigned long long)n * (unsigned long long)a->n_paths;
  pa.cursor = &hdr->cursor;
  pa.err = &hdr->err;
  pa.trunc_total = &hdr->trunc_total;
  pa.y_exp = pv.y_rule == PDD_Y_EXP;
  pa.max_blocks = max_blocks;
  pa.block_threads = block_threads;
  pa.iter_mode = ctx_iter_mode(problem_ctx(problem));
  pa.claim = ctx_claim(problem_ctx(problem));
  pa.n_segs = 1;
  SegArgs& sg = pa.seg[0];
  sg.cx = a->coords[0];
  sg.cy = a->coords[1];
  sg.cz = pv.dim == 3 ? a->coords[2] : a->coords[0];
  sg.begin = 0;
  sg.total = pa.total;
  sg.n_paths = (unsigned long long)a->n_paths;
  sg.n_nodes = (unsigned long long)n;
  sg.acc = acc;
  sg.path_off = 0;
  sg.emit_stride = (unsigned long long)a->n_paths;
  sg.grad = table;
  sg.emit_phi = emit ? a->path_phi : nullptr;
  sg.emit_xi = emit ? a->path_xi : nullptr;
  sg.emit_steps = emit ? a->path_steps : nullptr;
  sg.h = a->dt;
  sg.sqrt_h = std::sqrt(a->dt);
  const double c0 = pv.exit_rule == PDD_EXIT_GOBET_MENOZZI ? 0.5826 : 0.0;
  sg.thr0 = c0 * sg.sqrt_h;
  sg.key0 = (uint32_t)a->seed;
  sg.key1 = a->stream_tag;
  sg.seed_hi = (uint32_t)(a->seed >> 32);
  sg.grid_n = grid_n;
  sg.max_steps = (int)max_steps;
  int blocks = 0;
  e = launch_paths(pv.kind, pv.precision, cv, pa, pv.num_sms, pv.stream, &blocks);
  if (e != cudaSuccess) return fail(e, "path kernel launch");
  StatPtrs sp{};
  sp.mean_phi = out->mean_phi;
  sp.var_phi = out->var_phi;
  sp.mean_cv = out->mean_cv;
  sp.var_cv = out->var_cv;
  sp.cov_phi_xi = out->cov_phi_xi;
  sp.var_xi = out->var_xi;
  sp.rho = out->rho;
  sp.se_phi = out->se_phi;
  sp.se_cv = out->se_cv;
  sp.vr = out->vr;
  sp.pred_speedup = out->pred_speedup;
  sp.mean_steps = out->mean_steps;
  sp.n_paths = (unsigned long long*)out->n_paths;
  sp.n_truncated = (unsigned long long*)out->n_truncated;
  e = launch_finalize(acc, (uint32_t)n, a->kappa > 0.0 ? a->kappa : 1.0, sp, pv.stream);
  if (e != cudaSuccess) return fail(e, "finalize launch");
  *pv.launches += 2;
  if (a->flags & PDD_FLAG_ASYNC) return PDD_OK;
  ScratchHeader h{};
  e = cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, pv.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(pv.stream);
  if (e != cudaSuccess) return fail(e, "cudaStreamSynchronize");
  if (h.err != 0u) return error_word_status(h.err, "pdd_estimate_nodes_noalloc");
  if (h.cursor < pa.total) {
    set_error("pdd_estimate_nodes_noalloc: internal error, %llu of %llu paths scheduled",
              h.cursor, pa.total);
    return PDD_ERR_CUDA;
  }
  if (h.trunc_total > 0) {
    set_error("pdd_estimate_nodes_noalloc: %llu paths hit max_steps = %lld", h.trunc_total,
              (long long)max_steps);
    return PDD_WARN_TRUNCATED;
  }
  return PDD_OK;
}
