"""ctypes binding of libpdd.so (C ABI in include/pdd.h).

The ``pdd_*`` functions below have the names and arguments of the C entry
points; they only marshal arguments and turn non-OK statuses into
``PddError``.  ``Context`` and ``Problem`` are small conveniences that take
torch tensors (device memory and streams come from PyTorch) and return the
per-node statistics as tensors.  Every step of the computation runs in the
library's CUDA kernels; if the library is missing this module raises -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpdd.so")
# the bounds-checked build of the same library (build.build(bounds=True))
LIB_BOUNDS_PATH = os.path.join(HERE, "libpdd_bounds.so")

# ---- constants mirrored from include/pdd.h --------------------------------
PDD_OK, PDD_ERR_INVALID, PDD_ERR_NOMEM, PDD_ERR_CUDA = 0, -1, -2, -3
PDD_ERR_TIMEOUT, PDD_ERR_BUSY, PDD_ERR_NOT_READY, PDD_ERR_CANCELLED = -4, -5, -6, -7
PDD_ERR_OVERFLOW, PDD_WARN_TRUNCATED, PDD_WARN_NOT_CONVERGED = -8, 1, 2
PDD_ERR_BOUNDS, PDD_ERR_DEADLINE = -9, -10
PDD_PROBLEM_CFG0_2D, PDD_PROBLEM_ANISO_2D, PDD_PROBLEM_CUBE_3D, PDD_PROBLEM_HARMONIC_2D = 0, 1, 2, 3
PDD_PROBLEM_PAPER_EX_2D = 4
PDD_EXIT_GOBET_MENOZZI, PDD_EXIT_NAIVE = 0, 1
PDD_Y_EULER, PDD_Y_EXP = 0, 1
PDD_PATH_FP32, PDD_PATH_FP64 = 0, 1
PDD_GRID_VALUES, PDD_GRID_GRADIENT = 0, 1
PDD_DTYPE_F32, PDD_DTYPE_F64 = 0, 1
PDD_CV_NONE, PDD_CV_EXACT = -1, -2
PDD_MAX_GRIDS = 8
PDD_FLAG_EMIT_PATHS, PDD_FLAG_ASYNC, PDD_FLAG_GRAPH = 1, 2, 4
PDD_MAX_LEVELS = 128
PDD_RECORD_WORDS = 16
PDD_MLMC_MAX_LEVELS = 16

STAT_FIELDS = ["mean_phi", "var_phi", "mean_cv", "var_cv", "cov_phi_xi", "var_xi", "rho",
               "se_phi", "se_cv", "vr", "pred_speedup", "mean_steps"]
COUNT_FIELDS = ["n_paths", "n_truncated"]


class PddError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"pdd status {status}: {message}")
        self.status = status


class ProblemDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("exit_rule", ctypes.c_int32),
                ("y_rule", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_steps", ctypes.c_int64)]


class GridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("kind", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("on_device", ctypes.c_int32), ("data", ctypes.c_void_p)]


class EstimateArgs(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("coords", ctypes.c_void_p * 3),
                ("coords_on_device", ctypes.c_int32), ("grid_id", ctypes.c_int32),
                ("n_paths", ctypes.c_int64), ("dt", ctypes.c_double), ("kappa", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("stream_tag", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("path_phi", ctypes.c_void_p),
                ("path_xi", ctypes.c_void_p), ("path_steps", ctypes.c_void_p)]


class NodeStats(ctypes.Structure):
    _fields_ = ([("on_device", ctypes.c_int32), ("reserved", ctypes.c_int32)]
                + [(f, ctypes.c_void_p) for f in STAT_FIELDS + COUNT_FIELDS])


class FitArgs(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("coords", ctypes.c_void_p * 3),
                ("grid_id", ctypes.c_int32), ("n_h", ctypes.c_int32), ("h_min", ctypes.c_double),
                ("h_max", ctypes.c_double), ("n_paths", ctypes.c_int64),
                ("delta", ctypes.c_double), ("q", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("stream_tag_base", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


FIT_FIELDS = ["E_phi", "beta", "V_phi", "alpha", "E_tau", "K", "cov_phi_psi", "V_psi",
              "rho_phi_psi"]


class FitOut(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in FIT_FIELDS] + [("cloud", ctypes.c_void_p)]


class ScheduleArgs(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64)] + [(f, ctypes.c_void_p) for f in
                ("K", "beta", "alpha", "V_phi", "V_psi", "rho_phi_psi")] + [
                (f, ctypes.c_double) for f in ("delta", "kappa", "a0", "min_speedup")]


class ServerDesc(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("quantum_path_steps", ctypes.c_int64), ("device_arena_bytes", ctypes.c_size_t),
                ("policy", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("deadline_s", ctypes.c_double), ("rate_hint", ctypes.c_double)]


PDD_SERVE_FAIR, PDD_SERVE_SHORTEST, PDD_SERVE_EARLIEST_DEADLINE = 0, 1, 2
PDD_ITER_AUTO, PDD_ITER_SHORT, PDD_ITER_LONG = 0, 1, 2


class MlmcArgs(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("coords", ctypes.c_void_p * 3),
                ("grid_id", ctypes.c_int32), ("min_levels", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("dt0", ctypes.c_double), ("n_pilot", ctypes.c_int64),
                ("target_rmse", ctypes.c_double), ("alpha", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("stream_tag_base", ctypes.c_uint32),
                ("reserved2", ctypes.c_uint32)]


class MlmcOut(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_void_p), ("variance", ctypes.c_void_p),
                ("extrapolated", ctypes.c_void_p), ("extrap_variance", ctypes.c_void_p),
                ("n_levels", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("n_paths", ctypes.c_int64 * PDD_MLMC_MAX_LEVELS),
                ("var_mean", ctypes.c_double * PDD_MLMC_MAX_LEVELS),
                ("cost_mean", ctypes.c_double * PDD_MLMC_MAX_LEVELS),
                ("corr_rms", ctypes.c_double * PDD_MLMC_MAX_LEVELS),
                ("bias_estimate", ctypes.c_double), ("path_steps", ctypes.c_int64)]


SERVER_STAT_FIELDS = ["submitted", "admitted", "rejected_busy", "rejected_invalid",
                      "rejected_nomem", "completed", "cancelled", "failed", "launches", "pending",
                      "active", "path_steps", "rejected_deadline", "completed_path_steps",
                      "backlog_path_steps", "rate_path_steps_per_s"]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in SERVER_STAT_FIELDS]


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("pdd_abi_version", ctypes.c_int, []),
    ("pdd_last_error", ctypes.c_char_p, []),
    ("pdd_ctx_create", ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    ("pdd_ctx_destroy", None, [ctypes.c_void_p]),
    ("pdd_ctx_set_stream", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("pdd_ctx_set_timing", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("pdd_ctx_kernel_time", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int64]),
    ("pdd_ctx_launch_count", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    ("pdd_ctx_graph_count", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    ("pdd_ctx_set_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("pdd_ctx_abort", ctypes.c_int, [ctypes.c_void_p]),
    ("pdd_ctx_set_iteration", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("pdd_ctx_set_claim", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("pdd_ctx_get_claim", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("pdd_ctx_get_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    ("pdd_estimate_levels", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                           ctypes.POINTER(EstimateArgs),
                                           ctypes.POINTER(NodeStats), ctypes.c_uint32]),
    ("pdd_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EstimateArgs),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_double)]),
    ("pdd_create_problem", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ProblemDesc),
                                          ctypes.POINTER(ctypes.c_void_p)]),
    ("pdd_destroy_problem", ctypes.c_int, [ctypes.c_void_p]),
    ("pdd_set_control_grid", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(GridDesc)]),
    ("pdd_estimate_nodes", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EstimateArgs),
                                          ctypes.POINTER(NodeStats)]),
    ("pdd_accumulate", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EstimateArgs),
                                      ctypes.c_uint64, ctypes.c_void_p]),
    ("pdd_finalize_records", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_double, ctypes.POINTER(NodeStats)]),
    ("pdd_records_merge", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    ("pdd_fit_constants", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(FitArgs),
                                         ctypes.POINTER(FitOut)]),
    ("pdd_schedule", ctypes.c_int, [ctypes.POINTER(ScheduleArgs), ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("pdd_debug_bounds_selftest", ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
    ("pdd_balanced_plan", ctypes.c_int, [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    ("pdd_schedule_predict", ctypes.c_int, [ctypes.POINTER(ScheduleArgs), ctypes.c_double,
                                            ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    ("pdd_estimate_coupled", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EstimateArgs),
                                            ctypes.POINTER(NodeStats), ctypes.POINTER(NodeStats)]),
    ("pdd_accumulate_coupled", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EstimateArgs),
                                              ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    ("pdd_mlmc_allocate", ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_double, ctypes.c_void_p]),
    ("pdd_mlmc", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(MlmcArgs),
                                ctypes.POINTER(MlmcOut)]),
    ("pdd_server_create", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerDesc),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    ("pdd_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(EstimateArgs),
                                  ctypes.POINTER(ctypes.c_uint64)]),
    ("pdd_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(NodeStats),
                                ctypes.c_int]),
    ("pdd_cancel", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("pdd_server_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    ("pdd_server_inject_fault", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("pdd_server_destroy", None, [ctypes.c_void_p]),
    ("pdd_estimate_nodes_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EstimateArgs),
                                                  ctypes.POINTER(NodeStats)]),
    ("pdd_debug_philox", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64]),
    ("pdd_debug_philox_curand", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_int64]),
    ("pdd_debug_normals", ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("pdd_debug_issue_rate", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]),
]


def lib():
    """Load libpdd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
            l = ctypes.CDLL(LIB_PATH)
            for name, res, args in _SIGS:
                fn = getattr(l, name)
                fn.restype = res
                fn.argtypes = args
            _lib = l
        return _lib


def bounds_selftest() -> int:
    """Error word of the bounds-check self-test (62 in the bounds-checked
    build, 0 in the release build)."""
    bits = ctypes.c_uint32(0)
    _check(lib().pdd_debug_bounds_selftest(ctypes.byref(bits)))
    return bits.value


def _check(status: int) -> int:
    if status < 0:
        raise PddError(status, lib().pdd_last_error().decode(errors="replace"))
    return status


# ---- thin wrappers with the C names -----------------------------------------
def pdd_abi_version() -> int:
    return lib().pdd_abi_version()


def pdd_last_error() -> str:
    return lib().pdd_last_error().decode(errors="replace")


def pdd_ctx_create(device: int, cuda_stream: int | None, mem_budget: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().pdd_ctx_create(device, cuda_stream, mem_budget, ctypes.byref(h)))
    return h.value


def pdd_ctx_destroy(ctx: int) -> None:
    lib().pdd_ctx_destroy(ctx)


def pdd_ctx_set_stream(ctx: int, cuda_stream: int | None) -> None:
    _check(lib().pdd_ctx_set_stream(ctx, cuda_stream))


def pdd_ctx_set_timing(ctx: int, enable: bool) -> None:
    _check(lib().pdd_ctx_set_timing(ctx, int(enable)))


def pdd_ctx_kernel_time(ctx: int, capacity: int = 4096) -> tuple[float, int, list[float]]:
    """(total ms, launches, per-launch ms) of the timed path-kernel launches."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    per = (ctypes.c_double * capacity)()
    _check(lib().pdd_ctx_kernel_time(ctx, ctypes.byref(ms), ctypes.byref(n), per, capacity))
    return ms.value, n.value, list(per[: min(n.value, capacity)])


def pdd_ctx_launch_count(ctx: int) -> int:
    n = ctypes.c_int64()
    _check(lib().pdd_ctx_launch_count(ctx, ctypes.byref(n)))
    return n.value


def pdd_ctx_graph_count(ctx: int) -> int:
    n = ctypes.c_int64()
    _check(lib().pdd_ctx_graph_count(ctx, ctypes.byref(n)))
    return n.value


def pdd_ctx_set_launch(ctx: int, block_threads: int, max_blocks: int) -> None:
    _check(lib().pdd_ctx_set_launch(ctx, block_threads, max_blocks))


def pdd_estimate_levels(problem: int, levels, outs, flags: int = 0) -> int:
    """levels: sequence of EstimateArgs; outs: sequence of NodeStats."""
    n = len(levels)
    la = (EstimateArgs * n)(*levels)
    lo = (NodeStats * n)(*outs)
    return _check(lib().pdd_estimate_levels(problem, n, la, lo, flags))


def pdd_autotune(problem: int, sample: EstimateArgs) -> tuple[int, int, float]:
    t, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().pdd_autotune(problem, ctypes.byref(sample), ctypes.byref(t), ctypes.byref(b),
                              ctypes.byref(ms)))
    return t.value, b.value, ms.value


def pdd_create_problem(ctx: int, desc: ProblemDesc) -> int:
    h = ctypes.c_void_p()
    _check(lib().pdd_create_problem(ctx, ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def pdd_destroy_problem(problem: int) -> None:
    _check(lib().pdd_destroy_problem(problem))


def pdd_set_control_grid(problem: int, grid_id: int, desc: GridDesc) -> None:
    _check(lib().pdd_set_control_grid(problem, grid_id, ctypes.byref(desc)))


def pdd_estimate_nodes(problem: int, args: EstimateArgs, out: NodeStats) -> int:
    """Returns PDD_OK or PDD_WARN_TRUNCATED; raises on errors."""
    return _check(lib().pdd_estimate_nodes(problem, ctypes.byref(args), ctypes.byref(out)))


PDD_NOALLOC_MAX_NODES = 4096


def pdd_accumulate(problem: int, args: EstimateArgs, path_offset: int, records_ptr: int) -> int:
    return _check(lib().pdd_accumulate(problem, ctypes.byref(args), path_offset, records_ptr))


def pdd_finalize_records(ctx: int, records_ptr: int, n_nodes: int, kappa: float,
                         out: NodeStats) -> None:
    _check(lib().pdd_finalize_records(ctx, records_ptr, n_nodes, kappa, ctypes.byref(out)))


def pdd_records_merge(dst_ptr: int, src_ptr: int, n_nodes: int) -> None:
    _check(lib().pdd_records_merge(dst_ptr, src_ptr, n_nodes))


def pdd_fit_constants(problem: int, args: FitArgs, out: FitOut) -> int:
    return _check(lib().pdd_fit_constants(problem, ctypes.byref(args), ctypes.byref(out)))


def pdd_schedule(K, beta, alpha, V_phi, V_psi, rho, delta: float, kappa: float, a0: float,
                 min_speedup: float = 1.5, max_levels: int = 20):
    """Algorithm 4 (host computation in the library): returns (a, speedup)
    with a[0] = a0 < a[1] < ... and the predicted speedup of every step."""
    import numpy as np
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (K, beta, alpha, V_phi, V_psi, rho)]
    args = ScheduleArgs(arrs[0].size, *[x.ctypes.data for x in arrs], delta, kappa, a0,
                        min_speedup)
    a = np.zeros(max_levels + 1)
    sp = np.zeros(max_levels + 1)
    n = ctypes.c_int()
    _check(lib().pdd_schedule(ctypes.byref(args), a.ctypes.data, sp.ctypes.data, max_levels,
                              ctypes.byref(n)))
    J = n.value
    n_sp = J + 1 if J < max_levels else J
    return a[: J + 1].copy(), sp[:n_sp].copy()


def pdd_balanced_plan(a: float, beta, var, q: float = 2.0, delta: float = 1.0,
                      h_min: float = 1e-7, h_max: float = 0.1, n_min: int = 2,
                      n_max: int = (1 << 32) - 1):
    """Balanced time step and path count per node (eq. F:N_y_h): returns
    (h, n_paths) numpy arrays."""
    import numpy as np
    b = np.ascontiguousarray(beta, dtype=np.float64)
    v = np.ascontiguousarray(var, dtype=np.float64)
    h = np.zeros(b.size)
    n = np.zeros(b.size, dtype=np.int64)
    _check(lib().pdd_balanced_plan(b.size, a, q, delta, b.ctypes.data, v.ctypes.data, h_min,
                                   h_max, n_min, n_max, h.ctypes.data, n.ctypes.data))
    return h, n


def pdd_schedule_predict(K, beta, alpha, V_phi, V_psi, rho, delta: float, a: float, aj: float):
    """Per-node predicted rho^2[phi_h, xi_h] and path-step cost of the level at
    tolerance aj using the control variate of the level at tolerance a
    (a <= 0: plain level); returns (rho2, cost)."""
    import numpy as np
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (K, beta, alpha, V_phi, V_psi, rho)]
    args = ScheduleArgs(arrs[0].size, *[x.ctypes.data for x in arrs], delta, 1.0, aj, 1.5)
    rho2 = np.zeros(arrs[0].size)
    cost = np.zeros(arrs[0].size)
    _check(lib().pdd_schedule_predict(ctypes.byref(args), a, aj, rho2.ctypes.data,
                                      cost.ctypes.data))
    return rho2, cost


def pdd_estimate_coupled(problem: int, args: EstimateArgs, out_fine: NodeStats,
                         out_diff: NodeStats) -> int:
    return _check(lib().pdd_estimate_coupled(problem, ctypes.byref(args), ctypes.byref(out_fine),
                                             ctypes.byref(out_diff)))


def pdd_accumulate_coupled(problem: int, args: EstimateArgs, path_offset: int, rec_fine_ptr: int,
                           rec_diff_ptr: int) -> int:
    return _check(lib().pdd_accumulate_coupled(problem, ctypes.byref(args), path_offset,
                                               rec_fine_ptr, rec_diff_ptr))


def pdd_mlmc_allocate(var_mean, cost_mean, target_rmse: float):
    """Sample counts of the multilevel levels (host computation in the
    library); returns (status, counts)."""
    import numpy as np
    V = np.ascontiguousarray(var_mean, dtype=np.float64)
    C = np.ascontiguousarray(cost_mean, dtype=np.float64)
    N = np.zeros(V.size, dtype=np.int64)
    st = _check(lib().pdd_mlmc_allocate(V.size, V.ctypes.data, C.ctypes.data, target_rmse,
                                        N.ctypes.data))
    return st, N


def pdd_mlmc(problem: int, args: MlmcArgs, out: MlmcOut) -> int:
    """PDD_OK, PDD_WARN_NOT_CONVERGED or PDD_WARN_TRUNCATED; raises on errors."""
    return _check(lib().pdd_mlmc(problem, ctypes.byref(args), ctypes.byref(out)))


def pdd_server_create(ctx: int, desc: ServerDesc | None = None) -> int:
    h = ctypes.c_void_p()
    _check(lib().pdd_server_create(ctx, ctypes.byref(desc) if desc is not None else None,
                                   ctypes.byref(h)))
    return h.value


def pdd_submit(server: int, problem: int, args: EstimateArgs) -> int:
    t = ctypes.c_uint64()
    _check(lib().pdd_submit(server, problem, ctypes.byref(args), ctypes.byref(t)))
    return t.value


def pdd_poll(server: int, ticket: int, out: NodeStats, timeout_us: int) -> int:
    """Returns the raw status (PDD_OK, PDD_ERR_NOT_READY, PDD_ERR_TIMEOUT,
    PDD_ERR_CANCELLED or another error) without raising."""
    return lib().pdd_poll(server, ticket, ctypes.byref(out), timeout_us)


def pdd_cancel(server: int, ticket: int) -> None:
    _check(lib().pdd_cancel(server, ticket))


def pdd_server_get_stats(server: int) -> dict:
    st = ServerStats()
    _check(lib().pdd_server_get_stats(server, ctypes.byref(st)))
    return {f: getattr(st, f) for f in SERVER_STAT_FIELDS}


def pdd_server_inject_fault(server: int, fault: int) -> None:
    _check(lib().pdd_server_inject_fault(server, fault))


def pdd_server_destroy(server: int) -> None:
    lib().pdd_server_destroy(server)


def pdd_estimate_nodes_noalloc(problem: int, args: EstimateArgs, out: NodeStats) -> int:
    """Allocation-free estimate for callers that cannot let the library
    allocate device memory (device inputs and outputs only, at most
    PDD_NOALLOC_MAX_NODES nodes; see include/pdd.h).  Returns PDD_OK or
    PDD_WARN_TRUNCATED; raises on errors."""
    return _check(lib().pdd_estimate_nodes_noalloc(problem, ctypes.byref(args),
                                                   ctypes.byref(out)))


def pdd_debug_philox(ctr_ptr: int, key_ptr: int, out_ptr: int, n: int) -> None:
    _check(lib().pdd_debug_philox(ctr_ptr, key_ptr, out_ptr, n))


def pdd_debug_philox_curand(ctr_ptr: int, key_ptr: int, out_ptr: int, n: int) -> None:
    _check(lib().pdd_debug_philox_curand(ctr_ptr, key_ptr, out_ptr, n))


def pdd_debug_normals(seed: int, tag: int, node: int, path: int, first: int, count: int,
                      precision: int, out_f32: int | None, out_f64: int | None) -> None:
    _check(lib().pdd_debug_normals(seed, tag, node, path, first, count, precision, out_f32,
                                   out_f64))


# ---- torch conveniences ------------------------------------------------------
def _torch():
    import torch
    return torch


class Context:
    """A library context on one device, enqueuing on a torch stream."""

    def __init__(self, device: int = 0, stream=None, mem_budget: int = 0):
        """stream: a torch.cuda.Stream to enqueue on; by default a new
        (non-default) torch stream, exposed as ``self.stream`` so callers can
        order their own work and CUDA events on it."""
        torch = _torch()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.Stream(device)
        if self.stream.cuda_stream == 0:
            raise ValueError("pass a non-default stream (handle 0 means 'library-owned')")
        self._lib = lib()
        self.handle = pdd_ctx_create(device, self.stream.cuda_stream, mem_budget)
        # Handles of the servers and problems still open on this context, held
        # here and by those objects (a plain shared dict, not weak references,
        # which the garbage collector clears before it runs the finalisers of a
        # reference cycle): close() destroys what is still open first, and a
        # later close() of such an object is a no-op.  Each entry keeps the
        # library the object was created with.
        self._owned = {"servers": {}, "problems": {}}

    def set_stream(self, stream) -> None:
        pdd_ctx_set_stream(self.handle, stream.cuda_stream)
        self.stream = stream

    def set_timing(self, enable: bool) -> None:
        pdd_ctx_set_timing(self.handle, enable)

    def kernel_time(self) -> tuple[float, int, list[float]]:
        return pdd_ctx_kernel_time(self.handle)

    def launch_count(self) -> int:
        return pdd_ctx_launch_count(self.handle)

    def graph_count(self) -> int:
        return pdd_ctx_graph_count(self.handle)

    def finalize_records(self, records, kappa: float = 1.0) -> dict:
        """Per-node statistics (CUDA tensors) of device records."""
        torch = _torch()
        n = records.shape[0]
        res, out = {}, NodeStats()
        out.on_device = 1
        for f in STAT_FIELDS:
            res[f] = torch.empty(n, dtype=torch.float64, device=records.device)
            setattr(out, f, res[f].data_ptr())
        for f in COUNT_FIELDS:
            res[f] = torch.empty(n, dtype=torch.int64, device=records.device)
            setattr(out, f, res[f].data_ptr())
        torch.cuda.synchronize()
        pdd_finalize_records(self.handle, records.data_ptr(), n, kappa, out)
        return res

    def set_launch(self, block_threads: int = 0, max_blocks: int = 0) -> None:
        pdd_ctx_set_launch(self.handle, block_threads, max_blocks)

    def set_iteration(self, mode: int) -> None:
        """Euler steps per iteration: PDD_ITER_AUTO / _SHORT / _LONG."""
        _check(self._lib.pdd_ctx_set_iteration(self.handle, mode))

    def set_claim(self, paths_per_lane: int) -> None:
        """Paths per lane a warp claims from the cursor at once (0: automatic)."""
        _check(self._lib.pdd_ctx_set_claim(self.handle, paths_per_lane))

    def get_claim(self) -> int:
        v = ctypes.c_int()
        _check(self._lib.pdd_ctx_get_claim(self.handle, ctypes.byref(v)))
        return v.value

    def get_launch(self) -> tuple[int, int, int]:
        """(block_threads, max_blocks, iteration mode) of the context."""
        v = [ctypes.c_int() for _ in range(3)]
        _check(self._lib.pdd_ctx_get_launch(self.handle, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def abort(self) -> None:
        """Stop the work in flight on this context (pdd_ctx_abort); safe to
        call from another thread while an estimate runs."""
        _check(self._lib.pdd_ctx_abort(self.handle))

    def close(self) -> None:
        if self.handle:
            for kind, fn in (("servers", "pdd_server_destroy"),
                             ("problems", "pdd_destroy_problem")):
                for h, l in list(self._owned[kind].items()):
                    getattr(l, fn)(h)
                self._owned[kind].clear()
            self._lib.pdd_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _close_owned(owned: dict, handle, fn: str) -> None:
    """Destroy `handle` unless its context already did (see Context)."""
    l = owned.pop(handle, None)
    if l is not None:
        getattr(l, fn)(handle)


class Problem:
    """A built-in problem with up to PDD_MAX_GRIDS control grids."""

    def __init__(self, ctx: Context, kind: int, exit_rule: int = PDD_EXIT_GOBET_MENOZZI,
                 y_rule: int = PDD_Y_EULER, precision: int = PDD_PATH_FP32, max_steps: int = 0):
        self.ctx = ctx
        self.kind = kind
        self.dim = 3 if kind == PDD_PROBLEM_CUBE_3D else 2
        self.precision = precision
        self.handle = pdd_create_problem(ctx.handle, ProblemDesc(kind, exit_rule, y_rule,
                                                                 precision, max_steps))
        self._owned = ctx._owned["problems"]
        self._owned[self.handle] = ctx._lib

    def set_control_grid(self, grid_id: int, data, kind: int = PDD_GRID_VALUES) -> None:
        """data: numpy array or torch tensor (float32/float64, host or CUDA)
        of shape (n,)*D (VALUES) or (n,)*D + (D,) (GRADIENT), x fastest."""
        torch = _torch()
        import numpy as np
        if isinstance(data, np.ndarray):
            data = torch.from_numpy(np.ascontiguousarray(data))
        data = data.contiguous()
        if data.dtype not in (torch.float32, torch.float64):
            raise TypeError("grid data must be float32 or float64")
        n = data.shape[0]
        desc = GridDesc(n, kind, PDD_DTYPE_F32 if data.dtype == torch.float32 else PDD_DTYPE_F64,
                        int(data.is_cuda), data.data_ptr())
        pdd_set_control_grid(self.handle, grid_id, desc)

    def _prepare(self, nodes, n_paths, dt, grid_id, seed, stream_tag, kappa, emit_paths,
                 device_out, host_inputs, pin_host):
        torch = _torch()
        import numpy as np
        dev = torch.device("cuda", self.ctx.device)
        if isinstance(nodes, (list, tuple)):
            # pre-split SoA columns (float32, contiguous), used as given
            cols = list(nodes)
            n = cols[0].shape[0]
            if any(c.is_cuda == host_inputs or c.dtype != torch.float32 for c in cols):
                raise ValueError("columns must be float32 and on the side host_inputs says")
        else:
            if isinstance(nodes, np.ndarray):
                nodes = torch.from_numpy(np.ascontiguousarray(nodes, dtype=np.float32))
            nodes = nodes.to(torch.float32)
            n = nodes.shape[0]
            if host_inputs:
                cols = [nodes[:, j].contiguous().cpu() for j in range(self.dim)]
            else:
                cols = [nodes[:, j].contiguous().to(dev) for j in range(self.dim)]
        args = EstimateArgs()
        args.n_nodes = n
        for j in range(3):
            args.coords[j] = cols[j].data_ptr() if j < self.dim else None
        args.coords_on_device = 0 if host_inputs else 1
        args.grid_id = grid_id
        args.n_paths = n_paths
        args.dt = dt
        args.kappa = kappa
        args.seed = seed
        args.stream_tag = stream_tag
        args.flags = PDD_FLAG_EMIT_PATHS if emit_paths else 0
        res = {}
        if emit_paths:
            res["phi"] = torch.empty((n, n_paths), dtype=torch.float32, device=dev)
            res["xi"] = torch.empty((n, n_paths), dtype=torch.float32, device=dev)
            res["steps"] = torch.empty((n, n_paths), dtype=torch.int32, device=dev)
            args.path_phi = res["phi"].data_ptr()
            args.path_xi = res["xi"].data_ptr()
            args.path_steps = res["steps"].data_ptr()
        out = NodeStats()
        out.on_device = 1 if device_out else 0
        odev = dev if device_out else torch.device("cpu")
        pin = (not device_out) and pin_host
        for f in STAT_FIELDS:
            res[f] = torch.empty(n, dtype=torch.float64, device=odev, pin_memory=pin)
            setattr(out, f, res[f].data_ptr())
        for f in COUNT_FIELDS:
            res[f] = torch.empty(n, dtype=torch.int64, device=odev, pin_memory=pin)
            setattr(out, f, res[f].data_ptr())
        res["_keep"] = cols  # inputs must outlive an asynchronous call
        return args, out, res

    def estimate(self, nodes, n_paths: int, dt: float, grid_id: int = PDD_CV_NONE,
                 seed: int = 1234, stream_tag: int = 0, kappa: float = 1.0,
                 emit_paths: bool = False, device_out: bool = True, async_: bool = False,
                 host_inputs: bool = False, pin_host: bool = False):
        """Estimate every node.  nodes: (n, D) tensor or array of coordinates,
        or a list of D contiguous float32 columns.  Returns a dict of per-node
        tensors (and per-path tensors when emit_paths), plus 'status'.
        host_inputs/device_out choose host or device buffers for the C call;
        pin_host allocates host outputs in page-locked memory."""
        args, out, res = self._prepare(nodes, n_paths, dt, grid_id, seed, stream_tag, kappa,
                                       emit_paths, device_out, host_inputs, pin_host)
        if async_:
            args.flags |= PDD_FLAG_ASYNC
        res["status"] = pdd_estimate_nodes(self.handle, args, out)
        return res

    def estimate_levels(self, levels, async_: bool = False, graph: bool = False,
                        device_out: bool = True, host_inputs: bool = False):
        """Several levels in one launch.  levels: list of dicts with the
        keyword arguments of estimate() (nodes, n_paths, dt, grid_id, seed,
        stream_tag, kappa, emit_paths).  Returns (status, [per-level dict])."""
        prepared = []
        for lv in levels:
            prepared.append(self._prepare(lv["nodes"], lv["n_paths"], lv["dt"],
                                          lv.get("grid_id", PDD_CV_NONE), lv.get("seed", 1234),
                                          lv.get("stream_tag", 0), lv.get("kappa", 1.0),
                                          lv.get("emit_paths", False), device_out, host_inputs,
                                          False))
        flags = (PDD_FLAG_ASYNC if async_ else 0) | (PDD_FLAG_GRAPH if graph else 0)
        st = pdd_estimate_levels(self.handle, [p[0] for p in prepared], [p[1] for p in prepared],
                                 flags)
        return st, [p[2] for p in prepared]

    def estimate_coupled(self, nodes, n_paths: int, dt: float, grid_id: int = PDD_CV_NONE,
                         seed: int = 1234, stream_tag: int = 0, emit_paths: bool = False):
        """Multilevel coupling (fine dt/2, coarse dt).  Returns (fine, diff)
        dicts of per-node CUDA tensors; with emit_paths, fine['phi'] etc. hold
        the fine paths and diff['phi'] etc. the coarse paths."""
        torch = _torch()
        args, out_f, res_f = self._prepare(nodes, n_paths, dt, grid_id, seed, stream_tag, 1.0,
                                           False, True, False, False)
        _, out_d, res_d = self._prepare(nodes, n_paths, dt, grid_id, seed, stream_tag, 1.0,
                                        False, True, False, False)
        if emit_paths:
            n = args.n_nodes
            dev = torch.device("cuda", self.ctx.device)
            phi = torch.empty((2, n, n_paths), dtype=torch.float32, device=dev)
            xi = torch.empty((2, n, n_paths), dtype=torch.float32, device=dev)
            st = torch.empty((2, n, n_paths), dtype=torch.int32, device=dev)
            args.flags |= PDD_FLAG_EMIT_PATHS
            args.path_phi, args.path_xi, args.path_steps = phi.data_ptr(), xi.data_ptr(), st.data_ptr()
            res_f.update(phi=phi[0], xi=xi[0], steps=st[0])
            res_d.update(phi=phi[1], xi=xi[1], steps=st[1])
        res_f["status"] = pdd_estimate_coupled(self.handle, args, out_f, out_d)
        return res_f, res_d

    def accumulate(self, nodes, n_paths: int, dt: float, records, path_offset: int = 0,
                   grid_id: int = PDD_CV_NONE, seed: int = 1234, stream_tag: int = 0):
        """Add paths path_offset .. path_offset+n_paths-1 of every node into
        `records` (int64 CUDA tensor of shape (n_nodes, PDD_RECORD_WORDS))."""
        args, _, keep = self._prepare(nodes, n_paths, dt, grid_id, seed, stream_tag, 1.0, False,
                                      True, False, False)
        return pdd_accumulate(self.handle, args, path_offset, records.data_ptr())

    def accumulate_coupled(self, nodes, n_paths: int, dt: float, rec_fine, rec_diff,
                           path_offset: int = 0, grid_id: int = PDD_CV_NONE, seed: int = 1234,
                           stream_tag: int = 0):
        """Add coupled pairs path_offset .. path_offset+n_paths-1 of every node
        into the fine / difference records (int64 CUDA tensors (n_nodes,
        PDD_RECORD_WORDS))."""
        args, _, keep = self._prepare(nodes, n_paths, dt, grid_id, seed, stream_tag, 1.0, False,
                                      True, False, False)
        return pdd_accumulate_coupled(self.handle, args, path_offset, rec_fine.data_ptr(),
                                      rec_diff.data_ptr())

    def mlmc(self, nodes, dt0: float, target_rmse: float, grid_id: int = PDD_CV_NONE,
             min_levels: int = 2, max_levels: int = 8, n_pilot: int = 1000, alpha: float = 1.0,
             seed: int = 1234, stream_tag_base: int = 0):
        """Multilevel Monte Carlo estimate of the nodal values (pdd_mlmc).
        Returns a dict: status, per-node numpy arrays estimate / variance /
        extrapolated / extrap_variance, and the per-level counts and moments."""
        import numpy as np
        torch = _torch()
        dev = torch.device("cuda", self.ctx.device)
        nodes = np.asarray(nodes, dtype=np.float32).reshape(-1, self.dim)
        cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).to(dev)
                for j in range(self.dim)]
        n = nodes.shape[0]
        a = MlmcArgs()
        a.n_nodes = n
        for j in range(3):
            a.coords[j] = cols[j].data_ptr() if j < self.dim else None
        a.grid_id, a.min_levels, a.max_levels = grid_id, min_levels, max_levels
        a.dt0, a.n_pilot, a.target_rmse, a.alpha = dt0, n_pilot, target_rmse, alpha
        a.seed, a.stream_tag_base = seed, stream_tag_base
        arrs = {k: np.zeros(n) for k in ("estimate", "variance", "extrapolated", "extrap_variance")}
        o = MlmcOut()
        for k, v in arrs.items():
            setattr(o, k, v.ctypes.data)
        st = pdd_mlmc(self.handle, a, o)
        L = o.n_levels
        return dict(status=st, n_levels=L, rounds=o.rounds, bias_estimate=o.bias_estimate,
                    path_steps=o.path_steps, n_paths=np.array(o.n_paths[:L], dtype=np.int64),
                    var_mean=np.array(o.var_mean[:L]), cost_mean=np.array(o.cost_mean[:L]),
                    corr_rms=np.array(o.corr_rms[:L]), **arrs)

    def fit_constants(self, nodes, n_paths: int, h_min: float, h_max: float, n_h: int,
                      grid_id: int = PDD_CV_NONE, delta: float = 1.0, q: float = 2.0,
                      seed: int = 1234, stream_tag_base: int = 0):
        """Algorithm 3 on the GPU; returns a dict of per-node numpy arrays and
        the cloud (n_nodes, n_h, 6)."""
        import numpy as np
        torch = _torch()
        dev = torch.device("cuda", self.ctx.device)
        nodes = np.asarray(nodes, dtype=np.float32).reshape(-1, self.dim)
        cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).to(dev)
                for j in range(self.dim)]
        n = nodes.shape[0]
        a = FitArgs()
        a.n_nodes = n
        for j in range(3):
            a.coords[j] = cols[j].data_ptr() if j < self.dim else None
        a.grid_id, a.n_h, a.h_min, a.h_max = grid_id, n_h, h_min, h_max
        a.n_paths, a.delta, a.q, a.seed, a.stream_tag_base = n_paths, delta, q, seed, stream_tag_base
        res = {f: np.zeros(n) for f in FIT_FIELDS}
        res["cloud"] = np.zeros((n, n_h, 6))
        out = FitOut()
        for f in FIT_FIELDS + ["cloud"]:
            setattr(out, f, res[f].ctypes.data)
        torch.cuda.synchronize()
        res["status"] = pdd_fit_constants(self.handle, a, out)
        return res

    def autotune(self, nodes, n_paths: int, dt: float, grid_id: int = PDD_CV_NONE,
                 seed: int = 1234, stream_tag: int = 0):
        """Pick the fastest launch shape for this kind of call; returns
        (block_threads, max_blocks, ms)."""
        args, _, keep = self._prepare(nodes, n_paths, dt, grid_id, seed, stream_tag, 1.0, False,
                                      True, False, False)
        return pdd_autotune(self.handle, args)

    def estimate_on_stream(self, *a, **kw):
        """estimate() with the output tensors allocated on the context's
        stream (so torch's caching allocator orders their reuse after the
        library's kernels)."""
        torch = _torch()
        with torch.cuda.stream(self.ctx.stream):
            return self.estimate(*a, **kw)

    def close(self) -> None:
        if self.handle:
            _close_owned(self._owned, self.handle, "pdd_destroy_problem")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server on a context (see pdd_server_create)."""

    def __init__(self, ctx: Context, max_active: int = 0, max_queue: int = 0,
                 quantum_path_steps: int = 0, device_arena_bytes: int = 0,
                 policy: int = PDD_SERVE_FAIR, deadline_s: float = 0.0,
                 rate_hint: float = 0.0):
        self.ctx = ctx
        self.handle = pdd_server_create(ctx.handle, ServerDesc(max_active, max_queue,
                                                               quantum_path_steps,
                                                               device_arena_bytes, policy, 0,
                                                               deadline_s, rate_hint))
        self._owned = ctx._owned["servers"]
        self._owned[self.handle] = ctx._lib

    def submit(self, problem: Problem, nodes, n_paths: int, dt: float,
               grid_id: int = PDD_CV_NONE, seed: int = 1234, stream_tag: int = 0,
               kappa: float = 1.0, flags: int = 0) -> int:
        """nodes: (n, D) numpy array (host); the library copies it."""
        import numpy as np
        nodes = np.asarray(nodes, dtype=np.float32).reshape(-1, problem.dim)
        cols = [np.ascontiguousarray(nodes[:, j]) for j in range(problem.dim)]
        a = EstimateArgs()
        a.n_nodes = nodes.shape[0]
        for j in range(3):
            a.coords[j] = cols[j].ctypes.data if j < problem.dim else None
        a.coords_on_device = 0
        a.grid_id = grid_id
        a.n_paths = n_paths
        a.dt = dt
        a.kappa = kappa
        a.seed = seed
        a.stream_tag = stream_tag
        a.flags = flags
        return pdd_submit(self.handle, problem.handle, a)

    def poll(self, ticket: int, n_nodes: int, timeout_us: int = 0):
        """(status, results) -- results is a dict of numpy arrays when status
        is PDD_OK, else None."""
        import numpy as np
        res = {f: np.empty(n_nodes) for f in STAT_FIELDS}
        res.update({f: np.empty(n_nodes, dtype=np.int64) for f in COUNT_FIELDS})
        out = NodeStats()
        out.on_device = 0
        for f in STAT_FIELDS + COUNT_FIELDS:
            setattr(out, f, res[f].ctypes.data if n_nodes else None)
        st = pdd_poll(self.handle, ticket, out, min(int(timeout_us), 2**31 - 1))
        return st, (res if st == PDD_OK else None)

    def cancel(self, ticket: int) -> None:
        pdd_cancel(self.handle, ticket)

    def stats(self) -> dict:
        return pdd_server_get_stats(self.handle)

    def inject_fault(self, fault: int) -> None:
        pdd_server_inject_fault(self.handle, fault)

    def close(self) -> None:
        if self.handle:
            _close_owned(self._owned, self.handle, "pdd_server_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pdd_debug_issue_rate(kind: int, iters: int) -> tuple[float, float]:
    """Issue-rate probe of one instruction class on the current device:
    returns (thread-operations per second, kernel milliseconds)."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().pdd_debug_issue_rate(kind, iters, ctypes.byref(ops), ctypes.byref(ms)))
    return ops.value, ms.value
