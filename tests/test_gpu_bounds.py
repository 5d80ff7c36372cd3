"""The bounds-checked build of the library (libpdd_bounds.so, compiled with
-DPDD_DEBUG_BOUNDS=1) on valid inputs.

Its kernels check every control-grid cell, flat path index, segment, node,
record slot, exit-ring fill and per-path output index against its buffer; a
violation sets a bit of the launch's error word (the guarded access is
skipped, nothing traps) and the call returns PDD_ERR_BOUNDS.  It stands in
for a memory checker, which this environment does not offer.

* a self-test shows every check can fire (without any out-of-range access);
* the parity cases (FP32 and FP64 paths), a multi-segment launch and the
  multilevel coupling run with the error word zero, and the bounds-checked
  paths still match the oracle.
"""
import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W
from parity import PATH_FRAC, compare_paths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bounds_env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    build.build(bounds=True)
    oracle.build()
    release_bits = pdd.bounds_selftest()
    saved = (pdd._lib, pdd.LIB_PATH)
    pdd._lib, pdd.LIB_PATH = None, pdd.LIB_BOUNDS_PATH
    ctx = pdd.Context(0)
    yield {"torch": torch, "oracle": oracle, "pdd": pdd, "ctx": ctx,
           "release_bits": release_bits}
    ctx.close()
    pdd._lib, pdd.LIB_PATH = saved


def test_every_check_can_fire(bounds_env):
    pdd = bounds_env["pdd"]
    assert bounds_env["release_bits"] == 0
    assert pdd.bounds_selftest() == 62
    assert pdd.lib()._name.endswith("libpdd_bounds.so")


def test_parity_cases_in_bounds(bounds_env):
    from test_gpu_parity import CASES, _run_case
    for case in CASES:
        for precision in (0, 1):
            g, ref = _run_case(bounds_env, case, precision=precision)
            assert g["status"] in (0, bounds_env["pdd"].PDD_WARN_TRUNCATED), case[0]
            if precision == 0:
                p = compare_paths(g, ref)
                assert p["frac_ok"] >= PATH_FRAC, (case[0], p)


def test_levels_and_coupling_in_bounds(bounds_env):
    torch, pdd = bounds_env["torch"], bounds_env["pdd"]
    prob = pdd.Problem(bounds_env["ctx"], pdd.PDD_PROBLEM_CFG0_2D)
    for slot, eps in enumerate((1e-1, 1e-2)):
        prob.set_control_grid(slot, W.control_grid(0, 65, eps))
    nodes = W.workload_nodes("c1")
    levels = [dict(nodes=nodes[::8], n_paths=700, dt=1e-3, grid_id=0, stream_tag=1),
              dict(nodes=nodes[1::16], n_paths=333, dt=4e-4, grid_id=1, stream_tag=2,
                   emit_paths=True),
              dict(nodes=nodes[3::32], n_paths=1000, dt=2e-3, grid_id=-1, stream_tag=3)]
    st, _ = prob.estimate_levels(levels)
    assert st == 0
    fine, diff = prob.estimate_coupled(nodes[::16], 500, 2e-3, grid_id=0, emit_paths=True)
    assert fine["status"] == 0
    # more than 512 nodes: records in global memory instead of the block cache
    big = prob.estimate(W.workload_nodes("c4")[:1000], 50, 1e-3, grid_id=1)
    assert big["status"] == 0
    prob.close()
    p3 = pdd.Problem(bounds_env["ctx"], pdd.PDD_PROBLEM_CUBE_3D)
    p3.set_control_grid(0, W.control_grid(2, 33, 1e-2))
    r = p3.estimate(W.workload_nodes("c2")[::97], 200, 1e-3, grid_id=0, emit_paths=True)
    assert r["status"] == 0
    f3, _ = p3.estimate_coupled(W.workload_nodes("c2")[::301], 100, 2e-3, grid_id=0)
    assert f3["status"] == 0
    p3.close()
