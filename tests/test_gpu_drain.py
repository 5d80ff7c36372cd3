"""Drain iterations compute what the ordinary iterations compute.

Once a launch's path cursor is exhausted, the idle lanes of a warp draw the
Philox blocks and normals of the lanes still running, which read them with
warp shuffles.  A path's stream is fixed by its (seed, stream_tag, node, path)
key, so a path must give the same phi, xi and exit index, bit for bit,
whether it ran in the ordinary iterations or in the drain.  A launch with a
few paths per node runs its paths almost entirely in the drain (a warp enters
it at its first lane refill after the cursor ran out); the same first paths
of a launch with thousands of paths per node are issued first and run in the
ordinary iterations.  Both are compared here: 2D and 3D, plain and with the
control variate, FP32 and FP64 paths, single-segment and segment-table
launches, and several counts of running lanes per warp (1 to 32 paths).
"""
import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    ctx = pdd.Context(0)
    yield torch, pdd, ctx
    ctx.close()


def _same_paths(small, big, k):
    for f in ("phi", "xi", "steps"):
        a = small[f].cpu().numpy()[:, :k]
        b = big[f].cpu().numpy()[:, :k]
        assert np.array_equal(a, b), (f, int(np.sum(a != b)))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("grid", [False, True])
def test_drain_equals_ordinary_2d(env, precision, grid):
    torch, pdd, ctx = env
    prec = pdd.PDD_PATH_FP64 if precision == "fp64" else pdd.PDD_PATH_FP32
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D, precision=prec)
    gid = pdd.PDD_CV_NONE
    if grid:
        prob.set_control_grid(0, W.control_grid(0, 129, 1e-2))
        gid = 0
    nodes = W.workload_nodes("c1")[::4]  # 64 nodes
    big = prob.estimate(nodes, 1500 if precision == "fp32" else 300, 1e-3, grid_id=gid,
                        stream_tag=11, emit_paths=True)
    assert big["status"] == 0
    for n_small in (1, 2, 5, 17):  # 64 .. 1088 paths: 2 .. 34 warps, all lane counts
        small = prob.estimate(nodes, n_small, 1e-3, grid_id=gid, stream_tag=11,
                              emit_paths=True)
        assert small["status"] == 0
        _same_paths(small, big, n_small)
    prob.close()


@pytest.mark.parametrize("grid", [False, True])
def test_drain_equals_ordinary_3d(env, grid):
    torch, pdd, ctx = env
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CUBE_3D)
    gid = pdd.PDD_CV_NONE
    if grid:
        prob.set_control_grid(0, W.control_grid(2, 33, 1e-2))
        gid = 0
    nodes = W.workload_nodes("c2")[::72]  # 128 nodes
    big = prob.estimate(nodes, 1000, 1e-3, grid_id=gid, stream_tag=12, emit_paths=True)
    assert big["status"] == 0
    for n_small in (1, 3, 8):
        small = prob.estimate(nodes, n_small, 1e-3, grid_id=gid, stream_tag=12,
                              emit_paths=True)
        assert small["status"] == 0
        _same_paths(small, big, n_small)
    prob.close()


def test_drain_equals_ordinary_segment_table(env):
    torch, pdd, ctx = env
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, 129, 1e-1))
    prob.set_control_grid(1, W.control_grid(0, 129, 1e-2))
    nodes = W.workload_nodes("c1")

    def levels(n0, n1):
        return [dict(nodes=nodes[::8], n_paths=n0, dt=2e-3, grid_id=0, stream_tag=21,
                     emit_paths=True),
                dict(nodes=nodes[3::8], n_paths=n1, dt=5e-4, grid_id=1, stream_tag=22,
                     emit_paths=True)]

    st, big = prob.estimate_levels(levels(2000, 800))
    assert st == 0
    st, small = prob.estimate_levels(levels(3, 2))
    assert st == 0
    _same_paths(small[0], big[0], 3)
    _same_paths(small[1], big[1], 2)
    prob.close()


def test_drain_truncation(env):
    """A path cut at max_steps inside a drain iteration ends with the same
    record as in an ordinary one (exit index = max_steps, truncated count)."""
    torch, pdd, ctx = env
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D, max_steps=150)
    nodes = W.workload_nodes("c1")[::8]
    big = prob.estimate(nodes, 2000, 1e-4, stream_tag=13, emit_paths=True)
    small = prob.estimate(nodes, 2, 1e-4, stream_tag=13, emit_paths=True)
    assert big["status"] == pdd.PDD_WARN_TRUNCATED and small["status"] == pdd.PDD_WARN_TRUNCATED
    assert int(small["n_truncated"].sum()) > 0
    assert int(small["steps"].max()) == 150
    _same_paths(small, big, 2)
    prob.close()
