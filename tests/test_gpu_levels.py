"""Several levels in one persistent launch, CUDA-graph replay, launch shapes
and the autotuner -- all through the C ABI.

The per-node sums are exact integers keyed by (node, path), and every path's
random stream is fixed by its key, so the results of a multi-level launch, of
a replayed graph and of any launch shape must equal, bit for bit, those of one
pdd_estimate_nodes call per level (which the parity tests compare with the
oracle).
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


def _same(pdd, a, b, emit=False):
    for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
        x, y = a[f].cpu().numpy(), b[f].cpu().numpy()
        assert np.array_equal(x, y, equal_nan=True), f
    if emit:
        for f in ("phi", "xi", "steps"):
            assert np.array_equal(a[f].cpu().numpy(), b[f].cpu().numpy()), f


def _levels_2d():
    nodes = W.workload_nodes("c1")
    return [
        dict(nodes=nodes[::8], n_paths=700, dt=1e-3, grid_id=0, stream_tag=1, kappa=1.3),
        dict(nodes=nodes[1::16], n_paths=333, dt=4e-4, grid_id=1, stream_tag=2, emit_paths=True),
        dict(nodes=nodes[3::32], n_paths=1000, dt=2e-3, grid_id=-1, stream_tag=3),
        dict(nodes=nodes[:0], n_paths=10, dt=1e-3, grid_id=0, stream_tag=4),  # empty level
        dict(nodes=nodes[5::64], n_paths=64, dt=1e-2, grid_id=2, stream_tag=5, seed=99 + (7 << 32)),
    ]


def test_levels_equal_separate_calls_2d(env):
    torch, pdd, ctx = env
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    for slot, eps in enumerate((1e-1, 1e-2, 1e-3)):
        prob.set_control_grid(slot, W.control_grid(0, 129, eps))
    levels = _levels_2d()
    st, multi = prob.estimate_levels(levels)
    assert st == 0
    for lv, got in zip(levels, multi):
        kw = {k: v for k, v in lv.items() if k != "nodes"}
        ref = prob.estimate(lv["nodes"], **kw)
        _same(pdd, got, ref, emit=lv.get("emit_paths", False))
    # host buffers through the same call
    st, hostres = prob.estimate_levels(levels, device_out=False, host_inputs=True)
    for a, b in zip(multi, hostres):
        _same(pdd, a, b)
    prob.close()


def test_levels_equal_separate_calls_3d_cascade(env):
    torch, pdd, ctx = env
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CUBE_3D)
    for slot, eps in enumerate((1e-1, 1e-2, 1e-3)):
        prob.set_control_grid(slot, W.control_grid(2, 33, eps))
    nodes = W.workload_nodes("c2")
    levels = [dict(nodes=nodes[::97], n_paths=500, dt=1e-2, grid_id=0, stream_tag=1),
              dict(nodes=nodes[1::193], n_paths=300, dt=1e-3, grid_id=1, stream_tag=2),
              dict(nodes=nodes[2::769], n_paths=100, dt=2e-4, grid_id=2, stream_tag=3)]
    st, multi = prob.estimate_levels(levels)
    assert st == 0
    for lv, got in zip(levels, multi):
        kw = {k: v for k, v in lv.items() if k != "nodes"}
        _same(pdd, got, prob.estimate(lv["nodes"], **kw))
    prob.close()


def test_graph_replay_and_recapture(env):
    torch, pdd, ctx = env
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, 65, 1e-2))
    nodes = W.workload_nodes("c1")[::4]
    lv = [dict(nodes=nodes, n_paths=400, dt=1e-3, grid_id=0, stream_tag=1),
          dict(nodes=nodes[::2], n_paths=200, dt=2e-3, grid_id=-1, stream_tag=2)]
    prepared = [prob._prepare(l["nodes"], l["n_paths"], l["dt"], l["grid_id"], 1234,
                              l["stream_tag"], 1.0, False, True, False, False) for l in lv]
    args = [p[0] for p in prepared]
    outs = [p[1] for p in prepared]
    g0 = ctx.graph_count()
    results = []
    for _ in range(3):
        assert pdd.pdd_estimate_levels(prob.handle, args, outs, pdd.PDD_FLAG_GRAPH) == 0
        results.append([{f: p[2][f].clone() for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS}
                        for p in prepared])
    assert ctx.graph_count() == g0 + 1  # captured once, replayed twice
    for r in results[1:]:
        for a, b in zip(results[0], r):
            _same(pdd, a, b)
    ref = prob.estimate_levels(lv)[1]
    for a, b in zip(results[0], ref):
        _same(pdd, a, b)
    args[0].dt = 5e-4  # different arguments: a new capture
    assert pdd.pdd_estimate_levels(prob.handle, args, outs, pdd.PDD_FLAG_GRAPH) == 0
    assert ctx.graph_count() == g0 + 2
    with pytest.raises(pdd.PddError):  # graphs need device buffers
        hargs, houts, _ = prob._prepare(nodes, 10, 1e-3, 0, 1, 1, 1.0, False, False, True, False)
        pdd.pdd_estimate_levels(prob.handle, [hargs], [houts], pdd.PDD_FLAG_GRAPH)
    prob.close()


def test_launch_shape_and_autotuner_do_not_change_results(env):
    torch, pdd, ctx = env
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, 129, 1e-2))
    nodes = W.workload_nodes("c1")[::8]
    ref = prob.estimate(nodes, 900, 1e-3, grid_id=0)
    for threads, max_blocks in ((128, 0), (512, 0), (256, 4), (64, 1), (0, 0)):
        ctx.set_launch(threads, max_blocks)
        _same(pdd, ref, prob.estimate(nodes, 900, 1e-3, grid_id=0))
    # steps per iteration (scheduling quantum): short, long and automatic, on a
    # 2D and a 3D problem
    for mode in (pdd.PDD_ITER_SHORT, pdd.PDD_ITER_LONG, pdd.PDD_ITER_AUTO):
        ctx.set_iteration(mode)
        _same(pdd, ref, prob.estimate(nodes, 900, 1e-3, grid_id=0))
    # paths per lane claimed from the cursor at once
    for claim in (1, 2, 16, 64, 0):
        ctx.set_claim(claim)
        assert ctx.get_claim() == claim
        _same(pdd, ref, prob.estimate(nodes, 900, 1e-3, grid_id=0))
        _same(pdd, ref, prob.estimate(nodes, 900, 1e-3, grid_id=0))
    p3 = pdd.Problem(ctx, pdd.PDD_PROBLEM_CUBE_3D)
    p3.set_control_grid(0, W.control_grid(2, 33, 1e-2))
    n3 = W.workload_nodes("c2")[::97]
    ref3 = p3.estimate(n3, 300, 1e-3, grid_id=0)
    for mode in (pdd.PDD_ITER_SHORT, pdd.PDD_ITER_LONG):
        ctx.set_iteration(mode)
        _same(pdd, ref3, p3.estimate(n3, 300, 1e-3, grid_id=0))
    ctx.set_claim(8)
    _same(pdd, ref3, p3.estimate(n3, 300, 1e-3, grid_id=0))
    ctx.set_claim(0)
    ctx.set_iteration(pdd.PDD_ITER_AUTO)
    p3.close()
    t, b, ms = prob.autotune(nodes, 900, 1e-3, grid_id=0)
    assert t in (128, 256, 512) and b >= 0 and ms > 0
    assert ctx.get_launch()[:2] == (t, b)
    assert ctx.get_launch()[2] in (pdd.PDD_ITER_AUTO, pdd.PDD_ITER_SHORT, pdd.PDD_ITER_LONG)
    _same(pdd, ref, prob.estimate(nodes, 900, 1e-3, grid_id=0))
    with pytest.raises(pdd.PddError):
        ctx.set_launch(100, 0)
    with pytest.raises(pdd.PddError):
        ctx.set_iteration(7)
    for bad in (-1, 3, 128):
        with pytest.raises(pdd.PddError):
            ctx.set_claim(bad)
    assert ctx.get_claim() in (0, 1, 4, 16)
    ctx.set_launch(0, 0)
    ctx.set_iteration(pdd.PDD_ITER_AUTO)
    ctx.set_claim(0)
    prob.close()


def test_levels_reject_mixed_exact_and_grid(env):
    torch, pdd, ctx = env
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, 33, 1e-2))
    nodes = W.workload_nodes("c0")
    with pytest.raises(pdd.PddError) as e:
        prob.estimate_levels([dict(nodes=nodes, n_paths=10, dt=1e-3, grid_id=0),
                              dict(nodes=nodes, n_paths=10, dt=1e-3, grid_id=pdd.PDD_CV_EXACT)])
    assert e.value.status == pdd.PDD_ERR_INVALID
    prob.close()


def test_record_cache_boundary(env):
    """Launches whose nodes fit the per-block shared-memory record cache (at
    most 512 node records) and launches that add into the global records
    directly give the same bits: the first 512 of 513 nodes (cache off)
    against the same 512 nodes alone (cache on), and two levels of 256 nodes
    (cache on) against 300 + 256 nodes (cache off).  Short paths (dt 1e-2)
    make many exits per step, so the exit rings drain often."""
    torch, pdd, ctx = env
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, 65, 1e-2))
    rng = np.random.default_rng(17)
    nodes = W.random_interface_nodes(rng, 513)
    for dt, n_paths in ((1e-2, 3000), (1e-3, 400)):
        big = prob.estimate(nodes, n_paths, dt, grid_id=0, stream_tag=3, emit_paths=True)
        small = prob.estimate(nodes[:512], n_paths, dt, grid_id=0, stream_tag=3, emit_paths=True)
        for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
            assert np.array_equal(big[f].cpu().numpy()[:512], small[f].cpu().numpy(),
                                  equal_nan=True), (dt, f)
        for f in ("phi", "xi", "steps"):
            assert np.array_equal(big[f].cpu().numpy()[:512], small[f].cpu().numpy()), (dt, f)
    lv_cached = [dict(nodes=nodes[:256], n_paths=2000, dt=1e-2, grid_id=0, stream_tag=5),
                 dict(nodes=nodes[256:512], n_paths=1500, dt=2e-3, grid_id=-1, stream_tag=6)]
    lv_global = [dict(nodes=nodes[:300], n_paths=2000, dt=1e-2, grid_id=0, stream_tag=5),
                 dict(nodes=nodes[256:512], n_paths=1500, dt=2e-3, grid_id=-1, stream_tag=6)]
    a = prob.estimate_levels(lv_cached)[1]
    b = prob.estimate_levels(lv_global)[1]
    for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
        assert np.array_equal(a[0][f].cpu().numpy(), b[0][f].cpu().numpy()[:256],
                              equal_nan=True), f
        assert np.array_equal(a[1][f].cpu().numpy(), b[1][f].cpu().numpy(), equal_nan=True), f
    prob.close()
