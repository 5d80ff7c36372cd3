"""Serving (continuous batching) through the C ABI.

Requests of different sizes, path counts, time steps and control grids are
submitted together; each result must equal, bit for bit, the same request run
alone with pdd_estimate_nodes (exact sums keyed by node and path).  Admission
control, cancellation and host-side fault injection must leave the other
requests' results unchanged.
"""
import time

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
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, 129, 1e-1))
    prob.set_control_grid(1, W.control_grid(0, 129, 1e-2))
    yield torch, pdd, ctx, prob
    prob.close()
    ctx.close()


def _requests(seed=3, count=12):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(1, 200))
        out.append(dict(nodes=W.random_interface_nodes(rng, n), n_paths=int(rng.integers(50, 3000)),
                        dt=float(rng.choice([1e-2, 1e-3, 2e-4])),
                        grid_id=int(rng.choice([-1, 0, 1])), stream_tag=100 + i,
                        seed=1234 + (i % 3)))
    return out


def _alone(prob, r):
    res = prob.estimate(r["nodes"], r["n_paths"], r["dt"], grid_id=r["grid_id"], seed=r["seed"],
                        stream_tag=r["stream_tag"])
    return {k: v.cpu().numpy() for k, v in res.items() if hasattr(v, "cpu")}


def _same(pdd, a, b):
    for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
        assert np.array_equal(a[f], b[f], equal_nan=True), f


def _wait(srv, t, n, timeout_s=120):
    st, res = srv.poll(t, n, int(timeout_s * 1e6))
    return st, res


def test_mix_equals_alone(env):
    torch, pdd, ctx, prob = env
    reqs = _requests()
    srv = pdd.Server(ctx, max_active=8, quantum_path_steps=20_000_000)
    tickets = [srv.submit(prob, r["nodes"], r["n_paths"], r["dt"], grid_id=r["grid_id"],
                          seed=r["seed"], stream_tag=r["stream_tag"]) for r in reqs]
    for r, t in zip(reqs, tickets):
        st, res = _wait(srv, t, len(r["nodes"]))
        assert st == pdd.PDD_OK, pdd.pdd_last_error()
        _same(pdd, res, _alone(prob, r))
    s = srv.stats()
    assert s["completed"] == len(reqs) and s["admitted"] == len(reqs)
    assert s["launches"] > len(reqs) // 8  # requests were spread over several launches
    # the launches' executed path-steps are exactly the requests' exit indices
    steps = sum(int(np.rint(_alone(prob, r)["mean_steps"] * r["n_paths"]).sum()) for r in reqs)
    assert s["path_steps"] == steps
    srv.close()


def test_arrivals_while_running(env):
    torch, pdd, ctx, prob = env
    srv = pdd.Server(ctx, max_active=4, quantum_path_steps=5_000_000)
    big = dict(nodes=W.workload_nodes("c1")[::4], n_paths=4000, dt=2e-4, grid_id=1,
               stream_tag=7, seed=5)
    tb = srv.submit(prob, big["nodes"], big["n_paths"], big["dt"], grid_id=1, seed=5,
                    stream_tag=7)
    st, _ = srv.poll(tb, len(big["nodes"]), 0)
    assert st == pdd.PDD_ERR_NOT_READY
    small = _requests(seed=9, count=6)
    ts = []
    for r in small:  # arrive while the big request runs
        time.sleep(0.005)
        ts.append(srv.submit(prob, r["nodes"], r["n_paths"], r["dt"], grid_id=r["grid_id"],
                             seed=r["seed"], stream_tag=r["stream_tag"]))
    for r, t in zip(small, ts):
        st, res = _wait(srv, t, len(r["nodes"]))
        assert st == pdd.PDD_OK
        _same(pdd, res, _alone(prob, r))
    st, res = _wait(srv, tb, len(big["nodes"]))
    assert st == pdd.PDD_OK
    _same(pdd, res, _alone(prob, big))
    srv.close()


def test_admission_cancel_and_faults(env):
    torch, pdd, ctx, prob = env
    reqs = _requests(seed=21, count=6)
    # a tiny arena: requests queue for memory; a request larger than it is refused
    srv = pdd.Server(ctx, max_active=2, max_queue=3, quantum_path_steps=10_000_000,
                     device_arena_bytes=200 * 256 * 2)
    with pytest.raises(pdd.PddError) as e:
        srv.submit(prob, W.workload_nodes("c4")[:4000], 10, 1e-3)
    assert e.value.status == pdd.PDD_ERR_NOMEM
    with pytest.raises(pdd.PddError) as e:
        srv.submit(prob, reqs[0]["nodes"], 10, 1e-3, flags=pdd.PDD_FLAG_EMIT_PATHS)
    assert e.value.status == pdd.PDD_ERR_INVALID
    with pytest.raises(pdd.PddError):
        srv.submit(prob, reqs[0]["nodes"], 10, 1e-3, grid_id=6)
    srv.close()

    srv = pdd.Server(ctx, max_active=2, max_queue=4, quantum_path_steps=10_000_000)
    long_req = dict(nodes=W.workload_nodes("c1"), n_paths=200_000, dt=1e-4, grid_id=1,
                    stream_tag=1, seed=1)
    t_long = srv.submit(prob, long_req["nodes"], long_req["n_paths"], 1e-4, grid_id=1)
    deadline = time.time() + 30
    while srv.stats()["admitted"] < 1 and time.time() < deadline:
        time.sleep(0.001)
    srv.inject_fault(1)  # the next admission fails
    t_fail = srv.submit(prob, reqs[0]["nodes"], reqs[0]["n_paths"], reqs[0]["dt"])
    tickets = []
    busy = 0
    for r in reqs[1:]:
        try:
            tickets.append((r, srv.submit(prob, r["nodes"], r["n_paths"], r["dt"],
                                          grid_id=r["grid_id"], seed=r["seed"],
                                          stream_tag=r["stream_tag"])))
        except pdd.PddError as ex:
            assert ex.status == pdd.PDD_ERR_BUSY
            busy += 1
    srv.cancel(t_long)
    st, _ = _wait(srv, t_long, len(long_req["nodes"]))
    assert st == pdd.PDD_ERR_CANCELLED
    st, _ = _wait(srv, t_fail, len(reqs[0]["nodes"]))
    assert st == pdd.PDD_ERR_NOMEM
    for r, t in tickets:
        st, res = _wait(srv, t, len(r["nodes"]))
        assert st == pdd.PDD_OK
        _same(pdd, res, _alone(prob, r))
    s = srv.stats()
    assert s["rejected_busy"] == busy and s["cancelled"] == 1 and s["failed"] == 1
    # a request dropped mid-flight (its worker lost) leaves the others intact
    srv.inject_fault(2)
    more = _requests(seed=33, count=3)
    tk = [srv.submit(prob, r["nodes"], r["n_paths"], r["dt"], grid_id=r["grid_id"],
                     seed=r["seed"], stream_tag=r["stream_tag"]) for r in more]
    statuses = []
    for r, t in zip(more, tk):
        st, res = _wait(srv, t, len(r["nodes"]))
        statuses.append(st)
        if st == pdd.PDD_OK:
            _same(pdd, res, _alone(prob, r))
    assert statuses.count(pdd.PDD_ERR_CANCELLED) == 1
    assert statuses.count(pdd.PDD_OK) == len(more) - 1
    with pytest.raises(pdd.PddError):
        srv.cancel(123456789)
    srv.close()


def test_destroy_with_work_in_flight(env):
    torch, pdd, ctx, prob = env
    srv = pdd.Server(ctx, max_active=2, quantum_path_steps=5_000_000)
    for r in _requests(seed=44, count=5):
        srv.submit(prob, r["nodes"], r["n_paths"], r["dt"], grid_id=r["grid_id"])
    srv.close()  # cancels and waits for the launches in flight; must return
    torch.cuda.synchronize()


def test_concurrent_clients(env):
    """Four client threads submit and poll at the same time (the binding
    releases the interpreter lock in every C call); every result equals the
    same request run alone."""
    import threading
    torch, pdd, ctx, prob = env
    srv = pdd.Server(ctx, max_active=8, max_queue=64, quantum_path_steps=10_000_000)
    per_client = [_requests(seed=100 + c, count=5) for c in range(4)]
    for c, reqs in enumerate(per_client):
        for i, r in enumerate(reqs):
            r["stream_tag"] = 1000 + 10 * c + i
    got, errors = {}, []

    def client(c):
        try:
            tickets = [srv.submit(prob, r["nodes"], r["n_paths"], r["dt"], grid_id=r["grid_id"],
                                  seed=r["seed"], stream_tag=r["stream_tag"])
                       for r in per_client[c]]
            for i, (r, t) in enumerate(zip(per_client[c], tickets)):
                st, res = _wait(srv, t, len(r["nodes"]))
                got[(c, i)] = (st, res)
        except Exception as ex:  # reported in the main thread
            errors.append(repr(ex))

    threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    assert not errors, errors
    assert len(got) == 20
    srv.close()
    for c, reqs in enumerate(per_client):
        for i, r in enumerate(reqs):
            st, res = got[(c, i)]
            assert st == pdd.PDD_OK
            _same(pdd, res, _alone(prob, r))


def test_shortest_first_policy(env):
    """PDD_SERVE_SHORTEST gives the launches to the requests with the least
    remaining work: small requests submitted after a large one finish while it
    is still running; every result still equals the request run alone."""
    torch, pdd, ctx, prob = env
    srv = pdd.Server(ctx, max_active=8, quantum_path_steps=500_000_000,
                     policy=pdd.PDD_SERVE_SHORTEST)
    big = dict(nodes=W.workload_nodes("c1"), n_paths=200_000, dt=1e-4, grid_id=1,
               stream_tag=70, seed=3)
    tb = srv.submit(prob, big["nodes"], big["n_paths"], big["dt"], grid_id=1, seed=3,
                    stream_tag=70)
    small = _requests(seed=51, count=6)
    ts = [srv.submit(prob, r["nodes"], r["n_paths"], r["dt"], grid_id=r["grid_id"],
                     seed=r["seed"], stream_tag=r["stream_tag"]) for r in small]
    for r, t in zip(small, ts):
        st, res = _wait(srv, t, len(r["nodes"]))
        assert st == pdd.PDD_OK
        _same(pdd, res, _alone(prob, r))
    st, _ = srv.poll(tb, len(big["nodes"]), 0)
    assert st == pdd.PDD_ERR_NOT_READY  # the large request is still running
    st, res = _wait(srv, tb, len(big["nodes"]))
    assert st == pdd.PDD_OK
    _same(pdd, res, _alone(prob, big))
    srv.close()
    with pytest.raises(pdd.PddError):
        pdd.Server(ctx, policy=7)


def test_deadline_admission_and_goodput(env):
    """Admission by predicted work: with a deadline, a request whose predicted
    path-steps cannot finish in time is refused at once (PDD_ERR_DEADLINE,
    counted apart); admitted requests complete, so the completed path-steps
    are the executed ones (goodput 1) and the results still equal the
    requests run alone."""
    torch, pdd, ctx, prob = env
    srv = pdd.Server(ctx, max_active=16, max_queue=64, deadline_s=2.0, rate_hint=1e11)
    rng = np.random.default_rng(17)
    big = W.random_interface_nodes(rng, 4096)
    # ~4096 x 1e6 x 1,200 path-steps: hours of work, far beyond 2 s
    with pytest.raises(pdd.PddError) as e:
        srv.submit(prob, big, 1_000_000, 1e-4, grid_id=1, stream_tag=7)
    assert e.value.status == pdd.PDD_ERR_DEADLINE
    small = _requests(seed=5, count=6)
    tickets = [srv.submit(prob, r["nodes"], r["n_paths"], r["dt"], grid_id=r["grid_id"],
                          seed=r["seed"], stream_tag=r["stream_tag"]) for r in small]
    for t, r in zip(tickets, small):
        st, res = _wait(srv, t, len(r["nodes"]))
        assert st == pdd.PDD_OK
        _same(pdd, res, _alone(prob, r))
    s = srv.stats()
    assert s["rejected_deadline"] == 1 and s["rejected_busy"] == 0
    assert s["completed"] == len(small)
    assert s["completed_path_steps"] > 0
    assert abs(s["completed_path_steps"] - s["path_steps"]) <= 0.01 * s["path_steps"]
    assert s["backlog_path_steps"] == 0 and s["rate_path_steps_per_s"] > 0
    srv.close()


def test_backlog_refusal(env):
    """The deadline counts the queued and running work: a request that fits
    alone is refused while a similar one, just admitted, is still running."""
    torch, pdd, ctx, prob = env
    srv = pdd.Server(ctx, max_active=4, max_queue=64, deadline_s=0.5, rate_hint=1e11)
    nodes = W.workload_nodes("c1")
    # ~256 x 1.3e5 x 1,100 = 3.7e10 path-steps: predicted 0.37 s at the assumed
    # rate (the first call also runs the exit-time pilot of this time step)
    t1 = srv.submit(prob, nodes, 130_000, 1e-4, grid_id=1, stream_tag=301)
    with pytest.raises(pdd.PddError) as e:  # submitted at once, behind the first
        srv.submit(prob, nodes, 130_000, 1e-4, grid_id=1, stream_tag=302)
    assert e.value.status == pdd.PDD_ERR_DEADLINE
    assert b"deadline" in pdd.lib().pdd_last_error()
    st, _ = _wait(srv, t1, len(nodes))
    assert st == pdd.PDD_OK
    s = srv.stats()
    assert s["rejected_deadline"] == 1 and s["completed"] == 1
    # with the first one done, the same request fits again
    t3 = srv.submit(prob, nodes, 130_000, 1e-4, grid_id=1, stream_tag=303)
    st, _ = _wait(srv, t3, len(nodes))
    assert st == pdd.PDD_OK
    srv.close()


def test_earliest_deadline_bounds_latency(env):
    """Earliest-deadline policy with a deadline: under a burst far above
    capacity the admitted requests are served in submission order and each
    completes within the deadline (with slack for the predicted rate), the
    rest is refused at once, and no executed work is thrown away."""
    torch, pdd, ctx, prob = env
    deadline = 1.0
    srv = pdd.Server(ctx, max_active=32, max_queue=64, deadline_s=deadline,
                     policy=pdd.PDD_SERVE_EARLIEST_DEADLINE)
    nodes = W.workload_nodes("c1")
    # prime the (problem, dt) estimate and the measured rate with one request
    t = srv.submit(prob, nodes, 20_000, 1e-4, grid_id=1, stream_tag=500)
    assert _wait(srv, t, len(nodes))[0] == pdd.PDD_OK
    admitted, refused = {}, 0
    for i in range(40):  # each ~5.6e9 path-steps: ~25-40 ms of GPU work
        try:
            tk = srv.submit(prob, nodes, 20_000, 1e-4, grid_id=1, stream_tag=501 + i)
            admitted[tk] = time.perf_counter()
        except pdd.PddError as e:
            assert e.status == pdd.PDD_ERR_DEADLINE
            refused += 1
    assert admitted and refused
    lat = []
    for tk, t0 in admitted.items():
        st, _ = _wait(srv, tk, len(nodes))
        assert st == pdd.PDD_OK
        lat.append(time.perf_counter() - t0)
    assert max(lat) <= 2.0 * deadline, max(lat)
    s = srv.stats()
    assert s["rejected_deadline"] == refused
    assert abs(s["completed_path_steps"] - s["path_steps"]) <= 0.01 * s["path_steps"]
    srv.close()
