"""Synthetic input layouts: node counts and placement of every workload."""
import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W


@pytest.mark.parametrize("name,count", [("c0", 24), ("c1", 256), ("c2", 9216), ("c4", 31744),
                                        ("paper", 18)])
def test_node_counts(name, count):
    nodes = W.workload_nodes(name)
    assert nodes.shape[0] == count and nodes.dtype == np.float32
    assert np.all((nodes > 0) & (nodes < 1))
    assert np.unique(nodes, axis=0).shape[0] == count


def test_nodes_lie_on_interfaces():
    for name in ("c0", "c1", "c4"):
        w = W.WORKLOADS[name]
        S = w["subdomains"]
        nodes = W.workload_nodes(name).astype(np.float64)
        on_line = np.isclose(nodes * S, np.round(nodes * S), atol=1e-5)
        assert np.all(on_line.any(axis=1))
    nodes = W.workload_nodes("c2").astype(np.float64)
    on_plane = np.isclose(nodes * 4, np.round(nodes * 4), atol=1e-5)
    assert np.all(on_plane.any(axis=1))


def test_c0_node_order():
    nodes = W.workload_nodes("c0")
    # first the x = 1/2 line (segment y in (0, 1/2), then (1/2, 1)), then y = 1/2
    assert np.allclose(nodes[0], [0.5, 0.5 / 7])
    assert np.allclose(nodes[6], [0.5, 0.5 + 0.5 / 7])
    assert np.allclose(nodes[12], [0.5 / 7, 0.5])


def test_control_grid_vanishing_bump():
    for kind, n in ((0, 17), (2, 9)):
        g = W.control_grid(kind, n, 0.1)
        lin = np.linspace(0, 1, n)
        if kind == 2:
            Z, Y, X = np.meshgrid(lin, lin, lin, indexing="ij")
            u = W.exact_u(2, np.stack([X, Y, Z], -1))
            assert np.allclose(g[0], u[0]) and np.allclose(g[:, :, -1], u[:, :, -1])
        else:
            Y, X = np.meshgrid(lin, lin, indexing="ij")
            u = W.exact_u(0, np.stack([X, Y], -1))
            assert np.allclose(g[0], u[0]) and np.allclose(g[:, 0], u[:, 0])
        assert not np.allclose(g, u)


def test_serving_requests_seeded():
    a = W.serving_requests(5, 200.0, 0.5)
    b = W.serving_requests(5, 200.0, 0.5)
    assert len(a) == len(b) > 20
    assert all(x["n_nodes"] == y["n_nodes"] and x["arrival"] == y["arrival"] for x, y in zip(a, b))
    assert all(1 <= r["n_nodes"] <= 4096 and r["nodes"].shape == (r["n_nodes"], 2) for r in a)
