"""Shared comparison rules for GPU-vs-oracle parity tests.

Per path: the GPU's exit index k must equal the oracle's (an FP32 rounding
can move a path across the shrunken boundary one step early or late -- an
"exit-step flip"; flips are counted), and phi and xi must agree within
PATH_ATOL; at least PATH_FRAC of all paths must pass both.
Per node: means within 1e-5 relative, or within 3 combined standard errors.
"""
import numpy as np

PATH_ATOL = 1e-4
PATH_FRAC = 0.999
NODE_RTOL = 1e-5


def compare_paths(gpu, ref, atol=PATH_ATOL):
    phi = gpu["phi"].cpu().numpy().astype(np.float64)
    xi = gpu["xi"].cpu().numpy().astype(np.float64)
    steps = gpu["steps"].cpu().numpy().astype(np.int64)
    same = steps == ref["steps"]
    close = (np.abs(phi - ref["phi"]) <= atol) & (np.abs(xi - ref["xi"]) <= atol)
    ok = same & close
    err_phi = np.abs(phi - ref["phi"])[same]
    err_xi = np.abs(xi - ref["xi"])[same]
    return {
        "n": ok.size,
        "frac_ok": float(ok.mean()),
        "flips": int((~same).sum()),
        "max_err_phi": float(err_phi.max()) if err_phi.size else 0.0,
        "max_err_xi": float(err_xi.max()) if err_xi.size else 0.0,
    }


def node_tolerance(ref_mean, se_gpu, se_ref):
    return np.maximum(NODE_RTOL * np.abs(ref_mean), 3.0 * np.sqrt(se_gpu**2 + se_ref**2))


def compare_nodes(gpu, ref):
    out = {}
    for m, se in (("mean_phi", "se_phi"), ("mean_cv", "se_cv")):
        g = gpu[m].cpu().numpy()
        sg = gpu[se].cpu().numpy()
        tol = node_tolerance(ref[m], sg, ref[se])
        err = np.abs(g - ref[m])
        with np.errstate(divide="ignore", invalid="ignore"):
            # nodes whose paths all finish at k = 0 have zero error and zero tolerance
            rel = np.where(err > 0, err / np.abs(ref[m]), 0.0)
            over = np.where(err > 0, err / tol, 0.0)
        out[m] = {"ok": bool(np.all(err <= tol)), "max_rel": float(np.max(rel)),
                  "max_err_over_tol": float(np.max(over))}
    return out


def stats_from_paths(phi, xi, steps):
    """Numpy two-pass statistics of the GPU's own emitted per-path arrays."""
    phi = phi.astype(np.float64)
    xi = xi.astype(np.float64)
    psi = phi + xi
    return {
        "mean_phi": phi.mean(1), "var_phi": phi.var(1, ddof=1),
        "mean_cv": psi.mean(1), "var_cv": psi.var(1, ddof=1),
        "mean_steps": steps.astype(np.float64).mean(1),
    }
