"""Running the levels that Algorithm 4 schedules (the nodal loop of
Algorithm 5) through the library.

Algorithm 4 turns the fitted nodal constants (Algorithm 3) into a tolerance
sequence a_0 < a_1 < ... < a_J.  Algorithm 5 then runs PlainPDD at a_J and,
for j = J-1 .. 0, the level at tolerance a_j with the control variate of the
previous, coarser level; for every node and level the time step and path
count are the balanced ones of eq. F:N_y_h (bias a_j/2, statistical error
a_j/2).  This module only plans and marshals: the per-node (h, N) come from
pdd_balanced_plan, the model's predictions from pdd_schedule_predict, and
every path runs in the library's kernels (pdd_estimate_levels).

The previous iterates are synthetic here (the subdomain solves that would
build them are not part of this library): level j < J reads the control grid
the caller loaded into slot j, standing in for the iterate of tolerance
a_{j+1}.

Levels share one launch.  A launch holds at most 128 segments, and a segment
has one time step and one path count, so each level's nodes are cut into
contiguous groups, sorted by their planned time step for the pilot and, once
every node's N is known, by whichever of h or the per-node cost N E[tau] / h
predicts the cheaper launch; a group runs at the smallest h and the largest N
of its nodes (both stay within the tolerance), on a random stream of its own.  The path count of a controlled level needs
V[phi + xi] at that level's h, which only a run can give: a pilot launch of
`n_pilot` paths per node measures every level's variances first (its cost is
reported apart).
"""
from __future__ import annotations

import time

import numpy as np

from . import pdd


FIT_KEYS = ("K", "beta", "alpha", "V_phi", "V_psi", "rho_phi_psi", "E_tau")


def fitted_subset(fit, nodes):
    """The nodes Algorithm 3 could fit (finite constants, V[phi] > 0, beta !=
    0) and their constants; returns (mask, fit_subset, nodes_subset)."""
    ok = np.ones(len(fit["beta"]), dtype=bool)
    for k in FIT_KEYS:
        ok &= np.isfinite(np.asarray(fit[k]))
    ok &= (np.asarray(fit["V_phi"]) > 0) & (np.asarray(fit["beta"]) != 0)
    return ok, {k: np.asarray(fit[k])[ok] for k in FIT_KEYS}, np.asarray(nodes)[ok]


def group_nodes(key, groups):
    """Contiguous groups of node indices sorted by `key` (at most `groups`)."""
    order = np.argsort(np.asarray(key), kind="stable")
    return [g for g in np.array_split(order, max(1, min(groups, order.size))) if g.size]


def grouped_cost(groups, h, n_paths, e_tau):
    """Predicted path-steps of a level run as `groups` (each group at the
    smallest h and the largest N of its nodes): sum over nodes of
    N_group E[tau_i] / h_group."""
    return float(sum(np.max(n_paths[g]) * np.sum(e_tau[g]) / np.min(h[g]) for g in groups))


def partition(order, h, n_paths, e_tau, groups):
    """Cut the nodes, taken in `order`, into at most `groups` contiguous
    groups of least grouped_cost (dynamic programming over the cut points:
    best[k][j] = min over i of best[k-1][i] + cost of nodes i..j-1)."""
    hh, nn, ee = h[order], n_paths[order], e_tau[order]
    n = order.size
    groups = max(1, min(groups, n))
    ce = np.concatenate([[0.0], np.cumsum(ee)])
    # cost[i, j] of the group order[i:j] (j > i): max N, min h over the range
    cost = np.full((n + 1, n + 1), np.inf)
    for i in range(n):
        mx = np.maximum.accumulate(nn[i:])
        mn = np.minimum.accumulate(hh[i:])
        cost[i, i + 1:] = mx * (ce[i + 1:] - ce[i]) / mn
    best = np.full(n + 1, np.inf)
    best[0] = 0.0
    cut = np.zeros((groups + 1, n + 1), dtype=np.int64)
    for k in range(1, groups + 1):
        tot = best[:, None] + cost  # [i, j]: best with k-1 groups up to i, then i..j-1
        arg = np.argmin(tot, axis=0)
        new_best = tot[arg, np.arange(n + 1)]
        cut[k] = arg
        best = np.minimum(best, new_best) if k > 1 else new_best
        cut[k] = np.where(new_best <= best, arg, -1)
    # walk back: at each k the cut that reached j (fewer groups when they tie)
    out, j, k = [], n, groups
    while j > 0:
        while k > 0 and cut[k, j] < 0:
            k -= 1
        i = int(cut[k, j])
        out.append(order[i:j])
        j, k = i, k - 1
    return out[::-1]


def regroup(h, n_paths, e_tau, groups, dp_max_nodes=2048):
    """The cheapest grouping of one level's nodes by predicted cost
    (grouped_cost): contiguous groups of the nodes in order of h (the time
    step) or of N (the path count), cut by dynamic programming (O(n^2) memory
    and O(n^2 groups) time: equal-size groups above dp_max_nodes nodes)."""
    if h.size > dp_max_nodes:
        cands = [group_nodes(h, groups), group_nodes(n_paths, groups)]
    else:
        cands = [partition(np.argsort(h, kind="stable"), h, n_paths, e_tau, groups),
                 partition(np.argsort(n_paths, kind="stable"), h, n_paths, e_tau, groups)]
    costs = [grouped_cost(g, h, n_paths, e_tau) for g in cands]
    return cands[int(np.argmin(costs))], min(costs)


def plan_levels(fit, a, q=2.0, delta=1.0, h_min=1e-5, h_max=1e-2, max_segments=128):
    """Per level j = 0..J of the tolerance sequence `a` (a[0] the target): the
    planned time step of every node (eq. F:N_y_h with the fitted beta), the
    node groups of the level's segments, the model's predicted rho^2 and
    path-step cost per node (pdd_schedule_predict: level J plain, level j < J
    with the control variate of tolerance a[j+1])."""
    J = len(a) - 1
    per_level = max(1, max_segments // (J + 1))
    levels = []
    for j in range(J + 1):
        h, _ = pdd.pdd_balanced_plan(a[j], fit["beta"], fit["V_phi"], q=q, delta=delta,
                                     h_min=h_min, h_max=h_max)
        coarse = a[j + 1] if j < J else -1.0
        rho2, cost = pdd.pdd_schedule_predict(fit["K"], fit["beta"], fit["alpha"],
                                              fit["V_phi"], fit["V_psi"], fit["rho_phi_psi"],
                                              delta, coarse, a[j])
        levels.append({"j": j, "a": float(a[j]), "controlled": j < J, "h": h,
                       "groups": group_nodes(h, per_level), "pred_rho2": rho2,
                       "pred_path_steps": cost})
    return levels


def _segments(prob, cols_of, levels, n_paths_of, seed, tag_base, emit=False):
    """pdd_estimate_levels arguments for every group of every level."""
    segs = []
    for lv in levels:
        gid = lv["j"] if lv["controlled"] else pdd.PDD_CV_NONE
        for gi, idx in enumerate(lv["groups"]):
            n_paths = int(n_paths_of(lv, idx))
            tag = tag_base + 256 * lv["j"] + gi
            args, out, res = prob._prepare(cols_of(idx), n_paths, float(lv["h"][idx].min()), gid,
                                           seed, tag, 1.0, emit, True, False, False)
            segs.append((lv, idx, n_paths, tag, args, out, res))
    return segs


def run_levels(prob, nodes, levels, q=2.0, n_pilot=2000, seed=1234, tag_base=4096,
               n_max=(1 << 32) - 1, emit=False, e_tau=None):
    """Pilot, then all levels in one launch.  Returns per-level observations
    and the wall time of the main launch.  `nodes`: (n, D) float32 array;
    `e_tau`: per-node expected exit times (Algorithm 3's), which weigh the
    regrouping of each level by predicted cost (equal weights without)."""
    import torch
    dev = torch.device("cuda", prob.ctx.device)
    nodes = np.ascontiguousarray(nodes, dtype=np.float32)
    D = nodes.shape[1]
    cache = {}

    def cols_of(idx):
        key = idx.tobytes()
        if key not in cache:
            cache[key] = [torch.from_numpy(np.ascontiguousarray(nodes[idx, d])).to(dev)
                          for d in range(D)]
        return cache[key]

    n = nodes.shape[0]
    # pilot: the variance of each level's score at its own time steps
    pilot = _segments(prob, cols_of, levels, lambda lv, idx: n_pilot, seed, tag_base + 65536)
    t0 = time.perf_counter()
    st = pdd.pdd_estimate_levels(prob.handle, [s[4] for s in pilot], [s[5] for s in pilot], 0)
    pilot_s = time.perf_counter() - t0
    pilot_steps = 0.0
    var = [np.zeros(n) for _ in levels]
    for lv, idx, n_paths, _, _, _, res in pilot:
        key = "var_cv" if lv["controlled"] else "var_phi"
        var[lv["j"]][idx] = res[key].cpu().numpy()
        pilot_steps += float(res["mean_steps"].cpu().numpy().sum()) * n_paths
    e_tau = np.asarray(e_tau if e_tau is not None else np.ones(n), dtype=np.float64)
    for lv in levels:
        _, N = pdd.pdd_balanced_plan(lv["a"], np.zeros(n), var[lv["j"]], q=q, n_max=n_max)
        lv["n_paths"] = N
        lv["pilot_var"] = var[lv["j"]]
        # with every node's N known, group the main launch by predicted cost
        per_node = float(np.sum(N * e_tau / lv["h"]))
        lv["groups"], grouped = regroup(lv["h"], N.astype(np.float64), e_tau, len(lv["groups"]))
        lv["grouping_inflation"] = grouped / per_node if per_node > 0 else 1.0
    main = _segments(prob, cols_of, levels, lambda lv, idx: lv["n_paths"][idx].max(), seed,
                     tag_base, emit=emit)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_main = pdd.pdd_estimate_levels(prob.handle, [s[4] for s in main], [s[5] for s in main], 0)
    wall = time.perf_counter() - t0
    obs = []
    for lv in levels:
        est = np.zeros(n)
        rho = np.zeros(n)
        steps = 0.0
        paths = 0
        se = np.zeros(n)
        for lvx, idx, n_paths, tag, _, _, res in main:
            if lvx is not lv:
                continue
            key = "mean_cv" if lv["controlled"] else "mean_phi"
            est[idx] = res[key].cpu().numpy()
            se[idx] = res["se_cv" if lv["controlled"] else "se_phi"].cpu().numpy()
            rho[idx] = res["rho"].cpu().numpy()
            steps += float(res["mean_steps"].cpu().numpy().sum()) * n_paths
            paths += n_paths * idx.size
        obs.append({"estimate": est, "se": se, "rho": rho, "path_steps": steps, "paths": paths})
    return {"status": int(st_main), "pilot_status": int(st), "wall_s": wall,
            "pilot_s": pilot_s, "pilot_path_steps": pilot_steps, "levels": obs,
            "segments": [(s[0]["j"], s[1], s[2], s[3], float(s[0]["h"][s[1]].min()), s[6])
                         for s in main]}


def predicted_plain_steps(fit, a0, delta=1.0):
    """Predicted path-steps of PlainPDD(a0) (eq. F:PlainPDD_cost without the
    subdomain solves)."""
    p = 2.0 + 1.0 / delta
    return float(np.sum(np.asarray(fit["K"]) * np.asarray(fit["V_phi"])) / a0**p)


def summary(levels, run, u, kappa, fit, a0, delta=1.0):
    """Table 3 analogue: per level predicted vs observed path-steps and mean
    |rho|, and the cumulative speedups."""
    rows = []
    tot_pred, tot_obs = 0.0, 0.0
    for lv, ob in zip(levels, run["levels"]):
        k = kappa if lv["controlled"] else 1.0
        pred = float(np.sum(lv["pred_path_steps"]))
        rows.append({
            "tolerance": lv["a"], "controlled": lv["controlled"],
            "h_median": float(np.median(lv["h"])), "segments": len(lv["groups"]),
            "paths": ob["paths"],
            "pred_path_steps": pred, "obs_path_steps": ob["path_steps"],
            "pred_mean_abs_rho": float(np.mean(np.sqrt(lv["pred_rho2"]))) if lv["controlled"]
            else None,
            "obs_mean_abs_rho": float(np.mean(np.abs(ob["rho"]))) if lv["controlled"] else None,
            "rmse_vs_exact": float(np.sqrt(np.mean((ob["estimate"] - u) ** 2))),
            "max_se_over_half_tolerance": float(np.max(2.0 * ob["se"] / lv["a"])),
            "grouping_inflation": float(lv.get("grouping_inflation", 1.0)),
        })
        tot_pred += k * pred
        tot_obs += k * ob["path_steps"]
    return {"rows": rows, "pred_cumulative_speedup": predicted_plain_steps(fit, a0, delta) / tot_pred,
            "pred_cost": tot_pred, "obs_cost": tot_obs}
