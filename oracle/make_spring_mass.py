"""Write the initial states of the spring-mass experiment (Section IV-A) to
paper_2107_01745_b300/data/spring_mass_x0.json.

TEST-INPUT GENERATOR: run once by hand; the library never imports it.

The paper samples 300 initial states "uniformly from the problem's domain", the set of x0 for
which the stochastic optimal control problem is feasible.  Reading: draw x0 uniformly from
the state box (|p| <= p_max, |v| <= v_max; each component alone reaches its bounds inside the
domain, so no smaller box contains it) with numpy's PCG64 from a fixed seed, decide
feasibility of the whole scenario tree (every node's state in its box, every input in its
box, dynamics exact) and keep the first 300 feasible draws in draw order.  A draw is feasible
if the saturated LQR policy keeps every node in the box (a feasible point, found quickly),
else if one linear program says so (scipy HiGHS, interior point, 20 s limit); draws the LP
does not decide within the limit are rejected and counted.  Draws the LP does not decide within the
limit are rejected and counted.  The position bound is not given in the paper: p_max = 8 m.

    python -m oracle.make_spring_mass [workers]
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np
import scipy.optimize
import scipy.sparse

from paper_2107_01745_b300 import workloads as W

SEED = 6
COUNT = 300
P_MAX = 8.0
OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2107_01745_b300", "data",
                   "spring_mass_x0.json")


def _tree_lp(x0: np.ndarray | None):
    """Constraint data of the scenario-tree feasibility LP: variables [x0 (if free)] + the
    states of nodes 1.. + the inputs of the nonleaf nodes, dynamics as equalities, boxes as
    bounds (x0 free within the state box)."""
    p = W.spring_mass(np.zeros(10) if x0 is None else x0, p_max=P_MAX)
    t = p.tree
    nn, npl, nx, nu = t.num_nodes, t.num_nonleaf, p.nx, p.nu
    f0 = nx if x0 is None else 0          # x0 columns first when free
    nxv = (nn - 1) * nx
    nv = f0 + nxv + npl * nu
    A, B = p.A[1], p.B[1]
    ai, aj = np.nonzero(A)
    bi, bj = np.nonzero(B)
    rows, cols, vals = [], [], []
    beq = np.zeros(nxv)
    for j in range(1, nn):
        i = int(t.parent[j])
        r0 = (j - 1) * nx
        rows.extend(range(r0, r0 + nx))
        cols.extend(range(f0 + r0, f0 + r0 + nx))
        vals.extend([1.0] * nx)
        if i > 0 or x0 is None:
            rows.extend(r0 + ai)
            cols.extend((f0 + (i - 1) * nx if i > 0 else 0) + aj)
            vals.extend(-A[ai, aj])
        rows.extend(r0 + bi)
        cols.extend(f0 + nxv + i * nu + bj)
        vals.extend(-B[bi, bj])
        beq[r0:r0 + nx] = p.c[j] + (A @ p.x0 if (i == 0 and x0 is not None) else 0.0)
    Aeq = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(nxv, nv))
    lb = np.concatenate([p.xlo] * (1 if x0 is None else 0) + [np.tile(p.xlo, nn - 1), np.tile(p.ulo, npl)])
    ub = np.concatenate([p.xhi] * (1 if x0 is None else 0) + [np.tile(p.xhi, nn - 1), np.tile(p.uhi, npl)])
    return Aeq, beq, np.stack([lb, ub], 1), nv


def feasibility_status(x0: np.ndarray) -> int:
    """scipy linprog status of the feasibility LP at x0: 0 feasible, 2 infeasible, else undecided."""
    Aeq, beq, bounds, nv = _tree_lp(np.asarray(x0, dtype=np.float64))
    res = scipy.optimize.linprog(np.zeros(nv), A_eq=Aeq, b_eq=beq, bounds=bounds, method="highs-ipm",
                                 options={"time_limit": 20.0})
    return int(res.status)


_POLICY = {}


def policy_feasible(x0: np.ndarray) -> bool:
    """A quick certificate: the saturated LQR policy u = clip(-K x, u_min, u_max) (K of the
    nominal system's Riccati equation with the stage weights) keeps every node of the tree
    inside the state box.  True proves feasibility; False decides nothing."""
    import scipy.linalg
    if "K" not in _POLICY:
        p = W.spring_mass(np.zeros(10), p_max=P_MAX)
        A, B = p.A[1], p.B[1]
        Q, R = np.diag(p.Q), np.diag(p.R)
        P = scipy.linalg.solve_discrete_are(A, B, Q, R)
        _POLICY["K"] = np.linalg.solve(R + B.T @ P @ B, B.T @ P @ A)
        _POLICY["p"] = p
    K, p = _POLICY["K"], _POLICY["p"]
    t = p.tree
    A, B = p.A[1], p.B[1]
    X = np.empty((t.num_nodes, p.nx))
    X[0] = x0
    for s in range(1, t.horizon + 1):
        nodes = t.stage_nodes(s)
        par = t.parent[nodes]
        U = np.clip(-X[par] @ K.T, p.ulo, p.uhi)
        X[nodes] = X[par] @ A.T + U @ B.T + p.c[nodes]
        if np.any(X[nodes] < p.xlo) or np.any(X[nodes] > p.xhi):
            return False
    return True


def classify(x0: np.ndarray) -> tuple[int, bool]:
    """(status, by_policy): status 0 feasible, 2 infeasible, else undecided."""
    if policy_feasible(x0):
        return 0, True
    return feasibility_status(x0), False


def domain_extent(job) -> float:
    """min (sign = +1) or max (sign = -1) of x0[k] over the problem's domain."""
    k, sign = job
    Aeq, beq, bounds, nv = _tree_lp(None)
    c = np.zeros(nv)
    c[k] = sign
    res = scipy.optimize.linprog(c, A_eq=Aeq, b_eq=beq, bounds=bounds, method="highs-ipm")
    assert res.status == 0, res.message
    return float(res.x[k])


def draws(n: int, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """n states uniform in the box [lo, hi] (a box that contains the domain)."""
    rng = np.random.default_rng(SEED)
    return lo + (hi - lo) * rng.random((n, lo.size))


def main(workers: int = 6):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    keep, status, by_policy = [], [], []
    M = W.SPRING_MASS["masses"]
    hi = np.concatenate([np.full(M, P_MAX), np.full(M, W.SPRING_MASS["v_max"])])
    X = draws(20000, -hi, hi)
    with ctx.Pool(workers) as pool:
        # results come back in draw order; the pool stops once COUNT draws are feasible
        for k, (s, pol) in enumerate(pool.imap(classify, list(X), chunksize=1)):
            status.append(s)
            by_policy.append(pol)
            if s == 0:
                keep.append(X[k])
                if len(keep) % 20 == 0:
                    print(f"{k + 1} drawn, {len(keep)} feasible", flush=True)
                if len(keep) == COUNT:
                    pool.terminate()
                    break
    # the draws decided up to the last kept one
    last = 0
    cnt = 0
    for idx, s in enumerate(status):
        if s == 0:
            cnt += 1
            if cnt == COUNT:
                last = idx + 1
                break
    st_used = status[:last]
    doc = {"seed": SEED, "p_max": P_MAX, "v_max": W.SPRING_MASS["v_max"], "count": len(keep), "draws": last,
           "certified_by_policy": int(sum(by_policy[:last])),
           "rejected_infeasible": sum(s == 2 for s in st_used), "rejected_undecided": sum(s not in (0, 2) for s in st_used),
           "x0": [list(map(float, x)) for x in keep]}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT, {k: v for k, v in doc.items() if k != "x0"})


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 6)
