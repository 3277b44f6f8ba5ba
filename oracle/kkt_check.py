"""FP64 optimality residuals of a primal-dual pair (x, u, y), node by node.

TEST INFRASTRUCTURE ONLY: used by the tests, never by the library.  It shares no code with the
CUDA path.

A pair solves the problem of Section II when (Section II-D, and the termination meaning given
with Algorithm 1):

* x, u satisfy the dynamics of eq. system_dynamics_tree, x^j = A^j x^i + B^j u^i + c^j for every
  child j of i, with x^0 = p;
* (x, u) minimises f(x) + <y, Hx> over the dynamics (x = x(y) of Algorithm 3), i.e. with one
  multiplier mu^j per dynamics equation (costate),
      leaf l:          mu^l = 2 pi^l P_N x^l + pi^l p_N + y^l
      nonleaf j >= 1:  mu^j = 2 pi^j Q x^j + pi^j q + y_x^j + sum_{c in child(j)} A^c' mu^c
      nonleaf i:       0    = 2 pi^i R u^i + pi^i r + y_u^i + sum_{c in child(i)} B^c' mu^c
  (the cost of Section II-B without the factor 1/2); the last line is the stationarity residual;
* y is in the subdifferential of g at Hx, per component k of the dual layout with h = (Hx)_k:
  - g_k the indicator of [lo_k, hi_k] (kind 0): lo <= h <= hi (feasibility), y_k = 0 strictly
    inside (complementarity), y_k >= 0 at the upper bound and y_k <= 0 at the lower one (sign);
  - g_k = rho dist(h, [lo, hi]) (kind 1): the subdifferential is {rho} above the box, {-rho}
    below it, {0} strictly inside, [0, rho] at hi, [-rho, 0] at lo ([-rho, rho] for a point box);
  - g_k = rho Huber_delta(dist(h, [lo, hi])) (kind 2): differentiable, derivative
    rho min(d, delta) sign, d the distance, sign +1 above the box and -1 below it.
  The root's state block is the parameter and carries no term (its y must be zero).

With general constraint maps (Section II-C: z^i = F x^i + G u^i, z^l = FN x^l) the same conditions
hold with H'y in place of y in the costates and u equations (per nonleaf node F'y^i for the state
part and G'y^i for the input part, FN'y^l at a leaf) and with the box on z, the root's block
included (x^0 = x0).

kkt_residuals returns the six numbers that stotree_kkt_check defines (largest violations, with
points within tol_active of a bound counted as lying on it):
  dynamics, stationarity, feasibility (hard components), complementarity (hard components
  strictly inside; soft components whose subdifferential is one value: distance of y to it),
  sign (hard components at one bound; soft components at a kink: distance of y to the interval),
  gap: the sum over the components of the Fenchel-Young gap g_k(h) + g_k*(y_k) - y_k h >= 0 (Section
  II-D: with x = x(y) it is the primal objective f(x) + g(Hx) minus the dual objective at y), with
  the box's g taken as 0 (feasibility is reported apart) and the conjugates' domains not imposed.
"""
from __future__ import annotations

import numpy as np


def _dual_block(p, i):
    """(offset, length) of node i's block in a dual-sized vector."""
    nx, nu = p.nx, p.nu
    npn = p.tree.num_nonleaf
    if i < npn:
        return i * (nx + nu), nx + nu
    return npn * (nx + nu) + (i - npn) * nx, nx


def _ht_blocks(p, y):
    """H'y in the [x; u] layout (the selection maps: y itself)."""
    if not p.general:
        return np.asarray(y, dtype=np.float64)
    t = p.tree
    npn, nn, nx, nu = t.num_nonleaf, t.num_nodes, p.nx, p.nu
    nc, ncn = p.F.shape[0], p.FN.shape[0]
    out = np.empty(npn * (nx + nu) + (nn - npn) * nx)
    for i in range(nn):
        if i < npn:
            yi = y[i * nc:(i + 1) * nc]
            out[i * (nx + nu):i * (nx + nu) + nx] = p.F.T @ yi
            out[i * (nx + nu) + nx:(i + 1) * (nx + nu)] = p.G.T @ yi
        else:
            o = npn * nc + (i - npn) * ncn
            out[npn * (nx + nu) + (i - npn) * nx:npn * (nx + nu) + (i - npn + 1) * nx] = p.FN.T @ y[o:o + ncn]
    return out


def _fy_gap(h, y, lo, hi, kind, rho, delta):
    """g(h) + g*(y) - y h for one component (see the module docstring).  The support function of
    [lo, hi] is hi y for y > 0 and lo y for y < 0; g is 0 (box), rho d (kind 1) or rho Huber_delta(d)
    (kind 2) with d the distance of h to the box; g* adds y^2 / (2 rho) for Huber."""
    if y > 0:
        t = y * (hi - h)
    elif y < 0:
        t = y * (lo - h)
    else:
        t = 0.0
    if kind != 0:
        d = max(lo - h, 0.0) + max(h - hi, 0.0)
        if kind == 1:
            t += rho * d
        else:
            t += rho * (0.5 * d * d if d <= delta else delta * (d - 0.5 * delta)) + y * y / (2.0 * rho)
    return t


def _component_terms(p):
    """Per component of [x; u]: lo, hi, kind, rho, delta (hard box when no penalty is set)."""
    lo = np.concatenate([np.asarray(p.xlo, float), np.asarray(p.ulo, float)])
    hi = np.concatenate([np.asarray(p.xhi, float), np.asarray(p.uhi, float)])
    n = p.nx + p.nu
    if getattr(p, "pen_kind", None) is None:
        return lo, hi, np.zeros(n, dtype=int), np.zeros(n), np.ones(n)
    return lo, hi, np.asarray(p.pen_kind, int), np.asarray(p.pen_rho, float), np.asarray(p.pen_delta, float)


def kkt_residuals(p, x0, x, u, y, tol_active):
    """The five residuals of (x [Nn][nx], u [Np][nu], y [m] unscaled) for the root state x0."""
    t = p.tree
    nx, nu = p.nx, p.nu
    nn, npn = t.num_nodes, t.num_nonleaf
    prob, parent = np.asarray(t.prob, float), np.asarray(t.parent)
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    y_dual = np.asarray(y, dtype=np.float64)
    y = _ht_blocks(p, y_dual)  # the dual as it enters the costates and u equations
    x0 = np.asarray(x0, dtype=np.float64)
    Q, R, PN = (np.asarray(v, float) for v in (p.Q, p.R, p.PN))
    q, r, pN = (np.asarray(v, float) for v in (p.q, p.r, p.pN))

    def xstate(i):  # the root's state is the parameter
        return x0 if i == 0 else x[i]

    # dynamics of every non-root node
    dyn = 0.0
    for j in range(1, nn):
        i = parent[j]
        res = x[j] - (p.A[j] @ xstate(i) + p.B[j] @ u[i] + p.c[j])
        dyn = max(dyn, float(np.max(np.abs(res))))

    # costates from the leaves up (children have larger indices than their parent), and the
    # input stationarity at every nonleaf node
    mu = np.zeros((nn, nx))
    sumA = np.zeros((nn, nx))  # sum over children c of A^c' mu^c
    sumB = np.zeros((nn, nu))  # sum over children c of B^c' mu^c
    stat = 0.0
    for j in range(nn - 1, -1, -1):
        o, _ = _dual_block(p, j)
        if j >= npn:
            mu[j] = 2.0 * prob[j] * PN * x[j] + prob[j] * pN + y[o:o + nx]
        else:
            ru = 2.0 * prob[j] * R * u[j] + prob[j] * r + y[o + nx:o + nx + nu] + sumB[j]
            stat = max(stat, float(np.max(np.abs(ru))))
            if j > 0:
                mu[j] = 2.0 * prob[j] * Q * x[j] + prob[j] * q + y[o:o + nx] + sumA[j]
        if j > 0:
            sumA[parent[j]] += p.A[j].T @ mu[j]
            sumB[parent[j]] += p.B[j].T @ mu[j]

    if p.general:
        return {"dynamics": dyn, "stationarity": stat, **_box_on_z(p, x0, x, u, y_dual, tol_active)}
    # the nonsmooth term, component by component
    lo, hi, kind, rho, delta = _component_terms(p)
    feas = comp = sign = gap = 0.0
    for i in range(nn):
        o, n = _dual_block(p, i)
        h = np.concatenate([xstate(i), u[i]]) if i < npn else x[i]
        for k in range(n):
            yk, hk = float(y[o + k]), float(h[k])
            if i == 0 and k < nx:  # the parameter: no term, so y must vanish
                comp = max(comp, abs(yk))
                continue
            gap += _fy_gap(hk, yk, lo[k], hi[k], kind[k], rho[k], delta[k])
            if kind[k] == 0:
                feas = max(feas, lo[k] - hk, hk - hi[k], 0.0)
                at_hi, at_lo = hk >= hi[k] - tol_active, hk <= lo[k] + tol_active
                if not at_hi and not at_lo:
                    comp = max(comp, abs(yk))
                elif at_hi and not at_lo:
                    sign = max(sign, -yk)
                elif at_lo and not at_hi:
                    sign = max(sign, yk)
                continue
            if kind[k] == 1:
                if hk > hi[k] + tol_active:
                    sub = (rho[k], rho[k])
                elif hk < lo[k] - tol_active:
                    sub = (-rho[k], -rho[k])
                else:
                    sub = (-rho[k] if hk <= lo[k] + tol_active else 0.0,
                           rho[k] if hk >= hi[k] - tol_active else 0.0)
            else:
                d = max(lo[k] - hk, 0.0) + max(hk - hi[k], 0.0)
                gd = rho[k] * min(d, delta[k])
                v = gd if hk > hi[k] else (-gd if hk < lo[k] else 0.0)
                sub = (v, v)
            viol = max(sub[0] - yk, yk - sub[1], 0.0)
            if sub[0] == sub[1]:
                comp = max(comp, viol)
            else:
                sign = max(sign, viol)
    return {"dynamics": dyn, "stationarity": stat, "feasibility": feas, "complementarity": comp, "sign": sign,
            "gap": gap}


def _box_on_z(p, x0, x, u, y, tol_active):
    """Feasibility, complementarity and sign of the box on z = F x + G u (FN x at the leaves)."""
    t = p.tree
    npn, nn = t.num_nonleaf, t.num_nodes
    nc, ncn = p.F.shape[0], p.FN.shape[0]
    feas = comp = sign = gap = 0.0
    for i in range(nn):
        if i < npn:
            z = p.F @ (x0 if i == 0 else x[i]) + p.G @ u[i]
            yi, lo, hi = y[i * nc:(i + 1) * nc], p.zlo, p.zhi
        else:
            o = npn * nc + (i - npn) * ncn
            z = p.FN @ x[i]
            yi, lo, hi = y[o:o + ncn], p.zNlo, p.zNhi
        for k in range(len(z)):
            zk, yk = float(z[k]), float(yi[k])
            gap += _fy_gap(zk, yk, lo[k], hi[k], 0, 0.0, 1.0)
            feas = max(feas, lo[k] - zk, zk - hi[k], 0.0)
            at_hi, at_lo = zk >= hi[k] - tol_active, zk <= lo[k] + tol_active
            if not at_hi and not at_lo:
                comp = max(comp, abs(yk))
            elif at_hi and not at_lo:
                sign = max(sign, -yk)
            elif at_lo and not at_hi:
                sign = max(sign, yk)
    return {"feasibility": feas, "complementarity": comp, "sign": sign, "gap": gap}

