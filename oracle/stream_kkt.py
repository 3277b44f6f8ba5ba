"""FP64 optimality residuals of a solve step, streamed over the nodes (large instances).

TEST INFRASTRUCTURE ONLY: used by the tests, never by the library.  It shares no code with the
CUDA path.

x(y) of Algorithm 3 is the minimiser of the inner problem (Section III-D)

    min  sum_i pi^i (x^i'Q x^i + u^i'R u^i + q'x^i + r'u^i) + sum_l pi^l (x^l'P_N x^l + p_N'x^l) + <y, Hx>
    s.t. x^0 = p,  x^j = A^j x^anc(j) + B^j u^anc(j) + c^j,

with Hx = [x^i; u^i] per nonleaf node and x^l per leaf (no 1/2 in the cost).  With a
multiplier mu^j per dynamics equation, stationarity reads

    leaf l:        mu^l = 2 pi^l P_N x^l + pi^l p_N + y^l
    nonleaf j > 0: mu^j = 2 pi^j Q x^j + pi^j q + y_x^j + sum_{c in child(j)} A^c' mu^c
    nonleaf i:     0    = 2 pi^i R u^i + pi^i r + y_u^i + sum_{c in child(i)} B^c' mu^c

so a candidate (x, u) is the solve step's result exactly when the dynamics hold and the u
equations hold with the mu defined by the first two lines.  This module computes those
residuals in FP64 from the leaves up, reading the per-node A, B, c in blocks of children (each
block is regenerated on demand), so no full per-node array is ever held.  The homogeneous
variant (Algorithm 4) drops c, q, r, p_N and p.
"""
from __future__ import annotations

import numpy as np


def solve_step_residuals(p, y, x, u, homogeneous=False, block=2048):
    """Residuals of a candidate (x [Nn][nx], u [Np][nu]) for the dual y (unscaled, dual layout).

    Returns a dict with the largest absolute residual of the dynamics and of the u equations,
    and the scales they are measured against (the largest |term| entering each equation)."""
    t = p.tree
    nx, nu = p.nx, p.nu
    nn, npn = t.num_nodes, t.num_nonleaf
    par, prob, stage = t.parent, t.prob, t.stage
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    hom = 0.0 if homogeneous else 1.0
    nxu = nx + nu
    Q, R, PN = np.asarray(p.Q, float), np.asarray(p.R, float), np.asarray(p.PN, float)
    q, r, pN = hom * np.asarray(p.q, float), hom * np.asarray(p.r, float), hom * np.asarray(p.pN, float)

    def ydx(i):  # x part of node i's dual block
        return y[i * nxu:i * nxu + nx] if i < npn else y[npn * nxu + (i - npn) * nx:npn * nxu + (i - npn + 1) * nx]

    # mu for every node, the child sums accumulated into the parents, stage by stage from the
    # leaves; each stage's children are read in blocks
    mu = np.zeros((nn, nx))
    accA = np.zeros((nn, nx))   # sum_c A^c' mu^c per parent
    accB = np.zeros((npn, nu))  # sum_c B^c' mu^c per parent
    dyn_res, dyn_scale = 0.0, 0.0
    soff = [int(np.searchsorted(stage, s)) for s in range(t.horizon + 2)]
    for s in range(t.horizon, 0, -1):
        f0, f1 = soff[s], soff[s + 1]
        # mu of the stage's nodes (their own children are done)
        for j in range(f0, f1):
            if j >= npn:
                mu[j] = 2.0 * prob[j] * PN * x[j] + prob[j] * pN + ydx(j)
            else:
                mu[j] = 2.0 * prob[j] * Q * x[j] + prob[j] * q + ydx(j) + accA[j]
        for b0 in range(f0, f1, block):
            b1 = min(f1, b0 + block)
            A = p.A[b0:b1]
            B = p.B[b0:b1]
            c = p.c[b0:b1]
            pp = par[b0:b1]
            xp = x[pp]
            up = u[pp]
            # dynamics: x^j - A^j x^i - B^j u^i - c^j
            ax = np.einsum("nij,nj->ni", A, xp)
            bu = np.einsum("nij,nj->ni", B, up)
            res = x[b0:b1] - ax - bu - hom * c
            dyn_res = max(dyn_res, float(np.max(np.abs(res))))
            dyn_scale = max(dyn_scale, float(np.max(np.abs(x[b0:b1]))), float(np.max(np.abs(ax))),
                            float(np.max(np.abs(bu))))
            # children's contributions to their parents
            np.add.at(accA, pp, np.einsum("nij,ni->nj", A, mu[b0:b1]))
            np.add.at(accB, pp, np.einsum("nij,ni->nj", B, mu[b0:b1]))
    # u equations of every nonleaf node
    yu = y[:npn * nxu].reshape(npn, nxu)[:, nx:]
    ru = 2.0 * prob[:npn, None] * R[None, :] * u + prob[:npn, None] * r[None, :] + yu + accB
    u_scale = max(float(np.max(np.abs(2.0 * prob[:npn, None] * R[None, :] * u))), float(np.max(np.abs(yu))),
                  float(np.max(np.abs(accB))))
    # the root state is the parameter
    root_res = float(np.max(np.abs(x[0] - hom * np.asarray(p.x0, float))))
    return {"dynamics": max(dyn_res, root_res), "dynamics_scale": dyn_scale, "u_eq": float(np.max(np.abs(ru))),
            "u_scale": u_scale}
