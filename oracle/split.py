"""The scenario-tree solve split across ranks by subtrees (FP64, numpy): the multi-GPU layout of
the method, restated on host ranks.

TEST INFRASTRUCTURE ONLY: used by the tests, never by the library.  It shares no code with the
CUDA path.

Section III-D makes every stage of Algorithms 3 and 4 parallel over its nodes, and a node's
backward step needs only its children, its forward step only its parent.  So below a split
stage t_s the tree falls apart into independent subtrees rooted at nodes(t_s):

* a rank owns whole subtrees (a contiguous block of the roots in nodes(t_s) and every node
  below them) and the dual entries of those nodes; the stages above t_s (the "top") are
  replicated on every rank, their dual entries counted once (by rank 0) in reductions;
* factor (Section III-D recursion): each rank runs it over its subtrees from the leaves up,
  then the P^r of every root r in nodes(t_s) is all-gathered once and every rank finishes the
  top itself;
* solve (Algorithm 3, or 4 when homogeneous): backward over the owned subtrees, one all-gather
  of the roots' s^r (nx reals per root), the top's backward and forward on every rank, then the
  forward over the owned subtrees from the roots' states;
* NAMA (Algorithm 2): the elementwise work is local; every inner product, the residual's
  infinity norm and the terms of the FBE are all-reduced (one scalar each).

The recursion formulas are those of the oracle's C code (stotree_oracle.c): leaf P^l = pi^l P_N;
parent Rbar = pi^i R + sum B'PB, M = sum B'PA, K = -Rbar^-1 M, P = pi^i Q + sum A'PA + M'K,
gu = sum B'Pc + pi^i r / 2, gx = sum A'Pc + pi^i q / 2; backward s^l = y^l/2 + pi^l p_N/2,
v = y_u/2 + sum B's + gu, ubar = -Rbar^-1 v, s = y_x/2 + sum A's + K'v + gx; forward u = K x + ubar,
x^j = A^j x^i + B^j u^i + c^j.  Hard boxes only (the indicator g of Section II-B).

`comm` is any object with rank, world, allgather(ndarray) -> list of ndarrays in rank order,
allreduce_sum(float) and allreduce_max(float); LocalComm is the one-rank case.  Calls are
counted in comm.calls by the helpers here.
"""
from __future__ import annotations

import numpy as np

from paper_2107_01745_b300.workloads import dual_offsets


class LocalComm:
    rank, world = 0, 1

    def allgather(self, a):
        return [np.asarray(a)]

    def allreduce_sum(self, v):
        return float(v)

    def allreduce_max(self, v):
        return float(v)


def _count(comm, kind):
    calls = getattr(comm, "calls", None)
    if calls is None:
        calls = {}
        comm.calls = calls
    calls[kind] = calls.get(kind, 0) + 1


def split_stage(tree, world):
    """The first stage with at least `world` nodes (each rank then owns at least one subtree)."""
    for t in range(tree.horizon + 1):
        if int(np.sum(tree.stage == t)) >= world:
            return t
    raise ValueError(f"no stage has {world} nodes")


class Plan:
    """Ownership of the nodes for `world` ranks with split stage ts: roots = nodes(ts) in index
    order, split into `world` contiguous blocks; a node at stage >= ts belongs to the owner of
    its ancestor at stage ts; nodes at stages < ts are the replicated top."""

    def __init__(self, tree, world, ts=None):
        self.ts = split_stage(tree, world) if ts is None else ts
        st = tree.stage
        self.roots = np.nonzero(st == self.ts)[0]
        if len(self.roots) < world:
            raise ValueError("fewer subtree roots than ranks")
        nr = len(self.roots)
        bounds = [r * nr // world for r in range(world + 1)]
        self.root_owner = np.empty(nr, dtype=int)
        for r in range(world):
            self.root_owner[bounds[r]:bounds[r + 1]] = r
        owner = np.full(tree.num_nodes, -1)
        for k, root in enumerate(self.roots):
            owner[root] = self.root_owner[k]
        for j in range(tree.num_nodes):
            if st[j] > self.ts:
                owner[j] = owner[tree.parent[j]]
        self.owner = owner  # -1 for the top
        self.world = world


class SplitRank:
    """One rank's part of the factor, the solve step and NAMA."""

    def __init__(self, p, plan, comm):
        t = p.tree
        self.p, self.plan, self.comm = p, plan, comm
        self.nx, self.nu = p.nx, p.nu
        self.Nn, self.Np = t.num_nodes, t.num_nonleaf
        self.rank = comm.rank
        owner = plan.owner
        self.mine = np.nonzero(owner == self.rank)[0]      # owned subtree nodes, index order
        self.top = np.nonzero(owner == -1)[0]              # replicated stages < ts
        self.my_roots = plan.roots[plan.root_owner == self.rank]
        self.off = dual_offsets(t, self.nx, self.nu)
        self.m = int(self.off[-1])
        # per dual element: its node, sqrt(pi), bounds, and the reduction weight (owned entries,
        # and the top's entries on rank 0 only, so that sums count every entry once)
        node_of = np.repeat(np.arange(self.Nn), np.diff(self.off))
        self.sq = np.sqrt(t.prob[node_of])
        lo, hi = np.empty(self.m), np.empty(self.m)
        for i in range(self.Nn):
            o = self.off[i]
            lo[o:o + self.nx], hi[o:o + self.nx] = p.xlo, p.xhi
            if i < self.Np:
                lo[o + self.nx:o + self.nx + self.nu], hi[o + self.nx:o + self.nx + self.nu] = p.ulo, p.uhi
        lo[:self.nx], hi[:self.nx] = -np.inf, np.inf
        self.lo, self.hi = lo, hi
        counted = owner[node_of] == self.rank
        if self.rank == 0:
            counted |= owner[node_of] == -1
        self.weight = counted.astype(float)
        self.present = (owner[node_of] == self.rank) | (owner[node_of] == -1)
        self._factor()

    # -- the Section III-D recursion ---------------------------------------------------
    def _factor_node(self, i):
        p, nx, nu = self.p, self.nx, self.nu
        pi = p.tree.prob[i]
        Rb = pi * np.diag(p.R)
        M = np.zeros((nu, nx))
        Pn = pi * np.diag(p.Q)
        gu = 0.5 * pi * np.asarray(p.r, float)
        gx = 0.5 * pi * np.asarray(p.q, float)
        c0 = p.tree.child_begin[i]
        for j in range(c0, c0 + p.tree.child_count[i]):
            Pj, Aj, Bj, cj = self.P[j], p.A[j], p.B[j], p.c[j]
            Rb = Rb + Bj.T @ Pj @ Bj
            M = M + Bj.T @ Pj @ Aj
            Pn = Pn + Aj.T @ Pj @ Aj
            gu = gu + Bj.T @ Pj @ cj
            gx = gx + Aj.T @ Pj @ cj
        K = -np.linalg.solve(Rb, M)
        Pn = Pn + M.T @ K
        self.P[i] = 0.5 * (Pn + Pn.T)
        self.K[i], self.Rb[i], self.gu[i], self.gx[i] = K, Rb, gu, gx

    def _factor(self):
        p, nx, nu = self.p, self.nx, self.nu
        self.P = np.zeros((self.Nn, nx, nx))
        self.K = np.zeros((self.Np, nu, nx))
        self.Rb = np.zeros((self.Np, nu, nu))
        self.gu = np.zeros((self.Np, nu))
        self.gx = np.zeros((self.Np, nx))
        for l in self.mine:
            if l >= self.Np:
                self.P[l] = p.tree.prob[l] * np.diag(p.PN)
        for i in sorted((i for i in self.mine if i < self.Np), key=lambda i: -p.tree.stage[i]):
            self._factor_node(i)
        # the roots' P, once, to every rank
        _count(self.comm, "allgather_P")
        parts = self.comm.allgather(self.P[self.my_roots])
        for r, part in enumerate(parts):
            self.P[self.plan.roots[self.plan.root_owner == r]] = part
        for i in sorted(self.top, key=lambda i: -p.tree.stage[i]):
            self._factor_node(i)

    # -- Algorithm 3 (homogeneous = False) / 4 (True) ----------------------------------
    def _backward_node(self, i, y, hom, s, ubar):
        p, nx, nu = self.p, self.nx, self.nu
        o = self.off[i]
        v = 0.5 * y[o + nx:o + nx + nu] + (0.0 if hom else self.gu[i])
        acc = 0.5 * y[o:o + nx] + (0.0 if hom else self.gx[i])
        c0 = p.tree.child_begin[i]
        for j in range(c0, c0 + p.tree.child_count[i]):
            v = v + p.B[j].T @ s[j]
            acc = acc + p.A[j].T @ s[j]
        ubar[i] = -np.linalg.solve(self.Rb[i], v)
        s[i] = acc + self.K[i].T @ v

    def _forward_node(self, i, hom, x, u, ubar):
        p = self.p
        u[i] = self.K[i] @ x[i] + ubar[i]
        c0 = p.tree.child_begin[i]
        for j in range(c0, c0 + p.tree.child_count[i]):
            x[j] = p.A[j] @ x[i] + p.B[j] @ u[i] + (0.0 if hom else p.c[j])

    def solve(self, y, homogeneous=False):
        """x(y), u(y) on the owned subtrees and the top (other rows zero).  y: full-length dual
        vector whose owned and top entries are set (unscaled)."""
        p, nx = self.p, self.nx
        hom = homogeneous
        s = np.zeros((self.Nn, nx))
        ubar = np.zeros((self.Np, self.nu))
        for l in self.mine:
            if l >= self.Np:
                o = self.off[l]
                s[l] = 0.5 * y[o:o + nx] + (0.0 if hom else 0.5 * p.tree.prob[l] * np.asarray(p.pN, float))
        for i in sorted((i for i in self.mine if i < self.Np), key=lambda i: -p.tree.stage[i]):
            self._backward_node(i, y, hom, s, ubar)
        # the one exchange of the solve: the roots' s
        _count(self.comm, "allgather_s")
        parts = self.comm.allgather(s[self.my_roots])
        for r, part in enumerate(parts):
            s[self.plan.roots[self.plan.root_owner == r]] = part
        for i in sorted(self.top, key=lambda i: -p.tree.stage[i]):
            self._backward_node(i, y, hom, s, ubar)
        x = np.zeros((self.Nn, nx))
        u = np.zeros((self.Np, self.nu))
        x[0] = 0.0 if hom else np.asarray(p.x0, float)
        for i in sorted(self.top, key=lambda i: p.tree.stage[i]):
            self._forward_node(i, hom, x, u, ubar)
        for i in sorted((i for i in self.mine if i < self.Np), key=lambda i: p.tree.stage[i]):
            self._forward_node(i, hom, x, u, ubar)
        return x, u

    def stack(self, x, u):
        """Hx in the dual layout (rows of nodes this rank does not hold are zero)."""
        nx, nu, npn = self.nx, self.nu, self.Np
        h = np.empty(self.m)
        h[:npn * (nx + nu)] = np.concatenate([x[:npn], u], axis=1).reshape(-1)
        h[npn * (nx + nu):] = x[npn:].reshape(-1)
        return np.where(self.present, h, 0.0)

    # -- reductions ------------------------------------------------------------------------
    def dot(self, a, b):
        _count(self.comm, "allreduce")
        return self.comm.allreduce_sum(float(np.sum(self.weight * a * b)))

    def max_abs(self, a):
        _count(self.comm, "allreduce")
        return self.comm.allreduce_max(float(np.max(np.abs(np.where(self.present, a, 0.0)))))

    def cost(self, x, u):
        """f(x) of Section II-B over the nodes this rank counts (owned, and the top on rank 0)."""
        p, pr, npn = self.p, self.p.tree.prob, self.Np
        counted = np.zeros(self.Nn, dtype=bool)
        counted[self.mine] = True
        if self.rank == 0:
            counted[self.top] = True
        f = 0.0
        for i in np.nonzero(counted)[0]:
            if i < npn:
                f += pr[i] * (x[i] @ (p.Q * x[i]) + u[i] @ (p.R * u[i]) + p.q @ x[i] + p.r @ u[i])
            else:
                f += pr[i] * (x[i] @ (p.PN * x[i]) + p.pN @ x[i])
        _count(self.comm, "allreduce")
        return self.comm.allreduce_sum(f)

    # -- Algorithm 2 ----------------------------------------------------------------------
    def point(self, yb, lam):
        """The same quantities as the oracle's fb_point (hard box): S Hx, z, R, T, phi, ||R||."""
        x, u = self.solve(self.sq * yb)
        h = self.sq * self.stack(x, u)
        v = h + yb / lam
        z = np.minimum(np.maximum(v, self.sq * self.lo), self.sq * self.hi)
        z = np.where(self.present, z, 0.0)
        r = z - h
        f = self.cost(x, u)
        phi = -(f + self.dot(yb, h - z) + 0.5 * lam * self.dot(h - z, h - z))
        return dict(y=yb, h=h, x=x, u=u, z=z, r=r, phi=phi, T=yb - lam * r,
                    res_inf=self.max_abs(r / self.sq))

    def lbfgs_apply(self, S, Y, g, lam):
        """Two-loop recursion (H0 = gamma I of the newest pair, lam I while empty) with
        all-reduced inner products."""
        if not S:
            return lam * g
        q = g.copy()
        rhos = [1.0 / self.dot(s, y) for s, y in zip(S, Y)]
        alphas = []
        for s, y, rho in zip(reversed(S), reversed(Y), reversed(rhos)):
            a = rho * self.dot(s, q)
            alphas.append(a)
            q = q - a * y
        gamma = self.dot(S[-1], Y[-1]) / self.dot(Y[-1], Y[-1])
        rv = gamma * q
        for (s, y, rho), a in zip(zip(S, Y, rhos), reversed(alphas)):
            b = rho * self.dot(y, rv)
            rv = rv + (a - b) * s
        return rv

    def nama(self, lam, tol=1e-8, mem=5, max_iter=1000, max_ls=30, eps_curv=1e-12):
        """Algorithm 2 from y = 0 with the oracle's readings (extrapolation w = y + tau d +
        (1 - tau)(T(y) - y), update y+ = T(w), largest accepted tau, FIFO memory).  Returns the
        scaled iterate (rows of other ranks zero), the iteration count and the residual history."""
        pt = self.point(np.zeros(self.m), lam)
        S, Y = [], []
        res = [pt["res_inf"]]
        k = 0
        while pt["res_inf"] > tol and k < max_iter:
            r = pt["r"]
            d = -self.lbfgs_apply(S, Y, r, lam)
            fb = pt["T"] - pt["y"]
            tau, wp = 1.0, None
            for _ in range(max_ls + 1):
                cand = self.point(pt["y"] + tau * d + (1.0 - tau) * fb, lam)
                if cand["phi"] <= pt["phi"]:
                    wp = cand
                    break
                tau *= 0.5
            if wp is None:
                wp = self.point(pt["T"].copy(), lam)
            new = self.point(wp["T"], lam)
            s = new["y"] - pt["y"]
            q = new["r"] - r
            if self.dot(s, q) > eps_curv * self.dot(s, s) * self.dot(r, r):
                S.append(s)
                Y.append(q)
                if len(S) > mem:
                    S.pop(0)
                    Y.pop(0)
            pt = new
            k += 1
            res.append(pt["res_inf"])
        return dict(ybar=pt["y"], x=pt["x"], u=pt["u"], iters=k, res=res, res_inf=pt["res_inf"])
