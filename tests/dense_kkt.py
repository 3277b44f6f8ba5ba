"""Dense reference solutions used to pin the oracle (tests only).

These build the scenario-tree problem of Section II as one dense equality- (or
active-set-) constrained QP and hand it to numpy.linalg.solve, so they share no
recursion, factorisation or ordering with the tree dynamic programme.
"""
import numpy as np


def _index(p):
    t = p.tree
    nn, npl, nx, nu = t.num_nodes, t.num_nonleaf, p.nx, p.nu
    uoff = {i: i * nu for i in range(npl)}
    xoff = {j: npl * nu + (j - 1) * nx for j in range(1, nn)}
    nv = npl * nu + (nn - 1) * nx
    return uoff, xoff, nv


def build_qp(p, y, homogeneous=False):
    """min 1/2 v'Gv + g'v  s.t.  E v = e  for  f(x) + <y, Hx>  under the dynamics.
    v = (u^0..u^{Np-1}, x^1..x^{Nn-1}); y is unscaled, dual-sized (the term <y, Hx> enters g
    through the rows of H, h_rows; with general constraint maps H is F, G, FN)."""
    t = p.tree
    nn, npl, nx, nu = t.num_nodes, t.num_nonleaf, p.nx, p.nu
    pr = t.prob
    uoff, xoff, nv = _index(p)
    G = np.zeros((nv, nv))
    g = np.zeros(nv)
    lin = 0.0 if homogeneous else 1.0
    for i in range(npl):
        o = uoff[i]
        G[o:o + nu, o:o + nu] = 2.0 * pr[i] * np.diag(p.R)
        g[o:o + nu] = lin * pr[i] * p.r
    for j in range(1, nn):
        o = xoff[j]
        if j < npl:
            G[o:o + nx, o:o + nx] = 2.0 * pr[j] * np.diag(p.Q)
            g[o:o + nx] = lin * pr[j] * p.q
        else:
            G[o:o + nx, o:o + nx] = 2.0 * pr[j] * np.diag(p.PN)
            g[o:o + nx] = lin * pr[j] * p.pN
    Hm, _ = h_rows(p)
    g = g + Hm.T @ np.asarray(y, dtype=np.float64)
    E = np.zeros(((nn - 1) * nx, nv))
    e = np.zeros((nn - 1) * nx)
    x0 = np.zeros(nx) if homogeneous else p.x0
    for j in range(1, nn):
        i = int(t.parent[j])
        row = (j - 1) * nx
        E[row:row + nx, xoff[j]:xoff[j] + nx] = np.eye(nx)
        E[row:row + nx, uoff[i]:uoff[i] + nu] = -p.B[j]
        rhs = (0.0 if homogeneous else 1.0) * p.c[j]
        if i == 0:
            rhs = rhs + p.A[j] @ x0
        else:
            E[row:row + nx, xoff[i]:xoff[i] + nx] = -p.A[j]
        e[row:row + nx] = rhs
    return G, g, E, e


def unpack(p, v, homogeneous=False):
    t = p.tree
    nn, npl, nx, nu = t.num_nodes, t.num_nonleaf, p.nx, p.nu
    uoff, xoff, _ = _index(p)
    x = np.zeros((nn, nx))
    x[0] = 0.0 if homogeneous else p.x0
    for j in range(1, nn):
        x[j] = v[xoff[j]:xoff[j] + nx]
    u = np.stack([v[uoff[i]:uoff[i] + nu] for i in range(npl)])
    return x, u


def dense_solve(p, y, homogeneous=False):
    """x(y): minimiser of f(x) + <y, Hx> over the dynamics, by one dense KKT solve."""
    G, g, E, e = build_qp(p, y, homogeneous)
    nv, nc = G.shape[0], E.shape[0]
    K = np.block([[G, E.T], [E, np.zeros((nc, nc))]])
    sol = np.linalg.solve(K, np.concatenate([-g, e]))
    return unpack(p, sol[:nv], homogeneous)


def h_rows(p):
    """Hx (laid out like y) as Hm v + const: the selection of [x^i; u^i] / x^l, or with general
    constraint maps F x^i + G u^i / FN x^l; the root state enters the constant."""
    t = p.tree
    nn, npl, nx, nu = t.num_nodes, t.num_nonleaf, p.nx, p.nu
    uoff, xoff, nv = _index(p)
    from paper_2107_01745_b300.workloads import problem_offsets
    off = problem_offsets(p)
    m = int(off[-1])
    Hm = np.zeros((m, nv))
    const = np.zeros(m)
    if p.general:
        nc, ncn = p.F.shape[0], p.FN.shape[0]
        for i in range(nn):
            o = off[i]
            if i < npl:
                if i == 0:
                    const[o:o + nc] = p.F @ p.x0
                else:
                    Hm[o:o + nc, xoff[i]:xoff[i] + nx] = p.F
                Hm[o:o + nc, uoff[i]:uoff[i] + nu] = p.G
            else:
                Hm[o:o + ncn, xoff[i]:xoff[i] + nx] = p.FN
        return Hm, const
    for i in range(nn):
        o = off[i]
        if i == 0:
            const[o:o + nx] = p.x0
        else:
            Hm[o:o + nx, xoff[i]:xoff[i] + nx] = np.eye(nx)
        if i < npl:
            Hm[o + nx:o + nx + nu, uoff[i]:uoff[i] + nu] = np.eye(nu)
    return Hm, const


def box_vectors(p):
    from paper_2107_01745_b300.workloads import dual_offsets, problem_offsets
    t = p.tree
    nx, nu = p.nx, p.nu
    off = problem_offsets(p)
    m = int(off[-1])
    lo, hi = np.empty(m), np.empty(m)
    if p.general:
        for i in range(t.num_nodes):
            o, o1 = off[i], off[i + 1]
            lo[o:o1], hi[o:o1] = (p.zlo, p.zhi) if i < t.num_nonleaf else (p.zNlo, p.zNhi)
        return lo, hi
    for i in range(t.num_nodes):
        o = off[i]
        lo[o:o + nx], hi[o:o + nx] = p.xlo, p.xhi
        if i < t.num_nonleaf:
            lo[o + nx:o + nx + nu], hi[o + nx:o + nx + nu] = p.ulo, p.uhi
    lo[:nx], hi[:nx] = -np.inf, np.inf
    return lo, hi


def active_set_qp(p, y_guess, thresh=1e-7):
    """Exact solution of the box-constrained primal QP for the active set read off a dual guess.

    Returns (x, u, y_exact, certified) where ``certified`` says whether the
    candidate satisfies every KKT condition: primal feasibility of the inactive
    bounds and the sign of every active multiplier."""
    G, g, E, e = build_qp(p, np.zeros_like(y_guess))
    Hm, const = h_rows(p)
    lo, hi = box_vectors(p)
    up = y_guess > thresh
    dn = y_guess < -thresh
    act = np.nonzero(up | dn)[0]
    C = Hm[act]
    b = np.where(up[act], hi[act], lo[act]) - const[act]
    nv, ne, na = G.shape[0], E.shape[0], act.size
    K = np.block([[G, E.T, C.T],
                  [E, np.zeros((ne, ne)), np.zeros((ne, na))],
                  [C, np.zeros((na, ne)), np.zeros((na, na))]])
    sol = np.linalg.solve(K, np.concatenate([-g, e, b]))
    v = sol[:nv]
    nu_act = sol[nv + ne:]
    y = np.zeros_like(y_guess)
    y[act] = nu_act
    hx = Hm @ v + const
    feas = np.all(hx <= hi + 1e-9) and np.all(hx >= lo - 1e-9)
    signs = np.all(nu_act[up[act]] >= -1e-12) and np.all(nu_act[dn[act]] <= 1e-12)
    x, u = unpack(p, v)
    return x, u, y, bool(feas and signs)


def feasible(p):
    """Is the box-constrained problem feasible?  One LP (scipy HiGHS) over the dense dynamics."""
    import scipy.optimize
    G, g, E, e = build_qp(p, np.zeros(p.num_dual))
    Hm, const = h_rows(p)
    lo, hi = box_vectors(p)
    keep = np.isfinite(lo) | np.isfinite(hi)
    A_ub = np.vstack([Hm[keep], -Hm[keep]])
    b_ub = np.concatenate([hi[keep] - const[keep], -(lo[keep] - const[keep])])
    fin = np.isfinite(b_ub)
    res = scipy.optimize.linprog(np.zeros(G.shape[0]), A_ub=A_ub[fin], b_ub=b_ub[fin], A_eq=E, b_eq=e,
                                 bounds=(None, None), method="highs")
    return res.status == 0


def boxed_problem(seed, frac=0.7, **kw):
    """Random ragged problem whose box is frac x the range of its unconstrained solution
    (the recipe of the paper-scale workload), relaxed until the LP says it is feasible."""
    from paper_2107_01745_b300 import workloads as W
    p = W.random_problem(seed, box_scale=1e6, **kw)
    x, u = dense_solve(p, np.zeros(p.num_dual))
    for f in (frac, frac + 0.1, frac + 0.2, 1.0):
        W.with_box(p, f * np.max(np.abs(x[1:]), axis=0), f * np.max(np.abs(u), axis=0))
        if feasible(p):
            p.name = f"boxed{seed}"
            return p
    raise RuntimeError("no feasible box")


def constrained_boxed_problem(seed, frac=0.7, **kw):
    """Random problem with general constraint maps z = F x + G u (FN x at the leaves) whose z box is
    frac x the range of z along its unconstrained solution, relaxed until the LP says it is
    feasible."""
    from paper_2107_01745_b300 import workloads as W
    p = W.constrained_problem(seed, **kw)
    x, u = dense_solve(p, np.zeros(p.num_dual))
    npl = p.tree.num_nonleaf
    zn = x[:npl] @ p.F.T + u @ p.G.T
    zl = x[npl:] @ p.FN.T
    for f in (frac, frac + 0.1, frac + 0.2, 1.0):
        zmax, zNmax = f * np.max(np.abs(zn), axis=0), f * np.max(np.abs(zl), axis=0)
        W.with_constraints(p, p.F, p.G, p.FN, -zmax, zmax, -zNmax, zNmax)
        if feasible(p):
            p.name = f"fg{seed}"
            return p
    raise RuntimeError("no feasible box")
