"""Pins of oracle/kkt_check.py, the FP64 optimality residuals of a primal-dual pair (CPU).

The residuals are checked against facts outside the module:

* at the exact solution of the box-constrained QP (dense active-set KKT solve, certified), all
  five vanish to rounding;
* a planted violation moves exactly the residual the optimality conditions say it moves, by the
  amount they fix in closed form: a leaf state off its dynamics by delta (dynamics = |delta|), an
  input moved by delta (stationarity = 2 pi R delta), a state pushed past its bound
  (feasibility), a multiplier strictly inside the box (complementarity), a multiplier of the
  wrong sign at an active bound (sign);
* at any input trajectory and dual, the stationarity residual equals the largest entry of the
  gradient of f(x(u)) + <y, Hx(u)>, taken by central differences of the rolled-out Lagrangian;
* for soft terms, the residual at hand-placed points equals the distance of y to the
  subdifferential written out by hand for that point.
"""
import numpy as np
import pytest

from oracle import kkt_check as KC
from paper_2107_01745_b300 import workloads as W
from tests import dense_kkt as D

PROBS = [D.boxed_problem(12, horizon=3, nx=3, nu=2), D.boxed_problem(16, horizon=3, nx=5, nu=3, frac=0.9),
         D.boxed_problem(17, horizon=4, nx=4, nu=2, frac=0.9)]


def _solution(p):
    """The certified QP solution: the active set comes from a long FP64 NAMA run of the oracle,
    the values from the dense active-set KKT system."""
    from oracle import oracle as O
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    res = O.nama(o, lam, tol=1e-11, max_iter=2000)
    x, u, y, ok = D.active_set_qp(p, res["y"], thresh=1e-7)
    assert ok
    return x, u, y


@pytest.fixture(scope="module", params=range(len(PROBS)), ids=lambda k: PROBS[k].name)
def solved(request):
    p = PROBS[request.param]
    return (p,) + _solution(p)


def _blk(p, i):
    return KC._dual_block(p, i)[0]


def test_zero_at_the_certified_solution(solved):
    p, x, u, y = solved
    r = KC.kkt_residuals(p, p.x0, x, u, y, tol_active=1e-8)
    scale = max(1.0, np.max(np.abs(y)), np.max(np.abs(x)))
    for k, v in r.items():
        assert v <= 1e-10 * scale, (k, v)
    # the QP has active constraints, so the sign and complementarity parts were exercised
    assert np.count_nonzero(np.abs(y) > 1e-7) > 0


def test_leaf_state_off_its_dynamics(solved):
    p, x, u, y = solved
    j = p.tree.num_nodes - 1
    x2 = x.copy()
    x2[j, 1 % p.nx] += 3e-3
    r = KC.kkt_residuals(p, p.x0, x2, u, y, tol_active=1e-8)
    assert abs(r["dynamics"] - 3e-3) <= 1e-12


def test_input_moved_changes_its_stationarity(solved):
    p, x, u, y = solved
    i, a = 0, p.nu - 1
    u2 = u.copy()
    u2[i, a] += 2e-3
    r = KC.kkt_residuals(p, p.x0, x, u2, y, tol_active=1e-8)
    expect = 2.0 * p.tree.prob[i] * p.R[a] * 2e-3
    assert abs(r["stationarity"] - expect) <= 1e-9 * expect + 1e-13


def _rollout(p, u):
    t = p.tree
    x = np.zeros((t.num_nodes, p.nx))
    x[0] = p.x0
    for j in range(1, t.num_nodes):
        i = t.parent[j]
        x[j] = p.A[j] @ x[i] + p.B[j] @ u[i] + p.c[j]
    return x


def _lagrangian(p, u, y):
    """f(x(u)) + <y, Hx(u)> with x(u) rolled out through the dynamics (cost of Section II-B)."""
    t = p.tree
    npn = t.num_nonleaf
    x = _rollout(p, u)
    pr = t.prob
    f = sum(pr[i] * (x[i] @ (p.Q * x[i]) + u[i] @ (p.R * u[i]) + p.q @ x[i] + p.r @ u[i]) for i in range(npn))
    f += sum(pr[l] * (x[l] @ (p.PN * x[l]) + p.pN @ x[l]) for l in range(npn, t.num_nodes))
    h = np.concatenate([np.concatenate([x[i], u[i]]) if i < npn else x[i] for i in range(t.num_nodes)])
    return f + y @ h


@pytest.mark.parametrize("seed", [7, 8])
def test_stationarity_is_the_reduced_gradient(seed):
    """For a trajectory that satisfies the dynamics, the u equations of the costate recursion are
    the gradient of f(x(u)) + <y, Hx(u)> in u (the adjoint method).  The function is quadratic, so
    central differences give that gradient exactly up to rounding, without any recursion."""
    p = W.random_problem(seed, horizon=4, nx=3, nu=2)
    rng = np.random.default_rng(seed)
    npn = p.tree.num_nonleaf
    u = rng.standard_normal((npn, p.nu))
    y = W.random_dual(p, seed + 1)
    x = _rollout(p, u)
    hstep = 1e-3
    grad = np.zeros_like(u)
    for i in range(npn):
        for a in range(p.nu):
            up, dn = u.copy(), u.copy()
            up[i, a] += hstep
            dn[i, a] -= hstep
            grad[i, a] = (_lagrangian(p, up, y) - _lagrangian(p, dn, y)) / (2 * hstep)
    r = KC.kkt_residuals(p, p.x0, x, u, y, tol_active=1e-8)
    g = float(np.max(np.abs(grad)))
    assert abs(r["stationarity"] - g) <= 1e-8 * g
    assert r["dynamics"] <= 1e-13 * max(1.0, float(np.max(np.abs(x))))


def test_state_past_its_bound_is_infeasible(solved):
    p, x, u, y = solved
    j = p.tree.num_nodes - 1
    x2 = x.copy()
    x2[j, 0] = p.xhi[0] + 0.25
    r = KC.kkt_residuals(p, p.x0, x2, u, y, tol_active=1e-8)
    assert abs(r["feasibility"] - 0.25) <= 1e-14


def test_multiplier_inside_the_box_breaks_complementarity(solved):
    p, x, u, y = solved
    h = np.concatenate([np.concatenate([x[i], u[i]]) if i < p.tree.num_nonleaf else x[i]
                        for i in range(p.tree.num_nodes)])
    lo, hi = D.box_vectors(p)
    inside = np.nonzero((h < hi - 1e-3) & (h > lo + 1e-3))[0]
    inside = inside[inside >= p.nx]  # not the root's state
    k = int(inside[len(inside) // 2])
    y2 = y.copy()
    y2[k] = -0.0375
    r = KC.kkt_residuals(p, p.x0, x, u, y2, tol_active=1e-8)
    assert abs(r["complementarity"] - 0.0375) <= 1e-14
    # and a nonzero dual on the root's state (the parameter carries no term) is caught too
    y3 = y.copy()
    y3[0] = 0.5
    assert abs(KC.kkt_residuals(p, p.x0, x, u, y3, tol_active=1e-8)["complementarity"] - 0.5) <= 1e-14


def test_wrong_sign_at_an_active_bound(solved):
    p, x, u, y = solved
    act = np.nonzero(np.abs(y) > 1e-6)[0]
    k = int(act[0])
    y2 = y.copy()
    y2[k] = -y[k]
    r = KC.kkt_residuals(p, p.x0, x, u, y2, tol_active=1e-8)
    assert abs(r["sign"] - abs(y[k])) <= 1e-12 * max(1.0, abs(y[k]))


def test_soft_terms_by_hand():
    """One component of each kind, placed by hand; the other components sit at zero multiplier
    strictly inside a loose box, so only the planted component contributes."""
    p = W.random_problem(5, horizon=1, nx=2, nu=1, box_scale=1.0)
    t = p.tree
    nn, npn = t.num_nodes, t.num_nonleaf
    W.with_box(p, np.array([1.0, 1.0]), np.array([1.0]))
    W.with_penalty(p, np.array([1, 2, 0]), np.array([2.0, 3.0, 0.0]), np.array([1.0, 0.5, 1.0]))
    x = np.zeros((nn, p.nx))
    u = np.zeros((npn, p.nu))
    y = np.zeros(p.num_dual)
    leaf = npn  # first leaf
    o = KC._dual_block(p, leaf)[0]

    def res(xv, yv, comp):
        x[:] = 0.0
        y[:] = 0.0
        x[leaf, comp] = xv
        y[o + comp] = yv
        return KC.kkt_residuals(p, p.x0, x, u, y, tol_active=1e-9)

    # kind 1 (rho = 2) above the box: subdifferential {2}
    assert abs(res(1.5, 0.5, 0)["complementarity"] - 1.5) <= 1e-15
    # kind 1 at the upper bound: [0, 2]; y = 2.5 is 0.5 away, y = 1 is inside
    assert abs(res(1.0, 2.5, 0)["sign"] - 0.5) <= 1e-15
    assert res(1.0, 1.0, 0)["sign"] == 0.0
    # kind 1 inside: {0}
    assert abs(res(0.2, -0.7, 0)["complementarity"] - 0.7) <= 1e-15
    # kind 2 (rho = 3, delta = 0.5) below the box by 0.2: derivative -3 * 0.2 = -0.6
    assert abs(res(-1.2, 0.0, 1)["complementarity"] - 0.6) <= 1e-12
    # beyond delta the derivative saturates at rho delta = 1.5
    assert abs(res(2.0, 1.0, 1)["complementarity"] - 0.5) <= 1e-12


FG_PROBS = [dict(seed=81, horizon=3, nx=3, nu=2, nc=4, ncN=2), dict(seed=85, horizon=4, nx=4, nu=2, nc=3, ncN=4)]


@pytest.mark.parametrize("kw", FG_PROBS, ids=lambda k: f"fg{k['seed']}")
def test_general_maps_zero_at_the_certified_solution_and_planted_violations(kw):
    """With general constraint maps: all five vanish at the certified QP solution; a multiplier of
    a z component strictly inside its box and a z component pushed past its bound are reported
    by their amounts; the stationarity residual is the reduced gradient (central differences)."""
    from oracle import oracle as O
    kw = dict(kw)
    seed = kw.pop("seed")
    p = D.constrained_boxed_problem(seed, **kw)
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    res = O.nama(o, lam, tol=1e-11, max_iter=5000)
    x, u, y, ok = D.active_set_qp(p, res["y"], thresh=1e-7)
    assert ok and np.count_nonzero(np.abs(y) > 1e-7) > 0
    r = KC.kkt_residuals(p, p.x0, x, u, y, tol_active=1e-8)
    scale = max(1.0, np.max(np.abs(y)), np.max(np.abs(x)))
    for k, v in r.items():
        assert v <= 1e-10 * scale, (k, v)
    h = o.stack(x, u)
    lo, hi = D.box_vectors(p)
    inside = np.nonzero((h < hi - 1e-3) & (h > lo + 1e-3))[0]
    y2 = y.copy()
    y2[int(inside[0])] = 0.04
    assert abs(KC.kkt_residuals(p, p.x0, x, u, y2, tol_active=1e-8)["complementarity"] - 0.04) <= 1e-14
    act = np.nonzero(np.abs(y) > 1e-6)[0]
    y3 = y.copy()
    y3[int(act[0])] = -y[int(act[0])]
    assert abs(KC.kkt_residuals(p, p.x0, x, u, y3, tol_active=1e-8)["sign"] - abs(y[int(act[0])])) <= 1e-12 * scale
    # stationarity at a rolled-out trajectory equals the reduced gradient of f + <y, Hx>
    rng = np.random.default_rng(seed)
    npl = p.tree.num_nonleaf
    uu = rng.standard_normal((npl, p.nu))
    yy = W.random_dual(p, seed + 1)
    xx = _rollout(p, uu)

    def lag(u_):
        xr = _rollout(p, u_)
        pr = p.tree.prob
        f = sum(pr[i] * (xr[i] @ (p.Q * xr[i]) + u_[i] @ (p.R * u_[i]) + p.q @ xr[i] + p.r @ u_[i]) for i in range(npl))
        f += sum(pr[l] * (xr[l] @ (p.PN * xr[l]) + p.pN @ xr[l]) for l in range(npl, p.tree.num_nodes))
        return f + yy @ o.stack(xr, u_)

    grad = np.zeros_like(uu)
    for i in range(npl):
        for a in range(p.nu):
            up, dn = uu.copy(), uu.copy()
            up[i, a] += 1e-3
            dn[i, a] -= 1e-3
            grad[i, a] = (lag(up) - lag(dn)) / 2e-3
    g = float(np.max(np.abs(grad)))
    assert abs(KC.kkt_residuals(p, p.x0, xx, uu, yy, tol_active=1e-8)["stationarity"] - g) <= 1e-8 * g


def test_gap_of_a_planted_interior_multiplier(solved):
    """A multiplier y_k < 0 on a component strictly inside its box adds y_k (lo_k - h_k) to the
    gap (the support function's lo y against y h); at the solution the gap is zero."""
    p, x, u, y = solved
    h = np.concatenate([np.concatenate([x[i], u[i]]) if i < p.tree.num_nonleaf else x[i]
                        for i in range(p.tree.num_nodes)])
    lo, hi = D.box_vectors(p)
    inside = np.nonzero((h < hi - 1e-3) & (h > lo + 1e-3))[0]
    inside = inside[inside >= p.nx]
    k = int(inside[0])
    y2 = y.copy()
    y2[k] = -0.0375
    base = KC.kkt_residuals(p, p.x0, x, u, y, tol_active=1e-8)["gap"]
    r = KC.kkt_residuals(p, p.x0, x, u, y2, tol_active=1e-8)
    assert abs(r["gap"] - base - 0.0375 * (h[k] - lo[k])) <= 1e-13


@pytest.mark.parametrize("soft", [False, True], ids=["box", "soft"])
def test_gap_is_primal_minus_dual_objective(soft):
    """At x = x(y) the gap equals the primal objective f(x) + g(Hx) minus the dual objective
    -fhat(y) - g*(y) of Section II-D, both taken from the oracle's solve step and its g, g*
    (a different route from the per-component formula); y is inside the conjugates' domains."""
    from oracle import oracle as O
    p = D.boxed_problem(17, horizon=4, nx=4, nu=2, frac=0.9)
    if soft:
        n = p.nx + p.nu
        W.with_penalty(p, np.array([1, 2] * (n // 2) + [0] * (n % 2)), 5.0 * np.ones(n), 0.4 * np.ones(n))
    o = O.LQOracle(p)
    rng = np.random.default_rng(11)
    for trial in range(3):
        y = 0.3 * W.random_dual(p, 20 + trial)
        x, u = o.solve(y)
        r = KC.kkt_residuals(p, p.x0, x, u, y, tol_active=1e-8)
        yb = y / o.sq
        h = o.hx(y)
        primal = o.cost(x, u) + (O.g_val(o, o.sq * h) if soft else 0.0)
        dual = -O.fhat(o, yb) - O.g_conj(o, yb)
        assert np.isfinite(dual)
        assert abs(r["gap"] - (primal - dual)) <= 1e-9 * max(1.0, abs(primal)), (trial, r["gap"], primal - dual)
        assert r["gap"] >= -1e-12
