"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to an independent fact: a dense KKT solve
(numpy.linalg), the discrete algebraic Riccati equation (scipy), exact finite
differences of a quadratic, the Moreau identity and a brute-force prox, the dense
BFGS update, an exact active-set QP solution with certified KKT signs, and an
independent accelerated dual projected-gradient run.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from paper_2107_01745_b300 import workloads as W
from oracle import oracle as O
from tests import dense_kkt as D

PROBLEMS = [W.tiny_fp64(0)] + [W.random_problem(s, horizon=h, nx=nx, nu=nu)
                               for s, h, nx, nu in [(1, 3, 3, 2), (2, 4, 2, 1), (3, 3, 5, 3), (4, 2, 1, 1)]]


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("p", PROBLEMS, ids=lambda p: p.name)
@pytest.mark.parametrize("homogeneous", [False, True])
def test_solve_matches_dense_kkt(p, homogeneous):
    """Algorithm 3/4 with the derived factor equals the dense KKT solution (Section III-D)."""
    o = O.LQOracle(p)
    y = W.random_dual(p, 11, scale=2.0)
    x, u = o.solve(y, homogeneous)
    xd, ud = D.dense_solve(p, y, homogeneous)
    assert _rel(x, xd) < 1e-10
    assert _rel(u, ud) < 1e-10


def test_chain_gain_matches_dare():
    """A one-child-per-node chain is a finite-horizon LQR; far from the leaves its gain is
    the infinite-horizon gain from scipy's discrete algebraic Riccati solver."""
    rng = np.random.default_rng(5)
    nx, nu, horizon = 4, 2, 250
    A0 = W.spectral_rescale(rng.standard_normal((nx, nx)), 1.2)
    B0 = rng.standard_normal((nx, nu))
    Qd = rng.uniform(0.5, 2.0, nx)
    Rd = rng.uniform(0.1, 1.0, nu)
    tree = W.tree_from_branching([1] * horizon)
    nn = tree.num_nodes
    A = np.broadcast_to(A0, (nn, nx, nx)).copy()
    B = np.broadcast_to(B0, (nn, nx, nu)).copy()
    p = W.Problem(tree=tree, nx=nx, nu=nu, A=A, B=B, c=np.zeros((nn, nx)), Q=Qd, R=Rd,
                  PN=np.ones(nx), q=np.zeros(nx), r=np.zeros(nu), pN=np.zeros(nx),
                  xlo=-np.ones(nx), xhi=np.ones(nx), ulo=-np.ones(nu), uhi=np.ones(nu),
                  x0=np.zeros(nx))
    o = O.LQOracle(p)
    P = scipy.linalg.solve_discrete_are(A0, B0, np.diag(Qd), np.diag(Rd))
    Kd = -np.linalg.solve(np.diag(Rd) + B0.T @ P @ B0, B0.T @ P @ A0)
    assert _rel(o.P[0], P) < 1e-9
    assert _rel(o.K[0], Kd) < 1e-9


@pytest.mark.parametrize("p", PROBLEMS[:3], ids=lambda p: p.name)
def test_affine_in_y(p):
    """x(y + tau d) - x(y) = tau x_lin(d): the dual-gradient map is affine and Algorithm 4
    is its linear part.  The literal x(y) + tau x(d) is wrong whenever c, q, r or p are nonzero."""
    o = O.LQOracle(p)
    y, d = W.random_dual(p, 1), W.random_dual(p, 2)
    tau = 0.37
    h0, hy, hd = o.hx(y + tau * d), o.hx(y), o.hx(d, homogeneous=True)
    assert _rel(h0 - hy, tau * hd) < 1e-12
    assert _rel(h0, hy + tau * o.hx(d)) > 1e-6


@pytest.mark.parametrize("p", PROBLEMS, ids=lambda p: p.name)
def test_grad_fhat_by_central_differences(p):
    """grad fhat(ybar) = -Hbar x(ybar): fhat is quadratic so central differences are exact."""
    o = O.LQOracle(p)
    yb = W.random_dual(p, 3)
    h, _, _ = O.hbar(o, yb)
    rng = np.random.default_rng(4)
    for _ in range(3):
        d = rng.standard_normal(o.m)
        eps = 1e-2
        fd = (O.fhat(o, yb + eps * d) - O.fhat(o, yb - eps * d)) / (2 * eps)
        assert abs(fd - (-np.dot(h, d))) < 1e-9 * max(1.0, abs(fd))


@pytest.mark.parametrize("p", PROBLEMS[:3], ids=lambda p: p.name)
def test_hessian_symmetric_psd_and_dense(p):
    """grad^2 fhat = -Hbar x_lin(.) is symmetric PSD and equals H dX/dy from the dense KKT."""
    o = O.LQOracle(p)
    Hs = np.stack([-O.hbar_lin(o, e) for e in np.eye(o.m)], axis=1)
    assert np.max(np.abs(Hs - Hs.T)) < 1e-12 * max(1.0, np.max(np.abs(Hs)))
    assert np.min(np.linalg.eigvalsh(0.5 * (Hs + Hs.T))) > -1e-12 * np.max(np.abs(Hs))
    cols = []
    for e in np.eye(o.m):
        x, u = D.dense_solve(p, o.sq * e, homogeneous=True)
        cols.append(-o.sq * o.stack(x, u))
    assert _rel(Hs, np.stack(cols, axis=1)) < 1e-10


@pytest.mark.parametrize("p_branch", [0.6, 1.0])
def test_prox_moreau_and_brute_force(p_branch):
    """prox_{lam g*} via Moreau equals the two-sided shrink and a scalar brute-force minimisation.
    The box is the preconditioned S Y (Section III-E); with p_branch = 1 every node branches, so
    sqrt(pi) < 1 below the root and a projection on the unscaled Y fails the identity."""
    p = W.random_problem(7, box_scale=0.5, p_branch=p_branch)
    o = O.LQOracle(p)
    if p_branch == 1.0:
        assert np.min(o.sq) < 0.75
    lam = 0.7
    rng = np.random.default_rng(8)
    v = 3.0 * rng.standard_normal(o.m)
    a = O.prox_g_conj(o, v, lam)
    b = O.prox_g_conj_closed(o, v, lam)
    assert np.max(np.abs(a - b)) < 1e-14
    # Moreau: prox_{lam g*}(v) + lam prox_{g/lam}(v/lam) = v
    assert np.max(np.abs(a + lam * O.proj_box(o, v / lam) - v)) < 1e-14
    lo, hi = o.sq * o.lo, o.sq * o.hi
    for k in rng.choice(np.arange(p.nx, o.m), size=12, replace=False):
        obj = lambda zz: max(lo[k] * zz, hi[k] * zz) + (zz - v[k]) ** 2 / (2 * lam)
        res = scipy.optimize.minimize_scalar(obj, bounds=(v[k] - 20, v[k] + 20), method="bounded",
                                             options={"xatol": 1e-12})
        assert abs(res.x - a[k]) < 1e-6


@pytest.mark.parametrize("p", PROBLEMS[:3], ids=lambda p: p.name)
def test_fbe_definition_vs_augmented_lagrangian(p):
    """The FBE of Section III-A equals -[f(x) + <y, Hx - z> + lam/2 ||Hx - z||^2]."""
    o = O.LQOracle(p)
    lam = 0.3
    for seed in range(3):
        yb = W.random_dual(p, 20 + seed)
        a = O.fbe_literal(o, yb, lam)
        b = O.fb_point(o, yb, lam)["phi"]
        assert abs(a - b) < 1e-12 * max(1.0, abs(a))


@pytest.mark.parametrize("p", PROBLEMS[:3], ids=lambda p: p.name)
def test_fbe_below_dual_objective(p):
    """phi_lam(y) <= fhat(y) + g*(y) for lam < 1/L, with equality at a dual solution."""
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m), iters=300)
    for seed in range(4):
        yb = W.random_dual(p, 30 + seed)
        assert O.fb_point(o, yb, lam)["phi"] <= O.fhat(o, yb) + O.g_conj(o, yb) + 1e-12
    res = O.nama(o, lam, tol=1e-11)
    yb = res["ybar"]
    dual_obj = O.fhat(o, yb) + O.g_conj(o, yb)
    assert abs(O.fb_point(o, yb, lam)["phi"] - dual_obj) < 1e-8 * max(1.0, abs(dual_obj))


@pytest.mark.parametrize("p", PROBLEMS[:3], ids=lambda p: p.name)
def test_fbe_gradient_by_central_differences(p):
    """grad phi = (I - lam grad^2 fhat) R, checked by central differences away from kinks."""
    o = O.LQOracle(p)
    lam = 0.2
    yb = W.random_dual(p, 40)
    g = O.fbe_grad(o, yb, lam)
    rng = np.random.default_rng(41)
    pt = O.fb_point(o, yb, lam)
    v = pt["h"] + yb / lam
    gap = np.minimum(np.abs(v - o.sq * o.lo), np.abs(v - o.sq * o.hi))
    assert np.min(gap) > 1e-4, "test point too close to a kink"
    for _ in range(3):
        d = rng.standard_normal(o.m)
        eps = 1e-7
        fd = (O.fb_point(o, yb + eps * d, lam)["phi"] - O.fb_point(o, yb - eps * d, lam)["phi"]) / (2 * eps)
        assert abs(fd - np.dot(g, d)) < 1e-6 * max(1.0, abs(fd))


def test_lbfgs_two_loop_equals_dense_bfgs():
    """The two-loop recursion applies the dense BFGS inverse update started from gamma I."""
    rng = np.random.default_rng(9)
    n, mem = 12, 5
    M = rng.standard_normal((n, n))
    Hq = M @ M.T + n * np.eye(n)
    lb = O.LBFGS(mem, lam=0.5)
    pairs = []
    for _ in range(8):
        s = rng.standard_normal(n)
        q = Hq @ s
        lb.push(s, q)
        pairs.append((s, q))
    pairs = pairs[-mem:]
    s_new, q_new = pairs[-1]
    Hinv = (np.dot(s_new, q_new) / np.dot(q_new, q_new)) * np.eye(n)
    for s, q in pairs:
        rho = 1.0 / np.dot(s, q)
        V = np.eye(n) - rho * np.outer(q, s)
        Hinv = V.T @ Hinv @ V + rho * np.outer(s, s)
    g = rng.standard_normal(n)
    assert np.max(np.abs(lb.apply(g) - Hinv @ g)) < 1e-12 * np.max(np.abs(Hinv @ g))
    assert np.allclose(O.LBFGS(mem, lam=0.5).apply(g), 0.5 * g)


@pytest.mark.parametrize("p", PROBLEMS[:3], ids=lambda p: p.name)
def test_power_iteration_lambda(p):
    """Power iteration's L estimate approaches the largest eigenvalue of grad^2 fhat."""
    o = O.LQOracle(p)
    Hs = np.stack([-O.hbar_lin(o, e) for e in np.eye(o.m)], axis=1)
    Lmax = np.max(np.linalg.eigvalsh(0.5 * (Hs + Hs.T)))
    lam, L = O.power_lambda(o, np.random.default_rng(1).standard_normal(o.m), iters=400)
    assert L <= Lmax * (1 + 1e-12)
    assert L > Lmax * (1 - 1e-6)
    assert abs(lam - 0.9 / L) < 1e-15


BOXED = [D.boxed_problem(s, horizon=3, nx=3, nu=2) for s in (12, 13)] + [W.tiny_fp64(0)]


@pytest.mark.parametrize("solver", ["nama", "minfbe"])
@pytest.mark.parametrize("p", BOXED, ids=lambda p: p.name)
def test_solver_reaches_certified_qp_solution(solver, p):
    """Algorithms 1 and 2 stop at ||z - Hx||_inf <= eps; their primal agrees with the exact
    active-set QP solution, whose KKT signs are certified independently."""
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    fn = O.nama if solver == "nama" else O.minfbe
    res = fn(o, lam, tol=1e-10, max_iter=500)
    assert res["status"] == "converged"
    assert res["res_inf"] <= 1e-10
    x, u, y, ok = D.active_set_qp(p, res["y"], thresh=1e-6)
    assert ok, "active set read from the solver's dual does not certify"
    assert _rel(res["x"], x) < 1e-8
    assert _rel(res["u"], u) < 1e-8
    assert _rel(res["y"], y) < 1e-6
    if np.any(np.abs(y) > 1e-6):
        assert solver and res["iters"] > 0
    # phi is monotone along the iterates (descent line search plus an FB step)
    phis = np.array(res["phi"])
    assert np.all(np.diff(phis) <= 1e-12 * np.maximum(1.0, np.abs(phis[:-1])))
    # duality gap: f(x*) = -(fhat(y*) + g*(y*))
    yb = res["ybar"]
    dual_val = O.fhat(o, yb) + O.g_conj(o, yb)
    primal_val = o.cost(res["x"], res["u"])
    assert abs(primal_val + dual_val) < 1e-7 * max(1.0, abs(primal_val))


@pytest.mark.parametrize("p", BOXED[:1] + [D.boxed_problem(s, horizon=4, nx=3, nu=2) for s in (19, 26)],
                         ids=lambda p: p.name)
def test_nama_line_search_reaches_the_forward_backward_step(p):
    """Algorithm 2's trial point w(tau) = ybar + tau d + (1 - tau)(T(ybar) - ybar) tends to the
    forward-backward step T(ybar) as tau -> 0, and for lam < 1/L that step lowers the FBE by
    at least (1 - lam L) lam / 2 ||R||^2 (Section III-A).  So while the residual is far from
    zero some halving is accepted and the tau = 0 fallback is never used; reading the
    extrapolation literally as ybar + tau d + (1 - tau) R makes the small trials approach
    ybar + R instead, where the test can fail at every halving."""
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    res = O.nama(o, lam, tol=1e-10, max_iter=500)
    assert res["status"] == "converged"
    taus, before = np.array(res["tau"]), np.array(res["res"][:-1])
    assert np.any(taus < 1.0), "the line search never halves on this problem: no evidence"
    assert not np.any((taus == 0.0) & (before > 1e-6))


def test_loose_box_stops_at_iteration_zero():
    """With a box that never binds, y* = 0 and both methods return x(0) without iterating."""
    p = W.random_problem(14, box_scale=1e6)
    o = O.LQOracle(p)
    for fn in (O.nama, O.minfbe):
        res = fn(o, 0.1, tol=1e-12)
        assert res["iters"] == 0 and res["res_inf"] == 0.0
        x, u = D.dense_solve(p, np.zeros(o.m))
        assert _rel(res["x"], x) < 1e-10


def _gpad(o, lam, iters):
    """Accelerated dual projected gradient (FISTA on the dual), independent of Algorithms 1-2."""
    y = np.zeros(o.m)
    w = y.copy()
    t = 1.0
    for _ in range(iters):
        h, _, _ = O.hbar(o, w)
        y_new = O.prox_g_conj(o, w + lam * h, lam)
        t_new = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        w = y_new + ((t - 1) / t_new) * (y_new - y)
        y, t = y_new, t_new
    return y


def test_nama_minfbe_and_gpad_agree_on_tiny():
    """On the tiny FP64 workload, MINFBE, NAMA and a long GPAD run agree."""
    p = BOXED[0]
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    a = O.nama(o, lam, tol=1e-10)
    b = O.minfbe(o, lam, tol=1e-10)
    yg = _gpad(o, lam, 6000)
    hg, xg, ug = O.hbar(o, yg)
    assert _rel(a["x"], b["x"]) < 1e-8
    assert _rel(a["x"], xg) < 1e-6
    assert _rel(a["y"], o.sq * yg) < 1e-5
