"""Pins of the oracle's step-size backtracking (Section III-B, eqs. original-backtracking and
simple-backtracking) against facts other than the oracle:

* L = ||grad^2 fhat|| of the preconditioned dual is taken from the dense KKT solve (no tree
  recursion), as the largest eigenvalue of the dense Hessian;
* the descent lemma: with lambda <= (1 - beta)/L the original test never fails, so no halving;
  from a lambda far above, halving stops at some lambda >= (1 - beta)/(2L);
* Lipschitz continuity: with lambda L <= eps'' the simple test never fails; from above,
  halving stops at some lambda >= eps''/(2L);
* the test as evaluated (second-order expansion with a Hessian-vector product) equals the
  literal test from fhat values wherever its margin is well above rounding;
* both methods still reach the exact active-set QP solution with certified KKT signs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W
from tests import dense_kkt as D

# problems whose box binds at y = 0 (residual of order 0.1 or more there)
BOXED = [D.boxed_problem(12, horizon=3, nx=3, nu=2), D.boxed_problem(17, horizon=4, nx=4, nu=2, frac=0.9),
         D.boxed_problem(16, horizon=3, nx=5, nu=3, frac=0.9)]


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


def _dense_L(p):
    """Largest eigenvalue of grad^2 fhat(ybar) = S H (dx/dy) S from the dense KKT solve."""
    t = p.tree
    off = W.dual_offsets(t, p.nx, p.nu)
    m = int(off[-1])
    sq = np.empty(m)
    for i in range(t.num_nodes):
        sq[off[i]:off[i + 1]] = np.sqrt(t.prob[i])
    Hm, _ = D.h_rows(p)
    _, _, nv = D._index(p)
    cols = []
    for e in np.eye(m):
        G, g, E, ee = D.build_qp(p, sq * e, homogeneous=True)
        K = np.block([[G, E.T], [E, np.zeros((E.shape[0], E.shape[0]))]])
        v = np.linalg.solve(K, np.concatenate([-g, ee]))[:nv]
        cols.append(-sq * (Hm @ v))
    Hs = np.stack(cols, axis=1)
    return float(np.max(np.linalg.eigvalsh(0.5 * (Hs + Hs.T))))


@pytest.fixture(scope="module", params=range(len(BOXED)), ids=lambda i: f"{BOXED[i].name}-nx{BOXED[i].nx}")
def case(request):
    p = BOXED[request.param]
    o = O.LQOracle(p)
    assert O.fb_point(o, np.zeros(o.m), 0.1)["res_inf"] > 0.1
    return p, o, _dense_L(p)


def _certified(p, res):
    x, u, y, ok = D.active_set_qp(p, res["y"], thresh=1e-6)
    assert ok
    assert _rel(res["x"], x) < 1e-8 and _rel(res["u"], u) < 1e-8


@pytest.mark.parametrize("method", ["nama", "minfbe"])
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_original_never_halves_below_one_over_L(case, method, beta):
    p, o, L = case
    fn = O.nama if method == "nama" else O.minfbe
    res = fn(o, (1.0 - beta) / L * (1 - 1e-9), tol=1e-10, backtrack="original", bt_beta=beta)
    assert res["status"] == "converged" and res["halvings"] == 0


@pytest.mark.parametrize("method", ["nama", "minfbe"])
def test_original_from_large_lambda(case, method):
    p, o, L = case
    beta = 0.1
    lam0 = 1e4 / L
    fn = O.nama if method == "nama" else O.minfbe
    res = fn(o, lam0, tol=1e-10, max_iter=2000, backtrack="original", bt_beta=beta)
    assert res["status"] == "converged"
    assert res["halvings"] >= 1
    # halving stops for good once lambda <= (1 - beta)/L; it may stop above (the test sees
    # only the curvature along R(w))
    assert (1.0 - beta) / (2.0 * L) * (1 - 1e-12) <= res["lam"] <= lam0 / 2
    assert res["lam"] == lam0 * 0.5 ** res["halvings"]
    _certified(p, res)


@pytest.mark.parametrize("method", ["nama", "minfbe"])
def test_simple_never_halves_below_eps_over_L(case, method):
    p, o, L = case
    eps = 0.25
    fn = O.nama if method == "nama" else O.minfbe
    res = fn(o, eps / L * (1 - 1e-9), tol=1e-10, backtrack="simple", bt_eps=eps)
    assert res["status"] == "converged" and res["halvings"] == 0


@pytest.mark.parametrize("method", ["nama", "minfbe"])
def test_simple_from_large_lambda(case, method):
    p, o, L = case
    eps = 0.25
    lam0 = 1e4 / L
    fn = O.nama if method == "nama" else O.minfbe
    res = fn(o, lam0, tol=1e-10, max_iter=2000, backtrack="simple", bt_eps=eps)
    assert res["status"] == "converged"
    assert res["halvings"] >= 1
    assert eps / (2.0 * L) * (1 - 1e-12) <= res["lam"] <= lam0 / 2
    _certified(p, res)


@pytest.mark.parametrize("scale", [0.3, 0.9, 1.5, 4.0])
def test_original_test_matches_literal_fhat_values(case, scale):
    """Far from the solution the literal eq. (original-backtracking) from fhat values and the
    exact expansion agree: excess = lam/2 (lam <R, grad^2 fhat R> - (1 - beta) ||R||^2)."""
    p, o, L = case
    lam, beta = scale / L, 0.2
    rng = np.random.default_rng(5)
    for _ in range(4):
        w = rng.standard_normal(o.m)
        w[:p.nx] = 0.0
        wp = O.fb_point(o, w, lam)
        new = O.fb_point(o, wp["T"], lam)
        lit = O.original_backtrack_excess(o, wp, new, lam, beta)
        R = wp["r"]
        HR = -O.hbar_lin(o, R)
        quad = 0.5 * lam * (lam * float(R @ HR) - (1.0 - beta) * float(R @ R))
        assert abs(lit - quad) <= 1e-9 * max(abs(quad), float(R @ R) * lam)
        assert O.original_backtrack_fails(o, wp, new, lam, beta) == (lit > 0)
    assert (scale <= 0.8) <= (not O.original_backtrack_fails(o, wp, new, lam, beta))


def test_bad_backtracking_arguments_rejected():
    o = O.LQOracle(BOXED[0])
    for kw in (dict(backtrack="armijo"), dict(backtrack="simple", bt_eps=0.5),
               dict(backtrack="original", bt_beta=1.0)):
        with pytest.raises(ValueError):
            O.nama(o, 0.1, **kw)
