"""Pins of the oracle's GPAD (accelerated dual projected gradient; Section III-F warm start,
Section IV comparison method) against things other than itself:

* the theta sequence against hand-computed values and the identity that defines Nesterov's
  sequence, (1 - theta_{k+1}) / theta_{k+1}^2 = 1 / theta_k^2;
* the iterates against FISTA (Beck and Teboulle 2009, the t_k form) written here on the dense
  dual, with x(y) from one dense KKT solve and the two-sided shrink as the prox: equal after
  every number of steps, which fixes the extrapolation coefficient and the step;
* the limit against the exact active-set QP solution with certified KKT signs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W
from tests import dense_kkt as D


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


def test_theta_sequence_hand_values():
    th = [O.gpad_theta(k) for k in range(8)]
    assert th[0] == 1.0
    assert abs(th[1] - (np.sqrt(5.0) - 1.0) / 2.0) < 1e-15
    # theta_2 by hand: (sqrt(theta_1^4 + 4 theta_1^2) - theta_1^2) / 2 with theta_1^2 = (3 - sqrt 5)/2
    t1s = (3.0 - np.sqrt(5.0)) / 2.0
    assert abs(th[2] - 0.5 * (np.sqrt(t1s * t1s + 4.0 * t1s) - t1s)) < 1e-15
    assert abs(th[2] - 1.0 / 2.1935271) < 1e-7  # 1 / t_3 of the Beck-Teboulle sequence
    # the first extrapolation coefficients: 0, 0, then 0.28175...
    coef = [th[k] * (1.0 / (th[k - 1] if k > 0 else 1.0) - 1.0) for k in range(4)]
    assert coef[0] == 0.0 and abs(coef[1]) < 1e-15 and abs(coef[2] - 0.2817535) < 1e-7
    for k in range(1, 8):
        assert abs((1.0 - th[k]) / th[k] ** 2 - 1.0 / th[k - 1] ** 2) < 1e-12
        assert th[k] <= 2.0 / (k + 2) + 1e-15


def _dense_dual(p):
    """Scaled-dual forward-backward map built from the dense KKT solve (no tree recursion)."""
    t = p.tree
    off = W.dual_offsets(t, p.nx, p.nu)
    m = int(off[-1])
    sq = np.empty(m)
    for i in range(t.num_nodes):
        sq[off[i]:off[i + 1]] = np.sqrt(t.prob[i])
    Hm, const = D.h_rows(p)
    lo, hi = D.box_vectors(p)
    _, _, nv = D._index(p)

    def hx(y):
        G, g, E, e = D.build_qp(p, y)
        K = np.block([[G, E.T], [E, np.zeros((E.shape[0], E.shape[0]))]])
        v = np.linalg.solve(K, np.concatenate([-g, e]))[:nv]
        return Hm @ v + const

    def T(w, lam):
        v = w + lam * sq * hx(sq * w)
        # prox of lam * (support function of the scaled box): two-sided shrink
        out = np.zeros_like(v)
        up, dn = v > lam * sq * hi, v < lam * sq * lo
        out[up] = v[up] - lam * (sq * hi)[up]
        out[dn] = v[dn] - lam * (sq * lo)[dn]
        return out

    return T, sq


@pytest.mark.parametrize("seed", [12, 13])
def test_gpad_iterates_equal_dense_fista(seed):
    p = D.boxed_problem(seed, horizon=3, nx=3, nu=2)
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    T, sq = _dense_dual(p)
    y0 = 0.3 * np.random.default_rng(seed).standard_normal(o.m)
    y0[:p.nx] = 0.0
    # FISTA, Beck-Teboulle form: y_1 = x_0, t_1 = 1, x_k = T(y_k),
    # y_{k+1} = x_k + (t_k - 1)/t_{k+1} (x_k - x_{k-1})
    x_prev = y0 / sq
    yk, tk = x_prev.copy(), 1.0
    for K in range(1, 26):
        xk = T(yk, lam)
        t_next = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
        yk = xk + ((tk - 1.0) / t_next) * (xk - x_prev)
        x_prev, tk = xk, t_next
        if K in (1, 2, 3, 7, 25):
            res = O.gpad(o, lam, y0=y0, tol=0.0, max_iter=K)
            assert res["iters"] == K and res["status"] == "not_converged"
            assert _rel(res["ybar"], yk) < 1e-11, K


@pytest.mark.parametrize("seed", [12, 13])
def test_gpad_reaches_certified_qp_solution(seed):
    p = D.boxed_problem(seed, horizon=3, nx=3, nu=2)
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    res = O.gpad(o, lam, tol=1e-9, max_iter=50000)
    assert res["status"] == "converged" and res["res_inf"] <= 1e-9
    x, u, y, ok = D.active_set_qp(p, res["y"], thresh=1e-5)
    assert ok
    assert _rel(res["x"], x) < 1e-7
    assert _rel(res["u"], u) < 1e-7
    # the same solution as Algorithm 2
    nm = O.nama(o, lam, tol=1e-10)
    assert _rel(res["x"], nm["x"]) < 1e-7


def test_gpad_zero_iterations_is_the_start_point():
    p = D.boxed_problem(12, horizon=3, nx=3, nu=2)
    o = O.LQOracle(p)
    res = O.gpad(o, 0.1, tol=0.0, max_iter=0)
    assert res["iters"] == 0 and np.all(res["ybar"] == 0.0) and o.solve_calls == 1
    x, u = D.dense_solve(p, np.zeros(o.m))
    assert _rel(res["x"], x) < 1e-10
