"""Pins of the oracle's general separable g (Section II-B: hard box, soft constraint as
rho * distance to the box, l1 as its point-box case, Huber of the distance) against facts
other than the oracle:

* the proximal map against brute-force scalar minimisation (scipy);
* the conjugate against a brute-force supremum, and +inf off its domain;
* Moreau's identity against the conjugate's own closed-form proximal map;
* Fenchel-Young equality at the proximal point;
* the FBE definition (with g*) against the augmented-Lagrangian form (with g);
* solver results against optimality conditions written here: x = x(y) from a dense KKT solve
  and y in the subdifferential of g at Hx, plus zero duality gap;
* the exact-penalty theorem: with rho above the hard problem's largest multiplier the soft
  problem has the hard problem's solution.
"""
import numpy as np
import pytest
import scipy.optimize

from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W
from tests import dense_kkt as D


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


class _Elems:
    """A stand-in oracle holding per-element data only (what the prox functions read)."""

    def __init__(self, n, rng, kinds=(0, 1, 2)):
        self.m = n
        self.sq = rng.uniform(0.05, 1.0, n)
        c = rng.uniform(-1, 1, n)
        w = rng.uniform(0.0, 1.0, n)
        w[rng.random(n) < 0.2] = 0.0  # point boxes: l1 / Huber around c
        self.lo, self.hi = c - w, c + w
        self.kind = rng.choice(np.asarray(kinds, dtype=np.int32), n)
        self.rho = rng.uniform(0.2, 3.0, n)
        self.delta = rng.uniform(0.05, 1.0, n)


def _g1(kind, lo, hi, rho, delta, z):
    d = max(lo - z, 0.0) + max(z - hi, 0.0)
    if kind == 0:
        return 0.0 if d == 0.0 else np.inf
    if kind == 1:
        return rho * d
    return rho * (0.5 * d * d if d <= delta else delta * (d - 0.5 * delta))


def test_prox_against_brute_force():
    rng = np.random.default_rng(0)
    e = _Elems(300, rng)
    for lam in (0.05, 0.7, 5.0):
        v = rng.uniform(-4, 4, e.m)
        z = O.prox_g(e, v, lam)
        for k in range(e.m):
            s = e.sq[k]
            if e.kind[k] == 0:
                ref = s * np.clip(v[k] / s, e.lo[k], e.hi[k])
            else:
                f = lambda zb: _g1(e.kind[k], e.lo[k], e.hi[k], e.rho[k], e.delta[k], zb / s) + 0.5 * lam * (zb - v[k]) ** 2
                lo_b, hi_b = min(v[k], s * e.lo[k]) - 1.0, max(v[k], s * e.hi[k]) + 1.0
                ref = scipy.optimize.minimize_scalar(f, bounds=(lo_b, hi_b), method="bounded",
                                                     options={"xatol": 1e-12}).x
            assert abs(z[k] - ref) < 1e-7, (k, e.kind[k])


def test_conjugate_against_brute_force_supremum():
    rng = np.random.default_rng(1)
    e = _Elems(120, rng, kinds=(1, 2))
    grid = np.linspace(-60.0, 60.0, 120001)
    for k in range(e.m):
        s = e.sq[k]
        lim = e.rho[k] if e.kind[k] == 1 else e.rho[k] * e.delta[k]
        y = rng.uniform(-0.95, 0.95) * lim / s  # inside the domain of g~*
        one = _Elems(1, rng)
        for name in ("sq", "lo", "hi", "kind", "rho", "delta"):
            setattr(one, name, np.asarray([getattr(e, name)[k]]))
        pts = np.concatenate([grid, [e.lo[k], e.hi[k]]])   # the kinks of g
        val = lambda zz: s * y * zz - _g1(e.kind[k], e.lo[k], e.hi[k], e.rho[k], e.delta[k], zz)
        vals = np.array([val(zz) for zz in pts])
        j = int(np.argmax(vals))
        # g~*(y) = sup_z <y, s z> - g(z): best grid point or kink, refined between its neighbours
        ref = scipy.optimize.minimize_scalar(lambda zz: -val(zz), bounds=(pts[j] - 1e-3, pts[j] + 1e-3),
                                             method="bounded", options={"xatol": 1e-12})
        sup = max(vals[j], -ref.fun)
        assert abs(O.g_conj(one, np.asarray([y])) - sup) < 1e-6 * max(1.0, abs(sup)), k
        # off the domain: +inf
        assert O.g_conj(one, np.asarray([1.5 * lim / s])) == np.inf


@pytest.mark.parametrize("lam", [0.03, 0.8, 6.0])
def test_moreau_identity_against_conjugate_closed_form(lam):
    rng = np.random.default_rng(2)
    e = _Elems(2000, rng)
    v = rng.uniform(-5, 5, e.m)
    a = O.prox_g_conj(e, v, lam)           # v - lam z(v / lam), from the prox of g
    b = O.prox_g_conj_closed(e, v, lam)    # from the conjugates' closed forms
    assert np.max(np.abs(a - b)) < 1e-12 * max(1.0, np.max(np.abs(v)))


def test_fenchel_young_equality_at_the_prox():
    rng = np.random.default_rng(3)
    e = _Elems(500, rng)
    for lam in (0.1, 2.0):
        v = rng.uniform(-3, 3, e.m)
        z = O.prox_g(e, v, lam)
        y = lam * (v - z)                  # in the subdifferential of g~ at z
        lhs = O.g_val(e, z) + O.g_conj(e, y)
        assert abs(lhs - float(y @ z)) < 1e-10 * max(1.0, abs(lhs))


def _penalised(seed, kinds, rho, delta=0.2, **kw):
    p = D.boxed_problem(seed, **kw)
    return W.with_penalty(p, kinds, rho, delta)


# soft states / hard inputs; Huber states; l1 on the inputs around 0 (point box) with hard states
def _cases():
    a = _penalised(12, [1, 1, 1, 0, 0], 0.4, horizon=3, nx=3, nu=2)
    a.name = "soft-x"
    b = _penalised(17, [2, 2, 2, 2, 0, 0], 3.0, delta=0.1, horizon=4, nx=4, nu=2, frac=0.9)
    b.name = "huber-x"
    c = _penalised(12, [0, 0, 0, 1, 1], 0.3, horizon=3, nx=3, nu=2)
    c.ulo, c.uhi = np.zeros(2), np.zeros(2)
    c.name = "l1-u"
    return [a, b, c]


CASES = _cases()


@pytest.mark.parametrize("p", CASES, ids=lambda p: p.name)
def test_fbe_definition_with_general_g(p):
    o = O.LQOracle(p)
    rng = np.random.default_rng(4)
    for lam in (0.05, 0.3):
        for _ in range(3):
            yb = 0.3 * rng.standard_normal(o.m)
            yb[:p.nx] = 0.0
            pt = O.fb_point(o, yb, lam)
            lit = O.fbe_literal(o, yb, lam)
            assert np.isfinite(lit)
            assert abs(pt["phi"] - lit) < 1e-11 * max(1.0, abs(lit))


def _subgradient_residual(p, o, y, h):
    """max over elements of dist(y_k, subdifferential of g_k at (Hx)_k), from the definitions
    (y and h unscaled).  Kink points are recognised within 1e-7."""
    out = 0.0
    for k in range(o.m):
        if k < p.nx:
            out = max(out, abs(y[k]))  # root state: no term, multiplier zero
            continue
        lo, hi, kind, rho, dl, z = o.lo[k], o.hi[k], o.kind[k], o.rho[k], o.delta[k], h[k]
        tol = 1e-7
        if kind == 0:
            lo_s = -np.inf if abs(z - lo) <= tol else 0.0
            hi_s = np.inf if abs(z - hi) <= tol else 0.0
        elif kind == 1:
            if z > hi + tol:
                lo_s = hi_s = rho
            elif z < lo - tol:
                lo_s = hi_s = -rho
            else:
                lo_s = -rho if abs(z - lo) <= tol else 0.0
                hi_s = rho if abs(z - hi) <= tol else 0.0
        else:
            d = max(lo - z, 0.0) + max(z - hi, 0.0)
            gd = rho * min(d, dl)
            lo_s = hi_s = gd if z > hi else (-gd if z < lo else 0.0)
        out = max(out, max(lo_s - y[k], y[k] - hi_s, 0.0))
    return out


@pytest.mark.parametrize("solver", ["nama", "minfbe", "gpad"])
@pytest.mark.parametrize("p", CASES, ids=lambda p: p.name)
def test_solvers_satisfy_optimality_with_general_g(p, solver):
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    fn = {"nama": O.nama, "minfbe": O.minfbe, "gpad": O.gpad}[solver]
    kw = dict(max_iter=200000) if solver == "gpad" else dict(max_iter=2000)
    res = fn(o, lam, tol=1e-10, **kw)
    assert res["status"] == "converged"
    y = res["y"]
    xd, ud = D.dense_solve(p, y)
    assert _rel(res["x"], xd) < 1e-8 and _rel(res["u"], ud) < 1e-8
    h = o.stack(xd, ud)
    assert _subgradient_residual(p, o, y, h) < 1e-6
    # zero duality gap: f(x) + g(Hx) = -(fhat(y) + g*(y))
    yb = res["ybar"]
    zb = O.prox_g(o, o.sq * h, 1e12)  # Hx itself where g is finite; projected for hard boxes
    primal = o.cost(xd, ud) + O.g_val(o, zb)
    dual = O.fhat(o, yb) + O.g_conj(o, yb)
    assert abs(primal + dual) < 1e-6 * max(1.0, abs(primal))
    if solver != "gpad":
        phis = np.array(res["phi"])
        assert np.all(np.diff(phis) <= 1e-12 * np.maximum(1.0, np.abs(phis[:-1])))


def test_exact_penalty_recovers_the_hard_solution():
    """Soft constraints rho dist(., box) with rho above the hard problem's largest multiplier
    (unscaled) have the hard problem's solution."""
    hard = D.boxed_problem(12, horizon=3, nx=3, nu=2)
    oh = O.LQOracle(hard)
    lam, _ = O.power_lambda(oh, np.random.default_rng(0).standard_normal(oh.m))
    rh = O.nama(oh, lam, tol=1e-11)
    ymax = float(np.max(np.abs(rh["y"])))
    assert ymax > 1e-3
    soft = W.with_penalty(D.boxed_problem(12, horizon=3, nx=3, nu=2), 1, 2.0 * ymax)
    os_ = O.LQOracle(soft)
    rs = O.nama(os_, lam, tol=1e-11, max_iter=5000)
    assert rs["status"] == "converged"
    assert _rel(rs["x"], rh["x"]) < 1e-7 and _rel(rs["u"], rh["u"]) < 1e-7
    # and below it the soft solution violates the box
    weak = W.with_penalty(D.boxed_problem(12, horizon=3, nx=3, nu=2), 1, 0.25 * ymax)
    ow = O.LQOracle(weak)
    rw = O.nama(ow, lam, tol=1e-11, max_iter=5000)
    hw = ow.stack(rw["x"], rw["u"])
    viol = np.max(np.maximum(ow.lo - hw, 0) + np.maximum(hw - ow.hi, 0))
    assert viol > 1e-4
