"""Pins of the oracle with general constraint maps z^i = F x^i + G u^i, z^l = FN x^l (Section II-C),
shared by all nodes, with a box on z (CPU).

Checked against facts outside the oracle's recursion: one dense KKT solve of the whole tree
problem with the term <y, Hx> built from the rows of H (tests/dense_kkt.py), the selection maps
F = [I; 0], G = [0; I], FN = I reproducing the selection problem, the dual Hessian symmetric,
PSD and equal to the dense Jacobian, exact central differences of fhat, the FBE definition
against its augmented-Lagrangian form, and NAMA, MINFBE and GPAD reaching the exact solution of
the constrained QP, whose active set is certified by its KKT signs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W
from tests import dense_kkt as D

SHAPES = [dict(seed=81, horizon=3, nx=3, nu=2, nc=4, ncN=2), dict(seed=85, horizon=4, nx=4, nu=2, nc=3, ncN=4),
          dict(seed=87, horizon=3, nx=2, nu=3, nc=7, ncN=1, max_branch=4)]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


def _problem(kw, boxed=True):
    kw = dict(kw)
    seed = kw.pop("seed")
    return D.constrained_boxed_problem(seed, **kw) if boxed else W.constrained_problem(seed, **kw)


@pytest.mark.parametrize("homogeneous", [False, True])
@pytest.mark.parametrize("kw", SHAPES, ids=lambda k: f"nc{k['nc']}")
def test_solve_matches_dense_kkt(kw, homogeneous):
    p = _problem(kw, boxed=False)
    o = O.LQOracle(p)
    assert o.m == p.num_dual and o.m != o.sel_m
    for seed in (1, 2):
        y = W.random_dual(p, seed)
        x, u = o.solve(y, homogeneous=homogeneous)
        xd, ud = D.dense_solve(p, y, homogeneous=homogeneous)
        assert _rel(x, xd) < 1e-11 and _rel(u, ud) < 1e-11
        Hm, const = D.h_rows(p)
        from tests.dense_kkt import _index
        uoff, xoff, nv = _index(p)
        v = np.zeros(nv)
        for i in range(p.tree.num_nonleaf):
            v[uoff[i]:uoff[i] + p.nu] = ud[i]
        for j in range(1, p.tree.num_nodes):
            v[xoff[j]:xoff[j] + p.nx] = xd[j]
        h_dense = Hm @ v + (0.0 if homogeneous else 1.0) * const
        assert _rel(o.hx(y, homogeneous=homogeneous), h_dense) < 1e-11


def test_selection_maps_reproduce_the_selection_problem():
    p = W.random_problem(84, horizon=3, nx=3, nu=2)
    g = W.random_problem(84, horizon=3, nx=3, nu=2)
    nx, nu = p.nx, p.nu
    F = np.vstack([np.eye(nx), np.zeros((nu, nx))])
    G = np.vstack([np.zeros((nx, nu)), np.eye(nu)])
    W.with_constraints(g, F, G, np.eye(nx), np.concatenate([p.xlo, p.ulo]), np.concatenate([p.xhi, p.uhi]),
                       p.xlo, p.xhi)
    o, og = O.LQOracle(p), O.LQOracle(g)
    assert og.m == o.m
    y = W.random_dual(p, 5)  # zero on the root's state block
    assert _rel(og.hx(y), o.hx(y)) < 1e-13
    # the general maps box the root's block too; the selection leaves its state free
    assert np.all(np.isfinite(og.lo[:nx])) and np.all(np.isinf(o.lo[:nx]))


@pytest.mark.parametrize("kw", SHAPES, ids=lambda k: f"nc{k['nc']}")
def test_hessian_symmetric_psd_and_dense(kw):
    p = _problem(kw, boxed=False)
    o = O.LQOracle(p)
    Hs = np.stack([-O.hbar_lin(o, e) for e in np.eye(o.m)], axis=1)
    assert np.max(np.abs(Hs - Hs.T)) <= 1e-10 * np.max(np.abs(Hs))
    assert np.min(np.linalg.eigvalsh(0.5 * (Hs + Hs.T))) >= -1e-10 * np.max(np.abs(Hs))
    cols = []
    for e in np.eye(o.m):
        x, u = D.dense_solve(p, o.sq * e, homogeneous=True)
        cols.append(-o.sq * o.stack(x, u))
    assert _rel(Hs, np.stack(cols, axis=1)) < 1e-10


@pytest.mark.parametrize("kw", SHAPES[:2], ids=lambda k: f"nc{k['nc']}")
def test_grad_fhat_by_central_differences(kw):
    p = _problem(kw, boxed=False)
    o = O.LQOracle(p)
    rng = np.random.default_rng(3)
    yb = rng.standard_normal(o.m)
    h, _, _ = O.hbar(o, yb)
    step = 1e-3
    fd = np.array([(O.fhat(o, yb + step * e) - O.fhat(o, yb - step * e)) / (2 * step) for e in np.eye(o.m)])
    assert _rel(fd, -h) < 1e-8


@pytest.mark.parametrize("kw", SHAPES, ids=lambda k: f"nc{k['nc']}")
def test_fbe_definition_vs_augmented_lagrangian(kw):
    p = _problem(kw)
    o = O.LQOracle(p)
    rng = np.random.default_rng(4)
    for lam in (0.05, 0.3):
        yb = rng.standard_normal(o.m)
        pt = O.fb_point(o, yb, lam)
        lit = O.fbe_literal(o, yb, lam)
        assert abs(pt["phi"] - lit) <= 1e-11 * max(1.0, abs(lit))


@pytest.mark.parametrize("solver", ["nama", "minfbe", "gpad"])
@pytest.mark.parametrize("kw", SHAPES, ids=lambda k: f"nc{k['nc']}")
def test_solvers_reach_certified_qp_solution(kw, solver):
    p = _problem(kw)
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    fn = {"nama": O.nama, "minfbe": O.minfbe, "gpad": O.gpad}[solver]
    res = fn(o, lam, tol=1e-10, max_iter=50000)
    assert res["status"] == "converged" and res["res_inf"] <= 1e-10
    x, u, y, ok = D.active_set_qp(p, res["y"], thresh=1e-6)
    assert ok, "active set read from the solver's dual does not certify"
    assert np.count_nonzero(np.abs(y) > 1e-6) > 0  # the z box binds
    assert _rel(res["x"], x) < 1e-8 and _rel(res["u"], u) < 1e-8
    assert _rel(res["y"], y) < 1e-6
