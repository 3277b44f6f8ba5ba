"""The spring-mass workload of Section IV-A: the generator against independent facts, and the
oracle's solvers on it.

* the zero-order hold against scipy.signal.cont2discrete;
* the continuous model: Newton's law by hand for one mass, energy dissipation of the
  undriven array (spring potential plus kinetic energy never increases), a stable spectrum;
* the Markov scenario tree: conditional probabilities of the children, stage marginals of the
  modes against the chain's distribution p_c P_c^t, the disturbance of each node's mode;
* the stored initial states: inside the state box, and (two of them) feasible by the LP;
* NAMA, MINFBE and GPAD reach the paper's tolerance 5e-4 at a stored initial state, with the
  optimality conditions of the solve step and a feasible primal.
"""
import numpy as np
import pytest
import scipy.signal

from oracle import oracle as O
from oracle import stream_kkt as SK
from paper_2107_01745_b300 import workloads as W

S = W.SPRING_MASS


def test_zoh_matches_scipy_cont2discrete():
    Ac, Bc = W.spring_mass_continuous()
    A, B = W.zoh(Ac, Bc, S["Ts"])
    Ad, Bd, *_ = scipy.signal.cont2discrete((Ac, Bc, np.eye(10), np.zeros((10, 4))), S["Ts"], method="zoh")
    assert np.max(np.abs(A - Ad)) < 1e-12 and np.max(np.abs(B - Bd)) < 1e-12


def test_continuous_model_by_hand_and_energy():
    Ac, Bc = W.spring_mass_continuous()
    m, k, b = S["mass"], S["k_s"], S["b_d"]
    # mass 2 (index 1): m v2' = -k (p2 - p1) - k (p2 - p3) - b (v2 - v1) - b (v2 - v3) + u1 - u2
    x = np.arange(1.0, 11.0)
    u = np.array([0.3, -0.7, 0.2, 0.5])
    p, v = x[:5], x[5:]
    acc = (-k * (p[1] - p[0]) - k * (p[1] - p[2]) - b * (v[1] - v[0]) - b * (v[1] - v[2]) + u[0] - u[1]) / m
    assert abs((Ac @ x + Bc @ u)[6] - acc) < 1e-14
    # the walls: mass 1 is tied to a fixed wall at p = 0
    acc1 = (-k * p[0] - k * (p[0] - p[1]) - b * v[0] - b * (v[0] - v[1]) - u[0]) / m
    assert abs((Ac @ x + Bc @ u)[5] - acc1) < 1e-14
    # energy E = m/2 |v|^2 + k/2 sum of squared spring extensions never increases undriven
    A, _ = W.zoh(Ac, Bc, S["Ts"])
    rng = np.random.default_rng(0)
    ext = lambda p: np.concatenate([[p[0]], np.diff(p), [-p[-1]]])
    E = lambda x: 0.5 * m * x[5:] @ x[5:] + 0.5 * k * ext(x[:5]) @ ext(x[:5])
    for _ in range(5):
        x = rng.standard_normal(10)
        for _ in range(40):
            xn = A @ x
            assert E(xn) <= E(x) * (1 + 1e-12)
            x = xn
    assert np.max(np.real(np.linalg.eigvals(Ac))) < 0


def test_markov_tree():
    p = W.spring_mass()
    t = p.tree
    tree, modes = W.markov_tree(S["horizon"], S["p_c"], S["P_c"])
    assert t.num_nodes == 2 ** (S["horizon"] + 1) - 1
    Pc = np.asarray(S["P_c"])
    for i in range(t.num_nonleaf):
        kids = range(t.child_begin[i], t.child_begin[i] + t.child_count[i])
        cond = t.prob[list(kids)] / t.prob[i]
        want = np.asarray(S["p_c"]) if i == 0 else Pc[modes[i]]
        assert np.allclose(cond, want, atol=1e-15)
        assert [modes[j] for j in kids] == [0, 1]
    dist = np.asarray(S["p_c"])
    for s in range(1, S["horizon"] + 1):
        nodes = t.stage_nodes(s)
        marg = np.array([t.prob[nodes][modes[nodes] == a].sum() for a in (0, 1)])
        assert np.allclose(marg, dist, atol=1e-12)
        dist = dist @ Pc
    assert np.all(p.c[1:][modes[1:] == 0] == 0.0) and np.all(p.c[1:][modes[1:] == 1] == 0.1)


def test_stored_initial_states():
    X, meta = W.spring_mass_x0s()
    assert X.shape == (300, 10) and meta["count"] == 300
    assert np.all(np.abs(X[:, :5]) <= meta["p_max"]) and np.all(np.abs(X[:, 5:]) <= meta["v_max"])
    assert meta["draws"] == 300 + meta["rejected_infeasible"] + meta["rejected_undecided"]


@pytest.mark.slow
def test_two_stored_states_are_feasible():
    from oracle.make_spring_mass import feasibility_status
    X, _ = W.spring_mass_x0s()
    assert feasibility_status(X[0]) == 0 and feasibility_status(X[-1]) == 0


@pytest.mark.parametrize("solver", ["nama", "minfbe", "gpad"])
def test_solvers_reach_the_papers_tolerance(solver):
    X, meta = W.spring_mass_x0s()
    p = W.spring_mass(X[0], p_max=meta["p_max"])
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    fn = {"nama": O.nama, "minfbe": O.minfbe, "gpad": O.gpad}[solver]
    res = fn(o, lam, tol=5e-4, max_iter=5000)
    assert res["status"] == "converged" and res["res_inf"] <= 5e-4
    r = SK.solve_step_residuals(p, res["y"], res["x"], res["u"], block=1024)
    assert r["dynamics"] <= 1e-12 * max(1.0, r["dynamics_scale"]) and r["u_eq"] <= 1e-10 * max(1.0, r["u_scale"])
    h = o.stack(res["x"], res["u"])
    viol = np.max(np.maximum(o.lo - h, 0) + np.maximum(h - o.hi, 0))
    assert viol <= 5e-4
