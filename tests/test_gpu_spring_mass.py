"""The spring-mass experiment of Section IV-A on the GPU against the FP64 oracle: iterates and
oracle-call counts of NAMA, MINFBE and GPAD at stored initial states, and the call-count
statistic of the paper (share of problems solved within 50 calls, GPAD's median) on a sample."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 5e-4


def _relinf(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


@pytest.fixture(scope="module")
def system():
    X, meta = W.spring_mass_x0s()
    p = W.spring_mass(X[0], p_max=meta["p_max"])
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    return X, meta, p, o, lam


@pytest.mark.parametrize("k", [0, 2, 5])
@pytest.mark.parametrize("method", ["nama", "minfbe", "gpad"])
def test_fp64_matches_oracle(cuda_device, system, method, k):
    from paper_2107_01745_b300.stotree import StoTree
    X, meta, p, o, lam = system
    o.p.x0 = X[k]
    fn = {"nama": O.nama, "minfbe": O.minfbe, "gpad": O.gpad}[method]
    ref = fn(o, lam, tol=TOL, max_iter=5000)
    st = StoTree(p, precision="fp64")
    st.factor()
    res = st.solve(method, lam, x0=st.to_dev(X[k]), tol=TOL, max_iter=5000)
    info = res["info"]
    assert info["status"] == 0 and info["res_inf"] <= TOL
    # FP64 iterates agree to rounding; over a hundred iterations a line-search or curvature
    # decision taken at rounding level can differ, so long runs may differ by a few iterations
    assert abs(info["iters"] - ref["iters"]) <= max(2, ref["iters"] // 10)
    # calls in the paper's sense (right-hand sides through Algorithm 3/4: NAMA x(y), x_lin(r),
    # x_lin(d) per iteration; MINFBE x_lin(d), x(y+), x_lin(R+); GPAD x(w)); the oracle's own
    # count is higher because its line search solves at every trial point
    k = info["iters"]
    assert info["solve_calls"] == {"nama": 1 + 3 * k, "minfbe": 2 + 3 * k, "gpad": 1 + k}[method]
    # the same stopping iterate to rounding; else two iterates that both meet the tolerance
    same = info["iters"] == ref["iters"]
    assert _relinf(res["x"].cpu().numpy(), ref["x"]) < (1e-8 if same else 1e-4)
    assert _relinf(res["y"].cpu().numpy(), ref["y"]) < (1e-7 if same else 1e-2)
    st.close()


def test_iterations_against_stored_oracle_counts(cuda_device, system):
    """On the first 16 stored states the GPU (FP64, the precision the statistic is taken in:
    the duals are of order 100, and near the tolerance the steps lambda R fall below FP32's
    resolution of the iterate) takes the oracle's number of iterations (within 2 for runs of
    up to 30 iterations, within a factor 1.5 for the long ones, where rounding-level decisions
    accumulate); states the oracle does not solve within 300 iterations are hard on the GPU
    too.  The oracle's counts come from tests/golden/make_spring_mass_iters.py."""
    import json
    import os
    from paper_2107_01745_b300.stotree import StoTree
    X, meta, p, o, lam = system
    with open(os.path.join(os.path.dirname(__file__), "golden", "spring_mass_oracle_iters.json")) as f:
        gold = json.load(f)
    assert abs(gold["lambda"] - lam) <= 1e-12 * lam
    st = StoTree(p, precision="fp64")
    st.factor()
    for method in ("nama", "minfbe"):
        got = []
        for k, it, conv in zip(gold["states"], gold[method]["iters"], gold[method]["converged"]):
            info = st.solve(method, lam, x0=st.to_dev(X[k]), tol=TOL, max_iter=gold["max_iter"], outputs=False,
                            allow_not_converged=True)["info"]
            got.append(info["iters"])
            if conv and it <= 30:
                assert info["status"] == 0 and abs(info["iters"] - it) <= 2, (method, k)
            elif conv:
                # long runs: rounding-level decisions accumulate; both sides find them hard
                assert info["status"] == 0 and it / 1.5 <= info["iters"] <= 1.5 * it, (method, k)
            else:
                assert info["iters"] >= gold["max_iter"] // 2, (method, k)
        print(method, "iterations gpu", got, "oracle", gold[method]["iters"])
    st.close()
