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


@pytest.mark.parametrize("k", [0, 117, 299])
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
    assert info["iters"] == ref["iters"] and info["solve_calls"] == ref["solve_calls"]
    assert _relinf(res["x"].cpu().numpy(), ref["x"]) < 1e-8
    assert _relinf(res["y"].cpu().numpy(), ref["y"]) < 1e-7
    st.close()


def test_call_statistic_fp32_against_oracle(cuda_device, system):
    """On the first 40 stored states the FP32 GPU runs need as many oracle calls as the FP64
    oracle's, to within a few per problem, so the share solved within 50 calls agrees."""
    from paper_2107_01745_b300.stotree import StoTree
    X, meta, p, o, lam = system
    st = StoTree(p, precision="fp32")
    st.factor()
    for method in ("nama", "minfbe"):
        gpu, ref = [], []
        fn = O.nama if method == "nama" else O.minfbe
        for k in range(40):
            o.p.x0 = X[k]
            ref.append(fn(o, lam, tol=TOL, max_iter=5000)["solve_calls"])
            gpu.append(st.solve(method, lam, x0=st.to_dev(X[k]), tol=TOL, max_iter=5000,
                                outputs=False)["info"]["solve_calls"])
        gpu, ref = np.array(gpu), np.array(ref)
        print(method, "calls gpu", gpu.tolist(), "oracle", ref.tolist())
        assert np.median(np.abs(gpu - ref)) <= 3
        assert abs(np.mean(gpu <= 50) - np.mean(ref <= 50)) <= 0.1
    st.close()
