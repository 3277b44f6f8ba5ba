"""Parity of the general separable g (soft constraints, l1, Huber; Section II-B) on the GPU
with the FP64 oracle: the proximal step and FBE element by element, the solvers' iterates
and results, and the FP64 optimality check of the results."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W
from tests import dense_kkt as D
from tests.test_penalty_oracle import CASES, _penalised

pytestmark = pytest.mark.gpu


def _st():
    from paper_2107_01745_b300.stotree import StoTree
    return StoTree


def _relinf(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("p", CASES, ids=lambda p: p.name)
def test_prox_and_fbe_at_a_point(cuda_device, p, prec, tol):
    """Zero iterations from a given y: z_lambda(y) and phi_lambda(y) as the oracle computes them."""
    o = O.LQOracle(p)
    st = _st()(p, precision=prec)
    st.factor()
    rng = np.random.default_rng(8)
    for lam in (0.05, 0.4):
        y = rng.standard_normal(o.m) * rng.choice([0.05, 3.0], o.m)
        y[:p.nx] = 0.0
        pt = O.fb_point(o, y / o.sq, lam)
        res = st.solve("nama", lam, y0=st.to_dev(y), tol=1e-300, max_iter=0, allow_not_converged=True)
        z = res["z"].double().cpu().numpy()
        assert _relinf(z, pt["z"] / o.sq) < tol
        assert abs(res["info"]["fbe"] - pt["phi"]) <= tol * max(1.0, abs(pt["phi"])) * 10
        assert abs(res["info"]["res_inf"] - pt["res_inf"]) <= tol * max(1.0, pt["res_inf"]) * 10


@pytest.mark.parametrize("method", ["nama", "minfbe", "gpad"])
@pytest.mark.parametrize("p", CASES, ids=lambda p: p.name)
def test_solvers_fp64_match_oracle(cuda_device, p, method):
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    fn = {"nama": O.nama, "minfbe": O.minfbe, "gpad": O.gpad}[method]
    cap = 200000 if method == "gpad" else 2000
    ref = fn(o, lam, tol=1e-10, max_iter=cap)
    st = _st()(p, precision="fp64")
    st.factor()
    res = st.solve(method, lam, tol=1e-10, max_iter=cap)
    info = res["info"]
    assert info["status"] == 0 and info["res_inf"] <= 1e-10
    # the iterates agree to rounding until line-search comparisons of FBE values at rounding
    # level (near the tolerance, and at the kinks of g) go the other way
    assert abs(info["iters"] - ref["iters"]) <= (2 if method == "gpad" else max(6, ref["iters"] // 5))
    assert _relinf(res["x"].cpu().numpy(), ref["x"]) < 1e-8
    assert _relinf(res["u"].cpu().numpy(), ref["u"]) < 1e-8
    assert _relinf(res["y"].cpu().numpy(), ref["y"]) < 1e-6
    kkt = st.kkt_check(st.to_dev(p.x0), res["x"], res["u"], res["y"], tol_active=1e-7)
    assert kkt["dynamics"] < 1e-12 and kkt["stationarity"] < 1e-9
    assert kkt["feasibility"] < 1e-9 and kkt["complementarity"] < 1e-7 and kkt["sign"] < 1e-7


@pytest.mark.parametrize("method", ["nama", "minfbe"])
def test_solvers_fp32_with_penalties(cuda_device, method):
    p = _penalised(16, [1, 1, 2, 2, 1, 0, 0, 1], 0.5, delta=0.2, horizon=3, nx=5, nu=3, frac=0.9)
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    ref = (O.nama if method == "nama" else O.minfbe)(o, lam, tol=1e-10)
    st = _st()(p, precision="fp32")
    st.factor()
    res = st.solve(method, lam, tol=1e-5, max_iter=2000)
    assert res["info"]["status"] == 0 and res["info"]["res_inf"] <= 1e-5
    assert _relinf(res["x"].cpu().numpy(), ref["x"]) < 1e-4
    assert _relinf(res["u"].cpu().numpy(), ref["u"]) < 1e-4


def test_penalty_validation(cuda_device):
    from paper_2107_01745_b300.stotree import StoError
    p = CASES[0]
    st = _st()(p, precision="fp32")
    n = p.nx + p.nu
    for kind, rho, delta in (([3] * n, 1.0, 1.0), ([1] * n, 0.0, 1.0), ([2] * n, 1.0, 0.0), ([1] * n, np.inf, 1.0)):
        with pytest.raises(StoError) as ei:
            st.set_penalty(kind, rho, delta)
        assert ei.value.code == 1


@pytest.fixture(scope="module")
def soft_paper_scale():
    """The paper-scale instance with its state bounds made soft (rho = 1 per unit of
    distance; inputs stay hard)."""
    p = W.paper_scale(2)
    W.with_penalty(p, [1] * p.nx + [0] * p.nu, 1.0)
    return p, O.LQOracle(p)


@pytest.mark.slow
def test_paper_scale_soft_states(cuda_device, soft_paper_scale):
    p, o = soft_paper_scale
    r0 = np.random.default_rng(7).standard_normal(o.m)
    lam, _ = O.power_lambda(o, r0)
    ref = O.nama(o, lam, tol=1e-4, max_iter=300)
    assert ref["status"] == "converged"
    st = _st()(p, precision="fp32")
    st.factor()
    res = st.solve("nama", lam, tol=1e-4, max_iter=300)
    print("paper-scale soft states", res["info"], "oracle iters", ref["iters"])
    assert res["info"]["status"] == 0 and res["info"]["res_inf"] <= 1e-4
    assert _relinf(res["x"].cpu().numpy(), ref["x"]) < 1e-3
    kkt = st.kkt_check(st.to_dev(p.x0), res["x"], res["u"], res["y"], tol_active=1e-3)
    print("paper-scale soft states KKT", kkt)
    assert kkt["dynamics"] < 1e-4 and kkt["feasibility"] < 2e-4
