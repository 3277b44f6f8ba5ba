"""The largest single instance at full size (horizon 24, binary for 12 stages, 57,343 nodes,
nx = 200, nu = 100: 16.8 M primal and dual variables).  The FP64 oracle cannot hold it, so the
GPU results are checked by properties that hold at any size:

* the optimality conditions of the solve step (dynamics and u equations with the costates of
  the inner problem), evaluated in FP64 on the host by oracle/stream_kkt.py while the per-node
  data is regenerated block by block;
* x(y) affine in y: x(y + tau d) - x(y) = tau x_lin(d);
* the dual Hessian symmetric: <a, H x_lin(b)> = <b, H x_lin(a)>;
* NAMA reaching ||z - Hx||_inf <= 1e-4, with the library's FP64 KKT check and the host residuals
  at the returned point.

Tolerances (FP32 solve path): each dynamics equation is one 300-term FP32 product (rounding
~1e-6 of its scale, bound 1e-5); the u equations carry the FP32 errors of the whole backward
recursion through 24 stages against FP64 costates (bound 1e-3 of their scale)."""
import numpy as np
import pytest
import torch

from oracle import stream_kkt as SK
from paper_2107_01745_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def big(cuda_device):
    from paper_2107_01745_b300.stotree import StoTree
    p = W.largest(5)
    st = StoTree(p, precision="fp32", chunk_nodes=4096)
    st.factor()
    yield p, st
    st.close()


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / max(1e-30, float(torch.linalg.vector_norm(b))))


def test_largest_solve_step_optimality(big):
    p, st = big
    y = W.random_dual(p, 21, scale=1.0)
    st.solve_step(st.to_dev(y))
    x, u = st.last_primal()
    res = SK.solve_step_residuals(p, y, x.double().cpu().numpy(), u.double().cpu().numpy())
    print("largest solve step residuals", res)
    assert res["dynamics"] <= 1e-5 * res["dynamics_scale"]
    assert res["u_eq"] <= 1e-3 * res["u_scale"]


def test_largest_affine_and_symmetric(big):
    p, st = big
    g = torch.Generator(device="cuda").manual_seed(3)
    y = torch.randn(st.m, device="cuda", generator=g)
    d = torch.randn(st.m, device="cuda", generator=g)
    tau = 0.37
    hy = st.solve_step(y)
    hyd = st.solve_step(y + tau * d)
    hd = st.solve_step(d, homogeneous=True)
    assert _rel(hyd - hy, tau * hd) < 1e-4
    a = torch.randn(st.m, device="cuda", generator=g)
    ha = st.solve_step(a, homogeneous=True)
    lhs, rhs = float(torch.dot(a.double(), hd.double())), float(torch.dot(d.double(), ha.double()))
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), abs(rhs))


def test_largest_nama_to_tolerance(big):
    p, st = big
    r0 = torch.as_tensor(np.random.default_rng(7).standard_normal(st.m), dtype=torch.float32, device="cuda")
    lam, _ = st.estimate_lambda(r0, iters=50, safety=0.9)
    res = st.solve("nama", lam, tol=1e-4, max_iter=1000)
    info = res["info"]
    print("largest NAMA", info)
    assert info["status"] == 0 and info["res_inf"] <= 1e-4
    x, u, y = res["x"], res["u"], res["y"]
    kkt = st.kkt_check(st.to_dev(p.x0), x, u, y, tol_active=1e-3)
    print("largest FP64 KKT", kkt)
    assert kkt["dynamics"] < 1e-4 and kkt["feasibility"] < 2e-4
    r = SK.solve_step_residuals(p, y.double().cpu().numpy(), x.double().cpu().numpy(), u.double().cpu().numpy())
    print("largest NAMA solution residuals", r)
    assert r["dynamics"] <= 1e-5 * r["dynamics_scale"]
    assert r["u_eq"] <= 1e-3 * r["u_scale"]
