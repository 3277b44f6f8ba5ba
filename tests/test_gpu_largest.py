"""The largest single instance (horizon 24, binary for 12 stages, 57,343 nodes, nx = 200,
nu = 100: 16.8 M primal and dual variables).

Element by element: a depth-truncated instance of the same recipe (the same generator, sizes,
box and twelve binary stages, cut at horizon 14: 16,383 nodes, 4.5 M duals) fits the FP64
oracle, so its solve step (every output entry, within the 1e-5 dual-gradient bound), its
primal trajectory, NAMA's solution and the FP64 optimality check are compared with the
oracle's.

At full size the FP64 oracle cannot hold the instance, so the GPU results are checked by
properties that hold at any size:

* the optimality conditions of the solve step (dynamics and u equations with the costates of
  the inner problem), evaluated in FP64 on the host by oracle/stream_kkt.py while the per-node
  data is regenerated block by block;
* x(y) affine in y: x(y + tau d) - x(y) = tau x_lin(d);
* the dual Hessian symmetric: <a, H x_lin(b)> = <b, H x_lin(a)>;
* NAMA reaching ||z - Hx||_inf <= 1e-4, with the library's FP64 KKT check and the host residuals
  at the returned point.

Tolerances (FP32 solve path): each dynamics equation is one 300-term FP32 product (rounding
~1e-6 of its scale, bound 1e-5); the u equations carry the FP32 errors of the whole backward
recursion through 24 stages against FP64 costates: bound 1e-5 of their scale at the duals the
solvers evaluate (the preconditioned random dual, NAMA's solution; measured 6e-7 at the
solution), 1e-4 at an unscaled random dual whose states are four orders larger."""
import numpy as np
import pytest
import torch

from oracle import stream_kkt as SK
from paper_2107_01745_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def truncated():
    from oracle import oracle as O
    p = W.largest_truncated(5, horizon=14)
    p.A, p.B, p.c = p.A[:], p.B[:], p.c[:]  # dense arrays for the oracle
    return p, O.LQOracle(p)


def _rel2(a, b):
    return float(np.linalg.norm(a - b) / max(1e-30, np.linalg.norm(b)))


def test_largest_recipe_truncated_solve_step_matches_oracle(cuda_device, truncated):
    from paper_2107_01745_b300.stotree import StoTree
    p, o = truncated
    st = StoTree(p, precision="fp32", chunk_nodes=4096)
    st.factor()
    for homog in (False, True):
        y = W.random_dual(p, 31 + homog)
        h = st.solve_step(st.to_dev(y), homogeneous=homog).double().cpu().numpy()
        assert _rel2(h, o.hx(y, homogeneous=homog)) < 1e-5, homog
    Y = np.stack([W.random_dual(p, 33), W.random_dual(p, 34)])
    H = st.solve_step(st.to_dev(Y)).double().cpu().numpy()
    for k in range(2):
        assert _rel2(H[k], o.hx(Y[k])) < 1e-5
    st.solve_step(st.to_dev(Y[1]))
    x, u = st.last_primal()
    xr, ur = o.solve(Y[1])
    assert _rel2(x.double().cpu().numpy(), xr) < 1e-5 and _rel2(u.double().cpu().numpy(), ur) < 1e-5
    st.close()


def test_largest_recipe_truncated_nama_matches_oracle(cuda_device, truncated):
    """NAMA to ||z - Hx||_inf <= 1e-4 on the truncated instance: the solution against the
    oracle's NAMA at the same tolerance and step, and the FP64 check against the oracle's
    residuals at the GPU's result."""
    from oracle import kkt_check as KC
    from oracle import oracle as O
    from paper_2107_01745_b300.stotree import StoTree
    p, o = truncated
    lam, _ = O.power_lambda(o, np.random.default_rng(7).standard_normal(o.m), iters=30)
    ref = O.nama(o, lam, tol=1e-4, max_iter=200)
    st = StoTree(p, precision="fp32", chunk_nodes=4096)
    st.factor()
    res = st.solve("nama", lam, tol=1e-4, max_iter=200)
    info = res["info"]
    print("truncated largest NAMA", info, "oracle iters", ref["iters"])
    assert info["status"] == 0 and info["res_inf"] <= 1e-4
    x, u, y = (res[k].double().cpu().numpy() for k in ("x", "u", "y"))
    dx = float(np.max(np.abs(x - ref["x"])) / max(1.0, np.max(np.abs(ref["x"]))))
    du = float(np.max(np.abs(u - ref["u"])) / max(1.0, np.max(np.abs(ref["u"]))))
    print("truncated largest relinf x, u", dx, du)
    assert dx < 1e-4 and du < 1e-4
    x0 = st.to_dev(p.x0)
    gpu = st.kkt_check(x0, res["x"], res["u"], res["y"], tol_active=1e-3)
    orc = KC.kkt_residuals(p, x0.double().cpu().numpy(), x, u, y, tol_active=1e-3)
    scale = max(1.0, float(np.max(np.abs(x))), float(np.max(np.abs(y))))
    for k in gpu:
        assert abs(gpu[k] - orc[k]) <= 1e-9 * abs(orc[k]) + 1e-13 * scale, (k, gpu[k], orc[k])
    st.close()


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


@pytest.mark.parametrize("kind", ["preconditioned", "unscaled"])
def test_largest_solve_step_optimality(big, kind):
    """The optimality conditions of x(y) at a dual of the form the solvers evaluate (y = sqrt(pi)
    ybar, ybar ~ N(0, 1): the preconditioned dual of Section III-E), within the 1e-5 bound, and
    at an unscaled N(0, 1) dual, whose states reach 1e4 against O(1) inputs, so the u equations
    cancel more and FP32 rounding of the recursion is bounded by 1e-4 of their scale."""
    p, st = big
    y = W.random_dual(p, 21, scale=1.0)
    if kind == "preconditioned":
        sq = np.sqrt(p.tree.prob[np.repeat(np.arange(p.tree.num_nodes), np.diff(W.dual_offsets(p.tree, p.nx, p.nu)))])
        y = sq * y
    st.solve_step(st.to_dev(y))
    x, u = st.last_primal()
    res = SK.solve_step_residuals(p, y, x.double().cpu().numpy(), u.double().cpu().numpy())
    print("largest solve step residuals", kind, res)
    assert res["dynamics"] <= 1e-5 * res["dynamics_scale"]
    assert res["u_eq"] <= (1e-5 if kind == "preconditioned" else 1e-4) * res["u_scale"]


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
    assert r["u_eq"] <= 1e-5 * r["u_scale"]
