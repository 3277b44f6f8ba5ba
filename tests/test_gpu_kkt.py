"""The library's FP64 optimality check (stotree_kkt_check) against the oracle's residuals.

oracle/kkt_check.py evaluates, in FP64 on the host, the five residuals the check reports
(dynamics, input stationarity through the costates, box feasibility, complementarity, sign of
the multipliers; for soft terms the distance of y to the subdifferential of g).  Both sides
take the same (x, u, y), so they differ only by summation order: they agree to 1e-9 relative
(of the residual, with a floor of 1e-13 of the data's scale).  The points: the GPU's own FP64
solution, and that solution with one planted violation each, which the check must report where
the optimality conditions say and by the planted amount."""
import numpy as np
import pytest
import torch

from oracle import kkt_check as KC
from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W
from tests import dense_kkt as D

pytestmark = pytest.mark.gpu

KEYS = ("dynamics", "stationarity", "feasibility", "complementarity", "sign", "gap")
BOXED = [D.boxed_problem(12, horizon=3, nx=3, nu=2), D.boxed_problem(17, horizon=4, nx=4, nu=2, frac=0.9),
         D.boxed_problem(16, horizon=3, nx=5, nu=3, frac=0.9)]


def _st():
    from paper_2107_01745_b300.stotree import StoTree
    return StoTree


def _agree(gpu, orc, scale):
    for k in KEYS:
        assert abs(gpu[k] - orc[k]) <= 1e-9 * abs(orc[k]) + 1e-13 * scale, (k, gpu[k], orc[k])


def _points(p, x, u, y):
    """The solution and five planted violations: (name, x, u, y, residual, amount)."""
    nn, npn = p.tree.num_nodes, p.tree.num_nonleaf
    leaf = nn - 1
    out = [("solution", x, u, y, None, 0.0)]
    x1 = x.copy()
    x1[leaf, 0] += 4e-3
    out.append(("state off its dynamics", x1, u, y, "dynamics", 4e-3))
    u1 = u.copy()
    u1[0, 0] += 3e-3
    out.append(("input moved", x, u1, y, "stationarity", 2.0 * p.R[0] * 3e-3))
    x2 = x.copy()
    x2[leaf, 0] = p.xhi[0] + 0.125
    out.append(("state past its bound", x2, u, y, "feasibility", 0.125))
    h = np.concatenate([np.concatenate([x[i], u[i]]) if i < npn else x[i] for i in range(nn)])
    lo, hi = D.box_vectors(p)
    inside = np.nonzero((h < hi - 1e-3) & (h > lo + 1e-3))[0]
    k = int(inside[inside >= p.nx][0])
    y1 = y.copy()
    y1[k] = 0.0625
    out.append(("multiplier inside the box", x, u, y1, "complementarity", 0.0625))
    act = np.nonzero(np.abs(y) > 1e-4)[0]
    ka = int(act[0])
    y2 = y.copy()
    y2[ka] = -y[ka]
    out.append(("multiplier of the wrong sign", x, u, y2, "sign", abs(y[ka])))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", BOXED, ids=lambda p: p.name)
def test_kkt_check_matches_oracle(cuda_device, p, prec):
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    st = _st()(p, precision=prec)
    st.factor()
    res = st.solve("nama", lam, tol=1e-10 if prec == "fp64" else 1e-5, max_iter=2000)
    # the points are taken in the handle's precision, so both sides see the same numbers
    x, u, y = (res[k].double().cpu().numpy() for k in ("x", "u", "y"))
    scale = max(1.0, float(np.max(np.abs(x))), float(np.max(np.abs(y))))
    x0 = st.to_dev(p.x0)
    x0h = x0.double().cpu().numpy()
    # bounds within tol_active count as active: the FP32 run stops within 1e-5 of them
    tol_act = 1e-6 if prec == "fp64" else 1e-4
    for name, xp, up, yp, key, amount in _points(p, x, u, y):
        gpu = st.kkt_check(x0, st.to_dev(xp), st.to_dev(up), st.to_dev(yp), tol_active=tol_act)
        xq, uq, yq = (st.to_dev(v).double().cpu().numpy() for v in (xp, up, yp))
        orc = KC.kkt_residuals(p, x0h, xq, uq, yq, tol_active=tol_act)
        _agree(gpu, orc, scale)
        if key is None:
            if prec == "fp64":
                assert max(gpu.values()) <= 1e-8 * scale, gpu
            continue
        # the planted residual is reported, by the planted amount (pi^0 = 1 for the root's
        # input); in FP32 the point itself carries the rounding of the stopped solution
        rel = 1e-9 if prec == "fp64" else 5e-2
        assert abs(gpu[key] - amount) <= rel * amount + 1e-12 * scale, (name, gpu[key], amount)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_kkt_check_soft_terms_matches_oracle(cuda_device, prec):
    """Soft (kind 1), Huber (kind 2) and hard components at the GPU's NAMA solution and at random
    points: the generalised residuals agree with the oracle's."""
    p = D.boxed_problem(16, horizon=3, nx=5, nu=3, frac=0.9)
    n = p.nx + p.nu
    kinds = np.array([1, 2, 0, 1, 2, 0, 1, 2][:n])
    W.with_penalty(p, kinds, np.linspace(0.5, 2.0, n), np.linspace(0.2, 0.6, n))
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    st = _st()(p, precision=prec)
    st.factor()
    res = st.solve("nama", lam, tol=1e-10 if prec == "fp64" else 1e-5, max_iter=3000)
    x0 = st.to_dev(p.x0)
    x0h = x0.double().cpu().numpy()
    rng = np.random.default_rng(3)
    pts = [tuple(res[k].double().cpu().numpy() for k in ("x", "u", "y"))]
    for _ in range(3):
        x, u, y = pts[0]
        pts.append((x + 0.3 * rng.standard_normal(x.shape), u + 0.3 * rng.standard_normal(u.shape),
                    y + 0.5 * rng.standard_normal(y.shape)))
    for x, u, y in pts:
        gpu = st.kkt_check(x0, st.to_dev(x), st.to_dev(u), st.to_dev(y), tol_active=1e-6)
        xq, uq, yq = (st.to_dev(v).double().cpu().numpy() for v in (x, u, y))
        orc = KC.kkt_residuals(p, x0h, xq, uq, yq, tol_active=1e-6)
        _agree(gpu, orc, max(1.0, float(np.max(np.abs(xq))), float(np.max(np.abs(yq)))))


@pytest.mark.slow
def test_kkt_check_paper_scale_matches_oracle(cuda_device):
    """The paper-scale instance (1.79 M duals): the check at the FP32 NAMA result and at that
    result with a dual moved inside the box, against the oracle's residuals."""
    p = W.paper_scale(2)
    st = _st()(p, precision="fp32")
    st.factor()
    r0 = torch.as_tensor(np.random.default_rng(7).standard_normal(st.m), dtype=torch.float32, device="cuda")
    lam, _ = st.estimate_lambda(r0, iters=50)
    res = st.solve("nama", lam, tol=1e-4, max_iter=300)
    x0 = st.to_dev(p.x0)
    x, u, y = (res[k].double().cpu().numpy() for k in ("x", "u", "y"))
    x0h = x0.double().cpu().numpy()
    scale = max(1.0, float(np.max(np.abs(x))), float(np.max(np.abs(y))))
    y1 = y.copy()
    k = p.nx + 7  # an input of the root; the box leaves it inside or active, either way a change
    y1[k] += 0.05
    for yp in (y, y1):
        gpu = st.kkt_check(x0, res["x"], res["u"], st.to_dev(yp), tol_active=1e-3)
        orc = KC.kkt_residuals(p, x0h, x, u, st.to_dev(yp).double().cpu().numpy(), tol_active=1e-3)
        print("paper-scale KKT", gpu, orc)
        _agree(gpu, orc, scale)
