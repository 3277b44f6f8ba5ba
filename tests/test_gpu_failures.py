"""Failure paths of the library, made on purpose without faulting the GPU.

* A dependency wait inside a solve round that gives up: the handle's wait limit is set to 0, so
  the first check that finds a child's (backward) or parent's (forward) work unfinished gives
  up, the round runs to its end without that input and raises the error word; the host reports
  STO_ERR_TIMEOUT (stotree_round_status after stotree_solve_step or the no-allocation step, or
  the solver itself), resets the round state, and the next round with the normal limit is
  exact again.  Nothing waits without a limit, so no launch can hang.
* NaN in the starting dual: the residual pass flags it and the solver returns
  STO_ERR_NUMERICAL instead of iterating.
* An Rbar = pi R + sum B'PB that is not positive definite (a NaN in one node's B, or B so large
  that B'PB overflows): the FP64 Cholesky of Section III-D's recursion finds a pivot that is
  not positive, and stotree_factor returns STO_ERR_NUMERICAL naming the parent node.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W

pytestmark = pytest.mark.gpu

TIMEOUT, NUMERICAL, NOT_READY = 6, 4, 3


def _st():
    from paper_2107_01745_b300.stotree import StoTree
    return StoTree


def _rel2(a, b):
    return float(np.linalg.norm(a - b) / max(1e-30, np.linalg.norm(b)))


def _chains():
    """Four chains of 40 nodes under two binary stages: every backward work item (a path of at
    most four nodes) but the first of each chain depends on the item below it, and those items
    are handed to different CTAs at the same time."""
    t = W.tree_from_branching([2, 2] + [1] * 40)
    return W.random_problem(61, tree=t, nx=48, nu=24)


@pytest.mark.parametrize("entry", ["solve_step", "noalloc"])
def test_dependency_wait_gives_up_and_is_reported(cuda_device, entry):
    from paper_2107_01745_b300.stotree import StoError
    p = _chains()
    o = O.LQOracle(p)
    st = _st()(p, precision="fp32")
    st.factor()
    y = W.random_dual(p, 5)
    yd = st.to_dev(y)
    run = st.solve_step if entry == "solve_step" else st.solve_step_noalloc
    st.set_wait_limit(0.0)
    codes = []
    for _ in range(3):
        run(yd)
        try:
            st.round_status()
            codes.append(0)
        except StoError as e:
            codes.append(e.code)
            assert "waiting" in str(e)
    assert TIMEOUT in codes, codes
    assert set(codes) <= {0, TIMEOUT}
    # the state was reset: with the normal limit the next rounds are exact and report no error
    st.set_wait_limit(1.5)
    for _ in range(2):
        h = run(yd).double().cpu().numpy()
        st.round_status()
        assert _rel2(h, o.hx(y)) < 1e-5


def test_solver_reports_a_dependency_timeout(cuda_device):
    from paper_2107_01745_b300.stotree import StoError
    p = _chains()
    st = _st()(p, precision="fp32")
    st.factor()
    st.set_wait_limit(0.0)
    seen = []
    for _ in range(3):
        try:
            st.solve("nama", 0.05, tol=1e-12, max_iter=3, allow_not_converged=True)
            seen.append(0)
        except StoError as e:
            seen.append(e.code)
    assert TIMEOUT in seen, seen
    st.set_wait_limit(1.5)
    res = st.solve("nama", 0.05, tol=1e-12, max_iter=3, allow_not_converged=True)
    assert res["info"]["iters"] == 3


def test_wait_limit_range_is_checked(cuda_device):
    from paper_2107_01745_b300.stotree import StoError
    st = _st()(W.random_problem(62, horizon=2, nx=2, nu=1), precision="fp32")
    for bad in (-1.0, 61.0, float("nan")):
        with pytest.raises(StoError) as ei:
            st.set_wait_limit(bad)
        assert ei.value.code == 1


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("method", ["nama", "minfbe", "gpad"])
def test_nan_in_the_starting_dual_is_numerical(cuda_device, prec, method):
    from paper_2107_01745_b300.stotree import StoError
    p = W.tiny_fp64(0)
    st = _st()(p, precision=prec)
    st.factor()
    y0 = np.zeros(st.m)
    y0[st.m // 2] = np.nan
    with pytest.raises(StoError) as ei:
        st.solve(method, 0.05, y0=st.to_dev(y0), tol=1e-8, max_iter=50)
    assert ei.value.code == NUMERICAL
    # the handle stays usable
    res = st.solve(method, 0.05, tol=1e-6 if prec == "fp32" else 1e-8, max_iter=5000)
    assert res["info"]["status"] == 0


@pytest.mark.parametrize("bad", ["nan", "overflow"])
def test_factor_rejects_rbar_not_positive_definite(cuda_device, bad):
    from paper_2107_01745_b300.stotree import StoError
    p = W.random_problem(63, horizon=3, nx=3, nu=2)
    j = p.tree.num_nodes - 1  # a leaf: its parent's Rbar = pi R + sum_j B^j' P^j B^j
    B = np.array(p.B[:], copy=True)
    if bad == "nan":
        B[j, 0, 0] = np.nan
    else:
        B[j] = 1e160  # B'PB overflows to inf; the second pivot of the Cholesky is then NaN
    p.B = B
    st = _st()(p, precision="fp64")
    with pytest.raises(StoError) as ei:
        st.factor()
    assert ei.value.code == NUMERICAL
    assert f"node {p.tree.parent[j]}" in str(ei.value)
    with pytest.raises(StoError) as ei:
        st.solve_step(st.to_dev(np.zeros(st.m)))
    assert ei.value.code == NOT_READY
