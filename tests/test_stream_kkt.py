"""Pins of the streamed optimality check (oracle/stream_kkt.py) and of the block-generated
largest instance: the independent dense KKT solution has zero residuals, a perturbation shows
up exactly where the equations say, and block generation is the same however it is sliced."""
import copy

import numpy as np
import pytest

from oracle import stream_kkt as SK
from paper_2107_01745_b300 import workloads as W
from tests import dense_kkt as D

PROBLEMS = [W.tiny_fp64(0), W.random_problem(1, horizon=3, nx=3, nu=2), W.random_problem(3, horizon=3, nx=5, nu=3)]


@pytest.mark.parametrize("p", PROBLEMS, ids=lambda p: p.name)
@pytest.mark.parametrize("homogeneous", [False, True])
def test_dense_kkt_solution_has_zero_residuals(p, homogeneous):
    y = W.random_dual(p, 13, scale=2.0)
    x, u = D.dense_solve(p, y, homogeneous)
    res = SK.solve_step_residuals(p, y, x, u, homogeneous=homogeneous, block=3)
    assert res["dynamics"] <= 1e-10 * max(1.0, res["dynamics_scale"])
    assert res["u_eq"] <= 1e-10 * max(1.0, res["u_scale"])


def test_perturbation_is_detected_where_it_enters():
    """Changing u^i by delta e_k leaves the costates alone (x is unchanged) and moves the u
    equation of node i by exactly 2 pi^i R_k delta; the dynamics of i's children break."""
    p = PROBLEMS[1]
    y = W.random_dual(p, 5)
    x, u = D.dense_solve(p, y)
    i, k, delta = 2, 1, 1e-3
    u2 = u.copy()
    u2[i, k] += delta
    res = SK.solve_step_residuals(p, y, x, u2)
    assert abs(res["u_eq"] - 2.0 * p.tree.prob[i] * p.R[k] * delta) < 1e-12
    assert res["dynamics"] > 0.1 * delta * np.min(np.abs(p.B[p.tree.child_begin[i]][:, k]).max())


@pytest.mark.parametrize("homogeneous", [False, True])
def test_root_state_is_checked_against_the_parameter(homogeneous):
    """x^0 is the parameter p (zero in Algorithm 4): a candidate whose root state is off by
    delta while every other equation is rebuilt around it (the solve step of the changed
    parameter) still violates x^0 = p by exactly delta."""
    p = PROBLEMS[1]
    y = W.random_dual(p, 6)
    delta = 2.5e-3
    shifted = copy.copy(p)
    shifted.x0 = np.asarray(p.x0, dtype=float) + delta * (np.arange(p.nx) == 1)
    if homogeneous:
        # Algorithm 4 has x^0 = 0: the solution for x^0 = delta e_1 solves the inhomogeneous
        # problem with c, q, r, p_N zero
        shifted.c = np.zeros_like(p.c)
        shifted.q, shifted.r, shifted.pN = np.zeros(p.nx), np.zeros(p.nu), np.zeros(p.nx)
        shifted.x0 = delta * (np.arange(p.nx) == 1)
    x, u = D.dense_solve(shifted, y)
    res = SK.solve_step_residuals(p, y, x, u, homogeneous=homogeneous, block=3)
    assert abs(res["dynamics"] - delta) < 1e-12
    assert res["u_eq"] <= 1e-10 * max(1.0, res["u_scale"])


def test_largest_blocks_are_slice_independent():
    p = W.largest_unboxed(5, tree=W.largest_tree(horizon=4, branch_stages=2))
    nn = p.tree.num_nodes
    A_all = p.A[0:nn]
    q = W.largest_unboxed(5, tree=W.largest_tree(horizon=4, branch_stages=2))
    for f, s in [(0, 3), (3, 7), (5, nn)]:
        assert np.array_equal(q.A[f:s], A_all[f:s])
        assert np.array_equal(q.B[f:s], p.B[f:s])
        assert np.array_equal(q.c[f:s], p.c[f:s])
    assert np.all(A_all[0] == 0.0) and np.all(p.c[0:1] == 0.0)
    # the recipe: perturbations of spectral-radius-0.98 A of size 0.02, B ~ N(0, 1/nx)
    A0 = np.linalg.eigvals(A_all[1:].mean(axis=0))
    assert abs(np.max(np.abs(A0)) - 0.98) < 0.05
    assert abs(np.std(p.B[1:nn]) - 1.0 / np.sqrt(p.nx)) < 0.01


def test_block_generated_problem_against_dense_kkt():
    """A small tree from the largest instance's generator: the streamed check of the dense
    solution is zero with blocks read in pieces."""
    p = W.largest_unboxed(5, tree=W.largest_tree(horizon=3, branch_stages=2))
    p.nx, p.nu = W.LARGEST_SHAPE["nx"], W.LARGEST_SHAPE["nu"]
    nn = p.tree.num_nodes
    dense = W.Problem(tree=p.tree, nx=p.nx, nu=p.nu, A=p.A[0:nn], B=p.B[0:nn], c=p.c[0:nn], Q=p.Q, R=p.R,
                      PN=p.PN, q=p.q, r=p.r, pN=p.pN, xlo=p.xlo, xhi=p.xhi, ulo=p.ulo, uhi=p.uhi, x0=p.x0)
    y = W.random_dual(dense, 3)
    x, u = D.dense_solve(dense, y)
    res = SK.solve_step_residuals(p, y, x, u, block=2)
    assert res["dynamics"] <= 1e-9 * max(1.0, res["dynamics_scale"])
    assert res["u_eq"] <= 1e-9 * max(1.0, res["u_scale"])
