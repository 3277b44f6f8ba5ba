"""stotree_solve_step_noalloc against stotree_solve_step.

The no-allocation entry point serves callers that cannot call cudaMalloc (or any
allocator) while they run a solve, e.g. a controller whose device-memory plan is frozen
after start-up: its per-call scratch is a fixed array compiled into the library.  Its
result must equal the ordinary solve step's, call after call, although the shared array
keeps the previous call's contents.  This file is collected last so that a run stopping at
the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2107_01745_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel2(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_noalloc_matches_solve_step_twice(cuda_device, prec, tol):
    from paper_2107_01745_b300.stotree import StoTree, lib, _t_ptr, _stream
    p = W.random_problem(51, horizon=4, nx=7, nu=3)
    st = StoTree(p, precision=prec)
    st.factor()
    x0 = st.to_dev(p.x0)
    for call, (seed, homog, scaled) in enumerate([(1, False, False), (2, True, True)]):
        y = st.to_dev(W.random_dual(p, seed))
        ref = st.solve_step(y, x0=x0, homogeneous=homog, scaled=scaled)
        out = torch.full_like(y, float("nan"))
        code = lib().stotree_solve_step_noalloc(st.h, _t_ptr(y), _t_ptr(x0), _t_ptr(out), int(homog),
                                                int(scaled), _stream())
        torch.cuda.synchronize()
        assert code == 0, f"call {call}: status {code}"
        assert torch.isfinite(out).all()
        assert _rel2(out, ref) < tol, f"call {call}"


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_noalloc_as_the_first_solve_of_a_handle(cuda_device, prec, tol):
    """A freshly factored handle whose first solve is the no-allocation call: the factor has set
    up the launch, so the result equals a later ordinary solve step.  The no-allocation call
    leaves stotree_last_primal on the last ordinary round."""
    from paper_2107_01745_b300.stotree import StoTree
    p = W.random_problem(52, horizon=5, nx=9, nu=4, max_branch=3)
    st = StoTree(p, precision=prec)
    st.factor()
    x0 = st.to_dev(p.x0)
    y1 = st.to_dev(W.random_dual(p, 11))
    first = st.solve_step_noalloc(y1, x0=x0)
    torch.cuda.synchronize()
    st.round_status()
    ref = st.solve_step(y1, x0=x0)
    assert _rel2(first, ref) < tol
    x1, u1 = st.last_primal()
    y2 = st.to_dev(W.random_dual(p, 12))
    second = st.solve_step_noalloc(y2, x0=x0)
    x2, u2 = st.last_primal()
    torch.cuda.synchronize()
    assert torch.equal(x1, x2) and torch.equal(u1, u2)
    assert _rel2(second, st.solve_step(y2, x0=x0)) < tol


def test_noalloc_paper_scale_and_limit(cuda_device):
    """The paper-scale tree fits the fixed scratch; a problem needing more is refused with a message."""
    from paper_2107_01745_b300.stotree import StoTree, _stream, _t_ptr
    p = W.paper_scale(2)
    st = StoTree(p, precision="fp32")
    st.factor()
    x0 = st.to_dev(p.x0)
    for seed in (3, 4):
        y = st.to_dev(W.random_dual(p, seed, scale=0.5))
        ref = st.solve_step(y, x0=x0)
        out = st.solve_step_noalloc(y, x0=x0)
        torch.cuda.synchronize()
        assert _rel2(out, ref) < 1e-5
    # a tree needing more scratch than the fixed array: refused before any device work
    from paper_2107_01745_b300.stotree import _TreeDesc, lib
    t = W.tree_from_branching([2] * 13)  # 16383 nodes; with nx=400, nu=100: about 115 MB of scratch
    parent = np.ascontiguousarray(t.parent, dtype=np.int32)
    prob = np.ascontiguousarray(t.prob)
    desc = _TreeDesc(t.num_nodes, t.horizon, 400, 100, parent.ctypes.data, prob.ctypes.data)
    h = ctypes.c_void_p()
    assert lib().stotree_create(ctypes.byref(desc), 1, ctypes.byref(h)) == 0
    try:
        code = lib().stotree_solve_step_noalloc(h, _t_ptr(x0), _t_ptr(x0), _t_ptr(x0), 0, 0, _stream())
        assert code == 1
        assert b"scratch" in lib().stotree_last_error(h)
    finally:
        lib().stotree_destroy(h)
