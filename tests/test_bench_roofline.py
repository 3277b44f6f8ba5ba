"""Host-side roofline accounting of bench.py and the library (CPU, no kernel launched): the
algorithmic bytes of a solve round counted node by node, the paper-scale figure the bench
reports, and the ncu traffic figure used only while the profiled kernel source is unchanged."""
import ctypes
import os
import re
import shutil

import numpy as np

import bench
from paper_2107_01745_b300 import workloads as W


class _Desc(ctypes.Structure):
    _fields_ = [("num_nodes", ctypes.c_int32), ("horizon", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("nu", ctypes.c_int32), ("parent", ctypes.c_void_p), ("prob", ctypes.c_void_p)]


def _solve_bytes(tree, nx, nu, prec):
    from paper_2107_01745_b300 import stotree
    L = stotree.lib()
    parent = np.ascontiguousarray(tree.parent, dtype=np.int32)
    prob = np.ascontiguousarray(tree.prob, dtype=np.float64)
    d = _Desc(tree.num_nodes, tree.horizon, nx, nu, parent.ctypes.data, prob.ctypes.data)
    h = ctypes.c_void_p()
    assert L.stotree_create(ctypes.byref(d), prec, ctypes.byref(h)) == 0
    try:
        mat, vec = ctypes.c_double(), ctypes.c_double()
        assert L.stotree_solve_bytes(h, ctypes.byref(mat), ctypes.byref(vec)) == 0
        return mat.value, vec.value
    finally:
        L.stotree_destroy(h)


def _count(tree, nx, nu, es):
    """Bytes one round must move, node by node: the backward pass reads A^j and B^j of every
    non-root node and, per parent, K^i and Rbar^-1; the forward pass reads A^j, B^j and K^i
    again.  Per right-hand side: y in, Hx out (a dual block per node), and s, ubar, x, u each
    written once and read once."""
    mat = vec = 0
    for i in range(tree.num_nodes):
        leaf = tree.child_count[i] == 0
        if i > 0:
            mat += 2 * (nx * nx + nx * nu)
        if not leaf:
            mat += 2 * nu * nx + nu * nu
        block = nx if leaf else nx + nu
        vec += 2 * block + 2 * nx + (0 if leaf else 2 * nu)
    return es * mat, es * vec


def test_solve_bytes_counted_node_by_node():
    rng = np.random.default_rng(3)
    for prec, es in ((1, 4), (0, 8)):
        for _ in range(3):
            tree = W.random_tree(rng, 4, max_branch=3, p_branch=0.6)
            nx, nu = int(rng.integers(1, 9)), int(rng.integers(1, 5))
            got = _solve_bytes(tree, nx, nu, prec)
            want = _count(tree, nx, nu, es)
            assert got == want


def test_paper_scale_round_streams_2_04_gb():
    """Branching 2 for ten stages, then one child per node to horizon 20 (12,287 nodes), nx = 100,
    nu = 50, FP32: each round reads 2.04 GB of matrices, the figure the bench and the profile
    summaries quote."""
    tree = W.tree_from_branching([2] * 10 + [1] * 10)
    assert tree.num_nodes == 12287 and int(np.sum(tree.child_count > 0)) == 11263
    mat, vec = _solve_bytes(tree, 100, 50, 1)
    assert round(mat / 1e9, 2) == 2.04
    assert (mat, vec) == _count(tree, 100, 50, 4)


def test_traffic_reported_only_for_the_profiled_source(tmp_path, monkeypatch):
    """bench.py takes the DRAM traffic per round from the committed ncu summary, weighted by the
    mix of one- and two-right-hand-side rounds, and reports none once solve.cu differs from the
    profiled source (its sha256 recorded in the summary)."""
    src_root = bench.ROOT
    for rel in ("profiles/k_tree_paper_scale.md", "paper_2107_01745_b300/csrc/solve.cu"):
        os.makedirs(tmp_path / os.path.dirname(rel), exist_ok=True)
        shutil.copy(os.path.join(src_root, rel), tmp_path / rel)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the copy of the summary names the copied source's hash (the committed summary may be older
    # than the source, in which case bench.py reports no traffic, as checked at the end)
    import hashlib
    src_hash = hashlib.sha256((tmp_path / "paper_2107_01745_b300/csrc/solve.cu").read_bytes()).hexdigest()
    md = tmp_path / "profiles/k_tree_paper_scale.md"
    md.write_text(re.sub(r"sha256 `[0-9a-f]{64}`", f"sha256 `{src_hash}`", md.read_text(), count=1))
    text = (tmp_path / "profiles/k_tree_paper_scale.md").read_text()
    t1 = int(re.search(r"traffic_bytes_per_round_1rhs: (\d+)", text).group(1))
    t2 = int(re.search(r"traffic_bytes_per_round_2rhs: (\d+)", text).group(1))
    # 10 rounds, 4 of them with two right-hand sides (14 right-hand sides in all)
    assert bench._traffic_per_launch(10, 14) == (6 * t1 + 4 * t2) / 10
    assert bench._traffic_per_launch(3, 3) == t1
    with open(tmp_path / "paper_2107_01745_b300/csrc/solve.cu", "a") as f:
        f.write("\n// changed\n")
    assert bench._traffic_per_launch(10, 14) is None
