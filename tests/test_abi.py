"""CPU-side checks of the C ABI: the library builds, loads and exports every declared entry point,
and host-side validation rejects bad trees and arguments (no kernel is launched)."""
import ctypes
import re
import os

import numpy as np
import pytest

from tests.conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "stotree.h")).read()
    return sorted(set(re.findall(r"STO_API\s+[^;]*?\b(sto(?:tree|batch|warm)_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libso():
    from paper_2107_01745_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libso):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libso, n), n
    from paper_2107_01745_b300 import stotree
    assert sorted(stotree.exported_symbols()) == names


def test_status_strings(libso):
    libso.stotree_status_str.restype = ctypes.c_char_p
    assert libso.stotree_status_str(0) == b"ok"
    assert libso.stotree_status_str(7) == b"iteration limit reached"


class _Desc(ctypes.Structure):
    _fields_ = [("num_nodes", ctypes.c_int32), ("horizon", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("nu", ctypes.c_int32), ("parent", ctypes.c_void_p), ("prob", ctypes.c_void_p)]


def _create(libso, parent, prob, nx=2, nu=1, prec=1):
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    prob = np.ascontiguousarray(prob, dtype=np.float64)
    horizon = 0
    st = [0]
    for i in range(1, len(parent)):
        st.append(st[parent[i]] + 1)
    horizon = max(st)
    d = _Desc(len(parent), horizon, nx, nu, parent.ctypes.data, prob.ctypes.data)
    h = ctypes.c_void_p()
    code = libso.stotree_create(ctypes.byref(d), prec, ctypes.byref(h))
    if code == 0:
        libso.stotree_destroy.argtypes = [ctypes.c_void_p]
        m = ctypes.c_int64()
        libso.stotree_sizes.argtypes = [ctypes.c_void_p] * 5
        libso.stotree_sizes(h, ctypes.byref(m), None, None, None)
        libso.stotree_destroy(h)
        return code, m.value
    return code, None


def test_create_validates_tree(libso):
    from paper_2107_01745_b300 import workloads as W
    t = W.tree_from_branching([2, 2])
    code, m = _create(libso, t.parent, t.prob, nx=2, nu=1)
    assert code == 0 and m == 3 * 3 + 4 * 2
    bad = t.prob.copy()
    bad[1] = 0.7  # children of the root no longer sum to 1
    assert _create(libso, t.parent, bad)[0] == 2
    par = t.parent.copy()
    par[3], par[4] = par[4], par[3]  # not stage-sorted / contiguous
    par[3] = 2
    assert _create(libso, par, t.prob)[0] == 2
    # leaf above the last stage
    t2 = W.tree_from_branching([[2], [1, 0 + 1]])
    assert _create(libso, t2.parent, t2.prob)[0] == 0
    ragged = np.array([-1, 0, 0, 1], dtype=np.int32)  # node 2 is a leaf at stage 1 < horizon 2
    assert _create(libso, ragged, np.array([1.0, 0.5, 0.5, 0.5]))[0] == 2


def test_create_rejects_bad_sizes(libso):
    from paper_2107_01745_b300 import workloads as W
    t = W.tree_from_branching([2])
    assert _create(libso, t.parent, t.prob, nx=0)[0] == 1
    assert _create(libso, t.parent, t.prob, nx=400, nu=200)[0] == 1
    assert _create(libso, t.parent, t.prob, nx=200, nu=100, prec=0)[0] == 1
    assert _create(libso, t.parent, t.prob, nx=200, nu=100, prec=1)[0] == 0


def test_missing_library_fails_loudly(monkeypatch):
    """No silent fallback: without the built library the binding raises before any work."""
    import paper_2107_01745_b300.stotree as S
    monkeypatch.setattr(S, "LIB_PATH", "/nonexistent/libstotree.so")
    monkeypatch.setattr(S, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        S.lib()
