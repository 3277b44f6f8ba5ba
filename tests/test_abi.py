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


def test_warm_create_validates_arguments(libso):
    """stowarm_create refuses bad sizes and trees before touching the device."""
    from paper_2107_01745_b300 import workloads as W
    from paper_2107_01745_b300.stotree import _WarmDesc
    t = W.tree_from_branching([2, 2])
    parent = np.ascontiguousarray(t.parent, dtype=np.int32)
    prob = np.ascontiguousarray(t.prob, dtype=np.float64)
    bad = prob.copy()
    bad[1] = 0.7  # children of the root no longer sum to 1

    def create(**kw):
        a = dict(num_nodes=len(parent), horizon=2, nx=3, nu=2, parent=parent.ctypes.data, prob=prob.ctypes.data,
                 hidden=256, batch=8192, seed=0)
        a.update(kw)
        h = ctypes.c_void_p()
        return libso.stowarm_create(ctypes.byref(_WarmDesc(**a)), ctypes.byref(h))

    # hidden width not a whole number of 128-row tiles; batch outside [256, 65536] or not a
    # multiple of the 256-row weight-gradient split; empty state; 4 nx + 1 features above 256
    for kw in (dict(hidden=192), dict(batch=128), dict(batch=131072), dict(batch=8000), dict(nx=0),
               dict(nx=64, nu=1), dict(parent=None)):
        assert create(**kw) == 1, kw
    assert create(prob=bad.ctypes.data) == 2


def test_batch_create_validates_groups(libso):
    """stobatch_create refuses groups outside the batched engine's shapes before touching the device."""
    from paper_2107_01745_b300.stotree import _GroupDesc
    nx, nu = 4, 2
    arrs = dict(A=np.eye(nx), B=np.ones((nx, nu)), Q=np.ones(nx), R=np.ones(nu), PN=np.ones(nx),
                xlo=-np.ones(nx), xhi=np.ones(nx), ulo=-np.ones(nu), uhi=np.ones(nu))

    def create(n=1, **kw):
        a = dict(horizon=3, branching=2, branch_stages=2, nx=nx, nu=nu, num_instances=2)
        a.update({k: v.ctypes.data for k, v in arrs.items()})
        a.update(kw)
        g = (_GroupDesc * 1)(_GroupDesc(**a))
        h = ctypes.c_void_p()
        return libso.stobatch_create(g, n, ctypes.byref(h))

    # nx <= 64, nu <= 32, horizon in [1, 64], branch_stages <= horizon, instances >= 1, data given
    for kw in (dict(nx=0), dict(nx=65), dict(nu=33), dict(horizon=0), dict(horizon=65), dict(branch_stages=4),
               dict(branching=0), dict(num_instances=0), dict(A=None), dict(uhi=None)):
        assert create(**kw) == 1, kw
    assert create(n=0) == 1


def test_noalloc_refusals_need_no_device(libso):
    """stotree_solve_step_noalloc checks its arguments, its fixed scratch limit and the factor
    before it looks up the scratch array, so these refusals come back on a host without a GPU.
    The limit is the one its declaration states: s, ubar, x and u of one right-hand side
    (each part rounded up to 256 bytes) plus the round's flags must fit 32 MiB.  On a star
    tree (a root with K leaves, nx = 100, nu = 50, FP32) the largest K that fits is accepted
    as far as the factor check, and K + 1 is refused with a message."""
    L = libso
    L.stotree_solve_step_noalloc.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int32] * 2 + [ctypes.c_void_p]
    L.stotree_last_error.argtypes = [ctypes.c_void_p]
    L.stotree_last_error.restype = ctypes.c_char_p
    L.stotree_destroy.argtypes = [ctypes.c_void_p]
    fake = ctypes.c_void_p(4096)  # never dereferenced: each call below is refused first
    nx, nu = 100, 50

    def a256(v):
        return (v + 255) // 256 * 256

    def need(k):
        nn = k + 1
        return a256(4 * nu) + 2 * a256(8 * nn * nx) + a256(8 * nu) + a256(8 * nn) + 256

    kmax = 1
    while need(kmax + 1) <= 32 << 20:
        kmax += 1

    def star(k):
        parent = np.zeros(k + 1, dtype=np.int32)
        parent[0] = -1
        prob = np.full(k + 1, 1.0 / k)
        prob[0] = 1.0
        d = _Desc(k + 1, 1, nx, nu, parent.ctypes.data, prob.ctypes.data)
        h = ctypes.c_void_p()
        assert L.stotree_create(ctypes.byref(d), 1, ctypes.byref(h)) == 0
        return h

    h = star(kmax)
    try:
        assert L.stotree_solve_step_noalloc(None, fake, fake, fake, 0, 0, None) == 1
        assert L.stotree_solve_step_noalloc(h, None, fake, fake, 0, 0, None) == 1
        assert L.stotree_solve_step_noalloc(h, fake, fake, None, 0, 0, None) == 1
        assert L.stotree_solve_step_noalloc(h, fake, None, fake, 0, 0, None) == 1  # x0 needed
        assert L.stotree_solve_step_noalloc(h, fake, None, fake, 1, 0, None) == 3  # not factored
        assert L.stotree_solve_step_noalloc(h, fake, fake, fake, 0, 1, None) == 3
    finally:
        L.stotree_destroy(h)
    h = star(kmax + 1)
    try:
        assert L.stotree_solve_step_noalloc(h, fake, fake, fake, 0, 0, None) == 1
        msg = L.stotree_last_error(h)
        assert b"scratch" in msg and str(need(kmax + 1)).encode() in msg
    finally:
        L.stotree_destroy(h)


_CTYPE_OF = {
    "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
    "size_t": ctypes.c_size_t, "double": ctypes.c_double, "float": ctypes.c_float, "sto_status": ctypes.c_int,
}
_HANDLES = {"stotree_t", "stobatch_t", "stowarm_t", "sto_stream_t"}


def _expected_ctype(ctype: str):
    ctype = ctype.replace("const ", "").strip()
    if ctype.endswith("*") or ctype in _HANDLES:
        return ctypes.c_void_p
    return _CTYPE_OF[ctype]


def test_binding_prototypes_match_the_header():
    """Every entry point declared in include/stotree.h has a ctypes prototype in the binding with
    the same number of arguments, each of the declared width and kind, and the declared result
    type.  Without one, ctypes would pass a 64-bit pointer as a 32-bit int, or a float as a
    double, and the call would read shifted or truncated arguments."""
    from paper_2107_01745_b300 import stotree
    L = stotree.lib()
    src = open(os.path.join(ROOT, "include", "stotree.h")).read()
    decls = re.findall(r"STO_API\s+([^;]*?)\b(sto(?:tree|batch|warm)_\w+)\s*\(([^)]*)\)\s*;", src, re.S)
    assert len(decls) == len(_declared())
    for ret, name, params in decls:
        fn = getattr(L, name)
        params = " ".join(params.split())
        decl = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        want = [_expected_ctype(re.match(r"(.*?)\w+$", p).group(1)) for p in decl]
        assert fn.argtypes is not None, f"{name}: no prototype"
        assert len(fn.argtypes) == len(want), f"{name}: {len(fn.argtypes)} arguments bound, {len(want)} declared"
        for k, (got, exp) in enumerate(zip(fn.argtypes, want)):
            assert got is exp or (exp is ctypes.c_void_p and got is ctypes.c_char_p), f"{name} argument {k}: {got} vs {exp}"
        ret = " ".join(ret.split())
        want_ret = {"void": None, "const char *": ctypes.c_char_p}.get(ret, ctypes.c_int)
        if ret == "sto_status":
            want_ret = ctypes.c_int
        assert fn.restype is want_ret, f"{name}: result {fn.restype} vs {ret}"


def test_wait_limit_and_round_status_refusals_need_no_device(libso):
    """stotree_set_wait_limit accepts 0..60 s and refuses anything else; stotree_round_status
    needs a handle with a bound workspace.  Both answer on a host without a GPU."""
    L = libso
    L.stotree_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_double]
    L.stotree_round_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.stotree_destroy.argtypes = [ctypes.c_void_p]
    parent = np.array([-1, 0, 0], dtype=np.int32)
    prob = np.array([1.0, 0.5, 0.5])
    d = _Desc(3, 1, 2, 1, parent.ctypes.data, prob.ctypes.data)
    h = ctypes.c_void_p()
    assert L.stotree_create(ctypes.byref(d), 1, ctypes.byref(h)) == 0
    try:
        for bad in (-1e-9, 60.5, float("nan"), float("inf")):
            assert L.stotree_set_wait_limit(h, bad) == 1, bad
        for ok in (0.0, 1e-6, 1.5, 60.0):
            assert L.stotree_set_wait_limit(h, ok) == 0, ok
        assert L.stotree_set_wait_limit(None, 1.0) == 1
        assert L.stotree_round_status(None, None) == 1
        assert L.stotree_round_status(h, None) == 3  # no workspace bound
    finally:
        L.stotree_destroy(h)


def test_set_dynamics_argument_checks_need_no_device(libso):
    """stotree_set_dynamics: c is required, A and B are given together or both NULL (NULL keeps
    the nodes' matrices and is refused for nodes that have none), the node range must lie in the
    tree; the checks answer before any device work (no workspace bound here: NOT_READY)."""
    L = libso
    vp = ctypes.c_void_p
    L.stotree_set_dynamics.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp]
    L.stotree_destroy.argtypes = [vp]
    parent = np.array([-1, 0, 0], dtype=np.int32)
    prob = np.array([1.0, 0.5, 0.5])
    d = _Desc(3, 1, 2, 1, parent.ctypes.data, prob.ctypes.data)
    h = ctypes.c_void_p()
    assert L.stotree_create(ctypes.byref(d), 1, ctypes.byref(h)) == 0
    A = np.zeros((3, 2, 2))
    B = np.zeros((3, 2, 1))
    c = np.zeros((3, 2))
    p = lambda a: a.ctypes.data
    try:
        assert L.stotree_set_dynamics(h, 0, 3, p(A), p(B), None, None) == 1   # no c
        assert L.stotree_set_dynamics(h, 0, 3, p(A), None, p(c), None) == 1   # B without A
        assert L.stotree_set_dynamics(h, 0, 3, None, p(B), p(c), None) == 1   # A without B
        assert L.stotree_set_dynamics(h, 1, 3, p(A), p(B), p(c), None) == 1   # past the last node
        assert L.stotree_set_dynamics(h, 0, 0, p(A), p(B), p(c), None) == 1   # empty range
        assert L.stotree_set_dynamics(h, 0, 3, p(A), p(B), p(c), None) == 3   # no workspace yet
        assert L.stotree_set_dynamics(h, 0, 3, None, None, p(c), None) == 3
    finally:
        L.stotree_destroy(h)
