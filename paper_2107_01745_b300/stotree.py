"""Python binding of libstotree (argument marshalling only).

Every function mirrors an entry point of ``include/stotree.h``; torch is used for device
memory and streams, and every computation runs in the library's CUDA kernels.  Loading
fails loudly when ``libstotree.so`` has not been built
(``python -m paper_2107_01745_b300.build``): there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstotree.so")

STO_FP64, STO_FP32 = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "invalid scenario tree", 3: "not ready", 4: "numerical failure",
          5: "CUDA error", 6: "timeout", 7: "not converged", 8: "workspace too small"}
STO_NOT_CONVERGED = 7


class StoError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}" + (f" ({detail})" if detail else ""))


class _TreeDesc(ctypes.Structure):
    _fields_ = [("num_nodes", ctypes.c_int32), ("horizon", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("nu", ctypes.c_int32), ("parent", ctypes.c_void_p), ("prob", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("tol", ctypes.c_double), ("eps_curv", ctypes.c_double),
                ("lbfgs_mem", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("max_ls", ctypes.c_int32),
                ("backtrack", ctypes.c_int32), ("bt_param", ctypes.c_double), ("max_halvings", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("solve_calls", ctypes.c_int32), ("status", ctypes.c_int32),
                ("ls_zero", ctypes.c_int32), ("launches", ctypes.c_int32), ("halvings", ctypes.c_int32),
                ("res_inf", ctypes.c_double), ("fbe", ctypes.c_double),
                ("ms", ctypes.c_double), ("lambda_", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_2107_01745_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, dbl, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
        sigs = {
            "stotree_create": [vp, i32, vp],
            "stotree_sizes": [vp, vp, vp, vp, vp],
            "stotree_workspace_size": [vp, vp],
            "stotree_bind_workspace": [vp, vp, sz, vp],
            "stotree_set_dynamics": [vp, i32, i32, vp, vp, vp, vp],
            "stotree_set_costs": [vp, vp, vp, vp, vp, vp, vp, vp],
            "stotree_set_box": [vp, vp, vp, vp, vp, vp],
            "stotree_set_penalty": [vp, vp, vp, vp, vp],
            "stotree_factor": [vp, i32, vp],
            "stotree_solve_step": [vp, vp, vp, vp, i32, i32, i32, vp],
            "stotree_solve_step_noalloc": [vp, vp, vp, vp, i32, i32, vp],
            "stotree_last_primal": [vp, vp, vp, vp],
            "stotree_set_wait_limit": [vp, dbl],
            "stotree_set_constraint_maps": [vp, i32, i32, vp, vp, vp],
            "stotree_set_zbox": [vp, vp, vp, vp, vp, vp],
            "stotree_round_status": [vp, vp],
            "stotree_estimate_lambda": [vp, vp, i32, dbl, vp, vp, vp],
            "stotree_nama_solve": [vp, vp, vp, vp, vp, vp, vp, vp, vp],
            "stotree_minfbe_solve": [vp, vp, vp, vp, vp, vp, vp, vp, vp],
            "stotree_gpad_solve": [vp, vp, vp, vp, vp, vp, vp, vp, vp],
            "stotree_kkt_check": [vp, vp, vp, vp, vp, dbl, vp, vp],
            "stotree_set_timing": [vp, i32],
            "stotree_get_timing": [vp, vp, vp, vp],
            "stotree_solve_bytes": [vp, vp, vp],
        }
        for name, args in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.stotree_destroy.argtypes = [vp]
        L.stotree_destroy.restype = None
        L.stotree_last_error.argtypes = [vp]
        L.stotree_last_error.restype = ctypes.c_char_p
        L.stotree_status_str.argtypes = [ctypes.c_int]
        L.stotree_status_str.restype = ctypes.c_char_p
        bsigs = {
            "stobatch_create": [vp, i32, vp],
            "stobatch_sizes": [vp, vp, vp, vp, vp],
            "stobatch_workspace_size": [vp, vp],
            "stobatch_bind_workspace": [vp, vp, sz, vp],
            "stobatch_set_instance": [vp, i32, i32, vp, vp, vp],
            "stobatch_factor": [vp, vp],
            "stobatch_solve_step": [vp, vp, vp, i32, i32, vp],
            "stobatch_nama_solve": [vp, vp, vp, vp, vp, vp, vp, vp],
            "stobatch_round_status": [vp, vp],
            "stobatch_round_config": [vp, i32, vp, vp, vp, vp],
            "stobatch_set_round_variant": [vp, i32, i32],
        }
        for name, args in bsigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.stobatch_destroy.argtypes = [vp]
        L.stobatch_destroy.restype = None
        L.stobatch_last_error.argtypes = [vp]
        L.stobatch_last_error.restype = ctypes.c_char_p
        i64, f32, u64 = ctypes.c_int64, ctypes.c_float, ctypes.c_uint64
        wsigs = {
            "stowarm_create": [vp, vp],
            "stowarm_dims": [vp, vp, vp, vp],
            "stowarm_workspace_size": [vp, vp],
            "stowarm_bind_workspace": [vp, vp, sz, vp],
            "stowarm_set_params": [vp, vp, vp],
            "stowarm_get_params": [vp, vp, vp],
            "stowarm_forward": [vp, vp, i32, vp, vp],
            "stowarm_gradients": [vp, vp, vp, vp, i32, vp, vp, vp],
            "stowarm_train_batch": [vp, vp, vp, vp, i32, f32, vp],
            "stowarm_set_draws": [vp, i32, vp, vp, vp],
            "stowarm_train": [vp, i32, f32, u64, vp, vp],
            "stowarm_predict": [vp, i32, i32, vp, vp],
            "stowarm_gemm_bf16": [vp, i64, vp, i64, vp, i64, i32, i32, i32, vp],
        }
        for name, args in wsigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.stowarm_destroy.argtypes = [vp]
        L.stowarm_destroy.restype = None
        L.stowarm_last_error.argtypes = [vp]
        L.stowarm_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def exported_symbols():
    return [n for n in ("stotree_create", "stotree_destroy", "stotree_set_constraint_maps", "stotree_set_zbox",
                        "stotree_sizes", "stotree_workspace_size",
                        "stotree_bind_workspace", "stotree_set_dynamics", "stotree_set_costs", "stotree_set_box", "stotree_set_penalty",
                        "stotree_factor", "stotree_solve_step", "stotree_solve_step_noalloc", "stotree_set_wait_limit",
                        "stotree_round_status", "stotree_last_primal", "stotree_estimate_lambda",
                        "stotree_nama_solve", "stotree_minfbe_solve", "stotree_gpad_solve", "stotree_kkt_check", "stotree_set_timing",
                        "stotree_get_timing", "stotree_solve_bytes", "stotree_status_str", "stotree_last_error",
                        "stobatch_create", "stobatch_destroy", "stobatch_sizes", "stobatch_workspace_size",
                        "stobatch_bind_workspace", "stobatch_set_instance", "stobatch_factor",
                        "stobatch_solve_step", "stobatch_nama_solve", "stobatch_round_status",
                        "stobatch_round_config", "stobatch_set_round_variant", "stobatch_last_error",
                        "stowarm_create", "stowarm_destroy", "stowarm_dims", "stowarm_workspace_size",
                        "stowarm_bind_workspace", "stowarm_set_params", "stowarm_get_params", "stowarm_forward",
                        "stowarm_gradients", "stowarm_train_batch", "stowarm_set_draws", "stowarm_train",
                        "stowarm_predict", "stowarm_gemm_bf16", "stowarm_last_error")]


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _t_ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class StoTree:
    """One scenario-tree problem on one GPU: handle, workspace and data."""

    def __init__(self, problem, precision: str = "fp32", device="cuda:0", chunk_nodes: int = 2048):
        self.device = torch.device(device)
        self.p = problem
        self.prec = STO_FP32 if precision == "fp32" else STO_FP64
        self.dtype = torch.float32 if self.prec == STO_FP32 else torch.float64
        t = problem.tree
        L = lib()
        self._parent = np.ascontiguousarray(t.parent, dtype=np.int32)
        self._prob = np.ascontiguousarray(t.prob, dtype=np.float64)
        desc = _TreeDesc(t.num_nodes, t.horizon, problem.nx, problem.nu, _np_ptr(self._parent), _np_ptr(self._prob))
        h = ctypes.c_void_p()
        self._check(L.stotree_create(ctypes.byref(desc), self.prec, ctypes.byref(h)), "stotree_create", handle=False)
        self.h = h
        self.general = bool(getattr(problem, "general", False))
        if self.general:  # general constraint maps: before the sizes and the workspace
            self._maps = [np.ascontiguousarray(a, dtype=np.float64) for a in (problem.F, problem.G, problem.FN)]
            self._check(L.stotree_set_constraint_maps(h, problem.F.shape[0], problem.FN.shape[0],
                                                      *[_np_ptr(a) for a in self._maps]), "set_constraint_maps")
        m, n = ctypes.c_int64(), ctypes.c_int64()
        npl, nl = ctypes.c_int32(), ctypes.c_int32()
        L.stotree_sizes(h, ctypes.byref(m), ctypes.byref(n), ctypes.byref(npl), ctypes.byref(nl))
        self.m, self.n, self.Np, self.Nl = m.value, n.value, npl.value, nl.value
        self.Nn, self.nx, self.nu = t.num_nodes, problem.nx, problem.nu
        wb = ctypes.c_size_t()
        L.stotree_workspace_size(h, ctypes.byref(wb))
        self.workspace_bytes = wb.value
        with torch.cuda.device(self.device):
            self.ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            st = _stream()
            self._check(L.stotree_bind_workspace(h, _t_ptr(self.ws), self.workspace_bytes, st), "bind_workspace")
            self._chunk = chunk_nodes
            self.set_dynamics(problem.A, problem.B, problem.c)
            self.set_costs(problem.Q, problem.R, problem.PN, problem.q, problem.r, problem.pN)
            if self.general:
                self.set_zbox(problem.zlo, problem.zhi, problem.zNlo, problem.zNhi)
            else:
                self.set_box(problem.xlo, problem.xhi, problem.ulo, problem.uhi)
            if getattr(problem, "pen_kind", None) is not None:
                self.set_penalty(problem.pen_kind, problem.pen_rho, problem.pen_delta)

    # -- plumbing -------------------------------------------------------------------------
    def _check(self, code, where, handle=True):
        if code != 0:
            detail = ""
            if handle and getattr(self, "h", None):
                detail = lib().stotree_last_error(self.h).decode()
            raise StoError(code, where, detail)

    def close(self):
        if getattr(self, "h", None):
            lib().stotree_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self, nrhs=1):
        return torch.zeros((nrhs, self.m) if nrhs > 1 else (self.m,), dtype=self.dtype, device=self.device)

    def to_dev(self, a):
        return torch.as_tensor(np.asarray(a), dtype=self.dtype).to(self.device).contiguous()

    # -- set-up ---------------------------------------------------------------------------
    def set_dynamics(self, A, B, c):
        """stotree_set_dynamics for every node, in chunks (A [Nn][nx][nx], B [Nn][nx][nu],
        c [Nn][nx]; A = B = None keeps the matrices and replaces the disturbances); the handle
        needs stotree_factor again before its next solve."""
        nn = self.p.tree.num_nodes
        for f in range(0, nn, self._chunk):
            n = min(self._chunk, nn - f)
            Af = None if A is None else np.ascontiguousarray(A[f:f + n], dtype=np.float64)
            Bf = None if B is None else np.ascontiguousarray(B[f:f + n], dtype=np.float64)
            cf = np.ascontiguousarray(c[f:f + n], dtype=np.float64)
            self._check(lib().stotree_set_dynamics(self.h, f, n, _np_ptr(Af) if Af is not None else None,
                                                   _np_ptr(Bf) if Bf is not None else None, _np_ptr(cf), _stream()),
                        "set_dynamics")

    def set_costs(self, Q, R, PN, q=None, r=None, pN=None):
        arr = [np.ascontiguousarray(v, dtype=np.float64) if v is not None else None for v in (Q, R, PN, q, r, pN)]
        self._keep_cost = arr
        ptrs = [_np_ptr(a) if a is not None else None for a in arr]
        self._check(lib().stotree_set_costs(self.h, *ptrs, _stream()), "set_costs")

    def set_penalty(self, kind, rho, delta):
        """Per-component kind of g (0 box, 1 rho dist, 2 rho Huber(dist)), see stotree_set_penalty."""
        n = self.nx + self.nu
        k = np.ascontiguousarray(np.broadcast_to(np.asarray(kind, dtype=np.int32), (n,)))
        r = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, dtype=np.float64), (n,)))
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(delta, dtype=np.float64), (n,)))
        self._check(lib().stotree_set_penalty(self.h, k.ctypes.data_as(ctypes.c_void_p), _np_ptr(r), _np_ptr(d),
                                              _stream()), "set_penalty")

    def set_zbox(self, zlo, zhi, zNlo, zNhi):
        """stotree_set_zbox: the box on z of the general constraint maps."""
        arr = [np.ascontiguousarray(v, dtype=np.float64) for v in (zlo, zhi, zNlo, zNhi)]
        self._check(lib().stotree_set_zbox(self.h, *[_np_ptr(a) for a in arr], _stream()), "set_zbox")

    def set_box(self, xlo, xhi, ulo, uhi):
        arr = [np.ascontiguousarray(v, dtype=np.float64) for v in (xlo, xhi, ulo, uhi)]
        self._check(lib().stotree_set_box(self.h, *[_np_ptr(a) for a in arr], _stream()), "set_box")

    def factor(self, sync=True):
        self._check(lib().stotree_factor(self.h, 1 if sync else 0, _stream()), "factor")

    # -- hot path -------------------------------------------------------------------------
    def solve_step(self, y, x0=None, homogeneous=False, scaled=False, out=None):
        """Algorithm 3 (or 4): y [m] or [nrhs, m] device tensor -> Hx of the same shape."""
        y = y.contiguous()
        nrhs = 1 if y.dim() == 1 else y.shape[0]
        out = torch.empty_like(y) if out is None else out
        x0 = x0 if x0 is not None else (None if homogeneous else self.to_dev(self.p.x0))
        self._check(lib().stotree_solve_step(self.h, _t_ptr(y), _t_ptr(x0), _t_ptr(out), nrhs,
                                             1 if homogeneous else 0, 1 if scaled else 0, _stream()), "solve_step")
        return out

    def solve_step_noalloc(self, y, x0=None, homogeneous=False, scaled=False, out=None):
        """stotree_solve_step_noalloc: one right-hand side, scratch in the library's static array."""
        y = y.contiguous()
        out = torch.empty_like(y) if out is None else out
        x0 = x0 if x0 is not None else (None if homogeneous else self.to_dev(self.p.x0))
        self._check(lib().stotree_solve_step_noalloc(self.h, _t_ptr(y), _t_ptr(x0), _t_ptr(out),
                                                     1 if homogeneous else 0, 1 if scaled else 0, _stream()),
                    "solve_step_noalloc")
        return out

    def set_wait_limit(self, seconds):
        """stotree_set_wait_limit: limit of each dependency wait inside a solve round."""
        self._check(lib().stotree_set_wait_limit(self.h, float(seconds)), "set_wait_limit")

    def round_status(self):
        """stotree_round_status: raises StoError (timeout) if a wait of the rounds since the last
        synchronising call gave up."""
        self._check(lib().stotree_round_status(self.h, _stream()), "round_status")

    def last_primal(self):
        x = torch.empty((self.Nn, self.nx), dtype=self.dtype, device=self.device)
        u = torch.empty((self.Np, self.nu), dtype=self.dtype, device=self.device)
        self._check(lib().stotree_last_primal(self.h, _t_ptr(x), _t_ptr(u), _stream()), "last_primal")
        return x, u

    def estimate_lambda(self, r0, iters=50, safety=0.9):
        r = r0.clone().contiguous()
        lam, L = ctypes.c_double(), ctypes.c_double()
        self._check(lib().stotree_estimate_lambda(self.h, _t_ptr(r), iters, safety, ctypes.byref(lam),
                                                  ctypes.byref(L), _stream()), "estimate_lambda")
        return lam.value, L.value

    def solve(self, method, lam, x0=None, y0=None, tol=1e-4, mem=5, max_iter=1000, max_ls=30, eps_curv=None,
              outputs=True, allow_not_converged=False, backtrack=None, bt_param=None, max_halvings=60):
        """Algorithm 1 (method='minfbe'), 2 (method='nama') or GPAD (method='gpad', the
        accelerated dual projected gradient of Sections III-F and IV).  Returns tensors and info.

        backtrack (Algorithms 1 and 2): None (fixed lambda), 'original' (eq. original-backtracking,
        bt_param = beta, default 0) or 'simple' (eq. simple-backtracking, bt_param = eps'',
        default 0.25); the info dict then reports the final 'lambda_' and the 'halvings'."""
        if eps_curv is None:
            eps_curv = 1e-12 if self.prec == STO_FP64 else 1e-8
        x0 = self.to_dev(self.p.x0) if x0 is None else x0
        y = self.vec() if y0 is None else y0.clone().contiguous()
        x = torch.empty((self.Nn, self.nx), dtype=self.dtype, device=self.device) if outputs else None
        u = torch.empty((self.Np, self.nu), dtype=self.dtype, device=self.device) if outputs else None
        z = torch.empty(self.m, dtype=self.dtype, device=self.device) if outputs else None
        bt_code = {None: 0, "original": 1, "simple": 2}[backtrack]
        if bt_param is None:
            bt_param = 0.25 if backtrack == "simple" else 0.0
        o = Opts(lam, tol, eps_curv, mem, max_iter, max_ls, bt_code, bt_param, max_halvings, 0)
        info = Info()
        fn = {"nama": lib().stotree_nama_solve, "minfbe": lib().stotree_minfbe_solve,
              "gpad": lib().stotree_gpad_solve}[method]
        code = fn(self.h, ctypes.byref(o), _t_ptr(x0), _t_ptr(y), _t_ptr(x), _t_ptr(u), _t_ptr(z),
                  ctypes.byref(info), _stream())
        if code != 0 and not (allow_not_converged and code == STO_NOT_CONVERGED):
            self._check(code, method)
        return dict(y=y, x=x, u=u, z=z, info=info.as_dict())

    def kkt_check(self, x0, x, u, y, tol_active=1e-6):
        out = (ctypes.c_double * 6)()
        self._check(lib().stotree_kkt_check(self.h, _t_ptr(x0), _t_ptr(x), _t_ptr(u), _t_ptr(y), tol_active, out,
                                            _stream()), "kkt_check")
        return dict(dynamics=out[0], stationarity=out[1], feasibility=out[2], complementarity=out[3],
                    sign=out[4], gap=out[5])

    # -- measurement ----------------------------------------------------------------------
    def set_timing(self, on=True):
        self._check(lib().stotree_set_timing(self.h, 1 if on else 0), "set_timing")

    def get_timing(self):
        ms, n, rhs = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        self._check(lib().stotree_get_timing(self.h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(rhs)),
                    "get_timing")
        return ms.value, n.value, rhs.value

    def solve_bytes(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        lib().stotree_solve_bytes(self.h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value


class _GroupDesc(ctypes.Structure):
    _fields_ = [("horizon", ctypes.c_int32), ("branching", ctypes.c_int32), ("branch_stages", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("nu", ctypes.c_int32), ("num_instances", ctypes.c_int32),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("PN", ctypes.c_void_p), ("xlo", ctypes.c_void_p), ("xhi", ctypes.c_void_p), ("ulo", ctypes.c_void_p),
                ("uhi", ctypes.c_void_p)]


class StoBatch:
    """Many instances in shape groups (workloads.Group) solved together on one GPU."""

    def __init__(self, groups, device="cuda:0"):
        self.device = torch.device(device)
        self.groups = groups
        L = lib()
        self._keep = []
        descs = (_GroupDesc * len(groups))()
        for k, g in enumerate(groups):
            arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (g.A, g.B, g.Q, g.R, g.PN, g.xlo, g.xhi,
                                                                        g.ulo, g.uhi)]
            self._keep.append(arrs)
            descs[k] = _GroupDesc(g.horizon, g.branching, g.branch_stages, g.nx, g.nu, g.num_instances,
                                  *[_np_ptr(a) for a in arrs])
        h = ctypes.c_void_p()
        code = L.stobatch_create(descs, len(groups), ctypes.byref(h))
        if code != 0:
            raise StoError(code, "stobatch_create")
        self.h = h
        M, n = ctypes.c_int64(), ctypes.c_int32()
        L.stobatch_sizes(h, ctypes.byref(M), ctypes.byref(n), None, None)
        self.M, self.ninst = M.value, n.value
        offs = np.zeros(self.ninst, dtype=np.int64)
        sizes = np.zeros(self.ninst, dtype=np.int64)
        L.stobatch_sizes(h, None, None, _np_ptr(offs), _np_ptr(sizes))
        self.offsets, self.sizes = offs, sizes
        wb = ctypes.c_size_t()
        L.stobatch_workspace_size(h, ctypes.byref(wb))
        self.workspace_bytes = wb.value
        with torch.cuda.device(self.device):
            self.ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            self._check(L.stobatch_bind_workspace(h, _t_ptr(self.ws), self.workspace_bytes, _stream()), "bind")
            for gi, g in enumerate(groups):
                for k in range(g.num_instances):
                    x0 = np.ascontiguousarray(g.x0[k], dtype=np.float64)
                    c = np.ascontiguousarray(g.c[k], dtype=np.float64)
                    self._check(L.stobatch_set_instance(h, gi, k, _np_ptr(x0), _np_ptr(c), _stream()),
                                "set_instance")

    def _check(self, code, where):
        if code != 0:
            raise StoError(code, where, lib().stobatch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().stobatch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factor(self):
        self._check(lib().stobatch_factor(self.h, _stream()), "factor")

    def vec(self):
        return torch.zeros(self.M, dtype=torch.float32, device=self.device)

    def split(self, v):
        """Per-instance views of a batch vector."""
        return [v[o:o + n] for o, n in zip(self.offsets, self.sizes)]

    def pack(self, per_instance):
        return torch.cat([torch.as_tensor(np.asarray(a), dtype=torch.float32) for a in per_instance]).to(self.device)

    def solve_step(self, y, homogeneous=False, scaled=False):
        out = torch.empty_like(y)
        self._check(lib().stobatch_solve_step(self.h, _t_ptr(y), _t_ptr(out), 1 if homogeneous else 0,
                                              1 if scaled else 0, _stream()), "solve_step")
        return out

    def nama(self, lambdas, tol=1e-4, mem=5, max_iter=500, max_ls=30, eps_curv=1e-8, y0=None, outputs=True,
             allow_not_converged=False):
        y = self.vec() if y0 is None else y0.clone().contiguous()
        z = self.vec() if outputs else None
        hx = self.vec() if outputs else None
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        o = Opts(0.0, tol, eps_curv, mem, max_iter, max_ls)
        infos = (Info * self.ninst)()
        code = lib().stobatch_nama_solve(self.h, ctypes.byref(o), _np_ptr(lam), _t_ptr(y), _t_ptr(z), _t_ptr(hx),
                                         infos, _stream())
        if code != 0 and not (allow_not_converged and code == STO_NOT_CONVERGED):
            self._check(code, "nama")
        return dict(y=y, z=z, hx=hx, infos=[i.as_dict() for i in infos])

    def round_status(self):
        """stobatch_round_status: raises StoError (timeout) if a wait of the rounds since the last
        synchronising call gave up."""
        self._check(lib().stobatch_round_status(self.h, _stream()), "round_status")

    def round_config(self, nrhs=1):
        """stobatch_round_config: the tuned tile (columns, CTA threads), the persistent launch's
        CTAs and the tuner's measured round time per candidate (-1: not applicable)."""
        tc, nt, ctas = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ms = (ctypes.c_double * 4)()
        self._check(lib().stobatch_round_config(self.h, nrhs, ctypes.byref(tc), ctypes.byref(nt), ctypes.byref(ctas),
                                                ms), "round_config")
        return dict(tile_cols=tc.value, cta_threads=nt.value, ctas=ctas.value,
                    tuned_ms={"tile32x128": ms[0], "tile32x256": ms[1], "tile64x256": ms[2], "column128": ms[3]})

    def set_round_variant(self, nrhs, variant):
        """stobatch_set_round_variant: fix the round kernel variant (0-3) instead of the tuner's."""
        self._check(lib().stobatch_set_round_variant(self.h, nrhs, variant), "set_round_variant")

    def group_lambdas(self, iters=50, safety=0.9, seed=7):
        """lambda per group from the single-instance power iteration on the group's first instance
        (the dual Hessian does not depend on x0 or c)."""
        out = []
        for g in self.groups:
            st = StoTree(g.instance(0), precision="fp32", device=self.device)
            st.factor()
            r0 = torch.as_tensor(np.random.default_rng(seed).standard_normal(st.m), dtype=torch.float32,
                                 device=self.device)
            out.append(st.estimate_lambda(r0, iters=iters, safety=safety)[0])
            st.close()
        return np.array(out)


class _WarmDesc(ctypes.Structure):
    _fields_ = [("num_nodes", ctypes.c_int32), ("horizon", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("nu", ctypes.c_int32), ("parent", ctypes.c_void_p), ("prob", ctypes.c_void_p),
                ("hidden", ctypes.c_int32), ("batch", ctypes.c_int32), ("seed", ctypes.c_uint64)]


def gemm_bf16(A, B):
    """C = A B' on the tensor cores: A [M, K], B [N, K] BF16 CUDA tensors -> FP32 [M, N]."""
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty(M, N, dtype=torch.float32, device=A.device)
    code = lib().stowarm_gemm_bf16(_t_ptr(A), A.stride(0), _t_ptr(B), B.stride(0), _t_ptr(C), C.stride(0), M, N, K,
                                   _stream())
    if code != 0:
        raise StoError(code, "stowarm_gemm_bf16")
    return C


class StoWarm:
    """Learned warm start (per-node perceptron on the tensor cores) for problems on one tree."""

    def __init__(self, tree, nx, nu, hidden=256, batch=8192, seed=0, device="cuda:0"):
        self.device = torch.device(device)
        self.tree = tree
        parent = np.ascontiguousarray(tree.parent, dtype=np.int32)
        prob = np.ascontiguousarray(tree.prob, dtype=np.float64)
        st = np.zeros(len(parent), dtype=np.int64)
        for i in range(1, len(parent)):
            st[i] = st[parent[i]] + 1
        horizon = int(st.max())
        nonleaf = np.zeros(len(parent), dtype=bool)
        nonleaf[parent[1:]] = True
        self.m = int(nonleaf.sum()) * (nx + nu) + int((~nonleaf).sum()) * nx
        d = _WarmDesc(len(parent), horizon, nx, nu, parent.ctypes.data, prob.ctypes.data, hidden, batch, seed)
        h = ctypes.c_void_p()
        L = lib()
        code = L.stowarm_create(ctypes.byref(d), ctypes.byref(h))
        if code != 0:
            raise StoError(code, "stowarm_create")
        self.h = h
        di, do, npar = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        L.stowarm_dims(h, ctypes.byref(di), ctypes.byref(do), ctypes.byref(npar))
        self.d_in, self.d_out, self.num_params = di.value, do.value, npar.value
        self.nx, self.nu, self.hidden, self.batch = nx, nu, hidden, batch
        wb = ctypes.c_size_t()
        L.stowarm_workspace_size(h, ctypes.byref(wb))
        with torch.cuda.device(self.device):
            self._raw = torch.empty(wb.value + 1024, dtype=torch.uint8, device=self.device)
            off = (-self._raw.data_ptr()) % 1024
            self.ws = self._raw[off:off + wb.value]
            self._check(L.stowarm_bind_workspace(h, _t_ptr(self.ws), wb.value, _stream()), "bind")
        self._draws = None

    def _check(self, code, where):
        if code != 0:
            raise StoError(code, where, lib().stowarm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().stowarm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        p = np.empty(self.num_params, dtype=np.float32)
        self._check(lib().stowarm_get_params(self.h, _np_ptr(p), _stream()), "get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.num_params
        self._check(lib().stowarm_set_params(self.h, _np_ptr(p), _stream()), "set_params")

    def unflatten(self, p):
        """Parameter vector -> dict in the oracle's shapes."""
        H, di, do = self.hidden, self.d_in, self.d_out
        out, k = {}, 0
        for name, shape in (("W1", (H, di)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (do, H)),
                            ("b3", (do,))):
            n = int(np.prod(shape))
            out[name] = np.asarray(p[k:k + n]).reshape(shape)
            k += n
        return out

    @staticmethod
    def flatten(d):
        return np.concatenate([np.ravel(d[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])

    def forward(self, X):
        X = X.contiguous().float()
        Y = torch.empty(X.shape[0], self.d_out, dtype=torch.float32, device=self.device)
        self._check(lib().stowarm_forward(self.h, _t_ptr(X), X.shape[0], _t_ptr(Y), _stream()), "forward")
        return Y

    def gradients(self, X, T, nvalid):
        X, T = X.contiguous().float(), T.contiguous().float()
        nv = nvalid.contiguous().to(torch.int32)
        g = torch.empty(self.num_params, dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        self._check(lib().stowarm_gradients(self.h, _t_ptr(X), _t_ptr(T), _t_ptr(nv), X.shape[0], _t_ptr(g),
                                            _t_ptr(loss), _stream()), "gradients")
        return g, float(loss.item())

    def train_batch(self, X, T, nvalid, lr=1e-3):
        X, T = X.contiguous().float(), T.contiguous().float()
        nv = nvalid.contiguous().to(torch.int32)
        self._check(lib().stowarm_train_batch(self.h, _t_ptr(X), _t_ptr(T), _t_ptr(nv), X.shape[0], lr, _stream()),
                    "train_batch")

    def set_draws(self, x0, c, y=None):
        """x0 [D, nx], c [D, Nn, nx], y [D, m] (unscaled duals) FP32 device tensors (kept alive here)."""
        self._draws = (x0.contiguous().float(), c.contiguous().float(), None if y is None else y.contiguous().float())
        x0, c, y = self._draws
        self._check(lib().stowarm_set_draws(self.h, x0.shape[0], _t_ptr(x0), _t_ptr(c), _t_ptr(y)), "set_draws")

    def train(self, steps, lr=1e-3, seed=0):
        hist = torch.empty(max(steps, 1), dtype=torch.float32, device=self.device)
        self._check(lib().stowarm_train(self.h, steps, lr, seed, _t_ptr(hist), _stream()), "train")
        return hist[:steps]

    def predict(self, draw0, num_draws, out=None):
        """Predicted unscaled duals of draws [draw0, draw0 + num_draws) as [num_draws, m]."""
        if out is None:
            out = torch.zeros(num_draws, self.m, dtype=torch.float32, device=self.device)
        self._check(lib().stowarm_predict(self.h, draw0, num_draws, _t_ptr(out), _stream()), "predict")
        return out
