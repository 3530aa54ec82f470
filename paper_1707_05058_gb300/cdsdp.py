"""ctypes binding of the C ABI in include/cdsdp.h (argument marshalling only).

Every step of the solver runs inside libcdsdp.so: the host preprocessing in
its C++ setup code and every iteration in its CUDA kernels.  This module only
converts arrays, allocates the device workspace through PyTorch and passes
pointers and the current CUDA stream.  Importing it fails loudly when the
library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcdsdp.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libcdsdp.so is not built ({LIB_PATH}); run __graft_entry__.build() first")

_lib = ctypes.CDLL(LIB_PATH)

PRIMAL, DUAL, HSDE = 0, 1, 2
FORMS = {"primal": PRIMAL, "dual": DUAL, "hsde": HSDE}
FP32, FP64 = 0, 1
SOLVED, MAX_ITER, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, NOT_PD = 0, 1, 2, 3, 4

_i32p = ctypes.POINTER(ctypes.c_int)
_f64p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_ll = ctypes.c_longlong


class Opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_iter", ctypes.c_int), ("rho", ctypes.c_double),
                ("precision", ctypes.c_int), ("use_graph", ctypes.c_int), ("check_every", ctypes.c_int),
                ("jacobi_max_sweeps", ctypes.c_int), ("warm_start", ctypes.c_int), ("profile", ctypes.c_int),
                ("component_stop", ctypes.c_int), ("adaptive_rho", ctypes.c_int), ("rho_mu", ctypes.c_double),
                ("rho_nu", ctypes.c_double), ("x_update", ctypes.c_int), ("proj_warps_div", ctypes.c_int),
                ("linear_solver", ctypes.c_int), ("cg_tol", ctypes.c_double), ("cg_max_steps", ctypes.c_int),
                ("proj_streams", ctypes.c_int), ("proj_cta_kernel", ctypes.c_int),
                ("row_threads", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("p", ctypes.c_int), ("max_clique", ctypes.c_int),
                ("nnz_pattern", _ll), ("n_d_lower", _ll), ("nnz_A", _ll), ("n_fill", _ll),
                ("chordal", ctypes.c_int), ("diag_factor", ctypes.c_int), ("upload_bytes", _ll),
                ("ncomp", ctypes.c_int), ("cached_factor", ctypes.c_int)]


_lib.cdsdp_default_opts.argtypes = [ctypes.POINTER(Opts)]
_lib.cdsdp_default_opts.restype = None
_lib.cdsdp_setup.argtypes = [ctypes.c_int, ctypes.c_int, _ll, _i32p, _i32p, _i32p, _f64p, _f64p,
                             _ll, _i32p, _i32p, _f64p, _ll, _i32p, _i32p, ctypes.POINTER(_vp)]
_lib.cdsdp_setup_scaled.argtypes = [ctypes.c_int, ctypes.c_int, _ll, _i32p, _i32p, _i32p, _f64p, _f64p,
                                    _ll, _i32p, _i32p, _f64p, _ll, _i32p, _i32p, ctypes.c_int, ctypes.POINTER(_vp)]
_lib.cdsdp_scaling.argtypes = [_vp, _f64p, _f64p, _f64p, _f64p]
_lib.cdsdp_scaling_batch.argtypes = [_vp, _i32p, _f64p, _f64p]
_lib.cdsdp_setup_flags.argtypes = [ctypes.c_int, ctypes.c_int, _ll, _i32p, _i32p, _i32p, _f64p, _f64p,
                                   _ll, _i32p, _i32p, _f64p, _ll, _i32p, _i32p, ctypes.c_int, ctypes.c_uint,
                                   ctypes.POINTER(_vp)]
SETUP_NO_FACTOR = 1
SETUP_MERGE_CLIQUES = 2
_lib.cdsdp_completion_sizes.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_ll), _vp]
_lib.cdsdp_complete.argtypes = [_vp, _vp, _vp, ctypes.c_size_t, _vp, _f64p, _vp]
_lib.cdsdp_setup_batch.argtypes = [ctypes.c_int, _i32p, _i32p, ctypes.POINTER(_ll), _i32p, _i32p, _i32p, _f64p,
                                   _f64p, ctypes.POINTER(_ll), _i32p, _i32p, _f64p, ctypes.POINTER(_ll), _i32p, _i32p,
                                   ctypes.c_int, ctypes.c_uint, ctypes.POINTER(_vp)]
_lib.cdsdp_info.argtypes = [_vp, ctypes.POINTER(Info)]
_lib.cdsdp_cliques.argtypes = [_vp, _i32p, _i32p]
_lib.cdsdp_pattern.argtypes = [_vp, _i32p, _i32p]
_lib.cdsdp_components.argtypes = [_vp, _i32p, _i32p]
_lib.cdsdp_component_results.argtypes = [_vp, _vp, _i32p, _i32p, _f64p]
_lib.cdsdp_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(Opts), ctypes.c_int, _vp, ctypes.POINTER(Opts),
                               _f64p, _i32p]
_lib.cdsdp_workspace_bytes.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
_lib.cdsdp_bind.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.c_int, _vp]
_lib.cdsdp_solve.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(Opts), _vp, _f64p, _f64p, _f64p, _f64p, _i32p, _f64p]
_lib.cdsdp_results.argtypes = [_vp, _vp, _f64p, _f64p, _f64p, _f64p, _f64p]
_lib.cdsdp_free.argtypes = [_vp]
_lib.cdsdp_profile.argtypes = [_vp, _f64p, _i32p, _f64p]
_lib.cdsdp_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _f64p]
_lib.cdsdp_profile_orders.argtypes = [_vp, _i32p, _f64p, _i32p, _i32p, _f64p]
_lib.cdsdp_profile_large.argtypes = [_vp, _f64p, _i32p, _i32p, _f64p, _f64p]
_lib.cdsdp_psd_project_large_bytes.argtypes = [ctypes.c_int, _i32p, ctypes.POINTER(ctypes.c_size_t)]
_lib.cdsdp_psd_project_large.argtypes = [ctypes.c_int, _i32p, ctypes.POINTER(_ll), _vp, _vp, _vp, ctypes.c_size_t,
                                         _vp]
PROJ_CLASSES = 22
_lib.cdsdp_strerror.argtypes = [ctypes.c_int]
_lib.cdsdp_strerror.restype = ctypes.c_char_p
_lib.cdsdp_psd_project.argtypes = [ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                                   ctypes.c_int, ctypes.c_int, _vp]

_lib.cdsdp_psd_violation_scratch_bytes.argtypes = [ctypes.c_int]
_lib.cdsdp_psd_violation_scratch_bytes.restype = ctypes.c_size_t
_lib.cdsdp_psd_violation.argtypes = [ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int, _vp,
                                     ctypes.c_size_t, _vp, _vp]
_lib.cdsdp_grad_workspace_bytes.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
_lib.cdsdp_unrolled_forward.argtypes = [_vp, ctypes.POINTER(Opts), ctypes.c_int, ctypes.c_int, _vp, _vp, _vp,
                                        ctypes.c_size_t, _vp, _vp]
_lib.cdsdp_unrolled_backward.argtypes = [_vp, ctypes.POINTER(Opts), ctypes.c_int, ctypes.c_int, _vp, _vp, _vp,
                                         ctypes.c_size_t, _vp, _vp, _vp, _vp]
_lib.cdsdp_psd_violation_noalloc.argtypes = [ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int,
                                             _vp, _vp]

EXPORTED = ["cdsdp_default_opts", "cdsdp_setup", "cdsdp_info", "cdsdp_cliques", "cdsdp_pattern",
            "cdsdp_workspace_bytes", "cdsdp_bind", "cdsdp_solve", "cdsdp_results", "cdsdp_free",
            "cdsdp_strerror", "cdsdp_psd_project", "cdsdp_profile", "cdsdp_psd_violation_scratch_bytes",
            "cdsdp_psd_violation", "cdsdp_psd_violation_noalloc", "cdsdp_grad_workspace_bytes",
            "cdsdp_unrolled_forward", "cdsdp_unrolled_backward", "cdsdp_components",
            "cdsdp_component_results", "cdsdp_autotune", "cdsdp_setup_scaled", "cdsdp_scaling", "cdsdp_scaling_batch",
            "cdsdp_completion_sizes", "cdsdp_complete", "cdsdp_setup_flags", "cdsdp_setup_batch",
            "cdsdp_fma_peak", "cdsdp_profile_orders", "cdsdp_psd_project_large_bytes",
            "cdsdp_psd_project_large", "cdsdp_profile_large"]


class CdsdpError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {strerror(status)} ({status})")
        self.status = status


def strerror(status: int) -> str:
    return _lib.cdsdp_strerror(int(status)).decode()


def default_opts(**kw) -> Opts:
    o = Opts()
    _lib.cdsdp_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp32": FP32, "fp64": FP64}[v]
        setattr(o, k, v)
    return o


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None and a.size else None


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Problem:
    """One SDP after the data preprocessing of Algorithms 1-3 (host only).

    scale_passes=None sets the data up as given (cdsdp_setup); an integer k >= 0
    scales it first as Section 7.1.3 describes, with k equilibration passes
    (cdsdp_setup_scaled); solutions come back in the original units.
    cache_factor=False skips the cached inverses (cdsdp_setup_flags with
    CDSDP_SETUP_NO_FACTOR): such a problem solves with linear_solver=1 only."""

    def __init__(self, prob, scale_passes=None, cache_factor=True, merge_cliques=False):
        (A_con, A_row, A_col, A_val, b, C_row, C_col, C_val, P_row, P_col) = prob.arrays()
        self._keep = (A_con, A_row, A_col, A_val, b, C_row, C_col, C_val, P_row, P_col)
        h = _vp()
        args = (int(prob.n), int(prob.m), A_con.size, _ptr(A_con, ctypes.c_int), _ptr(A_row, ctypes.c_int),
                _ptr(A_col, ctypes.c_int), _ptr(A_val, ctypes.c_double), _ptr(b, ctypes.c_double),
                C_row.size, _ptr(C_row, ctypes.c_int), _ptr(C_col, ctypes.c_int),
                _ptr(C_val, ctypes.c_double), P_row.size, _ptr(P_row, ctypes.c_int), _ptr(P_col, ctypes.c_int))
        if not cache_factor or merge_cliques:
            flags = (0 if cache_factor else SETUP_NO_FACTOR) | (SETUP_MERGE_CLIQUES if merge_cliques else 0)
            st = _lib.cdsdp_setup_flags(*args, -1 if scale_passes is None else int(scale_passes), flags,
                                        ctypes.byref(h))
            what = "cdsdp_setup_flags"
        elif scale_passes is None:
            st = _lib.cdsdp_setup(*args, ctypes.byref(h))
            what = "cdsdp_setup"
        else:
            st = _lib.cdsdp_setup_scaled(*args, int(scale_passes), ctypes.byref(h))
            what = "cdsdp_setup_scaled"
        if st != 0:
            raise CdsdpError(st, what)
        self._adopt(h)

    def _adopt(self, h):
        self._h = h
        self.workspace = None
        self.max_iter = 0
        self._summands = None
        inf = Info()
        _lib.cdsdp_info(self._h, ctypes.byref(inf))
        self.info = {f: getattr(inf, f) for f, _ in Info._fields_}

    @classmethod
    def batch(cls, problems, scale_passes=None, cache_factor=True):
        """A batch of independent SDPs as one handle (cdsdp_setup_batch): their
        direct sum, problem j numbered after problems 0..j-1.  `split` cuts a
        solution back into the problems'."""
        arrs = [p.arrays() for p in problems]
        cat_i = lambda k: np.ascontiguousarray(np.concatenate([a[k] for a in arrs]), dtype=np.int32)
        cat_f = lambda k: np.ascontiguousarray(np.concatenate([a[k] for a in arrs]), dtype=np.float64)
        A_con, A_row, A_col, A_val, b = cat_i(0), cat_i(1), cat_i(2), cat_f(3), cat_f(4)
        C_row, C_col, C_val, P_row, P_col = cat_i(5), cat_i(6), cat_f(7), cat_i(8), cat_i(9)
        n = np.array([p.n for p in problems], np.int32)
        m = np.array([p.m for p in problems], np.int32)
        nA = np.array([a[0].size for a in arrs], np.int64)
        nC = np.array([a[5].size for a in arrs], np.int64)
        nP = np.array([a[8].size for a in arrs], np.int64)
        self = cls.__new__(cls)
        self._keep = (A_con, A_row, A_col, A_val, b, C_row, C_col, C_val, P_row, P_col, n, m, nA, nC, nP)
        h = _vp()
        i64p = lambda a: a.ctypes.data_as(ctypes.POINTER(_ll))
        st = _lib.cdsdp_setup_batch(len(problems), _ptr(n, ctypes.c_int), _ptr(m, ctypes.c_int), i64p(nA),
                                    _ptr(A_con, ctypes.c_int), _ptr(A_row, ctypes.c_int), _ptr(A_col, ctypes.c_int),
                                    _ptr(A_val, ctypes.c_double), _ptr(b, ctypes.c_double), i64p(nC),
                                    _ptr(C_row, ctypes.c_int), _ptr(C_col, ctypes.c_int), _ptr(C_val, ctypes.c_double),
                                    i64p(nP), _ptr(P_row, ctypes.c_int), _ptr(P_col, ctypes.c_int),
                                    -1 if scale_passes is None else int(scale_passes),
                                    0 if cache_factor else SETUP_NO_FACTOR, ctypes.byref(h))
        if st != 0:
            raise CdsdpError(st, "cdsdp_setup_batch")
        self._adopt(h)
        self._summands = (n.astype(np.int64), m.astype(np.int64))
        return self

    def split(self, out):
        """Per-problem X, y, Z (and their pattern entries, local indices) of a
        solve of a handle made by `batch`."""
        if self._summands is None:
            raise ValueError("split() needs a handle made by Problem.batch")
        n, m = self._summands
        rows, cols = self.pattern()
        vo = np.concatenate([[0], np.cumsum(n)])
        mo = np.concatenate([[0], np.cumsum(m)])
        eo = np.searchsorted(cols, vo)  # pattern entries are column-major, so each problem's are contiguous
        res = []
        for j in range(len(n)):
            e0, e1 = eo[j], eo[j + 1]
            res.append({"rows": rows[e0:e1] - vo[j], "cols": cols[e0:e1] - vo[j],
                        "X": None if out.get("X") is None else out["X"][e0:e1],
                        "Z": None if out.get("Z") is None else out["Z"][e0:e1],
                        "y": None if out.get("y") is None else out["y"][mo[j]:mo[j + 1]]})
        return res

    def split_components(self, out):
        """Per independent component (cdsdp_components): its pattern entries
        (global indices), X, Z on them, its constraints and y on them."""
        vc, rc = self.components()
        rows, cols = self.pattern()
        ec = vc[cols]
        res = []
        for c in range(int(self.info["ncomp"])):
            ent = np.flatnonzero(ec == c)
            con = np.flatnonzero(rc == c)
            res.append({"entries": ent, "rows": rows[ent], "cols": cols[ent], "constraints": con,
                        "X": None if out.get("X") is None else out["X"][ent],
                        "Z": None if out.get("Z") is None else out["Z"][ent],
                        "y": None if out.get("y") is None else out["y"][con]})
        return res

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.cdsdp_free(h)
            self._h = None

    def cliques(self):
        p = self.info["p"]
        off = np.zeros(p + 1, np.int32)
        tot = int(self.info["n_d_lower"])  # upper bound on the vertex count
        vert = np.zeros(max(tot, 1), np.int32)
        _lib.cdsdp_cliques(self._h, _ptr(off, ctypes.c_int), _ptr(vert, ctypes.c_int))
        return off, vert[:off[-1]]

    def clique_list(self):
        off, vert = self.cliques()
        return [tuple(int(v) for v in vert[off[k]:off[k + 1]]) for k in range(len(off) - 1)]

    def pattern(self):
        nz = int(self.info["nnz_pattern"])
        r = np.zeros(nz, np.int32)
        c = np.zeros(nz, np.int32)
        _lib.cdsdp_pattern(self._h, _ptr(r, ctypes.c_int), _ptr(c, ctypes.c_int))
        return r, c

    def scaling(self):
        """(d [n], e [m], tau, sigma) of Section 7.1.3; ones for an unscaled handle."""
        d = np.zeros(int(self.info["n"]))
        e = np.zeros(int(self.info["m"]))
        tau = ctypes.c_double()
        sigma = ctypes.c_double()
        st = _lib.cdsdp_scaling(self._h, _ptr(d, ctypes.c_double), _ptr(e, ctypes.c_double), ctypes.byref(tau),
                                ctypes.byref(sigma))
        if st != 0:
            raise CdsdpError(st, "cdsdp_scaling")
        return d, e, tau.value, sigma.value

    def scaling_batch(self):
        """(tau [count], sigma [count]) of every SDP of a scaled batch
        (cdsdp_scaling_batch); one entry for any other handle."""
        n = ctypes.c_int(0)
        st = _lib.cdsdp_scaling_batch(self._h, ctypes.byref(n), None, None)
        if st != 0:
            raise CdsdpError(st, "cdsdp_scaling_batch")
        tau, sigma = np.zeros(n.value), np.zeros(n.value)
        st = _lib.cdsdp_scaling_batch(self._h, None, _ptr(tau, ctypes.c_double), _ptr(sigma, ctypes.c_double))
        if st != 0:
            raise CdsdpError(st, "cdsdp_scaling_batch")
        return tau, sigma

    def completion_sizes(self):
        """(device scratch bytes, doubles of the dense blocks, block offsets [ncomp + 1])."""
        sb = ctypes.c_size_t()
        we = _ll()
        offs = np.zeros(int(self.info["ncomp"]) + 1, np.int64)
        st = _lib.cdsdp_completion_sizes(self._h, ctypes.byref(sb), ctypes.byref(we),
                                         ctypes.c_void_p(offs.ctypes.data))
        if st != 0:
            raise CdsdpError(st, "cdsdp_completion_sizes")
        return sb.value, we.value, offs

    def complete(self, X, dense=True, stream=None, scratch=None, out=None):
        """Maximum-determinant completion (Section 7.1.1) of X (pattern values,
        host array or CUDA tensor).  Returns (W, logdet): W a CUDA float64
        tensor holding the dense blocks of the components back to back (None
        when dense=False), logdet a numpy array per component.  Raises
        CdsdpError with status NOT_PD when a clique block of X is not positive
        definite."""
        import torch
        sb, we, _ = self.completion_sizes()
        if not torch.is_tensor(X):
            X = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).cuda()
        X = X.contiguous()
        if scratch is None:
            scratch = torch.empty(sb, dtype=torch.uint8, device=X.device)
        W = None
        if dense:
            W = out if out is not None else torch.empty(we, dtype=torch.float64, device=X.device)
        ld = np.zeros(int(self.info["ncomp"]))
        st = _lib.cdsdp_complete(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(scratch.data_ptr()),
                                 scratch.numel(), ctypes.c_void_p(W.data_ptr()) if W is not None else None,
                                 _ptr(ld, ctypes.c_double), _stream_ptr(stream))
        if st != 0:
            raise CdsdpError(st, "cdsdp_complete")
        return W, ld

    def components(self):
        """(component of each vertex [n], component of each constraint [m])."""
        vc = np.zeros(int(self.info["n"]), np.int32)
        rc = np.zeros(int(self.info["m"]), np.int32)
        st = _lib.cdsdp_components(self._h, _ptr(vc, ctypes.c_int), _ptr(rc, ctypes.c_int))
        if st != 0:
            raise CdsdpError(st, "cdsdp_components")
        return vc, rc

    def component_results(self, stream=None):
        """Per-component (iterations, status, last stopping-test row [ncomp, 8])
        of the last solve."""
        nc = int(self.info["ncomp"])
        it = np.zeros(nc, np.int32)
        stt = np.zeros(nc, np.int32)
        res = np.zeros((nc, 8))
        st = _lib.cdsdp_component_results(self._h, _stream_ptr(stream), _ptr(it, ctypes.c_int),
                                          _ptr(stt, ctypes.c_int), _ptr(res, ctypes.c_double))
        if st != 0:
            raise CdsdpError(st, "cdsdp_component_results")
        return it, stt, res

    def workspace_bytes(self, max_iter):
        n = ctypes.c_size_t()
        st = _lib.cdsdp_workspace_bytes(self._h, int(max_iter), ctypes.byref(n))
        if st != 0:
            raise CdsdpError(st, "cdsdp_workspace_bytes")
        return n.value

    def bind(self, max_iter=2000, stream=None, device="cuda"):
        """Allocate the device workspace with PyTorch and upload the problem."""
        import torch
        nbytes = self.workspace_bytes(max_iter)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        st = _lib.cdsdp_bind(self._h, ctypes.c_void_p(ws.data_ptr()), nbytes, int(max_iter), _stream_ptr(stream))
        if st != 0:
            raise CdsdpError(st, "cdsdp_bind")
        self.workspace = ws
        self.max_iter = max_iter
        return self

    def solve(self, form="primal", stream=None, outputs=True, **opts):
        o = default_opts(**opts)
        if self.workspace is None or o.max_iter > self.max_iter:
            self.bind(max(o.max_iter, self.max_iter))
        nz, m = int(self.info["nnz_pattern"]), int(self.info["m"])
        X = np.zeros(nz) if outputs else None
        y = np.zeros(m) if outputs else None
        Z = np.zeros(nz) if outputs else None
        hist = np.zeros((o.max_iter, 8)) if outputs else None
        cert = np.zeros(max(nz, m)) if outputs else None
        iters = ctypes.c_int(0)
        st = _lib.cdsdp_solve(self._h, FORMS.get(form, form), ctypes.byref(o), _stream_ptr(stream),
                              _ptr(X, ctypes.c_double), _ptr(y, ctypes.c_double), _ptr(Z, ctypes.c_double),
                              _ptr(hist, ctypes.c_double), ctypes.byref(iters), _ptr(cert, ctypes.c_double))
        if st < 0:
            raise CdsdpError(st, "cdsdp_solve")
        out = dict(status=st, iters=iters.value)
        if outputs:
            out.update(X=X, y=y, Z=Z, hist=hist[:iters.value])
            if st == PRIMAL_INFEASIBLE:
                out["cert"] = cert[:m]
            elif st == DUAL_INFEASIBLE:
                out["cert"] = cert[:nz]
        return out

    def autotune(self, form="primal", iters=50, stream=None, **opts):
        """Fastest launch schedule for this problem: returns (options dict to
        pass to solve, list of ms per iteration of every candidate)."""
        o = default_opts(**opts)
        if self.workspace is None or self.max_iter < iters:
            self.bind(max(iters, self.max_iter or 0))
        tuned = Opts()
        ms = np.zeros(28)
        n = ctypes.c_int(0)
        st = _lib.cdsdp_autotune(self._h, FORMS.get(form, form), ctypes.byref(o), int(iters), _stream_ptr(stream),
                                 ctypes.byref(tuned), _ptr(ms, ctypes.c_double), ctypes.byref(n))
        if st < 0:
            raise CdsdpError(st, "cdsdp_autotune")
        return ({"x_update": tuned.x_update, "proj_warps_div": tuned.proj_warps_div, "warm_start": tuned.warm_start,
                 "proj_streams": tuned.proj_streams, "proj_cta_kernel": tuned.proj_cta_kernel,
                 "row_threads": tuned.row_threads},
                ms[:n.value].tolist())

    def profile(self):
        """(projection ms summed, projection launches, iteration ms summed) of
        the last solve run with profile=1."""
        a, c = ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int()
        st = _lib.cdsdp_profile(self._h, ctypes.byref(a), ctypes.byref(n), ctypes.byref(c))
        if st != 0:
            raise CdsdpError(st, "cdsdp_profile")
        return a.value, n.value, c.value

    def profile_orders(self):
        """Per size class of the projection kernels in the last profiled solve:
        a list of dicts (order, ms, launches, cliques, nominal_flops) for the
        non-empty classes (cdsdp_profile_orders)."""
        n = PROJ_CLASSES
        orders, launches, cliques = (ctypes.c_int * n)(), (ctypes.c_int * n)(), (ctypes.c_int * n)()
        ms, flops = (ctypes.c_double * n)(), (ctypes.c_double * n)()
        st = _lib.cdsdp_profile_orders(self._h, orders, ms, launches, cliques, flops)
        if st != 0:
            raise CdsdpError(st, "cdsdp_profile_orders")
        return [{"order": orders[c], "ms": ms[c], "launches": launches[c], "cliques": cliques[c],
                 "nominal_flops": flops[c]} for c in range(n) if cliques[c] > 0]

    def profile_large(self):
        """The cliques of order > 128 in the last profiled solve: dict of ms,
        launches, cliques, nominal_flops and tensor_flops (cdsdp_profile_large)."""
        ms, nom, ten = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n, cl = ctypes.c_int(), ctypes.c_int()
        st = _lib.cdsdp_profile_large(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(cl), ctypes.byref(nom),
                                      ctypes.byref(ten))
        if st != 0:
            raise CdsdpError(st, "cdsdp_profile_large")
        return {"ms": ms.value, "launches": n.value, "cliques": cl.value, "nominal_flops": nom.value,
                "tensor_flops": ten.value}

    # ---- differentiation through unrolled Algorithm 1 ----

    def problem_data(self, device="cuda"):
        """(c, b) of the problem as CUDA float64 tensors in the solver's
        coordinates (c on the lower pattern, pattern order)."""
        import torch
        r, cpat = self.pattern()
        index = {(int(i), int(j)): e for e, (i, j) in enumerate(zip(r, cpat))}
        c = np.zeros(len(r))
        (_, _, _, _, b, C_row, C_col, C_val, _, _) = self._keep
        for i, j, v in zip(C_row, C_col, C_val):
            c[index[(int(i), int(j))]] += v
        return (torch.tensor(c, dtype=torch.float64, device=device),
                torch.tensor(np.asarray(b), dtype=torch.float64, device=device))

    def _grad_ws(self, iters, ckpt_every, precision, device):
        import torch
        n = ctypes.c_size_t()
        st = _lib.cdsdp_grad_workspace_bytes(self._h, int(iters), int(ckpt_every),
                                             FP64 if precision == "fp64" else FP32, ctypes.byref(n))
        if st != 0:
            raise CdsdpError(st, "cdsdp_grad_workspace_bytes")
        return torch.empty(n.value, dtype=torch.uint8, device=device)

    def unrolled_forward(self, c, b, iters, ckpt_every, precision="fp32", rho=1.0, gws=None, stream=None):
        import torch
        if self.workspace is None or self.max_iter < ckpt_every:
            self.bind(max(ckpt_every, self.max_iter))
        if gws is None:
            gws = self._grad_ws(iters, ckpt_every, precision, c.device)
        o = default_opts(precision=precision, rho=rho)
        x = torch.empty(int(self.info["nnz_pattern"]), dtype=torch.float64, device=c.device)
        c = c.contiguous(); b = b.contiguous()
        st = _lib.cdsdp_unrolled_forward(self._h, ctypes.byref(o), int(iters), int(ckpt_every),
                                         ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                         ctypes.c_void_p(gws.data_ptr()), gws.numel(), ctypes.c_void_p(x.data_ptr()),
                                         _stream_ptr(stream))
        if st != 0:
            raise CdsdpError(st, "cdsdp_unrolled_forward")
        return x, gws

    def unrolled_backward(self, c, b, xbar, iters, ckpt_every, gws, precision="fp32", rho=1.0, stream=None):
        import torch
        o = default_opts(precision=precision, rho=rho)
        cbar = torch.empty_like(c)
        bbar = torch.empty_like(b)
        c = c.contiguous(); b = b.contiguous(); xbar = xbar.contiguous().to(torch.float64)
        st = _lib.cdsdp_unrolled_backward(self._h, ctypes.byref(o), int(iters), int(ckpt_every),
                                          ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                          ctypes.c_void_p(gws.data_ptr()), gws.numel(),
                                          ctypes.c_void_p(xbar.data_ptr()), ctypes.c_void_p(cbar.data_ptr()),
                                          ctypes.c_void_p(bbar.data_ptr()), _stream_ptr(stream))
        if st != 0:
            raise CdsdpError(st, "cdsdp_unrolled_backward")
        return cbar, bbar

    def results(self, stream=None):
        nz, m = int(self.info["nnz_pattern"]), int(self.info["m"])
        X, y, Z = np.zeros(nz), np.zeros(m), np.zeros(nz)
        st = _lib.cdsdp_results(self._h, _stream_ptr(stream), _ptr(X, ctypes.c_double), _ptr(y, ctypes.c_double),
                                _ptr(Z, ctypes.c_double), None, None)
        if st < 0:
            raise CdsdpError(st, "cdsdp_results")
        return X, y, Z


def psd_project(W, offsets, sizes, eig_offsets=None, vec_offsets=None, want_eig=False, max_sweeps=30, stream=None):
    """Batched PSD projection of lower-packed blocks (torch CUDA tensors).
    W: float32 or float64 [n_packed]; offsets int32 [p+1]; sizes int32 [p].
    Returns X (and eigenvalues, eigenvectors when want_eig)."""
    import torch
    p = int(sizes.numel())
    X = torch.empty_like(W)
    prec = FP64 if W.dtype == torch.float64 else FP32
    eig = vec = None
    if want_eig:
        eig = torch.empty(int(eig_offsets[-1].item()) if eig_offsets is not None else 0, dtype=W.dtype, device=W.device)
        vec = torch.empty(int(vec_offsets[-1].item()) if vec_offsets is not None else 0, dtype=W.dtype, device=W.device)
    maxs = int(sizes.max().item()) if p else 1
    st = _lib.cdsdp_psd_project(p, ctypes.c_void_p(offsets.data_ptr()), ctypes.c_void_p(sizes.data_ptr()), maxs,
                                ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                ctypes.c_void_p(eig.data_ptr()) if eig is not None else None,
                                ctypes.c_void_p(eig_offsets.data_ptr()) if eig is not None else None,
                                ctypes.c_void_p(vec.data_ptr()) if vec is not None else None,
                                ctypes.c_void_p(vec_offsets.data_ptr()) if vec is not None else None,
                                prec, int(max_sweeps), _stream_ptr(stream))
    if st != 0:
        raise CdsdpError(st, "cdsdp_psd_project")
    return (X, eig, vec) if want_eig else X


def psd_project_large(W, sizes, offsets=None, scratch=None, stream=None):
    """P(W_k) of float32 lower-packed blocks of order 129..8192 on the tensor
    cores (cdsdp_psd_project_large).  W: contiguous float32 CUDA tensor;
    sizes, offsets: host integer sequences (offsets default to back-to-back
    blocks).  Returns a new tensor like W."""
    import torch
    if W.dtype != torch.float32 or W.device.type != "cuda" or not W.is_contiguous():
        raise ValueError("W must be a contiguous float32 CUDA tensor")
    sz = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32))
    if offsets is None:
        offsets = np.concatenate([[0], np.cumsum(sz.astype(np.int64) * (sz + 1) // 2)[:-1]])
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    need = int(np.max(off + sz.astype(np.int64) * (sz + 1) // 2))
    if off.size != sz.size or need > W.numel():
        raise ValueError("offsets and sizes do not fit W")
    nbytes = ctypes.c_size_t()
    st = _lib.cdsdp_psd_project_large_bytes(int(sz.size), _ptr(sz, ctypes.c_int), ctypes.byref(nbytes))
    if st != 0:
        raise CdsdpError(st, "cdsdp_psd_project_large_bytes")
    if scratch is None or scratch.numel() < nbytes.value:
        scratch = torch.empty(nbytes.value, dtype=torch.uint8, device=W.device)
    X = torch.empty_like(W)
    st = _lib.cdsdp_psd_project_large(int(sz.size), _ptr(sz, ctypes.c_int), off.ctypes.data_as(ctypes.POINTER(_ll)),
                                      ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                      ctypes.c_void_p(scratch.data_ptr()), nbytes.value, _stream_ptr(stream))
    if st != 0:
        raise CdsdpError(st, "cdsdp_psd_project_large")
    return X


def _check_violation_args(W, offsets, sizes, alpha=None):
    """Refuse, with ValueError, arguments the kernel would read or write out
    of bounds: W float32 or float64, offsets and sizes int32 with
    len(offsets) == len(sizes) + 1, alpha float64 with one element or more;
    all contiguous CUDA tensors on one device.  Returns the precision code."""
    import torch
    if W.dtype not in (torch.float32, torch.float64):
        raise ValueError(f"W must be float32 or float64, not {W.dtype}")
    for name, t in (("offsets", offsets), ("sizes", sizes)):
        if t.dtype != torch.int32:
            raise ValueError(f"{name} must be int32, not {t.dtype}")
    if sizes.dim() != 1 or sizes.numel() < 1:
        raise ValueError("sizes must be a non-empty 1-D tensor")
    if offsets.dim() != 1 or offsets.numel() != sizes.numel() + 1:
        raise ValueError("offsets must hold len(sizes) + 1 entries")
    if alpha is not None and (alpha.dtype != torch.float64 or alpha.numel() < 1):
        raise ValueError("alpha must be a float64 tensor with at least one element")
    ts = [W, offsets, sizes] + ([alpha] if alpha is not None else [])
    if any(not t.is_contiguous() for t in ts):
        raise ValueError("W, offsets, sizes and alpha must be contiguous")
    if any(t.device.type != "cuda" for t in ts) or len({t.device for t in ts}) != 1:
        raise ValueError("W, offsets, sizes and alpha must be CUDA tensors on one device")
    return FP64 if W.dtype == torch.float64 else FP32


def fma_peak(precision="fp32", iters=None, stream=None):
    """Measured FMA throughput of the current GPU in TFLOP/s (float or double
    FMA chains over every SM; cdsdp_fma_peak)."""
    prec = FP64 if precision == "fp64" else FP32
    if iters is None:
        iters = 20000 if prec == FP64 else 100000
    out = ctypes.c_double()
    st = _lib.cdsdp_fma_peak(prec, int(iters), _stream_ptr(stream), ctypes.byref(out))
    if st != 0:
        raise CdsdpError(st, "cdsdp_fma_peak")
    return out.value


def psd_violation(W, offsets, sizes, max_sweeps=30, stream=None):
    """alpha = -min(0, min_k lambda_min(W_k)) of lower-packed blocks (torch
    CUDA tensors, layout of psd_project); returns a 1-element float64 CUDA
    tensor.  Scratch comes from a PyTorch allocation.  An order outside
    1..max(sizes) cannot occur here; the library writes NaN for one."""
    import torch
    prec = _check_violation_args(W, offsets, sizes)
    p = int(sizes.numel())
    nbytes = _lib.cdsdp_psd_violation_scratch_bytes(p)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=W.device)
    alpha = torch.empty(1, dtype=torch.float64, device=W.device)
    maxs = int(sizes.max().item())
    st = _lib.cdsdp_psd_violation(p, ctypes.c_void_p(offsets.data_ptr()), ctypes.c_void_p(sizes.data_ptr()), maxs,
                                  ctypes.c_void_p(W.data_ptr()), prec, int(max_sweeps),
                                  ctypes.c_void_p(scratch.data_ptr()), nbytes, ctypes.c_void_p(alpha.data_ptr()),
                                  _stream_ptr(stream))
    if st != 0:
        raise CdsdpError(st, "cdsdp_psd_violation")
    return alpha


def psd_violation_noalloc(W, offsets, sizes, alpha, max_sweeps=30, stream=None):
    """As psd_violation, through the entry point that allocates nothing: the
    caller passes the output `alpha` (float64 CUDA tensor, first element
    written) and the scratch is the library's fixed device array."""
    prec = _check_violation_args(W, offsets, sizes, alpha)
    p = int(sizes.numel())
    maxs = int(sizes.max().item())
    st = _lib.cdsdp_psd_violation_noalloc(p, ctypes.c_void_p(offsets.data_ptr()), ctypes.c_void_p(sizes.data_ptr()),
                                          maxs, ctypes.c_void_p(W.data_ptr()), prec, int(max_sweeps),
                                          ctypes.c_void_p(alpha.data_ptr()), _stream_ptr(stream))
    if st != 0:
        raise CdsdpError(st, "cdsdp_psd_violation_noalloc")
    return alpha


def unrolled_primal(problem, c, b, iters=500, ckpt_every=50, precision="fp32", rho=1.0):
    """x_N of `iters` unrolled iterations of Algorithm 1 as a differentiable
    function of c (lower pattern values) and b: gradients flow back through
    the library's reverse pass (Daleckii-Krein adjoint of the projections)."""
    import torch

    class _Unrolled(torch.autograd.Function):
        @staticmethod
        def forward(ctx, c_, b_):
            x, gws = problem.unrolled_forward(c_.detach(), b_.detach(), iters, ckpt_every, precision, rho)
            ctx.save_for_backward(c_.detach(), b_.detach())
            ctx.gws = gws
            return x

        @staticmethod
        def backward(ctx, xbar):
            c_, b_ = ctx.saved_tensors
            cbar, bbar = problem.unrolled_backward(c_, b_, xbar, iters, ckpt_every, ctx.gws, precision, rho)
            return cbar, bbar

    return _Unrolled.apply(c, b)
