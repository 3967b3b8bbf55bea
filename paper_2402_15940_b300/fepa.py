"""Python binding of the C-ABI library (include/fepa.h): argument marshalling only.

Every computation runs in the CUDA kernels of libfepa.so; torch provides device
memory and the current stream.  There is no CPU fallback: if the library is
missing, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfepa.so")

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_MESH, ERR_NOCONV, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7
ERR_NONFINITE = -8
MASS, DIFFUSION = 0, 1
PRECOND_NONE, PRECOND_JACOBI = 0, 1
MAX_ORDER = 8

_FORMS = {"mass": MASS, "diffusion": DIFFUSION, MASS: MASS, DIFFUSION: DIFFUSION}
_PRECONDS = {"none": PRECOND_NONE, "jacobi": PRECOND_JACOBI, None: PRECOND_NONE,
             PRECOND_NONE: PRECOND_NONE, PRECOND_JACOBI: PRECOND_JACOBI}

# (name, restype, argtypes) of every exported symbol; the CPU test checks them against the header.
_P, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class CgStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("status", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("precond_norm", ctypes.c_double), ("b_norm", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RefineStats(ctypes.Structure):
    _fields_ = [("outer_iterations", ctypes.c_int32), ("inner_iterations", ctypes.c_int32),
                ("status", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("b_norm", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchStats(ctypes.Structure):
    _fields_ = [("max_iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("dof_iterations", ctypes.c_double),
                ("max_rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class BatchRefineStats(ctypes.Structure):
    _fields_ = [("max_inner_iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("dof_iterations", ctypes.c_double), ("max_rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolverState(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("outer_iterations", ctypes.c_int32), ("rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


CG_GRAPH, CG_STREAM = 0, 1
SOLVER_CG, SOLVER_REFINED = 0, 1
BUSY = 1

SIGNATURES = [
    ("fepa_version", ctypes.c_char_p, []),
    ("fepa_last_error", ctypes.c_char_p, []),
    ("fepa_launch_count", _I64, []),
    ("fepa_op_create", ctypes.c_int, [_I32, _I32, _I32, _P, _I32, _I32, _I32, _P, ctypes.POINTER(_P)]),
    ("fepa_op_create_hex", ctypes.c_int, [_I64, _P, _I64, _P, _I32, _I32, _I32, _P, ctypes.POINTER(_P)]),
    ("fepa_hex_numbering", ctypes.c_int, [_I64, _I64, _P, _I32, _P, ctypes.POINTER(_I64)]),
    ("fepa_op_set_vertices", ctypes.c_int, [_P, _P, _I32]),
    ("fepa_op_destroy", None, [_P]),
    ("fepa_op_ndofs", _I64, [_P]),
    ("fepa_op_nelems", _I64, [_P]),
    ("fepa_op_q1d", _I32, [_P]),
    ("fepa_op_dcomps", _I32, [_P]),
    ("fepa_op_set_stream", ctypes.c_int, [_P, _P]),
    ("fepa_op_set_cg_mode", ctypes.c_int, [_P, _I32]),
    ("fepa_op_set_fused_dot", ctypes.c_int, [_P, _I32]),
    ("fepa_op_apply_f32_dot", ctypes.c_int, [_P, _P, _P, _P]),
    ("fepa_op_boundary_dofs", ctypes.c_int, [_P, _P, _I64, ctypes.POINTER(_I64)]),
    ("fepa_op_set_essential", ctypes.c_int, [_P, _P, _I64]),
    ("fepa_op_elem_dofs", ctypes.c_int, [_P, _P]),
    ("fepa_op_qdata", ctypes.c_int, [_P, _P]),
    ("fepa_op_qp_coords", ctypes.c_int, [_P, _P]),
    ("fepa_op_apply", ctypes.c_int, [_P, _P, _P]),
    ("fepa_op_apply_f32", ctypes.c_int, [_P, _P, _P]),
    ("fepa_op_set_f32_variant", ctypes.c_int, [_P, _I32]),
    ("fepa_op_f32_variant", _I32, [_P]),
    ("fepa_f32_variant_name", ctypes.c_char_p, [_I32]),
    ("fepa_op_set_f64_variant", ctypes.c_int, [_P, _I32]),
    ("fepa_op_f64_variant", _I32, [_P]),
    ("fepa_f64_variant_name", ctypes.c_char_p, [_I32]),
    ("fepa_op_diagonal", ctypes.c_int, [_P, _P]),
    ("fepa_op_rhs", ctypes.c_int, [_P, _P, _P]),
    ("fepa_op_rhs_sine", ctypes.c_int, [_P, _D, _P]),
    ("fepa_cg_solve", ctypes.c_int, [_P, _P, _P, _D, _I32, _I32, ctypes.POINTER(CgStats)]),
    ("fepa_cg_solve_host", ctypes.c_int, [_P, _P, _P, _D, _I32, _I32, ctypes.POINTER(CgStats)]),
    ("fepa_cg_iterations", ctypes.c_int, [_P, _P, _P, _I32, _I32, ctypes.POINTER(CgStats)]),
    ("fepa_solve_refined", ctypes.c_int, [_P, _P, _P, _D, _I32, _D, _I32, _I32, ctypes.POINTER(RefineStats)]),
    ("fepa_solve_reliable", ctypes.c_int, [_P, _P, _P, _D, _D, _I32, _I32, ctypes.POINTER(RefineStats)]),
    ("fepa_solve_reliable_host", ctypes.c_int, [_P, _P, _P, _D, _D, _I32, _I32, ctypes.POINTER(RefineStats)]),
    ("fepa_solve_refined_host", ctypes.c_int, [_P, _P, _P, _D, _I32, _D, _I32, _I32,
                                               ctypes.POINTER(RefineStats)]),
    ("fepa_solver_start", ctypes.c_int, [_P, _I32, _P, _P, _D, _I32, _I32, _D, _I32]),
    ("fepa_solver_advance", ctypes.c_int, [_P, _I32]),
    ("fepa_solver_poll", ctypes.c_int, [_P, _I32, ctypes.POINTER(SolverState)]),
    ("fepa_batch_create", ctypes.c_int, [_I32, _P, _P, _P, _P, _I32, _P, ctypes.POINTER(_P)]),
    ("fepa_batch_destroy", None, [_P]),
    ("fepa_batch_ndofs", _I64, [_P]),
    ("fepa_batch_offsets", ctypes.c_int, [_P, _P]),
    ("fepa_batch_groups", _I32, [_P]),
    ("fepa_batch_group_info", ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _P]),
    ("fepa_batch_set_stream", ctypes.c_int, [_P, _P]),
    ("fepa_batch_set_f64_variant", ctypes.c_int, [_P, _I32]),
    ("fepa_batch_apply", ctypes.c_int, [_P, _P, _P]),
    ("fepa_batch_solve", ctypes.c_int, [_P, _P, _P, _D, _I32, _I32, ctypes.POINTER(BatchStats), _P]),
    ("fepa_batch_solve_refined", ctypes.c_int,
     [_P, _P, _P, _D, _I32, _D, _I32, _I32, ctypes.POINTER(BatchRefineStats), _P]),
    ("fepa_batch_solve_reliable", ctypes.c_int,
     [_P, _P, _P, _D, _D, _I32, _I32, ctypes.POINTER(BatchRefineStats), _P]),
    ("fepa_mg_create", ctypes.c_int, [_P, _I32, _I32, _I32, ctypes.POINTER(_P)]),
    ("fepa_mg_update", ctypes.c_int, [_P]),
    ("fepa_mg_destroy", None, [_P]),
    ("fepa_mg_levels", _I32, [_P]),
    ("fepa_mg_level_info", ctypes.c_int, [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I64),
                                          ctypes.POINTER(_D)]),
    ("fepa_mg_prolong", ctypes.c_int, [_P, _I32, _P, _P]),
    ("fepa_mg_restrict", ctypes.c_int, [_P, _I32, _P, _P]),
    ("fepa_mg_smooth", ctypes.c_int, [_P, _I32, _P, _P]),
    ("fepa_mg_vcycle", ctypes.c_int, [_P, _P, _P]),
    ("fepa_mg_solve", ctypes.c_int, [_P, _P, _P, _D, _I32, ctypes.POINTER(CgStats)]),
    ("fepa_mg_solver_start", ctypes.c_int, [_P, _P, _P, _D, _I32]),
    ("fepa_mg_solver_advance", ctypes.c_int, [_P, _I32]),
    ("fepa_mg_solver_poll", ctypes.c_int, [_P, _I32, ctypes.POINTER(SolverState)]),
    ("fepa_cg_solve_noalloc", ctypes.c_int, [_P, _P, _P, _D, _I32, _I32, ctypes.POINTER(CgStats)]),
    ("fepa_test_set_first_wait_limit", ctypes.c_int, [_I32]),
]
NOALLOC_MAX_DOFS = 131072


class FepaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fepa error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfepa.so (built by paper_2402_15940_b300.build) and declare its symbols."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2402_15940_b300.build`")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != OK:
        raise FepaError(rc, load_library().fepa_last_error().decode())


def launch_count() -> int:
    return int(load_library().fepa_launch_count())


def test_set_first_wait_limit(iterations: int):
    """Testing only: poll limit of the FP32 TMA kernels' first bounded wait (-1: default)."""
    _check(load_library().fepa_test_set_first_wait_limit(int(iterations)))


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("fepa needs a CUDA device; no CPU fallback exists")
    return torch


def _dev_ptr(t, dtype, numel, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} must have {numel} entries, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def hex_numbering(nverts, conn, p):
    """(elem_dofs [E][(p+1)^3] int32, N): the DOF numbering fepa_op_create_hex uses for order p
    on a connectivity mesh (host computation in the library; no device needed)."""
    lib = load_library()
    c = np.ascontiguousarray(conn, dtype=np.int32)
    if c.ndim != 2 or c.shape[1] != 8:
        raise ValueError("conn must have shape (E, 8)")
    out = np.empty((c.shape[0], (int(p) + 1) ** 3), dtype=np.int32)
    nd = ctypes.c_int64()
    _check(lib.fepa_hex_numbering(int(nverts), c.shape[0], c.ctypes.data_as(ctypes.c_void_p), int(p),
                                  out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nd)))
    return out, int(nd.value)


class Operator:
    """A partial-assembly operator: hex mesh (structured grid, or vertices + element
    connectivity through Operator.from_hex) + H1 space of order p + form + D."""

    def __init__(self, nx, ny, nz, vertices, p, form="diffusion", q=0):
        torch = _torch()
        lib = load_library()
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        if v.shape != ((nx + 1) * (ny + 1) * (nz + 1), 3):
            raise ValueError("vertices must have shape ((nx+1)(ny+1)(nz+1), 3)")
        self._lib = lib
        self.nx, self.ny, self.nz, self.p = int(nx), int(ny), int(nz), int(p)
        self.nverts = v.shape[0]
        self.form = _FORMS[form]
        h = ctypes.c_void_p()
        stream = torch.cuda.current_stream().cuda_stream
        _check(lib.fepa_op_create(self.nx, self.ny, self.nz, v.ctypes.data_as(ctypes.c_void_p), self.p, int(q),
                                  self.form, ctypes.c_void_p(stream), ctypes.byref(h)))
        self._init_handle(h)

    @classmethod
    def from_hex(cls, vertices, conn, p, form="diffusion", q=0):
        """Operator on a conforming hexahedral mesh: vertices (nverts, 3), conn (E, 8) with the
        corners of each element in tensor-product order (corner (i, j, k) at i + 2j + 4k)."""
        torch = _torch()
        lib = load_library()
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        c = np.ascontiguousarray(conn, dtype=np.int32)
        if v.ndim != 2 or v.shape[1] != 3 or c.ndim != 2 or c.shape[1] != 8:
            raise ValueError("vertices must have shape (nverts, 3) and conn (E, 8)")
        self = cls.__new__(cls)
        self._lib = lib
        self.nx = self.ny = self.nz = None
        self.p, self.nverts = int(p), v.shape[0]
        self.form = _FORMS[form]
        h = ctypes.c_void_p()
        stream = torch.cuda.current_stream().cuda_stream
        _check(lib.fepa_op_create_hex(v.shape[0], v.ctypes.data_as(ctypes.c_void_p), c.shape[0],
                                      c.ctypes.data_as(ctypes.c_void_p), self.p, int(q), self.form,
                                      ctypes.c_void_p(stream), ctypes.byref(h)))
        self._init_handle(h)
        return self

    def _init_handle(self, h):
        lib = self._lib
        self._h = h
        self.N = int(lib.fepa_op_ndofs(h))
        self.E = int(lib.fepa_op_nelems(h))
        self.q = int(lib.fepa_op_q1d(h))
        self.dcomps = int(lib.fepa_op_dcomps(h))
        self.n = self.p + 1

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.fepa_op_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        torch = _torch()
        _check(self._lib.fepa_op_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def _vec(self, out):
        torch = _torch()
        return torch.empty(self.N, dtype=torch.float64, device="cuda") if out is None else out

    def set_vertices(self, vertices):
        """New vertex positions (numpy host array or CUDA float64 tensor); rebuilds D."""
        torch = _torch()
        nv = self.nverts
        self._sync_stream()
        if isinstance(vertices, torch.Tensor):
            ptr = _dev_ptr(vertices, torch.float64, 3 * nv, "vertices")
            _check(self._lib.fepa_op_set_vertices(self._h, ptr, 1))
        else:
            v = np.ascontiguousarray(vertices, dtype=np.float64)
            if v.size != 3 * nv:
                raise ValueError("vertices has the wrong size")
            _check(self._lib.fepa_op_set_vertices(self._h, v.ctypes.data_as(ctypes.c_void_p), 0))

    # -- space and data
    def boundary_dofs(self) -> np.ndarray:
        cnt = ctypes.c_int64()
        _check(self._lib.fepa_op_boundary_dofs(self._h, None, 0, ctypes.byref(cnt)))
        out = np.empty(cnt.value, dtype=np.int32)
        _check(self._lib.fepa_op_boundary_dofs(self._h, out.ctypes.data_as(ctypes.c_void_p), cnt.value,
                                               ctypes.byref(cnt)))
        return out

    def set_essential(self, dofs):
        d = np.ascontiguousarray(dofs, dtype=np.int32)
        self._sync_stream()
        _check(self._lib.fepa_op_set_essential(self._h, d.ctypes.data_as(ctypes.c_void_p), len(d)))

    def elem_dofs(self):
        torch = _torch()
        out = torch.empty((self.E, self.n ** 3), dtype=torch.int32, device="cuda")
        self._sync_stream()
        _check(self._lib.fepa_op_elem_dofs(self._h, ctypes.c_void_p(out.data_ptr())))
        return out

    def qdata(self):
        torch = _torch()
        out = torch.empty((self.E, self.dcomps, self.q ** 3), dtype=torch.float64, device="cuda")
        self._sync_stream()
        _check(self._lib.fepa_op_qdata(self._h, ctypes.c_void_p(out.data_ptr())))
        return out

    def qp_coords(self):
        torch = _torch()
        out = torch.empty((self.E, self.q ** 3, 3), dtype=torch.float64, device="cuda")
        self._sync_stream()
        _check(self._lib.fepa_op_qp_coords(self._h, ctypes.c_void_p(out.data_ptr())))
        return out

    # -- operator
    def apply(self, x, out=None):
        torch = _torch()
        y = self._vec(out)
        px = _dev_ptr(x, torch.float64, self.N, "x")
        py = _dev_ptr(y, torch.float64, self.N, "y")
        self._sync_stream()
        _check(self._lib.fepa_op_apply(self._h, px, py))
        return y

    def apply_f32(self, x, out=None):
        """FP32 action (the mixed-precision operator); x, out: float32 CUDA tensors."""
        torch = _torch()
        y = torch.empty(self.N, dtype=torch.float32, device="cuda") if out is None else out
        px = _dev_ptr(x, torch.float32, self.N, "x")
        py = _dev_ptr(y, torch.float32, self.N, "y")
        self._sync_stream()
        _check(self._lib.fepa_op_apply_f32(self._h, px, py))
        return y

    def apply_f32_dot(self, x, out=None, xax=None):
        """FP32 action and (x, A x) from the same kernel; returns (y, xax), xax a float64
        CUDA tensor of one element."""
        torch = _torch()
        y = torch.empty(self.N, dtype=torch.float32, device="cuda") if out is None else out
        d = torch.empty(1, dtype=torch.float64, device="cuda") if xax is None else xax
        px = _dev_ptr(x, torch.float32, self.N, "x")
        py = _dev_ptr(y, torch.float32, self.N, "y")
        pd = _dev_ptr(d, torch.float64, 1, "xax")
        self._sync_stream()
        _check(self._lib.fepa_op_apply_f32_dot(self._h, px, py, pd))
        return y, d

    def set_f32_variant(self, variant):
        """-1: autotune at next FP32 use; 0..3: force a compiled launch shape."""
        _check(self._lib.fepa_op_set_f32_variant(self._h, int(variant)))

    def f32_variant(self):
        v = int(self._lib.fepa_op_f32_variant(self._h))
        return v, self._lib.fepa_f32_variant_name(v).decode()

    def set_f64_variant(self, variant):
        """-1: autotune at next FP64 use; 0: FP64 pipe; 1: double-float on the FP32 pipe;
        2: double-float in half-size blocks."""
        _check(self._lib.fepa_op_set_f64_variant(self._h, int(variant)))

    def f64_variant(self):
        v = int(self._lib.fepa_op_f64_variant(self._h))
        return v, self._lib.fepa_f64_variant_name(v).decode()

    def set_fused_dot(self, enable=True):
        """FP32 inner CG: take (d, A d) from the action kernel (default) or a separate pass."""
        _check(self._lib.fepa_op_set_fused_dot(self._h, 1 if enable else 0))

    def set_cg_mode(self, mode):
        _check(self._lib.fepa_op_set_cg_mode(self._h, {"graph": CG_GRAPH, "stream": CG_STREAM}.get(mode, mode)))

    def diagonal(self, out=None):
        torch = _torch()
        y = self._vec(out)
        self._sync_stream()
        _check(self._lib.fepa_op_diagonal(self._h, _dev_ptr(y, torch.float64, self.N, "diag")))
        return y

    def rhs(self, f_qp, out=None):
        torch = _torch()
        b = self._vec(out)
        pf = _dev_ptr(f_qp, torch.float64, self.E * self.q ** 3, "f_qp")
        self._sync_stream()
        _check(self._lib.fepa_op_rhs(self._h, pf, _dev_ptr(b, torch.float64, self.N, "b")))
        return b

    def rhs_sine(self, scale=1.0, out=None):
        torch = _torch()
        b = self._vec(out)
        self._sync_stream()
        _check(self._lib.fepa_op_rhs_sine(self._h, float(scale), _dev_ptr(b, torch.float64, self.N, "b")))
        return b

    # -- solver
    def solve(self, b, x=None, rtol=1e-10, maxit=10000, precond="jacobi", raise_on_noconv=True):
        torch = _torch()
        x = torch.zeros(self.N, dtype=torch.float64, device="cuda") if x is None else x
        st = CgStats()
        self._sync_stream()
        rc = self._lib.fepa_cg_solve(self._h, _dev_ptr(b, torch.float64, self.N, "b"),
                                     _dev_ptr(x, torch.float64, self.N, "x"), float(rtol), int(maxit),
                                     _PRECONDS[precond], ctypes.byref(st))
        if rc != ERR_NOCONV or raise_on_noconv:
            _check(rc)
        return x, st.as_dict()

    def solve_host(self, b, x=None, rtol=1e-10, maxit=10000, precond="jacobi", raise_on_noconv=True):
        """Solve with host (numpy) buffers; copies happen inside the library call."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.N) if x is None else x
        if b.shape != (self.N,) or x.shape != (self.N,) or x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("b and x must be contiguous float64 arrays of length N")
        st = CgStats()
        self._sync_stream()
        rc = self._lib.fepa_cg_solve_host(self._h, b.ctypes.data_as(ctypes.c_void_p),
                                          x.ctypes.data_as(ctypes.c_void_p), float(rtol), int(maxit),
                                          _PRECONDS[precond], ctypes.byref(st))
        if rc != ERR_NOCONV or raise_on_noconv:
            _check(rc)
        return x, st.as_dict()

    def solve_refined(self, b, x=None, rtol=1e-10, max_outer=50, inner_rtol=1e-4, inner_maxit=20000,
                      precond="jacobi", raise_on_noconv=True):
        """FP64 iterative refinement around an FP32 Jacobi-PCG (mixed precision)."""
        torch = _torch()
        x = torch.zeros(self.N, dtype=torch.float64, device="cuda") if x is None else x
        st = RefineStats()
        self._sync_stream()
        rc = self._lib.fepa_solve_refined(self._h, _dev_ptr(b, torch.float64, self.N, "b"),
                                          _dev_ptr(x, torch.float64, self.N, "x"), float(rtol), int(max_outer),
                                          float(inner_rtol), int(inner_maxit), _PRECONDS[precond], ctypes.byref(st))
        if rc != ERR_NOCONV or raise_on_noconv:
            _check(rc)
        return x, st.as_dict()

    def solve_refined_host(self, b, x=None, rtol=1e-10, max_outer=50, inner_rtol=1e-4, inner_maxit=20000,
                           precond="jacobi"):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.N) if x is None else x
        if b.shape != (self.N,) or x.shape != (self.N,) or x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("b and x must be contiguous float64 arrays of length N")
        st = RefineStats()
        self._sync_stream()
        _check(self._lib.fepa_solve_refined_host(self._h, b.ctypes.data_as(ctypes.c_void_p),
                                                 x.ctypes.data_as(ctypes.c_void_p), float(rtol), int(max_outer),
                                                 float(inner_rtol), int(inner_maxit), _PRECONDS[precond],
                                                 ctypes.byref(st)))
        return x, st.as_dict()

    def solve_reliable(self, b, x=None, rtol=1e-10, delta=0.03, maxit=20000, precond="jacobi",
                       raise_on_noconv=True):
        """Mixed-precision CG with reliable updates: one FP32 recurrence, its residual
        replaced by the FP64 residual each time it falls by delta (Krylov space kept)."""
        torch = _torch()
        x = torch.zeros(self.N, dtype=torch.float64, device="cuda") if x is None else x
        st = RefineStats()
        self._sync_stream()
        rc = self._lib.fepa_solve_reliable(self._h, _dev_ptr(b, torch.float64, self.N, "b"),
                                           _dev_ptr(x, torch.float64, self.N, "x"), float(rtol), float(delta),
                                           int(maxit), _PRECONDS[precond], ctypes.byref(st))
        if rc != ERR_NOCONV or raise_on_noconv:
            _check(rc)
        return x, st.as_dict()

    def solve_reliable_host(self, b, x=None, rtol=1e-10, delta=0.03, maxit=20000, precond="jacobi"):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.N) if x is None else x
        if b.shape != (self.N,) or x.shape != (self.N,) or x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("b and x must be contiguous float64 arrays of length N")
        st = RefineStats()
        self._sync_stream()
        _check(self._lib.fepa_solve_reliable_host(self._h, b.ctypes.data_as(ctypes.c_void_p),
                                                  x.ctypes.data_as(ctypes.c_void_p), float(rtol), float(delta),
                                                  int(maxit), _PRECONDS[precond], ctypes.byref(st)))
        return x, st.as_dict()

    # -- resumable solve (continuous batching)
    def solver_start(self, b, x, kind="cg", rtol=1e-10, maxit=20000, max_outer=50, inner_rtol=1e-4,
                     precond="jacobi"):
        torch = _torch()
        k = {"cg": SOLVER_CG, "refined": SOLVER_REFINED}.get(kind, kind)
        _check(self._lib.fepa_solver_start(self._h, int(k), _dev_ptr(b, torch.float64, self.N, "b"),
                                           _dev_ptr(x, torch.float64, self.N, "x"), float(rtol), int(maxit),
                                           int(max_outer), float(inner_rtol), _PRECONDS[precond]))
        self._sv_keep = (b, x)   # the buffers must outlive the solve (kept once it has started)

    def solver_advance(self, iterations):
        _check(self._lib.fepa_solver_advance(self._h, int(iterations)))

    def solver_poll(self, blocking=False):
        """None while work is in flight (non-blocking), else the state dict."""
        st = SolverState()
        rc = self._lib.fepa_solver_poll(self._h, 1 if blocking else 0, ctypes.byref(st))
        if rc == BUSY:
            return None
        _check(rc)
        return st.as_dict()

    def iterations(self, b, x, iters, precond="jacobi"):
        torch = _torch()
        st = CgStats()
        self._sync_stream()
        _check(self._lib.fepa_cg_iterations(self._h, _dev_ptr(b, torch.float64, self.N, "b"),
                                            _dev_ptr(x, torch.float64, self.N, "x"), int(iters),
                                            _PRECONDS[precond], ctypes.byref(st)))
        return st.as_dict()


class Batch:
    """Many independent problems solved together (block-diagonal batch operator).

    problems: list of dicts with keys n=(nx, ny, nz), vertices (numpy), p, form."""

    def __init__(self, problems, essential_boundary=True):
        torch = _torch()
        lib = load_library()
        self._lib = lib
        cnt = len(problems)
        dims = np.ascontiguousarray([list(pr["n"]) for pr in problems], dtype=np.int32)
        self._verts = [np.ascontiguousarray(pr["vertices"], dtype=np.float64) for pr in problems]
        ptrs = (ctypes.c_void_p * cnt)(*[v.ctypes.data for v in self._verts])
        orders = np.ascontiguousarray([pr["p"] for pr in problems], dtype=np.int32)
        forms = np.ascontiguousarray([_FORMS[pr["form"]] for pr in problems], dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib.fepa_batch_create(cnt, dims.ctypes.data_as(ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p),
                                     orders.ctypes.data_as(ctypes.c_void_p), forms.ctypes.data_as(ctypes.c_void_p),
                                     1 if essential_boundary else 0,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(h)))
        self._h = h
        self.count = cnt
        self.N = int(lib.fepa_batch_ndofs(h))
        off = np.empty(cnt + 1, dtype=np.int64)
        _check(lib.fepa_batch_offsets(h, off.ctypes.data_as(ctypes.c_void_p)))
        self.offsets = off
        self.groups = int(lib.fepa_batch_groups(h))

    def group_info(self):
        """Per group: order, form, elements and the autotuner's picks (FP64 variant, FP32 tile
        elements per block; -1 / 0 until chosen)."""
        out = []
        for g in range(self.groups):
            o, f, v64, ne32 = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
            e = ctypes.c_int64()
            _check(self._lib.fepa_batch_group_info(self._h, g, ctypes.byref(o), ctypes.byref(f), ctypes.byref(e),
                                                   ctypes.byref(v64), ctypes.byref(ne32)))
            out.append({"p": o.value, "form": "diffusion" if f.value == DIFFUSION else "mass", "elements": e.value,
                        "f64_variant": v64.value, "f32_elements_per_block": ne32.value})
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fepa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        torch = _torch()
        _check(self._lib.fepa_batch_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def set_f64_variant(self, variant):
        """-1: measured choice per group; 0: FP64 pipe; 1: double-float on the FP32 pipe;
        2: double-float in half-size tiles."""
        _check(self._lib.fepa_batch_set_f64_variant(self._h, int(variant)))

    def apply(self, x, out=None):
        torch = _torch()
        y = torch.empty(self.N, dtype=torch.float64, device="cuda") if out is None else out
        self._sync_stream()
        _check(self._lib.fepa_batch_apply(self._h, _dev_ptr(x, torch.float64, self.N, "x"),
                                          _dev_ptr(y, torch.float64, self.N, "y")))
        return y

    def solve(self, b, x=None, rtol=1e-10, maxit=10000, precond="jacobi", raise_on_noconv=True):
        torch = _torch()
        x = torch.zeros(self.N, dtype=torch.float64, device="cuda") if x is None else x
        st = BatchStats()
        its = np.zeros(self.count, dtype=np.int32)
        self._sync_stream()
        rc = self._lib.fepa_batch_solve(self._h, _dev_ptr(b, torch.float64, self.N, "b"),
                                        _dev_ptr(x, torch.float64, self.N, "x"), float(rtol), int(maxit),
                                        _PRECONDS[precond], ctypes.byref(st), its.ctypes.data_as(ctypes.c_void_p))
        if rc != ERR_NOCONV or raise_on_noconv:
            _check(rc)
        d = st.as_dict()
        d["iterations"] = its
        return x, d

    def solve_refined(self, b, x=None, rtol=1e-10, max_outer=50, inner_rtol=1e-4, inner_maxit=20000,
                      precond="jacobi", raise_on_noconv=True):
        """FP64 iterative refinement around batched FP32 Jacobi-PCG corrections (every problem
        to rtol on its FP64 residual); stats["iterations"]: FP32 iterations per problem."""
        torch = _torch()
        x = torch.zeros(self.N, dtype=torch.float64, device="cuda") if x is None else x
        st = BatchRefineStats()
        its = np.zeros(self.count, dtype=np.int32)
        self._sync_stream()
        rc = self._lib.fepa_batch_solve_refined(self._h, _dev_ptr(b, torch.float64, self.N, "b"),
                                                _dev_ptr(x, torch.float64, self.N, "x"), float(rtol),
                                                int(max_outer), float(inner_rtol), int(inner_maxit),
                                                _PRECONDS[precond], ctypes.byref(st),
                                                its.ctypes.data_as(ctypes.c_void_p))
        if rc != ERR_NOCONV or raise_on_noconv:
            _check(rc)
        d = st.as_dict()
        d["iterations"] = its
        return x, d


    def solve_reliable(self, b, x=None, rtol=1e-10, delta=0.03, maxit=20000, precond="jacobi",
                       raise_on_noconv=True):
        """Batched mixed-precision CG with reliable updates (per-problem FP32 recurrences whose
        residuals are replaced by FP64 residuals); stats["iterations"]: FP32 iterations per problem,
        stats["outer_iterations"]: replacements."""
        torch = _torch()
        x = torch.zeros(self.N, dtype=torch.float64, device="cuda") if x is None else x
        st = BatchRefineStats()
        its = np.zeros(self.count, dtype=np.int32)
        self._sync_stream()
        rc = self._lib.fepa_batch_solve_reliable(self._h, _dev_ptr(b, torch.float64, self.N, "b"),
                                                 _dev_ptr(x, torch.float64, self.N, "x"), float(rtol), float(delta),
                                                 int(maxit), _PRECONDS[precond], ctypes.byref(st),
                                                 its.ctypes.data_as(ctypes.c_void_p))
        if rc != ERR_NOCONV or raise_on_noconv:
            _check(rc)
        d = st.as_dict()
        d["iterations"] = its
        return x, d


class Multigrid:
    """p-multigrid V-cycle over orders p, p/2, ..., 1 of an Operator's mesh and form."""

    def __init__(self, op: Operator, smooth_degree=2, coarse_degree=24, precision="fp64"):
        lib = load_library()
        self._lib, self.op = lib, op
        h = ctypes.c_void_p()
        op._sync_stream()
        self.precision = precision
        _check(lib.fepa_mg_create(op._h, int(smooth_degree), int(coarse_degree),
                                  {"fp64": 0, "fp32": 1}[precision], ctypes.byref(h)))
        self._h = h
        self._info()

    def _info(self):
        lib, h = self._lib, self._h
        self.levels = []
        for l in range(int(lib.fepa_mg_levels(h))):
            o, n, lam = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_double()
            _check(lib.fepa_mg_level_info(h, l, ctypes.byref(o), ctypes.byref(n), ctypes.byref(lam)))
            self.levels.append({"order": o.value, "ndofs": n.value, "lambda_max": lam.value})

    def update(self):
        """Follow the fine op after set_vertices: move every level's mesh, rebuild diagonals
        and eigenvalue bounds."""
        self.op._sync_stream()
        _check(self._lib.fepa_mg_update(self._h))
        self._info()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fepa_mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, level, out=None):
        torch = _torch()
        return torch.empty(self.levels[level]["ndofs"], dtype=torch.float64, device="cuda") if out is None else out

    def prolong(self, level, xc, out=None):
        torch = _torch()
        y = self._vec(level, out)
        _check(self._lib.fepa_mg_prolong(self._h, int(level),
                                         _dev_ptr(xc, torch.float64, self.levels[level + 1]["ndofs"], "xc"),
                                         _dev_ptr(y, torch.float64, self.levels[level]["ndofs"], "xf")))
        return y

    def restrict(self, level, rf, out=None):
        torch = _torch()
        y = self._vec(level + 1, out)
        _check(self._lib.fepa_mg_restrict(self._h, int(level),
                                          _dev_ptr(rf, torch.float64, self.levels[level]["ndofs"], "rf"),
                                          _dev_ptr(y, torch.float64, self.levels[level + 1]["ndofs"], "rc")))
        return y

    def smooth(self, level, b, out=None):
        torch = _torch()
        y = self._vec(level, out)
        n = self.levels[level]["ndofs"]
        _check(self._lib.fepa_mg_smooth(self._h, int(level), _dev_ptr(b, torch.float64, n, "b"),
                                        _dev_ptr(y, torch.float64, n, "x")))
        return y

    def vcycle(self, b, out=None):
        torch = _torch()
        y = self._vec(0, out)
        n = self.levels[0]["ndofs"]
        _check(self._lib.fepa_mg_vcycle(self._h, _dev_ptr(b, torch.float64, n, "b"),
                                        _dev_ptr(y, torch.float64, n, "x")))
        return y

    def solve(self, b, x=None, rtol=1e-10, maxit=1000):
        torch = _torch()
        n = self.levels[0]["ndofs"]
        x = torch.zeros(n, dtype=torch.float64, device="cuda") if x is None else x
        st = CgStats()
        self.op._sync_stream()
        _check(self._lib.fepa_mg_solve(self._h, _dev_ptr(b, torch.float64, n, "b"), _dev_ptr(x, torch.float64, n, "x"),
                                       float(rtol), int(maxit), ctypes.byref(st)))
        return x, st.as_dict()

    # -- resumable solve (a serving loop's form of solve)
    def solver_start(self, b, x, rtol=1e-10, maxit=1000):
        torch = _torch()
        n = self.levels[0]["ndofs"]
        self.op._sync_stream()
        _check(self._lib.fepa_mg_solver_start(self._h, _dev_ptr(b, torch.float64, n, "b"),
                                              _dev_ptr(x, torch.float64, n, "x"), float(rtol), int(maxit)))
        self._sv_keep = (b, x)   # the buffers must outlive the solve

    def solver_advance(self, iterations):
        _check(self._lib.fepa_mg_solver_advance(self._h, int(iterations)))

    def solver_poll(self, blocking=False):
        """None while work is in flight (non-blocking), else the state dict."""
        st = SolverState()
        rc = self._lib.fepa_mg_solver_poll(self._h, 1 if blocking else 0, ctypes.byref(st))
        if rc == BUSY:
            return None
        _check(rc)
        return st.as_dict()
