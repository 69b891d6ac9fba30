"""Python binding of libhs, the GB300 separation-of-variables compact-stencil solver.

The functions below carry the C ABI's names (include/hs.h) and only marshal
arguments: every step of a solve runs in the CUDA library.  There is no CPU
path: importing works without a GPU, but any call needs libhs.so (built by
``paper_1912_03565_gb300.build``) and a CUDA device, and raises otherwise.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CPU/host data are
staged by the library itself (host-to-device copies on the given stream).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhs.so")

# enums (include/hs.h)
HS_OK = 0
HS_WARN_NEAR_SINGULAR = 1
HS_WARN_NOT_CONVERGED = 2
HS_ERR_INVALID_ARG = -1
HS_ERR_UNSUPPORTED = -2
HS_ERR_OOM = -3
HS_ERR_CUDA = -4
HS_ERR_NO_COEFF = -5
HS_ERR_TIMEOUT = -6
HS_ERR_NONFINITE = -7
HS_HELMHOLTZ, HS_CONVDIFF = 0, 1
HS_BC_DIRICHLET = 0
HS_FP64, HS_MIXED = 0, 1
HS_CD_PAPER, HS_CD_CORRECTED = 0, 1
HS_F64, HS_F32 = 0, 1
HS_RHS_NODAL, HS_RHS_ASSEMBLED = 0, 1
HS_RESID_DF, HS_RESID_F64, HS_RESID_AUTO = 0, 1, 2
(HS_DST_STAGED, HS_DST_FUSED, HS_DST_GENERIC, HS_DST_TWOPASS, HS_DST_FUSED_WIDE, HS_DST_GEMM,
 HS_DST_HALF) = (0, 1, 2, 3, 4, 5, 6)
HS_AXIS_X, HS_AXIS_Y = 0, 1
HS_FACTOR_AUTO, HS_FACTOR_F32, HS_FACTOR_F64 = 0, 1, 2
HS_HOST_F_MAPPED, HS_HOST_U_MAPPED, HS_HOST_F_EARLY, HS_HOST_U_LATE = 1, 2, 4, 8
HS_ZFACE_DIRICHLET, HS_ZFACE_ROBIN = 0, 1
HS_SIDE_DIRICHLET, HS_SIDE_NEUMANN, HS_SIDE_DN, HS_SIDE_ND = 0, 1, 2, 3
HS_THOMAS_PIPE16_256, HS_THOMAS_PIPE8_128, HS_THOMAS_PLAIN16_256, HS_THOMAS_PIPE16_128 = 0, 1, 2, 3
HS_THOMAS_BAL8_512, HS_THOMAS_BAL16_256 = 4, 5
HS_INFO_MAX_ITERS = 8
HS_INFO_STAGES = 8
STAGES = ("rhs", "dst_x", "dst_y", "thomas", "idst_y", "idst_x", "residual", "total")

EXPORTED = ("hs_plan", "hs_set_coeff", "hs_set_refinement", "hs_set_refinement_tol",
            "hs_set_stage_timing", "hs_solve",
            "hs_residual", "hs_rhs_apply", "hs_fp64_fma_rate", "hs_check_finite",
            "hs_autotune_cache_save", "hs_autotune_cache_load", "hs_autotune_cache_clear",
            "hs_autotune_cache_count", "hs_stage_times", "hs_workspace_bytes", "hs_destroy",
            "hs_status_str", "hs_last_error", "hs_residual_static", "hs_batch_create",
            "hs_batch_set_io", "hs_batch_solve", "hs_batch_set_wait_limit", "hs_batch_set_tol",
            "hs_batch_set_residual_precision", "hs_batch_debug_stall", "hs_set_residual_precision",
            "hs_batch_set_variant", "hs_batch_get_variant", "hs_batch_autotune",
            "hs_batch_graph_kernels",
            "hs_set_transform_variant", "hs_get_transform_variant", "hs_autotune",
            "hs_set_thomas_variant", "hs_get_thomas_variant", "hs_set_host_io", "hs_host_io_wait",
            "hs_set_factor_precision",
            "hs_precond_create", "hs_precond_apply", "hs_precond_solve", "hs_precond_destroy",
            "hs_batch_workspace_bytes", "hs_batch_destroy",
            "hs_zplan", "hs_zplan_set_coeff", "hs_zplan_set_faces", "hs_zplan_set_sides",
            "hs_zsolve", "hs_zsolve_ex", "hs_zsolve_full", "hs_zplan_set_coeff6",
            "hs_zplan_set_precision", "hs_set_coeff_fn", "hs_zplan_set_stage_timing",
            "hs_zplan_stage_times",
            "hs_zplan_workspace_bytes", "hs_zplan_last_error", "hs_zplan_destroy")
HS_STATIC_MAX_NZ = 8192


class hs_boundary(ctypes.Structure):
    _fields_ = [("face", ctypes.c_void_p * 6), ("fnn", ctypes.c_void_p * 6)]


class hs_problem_desc(ctypes.Structure):
    _fields_ = [("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("Nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("order", ctypes.c_int), ("equation", ctypes.c_int), ("cd_variant", ctypes.c_int),
                ("c0", ctypes.c_void_p), ("c1", ctypes.c_void_p), ("c2", ctypes.c_void_p),
                ("nrhs", ctypes.c_int), ("f", ctypes.c_void_p), ("u", ctypes.c_void_p)]


HS_PRECOND_MAX_HIST = 64


class hs_precond_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("history", ctypes.c_double * HS_PRECOND_MAX_HIST)]


class hs_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double * HS_INFO_MAX_ITERS),
                ("min_pivot_ratio", ctypes.c_double),
                ("stage_ms", ctypes.c_float * HS_INFO_STAGES)]

    def as_dict(self):
        n = self.iterations
        return {"iterations": n, "rel_residual": list(self.rel_residual[:max(n, 1)]),
                "min_pivot_ratio": self.min_pivot_ratio,
                "stage_ms": dict(zip(STAGES, list(self.stage_ms)))}


# double (*)(double z, int deriv, void *user)
HS_COEFF_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p)


def hs_set_coeff_fn(plan, fn, cd_variant=1):
    """hs_set_coeff from a Python function fn(z, deriv) -> float (deriv 0, 1, 2)."""
    cb = HS_COEFF_FN(lambda z, d, _u: float(fn(z, d)))
    return _check(load().hs_set_coeff_fn(plan, cb, None, int(cd_variant)), "hs_set_coeff_fn",
                  plan)


class HsError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} {detail}".strip())


_lib = None


def load(path: Optional[str] = None):
    """Load libhs.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1912_03565_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.hs_plan.argtypes = [ctypes.POINTER(vp), ci, ci, ci, cd, cd, cd, ci, ci, ci, ci, ci]
    lib.hs_plan.restype = ci
    lib.hs_set_coeff.argtypes = [vp, vp, vp, vp, ci]
    lib.hs_set_coeff.restype = ci
    lib.hs_set_coeff_fn.argtypes = [vp, HS_COEFF_FN, vp, ci]
    lib.hs_set_coeff_fn.restype = ci
    lib.hs_set_refinement.argtypes = [vp, ci]
    lib.hs_set_refinement.restype = ci
    lib.hs_set_refinement_tol.argtypes = [vp, cd]
    lib.hs_set_refinement_tol.restype = ci
    lib.hs_set_stage_timing.argtypes = [vp, ci]
    lib.hs_set_stage_timing.restype = ci
    lib.hs_solve.argtypes = [vp, vp, ci, ci, ctypes.POINTER(hs_boundary), vp, ci, vp,
                             ctypes.POINTER(hs_info)]
    lib.hs_solve.restype = ci
    lib.hs_residual.argtypes = [vp, vp, ci, ci, ctypes.POINTER(hs_boundary), vp, vp,
                                ctypes.POINTER(cd), ctypes.POINTER(cd)]
    lib.hs_residual.restype = ci
    lib.hs_autotune_cache_save.argtypes = [ctypes.c_char_p]
    lib.hs_autotune_cache_save.restype = ci
    lib.hs_autotune_cache_load.argtypes = [ctypes.c_char_p]
    lib.hs_autotune_cache_load.restype = ci
    lib.hs_autotune_cache_clear.argtypes = []
    lib.hs_autotune_cache_clear.restype = ci
    lib.hs_autotune_cache_count.argtypes = [ctypes.POINTER(ci)]
    lib.hs_autotune_cache_count.restype = ci
    lib.hs_check_finite.argtypes = [vp, vp, ci, ctypes.c_size_t, vp,
                                    ctypes.POINTER(ctypes.c_ulonglong)]
    lib.hs_check_finite.restype = ci
    lib.hs_fp64_fma_rate.argtypes = [vp, ctypes.POINTER(cd)]
    lib.hs_fp64_fma_rate.restype = ci
    lib.hs_rhs_apply.argtypes = [vp, vp, ci, ci, ctypes.POINTER(hs_boundary), vp, vp]
    lib.hs_rhs_apply.restype = ci
    lib.hs_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.hs_stage_times.restype = ci
    lib.hs_residual_static.argtypes = [ci, ci, ci, cd, cd, cd, ci, ci, ci, vp, vp, vp, vp, vp, vp,
                                       ctypes.POINTER(cd), ctypes.POINTER(cd)]
    lib.hs_residual_static.restype = ci
    lib.hs_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(hs_problem_desc), ci, ci, ci]
    lib.hs_batch_create.restype = ci
    lib.hs_batch_set_io.argtypes = [vp, ci, vp, vp]
    lib.hs_batch_set_io.restype = ci
    lib.hs_batch_solve.argtypes = [vp, vp, ci]
    lib.hs_batch_solve.restype = ci
    lib.hs_batch_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    lib.hs_batch_set_wait_limit.restype = ci
    lib.hs_precond_create.argtypes = [ctypes.POINTER(vp), vp, vp]
    lib.hs_precond_create.restype = ci
    lib.hs_precond_apply.argtypes = [vp, vp, vp, vp]
    lib.hs_precond_apply.restype = ci
    lib.hs_precond_solve.argtypes = [vp, vp, vp, cd, ci, vp, ctypes.POINTER(hs_precond_info)]
    lib.hs_precond_solve.restype = ci
    lib.hs_precond_destroy.argtypes = [vp]
    lib.hs_precond_destroy.restype = ci
    lib.hs_set_factor_precision.argtypes = [vp, ci]
    lib.hs_set_factor_precision.restype = ci
    lib.hs_set_host_io.argtypes = [vp, ci]
    lib.hs_set_host_io.restype = ci
    lib.hs_host_io_wait.argtypes = [vp, vp]
    lib.hs_host_io_wait.restype = ci
    dp = ctypes.POINTER(cd)
    lib.hs_zplan.argtypes = [ctypes.POINTER(vp), ci, ci, ci, cd, cd, cd, ci]
    lib.hs_zplan.restype = ci
    lib.hs_zplan_set_coeff.argtypes = [vp, dp]
    lib.hs_zplan_set_coeff.restype = ci
    lib.hs_zplan_set_faces.argtypes = [vp, ci, dp, dp, ci, dp, dp]
    lib.hs_zplan_set_faces.restype = ci
    lib.hs_zplan_set_stage_timing.argtypes = [vp, ci]
    lib.hs_zplan_set_stage_timing.restype = ci
    lib.hs_zplan_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.hs_zplan_stage_times.restype = ci
    lib.hs_zplan_set_sides.argtypes = [vp, ci, ci]
    lib.hs_zplan_set_sides.restype = ci
    lib.hs_zsolve_ex.argtypes = [vp, vp, vp, vp, ctypes.POINTER(vp), vp, vp]
    lib.hs_zsolve_ex.restype = ci
    lib.hs_zsolve_full.argtypes = [vp, vp, vp, vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp]
    lib.hs_zsolve_full.restype = ci
    lib.hs_zplan_set_precision.argtypes = [vp, ci, ci]
    lib.hs_zplan_set_precision.restype = ci
    lib.hs_zplan_set_coeff6.argtypes = [vp, dp, dp, dp]
    lib.hs_zplan_set_coeff6.restype = ci
    lib.hs_zsolve.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.hs_zsolve.restype = ci
    lib.hs_zplan_workspace_bytes.argtypes = [vp]
    lib.hs_zplan_workspace_bytes.restype = ctypes.c_size_t
    lib.hs_zplan_last_error.argtypes = [vp]
    lib.hs_zplan_last_error.restype = ctypes.c_char_p
    lib.hs_zplan_destroy.argtypes = [vp]
    lib.hs_zplan_destroy.restype = None
    lib.hs_set_thomas_variant.argtypes = [vp, ci]
    lib.hs_set_thomas_variant.restype = ci
    lib.hs_get_thomas_variant.argtypes = [vp, ctypes.POINTER(ci)]
    lib.hs_get_thomas_variant.restype = ci
    lib.hs_set_transform_variant.argtypes = [vp, ci, ci]
    lib.hs_set_transform_variant.restype = ci
    lib.hs_get_transform_variant.argtypes = [vp, ci, ctypes.POINTER(ci)]
    lib.hs_get_transform_variant.restype = ci
    lib.hs_autotune.argtypes = [vp, vp, ci, ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(ctypes.c_float)]
    lib.hs_autotune.restype = ci
    lib.hs_batch_set_variant.argtypes = [vp, ci]
    lib.hs_batch_set_variant.restype = ci
    lib.hs_batch_get_variant.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    lib.hs_batch_get_variant.restype = ci
    lib.hs_batch_graph_kernels.argtypes = [vp, ctypes.POINTER(ci)]
    lib.hs_batch_graph_kernels.restype = ci
    lib.hs_batch_autotune.argtypes = [vp, vp, ci, ctypes.POINTER(ctypes.c_float)]
    lib.hs_batch_autotune.restype = ci
    lib.hs_batch_set_residual_precision.argtypes = [vp, ci]
    lib.hs_batch_set_residual_precision.restype = ci
    lib.hs_set_residual_precision.argtypes = [vp, ci]
    lib.hs_set_residual_precision.restype = ci
    lib.hs_batch_set_tol.argtypes = [vp, cd]
    lib.hs_batch_set_tol.restype = ci
    lib.hs_batch_debug_stall.argtypes = [vp, ci]
    lib.hs_batch_debug_stall.restype = ci
    lib.hs_batch_workspace_bytes.argtypes = [vp]
    lib.hs_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.hs_batch_destroy.argtypes = [vp]
    lib.hs_batch_destroy.restype = ci
    lib.hs_workspace_bytes.argtypes = [vp]
    lib.hs_workspace_bytes.restype = ctypes.c_size_t
    lib.hs_destroy.argtypes = [vp]
    lib.hs_destroy.restype = ci
    lib.hs_status_str.argtypes = [ci]
    lib.hs_status_str.restype = ctypes.c_char_p
    lib.hs_last_error.argtypes = [vp]
    lib.hs_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def status_str(s: int) -> str:
    try:
        return load().hs_status_str(int(s)).decode()
    except Exception:  # library missing: still describe the code
        return f"hs_status {s}"


def _check(st, where, plan=None):
    if st < 0:
        detail = ""
        if plan:
            detail = load().hs_last_error(plan).decode()
        raise HsError(st, where, detail)
    return st


def _ptr(a):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return getattr(stream, "cuda_stream", None) or None


# ------------------------------------------------------------------ C ABI calls


def hs_plan(Nx, Ny, Nz, Lx, Ly, Lz, order, equation=HS_HELMHOLTZ, bc=HS_BC_DIRICHLET,
            precision=HS_FP64, max_rhs=1):
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.hs_plan(ctypes.byref(h), Nx, Ny, Nz, Lx, Ly, Lz, order, equation, bc,
                       precision, max_rhs), "hs_plan")
    return h.value


def hs_set_coeff(plan, c0, c1=None, c2=None, cd_variant=HS_CD_CORRECTED):
    """c0, c1, c2: host float64 arrays of length Nz+2 (numpy)."""
    import numpy as np
    arrs = [None if c is None else np.ascontiguousarray(c, dtype=np.float64) for c in (c0, c1, c2)]
    return _check(load().hs_set_coeff(plan, *[_ptr(a) for a in arrs], cd_variant),
                  "hs_set_coeff", plan)


def hs_set_refinement(plan, sweeps):
    return _check(load().hs_set_refinement(plan, sweeps), "hs_set_refinement", plan)


def hs_set_refinement_tol(plan, tol):
    return _check(load().hs_set_refinement_tol(plan, float(tol)), "hs_set_refinement_tol", plan)


def hs_set_stage_timing(plan, on):
    return _check(load().hs_set_stage_timing(plan, 1 if on else 0), "hs_set_stage_timing", plan)


def make_boundary(faces: Optional[Sequence] = None, fnn: Optional[Sequence] = None):
    b = hs_boundary()
    for k in range(6):
        b.face[k] = _ptr(faces[k]) if faces is not None and faces[k] is not None else None
        b.fnn[k] = _ptr(fnn[k]) if fnn is not None and fnn[k] is not None else None
    return b


def hs_solve(plan, f, f_dtype, rhs_kind, bnd, u, nrhs=1, stream=None, info=False):
    """Returns (status, info dict or None).  bnd: hs_boundary or None."""
    inf = hs_info() if info else None
    st = load().hs_solve(plan, _ptr(f), f_dtype, rhs_kind,
                         ctypes.byref(bnd) if bnd is not None else None, _ptr(u), nrhs,
                         _stream_ptr(stream), ctypes.byref(inf) if inf is not None else None)
    _check(st, "hs_solve", plan)
    return st, (inf.as_dict() if inf is not None else None)


def hs_residual(plan, f, f_dtype, rhs_kind, bnd, u, stream=None):
    r = ctypes.c_double()
    n = ctypes.c_double()
    _check(load().hs_residual(plan, _ptr(f), f_dtype, rhs_kind,
                              ctypes.byref(bnd) if bnd is not None else None, _ptr(u),
                              _stream_ptr(stream), ctypes.byref(r), ctypes.byref(n)),
           "hs_residual", plan)
    return r.value, n.value


def hs_rhs_apply(plan, f, f_dtype, rhs_kind, bnd, F, stream=None):
    """The lifted right-hand side as a solve forms it (device arrays; FP64 plan:
    F FP64 [Nz][Ny][Nx]; mixed plan: F FP32 [2][Nz][Ny][Nx], hi then lo)."""
    return _check(load().hs_rhs_apply(plan, _ptr(f), f_dtype, rhs_kind,
                                      ctypes.byref(bnd) if bnd is not None else None, _ptr(F),
                                      _stream_ptr(stream)), "hs_rhs_apply", plan)


def hs_autotune_cache_save(path):
    _check(load().hs_autotune_cache_save(os.fsencode(path)), "hs_autotune_cache_save")


def hs_autotune_cache_load(path):
    _check(load().hs_autotune_cache_load(os.fsencode(path)), "hs_autotune_cache_load")


def hs_autotune_cache_clear():
    _check(load().hs_autotune_cache_clear(), "hs_autotune_cache_clear")


def hs_autotune_cache_count():
    n = ctypes.c_int()
    _check(load().hs_autotune_cache_count(ctypes.byref(n)), "hs_autotune_cache_count")
    return n.value


def hs_check_finite(plan, data, stream=None):
    """Number of NaN / infinite values of a float64 or float32 device tensor."""
    import torch
    if data.dtype not in (torch.float64, torch.float32) or not data.is_contiguous():
        raise ValueError("data must be a contiguous float64 or float32 tensor")
    n = ctypes.c_ulonglong()
    dt = HS_F64 if data.dtype == torch.float64 else HS_F32
    _check(load().hs_check_finite(plan, _ptr(data), dt, data.numel(), _stream_ptr(stream),
                                  ctypes.byref(n)), "hs_check_finite", plan)
    return n.value


def hs_fp64_fma_rate(stream=None):
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    t = ctypes.c_double()
    _check(load().hs_fp64_fma_rate(_stream_ptr(stream), ctypes.byref(t)), "hs_fp64_fma_rate")
    return t.value


def hs_stage_times(plan):
    """Per-stage device ms of the last solve (stage timing on), keyed by STAGES."""
    arr = (ctypes.c_float * HS_INFO_STAGES)()
    _check(load().hs_stage_times(plan, arr), "hs_stage_times", plan)
    return dict(zip(STAGES, list(arr)))


def hs_residual_static(Nx, Ny, Nz, Lx, Ly, Lz, order, equation, cd_variant, c0, c1, c2, F, u,
                       stream=None):
    """||F - A U||_2, ||F||_2 without any allocation in the library (F, u device arrays).

    The C side receives bare pointers, so the sizes and types are checked here:
    c0..c2 hold Nz + 2 values, F and u are contiguous FP64 arrays of Nx Ny Nz
    elements (torch tensors on the current CUDA device)."""
    import numpy as np
    arrs = [None if c is None else np.ascontiguousarray(c, dtype=np.float64) for c in (c0, c1, c2)]
    for name, a in zip(("c0", "c1", "c2"), arrs):
        if a is not None and a.size != Nz + 2:
            raise ValueError(f"{name} must hold Nz + 2 = {Nz + 2} values, got {a.size}")
    n = int(Nx) * int(Ny) * int(Nz)
    for name, a in (("F", F), ("u", u)):
        dt = getattr(a, "dtype", None)
        if str(dt) not in ("torch.float64", "float64"):
            raise ValueError(f"{name} must be float64, got {dt}")
        numel = a.numel() if hasattr(a, "numel") and callable(a.numel) else int(np.size(a))
        if numel != n:
            raise ValueError(f"{name} must hold Nx*Ny*Nz = {n} values, got {numel}")
        contig = a.is_contiguous() if hasattr(a, "is_contiguous") else bool(
            getattr(getattr(a, "flags", None), "c_contiguous", False))
        if not contig:
            raise ValueError(f"{name} must be contiguous")
    r = ctypes.c_double()
    n = ctypes.c_double()
    _check(load().hs_residual_static(Nx, Ny, Nz, Lx, Ly, Lz, order, equation, cd_variant,
                                     *[_ptr(a) for a in arrs], _ptr(F), _ptr(u),
                                     _stream_ptr(stream), ctypes.byref(r), ctypes.byref(n)),
           "hs_residual_static")
    return r.value, n.value


def hs_workspace_bytes(plan):
    return int(load().hs_workspace_bytes(plan))


def hs_destroy(plan):
    if plan:
        return _check(load().hs_destroy(plan), "hs_destroy")
    return HS_OK


def hs_last_error(plan):
    return load().hs_last_error(plan).decode()


def hs_status_str(s):
    return status_str(s)


def hs_batch_create(problems, f_dtype=HS_F32, sweeps=1):
    """problems: list of dicts with N (Nx,Ny,Nz), L, order, equation, cd_variant, c0, c1, c2,
    nrhs, f (device array), u (device array).  Returns (handle, keepalive)."""
    import numpy as np
    arr = (hs_problem_desc * len(problems))()
    keep = []
    for k, p in enumerate(problems):
        cs = [None if c is None else np.ascontiguousarray(c, dtype=np.float64)
              for c in (p["c0"], p.get("c1"), p.get("c2"))]
        keep.append(cs)
        d = arr[k]
        d.Nx, d.Ny, d.Nz = p["N"]
        d.Lx, d.Ly, d.Lz = p["L"]
        d.order, d.equation = p["order"], p.get("equation", HS_HELMHOLTZ)
        d.cd_variant = p.get("cd_variant", HS_CD_CORRECTED)
        d.c0, d.c1, d.c2 = [_ptr(c) for c in cs]
        d.nrhs = p["nrhs"]
        d.f, d.u = _ptr(p["f"]), _ptr(p["u"])
    h = ctypes.c_void_p()
    _check(load().hs_batch_create(ctypes.byref(h), arr, len(problems), f_dtype, sweeps),
           "hs_batch_create")
    return h.value


def hs_batch_set_io(batch, k, f, u):
    return _check(load().hs_batch_set_io(batch, k, _ptr(f), _ptr(u)), "hs_batch_set_io")


def hs_batch_solve(batch, stream=None, sync=True):
    st = load().hs_batch_solve(batch, _stream_ptr(stream), 1 if sync else 0)
    _check(st, "hs_batch_solve")
    return st


def hs_batch_set_wait_limit(batch, spins):
    return _check(load().hs_batch_set_wait_limit(batch, int(spins)), "hs_batch_set_wait_limit")


def hs_set_residual_precision(plan, mode):
    return _check(load().hs_set_residual_precision(plan, int(mode)), "hs_set_residual_precision",
                  plan)


def hs_batch_set_residual_precision(batch, mode):
    return _check(load().hs_batch_set_residual_precision(batch, int(mode)),
                  "hs_batch_set_residual_precision")


def hs_set_transform_variant(plan, axis, variant):
    return _check(load().hs_set_transform_variant(plan, int(axis), int(variant)),
                  "hs_set_transform_variant", plan)


def hs_precond_create(plan, K):
    """Preconditioner-mode workspace for plan (coefficients = K_ref(z)) and the
    device FP64 coefficient field K (kept referenced by the caller)."""
    out = ctypes.c_void_p()
    _check(load().hs_precond_create(ctypes.byref(out), plan, _ptr(K)), "hs_precond_create", plan)
    return out


def hs_precond_apply(pc, u, y, stream=None):
    return _check(load().hs_precond_apply(pc, _ptr(u), _ptr(y), _stream_ptr(stream)),
                  "hs_precond_apply")


def hs_precond_solve(pc, F, x, tol=1e-10, maxit=100, stream=None):
    """Returns (status, info dict); raises on errors (negative status)."""
    inf = hs_precond_info()
    st = _check(load().hs_precond_solve(pc, _ptr(F), _ptr(x), float(tol), int(maxit),
                                        _stream_ptr(stream), ctypes.byref(inf)),
                "hs_precond_solve")
    n = min(inf.iterations, HS_PRECOND_MAX_HIST)
    return st, {"iterations": inf.iterations, "rel_residual": inf.rel_residual,
                "history": list(inf.history[:n])}


def hs_precond_destroy(pc):
    return _check(load().hs_precond_destroy(pc), "hs_precond_destroy")


def hs_set_factor_precision(plan, mode):
    return _check(load().hs_set_factor_precision(plan, int(mode)), "hs_set_factor_precision", plan)


def hs_set_host_io(plan, mapped):
    return _check(load().hs_set_host_io(plan, int(mapped)), "hs_set_host_io", plan)


def hs_host_io_wait(plan, stream=None):
    """Make `stream` wait for the plan's queued copies of u to the host (HS_HOST_U_LATE)."""
    return _check(load().hs_host_io_wait(plan, _stream_ptr(stream)), "hs_host_io_wait", plan)


def hs_set_thomas_variant(plan, variant):
    return _check(load().hs_set_thomas_variant(plan, int(variant)), "hs_set_thomas_variant", plan)


def hs_get_thomas_variant(plan):
    v = ctypes.c_int()
    _check(load().hs_get_thomas_variant(plan, ctypes.byref(v)), "hs_get_thomas_variant", plan)
    return v.value


def hs_get_transform_variant(plan, axis):
    v = ctypes.c_int()
    _check(load().hs_get_transform_variant(plan, int(axis), ctypes.byref(v)),
           "hs_get_transform_variant", plan)
    return v.value


def hs_autotune(plan, stream=None, reps=3):
    """Keeps the fastest transform variant per axis; returns (ms_x, ms_y) per pass."""
    mx, my = ctypes.c_float(), ctypes.c_float()
    _check(load().hs_autotune(plan, _stream_ptr(stream), int(reps), ctypes.byref(mx),
                              ctypes.byref(my)), "hs_autotune", plan)
    return mx.value, my.value


def hs_batch_set_variant(batch, variant):
    return _check(load().hs_batch_set_variant(batch, int(variant)), "hs_batch_set_variant")


def hs_batch_get_variant(batch):
    """(variant, grid) of the batch's persistent kernel."""
    v, g = ctypes.c_int(), ctypes.c_int()
    _check(load().hs_batch_get_variant(batch, ctypes.byref(v), ctypes.byref(g)),
           "hs_batch_get_variant")
    return v.value, g.value


def hs_batch_graph_kernels(batch):
    """Kernel launches per hs_batch_solve (kernel nodes of the captured graph)."""
    k = ctypes.c_int()
    _check(load().hs_batch_graph_kernels(batch, ctypes.byref(k)), "hs_batch_graph_kernels")
    return k.value


def hs_batch_autotune(batch, stream=None, reps=2):
    """Times each kernel variant on the batch, keeps the fastest; returns its ms per solve."""
    ms = ctypes.c_float()
    _check(load().hs_batch_autotune(batch, _stream_ptr(stream), int(reps), ctypes.byref(ms)),
           "hs_batch_autotune")
    return ms.value


def hs_batch_set_tol(batch, tol):
    return _check(load().hs_batch_set_tol(batch, float(tol)), "hs_batch_set_tol")


def hs_batch_debug_stall(batch, on):
    return _check(load().hs_batch_debug_stall(batch, 1 if on else 0), "hs_batch_debug_stall")


def hs_batch_workspace_bytes(batch):
    return int(load().hs_batch_workspace_bytes(batch))


def hs_batch_destroy(batch):
    if batch:
        return _check(load().hs_batch_destroy(batch), "hs_batch_destroy")
    return HS_OK


# ------------------------------------------------------------------ convenience


class Solver:
    """Owns one plan; marshals torch / numpy arrays to hs_solve."""

    def __init__(self, Nx, Ny, Nz, Lx, Ly, Lz, order, equation=HS_HELMHOLTZ,
                 precision=HS_FP64, max_rhs=1):
        self.shape = (Nz, Ny, Nx)
        self.order, self.equation, self.precision = order, equation, precision
        self.plan = hs_plan(Nx, Ny, Nz, Lx, Ly, Lz, order, equation, HS_BC_DIRICHLET,
                            precision, max_rhs)

    def set_coeff(self, c0, c1=None, c2=None, cd_variant=HS_CD_CORRECTED):
        import numpy as np
        n = self.shape[0] + 2
        for name, c in (("c0", c0), ("c1", c1), ("c2", c2)):
            if c is not None and np.asarray(c).size != n:
                raise ValueError(f"{name} must hold Nz + 2 = {n} values")
        return hs_set_coeff(self.plan, c0, c1, c2, cd_variant)

    def solve(self, f, u, f_dtype=HS_F64, rhs_kind=HS_RHS_NODAL, faces=None, fnn=None, nrhs=1,
              stream=None, info=False):
        b = make_boundary(faces, fnn) if (faces is not None or fnn is not None) else None
        self._keep = (f, u, faces, fnn)  # arrays stay alive until the next call
        return hs_solve(self.plan, f, f_dtype, rhs_kind, b, u, nrhs, stream, info)

    def close(self):
        if getattr(self, "plan", None):
            hs_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------- complex k(z), Robin z-faces


def _pair(z):
    z = complex(z)
    return (ctypes.c_double * 2)(z.real, z.imag)


class ZSolver:
    """Complex k(z) and Robin / Dirichlet z-faces on the FP64 path (orders 2, 4).

    Arrays are planar complex float64 device tensors: f [2][Nz+2][Ny+2][Nx+2],
    g_lo / g_hi [2][ny][nx] (None = 0), u [2][Nz+2][ny][nx], with nx = Nx + 2 on a
    Neumann x-axis (set_sides), Nx + 1 on an axis with one face of each kind
    (HS_SIDE_DN: nodes 1..Nx+1; HS_SIDE_ND: nodes 0..Nx), else Nx; likewise ny."""

    def __init__(self, Nx, Ny, Nz, Lx, Ly, Lz, order):
        out = ctypes.c_void_p()
        _check(load().hs_zplan(ctypes.byref(out), Nx, Ny, Nz, Lx, Ly, Lz, order), "hs_zplan")
        self.plan = out
        self.shape = (Nx, Ny, Nz)

    def _err(self, st, where):
        if st < 0:
            raise HsError(st, where, load().hs_zplan_last_error(self.plan).decode())
        return st

    def set_coeff(self, K):
        import numpy as np
        K = np.asarray(K, dtype=np.complex128).ravel()
        if K.size != self.shape[2] + 2:
            raise ValueError(f"K must hold Nz + 2 = {self.shape[2] + 2} values")
        buf = np.ascontiguousarray(np.stack([K.real, K.imag], axis=-1).ravel())
        arr = (ctypes.c_double * buf.size)(*buf.tolist())
        return self._err(load().hs_zplan_set_coeff(self.plan, arr), "hs_zplan_set_coeff")

    def set_precision(self, precision, sweeps=1):
        """HS_FP64, or HS_MIXED: FP32 solves refined with FP64 residuals (Dirichlet sides)."""
        return self._err(load().hs_zplan_set_precision(self.plan, int(precision), int(sweeps)),
                         "hs_zplan_set_precision")

    def set_coeff6(self, K, Kz, Kzz):
        """K, K_z, K_zz at the Nz + 2 nodes (order 6; orders 2 and 4 read K only)."""
        import numpy as np

        def arr(v):
            v = np.asarray(v, dtype=np.complex128).ravel()
            if v.size != self.shape[2] + 2:
                raise ValueError(f"coefficients must hold Nz + 2 = {self.shape[2] + 2} values")
            buf = np.ascontiguousarray(np.stack([v.real, v.imag], axis=-1).ravel())
            return (ctypes.c_double * buf.size)(*buf.tolist())

        return self._err(load().hs_zplan_set_coeff6(self.plan, arr(K), arr(Kz), arr(Kzz)),
                         "hs_zplan_set_coeff6")

    def set_faces(self, lo_kind, alpha_lo=1.0, beta_lo=0.0, hi_kind=HS_ZFACE_DIRICHLET,
                  alpha_hi=1.0, beta_hi=0.0):
        return self._err(load().hs_zplan_set_faces(self.plan, int(lo_kind), _pair(alpha_lo),
                                                   _pair(beta_lo), int(hi_kind), _pair(alpha_hi),
                                                   _pair(beta_hi)), "hs_zplan_set_faces")

    def set_sides(self, x_kind, y_kind):
        return self._err(load().hs_zplan_set_sides(self.plan, int(x_kind), int(y_kind)),
                         "hs_zplan_set_sides")

    def solve(self, f, u, g_lo=None, g_hi=None, stream=None, side_data=None, fnn=None):
        """side_data: u_n on the (x-lo, x-hi, y-lo, y-hi) faces, planar complex
        [2][Nz+2][Ny+2] (x-faces) / [2][Nz+2][Nx+2] (y-faces); None entries = 0.
        Only Neumann faces take data (both faces of HS_SIDE_NEUMANN, the high face
        of HS_SIDE_DN, the low face of HS_SIDE_ND).  fnn (order 6): f_nn on the six
        faces, planar complex [2][Nz+2][Ny+2] (x), [2][Nz+2][Nx+2] (y),
        [2][Ny+2][Nx+2] (z); None entries = 0."""
        self._keep = (f, u, g_lo, g_hi, side_data, fnn)
        if fnn is not None:
            sd = None if side_data is None else (ctypes.c_void_p * 4)(*[_ptr(a) for a in side_data])
            fa = (ctypes.c_void_p * 6)(*[_ptr(a) for a in fnn])
            return self._err(load().hs_zsolve_full(self.plan, _ptr(f), _ptr(g_lo), _ptr(g_hi), sd,
                                                   fa, _ptr(u), _stream_ptr(stream)),
                             "hs_zsolve_full")
        if side_data is None:
            return self._err(load().hs_zsolve(self.plan, _ptr(f), _ptr(g_lo), _ptr(g_hi),
                                              _ptr(u), _stream_ptr(stream)), "hs_zsolve")
        sd = (ctypes.c_void_p * 4)(*[_ptr(a) for a in side_data])
        return self._err(load().hs_zsolve_ex(self.plan, _ptr(f), _ptr(g_lo), _ptr(g_hi), sd,
                                             _ptr(u), _stream_ptr(stream)), "hs_zsolve_ex")

    ZSTAGES = ("rhs", "transforms", "thomas", "inverse_transforms", "output")

    def set_stage_timing(self, on):
        return self._err(load().hs_zplan_set_stage_timing(self.plan, int(bool(on))),
                         "hs_zplan_set_stage_timing")

    def stage_times(self):
        ms = (ctypes.c_float * 5)()
        self._err(load().hs_zplan_stage_times(self.plan, ms), "hs_zplan_stage_times")
        return dict(zip(self.ZSTAGES, list(ms)))

    def workspace_bytes(self):
        return load().hs_zplan_workspace_bytes(self.plan)

    def close(self):
        if getattr(self, "plan", None):
            load().hs_zplan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
