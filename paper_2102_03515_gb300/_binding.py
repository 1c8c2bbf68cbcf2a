"""ctypes declarations of include/femamg.h and one Python function per entry point.

Device buffers are torch CUDA tensors (contiguous; float64 vectors, int32 index arrays);
``stream`` defaults to torch's current stream.  Failures raise :class:`FemError` with the
library's status and message, except FEM_ENOCONV from ``pcg_solve``, which is reported in
the returned result (the best iterate is written).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfemamg.so")

FEM_OK, FEM_EINVAL, FEM_ENOMEM, FEM_ECUDA, FEM_ENOCONV = 0, 1, 2, 3, 4
FEM_EBREAKDOWN, FEM_ECANCELLED, FEM_EDEVCHECK, FEM_EUNSUPPORTED = 5, 6, 7, 8
STATUS_NAMES = {0: "FEM_OK", 1: "FEM_EINVAL", 2: "FEM_ENOMEM", 3: "FEM_ECUDA", 4: "FEM_ENOCONV",
                5: "FEM_EBREAKDOWN", 6: "FEM_ECANCELLED", 7: "FEM_EDEVCHECK",
                8: "FEM_EUNSUPPORTED"}
FEM_TARGET = {"sine": 0, "box": 1, "bumps": 2, "sine_plus_one": 3, "quadvals": 4}
FEM_FMT_AUTO, FEM_FMT_STENCIL, FEM_FMT_CSR = 0, 1, 2
AMG_SMOOTHER_CHEBYSHEV, AMG_SMOOTHER_L1_JACOBI, AMG_SMOOTHER_SGS = 0, 1, 2
AMG_COARSEN_SA, AMG_COARSEN_RED_BLACK = 0, 1
AMG_ORDER_HASH, AMG_ORDER_NATURAL = 0, 1
AMG_PREC_FP64, AMG_PREC_FP32, AMG_PREC_BF16 = 0, 1, 2
PCG_STOP_RESIDUAL, PCG_STOP_PRECONDITIONED = 0, 1


class FemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class KuhnDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("xyz_host", C.POINTER(C.c_double))]


class Target(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nb", C.c_int32), ("centers_host", C.POINTER(C.c_double)),
                ("widths_host", C.POINTER(C.c_double)), ("amps_host", C.POINTER(C.c_double)),
                ("lo", C.c_double), ("hi", C.c_double), ("quadvals_dev", C.c_void_p)]


class AssembleOpts(C.Structure):
    _fields_ = [("format", C.c_int32), ("keep_pencil", C.c_int32)]


class SystemInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("N", C.c_int64), ("nnz", C.c_int64), ("h", C.c_double),
                ("rho", C.c_double), ("is_stencil", C.c_int32), ("has_pencil", C.c_int32)]


class AmgOpts(C.Structure):
    _fields_ = [("theta", C.c_double), ("smoother", C.c_int32), ("degree", C.c_int32),
                ("cheb_ratio", C.c_double), ("coarse_max", C.c_int32),
                ("max_levels", C.c_int32), ("precision", C.c_int32), ("seed", C.c_uint32),
                ("rho_setup", C.c_double), ("coarsening", C.c_int32), ("max_row", C.c_int32),
                ("order", C.c_int32)]


class HierInfo(C.Structure):
    _fields_ = [("levels", C.c_int32), ("rows", C.c_int64 * 32), ("nnz", C.c_int64 * 32),
                ("lmax", C.c_double * 32), ("setup_ms", C.c_double), ("pnnz", C.c_int64 * 32),
                ("rnnz", C.c_int64 * 32), ("finest_stencil", C.c_int32),
                ("colours", C.c_int32 * 32)]


class PcgOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("stop", C.c_int32),
                ("flexible", C.c_int32), ("use_x0", C.c_int32), ("use_graph", C.c_int32),
                ("cancel_host", C.POINTER(C.c_int32))]


class PcgResult(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("relres", C.c_double),
                ("prec_relres", C.c_double), ("solve_ms", C.c_double)]

    def as_dict(self):
        return {"iterations": self.iterations, "status": STATUS_NAMES.get(self.status),
                "relres": self.relres, "prec_relres": self.prec_relres,
                "solve_ms": self.solve_ms}


_lock = threading.Lock()
_lib = None
VP = C.c_void_p
P = C.POINTER

# name -> (restype, argtypes); this list mirrors include/femamg.h
class MeshDesc(C.Structure):
    _fields_ = [("nv", C.c_int64), ("nt", C.c_int64), ("xyz", P(C.c_double)),
                ("tet", P(C.c_int32)), ("dirichlet", P(C.c_uint8))]


class BddcOpts(C.Structure):
    _fields_ = [("slabs", C.c_int32), ("slab_begin", C.c_int32), ("slab_end", C.c_int32),
                ("inner_tol", C.c_double)]


# void (*)(double* buf, int64_t count, int32_t on_device, void* ctx)
ALLREDUCE_FN = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.c_int64, C.c_int32, C.c_void_p)


class ErrorsResult(C.Structure):
    _fields_ = [("l2sq", C.c_double), ("h1sq", C.c_double)]


class MeshInfo(C.Structure):
    _fields_ = [("nv", C.c_int64), ("nt", C.c_int64)]


class RefineStats(C.Structure):
    _fields_ = [("passes", C.c_int32), ("new_vertices", C.c_int64), ("new_tets", C.c_int64)]


SIGNATURES = {
    "fem_assemble": (C.c_int, [P(KuhnDesc), C.c_double, P(Target), P(AssembleOpts), VP, P(VP)]),
    "fem_system_get_info": (C.c_int, [VP, P(SystemInfo)]),
    "fem_system_get_rhs": (C.c_int, [VP, VP, VP]),
    "fem_assemble_rhs": (C.c_int, [VP, P(Target), VP, VP]),
    "fem_assemble_rhs_noalloc": (C.c_int, [VP, P(Target), VP, VP]),
    "fem_assemble_mesh": (C.c_int, [P(MeshDesc), C.c_double, P(Target), P(AssembleOpts), VP,
                                    P(VP)]),
    "fem_errors": (C.c_int, [VP, VP, P(Target), C.c_double, C.c_int32, VP, P(ErrorsResult)]),
    "fem_recover": (C.c_int, [VP, VP, P(Target), VP, VP, VP]),
    "fem_measure_fp64_rate": (C.c_int, [C.c_int32, VP, P(C.c_double)]),
    "fem_error_hm1": (C.c_int, [VP, VP, P(Target), C.c_double, C.c_double, VP, P(C.c_double),
                                P(PcgResult)]),
    "fem_error_indicator": (C.c_int, [VP, VP, P(Target), C.c_int32, VP, VP, P(C.c_double)]),
    "fem_mark_bulk": (C.c_int, [VP, C.c_int64, C.c_double, VP, VP, P(C.c_double),
                                P(C.c_int64)]),
    "fem_mesh_create": (C.c_int, [P(MeshDesc), VP, P(VP)]),
    "fem_mesh_get_info": (C.c_int, [VP, P(MeshInfo)]),
    "fem_mesh_download": (C.c_int, [VP, VP, VP, VP, VP]),
    "fem_mesh_refine": (C.c_int, [VP, VP, VP, P(RefineStats)]),
    "fem_assemble_on_mesh": (C.c_int, [VP, C.c_double, P(Target), P(AssembleOpts), VP, P(VP)]),
    "fem_mesh_destroy": (None, [VP]),
    "fem_system_export": (C.c_int, [VP, C.c_int32, VP, VP, VP, VP]),
    "fem_system_dof_vertices": (C.c_int, [VP, VP, VP]),
    "fem_spmv": (C.c_int, [VP, VP, VP, VP]),
    "fem_system_destroy": (None, [VP]),
    "amg_setup": (C.c_int, [VP, P(AmgOpts), VP, P(VP)]),
    "amg_default_opts": (None, [P(AmgOpts)]),
    "amg_hier_get_info": (C.c_int, [VP, P(HierInfo)]),
    "amg_hier_export": (C.c_int, [VP, C.c_int32, C.c_int32, VP, VP, VP, P(C.c_int64), VP]),
    "amg_vcycle": (C.c_int, [VP, VP, VP, VP]),
    "amg_vcycle_graph": (C.c_int, [VP, VP, VP, C.c_int32, VP, P(C.c_double)]),
    "fem_spmv_timed": (C.c_int, [VP, VP, VP, C.c_int32, VP, P(C.c_double)]),
    "fem_bddc_partition": (C.c_int, [C.c_int32, C.c_int32, P(C.c_int32), P(C.c_int64)]),
    "bddc_setup": (C.c_int, [VP, P(BddcOpts), ALLREDUCE_FN, VP, VP, P(VP)]),
    "bddc_solve": (C.c_int, [VP, VP, VP, P(PcgOpts), ALLREDUCE_FN, VP, VP, P(PcgResult)]),
    "bddc_get_setup_ms": (C.c_double, [VP]),
    "bddc_destroy": (None, [VP]),
    "amg_galerkin_timed": (C.c_int, [VP, C.c_int32, C.c_int32, VP, P(C.c_double),
                                     P(C.c_int64)]),
    "amg_hier_destroy": (None, [VP]),
    "pcg_default_opts": (None, [P(PcgOpts)]),
    "pcg_solve": (C.c_int, [VP, VP, VP, VP, C.c_int32, P(C.c_double), P(PcgOpts), VP,
                            P(PcgResult)]),
    "pcg_batch_create": (C.c_int, [VP, VP, C.c_int32, P(PcgOpts), VP, P(VP)]),
    "pcg_batch_admit": (C.c_int, [VP, VP, C.c_double, P(C.c_int32), VP]),
    "pcg_batch_step": (C.c_int, [VP, C.c_int32, VP]),
    "pcg_batch_poll": (C.c_int, [VP, P(C.c_int32), P(C.c_int32), P(C.c_double), VP]),
    "pcg_batch_retire": (C.c_int, [VP, C.c_int32, VP, VP]),
    "pcg_batch_footprint": (C.c_int64, [VP, VP, C.c_int32]),
    "pcg_batch_destroy": (None, [VP]),
    "fem_last_error": (C.c_char_p, []),
    "fem_autotune_report": (C.c_char_p, []),
    "fem_autotune_clear": (None, []),
    "fem_autotune_pin": (C.c_int, [C.c_char_p, C.c_int32]),
    "fem_version": (C.c_char_p, []),
    "fem_kernel_launches": (C.c_int64, []),
}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libfemamg.so is not built (run paper_2102_03515_gb300.build)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, what: str):
    if status != FEM_OK:
        raise FemError(status, lib().fem_last_error().decode() or what)


def _stream(stream):
    if stream is None:
        import torch
        return VP(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return VP(stream)
    return VP(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.is_contiguous(), "device buffers must be contiguous"
    return VP(t.data_ptr())


def _dp(a):
    return a.ctypes.data_as(P(C.c_double))


def fem_last_error() -> str:
    return lib().fem_last_error().decode()


def fem_version() -> str:
    return lib().fem_version().decode()


def fem_measure_fp64_rate(reps: int = 10, stream=None) -> float:
    """Measured FP64 FMA throughput of the current GPU, TFLOP/s."""
    v = C.c_double(0.0)
    _check(lib().fem_measure_fp64_rate(int(reps), _stream(stream), C.byref(v)),
           "fem_measure_fp64_rate")
    return v.value


def fem_kernel_launches() -> int:
    return int(lib().fem_kernel_launches())


def fem_autotune_report() -> dict:
    """The autotuner's choices and timings (parsed JSON)."""
    import json
    return json.loads(lib().fem_autotune_report().decode())


def fem_autotune_clear() -> None:
    lib().fem_autotune_clear()


def fem_autotune_pin(kernel: str, variant: int) -> None:
    """Force `variant` of a kernel family for every shape (variant < 0: unpin)."""
    _check(lib().fem_autotune_pin(kernel.encode(), int(variant)), "fem_autotune_pin")


# ------------------------------------------------------------------ system

def _target(target: dict, keep: list) -> Target:
    t = Target()
    t.kind = FEM_TARGET[target["kind"]]
    t.lo = float(target.get("lo", 0.25))
    t.hi = float(target.get("hi", 0.75))
    if target["kind"] == "quadvals":
        # ubar at the 4 load-vector points of every tet: a contiguous float64 device tensor
        v = target["values"]
        assert v.is_cuda and v.dtype.is_floating_point and v.element_size() == 8, \
            "quadvals: a float64 CUDA tensor [nt, 4]"
        v = v.contiguous()
        keep.append(v)
        t.quadvals_dev = v.data_ptr()
    if target["kind"] == "bumps":
        c = np.ascontiguousarray(target["centers"], dtype=np.float64)
        w = np.ascontiguousarray(target["widths"], dtype=np.float64)
        a = np.ascontiguousarray(target["amps"], dtype=np.float64)
        keep += [c, w, a]
        t.nb = len(w)
        t.centers_host, t.widths_host, t.amps_host = _dp(c), _dp(w), _dp(a)
    return t


def fem_assemble_rhs(sys, target: dict, f, stream=None):
    keep = []
    t = _target(target, keep)
    _check(lib().fem_assemble_rhs(sys, C.byref(t), _ptr(f), _stream(stream)), "fem_assemble_rhs")


def fem_errors(sys, u, target: dict, scale: float = 1.0, qlevel: int = 1, stream=None) -> dict:
    """{"l2sq": ||w - u_h||^2, "h1sq": ||grad(w - u_h)||^2} for w = scale * target."""
    keep = []
    t = _target(target, keep)
    r = ErrorsResult()
    _check(lib().fem_errors(sys, _ptr(u), C.byref(t), float(scale), int(qlevel), _stream(stream),
                            C.byref(r)), "fem_errors")
    return {"l2sq": r.l2sq, "h1sq": r.h1sq}


def fem_error_hm1(sys, u, target: dict, scale: float = 1.0, tol: float = 1e-10,
                  stream=None) -> dict:
    """{"hm1sq": r^T K^-1 r with r = scale * f(target) - M u, "solve": the stiffness solve's
    result} (the discrete H^-1 error of w - u_h, w = scale * target)."""
    keep = []
    t = _target(target, keep)
    v = C.c_double(0.0)
    r = PcgResult()
    st = lib().fem_error_hm1(sys, _ptr(u), C.byref(t), float(scale), float(tol),
                             _stream(stream), C.byref(v), C.byref(r))
    if st not in (FEM_OK, FEM_ENOCONV):   # FEM_ENOCONV: the value of the last iterate
        raise FemError(st, fem_last_error() or "fem_error_hm1")
    return {"hm1sq": v.value, "solve": r.as_dict()}


def fem_recover(sys, u, target: dict, z=None, p=None, stream=None):
    """Control z = (ubar - u) / rho and adjoint p = -rho u at the unknowns."""
    keep = []
    t = _target(target, keep)
    _check(lib().fem_recover(sys, _ptr(u), C.byref(t), _ptr(z) if z is not None else None,
                             _ptr(p) if p is not None else None, _stream(stream)), "fem_recover")


def fem_assemble_rhs_noalloc(sys, target: dict, f, stream=None):
    """fem_assemble_rhs for callers that cannot allocate device memory (n <= 64)."""
    keep = []
    t = _target(target, keep)
    _check(lib().fem_assemble_rhs_noalloc(sys, C.byref(t), _ptr(f), _stream(stream)),
           "fem_assemble_rhs_noalloc")


def fem_assemble(n: int, rho: float, target: dict, xyz=None, fmt: int = FEM_FMT_AUTO,
                 keep_pencil: bool = False, stream=None):
    """Assemble (rho K + M) u = f on the Kuhn mesh; returns the system handle."""
    keep = []
    d = KuhnDesc()
    d.n = n
    if xyz is not None:
        xa = np.ascontiguousarray(xyz, dtype=np.float64)
        assert xa.size == 3 * (n + 1) ** 3
        keep.append(xa)
        d.xyz_host = _dp(xa)
    t = _target(target, keep)
    o = AssembleOpts(fmt, 1 if keep_pencil else 0)
    h = VP()
    _check(lib().fem_assemble(C.byref(d), rho, C.byref(t), C.byref(o), _stream(stream),
                              C.byref(h)), "fem_assemble")
    return h


def fem_assemble_mesh(xyz, tets, dirichlet, rho: float, target: dict, keep_pencil: bool = False,
                      stream=None):
    """Assemble (rho K + M) u = f on a general tetrahedral mesh (host arrays: xyz [nv, 3],
    tets [nt, 4], dirichlet [nv] flags); returns the system handle."""
    keep = []
    xa = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    ta = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    da = np.ascontiguousarray(dirichlet, dtype=np.uint8).reshape(-1)
    assert len(da) == len(xa)
    keep += [xa, ta, da]
    d = MeshDesc(len(xa), len(ta), _dp(xa), ta.ctypes.data_as(P(C.c_int32)),
                 da.ctypes.data_as(P(C.c_uint8)))
    t = _target(target, keep)
    o = AssembleOpts(FEM_FMT_CSR, 1 if keep_pencil else 0)
    h = VP()
    _check(lib().fem_assemble_mesh(C.byref(d), rho, C.byref(t), C.byref(o), _stream(stream),
                                   C.byref(h)), "fem_assemble_mesh")
    return h


# ------------------------------------------------------------------ adaptive meshes

def fem_error_indicator(sys, u, target: dict, eta2, qlevel: int = 1, stream=None) -> float:
    """Residual indicator eta_T^2 of every tet into eta2 (device, nt doubles); returns the
    sum."""
    keep = []
    t = _target(target, keep)
    tot = C.c_double()
    _check(lib().fem_error_indicator(sys, _ptr(u), C.byref(t), int(qlevel), _ptr(eta2),
                                     _stream(stream), C.byref(tot)), "fem_error_indicator")
    return tot.value


def fem_mark_bulk(eta2, theta: float, mark, stream=None):
    """Bulk marking of eta2 (device doubles) into mark (device uint8); returns
    (threshold, number marked)."""
    thr = C.c_double()
    nm = C.c_int64()
    _check(lib().fem_mark_bulk(_ptr(eta2), int(eta2.numel()), float(theta), _ptr(mark),
                               _stream(stream), C.byref(thr), C.byref(nm)), "fem_mark_bulk")
    return thr.value, nm.value


def fem_mesh_create(xyz, tets, dirichlet, stream=None):
    """Copy a conforming tetrahedral mesh (host arrays) to the device; returns the handle."""
    xa = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    ta = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    da = np.ascontiguousarray(dirichlet, dtype=np.uint8).reshape(-1)
    assert len(da) == len(xa)
    d = MeshDesc(len(xa), len(ta), _dp(xa), ta.ctypes.data_as(P(C.c_int32)),
                 da.ctypes.data_as(P(C.c_uint8)))
    h = VP()
    _check(lib().fem_mesh_create(C.byref(d), _stream(stream), C.byref(h)), "fem_mesh_create")
    return h


def fem_mesh_get_info(mesh) -> dict:
    i = MeshInfo()
    _check(lib().fem_mesh_get_info(mesh, C.byref(i)), "fem_mesh_get_info")
    return {"nv": i.nv, "nt": i.nt}


def fem_mesh_download(mesh, stream=None):
    """(xyz [nv, 3], tets [nt, 4] int32, dirichlet [nv] uint8) as numpy arrays."""
    i = fem_mesh_get_info(mesh)
    xyz = np.empty((i["nv"], 3), dtype=np.float64)
    tets = np.empty((i["nt"], 4), dtype=np.int32)
    d = np.empty(i["nv"], dtype=np.uint8)
    _check(lib().fem_mesh_download(mesh, VP(xyz.ctypes.data), VP(tets.ctypes.data),
                                   VP(d.ctypes.data), _stream(stream)), "fem_mesh_download")
    return xyz, tets, d


def fem_mesh_refine(mesh, mark, stream=None) -> dict:
    """Longest-edge bisection of the tets with mark[t] != 0 (device uint8) and closure."""
    r = RefineStats()
    _check(lib().fem_mesh_refine(mesh, _ptr(mark), _stream(stream), C.byref(r)),
           "fem_mesh_refine")
    return {"passes": r.passes, "new_vertices": r.new_vertices, "new_tets": r.new_tets}


def fem_assemble_on_mesh(mesh, rho: float, target: dict, keep_pencil: bool = False,
                         stream=None):
    """fem_assemble_mesh on a device mesh; returns the system handle."""
    keep = []
    t = _target(target, keep)
    o = AssembleOpts(FEM_FMT_CSR, 1 if keep_pencil else 0)
    h = VP()
    _check(lib().fem_assemble_on_mesh(mesh, float(rho), C.byref(t), C.byref(o), _stream(stream),
                                      C.byref(h)), "fem_assemble_on_mesh")
    return h


def fem_mesh_destroy(mesh) -> None:
    lib().fem_mesh_destroy(mesh)


def fem_system_dof_vertices(sys, vert, stream=None):
    """vert (device int64 tensor [N]) <- the vertex index of every unknown."""
    _check(lib().fem_system_dof_vertices(sys, _ptr(vert), _stream(stream)),
           "fem_system_dof_vertices")


def fem_system_get_info(sys) -> dict:
    i = SystemInfo()
    _check(lib().fem_system_get_info(sys, C.byref(i)), "fem_system_get_info")
    return {"n": i.n, "N": i.N, "nnz": i.nnz, "h": i.h, "rho": i.rho,
            "is_stencil": bool(i.is_stencil), "has_pencil": bool(i.has_pencil)}


def fem_system_get_rhs(sys, f, stream=None):
    _check(lib().fem_system_get_rhs(sys, _ptr(f), _stream(stream)), "fem_system_get_rhs")


def fem_system_export(sys, which, rowptr, col, val, stream=None):
    _check(lib().fem_system_export(sys, which, _ptr(rowptr), _ptr(col), _ptr(val),
                                   _stream(stream)), "fem_system_export")


def fem_spmv(sys, x, y, stream=None):
    _check(lib().fem_spmv(sys, _ptr(x), _ptr(y), _stream(stream)), "fem_spmv")


def fem_spmv_timed(sys, x, y, reps: int = 20, stream=None) -> float:
    """y = A x applied `reps` times; returns the mean ms of one operator launch."""
    ms = C.c_double(0.0)
    _check(lib().fem_spmv_timed(sys, _ptr(x), _ptr(y), int(reps), _stream(stream), C.byref(ms)),
           "fem_spmv_timed")
    return ms.value


def fem_system_destroy(sys):
    lib().fem_system_destroy(sys)


# ------------------------------------------------------------------ AMG

def amg_default_opts(**kw) -> AmgOpts:
    o = AmgOpts()
    lib().amg_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def amg_setup(sys, stream=None, **kw):
    o = amg_default_opts(**kw)
    h = VP()
    _check(lib().amg_setup(sys, C.byref(o), _stream(stream), C.byref(h)), "amg_setup")
    return h


def amg_hier_get_info(h) -> dict:
    i = HierInfo()
    _check(lib().amg_hier_get_info(h, C.byref(i)), "amg_hier_get_info")
    L = i.levels
    return {"levels": L, "rows": list(i.rows[:L]), "nnz": list(i.nnz[:L]),
            "lmax": list(i.lmax[:L]), "setup_ms": i.setup_ms, "pnnz": list(i.pnnz[:L]),
            "rnnz": list(i.rnnz[:L]), "finest_stencil": bool(i.finest_stencil),
            "colours": list(i.colours[:L])}


def amg_vcycle_graph(h, r, z, reps: int = 20, stream=None) -> float:
    """z = V(r) applied `reps` times from a CUDA graph; returns ms per application."""
    ms = C.c_double(0.0)
    _check(lib().amg_vcycle_graph(h, _ptr(r), _ptr(z), int(reps), _stream(stream), C.byref(ms)),
           "amg_vcycle_graph")
    return ms.value


def amg_galerkin_timed(h, level: int = 0, reps: int = 5, stream=None):
    """Level `level`'s Galerkin product recomputed `reps` times: (ms per product, entries of
    A P)."""
    ms = C.c_double(0.0)
    ape = C.c_int64(0)
    _check(lib().amg_galerkin_timed(h, int(level), int(reps), _stream(stream), C.byref(ms),
                                    C.byref(ape)), "amg_galerkin_timed")
    return ms.value, int(ape.value)


def amg_hier_export(h, level, which, rowptr=None, col=None, val=None, stream=None) -> int:
    nnz = C.c_int64(0)
    _check(lib().amg_hier_export(h, level, which, _ptr(rowptr), _ptr(col), _ptr(val),
                                 C.byref(nnz), _stream(stream)), "amg_hier_export")
    return nnz.value


def amg_vcycle(h, r, z, stream=None):
    _check(lib().amg_vcycle(h, _ptr(r), _ptr(z), _stream(stream)), "amg_vcycle")


def amg_hier_destroy(h):
    lib().amg_hier_destroy(h)


# ------------------------------------------------------------------ PCG

def pcg_default_opts(**kw) -> PcgOpts:
    o = PcgOpts()
    lib().pcg_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def pcg_solve(sys, hier, f, u, nrhs: int = 1, rho_k=None, stream=None, **kw):
    """Solve; returns a list of per-column result dicts (one for nrhs = 1)."""
    o = pcg_default_opts(**kw)
    res = (PcgResult * nrhs)()
    rk = None
    if rho_k is not None:
        rk = np.ascontiguousarray(rho_k, dtype=np.float64)
        assert len(rk) == nrhs
    st = lib().pcg_solve(sys, hier, _ptr(f), _ptr(u), nrhs, _dp(rk) if rk is not None else None,
                         C.byref(o), _stream(stream), res)
    out = [res[i].as_dict() for i in range(nrhs)]
    if st not in (FEM_OK, FEM_ENOCONV):
        raise FemError(st, fem_last_error())
    return out


# ------------------------------------------------------------------ batch sessions

def pcg_batch_create(sys, hier, slots: int, stream=None, **kw):
    o = pcg_default_opts(**kw)
    h = VP()
    _check(lib().pcg_batch_create(sys, hier, slots, C.byref(o), _stream(stream), C.byref(h)),
           "pcg_batch_create")
    return h


def pcg_batch_admit(b, f, rho: float, stream=None) -> int:
    slot = C.c_int32(-1)
    _check(lib().pcg_batch_admit(b, _ptr(f), rho, C.byref(slot), _stream(stream)),
           "pcg_batch_admit")
    return slot.value


def pcg_batch_step(b, iters: int = 1, stream=None):
    _check(lib().pcg_batch_step(b, iters, _stream(stream)), "pcg_batch_step")


def pcg_batch_poll(b, slots: int, stream=None):
    st = np.zeros(slots, dtype=np.int32)
    it = np.zeros(slots, dtype=np.int32)
    rr = np.zeros(slots, dtype=np.float64)
    _check(lib().pcg_batch_poll(b, st.ctypes.data_as(P(C.c_int32)),
                                it.ctypes.data_as(P(C.c_int32)), _dp(rr), _stream(stream)),
           "pcg_batch_poll")
    return st, it, rr


def pcg_batch_retire(b, slot: int, u, stream=None):
    _check(lib().pcg_batch_retire(b, slot, _ptr(u), _stream(stream)), "pcg_batch_retire")


def pcg_batch_footprint(sys, hier, slots: int) -> int:
    return int(lib().pcg_batch_footprint(sys, hier, slots))


def pcg_batch_destroy(b):
    lib().pcg_batch_destroy(b)


# ------------------------------------------------------------------ BDDC (Sec. 3.2)

def fem_bddc_partition(n: int, slabs: int):
    """(layer_begin[0..slabs], interface unknowns) of the slab split; host only."""
    lb = (C.c_int32 * (slabs + 1))()
    ni = C.c_int64(0)
    _check(lib().fem_bddc_partition(int(n), int(slabs), lb, C.byref(ni)), "fem_bddc_partition")
    return [int(v) for v in lb], int(ni.value)


class _DevView:
    """A device buffer given by pointer and length, seen by torch without a copy."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3}


def make_allreduce(group=None):
    """The sum over the ranks of a torch.distributed group, as the library's all-reduce
    callback: device buffers are summed in place through the group's backend (NCCL on
    GPUs), host buffers through a CPU tensor.  Keep the returned object alive while the
    library may call it."""
    import numpy as np
    import torch
    import torch.distributed as dist

    def fn(buf, count, on_device, ctx):
        if count <= 0:
            return
        addr = C.cast(buf, C.c_void_p).value
        if on_device:
            t = torch.as_tensor(_DevView(addr, count), device="cuda")
            dist.all_reduce(t, group=group)
        else:
            a = np.ctypeslib.as_array(buf, shape=(int(count),))
            t = torch.from_numpy(a.copy())
            dist.all_reduce(t, group=group)
            a[:] = t.numpy()

    return ALLREDUCE_FN(fn)


def bddc_setup(sys, slabs: int, slab_begin: int = 0, slab_end: int = 0, inner_tol: float = 1e-13,
               allreduce=None, stream=None):
    o = BddcOpts(int(slabs), int(slab_begin), int(slab_end), float(inner_tol))
    h = VP()
    cb = allreduce if allreduce is not None else ALLREDUCE_FN()
    _check(lib().bddc_setup(sys, C.byref(o), cb, None, _stream(stream), C.byref(h)), "bddc_setup")
    return h


def bddc_solve(b, f, u, allreduce=None, stream=None, **kw):
    """Solve with the BDDC-preconditioned interface CG; returns the result dict."""
    o = pcg_default_opts(**kw)
    r = PcgResult()
    cb = allreduce if allreduce is not None else ALLREDUCE_FN()
    st = lib().bddc_solve(b, _ptr(f), _ptr(u), C.byref(o), cb, None, _stream(stream), C.byref(r))
    out = r.as_dict()
    if st not in (FEM_OK, FEM_ENOCONV):
        raise FemError(st, fem_last_error())
    return out


def bddc_get_setup_ms(b) -> float:
    return float(lib().bddc_get_setup_ms(b))


def bddc_destroy(b):
    lib().bddc_destroy(b)
