"""Python binding of libcmcg (ctypes; argument marshalling only).

Every function has the name of the C entry point it wraps (``include/cmcg.h``)
and does no arithmetic of its own: arrays are checked for dtype / shape /
contiguity and their pointers passed through.  Host entry points take numpy
arrays; ``*_device`` entry points take CUDA tensors (torch) whose
``data_ptr()`` is passed, and run on the handle's stream (set with
``cmcg_set_stream``).  If ``libcmcg.so`` is missing the import fails: there is
no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcmcg.so")

CMCG_OK = 0
CMCG_NOT_CONVERGED = 1
CMCG_PENDING = 2
CMCG_ERR_INVALID_ARG = -1
CMCG_ERR_NONCONFORMING_MESH = -2
CMCG_ERR_OUT_OF_MEMORY = -3
CMCG_ERR_UNSTABLE = -4
CMCG_ERR_CG_BREAKDOWN = -5
CMCG_ERR_NONFINITE = -6
CMCG_ERR_DEVICE_TIMEOUT = -7
CMCG_ERR_CUDA = -8
CMCG_ERR_NO_DEVICE = -9
CMCG_FP64, CMCG_FP32 = 0, 1
CMCG_FLUX_UPWIND, CMCG_FLUX_CENTRED = 0, 1


class cmcg_mesh(C.Structure):
    _fields_ = [("nv", C.c_int64), ("verts", C.POINTER(C.c_double)), ("nt", C.c_int64),
                ("tets", C.POINTER(C.c_int32)), ("face_tags", C.POINTER(C.c_uint8))]


class cmcg_options(C.Structure):
    _fields_ = [("order", C.c_int), ("precision", C.c_int), ("flux", C.c_int), ("steps_per_period", C.c_int),
                ("c_q", C.c_double), ("hbm_budget_bytes", C.c_int64), ("device", C.c_int),
                ("stage_variant", C.c_int), ("stage_overlap", C.c_int), ("launch_graphs", C.c_int),
                ("reserved", C.c_int * 4)]


class cmcg_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("periods", C.c_int), ("steps_per_period", C.c_int), ("status", C.c_int),
                ("rel_residual", C.c_double), ("dt", C.c_double), ("solve_ms", C.c_double),
                ("reserved", C.c_double * 5)]


class cmcg_problem(C.Structure):
    _fields_ = [("mesh", C.POINTER(cmcg_mesh)), ("eps", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)),
                ("omega", C.c_double)]


class cmcg_server_options(C.Structure):
    _fields_ = [("device", C.c_int), ("precision", C.c_int), ("max_batch", C.c_int), ("workers", C.c_int),
                ("max_wait_ms", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int),
                ("hbm_budget_bytes", C.c_int64), ("stage_variant", C.c_int), ("reserved", C.c_int * 7)]


class CMCGError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {cmcg_status_string(code)} ({code})")
        self.code = code


_dp = C.POINTER(C.c_double)
_vp = C.c_void_p


def _load() -> C.CDLL:
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libcmcg.so not built at {_LIB_PATH}; run paper_2106_02858_gb300/build.py "
                          "(or __graft_entry__.build())")
    lib = C.CDLL(_LIB_PATH)
    sig = {
        "cmcg_default_options": (None, [C.POINTER(cmcg_options)]),
        "cmcg_status_string": (C.c_char_p, [C.c_int]),
        "cmcg_validate": (C.c_int, [C.POINTER(cmcg_mesh), _dp, _dp, C.c_double, C.POINTER(cmcg_options),
                                    C.POINTER(C.c_int)]),
        "cmcg_reference_matrices": (C.c_int, [C.c_int, _dp, _dp, _dp, _dp, _dp]),
        "cmcg_create": (C.c_int, [C.POINTER(cmcg_mesh), _dp, _dp, C.c_double, C.POINTER(cmcg_options),
                                  C.POINTER(_vp)]),
        "cmcg_create_batch": (C.c_int, [C.c_int, C.POINTER(cmcg_problem), C.POINTER(cmcg_options), C.POINTER(_vp)]),
        "cmcg_batch_size": (C.c_int, [_vp]),
        "cmcg_get_problem": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "cmcg_solve_batch": (C.c_int, [_vp, C.POINTER(_dp), C.POINTER(_dp), C.c_double, C.c_int, C.POINTER(_dp),
                                       C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp), C.POINTER(cmcg_info)]),
        "cmcg_solve_batch_device": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.c_double, C.c_int,
                                              C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp),
                                              C.POINTER(cmcg_info)]),
        "cmcg_solve_batch_n": (C.c_int, [_vp, C.c_int, C.POINTER(_dp), C.POINTER(_dp), C.c_double, C.c_int,
                                         C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp),
                                         C.POINTER(cmcg_info)]),
        "cmcg_device_bytes": (C.c_int64, [_vp]),
        "cmcg_fw_solve": (C.c_int, [_vp, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp]),
        "cmcg_set_boundary_data": (C.c_int, [_vp, C.c_int, _dp, _dp]),
        "cmcg_set_conductivity": (C.c_int, [_vp, C.c_int, _dp]),
        "cmcg_fw_solve_batch": (C.c_int, [_vp, C.c_int, C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp),
                                          C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp)]),
        "cmcg_server_default_options": (None, [C.POINTER(cmcg_server_options)]),
        "cmcg_server_create": (C.c_int, [C.POINTER(cmcg_server_options), C.POINTER(_vp)]),
        "cmcg_server_add_model": (C.c_int, [_vp, C.POINTER(cmcg_mesh), _dp, _dp, C.c_double, C.c_int, C.c_int,
                                            C.POINTER(C.c_int)]),
        "cmcg_server_submit": (C.c_int, [_vp, C.c_int, _dp, _dp, C.POINTER(C.c_int64)]),
        "cmcg_server_poll": (C.c_int, [_vp, C.c_int64, C.c_int, _dp, _dp, _dp, _dp, C.POINTER(cmcg_info), _dp]),
        "cmcg_server_stats": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                        C.POINTER(C.c_int)]),
        "cmcg_server_destroy": (None, [_vp]),
        "cmcg_destroy": (None, [_vp]),
        "cmcg_set_stream": (C.c_int, [_vp, _vp]),
        "cmcg_get_tuning": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "cmcg_get_sizes": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "dgtd_apply": (C.c_int, [_vp, C.c_double, _dp, _dp, _dp, C.c_int, _dp]),
        "dgtd_period_forward": (C.c_int, [_vp, _dp, _dp, _dp, _dp, _dp, _dp]),
        "dgtd_period_adjoint": (C.c_int, [_vp, _dp, _dp]),
        "dgtd_period_forward_device": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "dgtd_period_adjoint_device": (C.c_int, [_vp, _vp, _vp]),
        "cmcg_solve": (C.c_int, [_vp, _dp, _dp, C.c_double, C.c_int, _dp, _dp, _dp, _dp, C.POINTER(cmcg_info)]),
        "cmcg_solve_device": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_int, _vp, _vp, _vp, _vp,
                                        C.POINTER(cmcg_info)]),
        "cmcg_kernel_launches": (C.c_int64, [_vp]),
        "cmcg_inner": (C.c_int, [_vp, _dp, _dp, C.POINTER(C.c_double)]),
        "cmcg_inner_noalloc": (C.c_int, [C.c_int, C.c_int64, _vp, _vp, _vp, _vp, _vp]),
        "cmcg_profile_enable": (C.c_int, [_vp, C.c_int]),
        "cmcg_measure_peaks": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "cmcg_partition_slabs": (C.c_int, [C.POINTER(cmcg_mesh), C.c_int, C.c_int, C.POINTER(C.c_int32)]),
        "cmcg_slot_admit": (C.c_int, [_vp, C.c_int, _dp, _dp]),
        "cmcg_slot_round": (C.c_int, [_vp, C.c_double, C.c_int, C.POINTER(C.c_int)]),
        "cmcg_slot_take": (C.c_int, [_vp, C.c_int, _dp, _dp, _dp, _dp, C.POINTER(cmcg_info)]),
        "cmcg_slot_state": (C.c_int, [_vp, C.c_int]),
        "cmcg_slot_state_bytes": (C.c_int64, [_vp, C.c_int]),
        "cmcg_slot_save": (C.c_int, [_vp, C.c_int, _vp, C.c_int64]),
        "cmcg_slot_restore": (C.c_int, [_vp, C.c_int, _vp, C.c_int64]),
        "cmcg_solve_multifreq": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(_dp), C.POINTER(_dp),
                                           C.c_double, C.c_int, C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp),
                                           C.POINTER(_dp), C.POINTER(cmcg_info)]),
        "cmcg_shard_plan": (C.c_int, [C.POINTER(cmcg_mesh), C.POINTER(C.c_int32), C.c_int, C.c_int,
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_uint8)]),
        "cmcg_create_sharded": (C.c_int, [C.POINTER(cmcg_mesh), _dp, _dp, C.c_double, C.POINTER(cmcg_options),
                                          C.c_int, C.POINTER(C.c_int32), C.POINTER(_vp)]),
        "cmcg_profile_read": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                        C.POINTER(C.c_int64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("cmcg_default_options", "cmcg_status_string", "cmcg_validate", "cmcg_reference_matrices", "cmcg_create",
            "cmcg_destroy", "cmcg_set_stream", "cmcg_get_sizes", "dgtd_apply", "dgtd_period_forward",
            "dgtd_period_adjoint", "dgtd_period_forward_device", "dgtd_period_adjoint_device", "cmcg_solve",
            "cmcg_solve_device", "cmcg_kernel_launches", "cmcg_profile_enable", "cmcg_profile_read",
            "cmcg_inner", "cmcg_inner_noalloc", "cmcg_get_tuning", "cmcg_create_batch", "cmcg_batch_size",
            "cmcg_get_problem", "cmcg_solve_batch", "cmcg_solve_batch_device", "cmcg_solve_batch_n",
            "cmcg_device_bytes", "cmcg_fw_solve", "cmcg_fw_solve_batch", "cmcg_set_boundary_data", "cmcg_server_default_options", "cmcg_server_create", "cmcg_server_add_model",
            "cmcg_server_submit", "cmcg_server_poll", "cmcg_server_stats", "cmcg_server_destroy",
            "cmcg_measure_peaks", "cmcg_set_conductivity", "cmcg_partition_slabs", "cmcg_shard_plan",
            "cmcg_create_sharded", "cmcg_solve_multifreq", "cmcg_slot_admit", "cmcg_slot_round", "cmcg_slot_take",
            "cmcg_slot_state", "cmcg_slot_state_bytes", "cmcg_slot_save", "cmcg_slot_restore")
CMCG_NOALLOC_MAX_TETS = 1048576


def library_path() -> str:
    return _LIB_PATH


def _f64(a, shape=None, name="array"):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError(f"{name}: expected {shape} elements, got {a.shape}")
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _dev(t):
    """data_ptr of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.itemsize == 8 and t.is_contiguous() and t.is_floating_point()):
        raise ValueError("device arguments must be contiguous float64 CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _check(rc: int, where: str, allow_not_converged: bool = False) -> int:
    if rc < 0 or (rc > 0 and not allow_not_converged):
        raise CMCGError(rc, where)
    return rc


# ---------------------------------------------------------------------------------------------
# Same-name wrappers.
# ---------------------------------------------------------------------------------------------

def cmcg_default_options(order: int = 1, precision: int = CMCG_FP64, flux: int = CMCG_FLUX_UPWIND,
                         steps_per_period: int = 0, c_q: float = 0.0, hbm_budget_bytes: int = 0,
                         device: int = 0, stage_variant: int = 0, stage_overlap: int = 0,
                         launch_graphs: int = 0) -> cmcg_options:
    o = cmcg_options()
    _lib.cmcg_default_options(C.byref(o))
    o.order, o.precision, o.flux, o.steps_per_period = order, precision, flux, steps_per_period
    o.c_q, o.hbm_budget_bytes, o.device, o.stage_variant = c_q, hbm_budget_bytes, device, stage_variant
    o.stage_overlap = stage_overlap
    o.launch_graphs = launch_graphs
    return o


def cmcg_status_string(code: int) -> str:
    return _lib.cmcg_status_string(int(code)).decode()


@dataclass
class MeshArrays:
    """Keeps the numpy arrays alive while a cmcg_mesh points at them."""

    verts: np.ndarray
    tets: np.ndarray
    tags: np.ndarray
    struct: cmcg_mesh


def make_mesh(verts, tets, tags) -> MeshArrays:
    v = np.ascontiguousarray(verts, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    g = np.ascontiguousarray(tags, dtype=np.uint8).reshape(-1, 4)
    if g.shape[0] != t.shape[0]:
        raise ValueError("tags must have one row per tetrahedron")
    m = cmcg_mesh(v.shape[0], v.ctypes.data_as(_dp), t.shape[0], t.ctypes.data_as(C.POINTER(C.c_int32)),
                  g.ctypes.data_as(C.POINTER(C.c_uint8)))
    return MeshArrays(v, t, g, m)


def cmcg_validate(mesh: MeshArrays, eps, mu, omega: float, opt: cmcg_options):
    """Returns (status, steps_per_period)."""
    e, m = _f64(eps), _f64(mu)
    steps = C.c_int(0)
    rc = _lib.cmcg_validate(C.byref(mesh.struct), _ptr(e), _ptr(m), float(omega), C.byref(opt), C.byref(steps))
    return rc, steps.value


def cmcg_reference_matrices(order: int):
    """(M, Dr, Ds, Dt, LIFT) of the library's reference element."""
    np_ = (order + 1) * (order + 2) * (order + 3) // 6
    nfp = (order + 1) * (order + 2) // 2
    M, Dr, Ds, Dt = (np.zeros((np_, np_)) for _ in range(4))
    L = np.zeros((np_, 4 * nfp))
    _check(_lib.cmcg_reference_matrices(order, _ptr(M), _ptr(Dr), _ptr(Ds), _ptr(Dt), _ptr(L)),
           "cmcg_reference_matrices")
    return M, Dr, Ds, Dt, L


class Handle:
    """Owns a cmcg_handle (cmcg_create / cmcg_create_batch / cmcg_destroy)."""

    def __init__(self, ptr: int, nt: int, np_: int, steps: int, dt: float, problems=None):
        self.ptr = C.c_void_p(ptr)
        self.nt, self.np, self.steps, self.dt = nt, np_, steps, dt
        self.problems = problems or [(nt, steps, dt)]  # (nt, steps, dt) per problem

    def close(self):
        if self.ptr is not None and self.ptr.value:
            _lib.cmcg_destroy(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def cmcg_create(mesh: MeshArrays, eps, mu, omega: float, opt: cmcg_options) -> Handle:
    e, m = _f64(eps), _f64(mu)
    out = C.c_void_p()
    _check(_lib.cmcg_create(C.byref(mesh.struct), _ptr(e), _ptr(m), float(omega), C.byref(opt), C.byref(out)),
           "cmcg_create")
    nt, np_, steps, dt, fl = C.c_int64(), C.c_int(), C.c_int(), C.c_double(), C.c_int64()
    _check(_lib.cmcg_get_sizes(out, C.byref(nt), C.byref(np_), C.byref(steps), C.byref(dt), C.byref(fl)),
           "cmcg_get_sizes")
    return Handle(out.value, nt.value, np_.value, steps.value, dt.value)


def cmcg_slot_admit(h: Handle, slot: int, j_re, j_im=None) -> None:
    nt = h.problems[slot][0]
    jr = _f64(j_re, (nt, 3, h.np), "j_re")
    ji = None if j_im is None else _f64(j_im, (nt, 3, h.np), "j_im")
    _check(_lib.cmcg_slot_admit(h.ptr, int(slot), _ptr(jr), _ptr(ji)), "cmcg_slot_admit")


def cmcg_slot_round(h: Handle, tol: float, max_iter: int):
    """One round; returns the slots whose result became ready."""
    n = len(h.problems)
    done = (C.c_int * n)()
    _check(_lib.cmcg_slot_round(h.ptr, float(tol), int(max_iter), done), "cmcg_slot_round")
    return [p for p in range(n) if done[p]]


def cmcg_slot_take(h: Handle, slot: int):
    """(e, h) complex (nt, 3, Np) and the report of a ready slot; the slot becomes empty."""
    nt = h.problems[slot][0]
    er, ei, hr, hi = (np.empty((nt, 3, h.np)) for _ in range(4))
    info = cmcg_info()
    rc = _lib.cmcg_slot_take(h.ptr, int(slot), _ptr(er), _ptr(ei), _ptr(hr), _ptr(hi), C.byref(info))
    _check(rc, "cmcg_slot_take", allow_not_converged=True)
    return er + 1j * ei, hr + 1j * hi, info


def cmcg_slot_state(h: Handle, slot: int) -> int:
    return int(_lib.cmcg_slot_state(h.ptr, int(slot)))


def cmcg_slot_save(h: Handle, slot: int) -> bytes:
    """Checkpoint of a busy slot (the slot becomes empty)."""
    n = int(_lib.cmcg_slot_state_bytes(h.ptr, int(slot)))
    if n < 0:
        raise CMCGError(n, "cmcg_slot_state_bytes")
    buf = C.create_string_buffer(n)
    _check(_lib.cmcg_slot_save(h.ptr, int(slot), buf, n), "cmcg_slot_save")
    return buf.raw


def cmcg_slot_restore(h: Handle, slot: int, state: bytes) -> None:
    buf = C.create_string_buffer(state, len(state))
    _check(_lib.cmcg_slot_restore(h.ptr, int(slot), buf, len(state)), "cmcg_slot_restore")


def cmcg_solve_multifreq(h: Handle, harmonics, j_re, j_im=None, tol: float = 1e-8, max_iter: int = 1000):
    """Several harmonics k * omega of the handle's base frequency in one CMCG solve: lists of
    (nt, 3, Np) sources per harmonic; returns ([e], [h]) complex per harmonic and the report."""
    K = len(harmonics)
    jr = [_field(h, j_re[k], 3, "j_re") for k in range(K)]
    ji = [None if (j_im is None or j_im[k] is None) else _field(h, j_im[k], 3, "j_im") for k in range(K)]
    outs = [[np.empty((h.nt, 3, h.np)) for _ in range(K)] for _ in range(4)]
    P = C.POINTER(C.c_double)
    arr = lambda xs: (P * K)(*[_ptr(x) if x is not None else P() for x in xs])
    harm = (C.c_int * K)(*[int(k) for k in harmonics])
    info = cmcg_info()
    rc = _lib.cmcg_solve_multifreq(h.ptr, K, harm, arr(jr), arr(ji), float(tol), int(max_iter), arr(outs[0]),
                                   arr(outs[1]), arr(outs[2]), arr(outs[3]), C.byref(info))
    _check(rc, "cmcg_solve_multifreq", allow_not_converged=True)
    return ([outs[0][k] + 1j * outs[1][k] for k in range(K)], [outs[2][k] + 1j * outs[3][k] for k in range(K)], info)


def cmcg_partition_slabs(mesh: MeshArrays, nparts: int, axis: int = 2) -> np.ndarray:
    """Slab partition: part index (int32) of every tetrahedron."""
    part = np.empty(mesh.struct.nt, dtype=np.int32)
    _check(_lib.cmcg_partition_slabs(C.byref(mesh.struct), int(nparts), int(axis),
                                     part.ctypes.data_as(C.POINTER(C.c_int32))), "cmcg_partition_slabs")
    return part


def cmcg_shard_plan(mesh: MeshArrays, part, nparts: int, p: int):
    """Local mesh of part p: dict with n_owned, global_of_local (owned, then ghosts),
    ghost_owner_part, ghost_owner_local and local_tags (n_local, 4)."""
    part = np.ascontiguousarray(part, dtype=np.int32)
    pp = part.ctypes.data_as(C.POINTER(C.c_int32))
    no, ng = C.c_int64(), C.c_int64()
    _check(_lib.cmcg_shard_plan(C.byref(mesh.struct), pp, int(nparts), int(p), C.byref(no), C.byref(ng),
                                None, None, None, None), "cmcg_shard_plan")
    nl = no.value + ng.value
    gl = np.empty(nl, np.int32)
    op, ol = np.empty(ng.value, np.int32), np.empty(ng.value, np.int32)
    tags = np.empty((nl, 4), np.uint8)
    i32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    _check(_lib.cmcg_shard_plan(C.byref(mesh.struct), pp, int(nparts), int(p), C.byref(no), C.byref(ng),
                                i32(gl), i32(op), i32(ol), tags.ctypes.data_as(C.POINTER(C.c_uint8))),
           "cmcg_shard_plan")
    return {"n_owned": no.value, "global_of_local": gl, "ghost_owner_part": op, "ghost_owner_local": ol,
            "local_tags": tags}


def cmcg_create_sharded(mesh: MeshArrays, eps, mu, omega: float, opt: cmcg_options, part) -> Handle:
    """One handle over the parts of ``part``; takes and returns fields of the whole mesh."""
    e, m = _f64(eps), _f64(mu)
    part = np.ascontiguousarray(part, dtype=np.int32)
    nparts = int(part.max()) + 1
    out = C.c_void_p()
    _check(_lib.cmcg_create_sharded(C.byref(mesh.struct), _ptr(e), _ptr(m), float(omega), C.byref(opt), nparts,
                                    part.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(out)), "cmcg_create_sharded")
    nt, np_, steps, dt, fl = C.c_int64(), C.c_int(), C.c_int(), C.c_double(), C.c_int64()
    _check(_lib.cmcg_get_sizes(out, C.byref(nt), C.byref(np_), C.byref(steps), C.byref(dt), C.byref(fl)),
           "cmcg_get_sizes")
    return Handle(out.value, nt.value, np_.value, steps.value, dt.value)


def cmcg_create_batch(problems, opt: cmcg_options) -> Handle:
    """``problems``: list of (MeshArrays, eps, mu, omega)."""
    keep = []
    arr = (cmcg_problem * len(problems))()
    for i, (mesh, eps, mu, omega) in enumerate(problems):
        e, m = _f64(eps), _f64(mu)
        keep += [mesh, e, m]
        arr[i] = cmcg_problem(C.pointer(mesh.struct), _ptr(e), _ptr(m), float(omega))
    out = C.c_void_p()
    _check(_lib.cmcg_create_batch(len(problems), arr, C.byref(opt), C.byref(out)), "cmcg_create_batch")
    n = _lib.cmcg_batch_size(out)
    probs = []
    for p in range(n):
        nt, steps, dt = C.c_int64(), C.c_int(), C.c_double()
        _check(_lib.cmcg_get_problem(out, p, C.byref(nt), C.byref(steps), C.byref(dt)), "cmcg_get_problem")
        probs.append((nt.value, steps.value, dt.value))
    np_ = (opt.order + 1) * (opt.order + 2) * (opt.order + 3) // 6
    return Handle(out.value, probs[0][0], np_, probs[0][1], probs[0][2], problems=probs)


def cmcg_batch_size(h: Handle) -> int:
    return int(_lib.cmcg_batch_size(h.ptr))


def cmcg_get_problem(h: Handle, p: int):
    nt, steps, dt = C.c_int64(), C.c_int(), C.c_double()
    _check(_lib.cmcg_get_problem(h.ptr, p, C.byref(nt), C.byref(steps), C.byref(dt)), "cmcg_get_problem")
    return nt.value, steps.value, dt.value


def cmcg_solve_batch(h: Handle, j_re, j_im=None, tol: float = 1e-8, max_iter: int = 1000):
    """j_re, j_im: lists of (nt_p, 3, Np) arrays.  Returns (list of e, list of h, list of cmcg_info)."""
    n = len(h.problems)
    jr = [_f64(j_re[p], (h.problems[p][0], 3, h.np), "j_re") for p in range(n)]
    ji = [None if (j_im is None or j_im[p] is None) else _f64(j_im[p], (h.problems[p][0], 3, h.np), "j_im")
          for p in range(n)]
    outs = [[np.empty((h.problems[p][0], 3, h.np)) for p in range(n)] for _ in range(4)]
    P = C.POINTER(C.c_double)
    arr = lambda xs: (P * n)(*[_ptr(x) if x is not None else P() for x in xs])
    infos = (cmcg_info * n)()
    rc = _lib.cmcg_solve_batch(h.ptr, arr(jr), arr(ji), float(tol), int(max_iter), arr(outs[0]), arr(outs[1]),
                               arr(outs[2]), arr(outs[3]), infos)
    _check(rc, "cmcg_solve_batch", allow_not_converged=True)
    e = [outs[0][p] + 1j * outs[1][p] for p in range(n)]
    hh = [outs[2][p] + 1j * outs[3][p] for p in range(n)]
    return e, hh, list(infos)


def cmcg_solve_batch_device(h: Handle, j_re, j_im, tol: float, max_iter: int, e_re, e_im, h_re, h_im):
    """Lists (one per problem) of contiguous float64 CUDA tensors; j_im entries may be None."""
    n = len(h.problems)
    arr = lambda xs: (C.c_void_p * n)(*[_dev(x) if x is not None else C.c_void_p() for x in xs])
    infos = (cmcg_info * n)()
    rc = _lib.cmcg_solve_batch_device(h.ptr, arr(j_re), arr(j_im if j_im is not None else [None] * n), float(tol),
                                      int(max_iter), arr(e_re), arr(e_im), arr(h_re), arr(h_im), infos)
    _check(rc, "cmcg_solve_batch_device", allow_not_converged=True)
    return list(infos)


def cmcg_destroy(h: Handle) -> None:
    h.close()


def cmcg_set_stream(h: Handle, stream) -> None:
    """``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(_lib.cmcg_set_stream(h.ptr, C.c_void_p(raw) if raw else None), "cmcg_set_stream")


def cmcg_get_sizes(h: Handle):
    nt, np_, steps, dt, fl = C.c_int64(), C.c_int(), C.c_int(), C.c_double(), C.c_int64()
    _check(_lib.cmcg_get_sizes(h.ptr, C.byref(nt), C.byref(np_), C.byref(steps), C.byref(dt), C.byref(fl)),
           "cmcg_get_sizes")
    return nt.value, np_.value, steps.value, dt.value, fl.value


def cmcg_get_tuning(h: Handle):
    """(variant in use, microseconds per stage of each timed variant or None)."""
    v = C.c_int()
    us = (C.c_double * 10)()
    _check(_lib.cmcg_get_tuning(h.ptr, C.byref(v), us), "cmcg_get_tuning")
    return v.value, [x if x >= 0 else None for x in us]


def cmcg_kernel_launches(h: Handle) -> int:
    return int(_lib.cmcg_kernel_launches(h.ptr))


def cmcg_inner(h: Handle, u, v) -> float:
    """(u, v)_{eps,mu} on the device (FP64 accumulation)."""
    u, v = _field(h, u, 6, "u"), _field(h, v, 6, "v")
    out = C.c_double()
    _check(_lib.cmcg_inner(h.ptr, _ptr(u), _ptr(v), C.byref(out)), "cmcg_inner")
    return out.value


def cmcg_inner_noalloc(order: int, nt: int, u, v, w, out, stream=None) -> None:
    """Allocation-free (u, v)_{eps,mu} for callers that cannot call cudaMalloc.

    u, v: float64 CUDA tensors (nt, 6, Np); w: (nt, 2) = (eps, mu) times
    |det(v1-v0, v2-v0, v3-v0)| per tetrahedron; out: a 1-element float64 CUDA
    tensor, written asynchronously on ``stream`` (torch stream, raw handle or
    None).  The first call on a device does a one-time set-up, so make it before
    any stream capture; overlapping calls race on the shared static scratch."""
    raw = getattr(stream, "cuda_stream", stream)
    rc = _lib.cmcg_inner_noalloc(int(order), int(nt), _dev(u), _dev(v), _dev(w), _dev(out),
                                 C.c_void_p(raw) if raw else None)
    if rc == CMCG_ERR_INVALID_ARG and nt > CMCG_NOALLOC_MAX_TETS:
        raise CMCGError(rc, f"cmcg_inner_noalloc: nt = {nt} exceeds the static scratch limit of "
                            f"{CMCG_NOALLOC_MAX_TETS} tetrahedra")
    _check(rc, "cmcg_inner_noalloc")


def cmcg_profile_enable(h: Handle, on: bool = True) -> None:
    _check(_lib.cmcg_profile_enable(h.ptr, int(bool(on))), "cmcg_profile_enable")


def cmcg_measure_peaks(device: int = 0):
    """(FP32 CUDA-core TFLOP/s, TF32 tensor-core TFLOP/s) measured on the device."""
    f, t = C.c_double(), C.c_double()
    _check(_lib.cmcg_measure_peaks(int(device), C.byref(f), C.byref(t)), "cmcg_measure_peaks")
    return f.value, t.value


def cmcg_profile_read(h: Handle):
    """Returns (free_sweep_ms, free_stage_launches, source_sweep_ms, source_stage_launches)."""
    fm, fs, sm, ss = C.c_double(), C.c_int64(), C.c_double(), C.c_int64()
    _check(_lib.cmcg_profile_read(h.ptr, C.byref(fm), C.byref(fs), C.byref(sm), C.byref(ss)), "cmcg_profile_read")
    return fm.value, fs.value, sm.value, ss.value


def _field(h: Handle, u, ncomp=6, name="field"):
    return _f64(u, (h.nt, ncomp, h.np), name)


def dgtd_apply(h: Handle, t: float, u, j_re=None, j_im=None, adjoint: bool = False) -> np.ndarray:
    u = _field(h, u, 6, "u")
    jr, ji = _field(h, j_re, 3, "j_re"), _field(h, j_im, 3, "j_im")
    out = np.empty((h.nt, 6, h.np))
    _check(_lib.dgtd_apply(h.ptr, float(t), _ptr(u), _ptr(jr), _ptr(ji), int(bool(adjoint)), _ptr(out)),
           "dgtd_apply")
    return out


def dgtd_period_forward(h: Handle, u0, j_re=None, j_im=None, filtered: bool = False):
    """Returns uT, or (uT, filt_re, filt_im) when ``filtered``."""
    u0 = _field(h, u0, 6, "u0")
    jr, ji = _field(h, j_re, 3, "j_re"), _field(h, j_im, 3, "j_im")
    uT = np.empty((h.nt, 6, h.np))
    fr = np.empty_like(uT) if filtered else None
    fi = np.empty_like(uT) if filtered else None
    _check(_lib.dgtd_period_forward(h.ptr, _ptr(u0), _ptr(jr), _ptr(ji), _ptr(uT), _ptr(fr), _ptr(fi)),
           "dgtd_period_forward")
    return (uT, fr, fi) if filtered else uT


def dgtd_period_adjoint(h: Handle, wT) -> np.ndarray:
    wT = _field(h, wT, 6, "wT")
    w0 = np.empty((h.nt, 6, h.np))
    _check(_lib.dgtd_period_adjoint(h.ptr, _ptr(wT), _ptr(w0)), "dgtd_period_adjoint")
    return w0


def dgtd_period_forward_device(h: Handle, u0, j_re, j_im, uT, filt_re=None, filt_im=None) -> None:
    _check(_lib.dgtd_period_forward_device(h.ptr, _dev(u0), _dev(j_re), _dev(j_im), _dev(uT), _dev(filt_re),
                                           _dev(filt_im)), "dgtd_period_forward_device")


def dgtd_period_adjoint_device(h: Handle, wT, w0) -> None:
    _check(_lib.dgtd_period_adjoint_device(h.ptr, _dev(wT), _dev(w0)), "dgtd_period_adjoint_device")


def cmcg_solve(h: Handle, j_re, j_im=None, tol: float = 1e-8, max_iter: int = 1000):
    """Returns (e, h_field, info) with e, h complex (nt, 3, Np)."""
    jr, ji = _field(h, j_re, 3, "j_re"), _field(h, j_im, 3, "j_im")
    er, ei, hr, hi = (np.empty((h.nt, 3, h.np)) for _ in range(4))
    info = cmcg_info()
    _check(_lib.cmcg_solve(h.ptr, _ptr(jr), _ptr(ji), float(tol), int(max_iter), _ptr(er), _ptr(ei), _ptr(hr),
                           _ptr(hi), C.byref(info)), "cmcg_solve", allow_not_converged=True)
    return er + 1j * ei, hr + 1j * hi, info


def cmcg_set_boundary_data(h: Handle, g_re, g_im=None, problem: int = 0) -> None:
    """Impedance-face data g, arrays (nt, 4, 3, Nfp) of problem `problem`; g_re None clears."""
    nt = h.problems[problem][0]
    nfp = {4: 3, 10: 6, 20: 10}[h.np]
    gr = None if g_re is None else _f64(g_re, (nt, 4, 3, nfp), "g_re")
    gi = None if (g_re is None or g_im is None) else _f64(g_im, (nt, 4, 3, nfp), "g_im")
    h._keep_b = (gr, gi)
    _check(_lib.cmcg_set_boundary_data(h.ptr, int(problem), _ptr(gr), _ptr(gi)), "cmcg_set_boundary_data")


def cmcg_set_conductivity(h: Handle, sigma, problem: int = 0) -> None:
    """Conductivity per tetrahedron (nt,) of problem `problem`; None removes it."""
    nt = h.problems[problem][0]
    sg = None if sigma is None else _f64(sigma, (nt,), "sigma")
    _check(_lib.cmcg_set_conductivity(h.ptr, int(problem), _ptr(sg)), "cmcg_set_conductivity")


def cmcg_fw_solve(h: Handle, j_re, j_im=None, periods: int = 1):
    """Limiting-amplitude baseline: F_psi(P_psi^periods 0).  Returns (e, h_field) complex (nt, 3, Np)."""
    jr, ji = _field(h, j_re, 3, "j_re"), _field(h, j_im, 3, "j_im")
    er, ei, hr, hi = (np.empty((h.nt, 3, h.np)) for _ in range(4))
    _check(_lib.cmcg_fw_solve(h.ptr, _ptr(jr), _ptr(ji), int(periods), _ptr(er), _ptr(ei), _ptr(hr), _ptr(hi)),
           "cmcg_fw_solve")
    return er + 1j * ei, hr + 1j * hi


def cmcg_fw_solve_batch(h: Handle, j_re, j_im=None, periods: int = 1):
    """Every problem of a batch handle; lists in and out as in cmcg_solve_batch."""
    n = len(h.problems)
    jr = [_f64(j_re[p], (h.problems[p][0], 3, h.np), "j_re") for p in range(n)]
    ji = [None if (j_im is None or j_im[p] is None) else _f64(j_im[p], (h.problems[p][0], 3, h.np), "j_im")
          for p in range(n)]
    outs = [[np.empty((h.problems[p][0], 3, h.np)) for p in range(n)] for _ in range(4)]
    P = C.POINTER(C.c_double)
    arr = lambda xs: (P * n)(*[_ptr(x) if x is not None else P() for x in xs])
    _check(_lib.cmcg_fw_solve_batch(h.ptr, int(periods), arr(jr), arr(ji), arr(outs[0]), arr(outs[1]), arr(outs[2]),
                                    arr(outs[3])), "cmcg_fw_solve_batch")
    return [outs[0][p] + 1j * outs[1][p] for p in range(n)], [outs[2][p] + 1j * outs[3][p] for p in range(n)]


def cmcg_solve_device(h: Handle, j_re, j_im, tol: float, max_iter: int, e_re, e_im, h_re, h_im) -> cmcg_info:
    info = cmcg_info()
    _check(_lib.cmcg_solve_device(h.ptr, _dev(j_re), _dev(j_im), float(tol), int(max_iter), _dev(e_re), _dev(e_im),
                                  _dev(h_re), _dev(h_im), C.byref(info)), "cmcg_solve_device",
           allow_not_converged=True)
    return info


def create_for_problem(problem, precision: int = CMCG_FP64, flux: int = CMCG_FLUX_UPWIND, steps_per_period: int = 0,
                       device: int = 0, hbm_budget_bytes: int = 0, stage_variant: int = 0, stage_overlap: int = 0,
                       launch_graphs: int = 0):
    """Convenience: cmcg_create from an ``inputs.Problem``; returns (handle, mesh arrays)."""
    mesh = make_mesh(problem.mesh.verts, problem.mesh.tets, problem.mesh.tags)
    opt = cmcg_default_options(order=problem.order, precision=precision, flux=flux,
                               steps_per_period=steps_per_period, device=device, hbm_budget_bytes=hbm_budget_bytes,
                               stage_variant=stage_variant, stage_overlap=stage_overlap,
                               launch_graphs=launch_graphs)
    return cmcg_create(mesh, problem.eps, problem.mu, problem.omega, opt), mesh


def cmcg_solve_batch_n(h: Handle, n: int, j_re, j_im=None, tol: float = 1e-8, max_iter: int = 1000):
    """Solve problems [0, n) of a batch handle; lists of n (nt_p, 3, Np) sources."""
    jr = [_f64(j_re[p], (h.problems[p][0], 3, h.np), "j_re") for p in range(n)]
    ji = [None if (j_im is None or j_im[p] is None) else _f64(j_im[p], (h.problems[p][0], 3, h.np), "j_im")
          for p in range(n)]
    outs = [[np.empty((h.problems[p][0], 3, h.np)) for p in range(n)] for _ in range(4)]
    P = C.POINTER(C.c_double)
    arr = lambda xs: (P * n)(*[_ptr(x) if x is not None else P() for x in xs])
    infos = (cmcg_info * n)()
    rc = _lib.cmcg_solve_batch_n(h.ptr, int(n), arr(jr), arr(ji), float(tol), int(max_iter), arr(outs[0]),
                                 arr(outs[1]), arr(outs[2]), arr(outs[3]), infos)
    _check(rc, "cmcg_solve_batch_n", allow_not_converged=True)
    return ([outs[0][p] + 1j * outs[1][p] for p in range(n)], [outs[2][p] + 1j * outs[3][p] for p in range(n)],
            list(infos))


def cmcg_device_bytes(h: Handle) -> int:
    return int(_lib.cmcg_device_bytes(h.ptr))


def cmcg_server_default_options(**kw) -> cmcg_server_options:
    o = cmcg_server_options()
    _lib.cmcg_server_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Server:
    """Owns a cmcg_server (cmcg_server_create / cmcg_server_destroy)."""

    def __init__(self, opt: cmcg_server_options):
        out = C.c_void_p()
        _check(_lib.cmcg_server_create(C.byref(opt), C.byref(out)), "cmcg_server_create")
        self.ptr = out
        self.models = {}  # model id -> (nt, Np)
        self._keep = []

    def close(self):
        if self.ptr is not None and self.ptr.value:
            _lib.cmcg_server_destroy(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cmcg_server_create(opt: cmcg_server_options) -> Server:
    return Server(opt)


def cmcg_server_add_model(s: Server, mesh: MeshArrays, eps, mu, omega: float, order: int, max_batch: int = 0) -> int:
    e, m = _f64(eps), _f64(mu)
    mid = C.c_int()
    _check(_lib.cmcg_server_add_model(s.ptr, C.byref(mesh.struct), _ptr(e), _ptr(m), float(omega), int(order),
                                      int(max_batch), C.byref(mid)), "cmcg_server_add_model")
    s.models[mid.value] = (mesh.tets.shape[0], (order + 1) * (order + 2) * (order + 3) // 6)
    return mid.value


def cmcg_server_submit(s: Server, model: int, j_re, j_im=None) -> int:
    nt, np_ = s.models[model]
    jr, ji = _f64(j_re, (nt, 3, np_), "j_re"), _f64(j_im, (nt, 3, np_), "j_im")
    t = C.c_int64()
    _check(_lib.cmcg_server_submit(s.ptr, int(model), _ptr(jr), _ptr(ji), C.byref(t)), "cmcg_server_submit")
    return t.value


def cmcg_server_poll(s: Server, ticket: int, model: int, wait: bool = True):
    """None while pending (wait=False); else (status, e, h, info, latency_ms, queue_ms)."""
    nt, np_ = s.models[model]
    er, ei, hr, hi = (np.empty((nt, 3, np_)) for _ in range(4))
    info = cmcg_info()
    lat = (C.c_double * 2)()
    rc = _lib.cmcg_server_poll(s.ptr, int(ticket), int(bool(wait)), _ptr(er), _ptr(ei), _ptr(hr), _ptr(hi),
                               C.byref(info), lat)
    if rc == CMCG_PENDING:
        return None
    _check(rc, "cmcg_server_poll", allow_not_converged=True)
    return rc, er + 1j * ei, hr + 1j * hi, info, lat[0], lat[1]


def cmcg_server_stats(s: Server):
    c, q, b, n = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int()
    _check(_lib.cmcg_server_stats(s.ptr, C.byref(c), C.byref(q), C.byref(b), C.byref(n)), "cmcg_server_stats")
    return {"completed": c.value, "queued": q.value, "bytes_in_use": b.value, "handles": n.value}


def cmcg_server_destroy(s: Server) -> None:
    s.close()
