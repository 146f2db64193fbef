"""GB300 flux-limited convection library -- Python binding of ``include/fl.h``.

The compute path is the CUDA library ``_build/libfl.so`` (hand-written
sm_103a kernels).  This module only marshals arguments: every ``fl_*``
function here has the name and argument order of the C entry point, takes
device buffers as integers or CUDA tensors, raises :class:`FLError` on a
non-zero status and returns the C outputs.  There is no CPU fallback: if the
library is not built, every call raises.

A few helpers sit on top (``Mesh``, ``step_rk``, ``conv_limited_apply``):
they allocate the caller-side workspace with PyTorch and pass the current
stream, nothing else.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfl.so")

FL_OK, FL_EINVAL, FL_ENOMEM, FL_ECUDA, FL_EUNSUPPORTED, FL_ENONFINITE, FL_ETIMEOUT, FL_EINDEX = \
    range(8)
STATUS_NAMES = ["FL_OK", "FL_EINVAL", "FL_ENOMEM", "FL_ECUDA", "FL_EUNSUPPORTED",
                "FL_ENONFINITE", "FL_ETIMEOUT", "FL_EINDEX"]
LIMITERS = {"upwind": 0, "central": 1, "minmod": 2, "vanleer": 3, "superbee": 4, "smart": 5}
FL_F32, FL_F64 = 0, 1
FL_RENUMBER = 1
FL_FIELD_CELL, FL_FIELD_FACE = 0, 1

# Exported symbols of include/fl.h (checked by the ABI test).
ABI_SYMBOLS = [
    "fl_last_error", "fl_version", "fl_mesh_create_structured", "fl_mesh_create",
    "fl_mesh_create_weighted",
    "fl_mesh_permutation", "fl_mesh_info", "fl_mesh_status", "fl_mesh_destroy",
    "fl_mesh_to_internal", "fl_mesh_to_user", "fl_mesh_create_local", "fl_mesh_local_info",
    "fl_halo_pack", "fl_halo_unpack",
    "fl_conv_limited_apply",
    "fl_face_selection", "fl_workspace_size", "fl_step_rk", "fl_step_rk_modulated",
    "fl_step_rk_noalloc", "fl_step_rk_blocked", "fl_step_rk_stage", "fl_step_rk_stage_planes",
    "fl_step_rk_stage_cells", "fl_step_rk_stage_box",
    "fl_velocity_prescale",
    "fl_conv_limited_adjoint",
    "fl_adjoint_workspace_size", "fl_step_rk_adjoint", "fl_step_rk_stage_adjoint",
    "fl_step_rk_stage_adjoint_planes", "fl_step_rk_stage_adjoint_cells",
    "fl_step_rk_stage_adjoint_box", "fl_step_rk_checkpointed",
    "fl_step_rk_adjoint_from_checkpoints", "fl_batch_create",
    "fl_batch_workspace_size", "fl_batch_step_rk", "fl_batch_tiling", "fl_batch_set_tiling",
    "fl_batch_destroy",
    "fl_alg_create", "fl_alg_destroy", "fl_alg_info", "fl_alg_workspace_size",
    "fl_alg_face_values", "fl_alg_step_euler",
    "fl_reduce_workspace_size", "fl_reduce_max_abs", "fl_reduce_mass",
]


class FLError(RuntimeError):
    def __init__(self, status, msg):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, msg))
        self.status = status


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile libfl.so (nvcc, sm_103a) in-tree; returns its path."""
    from . import _build_lib
    return _build_lib.build(force=force)


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: run paper_2110_03044_gb300.build() "
                               "(there is no CPU fallback)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D, U, SZ = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                               ctypes.c_uint, ctypes.c_size_t)
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "fl_last_error": (ctypes.c_char_p, []),
            "fl_version": (ctypes.c_char_p, []),
            "fl_mesh_create_structured": (I, [I, I, I, D, D, D, U, PP]),
            "fl_mesh_create": (I, [I64, I64, P, P, P, P, U, PP]),
            "fl_mesh_create_weighted": (I, [I64, I64, P, P, P, P, P, U, PP]),
            "fl_mesh_create_local": (I, [I64, I64, I64, I64, P, P, P, P, P, U, PP]),
            "fl_mesh_local_info": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
            "fl_halo_pack": (I, [P, I, P, P, I64, P, P]),
            "fl_halo_unpack": (I, [P, I, P, P, I64, P, P]),
            "fl_mesh_permutation": (I, [P, P, P, P]),
            "fl_mesh_info": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64),
                                 ctypes.POINTER(I)]),
            "fl_mesh_status": (I, [P, P]),
            "fl_mesh_destroy": (I, [P]),
            "fl_mesh_to_internal": (I, [P, I, I, P, P, P]),
            "fl_mesh_to_user": (I, [P, I, I, P, P, P]),
            "fl_conv_limited_apply": (I, [P, I, I, P, P, P, P, P]),
            "fl_face_selection": (I, [P, I, P, P, P]),
            "fl_workspace_size": (I, [P, I, I, ctypes.POINTER(SZ)]),
            "fl_step_rk": (I, [P, I, I, I, D, I64, P, P, P, SZ, P]),
            "fl_step_rk_modulated": (I, [P, I, I, I, D, I64, P, P, P, P, SZ, P]),
            "fl_step_rk_noalloc": (I, [P, I, I, I, D, I64, P, P, P]),
            "fl_step_rk_blocked": (I, [P, I, I, I, D, I64, P, P, P, SZ, P]),
            "fl_step_rk_stage": (I, [P, I, I, I, I, D, P, P, P, P, P, P]),
            "fl_step_rk_stage_planes": (I, [P, I, I, I, I, D, I, I, P, P, P, P, P, P]),
            "fl_step_rk_stage_cells": (I, [P, I, I, I, I, D, I64, I64, P, P, P, P, P, P]),
            "fl_step_rk_stage_box": (I, [P, I, I, I, I, D, I, I, I, I, P, P, P, P, P, P]),
            "fl_velocity_prescale": (I, [P, I, D, P, P, P]),
            "fl_conv_limited_adjoint": (I, [P, I, I, P, P, P, P, P]),
            "fl_adjoint_workspace_size": (I, [P, I, I, I64, I64, ctypes.POINTER(SZ)]),
            "fl_step_rk_stage_adjoint": (I, [P, I, I, I, I, D, P, P, P, P, P, P, P, P]),
            "fl_step_rk_stage_adjoint_planes": (I, [P, I, I, I, I, D, I, I, P, P, P, P, P, P, P,
                                                    P]),
            "fl_step_rk_stage_adjoint_cells": (I, [P, I, I, I, I, D, I64, I64, P, P, P, P, P, P,
                                                   P, P]),
            "fl_step_rk_stage_adjoint_box": (I, [P, I, I, I, I, D, I, I, I, I, P, P, P, P, P, P,
                                                 P, P]),
            "fl_step_rk_adjoint": (I, [P, I, I, I, D, I64, I64, P, P, P, P, P, SZ, P]),
            "fl_step_rk_checkpointed": (I, [P, I, I, I, D, I64, I64, P, P, P, SZ, P]),
            "fl_step_rk_adjoint_from_checkpoints": (I, [P, I, I, I, D, I64, I64, P, P, P, P,
                                                         SZ, P]),
            "fl_batch_create": (I, [I, PP, PP]),
            "fl_batch_workspace_size": (I, [P, I, I, ctypes.POINTER(SZ)]),
            "fl_batch_step_rk": (I, [P, I, I, I, ctypes.POINTER(D), I64, PP, PP, P, SZ, P]),
            "fl_batch_tiling": (I, [P, I, I, I, ctypes.POINTER(I), ctypes.POINTER(I),
                                    ctypes.POINTER(I), ctypes.POINTER(I)]),
            "fl_batch_set_tiling": (I, [P, I, I, I, I, I, I, I]),
            "fl_batch_destroy": (I, [P]),
            "fl_alg_create": (I, [I64, I64, P, P, P, P, ctypes.POINTER(P)]),
            "fl_alg_destroy": (I, [P]),
            "fl_alg_info": (I, [P, P, P, ctypes.POINTER(SZ)]),
            "fl_alg_workspace_size": (I, [P, ctypes.POINTER(SZ)]),
            "fl_alg_face_values": (I, [P, I, P, P, P, P, SZ, P]),
            "fl_alg_step_euler": (I, [P, I, D, I64, P, P, P, SZ, P]),
            "fl_reduce_workspace_size": (SZ, []),
            "fl_reduce_max_abs": (I, [I, P, I64, ctypes.POINTER(D), P, P]),
            "fl_reduce_mass": (I, [P, I, P, ctypes.POINTER(D), P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(st):
    if st != FL_OK:
        raise FLError(st, lib().fl_last_error().decode(errors="replace"))


# ------------------------------------------------------------- marshalling
def _ptr(x):
    """Device pointer of a tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError("expected a CUDA tensor or an integer device pointer, got %r" % type(x))


def _fptr(x, code):
    """Device pointer of a field buffer whose elements have the call's type
    (FL_F32 / FL_F64): a tensor of another dtype, or a CPU tensor, is
    refused here (the library checks sizes against allocations, which a
    wrong element type inside a larger cached block would pass)."""
    if hasattr(x, "dtype") and hasattr(x, "is_cuda"):
        import torch
        want = torch.float64 if code == FL_F64 else torch.float32
        if x.dtype != want:
            raise TypeError("field tensor has dtype %s, the call's dtype is %s" % (x.dtype, want))
        if not x.is_cuda:
            raise ValueError("field tensors must be CUDA tensors")
    return _ptr(x)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _lim(limiter):
    return LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)


def dtype_code(dtype):
    import torch
    if dtype in (torch.float64, "f64", "float64", FL_F64):
        return FL_F64
    if dtype in (torch.float32, "f32", "float32", FL_F32):
        return FL_F32
    raise ValueError("unsupported dtype %r" % (dtype,))


# ------------------------------------------------------ C entry points
def fl_version():
    return lib().fl_version().decode()


def fl_last_error():
    return lib().fl_last_error().decode(errors="replace")


def fl_mesh_create_structured(nx, ny, nz, hx, hy, hz, periodic_mask=7):
    h = ctypes.c_void_p()
    _check(lib().fl_mesh_create_structured(int(nx), int(ny), int(nz), float(hx), float(hy),
                                           float(hz), int(periodic_mask), ctypes.byref(h)))
    return h.value


def fl_mesh_create(n_cells, face_cells, face_normals, face_areas, cell_volumes, flags=0):
    import numpy as np
    fc = np.ascontiguousarray(face_cells, dtype=np.int32)
    nrm = np.ascontiguousarray(face_normals, dtype=np.float64)
    ar = np.ascontiguousarray(face_areas, dtype=np.float64)
    vol = np.ascontiguousarray(cell_volumes, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib().fl_mesh_create(int(n_cells), int(fc.shape[0]), fc.ctypes.data, nrm.ctypes.data,
                                ar.ctypes.data, vol.ctypes.data, int(flags), ctypes.byref(h)))
    return h.value


def fl_mesh_create_local(n_cells, n_owned, n_interior, face_cells, face_normals, face_areas,
                         cell_volumes, face_distances=None, flags=0):
    """The local mesh of one part of a partitioned face-based mesh (see fl.h)."""
    import numpy as np
    fc = np.ascontiguousarray(face_cells, dtype=np.int32)
    nrm = np.ascontiguousarray(face_normals, dtype=np.float64)
    ar = np.ascontiguousarray(face_areas, dtype=np.float64)
    vol = np.ascontiguousarray(cell_volumes, dtype=np.float64)
    dist = None
    if face_distances is not None:
        dist = np.ascontiguousarray(face_distances, dtype=np.float64)
        if dist.shape != (fc.shape[0],):
            raise ValueError("face_distances must hold one value per face")
    h = ctypes.c_void_p()
    _check(lib().fl_mesh_create_local(int(n_cells), int(n_owned), int(n_interior), int(fc.shape[0]),
                                      fc.ctypes.data, nrm.ctypes.data, ar.ctypes.data,
                                      vol.ctypes.data, None if dist is None else dist.ctypes.data,
                                      int(flags), ctypes.byref(h)))
    return h.value


def fl_mesh_local_info(mesh):
    """(n_owned, n_interior) of a mesh."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().fl_mesh_local_info(mesh, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def fl_halo_pack(mesh, dtype, src, index, n, dst, stream=None):
    """dst[i] = src[index[i]] for i < n (device arrays; index int32)."""
    c = dtype_code(dtype)
    _check(lib().fl_halo_pack(mesh, c, _fptr(src, c), _ptr(index), int(n), _fptr(dst, c),
                              _stream(stream)))


def fl_halo_unpack(mesh, dtype, src, index, n, dst, stream=None):
    """dst[index[i]] = src[i] for i < n (device arrays; index int32)."""
    c = dtype_code(dtype)
    _check(lib().fl_halo_unpack(mesh, c, _fptr(src, c), _ptr(index), int(n), _fptr(dst, c),
                                _stream(stream)))


def fl_mesh_create_weighted(n_cells, face_cells, face_normals, face_areas, cell_volumes,
                            face_distances, flags=0):
    import numpy as np
    fc = np.ascontiguousarray(face_cells, dtype=np.int32)
    nrm = np.ascontiguousarray(face_normals, dtype=np.float64)
    ar = np.ascontiguousarray(face_areas, dtype=np.float64)
    vol = np.ascontiguousarray(cell_volumes, dtype=np.float64)
    dist = np.ascontiguousarray(face_distances, dtype=np.float64)
    if dist.shape != (fc.shape[0],):
        raise ValueError("face_distances must hold one value per face")
    h = ctypes.c_void_p()
    _check(lib().fl_mesh_create_weighted(int(n_cells), int(fc.shape[0]), fc.ctypes.data,
                                         nrm.ctypes.data, ar.ctypes.data, vol.ctypes.data,
                                         dist.ctypes.data, int(flags), ctypes.byref(h)))
    return h.value


def fl_mesh_permutation(mesh):
    import numpy as np
    C, F, _ = fl_mesh_info(mesh)
    cp = np.empty(C, np.int32)
    fp = np.empty(F, np.int32)
    fl = np.empty(F, np.uint8)
    _check(lib().fl_mesh_permutation(mesh, cp.ctypes.data, fp.ctypes.data, fl.ctypes.data))
    return cp, fp, fl


def fl_mesh_info(mesh):
    c, f, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(lib().fl_mesh_info(mesh, ctypes.byref(c), ctypes.byref(f), ctypes.byref(k)))
    return c.value, f.value, k.value


def fl_mesh_status(mesh, stream=None):
    """Raise if a kernel on this mesh recorded a device-side error (syncs)."""
    _check(lib().fl_mesh_status(mesh, _stream(stream)))


def fl_mesh_destroy(mesh):
    _check(lib().fl_mesh_destroy(mesh))


def _kind(kind):
    if kind in ("cell", FL_FIELD_CELL):
        return FL_FIELD_CELL
    if kind in ("face", FL_FIELD_FACE):
        return FL_FIELD_FACE
    raise ValueError("field kind must be 'cell' or 'face', got %r" % (kind,))


def fl_mesh_to_internal(mesh, kind, dtype, src, dst, stream=None):
    """dst (internal order) <- src (user order) for a cell or face field."""
    c = dtype_code(dtype)
    _check(lib().fl_mesh_to_internal(mesh, _kind(kind), c, _fptr(src, c), _fptr(dst, c),
                                     _stream(stream)))


def fl_mesh_to_user(mesh, kind, dtype, src, dst, stream=None):
    """dst (user order) <- src (internal order) for a cell or face field."""
    c = dtype_code(dtype)
    _check(lib().fl_mesh_to_user(mesh, _kind(kind), c, _fptr(src, c), _fptr(dst, c),
                                 _stream(stream)))


def fl_conv_limited_apply(mesh, limiter, dtype, theta_c, u_f, rhs_c, theta_f=None, stream=None):
    c = dtype_code(dtype)
    _check(lib().fl_conv_limited_apply(mesh, _lim(limiter), c, _fptr(theta_c, c), _fptr(u_f, c),
                                       _fptr(rhs_c, c), _fptr(theta_f, c), _stream(stream)))


def fl_face_selection(mesh, dtype, u_f, sel, stream=None):
    c = dtype_code(dtype)
    _check(lib().fl_face_selection(mesh, c, _fptr(u_f, c), _ptr(sel), _stream(stream)))


def fl_workspace_size(mesh, dtype, rk_order):
    n = ctypes.c_size_t()
    _check(lib().fl_workspace_size(mesh, dtype_code(dtype), int(rk_order), ctypes.byref(n)))
    return n.value


def fl_step_rk(mesh, limiter, dtype, rk_order, dt, nsteps, theta, u_f, workspace,
               workspace_bytes, stream=None):
    c = dtype_code(dtype)
    _check(lib().fl_step_rk(mesh, _lim(limiter), c, int(rk_order), float(dt), int(nsteps),
                            _fptr(theta, c), _fptr(u_f, c), _ptr(workspace),
                            int(workspace_bytes), _stream(stream)))


def fl_step_rk_stage(mesh, limiter, dtype, rk_order, stage, dt, theta_n, x, y, u_f, w_f=None,
                     stream=None):
    """One RK stage y = a theta_n + b (x + dt R(x)) (see fl.h)."""
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_stage(mesh, _lim(limiter), c, int(rk_order), int(stage), float(dt),
                                  _fptr(theta_n, c), _fptr(x, c), _fptr(y, c), _fptr(u_f, c),
                                  _fptr(w_f, c), _stream(stream)))


def fl_step_rk_stage_planes(mesh, limiter, dtype, rk_order, stage, dt, z_begin, z_end, theta_n,
                            x, y, u_f, w_f=None, stream=None):
    """fl_step_rk_stage over the z planes [z_begin, z_end) of a structured
    mesh only (see fl.h)."""
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_stage_planes(mesh, _lim(limiter), c, int(rk_order), int(stage),
                                         float(dt), int(z_begin), int(z_end), _fptr(theta_n, c),
                                         _fptr(x, c), _fptr(y, c), _fptr(u_f, c), _fptr(w_f, c),
                                         _stream(stream)))


def fl_step_rk_stage_cells(mesh, limiter, dtype, rk_order, stage, dt, c_begin, c_end, theta_n,
                           x, y, u_f, w_f=None, stream=None):
    """fl_step_rk_stage over the owned cells [c_begin, c_end) of a local mesh
    only (see fl.h)."""
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_stage_cells(mesh, _lim(limiter), c, int(rk_order), int(stage),
                                        float(dt), int(c_begin), int(c_end), _fptr(theta_n, c),
                                        _fptr(x, c), _fptr(y, c), _fptr(u_f, c), _fptr(w_f, c),
                                        _stream(stream)))


def fl_step_rk_stage_box(mesh, limiter, dtype, rk_order, stage, dt, y_begin, y_end, z_begin,
                         z_end, theta_n, x, y, u_f, w_f=None, stream=None):
    """fl_step_rk_stage over the rows [y_begin, y_end) of the planes
    [z_begin, z_end) of a structured mesh only (see fl.h)."""
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_stage_box(mesh, _lim(limiter), c, int(rk_order), int(stage),
                                      float(dt), int(y_begin), int(y_end), int(z_begin),
                                      int(z_end), _fptr(theta_n, c), _fptr(x, c), _fptr(y, c),
                                      _fptr(u_f, c), _fptr(w_f, c), _stream(stream)))


def fl_velocity_prescale(mesh, dtype, dt, u_f, w_f, stream=None):
    """w_f = dt (A/V) u_f, the velocity fl_step_rk_stage takes in FP64."""
    c = dtype_code(dtype)
    _check(lib().fl_velocity_prescale(mesh, c, float(dt), _fptr(u_f, c), _fptr(w_f, c),
                                      _stream(stream)))


def fl_step_rk_blocked(mesh, limiter, dtype, rk_order, dt, nsteps, theta, u_f, workspace,
                       workspace_bytes, stream=None):
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_blocked(mesh, _lim(limiter), c, int(rk_order), float(dt),
                                    int(nsteps), _fptr(theta, c), _fptr(u_f, c),
                                    _ptr(workspace), int(workspace_bytes), _stream(stream)))


def fl_step_rk_modulated(mesh, limiter, dtype, rk_order, dt, nsteps, theta, u_f, g, workspace,
                         workspace_bytes, stream=None):
    """fl_step_rk where stage s of step n advects with g[n * S + s] * u_f;
    ``g`` is a host sequence of nsteps * S floats (S = 1 Euler, 3 SSP-RK3)."""
    import numpy as np
    S = 1 if int(rk_order) == 1 else 3
    gg = np.ascontiguousarray(np.asarray(g, dtype=np.float64).ravel())
    if gg.size < int(nsteps) * S:
        raise ValueError("need nsteps * stages velocity factors")
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_modulated(mesh, _lim(limiter), c, int(rk_order),
                                      float(dt), int(nsteps), _fptr(theta, c), _fptr(u_f, c),
                                      gg.ctypes.data_as(ctypes.c_void_p), _ptr(workspace),
                                      int(workspace_bytes), _stream(stream)))


def fl_step_rk_noalloc(mesh, limiter, dtype, rk_order, dt, nsteps, theta, u_f, stream=None):
    """fl_step_rk for callers that cannot allocate device memory: the stage
    buffers come from the library's built-in scratch area (see fl.h)."""
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_noalloc(mesh, _lim(limiter), c, int(rk_order), float(dt),
                                    int(nsteps), _fptr(theta, c), _fptr(u_f, c),
                                    _stream(stream)))


def fl_conv_limited_adjoint(mesh, limiter, dtype, theta_c, u_f, lambda_rhs, lambda_theta,
                            stream=None):
    c = dtype_code(dtype)
    _check(lib().fl_conv_limited_adjoint(mesh, _lim(limiter), c, _fptr(theta_c, c),
                                         _fptr(u_f, c), _fptr(lambda_rhs, c),
                                         _fptr(lambda_theta, c), _stream(stream)))


def fl_step_rk_stage_adjoint(mesh, limiter, dtype, rk_order, stage, dt, x, mu, lam_a, lam_b,
                             out, u_f, w_f=None, stream=None):
    """Reverse mode of one RK stage (see fl.h): dJ/dx_s, or for stage 0 of
    SSP-RK3 dJ/dtheta_n with theta_n's later uses (lam_a, lam_b)."""
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_stage_adjoint(mesh, _lim(limiter), c, int(rk_order), int(stage),
                                          float(dt), _fptr(x, c), _fptr(mu, c), _fptr(lam_a, c),
                                          _fptr(lam_b, c), _fptr(out, c), _fptr(u_f, c),
                                          _fptr(w_f, c), _stream(stream)))


def fl_step_rk_stage_adjoint_planes(mesh, limiter, dtype, rk_order, stage, dt, z_begin, z_end,
                                    x, mu, lam_a, lam_b, out, u_f, w_f=None, stream=None):
    """fl_step_rk_stage_adjoint over the z planes [z_begin, z_end) of a
    structured mesh only (see fl.h)."""
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_stage_adjoint_planes(
        mesh, _lim(limiter), c, int(rk_order), int(stage), float(dt), int(z_begin), int(z_end),
        _fptr(x, c), _fptr(mu, c), _fptr(lam_a, c), _fptr(lam_b, c), _fptr(out, c),
        _fptr(u_f, c), _fptr(w_f, c), _stream(stream)))


def fl_step_rk_stage_adjoint_cells(mesh, limiter, dtype, rk_order, stage, dt, c_begin, c_end, x,
                                   mu, lam_a, lam_b, out, u_f, w_f=None, stream=None):
    """fl_step_rk_stage_adjoint over the owned cells [c_begin, c_end) of a
    local mesh only (see fl.h)."""
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_stage_adjoint_cells(
        mesh, _lim(limiter), c, int(rk_order), int(stage), float(dt), int(c_begin), int(c_end),
        _fptr(x, c), _fptr(mu, c), _fptr(lam_a, c), _fptr(lam_b, c), _fptr(out, c),
        _fptr(u_f, c), _fptr(w_f, c), _stream(stream)))


def fl_step_rk_stage_adjoint_box(mesh, limiter, dtype, rk_order, stage, dt, y_begin, y_end,
                                 z_begin, z_end, x, mu, lam_a, lam_b, out, u_f, w_f=None,
                                 stream=None):
    """fl_step_rk_stage_adjoint over the rows [y_begin, y_end) of the planes
    [z_begin, z_end) of a structured mesh only (see fl.h)."""
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_stage_adjoint_box(
        mesh, _lim(limiter), c, int(rk_order), int(stage), float(dt), int(y_begin), int(y_end),
        int(z_begin), int(z_end), _fptr(x, c), _fptr(mu, c), _fptr(lam_a, c), _fptr(lam_b, c),
        _fptr(out, c), _fptr(u_f, c), _fptr(w_f, c), _stream(stream)))


def fl_adjoint_workspace_size(mesh, dtype, rk_order, nsteps, checkpoint_every):
    n = ctypes.c_size_t()
    _check(lib().fl_adjoint_workspace_size(mesh, dtype_code(dtype), int(rk_order), int(nsteps),
                                           int(checkpoint_every), ctypes.byref(n)))
    return n.value


def fl_step_rk_adjoint(mesh, limiter, dtype, rk_order, dt, nsteps, checkpoint_every, theta0, u_f,
                       lambda_T, lambda_0, workspace, workspace_bytes, stream=None):
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_adjoint(mesh, _lim(limiter), c, int(rk_order), float(dt),
                                    int(nsteps), int(checkpoint_every), _fptr(theta0, c),
                                    _fptr(u_f, c), _fptr(lambda_T, c), _fptr(lambda_0, c),
                                    _ptr(workspace), int(workspace_bytes), _stream(stream)))


def fl_step_rk_checkpointed(mesh, limiter, dtype, rk_order, dt, nsteps, checkpoint_every,
                            theta, u_f, workspace, workspace_bytes, stream=None):
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_checkpointed(mesh, _lim(limiter), c, int(rk_order), float(dt),
                                         int(nsteps), int(checkpoint_every), _fptr(theta, c),
                                         _fptr(u_f, c), _ptr(workspace), int(workspace_bytes),
                                         _stream(stream)))


def fl_step_rk_adjoint_from_checkpoints(mesh, limiter, dtype, rk_order, dt, nsteps,
                                        checkpoint_every, u_f, lambda_T, lambda_0, workspace,
                                        workspace_bytes, stream=None):
    c = dtype_code(dtype)
    _check(lib().fl_step_rk_adjoint_from_checkpoints(
        mesh, _lim(limiter), c, int(rk_order), float(dt), int(nsteps), int(checkpoint_every),
        _fptr(u_f, c), _fptr(lambda_T, c), _fptr(lambda_0, c), _ptr(workspace),
        int(workspace_bytes), _stream(stream)))


def fl_batch_create(meshes):
    arr = (ctypes.c_void_p * len(meshes))(*meshes)
    h = ctypes.c_void_p()
    _check(lib().fl_batch_create(len(meshes), arr, ctypes.byref(h)))
    return h.value


def fl_batch_workspace_size(batch, dtype, rk_order):
    n = ctypes.c_size_t()
    _check(lib().fl_batch_workspace_size(batch, dtype_code(dtype), int(rk_order),
                                         ctypes.byref(n)))
    return n.value


def fl_batch_step_rk(batch, limiter, dtype, rk_order, dts, nsteps, thetas, u_fs, workspace,
                     workspace_bytes, stream=None):
    n = len(thetas)
    dt_arr = (ctypes.c_double * n)(*[float(d) for d in dts])
    c = dtype_code(dtype)
    th_arr = (ctypes.c_void_p * n)(*[_fptr(t, c) for t in thetas])
    u_arr = (ctypes.c_void_p * n)(*[_fptr(u, c) for u in u_fs])
    _check(lib().fl_batch_step_rk(batch, _lim(limiter), c, int(rk_order), dt_arr,
                                  int(nsteps), th_arr, u_arr, _ptr(workspace),
                                  int(workspace_bytes), _stream(stream)))


def fl_batch_tiling(batch, limiter, dtype, rk_order):
    """(kind, cells_per_thread, warps, z_chunk) of the batch's decomposition."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().fl_batch_tiling(batch, _lim(limiter), dtype_code(dtype), int(rk_order),
                                 *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def fl_batch_set_tiling(batch, limiter, dtype, rk_order, kind, cells_per_thread, warps, z_chunk):
    _check(lib().fl_batch_set_tiling(batch, _lim(limiter), dtype_code(dtype), int(rk_order),
                                     int(kind), int(cells_per_thread), int(warps), int(z_chunk)))


def fl_batch_destroy(batch):
    _check(lib().fl_batch_destroy(batch))


def fl_alg_create(n_cells, face_cells, normals, areas, volumes):
    """Matrices of the algebraic formulation (E, T, -S, Pi, M in ELLPACK) on
    the current device from host face arrays; returns the handle."""
    import numpy as np
    fc = np.ascontiguousarray(face_cells, dtype=np.int32)
    nrm = np.ascontiguousarray(normals, dtype=np.float64)
    ar = np.ascontiguousarray(areas, dtype=np.float64)
    vol = np.ascontiguousarray(volumes, dtype=np.float64)
    h = ctypes.c_void_p()
    vp = ctypes.c_void_p
    _check(lib().fl_alg_create(int(n_cells), int(fc.shape[0]), fc.ctypes.data_as(vp),
                               nrm.ctypes.data_as(vp), ar.ctypes.data_as(vp),
                               vol.ctypes.data_as(vp), ctypes.byref(h)))
    return h.value


def fl_alg_destroy(alg):
    _check(lib().fl_alg_destroy(alg))


def fl_alg_info(alg):
    """(nnz[5], width[5], device bytes) for E, T, -S, Pi, M."""
    nnz = (ctypes.c_int64 * 5)()
    width = (ctypes.c_int32 * 5)()
    b = ctypes.c_size_t()
    _check(lib().fl_alg_info(alg, nnz, width, ctypes.byref(b)))
    return list(nnz), list(width), b.value


def fl_alg_workspace_size(alg):
    n = ctypes.c_size_t()
    _check(lib().fl_alg_workspace_size(alg, ctypes.byref(n)))
    return n.value


def fl_alg_face_values(alg, limiter, theta, u_f, theta_f, workspace, workspace_bytes,
                       stream=None):
    _check(lib().fl_alg_face_values(alg, _lim(limiter), _fptr(theta, FL_F64),
                                    _fptr(u_f, FL_F64), _fptr(theta_f, FL_F64),
                                    _ptr(workspace), int(workspace_bytes), _stream(stream)))


def fl_alg_step_euler(alg, limiter, dt, nsteps, theta, u_f, workspace, workspace_bytes,
                      stream=None):
    _check(lib().fl_alg_step_euler(alg, _lim(limiter), float(dt), int(nsteps),
                                   _fptr(theta, FL_F64), _fptr(u_f, FL_F64), _ptr(workspace),
                                   int(workspace_bytes),
                                   _stream(stream)))


def fl_reduce_workspace_size():
    return int(lib().fl_reduce_workspace_size())


def fl_reduce_max_abs(dtype, x, n, workspace, stream=None):
    out = ctypes.c_double()
    c = dtype_code(dtype)
    _check(lib().fl_reduce_max_abs(c, _fptr(x, c), int(n), ctypes.byref(out),
                                   _ptr(workspace), _stream(stream)))
    return out.value


def fl_reduce_mass(mesh, dtype, theta, workspace, stream=None):
    out = ctypes.c_double()
    c = dtype_code(dtype)
    _check(lib().fl_reduce_mass(mesh, c, _fptr(theta, c), ctypes.byref(out),
                                _ptr(workspace), _stream(stream)))
    return out.value


# ---------------------------------------------------------------- helpers
class Mesh:
    """Owns an ``fl_mesh`` handle."""

    def __init__(self, handle, dims=None, h=None):
        self.handle = handle
        self.n_cells, self.n_faces, self.kind = fl_mesh_info(handle)
        self.dims = dims
        self.h = h

    @classmethod
    def structured(cls, nx, ny=1, nz=1, hx=1.0, hy=1.0, hz=1.0):
        return cls(fl_mesh_create_structured(nx, ny, nz, hx, hy, hz, 7), (nx, ny, nz),
                   (hx, hy, hz))

    @classmethod
    def from_faces(cls, n_cells, face_cells, face_normals, face_areas, cell_volumes,
                   renumber=False, distances=None):
        """Face-based mesh; ``distances`` (one per face) makes it non-uniform
        (Algorithm 3's distance weights, fl_mesh_create_weighted)."""
        flags = FL_RENUMBER if renumber else 0
        if distances is not None:
            return cls(fl_mesh_create_weighted(n_cells, face_cells, face_normals, face_areas,
                                               cell_volumes, distances, flags))
        return cls(fl_mesh_create(n_cells, face_cells, face_normals, face_areas, cell_volumes,
                                  flags))

    def permutation(self):
        return fl_mesh_permutation(self.handle)

    def to_internal(self, field, kind="cell", stream=None):
        """A new CUDA tensor holding ``field`` (user order) in the library's
        internal order (fl_mesh_to_internal; a copy for meshes that were not
        renumbered)."""
        import torch
        out = torch.empty_like(field)
        fl_mesh_to_internal(self.handle, kind, field.dtype, field, out, stream)
        return out

    def to_user(self, field, kind="cell", stream=None):
        """A new CUDA tensor holding ``field`` (internal order) in user order
        (fl_mesh_to_user)."""
        import torch
        out = torch.empty_like(field)
        fl_mesh_to_user(self.handle, kind, field.dtype, field, out, stream)
        return out

    def close(self):
        if self.handle:
            fl_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dt_of(t):
    return dtype_code(t.dtype)


def workspace_for(mesh, dtype, rk_order, device="cuda"):
    import torch
    n = fl_workspace_size(mesh.handle, dtype, rk_order)
    return torch.empty(max(n, 1), dtype=torch.uint8, device=device), n


def step_rk(mesh, limiter, theta, u_f, dt, nsteps, rk_order=3, workspace=None, stream=None):
    """In-place ``nsteps`` steps on the CUDA tensor ``theta``."""
    if workspace is None:
        workspace, nbytes = workspace_for(mesh, theta.dtype, rk_order, theta.device)
    else:
        nbytes = workspace.numel() * workspace.element_size()
    fl_step_rk(mesh.handle, limiter, theta.dtype, rk_order, dt, nsteps, theta, u_f, workspace,
               nbytes, stream)
    return theta


def step_rk_blocked(mesh, limiter, theta, u_f, dt, nsteps, rk_order=3, workspace=None,
                    stream=None):
    """``step_rk`` with temporal blocking (structured meshes): one launch per
    SSP-RK3 step, or per three Euler steps."""
    if workspace is None:
        workspace, nbytes = workspace_for(mesh, theta.dtype, rk_order, theta.device)
    else:
        nbytes = workspace.numel() * workspace.element_size()
    fl_step_rk_blocked(mesh.handle, limiter, theta.dtype, rk_order, dt, nsteps, theta, u_f,
                       workspace, nbytes, stream)
    return theta


def step_rk_modulated(mesh, limiter, theta, u_f, dt, nsteps, g, rk_order=1, workspace=None,
                      stream=None):
    """In-place ``nsteps`` steps on ``theta`` with the stage velocities
    g[n * S + s] * u_f (a time-modulated flow)."""
    if workspace is None:
        workspace, nbytes = workspace_for(mesh, theta.dtype, rk_order, theta.device)
    else:
        nbytes = workspace.numel() * workspace.element_size()
    fl_step_rk_modulated(mesh.handle, limiter, theta.dtype, rk_order, dt, nsteps, theta, u_f, g,
                         workspace, nbytes, stream)
    return theta


class Algebraic:
    """The algebraic formulation (Algorithm 1 / Algorithm 5 as SpMV + kbin)
    of a face-based mesh, FP64, for comparison with the fused kernels."""

    def __init__(self, n_cells, face_cells, normals, areas, volumes):
        import torch
        self.handle = fl_alg_create(n_cells, face_cells, normals, areas, volumes)
        self.n_cells = int(n_cells)
        self.n_faces = int(len(areas))
        nb = fl_alg_workspace_size(self.handle)
        self.ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
        self.ws_bytes = nb

    def info(self):
        return fl_alg_info(self.handle)

    def face_values(self, limiter, theta, u_f, stream=None):
        import torch
        out = torch.empty(self.n_faces, dtype=torch.float64, device=theta.device)
        fl_alg_face_values(self.handle, limiter, theta, u_f, out, self.ws, self.ws_bytes, stream)
        return out

    def step_euler(self, limiter, theta, u_f, dt, nsteps, stream=None):
        fl_alg_step_euler(self.handle, limiter, dt, nsteps, theta, u_f, self.ws, self.ws_bytes,
                          stream)
        return theta

    def close(self):
        if getattr(self, "handle", None):
            fl_alg_destroy(self.handle)
            self.handle = None


def conv_limited_apply(mesh, limiter, theta, u_f, want_theta_f=False, stream=None):
    import torch
    rhs = torch.empty_like(theta)
    thf = torch.empty(mesh.n_faces, dtype=theta.dtype, device=theta.device) if want_theta_f \
        else None
    fl_conv_limited_apply(mesh.handle, limiter, theta.dtype, theta, u_f, rhs, thf, stream)
    return (rhs, thf) if want_theta_f else rhs


def face_selection(mesh, u_f, stream=None):
    import torch
    sel = torch.empty((mesh.n_faces, 4), dtype=torch.int32, device=u_f.device)
    fl_face_selection(mesh.handle, u_f.dtype, u_f, sel, stream)
    return sel
