"""CPU oracle for the flux-limited convection path (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2110_03044_gb300`` never imports, links or executes anything here, and
this package never imports the library: the two share no code.

Two independent references live here:

* ``fl_oracle.cpp`` -- the plain FP64 stencil definition (face loop + cell
  loop, Euler / SSP-RK3, tangent-linear and adjoint), compiled with
  ``-O2 -fno-fast-math -ffp-contract=off`` and loaded through ctypes;
* ``brute.py`` -- the paper's algebraic formulation (incidence, shift,
  adjacency, normal and sign matrices assembled densely in NumPy) for tiny
  meshes, used to pin the stencil oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fl_oracle.cpp")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")
# The mutation test (tests/test_oracle_mutations.py) points this at a
# deliberately broken build to show that the pins reject it.
MUTANT_LIB = os.environ.get("FL_ORACLE_MUTANT_LIB")

LIMITERS = {"upwind": 0, "central": 1, "minmod": 2, "vanleer": 3, "superbee": 4, "smart": 5}

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (g++, OpenMP, no FMA
    contraction, no fast-math)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-std=c++17",
           "-shared", "-fPIC", "-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if MUTANT_LIB:
            lib = ctypes.CDLL(MUTANT_LIB)
        else:
            build()
            lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        I = ctypes.c_int
        D = ctypes.c_double
        lib.orc_mesh_new.restype = P
        lib.orc_mesh_new.argtypes = [i64, i64, P, P, P, P]
        lib.orc_mesh_free.argtypes = [P]
        lib.orc_mesh_set_distances.argtypes = [P, P]
        lib.orc_psi.argtypes = [I, P, P, i64]
        lib.orc_psi_branch.argtypes = [I, P, P, P, i64]
        lib.orc_face_values.argtypes = [P, I, P, P, P, P, P, P]
        lib.orc_rhs.argtypes = [P, I, P, P, P]
        lib.orc_step.argtypes = [P, I, I, D, i64, P, P]
        lib.orc_stage.argtypes = [P, I, I, I, D, P, P, P, P]
        lib.orc_step_modulated.argtypes = [P, I, I, D, i64, P, P, P]
        lib.orc_step_tlm.argtypes = [P, I, I, D, i64, P, P, P]
        lib.orc_rhs_adjoint.argtypes = [P, I, P, P, P, P]
        lib.orc_gradient.argtypes = [P, I, I, D, i64, P, P, P, P, P]
        lib.orc_set_threads.argtypes = [I]
        lib.orc_set_threads.restype = I
        lib.orc_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lim_id(lim) -> int:
    return LIMITERS[lim] if isinstance(lim, str) else int(lim)


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the oracle; returns the count in use."""
    return _load().orc_set_threads(int(n))


class OracleMesh:
    """The oracle's own copy of a face-based mesh (see ``workloads.Mesh``)."""

    def __init__(self, mesh):
        lib = _load()
        self._keep = (
            np.ascontiguousarray(mesh.face_cells, dtype=np.int32),
            _f64(mesh.normals),
            _f64(mesh.areas),
            _f64(mesh.volumes),
        )
        fc, nrm, ar, vol = self._keep
        self.C = int(mesh.n_cells)
        self.F = int(fc.shape[0])
        self.h = lib.orc_mesh_new(self.C, self.F, _ptr(fc), _ptr(nrm), _ptr(ar), _ptr(vol))
        if not self.h:
            raise ValueError(lib.orc_last_error().decode())
        # face distances of a non-uniform mesh (Algorithm 3's weights)
        dist = getattr(mesh, "distances", None)
        if dist is not None:
            self._dist = _f64(dist)
            if lib.orc_mesh_set_distances(self.h, _ptr(self._dist)) != 0:
                raise ValueError(lib.orc_last_error().decode())

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_mesh_free(self.h)
            self.h = None


def _om(mesh):
    return mesh if isinstance(mesh, OracleMesh) else OracleMesh(mesh)


def psi(lim, r):
    r = _f64(r)
    out = np.empty_like(r)
    _load().orc_psi(lim_id(lim), _ptr(r), _ptr(out), r.size)
    return out


def psi_branch(lim, r):
    r = _f64(r)
    p = np.empty_like(r)
    d = np.empty_like(r)
    _load().orc_psi_branch(lim_id(lim), _ptr(r), _ptr(p), _ptr(d), r.size)
    return p, d


def face_values(mesh, lim, theta, u):
    om = _om(mesh)
    th, uu = _f64(theta), _f64(u)
    thf = np.empty(om.F)
    sel = np.empty((om.F, 4), np.int32)
    du = np.empty(om.F)
    dU = np.empty(om.F)
    _load().orc_face_values(om.h, lim_id(lim), _ptr(th), _ptr(uu), _ptr(thf), _ptr(sel),
                            _ptr(du), _ptr(dU))
    return {"theta_f": thf, "s": sel[:, 0].copy(), "C": sel[:, 1].copy(), "D": sel[:, 2].copy(),
            "U": sel[:, 3].copy(), "du": du, "dU": dU}


def rhs(mesh, lim, theta, u):
    om = _om(mesh)
    th, uu = _f64(theta), _f64(u)
    R = np.empty(om.C)
    _load().orc_rhs(om.h, lim_id(lim), _ptr(th), _ptr(uu), _ptr(R))
    return R


def step(mesh, lim, rk, dt, nsteps, u, theta):
    om = _om(mesh)
    th = _f64(theta).copy()
    uu = _f64(u)
    rc = _load().orc_step(om.h, lim_id(lim), int(rk), float(dt), int(nsteps), _ptr(uu), _ptr(th))
    if rc:
        raise ValueError(_lib.orc_last_error().decode())
    return th


def step_modulated(mesh, lim, rk, dt, nsteps, u, g, theta):
    """nsteps steps where stage s of step n uses the velocity g[n*S + s] * u
    (S = 1 for Euler, 3 for SSP-RK3)."""
    om = _om(mesh)
    th = _f64(theta).copy()
    uu = _f64(u)
    S = 1 if int(rk) == 1 else 3
    gg = _f64(g).ravel()
    if gg.size < int(nsteps) * S:
        raise ValueError("need nsteps * stages velocity factors")
    rc = _load().orc_step_modulated(om.h, lim_id(lim), int(rk), float(dt), int(nsteps), _ptr(uu),
                                    _ptr(gg), _ptr(th))
    if rc:
        raise ValueError(_lib.orc_last_error().decode())
    return th


def stage(mesh, lim, rk, st, dt, theta_n, x, u):
    om = _om(mesh)
    thn, xx, uu = _f64(theta_n), _f64(x), _f64(u)
    y = np.empty(om.C)
    _load().orc_stage(om.h, lim_id(lim), int(rk), int(st), float(dt), _ptr(thn), _ptr(xx),
                      _ptr(uu), _ptr(y))
    return y


def step_tlm(mesh, lim, rk, dt, nsteps, u, theta, dtheta):
    om = _om(mesh)
    th = _f64(theta).copy()
    dth = _f64(dtheta).copy()
    uu = _f64(u)
    rc = _load().orc_step_tlm(om.h, lim_id(lim), int(rk), float(dt), int(nsteps), _ptr(uu),
                              _ptr(th), _ptr(dth))
    if rc:
        raise ValueError(_lib.orc_last_error().decode())
    return th, dth


def rhs_adjoint(mesh, lim, theta, u, mu):
    om = _om(mesh)
    th, uu, m = _f64(theta), _f64(u), _f64(mu)
    out = np.empty(om.C)
    _load().orc_rhs_adjoint(om.h, lim_id(lim), _ptr(th), _ptr(uu), _ptr(m), _ptr(out))
    return out


def gradient(mesh, lim, rk, dt, nsteps, u, theta0, target):
    """Returns (J, dJ/dtheta0) for J = 0.5 ||theta_T - target||^2."""
    om = _om(mesh)
    th0, tg, uu = _f64(theta0), _f64(target), _f64(u)
    g = np.empty(om.C)
    J = ctypes.c_double(0.0)
    rc = _load().orc_gradient(om.h, lim_id(lim), int(rk), float(dt), int(nsteps), _ptr(uu),
                              _ptr(th0), _ptr(tg), _ptr(g), ctypes.byref(J))
    if rc:
        raise ValueError(_lib.orc_last_error().decode())
    return J.value, g
