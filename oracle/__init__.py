"""Plain FP64 CPU oracle of the nonlinear Newmark-beta ground-response step.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs use it.  The CUDA library never
imports, links or calls anything here, and this package shares no code with it:
the two meet only in the seeded inputs of ``paper_2604_02755_gb300.synth``.

The arithmetic lives in ``oracle.c`` (plain C, FP64); this module compiles it
with gcc and marshals arguments through ctypes.  It is built twice from that one
source: ``liboracle.so`` (single thread) and ``liboracle_omp.so`` (the same code
with -fopenmp, its independent element, node and spring loops split over the host
cores; every sum keeps the single-thread order, so the two agree bit for bit).

Parity: every function is pinned by tests under ``tests/test_oracle_*.py``
against closed forms, invariants, brute force and exact symbolic integrals
(see each test's docstring for the passage of the paper it follows).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_libs = {}

SPRING_DTYPE = np.dtype([("tau", "<f8"), ("gR", "<f8"), ("tR", "<f8"), ("gmax", "<f8"), ("dir", "<i4"),
                         ("mode", "<i4")])
assert SPRING_DTYPE.itemsize == 40


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so and liboracle_omp.so (gcc -O2, ISO C11 so that
    no multiply-add contraction happens, no fast-math)."""
    src = os.path.join(_HERE, "oracle.c")
    newest = max(os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h")))
    for path, extra in ((_LIB_PATH, []), (_OMP_PATH, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < newest:
            tmp = path + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared"] + extra +
                                  ["-o", tmp, src, "-lm"])
            os.replace(tmp, path)
    return _LIB_PATH


class Model(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_elems", C.c_int64), ("n_faces", C.c_int64),
                ("conn", C.c_void_p), ("X", C.c_void_p), ("mat", C.c_void_p), ("n_mat", C.c_int32),
                ("matprops", C.c_void_p), ("faces", C.c_void_p), ("FX", C.c_void_p), ("fmat", C.c_void_p),
                ("fkind", C.c_void_p), ("n_springs", C.c_int32), ("dt", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("f1", C.c_double), ("f2", C.c_double), ("n_samples", C.c_int64),
                ("acc", C.c_void_p), ("x0_prev", C.c_int32)]


class State(C.Structure):
    _fields_ = [("u", C.c_void_p), ("v", C.c_void_p), ("a", C.c_void_p), ("q", C.c_void_p), ("du", C.c_void_p),
                ("D", C.c_void_p), ("th", C.c_void_p), ("step", C.c_int64), ("iters", C.c_int32),
                ("relres", C.c_double)]


class RO(C.Structure):
    _fields_ = [("G0", C.c_double), ("gref", C.c_double), ("alpha", C.c_double), ("beta", C.c_double)]


def lib(omp: bool = False):
    """The single-thread oracle, or (omp=True) the OpenMP build of the same source."""
    if omp not in _libs:
        build()
        L = C.CDLL(_OMP_PATH if omp else _LIB_PATH)
        dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_void_p
        L.or_shape.argtypes = [vp, vp]
        L.or_shape_dref.argtypes = [vp, vp]
        L.or_grad.argtypes = [vp, vp, vp]
        L.or_grad.restype = C.c_double
        L.or_bmatrix.argtypes = [vp, vp]
        L.or_quad_points.argtypes = [vp, vp]
        L.or_element_stiffness.argtypes = [vp, vp, vp]
        L.or_element_mass.argtypes = [vp, C.c_double, vp]
        L.or_face_dashpot.argtypes = [vp, C.c_double, C.c_double, C.c_double, vp]
        L.or_ro_params.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(RO)]
        for f in ("or_ro_g", "or_ro_dg", "or_ro_F"):
            getattr(L, f).argtypes = [C.c_double, C.POINTER(RO)]
            getattr(L, f).restype = C.c_double
        L.or_spring_update.argtypes = [vp, C.c_double, C.c_double, C.POINTER(RO)]
        L.or_spring_update.restype = C.c_double
        L.or_spring_tangent.argtypes = [vp, C.POINTER(RO)]
        L.or_spring_tangent.restype = C.c_double
        L.or_spring_dirs.argtypes = [C.c_int, vp, dp]
        L.or_spring_dirs.restype = C.c_int
        L.or_point_update.argtypes = [C.c_int, vp, C.c_double, C.c_double, C.POINTER(RO), vp, vp, vp, vp]
        L.or_elastic_D.argtypes = [C.c_int, vp, C.c_double, C.c_double, C.c_double, vp]
        L.or_state_init.argtypes = [C.POINTER(Model), C.POINTER(State)]
        L.or_state_init.restype = C.c_int
        L.or_step.argtypes = [C.POINTER(Model), C.POINTER(State)]
        L.or_step.restype = C.c_int
        L.or_operator.argtypes = [C.POINTER(Model), vp, C.c_int, vp, vp]
        L.or_operator.restype = C.c_int
        L.or_colouring.argtypes = [C.c_int64, C.c_int64, vp, vp]
        L.or_colouring.restype = C.c_int
        L.or_input_velocity.argtypes = [C.POINTER(Model), C.c_int64, C.c_int]
        L.or_input_velocity.restype = C.c_double
        L.or_strain.argtypes = [C.POINTER(Model), C.c_int64, C.c_int, vp, vp]
        L.or_coarse_map.argtypes = [C.c_int64, C.c_int64, vp, vp, vp]
        L.or_coarse_map.restype = C.c_int64
        L.or_p1_grads.argtypes = [vp, vp, dp]
        L.or_coarse_operator.argtypes = [C.POINTER(Model), vp, C.c_int, C.c_int64, vp, vp, vp]
        L.or_coarse_operator.restype = C.c_int
        L.or_threads.argtypes = [C.c_int]
        L.or_threads.restype = C.c_int
        _libs[omp] = L
    return _libs[omp]


def threads(n: int = 0, omp: bool = True) -> int:
    """Set (n > 0) and return the thread count of the OpenMP build (1 for the plain one)."""
    return int(lib(omp).or_threads(int(n)))


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ element-level wrappers

def shape(L):
    L = np.ascontiguousarray(L, np.float64); N = np.zeros(10)
    lib().or_shape(_p(L), _p(N)); return N


def shape_dref(L):
    L = np.ascontiguousarray(L, np.float64); dN = np.zeros((10, 3))
    lib().or_shape_dref(_p(L), _p(dN)); return dN


def grad(X, L):
    X = np.ascontiguousarray(X, np.float64); L = np.ascontiguousarray(L, np.float64); G = np.zeros((10, 3))
    det = lib().or_grad(_p(X), _p(L), _p(G)); return G, det


def bmatrix(G):
    G = np.ascontiguousarray(G, np.float64); B = np.zeros((6, 30))
    lib().or_bmatrix(_p(G), _p(B)); return B


def quad_points():
    L = np.zeros((4, 4)); w = np.zeros(1)
    lib().or_quad_points(_p(L), _p(w)); return L, float(w[0])


def element_stiffness(X, D):
    X = np.ascontiguousarray(X, np.float64)
    D = np.ascontiguousarray(np.broadcast_to(D, (4, 6, 6)), np.float64)
    K = np.zeros((30, 30)); lib().or_element_stiffness(_p(X), _p(D), _p(K)); return K


def element_mass(X, rho):
    X = np.ascontiguousarray(X, np.float64); M = np.zeros((10, 10))
    lib().or_element_mass(_p(X), float(rho), _p(M)); return M


def face_dashpot(FX, rho, vs, vp):
    FX = np.ascontiguousarray(FX, np.float64); Cm = np.zeros((18, 18))
    lib().or_face_dashpot(_p(FX), float(rho), float(vs), float(vp), _p(Cm)); return Cm


def ro_params(rho, vs, gamma_ref, h_max) -> RO:
    p = RO(); lib().or_ro_params(rho, vs, gamma_ref, h_max, C.byref(p)); return p


def ro_g(tau, p): return lib().or_ro_g(float(tau), C.byref(p))
def ro_dg(tau, p): return lib().or_ro_dg(float(tau), C.byref(p))
def ro_F(gamma, p): return lib().or_ro_F(float(gamma), C.byref(p))


def spring_update(s: np.ndarray, g_new: float, dg: float, p: RO) -> float:
    """Updates the one-element SPRING_DTYPE array `s` in place; returns the tangent."""
    assert s.dtype == SPRING_DTYPE and s.size == 1
    return lib().or_spring_update(_p(s), float(g_new), float(dg), C.byref(p))


def spring_tangent(s: np.ndarray, p: RO) -> float:
    return lib().or_spring_tangent(_p(s), C.byref(p))


def spring_dirs(S: int):
    q = np.zeros((S, 6)); w = C.c_double()
    if lib().or_spring_dirs(S, _p(q), C.byref(w)) != 0:
        raise ValueError("need at least 5 springs")
    return q, w.value


def point_update(q, w, Kb, p, eps, deps, springs):
    q = np.ascontiguousarray(q, np.float64); eps = np.ascontiguousarray(eps, np.float64)
    deps = np.ascontiguousarray(deps, np.float64); D = np.zeros((6, 6))
    lib().or_point_update(q.shape[0], _p(q), float(w), float(Kb), C.byref(p), _p(eps), _p(deps), _p(springs), _p(D))
    return D


def elastic_D(q, w, Kb, G0):
    q = np.ascontiguousarray(q, np.float64); D = np.zeros((6, 6))
    lib().or_elastic_D(q.shape[0], _p(q), float(w), float(Kb), float(G0), _p(D)); return D


def colouring(conn: np.ndarray, n_nodes: int):
    conn = np.ascontiguousarray(conn, np.int32); col = np.zeros(conn.shape[0], np.int32)
    nc = lib().or_colouring(conn.shape[0], int(n_nodes), _p(conn), _p(col))
    if nc < 0:
        raise ValueError("more than 64 colours")
    return col, nc


def coarse_map(conn: np.ndarray, n_nodes: int):
    """(cid [N], par [N][2], n_coarse) of the two-level preconditioner's P2 -> P1 map."""
    conn = np.ascontiguousarray(conn, np.int32)
    cid = np.zeros(n_nodes, np.int32); par = np.zeros((n_nodes, 2), np.int32)
    nc = lib().or_coarse_map(conn.shape[0], int(n_nodes), _p(conn), _p(cid), _p(par))
    if nc < 0:
        raise ValueError("inconsistent quadratic mesh for the coarse map")
    return cid, par, int(nc)


def p1_grads(X):
    X = np.ascontiguousarray(X, np.float64); g = np.zeros((4, 3)); v = C.c_double()
    lib().or_p1_grads(_p(X), _p(g), C.byref(v)); return g, v.value


# ------------------------------------------------------------------ model level

MAT_KEYS = ("rho", "vs", "vp", "gamma_ref", "h_max", "rayleigh_h")


class Oracle:
    """The whole model on the CPU.  Inputs mirror the library's: node
    coordinates + connectivity (or explicit per-element node coordinates, which
    lets a test build laterally periodic columns), materials, boundary faces,
    springs per point, dt, tolerance and outcrop acceleration samples."""

    def __init__(self, xyz, conn, mat, materials, faces=None, face_elem=None, face_kind=None, n_springs=10,
                 dt=0.01, acc=None, tol=1e-8, max_iter=10000, f1=0.1, f2=2.5, x0_prev=True, elem_xyz=None,
                 face_xyz=None, omp=False):
        self.L = lib(omp)
        self.conn = np.ascontiguousarray(conn, np.int32)
        E = self.conn.shape[0]
        self.n_nodes = int(np.max(self.conn)) + 1 if xyz is None else int(np.asarray(xyz).shape[0])
        if elem_xyz is None:
            elem_xyz = np.asarray(xyz, np.float64)[self.conn]
        self.X = np.ascontiguousarray(elem_xyz, np.float64).reshape(E, 10, 3)
        self.mat = np.ascontiguousarray(mat, np.int32)
        self.matprops = np.ascontiguousarray([[m[k] for k in MAT_KEYS] for m in materials], np.float64)
        if faces is None:
            faces = np.zeros((0, 6), np.int32); face_elem = np.zeros(0, np.int32); face_kind = np.zeros(0, np.int32)
        self.faces = np.ascontiguousarray(faces, np.int32).reshape(-1, 6)
        F = self.faces.shape[0]
        self.fmat = np.ascontiguousarray(self.mat[np.asarray(face_elem, np.int64)] if F else np.zeros(0), np.int32)
        self.fkind = np.ascontiguousarray(face_kind, np.int32)
        if face_xyz is None:
            face_xyz = np.asarray(xyz, np.float64)[self.faces[:, :3]] if F else np.zeros((0, 3, 3))
        self.FX = np.ascontiguousarray(face_xyz, np.float64).reshape(F, 3, 3)
        self.acc = np.ascontiguousarray(acc if acc is not None else np.zeros((1, 3)), np.float64).reshape(-1, 3)
        self.S = int(n_springs)
        self.m = Model(n_nodes=self.n_nodes, n_elems=E, n_faces=F, conn=_p(self.conn), X=_p(self.X), mat=_p(self.mat),
                       n_mat=len(materials), matprops=_p(self.matprops), faces=_p(self.faces), FX=_p(self.FX),
                       fmat=_p(self.fmat), fkind=_p(self.fkind), n_springs=self.S, dt=float(dt), tol=float(tol),
                       max_iter=int(max_iter), f1=float(f1), f2=float(f2), n_samples=self.acc.shape[0],
                       acc=_p(self.acc), x0_prev=1 if x0_prev else 0)
        N = self.n_nodes
        self.u = np.zeros((N, 3)); self.v = np.zeros((N, 3)); self.a = np.zeros((N, 3))
        self.q = np.zeros((N, 3)); self.du = np.zeros((N, 3))
        self.D = np.zeros((E, 4, 6, 6))
        self.th = np.zeros((E, 4, self.S), SPRING_DTYPE)
        self.s = State(u=_p(self.u), v=_p(self.v), a=_p(self.a), q=_p(self.q), du=_p(self.du), D=_p(self.D),
                       th=_p(self.th), step=0, iters=0, relres=0.0)
        if self.L.or_state_init(C.byref(self.m), C.byref(self.s)) != 0:
            raise ValueError("oracle state init failed (n_springs >= 5 required)")

    @classmethod
    def from_workload(cls, wl, **kw):
        m = wl.mesh
        return cls(m.xyz, m.conn, m.mat, wl.materials, m.faces, m.face_elem, m.face_kind, wl.n_springs, wl.dt,
                   wl.wave, **kw)

    @property
    def step_index(self) -> int:
        return int(self.s.step)

    @property
    def iters(self) -> int:
        return int(self.s.iters)

    def step(self) -> int:
        rc = self.L.or_step(C.byref(self.m), C.byref(self.s))
        if rc != 0:
            raise RuntimeError("oracle step failed: %d" % rc)
        return self.iters

    def operator(self, which: str, x: np.ndarray, D=None) -> np.ndarray:
        code = {"K": 0, "M": 1, "Cb": 2, "A": 3, "Cr": 4}[which]
        x = np.ascontiguousarray(x, np.float64).reshape(self.n_nodes, 3)
        y = np.zeros_like(x)
        D = self.D if D is None else np.ascontiguousarray(D, np.float64)
        self.L.or_operator(C.byref(self.m), _p(D), code, _p(x), _p(y))
        return y

    def coarse_operator(self, which: str, xc: np.ndarray, cid: np.ndarray, n_coarse: int, D=None) -> np.ndarray:
        """y_c = Op_c x_c of the linear-element coarse model (K1, M1, Cb1 or A1)."""
        code = {"K": 0, "M": 1, "Cb": 2, "A": 3}[which]
        xc = np.ascontiguousarray(xc, np.float64).reshape(n_coarse, 3)
        yc = np.zeros_like(xc)
        D = self.D if D is None else np.ascontiguousarray(D, np.float64)
        cid = np.ascontiguousarray(cid, np.int32)
        if self.L.or_coarse_operator(C.byref(self.m), _p(D), code, int(n_coarse), _p(cid), _p(xc), _p(yc)) != 0:
            raise ValueError("bad coarse operator")
        return yc

    def input_velocity(self, n: int) -> np.ndarray:
        return np.array([self.L.or_input_velocity(C.byref(self.m), int(n), c) for c in range(3)])

    def strain(self, e: int, qp: int, u: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, np.float64); eps = np.zeros(6)
        self.L.or_strain(C.byref(self.m), int(e), int(qp), _p(u), _p(eps)); return eps
