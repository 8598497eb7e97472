"""Thin ctypes binding of the C ABI in include/ns.h (same function names).

Only argument marshalling lives here: every step of the time stepper runs in
the CUDA library libns.so.  Importing works without a GPU; loading the library
fails loudly if it has not been built (``paper_2604_02755_gb300.build.build()``),
and every call that needs the device fails with the library's own error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NS_OK = 0
NS_ERR = {-1: "NS_ERR_INVALID_ARG", -2: "NS_ERR_OOM_DEVICE", -3: "NS_ERR_OOM_PINNED", -4: "NS_ERR_CUDA",
          -5: "NS_ERR_BAD_MESH", -6: "NS_ERR_NOT_CONVERGED", -7: "NS_ERR_TIMEOUT", -8: "NS_ERR_STATE"}
NS_PREC_FP64, NS_PREC_FP64_IR, NS_PREC_FP64_IR16 = 0, 1, 2
NS_SCATTER_ATOMIC, NS_SCATTER_COLOUR = 0, 1
NS_STREAM_RING, NS_STREAM_ZERO_COPY = 0, 1
NS_FIELD = {"u": 0, "v": 1, "a": 2, "q": 3, "du": 4}
NS_OP = {"K": 0, "M": 1, "Cb": 2, "A": 3, "Cr": 4}

SPRING_DTYPE = np.dtype([("tau", "<f8"), ("gR", "<f8"), ("tR", "<f8"), ("gmax", "<f8"), ("dir", "<i4"),
                         ("mode", "<i4")])


class NsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (NS_ERR.get(code, "NS_ERR"), code, msg))
        self.code = code


class ns_config(C.Structure):
    _fields_ = [("n_springs", C.c_int32), ("dt", C.c_double), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32),
                ("x0_prev", C.c_int32), ("precision", C.c_int32), ("scatter", C.c_int32), ("chunk_elems", C.c_int64),
                ("ring_depth", C.c_int32), ("device_state_budget", C.c_int64), ("rayleigh_f1", C.c_double),
                ("rayleigh_f2", C.c_double), ("surface_ring_steps", C.c_int64), ("device", C.c_int32),
                ("timing", C.c_int32), ("inner_max_iter", C.c_int32), ("inner_tol", C.c_double),
                ("wait_timeout_s", C.c_double), ("graphs", C.c_int32), ("stage_elements", C.c_int32),
                ("l2_prefetch", C.c_int32), ("pair_operator", C.c_int32), ("stream_mode", C.c_int32),
                ("spring_tile_points", C.c_int32), ("spring_tile_blocks", C.c_int32),
                ("spring_tensor_cores", C.c_int32), ("fault_pinned_alloc", C.c_int32),
                ("fault_state_copy", C.c_int32), ("multigrid", C.c_int32), ("coarse_max_iter", C.c_int32),
                ("coarse_tol", C.c_double), ("shared_members", C.c_int32), ("local_gather", C.c_int32)]


class ns_material(C.Structure):
    _fields_ = [("rho", C.c_double), ("vs", C.c_double), ("vp", C.c_double), ("gamma_ref", C.c_double),
                ("h_max", C.c_double), ("rayleigh_h", C.c_double)]


class ns_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("cg_iters_total", C.c_int64), ("cg_iters_last", C.c_int32),
                ("inner_iters_last", C.c_int32), ("relres_last", C.c_double), ("kernel_launches", C.c_int64),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("resident_elems", C.c_int64),
                ("streamed_elems", C.c_int64), ("ms_rhs", C.c_double), ("ms_jacobi", C.c_double),
                ("ms_solve", C.c_double), ("ms_newmark", C.c_double), ("ms_springs", C.c_double),
                ("ms_step", C.c_double), ("n_ebe64", C.c_int64), ("n_ebe32", C.c_int64), ("n_spring", C.c_int64),
                ("ms_ebe64", C.c_double), ("ms_ebe32", C.c_double), ("ms_spring", C.c_double),
                ("ms_stream_wall", C.c_double), ("ms_advance", C.c_double),
                ("h2d_bytes_early", C.c_int64), ("inner_iters_total", C.c_int64),
                ("spring_moved", C.c_int64), ("spring_reversals", C.c_int64), ("spring_fp64_roots", C.c_int64),
                ("coarse_iters_total", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ns_tuning(C.Structure):
    _fields_ = [("n_tile", C.c_int32), ("tile_points", C.c_int32 * 16), ("tile_blocks", C.c_int32 * 16),
                ("tile_ms", C.c_float * 16), ("chosen_tile_points", C.c_int32), ("chosen_tile_blocks", C.c_int32),
                ("n_chunk", C.c_int32), ("chunk_elems", C.c_int64 * 6), ("chunk_gbps", C.c_float * 6),
                ("chosen_chunk_elems", C.c_int64)]

    def as_dict(self):
        return {"tile_points": list(self.tile_points[:self.n_tile]), "tile_blocks": list(self.tile_blocks[:self.n_tile]),
                "tile_ms": list(self.tile_ms[:self.n_tile]),
                "chosen_tile_points": self.chosen_tile_points, "chosen_tile_blocks": self.chosen_tile_blocks,
                "chunk_elems": list(self.chunk_elems[:self.n_chunk]), "chunk_gbps": list(self.chunk_gbps[:self.n_chunk]),
                "chosen_chunk_elems": self.chosen_chunk_elems}


class ns_server_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("device_budget", C.c_int64), ("pinned_budget", C.c_int64),
                ("max_active", C.c_int32), ("quantum_steps", C.c_int32), ("batch", C.c_int32)]


class ns_case(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("xyz", C.c_void_p), ("n_elems", C.c_int64), ("conn", C.c_void_p),
                ("mat", C.c_void_p), ("n_mat", C.c_int32), ("mats", C.c_void_p), ("n_faces", C.c_int64),
                ("faces", C.c_void_p), ("face_elem", C.c_void_p), ("face_kind", C.c_void_p), ("n_surf", C.c_int64),
                ("surf", C.c_void_p), ("n_samples", C.c_int64), ("acc", C.c_void_p), ("cfg", ns_config),
                ("n_steps", C.c_int64)]


class ns_case_stats(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("streamed", C.c_int32), ("batches", C.c_int32),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("device_bytes", C.c_int64), ("state_bytes", C.c_int64), ("elem_steps", C.c_int64),
                ("ms_device", C.c_double), ("kernel_launches", C.c_int64), ("t_reform", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


NS_CASE_QUEUED, NS_CASE_RUNNING, NS_CASE_DONE, NS_CASE_FAILED = 0, 1, 2, 3

EXPORTED = ["ns_config_default", "ns_create", "ns_upload_mesh", "ns_set_materials", "ns_set_boundary",
            "ns_set_ground_motion", "ns_advance", "ns_read_surface", "ns_read_state", "ns_write_state",
            "ns_read_nodal", "ns_write_nodal", "ns_apply_operator", "ns_spring_points", "ns_get_stats",
            "ns_reset_stats", "ns_checkpoint_size", "ns_checkpoint", "ns_restore", "ns_destroy", "ns_last_error",
            "ns_spring_directions", "ns_colour_elements", "ns_state_bytes", "ns_spring_points_noalloc",
            "ns_spring_points_noalloc_capacity", "ns_set_members", "ns_set_member_ground_motion",
            "ns_get_member_iters", "ns_set_member_springs", "ns_autotune", "ns_autotune_steps", "ns_apply_coarse_operator", "ns_coarse_map", "ns_case_bytes", "ns_server_create", "ns_server_submit", "ns_server_status",
            "ns_server_wait", "ns_server_result", "ns_server_release", "ns_server_destroy"]

_lib = None


def lib():
    """The loaded libns.so (raises if it was never built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError("libns.so is not built; run paper_2604_02755_gb300.build.build() "
                              "(or __graft_entry__.build()) first")
        L = C.CDLL(_build.LIB)
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        sig = {
            "ns_config_default": ([C.POINTER(ns_config)], None),
            "ns_create": ([C.POINTER(vp), C.POINTER(ns_config)], C.c_int),
            "ns_upload_mesh": ([vp, i64, vp, i64, vp, vp], C.c_int),
            "ns_set_materials": ([vp, i32, vp], C.c_int),
            "ns_set_boundary": ([vp, i64, vp, vp, vp, i64, vp], C.c_int),
            "ns_set_ground_motion": ([vp, i64, d, vp], C.c_int),
            "ns_advance": ([vp, i64], C.c_int),
            "ns_read_surface": ([vp, i64, i64, vp, vp, vp], C.c_int),
            "ns_read_state": ([vp, i64, i64, vp, vp], C.c_int),
            "ns_write_state": ([vp, i64, i64, vp, vp], C.c_int),
            "ns_read_nodal": ([vp, i32, vp], C.c_int),
            "ns_write_nodal": ([vp, i32, vp], C.c_int),
            "ns_apply_operator": ([vp, i32, vp, vp], C.c_int),
            "ns_spring_points": ([vp, i64, vp, vp, vp, vp, vp], C.c_int),
            "ns_get_stats": ([vp, C.POINTER(ns_stats)], C.c_int),
            "ns_reset_stats": ([vp], C.c_int),
            "ns_checkpoint_size": ([vp, C.POINTER(i64)], C.c_int),
            "ns_checkpoint": ([vp, vp, i64], C.c_int),
            "ns_restore": ([vp, vp, i64], C.c_int),
            "ns_destroy": ([vp], None),
            "ns_last_error": ([vp], C.c_char_p),
            "ns_spring_directions": ([i32, vp, C.POINTER(d)], C.c_int),
            "ns_colour_elements": ([i64, i64, vp, vp, C.POINTER(i32)], C.c_int),
            "ns_state_bytes": ([i64, i32], i64),
            "ns_spring_points_noalloc": ([vp, i64, vp, vp, vp, vp, vp], C.c_int),
            "ns_spring_points_noalloc_capacity": ([i32], i64),
            "ns_set_members": ([vp, i32, vp, vp], C.c_int),
            "ns_set_member_ground_motion": ([vp, i32, i64, d, vp], C.c_int),
            "ns_get_member_iters": ([vp, i32, vp], C.c_int),
            "ns_set_member_springs": ([vp, i32, vp], C.c_int),
            "ns_autotune": ([vp, C.POINTER(ns_tuning)], C.c_int),
            "ns_autotune_steps": ([vp, C.c_int32, C.POINTER(ns_tuning)], C.c_int),
            "ns_apply_coarse_operator": ([vp, i32, i64, vp, vp], C.c_int),
            "ns_coarse_map": ([i64, i64, vp, vp, vp, C.POINTER(i64)], C.c_int),
            "ns_case_bytes": ([C.POINTER(ns_case), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)], C.c_int),
            "ns_server_create": ([C.POINTER(vp), C.POINTER(ns_server_config)], C.c_int),
            "ns_server_submit": ([vp, C.POINTER(ns_case), C.POINTER(i64)], C.c_int),
            "ns_server_status": ([vp, i64, C.POINTER(ns_case_stats)], C.c_int),
            "ns_server_wait": ([vp, i64, d], C.c_int),
            "ns_server_result": ([vp, i64, vp, vp, vp], C.c_int),
            "ns_server_release": ([vp, i64], C.c_int),
            "ns_server_destroy": ([vp], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(ctx, rc):
    if rc != NS_OK:
        raise NsError(rc, lib().ns_last_error(ctx).decode())


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ------------------------------------------------------------------ same-name wrappers

def ns_config_default(**overrides) -> ns_config:
    cfg = ns_config()
    lib().ns_config_default(C.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def ns_create(cfg: ns_config):
    h = C.c_void_p()
    _check(None, lib().ns_create(C.byref(h), C.byref(cfg)))
    return h


def ns_upload_mesh(ctx, xyz, conn, mat):
    xyz = _f64(xyz); conn = _i32(conn); mat = _i32(mat)
    _check(ctx, lib().ns_upload_mesh(ctx, xyz.shape[0], _p(xyz), conn.shape[0], _p(conn), _p(mat)))


def ns_set_materials(ctx, materials):
    arr = (ns_material * len(materials))()
    for i, m in enumerate(materials):
        arr[i] = ns_material(m["rho"], m["vs"], m["vp"], m["gamma_ref"], m["h_max"], m["rayleigh_h"])
    _check(ctx, lib().ns_set_materials(ctx, len(materials), C.cast(arr, C.c_void_p)))


def ns_set_boundary(ctx, faces, face_elem, face_kind, surf):
    faces = _i32(faces).reshape(-1, 6); face_elem = _i32(face_elem); face_kind = _i32(face_kind); surf = _i32(surf)
    _check(ctx, lib().ns_set_boundary(ctx, faces.shape[0], _p(faces), _p(face_elem), _p(face_kind), surf.shape[0],
                                      _p(surf)))


def ns_set_ground_motion(ctx, acc, dt):
    acc = _f64(acc).reshape(-1, 3)
    _check(ctx, lib().ns_set_ground_motion(ctx, acc.shape[0], float(dt), _p(acc)))


def ns_set_members(ctx, elem_off, node_off):
    eo = np.ascontiguousarray(elem_off, np.int64); no = np.ascontiguousarray(node_off, np.int64)
    _check(ctx, lib().ns_set_members(ctx, eo.shape[0] - 1, _p(eo), _p(no)))


def ns_set_member_ground_motion(ctx, member, acc, dt):
    acc = _f64(acc).reshape(-1, 3)
    _check(ctx, lib().ns_set_member_ground_motion(ctx, int(member), acc.shape[0], float(dt), _p(acc)))


def ns_set_member_springs(ctx, S):
    S = np.ascontiguousarray(S, np.int32)
    _check(ctx, lib().ns_set_member_springs(ctx, S.shape[0], _p(S)))


def ns_get_member_iters(ctx, M):
    out = np.zeros(M, np.int32)
    _check(ctx, lib().ns_get_member_iters(ctx, int(M), _p(out)))
    return out


def ns_advance(ctx, nsteps):
    _check(ctx, lib().ns_advance(ctx, int(nsteps)))


def ns_read_surface(ctx, step0, nsteps, n_surf, fields=("u", "v", "a")):
    out = {k: np.zeros((nsteps, n_surf, 3)) for k in fields}
    _check(ctx, lib().ns_read_surface(ctx, int(step0), int(nsteps), _p(out.get("u")), _p(out.get("v")),
                                      _p(out.get("a"))))
    return out


def ns_read_state(ctx, e0, n, n_springs, theta=True, D=True):
    th = np.zeros((n, 4, n_springs), SPRING_DTYPE) if theta else None
    Dm = np.zeros((n, 4, 6, 6)) if D else None
    _check(ctx, lib().ns_read_state(ctx, int(e0), int(n), _p(th), _p(Dm)))
    return th, Dm


def ns_write_state(ctx, e0, theta=None, D=None):
    n = (theta.shape[0] if theta is not None else D.shape[0])
    th = None if theta is None else np.ascontiguousarray(theta, SPRING_DTYPE)
    Dm = None if D is None else _f64(D)
    _check(ctx, lib().ns_write_state(ctx, int(e0), int(n), _p(th), _p(Dm)))


def ns_read_nodal(ctx, field, n_nodes):
    out = np.zeros((n_nodes, 3))
    _check(ctx, lib().ns_read_nodal(ctx, NS_FIELD[field], _p(out)))
    return out


def ns_write_nodal(ctx, field, x):
    x = _f64(x)
    _check(ctx, lib().ns_write_nodal(ctx, NS_FIELD[field], _p(x)))


def ns_apply_operator(ctx, op, x):
    x = _f64(x).reshape(-1, 3)
    y = np.zeros_like(x)
    _check(ctx, lib().ns_apply_operator(ctx, NS_OP[op], _p(x), _p(y)))
    return y


def ns_apply_coarse_operator(ctx, op, xc):
    """y_c = Op_c x_c of the two-level preconditioner's coarse (linear-element) model."""
    xc = _f64(xc).reshape(-1, 3)
    yc = np.zeros_like(xc)
    _check(ctx, lib().ns_apply_coarse_operator(ctx, NS_OP[op], xc.shape[0], _p(xc), _p(yc)))
    return yc


def ns_coarse_map(conn, n_nodes):
    """(cid [N], par [N][2], n_coarse) of the coarse level (host-only helper)."""
    conn = _i32(conn)
    cid = np.zeros(int(n_nodes), np.int32); par = np.zeros((int(n_nodes), 2), np.int32); nc = C.c_int64()
    rc = lib().ns_coarse_map(conn.shape[0], int(n_nodes), _p(conn), _p(cid), _p(par), C.byref(nc))
    if rc != NS_OK:
        raise NsError(rc, "coarse map failed")
    return cid, par, nc.value


def ns_spring_points(ctx, mat, eps, deps, theta):
    mat = _i32(mat); eps = _f64(eps); deps = _f64(deps)
    theta = np.ascontiguousarray(theta, SPRING_DTYPE)
    D = np.zeros((mat.shape[0], 6, 6))
    _check(ctx, lib().ns_spring_points(ctx, mat.shape[0], _p(mat), _p(eps), _p(deps), _p(theta), _p(D)))
    return theta, D


def ns_spring_points_noalloc(ctx, mat, eps, deps, theta):
    """Same as ns_spring_points, through the entry point that allocates no device memory."""
    mat = _i32(mat); eps = _f64(eps); deps = _f64(deps)
    theta = np.ascontiguousarray(theta, SPRING_DTYPE)
    D = np.zeros((mat.shape[0], 6, 6))
    _check(ctx, lib().ns_spring_points_noalloc(ctx, mat.shape[0], _p(mat), _p(eps), _p(deps), _p(theta), _p(D)))
    return theta, D


def ns_spring_points_noalloc_capacity(S):
    return int(lib().ns_spring_points_noalloc_capacity(int(S)))


def ns_get_stats(ctx) -> dict:
    st = ns_stats()
    _check(ctx, lib().ns_get_stats(ctx, C.byref(st)))
    return st.as_dict()


def ns_autotune(ctx) -> dict:
    t = ns_tuning()
    _check(ctx, lib().ns_autotune(ctx, C.byref(t)))
    return t.as_dict()


def ns_autotune_steps(ctx, nsteps: int) -> dict:
    t = ns_tuning()
    _check(ctx, lib().ns_autotune_steps(ctx, int(nsteps), C.byref(t)))
    return t.as_dict()


def ns_reset_stats(ctx):
    _check(ctx, lib().ns_reset_stats(ctx))


def ns_checkpoint_size(ctx) -> int:
    n = C.c_int64()
    _check(ctx, lib().ns_checkpoint_size(ctx, C.byref(n)))
    return n.value


def ns_checkpoint(ctx) -> np.ndarray:
    buf = np.zeros(ns_checkpoint_size(ctx), np.uint8)
    _check(ctx, lib().ns_checkpoint(ctx, _p(buf), buf.size))
    return buf


def ns_restore(ctx, buf):
    buf = np.ascontiguousarray(buf, np.uint8)
    _check(ctx, lib().ns_restore(ctx, _p(buf), buf.size))


def ns_destroy(ctx):
    if ctx:
        lib().ns_destroy(ctx)


def ns_last_error(ctx) -> str:
    return lib().ns_last_error(ctx).decode()


def ns_spring_directions(S):
    q = np.zeros((S, 6)); w = C.c_double()
    rc = lib().ns_spring_directions(int(S), _p(q), C.byref(w))
    if rc != NS_OK:
        raise NsError(rc, "invalid spring count")
    return q, w.value


def ns_colour_elements(conn, n_nodes):
    conn = _i32(conn)
    col = np.zeros(conn.shape[0], np.int32); nc = C.c_int32()
    rc = lib().ns_colour_elements(conn.shape[0], int(n_nodes), _p(conn), _p(col), C.byref(nc))
    if rc != NS_OK:
        raise NsError(rc, "colouring failed")
    return col, nc.value


def ns_state_bytes(n_elems, S):
    return int(lib().ns_state_bytes(int(n_elems), int(S)))


# ------------------------------------------------------------------ convenience wrapper

class Simulation:
    """One context holding a workload (synth.Workload-like: mesh, materials,
    n_springs, dt, wave).  Methods call the same-name functions above."""

    def __init__(self, wl, **cfg_overrides):
        cfg = dict(n_springs=wl.n_springs, dt=wl.dt)
        cfg.update(cfg_overrides)
        self.cfg = ns_config_default(**cfg)
        self.ctx = ns_create(self.cfg)
        m = wl.mesh
        self.n_nodes, self.n_elems, self.n_surf = m.n_nodes, m.n_elems, int(m.surf.shape[0])
        self.S = wl.n_springs
        try:
            ns_upload_mesh(self.ctx, m.xyz, m.conn, m.mat)
            ns_set_materials(self.ctx, wl.materials)
            ns_set_boundary(self.ctx, m.faces, m.face_elem, m.face_kind, m.surf)
            ns_set_ground_motion(self.ctx, wl.wave, wl.dt)
        except Exception:
            self.close()
            raise

    def advance(self, n):
        ns_advance(self.ctx, n)

    def surface(self, step0, n, fields=("u", "v", "a")):
        return ns_read_surface(self.ctx, step0, n, self.n_surf, fields)

    def nodal(self, field):
        return ns_read_nodal(self.ctx, field, self.n_nodes)

    def state(self, e0=0, n=None, theta=True, D=True):
        n = self.n_elems - e0 if n is None else n
        return ns_read_state(self.ctx, e0, n, self.S, theta, D)

    def stats(self):
        return ns_get_stats(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            ns_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSimulation(Simulation):
    """Members advanced together in one context (synth.Ensemble-like: one mesh shared by
    all members, per-member materials and waves).  shared=True (default): the context
    stores the mesh once (ns_config.shared_members = M) and keeps per member only the
    tangent, spring state, materials and node vectors; shared=False: it holds the disjoint
    union of M copies of the mesh (synth.union_of_copies, ns_set_members).  Either way
    member m's surface response is rows [m * n_surf, (m + 1) * n_surf) of the context's
    surface record."""

    def __init__(self, ens, shared=True, **cfg_overrides):
        from . import synth
        M = len(ens.members)
        cfg = dict(n_springs=ens.n_springs, dt=ens.dt)
        if shared:
            cfg["shared_members"] = M
        cfg.update(cfg_overrides)
        self.cfg = ns_config_default(**cfg)
        self.ctx = ns_create(self.cfg)
        self.M = M
        nmb = int(ens.mesh.mat.max()) + 1
        assert all(len(mats) == nmb for mats in ens.members), "one material row per layer and member"
        m0 = ens.mesh
        self.member_surf = int(m0.surf.shape[0])
        self.n_nodes, self.n_elems, self.n_surf = M * m0.n_nodes, M * m0.n_elems, M * self.member_surf
        self.S = ens.n_springs
        try:
            table = [row for mats in ens.members for row in mats]
            if shared:
                ns_upload_mesh(self.ctx, m0.xyz, m0.conn, m0.mat)
                ns_set_materials(self.ctx, table)
                ns_set_boundary(self.ctx, m0.faces, m0.face_elem, m0.face_kind, m0.surf)
            else:
                U = synth.union_of_copies(m0, M, n_materials=nmb)
                ns_upload_mesh(self.ctx, U.mesh.xyz, U.mesh.conn, U.mesh.mat)
                ns_set_materials(self.ctx, table)
                ns_set_boundary(self.ctx, U.mesh.faces, U.mesh.face_elem, U.mesh.face_kind, U.mesh.surf)
                ns_set_members(self.ctx, U.elem_off, U.node_off)
            ns_set_ground_motion(self.ctx, ens.waves[0], ens.dt)
            for m in range(M):
                ns_set_member_ground_motion(self.ctx, m, ens.waves[m], ens.dt)
        except Exception:
            self.close()
            raise

    def member_surface(self, m, step0, n, fields=("u", "v", "a")):
        s = self.surface(step0, n, fields)
        k = self.member_surf
        return {f: a[:, m * k:(m + 1) * k] for f, a in s.items()}

    def member_iters(self):
        return ns_get_member_iters(self.ctx, self.M)


# ------------------------------------------------------------------ served ensemble (include/ns_server.h)

def _case(wl, n_steps, keep, **cfg_overrides):
    """ns_case for a workload (synth.Workload-like); `keep` collects the arrays it points to."""
    m = wl.mesh
    arrs = dict(xyz=_f64(m.xyz), conn=_i32(m.conn), mat=_i32(m.mat), faces=_i32(m.faces).reshape(-1, 6),
                face_elem=_i32(m.face_elem), face_kind=_i32(m.face_kind), surf=_i32(m.surf),
                acc=_f64(wl.wave).reshape(-1, 3))
    mats = (ns_material * len(wl.materials))()
    for i, r in enumerate(wl.materials):
        mats[i] = ns_material(r["rho"], r["vs"], r["vp"], r["gamma_ref"], r["h_max"], r["rayleigh_h"])
    keep.append((arrs, mats))
    cfg = dict(n_springs=wl.n_springs, dt=wl.dt)
    cfg.update(cfg_overrides)
    return ns_case(n_nodes=arrs["xyz"].shape[0], xyz=_p(arrs["xyz"]), n_elems=arrs["conn"].shape[0],
                   conn=_p(arrs["conn"]), mat=_p(arrs["mat"]), n_mat=len(wl.materials),
                   mats=C.cast(mats, C.c_void_p), n_faces=arrs["faces"].shape[0], faces=_p(arrs["faces"]),
                   face_elem=_p(arrs["face_elem"]), face_kind=_p(arrs["face_kind"]), n_surf=arrs["surf"].shape[0],
                   surf=_p(arrs["surf"]), n_samples=arrs["acc"].shape[0], acc=_p(arrs["acc"]),
                   cfg=ns_config_default(**cfg), n_steps=int(n_steps))


def ns_case_bytes(wl, n_steps, **cfg_overrides):
    keep = []
    c = _case(wl, n_steps, keep, **cfg_overrides)
    dev, st, dstr = C.c_int64(), C.c_int64(), C.c_int64()
    rc = lib().ns_case_bytes(C.byref(c), C.byref(dev), C.byref(st), C.byref(dstr))
    if rc != NS_OK:
        raise NsError(rc, "invalid case")
    return dev.value, st.value, dstr.value


class Server:
    """Served ensemble: cases queued first come first served and admitted into concurrent
    slots as device / pinned-host memory allows (include/ns_server.h)."""

    def __init__(self, device=0, device_budget=None, pinned_budget=0, max_active=4, quantum_steps=16, batch=0):
        if device_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            device_budget = int(free * 0.85)
        cfg = ns_server_config(device=device, device_budget=int(device_budget), pinned_budget=int(pinned_budget),
                               max_active=int(max_active), quantum_steps=int(quantum_steps), batch=int(batch))
        h = C.c_void_p()
        rc = lib().ns_server_create(C.byref(h), C.byref(cfg))
        if rc != NS_OK:
            raise NsError(rc, "server creation failed")
        self.h = h
        self.n_surf = {}
        self.n_steps = {}

    def submit(self, wl, n_steps, **cfg_overrides):
        keep = []
        c = _case(wl, n_steps, keep, **cfg_overrides)
        i = C.c_int64()
        rc = lib().ns_server_submit(self.h, C.byref(c), C.byref(i))
        if rc != NS_OK:
            raise NsError(rc, "submission refused")
        self.n_surf[i.value] = int(wl.mesh.surf.shape[0])
        self.n_steps[i.value] = int(n_steps)
        return i.value

    def status(self, i):
        st = ns_case_stats()
        rc = lib().ns_server_status(self.h, int(i), C.byref(st))
        if rc != NS_OK:
            raise NsError(rc, "unknown case")
        return st.as_dict()

    def wait(self, i, timeout_s=3600.0):
        rc = lib().ns_server_wait(self.h, int(i), float(timeout_s))
        if rc != NS_OK:
            raise NsError(rc, "wait failed")
        return self.status(i)

    def result(self, i, fields=("u", "v", "a")):
        shape = (self.n_steps[i], self.n_surf[i], 3)
        out = {k: np.zeros(shape) for k in fields}
        rc = lib().ns_server_result(self.h, int(i), _p(out.get("u")), _p(out.get("v")), _p(out.get("a")))
        if rc != NS_OK:
            raise NsError(rc, "case %d has no result" % i)
        return out

    def release(self, i):
        rc = lib().ns_server_release(self.h, int(i))
        if rc != NS_OK:
            raise NsError(rc, "release failed")

    def close(self):
        if self.h:
            lib().ns_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
