"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 2.3).

This module holds input preparation only -- meshes, boundary face lists,
surface node lists, material parameter tables and input waves.  It contains
none of the finite-element method's arithmetic (no shape functions, element
matrices, solver or constitutive law), so both the CUDA library and the CPU
oracle may take their inputs from it.

Mesh: a box split into hexahedra, each hexahedron split into six tetrahedra
along its (0,0,0)-(1,1,1) diagonal (Kuhn split), with a mid-edge node on every
tetrahedron edge (10-node quadratic tetrahedra, Sec. 2.1).  Because every Kuhn
edge joins two grid points whose indices differ by 0 or +1 per axis, the
quadratic node set is exactly the grid of half spacing, so node ids are
lexicographic indices of that doubled grid (x fastest).

Local node order of a tetrahedron: vertices 0-3, then edge nodes on the edges
(0,1), (1,2), (0,2), (0,3), (1,3), (2,3).  Vertex order is chosen so that the
signed volume det[x1-x0, x2-x0, x3-x0] / 6 is positive.

Boundary faces (Sec. 2.1: absorbing bottom and sides): six-node triangles,
vertices (f0, f1, f2) then edge nodes (f0,f1), (f1,f2), (f0,f2); kind 0 = bottom
(z = 0), kind 1 = side (x or y extreme).  The top surface z = Lz is traction
free and carries no face.

Random numbers: splitmix64 (Steele, Lea, Flood 2014), used counter-style: the
k-th draw (k = 1, 2, ...) of stream s under seed q is mix(q ^ (s * C) + k * G)
with G = 0x9E3779B97F4A7C15 and mix the splitmix64 output function.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM = np.uint64(0xD1B54A32D192ED03)

# edge (local vertex pair) -> local node index, for the order documented above
TET_EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))


def splitmix64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """Draws 1..n of splitmix64 stream `stream` under `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        s0 = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream) * _STREAM)
        z = s0 + (np.arange(1, n + 1, dtype=np.uint64) * _G)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(seed, n, stream) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n standard normal doubles by the Box-Muller transform of two uniform streams."""
    u1 = uniform01(seed, n, 2 * stream + 1)
    u2 = uniform01(seed, n, 2 * stream + 2)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------- materials

def soil(rho: float, vs: float, gamma_ref: float, h_max: float = 0.20, rayleigh_h: float = 0.02,
         poisson: float = 0.40) -> dict:
    """One material row: density, S and P wave speeds, spring reference strain,
    maximum hysteretic damping and Rayleigh damping ratio.  Vp follows from a
    Poisson ratio (0.40 gives Vp = sqrt(6) Vs)."""
    vp = vs * math.sqrt(2.0 * (1.0 - poisson) / (1.0 - 2.0 * poisson))
    return dict(rho=float(rho), vs=float(vs), vp=float(vp), gamma_ref=float(gamma_ref),
                h_max=float(h_max), rayleigh_h=float(rayleigh_h))


def two_layer_materials(rayleigh_h: float = 0.02) -> list:
    """Soft soil (Vs 150 m/s, rho 1700) over bedrock (Vs 600 m/s, rho 2000)."""
    return [soil(1700.0, 150.0, 5e-4, 0.20, rayleigh_h), soil(2000.0, 600.0, 1e-2, 0.20, rayleigh_h)]


def three_layer_materials(rayleigh_h: float = 0.02) -> list:
    """0-20 m Vs 150 / rho 1700, 20-60 m Vs 300 / rho 1850, bedrock Vs 600 / rho 2000."""
    return [soil(1700.0, 150.0, 5e-4, 0.20, rayleigh_h), soil(1850.0, 300.0, 7e-4, 0.20, rayleigh_h),
            soil(2000.0, 600.0, 1e-2, 0.20, rayleigh_h)]


# ----------------------------------------------------------------------------- mesh

@dataclass
class Mesh:
    xyz: np.ndarray          # [N,3] float64 node coordinates
    conn: np.ndarray         # [E,10] int32 element nodes (order in module docstring)
    mat: np.ndarray          # [E] int32 material index
    faces: np.ndarray        # [F,6] int32 boundary face nodes
    face_elem: np.ndarray    # [F] int32 element owning the face
    face_kind: np.ndarray    # [F] int32 0 bottom, 1 side
    surf: np.ndarray         # [Ns] int32 top-surface nodes
    dims: tuple = ()         # (nx, ny, nz) hexahedra
    size: tuple = ()         # (Lx, Ly, Lz) metres
    info: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.conn.shape[0])


_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
_PERM_SIGN = (1, -1, -1, 1, 1, -1)


def _kuhn_corners():
    """Corner offsets (4 x 3, in hexahedron units) of the six Kuhn tetrahedra,
    ordered to have positive orientation."""
    out = []
    for perm, sgn in zip(_PERMS, _PERM_SIGN):
        a, b, _ = perm
        c0 = np.zeros(3, dtype=np.int64)
        c1 = c0.copy(); c1[a] = 1
        c2 = c1.copy(); c2[b] = 1
        c3 = np.ones(3, dtype=np.int64)
        if sgn < 0:
            c1, c2 = c2, c1
        out.append(np.stack([c0, c1, c2, c3]))
    return np.stack(out)  # [6,4,3]


def smooth_field(seed: int, x: np.ndarray, y: np.ndarray, lx: float, ly: float, lo: float, hi: float,
                 modes: int = 4) -> np.ndarray:
    """Seeded smooth random field on [0,lx]x[0,ly]: a sum of a few low cosine modes
    with normal amplitudes, affinely mapped so its range over the box is [lo, hi]
    (exact range estimated on a 65x65 grid, then clipped)."""
    amp = normal(seed, modes * modes, stream=7).reshape(modes, modes)
    ph = uniform01(seed, 2 * modes * modes, stream=8).reshape(2, modes, modes) * 2.0 * np.pi

    def raw(xx, yy):
        f = np.zeros_like(xx, dtype=np.float64)
        for i in range(modes):
            for j in range(modes):
                if i == 0 and j == 0:
                    continue
                f += amp[i, j] / (1.0 + i * i + j * j) * np.cos(np.pi * i * xx / lx + ph[0, i, j]) * \
                    np.cos(np.pi * j * yy / ly + ph[1, i, j])
        return f

    gx, gy = np.meshgrid(np.linspace(0, lx, 65), np.linspace(0, ly, 65))
    g = raw(gx, gy)
    fmin, fmax = float(g.min()), float(g.max())
    f = raw(np.asarray(x, np.float64), np.asarray(y, np.float64))
    return np.clip(lo + (f - fmin) * (hi - lo) / max(fmax - fmin, 1e-300), lo, hi)


def kuhn_box(nx: int, ny: int, nz: int, lx: float, ly: float, lz: float, layer_depths=(),
             jitter: float = 0.0, seed: int = 0, x0: float = 0.0, y0: float = 0.0,
             domain: tuple | None = None) -> Mesh:
    """Structured box of nx*ny*nz hexahedra, six quadratic tetrahedra each.

    layer_depths: interfaces, depth below the top surface (metres), shallowest
      first; each entry is a float or a callable (x, y) -> depth.  Element
      material = number of interfaces shallower than its centroid.
    jitter: vertex perturbation as a fraction of the local hexahedron size
      (uniform in [-jitter, jitter] per axis; none across the boundary planes);
      mid-edge nodes stay at edge midpoints.
    x0, y0, domain: place this box at offset (x0, y0) inside a larger domain
      (Lx, Ly) -- used to cut a column out of a bigger model; the boundary
      planes are this box's own.
    """
    hx, hy, hz = lx / nx, ly / ny, lz / nz
    NX, NY, NZ = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    I, J, K = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    I = I.transpose(2, 1, 0).ravel(); J = J.transpose(2, 1, 0).ravel(); K = K.transpose(2, 1, 0).ravel()
    nn = NX * NY * NZ
    # vertex (even, even, even) positions, jittered
    xs = x0 + 0.5 * hx * I.astype(np.float64)
    ys = y0 + 0.5 * hy * J.astype(np.float64)
    zs = 0.5 * hz * K.astype(np.float64)
    xyz = np.stack([xs, ys, zs], axis=1)
    if jitter > 0.0:
        d = (uniform01(seed, 3 * nn, stream=3).reshape(nn, 3) * 2.0 - 1.0) * jitter * np.array([hx, hy, hz])
        d[(I == 0) | (I == NX - 1), 0] = 0.0
        d[(J == 0) | (J == NY - 1), 1] = 0.0
        d[(K == 0) | (K == NZ - 1), 2] = 0.0
        even = (I % 2 == 0) & (J % 2 == 0) & (K % 2 == 0)
        xyz[even] += d[even]
    # odd points: midpoint of the Kuhn edge through them (parity decides the endpoints)
    oi, oj, ok = I % 2, J % 2, K % 2
    odd = (oi + oj + ok) > 0
    lo_id = (I - oi) + NX * ((J - oj) + NY * (K - ok))
    hi_id = (I + oi) + NX * ((J + oj) + NY * (K + ok))
    xyz[odd] = 0.5 * (xyz[lo_id[odd]] + xyz[hi_id[odd]])

    corners = _kuhn_corners()  # [6,4,3]
    hi_, hj_, hk_ = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hi_ = hi_.transpose(2, 1, 0).ravel(); hj_ = hj_.transpose(2, 1, 0).ravel(); hk_ = hk_.transpose(2, 1, 0).ravel()
    nh = nx * ny * nz
    base = np.stack([hi_, hj_, hk_], axis=1)  # [nh,3]
    vd = 2 * (base[:, None, None, :] + corners[None, :, :, :])  # [nh,6,4,3] doubled coords of vertices
    vd = vd.reshape(nh * 6, 4, 3)
    ed = np.stack([(vd[:, a] + vd[:, b]) // 2 for a, b in TET_EDGES], axis=1)  # [E,6,3]
    allp = np.concatenate([vd, ed], axis=1)  # [E,10,3]
    conn = (allp[..., 0] + NX * (allp[..., 1] + NY * allp[..., 2])).astype(np.int32)

    # materials by centroid depth
    xc = xyz[conn[:, :4], :].mean(axis=1)
    depth = lz - xc[:, 2]
    mat = np.zeros(conn.shape[0], dtype=np.int32)
    for d in layer_depths:
        dd = d(xc[:, 0], xc[:, 1]) if callable(d) else np.full(conn.shape[0], float(d))
        mat += (depth > dd).astype(np.int32)

    # boundary faces: local face opposite vertex o
    face_local = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))
    edge_index = {e: 4 + i for i, e in enumerate(TET_EDGES)}
    f_nodes, f_elem, f_kind = [], [], []
    for tri in face_local:
        v = vd[:, tri, :]  # [E,3,3]
        bottom = np.all(v[:, :, 2] == 0, axis=1)
        side = (np.all(v[:, :, 0] == 0, axis=1) | np.all(v[:, :, 0] == NX - 1, axis=1) |
                np.all(v[:, :, 1] == 0, axis=1) | np.all(v[:, :, 1] == NY - 1, axis=1))
        sel = np.nonzero(bottom | side)[0]
        a, b, c = tri
        cols = [a, b, c, edge_index[tuple(sorted((a, b)))], edge_index[tuple(sorted((b, c)))],
                edge_index[tuple(sorted((a, c)))]]
        f_nodes.append(conn[sel][:, cols])
        f_elem.append(sel.astype(np.int32))
        f_kind.append(np.where(bottom[sel], 0, 1).astype(np.int32))
    f_elem = np.concatenate(f_elem)
    order = np.argsort(f_elem, kind="stable")
    faces = np.concatenate(f_nodes)[order].astype(np.int32)
    face_kind = np.concatenate(f_kind)[order]
    f_elem = f_elem[order]

    sI, sJ = np.meshgrid(np.arange(NX), np.arange(NY), indexing="ij")
    surf = (sI.T.ravel() + NX * (sJ.T.ravel() + NY * (NZ - 1))).astype(np.int32)

    m = Mesh(xyz=xyz, conn=np.ascontiguousarray(conn), mat=mat, faces=np.ascontiguousarray(faces),
             face_elem=f_elem, face_kind=face_kind, surf=surf, dims=(nx, ny, nz), size=(lx, ly, lz),
             info=dict(jitter=jitter, seed=seed, x0=x0, y0=y0))
    # orientation check (input sanity, not method arithmetic)
    e = xyz[conn[:, :4]]
    det = np.einsum("ij,ij->i", np.cross(e[:, 1] - e[:, 0], e[:, 2] - e[:, 0]), e[:, 3] - e[:, 0])
    if not np.all(det > 0):
        raise ValueError("generated mesh has non-positive tetrahedra")
    return m


def _spread3(v: np.ndarray) -> np.ndarray:
    """Spread the low 21 bits of v so that bit b lands on bit 3b (Morton interleave)."""
    x = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    for shift, mask in ((32, 0x1F00000000FFFF), (16, 0x1F0000FF0000FF), (8, 0x100F00F00F00F00F),
                        (4, 0x10C30C30C30C30C3), (2, 0x1249249249249249)):
        x = (x | (x << np.uint64(shift))) & np.uint64(mask)
    return x


def morton_keys(p: np.ndarray) -> np.ndarray:
    """Z-order keys of points p [n,3]: coordinates scaled to 21-bit integers over the
    bounding box, bits interleaved x, y, z."""
    lo, hi = p.min(axis=0), p.max(axis=0)
    q = np.floor((p - lo) / np.maximum(hi - lo, 1e-300) * float((1 << 21) - 1)).astype(np.int64)
    return _spread3(q[:, 0]) | (_spread3(q[:, 1]) << np.uint64(1)) | (_spread3(q[:, 2]) << np.uint64(2))


def renumber(mesh: Mesh, how: str = "morton", seed: int = 0) -> Mesh:
    """The same mesh with elements and nodes renumbered.

    how: "grid" (unchanged: the generator's lexicographic order), "morton" (elements by
    the Z-order key of their centroids, nodes by that of their positions) or "shuffled"
    (seeded random permutations of both -- the worst case for the operator's gathers).
    The surface node list keeps its order (so surface records line up), faces stay sorted
    by their owning element."""
    if how == "grid":
        return mesh
    E, N = mesh.n_elems, mesh.n_nodes
    if how == "morton":
        pe = np.argsort(morton_keys(mesh.xyz[mesh.conn[:, :4]].mean(axis=1)), kind="stable")
        pn = np.argsort(morton_keys(mesh.xyz), kind="stable")
    elif how == "shuffled":
        pe = np.argsort(splitmix64(seed, E, stream=7), kind="stable")
        pn = np.argsort(splitmix64(seed, N, stream=8), kind="stable")
    else:
        raise ValueError(f"unknown numbering {how!r}")
    inv_e = np.empty(E, dtype=np.int64)
    inv_e[pe] = np.arange(E)
    inv_n = np.empty(N, dtype=np.int64)
    inv_n[pn] = np.arange(N)
    fe = inv_e[mesh.face_elem]
    fo = np.argsort(fe, kind="stable")
    return Mesh(xyz=np.ascontiguousarray(mesh.xyz[pn]), conn=np.ascontiguousarray(inv_n[mesh.conn[pe]].astype(np.int32)),
                mat=np.ascontiguousarray(mesh.mat[pe]), faces=np.ascontiguousarray(inv_n[mesh.faces[fo]].astype(np.int32)),
                face_elem=np.ascontiguousarray(fe[fo].astype(np.int32)), face_kind=np.ascontiguousarray(mesh.face_kind[fo]),
                surf=inv_n[mesh.surf].astype(np.int32), dims=mesh.dims, size=mesh.size,
                info=dict(mesh.info, numbering=how))


# ----------------------------------------------------------------------------- input waves

def band_limited_wave(seed: int, nt: int, dt: float, f_lo: float = 0.1, f_hi: float = 2.5,
                      peak: float = 3.0, taper: float = 0.1, components: int = 3, taper_s: float = None) -> np.ndarray:
    """Seeded Gaussian acceleration [nt, components]: N(0,1) samples, band-passed
    by zeroing DFT bins outside [f_lo, f_hi], cosine-tapered over the first and
    last `taper` fraction (or, with taper_s, the first and last taper_s seconds),
    then scaled so each component's peak |a| = `peak`."""
    out = np.zeros((nt, components))
    f = np.fft.rfftfreq(nt, dt)
    keep = (f >= f_lo) & (f <= f_hi)
    nta = max(1, int(round(taper_s / dt if taper_s is not None else taper * nt)))
    w = np.ones(nt)
    ramp = 0.5 - 0.5 * np.cos(np.pi * np.arange(nta) / nta)
    w[:nta] = ramp
    w[nt - nta:] = np.minimum(w[nt - nta:], ramp[::-1])
    for c in range(components):
        z = normal(seed, nt, stream=16 + c)
        Z = np.fft.rfft(z)
        Z[~keep] = 0.0
        a = np.fft.irfft(Z, n=nt) * w
        pk = np.max(np.abs(a))
        out[:, c] = a * (peak / pk if pk > 0 else 0.0)
    return out


# ----------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    mesh: Mesh
    materials: list
    n_springs: int
    dt: float
    n_steps: int
    wave: np.ndarray  # [n_steps + 1, 3] outcrop acceleration samples at t = k dt


def tiny_two_layer(nt: int = 300, seed: int = 1, n_springs: int = 10, dims=(10, 10, 6)) -> Workload:
    """Plain FP64 tiny case: 200x200x60 m, two layers (interface 30 m deep),
    10x10x6 hexahedra -> 3,600 quadratic tetrahedra, 10 springs per point,
    dt = 0.01 s, 300 steps, 0.1-2.5 Hz Gaussian input scaled to 3 m/s^2."""
    nx, ny, nz = dims
    m = kuhn_box(nx, ny, nz, 200.0, 200.0, 60.0, layer_depths=(30.0,), jitter=0.0, seed=seed)
    w = band_limited_wave(seed, nt + 1, 0.01)
    return Workload("tiny two-layer 200x200x60 m, 10x10x6 hex -> 3600 P2 tets, 10 springs", m,
                    two_layer_materials(0.02), n_springs, 0.01, nt, w)


def large_interface_field(seed: int, lx: float = 800.0, ly: float = 800.0):
    """Random soft-layer bottom depth (20-60 m) of the large single model."""
    return lambda x, y: smooth_field(seed, x, y, lx, ly, 20.0, 60.0)


def large_single_model(nt: int = 2000, seed: int = 2, n_springs: int = 150, dims=(160, 160, 52),
                       column=None) -> Workload:
    """Single large model: 800x800x260 m at 5 m hexahedra (160x160x52 -> 7,987,200
    quadratic tetrahedra, 10,819,305 nodes), soft layer over bedrock with a seeded
    random interface 20-60 m deep, vertices jittered by up to 10% of h,
    150 springs per point, dt = 0.005 s.

    column=(i0, j0, ni, nj) cuts an ni x nj hexahedron column out of the same
    model (same spacing, interface and materials) -- a bounded sample of it."""
    nx, ny, nz = dims
    h = 800.0 / 160.0
    lx, ly, lz = nx * h, ny * h, nz * h
    iface = large_interface_field(seed)
    if column is None:
        m = kuhn_box(nx, ny, nz, lx, ly, lz, layer_depths=(iface,), jitter=0.1, seed=seed)
    else:
        i0, j0, ni, nj = column
        m = kuhn_box(ni, nj, nz, ni * h, nj * h, lz, layer_depths=(iface,), jitter=0.1, seed=seed,
                     x0=i0 * h, y0=j0 * h)
    w = band_limited_wave(seed, nt + 1, 0.005)
    return Workload("single large model 800x800x260 m, 5 m hex, 150 springs", m, two_layer_materials(0.02),
                    n_springs, 0.005, nt, w)


def main_motion_record(seed: int = 2, nt: int = 2000, dt: float = 0.005, taper_s: float = 0.2) -> np.ndarray:
    """Full-length input record of the large model (2000 steps of 0.005 s) whose strong
    part starts early: the same seeded band-limited Gaussian, tapered over 0.2 s at each
    end instead of a tenth of the record."""
    return band_limited_wave(seed, nt + 1, dt, taper_s=taper_s)


def lead_in_steps(dt: float, lz: float = 260.0, depth_max: float = 60.0, vs_soft: float = 150.0,
                  vs_rock: float = 600.0, taper_s: float = 0.2) -> int:
    """Steps until the input's S waves, past the taper, have crossed the bedrock and the
    deepest soft layer and reached the surface: (taper + (lz - d)/Vs_rock + d/Vs_soft) / dt
    with d the largest interface depth.  A timed window after this many steps sits in the
    strong motion of the soft layer, not in the quiet lead-in."""
    return int(math.ceil((taper_s + (lz - depth_max) / vs_rock + depth_max / vs_soft) / dt))


def precision_form_model(nt: int = 3000, seed: int = 4, n_springs: int = 50, dims=(64, 64, 41),
                         column=None) -> Workload:
    """Precision-form model: 320x320x205 m at 5 m hexahedra (64x64x41 -> 1,007,616
    quadratic tetrahedra, 1,381,203 nodes), three layers (0-20 m Vs 150, 20-60 m Vs 300,
    bedrock Vs 600), vertices jittered by up to 10% of h, 50 springs per point,
    dt = 0.005 s.  column=(i0, j0, ni, nj) cuts an ni x nj hexahedron column out of it."""
    nx, ny, nz = dims
    h = 5.0
    lz = nz * h
    if column is None:
        m = kuhn_box(nx, ny, nz, nx * h, ny * h, lz, layer_depths=(20.0, 60.0), jitter=0.1, seed=seed)
    else:
        i0, j0, ni, nj = column
        m = kuhn_box(ni, nj, nz, ni * h, nj * h, lz, layer_depths=(20.0, 60.0), jitter=0.1, seed=seed,
                     x0=i0 * h, y0=j0 * h)
    w = band_limited_wave(seed, nt + 1, 0.005)
    return Workload("precision-form model 320x320x205 m, 5 m hex, three layers, 50 springs", m,
                    three_layer_materials(0.02), n_springs, 0.005, nt, w)


@dataclass
class Ensemble:
    """Members sharing one mesh: member m has its own materials (same layering) and input."""
    name: str
    mesh: Mesh
    members: list            # [M] lists of material rows
    waves: list              # [M] arrays [n_steps + 1, 3]
    n_springs: int
    dt: float
    n_steps: int

    def member(self, m: int) -> Workload:
        return Workload("%s, member %d" % (self.name, m), self.mesh, self.members[m], self.n_springs, self.dt,
                        self.n_steps, self.waves[m])


def ensemble_members(M: int = 64, nt: int = 4000, seed: int = 3, n_springs: int = 50, dims=(40, 40, 21),
                     h: float = 4.0, interface_depth: float = 40.0) -> Ensemble:
    """Batched ensemble: M members on one shared mesh -- 160x160x84 m at 4 m hexahedra
    (40x40x21 -> 201,600 quadratic tetrahedra, 282,123 nodes), soil over bedrock with a
    planar interface 40 m deep, vertices jittered by up to 10% of h, 50 springs per point,
    dt = 0.005 s.  Per member (seeded): soil Vs ~ U(100, 300) m/s, reference strain
    ~ logU(1e-4, 1e-3), damping ratio ~ U(1, 5)% (Rayleigh, both layers), and an
    independent band-limited input wave."""
    nx, ny, nz = dims
    m = kuhn_box(nx, ny, nz, nx * h, ny * h, nz * h, layer_depths=(interface_depth,), jitter=0.1, seed=seed)
    u = uniform01(seed, 3 * M, stream=40).reshape(3, M)
    vs = 100.0 + 200.0 * u[0]
    gref = 10.0 ** (-4.0 + u[1])
    hr = 0.01 + 0.04 * u[2]
    members = [[soil(1700.0, float(vs[k]), float(gref[k]), 0.20, float(hr[k])),
                soil(2000.0, 600.0, 1e-2, 0.20, float(hr[k]))] for k in range(M)]
    waves = [band_limited_wave(seed * 1000 + 17 + k, nt + 1, 0.005) for k in range(M)]
    return Ensemble("batched ensemble, %d members on 160x160x84 m at 4 m, 50 springs" % M, m, members, waves,
                    n_springs, 0.005, nt)


@dataclass
class Union:
    mesh: Mesh
    elem_off: np.ndarray  # [M + 1]
    node_off: np.ndarray  # [M + 1]


def union_of_copies(mesh: Mesh, M: int, n_materials: int) -> Union:
    """Disjoint union of M copies of a mesh (copy m: nodes shifted by m * N, elements by
    m * E, material ids by m * n_materials, faces and surface nodes in copy order)."""
    N, E, F = mesh.n_nodes, mesh.n_elems, mesh.faces.shape[0]
    k = np.arange(M)
    xyz = np.tile(mesh.xyz, (M, 1))
    conn = (mesh.conn[None, :, :] + (k * N)[:, None, None]).reshape(M * E, 10).astype(np.int32)
    mat = (mesh.mat[None, :] + (k * n_materials)[:, None]).reshape(-1).astype(np.int32)
    faces = (mesh.faces[None, :, :] + (k * N)[:, None, None]).reshape(M * F, 6).astype(np.int32)
    face_elem = (mesh.face_elem[None, :] + (k * E)[:, None]).reshape(-1).astype(np.int32)
    face_kind = np.tile(mesh.face_kind, M).astype(np.int32)
    surf = (mesh.surf[None, :] + (k * N)[:, None]).reshape(-1).astype(np.int32)
    u = Mesh(xyz=xyz, conn=conn, mat=mat, faces=faces, face_elem=face_elem, face_kind=face_kind, surf=surf,
             dims=mesh.dims)
    return Union(u, np.arange(M + 1, dtype=np.int64) * E, np.arange(M + 1, dtype=np.int64) * N)


@dataclass
class Request:
    arrival_s: float
    workload: Workload
    n_steps: int


def served_trace(R: int = 12, rate_per_s: float = 4.0, seed: int = 5, step_scale: float = 0.01,
                 e_lo: float = 5e4, e_hi: float = 2e6, nz: int = 21, h: float = 4.0) -> list:
    """Served ensemble: R requests with Poisson arrivals (rate_per_s), meshes of
    log-uniform size in [e_lo, e_hi] elements (nx = ny hexahedra of h metres, nz deep,
    soil over bedrock at 40 m, jitter 10%), springs ~ U{20..150}, steps ~ U[1000, 4000]
    times step_scale, soil Vs ~ U(100, 300) m/s, reference strain ~ logU(1e-4, 1e-3),
    damping ~ U(1, 5)%, independent input waves, dt 0.005 s."""
    u = uniform01(seed, 8 * R, stream=60).reshape(8, R)
    t = np.cumsum(-np.log1p(-u[0]) / rate_per_s)
    out = []
    for k in range(R):
        E = math.exp(math.log(e_lo) + (math.log(e_hi) - math.log(e_lo)) * u[1, k])
        n = max(2, int(round(math.sqrt(E / (6.0 * nz)))))
        S = 20 + int(u[2, k] * 131) if u[2, k] < 1.0 else 150
        steps = max(1, int(round((1000 + 3000 * u[3, k]) * step_scale)))
        vs = 100.0 + 200.0 * u[4, k]
        gref = 10.0 ** (-4.0 + u[5, k])
        hr = 0.01 + 0.04 * u[6, k]
        m = kuhn_box(n, n, nz, n * h, n * h, nz * h, layer_depths=(40.0,), jitter=0.1, seed=seed * 100 + k)
        mats = [soil(1700.0, vs, gref, 0.20, hr), soil(2000.0, 600.0, 1e-2, 0.20, hr)]
        w = band_limited_wave(seed * 1000 + k, max(steps + 1, 400), 0.005)
        wl = Workload("request %d: %dx%dx%d hexahedra, %d springs" % (k, n, n, nz, S), m, mats, S, 0.005, steps, w)
        out.append(Request(float(t[k]), wl, steps))
    return out
