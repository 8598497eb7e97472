"""Pins of the oracle's two-level preconditioner pieces (Sec. 2.2: EBE-IPCG with a
multigrid preconditioner after [SC14]; reading: the coarse level is the linear
tetrahedral model on the same elements).

  * coarse map: every vertex of the quadratic mesh gets one coarse index (in ascending
    fine-node order), every edge node is interpolated from its own edge's end vertices --
    checked against the node coordinates (the edge node is the midpoint of its parents);
  * Galerkin identity: for straight elements the linear-element operator equals P^T A P,
    P the linear interpolation from the vertices to all quadratic nodes, because P maps a
    linear field to its exact quadratic representation and the quadratic element
    integrals are exact for it -- checked densely for K, M, the dashpots and the full A
    with random SPD point tangents (the coarse stiffness uses their mean);
  * closed forms: the coarse mass sums to rho V per direction, the coarse stiffness
    annihilates the six rigid-body modes.
"""
import numpy as np
import pytest

import oracle
from paper_2604_02755_gb300 import synth


def model(dims, seed=3):
    m = synth.kuhn_box(*dims, 40.0, 40.0, 30.0, layer_depths=(15.0,), jitter=0.1, seed=seed)
    wl = synth.Workload("c", m, synth.two_layer_materials(0.03), 10, 0.01, 10, synth.band_limited_wave(seed, 11, 0.01))
    return wl, oracle.Oracle.from_workload(wl)


def interp(par, n_coarse):
    N = par.shape[0]
    P = np.zeros((3 * N, 3 * n_coarse))
    for n in range(N):
        for c in range(3):
            if par[n, 0] == par[n, 1]:
                P[3 * n + c, 3 * par[n, 0] + c] = 1.0
            else:
                P[3 * n + c, 3 * par[n, 0] + c] = 0.5
                P[3 * n + c, 3 * par[n, 1] + c] = 0.5
    return P


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2), (3, 2, 2)])
def test_coarse_map(dims):
    wl, _ = model(dims)
    m = wl.mesh
    cid, par, nc = oracle.coarse_map(m.conn, m.n_nodes)
    verts = np.unique(m.conn[:, :4])
    assert nc == verts.size
    assert np.array_equal(np.nonzero(cid >= 0)[0], verts) and np.array_equal(cid[verts], np.arange(nc))
    fine_of = np.zeros(nc, np.int64)
    fine_of[cid[verts]] = verts
    edge = np.nonzero(cid < 0)[0]
    assert np.all(par[edge, 0] < par[edge, 1])
    mid = 0.5 * (m.xyz[fine_of[par[edge, 0]]] + m.xyz[fine_of[par[edge, 1]]])
    assert np.allclose(m.xyz[edge], mid, rtol=0, atol=1e-12)
    assert np.array_equal(par[verts, 0], cid[verts]) and np.array_equal(par[verts, 1], cid[verts])
    # an inconsistent mesh (an edge node listed under another edge) is refused
    bad = m.conn.copy()
    bad[0, 4], bad[0, 5] = bad[0, 5], bad[0, 4]
    with pytest.raises(ValueError):
        oracle.coarse_map(bad, m.n_nodes)


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2)])
def test_coarse_operator_is_galerkin(dims):
    wl, o = model(dims)
    m = wl.mesh
    cid, par, nc = oracle.coarse_map(m.conn, m.n_nodes)
    P = interp(par, nc)
    rng = np.random.default_rng(5)
    A_ = rng.normal(size=(m.n_elems, 4, 6, 6)) * 1e7
    D = np.einsum("epij,epkj->epik", A_, A_) + 1e8 * np.eye(6)
    for which in ("K", "M", "Cb", "A"):
        n3 = 3 * m.n_nodes
        Af = np.zeros((n3, n3))
        for j in range(n3):
            e = np.zeros(n3)
            e[j] = 1.0
            Af[:, j] = o.operator(which, e, D=D).ravel()
        Ac = np.zeros((3 * nc, 3 * nc))
        for j in range(3 * nc):
            e = np.zeros(3 * nc)
            e[j] = 1.0
            Ac[:, j] = o.coarse_operator(which, e, cid, nc, D=D).ravel()
        G = P.T @ Af @ P
        assert np.abs(Ac - G).max() <= 1e-12 * np.abs(G).max(), which
        assert np.abs(Ac - Ac.T).max() <= 1e-12 * np.abs(Ac).max(), which


def test_coarse_mass_and_rigid_modes():
    wl, o = model((2, 2, 2))
    m = wl.mesh
    cid, par, nc = oracle.coarse_map(m.conn, m.n_nodes)
    fine_of = np.zeros(nc, np.int64)
    verts = np.nonzero(cid >= 0)[0]
    fine_of[cid[verts]] = verts
    X = m.xyz[fine_of]
    # total mass: 1^T M1 1 per direction = sum of rho V
    rho = np.array([mm["rho"] for mm in wl.materials])[m.mat]
    vol = np.array([oracle.p1_grads(m.xyz[m.conn[e, :4]])[1] for e in range(m.n_elems)])
    ones = np.zeros((nc, 3))
    ones[:, 0] = 1.0
    assert abs(o.coarse_operator("M", ones, cid, nc)[:, 0].sum() - (rho * vol).sum()) <= 1e-12 * (rho * vol).sum()
    # rigid-body modes: three translations and three rotations
    K1 = lambda x: o.coarse_operator("K", x, cid, nc)
    scale = np.abs(K1(np.random.default_rng(0).normal(size=(nc, 3)))).max()
    for k in range(3):
        t = np.zeros((nc, 3))
        t[:, k] = 1.0
        assert np.abs(K1(t)).max() <= 1e-9 * scale
        w = np.zeros(3)
        w[k] = 1.0
        assert np.abs(K1(np.cross(w, X))).max() <= 1e-9 * scale * np.abs(X).max()
