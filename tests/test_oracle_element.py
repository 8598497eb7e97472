"""Pins of the oracle's element level (Sec. 2.1: quadratic tetrahedra, Eq. 2
K_e = sum_j w_j B^T D B with four points, consistent mass, dashpot faces).

Each check comes from outside the oracle: exact simplex integrals, rigid-body
modes, the constant-strain patch test, reproduction of linear fields."""
import numpy as np
import pytest

import oracle
from tests import exact_integrals as ex

RNG = np.random.default_rng(1234)


def random_tet(scale=3.0):
    while True:
        xv = RNG.normal(size=(4, 3)) * scale
        if ex.tet_volume(xv) > 0.5:
            return xv


def p2_nodes(xv):
    xv = np.asarray(xv)
    return np.vstack([xv] + [0.5 * (xv[a] + xv[b]) for a, b in ex.TET_EDGES])


def random_bary(n):
    L = RNG.random((n, 4))
    return L / L.sum(axis=1, keepdims=True)


def test_shape_partition_of_unity_and_nodal_delta():
    for L in random_bary(20):
        assert abs(oracle.shape(L).sum() - 1.0) < 1e-14
    nodes = np.vstack([np.eye(4)] + [0.5 * (np.eye(4)[a] + np.eye(4)[b]) for a, b in ex.TET_EDGES])
    for k, L in enumerate(nodes):
        N = oracle.shape(L)
        assert np.allclose(N, np.eye(10)[k], atol=1e-15)


def test_shape_reference_derivatives_by_finite_difference():
    # reference coordinates (xi, eta, zeta) = (L1, L2, L3), L0 = 1 - sum
    h = 1e-6
    for L in random_bary(5):
        dN = oracle.shape_dref(L)
        for c in range(3):
            Lp = L.copy(); Lm = L.copy()
            Lp[c + 1] += h; Lp[0] -= h
            Lm[c + 1] -= h; Lm[0] += h
            fd = (oracle.shape(Lp) - oracle.shape(Lm)) / (2 * h)
            assert np.allclose(dN[:, c], fd, atol=1e-8)


def test_gradients_reproduce_linear_fields_and_volume():
    xv = random_tet()
    X = p2_nodes(xv)
    for L in random_bary(6):
        G, det = oracle.grad(X, L)
        # grad of the coordinate field x is the identity; gradients sum to zero
        assert np.allclose(X.T @ G, np.eye(3), atol=1e-12)
        assert np.allclose(G.sum(axis=0), 0.0, atol=1e-12)
        assert abs(det / 6.0 - ex.tet_volume(xv)) < 1e-12 * abs(det)


def test_quadrature_points_degree_two_exact():
    L, w = oracle.quad_points()
    assert abs(4 * w - 1.0) < 1e-15
    # int L_j L_k dV / V = (1 + delta_jk) / 20
    for j in range(4):
        for k in range(4):
            approx = w * sum(L[q, j] * L[q, k] for q in range(4))
            assert abs(approx - (2.0 if j == k else 1.0) / 20.0) < 1e-15


def test_mass_matches_exact_integral_and_total():
    xv = random_tet()
    vol = ex.tet_volume(xv)
    rho = 1850.0
    M = oracle.element_mass(p2_nodes(xv), rho)
    Mex = ex.tet_mass_exact(vol, rho)
    assert np.allclose(M, Mex, rtol=0, atol=1e-12 * np.abs(Mex).max())
    assert abs(M.sum() - rho * vol) < 1e-12 * rho * vol
    assert np.allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    assert np.all(np.linalg.eigvalsh(M) > 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_stiffness_matches_exact_integral(seed):
    rng = np.random.default_rng(seed)
    xv = random_tet()
    A = rng.normal(size=(6, 6))
    D = A @ A.T + 6 * np.eye(6)  # any symmetric positive definite constant D
    K = oracle.element_stiffness(p2_nodes(xv), D)
    Kex = ex.tet_stiffness_exact(xv, D)
    assert np.abs(K - Kex).max() <= 1e-12 * np.abs(Kex).max()


def rigid_modes(X):
    modes = []
    for c in range(3):
        r = np.zeros((10, 3)); r[:, c] = 1.0; modes.append(r.ravel())
    for axis in np.eye(3):
        modes.append(np.cross(axis, X).ravel())
    return np.array(modes)


def test_stiffness_rigid_body_modes_and_spectrum():
    xv = random_tet()
    X = p2_nodes(xv)
    D = ex.hooke(4.0e8, 1.0e8)
    K = oracle.element_stiffness(X, D)
    for r in rigid_modes(X):
        assert np.linalg.norm(K @ r) <= 1e-12 * np.abs(K).max() * np.linalg.norm(r)
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert np.sum(np.abs(ev) < 1e-9 * ev.max()) == 6
    assert ev.min() > -1e-9 * ev.max()


def test_constant_strain_patch_test():
    """u = E x gives constant stress s = D eps; nodal forces are s . int grad N:
    zero at vertices, V s (grad L_a + grad L_b) at edge nodes."""
    xv = random_tet()
    X = p2_nodes(xv)
    E = RNG.normal(size=(3, 3))
    D = ex.hooke(3.0e8, 1.2e8)
    u = (X @ E.T).ravel()
    eps_t = 0.5 * (E + E.T)
    eps_v = np.array([eps_t[0, 0], eps_t[1, 1], eps_t[2, 2], 2 * eps_t[1, 2], 2 * eps_t[0, 2], 2 * eps_t[0, 1]])
    sv = D @ eps_v
    S = np.array([[sv[0], sv[5], sv[4]], [sv[5], sv[1], sv[3]], [sv[4], sv[3], sv[2]]])
    f = (oracle.element_stiffness(X, D) @ u).reshape(10, 3)
    gL = ex.bary_gradients(xv)
    vol = ex.tet_volume(xv)
    expect = np.zeros((10, 3))
    for k, (a, b) in enumerate(ex.TET_EDGES):
        expect[4 + k] = vol * S @ (gL[a] + gL[b])
    assert np.abs(f - expect).max() <= 1e-10 * np.abs(expect).max()


def test_face_dashpot_exact_and_directions():
    fx = np.array([[0.0, 0.0, 0.0], [4.0, 0.5, 0.0], [1.0, 3.0, 0.0]])
    area = 0.5 * np.linalg.norm(np.cross(fx[1] - fx[0], fx[2] - fx[0]))
    rho, vs, vp = 2000.0, 600.0, 1470.0
    Cm = oracle.face_dashpot(fx, rho, vs, vp)
    Mf = ex.tri_mass_exact(area)
    assert abs(Mf.sum() - area) < 1e-13 * area
    # normal is z: xx, yy blocks damp with rho Vs, zz with rho Vp, no coupling
    for r, c, val in ((0, 0, rho * vs), (1, 1, rho * vs), (2, 2, rho * vp), (0, 1, 0.0), (0, 2, 0.0), (1, 2, 0.0)):
        blk = Cm[r::3, c::3]
        assert np.allclose(blk, Mf * val, atol=1e-9 * rho * vp * area)
    # rotated face: the dashpot is rho [Vs I + (Vp - Vs) n n^T] for any orientation
    Q, _ = np.linalg.qr(RNG.normal(size=(3, 3)))
    fr = fx @ Q.T
    Cr = oracle.face_dashpot(fr, rho, vs, vp)
    n = Q @ np.array([0.0, 0.0, 1.0])
    T = rho * (vs * np.eye(3) + (vp - vs) * np.outer(n, n))
    assert np.allclose(Cr, np.kron(Mf, T), atol=1e-9 * rho * vp * area)
