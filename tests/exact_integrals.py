"""Exact integrals of polynomials in barycentric coordinates, used to pin the
oracle's quadrature-based element matrices by an independent route.

Identities used (standard results of simplex integration):
  tetrahedron of volume V:  int L0^a L1^b L2^c L3^d dV = 6 V a! b! c! d! / (a+b+c+d+3)!
  triangle of area A:       int l0^a l1^b l2^c dA     = 2 A a! b! c! / (a+b+c+2)!
Polynomials are dicts {exponent tuple: coefficient}; shape functions are
written homogeneously using sum(L) = 1.
"""
from math import factorial

import numpy as np

TET_EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))
TRI_EDGES = ((0, 1), (1, 2), (0, 2))


def _mono(n, **pw):
    e = [0] * n
    for k, v in pw.items():
        e[int(k[1:])] += v
    return tuple(e)


def pmul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0.0) + ca * cb
    return out


def padd(p, q, s=1.0):
    out = dict(p)
    for e, c in q.items():
        out[e] = out.get(e, 0.0) + s * c
    return out


def lin(n, i):
    e = [0] * n
    e[i] = 1
    return {tuple(e): 1.0}


def const(n, c):
    return {tuple([0] * n): c}


def quad_shape(n, edges):
    """Quadratic Lagrange shape functions on an n-vertex simplex, homogeneous of degree 2."""
    one = {}
    for i in range(n):
        one = padd(one, lin(n, i))
    N = []
    for i in range(n):
        N.append(pmul(lin(n, i), padd(pmul(const(n, 2.0), lin(n, i)), one, -1.0)))  # L_i (2 L_i - sum L)
    for a, b in edges:
        N.append(pmul(const(n, 4.0), pmul(lin(n, a), lin(n, b))))
    return N


def integrate_tet(p, vol):
    s = 0.0
    for e, c in p.items():
        s += c * 6.0 * vol * np.prod([factorial(k) for k in e]) / factorial(sum(e) + 3)
    return s


def integrate_tri(p, area):
    s = 0.0
    for e, c in p.items():
        s += c * 2.0 * area * np.prod([factorial(k) for k in e]) / factorial(sum(e) + 2)
    return s


def tet_mass_exact(vol, rho=1.0):
    N = quad_shape(4, TET_EDGES)
    return np.array([[rho * integrate_tet(pmul(N[a], N[b]), vol) for b in range(10)] for a in range(10)])


def tri_mass_exact(area):
    N = quad_shape(3, TRI_EDGES)
    return np.array([[integrate_tri(pmul(N[a], N[b]), area) for b in range(6)] for a in range(6)])


def bary_gradients(xv):
    """Gradients of the four barycentric coordinates of a straight tetrahedron
    (rows), from L = A^{-1} [1; x]."""
    A = np.vstack([np.ones(4), np.asarray(xv, np.float64).T])
    Ainv = np.linalg.inv(A)
    return Ainv[:, 1:]


def tet_volume(xv):
    xv = np.asarray(xv, np.float64)
    return np.linalg.det(np.stack([xv[1] - xv[0], xv[2] - xv[0], xv[3] - xv[0]])) / 6.0


def shape_gradient_linear_parts(xv):
    """Physical gradient of each quadratic shape function written as
    sum_j c[a, j, :] L_j (homogeneous linear in L).  Returns c [10, 4, 3]."""
    gL = bary_gradients(xv)
    c = np.zeros((10, 4, 3))
    for i in range(4):
        # d/dx [L_i (2 L_i - sum_k L_k)] with sum_k L_k = 1 identically -> (4 L_i - 1) gL_i
        # = 4 L_i gL_i - (sum_j L_j) gL_i
        for j in range(4):
            c[i, j] -= gL[i]
        c[i, i] += 4.0 * gL[i]
    for k, (a, b) in enumerate(TET_EDGES):
        c[4 + k, a] += 4.0 * gL[b]
        c[4 + k, b] += 4.0 * gL[a]
    return c


def bmatrix_from_grad(g):
    """6x30 strain-displacement matrix from 10 gradient vectors (xx yy zz yz xz xy)."""
    B = np.zeros((6, 30))
    for i in range(10):
        d = g[i]
        B[0, 3 * i] = d[0]; B[1, 3 * i + 1] = d[1]; B[2, 3 * i + 2] = d[2]
        B[3, 3 * i + 1] = d[2]; B[3, 3 * i + 2] = d[1]
        B[4, 3 * i] = d[2]; B[4, 3 * i + 2] = d[0]
        B[5, 3 * i] = d[1]; B[5, 3 * i + 1] = d[0]
    return B


def tet_stiffness_exact(xv, D):
    """int B^T D B dV for constant D: B = sum_j B_j L_j, int L_j L_k = V (1 + delta_jk) / 20."""
    vol = tet_volume(xv)
    c = shape_gradient_linear_parts(xv)
    Bj = [bmatrix_from_grad(c[:, j, :]) for j in range(4)]
    K = np.zeros((30, 30))
    for j in range(4):
        for k in range(4):
            K += Bj[j].T @ D @ Bj[k] * vol * (2.0 if j == k else 1.0) / 20.0
    return K


def hooke(lam, mu):
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(6), np.arange(6)] += np.array([2 * mu, 2 * mu, 2 * mu, mu, mu, mu])
    return D
