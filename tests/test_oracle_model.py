"""Pins of the oracle's model level: the Newmark-beta increment of Eq. 1 with
the updates below it (Sec. 2.1), the lagged tangent of Alg. 4, the block-Jacobi
PCG (Sec. 2.2) and the derived index data.

  * brute force: a dense solve of the same linear system on tiny meshes;
  * equilibrium after every step: M a^n + C^n v^n + q^n = f^n to the CG tolerance;
  * energy: undamped, unforced, linear => 1/2 v.M v + 1/2 u.K u is constant
    (the average-acceleration rule conserves it exactly);
  * the input velocity is the trapezoidal integral of the given acceleration;
  * element colouring is a valid greedy first-fit colouring.
"""
import numpy as np
import pytest
from scipy.integrate import cumulative_trapezoid

import oracle
from paper_2604_02755_gb300 import synth


def small_workload(dims=(2, 2, 2), nt=40, S=10, seed=3, linear=False, rayleigh_h=0.02, peak=3.0, dt=0.01):
    m = synth.kuhn_box(*dims, 40.0, 40.0, 30.0, layer_depths=(15.0,), jitter=0.1, seed=seed)
    mats = synth.two_layer_materials(rayleigh_h)
    if linear:
        for mm in mats:
            mm["gamma_ref"] = 1e30
    w = synth.band_limited_wave(seed, nt + 1, dt, peak=peak)
    return synth.Workload("small", m, mats, S, dt, nt, w)


def bottom_only(wl):
    m = wl.mesh
    sel = m.face_kind == 0
    return oracle.Oracle(m.xyz, m.conn, m.mat, wl.materials, m.faces[sel], m.face_elem[sel], m.face_kind[sel],
                         wl.n_springs, wl.dt, wl.wave)


def dense(o, which, D):
    n = o.n_nodes * 3
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        A[:, j] = o.operator(which, e, D=D).ravel()
    return A


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2)])
def test_pcg_matches_dense_solve(dims):
    wl = small_workload(dims=dims, nt=60)
    o = oracle.Oracle.from_workload(wl, tol=1e-13)
    ob = bottom_only(wl)
    dt = wl.dt
    for n in range(1, 4):
        D_prev = o.D.copy()
        u, v, a, q = o.u.copy(), o.v.copy(), o.a.copy(), o.q.copy()
        A = dense(o, "A", D_prev)
        assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
        vin = o.input_velocity(n)
        f = ob.operator("Cb", np.tile(vin, (o.n_nodes, 1)))
        Cv = o.operator("Cr", v, D=D_prev) + o.operator("Cb", v)
        b = f - q + Cv + o.operator("M", a + 4.0 / dt * v)
        du = np.linalg.solve(A, b.ravel()).reshape(-1, 3)
        o.step()
        assert np.abs(o.du - du).max() <= 1e-10 * np.abs(du).max()
        assert np.allclose(o.u, u + du, rtol=0, atol=1e-12 * np.abs(u + du).max())
        assert np.allclose(o.v, -v + 2.0 / dt * du, rtol=0, atol=1e-10 * np.abs(o.v).max())


def test_equilibrium_after_each_step():
    wl = small_workload(dims=(3, 3, 2), nt=80)
    o = oracle.Oracle.from_workload(wl)
    ob = bottom_only(wl)
    for n in range(1, 31):
        D_prev = o.D.copy()
        o.step()
        f = ob.operator("Cb", np.tile(o.input_velocity(n), (o.n_nodes, 1)))
        Cv = o.operator("Cr", o.v, D=D_prev) + o.operator("Cb", o.v)
        res = o.operator("M", o.a) + Cv + o.q - f
        scale = np.linalg.norm(o.operator("M", o.a)) + np.linalg.norm(f) + np.linalg.norm(o.q)
        assert np.linalg.norm(res) <= 5e-8 * scale, n
    assert (o.th["mode"] == 1).any()  # the history really was hysteretic


def test_linear_undamped_energy_conservation():
    wl = small_workload(dims=(2, 2, 2), linear=True, rayleigh_h=0.0, nt=10)
    m = wl.mesh
    o = oracle.Oracle(m.xyz, m.conn, m.mat, wl.materials, n_springs=wl.n_springs, dt=wl.dt, acc=np.zeros((1, 3)),
                      tol=1e-12)
    rng = np.random.default_rng(5)
    o.v[:] = rng.normal(size=o.v.shape) * 1e-3
    D0 = o.D.copy()

    def energy():
        return 0.5 * np.sum(o.v * o.operator("M", o.v)) + 0.5 * np.sum(o.u * o.operator("K", o.u, D=D0))

    e0 = energy()
    for _ in range(150):
        o.step()
    assert np.abs(o.D - D0).max() <= 1e-9 * np.abs(D0).max()
    assert abs(energy() - e0) <= 1e-8 * e0
    assert np.abs(o.u).max() > 1e-6  # it did move


def test_input_velocity_is_trapezoidal_integral():
    wl = small_workload(nt=100)
    o = oracle.Oracle.from_workload(wl)
    ref = cumulative_trapezoid(wl.wave, dx=wl.dt, axis=0, initial=0.0)
    for n in (0, 1, 7, 50, 100):
        assert np.allclose(o.input_velocity(n), ref[n], rtol=1e-13, atol=1e-15)
    # beyond the record the acceleration is zero
    assert np.allclose(o.input_velocity(150), ref[100] + 0.5 * wl.dt * wl.wave[100], rtol=1e-13)


def test_greedy_colouring_valid_and_first_fit():
    m = synth.kuhn_box(4, 3, 3, 40.0, 30.0, 30.0)
    col, nc = oracle.colouring(m.conn, m.n_nodes)
    assert col.max() + 1 == nc
    node_elems = {}
    for e, row in enumerate(m.conn):
        for nd in row:
            node_elems.setdefault(int(nd), []).append(e)
    for e, row in enumerate(m.conn):
        neigh = set()
        for nd in row:
            neigh.update(node_elems[int(nd)])
        neigh.discard(e)
        assert all(col[f] != col[e] for f in neigh)
        earlier = {col[f] for f in neigh if f < e}
        assert all(c in earlier for c in range(col[e]))


def test_openmp_build_is_bit_identical():
    """The OpenMP build of the oracle (its independent element, node and spring loops split
    over threads, every sum in the single-thread order) reproduces the single-thread build
    bit for bit, so timing it on all host cores times the same computation."""
    wl = small_workload(dims=(4, 3, 3), nt=40)
    out = []
    for omp in (False, True):
        if omp:
            assert oracle.threads(4) == 4
        o = oracle.Oracle.from_workload(wl, omp=omp)
        for _ in range(12):
            o.step()
        x = np.random.default_rng(1).normal(size=(o.n_nodes, 3))
        out.append((o.u.copy(), o.q.copy(), o.D.copy(), o.th.tobytes(), o.operator("A", x), o.operator("K", x)))
    for a, b in zip(*out):
        assert np.array_equal(a, b) if not isinstance(a, bytes) else a == b
    assert (o.th["mode"] == 1).any()
