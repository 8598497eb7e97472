"""Pins of the oracle's 1D spring law (Sec. 2.1: modified Ramberg-Osgood skeleton
with the Masing rule; 40 bytes of state per spring) and of the multi-spring
point (D from many 1D springs).

Closed forms and invariants used:
  * the reference strain is where the secant modulus is G0/2;
  * the tangent tends to G0 at vanishing strain;
  * a Masing branch leaving the skeleton at gamma_a reaches (-gamma_a, -tau_a),
    and a full cycle closes;
  * loop damping of RO + Masing: h = (2/pi) beta/(beta+2) (1 - G_sec/G0);
  * with every spring at G0 the multi-spring D is isotropic Hooke.
"""
import math

import numpy as np
import pytest

import oracle
from tests import exact_integrals as ex


def soft():
    return oracle.ro_params(1700.0, 150.0, 5e-4, 0.20)


def fresh():
    return np.zeros(1, oracle.SPRING_DTYPE)


def test_state_is_forty_bytes():
    assert oracle.SPRING_DTYPE.itemsize == 40


def test_parameters():
    p = soft()
    assert abs(p.G0 - 1700.0 * 150.0 ** 2) < 1e-6
    beta = 2 * math.pi * 0.2 / (2 - math.pi * 0.2)
    assert abs(p.beta - beta) < 1e-15 and abs(p.alpha - 2 ** beta) < 1e-14


@pytest.mark.parametrize("ratio", [1e-6, 1e-3, 0.1, 1.0, 3.0, 30.0, 1e3])
def test_skeleton_inverse(ratio):
    p = soft()
    g = ratio * p.gref
    tau = oracle.ro_F(g, p)
    assert abs(oracle.ro_g(tau, p) - g) <= 1e-13 * g
    assert oracle.ro_F(-g, p) == -tau
    assert 0 < tau <= p.G0 * g


def test_secant_half_at_reference_strain():
    p = soft()
    tau = oracle.ro_F(p.gref, p)
    assert abs(tau / p.gref / p.G0 - 0.5) < 1e-13


def test_tangent_tends_to_G0_and_decreases():
    p = soft()
    assert abs(1.0 / oracle.ro_dg(0.0, p) - p.G0) < 1e-6
    prev = p.G0 * (1 + 1e-12)
    for r in np.logspace(-6, 2, 30):
        G = 1.0 / oracle.ro_dg(oracle.ro_F(r * p.gref, p), p)
        assert G < prev
        prev = G
    G = 1.0 / oracle.ro_dg(oracle.ro_F(1e-7 * p.gref, p), p)
    assert abs(G / p.G0 - 1.0) < 1e-5


def drive(s, p, path):
    """Apply strain increments along `path` (list of strains); return stresses."""
    taus = []
    g_prev = path[0]
    for g in path[1:]:
        oracle.spring_update(s, g, g - g_prev, p)
        taus.append(float(s["tau"][0]))
        g_prev = g
    return np.array(taus)


def test_virgin_and_zero_increment():
    p = soft()
    s = fresh()
    G = oracle.spring_update(s, 0.0, 0.0, p)
    assert s["dir"][0] == 0 and s["tau"][0] == 0.0 and abs(G - p.G0) < 1e-6
    oracle.spring_update(s, 1e-4, 1e-4, p)
    assert s["dir"][0] == 1 and s["mode"][0] == 0
    before = s.copy()
    oracle.spring_update(s, 1e-4, 0.0, p)
    assert s.tobytes() == before.tobytes()


def test_masing_branch_reaches_opposite_skeleton_point_and_loop_closes():
    p = soft()
    ga = 4 * p.gref
    s = fresh()
    up = np.linspace(0.0, ga, 400)
    drive(s, p, up)
    tau_a = float(s["tau"][0])
    assert abs(tau_a - oracle.ro_F(ga, p)) < 1e-12 * tau_a
    down = np.linspace(ga, -ga, 801)
    drive(s, p, down)
    assert s["mode"][0] in (0, 1)
    assert abs(float(s["tau"][0]) + tau_a) < 1e-12 * tau_a
    back = np.linspace(-ga, ga, 801)
    drive(s, p, back)
    assert abs(float(s["tau"][0]) - tau_a) < 1e-12 * tau_a
    # beyond the previous maximum the skeleton is followed again
    drive(s, p, np.linspace(ga, 2 * ga, 50))
    assert s["mode"][0] == 0
    assert abs(float(s["tau"][0]) - oracle.ro_F(2 * ga, p)) < 1e-12 * tau_a
    assert abs(float(s["gmax"][0]) - 2 * ga) < 1e-18


@pytest.mark.parametrize("ratio", [0.3, 1.0, 5.0])
def test_loop_damping_closed_form(ratio):
    p = soft()
    ga = ratio * p.gref
    s = fresh()
    drive(s, p, np.linspace(0.0, ga, 2000))
    tau_a = float(s["tau"][0])
    n = 20000
    path = np.concatenate([np.linspace(ga, -ga, n + 1), np.linspace(-ga, ga, n + 1)[1:]])
    taus = drive(s, p, path)
    taus = np.concatenate([[tau_a], taus])
    area = np.sum(0.5 * (taus[1:] + taus[:-1]) * np.diff(path))  # closed loop integral of tau dgamma
    w_el = 0.5 * tau_a * ga
    h_num = abs(area) / (4 * math.pi * w_el)
    h_closed = 2 / math.pi * p.beta / (p.beta + 2) * (1 - tau_a / ga / p.G0)
    assert abs(h_num - h_closed) < 1e-6


def test_tangent_matches_finite_difference_on_skeleton_and_branch():
    p = soft()
    h = 1e-10
    for path in ([0.0, 3e-4, 9e-4], [0.0, 2e-3, 1e-3, 6e-4]):
        s = fresh()
        drive(s, p, path)
        G = oracle.spring_tangent(s, p)
        direction = np.sign(path[-1] - path[-2])
        s1 = s.copy(); s2 = s.copy()
        oracle.spring_update(s1, path[-1] + direction * h, direction * h, p)
        oracle.spring_update(s2, path[-1] + direction * 2 * h, direction * 2 * h, p)
        fd = (4 * float(s1["tau"][0]) - float(s2["tau"][0]) - 3 * float(s["tau"][0])) / (2 * h) * direction
        assert abs(fd - G) < 1e-5 * G


@pytest.mark.parametrize("S", [5, 10, 50, 150])
def test_multispring_elastic_limit_is_isotropic_hooke(S):
    q, w = oracle.spring_dirs(S)
    rho, vs, vp = 1700.0, 150.0, 150.0 * math.sqrt(6.0)
    G0 = rho * vs * vs
    Kb = rho * (vp * vp - 4.0 / 3.0 * vs * vs)
    D = oracle.elastic_D(q, w, Kb, G0)
    Dh = ex.hooke(Kb - 2.0 / 3.0 * G0, G0)
    assert np.abs(D - Dh).max() <= 1e-13 * np.abs(Dh).max()
    # spring strains are shear projections: no spring sees a volumetric strain
    assert np.abs(q[:, :3].sum(axis=1)).max() < 1e-12


def test_multispring_rejects_too_few_springs():
    with pytest.raises(ValueError):
        oracle.spring_dirs(4)


def test_multispring_point_D_symmetric_positive_definite_and_softening():
    S = 50
    q, w = oracle.spring_dirs(S)
    p = soft()
    rho, vs, vp = 1700.0, 150.0, 150.0 * math.sqrt(6.0)
    Kb = rho * (vp * vp - 4.0 / 3.0 * vs * vs)
    De = oracle.elastic_D(q, w, Kb, p.G0)
    rng = np.random.default_rng(7)
    springs = np.zeros(S, oracle.SPRING_DTYPE)
    eps = np.zeros(6)
    for k in range(60):
        deps = rng.normal(size=6) * 2e-4
        eps = eps + deps
        D = oracle.point_update(q, w, Kb, p, eps, deps, springs)
        assert np.abs(D - D.T).max() <= 1e-12 * np.abs(D).max()
        ev = np.linalg.eigvalsh(D)
        assert ev.min() > 0
        # softening: the tangent never exceeds the elastic one
        assert np.linalg.eigvalsh(De - D).min() > -1e-6 * np.abs(De).max()
    # tiny strains leave the point (almost) elastic
    springs = np.zeros(S, oracle.SPRING_DTYPE)
    d = np.full(6, 1e-12)
    D = oracle.point_update(q, w, Kb, p, d, d, springs)
    assert np.abs(D - De).max() <= 1e-6 * np.abs(De).max()
