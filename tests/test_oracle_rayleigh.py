"""Pin of the oracle's Rayleigh damping (Sec. 2.1: C^n from the damping ratio h^n).

The reading: C_r = alpha M + beta K with alpha and beta chosen so that the modal
damping ratio equals h at f1 = 0.1 Hz and f2 = 2.5 Hz.  This is checked through
properties of the assembled operators, not by retyping the formula:

  * modal damping: for every elastic mode phi_i of K phi = w^2 M phi (dense
    generalised eigenproblem from the oracle's own K and M), the Rayleigh operator
    is diagonal in the modal basis and zeta_i = phi_i.C_r phi_i / (2 w_i phi_i.M phi_i)
    lies on one curve zeta(w) = a/(2w) + b w/2; that curve, fitted over all modes,
    passes through h at 2 pi 0.1 Hz and at 2 pi 2.5 Hz.  A swapped alpha/beta, a
    frequency used for an angular frequency or a dropped factor 2 each move the
    curve off those two points;
  * free decay: one mode released from rest under the oracle's own Newmark-beta
    step (no forcing, no dashpots) decays per step by the factor the trapezoidal
    rule (the average-acceleration scheme) gives for a damped oscillator of that
    w and zeta -- the decay rate is read from the two-term recurrence the modal
    coordinate obeys.
"""
import numpy as np
import pytest
from scipy.linalg import eigh

import oracle
from paper_2604_02755_gb300 import synth


def linear_box(dims, h):
    m = synth.kuhn_box(*dims, 40.0, 40.0, 30.0, layer_depths=(15.0,), jitter=0.1, seed=7)
    mats = synth.two_layer_materials(h)
    for mm in mats:
        mm["gamma_ref"] = 1e30  # linear springs: the tangent stays elastic
    return m, mats


def dense(o, which):
    n = o.n_nodes * 3
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = o.operator(which, e).ravel()
    return 0.5 * (A + A.T)


def elastic_modes(o):
    K, M, Cr = dense(o, "K"), dense(o, "M"), dense(o, "Cr")
    w2, phi = eigh(K, M)
    keep = w2 > 1e-6 * w2.max()  # drop the six rigid-body modes (w = 0)
    assert (~keep).sum() == 6
    return np.sqrt(w2[keep]), phi[:, keep], K, M, Cr


@pytest.mark.parametrize("dims,h", [((1, 1, 1), 0.02), ((2, 2, 2), 0.05)])
def test_modal_damping_curve_hits_h_at_calibration_frequencies(dims, h):
    m, mats = linear_box(dims, h)
    o = oracle.Oracle(m.xyz, m.conn, m.mat, mats, n_springs=10, dt=0.01)
    w, phi, K, M, Cr = elastic_modes(o)
    # C_r is diagonal in the modal basis (proportional damping)
    Cm = phi.T @ Cr @ phi
    off = Cm - np.diag(np.diag(Cm))
    assert np.abs(off).max() <= 1e-9 * np.abs(np.diag(Cm)).max()
    mm = np.einsum("ji,jk,ki->i", phi, M, phi)
    zeta = np.diag(Cm) / (2.0 * w * mm)
    # zeta w = a/2 + b w^2/2 is linear in (a, b): fit over all elastic modes
    A = np.stack([0.5 * np.ones_like(w), 0.5 * w ** 2], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, zeta * w, rcond=None)
    assert np.abs(A @ np.array([a, b]) - zeta * w).max() <= 1e-9 * np.abs(zeta * w).max()

    def curve(f):
        om = 2.0 * np.pi * f
        return a / (2.0 * om) + b * om / 2.0

    assert abs(curve(0.1) - h) <= 1e-9 * h
    assert abs(curve(2.5) - h) <= 1e-9 * h
    # between the two frequencies the Rayleigh curve dips below h, outside it rises
    assert curve(0.5) < h and curve(0.05) > h and curve(10.0) > h


def test_free_decay_of_one_mode():
    h = 0.05
    m, mats = linear_box((1, 1, 1), h)
    dt = 0.002
    o = oracle.Oracle(m.xyz, m.conn, m.mat, mats, n_springs=10, dt=dt, acc=np.zeros((1, 3)), tol=1e-13)
    w, phi, K, M, Cr = elastic_modes(o)
    i = 0  # the lowest elastic mode
    wi = w[i]
    mode = phi[:, i].reshape(-1, 3)
    mm = phi[:, i] @ M @ phi[:, i]
    zeta = phi[:, i] @ Cr @ phi[:, i] / (2.0 * wi * mm)
    # consistent initial state: u = phi, v = 0, q = K u, a = -M^-1 K u = -w^2 phi
    o.u[:] = mode
    o.q[:] = (K @ phi[:, i]).reshape(-1, 3)
    o.a[:] = -wi ** 2 * mode
    c = [1.0]
    for _ in range(120):
        o.step()
        c.append(phi[:, i] @ M @ o.u.ravel() / mm)
    c = np.array(c)
    # the modal coordinate obeys c[n+1] = s c[n] - p c[n-1] with p = |z|^2, z the
    # per-step amplification of the trapezoidal rule
    Afit = np.stack([c[1:-1], -c[:-2]], axis=1)
    (s, p), *_ = np.linalg.lstsq(Afit, c[2:], rcond=None)
    lam = complex(-zeta * wi, wi * np.sqrt(1.0 - zeta ** 2))
    z = (1.0 + lam * dt / 2.0) / (1.0 - lam * dt / 2.0)
    assert abs(p - abs(z) ** 2) <= 1e-8
    assert abs(s - 2.0 * z.real) <= 1e-8
    # and the decay is that of damping ratio h-curve value, clearly nonzero
    assert abs(z) < 1.0 - 1e-4
