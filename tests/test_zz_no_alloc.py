"""The allocation-free spring entry point (for callers that cannot allocate device
memory when they call it) gives the same result as the allocating ns_spring_points,
called through the C ABI, on two calls in a row that carry the spring state forward.

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_2604_02755_gb300 import binding as B
from paper_2604_02755_gb300 import build, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    build.build()
    S = 50
    m = synth.kuhn_box(2, 2, 2, 20.0, 20.0, 20.0, layer_depths=(10.0,))
    wl = synth.Workload("noalloc", m, synth.two_layer_materials(0.02), S, 0.01, 10,
                        synth.band_limited_wave(3, 11, 0.01))
    rng = np.random.default_rng(21)
    npts = 48
    assert npts <= B.ns_spring_points_noalloc_capacity(S)
    mat = (np.arange(npts) % 2).astype(np.int32)
    th_a = np.zeros(npts * S, B.SPRING_DTYPE)
    th_b = np.zeros(npts * S, B.SPRING_DTYPE)
    eps = np.zeros((npts, 6))
    with B.Simulation(wl) as sim:
        for call in range(2):
            deps = rng.normal(size=(npts, 6)) * 10 ** rng.uniform(-5, -3, size=(npts, 1))
            eps = eps + deps
            th_a, Da = B.ns_spring_points(sim.ctx, mat, eps, deps, th_a)
            th_b, Db = B.ns_spring_points_noalloc(sim.ctx, mat, eps, deps, th_b)
            assert np.abs(Db - Da).max() <= 1e-12 * np.abs(Da).max(), call
            assert np.array_equal(th_a["dir"], th_b["dir"]) and np.array_equal(th_a["mode"], th_b["mode"])
            for f in ("tau", "gR", "tR", "gmax"):
                assert np.abs(th_a[f] - th_b[f]).max() <= 1e-12 * (np.abs(th_a[f]).max() + 1e-300), f
        assert (th_a["dir"] != 0).any()
        too_many = B.ns_spring_points_noalloc_capacity(S) + 1
        with pytest.raises(B.NsError) as ei:
            B.ns_spring_points_noalloc(sim.ctx, np.zeros(too_many, np.int32), np.zeros((too_many, 6)),
                                       np.zeros((too_many, 6)), np.zeros(too_many * S, B.SPRING_DTYPE))
        assert ei.value.code == -1


def test_noalloc_at_full_capacity():
    """As many points as the staging array holds at 150 springs per point: the last
    sub-arrays of the carve-up reach the end of the array (alignment slack included)."""
    build.build()
    S = 150
    m = synth.kuhn_box(2, 2, 2, 20.0, 20.0, 20.0, layer_depths=(10.0,))
    wl = synth.Workload("noalloc-full", m, synth.two_layer_materials(0.02), S, 0.01, 10,
                        synth.band_limited_wave(3, 11, 0.01))
    npts = B.ns_spring_points_noalloc_capacity(S)
    assert npts == (8 * 2 ** 20 - 11 * 256) // (556 + 80 * S)
    rng = np.random.default_rng(22)
    mat = (np.arange(npts) % 2).astype(np.int32)
    th_a = np.zeros(npts * S, B.SPRING_DTYPE)
    th_b = np.zeros(npts * S, B.SPRING_DTYPE)
    eps = np.zeros((npts, 6))
    with B.Simulation(wl) as sim:
        for call in range(2):
            deps = rng.normal(size=(npts, 6)) * 10 ** rng.uniform(-5, -3, size=(npts, 1))
            eps = eps + deps
            th_a, Da = B.ns_spring_points(sim.ctx, mat, eps, deps, th_a)
            th_b, Db = B.ns_spring_points_noalloc(sim.ctx, mat, eps, deps, th_b)
            assert np.abs(Db - Da).max() <= 1e-12 * np.abs(Da).max(), call
            assert th_a.tobytes() == th_b.tobytes() or all(
                np.abs(th_a[f] - th_b[f]).max() <= 1e-12 * (np.abs(th_a[f]).max() + 1e-300)
                for f in ("tau", "gR", "tR", "gmax"))
            assert np.array_equal(th_a["dir"], th_b["dir"]) and np.array_equal(th_a["mode"], th_b["mode"])
