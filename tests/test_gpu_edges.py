"""Degenerate and edge cases of the time stepper on the GPU: a record of zeros (zero
right-hand side: the CG's zero-right-hand-side exit, no spring ever loaded), the
smallest mesh (one hexahedron = 6 elements, far from a full block) without boundary
faces or surface nodes, driven only by an initial velocity, against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2604_02755_gb300 import binding as B
from paper_2604_02755_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    B.lib()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("precision", [B.NS_PREC_FP64, B.NS_PREC_FP64_IR, B.NS_PREC_FP64_IR16])
def test_zero_record_leaves_everything_at_rest(precision):
    m = synth.kuhn_box(3, 2, 3, 30.0, 20.0, 30.0, layer_depths=(15.0,), jitter=0.1, seed=2)
    wl = synth.Workload("zero", m, synth.two_layer_materials(0.02), 10, 0.01, 20, np.zeros((21, 3)))
    with B.Simulation(wl, surface_ring_steps=10, precision=precision) as sim:
        th0, D0 = sim.state()
        sim.advance(10)
        s = sim.surface(1, 10)
        th, D = sim.state()
        st = sim.stats()
    assert not np.any(s["u"]) and not np.any(s["v"]) and not np.any(s["a"])
    assert th.tobytes() == th0.tobytes()  # virgin springs
    # elastic tangent again, up to the rounding of its (double-float) accumulation over the springs
    assert np.max(np.abs(D - D0)) <= 1e-13 * np.max(np.abs(D0))
    assert st["cg_iters_last"] == 0


def test_single_hexahedron_without_boundary_against_oracle():
    m = synth.kuhn_box(1, 1, 1, 5.0, 5.0, 5.0, jitter=0.0, seed=1)
    mats = synth.two_layer_materials(0.02)[:1]
    rng = np.random.default_rng(4)
    v0 = rng.normal(size=(m.n_nodes, 3)) * 0.05
    nsteps = 12
    wl = synth.Workload("one hexahedron", m, mats, 10, 0.005, nsteps, np.zeros((nsteps + 1, 3)))
    cfg = B.ns_config_default(n_springs=10, dt=0.005)
    ctx = B.ns_create(cfg)
    try:
        B.ns_upload_mesh(ctx, m.xyz, m.conn, m.mat)
        B.ns_set_materials(ctx, mats)
        B.ns_set_boundary(ctx, np.zeros((0, 6), np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32),
                          np.zeros(0, np.int32))
        B.ns_set_ground_motion(ctx, wl.wave, wl.dt)
        B.ns_write_nodal(ctx, "v", v0)
        B.ns_advance(ctx, nsteps)
        u = B.ns_read_nodal(ctx, "u", m.n_nodes)
        th, _ = B.ns_read_state(ctx, 0, m.n_elems, 10)
    finally:
        B.ns_destroy(ctx)
    o = oracle.Oracle(m.xyz, m.conn, m.mat, mats, None, None, None, 10, wl.dt, wl.wave)
    o.v[:] = v0
    for _ in range(nsteps):
        o.step()
    assert m.n_elems == 6
    assert rel(u, o.u) <= 1e-6
    assert np.array_equal(th["dir"], o.th["dir"]) and np.array_equal(th["mode"], o.th["mode"])
