"""The two-level preconditioner (Sec. 2.2: EBE-IPCG with a multigrid preconditioner after
[SC14]) on the GPU against the oracle:

  * the coarse (linear-element) operator K1, M1, Cb1 and A1 against the oracle's, which
    is pinned to P^T A P (tests/test_oracle_coarse.py) -- FP32 arithmetic on the device,
    so to FP32 rounding of the element sums;
  * whole runs with the two-level preconditioner against the oracle's plain block-Jacobi
    PCG at the same 1e-8 tolerance (surface relative L2 <= 1e-6): the preconditioner
    changes the path to the solution, not the solution;
  * the coarse solve does work (coarse iterations counted) and the inner solve started
    from its interpolated solution needs fewer iterations than from zero.
"""
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


def small(dims=(4, 3, 3), nt=60, S=10, seed=5):
    m = synth.kuhn_box(*dims, 10.0 * dims[0], 10.0 * dims[1], 10.0 * dims[2], layer_depths=(15.0,), jitter=0.1,
                       seed=seed)
    w = synth.band_limited_wave(seed, nt + 1, 0.01)
    return synth.Workload("small", m, synth.two_layer_materials(0.02), S, 0.01, nt, w)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("scatter", [B.NS_SCATTER_ATOMIC, B.NS_SCATTER_COLOUR])
def test_coarse_operator_matches_oracle(scatter):
    wl = small(dims=(4, 3, 2))
    o = oracle.Oracle.from_workload(wl)
    cid, par, nc = oracle.coarse_map(wl.mesh.conn, wl.mesh.n_nodes)
    rng = np.random.default_rng(2)
    with B.Simulation(wl, precision=B.NS_PREC_FP64_IR, multigrid=1, scatter=scatter) as sim:
        E = wl.mesh.n_elems
        A = rng.normal(size=(E, 4, 6, 6)) * 1e7
        D = np.einsum("epij,epkj->epik", A, A) + 1e8 * np.eye(6)
        B.ns_write_state(sim.ctx, 0, D=D)
        xc = rng.normal(size=(nc, 3))
        for op in ("K", "M", "Cb", "A"):
            yg = B.ns_apply_coarse_operator(sim.ctx, op, xc)
            yo = o.coarse_operator(op, xc, cid, nc, D=D)
            assert np.abs(yg - yo).max() <= 2e-5 * np.abs(yo).max(), op


@pytest.mark.parametrize("precision,scatter", [(B.NS_PREC_FP64_IR, B.NS_SCATTER_ATOMIC),
                                               (B.NS_PREC_FP64_IR, B.NS_SCATTER_COLOUR),
                                               (B.NS_PREC_FP64_IR16, B.NS_SCATTER_ATOMIC)])
def test_multigrid_run_matches_oracle(precision, scatter):
    wl = small(dims=(4, 3, 3), nt=60)
    nsteps = 30
    o = oracle.Oracle.from_workload(wl, x0_prev=False)
    us, vs = [], []
    with B.Simulation(wl, surface_ring_steps=nsteps, precision=precision, multigrid=1, scatter=scatter,
                      x0_prev=0) as sim:
        for _ in range(nsteps):
            o.step()
            us.append(o.u[wl.mesh.surf].copy())
            vs.append(o.v[wl.mesh.surf].copy())
        sim.advance(nsteps)
        s = sim.surface(1, nsteps)
        th, _ = sim.state()
        st = sim.stats()
    assert rel(s["u"], np.array(us)) <= 1e-6
    assert rel(s["v"], np.array(vs)) <= 1e-6
    assert np.mean(th["mode"] == o.th["mode"]) > 0.999
    assert st["coarse_iters_total"] > 0


def test_coarse_start_cuts_inner_iterations():
    """A column of the large model (5 m hexahedra, dt 0.005 s, 150 springs): the inner FP32
    solve started from the interpolated coarse solution takes fewer iterations than from
    zero.  Both runs solve to 1e-12, where the record no longer depends on the path to the
    solution, and agree to 1e-6 (at 1e-8 the two preconditioners' stopping points differ
    by the tolerance's own effect, ~5e-5 on this record)."""
    wl = synth.large_single_model(column=(30, 30, 6, 6))
    wl.wave = synth.main_motion_record()
    n = 40
    out = {}
    for mg in (0, 1):
        with B.Simulation(wl, surface_ring_steps=n, precision=B.NS_PREC_FP64_IR, x0_prev=0, multigrid=mg,
                          inner_max_iter=200, cg_tol=1e-12) as sim:
            sim.advance(n)
            st = sim.stats()
            out[mg] = (sim.surface(1, n)["v"], st["inner_iters_total"], st["coarse_iters_total"], st["cg_iters_total"])
    print("inner iterations without / with the coarse start: %d / %d (coarse %d), outer %d / %d" % (
        out[0][1], out[1][1], out[1][2], out[0][3], out[1][3]))
    assert rel(out[1][0], out[0][0]) <= 1e-6
    assert out[1][2] > 0 and out[1][1] < out[0][1]
