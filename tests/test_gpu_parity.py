"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances:
  * element operators, spring points: 1e-12 relative (both sides FP64; only the
    summation order differs);
  * whole steps: relative L2 of surface displacement and velocity <= 1e-6
    (both sides stop CG at ||r|| <= 1e-8 ||b||; the solutions differ at the
    level of that tolerance, never above it);
  * index-valued state (spring direction and branch flags): bit-exact.
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


def small(dims=(3, 2, 2), S=10, nt=80, seed=5, jitter=0.1, peak=3.0):
    m = synth.kuhn_box(*dims, 30.0 * dims[0] / 3, 20.0 * dims[1] / 2, 30.0, layer_depths=(15.0,), jitter=jitter,
                       seed=seed)
    w = synth.band_limited_wave(seed, nt + 1, 0.01, peak=peak)
    return synth.Workload("small", m, synth.two_layer_materials(0.02), S, 0.01, nt, w)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("scatter,pair", [(B.NS_SCATTER_ATOMIC, 0), (B.NS_SCATTER_COLOUR, 0),
                                          (B.NS_SCATTER_ATOMIC, 1), (B.NS_SCATTER_COLOUR, 1)])
def test_operators_match_oracle(scatter, pair):
    """Element operators against the oracle's; pair = 1 runs them in double-float
    arithmetic on the FP32 pipes, which must still meet the FP64 bound."""
    wl = small(dims=(4, 3, 2))
    o = oracle.Oracle.from_workload(wl)
    rng = np.random.default_rng(0)
    with B.Simulation(wl, scatter=scatter, pair_operator=pair) as sim:
        # random symmetric positive definite tangents at every point
        E = wl.mesh.n_elems
        A = rng.normal(size=(E, 4, 6, 6)) * 1e7
        D = np.einsum("epij,epkj->epik", A, A) + 1e8 * np.eye(6)
        B.ns_write_state(sim.ctx, 0, D=D)
        x = rng.normal(size=(wl.mesh.n_nodes, 3))
        for op in ("K", "M", "Cb", "A", "Cr"):
            yg = B.ns_apply_operator(sim.ctx, op, x)
            yo = o.operator(op, x, D=D)
            assert np.abs(yg - yo).max() <= 1e-12 * np.abs(yo).max(), op


@pytest.mark.parametrize("S,tensor", [(50, 1), (50, 0), (150, 1), (12, 1)])
def test_spring_points_match_oracle(S, tensor):
    """Multi-spring points against the oracle, the tangent assembled on the tensor cores
    (digit products) or in double-float sums."""
    wl = small()
    q, w = oracle.spring_dirs(S)
    mats = wl.materials
    rng = np.random.default_rng(3)
    npts = 64
    mat = (np.arange(npts) % 2).astype(np.int32)
    th_g = np.zeros((npts, S), B.SPRING_DTYPE)
    th_o = np.zeros((npts, S), oracle.SPRING_DTYPE)
    eps = np.zeros((npts, 6))
    wl2 = synth.Workload(wl.name, wl.mesh, mats, S, wl.dt, wl.n_steps, wl.wave)
    with B.Simulation(wl2, spring_tensor_cores=tensor) as sim:
        for it in range(40 if S <= 50 else 12):
            scale = 10 ** rng.uniform(-6, -3, size=(npts, 1))
            deps = rng.normal(size=(npts, 6)) * scale
            if it == 5:
                deps[:4] = 0.0  # zero increments leave the state untouched
            eps = eps + deps
            th_g, Dg = B.ns_spring_points(sim.ctx, mat, eps, deps, th_g.reshape(-1))
            th_g = th_g.reshape(npts, S)
            for p in range(npts):
                mm = mats[mat[p]]
                ro = oracle.ro_params(mm["rho"], mm["vs"], mm["gamma_ref"], mm["h_max"])
                Kb = mm["rho"] * (mm["vp"] ** 2 - 4.0 / 3.0 * mm["vs"] ** 2)
                Do = oracle.point_update(q, w, Kb, ro, eps[p], deps[p], th_o[p])
                assert np.abs(Dg[p] - Do).max() <= 1e-12 * np.abs(Do).max(), (it, p)
            assert np.array_equal(th_g["dir"], th_o["dir"])
            assert np.array_equal(th_g["mode"], th_o["mode"])
            for f in ("tau", "tR"):
                scale = np.abs(th_o[f]).max() + 1e-300
                assert np.abs(th_g[f] - th_o[f]).max() <= 1e-12 * scale, f
            for f in ("gR", "gmax"):
                scale = np.abs(th_o[f]).max() + 1e-300
                assert np.abs(th_g[f] - th_o[f]).max() <= 1e-13 * scale, f
    assert (th_o["mode"] == 1).any() and (th_o["mode"] == 0).any()


def run_both(wl, nsteps, **cfg):
    o = oracle.Oracle.from_workload(wl)
    with B.Simulation(wl, surface_ring_steps=max(nsteps, 1), **cfg) as sim:
        for _ in range(nsteps):
            o.step()
        sim.advance(nsteps)
        out = dict(u=sim.nodal("u"), v=sim.nodal("v"), a=sim.nodal("a"), q=sim.nodal("q"), du=sim.nodal("du"),
                   surf=sim.surface(1, nsteps), state=sim.state(), stats=sim.stats())
    return o, out


def test_one_step_matches_oracle():
    wl = small(dims=(4, 3, 2), nt=40)
    o, g = run_both(wl, 1)
    for f in ("u", "v", "a", "q", "du"):
        assert rel(g[f], getattr(o, f)) <= 1e-7, f
    th, D = g["state"]
    assert rel(D, o.D) <= 1e-8
    assert np.array_equal(th["dir"], o.th["dir"]) and np.array_equal(th["mode"], o.th["mode"])
    assert abs(g["stats"]["cg_iters_last"] - o.iters) <= 2


@pytest.mark.parametrize("scatter,precision", [(B.NS_SCATTER_ATOMIC, B.NS_PREC_FP64),
                                               (B.NS_SCATTER_COLOUR, B.NS_PREC_FP64),
                                               (B.NS_SCATTER_ATOMIC, B.NS_PREC_FP64_IR),
                                               (B.NS_SCATTER_COLOUR, B.NS_PREC_FP64_IR),
                                               (B.NS_SCATTER_ATOMIC, B.NS_PREC_FP64_IR16),
                                               (B.NS_SCATTER_COLOUR, B.NS_PREC_FP64_IR16),
                                               (B.NS_SCATTER_ATOMIC, -1), (B.NS_SCATTER_COLOUR, -2)])
def test_thirty_steps_surface_parity(scatter, precision):
    """precision -1 / -2: the FP64 + FP32-inner / FP16-tangent forms with the FP64-accuracy
    operator applications in double-float arithmetic."""
    wl = small(dims=(4, 3, 3), nt=60)
    nsteps = 30
    o = oracle.Oracle.from_workload(wl)
    us, vs = [], []
    pair = int(precision < 0)
    precision = {-1: B.NS_PREC_FP64_IR, -2: B.NS_PREC_FP64_IR16}.get(precision, precision)
    with B.Simulation(wl, surface_ring_steps=nsteps, scatter=scatter, precision=precision,
                      pair_operator=pair) as sim:
        for _ in range(nsteps):
            o.step()
            us.append(o.u[wl.mesh.surf].copy())
            vs.append(o.v[wl.mesh.surf].copy())
        sim.advance(nsteps)
        s = sim.surface(1, nsteps)
        th, _ = sim.state()
    assert rel(s["u"], np.array(us)) <= 1e-6
    assert rel(s["v"], np.array(vs)) <= 1e-6
    # almost every spring ends in the same branch state
    assert np.mean(th["mode"] == o.th["mode"]) > 0.999
    assert (o.th["mode"] == 1).mean() > 0.01  # hysteresis happened


def test_colour_scatter_is_deterministic_and_streaming_is_invisible():
    """Deterministic scatter: repeated runs, state streamed through device chunk buffers
    (part or all of it, two ring depths) and state updated in place in pinned host memory
    (zero-copy) all give bit-identical fields, tangents and spring states."""
    wl = small(dims=(4, 3, 3), nt=60)
    n = 12
    S = wl.n_springs
    per_elem = B.ns_state_bytes(1, S)
    res = []
    for budget, chunk, ring, mode in ((-1, 100000, 3, 0), (-1, 100000, 3, 0), (per_elem * 37, 13, 3, 0), (0, 29, 2, 0),
                                      (per_elem * 37, 13, 3, B.NS_STREAM_ZERO_COPY)):
        with B.Simulation(wl, scatter=B.NS_SCATTER_COLOUR, surface_ring_steps=n, device_state_budget=budget,
                          chunk_elems=chunk, ring_depth=ring, stream_mode=mode) as sim:
            sim.advance(n)
            st = sim.stats()
            res.append((sim.nodal("u"), sim.nodal("v"), sim.state(), st))
    u0, v0, (th0, D0), _ = res[0]
    for u, v, (th, D), st in res[1:]:
        assert np.array_equal(u, u0) and np.array_equal(v, v0)
        assert np.array_equal(D, D0)
        assert th.tobytes() == th0.tobytes()
    assert res[2][3]["streamed_elems"] == wl.mesh.n_elems - 37
    assert res[3][3]["streamed_elems"] == wl.mesh.n_elems
    assert res[3][3]["h2d_bytes"] == n * wl.mesh.n_elems * per_elem
    # zero-copy: the kernel updated the host-resident springs in place
    assert res[4][3]["streamed_elems"] == wl.mesh.n_elems - 37
    assert res[4][3]["h2d_bytes"] == n * (wl.mesh.n_elems - 37) * per_elem


def test_checkpoint_restore_bit_identical():
    wl = small(dims=(3, 3, 2), nt=40)
    with B.Simulation(wl, scatter=B.NS_SCATTER_COLOUR) as a:
        a.advance(10)
        ua = a.nodal("u")
        tha, Da = a.state()
    with B.Simulation(wl, scatter=B.NS_SCATTER_COLOUR) as b:
        b.advance(4)
        ck = B.ns_checkpoint(b.ctx)
    with B.Simulation(wl, scatter=B.NS_SCATTER_COLOUR) as c:
        B.ns_restore(c.ctx, ck)
        assert c.stats()["steps"] == 4
        c.advance(6)
        assert np.array_equal(c.nodal("u"), ua)
        th, D = c.state()
        assert np.array_equal(D, Da) and th.tobytes() == tha.tobytes()


def test_errors_are_reported():
    wl = small()
    with B.Simulation(wl) as sim:
        with pytest.raises(B.NsError) as ei:
            B.ns_set_ground_motion(sim.ctx, wl.wave, 0.02)
        assert ei.value.code == -1
        with pytest.raises(B.NsError):
            sim.surface(1, 1)  # nothing advanced yet
    bad = small()
    bad.mesh.xyz[bad.mesh.conn[0, 4]] += 1.0  # curved edge
    with pytest.raises(B.NsError) as ei:
        B.Simulation(bad)
    assert ei.value.code == -5
    wl = small()
    with B.Simulation(wl, cg_max_iter=2) as sim:
        with pytest.raises(B.NsError) as ei:
            sim.advance(1)
        assert ei.value.code == -6


@pytest.mark.parametrize("precision,nsteps", [(B.NS_PREC_FP64, 60), (B.NS_PREC_FP64_IR, 60)])
def test_tiny_two_layer_case_parity(precision, nsteps):
    """The plain FP64 tiny case (200x200x60 m, 10x10x6 hexahedra -> 3,600 quadratic
    tetrahedra, 10 springs/point, dt 0.01 s) over its first steps."""
    wl = synth.tiny_two_layer()
    o = oracle.Oracle.from_workload(wl)
    us, vs = [], []
    with B.Simulation(wl, surface_ring_steps=nsteps, precision=precision) as sim:
        for _ in range(nsteps):
            o.step()
            us.append(o.u[wl.mesh.surf].copy())
            vs.append(o.v[wl.mesh.surf].copy())
        sim.advance(nsteps)
        s = sim.surface(1, nsteps)
    assert rel(s["u"], np.array(us)) <= 1e-6
    assert rel(s["v"], np.array(vs)) <= 1e-6


def test_tiny_two_layer_full_record():
    """All 300 steps of the tiny case, through the main motion.  Over this record the
    CG stopping tolerance itself decides the answer at the 1e-4 level: the oracle at
    1e-8 and at 1e-12 differ by 7.0e-5 in surface displacement (relative L2), while 1e-10
    and 1e-12 agree to 1.7e-10.  Parity is therefore checked with both sides solving to
    1e-12, where the answer no longer depends on the tolerance."""
    wl = synth.tiny_two_layer()
    nsteps = wl.n_steps
    o = oracle.Oracle.from_workload(wl, tol=1e-12)
    us, vs = [], []
    for _ in range(nsteps):
        o.step()
        us.append(o.u[wl.mesh.surf].copy())
        vs.append(o.v[wl.mesh.surf].copy())
    with B.Simulation(wl, surface_ring_steps=nsteps, precision=B.NS_PREC_FP64_IR, cg_tol=1e-12) as sim:
        sim.advance(nsteps)
        s = sim.surface(1, nsteps)
        th, _ = sim.state()
    assert rel(s["u"], np.array(us)) <= 1e-6
    assert rel(s["v"], np.array(vs)) <= 1e-6
    assert np.mean(th["mode"] == o.th["mode"]) > 0.999
    # the plain FP64 method with both sides at the paper's 1e-8, over the whole record:
    # reported beside the 1e-12 figure (the difference is the stopping tolerance's effect)
    o8 = oracle.Oracle.from_workload(wl, tol=1e-8)
    us8, vs8 = [], []
    for _ in range(nsteps):
        o8.step()
        us8.append(o8.u[wl.mesh.surf].copy())
        vs8.append(o8.v[wl.mesh.surf].copy())
    with B.Simulation(wl, surface_ring_steps=nsteps, precision=B.NS_PREC_FP64, cg_tol=1e-8) as sim:
        sim.advance(nsteps)
        s8 = sim.surface(1, nsteps)
    print("tiny full record: both at 1e-12 u %.2e v %.2e; plain FP64 both at 1e-8 u %.2e v %.2e" % (
        rel(s["u"], np.array(us)), rel(s["v"], np.array(vs)), rel(s8["u"], np.array(us8)),
        rel(s8["v"], np.array(vs8))))
    assert rel(s8["u"], np.array(us8)) <= 1e-3 and rel(s8["v"], np.array(vs8)) <= 1e-3


def incident(conn, node):
    return np.nonzero((conn == node).any(axis=1))[0]


def test_large_model_sampled_outputs():
    """The single large model at full size (7,987,200 elements, 150 springs/point,
    191.7 GB of spring state in HBM), one step in the benchmark's configuration,
    checked on sampled outputs the oracle computes one by one: the operator A at
    sampled nodes (through a sub-model of the incident elements and faces) and the
    multi-spring update of sampled elements from the device's strains."""
    wl = synth.large_single_model()
    m = wl.mesh
    rng = np.random.default_rng(11)
    samp_e = np.sort(rng.choice(m.n_elems, 6, replace=False))
    S = wl.n_springs
    with B.Simulation(wl, precision=B.NS_PREC_FP64_IR, surface_ring_steps=2) as sim:
        sim.advance(1)
        before = [B.ns_read_state(sim.ctx, int(e), 1, S) for e in samp_e]
        sim.advance(1)
        st = sim.stats()
        assert st["relres_last"] <= 1e-8
        u, du = sim.nodal("u"), sim.nodal("du")
        after = [B.ns_read_state(sim.ctx, int(e), 1, S) for e in samp_e]
        # spring update of sampled elements
        q, w = oracle.spring_dirs(S)
        Lq, _ = oracle.quad_points()
        for e, (thb, _), (tha, Da) in zip(samp_e, before, after):
            X = m.xyz[m.conn[e]]
            mm = wl.materials[m.mat[e]]
            ro = oracle.ro_params(mm["rho"], mm["vs"], mm["gamma_ref"], mm["h_max"])
            Kb = mm["rho"] * (mm["vp"] ** 2 - 4.0 / 3.0 * mm["vs"] ** 2)
            th = thb[0].copy()
            for qp in range(4):
                G, _ = oracle.grad(X, Lq[qp])
                Bm = oracle.bmatrix(G)
                eps = Bm @ u[m.conn[e]].ravel()
                deps = Bm @ du[m.conn[e]].ravel()
                Do = oracle.point_update(q, w, Kb, ro, eps, deps, th[qp])
                assert np.abs(Da[0, qp] - Do).max() <= 1e-11 * np.abs(Do).max()
            assert np.array_equal(th["dir"], tha[0]["dir"]) and np.array_equal(th["mode"], tha[0]["mode"])
            assert np.abs(th["tau"] - tha[0]["tau"]).max() <= 1e-11 * (np.abs(th["tau"]).max() + 1e-300)
        # operator at sampled nodes through the oracle on the incident sub-model
        x = rng.normal(size=(m.n_nodes, 3))
        y = B.ns_apply_operator(sim.ctx, "A", x)
        _, Dall = None, None
        for node in rng.choice(m.n_nodes, 4, replace=False):
            els = incident(m.conn, node)
            fcs = np.nonzero((m.faces == node).any(axis=1))[0]
            _, Dloc = zip(*[B.ns_read_state(sim.ctx, int(e), 1, S, theta=False) for e in els])
            Dloc = np.concatenate(Dloc)
            sub = oracle.Oracle(m.xyz, m.conn[els], m.mat[els], wl.materials, m.faces[fcs],
                                np.searchsorted(els, m.face_elem[fcs]), m.face_kind[fcs], S, wl.dt, wl.wave)
            yo = sub.operator("A", x, D=Dloc)
            assert np.abs(y[node] - yo[node]).max() <= 1e-12 * np.abs(yo[node]).max()


@pytest.mark.parametrize("precision", [B.NS_PREC_FP64, B.NS_PREC_FP64_IR])
def test_graph_replay_equals_direct_launches(precision):
    """Captured-and-replayed solver iterations run the same kernels in the same order as
    direct launches: with the deterministic scatter the two records agree bit for bit,
    and the launch counts agree."""
    wl = small(dims=(4, 3, 3), nt=40)
    out = []
    for graphs in (0, 1):
        with B.Simulation(wl, surface_ring_steps=20, scatter=B.NS_SCATTER_COLOUR, precision=precision,
                          graphs=graphs) as sim:
            sim.advance(20)
            s = sim.surface(1, 20)
            out.append((s["u"], s["v"], sim.stats()["kernel_launches"], sim.stats()["cg_iters_total"]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]


def test_staged_operator_equals_direct_loads():
    """The FP32 inner operator reading its element data from tiles staged in shared
    memory by bulk copies (stage 1), or its tangent rows copied per warp asynchronously
    (stage 2), computes what the per-thread-load kernel computes: all sides solve to
    1e-12, so the surface records agree to rounding (atomic scatter order)."""
    wl = small(dims=(6, 5, 4), nt=60)  # 720 elements: two full tiles and a ragged one
    out = []
    for staged in (0, 1, 2):
        for prec in (B.NS_PREC_FP64_IR, B.NS_PREC_FP64_IR16):
            with B.Simulation(wl, surface_ring_steps=30, precision=prec, stage_elements=staged, cg_tol=1e-12) as sim:
                sim.advance(30)
                out.append(sim.surface(1, 30)["v"])
    assert rel(out[2], out[0]) <= 1e-9 and rel(out[3], out[1]) <= 1e-9
    assert rel(out[4], out[0]) <= 1e-9 and rel(out[5], out[1]) <= 1e-9
    assert rel(out[1], out[0]) <= 1e-9  # FP16 storage only changes the preconditioner


def test_warp_staged_operator_matches_oracle():
    """The per-warp staged FP32 operator inside the flexible CG against the oracle's FP64
    PCG over thirty steps (surface relative L2 <= 1e-6), on a mesh whose last warp is
    ragged (720 elements = 22.5 warps)."""
    wl = small(dims=(6, 5, 4), nt=60)
    o = oracle.Oracle.from_workload(wl)
    us = []
    with B.Simulation(wl, surface_ring_steps=30, precision=B.NS_PREC_FP64_IR, stage_elements=2) as sim:
        for _ in range(30):
            o.step()
            us.append(o.v[wl.mesh.surf].copy())
        sim.advance(30)
        s = sim.surface(1, 30)
    assert rel(s["v"], np.array(us)) <= 1e-6


def test_autotune_steps_are_ordinary_steps():
    """The autotuner on the simulation's own steps: advancing 16 steps through it (14
    candidate launch shapes at 10 springs, two of them timed twice) gives the record of 16
    plain steps bit for bit (colour scatter, so that no atomic order differs between the
    runs), reports a time for every shape and keeps the fastest."""
    wl = small(dims=(4, 3, 3), nt=60)
    out = []
    for tune in (False, True):  # colour scatter: the order of every sum is fixed
        with B.Simulation(wl, scatter=B.NS_SCATTER_COLOUR, surface_ring_steps=22) as sim:
            sim.advance(2)
            if tune:
                t = B.ns_autotune_steps(sim.ctx, 16)
            else:
                sim.advance(16)
            sim.advance(4)
            out.append(sim.surface(1, 22))
    assert np.array_equal(out[0]["u"], out[1]["u"]) and np.array_equal(out[0]["v"], out[1]["v"])
    n = len(t["tile_ms"])
    assert n == 14 and all(0 < x < 1e29 for x in t["tile_ms"])
    k = int(np.argmin(t["tile_ms"]))
    assert (t["chosen_tile_points"], t["chosen_tile_blocks"]) == (t["tile_points"][k], t["tile_blocks"][k])
    with B.Simulation(wl) as sim:
        sim.advance(1)
        with pytest.raises(RuntimeError):
            B.ns_autotune_steps(sim.ctx, 3)  # fewer steps than launch shapes


def test_autotune_keeps_results_and_state():
    """The autotuner times block shapes on a copy of the state and chunk sizes by round
    trips through the ring; the run it tunes is bit-identical to an untuned one."""
    wl = small(dims=(4, 3, 3), nt=60)
    per_elem = B.ns_state_bytes(1, wl.n_springs)
    out = []
    for tune in (False, True):
        with B.Simulation(wl, scatter=B.NS_SCATTER_COLOUR, surface_ring_steps=12, device_state_budget=per_elem * 40,
                          chunk_elems=16, ring_depth=3) as sim:
            sim.advance(4)
            before = sim.state()
            if tune:
                t = B.ns_autotune(sim.ctx)
                after = sim.state()
                assert after[0].tobytes() == before[0].tobytes() and np.array_equal(after[1], before[1])
                assert t["chosen_tile_points"] in t["tile_points"] and min(t["tile_ms"]) > 0
                assert t["chosen_chunk_elems"] in t["chunk_elems"] and min(t["chunk_gbps"]) > 0
            sim.advance(8)
            out.append((sim.nodal("u"), sim.state()))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1][0].tobytes() == out[1][1][0].tobytes()


@pytest.mark.parametrize("precision,scatter", [(B.NS_PREC_FP64, B.NS_SCATTER_ATOMIC),
                                               (B.NS_PREC_FP64_IR, B.NS_SCATTER_ATOMIC),
                                               (B.NS_PREC_FP64_IR16, B.NS_SCATTER_ATOMIC),
                                               (B.NS_PREC_FP64, B.NS_SCATTER_COLOUR),
                                               (B.NS_PREC_FP64_IR, B.NS_SCATTER_COLOUR)])
def test_zero_start_parity(precision, scatter):
    """CG started from zero (no operator application for the initial residual) against
    the oracle started from zero.  Started from zero, the solve also accumulates the
    internal force q^n = q^{n-1} + K du from the iterations' own K p, so q is compared
    with the oracle's q, which applies K to the increment."""
    wl = small(dims=(4, 3, 3), nt=60)
    nsteps = 20
    o = oracle.Oracle.from_workload(wl, x0_prev=False)
    us = []
    with B.Simulation(wl, surface_ring_steps=nsteps, precision=precision, x0_prev=0, scatter=scatter) as sim:
        for _ in range(nsteps):
            o.step()
            us.append(o.u[wl.mesh.surf].copy())
        sim.advance(nsteps)
        s = sim.surface(1, nsteps)
        q = sim.nodal("q")
    assert rel(s["u"], np.array(us)) <= 1e-6
    assert rel(q, o.q) <= 1e-6


@pytest.mark.parametrize("how", ["morton", "shuffled"])
def test_renumbered_mesh_parity(how):
    """Morton-ordered and shuffled numberings of the same mesh (the second defeats the
    operator's gather locality) against the oracle on the same numbering."""
    import dataclasses
    base = small(dims=(4, 3, 3), nt=60)
    wl = dataclasses.replace(base, mesh=synth.renumber(base.mesh, how, seed=11))
    nsteps = 20
    o = oracle.Oracle.from_workload(wl)
    us = []
    with B.Simulation(wl, surface_ring_steps=nsteps, precision=B.NS_PREC_FP64_IR, x0_prev=0) as sim:
        for _ in range(nsteps):
            o.step()
            us.append(o.u[wl.mesh.surf].copy())
        sim.advance(nsteps)
        s = sim.surface(1, nsteps)
    assert rel(s["u"], np.array(us)) <= 1e-6


@pytest.mark.parametrize("mode", ["ring-part", "ring-all", "zero-copy"])
def test_streamed_state_matches_oracle(mode):
    """Spring state streamed from pinned host memory (Alg. 3) against the oracle, which
    keeps all of it in one array: part of the state through a ring of three device
    buffers, all of it through a ring of two, and part of it updated in place in pinned
    host memory (zero-copy)."""
    wl = small(dims=(4, 3, 3), nt=60)
    nsteps = 30
    per_elem = B.ns_state_bytes(1, wl.n_springs)
    cfg = {"ring-part": dict(device_state_budget=per_elem * 37, chunk_elems=13, ring_depth=3),
           "ring-all": dict(device_state_budget=0, chunk_elems=29, ring_depth=2),
           "zero-copy": dict(device_state_budget=per_elem * 37, stream_mode=B.NS_STREAM_ZERO_COPY)}[mode]
    o = oracle.Oracle.from_workload(wl)
    us, vs = [], []
    with B.Simulation(wl, surface_ring_steps=nsteps, **cfg) as sim:
        for _ in range(nsteps):
            o.step()
            us.append(o.u[wl.mesh.surf].copy())
            vs.append(o.v[wl.mesh.surf].copy())
        sim.advance(nsteps)
        s = sim.surface(1, nsteps)
        th, _ = sim.state()
        st = sim.stats()
    assert st["streamed_elems"] == wl.mesh.n_elems - (0 if mode == "ring-all" else 37)
    assert st["h2d_bytes"] >= nsteps * st["streamed_elems"] * per_elem
    assert rel(s["u"], np.array(us)) <= 1e-6
    assert rel(s["v"], np.array(vs)) <= 1e-6
    assert np.mean(th["mode"] == o.th["mode"]) > 0.999 and np.mean(th["dir"] == o.th["dir"]) > 0.999
    assert (o.th["mode"] == 1).mean() > 0.01


def test_main_motion_column_matches_oracle():
    """A 3 x 3 x 52 hexahedron column of the single large model (2,808 elements, 150
    springs per point, dt 0.005 s) driven by a full-length record through its strong
    motion: the timed window of the benchmark starts after the S waves have crossed the
    bedrock and the deepest soft layer (synth.lead_in_steps), and this run goes 40 steps
    past that.  The oracle (OpenMP build, all host cores) and the benchmark's solver form
    (flexible FP64 CG with the FP32 inner solve, started from zero) both solve to 1e-12,
    where the answer no longer depends on the stopping tolerance; springs must have
    reversed both on the skeleton and on Masing branches.  With both sides at the
    paper's 1e-8 the records differ by the tolerance's own effect, reported here."""
    wl = synth.large_single_model(column=(40, 40, 3, 3))
    wl.wave = synth.main_motion_record()
    nsteps = synth.lead_in_steps(wl.dt) + 40
    surf = wl.mesh.surf
    oracle.threads(0)

    def run_oracle(tol, track):
        o = oracle.Oracle.from_workload(wl, tol=tol, x0_prev=False, omp=True)
        us, vs = [], []
        skel = branch = 0
        prev_mode, prev_gR = o.th["mode"].copy(), o.th["gR"].copy()
        for _ in range(nsteps):
            o.step()
            us.append(o.u[surf].copy())
            vs.append(o.v[surf].copy())
            if track:
                mode, gR = o.th["mode"], o.th["gR"]
                skel += int(((prev_mode == 0) & (mode == 1)).sum())
                branch += int(((prev_mode == 1) & (mode == 1) & (gR != prev_gR)).sum())
                prev_mode, prev_gR = mode.copy(), gR.copy()
        return o, np.array(us), np.array(vs), skel, branch

    o, us, vs, skel, branch = run_oracle(1e-12, True)
    assert skel > 0 and branch > 0, (skel, branch)
    with B.Simulation(wl, surface_ring_steps=nsteps, precision=B.NS_PREC_FP64_IR, x0_prev=0, cg_tol=1e-12) as sim:
        sim.advance(nsteps)
        s = sim.surface(1, nsteps)
        th, _ = sim.state()
        st = sim.stats()
    eu, ev = rel(s["u"], us), rel(s["v"], vs)
    print("main-motion column, both at 1e-12: u %.2e v %.2e; reversals skeleton %d branch %d" % (eu, ev, skel, branch))
    assert eu <= 1e-6 and ev <= 1e-6
    assert np.mean(th["mode"] == o.th["mode"]) > 0.999 and np.mean(th["dir"] == o.th["dir"]) > 0.999
    assert st["spring_reversals"] > 0
    # both at the paper's tolerance 1e-8 (plain FP64 PCG on the GPU): the difference is the
    # stopping tolerance's own effect on a path-dependent history, reported
    _, us8, vs8, _, _ = run_oracle(1e-8, False)
    with B.Simulation(wl, surface_ring_steps=nsteps, precision=B.NS_PREC_FP64, x0_prev=0, cg_tol=1e-8) as sim:
        sim.advance(nsteps)
        s8 = sim.surface(1, nsteps)
    print("main-motion column, both at 1e-8: u %.2e v %.2e; oracle 1e-8 vs 1e-12: u %.2e v %.2e" % (
        rel(s8["u"], us8), rel(s8["v"], vs8), rel(us8, us), rel(vs8, vs)))
    assert rel(s8["u"], us8) <= 1e-3 and rel(s8["v"], vs8) <= 1e-3


@pytest.mark.parametrize("precision", [B.NS_PREC_FP64_IR, B.NS_PREC_FP64_IR16])
def test_local_gather_operator_equals_direct(precision):
    """The FP32 inner operator gathering each block's distinct nodes into shared memory
    (local connectivity, shared-memory force sums, one global atomic per node) computes what
    the per-element gathers compute: both solve to 1e-12, so the records agree to the
    rounding of the FP32 sums' order; and against the oracle at 1e-8."""
    wl = small(dims=(6, 5, 4), nt=60)  # 720 elements: two full blocks of 256 and a ragged one
    out = []
    for lg in (0, 1):
        with B.Simulation(wl, surface_ring_steps=30, precision=precision, local_gather=lg, cg_tol=1e-12,
                          x0_prev=0) as sim:
            sim.advance(30)
            out.append(sim.surface(1, 30)["v"])
    assert rel(out[1], out[0]) <= 1e-9
    o = oracle.Oracle.from_workload(wl, x0_prev=False)
    vs = []
    for _ in range(30):
        o.step()
        vs.append(o.v[wl.mesh.surf].copy())
    with B.Simulation(wl, surface_ring_steps=30, precision=precision, local_gather=1, x0_prev=0) as sim:
        sim.advance(30)
        assert rel(sim.surface(1, 30)["v"], np.array(vs)) <= 1e-6
