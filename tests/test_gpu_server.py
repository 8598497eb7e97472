"""Served ensemble (include/ns_server.h): cases of uneven size submitted while others
run are admitted as slots and memory free up, their kernels overlap on the device, and
each result is the same as the case run alone -- bit for bit with the deterministic
(colour) scatter, which leaves summation order as the only freedom and fixes it."""
import numpy as np
import pytest

from paper_2604_02755_gb300 import binding as B
from paper_2604_02755_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    B.lib()


def case(dims, S, seed, nt=120):
    m = synth.kuhn_box(*dims, 10.0 * dims[0], 10.0 * dims[1], 5.0 * dims[2], layer_depths=(20.0,), jitter=0.1,
                       seed=seed)
    w = synth.band_limited_wave(seed, nt + 1, 0.005)
    mats = [synth.soil(1700.0, 120.0 + 20 * seed, 5e-4, 0.20, 0.02), synth.soil(2000.0, 600.0, 1e-2, 0.20, 0.02)]
    return synth.Workload("case %d" % seed, m, mats, S, 0.005, nt, w)


CASES = [((3, 2, 8), 10, 1, B.NS_PREC_FP64_IR), ((4, 3, 8), 20, 2, B.NS_PREC_FP64),
         ((2, 2, 10), 15, 3, B.NS_PREC_FP64_IR16), ((5, 2, 8), 10, 4, B.NS_PREC_FP64_IR)]
NSTEPS = 25


def alone(wl, prec):
    with B.Simulation(wl, surface_ring_steps=NSTEPS, precision=prec, scatter=B.NS_SCATTER_COLOUR) as sim:
        sim.advance(NSTEPS)
        return sim.surface(1, NSTEPS)


def test_results_in_the_mix_equal_results_alone():
    wls = [(case(d, S, seed), prec) for d, S, seed, prec in CASES]
    ref = [alone(wl, prec) for wl, prec in wls]
    with B.Server(max_active=4, quantum_steps=5) as srv:
        ids = [srv.submit(wl, NSTEPS, precision=prec, scatter=B.NS_SCATTER_COLOUR) for wl, prec in wls]
        st = [srv.wait(i, 600) for i in ids]
        got = [srv.result(i) for i in ids]
    for k in range(len(wls)):
        assert st[k]["state"] == B.NS_CASE_DONE and st[k]["error"] == 0
        for f in ("u", "v", "a"):
            assert np.array_equal(got[k][f], ref[k][f]), (k, f)
    # they were in flight together
    assert max(s["t_admit"] for s in st) < min(s["t_done"] for s in st)


def test_admission_waits_for_memory_and_streams_when_it_must():
    wls = [case((3, 2, 8), 10, s) for s in (5, 6, 7)]
    dev, state, dstr = B.ns_case_bytes(wls[0], NSTEPS, scatter=B.NS_SCATTER_COLOUR)
    ref = [alone(wl, B.NS_PREC_FP64) for wl in wls]
    # room for one resident case at a time: the others queue and follow one by one
    with B.Server(device_budget=int(dev * 1.5), max_active=4, quantum_steps=5) as srv:
        ids = [srv.submit(wl, NSTEPS, scatter=B.NS_SCATTER_COLOUR) for wl in wls]
        st = [srv.wait(i, 600) for i in ids]
        got = [srv.result(i)["v"] for i in ids]
    for k in range(3):
        assert np.array_equal(got[k], ref[k]["v"])
        assert st[k]["streamed"] == 0
    for k in range(1, 3):
        assert st[k]["t_admit"] >= st[k - 1]["t_done"]
    # too little device memory for a resident state, enough pinned host memory: streamed
    # (through a ring of three 32-element chunks)
    dev, state, dstr = B.ns_case_bytes(wls[0], NSTEPS, scatter=B.NS_SCATTER_COLOUR, chunk_elems=32, ring_depth=3)
    budget = (dstr + dev) // 2
    assert dstr < budget < dev
    with B.Server(device_budget=budget, pinned_budget=4 * state, max_active=2, quantum_steps=5) as srv:
        i = srv.submit(wls[0], NSTEPS, scatter=B.NS_SCATTER_COLOUR, chunk_elems=32, ring_depth=3)
        s = srv.wait(i, 600)
        v = srv.result(i)["v"]
        assert s["streamed"] == 1 and s["state"] == B.NS_CASE_DONE
    assert np.array_equal(v, ref[0]["v"])
    # a case that fits neither way is refused at submission
    with B.Server(device_budget=dstr // 2, pinned_budget=0, max_active=1) as srv:
        with pytest.raises(B.NsError) as ei:
            srv.submit(wls[0], NSTEPS)
        assert ei.value.code == -2


def test_served_case_matches_oracle():
    """Cases run through the server in a mix of four (atomic scatter, their kernels
    overlapping on the device) against the FP64 oracle run on each case alone."""
    import oracle
    n = 60
    wls = [(case(d, S, seed), prec) for d, S, seed, prec in CASES]
    with B.Server(max_active=4, quantum_steps=7) as srv:
        ids = [srv.submit(wl, n, precision=prec) for wl, prec in wls]
        st = [srv.wait(i, 600) for i in ids]
        got = [srv.result(i) for i in ids]
    assert max(s["t_admit"] for s in st) < min(s["t_done"] for s in st)
    for k in (0, 1, 2):
        wl = wls[k][0]
        o = oracle.Oracle.from_workload(wl)
        us, vs = [], []
        for _ in range(n):
            o.step()
            us.append(o.u[wl.mesh.surf].copy())
            vs.append(o.v[wl.mesh.surf].copy())
        for f, ref in (("u", np.array(us)), ("v", np.array(vs))):
            err = np.linalg.norm(got[k][f] - ref) / np.linalg.norm(ref)
            assert err <= 1e-6, (k, f, err)


def test_batched_serving_matches_alone_and_oracle():
    """Continuous batching (batch = 1): cases of one solver class with different meshes and
    springs per point run as the members of one batched context, re-formed whenever a case
    arrives or finishes; each record equals the case run alone (both solving to 1e-12, the
    atomic sums leaving rounding only: 1e-9) and the FP64 oracle (1e-6)."""
    import time

    import oracle
    spec = [((3, 2, 8), 10, 1, 110), ((4, 3, 8), 20, 2, 40), ((2, 2, 10), 15, 3, 55), ((5, 2, 8), 12, 4, 25)]
    wls = [case(d, S, seed, nt=160) for d, S, seed, n in spec]  # 0.8 s records (shorter ones band-pass to zero)
    steps = [n for *_, n in spec]
    kw = dict(precision=B.NS_PREC_FP64_IR, cg_tol=1e-12)
    with B.Server(max_active=4, quantum_steps=5, batch=1) as srv:
        ids = [srv.submit(wls[0], steps[0], **kw)]
        time.sleep(0.2)  # the others arrive while the first one runs
        ids += [srv.submit(w, n, **kw) for w, n in zip(wls[1:], steps[1:])]
        st = [srv.wait(i, 600) for i in ids]
        got = [srv.result(i) for i in ids]
    assert all(s["state"] == B.NS_CASE_DONE and s["error"] == 0 for s in st)
    # the longest case saw the batch re-formed as the others joined (and left)
    assert st[0]["batches"] >= 2, st[0]
    for k, (wl, n) in enumerate(zip(wls, steps)):
        with B.Simulation(wl, surface_ring_steps=n, **kw) as sim:
            sim.advance(n)
            ref = sim.surface(1, n)
        for f in ("u", "v"):
            err = np.linalg.norm(got[k][f] - ref[f]) / np.linalg.norm(ref[f])
            assert err <= 1e-9, (k, f, err)
    wl, n = wls[1], steps[1]
    o = oracle.Oracle.from_workload(wl, tol=1e-12)
    vs = []
    for _ in range(n):
        o.step()
        vs.append(o.v[wl.mesh.surf].copy())
    err = np.linalg.norm(got[1]["v"] - np.array(vs)) / np.linalg.norm(np.array(vs))
    assert err <= 1e-6, err


def test_member_springs_validation():
    """Per-member springs: after the members, before the first step, all state resident."""
    wls = [case((3, 2, 8), 10, 1), case((3, 2, 8), 10, 2)]
    U = synth.union_of_copies(wls[0].mesh, 2, n_materials=2)
    ctx = B.ns_create(B.ns_config_default(n_springs=10, dt=0.005))
    try:
        B.ns_upload_mesh(ctx, U.mesh.xyz, U.mesh.conn, U.mesh.mat)
        B.ns_set_materials(ctx, wls[0].materials + wls[1].materials)
        B.ns_set_boundary(ctx, U.mesh.faces, U.mesh.face_elem, U.mesh.face_kind, U.mesh.surf)
        with pytest.raises(B.NsError):  # no members yet
            B.ns_set_member_springs(ctx, [10, 20])
        B.ns_set_members(ctx, U.elem_off, U.node_off)
        with pytest.raises(B.NsError):  # too few springs
            B.ns_set_member_springs(ctx, [10, 4])
        B.ns_set_member_springs(ctx, [10, 20])
        B.ns_set_ground_motion(ctx, wls[0].wave, 0.005)
        B.ns_advance(ctx, 3)
        with pytest.raises(B.NsError):  # set once
            B.ns_set_member_springs(ctx, [10, 20])
        with pytest.raises(B.NsError):  # the spring state of mixed members is not readable
            B.ns_read_state(ctx, 0, 1, 10)
    finally:
        B.ns_destroy(ctx)
