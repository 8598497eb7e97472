"""Batched members: several independent cases of the method in one context, advanced by
the same launches, each with its own CG -- either members sharing one mesh (its
connectivity and geometry stored once, Alg. 4's problem sets on one mesh) or the
disjoint union of the members' meshes.  A member's result must not depend on the
others: every member of the batch matches the same case run alone (both sides stopping
CG at 1e-12, where the answer no longer depends on the stopping point, so only summation
order separates them), and one member matches the FP64 oracle at the stated 1e-6."""
import numpy as np
import pytest

import oracle
from paper_2604_02755_gb300 import binding as B
from paper_2604_02755_gb300 import build, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    B.lib()


def ensemble(M=3, nt=200):
    # 3 x 2 x 12 hexahedra of 4 m (48 m deep, soil over bedrock at 40 m), 10 springs
    return synth.ensemble_members(M=M, nt=nt, dims=(3, 2, 12), n_springs=10)


@pytest.mark.parametrize("precision,x0_prev,shared", [(B.NS_PREC_FP64, 1, True), (B.NS_PREC_FP64_IR, 1, True),
                                                     (B.NS_PREC_FP64_IR16, 1, True), (B.NS_PREC_FP64, 0, True),
                                                     (B.NS_PREC_FP64_IR, 0, True), (B.NS_PREC_FP64_IR, 1, False),
                                                     (B.NS_PREC_FP64, 0, False)])
def test_members_match_their_runs_alone(precision, x0_prev, shared):
    ens = ensemble()
    nsteps = 30
    with B.BatchSimulation(ens, shared=shared, surface_ring_steps=nsteps, precision=precision, cg_tol=1e-12,
                           x0_prev=x0_prev) as bs:
        bs.advance(nsteps)
        got = [bs.member_surface(m, 1, nsteps) for m in range(bs.M)]
        its = bs.member_iters()
        th_all, _ = bs.state()
    E = ens.mesh.n_elems
    for m in range(len(ens.members)):
        with B.Simulation(ens.member(m), surface_ring_steps=nsteps, precision=precision, cg_tol=1e-12,
                          x0_prev=x0_prev) as sim:
            sim.advance(nsteps)
            alone = sim.surface(1, nsteps)
            th, _ = sim.state()
            it = sim.stats()["cg_iters_last"]
        assert rel(got[m]["u"], alone["u"]) <= 1e-9, m
        assert rel(got[m]["v"], alone["v"]) <= 1e-9, m
        assert abs(int(its[m]) - it) <= 1
        assert np.array_equal(th_all["mode"][m * E:(m + 1) * E], th["mode"])
    # the members are different cases
    assert rel(got[0]["u"], got[1]["u"]) > 1e-3


@pytest.mark.parametrize("shared", [True, False])
def test_member_matches_oracle(shared):
    """Both sides at CG tolerance 1e-12: in these first steps of the record the surface
    moves by ~1e-7 m and the oracle alone changes by 2.9e-5 (relative L2) between
    tolerances 1e-8 and 1e-12, so only the tolerance-independent answer is compared."""
    ens = ensemble()
    nsteps = 30
    with B.BatchSimulation(ens, shared=shared, surface_ring_steps=nsteps, precision=B.NS_PREC_FP64_IR,
                           cg_tol=1e-12) as bs:
        bs.advance(nsteps)
        got = bs.member_surface(2, 1, nsteps)
    o = oracle.Oracle.from_workload(ens.member(2), tol=1e-12)
    us, vs = [], []
    for _ in range(nsteps):
        o.step()
        us.append(o.u[ens.mesh.surf].copy())
        vs.append(o.v[ens.mesh.surf].copy())
    assert rel(got["u"], np.array(us)) <= 1e-6
    assert rel(got["v"], np.array(vs)) <= 1e-6


def test_member_validation():
    ens = ensemble(M=2, nt=200)
    U = synth.union_of_copies(ens.mesh, 2, n_materials=2)
    cfg = B.ns_config_default(n_springs=10, dt=ens.dt)
    ctx = B.ns_create(cfg)
    try:
        B.ns_upload_mesh(ctx, U.mesh.xyz, U.mesh.conn, U.mesh.mat)
        B.ns_set_materials(ctx, ens.members[0] + ens.members[1])
        B.ns_set_boundary(ctx, U.mesh.faces, U.mesh.face_elem, U.mesh.face_kind, U.mesh.surf)
        bad = U.node_off.copy()
        bad[1] -= 1  # the last node of copy 0 assigned to copy 1
        with pytest.raises(B.NsError) as ei:
            B.ns_set_members(ctx, U.elem_off, bad)
        assert ei.value.code == -5  # NS_ERR_BAD_MESH
        with pytest.raises(B.NsError):
            B.ns_set_members(ctx, U.elem_off[:-1], U.node_off[:-1])  # does not cover the mesh
        B.ns_set_members(ctx, U.elem_off, U.node_off)
        B.ns_set_ground_motion(ctx, ens.waves[0], ens.dt)
        with pytest.raises(B.NsError):
            B.ns_set_member_ground_motion(ctx, 2, ens.waves[1], ens.dt)  # no member 2
        with pytest.raises(B.NsError):
            B.ns_set_member_ground_motion(ctx, 1, ens.waves[1][:-1], ens.dt)  # other length
        B.ns_set_member_ground_motion(ctx, 1, ens.waves[1], ens.dt)
        B.ns_advance(ctx, 2)
        assert B.ns_get_member_iters(ctx, 2).min() > 0
    finally:
        B.ns_destroy(ctx)


def test_shared_mesh_equals_disjoint_union():
    """Members on one stored mesh compute what the disjoint union of their meshes computes:
    the same spring states and, both at 1e-12, the same records to summation order."""
    ens = ensemble(M=4)
    nsteps = 25
    out = []
    for shared in (True, False):
        with B.BatchSimulation(ens, shared=shared, surface_ring_steps=nsteps, precision=B.NS_PREC_FP64_IR,
                               cg_tol=1e-12, x0_prev=0) as bs:
            bs.advance(nsteps)
            out.append((bs.surface(1, nsteps)["v"], bs.state()[0], bs.member_iters()))
    assert rel(out[0][0], out[1][0]) <= 1e-9
    assert np.mean(out[0][1]["mode"] == out[1][1]["mode"]) > 0.999
    assert np.abs(out[0][2].astype(int) - out[1][2].astype(int)).max() <= 1


def test_shared_mesh_validation():
    ens = ensemble(M=2, nt=200)
    with pytest.raises(B.NsError) as ei:  # members of a shared mesh need the atomic scatter
        B.ns_create(B.ns_config_default(shared_members=2, scatter=B.NS_SCATTER_COLOUR))
    assert ei.value.code == -1
    ctx = B.ns_create(B.ns_config_default(n_springs=10, dt=ens.dt, shared_members=2))
    try:
        m = ens.mesh
        B.ns_upload_mesh(ctx, m.xyz, m.conn, m.mat)
        with pytest.raises(B.NsError):  # two members need four material rows
            B.ns_set_materials(ctx, ens.members[0])
        B.ns_set_materials(ctx, ens.members[0] + ens.members[1])
        B.ns_set_boundary(ctx, m.faces, m.face_elem, m.face_kind, m.surf)
        with pytest.raises(B.NsError) as ei:  # the members are already set
            B.ns_set_members(ctx, [0, m.n_elems, 2 * m.n_elems], [0, m.n_nodes, 2 * m.n_nodes])
        assert ei.value.code == -8
        B.ns_set_ground_motion(ctx, ens.waves[0], ens.dt)
        B.ns_set_member_ground_motion(ctx, 1, ens.waves[1], ens.dt)
        B.ns_advance(ctx, 2)
        assert B.ns_get_member_iters(ctx, 2).min() > 0
    finally:
        B.ns_destroy(ctx)
