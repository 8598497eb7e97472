"""Host side of the batched members: the union-of-copies mesh and the ensemble draws."""
import numpy as np

from paper_2604_02755_gb300 import synth


def test_union_of_copies_is_a_disjoint_union():
    ens = synth.ensemble_members(M=3, nt=5, dims=(3, 2, 12), n_springs=10)
    m = ens.mesh
    U = synth.union_of_copies(m, 3, n_materials=2)
    N, E, F = m.n_nodes, m.n_elems, m.faces.shape[0]
    assert list(U.elem_off) == [0, E, 2 * E, 3 * E] and list(U.node_off) == [0, N, 2 * N, 3 * N]
    for k in range(3):
        c = U.mesh.conn[k * E:(k + 1) * E]
        assert c.min() >= k * N and c.max() < (k + 1) * N  # no node shared between copies
        assert np.array_equal(c - k * N, m.conn)
        assert np.array_equal(U.mesh.mat[k * E:(k + 1) * E], m.mat + 2 * k)
        assert np.array_equal(U.mesh.xyz[k * N:(k + 1) * N], m.xyz)
        fe = U.mesh.face_elem[k * F:(k + 1) * F]
        assert fe.min() >= k * E and fe.max() < (k + 1) * E  # faces ordered by copy
        assert np.array_equal(U.mesh.faces[k * F:(k + 1) * F] - k * N, m.faces)
        assert np.array_equal(U.mesh.surf[k * len(m.surf):(k + 1) * len(m.surf)] - k * N, m.surf)


def test_ensemble_member_draws():
    ens = synth.ensemble_members(M=64, nt=1000, dims=(2, 2, 12))
    vs = np.array([mm[0]["vs"] for mm in ens.members])
    gr = np.array([mm[0]["gamma_ref"] for mm in ens.members])
    hr = np.array([mm[0]["rayleigh_h"] for mm in ens.members])
    assert vs.min() >= 100 and vs.max() <= 300 and vs.std() > 30
    assert gr.min() >= 1e-4 and gr.max() <= 1e-3
    assert hr.min() >= 0.01 and hr.max() <= 0.05
    assert all(mm[1]["vs"] == 600.0 for mm in ens.members)  # shared bedrock
    # independent inputs, each scaled to a 3 m/s^2 peak
    assert abs(np.corrcoef(ens.waves[0][:, 0], ens.waves[1][:, 0])[0, 1]) < 0.5
    assert np.allclose([np.abs(w).max(axis=0) for w in ens.waves], 3.0)


def test_case_bytes_accounting():
    from paper_2604_02755_gb300 import binding as B
    from paper_2604_02755_gb300 import build
    build.build()
    wl = synth.tiny_two_layer(nt=20)
    E = wl.mesh.n_elems
    dev, st, dstr = B.ns_case_bytes(wl, 20, precision=B.NS_PREC_FP64, chunk_elems=100)
    assert st == E * 4 * wl.n_springs * 40  # 40 B per spring, 4 points per element (Sec. 2.1)
    assert dev > st and dstr == dev - st + 3 * 100 * 4 * wl.n_springs * 40  # a ring of 3 chunks instead
    dev1, _, dstr1 = B.ns_case_bytes(wl, 20, precision=B.NS_PREC_FP64)
    assert dev1 == dev and dstr1 > dev  # 100,000-element chunks: the ring holds more than the state
    dev_ir, _, _ = B.ns_case_bytes(wl, 20, precision=B.NS_PREC_FP64_IR)
    dev_16, _, _ = B.ns_case_bytes(wl, 20, precision=B.NS_PREC_FP64_IR16)
    assert dev < dev_16 < dev_ir  # FP32 copy of D > FP16 copy > none
    dev_s, st_s, _ = B.ns_case_bytes(wl, 20, n_springs=150, precision=B.NS_PREC_FP64)
    assert st_s == 15 * st and dev_s - dev == st_s - st
