"""Element and node numbering of the synthetic meshes (Morton order of centroids, or a
seeded shuffle that defeats the operator's gather locality).  A renumbered mesh is the
same mesh: the same tetrahedra, the same surface points in the same order, faces owned by
elements that contain them; and the method's answer does not depend on the numbering
(the oracle's surface response agrees to summation-order rounding)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2604_02755_gb300 import synth


def mesh():
    return synth.kuhn_box(4, 3, 3, 40.0, 30.0, 30.0, layer_depths=(15.0,), jitter=0.1, seed=2)


@pytest.mark.parametrize("how", ["morton", "shuffled"])
def test_renumbered_mesh_is_the_same_mesh(how):
    m = mesh()
    r = synth.renumber(m, how, seed=1)
    assert r.n_elems == m.n_elems and r.n_nodes == m.n_nodes
    # a permutation of nodes and elements, not a different mesh
    assert sorted(np.unique(r.conn).tolist()) == list(range(r.n_nodes))
    key = lambda mm: np.sort(np.round(mm.xyz[mm.conn].reshape(mm.n_elems, -1), 9), axis=0)
    assert np.array_equal(key(m), key(r))
    mats = lambda mm: sorted(zip(np.round(mm.xyz[mm.conn[:, :4]].mean(axis=1), 9).tolist(), mm.mat.tolist()))
    assert mats(m) == mats(r)
    assert np.array_equal(m.xyz[m.surf], r.xyz[r.surf])
    assert np.all(np.diff(r.face_elem) >= 0)
    for f in range(len(r.faces)):
        assert set(r.faces[f]) <= set(r.conn[r.face_elem[f]])
    assert np.array_equal(np.sort(m.face_kind), np.sort(r.face_kind))
    if how == "shuffled":
        assert not np.array_equal(r.conn, m.conn)


def test_morton_keys_order_the_octants():
    # the eight corners of a cube: key bit 0 is x, bit 1 y, bit 2 z
    p = np.array([[x, y, z] for z in (0.0, 1.0) for y in (0.0, 1.0) for x in (0.0, 1.0)])
    k = synth.morton_keys(p)
    assert np.array_equal(np.argsort(k), np.arange(8))
    x = 0x1249249249249249  # 21 set bits of x at bit positions 0, 3, ..., 60
    assert int(k[1]) == x and int(k[2]) == x << 1 and int(k[4]) == x << 2 and int(k[7]) == (1 << 63) - 1


@pytest.mark.parametrize("how", ["morton", "shuffled"])
def test_oracle_answer_does_not_depend_on_numbering(how):
    m = mesh()
    w = synth.band_limited_wave(5, 201, 0.01, peak=3.0)  # long enough to hold the 0.1-2.5 Hz band
    base = synth.Workload("numbering", m, synth.two_layer_materials(0.02), 10, 0.01, 200, w)
    alt = dataclasses.replace(base, mesh=synth.renumber(m, how, seed=3))
    out = []
    for wl in (base, alt):
        o = oracle.Oracle.from_workload(wl, tol=1e-13)
        for _ in range(8):
            o.step()
        out.append(o.u[wl.mesh.surf].copy())
    scale = np.max(np.abs(out[0]))
    assert scale > 0
    assert np.max(np.abs(out[0] - out[1])) <= 1e-9 * scale
