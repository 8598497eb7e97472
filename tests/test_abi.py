"""The C-ABI library builds, loads, exports every entry point that the headers under
include/ declare, and its host-only helpers agree with the oracle's independent
re-derivations (no device work)."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2604_02755_gb300 import binding, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return binding.lib()


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(ns_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert sorted(binding.EXPORTED) == names


def test_spring_directions_match_oracle():
    for S in (5, 10, 50, 150):
        qg, wg = binding.ns_spring_directions(S)
        qo, wo = oracle.spring_dirs(S)
        assert wg == wo
        assert np.abs(qg - qo).max() <= 1e-12 * np.abs(qo).max()
    with pytest.raises(binding.NsError):
        binding.ns_spring_directions(4)


def test_colouring_bit_exact_with_oracle():
    m = synth.kuhn_box(6, 5, 4, 60.0, 50.0, 40.0, jitter=0.1, seed=3)
    cg, ncg = binding.ns_colour_elements(m.conn, m.n_nodes)
    co, nco = oracle.colouring(m.conn, m.n_nodes)
    assert ncg == nco
    assert np.array_equal(cg, co)


def test_state_bytes_match_paper_sizing():
    assert binding.ns_state_bytes(1, 150) == 24000
    assert binding.ns_state_bytes(7987200, 150) == 7987200 * 24000


def test_create_without_device_reports_an_error_code():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(binding.NsError) as ei:
        binding.ns_create(binding.ns_config_default())
    assert ei.value.code == -4


@pytest.mark.parametrize("bad", [dict(n_springs=3), dict(spring_tile_points=6), dict(spring_tile_points=2),
                                 dict(n_springs=150, spring_tile_points=256), dict(spring_tile_blocks=3),
                                 dict(precision=7), dict(stream_mode=2), dict(inner_max_iter=0),
                                 dict(inner_tol=0.0), dict(ring_depth=1)])
def test_invalid_config_rejected_before_device_use(bad):
    """Out-of-range settings are refused by ns_create before any device call: a spring
    tile that is not a multiple of 4 points or whose float pairs exceed 200 KB of shared
    memory, a register budget other than 1 or 4 blocks per SM, unknown enums, and so on."""
    with pytest.raises(binding.NsError) as ei:
        binding.ns_create(binding.ns_config_default(**bad))
    assert ei.value.code == -1


@pytest.mark.parametrize("dims", [(3, 2, 2), (6, 5, 4)])
def test_coarse_map_bit_exact_with_oracle(dims):
    """The two-level preconditioner's P2 -> P1 map (host code of the library) equals the
    oracle's independent derivation index for index."""
    m = synth.kuhn_box(*dims, 10.0 * dims[0], 10.0 * dims[1], 10.0 * dims[2], jitter=0.1, seed=4)
    cg, pg, ncg = binding.ns_coarse_map(m.conn, m.n_nodes)
    co, po, nco = oracle.coarse_map(m.conn, m.n_nodes)
    assert ncg == nco and np.array_equal(cg, co) and np.array_equal(pg, po)
    bad = m.conn.copy()
    bad[0, 4], bad[0, 5] = bad[0, 5], bad[0, 4]
    with pytest.raises(binding.NsError) as ei:
        binding.ns_coarse_map(bad, m.n_nodes)
    assert ei.value.code == -5


@pytest.mark.parametrize("bad", [dict(multigrid=1), dict(multigrid=2, precision=1),
                                 dict(multigrid=1, precision=1, coarse_max_iter=0),
                                 dict(multigrid=1, precision=1, coarse_tol=0.0)])
def test_invalid_multigrid_config_rejected(bad):
    """The two-level preconditioner needs a flexible solver form and sane coarse limits."""
    with pytest.raises(binding.NsError) as ei:
        binding.ns_create(binding.ns_config_default(**bad))
    assert ei.value.code == -1
