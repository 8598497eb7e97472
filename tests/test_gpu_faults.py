"""Failure handling made on the host, never by faulting the GPU:

  * the k-th pinned host allocation of a context fails (injected) and surfaces as
    NS_ERR_OOM_PINNED from the call that made it;
  * the k-th state-stream copy (a chunk's H2D or D2H of Alg. 3) fails before it is
    issued and surfaces as NS_ERR_CUDA from ns_advance; the context still answers and is
    destroyed cleanly;
  * a bounded host wait that runs out (a wait limit far below one step's device time)
    surfaces as NS_ERR_TIMEOUT; the device work it gave up on still completes and the
    context is destroyed cleanly;
  * CG reaching its iteration limit is NS_ERR_NOT_CONVERGED (tests/test_gpu_parity.py).
"""
import numpy as np
import pytest

from paper_2604_02755_gb300 import binding as B
from paper_2604_02755_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    B.lib()


def small(dims=(4, 3, 3), S=10, nt=40):
    m = synth.kuhn_box(*dims, 40.0, 30.0, 30.0, layer_depths=(15.0,), jitter=0.1, seed=5)
    return synth.Workload("small", m, synth.two_layer_materials(0.02), S, 0.01, nt,
                          synth.band_limited_wave(5, nt + 1, 0.01))


def test_injected_pinned_allocation_failure():
    wl = small()
    per_elem = B.ns_state_bytes(1, wl.n_springs)
    # ns_create makes two pinned allocations; the streamed state's six arrays come next
    with pytest.raises(B.NsError) as ei:
        B.Simulation(wl, device_state_budget=per_elem * 10, chunk_elems=16, fault_pinned_alloc=4)
    assert ei.value.code == -3 and "injected" in str(ei.value)
    # the same configuration without the fault runs
    with B.Simulation(wl, device_state_budget=per_elem * 10, chunk_elems=16) as sim:
        sim.advance(2)
    # the first allocation of ns_create itself
    with pytest.raises(B.NsError) as ei:
        B.Simulation(wl, fault_pinned_alloc=1)
    assert ei.value.code == -3


def test_injected_state_copy_failure():
    wl = small()
    per_elem = B.ns_state_bytes(1, wl.n_springs)
    n_streamed = wl.mesh.n_elems - 10
    chunks = -(-n_streamed // 16)
    k = 2 * chunks + 3  # inside the second step's pipeline (each chunk: one H2D, one D2H)
    with B.Simulation(wl, device_state_budget=per_elem * 10, chunk_elems=16, ring_depth=3,
                      fault_state_copy=k) as sim:
        sim.advance(1)
        with pytest.raises(B.NsError) as ei:
            sim.advance(3)
        assert ei.value.code == -4 and "injected" in str(ei.value)
        st = sim.stats()
        assert st["steps"] == 1  # the failing step was not counted
        sim.nodal("u")  # the context still answers


def test_bounded_host_wait_times_out():
    wl = small(dims=(8, 8, 6), nt=40)
    with B.Simulation(wl, wait_timeout_s=1e-7, precision=B.NS_PREC_FP64_IR) as sim:
        with pytest.raises(B.NsError) as ei:
            sim.advance(20)
        assert ei.value.code == -7
    # a normal limit on the same model completes
    with B.Simulation(wl, precision=B.NS_PREC_FP64_IR) as sim:
        sim.advance(2)


def test_spring_counters():
    """The spring kernel's counts: every spring moves once the input reaches it, some
    reverse (hysteresis), and the counts reset with the statistics."""
    wl = small(nt=60)
    with B.Simulation(wl) as sim:
        sim.advance(30)
        st = sim.stats()
        n_spr = wl.mesh.n_elems * 4 * wl.n_springs
        assert 0 < st["spring_moved"] <= 30 * n_spr
        assert 0 < st["spring_reversals"] <= st["spring_moved"]
        assert 0 <= st["spring_fp64_roots"] <= st["spring_moved"]
        B.ns_reset_stats(sim.ctx)
        assert sim.stats()["spring_moved"] == 0
        sim.advance(1)
        st1 = sim.stats()
        assert 0 < st1["spring_moved"] <= n_spr
