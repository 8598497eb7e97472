"""The per-spring and per-element state sizes the paper prints (Sec. 2.1, 2.3)."""
import json
import os

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "state_sizing.json")))


def test_oracle_spring_state_matches_paper_sizes():
    assert oracle.SPRING_DTYPE.itemsize == GOLD["bytes_per_spring"]
    per_elem = oracle.SPRING_DTYPE.itemsize * GOLD["springs_per_point"] * GOLD["points_per_element"]
    assert per_elem == GOLD["bytes_per_element"]
    two_parts = GOLD["resident_partitions"] * GOLD["partition_elements"] * per_elem / 1e9
    assert abs(two_parts - GOLD["partition_gpu_increment_gb_approx"]) < 0.5
