"""Host-side pieces of bench.py that run before any GPU work: the workload
table, the variant list and the description of every workload (a missing
key there would only show up in a GPU run)."""
from __future__ import annotations

import bench
from paper_1106_3678_gb300 import workloads as W


def test_variants_and_default_are_known_workloads():
    assert bench.DEFAULT in bench.WORKLOADS
    assert set(bench.VARIANTS) <= set(bench.WORKLOADS)
    assert len(set(bench.VARIANTS)) == len(bench.VARIANTS)
    assert bench.DEFAULT not in bench.VARIANTS


def test_every_workload_has_a_description():
    A = W.cd2d(4)
    for name, wl in bench.WORKLOADS.items():
        d = bench._variant_desc(name, wl, [(A, None, None)])
        assert isinstance(d, str) and d, name


def test_headline_conversion_count_is_set():
    # the reference arm converts its per-iteration time with this count
    assert bench.WORKLOADS[bench.DEFAULT]["iters"] > 0
    assert bench.NCU_DRAM_BYTES_PER_ITER is None or bench.NCU_DRAM_BYTES_PER_ITER > 0


def test_pairs_name_known_workloads_and_converged_rule():
    for name, base, key in bench.PAIRS:
        assert name in bench.WORKLOADS and base in bench.WORKLOADS and key.startswith("speedup")
    assert bench._converged({"flags": [0, 0], "true_relres": [1e-11, 9e-11]}, 1e-10) is True
    assert bench._converged({"flags": [0, 1], "true_relres": [1e-11, 9e-11]}, 1e-10) is False
    assert bench._converged({"flags": [0], "true_relres": [2e-10]}, 1e-10) is False
    assert bench._converged({"flags": [0], "true_relres_max": 5e-11}, 1e-10) is True


def test_fused_column_rule_mirrors_the_library_rule():
    # the rule documented with mlb_tuning.qd_fused in include/mlbicgstab.h
    assert bench._qd_rule(4, False) == 4 and bench._qd_rule(4, False, True) == 4
    assert bench._qd_rule(8, False) == 1 and bench._qd_rule(16, False) == 1
    assert bench._qd_rule(8, False, True) == 2 and bench._qd_rule(16, False, True) == 2
    assert bench._qd_rule(4, True) == 2 and bench._qd_rule(3, False) == 2
    assert bench._qd_rule(1, False) == 1 and bench._qd_rule(1, True) == 1
