"""Host logic of bench.py's CPU baselines (no GPU): the bounded oracle sample and
the all-cores run of it in spawned processes."""
import bench
import labfm_inputs as li


def test_oracle_sample_counts_its_node_evaluations():
    ns = li.tgv_lattice(32, m=4, h_over_s=1.7, jitter=0.3, seed=1)
    sample = bench.OracleSample(ns, rows=64, seed=3)
    assert sample.n == 64 and len(sample.rows) == 64
    sample.step()  # four eq. icns evaluations at the 64 rows
    assert "64 random nodes" in sample.describe()


def test_oracle_all_cores_spawns_and_times():
    value, wall = bench.oracle_all_cores(32, reps=1, cores=2, rows=64)
    assert value > 0 and wall > 0


def test_oracle_all_cores_reports_a_worker_failure():
    import pytest
    with pytest.raises(RuntimeError, match="oracle worker failed"):
        bench.oracle_all_cores(32, reps=1, cores=2, rows=-1)
