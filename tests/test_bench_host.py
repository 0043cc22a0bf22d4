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


def test_clock_summary_separates_the_timed_window(tmp_path):
    # nvidia-smi lines (timestamp first) are summarised over the sampler's lifetime and,
    # separately, over the samples inside the timed window
    import datetime
    import time
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.path = str(tmp_path / "clocks.csv")
    cs.keep = True
    cs.proc = object()
    now = time.time()
    with open(cs.path, "w") as f:
        for k in range(5):
            t = datetime.datetime.fromtimestamp(now + 0.1 * k).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
            cap = "Active" if k == 4 else "Not Active"
            f.write(f"{t}, 0, {2070 - k}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {cap}\n")
        f.write("garbage line\n")
    out = cs.summary(window=(now + 0.05, now + 0.35))
    assert out["samples"] == 5 and out["sm_max_mhz"] == 2070.0 and out["reasons"] == ["sw_power_cap"]
    tw = out["timed_window"]
    assert tw["samples"] == 3 and tw["sm_mhz"] == 2068.0 and tw["reasons"] == []
