"""Host-side logic of bench.py that needs no GPU: the workload recipes, the
recorded-traffic lookup, the roofline denominators and the oracle timing
used for the CPU baseline (both generators)."""
import json
import os

import numpy as np
import pytest

import bench
import oracle.mt as omt
from paper_1501_07701_gb300 import workloads


def test_uneven_workload_recipe():
    w, desc = bench.workload("uneven", 0)
    assert w["mexp"] == 11213 and w["seeds"].size == 10000
    assert np.array_equal(w["seeds"], np.arange(10000, dtype=np.uint32))
    counts = w["counts"]
    assert counts.min() >= 1 << 10 and counts.max() < 1 << 22
    assert int(counts.sum()) == 5121292474          # the figure the bench reports
    assert "10000" in desc and "11213" in desc


def test_workload_overrides():
    w, desc = bench.workload("uneven", 0, mexp=3217)
    assert w["mexp"] == 3217 and "3217" in desc
    w, desc = bench.workload("equal", 0, streams=8, count=100, generator="original-MT p 3217")
    assert w["seeds"].size == 8 and np.all(w["counts"] == 100) and "original-MT" in desc
    w, _ = bench.workload("uneven", 0, streams=5, param_sets=3)
    assert w["seeds"].size == 5 and w["param_seeds"] is not None
    assert len(set(int(k) for k in w["param_seeds"])) == 3
    with pytest.raises(SystemExit):
        bench.workload("nosuch", 0)


def test_ranks_get_distinct_seeds():
    a, _ = bench.workload("equal", 0, streams=16, count=4)
    b, _ = bench.workload("equal", 1, streams=16, count=4)
    assert not set(a["seeds"].tolist()) & set(b["seeds"].tolist())


def test_recorded_traffic_matches_the_current_source():
    t = bench.recorded_traffic("mtgp_fast_kernel", "uneven")
    assert t is not None, "profiles/fast_kernel_uneven_traffic.md was taken on another kernel source"
    w, _ = bench.workload("uneven", 0)
    alg = 4.0 * int(w["counts"].sum()) + 8.0 * 351 * 10000
    assert 0.99 * alg < t <= alg                    # no re-reads: traffic within 1 % of algorithmic
    assert bench.recorded_traffic("mtgp_fast_kernel", "equal") is None


def test_hbm_peak_reads_the_measured_file():
    peak, src = bench.hbm_peak()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path) and json.load(open(path)).get("hbm_gbs"):
        assert src == "measured" and peak == json.load(open(path))["hbm_gbs"]
    else:
        assert (peak, src) == (6800.0, "fallback")


@pytest.mark.parametrize("generator", ["mtgp", "mt"])
def test_oracle_rate_counts_whole_streams(generator):
    w, _ = bench.workload("uneven", 0, streams=40)
    mt_params = omt.params_generate(3217, workloads.PARAM_SEED) if generator == "mt" else None
    rate, numbers, secs, streams = bench.oracle_rate(w, 0.2, 2, max_batch=1 << 22, mt_params=mt_params)
    assert rate > 0 and secs > 0 and 1 <= streams <= 40
    order = np.random.default_rng(0).permutation(40)[:streams]
    assert numbers == int(w["counts"][order].sum())


def test_split_piece_specs():
    total, sms = 5121292474, 152
    assert bench.split_piece("0", total, sms) == 0 and bench.split_piece("", total, sms) == 0
    assert bench.split_piece("auto", total, sms) == -(-total // (sms * 16)) == 2105795
    assert bench.split_piece("auto48", total, sms) == -(-total // (sms * 48))
    assert bench.split_piece("16384", total, sms) == 16384
    assert bench.split_piece("10", total, sms) == 64          # the smallest piece the library takes
    assert bench.split_piece("auto48", 1000, sms) == 64
