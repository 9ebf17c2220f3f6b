"""Host-side helpers of the benchmark, on the CPU: the reduction of an ncu
launch list to per-kernel shares, kernel-name shortening, the whole-job value,
and the oracle's recorded counts and sampled solution."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

_HDR = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
        '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')


def _row(i, name, unit, value):
    return (f'"{i}","1","python3","h","{name}","1","13","(256, 1, 1)","(8, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","gpu__time_duration.sum","{unit}","{value}"\n')


def test_kernel_short_name():
    assert bench._kernel_short_name(
        "void pc::<unnamed>::k_rowprod_warp<pc::<unnamed>::GalSrc, 2>(int, const int *)") == \
        "k_rowprod_warp<GalSrc, 2>"
    assert bench._kernel_short_name("<unnamed>::k_check_finite(long, const double *, int *)") == \
        "k_check_finite"
    assert bench._kernel_short_name("pc::(anonymous namespace)::k_scan<int, int>(long, const int *)") == \
        "k_scan<int, int>"
    assert bench._kernel_short_name("void pc::<unnamed>::k_res_stream<float, (bool)0>(int)") == \
        "k_res_stream<float, (bool)0>"


def test_summarize_launches_shares(tmp_path, capsys):
    p = tmp_path / "launches.csv"
    p.write_text("==PROF== Connected to process 1\n" + _HDR +
                 _row(0, "pc::<unnamed>::k_a(int)", "ns", "1,000") +
                 _row(1, "pc::<unnamed>::k_b<float>(int)", "usecond", "3") +
                 _row(2, "pc::<unnamed>::k_a(int)", "ns", "1000") +
                 _row(3, "pc::<unnamed>::k_c(int)", "msecond", "0.005"))
    bench.summarize_launches(str(p))
    out = capsys.readouterr().out.splitlines()
    assert out[0].startswith("launches: 4 ") and "0.010 ms" in out[0]
    body = {ln.split()[0]: ln.split()[1:] for ln in out[2:]}
    # sorted by total time: k_c 5 us, k_b 3 us, k_a 2 us (two launches)
    assert [ln.split()[0] for ln in out[2:]] == ["k_c", "k_b<float>", "k_a"]
    assert body["k_a"] == ["2", "0.002", "20.00%"]
    assert body["k_c"] == ["1", "0.005", "50.00%"]


def test_job_value_counts_every_rank():
    # replicas: each of N ranks solves n unknowns; value = N n / slowest time
    assert bench.job_value(1000, 1, 500.0) == 2000.0
    assert bench.job_value(1000, 4, 500.0) == 8000.0


def test_oracle_counts_and_sample_error(tmp_path, monkeypatch):
    import json

    import numpy as np
    rec = {"C5-mid": {"resetups": 6, "cycles": 300, "wcycles": 14, "iters": 20, "n": 10,
                      "seconds": 1.0, "host": "h", "sample_idx": [1, 3], "sample_x": [2.0, -1.0]}}
    p = tmp_path / "solves.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "GOLDEN_SOLVES", str(p))
    c = bench.oracle_counts("C5")          # stands in through the same recipe
    assert c["from"] == "C5-mid" and c["builds"] == 7 and c["cycles"] == 300 and c["wcycles"] == 14
    assert bench.oracle_counts("C2") is None
    x = np.zeros(10); x[1], x[3] = 2.0, -1.0 + 1e-3
    e = bench.error_vs_recorded_oracle("C5-mid", x)
    assert abs(e["value"] - 1e-3 / np.sqrt(5.0)) < 1e-12
    assert bench.error_vs_recorded_oracle("C5", x) is None
