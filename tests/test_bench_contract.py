"""The benchmark's reference arm (the CPU oracle on host cores) runs without a
GPU and prints the one-line JSON contract; the throughput model of Sec. V
reproduces the paper's Tables I and II."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-seconds", "1"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "Gbps" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["N"] == 2048 and d["config"]["L"] == 32 and d["config"]["workload"]


def _tables_1_2():
    lat, tp, k = {}, {}, None
    with open(os.path.join(ROOT, "tests", "golden", "adaptive_throughput_tables_1_2.txt")) as fh:
        for line in fh:
            f = line.split()
            if not f or f[0].startswith("#"):
                continue
            if f[0] == "k":
                k = float(f[1])
            elif f[0] == "latency":
                lat[int(f[1])] = float(f[2])
            else:
                tp[(int(f[1]), float(f[2]))] = float(f[3])
    return k, lat, tp


def test_adaptive_throughput_reproduces_table_2():
    """Eq. (tp) against the paper's own tables. The Fast-SSC latency is not
    printed; the 4.5 dB column, equal for both list sizes, gives it (the
    Fast-SSC pass almost never fails there). At each lower point one FER_F,
    solved from the L = 8 row and Table I's L = 8 latency, must then predict
    the L = 32 row from Table I's L = 32 latency."""
    sys.path.insert(0, ROOT)
    import bench
    k, lat, tp = _tables_1_2()
    lat_f = k / tp[(8, 4.5)]
    assert tp[(32, 4.5)] == tp[(8, 4.5)]
    for pays_both, tol in ((True, 0.02), (False, 0.10)):
        for db in (3.5, 4.0):
            cost8 = k / tp[(8, db)]
            fer_f = (cost8 - lat_f) / (lat[8] if pays_both else lat[8] - lat_f)
            assert 0.0 < fer_f < 1.0
            assert bench.adaptive_throughput(k, fer_f, lat_f, lat[8], pays_both) == pytest.approx(tp[(8, db)])
            pred = bench.adaptive_throughput(k, fer_f, lat_f, lat[32], pays_both)
            assert pred == pytest.approx(tp[(32, db)], rel=tol), (pays_both, db, pred)
    # the end points: no failures gives the Fast-SSC rate, all failures the list
    # rate (printed form) or the rate of both passes in a row
    assert bench.adaptive_throughput(k, 0.0, lat_f, lat[32]) == pytest.approx(k / lat_f)
    assert bench.adaptive_throughput(k, 1.0, lat_f, lat[32], False) == pytest.approx(k / lat[32])
    assert bench.adaptive_throughput(k, 1.0, lat_f, lat[32]) == pytest.approx(k / (lat_f + lat[32]))
    # and the list decoder alone at L = 32: 4.0 Mbps (Sec. VI-B)
    assert round(k / lat[32], 1) == 4.0


def test_metric_comparisons_fit_the_line_tail():
    """The bench line keeps its last blocks short: the FER sweep of both codes
    (60 points), the serving figures and the two batched-vs-plain pairs must
    fit in the final 3000 characters of the printed line."""
    sys.path.insert(0, ROOT)
    import bench
    rows = []
    for code, Ls in (("(1024,860)", (2, 4, 8, 32)), ("(2048,1723)", (8, 32))):
        for L in Ls:
            for dt in ("f32", "i8"):
                for eb in (3.5, 3.75, 4.0, 4.25, 4.5):
                    rows.append({"code": code, "L": L, "dtype": dt, "ebn0_db": eb, "frames": 1048576,
                                 "errors_fast": 123456, "errors_scl": 123457, "mcnemar_p": 0.123456789,
                                 "fer_match": True, "underpowered": False})
    fer = bench.compact_fer({"rows": rows})
    assert sum(len(v) for k, v in fer.items() if k.startswith("(")) == 60
    head = {"workload": "(2048,1723) CRC-32 L=32, one class, the plain form's 1048576 frames per GPU",
            "value": 3.123456789, "plain_value": 2.987654321, "ms_per_step": 567.891234, "plain_ms_per_step": 590.1234,
            "graph_replay": True, "results_equal_plain": True, "roofline": {"frac": 0.0412345, "plain_frac": 0.04}}
    tail = {"fer": fer,
            "serving": {"offered_frames_per_s": 200000.0, "requests": 1234, "frames": 1612345,
                        "p50_ms": 0.423456789, "p99_ms": 4.123456789, "info_gbps": 0.19123456789,
                        "p99_ms_by_frames": {"1-16": 1.123456789, "17-256": 2.123456789, "257-4096": 5.123456789}},
            "batched": {"value": 5.3123456789, "plain_value": 4.6312345678, "ms_per_step": 123.456789,
                        "plain_ms_per_step": 140.123456789, "plain_launches_per_step": 125,
                        "results_equal_plain": True},
            "batched_headline": bench.compact_headline(head)}
    text = json.dumps(tail)
    assert len(text) < 3000, len(text)
    assert bench.compact_headline(dict(head, value=None, roofline=None))["batched_over_plain"] is None
