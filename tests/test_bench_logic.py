"""Host logic of the benchmark and of the oracle's statistics (CPU only):
the byte model and roofline arithmetic, the per-workload table choice, the
serving trace, and the oracle's IsNeighbor count."""
import argparse
import importlib.util
import json
import os

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_roofline_closed_form(bench):
    wl = dict(bench.WORKLOADS["c2"])
    moves, walks, ms = 1_000_000, 10_000, 1.0
    roof = bench.roofline(wl, moves, walks, ms, None, {"loads_per_s": 5e11}, 1e12)
    # ALIAS: one 32-byte record + a 4-byte path entry per move; 12 B + a row pair per walk
    want = moves * 36 + walks * (12 + 36)
    assert roof["algorithmic_bytes_per_launch"] == want
    assert roof["achieved"] == pytest.approx(want / 1e-3 / 1e9, rel=1e-3)
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    assert roof["peak"] == pytest.approx(peak)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"], abs=1e-4)  # rounded to 4 places
    assert roof["frac_of_gather_ceiling"] == pytest.approx(2.0)
    # NAIVE with row records: one 16-byte record (one sector) per move, the source's row pair per walk
    wl1 = dict(bench.WORKLOADS["c1"])
    r1 = bench.roofline(wl1, moves, walks, ms, None, None, 1.0, records=True, kernel="walk_plain")
    assert r1["algorithmic_bytes_per_launch"] == int(moves * 36 + walks * (12 + 36))
    assert r1["kernel"] == "walk_plain"
    r0 = bench.roofline(wl1, moves, walks, ms, None, None, 1.0)
    assert r0["algorithmic_bytes_per_launch"] == int(moves * (36 + 32 + 4) + walks * 12)


def test_table_choice(bench):
    on = argparse.Namespace(paper_paths=False)
    off = argparse.Namespace(paper_paths=True)
    assert bench.tables_of(bench.WORKLOADS["c2"], on) == 0
    assert bench.table_names(bench.tables_of(bench.WORKLOADS["c3"], on)) == ["row_records", "neighbor_hash"]
    assert bench.table_names(bench.tables_of(bench.WORKLOADS["c4"], on)) == ["label_index"]
    for c in bench.WORKLOADS:
        assert bench.tables_of(bench.WORKLOADS[c], off) == 0
    # the flags are the library's
    import paper_2107_11983_gb300 as trw
    assert bench.TABLE_FLAGS == {"row_records": trw.PREP_ROW_RECORDS, "neighbor_hash": trw.PREP_NEIGHBOR_HASH,
                                 "label_index": trw.PREP_LABEL_INDEX}


def test_serve_trace_mix(bench):
    g = synth.rmat(10)
    t1, r1 = bench.serve_trace(g, 4000, 2000.0)
    t2, r2 = bench.serve_trace(g, 4000, 2000.0)
    assert np.array_equal(t1, t2) and len(r1) == len(r2) == 4000  # deterministic
    assert t1[0] == 0 and np.all(np.diff(t1) >= 0)
    assert abs(t1[-1] / 3999 - 1 / 2000.0) < 0.1 / 2000.0       # Poisson rate
    algos = np.array([r["algo"] for r in r1])
    assert abs(np.mean(algos == 2) - 0.90) < 0.02                # PPR share
    assert abs(np.mean(algos == 1) - 0.05) < 0.015
    assert abs(np.mean(algos == 3) - 0.05) < 0.015
    for r in r1:
        n = r["sources"].shape[0] * r.get("walks_per_source", 1)
        if r["algo"] == 2:
            assert 1000 <= n <= 100000 and r.get("endpoints")
        else:
            assert 10000 <= n <= 1000000 and r["max_len"] == 80


def test_oracle_deciding_checks():
    g = synth.rmat(9, seed=5)
    src = synth.vertex_sources(g.nv)
    flat = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, src, 30, 1, n2v_p=1.0, n2v_q=1.0)
    assert flat.stats["checks"] == 0                  # every class always accepted: no check decides
    assert flat.stats["attempts"] == flat.stats["moves"]
    biased = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, src, 30, 1, n2v_p=0.5, n2v_q=2.0)
    st = biased.stats
    assert 0 < st["checks"] < st["attempts"]
    # p=0.5, q=2: T_ret always, T_nb = 1/2, T_far = 1/4 of p* = 2; a check decides when the
    # dart falls in [2^30, 2^31), a quarter of the non-return attempts after the first step
    frac = st["checks"] / (st["attempts"] - len(src))
    assert 0.15 < frac < 0.26


def test_sampler_workloads(bench):
    import paper_2107_11983_gb300 as trw
    wl = dict(bench.WORKLOADS["c2"], sampler="its_guided")
    kw = bench.walk_kwargs(wl)
    assert kw == {"sampler": trw.SAMPLER_ITS, "max_weight": bench.SWEEP_BOUND}
    assert bench.SAMPLER_PREP == {"its": trw.PREP_ITS, "its_guided": trw.PREP_ITS_GUIDE, "rej": trw.PREP_REJ}
    r = bench.roofline(wl, 1000, 10, 1.0, None, None, 1.0)
    assert r["bytes_per_move"] == 68  # the cell's record, the answer's record, the path entry
    assert bench.roofline(dict(wl, sampler="rej"), 1000, 10, 1.0, None, None, 1.0) is None  # needs the oracle model
    cpu = {"model_bytes_per_move": 100.0}
    assert bench.roofline(dict(wl, sampler="rej"), 1000, 10, 1.0, cpu, None, 1.0)["bytes_per_move"] == 100.0
    assert bench.walk_kwargs(bench.WORKLOADS["c2"]) == {}


@pytest.mark.parametrize("config", ["c1", "c4"])
def test_reference_arm_line(config):
    """bench.py --impl reference: one JSON line with the contract's keys, the
    oracle timed on the host cores over a sample no larger than the batch; a
    workload it does not walk gives the one-line unavailable form."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", config,
                        "--steps", "2", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    if config == "c4":
        assert set(d) == {"impl", "unavailable"}
        return
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["metric"] == "walk steps/sec" and d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["value"] > 0
    assert d["config"]["workload"] == "deepwalk-rmat-s14"
    assert d["config"]["walks_per_step"] == 1 << 14  # the whole batch: smaller than the per-core sample
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert str(1 << 14) in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_traffic_scales_captured_bytes_per_move(bench, monkeypatch):
    """The bench's `traffic` is a committed capture's DRAM bytes per move times
    the moves of the timed launch, and null once the kernel source changed."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    key = "walk_persistent/deepwalk-weighted-alias-rmat-s22"
    e = rec[key]
    assert e["source_hash"] == bench.kernel_source_hash(), "traffic.json was captured from another kernel source"
    assert bench.ncu_traffic(key, e["moves"]) == e["dram_bytes"]
    assert bench.ncu_traffic(key, 2 * e["moves"]) == 2 * e["dram_bytes"]
    assert bench.ncu_traffic("walk_persistent/no-such-workload", 1000) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic(key, e["moves"]) is None
