"""Host logic of bench.py that needs no GPU: the source digest that keeps a
profiled DRAM-traffic figure tied to the kernel code it was captured on, the
partition of a batch over ranks, and the reference arm's JSON line."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench

SRC = '''// header comment
__global__ void k(float *x, int n) {   /* a block
   comment */
    const char *s = "// not a comment";
    if (threadIdx.x < n) x[threadIdx.x] *= 2.f;
}
'''

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_comment_and_whitespace_edits_keep_the_digest():
    edited = SRC.replace("// header comment", "// another header\n// over two lines")
    edited = edited.replace("a block\n   comment", "reworded")
    edited = edited.replace("x[threadIdx.x] *= 2.f;", "x[threadIdx.x]   *=   2.f;   // doubled")
    assert bench.code_digest(edited) == bench.code_digest(SRC)


def test_code_edits_change_the_digest():
    assert bench.code_digest(SRC.replace("2.f", "3.f")) != bench.code_digest(SRC)
    assert bench.code_digest(SRC.replace("< n", "<= n")) != bench.code_digest(SRC)
    # comment markers inside a string literal are code
    assert bench.code_digest(SRC.replace('"// not a comment"', '"// changed"')) != bench.code_digest(SRC)


def test_profiled_traffic_scales_with_units_and_needs_the_captured_code(monkeypatch):
    assert bench.profiled_traffic("no such class", 10) is None
    rec = dict(bench.PROFILED_TRAFFIC["tc"])
    rec["sha256"] = bench.code_digest("".join(open(os.path.join(ROOT, f)).read() for f in rec["file"]))
    rec["bytes_per_unit"] = 1000.0
    monkeypatch.setitem(bench.PROFILED_TRAFFIC, "tc", rec)
    assert bench.profiled_traffic("tc", 7.5) == pytest.approx(7500.0)
    assert bench.profiled_traffic("tc", 0) is None
    rec2 = dict(rec, sha256="0" * 64)     # the kernel changed since the capture
    monkeypatch.setitem(bench.PROFILED_TRAFFIC, "tc", rec2)
    assert bench.profiled_traffic("tc", 7.5) is None


def test_partition_is_greedy_by_work_and_covers_every_system():
    works = [5.0, 9.0, 1.0, 7.0, 3.0, 3.0]
    parts = bench.partition(works, 2)
    assert sorted(i for p in parts for i in p) == list(range(len(works)))
    # LPT: 9 -> r0, 7 -> r1, 5 -> r1 (7 < 9), 3 -> r0 (9 < 12), 3 -> r1 (12 = 12: lowest rank r0?)
    loads = [sum(works[i] for i in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(works)
    assert parts == bench.partition(works, 2)          # deterministic
    assert bench.partition(works, 1) == [list(range(6))]
    # more ranks than systems: the extra ranks get nothing
    assert [len(p) for p in bench.partition([1.0, 2.0], 4)] == [1, 1, 0, 0]


def test_work_estimate_counts_block_triples_of_h0_squared():
    from synth import make_chain
    s = make_chain(12, opa=4, b=4, spacing=2.8, cutoff=8.0, seed=0, dirs=("x",))
    k = np.diff(s.h0.row_ptr)
    assert bench.work_estimate(s) == float(np.sum(k * k))


def test_partitioned_job_time_counts_one_workload():
    import torch
    assert bench.job_seconds_per_solve(3.0, 3, 1, None, torch, None, replicas=False) == pytest.approx(1.0)
    assert bench.job_seconds_per_solve(3.0, 3, 1, None, torch, None, replicas=True) == pytest.approx(1.0)


def test_dense_oracle_refuses_large_systems():
    class M:
        n = bench.DENSE_MAX_N + 1
    with pytest.raises(ValueError):
        bench.dense(M())


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times a full CPU oracle solve (no GPU
    needed) and prints one JSON line with the keys the contract asks for."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "cluster", "--atoms", "60",
                        "--steps", "1", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "s" and line["value"] > 0
    assert line["higher_is_better"] is False and line["steps"] == 1 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["scaled_to_workload"]["kind"] == "model"
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("cluster-60-atoms") and line["config"]["atoms"] == 60
    assert line["config"]["sample"]["atoms"] == 60 and line["config"]["sample"]["iterations"] > 5


def test_oracle_sample_is_a_carve_out_of_the_smallest_cluster():
    from synth import make_chain, make_cluster
    systems = [make_chain(300, opa=8, b=32, spacing=2.8, cutoff=8.0, seed=1, dirs=("x",)),
               make_cluster(400, opa=8, b=32, cutoff=10.0, seed=2, dirs=("x",)),
               make_cluster(300, opa=8, b=32, cutoff=10.0, seed=3, dirs=("x",))]
    s, k, desc = bench.oracle_sample_system(systems)
    assert k == 2 and s.n_atoms == bench.SAMPLE_ATOMS and s.n == bench.SAMPLE_ATOMS * 8
    assert "system 2" in desc
