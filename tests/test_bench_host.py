"""Host logic of bench.py that needs no GPU: the source digest that keeps a
profiled DRAM-traffic figure tied to the kernel code it was captured on."""

import bench

SRC = '''// header comment
__global__ void k(float *x, int n) {   /* a block
   comment */
    const char *s = "// not a comment";
    if (threadIdx.x < n) x[threadIdx.x] *= 2.f;
}
'''


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


def test_recorded_traffic_only_for_its_workload():
    assert bench.profiled_traffic("tc", "some other workload") is None
    assert bench.profiled_traffic("no such class", bench.WORKLOAD) is None


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the CPU oracle (no GPU needed) and
    prints one JSON line with the keys the benchmark contract asks for."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--atoms", "60", "--steps", "1",
                        "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "s" and line["value"] > 0
    assert line["higher_is_better"] is False and line["steps"] == 1 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("cluster-60-atoms") and line["config"]["atoms"] == 60
