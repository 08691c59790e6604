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
