"""The kernel-source hash that gates the benchmark's ncu traffic figure covers code only:
comments and whitespace leave it unchanged, any code change moves it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SRC = """// kernel
__global__ void k(int* a) {  /* one
                                 two */
    a[0] = 1;   // store
}
"""


def test_comments_and_whitespace_do_not_count():
    base = bench.code_only(SRC)
    assert base == "__global__voidk(int*a){a[0]=1;}"
    assert bench.code_only(SRC + "\n// note\n/* note */\n\n   ") == base
    assert bench.code_only(SRC.replace("    a[0]", "\ta[0]")) == base
    assert bench.code_only(SRC.replace("a[0] = 1", "a[0] = 2")) != base


def test_hash_is_stable():
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert len(bench.kernel_source_hash()) == 16
