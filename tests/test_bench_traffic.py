"""The key that ties committed ncu traffic counters to a kernel's code (bench.py's `traffic` field).

A counter recorded for some code must stop being reported once that code changes, and only then:
comment and blank-line edits keep the key, any code edit in scope changes it, and text past the
kernel's end marker is out of scope.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KERNEL = """// header comment
#include "x.cuh"
/* a block
   comment */
__global__ void k_a(int* p) {
  p[0] = 1;   // trailing comment
}
// END OF k_a
__global__ void k_b(int* p) { p[0] = 2; }
"""


def _hash(tmp_path, text, until="// END OF k_a"):
    (tmp_path / "k.cu").write_text(text)
    (tmp_path / "x.cuh").write_text("#define X 1\n")
    old = bench.ROOT
    bench.ROOT = str(tmp_path)
    try:
        return bench._code_hash([{"file": "k.cu", "until": until}, {"file": "x.cuh"}])
    finally:
        bench.ROOT = old


def test_comments_and_blank_lines_keep_the_key(tmp_path):
    h = _hash(tmp_path, KERNEL)
    edited = KERNEL.replace("// trailing comment", "// another remark").replace("/* a block", "/* edited block")
    edited = edited.replace("p[0] = 1;", "\n\np[0] = 1;   ")
    assert _hash(tmp_path, edited) == h


def test_a_code_edit_in_scope_changes_the_key(tmp_path):
    h = _hash(tmp_path, KERNEL)
    assert _hash(tmp_path, KERNEL.replace("p[0] = 1;", "p[0] = 3;")) != h
    # an included header is in scope too
    (tmp_path / "k.cu").write_text(KERNEL)
    (tmp_path / "x.cuh").write_text("#define X 2\n")
    old = bench.ROOT
    bench.ROOT = str(tmp_path)
    try:
        h2 = bench._code_hash([{"file": "k.cu", "until": "// END OF k_a"}, {"file": "x.cuh"}])
    finally:
        bench.ROOT = old
    assert h2 != h


def test_text_after_the_kernel_is_out_of_scope(tmp_path):
    h = _hash(tmp_path, KERNEL)
    assert _hash(tmp_path, KERNEL.replace("p[0] = 2;", "p[0] = 7;")) == h
    # a missing end marker never matches
    assert _hash(tmp_path, KERNEL, until="// no such marker") is None


def test_traffic_is_reported_only_for_matching_code(tmp_path, monkeypatch):
    (tmp_path / "k.cu").write_text(KERNEL)
    (tmp_path / "x.cuh").write_text("#define X 1\n")
    (tmp_path / "profiles").mkdir()
    scope = [{"file": "k.cu", "until": "// END OF k_a"}, {"file": "x.cuh"}]
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"k_a@w": {"scope": scope, "code_sha256_16": bench._code_hash(scope), "dram_bytes_per_launch": 1234}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench._traffic("k_a@w") == 1234
    assert bench._traffic("k_b@w") is None
    (tmp_path / "k.cu").write_text(KERNEL.replace("p[0] = 1;", "p[0] = 5;"))
    assert bench._traffic("k_a@w") is None
