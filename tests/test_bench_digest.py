"""bench.source_digest: a profile is retired by a change to the code of its
kernel or headers, not by a change to their comments or layout."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_text_drops_comments_and_layout(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f(int x) {  // one\n  return x + 1; /* two\n lines */\n}\n")
    b.write_text("/* header */\nint f(int x) {\n\n    return x + 1;\n}  // end\n")
    assert bench._code_text(str(a)) == bench._code_text(str(b)) == "int f(int x) { return x + 1; }"


def test_code_text_sees_code_changes(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f(int x) { return x + 1; }\n")
    b.write_text("int f(int x) { return x + 2; }\n")
    assert bench._code_text(str(a)) != bench._code_text(str(b))

