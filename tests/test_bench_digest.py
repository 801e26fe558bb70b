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



def test_public_header_prototypes_do_not_count(tmp_path):
    """A new entry point in include/mtp.h is host interface: the profiles of
    the kernels stay valid; a change to a type the kernels use retires them."""
    d = tmp_path / "include"
    d.mkdir()
    h = d / "mtp.h"
    base = "typedef struct { int a; } mtp_x;\nmtp_status mtp_f(mtp_x* p, int n);\n"
    h.write_text(base)
    t0 = bench._code_text(str(h))
    h.write_text(base + "/* new */\nmtp_status mtp_g(const float* d, int32_t k,\n                  void* s);\n"
                 "const char* mtp_name(const mtp_x* p);\n")
    assert bench._code_text(str(h)) == t0 == "typedef struct { int a; } mtp_x;"
    h.write_text(base.replace("int a;", "int a; int b;"))
    assert bench._code_text(str(h)) != t0
