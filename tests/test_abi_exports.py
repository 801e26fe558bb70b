"""CPU checks of the boundary: libmtp.so builds for sm_103a, loads, exports
every function include/mtp.h declares, and the product package never
reaches the oracle."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2505_01059_gb300")


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "mtp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mtp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_01059_gb300 import _build, mtp
    _build.build_library()
    return mtp.load_library()


def test_library_exports_every_declared_function(lib):
    declared = _declared_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    from paper_2505_01059_gb300 import mtp
    assert sorted(mtp.EXPORTS) == declared


def test_problem_struct_layout_matches(lib):
    import ctypes
    from paper_2505_01059_gb300 import mtp
    assert lib.mtp_problem_bytes() == ctypes.sizeof(mtp.MtpProblem)


def test_product_never_imports_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    assert not any(a.name.split(".")[0] == "oracle" for a in node.names), f
                if isinstance(node, ast.ImportFrom):
                    assert (node.module or "").split(".")[0] != "oracle", f
    for dirpath, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            assert "oracle" not in open(os.path.join(dirpath, f)).read().lower(), f


def test_missing_library_fails_loudly(tmp_path):
    from paper_2505_01059_gb300 import mtp
    with pytest.raises(RuntimeError):
        mtp.load_library.__wrapped__(str(tmp_path / "nope.so")) if hasattr(
            mtp.load_library, "__wrapped__") else _fresh_load(mtp, str(tmp_path / "nope.so"))


def _fresh_load(mtp, path):
    saved = mtp._lib
    mtp._lib = None
    try:
        return mtp.load_library(path)
    finally:
        mtp._lib = saved


def test_workloads_hold_no_planner_arithmetic():
    # the shared input module imports only numpy: it draws task parameters,
    # never a step of the planner
    tree = ast.parse(open(os.path.join(PKG, "workloads.py")).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            mods.add(node.module)
    assert mods <= {"numpy", "__future__"}, mods


@pytest.mark.parametrize("bad,word", [
    (dict(E=0), "E"), (dict(E=10_000), "E"), (dict(beta=1.5), "beta"), (dict(alpha=1.0), "alpha"),
    (dict(M=0), "M"), (dict(sigma_min=0.0), "sigma"), (dict(interp="bspline", degree=9), "degree"),
    (dict(dt=0.0), "dt"), (dict(B=0), "B"),
])
def test_invalid_problems_rejected_before_any_device_work(lib, bad, word):
    """mtp_create validates the problem on the host first: an invalid one is
    refused with MTP_ERR_INVALID_ARG and a message naming the field, with or
    without a GPU."""
    from paper_2505_01059_gb300 import mtp, workloads as W
    spec = dict(W.pointmass(B=512), **bad)
    with pytest.raises(mtp.MtpError) as ei:
        mtp.mtp_create(spec)
    assert ei.value.status == 1
    assert word.lower() in str(ei.value).lower()
