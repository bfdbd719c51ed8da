"""The C-ABI library builds, loads and exports every entry point declared in include/otgb.h
(no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "otgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ot_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1009_6039_gb300 as ot
    return ot


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ot_plan_create", "ot_solve", "ot_solve_batched", "ot_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ot_[a-z_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    assert sorted(lib.EXPORTS) == _declared()


def test_binding_names_match_abi(lib):
    for n in _declared():
        assert callable(getattr(lib, n)), n


def test_strerror_without_gpu(lib):
    assert lib.ot_strerror(0) == "ok"
    assert "converge" in lib.ot_strerror(lib.OT_ENOCONV)
    assert lib.ot_strerror(-99) == "unknown status"
    assert "wait" in lib.ot_strerror(lib.OT_ETIMEOUT)


def test_build_is_arm_portable():
    # host code must build on the aarch64 GPU hosts: no x86 intrinsics or -march flags
    for d in ("paper_1009_6039_gb300/csrc", "oracle"):
        for fn in os.listdir(os.path.join(ROOT, d)):
            if fn.endswith((".cu", ".cuh", ".c", ".h")):
                s = open(os.path.join(ROOT, d, fn)).read()
                assert "immintrin" not in s and "xmmintrin" not in s, fn
    b = open(os.path.join(ROOT, "paper_1009_6039_gb300", "build.py")).read()
    assert "march" not in b


def test_binding_constants_match_the_header(lib):
    # every OT_OPT_*, OT_PROF_* and status code of the header has the same value in the binding
    src = open(os.path.join(ROOT, "include", "otgb.h")).read()
    defs = dict((k, int(v)) for k, v in re.findall(
        r"#define\s+(OT_(?:OPT|PROF|E|OK)[A-Z0-9_]*)\s+\(?(-?\d+)\)?", src))
    assert len(defs) > 30
    for name, value in defs.items():
        if name.startswith("OT_PROF_"):
            if name == "OT_PROF_CLASSES":
                assert len(lib.PROF_CLASSES) == value
            continue
        assert getattr(lib, name) == value, name
    # the Plan option names cover every option key
    keys = {v for k, v in defs.items() if k.startswith("OT_OPT_")}
    assert keys == set(lib.Plan._keys.values())
