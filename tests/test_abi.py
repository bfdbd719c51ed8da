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


def _struct_fields(name):
    src = open(os.path.join(ROOT, "include", "otgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct\s*\{(.*?)\}\s*%s;" % name, src, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, names = decl.split(None, 1)
        fields += [(typ, n.strip()) for n in names.split(",")]
    return fields


def test_stats_struct_layout_matches_the_header(lib, tmp_path):
    # the binding's ot_stats has the header's fields in the header's order, with the offsets
    # and size a C compiler gives them
    import ctypes
    fields = _struct_fields("ot_stats")
    ctypes_of = {"int32_t": ctypes.c_int32, "double": ctypes.c_double}
    assert [n for _, n in fields] == [n for n, _ in lib.ot_stats._fields_]
    for (typ, n), (m, ct) in zip(fields, lib.ot_stats._fields_):
        assert ctypes_of[typ] is ct, n
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "otgb.h"\nint main(void) {\n'
                    + "".join('  printf("%%zu\\n", offsetof(ot_stats, %s));\n' % n
                              for _, n in fields)
                    + '  printf("%zu\\n", sizeof(ot_stats));\n  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[:-1] == [getattr(lib.ot_stats, n).offset for _, n in fields]
    assert out[-1] == ctypes.sizeof(lib.ot_stats)
