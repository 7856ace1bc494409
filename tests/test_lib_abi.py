"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/gt.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gt_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2311_02573_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert {"gt_build", "gt_insert", "gt_query", "gt_exhaustive"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    from paper_2311_02573_gb300 import gt
    assert set(gt.ENTRY_POINTS) <= _declared()


def test_struct_layouts_match_header():
    # the binding's ctypes structs mirror the header's field order and sizes
    from paper_2311_02573_gb300 import gt
    assert ctypes.sizeof(gt.BuildOpts) == 8 + 8 + 8 + 4 + 4 + 4 + 4
    assert gt.BuildOpts.layout.offset == 32 and gt.BuildOpts.prefix_level.offset == 36
    assert ctypes.sizeof(gt.QueryOpts) == 8 + 4 + 4 + 8 + 8 + 4 + 4 + 8 + 4 + 4
    assert ctypes.sizeof(gt.CSR) == 8 + 8 + 8 + 4 + 4
    assert gt.QueryStats.level_tests.offset == 7 * 8 + 2 * 4
    assert gt.QueryStats.launches.offset == 7 * 8 + 2 * 4 + 64 * 8 + 8
    assert ctypes.sizeof(gt.QueryStats) == 7 * 8 + 2 * 4 + 64 * 8 + 8 + 2 * 8 + 8 * 4 + 3 * 8
    assert ctypes.sizeof(gt.AutotuneResult) == 4 * (3 + 1 + 9 + 9 + 8 + 4 + 1)
    assert ctypes.sizeof(gt.ServerOpts) == 8 + 4 + 4 + 8 + 8 + 8 + 4 + 4
    assert gt.ServerOpts.schedule.offset == 40
    assert ctypes.sizeof(gt.ServerStats) == 16 * 8
    assert ctypes.sizeof(gt.TreeInfo) == 8 + 8 + 4 * 8
