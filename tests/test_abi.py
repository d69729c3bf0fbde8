"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/claw.h
declares; the Python binding declares a signature for each (no GPU needed)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "claw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(claw_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1808_02638_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (claw_[a-z_0-9]+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    assert len(declared_symbols()) >= 18


def test_library_loads_and_binding_covers_the_header():
    from paper_1808_02638_gb300 import build, claw
    build.build()
    L = ctypes.CDLL(claw.LIB_PATH)
    for s in declared_symbols():
        assert hasattr(L, s)
        assert s in claw._SIGNATURES, s
    assert claw.load().claw_strerror(5).decode() == "NaN or Inf in the state"


def test_binding_structs_match_header_layout():
    from paper_1808_02638_gb300 import claw
    # claw_box: 6 int32 + 2 int64; claw_problem: 4 doubles, 3 ints, 8 ratios, 1 double, ...
    assert ctypes.sizeof(claw.claw_box) == 40
    assert claw.claw_problem.cfl.offset == 4 * 8 + 3 * 4 + 8 * 4 + 4   # aligned to 8
    assert claw.claw_problem.rho0.offset % 8 == 0


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1808_02638_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "claw_oracle" not in text, f
