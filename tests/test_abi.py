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


def test_binding_structs_match_header_layout(tmp_path):
    # the C compiler's offsets of every field of the header's structs equal the binding's
    from paper_1808_02638_gb300 import claw
    structs = {"claw_problem": claw.claw_problem, "claw_box": claw.claw_box, "claw_fill_job": claw.claw_fill_job}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "claw.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln)}
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1808_02638_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "claw_oracle" not in text, f
