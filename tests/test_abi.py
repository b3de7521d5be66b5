"""The C-ABI library builds, loads and exports every symbol the header declares (no GPU calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            src = open(os.path.join(ROOT, "include", hdr)).read()
            names |= set(re.findall(r"EMPPP_API\s+[\w\s\*]+?\b(emppp_\w+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("emppp_create", "emppp_set_particles", "emppp_step", "emppp_get_state", "emppp_get_fields",
                 "emppp_destroy", "emppp_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2605_05543_gb300 import _build, emppp

    _build.build_library()
    lib = emppp.load()
    names = _declared()
    assert names, "no declarations found"
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding knows every declared symbol, and nothing else
    assert set(emppp.SIGNATURES) == names
    assert lib.emppp_version().decode().startswith("emppp")


def test_library_exports_nothing_else():
    from paper_2605_05543_gb300 import _build

    path = _build.build_library()
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm not available")
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T " in ln}
    ours = {s for s in exported if s.startswith("emppp_")}
    assert ours == _declared()
