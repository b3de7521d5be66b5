"""The debug build of the library (GB300): its pair kernels check every history-window offset they turn into
a ring slot, and every source and target index, against its range, and record a failure in the device error
word (kErrBounds) instead of trapping. compute-sanitizer is not available on this machine, so this build is the
bounds check of the kernels. Every instance family runs on small systems (both precisions, the three
proposals, eq:mid, the history window, a wider tile, a wrapped ring, the bracket dump) in a child process
that loads the debug build: no check fails (status OK after every step) and the fields match the oracle
(1e-12 FP64, 1e-5 mixed) as in the release build.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from gpu_helpers import field_errors, history_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import _build, emppp  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from debug_build_cases import CASES  # noqa: E402


def test_debug_build_checks_pass_and_fields_match_oracle(tmp_path):
    _build.build_library(debug=True)
    path = str(tmp_path / "debug_cases.npz")
    env = dict(os.environ, EMPPP_DEBUG_LIB="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_cases.py"), path], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(path)
    for name, (N, n, D, sigma, precision, proposal, extra) in CASES.items():
        assert int(got[name + "/status"]) == emppp.OK, name
        h = history_case(N, n, sigma=sigma, seed=31 + N)
        variant = oracle.MIDPOINT if extra.get("reconstruction") == "midpoint" else 0
        E_ref, B_ref, _, M = oracle.self_fields(h.T, h.W, h.V, n, D, mags=True, variant=variant)
        eE, eB = field_errors(got[name + "/E"], got[name + "/B"], E_ref, B_ref, M)
        tol = 1e-12 if precision == "fp64" else 1e-5
        assert eE <= tol and eB <= tol, (name, eE, eB)
        if name + "/brackets" in got:
            assert np.array_equal(got[name + "/brackets"], oracle.bracket_table(h.T, h.W, n, D)), name
