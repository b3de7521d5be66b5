"""Cases run on the debug build of the library (a child process with EMPPP_DEBUG_LIB=1): every pair-kernel
instance family on small systems. Writes each case's fields and its status after the step to an npz file
(argv[1]); test_gpu_debug_build.py compares them with the oracle."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

from gpu_helpers import DT, history_case, window  # noqa: E402
from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

# name: (N, n, D, sigma, precision, proposal, extra)
CASES = {
    "fp64_tiles": (300, 60, 128, 10e-6, "fp64", "closed_form", {}),
    "fp64_bisect_wrapped": (517, 90, 48, 5e-6, "fp64", "bisect", {}),
    "fp64_mlp": (300, 60, 128, 10e-6, "fp64", "mlp", {}),
    "fp64_midpoint": (300, 60, 128, 10e-6, "fp64", "closed_form", {"reconstruction": "midpoint"}),
    "mixed_tiles": (300, 60, 128, 10e-6, "mixed", "closed_form", {}),
    "mixed_bisect_wrapped": (517, 90, 48, 5e-6, "mixed", "bisect", {}),
    "mixed_mlp": (300, 60, 128, 10e-6, "mixed", "mlp", {}),
    "mixed_window": (517, 90, 48, 5e-6, "mixed", "closed_form", {"window": True}),
    "mixed_shape_256": (517, 90, 48, 5e-6, "mixed", "closed_form", {"shape": (256, 8)}),
}


def run_case(N, n, D, sigma, precision, proposal, extra):
    h = history_case(N, n, sigma=sigma, seed=31 + N)
    T, W, V, u = window(h, D)
    kw = {k: v for k, v in extra.items() if k in ("reconstruction",)}
    with emppp.Solver(N, D, DT, precision=precision, proposal=proposal, **kw) as s:
        s.set_history(n, T, W, V, u)
        if proposal == "mlp":
            s.set_proposal(inputs.mlp_init_params(5))
        if extra.get("window"):
            s.set_tuning(targets_per_block=128, sources_per_sum=32, history_window=1)
        if "shape" in extra:
            s.set_tuning(targets_per_block=extra["shape"][0], sources_per_sum=extra["shape"][1])
        # the bracket dump instance, on the stored state itself (before the step moves it)
        brackets = s.bracket_dump()[0] if proposal == "closed_form" and not extra else None
        s.step(1)
        status = emppp.OK
        try:
            s.get_state()
        except emppp.EmpppError as e:
            status = e.status
        E, B = s.get_fields()
    return E, B, status, brackets


def main(path):
    assert emppp.library_path().endswith("libemppp_debug.so")
    emppp.load()
    out = {}
    for name, case in CASES.items():
        E, B, status, brackets = run_case(*case)
        out[name + "/E"], out[name + "/B"], out[name + "/status"] = E, B, np.array(status)
        if brackets is not None:
            out[name + "/brackets"] = brackets
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
