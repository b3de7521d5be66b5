"""The benchmark configurations run at their stated sizes, against the FP64 oracle's own runs (GB300).

Every expected value here comes from the oracle alone, run by the committed scripts in tests/golden/ on the
seeded bunch: the GPU's state is never handed to the oracle.

N = 4096 uniform-field run (Sec. 2.2 eq:dt / eq:linear, Sec. 2.3 Higuera-Cary, Sec. 2.6 background field):
sigma = 10 um, gamma0 = 3, B = 5e-5 T along x, dt = 1e-15 s, depth 512 (the window slides from step 512 on),
2000 steps from t = 0, seed 0; the oracle's run is tests/golden/cfg2_oracle_run.npz.
  - positions of all particles after 1, 100, 511, 512, 1000, 1500 and 2000 steps: max_i |dx_i| / sigma_rms
    <= 1e-9 on the FP64 path; the error at every checkpoint is recorded (its growth per step);
  - fields of 256 sampled targets at steps 0 and 1 (the same state on both sides, up to rounding):
    <= 1e-12 of sum_j |F_ij| (FP64), <= 1e-5 (mixed); at steps 511, 512, 1000 and 1999 the two runs'
    states differ by the position error above, and the field difference is held to FIELD_TRAJ_TOL.

N = 65536 free-expansion run (the benchmark's bunch: sigma = 20 um, gamma0 = 3, dt = 1e-15 s, depth 1024),
500 steps from t = 0 on the FP64 and the mixed path from the same seed. A 500-step oracle run of 65536
particles is out of reach of a host; the oracle's first full step is tests/golden/cfg3_oracle_start.npz:
  - fields of 64 sampled targets at steps 0 and 1 (<= 1e-12 FP64, <= 1e-5 mixed) and their positions after
    1 and 2 steps (<= 1e-12 of the bunch size);
  - at steps 250 and 499 the mixed path evaluates the FP64 path's state (a second solver given that
    history), and after 500 steps the two paths' positions are compared: stated numbers, with bars. The
    FP64 kernel at N = 65536 mid-run against the oracle is test_gpu_fp64.py::test_full_size_sampled_targets
    (a seeded step-250 history).
"""
import json
import os

import numpy as np
import pytest

from gpu_helpers import record, sigma_rms

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FIELD_TOL = {"fp64": 1e-12, "mixed": 1e-5}
POS_TOL_FP64 = 1e-9
# mixed path: positions against the oracle's run after the stated steps (measured 8.7e-10 of the bunch size
# after 2000 steps of the N = 4096 run) and against the FP64 path after 500 steps (measured 2.0e-11); the bar
# leaves a factor of about 10
POS_TOL_MIXED = 1e-8
# fields of two runs whose states have drifted apart by the position error (FP64: measured 1.9e-12 at step
# 1999, where the positions differ by 2.5e-14 of the bunch size; mixed: the mixed path's own bar)
FIELD_TRAJ_TOL = {"fp64": 1e-10, "mixed": 1e-5}


def _field_err(F, F_ref, M):
    return float(np.max(np.abs(F - F_ref) / np.maximum(M, 1e-300)))


def _golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"golden file {name} not generated (see tests/golden/make_*.py)")
    G = np.load(path)
    return G, json.loads(str(G["meta"]))


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_cfg2_uniform_field_2000_steps(path):
    G, meta = _golden("cfg2_oracle_run.npz")
    N, D, dt, steps = meta["N"], meta["D"], meta["dt"], meta["steps"]
    b_uni = np.array(meta["B"])
    tg = G["targets"]
    pos_steps, field_steps = set(meta["pos_steps"]), set(meta["field_steps"])
    bunch = inputs.gaussian_bunch(N, meta["sigma"], meta["gamma0"], seed=meta["seed"])
    bext = emppp.bext_uniform(b_uni)
    stream = torch.cuda.Stream()
    pos_err, field_err = {}, {}
    with emppp.Solver(N, D, dt, precision=path, proposal="closed_form", stream=stream) as s:
        s.set_particles(bunch.x.copy(), bunch.u.copy())
        n = 0
        while True:
            if n in pos_steps:
                x, u, t, nn = s.get_state()
                assert nn == n and t == float(G[f"t_{n}"][0])
                xg = G[f"x_{n}"]
                pos_err[n] = float(np.max(np.linalg.norm(x - xg, axis=1)) / sigma_rms(xg))
            if n in field_steps:
                s.step(1, bext)
                E, B = s.get_fields()
                M = G[f"M_{n}"]
                # get_fields and the oracle's step both report B_self + B_ext
                field_err[n] = (_field_err(E[tg], G[f"E_{n}"], M[:, 0:1]),
                                _field_err(B[tg] - b_uni, G[f"B_{n}"] - b_uni, M[:, 1:2]))
                n += 1
                continue
            nxt = [k for k in sorted(pos_steps | field_steps) if k > n]
            if not nxt:
                break
            s.step(nxt[0] - n, bext)
            n = nxt[0]
    assert n == steps
    record(f"cfg2_{path}", dict(position_error_over_sigma=pos_err, field_error=field_err))
    print(path, "positions", pos_err, "fields", field_err)
    for k, (eE, eB) in field_err.items():
        bar = FIELD_TOL[path] if k <= 1 else FIELD_TRAJ_TOL[path]
        assert eE <= bar and eB <= bar, (k, eE, eB)
    bar = POS_TOL_FP64 if path == "fp64" else POS_TOL_MIXED
    for k, e in pos_err.items():
        assert e <= bar, (k, e)


CFG3 = dict(N=65536, sigma=20e-6, gamma0=3.0, dt=1e-15, D=1024, steps=500, seed=0)
CFG3_CROSS = (250, 499)


def _cfg3_run(path, G, keep_at=()):
    """500 steps from t = 0: fields of steps 0 and 1 and positions after 1 and 2 steps of the golden
    targets; the history at the steps in keep_at; the final positions."""
    c = CFG3
    tg = G["targets"]
    bunch = inputs.gaussian_bunch(c["N"], c["sigma"], c["gamma0"], seed=c["seed"])
    stream = torch.cuda.Stream()
    res, kept = {}, {}
    with emppp.Solver(c["N"], c["D"], c["dt"], precision=path, proposal="closed_form", stream=stream) as s:
        s.set_particles(bunch.x.copy(), bunch.u.copy())
        for k in (0, 1):
            s.step(1)
            E, B = s.get_fields()
            x, u, _, _ = s.get_state()
            M = G[f"M_{k}"]
            res[f"E_{k}"] = _field_err(E[tg], G[f"E_{k}"], M[:, 0:1])
            res[f"B_{k}"] = _field_err(B[tg], G[f"B_{k}"], M[:, 1:2])
            res[f"x_{k + 1}"] = float(np.max(np.linalg.norm(x[tg] - G[f"x_{k + 1}"], axis=1)) / sigma_rms(x))
            res[f"u_{k + 1}"] = float(np.max(np.abs(u[tg] - G[f"u_{k + 1}"])) / np.max(np.abs(G[f"u_{k + 1}"])))
        n = 2
        for k in sorted(keep_at):
            s.step(k - n)
            n = k
            kept[k] = s.get_history()
        s.step(c["steps"] - n)
        x_end, _, _, n_end = s.get_state()
        assert n_end == c["steps"]
    return res, x_end, kept


def test_cfg3_500_steps_fp64_and_mixed():
    G, meta = _golden("cfg3_oracle_start.npz")
    c = CFG3
    assert meta["N"] == c["N"] and meta["D"] == c["D"]
    r64, x64, kept = _cfg3_run("fp64", G, keep_at=CFG3_CROSS)
    rmx, xmx, _ = _cfg3_run("mixed", G)
    # the mixed path on the FP64 path's own state at steps 250 and 499, against the FP64 path's fields
    cross = {}
    for k, (n, T, W, V, u) in kept.items():
        F = {}
        for path in ("fp64", "mixed"):
            with emppp.Solver(c["N"], c["D"], c["dt"], precision=path, proposal="closed_form") as s:
                s.set_history(n, T, W, V, u)
                s.step(1)
                F[path] = s.get_fields()
        nE = np.linalg.norm(F["fp64"][0], axis=1)
        nB = np.linalg.norm(F["fp64"][1], axis=1)
        cross[k] = dict(E_rel_norm_max=float(np.max(np.linalg.norm(F["mixed"][0] - F["fp64"][0], axis=1) / nE)),
                        B_rel_norm_max=float(np.max(np.linalg.norm(F["mixed"][1] - F["fp64"][1], axis=1) / nB)),
                        E_rel_norm_median=float(np.median(np.linalg.norm(F["mixed"][0] - F["fp64"][0], axis=1) / nE)))
    drift = float(np.max(np.linalg.norm(xmx - x64, axis=1)) / sigma_rms(x64))
    record("cfg3", dict(fp64_vs_oracle=r64, mixed_vs_oracle=rmx, mixed_vs_fp64_path_same_state=cross,
                        mixed_vs_fp64_positions_after_500=drift))
    print("fp64", r64, "mixed", rmx, "cross", cross, "drift", drift)
    for path, r in (("fp64", r64), ("mixed", rmx)):
        for k in (0, 1):
            assert r[f"E_{k}"] <= FIELD_TOL[path] and r[f"B_{k}"] <= FIELD_TOL[path], (path, k, r)
        for k in (1, 2):
            # after one or two steps the self fields have moved the positions by far less than 1e-12 of the
            # bunch size: both paths' pushes (FP64) agree with the oracle's to rounding
            assert r[f"x_{k}"] <= 1e-12 and r[f"u_{k}"] <= (1e-12 if path == "fp64" else 1e-10), (path, k, r)
    for k, e in cross.items():
        # normwise |E_i| is the net field, which cancels at the bunch centre: the bar is the mixed path's
        # 1e-5 of sum_j |E_ij| scaled by the largest cancellation ratio seen (design notes)
        assert e["E_rel_norm_median"] <= 1e-5, (k, e)
    assert drift <= POS_TOL_MIXED, drift
