"""Diagnostics of the library on the GB300: the FP64 kernel's reciprocal against the correctly rounded
quotient, and the ALU throughput probes that give the benchmark its measured roofline denominators."""
import numpy as np
import pytest

from gpu_helpers import record

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2605_05543_gb300 import emppp, inputs  # noqa: E402

ULP_BAR = 2.0  # the bar stated with emppp_reciprocal_probe in include/emppp.h


def _ulps(y, ref):
    return np.abs(y - ref) / np.spacing(np.abs(ref))


def test_reciprocal_within_two_ulp():
    """1 / x of the FP64 pair kernel (approximate reciprocal + two Newton-Raphson steps) over the arguments
    the kernel passes and across the whole normal range it is stated for. numpy's 1.0 / x is IEEE
    division, correctly rounded, so the distance is counted in units in the last place of the quotient."""
    rng = np.random.default_rng(7)
    c = inputs.C_LIGHT
    parts = [
        # eta . v' = R (c - eta_hat . v): R from 1e-12 m to 1 m, 1 - beta cos psi from 1e-6 to 2
        rng.uniform(-12, 0, 200000),
        # C2 = c^2 - |v|^2 and the denominators of the root of eq:dt
        np.log10(c * c) + rng.uniform(-8, 0, 200000),
        # the stated range, log-uniform over the exponents
        rng.uniform(-1021.9 * np.log10(2), 1021.9 * np.log10(2), 400000),
    ]
    x = np.concatenate([10.0 ** p for p in parts[:2]] + [10.0 ** parts[2]])
    x = x * (1.0 + rng.uniform(0, 1e-3, x.size))  # random mantissas
    edges = np.array([2.0 ** -1022 * 1.0000001, 2.0 ** 1022, 1.0, 2.0, 0.5, 3.0, 1.0 / 3.0, c, c * c,
                      np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0)])
    x = np.concatenate([x, edges])
    y = emppp.reciprocal_probe(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = 1.0 / x
    u = _ulps(y, ref)
    record("reciprocal", dict(max_ulp=float(u.max()), mean_ulp=float(u.mean()),
                              exact_fraction=float(np.mean(u == 0)), samples=int(x.size)))
    assert np.all(np.isfinite(y))
    assert u.max() <= ULP_BAR, (u.max(), x[np.argmax(u)])
    # powers of two have exact reciprocals
    p2 = 2.0 ** np.arange(-1000, 1001, 37, dtype=np.float64)
    y2 = emppp.reciprocal_probe(torch.from_numpy(p2).cuda()).cpu().numpy()
    assert np.array_equal(y2, 1.0 / p2)


def test_peak_probe_is_plausible():
    p = emppp.measure_peaks()
    sms = p["sms"]
    # nominal at the GB300's maximum SM clock (2.07 GHz): 128 FP32 lanes, 2 FP64 lanes, 16 MUFU lanes per SM
    nominal = dict(fp32_flops=sms * 128 * 2 * 2.07e9, fp64_flops=sms * 2 * 2 * 2.07e9, mufu_ops=sms * 16 * 2.07e9)
    record("peaks", {**p, **{k + "_nominal": v for k, v in nominal.items()}})
    for k, v in nominal.items():
        # a probe that does the work reaches a large fraction of the pipe at the clock under load, and
        # cannot exceed it
        assert 0.3 * v <= p[k] <= 1.25 * v, (k, p[k], v)
