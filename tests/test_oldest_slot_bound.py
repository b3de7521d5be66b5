"""The mixed path's oldest-slot bound, restated in numpy FP32 and checked against exact arithmetic (CPU).

A pair predicted beyond the stored history needs the node test of the oldest slot k0: |r - w_k0|^2 against
that slot's FP32 upper threshold T (Sec. 2.2). The pair kernel decides it without loading slot k0's record:
with d = r - w_n from the hi/lo split present records and the source's chord c = w_n - w_k0 (FP64, rounded
to FP32), it accepts when fl32(2 d.c + fl32(|d|^2 (1 - 32u))) exceeds the per-source threshold
T (1 + 32u) - |c|^2 (1 - 32u), formed in FP64 and rounded up. The argument is that an accepted pair has an
exact |r - w_k0|^2 above T (1 + 32u), so that the FP32 node test itself is true at its first comparison.

Here the kernel's operations are written out in float32 (each operation rounded to nearest, the final
multiply-add once), with and without contraction of the dot products into fused multiply-adds, for
geometries whose |r - w_k0| lies within a relative 1e-8 to 1e-3 of sqrt(T) on either side, chords up
to the light-travel distance and target-source separations from near zero upwards. Checked:
  - soundness: every accepted pair has an exact |r - w_k0|^2 (rational arithmetic on the FP64
    positions) above T (1 + 24u), and its FP32 node-test value (from the hi/lo records of r and w_k0)
    above T;
  - usefulness: every pair 1e-4 or more outside the sphere, with the split origin close enough for the
    FP32 band, is accepted.
"""
from fractions import Fraction

import numpy as np

U = 2.0 ** -24
F32 = np.float32


def split(x, origin):
    """hi/lo FP32 split of FP64 coordinates about an origin, as the shadow ring stores them."""
    y = x - origin
    hi = y.astype(np.float32)
    lo = (y - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def separation(rh, rl, wh, wl):
    """(r_hi - w_hi) + (r_lo - w_lo), each operation rounded to FP32."""
    return (rh - wh) + (rl - wl)


def fma32(a, b, c):
    """a b + c rounded once to FP32 (the product of two FP32 values is exact in FP64)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def dot32(a, b, fused):
    if fused:
        return fma32(a[:, 2], b[:, 2], fma32(a[:, 1], b[:, 1], a[:, 0] * b[:, 0]))
    return a[:, 0] * b[:, 0] + a[:, 1] * b[:, 1] + a[:, 2] * b[:, 2]


def round_up32(x):
    f = x.astype(np.float32)
    low = f.astype(np.float64) < x
    f[low] = np.nextafter(f[low], np.float32(np.inf))
    return f


def geometry(n, seed):
    """n pairs: the oldest stored position w_k0, the present position w_n = w_k0 + c and the target r,
    with |r - w_k0| = sqrt(T) (1 + eps); T an FP32 threshold of (c (t_n - t_k0))^2."""
    rng = np.random.default_rng(seed)
    L = 10.0 ** rng.uniform(-7, -3, n)  # light-travel distance c (t_n - t_k0), m
    T = (L * L).astype(np.float32).astype(np.float64)
    origin = rng.normal(size=(n, 3)) * 1e-4
    wk0 = origin + rng.normal(size=(n, 3)) * 10.0 ** rng.uniform(-6, -3.5, (n, 1))
    cdir = rng.normal(size=(n, 3))
    cdir /= np.linalg.norm(cdir, axis=1, keepdims=True)
    beta = rng.uniform(0.0, 0.999, n)
    beta[: n // 8] = 0.0  # a source at rest (c = 0)
    wn = wk0 + cdir * (beta * L)[:, None]
    # target direction from w_k0: random, towards the present position, or away from it
    rdir = rng.normal(size=(n, 3))
    mode = rng.integers(0, 3, n)
    rdir[mode == 1] = cdir[mode == 1] + 0.05 * rdir[mode == 1]
    rdir[mode == 2] = -cdir[mode == 2] + 0.05 * rdir[mode == 2]
    rdir /= np.linalg.norm(rdir, axis=1, keepdims=True)
    sign = rng.choice([-1.0, 1.0], n)
    eps = sign * 10.0 ** rng.uniform(-8, -3, n)
    r = wk0 + rdir * (np.sqrt(T) * (1.0 + eps))[:, None]
    return T, origin, wk0, wn, r, eps


def bound_and_test(T, origin, wk0, wn, r, fused):
    rh, rl = split(r, origin)
    nh, nl = split(wn, origin)
    kh, kl = split(wk0, origin)
    # per source, FP64: the chord and the bound's threshold
    c64 = wn - wk0
    cc = np.sum(c64 * c64, axis=1)
    thr = round_up32(T * (1.0 + 32 * U) - cc * (1.0 - 32 * U))
    c32 = c64.astype(np.float32)
    # per pair, FP32: the bound
    d = separation(rh, rl, nh, nl)
    dd = dot32(d, d, fused)
    dc = dot32(d, c32, fused)
    accept = fma32(np.full_like(dc, 2.0), dc, dd * F32(1.0 - 32 * U)) > thr
    # the node test's own FP32 value at slot k0
    dk = separation(rh, rl, kh, kl)
    D2k = dot32(dk, dk, fused)
    return accept, D2k


def exact_sq(a, b):
    return [sum((Fraction(float(x)) - Fraction(float(y))) ** 2 for x, y in zip(a[i], b[i])) for i in range(len(a))]


def test_bound_is_sound_and_useful():
    n = 40000
    T, origin, wk0, wn, r, eps = geometry(n, seed=2605)
    for fused in (False, True):
        accept, D2k = bound_and_test(T, origin, wk0, wn, r, fused)
        idx = np.nonzero(accept)[0]
        assert len(idx) > n // 4, len(idx)
        # the FP32 node test at slot k0 is true at its first comparison
        assert np.all(D2k[idx].astype(np.float64) > T[idx])
        # the exact distance is beyond the threshold with the stated margin (checked on the accepted pairs
        # closest to the sphere, where it is tight, and a sample of the rest)
        order = idx[np.argsort(np.abs(eps[idx]))]
        check = np.concatenate([order[:400], order[400::97]])
        q = exact_sq(r[check], wk0[check])
        for k, qi in zip(check, q):
            assert qi > Fraction(float(T[k])) * (1 + Fraction(24, 2 ** 24)), (k, eps[k])
        # nothing inside the sphere is accepted
        assert not np.any(accept & (eps < 0))
        # every pair 1e-4 or more outside the sphere is accepted
        assert np.all(accept[eps >= 1e-4])


def test_bound_never_accepts_inside_near_cancellation():
    """Targets close to the present position (|d| far below |c|): |d|^2 + 2 d.c + |c|^2 cancels almost
    entirely against |c|^2, the regime where the FP32 terms' errors matter most."""
    rng = np.random.default_rng(7)
    n = 20000
    L = 10.0 ** rng.uniform(-6, -4, n)
    T = (L * L).astype(np.float32).astype(np.float64)
    origin = np.zeros((n, 3))
    wk0 = rng.normal(size=(n, 3)) * 1e-5
    cdir = rng.normal(size=(n, 3))
    cdir /= np.linalg.norm(cdir, axis=1, keepdims=True)
    wn = wk0 + cdir * (np.sqrt(T) * rng.uniform(0.9, 0.999999, n))[:, None]
    ddir = rng.normal(size=(n, 3))
    ddir /= np.linalg.norm(ddir, axis=1, keepdims=True)
    r = wn + ddir * (np.sqrt(T) * 10.0 ** rng.uniform(-7, -1, n))[:, None]
    for fused in (False, True):
        accept, D2k = bound_and_test(T, origin, wk0, wn, r, fused)
        q = np.array([float(x) for x in exact_sq(r, wk0)])
        # accepted pairs are outside with margin; pairs inside (or on) the sphere are never accepted
        assert np.all(q[accept] > T[accept] * (1 + 24 * U))
        assert np.all(D2k[accept].astype(np.float64) > T[accept])
        assert not np.any(accept & (q <= T))
