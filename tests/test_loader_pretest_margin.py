"""The loader's float pre-test of the Maxwell-Juttner draw (ratio of
uniforms): evaluated in float32 in the kernel's order of operations
(a -> float, u = v/a, gamma - 1 = u^2/(sqrt(1 + u^2) + 1), times 1/theta in
float, 2 logf(a)), it may decide a round only when its two sides differ by
more than 4e-6 (|lhs| + |rhs|) + 1e-6.  Over a million rounds per
temperature no decision it takes differs from the FP64 test's, and it
leaves fewer than 1e-4 of the rounds to the FP64 test."""
import numpy as np
import pytest


@pytest.mark.parametrize("theta", [0.1, 0.3, 0.3 / 1836, 1.0, 3e-3])
def test_float_pretest_never_contradicts_fp64(theta):
    rng = np.random.default_rng(7)
    n = 1_000_000
    a = (rng.integers(0, 2 ** 53, n) + 1.0) * 2.0 ** -53
    w = 2.0 * ((rng.integers(0, 2 ** 53, n) + 1.0) * 2.0 ** -53) - 1.0
    gs = theta + np.sqrt(theta * theta + 1.0)
    bmax = np.sqrt(2 * theta * gs) * np.exp(-(gs - 1) / (2 * theta))
    vv = bmax * w
    u = vv / a
    exact = 2 * np.log(a) <= -(u * u / (np.sqrt(1 + u * u) + 1)) / theta
    f = np.float32
    af = a.astype(f)
    uf = (vv.astype(f) / af).astype(f)
    u2 = (uf * uf).astype(f)
    rf = (-(u2 / (np.sqrt(f(1) + u2).astype(f) + f(1))).astype(f) * (f(1) / f(theta))).astype(f)
    lf = (f(2) * np.log(af).astype(f)).astype(f)
    m = f(4e-6) * (np.abs(rf) + np.abs(lf)) + f(1e-6)
    acc, rej = lf <= rf - m, lf > rf + m
    assert not np.any(acc & ~exact) and not np.any(rej & exact)
    assert (acc | rej).mean() > 1 - 1e-4
