"""The pivot reciprocal of the eliminations (one third-order step r (1 + e + e^2) from a
single-precision seed, qcs_common.cuh) against the correctly rounded 1/d of the host's IEEE
division: every pivot step of every FP64 path divides by |pivot|^2 through it, so its error
enters each Gauss vector.  Bound: 2 ulp (the step's truncation error e^3 < 2^-57 plus the
last FMA's rounding); the values outside the seed's exponent range take the device's IEEE
division and must match exactly."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2506_22408_gb300 import qcs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def ulp_distance(a, b):
    """Distance in units in the last place between non-negative finite doubles."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_reciprocal_within_two_ulp_over_the_seed_range(ctx):
    rng = np.random.default_rng(21)
    # mantissas uniform in [1, 2), exponents over the whole seed range and beyond
    m = 1.0 + rng.random(200_000)
    e = rng.integers(-140, 141, size=m.size)
    d = np.ldexp(m, e)
    # powers of two, values next to them, and the edges of the seed's exponent range
    edges = np.ldexp(1.0, np.arange(-130, 131))
    d = np.concatenate([d, edges, np.nextafter(edges, 0), np.nextafter(edges, np.inf)])
    r = ctx.selftest_reciprocal(torch.from_numpy(d).cuda()).cpu().numpy()
    want = 1.0 / d
    dist = ulp_distance(r, want)
    assert dist.max() <= 2, (dist.max(), d[np.argmax(dist)])
    # most results are the correctly rounded ones
    assert (dist == 0).mean() > 0.9


def test_reciprocal_outside_the_seed_range_is_the_division(ctx):
    d = np.array([0.0, 5e-324, 1e-310, 2.0 ** -126, 2.0 ** -400, 2.0 ** 126, 1e300, np.inf, np.nan])
    r = ctx.selftest_reciprocal(torch.from_numpy(d).cuda()).cpu().numpy()
    with np.errstate(divide="ignore", over="ignore"):
        want = 1.0 / d
    assert np.isposinf(r[0]) and np.isnan(r[-1]) and r[-2] == 0.0
    fin = np.isfinite(want)
    assert np.array_equal(r[fin], want[fin])


def test_reciprocal_rejects_bad_arguments(ctx):
    with pytest.raises(ValueError):
        ctx.selftest_reciprocal(torch.ones(4, dtype=torch.float32, device="cuda"))
    r = ctx.selftest_reciprocal(torch.empty(0, dtype=torch.float64, device="cuda"))
    assert r.numel() == 0
