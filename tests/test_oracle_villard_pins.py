"""Pins of the oracle's Villard-variant resultant (Sec. 5.2, the variant of Algorithm 6 with
values of H, an interpolant basis of [H; -I] and det Q) -- CPU only.

The resultant is unique, so the output must equal the direct method's oracle (itself pinned by
root products, Sylvester determinants and the Poisson formula in tests/test_oracle_pins.py) and
must agree with det of the Sylvester matrix computed in pure Python at sample points
(tests/pyref.py), for every block size m, unequal degrees and several primes.  A common factor
of f and g makes Res identically zero: no point is usable and the oracle reports it.
"""
import random

import numpy as np
import pytest

import oracle
import synth
from tests import pyref

P60 = 1152921504606846883


def _fg(seed, p, dxf, dyf, dxg, dyg):
    g = synth.rng(seed)
    return synth.uniform(g, (dyf + 1, dxf + 1), p, np.uint64), synth.uniform(g, (dyg + 1, dxg + 1), p, np.uint64)


CASES = [
    # p, dxf, dyf, dxg, dyg, m
    (P60, 6, 6, 6, 6, 2),
    (P60, 12, 12, 12, 12, 0),
    (P60, 9, 5, 4, 7, 3),
    (998244353, 10, 7, 10, 7, 1),
    (10007, 5, 6, 7, 4, 2),
    (P60, 3, 8, 3, 8, 4),
    (P60, 8, 3, 8, 3, 3),
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_{c[1]}x{c[2]}_{c[3]}x{c[4]}_m{c[5]}" for c in CASES])
def test_villard_equals_direct_method(case):
    p, dxf, dyf, dxg, dyg, m = case
    f, g = _fg(sum(case) & 0xffff, p, dxf, dyf, dxg, dyg)
    assert np.array_equal(oracle.bivariate_resultant_villard(p, f, g, m), oracle.bivariate_resultant(p, f, g))


@pytest.mark.parametrize("p", [10007, P60])
def test_villard_matches_sylvester_determinants(p):
    dxf, dyf, dxg, dyg = 4, 5, 3, 4
    f, g = _fg(p % 1000, p, dxf, dyf, dxg, dyg)
    R = oracle.bivariate_resultant_villard(p, f, g, 2)
    rnd = random.Random(5)
    for _ in range(4):
        x = rnd.randrange(p)
        fa = [pyref.horner(p, f[j], x) for j in range(dyf + 1)]
        ga = [pyref.horner(p, g[j], x) for j in range(dyg + 1)]
        assert pyref.horner(p, R, x) == pyref.det_mod(p, pyref.sylvester(fa, ga))


def test_villard_common_factor_has_no_usable_point():
    p = 10007
    h = np.array([[3, 1], [2, 0]], dtype=np.uint64)            # 3 + x + 2 z
    f0, g0 = _fg(3, p, 2, 2, 2, 2)
    # f = h f0, g = h g0 as bivariate products
    fx = np.zeros((4, 4), dtype=np.uint64)
    gx = np.zeros((4, 4), dtype=np.uint64)
    for j1 in range(2):
        for i1 in range(2):
            for j2 in range(3):
                for i2 in range(3):
                    fx[j1 + j2, i1 + i2] = (int(fx[j1 + j2, i1 + i2]) + int(h[j1, i1]) * int(f0[j2, i2])) % p
                    gx[j1 + j2, i1 + i2] = (int(gx[j1 + j2, i1 + i2]) + int(h[j1, i1]) * int(g0[j2, i2])) % p
    with pytest.raises(ValueError):
        oracle.bivariate_resultant_villard(p, fx, gx, 2)


def test_villard_non_generic_input_is_reported():
    """f constant in x: the denominator of H is a proper factor of Res, det Q is no longer a
    constant multiple of it, and the oracle's check against Res at the delta points reports it
    (the direct method still gives the resultant)."""
    p = P60
    f, g = _fg(15, p, 0, 5, 4, 6)
    with pytest.raises(ValueError, match="not generic"):
        oracle.bivariate_resultant_villard(p, f, g, 0)
    assert oracle.bivariate_resultant(p, f, g).any()
