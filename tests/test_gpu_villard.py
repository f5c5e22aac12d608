"""GPU parity of bivariate_resultant_villard (Sec. 5.2, the variant of Algorithm 6: values of
a block of the inverse Sylvester matrix by one extended Euclid per point, PM-IntBasis on
[H; -I], det Q at geometric points, normalisation) against the oracle.

The resultant is unique, so the device output must equal the oracle's resultant bit for bit:
small shapes against both oracle methods, every block size m including m = 1 (scalar
reconstruction), unequal degrees, and the deg 150 / 150 workload against the fingerprint of
the oracle's output.  A common factor makes Res vanish at every point: no progression is
usable and the call reports it.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P60 = 1152921504606846883
P62 = 4611686018427387847
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "golden.json")


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_04356_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def _gpu(ctx, primes, fs, gs, m=0):
    from paper_1905_04356_gb300 import pmat
    f = pmat.to_device(np.stack(fs))
    g = pmat.to_device(np.stack(gs))
    R = pmat.bivariate_resultant_villard(ctx, primes, f, g, m)
    ctx.sync()
    return pmat.to_host(R)


def _fg(seed, p, dxf, dyf, dxg, dyg):
    g = synth.rng(seed)
    return synth.uniform(g, (dyf + 1, dxf + 1), p, np.uint64), synth.uniform(g, (dyg + 1, dxg + 1), p, np.uint64)


CASES = [
    # p, dxf, dyf, dxg, dyg, m
    (P60, 6, 6, 6, 6, 2),
    (P60, 12, 12, 12, 12, 0),
    (P60, 9, 5, 4, 7, 3),
    (synth.P998, 10, 7, 10, 7, 1),
    (P60, 3, 8, 3, 8, 4),
    (P60, 8, 3, 8, 3, 3),
    (P62, 20, 20, 20, 20, 0),
    (P60, 1, 1, 1, 1, 1),
    (P60, 40, 30, 35, 25, 5),
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_{c[1]}x{c[2]}_{c[3]}x{c[4]}_m{c[5]}" for c in CASES])
def test_villard_matches_oracle(ctx, case):
    p, dxf, dyf, dxg, dyg, m = case
    f, g = _fg(sum(case) & 0xffff, p, dxf, dyf, dxg, dyg)
    got = _gpu(ctx, [p], [f], [g], m)[0]
    want = oracle.bivariate_resultant(p, f, g)
    assert np.array_equal(got, want)
    if dxf + dyf <= 24:
        assert np.array_equal(got, oracle.bivariate_resultant_villard(p, f, g, m))


def test_villard_150_full_size(ctx):
    """deg_x = deg_y = 150, 60-bit prime, m = 8: the whole output against the oracle's fingerprint."""
    gold = json.load(open(GOLDEN))["resultant_150"]
    W = synth.resultant_c5(0, nprimes=1)
    got = _gpu(ctx, W["primes"], W["f"], W["g"])[0]
    assert list(got.shape) == gold["shape"]
    for i, v in gold["samples"]:
        assert int(got[i]) == v
    assert hashlib.sha256(np.ascontiguousarray(got).tobytes()).hexdigest() == gold["sha256"]


def test_villard_two_primes(ctx):
    f1, g1 = _fg(11, P60, 7, 6, 7, 6)
    f2, g2 = _fg(12, P62, 7, 6, 7, 6)
    got = _gpu(ctx, [P60, P62], [f1, f2], [g1, g2])
    assert np.array_equal(got[0], oracle.bivariate_resultant(P60, f1, g1))
    assert np.array_equal(got[1], oracle.bivariate_resultant(P62, f2, g2))


def test_villard_common_factor_is_reported(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    p = P60
    f0, g0 = _fg(3, p, 2, 2, 2, 2)
    h = [[3, 1], [2, 0]]                                     # 3 + x + 2 y
    f = np.zeros((4, 4), dtype=np.uint64)
    g = np.zeros((4, 4), dtype=np.uint64)
    for j1 in range(2):
        for i1 in range(2):
            for j2 in range(3):
                for i2 in range(3):
                    f[j1 + j2, i1 + i2] = (int(f[j1 + j2, i1 + i2]) + h[j1][i1] * int(f0[j2, i2])) % p
                    g[j1 + j2, i1 + i2] = (int(g[j1 + j2, i1 + i2]) + h[j1][i1] * int(g0[j2, i2])) % p
    with pytest.raises(PmError) as e:
        _gpu(ctx, [p], [f], [g], 2)
    assert e.value.code == pmat.PM_EUNSUPPORTED


def test_villard_rejects_bad_arguments(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    f, g = _fg(1, P60, 3, 0, 3, 2)                           # y-degree 0
    with pytest.raises(PmError) as e:
        _gpu(ctx, [P60], [f], [g], 1)
    assert e.value.code == pmat.PM_EINVAL


@pytest.mark.parametrize("degs", [(6, 4, 0, 5), (3, 2, 3, 2)], ids=["g_const_in_x", "small"])
def test_villard_degenerate_x_degrees(ctx, degs):
    """g constant in x, and a small case with m = 2: the resultant equals the direct method's."""
    dxf, dyf, dxg, dyg = degs
    f, g = _fg(sum(degs), P60, dxf, dyf, dxg, dyg)
    got = _gpu(ctx, [P60], [f], [g], 0)[0]
    assert np.array_equal(got, oracle.bivariate_resultant(P60, f, g))


def test_villard_non_generic_input_is_refused(ctx):
    """f constant in x (degrees 0 / 5 against 4 / 6): H's denominator is a proper factor of Res,
    the oracle's own check reports the input as not generic, and the device's check of the
    normalised det Q against Res at the delta points must refuse it (PM_EUNSUPPORTED) rather
    than return a wrong resultant."""
    from paper_1905_04356_gb300 import PmError, pmat
    f, g = _fg(15, P60, 0, 5, 4, 6)
    with pytest.raises(ValueError, match="not generic"):
        oracle.bivariate_resultant_villard(P60, f, g, 0)
    with pytest.raises(PmError) as e:
        _gpu(ctx, [P60], [f], [g], 0)
    assert e.value.code == pmat.PM_EUNSUPPORTED
