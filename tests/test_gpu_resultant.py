"""GPU parity of bivariate_resultant (direct method, Sec. 5.2) against the oracle."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P60 = 1152921504606846883
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


def _gpu(ctx, primes, fs, gs):
    from paper_1905_04356_gb300 import pmat
    f = pmat.to_device(np.stack(fs))
    g = pmat.to_device(np.stack(gs))
    R = pmat.bivariate_resultant(ctx, primes, f, g)
    ctx.sync()
    return pmat.to_host(R)


@pytest.mark.parametrize("degs", [(1, 1, 1, 1), (2, 3, 3, 2), (0, 2, 2, 1), (5, 4, 3, 6), (20, 20, 20, 20),
                                  (40, 30, 25, 35), (7, 0, 3, 5)])
def test_resultant_matches_oracle(ctx, degs):
    dxf, dyf, dxg, dyg = degs
    g0 = synth.rng(sum(degs))
    primes = [P60, synth.random_prime(g0, 60), synth.random_prime(g0, 50)]
    fs, gs, exp = [], [], []
    for p in primes:
        f = synth.uniform(g0, (dyf + 1, dxf + 1), p, np.uint64)
        g = synth.uniform(g0, (dyg + 1, dxg + 1), p, np.uint64)
        f[dyf, 0] = max(int(f[dyf, 0]), 1)   # leading y-coefficient not identically zero
        g[dyg, 0] = max(int(g[dyg, 0]), 1)
        fs.append(f); gs.append(g); exp.append(oracle.bivariate_resultant(p, f, g))
    got = _gpu(ctx, primes, fs, gs)
    for i in range(len(primes)):
        assert np.array_equal(got[i], exp[i]), (degs, i)


def test_leading_coefficient_vanishing_at_one(ctx):
    """lc_y(f) = x - 1 vanishes at x = 1, the first point of every progression:
    the device must move to scaled points and still match."""
    p = 10007
    g0 = synth.rng(5)
    f = synth.uniform(g0, (3, 3), p, np.uint64)
    f[2] = [p - 1, 1, 0]
    g = synth.uniform(g0, (3, 3), p, np.uint64)
    g[2, 2] = 1
    got = _gpu(ctx, [p], [f], [g])
    assert np.array_equal(got[0], oracle.bivariate_resultant(p, f, g))


def test_resultant_150_full_size(ctx):
    """deg_x = deg_y = 150, 60-bit prime: the whole output against the oracle's fingerprint."""
    gold = json.load(open(GOLDEN))["resultant_150"]
    W = synth.resultant_c5(0, nprimes=1)
    assert W["primes"][0] == gold["p"]
    got = _gpu(ctx, W["primes"], W["f"], W["g"])[0]
    assert list(got.shape) == gold["shape"]
    for i, v in gold["samples"]:
        assert int(got[i]) == v
    assert hashlib.sha256(np.ascontiguousarray(got).tobytes()).hexdigest() == gold["sha256"]


def test_resultant_16_prime_batch(ctx):
    """The same integer inputs modulo 16 primes: every instance's whole output against the
    oracle's fingerprint for its prime (tests/golden/make_golden.py, one oracle resultant per
    prime), plus sampled coefficients."""
    gold = json.load(open(GOLDEN))["resultant_150_16primes"]
    W = synth.resultant_c5(0, nprimes=16)
    assert [int(p) for p in W["primes"]] == gold["primes"]
    got = _gpu(ctx, W["primes"], W["f"], W["g"])
    assert list(got.shape) == gold["shape"]
    for i in range(16):
        for j, v in gold["samples"][i]:
            assert int(got[i][j]) == v, (i, j)
        assert hashlib.sha256(np.ascontiguousarray(got[i]).tobytes()).hexdigest() == gold["sha256"][i], i
