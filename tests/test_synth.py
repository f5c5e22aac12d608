"""The seeded input generators (synth.py, no arithmetic of the method): determinism, the
60-bit prime draw, value ranges, widths and the batch recipe."""
import numpy as np
import pytest

import synth


def test_same_seed_same_inputs_and_different_seed_different_inputs():
    a, b, c = synth.product_c2(0, m=4, d=64), synth.product_c2(0, m=4, d=64), synth.product_c2(1, m=4, d=64)
    assert a["p"] == b["p"] and np.array_equal(a["A"], b["A"]) and np.array_equal(a["B"], b["B"])
    assert a["p"] != c["p"] or not np.array_equal(a["A"], c["A"])


@pytest.mark.parametrize("seed", [0, 1, 7])
def test_random_60_bit_prime(seed):
    sympy = pytest.importorskip("sympy")
    p = synth.random_prime(synth.rng(seed), 60)
    assert (1 << 59) <= p < (1 << 60) and p % 2 == 1
    assert sympy.isprime(p)


def test_primality_test_against_sympy():
    sympy = pytest.importorskip("sympy")
    g = np.random.default_rng(3)
    for n in [0, 1, 2, 3, 4, 561, 1105, 998244353, (1 << 61) - 1, 3215031751, 2152302898747] + \
            [int(x) for x in g.integers(1, 1 << 62, size=200, dtype=np.uint64)]:
        assert synth.is_prime(n) == sympy.isprime(n), n


def test_values_are_reduced_and_width_follows_the_modulus():
    g = synth.rng(5)
    x = synth.uniform(g, (3, 4, 100), 97)
    assert x.dtype == np.uint32 and int(x.max()) < 97
    y = synth.uniform(g, (2, 2, 50), synth.random_prime(g, 60))
    assert y.dtype == np.uint64


def test_bench_workload_shapes():
    W = synth.product_c2(0)
    assert W["A"].shape == (32, 32, 4096) and W["B"].shape == (32, 32, 4096) and W["A"].dtype == np.uint64
    W2 = synth.product_c2(0, ntt_prime=True, m=2, d=8)
    assert W2["p"] == synth.P998 and W2["A"].dtype == np.uint32


def test_batch_recipe():
    items = synth.batch_c4(0, count=64)
    assert len(items) == 64
    for i, it in enumerate(items):
        assert 2 <= min(it["m"], it["n"], it["k"]) and max(it["m"], it["n"], it["k"]) <= 64
        assert 64 <= it["d"] <= 16384
        assert (it["p"] == synth.P998) == (i % 2 == 0)
        assert it["A"].shape == (it["m"], it["n"], it["d"]) and it["B"].shape == (it["n"], it["k"], it["d"])
