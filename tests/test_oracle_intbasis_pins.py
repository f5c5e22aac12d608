"""Pins of the oracle's interpolant bases (Sec. 3, Algorithms 4 and 5) -- CPU only.

M-IntBasis is checked against what the definition fixes: every row p of P satisfies
p(alpha_l) E_l = 0 (evaluated by Horner in tests/pyref.py); det P = lambda prod_l (x - alpha_l)^n
for generic E; P is s-ordered weak Popov with the returned s-row-degree; the row degrees sum to
n sigma for a generic uniform shift; over F_5 the module elements of bounded s-degree, counted by
enumeration, match the predictable-degree count.  PM-IntBasis equals M-IntBasis bit for bit for
every threshold (both are the canonical s-ordered weak Popov basis the algorithms produce).
"""
import itertools
import random

import numpy as np
import pytest

import oracle
from tests import pyref
from tests.test_oracle_pins import _rand_pmat, _rdeg_py, _weak_popov_pivots_on_diagonal

P60 = 1152921504606846883


def _points(rnd, p, k):
    pts = set()
    while len(pts) < k:
        pts.add(rnd.randrange(p))
    return sorted(pts, key=lambda _: rnd.random())


@pytest.mark.parametrize("p", [97, P60])
@pytest.mark.parametrize("mns", [(2, 1, 6), (4, 2, 9), (5, 3, 7), (6, 2, 13)])
def test_mintbasis_interpolant_properties(p, mns):
    m, n, sigma = mns
    rnd = random.Random(m * 100 + n * 10 + sigma)
    E = _rand_pmat(rnd, p, m, n, sigma)
    alpha = _points(rnd, p, sigma)
    for s in ([0] * m, [rnd.randrange(-3, 4) for _ in range(m)]):
        P, rd = oracle.mintbasis(p, E, alpha, s)
        for l, a in enumerate(alpha):
            Pa = pyref.eval_pmat(p, P.tolist(), a)
            El = [[int(E[i, j, l]) for j in range(n)] for i in range(m)]
            assert all(v == 0 for row in pyref.matmul(p, Pa, El) for v in row), l
        b1, b2 = 3, 5
        while b1 in alpha or b2 in alpha:
            b1, b2 = b1 + 2, b2 + 2
        D1 = pyref.det_mod(p, pyref.eval_pmat(p, P.tolist(), b1))
        D2 = pyref.det_mod(p, pyref.eval_pmat(p, P.tolist(), b2))
        W1, W2 = 1, 1
        for a in alpha:
            W1 = W1 * pow((b1 - a) % p, n, p) % p
            W2 = W2 * pow((b2 - a) % p, n, p) % p
        assert D1 != 0 and D1 * W2 % p == D2 * W1 % p
        assert _weak_popov_pivots_on_diagonal(P, s)
        assert list(rd) == _rdeg_py(P, s)
        if all(v == 0 for v in s) and p > 1000:
            assert sum(rd) == n * sigma


@pytest.mark.parametrize("p", [97, P60])
def test_pmintbasis_equals_mintbasis_for_every_threshold(p):
    rnd = random.Random(7)
    m, n, sigma = 4, 2, 19
    E = _rand_pmat(rnd, p, m, n, sigma)
    geo = [3 * pow(5, l, p) % p for l in range(sigma)]               # c q^l
    for alpha in (geo, _points(rnd, p, sigma)):
        s = [rnd.randrange(-2, 3) for _ in range(m)]
        P, rd = oracle.mintbasis(p, E, alpha, s)
        for T in (1, 2, 3, 5, 8, sigma):
            P2, rd2 = oracle.pmintbasis(p, E, alpha, s, T)
            assert np.array_equal(P2, P) and list(rd2) == list(rd), T


def test_mintbasis_dimension_counts_brute_force():
    """Over F_5, count interpolants of bounded s-degree by enumeration and compare with the
    predictable-degree count sum_i max(0, delta - rdeg_i + 1)."""
    p = 5
    rnd = random.Random(3)
    for (m, n, sigma, s) in ((2, 1, 3, (0, 0)), (2, 1, 4, (1, 0)), (3, 1, 2, (0, 0, 0)), (3, 2, 2, (0, 1, 0))):
        E = _rand_pmat(rnd, p, m, n, sigma)
        alpha = _points(rnd, p, sigma)
        P, rd = oracle.mintbasis(p, E, alpha, list(s))
        for delta in range(max(s), max(s) + 3):
            slots = [delta - sj + 1 if delta - sj >= 0 else 0 for sj in s]
            total = sum(slots)
            if p ** total > 200000:
                continue
            count = 0
            for vals in itertools.product(range(p), repeat=total):
                vec, pos = [], 0
                for j in range(m):
                    vec.append(list(vals[pos: pos + slots[j]]) or [0])
                    pos += slots[j]
                ok = all(sum(pyref.horner(p, vec[j], a) * int(E[j, c, l]) for j in range(m)) % p == 0
                         for l, a in enumerate(alpha) for c in range(n))
                count += ok
            dim = round(np.log(count) / np.log(p))
            assert p ** dim == count
            assert dim == sum(max(0, delta - int(r) + 1) for r in rd)


@pytest.mark.parametrize("p", [7, 97, P60])
def test_pmat_eval_is_the_power_sum(p):
    """oracle.pmat_eval (Horner) against sum_e X_e a^e taken with Python integers."""
    rnd = random.Random(p & 0xffff)
    X = _rand_pmat(rnd, p, 3, 4, 9)
    for a in (0, 1, p - 1, rnd.randrange(p)):
        got = oracle.pmat_eval(p, X, a)
        for i in range(3):
            for j in range(4):
                want = sum(int(X[i, j, e]) * pow(a, e, p) for e in range(9)) % p
                assert int(got[i, j]) == want
