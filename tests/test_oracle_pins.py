"""Pins of the CPU oracle against things other than itself (CPU only).

Products (Sec. 2): Kronecker-substitution products, random-point identities
(Schwartz-Zippel), closed forms, identity / shift matrices, extreme values.
Algorithm 1: the t-Popov conditions + basis certificate (Q.R = 0 mod x and
det Q = x^rank).  Algorithms 2-3: P.F = 0 mod x^d, deg det P = n d for generic
F, s-ordered weak Popov pivots, brute-force dimension counts of the module
over tiny fields, and PM-Basis == M-Basis for every threshold.
Resultants (Sec. 5.2): Res(prod(y-a_i), prod(y-b_j)) = prod(a_i - b_j),
Sylvester determinants, the Poisson product formula for bivariate inputs.
"""
import itertools
import random

import numpy as np
import pytest

import oracle
import synth
from tests import pyref

P60 = 1152921504606846883  # 2^60 - 93, checked prime below
P62 = 4611686018427387847  # 2^62 - 57, checked prime below


def test_test_primes_are_prime():
    assert synth.is_prime(P60) and synth.is_prime(P62) and synth.is_prime(synth.P998)
    assert not synth.is_prime(P60 + 2)


def _rand_pmat(rnd, p, r, c, length):
    return np.array([[[rnd.randrange(p) for _ in range(length)] for _ in range(c)] for _ in range(r)],
                    dtype=np.uint64)


# ============================================================ products
@pytest.mark.parametrize("p", [5, 97, synth.P998, P60, P62])
@pytest.mark.parametrize("shape", [(1, 1, 1, 1, 1), (3, 2, 4, 7, 5), (2, 3, 1, 1, 9), (4, 4, 4, 6, 6)])
def test_product_matches_kronecker_substitution(p, shape):
    m, n, k, dA, dB = shape
    rnd = random.Random(hash((p, shape)) & 0xffff)
    A = _rand_pmat(rnd, p, m, n, dA)
    B = _rand_pmat(rnd, p, n, k, dB)
    ref = np.array(pyref.ks_pmat_mul(p, A.tolist(), B.tolist()), dtype=np.uint64)
    full = oracle.pmat_mul(p, A, B)
    assert np.array_equal(full, ref)
    # truncation: prefix of the exact product, zero beyond its length
    for t in (1, (dA + dB) // 2, dA + dB - 1, dA + dB + 3):
        tr = oracle.pmat_mul_trunc(p, A, B, t)
        exp = np.zeros((m, k, t), dtype=np.uint64)
        L = min(t, dA + dB - 1)
        exp[:, :, :L] = ref[:, :, :L]
        assert np.array_equal(tr, exp)
    # middle product: the slice of degrees c..c+d-1
    for c, d in ((0, 1), (dA - 1, dB - dA + 1 if dB >= dA else 1), (1, dA + dB - 2)):
        if d <= 0:
            continue
        mp = oracle.pmat_middle_product(p, A, B, c, d)
        exp = np.zeros((m, k, d), dtype=np.uint64)
        hi = min(c + d, dA + dB - 1)
        if hi > c:
            exp[:, :, : hi - c] = ref[:, :, c:hi]
        assert np.array_equal(mp, exp)
    # single coefficients
    for _ in range(5):
        i, kk, t = rnd.randrange(m), rnd.randrange(k), rnd.randrange(dA + dB - 1)
        assert oracle.pmat_coeff(p, A, B, i, kk, t) == int(ref[i, kk, t])


def test_scalar_degree_zero_brute_force():
    for p in (2, 3, 7, synth.P998, P60, P62):
        for a, b in ((0, 0), (1, p - 1), (p - 1, p - 1), (p // 2, p // 3)):
            A = np.array([[[a]]], dtype=np.uint64)
            B = np.array([[[b]]], dtype=np.uint64)
            assert int(oracle.pmat_mul(p, A, B)[0, 0, 0]) == a * b % p


@pytest.mark.parametrize("p", [synth.P998, P60])
def test_random_point_identity(p):
    """C(alpha) = A(alpha) B(alpha) for random alpha (Schwartz-Zippel)."""
    rnd = random.Random(7)
    m, n, k, dA, dB = 5, 3, 2, 40, 33
    A = _rand_pmat(rnd, p, m, n, dA)
    B = _rand_pmat(rnd, p, n, k, dB)
    Cf = oracle.pmat_mul(p, A, B)
    for _ in range(3):
        x = rnd.randrange(p)
        lhs = pyref.eval_pmat(p, Cf.tolist(), x)
        rhs = pyref.matmul(p, pyref.eval_pmat(p, A.tolist(), x), pyref.eval_pmat(p, B.tolist(), x))
        assert lhs == rhs


def test_transposed_operand_is_caught():
    """A plausible mistake (swapping the operand order) changes the result."""
    p = 97
    rnd = random.Random(3)
    A = _rand_pmat(rnd, p, 2, 2, 3)
    B = _rand_pmat(rnd, p, 2, 2, 3)
    assert not np.array_equal(oracle.pmat_mul(p, A, B), oracle.pmat_mul(p, B, A))


def test_binomial_closed_form():
    p = synth.P998
    import math
    a, b = 37, 52
    A = np.array([[[math.comb(a, i) % p for i in range(a + 1)]]], dtype=np.uint64)
    B = np.array([[[math.comb(b, i) % p for i in range(b + 1)]]], dtype=np.uint64)
    C = oracle.pmat_mul(p, A, B)[0, 0]
    assert [int(v) for v in C] == [math.comb(a + b, i) % p for i in range(a + b + 1)]


def test_geometric_closed_form():
    p = P60
    n = 50
    A = np.array([[[1, p - 1]]], dtype=np.uint64)          # 1 - x
    B = np.ones((1, 1, n), dtype=np.uint64)                   # 1 + x + ... + x^(n-1)
    C = oracle.pmat_mul(p, A, B)[0, 0]
    exp = [1] + [0] * (n - 1) + [p - 1]                       # 1 - x^n
    assert [int(v) for v in C] == exp


def test_identity_and_shift():
    p = P60
    rnd = random.Random(11)
    m, n, d = 3, 4, 9
    A = _rand_pmat(rnd, p, m, n, d)
    I = np.zeros((n, n, 1), dtype=np.uint64)
    for i in range(n):
        I[i, i, 0] = 1
    assert np.array_equal(oracle.pmat_mul(p, A, I), A)
    s = 4
    Xs = np.zeros((m, m, s + 1), dtype=np.uint64)
    for i in range(m):
        Xs[i, i, s] = 1
    C = oracle.pmat_mul(p, Xs, A)
    assert np.array_equal(C[:, :, s:], A) and not C[:, :, :s].any()


def test_overflow_extremes():
    """All coefficients p-1 with long inner sums: exact against big integers."""
    for p in (P60, P62):
        m, n, k, dA, dB = 2, 40, 2, 300, 300
        A = np.full((m, n, dA), p - 1, dtype=np.uint64)
        B = np.full((n, k, dB), p - 1, dtype=np.uint64)
        C = oracle.pmat_mul(p, A, B)
        for t in (0, 150, 299, 450, 598):
            terms = min(t, dA - 1) - max(0, t - dB + 1) + 1
            assert int(C[0, 1, t]) == (n * terms * (p - 1) ** 2) % p


# ============================================================ Algorithm 1
def _popov_checks(p, R, t, Q, rank):
    """Q is the t-Popov approximant basis of (R, order 1)."""
    m, n = R.shape
    Q0 = Q[:, :, 0].astype(object)
    Q1 = Q[:, :, 1].astype(object)
    # Q.R = 0 mod x  <=>  Q(0).R = 0
    prod = pyref.matmul(p, Q0.tolist(), R.astype(object).tolist())
    assert all(v == 0 for row in prod for v in row)
    # rank agrees with an independent elimination, det Q = x^rank
    assert rank == pyref.rank_mod(p, R.tolist())
    for x in (2, 3, 5):
        if x >= p:
            continue
        Qx = [[(int(Q0[i][j]) + int(Q1[i][j]) * x) % p for j in range(m)] for i in range(m)]
        assert pyref.det_mod(p, Qx) == pow(x, rank, p)
    # t-Popov: the t-pivot (rightmost entry reaching the t-degree) of row i is
    # on the diagonal, pivots are monic, and each pivot has degree larger than
    # every other entry of its column.
    def deg(i, j):
        if Q1[i][j]:
            return 1
        return 0 if Q0[i][j] else -1
    for i in range(m):
        rd = max(deg(i, j) + t[j] for j in range(m) if deg(i, j) >= 0)
        piv = max(j for j in range(m) if deg(i, j) >= 0 and deg(i, j) + t[j] == rd)
        assert piv == i
        lead = Q1[i][i] if deg(i, i) == 1 else Q0[i][i]
        assert lead == 1
        for r in range(m):
            if r != i:
                assert deg(r, i) < deg(i, i)


@pytest.mark.parametrize("p", [2, 3, 5, 97, P60])
def test_mbasis1_is_t_popov(p):
    rnd = random.Random(p % 1000)
    for trial in range(40):
        m = rnd.randrange(1, 7)
        n = rnd.randrange(1, 5)
        R = np.array([[rnd.randrange(p) if rnd.random() < 0.8 else 0 for _ in range(n)]
                      for _ in range(m)], dtype=np.uint64)
        if trial % 5 == 0:            # rank-deficient rows: duplicate / scaled rows
            R[-1] = R[0] * 2 % p
        t = [rnd.randrange(-2, 3) for _ in range(m)]
        Q, rank = oracle.mbasis1(p, R, t)
        _popov_checks(p, R, t, Q, rank)


# ============================================================ Algorithms 2 and 3
def _series_product_mod(p, P, F, d):
    """P.F mod x^d with Kronecker substitution (pure Python)."""
    C = pyref.ks_pmat_mul(p, P.tolist(), F.tolist())
    return [[row[:d] for row in Ci] for Ci in C]


def _rdeg_py(P, s):
    m, c, L = P.shape
    out = []
    for i in range(m):
        best = None
        for j in range(c):
            nz = np.nonzero(P[i, j])[0]
            if len(nz):
                v = int(nz[-1]) + int(s[j])
                best = v if best is None else max(best, v)
        out.append(best)
    return out


def _weak_popov_pivots_on_diagonal(P, s):
    m = P.shape[0]
    rd = _rdeg_py(P, s)
    for i in range(m):
        piv = None
        for j in range(m):
            nz = np.nonzero(P[i, j])[0]
            if len(nz) and int(nz[-1]) + int(s[j]) == rd[i]:
                piv = j
        if piv != i:
            return False
    return True


@pytest.mark.parametrize("p", [97, P60])
@pytest.mark.parametrize("mnd", [(2, 1, 6), (4, 2, 9), (5, 3, 7), (6, 2, 13)])
def test_mbasis_approximant_properties(p, mnd):
    m, n, d = mnd
    rnd = random.Random(m * 100 + n * 10 + d)
    F = _rand_pmat(rnd, p, m, n, d + 2)
    for s in ([0] * m, [rnd.randrange(-3, 4) for _ in range(m)]):
        P, rd = oracle.mbasis(p, F, d, s)
        # P.F = 0 mod x^d
        prod = _series_product_mod(p, P, F, d)
        assert all(v == 0 for Ci in prod for row in Ci for v in row)
        # deg det P = n d, det P = lambda x^(n d) (generic F, checked at 2 points)
        x1, x2 = 3, 5
        D1 = pyref.det_mod(p, pyref.eval_pmat(p, P.tolist(), x1))
        D2 = pyref.det_mod(p, pyref.eval_pmat(p, P.tolist(), x2))
        assert D1 != 0 and D2 != 0
        assert D1 * pow(x2, n * d, p) % p == D2 * pow(x1, n * d, p) % p
        # s-ordered weak Popov, and the returned s-row-degree
        assert _weak_popov_pivots_on_diagonal(P, s)
        assert list(rd) == _rdeg_py(P, s)
        # generic uniform shift: sum of row degrees = n d
        if all(v == 0 for v in s) and p > 1000:
            assert sum(rd) == n * d


@pytest.mark.parametrize("p", [97, P60])
def test_pmbasis_equals_mbasis_for_every_threshold(p):
    rnd = random.Random(5)
    for (m, n, d) in ((4, 2, 16), (3, 1, 11), (6, 3, 20), (5, 2, 33)):
        F = _rand_pmat(rnd, p, m, n, d)
        for s in ([0] * m, [rnd.randrange(-4, 5) for _ in range(m)]):
            P, rd = oracle.mbasis(p, F, d, s)
            for T in (1, 2, 3, 5, 8, d):
                P2, rd2 = oracle.pmbasis(p, F, d, s, T=T)
                assert np.array_equal(P, P2), (m, n, d, T)
                assert np.array_equal(rd, rd2)


def test_mbasis_dimension_counts_brute_force():
    """Over F_3, count module elements of bounded s-degree by enumeration and
    compare with the predictable-degree count sum_i max(0, delta - rdeg_i + 1)."""
    p = 3
    rnd = random.Random(1)
    for (m, n, d, s) in ((2, 1, 3, (0, 0)), (2, 1, 4, (1, 0)), (3, 1, 2, (0, 0, 0)), (3, 2, 2, (0, 1, 0))):
        F = _rand_pmat(rnd, p, m, n, d)
        P, rd = oracle.mbasis(p, F, d, list(s))
        for delta in range(max(s), max(s) + 3):
            bounds = [delta - sj for sj in s]
            if min(bounds) < -1:
                continue
            slots = [b + 1 if b >= 0 else 0 for b in bounds]
            total = sum(slots)
            if p ** total > 60000:
                continue
            count = 0
            for vals in itertools.product(range(p), repeat=total):
                vec, pos = [], 0
                for j in range(m):
                    vec.append(list(vals[pos: pos + slots[j]]) or [0])
                    pos += slots[j]
                ok = True
                for c in range(n):
                    acc = [0] * d
                    for j in range(m):
                        prod = pyref.ks_polymul(vec[j], [int(v) for v in F[j, c]])
                        for t in range(min(d, len(prod))):
                            acc[t] += prod[t]
                    if any(v % p for v in acc):
                        ok = False
                        break
                count += ok
            dim = round(np.log(count) / np.log(p))
            assert p ** dim == count
            assert dim == sum(max(0, delta - int(r) + 1) for r in rd)


# ============================================================ resultants
@pytest.mark.parametrize("p", [101, synth.P998, P60])
def test_univariate_resultant_root_product(p):
    rnd = random.Random(p % 977)
    for _ in range(10):
        a = [rnd.randrange(p) for _ in range(rnd.randrange(1, 8))]
        b = [rnd.randrange(p) for _ in range(rnd.randrange(1, 8))]
        if rnd.random() < 0.3:
            b[0] = a[0]                     # a common root: resultant 0
        A, B = [1], [1]
        for r in a:
            A = pyref.pmul(p, A, [(-r) % p, 1])
        for r in b:
            B = pyref.pmul(p, B, [(-r) % p, 1])
        exp = 1
        for x in a:
            for y in b:
                exp = exp * (x - y) % p
        assert oracle.univ_resultant(p, A, B) == exp


@pytest.mark.parametrize("p", [7, 101, P60])
def test_univariate_resultant_sylvester(p):
    rnd = random.Random(p % 1013)
    for _ in range(30):
        da, db = rnd.randrange(0, 7), rnd.randrange(0, 7)
        A = [rnd.randrange(p) for _ in range(da)] + [rnd.randrange(1, p)]
        B = [rnd.randrange(p) for _ in range(db)] + [rnd.randrange(1, p)]
        exp = pyref.det_mod(p, pyref.sylvester(A, B)) if da + db else 1
        assert oracle.univ_resultant(p, A, B) == exp


def _bivariate_sylvester_reference(p, f, g):
    """det of the Sylvester matrix in y over F_p[x]: values at D+1 points, Lagrange."""
    dyf, dxf = f.shape[0] - 1, f.shape[1] - 1
    dyg, dxg = g.shape[0] - 1, g.shape[1] - 1
    D = dxf * dyg + dxg * dyf
    xs = list(range(p - 1, p - 2 - D, -1))      # points from the top: no overlap with the oracle's
    ys = []
    for x in xs:
        fa = [pyref.horner(p, f[j], x) for j in range(dyf + 1)]
        ga = [pyref.horner(p, g[j], x) for j in range(dyg + 1)]
        ys.append(pyref.det_mod(p, pyref.sylvester(fa, ga)) if dyf + dyg else 1)
    return pyref.lagrange(p, xs, ys)


@pytest.mark.parametrize("p", [10007, P60])
def test_bivariate_resultant_sylvester_tiny(p):
    rnd = random.Random(3)
    for (dxf, dyf, dxg, dyg) in ((1, 1, 1, 1), (2, 3, 3, 2), (3, 2, 1, 3), (0, 2, 2, 1), (2, 1, 0, 1)):
        f = np.array([[rnd.randrange(p) for _ in range(dxf + 1)] for _ in range(dyf + 1)], dtype=np.uint64)
        g = np.array([[rnd.randrange(p) for _ in range(dxg + 1)] for _ in range(dyg + 1)], dtype=np.uint64)
        R = oracle.bivariate_resultant(p, f, g)
        assert [int(v) for v in R] == _bivariate_sylvester_reference(p, f, g)


def test_bivariate_resultant_skips_vanishing_leading_coefficients():
    """lc_y(f) = x (x - 1) vanishes at the first two points; the result must not change."""
    p = 10007
    rnd = random.Random(9)
    dxf, dyf, dxg, dyg = 2, 2, 2, 2
    f = np.array([[rnd.randrange(p) for _ in range(dxf + 1)] for _ in range(dyf + 1)], dtype=np.uint64)
    f[dyf] = [0, p - 1, 1]           # x^2 - x
    g = np.array([[rnd.randrange(p) for _ in range(dxg + 1)] for _ in range(dyg + 1)], dtype=np.uint64)
    R = oracle.bivariate_resultant(p, f, g)
    assert [int(v) for v in R] == _bivariate_sylvester_reference(p, f, g)


def test_bivariate_resultant_poisson_formula():
    """f = prod_i (y - a_i(x)), a_i linear: Res_y(f, g) = prod_i g(x, a_i(x))."""
    p = P60
    rnd = random.Random(21)
    dyf, dxg, dyg = 3, 4, 3
    roots = [[rnd.randrange(p), rnd.randrange(p)] for _ in range(dyf)]   # a_i(x) = r0 + r1 x
    # f as a polynomial in y with coefficients in F_p[x] (lists, low first)
    fy = [[1]]
    for r in roots:
        lin = [[(-r[0]) % p, (-r[1]) % p], [1]]    # (y - a_i(x))
        new = [[0] for _ in range(len(fy) + 1)]
        for j, cj in enumerate(fy):
            for e, ce in enumerate(lin):
                new[j + e] = pyref.padd(p, new[j + e], pyref.pmul(p, cj, ce))
        fy = new
    dxf = max(len(c) for c in fy) - 1
    f = np.zeros((dyf + 1, dxf + 1), dtype=np.uint64)
    for j, c in enumerate(fy):
        f[j, : len(c)] = c
    g = np.array([[rnd.randrange(p) for _ in range(dxg + 1)] for _ in range(dyg + 1)], dtype=np.uint64)
    # prod_i g(x, a_i(x)) by plain polynomial arithmetic in x
    exp = [1]
    for r in roots:
        val = [0]
        lin = [r[0], r[1]]
        powy = [1]
        for j in range(dyg + 1):
            val = pyref.padd(p, val, pyref.pmul(p, [int(v) for v in g[j]], powy))
            powy = pyref.pmul(p, powy, lin)
        exp = pyref.pmul(p, exp, val)
    R = oracle.bivariate_resultant(p, f, g)
    D = dxf * dyg + dxg * dyf
    exp = (exp + [0] * (D + 1))[: D + 1]
    assert [int(v) for v in R] == exp
