"""Pins of the oracle's truncated inverse (Sec. 4, linear system solving by lifting) -- CPU only.

The truncated inverse X = A^-1 mod x^t is the unique power series with A.X = I mod x^t (for
A(0) invertible).  It is checked against: the defining identity on both sides, with products
taken by Kronecker substitution (tests/pyref.py, not the oracle's product code); the scalar
geometric series 1 / (1 - a x); the finite inverse of I + x N for nilpotent N; block-diagonal
structure; the prefix property in t; determinants for the constant inverse; singular A(0).
"""
import random

import numpy as np
import pytest

import oracle
import synth
from tests import pyref

P60 = 1152921504606846883
P62 = 4611686018427387847
PRIMES = [2, 3, 97, synth.P998, P60, P62]


def _rand(rnd, p, r, c, length):
    return np.array([[[rnd.randrange(p) for _ in range(length)] for _ in range(c)] for _ in range(r)],
                    dtype=np.uint64)


def _rand_invertible_const(rnd, p, n):
    """A random invertible constant matrix: a product of unit lower and upper triangular ones."""
    Lm = [[(1 if i == j else (rnd.randrange(p) if i > j else 0)) for j in range(n)] for i in range(n)]
    Um = [[(1 if i == j else (rnd.randrange(p) if i < j else 0)) for j in range(n)] for i in range(n)]
    return [[sum(Lm[i][l] * Um[l][j] for l in range(n)) % p for j in range(n)] for i in range(n)]


def _identity_series(n, t):
    I = np.zeros((n, n, t), dtype=np.uint64)
    for i in range(n):
        I[i, i, 0] = 1
    return I


@pytest.mark.parametrize("p", PRIMES)
def test_matinv_against_determinant_and_product(p):
    rnd = random.Random(p & 0xffff)
    for n in (1, 2, 5):
        M = _rand_invertible_const(rnd, p, n)
        inv = oracle.matinv(p, np.array(M, dtype=np.uint64)).tolist()
        prod = [[sum(M[i][l] * inv[l][j] for l in range(n)) % p for j in range(n)] for i in range(n)]
        assert prod == [[1 if i == j else 0 for j in range(n)] for i in range(n)]
        assert pyref.det_mod(p, M) != 0
    S = [[1, 2, 3], [2, 4, 6], [0, 1, 1]]          # rank 2 over every field
    assert pyref.det_mod(p, [[v % p for v in r] for r in S]) == 0
    with pytest.raises(oracle.SingularError):
        oracle.matinv(p, np.array([[v % p for v in r] for r in S], dtype=np.uint64))


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("n,dA,t", [(1, 1, 1), (1, 4, 9), (2, 3, 7), (3, 5, 12), (4, 9, 6), (2, 40, 33)])
def test_inverse_defining_identity_both_sides(p, n, dA, t):
    rnd = random.Random(hash((p, n, dA, t)) & 0xffff)
    A = _rand(rnd, p, n, n, dA)
    A[:, :, 0] = np.array(_rand_invertible_const(rnd, p, n), dtype=np.uint64)
    X = oracle.inv_trunc(p, A, t)
    assert X.shape == (n, n, t)
    I = _identity_series(n, t)
    AX = np.array(pyref.ks_pmat_mul(p, A.tolist(), X.tolist()), dtype=np.uint64)[:, :, :t]
    XA = np.array(pyref.ks_pmat_mul(p, X.tolist(), A.tolist()), dtype=np.uint64)[:, :, :t]
    pad = lambda M: np.pad(M, ((0, 0), (0, 0), (0, t - M.shape[2]))) if M.shape[2] < t else M
    assert np.array_equal(pad(AX), I) and np.array_equal(pad(XA), I)


@pytest.mark.parametrize("p", [97, synth.P998, P60, P62])
def test_scalar_geometric_series(p):
    a = 123456789 % p
    A = np.array([[[1, (p - a) % p]]], dtype=np.uint64)       # 1 - a x
    X = oracle.inv_trunc(p, A, 40)
    assert [int(v) for v in X[0, 0]] == [pow(a, j, p) for j in range(40)]


@pytest.mark.parametrize("p", [5, 97, P60])
def test_nilpotent_perturbation_has_finite_inverse(p):
    """(I + x N)^-1 = sum_{j<n} (-x N)^j for N strictly upper triangular (N^n = 0)."""
    rnd = random.Random(7)
    n, t = 4, 9
    N = [[(rnd.randrange(p) if j > i else 0) for j in range(n)] for i in range(n)]
    A = np.zeros((n, n, 2), dtype=np.uint64)
    for i in range(n):
        A[i, i, 0] = 1
        for j in range(n):
            A[i, j, 1] = N[i][j]
    exp = np.zeros((n, n, t), dtype=np.uint64)
    Pw = [[1 if i == j else 0 for j in range(n)] for i in range(n)]
    for d in range(t):
        sgn = 1 if d % 2 == 0 else p - 1
        for i in range(n):
            for j in range(n):
                exp[i, j, d] = Pw[i][j] * sgn % p
        Pw = [[sum(Pw[i][l] * N[l][j] for l in range(n)) % p for j in range(n)] for i in range(n)]
    assert np.array_equal(oracle.inv_trunc(p, A, t), exp)
    assert not exp[:, :, n:].any()


def test_block_diagonal_and_prefix():
    p = synth.P998
    rnd = random.Random(3)
    A1, A2 = _rand(rnd, p, 2, 2, 6), _rand(rnd, p, 3, 3, 6)
    A1[:, :, 0] = np.array(_rand_invertible_const(rnd, p, 2), dtype=np.uint64)
    A2[:, :, 0] = np.array(_rand_invertible_const(rnd, p, 3), dtype=np.uint64)
    A = np.zeros((5, 5, 6), dtype=np.uint64)
    A[:2, :2], A[2:, 2:] = A1, A2
    X = oracle.inv_trunc(p, A, 20)
    assert np.array_equal(X[:2, :2], oracle.inv_trunc(p, A1, 20))
    assert np.array_equal(X[2:, 2:], oracle.inv_trunc(p, A2, 20))
    assert not X[:2, 2:].any() and not X[2:, :2].any()
    assert np.array_equal(oracle.inv_trunc(p, A, 7), X[:, :, :7])


def test_constant_matrix_and_singular_constant_term():
    p = 97
    rnd = random.Random(5)
    M = np.array(_rand_invertible_const(rnd, p, 3), dtype=np.uint64)
    X = oracle.inv_trunc(p, M[:, :, None], 5)
    assert np.array_equal(X[:, :, 0], oracle.matinv(p, M)) and not X[:, :, 1:].any()
    # A = diag(x, 1) is invertible over F_p(x) but A(0) is singular: no power-series inverse
    A = np.zeros((2, 2, 2), dtype=np.uint64)
    A[0, 0, 1] = 1
    A[1, 1, 0] = 1
    with pytest.raises(oracle.SingularError):
        oracle.inv_trunc(p, A, 4)


# ------------------------------------------------------------ series solution (Dixon's output)
@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("n,dA,db,N", [(1, 1, 1, 1), (1, 3, 2, 10), (2, 4, 4, 13), (3, 5, 2, 20), (4, 3, 6, 9)])
def test_series_solution_defining_identity(p, n, dA, db, N):
    """A.v = b mod x^N with Kronecker-substitution products."""
    rnd = random.Random(hash((p, n, dA, db, N)) & 0xffff)
    A = _rand(rnd, p, n, n, dA)
    A[:, :, 0] = np.array(_rand_invertible_const(rnd, p, n), dtype=np.uint64)
    b = _rand(rnd, p, n, 1, db)
    v = oracle.solve_series(p, A, b, N)
    assert v.shape == (n, 1, N)
    Av = np.array(pyref.ks_pmat_mul(p, A.tolist(), v.tolist()), dtype=object)
    got = [[[int(Av[i, 0, t]) if t < Av.shape[2] else 0 for t in range(N)]] for i in range(n)]
    exp = [[[int(b[i, 0, t]) if t < db else 0 for t in range(N)]] for i in range(n)]
    assert got == exp


@pytest.mark.parametrize("p", [97, synth.P998, P62])
def test_series_solution_scalar_closed_form(p):
    """(1 - a x) v = 1 + c x: v_0 = 1, v_j = a^(j-1) (a + c) for j >= 1."""
    a, c = 1234567 % p, 7654321 % p
    A = np.array([[[1, (p - a) % p]]], dtype=np.uint64)
    b = np.array([[[1, c]]], dtype=np.uint64)
    v = oracle.solve_series(p, A, b, 30)
    assert [int(x) for x in v[0, 0]] == [1] + [pow(a, j - 1, p) * (a + c) % p for j in range(1, 30)]


def test_series_solution_prefix_and_singular():
    p = synth.P998
    rnd = random.Random(9)
    A = _rand(rnd, p, 3, 3, 4)
    A[:, :, 0] = np.array(_rand_invertible_const(rnd, p, 3), dtype=np.uint64)
    b = _rand(rnd, p, 3, 1, 4)
    assert np.array_equal(oracle.solve_series(p, A, b, 8), oracle.solve_series(p, A, b, 20)[:, :, :8])
    S = np.zeros((2, 2, 2), dtype=np.uint64)
    S[0, 0, 1] = 1
    S[1, 1, 0] = 1
    with pytest.raises(oracle.SingularError):
        oracle.solve_series(p, S, np.ones((2, 1, 1), dtype=np.uint64), 4)


# ------------------------------------------------------------ high-order lifting slices
@pytest.mark.parametrize("p", [97, synth.P998, P62])
@pytest.mark.parametrize("D", [1, 3, 5])
def test_slices_sit_at_the_stated_degrees(p, D):
    """A = 1 - a x^D (length D + 1): A^-1 = sum_j a^j x^(jD), so slice i, coefficients
    (2^i - 1) D .. (2^i + 1) D, is a^(2^i - 1), 0 .. 0, a^(2^i), 0 .. 0, a^(2^i + 1) with D - 1
    zeros between."""
    a = 98765 % p
    A = np.zeros((1, 1, D + 1), dtype=np.uint64)
    A[0, 0, 0] = 1
    A[0, 0, D] = (p - a) % p
    K = 5
    S = oracle.inv_slices(p, A, K)
    for i in range(K):
        exp = [0] * (2 * D + 1)
        for j, e in ((0, (1 << i) - 1), (D, 1 << i), (2 * D, (1 << i) + 1)):
            exp[j] = pow(a, e, p)
        assert [int(v) for v in S[i, 0, 0]] == exp, i


def test_slices_match_the_truncated_inverse_and_the_recurrence():
    """Slice i is the truncated inverse's coefficients (2^i - 1) D .. (2^i + 1) D, and for i >= 1
    coefficients D .. 2D of A.S_i vanish (they are coefficients of A.A^-1 = I above degree D)."""
    p = synth.P998
    rnd = random.Random(13)
    n, dA, K = 3, 5, 4
    D = dA - 1
    A = _rand(rnd, p, n, n, dA)
    A[:, :, 0] = np.array(_rand_invertible_const(rnd, p, n), dtype=np.uint64)
    S = oracle.inv_slices(p, A, K)
    X = oracle.inv_trunc(p, A, ((1 << (K - 1)) + 1) * D + 1)
    for i in range(K):
        s0 = ((1 << i) - 1) * D
        assert np.array_equal(S[i], X[:, :, s0:s0 + 2 * D + 1])
        if i >= 1:
            AS = np.array(pyref.ks_pmat_mul(p, A.tolist(), S[i].tolist()), dtype=object)
            assert not any(int(AS[r, c, t]) for r in range(n) for c in range(n) for t in range(D, 2 * D + 1))
