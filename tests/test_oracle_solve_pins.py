"""Pins of the oracle's lifting solver (Sec. 4, linear system solving: series solution, then
vector rational reconstruction by an approximant basis) -- CPU only.

What the definition fixes, checked with independent pure-Python arithmetic (tests/pyref.py):
A u = f b as a polynomial identity (Kronecker-substitution products), f monic, the degree bounds
of Cramer's rule; f = the monic determinant of A for generic inputs (determinant interpolated
from values by Lagrange's formula); a smaller denominator when the system decouples (block
diagonal A, right-hand side in one block); u = b, f = 1 for A = I; the scalar case against the
reduced fraction c / a computed by a Euclidean gcd in Python.
"""
import random

import numpy as np
import pytest

import oracle
from tests import pyref

P60 = 1152921504606846883


def _rand(rnd, p, shape):
    out = np.zeros(shape, dtype=np.uint64)
    flat = out.reshape(-1)
    for i in range(flat.size):
        flat[i] = rnd.randrange(p)
    return out


def _trim(a):
    a = [int(x) for x in a]
    while a and a[-1] == 0:
        a.pop()
    return a


def _det_poly(p, A):
    """det A(x) by evaluation at deg + 1 points and Lagrange interpolation."""
    n, _, dA = A.shape
    D = n * (dA - 1)
    xs = list(range(1, D + 2))
    ys = [pyref.det_mod(p, pyref.eval_pmat(p, A.tolist(), x)) for x in xs]
    return _trim(pyref.lagrange(p, xs, ys))


def _monic(p, a):
    a = _trim(a)
    inv = pow(a[-1], p - 2, p)
    return [x * inv % p for x in a]


def _check_identity(p, A, b, u, f):
    n = A.shape[0]
    Au = pyref.ks_pmat_mul(p, A.tolist(), u.tolist())
    for i in range(n):
        assert _trim(Au[i][0]) == _trim(pyref.pmul(p, [int(x) for x in f], [int(x) for x in b[i, 0]])), i


@pytest.mark.parametrize("p", [97, 998244353, P60])
@pytest.mark.parametrize("n,dA,db", [(1, 3, 2), (2, 3, 3), (3, 2, 4), (3, 4, 1), (4, 3, 3)])
def test_solution_identity_and_generic_denominator(p, n, dA, db):
    rnd = random.Random(p % 1000 + 10 * n + dA + 100 * db)
    while True:
        A = _rand(rnd, p, (n, n, dA))
        if pyref.det_mod(p, A[:, :, 0].tolist()):
            break
    b = _rand(rnd, p, (n, 1, db))
    u, f = oracle.solve(p, A, b)
    _check_identity(p, A, b, u, f)
    assert _trim(f)[-1] == 1                      # monic
    assert len(_trim(f)) - 1 <= n * (dA - 1)
    for i in range(n):
        assert len(_trim(u[i, 0])) - 1 <= (n - 1) * (dA - 1) + db - 1
    if p > 1000:                                   # generic: the denominator is det A
        assert _trim(f) == _monic(p, _det_poly(p, A))


@pytest.mark.parametrize("p", [101, P60])
def test_decoupled_system_has_the_block_denominator(p):
    """A = diag(A1, A2), b = [b1; 0]: the minimal denominator is det A1 (monic), of degree
    below deg det A, and the second block of u vanishes."""
    rnd = random.Random(p % 977)
    n1, n2, dA = 2, 2, 3
    while True:
        A1 = _rand(rnd, p, (n1, n1, dA))
        A2 = _rand(rnd, p, (n2, n2, dA))
        if pyref.det_mod(p, A1[:, :, 0].tolist()) and pyref.det_mod(p, A2[:, :, 0].tolist()):
            break
    A = np.zeros((n1 + n2, n1 + n2, dA), dtype=np.uint64)
    A[:n1, :n1] = A1
    A[n1:, n1:] = A2
    b = np.zeros((n1 + n2, 1, 2), dtype=np.uint64)
    b[:n1] = _rand(rnd, p, (n1, 1, 2))
    u, f = oracle.solve(p, A, b)
    _check_identity(p, A, b, u, f)
    assert _trim(f) == _monic(p, _det_poly(p, A1))
    assert len(_trim(f)) - 1 < len(_det_poly(p, A)) - 1
    assert not u[n1:].any()


def test_identity_matrix_gives_the_right_hand_side():
    p = P60
    rnd = random.Random(3)
    n = 3
    A = np.zeros((n, n, 1), dtype=np.uint64)
    for i in range(n):
        A[i, i, 0] = 1
    b = _rand(rnd, p, (n, 1, 5))
    u, f = oracle.solve(p, A, b)
    assert _trim(f) == [1]
    assert np.array_equal(u[:, :, :5], b)


def _pgcd(p, a, b):
    a, b = _trim(a), _trim(b)
    while b:
        inv = pow(b[-1], p - 2, p)
        while len(a) >= len(b):
            c = a[-1] * inv % p
            sh = len(a) - len(b)
            for i, x in enumerate(b):
                a[sh + i] = (a[sh + i] - c * x) % p
            a = _trim(a)
            if not a:
                break
        a, b = b, a
    return _monic(p, a)


def _pdiv_exact(p, a, g):
    a, g = _trim(a), _trim(g)
    q = [0] * (len(a) - len(g) + 1)
    inv = pow(g[-1], p - 2, p)
    while len(a) >= len(g):
        c = a[-1] * inv % p
        sh = len(a) - len(g)
        q[sh] = c
        for i, x in enumerate(g):
            a[sh + i] = (a[sh + i] - c * x) % p
        a = _trim(a)
    assert not a
    return q


@pytest.mark.parametrize("p", [97, P60])
def test_scalar_case_is_the_reduced_fraction(p):
    """n = 1: u / f = c / a in lowest terms with f monic; a common factor planted in a and c
    must cancel."""
    rnd = random.Random(p % 991)
    g = [rnd.randrange(1, p) for _ in range(3)]          # common factor, degree 2
    a1 = [rnd.randrange(1, p)] + [rnd.randrange(p) for _ in range(3)]
    c1 = [rnd.randrange(p) for _ in range(2)] + [rnd.randrange(1, p)]
    a = pyref.pmul(p, g, a1)
    c = pyref.pmul(p, g, c1)
    A = np.array([[a]], dtype=np.uint64)
    b = np.array([[c]], dtype=np.uint64)
    u, f = oracle.solve(p, A, b)
    gg = _pgcd(p, a, c)
    fa = _monic(p, _pdiv_exact(p, a, gg))
    assert _trim(f) == fa
    lc_inv = pow(_trim(_pdiv_exact(p, a, gg))[-1], p - 2, p)
    assert _trim(u[0, 0]) == _trim([x * lc_inv % p for x in _pdiv_exact(p, c, gg)])
