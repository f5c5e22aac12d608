"""Independent pure-Python helpers used to PIN the oracle.

None of these restates the oracle's own formulas: products go through
Kronecker substitution (one big-integer multiplication), evaluation through
Horner's rule, determinants through Gaussian elimination, interpolation
through Lagrange's formula.  They are slow and meant for small inputs only.
"""
from __future__ import annotations

import random


# ---------------------------------------------------------------- products
def ks_polymul(a, b):
    """Exact integer product of two coefficient lists by Kronecker substitution."""
    if not a or not b:
        return []
    bound = max(a) * max(b) * min(len(a), len(b)) + 1
    bits = bound.bit_length() + 1
    A = 0
    for c in reversed(a):
        A = (A << bits) | int(c)
    Bv = 0
    for c in reversed(b):
        Bv = (Bv << bits) | int(c)
    P = A * Bv
    mask = (1 << bits) - 1
    out = []
    for _ in range(len(a) + len(b) - 1):
        out.append(P & mask)
        P >>= bits
    return out


def ks_pmat_mul(p, A, B):
    """A (m x n x dA), B (n x k x dB) as nested lists or arrays -> m x k lists mod p."""
    m, n, dA = len(A), len(A[0]), len(A[0][0])
    k, dB = len(B[0]), len(B[0][0])
    L = dA + dB - 1
    C = [[[0] * L for _ in range(k)] for _ in range(m)]
    for i in range(m):
        for kk in range(k):
            acc = [0] * L
            for l in range(n):
                prod = ks_polymul([int(x) for x in A[i][l]], [int(x) for x in B[l][kk]])
                for t, v in enumerate(prod):
                    acc[t] += v
            C[i][kk] = [v % p for v in acc]
    return C


def horner(p, coeffs, x):
    v = 0
    for c in reversed(list(coeffs)):
        v = (v * x + int(c)) % p
    return v


def eval_pmat(p, X, x):
    return [[horner(p, X[i][j], x) for j in range(len(X[0]))] for i in range(len(X))]


def matmul(p, A, B):
    n, k = len(B), len(B[0])
    return [[sum(A[i][l] * B[l][j] for l in range(n)) % p for j in range(k)] for i in range(len(A))]


# ---------------------------------------------------------------- linear algebra
def det_mod(p, M):
    M = [[int(x) % p for x in row] for row in M]
    n = len(M)
    det = 1
    for c in range(n):
        piv = next((r for r in range(c, n) if M[r][c]), None)
        if piv is None:
            return 0
        if piv != c:
            M[c], M[piv] = M[piv], M[c]
            det = -det
        det = det * M[c][c] % p
        inv = pow(M[c][c], p - 2, p)
        for r in range(c + 1, n):
            f = M[r][c] * inv % p
            if f:
                M[r] = [(x - f * y) % p for x, y in zip(M[r], M[c])]
    return det % p


def rank_mod(p, M):
    M = [[int(x) % p for x in row] for row in M]
    rows, cols = len(M), len(M[0]) if M else 0
    r = 0
    for c in range(cols):
        piv = next((i for i in range(r, rows) if M[i][c]), None)
        if piv is None:
            continue
        M[r], M[piv] = M[piv], M[r]
        inv = pow(M[r][c], p - 2, p)
        for i in range(rows):
            if i != r and M[i][c]:
                f = M[i][c] * inv % p
                M[i] = [(x - f * y) % p for x, y in zip(M[i], M[r])]
        r += 1
    return r


def sylvester(A, B):
    """Sylvester matrix of A (degree a) and B (degree b), coefficients low-first.

    Rows 0..b-1 hold shifted copies of A, rows b..b+a-1 shifted copies of B,
    highest degree first, so that det = Res(A, B) = lc(A)^b lc(B)^a prod(ai - bj).
    """
    a, b = len(A) - 1, len(B) - 1
    n = a + b
    S = [[0] * n for _ in range(n)]
    for r in range(b):
        for i, c in enumerate(reversed(A)):
            S[r][r + i] = c
    for r in range(a):
        for i, c in enumerate(reversed(B)):
            S[b + r][r + i] = c
    return S


def lagrange(p, xs, ys):
    """Coefficients (low first) of the interpolating polynomial, by Lagrange."""
    n = len(xs)
    out = [0] * n
    for i in range(n):
        num = [1]
        den = 1
        for j in range(n):
            if j == i:
                continue
            num = [(c1 - xs[j] * c0) % p for c0, c1 in zip(num + [0], [0] + num)]
            den = den * (xs[i] - xs[j]) % p
        f = ys[i] * pow(den, p - 2, p) % p
        for t in range(n):
            out[t] = (out[t] + f * num[t]) % p
    return out


# ---------------------------------------------------------------- polynomials
def pmul(p, a, b):
    return [v % p for v in ks_polymul([x % p for x in a], [x % p for x in b])]


def padd(p, a, b):
    n = max(len(a), len(b))
    return [((a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0)) % p for i in range(n)]


def rand_prime(bits, rnd: random.Random):
    import synth
    while True:
        c = rnd.randrange(1 << (bits - 1), 1 << bits) | 1
        if synth.is_prime(c):
            return c
