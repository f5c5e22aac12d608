"""Seeded synthetic inputs shared by the CPU oracle, the GPU tests and bench.py.

This module holds no arithmetic of the method itself (no products, no bases,
no resultants): it only draws moduli and coefficient arrays from a seeded
NumPy PCG64 generator, with the shapes and value distributions of the
paper's random workloads (Sec. 1 "Experiments": random inputs modulo a random
60-bit prime; Sec. 3 tables: random matrices of given degree; Sec. 5.2:
random dense bivariate polynomials of given partial degrees).

Conventions
-----------
* A polynomial matrix with r x c entries of length ``len`` is a NumPy array of
  shape (r, c, len); coefficient t of entry (i, j) is ``X[i, j, t]``.  This is
  the entry-major, row-major layout the C-ABI expects.
* Coefficients are uniform in [0, p), stored as uint32 when p < 2**32 and as
  uint64 otherwise.
"""
from __future__ import annotations

import math

import numpy as np

P998 = 998244353  # the NTT-friendly 30-bit prime named by the product workloads

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (bases: the first 12 primes).

    Used only to draw moduli for synthetic inputs.
    """
    if n < 2:
        return False
    for b in _MR_BASES:
        if n % b == 0:
            return n == b
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def random_prime(g: np.random.Generator, bits: int = 60) -> int:
    """First uniform odd integer in [2^(bits-1), 2^bits) that passes Miller-Rabin."""
    lo = 1 << (bits - 1)
    while True:
        c = int(g.integers(lo, 1 << bits, dtype=np.uint64)) | 1
        if is_prime(c):
            return c


def dtype_for(p: int):
    return np.uint32 if p < (1 << 32) else np.uint64


def uniform(g: np.random.Generator, shape, p: int, dtype=None) -> np.ndarray:
    """Coefficients uniform in [0, p)."""
    dt = dtype or dtype_for(p)
    return g.integers(0, p, size=shape, dtype=np.uint64).astype(dt)


def pmat(g, r: int, c: int, length: int, p: int, dtype=None) -> np.ndarray:
    return uniform(g, (r, c, length), p, dtype)


# --------------------------------------------------------------------------
# The five workloads (sizes as in the product / PM-Basis / resultant tables)
# --------------------------------------------------------------------------

def product_c1(seed: int = 0):
    """4x4 . 4x4, entries of degree < 256, p = 998244353, uint32."""
    g = rng(seed)
    A = pmat(g, 4, 4, 256, P998)
    B = pmat(g, 4, 4, 256, P998)
    return dict(p=P998, A=A, B=B)


def product_c2(seed: int = 0, ntt_prime: bool = False, m: int = 32, d: int = 4096):
    """32x32 . 32x32, entries of degree < 4096.

    ``ntt_prime=False``: p is a random 60-bit prime drawn from the seed, uint64.
    ``ntt_prime=True``: the same shapes modulo 998244353, uint32.
    """
    g = rng(seed)
    p60 = random_prime(g, 60)
    p = P998 if ntt_prime else p60
    A = pmat(g, m, m, d, p)
    B = pmat(g, m, m, d, p)
    return dict(p=p, A=A, B=B)


def inverse_w(seed: int = 0, n: int = 32, d: int = 4096, t: int = 4096):
    """A (n x n, degree < d) modulo a random 60-bit prime and the truncation order t.

    A(0) is uniform, hence invertible except with probability < n / p.
    """
    g = rng(seed)
    p = random_prime(g, 60)
    A = pmat(g, n, n, d, p, np.uint64)
    return dict(p=p, A=A, t=t)


def solve_w(seed: int = 0, n: int = 32, d: int = 4096, digits: int = 8):
    """A (n x n) and b (n x 1) of degree < d modulo a random 60-bit prime; the series solution is
    wanted mod x^(digits d)."""
    g = rng(seed)
    p = random_prime(g, 60)
    A = pmat(g, n, n, d, p, np.uint64)
    b = pmat(g, n, 1, d, p, np.uint64)
    return dict(p=p, A=A, b=b, N=digits * d)


def linsolve_w(seed: int = 0, n: int = 16, d: int = 256):
    """A (n x n, length d) and b (n x 1, length d) modulo a random 60-bit prime."""
    g = rng(seed)
    p = random_prime(g, 60)
    A = pmat(g, n, n, d, p, np.uint64)
    b = pmat(g, n, 1, d, p, np.uint64)
    return dict(p=p, A=A, b=b)


def pmbasis_c3(seed: int = 0, m: int = 32, n: int = 16, d: int = 8192):
    """F (m x n, length d) modulo a random 60-bit prime, uniform shift 0."""
    g = rng(seed)
    p = random_prime(g, 60)
    F = pmat(g, m, n, d, p, np.uint64)
    return dict(p=p, F=F, d=d, shift=np.zeros(m, dtype=np.int64))


def intbasis_w(seed: int = 0, m: int = 32, n: int = 16, sigma: int = 8192):
    """E (m x n, sigma matrices) modulo a random 60-bit prime at the points c q^l with c, q
    drawn uniformly from [2, p - 1), uniform shift 0."""
    g = rng(seed)
    p = random_prime(g, 60)
    E = pmat(g, m, n, sigma, p, np.uint64)
    c = int(g.integers(2, p - 1))
    q = int(g.integers(2, p - 1))
    return dict(p=p, E=E, c=c, q=q, shift=np.zeros(m, dtype=np.int64))


def loguniform_int(g, lo: int, hi: int) -> int:
    """floor(exp(U[ln lo, ln (hi+1))))."""
    return int(math.floor(math.exp(g.uniform(math.log(lo), math.log(hi + 1)))))


def batch_c4(seed: int = 0, count: int = 512, dim=(2, 64), deg=(64, 16384)):
    """``count`` independent products with log-uniform m, n, k and degree bound.

    Even-indexed products are modulo 998244353 (uint32), odd-indexed ones modulo
    a fresh random 60-bit prime each (uint64).  Both operands of product i have
    length d_i.
    """
    g = rng(seed)
    out = []
    for i in range(count):
        m = loguniform_int(g, *dim)
        n = loguniform_int(g, *dim)
        k = loguniform_int(g, *dim)
        d = loguniform_int(g, *deg)
        p = P998 if i % 2 == 0 else random_prime(g, 60)
        out.append(dict(p=p, m=m, n=n, k=k, d=d))
    for item in out:
        item["A"] = pmat(g, item["m"], item["n"], item["d"], item["p"])
        item["B"] = pmat(g, item["n"], item["k"], item["d"], item["p"])
    return out


def resultant_c5(seed: int = 0, dx: int = 150, dy: int = 150, nprimes: int = 1):
    """Dense f, g in F_p[x, y] with deg_x = dx, deg_y = dy.

    ``f[j, i]`` is the coefficient of x^i y^j.  One set of integer coefficients
    uniform in [0, p_1) is drawn and reduced modulo each of p_1..p_nprimes
    (p_1 first; the others are the next random 60-bit primes from the seed).
    """
    g = rng(seed)
    primes = [random_prime(g, 60)]
    f = uniform(g, (dy + 1, dx + 1), primes[0], np.uint64)
    gg = uniform(g, (dy + 1, dx + 1), primes[0], np.uint64)
    while len(primes) < nprimes:
        q = random_prime(g, 60)
        if q not in primes:
            primes.append(q)
    fs = [f % np.uint64(q) for q in primes]
    gs = [gg % np.uint64(q) for q in primes]
    return dict(primes=primes, f=fs, g=gs, dx=dx, dy=dy)
