"""CPU oracle for polynomial-matrix arithmetic over F_p -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()``, the golden-value script under
``tests/golden/`` and the CPU-baseline leg of ``bench.py`` may import this
package.  The product library never does: it shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, unsigned __int128, OpenMP).
This module only marshals NumPy arrays into it.  Each wrapper names the part
of the paper its C function follows:

* ``pmat_mul`` / ``pmat_mul_trunc`` / ``pmat_middle_product`` / ``pmat_coeff``:
  Sec. 2, polynomial (matrix) multiplication and MiddleProduct(F, G, c, d).
* ``mbasis1``: Algorithm 1.  ``mbasis``: Algorithm 2.  ``pmbasis``: Algorithm 3.
  ``mintbasis``: Algorithm 4.  ``pmintbasis``: Algorithm 5.
* ``univ_resultant`` / ``bivariate_resultant``: Sec. 5.2, the direct
  evaluation / Euclid / interpolation method.
* ``matinv`` / ``inv_trunc``: Sec. 4 (linear system solving by lifting): the
  inverse of a constant matrix and the truncated inverse A^-1 mod x^t, by
  definition.  ``solve_series``: the series solution A^-1 b mod x^N (what
  Dixon's lifting computes), by definition.  ``inv_slices``: the high-order
  lifting slices of A^-1, read off the truncated inverse.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB_PATH, build

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(
            os.path.join(os.path.dirname(__file__), "oracle.c")
        ):
            build()
        L = C.CDLL(LIB_PATH)
        u64, i64, i32 = C.c_uint64, C.c_int64, C.c_int
        P = C.c_void_p
        L.orc_pmat_coeff.restype = u64
        L.orc_pmat_coeff.argtypes = [u64, i32, i32, i32, P, i64, P, i64, i32, i32, i64]
        L.orc_pmat_slice.restype = None
        L.orc_pmat_slice.argtypes = [u64, i32, i32, i32, P, i64, P, i64, i64, i64, P]
        L.orc_mbasis1.restype = i32
        L.orc_mbasis1.argtypes = [u64, i32, i32, P, P, P]
        L.orc_mbasis.restype = None
        L.orc_mbasis.argtypes = [u64, i32, i32, P, i64, i64, P, P, P]
        L.orc_pmbasis.restype = None
        L.orc_pmbasis.argtypes = [u64, i32, i32, P, i64, i64, P, i64, P, P]
        L.orc_rdeg.restype = None
        L.orc_rdeg.argtypes = [i32, i32, P, i64, P, P]
        L.orc_univ_resultant.restype = u64
        L.orc_univ_resultant.argtypes = [u64, P, i64, P, i64]
        L.orc_bivariate_resultant.restype = i32
        L.orc_bivariate_resultant.argtypes = [u64, i32, i32, P, i32, i32, P, P]
        L.orc_powmod.restype = u64
        L.orc_powmod.argtypes = [u64, u64, u64]
        L.orc_invmod.restype = u64
        L.orc_invmod.argtypes = [u64, u64]
        L.orc_matinv.restype = i32
        L.orc_matinv.argtypes = [u64, i32, P, P]
        L.orc_inv_trunc.restype = i32
        L.orc_inv_trunc.argtypes = [u64, i32, P, i64, i64, P]
        L.orc_inv_slices.restype = i32
        L.orc_inv_slices.argtypes = [u64, i32, P, i64, i32, P]
        L.orc_mintbasis.restype = None
        L.orc_mintbasis.argtypes = [u64, i32, i32, P, i64, P, P, P, P]
        L.orc_pmintbasis.restype = None
        L.orc_pmintbasis.argtypes = [u64, i32, i32, P, i64, P, P, i64, P, P]
        L.orc_bivariate_resultant_villard.restype = i32
        L.orc_bivariate_resultant_villard.argtypes = [u64, i32, i32, P, i32, i32, P, i32, P]
        L.orc_scale.restype = None
        L.orc_scale.argtypes = [u64, P, i64, u64]
        L.orc_pmat_eval.restype = None
        L.orc_pmat_eval.argtypes = [u64, i32, i32, P, i64, u64, P]
        L.orc_solve_series.restype = i32
        L.orc_solve_series.argtypes = [u64, i32, P, i64, P, i64, i64, P]
        _lib = L
    return _lib


def _u64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x).astype(np.uint64, copy=False))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def pmat_slice(p, A, B, c0, length, threads=None):
    """Coefficients c0 .. c0+length-1 of A.B (A: m x n x dA, B: n x k x dB)."""
    A, B = _u64(A), _u64(B)
    m, n, dA = A.shape
    n2, k, dB = B.shape
    assert n == n2
    Cout = np.zeros((m, k, length), dtype=np.uint64)
    _with_threads(threads, lambda: lib().orc_pmat_slice(
        p, m, n, k, _ptr(A), dA, _ptr(B), dB, c0, length, _ptr(Cout)))
    return Cout


def pmat_mul(p, A, B, threads=None):
    return pmat_slice(p, A, B, 0, A.shape[2] + B.shape[2] - 1, threads)


def pmat_mul_trunc(p, A, B, t, threads=None):
    return pmat_slice(p, A, B, 0, t, threads)


def pmat_middle_product(p, A, B, c, d, threads=None):
    return pmat_slice(p, A, B, c, d, threads)


def pmat_coeff(p, A, B, i, k, t):
    A, B = _u64(A), _u64(B)
    m, n, dA = A.shape
    _, kk, dB = B.shape
    return int(lib().orc_pmat_coeff(p, m, n, kk, _ptr(A), dA, _ptr(B), dB, i, k, t))


def mbasis1(p, R, t):
    """Algorithm 1: returns (Q as m x m x 2 array [const, x-coeff], rank)."""
    R = _u64(R)
    m, n = R.shape
    t = np.ascontiguousarray(np.asarray(t, dtype=np.int64))
    Q = np.zeros((m, m, 2), dtype=np.uint64)
    rank = lib().orc_mbasis1(p, m, n, _ptr(R), _ptr(t), _ptr(Q))
    return Q, rank


def mbasis(p, F, d, s, threads=None):
    """Algorithm 2: returns (P as m x m x (d+1), rdeg_s(P))."""
    F = _u64(F)
    m, n, lenF = F.shape
    s = np.ascontiguousarray(np.asarray(s, dtype=np.int64))
    P = np.zeros((m, m, d + 1), dtype=np.uint64)
    rd = np.zeros(m, dtype=np.int64)
    _with_threads(threads, lambda: lib().orc_mbasis(
        p, m, n, _ptr(F), lenF, d, _ptr(s), _ptr(P), _ptr(rd)))
    return P, rd


def pmbasis(p, F, d, s, T=32, threads=None):
    """Algorithm 3 with threshold T: returns (P as m x m x (d+1), rdeg_s(P))."""
    F = _u64(F)
    m, n, lenF = F.shape
    s = np.ascontiguousarray(np.asarray(s, dtype=np.int64))
    P = np.zeros((m, m, d + 1), dtype=np.uint64)
    rd = np.zeros(m, dtype=np.int64)
    _with_threads(threads, lambda: lib().orc_pmbasis(
        p, m, n, _ptr(F), lenF, d, _ptr(s), T, _ptr(P), _ptr(rd)))
    return P, rd


def mintbasis(p, E, alpha, s):
    """Algorithm 4: E is m x n x sigma (E[:, :, l] = E_l at point alpha[l]); returns (P, rdeg_s(P))."""
    E = _u64(E)
    m, n, sigma = E.shape
    al = _u64(alpha)
    s = np.ascontiguousarray(np.asarray(s, dtype=np.int64))
    P = np.zeros((m, m, sigma + 1), dtype=np.uint64)
    rd = np.zeros(m, dtype=np.int64)
    lib().orc_mintbasis(p, m, n, _ptr(E), sigma, _ptr(al), _ptr(s), _ptr(P), _ptr(rd))
    return P, rd


def pmintbasis(p, E, alpha, s, T=32):
    """Algorithm 5 with threshold T: returns (P, rdeg_s(P))."""
    E = _u64(E)
    m, n, sigma = E.shape
    al = _u64(alpha)
    s = np.ascontiguousarray(np.asarray(s, dtype=np.int64))
    P = np.zeros((m, m, sigma + 1), dtype=np.uint64)
    rd = np.zeros(m, dtype=np.int64)
    lib().orc_pmintbasis(p, m, n, _ptr(E), sigma, _ptr(al), _ptr(s), T, _ptr(P), _ptr(rd))
    return P, rd


def pmat_eval(p, X, a):
    """X(a) for an r x c x len polynomial matrix: an r x c uint64 array."""
    X = _u64(X)
    r, c, length = X.shape
    out = np.zeros((r, c), dtype=np.uint64)
    lib().orc_pmat_eval(p, r, c, _ptr(X), length, a, _ptr(out))
    return out


def rdeg(P, s):
    P = _u64(P)
    m, c, length = P.shape
    s = np.ascontiguousarray(np.asarray(s, dtype=np.int64))
    out = np.zeros(m, dtype=np.int64)
    lib().orc_rdeg(m, c, _ptr(P), length, _ptr(s), _ptr(out))
    return out


def univ_resultant(p, a, b):
    """Res(a, b) for coefficient lists (low degree first) with nonzero leading terms."""
    a, b = _u64(a), _u64(b)
    return int(lib().orc_univ_resultant(p, _ptr(a), len(a) - 1, _ptr(b), len(b) - 1))


def bivariate_resultant(p, f, g, threads=None):
    """Res_y(f, g) with f[j, i] = coeff of x^i y^j; returns D+1 coefficients."""
    f, g = _u64(f), _u64(g)
    dyf, dxf = f.shape[0] - 1, f.shape[1] - 1
    dyg, dxg = g.shape[0] - 1, g.shape[1] - 1
    D = dxf * dyg + dxg * dyf
    R = np.zeros(D + 1, dtype=np.uint64)
    rc = []
    _with_threads(threads, lambda: rc.append(lib().orc_bivariate_resultant(
        p, dxf, dyf, _ptr(f), dxg, dyg, _ptr(g), _ptr(R))))
    if rc[0] != 0:
        raise ValueError("too few evaluation points in F_p")
    return R


def villard_m(dyf, dyg, dxf, dxg):
    """Default block size of the Villard variant: ceil(n^0.4) for the partial degree
    n = max of the degrees (the choice reported in Sec. 5.2), at most min(dyf, dyg)."""
    import math
    n = max(dxf, dxg, dyf, dyg)
    m = 1
    while m ** 2.5 < n:      # smallest m with m >= n^0.4
        m += 1
    return max(1, min(m, dyf, dyg))


def bivariate_resultant_villard(p, f, g, m=0, threads=None):
    """Res_y(f, g) by the variant of Algorithm 6 (Sec. 5.2); same layout and output as
    bivariate_resultant.  m = 0 takes villard_m."""
    f, g = _u64(f), _u64(g)
    dyf, dxf = f.shape[0] - 1, f.shape[1] - 1
    dyg, dxg = g.shape[0] - 1, g.shape[1] - 1
    if m <= 0:
        m = villard_m(dyf, dyg, dxf, dxg)
    D = dxf * dyg + dxg * dyf
    R = np.zeros(D + 1, dtype=np.uint64)
    rc = []
    _with_threads(threads, lambda: rc.append(lib().orc_bivariate_resultant_villard(
        p, dxf, dyf, _ptr(f), dxg, dyg, _ptr(g), m, _ptr(R))))
    if rc[0] == 1:
        raise ValueError("too few evaluation points in F_p")
    if rc[0] == 2:
        raise ValueError("det Q vanishes at the normalisation point: input not generic")
    if rc[0] == 3:
        raise ValueError("det Q is not a constant multiple of Res: input not generic")
    return R


class SingularError(ValueError):
    """A constant matrix (or A(0)) is not invertible modulo p."""


def matinv(p, M):
    """Inverse of the n x n matrix M over F_p (p prime)."""
    M = _u64(M)
    n = M.shape[0]
    out = np.zeros((n, n), dtype=np.uint64)
    if lib().orc_matinv(p, n, _ptr(M), _ptr(out)):
        raise SingularError("singular matrix mod p")
    return out


def inv_trunc(p, A, t, threads=None):
    """A^-1 mod x^t (A: n x n x dA with A(0) invertible mod the prime p): n x n x t."""
    A = _u64(A)
    n, n2, dA = A.shape
    assert n == n2
    X = np.zeros((n, n, t), dtype=np.uint64)
    rc = []
    _with_threads(threads, lambda: rc.append(lib().orc_inv_trunc(p, n, _ptr(A), dA, t, _ptr(X))))
    if rc[0]:
        raise SingularError("A(0) is singular mod p")
    return X


def solve_series(p, A, b, N, threads=None):
    """A^-1 b mod x^N (A: n x n x dA with A(0) invertible mod the prime p, b: n x 1 x db): n x 1 x N."""
    A, b = _u64(A), _u64(b)
    n, n2, dA = A.shape
    assert n == n2 and b.shape[0] == n and b.shape[1] == 1
    v = np.zeros((n, 1, N), dtype=np.uint64)
    rc = []
    _with_threads(threads, lambda: rc.append(lib().orc_solve_series(p, n, _ptr(A), dA, _ptr(b), b.shape[2], N,
                                                                       _ptr(v))))
    if rc[0]:
        raise SingularError("A(0) is singular mod p")
    return v


def solve(p, A, b, threads=None):
    """Sec. 4, linear system solving by lifting: (u, f) with A u = f b, f monic of minimal degree
    (A: n x n x dA with A(0) invertible mod the prime p, b: n x 1 x db).

    The steps of the lifting solver: v = A^-1 b mod x^N (the series solution above, which is
    what the truncated inverse and Dixon's lifting compute), then vector rational reconstruction
    by an approximant basis of the (n+1) x n matrix [v^T; -I] at order N.  With
    D1 = n (dA - 1) >= deg f and D2 = (n - 1)(dA - 1) + db - 1 >= deg u (Cramer's rule) and
    N = D1 + D2 + 1, the basis is taken for the shift (-D1, -D2, ..., -D2): its one row of
    non-positive shifted degree is [f, u^T] up to a constant, since two solutions within the
    degree bounds agree modulo x^N on a polynomial identity of degree < N.  Returns
    (u as n x 1 x (D2+1), f as D1+1 coefficients), both normalised so that f is monic.
    """
    A, b = _u64(A), _u64(b)
    n, n2, dA = A.shape
    assert n == n2 and b.shape[0] == n and b.shape[1] == 1
    db = b.shape[2]
    D1 = n * (dA - 1)
    D2 = (n - 1) * (dA - 1) + db - 1
    N = D1 + D2 + 1
    v = solve_series(p, A, b, N, threads)
    F = np.zeros((n + 1, n, N), dtype=np.uint64)
    F[0] = v[:, 0, :]
    for i in range(n):
        F[1 + i, i, 0] = (p - 1) % p
    s = [-D1] + [-D2] * n
    P, rd = pmbasis(p, F, N, s, threads=threads)
    r = int(np.argmin(rd))
    if rd[r] > 0:
        raise SingularError("no solution within the degree bounds")
    f = np.ascontiguousarray(P[r, 0, :D1 + 1])
    u = np.ascontiguousarray(P[r, 1:, :D2 + 1]).reshape(n, 1, D2 + 1)
    nz = np.nonzero(f)[0]
    lc = int(f[nz[-1]])
    inv = powmod(lc, p - 2, p)
    lib().orc_scale(p, _ptr(f), f.size, inv)
    lib().orc_scale(p, _ptr(u), u.size, inv)
    return u, f


def inv_slices(p, A, K, threads=None):
    """High-order lifting slices: K x n x n x (2D+1) with slice i = coefficients
    (2^i - 1) D .. (2^i + 1) D of A^-1 (A: n x n x dA, D = dA - 1, A(0) invertible)."""
    A = _u64(A)
    n, n2, dA = A.shape
    assert n == n2 and dA >= 2
    S = np.zeros((K, n, n, 2 * (dA - 1) + 1), dtype=np.uint64)
    rc = []
    _with_threads(threads, lambda: rc.append(lib().orc_inv_slices(p, n, _ptr(A), dA, K, _ptr(S))))
    if rc[0]:
        raise SingularError("A(0) is singular mod p")
    return S


def powmod(a, e, p):
    return int(lib().orc_powmod(a, e, p))


def _with_threads(threads, fn):
    """Run fn with OMP_NUM_THREADS-equivalent control through libgomp."""
    if threads is None:
        return fn()
    try:
        gomp = C.CDLL("libgomp.so.1")
        old = gomp.omp_get_max_threads()
        gomp.omp_set_num_threads(int(threads))
        try:
            return fn()
        finally:
            gomp.omp_set_num_threads(old)
    except OSError:
        return fn()


def max_threads() -> int:
    lib()
    try:
        return int(C.CDLL("libgomp.so.1").omp_get_max_threads())
    except OSError:
        return 1
