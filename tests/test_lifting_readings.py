"""CPU checks of two derivations the device code rests on (no GPU, no CUDA code involved).

1. The series solution by high-order lifting (Sec. 4): the residue jumps through the slices and
   the binary tree of residue positions, run here with the oracle's exact products and slices,
   must give the oracle's series solution A^-1 b mod x^N; and the positions (x + popcount x) D,
   x < 2^k, are at most 2D apart and cover N.
2. The explicit CRT sum's quotient: for the NTT prime table (recomputed here with its own
   primality test) the 64-bit fixed-point sum gives floor(sum t_i / q_i) exactly, at random
   values and at the coefficient bound, for shapes whose primes exceed the bound by as little
   as 0.013 bits.
"""
import math
import random

import numpy as np
import pytest

import oracle
import synth

P60 = 1152921504606846883


# ------------------------------------------------------------ high-order lifting
def _levels(D, N):
    k = 0
    while ((1 << k) + k + 1) * D + 1 < N:
        k += 1
    return k


def _hol_series(p, A, b, N):
    """A^-1 b mod x^N by residue jumps through the slices (the steps of the device routine,
    with the oracle's products)."""
    n, _, dA = A.shape
    D = dA - 1
    k = _levels(D, N)
    S = oracle.inv_slices(p, A, max(k, 1))
    W = {0: np.zeros((n, 1, D + 1), dtype=np.uint64)}
    W[0][:, :, :b.shape[2]] = b
    for i in range(k - 1, -1, -1):
        for x in range(0, 1 << k, 1 << (i + 1)):
            U = oracle.pmat_slice(p, S[i], W[x], D, D)             # coefficients D .. 2D-1 of S_i w
            R = oracle.pmat_slice(p, A, U, D, D)                    # coefficients D .. 2D-1 of A U
            w = np.zeros((n, 1, D + 1), dtype=np.uint64)
            w[:, :, :D] = (p - R) % p
            W[x + (1 << i)] = w
    v = np.zeros((n, 1, N), dtype=np.uint64)
    done = np.zeros(N, dtype=bool)
    for x, w in W.items():
        pos = (x + bin(x).count("1")) * D
        Y = oracle.pmat_slice(p, S[0], w, 0, 2 * D + 1)          # S_0 w mod x^(2D+1)
        for t in range(2 * D + 1):
            if pos + t < N:
                if done[pos + t]:
                    assert v[0, 0, pos + t] == Y[0, 0, t]          # overlapping windows agree
                v[:, :, pos + t] = Y[:, :, t]
                done[pos + t] = True
    assert done.all()
    return v


@pytest.mark.parametrize("p,n,dA,db,N", [(P60, 3, 5, 5, 120), (97, 2, 3, 2, 64), (synth.P998, 4, 9, 4, 300),
                                         (P60, 2, 2, 1, 40), (101, 3, 6, 6, 11)])
def test_high_order_lifting_steps_give_the_series_solution(p, n, dA, db, N):
    g = synth.rng(n * 1000 + dA * 10 + db)
    while True:
        A = synth.uniform(g, (n, n, dA), p, np.uint64)
        try:
            oracle.matinv(p, A[:, :, 0])
            break
        except Exception:
            continue
    b = synth.uniform(g, (n, 1, db), p, np.uint64)
    assert np.array_equal(_hol_series(p, A, b, N), oracle.solve_series(p, A, b, N))


@pytest.mark.parametrize("k", range(0, 9))
def test_residue_positions_are_at_most_2D_apart_and_cover(k):
    pos = sorted({x + bin(x).count("1") for x in range(1 << k)})   # in units of D
    assert pos[0] == 0
    assert all(b - a <= 2 for a, b in zip(pos, pos[1:]))
    assert pos[-1] == (1 << k) - 1 + k            # so windows of 2D + 1 reach (2^k + k + 1) D
    # jumps compose: the residue x + 2^i (bit i of x clear) sits K_i = 2^i + 1 units further
    for i in range(k):
        for x in range(0, 1 << k, 1 << (i + 1)):
            fx = x + bin(x).count("1")
            fy = (x + (1 << i)) + bin(x + (1 << i)).count("1")
            assert fy - fx == (1 << i) + 1


# ------------------------------------------------------------ explicit CRT quotient
def _is_prime(n):
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for s in small:
        if n % s == 0:
            return n == s
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _ntt_primes():
    """The six largest primes c 2^20 + 1 below 2^30."""
    out, c = [], (1 << 10)
    while len(out) < 6:
        c -= 1
        if _is_prime(c * (1 << 20) + 1):
            out.append(c * (1 << 20) + 1)
    return out


def _primes_for(p, n, dmin):
    need = math.log2(n) + math.log2(dmin) + 2 * math.log2(p - 1)
    have, pr = 0.0, []
    for q in _ntt_primes():
        pr.append(q)
        have += math.log2(q)
        if have > need + 0.01:
            return pr
    raise AssertionError("table too small")


@pytest.mark.parametrize("p,n,dmin", [(144115188075855859, 4, 14), (72057594037927931, 7, 32), (P60, 32, 4096),
                                      (4611686018427387847, 128, 1 << 19), (1000000007, 1, 1), (97, 2, 3)])
def test_fixed_point_crt_quotient_is_exact(p, n, dmin):
    pr = _primes_for(p, n, dmin)
    assert min(pr) > 1 << 29                       # floor(2^59 / q) fits 32 bits
    M = math.prod(pr)
    bound = n * dmin * (p - 1) ** 2
    rnd = random.Random(p % 1000 + n)
    for X in [0, 1, bound, bound - 1] + [rnd.randrange(bound + 1) for _ in range(300)]:
        t = [(X % q) * pow(M // q, -1, q) % q for q in pr]
        s = sum(ti * ((1 << 59) // q) for ti, q in zip(t, pr))
        assert s < 1 << 64
        k = (s + (1 << 33)) >> 59
        assert k == sum(ti * (M // q) for ti, q in zip(t, pr)) // M
        assert (sum(ti * (M // q) for ti, q in zip(t, pr)) - k * M) == X
