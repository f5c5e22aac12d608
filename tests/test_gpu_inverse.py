"""GPU parity of the truncated inverse A^-1 mod x^t (Sec. 4, lifting: matrix Newton iteration).

Bit-exact against the oracle's coefficient recurrence at sizes it finishes quickly (moduli
2, 3, 97, 2^32 - 5, 998244353, 60- and 62-bit; t = 1, 2, odd and power-of-two lengths; A
shorter and longer than t; n up to 32, i.e. several pointwise tiles).  At the full size (32 x
32, dA = t = 4096, 60-bit p) the output is checked by the defining identity A.X = I mod x^t on
sampled coefficients the oracle computes one by one, and its prefix against the oracle's inverse
of A mod x^64 (X mod x^64 depends only on A mod x^64).
"""
import random

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P60 = 1152921504606846883
P62 = 4611686018427387847
P32 = 4294967291


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


def _matrix(seed, p, n, dA, w):
    """A random n x n x dA matrix mod p whose constant term is invertible (a product of unit
    lower and upper triangular matrices)."""
    g = synth.rng(seed)
    dt = np.uint32 if w == 4 else np.uint64
    A = synth.uniform(g, (n, n, dA), p, dt)
    rnd = random.Random(seed)
    Lm = [[(1 if i == j else (rnd.randrange(p) if i > j else 0)) for j in range(n)] for i in range(n)]
    Um = [[(1 if i == j else (rnd.randrange(p) if i < j else 0)) for j in range(n)] for i in range(n)]
    A0 = [[sum(Lm[i][l] * Um[l][j] for l in range(n)) % p for j in range(n)] for i in range(n)]
    A[:, :, 0] = np.array(A0, dtype=np.uint64).astype(dt)
    return A


def _gpu_inv(ctx, p, A, t):
    from paper_1905_04356_gb300 import pmat
    X = pmat.pmat_inv_trunc(ctx, p, pmat.to_device(A), t)
    ctx.sync()
    return pmat.to_host(X)


CASES = [
    # p, w, n, dA, t
    (synth.P998, 4, 4, 50, 300),
    (P60, 8, 3, 17, 100),
    (P62, 8, 2, 200, 129),
    (97, 4, 6, 7, 64),
    (2, 4, 5, 30, 70),
    (3, 4, 3, 3, 33),
    (P32, 4, 4, 10, 20),
    (P60, 8, 5, 9, 1),
    (P60, 8, 5, 9, 2),
    (synth.P998, 4, 3, 1, 40),        # constant matrix: X = A^-1, zero beyond
    (P60, 8, 1, 600, 513),
    (P60, 8, 32, 64, 200),            # 32 x 32: full pointwise block tiles
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_w{c[1]}_n{c[2]}_dA{c[3]}_t{c[4]}" for c in CASES])
def test_inverse_matches_oracle(ctx, case):
    p, w, n, dA, t = case
    A = _matrix(hash(case) & 0xffff, p, n, dA, w)
    got = _gpu_inv(ctx, p, A, t)
    exp = oracle.inv_trunc(p, A, t)
    assert got.shape == (n, n, t)
    assert np.array_equal(got.astype(np.uint64), exp)


def test_full_size_identity_sampled(ctx):
    """32 x 32, dA = t = 4096, 60-bit p: A.X = I mod x^t on sampled coefficients."""
    p, n, t = P60, 32, 4096
    A = _matrix(11, p, n, t, 8)
    X = _gpu_inv(ctx, p, A, t).astype(np.uint64)
    rnd = random.Random(2)
    picks = [(0, 0, 0), (3, 3, 0), (1, 2, 0), (5, 5, t - 1), (31, 0, t - 1)] + \
        [(rnd.randrange(n), rnd.randrange(n), rnd.randrange(t)) for _ in range(60)]
    for i, k, j in picks:
        assert oracle.pmat_coeff(p, A, X, i, k, j) == (1 if (i == k and j == 0) else 0), (i, k, j)
    assert np.array_equal(X[:, :, :64], oracle.inv_trunc(p, A[:, :, :64], 64))


def test_singular_constant_term_is_reported(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    p = 97
    A = np.zeros((2, 2, 3), dtype=np.uint32)
    A[0, 0, 1] = 1                                        # diag(x, 1): A(0) singular
    A[1, 1, 0] = 1
    pmat.pmat_inv_trunc(ctx, p, pmat.to_device(A), 8)
    with pytest.raises(PmError) as e:
        ctx.sync()
    assert e.value.code == pmat.PM_EDOMAIN
    # the context stays usable
    B = _matrix(5, p, 3, 4, 4)
    assert np.array_equal(_gpu_inv(ctx, p, B, 9).astype(np.uint64), oracle.inv_trunc(p, B, 9))


def test_argument_errors(ctx):
    import torch
    from paper_1905_04356_gb300 import PmError, pmat
    A = torch.zeros((3, 3, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(PmError) as e:
        pmat.pmat_inv_trunc(ctx, P60, A, 4)                 # w = 4 with p >= 2^32
    assert e.value.code == pmat.PM_EINVAL
    with pytest.raises(PmError) as e:
        pmat.pmat_inv_trunc(ctx, 97, A, 0)                  # t = 0
    assert e.value.code == pmat.PM_EINVAL
    big = torch.zeros((129, 129, 1), dtype=torch.int32, device="cuda")
    with pytest.raises(PmError) as e:
        pmat.pmat_inv_trunc(ctx, 97, big, 2)
    assert e.value.code == pmat.PM_EUNSUPPORTED


# ------------------------------------------------------------ series solution by Dixon's lifting
def _vector(seed, p, n, db, w):
    g = synth.rng(seed)
    return synth.uniform(g, (n, 1, db), p, np.uint32 if w == 4 else np.uint64)


def _gpu_solve(ctx, p, A, b, N):
    from paper_1905_04356_gb300 import pmat
    v = pmat.pmat_solve_series(ctx, p, pmat.to_device(A), pmat.to_device(b), N)
    ctx.sync()
    return pmat.to_host(v)


SOLVE_CASES = [
    # p, w, n, dA, db, N  (delta = max(dA, db) is the Dixon digit length)
    (synth.P998, 4, 4, 50, 30, 300),
    (P60, 8, 3, 17, 17, 100),
    (P62, 8, 2, 20, 40, 129),
    (97, 4, 5, 7, 3, 64),
    (2, 4, 5, 30, 10, 70),
    (3, 4, 3, 3, 3, 33),
    (P60, 8, 32, 64, 64, 256),       # 32 x 32: staged pointwise blocks with k = 1
    (P60, 8, 4, 40, 40, 25),         # N below one digit
    (synth.P998, 4, 3, 9, 9, 1),
]


@pytest.mark.parametrize("case", SOLVE_CASES, ids=[f"p{c[0]}_w{c[1]}_n{c[2]}_dA{c[3]}_db{c[4]}_N{c[5]}"
                                                   for c in SOLVE_CASES])
def test_series_solution_matches_oracle(ctx, case):
    p, w, n, dA, db, N = case
    A = _matrix(hash(case) & 0xffff, p, n, dA, w)
    b = _vector(hash(case) & 0xfff, p, n, db, w)
    got = _gpu_solve(ctx, p, A, b, N)
    assert got.shape == (n, 1, N)
    assert np.array_equal(got.astype(np.uint64), oracle.solve_series(p, A, b, N))


def test_series_solution_full_size_sampled(ctx):
    """32 x 32, dA = db = 4096, N = 8 digits: A.v = b mod x^N on sampled coefficients."""
    p, n, d, N = P60, 32, 4096, 8 * 4096
    A = _matrix(21, p, n, d, 8)
    b = _vector(22, p, n, d, 8)
    v = _gpu_solve(ctx, p, A, b, N).astype(np.uint64)
    rnd = random.Random(4)
    picks = [(0, 0), (7, 4095), (31, 4096), (3, N - 1)] + [(rnd.randrange(n), rnd.randrange(N)) for _ in range(40)]
    for i, t in picks:
        exp = int(b[i, 0, t]) if t < d else 0
        assert oracle.pmat_coeff(p, A, v, i, 0, t) == exp, (i, t)
    assert np.array_equal(v[:, :, :64], oracle.solve_series(p, A[:, :, :64], b[:, :, :64], 64))


def test_series_solution_singular_constant_term(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    A = np.zeros((2, 2, 3), dtype=np.uint32)
    A[0, 0, 1] = 1
    A[1, 1, 0] = 1
    pmat.pmat_solve_series(ctx, 97, pmat.to_device(A), pmat.to_device(np.ones((2, 1, 2), dtype=np.uint32)), 8)
    with pytest.raises(PmError) as e:
        ctx.sync()
    assert e.value.code == pmat.PM_EDOMAIN


# ------------------------------------------------------------ high-order lifting slices
SLICE_CASES = [
    # p, w, n, dA, K
    (synth.P998, 4, 3, 5, 5),
    (P60, 8, 2, 9, 4),
    (P62, 8, 4, 3, 6),
    (97, 4, 5, 7, 4),
    (2, 4, 3, 4, 4),
    (P60, 8, 32, 17, 4),             # 32 x 32 blocks
    (synth.P998, 4, 1, 2, 8),        # D = 1
    (P60, 8, 3, 6, 1),               # slice 0 only
]


@pytest.mark.parametrize("case", SLICE_CASES, ids=[f"p{c[0]}_w{c[1]}_n{c[2]}_dA{c[3]}_K{c[4]}" for c in SLICE_CASES])
def test_inverse_slices_match_oracle(ctx, case):
    from paper_1905_04356_gb300 import pmat
    p, w, n, dA, K = case
    A = _matrix(hash(case) & 0xffff, p, n, dA, w)
    S = pmat.pmat_inv_slices(ctx, p, pmat.to_device(A), K)
    ctx.sync()
    got = pmat.to_host(S).astype(np.uint64)
    assert got.shape == (K, n, n, 2 * dA - 1)
    assert np.array_equal(got, oracle.inv_slices(p, A, K))


def test_inverse_slices_full_size_properties(ctx):
    """32 x 32, dA = 4096 (D = 4095), 5 slices (the last one reaches degree 17 D): slice 0's
    prefix against the oracle, slice 1's lower half equal to slice 0's upper part (both are
    coefficients D .. 2D-1 of A^-1), and A.S_i zero in degrees D .. 2D on sampled entries."""
    from paper_1905_04356_gb300 import pmat
    p, n, dA, K = P60, 32, 4096, 5
    D = dA - 1
    A = _matrix(31, p, n, dA, 8)
    S = pmat.to_host(pmat.pmat_inv_slices(ctx, p, pmat.to_device(A), K)).astype(np.uint64)
    ctx.sync()
    assert np.array_equal(S[0][:, :, :64], oracle.inv_trunc(p, A[:, :, :64], 64))
    assert np.array_equal(S[1][:, :, :D], S[0][:, :, D:2 * D])
    rnd = random.Random(8)
    for i in (1, K - 1):
        for _ in range(12):
            r, c, t = rnd.randrange(n), rnd.randrange(n), rnd.randrange(D, 2 * D + 1)
            assert oracle.pmat_coeff(p, A, S[i], r, c, t) == 0, (i, r, c, t)


# ------------------------------------------------------------ series solution by high-order lifting
HOL_CASES = [
    # p, w, n, dA, db, N   (D = dA - 1; k levels, 2^k residues: the least k with (2^k + k + 1) D + 1 >= N)
    (P60, 8, 4, 9, 9, 200),          # k = 5
    (synth.P998, 4, 3, 17, 5, 1000),  # k = 6, db < dA
    (P60, 8, 5, 40, 40, 50),         # k = 0: N <= 2D + 1, one product by S_0
    (P60, 8, 5, 40, 12, 79),         # k = 0 at the bound 2D + 1
    (P60, 8, 5, 40, 12, 80),         # k = 1
    (97, 4, 1, 3, 1, 500),           # n = 1, D = 2, k = 8: 256 residues
    (2, 4, 3, 5, 5, 90),             # p = 2
    (P62, 8, 2, 2, 2, 37),           # D = 1
    (P60, 8, 32, 33, 33, 700),       # 32 x 32 blocks, k = 5
    (synth.P998, 4, 3, 9, 9, 1),     # N = 1
]


@pytest.mark.parametrize("case", HOL_CASES, ids=[f"p{c[0]}_w{c[1]}_n{c[2]}_dA{c[3]}_db{c[4]}_N{c[5]}"
                                                 for c in HOL_CASES])
def test_series_solution_by_high_order_lifting_matches_oracle(ctx, case):
    from paper_1905_04356_gb300 import pmat
    p, w, n, dA, db, N = case
    A = _matrix(hash(case) & 0xffff, p, n, dA, w)
    b = _vector(hash(case) & 0xfff, p, n, db, w)
    v = pmat.pmat_solve_series_hol(ctx, p, pmat.to_device(A), pmat.to_device(b), N)
    ctx.sync()
    got = pmat.to_host(v).astype(np.uint64)
    assert got.shape == (n, 1, N)
    assert np.array_equal(got, oracle.solve_series(p, A, b, N))


def test_series_solution_by_high_order_lifting_full_size(ctx):
    """32 x 32, dA = db = 4096, N = 8 digits (k = 3 levels, 8 residues): identical to Dixon's
    lifting on every coefficient, A.v = b mod x^N on sampled coefficients (oracle), and the
    prefix against the oracle."""
    from paper_1905_04356_gb300 import pmat
    p, n, d, N = P60, 32, 4096, 8 * 4096
    A = _matrix(21, p, n, d, 8)
    b = _vector(22, p, n, d, 8)
    Ad, bd = pmat.to_device(A), pmat.to_device(b)
    v = pmat.to_host(pmat.pmat_solve_series_hol(ctx, p, Ad, bd, N)).astype(np.uint64)
    v2 = pmat.to_host(pmat.pmat_solve_series(ctx, p, Ad, bd, N)).astype(np.uint64)
    ctx.sync()
    assert np.array_equal(v, v2)
    rnd = random.Random(5)
    picks = [(0, 0), (9, 4095), (31, 8190), (5, 20475), (3, N - 1)] + \
        [(rnd.randrange(n), rnd.randrange(N)) for _ in range(30)]
    for i, t in picks:
        exp = int(b[i, 0, t]) if t < d else 0
        assert oracle.pmat_coeff(p, A, v, i, 0, t) == exp, (i, t)
    assert np.array_equal(v[:, :, :64], oracle.solve_series(p, A[:, :, :64], b[:, :, :64], 64))


def test_series_solution_by_high_order_lifting_argument_errors(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    A = pmat.to_device(_matrix(3, 97, 2, 3, 4))
    for (Ab, bb, N) in ((pmat.to_device(_matrix(3, 97, 2, 1, 4)), pmat.to_device(_vector(1, 97, 2, 1, 4)), 8),  # dA < 2
                        (A, pmat.to_device(_vector(1, 97, 2, 4, 4)), 8),                                      # db > dA
                        (A, pmat.to_device(_vector(1, 97, 2, 3, 4)), 2000)):                                  # > 256 residues
        with pytest.raises(PmError) as e:
            pmat.pmat_solve_series_hol(ctx, 97, Ab, bb, N)
        assert e.value.code == pmat.PM_EINVAL


def test_series_solution_by_high_order_lifting_singular_constant_term(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    A = np.zeros((2, 2, 3), dtype=np.uint32)
    A[0, 0, 1] = 1
    A[1, 1, 0] = 1
    pmat.pmat_solve_series_hol(ctx, 97, pmat.to_device(A), pmat.to_device(np.ones((2, 1, 2), dtype=np.uint32)), 40)
    with pytest.raises(PmError) as e:
        ctx.sync()
    assert e.value.code == pmat.PM_EDOMAIN
