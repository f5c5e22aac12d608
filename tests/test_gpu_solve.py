"""GPU parity of the lifting solver pmat_solve (Sec. 4: series solution by Dixon's lifting, then
vector rational reconstruction by PM-Basis) against the oracle's solver.

The pair (u, f) with A u = f b and f monic of minimal degree is unique, so the device output must
match the oracle bit for bit, degrees included.  Cases: several primes (97 makes the
reconstruction's residuals singular often), n = 1, constant A, a decoupled system whose
denominator is smaller than det A, singular A(0), and the bench workload (16 x 16, length 256)
checked by A u = f b on coefficients the oracle computes one by one.
"""
import random

import numpy as np
import pytest

import oracle
import synth
from tests.test_gpu_inverse import P60, P62, _matrix, _vector

pytestmark = pytest.mark.gpu


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


def _gpu(ctx, p, A, b):
    from paper_1905_04356_gb300 import pmat
    u, f, df, du = pmat.pmat_solve(ctx, p, pmat.to_device(A), pmat.to_device(b))
    return pmat.to_host(u), pmat.to_host(f), df, du


def _deg(a):
    nz = np.nonzero(a)[0]
    return int(nz[-1]) if len(nz) else -1


CASES = [
    # p, n, dA, db
    (P60, 1, 5, 3),
    (P60, 3, 4, 4),
    (P60, 4, 64, 64),
    (P62, 2, 9, 17),
    (synth.P998, 5, 6, 2),
    (97, 4, 5, 5),
    (101, 6, 3, 4),
    (P60, 3, 1, 7),          # constant A: f = 1
    (P60, 8, 16, 1),
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_n{c[1]}_dA{c[2]}_db{c[3]}" for c in CASES])
def test_solve_matches_oracle(ctx, case):
    p, n, dA, db = case
    A = _matrix(hash(case) & 0xffff, p, n, dA, 8)
    b = _vector(hash(case) & 0xfff, p, n, db, 8)
    u, f, df, du = _gpu(ctx, p, A, b)
    ue, fe = oracle.solve(p, A, b)
    assert np.array_equal(f, fe)
    assert np.array_equal(u, ue)
    assert df == _deg(fe) and du == max(_deg(ue[i, 0]) for i in range(n))


def test_solve_decoupled_system(ctx):
    """Block-diagonal A with b in the first block: the denominator is that block's determinant."""
    p = P60
    A1 = _matrix(5, p, 3, 6, 8)
    A2 = _matrix(6, p, 2, 6, 8)
    A = np.zeros((5, 5, 6), dtype=np.uint64)
    A[:3, :3] = A1
    A[3:, 3:] = A2
    b = np.zeros((5, 1, 4), dtype=np.uint64)
    b[:3] = _vector(7, p, 3, 4, 8)
    u, f, df, du = _gpu(ctx, p, A, b)
    ue, fe = oracle.solve(p, A, b)
    assert np.array_equal(f, fe) and np.array_equal(u, ue)
    assert df == 3 * 5 and not u[3:].any()


def test_solve_singular_constant_term(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    p = P60
    A = _matrix(8, p, 3, 4, 8)
    A[1, :, 0] = A[0, :, 0]
    b = _vector(9, p, 3, 4, 8)
    with pytest.raises(PmError) as e:
        pmat.pmat_solve(ctx, p, pmat.to_device(A), pmat.to_device(b))
    assert e.value.code == pmat.PM_EDOMAIN


def test_solve_bench_workload_identity(ctx):
    """16 x 16, length 256 (the bench workload): f monic of degree n (dA - 1) (generic), and
    A u = f b on sampled coefficients."""
    W = synth.linsolve_w(0)
    p, A, b = W["p"], W["A"], W["b"]
    n, _, dA = A.shape
    u, f, df, du = _gpu(ctx, p, A, b)
    assert df == n * (dA - 1) and int(f[df]) == 1
    D = len(f) - 1 + u.shape[2] - 1
    rnd = random.Random(2)
    F = f.reshape(1, 1, -1)
    for _ in range(24):
        i, t = rnd.randrange(n), rnd.randrange(D + 1)
        lhs = oracle.pmat_coeff(p, A, u, i, 0, t)
        rhs = oracle.pmat_coeff(p, F, np.ascontiguousarray(b[i:i + 1]), 0, 0, t)
        assert lhs == rhs, (i, t)


@pytest.mark.parametrize("case", [(3, 2, 3, 2), (P60, 1, 1, 1), (5, 3, 2, 3)], ids=["F3", "constant_1x1", "F5"])
def test_solve_small_fields_and_trivial(ctx, case):
    """Tiny fields (many singular residuals in the reconstruction) and the constant 1 x 1 system."""
    p, n, dA, db = case
    for seed in range(4):
        A = _matrix(1000 + seed, p, n, dA, 8)
        b = _vector(2000 + seed, p, n, db, 8)
        u, f, df, du = _gpu(ctx, p, A, b)
        ue, fe = oracle.solve(p, A, b)
        assert np.array_equal(f, fe) and np.array_equal(u, ue), seed
