"""GPU parity of pmat_mul_vdm: products by Vandermonde-matrix evaluation and interpolation
(dense tensor-core products mod p) against the oracle, and equal to pmat_mul at sizes the oracle
only samples."""
import random

import numpy as np
import pytest

import oracle
import synth

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


CASES = [
    # p, m, n, k, dA, dB
    (synth.P998, 1, 1, 1, 1, 1),
    (synth.P998, 4, 4, 4, 256, 256),       # the 4x4 length-256 workload
    (synth.P998, 3, 5, 2, 17, 33),         # lengths not multiples of 16
    (synth.P998, 7, 9, 6, 300, 200),
    (synth.P998, 130, 3, 2, 40, 20),       # more than 128 entries: several row blocks
    (synth.P998, 2, 40, 3, 700, 900),
    (7340033, 5, 3, 4, 100, 60),           # 7 2^20 + 1
    (synth.P998, 33, 2, 35, 5, 70),        # output columns in several 32-column blocks
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_{c[1]}x{c[2]}x{c[3]}_{c[4]}_{c[5]}" for c in CASES])
def test_vdm_matches_oracle(ctx, case):
    from paper_1905_04356_gb300 import pmat
    p, m, n, k, dA, dB = case
    g = synth.rng(sum(case) & 0xffff)
    A = synth.uniform(g, (m, n, dA), p, np.uint32)
    B = synth.uniform(g, (n, k, dB), p, np.uint32)
    C = pmat.pmat_mul_vdm(ctx, p, pmat.to_device(A), pmat.to_device(B))
    ctx.sync()
    assert np.array_equal(pmat.to_host(C).astype(np.uint64), oracle.pmat_mul(p, A, B))


def test_vdm_extreme_inputs(ctx):
    """Every coefficient p - 1: digits at their largest, the drained sums at the exactness bound."""
    from paper_1905_04356_gb300 import pmat
    p = synth.P998
    A = np.full((6, 64, 130), p - 1, dtype=np.uint32)
    B = np.full((64, 5, 129), p - 1, dtype=np.uint32)
    C = pmat.pmat_mul_vdm(ctx, p, pmat.to_device(A), pmat.to_device(B))
    ctx.sync()
    assert np.array_equal(pmat.to_host(C).astype(np.uint64), oracle.pmat_mul(p, A, B))


@pytest.mark.parametrize("shape", [(64, 64, 64, 1024), (128, 16, 128, 512)])
def test_vdm_equals_pmat_mul_and_oracle_samples(ctx, shape):
    """Larger shapes: every coefficient equal to pmat_mul's (NTT path), sampled ones to the oracle."""
    from paper_1905_04356_gb300 import pmat
    m, n, k, d = shape
    p = synth.P998
    g = synth.rng(m + n + k + d)
    A = synth.uniform(g, (m, n, d), p, np.uint32)
    B = synth.uniform(g, (n, k, d), p, np.uint32)
    dA_, dB_ = pmat.to_device(A), pmat.to_device(B)
    C1 = pmat.to_host(pmat.pmat_mul_vdm(ctx, p, dA_, dB_))
    C2 = pmat.to_host(pmat.pmat_mul(ctx, p, dA_, dB_))
    ctx.sync()
    assert np.array_equal(C1, C2)
    rnd = random.Random(3)
    for _ in range(6):
        i, kk, t = rnd.randrange(m), rnd.randrange(k), rnd.randrange(2 * d - 1)
        assert int(C1[i, kk, t]) == oracle.pmat_coeff(p, A, B, i, kk, t)


def test_vdm_rejects_unsupported_moduli(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    A = pmat.to_device(np.ones((2, 2, 8), dtype=np.uint32))
    with pytest.raises(PmError) as e:
        pmat.pmat_mul_vdm(ctx, 1000000007, A, A)      # 2^4 does not divide p - 1 far enough
    assert e.value.code == pmat.PM_EUNSUPPORTED
