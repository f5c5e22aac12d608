"""GPU parity of the one-launch product path (small products modulo an NTT prime used directly:
at most 2^10 transform points, inner dimension <= 16, all transforms in the shared memory of one
8-CTA cluster) against the oracle, at the edges of where it applies, and that it is one launch
per product."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P7 = 7340033          # 7 2^20 + 1


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
    # p, w, m, n, k, dA, dB, one launch
    (synth.P998, 4, 4, 4, 4, 256, 256, True),     # the 4 x 4 length-256 workload: 512 points
    (synth.P998, 4, 1, 1, 1, 1, 1, True),         # 16 points (the shortest transform)
    (synth.P998, 8, 3, 5, 2, 17, 33, True),       # 64-bit storage
    (P7, 4, 2, 16, 3, 100, 100, True),            # inner dimension 16: sums of 16 products (88 KB)
    (P7, 4, 2, 16, 3, 300, 200, True),            # 512 points over the cluster's 8 CTAs
    (synth.P998, 4, 16, 16, 16, 400, 300, False),  # 768 entries of 1024 points: too large, batched path
    (synth.P998, 4, 2, 17, 3, 30, 20, False),     # inner dimension 17: the batched path
    (synth.P998, 4, 1, 2, 1, 600, 425, True),     # output length 1024: 2^10 points
    (synth.P998, 4, 1, 2, 1, 600, 426, False),    # output length 1025: 2^11 points, batched path
    (P7, 8, 6, 7, 5, 100, 90, True),
    (1152921504606846883, 8, 2, 2, 2, 50, 50, False),   # 2^60 - 93: CRT primes, batched path
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_w{c[1]}_{c[2]}x{c[3]}x{c[4]}_{c[5]}_{c[6]}" for c in CASES])
def test_small_product_matches_oracle(ctx, case):
    from paper_1905_04356_gb300 import pmat
    p, w, m, n, k, dA, dB, one = case
    dt = np.uint32 if w == 4 else np.uint64
    g = synth.rng(dA * 7 + dB)
    A = synth.uniform(g, (m, n, dA), p, dt)
    B = synth.uniform(g, (n, k, dB), p, dt)
    dA_, dB_ = pmat.to_device(A), pmat.to_device(B)
    pmat.pmat_mul(ctx, p, dA_, dB_)            # first call: prime slot and twiddle tables
    ctx.sync()
    n0 = ctx.launches()
    C = pmat.pmat_mul(ctx, p, dA_, dB_)
    ctx.sync()
    launches = ctx.launches() - n0
    assert np.array_equal(pmat.to_host(C).astype(np.uint64), oracle.pmat_mul(p, A, B))
    if one:
        assert launches == 1
    else:
        assert launches > 1


def test_small_product_extreme_inputs(ctx):
    """Every coefficient p - 1 and inner dimension 16: the pointwise sums at their largest."""
    from paper_1905_04356_gb300 import pmat
    p = synth.P998
    A = np.full((3, 16, 200), p - 1, dtype=np.uint32)
    B = np.full((16, 2, 311), p - 1, dtype=np.uint32)
    C = pmat.pmat_mul(ctx, p, pmat.to_device(A), pmat.to_device(B))
    ctx.sync()
    assert np.array_equal(pmat.to_host(C).astype(np.uint64), oracle.pmat_mul(p, A, B))
