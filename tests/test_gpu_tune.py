"""The autotuner: pm_tune_product times the pointwise forms that apply to a shape and records
the fastest; pm_tune_basis picks PM-Basis's threshold.  Products and bases computed after tuning
(in the automatic mode, which takes the recorded choice) are checked against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P60 = 1152921504606846883


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


@pytest.mark.parametrize("p,w,m,n,k,dA,dB,forms", [
    (P60, 8, 32, 32, 32, 300, 200, {1, 6, 2}),          # CUDA-core tiles (4 x 8, 4 x 4) and the tensor-core form
    (synth.P998, 4, 5, 4, 7, 500, 400, {1, 6, 2, 3}),   # n <= 8: the streaming form too
    (P60, 8, 40, 20, 1, 64, 100, {1, 6, 2, 4}),         # k = 1: the matrix-vector form too (m > 32: no tensor)
    (97, 4, 64, 48, 40, 30, 20, {1, 6, 5}),             # beyond the tensor-core digit shapes
    (synth.P998, 4, 36, 57, 51, 300, 300, {1, 6}),      # ragged k: 4-column thread tiles waste less
])
def test_tuned_products_match_oracle(ctx, p, w, m, n, k, dA, dB, forms):
    from paper_1905_04356_gb300 import pmat
    form, bi, bk, ns, ncand = pmat.tune_product(ctx, p, w, m, n, k, dA, dB, reps=2)
    allowed = forms if m <= 32 else forms - {2}
    assert form in allowed and ns > 0 and ncand >= len(allowed)
    if form in (1, 6):
        assert bi >= 1 and bk >= 1 and bi * bk <= 32
    g = synth.rng(m * 1000 + n * 10 + k)
    dt = np.uint32 if w == 4 else np.uint64
    A = synth.uniform(g, (m, n, dA), p, dt)
    B = synth.uniform(g, (n, k, dB), p, dt)
    C = pmat.pmat_mul(ctx, p, pmat.to_device(A), pmat.to_device(B))   # automatic mode: the tuned form
    ctx.sync()
    assert np.array_equal(pmat.to_host(C).astype(np.uint64), oracle.pmat_mul(p, A, B))


def test_tuned_threshold_pm_basis_matches_oracle(ctx):
    from paper_1905_04356_gb300 import pmat
    g = synth.rng(77)
    p = synth.random_prime(g, 60)
    T, ns = pmat.tune_basis(ctx, p, 6, 3, 200, reps=1)
    assert T in (8, 16, 32, 64, 128) and ns > 0
    F = synth.uniform(g, (6, 3, 200), p, np.uint64)
    shift = [0, 3, 1, 0, 2, 5]
    P, rd = pmat.pm_basis(ctx, p, pmat.to_device(F), 200, shift)
    ctx.sync()
    Pexp, rdexp = oracle.mbasis(p, F, 200, shift)
    assert np.array_equal(pmat.to_host(P), Pexp) and list(rd) == list(rdexp)
    ctx.set_option(pmat.PM_OPT_THRESHOLD, 32)


def test_tuner_rejects_bad_arguments(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    with pytest.raises(PmError):
        pmat.tune_product(ctx, P60, 8, 0, 1, 1, 10, 10)
    with pytest.raises(PmError):
        pmat.tune_basis(ctx, 4, 2, 1, 10)
