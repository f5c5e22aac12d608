"""GPU parity of PM-Basis (Algorithm 3 on the device) against the oracle.

The oracle computes M-Basis (Algorithm 2) by definition; the CPU pins show it
equals PM-Basis for every threshold, so the device result must match it on
every coefficient, and the returned rdeg_s(P) must match too.  Tiny primes
make the residual matrices singular often, which exercises the device's
non-generic elimination path; random shifts exercise the (shift, index)
ordering of Algorithm 1.
"""
import random

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


def _run(ctx, p, F, d, s, T=None):
    from paper_1905_04356_gb300 import pmat
    if T is not None:
        ctx.set_option(pmat.PM_OPT_THRESHOLD, T)
    try:
        P, rd = pmat.pm_basis(ctx, p, pmat.to_device(F), d, s)
        ctx.sync()
    finally:
        ctx.set_option(pmat.PM_OPT_THRESHOLD, 32)
    return pmat.to_host(P), rd


CASES = [
    # p, m, n, d, T
    (P60, 2, 1, 6, 32),
    (P60, 4, 2, 16, 4),
    (P60, 5, 3, 33, 8),
    (P60, 6, 2, 20, 1),
    (P60, 8, 4, 100, 32),
    (P60, 32, 16, 64, 32),
    (P60, 32, 16, 200, 16),
    (P60, 4, 2, 1024, 32),   # nodes of order 1024 and 512: node products at half length
    (97, 3, 1, 512, 32),     # the same at order 512, small field
    (97, 4, 2, 16, 4),
    (7, 5, 2, 23, 3),
    (3, 3, 1, 12, 32),
    (synth.P998, 6, 3, 40, 8),
    (P60, 3, 3, 10, 4),      # m = n: no fast path
    (P60, 2, 4, 9, 32),      # m < n
    (2, 4, 2, 40, 8),        # p = 2: the leaves on bits
    (2, 6, 3, 100, 32),
    (2, 32, 16, 200, 16),
    (2, 3, 1, 1024, 32),     # p = 2 with node products at half length
    (2, 2, 4, 9, 32),
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_{c[1]}x{c[2]}_d{c[3]}_T{c[4]}" for c in CASES])
def test_pm_basis_matches_oracle(ctx, case):
    p, m, n, d, T = case
    g = synth.rng(sum(case) & 0xffff)
    F = synth.uniform(g, (m, n, d), p, np.uint64)
    rnd = random.Random(d)
    for s in ([0] * m, [rnd.randrange(-5, 6) for _ in range(m)]):
        P, rd = _run(ctx, p, F, d, s, T)
        Pexp, rdexp = oracle.mbasis(p, F, d, s)
        assert np.array_equal(P, Pexp), (case, s)
        assert np.array_equal(rd, rdexp), (case, s)


def test_pm_basis_short_input_is_zero_padded(ctx):
    """Only F mod x^d is read; a shorter F behaves as if padded with zeros."""
    p, m, n, d = P60, 4, 2, 24
    g = synth.rng(9)
    F = synth.uniform(g, (m, n, 10), p, np.uint64)
    P, rd = _run(ctx, p, F, d, [0] * m, 4)
    Fp = np.zeros((m, n, d), dtype=np.uint64)
    Fp[:, :, :10] = F
    Pexp, rdexp = oracle.mbasis(p, Fp, d, [0] * m)
    assert np.array_equal(P, Pexp) and np.array_equal(rd, rdexp)


def test_pm_basis_rejects_even_modulus(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    F = pmat.to_device(np.ones((2, 1, 4), dtype=np.uint64))
    with pytest.raises(PmError) as e:
        pmat.pm_basis(ctx, 1 << 20, F, 4, [0, 0])
    assert e.value.code == pmat.PM_EINVAL


@pytest.mark.parametrize("case", [(P60, 6, 2, 40, 8), (97, 5, 3, 30, 32), (P60, 32, 16, 96, 32), (2, 6, 2, 40, 8)])
def test_single_cta_leaf_matches_oracle(ctx, case):
    """The one-CTA leaf kernel (basis in global memory) gives the same bases."""
    from paper_1905_04356_gb300 import pmat
    p, m, n, d, T = case
    g = synth.rng(77 + d)
    F = synth.uniform(g, (m, n, d), p, np.uint64)
    s = [(i * 7) % 5 - 2 for i in range(m)]
    ctx.set_option(pmat.PM_OPT_LEAF_CLUSTER, 0)
    try:
        P, rd = _run(ctx, p, F, d, s, T)
    finally:
        ctx.set_option(pmat.PM_OPT_LEAF_CLUSTER, 1)
    Pexp, rdexp = oracle.mbasis(p, F, d, s)
    assert np.array_equal(P, Pexp) and np.array_equal(rd, rdexp)


def test_pm_basis_32x16_order_8192_matches_oracle_fingerprint(ctx):
    """F 32 x 16, order 8192, 60-bit prime, shift 0: the whole basis against the SHA-256 of
    the oracle's M-Basis output (and its row degrees)."""
    import hashlib
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "golden.json")))["pmbasis_32x16_d8192"]
    W = synth.pmbasis_c3(0)
    assert W["p"] == gold["p"]
    P, rd = _run(ctx, W["p"], W["F"], W["d"], W["shift"], 32)
    assert list(P.shape) == gold["shape"]
    assert [int(v) for v in rd] == gold["rdeg"]
    assert sum(gold["rdeg"]) == 16 * 8192
    flat = P.reshape(-1)
    for i, v in gold["samples"]:
        assert int(flat[i]) == v
    assert hashlib.sha256(np.ascontiguousarray(P).tobytes()).hexdigest() == gold["sha256"]
