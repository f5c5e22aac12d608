"""GPU parity of the product path (C-ABI -> CUDA) against the CPU oracle.

Bit-exact: every residue of every tested output must match (the products
are exact; there is no tolerance).  Sizes span several transform tiles, the
column path (transforms longer than 2^14 points) and ragged lengths; the
full-size workloads are checked on sampled coefficients the oracle computes
one by one.
"""
import random

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P60 = 1152921504606846883          # 2^60 - 93
P62 = 4611686018427387847          # 2^62 - 57
P32 = 4294967291                   # 2^32 - 5: word-size, no 2-power roots of unity
COMPOSITE = 1000000000             # products are ring operations: any p >= 2


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


def _dt(p, w):
    return np.uint32 if w == 4 else np.uint64


def _rand(g, p, shape, w):
    return synth.uniform(g, shape, p, _dt(p, w))


def _gpu(ctx, fn, p, A, B, *args):
    from paper_1905_04356_gb300 import pmat
    dA, dB = pmat.to_device(A), pmat.to_device(B)
    out = getattr(pmat, fn)(ctx, p, dA, dB, *args)
    ctx.sync()
    return pmat.to_host(out)


CASES = [
    # p, w, m, n, k, dA, dB
    (synth.P998, 4, 1, 1, 1, 1, 1),
    (synth.P998, 4, 4, 4, 4, 256, 256),
    (synth.P998, 8, 3, 5, 2, 17, 33),
    (synth.P998, 4, 7, 3, 9, 300, 1000),
    (P60, 8, 1, 1, 1, 1, 1),
    (P60, 8, 3, 5, 2, 17, 33),
    (P60, 8, 5, 17, 6, 700, 513),
    (P62, 8, 2, 9, 3, 129, 64),
    (P32, 4, 4, 6, 5, 200, 77),
    (97, 4, 6, 6, 6, 40, 41),
    (2, 4, 3, 3, 3, 50, 20),
    (COMPOSITE, 4, 3, 4, 2, 90, 45),
    (P60, 8, 2, 3, 2, 4000, 4500),        # L = 2^13, one CTA per transform
    (synth.P998, 4, 2, 2, 3, 5000, 4000),  # L = 2^14: one CTA of 1024 threads
    (P60, 8, 2, 2, 1, 9000, 7000),         # L = 2^14, 5 primes
    (synth.P998, 4, 1, 2, 1, 9000, 8000),  # L = 2^15, inputs <= 2^14: odd half twisted, inverse in one CTA
    (P60, 8, 1, 1, 2, 9000, 8000),         # L = 2^15, 5 primes
    (P60, 8, 1, 1, 1, 20000, 100),         # L = 2^15, A longer than 2^14: A by the column pass, B twisted
    (synth.P998, 4, 1, 1, 2, 17000, 16000),  # L = 2^16: column passes both ways
    # pointwise block plans: a slice left empty in the last inner chunk (n = 32 + 5),
    # 2 x 2 block tiles with two chunks, uneven tiles, several column tiles, 4 slices
    (P60, 8, 4, 37, 8, 50, 40),
    (synth.P998, 4, 64, 64, 64, 40, 30),
    (P60, 8, 36, 57, 51, 70, 50),
    (P62, 8, 33, 2, 70, 25, 25),
    (97, 4, 2, 300, 2, 30, 20),
    # inner dimension 1 (outer products, streaming kernel): many rows, k = 1 and k = 5
    (P60, 8, 37, 1, 5, 300, 200),
    (synth.P998, 4, 300, 1, 1, 151, 4000),
    # matrix-vector products (k = 1, 8 < n <= 64, streaming kernel with a padded register block)
    (P60, 8, 32, 32, 1, 100, 90),
    (synth.P998, 4, 5, 17, 1, 60, 70),
    (97, 4, 3, 64, 1, 30, 20),
    (P62, 8, 7, 40, 1, 50, 50),
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_w{c[1]}_{c[2]}x{c[3]}x{c[4]}_{c[5]}_{c[6]}" for c in CASES])
def test_full_product_matches_oracle(ctx, case):
    p, w, m, n, k, dA, dB = case
    g = synth.rng(hash(case) & 0xffffffff)
    A = _rand(g, p, (m, n, dA), w)
    B = _rand(g, p, (n, k, dB), w)
    got = _gpu(ctx, "pmat_mul", p, A, B)
    exp = oracle.pmat_mul(p, A, B)
    assert got.shape == exp.shape
    assert np.array_equal(got.astype(np.uint64), exp)


@pytest.mark.parametrize("case", [(P60, 8, 3, 4, 5, 100, 60), (synth.P998, 4, 4, 2, 3, 333, 222),
                                  (P32, 4, 2, 3, 2, 3000, 3100),
                                  (P60, 8, 1, 1, 1, 9000, 8000)])   # 2^15 points: the one-CTA inverse's slice
def test_truncated_product_matches_oracle(ctx, case):
    p, w, m, n, k, dA, dB = case
    g = synth.rng(7)
    A = _rand(g, p, (m, n, dA), w)
    B = _rand(g, p, (n, k, dB), w)
    for t in (1, 17, min(dA, dB), dA + dB - 1, dA + dB + 40):
        got = _gpu(ctx, "pmat_mul_trunc", p, A, B, t)
        exp = oracle.pmat_mul_trunc(p, A, B, t)
        assert np.array_equal(got.astype(np.uint64), exp), t


@pytest.mark.parametrize("p,w", [(P60, 8), (synth.P998, 4)])
def test_middle_product_matches_oracle(ctx, p, w):
    g = synth.rng(11)
    m, n, k = 3, 4, 2
    # (c, d, dA, dB): the paper's c = d case, the PM-Basis residual shape
    # (dA = c + 1, dB = c + d), and shorter operands
    for c, d, dA, dB in ((64, 64, 64, 128), (33, 32, 34, 65), (500, 300, 501, 800), (10, 5, 3, 9),
                         (4096, 4096, 4097, 8192), (0, 7, 1, 7)):
        A = _rand(g, p, (m, n, dA), w)
        B = _rand(g, p, (n, k, dB), w)
        got = _gpu(ctx, "pmat_middle_product", p, A, B, c, d)
        exp = oracle.pmat_middle_product(p, A, B, c, d)
        assert np.array_equal(got.astype(np.uint64), exp), (c, d, dA, dB)


@pytest.mark.parametrize("p,w", [(P60, 8), (synth.P998, 4)])
def test_long_middle_product_matches_oracle(ctx, p, w):
    """Middle products at 2^15 transform points: A (c + 1 <= 2^14 coefficients) twisted, B longer
    than 2^14 by the column pass, the one-CTA inverse writing the coefficients from c on."""
    g = synth.rng(13)
    for c, d, dA, dB in ((12000, 12000, 12001, 24000), (9000, 7000, 9001, 16000)):
        A = _rand(g, p, (1, 1, dA), w)
        B = _rand(g, p, (1, 1, dB), w)
        got = _gpu(ctx, "pmat_middle_product", p, A, B, c, d)
        exp = oracle.pmat_middle_product(p, A, B, c, d)
        assert np.array_equal(got.astype(np.uint64), exp), (c, d, dA, dB)


def test_long_transform_sampled(ctx):
    """1 x 2 . 2 x 1 with lengths 40000 / 30000: L = 2^17 (column path, 3 top stages)."""
    p = P60
    g = synth.rng(3)
    A = _rand(g, p, (1, 2, 40000), 8)
    B = _rand(g, p, (2, 1, 30000), 8)
    got = _gpu(ctx, "pmat_mul", p, A, B)
    rnd = random.Random(1)
    for t in [0, 1, 29999, 39999, 69998] + [rnd.randrange(69999) for _ in range(40)]:
        assert int(got[0, 0, t]) == oracle.pmat_coeff(p, A, B, 0, 0, t), t


@pytest.mark.parametrize("ntt_prime", [False, True], ids=["p60", "p998"])
def test_c2_full_size_sampled(ctx, ntt_prime):
    """32x32 . 32x32, degree < 4096: sampled coefficients vs the oracle."""
    W = synth.product_c2(0, ntt_prime=ntt_prime)
    p, A, B = W["p"], W["A"], W["B"]
    got = _gpu(ctx, "pmat_mul", p, A, B)
    assert got.shape == (32, 32, 8191)
    rnd = random.Random(5)
    picks = [(0, 0, 0), (31, 31, 8190), (5, 7, 4095)] + \
        [(rnd.randrange(32), rnd.randrange(32), rnd.randrange(8191)) for _ in range(150)]
    for (i, kk, t) in picks:
        assert int(got[i, kk, t]) == oracle.pmat_coeff(p, A, B, i, kk, t), (i, kk, t)


def test_c1_full(ctx):
    W = synth.product_c1(0)
    got = _gpu(ctx, "pmat_mul", W["p"], W["A"], W["B"])
    exp = oracle.pmat_mul(W["p"], W["A"], W["B"])
    assert got.dtype == np.uint32 and np.array_equal(got.astype(np.uint64), exp)


def test_argument_errors(ctx):
    import torch
    from paper_1905_04356_gb300 import PmError, pmat
    A = torch.zeros((2, 3, 5), dtype=torch.int64, device="cuda")
    B = torch.zeros((3, 2, 5), dtype=torch.int64, device="cuda")
    with pytest.raises(PmError) as e:
        pmat.pmat_middle_product(ctx, P60, A, B, 2, 3)       # dA = 5 > c + 1
    assert e.value.code == pmat.PM_EINVAL
    with pytest.raises(PmError) as e:
        pmat.pmat_mul(ctx, 1, A, B)                           # p < 2
    assert e.value.code == pmat.PM_EINVAL
    A4 = torch.zeros((2, 3, 5), dtype=torch.int32, device="cuda")
    B4 = torch.zeros((3, 2, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(PmError) as e:
        pmat.pmat_mul(ctx, P60, A4, B4)                       # w = 4 with p >= 2^32
    assert e.value.code == pmat.PM_EINVAL


def test_debug_check_rejects_unreduced_input(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    A = np.full((2, 2, 4), 200, dtype=np.uint32)          # >= p = 97
    B = np.ones((2, 2, 4), dtype=np.uint32)
    ctx.set_option(pmat.PM_OPT_DEBUG_CHECKS, 1)
    try:
        with pytest.raises(PmError) as e:
            _gpu(ctx, "pmat_mul", 97, A, B)
        assert e.value.code == pmat.PM_EDOMAIN
    finally:
        ctx.set_option(pmat.PM_OPT_DEBUG_CHECKS, 0)


@pytest.mark.parametrize("name,ntt_prime", [("product_32x32_p60", False), ("product_32x32_p998", True)])
def test_c2_full_output_matches_oracle_fingerprint(ctx, name, ntt_prime):
    """The whole 32x32 . 32x32, length-4096 product against the SHA-256 of the oracle's output."""
    import hashlib
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "golden.json")))[name]
    W = synth.product_c2(0, ntt_prime=ntt_prime)
    assert W["p"] == gold["p"]
    got = _gpu(ctx, "pmat_mul", W["p"], W["A"], W["B"]).astype(np.uint64)
    assert list(got.shape) == gold["shape"]
    flat = got.reshape(-1)
    for i, v in gold["samples"]:
        assert int(flat[i]) == v
    assert hashlib.sha256(np.ascontiguousarray(got).tobytes()).hexdigest() == gold["sha256"]


@pytest.mark.parametrize("case", [(P60, 8, 32, 32, 32, 300, 200), (synth.P998, 4, 5, 7, 3, 100, 90),
                                  (P60, 8, 32, 32, 16, 64, 130), (97, 4, 17, 9, 31, 40, 33),
                                  (P62, 8, 32, 1, 32, 20, 20), (P60, 8, 3, 17, 5, 9, 8),
                                  (P60, 8, 32, 20, 32, 33, 40), (synth.P998, 4, 32, 16, 32, 5, 4),
                                  (2, 4, 6, 32, 7, 50, 61), (3, 4, 1, 1, 1, 3, 2), (P60, 8, 1, 32, 1, 7, 1000),
                                  (synth.P998, 4, 31, 31, 31, 1, 1)])
def test_tensor_core_and_cuda_core_pointwise_agree_with_oracle(ctx, case):
    """Both pointwise forms (balanced 8-bit digits in fp16 on tcgen05, 64-bit lazy sums on CUDA
    cores) give the oracle's product bit for bit: full and ragged inner dimensions (n = 17, 20
    leave zero digits up to the MMA's 16-step), one-row / one-column shapes, p = 2 and 3,
    transform lengths from 16 points."""
    from paper_1905_04356_gb300 import pmat
    p, w, m, n, k, dA, dB = case
    g = synth.rng(31 + m * n * k)
    A = _rand(g, p, (m, n, dA), w)
    B = _rand(g, p, (n, k, dB), w)
    exp = oracle.pmat_mul(p, A, B)
    try:
        for mode in (1, 2):
            ctx.set_option(pmat.PM_OPT_POINTWISE, mode)
            got = _gpu(ctx, "pmat_mul", p, A, B)
            assert np.array_equal(got.astype(np.uint64), exp), mode
    finally:
        ctx.set_option(pmat.PM_OPT_POINTWISE, 0)


def test_bounded_wait_gives_up_and_context_stays_usable(ctx):
    """The tensor-core kernel's wait for its MMA is bounded.  With the test hook, block 0 issues
    no MMA for its first point (nothing in flight), its wait gives up, the kernel frees its
    tensor memory and returns, and pm_sync reports PM_ETIMEOUT; the next products on the same
    context are exact."""
    from paper_1905_04356_gb300 import PmError, pmat
    p = P60
    g = synth.rng(31)
    A = synth.uniform(g, (4, 4, 64), p, np.uint64)
    B = synth.uniform(g, (4, 4, 64), p, np.uint64)
    dA, dB = pmat.to_device(A), pmat.to_device(B)
    ctx.set_option(pmat.PM_OPT_POINTWISE, 2)
    ctx.set_option(pmat.PM_OPT_TEST_WITHHOLD_MMA, 1)
    try:
        pmat.pmat_mul(ctx, p, dA, dB)
        with pytest.raises(PmError) as e:
            ctx.sync()
        assert e.value.code == pmat.PM_ETIMEOUT
    finally:
        ctx.set_option(pmat.PM_OPT_TEST_WITHHOLD_MMA, 0)
    try:
        for mode in (2, 1):
            ctx.set_option(pmat.PM_OPT_POINTWISE, mode)
            got = pmat.to_host(pmat.pmat_mul(ctx, p, dA, dB))
            ctx.sync()
            assert np.array_equal(got, oracle.pmat_mul(p, A, B)), mode
    finally:
        ctx.set_option(pmat.PM_OPT_POINTWISE, 0)


def test_work_counters_count_each_product(ctx):
    """pm_work_counters: compulsory bytes, pointwise MACs and butterflies of a product modulo
    998244353 (one prime, L the next power of two above the output length)."""
    from paper_1905_04356_gb300 import pmat
    p, m, n, k, dA, dB = synth.P998, 3, 5, 2, 17, 33
    g = synth.rng(77)
    A = synth.uniform(g, (m, n, dA), p, np.uint32)
    B = synth.uniform(g, (n, k, dB), p, np.uint32)
    ctx.work(reset=True)
    pmat.pmat_mul(ctx, p, pmat.to_device(A), pmat.to_device(B))
    ctx.sync()
    w = ctx.work(reset=True)
    lenC = dA + dB - 1
    lg = max(4, (lenC - 1).bit_length())
    L = 1 << lg
    assert w["bytes"] == (m * n * dA + n * k * dB + m * k * lenC) * 4
    assert w["macs"] == L * m * n * k
    assert w["butterflies"] == (m * n + n * k + m * k) * (L // 2) * lg


@pytest.mark.parametrize("p,n,d", [(144115188075855859, 4, 14), (72057594037927931, 7, 32), (P62, 8, 64),
                                   (P60, 32, 300)])
def test_extreme_coefficients_at_the_crt_bound(ctx, p, n, d):
    """Every input coefficient p - 1: the middle coefficients of the lifted product reach
    n d (p - 1)^2, the bound the prime count is chosen from.  The first two shapes leave 0.013
    bits between that bound and the product of the 4 primes, the hardest case for the CRT
    quotient (X / M = 0.991)."""
    A = np.full((3, n, d), p - 1, dtype=np.uint64)
    B = np.full((n, 2, d + 3), p - 1, dtype=np.uint64)
    got = _gpu(ctx, "pmat_mul", p, A, B)
    assert np.array_equal(got.astype(np.uint64), oracle.pmat_mul(p, A, B))


@pytest.mark.parametrize("name,ntt_prime", [("product_32x32_p60", False), ("product_32x32_p998", True)])
def test_tensor_core_c2_full_output_matches_oracle_fingerprint(ctx, name, ntt_prime):
    """The whole 32x32 . 32x32, length-4096 product with the tensor-core pointwise form, against
    the SHA-256 of the oracle's output (the launch configuration the bench times)."""
    import hashlib
    import json
    import os
    from paper_1905_04356_gb300 import pmat
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "golden.json")))[name]
    W = synth.product_c2(0, ntt_prime=ntt_prime)
    ctx.set_option(pmat.PM_OPT_POINTWISE, 2)
    try:
        got = _gpu(ctx, "pmat_mul", W["p"], W["A"], W["B"]).astype(np.uint64)
    finally:
        ctx.set_option(pmat.PM_OPT_POINTWISE, 0)
    assert hashlib.sha256(np.ascontiguousarray(got).tobytes()).hexdigest() == gold["sha256"]


@pytest.mark.parametrize("p,w", [(P60, 8), (synth.P998, 4), (P62, 8)])
def test_tensor_core_extreme_inputs(ctx, p, w):
    """All inputs p - 1 (and all zero in one operand block) through the tensor-core form."""
    from paper_1905_04356_gb300 import pmat
    dt = np.uint32 if w == 4 else np.uint64
    A = np.full((32, 32, 257), p - 1, dtype=dt)
    B = np.full((32, 32, 255), p - 1, dtype=dt)
    B[:, :16, :] = 0
    exp = oracle.pmat_mul(p, A, B)
    ctx.set_option(pmat.PM_OPT_POINTWISE, 2)
    try:
        got = _gpu(ctx, "pmat_mul", p, A, B)
    finally:
        ctx.set_option(pmat.PM_OPT_POINTWISE, 0)
    assert np.array_equal(got.astype(np.uint64), exp)


@pytest.mark.parametrize("case", [(P60, 8, 64, 64, 64, 100, 80), (synth.P998, 4, 128, 40, 100, 50, 60),
                                  (97, 4, 70, 17, 33, 20, 30), (P60, 8, 128, 128, 128, 30, 40),
                                  (P62, 8, 65, 1, 200, 9, 7), (2, 4, 64, 300, 3, 5, 6)])
def test_tensor_core_dense_pointwise_matches_oracle(ctx, case):
    """The tensor-core dense form (PM_OPT_POINTWISE = 3: every point's m x n . n x k product as a
    dense product of fp16 digits, drained every 256 inner entries) against the oracle: m = 64 and
    above, ragged n and k, inner dimensions from 1 to 300, moduli 2 to 62 bits."""
    from paper_1905_04356_gb300 import pmat
    p, w, m, n, k, dA, dB = case
    g = synth.rng(41 + m * n * k)
    A = _rand(g, p, (m, n, dA), w)
    B = _rand(g, p, (n, k, dB), w)
    ctx.set_option(pmat.PM_OPT_POINTWISE, 3)
    try:
        got = _gpu(ctx, "pmat_mul", p, A, B)
    finally:
        ctx.set_option(pmat.PM_OPT_POINTWISE, 0)
    assert np.array_equal(got.astype(np.uint64), oracle.pmat_mul(p, A, B))



@pytest.mark.parametrize("case", [(synth.P998, 4, 36, 57, 51, 60, 70), (P60, 8, 33, 40, 13, 30, 20),
                                  (synth.P998, 4, 5, 3, 7, 100, 90), (97, 4, 1, 1, 1, 3, 2),
                                  (P62, 8, 9, 70, 6, 20, 17), (synth.P998, 4, 64, 16, 64, 5, 4),
                                  (2, 4, 3, 33, 130, 9, 10)])
def test_cuda_core_4x4_thread_tiles_match_oracle(ctx, case):
    """The staged CUDA-core form with 4 x 4 thread tiles (PM_OPT_POINTWISE = 4) against the
    oracle: k not a multiple of 4 (the last thread tile's columns past k read unused staging
    words and are never stored), odd m, inner dimensions over several 32-entry chunks (40, 57,
    70), chunks split into slices when the block tile leaves slots free (9 x 70 . 70 x 6: 4
    slices, 3 x 33 . 33 x 130: 2), full 32-slot blocks (64 x 16 . 16 x 64), n <= 8 (the
    streaming form's shapes taken by the staged kernel), one-entry products, wide k (130
    columns: several column blocks), moduli 2 to 62 bits through the CRT."""
    from paper_1905_04356_gb300 import pmat
    p, w, m, n, k, dA, dB = case
    g = synth.rng(53 + m * n * k)
    A = _rand(g, p, (m, n, dA), w)
    B = _rand(g, p, (n, k, dB), w)
    ctx.set_option(pmat.PM_OPT_POINTWISE, 4)
    try:
        got = _gpu(ctx, "pmat_mul", p, A, B)
    finally:
        ctx.set_option(pmat.PM_OPT_POINTWISE, 0)
    assert np.array_equal(got.astype(np.uint64), oracle.pmat_mul(p, A, B))


def test_cuda_core_4x4_extreme_inputs(ctx):
    """Every coefficient p - 1 through the 4 x 4 thread tiles: the lazy 64-bit sums at their
    largest over 16-product groups and several chunks."""
    from paper_1905_04356_gb300 import pmat
    p = synth.P998
    A = np.full((7, 45, 40), p - 1, dtype=np.uint32)
    B = np.full((45, 11, 33), p - 1, dtype=np.uint32)
    ctx.set_option(pmat.PM_OPT_POINTWISE, 4)
    try:
        got = _gpu(ctx, "pmat_mul", p, A, B)
    finally:
        ctx.set_option(pmat.PM_OPT_POINTWISE, 0)
    assert np.array_equal(got.astype(np.uint64), oracle.pmat_mul(p, A, B))
