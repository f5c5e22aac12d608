"""GPU parity of pmat_mul_host (the product from and to host memory, copies overlapped with the
stages) against the CPU oracle.

The shapes exercise every chunking branch: small operands (one forward launch for both), A or B
of 8 MB or more (two row chunks each, transformed as they land), one output chunk (the default,
consecutive calls overlapping) and N output chunks set by option (more chunks than output
entries included); transforms longer than 2^14 points (column passes), the direct NTT-prime
mode with 32-bit words, pageable and pinned host buffers.
The full-size 32x32 products are checked against the SHA-256 of the oracle's output.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P60 = 1152921504606846883
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


def _host_tensor(a, pinned):
    import torch
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32))
    return t.pin_memory() if pinned else t


def _run(ctx, p, A, B, pinned=True):
    from paper_1905_04356_gb300 import pmat
    C = pmat.pmat_mul_host(ctx, p, _host_tensor(A, pinned), _host_tensor(B, pinned))
    ctx.sync()
    c = C.numpy()
    return c.view(np.uint64) if c.dtype == np.int64 else c.view(np.uint32)


CASES = [
    # p, w, m, n, k, dA, dB, pinned
    (P60, 8, 3, 5, 2, 17, 33, True),            # tiny: one chunk everywhere
    (synth.P998, 4, 7, 3, 9, 300, 1000, False),  # direct mode, 32-bit words, pageable buffers
    (P60, 8, 16, 1, 16, 2100, 2100, True),      # 8.6 MB of output
    (P60, 8, 2, 1, 64, 4096, 4096, True),       # m = 2
    (P60, 8, 64, 2, 2, 8200, 8, True),          # A of 8.4 MB: 2 row chunks
    (P60, 8, 8, 2, 16, 64, 32768, True),        # B of 8.4 MB: 2 row chunks, L = 2^16 (column passes)
    (P32, 4, 9, 2, 16, 700, 1500, True),        # 32-bit words through the CRT
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_w{c[1]}_{c[2]}x{c[3]}x{c[4]}_{c[5]}_{c[6]}" for c in CASES])
def test_host_product_matches_oracle(ctx, case):
    p, w, m, n, k, dA, dB, pinned = case
    dt = np.uint32 if w == 4 else np.uint64
    g = synth.rng((m * 131 + k * 7 + dB) & 0xffff)
    A = synth.uniform(g, (m, n, dA), p, dt)
    B = synth.uniform(g, (n, k, dB), p, dt)
    got = _run(ctx, p, A, B, pinned)
    want = oracle.pmat_mul(p, A.astype(np.uint64), B.astype(np.uint64))
    assert got.shape == want.shape
    assert np.array_equal(got.astype(np.uint64), want)


@pytest.mark.parametrize("name,ntt_prime", [("product_32x32_p60", False), ("product_32x32_p998", True)])
def test_host_product_full_size_matches_oracle_fingerprint(ctx, name, ntt_prime):
    """The bench product (32x32 . 32x32, length 4096) from host memory, against the SHA-256 of
    the oracle's output."""
    import hashlib
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "golden.json")))[name]
    W = synth.product_c2(0, ntt_prime=ntt_prime)
    assert W["p"] == gold["p"]
    got = _run(ctx, W["p"], W["A"], W["B"]).astype(np.uint64)
    assert list(got.shape) == gold["shape"]
    assert hashlib.sha256(np.ascontiguousarray(got).tobytes()).hexdigest() == gold["sha256"]


@pytest.mark.parametrize("case", [CASES[2], CASES[4], CASES[5]], ids=["out4", "A_rows", "B_rows_cols"])
def test_host_product_latency_form(ctx, case):
    """An explicit output chunk count (the latency form): 4 output chunks pipelined with their
    downloads, with A or B in two row chunks where they are 8 MB or more."""
    from paper_1905_04356_gb300 import pmat
    p, w, m, n, k, dA, dB, pinned = case
    g = synth.rng((m * 17 + dB) & 0xffff)
    A = synth.uniform(g, (m, n, dA), p, np.uint64)
    B = synth.uniform(g, (n, k, dB), p, np.uint64)
    ctx.set_option(pmat.PM_OPT_HOST_CHUNKS, 4)
    try:
        got = _run(ctx, p, A, B, pinned)
    finally:
        ctx.set_option(pmat.PM_OPT_HOST_CHUNKS, 0)
    assert np.array_equal(got, oracle.pmat_mul(p, A, B))


@pytest.mark.parametrize("chunks", [1, 3, 7, 40])
def test_host_product_chunk_counts(ctx, chunks):
    """Any output chunk count gives the same exact product (40 > the 36 output entries)."""
    from paper_1905_04356_gb300 import pmat
    g = synth.rng(700 + chunks)
    A = synth.uniform(g, (4, 3, 900), P60, np.uint64)
    B = synth.uniform(g, (3, 9, 1100), P60, np.uint64)
    ctx.set_option(pmat.PM_OPT_HOST_CHUNKS, chunks)
    try:
        got = _run(ctx, P60, A, B)
    finally:
        ctx.set_option(pmat.PM_OPT_HOST_CHUNKS, 0)
    assert np.array_equal(got, oracle.pmat_mul(P60, A, B))


def test_host_product_rejects_device_tensors(ctx):
    import torch
    from paper_1905_04356_gb300 import pmat
    A = torch.zeros((2, 2, 4), dtype=torch.int64, device="cuda")
    with pytest.raises(TypeError):
        pmat.pmat_mul_host(ctx, P60, A, A)


def test_host_product_then_device_work_is_ordered(ctx):
    """A device product issued right after a host product on the same context reuses the
    workspace; both results must be exact."""
    from paper_1905_04356_gb300 import pmat
    g = synth.rng(4242)
    A = synth.uniform(g, (16, 1, 2100), P60, np.uint64)
    B = synth.uniform(g, (1, 16, 2100), P60, np.uint64)
    A2 = synth.uniform(g, (4, 4, 300), P60, np.uint64)
    B2 = synth.uniform(g, (4, 4, 300), P60, np.uint64)
    C = pmat.pmat_mul_host(ctx, P60, _host_tensor(A, True), _host_tensor(B, True))
    C2 = pmat.pmat_mul(ctx, P60, pmat.to_device(A2), pmat.to_device(B2))
    ctx.sync()
    assert np.array_equal(C.numpy().view(np.uint64), oracle.pmat_mul(P60, A, B))
    assert np.array_equal(pmat.to_host(C2), oracle.pmat_mul(P60, A2, B2))


def test_host_products_back_to_back(ctx):
    """Consecutive host products overlap (alternating staging sets, downloads joined lazily):
    five calls with different inputs and outputs, one sync, every result exact; then a device
    product on the same context, which must wait for the pending downloads."""
    from paper_1905_04356_gb300 import pmat
    g = synth.rng(8080)
    shapes = [(16, 1, 16, 2100, 2100), (16, 1, 16, 2100, 2100), (8, 4, 8, 900, 3000), (16, 1, 16, 2100, 2100),
              (8, 4, 8, 900, 3000)]
    ins, outs = [], []
    for (m, n, k, dA, dB) in shapes:
        A = synth.uniform(g, (m, n, dA), P60, np.uint64)
        B = synth.uniform(g, (n, k, dB), P60, np.uint64)
        ins.append((A, B))
        outs.append(pmat.pmat_mul_host(ctx, P60, _host_tensor(A, True), _host_tensor(B, True)))
    A2 = synth.uniform(g, (4, 4, 300), P60, np.uint64)
    B2 = synth.uniform(g, (4, 4, 300), P60, np.uint64)
    C2 = pmat.pmat_mul(ctx, P60, pmat.to_device(A2), pmat.to_device(B2))
    ctx.sync()
    for (A, B), C in zip(ins, outs):
        assert np.array_equal(C.numpy().view(np.uint64), oracle.pmat_mul(P60, A, B))
    assert np.array_equal(pmat.to_host(C2), oracle.pmat_mul(P60, A2, B2))
