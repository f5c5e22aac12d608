"""GPU parity of pmat_mul_batched (uneven products binned by transform length)."""
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


def test_mixed_batch_full_oracle(ctx):
    """40 products: primes 998244353 / 60-bit / small / word-size, lengths 1 .. 9000."""
    from paper_1905_04356_gb300 import pmat
    rnd = random.Random(4)
    g = synth.rng(4)
    primes = [(synth.P998, 4), (P60, 8), (97, 4), (4294967291, 4), (synth.random_prime(g, 60), 8)]
    items, host = [], []
    for i in range(40):
        p, w = primes[i % len(primes)]
        m, n, k = rnd.randint(1, 7), rnd.randint(1, 7), rnd.randint(1, 7)
        dA = rnd.choice([1, 3, 50, 200, 700, 3000, 5000]) if i % 9 else 9000
        dB = rnd.choice([1, 2, 60, 400, 2500]) if i % 9 else 6000
        dt = np.uint32 if w == 4 else np.uint64
        A = synth.uniform(g, (m, n, dA), p, dt)
        B = synth.uniform(g, (n, k, dB), p, dt)
        host.append((p, A, B))
        items.append((p, pmat.to_device(A), pmat.to_device(B)))
    outs = pmat.pmat_mul_batched(ctx, items)
    ctx.sync()
    for (p, A, B), C in zip(host, outs):
        assert np.array_equal(pmat.to_host(C).astype(np.uint64), oracle.pmat_mul(p, A, B))


def test_batched_512_sampled():
    """The 512-product workload (log-uniform m, n, k in [2, 64], lengths in [64, 16384],
    half mod 998244353, half mod 60-bit primes): 4 sampled coefficients per product."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_04356_gb300 import Context, pmat
    ctx = Context(0)
    items = synth.batch_c4(0)
    dev = [(it["p"], pmat.to_device(it["A"]), pmat.to_device(it["B"])) for it in items]
    outs = pmat.pmat_mul_batched(ctx, dev)
    ctx.sync()
    rnd = random.Random(8)
    for it, C in zip(items, outs):
        m, k, d = it["m"], it["k"], it["d"]
        picks = [(0, 0, 0), (m - 1, k - 1, 2 * d - 2)] + \
            [(rnd.randrange(m), rnd.randrange(k), rnd.randrange(2 * d - 1)) for _ in range(2)]
        idx = torch.tensor([(i * k + kk) * (2 * d - 1) + t for (i, kk, t) in picks], device=C.device)
        got = pmat.to_host(C.reshape(-1)[idx])
        for (i, kk, t), v in zip(picks, got):
            assert int(v) == oracle.pmat_coeff(it["p"], it["A"], it["B"], i, kk, t), (it["m"], it["n"], k, d, i, kk, t)
    ctx.close()
