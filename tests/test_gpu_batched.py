"""GPU parity of pmat_mul_batched (uneven products binned by transform length)."""
import os
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


def _eval_all(p, X, alpha):
    """X(alpha) for every entry (the oracle's Horner evaluation)."""
    return oracle.pmat_eval(p, X, alpha)


def test_batched_512_every_entry_at_random_points():
    """The 512-product workload (log-uniform m, n, k in [2, 64], lengths in [64, 16384], half mod
    998244353, half mod 60-bit primes): every output entry of every product is checked at two
    seeded random points alpha, C(alpha) = A(alpha) . B(alpha) mod p, with A(alpha), B(alpha) and
    C(alpha) evaluated by the oracle's Horner rule and the matrix product taken by the oracle.  A
    wrong entry of degree < 2d - 1 passes one point with probability below 2d / p (Schwartz-Zippel),
    and a single wrong coefficient c_t never passes (it shifts C(alpha) by a nonzero multiple of
    alpha^t)."""
    import concurrent.futures as cf

    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_04356_gb300 import Context, pmat
    ctx = Context(0)
    items = synth.batch_c4(0)
    dev = [(it["p"], pmat.to_device(it["A"]), pmat.to_device(it["B"])) for it in items]
    outs = pmat.pmat_mul_batched(ctx, dev)
    ctx.sync()
    del dev
    rnd = random.Random(8)
    alphas = [(rnd.randrange(1, it["p"]), rnd.randrange(1, it["p"])) for it in items]

    def check(idx):
        it, al = items[idx], alphas[idx]
        C = pmat.to_host(outs[idx])
        assert C.shape == (it["m"], it["k"], 2 * it["d"] - 1)
        for a in al:
            lhs = _eval_all(it["p"], C, a)
            Aa = _eval_all(it["p"], it["A"], a)[:, :, None]
            Ba = _eval_all(it["p"], it["B"], a)[:, :, None]
            rhs = oracle.pmat_mul(it["p"], Aa, Ba, threads=1)[:, :, 0]
            bad = np.argwhere(lhs != rhs)
            assert bad.size == 0, (idx, it["m"], it["n"], it["k"], it["d"], bad[:4].tolist())
        return idx

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        done = list(ex.map(check, range(len(items))))
    assert len(done) == 512
    ctx.close()
