"""The product entry points inside CUDA graphs: captured once on the context's stream, then
replayed on new inputs written into the same buffers, every replay bit-exact against the oracle.

pmat_mul sizes its workspace and twiddle tables on its first call, so a warm-up call precedes
the capture.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P60 = 1152921504606846883


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_04356_gb300 import Context, build
    build.build()
    s = torch.cuda.Stream()
    ctx = Context(0, stream=s)
    yield ctx, s
    ctx.close()


CASES = [(P60, 8, 6, 5, 4, 700, 900), (synth.P998, 4, 5, 7, 3, 300, 200), (P60, 8, 32, 32, 32, 64, 64)]


def _dev_like(a):
    import torch
    return torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)).cuda()


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_{c[2]}x{c[3]}x{c[4]}_{c[5]}_{c[6]}" for c in CASES])
def test_product_graph_replay(env, case):
    import torch
    from paper_1905_04356_gb300 import pmat
    ctx, s = env
    p, w, m, n, k, dA, dB = case
    dt = np.uint32 if w == 4 else np.uint64
    g0 = synth.rng(sum(case) & 0xffff)
    A = _dev_like(synth.uniform(g0, (m, n, dA), p, dt))
    B = _dev_like(synth.uniform(g0, (n, k, dB), p, dt))
    C = torch.empty((m, k, dA + dB - 1), dtype=A.dtype, device="cuda")

    def call():
        pmat.pmat_mul(ctx, p, A, B, out=C)

    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        call()                                     # warm-up: workspace and tables
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        call()
    for trial in range(3):
        An = synth.uniform(g0, (m, n, dA), p, dt)
        Bn = synth.uniform(g0, (n, k, dB), p, dt)
        A.copy_(_dev_like(An))
        B.copy_(_dev_like(Bn))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        got = got.view(np.uint64) if got.dtype == np.int64 else got.view(np.uint32)
        assert np.array_equal(got.astype(np.uint64), oracle.pmat_mul(p, An.astype(np.uint64), Bn.astype(np.uint64))), trial


def test_batched_graph_replay(env):
    """pmat_mul_batched inside a CUDA graph: a mixed batch (moduli 998244353, 60-bit, 97 and
    2^32 - 5; transform lengths from 16 to 2^15 points, so the column passes run too) is captured
    once after a warm-up call and replayed three times on fresh inputs, every product of every
    replay equal to the oracle's."""
    import random

    import torch
    from paper_1905_04356_gb300 import pmat
    ctx, s = env
    rnd = random.Random(12)
    g0 = synth.rng(12)
    primes = [(synth.P998, 4), (P60, 8), (97, 4), (4294967291, 4), (synth.random_prime(g0, 60), 8)]
    shapes = []
    for i in range(14):
        p, w = primes[i % len(primes)]
        m, n, k = rnd.randint(1, 6), rnd.randint(1, 6), rnd.randint(1, 6)
        dA = rnd.choice([1, 7, 100, 900, 3000]) if i % 7 else 9000
        dB = rnd.choice([1, 5, 300, 2000]) if i % 7 else 8000
        shapes.append((p, w, m, n, k, dA, dB))
    def draw():
        return [(synth.uniform(g0, (m, n, dA), p, np.uint32 if w == 4 else np.uint64),
                 synth.uniform(g0, (n, k, dB), p, np.uint32 if w == 4 else np.uint64))
                for (p, w, m, n, k, dA, dB) in shapes]
    host = draw()
    dev = [(_dev_like(A), _dev_like(B)) for A, B in host]
    outs = [torch.empty((m, k, dA + dB - 1), dtype=dev[i][0].dtype, device="cuda")
            for i, (p, w, m, n, k, dA, dB) in enumerate(shapes)]
    items = [(shapes[i][0], dev[i][0], dev[i][1]) for i in range(len(shapes))]
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        pmat.pmat_mul_batched(ctx, items, outs)   # warm-up: workspace and tables
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pmat.pmat_mul_batched(ctx, items, outs)
    for trial in range(3):
        host = draw()
        for (A, B), (dA_, dB_) in zip(host, dev):
            dA_.copy_(_dev_like(A))
            dB_.copy_(_dev_like(B))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for i, ((A, B), C) in enumerate(zip(host, outs)):
            got = pmat.to_host(C).astype(np.uint64)
            assert np.array_equal(got, oracle.pmat_mul(shapes[i][0], A, B)), (trial, i, shapes[i])
