"""pmat_mul_noalloc: the product for callers that cannot allocate device memory.

It must give exactly what pmat_mul gives (bit for bit: products over F_p are
exact), on consecutive calls that reuse its fixed scratch array, and must
refuse work that does not fit that array.  This file sorts last so that a run
stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes as C

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
    ctx = Context(0)
    yield ctx
    ctx.close()


def _noalloc(p, A, B):
    import torch
    from paper_1905_04356_gb300 import pmat
    m, n, dA = A.shape
    _, k, dB = B.shape
    out = torch.empty((m, k, dA + dB - 1), dtype=A.dtype, device=A.device)
    stream = torch.cuda.current_stream().cuda_stream
    rc = pmat.lib().pmat_mul_noalloc(p, pmat.width(A), m, n, k, A.data_ptr(), dA, B.data_ptr(), dB,
                                     out.data_ptr(), C.c_void_p(stream))
    assert rc == pmat.PM_OK, pmat.STATUS_NAMES.get(rc, rc)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("p,w,shape", [
    (synth.P998, 4, (4, 4, 4, 256, 256)),      # one NTT prime, written directly
    (P60, 8, (5, 3, 4, 700, 900)),             # 5 CRT primes
    (P60, 8, (1, 2, 1, 9000, 8000)),           # 2^14-point transforms (column pass)
    (1000000007, 4, (3, 5, 2, 300, 200)),      # CRT into uint32 output (p not an NTT prime)
    (1 << 32, 4, (2, 3, 2, 100, 120)),         # even p: Garner's mixed radix
    (3, 4, (2, 1, 2, 2, 2)),                   # one CRT prime, not used directly
])
def test_noalloc_matches_pmat_mul_twice(env, p, w, shape):
    from paper_1905_04356_gb300 import pmat
    m, n, k, dA, dB = shape
    dt = np.uint32 if w == 4 else np.uint64
    for call in range(2):                       # two calls in a row share the scratch array
        g = synth.rng(100 + call)
        A = pmat.to_device(synth.uniform(g, (m, n, dA), p, dt))
        B = pmat.to_device(synth.uniform(g, (n, k, dB), p, dt))
        got = pmat.to_host(_noalloc(p, A, B))
        ref = pmat.pmat_mul(env, p, A, B)
        env.sync()
        assert np.array_equal(got, pmat.to_host(ref)), call
        if dA * dB * m * n * k <= 10 ** 8:          # small enough for the oracle too
            exp = oracle.pmat_mul(p, pmat.to_host(A), pmat.to_host(B))
            assert np.array_equal(got.astype(np.uint64), exp), call


def test_noalloc_rejects_work_beyond_its_scratch(env):
    import torch
    from paper_1905_04356_gb300 import pmat
    A = torch.zeros((32, 32, 4096), dtype=torch.int64, device="cuda")
    B = torch.zeros((32, 32, 4096), dtype=torch.int64, device="cuda")
    out = torch.empty((32, 32, 8191), dtype=torch.int64, device="cuda")
    rc = pmat.lib().pmat_mul_noalloc(P60, 8, 32, 32, 32, A.data_ptr(), 4096, B.data_ptr(), 4096, out.data_ptr(),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == pmat.PM_ESCRATCH
    rc = pmat.lib().pmat_mul_noalloc(P60, 8, 0, 1, 1, A.data_ptr(), 1, B.data_ptr(), 1, out.data_ptr(), None)
    assert rc == pmat.PM_EINVAL
    # a length beyond 2^20 is refused before dA + dB - 1 is formed (nothing runs, nothing is read)
    rc = pmat.lib().pmat_mul_noalloc(P60, 8, 1, 1, 1, A.data_ptr(), (1 << 62), B.data_ptr(), (1 << 62),
                                     out.data_ptr(), None)
    assert rc == pmat.PM_EINVAL
