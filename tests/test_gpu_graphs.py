"""The product entry points inside CUDA graphs: captured once on the context's stream, then
replayed on new inputs written into the same buffers, every replay bit-exact against the oracle.

pmat_mul sizes its workspace and twiddle tables on its first call, so a warm-up call precedes
the capture; pmat_mul_noalloc needs none (its scratch is a fixed device array).
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
@pytest.mark.parametrize("entry", ["pmat_mul", "pmat_mul_noalloc"])
def test_product_graph_replay(env, case, entry):
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
        if entry == "pmat_mul":
            pmat.pmat_mul(ctx, p, A, B, out=C)
        else:
            rc = pmat.lib().pmat_mul_noalloc(p, w, m, n, k, A.data_ptr(), dA, B.data_ptr(), dB, C.data_ptr(),
                                             s.cuda_stream)
            assert rc == 0

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
