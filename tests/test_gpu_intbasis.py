"""GPU parity of PM-IntBasis (Algorithm 5 on the device, geometric points) against the oracle.

The device computes the basis at the points alpha_l = c q^l: leaves run Algorithm 4 on the
list of residuals P(alpha_l) E_l, nodes evaluate P1 at the second half of the points by a
chirp middle product.  The CPU pins show that the oracle's PM-IntBasis equals its
M-IntBasis for every threshold, so the device output must match the oracle on every
coefficient, and rdeg_s(P) too.  Tiny primes make residuals singular and points repeat
(q of small order), q = 1 puts every point at c, c = 0 puts them all at 0.
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


def _run(ctx, p, E, c, q, s, T=None, cluster=1):
    from paper_1905_04356_gb300 import pmat
    if T is not None:
        ctx.set_option(pmat.PM_OPT_THRESHOLD, T)
    ctx.set_option(pmat.PM_OPT_LEAF_CLUSTER, cluster)
    try:
        P, rd = pmat.pm_intbasis(ctx, p, pmat.to_device(E), c, q, s)
        ctx.sync()
    finally:
        ctx.set_option(pmat.PM_OPT_THRESHOLD, 32)
        ctx.set_option(pmat.PM_OPT_LEAF_CLUSTER, 1)
    return pmat.to_host(P), rd


def _points(p, c, q, sigma):
    return [c * pow(q, l, p) % p for l in range(sigma)]


CASES = [
    # p, m, n, sigma, T, c, q
    (P60, 2, 1, 6, 32, 3, 5),
    (P60, 4, 2, 16, 4, 7, 11),
    (P60, 5, 3, 33, 8, 2, 3),
    (P60, 6, 2, 20, 1, 9, 2),
    (P60, 8, 4, 100, 32, 5, 7),
    (P60, 32, 16, 64, 32, 3, 7),
    (P60, 32, 16, 200, 16, 11, 13),
    (P60, 16, 8, 150, 32, 5, 3),       # the [H; -I] shape of the resultant variant
    (97, 4, 2, 16, 4, 3, 5),           # q of order 96
    (7, 5, 2, 23, 3, 3, 2),            # q of order 3: points repeat
    (3, 3, 1, 12, 32, 1, 2),
    (synth.P998, 6, 3, 40, 8, 3, 3),
    (P60, 3, 3, 10, 4, 4, 6),          # m = n
    (P60, 2, 4, 9, 32, 5, 2),          # m < n
    (P60, 4, 2, 20, 4, 6, 1),          # q = 1: every point is c
    (P60, 4, 2, 20, 4, 0, 5),          # c = 0: every point is 0
    (2, 4, 2, 30, 4, 1, 1),            # p = 2: every point is 1 (the leaves on bits)
    (2, 6, 3, 64, 16, 0, 1),           # p = 2, every point 0
    (2, 32, 16, 100, 32, 1, 1),
]


@pytest.mark.parametrize("case", CASES, ids=[f"p{c[0]}_{c[1]}x{c[2]}_s{c[3]}_T{c[4]}" for c in CASES])
def test_pm_intbasis_matches_oracle(ctx, case):
    p, m, n, sigma, T, c, q = case
    g = synth.rng(sum(case) & 0xffff)
    E = synth.uniform(g, (m, n, sigma), p, np.uint64)
    rnd = random.Random(sigma)
    alpha = _points(p, c, q, sigma)
    for s in ([0] * m, [rnd.randrange(-5, 6) for _ in range(m)]):
        P, rd = _run(ctx, p, E, c, q, s, T)
        Pexp, rdexp = oracle.pmintbasis(p, E, alpha, s, T)
        assert np.array_equal(P, Pexp), (case, s)
        assert np.array_equal(rd, rdexp), (case, s)


@pytest.mark.parametrize("case", [(P60, 6, 2, 40, 8, 3, 5), (97, 5, 3, 30, 32, 5, 3), (P60, 32, 16, 96, 32, 7, 3),
                                  (2, 5, 3, 30, 32, 1, 1)])
def test_single_cta_leaf_matches_oracle(ctx, case):
    """The one-CTA interpolant leaf (basis in global memory) gives the same bases."""
    p, m, n, sigma, T, c, q = case
    g = synth.rng(91 + sigma)
    E = synth.uniform(g, (m, n, sigma), p, np.uint64)
    s = [(i * 7) % 5 - 2 for i in range(m)]
    P, rd = _run(ctx, p, E, c, q, s, T, cluster=0)
    Pexp, rdexp = oracle.pmintbasis(p, E, _points(p, c, q, sigma), s, T)
    assert np.array_equal(P, Pexp) and np.array_equal(rd, rdexp)


def test_pm_intbasis_32x16_1024_points_matches_oracle(ctx):
    """Several recursion levels with chirp evaluations of length up to 1024."""
    p, m, n, sigma = P60, 32, 16, 1024
    E = synth.uniform(synth.rng(5), (m, n, sigma), p, np.uint64)
    c, q = 5, 3
    P, rd = _run(ctx, p, E, c, q, [0] * m, 32)
    Pexp, rdexp = oracle.pmintbasis(p, E, _points(p, c, q, sigma), [0] * m, 32)
    assert np.array_equal(P, Pexp) and np.array_equal(rd, rdexp)


def test_pm_intbasis_full_size_properties(ctx):
    """E 32 x 16 at 8192 geometric points (the bench workload): every sampled point is
    interpolated (P(alpha_l) E_l = 0 by the oracle's evaluation), the basis is s-ordered
    weak Popov with the returned s-row-degree, and the degrees sum to n sigma (generic E)."""
    W = synth.intbasis_w(0)
    p, E, c, q, s = W["p"], W["E"], W["c"], W["q"], W["shift"]
    m, n, sigma = E.shape
    P, rd = _run(ctx, p, E, c, q, s, 32)
    assert np.array_equal(rd, oracle.rdeg(P, s))
    assert int(rd.sum()) == n * sigma
    # s-ordered weak Popov: the s-pivot of row i (rightmost column reaching its s-degree)
    # sits in column i (generic case)
    nz = P != 0
    deg = np.where(nz.any(-1), sigma - np.argmax(nz[..., ::-1], axis=-1), -(1 << 40)) + np.asarray(s)[None, :]
    for i in range(m):
        top = deg[i].max()
        assert top == rd[i] and deg[i, i] == top and (deg[i, i + 1:] < top).all(), i
    rnd = random.Random(1)
    for l in [0, 1, sigma // 2 - 1, sigma // 2, sigma - 1] + [rnd.randrange(sigma) for _ in range(3)]:
        a = c * pow(q, l, p) % p
        Pa = oracle.pmat_eval(p, P, a)
        El = np.ascontiguousarray(E[:, :, l:l + 1])
        prod = oracle.pmat_mul(p, Pa.reshape(m, m, 1), El)
        assert not prod.any(), l


def test_pm_intbasis_rejects_bad_arguments(ctx):
    from paper_1905_04356_gb300 import PmError, pmat
    E = pmat.to_device(np.ones((2, 1, 4), dtype=np.uint64))
    for p, c, q in [(1 << 20, 1, 2), (P60, 1, 0), (P60, P60, 2), (P60, 1, P60)]:
        with pytest.raises(PmError) as e:
            pmat.pm_intbasis(ctx, p, E, c, q, [0, 0])
        assert e.value.code == pmat.PM_EINVAL


@pytest.mark.parametrize("case", [(P60, 3, 2, 1, 32, 5, 3, 1), (P60, 4, 2, 17, 1, 2, 3, 0), (97, 2, 3, 12, 2, 3, 5, 1),
                                  (P60, 5, 5, 9, 4, 7, 2, 1)],
                         ids=["one_point", "T1_one_cta", "m_lt_n_p97", "m_eq_n"])
def test_pm_intbasis_edge_cases(ctx, case):
    """One point; threshold 1 with the one-CTA leaf; m < n over F_97; m = n (no fast path)."""
    p, m, n, sigma, T, c, q, cluster = case
    g = synth.rng(sum(case) & 0xfff)
    E = synth.uniform(g, (m, n, sigma), p, np.uint64)
    s = [(3 * i) % 4 - 1 for i in range(m)]
    P, rd = _run(ctx, p, E, c, q, s, T, cluster=cluster)
    Pexp, rdexp = oracle.pmintbasis(p, E, _points(p, c, q, sigma), s, T)
    assert np.array_equal(P, Pexp) and np.array_equal(rd, rdexp)
