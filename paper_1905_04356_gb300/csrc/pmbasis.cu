// pmbasis.cu -- PM-Basis (Sec. 3, Algorithm 3) on the device.
//
// Nodes of the recursion: the residual R = MiddleProduct(P1, F, ceil(e/2),
// floor(e/2)) and the product P2 . P1, both through the product hot path
// (prod_slice: NTT -> pointwise -> inverse NTT -> CRT).  Leaves (order e <= T):
// k_mbasis_leaf runs Algorithm 2 (M-Basis) with Algorithm 1 (M-Basis-1) in one
// CTA, in Montgomery arithmetic modulo the word-size prime p.
//
// Shifts stay on the device: a leaf returns rdeg_s(P) by the predictable-degree
// property (independent rows of M-Basis-1 gain x, so their shifted degree grows
// by one; P is s-reduced at every step), and a node returns the shift of its
// right child, rdeg_s(P2 P1) = rdeg_{rdeg_s(P1)}(P2).  Nothing is read back
// before the end of the call.
//
// Leaf, step k (Algorithm 2): R = coefficient k of P.F, read from a residual
// series G kept equal to P.F (G <- Q.G each step, the "list of residuals"
// variant of Sec. 3); rows are visited in increasing (shift, index) order
// (Algorithm 1).  Rows of P and G are kept multiplied by known nonzero
// constants lambda_i, so no modular inversion is needed per step: the generic
// case (the first n rows in that order are independent) is solved by
// fraction-free Gauss-Jordan, any other case by a fraction-free elimination in
// row order; rows are normalised once when the leaf ends.
#include <cooperative_groups.h>
#include <cstring>
#include <vector>

#include "host.h"

#define CKI(call)                                                       \
    do {                                                                \
        int _rc = (call);                                               \
        if (_rc) return _rc;                                            \
    } while (0)

struct LeafArgs {
    u64 p, pn, r2, one;      // p, -p^-1 mod 2^64, 2^128 mod p, 2^64 mod p
    int m, n, T, chunk;      // dimensions, leaf order, terms per Montgomery reduction
    const u64 *F;            // m x n, entry stride sF, plain values in [0, p)
    i64 sF;
    const i64 *s_in;         // shift (device)
    i64 *s_out;              // rdeg_s(P) (device)
    u64 *P;                  // m x m, length T + 1, entry stride sP (plain)
    i64 sP;
    u64 *G0, *G1;            // residual series, m x n x T (Montgomery), double buffer
    u64 *P0, *P1;            // basis, m x m x (T + 1) (Montgomery), double buffer
    const u64 *alpha;        // interpolant leaves: the T points (Montgomery); null for approximants
};

#define LEAF_CL_MAX 16       // leaf cluster size (CTAs), the largest tried

namespace leaf_odd {
#define LEAF_F2 false
#include "leaf_impl.cuh"
#undef LEAF_F2
}  // namespace leaf_odd

namespace leaf_f2 {
#define LEAF_F2 true
#include "leaf_impl.cuh"
#undef LEAF_F2
}  // namespace leaf_f2

namespace leaf_rt {
#define LEAF_F2 (p == 2)
#include "leaf_impl.cuh"
#undef LEAF_F2
}  // namespace leaf_rt

using namespace leaf_rt;    // the node kernels below test the modulus at run time

static size_t elim_bytes(int m, int n)
{
    const int mx = m > n ? m : n;
    const size_t words = (size_t)m + (size_t)m * m + (size_t)n * m + mx + (n + 1) + (size_t)n * n + (size_t)n * m + n + m +
                         (size_t)m * mx;
    return words * 8 + ((size_t)4 * m + 2 * n + 8) * 4;
}

static size_t leaf_smem(int m, int n)
{
    return (size_t)2 * m * 8 + (size_t)m * n * 8 + elim_bytes(m, n) + 64;
}

static size_t leaf_cl_smem(int m, int n, int T, int LEAF_CL)
{
    const int ngm = (n + LEAF_CL - 1) / LEAF_CL, npm = (m + LEAF_CL - 1) / LEAF_CL;
    return (size_t)2 * m * 8 + (size_t)2 * m * n * 8 + (size_t)2 * m * ngm * T * 8 + (size_t)2 * m * npm * (T + 1) * 8 +
           2 * elim_bytes(m, n) + 64;
}

// ------------------------------------------------------------------ host recursion
namespace {

struct PmbCtx {
    pm_ctx *ctx;
    bool use_cluster;
    LeafArgs base;     // p-dependent constants + leaf scratch
    int m, n;
    int64_t T;
    // interpolant bases at the points c q^l (Algorithm 5): the points (Montgomery), the
    // chirp q^C(t) (plain) and q^-C(t) (Montgomery), t < sigma; c and q (plain)
    const u64 *alpha, *h, *hinv;
    u64 c, q;
};

// Bytes of arena the recursion on order e needs (P1, shifts, R, P2 per level).
size_t al256(size_t x) { return (x + 255) / 256 * 256; }

size_t rec_bytes(int m, int n, int64_t e, int64_t T)
{
    if (e <= T) return 0;
    const int64_t e1 = (e + 1) / 2, e2 = e / 2;
    const size_t own = al256((size_t)m * m * (e1 + 1) * 8) + al256((size_t)m * 8) + al256((size_t)m * n * e2 * 8) +
                       al256((size_t)m * m * (e2 + 1) * 8);
    size_t left = rec_bytes(m, n, e1, T), right = rec_bytes(m, n, e2, T);
    return own + (left > right ? left : right);
}

// alpha: null for an approximant leaf, else the leaf's e points (Montgomery form).
int leaf(PmbCtx &C, const u64 *F, int64_t sF, int64_t e, const i64 *s_in, u64 *P, int64_t sP, i64 *s_out,
         const u64 *alpha = nullptr)
{
    pm_ctx *ctx = C.ctx;
    LeafArgs A = C.base;
    A.T = (int)e;
    A.F = F; A.sF = sF; A.s_in = s_in; A.s_out = s_out; A.P = P; A.sP = sP;
    A.alpha = alpha;
    const bool f2 = A.p == 2;              // leaves on bits, else Montgomery arithmetic
    void (*k_cl)(LeafArgs) = f2 ? (alpha ? leaf_f2::k_mbasis_leaf_cl<true> : leaf_f2::k_mbasis_leaf_cl<false>)
                                : (alpha ? leaf_odd::k_mbasis_leaf_cl<true> : leaf_odd::k_mbasis_leaf_cl<false>);
    void (*k_one)(LeafArgs) = f2 ? (alpha ? leaf_f2::k_mbasis_leaf<true> : leaf_f2::k_mbasis_leaf<false>)
                                 : (alpha ? leaf_odd::k_mbasis_leaf<true> : leaf_odd::k_mbasis_leaf<false>);
    int tok = stage_begin(ctx, PM_STAGE_LEAF);
    bool done = false;
    if (C.use_cluster) {
        for (int clsz = LEAF_CL_MAX; clsz >= 8 && !done; clsz /= 2) {
            const size_t smc = leaf_cl_smem(C.m, C.n, (int)e, clsz);
            if (smc > 200 * 1024) continue;
            cudaFuncSetAttribute(k_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
            if (clsz > 8) cudaFuncSetAttribute(k_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(clsz);
            cfg.blockDim = dim3(512);
            cfg.dynamicSmemBytes = smc;
            cfg.stream = ctx->stream;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = clsz;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int ncl = 0;
            if (cudaOccupancyMaxActiveClusters(&ncl, k_cl, &cfg) != cudaSuccess || ncl < 1) {
                cudaGetLastError();
                continue;
            }
            if (cudaLaunchKernelEx(&cfg, k_cl, A) == cudaSuccess) done = true;
            else cudaGetLastError();
        }
    }
    if (!done) {
        // the opt-in is needed whenever static + dynamic shared memory exceed 48 KB
        const size_t sm = leaf_smem(C.m, C.n);
        cudaFuncSetAttribute(k_one, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_one<<<1, 512, sm, ctx->stream>>>(A);
    }
    ctx->launches++;
    cudaError_t err = cudaGetLastError();
    stage_end(ctx, tok);
    return pm_cuda(ctx, err, "k_mbasis_leaf");
}

// Coefficient e of P = P2 P1 (the product of the top coefficients, P2[t2] P1[t1], t1 + t2 = e),
// written to P[e] and taken off P[0]: a cyclic product of length e folds it onto coefficient 0.
__global__ void k_wrap_top(const LeafArgs A, const u64 *P2, i64 s2, i64 t2, const u64 *P1, i64 s1, i64 t1, u64 *P,
                           i64 sP, int m, i64 e)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= m * m) return;
    const int i = x / m, j = x - i * m;
    u64 acc = 0;                                        // sum of a b 2^-64 (Montgomery products)
    for (int l = 0; l < m; l++)
        acc = add64(acc, mmul(P2[(i64)(i * m + l) * s2 + t2], P1[(i64)(l * m + j) * s1 + t1], A), A.p);
    const u64 ce = mmul(acc, A.r2, A);                  // times 2^128 2^-64: the plain sum
    u64 *c = P + (i64)x * sP;
    c[e] = ce;
    c[0] = sub64(c[0], ce, A.p);
}

// Step 6 of Algorithms 3 and 5: P = P2 P1, P2 of length l2 and P1 of length l1, l1 + l2 - 1 = e + 1
// coefficients.  When e is a power of two those need a transform of 2e points; a cyclic product
// of length e instead folds only coefficient e onto coefficient 0, so that one coefficient is
// computed apart (k_wrap_top) and the transforms are half as long.  Below order 512 the
// products are launch-bound and the extra launch costs more than it saves.
#define PMB_WRAP_MIN 512
int node_product(pm_ctx *ctx, const LeafArgs &A, int m, const u64 *P2, int64_t l2, const u64 *P1, int64_t l1,
                 int64_t e, u64 *P, int64_t sP)
{
    if (e < PMB_WRAP_MIN || (e & (e - 1)) != 0)
        return prod_slice(ctx, A.p, 8, m, m, m, P2, l2, l2, P1, l1, l1, 0, e + 1, ceil_log2(e + 1), P, sP);
    CKI(prod_slice(ctx, A.p, 8, m, m, m, P2, l2, l2, P1, l1, l1, 0, e, ceil_log2(e), P, sP));
    int tok = stage_begin(ctx, PM_STAGE_OTHER);
    k_wrap_top<<<(m * m + 127) / 128, 128, 0, ctx->stream>>>(A, P2, l2, l2 - 1, P1, l1, l1 - 1, P, sP, m, e);
    ctx->launches++;
    cudaError_t err = cudaGetLastError();
    stage_end(ctx, tok);
    return pm_cuda(ctx, err, "k_wrap_top");
}

int rec(PmbCtx &C, const u64 *F, int64_t sF, int64_t e, const i64 *s_in, u64 *P, int64_t sP, i64 *s_out)
{
    if (e <= C.T) return leaf(C, F, sF, e, s_in, P, sP, s_out);
    pm_ctx *ctx = C.ctx;
    const int m = C.m, n = C.n;
    const int64_t e1 = (e + 1) / 2, e2 = e / 2;
    const size_t mark = ctx->arena.used;
    u64 *P1 = (u64 *)arena_alloc(ctx, (size_t)m * m * (e1 + 1) * 8);
    i64 *s1 = (i64 *)arena_alloc(ctx, (size_t)m * 8);
    u64 *R = (u64 *)arena_alloc(ctx, (size_t)m * n * e2 * 8);
    u64 *P2 = (u64 *)arena_alloc(ctx, (size_t)m * m * (e2 + 1) * 8);
    if (!P1 || !s1 || !R || !P2) return pm_fail(ctx, PM_ENOMEM, "PM-Basis arena exhausted");
    // step 2: P1 = PM-Basis(F mod x^e1, e1, s)
    CKI(rec(C, F, sF, e1, s_in, P1, e1 + 1, s1));
    // step 3: R = MiddleProduct(P1, F mod x^e, e1, e2)
    CKI(prod_slice(ctx, C.base.p, 8, m, m, n, P1, e1 + 1, e1 + 1, F, e, sF, e1, e2, ceil_log2(e), R, e2));
    // steps 4-5: P2 = PM-Basis(R, e2, rdeg_s(P1))
    CKI(rec(C, R, e2, e2, s1, P2, e2 + 1, s_out));
    // step 6: P = P2 P1 (degree <= e)
    CKI(node_product(ctx, C.base, m, P2, e2 + 1, P1, e1 + 1, e, P, sP));
    ctx->arena.used = mark;
    return PM_OK;
}

// ------------------------------------------------------------------ interpolant bases (Algorithm 5)
// Points alpha_l = c q^l.  The residual of a node, R_l = P1(alpha_{o+e1+l}) E_{e1+l},
// needs P1 at a geometric progression: with C(t) = t (t - 1) / 2 and c' = c q^(o+e1),
// P1(c' q^i) = q^-C(i) sum_e (a_e c'^e q^-C(e)) q^C(i+e) (Sec. 2, evaluation at a
// geometric progression), the middle product of the scaled, reversed coefficients of
// every entry of P1 with the chirp q^C(t) on the product hot path; then a batch of
// e2 constant m x m by m x n products mod p.

// alpha_t = c q^t (Montgomery), h_t = q^C(t) (plain), hinv_t = q^-C(t) (Montgomery)
__global__ void k_ip_tables(const LeafArgs A, u64 qm, u64 qim, u64 cm, u64 *alpha, u64 *h, u64 *hinv, int64_t N)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const u64 c2 = (u64)t * (u64)(t > 0 ? t - 1 : 0) / 2;
        alpha[t] = mmul(cm, mpow(qm, (u64)t, A), A);
        h[t] = mmul(mpow(qm, c2, A), 1, A);
        hinv[t] = mpow(qim, c2, A);
    }
}

// u_e = c'^e q^-C(e) (Montgomery), e < E
__global__ void k_ip_uvec(const LeafArgs A, u64 cpm, const u64 *hinv, u64 *u, int E)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
        u[e] = mmul(mpow(cpm, (u64)e, A), hinv[e], A);
}

// U[r][E-1-e] = P1[r][e] u_e (plain), r < rows
__global__ void k_ip_prep(const LeafArgs A, const u64 *P1, int64_t sP1, const u64 *u, u64 *U, int64_t rows, int E)
{
    const int64_t total = rows * E;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = x / E;
        const int e = (int)(x % E);
        U[r * E + (E - 1 - e)] = mmul(P1[r * sP1 + e], u[e], A);
    }
}

// R[i][j][l] = q^-C(l) sum_k S[i][k][l] E[k][j][l], l < L: S holds q^C(l) P1(c' q^l)
// (m x m, entry stride L), E the second half of the points (entry stride sE), plain values.
__global__ void k_ip_resid(const LeafArgs A, const u64 *S, const u64 *E, int64_t sE, const u64 *hinv, u64 *R,
                           int64_t L)
{
    const int m = A.m, n = A.n;
    const int64_t total = (int64_t)m * n * L;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = x % L, e = x / L;
        const int i = (int)(e / n), j = (int)(e % n);
        u64 hi = 0, lo = 0, acc = 0;
        int cnt = 0;
        for (int k = 0; k < m; k++) {
            mac128(hi, lo, S[((int64_t)i * m + k) * L + l], E[((int64_t)k * n + j) * sE + l]);
            if (++cnt == A.chunk) { acc = add64(acc, fm_redc(hi, lo, A.p, A.pn), A.p); hi = lo = 0; cnt = 0; }
        }
        acc = add64(acc, fm_redc(hi, lo, A.p, A.pn), A.p);   // sum / 2^64
        R[x] = mmul(mmul(acc, hinv[l], A), A.r2, A);
    }
}

int ip_grid(int64_t total)
{
    const int64_t b = (total + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

size_t rec_ip_bytes(int m, int n, int64_t e, int64_t T)
{
    if (e <= T) return 0;
    const int64_t e1 = (e + 1) / 2, e2 = e / 2;
    const size_t mm = (size_t)m * m;
    const size_t own = 2 * al256(mm * (e1 + 1) * 8) + al256((size_t)m * 8) + al256((size_t)(e1 + 1) * 8) +
                       al256(mm * e2 * 8) + al256((size_t)m * n * e2 * 8) + al256(mm * (e2 + 1) * 8);
    size_t left = rec_ip_bytes(m, n, e1, T), right = rec_ip_bytes(m, n, e2, T);
    return own + (left > right ? left : right);
}

// P (m x m, length e + 1, stride sP) = PM-IntBasis of E (m x n, e points from point o,
// entry stride sE) for the shift s_in; s_out = rdeg_s(P).
int rec_ip(PmbCtx &C, const u64 *E, int64_t sE, int64_t e, int64_t o, const i64 *s_in, u64 *P, int64_t sP, i64 *s_out)
{
    if (e <= C.T) return leaf(C, E, sE, e, s_in, P, sP, s_out, C.alpha + o);
    pm_ctx *ctx = C.ctx;
    const int m = C.m, n = C.n;
    const LeafArgs &A = C.base;
    const int64_t e1 = (e + 1) / 2, e2 = e / 2, E1 = e1 + 1, mm = (int64_t)m * m;
    const size_t mark = ctx->arena.used;
    u64 *P1 = (u64 *)arena_alloc(ctx, (size_t)mm * E1 * 8);
    i64 *s1 = (i64 *)arena_alloc(ctx, (size_t)m * 8);
    u64 *U = (u64 *)arena_alloc(ctx, (size_t)mm * E1 * 8);
    u64 *u = (u64 *)arena_alloc(ctx, (size_t)E1 * 8);
    u64 *S = (u64 *)arena_alloc(ctx, (size_t)mm * e2 * 8);
    u64 *R = (u64 *)arena_alloc(ctx, (size_t)m * n * e2 * 8);
    u64 *P2 = (u64 *)arena_alloc(ctx, (size_t)mm * (e2 + 1) * 8);
    if (!P1 || !s1 || !U || !u || !S || !R || !P2) return pm_fail(ctx, PM_ENOMEM, "PM-IntBasis arena exhausted");
    // step 2: P1 = PM-IntBasis(E_0 .. E_{e1-1}, alpha_o .. alpha_{o+e1-1}, s)
    CKI(rec_ip(C, E, sE, e1, o, s_in, P1, E1, s1));
    // step 3: R_l = P1(alpha_{o+e1+l}) E_{e1+l}, l < e2
    {
        const u64 cp = host_mulmod(C.c % A.p, host_powmod(C.q, (uint64_t)(o + e1), A.p), A.p);
        const u64 cpm = host_mulmod(cp, A.one, A.p);
        int tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_ip_uvec<<<ip_grid(E1), 256, 0, ctx->stream>>>(A, cpm, C.hinv, u, (int)E1);
        k_ip_prep<<<ip_grid(mm * E1), 256, 0, ctx->stream>>>(A, P1, E1, u, U, mm, (int)E1);
        ctx->launches += 2;
        cudaError_t err = cudaGetLastError();
        stage_end(ctx, tok);
        CKI(pm_cuda(ctx, err, "k_ip_prep"));
        CKI(prod_slice(ctx, A.p, 8, (int)mm, 1, 1, U, E1, E1, C.h, e1 + e2, e1 + e2, e1, e2, ceil_log2(e1 + e2), S, e2));
        tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_ip_resid<<<ip_grid((int64_t)m * n * e2), 256, 0, ctx->stream>>>(A, S, E + e1, sE, C.hinv, R, e2);
        ctx->launches++;
        err = cudaGetLastError();
        stage_end(ctx, tok);
        CKI(pm_cuda(ctx, err, "k_ip_resid"));
    }
    // steps 4-5: P2 = PM-IntBasis(R, alpha_{o+e1} .. alpha_{o+e-1}, rdeg_s(P1))
    CKI(rec_ip(C, R, e2, e2, o + e1, s1, P2, e2 + 1, s_out));
    // step 6: P = P2 P1 (degree <= e)
    CKI(node_product(ctx, A, m, P2, e2 + 1, P1, E1, e, P, sP));
    ctx->arena.used = mark;
    return PM_OK;
}

// Constants and leaf scratch shared by both entry points.
int pmb_setup(pm_ctx *ctx, PmbCtx &C, uint64_t p, int m, int n, int64_t Tl, size_t extra)
{
    C.ctx = ctx;
    C.use_cluster = ctx->opt_leaf_cluster != 0;
    C.m = m;
    C.n = n;
    C.T = ctx->opt_T;
    C.alpha = C.h = C.hinv = nullptr;
    C.c = C.q = 0;
    LeafArgs &A = C.base;
    memset(&A, 0, sizeof(A));
    A.p = p;
    uint64_t inv = 1;                       // p^-1 mod 2^64 by Newton iteration
    for (int i = 0; i < 7; i++) inv *= 2 - p * inv;
    A.pn = (uint64_t)0 - inv;
    A.one = (uint64_t)(((unsigned __int128)1 << 64) % p);
    A.r2 = (uint64_t)((unsigned __int128)A.one * A.one % p);
    if (p == 2) A.one = A.r2 = 1;           // bits: the Montgomery form is the identity
    A.m = m;
    A.n = n;
    uint64_t ch = ~0ull / p;
    A.chunk = (int)(ch > 16 ? 16 : ch);
    const size_t leafG = (size_t)m * n * Tl * 8, leafP = (size_t)m * m * (Tl + 1) * 8;
    CKI(arena_reserve(ctx, extra + 2 * al256(leafG) + 2 * al256(leafP)));
    A.G0 = (u64 *)arena_alloc(ctx, leafG);
    A.G1 = (u64 *)arena_alloc(ctx, leafG);
    A.P0 = (u64 *)arena_alloc(ctx, leafP);
    A.P1 = (u64 *)arena_alloc(ctx, leafP);
    if (!A.G0 || !A.G1 || !A.P0 || !A.P1) return pm_fail(ctx, PM_ENOMEM, "arena too small");
    return PM_OK;
}

int pmb_check(pm_ctx *ctx, uint64_t p, int m, int n, int64_t d)
{
    if (m < 1 || n < 1 || d < 1) return pm_fail(ctx, PM_EINVAL, "need m, n >= 1 and an order >= 1");
    if (p < 2 || (p > 2 && !(p & 1)) || p >= (1ull << 62)) return pm_fail(ctx, PM_EINVAL, "need a prime p < 2^62");
    if (m > 128 || n > 128) return pm_fail(ctx, PM_EUNSUPPORTED, "m, n <= 128 supported");
    if (d + 1 > (1 << PM_MAX_LOG2L)) return pm_fail(ctx, PM_EINVAL, "order too large for the transforms");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    if (leaf_smem(m, n) > 200 * 1024) return pm_fail(ctx, PM_EUNSUPPORTED, "leaf workspace too large");
    return PM_OK;
}

}  // namespace

extern "C" int pm_intbasis(pm_ctx *ctx, uint64_t p, int m, int n, const void *E, int64_t sigma, uint64_t c,
                           uint64_t q, const int64_t *shift, void *P, int64_t *rdeg_out)
{
    if (!ctx) return PM_EINVAL;
    CKI(pmb_check(ctx, p, m, n, sigma));
    if (!E || !shift || !P || !rdeg_out) return pm_fail(ctx, PM_EINVAL, "null buffer");
    if (c >= p || q == 0 || q >= p) return pm_fail(ctx, PM_EINVAL, "need c in [0, p) and q in [1, p)");
    PmbCtx C;
    const int64_t T = ctx->opt_T, Tl = sigma < T ? sigma : T;
    const size_t need = rec_ip_bytes(m, n, sigma, T) + 3 * al256((size_t)sigma * 8) + 2 * al256((size_t)m * 8);
    CKI(pmb_setup(ctx, C, p, m, n, Tl, need));
    const LeafArgs &A = C.base;
    u64 *alpha = (u64 *)arena_alloc(ctx, (size_t)sigma * 8);
    u64 *h = (u64 *)arena_alloc(ctx, (size_t)sigma * 8);
    u64 *hinv = (u64 *)arena_alloc(ctx, (size_t)sigma * 8);
    i64 *s_in = (i64 *)arena_alloc(ctx, (size_t)m * 8);
    i64 *s_out = (i64 *)arena_alloc(ctx, (size_t)m * 8);
    if (!alpha || !h || !hinv || !s_in || !s_out) return pm_fail(ctx, PM_ENOMEM, "arena too small");
    C.alpha = alpha;
    C.h = h;
    C.hinv = hinv;
    C.c = c;
    C.q = q;
    {
        const u64 qm = host_mulmod(q, A.one, p), qim = host_mulmod(host_powmod(q, p - 2, p), A.one, p);
        const u64 cm = host_mulmod(c, A.one, p);
        int tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_ip_tables<<<ip_grid(sigma), 256, 0, ctx->stream>>>(A, qm, qim, cm, alpha, h, hinv, sigma);
        ctx->launches++;
        cudaError_t err = cudaGetLastError();
        stage_end(ctx, tok);
        CKI(pm_cuda(ctx, err, "k_ip_tables"));
    }
    CKI(pm_cuda(ctx, cudaMemcpyAsync(s_in, shift, (size_t)m * 8, cudaMemcpyHostToDevice, ctx->stream), "shift H2D"));
    CKI(rec_ip(C, (const u64 *)E, sigma, sigma, 0, s_in, (u64 *)P, sigma + 1, s_out));
    CKI(pm_cuda(ctx, cudaMemcpyAsync(rdeg_out, s_out, (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream), "rdeg D2H"));
    CKI(pm_cuda(ctx, cudaStreamSynchronize(ctx->stream), "pm_intbasis sync"));
    return PM_OK;
}

extern "C" int pm_basis(pm_ctx *ctx, uint64_t p, int m, int n, const void *F, int64_t lenF, int64_t d,
                        const int64_t *shift, void *P, int64_t *rdeg_out)
{
    if (!ctx) return PM_EINVAL;
    CKI(pmb_check(ctx, p, m, n, d));
    if (lenF < 1) return pm_fail(ctx, PM_EINVAL, "need lenF >= 1");
    if (!F || !shift || !P || !rdeg_out) return pm_fail(ctx, PM_EINVAL, "null buffer");
    PmbCtx C;
    const int64_t T = ctx->opt_T, Tl = d < T ? d : T;   // largest leaf order
    // arena: recursion buffers + leaf scratch + the two shift vectors
    const size_t padF = lenF < d ? al256((size_t)m * n * d * 8) : 0;
    CKI(pmb_setup(ctx, C, p, m, n, Tl, rec_bytes(m, n, d, T) + 2 * al256((size_t)m * 8) + padF));
    i64 *s_in = (i64 *)arena_alloc(ctx, (size_t)m * 8);
    i64 *s_out = (i64 *)arena_alloc(ctx, (size_t)m * 8);
    if (!s_in || !s_out) return pm_fail(ctx, PM_ENOMEM, "arena too small");
    // only F mod x^d is read: a shorter F is copied into a zero-padded buffer of length d
    const u64 *Fd = (const u64 *)F;
    int64_t sF = lenF;
    if (lenF < d) {
        u64 *Fp = (u64 *)arena_alloc(ctx, (size_t)m * n * d * 8);
        if (!Fp) return pm_fail(ctx, PM_ENOMEM, "arena too small");
        CKI(pm_cuda(ctx, cudaMemsetAsync(Fp, 0, (size_t)m * n * d * 8, ctx->stream), "pad F"));
        CKI(pm_cuda(ctx, cudaMemcpy2DAsync(Fp, (size_t)d * 8, F, (size_t)lenF * 8, (size_t)lenF * 8, (size_t)m * n,
                                           cudaMemcpyDeviceToDevice, ctx->stream), "copy F"));
        Fd = Fp;
        sF = d;
    }
    CKI(pm_cuda(ctx, cudaMemcpyAsync(s_in, shift, (size_t)m * 8, cudaMemcpyHostToDevice, ctx->stream), "shift H2D"));
    CKI(rec(C, Fd, sF, d, s_in, (u64 *)P, d + 1, s_out));
    CKI(pm_cuda(ctx, cudaMemcpyAsync(rdeg_out, s_out, (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream), "rdeg D2H"));
    CKI(pm_cuda(ctx, cudaStreamSynchronize(ctx->stream), "pm_basis sync"));
    return PM_OK;
}
