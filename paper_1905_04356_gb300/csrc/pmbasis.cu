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
};

// ------------------------------------------------------------------ device arithmetic
__device__ __forceinline__ u64 redc128(u64 hi, u64 lo, u64 p, u64 pn)
{
    // (hi 2^64 + lo) / 2^64 mod p for hi 2^64 + lo < p 2^64
    u64 m = lo * pn;
    u64 r = hi + __umul64hi(m, p) + (lo != 0);
    return csub64(r, p);
}
__device__ __forceinline__ void mac128(u64 &hi, u64 &lo, u64 a, u64 b)
{
    u64 l = a * b, h = __umul64hi(a, b);
    lo += l;
    hi += h + (lo < l);
}
__device__ __forceinline__ u64 mmul(u64 a, u64 b, const LeafArgs &A) { return mont_mul(a, b, A.p, A.pn); }
__device__ u64 mpow(u64 a, u64 e, const LeafArgs &A)
{
    u64 r = A.one;
    while (e) {
        if (e & 1) r = mmul(r, a, A);
        a = mmul(a, a, A);
        e >>= 1;
    }
    return r;
}

// ------------------------------------------------------------------ leaf kernel
// Shared memory (dynamic): t[m] i64, lam[m], kap[m], W[m][m], R[m][n], M[n][m],
// piv[n], ord[m], ind[m], misc.
__global__ void __launch_bounds__(512) k_mbasis_leaf(const LeafArgs A)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int m = A.m, n = A.n, T = A.T;
    const u64 p = A.p;
    const int tid = threadIdx.x, nth = blockDim.x;
    i64 *t = (i64 *)smraw;
    u64 *lam = (u64 *)(t + m);
    u64 *kap = lam + m;
    u64 *W = kap + m;               // W[j*m + i]: -(coefficient of e_i) in the scaled row j of Q
    u64 *R = W + m * m;             // R[i*n + c]
    u64 *M = R + m * n;             // M[c*m + pos]  (Gauss-Jordan on [R_I^T | R_D^T])
    u64 *fac = M + n * m;           // column snapshot, n
    u64 *dpr = fac + (m > n ? m : n);   // pivots / prefix products, n + 1
    u64 *bas = dpr + n + 1;         // general path: basis vectors [n][n]
    u64 *tb = bas + n * n;          // general path: transformations [n][m]
    u64 *vv = tb + n * m;           // general path: v[n], tv[m]
    u64 *tv = vv + n;
    int *ord = (int *)(tv + m);
    int *ind = ord + m;             // 1 = independent at this step
    int *pcs = ind + m;             // general path: pivot columns [n]
    int *misc = pcs + n;            // misc[0] = fast path ok, misc[1] = pivot row, misc[2] = rank, misc[3] = pc

    u64 *G = A.G0, *Gn = A.G1, *P = A.P0, *Pn = A.P1;
    for (int i = tid; i < m; i += nth) { t[i] = A.s_in[i]; lam[i] = A.one; }
    for (int x = tid; x < m * n * T; x += nth) {
        const int a = x % T, e = x / T;
        G[x] = mmul(A.F[(i64)e * A.sF + a], A.r2, A);
    }
    const int LP = T + 1;
    for (int x = tid; x < m * m * LP; x += nth) {
        const int a = x % LP, e = x / LP;
        P[x] = (a == 0 && (e / m) == (e % m)) ? A.one : 0;
    }
    __syncthreads();

    for (int k = 0; k < T; k++) {
        // ---- order rows by (t_i, i); gather the residual R = G[:, :, k]
        for (int i = tid; i < m; i += nth) {
            int r = 0;
            const i64 ti = t[i];
            for (int j = 0; j < m; j++) r += (t[j] < ti) || (t[j] == ti && j < i);
            ord[r] = i;
            ind[i] = 0;
            kap[i] = A.one;
        }
        for (int x = tid; x < m * n; x += nth) R[x] = G[(i64)x * T + k];
        for (int x = tid; x < m * m; x += nth) W[x] = 0;
        if (tid == 0) misc[0] = 0;
        __syncthreads();

        // ---- fast path: the first n rows in order are independent (needs m > n)
        if (m > n) {
            for (int x = tid; x < n * m; x += nth) {
                const int c = x / m, pos = x % m;
                M[x] = R[ord[pos] * n + c];
            }
            if (tid == 0) misc[0] = 1;
            __syncthreads();
            for (int s = 0; s < n; s++) {
                if (tid == 0) {
                    int r = -1;
                    for (int c = s; c < n; c++) if (M[c * m + s]) { r = c; break; }
                    misc[1] = r;
                    if (r < 0) misc[0] = 0;
                }
                __syncthreads();
                const int r = misc[1];
                if (r < 0) break;
                if (r != s)
                    for (int col = tid; col < m; col += nth) {
                        u64 a = M[s * m + col];
                        M[s * m + col] = M[r * m + col];
                        M[r * m + col] = a;
                    }
                __syncthreads();
                for (int c = tid; c < n; c += nth) fac[c] = M[c * m + s];
                __syncthreads();
                const u64 pv = M[s * m + s];
                for (int x = tid; x < n * m; x += nth) {
                    const int c = x / m, col = x % m;
                    if (c == s) continue;
                    const u64 f = fac[c];
                    M[x] = sub64(mmul(pv, M[x], A), mmul(f, M[s * m + col], A), p);
                }
                __syncthreads();
            }
            if (misc[0]) {
                // prefix / suffix products of the pivots d_r = M[r][r]:
                // W[j][ord[r]] = -Y[r][j] prod_{r' != r} d_r', kap_j = prod d
                if (tid == 0) {
                    u64 acc = A.one;
                    for (int r = 0; r < n; r++) { dpr[r] = acc; acc = mmul(acc, M[r * m + r], A); }
                    dpr[n] = acc;   // product of all pivots
                    u64 suf = A.one;
                    for (int r = n - 1; r >= 0; r--) { fac[r] = mmul(dpr[r], suf, A); suf = mmul(suf, M[r * m + r], A); }
                }
                __syncthreads();
                for (int x = tid; x < (m - n) * n; x += nth) {
                    const int jp = n + x / n, r = x % n;
                    const int j = ord[jp], i = ord[r];
                    const u64 w = mmul(M[r * m + jp], fac[r], A);   // the relation's coefficient of R_i
                    W[j * m + i] = w ? p - w : 0;                   // stored negated: Q'_j = kap_j e_j - w e_i
                }
                for (int pos = tid; pos < m; pos += nth) {
                    const int i = ord[pos];
                    if (pos < n) ind[i] = 1;
                    else kap[i] = dpr[n];
                }
            }
            __syncthreads();
        }

        // ---- general path: rows in order, fraction-free common-denominator elimination
        if (!misc[0]) {
            for (int x = tid; x < m * m; x += nth) W[x] = 0;
            if (tid == 0) { misc[2] = 0; dpr[0] = A.one; }
            __syncthreads();
            for (int pos = 0; pos < m; pos++) {
                const int r = ord[pos];
                const int rank = misc[2];
                const u64 D = dpr[0];
                // v = D R_r - sum_b R_r[pc_b] bas_b ; tv = D e_r - sum_b R_r[pc_b] tb_b
                for (int x = tid; x < n + m; x += nth) {
                    u64 acc;
                    if (x < n) {
                        acc = mmul(D, R[r * n + x], A);
                        for (int b = 0; b < rank; b++)
                            acc = sub64(acc, mmul(R[r * n + pcs[b]], bas[b * n + x], A), p);
                        vv[x] = acc;
                    } else {
                        const int i = x - n;
                        acc = (i == r) ? D : 0;
                        for (int b = 0; b < rank; b++)
                            acc = sub64(acc, mmul(R[r * n + pcs[b]], tb[b * m + i], A), p);
                        tv[i] = acc;
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    int pc = -1;
                    for (int c = 0; c < n; c++) if (vv[c]) { pc = c; break; }
                    misc[3] = pc;
                }
                __syncthreads();
                const int pc = misc[3];
                if (pc >= 0) {
                    const u64 pv = vv[pc];
                    for (int b = tid; b < rank; b += nth) fac[b] = bas[b * n + pc];
                    __syncthreads();
                    for (int x = tid; x < rank * (n + m); x += nth) {
                        const int b = x / (n + m), c = x % (n + m);
                        if (c < n) bas[b * n + c] = sub64(mmul(pv, bas[b * n + c], A), mmul(fac[b], vv[c], A), p);
                        else tb[b * m + (c - n)] = sub64(mmul(pv, tb[b * m + (c - n)], A), mmul(fac[b], tv[c - n], A), p);
                    }
                    for (int c = tid; c < n + m; c += nth) {
                        if (c < n) bas[rank * n + c] = mmul(D, vv[c], A);
                        else tb[rank * m + (c - n)] = mmul(D, tv[c - n], A);
                    }
                    __syncthreads();
                    if (tid == 0) { pcs[rank] = pc; misc[2] = rank + 1; dpr[0] = mmul(pv, D, A); ind[r] = 1; }
                } else {
                    // dependent: Q'_r = tv (tv[r] = D), i.e. kap_r = D, W[r][i] = tv[i] for i != r
                    for (int i = tid; i < m; i += nth)
                        if (i != r) W[r * m + i] = tv[i];
                    if (tid == 0) kap[r] = D;
                }
                __syncthreads();
            }
        }
        __syncthreads();

        // ---- updates: G <- Q' G (coefficients k+1 .. T-1), P <- Q' P, lam, t
        // independent rows: x . row (shift by one coefficient); dependent j: kap_j row_j + sum_i W[j][i] row_i
        const int chunk = A.chunk;
        const int ngl = T - k - 1;
        for (int x = tid; x < m * n * ngl; x += nth) {
            const int a = k + 1 + x % ngl, e = x / ngl, j = e / n, c = e % n;
            u64 val;
            if (ind[j]) val = G[(i64)e * T + a - 1];
            else {
                u64 hi = 0, lo = 0, accm = 0;
                int cnt = 1;
                mac128(hi, lo, kap[j], G[(i64)e * T + a]);
                for (int i = 0; i < m; i++) {
                    const u64 w = W[j * m + i];
                    if (!w) continue;
                    mac128(hi, lo, w, G[((i64)i * n + c) * T + a]);
                    if (++cnt == chunk) { accm = add64(accm, redc128(hi, lo, p, A.pn), p); hi = lo = 0; cnt = 0; }
                }
                val = add64(accm, redc128(hi, lo, p, A.pn), p);
            }
            Gn[(i64)e * T + a] = val;
        }
        const int np = k + 2;   // P has degree <= k before the step, <= k + 1 after
        for (int x = tid; x < m * m * np; x += nth) {
            const int a = x % np, e = x / np, j = e / m, c = e % m;
            u64 val;
            if (ind[j]) val = a ? P[(i64)e * LP + a - 1] : 0;
            else if (a == k + 1) val = 0;
            else {
                u64 hi = 0, lo = 0, accm = 0;
                int cnt = 1;
                mac128(hi, lo, kap[j], P[(i64)e * LP + a]);
                for (int i = 0; i < m; i++) {
                    const u64 w = W[j * m + i];
                    if (!w) continue;
                    mac128(hi, lo, w, P[((i64)i * m + c) * LP + a]);
                    if (++cnt == chunk) { accm = add64(accm, redc128(hi, lo, p, A.pn), p); hi = lo = 0; cnt = 0; }
                }
                val = add64(accm, redc128(hi, lo, p, A.pn), p);
            }
            Pn[(i64)e * LP + a] = val;
        }
        __syncthreads();
        for (int i = tid; i < m; i += nth) {
            if (ind[i]) t[i] += 1;
            else lam[i] = mmul(kap[i], lam[i], A);
        }
        { u64 *s = G; G = Gn; Gn = s; s = P; P = Pn; Pn = s; }
        __syncthreads();
    }

    // ---- normalise rows (P_true = lam^-1 P) and leave Montgomery form
    for (int i = tid; i < m; i += nth) {
        const u64 inv = mpow(lam[i], p - 2, A);     // Montgomery form of lam_i^-1
        kap[i] = mmul(inv, 1, A);                   // plain lam_i^-1
        A.s_out[i] = t[i];
    }
    __syncthreads();
    for (int x = tid; x < m * m * LP; x += nth) {
        const int a = x % LP, e = x / LP, i = e / m;
        A.P[(i64)e * A.sP + a] = mmul(P[x], kap[i], A);
    }
}

static size_t leaf_smem(int m, int n)
{
    const int mx = m > n ? m : n;
    size_t words = (size_t)m * 3 + (size_t)m * m + (size_t)m * n + (size_t)n * m + mx + (n + 1) + (size_t)n * n +
                   (size_t)n * m + n + m;
    return words * 8 + (size_t)(3 * m + n + 8) * 4 + 64;
}

// ------------------------------------------------------------------ host recursion
namespace {

struct PmbCtx {
    pm_ctx *ctx;
    LeafArgs base;     // p-dependent constants + leaf scratch
    int m, n;
    int64_t T;
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

int leaf(PmbCtx &C, const u64 *F, int64_t sF, int64_t e, const i64 *s_in, u64 *P, int64_t sP, i64 *s_out)
{
    pm_ctx *ctx = C.ctx;
    LeafArgs A = C.base;
    A.T = (int)e;
    A.F = F; A.sF = sF; A.s_in = s_in; A.s_out = s_out; A.P = P; A.sP = sP;
    const size_t sm = leaf_smem(C.m, C.n);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_mbasis_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int tok = stage_begin(ctx, PM_STAGE_LEAF);
    k_mbasis_leaf<<<1, 512, sm, ctx->stream>>>(A);
    ctx->launches++;
    cudaError_t err = cudaGetLastError();
    stage_end(ctx, tok);
    return pm_cuda(ctx, err, "k_mbasis_leaf");
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
    CKI(prod_slice(ctx, C.base.p, 8, m, m, m, P2, e2 + 1, e2 + 1, P1, e1 + 1, e1 + 1, 0, e + 1, ceil_log2(e + 1), P,
                   sP));
    ctx->arena.used = mark;
    return PM_OK;
}

}  // namespace

extern "C" int pm_basis(pm_ctx *ctx, uint64_t p, int m, int n, const void *F, int64_t lenF, int64_t d,
                        const int64_t *shift, void *P, int64_t *rdeg_out)
{
    if (!ctx) return PM_EINVAL;
    if (m < 1 || n < 1 || d < 1 || lenF < 1) return pm_fail(ctx, PM_EINVAL, "need m, n, d, lenF >= 1");
    if (p < 3 || !(p & 1) || p >= (1ull << 62)) return pm_fail(ctx, PM_EINVAL, "pm_basis needs an odd prime p < 2^62");
    if (m > 128 || n > 128) return pm_fail(ctx, PM_EUNSUPPORTED, "pm_basis supports m, n <= 128");
    if (!F || !shift || !P || !rdeg_out) return pm_fail(ctx, PM_EINVAL, "null buffer");
    if (d + 1 > (1 << PM_MAX_LOG2L)) return pm_fail(ctx, PM_EINVAL, "order too large for the transforms");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    const size_t sm = leaf_smem(m, n);
    if (sm > 200 * 1024) return pm_fail(ctx, PM_EUNSUPPORTED, "leaf workspace too large");

    PmbCtx C;
    C.ctx = ctx;
    C.m = m;
    C.n = n;
    C.T = ctx->opt_T;
    const int64_t Tl = d < C.T ? d : C.T;   // largest leaf order
    LeafArgs &A = C.base;
    memset(&A, 0, sizeof(A));
    A.p = p;
    uint64_t inv = 1;                       // p^-1 mod 2^64 by Newton iteration
    for (int i = 0; i < 7; i++) inv *= 2 - p * inv;
    A.pn = (uint64_t)0 - inv;
    A.one = (uint64_t)(((unsigned __int128)1 << 64) % p);
    A.r2 = (uint64_t)((unsigned __int128)A.one * A.one % p);
    A.m = m;
    A.n = n;
    uint64_t ch = ~0ull / p;
    A.chunk = (int)(ch > 16 ? 16 : ch);

    // arena: recursion buffers + leaf scratch + the two shift vectors
    const size_t leafG = (size_t)m * n * Tl * 8, leafP = (size_t)m * m * (Tl + 1) * 8;
    const size_t padF = lenF < d ? al256((size_t)m * n * d * 8) : 0;
    const size_t need = rec_bytes(m, n, d, C.T) + 2 * al256(leafG) + 2 * al256(leafP) + 2 * al256((size_t)m * 8) + padF;
    CKI(arena_reserve(ctx, need));
    A.G0 = (u64 *)arena_alloc(ctx, leafG);
    A.G1 = (u64 *)arena_alloc(ctx, leafG);
    A.P0 = (u64 *)arena_alloc(ctx, leafP);
    A.P1 = (u64 *)arena_alloc(ctx, leafP);
    i64 *s_in = (i64 *)arena_alloc(ctx, (size_t)m * 8);
    i64 *s_out = (i64 *)arena_alloc(ctx, (size_t)m * 8);
    if (!A.G0 || !A.G1 || !A.P0 || !A.P1 || !s_in || !s_out) return pm_fail(ctx, PM_ENOMEM, "arena too small");
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
