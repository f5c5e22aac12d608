// inverse.cu -- truncated inverse of a polynomial matrix (Sec. 4, "Linear
// system solving": the lifting solver first computes S = A^-1 mod x^t by
// matrix Newton iteration).
//
// Constant term: X_0 = A(0)^-1 by fraction-free Gauss-Jordan in one CTA
// (Montgomery arithmetic for odd p, bit arithmetic for p = 2), rows divided
// by their diagonal entries at the end, so one modular inversion per row.
// Newton step k -> kk = min(2k, t): since A.X_k = I mod x^k,
//   E = coefficients k .. kk-1 of A.X_k               (middle product)
//   X_kk = X_k - x^k (X_k . E mod x^(kk-k))           (truncated product)
// both through the product hot path (prod_slice), then one negation pass.
#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include "host.h"

struct InvArith {
    u64 p, pn, one, r2;     // Montgomery constants (odd p)
    int two;                // p = 2: plain bit arithmetic
};

__device__ __forceinline__ u64 ia_mul(const InvArith &F, u64 a, u64 b)
{
    return F.two ? (a & b) : mont_mul(a, b, F.p, F.pn);
}
__device__ __forceinline__ u64 ia_in(const InvArith &F, u64 a) { return F.two ? a : mont_mul(a, F.r2, F.p, F.pn); }
__device__ __forceinline__ u64 ia_out(const InvArith &F, u64 a) { return F.two ? a : mont_mul(a, 1, F.p, F.pn); }
__device__ u64 ia_inv(const InvArith &F, u64 a)         // a^(p-2), a != 0 (Fermat)
{
    if (F.two) return 1;
    u64 r = F.one, e = F.p - 2;
    while (e) {
        if (e & 1) r = mont_mul(r, a, F.p, F.pn);
        a = mont_mul(a, a, F.p, F.pn);
        e >>= 1;
    }
    return r;
}

// M: scratch n x 2n (row-major) in global memory.  On success X_0 goes to
// X[(i n + j) sX]; if A(0) is singular the status word gets PM_EDOMAIN.
__global__ void __launch_bounds__(1024) k_inv0(InvArith F, const void *A, int w, i64 sA, int n, u64 *M, void *X,
                                               i64 sX, int *status)
{
    __shared__ int piv;
    __shared__ u64 fcol[128];
    const int tid = threadIdx.x, nth = blockDim.x, n2 = 2 * n;
    for (int x = tid; x < n * n2; x += nth) {
        const int i = x / n2, j = x - i * n2;
        u64 v;
        if (j < n) {
            const i64 idx = ((i64)i * n + j) * sA;
            v = ia_in(F, w == 8 ? ((const u64 *)A)[idx] : ((const u32 *)A)[idx]);
        } else v = (j - n == i) ? F.one : 0;
        M[x] = v;
    }
    __syncthreads();
    for (int c = 0; c < n; c++) {
        if (tid == 0) piv = n;
        __syncthreads();
        for (int r = c + tid; r < n; r += nth)
            if (M[(i64)r * n2 + c]) atomicMin(&piv, r);
        __syncthreads();
        const int r = piv;
        if (r == n) {                                  // uniform: no pivot in column c
            if (tid == 0) atomicCAS(status, 0, PM_EDOMAIN);
            return;
        }
        if (r != c)
            for (int j = tid; j < n2; j += nth) {
                const u64 a = M[(i64)r * n2 + j];
                M[(i64)r * n2 + j] = M[(i64)c * n2 + j];
                M[(i64)c * n2 + j] = a;
            }
        __syncthreads();
        for (int i = tid; i < n; i += nth) fcol[i] = M[(i64)i * n2 + c];
        __syncthreads();
        const u64 pv = fcol[c];
        // rows i != c: row_i <- pv row_i - M[i][c] row_c (fraction-free)
        for (int x = tid; x < n * n2; x += nth) {
            const int i = x / n2, j = x - i * n2;
            if (i == c) continue;
            M[x] = sub64(ia_mul(F, pv, M[x]), ia_mul(F, fcol[i], M[(i64)c * n2 + j]), F.p);
        }
        __syncthreads();
    }
    // the left half is now diagonal: X_0 = diag(d)^-1 . right half
    for (int i = tid; i < n; i += nth) fcol[i] = ia_inv(F, M[(i64)i * n2 + i]);
    __syncthreads();
    for (int x = tid; x < n * n; x += nth) {
        const int i = x / n, j = x - i * n;
        const u64 v = ia_out(F, ia_mul(F, fcol[i], M[(i64)i * n2 + n + j]));
        const i64 o = (i64)x * sX;
        if (w == 8) ((u64 *)X)[o] = v;
        else ((u32 *)X)[o] = (u32)v;
    }
}

// X[e sX + off + j] <- -X[e sX + off + j] mod p for e < count, j < h.
__global__ void k_negate_slice(void *X, int w, i64 sX, i64 off, i64 h, i64 count, u64 p)
{
    const i64 total = count * h;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < total; x += (i64)gridDim.x * blockDim.x) {
        const i64 e = x / h, o = e * sX + off + (x - e * h);
        if (w == 8) {
            const u64 v = ((u64 *)X)[o];
            ((u64 *)X)[o] = v ? p - v : 0;
        } else {
            const u32 v = ((u32 *)X)[o];
            ((u32 *)X)[o] = v ? (u32)p - v : 0;
        }
    }
}

// E (count entries of length len) <- the identity: coefficient 0 of the diagonal entries is 1
__global__ void k_identity(void *E, int w, int n, i64 len)
{
    const i64 total = (i64)n * n * len;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < total; x += (i64)gridDim.x * blockDim.x) {
        const i64 e = x / len, t = x - e * len;
        const u64 v = (t == 0 && e / n == e % n) ? 1 : 0;
        if (w == 8) ((u64 *)E)[x] = v;
        else ((u32 *)E)[x] = (u32)v;
    }
}

#define CKI(call)                                                       \
    do {                                                                \
        int _rc = (call);                                               \
        if (_rc) return _rc;                                            \
    } while (0)

static int check_inverse_args(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA, int64_t t, void *X)
{
    if (w != 4 && w != 8) return pm_fail(ctx, PM_EINVAL, "w must be 4 or 8");
    if (p < 2 || (w == 4 && p >= (1ull << 32)) || (w == 8 && p >= (1ull << 62)))
        return pm_fail(ctx, PM_EINVAL, "need 2 <= p < 2^32 (w = 4) or 2^62 (w = 8)");
    if (n < 1 || dA < 1 || t < 1) return pm_fail(ctx, PM_EINVAL, "need n, dA, t >= 1");
    if (n > 128) return pm_fail(ctx, PM_EUNSUPPORTED, "n <= 128 is supported");
    if (t > (int64_t(1) << (PM_MAX_LOG2L - 1))) return pm_fail(ctx, PM_EINVAL, "length too large for the transforms");
    if (!A || !X) return pm_fail(ctx, PM_EINVAL, "null buffer");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    return PM_OK;
}

static InvArith inv_arith(uint64_t p)
{
    InvArith F;
    memset(&F, 0, sizeof(F));
    F.p = p;
    F.two = p == 2;
    if (!F.two) {
        uint64_t inv = 1;                   // p^-1 mod 2^64 by Newton iteration
        for (int i = 0; i < 7; i++) inv *= 2 - p * inv;
        F.pn = (uint64_t)0 - inv;
        F.one = (uint64_t)(((unsigned __int128)1 << 64) % p);
        F.r2 = (uint64_t)((unsigned __int128)F.one * F.one % p);
    } else {
        F.one = 1;
    }
    return F;
}

static void negate_slice(pm_ctx *ctx, void *X, int w, int64_t sX, int64_t off, int64_t h, int64_t count, uint64_t p)
{
    const int64_t tot = count * h;
    int grid = (int)((tot + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_negate_slice<<<grid, 256, 0, ctx->stream>>>(X, w, sX, off, h, count, p);
    ctx->launches++;
}

// X = A^-1 mod x^t with scratch M (n x 2n u64) and E (n x n x max(t/2, 1) words of width w).
static int inv_trunc_core(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA, int64_t t, void *X,
                          u64 *M, void *E)
{
    const InvArith F = inv_arith(p);
    const int64_t nn = (int64_t)n * n;
    k_inv0<<<1, 1024, 0, ctx->stream>>>(F, A, w, dA, n, M, X, t, ctx->d_status);
    ctx->launches++;
    CKI(pm_cuda(ctx, cudaGetLastError(), "k_inv0"));
    // every coefficient 1 .. t-1 of X is written by exactly one Newton step
    for (int64_t k = 1; k < t;) {
        const int64_t kk = 2 * k < t ? 2 * k : t, h = kk - k;
        const int64_t dAe = dA < kk ? dA : kk;
        // E = coefficients k .. kk-1 of A . X_k: product length <= kk + k - 1, cyclic length
        // L >= kk puts every aliased coefficient below k
        CKI(prod_slice(ctx, p, w, n, n, n, A, dAe, dA, X, k, t, k, h, ceil_log2(kk), E, h));
        // X[k .. kk) = X_k . E mod x^h (no aliasing), then negated
        const int64_t dX = k < h ? k : h;
        CKI(prod_slice(ctx, p, w, n, n, n, X, dX, t, E, h, h, 0, h, ceil_log2(dX + h - 1), (char *)X + k * w, t));
        negate_slice(ctx, X, w, t, k, h, nn, p);
        CKI(pm_cuda(ctx, cudaGetLastError(), "k_negate_slice"));
        k = kk;
    }
    return PM_OK;
}

static size_t inv_scratch_words(int n, int64_t t, int w, size_t *bE)
{
    const int64_t hmax = t / 2 > 0 ? t / 2 : 1;
    *bE = (size_t)n * n * (size_t)hmax * w;
    return (size_t)n * n * 2;
}

extern "C" int pmat_inv_trunc(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA, int64_t t, void *X)
{
    if (!ctx) return PM_EINVAL;
    CKI(check_inverse_args(ctx, p, w, n, A, dA, t, X));
    size_t bE;
    const size_t wM = inv_scratch_words(n, t, w, &bE);
    CKI(arena_reserve(ctx, wM * 8 + bE + 512));
    u64 *M = (u64 *)arena_alloc(ctx, wM * 8);
    void *E = arena_alloc(ctx, bE);
    if (!M || !E) return pm_fail(ctx, PM_ENOMEM, "arena too small");
    return inv_trunc_core(ctx, p, w, n, A, dA, t, X, M, E);
}

// Dixon's lifting (Sec. 4): with delta = max(dA, db) and S = A^-1 mod x^delta,
//   y_i = S r_i mod x^delta,  r_{i+1} = (r_i - A y_i) / x^delta = -(coefficients
//   delta .. 2 delta - 1 of A y_i)   (r_i has length delta and A y_i = r_i mod x^delta),
// from r_0 = b; v = sum_i y_i x^(i delta).  Both steps are products on the hot path.
extern "C" int pmat_solve_series(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA, const void *b,
                                 int64_t db, int64_t N, void *v)
{
    if (!ctx) return PM_EINVAL;
    CKI(check_inverse_args(ctx, p, w, n, A, dA, N, v));
    if (db < 1 || !b) return pm_fail(ctx, PM_EINVAL, "need db >= 1 and b");
    const int64_t delta = dA > db ? dA : db;
    if (2 * delta > (int64_t(1) << PM_MAX_LOG2L)) return pm_fail(ctx, PM_EINVAL, "degree too large for the transforms");
    size_t bE;
    const size_t wM = inv_scratch_words(n, delta, w, &bE);
    const size_t bS = (size_t)n * n * delta * w, bR = (size_t)n * delta * w;
    // S and A are the same in every full digit: their transforms are kept after the first
    const int lgS = ceil_log2(2 * delta - 1) < 4 ? 4 : ceil_log2(2 * delta - 1);
    const int lgA = ceil_log2(dA + delta - 1) < 4 ? 4 : ceil_log2(dA + delta - 1);
    const bool cache = N > 2 * delta;                 // at least two full digits reuse them
    const size_t bTS = cache ? prod_operand_bytes(ctx, p, n, delta, lgS, (int64_t)n * n) : 0;
    const size_t bTA = cache ? prod_operand_bytes(ctx, p, n, dA, lgA, (int64_t)n * n) : 0;
    CKI(arena_reserve(ctx, wM * 8 + bE + bS + bR + bTS + bTA + 6 * 256));
    u64 *M = (u64 *)arena_alloc(ctx, wM * 8);
    void *E = arena_alloc(ctx, bE);
    void *S = arena_alloc(ctx, bS);
    void *R = arena_alloc(ctx, bR);
    u32 *TS = bTS ? (u32 *)arena_alloc(ctx, bTS) : nullptr;
    u32 *TA = bTA ? (u32 *)arena_alloc(ctx, bTA) : nullptr;
    if (!M || !E || !S || !R || (bTS && !TS) || (bTA && !TA)) return pm_fail(ctx, PM_ENOMEM, "arena too small");
    CKI(inv_trunc_core(ctx, p, w, n, A, dA, delta, S, M, E));
    // r_0 = b, zero-padded to length delta
    CKI(pm_cuda(ctx, cudaMemsetAsync(R, 0, bR, ctx->stream), "residual"));
    CKI(pm_cuda(ctx, cudaMemcpy2DAsync(R, (size_t)delta * w, b, (size_t)db * w, (size_t)db * w, (size_t)n,
                                       cudaMemcpyDeviceToDevice, ctx->stream), "residual"));
    for (int64_t i = 0, off = 0; off < N; i++, off += delta) {
        const int64_t len = N - off < delta ? N - off : delta;
        char *y = (char *)v + off * w;
        // y_i = S r_i mod x^len (no aliasing)
        ProdReq q1;
        q1.p = p; q1.w = w; q1.m = n; q1.n = n; q1.k = 1;
        q1.lg = ceil_log2(2 * len - 1) < 4 ? 4 : ceil_log2(2 * len - 1);
        q1.A = S; q1.dA = len; q1.sA = delta; q1.B = R; q1.dB = len; q1.sB = delta;
        q1.off = 0; q1.len = len; q1.C = y; q1.sC = N;
        if (TS && len == delta) {                      // full digits: S's transforms kept after the first
            if (i == 0) q1.At_out = TS;
            else q1.At = TS;
        }
        CKI(prod_batch(ctx, &q1, 1));
        if (off + delta >= N) break;
        // r_{i+1} = -(coefficients delta .. 2 delta - 1 of A y_i) (no aliasing)
        ProdReq q2;
        q2.p = p; q2.w = w; q2.m = n; q2.n = n; q2.k = 1; q2.lg = lgA;
        q2.A = A; q2.dA = dA; q2.sA = dA; q2.B = y; q2.dB = delta; q2.sB = N;
        q2.off = delta; q2.len = delta; q2.C = R; q2.sC = delta;
        if (TA) {                                      // A's transforms, likewise
            if (i == 0) q2.At_out = TA;
            else q2.At = TA;
        }
        CKI(prod_batch(ctx, &q2, 1));
        negate_slice(ctx, R, w, delta, 0, delta, n, p);
        CKI(pm_cuda(ctx, cudaGetLastError(), "k_negate_slice"));
    }
    return PM_OK;
}

// High-order lifting (Sec. 4; Storjohann): the slices S_i = coefficients (2^i - 1) D ..
// (2^i + 1) D of X = A^-1, D = dA - 1, with the residues E_m = x^-m (I - A (X mod x^m)) =
// A (X div x^m) mod x^(D+1) (degree <= D).  From X = (X mod x^m) + x^m X E_m, with
// c = 2^i D:
//   lower half of S_{i+1} = coefficients D .. 2D-1 of S_i E_{c-D}
//   upper half of S_{i+1} = coefficients D .. 2D   of S_i E_c
//   E_{2c-D} = A . S_{i+1}[0 .. D] mod x^(D+1),  E_2c = A . S_{i+1}[D .. 2D] mod x^(D+1)
// from S_0 = A^-1 mod x^(2D+1) (Newton), E_0 = I and E_D = A . S_0[D .. 2D] mod x^(D+1):
// four products per slice, two by two in one batched call.
extern "C" int pmat_inv_slices(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA, int K, void *S)
{
    if (!ctx) return PM_EINVAL;
    if (dA < 2 || K < 1 || K > 24) return pm_fail(ctx, PM_EINVAL, "need dA >= 2 and 1 <= K <= 24");
    const int64_t D = dA - 1, W = 2 * D + 1;
    CKI(check_inverse_args(ctx, p, w, n, A, dA, W, S));
    if (3 * D + 1 > (int64_t(1) << PM_MAX_LOG2L)) return pm_fail(ctx, PM_EINVAL, "degree too large for the transforms");
    const size_t nn = (size_t)n * n;
    size_t bE;
    const size_t wM = inv_scratch_words(n, W, w, &bE);
    const size_t bR = nn * (size_t)(D + 1) * w;
    // cyclic lengths without aliasing: an output window [off, off + len) of a product of length P
    // needs L >= max(P - off, off + len).  E = A S_i[..] mod x^(D+1): P = 2D + 1, off = 0.
    // Halves of S_{i+1}: S_i (2D + 1) by E (D + 1), P = 3D + 1, off = D, len <= D + 1: L >= 2D + 1.
    const int lgE = ceil_log2(2 * D + 1) < 4 ? 4 : ceil_log2(2 * D + 1);
    const int lgS = lgE;
    // transforms kept across products: S_i's for its two products, A's for all of them
    const size_t bTS = K > 1 ? prod_operand_bytes(ctx, p, n, D + 1, lgS, (int64_t)nn) : 0;
    const size_t bTA = K > 1 ? prod_operand_bytes(ctx, p, n, dA, lgE, (int64_t)nn) : 0;
    CKI(arena_reserve(ctx, wM * 8 + bE + 2 * bR + bTS + bTA + 6 * 256));
    u64 *M = (u64 *)arena_alloc(ctx, wM * 8);
    void *E = arena_alloc(ctx, bE);
    char *Elo = (char *)arena_alloc(ctx, bR), *Ehi = (char *)arena_alloc(ctx, bR);
    u32 *TS = bTS ? (u32 *)arena_alloc(ctx, bTS) : nullptr;
    u32 *TA = bTA ? (u32 *)arena_alloc(ctx, bTA) : nullptr;
    if (!M || !E || !Elo || !Ehi || (bTS && !TS) || (bTA && !TA)) return pm_fail(ctx, PM_ENOMEM, "arena too small");
    char *S0 = (char *)S;
    const size_t slice = nn * (size_t)W * w;
    CKI(inv_trunc_core(ctx, p, w, n, A, dA, W, S0, M, E));
    if (K == 1) return PM_OK;
    {
        const int64_t tot = (int64_t)nn * (D + 1);
        int grid = (int)((tot + 255) / 256);
        if (grid > 4096) grid = 4096;
        k_identity<<<grid, 256, 0, ctx->stream>>>(Elo, w, n, D + 1);
        ctx->launches++;
        CKI(pm_cuda(ctx, cudaGetLastError(), "k_identity"));
    }
    auto req = [&](const void *Ap, int64_t da, int64_t sa, const void *Bp, int64_t db, int64_t sb, int64_t off,
                   int64_t len, int lg, void *Cp, int64_t sc) {
        ProdReq q;
        q.p = p; q.w = w; q.m = n; q.n = n; q.k = n; q.lg = lg < 4 ? 4 : lg;
        q.A = Ap; q.dA = da; q.sA = sa; q.B = Bp; q.dB = db; q.sB = sb;
        q.off = off; q.len = len; q.C = Cp; q.sC = sc;
        return q;
    };
    {
        ProdReq q = req(A, dA, dA, S0 + D * w, D + 1, W, 0, D + 1, lgE, Ehi, D + 1);   // E_D
        q.At_out = TA;                                   // A's transforms, for every later product
        CKI(prod_batch(ctx, &q, 1));
    }
    for (int i = 1; i < K; i++) {
        const char *Sp = S0 + (size_t)(i - 1) * slice;
        char *Sc = S0 + (size_t)i * slice;
        ProdReq q[2] = {req(Sp, W, W, Elo, D + 1, D + 1, D, D, lgS, Sc, W),                    // lower half
                        req(Sp, W, W, Ehi, D + 1, D + 1, D, D + 1, lgS, Sc + D * w, W)};       // upper half
        q[0].At_out = TS;                                // the forward stage of the call fills TS
        q[1].At = TS;                                    // before its pointwise stage reads it
        CKI(prod_batch(ctx, q, 2));
        if (i + 1 < K) {
            ProdReq r[2] = {req(A, dA, dA, Sc, D + 1, W, 0, D + 1, lgE, Elo, D + 1),
                            req(A, dA, dA, Sc + D * w, D + 1, W, 0, D + 1, lgE, Ehi, D + 1)};
            r[0].At = TA;
            r[1].At = TA;
            CKI(prod_batch(ctx, r, 2));
        }
    }
    return PM_OK;
}

// ------------------------------------------------------------------ high-order lifting solution
// A^-1 b mod x^N from the slices (Sec. 4, high-order lifting used for system solving).  With
// X = A^-1, D = dA - 1 and rho_m(w) = x^-m (w - A (X w mod x^m)), the residue of w at position m:
//   X w = (X w mod x^m) + x^m X rho_m(w),   rho_(m1 + m2) = rho_m2 o rho_m1,
// and for deg w <= D, rho_m(w) (degree < D) depends only on coefficients m - D .. m - 1 of X w:
//   rho_m(w) = -(coefficients D .. 2D - 1 of A U),   U = coefficients m - D .. m - 1 of X w.
// For m = K_i = (2^i + 1) D, U = coefficients D .. 2D - 1 of S_i w: slice S_i holds exactly the
// coefficients of X those need.  Residues of b are made in a binary tree: level i = k - 1 .. 0
// moves every residue made so far one jump K_i further, so after k levels there is one residue
// at position f(x) D for every x < 2^k, f(x) = x + popcount(x) (x's bits name its jumps).  Since
// f(x + 1) - f(x) <= 2, sorted positions are at most 2D apart, and each residue w at position P
// gives v's coefficients P .. P + 2D as S_0 w mod x^(2D + 1).  Every level is two products over
// all of its residues at once, one matrix product by S_i and one by A, where Dixon's lifting
// takes ceil(N / delta) matrix-vector steps one after the other.
//
// Storage: the residues are the columns of an n x 2^k matrix W (entries of length D + 1), column
// j holding x = the k-bit reversal of j; level i then reads columns [0, c) and writes [c, 2c),
// c = 2^(k-1-i), both contiguous column blocks.
namespace {

#define HOL_MAXR 256

struct HolTable {
    int cnt;                  // distinct residue positions, ascending
    int col[HOL_MAXR];        // residue column at each
    i64 pos[HOL_MAXR];
};

// v[r][t] = Y[r][j][t - pos_j], j the residue with the largest position <= t.
__global__ void k_hol_assemble(void *v, int w, int n, i64 N, const void *Y, int R, i64 Ws,
                               const __grid_constant__ HolTable T)
{
    const i64 total = (i64)n * N;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < total; x += (i64)gridDim.x * blockDim.x) {
        const i64 r = x / N, t = x - r * N;
        int lo = 0, hi = T.cnt - 1;                   // last entry with pos <= t (pos[0] = 0)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (T.pos[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const i64 src = ((r * R + T.col[lo]) * Ws) + (t - T.pos[lo]);
        if (w == 8) ((u64 *)v)[x] = ((const u64 *)Y)[src];
        else ((u32 *)v)[x] = ((const u32 *)Y)[src];
    }
}

int bitrev(int x, int k)
{
    int r = 0;
    for (int i = 0; i < k; i++) r |= ((x >> i) & 1) << (k - 1 - i);
    return r;
}

}  // namespace

extern "C" int pmat_solve_series_hol(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA,
                                     const void *b, int64_t db, int64_t N, void *v)
{
    if (!ctx) return PM_EINVAL;
    CKI(check_inverse_args(ctx, p, w, n, A, dA, N, v));
    if (db < 1 || !b) return pm_fail(ctx, PM_EINVAL, "need db >= 1 and b");
    if (dA < 2 || db > dA) return pm_fail(ctx, PM_EINVAL, "high-order lifting needs dA >= 2 and db <= dA");
    const int64_t D = dA - 1, Ws = 2 * D + 1, Lw = D + 1;
    if (3 * D + 1 > (int64_t(1) << PM_MAX_LOG2L)) return pm_fail(ctx, PM_EINVAL, "degree too large for the transforms");
    int k = 0;
    while (((int64_t(1) << k) + k + 1) * D + 1 < N) k++;
    if ((1 << k) > HOL_MAXR) return pm_fail(ctx, PM_EINVAL, "N needs more than 256 residues at this degree");
    const int R = 1 << k, K = k > 0 ? k : 1, half = R > 1 ? R / 2 : 1;

    // residue positions: sorted, distinct, gaps <= 2D, the last within 2D of N - 1
    HolTable T;
    {
        std::vector<std::pair<int64_t, int>> ps;
        for (int j = 0; j < R; j++) {
            const int x = bitrev(j, k);
            ps.push_back({(int64_t)(x + __builtin_popcount((unsigned)x)) * D, j});
        }
        std::sort(ps.begin(), ps.end());
        T.cnt = 0;
        for (auto &e : ps)
            if (T.cnt == 0 || T.pos[T.cnt - 1] != e.first) { T.pos[T.cnt] = e.first; T.col[T.cnt] = e.second; T.cnt++; }
        for (int i = 1; i < T.cnt; i++)
            if (T.pos[i] - T.pos[i - 1] > 2 * D) return pm_fail(ctx, PM_EINVAL, "internal: residue gap");
        if (N - 1 - T.pos[T.cnt - 1] > 2 * D) return pm_fail(ctx, PM_EINVAL, "internal: residue coverage");
    }

    const size_t nn = (size_t)n * n;
    const size_t bS = (size_t)K * nn * Ws * w, bW = (size_t)n * R * Lw * w, bY = (size_t)n * R * Ws * w;
    const size_t bT1 = (size_t)n * half * Lw * w, bU = (size_t)n * half * D * w;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t total = al(bS) + al(bW) + al(bY) + 2 * al(bT1) + al(bU);
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, total, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return pm_fail(ctx, PM_ENOMEM, "pmat_solve_series_hol workspace allocation failed");
    }
    char *S = buf, *Wm = S + al(bS), *Y = Wm + al(bW), *T1 = Y + al(bY), *T2 = T1 + al(bT1), *U = T2 + al(bT1);
    int rc = PM_OK;
    auto req = [&](const void *Ap, int64_t da, int64_t sa, const void *Bp, int64_t dbb, int64_t sb, int kk,
                   int64_t off, int64_t len, int lg, void *Cp, int64_t sc) {
        ProdReq q;
        q.p = p; q.w = w; q.m = n; q.n = n; q.k = kk; q.lg = lg < 4 ? 4 : lg;
        q.A = Ap; q.dA = da; q.sA = sa; q.B = Bp; q.dB = dbb; q.sB = sb;
        q.off = off; q.len = len; q.C = Cp; q.sC = sc;
        return q;
    };
    do {
        // slices S_0 .. S_(K-1)
        if ((rc = pmat_inv_slices(ctx, p, w, n, A, dA, K, S))) break;
        // W = [b, 0, ...]
        if ((rc = pm_cuda(ctx, cudaMemsetAsync(Wm, 0, bW, ctx->stream), "residues"))) break;
        if ((rc = pm_cuda(ctx, cudaMemcpy2DAsync(Wm, (size_t)R * Lw * w, b, (size_t)db * w, (size_t)db * w, (size_t)n,
                                                 cudaMemcpyDeviceToDevice, ctx->stream), "residues")))
            break;
        // cyclic lengths without aliasing (an output window [off, off + len) of a product of
        // length P needs L >= max(P - off, off + len)): S_i (2D + 1) by W (D + 1), window
        // [D, 2D): 2D + 1; A (D + 1) by U (D), window [D, 2D): 2D; S_0 by W mod x^(2D + 1): 3D + 1
        const int lgU = ceil_log2(2 * D + 1), lgR = ceil_log2(2 * D), lgY = ceil_log2(3 * D + 1);
        for (int i = k - 1; i >= 0 && !rc; i--) {
            const int c = 1 << (k - 1 - i);
            const char *Si = S + (size_t)i * nn * Ws * w;
            // the level's residues as an n x c block, then U = coefficients D .. 2D-1 of S_i . block
            if ((rc = pm_cuda(ctx, cudaMemcpy2DAsync(T1, (size_t)c * Lw * w, Wm, (size_t)R * Lw * w, (size_t)c * Lw * w,
                                                     (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream), "gather")))
                break;
            ProdReq q1 = req(Si, Ws, Ws, T1, Lw, Lw, c, D, D, lgU, U, D);
            if ((rc = prod_batch(ctx, &q1, 1))) break;
            // new residues -(coefficients D .. 2D-1 of A . U), degree < D (coefficient D stays 0)
            if ((rc = pm_cuda(ctx, cudaMemsetAsync(T2, 0, (size_t)n * c * Lw * w, ctx->stream), "residues"))) break;
            ProdReq q2 = req(A, dA, dA, U, D, D, c, D, D, lgR, T2, Lw);
            if ((rc = prod_batch(ctx, &q2, 1))) break;
            negate_slice(ctx, T2, w, Lw, 0, D, (int64_t)n * c, p);
            if ((rc = pm_cuda(ctx, cudaGetLastError(), "k_negate_slice"))) break;
            if ((rc = pm_cuda(ctx, cudaMemcpy2DAsync(Wm + (size_t)c * Lw * w, (size_t)R * Lw * w, T2,
                                                     (size_t)c * Lw * w, (size_t)c * Lw * w, (size_t)n,
                                                     cudaMemcpyDeviceToDevice, ctx->stream), "scatter")))
                break;
        }
        if (rc) break;
        // v's coefficients from every residue: Y = S_0 . W mod x^(2D + 1), then assembled
        ProdReq qy = req(S, Ws, Ws, Wm, Lw, Lw, R, 0, Ws, lgY, Y, Ws);
        if ((rc = prod_batch(ctx, &qy, 1))) break;
        const int64_t tot = (int64_t)n * N;
        int grid = (int)((tot + 255) / 256);
        if (grid > 152 * 16) grid = 152 * 16;
        k_hol_assemble<<<grid, 256, 0, ctx->stream>>>(v, w, n, N, Y, R, Ws, T);
        ctx->launches++;
        rc = pm_cuda(ctx, cudaGetLastError(), "k_hol_assemble");
    } while (0);
    cudaFreeAsync(buf, ctx->stream);
    return rc;
}
