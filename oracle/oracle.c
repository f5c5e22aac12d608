/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for polynomial-matrix
 * arithmetic over F_p (Hyun, Neiger, Schost, ISSAC 2019, arXiv 1905.04356).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the golden-value script and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Every value is a uint64_t residue in [0, p), with 2 <= p < 2^63.  All
 * arithmetic is exact: products are accumulated in unsigned __int128 and
 * reduced with the compiler's 128-bit remainder.  There is no blocking, no
 * transform and no reordering beyond what each definition states.
 *
 * Layout: a polynomial matrix X with r x c entries of length len is stored
 * entry-major, row-major: coefficient t of entry (i,j) is X[(i*c + j)*len + t].
 *
 * What each function follows:
 *   orc_pmat_slice   Sec. 2 "Polynomial matrix multiplication" and
 *                    "Polynomial multiplication": the product A.B, its
 *                    truncation mod x^t, and MiddleProduct(F,G,c,d) = the
 *                    coefficients of degrees c..c+d-1 of FG, all read as
 *                    slices of the plain convolution sum.
 *   orc_mbasis1      Algorithm 1 (M-Basis-1): the s-Popov approximant basis
 *                    at order 1, by Gaussian elimination over rows taken in
 *                    increasing (shift, index) order.
 *   orc_mbasis       Algorithm 2 (M-Basis): residual = coefficient k of P.F,
 *                    Q = M-Basis-1(residual, t), P <- Q.P, t <- rdeg_s(P).
 *   orc_pmbasis      Algorithm 3 (PM-Basis): divide and conquer with the
 *                    threshold T, the first half of order ceil(d/2), and the
 *                    residual as a middle product.
 *   orc_mintbasis    Algorithm 4 (M-IntBasis): R = P(alpha_k) E_k, Q =
 *                    M-Basis-1(R, t) with x read as x - alpha_k, P <- Q.P,
 *                    t <- rdeg_s(P) (Sec. 3, "Interpolant bases").
 *   orc_pmat_eval    value of every entry of a polynomial matrix at a point
 *                    (Horner), to check P(alpha_l) E_l = 0.
 *   orc_pmintbasis   Algorithm 5 (PM-IntBasis): divide and conquer with the
 *                    threshold T, the residual being P1 evaluated at the second
 *                    half of the points times the second half of E.
 *   orc_bivariate_resultant_villard
 *                    Sec. 5.2, the variant of Algorithm 6: values of the
 *                    top-right block H of the inverse Sylvester matrix, an
 *                    interpolant basis of [H; -I] giving H = Q^-1 R, det Q
 *                    normalised by one direct value of the resultant.
 *   orc_univ_resultant / orc_bivariate_resultant
 *                    Sec. 5.2, the "Direct" method: evaluate in x, take
 *                    univariate resultants in y by the Euclidean algorithm,
 *                    interpolate (Newton divided differences).
 *   orc_matinv / orc_inv_trunc
 *                    Sec. 4, "Linear system solving": the truncated inverse
 *                    S = A^-1 mod x^t of a polynomial matrix with A(0)
 *                    invertible, taken by its definition -- the power series
 *                    X with A.X = I mod x^t, coefficient by coefficient:
 *                    X_0 = A_0^-1, X_j = -A_0^-1 (A_1 X_{j-1} + ... + A_j X_0).
 *   orc_inv_slices   Sec. 4, high-order lifting: the slices S_i of A^-1,
 *                    coefficients (2^i - 1)(d - 1) .. (2^i + 1)(d - 1) of the
 *                    truncated inverse above (d = the length of A).
 *   orc_scale        multiplication of a coefficient array by a constant (the
 *                    normalisation of the lifting solver's output, Sec. 4).
 *   orc_solve_series Sec. 4, lifting: the power-series solution
 *                    v = A^-1 b mod x^N that Dixon's algorithm produces, by
 *                    its definition A.v = b mod x^N: v_0 = A_0^-1 b_0,
 *                    v_j = A_0^-1 (b_j - A_1 v_{j-1} - ... - A_j v_0).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;
typedef uint64_t u64;
typedef int64_t i64;

/* ------------------------------------------------------------------ */
/* Field arithmetic in F_p                                              */
/* ------------------------------------------------------------------ */

static inline u64 f_add(u64 a, u64 b, u64 p) { u64 s = a + b; return s >= p ? s - p : s; }
static inline u64 f_sub(u64 a, u64 b, u64 p) { return a >= b ? a - b : a + (p - b); }
static inline u64 f_mul(u64 a, u64 b, u64 p) { return (u64)(((u128)a * b) % p); }
static inline u64 f_neg(u64 a, u64 p) { return a ? p - a : 0; }

u64 orc_powmod(u64 a, u64 e, u64 p)
{
    u64 r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = f_mul(r, a, p);
        a = f_mul(a, a, p);
        e >>= 1;
    }
    return r;
}

/* Inverse by the extended Euclidean algorithm on integers; 0 if a = 0. */
u64 orc_invmod(u64 a, u64 p)
{
    i128 r0 = (i128)p, r1 = (i128)(a % p), s0 = 0, s1 = 1;
    if (r1 == 0) return 0;
    while (r1 != 0) {
        i128 q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    /* r0 = gcd = 1 for prime p; s0 * a = 1 mod p */
    i128 v = s0 % (i128)p;
    if (v < 0) v += (i128)p;
    return (u64)v;
}

/* Accumulator for sums of products < 2^126: reduced whenever it reaches 2^126. */
static inline void acc_add(u128 *acc, u64 a, u64 b, u64 p)
{
    *acc += (u128)a * b;
    if (*acc >> 126) *acc %= p;
}

/* ------------------------------------------------------------------ */
/* Products: C (m x k, len) = coefficients c0 .. c0+len-1 of A.B        */
/* A is m x n with entries of length dA; B is n x k with length dB.     */
/* Coefficient t of entry (i,kk) is sum_l sum_{a+b=t} A_il[a] B_lk[b].  */
/* pmat_mul is the slice [0, dA+dB-1); pmat_mul_trunc(t) is [0, t);     */
/* MiddleProduct(A,B,c,d) is [c, c+d).                                   */
/* ------------------------------------------------------------------ */

u64 orc_pmat_coeff(u64 p, int m, int n, int k, const u64 *A, i64 dA, const u64 *B, i64 dB,
                   int i, int kk, i64 t)
{
    (void)m;
    u128 acc = 0;
    if (t < 0 || t > dA + dB - 2) return 0;
    i64 a_lo = t - (dB - 1) > 0 ? t - (dB - 1) : 0;
    i64 a_hi = t < dA - 1 ? t : dA - 1;
    for (int l = 0; l < n; l++) {
        const u64 *Ail = A + ((i64)i * n + l) * dA;
        const u64 *Blk = B + ((i64)l * k + kk) * dB;
        for (i64 a = a_lo; a <= a_hi; a++) acc_add(&acc, Ail[a], Blk[t - a], p);
    }
    return (u64)(acc % p);
}

void orc_pmat_slice(u64 p, int m, int n, int k, const u64 *A, i64 dA, const u64 *B, i64 dB,
                    i64 c0, i64 len, u64 *C)
{
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int i = 0; i < m; i++)
        for (int kk = 0; kk < k; kk++) {
            u64 *out = C + ((i64)i * k + kk) * len;
            for (i64 t = 0; t < len; t++)
                out[t] = orc_pmat_coeff(p, m, n, k, A, dA, B, dB, i, kk, c0 + t);
        }
}

void orc_pmat_mul(u64 p, int m, int n, int k, const u64 *A, i64 dA, const u64 *B, i64 dB, u64 *C)
{
    orc_pmat_slice(p, m, n, k, A, dA, B, dB, 0, dA + dB - 1, C);
}

void orc_pmat_mul_trunc(u64 p, int m, int n, int k, const u64 *A, i64 dA, const u64 *B, i64 dB,
                        i64 t, u64 *C)
{
    orc_pmat_slice(p, m, n, k, A, dA, B, dB, 0, t, C);
}

void orc_pmat_middle_product(u64 p, int m, int n, int k, const u64 *A, i64 dA, const u64 *B,
                             i64 dB, i64 c, i64 d, u64 *C)
{
    orc_pmat_slice(p, m, n, k, A, dA, B, dB, c, d, C);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1, M-Basis-1(R, t): R in F_p^{m x n}, shift t in Z^m.      */
/* Output Q (m x m, degree <= 1) as Q[(i*m + j)*2 + e], e = 0 constant,  */
/* e = 1 coefficient of x.  Returns the rank of R.                       */
/*                                                                     */
/* Rows are visited in increasing (t_i, i) order (the s-pivot is the     */
/* rightmost entry reaching the s-degree, so among equal shifts a later  */
/* index is the pivot of a kernel row).  A row that is independent of    */
/* the rows before it becomes x.e_i; a dependent row j becomes           */
/* e_j - sum c_ji e_i, its unique expression over the earlier            */
/* independent rows.  This is the t-Popov basis of the order-1 module,   */
/* which is unique.                                                      */
/* ------------------------------------------------------------------ */

int orc_mbasis1(u64 p, int m, int n, const u64 *R, const i64 *t, u64 *Q)
{
    int *order = (int *)malloc(sizeof(int) * m);
    int *piv = (int *)malloc(sizeof(int) * m);
    u64 *bv = (u64 *)calloc((size_t)m * n, sizeof(u64));  /* echelon rows, pivot 1 */
    u64 *bc = (u64 *)calloc((size_t)m * m, sizeof(u64));  /* bv[b] = sum_i bc[b][i] R_i */
    u64 *v = (u64 *)malloc(sizeof(u64) * n);
    u64 *tv = (u64 *)malloc(sizeof(u64) * m);
    int rank = 0;

    /* stable insertion sort of row indices by shift */
    for (int i = 0; i < m; i++) {
        int j = i;
        while (j > 0 && t[order[j - 1]] > t[i]) { order[j] = order[j - 1]; j--; }
        order[j] = i;
    }
    memset(Q, 0, sizeof(u64) * (size_t)m * m * 2);

    for (int oi = 0; oi < m; oi++) {
        int r = order[oi];
        for (int c = 0; c < n; c++) v[c] = R[(i64)r * n + c];
        memset(tv, 0, sizeof(u64) * m);
        tv[r] = 1;
        for (int b = 0; b < rank; b++) {
            u64 f = v[piv[b]];
            if (!f) continue;
            for (int c = 0; c < n; c++) v[c] = f_sub(v[c], f_mul(f, bv[(i64)b * n + c], p), p);
            for (int c = 0; c < m; c++) tv[c] = f_sub(tv[c], f_mul(f, bc[(i64)b * m + c], p), p);
        }
        int pc = -1;
        for (int c = 0; c < n; c++) if (v[c]) { pc = c; break; }
        if (pc >= 0) {
            u64 inv = orc_invmod(v[pc], p);
            for (int c = 0; c < n; c++) bv[(i64)rank * n + c] = f_mul(v[c], inv, p);
            for (int c = 0; c < m; c++) bc[(i64)rank * m + c] = f_mul(tv[c], inv, p);
            piv[rank++] = pc;
            Q[((i64)r * m + r) * 2 + 1] = 1;            /* x . e_r */
        } else {
            for (int c = 0; c < m; c++) Q[((i64)r * m + c) * 2 + 0] = tv[c];
        }
    }
    free(order); free(piv); free(bv); free(bc); free(v); free(tv);
    return rank;
}

/* rdeg_s(P)_i = max_j (deg P_ij + s_j) over the nonzero entries of row i
 * (Sec. 3, definition of the s-degree); a zero row gets INT64_MIN. */
void orc_rdeg(int m, int c, const u64 *P, i64 len, const i64 *s, i64 *out)
{
    for (int i = 0; i < m; i++) {
        i64 best = INT64_MIN;
        for (int j = 0; j < c; j++) {
            const u64 *e = P + ((i64)i * c + j) * len;
            i64 dg = -1;
            for (i64 a = len - 1; a >= 0; a--) if (e[a]) { dg = a; break; }
            if (dg >= 0 && dg + s[j] > best) best = dg + s[j];
        }
        out[i] = best;
    }
}

/* ------------------------------------------------------------------ */
/* Algorithm 2, M-Basis(F, d, s).  F is m x n with entries of length     */
/* lenF (coefficients beyond lenF are zero).  Output P (m x m, length    */
/* d+1) and rdeg_s(P).                                                   */
/* ------------------------------------------------------------------ */

void orc_mbasis(u64 p, int m, int n, const u64 *F, i64 lenF, i64 d, const i64 *s,
                u64 *P, i64 *rdeg)
{
    const i64 len = d + 1;
    u64 *R = (u64 *)malloc(sizeof(u64) * (size_t)m * n);
    u64 *Q = (u64 *)malloc(sizeof(u64) * (size_t)m * m * 2);
    u64 *Pn = (u64 *)calloc((size_t)m * m * len, sizeof(u64));
    i64 *t = (i64 *)malloc(sizeof(i64) * m);
    i64 degP = 0; /* every entry of P has degree <= degP */

    memset(P, 0, sizeof(u64) * (size_t)m * m * len);
    for (int i = 0; i < m; i++) P[((i64)i * m + i) * len] = 1;
    for (int i = 0; i < m; i++) t[i] = s[i];

    for (i64 k = 0; k < d; k++) {
        /* a. residual R = coefficient of degree k of P.F */
#pragma omp parallel for collapse(2) schedule(static)
        for (int i = 0; i < m; i++)
            for (int j = 0; j < n; j++) {
                u128 acc = 0;
                for (int l = 0; l < m; l++) {
                    const u64 *Pil = P + ((i64)i * m + l) * len;
                    const u64 *Flj = F + ((i64)l * n + j) * lenF;
                    i64 amax = degP < k ? degP : k;
                    for (i64 a = 0; a <= amax; a++) {
                        i64 b = k - a;
                        if (b < lenF) acc_add(&acc, Pil[a], Flj[b], p);
                    }
                }
                R[(i64)i * n + j] = (u64)(acc % p);
            }
        /* b. Q = M-Basis-1(R, t) */
        orc_mbasis1(p, m, n, R, t, Q);
        /* c. P <- Q.P (Q has degree <= 1) */
        i64 degN = degP + 1 < d ? degP + 1 : d;
#pragma omp parallel for collapse(2) schedule(static)
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) {
                u64 *out = Pn + ((i64)i * m + j) * len;
                for (i64 a = 0; a <= degN; a++) {
                    u128 acc = 0;
                    for (int l = 0; l < m; l++) {
                        u64 q0 = Q[((i64)i * m + l) * 2 + 0], q1 = Q[((i64)i * m + l) * 2 + 1];
                        const u64 *Plj = P + ((i64)l * m + j) * len;
                        if (q0 && a <= degP) acc_add(&acc, q0, Plj[a], p);
                        if (q1 && a >= 1 && a - 1 <= degP) acc_add(&acc, q1, Plj[a - 1], p);
                    }
                    out[a] = (u64)(acc % p);
                }
            }
        degP = degN;
        memcpy(P, Pn, sizeof(u64) * (size_t)m * m * len);
        /* ... and t <- rdeg_s(P) */
        orc_rdeg(m, m, P, len, s, t);
    }
    for (int i = 0; i < m; i++) rdeg[i] = t[i];
    free(R); free(Q); free(Pn); free(t);
}

/* ------------------------------------------------------------------ */
/* Algorithm 3, PM-Basis(F, d, s) with threshold T (M-Basis if d <= T). */
/* ------------------------------------------------------------------ */

void orc_pmbasis(u64 p, int m, int n, const u64 *F, i64 lenF, i64 d, const i64 *s, i64 T,
                 u64 *P, i64 *rdeg)
{
    if (d <= T) { orc_mbasis(p, m, n, F, lenF, d, s, P, rdeg); return; }
    const i64 d1 = (d + 1) / 2, d2 = d / 2;
    /* F mod x^d as a dense m x n matrix of length d */
    u64 *Fd = (u64 *)calloc((size_t)m * n * d, sizeof(u64));
    for (i64 e = 0; e < (i64)m * n; e++)
        for (i64 a = 0; a < d && a < lenF; a++) Fd[e * d + a] = F[e * lenF + a];
    /* step 2: P1 = PM-Basis(F mod x^d1, d1, s) */
    u64 *P1 = (u64 *)malloc(sizeof(u64) * (size_t)m * m * (d1 + 1));
    i64 *t1 = (i64 *)malloc(sizeof(i64) * m);
    orc_pmbasis(p, m, n, Fd, d, d1, s, T, P1, t1);
    /* step 3: R = MiddleProduct(P1, F, d1, d2): coefficients d1..d-1 of P1.F */
    u64 *Rm = (u64 *)malloc(sizeof(u64) * (size_t)m * n * (d2 > 0 ? d2 : 1));
    orc_pmat_middle_product(p, m, m, n, P1, d1 + 1, Fd, d, d1, d2, Rm);
    /* step 4: t = rdeg_s(P1) (returned above); step 5: P2 = PM-Basis(R, d2, t) */
    u64 *P2 = (u64 *)malloc(sizeof(u64) * (size_t)m * m * (d2 + 1));
    i64 *t2 = (i64 *)malloc(sizeof(i64) * m);
    orc_pmbasis(p, m, n, Rm, d2, d2, t1, T, P2, t2);
    /* step 6: P = P2.P1, degree <= d */
    orc_pmat_slice(p, m, m, m, P2, d2 + 1, P1, d1 + 1, 0, d + 1, P);
    orc_rdeg(m, m, P, d + 1, s, rdeg);
    free(Fd); free(P1); free(t1); free(Rm); free(P2); free(t2);
}

/* ------------------------------------------------------------------ */
/* Resultants                                                           */
/* ------------------------------------------------------------------ */

static i64 poly_deg(const u64 *a, i64 len)
{
    for (i64 i = len - 1; i >= 0; i--) if (a[i]) return i;
    return -1;
}

/* Res(A, B) for A of degree a and B of degree b (actual degrees, both >= 0)
 * by the Euclidean algorithm: with R = A mod B of degree r,
 *   Res(A, B) = (-1)^(a b) lc(B)^(a - r) Res(B, R),
 * Res(A, c) = c^a for a nonzero constant c, and Res = 0 when a remainder
 * vanishes before a constant is reached.  Res(A,B) = lc(A)^b lc(B)^a
 * prod (alpha_i - beta_j) over the roots. */
u64 orc_univ_resultant(u64 p, const u64 *A0, i64 a, const u64 *B0, i64 b)
{
    u64 *A = (u64 *)malloc(sizeof(u64) * (a + 1));
    u64 *B = (u64 *)malloc(sizeof(u64) * (b + 1));
    memcpy(A, A0, sizeof(u64) * (a + 1));
    memcpy(B, B0, sizeof(u64) * (b + 1));
    u64 acc = 1 % p;
    for (;;) {
        if (b == 0) { acc = f_mul(acc, orc_powmod(B[0], (u64)a, p), p); break; }
        if (a == 0) { acc = f_mul(acc, orc_powmod(A[0], (u64)b, p), p); break; }
        /* A <- A mod B, by long division from the top coefficient down */
        u64 ilc = orc_invmod(B[b], p);
        for (i64 da = a; da >= b; da--) {
            u64 f = f_mul(A[da], ilc, p);
            if (!f) continue;
            for (i64 i = 0; i <= b; i++)
                A[da - b + i] = f_sub(A[da - b + i], f_mul(f, B[i], p), p);
        }
        i64 r = poly_deg(A, a < b ? a + 1 : b);
        if (r < 0) { acc = 0; break; }
        if ((a & 1) && (b & 1)) acc = f_neg(acc, p);
        acc = f_mul(acc, orc_powmod(B[b], (u64)(a - r), p), p);
        /* (A, B) <- (B, R) */
        u64 *tmp = A; A = B; B = tmp;
        a = b; b = r;
    }
    free(A); free(B);
    return acc;
}

/* Res_y(f, g) in F_p[x] with formal y-degrees dyf, dyg.
 * f[j*(dxf+1) + i] = coefficient of x^i y^j (likewise g).
 * R receives D+1 coefficients, D = dxf*dyg + dxg*dyf (the degree bound).
 * Points x = 0, 1, 2, ... where lc_y(f)(x) lc_y(g)(x) = 0 are skipped, so at
 * the points used the univariate degrees equal the formal ones and the
 * resultant specialises.  Returns 0 on success, -1 if p has too few points. */
/* R (N coefficients) interpolating the values vs (overwritten) at the increasing
 * non-negative integer points xs, by Newton divided differences. */
static void interp_int_points(u64 p, const u64 *xs, u64 *vs, i64 N, u64 *R)
{
    /* Newton divided differences; x_i - x_{i-j} is a positive integer at most
     * xs[N-1], so a table of inverses of 1..xs[N-1] serves every level.
     * Level j: c_i <- (c_i - c_{i-1}) / (x_i - x_{i-j}) for i >= j. */
    u64 xmax = xs[N - 1];
    u64 *inv = (u64 *)malloc(sizeof(u64) * (xmax + 2));
    u64 *c = vs, *c2 = (u64 *)malloc(sizeof(u64) * N);
    inv[0] = 0;
#pragma omp parallel for schedule(static)
    for (i64 e = 1; e <= (i64)xmax; e++) inv[e] = orc_invmod((u64)e, p);
    for (i64 j = 1; j < N; j++) {
#pragma omp parallel for schedule(static) if (N - j > 4096)
        for (i64 i = j; i < N; i++)
            c2[i] = f_mul(f_sub(c[i], c[i - 1], p), inv[xs[i] - xs[i - j]], p);
        memcpy(c + j, c2 + j, sizeof(u64) * (N - j));
    }
    /* Newton form -> monomial form, from the innermost factor out:
     * R <- R.(x - x_i) + c_i for i = N-2 .. 0, starting from R = c_{N-1}. */
    u64 *Rn = c2;
    memset(R, 0, sizeof(u64) * N);
    R[0] = c[N - 1];
    for (i64 i = N - 2, deg = 0; i >= 0; i--, deg++) {
        u64 xi = xs[i];
        Rn[deg + 1] = R[deg];
#pragma omp parallel for schedule(static) if (deg > 4096)
        for (i64 e = 1; e <= deg; e++) Rn[e] = f_sub(R[e - 1], f_mul(xi, R[e], p), p);
        Rn[0] = f_sub(c[i], f_mul(xi, R[0], p), p);
        memcpy(R, Rn, sizeof(u64) * (deg + 2));
    }
    free(c2);
    free(inv);
}

int orc_bivariate_resultant(u64 p, int dxf, int dyf, const u64 *f, int dxg, int dyg,
                            const u64 *g, u64 *R)
{
    const i64 D = (i64)dxf * dyg + (i64)dxg * dyf;
    const i64 N = D + 1;
    u64 *xs = (u64 *)malloc(sizeof(u64) * N);
    u64 *vs = (u64 *)malloc(sizeof(u64) * N);
    /* choose the points */
    i64 cnt = 0;
    for (u64 x = 0; cnt < N; x++) {
        if (x >= p) { free(xs); free(vs); return -1; }
        u64 lf = 0, lg = 0;
        for (int i = dxf; i >= 0; i--) lf = f_add(f_mul(lf, x, p), f[(i64)dyf * (dxf + 1) + i], p);
        for (int i = dxg; i >= 0; i--) lg = f_add(f_mul(lg, x, p), g[(i64)dyg * (dxg + 1) + i], p);
        if (lf && lg) xs[cnt++] = x;
    }
    /* values: univariate resultants of the specialisations */
#pragma omp parallel
    {
        u64 *fa = (u64 *)malloc(sizeof(u64) * (dyf + 1));
        u64 *ga = (u64 *)malloc(sizeof(u64) * (dyg + 1));
#pragma omp for schedule(dynamic, 16)
        for (i64 t = 0; t < N; t++) {
            u64 x = xs[t];
            for (int j = 0; j <= dyf; j++) {
                u64 v = 0;
                for (int i = dxf; i >= 0; i--) v = f_add(f_mul(v, x, p), f[(i64)j * (dxf + 1) + i], p);
                fa[j] = v;
            }
            for (int j = 0; j <= dyg; j++) {
                u64 v = 0;
                for (int i = dxg; i >= 0; i--) v = f_add(f_mul(v, x, p), g[(i64)j * (dxg + 1) + i], p);
                ga[j] = v;
            }
            vs[t] = orc_univ_resultant(p, fa, dyf, ga, dyg);
        }
        free(fa); free(ga);
    }
    interp_int_points(p, xs, vs, N, R);
    free(xs); free(vs);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Truncated inverse (Sec. 4, linear system solving by lifting)         */
/* ------------------------------------------------------------------ */

/* Inverse of the n x n constant matrix M (row-major) by Gauss-Jordan
 * elimination over F_p (p prime) on [M | I]: pivot = the first row at or
 * below the current one with a nonzero entry in the column.  Returns 0 and
 * writes Minv, or 1 if M is singular. */
int orc_matinv(u64 p, int n, const u64 *M, u64 *Minv)
{
    int w = 2 * n;
    u64 *T = (u64 *)malloc(sizeof(u64) * (size_t)n * w);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < w; j++)
            T[(size_t)i * w + j] = j < n ? M[(size_t)i * n + j] % p : (j - n == i ? 1 % p : 0);
    for (int c = 0; c < n; c++) {
        int r = -1;
        for (int i = c; i < n; i++) if (T[(size_t)i * w + c]) { r = i; break; }
        if (r < 0) { free(T); return 1; }
        if (r != c)
            for (int j = 0; j < w; j++) {
                u64 t = T[(size_t)r * w + j];
                T[(size_t)r * w + j] = T[(size_t)c * w + j];
                T[(size_t)c * w + j] = t;
            }
        u64 iv = orc_invmod(T[(size_t)c * w + c], p);
        for (int j = 0; j < w; j++) T[(size_t)c * w + j] = f_mul(T[(size_t)c * w + j], iv, p);
        for (int i = 0; i < n; i++) {
            if (i == c) continue;
            u64 f = T[(size_t)i * w + c];
            if (!f) continue;
            for (int j = 0; j < w; j++)
                T[(size_t)i * w + j] = f_sub(T[(size_t)i * w + j], f_mul(f, T[(size_t)c * w + j], p), p);
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Minv[(size_t)i * n + j] = T[(size_t)i * w + n + j];
    free(T);
    return 0;
}

/* X (n x n, length t) = A^-1 mod x^t for A (n x n, length dA), by the
 * recurrence X_j = -A_0^-1 sum_{i=1..min(j, dA-1)} A_i X_{j-i}.  Returns 0, or
 * 1 if A(0) is singular (X untouched). */
int orc_inv_trunc(u64 p, int n, const u64 *A, i64 dA, i64 t, u64 *X)
{
    size_t nn = (size_t)n * n;
    u64 *A0 = (u64 *)calloc(nn, sizeof(u64)), *A0i = (u64 *)calloc(nn, sizeof(u64));
    u64 *Sj = (u64 *)malloc(sizeof(u64) * nn);
    for (size_t e = 0; e < nn; e++) A0[e] = A[e * dA];
    if (orc_matinv(p, n, A0, A0i)) { free(A0); free(A0i); free(Sj); return 1; }
    memset(X, 0, sizeof(u64) * nn * t);
    for (size_t e = 0; e < nn; e++) X[e * t] = A0i[e];
    for (i64 j = 1; j < t; j++) {
        /* S_j = sum_{i=1..min(j, dA-1)} A_i X_{j-i} */
#pragma omp parallel for schedule(static) if (nn >= 64)
        for (size_t e = 0; e < nn; e++) {
            int r = (int)(e / n), c = (int)(e % n);
            u128 acc = 0;
            for (i64 i = 1; i <= j && i < dA; i++)
                for (int l = 0; l < n; l++)
                    acc_add(&acc, A[((size_t)r * n + l) * dA + i], X[((size_t)l * n + c) * t + (j - i)], p);
            Sj[e] = (u64)(acc % p);
        }
        /* X_j = -A_0^-1 S_j */
        for (int r = 0; r < n; r++)
            for (int c = 0; c < n; c++) {
                u64 v = 0;
                for (int l = 0; l < n; l++) v = f_add(v, f_mul(A0i[(size_t)r * n + l], Sj[(size_t)l * n + c], p), p);
                X[((size_t)r * n + c) * t + j] = f_neg(v, p);
            }
    }
    free(A0); free(A0i); free(Sj);
    return 0;
}

/* v (n x 1, length N) = A^-1 b mod x^N for A (n x n, length dA) with A(0)
 * invertible and b (n x 1, length db): v_j = A_0^-1 (b_j - sum_{i=1..j} A_i v_{j-i}).
 * Returns 0, or 1 if A(0) is singular (v untouched). */
int orc_solve_series(u64 p, int n, const u64 *A, i64 dA, const u64 *b, i64 db, i64 N, u64 *v)
{
    size_t nn = (size_t)n * n;
    u64 *A0 = (u64 *)calloc(nn, sizeof(u64)), *A0i = (u64 *)calloc(nn, sizeof(u64));
    u64 *rj = (u64 *)malloc(sizeof(u64) * n);
    for (size_t e = 0; e < nn; e++) A0[e] = A[e * dA];
    if (orc_matinv(p, n, A0, A0i)) { free(A0); free(A0i); free(rj); return 1; }
    memset(v, 0, sizeof(u64) * (size_t)n * N);
    for (i64 j = 0; j < N; j++) {
        /* r_j = b_j - sum_{i=1..min(j, dA-1)} A_i v_{j-i} */
        for (int r = 0; r < n; r++) {
            u128 acc = 0;
            for (i64 i = 1; i <= j && i < dA; i++)
                for (int l = 0; l < n; l++) acc_add(&acc, A[((size_t)r * n + l) * dA + i], v[(size_t)l * N + (j - i)], p);
            const u64 bj = j < db ? b[(size_t)r * db + j] % p : 0;
            rj[r] = f_sub(bj, (u64)(acc % p), p);
        }
        for (int r = 0; r < n; r++) {
            u128 acc = 0;
            for (int l = 0; l < n; l++) acc_add(&acc, A0i[(size_t)r * n + l], rj[l], p);
            v[(size_t)r * N + j] = (u64)(acc % p);
        }
    }
    free(A0); free(A0i); free(rj);
    return 0;
}

/* The high-order lifting slices (Sec. 4): S_i (n x n, length 2D + 1, D = dA - 1) =
 * coefficients (2^i - 1) D .. (2^i + 1) D of A^-1, for i = 0 .. K-1, read off the
 * truncated inverse.  Output S[((i n + r) n + c)(2D + 1) + t].  Returns 0, or 1 if
 * A(0) is singular. */
int orc_inv_slices(u64 p, int n, const u64 *A, i64 dA, int K, u64 *S)
{
    const i64 D = dA - 1, w = 2 * D + 1;
    const i64 t = ((i64)1 << (K - 1)) * D + D + 1;          /* through (2^(K-1) + 1) D */
    size_t nn = (size_t)n * n;
    u64 *X = (u64 *)malloc(sizeof(u64) * nn * t);
    if (orc_inv_trunc(p, n, A, dA, t, X)) { free(X); return 1; }
    for (int i = 0; i < K; i++) {
        const i64 s0 = (((i64)1 << i) - 1) * D;
        for (size_t e = 0; e < nn; e++)
            for (i64 j = 0; j < w; j++) S[((size_t)i * nn + e) * w + j] = X[e * t + s0 + j];
    }
    free(X);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Interpolant bases (Sec. 3, Algorithms 4 and 5)                       */
/* ------------------------------------------------------------------ */

/* P(a) for an entry of length len (Horner). */
static u64 poly_eval(const u64 *f, i64 len, u64 a, u64 p)
{
    u64 v = 0;
    for (i64 e = len - 1; e >= 0; e--) v = f_add(f_mul(v, a, p), f[e], p);
    return v;
}

/* x[i] <- c x[i] mod p for i < count. */
void orc_scale(u64 p, u64 *x, i64 count, u64 c)
{
    for (i64 i = 0; i < count; i++) x[i] = f_mul(x[i] % p, c % p, p);
}

/* out[e] = X_e(a) for the r x c entries of X (length len), by Horner's rule. */
void orc_pmat_eval(u64 p, int r, int c, const u64 *X, i64 len, u64 a, u64 *out)
{
    for (i64 e = 0; e < (i64)r * c; e++) out[e] = poly_eval(X + e * len, len, a % p, p);
}

/* Algorithm 4: E[(i n + j) sigma + l] = entry (i, j) of E_l, points alpha[l];
 * P: m x m, length sigma + 1; rdeg = rdeg_s(P). */
void orc_mintbasis(u64 p, int m, int n, const u64 *E, i64 sigma, const u64 *alpha, const i64 *s,
                   u64 *P, i64 *rdeg)
{
    const i64 len = sigma + 1;
    u64 *R = (u64 *)malloc(sizeof(u64) * (size_t)m * n);
    u64 *Q = (u64 *)malloc(sizeof(u64) * (size_t)m * m * 2);
    u64 *Pv = (u64 *)malloc(sizeof(u64) * (size_t)m * m);
    u64 *Pn = (u64 *)calloc((size_t)m * m * len, sizeof(u64));
    i64 *t = (i64 *)malloc(sizeof(i64) * m);
    i64 degP = 0;
    memset(P, 0, sizeof(u64) * (size_t)m * m * len);
    for (int i = 0; i < m; i++) P[((i64)i * m + i) * len] = 1;
    for (int i = 0; i < m; i++) t[i] = s[i];
    for (i64 k = 0; k < sigma; k++) {
        const u64 a = alpha[k] % p;
        /* a. R = P(alpha_k) E_k */
        for (i64 e = 0; e < (i64)m * m; e++) Pv[e] = poly_eval(P + e * len, degP + 1, a, p);
        for (int i = 0; i < m; i++)
            for (int j = 0; j < n; j++) {
                u128 acc = 0;
                for (int l = 0; l < m; l++) acc_add(&acc, Pv[(i64)i * m + l], E[((i64)l * n + j) * sigma + k], p);
                R[(i64)i * n + j] = (u64)(acc % p);
            }
        /* b. Q = M-Basis-1(R, t), x read as x - alpha_k: Q0 <- Q0 - alpha_k Q1 */
        orc_mbasis1(p, m, n, R, t, Q);
        for (i64 e = 0; e < (i64)m * m; e++) Q[e * 2] = f_sub(Q[e * 2], f_mul(a, Q[e * 2 + 1], p), p);
        /* c. P <- Q.P, t <- rdeg_s(P) */
        const i64 degN = degP + 1 < sigma ? degP + 1 : sigma;
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) {
                u64 *out = Pn + ((i64)i * m + j) * len;
                for (i64 c = 0; c <= degN; c++) {
                    u128 acc = 0;
                    for (int l = 0; l < m; l++) {
                        const u64 q0 = Q[((i64)i * m + l) * 2], q1 = Q[((i64)i * m + l) * 2 + 1];
                        const u64 *Plj = P + ((i64)l * m + j) * len;
                        if (q0 && c <= degP) acc_add(&acc, q0, Plj[c], p);
                        if (q1 && c >= 1 && c - 1 <= degP) acc_add(&acc, q1, Plj[c - 1], p);
                    }
                    out[c] = (u64)(acc % p);
                }
            }
        degP = degN;
        memcpy(P, Pn, sizeof(u64) * (size_t)m * m * len);
        orc_rdeg(m, m, P, len, s, t);
    }
    for (int i = 0; i < m; i++) rdeg[i] = t[i];
    free(R); free(Q); free(Pv); free(Pn); free(t);
}

/* Algorithm 5 with threshold T (Algorithm 4 if sigma <= T). */
void orc_pmintbasis(u64 p, int m, int n, const u64 *E, i64 sigma, const u64 *alpha, const i64 *s, i64 T,
                    u64 *P, i64 *rdeg)
{
    if (sigma <= T) { orc_mintbasis(p, m, n, E, sigma, alpha, s, P, rdeg); return; }
    const i64 s1 = (sigma + 1) / 2, s2 = sigma / 2;
    /* step 2: P1 = PM-IntBasis(E_1..s1, alpha_1..s1, s) */
    u64 *E1 = (u64 *)malloc(sizeof(u64) * (size_t)m * n * s1);
    for (i64 e = 0; e < (i64)m * n; e++)
        for (i64 l = 0; l < s1; l++) E1[e * s1 + l] = E[e * sigma + l];
    u64 *P1 = (u64 *)malloc(sizeof(u64) * (size_t)m * m * (s1 + 1));
    i64 *t1 = (i64 *)malloc(sizeof(i64) * m);
    orc_pmintbasis(p, m, n, E1, s1, alpha, s, T, P1, t1);
    /* step 3: R_l = P1(alpha_{s1+l}) E_{s1+l} */
    u64 *R = (u64 *)malloc(sizeof(u64) * (size_t)m * n * (s2 > 0 ? s2 : 1));
    u64 *Pv = (u64 *)malloc(sizeof(u64) * (size_t)m * m);
    for (i64 l = 0; l < s2; l++) {
        const u64 a = alpha[s1 + l] % p;
        for (i64 e = 0; e < (i64)m * m; e++) Pv[e] = poly_eval(P1 + e * (s1 + 1), s1 + 1, a, p);
        for (int i = 0; i < m; i++)
            for (int j = 0; j < n; j++) {
                u128 acc = 0;
                for (int k = 0; k < m; k++) acc_add(&acc, Pv[(i64)i * m + k], E[((i64)k * n + j) * sigma + s1 + l], p);
                R[((i64)i * n + j) * s2 + l] = (u64)(acc % p);
            }
    }
    /* steps 4-5: t = rdeg_s(P1); P2 = PM-IntBasis(R, alpha_{s1+1..sigma}, t) */
    u64 *P2 = (u64 *)malloc(sizeof(u64) * (size_t)m * m * (s2 + 1));
    i64 *t2 = (i64 *)malloc(sizeof(i64) * m);
    orc_pmintbasis(p, m, n, R, s2, alpha + s1, t1, T, P2, t2);
    /* step 6: P = P2 P1 */
    orc_pmat_slice(p, m, m, m, P2, s2 + 1, P1, s1 + 1, 0, sigma + 1, P);
    orc_rdeg(m, m, P, sigma + 1, s, rdeg);
    free(E1); free(P1); free(t1); free(R); free(Pv); free(P2); free(t2);
}

/* det M mod p (M: n x n, row-major, destroyed) by Gaussian elimination. */
static u64 det_destroy(u64 p, int n, u64 *M)
{
    u64 det = 1 % p;
    for (int c = 0; c < n; c++) {
        int r = -1;
        for (int i = c; i < n; i++) if (M[(size_t)i * n + c]) { r = i; break; }
        if (r < 0) return 0;
        if (r != c) {
            for (int j = 0; j < n; j++) {
                u64 t = M[(size_t)r * n + j];
                M[(size_t)r * n + j] = M[(size_t)c * n + j];
                M[(size_t)c * n + j] = t;
            }
            det = f_neg(det, p);
        }
        const u64 pv = M[(size_t)c * n + c];
        det = f_mul(det, pv, p);
        const u64 iv = orc_invmod(pv, p);
        for (int i = c + 1; i < n; i++) {
            const u64 fct = f_mul(M[(size_t)i * n + c], iv, p);
            if (!fct) continue;
            for (int j = c; j < n; j++)
                M[(size_t)i * n + j] = f_sub(M[(size_t)i * n + j], f_mul(fct, M[(size_t)c * n + j], p), p);
        }
    }
    return det;
}

/* The specialisations a(z) = f(x, z), b(z) = g(x, z) at x. */
static void specialise(u64 p, int dx, int dy, const u64 *f, u64 x, u64 *out)
{
    for (int j = 0; j <= dy; j++) {
        u64 v = 0;
        for (int i = dx; i >= 0; i--) v = f_add(f_mul(v, x, p), f[(i64)j * (dx + 1) + i], p);
        out[j] = v;
    }
}

/* det of the top-left m x m block of the 2m x 2m basis P (entries of length len) at x. */
static u64 det_at_first(u64 p, int m, int mm, const u64 *P, i64 len, u64 x, u64 *Qv)
{
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) Qv[i * m + j] = poly_eval(P + ((i64)i * mm + j) * len, len, x, p);
    return det_destroy(p, m, Qv);
}

/* Sec. 5.2, the variant of Algorithm 6 (Determinant) for Res_z(f, g): with P(x) the
 * Sylvester matrix of f, g in z (nu = dyf + dyg), H the m x m block of P^-1 named below,
 * delta = 2 ceil(nu / m) d + 1 values of H, an interpolant basis of [H; -I] (Algorithm 5)
 * whose first m rows give (Q, R) with H = Q^-1 R (the fraction-reconstruction statement of
 * Sec. 3), det Q = lambda Res (generic input), lambda fixed by one direct value of Res.
 * P(x) is the matrix of (u, v) -> u f + v g on the unknowns (u_0 .. u_{dyg-1}, v_0 ..
 * v_{dyf-1}) with the equations ordered by decreasing power of z; H is its top-right
 * quadrant: H[i][j] = u_i of the solution of u f + v g = z^(m-1-j).  Columns are taken here
 * in increasing power (H J, J the reversal), which leaves Q unchanged.
 * Points: the smallest non-negative integers where both leading coefficients and Res are
 * nonzero (delta of them) for H; 0 .. D for det Q.  Returns 0, or 1 when the points run out
 * (Res identically zero, or p too small), 2 when det Q vanishes at the normalisation point,
 * 3 when the normalised det Q differs from Res at one of the delta points (2 and 3: the input
 * is not generic). */
int orc_bivariate_resultant_villard(u64 p, int dxf, int dyf, const u64 *f, int dxg, int dyg, const u64 *g, int m,
                                    u64 *R)
{
    const int nu = dyf + dyg, d = dxf > dxg ? dxf : dxg;
    const i64 delta = 2 * (i64)((nu + m - 1) / m) * d + 1;
    const i64 D = (i64)dxf * dyg + (i64)dxg * dyf, N = D + 1;
    u64 *xs = (u64 *)malloc(sizeof(u64) * delta);
    u64 *E = (u64 *)calloc((size_t)2 * m * m * delta, sizeof(u64));
    u64 *S = (u64 *)malloc(sizeof(u64) * (size_t)nu * nu);
    u64 *Si = (u64 *)malloc(sizeof(u64) * (size_t)nu * nu);
    u64 *fa = (u64 *)malloc(sizeof(u64) * (dyf + 1));
    u64 *ga = (u64 *)malloc(sizeof(u64) * (dyg + 1));
    int rc = 0;
    i64 cnt = 0;
    u64 res0 = 0;
    /* at most D + dxf + dxg integers are roots of Res or of a leading coefficient */
    const u64 xlim = (u64)(delta + D + dxf + dxg + 1);
    for (u64 x = 0; cnt < delta; x++) {
        if (x >= p || x >= xlim) { rc = 1; break; }
        specialise(p, dxf, dyf, f, x, fa);
        specialise(p, dxg, dyg, g, x, ga);
        if (!fa[dyf] || !ga[dyg]) continue;
        /* Sylvester matrix, equation row r <-> coefficient of z^(nu-1-r) */
        memset(S, 0, sizeof(u64) * (size_t)nu * nu);
        for (int j = 0; j < dyg; j++)
            for (int t = 0; t <= dyf; t++) S[(size_t)(nu - 1 - (j + t)) * nu + j] = fa[t];
        for (int j = 0; j < dyf; j++)
            for (int t = 0; t <= dyg; t++) S[(size_t)(nu - 1 - (j + t)) * nu + dyg + j] = ga[t];
        if (orc_matinv(p, nu, S, Si)) continue;      /* Res(x) = 0 */
        if (cnt == 0) res0 = orc_univ_resultant(p, fa, dyf, ga, dyg);
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++)                 /* column nu-1-j <-> z^j */
                E[((i64)i * m + j) * delta + cnt] = Si[(size_t)i * nu + (nu - 1 - j)];
        xs[cnt++] = x;
    }
    if (!rc) {
        for (int i = 0; i < m; i++)
            for (i64 l = 0; l < delta; l++) E[((i64)(m + i) * m + i) * delta + l] = f_neg(1 % p, p);
        const int mm = 2 * m;
        u64 *P = (u64 *)malloc(sizeof(u64) * (size_t)mm * mm * (delta + 1));
        i64 *s0 = (i64 *)calloc(mm, sizeof(i64)), *rd = (i64 *)malloc(sizeof(i64) * mm);
        orc_pmintbasis(p, mm, m, E, delta, xs, s0, 32, P, rd);
        /* det Q at 0 .. D and at the normalisation point xs[0] */
        u64 *ys = (u64 *)malloc(sizeof(u64) * N), *pts = (u64 *)malloc(sizeof(u64) * N);
        u64 *Qv = (u64 *)malloc(sizeof(u64) * (size_t)m * m);
        const i64 len = delta + 1;
        for (i64 t = 0; t <= N; t++) {
            const u64 x = t < N ? (u64)t : xs[0];
            for (int i = 0; i < m; i++)
                for (int j = 0; j < m; j++) Qv[i * m + j] = poly_eval(P + ((i64)i * mm + j) * len, len, x, p);
            const u64 dq = det_destroy(p, m, Qv);
            if (t < N) { ys[t] = dq; pts[t] = x; }
            else if (!dq) rc = 2;
            else {
                const u64 scale = f_mul(res0, orc_invmod(dq, p), p);
                for (i64 k = 0; k < N; k++) ys[k] = f_mul(ys[k], scale, p);
            }
        }
        /* The properties the method rests on hold for generic input only: det Q must be a
         * constant multiple of Res.  Check the normalised det Q against Res at the delta
         * points (det Q evaluated there by Horner, Res by the univariate resultant). */
        const u64 sc = rc ? 0 : f_mul(res0, orc_invmod(det_at_first(p, m, mm, P, len, xs[0], Qv), p), p);
        for (i64 l = 0; !rc && l < delta; l++) {
            const u64 dq = det_at_first(p, m, mm, P, len, xs[l], Qv);
            specialise(p, dxf, dyf, f, xs[l], fa);
            specialise(p, dxg, dyg, g, xs[l], ga);
            if (f_mul(dq, sc, p) != orc_univ_resultant(p, fa, dyf, ga, dyg)) rc = 3;
        }
        if (!rc) interp_int_points(p, pts, ys, N, R);
        free(P); free(s0); free(rd); free(ys); free(pts); free(Qv);
    }
    free(xs); free(E); free(S); free(Si); free(fa); free(ga);
    return rc;
}
