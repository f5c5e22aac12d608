// resultant.cu -- bivariate resultant Res_y(f, g) in F_p[x] (Sec. 5.2, the
// direct evaluation / interpolation method), on the device.
//
// With N = D + 1 points (D = dxf dyg + dxg dyf bounds deg Res), q = alpha:
//  1. Evaluation of every x-coefficient polynomial of f and g at the geometric
//     progression 1, q, ..., q^(N-1) (Sec. 2: evaluation at geometric
//     progressions in O(M(d))): with C(t) = t (t - 1) / 2, i e = C(i+e) - C(i)
//     - C(e), so F(q^i) = q^-C(i) sum_e (F_e q^-C(e)) q^C(i+e): a middle product
//     of the scaled, reversed coefficients with the chirp h_t = q^C(t), run on
//     the product hot path (pmat_middle_product of a J x 1 by a 1 x 1 matrix).
//  2. At each point, the univariate resultant by the Euclidean algorithm
//     (Res(A,B) = (-1)^(ab) lc(B)^(a-r) Res(B, A mod B)), one warp per point,
//     pseudo-remainders so that no inversion is needed until the end.
//  3. Interpolation at the geometric progression: with w_t = prod_{l=1..t}
//     (q^l - 1), the Newton coefficients c_k satisfy sum_i (v_i / w_i) x^i =
//     (sum_k c_k q^C(k) x^k)(sum_t x^t / w_t), and the series of 1 / w_t has
//     the inverse sum_t (-1)^t q^C(t) x^t / w_t (q-exponential identity); the
//     Newton-to-monomial change of basis is, by the q-binomial theorem,
//     R_m w_m = sum_t c_{m+t} w_{m+t} (-1)^t q^C(t) / w_t.  Both are
//     truncated products of length N on the hot path.
// The Villard variant (bivariate_resultant_villard, Sec. 5.2 over Algorithm 6) shares the
// evaluation, the interpolation and the product path; its own kernels are the per-point
// extended Euclid that yields H(alpha) and Res(alpha), the per-point determinant of Q and the
// normalisation; the interpolant basis comes from pm_intbasis.
//
// The points are c q^i (the substitution x -> c x, undone on the result's
// coefficients): they must be distinct (q^l != 1 for 0 < l < N) and keep the
// leading y-coefficients nonzero; a pair (c, q) that fails either is replaced
// by the next candidate.  By uniqueness of the resultant the output does not
// depend on the points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host.h"

#define CKI(call)                                                       \
    do {                                                                \
        int _rc = (call);                                               \
        if (_rc) return _rc;                                            \
    } while (0)

#define RES_MAXI 16   // instances per launch

struct ResInst {
    u64 p, pn, one, r2;     // Montgomery constants (R = 2^64)
    u64 qm, qim;            // q and q^-1, Montgomery form
    u64 cm, cim;            // point scale c and c^-1, Montgomery form (points are c q^i)
    const u64 *f, *g;       // inputs (plain), f[j*(dxf+1) + i]
    u64 *R;                 // output (plain), N values
    u64 *qp, *h, *hinv;     // q^t, q^C(t), q^-C(t) (Montgomery), t < NE
    u64 *Ua, *Hb;           // evaluation operands (plain): J x E and NE
    u64 *S;                 // evaluation output J x N (plain)
    u64 *Vt;                // values, point-major N x J (Montgomery)
    u64 *v;                 // resultant values (plain), N
    u64 *w, *winv;          // w_t and 1 / w_t (Montgomery), N
    u64 *Va, *Eb, *Cp, *Ur, *Y;   // interpolation operands / outputs (plain), N
};

struct ResPack {
    int count;
    int dxf, dyf, dxg, dyg;
    int E, J, N, NE;        // E = max(dxf, dxg) + 1, J = dyf + dyg + 2, NE = N + E - 1
    int *flag;              // bit 1: q^l = 1 for some 0 < l < N; bit 2: a leading coefficient vanishes
    ResInst in[RES_MAXI];
};

__device__ __forceinline__ u64 mm(u64 a, u64 b, const ResInst &I) { return mont_mul(a, b, I.p, I.pn); }
__device__ u64 mpw(u64 a, u64 e, const ResInst &I)
{
    u64 r = I.one;
    while (e) {
        if (e & 1) r = mm(r, a, I);
        a = mm(a, a, I);
        e >>= 1;
    }
    return r;
}

// ------------------------------------------------------------------ 1. powers, evaluation operands
__global__ void k_res_powers(const __grid_constant__ ResPack P)
{
    const ResInst &I = P.in[blockIdx.y];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P.NE; t += gridDim.x * blockDim.x) {
        const u64 c2 = (u64)t * (u64)(t > 0 ? t - 1 : 0) / 2;
        const u64 qt = mpw(I.qm, (u64)t, I);
        I.qp[t] = qt;
        I.h[t] = mpw(I.qm, c2, I);
        I.hinv[t] = mpw(I.qim, c2, I);
        I.Hb[t] = mm(I.h[t], 1, I);
        if (t >= 1 && t < P.N && qt == I.one) atomicOr(P.flag, 1);
    }
}

// Ua[j][E-1-e] = coefficient e of row j times q^-C(e); rows 0..dyf from f, then g.
__global__ void k_res_prep_eval(const __grid_constant__ ResPack P)
{
    const ResInst &I = P.in[blockIdx.y];
    const int total = P.J * P.E;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < total; x += gridDim.x * blockDim.x) {
        const int j = x / P.E, e = x % P.E;
        u64 c = 0;
        if (j <= P.dyf) { if (e <= P.dxf) c = I.f[(i64)j * (P.dxf + 1) + e]; }
        else { const int jg = j - P.dyf - 1; if (e <= P.dxg) c = I.g[(i64)jg * (P.dxg + 1) + e]; }
        c = mm(c, mpw(I.cm, (u64)e, I), I);                         // x -> c x: coefficient e times c^e
        I.Ua[(i64)j * P.E + (P.E - 1 - e)] = mm(c, I.hinv[e], I);   // plain x Montgomery = plain
    }
}

// values F_j(q^i) = q^-C(i) S[j][i], stored point-major in Montgomery form; leading
// y-coefficients must not vanish.
__global__ void k_res_eval_finish(const __grid_constant__ ResPack P)
{
    const ResInst &I = P.in[blockIdx.y];
    const i64 total = (i64)P.J * P.N;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < total; x += (i64)gridDim.x * blockDim.x) {
        const int j = (int)(x / P.N), i = (int)(x % P.N);
        const u64 val = mm(I.S[x], I.hinv[i], I);
        if ((j == P.dyf || j == P.J - 1) && val == 0) atomicOr(P.flag, 2);
        I.Vt[(i64)i * P.J + j] = mm(val, I.r2, I);
    }
}

// ------------------------------------------------------------------ 2. Euclid, one warp per point
__device__ __forceinline__ int warp_deg(const u64 *A, int start)
{
    const int lane = threadIdx.x & 31;
    for (int base = start & ~31; base >= 0; base -= 32) {
        const int c = base + lane;
        const unsigned b = __ballot_sync(0xffffffffu, c <= start && A[c] != 0);
        if (b) return base + 31 - __clz(b);
    }
    return -1;
}

// Res(A, B) = (-1)^(ab) lc(B)^(a-r) Res(B, A mod B); with s pseudo-division steps
// A_s = lc(B)^s A mod B, Res(B, A_s) = lc(B)^(s b) Res(B, A mod B).  Each remainder
// step records (lc(B), a - r, s b) in shared memory; the powers are taken at the end,
// 32 records at a time across the lanes.  Two steps with shifts sh and sh - 1 are
// fused: A <- lc(B)^2 A - lc(B) lc(A) x^sh B - t x^(sh-1) B, t = lc(B) A[da-1] -
// lc(A) B[b-1] (t = 0 only means the degree fell further; the relation still holds).
__global__ void __launch_bounds__(256) k_res_euclid(const __grid_constant__ ResPack P, int dmax)
{
    extern __shared__ u64 sme[];
    const ResInst &I = P.in[blockIdx.y];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int pt = blockIdx.x * (blockDim.x >> 5) + wid;
    if (pt >= P.N) return;
    const int nrec = dmax + 2;
    u64 *A = sme + (size_t)wid * (2 * (dmax + 1) + 3 * nrec);
    u64 *B = A + (dmax + 1);
    u64 *rl = B + (dmax + 1);            // lc(B) per remainder step
    u64 *rn = rl + nrec;                 // exponent a - r
    u64 *rd = rn + nrec;                 // exponent s b
    const u64 *val = I.Vt + (i64)pt * P.J;
    int a = P.dyf, b = P.dyg;
    for (int c = lane; c <= a; c += 32) A[c] = val[c];
    for (int c = lane; c <= b; c += 32) B[c] = val[P.dyf + 1 + c];
    __syncwarp();
    u64 tail = I.one;                    // lc^deg factor of the last step
    bool neg = false, zero = false;
    int nr = 0;
    for (;;) {
        if (b == 0) { tail = mpw(B[0], (u64)a, I); break; }
        if (a == 0) { tail = mpw(A[0], (u64)b, I); break; }
        if (a < b) {                                // Res(A, B) = (-1)^(ab) Res(B, A)
            u64 *sw = A; A = B; B = sw;
            int t = a; a = b; b = t;
            neg ^= (a & b & 1);
        }
        const u64 lcB = B[b];
        const u64 lcB2 = mm(lcB, lcB, I);
        int da = a, s = 0;
        while (da >= b) {
            const u64 lcA = A[da];
            const int sh = da - b;
            if (sh >= 1) {
                const u64 t = mont_msub(lcB, A[da - 1], lcA, B[b - 1], I.p, I.pn);
                const u64 f1 = mm(lcB, lcA, I);
                __syncwarp();                       // every lane has read A[da], A[da - 1]
                for (int c = lane; c <= da - 2; c += 32) {
                    u64 x;
                    if (c >= sh) x = mont_msub2(lcB2, A[c], f1, B[c - sh], t, B[c - sh + 1], I.p, I.pn);
                    else if (c == sh - 1) x = mont_msub(lcB2, A[c], t, B[0], I.p, I.pn);
                    else x = mm(lcB2, A[c], I);
                    A[c] = x;
                }
                s += 2;
                __syncwarp();                       // the new coefficients are visible to the whole warp
                da = warp_deg(A, da - 2);
            } else {
                __syncwarp();
                for (int c = lane; c <= da - 1; c += 32) A[c] = mont_msub(lcB, A[c], lcA, B[c], I.p, I.pn);
                s += 1;
                __syncwarp();
                da = warp_deg(A, da - 1);
            }
            __syncwarp();
        }
        const int r = da;
        if (r < 0) { zero = true; break; }
        neg ^= (a & b & 1);
        if (lane == 0) { rl[nr] = lcB; rn[nr] = (u64)(a - r); rd[nr] = (u64)s * (u64)b; }
        nr++;
        u64 *sw = A; A = B; B = sw;                // (A, B) <- (B, R)
        a = b;
        b = r;
    }
    __syncwarp();
    if (zero) {
        if (lane == 0) I.v[pt] = 0;
        return;
    }
    // num = prod lc^(a-r), den = prod lc^(s b): 32 records at a time
    u64 num = I.one, den = I.one;
    for (int i = lane; i < nr; i += 32) {
        num = mm(num, mpw(rl[i], rn[i], I), I);
        den = mm(den, mpw(rl[i], rd[i], I), I);
    }
    for (int o = 16; o >= 1; o >>= 1) {
        num = mm(num, __shfl_xor_sync(0xffffffffu, num, o), I);
        den = mm(den, __shfl_xor_sync(0xffffffffu, den, o), I);
    }
    if (lane == 0) {
        u64 res = mm(mm(num, tail, I), mpw(den, I.p - 2, I), I);
        res = mm(res, 1, I);
        if (neg && res) res = I.p - res;
        I.v[pt] = res;
    }
}

// ------------------------------------------------------------------ 3. interpolation
// w_t = prod_{l=1..t} (q^l - 1) and 1 / w_t, one block of 1024 threads per instance:
// chunked prefix / suffix products, one inversion.
__global__ void __launch_bounds__(1024) k_res_wscan(const __grid_constant__ ResPack P)
{
    __shared__ u64 pre[1024], suf[1024];
    const ResInst &I = P.in[blockIdx.x];
    const int N = P.N, tid = threadIdx.x;
    const int per = (N + 1023) / 1024;
    const int lo = tid * per, hi = min(N, lo + per);
    auto fac = [&](int t) -> u64 { return t >= 1 ? sub64(I.qp[t], I.one, I.p) : I.one; };
    u64 a = I.one;
    for (int t = lo; t < hi; t++) a = mm(a, fac(t), I);
    pre[tid] = a;
    suf[tid] = a;
    __syncthreads();
    // inclusive scans (Hillis-Steele), forward for prefixes and backward for suffixes
    for (int o = 1; o < 1024; o <<= 1) {
        u64 x = tid >= o ? pre[tid - o] : I.one;
        u64 y = tid + o < 1024 ? suf[tid + o] : I.one;
        __syncthreads();
        pre[tid] = mm(pre[tid], x, I);
        suf[tid] = mm(suf[tid], y, I);
        __syncthreads();
    }
    const u64 total = pre[1023];
    const u64 tinv = mpw(total, I.p - 2, I);       // 1 / w_{N-1}
    u64 run = tid ? pre[tid - 1] : I.one;           // product of the factors before this chunk
    for (int t = lo; t < hi; t++) { run = mm(run, fac(t), I); I.w[t] = run; }
    // 1 / w_t = (1 / w_{N-1}) prod_{l = t+1 .. N-1} (q^l - 1)
    u64 after = tid + 1 < 1024 ? suf[tid + 1] : I.one;
    for (int t = hi - 1; t >= lo; t--) { I.winv[t] = mm(tinv, after, I); after = mm(after, fac(t), I); }
}

// V_i = v_i / w_i and E_t = (-1)^t q^C(t) / w_t (plain)
__global__ void k_res_interp1(const __grid_constant__ ResPack P)
{
    const ResInst &I = P.in[blockIdx.y];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P.N; t += gridDim.x * blockDim.x) {
        I.Va[t] = mm(I.v[t], I.winv[t], I);
        u64 e = mm(mm(I.h[t], I.winv[t], I), 1, I);
        if ((t & 1) && e) e = I.p - e;
        I.Eb[t] = e;
    }
}

// c_k = C'_k q^-C(k); u_k = c_k w_k; Ur[N-1-k] = u_k (plain)
__global__ void k_res_interp2(const __grid_constant__ ResPack P)
{
    const ResInst &I = P.in[blockIdx.y];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.N; k += gridDim.x * blockDim.x) {
        const u64 c = mm(I.Cp[k], I.hinv[k], I);
        I.Ur[P.N - 1 - k] = mm(c, I.w[k], I);
    }
}

// R_m = Y_{N-1-m} / w_m (plain)
__global__ void k_res_interp3(const __grid_constant__ ResPack P)
{
    const ResInst &I = P.in[blockIdx.y];
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P.N; m += gridDim.x * blockDim.x)
        I.R[m] = mm(mm(I.Y[P.N - 1 - m], I.winv[m], I), mpw(I.cim, (u64)m, I), I);   // undo x -> c x
}


// ------------------------------------------------------------------ Villard variant (Sec. 5.2)
// Algorithm 6 with values: H(alpha) = top-right m x m block of P(alpha)^-1, P the Sylvester
// matrix of f(alpha, z), g(alpha, z) as the map (u, v) -> u f + v g with the equations
// ordered by decreasing power of z.  Column j (taken here in increasing power, which leaves
// the fraction denominator unchanged) is the u-part of the solution of u f + v g = z^j:
// u = z^j s mod g with s f + t g = 1 (extended Euclid), so H[i][j] = [z^i] (z^j s mod g).
#define VIL_WARPS 4
#define VIL_MMAX 16

// One warp per point l < P.N: the extended Euclidean algorithm on (f_alpha, g_alpha) by
// pseudo-division, tracking the cofactor of f and Res(f_alpha, g_alpha); writes H(alpha_l) and
// the -I block into Eip (2m x m x P.N, plain) and Res into resv[l] (plain); Res = 0 sets flag
// bit 4.  Each quotient term is one pseudo-division step A <- lc(B) A - lc(A) y^sh B, applied
// to the cofactor alike (the relation A = s_A f + t_A g is linear), so no inversion is needed
// until the end: with s steps, prem = lc(B)^s (A mod B), hence Res(A, B) = (-1)^(ab)
// lc(B)^(a-r) Res(B, prem) / lc(B)^(s b); the factors are recorded per remainder and the
// powers taken at the end (one inversion), and the final constant B0 = s_B f + t_B g gives
// s = s_B / B0 (another).  H then needs lc(g)^-1 (a third).
__global__ void __launch_bounds__(32 * VIL_WARPS) k_vil_xgcd(const __grid_constant__ ResPack P, int dmax, int m,
                                                            u64 *Eip, u64 *resv)
{
    extern __shared__ u64 smv[];
    const ResInst &I = P.in[0];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int pt = blockIdx.x * VIL_WARPS + wid;
    if (pt >= P.N) return;
    const int W = dmax + 2;
    u64 *A = smv + (size_t)wid * 8 * W, *B = A + W, *sA = B + W, *sB = sA + W, *G = sB + W;
    u64 *rl = G + W, *rn = rl + W, *rd = rn + W;       // per remainder: lc(B), a - r, s b
    const u64 *val = I.Vt + (i64)pt * P.J;
    for (int c = lane; c < W; c += 32) {
        A[c] = c <= P.dyf ? val[c] : 0;
        B[c] = c <= P.dyg ? val[P.dyf + 1 + c] : 0;
        G[c] = B[c];
        sA[c] = c == 0 ? I.one : 0;
        sB[c] = 0;
    }
    __syncwarp();
    int a = P.dyf, b = P.dyg, dsA = 0, dsB = -1, nr = 0;
    bool neg = false, zero = false;
    while (b > 0) {
        const u64 lcB = B[b];
        int da = a, st = 0;
        while (da >= b) {
            const u64 lcA = A[da];
            const int sh = da - b;
            const int top = dsA > sh + dsB ? dsA : sh + dsB;
            __syncwarp();                                // every lane has read A[da]
            for (int i = lane; i < da; i += 32)
                A[i] = i >= sh ? mont_msub(lcB, A[i], lcA, B[i - sh], I.p, I.pn) : mm(lcB, A[i], I);
            for (int i = lane; i <= top && i < W; i += 32) {
                const u64 y = (i >= sh && i - sh <= dsB) ? sB[i - sh] : 0;
                sA[i] = mont_msub(lcB, sA[i], lcA, y, I.p, I.pn);
            }
            dsA = top < W - 1 ? top : W - 1;
            st++;
            __syncwarp();
            if (lane == 0) A[da] = 0;
            __syncwarp();
            da = da > 0 ? warp_deg(A, da - 1) : -1;
        }
        const int r = da;
        if (r < 0) { zero = true; break; }
        neg ^= (a & b & 1);
        if (lane == 0) { rl[nr] = lcB; rn[nr] = (u64)(a - r); rd[nr] = (u64)st * (u64)b; }
        nr++;
        u64 *t = A; A = B; B = t;                        // (A, B) <- (B, prem), cofactors alike
        t = sA; sA = sB; sB = t;
        a = b; b = r;
        const int d2 = dsA; dsA = dsB; dsB = d2;
        __syncwarp();
    }
    u64 *H = Eip;
    const i64 sig = P.N;
    if (zero) {
        for (int x = lane; x < 2 * m * m; x += 32) H[(i64)x * sig + pt] = 0;
        if (lane == 0) { resv[pt] = 0; atomicOr(P.flag, 4); }
        return;
    }
    // Res = (-1)^.. prod lc^(a-r) B0^a / prod lc^(s b): 32 records at a time, one inversion
    const u64 b0 = B[0];
    u64 num = I.one, den = I.one;
    for (int i = lane; i < nr; i += 32) {
        num = mm(num, mpw(rl[i], rn[i], I), I);
        den = mm(den, mpw(rl[i], rd[i], I), I);
    }
    for (int o = 16; o >= 1; o >>= 1) {
        num = mm(num, __shfl_xor_sync(0xffffffffu, num, o), I);
        den = mm(den, __shfl_xor_sync(0xffffffffu, den, o), I);
    }
    if (lane == 0) {
        u64 res = mm(mm(mm(num, mpw(b0, (u64)a, I), I), mpw(den, I.p - 2, I), I), 1, I);
        if (neg && res) res = I.p - res;
        resv[pt] = res;
    }
    const u64 binv = mpw(b0, I.p - 2, I);
    const int n2 = P.dyg;
    u64 *u = sA, *tmp = A;                               // sA and A are free now
    for (int c = lane; c < W; c += 32) u[c] = c < n2 ? mm(sB[c], binv, I) : 0;
    __syncwarp();
    const u64 ginv = mpw(G[n2], I.p - 2, I);
    for (int j = 0; j < m; j++) {
        for (int i = lane; i < m; i += 32) H[((i64)i * m + j) * sig + pt] = mm(u[i], 1, I);
        if (j + 1 == m) break;
        const u64 t = mm(u[n2 - 1], ginv, I);            // u <- y u mod g
        for (int i = lane; i < n2; i += 32) tmp[i] = sub64(i ? u[i - 1] : 0, mm(t, G[i], I), I.p);
        __syncwarp();
        for (int i = lane; i < n2; i += 32) u[i] = tmp[i];
        __syncwarp();
    }
    for (int x = lane; x < m * m; x += 32) {
        const int i = x / m, j = x % m;
        H[((i64)(m + i) * m + j) * sig + pt] = i == j ? I.p - 1 : 0;
    }
}

// ue[e] = c^e q^-C(e) (Montgomery), e < LQ
__global__ void k_vil_uvec(const __grid_constant__ ResPack P, u64 *ue, int LQ)
{
    const ResInst &I = P.in[0];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < LQ; e += gridDim.x * blockDim.x)
        ue[e] = mm(mpw(I.cm, (u64)e, I), I.hinv[e], I);
}

// Ua2[r][LQ-1-e] = Q_r[e] ue[e] (plain), r = i m + j for the top-left m x m block of the
// 2m x 2m basis Pb (entry stride sP)
__global__ void k_vil_prep_q(const __grid_constant__ ResPack P, const u64 *Pb, i64 sP, int m, const u64 *ue, u64 *Ua2,
                             int LQ)
{
    const ResInst &I = P.in[0];
    const i64 total = (i64)m * m * LQ;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < total; x += (i64)gridDim.x * blockDim.x) {
        const int e = (int)(x % LQ), r = (int)(x / LQ), i = r / m, j = r % m;
        Ua2[(i64)r * LQ + (LQ - 1 - e)] = mm(Pb[((i64)i * 2 * m + j) * sP + e], ue[e], I);
    }
}

// v[l] = det Q(c q^l) (plain), l < P.N: Q(c q^l)[i][j] = q^-C(l) S2[i m + j][l]
__global__ void k_vil_det(const __grid_constant__ ResPack P, const u64 *S2, int m, u64 *v)
{
    const ResInst &I = P.in[0];
    u64 M[VIL_MMAX * VIL_MMAX];
    for (i64 l = blockIdx.x * (i64)blockDim.x + threadIdx.x; l < P.N; l += (i64)gridDim.x * blockDim.x) {
        const u64 hl = mm(I.hinv[l], I.r2, I);     // q^-C(l) R^2: plain x this = Montgomery form
        for (int x = 0; x < m * m; x++) M[x] = mm(S2[(i64)x * P.N + l], hl, I);
        u64 det = I.one;
        bool neg = false;
        for (int c = 0; c < m && det; c++) {
            int r = c;
            while (r < m && M[r * m + c] == 0) r++;
            if (r == m) { det = 0; break; }
            if (r != c) {
                for (int j = c; j < m; j++) { const u64 t = M[r * m + j]; M[r * m + j] = M[c * m + j]; M[c * m + j] = t; }
                neg = !neg;
            }
            const u64 pv = M[c * m + c];
            det = mm(det, pv, I);
            const u64 pinv = mpw(pv, I.p - 2, I);
            for (int r2 = c + 1; r2 < m; r2++) {
                const u64 fct = mm(M[r2 * m + c], pinv, I);
                if (!fct) continue;
                for (int j = c + 1; j < m; j++) M[r2 * m + j] = sub64(M[r2 * m + j], mm(fct, M[c * m + j], I), I.p);
            }
        }
        u64 d = mm(det, 1, I);
        if (neg && d) d = I.p - d;
        v[l] = d;
    }
}

// sc[0] = Res(alpha_0) / det Q(alpha_0) (Montgomery); det Q(alpha_0) = 0 sets flag bit 16
__global__ void k_vil_norm(const __grid_constant__ ResPack P, const u64 *resv, const u64 *v, u64 *sc)
{
    const ResInst &I = P.in[0];
    if (threadIdx.x || blockIdx.x) return;
    if (v[0] == 0) { atomicOr(P.flag, 16); sc[0] = 0; return; }
    sc[0] = mm(mm(resv[0], I.r2, I), mpw(mm(v[0], I.r2, I), I.p - 2, I), I);
}

// v[l] <- v[l] sc; the first nchk values must equal the directly computed resultants (else
// flag bit 8: det Q is not a constant multiple of Res, the input is not generic)
__global__ void k_vil_scale(const __grid_constant__ ResPack P, const u64 *resv, const u64 *sc, u64 *v, int nchk)
{
    const ResInst &I = P.in[0];
    const u64 c = sc[0];
    for (i64 l = blockIdx.x * (i64)blockDim.x + threadIdx.x; l < P.N; l += (i64)gridDim.x * blockDim.x) {
        const u64 x = mm(v[l], c, I);
        v[l] = x;
        if (l < nchk && x != resv[l]) atomicOr(P.flag, 8);
    }
}

// ------------------------------------------------------------------ host driver
static uint64_t mont_pn(uint64_t p)
{
    uint64_t inv = 1;
    for (int i = 0; i < 7; i++) inv *= 2 - p * inv;
    return (uint64_t)0 - inv;
}

static int res_batch(pm_ctx *ctx, int cnt, const uint64_t *primes, const uint64_t *alphas, const uint64_t *scales,
                     int dxf, int dyf,
                     const u64 *f, int dxg, int dyg, const u64 *g, u64 *R, int *h_flag)
{
    const int64_t D = (int64_t)dxf * dyg + (int64_t)dxg * dyf;
    const int N = (int)(D + 1), E = (dxf > dxg ? dxf : dxg) + 1, J = dyf + dyg + 2, NE = N + E - 1;
    const size_t nf = (size_t)(dyf + 1) * (dxf + 1), ng = (size_t)(dyg + 1) * (dxg + 1);
    ResPack pk;
    memset(&pk, 0, sizeof(pk));
    pk.count = cnt; pk.dxf = dxf; pk.dyf = dyf; pk.dxg = dxg; pk.dyg = dyg;
    pk.E = E; pk.J = J; pk.N = N; pk.NE = NE;
    const size_t per = (size_t)NE * 8 * 4 + (size_t)J * E * 8 + (size_t)J * N * 8 * 2 + (size_t)N * 8 * 8 + 16 * 256;
    CKI(arena_reserve(ctx, per * cnt + 256));
    pk.flag = (int *)arena_alloc(ctx, 256);
    for (int i = 0; i < cnt; i++) {
        ResInst &I = pk.in[i];
        const uint64_t p = primes[i];
        I.p = p;
        I.pn = mont_pn(p);
        I.one = (uint64_t)(((unsigned __int128)1 << 64) % p);
        I.r2 = (uint64_t)((unsigned __int128)I.one * I.one % p);
        I.qm = (uint64_t)((unsigned __int128)(alphas[i] % p) * I.one % p);
        I.qim = (uint64_t)((unsigned __int128)host_powmod(alphas[i] % p, p - 2, p) * I.one % p);
        I.cm = (uint64_t)((unsigned __int128)(scales[i] % p) * I.one % p);
        I.cim = (uint64_t)((unsigned __int128)host_powmod(scales[i] % p, p - 2, p) * I.one % p);
        I.f = f + i * nf;
        I.g = g + i * ng;
        I.R = R + (size_t)i * N;
        auto A = [&](size_t n) { return (u64 *)arena_alloc(ctx, n * 8); };
        I.qp = A(NE); I.h = A(NE); I.hinv = A(NE); I.Hb = A(NE);
        I.Ua = A((size_t)J * E); I.S = A((size_t)J * N); I.Vt = A((size_t)J * N);
        I.v = A(N); I.w = A(N); I.winv = A(N); I.Va = A(N); I.Eb = A(N); I.Cp = A(N); I.Ur = A(N); I.Y = A(N);
        if (!I.Y) return pm_fail(ctx, PM_ENOMEM, "resultant arena exhausted");
    }
    CKI(pm_cuda(ctx, cudaMemsetAsync(pk.flag, 0, sizeof(int), ctx->stream), "flag"));
    const dim3 grid((NE + 255) / 256 < 1024 ? (NE + 255) / 256 : 1024, cnt);
    int tok = stage_begin(ctx, PM_STAGE_OTHER);
    k_res_powers<<<grid, 256, 0, ctx->stream>>>(pk);
    k_res_prep_eval<<<dim3((J * E + 255) / 256, cnt), 256, 0, ctx->stream>>>(pk);
    ctx->launches += 2;
    CKI(pm_cuda(ctx, cudaGetLastError(), "resultant prep"));
    stage_end(ctx, tok);
    // 1. evaluation: one middle product per instance (J x 1 times 1 x 1)
    {
        std::vector<ProdReq> rq(cnt);
        for (int i = 0; i < cnt; i++) {
            ProdReq &q = rq[i];
            q.p = primes[i]; q.w = 8; q.m = J; q.n = 1; q.k = 1;
            q.A = pk.in[i].Ua; q.dA = E; q.sA = E;
            q.B = pk.in[i].Hb; q.dB = NE; q.sB = NE;
            q.off = E - 1; q.len = N; q.C = pk.in[i].S; q.sC = N;
            q.lg = ceil_log2((int64_t)E - 1 + N);
            if (q.lg < 4) q.lg = 4;
        }
        CKI(prod_batch(ctx, rq.data(), cnt));
    }
    tok = stage_begin(ctx, PM_STAGE_OTHER);
    k_res_eval_finish<<<dim3(1024, cnt), 256, 0, ctx->stream>>>(pk);
    ctx->launches++;
    CKI(pm_cuda(ctx, cudaGetLastError(), "resultant eval"));
    // the flag decides whether this q is usable
    CKI(pm_cuda(ctx, cudaMemcpyAsync(h_flag, pk.flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "flag"));
    CKI(pm_cuda(ctx, cudaStreamSynchronize(ctx->stream), "flag sync"));
    stage_end(ctx, tok);
    if (*h_flag) return PM_OK;
    // 2. univariate resultants, one warp per point
    tok = stage_begin(ctx, PM_STAGE_OTHER);
    {
        const int dmax = dyf > dyg ? dyf : dyg;
        const size_t sm = (size_t)8 * (2 * (dmax + 1) + 3 * (dmax + 2)) * 8;
        if (sm > 48 * 1024) cudaFuncSetAttribute(k_res_euclid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_res_euclid<<<dim3((N + 7) / 8, cnt), 256, sm, ctx->stream>>>(pk, dmax);
        k_res_wscan<<<cnt, 1024, 0, ctx->stream>>>(pk);
        k_res_interp1<<<dim3((N + 255) / 256, cnt), 256, 0, ctx->stream>>>(pk);
        ctx->launches += 3;
        CKI(pm_cuda(ctx, cudaGetLastError(), "resultant euclid"));
    }
    stage_end(ctx, tok);
    // 3. interpolation: two truncated products of length N
    std::vector<ProdReq> rq(cnt);
    auto trunc_req = [&](int i, const u64 *Aop, const u64 *Bop, u64 *Cout) {
        ProdReq &q = rq[i];
        q.p = primes[i]; q.w = 8; q.m = 1; q.n = 1; q.k = 1;
        q.A = Aop; q.dA = N; q.sA = N; q.B = Bop; q.dB = N; q.sB = N;
        q.off = 0; q.len = N; q.C = Cout; q.sC = N;
        q.lg = ceil_log2(2 * (int64_t)N - 1);
        if (q.lg < 4) q.lg = 4;
    };
    for (int i = 0; i < cnt; i++) trunc_req(i, pk.in[i].Va, pk.in[i].Eb, pk.in[i].Cp);
    CKI(prod_batch(ctx, rq.data(), cnt));
    tok = stage_begin(ctx, PM_STAGE_OTHER);
    k_res_interp2<<<dim3((N + 255) / 256, cnt), 256, 0, ctx->stream>>>(pk);
    ctx->launches++;
    CKI(pm_cuda(ctx, cudaGetLastError(), "resultant interp"));
    stage_end(ctx, tok);
    for (int i = 0; i < cnt; i++) trunc_req(i, pk.in[i].Ur, pk.in[i].Eb, pk.in[i].Y);
    CKI(prod_batch(ctx, rq.data(), cnt));
    tok = stage_begin(ctx, PM_STAGE_OTHER);
    k_res_interp3<<<dim3((N + 255) / 256, cnt), 256, 0, ctx->stream>>>(pk);
    ctx->launches++;
    CKI(pm_cuda(ctx, cudaGetLastError(), "resultant interp"));
    stage_end(ctx, tok);
    return PM_OK;
}

extern "C" int bivariate_resultant(pm_ctx *ctx, int nprimes, const uint64_t *primes, int dxf, int dyf, const void *f,
                                   int dxg, int dyg, const void *g, void *R)
{
    if (!ctx) return PM_EINVAL;
    if (nprimes < 1 || !primes || !f || !g || !R) return pm_fail(ctx, PM_EINVAL, "bad arguments");
    if (dxf < 0 || dyf < 0 || dxg < 0 || dyg < 0) return pm_fail(ctx, PM_EINVAL, "negative degree");
    if (dyf > 2047 || dyg > 2047) return pm_fail(ctx, PM_EUNSUPPORTED, "y-degree above 2047");
    const int64_t D = (int64_t)dxf * dyg + (int64_t)dxg * dyf;
    const int E = (dxf > dxg ? dxf : dxg) + 1;
    if (2 * (D + 1) - 1 > (1 << PM_MAX_LOG2L) || D + E > (1 << PM_MAX_LOG2L))
        return pm_fail(ctx, PM_EINVAL, "resultant degree too large for the transforms");
    for (int i = 0; i < nprimes; i++)
        if (!(primes[i] & 1) || primes[i] < 3 || primes[i] >= (1ull << 62) || primes[i] <= (uint64_t)(2 * (D + 1)))
            return pm_fail(ctx, PM_EINVAL, "each prime must be odd, below 2^62 and above 2(D+1)");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    const size_t nf = (size_t)(dyf + 1) * (dxf + 1), ng = (size_t)(dyg + 1) * (dxg + 1);
    const size_t N = (size_t)D + 1;
    for (int i0 = 0; i0 < nprimes; i0 += RES_MAXI) {
        const int cnt = nprimes - i0 < RES_MAXI ? nprimes - i0 : RES_MAXI;
        std::vector<uint64_t> alpha(cnt, 3), scale(cnt, 1);
        // candidates (c, q) = (1, 3), (2, 5), (3, 7), ...: a batch is retried with the
        // next candidate of each failing instance (the flag is per batch)
        for (int attempt = 0;; attempt++) {
            if (attempt >= 64) return pm_fail(ctx, PM_EUNSUPPORTED, "no usable geometric progression found");
            int flag = 0;
            CKI(res_batch(ctx, cnt, primes + i0, alpha.data(), scale.data(), dxf, dyf, (const u64 *)f + i0 * nf, dxg, dyg,
                          (const u64 *)g + i0 * ng, (u64 *)R + i0 * N, &flag));
            if (!flag) break;
            if (cnt > 1) {   // find which instances fail by running them alone
                bool any = false;
                for (int i = 0; i < cnt; i++) {
                    int fl = 0;
                    CKI(res_batch(ctx, 1, primes + i0 + i, &alpha[i], &scale[i], dxf, dyf, (const u64 *)f + (i0 + i) * nf, dxg,
                                  dyg, (const u64 *)g + (i0 + i) * ng, (u64 *)R + (i0 + i) * N, &fl));
                    if (fl) { alpha[i] += 2; scale[i] += 1; any = true; }
                }
                if (!any) break;
            } else {
                alpha[0] += 2;
                scale[0] += 1;
            }
        }
    }
    return PM_OK;
}

// ------------------------------------------------------------------ Villard variant, host
// One prime, points c q^l.  flag bits: 1 points not distinct, 2 a leading coefficient
// vanishes at an H point, 4 Res vanishes at an H point, 16 det Q vanishes at the first
// point (all four: try the next (c, q)); 8 det Q is not a multiple of Res (input not generic).
static int vil_one(pm_ctx *ctx, uint64_t p, uint64_t q, uint64_t c, int dxf, int dyf, const u64 *f, int dxg, int dyg,
                   const u64 *g, int m, u64 *R, int *h_flag)
{
    const int nu = dyf + dyg, d = dxf > dxg ? dxf : dxg, E = d + 1, J = dyf + dyg + 2, dmax = dyf > dyg ? dyf : dyg;
    const int64_t D = (int64_t)dxf * dyg + (int64_t)dxg * dyf, N = D + 1;
    const int64_t delta = 2 * (int64_t)((nu + m - 1) / m) * d + 1;
    const int64_t NP = N > delta ? N : delta;                   // points covered by the tables
    const int64_t NE = NP + (E > delta + 1 ? E : delta + 1);    // chirp length bound
    const int64_t m2 = 2 * m;
    // buffers (stream-ordered; pm_intbasis below owns the driver arena)
    const size_t words = 4 * (size_t)NE + (size_t)J * E + 2 * (size_t)J * delta + (size_t)m2 * m * delta + delta +
                         (size_t)m2 * m2 * (delta + 1) + (size_t)m * m * (delta + 1) + (delta + 1) +
                         (size_t)m * m * N + 9 * (size_t)N + 64;
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, words * 8 + 32 * 256, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return pm_fail(ctx, PM_ENOMEM, "Villard resultant workspace allocation failed");
    }
    size_t used = 0;
    auto A = [&](size_t n) { u64 *r = (u64 *)(buf + used); used += (n * 8 + 255) & ~size_t(255); return r; };
    ResPack pk;
    memset(&pk, 0, sizeof(pk));
    pk.count = 1; pk.dxf = dxf; pk.dyf = dyf; pk.dxg = dxg; pk.dyg = dyg;
    pk.E = E; pk.J = J;
    ResInst &I = pk.in[0];
    I.p = p;
    I.pn = mont_pn(p);
    I.one = (uint64_t)(((unsigned __int128)1 << 64) % p);
    I.r2 = (uint64_t)((unsigned __int128)I.one * I.one % p);
    I.qm = (uint64_t)((unsigned __int128)(q % p) * I.one % p);
    I.qim = (uint64_t)((unsigned __int128)host_powmod(q % p, p - 2, p) * I.one % p);
    I.cm = (uint64_t)((unsigned __int128)(c % p) * I.one % p);
    I.cim = (uint64_t)((unsigned __int128)host_powmod(c % p, p - 2, p) * I.one % p);
    I.f = f; I.g = g; I.R = R;
    I.qp = A(NE); I.h = A(NE); I.hinv = A(NE); I.Hb = A(NE);
    I.Ua = A((size_t)J * E); I.S = A((size_t)J * delta); I.Vt = A((size_t)J * delta);
    u64 *Eip = A((size_t)m2 * m * delta), *resv = A(delta), *Pb = A((size_t)m2 * m2 * (delta + 1));
    u64 *Ua2 = A((size_t)m * m * (delta + 1)), *ue = A(delta + 1), *S2 = A((size_t)m * m * N);
    I.v = A(N); I.w = A(N); I.winv = A(N); I.Va = A(N); I.Eb = A(N); I.Cp = A(N); I.Ur = A(N); I.Y = A(N);
    u64 *sc = A(8);
    pk.flag = (int *)A(8);
    int rc = PM_OK;
    do {
        if ((rc = pm_cuda(ctx, cudaMemsetAsync(pk.flag, 0, sizeof(int), ctx->stream), "flag"))) break;
        // chirp tables for every length below, distinctness of the NP points
        ResPack pt = pk;
        pt.N = (int)NP; pt.NE = (int)NE;
        int tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_res_powers<<<(int)((NE + 255) / 256 < 1024 ? (NE + 255) / 256 : 1024), 256, 0, ctx->stream>>>(pt);
        // 1. f, g at the delta points (chirp middle product), point-major Montgomery values
        ResPack pe = pk;
        pe.N = (int)delta; pe.NE = (int)(delta + E - 1);
        k_res_prep_eval<<<(J * E + 255) / 256, 256, 0, ctx->stream>>>(pe);
        ctx->launches += 2;
        stage_end(ctx, tok);
        if ((rc = pm_cuda(ctx, cudaGetLastError(), "Villard prep"))) break;
        {
            ProdReq r1;
            r1.p = p; r1.w = 8; r1.m = J; r1.n = 1; r1.k = 1;
            r1.A = I.Ua; r1.dA = E; r1.sA = E; r1.B = I.Hb; r1.dB = delta + E - 1; r1.sB = delta + E - 1;
            r1.off = E - 1; r1.len = delta; r1.C = I.S; r1.sC = delta;
            r1.lg = ceil_log2((int64_t)E - 1 + delta);
            if (r1.lg < 4) r1.lg = 4;
            if ((rc = prod_batch(ctx, &r1, 1))) break;
        }
        tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_res_eval_finish<<<1024, 256, 0, ctx->stream>>>(pe);
        // 2. H(alpha_l) and Res(alpha_l) by the extended Euclidean algorithm, one warp per point
        const size_t smv = (size_t)VIL_WARPS * 8 * (dmax + 2) * 8;
        if (smv > 48 * 1024) cudaFuncSetAttribute(k_vil_xgcd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv);
        k_vil_xgcd<<<(int)((delta + VIL_WARPS - 1) / VIL_WARPS), 32 * VIL_WARPS, smv, ctx->stream>>>(pe, dmax, m, Eip,
                                                                                                     resv);
        ctx->launches += 2;
        stage_end(ctx, tok);
        if ((rc = pm_cuda(ctx, cudaGetLastError(), "Villard Euclid"))) break;
        if ((rc = pm_cuda(ctx, cudaMemcpyAsync(h_flag, pk.flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
                          "flag")))
            break;
        if ((rc = pm_cuda(ctx, cudaStreamSynchronize(ctx->stream), "flag sync"))) break;
        if (*h_flag) break;
        // 3. interpolant basis of [H; -I] at the delta points (Algorithm 5); Q = its top-left block
        std::vector<int64_t> s0(m2, 0), rdeg(m2, 0);
        if ((rc = pm_intbasis(ctx, p, (int)m2, m, Eip, delta, c % p, q % p, s0.data(), Pb, rdeg.data()))) break;
        int64_t LQ = 1;
        for (int i = 0; i < m; i++) LQ = rdeg[i] + 1 > LQ ? rdeg[i] + 1 : LQ;
        if (LQ > delta + 1) LQ = delta + 1;
        // 4. det Q at the N points c q^l: chirp evaluation of the m^2 entries, a determinant per point
        ResPack pq = pk;
        pq.N = (int)N;
        tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_vil_uvec<<<(int)((LQ + 255) / 256), 256, 0, ctx->stream>>>(pq, ue, (int)LQ);
        k_vil_prep_q<<<(int)(((int64_t)m * m * LQ + 255) / 256 < 4096 ? ((int64_t)m * m * LQ + 255) / 256 : 4096), 256,
                       0, ctx->stream>>>(pq, Pb, delta + 1, m, ue, Ua2, (int)LQ);
        ctx->launches += 2;
        stage_end(ctx, tok);
        if ((rc = pm_cuda(ctx, cudaGetLastError(), "Villard Q prep"))) break;
        {
            ProdReq r2;
            r2.p = p; r2.w = 8; r2.m = m * m; r2.n = 1; r2.k = 1;
            r2.A = Ua2; r2.dA = LQ; r2.sA = LQ; r2.B = I.Hb; r2.dB = N + LQ - 1; r2.sB = N + LQ - 1;
            r2.off = LQ - 1; r2.len = N; r2.C = S2; r2.sC = N;
            r2.lg = ceil_log2(LQ - 1 + N);
            if (r2.lg < 4) r2.lg = 4;
            if ((rc = prod_batch(ctx, &r2, 1))) break;
        }
        tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_vil_det<<<(int)((N + 127) / 128), 128, 0, ctx->stream>>>(pq, S2, m, I.v);
        k_vil_norm<<<1, 32, 0, ctx->stream>>>(pq, resv, I.v, sc);
        k_vil_scale<<<(int)((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024), 256, 0, ctx->stream>>>(
            pq, resv, sc, I.v, (int)(delta < N ? delta : N));
        ctx->launches += 3;
        stage_end(ctx, tok);
        if ((rc = pm_cuda(ctx, cudaGetLastError(), "Villard det"))) break;
        if ((rc = pm_cuda(ctx, cudaMemcpyAsync(h_flag, pk.flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
                          "flag")))
            break;
        if ((rc = pm_cuda(ctx, cudaStreamSynchronize(ctx->stream), "flag sync"))) break;
        if (*h_flag) break;
        // 5. interpolation at the N points (as in the direct method)
        tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_res_wscan<<<1, 1024, 0, ctx->stream>>>(pq);
        k_res_interp1<<<(int)((N + 255) / 256), 256, 0, ctx->stream>>>(pq);
        ctx->launches += 2;
        stage_end(ctx, tok);
        if ((rc = pm_cuda(ctx, cudaGetLastError(), "Villard interp"))) break;
        ProdReq ri;
        ri.p = p; ri.w = 8; ri.m = 1; ri.n = 1; ri.k = 1;
        ri.dA = N; ri.sA = N; ri.dB = N; ri.sB = N; ri.off = 0; ri.len = N; ri.sC = N;
        ri.lg = ceil_log2(2 * N - 1);
        if (ri.lg < 4) ri.lg = 4;
        ri.A = I.Va; ri.B = I.Eb; ri.C = I.Cp;
        if ((rc = prod_batch(ctx, &ri, 1))) break;
        tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_res_interp2<<<(int)((N + 255) / 256), 256, 0, ctx->stream>>>(pq);
        ctx->launches++;
        stage_end(ctx, tok);
        ri.A = I.Ur; ri.B = I.Eb; ri.C = I.Y;
        if ((rc = prod_batch(ctx, &ri, 1))) break;
        tok = stage_begin(ctx, PM_STAGE_OTHER);
        k_res_interp3<<<(int)((N + 255) / 256), 256, 0, ctx->stream>>>(pq);
        ctx->launches++;
        stage_end(ctx, tok);
        rc = pm_cuda(ctx, cudaGetLastError(), "Villard interp");
    } while (0);
    cudaFreeAsync(buf, ctx->stream);
    return rc;
}

extern "C" int bivariate_resultant_villard(pm_ctx *ctx, int nprimes, const uint64_t *primes, int dxf, int dyf,
                                           const void *f, int dxg, int dyg, const void *g, int m, void *R)
{
    if (!ctx) return PM_EINVAL;
    if (nprimes < 1 || !primes || !f || !g || !R) return pm_fail(ctx, PM_EINVAL, "bad arguments");
    if (dxf < 0 || dxg < 0 || dyf < 1 || dyg < 1) return pm_fail(ctx, PM_EINVAL, "need dyf, dyg >= 1 and dxf, dxg >= 0");
    if (dxf == 0 && dxg == 0) return pm_fail(ctx, PM_EINVAL, "need an x-degree >= 1");
    if (dyf > 2047 || dyg > 2047) return pm_fail(ctx, PM_EUNSUPPORTED, "y-degree above 2047");
    if (m <= 0) {   // ceil(n^0.4) for the partial degree n (Sec. 5.2)
        const int n = std::max(std::max(dxf, dxg), std::max(dyf, dyg));
        m = 1;
        while (std::pow((double)m, 2.5) < (double)n) m++;
    }
    m = std::min(m, std::min(dyf, dyg));
    if (m > VIL_MMAX) return pm_fail(ctx, PM_EUNSUPPORTED, "block size m above 16");
    const int nu = dyf + dyg, d = std::max(dxf, dxg);
    const int64_t D = (int64_t)dxf * dyg + (int64_t)dxg * dyf, N = D + 1;
    const int64_t delta = 2 * (int64_t)((nu + m - 1) / m) * d + 1;
    const int64_t NP = std::max(N, delta);
    if (2 * N - 1 > (1 << PM_MAX_LOG2L) || NP + delta + d + 1 > (1 << PM_MAX_LOG2L) || delta + 1 > (1 << PM_MAX_LOG2L))
        return pm_fail(ctx, PM_EINVAL, "resultant degree too large for the transforms");
    for (int i = 0; i < nprimes; i++)
        if (!(primes[i] & 1) || primes[i] < 3 || primes[i] >= (1ull << 62) || primes[i] <= (uint64_t)(2 * NP))
            return pm_fail(ctx, PM_EINVAL, "each prime must be odd, below 2^62 and above twice the point count");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    const size_t nf = (size_t)(dyf + 1) * (dxf + 1), ng = (size_t)(dyg + 1) * (dxg + 1);
    for (int i = 0; i < nprimes; i++) {
        uint64_t q = 3, c = 1;
        for (int attempt = 0;; attempt++) {
            if (attempt >= 64) return pm_fail(ctx, PM_EUNSUPPORTED, "no usable geometric progression found");
            int flag = 0;
            CKI(vil_one(ctx, primes[i], q, c, dxf, dyf, (const u64 *)f + i * nf, dxg, dyg, (const u64 *)g + i * ng, m,
                        (u64 *)R + (size_t)i * N, &flag));
            if (!flag) break;
            if (flag & 8) return pm_fail(ctx, PM_EUNSUPPORTED, "input not generic for the Villard variant");
            q += 2;
            c += 1;
        }
    }
    return PM_OK;
}
