// common.cuh -- shared device arithmetic and job descriptors of libpmat.
//
// Modular arithmetic is written from the published methods:
//  * Shoup's precomputed-quotient multiplication (V. Shoup, NTL; "Harvey,
//    Faster arithmetic for number-theoretic transforms", 2014, Sec. 2): for a
//    constant w < q and w' = floor(w 2^32 / q), x w mod q lies in [0, 2q).
//  * Harvey's lazy butterflies (same paper, Algorithms 4 and 5): values are
//    kept in [0, 2q) (Gentleman-Sande, forward) or [0, 4q) (Cooley-Tukey,
//    inverse), which needs q < 2^30.
//  * Barrett reduction (P. Barrett, CRYPTO 1986) with mu = floor(2^64 / p).
//  * Montgomery multiplication (P. L. Montgomery, Math. Comp. 1985) with
//    R = 2^64 for odd p < 2^63.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef uint32_t u32;
typedef uint64_t u64;
typedef int64_t i64;

#define PM_MAX_LOG2L 20      // largest transform: 2^20 points
#define PM_LB_LOG2 14        // transforms up to 2^14 points run in one CTA
#define PM_MAXJ 32           // job descriptors per launch
#define PM_MAXK 6            // CRT primes per product

// ---------------------------------------------------------------- 32-bit
__device__ __forceinline__ u32 shoup_mul(u32 x, u32 w, u32 ws, u32 q)
{
    return x * w - __umulhi(x, ws) * q;   // in [0, 2q) for any x < 2^32
}
__device__ __forceinline__ u32 csub(u32 x, u32 m) { return min(x, x - m); }  // x < 2m -> [0,m)

// Gentleman-Sande (DIF) butterfly, inputs and outputs in [0, 2q):
// (X, Y) -> (X + Y, (X - Y) w)
__device__ __forceinline__ void bfly_dif(u32 &X, u32 &Y, uint2 w, u32 q, u32 q2)
{
    u32 s = X + Y;
    u32 d = X - Y + q2;
    X = csub(s, q2);
    Y = shoup_mul(d, w.x, w.y, q);
}
// Cooley-Tukey (DIT) butterfly, inputs and outputs in [0, 4q):
// (X, Y) -> (X + Y w, X - Y w)
__device__ __forceinline__ void bfly_dit(u32 &X, u32 &Y, uint2 w, u32 q, u32 q2)
{
    u32 x = csub(X, q2);
    u32 t = shoup_mul(Y, w.x, w.y, q);
    X = x + t;
    Y = x - t + q2;
}

// Per-prime constants carried by every job.
struct PrimeDev {
    u32 q, q2;         // q, 2q
    u32 r32, r32s;     // 2^32 mod q, Shoup companion
    u32 ones;          // floor(2^32 / q): Shoup companion of 1
    u32 linv, linvs;   // L^-1 mod q for the job's transform length, companion
    const uint2 *twf;  // twf[h + r] = (omega_{2h}^r, companion), h = 1, 2, 4, ...
    const uint2 *twi;  // inverse roots
};

// x mod q in [0, q) for x < 2^64 (x = hi 2^32 + lo, both folded by Shoup)
__device__ __forceinline__ u32 reduce64(u64 x, const PrimeDev &P)
{
    u32 hi = (u32)(x >> 32), lo = (u32)x;
    u32 s = shoup_mul(hi, P.r32, P.r32s, P.q) + shoup_mul(lo, 1u, P.ones, P.q);  // < 4q
    return csub(csub(s, P.q2), P.q);
}

// ---------------------------------------------------------------- 64-bit
__device__ __forceinline__ u64 shoup_mul64(u64 x, u64 w, u64 ws, u64 p)
{
    return x * w - __umul64hi(x, ws) * p;  // in [0, 2p), p < 2^63
}
__device__ __forceinline__ u64 csub64(u64 x, u64 m) { return x >= m ? x - m : x; }
__device__ __forceinline__ u64 barrett64(u64 x, u64 p, u64 mu)
{
    u64 r = x - __umul64hi(x, mu) * p;     // in [0, 2p)
    return csub64(r, p);
}
// Montgomery product a b R^-1 mod p for a, b < p, p odd < 2^63, pn = -p^-1 mod 2^64
__device__ __forceinline__ u64 mont_mul(u64 a, u64 b, u64 p, u64 pn)
{
    u64 lo = a * b, hi = __umul64hi(a, b);
    u64 m = lo * pn;
    u64 r = hi + __umul64hi(m, p) + (lo != 0);
    return csub64(r, p);
}
// Montgomery reduction of a 128-bit T = hi 2^64 + lo < p 2^64: T 2^-64 mod p
__device__ __forceinline__ u64 redc128(u64 hi, u64 lo, u64 p, u64 pn)
{
    u64 m = lo * pn;
    u64 r = hi + __umul64hi(m, p) + (lo != 0);
    return csub64(r, p);
}
// (hi, lo) <- (hi, lo) - b y, plus p 2^64 when that goes negative: keeps T in [0, p 2^64)
__device__ __forceinline__ void sub128_mod(u64 &hi, u64 &lo, u64 b, u64 y, u64 p)
{
    const u64 l2 = b * y, h2 = __umul64hi(b, y);
    const u64 b1 = lo < l2;
    const bool neg = hi < h2 || (hi == h2 && b1);
    lo -= l2;
    hi = hi - h2 - b1 + (neg ? p : 0);
}
// Montgomery forms with one reduction: (a x - b y) 2^-64 mod p and
// (a x - b y - c z) 2^-64 mod p, for operands below p < 2^62
__device__ __forceinline__ u64 mont_msub(u64 a, u64 x, u64 b, u64 y, u64 p, u64 pn)
{
    u64 lo = a * x, hi = __umul64hi(a, x);
    sub128_mod(hi, lo, b, y, p);
    return redc128(hi, lo, p, pn);
}
__device__ __forceinline__ u64 mont_msub2(u64 a, u64 x, u64 b, u64 y, u64 c, u64 z, u64 p, u64 pn)
{
    u64 lo = a * x, hi = __umul64hi(a, x);
    sub128_mod(hi, lo, b, y, p);
    sub128_mod(hi, lo, c, z, p);
    return redc128(hi, lo, p, pn);
}
__device__ __forceinline__ u64 add64(u64 a, u64 b, u64 p) { u64 s = a + b; return s >= p ? s - p : s; }
__device__ __forceinline__ u64 sub64(u64 a, u64 b, u64 p) { return a >= b ? a - b : a + (p - b); }

// ---------------------------------------------------------------- jobs
// Forward transform of `count` blocks of 2^lg points.  Block e reads
// src + e*src_stride (src_len values, zero beyond) and writes dst + e*dst_stride.
// src_mode: 0 = u32 already in [0, 2q), 4 = user u32 in [0,p), 8 = user u64; with
// PM_FWD_TWIST added, the job is the second half of a 2^(LG+1)-point transform of at most 2^LG
// coefficients: the radix-2 stage over the halves maps (x_i, 0) to (x_i, x_i w^i), w of
// order 2^(LG+1), so coefficient i is multiplied by w^i on load and the 2^LG-point block
// transform gives the odd half directly (the even half is the plain block transform).
#define PM_FWD_TWIST 0x100
// grp: 0, or (G << 8) | g for job g of an interleave group of G consecutive jobs in the pack (the
// same source modulo G primes, equal block counts): the group's blocks alternate between its
// jobs, so the G CTAs that read the same source entries run side by side and all but the first
// find them in L2.
struct FwdJob {
    const void *src;
    u32 *dst;
    i64 src_stride, dst_stride;
    int src_len, src_mode, count, grp;
    PrimeDev P;
};
// Inverse transform.  dst_mode: 0 = u32 staging (unscaled, all points),
// 1 = u32 residues (scaled, [0,q)), 4 / 8 = final u32 / u64 values (p = q).
// Points x in [out_off, out_off + out_len) are written to dst + e*dst_stride + (x - out_off).
struct InvJob {
    const u32 *src;
    void *dst;
    i64 src_stride, dst_stride;
    int out_off, out_len, dst_mode, count;
    PrimeDev P;
};
// Column pass for transforms longer than 2^PM_LB_LOG2: the top stages act on
// columns c + j 2^PM_LB_LOG2 of each entry.
struct ColJob {
    const void *src;   // fwd: user/u32 source (mode as FwdJob); inv: u32
    void *dst;         // fwd: u32 [entry][L]; inv: as InvJob
    i64 src_stride, dst_stride;
    int src_len, mode, count, out_off, out_len, _pad;
    PrimeDev P;
};
// Pointwise products at every transform point: C_j = A_j B_j mod q.
// The CUDA-core kernel's block plan (pw_plan_tile): block tiles of bi x bk thread tiles of
// 4 x cw outputs (nbk tiles across k, ntile per transform point group), the inner
// dimension staged lc <= 32 at a time and split into ns contiguous slices; mg_* are
// division magics ceil(2^31 / d) for d = lc, the last chunk, the tile width and the
// last tile's width; smem = dynamic shared memory in bytes.
struct PwJob {
    const u32 *A, *B;
    u32 *C;
    int m, n, k, L;
    int bi, bk, ns, lc, nbk, ntile, smem;
    int cw;             // columns per thread tile: 8 or 4
    u32 mg_lc, mg_lt, mg_cb, mg_ct;
    PrimeDev P;
};
// Garner CRT of K residue planes into values mod p.
struct CrtJob {
    const u32 *res;     // [K][count], count = entries * len
    void *dst;          // entry e, position t -> dst[e * dst_stride + t], u32 or u64
    i64 count, len, dst_stride;
    int K, w;
    u64 p, mu;          // p and floor(2^64/p)
    u32 q[PM_MAXK];
    u32 c[PM_MAXK][PM_MAXK], cs[PM_MAXK][PM_MAXK];   // q_j^-1 mod q_i, companions
    u64 qm[PM_MAXK], qms[PM_MAXK];                   // q_i mod p, Shoup-64 companions
    int small_p;        // p <= 2^30: residues need a reduction mod p
    // explicit CRT sum (mode 1, odd p): X = sum_i t_i M_i - k M with M_i = M / q_i,
    // t_i = r_i M_i^-1 mod q_i and k = floor(sum_i t_i / q_i); mode 0: Garner
    int mode;
    u32 gi[PM_MAXK], gis[PM_MAXK];                   // M_i^-1 mod q_i, Shoup companions
    u32 W[PM_MAXK];                                  // floor(2^59 / q_i)
    u64 Cm[PM_MAXK + 1];                             // (M_i mod p) 2^64 mod p; (-M mod p) 2^64 mod p last
    u64 pn;                                          // -p^-1 mod 2^64
};

template <typename J>
struct JobPack {
    int njobs;
    int blk_start[PM_MAXJ + 1];
    J jobs[PM_MAXJ];
};

// ---------------------------------------------------------------- launchers
// All return cudaError_t of the launch; `launches` is incremented per launch.
cudaError_t launch_twiddles(uint2 *twf, uint2 *twi, u32 q, const u32 *roots_f, const u32 *roots_i,
                            int maxlog, cudaStream_t st, long long *launches);
cudaError_t launch_ntt_fwd_block(const JobPack<FwdJob> &pk, int lg, cudaStream_t st, long long *launches);
cudaError_t launch_ntt_inv_block(const JobPack<InvJob> &pk, int lg, cudaStream_t st, long long *launches);
cudaError_t launch_ntt_fwd_cols(const JobPack<ColJob> &pk, int lg, cudaStream_t st, long long *launches);
cudaError_t launch_ntt_inv_cols(const JobPack<ColJob> &pk, int lg, cudaStream_t st, long long *launches);
// 2^15-point inverse transforms, one CTA per entry (jobs as for launch_ntt_inv_block, src stride 2^15).
cudaError_t launch_ntt_inv_pair(const JobPack<InvJob> &pk, cudaStream_t st, long long *launches);
// A whole product modulo an NTT prime q = p in one CTA (small.cu): A (m x n x dA), B (n x k x dB)
// and C (m x k x len, len = dA + dB - 1) contiguous in the caller's width w; L = 2^lg points,
// n <= 16 (the pointwise sums stay below 2^64), small_product_smem(...) bytes of shared memory.
struct SmallJob {
    const void *A, *B;
    void *C;
    int w, m, n, k, dA, dB, len, lg;
    PrimeDev P;
};
size_t small_product_smem(int m, int n, int k, int lg);
cudaError_t launch_small_product(const SmallJob &J, cudaStream_t st);
// every job of the pack has the same thread-tile width (cw); cudaErrorInvalidValue otherwise
cudaError_t launch_pointwise(const JobPack<PwJob> &pk, cudaStream_t st, long long *launches);
int pw_plan(PwJob &j);
int pw_plan_tile(PwJob &j, int bi, int bk, int cw);
int pw_tiles(const PwJob &j, int *bi_out, int *bk_out, int max, int cw, long long *cost0 = nullptr);
cudaError_t launch_pointwise_sn(const JobPack<PwJob> &pk, cudaStream_t st, long long *launches);
bool pws_supported(const PwJob &j);
int pws_blocks(const PwJob &j);
cudaError_t launch_pointwise_mv(const JobPack<PwJob> &pk, cudaStream_t st, long long *launches);
bool pwv_supported(const PwJob &j);
int pwv_blocks(const PwJob &j);
cudaError_t launch_crt(const JobPack<CrtJob> &pk, cudaStream_t st, long long *launches);
void crt_setup(CrtJob &J, const u32 *q, int K, uint64_t p);
// Host set-up of the NTT primes (primes.cu).
uint64_t host_mulmod(uint64_t a, uint64_t b, uint64_t p);
uint64_t host_powmod(uint64_t a, uint64_t e, uint64_t p);
bool ntt_is_prime32(uint64_t n);                          // deterministic below 2^32
void ntt_roots(uint32_t q, uint32_t *rf, uint32_t *ri);   // [PM_MAX_LOG2L + 1]: 2^l-th roots and inverses (0: none)
int ntt_prime_table(uint32_t *out, int maxk);             // CRT primes c 2^20 + 1 < 2^30, largest first
cudaError_t launch_pointwise_tc(const JobPack<PwJob> &pk, int *status, cudaStream_t st, long long *launches,
                                int withhold = 0);
bool tc_supported(const PwJob &j);
int tc_blocks(const PwJob &j);
int fwd_block_threads(int lg);
int blocks_per_entry_cols(int lg);
int crt_blocks(const CrtJob &j);
