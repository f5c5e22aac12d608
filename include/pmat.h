/*
 * pmat.h -- C ABI of libpmat: exact univariate polynomial-matrix arithmetic
 * over F_p on one GB300 GPU (sm_103a).
 *
 * Operations (Hyun, Neiger, Schost, "Implementations of efficient univariate
 * polynomial matrix algorithms and application to bivariate resultants",
 * ISSAC 2019):
 *   pmat_mul, pmat_mul_trunc      Sec. 2, "Polynomial matrix multiplication"
 *   pmat_middle_product           Sec. 2, "Polynomial multiplication":
 *                                 MiddleProduct(F, G, c, d)
 *   pmat_mul_vdm                  the same by Vandermonde-matrix evaluation and
 *                                 interpolation (Sec. 2, dense products on the
 *                                 tensor cores)
 *   pmat_mul_batched              many independent products in one call
 *   pmat_mul_host                 the same product from and to host memory,
 *                                 copies overlapped with the stages
 *   pm_basis                      Sec. 3, Algorithm 3 (PM-Basis) over
 *                                 Algorithms 1-2 (M-Basis-1, M-Basis)
 *   pm_intbasis                   Sec. 3, Algorithm 5 (PM-IntBasis) over
 *                                 Algorithm 4 (M-IntBasis), geometric points
 *   bivariate_resultant           Sec. 5.2, resultant of bivariate
 *                                 polynomials (the direct method)
 *   bivariate_resultant_villard   Sec. 5.2, the same by the variant of
 *                                 Algorithm 6 (values of a block of the
 *                                 inverse Sylvester matrix, PM-IntBasis)
 *   pmat_inv_trunc                Sec. 4, "Linear system solving": the
 *                                 truncated inverse A^-1 mod x^t by matrix
 *                                 Newton iteration
 *   pmat_solve_series             Sec. 4, lifting: A^-1 b mod x^N by Dixon's
 *                                 algorithm over the truncated inverse
 *   pmat_inv_slices               Sec. 4, high-order lifting: slices of A^-1
 *                                 at degrees around 2^i (d - 1)
 *   pmat_solve_series_hol         Sec. 4, high-order lifting: A^-1 b mod x^N
 *                                 from the slices
 *   pmat_solve                    Sec. 4, lifting solver: (u, f) with
 *                                 A u = f b by Dixon's lifting and vector
 *                                 rational reconstruction (PM-Basis)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * * A polynomial matrix X with r x c entries of length len is one contiguous
 *   array in DEVICE memory, entry-major and row-major: coefficient t of entry
 *   (i, j) is X[(i*c + j)*len + t].
 * * Element width w is 4 (uint32_t, requires p < 2^32) or 8 (uint64_t,
 *   requires p < 2^62).  Inputs must be reduced into [0, p); outputs are.
 * * p >= 2.  Products are ring operations and accept any such p; pm_basis,
 *   pm_intbasis and pmat_inv_trunc need p prime (not checked, as for a field
 *   type), 2 included; the resultants need p odd (checked).
 * * The caller owns every input and output buffer; outputs must not alias
 *   inputs.  The context owns its workspace, twiddle tables and plans.
 * * All calls are asynchronous and ordered on the context's stream.  A
 *   status returned by a call covers argument checking and launch errors;
 *   pm_sync() waits for the stream and returns the first deferred error.
 * * Every function returns an int status (PM_OK = 0 or a PM_E* code below)
 *   and never throws.  pm_last_error() gives a message for the last failure.
 * * Maximum transform length is 2^20 points: a product whose result needs
 *   more returns PM_EINVAL.
 */
#ifndef PMAT_H
#define PMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PM_OK = 0,
    PM_EINVAL = 1,       /* bad argument (dimension, length, modulus, width) */
    PM_EDOMAIN = 2,      /* an input coefficient is not in [0, p) (debug check), or
                            A(0) is singular in pmat_inv_trunc / pmat_solve_series /
                            pmat_inv_slices (deferred, pm_sync) */
    PM_ENOMEM = 3,       /* device workspace allocation failed */
    PM_ECUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    PM_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
    PM_EUNSUPPORTED = 6, /* valid request outside what this build handles */
    PM_ESCRATCH = 7      /* request needs more than the fixed scratch array of pmat_mul_noalloc */
};

typedef struct pm_ctx pm_ctx;

/* Option keys for pm_set_option. */
enum {
    PM_OPT_POINTWISE = 1,   /* 0 = auto (the cost-model rules, or the form pm_tune_product
                               recorded for the shape), 1 = CUDA-core 64-bit products,
                               2 = tensor-core digit products, four points per MMA, where
                               m, n, k <= 32 (CUDA cores elsewhere), 3 = tensor-core dense
                               products per point where m >= 64 (CUDA cores elsewhere),
                               4 = CUDA-core staged products in 4 x 4 thread tiles (every
                               shape) */
    PM_OPT_THRESHOLD = 2,   /* PM-Basis threshold T (>= 1): M-Basis when order <= T;
                               default 32 (Sec. 3, "Interpolant bases") */
    PM_OPT_DEBUG_CHECKS = 3, /* 1 = check inputs are in [0, p) (PM_EDOMAIN) */
    PM_OPT_STAGE_TIMING = 4, /* 1 = record CUDA events around every stage (see pm_stage_times) */
    PM_OPT_LEAF_CLUSTER = 5, /* PM-Basis / PM-IntBasis leaves: 1 = a cluster of up to 16 CTAs with
                                the basis in shared memory (default), 0 = one CTA with the basis
                                in global memory */
    PM_OPT_HOST_CHUNKS = 6,  /* pmat_mul_host output chunks: 0 (default) = one, the fastest
                                for calls in a row (a call's download overlaps the next call);
                                N >= 1 = N chunks of output entries whose inverse transforms,
                                recombination and copy back are pipelined, for the latency of
                                a call on its own */
    PM_OPT_TEST_WITHHOLD_MMA = 7 /* test hook for the bounded device waits: 1 = the tensor-core
                                pointwise kernel issues no MMA for its first point in block 0,
                                so that block's wait gives up after 1024 polls; the call's
                                output is undefined and pm_sync returns PM_ETIMEOUT.  Nothing
                                is in flight when the wait gives up.  Default 0. */
};

/* Stages reported by pm_stage_times. */
enum {
    PM_STAGE_FWD = 0,        /* forward transforms (reduction mod q fused) */
    PM_STAGE_POINTWISE = 1,  /* pointwise products at the transform points */
    PM_STAGE_INV = 2,        /* inverse transforms (scaling and slice fused) */
    PM_STAGE_CRT = 3,        /* multi-prime recombination */
    PM_STAGE_LEAF = 4,       /* PM-Basis leaves (Algorithm 2 on the device) */
    PM_STAGE_OTHER = 5,      /* driver kernels: shifts, scalings, Euclid */
    PM_NSTAGES = 8
};

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * owned by the caller (kept, not destroyed; cudaStreamLegacy selects the
 * legacy default stream), or NULL for a context-owned non-blocking stream.
 * *ctx receives the handle.  Returns PM_EINVAL on a bad device, PM_ECUDA on a
 * runtime failure. */
int pm_create(pm_ctx **ctx, int device, void *cuda_stream);

/* Destroy a context: synchronises its stream, frees its device memory. */
int pm_destroy(pm_ctx *ctx);

/* Set an option (keys above).  PM_EINVAL on an unknown key or bad value. */
int pm_set_option(pm_ctx *ctx, int key, int64_t value);

/* Replace the stream used by later calls (NULL = the context's own). */
int pm_set_stream(pm_ctx *ctx, void *cuda_stream);

/* Wait for all work queued on the context's stream; return the first
 * deferred error (kernel fault, device-side timeout) or PM_OK. */
int pm_sync(pm_ctx *ctx);

/* Message for the last non-OK status on this context (never NULL). */
const char *pm_last_error(pm_ctx *ctx);

/* Number of CUDA kernel launches issued by this context since creation
 * (a diagnostic counter; it includes set-up kernels). */
int64_t pm_kernel_launches(pm_ctx *ctx);

/* Algorithmic work of every product this context ran since creation (or the
 * last reset), whichever entry point or driver issued it: out3[0] = the
 * compulsory bytes (inputs read once, outputs written once), out3[1] = the
 * pointwise modular multiply-adds (primes x transform points x m n k),
 * out3[2] = the NTT butterflies (primes x transforms x (L/2) log2 L).  HOST
 * int64_t[3].  reset != 0 zeroes the counters after reading them. */
int pm_work_counters(pm_ctx *ctx, int64_t *out3, int reset);

/* With PM_OPT_STAGE_TIMING on, every stage of every call is bracketed by
 * CUDA events on the context's stream.  This call synchronises the stream,
 * adds the elapsed times of all stages recorded since the previous call into
 * ms[PM_NSTAGES] and their launch counts into launches[PM_NSTAGES] (host
 * arrays, overwritten), and clears the record.  Either pointer may be NULL. */
int pm_stage_times(pm_ctx *ctx, double *ms, int64_t *launches);

/* C (m x k, length dA+dB-1) = A (m x n, length dA) . B (n x k, length dB)
 * mod p.  Sec. 2, "Polynomial matrix multiplication": evaluation and
 * interpolation at roots of unity; for moduli without suitable roots the
 * product is lifted to Z[x] and taken modulo several NTT primes, then
 * recombined (the "3-primes" approach, with as many primes as the integer
 * coefficients need).  Requires m, n, k, dA, dB >= 1. */
int pmat_mul(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k,
             const void *A, int64_t dA, const void *B, int64_t dB, void *C);

/* pmat_mul with A, B and C in HOST memory (same layouts).  Uploads and
 * downloads run on two streams owned by the context, overlapped with the
 * stages: B and A are transformed as their row chunks land, the pointwise
 * products run once, and the output entries are inverse-transformed,
 * recombined and copied back in chunks, each copy overlapping the next
 * chunk's work.  Consecutive calls overlap too: they alternate between two
 * device staging sets, so a call's download runs during the next call's
 * work, and the next call's upload during this call's.  The context's
 * stream does not wait for the downloads until something needs them: the
 * next device product on the context, pm_sync, pm_set_stream or
 * pm_host_join.  Page-locked (pinned) host buffers are needed for the copies
 * to overlap; pageable ones give the same result.  C is complete after
 * pm_sync() (or after pm_host_join() and the stream's completion), and A, B,
 * C must stay valid until then.  Returns PM_EUNSUPPORTED when the product's
 * device workspace would exceed 16 GB (use pmat_mul on device buffers). */
int pmat_mul_host(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k,
                  const void *A, int64_t dA, const void *B, int64_t dB, void *C);

/* Make the context's stream wait for every download pmat_mul_host has
 * issued, so that work or events recorded on the stream afterwards follow
 * them.  Does not block the host. */
int pm_host_join(pm_ctx *ctx);

/* C (m x k, length t) = A . B mod x^t (Sec. 2; the truncated product used by
 * Newton iteration in Sec. 4, "Linear system solving").  Requires t >= 1;
 * coefficients of degree >= dA+dB-1 are zero. */
int pmat_mul_trunc(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k,
                   const void *A, int64_t dA, const void *B, int64_t dB, int64_t t, void *C);

/* C (m x k, length d) = MiddleProduct(A, B, c, d): the coefficients of
 * degrees c .. c+d-1 of A . B (Sec. 2, "Polynomial multiplication").
 * The paper states it for A of length c and B of length c+d; this entry
 * point also accepts A of length c+1, the case of the PM-Basis residual
 * (Algorithm 3, step 3).  Requires 1 <= dA <= c+1, 1 <= dB <= c+d, d >= 1. */
int pmat_middle_product(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k,
                        const void *A, int64_t dA, const void *B, int64_t dB,
                        int64_t c, int64_t d, void *C);

/* One product of a batch: C_i = A_i . B_i mod p_i, full length dA+dB-1.
 * Descriptors live in HOST memory; the matrices in device memory. */
typedef struct {
    uint64_t p;
    int w, m, n, k;
    const void *A;
    int64_t dA;
    const void *B;
    int64_t dB;
    void *C;
} pmat_desc;

/* `count` independent products (each as pmat_mul) in one call: work of all
 * products is binned by transform length and run by shared launches.  On a
 * bad descriptor returns PM_EINVAL and runs nothing. */
int pmat_mul_batched(pm_ctx *ctx, int count, const pmat_desc *descs);

/* pmat_mul without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * code being captured into a CUDA graph that must hold no allocation nodes,
 * code running under a framework whose pool owns all device memory, or a
 * process with a device-memory budget fixed at start-up.  It computes what
 * pmat_mul computes (same arguments, same result) on the CUDA stream
 * `cuda_stream` (NULL = the legacy default stream) of the CURRENT device, and
 * takes no context.
 * Scratch: one file-scope device array of 64 MiB, held by every GPU that
 * loads the library until the process exits.  A product whose scratch need
 *   K * (2 * al(2^lg * 8) + al(m n 2^lg 4) + al(n k 2^lg 4) + al(m k 2^lg 4))
 *   + (K > 1 or p not an NTT prime ? K * m k (dA+dB-1) * 4 : 0)
 * (2^lg = the transform length >= dA+dB-1, K = the number of NTT primes,
 * al = round up to 256 bytes) exceeds 64 MiB is rejected with PM_ESCRATCH
 * before anything runs.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current), so make
 * that first call before any stream capture.  Every call overwrites the
 * array: calls that overlap on the GPU (several streams or host threads)
 * race and must be serialised by the caller.  Calls no cudaMalloc, cudaFree
 * or other allocating routine.  Returns PM_EINVAL on bad arguments (a length
 * above 2^20 included), PM_EUNSUPPORTED when the product needs more CRT primes
 * than the table holds, PM_ESCRATCH as above, PM_ECUDA on a runtime or launch
 * failure. */
int pmat_mul_noalloc(uint64_t p, int w, int m, int n, int k,
                     const void *A, int64_t dA, const void *B, int64_t dB, void *C,
                     void *cuda_stream);

/* PM-Basis (Sec. 3, Algorithm 3; leaves: Algorithm 2 with Algorithm 1).
 * F: m x n matrix of uint64_t (w = 8) with entries of length lenF in device
 * memory; only F mod x^d is read (requires lenF >= 1; missing coefficients are
 * zero).  shift: HOST int64_t[m].  P: DEVICE output, m x m entries of length
 * d+1, an s-ordered weak Popov approximant basis of (F, d).  rdeg_out: HOST
 * int64_t[m] receiving rdeg_s(P) (this call therefore synchronises the
 * stream).  Requires p prime (p = 2 included: the leaves then work on bits),
 * 1 <= n, 1 <= m, d >= 1. */
int pm_basis(pm_ctx *ctx, uint64_t p, int m, int n, const void *F, int64_t lenF,
             int64_t d, const int64_t *shift, void *P, int64_t *rdeg_out);

/* PM-IntBasis (Sec. 3, "Interpolant bases", Algorithm 5; leaves: Algorithm 4)
 * at the geometric progression of points alpha_l = c q^l, l < sigma.
 * E: DEVICE uint64_t, m x n entries of length sigma, E[(i*n + j)*sigma + l] =
 * entry (i, j) of the matrix E_l attached to alpha_l.  shift: HOST
 * int64_t[m].  P: DEVICE output, m x m entries of length sigma+1, the
 * s-ordered weak Popov interpolant basis with P(alpha_l) E_l = 0 for every l
 * that Algorithm 4 returns (Algorithm 5 returns the same basis).  rdeg_out:
 * HOST int64_t[m] receiving rdeg_s(P) (this call synchronises the stream).
 * The residual of a node (P1 at the second half of the points) is evaluated
 * by a chirp middle product on the product path.  Requires p a prime < 2^62
 * (2 included), c in [0, p), q in [1, p), 1 <= m, n <= 128, sigma >= 1; the points
 * need not be distinct.  Returns PM_EINVAL on bad arguments. */
int pm_intbasis(pm_ctx *ctx, uint64_t p, int m, int n, const void *E, int64_t sigma,
                uint64_t c, uint64_t q, const int64_t *shift, void *P, int64_t *rdeg_out);

/* Res_y(f, g) in F_p[x] for f, g in F_p[x, y] with formal y-degrees dyf,
 * dyg and x-degrees <= dxf, dxg (Sec. 5.2, the direct evaluation /
 * interpolation method).  f: DEVICE uint64_t[(dyf+1)*(dxf+1)] with
 * f[j*(dxf+1) + i] = coefficient of x^i y^j (likewise g).  R: DEVICE
 * uint64_t[nprimes][D+1], D = dxf*dyg + dxg*dyf; instance i is computed
 * modulo primes[i] (HOST array) from f + i*(dyf+1)*(dxf+1) and
 * g + i*(dyg+1)*(dxg+1).  Requires every prime odd and larger than 2(D+1),
 * the leading y-coefficients not identically zero.  Returns PM_EUNSUPPORTED
 * when no usable geometric progression is found. */
int bivariate_resultant(pm_ctx *ctx, int nprimes, const uint64_t *primes,
                        int dxf, int dyf, const void *f, int dxg, int dyg, const void *g,
                        void *R);

/* Res_y(f, g) by the variant of Algorithm 6 in Sec. 5.2 (same layouts, output
 * and conventions as bivariate_resultant).  With P(x) the Sylvester matrix of
 * f, g in y (nu = dyf + dyg, entries of degree <= d = max(dxf, dxg)) and H the
 * top-right m x m block of P^-1 (equations ordered by decreasing power of y):
 * H at delta = 2 ceil(nu / m) d + 1 points c q^l by one extended Euclidean
 * algorithm per point; pm_intbasis on [H; -I] gives H = Q^-1 R (Sec. 3,
 * fraction reconstruction); det Q at the D + 1 points, normalised by Res at
 * the first point, is interpolated.  Requires generic input: every value of
 * the normalised det Q at the delta points is checked against Res there, and
 * a mismatch returns PM_EUNSUPPORTED.  m = 0 takes ceil(n^0.4) for the
 * largest partial degree n (the choice of Sec. 5.2), clamped to min(dyf,
 * dyg); m <= 16.  Requires dyf, dyg >= 1, an x-degree >= 1, every prime odd,
 * below 2^62 and above 2 max(D + 1, delta).  Synchronises the stream. */
int bivariate_resultant_villard(pm_ctx *ctx, int nprimes, const uint64_t *primes,
                                int dxf, int dyf, const void *f, int dxg, int dyg,
                                const void *g, int m, void *R);

/* Truncated inverse (Sec. 4, "Linear system solving", lifting: S = A^-1 mod
 * x^t by matrix Newton iteration).  A: DEVICE n x n matrix with entries of
 * length dA (width w); X: DEVICE output, n x n entries of length t, the unique
 * power series with A.X = I mod x^t.  Newton step k -> 2k: E = coefficients
 * k..2k-1 of A.X_k (a middle product), X_2k = X_k - x^k (X_k . E mod x^k) (a
 * truncated product); the constant term is A(0)^-1 by Gauss-Jordan on the
 * device.  Requires p prime, 1 <= n <= 128, dA >= 1, 1 <= t <= 2^19.  A(0)
 * singular mod p is found on the device: X is then undefined and pm_sync
 * returns PM_EDOMAIN.  Asynchronous; uses the context's driver arena. */
int pmat_inv_trunc(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA,
                   int64_t t, void *X);

/* Power-series solution of A v = b (Sec. 4, "Linear system solving", lifting:
 * Dixon's algorithm).  A: DEVICE n x n matrix, entries of length dA (width w);
 * b: DEVICE n x 1 matrix, entries of length db; v: DEVICE output n x 1, entries
 * of length N, v = A^-1 b mod x^N.  With delta = max(dA, db) and S = A^-1 mod
 * x^delta (pmat_inv_trunc's method): y_i = S r_i mod x^delta, r_{i+1} = (r_i -
 * A y_i) / x^delta from r_0 = b, v = sum_i y_i x^(i delta): ceil(N / delta)
 * truncated products and middle products on the hot path.  Requires p prime,
 * 1 <= n <= 128, dA, db, N >= 1, 2 delta <= 2^20, N <= 2^19.  A(0) singular:
 * v is undefined and pm_sync returns PM_EDOMAIN.  Asynchronous; uses the
 * context's driver arena. */
int pmat_solve_series(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA,
                      const void *b, int64_t db, int64_t N, void *v);

/* Linear system solving by lifting (Sec. 4, "Linear system solving"): the
 * pair (u, f) with A u = f b, f monic of minimal degree.  A: DEVICE n x n
 * matrix of uint64_t, entries of length dA, A(0) invertible mod p; b: DEVICE
 * n x 1, entries of length db.  With D1 = n (dA - 1) and D2 = (n - 1)(dA - 1)
 * + db - 1 (Cramer's bounds on deg f and deg u): v = A^-1 b mod x^N, N = D1 +
 * D2 + 1 (pmat_solve_series), then vector rational reconstruction by an
 * approximant basis of [v^T; -I] at order N for the shift (-D1, -D2, ...,
 * -D2) (pm_basis): its row of non-positive shifted degree is [f, u^T].
 * Outputs: u DEVICE n x 1 of length D2 + 1, f DEVICE length D1 + 1 (zero
 * beyond the degrees), deg_out HOST int64_t[2] = (deg f, deg u; -1 for
 * u = 0).  Synchronises the stream.  Requires p an odd prime < 2^62,
 * 1 <= n <= 127, dA, db >= 1, N <= 2^19.  A(0) singular: PM_EDOMAIN. */
int pmat_solve(pm_ctx *ctx, uint64_t p, int n, const void *A, int64_t dA,
               const void *b, int64_t db, void *u, void *f, int64_t *deg_out);

/* High-order lifting slices (Sec. 4, "Linear system solving": Storjohann's
 * high-order lifting).  A: DEVICE n x n matrix, entries of length dA >= 2 (width
 * w), A(0) invertible; D = dA - 1.  S: DEVICE output, K slices of n x n entries
 * of length 2D + 1: coefficient t of entry (r, c) of slice i, at
 * S[((i n + r) n + c)(2D + 1) + t], is coefficient (2^i - 1) D + t of A^-1.
 * Slice 0 is A^-1 mod x^(2D+1) by Newton iteration; each further slice takes
 * four products of degree about D on the hot path, through the residues
 * E_m = x^-m (I - A (A^-1 mod x^m)) at m = 2^i D - D and 2^i D.  Requires p
 * prime, 1 <= n <= 128, 1 <= K <= 24, 3D + 1 <= 2^20.  A(0) singular: S is
 * undefined and pm_sync returns PM_EDOMAIN.  Asynchronous; uses the driver arena. */
int pmat_inv_slices(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA, int K,
                    void *S);

/* Power-series solution of A v = b by high-order lifting (Sec. 4, "Linear
 * system solving": Storjohann's high-order lifting; the paper's table there
 * sets it against Dixon's lifting).  Same arguments and the same result as
 * pmat_solve_series: v = A^-1 b mod x^N (DEVICE n x 1, entries of length N).
 * Method: with D = dA - 1, X = A^-1 and the residues rho_m(w) = x^-m (w - A
 * (X w mod x^m)), the k slices S_0 .. S_(k-1) of pmat_inv_slices give jumps
 * rho_(K_i), K_i = (2^i + 1) D, each two products (by S_i, then by A); k levels
 * of a binary tree put 2^k residues of b at positions (x + popcount x) D,
 * x < 2^k, at most 2D apart, and S_0 times all of them at once gives v.  k is
 * the least with (2^k + k + 1) D + 1 >= N.  Requires p prime, 1 <= n <= 128,
 * dA >= 2, 1 <= db <= dA, 3D + 1 <= 2^20, N <= 2^19 and 2^k <= 256
 * (PM_EINVAL otherwise).  A(0) singular: v is undefined and pm_sync returns
 * PM_EDOMAIN.  Allocates its buffers on the context's stream (stream-ordered)
 * and uses the driver arena for the slices.  Asynchronous. */
int pmat_solve_series_hol(pm_ctx *ctx, uint64_t p, int w, int n, const void *A, int64_t dA,
                          const void *b, int64_t db, int64_t N, void *v);

/* C (m x k, length dA+dB-1) = A . B mod p by evaluation and interpolation as
 * multiplications by Vandermonde matrices (Sec. 2, "Polynomial matrix
 * multiplication": the variant after Doliskani, Giorgi, Lebreton and Schost,
 * where evaluation / interpolation become products of matrices over F_p of
 * sizes about (d x d) by (d x n^2)).  The points are the powers of w of order L
 * (L = the power of two >= dA + dB - 1, at least 32), so the interpolation
 * matrix is the explicit inverse L^-1 w^(-t j); the evaluations T = X V^T, the
 * interpolation C = T_C W^T are dense products mod p on the tensor cores
 * (fp16 digits of balanced radix 256, fp32 accumulation drained every 64 inner
 * entries), the pointwise products those of pmat_mul.  Same layouts and result
 * as pmat_mul; A, B, C are uint32_t (w = 4).  Requires p a prime below 2^30 with
 * L | p - 1 (an NTT prime for the length, e.g. 998244353) -- PM_EUNSUPPORTED
 * otherwise -- and 1 <= dA, dB <= 2^15, m, n, k >= 1 (PM_EINVAL).  Uses the
 * context's workspace; asynchronous on the context's stream. */
int pmat_mul_vdm(pm_ctx *ctx, uint64_t p, int m, int n, int k, const void *A, int64_t dA, const void *B,
                 int64_t dB, void *C);

/* Autotuner for the pointwise products of a product shape (Sec. 2, "Polynomial
 * matrix multiplication": the n^omega d term).  Times every pointwise form that
 * applies to an m x n . n x k product of lengths dA, dB modulo p -- the
 * CUDA-core form with each of its (up to) four best block tiles by the cost
 * model, for thread tiles of 4 x 8 and of 4 x 4 outputs, the streaming form
 * (n <= 8), the matrix-vector form (k = 1), the tensor-core digit form
 * (m, n, k <= 32) -- over `reps` products each (after
 * one warm-up) on zero inputs (the kernels' time does not depend on the
 * values), and records the fastest in the context: later products of the same
 * (m, n, k, transform length) take it when PM_OPT_POINTWISE is 0 (auto).
 * out: HOST int64_t[5] = form (1 CUDA-core block tile of 4 x 8 thread tiles,
 * 2 tensor-core four points per MMA, 3 streaming, 4 matrix-vector, 5 tensor-core
 * dense products per point, tried where m >= 64, 6 CUDA-core block tile of 4 x 4
 * thread tiles), bi, bk (the block tile of forms 1 and 6, else 0), the
 * winner's pointwise-stage time per product in ns, the number of candidates.
 * Allocates and frees its scratch on the context's stream, synchronises it and
 * discards earlier stage-timing records.  Requires 1 <= reps <= 1000 and the
 * product arguments of pmat_mul; PM_EINVAL otherwise. */
int pm_tune_product(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, int64_t dA, int64_t dB, int reps,
                    int64_t *out);

/* Autotuner for PM-Basis's threshold T (Sec. 3, Algorithm 3: orders <= T run
 * M-Basis at a leaf).  Times pm_basis on seeded pseudo-random F (m x n, order d,
 * uniform shift 0) modulo the odd prime p for T in {8, 16, 32, 64, 128} (those
 * <= d, and 8), `reps` calls each after one warm-up, and sets the context's
 * threshold (PM_OPT_THRESHOLD) to the fastest.  out: HOST int64_t[2] = T, its
 * time per call in ns.  Allocates and frees its scratch on the context's
 * stream and synchronises it.  Requires 1 <= reps <= 100; PM_EINVAL otherwise. */
int pm_tune_basis(pm_ctx *ctx, uint64_t p, int m, int n, int64_t d, int reps, int64_t *out);

/* Measured rate of dense tensor-core MMA on device `device`: tcgen05.mma of
 * kind::f16 (fp16 x fp16 operands in shared memory, fp32 accumulator in tensor
 * memory) of shape 128 x n_cols x 16, `iters` back to back per SM on every SM,
 * timed by CUDA events (best of three launches after one warm-up).  The paper
 * has no counterpart: it is the tensor peak the tensor-core pointwise products
 * (Sec. 2, the n^omega d term) are measured against.  *tflops receives
 * 2 * 128 * n_cols * 16 * iters * SMs / time.  Requires 16 <= n_cols <= 256,
 * n_cols a multiple of 16, 1 <= iters <= 2^20.  Allocates a status word and
 * synchronises; returns PM_ETIMEOUT if the bounded wait for the MMAs ran out. */
int pm_mma_rate(int device, int n_cols, int iters, double *tflops);

#ifdef __cplusplus
}
#endif

#endif /* PMAT_H */
