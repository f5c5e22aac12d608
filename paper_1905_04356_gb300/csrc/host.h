// host.h -- host-side context and the internal product entry shared by the
// C-ABI products, PM-Basis and the resultant driver.
#pragma once
#include <cstdint>
#include <deque>
#include <string>
#include <vector>

#include "common.cuh"
#include "pmat.h"

struct PrimeSlot {
    u32 q = 0;
    int maxlog = 0;               // tables cover transforms up to 2^maxlog points
    uint2 *twf = nullptr, *twi = nullptr;
    u32 rf[PM_MAX_LOG2L + 1], ri[PM_MAX_LOG2L + 1];
};

struct Arena {                    // bump allocator over one device buffer
    char *base = nullptr;
    size_t size = 0, used = 0;
};

struct pm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own = nullptr;
    std::string err = "no error";
    int opt_pointwise = 0, opt_debug = 0;
    int64_t opt_T = 32;
    std::vector<PrimeSlot> table;     // CRT primes, largest first
    std::deque<PrimeSlot> direct;     // NTT-friendly moduli used directly (p = q); stable addresses
    void *ws = nullptr;
    size_t ws_size = 0;
    long long launches = 0;
    int64_t work[3] = {0, 0, 0};      // product work: compulsory bytes, pointwise MACs, butterflies
    int *d_status = nullptr;          // deferred device status (0 = OK)
    Arena arena;                      // driver buffers (PM-Basis, resultant)
    int opt_timing = 0;
    int opt_leaf_cluster = 1;         // PM-Basis leaves on a CTA cluster (0 = one CTA)
    int opt_host_chunks = 0;          // pmat_mul_host output chunks (0 = automatic)
    int opt_withhold = 0;             // test hook: the tensor-core pointwise kernel withholds an MMA
    // pointwise forms picked by pm_tune_product, per (m, n, k, transform length): form 1 = CUDA-core
    // block tile (bi, bk) of 4 x 8 thread tiles, 2 = tensor-core (four points per MMA, m, n, k <=
    // 32), 3 = streaming (n <= 8), 4 = matrix-vector (k = 1), 5 = tensor-core dense products per
    // point (m >= 64), 6 = CUDA-core block tile (bi, bk) of 4 x 4 thread tiles
    struct Tune { int m, n, k, lg, form, bi, bk; };
    std::vector<Tune> tune;
    int force_form = -1, force_bi = 0, force_bk = 0;   // the tuner's candidate while it times one
    // form 5: the tensor-core dense products per point (digit chunks of every point's A_j, B_j^T)
    void *gemm_ws = nullptr;
    size_t gemm_size = 0;
    struct Mark { int stage; cudaEvent_t a, b; long long launches; };
    std::vector<Mark> marks;          // recorded stage intervals
    std::vector<cudaEvent_t> spare;   // reusable events
    // pmat_mul_host: uploads and downloads on their own streams (created on first use), two
    // staging sets used by alternate calls so that one call's download overlaps the next
    // call's work; the context's stream joins the downloads lazily (host_join)
    cudaStream_t up = nullptr, dn = nullptr;
    std::vector<cudaEvent_t> hev;     // per-chunk ordering events
    cudaEvent_t in_free[2] = {nullptr, nullptr};   // staging set's inputs consumed (context stream)
    cudaEvent_t out_free[2] = {nullptr, nullptr};  // staging set's outputs downloaded (dn)
    cudaEvent_t ws_ready = nullptr;                // workspace (re)allocated (context stream)
    bool in_rec[2] = {false, false}, out_rec[2] = {false, false};
    bool host_pending = false;        // downloads the context's stream has not joined yet
    int host_parity = 0;
    size_t host_stage = 0;            // bytes of one staging set in the current layout
    void *host_ws = nullptr;          // the workspace the staging sets were laid out in
};

// Make the context's stream wait for every pending pmat_mul_host download (no-op if none).
int host_join(pm_ctx *ctx);

// Stage timing: stage_begin returns a token; stage_end closes it.
int stage_begin(pm_ctx *ctx, int stage);
void stage_end(pm_ctx *ctx, int token);

int pm_fail(pm_ctx *ctx, int code, const std::string &msg);
int pm_cuda(pm_ctx *ctx, cudaError_t e, const char *what);

// Device workspace of at least `bytes` (grows stream-ordered).
int ws_reserve(pm_ctx *ctx, size_t bytes, void **out);
// Arena: reset / reserve-grow / allocate (256-byte aligned).
int arena_reserve(pm_ctx *ctx, size_t bytes);
void *arena_alloc(pm_ctx *ctx, size_t bytes);

// C (m x k, entry stride sC) = coefficients off .. off+len-1 of A . B mod p,
// A: m x n, length dA, entry stride sA; B: n x k, length dB, stride sB.
// L is the cyclic transform length (power of 2, >= 16) chosen by the caller
// so that no aliased coefficient lands in [off, off+len) except beyond L
// (positions >= L of the slice are set to zero).
int prod_slice(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA, int64_t sA,
               const void *B, int64_t dB, int64_t sB, int64_t off, int64_t len, int lg, void *C, int64_t sC);

// One product request (the arguments of prod_slice).  An operand A used by many products
// can keep its transforms: At_out receives them (all primes, [prime][entry][L] words, prime
// stride prod_operand_bytes / K), At supplies them instead of transforming A again; both are
// valid for requests with the same p, inner dimension, min(dA, dB) and transform length.
struct ProdReq {
    uint64_t p;
    int w, m, n, k, lg;
    const void *A, *B;
    void *C;
    int64_t dA, sA, dB, sB, off, len, sC;
    const u32 *At = nullptr;
    u32 *At_out = nullptr;
};

// Bytes of an At / At_out buffer for an operand of `entries` entries in requests with these
// parameters (0 if the modulus cannot be handled).
size_t prod_operand_bytes(pm_ctx *ctx, uint64_t p, int n, int64_t dmin, int lg, int64_t entries);
// Run many independent product requests: planned together, their jobs binned by
// transform length into shared launches, the workspace chunked under a cap.
int prod_batch(pm_ctx *ctx, const ProdReq *reqs, int count);

int ceil_log2(int64_t x);

// The pointwise stage of the product path on transforms computed elsewhere, and the work
// counters of a Vandermonde product (vdm.cu).
int run_pointwise(pm_ctx *ctx, u32 *A, u32 *B, u32 *C, int m, int n, int k, int lg, const PrimeDev &D);
void count_work_vdm(pm_ctx *ctx, int lg, int m, int n, int k, int64_t dA, int64_t dB, int64_t len);
// C (M x N, row stride ldc) = A B^T mod the prime of P from tensor-core digit chunks (vdm.cu).
int vd_modgemm(pm_ctx *ctx, const unsigned char *Ad, const unsigned char *Bd, int M, int N, int nks, u32 *C, int64_t ldc,
               const PrimeDev &P);
// Pointwise products of one job as a batch of dense tensor-core products over its points (vdm.cu).
int pointwise_gemm(pm_ctx *ctx, const PwJob &j);

