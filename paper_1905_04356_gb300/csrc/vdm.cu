// vdm.cu -- polynomial-matrix products by evaluation and interpolation done as
// multiplications by Vandermonde matrices (Sec. 2, "Polynomial matrix
// multiplication": the variant after Doliskani, Giorgi, Lebreton and Schost,
// where the O(n^2 M(d)) evaluation / interpolation part becomes products of
// matrices over F_p of sizes about (d x d) by (d x n^2)).
//
// The points are the powers of an element w of order L (an NTT prime p, L the
// power of two above the output length), so the evaluation matrix is
// V[j][l] = w^(j l) and the interpolation matrix is its inverse,
// W[t][j] = L^-1 w^(-t j).  Then, with X_A the m n entries of A as rows of
// their dA coefficients (the caller's layout):
//     T_A = X_A V_A^T   (m n x L, V_A = V restricted to l < dA),  T_B alike,
//     T_C(e)[j] = sum over the inner dimension of T_A T_B at every point j
//                 (the pointwise products of the product path),
//     C   = T_C W^T    (m k x (dA + dB - 1)).
// Each of the three is a dense product C = A B^T mod p on the tensor cores.
//
// The tensor-core modular product (k_modgemm).  Residues are split once into
// balanced radix-256 digits in fp16 (d_0..d_2 in [-128, 127], d_3 in [0, 64],
// the bytes of r + 0x80808080 minus 128) and stored in chunks that are the
// shared-memory operand tiles of one 16-wide K-step in the no-swizzle K-major
// core-matrix layout: an A chunk holds the four digit tiles of 128 rows (16 KB),
// a B chunk the four digit blocks of 64 rows stacked as 256 MMA rows (8 KB).
// One CTA per SM, persistent over 128 x 64 output tiles: per K-step, four
// tcgen05.mma of 128 x 256 x 16 (digit x of A against [B_0 B_1 B_2 B_3]) write
// tensor-memory columns [64x, 64x + 256), so column block w accumulates
// E_w = sum_{x+y=w} A_x B_y (7 x 64 columns).  N = 256 halves the operand bytes
// per product against N = 128, which is what bounds this MMA shape.
// A digit product is at most 2^14 in magnitude and E_w has at most 4 x 256 of
// them per 256 inner entries, so every partial sum is an integer of magnitude
// <= 2^24, exact in fp32 (2^24 itself only when every term is the largest).
// After every 16 K-steps the seven accumulators are drained: E_1..E_4 converted
// to int32 by F2I, E_0, E_5 and E_6 (|E| <= 2^22: one product term of digits
// d_0 d_0, two of d_2 d_3, one of d_3 d_3) by adding 1.5 2^23 in fp32 and taking
// the low bits; then sum_w (256^w mod p) E_w + the running residue mod p.  The
// first K-step of a chunk clears the accumulators without stores: an MMA of a
// zero A tile into columns [192, 448) and the x = 0 MMA with accumulation off.
// Roles: warp 8 issues the chunks' bulk copies (cp.async.bulk, mbarrier
// transaction counts) into a ring of 8 stages, warp 9's first thread the MMAs,
// warps 0-7 (lane quarter w % 4, 32-column half w / 4) drain the accumulators
// and write finished tiles; the MMAs of a chunk wait for the previous drain.
// Every wait is bounded: after a timeout PM_ETIMEOUT is recorded, later waits
// return at once and the loops run out (output undefined); before the CTA exits
// the producer waits (bounded) for its copies and the MMA thread for its MMAs.
#include <cuda_fp16.h>
#include <cstring>
#include <vector>

#include "host.h"

#define VD_STAGES 8
#define VD_BN 64             // output columns per tile (B rows per chunk)
#define VD_ACHUNK 16384      // 128 rows x 16 K fp16 x 4 digits
#define VD_BCHUNK 8192       // 64 rows x 16 K fp16 x 4 digits (256 MMA rows)
#define VD_STAGE (VD_ACHUNK + VD_BCHUNK)
#define VD_ZERO 4096         // a zero 128 x 16 A operand (clears accumulator columns)
#define VD_SMEM (VD_STAGES * VD_STAGE + VD_ZERO)
#define VD_EPI 8             // drain warps: lane quarter w % 4, column half w / 4
#define VD_THREADS (32 * VD_EPI + 64)
#define VD_COLS 512          // tensor-memory columns (7 x 64 used)
#define VD_KC 16             // K-steps per drain (256 inner entries)

#define CKI(call)                                                       \
    do {                                                                \
        int _rc = (call);                                               \
        if (_rc) return _rc;                                            \
    } while (0)

namespace {

struct MgJob {
    const unsigned char *Ad, *Bd;   // digit chunks: A [row block][K-step] (16 KB), B [row block][K-step] (4 KB)
    i64 sAd, sBd;                   // bytes between the chunk sets of consecutive batch members
    u32 *C;                         // C[b sCb + i ldc + j ldj] for i < M, j < N, in [0, p)
    i64 ldc, ldj, sCb;
    int M, N, nks, nbN, tiles;      // rows, columns, K-steps, 64-column blocks, tiles per member
    PrimeDev P;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row r, inner 8 kk8 .. 8 kk8 + 7) in a 128 x 16 fp16 tile (K-major, no swizzle:
// 8-row x 16-byte core matrices, LBO 128 B between the two K-adjacent ones, SBO 256 B between
// 8-row groups)
__device__ __forceinline__ int op_off(int r, int kk8) { return (r >> 3) * 256 + kk8 * 128 + (r & 7) * 16; }

__device__ __forceinline__ uint64_t op_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           (1ull << 46);
}

// fp16 pair of digit x of two biased residues (bytes x of t0 and t1 as 0x6400 | byte, minus 1152)
__device__ __forceinline__ uint32_t digit_pair(uint32_t t0, uint32_t t1, int x)
{
    // prmt selector nibbles (nibble j picks result byte j from {t1, t0}, 4..7 = t1):
    // bytes 0 and 2 are byte x of t0 and byte x of t1 (bytes 1 and 3 are masked off)
    const uint32_t sel = (uint32_t)x | ((uint32_t)x << 4) | ((uint32_t)(4 + x) << 8) | ((uint32_t)(4 + x) << 12);
    uint32_t w;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(w) : "r"(t0), "r"(t1), "r"(sel));
    w = (w & 0x00FF00FFu) | 0x64006400u;
    const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&w), __halves2half2(__ushort_as_half(0x6480),
                                                                                      __ushort_as_half(0x6480)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// digits of 8 residues r[0..7] (inner entries 8 kk8 .. of one row) into the chunk layout.
// bmode: 0 = A chunks (128 rows, digit x tile at 4096 x), 1 = B chunks (64 rows, digit x at rows
// 64 x + r); chunk (row block, K-step) at base + (rb nks + ks) chunk bytes
__device__ __forceinline__ void put_digits(unsigned char *base, int bmode, int nks, int row, int k8, const u32 (&r)[8])
{
    u32 t[8];
#pragma unroll
    for (int i = 0; i < 8; i++) t[i] = r[i] + 0x80808080u;
    const int ks = k8 >> 1, kk8 = k8 & 1;
#pragma unroll
    for (int x = 0; x < 4; x++) {
        uint4 h;
        h.x = digit_pair(t[0], t[1], x);
        h.y = digit_pair(t[2], t[3], x);
        h.z = digit_pair(t[4], t[5], x);
        h.w = digit_pair(t[6], t[7], x);
        unsigned char *dst = bmode == 0
            ? base + ((size_t)(row >> 7) * nks + ks) * VD_ACHUNK + x * 4096 + op_off(row & 127, kk8)
            : base + ((size_t)(row >> 6) * nks + ks) * VD_BCHUNK + op_off(64 * x + (row & 63), kk8);
        *(uint4 *)dst = h;
    }
}

// digits of `batch` matrices of rows x K u32 residues in [0, p): element (b, row, l) at
// src[b sb + row srow + l sl], chunk set of member b at dst + b sdst.  bfast: consecutive threads
// take consecutive members (coalesced when sb = 1: the transform-domain layout), else
// consecutive octets of a row (coalesced when sl = 1: row-major matrices).
__global__ void k_vd_digits(const u32 *src, i64 sb, i64 srow, i64 sl, int batch, int rows, int K, int nks, int bmode,
                            unsigned char *dst, i64 sdst, int bfast)
{
    const int nk8 = (K + 7) >> 3;
    const i64 total = (i64)batch * rows * nk8;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < total; x += (i64)gridDim.x * blockDim.x) {
        int b, row, k8;
        if (bfast) { b = (int)(x % batch); const i64 y = x / batch; row = (int)(y / nk8); k8 = (int)(y % nk8); }
        else { k8 = (int)(x % nk8); const i64 y = x / nk8; row = (int)(y % rows); b = (int)(y / rows); }
        const u32 *s = src + b * sb + row * srow;
        u32 r[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int l = 8 * k8 + i;
            r[i] = l < K ? s[l * sl] : 0u;
        }
        put_digits(dst + b * sdst, bmode, nks, row, k8, r);
    }
}

// w^i mod p for i < L (p < 2^30)
__global__ void k_vd_powers(u32 *tab, int L, u32 w, u32 p)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
        u64 r = 1, b = w;
        for (u32 e = (u32)i; e; e >>= 1, b = b * b % p)
            if (e & 1) r = r * b % p;
        tab[i] = (u32)r;
    }
}

// digits (B chunks) of the matrix M[j][l] = s w^(sgn j l) for j < rows, l < K: the
// evaluation matrix (s = 1, sgn = +1) or the interpolation matrix (s = L^-1, sgn = -1)
__global__ void k_vd_matrix(const u32 *tab, int L, int rows, int K, int nks, int neg, u32 scale, u32 p,
                            unsigned char *dst)
{
    const int nk8 = (K + 7) >> 3;
    const i64 total = (i64)rows * nk8;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < total; x += (i64)gridDim.x * blockDim.x) {
        const int row = (int)(x / nk8), k8 = (int)(x % nk8);
        u32 r[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int l = 8 * k8 + i;
            u32 v = 0;
            if (l < K) {
                const u32 e = (u32)(((u64)row * (u64)l) & (u64)(L - 1));
                v = tab[neg ? (e ? (u32)L - e : 0u) : e];
                v = (u32)((u64)v * scale % p);
            }
            r[i] = v;
        }
        put_digits(dst, 1, nks, row, k8, r);
    }
}

__device__ __forceinline__ bool vd_wait(uint32_t bar, uint32_t parity, volatile int *abort, int *status)
{
    if (*abort) return false;
    for (int it = 0; it < (1 << 24); it++) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(bar), "r"(parity));
        if (done) return true;
        if ((it & 255) == 255 && *abort) return false;
    }
    *abort = 1;
    atomicExch(status, PM_ETIMEOUT);
    return false;
}

__device__ __forceinline__ void tmem_ld4(uint32_t addr, uint32_t *d)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]) : "r"(addr));
}

__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

// bounded wait that ignores the abort flag (teardown: copies and MMAs land before exit)
__device__ __forceinline__ void vd_wait_raw(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; it++)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(bar), "r"(parity));
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// integer value of an fp32 holding an integer of magnitude <= 2^22
__device__ __forceinline__ int small_f2i(uint32_t f)
{
    return __float_as_int(__fadd_rn(__uint_as_float(f), 12582912.0f)) - 0x4B400000;
}

__global__ void __launch_bounds__(VD_THREADS, 1) k_modgemm(const __grid_constant__ MgJob J, int total_tiles, int *status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    // full[S], empty[S], accumulators full, accumulators drained, final drain
    __shared__ __align__(8) uint64_t bars[2 * VD_STAGES + 3];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    volatile int *abort_ = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t b_full = smem_u32(&bars[0]), b_empty = smem_u32(&bars[VD_STAGES]),
                   b_accf = smem_u32(&bars[2 * VD_STAGES]), b_acce = smem_u32(&bars[2 * VD_STAGES + 1]),
                   b_drain = smem_u32(&bars[2 * VD_STAGES + 2]);
    unsigned char *zero = sm + VD_STAGES * VD_STAGE;
    for (int x = tid; x < VD_ZERO / 16; x += VD_THREADS) ((uint4 *)zero)[x] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // the zero tile, for the tensor core
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(VD_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < 2 * VD_STAGES + 3; b++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[b])),
                         "r"(b == 2 * VD_STAGES + 1 ? 32 * VD_EPI : 1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const int nks = J.nks, nkc = (nks + VD_KC - 1) / VD_KC;

    if (warp == VD_EPI) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            int ksg = 0;                      // K-steps issued by this CTA
            for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
                const int bm = t / J.tiles, tl = t % J.tiles, mb = tl / J.nbN, nb = tl % J.nbN;
                const unsigned char *Ab = J.Ad + bm * J.sAd + (size_t)mb * nks * VD_ACHUNK,
                                    *Bb = J.Bd + bm * J.sBd + (size_t)nb * nks * VD_BCHUNK;
                for (int ks = 0; ks < nks; ks++, ksg++) {
                    const int s = ksg % VD_STAGES;
                    if (ksg >= VD_STAGES) vd_wait(b_empty + 8 * s, (uint32_t)((ksg / VD_STAGES - 1) & 1), abort_, status);
                    const uint32_t dst = smem_u32(sm + s * VD_STAGE), bar = b_full + 8 * s;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(VD_STAGE) : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(dst), "l"(Ab + (size_t)ks * VD_ACHUNK), "r"(VD_ACHUNK), "r"(bar) : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(dst + VD_ACHUNK), "l"(Bb + (size_t)ks * VD_BCHUNK), "r"(VD_BCHUNK), "r"(bar)
                                 : "memory");
                }
            }
            // the copies still in flight land before the CTA exits
            for (int k2 = ksg - VD_STAGES < 0 ? 0 : ksg - VD_STAGES; k2 < ksg; k2++)
                vd_wait_raw(b_full + 8 * (k2 % VD_STAGES), (uint32_t)((k2 / VD_STAGES) & 1));
        }
    } else if (warp == VD_EPI + 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            // D f32 (bit 4), A and B fp16, K-major; N = 256 (>> 3 at bit 17), M = 128 (>> 4 at bit 24)
            const uint32_t idesc = (1u << 4) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
            const uint64_t zd = op_desc(smem_u32(zero));
            int ksg = 0, g = 0;               // K-steps and accumulator chunks of this CTA
            for (int t = blockIdx.x; t < total_tiles; t += gridDim.x)
                for (int kc = 0; kc < nkc; kc++, g++) {
                    if (g >= 1) vd_wait(b_acce, (uint32_t)((g - 1) & 1), abort_, status);   // previous chunk drained
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const int k1 = (kc + 1) * VD_KC < nks ? (kc + 1) * VD_KC : nks;
                    for (int ks = kc * VD_KC; ks < k1; ks++, ksg++) {
                        const int s = ksg % VD_STAGES;
                        vd_wait(b_full + 8 * s, (uint32_t)((ksg / VD_STAGES) & 1), abort_, status);
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint32_t st = smem_u32(sm + s * VD_STAGE);
                        const uint64_t bd = op_desc(st + VD_ACHUNK);
                        const uint32_t first = ks == kc * VD_KC;
                        if (first) mma_f16(tmem + 192u, zd, bd, idesc, 0u);     // columns [192, 448) <- 0
#pragma unroll
                        for (int x = 0; x < 4; x++)
                            mma_f16(tmem + 64u * x, op_desc(st + 4096 * x), bd, idesc, (first && x == 0) ? 0u : 1u);
                        commit(b_empty + 8 * s);
                    }
                    commit(b_accf);
                }
            commit(b_drain);                 // every MMA of this CTA has completed
            vd_wait_raw(b_drain, 0u);
        }
    } else {
        // ---------------------------------------------------------------- drain (warps 0-7)
        const int half = warp >> 2;
        const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32u * half;
        const u32 q = J.P.q;
        u32 cw[7];
#pragma unroll
        for (int w = 0; w < 7; w++) cw[w] = (u32)((1ull << (8 * w)) % q);
        const i64 off = (i64)q << 28;          // > 7 q 2^24 >= |sum_w cw_w E_w|: keeps the sums positive
        int g = 0;
        for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
            const int bm = t / J.tiles, tl = t % J.tiles, mb = tl / J.nbN, nb = tl % J.nbN;
            u32 acc[32];
#pragma unroll
            for (int c = 0; c < 32; c++) acc[c] = 0;
            for (int kc = 0; kc < nkc; kc++, g++) {
                if (lane == 0) vd_wait(b_accf, (uint32_t)(g & 1), abort_, status);
                __syncwarp();
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int gg = 0; gg < 8; gg++) {              // 4 columns at a time: 7 loads, one wait
                    uint32_t d[7][4];
#pragma unroll
                    for (int w = 0; w < 7; w++) tmem_ld4(tq + 64u * w + 4u * gg, d[w]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    if (gg == 7) {
                        // every value of the chunk is in registers: the MMAs may overwrite
                        asm volatile("tcgen05.fence::before_thread_sync;");
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b_acce) : "memory");
                    }
#pragma unroll
                    for (int cc = 0; cc < 4; cc++) {
                        i64 x = off + acc[4 * gg + cc];
                        x += (i64)(int)cw[0] * (i64)small_f2i(d[0][cc]);
#pragma unroll
                        for (int w = 1; w < 5; w++) x += (i64)(int)cw[w] * (i64)__float2int_rn(__uint_as_float(d[w][cc]));
                        x += (i64)(int)cw[5] * (i64)small_f2i(d[5][cc]);
                        x += (i64)(int)cw[6] * (i64)small_f2i(d[6][cc]);
                        acc[4 * gg + cc] = reduce64((u64)x, J.P);
                    }
                }
            }
            const int row = mb * 128 + 32 * (warp & 3) + lane, c0 = nb * VD_BN + 32 * half;
            if (row < J.M && c0 < J.N) {
                u32 *dst = J.C + bm * J.sCb + (i64)row * J.ldc + (i64)c0 * J.ldj;
                const int nc = J.N - c0 < 32 ? J.N - c0 : 32;
#pragma unroll
                for (int c = 0; c < 32; c++)
                    if (c < nc) dst[c * J.ldj] = acc[c];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(VD_COLS));
}

size_t al256v(size_t x) { return (x + 255) & ~size_t(255); }

int grid_for(i64 total) { return (int)(total / 256 + 1 < 4096 ? total / 256 + 1 : 4096); }

}  // namespace

// C_b (M x N: element (i, j) at C + b sCb + i ldc + j ldj) = A_b B_b^T mod the prime of P for
// b < batch, from digit chunk sets sAd / sBd bytes apart (one launch).
int vd_modgemm_batched(pm_ctx *ctx, const unsigned char *Ad, int64_t sAd, const unsigned char *Bd, int64_t sBd,
                       int batch, int M, int N, int nks, u32 *C, int64_t ldc, int64_t ldj, int64_t sCb,
                       const PrimeDev &P)
{
    MgJob J;
    J.Ad = Ad; J.Bd = Bd; J.sAd = sAd; J.sBd = sBd;
    J.C = C; J.ldc = ldc; J.ldj = ldj; J.sCb = sCb;
    J.M = M; J.N = N; J.nks = nks; J.nbN = (N + VD_BN - 1) / VD_BN; J.tiles = ((M + 127) / 128) * J.nbN; J.P = P;
    const int64_t tiles = (int64_t)batch * J.tiles;
    if (tiles > 0x7fffffffLL) return pm_fail(ctx, PM_EUNSUPPORTED, "modular product grid too large");
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess || sms < 1) return pm_cuda(ctx, e != cudaSuccess ? e : cudaErrorInvalidDevice, "SM count");
    e = cudaFuncSetAttribute(k_modgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, VD_SMEM);
    if (e != cudaSuccess) return pm_cuda(ctx, e, "cudaFuncSetAttribute");
    const int grid = tiles < sms ? (int)tiles : sms;      // persistent: one CTA per SM
    k_modgemm<<<grid, VD_THREADS, VD_SMEM, ctx->stream>>>(J, (int)tiles, ctx->d_status);
    ctx->launches++;
    return pm_cuda(ctx, cudaGetLastError(), "k_modgemm");
}

// C (M x N, row stride ldc) = A B^T mod the prime of P, from digit chunks (one launch).
int vd_modgemm(pm_ctx *ctx, const unsigned char *Ad, const unsigned char *Bd, int M, int N, int nks, u32 *C, int64_t ldc,
               const PrimeDev &P)
{
    return vd_modgemm_batched(ctx, Ad, 0, Bd, 0, 1, M, N, nks, C, ldc, 1, 0, P);
}

// Bytes of the digit chunks of a member: rows in blocks of 128 (A) or 64 (B), K in steps of 16.
static size_t vd_chunk_bytes(int rows, int K, int bmode)
{
    const int nks = (K + 15) / 16;
    return bmode == 0 ? (size_t)((rows + 127) / 128) * nks * VD_ACHUNK
                      : (size_t)((rows + VD_BN - 1) / VD_BN) * nks * VD_BCHUNK;
}

// The pointwise products C_j = A_j B_j mod q at the L transform points as a batch of dense
// products on the tensor cores: A_j (m x n) and B_j^T (k x n) are gathered from the
// transform-domain layout [entry][L] into digit chunks, C_j is written back into it.
int pointwise_gemm(pm_ctx *ctx, const PwJob &j)
{
    const int m = j.m, n = j.n, k = j.k, L = j.L, nks = (n + 15) / 16;
    const size_t bA = al256v(vd_chunk_bytes(m, n, 0)), bB = al256v(vd_chunk_bytes(k, n, 1));
    const size_t need = (size_t)L * (bA + bB);
    if (need > ctx->gemm_size) {
        if (ctx->gemm_ws) CKI(pm_cuda(ctx, cudaFreeAsync(ctx->gemm_ws, ctx->stream), "cudaFreeAsync"));
        ctx->gemm_ws = nullptr;
        ctx->gemm_size = 0;
        if (cudaMallocAsync(&ctx->gemm_ws, need, ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return pm_fail(ctx, PM_ENOMEM, "pointwise digit scratch allocation failed");
        }
        ctx->gemm_size = need;
    }
    unsigned char *Ad = (unsigned char *)ctx->gemm_ws, *Bd = Ad + (size_t)L * bA;
    CKI(pm_cuda(ctx, cudaMemsetAsync(Ad, 0, need, ctx->stream), "cudaMemsetAsync"));
    const int64_t tA = (int64_t)L * m * ((n + 7) / 8), tB = (int64_t)L * k * ((n + 7) / 8);
    // A_j[i][l] = A[(i n + l) L + j]; B_j^T[c][l] = B[(l k + c) L + j]
    k_vd_digits<<<grid_for(tA), 256, 0, ctx->stream>>>(j.A, 1, (int64_t)n * L, L, L, m, n, nks, 0, Ad, (int64_t)bA, 1);
    k_vd_digits<<<grid_for(tB), 256, 0, ctx->stream>>>(j.B, 1, L, (int64_t)k * L, L, k, n, nks, 1, Bd, (int64_t)bB, 1);
    ctx->launches += 2;
    CKI(pm_cuda(ctx, cudaGetLastError(), "k_vd_digits"));
    // C_j[i][c] = C[(i k + c) L + j]
    return vd_modgemm_batched(ctx, Ad, (int64_t)bA, Bd, (int64_t)bB, L, m, k, nks, j.C, (int64_t)k * L, L, 1, j.P);
}

extern "C" int pmat_mul_vdm(pm_ctx *ctx, uint64_t p, int m, int n, int k, const void *A, int64_t dA, const void *B,
                            int64_t dB, void *C)
{
    if (!ctx) return PM_EINVAL;
    if (m < 1 || n < 1 || k < 1 || dA < 1 || dB < 1 || !A || !B || !C)
        return pm_fail(ctx, PM_EINVAL, "pmat_mul_vdm: bad arguments");
    if (dA > (1 << 15) || dB > (1 << 15)) return pm_fail(ctx, PM_EINVAL, "pmat_mul_vdm: lengths above 2^15");
    const int64_t len = dA + dB - 1;
    const int lg0 = ceil_log2(len), lg = lg0 < 5 ? 5 : lg0;
    const int64_t L = int64_t(1) << lg;
    if (p >= (1ull << 30) || p < 3 || ((p - 1) % (uint64_t)L) != 0 || !ntt_is_prime32(p))
        return pm_fail(ctx, PM_EUNSUPPORTED, "pmat_mul_vdm: p must be a prime below 2^30 with 2^lg | p - 1");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    CKI(host_join(ctx));
    const u32 q = (u32)p;
    u32 rf[PM_MAX_LOG2L + 1], ri[PM_MAX_LOG2L + 1];
    ntt_roots(q, rf, ri);
    PrimeDev P;
    memset(&P, 0, sizeof(P));
    P.q = q; P.q2 = 2 * q;
    P.r32 = (u32)((1ull << 32) % q);
    P.r32s = (u32)(((uint64_t)P.r32 << 32) / q);
    P.ones = (u32)((1ull << 32) / q);
    const u32 linv = (u32)host_powmod((uint64_t)L % q, q - 2, q);
    // workspace
    const int64_t eA = (int64_t)m * n, eB = (int64_t)n * k, eC = (int64_t)m * k;
    const int nkA = (int)((dA + 15) / 16), nkB = (int)((dB + 15) / 16), nkL = (int)(L / 16);
    const size_t bXA = al256v((size_t)((eA + 127) / 128) * nkA * VD_ACHUNK), bXB = al256v((size_t)((eB + 127) / 128) * nkB * VD_ACHUNK);
    const size_t bVA = al256v(vd_chunk_bytes(L, (int)dA, 1)), bVB = al256v(vd_chunk_bytes(L, (int)dB, 1));
    const size_t bTC = al256v((size_t)((eC + 127) / 128) * nkL * VD_ACHUNK), bW = al256v(vd_chunk_bytes((int)len, L, 1));
    const size_t bdig = bXA + bXB + bVA + bVB + bTC + bW;
    const size_t bTa = al256v((size_t)eA * L * 4), bTb = al256v((size_t)eB * L * 4), bTc = al256v((size_t)eC * L * 4);
    const size_t btab = al256v((size_t)L * 4);
    void *ws = nullptr;
    CKI(ws_reserve(ctx, bdig + bTa + bTb + bTc + btab + 256, &ws));
    unsigned char *cur = (unsigned char *)ws;
    unsigned char *XA = cur; cur += bXA;
    unsigned char *XB = cur; cur += bXB;
    unsigned char *VA = cur; cur += bVA;
    unsigned char *VB = cur; cur += bVB;
    unsigned char *TCd = cur; cur += bTC;
    unsigned char *Wd = cur; cur += bW;
    u32 *TA = (u32 *)cur; cur += bTa;
    u32 *TB = (u32 *)cur; cur += bTb;
    u32 *TC = (u32 *)cur; cur += bTc;
    u32 *tab = (u32 *)cur;
    count_work_vdm(ctx, lg, m, n, k, dA, dB, len);
    // ---- evaluation: T_A = X_A V_A^T, T_B = X_B V_B^T (digits first; padding digits are zero)
    int tok = stage_begin(ctx, PM_STAGE_FWD);
    CKI(pm_cuda(ctx, cudaMemsetAsync(ws, 0, bdig, ctx->stream), "cudaMemsetAsync"));
    k_vd_powers<<<grid_for(L), 256, 0, ctx->stream>>>(tab, (int)L, rf[lg], q);
    k_vd_digits<<<grid_for(eA * ((dA + 7) / 8)), 256, 0, ctx->stream>>>((const u32 *)A, 0, dA, 1, 1, (int)eA, (int)dA, nkA,
                                                                          0, XA, 0, 0);
    k_vd_digits<<<grid_for(eB * ((dB + 7) / 8)), 256, 0, ctx->stream>>>((const u32 *)B, 0, dB, 1, 1, (int)eB, (int)dB, nkB,
                                                                          0, XB, 0, 0);
    k_vd_matrix<<<grid_for(L * ((dA + 7) / 8)), 256, 0, ctx->stream>>>(tab, (int)L, (int)L, (int)dA, nkA, 0, 1u, q, VA);
    k_vd_matrix<<<grid_for(L * ((dB + 7) / 8)), 256, 0, ctx->stream>>>(tab, (int)L, (int)L, (int)dB, nkB, 0, 1u, q, VB);
    k_vd_matrix<<<grid_for(len * (L / 8)), 256, 0, ctx->stream>>>(tab, (int)L, (int)len, (int)L, nkL, 1, linv, q, Wd);
    ctx->launches += 6;
    CKI(pm_cuda(ctx, cudaGetLastError(), "Vandermonde set-up"));
    CKI(vd_modgemm(ctx, XA, VA, (int)eA, (int)L, nkA, TA, L, P));
    CKI(vd_modgemm(ctx, XB, VB, (int)eB, (int)L, nkB, TB, L, P));
    stage_end(ctx, tok);
    // ---- pointwise products at the L points (the product path's kernels)
    tok = stage_begin(ctx, PM_STAGE_POINTWISE);
    CKI(run_pointwise(ctx, TA, TB, TC, m, n, k, lg, P));
    stage_end(ctx, tok);
    // ---- interpolation: C = T_C W^T
    tok = stage_begin(ctx, PM_STAGE_INV);
    k_vd_digits<<<grid_for(eC * (L / 8)), 256, 0, ctx->stream>>>(TC, 0, L, 1, 1, (int)eC, (int)L, nkL, 0, TCd, 0, 0);
    ctx->launches++;
    CKI(pm_cuda(ctx, cudaGetLastError(), "k_vd_digits"));
    CKI(vd_modgemm(ctx, TCd, Wd, (int)eC, (int)len, nkL, (u32 *)C, len, P));
    stage_end(ctx, tok);
    return PM_OK;
}
