// small.cu -- the whole product A . B mod p in one launch of one CTA cluster, for small products
// modulo an NTT prime (Sec. 2, "Polynomial matrix multiplication": evaluation at the L-th
// roots of unity, pointwise products, interpolation).  A 4 x 4 . 4 x 4 product of length-256
// entries is a few microseconds of work; done as the batched path's three launches (forward
// transforms, pointwise products, inverse transforms) with their job packs it costs three
// launch latencies and the host's planning.  Here, on a cluster of SMALL_CL CTAs:
//   1. CTA r takes the input entries e = r, r + SMALL_CL, ... (the m n entries of A, then the
//      n k of B), reduced mod q and zero-padded to L points, into its shared memory;
//   2. Gentleman-Sande (DIF) transforms of each, natural order in, bit-reversed order out,
//      the twiddle of butterfly o in a block of 2h points w_{2h}^o (the context's tables, staged
//      in shared memory); stages taken two at a time (a thread does both stages on four points);
//   3. after a cluster barrier, CTA r takes the output entries e = r, r + SMALL_CL, ...:
//      C_ik(x) = sum_l A_il(x) B_lk(x) at each point, the transforms of A_il and B_lk read from
//      the CTAs that hold them (distributed shared memory), one 64-bit sum of at most 16
//      products of residues below 2^30 (exact) reduced once;
//   4. Cooley-Tukey (DIT) inverse transforms, bit-reversed in, natural out, scaled by L^-1,
//      and the dA + dB - 1 coefficients of each entry written in the caller's width;
//   5. a last cluster barrier, so that no CTA leaves while a peer may read its memory.
// Every value is kept in [0, q) between steps.  One block barrier per pair of butterfly stages.
#include <cooperative_groups.h>

#include "host.h"

#define SMALL_CL 8           // CTAs of the cluster
#define SMALL_THREADS 512

namespace {

__device__ __forceinline__ u32 add_q(u32 a, u32 b, u32 q)
{
    const u32 s = a + b;
    return s >= q ? s - q : s;
}

// butterflies of one stage over `rows` rows of L points at R (row stride L): DIF (INV = false,
// twiddles tw[h + o] = w_{2h}^o) or DIT (INV = true, inverse twiddles)
template <bool INV>
__device__ __forceinline__ void stage(u32 *R, int rows, int lg, int h, const uint2 *tw, u32 q)
{
    const int half = 1 << (lg - 1);
    for (int x = threadIdx.x; x < rows * half; x += blockDim.x) {
        const int row = x >> (lg - 1), r = x & (half - 1), o = r & (h - 1);
        u32 *P = R + ((size_t)row << lg) + ((r - o) << 1) + o;
        const uint2 w = tw[h + o];
        const u32 a = P[0], b = P[h];
        if (!INV) {
            P[0] = add_q(a, b, q);
            P[h] = csub(shoup_mul(a + q - b, w.x, w.y, q), q);
        } else {
            const u32 t = csub(shoup_mul(b, w.x, w.y, q), q);
            P[0] = add_q(a, t, q);
            P[h] = add_q(a, q - t, q);
        }
    }
}

// two DIF stages, half sizes h and h / 2 (h >= 2), on the quads P0 .. P3 = base + {0, 1, 2, 3} h / 2
// of every block of 2h points (base = block start + o, o < h / 2): the same butterflies as two
// calls of stage<false>, without the barrier between them
__device__ __forceinline__ void stage2_dif(u32 *R, int rows, int lg, int h, const uint2 *tw, u32 q)
{
    const int quarter = 1 << (lg - 2), hh = h >> 1;
    for (int x = threadIdx.x; x < rows * quarter; x += blockDim.x) {
        const int row = x >> (lg - 2), r = x & (quarter - 1), o = r & (hh - 1);
        u32 *P = R + ((size_t)row << lg) + ((r - o) << 2) + o;
        u32 a0 = P[0], a1 = P[hh], a2 = P[h], a3 = P[h + hh];
        const uint2 w0 = tw[h + o], w1 = tw[h + o + hh], w2 = tw[hh + o];
        u32 t;
        t = add_q(a0, a2, q); a2 = csub(shoup_mul(a0 + q - a2, w0.x, w0.y, q), q); a0 = t;
        t = add_q(a1, a3, q); a3 = csub(shoup_mul(a1 + q - a3, w1.x, w1.y, q), q); a1 = t;
        t = add_q(a0, a1, q); a1 = csub(shoup_mul(a0 + q - a1, w2.x, w2.y, q), q); a0 = t;
        t = add_q(a2, a3, q); a3 = csub(shoup_mul(a2 + q - a3, w2.x, w2.y, q), q); a2 = t;
        P[0] = a0; P[hh] = a1; P[h] = a2; P[h + hh] = a3;
    }
}

// two DIT stages, half sizes h and 2h, on the quads P0 .. P3 = base + {0, 1, 2, 3} h of every
// block of 4h points (o < h): the same butterflies as two calls of stage<true>
__device__ __forceinline__ void stage2_dit(u32 *R, int rows, int lg, int h, const uint2 *tw, u32 q)
{
    const int quarter = 1 << (lg - 2);
    for (int x = threadIdx.x; x < rows * quarter; x += blockDim.x) {
        const int row = x >> (lg - 2), r = x & (quarter - 1), o = r & (h - 1);
        u32 *P = R + ((size_t)row << lg) + ((r - o) << 2) + o;
        u32 a0 = P[0], a1 = P[h], a2 = P[2 * h], a3 = P[3 * h];
        const uint2 w0 = tw[h + o], w1 = tw[2 * h + o], w2 = tw[3 * h + o];
        u32 t;
        t = csub(shoup_mul(a1, w0.x, w0.y, q), q); a1 = add_q(a0, q - t, q); a0 = add_q(a0, t, q);
        t = csub(shoup_mul(a3, w0.x, w0.y, q), q); a3 = add_q(a2, q - t, q); a2 = add_q(a2, t, q);
        t = csub(shoup_mul(a2, w1.x, w1.y, q), q); a2 = add_q(a0, q - t, q); a0 = add_q(a0, t, q);
        t = csub(shoup_mul(a3, w2.x, w2.y, q), q); a3 = add_q(a1, q - t, q); a1 = add_q(a1, t, q);
        P[0] = a0; P[h] = a1; P[2 * h] = a2; P[3 * h] = a3;
    }
}

__global__ void __launch_bounds__(SMALL_THREADS) k_small_product(const __grid_constant__ SmallJob J)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) u32 sh[];
    const int lg = J.lg, L = 1 << lg;
    const int eA = J.m * J.n, eB = J.n * J.k, eC = J.m * J.k, eX = eA + eB;
    const int rk = (int)cl.block_rank(), tid = threadIdx.x, nth = blockDim.x;
    const int nx = (eX - rk + SMALL_CL - 1) / SMALL_CL, ny = (eC - rk + SMALL_CL - 1) / SMALL_CL;   // entries here
    const int sx = (eX + SMALL_CL - 1) / SMALL_CL;           // input slots per CTA (the same in every CTA)
    const u32 q = J.P.q;
    uint2 *twf = (uint2 *)sh, *twi = twf + L;
    u32 *X = (u32 *)(twi + L);                               // [sx][L]: input entry rk + SMALL_CL s in slot s
    u32 *Y = X + ((size_t)sx << lg);                         // [ny][L]
    for (int i = tid; i < L; i += nth) { twf[i] = J.P.twf[i]; twi[i] = J.P.twi[i]; }
    // 1. this CTA's input entries, values mod q
    for (int x = tid; x < (nx << lg); x += nth) {
        const int s = x >> lg, t = x & (L - 1), e = rk + SMALL_CL * s;
        const bool isA = e < eA;
        const int d = isA ? J.dA : J.dB;
        u32 v = 0;
        if (t < d) {
            const i64 idx = (i64)(isA ? e : e - eA) * d + t;
            const void *src = isA ? J.A : J.B;
            if (J.w == 8) v = reduce64(((const u64 *)src)[idx], J.P);
            else v = csub(shoup_mul(((const u32 *)src)[idx], 1u, J.P.ones, q), q);
        }
        X[x] = v;
    }
    __syncthreads();
    // 2. forward transforms: stages h = L/2, ..., 1, two at a time while h >= 2
    for (int h = L >> 1; h >= 1;) {
        if (h >= 2) { stage2_dif(X, nx, lg, h, twf, q); h >>= 2; }
        else { stage<false>(X, nx, lg, h, twf, q); h >>= 1; }
        __syncthreads();
    }
    cl.sync();                                               // every input transform is in place
    // 3. pointwise products of this CTA's output entries, operands from the CTAs that hold them
    for (int x = tid; x < (ny << lg); x += nth) {
        const int s = x >> lg, pt = x & (L - 1), e = rk + SMALL_CL * s, i = e / J.k, c = e - i * J.k;
        u64 acc = 0;
#pragma unroll 4
        for (int l = 0; l < J.n; l++) {
            const int ea = i * J.n + l, eb = eA + l * J.k + c;
            const u32 *Xa = cl.map_shared_rank(X, ea % SMALL_CL), *Xb = cl.map_shared_rank(X, eb % SMALL_CL);
            acc += (u64)Xa[((size_t)(ea / SMALL_CL) << lg) + pt] * Xb[((size_t)(eb / SMALL_CL) << lg) + pt];
        }
        Y[x] = reduce64(acc, J.P);
    }
    __syncthreads();
    // 4. inverse transforms: stages h = 1, ..., L/2, two at a time while 2h <= L/2
    for (int h = 1; h <= (L >> 1);) {
        if (2 * h <= (L >> 1)) { stage2_dit(Y, ny, lg, h, twi, q); h <<= 2; }
        else { stage<true>(Y, ny, lg, h, twi, q); h <<= 1; }
        __syncthreads();
    }
    // 5. scaled coefficients 0 .. len - 1 of this CTA's output entries
    for (int x = tid; x < ny * J.len; x += nth) {
        const int s = x / J.len, t = x - s * J.len, e = rk + SMALL_CL * s;
        const u32 v = csub(shoup_mul(Y[((size_t)s << lg) + t], J.P.linv, J.P.linvs, q), q);
        const i64 o = (i64)e * J.len + t;
        if (J.w == 8) ((u64 *)J.C)[o] = v;
        else ((u32 *)J.C)[o] = v;
    }
    cl.sync();                                               // no CTA leaves while a peer may read it
}

}  // namespace

size_t small_product_smem(int m, int n, int k, int lg)
{
    const size_t L = (size_t)1 << lg, ex = (size_t)m * n + (size_t)n * k, ec = (size_t)m * k;
    return 2 * L * sizeof(uint2) + ((ex + SMALL_CL - 1) / SMALL_CL + (ec + SMALL_CL - 1) / SMALL_CL) * L * sizeof(u32);
}

cudaError_t launch_small_product(const SmallJob &J, cudaStream_t st)
{
    static size_t set = 0;                                   // the attribute set for up to `set` bytes
    const size_t sm = small_product_smem(J.m, J.n, J.k, J.lg);
    if (sm > set) {
        cudaError_t e = cudaFuncSetAttribute(k_small_product, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        set = 200 * 1024;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(SMALL_CL);
    cfg.blockDim = dim3(SMALL_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = SMALL_CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_small_product, J);
}
