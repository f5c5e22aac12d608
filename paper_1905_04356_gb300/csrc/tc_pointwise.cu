// tc_pointwise.cu -- pointwise matrix products on the tensor cores (tcgen05).
//
// At every transform point j, C_j = A_j B_j mod q (Sec. 2, "Polynomial matrix
// multiplication": the n^omega d term), for m, n, k <= 32.  Each 30-bit residue
// is split into four 8-bit limbs, a = sum_u a_u 2^(8u); limbs are exact in
// bf16, every limb product is below 2^16 and every sum of n <= 32 of them is
// below 2^21, so one tcgen05.mma of kind::f16 (bf16 x bf16, fp32 accumulator in
// tensor memory) computes all limb products exactly:
//     D (128 x 4kp) = A_limb (128 x n) . B_limb (n x 4kp),
// with row 4i + u of A_limb = limb u of row i of A_j, and column v kp + c of
// B_limb = limb v of column c of B_j.  The CUDA cores then recombine
//     C(i, c) = sum_u 2^(8u) sum_v 2^(8v) D(4i + u, v kp + c)  mod q:
// the four u of one output sit in four adjacent lanes (tensor-memory lane =
// row), so they combine with two shuffles.
//
// A block takes 8 consecutive points of one prime: the residues of all entries
// for those points are staged in shared memory with 16-byte loads (the
// transform domain is entry-major, point-minor), then point by point: limb
// operands are written in the no-swizzle K-major core-matrix layout, one thread
// issues the MMA(s) and commits to an mbarrier (bounded wait), the accumulator
// is read back with tcgen05.ld, results are staged and finally written back
// 32 bytes per entry.
#include <cuda_bf16.h>

#include "common.cuh"
#include "pmat.h"

#define TC_PTS 8          // points per block
#define TC_THREADS 128    // four warps: tensor-memory lanes 0..127

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// (row r, k) of an R x 32 bf16 tile, K-major, no swizzle: 8-row x 16-byte core
// matrices, 128 B between K-adjacent ones (LBO), 512 B between 8-row groups (SBO)
__device__ __forceinline__ int tc_off(int r, int k) { return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t f32_to_u(uint32_t bits)
{
    // exact nonnegative integer below 2^23 held in an fp32: add 2^23 and read the mantissa
    return __float_as_uint(__uint_as_float(bits) + 8388608.0f) - 0x4B000000u;
}

int tc_blocks(const PwJob &j) { return (j.L + TC_PTS - 1) / TC_PTS; }

template <int KP>
__global__ void __launch_bounds__(TC_THREADS) k_pointwise_tc(const __grid_constant__ JobPack<PwJob> pk, int *status,
                                                              int withhold)
{
    constexpr int N = 4 * KP;                      // MMA N (columns: limb v, column c)
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int b = blockIdx.x;
    int jb = 0;
    while (b >= pk.blk_start[jb + 1]) jb++;
    const PwJob &J = pk.jobs[jb];
    const int m = J.m, n = J.n, k = J.k, L = J.L;
    const u32 q = J.P.q, q2 = J.P.q2, r32 = J.P.r32, r32s = J.P.r32s, ones = J.P.ones;
    const int j0 = (b - pk.blk_start[jb]) * TC_PTS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    unsigned char *opA = sm;                       // 128 x 32 bf16
    unsigned char *opB = sm + 8192;                // N x 32 bf16
    u32 *rawA = (u32 *)(sm + 16384);               // [m n][TC_PTS]
    u32 *rawB = rawA + 1024 * TC_PTS;              // [n k][TC_PTS]
    u32 *outC = rawB + 1024 * TC_PTS;              // [m k][TC_PTS]

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(N < 32 ? 32 : N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // stage the 8 points of every entry: 32 contiguous bytes per entry (L is a multiple of 16)
    const int eA = m * n, eB = n * k;
    for (int x = tid; x < (eA + eB) * 2; x += TC_THREADS) {
        const int e = x >> 1, h = x & 1;
        const u32 *src = e < eA ? J.A + (i64)e * L : J.B + (i64)(e - eA) * L;
        const uint4 v = *(const uint4 *)(src + j0 + 4 * h);
        u32 *dst = (e < eA ? rawA + e * TC_PTS : rawB + (e - eA) * TC_PTS) + 4 * h;
        *(uint4 *)dst = v;
    }
    // zero both operand tiles once: padding rows / columns stay zero for every point
    for (int x = tid; x < (8192 + N * 64) / 16; x += TC_THREADS) ((uint4 *)sm)[x] = make_uint4(0, 0, 0, 0);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
    const int ksteps = (n + 15) >> 4;
    // per-lane recombination constant 2^(8u) mod q, u = lane & 3 (row 4i + u)
    const int u = lane & 3;
    const u32 wu = (u32)(((1ull << (8 * u)) % q));
    const u32 wus = (u32)(((u64)wu << 32) / q);
    bool ok = true;

    for (int pp = 0; pp < TC_PTS; pp++) {
        // ---- limb operands for point j0 + pp
        for (int x = tid; x < m * ((n + 1) >> 1); x += TC_THREADS) {
            const int i = x / ((n + 1) >> 1), l = 2 * (x % ((n + 1) >> 1));
            const u32 a0 = rawA[(i * n + l) * TC_PTS + pp];
            const u32 a1 = l + 1 < n ? rawA[(i * n + l + 1) * TC_PTS + pp] : 0u;
#pragma unroll
            for (int uu = 0; uu < 4; uu++) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn((float)((a0 >> (8 * uu)) & 255u), (float)((a1 >> (8 * uu)) & 255u));
                *(__nv_bfloat162 *)(opA + tc_off(4 * i + uu, l)) = h2;
            }
        }
        for (int x = tid; x < k * ((n + 1) >> 1); x += TC_THREADS) {
            const int c = x / ((n + 1) >> 1), l = 2 * (x % ((n + 1) >> 1));
            const u32 b0 = rawB[(l * k + c) * TC_PTS + pp];
            const u32 b1 = l + 1 < n ? rawB[((l + 1) * k + c) * TC_PTS + pp] : 0u;
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn((float)((b0 >> (8 * v)) & 255u), (float)((b1 >> (8 * v)) & 255u));
                *(__nv_bfloat162 *)(opB + tc_off(v * KP + c, l)) = h2;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // withhold (test hook): block 0 issues no MMA for its first point, so nothing is in
        // flight and its wait below must give up
        const bool issue = !(withhold && blockIdx.x == 0 && pp == 0);
        if (tid == 0 && issue) {
            for (int ks = 0; ks < ksteps; ks++) {
                const uint64_t ad = tc_desc(smem_u32(opA) + ks * 256), bd = tc_desc(smem_u32(opB) + ks * 256);
                asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(ks));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&mbar)));
        }
        // ---- bounded wait for the MMA (phase pp & 1)
        uint32_t done = 0;
        const int polls = issue ? (1 << 24) : (1 << 10);   // short only where nothing was issued
        for (int it = 0; it < polls && !done; it++)
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                         " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(&mbar)), "r"((uint32_t)(pp & 1)));
        ok = __syncthreads_and(done) != 0;           // one decision for the whole block
        if (!ok) {
            if (tid == 0) atomicExch(status, PM_ETIMEOUT);
            // MMAs that were issued may still write tensor memory: before it is freed, wait
            // (bounded again) for their commit; past that second limit the block frees it
            // anyway so that the SM's tensor memory is not held forever, and the context's
            // tensor memory contents are undefined (PM_ETIMEOUT is already recorded)
            if (issue)
                for (int it = 0; it < (1 << 24) && !done; it++)
                    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                                 " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(&mbar)), "r"((uint32_t)(pp & 1)));
            __syncthreads();
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- epilogue: warp w reads tensor-memory lanes 32w..32w+31 (rows 4i + u, i = 8w + lane/4)
        {
            u32 d[N];
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 32) {
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                             "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                             : "=r"(d[c0 + 0]), "=r"(d[c0 + 1]), "=r"(d[c0 + 2]), "=r"(d[c0 + 3]), "=r"(d[c0 + 4]),
                               "=r"(d[c0 + 5]), "=r"(d[c0 + 6]), "=r"(d[c0 + 7]), "=r"(d[c0 + 8]), "=r"(d[c0 + 9]),
                               "=r"(d[c0 + 10]), "=r"(d[c0 + 11]), "=r"(d[c0 + 12]), "=r"(d[c0 + 13]), "=r"(d[c0 + 14]),
                               "=r"(d[c0 + 15]), "=r"(d[c0 + 16]), "=r"(d[c0 + 17]), "=r"(d[c0 + 18]), "=r"(d[c0 + 19]),
                               "=r"(d[c0 + 20]), "=r"(d[c0 + 21]), "=r"(d[c0 + 22]), "=r"(d[c0 + 23]), "=r"(d[c0 + 24]),
                               "=r"(d[c0 + 25]), "=r"(d[c0 + 26]), "=r"(d[c0 + 27]), "=r"(d[c0 + 28]), "=r"(d[c0 + 29]),
                               "=r"(d[c0 + 30]), "=r"(d[c0 + 31])
                             : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            const int i = 8 * warp + (lane >> 2);
#pragma unroll
            for (int c = 0; c < KP; c++) {
                const u64 S = (u64)f32_to_u(d[c]) + ((u64)f32_to_u(d[KP + c]) << 8) +
                              ((u64)f32_to_u(d[2 * KP + c]) << 16) + ((u64)f32_to_u(d[3 * KP + c]) << 24);
                const u32 hi = (u32)(S >> 32), lo = (u32)S;
                u32 s = shoup_mul(hi, r32, r32s, q) + shoup_mul(lo, 1u, ones, q);   // < 4q
                s = csub(csub(s, q2), q);
                u32 t = csub(shoup_mul(s, wu, wus, q), q);                          // times 2^(8u)
                t = csub(t + __shfl_xor_sync(0xffffffffu, t, 1), q);
                t = csub(t + __shfl_xor_sync(0xffffffffu, t, 2), q);
                if (u == 0 && i < m && c < k) outC[(i * k + c) * TC_PTS + pp] = t;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    // ---- write the 8 points of every output entry (32 bytes each)
    if (ok)
        for (int x = tid; x < m * k * 2; x += TC_THREADS) {
            const int e = x >> 1, h = x & 1;
            *(uint4 *)(J.C + (i64)e * L + j0 + 4 * h) = *(const uint4 *)(outC + e * TC_PTS + 4 * h);
        }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N < 32 ? 32 : N));
}

static size_t tc_smem() { return 16384 + 3 * 1024 * TC_PTS * 4; }   // operands + raw A, raw B, staged C

bool tc_supported(const PwJob &j) { return j.m <= 32 && j.n <= 32 && j.k <= 32 && j.L >= 16; }

cudaError_t launch_pointwise_tc(const JobPack<PwJob> &pk, int *status, cudaStream_t st, long long *launches,
                                int withhold)
{
    int kmax = 0;
    for (int i = 0; i < pk.njobs; i++) kmax = pk.jobs[i].k > kmax ? pk.jobs[i].k : kmax;
    const size_t sm = tc_smem();
    if (kmax <= 16) {
        cudaFuncSetAttribute(k_pointwise_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_pointwise_tc<16><<<pk.blk_start[pk.njobs], TC_THREADS, sm, st>>>(pk, status, withhold);
    } else {
        cudaFuncSetAttribute(k_pointwise_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_pointwise_tc<32><<<pk.blk_start[pk.njobs], TC_THREADS, sm, st>>>(pk, status, withhold);
    }
    ++*launches;
    return cudaGetLastError();
}
