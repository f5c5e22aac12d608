// tc_pointwise.cu -- pointwise matrix products on the tensor cores (tcgen05).
//
// At every transform point j, C_j = A_j B_j mod q (Sec. 2, "Polynomial matrix
// multiplication": the n^omega d term), for m, n, k <= 32.  GB300 has no
// integer tensor MMA (.kind::i8 does not exist for sm_103a), so residues are
// split into small signed digits that fp16 holds exactly and the products run
// as tcgen05.mma of kind::f16 with fp32 accumulation in tensor memory.
//
// Digits.  A residue r in [0, q), q < 2^30, is written r = sum_x d_x 256^x with
// balanced digits d_0..d_2 in [-128, 127] and d_3 in [0, 64]: the bytes of
// t = r + 0x80808080 minus 128 (no carry leaves t, since r + 0x80808080 <
// 2^32).  A digit is made fp16 from its biased byte b as the bit pattern
// 0x6400 | b (= 1024 + b) minus 1152, exactly.
//
// Weights summed in the MMA.  With A = sum_x 256^x A_x and B = sum_y 256^y B_y,
//     A B = sum_w 256^w E_w,   E_w = sum_{x+y=w} A_x B_y,   w = 0..6.
// Digit products are at most 2^14 in magnitude; E_w has at most 4 x n <= 128
// of them, so |E_w| <= 2^21 and every partial sum of the fp32 accumulation is
// an integer below 2^24: the sums are exact.  The MMA for digit x of A takes
// B's four digit blocks side by side, [B_0 B_1 B_2 B_3] (N = 128), and writes
// tensor-memory columns [32x, 32x + 128): block y lands on E_(x+y).  Seven
// accumulators of 32 columns hold E_0..E_6.
//
// Four points per MMA.  An MMA has M = 128 rows, a 32 x 32 product only 32:
// the 128 rows of the A operand are the rows of four consecutive points
// (row 32 pt + i), and the MMA for point pt uses point pt's B with the
// instruction's disable-output-lane mask set for every lane outside quarter
// pt, so only lanes 32 pt .. 32 pt + 31 accumulate.  Lane quarter pt is read
// by warps pt and pt + 4, which therefore own point pt's outputs.
//
// Epilogue.  An exact fp32 integer |v| <= 2^22 plus 1.5 2^23 has the bit
// pattern 0x4B400000 + v, so E_w costs one FADD.  C = sum_w (256^w mod q) E_w
// is formed with 64-bit multiply-adds (|C| < 2^54, offset by q 2^25 to stay
// positive) and reduced mod q once.  The accumulators are then cleared with
// tcgen05.st for the next tile.
//
// Work split.  A CTA (256 threads, two per SM: 112 KB of shared memory and 256
// tensor-memory columns each) loops over tiles of four points, in half-tiles
// of 16 inner-dimension entries (one MMA K-step each).  The residues of a tile
// (16 bytes per entry) arrive by cp.async in a staging buffer while the
// previous tile runs.  The operands of consecutive half-tiles alternate
// between two stage buffers, so the digits of half-tile q + 1 are written
// while the MMAs of half-tile q run.  For a half-tile every thread takes 8
// consecutive inner-dimension entries of one row of A (or one column of B):
// digits, one 16-byte shared-memory store per point and digit in the
// no-swizzle K-major core-matrix layout.  One thread issues the MMAs and commits them to an
// mbarrier; the wait is bounded (PM_ETIMEOUT), and after a timeout with MMAs in
// flight the block waits again (bounded) for their commit before it frees the
// tensor memory.  Outputs go through shared memory and leave as one 16-byte
// store per entry (four points).
#include <cuda_fp16.h>

#include "common.cuh"
#include "pmat.h"

#define TC_PTS 4           // points per tile (one MMA group)
#define TC_THREADS 256     // eight warps: two per tensor-memory lane quarter
#define TC_COLS 256        // tensor-memory columns allocated (7 x 32 used)
#define TC_HALF 16384      // one operand tile of a half-tile: 128 rows x 16 K fp16 x 4 tiles
#define TC_STAGE (2 * TC_HALF)   // A (4 digits) and B (4 points) of one half-tile
#define TC_RAW 32768       // residues of a tile: 2048 entries x 16 bytes (XOR-swizzled slots)
#define TC_OUTB 16384      // staged outputs [point][row][column ^ row], 4 x 32 x 32 words
#define TC_SMEM (2 * TC_STAGE + TC_RAW + TC_OUTB)

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row r, inner index 8 kk8 .. 8 kk8 + 7) in a 128 x 16 fp16 tile, K-major, no
// swizzle: 8-row x 16-byte core matrices, LBO = 128 B between the two K-adjacent ones, SBO =
// 256 B between 8-row groups
__device__ __forceinline__ int op_off(int r, int kk8) { return (r >> 3) * 256 + kk8 * 128 + (r & 7) * 16; }

__device__ __forceinline__ uint64_t op_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           (1ull << 46);
}

// 16-byte slot of staged entry e (A entries first, then B): the low three bits XORed with bits
// 3..5 and 6..8, so the octet reads of a warp (and the cp.async writes) spread evenly over the
// eight 16-byte bank groups
__device__ __forceinline__ int raw_slot(int e) { return e ^ (((e >> 3) ^ (e >> 6)) & 7); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
}

__device__ __forceinline__ int find_tile_job(const JobPack<PwJob> &pk, int tile)
{
    int jb = 0;
    while (tile >= pk.blk_start[jb + 1]) jb++;
    return jb;
}

// residues of points j0 .. j0 + 3 of every entry of A and B into the staging buffer
__device__ __forceinline__ void prefetch_tile(const JobPack<PwJob> &pk, int tile, unsigned char *raw, int tid)
{
    const PwJob &J = pk.jobs[find_tile_job(pk, tile)];
    const int eA = J.m * J.n, eT = eA + J.n * J.k, j0 = (tile - pk.blk_start[find_tile_job(pk, tile)]) * TC_PTS;
    for (int e = tid; e < eT; e += TC_THREADS) {
        const u32 *src = e < eA ? J.A + (i64)e * J.L : J.B + (i64)(e - eA) * J.L;
        cp_async16(smem_u32(raw + raw_slot(e) * 16), src + j0);
    }
    asm volatile("cp.async.commit_group;");
}

// fp16 pair of digit x of two biased residues: bytes x of t0 and t1 as 0x6400 | byte, minus 1152
__device__ __forceinline__ uint32_t digit_pair(uint32_t t0, uint32_t t1, uint32_t sel)
{
    uint32_t w;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(w) : "r"(t0), "r"(t1), "r"(sel));
    w = (w & 0x00FF00FFu) | 0x64006400u;
    const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&w), __halves2half2(__ushort_as_half(0x6480),
                                                                                      __ushort_as_half(0x6480)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// digits of half-tile h (inner entries 16 h .. 16 h + 15) into one stage buffer
__device__ __forceinline__ void produce_half(const PwJob &J, const unsigned char *raw, unsigned char *stage, int h,
                                             int tid)
{
    const int m = J.m, n = J.n, k = J.k;
    unsigned char *opA = stage, *opB = stage + TC_HALF;
    for (int o = tid; o < 2 * (m + k); o += TC_THREADS) {
        const bool isA = o < 2 * m;
        const int rc = (isA ? o : o - 2 * m) >> 1, oct = o & 1;   // row i of A or column c of B; octet
        const int l0 = 16 * h + 8 * oct;
        uint4 v[8];
#pragma unroll
        for (int t = 0; t < 8; t++) {
            const int l = l0 + t;
            v[t] = make_uint4(0, 0, 0, 0);                     // entries l >= n are zero digits
            if (l < n) v[t] = *(const uint4 *)(raw + raw_slot(isA ? rc * n + l : m * n + l * k + rc) * 16);
        }
#pragma unroll
        for (int pt = 0; pt < TC_PTS; pt++) {
            u32 t8[8];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const u32 r = pt == 0 ? v[t].x : pt == 1 ? v[t].y : pt == 2 ? v[t].z : v[t].w;
                t8[t] = r + 0x80808080u;                       // transforms are in [0, q)
            }
#pragma unroll
            for (int x = 0; x < 4; x++) {
                // prmt selector nibbles (nibble j picks result byte j from {t1, t0}, 4..7 = t1):
                // bytes 0 and 2 are byte x of t0 and byte x of t1 (bytes 1 and 3 are masked off)
                const u32 sel = (u32)x | ((u32)x << 4) | ((u32)(4 + x) << 8) | ((u32)(4 + x) << 12);
                uint4 hv;
                hv.x = digit_pair(t8[0], t8[1], sel);
                hv.y = digit_pair(t8[2], t8[3], sel);
                hv.z = digit_pair(t8[4], t8[5], sel);
                hv.w = digit_pair(t8[6], t8[7], sel);
                // A: tile of digit x, row 32 pt + i; B: tile of point pt, row 32 x + c
                unsigned char *dst = isA ? opA + x * 4096 + op_off(32 * pt + rc, oct)
                                         : opB + pt * 4096 + op_off(32 * x + rc, oct);
                *(uint4 *)dst = hv;
            }
        }
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int polls)
{
    uint32_t done = 0;
    for (int it = 0; it < polls && !done; it++)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(bar), "r"(parity));
    return done != 0;
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t *d)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7])
                 : "r"(addr));
}

__device__ __forceinline__ void tmem_zero16(uint32_t addr)
{
    const uint32_t z = 0;
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};"
                 ::"r"(addr), "r"(z));
}

// one MMA: D[lanes of quarter pt, columns col ..] += A . B, K = 16
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, int pt)
{
    const uint32_t on = 0u, off = 0xFFFFFFFFu;
    const uint32_t m0 = pt == 0 ? on : off, m1 = pt == 1 ? on : off, m2 = pt == 2 ? on : off, m3 = pt == 3 ? on : off;
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, 1, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, {%4, %5, %6, %7}, p;\n}\n"
                 ::"r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(m0), "r"(m1), "r"(m2), "r"(m3));
}

// the 16 MMAs of a half-tile, committed to the stage's mbarrier (one thread)
__device__ __forceinline__ void issue_half(uint32_t tmem, const unsigned char *stage, uint32_t idesc, uint32_t bar)
{
    for (int pt = 0; pt < TC_PTS; pt++)
        for (int x = 0; x < 4; x++)
            mma_f16(tmem + 32u * x, op_desc(smem_u32(stage + x * 4096)), op_desc(smem_u32(stage + TC_HALF + pt * 4096)),
                    idesc, pt);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

__device__ __forceinline__ void sync_stage()
{
    asm volatile("fence.proxy.async.shared::cta;");     // generic-proxy stores seen by the MMAs
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

}  // namespace

int tc_blocks(const PwJob &j) { return j.L / TC_PTS; }

__global__ void __launch_bounds__(TC_THREADS, 2) k_pointwise_tc(const __grid_constant__ JobPack<PwJob> pk, int *status,
                                                                 int withhold)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    unsigned char *raw = sm + 2 * TC_STAGE;
    u32 *outC = (u32 *)(sm + 2 * TC_STAGE + TC_RAW);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, chalf = warp >> 2;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t tq = tmem + ((uint32_t)(32 * quarter) << 16) + 16u * chalf;   // this warp's lanes, column half
#pragma unroll
    for (int w = 0; w < 7; w++) tmem_zero16(tq + 32u * w);
    asm volatile("tcgen05.wait::st.sync.aligned;");
    // D f32 (bit 4), A and B fp16 (formats 0), both K-major; N = 128 (>> 3 at bit 17), M = 128 (>> 4 at bit 24)
    const uint32_t idesc = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

    const int ntiles = pk.blk_start[pk.njobs];
    if (blockIdx.x >= ntiles) {
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
        return;
    }
    // Half-stage q (half h of tile t) uses stage buffer q & 1 and commits to mbar[q & 1]; with
    // nph[s] the commits made to mbar[s] so far, the latest one completes the phase of parity
    // (nph[s] - 1) & 1.  The test hook's withheld first half-stage counts as a commit that never
    // arrives (its wait must run out); rc[s] counts the commits really issued.
    // bit b of `odd` = nph[b] & 1, bit b of `real` = (rc[b] > 0)
    uint32_t odd = 0, real = 0;
    int qs = 0;                               // half-stages issued
    bool ok = true, inflight = false;
    // prologue: the first tile's residues, its first half's digits and MMAs
    int tile = blockIdx.x;
    prefetch_tile(pk, tile, raw, tid);
    asm volatile("cp.async.wait_all;");
    __syncthreads();
    {
        const PwJob &J = pk.jobs[find_tile_job(pk, tile)];
        produce_half(J, raw, sm, 0, tid);
        sync_stage();
        if ((J.n + 15) >> 4 == 1 && tile + (int)gridDim.x < ntiles) prefetch_tile(pk, tile + gridDim.x, raw, tid);
        const bool issue = !(withhold && blockIdx.x == 0);
        if (tid == 0 && issue) issue_half(tmem, sm, idesc, smem_u32(&mbar[0]));
        odd = 1;
        real = issue ? 1 : 0;
        inflight = issue;
        qs = 1;
    }
    int cur = -1;
    u32 cw[7] = {0, 0, 0, 0, 0, 0, 0};
    u64 k0 = 0;
    int h = 0;                                // the half of `tile` last issued
    while (true) {
        const PwJob &J = pk.jobs[find_tile_job(pk, tile)];
        const int ksteps = (J.n + 15) >> 4;
        const int q = qs - 1, s = q & 1;      // the half-stage in flight
        const bool last = h == ksteps - 1;
        // ---- the next half-stage: (tile, h + 1) or (next tile, 0)
        const int ntile = last ? tile + (int)gridDim.x : tile;
        const int nh = last ? 0 : h + 1;
        const bool has_next = ntile < ntiles;
        if (has_next) {
            if (last) {                       // the next tile's residues (prefetched) must have landed
                asm volatile("cp.async.wait_all;");
                __syncthreads();
            }
            // stage buffer s ^ 1 is free once half-stage q - 1 has completed
            if (q >= 1) {
                const bool withheld = withhold && blockIdx.x == 0 && q == 1;   // half-stage 0 had no MMAs
                bool fin = mbar_wait(smem_u32(&mbar[s ^ 1]), ((odd >> (s ^ 1)) & 1) ^ 1, withheld ? (1 << 10) : (1 << 24));
                fin = __syncthreads_and(fin) != 0;
                if (!fin) { ok = false; break; }
            }
            const PwJob &NJ = pk.jobs[find_tile_job(pk, ntile)];
            produce_half(NJ, raw, sm + (s ^ 1) * TC_STAGE, nh, tid);
            sync_stage();
            // the staging buffer is free after the next tile's last half: its successor's residues
            if (nh == ((NJ.n + 15) >> 4) - 1 && ntile + (int)gridDim.x < ntiles)
                prefetch_tile(pk, ntile + gridDim.x, raw, tid);
        }
        if (last) {
            // ---- epilogue of `tile` once its last half-stage has completed
            const bool waited_short = withhold && blockIdx.x == 0 && q == 0;
            bool fin = mbar_wait(smem_u32(&mbar[s]), ((odd >> s) & 1) ^ 1, waited_short ? (1 << 10) : (1 << 24));
            fin = __syncthreads_and(fin) != 0;
            if (!fin) { ok = false; break; }
            inflight = false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int m = J.m, k = J.k, L = J.L, jb = find_tile_job(pk, tile);
            const int j0 = (tile - pk.blk_start[jb]) * TC_PTS;
            if (jb != cur) {                  // per job: 256^w mod q and the folded offset
                cur = jb;
                u64 sum = 0;
#pragma unroll
                for (int w = 0; w < 7; w++) {
                    cw[w] = (u32)((1ull << (8 * w)) % J.P.q);
                    sum += cw[w];
                }
                k0 = ((u64)J.P.q << 25) - sum * 0x4B400000ull;   // q 2^25 - sum_w cw_w bits(1.5 2^23), mod 2^64
            }
            {
                const int i = lane, pt = quarter;
#pragma unroll
                for (int half = 0; half < 2; half++) {          // 8 columns at a time: 7 loads, one wait
                    uint32_t d[7][8];
#pragma unroll
                    for (int w = 0; w < 7; w++) tmem_ld8(tq + 32u * w + 8u * half, d[w]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                    for (int cc = 0; cc < 8; cc++) {
                        u64 acc = k0;
#pragma unroll
                        for (int w = 0; w < 7; w++) {
                            const u32 bits = __float_as_uint(__uint_as_float(d[w][cc]) + 12582912.0f);
                            acc += (u64)bits * cw[w];
                        }
                        const int c = 16 * chalf + 8 * half + cc;
                        if (i < m && c < k) outC[(pt * 32 + i) * 32 + (c ^ i)] = reduce64(acc, J.P);
                    }
                }
#pragma unroll
                for (int w = 0; w < 7; w++) tmem_zero16(tq + 32u * w);   // cleared for the next tile
                asm volatile("tcgen05.wait::st.sync.aligned;");
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            // ---- outputs: four points of every entry, one 16-byte store each
            for (int i = warp; i < m; i += TC_THREADS / 32)     // row i, column = lane
                if (lane < k) {
                    const int o = i * 32 + (lane ^ i);
                    *(uint4 *)(J.C + (i64)(i * k + lane) * L + j0) =
                        make_uint4(outC[o], outC[1024 + o], outC[2048 + o], outC[3072 + o]);
                }
        }
        if (!has_next) break;
        // ---- MMAs of the next half-stage (after the epilogue cleared the accumulators)
        if (tid == 0) issue_half(tmem, sm + (s ^ 1) * TC_STAGE, idesc, smem_u32(&mbar[s ^ 1]));
        odd ^= 1u << (s ^ 1);
        real |= 1u << (s ^ 1);
        inflight = true;
        qs++;
        if (last) {
            // the staged outputs are rewritten by the next epilogue only after its barrier
            __syncthreads();
        }
        tile = ntile;
        h = nh;
    }
    if (!ok) {
        if (tid == 0) atomicExch(status, PM_ETIMEOUT);
        // MMAs that were issued may still write tensor memory: wait (bounded) for their commits
        // before it is freed; past that limit it is freed anyway (contents undefined)
        if (inflight)
            for (int b = 0; b < 2; b++)
                if ((real >> b) & 1) mbar_wait(smem_u32(&mbar[b]), ((odd >> b) & 1) ^ 1, 1 << 24);
    }
    asm volatile("cp.async.wait_all;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
}

bool tc_supported(const PwJob &j) { return j.m <= 32 && j.n <= 32 && j.k <= 32 && j.L >= 16; }

cudaError_t launch_pointwise_tc(const JobPack<PwJob> &pk, int *status, cudaStream_t st, long long *launches,
                                int withhold)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
    }
    const cudaError_t e = cudaFuncSetAttribute(k_pointwise_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    const int tiles = pk.blk_start[pk.njobs];
    const int grid = tiles < 2 * sms ? tiles : 2 * sms;
    k_pointwise_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(pk, status, withhold);
    ++*launches;
    return cudaGetLastError();
}
