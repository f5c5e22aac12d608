// ntt.cu -- batched number-theoretic transforms over NTT primes q < 2^30.
//
// Evaluation / interpolation at roots of unity (Sec. 2, "Polynomial matrix
// multiplication": "For FFT primes, we use evaluation/interpolation at roots
// of unity").  Design for sm_103a:
//  * Forward: Gentleman-Sande (decimation in frequency), natural order in,
//    bit-reversed order out.  Inverse: Cooley-Tukey (decimation in time),
//    bit-reversed order in, natural order out.  Pointwise products do not care
//    about the order of the points, so no bit-reversal pass exists.
//  * Each thread owns 16 values and runs 4 butterfly stages in registers
//    (radix 16); passes exchange data through padded shared memory.  The first
//    forward pass reads the caller's coefficients directly (reduction mod q and
//    zero padding fused), the last inverse pass writes the requested slice
//    directly (scaling by L^-1 fused).
//  * Transforms longer than 2^13 points: a column kernel runs the top stages
//    on 32-column tiles (coalesced rows), the block kernel the bottom 13.
//  * Twiddles: one table per prime, twf[h + r] = omega_{2h}^r with its Shoup
//    companion, so every stage reads a contiguous run and any transform length
//    shares the same table.
#include "common.cuh"

__device__ __forceinline__ int spad(int x) { return x + (x >> 5); }

// ------------------------------------------------------------------ tables
struct Roots {
    u32 f[PM_MAX_LOG2L + 1];   // f[l]: primitive 2^l-th root of unity
    u32 i[PM_MAX_LOG2L + 1];   // its inverse
};

__device__ __forceinline__ u32 powmod32(u32 a, u32 e, u32 q)
{
    u64 r = 1, b = a;
    while (e) {
        if (e & 1) r = r * b % q;
        b = b * b % q;
        e >>= 1;
    }
    return (u32)r;
}

__global__ void k_twiddles(uint2 *twf, uint2 *twi, u32 q, Roots roots, int maxlog)
{
    const int n = 1 << maxlog;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x + 1; e < n; e += gridDim.x * blockDim.x) {
        int l = 31 - __clz(e);            // h = 2^l
        u32 r = (u32)e - (1u << l);
        u32 wf = powmod32(roots.f[l + 1], r, q);
        u32 wi = powmod32(roots.i[l + 1], r, q);
        twf[e] = make_uint2(wf, (u32)(((u64)wf << 32) / q));
        twi[e] = make_uint2(wi, (u32)(((u64)wi << 32) / q));
    }
}

cudaError_t launch_twiddles(uint2 *twf, uint2 *twi, u32 q, const u32 *rf, const u32 *ri, int maxlog,
                            cudaStream_t st, long long *launches)
{
    Roots R;
    for (int l = 0; l <= PM_MAX_LOG2L; l++) { R.f[l] = rf[l]; R.i[l] = ri[l]; }
    int n = 1 << maxlog;
    int grid = (n + 255) / 256;
    if (grid > 4096) grid = 4096;
    k_twiddles<<<grid, 256, 0, st>>>(twf, twi, q, R, maxlog);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ loads
// Load one coefficient and bring it into [0, 2q) (user data: [0, q)).
__device__ __forceinline__ u32 load_coeff(const void *src, int mode, i64 idx, const PrimeDev &P)
{
    if (mode == 8) return reduce64(__ldg((const u64 *)src + idx), P);
    u32 x = __ldg((const u32 *)src + idx);
    if (mode == 4) return csub(shoup_mul(x, 1u, P.ones, P.q), P.q);
    return x;
}

// Radix-2^r group of the forward (DIF) transform: stages with half sizes
// lo*2^(r-1), ..., lo.  v[o + j] holds point base + j*lo; gl = base mod lo.
template <int r>
__device__ __forceinline__ void grp_dif(u32 (&v)[16], int o, int gl, int lo, const uint2 *__restrict__ tw,
                                        u32 q, u32 q2)
{
    constexpr int R = 1 << r;
#pragma unroll
    for (int i = 0; i < r; i++) {
        const int lh = R >> (i + 1);
        const uint2 *t = tw + lo * lh + gl;
#pragma unroll
        for (int jj = 0; jj < lh; jj++) {
            const uint2 w = __ldg(t + jj * lo);
#pragma unroll
            for (int b = 0; b < R; b += 2 * lh) bfly_dif(v[o + b + jj], v[o + b + jj + lh], w, q, q2);
        }
    }
}

// Inverse (DIT) group: the same pairs, half sizes lo, 2lo, ..., lo*2^(r-1).
template <int r>
__device__ __forceinline__ void grp_dit(u32 (&v)[16], int o, int gl, int lo, const uint2 *__restrict__ tw,
                                        u32 q, u32 q2)
{
    constexpr int R = 1 << r;
#pragma unroll
    for (int i = r - 1; i >= 0; i--) {
        const int lh = R >> (i + 1);
        const uint2 *t = tw + lo * lh + gl;
#pragma unroll
        for (int jj = 0; jj < lh; jj++) {
            const uint2 w = __ldg(t + jj * lo);
#pragma unroll
            for (int b = 0; b < R; b += 2 * lh) bfly_dit(v[o + b + jj], v[o + b + jj + lh], w, q, q2);
        }
    }
}

__device__ __forceinline__ int find_job(const int *blk_start, int b)
{
    int j = 0;
    while (b >= blk_start[j + 1]) j++;
    return j;
}

// ------------------------------------------------------------------ forward, block
// First pass of radix 2^r (r = 1..4): groups g + j*lo with lo = L >> r; each
// thread takes 16 >> r groups.  Reads the source, writes shared memory (or
// the destination when this pass is also the last one, L = 16).
template <int r>
__device__ __forceinline__ void fwd_first(u32 (&v)[16], u32 *X, const FwdJob &J, i64 e, bool act, int lg,
                                          int tid, int tpt)
{
    constexpr int R = 1 << r;
    const int L = 1 << lg, lo = L >> r;
    const u32 q = J.P.q, q2 = J.P.q2;
    const char *src = (const char *)J.src;
    const i64 sb = e * J.src_stride;
#pragma unroll
    for (int it = 0; it < (16 >> r); it++) {
        const int g = tid + it * tpt;
#pragma unroll
        for (int j = 0; j < R; j++) {
            const int x = g + j * lo;
            v[it * R + j] = (act && x < J.src_len) ? load_coeff(src, J.src_mode, sb + x, J.P) : 0u;
        }
        grp_dif<r>(v, it * R, g & (lo - 1), lo, J.P.twf, q, q2);
    }
    if (lg == r) {   // single pass (L = 16): final values, contiguous
        if (act) {
            u32 *d = J.dst + e * J.dst_stride;
#pragma unroll
            for (int j = 0; j < 16; j++) d[j] = csub(v[j], q);
        }
        return;
    }
#pragma unroll
    for (int it = 0; it < (16 >> r); it++) {
        const int g = tid + it * tpt;
#pragma unroll
        for (int j = 0; j < R; j++) X[spad(g + j * lo)] = v[it * R + j];
    }
}

__global__ void __launch_bounds__(512, 3) k_ntt_fwd_block(const __grid_constant__ JobPack<FwdJob> pk, int lg)
{
    extern __shared__ u32 sm[];
    const int b = blockIdx.x;
    const int jb = find_job(pk.blk_start, b);
    const FwdJob &J = pk.jobs[jb];
    const int L = 1 << lg, tpt = L >> 4, tpb = blockDim.x / tpt;
    const int lt = threadIdx.x / tpt, tid = threadIdx.x - lt * tpt;
    const i64 e = (i64)(b - pk.blk_start[jb]) * tpb + lt;
    const bool act = e < J.count;
    u32 *X = sm + lt * (L + (L >> 5));
    const u32 q = J.P.q, q2 = J.P.q2;
    u32 v[16];

    const int b0 = ((lg - 1) & 3) + 1;
    switch (b0) {
    case 1: fwd_first<1>(v, X, J, e, act, lg, tid, tpt); break;
    case 2: fwd_first<2>(v, X, J, e, act, lg, tid, tpt); break;
    case 3: fwd_first<3>(v, X, J, e, act, lg, tid, tpt); break;
    default: fwd_first<4>(v, X, J, e, act, lg, tid, tpt); break;
    }
    if (lg == b0) return;
    for (int s0 = b0; s0 < lg; s0 += 4) {
        __syncthreads();
        const int llo = lg - s0 - 4, lo = 1 << llo;
        const int g = tid, gl = g & (lo - 1);
        const int base = ((g >> llo) << (llo + 4)) + gl;
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = X[spad(base + j * lo)];
        grp_dif<4>(v, 0, gl, lo, J.P.twf, q, q2);
        if (llo == 0) {
            if (act) {
                uint4 *d = (uint4 *)(J.dst + e * J.dst_stride + base);
#pragma unroll
                for (int j = 0; j < 4; j++)
                    d[j] = make_uint4(csub(v[4 * j], q), csub(v[4 * j + 1], q), csub(v[4 * j + 2], q),
                                      csub(v[4 * j + 3], q));
            }
        } else {
            // each thread writes back exactly the points it read: no barrier needed here
#pragma unroll
            for (int j = 0; j < 16; j++) X[spad(base + j * lo)] = v[j];
        }
    }
}

// ------------------------------------------------------------------ inverse, block
__device__ __forceinline__ void store_out(const InvJob &J, i64 e, int x, u32 val)
{
    if (J.dst_mode == 0) {
        ((u32 *)J.dst)[e * J.dst_stride + x] = val;
        return;
    }
    const int t = x - J.out_off;
    if (t < 0 || t >= J.out_len) return;
    u32 y = csub(shoup_mul(val, J.P.linv, J.P.linvs, J.P.q), J.P.q);
    if (J.dst_mode == 8) ((u64 *)J.dst)[e * J.dst_stride + t] = y;
    else ((u32 *)J.dst)[e * J.dst_stride + t] = y;
}

template <int r>
__device__ __forceinline__ void inv_last(u32 (&v)[16], const u32 *X, const InvJob &J, i64 e, bool act, int lg,
                                         int tid, int tpt, bool from_regs)
{
    constexpr int R = 1 << r;
    const int L = 1 << lg, lo = L >> r;
    const u32 q = J.P.q, q2 = J.P.q2;
#pragma unroll
    for (int it = 0; it < (16 >> r); it++) {
        const int g = tid + it * tpt;
        if (!from_regs) {
#pragma unroll
            for (int j = 0; j < R; j++) v[it * R + j] = X[spad(g + j * lo)];
        }
        grp_dit<r>(v, it * R, g & (lo - 1), lo, J.P.twi, q, q2);
        if (act) {
#pragma unroll
            for (int j = 0; j < R; j++) store_out(J, e, g + j * lo, v[it * R + j]);
        }
    }
}

__global__ void __launch_bounds__(512, 3) k_ntt_inv_block(const __grid_constant__ JobPack<InvJob> pk, int lg)
{
    extern __shared__ u32 sm[];
    const int b = blockIdx.x;
    const int jb = find_job(pk.blk_start, b);
    const InvJob &J = pk.jobs[jb];
    const int L = 1 << lg, tpt = L >> 4, tpb = blockDim.x / tpt;
    const int lt = threadIdx.x / tpt, tid = threadIdx.x - lt * tpt;
    const i64 e = (i64)(b - pk.blk_start[jb]) * tpb + lt;
    const bool act = e < J.count;
    u32 *X = sm + lt * (L + (L >> 5));
    const u32 q = J.P.q, q2 = J.P.q2;
    u32 v[16];
    const int b0 = ((lg - 1) & 3) + 1;

    if (lg == b0) {   // L = 16: one radix-16 pass straight from the source
        const u32 *s = J.src + e * J.src_stride;
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = act ? s[j] : 0u;
        inv_last<4>(v, X, J, e, act, lg, tid, tpt, true);
        return;
    }
    // radix-16 passes, lo = 1, 16, 256, ... over the low lg - b0 stages
    for (int s0 = 0; s0 < lg - b0; s0 += 4) {
        const int llo = s0, lo = 1 << llo;
        const int g = tid, gl = g & (lo - 1);
        const int base = ((g >> llo) << (llo + 4)) + gl;
        if (s0 == 0) {
            if (act) {
                const uint4 *s = (const uint4 *)(J.src + e * J.src_stride + base);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    uint4 t = s[j];
                    v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = 0u;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = X[spad(base + j * lo)];
        }
        grp_dit<4>(v, 0, gl, lo, J.P.twi, q, q2);
#pragma unroll
        for (int j = 0; j < 16; j++) X[spad(base + j * lo)] = v[j];
        __syncthreads();
    }
    switch (b0) {
    case 1: inv_last<1>(v, X, J, e, act, lg, tid, tpt, false); break;
    case 2: inv_last<2>(v, X, J, e, act, lg, tid, tpt, false); break;
    case 3: inv_last<3>(v, X, J, e, act, lg, tid, tpt, false); break;
    default: inv_last<4>(v, X, J, e, act, lg, tid, tpt, false); break;
    }
}

int fwd_block_threads(int lg)
{
    const int tpt = (1 << lg) >> 4;
    return tpt >= 256 ? tpt : 256;
}

static int block_smem(int lg, int threads)
{
    const int L = 1 << lg, tpt = L >> 4, tpb = threads / tpt;
    return tpb * (L + (L >> 5)) * (int)sizeof(u32);
}

template <typename Pack>
static int pack_blocks(const Pack &pk) { return pk.blk_start[pk.njobs]; }

cudaError_t launch_ntt_fwd_block(const JobPack<FwdJob> &pk, int lg, cudaStream_t st, long long *launches)
{
    const int th = fwd_block_threads(lg), sm = block_smem(lg, th);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_ntt_fwd_block, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    k_ntt_fwd_block<<<pack_blocks(pk), th, sm, st>>>(pk, lg);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_ntt_inv_block(const JobPack<InvJob> &pk, int lg, cudaStream_t st, long long *launches)
{
    const int th = fwd_block_threads(lg), sm = block_smem(lg, th);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_ntt_inv_block, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    k_ntt_inv_block<<<pack_blocks(pk), th, sm, st>>>(pk, lg);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ column passes
// Transform length L = 2^lg > 2^13: R1 = L / 2^13 rows per column.  A block takes
// a tile of TC = 4096 / R1 consecutive columns (at least 32) and all R1 rows, so
// every tile holds 4096 points; rows of a tile are contiguous runs of TC words.
#define COLS_POINTS 4096

__host__ __device__ __forceinline__ int cols_tile(int lg)
{
    const int r1 = 1 << (lg - PM_LB_LOG2);
    const int tc = COLS_POINTS / r1;
    return tc < 32 ? 32 : tc;
}

int blocks_per_entry_cols(int lg) { return (1 << PM_LB_LOG2) / cols_tile(lg); }

__global__ void __launch_bounds__(256) k_ntt_fwd_cols(const __grid_constant__ JobPack<ColJob> pk, int lg)
{
    extern __shared__ u32 sm[];
    const int b = blockIdx.x;
    const int jb = find_job(pk.blk_start, b);
    const ColJob &J = pk.jobs[jb];
    const int TC = cols_tile(lg), tiles = (1 << PM_LB_LOG2) / TC;
    const int rel = b - pk.blk_start[jb];
    const i64 e = rel / tiles;
    const int c0 = (rel % tiles) * TC;
    const int R1 = 1 << (lg - PM_LB_LOG2), LB = 1 << PM_LB_LOG2;
    const u32 q = J.P.q, q2 = J.P.q2;
    const char *src = (const char *)J.src;
    const i64 sb = e * J.src_stride;

    for (int idx = threadIdx.x; idx < R1 * TC; idx += blockDim.x) {
        const int row = idx / TC, cc = idx % TC;
        const int x = c0 + cc + row * LB;
        sm[idx] = x < J.src_len ? load_coeff(src, J.mode, sb + x, J.P) : 0u;
    }
    __syncthreads();
    for (int hr = R1 >> 1; hr >= 1; hr >>= 1) {
        const int h = hr * LB;
        for (int bi = threadIdx.x; bi < (R1 >> 1) * TC; bi += blockDim.x) {
            const int cc = bi % TC, pj = bi / TC;
            const int jj = pj & (hr - 1), j0 = ((pj / hr) * 2 * hr) + jj;
            const uint2 w = __ldg(J.P.twf + h + c0 + cc + jj * LB);
            bfly_dif(sm[j0 * TC + cc], sm[(j0 + hr) * TC + cc], w, q, q2);
        }
        __syncthreads();
    }
    u32 *d = (u32 *)J.dst + e * J.dst_stride;
    for (int idx = threadIdx.x; idx < R1 * TC; idx += blockDim.x) {
        const int row = idx / TC, cc = idx % TC;
        d[c0 + cc + row * LB] = sm[idx];
    }
}

__global__ void __launch_bounds__(256) k_ntt_inv_cols(const __grid_constant__ JobPack<ColJob> pk, int lg)
{
    extern __shared__ u32 sm[];
    const int b = blockIdx.x;
    const int jb = find_job(pk.blk_start, b);
    const ColJob &J = pk.jobs[jb];
    const int TC = cols_tile(lg), tiles = (1 << PM_LB_LOG2) / TC;
    const int rel = b - pk.blk_start[jb];
    const i64 e = rel / tiles;
    const int c0 = (rel % tiles) * TC;
    const int R1 = 1 << (lg - PM_LB_LOG2), LB = 1 << PM_LB_LOG2;
    const u32 q = J.P.q, q2 = J.P.q2;
    const u32 *s = (const u32 *)J.src + e * J.src_stride;

    for (int idx = threadIdx.x; idx < R1 * TC; idx += blockDim.x) {
        const int row = idx / TC, cc = idx % TC;
        sm[idx] = s[c0 + cc + row * LB];
    }
    __syncthreads();
    for (int hr = 1; hr < R1; hr <<= 1) {
        const int h = hr * LB;
        for (int bi = threadIdx.x; bi < (R1 >> 1) * TC; bi += blockDim.x) {
            const int cc = bi % TC, pj = bi / TC;
            const int jj = pj & (hr - 1), j0 = ((pj / hr) * 2 * hr) + jj;
            const uint2 w = __ldg(J.P.twi + h + c0 + cc + jj * LB);
            bfly_dit(sm[j0 * TC + cc], sm[(j0 + hr) * TC + cc], w, q, q2);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < R1 * TC; idx += blockDim.x) {
        const int row = idx / TC, cc = idx % TC;
        const int x = c0 + cc + row * LB;
        const int t = x - J.out_off;
        if (t < 0 || t >= J.out_len) continue;
        u32 y = csub(shoup_mul(sm[idx], J.P.linv, J.P.linvs, q), q);
        if (J.mode == 8) ((u64 *)J.dst)[e * J.dst_stride + t] = y;
        else ((u32 *)J.dst)[e * J.dst_stride + t] = y;
    }
}

cudaError_t launch_ntt_fwd_cols(const JobPack<ColJob> &pk, int lg, cudaStream_t st, long long *launches)
{
    const int sm = (1 << (lg - PM_LB_LOG2)) * cols_tile(lg) * (int)sizeof(u32);
    k_ntt_fwd_cols<<<pack_blocks(pk), 256, sm, st>>>(pk, lg);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_ntt_inv_cols(const JobPack<ColJob> &pk, int lg, cudaStream_t st, long long *launches)
{
    const int sm = (1 << (lg - PM_LB_LOG2)) * cols_tile(lg) * (int)sizeof(u32);
    k_ntt_inv_cols<<<pack_blocks(pk), 256, sm, st>>>(pk, lg);
    ++*launches;
    return cudaGetLastError();
}
