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
//  * Transforms longer than 2^14 points: a column kernel runs the top stages
//    on column tiles (coalesced rows), the block kernel the bottom 14.
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

// Twiddle-table entries kept in shared memory per block: the radix-16 passes of stride 16 and 1
// read entries lo h + gl + j lo < 16 lo, all below 256 and below the transform length L (lo <=
// L / 16).  A block stages min(TW_SH, L) entries: every table holds at least L (it is built for
// the longest transform of its prime so far), not necessarily 256.
#define TW_SH 256

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
// lo*2^(r-1), ..., lo.  v[o + j] holds point base + j*lo; gl = base mod lo.  SH: tw is the
// block's shared-memory copy of the table's first TW_SH entries (plain loads), else the table
// in global memory (read-only loads).
template <int r, bool SH = false>
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
            const uint2 w = SH ? t[jj * lo] : __ldg(t + jj * lo);
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
// Kernels are instantiated per transform length 2^LG (LG = 4..13), so every pass's
// stride lo is a compile-time constant: with the padded index spad(x) = x + x/32
// and a group base b (b mod lo = gl < lo, b / lo a multiple of 16),
// spad(b + j lo) = spad(b) + j lo + (j lo) / 32, i.e. immediate offsets.
template <int LO>
__device__ __forceinline__ constexpr int poff(int j) { return j * LO + ((j * LO) >> 5); }

// Coefficients x and x + 1 (x even) of an entry, as load_coeff, zero from src_len on: one
// vector load when the pair is aligned (vec) and inside the entry.
__device__ __forceinline__ void load_pair(const void *src, int mode, i64 idx, int x, int len, bool vec,
                                          const PrimeDev &P, u32 &a, u32 &b)
{
    if (vec && x + 1 < len) {
        if (mode == 8) {
            const ulonglong2 t = __ldg((const ulonglong2 *)((const u64 *)src + idx));
            a = reduce64(t.x, P);
            b = reduce64(t.y, P);
        } else {
            const uint2 t = __ldg((const uint2 *)((const u32 *)src + idx));
            a = mode == 4 ? csub(shoup_mul(t.x, 1u, P.ones, P.q), P.q) : t.x;
            b = mode == 4 ? csub(shoup_mul(t.y, 1u, P.ones, P.q), P.q) : t.y;
        }
    } else {
        a = x < len ? load_coeff(src, mode, idx, P) : 0u;
        b = x + 1 < len ? load_coeff(src, mode, idx + 1, P) : 0u;
    }
}

template <int LG, int R0, bool TWIST>
__device__ __forceinline__ void fwd_first_t(u32 (&v)[16], u32 *X, const FwdJob &J, i64 e, bool act, int tid)
{
    constexpr int L = 1 << LG, TPT = L >> 4, R = 1 << R0, LO = L >> R0;
    const u32 q = J.P.q, q2 = J.P.q2;
    const char *src = (const char *)J.src;
    const i64 sb = e * J.src_stride;
    // the flag bit is set only on twisted jobs, so the plain path reads the field as it is
#define FWD_MODE (TWIST ? (J.src_mode & 0xff) : J.src_mode)
    // coefficient x times w^x (w of order 2L: twf[L + x]) for the odd half of a 2L-point transform
    auto tw = [&](u32 a, int x) -> u32 {
        if constexpr (!TWIST) return a;
        const uint2 w = __ldg(J.P.twf + L + x);
        return csub(shoup_mul(a, w.x, w.y, q), q);
    };
    if constexpr (R0 == 1 && LG > 1) {
        // radix-2 stage: the thread takes groups g0 = 2 (tid + u TPT) and g0 + 1 (u < 4), so each
        // pair of points is one vector load of the input and the two twiddles one 16-byte load
        const int wsz = FWD_MODE == 8 ? 16 : 8;
        const bool vec = ((reinterpret_cast<uintptr_t>(src) + (uintptr_t)(sb * (FWD_MODE == 8 ? 8 : 4))) &
                          (uintptr_t)(wsz - 1)) == 0;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int g0 = 2 * (tid + u * TPT);
#pragma unroll
            for (int j = 0; j < 2; j++) {
                u32 a = 0u, b2 = 0u;
                if (act) load_pair(src, FWD_MODE, sb + g0 + j * LO, g0 + j * LO, J.src_len, vec, J.P, a, b2);
                v[4 * u + j] = tw(a, g0 + j * LO);
                v[4 * u + 2 + j] = tw(b2, g0 + j * LO + 1);
            }
            const uint4 w2 = __ldg((const uint4 *)(J.P.twf + LO + g0));
            bfly_dif(v[4 * u], v[4 * u + 1], make_uint2(w2.x, w2.y), q, q2);
            bfly_dif(v[4 * u + 2], v[4 * u + 3], make_uint2(w2.z, w2.w), q, q2);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                u32 *xb = X + spad(2 * (tid + u * TPT) + h);
#pragma unroll
                for (int j = 0; j < 2; j++) xb[poff<LO>(j)] = v[4 * u + 2 * h + j];
            }
        }
        return;
    }
#pragma unroll
    for (int it = 0; it < (16 >> R0); it++) {
        const int g = tid + it * TPT;
#pragma unroll
        for (int j = 0; j < R; j++) {
            const int x = g + j * LO;
            v[it * R + j] = (act && x < J.src_len) ? tw(load_coeff(src, FWD_MODE, sb + x, J.P), x) : 0u;
        }
        grp_dif<R0>(v, it * R, g & (LO - 1), LO, J.P.twf, q, q2);
    }
    if (LG == R0) {
        if (act) {
            u32 *d = J.dst + e * J.dst_stride;
#pragma unroll
            for (int j = 0; j < 16; j++) d[j] = csub(v[j], q);
        }
        return;
    }
#pragma unroll
    for (int it = 0; it < (16 >> R0); it++) {
        const int g = tid + it * TPT;
        u32 *xb = X + spad(g);
#pragma unroll
        for (int j = 0; j < R; j++) xb[poff<LO>(j)] = v[it * R + j];
    }
}

#undef FWD_MODE

// The group of 16 points that thread t takes in a radix-16 pass.  In the stride-16 pass two
// adjacent blocks of 256 points are 264 padded words apart, 8 banks, so the half-warps' 16-bank
// windows would overlap (2-way conflicts on every load and store); with REMAP the half-warps
// take blocks two apart instead (528 words, 16 banks): warp w holds blocks 4 (w / 2) + w % 2
// and that + 2.  A bijection on the groups when TPT is a multiple of 64; other passes and
// shorter transforms keep t.  Measured on GB300: inverse transforms 1 % faster at 2^13 and 2^14
// points, forward 2 % faster at 2^14 points but 2 % slower at 2^13 (its register allocation
// under the 32-register cap changes), so the forward transform remaps at 2^14 points only.
template <int LO, int TPT, bool REMAP>
__device__ __forceinline__ int pass_group(int t)
{
    if constexpr (REMAP && LO == 16 && TPT >= 64) {
        const int w = t >> 5, h = (t >> 4) & 1;
        return ((((w >> 1) << 2) + (w & 1) + (h << 1)) << 4) + (t & 15);
    } else {
        return t;
    }
}

// one radix-16 pass of the forward transform with constant stride LO
template <int LG, int LO, bool LAST>
__device__ __forceinline__ void fwd_pass16(u32 (&v)[16], u32 *X, const FwdJob &J, i64 e, bool act, int tid,
                                           const uint2 *twS)
{
    constexpr int LLO = (LO == 1) ? 0 : (LO == 2) ? 1 : (LO == 4) ? 2 : (LO == 8) ? 3 : (LO == 16) ? 4 : (LO == 32) ? 5 :
                        (LO == 64) ? 6 : (LO == 128) ? 7 : (LO == 256) ? 8 : 9;
    const u32 q = J.P.q, q2 = J.P.q2;
    const int g = pass_group<LO, (1 << LG) / 16, LG == PM_LB_LOG2>(tid), gl = g & (LO - 1);
    const int base = ((g >> LLO) << (LLO + 4)) + gl;
    __syncthreads();
    const u32 *xb = X + spad(base);
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = xb[poff<LO>(j)];
    if constexpr (LO <= 16) grp_dif<4, true>(v, 0, gl, LO, twS, q, q2);   // twiddles 1 .. 255
    else grp_dif<4>(v, 0, gl, LO, J.P.twf, q, q2);
    if (LAST) {
        if (act) {
            uint4 *d = (uint4 *)(J.dst + e * J.dst_stride + base);
#pragma unroll
            for (int j = 0; j < 4; j++)
                d[j] = make_uint4(csub(v[4 * j], q), csub(v[4 * j + 1], q), csub(v[4 * j + 2], q), csub(v[4 * j + 3], q));
        }
    } else {
        u32 *xw = X + spad(base);   // each thread writes back exactly the points it read
#pragma unroll
        for (int j = 0; j < 16; j++) xw[poff<LO>(j)] = v[j];
    }
}

// 2^14 points: one CTA of 1024 threads (two per SM); shorter transforms: 512 threads, four CTAs per SM
template <int LG>
__global__ void __launch_bounds__(LG == 14 ? 1024 : 512, LG == 14 ? 2 : 4) k_ntt_fwd_block(const __grid_constant__ JobPack<FwdJob> pk)
{
    extern __shared__ u32 sm[];
    constexpr int L = 1 << LG, TPT = L >> 4, B0 = ((LG - 1) & 3) + 1;
    const int b = blockIdx.x;
    int jb = find_job(pk.blk_start, b), lb = b - pk.blk_start[jb];
    if (const int g = pk.jobs[jb].grp) {   // interleave group: block rel -> job rel % G, block rel / G
        const int G = g >> 8, first = jb - (g & 255), rel = b - pk.blk_start[first];
        jb = first + rel % G;
        lb = rel / G;
    }
    const FwdJob &J = pk.jobs[jb];
    const int tpb = blockDim.x / TPT;
    const int lt = threadIdx.x / TPT, tid = threadIdx.x - lt * TPT;
    const i64 e = (i64)lb * tpb + lt;
    const bool act = e < J.count;
    u32 *X = sm + lt * (L + (L >> 5));
    // the twiddle table's first TW_SH entries in shared memory, for the passes of stride <= 16
    // (visible from the first pass's barrier on)
    uint2 *twS = (uint2 *)(sm + tpb * (L + (L >> 5)));
    if constexpr (LG - B0 >= 4)
        for (int i = threadIdx.x; i < (L < TW_SH ? L : TW_SH); i += blockDim.x) twS[i] = __ldg(J.P.twf + i);
    u32 v[16];
    // the twisted load is compiled only into the 2^14-point kernel, the one whose jobs can carry it
    if constexpr (LG == PM_LB_LOG2) {
        if (J.src_mode & PM_FWD_TWIST) fwd_first_t<LG, B0, true>(v, X, J, e, act, tid);
        else fwd_first_t<LG, B0, false>(v, X, J, e, act, tid);
    } else {
        fwd_first_t<LG, B0, false>(v, X, J, e, act, tid);
    }
    // radix-16 passes: stride L >> (B0 + 4), L >> (B0 + 8), ..., 1
    if constexpr (LG - B0 >= 4) fwd_pass16<LG, (L >> (B0 + 4)), (LG - B0 == 4)>(v, X, J, e, act, tid, twS);
    if constexpr (LG - B0 >= 8) fwd_pass16<LG, (L >> (B0 + 8)), (LG - B0 == 8)>(v, X, J, e, act, tid, twS);
    if constexpr (LG - B0 >= 12) fwd_pass16<LG, (L >> (B0 + 12)), (LG - B0 == 12)>(v, X, J, e, act, tid, twS);
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

template <int LG, int R0>
__device__ __forceinline__ void inv_last_t(u32 (&v)[16], const u32 *X, const InvJob &J, i64 e, bool act, int tid,
                                           bool from_regs)
{
    constexpr int L = 1 << LG, TPT = L >> 4, R = 1 << R0, LO = L >> R0;
    const u32 q = J.P.q, q2 = J.P.q2;
#pragma unroll
    for (int it = 0; it < (16 >> R0); it++) {
        const int g = tid + it * TPT;
        if (!from_regs) {
            const u32 *xb = X + spad(g);
#pragma unroll
            for (int j = 0; j < R; j++) v[it * R + j] = xb[poff<LO>(j)];
        }
        grp_dit<R0>(v, it * R, g & (LO - 1), LO, J.P.twi, q, q2);
        if (act) {
#pragma unroll
            for (int j = 0; j < R; j++) store_out(J, e, g + j * LO, v[it * R + j]);
        }
    }
}

// one radix-16 pass of the inverse transform with constant stride LO
template <int LG, int LO, bool FIRST>
__device__ __forceinline__ void inv_pass16(u32 (&v)[16], u32 *X, const InvJob &J, i64 e, bool act, int tid)
{
    constexpr int LLO = (LO == 1) ? 0 : (LO == 2) ? 1 : (LO == 4) ? 2 : (LO == 8) ? 3 : (LO == 16) ? 4 : (LO == 32) ? 5 :
                        (LO == 64) ? 6 : (LO == 128) ? 7 : (LO == 256) ? 8 : 9;
    const u32 q = J.P.q, q2 = J.P.q2;
    const int g = pass_group<LO, (1 << LG) / 16, true>(tid), gl = g & (LO - 1);
    const int base = ((g >> LLO) << (LLO + 4)) + gl;
    if (FIRST) {
        if (act) {
            const uint4 *s4 = (const uint4 *)(J.src + e * J.src_stride + base);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                uint4 t = s4[j];
                v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = 0u;
        }
    } else {
        const u32 *xb = X + spad(base);
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = xb[poff<LO>(j)];
    }
    grp_dit<4>(v, 0, gl, LO, J.P.twi, q, q2);
    u32 *xw = X + spad(base);
#pragma unroll
    for (int j = 0; j < 16; j++) xw[poff<LO>(j)] = v[j];
    __syncthreads();
}

template <int LG>
__global__ void __launch_bounds__(LG == 14 ? 1024 : 512, LG == 14 ? 2 : 4) k_ntt_inv_block(const __grid_constant__ JobPack<InvJob> pk)
{
    extern __shared__ u32 sm[];
    constexpr int L = 1 << LG, TPT = L >> 4, B0 = ((LG - 1) & 3) + 1;
    const int b = blockIdx.x;
    const int jb = find_job(pk.blk_start, b);
    const InvJob &J = pk.jobs[jb];
    const int tpb = blockDim.x / TPT;
    const int lt = threadIdx.x / TPT, tid = threadIdx.x - lt * TPT;
    const i64 e = (i64)(b - pk.blk_start[jb]) * tpb + lt;
    const bool act = e < J.count;
    u32 *X = sm + lt * (L + (L >> 5));
    u32 v[16];
    if constexpr (LG == B0) {   // L = 16: one radix-16 pass straight from the source
        const u32 *s = J.src + e * J.src_stride;
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = act ? s[j] : 0u;
        inv_last_t<LG, 4>(v, X, J, e, act, tid, true);
        return;
    } else {
        // radix-16 passes, stride 1, 16, 256 over the low LG - B0 stages
        inv_pass16<LG, 1, true>(v, X, J, e, act, tid);
        if constexpr (LG - B0 >= 8) inv_pass16<LG, 16, false>(v, X, J, e, act, tid);
        if constexpr (LG - B0 >= 12) inv_pass16<LG, 256, false>(v, X, J, e, act, tid);
        inv_last_t<LG, B0>(v, X, J, e, act, tid, false);
    }
}

int fwd_block_threads(int lg)
{
    const int tpt = (1 << lg) >> 4;
    return tpt >= 256 ? tpt : 256;
}

// tw: room for the forward kernel's shared-memory twiddles
static int block_smem(int lg, int threads, bool tw)
{
    const int L = 1 << lg, tpt = L >> 4, tpb = threads / tpt;
    return tpb * (L + (L >> 5)) * (int)sizeof(u32) + (tw ? TW_SH * (int)sizeof(uint2) : 0);
}

template <typename Pack>
static int pack_blocks(const Pack &pk) { return pk.blk_start[pk.njobs]; }

// ------------------------------------------------------------------ inverse, 2^15 points
// Inverse transform of 2^15 points in one CTA (1024 threads): the 2^14-point inverse of the
// even half (the first 2^14 transform values) goes to shared memory, then that of the odd
// half, whose last pass ends with the radix-2 step over the halves,
// (y0_x, y1_x) -> (y0_x + y1_x w^-x, y0_x - y1_x w^-x) with w of order 2^15, and writes
// points x and x + 2^14 as the job asks (store_out: scaled by 2^-15, the slice, the width).
// This replaces the column pass over the halves and its staging round trip.
template <int LG, int R0, bool ODD>
__device__ __forceinline__ void inv_last_half(u32 (&v)[16], const u32 *X, u32 *S0, const InvJob &J, i64 e, bool act,
                                              int tid)
{
    constexpr int L = 1 << LG, TPT = L >> 4, R = 1 << R0, LO = L >> R0;
    const u32 q = J.P.q, q2 = J.P.q2;
#pragma unroll
    for (int it = 0; it < (16 >> R0); it++) {
        const int g = tid + it * TPT;
        const u32 *xb = X + spad(g);
#pragma unroll
        for (int j = 0; j < R; j++) v[it * R + j] = xb[poff<LO>(j)];
        grp_dit<R0>(v, it * R, g & (LO - 1), LO, J.P.twi, q, q2);
#pragma unroll
        for (int j = 0; j < R; j++) {
            const int x = g + j * LO;
            if (!ODD) {
                S0[x] = v[it * R + j];
            } else {
                u32 a = S0[x], b = v[it * R + j];
                bfly_dit(a, b, __ldg(J.P.twi + L + x), q, q2);
                if (act) {
                    store_out(J, e, x, a);
                    store_out(J, e, x + L, b);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(1024, 1) k_ntt_inv_pair(const __grid_constant__ JobPack<InvJob> pk)
{
    extern __shared__ u32 sm[];
    constexpr int LG = PM_LB_LOG2, L = 1 << LG, B0 = ((LG - 1) & 3) + 1;
    static_assert(LG == 14, "the pass sequence below is that of 2^14 points");
    const int b = blockIdx.x;
    const int jb = find_job(pk.blk_start, b);
    const InvJob &J = pk.jobs[jb];
    const int tid = threadIdx.x;
    const i64 e = b - pk.blk_start[jb];
    const bool act = e < J.count;
    u32 *X = sm, *S0 = sm + L + (L >> 5);
    u32 v[16];
    InvJob H = J;                                       // the even half: values 0 .. 2^14 - 1
    inv_pass16<LG, 1, true>(v, X, H, e, act, tid);
    inv_pass16<LG, 16, false>(v, X, H, e, act, tid);
    inv_pass16<LG, 256, false>(v, X, H, e, act, tid);
    inv_last_half<LG, B0, false>(v, X, S0, H, e, act, tid);
    __syncthreads();
    H.src = J.src + L;                                  // the odd half
    inv_pass16<LG, 1, true>(v, X, H, e, act, tid);
    inv_pass16<LG, 16, false>(v, X, H, e, act, tid);
    inv_pass16<LG, 256, false>(v, X, H, e, act, tid);
    inv_last_half<LG, B0, true>(v, X, S0, J, e, act, tid);
}

cudaError_t launch_ntt_inv_pair(const JobPack<InvJob> &pk, cudaStream_t st, long long *launches)
{
    constexpr int L = 1 << PM_LB_LOG2;
    const int sm = (L + (L >> 5) + L) * (int)sizeof(u32);
    cudaError_t e = cudaFuncSetAttribute(k_ntt_inv_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    k_ntt_inv_pair<<<pack_blocks(pk), 1024, sm, st>>>(pk);
    ++*launches;
    return cudaGetLastError();
}


template <int LG>
static cudaError_t fwd_lg(const JobPack<FwdJob> &pk, cudaStream_t st)
{
    const int th = fwd_block_threads(LG), sm = block_smem(LG, th, true);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_ntt_fwd_block<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    k_ntt_fwd_block<LG><<<pack_blocks(pk), th, sm, st>>>(pk);
    return cudaGetLastError();
}

template <int LG>
static cudaError_t inv_lg(const JobPack<InvJob> &pk, cudaStream_t st)
{
    const int th = fwd_block_threads(LG), sm = block_smem(LG, th, false);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_ntt_inv_block<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    k_ntt_inv_block<LG><<<pack_blocks(pk), th, sm, st>>>(pk);
    return cudaGetLastError();
}

cudaError_t launch_ntt_fwd_block(const JobPack<FwdJob> &pk, int lg, cudaStream_t st, long long *launches)
{
    ++*launches;
    switch (lg) {
    case 4: return fwd_lg<4>(pk, st);
    case 5: return fwd_lg<5>(pk, st);
    case 6: return fwd_lg<6>(pk, st);
    case 7: return fwd_lg<7>(pk, st);
    case 8: return fwd_lg<8>(pk, st);
    case 9: return fwd_lg<9>(pk, st);
    case 10: return fwd_lg<10>(pk, st);
    case 11: return fwd_lg<11>(pk, st);
    case 12: return fwd_lg<12>(pk, st);
    case 13: return fwd_lg<13>(pk, st);
    case 14: return fwd_lg<14>(pk, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ntt_inv_block(const JobPack<InvJob> &pk, int lg, cudaStream_t st, long long *launches)
{
    ++*launches;
    switch (lg) {
    case 4: return inv_lg<4>(pk, st);
    case 5: return inv_lg<5>(pk, st);
    case 6: return inv_lg<6>(pk, st);
    case 7: return inv_lg<7>(pk, st);
    case 8: return inv_lg<8>(pk, st);
    case 9: return inv_lg<9>(pk, st);
    case 10: return inv_lg<10>(pk, st);
    case 11: return inv_lg<11>(pk, st);
    case 12: return inv_lg<12>(pk, st);
    case 13: return inv_lg<13>(pk, st);
    case 14: return inv_lg<14>(pk, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ column passes
// Transform length L = 2^lg > 2^14: R1 = L / 2^14 rows per column.  A block takes
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
