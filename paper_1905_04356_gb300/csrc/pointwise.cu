// pointwise.cu -- pointwise matrix products in the transform domain and the
// multi-prime CRT recombination.
//
// Pointwise: at every evaluation point j, C_j = A_j B_j mod q (Sec. 2,
// "Polynomial matrix multiplication": the n^omega d term of the cost).  This
// is the CUDA-core form: each thread owns one point and a 4 x 8 tile of
// outputs; 30-bit residues multiply into 64-bit lazy accumulators (16 terms
// below 2^64, one mad.wide.u32 each), folded mod q every 16 terms.  Loads are coalesced across the
// points of a warp (the transform domain is entry-major, point-minor).
//
// CRT: for moduli without suitable roots of unity the product is lifted to
// Z[x] and computed modulo K NTT primes (Sec. 2, "3-primes multiplication";
// here K is the least count whose product bounds the integer coefficients).
// Garner's mixed-radix algorithm recovers the integer coefficient, and a
// Horner pass in F_p reduces it mod p.
#include "common.cuh"

#define PW_TI 4      // output rows per thread
#define PW_TK 8      // output columns per thread
#define PW_PTS 128   // points (threads) per block

__device__ __forceinline__ int find_job_pw(const int *blk_start, int b)
{
    int j = 0;
    while (b >= blk_start[j + 1]) j++;
    return j;
}

int pw_blocks(const PwJob &j)
{
    const int npb = (j.L + PW_PTS - 1) / PW_PTS;
    return npb * ((j.m + PW_TI - 1) / PW_TI) * ((j.k + PW_TK - 1) / PW_TK);
}

__device__ __forceinline__ void mad_wide(u64 &acc, u32 a, u32 b)
{
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// One thread: one point, a PW_TI x PW_TK tile of outputs.  Rows / columns past
// the matrix edge read a valid row (the last one) and are not stored, so the
// inner loop carries no predicates.
__global__ void __launch_bounds__(PW_PTS) k_pointwise(const __grid_constant__ JobPack<PwJob> pk)
{
    const int b = blockIdx.x;
    const int jb = find_job_pw(pk.blk_start, b);
    const PwJob &J = pk.jobs[jb];
    const int m = J.m, n = J.n, k = J.k, Li = J.L;
    const u32 q = J.P.q, q2 = J.P.q2, r32 = J.P.r32, r32s = J.P.r32s, ones = J.P.ones;
    int rel = b - pk.blk_start[jb];
    const int npb = (Li + PW_PTS - 1) / PW_PTS, ntk = (k + PW_TK - 1) / PW_TK;
    const int pb = rel % npb;
    rel /= npb;
    const int tk = rel % ntk, ti = rel / ntk;
    const int pt = pb * PW_PTS + threadIdx.x;
    if (pt >= Li) return;
    const int i0 = ti * PW_TI, k0 = tk * PW_TK;
    const i64 L = Li;

    const u32 *pa[PW_TI], *pbp[PW_TK];
#pragma unroll
    for (int a = 0; a < PW_TI; a++) pa[a] = J.A + (i64)min(i0 + a, m - 1) * n * L + pt;
#pragma unroll
    for (int c = 0; c < PW_TK; c++) pbp[c] = J.B + (i64)min(k0 + c, k - 1) * L + pt;
    const i64 sb = (i64)k * L;   // B stride between consecutive l

    u32 part[PW_TI][PW_TK];
#pragma unroll
    for (int a = 0; a < PW_TI; a++)
#pragma unroll
        for (int c = 0; c < PW_TK; c++) part[a][c] = 0;

    for (int l0 = 0; l0 < n; l0 += 16) {
        const int lend = min(n, l0 + 16);
        u64 acc[PW_TI][PW_TK];
#pragma unroll
        for (int a = 0; a < PW_TI; a++)
#pragma unroll
            for (int c = 0; c < PW_TK; c++) acc[a][c] = 0;
        for (int l = l0; l < lend; l++) {
            u32 av[PW_TI], bv[PW_TK];
#pragma unroll
            for (int a = 0; a < PW_TI; a++) av[a] = __ldg(pa[a] + (i64)l * L);
#pragma unroll
            for (int c = 0; c < PW_TK; c++) bv[c] = __ldg(pbp[c] + (i64)l * sb);
#pragma unroll
            for (int a = 0; a < PW_TI; a++)
#pragma unroll
                for (int c = 0; c < PW_TK; c++) mad_wide(acc[a][c], av[a], bv[c]);
        }
        // fold: acc < 16 q^2 < 2^64; acc = hi 2^32 + lo -> [0, q)
#pragma unroll
        for (int a = 0; a < PW_TI; a++)
#pragma unroll
            for (int c = 0; c < PW_TK; c++) {
                const u32 hi = (u32)(acc[a][c] >> 32), lo = (u32)acc[a][c];
                u32 s2 = shoup_mul(hi, r32, r32s, q) + shoup_mul(lo, 1u, ones, q);    // < 4q
                s2 = csub(csub(s2, q2), q);
                part[a][c] = csub(part[a][c] + s2, q);
            }
    }
#pragma unroll
    for (int a = 0; a < PW_TI; a++)
#pragma unroll
        for (int c = 0; c < PW_TK; c++)
            if (i0 + a < m && k0 + c < k) J.C[((i64)(i0 + a) * k + k0 + c) * L + pt] = part[a][c];
}

cudaError_t launch_pointwise(const JobPack<PwJob> &pk, cudaStream_t st, long long *launches)
{
    k_pointwise<<<pk.blk_start[pk.njobs], PW_PTS, 0, st>>>(pk);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ staged CUDA-core form
// A block takes 8 consecutive points of one prime.  The residues of every entry at
// those points are staged in shared memory (32-byte coalesced reads; rows padded to
// 9 words), then each thread computes a 4 x 8 output tile at one point: warp w owns
// output rows 4w.., lane = 8 * (column tile) + point.  Within a warp the A reads are
// broadcasts and the B reads fall in distinct banks.  Outputs are staged and
// written back 32 bytes per entry.  Needs m n, n k, m k <= 1024 (else k_pointwise).
#define PS_PTS 8
#define PS_ROW 9
#define PS_THREADS 256

int pws_blocks(const PwJob &j) { return (j.L + PS_PTS - 1) / PS_PTS; }
bool pws_supported(const PwJob &j) { return j.m * j.n <= 1024 && j.n * j.k <= 1024 && j.m * j.k <= 1024 && j.L >= 16; }

__global__ void __launch_bounds__(PS_THREADS, 2) k_pointwise_s(const __grid_constant__ JobPack<PwJob> pk)
{
    extern __shared__ __align__(16) u32 sms[];
    const int b = blockIdx.x;
    const int jb = find_job_pw(pk.blk_start, b);
    const PwJob &J = pk.jobs[jb];
    const int m = J.m, n = J.n, k = J.k, L = J.L;
    const u32 q = J.P.q, q2 = J.P.q2, r32 = J.P.r32, r32s = J.P.r32s, ones = J.P.ones;
    const int j0 = (b - pk.blk_start[jb]) * PS_PTS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int eA = m * n, eB = n * k, eC = m * k;
    u32 *rA = sms, *rB = sms + eA * PS_ROW, *rC = rB + eB * PS_ROW;

    for (int x = tid; x < (eA + eB) * 2; x += PS_THREADS) {
        const int e = x >> 1, h = x & 1;
        const u32 *src = e < eA ? J.A + (i64)e * L : J.B + (i64)(e - eA) * L;
        const uint4 v = *(const uint4 *)(src + j0 + 4 * h);
        u32 *dst = (e < eA ? rA + e * PS_ROW : rB + (e - eA) * PS_ROW) + 4 * h;
        dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w;
    }
    __syncthreads();

    const int pp = lane & 7, tkl = lane >> 3;                 // point, column tile within the warp
    const int nti = (m + PW_TI - 1) / PW_TI, ntk = (k + PW_TK - 1) / PW_TK;
    // work items: (row tile ti, column-tile group tg); a warp takes 4 column tiles of one row tile
    const int ngroups = (ntk + 3) / 4;
    for (int item = warp; item < nti * ngroups; item += PS_THREADS / 32) {
        const int ti = item / ngroups, tk = (item % ngroups) * 4 + tkl;
        const int i0 = ti * PW_TI, k0 = tk * PW_TK;
        const bool live = tk < ntk;
        int oa[PW_TI], ob[PW_TK];                              // 32-bit shared-memory offsets
#pragma unroll
        for (int a = 0; a < PW_TI; a++) oa[a] = min(i0 + a, m - 1) * n * PS_ROW + pp;
#pragma unroll
        for (int c = 0; c < PW_TK; c++) ob[c] = min(k0 + c, k - 1) * PS_ROW + pp;
        const int sbk = k * PS_ROW;
        // 64-bit accumulators as (hi, lo) words with a carry chain per product;
        // acc < q + 15 (q - 1)^2 < 2^64: fold to [0, q) every 15 products
        u32 alo[PW_TI][PW_TK], ahi[PW_TI][PW_TK];
#pragma unroll
        for (int a = 0; a < PW_TI; a++)
#pragma unroll
            for (int c = 0; c < PW_TK; c++) { alo[a][c] = 0; ahi[a][c] = 0; }
        for (int l0 = 0; l0 < n; l0 += 15) {
            const int lend = min(n, l0 + 15);
#pragma unroll 3
            for (int l = l0; l < lend; l++) {
                u32 av[PW_TI], bv[PW_TK];
#pragma unroll
                for (int a = 0; a < PW_TI; a++) av[a] = rA[oa[a] + l * PS_ROW];
#pragma unroll
                for (int c = 0; c < PW_TK; c++) bv[c] = rB[ob[c] + l * sbk];
#pragma unroll
                for (int a = 0; a < PW_TI; a++)
#pragma unroll
                    for (int c = 0; c < PW_TK; c++)
                        asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;"
                            : "+r"(alo[a][c]), "+r"(ahi[a][c]) : "r"(av[a]), "r"(bv[c]));
            }
#pragma unroll
            for (int a = 0; a < PW_TI; a++)
#pragma unroll
                for (int c = 0; c < PW_TK; c++) {
                    u32 s2 = shoup_mul(ahi[a][c], r32, r32s, q) + shoup_mul(alo[a][c], 1u, ones, q);
                    alo[a][c] = csub(csub(s2, q2), q);
                    ahi[a][c] = 0;
                }
        }
        if (live) {
#pragma unroll
            for (int a = 0; a < PW_TI; a++)
#pragma unroll
                for (int c = 0; c < PW_TK; c++)
                    if (i0 + a < m && k0 + c < k) rC[((i0 + a) * k + k0 + c) * PS_ROW + pp] = alo[a][c];
        }
    }
    __syncthreads();
    for (int x = tid; x < eC * 2; x += PS_THREADS) {
        const int e = x >> 1, h = x & 1;
        const u32 *s4 = rC + e * PS_ROW + 4 * h;
        *(uint4 *)(J.C + (i64)e * L + j0 + 4 * h) = make_uint4(s4[0], s4[1], s4[2], s4[3]);
    }
}

cudaError_t launch_pointwise_s(const JobPack<PwJob> &pk, cudaStream_t st, long long *launches)
{
    int mx = 0;
    for (int i = 0; i < pk.njobs; i++) {
        const PwJob &j = pk.jobs[i];
        const int t = (j.m * j.n + j.n * j.k + j.m * j.k) * PS_ROW * 4;
        mx = t > mx ? t : mx;
    }
    if (mx > 48 * 1024) cudaFuncSetAttribute(k_pointwise_s, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    k_pointwise_s<<<pk.blk_start[pk.njobs], PS_THREADS, mx, st>>>(pk);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ CRT
#define CRT_THREADS 256
#define CRT_PER_THREAD 4

int crt_blocks(const CrtJob &j)
{
    const i64 per = (i64)CRT_THREADS * CRT_PER_THREAD;
    return (int)((j.count + per - 1) / per);
}

template <int K>
__device__ __forceinline__ void crt_one(const CrtJob &J, i64 idx)
{
    u32 v[K];
    // Garner: v_i = (...((r_i - v_0) c_i0 - v_1) c_i1 ... - v_{i-1}) c_i,i-1 mod q_i
#pragma unroll
    for (int i = 0; i < K; i++) {
        const u32 qi = J.q[i];
        u32 t = __ldg(J.res + (i64)i * J.count + idx);
#pragma unroll
        for (int j = 0; j < i; j++) {
            const u32 vj = csub(v[j], qi);              // v_j < q_j < 2 q_i
            t = csub(shoup_mul(t + qi - vj, J.c[i][j], J.cs[i][j], qi), qi);
        }
        v[i] = t;
    }
    // X = v_0 + q_0 (v_1 + q_1 (v_2 + ...)) reduced mod p by Horner
    u64 y = J.small_p ? barrett64(v[K - 1], J.p, J.mu) : v[K - 1];
#pragma unroll
    for (int i = K - 2; i >= 0; i--) {
        u64 z = shoup_mul64(y, J.qm[i], J.qms[i], J.p);              // [0, 2p)
        z += J.small_p ? barrett64(v[i], J.p, J.mu) : v[i];         // [0, 3p)
        y = csub64(csub64(z, J.p), J.p);
    }
    const i64 e = idx / J.len, o = e * J.dst_stride + (idx - e * J.len);
    if (J.w == 8) ((u64 *)J.dst)[o] = y;
    else ((u32 *)J.dst)[o] = (u32)y;
}

__global__ void __launch_bounds__(CRT_THREADS) k_crt(const __grid_constant__ JobPack<CrtJob> pk)
{
    const int b = blockIdx.x;
    const int jb = find_job_pw(pk.blk_start, b);
    const CrtJob &J = pk.jobs[jb];
    const i64 start = (i64)(b - pk.blk_start[jb]) * CRT_THREADS * CRT_PER_THREAD + threadIdx.x;
#pragma unroll
    for (int it = 0; it < CRT_PER_THREAD; it++) {
        const i64 idx = start + (i64)it * CRT_THREADS;
        if (idx >= J.count) return;
        switch (J.K) {
        case 1: crt_one<1>(J, idx); break;
        case 2: crt_one<2>(J, idx); break;
        case 3: crt_one<3>(J, idx); break;
        case 4: crt_one<4>(J, idx); break;
        case 5: crt_one<5>(J, idx); break;
        default: crt_one<6>(J, idx); break;
        }
    }
}

cudaError_t launch_crt(const JobPack<CrtJob> &pk, cudaStream_t st, long long *launches)
{
    k_crt<<<pk.blk_start[pk.njobs], CRT_THREADS, 0, st>>>(pk);
    ++*launches;
    return cudaGetLastError();
}
