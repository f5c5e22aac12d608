// pointwise.cu -- pointwise matrix products in the transform domain and the
// multi-prime CRT recombination.
//
// Pointwise: at every evaluation point j, C_j = A_j B_j mod q (Sec. 2,
// "Polynomial matrix multiplication": the n^omega d term of the cost).  This
// is the CUDA-core form: a block takes 8 consecutive points and stages the
// residues it needs in shared memory; each thread owns one point and a 4 x 8
// (or 4 x 4) tile of outputs, multiplying 30-bit residues into 64-bit lazy
// accumulators (one 32 x 32 -> 64-bit multiply-add per product) folded mod q
// every 16 products.
//
// CRT: for moduli without suitable roots of unity the product is lifted to
// Z[x] and computed modulo K NTT primes (Sec. 2, "3-primes multiplication";
// here K is the least count whose product bounds the integer coefficients).
// For odd p the integer coefficient is never formed: its value mod p is the
// explicit CRT sum with an exact fixed-point quotient (crt_sum).  For even p,
// Garner's mixed-radix algorithm recovers it and a Horner pass in F_p reduces
// it mod p.
#include "common.cuh"

#define PS_PTS 8        // points per block
#define PS_ROW 9        // shared-memory words per staged entry: 8 points + 1 pad
#define PS_THREADS 256  // 8 warps = 32 slots of 8 lanes (one lane per point)
#define PS_LC 32        // inner-dimension entries staged per chunk
#define PS_PA 290       // A-row pitch (words): >= 32 * 9 and = 2 mod 8, so thread tiles
                        // 4 rows apart start 8 banks apart
#define PS_PB 289       // B-column pitch (words, B staged column-major) for 8-column thread
                        // tiles: odd, so thread tiles 8 columns apart start 8 banks apart
#define PS_PB4 290      // the same for 4-column thread tiles: = 2 mod 8, so thread tiles 4
                        // columns apart start 8 banks apart
#define PS_WORDS 28160  // shared-memory budget per block (110 KB: 2 blocks per SM)
#define PW4_MINB 4      // blocks per SM of the 4 x 4 thread-tile instance (64 registers)
#define PS_WORDS4 ((228 * 1024 / PW4_MINB - 1024) / 4)   // its budget: PW4_MINB blocks fit an SM

__device__ __forceinline__ int find_job_pw(const int *blk_start, int b)
{
    int j = 0;
    while (b >= blk_start[j + 1]) j++;
    return j;
}

static u32 magic31(int d) { return (u32)(((1ull << 31) + d - 1) / d); }

// Block plan.  The m x k output is cut into block tiles of bi x bk thread tiles
// (4 x cw outputs each, cw = 8 or 4, bi bk <= 32 slots), chosen to minimise the lanes spent
// on thread tiles plus the entries staged, within the shared-memory budget; the inner
// dimension n is staged PS_LC entries at a time and, when a block tile leaves slots
// free, each chunk is split into ns contiguous slices whose partial sums are added
// at the end.  4-column thread tiles waste at most 3 columns of a ragged k (8-column ones up
// to 7) for one more shared-memory load per 8 products (8 loads per 16 multiply-adds against
// 12 per 32).
static int pw_pitch(int cw) { return cw == 4 ? PS_PB4 : PS_PB; }

// Block tiles (bi, bk) of 4 x cw thread tiles that fit, in increasing order of the cost model
// (at most `max`; ties keep the loop order); *cost0 (if given) = the first one's cost.
// Cost of a block: 8 cw per thread tile (its 4 cw multiply-adds per inner entry, with their
// loads), rounded up to warps of 4 slots, plus 16 per staged row or column and 64 fixed.
int pw_tiles(const PwJob &j, int *bi_out, int *bk_out, int max, int cw, long long *cost0)
{
    const int nti = (j.m + 3) / 4, ntk = (j.k + cw - 1) / cw, pb = pw_pitch(cw);
    long long cost[256];
    int cbi[256], cbk[256], nc = 0;                  // bi bk <= 32: at most 130 candidates
    for (int bi = 1; bi <= nti && bi <= 32; bi++)
        for (int bk = 1; bk <= ntk && bi * bk <= 32; bk++) {
            if (bi * 4 * PS_PA + bk * cw * pb > (cw == 4 ? PS_WORDS4 : PS_WORDS)) continue;
            const long long nb = (long long)((nti + bi - 1) / bi) * ((ntk + bk - 1) / bk);
            cost[nc] = nb * (((bi * bk + 3) / 4) * 4 * 8 * cw + (bi * 4 + bk * cw) * 16 + 64);
            cbi[nc] = bi;
            cbk[nc] = bk;
            nc++;
        }
    int out = 0;
    for (; out < max && out < nc; out++) {           // selection of the cheapest remaining
        int best = -1;
        for (int c = 0; c < nc; c++)
            if (cost[c] >= 0 && (best < 0 || cost[c] < cost[best])) best = c;
        bi_out[out] = cbi[best];
        bk_out[out] = cbk[best];
        if (out == 0 && cost0) *cost0 = cost[best];
        cost[best] = -1;
    }
    return out;
}

// The default plan: the cheaper of the best 4 x 8 and the best 4 x 4 block tile, the latter's
// cost weighted by 7/8 for its occupancy (4 blocks per SM against 2; fitted to the measured
// pointwise times of six shapes of the 512-product batch and the 32 x 32 step on GB300).
int pw_plan(PwJob &j)
{
    int bi = 1, bk = 1, bi4 = 1, bk4 = 1;
    long long c8 = 0, c4 = 0;
    pw_tiles(j, &bi, &bk, 1, 8, &c8);
    pw_tiles(j, &bi4, &bk4, 1, 4, &c4);
    if (c4 * 7 < c8 * 8) return pw_plan_tile(j, bi4, bk4, 4);
    return pw_plan_tile(j, bi, bk, 8);
}

// The plan for block tile (bi, bk) of 4 x cw thread tiles (one that pw_tiles lists).  Returns
// the block count.
int pw_plan_tile(PwJob &j, int bi, int bk, int cw)
{
    const int nti = (j.m + 3) / 4, ntk = (j.k + cw - 1) / cw;
    j.bi = bi;
    j.bk = bk;
    j.cw = cw;
    const int items = j.bi * j.bk, rb = j.bi * 4, cb = j.bk * cw;
    j.lc = j.n < PS_LC ? j.n : PS_LC;
    j.ns = 1;                                                  // slices of >= 8 products per chunk
    while (items * j.ns * 2 <= 32 && j.ns * 2 * 8 <= j.lc) j.ns *= 2;
    const int stage = rb * PS_PA + cb * pw_pitch(cw), red = j.ns * rb * cb * PS_ROW;
    j.smem = (stage > red ? stage : red) * 4;
    j.nbk = (ntk + j.bk - 1) / j.bk;
    j.ntile = ((nti + j.bi - 1) / j.bi) * j.nbk;
    const int nch = (j.n + j.lc - 1) / j.lc;
    j.mg_lc = magic31(j.lc);
    j.mg_lt = magic31(j.n - (nch - 1) * j.lc);
    j.mg_cb = magic31(cb);
    j.mg_ct = magic31(j.k - (j.nbk - 1) * cb);
    return (j.L / PS_PTS) * j.ntile;
}

template <int OFF>
__device__ __forceinline__ u32 lds(u32 addr)
{
    u32 v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(OFF));
    return v;
}

// One product of residues below 2^30 into a 64-bit accumulator: one 32 x 32 -> 64-bit
// multiply-add (measured on GB300 3-4 % faster in this kernel than a carry chain of two 32-bit
// multiply-adds on the accumulator's halves).
__device__ __forceinline__ void pw_mac(u64 &acc, u32 a, u32 b) { acc += (u64)a * b; }

// One inner-dimension step l + U of a 4 x CW thread tile: A rows at fa + a PS_PA words,
// B columns at fb + c PB words, consecutive l 9 words apart.
template <int U, int CW>
__device__ __forceinline__ void pw_step(u64 (&acc)[4][CW], u32 fa, u32 fb)
{
    constexpr int PB = CW == 4 ? PS_PB4 : PS_PB;
    u32 av[4], bv[CW];
    av[0] = lds<U * 36>(fa);
    av[1] = lds<U * 36 + 4 * PS_PA>(fa);
    av[2] = lds<U * 36 + 8 * PS_PA>(fa);
    av[3] = lds<U * 36 + 12 * PS_PA>(fa);
    bv[0] = lds<U * 36>(fb);
    bv[1] = lds<U * 36 + 4 * PB>(fb);
    bv[2] = lds<U * 36 + 8 * PB>(fb);
    bv[3] = lds<U * 36 + 12 * PB>(fb);
    if constexpr (CW == 8) {
        bv[4] = lds<U * 36 + 16 * PB>(fb);
        bv[5] = lds<U * 36 + 20 * PB>(fb);
        bv[6] = lds<U * 36 + 24 * PB>(fb);
        bv[7] = lds<U * 36 + 28 * PB>(fb);
    }
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < CW; c++) pw_mac(acc[a][c], av[a], bv[c]);
}

// acc < 2^64 -> its value mod q in [0, q)
__device__ __forceinline__ u32 pw_reduce(u64 acc, u32 q, u32 q2, u32 r32, u32 r32s, u32 ones)
{
    const u32 s2 = shoup_mul((u32)(acc >> 32), r32, r32s, q) + shoup_mul((u32)acc, 1u, ones, q);
    return csub(csub(s2, q2), q);
}

// One block: 8 consecutive points of one transform and one block tile of the output.
// Thread (warp w, lane) has slot 4 w + lane / 8 -> (slice, thread tile) and point
// lane % 8.  Per chunk of <= 32 inner entries, the A rows and B columns of the block
// tile are staged (32-byte coalesced reads: the 8 points of an entry, four 16-byte
// loads in flight per thread), then every live slot accumulates its 4 x CW tile over
// its slice of the chunk.  Thread-tile rows / columns past the matrix edge read
// unused staging words and are never stored, so the inner loop carries no
// predicates.  Partial tiles go through shared memory, slices are summed, and each
// entry's 8 points are written back as two 16-byte stores.
//
// Accumulation: acc < 2^32 + 2q + 16 (q - 1)^2 < 2^64 for q < 2^30, so after every 16
// products acc is folded lazily to lo + (hi 2^32 mod q) < 2^32 + 2q, and reduced to
// [0, q) once at the end.
template <int CW>
__device__ __forceinline__ void pw_block(const PwJob &J, int rel, u32 *sms)
{
    constexpr int PB = CW == 4 ? PS_PB4 : PS_PB;
    const int n = J.n, k = J.k, L = J.L, ns = J.ns, lc = J.lc, bk = J.bk;
    const u32 q = J.P.q, q2 = J.P.q2, r32 = J.P.r32, r32s = J.P.r32s, ones = J.P.ones;
    const int tile = rel % J.ntile, j0 = (rel / J.ntile) * PS_PTS;
    const int rb = J.bi * 4, cb = bk * CW;
    const int r0 = (tile / J.nbk) * rb, c0 = (tile % J.nbk) * cb;
    const int rows = min(J.m - r0, rb), cols = min(k - c0, cb);
    const int tid = threadIdx.x, lane = tid & 31, pp = lane & 7;
    const int slot = (tid >> 5) * 4 + (lane >> 3), items = J.bi * bk;
    const int item = slot % items, slice = slot / items;
    const bool live = slice < ns;
    const int ti = item / bk, tk = item % bk;
    u32 *rA = sms, *rB = sms + rb * PS_PA;
    const u32 sA = (u32)__cvta_generic_to_shared(rA) + (ti * 4 * PS_PA + pp) * 4;
    const u32 sB = (u32)__cvta_generic_to_shared(rB) + (tk * CW * PB + pp) * 4;

    u64 acc[4][CW];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < CW; c++) acc[a][c] = 0;
    bool lazy = false;                                         // accumulators not yet in [0, q)

    for (int l0 = 0; l0 < n; l0 += lc) {
        const int lcv = min(lc, n - l0);
        if (l0) __syncthreads();                               // the previous chunk is consumed
        // stage: entry e < nA is A (row, l) = divmod(e, lcv), else B (l, col) = divmod(e - nA, cols)
        {
            const int nA = rows * lcv, tot = (nA + lcv * cols) * 2;
            const u32 mA = lcv == lc ? J.mg_lc : J.mg_lt, mB = cols == cb ? J.mg_cb : J.mg_ct;
            for (int x0 = tid; x0 < tot; x0 += 4 * PS_THREADS) {
                uint4 v[4];
                u32 *d[4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int x = min(x0 + i * PS_THREADS, tot - 1);
                    const int e = x >> 1, h = x & 1;
                    const bool isA = e < nA;
                    const int f = isA ? e : e - nA, dv = isA ? lcv : cols;
                    const int qt = (int)__umulhi((u32)f << 1, isA ? mA : mB), rm = f - qt * dv;
                    const u32 *src = isA ? J.A + (i64)((r0 + qt) * n + l0 + rm) * L
                                         : J.B + (i64)((l0 + qt) * k + c0 + rm) * L;
                    d[i] = (isA ? rA + qt * PS_PA + rm * PS_ROW : rB + rm * PB + qt * PS_ROW) + 4 * h;
                    v[i] = __ldg((const uint4 *)(src + j0 + 4 * h));
                }
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if (x0 + i * PS_THREADS < tot) { d[i][0] = v[i].x; d[i][1] = v[i].y; d[i][2] = v[i].z; d[i][3] = v[i].w; }
            }
        }
        __syncthreads();
        if (live) {
            // this slice's contiguous share of the chunk, in groups of 16 products
            const int per = (lcv + ns - 1) / ns, lb = slice * per, le = min(lcv, lb + per);
            u32 fa = sA + lb * PS_ROW * 4, fb = sB + lb * PS_ROW * 4;
            for (int g = lb; g < le; g += 16) {
                int cnt = min(le, g + 16) - g;
                for (; cnt >= 8; cnt -= 8) {
                    pw_step<0, CW>(acc, fa, fb); pw_step<1, CW>(acc, fa, fb);
                    pw_step<2, CW>(acc, fa, fb); pw_step<3, CW>(acc, fa, fb);
                    pw_step<4, CW>(acc, fa, fb); pw_step<5, CW>(acc, fa, fb);
                    pw_step<6, CW>(acc, fa, fb); pw_step<7, CW>(acc, fa, fb);
                    fa += 8 * PS_ROW * 4; fb += 8 * PS_ROW * 4;
                }
                for (; cnt > 0; cnt--) {
                    pw_step<0, CW>(acc, fa, fb);
                    fa += PS_ROW * 4; fb += PS_ROW * 4;
                }
                if (g + 16 < le || l0 + lc < n) {
                    // more products follow: acc <- lo + (hi 2^32 mod q)
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int c = 0; c < CW; c++)
                            acc[a][c] = (u64)(u32)acc[a][c] + shoup_mul((u32)(acc[a][c] >> 32), r32, r32s, q);
                    lazy = true;
                } else {
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int c = 0; c < CW; c++) acc[a][c] = pw_reduce(acc[a][c], q, q2, r32, r32s, ones);
                    lazy = false;
                }
            }
        }
    }
    if (lazy) {                                                // a slice empty in the last chunk
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < CW; c++) acc[a][c] = pw_reduce(acc[a][c], q, q2, r32, r32s, ones);
    }
    __syncthreads();
    // partial tiles: red[slice][row][col][point]
    u32 *red = sms;
    if (live) {
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < CW; c++) {
                const int r = ti * 4 + a, cc = tk * CW + c;
                if (r < rows && cc < cols) red[((slice * rb + r) * cb + cc) * PS_ROW + pp] = (u32)acc[a][c];
            }
    }
    __syncthreads();
    const u32 mC = cols == cb ? J.mg_cb : J.mg_ct;
    for (int x = tid; x < rows * cols * 2; x += PS_THREADS) {
        const int e = x >> 1, h = x & 1;
        const int r = (int)__umulhi((u32)e << 1, mC), c = e - r * cols;
        uint4 o;
        if (ns == 1) {
            const u32 *s4 = red + (r * cb + c) * PS_ROW + 4 * h;
            o = make_uint4(s4[0], s4[1], s4[2], s4[3]);
        } else {
            u32 w[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                u64 s = 0;                                     // ns <= 32 terms < q: s < 2^35
                for (int sl = 0; sl < ns; sl++) s += red[((sl * rb + r) * cb + c) * PS_ROW + 4 * h + t];
                w[t] = pw_reduce(s, q, q2, r32, r32s, ones);
            }
            o = make_uint4(w[0], w[1], w[2], w[3]);
        }
        *(uint4 *)(J.C + (i64)((r0 + r) * k + c0 + c) * L + j0 + 4 * h) = o;
    }
}

// A block's job by a scan of the pack's block counts, then its tile.  One instance per thread-tile
// width (a single kernel holding both spills the 4 x 8 tile's accumulators).
template <int CW>
__global__ void __launch_bounds__(PS_THREADS, CW == 4 ? PW4_MINB : 2) k_pointwise(const __grid_constant__ JobPack<PwJob> pk)
{
    extern __shared__ __align__(16) u32 sms[];
    const int b = blockIdx.x;
    const int jb = find_job_pw(pk.blk_start, b);
    pw_block<CW>(pk.jobs[jb], b - pk.blk_start[jb], sms);
}

cudaError_t launch_pointwise(const JobPack<PwJob> &pk, cudaStream_t st, long long *launches)
{
    int mx = 0;
    for (int i = 0; i < pk.njobs; i++) {
        if (pk.jobs[i].cw != pk.jobs[0].cw) return cudaErrorInvalidValue;
        mx = pk.jobs[i].smem > mx ? pk.jobs[i].smem : mx;
    }
    const bool four = pk.jobs[0].cw == 4;
    if (mx > 48 * 1024) {
        const cudaError_t e = four ? cudaFuncSetAttribute(k_pointwise<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)
                                   : cudaFuncSetAttribute(k_pointwise<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e != cudaSuccess) return e;
    }
    if (four) {                       // the whole carveout for shared memory, so PW4_MINB blocks fit
        const cudaError_t e = cudaFuncSetAttribute(k_pointwise<4>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    if (four) k_pointwise<4><<<pk.blk_start[pk.njobs], PS_THREADS, mx, st>>>(pk);
    else k_pointwise<8><<<pk.blk_start[pk.njobs], PS_THREADS, mx, st>>>(pk);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ small inner dimension
// C = A B at every point for n <= PWS_NMAX: the work is n multiply-adds per output, so
// the kernel is bound by the m k output writes.  One thread per point keeps an n x 8
// block of B's residues in registers and streams PWS_ROWS rows of A (n residues each);
// an output is one 64-bit sum of n <= 8 products below 2^60, reduced once.  Every
// access is coalesced across the points of a warp.  Blocks: points x row groups x
// column chunks of 8 (n <= 4) or 4 (n > 4, to stay near 100 registers).
#define PWS_THREADS 256
#define PWS_ROWS 16
#define PWS_NMAX 8

static int pws_kc(int n) { return n <= 4 ? 8 : 4; }

int pws_blocks(const PwJob &j)
{
    const int kc = pws_kc(j.n);
    return ((j.L + PWS_THREADS - 1) / PWS_THREADS) * ((j.m + PWS_ROWS - 1) / PWS_ROWS) * ((j.k + kc - 1) / kc);
}
bool pws_supported(const PwJob &j) { return j.n <= PWS_NMAX; }

template <int N, int PWS_KC>
__global__ void __launch_bounds__(PWS_THREADS) k_pointwise_sn(const __grid_constant__ JobPack<PwJob> pk)
{
    const int b = blockIdx.x;
    const int jb = find_job_pw(pk.blk_start, b);
    const PwJob &J = pk.jobs[jb];
    const int L = J.L, k = J.k;
    const int npb = (L + PWS_THREADS - 1) / PWS_THREADS, nrg = (J.m + PWS_ROWS - 1) / PWS_ROWS;
    int rel = b - pk.blk_start[jb];
    const int pt = (rel % npb) * PWS_THREADS + threadIdx.x;
    rel /= npb;
    const int i0 = (rel % nrg) * PWS_ROWS, c0 = (rel / nrg) * PWS_KC;
    if (pt >= L) return;
    const int kcv = min(PWS_KC, k - c0);
    u32 bv[N][PWS_KC];
#pragma unroll
    for (int l = 0; l < N; l++)
#pragma unroll
        for (int c = 0; c < PWS_KC; c++) bv[l][c] = c < kcv ? __ldg(J.B + ((i64)l * k + c0 + c) * L + pt) : 0u;
    const int i1 = min(J.m, i0 + PWS_ROWS);
    for (int i = i0; i < i1; i++) {
        u32 av[N];
#pragma unroll
        for (int l = 0; l < N; l++) av[l] = __ldg(J.A + ((i64)i * N + l) * L + pt);
#pragma unroll
        for (int c = 0; c < PWS_KC; c++) {
            if (c < kcv) {
                u64 acc = 0;
#pragma unroll
                for (int l = 0; l < N; l++) acc += (u64)av[l] * bv[l][c];
                __stcs(J.C + ((i64)i * k + c0 + c) * L + pt, reduce64(acc, J.P));
            }
        }
    }
}

// one launch per inner dimension n (every job of the pack has the same n)
cudaError_t launch_pointwise_sn(const JobPack<PwJob> &pk, cudaStream_t st, long long *launches)
{
    const int nb = pk.blk_start[pk.njobs];
    switch (pk.jobs[0].n) {
    case 1: k_pointwise_sn<1, 8><<<nb, PWS_THREADS, 0, st>>>(pk); break;
    case 2: k_pointwise_sn<2, 8><<<nb, PWS_THREADS, 0, st>>>(pk); break;
    case 3: k_pointwise_sn<3, 8><<<nb, PWS_THREADS, 0, st>>>(pk); break;
    case 4: k_pointwise_sn<4, 8><<<nb, PWS_THREADS, 0, st>>>(pk); break;
    case 5: k_pointwise_sn<5, 4><<<nb, PWS_THREADS, 0, st>>>(pk); break;
    case 6: k_pointwise_sn<6, 4><<<nb, PWS_THREADS, 0, st>>>(pk); break;
    case 7: k_pointwise_sn<7, 4><<<nb, PWS_THREADS, 0, st>>>(pk); break;
    case 8: k_pointwise_sn<8, 4><<<nb, PWS_THREADS, 0, st>>>(pk); break;
    default: return cudaErrorInvalidValue;
    }
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ matrix-vector (k = 1)
// c_i = sum_l A[i][l] b_l at every point, 8 < n <= PWV_NMAX: one thread per point keeps
// b (n residues, zero-padded to NB) in registers and streams PWV_ROWS rows of A; each
// output is a 64-bit (hi, lo) carry-chain sum, folded lazily to lo + (hi 2^32 mod q)
// every 16 products (below 2^32 + 2q + 16 (q-1)^2 < 2^64) and reduced once.  Bound by
// reading A once.
#define PWV_THREADS 256
#define PWV_ROWS 16
#define PWV_NMAX 64

int pwv_blocks(const PwJob &j) { return ((j.L + PWV_THREADS - 1) / PWV_THREADS) * ((j.m + PWV_ROWS - 1) / PWV_ROWS); }
bool pwv_supported(const PwJob &j) { return j.k == 1 && j.n > PWS_NMAX && j.n <= PWV_NMAX; }

template <int NB>
__global__ void __launch_bounds__(PWV_THREADS) k_pointwise_mv(const __grid_constant__ JobPack<PwJob> pk)
{
    const int b = blockIdx.x;
    const int jb = find_job_pw(pk.blk_start, b);
    const PwJob &J = pk.jobs[jb];
    const int L = J.L, n = J.n;
    const u32 q = J.P.q, r32 = J.P.r32, r32s = J.P.r32s;
    const int npb = (L + PWV_THREADS - 1) / PWV_THREADS;
    const int rel = b - pk.blk_start[jb];
    const int pt = (rel % npb) * PWV_THREADS + threadIdx.x, i0 = (rel / npb) * PWV_ROWS;
    if (pt >= L) return;
    u32 bv[NB];
#pragma unroll
    for (int l = 0; l < NB; l++) bv[l] = l < n ? __ldg(J.B + (i64)l * L + pt) : 0u;
    const int i1 = min(J.m, i0 + PWV_ROWS);
    for (int i = i0; i < i1; i++) {
        const u32 *arow = J.A + (i64)i * n * L + pt;
        u32 lo = 0, hi = 0;
#pragma unroll
        for (int l0 = 0; l0 < NB; l0 += 16) {
#pragma unroll
            for (int l = l0; l < l0 + 16; l++) {
                const u32 a = l < n ? __ldcs(arow + (i64)l * L) : 0u;
                asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;" : "+r"(lo), "+r"(hi) : "r"(a), "r"(bv[l]));
            }
            if (l0 + 16 < NB) {
                const u32 t = shoup_mul(hi, r32, r32s, q);
                asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, 0, 0;" : "+r"(lo), "=r"(hi) : "r"(t));
            }
        }
        J.C[(i64)i * L + pt] = reduce64(((u64)hi << 32) | lo, J.P);
    }
}

cudaError_t launch_pointwise_mv(const JobPack<PwJob> &pk, cudaStream_t st, long long *launches)
{
    int nmax = 0;
    for (int i = 0; i < pk.njobs; i++) nmax = pk.jobs[i].n > nmax ? pk.jobs[i].n : nmax;
    const int nb = pk.blk_start[pk.njobs];
    if (nmax <= 16) k_pointwise_mv<16><<<nb, PWV_THREADS, 0, st>>>(pk);
    else if (nmax <= 32) k_pointwise_mv<32><<<nb, PWV_THREADS, 0, st>>>(pk);
    else k_pointwise_mv<64><<<nb, PWV_THREADS, 0, st>>>(pk);
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

// Value y of flat output index idx (entry idx / len, position idx mod len) to dst.
__device__ __forceinline__ void crt_store(const CrtJob &J, i64 idx, u64 y)
{
    i64 o = idx;
    if (J.dst_stride != J.len) {
        const i64 e = idx / J.len;
        o = e * J.dst_stride + (idx - e * J.len);
    }
    if (J.w == 8) ((u64 *)J.dst)[o] = y;
    else ((u32 *)J.dst)[o] = (u32)y;
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
    crt_store(J, idx, y);
}

// The explicit CRT sum (mode 1).  With t_i = r_i M_i^-1 mod q_i, sum_i t_i / q_i = k + X / M
// for the integer X < M that the residues stand for, and X mod p = sum_i t_i (M_i mod p) -
// k (M mod p).  k: s = sum_i t_i floor(2^59 / q_i) lies in (2^59 sum_i t_i / q_i - 2^33,
// 2^59 sum_i t_i / q_i] (sum_i t_i < 6 2^30), so (s + 2^33) >> 59 = k whenever X / M <
// 1 - 2^-26, which the prime count guarantees (M > 2^0.01 times the bound on X).  The sum
// mod p: terms t (M_i mod p) 2^64 mod p accumulated in 128 bits (below (K + 1) 2^30 p, so
// below p 2^64) and one Montgomery reduction.
// (w2, w1, w0) += a b for a < 2^32, b = b0 + b1 2^32 < 2^64: a b0 into words 0 and 1, a b1 into
// words 1 and 2, one carry chain of 32-bit multiply-adds (the sum stays below 2^96)
__device__ __forceinline__ void mac96(u32 &w0, u32 &w1, u32 &w2, u32 a, u64 b)
{
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;\n\t"
        "mad.lo.cc.u32 %1, %3, %5, %1;\n\t"
        "madc.hi.u32 %2, %3, %5, %2;"
        : "+r"(w0), "+r"(w1), "+r"(w2) : "r"(a), "r"((u32)b), "r"((u32)(b >> 32)));
}

template <int K>
__device__ __forceinline__ void crt_sum(const CrtJob &J, i64 idx)
{
    u64 s = 0;
    u32 w0 = 0, w1 = 0, w2 = 0;                      // the 128-bit sum below (K + 1) 2^30 p < 2^95
#pragma unroll
    for (int i = 0; i < K; i++) {
        const u32 qi = J.q[i];
        const u32 r = __ldg(J.res + (i64)i * J.count + idx);
        const u32 t = csub(shoup_mul(r, J.gi[i], J.gis[i], qi), qi);
        s += (u64)t * J.W[i];
        mac96(w0, w1, w2, t, J.Cm[i]);
    }
    const u32 k = (u32)((s + (1ull << 33)) >> 59);
    mac96(w0, w1, w2, k, J.Cm[K]);
    crt_store(J, idx, redc128(w2, ((u64)w1 << 32) | w0, J.p, J.pn));
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
        if (J.mode == 1) {
            switch (J.K) {
            case 2: crt_sum<2>(J, idx); break;
            case 3: crt_sum<3>(J, idx); break;
            case 4: crt_sum<4>(J, idx); break;
            case 5: crt_sum<5>(J, idx); break;
            default: crt_sum<6>(J, idx); break;
            }
            continue;
        }
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
