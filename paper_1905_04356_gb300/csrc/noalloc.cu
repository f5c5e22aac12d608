// noalloc.cu -- pmat_mul_noalloc: the full product A . B mod p without any
// device allocation, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden --
// inside a CUDA stream capture that must not contain allocation nodes, under a
// host framework whose memory pool owns the whole device, or in a process
// that has a fixed device-memory budget and must never grow it after set-up.
// pmat_mul allocates (a growing workspace, twiddle tables, a context); this
// entry point takes no context and uses one fixed array instead.
//
// All scratch (twiddle tables, transform-domain buffers, CRT residues) lives
// in g_pm_scratch, a file-scope __device__ array of PM_NOALLOC_SCRATCH_BYTES
// (64 MiB).  Every GPU that loads this library holds that array until the
// process exits.  Host code cannot use the symbol as a device address, so the
// first call on each device (with that device current) looks the address up
// with cudaGetSymbolAddress and caches it; that first call must therefore
// happen before any stream capture.  Every call shares the array and
// overwrites it; nothing in it needs to start at zero (each stage writes every
// value the next stage reads).  Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on the array: serialise them.
//
// The work is the same four kernels as pmat_mul (forward transforms with the
// reduction fused, pointwise products, inverse transforms with the slice
// fused, CRT recombination: the explicit CRT sum for odd p, Garner's mixed
// radix for even p or a single prime; see pointwise.cu), launched on the
// caller's stream.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "pmat.h"

#define PM_NOALLOC_SCRATCH_BYTES (64ull << 20)
#define PM_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_pm_scratch[PM_NOALLOC_SCRATCH_BYTES];

namespace {

struct StaticPrime {
    u32 q;
    u32 rf[PM_MAX_LOG2L + 1], ri[PM_MAX_LOG2L + 1];
};

void make_prime(StaticPrime &s, u32 q)
{
    s.q = q;
    ntt_roots(q, s.rf, s.ri);
}

std::once_flag g_table_once;
std::vector<StaticPrime> g_table;        // CRT primes q = c 2^20 + 1 < 2^30, largest first
std::mutex g_dev_mu;
void *g_dev_scratch[PM_NOALLOC_MAX_DEVICES];

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

PrimeDev dev_prime(const StaticPrime &s, int lg, const uint2 *twf, const uint2 *twi)
{
    PrimeDev P;
    const uint64_t q = s.q;
    P.q = s.q;
    P.q2 = 2 * s.q;
    P.r32 = (u32)((1ull << 32) % q);
    P.r32s = (u32)(((uint64_t)P.r32 << 32) / q);
    P.ones = (u32)((1ull << 32) / q);
    P.linv = (u32)host_powmod((1ull << lg) % q, q - 2, q);
    P.linvs = (u32)(((uint64_t)P.linv << 32) / q);
    P.twf = twf;
    P.twi = twi;
    return P;
}

template <typename J>
void add(JobPack<J> &pk, const J &j, int blocks)
{
    pk.jobs[pk.njobs] = j;
    pk.blk_start[pk.njobs + 1] = pk.blk_start[pk.njobs] + blocks;
    pk.njobs++;
}

}  // namespace

extern "C" int pmat_mul_noalloc(uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA, const void *B,
                                int64_t dB, void *C, void *cuda_stream)
{
    if (m < 1 || n < 1 || k < 1 || dA < 1 || dB < 1 || p < 2 || (w != 4 && w != 8) ||
        (w == 4 && p > (1ull << 32)) || p >= (1ull << 62) || !A || !B || !C)
        return PM_EINVAL;
    // each length bounded before their sum is formed (no overflow of dA + dB - 1)
    if (dA > (int64_t(1) << PM_MAX_LOG2L) || dB > (int64_t(1) << PM_MAX_LOG2L)) return PM_EINVAL;
    const int64_t len = dA + dB - 1;
    int lg = 4;
    while ((int64_t(1) << lg) < len) lg++;
    if (lg > PM_MAX_LOG2L) return PM_EINVAL;
    const int64_t L = int64_t(1) << lg;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // primes: p itself when it is an NTT prime for this length, else the CRT table
    std::call_once(g_table_once, [] {
        uint32_t qs[PM_MAXK];
        const int nq = ntt_prime_table(qs, PM_MAXK);
        for (int i = 0; i < nq; i++) { g_table.emplace_back(); make_prime(g_table.back(), qs[i]); }
    });
    std::vector<StaticPrime> pr;
    bool direct = false;
    if (p < (1ull << 30) && p > 2 && ((p - 1) % (uint64_t)L) == 0 && ntt_is_prime32(p)) {
        pr.emplace_back();
        make_prime(pr.back(), (u32)p);
        direct = true;
    } else {
        const int64_t dmin = dA < dB ? dA : dB;
        const double need = std::log2((double)n) + std::log2((double)dmin) + 2.0 * std::log2((double)(p - 1 ? p - 1 : 1));
        double have = 0;
        for (auto &s : g_table) {
            pr.push_back(s);
            have += std::log2((double)s.q);
            if (have > need + 0.01) break;
        }
        if (have <= need + 0.01) return PM_EUNSUPPORTED;
    }
    const int K = (int)pr.size();

    // scratch layout: per prime two twiddle tables, then the transform buffers
    const size_t eA = (size_t)m * n, eB = (size_t)n * k, eC = (size_t)m * k;
    const size_t btw = al256((size_t(1) << lg) * sizeof(uint2));
    const size_t bA = al256(eA * L * 4), bB = al256(eB * L * 4), bC = al256(eC * L * 4);
    const size_t bR = direct ? 0 : eC * (size_t)len * 4;
    const size_t need_bytes = K * (2 * btw + bA + bB + bC) + K * bR;
    if (need_bytes > PM_NOALLOC_SCRATCH_BYTES) return PM_ESCRATCH;

    // once per device, with that device current: the array's device address
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= PM_NOALLOC_MAX_DEVICES) return PM_ECUDA;
    char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        if (!g_dev_scratch[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_pm_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return PM_ECUDA;
            }
            g_dev_scratch[dev] = ptr;
        }
        scratch = (char *)g_dev_scratch[dev];
    }

    long long launches = 0;
    std::vector<PrimeDev> P(K);
    char *cur = scratch;
    for (int i = 0; i < K; i++) {
        uint2 *twf = (uint2 *)cur, *twi = (uint2 *)(cur + btw);
        cur += 2 * btw;
        if (launch_twiddles(twf, twi, pr[i].q, pr[i].rf, pr[i].ri, lg, st, &launches) != cudaSuccess) return PM_ECUDA;
        P[i] = dev_prime(pr[i], lg, twf, twi);
    }
    u32 *Ah = (u32 *)cur, *Bh = (u32 *)(cur + K * bA), *Ch = (u32 *)(cur + K * (bA + bB));
    u32 *Rs = (u32 *)(cur + K * (bA + bB + bC));
    const int LBL = PM_LB_LOG2;

    // forward transforms
    {
        JobPack<FwdJob> pk; pk.njobs = 0; pk.blk_start[0] = 0;
        JobPack<ColJob> pc; pc.njobs = 0; pc.blk_start[0] = 0;
        for (int i = 0; i < K; i++)
            for (int opnd = 0; opnd < 2; opnd++) {
                const void *src = opnd ? B : A;
                const int64_t d = opnd ? dB : dA;
                const int ent = (int)(opnd ? eB : eA);
                u32 *dst = (u32 *)((char *)(opnd ? Bh : Ah) + i * (opnd ? bB : bA));
                if (lg <= LBL) {
                    FwdJob j;
                    j.src = src; j.dst = dst; j.src_stride = d; j.dst_stride = L; j.src_len = (int)d; j.src_mode = w;
                    j.count = ent; j.grp = 0; j.P = P[i];
                    const int epb = fwd_block_threads(lg) / (int)(L >> 4);
                    add(pk, j, (ent + epb - 1) / epb);
                } else {
                    ColJob c;
                    c.src = src; c.dst = dst; c.src_stride = d; c.dst_stride = L; c.src_len = (int)d; c.mode = w;
                    c.count = ent; c.out_off = 0; c.out_len = 0; c._pad = 0; c.P = P[i];
                    add(pc, c, ent * blocks_per_entry_cols(lg));
                    const int64_t nb = L >> LBL;
                    FwdJob j;
                    j.src = dst; j.dst = dst; j.src_stride = 1 << LBL; j.dst_stride = 1 << LBL; j.src_len = 1 << LBL;
                    j.src_mode = 0; j.count = (int)(ent * nb); j.grp = 0; j.P = P[i];
                    const int epb = fwd_block_threads(LBL) / ((1 << LBL) >> 4);
                    add(pk, j, (int)((ent * nb + epb - 1) / epb));
                }
            }
        if (pc.njobs && launch_ntt_fwd_cols(pc, lg, st, &launches) != cudaSuccess) return PM_ECUDA;
        if (launch_ntt_fwd_block(pk, lg > LBL ? LBL : lg, st, &launches) != cudaSuccess) return PM_ECUDA;
    }
    // pointwise products
    {
        JobPack<PwJob> pk; pk.njobs = 0; pk.blk_start[0] = 0;
        for (int i = 0; i < K; i++) {
            PwJob j;
            memset(&j, 0, sizeof(j));
            j.A = (u32 *)((char *)Ah + i * bA); j.B = (u32 *)((char *)Bh + i * bB); j.C = (u32 *)((char *)Ch + i * bC);
            j.m = m; j.n = n; j.k = k; j.L = (int)L; j.P = P[i];
            const int nb = pw_plan(j);
            add(pk, j, nb);
        }
        if (launch_pointwise(pk, st, &launches) != cudaSuccess) return PM_ECUDA;
    }
    // inverse transforms, scaled, the whole product
    {
        const int mode = direct ? w : 1;
        JobPack<InvJob> pk; pk.njobs = 0; pk.blk_start[0] = 0;
        JobPack<ColJob> pc; pc.njobs = 0; pc.blk_start[0] = 0;
        for (int i = 0; i < K; i++) {
            u32 *src = (u32 *)((char *)Ch + i * bC);
            void *dst = direct ? C : (void *)((char *)Rs + i * bR);
            if (lg <= LBL) {
                InvJob j;
                j.src = src; j.dst = dst; j.src_stride = L; j.dst_stride = len; j.out_off = 0; j.out_len = (int)len;
                j.dst_mode = mode; j.count = (int)eC; j.P = P[i];
                const int epb = fwd_block_threads(lg) / (int)(L >> 4);
                add(pk, j, (int)((eC + epb - 1) / epb));
            } else {
                const int64_t nb = L >> LBL;
                InvJob j;
                j.src = src; j.dst = src; j.src_stride = 1 << LBL; j.dst_stride = 1 << LBL; j.out_off = 0; j.out_len = 0;
                j.dst_mode = 0; j.count = (int)(eC * nb); j.P = P[i];
                const int epb = fwd_block_threads(LBL) / ((1 << LBL) >> 4);
                add(pk, j, (int)((eC * nb + epb - 1) / epb));
                ColJob c;
                c.src = src; c.dst = dst; c.src_stride = L; c.dst_stride = len; c.src_len = 0; c.mode = mode;
                c.count = (int)eC; c.out_off = 0; c.out_len = (int)len; c._pad = 0; c.P = P[i];
                add(pc, c, (int)eC * blocks_per_entry_cols(lg));
            }
        }
        if (launch_ntt_inv_block(pk, lg > LBL ? LBL : lg, st, &launches) != cudaSuccess) return PM_ECUDA;
        if (pc.njobs && launch_ntt_inv_cols(pc, lg, st, &launches) != cudaSuccess) return PM_ECUDA;
    }
    // CRT
    if (!direct) {
        JobPack<CrtJob> pk; pk.njobs = 0; pk.blk_start[0] = 0;
        CrtJob j;
        memset(&j, 0, sizeof(j));
        u32 qs[PM_MAXK];
        for (int i = 0; i < K; i++) qs[i] = pr[i].q;
        crt_setup(j, qs, K, p);
        j.res = Rs; j.dst = C; j.count = (int64_t)eC * len; j.len = len; j.dst_stride = len; j.w = w;
        add(pk, j, crt_blocks(j));
        if (launch_crt(pk, st, &launches) != cudaSuccess) return PM_ECUDA;
    }
    return PM_OK;
}
