// api.cu -- context management and the product entry points of the C ABI.
//
// Products (Sec. 2, "Polynomial matrix multiplication"): forward transforms
// of every entry of A and B, pointwise m x n . n x k products at every point,
// inverse transforms with the requested slice, and -- when p itself has no
// suitable roots of unity -- the same modulo K NTT primes followed by CRT.
// Transform lengths: full product L >= dA + dB - 1; truncated product mod x^t
// L >= min(dA,t) + min(dB,t) - 1; middle product of degrees c..c+d-1
// L >= c + d, since every aliased coefficient then lands below c.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "host.h"

// ------------------------------------------------------------------ errors
int pm_fail(pm_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int pm_cuda(pm_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PM_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return pm_fail(ctx, PM_ENOMEM, m);
    return pm_fail(ctx, PM_ECUDA, m);
}

#define CK(call)                                                        \
    do {                                                                \
        int _rc = pm_cuda(ctx, (call), #call);                          \
        if (_rc) return _rc;                                            \
    } while (0)
#define CKI(call)                                                       \
    do {                                                                \
        int _rc = (call);                                               \
        if (_rc) return _rc;                                            \
    } while (0)

int ceil_log2(int64_t x)
{
    int l = 0;
    while ((int64_t(1) << l) < x) l++;
    return l;
}

static void slot_init(PrimeSlot &s, uint32_t q)
{
    s.q = q;
    ntt_roots(q, s.rf, s.ri);
}

static int slot_tables(pm_ctx *ctx, PrimeSlot &s, int lg)
{
    if (s.maxlog >= lg && s.twf) return PM_OK;
    int want = lg < PM_LB_LOG2 ? PM_LB_LOG2 : lg;
    if (s.rf[want] == 0) want = lg;
    size_t bytes = (size_t(1) << want) * sizeof(uint2);
    if (s.twf) { CK(cudaFreeAsync(s.twf, ctx->stream)); CK(cudaFreeAsync(s.twi, ctx->stream)); }
    s.twf = s.twi = nullptr;
    CK(cudaMallocAsync((void **)&s.twf, bytes, ctx->stream));
    CK(cudaMallocAsync((void **)&s.twi, bytes, ctx->stream));
    CK(launch_twiddles(s.twf, s.twi, s.q, s.rf, s.ri, want, ctx->stream, &ctx->launches));
    s.maxlog = want;
    return PM_OK;
}

static PrimeDev prime_dev(const PrimeSlot &s, int lg)
{
    PrimeDev P;
    const uint64_t q = s.q;
    P.q = s.q;
    P.q2 = 2 * s.q;
    P.r32 = (u32)((1ull << 32) % q);
    P.r32s = (u32)(((uint64_t)P.r32 << 32) / q);
    P.ones = (u32)((1ull << 32) / q);
    uint64_t L = 1ull << lg;
    P.linv = (u32)host_powmod(L % q, q - 2, q);
    P.linvs = (u32)(((uint64_t)P.linv << 32) / q);
    P.twf = s.twf;
    P.twi = s.twi;
    return P;
}

// ------------------------------------------------------------------ memory
int host_join(pm_ctx *ctx)
{
    if (!ctx->host_pending) return PM_OK;
    for (int b = 0; b < 2; b++)
        if (ctx->out_rec[b]) CK(cudaStreamWaitEvent(ctx->stream, ctx->out_free[b], 0));
    ctx->host_pending = false;
    return PM_OK;
}

int ws_reserve(pm_ctx *ctx, size_t bytes, void **out)
{
    if (bytes > ctx->ws_size) {
        size_t want = bytes + (bytes >> 3);
        if (ctx->ws) CK(cudaFreeAsync(ctx->ws, ctx->stream));
        ctx->ws = nullptr;
        ctx->ws_size = 0;
        cudaError_t e = cudaMallocAsync(&ctx->ws, want, ctx->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->ws = nullptr;
            return pm_fail(ctx, PM_ENOMEM, "workspace allocation failed");
        }
        ctx->ws_size = want;
    }
    *out = ctx->ws;
    return PM_OK;
}

int arena_reserve(pm_ctx *ctx, size_t bytes)
{
    Arena &a = ctx->arena;
    a.used = 0;
    if (bytes <= a.size) return PM_OK;
    if (a.base) CK(cudaFreeAsync(a.base, ctx->stream));
    a.base = nullptr;
    a.size = 0;
    cudaError_t e = cudaMallocAsync((void **)&a.base, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        a.base = nullptr;
        return pm_fail(ctx, PM_ENOMEM, "driver arena allocation failed");
    }
    a.size = bytes;
    return PM_OK;
}

void *arena_alloc(pm_ctx *ctx, size_t bytes)
{
    Arena &a = ctx->arena;
    size_t off = (a.used + 255) & ~size_t(255);
    if (off + bytes > a.size) return nullptr;
    a.used = off + bytes;
    return a.base + off;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ------------------------------------------------------------------ stage timing
static cudaEvent_t take_event(pm_ctx *ctx)
{
    cudaEvent_t e = nullptr;
    if (!ctx->spare.empty()) { e = ctx->spare.back(); ctx->spare.pop_back(); }
    else cudaEventCreate(&e);
    return e;
}

// Every stage is also an NVTX range (named by stage) for timeline tools; the ranges cost a
// function-pointer test when no tool is attached.
static const char *const kStageNames[PM_NSTAGES] = {"pm:fwd_ntt", "pm:pointwise", "pm:inv_ntt", "pm:crt", "pm:leaf",
                                                    "pm:other"};

int stage_begin(pm_ctx *ctx, int stage)
{
    nvtxRangePushA(stage >= 0 && stage < PM_NSTAGES ? kStageNames[stage] : "pm:stage");
    if (!ctx->opt_timing) return -1;
    pm_ctx::Mark mk;
    mk.stage = stage;
    mk.a = take_event(ctx);
    mk.b = take_event(ctx);
    mk.launches = ctx->launches;
    cudaEventRecord(mk.a, ctx->stream);
    ctx->marks.push_back(mk);
    return (int)ctx->marks.size() - 1;
}

void stage_end(pm_ctx *ctx, int token)
{
    nvtxRangePop();
    if (token < 0 || token >= (int)ctx->marks.size()) return;
    pm_ctx::Mark &mk = ctx->marks[token];
    mk.launches = ctx->launches - mk.launches;
    cudaEventRecord(mk.b, ctx->stream);
}

// ------------------------------------------------------------------ primes per product
// The product is exact over Z when prod q_i exceeds the largest integer
// coefficient n . min(dA, dB) . (p-1)^2.
static int choose_primes(pm_ctx *ctx, uint64_t p, int n, int64_t dmin, int lg, std::vector<PrimeSlot *> &out,
                         bool &direct)
{
    out.clear();
    direct = false;
    if (p < (1ull << 30) && p > 2 && ((p - 1) % (1ull << lg)) == 0) {
        for (auto &s : ctx->direct)                   // a slot exists only for a prime: no test again
            if (s.q == p) { out.push_back(&s); direct = true; return PM_OK; }
    }
    if (p < (1ull << 30) && p > 2 && ((p - 1) % (1ull << lg)) == 0 && ntt_is_prime32(p)) {
        ctx->direct.emplace_back();
        slot_init(ctx->direct.back(), (u32)p);
        out.push_back(&ctx->direct.back());
        direct = true;
        return PM_OK;
    }
    const double need = std::log2((double)n) + std::log2((double)dmin) + 2.0 * std::log2((double)(p - 1 ? p - 1 : 1));
    double have = 0;
    for (auto &s : ctx->table) {
        out.push_back(&s);
        have += std::log2((double)s.q);
        if (have > need + 0.01) break;
    }
    if (have <= need + 0.01) return pm_fail(ctx, PM_EUNSUPPORTED, "product needs more CRT primes than the table holds");
    return PM_OK;
}

static void fill_crt(CrtJob &J, const std::vector<PrimeSlot *> &pr, uint64_t p)
{
    u32 q[PM_MAXK];
    for (size_t i = 0; i < pr.size(); i++) q[i] = pr[i]->q;
    crt_setup(J, q, (int)pr.size(), p);
}

// ------------------------------------------------------------------ checks
__global__ void k_check_range(const void *x, int64_t count, int w, uint64_t p, int *status)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t v = w == 8 ? ((const uint64_t *)x)[i] : ((const uint32_t *)x)[i];
        if (v >= p) atomicCAS(status, 0, PM_EDOMAIN);
    }
}

static int debug_check(pm_ctx *ctx, const void *x, int64_t count, int w, uint64_t p)
{
    if (!ctx->opt_debug) return PM_OK;
    k_check_range<<<256, 256, 0, ctx->stream>>>(x, count, w, p, ctx->d_status);
    ctx->launches++;
    CK(cudaGetLastError());
    int st = 0;
    CK(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (st == PM_EDOMAIN) {
        CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
        return pm_fail(ctx, PM_EDOMAIN, "input coefficient not in [0, p)");
    }
    return PM_OK;
}

// ------------------------------------------------------------------ product core
template <typename J>
static void pack_add(JobPack<J> &pk, const J &job, int blocks)
{
    const int n = pk.njobs;
    pk.jobs[n] = job;
    pk.blk_start[n + 1] = pk.blk_start[n] + blocks;
    pk.njobs = n + 1;
}

template <typename J>
static void pack_reset(JobPack<J> &pk)
{
    pk.njobs = 0;
    pk.blk_start[0] = 0;
}

static int fwd_entries_per_block(int lg)
{
    const int tpt = (1 << lg) >> 4, th = fwd_block_threads(lg);
    return th / tpt;
}

// Forward jobs of one operand modulo one prime (a column pass first when L > 2^14, except for
// 2^15 points and inputs of at most 2^14 coefficients: two block jobs, the odd half twisted).
static void add_forward(const PrimeDev &P, const void *src, int mode, int64_t src_stride, int64_t src_len,
                        int entries, u32 *dst, int lg, std::vector<FwdJob> &blk, std::vector<int> &blk_n,
                        std::vector<ColJob> &col, std::vector<int> &col_n)
{
    const int64_t L = int64_t(1) << lg;
    if (lg == PM_LB_LOG2 + 1 && src_len <= (int64_t(1) << PM_LB_LOG2)) {
        const int epb = fwd_entries_per_block(PM_LB_LOG2);
        for (int h = 0; h < 2; h++) {
            FwdJob j;
            j.src = src; j.dst = dst + ((size_t)h << PM_LB_LOG2); j.src_stride = src_stride; j.dst_stride = L;
            j.src_len = (int)src_len; j.src_mode = mode | (h ? PM_FWD_TWIST : 0); j.count = entries; j.grp = 0; j.P = P;
            blk.push_back(j);
            blk_n.push_back((entries + epb - 1) / epb);
        }
        return;
    }
    if (lg <= PM_LB_LOG2) {
        FwdJob j;
        j.src = src; j.dst = dst; j.src_stride = src_stride; j.dst_stride = L;
        j.src_len = (int)src_len; j.src_mode = mode; j.count = entries; j.grp = 0; j.P = P;
        const int epb = fwd_entries_per_block(lg);
        blk.push_back(j);
        blk_n.push_back((entries + epb - 1) / epb);
    } else {
        ColJob c;
        c.src = src; c.dst = dst; c.src_stride = src_stride; c.dst_stride = L;
        c.src_len = (int)src_len; c.mode = mode; c.count = entries; c.out_off = 0; c.out_len = 0; c._pad = 0; c.P = P;
        col.push_back(c);
        col_n.push_back(entries * blocks_per_entry_cols(lg));
        FwdJob j;
        const int64_t nb = L >> PM_LB_LOG2;
        j.src = dst; j.dst = dst; j.src_stride = 1 << PM_LB_LOG2; j.dst_stride = 1 << PM_LB_LOG2;
        j.src_len = 1 << PM_LB_LOG2; j.src_mode = 0; j.count = (int)(entries * nb); j.grp = 0; j.P = P;
        const int epb = fwd_entries_per_block(PM_LB_LOG2);
        blk.push_back(j);
        blk_n.push_back((int)((entries * nb + epb - 1) / epb));
    }
}

// Launch a list of jobs in packs of PM_MAXJ.
template <typename J, typename F>
static int launch_packs(pm_ctx *ctx, const std::vector<J> &jobs, const std::vector<int> &nblk, F launch)
{
    size_t i = 0;
    while (i < jobs.size()) {
        JobPack<J> pk;
        pack_reset(pk);
        while (i < jobs.size() && pk.njobs < PM_MAXJ) { pack_add(pk, jobs[i], nblk[i]); i++; }
        CK(launch(pk));
    }
    return PM_OK;
}

// Jobs [g0, blk.size()) transform one source modulo different primes (one job each, or the two
// halves of each 2^15-point transform), all reading the source with the same number of blocks:
// mark them an interleave group.  Block jobs after a column pass read their own staging
// arrays and stay ungrouped.
static void group_forward(std::vector<FwdJob> &blk, size_t g0, int lg)
{
    const size_t G = blk.size() - g0;
    if (lg > PM_LB_LOG2 + 1 || G < 2 || G > 255) return;
    for (size_t i = g0; i < blk.size(); i++)
        if ((blk[i].src_mode & 0xff) == 0 || blk[i].count != blk[g0].count) return;
    for (size_t i = 0; i < G; i++) blk[g0 + i].grp = (int)((G << 8) | i);
}

// Forward block jobs in packs of PM_MAXJ that never split an interleave group.
static int launch_fwd_packs(pm_ctx *ctx, const std::vector<FwdJob> &jobs, const std::vector<int> &nblk, int blg)
{
    size_t i = 0;
    while (i < jobs.size()) {
        JobPack<FwdJob> pk;
        pack_reset(pk);
        while (i < jobs.size()) {
            const int G = jobs[i].grp ? jobs[i].grp >> 8 : 1;
            if (pk.njobs + G > PM_MAXJ) break;
            for (int g = 0; g < G; g++, i++) pack_add(pk, jobs[i], nblk[i]);
        }
        CK(launch_ntt_fwd_block(pk, blg, ctx->stream, &ctx->launches));
    }
    return PM_OK;
}

// Forward jobs of one transform length: column passes first, then the blocks.
static int launch_fwd_lists(pm_ctx *ctx, const std::vector<FwdJob> &blk, const std::vector<int> &bn,
                            const std::vector<ColJob> &col, const std::vector<int> &cn, int lg)
{
    if (!col.empty())
        CKI(launch_packs(ctx, col, cn, [&](const JobPack<ColJob> &pk) {
            return launch_ntt_fwd_cols(pk, lg, ctx->stream, &ctx->launches); }));
    if (!blk.empty()) CKI(launch_fwd_packs(ctx, blk, bn, lg > PM_LB_LOG2 ? PM_LB_LOG2 : lg));
    return PM_OK;
}

// Algorithmic work of one product (the measure the roofline fractions use): the compulsory
// bytes (inputs read once, the output written once), the pointwise modular multiply-adds
// (K primes x L points x m n k) and the butterflies of every transform (K (mn + nk + mk)
// transforms of (L/2) lg L butterflies).
static void count_work(pm_ctx *ctx, int K, int lg, int w, int m, int n, int k, int64_t dA, int64_t dB, int64_t len)
{
    const int64_t L = int64_t(1) << lg;
    ctx->work[0] += ((int64_t)m * n * dA + (int64_t)n * k * dB + (int64_t)m * k * len) * w;
    ctx->work[1] += (int64_t)K * L * m * n * k;
    ctx->work[2] += (int64_t)K * ((int64_t)m * n + (int64_t)n * k + (int64_t)m * k) * (L / 2) * lg;
}

namespace {
struct Plan {
    std::vector<PrimeSlot *> pr;
    bool direct;
    size_t bA, bB, bC, bR, total;
    int64_t out_len;
};

// Pointwise jobs sorted by kernel form.
struct PwLists {
    std::vector<PwJob> jobs, jobs4, tjobs, sjobs[9], vjobs, gjobs;    // jobs: 4 x 8 thread tiles, jobs4: 4 x 4
    std::vector<int> nb, nb4, tnb, snb[9], vnb;
};

// Inverse-transform jobs of one transform length (a column pass after the blocks when L > 2^14).
struct InvLists {
    std::vector<InvJob> blk;
    std::vector<int> bn;
    std::vector<ColJob> col;
    std::vector<int> cn;
    std::vector<InvJob> pair;       // 2^15 points: both halves and the step over them in one CTA
    std::vector<int> pn;
};
}  // namespace

// Prime i's transforms of a request's A: the caller's (At, At_out) or the workspace's.
static u32 *a_transform(const ProdReq &q, const Plan &P, char *ws_A, size_t i)
{
    if (q.At) return (u32 *)q.At + i * (P.bA / 4);
    if (q.At_out) return q.At_out + i * (P.bA / 4);
    return (u32 *)(ws_A + i * P.bA);
}

size_t prod_operand_bytes(pm_ctx *ctx, uint64_t p, int n, int64_t dmin, int lg, int64_t entries)
{
    std::vector<PrimeSlot *> pr;
    bool direct = false;
    if (choose_primes(ctx, p, n, dmin, lg, pr, direct)) return 0;
    return pr.size() * align256((size_t)entries * ((size_t)1 << lg) * 4);
}

// Pointwise m x n . n x k products at every point of one prime's transforms: tensor-core limb
// products where the shape allows (m, n, k <= 32) when that form is requested, small inner
// dimensions (n <= 8) by a streaming kernel (one launch per n), matrix-vector products
// (k = 1, n <= 64) by another, the staged CUDA-core 64-bit form otherwise (4 x 8 or 4 x 4
// thread tiles by the cost model, or as the tuner recorded or option 4 asks).
// With PM_OPT_POINTWISE = 0 a form recorded by pm_tune_product for the same (m, n, k, length) is
// taken; otherwise (and for forms that do not apply) the rules above.
static void add_pointwise(pm_ctx *ctx, PwLists &pl, u32 *A, u32 *B, u32 *C, int m, int n, int k, int lg,
                          const PrimeDev &D)
{
    PwJob j;
    memset(&j, 0, sizeof(j));
    j.A = A; j.B = B; j.C = C;
    j.m = m; j.n = n; j.k = k; j.L = 1 << lg; j.P = D;
    int form = 0, bi = 0, bk = 0;
    if (ctx->force_form >= 0) { form = ctx->force_form; bi = ctx->force_bi; bk = ctx->force_bk; }
    else if (ctx->opt_pointwise == 2) form = 2;
    else if (ctx->opt_pointwise == 0)
        for (const auto &t : ctx->tune)
            if (t.m == m && t.n == n && t.k == k && t.lg == lg) { form = t.form; bi = t.bi; bk = t.bk; break; }
    if (ctx->opt_pointwise == 3 && ctx->force_form < 0) form = 5;
    if (ctx->opt_pointwise == 4 && ctx->force_form < 0) {          // 4 x 4 thread tiles, cost-model block
        form = 6;
        pw_tiles(j, &bi, &bk, 1, 4);
    }
    // automatic rule, measured on GB300: the dense tensor-core form wins for large per-point
    // products (512 x 512 . 512 x 512 at 256 points: 4.04 ms against 6.21 ms on CUDA cores) and
    // loses at 128 x 128 . 128 x 128 (1.22 against 0.81 ms)
    if (ctx->opt_pointwise == 0 && form == 0 && ctx->force_form < 0 && m >= 256 && n >= 256 && k >= 256) form = 5;
    if (form == 5 && j.m >= 64) { pl.gjobs.push_back(j); return; }
    if (form == 2 && tc_supported(j)) { pl.tjobs.push_back(j); pl.tnb.push_back(tc_blocks(j)); }
    else if (form == 1 && bi > 0 && bk > 0) { const int nbk = pw_plan_tile(j, bi, bk, 8); pl.jobs.push_back(j); pl.nb.push_back(nbk); }
    else if (form == 6 && bi > 0 && bk > 0) { const int nbk = pw_plan_tile(j, bi, bk, 4); pl.jobs4.push_back(j); pl.nb4.push_back(nbk); }
    else if (form == 4 && pwv_supported(j)) { pl.vjobs.push_back(j); pl.vnb.push_back(pwv_blocks(j)); }
    else if ((form == 0 || form == 3 || form == 2) && pws_supported(j)) { pl.sjobs[j.n].push_back(j); pl.snb[j.n].push_back(pws_blocks(j)); }
    else if ((form == 0 || form == 2) && pwv_supported(j)) { pl.vjobs.push_back(j); pl.vnb.push_back(pwv_blocks(j)); }
    else {
        const int nbk = pw_plan(j);
        (j.cw == 4 ? pl.jobs4 : pl.jobs).push_back(j);
        (j.cw == 4 ? pl.nb4 : pl.nb).push_back(nbk);
    }
}

static int launch_pointwise_lists(pm_ctx *ctx, const PwLists &pl)
{
    if (!pl.jobs.empty())
        CKI(launch_packs(ctx, pl.jobs, pl.nb, [&](const JobPack<PwJob> &pk) {
            return launch_pointwise(pk, ctx->stream, &ctx->launches); }));
    if (!pl.jobs4.empty())
        CKI(launch_packs(ctx, pl.jobs4, pl.nb4, [&](const JobPack<PwJob> &pk) {
            return launch_pointwise(pk, ctx->stream, &ctx->launches); }));
    if (!pl.vjobs.empty())
        CKI(launch_packs(ctx, pl.vjobs, pl.vnb, [&](const JobPack<PwJob> &pk) {
            return launch_pointwise_mv(pk, ctx->stream, &ctx->launches); }));
    for (int nn = 1; nn <= 8; nn++)
        if (!pl.sjobs[nn].empty())
            CKI(launch_packs(ctx, pl.sjobs[nn], pl.snb[nn], [&](const JobPack<PwJob> &pk) {
                return launch_pointwise_sn(pk, ctx->stream, &ctx->launches); }));
    if (!pl.tjobs.empty())
        CKI(launch_packs(ctx, pl.tjobs, pl.tnb, [&](const JobPack<PwJob> &pk) {
            return launch_pointwise_tc(pk, ctx->d_status, ctx->stream, &ctx->launches, ctx->opt_withhold); }));
    for (const PwJob &j : pl.gjobs) CKI(pointwise_gemm(ctx, j));
    return PM_OK;
}

// The pointwise stage alone, for transforms computed elsewhere (the Vandermonde products).
int run_pointwise(pm_ctx *ctx, u32 *A, u32 *B, u32 *C, int m, int n, int k, int lg, const PrimeDev &D)
{
    PwLists pl;
    add_pointwise(ctx, pl, A, B, C, m, n, k, lg, D);
    return launch_pointwise_lists(ctx, pl);
}

// Work of a Vandermonde product (one prime): its compulsory bytes and pointwise multiply-adds.
void count_work_vdm(pm_ctx *ctx, int lg, int m, int n, int k, int64_t dA, int64_t dB, int64_t len)
{
    ctx->work[0] += ((int64_t)m * n * dA + (int64_t)n * k * dB + (int64_t)m * k * len) * 4;
    ctx->work[1] += (int64_t)(int64_t(1) << lg) * m * n * k;
}

// Inverse transforms of eC entries (src, stride L) modulo one prime; coefficients off ..
// off+out_len-1 of each go to dst (entry stride dstride) in the given mode (1 = u32 residues,
// 4 / 8 = the caller's element width).
static void add_inverse(InvLists &il, const PrimeDev &D, u32 *src, void *dst, int64_t dstride, int mode,
                        int64_t off, int64_t out_len, int64_t eC, int lg)
{
    const int64_t L = int64_t(1) << lg;
    if (lg <= PM_LB_LOG2 || lg == PM_LB_LOG2 + 1) {
        InvJob j;
        j.src = src; j.dst = dst; j.src_stride = L; j.dst_stride = dstride;
        j.out_off = (int)off; j.out_len = (int)out_len; j.dst_mode = mode; j.count = (int)eC; j.P = D;
        if (lg > PM_LB_LOG2) {
            il.pair.push_back(j);
            il.pn.push_back((int)eC);
            return;
        }
        const int epb = fwd_entries_per_block(lg);
        il.blk.push_back(j);
        il.bn.push_back((int)((eC + epb - 1) / epb));
    } else {
        const int64_t nbk = L >> PM_LB_LOG2;
        InvJob j;
        j.src = src; j.dst = src; j.src_stride = 1 << PM_LB_LOG2; j.dst_stride = 1 << PM_LB_LOG2;
        j.out_off = 0; j.out_len = 0; j.dst_mode = 0; j.count = (int)(eC * nbk); j.P = D;
        const int epb = fwd_entries_per_block(PM_LB_LOG2);
        il.blk.push_back(j);
        il.bn.push_back((int)((eC * nbk + epb - 1) / epb));
        ColJob c;
        c.src = src; c.dst = dst; c.src_stride = L; c.dst_stride = dstride;
        c.src_len = 0; c.mode = mode; c.count = (int)eC; c.out_off = (int)off;
        c.out_len = (int)out_len; c._pad = 0; c.P = D;
        il.col.push_back(c);
        il.cn.push_back((int)eC * blocks_per_entry_cols(lg));
    }
}

static int launch_inverse_lists(pm_ctx *ctx, const InvLists &il, int lg)
{
    if (!il.blk.empty()) {
        const int blg = lg > PM_LB_LOG2 ? PM_LB_LOG2 : lg;
        CKI(launch_packs(ctx, il.blk, il.bn, [&](const JobPack<InvJob> &pk) {
            return launch_ntt_inv_block(pk, blg, ctx->stream, &ctx->launches); }));
    }
    if (!il.col.empty())
        CKI(launch_packs(ctx, il.col, il.cn, [&](const JobPack<ColJob> &pk) {
            return launch_ntt_inv_cols(pk, lg, ctx->stream, &ctx->launches); }));
    if (!il.pair.empty())
        CKI(launch_packs(ctx, il.pair, il.pn, [&](const JobPack<InvJob> &pk) {
            return launch_ntt_inv_pair(pk, ctx->stream, &ctx->launches); }));
    return PM_OK;
}

#define PM_BATCH_WS_CAP (16ull << 30)   // workspace bytes per chunk of a batch

int prod_batch(pm_ctx *ctx, const ProdReq *reqs, int count)
{
    CKI(host_join(ctx));   // the workspace may hold a staging set a download still reads
    // ---- plan every request; size the twiddle tables before any job takes their addresses
    std::vector<Plan> plan(count);
    for (int r = 0; r < count; r++) {
        const ProdReq &q = reqs[r];
        if (q.lg > PM_MAX_LOG2L) return pm_fail(ctx, PM_EINVAL, "transform longer than 2^20 points");
        Plan &P = plan[r];
        CKI(choose_primes(ctx, q.p, q.n, q.dA < q.dB ? q.dA : q.dB, q.lg, P.pr, P.direct));
        const int64_t L = int64_t(1) << q.lg;
        const size_t eA = (size_t)q.m * q.n, eB = (size_t)q.n * q.k, eC = (size_t)q.m * q.k;
        P.bA = align256(eA * L * 4);
        P.bB = align256(eB * L * 4);
        P.bC = align256(eC * L * 4);
        P.bR = P.direct ? 0 : eC * (size_t)q.len * 4;     // packed planes: the CRT kernel reads res + i * count
        P.total = P.pr.size() * (P.bA + P.bB + P.bC) + align256(P.pr.size() * P.bR);
        P.out_len = q.off + q.len <= L ? q.len : (q.off < L ? L - q.off : 0);
    }
    for (int r = 0; r < count; r++)
        for (auto *s : plan[r].pr) CKI(slot_tables(ctx, *s, reqs[r].lg));
    for (int r = 0; r < count; r++) {
        const ProdReq &q = reqs[r];
        count_work(ctx, (int)plan[r].pr.size(), q.lg, q.w, q.m, q.n, q.k, q.dA, q.dB, q.len);
    }

    // ---- chunks under the workspace cap
    int r0 = 0;
    while (r0 < count) {
        size_t tot = plan[r0].total;
        int r1 = r0 + 1;
        while (r1 < count && tot + plan[r1].total <= PM_BATCH_WS_CAP) tot += plan[r1].total, r1++;
        void *ws = nullptr;
        CKI(ws_reserve(ctx, tot + 256, &ws));
        struct Bufs { char *A, *B, *C, *R; };
        std::vector<Bufs> buf(r1 - r0);
        char *cur = (char *)ws;
        for (int r = r0; r < r1; r++) {
            const Plan &P = plan[r];
            const size_t K = P.pr.size();
            Bufs &b = buf[r - r0];
            b.A = cur; cur += K * P.bA;
            b.B = cur; cur += K * P.bB;
            b.C = cur; cur += K * P.bC;
            b.R = cur; cur += align256(K * P.bR);
        }
        // 1. forward transforms, binned by transform length
        int tok = stage_begin(ctx, PM_STAGE_FWD);
        for (int lg = 4; lg <= PM_MAX_LOG2L; lg++) {
            std::vector<FwdJob> blk; std::vector<int> bn;
            std::vector<ColJob> col; std::vector<int> cn;
            for (int r = r0; r < r1; r++) {
                const ProdReq &q = reqs[r];
                if (q.lg != lg) continue;
                const Plan &P = plan[r];
                const Bufs &b = buf[r - r0];
                // operand by operand, every prime of one operand side by side (one interleave group)
                if (!q.At) {                            // A's transforms: computed (kept if asked)
                    const size_t g0 = blk.size();
                    for (size_t i = 0; i < P.pr.size(); i++)
                        add_forward(prime_dev(*P.pr[i], lg), q.A, q.w, q.sA, q.dA, q.m * q.n, a_transform(q, P, b.A, i),
                                    lg, blk, bn, col, cn);
                    group_forward(blk, g0, lg);
                }
                const size_t g0 = blk.size();
                for (size_t i = 0; i < P.pr.size(); i++)
                    add_forward(prime_dev(*P.pr[i], lg), q.B, q.w, q.sB, q.dB, q.n * q.k, (u32 *)(b.B + i * P.bB), lg,
                                blk, bn, col, cn);
                group_forward(blk, g0, lg);
            }
            CKI(launch_fwd_lists(ctx, blk, bn, col, cn, lg));
        }
        stage_end(ctx, tok);
        // 2. pointwise products (jobs of any length share launches)
        tok = stage_begin(ctx, PM_STAGE_POINTWISE);
        {
            PwLists pl;
            for (int r = r0; r < r1; r++) {
                const ProdReq &q = reqs[r];
                const Plan &P = plan[r];
                const Bufs &b = buf[r - r0];
                for (size_t i = 0; i < P.pr.size(); i++)
                    add_pointwise(ctx, pl, a_transform(q, P, b.A, i), (u32 *)(b.B + i * P.bB), (u32 *)(b.C + i * P.bC),
                                  q.m, q.n, q.k, q.lg, prime_dev(*P.pr[i], q.lg));
            }
            CKI(launch_pointwise_lists(ctx, pl));
        }
        stage_end(ctx, tok);
        // 3. inverse transforms, scaled, writing each slice, binned by length
        tok = stage_begin(ctx, PM_STAGE_INV);
        for (int lg = 4; lg <= PM_MAX_LOG2L; lg++) {
            InvLists il;
            for (int r = r0; r < r1; r++) {
                const ProdReq &q = reqs[r];
                if (q.lg != lg) continue;
                const Plan &P = plan[r];
                const Bufs &b = buf[r - r0];
                for (size_t i = 0; i < P.pr.size(); i++)
                    add_inverse(il, prime_dev(*P.pr[i], lg), (u32 *)(b.C + i * P.bC),
                                P.direct ? q.C : (void *)(b.R + i * P.bR), P.direct ? q.sC : q.len, P.direct ? q.w : 1,
                                q.off, P.out_len, (int64_t)q.m * q.k, lg);
            }
            CKI(launch_inverse_lists(ctx, il, lg));
        }
        stage_end(ctx, tok);
        // 4. CRT recombination into values mod p
        tok = stage_begin(ctx, PM_STAGE_CRT);
        {
            std::vector<CrtJob> jobs; std::vector<int> nb;
            for (int r = r0; r < r1; r++) {
                const Plan &P = plan[r];
                if (P.direct) continue;
                const ProdReq &q = reqs[r];
                CrtJob j;
                memset(&j, 0, sizeof(j));
                fill_crt(j, P.pr, q.p);
                j.res = (const u32 *)buf[r - r0].R; j.dst = q.C; j.count = (int64_t)q.m * q.k * q.len;
                j.len = q.len; j.dst_stride = q.sC; j.w = q.w;
                jobs.push_back(j);
                nb.push_back(crt_blocks(j));
            }
            if (!jobs.empty())
                CKI(launch_packs(ctx, jobs, nb, [&](const JobPack<CrtJob> &pk) {
                    return launch_crt(pk, ctx->stream, &ctx->launches); }));
        }
        stage_end(ctx, tok);
        // 5. slice positions beyond the transform length are zero
        for (int r = r0; r < r1; r++) {
            const ProdReq &q = reqs[r];
            const Plan &P = plan[r];
            if (P.out_len < q.len) {
                const int64_t z0 = P.out_len > 0 ? P.out_len : 0;
                CK(cudaMemset2DAsync((char *)q.C + z0 * q.w, (size_t)q.sC * q.w, 0, (size_t)(q.len - z0) * q.w,
                                     (size_t)q.m * q.k, ctx->stream));
            }
        }
        r0 = r1;
    }
    return PM_OK;
}

int prod_slice(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA, int64_t sA,
               const void *B, int64_t dB, int64_t sB, int64_t off, int64_t len, int lg, void *C, int64_t sC)
{
    ProdReq q;
    q.p = p; q.w = w; q.m = m; q.n = n; q.k = k; q.lg = lg < 4 ? 4 : lg;
    q.A = A; q.B = B; q.C = C; q.dA = dA; q.sA = sA; q.dB = dB; q.sB = sB; q.off = off; q.len = len; q.sC = sC;
    return prod_batch(ctx, &q, 1);
}

// Small products modulo an NTT prime used directly (L <= 2^10 points, n <= 16, the transforms of
// all entries in at most 160 KB of shared memory) in one CTA and one launch (small.cu), instead
// of the batched path's three launches; not when a pointwise form is forced (the tests of each
// form must reach it).  The launch is recorded as the forward stage.  done = false: not taken.
static int small_product(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA,
                         const void *B, int64_t dB, void *C, int64_t len, int lg, bool &done)
{
    done = false;
    const int lg4 = lg < 4 ? 4 : lg;
    if (lg4 > 10 || n > 16 || ctx->force_form >= 0 || ctx->opt_pointwise != 0) return PM_OK;
    if (p >= (1ull << 30) || p < 3 || ((p - 1) % (1ull << lg4)) != 0) return PM_OK;
    if (small_product_smem(m, n, k, lg4) > 160 * 1024) return PM_OK;
    std::vector<PrimeSlot *> pr;
    bool direct = false;
    CKI(choose_primes(ctx, p, n, dA < dB ? dA : dB, lg4, pr, direct));
    if (!direct) return PM_OK;
    CKI(host_join(ctx));
    CKI(slot_tables(ctx, *pr[0], lg4));
    count_work(ctx, 1, lg4, w, m, n, k, dA, dB, len);
    SmallJob J;
    J.A = A; J.B = B; J.C = C;
    J.w = w; J.m = m; J.n = n; J.k = k; J.dA = (int)dA; J.dB = (int)dB; J.len = (int)len; J.lg = lg4;
    J.P = prime_dev(*pr[0], lg4);
    const int tok = stage_begin(ctx, PM_STAGE_FWD);
    ctx->launches++;
    const cudaError_t e = launch_small_product(J, ctx->stream);
    stage_end(ctx, tok);
    CKI(pm_cuda(ctx, e, "k_small_product"));
    done = true;
    return PM_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int pm_create(pm_ctx **out, int device, void *cuda_stream)
{
    if (!out) return PM_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return PM_EINVAL;
    }
    pm_ctx *ctx = new (std::nothrow) pm_ctx();
    if (!ctx) return PM_ENOMEM;
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return PM_ECUDA; }
    if (cuda_stream) ctx->stream = (cudaStream_t)cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return PM_ECUDA; }
        ctx->stream = ctx->own;
    }
    if (cudaMalloc((void **)&ctx->d_status, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->own) cudaStreamDestroy(ctx->own);
        delete ctx;
        return PM_ECUDA;
    }
    // CRT primes: q = c 2^20 + 1 < 2^30, largest first (all in (2^29, 2^30))
    uint32_t qs[PM_MAXK];
    const int nq = ntt_prime_table(qs, PM_MAXK);
    for (int i = 0; i < nq; i++) {
        ctx->table.emplace_back();
        slot_init(ctx->table.back(), qs[i]);
    }
    *out = ctx;
    return PM_OK;
}

int pm_destroy(pm_ctx *ctx)
{
    if (!ctx) return PM_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &s : ctx->table) { cudaFree(s.twf); cudaFree(s.twi); }
    for (auto &s : ctx->direct) { cudaFree(s.twf); cudaFree(s.twi); }
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->arena.base) cudaFree(ctx->arena.base);
    if (ctx->gemm_ws) cudaFree(ctx->gemm_ws);
    if (ctx->d_status) cudaFree(ctx->d_status);
    for (auto &mk : ctx->marks) { cudaEventDestroy(mk.a); cudaEventDestroy(mk.b); }
    for (auto e : ctx->spare) cudaEventDestroy(e);
    if (ctx->up) cudaStreamSynchronize(ctx->up);
    if (ctx->dn) cudaStreamSynchronize(ctx->dn);
    for (auto e : ctx->hev) cudaEventDestroy(e);
    for (int i = 0; i < 2; i++) {
        if (ctx->in_free[i]) cudaEventDestroy(ctx->in_free[i]);
        if (ctx->out_free[i]) cudaEventDestroy(ctx->out_free[i]);
    }
    if (ctx->ws_ready) cudaEventDestroy(ctx->ws_ready);
    if (ctx->up) cudaStreamDestroy(ctx->up);
    if (ctx->dn) cudaStreamDestroy(ctx->dn);
    if (ctx->own) cudaStreamDestroy(ctx->own);
    delete ctx;
    return PM_OK;
}

int pm_set_option(pm_ctx *ctx, int key, int64_t value)
{
    if (!ctx) return PM_EINVAL;
    switch (key) {
    case PM_OPT_POINTWISE:
        if (value < 0 || value > 4) return pm_fail(ctx, PM_EINVAL, "pointwise path must be 0, 1, 2, 3 or 4");
        ctx->opt_pointwise = (int)value;
        return PM_OK;
    case PM_OPT_THRESHOLD:
        if (value < 1) return pm_fail(ctx, PM_EINVAL, "threshold must be >= 1");
        ctx->opt_T = value;
        return PM_OK;
    case PM_OPT_DEBUG_CHECKS:
        ctx->opt_debug = value ? 1 : 0;
        return PM_OK;
    case PM_OPT_STAGE_TIMING:
        ctx->opt_timing = value ? 1 : 0;
        return PM_OK;
    case PM_OPT_LEAF_CLUSTER:
        ctx->opt_leaf_cluster = value ? 1 : 0;
        return PM_OK;
    case PM_OPT_TEST_WITHHOLD_MMA:
        ctx->opt_withhold = value ? 1 : 0;
        return PM_OK;
    case PM_OPT_HOST_CHUNKS:
        if (value < 0 || value > (1 << 20)) return pm_fail(ctx, PM_EINVAL, "host chunk count out of range");
        ctx->opt_host_chunks = (int)value;
        return PM_OK;
    default:
        return pm_fail(ctx, PM_EINVAL, "unknown option key");
    }
}

int pm_set_stream(pm_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return PM_EINVAL;
    CKI(host_join(ctx));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->stream = cuda_stream ? (cudaStream_t)cuda_stream : ctx->own;
    if (!ctx->stream) {
        CK(cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking));
        ctx->stream = ctx->own;
    }
    return PM_OK;
}

int pm_sync(pm_ctx *ctx)
{
    if (!ctx) return PM_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CKI(host_join(ctx));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->up) CK(cudaStreamSynchronize(ctx->up));   // also copies a failed call left in flight
    if (ctx->dn) CK(cudaStreamSynchronize(ctx->dn));
    int st = 0;
    CK(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
        return pm_fail(ctx, st, st == PM_ETIMEOUT ? "device-side wait timed out" : "device status error");
    }
    return PM_OK;
}

const char *pm_last_error(pm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t pm_kernel_launches(pm_ctx *ctx) { return ctx ? ctx->launches : -1; }

int pm_work_counters(pm_ctx *ctx, int64_t *out3, int reset)
{
    if (!ctx || !out3) return PM_EINVAL;
    for (int i = 0; i < 3; i++) out3[i] = ctx->work[i];
    if (reset)
        for (int i = 0; i < 3; i++) ctx->work[i] = 0;
    return PM_OK;
}

int pm_stage_times(pm_ctx *ctx, double *ms, int64_t *launches)
{
    if (!ctx) return PM_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ms) for (int i = 0; i < PM_NSTAGES; i++) ms[i] = 0;
    if (launches) for (int i = 0; i < PM_NSTAGES; i++) launches[i] = 0;
    for (auto &mk : ctx->marks) {
        float t = 0;
        CK(cudaEventElapsedTime(&t, mk.a, mk.b));
        if (ms) ms[mk.stage] += t;
        if (launches) launches[mk.stage] += mk.launches;
        ctx->spare.push_back(mk.a);
        ctx->spare.push_back(mk.b);
    }
    ctx->marks.clear();
    return PM_OK;
}

static int check_common(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA,
                        const void *B, int64_t dB, const void *C, bool device_inputs = true)
{
    if (!ctx) return PM_EINVAL;
    if (m < 1 || n < 1 || k < 1) return pm_fail(ctx, PM_EINVAL, "dimensions must be >= 1");
    if (dA < 1 || dB < 1) return pm_fail(ctx, PM_EINVAL, "lengths must be >= 1");
    if (p < 2) return pm_fail(ctx, PM_EINVAL, "modulus must be >= 2");
    if (w != 4 && w != 8) return pm_fail(ctx, PM_EINVAL, "element width must be 4 or 8");
    if (w == 4 && p > (1ull << 32)) return pm_fail(ctx, PM_EINVAL, "w = 4 needs p <= 2^32");
    if (p >= (1ull << 62)) return pm_fail(ctx, PM_EINVAL, "p must be below 2^62");
    if (!A || !B || !C) return pm_fail(ctx, PM_EINVAL, "null buffer");
    if (dA > (1 << PM_MAX_LOG2L) || dB > (1 << PM_MAX_LOG2L)) return pm_fail(ctx, PM_EINVAL, "length exceeds 2^20");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    if (device_inputs) {
        CKI(debug_check(ctx, A, (int64_t)m * n * dA, w, p));
        CKI(debug_check(ctx, B, (int64_t)n * k * dB, w, p));
    }
    return PM_OK;
}

// Rows [r0, r1) of chunk c when `rows` rows are cut into `nc` nearly equal chunks.
static void chunk_rows(int rows, int nc, int c, int &r0, int &r1)
{
    r0 = (int)((int64_t)rows * c / nc);
    r1 = (int)((int64_t)rows * (c + 1) / nc);
}

// The full product with A, B and C in host memory.  The uploads run on a second stream, B then
// A, each in up to two row chunks transformed as they land; the pointwise products run once over
// the whole product (cutting them by rows would reload B's transforms per chunk); the inverse
// transforms and the CRT then run in chunks of output entries, each copied back on the copy
// stream while the next chunk computes.
static int mul_host(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA,
                    const void *B, int64_t dB, void *C)
{
    const int64_t len = dA + dB - 1;
    const int lg = ceil_log2(len) < 4 ? 4 : ceil_log2(len);
    if (lg > PM_MAX_LOG2L) return pm_fail(ctx, PM_EINVAL, "product longer than 2^20");
    const int64_t L = int64_t(1) << lg;
    std::vector<PrimeSlot *> pr;
    bool direct = false;
    CKI(choose_primes(ctx, p, n, dA < dB ? dA : dB, lg, pr, direct));
    for (auto *sl : pr) CKI(slot_tables(ctx, *sl, lg));
    const size_t K = pr.size();
    count_work(ctx, (int)K, lg, w, m, n, k, dA, dB, len);
    const size_t eA = (size_t)m * n, eB = (size_t)n * k, eC = (size_t)m * k;
    const size_t bAh = eA * dA * w, bBh = eB * dB * w, bCh = eC * len * w;
    const size_t bA = align256(eA * L * 4), bB = align256(eB * L * 4), bC = align256(eC * L * 4);
    const size_t bR = direct ? 0 : K * eC * len * 4;
    const size_t stage = align256(bAh) + align256(bBh) + align256(bCh);   // one staging set
    const size_t total = 2 * stage + K * (bA + bB + bC) + align256(bR);
    if (total > PM_BATCH_WS_CAP) return pm_fail(ctx, PM_EUNSUPPORTED, "pmat_mul_host: product too large for one pass");
    // Chunking.  Inputs of 8 MB or more come in two row chunks, each transformed as it lands.
    // Output: consecutive calls overlap, so this call's download runs during the next call's
    // upload and work, and one output chunk is fastest for calls in a row (measured: 0.90 ms per
    // 32x32, length-4096 product, against 0.96 ms with 6 output chunks).  An explicit chunk
    // count N (latency, for a call on its own) pipelines N output chunks with their downloads.
    const int ncA = (bAh >= (8u << 20) && m >= 2) ? 2 : 1;
    const int ncB = (bBh >= (8u << 20) && n >= 2) ? 2 : 1;
    int ncO = ctx->opt_host_chunks > 0 ? ctx->opt_host_chunks : 1;
    if ((size_t)ncO > eC) ncO = (int)eC;
    const bool chunked = ncA > 1 || ncB > 1;
    // A new layout or a larger workspace: let every pending download finish first (the old
    // staging sets may move), and make the uploads wait for the (re)allocation.
    const bool relayout = stage != ctx->host_stage || total + 256 > ctx->ws_size;
    if (relayout) {
        CKI(host_join(ctx));
        ctx->in_rec[0] = ctx->in_rec[1] = ctx->out_rec[0] = ctx->out_rec[1] = false;
        ctx->host_stage = stage;
    }
    void *ws = nullptr;
    CKI(ws_reserve(ctx, total + 256, &ws));
    // the workspace moved (this call or another user grew it): the staging sets are new memory
    // that the upload stream may touch only after its allocation on the context's stream
    const bool moved = ws != ctx->host_ws;
    if (moved) {
        ctx->in_rec[0] = ctx->in_rec[1] = ctx->out_rec[0] = ctx->out_rec[1] = false;
        ctx->host_ws = ws;
    }
    const int sb = ctx->host_parity;                   // this call's staging set
    ctx->host_parity ^= 1;
    char *cur = (char *)ws + sb * stage;
    char *Ad = cur; cur += align256(bAh);
    char *Bd = cur; cur += align256(bBh);
    char *Cd = cur;
    cur = (char *)ws + 2 * stage;
    char *TA = cur; cur += K * bA;
    char *TB = cur; cur += K * bB;
    char *TC = cur; cur += K * bC;
    char *R = cur;
    if (!ctx->up) CK(cudaStreamCreateWithFlags(&ctx->up, cudaStreamNonBlocking));
    if (!ctx->dn) CK(cudaStreamCreateWithFlags(&ctx->dn, cudaStreamNonBlocking));
    for (int i = 0; i < 2; i++) {
        if (!ctx->in_free[i]) CK(cudaEventCreateWithFlags(&ctx->in_free[i], cudaEventDisableTiming));
        if (!ctx->out_free[i]) CK(cudaEventCreateWithFlags(&ctx->out_free[i], cudaEventDisableTiming));
    }
    if (!ctx->ws_ready) CK(cudaEventCreateWithFlags(&ctx->ws_ready, cudaEventDisableTiming));
    const int nev = ncA + ncB + ncO;
    while ((int)ctx->hev.size() < nev) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->hev.push_back(e);
    }
    cudaEvent_t *ev = ctx->hev.data();   // B chunks, A chunks, output chunks
    cudaEvent_t *evB = ev, *evA = evB + ncB, *evO = evA + ncA;
    cudaStream_t cs = ctx->up;
    if (relayout || moved) {                           // the workspace exists in stream order
        CK(cudaEventRecord(ctx->ws_ready, ctx->stream));
        CK(cudaStreamWaitEvent(cs, ctx->ws_ready, 0));
    }
    // the staging set's previous inputs have been transformed (the call two back)
    if (ctx->in_rec[sb]) CK(cudaStreamWaitEvent(cs, ctx->in_free[sb], 0));
    // uploads, then the forward transforms of each chunk once it has landed
    struct Up { const char *h; char *d; int rows, ncol; int64_t dl; char *T; size_t bT; cudaEvent_t *e; int nc; };
    const Up ups[2] = {{(const char *)B, Bd, n, k, dB, TB, bB, evB, ncB}, {(const char *)A, Ad, m, n, dA, TA, bA, evA, ncA}};
    for (const Up &u : ups)
        for (int c = 0; c < u.nc; c++) {
            int r0, r1;
            chunk_rows(u.rows, u.nc, c, r0, r1);
            const size_t o = (size_t)r0 * u.ncol * u.dl * w, sz = (size_t)(r1 - r0) * u.ncol * u.dl * w;
            CK(cudaMemcpyAsync(u.d + o, u.h + o, sz, cudaMemcpyHostToDevice, cs));
            CK(cudaEventRecord(u.e[c], cs));
        }
    if (!chunked) {                                    // small operands: one launch for both
        for (const Up &u : ups) {
            CK(cudaStreamWaitEvent(ctx->stream, u.e[0], 0));
            CKI(debug_check(ctx, u.d, (int64_t)u.rows * u.ncol * u.dl, w, p));
        }
        int tok = stage_begin(ctx, PM_STAGE_FWD);
        std::vector<FwdJob> blk; std::vector<int> bn;
        std::vector<ColJob> col; std::vector<int> cn;
        for (const Up &u : ups) {
            const size_t g0 = blk.size();
            for (size_t i = 0; i < K; i++)
                add_forward(prime_dev(*pr[i], lg), u.d, w, u.dl, u.dl, u.rows * u.ncol, (u32 *)(u.T + i * u.bT), lg,
                            blk, bn, col, cn);
            group_forward(blk, g0, lg);
        }
        CKI(launch_fwd_lists(ctx, blk, bn, col, cn, lg));
        stage_end(ctx, tok);
    }
    for (const Up &u : ups)
        for (int c = 0; chunked && c < u.nc; c++) {
            int r0, r1;
            chunk_rows(u.rows, u.nc, c, r0, r1);
            CK(cudaStreamWaitEvent(ctx->stream, u.e[c], 0));
            CKI(debug_check(ctx, u.d + (size_t)r0 * u.ncol * u.dl * w, (int64_t)(r1 - r0) * u.ncol * u.dl, w, p));
            int tok = stage_begin(ctx, PM_STAGE_FWD);
            std::vector<FwdJob> blk; std::vector<int> bn;
            std::vector<ColJob> col; std::vector<int> cn;
            for (size_t i = 0; i < K; i++)
                add_forward(prime_dev(*pr[i], lg), u.d + (size_t)r0 * u.ncol * u.dl * w, w, u.dl, u.dl,
                            (r1 - r0) * u.ncol, (u32 *)(u.T + i * u.bT) + (size_t)r0 * u.ncol * L, lg, blk, bn, col,
                            cn);
            group_forward(blk, 0, lg);
            CKI(launch_fwd_lists(ctx, blk, bn, col, cn, lg));
            stage_end(ctx, tok);
        }
    CK(cudaEventRecord(ctx->in_free[sb], ctx->stream));   // this staging set's inputs are consumed
    ctx->in_rec[sb] = true;
    int tok = stage_begin(ctx, PM_STAGE_POINTWISE);
    {
        PwLists pl;
        for (size_t i = 0; i < K; i++)
            add_pointwise(ctx, pl, (u32 *)(TA + i * bA), (u32 *)(TB + i * bB), (u32 *)(TC + i * bC), m, n, k, lg,
                          prime_dev(*pr[i], lg));
        CKI(launch_pointwise_lists(ctx, pl));
    }
    stage_end(ctx, tok);
    // the staging set's previous outputs have been downloaded (the call two back)
    if (ctx->out_rec[sb]) CK(cudaStreamWaitEvent(ctx->stream, ctx->out_free[sb], 0));
    // output entries [e0, e1) per chunk: inverse transforms, CRT (residue planes of the chunk
    // packed: K planes of (e1 - e0) * len words), copy back
    for (int c = 0; c < ncO; c++) {
        const int64_t e0 = (int64_t)eC * c / ncO, e1 = (int64_t)eC * (c + 1) / ncO, ce = e1 - e0;
        char *Rc = R + K * (size_t)e0 * len * 4;
        char *Cc = Cd + (size_t)e0 * len * w;
        tok = stage_begin(ctx, PM_STAGE_INV);
        {
            InvLists il;
            for (size_t i = 0; i < K; i++)
                add_inverse(il, prime_dev(*pr[i], lg), (u32 *)(TC + i * bC) + (size_t)e0 * L,
                            direct ? (void *)Cc : (void *)(Rc + i * (size_t)ce * len * 4), len, direct ? w : 1, 0, len,
                            ce, lg);
            CKI(launch_inverse_lists(ctx, il, lg));
        }
        stage_end(ctx, tok);
        if (!direct) {
            tok = stage_begin(ctx, PM_STAGE_CRT);
            CrtJob j;
            memset(&j, 0, sizeof(j));
            fill_crt(j, pr, p);
            j.res = (const u32 *)Rc; j.dst = Cc; j.count = ce * len; j.len = len; j.dst_stride = len; j.w = w;
            std::vector<CrtJob> jobs(1, j);
            std::vector<int> nb(1, crt_blocks(j));
            CKI(launch_packs(ctx, jobs, nb, [&](const JobPack<CrtJob> &pk) {
                return launch_crt(pk, ctx->stream, &ctx->launches); }));
            stage_end(ctx, tok);
        }
        CK(cudaEventRecord(evO[c], ctx->stream));
        CK(cudaStreamWaitEvent(ctx->dn, evO[c], 0));
        CK(cudaMemcpyAsync((char *)C + (size_t)e0 * len * w, Cc, (size_t)ce * len * w, cudaMemcpyDeviceToHost,
                           ctx->dn));
    }
    CK(cudaEventRecord(ctx->out_free[sb], ctx->dn));
    ctx->out_rec[sb] = true;
    ctx->host_pending = true;     // joined by host_join: the next device product, pm_sync, pm_host_join
    return PM_OK;
}

int pmat_mul(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA, const void *B,
             int64_t dB, void *C)
{
    CKI(check_common(ctx, p, w, m, n, k, A, dA, B, dB, C));
    const int64_t len = dA + dB - 1;
    const int lg = ceil_log2(len);
    if (lg > PM_MAX_LOG2L) return pm_fail(ctx, PM_EINVAL, "product longer than 2^20");
    bool done = false;
    CKI(small_product(ctx, p, w, m, n, k, A, dA, B, dB, C, len, lg, done));
    if (done) return PM_OK;
    return prod_slice(ctx, p, w, m, n, k, A, dA, dA, B, dB, dB, 0, len, lg, C, len);
}

int pm_host_join(pm_ctx *ctx)
{
    if (!ctx) return PM_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    return host_join(ctx);
}

int pmat_mul_host(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA, const void *B,
                  int64_t dB, void *C)
{
    CKI(check_common(ctx, p, w, m, n, k, A, dA, B, dB, C, false));
    return mul_host(ctx, p, w, m, n, k, A, dA, B, dB, C);
}

int pmat_mul_trunc(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA, const void *B,
                   int64_t dB, int64_t t, void *C)
{
    CKI(check_common(ctx, p, w, m, n, k, A, dA, B, dB, C));
    if (t < 1) return pm_fail(ctx, PM_EINVAL, "t must be >= 1");
    const int64_t a = dA < t ? dA : t, b = dB < t ? dB : t;
    const int lg = ceil_log2(a + b - 1);
    if (lg > PM_MAX_LOG2L) return pm_fail(ctx, PM_EINVAL, "product longer than 2^20");
    return prod_slice(ctx, p, w, m, n, k, A, a, dA, B, b, dB, 0, t, lg, C, t);
}

int pmat_middle_product(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, const void *A, int64_t dA,
                        const void *B, int64_t dB, int64_t c, int64_t d, void *C)
{
    CKI(check_common(ctx, p, w, m, n, k, A, dA, B, dB, C));
    if (c < 0 || d < 1) return pm_fail(ctx, PM_EINVAL, "need c >= 0, d >= 1");
    if (dA > c + 1) return pm_fail(ctx, PM_EINVAL, "middle product needs dA <= c + 1");
    if (dB > c + d) return pm_fail(ctx, PM_EINVAL, "middle product needs dB <= c + d");
    const int lg = ceil_log2(c + d);
    if (lg > PM_MAX_LOG2L) return pm_fail(ctx, PM_EINVAL, "product longer than 2^20");
    return prod_slice(ctx, p, w, m, n, k, A, dA, dA, B, dB, dB, c, d, lg, C, d);
}

}  // extern "C"
