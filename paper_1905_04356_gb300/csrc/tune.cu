// tune.cu -- the autotuner: measured choice of the pointwise form and block tile of a product
// shape, and of PM-Basis's threshold T.
//
// Products (Sec. 2, "Polynomial matrix multiplication"): the pointwise stage (the n^omega d
// term) has several forms -- the CUDA-core kernel with a block tile (bi, bk) of 4 x 8 thread
// tiles, a streaming kernel for n <= 8, a matrix-vector kernel for k = 1, and the tensor-core
// digit form for m, n, k <= 32 -- and the cost model that picks a tile by default is an
// estimate.  pm_tune_product times every form that applies (the CUDA-core one with its best
// tiles by the cost model) on the product's own shape and records the fastest per (m, n, k,
// transform length); later products of that shape in the automatic mode take it.
//
// PM-Basis (Sec. 3, Algorithm 3): leaves of order <= T run M-Basis, larger orders recurse on
// two halves with products in between; T trades the leaf chain's cost per order step against
// the products' cost.  pm_tune_basis times pm_basis on seeded pseudo-random input for a set of
// thresholds and keeps the fastest in the context.
#include <cstring>
#include <vector>

#include "host.h"


namespace {

// x[i] = splitmix64(seed + i) mod p, the seeded input of the threshold timing
__global__ void k_tune_fill(uint64_t *x, int64_t count, uint64_t p, uint64_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = z % p;
    }
}

struct Cand { int form, bi, bk; };

}  // namespace

extern "C" {

int pm_tune_product(pm_ctx *ctx, uint64_t p, int w, int m, int n, int k, int64_t dA, int64_t dB, int reps,
                    int64_t *out)
{
    if (!ctx || !out) return PM_EINVAL;
    if (m < 1 || n < 1 || k < 1 || dA < 1 || dB < 1 || reps < 1 || reps > 1000 || (w != 4 && w != 8) || p < 2 ||
        (w == 4 && p > (1ull << 32)) || p >= (1ull << 62) || dA > (1 << PM_MAX_LOG2L) || dB > (1 << PM_MAX_LOG2L))
        return pm_fail(ctx, PM_EINVAL, "pm_tune_product: bad arguments");
    const int64_t len = dA + dB - 1;
    const int lg0 = ceil_log2(len), lg = lg0 < 4 ? 4 : lg0;
    if (lg > PM_MAX_LOG2L) return pm_fail(ctx, PM_EINVAL, "pm_tune_product: product longer than 2^20");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    // candidate forms for this shape
    PwJob j;
    memset(&j, 0, sizeof(j));
    j.m = m; j.n = n; j.k = k; j.L = 1 << lg;
    std::vector<Cand> cands;
    int tbi[4], tbk[4];
    const int nt = pw_tiles(j, tbi, tbk, 4, 8);
    for (int t = 0; t < nt; t++) cands.push_back({1, tbi[t], tbk[t]});
    const int nt4 = pw_tiles(j, tbi, tbk, 4, 4);
    for (int t = 0; t < nt4; t++) cands.push_back({6, tbi[t], tbk[t]});
    if (tc_supported(j)) cands.push_back({2, 0, 0});
    if (pws_supported(j)) cands.push_back({3, 0, 0});
    if (pwv_supported(j)) cands.push_back({4, 0, 0});
    if (m >= 64) cands.push_back({5, 0, 0});
    // zero inputs (the kernels' time does not depend on the values) and the output
    const size_t bA = (size_t)m * n * dA * w, bB = (size_t)n * k * dB * w, bC = (size_t)m * k * len * w;
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, bA + bB + bC + 512, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return pm_fail(ctx, PM_ENOMEM, "pm_tune_product: scratch allocation failed");
    }
    char *A = buf, *B = buf + ((bA + 255) & ~size_t(255)), *C = B + ((bB + 255) & ~size_t(255));
    int rc = pm_cuda(ctx, cudaMemsetAsync(buf, 0, bA + bB + 512, ctx->stream), "cudaMemsetAsync");
    const int timing = ctx->opt_timing;
    double best_ms = -1;
    Cand best{0, 0, 0};
    if (!rc) {
        ctx->opt_timing = 1;
        rc = pm_stage_times(ctx, nullptr, nullptr);                  // earlier records dropped
        for (size_t c = 0; !rc && c < cands.size(); c++) {
            ctx->force_form = cands[c].form;
            ctx->force_bi = cands[c].bi;
            ctx->force_bk = cands[c].bk;
            rc = prod_slice(ctx, p, w, m, n, k, A, dA, dA, B, dB, dB, 0, len, lg, C, len);   // warm-up
            if (!rc) rc = pm_stage_times(ctx, nullptr, nullptr);
            for (int r = 0; !rc && r < reps; r++) rc = prod_slice(ctx, p, w, m, n, k, A, dA, dA, B, dB, dB, 0, len, lg, C, len);
            double ms[PM_NSTAGES];
            if (!rc) rc = pm_stage_times(ctx, ms, nullptr);
            if (!rc && (best_ms < 0 || ms[PM_STAGE_POINTWISE] < best_ms)) {
                best_ms = ms[PM_STAGE_POINTWISE];
                best = cands[c];
            }
        }
        ctx->force_form = -1;
        ctx->opt_timing = timing;
    }
    cudaFreeAsync(buf, ctx->stream);
    if (rc) return rc;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "stream synchronisation failed");
    bool found = false;
    for (auto &t : ctx->tune)
        if (t.m == m && t.n == n && t.k == k && t.lg == lg) { t.form = best.form; t.bi = best.bi; t.bk = best.bk; found = true; }
    if (!found) ctx->tune.push_back({m, n, k, lg, best.form, best.bi, best.bk});
    out[0] = best.form;
    out[1] = best.bi;
    out[2] = best.bk;
    out[3] = (int64_t)(best_ms / reps * 1e6);
    out[4] = (int64_t)cands.size();
    return PM_OK;
}

int pm_tune_basis(pm_ctx *ctx, uint64_t p, int m, int n, int64_t d, int reps, int64_t *out)
{
    if (!ctx || !out) return PM_EINVAL;
    if (m < 1 || n < 1 || d < 1 || reps < 1 || reps > 100 || p < 3 || !(p & 1) || p >= (1ull << 62))
        return pm_fail(ctx, PM_EINVAL, "pm_tune_basis: bad arguments");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    const size_t bF = (size_t)m * n * d * 8, bP = (size_t)m * m * (d + 1) * 8;
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, bF + bP + 256, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return pm_fail(ctx, PM_ENOMEM, "pm_tune_basis: scratch allocation failed");
    }
    uint64_t *F = (uint64_t *)buf, *P = (uint64_t *)(buf + ((bF + 255) & ~size_t(255)));
    k_tune_fill<<<256, 256, 0, ctx->stream>>>(F, (int64_t)m * n * d, p, 0x243F6A8885A308D3ull);
    ctx->launches++;
    int rc = pm_cuda(ctx, cudaGetLastError(), "k_tune_fill");
    std::vector<int64_t> shift(m, 0), rdeg(m, 0);
    const int64_t T0 = ctx->opt_T;
    int64_t bestT = T0;
    double best_ms = -1;
    cudaEvent_t a = nullptr, b = nullptr;
    if (!rc) rc = pm_cuda(ctx, cudaEventCreate(&a), "cudaEventCreate");
    if (!rc) rc = pm_cuda(ctx, cudaEventCreate(&b), "cudaEventCreate");
    for (int64_t T : {8, 16, 32, 64, 128}) {
        if (rc || (T > d && T != 8)) continue;
        ctx->opt_T = T;
        rc = pm_basis(ctx, p, m, n, F, d, d, shift.data(), P, rdeg.data());     // warm-up
        if (!rc) rc = pm_cuda(ctx, cudaEventRecord(a, ctx->stream), "cudaEventRecord");
        for (int r = 0; !rc && r < reps; r++) rc = pm_basis(ctx, p, m, n, F, d, d, shift.data(), P, rdeg.data());
        if (!rc) rc = pm_cuda(ctx, cudaEventRecord(b, ctx->stream), "cudaEventRecord");
        if (!rc) rc = pm_cuda(ctx, cudaEventSynchronize(b), "cudaEventSynchronize");
        float ms = 0;
        if (!rc) rc = pm_cuda(ctx, cudaEventElapsedTime(&ms, a, b), "cudaEventElapsedTime");
        if (!rc && (best_ms < 0 || ms < best_ms)) { best_ms = ms; bestT = T; }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFreeAsync(buf, ctx->stream);
    ctx->opt_T = rc ? T0 : bestT;
    if (rc) return rc;
    out[0] = bestT;
    out[1] = (int64_t)(best_ms / reps * 1e6);
    return PM_OK;
}

}  // extern "C"
