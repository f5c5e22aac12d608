// solve.cu -- linear system solving by lifting (Sec. 4, "Linear system solving"): the pair
// (u, f) with A u = f b and f of minimal degree, for A square with A(0) invertible.
//
//  1. v = A^-1 b mod x^N by the truncated inverse and Dixon's lifting (pmat_solve_series).
//  2. Vector rational reconstruction: an approximant basis of the (n+1) x n matrix
//     F = [v^T; -I] at order N (pm_basis).  With D1 = n (dA - 1) >= deg f and
//     D2 = (n - 1)(dA - 1) + db - 1 >= deg u (Cramer's rule), N = D1 + D2 + 1 and the shift
//     (-D1, -D2, ..., -D2), the basis has exactly one row of non-positive shifted degree,
//     [f, u^T] up to a constant: two solutions within the degree bounds give
//     g u - f w = 0 mod x^N with deg < N, so they are proportional.
//  3. That row is picked from the returned shifted row degrees and normalised on the device
//     so that f is monic.
#include <vector>

#include "host.h"

namespace {

struct SolveK {
    u64 p, pn, one, r2;     // Montgomery constants (R = 2^64)
};

__device__ u64 s_pow(u64 a, u64 e, const SolveK &K)
{
    u64 r = K.one;
    while (e) {
        if (e & 1) r = mont_mul(r, a, K.p, K.pn);
        a = mont_mul(a, a, K.p, K.pn);
        e >>= 1;
    }
    return r;
}

// F[(1 + i) n + i][0] = p - 1: the -I block below the series row.
__global__ void k_minus_identity(u64 *F, int n, int64_t N, u64 pm1)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        F[((int64_t)(1 + i) * n + i) * N] = pm1;
}

// One block: deg f (largest nonzero index of f = P[row][0]) and the Montgomery form of
// lc(f)^-1 into sc[0]; deg[0] = deg f (-1 when f = 0), deg[1] reset for the next kernel.
__global__ void __launch_bounds__(1024) k_solve_lead(const u64 *f, int64_t D1, SolveK K, u64 *sc, int64_t *deg)
{
    __shared__ int64_t dmax;
    if (threadIdx.x == 0) dmax = -1;
    __syncthreads();
    int64_t loc = -1;
    for (int64_t i = threadIdx.x; i <= D1; i += blockDim.x)
        if (f[i]) loc = i;
    if (loc >= 0) atomicMax((long long *)&dmax, (long long)loc);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t d = dmax;
        deg[0] = d;
        deg[1] = -1;
        sc[0] = d >= 0 ? s_pow(mont_mul(f[d], K.r2, K.p, K.pn), K.p - 2, K) : 0;
    }
}

// f_out[i] = f[i] / lc (i <= D1), u_out[j][i] = u_j[i] / lc (i <= D2); deg[1] = max deg u_j.
__global__ void k_solve_scale(const u64 *P, int64_t row0, int64_t sP, int n, int64_t D1, int64_t D2, SolveK K,
                              const u64 *sc, u64 *f_out, u64 *u_out, int64_t *deg)
{
    const u64 c = sc[0];
    const int64_t nf = D1 + 1, nu = (int64_t)n * (D2 + 1);
    int64_t dloc = -1;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nf + nu; x += (int64_t)gridDim.x * blockDim.x) {
        if (x < nf) {
            f_out[x] = mont_mul(P[row0 + x], c, K.p, K.pn);
        } else {
            const int64_t y = x - nf, j = y / (D2 + 1), i = y % (D2 + 1);
            const u64 v = P[row0 + (1 + j) * sP + i];
            u_out[y] = mont_mul(v, c, K.p, K.pn);
            if (v && i > dloc) dloc = i;
        }
    }
    if (dloc >= 0) atomicMax((long long *)&deg[1], (long long)dloc);
}

int grid_for(int64_t total)
{
    const int64_t b = (total + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

}  // namespace

extern "C" int pmat_solve(pm_ctx *ctx, uint64_t p, int n, const void *A, int64_t dA, const void *b, int64_t db,
                          void *u, void *f, int64_t *deg_out)
{
    if (!ctx) return PM_EINVAL;
    if (n < 1 || n > 127) return pm_fail(ctx, PM_EINVAL, "pmat_solve needs 1 <= n <= 127");
    if (dA < 1 || db < 1) return pm_fail(ctx, PM_EINVAL, "lengths must be >= 1");
    if (p < 3 || !(p & 1) || p >= (1ull << 62)) return pm_fail(ctx, PM_EINVAL, "pmat_solve needs an odd prime p < 2^62");
    if (!A || !b || !u || !f || !deg_out) return pm_fail(ctx, PM_EINVAL, "null buffer");
    const int64_t D1 = (int64_t)n * (dA - 1), D2 = (int64_t)(n - 1) * (dA - 1) + db - 1, N = D1 + D2 + 1;
    if (N > (int64_t(1) << 19)) return pm_fail(ctx, PM_EINVAL, "system too large: the series order exceeds 2^19");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    SolveK K;
    K.p = p;
    uint64_t inv = 1;                       // p^-1 mod 2^64 by Newton iteration
    for (int i = 0; i < 7; i++) inv *= 2 - p * inv;
    K.pn = (uint64_t)0 - inv;
    K.one = (uint64_t)(((unsigned __int128)1 << 64) % p);
    K.r2 = (uint64_t)((unsigned __int128)K.one * K.one % p);

    const int m = n + 1;
    const size_t bv = (size_t)n * N * 8, bF = (size_t)m * n * N * 8, bP = (size_t)m * m * (N + 1) * 8;
    char *buf = nullptr;
    const size_t total = bv + bF + bP + 256;
    if (cudaMallocAsync((void **)&buf, total, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return pm_fail(ctx, PM_ENOMEM, "pmat_solve workspace allocation failed");
    }
    u64 *v = (u64 *)buf, *F = (u64 *)(buf + bv), *P = (u64 *)(buf + bv + bF);
    u64 *sc = (u64 *)(buf + bv + bF + bP);
    int64_t *deg = (int64_t *)(sc + 2);
    int rc = PM_OK;
    do {
        // 1. v = A^-1 b mod x^N
        if ((rc = pmat_solve_series(ctx, p, 8, n, A, dA, b, db, N, v))) break;
        // 2. F = [v^T; -I], approximant basis at order N for the shift (-D1, -D2, ..., -D2)
        if ((rc = pm_cuda(ctx, cudaMemsetAsync(F, 0, bF, ctx->stream), "clear F"))) break;
        if ((rc = pm_cuda(ctx, cudaMemcpyAsync(F, v, bv, cudaMemcpyDeviceToDevice, ctx->stream), "copy v"))) break;
        k_minus_identity<<<1, 128, 0, ctx->stream>>>(F, n, N, p - 1);
        ctx->launches++;
        if ((rc = pm_cuda(ctx, cudaGetLastError(), "k_minus_identity"))) break;
        std::vector<int64_t> shift(m, -D2), rdeg(m, 0);
        shift[0] = -D1;
        if ((rc = pm_basis(ctx, p, m, n, F, N, N, shift.data(), P, rdeg.data()))) break;
        if ((rc = pm_sync(ctx))) break;    // A(0) singular is reported here (deferred status)
        // 3. the row of non-positive shifted degree, normalised to a monic f
        int r = 0;
        for (int i = 1; i < m; i++)
            if (rdeg[i] < rdeg[r]) r = i;
        if (rdeg[r] > 0) { rc = pm_fail(ctx, PM_EDOMAIN, "no solution within the degree bounds"); break; }
        const int64_t row0 = (int64_t)r * m * (N + 1);
        k_solve_lead<<<1, 1024, 0, ctx->stream>>>(P + row0, D1, K, sc, deg);
        k_solve_scale<<<grid_for(D1 + 1 + (int64_t)n * (D2 + 1)), 256, 0, ctx->stream>>>(
            P, row0, N + 1, n, D1, D2, K, sc, (u64 *)f, (u64 *)u, deg);
        ctx->launches += 2;
        if ((rc = pm_cuda(ctx, cudaGetLastError(), "k_solve_scale"))) break;
        if ((rc = pm_cuda(ctx, cudaMemcpyAsync(deg_out, deg, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream),
                          "degrees D2H")))
            break;
        if ((rc = pm_cuda(ctx, cudaStreamSynchronize(ctx->stream), "pmat_solve sync"))) break;
        if (deg_out[0] < 0) rc = pm_fail(ctx, PM_EDOMAIN, "reconstructed denominator is zero");
    } while (0);
    cudaFreeAsync(buf, ctx->stream);
    return rc;
}
