// drivers.cu -- pmat_mul_batched: many independent products through one
// planned batch (jobs binned by transform length into shared launches).
#include <cstring>
#include <vector>

#include "host.h"

#define CKI(call)                                                       \
    do {                                                                \
        int _rc = (call);                                               \
        if (_rc) return _rc;                                            \
    } while (0)

extern "C" {

int pmat_mul_batched(pm_ctx *ctx, int count, const pmat_desc *d)
{
    if (!ctx) return PM_EINVAL;
    if (count < 0 || (count > 0 && !d)) return pm_fail(ctx, PM_EINVAL, "bad descriptor array");
    for (int i = 0; i < count; i++) {
        const pmat_desc &x = d[i];
        if (x.m < 1 || x.n < 1 || x.k < 1 || x.dA < 1 || x.dB < 1 || x.p < 2 || (x.w != 4 && x.w != 8) ||
            (x.w == 4 && x.p > (1ull << 32)) || x.p >= (1ull << 62) || !x.A || !x.B || !x.C ||
            ceil_log2(x.dA + x.dB - 1) > PM_MAX_LOG2L)
            return pm_fail(ctx, PM_EINVAL, "bad descriptor " + std::to_string(i));
    }
    std::vector<ProdReq> reqs(count);
    for (int i = 0; i < count; i++) {
        const pmat_desc &x = d[i];
        ProdReq &q = reqs[i];
        q.p = x.p; q.w = x.w; q.m = x.m; q.n = x.n; q.k = x.k;
        q.A = x.A; q.B = x.B; q.C = x.C;
        q.dA = x.dA; q.sA = x.dA; q.dB = x.dB; q.sB = x.dB;
        q.off = 0; q.len = x.dA + x.dB - 1; q.sC = q.len;
        const int lg = ceil_log2(q.len);
        q.lg = lg < 4 ? 4 : lg;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pm_fail(ctx, PM_ECUDA, "cudaSetDevice failed");
    return prod_batch(ctx, reqs.data(), count);
}

}  // extern "C"
