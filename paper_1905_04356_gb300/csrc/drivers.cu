// drivers.cu -- entry points built on the product core: batched products,
// PM-Basis (Algorithm 3) and the bivariate resultant (Sec. 5.2).
#include <cstring>

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
    for (int i = 0; i < count; i++) {
        const pmat_desc &x = d[i];
        const int64_t len = x.dA + x.dB - 1;
        CKI(prod_slice(ctx, x.p, x.w, x.m, x.n, x.k, x.A, x.dA, x.dA, x.B, x.dB, x.dB, 0, len, ceil_log2(len), x.C,
                       len));
    }
    return PM_OK;
}

int bivariate_resultant(pm_ctx *ctx, int nprimes, const uint64_t *primes, int dxf, int dyf, const void *f, int dxg,
                        int dyg, const void *g, void *R)
{
    (void)nprimes; (void)primes; (void)dxf; (void)dyf; (void)f; (void)dxg; (void)dyg; (void)g; (void)R;
    if (!ctx) return PM_EINVAL;
    return pm_fail(ctx, PM_EUNSUPPORTED, "bivariate_resultant not built yet");
}

}  // extern "C"
