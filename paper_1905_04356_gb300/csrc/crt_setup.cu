// crt_setup.cu -- host set-up of the multi-prime CRT constants (Sec. 2, "3-primes
// multiplication": the product lifted to Z[x] and computed modulo K NTT primes), shared by
// the context's product path and the allocation-free entry point.  The kernel that uses them
// (k_crt) and the arithmetic they serve are described in pointwise.cu.
#include "common.cuh"

// Host set-up of the constants of a CRT job over the primes q[0 .. K-1] (every one above 2^29)
// for values mod p: Garner's tables always, the explicit sum's for odd p and K >= 2.
void crt_setup(CrtJob &J, const u32 *q, int K, uint64_t p)
{
    J.K = K;
    J.p = p;
    J.mu = (uint64_t)(((unsigned __int128)1 << 64) / p);
    J.small_p = p <= (1ull << 30);
    for (int i = 0; i < K; i++) {
        const uint64_t qi = q[i];
        J.q[i] = (u32)qi;
        for (int j = 0; j < i; j++) {
            const uint64_t c = host_powmod(q[j] % qi, qi - 2, qi);
            J.c[i][j] = (u32)c;
            J.cs[i][j] = (u32)((c << 32) / qi);
        }
        J.qm[i] = qi % p;
        J.qms[i] = (uint64_t)(((unsigned __int128)J.qm[i] << 64) / p);
    }
    J.mode = (p & 1) && K >= 2 ? 1 : 0;                 // Montgomery reduction needs p odd
    if (!J.mode) return;
    const uint64_t r64 = (uint64_t)(((unsigned __int128)1 << 64) % p);   // 2^64 mod p
    uint64_t Mp = 1 % p;
    for (int i = 0; i < K; i++) {
        const uint64_t qi = q[i];
        uint64_t mi_q = 1, mi_p = 1 % p;
        for (int j = 0; j < K; j++)
            if (j != i) {
                mi_q = host_mulmod(mi_q, q[j] % qi, qi);
                mi_p = host_mulmod(mi_p, q[j] % p, p);
            }
        const uint64_t g = host_powmod(mi_q, qi - 2, qi);
        J.gi[i] = (u32)g;
        J.gis[i] = (u32)((g << 32) / qi);
        J.W[i] = (u32)((1ull << 59) / qi);
        J.Cm[i] = host_mulmod(mi_p, r64, p);
        Mp = host_mulmod(Mp, qi % p, p);
    }
    J.Cm[K] = host_mulmod((p - Mp) % p, r64, p);
    uint64_t inv = 1;                                   // p^-1 mod 2^64 by Newton iteration
    for (int it = 0; it < 7; it++) inv *= 2 - p * inv;
    J.pn = (uint64_t)0 - inv;
}
