// primes.cu -- host set-up of the NTT primes, shared by the context's product path, the
// allocation-free entry point and the CRT constants.
//
// The CRT primes are q = c 2^20 + 1 < 2^30 (Sec. 2, "3-primes multiplication": the product is
// lifted to Z[x] and computed modulo primes with 2^20-th roots of unity).  Primality is
// decided by deterministic Miller-Rabin (bases 2, 7 and 61 are enough below 4.76e9, Jaeschke
// 1993), a generator of F_q^* by trial factorisation of q - 1, and the 2^l-th roots as
// g^((q-1)/2^l).
#include <vector>

#include "common.cuh"

uint64_t host_mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((unsigned __int128)a * b % p); }

uint64_t host_powmod(uint64_t a, uint64_t e, uint64_t p)
{
    uint64_t r = 1 % p;
    for (a %= p; e; e >>= 1, a = host_mulmod(a, a, p))
        if (e & 1) r = host_mulmod(r, a, p);
    return r;
}

bool ntt_is_prime32(uint64_t n)
{
    if (n < 2 || n >= (1ull << 32)) return false;
    for (uint64_t s : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 61ull})
        if (n % s == 0) return n == s;
    uint64_t d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; r++; }
    for (uint64_t a : {2ull, 7ull, 61ull}) {
        uint64_t x = host_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r && comp; i++) {
            x = host_mulmod(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

void ntt_roots(uint32_t q, uint32_t *rf, uint32_t *ri)
{
    std::vector<uint64_t> f;                   // prime factors of q - 1
    uint64_t m = q - 1;
    for (uint64_t d = 2; d * d <= m; d++)
        if (m % d == 0) {
            f.push_back(d);
            while (m % d == 0) m /= d;
        }
    if (m > 1) f.push_back(m);
    uint64_t g = 2;
    for (;; g++) {
        bool ok = true;
        for (uint64_t d : f)
            if (host_powmod(g, (q - 1) / d, q) == 1) { ok = false; break; }
        if (ok) break;
    }
    for (int l = 0; l <= PM_MAX_LOG2L; l++) {
        if (((uint64_t)(q - 1) % (1ull << l)) != 0) { rf[l] = ri[l] = 0; continue; }
        const uint64_t w = host_powmod(g, (q - 1) >> l, q);
        rf[l] = (uint32_t)w;
        ri[l] = (uint32_t)host_powmod(w, q - 2, q);
    }
}

int ntt_prime_table(uint32_t *out, int maxk)
{
    int K = 0;
    for (uint64_t c = 1023; c >= 512 && K < maxk; c--)
        if (ntt_is_prime32((c << 20) + 1)) out[K++] = (uint32_t)((c << 20) + 1);
    return K;
}
