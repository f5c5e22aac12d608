// leaf_impl.cuh -- device side of PM-Basis / PM-IntBasis (Sec. 3, Algorithms 1-2 and 4 at
// the leaves of Algorithms 3 and 5): field arithmetic, Algorithm 1 with scaled rows, and the two
// leaf kernels.  pmbasis.cu includes this file three times, in namespaces that fix LEAF_F2:
// false (odd p, Montgomery arithmetic), true (p = 2, bits) and the run-time test (p == 2) used
// by the node kernels, so that the leaves carry no test of the modulus.
// ------------------------------------------------------------------ device arithmetic
// Field arithmetic: Montgomery products (R = 2^64) for odd p.  For p = 2 the elements are bits
// and the "Montgomery form" is the identity (one = r2 = 1): a product is an AND, a x - b y
// (- c z) an XOR, and the reduction of an integer sum its parity.  LEAF_F2 selects the form:
// a constant in the leaf instantiations, the test p == 2 in the node kernels'.
__device__ __forceinline__ u64 fm_mul(u64 a, u64 b, u64 p, u64 pn) { return LEAF_F2 ? (a & b) : mont_mul(a, b, p, pn); }
__device__ __forceinline__ u64 fm_msub(u64 a, u64 x, u64 b, u64 y, u64 p, u64 pn)
{
    return LEAF_F2 ? ((a & x) ^ (b & y)) : mont_msub(a, x, b, y, p, pn);
}
__device__ __forceinline__ u64 fm_msub2(u64 a, u64 x, u64 b, u64 y, u64 c, u64 z, u64 p, u64 pn)
{
    return LEAF_F2 ? ((a & x) ^ (b & y) ^ (c & z)) : mont_msub2(a, x, b, y, c, z, p, pn);
}
__device__ __forceinline__ u64 fm_redc(u64 hi, u64 lo, u64 p, u64 pn) { return LEAF_F2 ? (lo & 1) : redc128(hi, lo, p, pn); }
__device__ __forceinline__ void mac128(u64 &hi, u64 &lo, u64 a, u64 b)
{
    u64 l = a * b, h = __umul64hi(a, b);
    lo += l;
    hi += h + (lo < l);
}
__device__ __forceinline__ u64 mmul(u64 a, u64 b, const LeafArgs &A) { return fm_mul(a, b, A.p, A.pn); }
__device__ u64 mpow(u64 a, u64 e, const LeafArgs &A)
{
    u64 r = A.one;
    while (e) {
        if (e & 1) r = mmul(r, a, A);
        a = mmul(a, a, A);
        e >>= 1;
    }
    return r;
}

// ------------------------------------------------------------------ Algorithm 1 with scaled rows
// Shared-memory scratch of the elimination (all pointers into shared memory).
struct ElimSm {
    u64 *kap, *W, *M, *fac, *dpr, *bas, *tb, *vv, *tv;
    int *ord, *ind, *pcs, *misc, *perm;
    u64 *Wc;     // compact relation: Wc[j * n + b] = W[j][ilist[b]], b < nind
    int *ilist;  // independent rows, misc[4] = their count
    int *ipos;   // ipos[ilist[b]] = b
};

__device__ __forceinline__ size_t elim_words(int m, int n)
{
    const int mx = m > n ? m : n;
    return (size_t)m + (size_t)m * m + (size_t)n * m + mx + (n + 1) + (size_t)n * n + (size_t)n * m + n + m +
           (size_t)m * (mx);
}

__device__ __forceinline__ int elim_ints(int m, int n) { return 4 * m + 2 * n + 8; }

__device__ ElimSm elim_carve(u64 *w, int *ip, int m, int n)
{
    ElimSm E;
    const int mx = m > n ? m : n;
    E.kap = w; w += m;
    E.W = w; w += (size_t)m * m;
    E.M = w; w += (size_t)n * m;
    E.fac = w; w += mx;
    E.dpr = w; w += n + 1;
    E.bas = w; w += (size_t)n * n;
    E.tb = w; w += (size_t)n * m;
    E.vv = w; w += n;
    E.tv = w; w += m;
    E.Wc = w;
    E.ord = ip; ip += m;
    E.ind = ip; ip += m;
    E.pcs = ip; ip += n;
    E.perm = ip; ip += n;
    E.misc = ip; ip += 8;
    E.ilist = ip; ip += m;
    E.ipos = ip;
    return E;
}

// Fraction-free Gauss-Jordan of the n x m matrix M[c][col] = R[ord[col]][c] (n <= 64,
// m <= 128; the result is left in E.M) by the
// first GJ_WARPS warps of the block: lanes own columns, warps own rows (row c in
// warp c % GJ_WARPS), values stay in registers.  Pivot of column s: the lowest row
// not yet used with a nonzero entry.  One named barrier per pivot step: every warp
// publishes its candidate row (index and values) into a buffer alternating with the
// step's parity, then all warps read the winner's row.  Pivot step s updates every
// row c != r_s as row_c <- pv_s row_c - M[c][s] row_{r_s}, so the diagonal of row r_s
// ends as d_s = prod_{s' >= s} pv_s', the common multiple of the d_s is
// D = prod pv = d_0, and D / d_s = prod_{s' < s} pv_s' is recorded as E.fac[s]
// (E.dpr[n] = D).  Returns true (uniformly) when every column had a pivot; E.M then
// holds the result and E.perm[s] the pivot row of column s.
#define GJ_WARPS 8
#define GJ_CPL_MAX 4

template <int GJ_RPW, int GJ_CPL>
__device__ bool gj_regs(const LeafArgs &A, const u64 *R, ElimSm &E, int (*cand)[GJ_WARPS],
                        u64 (*crow)[GJ_WARPS][32 * GJ_CPL_MAX], int *failp, int gn)
{
    int &fail = *failp;
    const int m = A.m, n = A.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u64 p = A.p, pn = A.pn;
    const bool grp = warp < GJ_WARPS;
    u64 v[GJ_RPW][GJ_CPL];
    if (tid == 0) fail = 0;
    if (grp) {
#pragma unroll
        for (int i = 0; i < GJ_RPW; i++)
#pragma unroll
            for (int t = 0; t < GJ_CPL; t++) {
                const int c = warp + GJ_WARPS * i, col = lane + 32 * t;
                v[i][t] = (c < n && col < m) ? R[E.ord[col] * n + c] : 0;   // M[c][col] = R[ord[col]][c]
            }
        unsigned long long used = 0;
        u64 pre = A.one;                                // prod of the pivots so far (thread 0)
        int s = 0;
        for (; s < n; s++) {
            const int ls = s & 31, ts = s >> 5, bf = s & 1;
            // this warp's candidate: lowest unused own row with a nonzero entry in column s
            int mine = 0x7fffffff, slot = 0;
#pragma unroll
            for (int i = GJ_RPW - 1; i >= 0; i--) {
                const int c = warp + GJ_WARPS * i;
                u64 x = 0;
#pragma unroll
                for (int t = 0; t < GJ_CPL; t++) x = (t == ts) ? v[i][t] : x;
                if (c < n && !((used >> c) & 1ull) && x) { mine = c; slot = i; }
            }
            mine = __shfl_sync(0xffffffffu, mine, ls);
            slot = __shfl_sync(0xffffffffu, slot, ls);
            if (lane == 0) cand[bf][warp] = mine;
            if (mine != 0x7fffffff) {
#pragma unroll
                for (int t = 0; t < GJ_CPL; t++) {
                    u64 x = 0;
#pragma unroll
                    for (int i = 0; i < GJ_RPW; i++) x = (i == slot) ? v[i][t] : x;
                    crow[bf][warp][lane + 32 * t] = x;
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(GJ_WARPS * 32));
            int r = 0x7fffffff;
#pragma unroll
            for (int w = 0; w < GJ_WARPS; w++) r = min(r, cand[bf][w]);
            if (r == 0x7fffffff) break;                 // uniform over the group
            used |= 1ull << r;
            const u64 *prow = crow[bf][r % GJ_WARPS];
            const u64 pv = prow[s];
            if (tid == 0) {
                E.perm[s] = r;
                E.fac[s] = pre;
                pre = fm_mul(pre, pv, p, pn);
            }
#pragma unroll
            for (int i = 0; i < GJ_RPW; i++) {
                const int c = warp + GJ_WARPS * i;
                if (c >= n || c == r) continue;         // uniform within the warp
                u64 x = 0;
#pragma unroll
                for (int t = 0; t < GJ_CPL; t++) x = (t == ts) ? v[i][t] : x;
                const u64 f = __shfl_sync(0xffffffffu, x, ls);
#pragma unroll
                for (int t = 0; t < GJ_CPL; t++) v[i][t] = fm_msub(pv, v[i][t], f, prow[lane + 32 * t], p, pn);
            }
        }
        if (tid == 0) {
            if (s != n) fail = 1;
            E.dpr[n] = pre;
        }
#pragma unroll
        for (int i = 0; i < GJ_RPW; i++)
#pragma unroll
            for (int t = 0; t < GJ_CPL; t++) {
                const int c = warp + GJ_WARPS * i, col = lane + 32 * t;
                if (c < n && col < m) E.M[c * m + col] = v[i][t];
            }
    }
    asm volatile("bar.sync 2, %0;" ::"r"(gn));
    return fail == 0;
}

// The same elimination for 8 < n <= 16 and m <= 32 with the columns owned by lanes: warp w holds
// columns 4w .. 4w + 3, lane l row l % 16 of columns 4w + 2 (l / 16) and the next.  Pivot step
// s: the warp holding column s finds its lowest unused row with a nonzero entry by one ballot
// and publishes the column (the factors M[c][s] of the update) into a buffer alternating with
// the step's parity; after one named barrier every thread reads its factor and takes the
// pivot row's entries of its two columns from its own warp by shuffles, so no step waits on
// more than one exchange through shared memory (the row-owned layout of gj_regs needs a
// cross-warp search for the pivot row and a broadcast of the whole row).  The pivots are kept
// and turned into the prefix products E.fac after the loop.  Same pivots, same updates, same
// outputs as gj_regs.
__device__ bool gj_cols16(const LeafArgs &A, const u64 *R, ElimSm &E, int gn)
{
    __shared__ u64 fbuf[2][16];
    __shared__ int rbuf[2];
    __shared__ u64 pvs[16];
    __shared__ int fail;
    const int m = A.m, n = A.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u64 p = A.p, pn = A.pn;
    const int c = lane & 15, cp = lane >> 4, col0 = 4 * warp + 2 * cp;
    if (warp < GJ_WARPS) {
        u64 v0 = (c < n && col0 < m) ? R[E.ord[col0] * n + c] : 0;
        u64 v1 = (c < n && col0 + 1 < m) ? R[E.ord[col0 + 1] * n + c] : 0;
        unsigned used = 0;
        int s = 0;
        for (; s < n; s++) {
            const int bf = s & 1, oc = s & 1, ocp = (s >> 1) & 1;
            if (warp == (s >> 2)) {
                const u64 x = oc ? v1 : v0;
                const bool cand = cp == ocp && c < n && !((used >> c) & 1u) && x != 0;
                const unsigned bits = (__ballot_sync(0xffffffffu, cand) >> (16 * ocp)) & 0xFFFFu;
                if (cp == ocp) fbuf[bf][c] = x;
                if (lane == 0) rbuf[bf] = bits ? __ffs(bits) - 1 : -1;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(GJ_WARPS * 32));
            const int r = rbuf[bf];
            if (r < 0) break;                                // uniform over the group
            used |= 1u << r;
            const u64 fc = fbuf[bf][c], pv = fbuf[bf][r];
            const u64 q0 = __shfl_sync(0xffffffffu, v0, r + 16 * cp), q1 = __shfl_sync(0xffffffffu, v1, r + 16 * cp);
            if (c != r) {
                v0 = fm_msub(pv, v0, fc, q0, p, pn);
                v1 = fm_msub(pv, v1, fc, q1, p, pn);
            }
            if (tid == 0) { E.perm[s] = r; pvs[s] = pv; }
        }
        const bool ok = s == n;
        asm volatile("bar.sync 1, %0;" ::"r"(GJ_WARPS * 32));   // pvs complete
        if (ok) {
            if (warp == 0) {
                // E.fac[s] = prod_{s' < s} pv_s' (exclusive prefix products), E.dpr[n] = all of them
                u64 x = lane < n ? pvs[lane] : A.one;
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) {
                    const u64 y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x = fm_mul(x, y, p, pn);
                }
                const u64 ex = __shfl_up_sync(0xffffffffu, x, 1);
                if (lane < n) E.fac[lane] = lane ? ex : A.one;
                if (lane == n - 1) E.dpr[n] = x;
            }
            if (c < n && col0 < m) E.M[c * m + col0] = v0;
            if (c < n && col0 + 1 < m) E.M[c * m + col0 + 1] = v1;
        }
        if (tid == 0) fail = !ok;
    }
    asm volatile("bar.sync 2, %0;" ::"r"(gn));
    return fail == 0;
}

// Register tile: GJ_RPW rows per warp (n <= 8 GJ_RPW), GJ_CPL columns per lane (m <= 32 GJ_CPL).
// Called by the elimination group (warps 0 .. gn/32 - 1, gn >= GJ_WARPS * 32), which it
// leaves through named barrier 2.
__device__ bool gj_dispatch(const LeafArgs &A, const u64 *R, ElimSm &E, int gn)
{
    __shared__ int cand[2][GJ_WARPS];
    __shared__ u64 crow[2][GJ_WARPS][32 * GJ_CPL_MAX];
    __shared__ int fail;
    const int rpw = (A.n + GJ_WARPS - 1) / GJ_WARPS, cpl = (A.m + 31) / 32;
    if (gn < GJ_WARPS * 32) return false;          // the named barrier needs GJ_WARPS full warps
    // the column-owned form for 8 < n <= 16 (measured: 32 x 16 bases 15.5 -> 14.1 us per order
    // step); for n <= 8 the row-owned form holds one row per warp, one update per thread and
    // pivot, and is faster (the Villard variant's 16 x 8 bases: 93 against 76 ms of leaves)
    if (A.n > 8 && A.n <= 16 && A.m <= 32) return gj_cols16(A, R, E, gn);
    if (cpl == 1) {
        if (rpw <= 1) return gj_regs<1, 1>(A, R, E, cand, crow, &fail, gn);
        if (rpw <= 2) return gj_regs<2, 1>(A, R, E, cand, crow, &fail, gn);
        if (rpw <= 4) return gj_regs<4, 1>(A, R, E, cand, crow, &fail, gn);
    } else if (cpl == 2) {
        if (rpw <= 2) return gj_regs<2, 2>(A, R, E, cand, crow, &fail, gn);
        if (rpw <= 4) return gj_regs<4, 2>(A, R, E, cand, crow, &fail, gn);
        if (rpw <= 8) return gj_regs<8, 2>(A, R, E, cand, crow, &fail, gn);
    } else if (cpl <= 4) {
        if (rpw <= 4) return gj_regs<4, 4>(A, R, E, cand, crow, &fail, gn);
        if (rpw <= 8) return gj_regs<8, 4>(A, R, E, cand, crow, &fail, gn);
    }
    return false;   // shapes beyond the register tile take the row-order elimination
}

// Algorithm 1 on the residual R (m x n, Montgomery) with shift t: rows visited in
// increasing (t_i, i) order (rows with a zero residual may be moved last: same output).  Output: ind[i] = 1 for rows that become x e_i; for the
// other rows j, the scaled relation kap_j R_j = -sum_i W[j][i] R_i (W stored
// negated), i.e. the row of Q is kap_j e_j + sum_i W[j][i] e_i.  Called by the
// elimination group: warps 0 .. gn/32 - 1 of the block (tid < gn, gn a multiple of 32
// and >= 256), synchronised by named barrier 2, with which it ends.
#define EBAR() asm volatile("bar.sync 2, %0;" ::"r"(nth))
// Fast path of Algorithm 1: Gauss-Jordan on [R_I^T | R_D^T] (n x m), I = the first n rows of
// E.ord; false (nothing written but scratch) when those rows are dependent.
__device__ __forceinline__ bool mbasis1_fast(const LeafArgs &A, const u64 *R, ElimSm &E, int nth)
{
    const int m = A.m, n = A.n, tid = threadIdx.x;
    const u64 p = A.p;
    // the independent rows are known before the elimination: list them in index order
    for (int pos = tid; pos < m; pos += nth) E.ind[E.ord[pos]] = pos < n;
    EBAR();
    if (tid < 32) {
        int base = 0;
        for (int i0 = 0; i0 < m; i0 += 32) {
            const int i = i0 + tid;
            const bool f = i < m && E.ind[i];
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (f) {
                const int b = base + __popc(bal & ((1u << tid) - 1u));
                E.ilist[b] = i;
                E.ipos[i] = b;
            }
            base += __popc(bal);
        }
        if (tid == 0) E.misc[4] = base;
    }
    const bool ok = gj_dispatch(A, R, E, nth);
    if (ok) {
        // E.fac[s] = D / d_s and E.dpr[n] = D come from the elimination; the relation of
        // dependent row j on independent row i = ord[s] goes to Wc[j][ipos[i]]
        for (int x = tid; x < (m - n) * n; x += nth) {
            const int jp = n + x / n, s2 = x % n;
            const int j = E.ord[jp], i = E.ord[s2];
            const u64 w = fm_mul(E.M[E.perm[s2] * m + jp], E.fac[s2], p, A.pn);
            E.Wc[j * n + E.ipos[i]] = w ? p - w : 0;
        }
        for (int pos = n + tid; pos < m; pos += nth) E.kap[E.ord[pos]] = E.dpr[n];
    }
    EBAR();
    return ok;
}

// Rows whose residual is zero, moved to the end of E.ord for a second try of the fast path.
// Such rows are dependent with the trivial relation (their row of Q is e_j) wherever they
// come, and change neither the independent set nor the other rows' relations, so the output
// is still Algorithm 1's.  This keeps the fast path once a row has become an approximant of
// every order (the solution row of a reconstruction).  False (order unchanged) when no row is
// zero.
__device__ __forceinline__ bool zero_rows_last(const LeafArgs &A, const u64 *R, const i64 *t, ElimSm &E, int nth)
{
    const int m = A.m, n = A.n, tid = threadIdx.x, lane = tid & 31;
    // one warp per row, lanes over the columns, one vote; flags in E.ipos (m ints, rewritten
    // by the fast path's listing only after the reordering has read them)
    for (int i = tid >> 5; i < m; i += nth >> 5) {
        bool nz = false;
        for (int c = lane; c < n; c += 32) nz |= R[i * n + c] != 0;
        nz = __any_sync(0xffffffffu, nz);
        if (lane == 0) E.ipos[i] = !nz;
    }
    EBAR();
    int nzero = 0;
    for (int j = 0; j < m; j++) nzero += E.ipos[j];
    if (nzero == 0) return false;        // uniform: every thread read the same flags
    for (int i = tid; i < m; i += nth) {
        int r = 0;
        const i64 ti = t[i];
        const int zi = E.ipos[i];
        for (int j = 0; j < m; j++) {
            const int zj = E.ipos[j];
            r += (zj < zi) || (zj == zi && ((t[j] < ti) || (t[j] == ti && j < i)));
        }
        E.ord[r] = i;
    }
    EBAR();
    return true;
}

__device__ void mbasis1_scaled(const LeafArgs &A, const u64 *R, const i64 *t, ElimSm &E, int gn)
{
    const int m = A.m, n = A.n, tid = threadIdx.x, nth = gn;
    const u64 p = A.p;
    for (int i = tid; i < m; i += nth) {
        int r = 0;
        const i64 ti = t[i];
        for (int j = 0; j < m; j++) r += (t[j] < ti) || (t[j] == ti && j < i);
        E.ord[r] = i;
        E.kap[i] = A.one;
    }
    EBAR();
    if (m > n) {
        if (mbasis1_fast(A, R, E, nth)) return;
        if (zero_rows_last(A, R, t, E, nth) && mbasis1_fast(A, R, E, nth)) return;
    }
    {
        // general path: rows in order, fraction-free common-denominator elimination
        for (int x = tid; x < m * m; x += nth) E.W[x] = 0;
        for (int i = tid; i < m; i += nth) E.ind[i] = 0;
        if (tid == 0) { E.misc[2] = 0; E.dpr[0] = A.one; }
        EBAR();
        for (int pos = 0; pos < m; pos++) {
            const int r = E.ord[pos];
            const int rank = E.misc[2];
            const u64 D = E.dpr[0];
            for (int x = tid; x < n + m; x += nth) {
                u64 acc;
                if (x < n) {
                    acc = fm_mul(D, R[r * n + x], p, A.pn);
                    for (int b = 0; b < rank; b++)
                        acc = sub64(acc, fm_mul(R[r * n + E.pcs[b]], E.bas[b * n + x], p, A.pn), p);
                    E.vv[x] = acc;
                } else {
                    const int i = x - n;
                    acc = (i == r) ? D : 0;
                    for (int b = 0; b < rank; b++)
                        acc = sub64(acc, fm_mul(R[r * n + E.pcs[b]], E.tb[b * m + i], p, A.pn), p);
                    E.tv[i] = acc;
                }
            }
            EBAR();
            if (tid == 0) {
                int pc = -1;
                for (int c = 0; c < n; c++) if (E.vv[c]) { pc = c; break; }
                E.misc[3] = pc;
            }
            EBAR();
            const int pc = E.misc[3];
            if (pc >= 0) {
                const u64 pv = E.vv[pc];
                for (int b = tid; b < rank; b += nth) E.fac[b] = E.bas[b * n + pc];
                EBAR();
                for (int x = tid; x < rank * (n + m); x += nth) {
                    const int b = x / (n + m), c = x % (n + m);
                    if (c < n) E.bas[b * n + c] = sub64(fm_mul(pv, E.bas[b * n + c], p, A.pn), fm_mul(E.fac[b], E.vv[c], p, A.pn), p);
                    else E.tb[b * m + (c - n)] = sub64(fm_mul(pv, E.tb[b * m + (c - n)], p, A.pn),
                                                      fm_mul(E.fac[b], E.tv[c - n], p, A.pn), p);
                }
                for (int c = tid; c < n + m; c += nth) {
                    if (c < n) E.bas[rank * n + c] = fm_mul(D, E.vv[c], p, A.pn);
                    else E.tb[rank * m + (c - n)] = fm_mul(D, E.tv[c - n], p, A.pn);
                }
                EBAR();
                if (tid == 0) { E.pcs[rank] = pc; E.misc[2] = rank + 1; E.dpr[0] = fm_mul(pv, D, p, A.pn); E.ind[r] = 1; }
            } else {
                // dependent: the row of Q is tv (tv[r] = D): kap_r = D, W[r][i] = tv[i]
                for (int i = tid; i < m; i += nth)
                    if (i != r) E.W[r * m + i] = E.tv[i];
                if (tid == 0) E.kap[r] = D;
            }
            EBAR();
        }
    }
    EBAR();
    // compact form of the relations: the independent rows in index order, and for
    // every dependent row its coefficients on them
    if (tid < 32) {
        int base = 0;
        for (int i0 = 0; i0 < m; i0 += 32) {
            const int i = i0 + tid;
            const bool f = i < m && E.ind[i];
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (f) E.ilist[base + __popc(bal & ((1u << tid) - 1u))] = i;
            base += __popc(bal);
        }
        if (tid == 0) E.misc[4] = base;
    }
    EBAR();
    const int nind = E.misc[4];
    for (int x = tid; x < m * nind; x += nth) {
        const int j = x / nind, b = x % nind;
        E.Wc[j * n + b] = E.W[j * m + E.ilist[b]];
    }
    EBAR();
}

// New value of one coefficient of a dependent row j: kap_j X[j] + sum_i W[j][i] X[i],
// X[i] at stride `rs` between rows, lazy 128-bit sums reduced every `chunk` terms.
__device__ __forceinline__ u64 dep_combine(const LeafArgs &A, const ElimSm &E, int j, const u64 *X, i64 rs)
{
    const int n = A.n, nind = E.misc[4];
    const u64 *wc = E.Wc + (size_t)j * n;
    u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0, accm = 0;   // two independent chains (even / odd terms)
    int c0 = 1, c1 = 0;
    mac128(h0, l0, E.kap[j], X[(i64)j * rs]);
    int b = 0;
    for (; b + 1 < nind; b += 2) {
        mac128(h1, l1, wc[b], X[(i64)E.ilist[b] * rs]);
        mac128(h0, l0, wc[b + 1], X[(i64)E.ilist[b + 1] * rs]);
        if (++c1 == A.chunk) { accm = add64(accm, fm_redc(h1, l1, A.p, A.pn), A.p); h1 = l1 = 0; c1 = 0; }
        if (++c0 == A.chunk) { accm = add64(accm, fm_redc(h0, l0, A.p, A.pn), A.p); h0 = l0 = 0; c0 = 0; }
    }
    if (b < nind) mac128(h1, l1, wc[b], X[(i64)E.ilist[b] * rs]);   // c1 < chunk here
    accm = add64(accm, fm_redc(h0, l0, A.p, A.pn), A.p);
    return add64(accm, fm_redc(h1, l1, A.p, A.pn), A.p);
}

// ------------------------------------------------------------------ leaf kernel, one CTA
// G and P in global memory (double-buffered); for shapes whose slices do not fit
// the cluster kernel's shared memory.
// IP: interpolant leaf (Algorithm 4): the residual list holds P(alpha_l) E_l, independent
// rows are multiplied by (x - alpha_k) (by alpha_l - alpha_k in the list) instead of x.
template <bool IP>
__global__ void __launch_bounds__(512) k_mbasis_leaf(const LeafArgs A)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int m = A.m, n = A.n, T = A.T;
    const int tid = threadIdx.x, nth = blockDim.x;
    i64 *t = (i64 *)smraw;
    u64 *lam = (u64 *)(t + m);
    u64 *R = lam + m;
    u64 *ew = R + (size_t)m * n;
    int *ei = (int *)(ew + elim_words(m, n));
    ElimSm E = elim_carve(ew, ei, m, n);

    u64 *G = A.G0, *Gn = A.G1, *P = A.P0, *Pn = A.P1;
    for (int i = tid; i < m; i += nth) { t[i] = A.s_in[i]; lam[i] = A.one; }
    for (int x = tid; x < m * n * T; x += nth) {
        const int a = x % T, e = x / T;
        G[x] = mmul(A.F[(i64)e * A.sF + a], A.r2, A);
    }
    const int LP = T + 1;
    for (int x = tid; x < m * m * LP; x += nth) {
        const int a = x % LP, e = x / LP;
        P[x] = (a == 0 && (e / m) == (e % m)) ? A.one : 0;
    }
    __syncthreads();
    for (int k = 0; k < T; k++) {
        for (int x = tid; x < m * n; x += nth) R[x] = G[(i64)x * T + k];
        __syncthreads();
        mbasis1_scaled(A, R, t, E, nth);
        const int ngl = T - k - 1;
        for (int x = tid; x < m * n * ngl; x += nth) {
            const int a = k + 1 + x % ngl, e = x / ngl, j = e / n, c = e % n;
            u64 val;
            if (!E.ind[j]) val = dep_combine(A, E, j, G + (i64)c * T + a, (i64)n * T);
            else if (IP) val = mmul(sub64(A.alpha[a], A.alpha[k], A.p), G[(i64)e * T + a], A);
            else val = G[(i64)e * T + a - 1];
            Gn[(i64)e * T + a] = val;
        }
        const int np = k + 2;
        for (int x = tid; x < m * m * np; x += nth) {
            const int a = x % np, e = x / np, j = e / m, c = e % m;
            u64 val;
            if (E.ind[j]) {
                val = a ? P[(i64)e * LP + a - 1] : 0;
                if (IP && a <= k) val = sub64(val, mmul(A.alpha[k], P[(i64)e * LP + a], A), A.p);
            } else if (a == k + 1) val = 0;
            else val = dep_combine(A, E, j, P + (i64)c * LP + a, (i64)m * LP);
            Pn[(i64)e * LP + a] = val;
        }
        __syncthreads();
        for (int i = tid; i < m; i += nth) {
            if (E.ind[i]) t[i] += 1;
            else lam[i] = mmul(E.kap[i], lam[i], A);
        }
        { u64 *s2 = G; G = Gn; Gn = s2; s2 = P; P = Pn; Pn = s2; }
        __syncthreads();
    }
    for (int i = tid; i < m; i += nth) {
        E.kap[i] = mmul(mpow(lam[i], A.p - 2, A), 1, A);   // plain lam_i^-1
        A.s_out[i] = t[i];
    }
    __syncthreads();
    for (int x = tid; x < m * m * LP; x += nth) {
        const int a = x % LP, e = x / LP, i = e / m;
        A.P[(i64)e * A.sP + a] = mmul(P[x], E.kap[i], A);
    }
}

// ------------------------------------------------------------------ leaf kernel, CTA cluster
// LEAF_CL CTAs; CTA r owns the G columns [r n / CL, (r+1) n / CL) and the P columns
// [r m / CL, (r+1) m / CL), both in its shared memory.  The order steps are pipelined
// over two warp groups: at step k, warps 0 .. LEAF_EW-1 run the elimination of the
// residual R_k (Algorithm 1) while the other warps apply the previous step's Q_{k-1} to
// the rest of G (coefficients >= k+1) and to P.  Then every thread helps with the one
// thing the next elimination waits for: coefficient k+1 of Q_k G, this CTA's columns of
// R_{k+1}, written into every CTA's residual buffer (distributed shared memory) before
// one cluster barrier.  G, P, the residuals and the elimination outputs are
// double-buffered by step parity.
#define LEAF_EW 8

// Q_k applied to this CTA's slices (k = the step of E): G coefficients a >= k+2 of
// Gs -> Gd (skipped when G is null) and P coefficients 0 .. k+1 of Ps -> Pd, by threads
// ut = 0 .. un-1.
template <bool IP>
__device__ void leaf_apply(const LeafArgs &A, const ElimSm &E, int k, const u64 *Gs, u64 *Gd, const u64 *Ps, u64 *Pd,
                           int ng, int ngm, int np_, int npm, int ut, int un)
{
    const int m = A.m, T = A.T, LP = T + 1;
    if (Gs) {
        const int ngl = T - k - 2;
        for (int x = ut; x < m * ng * ngl; x += un) {
            const int a = k + 2 + x % ngl, e = x / ngl, j = e / ng, c = e % ng;
            const i64 o = ((i64)j * ngm + c) * T + a;
            u64 val;
            if (!E.ind[j]) val = dep_combine(A, E, j, Gs + (i64)c * T + a, (i64)ngm * T);
            else if (IP) val = mmul(sub64(A.alpha[a], A.alpha[k], A.p), Gs[o], A);
            else val = Gs[o - 1];
            Gd[o] = val;
        }
    }
    const int npc = k + 2;
    for (int x = ut; x < m * np_ * npc; x += un) {
        const int a = x % npc, e = x / npc, j = e / np_, c = e % np_;
        const i64 o = ((i64)j * npm + c) * LP + a;
        u64 val;
        if (E.ind[j]) {
            val = a ? Ps[o - 1] : 0;
            if (IP && a <= k) val = sub64(val, mmul(A.alpha[k], Ps[o], A), A.p);
        } else if (a == k + 1) val = 0;
        else val = dep_combine(A, E, j, Ps + (i64)c * LP + a, (i64)npm * LP);
        Pd[o] = val;
    }
}

template <bool IP>
__global__ void __launch_bounds__(512) k_mbasis_leaf_cl(const LeafArgs A)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int LEAF_CL = (int)cl.num_blocks();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int m = A.m, n = A.n, T = A.T, LP = T + 1;
    const int tid = threadIdx.x, nth = blockDim.x, egn = LEAF_EW * 32;
    const int rk = (int)cl.block_rank();
    const int g0 = rk * n / LEAF_CL, g1 = (rk + 1) * n / LEAF_CL, ng = g1 - g0;
    const int p0 = rk * m / LEAF_CL, p1 = (rk + 1) * m / LEAF_CL, np_ = p1 - p0;
    const int ngm = (n + LEAF_CL - 1) / LEAF_CL, npm = (m + LEAF_CL - 1) / LEAF_CL;
    const size_t ewn = elim_words(m, n);
    const int ein = elim_ints(m, n);
    i64 *t = (i64 *)smraw;
    u64 *lam = (u64 *)(t + m);
    u64 *Rb = lam + m;                                  // 2 x m x n
    u64 *G0 = Rb + 2 * (size_t)m * n, *G1 = G0 + (size_t)m * ngm * T;
    u64 *P0 = G1 + (size_t)m * ngm * T, *P1 = P0 + (size_t)m * npm * LP;
    u64 *ew = P1 + (size_t)m * npm * LP;               // 2 elimination outputs
    int *ei = (int *)(ew + 2 * ewn);

    // G slice: G0[(i*ngm + cl)*T + a] = F[i][g0 + cl][a]; P slice: identity columns
    for (int i = tid; i < m; i += nth) { t[i] = A.s_in[i]; lam[i] = A.one; }
    for (int x = tid; x < m * ng * T; x += nth) {
        const int a = x % T, e = x / T, i = e / ng, c = e % ng;
        G0[((i64)i * ngm + c) * T + a] = mmul(A.F[((i64)i * n + g0 + c) * A.sF + a], A.r2, A);
    }
    for (int x = tid; x < m * np_ * LP; x += nth) {
        const int a = x % LP, e = x / LP, i = e / np_, c = e % np_;
        P0[((i64)i * npm + c) * LP + a] = (a == 0 && i == p0 + c) ? A.one : 0;
    }
    __syncthreads();
    // R_0: coefficient 0 of this CTA's G columns, to every CTA
    for (int x = tid; x < LEAF_CL * m * ng; x += nth) {
        const int dst = x / (m * ng), e = x % (m * ng), i = e / ng, c = e % ng;
        u64 *rR = cl.map_shared_rank(Rb, dst);
        rR[i * n + g0 + c] = G0[((i64)i * ngm + c) * T];
    }
    for (int k = 0; k < T; k++) {
        cl.sync();                                      // R_k is complete in every CTA
        const u64 *R = Rb + (size_t)(k & 1) * m * n;
        const ElimSm Ek = elim_carve(ew + (k & 1) * ewn, ei + (k & 1) * ein, m, n);
        u64 *Gk = (k & 1) ? G1 : G0;                   // G after k steps (coefficients >= k+1)
        if (tid < egn) {
            ElimSm Ew = Ek;
            mbasis1_scaled(A, R, t, Ew, egn);
        } else if (k > 0) {
            const ElimSm Ep = elim_carve(ew + ((k - 1) & 1) * ewn, ei + ((k - 1) & 1) * ein, m, n);
            leaf_apply<IP>(A, Ep, k - 1, (k & 1) ? G0 : G1, Gk, (k & 1) ? P0 : P1, (k & 1) ? P1 : P0, ng, ngm, np_,
                           npm, tid - egn, nth - egn);
        }
        __syncthreads();
        if (k + 1 < T) {
            // R_{k+1}: coefficient k+1 of Q_k G for this CTA's columns, to every CTA.  Entry
            // (j, c) is taken by 16 threads: the kap term and the independent rows' terms are
            // spread over them and summed by shuffles (every lane takes part), and thread h
            // stores the entry into CTA h.
            u64 *Rn = Rb + (size_t)((k + 1) & 1) * m * n;
            const int nind = Ek.misc[4], h = tid & 15;
            const i64 rs = (i64)ngm * T;
            for (int e0 = 0; e0 < m * ng; e0 += nth / 16) {
                const int e = e0 + tid / 16;
                const bool act = e < m * ng;
                const int j = act ? e / ng : 0, c = act ? e % ng : 0;
                const bool dep = act && !Ek.ind[j];
                const u64 *X = Gk + (i64)c * T + k + 1;
                u64 hi = 0, lo = 0, acc = 0;
                if (dep) {
                    int cnt = 0;
                    if (h == 0) { mac128(hi, lo, Ek.kap[j], X[(i64)j * rs]); cnt = 1; }
                    for (int b = h; b < nind; b += 16) {
                        mac128(hi, lo, Ek.Wc[j * n + b], X[(i64)Ek.ilist[b] * rs]);
                        if (++cnt == A.chunk) { acc = add64(acc, fm_redc(hi, lo, A.p, A.pn), A.p); hi = lo = 0; cnt = 0; }
                    }
                }
                u64 val = add64(acc, fm_redc(hi, lo, A.p, A.pn), A.p);
#pragma unroll
                for (int o = 8; o >= 1; o >>= 1) val = add64(val, __shfl_xor_sync(0xffffffffu, val, o, 16), A.p);
                if (act && !dep)   // independent rows: x R_k (approximants), (alpha_{k+1} - alpha_k) G_{k+1} (interpolants)
                    val = IP ? mmul(sub64(A.alpha[k + 1], A.alpha[k], A.p), X[(i64)j * rs], A) : R[j * n + g0 + c];
                if (act && h < LEAF_CL) cl.map_shared_rank(Rn, h)[j * n + g0 + c] = val;
            }
        }
        for (int i = tid; i < m; i += nth) {
            if (Ek.ind[i]) t[i] += 1;
            else lam[i] = mmul(Ek.kap[i], lam[i], A);
        }
    }
    // P after T steps: Q_{T-1} applied to P after T-1 steps
    __syncthreads();
    {
        const ElimSm El = elim_carve(ew + ((T - 1) & 1) * ewn, ei + ((T - 1) & 1) * ein, m, n);
        leaf_apply<IP>(A, El, T - 1, nullptr, nullptr, ((T - 1) & 1) ? P1 : P0, (T & 1) ? P1 : P0, ng, ngm, np_, npm,
                       tid, nth);
    }
    __syncthreads();
    for (int i = tid; i < m; i += nth) lam[i] = mmul(mpow(lam[i], A.p - 2, A), 1, A);   // plain lam_i^-1
    if (rk == 0)
        for (int i = tid; i < m; i += nth) A.s_out[i] = t[i];
    __syncthreads();
    const u64 *Pf = (T & 1) ? P1 : P0;
    for (int x = tid; x < m * np_ * LP; x += nth) {
        const int a = x % LP, e = x / LP, i = e / np_, c = e % np_;
        A.P[((i64)i * m + p0 + c) * A.sP + a] = mmul(Pf[((i64)i * npm + c) * LP + a], lam[i], A);
    }
    cl.sync();   // no CTA leaves while others may still access its shared memory
}

#undef EBAR
