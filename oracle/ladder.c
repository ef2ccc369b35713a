/*
 * CPU rungs of the local-energy speed-up ladder (Sec. 4.3, Fig. speedup-eloc).
 * TEST INFRASTRUCTURE ONLY, like oracle.c: the benchmark's CPU baseline times
 * them and the tests check them; the product path never loads them.
 *
 * Every rung computes the same sum, Eq. (Eloc) restricted to x' in S (the
 * sample-aware set of Sec. 3.4 (4)), over the grouped Hamiltonian of Alg. 1
 * (the compressed structure, technique (1), which the paper keeps in every
 * rung).  They differ only in the techniques the figure adds one by one:
 *
 *   rung 0, bare      -- no fusion, no sample-aware skip, no integer table:
 *                        for x, every group's coefficient H_{x x'} is formed
 *                        and the nonzero (x', H) pairs are stored first; then
 *                        each stored x' is searched for in S, kept as boolean
 *                        tuples (one byte per qubit, Sec. 3.4 (5)) in
 *                        byte-wise order, by binary search with byte-wise
 *                        comparison.
 *   rung 1, SA+FUSE   -- x' is searched for first (same tuple search); its
 *                        coefficient is formed only when x' is in S and added
 *                        to E_loc(x) at once (Sec. 3.4 (2), (4)).
 *   rung 2, +LUT      -- S as sorted integer keys, found by binary search on
 *                        one or two 64-bit compares (Sec. 3.4 (5)).
 * The paper does not say how its first two rungs searched the tuples; a
 * binary search over them is the reading taken here.
 *
 * Sign of a string: (-1)^{popc(x & yz_t)} with x the sample (the row), the
 * coefficients already folded by Re((-i)^{nY}) (Alg. 1).  OpenMP over samples.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LMAXW 2
#define LMAXN 128

static int lpopc(uint64_t v) { return __builtin_popcountll(v); }

static void to_tuple(const uint64_t *x, int N, uint8_t *t) {
    for (int q = 0; q < N; ++q) t[q] = (uint8_t)((x[q >> 6] >> (q & 63)) & 1u);
}

static int64_t bsearch_tuples(const uint8_t *tuples, int64_t n, int N, const uint8_t *t) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        const int c = memcmp(tuples + mid * N, t, (size_t)N);
        if (c == 0) return mid;
        if (c < 0)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

static int lkey_cmp(const uint64_t *a, const uint64_t *b, int W) {
    for (int w = W - 1; w >= 0; --w) {
        if (a[w] < b[w]) return -1;
        if (a[w] > b[w]) return 1;
    }
    return 0;
}

static int64_t bsearch_keys(const uint64_t *keys, int64_t n, const uint64_t *k, int W) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        const int c = lkey_cmp(&keys[mid * W], k, W);
        if (c == 0) return mid;
        if (c < 0)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/* H_{x, x ^ xy_m} = sum over the strings of group m */
static double group_coef(const uint64_t *x, int W, int64_t b, int64_t e, const uint64_t *yz,
                         const double *coef) {
    double h = 0.0;
    for (int64_t t = b; t < e; ++t) {
        int par = 0;
        for (int w = 0; w < W; ++w) par += lpopc(x[w] & yz[t * W + w]);
        h += (par & 1) ? -coef[t] : coef[t];
    }
    return h;
}

/* rung: 0 bare, 1 SA+FUSE, 2 +LUT.
 * groups: gxy[n_groups][W] masks, goff[n_groups + 1] string offsets, strings
 *   yz[n_terms][W], coef[n_terms].
 * S: keys[n_s][W] sorted ascending (most significant word first) with
 *   logpsi[2i], logpsi[2i + 1] = log|psi|, phase of keys row i (rung 2);
 *   tuples[n_s][N] the same rows as bytes, sorted in memcmp order, with
 *   tlogpsi in that order (rungs 0 and 1).
 * x[n_x][W]: the rows to evaluate (each in S); out[2i], out[2i+1] = E_loc.
 * Returns 0, or -1 (a row not in S, or no memory). */
int ladder_eloc(int rung, int N, int W, int64_t n_groups, const uint64_t *gxy, const int64_t *goff,
                const uint64_t *yz, const double *coef, int64_t n_s, const uint64_t *keys,
                const double *logpsi, const uint8_t *tuples, const double *tlogpsi, int64_t n_x,
                const uint64_t *x, double *out) {
    if (W < 1 || W > LMAXW || N < 1 || N > LMAXN || rung < 0 || rung > 2) return -1;
    int bad = 0;
#pragma omp parallel reduction(| : bad)
    {
        uint64_t *lx = NULL;
        double *lh = NULL;
        if (rung == 0) {
            lx = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_groups > 0 ? n_groups : 1) * W);
            lh = (double *)malloc(sizeof(double) * (size_t)(n_groups > 0 ? n_groups : 1));
            if (!lx || !lh) bad = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < n_x; ++i) {
            if (bad) continue;
            const uint64_t *xi = &x[i * W];
            uint8_t t[LMAXN];
            uint64_t xp[LMAXW];
            int64_t self;
            const double *lp = rung == 2 ? logpsi : tlogpsi;
            if (rung == 2) {
                self = bsearch_keys(keys, n_s, xi, W);
            } else {
                to_tuple(xi, N, t);
                self = bsearch_tuples(tuples, n_s, N, t);
            }
            if (self < 0) {
                bad = 1;
                continue;
            }
            const double la = lp[2 * self], ph = lp[2 * self + 1];
            double er = 0.0, ei = 0.0;
            if (rung == 0) {
                int64_t k = 0;
                for (int64_t m = 0; m < n_groups; ++m) {
                    for (int w = 0; w < W; ++w) lx[k * W + w] = xi[w] ^ gxy[m * W + w];
                    const double h = group_coef(xi, W, goff[m], goff[m + 1], yz, coef);
                    if (h != 0.0) lh[k++] = h;
                }
                for (int64_t q = 0; q < k; ++q) {
                    to_tuple(&lx[q * W], N, t);
                    const int64_t j = bsearch_tuples(tuples, n_s, N, t);
                    if (j < 0) continue;
                    const double mag = exp(lp[2 * j] - la), d = lp[2 * j + 1] - ph;
                    er += lh[q] * mag * cos(d);
                    ei += lh[q] * mag * sin(d);
                }
            } else {
                for (int64_t m = 0; m < n_groups; ++m) {
                    for (int w = 0; w < W; ++w) xp[w] = xi[w] ^ gxy[m * W + w];
                    int64_t j;
                    if (rung == 2) {
                        j = bsearch_keys(keys, n_s, xp, W);
                    } else {
                        to_tuple(xp, N, t);
                        j = bsearch_tuples(tuples, n_s, N, t);
                    }
                    if (j < 0) continue;
                    const double h = group_coef(xi, W, goff[m], goff[m + 1], yz, coef);
                    const double mag = exp(lp[2 * j] - la), d = lp[2 * j + 1] - ph;
                    er += h * mag * cos(d);
                    ei += h * mag * sin(d);
                }
            }
            out[2 * i] = er;
            out[2 * i + 1] = ei;
        }
        free(lx);
        free(lh);
    }
    return bad ? -1 : 0;
}
