/*
 * CPU oracle, plain C, FP64.  TEST INFRASTRUCTURE ONLY: tests, the smoke
 * check and the CPU baseline of the benchmark use it; the product path never
 * loads it.  It shares no code with the CUDA library.
 *
 * Contents
 *   oracle_jw_build   -- the qubit Hamiltonian of Eq. (eham) -> Eq. (sham) by
 *                        direct Jordan-Wigner operator algebra: every ladder
 *                        operator is a sum of two Pauli strings, every
 *                        one- and two-body term is the product of its ladder
 *                        operators, equal strings are merged (Sec. 2.3).
 *   oracle_coupled    -- for one bitstring x, the matrix row H_{x x'} over all
 *                        x' reached by the (ungrouped) Pauli strings.
 *   oracle_eloc_lut   -- Eq. (Eloc) with psi(x') read from a table of the
 *                        samples S: the sample-aware sum of Sec. 3.4 (4).
 *
 * Conventions (stated here, not derived from the CUDA code):
 *   qubit j is bit j%64 of word j/64; |1> = occupied.
 *   Pauli string in "Y form": mask xy marks qubits carrying X or Y, mask yz
 *   marks qubits carrying Y or Z (the pmXY / pmYZ pair of Alg. 1).
 *   a^dag_j = Z_{<j} (X_j - i Y_j)/2,  a_j = Z_{<j} (X_j + i Y_j)/2.
 *   P|x> = i^{nY} (-1)^{popc(x & yz)} |x ^ xy>  (Y|b> = i(-1)^b |1-b>).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXW 2

typedef struct {
    uint64_t xy[MAXW], yz[MAXW];
    double re, im;
} pstr;

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

/* Product of two single-qubit Paulis in the textbook table
 *   XY = iZ, YZ = iX, ZX = iY, YX = -iZ, ZY = -iX, XZ = -iY, PP = I.
 * Written over whole words: with sigma(a,b) = i^{ab} X^a Z^b per qubit
 * (a = xy bit, b = yz bit), sigma1 sigma2 = i^{a1b1 + a2b2 + 2 b1a2 - a3b3}
 * sigma3, and the exponent adds up over qubits. */
static void pmul(const pstr *A, const pstr *B, pstr *C, int W) {
    int k = 0;
    for (int w = 0; w < W; ++w) {
        uint64_t a1 = A->xy[w], b1 = A->yz[w], a2 = B->xy[w], b2 = B->yz[w];
        uint64_t a3 = a1 ^ a2, b3 = b1 ^ b2;
        k += popc64(a1 & b1) + popc64(a2 & b2) + 2 * popc64(b1 & a2) - popc64(a3 & b3);
        C->xy[w] = a3;
        C->yz[w] = b3;
    }
    k = ((k % 4) + 4) % 4;
    /* (re + i im) * i^k */
    double re = A->re * B->re - A->im * B->im;
    double im = A->re * B->im + A->im * B->re;
    for (int t = 0; t < k; ++t) {
        double r2 = -im, i2 = re;
        re = r2;
        im = i2;
    }
    C->re = re;
    C->im = im;
}

/* ladder operator j as two strings: Z_{<j} X_j and Z_{<j} Y_j with
 * coefficients 1/2 and -i/2 (creation) or +i/2 (annihilation). */
static void ladder(int j, int dag, int W, pstr out[2]) {
    memset(out, 0, 2 * sizeof(pstr));
    for (int q = 0; q < j; ++q) {
        out[0].yz[q / 64] |= 1ull << (q % 64);
        out[1].yz[q / 64] |= 1ull << (q % 64);
    }
    out[0].xy[j / 64] |= 1ull << (j % 64);          /* X_j */
    out[1].xy[j / 64] |= 1ull << (j % 64);          /* Y_j */
    out[1].yz[j / 64] |= 1ull << (j % 64);
    out[0].re = 0.5;
    out[0].im = 0.0;
    out[1].re = 0.0;
    out[1].im = dag ? -0.5 : 0.5;
    (void)W;
}

/* ---- open-addressing map from a Pauli string to its summed coefficient ---- */
typedef struct {
    pstr *slot;
    uint8_t *used;
    int64_t cap, n;
    int W;
} pmap;

static uint64_t hkey(const pstr *p, int W) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (int w = 0; w < W; ++w) {
        h ^= p->xy[w] + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
        h ^= p->yz[w] + 0x8CB92BA72F3D8DD7ull + (h << 6) + (h >> 2);
    }
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    return h;
}

static int same(const pstr *a, const pstr *b, int W) {
    for (int w = 0; w < W; ++w)
        if (a->xy[w] != b->xy[w] || a->yz[w] != b->yz[w]) return 0;
    return 1;
}

static int pmap_init(pmap *m, int64_t cap, int W) {
    m->cap = cap;
    m->n = 0;
    m->W = W;
    m->slot = (pstr *)calloc((size_t)cap, sizeof(pstr));
    m->used = (uint8_t *)calloc((size_t)cap, 1);
    return (m->slot && m->used) ? 0 : -1;
}

static void pmap_free(pmap *m) {
    free(m->slot);
    free(m->used);
    m->slot = NULL;
    m->used = NULL;
}

static int pmap_add(pmap *m, const pstr *p);

static int pmap_grow(pmap *m) {
    pmap big;
    if (pmap_init(&big, m->cap * 2, m->W)) return -1;
    for (int64_t i = 0; i < m->cap; ++i)
        if (m->used[i]) pmap_add(&big, &m->slot[i]);
    pmap_free(m);
    *m = big;
    return 0;
}

static int pmap_add(pmap *m, const pstr *p) {
    if (2 * (m->n + 1) > m->cap && pmap_grow(m)) return -1;
    int64_t i = (int64_t)(hkey(p, m->W) & (uint64_t)(m->cap - 1));
    while (m->used[i]) {
        if (same(&m->slot[i], p, m->W)) {
            m->slot[i].re += p->re;
            m->slot[i].im += p->im;
            return 0;
        }
        i = (i + 1) & (m->cap - 1);
    }
    m->used[i] = 1;
    m->slot[i] = *p;
    m->n++;
    return 0;
}

/* ---- Hamiltonian ---- */
static pmap g_ham;
static int g_ham_ready = 0;

static void add_product(pmap *m, pstr *const ops[], int nops, double scale, int W) {
    /* expand the product of nops two-string sums into 2^nops strings */
    int combos = 1 << nops;
    for (int c = 0; c < combos; ++c) {
        pstr acc;
        memset(&acc, 0, sizeof acc);
        acc.re = scale;
        for (int k = 0; k < nops; ++k) {
            pstr t;
            pmul(&acc, &ops[k][(c >> k) & 1], &t, W);
            acc = t;
        }
        pmap_add(m, &acc);
    }
}

/* Builds H = e_core + sum_{pq,s} h_pq a+_{ps} a_{qs}
 *          + 1/2 sum_{pqrs,s t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
 * with spin orbital P = 2p + s.  Returns the number of merged strings (all
 * of them, before any fold or drop), or -1 on allocation failure. */
int64_t oracle_jw_build(int n_spatial, const double *h, const double *eri, double e_core) {
    int n = n_spatial, N = 2 * n, W = (N + 63) / 64;
    if (W > MAXW) return -1;
    if (g_ham_ready) pmap_free(&g_ham);
    if (pmap_init(&g_ham, 1 << 16, W)) return -1;
    g_ham_ready = 1;
    pstr ident;
    memset(&ident, 0, sizeof ident);
    ident.re = e_core;
    pmap_add(&g_ham, &ident);

    pstr A[2], B[2], C[2], D[2];
    for (int s = 0; s < 2; ++s)
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double v = h[p * n + q];
                if (v == 0.0) continue;
                ladder(2 * p + s, 1, W, A);
                ladder(2 * q + s, 0, W, B);
                pstr *ops[2] = {A, B};
                add_product(&g_ham, ops, 2, v, W);
            }
    for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t)
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q)
                    for (int r = 0; r < n; ++r)
                        for (int u = 0; u < n; ++u) {
                            double v = eri[((p * n + q) * n + r) * n + u];
                            if (v == 0.0) continue;
                            int P = 2 * p + s, Q = 2 * q + s, R = 2 * r + t, S = 2 * u + t;
                            if (P == R || Q == S) continue; /* a+_j a+_j = a_j a_j = 0 */
                            ladder(P, 1, W, A);
                            ladder(R, 1, W, B);
                            ladder(S, 0, W, C);
                            ladder(Q, 0, W, D);
                            pstr *ops[4] = {A, B, C, D};
                            add_product(&g_ham, ops, 4, 0.5 * v, W);
                        }
    return g_ham.n;
}

/* copy the merged strings out (any order); arrays sized by the count above */
int oracle_jw_fetch(uint64_t *xy, uint64_t *yz, double *re, double *im) {
    if (!g_ham_ready) return -1;
    int W = g_ham.W;
    int64_t k = 0;
    for (int64_t i = 0; i < g_ham.cap; ++i) {
        if (!g_ham.used[i]) continue;
        for (int w = 0; w < W; ++w) {
            xy[k * W + w] = g_ham.slot[i].xy[w];
            yz[k * W + w] = g_ham.slot[i].yz[w];
        }
        re[k] = g_ham.slot[i].re;
        im[k] = g_ham.slot[i].im;
        ++k;
    }
    pmap_free(&g_ham);
    g_ham_ready = 0;
    return 0;
}

/* ---- matrix rows and local energies ---- */
typedef struct {
    uint64_t key[MAXW];
    double v;
    int64_t order;
} rowent;

typedef struct {
    rowent *e;
    uint8_t *used;
    int64_t *ins; /* insertion order -> slot */
    int64_t cap, n;
} rowmap;

static uint64_t rhash(const uint64_t *k, int W) {
    uint64_t h = 0x2545F4914F6CDD1Dull;
    for (int w = 0; w < W; ++w) {
        h ^= k[w];
        h *= 0x9E3779B97F4A7C15ull;
        h ^= h >> 29;
    }
    return h;
}

static int rowmap_init(rowmap *m, int64_t cap) {
    m->cap = cap;
    m->n = 0;
    m->e = (rowent *)malloc((size_t)cap * sizeof(rowent));
    m->used = (uint8_t *)calloc((size_t)cap, 1);
    m->ins = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    return (m->e && m->used && m->ins) ? 0 : -1;
}

static void rowmap_free(rowmap *m) {
    free(m->e);
    free(m->used);
    free(m->ins);
}

static void rowmap_clear(rowmap *m) {
    for (int64_t k = 0; k < m->n; ++k) m->used[m->ins[k]] = 0;
    m->n = 0;
}

static void rowmap_add(rowmap *m, const uint64_t *key, double v, int W) {
    int64_t i = (int64_t)(rhash(key, W) & (uint64_t)(m->cap - 1));
    while (m->used[i]) {
        int eq = 1;
        for (int w = 0; w < W; ++w) eq &= (m->e[i].key[w] == key[w]);
        if (eq) {
            m->e[i].v += v;
            return;
        }
        i = (i + 1) & (m->cap - 1);
    }
    m->used[i] = 1;
    for (int w = 0; w < W; ++w) m->e[i].key[w] = key[w];
    m->e[i].v = v;
    m->e[i].order = m->n;
    m->ins[m->n++] = i;
}

static int64_t pow2_at_least(int64_t v) {
    int64_t c = 1;
    while (c < v) c <<= 1;
    return c;
}

/* H_{x x'} = <x|H|x'> = sum_t coef_t <x|P_t|x'>, where the folded coefficient
 * coef_t = Re(c_t) Re((-i)^{nY}) already carries i^{nY} (Alg. 1), so
 * <x|P_t|x'> contributes coef_t (-1)^{popc(x' & yz_t)} when x = x' ^ xy_t. */
static void row_of(const uint64_t *x, int W, int64_t n_terms, const uint64_t *xy,
                   const uint64_t *yz, const double *coef, rowmap *m) {
    rowmap_clear(m);
    uint64_t xp[MAXW];
    for (int64_t t = 0; t < n_terms; ++t) {
        int par = 0;
        for (int w = 0; w < W; ++w) {
            xp[w] = x[w] ^ xy[t * W + w];
            par += popc64(xp[w] & yz[t * W + w]);
        }
        rowmap_add(m, xp, (par & 1) ? -coef[t] : coef[t], W);
    }
}

static int in_sector(const uint64_t *x, int W, int n_alpha, int n_beta) {
    const uint64_t EVEN = 0x5555555555555555ull;
    int a = 0, b = 0;
    for (int w = 0; w < W; ++w) {
        a += popc64(x[w] & EVEN);
        b += popc64(x[w] & ~EVEN);
    }
    return a == n_alpha && b == n_beta;
}

/* All x' with the sector's electron counts that some string couples to x
 * (accidental zeros kept), in first-reached order.  Returns the count, or
 * -1 if cap is too small. */
int64_t oracle_coupled(int W, int64_t n_terms, const uint64_t *xy, const uint64_t *yz,
                       const double *coef, const uint64_t *x, int n_alpha, int n_beta,
                       uint64_t *out_x, double *out_h, int64_t cap) {
    rowmap m;
    if (rowmap_init(&m, pow2_at_least(2 * n_terms + 2))) return -1;
    row_of(x, W, n_terms, xy, yz, coef, &m);
    int64_t k = 0;
    for (int64_t o = 0; o < m.n; ++o) {
        rowent *e = &m.e[m.ins[o]];
        if (!in_sector(e->key, W, n_alpha, n_beta)) continue;
        if (k >= cap) {
            rowmap_free(&m);
            return -1;
        }
        for (int w = 0; w < W; ++w) out_x[k * W + w] = e->key[w];
        out_h[k] = e->v;
        ++k;
    }
    rowmap_free(&m);
    return k;
}

static int key_cmp(const uint64_t *a, const uint64_t *b, int W) {
    for (int w = W - 1; w >= 0; --w) {
        if (a[w] < b[w]) return -1;
        if (a[w] > b[w]) return 1;
    }
    return 0;
}

/* binary search in the sorted sample table (the id_lut of Alg. 2) */
static int64_t find_key(const uint64_t *lut, int64_t n, const uint64_t *k, int W) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = key_cmp(&lut[mid * W], k, W);
        if (c == 0) return mid;
        if (c < 0)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/* Eq. (Eloc) restricted to x' in S (Sec. 3.4 (4)).
 * lut: the samples S, sorted ascending (most significant word first), with
 * lut_logpsi[2i], lut_logpsi[2i+1] = log|psi|, phase of lut row i.
 * x: the bitstrings to evaluate (each must be in S).
 * out[2i], out[2i+1] = Re, Im of E_loc(x_i). */
int oracle_eloc_lut(int W, int64_t n_terms, const uint64_t *xy, const uint64_t *yz,
                    const double *coef, int64_t n_lut, const uint64_t *lut,
                    const double *lut_logpsi, int64_t n_x, const uint64_t *x, int n_alpha,
                    int n_beta, double *out) {
    int bad = 0;
#pragma omp parallel reduction(| : bad)
    {
        rowmap m;
        if (rowmap_init(&m, pow2_at_least(2 * n_terms + 2))) {
            bad = 1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t i = 0; i < n_x; ++i) {
                const uint64_t *xi = &x[i * W];
                int64_t self = find_key(lut, n_lut, xi, W);
                if (self < 0) {
                    bad = 1;
                    continue;
                }
                double la = lut_logpsi[2 * self], ph = lut_logpsi[2 * self + 1];
                row_of(xi, W, n_terms, xy, yz, coef, &m);
                double er = 0.0, ei = 0.0;
                for (int64_t o = 0; o < m.n; ++o) {
                    rowent *e = &m.e[m.ins[o]];
                    if (!in_sector(e->key, W, n_alpha, n_beta)) continue;
                    int64_t j = find_key(lut, n_lut, e->key, W);
                    if (j < 0) continue;
                    double mag = exp(lut_logpsi[2 * j] - la);
                    double d = lut_logpsi[2 * j + 1] - ph;
                    er += e->v * mag * cos(d);
                    ei += e->v * mag * sin(d);
                }
                out[2 * i] = er;
                out[2 * i + 1] = ei;
            }
            rowmap_free(&m);
        }
    }
    return bad ? -1 : 0;
}
