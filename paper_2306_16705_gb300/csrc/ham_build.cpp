// Host builder of the grouped Pauli-string Hamiltonian (Sec. 2.3, Eq. sham;
// Alg. 1; Sec. 3.4 (1)).
//
// Every Pauli string is written as F(a, b) = prod_q X_q^{a_q} Z_q^{b_q}
// (X before Z on each qubit), which makes every coefficient real:
//   a+_j = 1/2 F(e_j, z_<j) + 1/2 F(e_j, z_<=j),
//   a_j  = 1/2 F(e_j, z_<j) - 1/2 F(e_j, z_<=j),
//   F(a1,b1) F(a2,b2) = (-1)^{popc(b1 & a2)} F(a1^a2, b1^b2).
// Since X Z = -iY on a qubit, F(a, b) = (-i)^{popc(a&b)} P with P the Pauli
// string of X/Y mask a and Y/Z mask b, so the coefficient c of P is
// r (-i)^{nY} and Alg. 1's folded coefficient Re(c) Re((-i)^{nY}) is r for
// an even number of Y and 0 for an odd number.  With that, a string acts as
// F(a,b)|x> = (-1)^{popc(x & b)} |x ^ a>, which is the sign rule the kernels
// use.
//
// Work is split over OpenMP threads by a hash of the X mask (all products of
// one term share it), each thread merging equal strings in its own table.
#include <omp.h>
#include <parallel/algorithm>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hashfn.h"
#include "internal.h"

namespace nnqs {
namespace {

struct Ent {
    uint64_t a[2], b[2];
    double r;
};

class StrMap {
   public:
    explicit StrMap(int W) : W_(W) { rehash(1 << 12); }
    void add(const uint64_t *a, const uint64_t *b, double r) {
        if (2 * (n_ + 1) > cap_) rehash(cap_ * 2);
        size_t i = slot_of(a, b);
        while (used_[i]) {
            Ent &e = ent_[i];
            if (e.a[0] == a[0] && e.b[0] == b[0] && (W_ == 1 || (e.a[1] == a[1] && e.b[1] == b[1]))) {
                e.r += r;
                return;
            }
            i = (i + 1) & (cap_ - 1);
        }
        used_[i] = 1;
        Ent &e = ent_[i];
        e.a[0] = a[0];
        e.b[0] = b[0];
        e.a[1] = W_ > 1 ? a[1] : 0;
        e.b[1] = W_ > 1 ? b[1] : 0;
        e.r = r;
        ++n_;
    }
    template <class F>
    void for_each(F f) const {
        for (size_t i = 0; i < cap_; ++i)
            if (used_[i]) f(ent_[i]);
    }

   private:
    size_t slot_of(const uint64_t *a, const uint64_t *b) const {
        uint64_t h = W_ == 1 ? hash_key2(a[0], b[0]) : hash_key2(a[0] ^ mix64(a[1]), b[0] ^ mix64(b[1] + 1));
        return h & (cap_ - 1);
    }
    void rehash(size_t cap) {
        std::vector<Ent> old = std::move(ent_);
        std::vector<uint8_t> oldu = std::move(used_);
        ent_.assign(cap, Ent{});
        used_.assign(cap, 0);
        cap_ = cap;
        n_ = 0;
        for (size_t i = 0; i < old.size(); ++i)
            if (oldu[i]) add(old[i].a, old[i].b, old[i].r);
    }
    int W_;
    size_t cap_ = 0, n_ = 0;
    std::vector<Ent> ent_;
    std::vector<uint8_t> used_;
};

inline void below_mask(int j, uint64_t m[2]) {
    m[0] = j >= 64 ? ~0ull : ((1ull << j) - 1);
    m[1] = j >= 64 ? ((1ull << (j - 64)) - 1) : 0ull;
}

// Expands scale * op_0 op_1 ... op_{n-1} (ladder operators j[k], creation
// when cre[k]) into its 2^n strings and adds those with an even number of Y
// to the map.  The odd ones fold to zero (Re((-i)^{nY}) = 0, Alg. 1) and
// never share a key with an even one, so leaving them out changes no kept
// coefficient and halves the insertions.
void expand(StrMap &map, int nops, const int *j, const bool *cre, double scale) {
    uint64_t a[2] = {0, 0}, base[2] = {0, 0};
    int fixed_parity = 0;
    for (int k = 0; k < nops; ++k) {
        a[j[k] >> 6] ^= 1ull << (j[k] & 63);
        uint64_t m[2];
        below_mask(j[k], m);
        base[0] ^= m[0];
        base[1] ^= m[1];
        for (int l = k + 1; l < nops; ++l) fixed_parity += (j[l] < j[k]);
    }
    const double w = scale / double(1 << nops);
    for (int t = 0; t < (1 << nops); ++t) {
        uint64_t b[2] = {base[0], base[1]};
        int parity = fixed_parity;
        double c = w;
        for (int k = 0; k < nops; ++k) {
            if (!((t >> k) & 1)) continue;
            b[j[k] >> 6] ^= 1ull << (j[k] & 63);
            if (!cre[k]) c = -c;
            for (int l = k + 1; l < nops; ++l) parity += (j[l] == j[k]);
        }
        if ((__builtin_popcountll(a[0] & b[0]) + __builtin_popcountll(a[1] & b[1])) & 1) continue;
        map.add(a, b, (parity & 1) ? -c : c);
    }
}

inline uint64_t xmask_hash(const int *j, int nops) {
    uint64_t a[2] = {0, 0};
    for (int k = 0; k < nops; ++k) a[j[k] >> 6] ^= 1ull << (j[k] & 63);
    return hash_key2(a[0], a[1]);
}

inline bool key_less(const Ent &x, const Ent &y) {
    if (x.a[1] != y.a[1]) return x.a[1] < y.a[1];
    if (x.a[0] != y.a[0]) return x.a[0] < y.a[0];
    if (x.b[1] != y.b[1]) return x.b[1] < y.b[1];
    return x.b[0] < y.b[0];
}

inline int popc(uint64_t v) { return __builtin_popcountll(v); }

}  // namespace

nnqs_status build_pauli_host(int n_spatial, const double *h, const double *eri, double e_core,
                             double drop_tol, nnqs_ham *H) {
    const int n = n_spatial, N = 2 * n, W = (N + 63) / 64;
    H->n_spatial = n;
    H->n_qubits = N;
    H->W = W;
    const int T = std::max(1, omp_get_max_threads());
    std::vector<std::vector<Ent>> parts(T);
    bool oom = false;

#pragma omp parallel num_threads(T)
    {
        const int me = omp_get_thread_num();
        try {
            StrMap map(W);
            if (e_core != 0.0 && hash_key2(0, 0) % T == (uint64_t)me) {
                uint64_t z[2] = {0, 0};
                map.add(z, z, e_core);  // identity string, X mask 0
            }
            int j[4];
            bool cre[4];
            for (int s = 0; s < 2; ++s)
                for (int p = 0; p < n; ++p)
                    for (int q = 0; q < n; ++q) {
                        double v = h[p * n + q];
                        if (v == 0.0) continue;
                        j[0] = 2 * p + s;
                        cre[0] = true;
                        j[1] = 2 * q + s;
                        cre[1] = false;
                        if (xmask_hash(j, 2) % T != (uint64_t)me) continue;
                        expand(map, 2, j, cre, v);
                    }
            for (int s = 0; s < 2; ++s)
                for (int t = 0; t < 2; ++t)
                    for (int p = 0; p < n; ++p)
                        for (int q = 0; q < n; ++q)
                            for (int r = 0; r < n; ++r)
                                for (int u = 0; u < n; ++u) {
                                    const double v = eri[((size_t(p) * n + q) * n + r) * n + u];
                                    if (v == 0.0) continue;
                                    j[0] = 2 * p + s;  // a+_{p s}
                                    j[1] = 2 * r + t;  // a+_{r t}
                                    j[2] = 2 * u + t;  // a_{s t}
                                    j[3] = 2 * q + s;  // a_{q s}
                                    if (j[0] == j[1] || j[2] == j[3]) continue;  // a+a+ or aa on one orbital
                                    cre[0] = cre[1] = true;
                                    cre[2] = cre[3] = false;
                                    if (xmask_hash(j, 4) % T != (uint64_t)me) continue;
                                    expand(map, 4, j, cre, 0.5 * v);
                                }
            std::vector<Ent> &out = parts[me];
            map.for_each([&](const Ent &e) {
                int ny = popc(e.a[0] & e.b[0]) + popc(e.a[1] & e.b[1]);
                if (ny & 1) return;  // Re((-i)^{nY}) = 0: folded away (Alg. 1)
                if (!(std::fabs(e.r) >= drop_tol)) return;
                out.push_back(e);
            });
        } catch (...) {
#pragma omp critical
            oom = true;
        }
    }
    if (oom) return set_error(NNQS_E_NOMEM, "host allocation failed while merging Pauli strings");

    size_t total = 0;
    for (auto &p : parts) total += p.size();
    std::vector<Ent> all;
    all.reserve(total);
    for (auto &p : parts) {
        all.insert(all.end(), p.begin(), p.end());
        std::vector<Ent>().swap(p);
    }
    __gnu_parallel::sort(all.begin(), all.end(), key_less);

    H->n_terms = (int64_t)all.size();
    H->tyz.resize(all.size() * W);
    H->tcoef.resize(all.size());
    H->gxy.clear();
    H->goff.clear();
    H->max_group = 0;
    for (size_t i = 0; i < all.size(); ++i) {
        const Ent &e = all[i];
        bool fresh = (i == 0) || e.a[0] != all[i - 1].a[0] || e.a[1] != all[i - 1].a[1];
        if (fresh) {
            for (int w = 0; w < W; ++w) H->gxy.push_back(e.a[w]);
            H->goff.push_back((int64_t)i);
        }
        for (int w = 0; w < W; ++w) H->tyz[i * W + w] = e.b[w];
        H->tcoef[i] = e.r;
    }
    H->goff.push_back((int64_t)all.size());
    H->n_groups = (int64_t)H->goff.size() - 1;
    for (int64_t g = 0; g < H->n_groups; ++g)
        H->max_group = std::max<int64_t>(H->max_group, H->goff[g + 1] - H->goff[g]);
    return NNQS_OK;
}

uint64_t hash_words(const uint64_t *k, int W) { return W == 1 ? hash_key1(k[0]) : hash_key2(k[0], k[1]); }

nnqs_status upload_ham(nnqs_ham *H) {
    const int W = H->W;
    const int64_t G = H->n_groups, T = H->n_terms;
    if (T >= (int64_t(1) << 32)) return set_error(NNQS_E_UNSUPPORTED, "more than 2^32 Pauli strings");
    std::vector<uint32_t> off32(G + 1);
    for (int64_t g = 0; g <= G; ++g) off32[g] = (uint32_t)H->goff[g];
    std::vector<uint8_t> spin(G);
    H->max_xy_weight = 0;
    for (int64_t g = 0; g < G; ++g) {
        int pa = 0, pb = 0;
        for (int w = 0; w < W; ++w) {
            pa += popc(H->gxy[g * W + w] & kEven);
            pb += popc(H->gxy[g * W + w] & ~kEven);
        }
        H->max_xy_weight = std::max(H->max_xy_weight, pa + pb);
        spin[g] = ((pa & 1) || (pb & 1) || pa > 30 || pb > 30) ? 0xFF : uint8_t((pa / 2) | ((pb / 2) << 4));
    }
    // group hash: X/Y mask -> group index, load <= 0.5
    int64_t cap = 2;
    while (cap < 2 * G) cap <<= 1;
    std::vector<uint64_t> hk(size_t(cap) * W, ~0ull);
    std::vector<int32_t> hv(cap, -1);
    for (int64_t g = 0; g < G; ++g) {
        uint64_t i = hash_words(&H->gxy[g * W], W) & uint64_t(cap - 1);
        while (hv[i] >= 0) i = (i + 1) & uint64_t(cap - 1);
        for (int w = 0; w < W; ++w) hk[i * W + w] = H->gxy[g * W + w];
        hv[i] = (int32_t)g;
    }
    H->ghcap = cap;

    auto up = [&](void **dst, const void *src, size_t bytes) -> nnqs_status {
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(dst, bytes);
        if (e != cudaSuccess) return cuda_error(e, "cudaMalloc (Hamiltonian tables)");
        H->device_bytes += bytes;
        if (src) {
            e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy (Hamiltonian tables)");
        }
        return NNQS_OK;
    };
    NNQS_TRY(up((void **)&H->d_gxy, H->gxy.data(), H->gxy.size() * 8));
    NNQS_TRY(up((void **)&H->d_goff, off32.data(), off32.size() * 4));
    NNQS_TRY(up((void **)&H->d_gspin, spin.data(), spin.size()));
    NNQS_TRY(up((void **)&H->d_tyz, H->tyz.data(), H->tyz.size() * 8));
    NNQS_TRY(up((void **)&H->d_tcoef, H->tcoef.data(), H->tcoef.size() * 8));
    NNQS_TRY(up((void **)&H->d_ghkeys, hk.data(), hk.size() * 8));
    NNQS_TRY(up((void **)&H->d_ghvals, hv.data(), hv.size() * 4));
    return NNQS_OK;
}

}  // namespace nnqs
