// Holstein basis helpers shared by the SELL build, the matrix-free operator and the host ABI
// (not part of the ABI).  See cheb_holstein.cu for the ranking.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "cheb_internal.cuh"

namespace cheb {

constexpr int HOL_MAX_L = 64;

// binomial table: C(m, j) at [m * (L + 2) + j], m in [0, nph + L + 1], j in [0, L + 1]
struct Binom {
    const int64_t* t;
    int L;
    __host__ __device__ int64_t operator()(int m, int j) const {
        if (m < 0 || j < 0 || j > m) return 0;
        return t[(int64_t)m * (L + 2) + j];
    }
};

inline bool make_binom(int L, int nph, std::vector<int64_t>& tab)
{
    const int mmax = nph + L + 1;
    tab.assign((size_t)(mmax + 1) * (L + 2), 0);
    for (int m = 0; m <= mmax; ++m) {
        tab[(size_t)m * (L + 2) + 0] = 1;
        for (int j = 1; j <= std::min(m, L + 1); ++j) {
            const int64_t a = tab[(size_t)(m - 1) * (L + 2) + j - 1];
            const int64_t b = (j <= m - 1) ? tab[(size_t)(m - 1) * (L + 2) + j] : 0;
            if (a > INT64_MAX - b) return false;
            tab[(size_t)m * (L + 2) + j] = a + b;
        }
    }
    return true;
}

__host__ __device__ inline int64_t hol_rank(const Binom& C, int L, int nph, const uint8_t* occ)
{
    int64_t r = 0;
    int R = nph;
    for (int j = 0; j < L; ++j) {
        const int n = occ[j];
        r += C(R + L - j, L - j) - C(R - n + L - j, L - j);
        R -= n;
    }
    return r;
}

__host__ __device__ inline void hol_unrank(const Binom& C, int L, int nph, int64_t p, uint8_t* occ)
{
    int R = nph;
    for (int j = 0; j < L; ++j) {
        const int m = L - 1 - j;
        int v = 0;
        while (v < R) {
            const int64_t cnt = C(R - v + m, m);  // tuples of the last m sites with sum <= R - v
            if (p < cnt) break;
            p -= cnt;
            ++v;
        }
        occ[j] = (uint8_t)v;
        R -= v;
    }
}

// ---- on-device construction of the SELL-C (C = 32) matrix ------------------------------------
struct HolParams {
    int L, nph, periodic;
    int64_t dph, n;
    double t, omega0, g;
    const double* delta;  // [L] or NULL
    const double* gsite;  // [L] or NULL
    Binom C;
};

// Matrix elements of Eq. ghm shared by the stored and the matrix-free operators, so both use
// the same double before scaling: diagonal Delta_e + w0 * (total phonon number) and the
// phonon term -g_e w0 sqrt(m) between occupations m - 1 and m at the electron site.
__host__ __device__ inline double hol_diag_value(const HolParams& P, int e, int ntot)
{
    return (P.delta ? P.delta[e] : 0.0) + P.omega0 * (double)ntot;
}
__host__ __device__ inline double hol_phonon_value(const HolParams& P, int e, int m)
{
    const double ge = P.gsite ? P.gsite[e] : P.g;
    return -ge * P.omega0 * sqrt((double)m);
}


// ---- phonon neighbours without a stored matrix (matrix-free operator, Sec. 3.3) -------------
// With G(j, R) = C(R + L - j, L - j), the number of tuples on sites j..L-1 with sum <= R, and
// Pascal's rule C(N + 1, K + 1) - C(N, K) = C(N, K + 1), the rank formula telescopes to
//     rank(n) = G(0, nph) - (R_L + 1) - sum_{j=1}^{L-1} C(R_j + L - j, L - j + 1),
// a function of the remaining budgets R_j alone.  Raising n_e by one lowers R_j by one for
// every j > e, hence
//     rank(n + 1_e) - rank(n) = 1 + sum_{j=e+1}^{L-1} G(j, R_j - 1)    (needs sum n < nph)
//     rank(n) - rank(n - 1_e) = 1 + sum_{j=e+1}^{L-1} G(j, R_j)        (needs n_e > 0)
// with R_j of n.  Both sums run over the sites after e, so one pass from e = L-1 down to 0
// gives the two offsets of every electron site from a single unranking.  Occupations are
// packed 4 bits per site (nph <= 15) in two words (L <= 32).
constexpr int HOLMF_MAX_L = 32;
constexpr int HOLMF_MAX_NPH = 15;

// Tuple counts of the walk: G(j, R) = C(R + L - j, L - j), stored as the pair
// (G(j, R - 1), G(j, R)) at t[j * w + R] (G(j, -1) = 0), j in [0, L], R in [0, nph],
// w = nph + 1.  Every value is below Dph < 2^31.
struct HolG {
    const int2* t;
    int w;
    __host__ __device__ int2 pair(int j, int R) const { return t[j * w + R]; }
    __host__ __device__ int32_t operator()(int j, int R) const { return t[j * w + R].y; }
};

inline void make_hol_g(int L, int nph, const std::vector<int64_t>& binom, std::vector<int2>& g)
{
    Binom C{binom.data(), L};
    const int w = nph + 1;
    g.assign((size_t)(L + 1) * w, make_int2(0, 0));
    for (int j = 0; j <= L; ++j)
        for (int R = 0; R <= nph; ++R)
            g[(size_t)j * w + R] = make_int2(R > 0 ? (int32_t)C(R - 1 + L - j, L - j) : 0,
                                             (int32_t)C(R + L - j, L - j));
}

// Occupations of phonon rank p, packed 4 bits per site with site L-1 in the lowest bits of
// lo (sites L-17 .. 0 continue in hi), and their sum.
template <class GT>
__host__ __device__ inline int hol_unrank_packed(const GT& G, int L, int nph, int32_t p,
                                                 uint64_t& lo, uint64_t& hi)
{
    lo = 0;
    hi = 0;
    int R = nph;
    for (int j = 0; j < L; ++j) {
        int v = 0;
        while (v < R) {
            const int32_t cnt = G(j + 1, R - v);  // tuples of sites j+1.. with sum <= R - v
            if (p < cnt) break;
            p -= cnt;
            ++v;
        }
        const int q = L - 1 - j;
        if (q < 16) lo |= (uint64_t)v << (4 * q);
        else hi |= (uint64_t)v << (4 * (q - 16));
        R -= v;
    }
    return nph - R;
}

// Walk over the electron sites e = L-1, L-2, ..., 0 of one phonon configuration n: step(e)
// returns n_e and the offsets up = rank(n + 1_e) - rank(n) (0 when sum n = nph) and
// dn = rank(n) - rank(n - 1_e) (0 when n_e = 0).  Offsets are below Dph < 2^31.
struct HolWalk {
    uint64_t lo, hi;   // occupations still to visit, the next one in the lowest 4 bits
    int ntot, after;   // total phonon number; sum of n_j over the sites already passed (j > e)
    int32_t su, sd;    // sum_{j > e} G(j, R_j - 1) and G(j, R_j)

    template <class GT>
    __host__ __device__ void begin(const GT& G, int L, int nph, int32_t p) {
        ntot = hol_unrank_packed(G, L, nph, p, lo, hi);
        after = 0;
        su = 0;
        sd = 0;
    }
    template <class GT>
    __host__ __device__ int step(const GT& G, int L, int nph, int e, int32_t& up, int32_t& dn) {
        if (e + 1 < L) {
            const int2 g = G.pair(e + 1, nph - ntot + after);  // at R_{e+1}
            su += g.x;
            sd += g.y;
        }
        const int ne = (int)(lo & 15u);
        lo = (lo >> 4) | (hi << 60);
        hi >>= 4;
        up = ntot < nph ? 1 + su : 0;
        dn = ne > 0 ? 1 + sd : 0;
        after += ne;
        return ne;
    }
};

}  // namespace cheb
