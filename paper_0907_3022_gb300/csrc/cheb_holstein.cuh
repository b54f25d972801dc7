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

// G(j, R) at t[j * w + R], j in [0, L], R in [0, nph], w = nph + 1 (values < 2^31)
struct HolG {
    const int32_t* t;
    int w;
    __host__ __device__ int64_t operator()(int j, int R) const { return t[j * w + R]; }
};

inline void make_hol_g(int L, int nph, const std::vector<int64_t>& binom, std::vector<int32_t>& g)
{
    Binom C{binom.data(), L};
    g.assign((size_t)(L + 1) * (nph + 1), 0);
    for (int j = 0; j <= L; ++j)
        for (int R = 0; R <= nph; ++R) g[(size_t)j * (nph + 1) + R] = (int32_t)C(R + L - j, L - j);
}

__host__ __device__ inline int hol_occ(uint64_t lo, uint64_t hi, int j)
{
    return (int)(((j < 16) ? (lo >> (4 * j)) : (hi >> (4 * (j - 16)))) & 15u);
}

// occupations of phonon rank p (packed) and their sum
template <class GT>
__host__ __device__ inline int hol_unrank_packed(const GT& G, int L, int nph, int64_t p,
                                                 uint64_t& lo, uint64_t& hi)
{
    lo = 0;
    hi = 0;
    int R = nph;
    for (int j = 0; j < L; ++j) {
        int v = 0;
        while (v < R) {
            const int64_t cnt = G(j + 1, R - v);  // tuples of sites j+1.. with sum <= R - v
            if (p < cnt) break;
            p -= cnt;
            ++v;
        }
        if (j < 16) lo |= (uint64_t)v << (4 * j);
        else hi |= (uint64_t)v << (4 * (j - 16));
        R -= v;
    }
    return nph - R;
}

// f(e, n_e, up, dn) for e = L-1 down to 0, with up = rank(n + 1_e) - rank(n) (0 when
// sum n = nph) and dn = rank(n) - rank(n - 1_e) (0 when n_e = 0)
template <class GT, class F>
__host__ __device__ inline void hol_phonon_walk(const GT& G, int L, int nph, uint64_t lo,
                                                uint64_t hi, int ntot, F&& f)
{
    int64_t su = 0, sd = 0;
    int after = 0;  // sum of n_j over j > e
    for (int e = L - 1; e >= 0; --e) {
        if (e + 1 < L) {
            const int Rn = nph - ntot + after;  // R_{e+1}
            sd += G(e + 1, Rn);
            if (Rn >= 1) su += G(e + 1, Rn - 1);
        }
        const int ne = hol_occ(lo, hi, e);
        f(e, ne, ntot < nph ? 1 + su : (int64_t)0, ne > 0 ? 1 + sd : (int64_t)0);
        after += ne;
    }
}

}  // namespace cheb
