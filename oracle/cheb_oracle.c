/*
 * Oracle for the Chebyshev time-evolution method (Fehske et al., "Numerical approaches to
 * time evolution of complex quantum systems", Sec. 2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded FP64 reference
 * that the CUDA library is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the library never calls it and shares no code
 * with it.  Everything here is written for a reader to check against the paper by eye:
 * no blocking, no fusion, no reordering beyond what the equations state.
 *
 * Contents
 *   rescaling of H into [-1,1] ......................... Sec. 2.2, text after Eq. (U_1)
 *   expansion coefficients c_k (integral definition) ... Sec. 2.2, Eq. (c_k)
 *   truncation order M ................................. Sec. 2.2, Eq. (dec_Bessel) and text
 *   Chebyshev step  U(dt) psi = sum_k C_k v_k .......... Sec. 2.2, Eqs. (U_1), (rec)
 *   operators as explicit sparse matrices (CSR):
 *     1D finite-difference grid ........................ Sec. 3.1
 *     honeycomb tight-binding ribbon, zigzag edges ..... Sec. 3.2, Eq. (model)
 *     Holstein chain in a truncated phonon basis ....... Sec. 3.3, Eq. (ghm)
 *   observables <n_i>, <b_i^+ b_i>, chi_ii ............. Sec. 3.3 (Fig. 3 caption)
 *   reverse-mode gradient of a region probability w.r.t. the on-site potential: no
 *   counterpart in the paper; it differentiates Eqs. (U_1) and (rec) with a, b held fixed.
 *
 * Vectors cross this interface as interleaved (re, im) doubles, i.e. C99 double complex.
 * Functions return 0 on success and a negative number on a bad argument.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------------------ */
/* Rescaling, Sec. 2.2: b = (Emax + Emin)/2, a = (Emax - Emin + eps)/2,                  */
/* eps = alpha (Emax - Emin), so the spectrum of (H - b)/a lies in [-1/(1+alpha), 1/(1+alpha)]. */
/* ------------------------------------------------------------------------------------ */
int oracle_rescale(double emin, double emax, double alpha, double* a, double* b)
{
    if (!(emax >= emin) || !(alpha >= 0.0)) return -1;
    double eps = alpha * (emax - emin);
    *b = 0.5 * (emax + emin);
    *a = 0.5 * (emax - emin + eps);
    if (!(*a > 0.0)) return -2;
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Expansion coefficients, Sec. 2.2, Eq. (c_k):                                           */
/*   c_k(z) = int_{-1}^{1} T_k(x) e^{-i x z} / (pi sqrt(1-x^2)) dx                        */
/* With x = cos(theta) this is (1/pi) int_0^pi cos(k theta) e^{-i z cos theta} d theta,   */
/* i.e. (1/2pi) int_0^{2pi} cos(k theta) e^{-i z cos theta} d theta.  The integrand is    */
/* smooth and 2pi-periodic, so the trapezoidal rule on P equally spaced nodes is exact     */
/* up to the aliased terms c_{mP +- k}, m >= 1, which vanish to machine precision once     */
/* P - k is well past z.  The oracle evaluates that sum directly.                         */
/*                                                                                          */
/* The multipliers of T_k(H~) psi in Eq. (U_1) are                                         */
/*   C_k = e^{-i b dt} (2 - delta_k0) c_k(a dt),                                           */
/* and M is the largest k <= kmax with |C_k| >= tol (coefficients beyond M are dropped,    */
/* as the text after Eq. (dec_Bessel) describes).  C has room for kmax + 1 entries.        */
/* ------------------------------------------------------------------------------------ */
static long next_pow2(long x)
{
    long p = 1;
    while (p < x) p <<= 1;
    return p;
}

int oracle_bessel_coeffs(double z, int kmax, double* c_out /* 2*(kmax+1): c_k(z) */)
{
    if (kmax < 0 || !(z >= 0.0)) return -1;
    long P = next_pow2(2 * (long)kmax + 2 * (long)ceil(z) + 256);
    /* Node values.  The phase z cos(theta_j) reaches z, so each node is evaluated in long
       double (cos reduced to the first octant by symmetry, then e^{-i phase}) and rounded to
       double once; the rounding error of a double phase (~ z * 1e-16) would otherwise put a
       noise floor near 1e-15 under the coefficients. */
    double* ctab = (double*)malloc(sizeof(double) * (size_t)P);
    cplx* f = (cplx*)malloc(sizeof(cplx) * (size_t)P);
    if (!ctab || !f) { free(ctab); free(f); return -3; }
    const long double twopi = 2.0L * acosl(-1.0L);
    for (long m = 0; m < P; ++m) {
        long q = m;
        long double sgn = 1.0L;
        if (q > P / 2) q = P - q;                       /* cos(2pi - t) = cos t  */
        if (q > P / 4) { q = P / 2 - q; sgn = -1.0L; }  /* cos(pi - t) = -cos t  */
        long double v;
        if (q <= P / 8) v = cosl(twopi * (long double)q / (long double)P);
        else v = sinl(twopi * (long double)(P / 4 - q) / (long double)P);
        v *= sgn;
        long double ph = (long double)z * v;
        ctab[m] = (double)v;
        f[m] = (double)cosl(ph) - I * (double)sinl(ph);
    }
    for (int k = 0; k <= kmax; ++k) {
        cplx s = 0.0;
        for (long j = 0; j < P; ++j) {
            long idx = (long)(((int64_t)k * (int64_t)j) & (int64_t)(P - 1)); /* k j mod P */
            s += ctab[idx] * f[j];
        }
        s /= (double)P;
        c_out[2 * k] = creal(s);
        c_out[2 * k + 1] = cimag(s);
    }
    free(ctab);
    free(f);
    return 0;
}

int oracle_coeffs(double a, double b, double dt, double tol, int kmax, double* C_out, int* M_out)
{
    if (!(a > 0.0) || kmax < 1) return -1;
    double z = a * dt;
    double* c = (double*)malloc(sizeof(double) * 2 * (size_t)(kmax + 1));
    if (!c) return -3;
    int rc = oracle_bessel_coeffs(z, kmax, c);
    if (rc) { free(c); return rc; }
    cplx phase = cexp(-I * b * dt);
    int M = 0;
    for (int k = 0; k <= kmax; ++k) {
        cplx ck = (c[2 * k] + I * c[2 * k + 1]) * (k == 0 ? 1.0 : 2.0) * phase;
        C_out[2 * k] = creal(ck);
        C_out[2 * k + 1] = cimag(ck);
        if (cabs(ck) >= tol) M = k;
    }
    free(c);
    if (M < 1) M = 1;
    *M_out = M;
    return (M == kmax) ? -4 : 0; /* -4: the cutoff was not reached below kmax */
}

/* ------------------------------------------------------------------------------------ */
/* Sparse operators as explicit CSR matrices (real symmetric H).                           */
/* ------------------------------------------------------------------------------------ */
typedef struct oracle_op {
    long n, nnz, cap;
    long* rowptr;
    long* col;
    double* val;
    /* Holstein bookkeeping (NULL for the lattices) */
    int hol_L, hol_nph;
    long hol_dph;
    unsigned char* hol_occ; /* [dph][L] phonon occupations in basis order */
} oracle_op;

static oracle_op* op_new(long n, long cap)
{
    oracle_op* H = (oracle_op*)calloc(1, sizeof(oracle_op));
    if (!H) return NULL;
    H->n = n;
    H->cap = cap > 0 ? cap : 1;
    H->rowptr = (long*)calloc((size_t)n + 1, sizeof(long));
    H->col = (long*)malloc(sizeof(long) * (size_t)H->cap);
    H->val = (double*)malloc(sizeof(double) * (size_t)H->cap);
    if (!H->rowptr || !H->col || !H->val) {
        free(H->rowptr); free(H->col); free(H->val); free(H);
        return NULL;
    }
    return H;
}

static void op_push(oracle_op* H, long col, double val)
{
    /* capacities are computed exactly by the builders; this never grows */
    H->col[H->nnz] = col;
    H->val[H->nnz] = val;
    H->nnz++;
}

void oracle_op_free(oracle_op* H)
{
    if (!H) return;
    free(H->rowptr); free(H->col); free(H->val); free(H->hol_occ);
    free(H);
}

long oracle_op_dim(const oracle_op* H) { return H->n; }
long oracle_op_nnz(const oracle_op* H) { return H->nnz; }

void oracle_op_export(const oracle_op* H, long* rowptr, long* col, double* val)
{
    memcpy(rowptr, H->rowptr, sizeof(long) * (size_t)(H->n + 1));
    memcpy(col, H->col, sizeof(long) * (size_t)H->nnz);
    memcpy(val, H->val, sizeof(double) * (size_t)H->nnz);
}

/* y = H x */
void oracle_op_apply(const oracle_op* H, const double* xin, double* yout)
{
    const cplx* x = (const cplx*)xin;
    cplx* y = (cplx*)yout;
    for (long i = 0; i < H->n; ++i) {
        cplx s = 0.0;
        for (long p = H->rowptr[i]; p < H->rowptr[i + 1]; ++p) s += H->val[p] * x[H->col[p]];
        y[i] = s;
    }
}

/* 1D grid, Sec. 3.1: H = -(1/2) d^2/dx^2 + V(x) (hbar = m = 1) with the 3-point stencil
   psi'' ~ (psi_{i-1} - 2 psi_i + psi_{i+1}) / dx^2 and psi = 0 outside the grid.          */
oracle_op* oracle_op_lattice1d(long n, double dx, const double* V)
{
    if (n < 1 || !(dx > 0.0)) return NULL;
    oracle_op* H = op_new(n, 3 * n);
    if (!H) return NULL;
    double kin = 1.0 / (dx * dx);
    for (long i = 0; i < n; ++i) {
        if (i > 0) op_push(H, i - 1, -0.5 * kin);
        op_push(H, i, kin + V[i]);
        if (i + 1 < n) op_push(H, i + 1, -0.5 * kin);
        H->rowptr[i + 1] = H->nnz;
    }
    return H;
}

/* Honeycomb ribbon, Sec. 3.2, Eq. (model): H = -t sum_<ij> (c_i^+ c_j + h.c.) + sum_j eps_j n_j.
   Brick-wall picture of the honeycomb lattice: site (r, c) with r in [0, W) across the ribbon
   and c in [0, L) along it, index r*L + c.  Its three neighbours are (r, c-1), (r, c+1) and
   (r+1, c) when r + c is even, (r-1, c) when r + c is odd.  Rows r are zigzag chains, so the
   edges r = 0 and r = W-1 are zigzag edges and the columns c = 0 and c = L-1 armchair edges:
   a ribbon with armchair edges along its length is the same lattice with the long direction
   across the rows (W = length, L = number of dimer lines).  periodic = 1 wraps both
   directions (a torus; needs W and L even), periodic = 2 wraps the rows only (an armchair
   ribbon made infinite along its length; needs W even); both serve only to check spectra
   against closed forms.                                                                     */
static long hc_index(int W, int L, int r, int c, int periodic)
{
    if (periodic == 1) {
        r = (r % W + W) % W;
        c = (c % L + L) % L;
    } else if (periodic == 2) {
        if (c < 0 || c >= L) return -1;
        r = (r % W + W) % W;
    } else if (r < 0 || r >= W || c < 0 || c >= L) {
        return -1;
    }
    return (long)r * L + c;
}

oracle_op* oracle_op_honeycomb(int W, int L, double t, const double* eps, int periodic)
{
    if (W < 1 || L < 1 || periodic < 0 || periodic > 2) return NULL;
    if (periodic == 1 && ((W % 2) || (L % 2) || W < 2 || L < 4)) return NULL;
    if (periodic == 2 && ((W % 2) || W < 4)) return NULL;
    long n = (long)W * L;
    oracle_op* H = op_new(n, 4 * n);
    if (!H) return NULL;
    for (int r = 0; r < W; ++r) {
        for (int c = 0; c < L; ++c) {
            long i = (long)r * L + c;
            int rv = ((r + c) % 2 == 0) ? r + 1 : r - 1;
            long nb[3] = {hc_index(W, L, r, c - 1, periodic), hc_index(W, L, r, c + 1, periodic),
                          hc_index(W, L, rv, c, periodic)};
            op_push(H, i, eps ? eps[i] : 0.0);
            for (int q = 0; q < 3; ++q)
                if (nb[q] >= 0) op_push(H, nb[q], -t);
            H->rowptr[i + 1] = H->nnz;
        }
    }
    return H;
}

/* Holstein chain, Sec. 3.3, Eq. (ghm), one spinless electron:
     H = sum_i Delta_i n_i - t sum_i (c_i^+ c_{i+1} + h.c.)
         - sum_i g_i omega0 (b_i^+ + b_i) n_i + omega0 sum_i b_i^+ b_i,
   in the basis |e; n_0 .. n_{L-1}> with n_0 + ... + n_{L-1} <= nph (the truncation of
   Sec. 3.3).  Basis order: index = e * Dph + rank(n), rank(n) the position of the tuple n in
   the lexicographically sorted list of all admissible tuples (n_0 most significant).  The
   oracle lists that set by brute force and finds ranks by binary search.
   periodic != 0 adds the bond (L-1, 0); it needs L >= 3 so that the two bonds of a site are
   distinct.  Delta and g may be NULL (zero and g_uniform).                                 */
static long hol_count(int L, int nph)
{
    /* number of tuples of L non-negative integers with sum <= nph, by enumeration */
    if (L == 0) return 1;
    long s = 0;
    for (int v = 0; v <= nph; ++v) s += hol_count(L - 1, nph - v);
    return s;
}

static void hol_fill(unsigned char* occ, int L, int nph, int pos, unsigned char* cur, long* row)
{
    if (pos == L) {
        memcpy(occ + (size_t)(*row) * L, cur, (size_t)L);
        (*row)++;
        return;
    }
    for (int v = 0; v <= nph; ++v) {
        cur[pos] = (unsigned char)v;
        hol_fill(occ, L, nph - v, pos + 1, cur, row);
    }
}

static long hol_find(const oracle_op* H, const unsigned char* key)
{
    long lo = 0, hi = H->hol_dph - 1;
    while (lo <= hi) {
        long mid = lo + (hi - lo) / 2;
        int c = memcmp(H->hol_occ + (size_t)mid * H->hol_L, key, (size_t)H->hol_L);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

oracle_op* oracle_op_holstein(int L, int nph, int periodic, double t, double omega0,
                              double g_uniform, const double* Delta, const double* g)
{
    if (L < 1 || nph < 0 || nph > 255 || (periodic && L < 3)) return NULL;
    long dph = hol_count(L, nph);
    long n = (long)L * dph;
    oracle_op* H = op_new(n, 5 * n);
    if (!H) return NULL;
    H->hol_L = L;
    H->hol_nph = nph;
    H->hol_dph = dph;
    H->hol_occ = (unsigned char*)malloc((size_t)dph * (size_t)L);
    unsigned char* cur = (unsigned char*)calloc((size_t)L, 1);
    unsigned char* key = (unsigned char*)calloc((size_t)L, 1);
    if (!H->hol_occ || !cur || !key) { free(cur); free(key); oracle_op_free(H); return NULL; }
    long row = 0;
    hol_fill(H->hol_occ, L, nph, 0, cur, &row);

    for (int e = 0; e < L; ++e) {
        double ge = g ? g[e] : g_uniform;
        for (long p = 0; p < dph; ++p) {
            long i = (long)e * dph + p;
            const unsigned char* occ = H->hol_occ + (size_t)p * L;
            int ntot = 0;
            for (int j = 0; j < L; ++j) ntot += occ[j];
            /* diagonal: Delta_e n_e + omega0 sum_j n_j */
            op_push(H, i, (Delta ? Delta[e] : 0.0) + omega0 * ntot);
            /* hopping: the electron moves to e-1 or e+1, phonons unchanged */
            int el = e - 1, er = e + 1;
            if (periodic) { el = (el + L) % L; er = er % L; }
            if (el >= 0) op_push(H, (long)el * dph + p, -t);
            if (er < L) op_push(H, (long)er * dph + p, -t);
            /* coupling at the electron site: b_e^+ raises n_e (sqrt(n_e+1)), b_e lowers it (sqrt(n_e)) */
            if (ntot < nph) {
                memcpy(key, occ, (size_t)L);
                key[e]++;
                long q = hol_find(H, key);
                op_push(H, (long)e * dph + q, -ge * omega0 * sqrt((double)occ[e] + 1.0));
            }
            if (occ[e] > 0) {
                memcpy(key, occ, (size_t)L);
                key[e]--;
                long q = hol_find(H, key);
                op_push(H, (long)e * dph + q, -ge * omega0 * sqrt((double)occ[e]));
            }
            H->rowptr[i + 1] = H->nnz;
        }
    }
    free(cur);
    free(key);
    return H;
}

long oracle_holstein_dim_phonon(const oracle_op* H) { return H->hol_dph; }

/* basis state of index idx: electron site and the L occupations */
int oracle_holstein_state(const oracle_op* H, long idx, int* e, unsigned char* occ)
{
    if (!H->hol_occ || idx < 0 || idx >= H->n) return -1;
    *e = (int)(idx / H->hol_dph);
    memcpy(occ, H->hol_occ + (size_t)(idx % H->hol_dph) * H->hol_L, (size_t)H->hol_L);
    return 0;
}

/* index of |e; occ>, -1 if the tuple is not in the truncated basis */
long oracle_holstein_index(const oracle_op* H, int e, const unsigned char* occ)
{
    if (!H->hol_occ || e < 0 || e >= H->hol_L) return -1;
    long q = hol_find(H, occ);
    return q < 0 ? -1 : (long)e * H->hol_dph + q;
}

/* Observables of Fig. 3 for a normalised state: dens[i] = <n_i>, phon[i] = <b_i^+ b_i>,
   chi[i] = <n_i (b_i + b_i^+)> (the coupling operator restricted to the truncated basis). */
int oracle_holstein_observables(const oracle_op* H, const double* psin, double* dens,
                                double* phon, double* chi)
{
    if (!H->hol_occ) return -1;
    const cplx* psi = (const cplx*)psin;
    int L = H->hol_L;
    unsigned char* key = (unsigned char*)malloc((size_t)L);
    if (!key) return -3;
    for (int i = 0; i < L; ++i) dens[i] = phon[i] = chi[i] = 0.0;
    for (long idx = 0; idx < H->n; ++idx) {
        int e = (int)(idx / H->hol_dph);
        const unsigned char* occ = H->hol_occ + (size_t)(idx % H->hol_dph) * L;
        double w = creal(psi[idx] * conj(psi[idx]));
        dens[e] += w;
        for (int i = 0; i < L; ++i) phon[i] += w * occ[i];
        /* <psi| n_e b_e^+ |psi> + c.c. : pair (idx) with the state one phonon higher at e */
        memcpy(key, occ, (size_t)L);
        key[e]++;
        long q = hol_find(H, key);
        if (q >= 0) {
            long up = (long)e * H->hol_dph + q;
            chi[e] += 2.0 * creal(conj(psi[up]) * psi[idx]) * sqrt((double)occ[e] + 1.0);
        }
    }
    free(key);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* One Chebyshev step, Sec. 2.2, Eqs. (U_1) and (rec):                                     */
/*   H~ = (H - b)/a;  v_0 = psi;  v_1 = H~ v_0;  v_{k+1} = 2 H~ v_k - v_{k-1};            */
/*   psi <- sum_{k=0}^{M} C_k v_k   with C_k = e^{-i b dt}(2 - delta_k0) c_k(a dt).        */
/* ------------------------------------------------------------------------------------ */
static void apply_scaled(const oracle_op* H, double a, double b, const cplx* x, cplx* y)
{
    oracle_op_apply(H, (const double*)x, (double*)y);
    for (long i = 0; i < H->n; ++i) y[i] = (y[i] - b * x[i]) / a;
}

int oracle_cheb_step(const oracle_op* H, double a, double b, const double* Cin, int M,
                     double* psin)
{
    if (M < 1 || !(a > 0.0)) return -1;
    long n = H->n;
    const cplx* C = (const cplx*)Cin;
    cplx* psi = (cplx*)psin;
    cplx* vprev = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* vcur = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* vnext = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    if (!vprev || !vcur || !vnext || !out) { free(vprev); free(vcur); free(vnext); free(out); return -3; }
    memcpy(vprev, psi, sizeof(cplx) * (size_t)n);          /* v_0 */
    apply_scaled(H, a, b, vprev, vcur);                      /* v_1 = H~ v_0 */
    for (long i = 0; i < n; ++i) out[i] = C[0] * vprev[i] + C[1] * vcur[i];
    for (int k = 1; k < M; ++k) {
        apply_scaled(H, a, b, vcur, vnext);                  /* H~ v_k */
        for (long i = 0; i < n; ++i) vnext[i] = 2.0 * vnext[i] - vprev[i];   /* v_{k+1} */
        for (long i = 0; i < n; ++i) out[i] += C[k + 1] * vnext[i];
        cplx* tmp = vprev; vprev = vcur; vcur = vnext; vnext = tmp;
    }
    memcpy(psi, out, sizeof(cplx) * (size_t)n);
    free(vprev); free(vcur); free(vnext); free(out);
    return 0;
}

/* nsteps Chebyshev steps in place; the multi-vector form evolves nvec vectors stored
   [site][vec] (each one independently, one after the other). */
int oracle_cheb_evolve(const oracle_op* H, double a, double b, const double* C, int M,
                       int nsteps, double* psin)
{
    for (int s = 0; s < nsteps; ++s) {
        int rc = oracle_cheb_step(H, a, b, C, M, psin);
        if (rc) return rc;
    }
    return 0;
}

/* <psi|psi> and <psi|H|psi> */
void oracle_norm_energy(const oracle_op* H, const double* psin, double* norm2, double* energy)
{
    const cplx* psi = (const cplx*)psin;
    cplx* y = (cplx*)malloc(sizeof(cplx) * (size_t)H->n);
    oracle_op_apply(H, psin, (double*)y);
    double nn = 0.0;
    cplx e = 0.0;
    for (long i = 0; i < H->n; ++i) {
        nn += creal(conj(psi[i]) * psi[i]);
        e += conj(psi[i]) * y[i];
    }
    *norm2 = nn;
    *energy = creal(e);
    free(y);
}

/* ------------------------------------------------------------------------------------ */
/* Gradient of P = psi_n^+ Pi psi_n, psi_{s+1} = U psi_s (U from Eq. (U_1), a and b fixed),  */
/* with respect to the diagonal entries V_i of H (dH~/dV_i = e_i e_i^T / a).                */
/* No counterpart in the paper: this is reverse-mode differentiation of Eqs. (U_1), (rec).  */
/* Convention: for real P, xbar = dP/d(conj x), so dP = 2 Re(xbar^+ dx).                    */
/*   lambda_n = Pi psi_n;  for each step s = n-1 .. 0 (forward vectors v_k of that step):   */
/*     vbar_k = conj(C_k) lambda_{s+1}                  for k = 0..M                        */
/*     for k = M-1 .. 1:  vbar_k += 2 H~ vbar_{k+1};  vbar_{k-1} -= vbar_{k+1};             */
/*                        grad_i += (4/a) Re(conj(vbar_{k+1,i}) v_{k,i})                    */
/*     vbar_0 += H~ vbar_1;  grad_i += (2/a) Re(conj(vbar_{1,i}) v_{0,i})                   */
/*     lambda_s = vbar_0.                                                                    */
/* The oracle keeps every psi_s and every v_k of the step being reversed.                   */
/* mask[i] != 0 marks the sites of the region Pi.  lambda0 (optional) receives lambda_0.    */
/* ------------------------------------------------------------------------------------ */
int oracle_adjoint_region(const oracle_op* H, double a, double b, const double* Cin, int M,
                          int nsteps, const double* psi0, const unsigned char* mask,
                          double* grad, double* P_out, double* lambda0)
{
    if (M < 1 || nsteps < 0) return -1;
    long n = H->n;
    const cplx* C = (const cplx*)Cin;
    cplx* traj = (cplx*)malloc(sizeof(cplx) * (size_t)n * (size_t)(nsteps + 1));
    cplx* v = (cplx*)malloc(sizeof(cplx) * (size_t)n * (size_t)(M + 1));
    cplx* vbar = (cplx*)malloc(sizeof(cplx) * (size_t)n * (size_t)(M + 1));
    cplx* lam = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    if (!traj || !v || !vbar || !lam || !tmp) {
        free(traj); free(v); free(vbar); free(lam); free(tmp);
        return -3;
    }
    memcpy(traj, psi0, sizeof(cplx) * (size_t)n);
    for (int s = 0; s < nsteps; ++s) {
        memcpy(traj + (size_t)(s + 1) * n, traj + (size_t)s * n, sizeof(cplx) * (size_t)n);
        int rc = oracle_cheb_step(H, a, b, Cin, M, (double*)(traj + (size_t)(s + 1) * n));
        if (rc) { free(traj); free(v); free(vbar); free(lam); free(tmp); return rc; }
    }
    const cplx* psin = traj + (size_t)nsteps * n;
    double P = 0.0;
    for (long i = 0; i < n; ++i) {
        lam[i] = mask[i] ? psin[i] : 0.0;
        P += mask[i] ? creal(conj(psin[i]) * psin[i]) : 0.0;
        grad[i] = 0.0;
    }
    *P_out = P;
    for (int s = nsteps - 1; s >= 0; --s) {
        /* forward vectors of step s */
        memcpy(v, traj + (size_t)s * n, sizeof(cplx) * (size_t)n);
        apply_scaled(H, a, b, v, v + n);
        for (int k = 1; k < M; ++k) {
            apply_scaled(H, a, b, v + (size_t)k * n, v + (size_t)(k + 1) * n);
            for (long i = 0; i < n; ++i)
                v[(size_t)(k + 1) * n + i] = 2.0 * v[(size_t)(k + 1) * n + i] - v[(size_t)(k - 1) * n + i];
        }
        /* reverse sweep */
        for (int k = 0; k <= M; ++k)
            for (long i = 0; i < n; ++i) vbar[(size_t)k * n + i] = conj(C[k]) * lam[i];
        for (int k = M - 1; k >= 1; --k) {
            cplx* vb1 = vbar + (size_t)(k + 1) * n;
            apply_scaled(H, a, b, vb1, tmp);
            for (long i = 0; i < n; ++i) {
                vbar[(size_t)k * n + i] += 2.0 * tmp[i];
                vbar[(size_t)(k - 1) * n + i] -= vb1[i];
                grad[i] += (4.0 / a) * creal(conj(vb1[i]) * v[(size_t)k * n + i]);
            }
        }
        apply_scaled(H, a, b, vbar + n, tmp);
        for (long i = 0; i < n; ++i) {
            vbar[i] += tmp[i];
            grad[i] += (2.0 / a) * creal(conj(vbar[n + i]) * v[i]);
        }
        memcpy(lam, vbar, sizeof(cplx) * (size_t)n);
    }
    if (lambda0) memcpy(lambda0, lam, sizeof(cplx) * (size_t)n);
    free(traj); free(v); free(vbar); free(lam); free(tmp);
    return 0;
}
