// Matrix-free Holstein operator (Sec. 3.3): the fused recurrence of Eq. rec with the matrix
// elements of Eq. ghm recomputed from the basis indices in every launch instead of read from
// a stored matrix, as the paper does for its 18-site chain.
//
// Rows are e * Dph + r (electron site e, phonon rank r).  One thread takes one phonon
// configuration r (and one vector) for all L electron sites: it unranks r once and walks
// e = L-1 .. 0 with hol_phonon_walk, which yields the ranks of n +- 1_e.  Electron hops keep r,
// so the hop terms of row (e, r) are the values the thread loaded for rows (e +- 1, r): every
// element of T_j is read once, plus the two phonon gathers T_j[e Dph + rank(n +- 1_e)], which
// stay inside the slab of electron site e.  Per row and order the launch moves
// T_j, T_{j-1}, T_{j+1} and the accumulator (read and write) and nothing else: no matrix, no
// stored diagonal (complex64: 40 bytes per row instead of about 70 with the SELL matrix).
//
// The sums are formed in the order of the stored rows (hop to e-1, hop to e+1, phonon up,
// phonon down, then the diagonal) with the same scaled values, so the stored and the
// matrix-free operators give the same T_{j+1}.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "cheb_device.cuh"
#include "cheb_holstein.cuh"
#include "cheb_internal.cuh"

namespace cheb {

struct HolMFArgs {
    int32_t L, nph, periodic, energy_only;
    int64_t dph;
    const int32_t* G;     // [(L + 1)(nph + 1)], see HolG
    const void* dtab;     // R [L][nph + 1]: 2 (Delta_e + w0 s - b)/a, s = total phonon number
    const void* qtab;     // R [L][nph + 1]: 2 (-g_e w0 sqrt(m))/a
    int64_t tile_units;   // (phonon configuration, vector) pairs per tile
    int32_t ntiles;
    double* energy_out;   // energy_only: <psi|H|psi> per vector
};

// Last CTA: sum the per-tile partials (threads stride over tiles, then a fixed-order block
// tree) and write (||psi||^2, <psi|H|psi>) per vector, or the energy alone.
__device__ void holmf_finalize(const RecArgs& a, const HolMFArgs& m, const DevBlock& B,
                               double* smem)
{
    __shared__ unsigned int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(a.done_counter, 1u);
        s_last = (t == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nv = a.nvec;
    for (int v = 0; v < nv; ++v) {
        double val[2] = {0.0, 0.0};
        for (int t = threadIdx.x; t < m.ntiles; t += blockDim.x) {
            val[0] += __ldcg(a.partials + ((size_t)t * nv + v) * 2 + 0);
            val[1] += __ldcg(a.partials + ((size_t)t * nv + v) * 2 + 1);
        }
        block_reduce_groups<2>(val, 1, smem, smem + 1024);  // totals in smem[1024..1025]
        if (threadIdx.x == 0) {
            const double n2 = smem[1024], eh = smem[1025];
            const double E = B.a * eh + B.b * n2;  // <H> = a <H~> + b ||psi||^2
            if (m.energy_out) {
                m.energy_out[v] = E;
            } else {
                a.red_out[(size_t)v * 2 + 0] = n2;
                a.red_out[(size_t)v * 2 + 1] = E;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *a.done_counter = 0u;
}

template <typename R>
__global__ void __launch_bounds__(512) k_rec_holmf(RecArgs a, HolMFArgs m)
{
    using C = typename V2<R>::C;
    using U = SiteUpdate<R>;
    __shared__ int32_t sG[(HOLMF_MAX_L + 1) * (HOLMF_MAX_NPH + 1)];
    __shared__ R sD[HOLMF_MAX_L * (HOLMF_MAX_NPH + 1)];
    __shared__ R sQ[HOLMF_MAX_L * (HOLMF_MAX_NPH + 1)];
    __shared__ double s_red[16 * 32 * 2 + 2];
    const int w = m.nph + 1;
    for (int i = threadIdx.x; i < (m.L + 1) * w; i += blockDim.x) sG[i] = m.G[i];
    for (int i = threadIdx.x; i < m.L * w; i += blockDim.x) {
        sD[i] = static_cast<const R*>(m.dtab)[i];
        sQ[i] = static_cast<const R*>(m.qtab)[i];
    }
    __syncthreads();
    const HolG G{sG, w};
    const int nv = a.nvec;
    const int L = m.L, nph = m.nph;
    const bool periodic = m.periodic != 0;
    const int64_t es = m.dph * nv;  // distance between the rows of neighbouring electron sites
    const C* __restrict__ cur = static_cast<const C*>(a.cur);
    C* __restrict__ prev = static_cast<C*>(a.prev);
    C* __restrict__ out1 = static_cast<C*>(a.out1);
    C* __restrict__ psi = static_cast<C*>(a.psi);
    C* __restrict__ tail = static_cast<C*>(a.tail);
    const C* __restrict__ qc = static_cast<const C*>(a.qcoef);
    const DevBlock B = a.blocks[0];
    const int k = a.j + 1;
    const bool first = (a.mode == REC_FIRST);
    const bool store = !m.energy_only;
    const R beta = (R)B.beta;
    const C zero = V2<R>::make(0, 0);
    C qk = zero, q0 = zero, q1 = zero, ph = zero, pl = zero;
    bool last = false, to_tail = false, read_psi = false, read_tail = false, read_psi_last = false;
    if (!first) {
        qk = qc[B.coef_off + k];
        if (a.mode == REC_SECOND) {
            q0 = qc[B.coef_off + 0];
            q1 = qc[B.coef_off + 1];
        }
        last = (k == B.M);
        split_const<R>(B.ph_re, ph.x, pl.x);
        split_const<R>(B.ph_im, ph.y, pl.y);
        to_tail = k > B.ksplit;
        const bool gen = (a.mode == REC_GENERAL);
        read_psi = gen && !to_tail;
        read_tail = gen && to_tail && (k > B.ksplit + 1);
        read_psi_last = last && to_tail;
    }
    const int64_t units = m.dph * nv;
    for (int t = blockIdx.x; t < m.ntiles; t += gridDim.x) {
        R part0 = 0, part1 = 0;
        const int64_t u1 = min((int64_t)(t + 1) * m.tile_units, units);
        for (int64_t u = (int64_t)t * m.tile_units + threadIdx.x; u < u1; u += blockDim.x) {
            const int64_t r = u / nv;
            const int v = (int)(u - r * nv);
            uint64_t lo, hi;
            const int ntot = hol_unrank_packed(G, L, nph, r, lo, hi);
            const int64_t col = r * nv + v;  // element (e, r, v) at e * es + col
            const C xlast = cur[(int64_t)(L - 1) * es + col];
            C xr = periodic ? cur[col] : zero;  // T_j at e + 1 (e = L-1: site 0 if periodic)
            C xc = xlast;                        // T_j at e
            hol_phonon_walk(G, L, nph, lo, hi, ntot, [&](int e, int ne, int64_t up, int64_t dn) {
                const int64_t base = (int64_t)e * es + col;
                C xl = zero;  // T_j at e - 1 (e = 0: site L-1 if periodic)
                if (e > 0) xl = cur[base - es];
                else if (periodic) xl = xlast;
                C p = zero, acc = zero, ps = zero, xu = zero, xd = zero;
                if (!first) p = prev[base];
                if (read_psi) acc = psi[base];
                else if (read_tail) acc = tail[base];
                if (read_psi_last) ps = psi[base];
                if (up) xu = cur[base + up * nv];
                if (dn) xd = cur[base - dn * nv];
                // h = 2 H~ x - p, terms in the stored-row order
                C h = V2<R>::make(-p.x, -p.y);
                if (e > 0 || periodic) {
                    h.x = fma(beta, xl.x, h.x);
                    h.y = fma(beta, xl.y, h.y);
                }
                if (e + 1 < L || periodic) {
                    h.x = fma(beta, xr.x, h.x);
                    h.y = fma(beta, xr.y, h.y);
                }
                if (up) {
                    const R qv = sQ[e * w + ne + 1];
                    h.x = fma(qv, xu.x, h.x);
                    h.y = fma(qv, xu.y, h.y);
                }
                if (dn) {
                    const R qv = sQ[e * w + ne];
                    h.x = fma(qv, xd.x, h.x);
                    h.y = fma(qv, xd.y, h.y);
                }
                const R d = sD[e * w + ntot];
                h.x = fma(d, xc.x, h.x);
                h.y = fma(d, xc.y, h.y);
                if (first) {
                    const C t1 = V2<R>::make((R)0.5 * h.x, (R)0.5 * h.y);
                    part0 = fma(xc.x, xc.x, fma(xc.y, xc.y, part0));
                    part1 = fma(xc.x, t1.x, fma(xc.y, t1.y, part1));
                    if (store) {
                        prev[base] = xc;
                        out1[base] = t1;
                    }
                } else {
                    prev[base] = h;  // T_{j+1} over T_{j-1}
                    if (a.mode == REC_SECOND) {
                        U::accum(acc, q0, p, 0);
                        U::accum(acc, q1, xc, 1);
                        U::accum(acc, qk, h, 2);
                    } else {
                        U::accum(acc, qk, h, k);
                    }
                    if (last) {
                        if (read_psi_last) acc = V2<R>::make(ps.x + acc.x, ps.y + acc.y);
                        acc = U::phase(acc, ph, pl);
                        const double t2 = (double)h.x * h.x + (double)h.y * h.y;
                        if (!(t2 <= 4.0 * a.norm2[(size_t)v * 2])) atomicOr(a.errflag, 1);
                        psi[base] = acc;
                    } else {
                        (to_tail ? tail : psi)[base] = acc;
                    }
                }
                xr = xc;
                xc = xl;
            });
        }
        if (first) {
            double dpart[2] = {(double)part0, (double)part1};
            block_reduce_groups<2>(dpart, nv, s_red, a.partials + (size_t)t * nv * 2);
        }
    }
    if (first) holmf_finalize(a, m, B, s_red);
}

// scaled tables from the same matrix elements as the stored rows
template <typename R>
__global__ void k_holmf_tables(HolParams P, double a, double b, R* dtab, R* qtab)
{
    const int w = P.nph + 1;
    for (int i = threadIdx.x; i < P.L * w; i += blockDim.x) {
        const int e = i / w, s = i % w;
        dtab[i] = (R)(2.0 * (hol_diag_value(P, e, s) - b) / a);
        qtab[i] = (R)(2.0 * hol_phonon_value(P, e, s) / a);
    }
}

int holmf_build(Plan* p)
{
    const cheb_ham_desc& h = p->desc;
    const int L = h.hol_sites, nph = h.hol_nph;
    std::vector<int64_t> tab;
    if (!make_binom(L, nph, tab)) return fail(CHEB_ERR_INVALID, "Holstein basis too large");
    // the binomial table also serves the observables (unranking of the phonon tuples)
    CHEB_CUDA(cudaMalloc(&p->d_binom, tab.size() * sizeof(int64_t)));
    CHEB_CUDA(cudaMemcpy(p->d_binom, tab.data(), tab.size() * sizeof(int64_t),
                         cudaMemcpyHostToDevice));
    std::vector<int32_t> g;
    make_hol_g(L, nph, tab, g);
    CHEB_CUDA(cudaMalloc(&p->d_holmf_G, g.size() * sizeof(int32_t)));
    CHEB_CUDA(cudaMemcpy(p->d_holmf_G, g.data(), g.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    const size_t nt = (size_t)L * (nph + 1);
    CHEB_CUDA(cudaMalloc(&p->d_holmf_dtab, nt * p->real_size()));
    CHEB_CUDA(cudaMalloc(&p->d_holmf_qtab, nt * p->real_size()));
    HolParams P{};
    P.L = L;
    P.nph = nph;
    P.periodic = h.hol_periodic;
    P.dph = p->hol_dph;
    P.n = p->n_sites;
    P.t = h.hop;
    P.omega0 = h.omega0;
    P.g = h.g;
    P.delta = h.onsite;
    P.gsite = h.hol_g;
    const DevBlock& B = p->hblocks[0];
    if (p->prec == CHEB_C128)
        k_holmf_tables<double><<<1, 256, 0, p->stream>>>(P, B.a, B.b,
                                                         static_cast<double*>(p->d_holmf_dtab),
                                                         static_cast<double*>(p->d_holmf_qtab));
    else
        k_holmf_tables<float><<<1, 256, 0, p->stream>>>(P, B.a, B.b,
                                                        static_cast<float*>(p->d_holmf_dtab),
                                                        static_cast<float*>(p->d_holmf_qtab));
    p->launches++;
    CHEB_CUDA(cudaGetLastError());
    // partials for the smallest tile (128 threads, one unit each)
    const int64_t units = p->hol_dph * p->nvec;
    const size_t need = (size_t)((units + 127) / 128) * p->nvec * 2;
    CHEB_CUDA(cudaMalloc(&p->d_holmf_partials, need * sizeof(double)));
    p->holmf_partials_cap = need;
    CHEB_CUDA(cudaStreamSynchronize(p->stream));
    return CHEB_OK;
}

static int holmf_launch(Plan* p, const RecArgs& a0, double* energy_out, cudaStream_t s)
{
    HolMFArgs m{};
    m.L = p->desc.hol_sites;
    m.nph = p->desc.hol_nph;
    m.periodic = p->desc.hol_periodic;
    m.energy_only = energy_out ? 1 : 0;
    m.dph = p->hol_dph;
    m.G = p->d_holmf_G;
    m.dtab = p->d_holmf_dtab;
    m.qtab = p->d_holmf_qtab;
    const int th = p->threads;
    m.tile_units = (int64_t)th * std::max(1, p->spt);
    const int64_t units = p->hol_dph * p->nvec;
    const int64_t ntiles = (units + m.tile_units - 1) / m.tile_units;
    if ((size_t)ntiles * p->nvec * 2 > p->holmf_partials_cap || ntiles > INT32_MAX)
        return fail(CHEB_ERR_INVALID, "matrix-free Holstein: tile count exceeds the partials buffer");
    m.ntiles = (int32_t)ntiles;
    m.energy_out = energy_out;
    RecArgs a = a0;
    a.partials = p->d_holmf_partials;
    int grid = (int)ntiles;
    if (p->grid_cap > 0 && grid > p->grid_cap) grid = p->grid_cap;
    if (p->prec == CHEB_C128)
        k_rec_holmf<double><<<grid, th, 0, s>>>(a, m);
    else
        k_rec_holmf<float><<<grid, th, 0, s>>>(a, m);
    p->launches++;
    CHEB_CUDA(cudaGetLastError());
    return CHEB_OK;
}

int launch_holmf(Plan* p, const RecArgs& a, cudaStream_t s) { return holmf_launch(p, a, nullptr, s); }

// <psi|H|psi> per vector through the matrix-free operator (FIRST-mode sums, nothing stored)
int launch_holmf_energy(Plan* p, const void* psi, double* out, cudaStream_t s)
{
    RecArgs a{};
    a.nvec = p->nvec;
    a.blocks = p->d_blocks;
    a.mode = REC_FIRST;
    a.j = 0;
    a.cur = psi;
    a.done_counter = p->d_counter;
    a.red_out = nullptr;
    a.errflag = p->d_err;
    return holmf_launch(p, a, out, s);
}

}  // namespace cheb
