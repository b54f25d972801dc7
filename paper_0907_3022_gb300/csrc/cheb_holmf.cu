// Matrix-free Holstein operator (Sec. 3.3): the fused recurrence of Eq. rec with the matrix
// elements of Eq. ghm recomputed from the basis indices in every launch instead of read from
// a stored matrix, as the paper does for its 18-site chain.
//
// Rows are e * Dph + r (electron site e, phonon rank r).  One thread takes one phonon
// configuration r (and one vector) for all L electron sites: it unranks r once and walks
// e = L-1 .. 0 with HolWalk, which yields the ranks of n +- 1_e.  Electron hops keep r,
// so the hop terms of row (e, r) are the values the thread loaded for rows (e +- 1, r): every
// element of T_j is read once, plus the two phonon gathers T_j[e Dph + rank(n +- 1_e)], which
// stay inside the slab of electron site e.  Per row and order the launch moves T_j, T_{j-1}
// and T_{j+1}, and every third launch the accumulator (read and write, see AccGroup): no
// matrix and no stored diagonal (complex64: 24 + 16/3 bytes per row and order).
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
    const int2* G;        // [(L + 1)(nph + 1)], see HolG
    const void* dtab;     // R [L][nph + 1]: 2 (Delta_e + w0 s - b)/a, s = total phonon number
    const void* qtab;     // R [L][nph + 1]: 2 (-g_e w0 sqrt(m))/a
    uint32_t tile_units;  // (phonon configuration, vector) pairs per tile
    int32_t ntiles;
    int32_t log2_nvec;
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

// One launch of the recurrence for the mode MODE (REC_FIRST / REC_SECOND / REC_GENERAL);
// each thread advances NR phonon configurations in lockstep (NR = 2 doubles the loads in
// flight per thread).  MINB > 1 caps the registers so that MINB blocks of 256 threads fit
// on an SM (more warps to hide the gather latency; launches then use <= 256 threads).
// LT > 0 compiles the walk over the electron sites for a chain of exactly LT sites (the
// 12-site configuration and the paper's 18 sites): offsets and site tests become constants.
template <typename R, int MODE, int NR, int MINB, int LT>
__global__ void __launch_bounds__(MINB > 1 ? 256 : 512, MINB) k_rec_holmf(RecArgs a, HolMFArgs m)
{
    using C = typename V2<R>::C;
    using U = SiteUpdate<R>;
    constexpr bool FIRST = (MODE == REC_FIRST);
    constexpr bool SECOND = (MODE == REC_SECOND);
    __shared__ int2 sG[(HOLMF_MAX_L + 1) * (HOLMF_MAX_NPH + 1)];
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
    const int nv = a.nvec, lnv = m.log2_nvec;
    const int L = LT > 0 ? LT : m.L, nph = m.nph;  // LT > 0: chain length fixed at compile time
    const bool periodic = m.periodic != 0;
    // element offsets fit 32 bits (rows * nvec < 2^32 is checked at plan creation)
    const uint32_t units = (uint32_t)m.dph << lnv;
    const uint32_t es = units;  // distance between the rows of neighbouring electron sites
    const C* __restrict__ cur = static_cast<const C*>(a.cur);
    C* __restrict__ prev = static_cast<C*>(a.prev);
    C* __restrict__ out1 = static_cast<C*>(a.out1);
    C* __restrict__ psi = static_cast<C*>(a.psi);
    C* __restrict__ tail = static_cast<C*>(a.tail);
    const C* __restrict__ qc = static_cast<const C*>(a.qcoef);
    const DevBlock B = a.blocks[0];
    const int k = a.j + 1;
    const bool store = !m.energy_only;
    const R beta = (R)B.beta;
    const C zero = V2<R>::make(0, 0);
    const AccGroup ag(FIRST ? 1 : k, B.M, B.ksplit);
    C qm2 = zero, qm1 = zero, qk = zero, ph = zero, pl = zero;
    if (!FIRST) {
        qk = qc[B.coef_off + k];
        if (ag.n >= 2) qm1 = qc[B.coef_off + k - 1];
        if (ag.n >= 3) qm2 = qc[B.coef_off + k - 2];
        split_const<R>(B.ph_re, ph.x, pl.x);
        split_const<R>(B.ph_im, ph.y, pl.y);
    }
    C* __restrict__ accp = ag.to_tail ? tail : psi;
    for (int t = blockIdx.x; t < m.ntiles; t += gridDim.x) {
        R part0 = 0, part1 = 0;
        double dpart0 = 0.0, dpart1 = 0.0;  // energy-only launches (observables): FP64 terms
        const uint32_t ub = (uint32_t)t * m.tile_units;
        const uint32_t u1 = min(ub + m.tile_units, units);
        for (uint32_t u0 = ub + threadIdx.x; u0 < u1; u0 += NR * blockDim.x) {
            // unit u = r * nvec + v is also the offset of element (e = 0, r, v)
            HolWalk W[NR];
            uint32_t col[NR];
            bool ok[NR];
            C xr[NR], xc[NR], xlast[NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const uint32_t u = u0 + i * blockDim.x;
                ok[i] = u < u1;
                col[i] = ok[i] ? u : u0;  // a missing configuration repeats the first, unstored
                W[i].begin(G, L, nph, (int32_t)(col[i] >> lnv));
                xlast[i] = cur[(uint32_t)(L - 1) * es + col[i]];
                xr[i] = periodic ? cur[col[i]] : zero;  // T_j at e + 1 (e = L-1: site 0)
                xc[i] = xlast[i];                        // T_j at e
            }
#pragma unroll (LT > 0 ? LT : 1)
            for (int e = L - 1; e >= 0; --e) {
                C xl[NR], p[NR], acc[NR], ps[NR], xu[NR], xd[NR];
                int ne[NR];
                // every load of this electron site first
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    int32_t up, dn;
                    ne[i] = W[i].step(G, L, nph, e, up, dn);
                    const uint32_t base = (uint32_t)e * es + col[i];
                    xl[i] = (e > 0) ? cur[base - es] : (periodic ? xlast[i] : zero);
                    p[i] = FIRST ? zero : (SECOND ? psi[base] : prev[base]);  // T_{k-2}
                    acc[i] = ag.read_acc ? accp[base] : zero;
                    ps[i] = ag.read_psi_last ? psi[base] : zero;
                    xu[i] = up ? cur[base + ((uint32_t)up << lnv)] : zero;
                    xd[i] = dn ? cur[base - ((uint32_t)dn << lnv)] : zero;
                    if (!up) ne[i] |= 1 << 8;  // flags: no raising / no lowering term
                    if (!dn) ne[i] |= 1 << 9;
                }
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    const uint32_t base = (uint32_t)e * es + col[i];
                    const int n_e = ne[i] & 255;
                    // h = 2 H~ x - p, terms in the stored-row order
                    C h = V2<R>::make(-p[i].x, -p[i].y);
                    if (e > 0 || periodic) {
                        h.x = fma(beta, xl[i].x, h.x);
                        h.y = fma(beta, xl[i].y, h.y);
                    }
                    if (e + 1 < L || periodic) {
                        h.x = fma(beta, xr[i].x, h.x);
                        h.y = fma(beta, xr[i].y, h.y);
                    }
                    if (!(ne[i] & (1 << 8))) {
                        const R qv = sQ[e * w + n_e + 1];
                        h.x = fma(qv, xu[i].x, h.x);
                        h.y = fma(qv, xu[i].y, h.y);
                    }
                    if (!(ne[i] & (1 << 9))) {
                        const R qv = sQ[e * w + n_e];
                        h.x = fma(qv, xd[i].x, h.x);
                        h.y = fma(qv, xd[i].y, h.y);
                    }
                    const R d = sD[e * w + W[i].ntot];
                    h.x = fma(d, xc[i].x, h.x);
                    h.y = fma(d, xc[i].y, h.y);
                    if (FIRST) {
                        const C t1 = V2<R>::make((R)0.5 * h.x, (R)0.5 * h.y);
                        if (ok[i] && store) {
                            part0 = fma(xc[i].x, xc[i].x, fma(xc[i].y, xc[i].y, part0));
                            part1 = fma(xc[i].x, t1.x, fma(xc[i].y, t1.y, part1));
                            out1[base] = t1;
                        } else if (ok[i]) {
                            // energy of psi for cheb_observables: the row of 2 H~ psi in the
                            // vector precision, its products and sums with psi in FP64
                            dpart0 += (double)xc[i].x * xc[i].x + (double)xc[i].y * xc[i].y;
                            dpart1 += (double)xc[i].x * t1.x + (double)xc[i].y * t1.y;
                        }
                    } else if (ok[i]) {
                        prev[base] = h;  // T_k over T_{k-2}
                        if (ag.upd) {
                            C ac = acc[i];
                            if (ag.n >= 3) U::accum(ac, qm2, p[i], k - 2);
                            if (ag.n >= 2) U::accum(ac, qm1, xc[i], k - 1);
                            U::accum(ac, qk, h, k);
                            if (ag.last) {
                                if (ag.read_psi_last) ac = V2<R>::make(ps[i].x + ac.x, ps[i].y + ac.y);
                                ac = U::phase(ac, ph, pl);
                                // growth check |T_M|^2 <= 4 ||psi||^2 in the vector precision
                                const R t2 = fma(h.x, h.x, h.y * h.y);
                                const int v = (int)(col[i] & (nv - 1));
                                if (!(t2 <= (R)(4.0 * a.norm2[(size_t)v * 2]))) atomicOr(a.errflag, 1);
                                psi[base] = ac;
                            } else {
                                accp[base] = ac;
                            }
                        }
                    }
                    xr[i] = xc[i];
                    xc[i] = xl[i];
                }
            }
        }
        if (FIRST) {
            if (!store || !Split<R>::on) {  // FP64 tree
                double dpart[2] = {store ? (double)part0 : dpart0, store ? (double)part1 : dpart1};
                block_reduce_groups<2>(dpart, nv, s_red, a.partials + (size_t)t * nv * 2);
            } else {  // complex64 recurrence (divergence-check norm): FP32 warp tree, FP64 block sum
                float fpart[2] = {(float)part0, (float)part1};
                block_reduce_groups_f<2>(fpart, nv, s_red, a.partials + (size_t)t * nv * 2);
            }
        }
    }
    if (FIRST) holmf_finalize(a, m, B, s_red);
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
    std::vector<int2> g;
    make_hol_g(L, nph, tab, g);
    CHEB_CUDA(cudaMalloc(&p->d_holmf_G, g.size() * sizeof(int2)));
    CHEB_CUDA(cudaMemcpy(p->d_holmf_G, g.data(), g.size() * sizeof(int2), cudaMemcpyHostToDevice));
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

template <typename R, int NR, int MINB, int LT>
static void launch_lt(const RecArgs& a, const HolMFArgs& m, int grid, int th, cudaStream_t s)
{
    if (a.mode == REC_FIRST) k_rec_holmf<R, REC_FIRST, NR, MINB, LT><<<grid, th, 0, s>>>(a, m);
    else if (a.mode == REC_SECOND) k_rec_holmf<R, REC_SECOND, NR, MINB, LT><<<grid, th, 0, s>>>(a, m);
    else k_rec_holmf<R, REC_GENERAL, NR, MINB, LT><<<grid, th, 0, s>>>(a, m);
}

template <typename R, int NR, int MINB>
static void launch_nr(const RecArgs& a, const HolMFArgs& m, int grid, int th, cudaStream_t s)
{
    if constexpr (NR == 1) {
        if (m.L == 12) return launch_lt<R, NR, MINB, 12>(a, m, grid, th, s);
        if (m.L == 18) return launch_lt<R, NR, MINB, 18>(a, m, grid, th, s);
    }
    launch_lt<R, NR, MINB, 0>(a, m, grid, th, s);
}

// variants: 0 = one configuration per thread, 1 = the same with 5 blocks of 256 threads
// per SM, 2 = two configurations per thread
template <typename R>
static void launch_modes(const RecArgs& a, const HolMFArgs& m, int variant, int grid, int th,
                         cudaStream_t s)
{
    if (variant == 2) launch_nr<R, 2, 1>(a, m, grid, th, s);
    else if (variant == 1) launch_nr<R, 1, 5>(a, m, grid, th, s);
    else launch_nr<R, 1, 1>(a, m, grid, th, s);
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
    m.tile_units = (uint32_t)(th * std::max(1, p->spt));
    const int64_t units = p->hol_dph * p->nvec;
    const int64_t ntiles = (units + m.tile_units - 1) / m.tile_units;
    if ((size_t)ntiles * p->nvec * 2 > p->holmf_partials_cap || ntiles > INT32_MAX)
        return fail(CHEB_ERR_INVALID, "matrix-free Holstein: tile count exceeds the partials buffer");
    m.ntiles = (int32_t)ntiles;
    m.energy_out = energy_out;
    m.log2_nvec = 0;
    while ((1 << m.log2_nvec) < p->nvec) ++m.log2_nvec;
    RecArgs a = a0;
    a.partials = p->d_holmf_partials;
    int grid = (int)ntiles;
    if (p->grid_cap > 0 && grid > p->grid_cap) grid = p->grid_cap;
    const int variant = p->holmf_variant;
    if (variant == 1 && th > 256)
        return fail(CHEB_ERR_INVALID, "matrix-free Holstein: variant 1 needs <= 256 threads");
    if (p->prec == CHEB_C128) launch_modes<double>(a, m, variant, grid, th, s);
    else launch_modes<float>(a, m, variant, grid, th, s);
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
