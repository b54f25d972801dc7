// Holstein chain in a truncated phonon basis (Sec. 3.3, Eq. ghm): basis ranking, on-device
// SELL-C construction of H, and the observables of Fig. 3.
//
// Basis: |e; n_0 .. n_{L-1}> with n_0 + ... + n_{L-1} <= nph, index e * Dph + rank(n), where
// rank(n) is the position of n in the lexicographic order of all admissible tuples (n_0 most
// significant).  With R_j = nph - (n_0 + ... + n_{j-1}) the tuples that precede n and share
// its first j entries but have a smaller j-th entry number
//     sum_{v < n_j} C(R_j - v + L-1-j, L-1-j) = C(R_j + L-j, L-j) - C(R_j - n_j + L-j, L-j)
// (hockey-stick identity), so rank(n) = sum_j [C(R_j + L-j, L-j) - C(R_j - n_j + L-j, L-j)]
// costs O(L) with a binomial table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "cheb_holstein.cuh"
#include "cheb_internal.cuh"

namespace cheb {

// off-diagonal entries of row i in a fixed order: hop to e-1, hop to e+1, phonon up, down
__device__ inline int hol_row(const HolParams& P, int64_t i, int64_t* col, double* val,
                              double* diag)
{
    const int e = (int)(i / P.dph);
    const int64_t p = i - (int64_t)e * P.dph;
    uint8_t occ[HOL_MAX_L];
    hol_unrank(P.C, P.L, P.nph, p, occ);
    int ntot = 0;
    for (int j = 0; j < P.L; ++j) ntot += occ[j];
    *diag = hol_diag_value(P, e, ntot);
    int cnt = 0;
    int el = e - 1, er = e + 1;
    if (P.periodic) {
        el = (el + P.L) % P.L;
        er = er % P.L;
    }
    if (el >= 0) { col[cnt] = (int64_t)el * P.dph + p; val[cnt] = -P.t; ++cnt; }
    if (er < P.L) { col[cnt] = (int64_t)er * P.dph + p; val[cnt] = -P.t; ++cnt; }
    const int ne = occ[e];
    if (ntot < P.nph) {
        occ[e] = (uint8_t)(ne + 1);
        col[cnt] = (int64_t)e * P.dph + hol_rank(P.C, P.L, P.nph, occ);
        val[cnt] = hol_phonon_value(P, e, ne + 1);
        ++cnt;
        occ[e] = (uint8_t)ne;
    }
    if (ne > 0) {
        occ[e] = (uint8_t)(ne - 1);
        col[cnt] = (int64_t)e * P.dph + hol_rank(P.C, P.L, P.nph, occ);
        val[cnt] = hol_phonon_value(P, e, ne);
        ++cnt;
        occ[e] = (uint8_t)ne;
    }
    return cnt;
}

// off-diagonal count of every row
__global__ void k_hol_rowlen(HolParams P, uint8_t* rowlen)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    int64_t col[4];
    double val[4], d;
    rowlen[i] = (uint8_t)hol_row(P, i, col, val, &d);
}

// sum of n bytes into *out (grid-stride, one atomic per warp)
__global__ void k_sum_u8(const uint8_t* x, int64_t n, unsigned long long* out)
{
    unsigned long long t = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        t += x[i];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, t);
}

// SELL-C-sigma row order: inside every window of sigma consecutive rows the rows are ordered by
// decreasing off-diagonal count, rows of equal count keeping their order (stable), so that the
// C = 32 rows of a chunk have nearly equal lengths and the chunk pads little.  One CTA per
// window: counts per length, then positions from warp ballots in passes of blockDim rows.
// perm[position] = row.
__global__ void k_sell_sigma_perm(const uint8_t* rowlen, int64_t n, int sigma, int32_t* perm)
{
    __shared__ int cnt[5], base[5];
    __shared__ int wtot[32][5];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int64_t w0 = (int64_t)blockIdx.x * sigma;
    const int64_t w1 = min(n, w0 + (int64_t)sigma);
    if (tid < 5) cnt[tid] = 0;
    __syncthreads();
    for (int64_t i = w0 + tid; i < w1; i += blockDim.x) atomicAdd(&cnt[4 - rowlen[i]], 1);
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int c = 0; c < 5; ++c) {
            base[c] = acc;
            acc += cnt[c];
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t b0 = w0; b0 < w1; b0 += blockDim.x) {
        const int64_t i = b0 + tid;
        const int c = i < w1 ? 4 - rowlen[i] : -1;  // class 0 = longest rows
        int lanepre = 0;
        for (int cc = 0; cc < 5; ++cc) {
            const unsigned m = __ballot_sync(0xffffffffu, c == cc);
            if (lane == 0) wtot[warp][cc] = __popc(m);
            if (c == cc) lanepre = __popc(m & lt);
        }
        __syncthreads();
        if (c >= 0) {
            int pre = 0;
            for (int w = 0; w < warp; ++w) pre += wtot[w][c];
            perm[w0 + base[c] + pre + lanepre] = (int32_t)i;
        }
        __syncthreads();
        if (tid < 5) {
            int t = 0;
            for (int w = 0; w < nw; ++w) t += wtot[w][tid];
            base[tid] += t;
        }
        __syncthreads();
    }
}

// chunk lengths: the longest row of each chunk of 32 positions (row of a position: perm, or the
// identity without sorting)
__global__ void k_hol_chunklen(HolParams P, const uint8_t* rowlen, const int32_t* perm,
                               int64_t nchunks, int32_t* chunk_len)
{
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t pos = gtid;  // one thread per position; warps are chunks
    int len = 0;
    if (pos < P.n) len = rowlen[perm ? (int64_t)perm[pos] : pos];
    for (int off = 16; off > 0; off >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, off));
    if ((threadIdx.x & 31) == 0 && (gtid >> 5) < nchunks) chunk_len[gtid >> 5] = len;
}

template <typename R>
__global__ void k_hol_fill(HolParams P, const int32_t* perm, const int64_t* chunk_off,
                           const int32_t* chunk_len, int32_t* scol, R* sval, double* sval_raw,
                           uint8_t* rowlen, double* diag_raw, R* diag_scaled, double a, double b)
{
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // storage position
    if (pos >= P.n) return;
    const int64_t i = perm ? (int64_t)perm[pos] : pos;                    // its row
    int64_t col[4];
    double val[4], d;
    const int cnt = hol_row(P, i, col, val, &d);
    const int64_t ch = pos >> 5;
    const int lane = (int)(pos & 31);
    const int len = chunk_len[ch];
    const int64_t off = chunk_off[ch] + lane;
    for (int e = 0; e < len; ++e) {
        const bool real = e < cnt;
        scol[off + (int64_t)e * 32] = real ? (int32_t)col[e] : (int32_t)i;
        sval[off + (int64_t)e * 32] = real ? (R)(2.0 * val[e] / a) : (R)0;
        if (sval_raw) sval_raw[off + (int64_t)e * 32] = real ? val[e] : 0.0;
    }
    if (rowlen) rowlen[i] = (uint8_t)cnt;
    if (diag_raw) diag_raw[i] = d;
    diag_scaled[i] = (R)(2.0 * (d - b) / a);
}

int holstein_build(Plan* p)
{
    const cheb_ham_desc& h = p->desc;
    const int L = h.hol_sites, nph = h.hol_nph;
    std::vector<int64_t> tab;
    if (!make_binom(L, nph, tab)) return fail(CHEB_ERR_INVALID, "Holstein basis too large");
    const int64_t dph = tab[(size_t)(nph + L) * (L + 2) + L];
    const int64_t n = (int64_t)L * dph;
    if (n >= ((int64_t)1 << 31) - 64) return fail(CHEB_ERR_INVALID, "Holstein dimension >= 2^31");
    p->hol_dph = dph;
    CHEB_CUDA(cudaMalloc(&p->d_binom, tab.size() * sizeof(int64_t)));
    CHEB_CUDA(cudaMemcpy(p->d_binom, tab.data(), tab.size() * sizeof(int64_t),
                         cudaMemcpyHostToDevice));
    HolParams P;
    P.L = L;
    P.nph = nph;
    P.periodic = h.hol_periodic;
    P.dph = dph;
    P.n = n;
    P.t = h.hop;
    P.omega0 = h.omega0;
    P.g = h.g;
    P.delta = h.onsite;
    P.gsite = h.hol_g;
    P.C = Binom{p->d_binom, L};
    // unscaled copies (CSR export) only for bases up to 2^27 rows
    const bool keep_raw = n <= ((int64_t)1 << 27);

    const int64_t nchunks = (n + 31) / 32;
    p->sell_nchunks = nchunks;
    CHEB_CUDA(cudaMalloc(&p->d_sell_chunk_len, nchunks * sizeof(int32_t)));
    CHEB_CUDA(cudaMalloc(&p->d_sell_chunk_off, (nchunks + 1) * sizeof(int64_t)));
    const int th = 256;
    // row lengths (kept for the CSR export and the energy when the basis is small), then the
    // sigma-window order of the rows
    uint8_t* rowlen = nullptr;
    CHEB_CUDA(cudaMalloc(&rowlen, (size_t)n));
    k_hol_rowlen<<<(unsigned)((n + th - 1) / th), th, 0, p->stream>>>(P, rowlen);
    p->launches++;
    CHEB_CUDA(cudaGetLastError());
    if (p->sell_sigma > 1) {
        CHEB_CUDA(cudaMalloc(&p->d_sell_perm, (size_t)n * sizeof(int32_t)));
        const int64_t nwin = (n + p->sell_sigma - 1) / p->sell_sigma;
        k_sell_sigma_perm<<<(unsigned)nwin, std::min(p->sell_sigma, 1024), 0, p->stream>>>(
            rowlen, n, p->sell_sigma, p->d_sell_perm);
        p->launches++;
        CHEB_CUDA(cudaGetLastError());
    }
    const int64_t blocks = (nchunks * 32 + th - 1) / th;
    k_hol_chunklen<<<(unsigned)blocks, th, 0, p->stream>>>(P, rowlen, p->d_sell_perm, nchunks,
                                                          p->d_sell_chunk_len);
    p->launches++;
    CHEB_CUDA(cudaGetLastError());
    std::vector<int32_t> len(nchunks);
    CHEB_CUDA(cudaMemcpyAsync(len.data(), p->d_sell_chunk_len, nchunks * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, p->stream));
    CHEB_CUDA(cudaStreamSynchronize(p->stream));
    std::vector<int64_t> off(nchunks + 1);
    off[0] = 0;
    for (int64_t c = 0; c < nchunks; ++c) off[c + 1] = off[c] + (int64_t)len[c] * 32;
    p->sell_nnz_stored = off[nchunks];
    CHEB_CUDA(cudaMemcpy(p->d_sell_chunk_off, off.data(), (nchunks + 1) * sizeof(int64_t),
                         cudaMemcpyHostToDevice));
    const size_t ns = (size_t)std::max<int64_t>(p->sell_nnz_stored, 1);
    CHEB_CUDA(cudaMalloc(&p->d_sell_col, ns * sizeof(int32_t)));
    CHEB_CUDA(cudaMalloc(&p->d_sell_val, ns * p->real_size()));
    if (keep_raw) {
        CHEB_CUDA(cudaMalloc(&p->d_sell_val_raw, ns * sizeof(double)));
        CHEB_CUDA(cudaMalloc(&p->d_hol_diag_raw, (size_t)n * sizeof(double)));
        p->d_hol_rowlen = rowlen;
        rowlen = nullptr;
    }
    const DevBlock& B = p->hblocks[0];
    const unsigned gb = (unsigned)((n + th - 1) / th);
    if (p->prec == CHEB_C128)
        k_hol_fill<double><<<gb, th, 0, p->stream>>>(
            P, p->d_sell_perm, p->d_sell_chunk_off, p->d_sell_chunk_len, p->d_sell_col,
            static_cast<double*>(p->d_sell_val), p->d_sell_val_raw, nullptr,
            p->d_hol_diag_raw, static_cast<double*>(p->d_diag), B.a, B.b);
    else
        k_hol_fill<float><<<gb, th, 0, p->stream>>>(
            P, p->d_sell_perm, p->d_sell_chunk_off, p->d_sell_chunk_len, p->d_sell_col,
            static_cast<float*>(p->d_sell_val), p->d_sell_val_raw, nullptr,
            p->d_hol_diag_raw, static_cast<float*>(p->d_diag), B.a, B.b);
    p->launches++;
    CHEB_CUDA(cudaGetLastError());
    CHEB_CUDA(cudaStreamSynchronize(p->stream));
    // off-diagonal entries of the matrix without padding (padding statistics)
    unsigned long long* d_cnt = nullptr;
    CHEB_CUDA(cudaMalloc(&d_cnt, sizeof(unsigned long long)));
    CHEB_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), p->stream));
    k_sum_u8<<<(unsigned)std::min<int64_t>((n + th - 1) / th, 4096), th, 0, p->stream>>>(
        p->d_hol_rowlen ? p->d_hol_rowlen : rowlen, n, d_cnt);
    p->launches++;
    unsigned long long nz = 0;
    CHEB_CUDA(cudaMemcpyAsync(&nz, d_cnt, sizeof(nz), cudaMemcpyDeviceToHost, p->stream));
    CHEB_CUDA(cudaStreamSynchronize(p->stream));
    cudaFree(d_cnt);
    if (rowlen) cudaFree(rowlen);
    p->sell_nnz_offdiag = (int64_t)nz;
    return CHEB_OK;
}

// ---- observables ------------------------------------------------------------------------------
// Work items of a Holstein plan never straddle two electron sites, so density and chi of an
// item belong to the single slot e = first / Dph.  Per item partials:
//   [item][0][v]            <n_e> part            (density)
//   [item][1][v]            <n_e (b_e + b_e^+)>   (chi)
//   [item][2 + i][v]        <b_i^+ b_i> part      (phonon), i < L
//   energy: [item][0][v] = <x|H x> part
template <typename R>
__global__ void k_hol_obs(HolParams P, const WorkItem* items, int nitems, const void* psi_,
                          int nvec, int kind, const int32_t* perm, const int64_t* chunk_off,
                          const int32_t* chunk_len, const int32_t* scol, const R* sval,
                          const R* dscaled, double a, double b, double* partials, int nslot)
{
    using C = typename CT<R>::type;
    const C* psi = static_cast<const C*>(psi_);
    __shared__ double s_red[32];
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const WorkItem it = items[w];
        for (int v = 0; v < nvec; ++v) {
            for (int slot = 0; slot < nslot; ++slot) {
                double acc = 0.0;
                for (int64_t u = threadIdx.x; u < it.count; u += blockDim.x) {
                    int64_t i = it.first + u;
                    if (kind == CHEB_OBS_ENERGY) {
                        // <x|H|x> = (a/2) <x|2H~ x> + b |x|^2 from the scaled matrix the
                        // recurrence uses (padding entries are zero); the sum runs over the
                        // matrix's storage positions, row = perm[position] when sorted
                        const int64_t pos = i;
                        if (perm) i = perm[pos];
                        const C x = psi[i * nvec + v];
                        const double wgt = (double)x.x * x.x + (double)x.y * x.y;
                        const double d = (double)dscaled[i];
                        double hx = d * x.x, hy = d * x.y;
                        const int64_t ch = pos >> 5;
                        const int64_t off = chunk_off[ch] + (pos & 31);
                        for (int e = 0; e < chunk_len[ch]; ++e) {
                            const C y = psi[(int64_t)scol[off + (int64_t)e * 32] * nvec + v];
                            const double w = (double)sval[off + (int64_t)e * 32];
                            hx += w * y.x;
                            hy += w * y.y;
                        }
                        acc += 0.5 * a * ((double)x.x * hx + (double)x.y * hy) + b * wgt;
                        continue;
                    }
                    const C x = psi[i * nvec + v];
                    const double wgt = (double)x.x * x.x + (double)x.y * x.y;
                    if (kind == CHEB_OBS_HOL_DENSITY) {
                        acc += wgt;
                    } else {
                        const int e = (int)(i / P.dph);
                        uint8_t occ[HOL_MAX_L];
                        hol_unrank(P.C, P.L, P.nph, i - (int64_t)e * P.dph, occ);
                        if (kind == CHEB_OBS_HOL_PHONON) {
                            acc += wgt * (double)occ[slot];
                        } else {  // chi: pair this row with the state one phonon higher at e
                            int ntot = 0;
                            for (int j = 0; j < P.L; ++j) ntot += occ[j];
                            if (ntot < P.nph) {
                                const int ne = occ[e];
                                occ[e] = (uint8_t)(ne + 1);
                                const int64_t up = (int64_t)e * P.dph + hol_rank(P.C, P.L, P.nph, occ);
                                const C y = psi[up * nvec + v];
                                acc += 2.0 * ((double)y.x * x.x + (double)y.y * x.y) * sqrt((double)ne + 1.0);
                            }
                        }
                    }
                }
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
                __syncthreads();
                if (threadIdx.x == 0) {
                    double t = 0.0;
                    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_red[q];
                    partials[((size_t)w * nslot + slot) * nvec + v] = t;
                }
                __syncthreads();
            }
        }
    }
}

__global__ void k_hol_obs_finalize(const WorkItem* items, int nitems, int64_t dph, int L,
                                   int nvec, int kind, int nslot, const double* partials,
                                   double* out)
{
    // out: density/chi/phonon [L][nvec]; energy [nvec]
    const int nout = (kind == CHEB_OBS_ENERGY) ? nvec : L * nvec;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += gridDim.x * blockDim.x) {
        const int i = o / nvec, v = o % nvec;
        double t = 0.0;
        for (int w = 0; w < nitems; ++w) {
            const int e = (int)(items[w].first / dph);
            if (kind == CHEB_OBS_HOL_PHONON) {
                t += partials[((size_t)w * nslot + i) * nvec + v];
            } else if (kind == CHEB_OBS_ENERGY) {
                t += partials[((size_t)w * nslot + 0) * nvec + v];
            } else if (e == i) {
                t += partials[((size_t)w * nslot + 0) * nvec + v];
            }
        }
        out[o] = t;
    }
}

static int hol_obs_common(Plan* p, const void* psi, int kind, double* out, cudaStream_t s)
{
    const cheb_ham_desc& h = p->desc;
    HolParams P;
    P.L = h.hol_sites;
    P.nph = h.hol_nph;
    P.periodic = h.hol_periodic;
    P.dph = p->hol_dph;
    P.n = p->n_sites;
    P.t = h.hop;
    P.omega0 = h.omega0;
    P.g = h.g;
    P.delta = nullptr;
    P.C = Binom{p->d_binom, P.L};
    const int nslot = (kind == CHEB_OBS_HOL_PHONON) ? P.L : 1;
    const int nitems = (int)p->hitems.size();
    const size_t need = (size_t)nitems * nslot * p->nvec;
    if (p->obs_scratch_cap < need) {
        if (p->d_obs_scratch) cudaFree(p->d_obs_scratch);
        p->d_obs_scratch = nullptr;
        p->obs_scratch_cap = 0;
        CHEB_CUDA(cudaMalloc(&p->d_obs_scratch, need * sizeof(double)));
        p->obs_scratch_cap = need;
    }
    const int grid = std::min(nitems, 65535);
    const double ba = p->hblocks[0].a, bb = p->hblocks[0].b;
    if (p->prec == CHEB_C128)
        k_hol_obs<double><<<grid, 256, 0, s>>>(P, p->d_items, nitems, psi, p->nvec, kind,
                                               p->d_sell_perm, p->d_sell_chunk_off, p->d_sell_chunk_len,
                                               p->d_sell_col, static_cast<const double*>(p->d_sell_val),
                                               static_cast<const double*>(p->d_diag), ba, bb,
                                               p->d_obs_scratch, nslot);
    else
        k_hol_obs<float><<<grid, 256, 0, s>>>(P, p->d_items, nitems, psi, p->nvec, kind,
                                              p->d_sell_perm, p->d_sell_chunk_off, p->d_sell_chunk_len,
                                              p->d_sell_col, static_cast<const float*>(p->d_sell_val),
                                              static_cast<const float*>(p->d_diag), ba, bb,
                                              p->d_obs_scratch, nslot);
    k_hol_obs_finalize<<<1, 256, 0, s>>>(p->d_items, nitems, p->hol_dph, P.L, p->nvec, kind,
                                         nslot, p->d_obs_scratch, out);
    p->launches += 2;
    CHEB_CUDA(cudaGetLastError());
    return CHEB_OK;
}

int launch_holstein_observable(Plan* p, const void* psi, int kind, double* out, cudaStream_t s)
{
    return hol_obs_common(p, psi, kind, out, s);
}

int launch_holstein_energy(Plan* p, const void* psi, double* out, cudaStream_t s)
{
    return hol_obs_common(p, psi, CHEB_OBS_ENERGY, out, s);
}

}  // namespace cheb

using namespace cheb;

// ---- host ABI ---------------------------------------------------------------------------------
extern "C" int64_t cheb_holstein_dim_phonon(int L, int nph)
{
    if (L < 1 || L > HOL_MAX_L || nph < 0 || nph > 255) return -1;
    std::vector<int64_t> tab;
    if (!make_binom(L, nph, tab)) return -1;
    return tab[(size_t)(nph + L) * (L + 2) + L];
}

extern "C" int cheb_holstein_rank(int L, int nph, const uint8_t* occ, int e, int64_t* idx)
{
    if (!occ || !idx || L < 1 || L > HOL_MAX_L || nph < 0 || nph > 255 || e < 0 || e >= L)
        return fail(CHEB_ERR_INVALID, "cheb_holstein_rank: bad arguments");
    int s = 0;
    for (int j = 0; j < L; ++j) s += occ[j];
    if (s > nph) return fail(CHEB_ERR_INVALID, "cheb_holstein_rank: occupation sum > nph");
    std::vector<int64_t> tab;
    if (!make_binom(L, nph, tab)) return fail(CHEB_ERR_INVALID, "cheb_holstein_rank: overflow");
    Binom C{tab.data(), L};
    const int64_t dph = C(nph + L, L);
    *idx = (int64_t)e * dph + hol_rank(C, L, nph, occ);
    return CHEB_OK;
}

extern "C" int cheb_holstein_unrank(int L, int nph, int64_t idx, uint8_t* occ, int* e)
{
    if (!occ || !e || L < 1 || L > HOL_MAX_L || nph < 0 || nph > 255)
        return fail(CHEB_ERR_INVALID, "cheb_holstein_unrank: bad arguments");
    std::vector<int64_t> tab;
    if (!make_binom(L, nph, tab)) return fail(CHEB_ERR_INVALID, "cheb_holstein_unrank: overflow");
    Binom C{tab.data(), L};
    const int64_t dph = C(nph + L, L);
    if (idx < 0 || idx >= (int64_t)L * dph)
        return fail(CHEB_ERR_INVALID, "cheb_holstein_unrank: index out of range");
    *e = (int)(idx / dph);
    hol_unrank(C, L, nph, idx - (int64_t)(*e) * dph, occ);
    return CHEB_OK;
}

extern "C" int cheb_holstein_phonon_neighbors(int L, int nph, int64_t p0, int64_t count,
                                              int64_t* up, int64_t* dn)
{
    if (!up || !dn || L < 1 || L > HOLMF_MAX_L || nph < 0 || nph > HOLMF_MAX_NPH || p0 < 0 ||
        count < 0)
        return fail(CHEB_ERR_INVALID, "cheb_holstein_phonon_neighbors: bad arguments");
    std::vector<int64_t> tab;
    if (!make_binom(L, nph, tab)) return fail(CHEB_ERR_INVALID, "cheb_holstein_phonon_neighbors: overflow");
    const int64_t dph = Binom{tab.data(), L}(nph + L, L);
    if (dph >= ((int64_t)1 << 31) || p0 + count > dph)
        return fail(CHEB_ERR_INVALID, "cheb_holstein_phonon_neighbors: ranks out of range");
    std::vector<int2> g;
    make_hol_g(L, nph, tab, g);
    const HolG G{g.data(), nph + 1};
    for (int64_t i = 0; i < count; ++i) {
        const int64_t p = p0 + i;
        HolWalk W;
        W.begin(G, L, nph, (int32_t)p);
        for (int e = L - 1; e >= 0; --e) {
            int32_t du, dd;
            W.step(G, L, nph, e, du, dd);
            up[i * L + e] = du ? p + du : -1;
            dn[i * L + e] = dd ? p - dd : -1;
        }
    }
    return CHEB_OK;
}
