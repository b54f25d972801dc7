// One whole time step of a small 1D grid (Sec. 3.1; Eqs. U_1 and rec) in a single launch on a
// thread-block cluster.
//
// The 3-point chain of n sites is split over the CL CTAs of one cluster (a contiguous chunk per
// CTA).  T_{k-1} lives in shared memory (two buffers, read T_{k-1} / write T_k), T_{k-2} and the
// accumulators of Eq. U_1 of a thread's own sites stay in registers, and a CTA reads the two
// neighbouring values beyond its chunk straight from the neighbour CTA's shared memory
// (distributed shared memory).  One cluster barrier separates consecutive orders, so the M
// orders of a step cost M barriers instead of M kernel launches, and the DRAM sees psi once
// in and once out.  Every thread runs the same number of barriers (no early exit).
//
// Spreading the chain over several SMs matters for complex128: one SM does about two FP64
// fused multiply-adds per clock on this GPU.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "cheb_device.cuh"
#include "cheb_internal.cuh"

namespace cg = cooperative_groups;

namespace cheb {

static constexpr int CL_MAX_CTAS = 16;  // CTAs per cluster: 8 (portable) or 16
static constexpr int CL_MAX_SPT = 4;    // sites per thread
static constexpr int CL_THREADS = 1024;
static constexpr int64_t CL_MAX_SITES = (int64_t)8 * CL_THREADS * CL_MAX_SPT;

struct ClusterArgs {
    void* psi;                // [n] in: T_0; out: psi(t + dt)
    const void* diag;         // R [n]: 2 (H_ii - b) / a
    const void* qcoef;        // C (hi, lo) per order
    const DevBlock* blocks;   // block 0: M, ksplit, beta, a, b, phase
    int32_t n;
    int32_t chunk;            // sites per CTA
    double* red_out;          // [2]: ||psi||^2, <psi|H|psi>
    int* errflag;
};

template <typename R, int SPT>
__global__ void __launch_bounds__(CL_THREADS) k_step_cluster(ClusterArgs a)
{
    using C = typename V2<R>::C;
    using U = SiteUpdate<R>;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ float4 cl_smem_raw[];
    C* const buf0 = reinterpret_cast<C*>(cl_smem_raw);  // [chunk]
    C* const buf1 = buf0 + a.chunk;                       // [chunk]
    __shared__ double s_red[32 * 2];
    __shared__ double s_tot[2];

    const int rank = (int)cluster.block_rank();
    const int nctas = (int)cluster.num_blocks();
    const int lo = rank * a.chunk;
    const int cnt = max(0, min(a.n, lo + a.chunk) - lo);
    const bool has_left = rank > 0 && lo > 0;
    const bool has_right = rank + 1 < nctas && lo + cnt < a.n;
    // the neighbours' buffers, seen through distributed shared memory
    C* const l0 = has_left ? cluster.map_shared_rank(buf0, rank - 1) : buf0;
    C* const l1 = has_left ? cluster.map_shared_rank(buf1, rank - 1) : buf1;
    C* const r0 = has_right ? cluster.map_shared_rank(buf0, rank + 1) : buf0;
    C* const r1 = has_right ? cluster.map_shared_rank(buf1, rank + 1) : buf1;

    const DevBlock B = a.blocks[0];
    const C* __restrict__ qc = static_cast<const C*>(a.qcoef);
    const R* __restrict__ diag = static_cast<const R*>(a.diag);
    C* __restrict__ psi = static_cast<C*>(a.psi);
    R bh, bl;
    split_const<R>(B.beta, bh, bl);
    C ph, pl;
    split_const<R>(B.ph_re, ph.x, pl.x);
    split_const<R>(B.ph_im, ph.y, pl.y);
    const int tid = threadIdx.x;
    const C zero = V2<R>::make(0, 0);

    // own sites li = tid + j * blockDim.x: T_0 into shared memory, d and the accumulators
    C p[SPT], acc[SPT], tl[SPT];
    R d[SPT];
    const C q0 = qc[B.coef_off + 0];
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int li = tid + j * (int)blockDim.x;
        p[j] = zero;
        acc[j] = zero;
        tl[j] = zero;
        d[j] = 0;
        if (li < cnt) {
            const C x = psi[lo + li];
            buf0[li] = x;
            d[j] = diag[lo + li];
            U::accum(acc[j], q0, x, 0);
        }
    }
    cluster.sync();

    // orders k = 1 .. M: T_k from T_{k-1} (shared, buffer (k-1) & 1) and T_{k-2} (registers)
    R part0 = 0, part1 = 0;
    for (int k = 1; k <= B.M; ++k) {
        const C* cur = (k & 1) ? buf0 : buf1;
        C* nxt = (k & 1) ? buf1 : buf0;
        const C* curl = (k & 1) ? l0 : l1;
        const C* curr = (k & 1) ? r0 : r1;
        const C qk = qc[B.coef_off + k];
        const bool to_tail = k > B.ksplit;
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const int li = tid + j * (int)blockDim.x;
            if (li < cnt) {
                const C x = cur[li];
                const C yl = li > 0 ? cur[li - 1] : (has_left ? curl[a.chunk - 1] : zero);
                const C yr = li + 1 < cnt ? cur[li + 1] : (has_right ? curr[0] : zero);
                const R sx = yl.x + yr.x, sy = yl.y + yr.y;
                R hx = -p[j].x, hy = -p[j].y;
                if constexpr (Split<R>::on) {  // complex64: beta as a float-float pair
                    hx = fma(bl, sx, hx);
                    hy = fma(bl, sy, hy);
                }
                hx = fma(bh, sx, hx);
                hy = fma(bh, sy, hy);
                hx = fma(d[j], x.x, hx);
                hy = fma(d[j], x.y, hy);
                if (k == 1) {  // T_1 = H~ T_0
                    hx *= (R)0.5;
                    hy *= (R)0.5;
                    part0 = fma(x.x, x.x, fma(x.y, x.y, part0));
                    part1 = fma(x.x, hx, fma(x.y, hy, part1));
                }
                const C h = V2<R>::make(hx, hy);
                nxt[li] = h;
                p[j] = x;
                U::accum(to_tail ? tl[j] : acc[j], qk, h, k);
                // growth check |T_M|^2 <= 4 ||psi||^2: s_tot is written by the k = 1 sums below
                // and read from k = 2 on (every plan has M >= 2, cheb_coeffs raises M = 1)
                if (k == B.M && k >= 2) {
                    const R t2 = fma(h.x, h.x, h.y * h.y);
                    if (!(t2 <= (R)(4.0 * s_tot[0]))) atomicOr(a.errflag, 1);
                }
            }
        }
        if (k == 1) {
            // ||T_0||^2 and <T_0|H~ T_0>: warp tree, CTA sum, then every CTA adds the
            // cluster's partials read from the other CTAs' shared memory
            double v0 = (double)part0, v1 = (double)part1;
            for (int off = 16; off > 0; off >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, off);
                v1 += __shfl_xor_sync(0xffffffffu, v1, off);
            }
            if ((tid & 31) == 0) {
                s_red[(tid >> 5) * 2 + 0] = v0;
                s_red[(tid >> 5) * 2 + 1] = v1;
            }
            __syncthreads();
            if (tid == 0) {
                double t0 = 0.0, t1 = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    t0 += s_red[w * 2 + 0];
                    t1 += s_red[w * 2 + 1];
                }
                s_red[62] = t0;
                s_red[63] = t1;
            }
            cluster.sync();
            if (tid == 0) {
                double t0 = 0.0, t1 = 0.0;
                for (int r = 0; r < nctas; ++r) {
                    const double* rs = cluster.map_shared_rank(s_red, r);
                    t0 += rs[62];
                    t1 += rs[63];
                }
                s_tot[0] = t0;
                s_tot[1] = t1;
                if (rank == 0) {
                    a.red_out[0] = t0;
                    a.red_out[1] = B.a * t1 + B.b * t0;  // <H> = a <H~> + b ||psi||^2
                }
            }
        }
        cluster.sync();  // T_k complete everywhere (and the k = 1 sums read) before order k + 1
    }
    // psi(t + dt) = e^{-i b dt} (accumulator + tail)
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int li = tid + j * (int)blockDim.x;
        if (li < cnt) {
            const C s = V2<R>::make(acc[j].x + tl[j].x, acc[j].y + tl[j].y);
            psi[lo + li] = U::phase(s, ph, pl);
        }
    }
}

// 1D grids of at most 8 * 1024 * 4 sites, one vector
bool cluster_eligible(const Plan* p)
{
    return p->desc.kind == CHEB_LAT1D && p->nvec == 1 && !p->desc.onsite_per_vec &&
           p->n_sites <= CL_MAX_SITES;
}

// chunk of sites per CTA, threads per CTA (one per site up to 1024) and sites per thread
static void cluster_shape(const Plan* p, int ctas, int* chunk, int* threads, int* spt, size_t* smem)
{
    const int n = (int)p->n_sites;
    *chunk = (n + ctas - 1) / ctas;
    *threads = std::max(32, std::min(CL_THREADS, (*chunk + 31) / 32 * 32));
    const int need = (*chunk + *threads - 1) / *threads;
    *spt = need <= 1 ? 1 : (need <= 2 ? 2 : 4);
    *smem = 2 * (size_t)(*chunk) * p->cplx_size();
}

template <typename R, int SPT>
static int cluster_attr(size_t smem)
{
    // never below the default 48 KB: a later launch with a larger chunk must not be refused
    CHEB_CUDA(cudaFuncSetAttribute(k_step_cluster<R, SPT>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)std::max<size_t>(smem, 48 * 1024)));
    CHEB_CUDA(cudaFuncSetAttribute(k_step_cluster<R, SPT>,
                                   cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return CHEB_OK;
}

template <typename R, int SPT>
static int cluster_fits(int ctas, int threads, size_t smem, int* fits)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    CHEB_CUDA(cudaOccupancyMaxActiveClusters(&n, k_step_cluster<R, SPT>, &cfg));
    *fits = n > 0;
    return CHEB_OK;
}

template <typename R>
static int cluster_prepare_r(int ctas, int spt, int threads, size_t smem, int* fits)
{
    int rc = CHEB_OK;
    if (spt == 1) rc = cluster_attr<R, 1>(smem);
    else if (spt == 2) rc = cluster_attr<R, 2>(smem);
    else rc = cluster_attr<R, 4>(smem);
    if (rc) return rc;
    if (spt == 1) return cluster_fits<R, 1>(ctas, threads, smem, fits);
    if (spt == 2) return cluster_fits<R, 2>(ctas, threads, smem, fits);
    return cluster_fits<R, 4>(ctas, threads, smem, fits);
}

// Set the kernel's attributes for a cluster of `ctas` CTAs; CHEB_ERR_UNSUPPORTED if the
// device cannot schedule such a cluster.
int cluster_configure(Plan* p, int ctas)
{
    if (ctas != 8 && ctas != CL_MAX_CTAS) return fail(CHEB_ERR_INVALID, "cluster size must be 8 or 16");
    int chunk, threads, spt, fits = 0;
    size_t smem;
    cluster_shape(p, ctas, &chunk, &threads, &spt, &smem);
    const int rc = p->prec == CHEB_C128 ? cluster_prepare_r<double>(ctas, spt, threads, smem, &fits)
                                        : cluster_prepare_r<float>(ctas, spt, threads, smem, &fits);
    if (rc) return rc;
    return fits ? CHEB_OK : fail(CHEB_ERR_UNSUPPORTED, "the device cannot schedule this cluster");
}

template <typename R, int SPT>
static cudaError_t cluster_go_t(const ClusterArgs& a, int ctas, int threads, size_t smem,
                                cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_cluster<R, SPT>, a);
}

template <typename R>
static cudaError_t cluster_go(const ClusterArgs& a, int ctas, int spt, int threads, size_t smem,
                              cudaStream_t s)
{
    if (spt == 1) return cluster_go_t<R, 1>(a, ctas, threads, smem, s);
    if (spt == 2) return cluster_go_t<R, 2>(a, ctas, threads, smem, s);
    return cluster_go_t<R, 4>(a, ctas, threads, smem, s);
}

int cluster_launch(Plan* p, void* psi, cudaStream_t s)
{
    const int ctas = p->cluster;
    int chunk, threads, spt;
    size_t smem;
    cluster_shape(p, ctas, &chunk, &threads, &spt, &smem);
    ClusterArgs a{};
    a.psi = psi;
    a.diag = p->d_diag;
    a.qcoef = p->d_qcoef;
    a.blocks = p->d_blocks;
    a.n = (int32_t)p->n_sites;
    a.chunk = chunk;
    a.red_out = p->d_red;
    a.errflag = p->d_err;
    const cudaError_t e = p->prec == CHEB_C128 ? cluster_go<double>(a, ctas, spt, threads, smem, s)
                                               : cluster_go<float>(a, ctas, spt, threads, smem, s);
    if (e != cudaSuccess) {
        cudaGetLastError();  // a refused launch leaves no error behind for later calls
        return cuda_fail(e, "cluster step launch");
    }
    p->launches++;
    return CHEB_OK;
}

}  // namespace cheb
