// One whole time step of a small 1D grid (Sec. 3.1; Eqs. U_1 and rec) in a single launch on a
// thread-block cluster.
//
// The 3-point chain of n sites is split over the CL CTAs of one cluster (a contiguous chunk per
// CTA).  A CTA keeps T_{k-1} and T_{k-2} of its chunk in shared memory with margins of S sites
// on both sides, and runs the orders in super-steps of S: at the start of a super-step it
// copies the S edge values of T_{k-1} and the S - 1 edge values of T_{k-2} of each
// neighbouring CTA (distributed shared memory) into its margins; after a cluster barrier it
// forms the S orders alone, order o of the super-step over its chunk widened by S - 1 - o
// sites on each side (the widened part recomputes the neighbours' edge sites, each order
// needing one site less), with only CTA barriers between orders; a second cluster barrier ends
// the super-step.  The M orders of a step cost about 2 M / S cluster barriers (one per order
// with S = 1), and the DRAM sees psi once in and once out.  Sites beyond the chain read as
// zero.  Every thread runs the same number of barriers (no early exit).
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
static constexpr int CL_MAX_SPT = 4;    // positions per thread
static constexpr int CL_THREADS = 1024;
static constexpr int64_t CL_MAX_SITES = (int64_t)8 * CL_THREADS * 4;

struct ClusterArgs {
    void* psi;                // [n] in: T_0; out: psi(t + dt)
    const void* diag;         // R [n]: 2 (H_ii - b) / a
    const void* qcoef;        // C (hi, lo) per order
    const DevBlock* blocks;   // block 0: M, ksplit, beta, a, b, phase
    int32_t n;
    int32_t chunk;            // sites per CTA
    int32_t S;                // orders per super-step, 1 <= S <= chunk
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
    const int S = a.S;
    // two buffers of chunk + 2 S, site i of the chunk (i in [-S, chunk + S)) at i + S
    C* bA = reinterpret_cast<C*>(cl_smem_raw) + S;  // T_{k-1}
    C* bB = bA + (a.chunk + 2 * S);                  // T_{k-2}, overwritten by T_k
    __shared__ double s_red[32 * 2];
    __shared__ double s_tot[2];

    const int rank = (int)cluster.block_rank();
    const int nctas = (int)cluster.num_blocks();
    const int lo = rank * a.chunk;
    const int cnt = max(0, min(a.n, lo + a.chunk) - lo);
    const bool has_left = rank > 0 && lo > 0;
    const bool has_right = rank + 1 < nctas && lo + cnt < a.n;

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
    const int nth = (int)blockDim.x;
    const C zero = V2<R>::make(0, 0);

    // both buffers zero (margins and sites beyond the chain stay zero unless copied)
    for (int i = tid; i < 2 * (a.chunk + 2 * S); i += nth) reinterpret_cast<C*>(cl_smem_raw)[i] = zero;
    __syncthreads();
    // positions i = tid - (S - 1) + j nth cover the widest order's [-(S - 1), cnt + S - 1);
    // own sites (0 <= i < cnt): T_0 into shared memory and the accumulators
    C acc[SPT], tl[SPT];
    R d[SPT];
    const C q0 = qc[B.coef_off + 0];
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int i = tid - (S - 1) + j * nth;
        const int gi = lo + i;
        acc[j] = zero;
        tl[j] = zero;
        d[j] = (gi >= 0 && gi < a.n && i < cnt + S - 1) ? diag[gi] : (R)0;
        if (i >= 0 && i < cnt) {
            const C x = psi[gi];
            bA[i] = x;
            U::accum(acc[j], q0, x, 0);
        }
    }
    cluster.sync();

    R part0 = 0, part1 = 0;
    for (int k0 = 1; k0 <= B.M; k0 += S) {
        const int ns = min(S, B.M - k0 + 1);
        // margins: T_{k0-1} at S sites and T_{k0-2} at S - 1 sites beyond each end of the chunk,
        // from the neighbours' buffers (the same offsets: every CTA swaps its buffers alike)
        if (tid < 2 * S) {
            const int t = tid < S ? tid : tid - S;
            C va = zero, vb = zero;
            if (tid < S) {  // site -1 - t: the left neighbour's site chunk - 1 - t
                if (has_left) {
                    va = cluster.map_shared_rank(bA, rank - 1)[a.chunk - 1 - t];
                    if (t < S - 1) vb = cluster.map_shared_rank(bB, rank - 1)[a.chunk - 1 - t];
                }
                bA[-1 - t] = va;
                if (t < S - 1) bB[-1 - t] = vb;
            } else {  // site cnt + t: the right neighbour's site t (zero beyond the chain)
                if (has_right && lo + cnt + t < a.n) {
                    va = cluster.map_shared_rank(bA, rank + 1)[t];
                    if (t < S - 1) vb = cluster.map_shared_rank(bB, rank + 1)[t];
                }
                bA[cnt + t] = va;
                if (t < S - 1) bB[cnt + t] = vb;
            }
        }
        cluster.sync();  // every CTA has its margins before any buffer changes
        for (int o = 0; o < ns; ++o) {
            const int k = k0 + o;
            const int hw = S - 1 - o;  // sites formed beyond each end at this order
            const C qk = qc[B.coef_off + k];
            const bool to_tail = k > B.ksplit;
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
                const int i = tid - (S - 1) + j * nth;
                const int gi = lo + i;
                if (i >= -hw && i < cnt + hw && gi >= 0 && gi < a.n) {
                    const C x = bA[i];
                    const C yl = bA[i - 1];
                    const C yr = bA[i + 1];
                    const C pv = bB[i];
                    const R sx = yl.x + yr.x, sy = yl.y + yr.y;
                    R hx = -pv.x, hy = -pv.y;
                    if constexpr (Split<R>::on) {  // complex64: beta as a float-float pair
                        hx = fma(bl, sx, hx);
                        hy = fma(bl, sy, hy);
                    }
                    hx = fma(bh, sx, hx);
                    hy = fma(bh, sy, hy);
                    hx = fma(d[j], x.x, hx);
                    hy = fma(d[j], x.y, hy);
                    const bool own = i >= 0 && i < cnt;
                    if (k == 1) {  // T_1 = H~ T_0 (T_{-1} = 0)
                        hx *= (R)0.5;
                        hy *= (R)0.5;
                        if (own) {
                            part0 = fma(x.x, x.x, fma(x.y, x.y, part0));
                            part1 = fma(x.x, hx, fma(x.y, hy, part1));
                        }
                    }
                    const C h = V2<R>::make(hx, hy);
                    bB[i] = h;  // T_k over T_{k-2} (this thread's own position)
                    if (own) {
                        U::accum(to_tail ? tl[j] : acc[j], qk, h, k);
                        // growth check |T_M|^2 <= 4 ||psi||^2: s_tot is written by the k = 1
                        // sums below and read from k = 2 on (every plan has M >= 2)
                        if (k == B.M && k >= 2) {
                            const R t2 = fma(h.x, h.x, h.y * h.y);
                            if (!(t2 <= (R)(4.0 * s_tot[0]))) atomicOr(a.errflag, 1);
                        }
                    }
                }
            }
            C* const t = bA;  // T_k becomes the next order's T_{k-1}
            bA = bB;
            bB = t;
            __syncthreads();
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
                    for (int w = 0; w < (nth >> 5); ++w) {
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
                __syncthreads();
            }
        }
        cluster.sync();  // the super-step's edges are complete before the neighbours copy them
    }
    // psi(t + dt) = e^{-i b dt} (accumulator + tail)
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int i = tid - (S - 1) + j * nth;
        if (i >= 0 && i < cnt) {
            const C sum = V2<R>::make(acc[j].x + tl[j].x, acc[j].y + tl[j].y);
            psi[lo + i] = U::phase(sum, ph, pl);
        }
    }
}

// 1D grids of at most 8 * 1024 * 4 sites, one vector
bool cluster_eligible(const Plan* p)
{
    return p->desc.kind == CHEB_LAT1D && p->nvec == 1 && !p->desc.onsite_per_vec &&
           p->n_sites <= CL_MAX_SITES;
}

// chunk of sites per CTA, orders per super-step, threads per CTA (one per position of the
// widest order up to 1024) and positions per thread
static void cluster_shape(const Plan* p, int ctas, int* chunk, int* S, int* threads, int* spt,
                          size_t* smem)
{
    const int n = (int)p->n_sites;
    *chunk = (n + ctas - 1) / ctas;
    // orders per super-step: the redundant edge work grows with S / chunk, the cluster barriers
    // fall as 1 / S; measured on the 2048-point grid (16 CTAs): complex128 flat from S = 16 to
    // 32 (FP64 bound), complex64 best near 48-64.  S <= chunk (margins come from the direct
    // neighbours only) and the widest order's chunk + 2 (S - 1) positions fit CL_MAX_SPT per
    // thread.
    const int want = p->prec == CHEB_C128 ? std::min(32, *chunk / 4) : std::min(64, *chunk / 2);
    *S = std::max(1, std::min({want, *chunk, 1 + (CL_MAX_SPT * CL_THREADS - *chunk) / 2}));
    const int pos = *chunk + 2 * (*S - 1);
    *threads = std::max(32, std::min(CL_THREADS, (pos + 31) / 32 * 32));
    const int need = (pos + *threads - 1) / *threads;
    *spt = need <= 1 ? 1 : (need <= 2 ? 2 : CL_MAX_SPT);
    *smem = 2 * (size_t)(*chunk + 2 * *S) * p->cplx_size();
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
    int chunk, S, threads, spt, fits = 0;
    size_t smem;
    cluster_shape(p, ctas, &chunk, &S, &threads, &spt, &smem);
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
    int chunk, S, threads, spt;
    size_t smem;
    cluster_shape(p, ctas, &chunk, &S, &threads, &spt, &smem);
    ClusterArgs a{};
    a.psi = psi;
    a.diag = p->d_diag;
    a.qcoef = p->d_qcoef;
    a.blocks = p->d_blocks;
    a.n = (int32_t)p->n_sites;
    a.chunk = chunk;
    a.S = S;
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
