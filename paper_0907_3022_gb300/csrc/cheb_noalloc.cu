// Plan-free region norm that allocates no device memory.
//
// Some callers may not allocate device memory at the point where they need a norm:
// latency-critical loops that cannot afford the device-wide synchronisation of cudaMalloc and
// cudaFree, and host programs that own all device memory through their own pool and forbid
// libraries from allocating behind their back.  cheb_region_norm_noalloc serves them: it is
// the per-tile-partials reduction of cheb_observables (CHEB_OBS_NORM2 / CHEB_OBS_PROB_COLS)
// with its scratch in a fixed-size array compiled into the library instead of plan memory.
//
// The scratch is g_noalloc_partials below: CHEB_NOALLOC_MAX_PARTIALS doubles (512 KiB) that
// every GPU which loads the library holds until the process exits.  In host code the
// symbol's name is only a host-side stand-in, so the device address is looked up once per
// device with cudaGetSymbolAddress (on the first call made with that device current) and
// cached.  All calls share the array and it keeps the last call's contents; every slot a call
// reads was written earlier in the same call, so nothing needs clearing, but calls whose
// kernels overlap on the GPU (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "cheb_internal.cuh"

namespace cheb {

static __device__ __align__(256) double g_noalloc_partials[CHEB_NOALLOC_MAX_PARTIALS];

static constexpr int kNoallocTile = 1024;  // sites per CTA
static constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kMaxDevices] = {};

// partials[b * nvec + v] = sum over the sites of tile b with column > col_min of |psi_v|^2
template <typename R>
__global__ void k_region_norm_partials(const void* psi_, int64_t n_sites, int32_t L, int nvec,
                                       int64_t col_min, double* partials)
{
    using C = typename CT<R>::type;
    const C* psi = static_cast<const C*>(psi_);
    __shared__ double s_red[32];
    const int64_t first = (int64_t)blockIdx.x * kNoallocTile;
    const int64_t last = min(first + (int64_t)kNoallocTile, n_sites);
    for (int v = 0; v < nvec; ++v) {
        double acc = 0.0;
        for (int64_t i = first + threadIdx.x; i < last; i += blockDim.x) {
            if (i % L > col_min) {
                const C x = psi[i * nvec + v];
                acc += (double)x.x * x.x + (double)x.y * x.y;
            }
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
            partials[(int64_t)blockIdx.x * nvec + v] = t;
        }
        __syncthreads();
    }
}

// out[v] = sum over the tiles: one warp per vector, lane l sums tiles l, l + 32, ... in order,
// then a fixed xor tree (the summation order depends on the tile count only)
__global__ void k_region_norm_finalize(const double* partials, int ntiles, int nvec, double* out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = warp; v < nvec; v += blockDim.x >> 5) {
        double t = 0.0;
        for (int b = lane; b < ntiles; b += 32) t += partials[(int64_t)b * nvec + v];
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) out[v] = t;
    }
}

// Device address of the scratch array on the current device (looked up once per device).
static int noalloc_scratch(double** out)
{
    int dev = 0;
    CHEB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(CHEB_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        CHEB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partials));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return CHEB_OK;
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_region_norm_noalloc(const void* psi, int prec, int64_t n_sites, int32_t L,
                                        int nvec, int64_t col_min, double* out, void* stream)
{
    if (!psi || !out) return fail(CHEB_ERR_INVALID, "cheb_region_norm_noalloc: NULL pointer");
    if (prec != CHEB_C128 && prec != CHEB_C64) return fail(CHEB_ERR_INVALID, "bad precision");
    if (n_sites < 1 || L < 1 || nvec < 1)
        return fail(CHEB_ERR_INVALID, "cheb_region_norm_noalloc: need n_sites, L, nvec >= 1");
    if (!aligned16(psi) || !aligned16(out))
        return fail(CHEB_ERR_ALIGN, "cheb_region_norm_noalloc: pointers must be 16-byte aligned");
    const int64_t ntiles = (n_sites + kNoallocTile - 1) / kNoallocTile;
    if (ntiles * (int64_t)nvec > CHEB_NOALLOC_MAX_PARTIALS)
        return fail(CHEB_ERR_INVALID,
                    "cheb_region_norm_noalloc: ceil(n_sites/1024) * nvec exceeds "
                    "CHEB_NOALLOC_MAX_PARTIALS (65536); use cheb_observables on a plan");
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == CHEB_C128)
        k_region_norm_partials<double><<<(unsigned)ntiles, 256, 0, s>>>(psi, n_sites, L, nvec,
                                                                          col_min, scratch);
    else
        k_region_norm_partials<float><<<(unsigned)ntiles, 256, 0, s>>>(psi, n_sites, L, nvec,
                                                                         col_min, scratch);
    CHEB_CUDA(cudaGetLastError());
    k_region_norm_finalize<<<1, 256, 0, s>>>(scratch, (int)ntiles, nvec, out);
    CHEB_CUDA(cudaGetLastError());
    return CHEB_OK;
}
