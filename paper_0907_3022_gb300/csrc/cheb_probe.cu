// Micro-kernels that measure the peaks the roofline of a kernel is quoted against when no
// external figure exists for them: the shared-memory load bandwidth of the whole GPU, and the
// FP64 and FP32 fused multiply-add rates.  The paper has no counterpart (measurement only).
//
// Each probe runs a fixed amount of work on every SM (grid = SMs x resident CTAs), timed with
// CUDA events on the caller's stream after one warm-up launch; the best of three timed
// launches is reported.  The loops carry enough independent work per thread to keep the unit
// busy, and their results feed one conditional store so that nothing is optimised away.
#include <cuda_runtime.h>

#include <algorithm>

#include "cheb_internal.cuh"

namespace cheb {

static constexpr int PROBE_SMEM_THREADS = 1024;
static constexpr int PROBE_SMEM_ELEMS = 2048;  // float4 elements: 32 KiB per CTA
static constexpr int PROBE_SMEM_ITERS = 2048;

// Every thread reads 16-byte elements at (tid + 512 j + 32 it) mod 2048: consecutive lanes read
// consecutive elements, so a warp's request touches each bank four times (the minimum for
// 512 bytes) and the loads stream at the shared-memory pipe's rate.
__global__ void __launch_bounds__(PROBE_SMEM_THREADS) k_probe_smem(float* sink, int iters)
{
    __shared__ float4 buf[PROBE_SMEM_ELEMS];
    for (int i = threadIdx.x; i < PROBE_SMEM_ELEMS; i += blockDim.x)
        buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    int idx = threadIdx.x;
    for (int it = 0; it < iters; ++it) {
        // four independent loads per iteration, combined with integer-exact adds
        const float4 x0 = buf[idx];
        const float4 x1 = buf[(idx + 512) & (PROBE_SMEM_ELEMS - 1)];
        const float4 x2 = buf[(idx + 1024) & (PROBE_SMEM_ELEMS - 1)];
        const float4 x3 = buf[(idx + 1536) & (PROBE_SMEM_ELEMS - 1)];
        a0.x += x0.x; a0.y += x0.y; a0.z += x0.z; a0.w += x0.w;
        a1.x += x1.x; a1.y += x1.y; a1.z += x1.z; a1.w += x1.w;
        a2.x += x2.x; a2.y += x2.y; a2.z += x2.z; a2.w += x2.w;
        a3.x += x3.x; a3.y += x3.y; a3.z += x3.z; a3.w += x3.w;
        idx = (idx + 32) & (PROBE_SMEM_ELEMS - 1);
    }
    const float s = a0.x + a0.y + a0.z + a0.w + a1.x + a1.y + a1.z + a1.w + a2.x + a2.y + a2.z +
                    a2.w + a3.x + a3.y + a3.z + a3.w;
    if (s == -1.f) sink[0] = s;  // never true: keeps the loads
}

// FMA chains: 8 independent accumulators per thread, x = x * m + c
template <typename R>
__global__ void __launch_bounds__(256) k_probe_fma(R* sink, int iters, R m, R c)
{
    R x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (R)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], m, c);
    }
    R s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == (R)-1) sink[0] = s;
}

static int probe_time(cudaStream_t s, int kind, int sms, float* sink, double* value)
{
    cudaEvent_t e0, e1;
    CHEB_CUDA(cudaEventCreate(&e0));
    CHEB_CUDA(cudaEventCreate(&e1));
    double best = 0.0;
    int rc = CHEB_OK;
    for (int rep = 0; rep < 4 && !rc; ++rep) {  // rep 0 warms up
        double work = 0.0;
        cudaError_t e = cudaEventRecord(e0, s);
        if (kind == CHEB_PEAK_SMEM_LOAD_GBS) {
            const int grid = sms * 2;  // two 1024-thread CTAs per SM (32 KiB each)
            k_probe_smem<<<grid, PROBE_SMEM_THREADS, 0, s>>>(sink, PROBE_SMEM_ITERS);
            work = (double)grid * PROBE_SMEM_THREADS * PROBE_SMEM_ITERS * 4 * 16;  // bytes
        } else if (kind == CHEB_PEAK_FP64_GFLOPS) {
            const int grid = sms * 8, iters = 4096;
            k_probe_fma<double><<<grid, 256, 0, s>>>(reinterpret_cast<double*>(sink), iters,
                                                     0.999999, 1e-7);
            work = (double)grid * 256 * iters * 8 * 2;  // flops
        } else {
            const int grid = sms * 8, iters = 16384;
            k_probe_fma<float><<<grid, 256, 0, s>>>(sink, iters, 0.999999f, 1e-7f);
            work = (double)grid * 256 * iters * 8 * 2;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "peak probe");
            break;
        }
        if (rep > 0 && ms > 0.f) best = std::max(best, work / (ms * 1e-3) / 1e9);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) *value = best;
    return rc;
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_measure_peak(int kind, void* stream, double* value)
{
    if (!value) return fail(CHEB_ERR_INVALID, "cheb_measure_peak: NULL value");
    if (kind != CHEB_PEAK_SMEM_LOAD_GBS && kind != CHEB_PEAK_FP64_GFLOPS &&
        kind != CHEB_PEAK_FP32_GFLOPS)
        return fail(CHEB_ERR_INVALID, "cheb_measure_peak: unknown kind");
    int dev = 0, sms = 0;
    CHEB_CUDA(cudaGetDevice(&dev));
    CHEB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* sink = nullptr;
    CHEB_CUDA(cudaMalloc(&sink, 64));
    const int rc = probe_time(static_cast<cudaStream_t>(stream), kind, sms, sink, value);
    cudaFree(sink);
    return rc;
}
