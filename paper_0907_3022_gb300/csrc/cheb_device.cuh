// Device helpers shared by the recurrence kernels (not part of the ABI): complex vector
// types, vector loads, the deterministic block reduction and the per-site accumulation of
// psi with float-float constants.
#pragma once

#include <cuda_runtime.h>

#include "cheb_internal.cuh"

namespace cheb {

// ---- small complex helpers ---------------------------------------------------------------
template <typename R> struct V2;
template <> struct V2<double> {
    using C = double2;
    static __device__ __forceinline__ C make(double x, double y) { return make_double2(x, y); }
};
template <> struct V2<float> {
    using C = float2;
    static __device__ __forceinline__ C make(float x, float y) { return make_float2(x, y); }
};

// Load / store VPT consecutive complex values with the widest aligned accesses.
template <typename R, int VPT> struct VecIO {
    using C = typename V2<R>::C;
    static __device__ __forceinline__ void load(const C* __restrict__ p, C (&o)[VPT]) {
#pragma unroll
        for (int v = 0; v < VPT; ++v) o[v] = p[v];
    }
    static __device__ __forceinline__ void store(C* __restrict__ p, const C (&o)[VPT]) {
#pragma unroll
        for (int v = 0; v < VPT; ++v) p[v] = o[v];
    }
};
template <> struct VecIO<float, 2> {
    static __device__ __forceinline__ void load(const float2* __restrict__ p, float2 (&o)[2]) {
        float4 t = *reinterpret_cast<const float4*>(p);
        o[0] = make_float2(t.x, t.y);
        o[1] = make_float2(t.z, t.w);
    }
    static __device__ __forceinline__ void store(float2* __restrict__ p, const float2 (&o)[2]) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
    }
};
template <> struct VecIO<float, 4> {
    static __device__ __forceinline__ void load(const float2* __restrict__ p, float2 (&o)[4]) {
        float4 t0 = reinterpret_cast<const float4*>(p)[0];
        float4 t1 = reinterpret_cast<const float4*>(p)[1];
        o[0] = make_float2(t0.x, t0.y);
        o[1] = make_float2(t0.z, t0.w);
        o[2] = make_float2(t1.x, t1.y);
        o[3] = make_float2(t1.z, t1.w);
    }
    static __device__ __forceinline__ void store(float2* __restrict__ p, const float2 (&o)[4]) {
        reinterpret_cast<float4*>(p)[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        reinterpret_cast<float4*>(p)[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
    }
};

// ---- deterministic block reduction of NSUM values per thread, grouped by vector group -------
// Threads with the same (threadIdx.x % nvg) hold partials of the same vector group (nvg is a
// power of two <= 32).  Thread t < nvg * NSUM writes the block total of value t % NSUM of
// group t / NSUM to gout[t].  The tree order is fixed, so results are bitwise reproducible.
template <int NSUM>
__device__ __forceinline__ void block_reduce_groups(double (&val)[NSUM], int nvg, double* smem,
                                                    double* gout)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int s = 0; s < NSUM; ++s) {
        double x = val[s];
        for (int off = 16; off >= nvg; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        val[s] = x;
    }
    if (lane < nvg) {
#pragma unroll
        for (int s = 0; s < NSUM; ++s) smem[(warp * nvg + lane) * NSUM + s] = val[s];
    }
    __syncthreads();
    if ((int)threadIdx.x < nvg * NSUM) {
        const int g = threadIdx.x / NSUM, s = threadIdx.x % NSUM;
        double acc = 0.0;
        for (int w = 0; w < nwarps; ++w) acc += smem[(w * nvg + g) * NSUM + s];
        gout[threadIdx.x] = acc;
    }
    __syncthreads();
}

// The same for FP32 per-thread values (complex64 plans): the warp-level tree runs in FP32
// (fixed pairwise order, relative error <= 5 ulp of the warp's sum of magnitudes), the
// block-level sum in FP64.  FP64 arithmetic runs at ~1/64 of the FP32 rate on this GPU, and
// a butterfly of NSUM doubles per thread cost more than the kernels' own site updates.
template <int NSUM>
__device__ __forceinline__ void block_reduce_groups_f(float (&val)[NSUM], int nvg, double* smem,
                                                      double* gout)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int s = 0; s < NSUM; ++s) {
        float x = val[s];
        for (int off = 16; off >= nvg; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        val[s] = x;
    }
    if (lane < nvg) {
#pragma unroll
        for (int s = 0; s < NSUM; ++s) smem[(warp * nvg + lane) * NSUM + s] = (double)val[s];
    }
    __syncthreads();
    if ((int)threadIdx.x < nvg * NSUM) {
        const int g = threadIdx.x / NSUM, s = threadIdx.x % NSUM;
        double acc = 0.0;
        for (int w = 0; w < nwarps; ++w) acc += smem[(w * nvg + g) * NSUM + s];
        gout[threadIdx.x] = acc;
    }
    __syncthreads();
}

// ---- the fused recurrence: shared per-site update ----------------------------------------
// complex64 plans carry the per-block constants (q_k, beta, e^{-i b dt}) as unevaluated sums
// hi + lo of two floats: rounding each to one float would make every step's propagator
// non-unitary by ~1e-7 in the same direction, and the norm would drift linearly in time.
template <typename R> struct Split { static constexpr bool on = false; };
template <> struct Split<float> { static constexpr bool on = true; };

template <typename R>
__device__ __forceinline__ void split_const(double v, R& hi, R& lo)
{
    hi = (R)v;
    lo = Split<R>::on ? (R)(v - (double)hi) : (R)0;
}

template <typename R>
struct SiteUpdate {
    using C = typename V2<R>::C;
    static constexpr bool SP = Split<R>::on;

    // acc += (-i)^k q T  with the sign of (-i)^k folded into q = qh + ql
    static __device__ __forceinline__ void accum(C& acc, const C q, const C t, const int k) {
        if ((k & 1) == 0) {
            if (SP) {
                acc.x = fma(q.y, t.x, acc.x);
                acc.y = fma(q.y, t.y, acc.y);
            }
            acc.x = fma(q.x, t.x, acc.x);
            acc.y = fma(q.x, t.y, acc.y);
        } else {  // -i q t = (q t.y, -q t.x)
            if (SP) {
                acc.x = fma(q.y, t.y, acc.x);
                acc.y = fma(-q.y, t.x, acc.y);
            }
            acc.x = fma(q.x, t.y, acc.x);
            acc.y = fma(-q.x, t.x, acc.y);
        }
    }
    // acc * (ph + pl), ph and pl complex with e^{-i b dt} = ph + pl
    static __device__ __forceinline__ C phase(const C acc, const C ph, const C pl) {
        R rx = 0, ry = 0;
        if (SP) {
            rx = fma(pl.x, acc.x, -pl.y * acc.y);
            ry = fma(pl.x, acc.y, pl.y * acc.x);
        }
        rx = fma(ph.x, acc.x, fma(-ph.y, acc.y, rx));
        ry = fma(ph.x, acc.y, fma(ph.y, acc.x, ry));
        return V2<R>::make(rx, ry);
    }
};

}  // namespace cheb
