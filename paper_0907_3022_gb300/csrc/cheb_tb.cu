// Temporally blocked Chebyshev recurrence for complex64 brick-wall stencils (Sec. 2.2,
// Eqs. U_1 and rec; ribbons of Sec. 3.2, the 1D grid as W = 1).
//
// One launch forms s consecutive orders k = ka .. kb for every ribbon.  A CTA owns a tile
// of one ribbon: the interior [r0, r1) x [c0, c1) plus a halo on every side that is not a
// ribbon edge (the region [R0, R1) x [C0, C1)): s columns left and right, ceil(s / 2) rows
// above and below, since on the brick wall a site d rows away is at least 2d - 1 bonds away.
// It loads T_{ka-2}, T_{ka-1} and the on-site data d of the region into shared memory once,
// then runs the s recurrence orders there: the i-th order is computed at the sites whose
// bond distance to the open sides exceeds i, which is exactly where its inputs are still
// valid, and the interior keeps all s.  The
// weighted sum of the s new orders for the interior sites stays in registers.  At the end
// the interior's last two vectors go to the other global buffer pair (the neighbouring CTAs
// are still reading this pair as their halo) and the partial sum goes to an accumulator:
//   E   (main accumulator)  for launches that start at an order <= ksplit,
//   tail                    for launches that start later (|q_k| < 2^-8, see cheb_kernels.cu),
// and psi = e^{-i b dt} (E + tail + partial) at the launch holding the ribbon's last order M.
// psi itself is read only by the first launch (as T_0) and written only at order M; the
// first launch never holds order M (the host keeps s_0 < min M).
//
// Per site and s orders the launch moves 2 vectors + d of the region in and 2 vectors of
// the interior out, plus the accumulator: about (2 nv 8 + 4) * halo + 3 nv 8 bytes instead
// of s * (5 nv 8 + 4) for s single-order launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "cheb_internal.cuh"

namespace cheb {

// Shared memory of one CTA: two float2 planes per vector and the float on-site plane, for a
// region of TPB * SPT sites (plus one zero element per plane).
__host__ __device__ constexpr size_t tb_smem(int nv, int spt, int tpb)
{
    // each plane holds tpb * spt sites and one zero element (the neighbour outside a ribbon)
    return 2 * (size_t)nv * ((size_t)tpb * spt + 1) * sizeof(float2) + (size_t)tpb * spt * sizeof(float);
}

// CTAs per SM the launch bounds ask for: 256-thread CTAs as tuned (3 up to 4 sites per
// thread, else 2); larger CTAs as many as shared memory (227 KB per SM) and the 2048-thread
// limit allow
__host__ __device__ constexpr int tb_min_blocks(int nv, int spt, int tpb)
{
    if (tpb == 256) return spt <= 4 ? 3 : 2;
    const size_t by_smem = 232448 / (tb_smem(nv, spt, tpb) + 1024);
    const size_t by_threads = 2048 / tpb;
    const size_t b = by_smem < by_threads ? by_smem : by_threads;
    return b < 1 ? 1 : (int)b;
}

// The last halo shrink (order index within the launch) at which region position (rr, cc) of an
// RH x RW region is still formed: its bond distance to the region's open sides less one.  A
// site d rows from an open row side is 2d - 1 bonds from it when its vertical bond points that
// way, else 2d (the vertical bonds alternate), so rows stay valid about twice as long as
// columns.  1 << 20 where no side is open.  Used by the kernels and by the host work model.
__host__ __device__ __forceinline__ int tb_limit(int rr, int cc, int RH, int RW, bool up,
                                                 bool open_t, bool open_b, bool open_l,
                                                 bool open_r)
{
    int dl = 1 << 20;
    if (open_t) dl = min(dl, 2 * rr + (up ? 0 : 1));
    if (open_b) dl = min(dl, 2 * (RH - 1 - rr) + (up ? 1 : 0));
    if (open_l) dl = min(dl, cc);
    if (open_r) dl = min(dl, RW - 1 - cc);
    return dl;
}

// Shared-memory planes: one float2 plane for a single vector, else one float4 plane per pair
// of vectors (vectors 2p and 2p + 1 of a site side by side), so that region loads, neighbour
// reads and stores move 16 bytes at a time.
template <int NV> struct TBPlane {
    using T = float4;
    static constexpr int NP = NV / 2;  // planes
    static constexpr int PER = 2;      // vectors per plane element
};
template <> struct TBPlane<1> {
    using T = float2;
    static constexpr int NP = 1;
    static constexpr int PER = 1;
};

__device__ __forceinline__ float2 tb_get(const float2& t, int) { return t; }
__device__ __forceinline__ float2 tb_get(const float4& t, int c)
{
    return c ? make_float2(t.z, t.w) : make_float2(t.x, t.y);
}
__device__ __forceinline__ void tb_set(float2& t, int, const float2 v) { t = v; }
__device__ __forceinline__ void tb_set(float4& t, int c, const float2 v)
{
    if (c) {
        t.z = v.x;
        t.w = v.y;
    } else {
        t.x = v.x;
        t.y = v.y;
    }
}
template <typename T> __device__ __forceinline__ T tb_zero();
template <> __device__ __forceinline__ float2 tb_zero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ float4 tb_zero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// split of a double into hi + lo floats
__device__ __forceinline__ void tb_split(double x, float& hi, float& lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// acc += (-i)^k q T with the sign of (-i)^k folded into q = (hi, lo)
__device__ __forceinline__ void tb_accum(float2& acc, const float2 q, const float2 t, const int k)
{
    if ((k & 1) == 0) {
        acc.x = fmaf(q.y, t.x, acc.x);
        acc.y = fmaf(q.y, t.y, acc.y);
        acc.x = fmaf(q.x, t.x, acc.x);
        acc.y = fmaf(q.x, t.y, acc.y);
    } else {
        acc.x = fmaf(q.y, t.y, acc.x);
        acc.y = fmaf(-q.y, t.x, acc.y);
        acc.x = fmaf(q.x, t.y, acc.x);
        acc.y = fmaf(-q.x, t.x, acc.y);
    }
}

__device__ __forceinline__ float2 tb_phase(const float2 a, const float2 ph, const float2 pl)
{
    float rx = fmaf(pl.x, a.x, -pl.y * a.y);
    float ry = fmaf(pl.x, a.y, pl.y * a.x);
    rx = fmaf(ph.x, a.x, fmaf(-ph.y, a.y, rx));
    ry = fmaf(ph.x, a.y, fmaf(ph.y, a.x, ry));
    return make_float2(rx, ry);
}

// asynchronous global -> shared copies (no registers in between)
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_el(float2* sdst, const float2* gsrc) { cp_async8(sdst, gsrc); }
__device__ __forceinline__ void cp_async_el(float4* sdst, const float4* gsrc) { cp_async16(sdst, gsrc); }
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <int NV, int SPT, bool FIRST, int TPB>
__global__ void __launch_bounds__(TPB, tb_min_blocks(NV, SPT, TPB)) k_rec_tb(TBArgs a)
{
    using PT = typename TBPlane<NV>::T;
    constexpr int NP = TBPlane<NV>::NP, PER = TBPlane<NV>::PER;
    constexpr int TB_THREADS = TPB;
    constexpr int RMAX = TB_THREADS * SPT;
    constexpr int RP = RMAX + 1;  // plane stride; element RMAX of every plane stays zero
    extern __shared__ float4 tb_smem_raw[];
    PT* const sP0 = reinterpret_cast<PT*>(tb_smem_raw);       // [NP][RP]
    PT* const sQ0 = sP0 + NP * RP;                              // [NP][RP]
    float* const sD = reinterpret_cast<float*>(sQ0 + NP * RP);  // [RMAX]
    __shared__ double s_red[(TB_THREADS / 32) * 2 * NV];

    // global vectors seen as NP plane elements per site
    const PT* __restrict__ in_prev = static_cast<const PT*>(a.in_prev);
    const PT* __restrict__ in_cur = static_cast<const PT*>(a.in_cur);
    PT* __restrict__ out_prev = static_cast<PT*>(a.out_prev);
    PT* __restrict__ out_cur = static_cast<PT*>(a.out_cur);
    PT* __restrict__ accE = static_cast<PT*>(a.acc_main);
    PT* __restrict__ tail = static_cast<PT*>(a.tail);
    PT* __restrict__ psi = static_cast<PT*>(a.psi);
    const float* __restrict__ diag = static_cast<const float*>(a.diag);
    const float2* __restrict__ qc = static_cast<const float2*>(a.qcoef);
    const int tid = threadIdx.x;
    constexpr bool first = FIRST;  // ka == 1: T_0 = psi, no T_{-1}; norm and energy partials
    if (tid < 2 * NP) sP0[(tid / NP) * NP * RP + (tid % NP) * RP + RMAX] = tb_zero<PT>();

    for (int w = blockIdx.x; w < a.ntiles; w += gridDim.x) {
        const TBTile T = a.tiles[w];
        const DevBlock B = a.blocks[T.block];
        // per-thread norm / energy terms of the first launch: a thread sums only its SPT
        // sites, in FP32 (FP64 arithmetic is ~1/32 the FP32 rate on this GPU); the block and
        // grid reductions that follow are FP64
        float part[FIRST ? 2 * NV : 1];
#pragma unroll
        for (int q = 0; q < (FIRST ? 2 * NV : 1); ++q) part[q] = 0.f;
        if (a.ka <= B.M) {
            const int ke = min(a.kb, B.M);
            const bool done = (ke == B.M);
            const int RW = T.C1 - T.C0, RH = T.R1 - T.R0;
            const int nreg = RW * RH;
            // idx / RW as (idx * ceil(2^32 / RW)) >> 32: exact because idx * (RW - 1) stays far
            // below 2^32 (idx < RMAX <= 8192)
            const unsigned long long invRW = ((1ull << 32) + (unsigned)RW - 1u) / (unsigned)RW;
            const bool open_t = T.R0 > 0, open_b = T.R1 < B.W, open_l = T.C0 > 0, open_r = T.C1 < B.L;
            // per position tid + j * TPB of the row-major region: the shared-memory indices of
            // its three neighbours (RMAX, the zero element, where the ribbon has none) and
            // the last halo shrink at which it is still computed (its distance to the open
            // sides of the region; -1 outside the region)
            int nbl[SPT], nbr[SPT], nbv[SPT], dlim[SPT];
            bool inter[SPT];
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
                const int idx = tid + j * TB_THREADS;
                const int rr = (int)(((unsigned long long)idx * invRW) >> 32), cc = idx - rr * RW;
                const int r = T.R0 + rr, c = T.C0 + cc;
                const bool up = (r + c) & 1;  // vertical neighbour r-1 (else r+1)
                nbl[j] = c > 0 ? idx - 1 : RMAX;
                nbr[j] = c + 1 < B.L ? idx + 1 : RMAX;
                nbv[j] = up ? (r > 0 ? idx - RW : RMAX) : (r + 1 < B.W ? idx + RW : RMAX);
                // sites never computed (limit 0) never read their neighbours
                dlim[j] = idx < nreg ? tb_limit(rr, cc, RH, RW, up, open_t, open_b, open_l, open_r)
                                     : -1;
                inter[j] = idx < nreg && (r >= T.r0) && (r < T.r1) && (c >= T.c0) && (c < T.c1);
            }
            // ---- load the region: asynchronous copies straight into shared memory ---------
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
                const int idx = tid + j * TB_THREADS;
                if (idx < nreg) {
                    const int rr = (int)(((unsigned long long)idx * invRW) >> 32), cc = idx - rr * RW;
                    const int64_t g = B.offset + (int64_t)(T.R0 + rr) * B.L + (T.C0 + cc);
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        cp_async_el(&sQ0[p * RP + idx], &in_cur[g * NP + p]);
                        if (first) sP0[p * RP + idx] = tb_zero<PT>();
                        else cp_async_el(&sP0[p * RP + idx], &in_prev[g * NP + p]);
                    }
                    cp_async4(&sD[idx], &diag[g]);
                }
            }
            float2 acc[SPT][NV];
            const bool to_main = first || (a.ka <= B.ksplit);
            const bool tail_has = a.prev_ka > B.ksplit;  // an earlier launch wrote the tail
            // the accumulator this launch continues, read now so that its latency hides behind
            // the region copies: E (main), the tail, or E + tail at the ribbon's last order
            const bool read_e = !first && (to_main || done);
            const bool read_t = !first && !to_main && tail_has;
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
                PT eP[NP], tP[NP];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    eP[p] = tb_zero<PT>();
                    tP[p] = tb_zero<PT>();
                }
                if (inter[j] && (read_e || read_t)) {
                    const int idx = tid + j * TB_THREADS;
                    const int rr = (int)(((unsigned long long)idx * invRW) >> 32), cc = idx - rr * RW;
                    const int64_t g = B.offset + (int64_t)(T.R0 + rr) * B.L + (T.C0 + cc);
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (read_e) eP[p] = accE[g * NP + p];
                        if (read_t) tP[p] = tail[g * NP + p];
                    }
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) {
#pragma unroll
                    for (int cv = 0; cv < PER; ++cv) {
                        const float2 e = tb_get(eP[p], cv), t2 = tb_get(tP[p], cv);
                        // the tail alone for a tail launch; E + tail when the ribbon ends here
                        acc[j][p * PER + cv] = (read_e && read_t)
                                                   ? make_float2(e.x + t2.x, e.y + t2.y)
                                                   : (read_t ? t2 : e);
                    }
                }
            }
            const float bh = (float)B.beta;  // exact: complex64 lattice plans choose a so
            cp_async_wait_all();
            __syncthreads();
            float dreg[SPT];  // the on-site values of this thread's sites, read once per tile
#pragma unroll
            for (int j = 0; j < SPT; ++j) dreg[j] = sD[min(tid + j * TB_THREADS, RMAX - 1)];
            if (first) {  // q_0 T_0
                const float2 q0 = qc[B.coef_off + 0];
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    if (!inter[j]) continue;
                    const int idx = tid + j * TB_THREADS;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const PT x = sQ0[p * RP + idx];
#pragma unroll
                        for (int c = 0; c < PER; ++c) tb_accum(acc[j][p * PER + c], q0, tb_get(x, c), 0);
                    }
                }
            }
            // ---- s recurrence orders in shared memory -------------------------------------
            PT* sP = sP0;
            PT* sQ = sQ0;
            float2 qn = qc[B.coef_off + a.ka];  // q_k read one order ahead
            for (int k = a.ka; k <= ke; ++k) {
                const int sh = k - a.ka + 1;  // order k is computed on the region shrunk by sh
                const float2 qk = qn;
                if (k < ke) qn = qc[B.coef_off + k + 1];
                PT* __restrict__ Pw = sP;        // T_{k-2} in, T_k out (own site only)
                const PT* __restrict__ Qr = sQ;  // T_{k-1}, read at the site and neighbours
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    if (dlim[j] < sh) continue;
                    const int idx = tid + j * TB_THREADS;
                    const float d = dreg[j];
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const PT* Q = Qr + p * RP;
                        const PT xP = Q[idx];
                        const PT ylP = Q[nbl[j]];
                        const PT yrP = Q[nbr[j]];
                        const PT yvP = Q[nbv[j]];
                        const PT pP = Pw[p * RP + idx];
                        PT hP;
#pragma unroll
                        for (int cv = 0; cv < PER; ++cv) {
                            const float2 x = tb_get(xP, cv), yl = tb_get(ylP, cv);
                            const float2 yr = tb_get(yrP, cv), yv = tb_get(yvP, cv);
                            const float2 pv = tb_get(pP, cv);
                            const float sx = (yl.x + yr.x) + yv.x;
                            const float sy = (yl.y + yr.y) + yv.y;
                            // beta is a float32 number in complex64 lattice plans
                            float hx = fmaf(bh, sx, -pv.x), hy = fmaf(bh, sy, -pv.y);
                            hx = fmaf(d, x.x, hx);
                            hy = fmaf(d, x.y, hy);
                            if (k == 1) {  // T_1 = H~ T_0 (p = 0)
                                hx *= 0.5f;
                                hy *= 0.5f;
                            }
                            const float2 h = make_float2(hx, hy);
                            tb_set(hP, cv, h);
                            if (inter[j]) {
                                const int v = p * PER + cv;
                                tb_accum(acc[j][v], qk, h, k);
                                if constexpr (FIRST) {
                                    if (k == 1) {
                                        part[2 * v + 0] = fmaf(x.x, x.x, fmaf(x.y, x.y, part[2 * v + 0]));
                                        part[2 * v + 1] = fmaf(x.x, h.x, fmaf(x.y, h.y, part[2 * v + 1]));
                                    }
                                }
                            }
                        }
                        Pw[p * RP + idx] = hP;
                    }
                }
                __syncthreads();
                PT* tmp = sP;
                sP = sQ;
                sQ = tmp;
            }
            // ---- write back: sQ = T_ke, sP = T_{ke-1} ----------------------------------------
            float lim4[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v)
                lim4[v] = done ? (float)(4.0 * a.norm2[((size_t)T.block * NV + v) * 2]) : 0.f;
            float2 ph, pl;
            tb_split(B.ph_re, ph.x, pl.x);
            tb_split(B.ph_im, ph.y, pl.y);
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
                if (!inter[j]) continue;
                const int idx = tid + j * TB_THREADS;
                const int rr = (int)(((unsigned long long)idx * invRW) >> 32), cc = idx - rr * RW;
                const int64_t g = B.offset + (int64_t)(T.R0 + rr) * B.L + (T.C0 + cc);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const PT tkP = sQ[p * RP + idx];
                    PT aP;
#pragma unroll
                    for (int cv = 0; cv < PER; ++cv) tb_set(aP, cv, acc[j][p * PER + cv]);
                    if (!done) {
                        out_cur[g * NP + p] = tkP;
                        out_prev[g * NP + p] = sP[p * RP + idx];
                        if (to_main) accE[g * NP + p] = aP;
                        else tail[g * NP + p] = aP;
                    } else {
                        PT oP;
#pragma unroll
                        for (int cv = 0; cv < PER; ++cv) {
                            const int v = p * PER + cv;
                            tb_set(oP, cv, tb_phase(acc[j][v], ph, pl));  // E + tail + partial
                            // growth check |T_M|^2 <= 4 ||psi||^2, in FP32 (a divergence test)
                            const float2 tk = tb_get(tkP, cv);
                            const float t2 = fmaf(tk.x, tk.x, tk.y * tk.y);
                            if (!(t2 <= lim4[v])) atomicOr(a.errflag, 1);
                        }
                        psi[g * NP + p] = oP;
                    }
                }
            }
        }
        if constexpr (FIRST) {
            // per-tile partials of ||T_0||^2 and <T_0|H~ T_0>, fixed-order reduction: FP32
            // tree inside each warp (FP64 runs at ~1/64 of the FP32 rate here), FP64 across
            // the warps
            const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
            for (int q = 0; q < 2 * NV; ++q) {
                float xs = part[q];
                for (int off = 16; off > 0; off >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, off);
                if (lane == 0) s_red[warp * 2 * NV + q] = (double)xs;
            }
            __syncthreads();
            if (tid < 2 * NV) {
                double t = 0.0;
                for (int q = 0; q < TB_THREADS / 32; ++q) t += s_red[q * 2 * NV + tid];
                a.partials[(size_t)w * NV * 2 + tid] = t;
            }
        }
        __syncthreads();  // shared memory is reused by the next tile
    }
    if constexpr (FIRST) {
        __shared__ unsigned int s_last;
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = (atomicAdd(a.done_counter, 1u) == gridDim.x - 1) ? 1u : 0u;
        __syncthreads();
        if (s_last) {
            __threadfence();
            // one warp per (ribbon, vector) slot: lane l sums tiles l, l + 32, ..., then a
            // fixed xor tree (the order depends on the tile count only, not on timing)
            const int lane = tid & 31, warp = tid >> 5;
            for (int slot = warp; slot < a.nblocks * NV; slot += TB_THREADS / 32) {
                const int q = slot / NV, v = slot % NV;
                const int it1 = a.block_tile_begin[q + 1];
                double n2 = 0.0, eh = 0.0;
#pragma unroll 4
                for (int it = a.block_tile_begin[q] + lane; it < it1; it += 32) {
                    n2 += __ldcg(a.partials + ((size_t)it * NV + v) * 2 + 0);
                    eh += __ldcg(a.partials + ((size_t)it * NV + v) * 2 + 1);
                }
                for (int off = 16; off > 0; off >>= 1) {
                    n2 += __shfl_xor_sync(0xffffffffu, n2, off);
                    eh += __shfl_xor_sync(0xffffffffu, eh, off);
                }
                if (lane == 0) {
                    const DevBlock Bq = a.blocks[q];
                    a.red_out[(size_t)slot * 2 + 0] = n2;
                    a.red_out[(size_t)slot * 2 + 1] = Bq.a * eh + Bq.b * n2;
                }
            }
            if (tid == 0) *a.done_counter = 0u;
        }
    }
}

size_t tb_smem_bytes(int nv, int spt, int tpb) { return tb_smem(nv, spt, tpb); }

template <int NV, int SPT, int TPB>
static int tb_launch_t(const TBArgs& a, int grid, cudaStream_t s)
{
    const size_t smem = tb_smem(NV, SPT, TPB);
    if (a.ka == 1) k_rec_tb<NV, SPT, true, TPB><<<grid, TPB, smem, s>>>(a);
    else k_rec_tb<NV, SPT, false, TPB><<<grid, TPB, smem, s>>>(a);
    CHEB_CUDA(cudaGetLastError());
    return CHEB_OK;
}

template <int NV, int SPT, int TPB>
static int tb_attr_t()
{
    const int smem = (int)tb_smem(NV, SPT, TPB);
    CHEB_CUDA(cudaFuncSetAttribute(k_rec_tb<NV, SPT, true, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CHEB_CUDA(cudaFuncSetAttribute(k_rec_tb<NV, SPT, false, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return CHEB_OK;
}

// The (vectors, sites per thread, threads per CTA) shapes compiled: regions of 256 x 4..8
// sites (2-3 CTAs per SM) and one large CTA per SM (512 or 1024 threads) with the largest
// region the shared memory holds for the vector count.
#define CHEB_TB_SHAPES(X)                                                                  \
    X(4, 4, 256) X(2, 4, 256) X(1, 4, 256) X(4, 6, 256) X(2, 6, 256) X(1, 6, 256)          \
    X(2, 8, 256) X(1, 8, 256) X(4, 3, 512) X(4, 4, 512) X(4, 6, 512) X(4, 2, 1024)         \
    X(4, 3, 1024) X(2, 6, 1024) X(1, 8, 1024)

bool tb_supported(int nv, int spt, int tpb)
{
#define CHEB_TB_IS(NV, SPT, TPB) if (nv == NV && spt == SPT && tpb == TPB) return true;
    CHEB_TB_SHAPES(CHEB_TB_IS)
#undef CHEB_TB_IS
    return false;
}

// Allow the dynamic shared memory of the (nv, spt, tpb) instantiation; called while the
// schedule is prepared, outside any stream capture.
int tb_configure(int nv, int spt, int tpb)
{
#define CHEB_TB_ATTR(NV, SPT, TPB) if (nv == NV && spt == SPT && tpb == TPB) return tb_attr_t<NV, SPT, TPB>();
    CHEB_TB_SHAPES(CHEB_TB_ATTR)
#undef CHEB_TB_ATTR
    return fail(CHEB_ERR_UNSUPPORTED, "temporal blocking: unsupported nvec / sites per thread / threads");
}

int tb_launch(Plan* p, const TBArgs& a, cudaStream_t s)
{
    int grid = a.ntiles;
    if (p->tb_grid_cap > 0 && grid > p->tb_grid_cap) grid = p->tb_grid_cap;
    if (grid < 1) return CHEB_OK;
    int rc = CHEB_ERR_UNSUPPORTED;
    const int nv = p->nvec, spt = p->tb_spt, tpb = p->tb_tpb;
#define CHEB_TB_GO(NV, SPT, TPB) if (nv == NV && spt == SPT && tpb == TPB) rc = tb_launch_t<NV, SPT, TPB>(a, grid, s); else
    CHEB_TB_SHAPES(CHEB_TB_GO) {}
#undef CHEB_TB_GO
    if (rc == CHEB_ERR_UNSUPPORTED)
        return fail(rc, "temporal blocking: unsupported nvec / sites per thread / threads");
    p->launches++;
    return rc;
}

// Widest region row that fits rmax positions with rh rows: rmax / rh sites per row, or with
// padded rows (align > 0; the register-run kernel) a row stride that is a multiple of align
// and leaves at least one zero pad after every row, with one position to spare.
static int tb_width_cap(int rmax, int rh, int align)
{
    if (align <= 0) return rmax / rh;
    return (((rmax - 1) / rh) & ~(align - 1)) - 1;
}

// Tiles for a halo of s: row bands chosen for the least halo waste, then as many interior
// columns as the region budget (rmax positions: threads * sites per thread) allows.  Returns
// false if a ribbon cannot be tiled (the region of one interior column would not fit).
bool tb_tiles_of_ribbon(int W, int L, int s, int rmax, int block, std::vector<TBTile>& tiles,
                        int align, bool uniform)
{
    // halo widths for s orders: s columns, but only ceil(s / 2) rows, since d rows away is at
    // least 2d - 1 bonds on the brick wall (the kernel's validity distance counts the same way)
    const int hr = (s + 1) / 2;
    // row bands: pick the band count whose tiles waste the least region on halos
    int best_nbr = -1;
    double best_eff = 0.0;
    for (int nbr = 1; nbr <= W; ++nbr) {
        const int tr = (W + nbr - 1) / nbr;
        const int rh = std::min(W, tr + (nbr > 1 ? 2 * hr : 0));  // worst band
        const int wcap = tb_width_cap(rmax, rh, align);
        const int tcmax = wcap - (L > wcap ? 2 * s : 0);
        if (tcmax < 1) continue;
        const int tc = std::min(tcmax, L);
        const double eff = (double)tr * tc / ((double)rh * (tc + (L > tc ? 2 * s : 0)));
        if (eff > best_eff * 1.02) {
            best_eff = eff;
            best_nbr = nbr;
        }
        if (tr <= 2 * hr) break;
    }
    if (best_nbr < 0) return false;
    const int tr = (W + best_nbr - 1) / best_nbr;
    // padded regions for boxes: every band takes its width from the tallest band's height, so
    // that one row stride and one box of (stride x tallest rows) fit every tile of the ribbon
    const int rh_max = std::min(W, tr + (best_nbr > 1 ? 2 * hr : 0));
    const size_t first_tile = tiles.size();
    for (int r0 = 0; r0 < W; r0 += tr) {
        const int r1 = std::min(W, r0 + tr);
        const int R0 = std::max(0, r0 - hr), R1 = std::min(W, r1 + hr);
        const int rh = R1 - R0;
        int tc = tb_width_cap(rmax, uniform ? rh_max : rh, align);
        if (tc < L) tc -= 2 * s;  // halo on both column sides
        if (tc < 1) return false;
        const int nbc = (L + tc - 1) / tc;
        tc = (L + nbc - 1) / nbc;
        for (int c0 = 0; c0 < L; c0 += tc) {
            const int c1 = std::min(L, c0 + tc);
            TBTile t{};
            t.block = block;
            t.R0 = R0;
            t.R1 = R1;
            t.C0 = std::max(0, c0 - s);
            t.C1 = std::min(L, c1 + s);
            t.r0 = r0;
            t.r1 = r1;
            t.c0 = c0;
            t.c1 = c1;
            const int64_t RW = t.C1 - t.C0, RH = t.R1 - t.R0;
            const int64_t S = align > 0 ? (RW + align) & ~(int64_t)(align - 1) : RW;
            const int64_t used = align > 0 ? 1 + RH * S : RH * RW;
            if (RW < 1 || used > rmax) return false;
            t.S = (int32_t)S;
            t.BH = (int32_t)RH;
            tiles.push_back(t);
        }
    }
    if (align > 0 && uniform) {  // the ribbon's common stride and box height
        int S = 0, BH = 0;
        for (size_t i = first_tile; i < tiles.size(); ++i) {
            S = std::max(S, (tiles[i].C1 - tiles[i].C0 + align) & ~(align - 1));
            BH = std::max(BH, tiles[i].R1 - tiles[i].R0);
        }
        if (1 + (int64_t)BH * S > rmax) return false;
        for (size_t i = first_tile; i < tiles.size(); ++i) {
            tiles[i].S = S;
            tiles[i].BH = BH;
        }
    }
    return true;
}

bool tb_build_tiles(const Plan* p, int s, std::vector<TBTile>& tiles, std::vector<int32_t>& begin)
{
    const int rmax = p->tb_tpb * p->tb_spt;
    const bool runs = p->tb_kernel == CHEB_TB_RUNS || p->tb_kernel == CHEB_TB_RUNS_TMA;
    const bool boxes_wanted = p->tb_kernel == CHEB_TB_RUNS_TMA && p->nvec >= 2;
    const int align = runs ? (p->nvec >= 2 ? 4 : 8) : 0;
    tiles.clear();
    begin.assign(p->nblocks + 1, 0);
    for (int q = 0; q < p->nblocks; ++q) {
        begin[q] = (int32_t)tiles.size();
        const DevBlock& B = p->hblocks[q];
        const size_t t0 = tiles.size();
        if (!tb_tiles_of_ribbon(B.W, B.L, s, rmax, q, tiles, align, boxes_wanted)) return false;
        // register-run kernel with boxes, pairs of vectors: boxes of (stride x rows) up to
        // 256 x 256
        const bool boxes = boxes_wanted && tiles[t0].S <= 256 && tiles[t0].BH <= 256 &&
                           tbr_tma_available();
        for (size_t i = t0; i < tiles.size(); ++i) tiles[i].tma = boxes ? 1 : 0;
    }
    begin[p->nblocks] = (int32_t)tiles.size();
    return true;
}

// Host work model of one blocked launch (cheb_plan_step_model): the tiles of set `tiles`
// forming orders ka..kb, counted the way k_rec_tb runs them.
void tb_model_launch(const Plan* p, const std::vector<TBTile>& tiles, int ka, int kb,
                     int prev_ka, TBModel& m)
{
    const int nv = p->nvec;
    const double pt = nv >= 2 ? 16.0 : 8.0;  // bytes of one plane element
    const double np = nv >= 2 ? nv / 2 : 1;   // planes
    const int rmax = p->tb_tpb * p->tb_spt;
    const bool first = ka == 1;
    for (const TBTile& T : tiles) {
        const DevBlock& B = p->hblocks[T.block];
        if (ka > B.M) continue;
        const int ke = std::min(kb, (int)B.M), ns = ke - ka + 1;
        const bool done = ke == B.M;
        const int RW = T.C1 - T.C0, RH = T.R1 - T.R0;
        const double nreg = (double)RW * RH;
        const double inter = (double)(T.r1 - T.r0) * (T.c1 - T.c0);
        const bool ot = T.R0 > 0, ob = T.R1 < B.W, ol = T.C0 > 0, orr = T.C1 < B.L;
        double computed = 0.0;
        for (int rr = 0; rr < RH; ++rr)
            for (int cc = 0; cc < RW; ++cc) {
                const bool up = ((T.R0 + rr) + (T.C0 + cc)) & 1;
                computed += std::min(ns, tb_limit(rr, cc, RH, RW, up, ot, ob, ol, orr));
            }
        m.useful += inter * ns;
        m.computed += computed;
        // per formed site-order and plane: own site, three neighbours and T_{k-2} read, T_k
        // written; region copies (two planes and d in; the first launch zeroes T_{-1}); the
        // on-site values read once per thread slot; q_0 T_0 (first launch); the interior read
        // back for the write-out (both vectors, or T_M only at the ribbon's last order)
        m.smem += computed * np * 6.0 * pt + nreg * (2.0 * np * pt + 4.0) + (double)rmax * 4.0 +
                  (first ? inter * np * pt : 0.0) + inter * np * pt * (done ? 1.0 : 2.0);
        // between L2 and the SM: the region's inputs, the interior's accumulator in and
        // outputs (the algorithmic DRAM count takes the inputs once per interior site)
        const double vin = first ? 1.0 : 2.0;
        const bool to_main = first || ka <= B.ksplit;
        const bool read_e = !first && (to_main || done);
        const bool read_t = !first && !to_main && prev_ka > B.ksplit;
        const double acc_in = (read_e ? 1.0 : 0.0) + (read_t ? 1.0 : 0.0);
        const double outs = done ? 1.0 : 3.0;  // psi, or T_{ke-1}, T_ke and the accumulator
        m.l2 += nreg * (vin * np * pt + 4.0) + inter * np * pt * (acc_in + outs);
    }
}

}  // namespace cheb
