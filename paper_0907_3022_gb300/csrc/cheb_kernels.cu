// Fused Chebyshev recurrence kernel (Sec. 2.2, Eqs. U_1 and rec) and FP64 reductions.
//
// One launch forms T_{j+1} for every block whose order M reaches j+1:
//   FIRST   (j = 0):  T_1 = H~ psi                    -> B = T_1
//                     and per (block, vec) ||psi||^2, <psi|H~ psi>   (deterministic FP64)
//   SECOND  (j = 1):  T_2 = 2 H~ T_1 - T_0 (T_0 = psi) -> A = T_2,
//                     psi = q_0 T_0 + q_1' T_1 + q_2 T_2
//   GENERAL (j >= 2): T_{j+1} = 2 H~ T_j - T_{j-1}     -> over T_{j-1};
//                     at j+1 = 2 (mod 3): psi += q'_{j-1} T_{j-1} + q'_j T_j + q'_{j+1} T_{j+1};
//                     at j+1 = M: the orders left, then psi *= e^{-i b dt}
// (the accumulator is touched by every third launch, see AccGroup).
// complex64 plans send the orders with |q_k| < 2^-8 (k > ksplit) to a second accumulator
// "tail" and add it to psi at the last order: added straight into psi, terms smaller than
// half an ulp of psi would be rounded away every time, which truncates the series early
// and makes the norm decay linearly in time (~1e-8 per step at M = 20).
// where q_k = sign (2 - delta_k0) J_k(a dt) is real and the factor (-i)^k is applied by the
// parity of k (even k: +/- real, odd k: +/- imaginary), so the accumulation costs two FMAs
// per complex value.  2 H~ x at a site is d_i x_i + beta * (sum of neighbour values) with
// d_i = 2 (H_ii - b)/a stored per site and beta = 2 h_offdiag / a per block (stencils), or
// d_i x_i + sum_j v_ij x_j with v_ij = 2 H_ij / a stored in SELL-C order (Holstein).
//
// Memory per site and order (GENERAL, one vector): read T_j (+ neighbours, from cache),
// T_{j-1}, d_i; write T_{j+1}; every third order also read and write psi.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "cheb_device.cuh"
#include "cheb_internal.cuh"

namespace cheb {

// Finalize FIRST-mode reductions: the last CTA to finish sums the per-item partials of each
// block and writes (||psi||^2, <psi|H|psi>) per (block, vec).  One warp per (block, vec)
// slot: lane l sums items l, l + 32, ... in order, then a fixed xor tree, so the summation
// order depends on the item count only (a single thread per slot walked thousands of
// partials out of L2 one after another).
__device__ void finalize_first(const RecArgs& a)
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int slot = warp; slot < a.nblocks * nv; slot += nwarps) {
        const int q = slot / nv, v = slot % nv;
        const int it1 = a.block_item_begin[q + 1];
        double n2 = 0.0, eh = 0.0;
#pragma unroll 8
        for (int it = a.block_item_begin[q] + lane; it < it1; it += 32) {
            n2 += __ldcg(a.partials + ((size_t)it * nv + v) * 2 + 0);
            eh += __ldcg(a.partials + ((size_t)it * nv + v) * 2 + 1);
        }
        for (int off = 16; off > 0; off >>= 1) {
            n2 += __shfl_xor_sync(0xffffffffu, n2, off);
            eh += __shfl_xor_sync(0xffffffffu, eh, off);
        }
        if (lane == 0) {
            const DevBlock B = a.blocks[q];
            a.red_out[(size_t)slot * 2 + 0] = n2;
            a.red_out[(size_t)slot * 2 + 1] = B.a * eh + B.b * n2;  // <H> = a <H~> + b ||psi||^2
        }
    }
    if (threadIdx.x == 0) *a.done_counter = 0u;  // ready for the next FIRST launch
}

// ---- operators: off-diagonal part of 2 H~ x at one (site, vector group) --------------------
// Stencil: beta * (sum of the brick-wall neighbours); 1D grid = one ribbon with W = 1.
template <typename R, int VPT>
struct StencilOp {
    using C = typename V2<R>::C;
    using IO = VecIO<R, VPT>;
    R bh, bl;
    int32_t W, L;
    __device__ __forceinline__ void init(const RecArgs&, const DevBlock& B) {
        split_const<R>(B.beta, bh, bl);
        W = B.W;
        L = B.L;
    }
    // adds beta * s to acc (acc holds -T_{j-1} or 0)
    __device__ __forceinline__ void offdiag(const RecArgs&, const C* __restrict__ cur, int64_t sl,
                                            int64_t, int64_t base, int, int nv,
                                            C (&acc)[VPT]) const {
        const int r = (int)(sl / L);
        const int c = (int)(sl - (int64_t)r * L);
        const int vr = ((r + c) & 1) ? r - 1 : r + 1;
        const bool hl = c > 0, hr = c + 1 < L, hv = (vr >= 0) && (vr < W);
        C nl[VPT], nr[VPT], nvv[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) nl[v] = nr[v] = nvv[v] = V2<R>::make(0, 0);
        if (hl) IO::load(cur + base - nv, nl);
        if (hr) IO::load(cur + base + nv, nr);
        if (hv) IO::load(cur + base + (int64_t)(vr - r) * L * nv, nvv);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const R sx = nl[v].x + nr[v].x + nvv[v].x;
            const R sy = nl[v].y + nr[v].y + nvv[v].y;
            if (Split<R>::on) {
                acc[v].x = fma(bl, sx, acc[v].x);
                acc[v].y = fma(bl, sy, acc[v].y);
            }
            acc[v].x = fma(bh, sx, acc[v].x);
            acc[v].y = fma(bh, sy, acc[v].y);
        }
    }
};

// SELL-C (C = 32): entries v_ij = 2 H_ij / a stored column-major per chunk of 32 rows.
template <typename R, int VPT>
struct SellOp {
    using C = typename V2<R>::C;
    using IO = VecIO<R, VPT>;
    __device__ __forceinline__ void init(const RecArgs&, const DevBlock&) {}
    // pos: the row's storage position (the row itself without sigma sorting)
    __device__ __forceinline__ void offdiag(const RecArgs& a, const C* __restrict__ cur, int64_t pos,
                                            int64_t, int64_t, int g, int nv,
                                            C (&acc)[VPT]) const {
        const R* __restrict__ sval = static_cast<const R*>(a.sell_val);
        const int64_t chunk = pos >> 5;
        const int64_t off = a.sell_chunk_off[chunk] + (pos & 31);
        const int len = a.sell_chunk_len[chunk];
        // complex128: the first EU entries (every Holstein row has 2 to 4) with all column
        // indices and values first, then all gathers, so that a row's dependent loads overlap
        // (10 % faster); complex64 keeps one entry at a time, whose fewer registers leave more
        // warps to hide the gathers (the batched form was 20 % slower there)
        constexpr int EU = sizeof(R) == 8 ? 4 : 0;
        if constexpr (EU > 0) {
            int col[EU];
            R val[EU];
#pragma unroll
            for (int e = 0; e < EU; ++e) {
                col[e] = e < len ? a.sell_col[off + (int64_t)e * 32] : 0;
                val[e] = e < len ? sval[off + (int64_t)e * 32] : (R)0;
            }
            C y[EU][VPT];
#pragma unroll
            for (int e = 0; e < EU; ++e)
                if (e < len) IO::load(cur + (int64_t)col[e] * nv + (int64_t)g * VPT, y[e]);
#pragma unroll
            for (int e = 0; e < EU; ++e) {
                if (e < len) {
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        acc[v].x = fma(val[e], y[e][v].x, acc[v].x);
                        acc[v].y = fma(val[e], y[e][v].y, acc[v].y);
                    }
                }
            }
        }
        for (int e = EU; e < len; ++e) {
            const int c = a.sell_col[off + (int64_t)e * 32];
            const R v0 = sval[off + (int64_t)e * 32];
            C z[VPT];
            IO::load(cur + (int64_t)c * nv + (int64_t)g * VPT, z);
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                acc[v].x = fma(v0, z[v].x, acc[v].x);
                acc[v].y = fma(v0, z[v].y, acc[v].y);
            }
        }
    }
};

// ---- the fused recurrence kernel -------------------------------------------------------------
template <typename R, int VPT, template <typename, int> class Op>
__global__ void __launch_bounds__(512) k_rec(RecArgs a)
{
    using C = typename V2<R>::C;
    using U = SiteUpdate<R>;
    using IO = VecIO<R, VPT>;
    __shared__ double s_red[16 * 32 * 2];  // [warps][nvg][2 VPT]
    const int nv = a.nvec;
    const int nvg = nv / VPT;
    const C* __restrict__ cur = static_cast<const C*>(a.cur);
    C* __restrict__ prev = static_cast<C*>(a.prev);
    C* __restrict__ out1 = static_cast<C*>(a.out1);
    C* __restrict__ psi = static_cast<C*>(a.psi);
    C* __restrict__ tail = static_cast<C*>(a.tail);
    const R* __restrict__ diag = static_cast<const R*>(a.diag);
    const C* __restrict__ qc = static_cast<const C*>(a.qcoef);  // (hi, lo) per k
    const int k = a.j + 1;  // order formed by this launch
    const bool first = (a.mode == REC_FIRST);
    const bool second = (a.mode == REC_SECOND);

    for (int w = blockIdx.x; w < a.nitems; w += gridDim.x) {
        const WorkItem it = a.items[w];
        const DevBlock B = a.blocks[it.block];
        // per-thread norm / energy terms (FIRST): in the vector precision, since a thread sums
        // only its few sites (FP64 arithmetic is ~1/32 the FP32 rate on this GPU); the block
        // and grid reductions that follow are FP64
        R part[2 * VPT];
#pragma unroll
        for (int s = 0; s < 2 * VPT; ++s) part[s] = (R)0;
        if (k <= B.M) {
            Op<R, VPT> op;
            op.init(a, B);
            const int64_t units = it.count * nvg;  // (site, vector group) pairs in the tile
            const AccGroup ag(k, B.M, B.ksplit);
            C qm2 = V2<R>::make(0, 0), qm1 = qm2, qk = qm2;
            if (!first) {
                qk = qc[B.coef_off + k];
                if (ag.n >= 2) qm1 = qc[B.coef_off + k - 1];
                if (ag.n >= 3) qm2 = qc[B.coef_off + k - 2];
            }
            C ph, pl;
            split_const<R>(B.ph_re, ph.x, pl.x);
            split_const<R>(B.ph_im, ph.y, pl.y);
            C* __restrict__ accp = ag.to_tail ? tail : psi;
            for (int64_t u = threadIdx.x; u < units; u += blockDim.x) {
                // site within the block; for a sigma-sorted SELL matrix the storage position,
                // whose row is sell_perm[position]
                const int64_t sl = it.first + u / nvg;
                const int g = (int)(u % nvg);
                const int64_t gs = B.offset + (a.sell_perm ? (int64_t)__ldg(a.sell_perm + sl) : sl);
                const int64_t base = gs * nv + (int64_t)g * VPT;
                // every load of this site first, then arithmetic and stores
                C x[VPT], p[VPT], acc[VPT], ps[VPT];
                R d[VPT];
                IO::load(cur + base, x);
                if (first) {
#pragma unroll
                    for (int v = 0; v < VPT; ++v) p[v] = V2<R>::make(0, 0);
                } else {
                    IO::load((second ? psi : prev) + base, p);  // T_{k-2} (SECOND: T_0 = psi)
                }
                if (ag.read_acc) {
                    IO::load(accp + base, acc);
                } else {
#pragma unroll
                    for (int v = 0; v < VPT; ++v) acc[v] = V2<R>::make(0, 0);
                }
                if (ag.read_psi_last) IO::load(psi + base, ps);
#pragma unroll
                for (int v = 0; v < VPT; ++v) d[v] = a.diag_per_vec ? diag[base + v] : diag[gs];
                // h = 2 H~ x - p  (FIRST: p = 0)
                C h[VPT];
#pragma unroll
                for (int v = 0; v < VPT; ++v) h[v] = V2<R>::make(-p[v].x, -p[v].y);
                op.offdiag(a, cur, sl, gs, base, g, nv, h);
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    h[v].x = fma(d[v], x[v].x, h[v].x);
                    h[v].y = fma(d[v], x[v].y, h[v].y);
                }
                if (first) {
                    C t1[VPT];
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        t1[v] = V2<R>::make((R)0.5 * h[v].x, (R)0.5 * h[v].y);
                        part[2 * v + 0] = fma(x[v].x, x[v].x, fma(x[v].y, x[v].y, part[2 * v + 0]));
                        part[2 * v + 1] = fma(x[v].x, t1[v].x, fma(x[v].y, t1[v].y, part[2 * v + 1]));
                    }
                    IO::store(out1 + base, t1);
                } else {
                    IO::store(prev + base, h);  // T_k over T_{k-2}
                    if (ag.upd) {
#pragma unroll
                        for (int v = 0; v < VPT; ++v) {
                            if (ag.n >= 3) U::accum(acc[v], qm2, p[v], k - 2);
                            if (ag.n >= 2) U::accum(acc[v], qm1, x[v], k - 1);
                            U::accum(acc[v], qk, h[v], k);
                        }
                        if (ag.last) {
                            if (ag.read_psi_last) {  // psi + (tail + newest orders)
#pragma unroll
                                for (int v = 0; v < VPT; ++v)
                                    acc[v] = V2<R>::make(ps[v].x + acc[v].x, ps[v].y + acc[v].y);
                            }
#pragma unroll
                            for (int v = 0; v < VPT; ++v) {
                                acc[v] = U::phase(acc[v], ph, pl);
                                // growth check |T_M|^2 <= 4 ||psi||^2 in the vector precision
                                const R t2 = fma(h[v].x, h[v].x, h[v].y * h[v].y);
                                const R lim = (R)(4.0 * a.norm2[((size_t)it.block * nv + g * VPT + v) * 2]);
                                if (!(t2 <= lim)) atomicOr(a.errflag, 1);
                            }
                            IO::store(psi + base, acc);
                        } else {
                            IO::store(accp + base, acc);
                        }
                    }
                }
            }
        }
        if (first) {
            // partials[w][vec][2] = (||x||^2, <x|H~x>) of this tile; (g, v, comp) -> g*2VPT + 2v + comp
            if constexpr (Split<R>::on) {  // complex64: FP32 warp tree, FP64 block sum
                block_reduce_groups_f<2 * VPT>(part, nvg, s_red, a.partials + (size_t)w * nv * 2);
            } else {
                double dpart[2 * VPT];
#pragma unroll
                for (int s = 0; s < 2 * VPT; ++s) dpart[s] = (double)part[s];
                block_reduce_groups<2 * VPT>(dpart, nvg, s_red, a.partials + (size_t)w * nv * 2);
            }
        }
    }
    if (first) finalize_first(a);
}

// ---- dispatch ---------------------------------------------------------------------------
template <typename R, int VPT>
static void launch_t(const RecArgs& a, int op, int grid, int threads, cudaStream_t s)
{
    if (op == OP_STENCIL)
        k_rec<R, VPT, StencilOp><<<grid, threads, 0, s>>>(a);
    else
        k_rec<R, VPT, SellOp><<<grid, threads, 0, s>>>(a);
}

// vectors per thread: the plan's tuned value when it divides nvec, else the widest group
// that keeps 16-byte accesses (complex128: 1 value; complex64: up to 4 values)
int vpt_for(int prec, int nvec, int want)
{
    if (want > 0 && nvec % want == 0 && (want == 1 || want == 2 || (want == 4 && prec == CHEB_C64)))
        return want;
    if (prec == CHEB_C128) return 1;
    if (nvec % 4 == 0) return 4;
    if (nvec % 2 == 0) return 2;
    return 1;
}

int launch_recurrence(Plan* p, const RecArgs& a, int op, int prec, cudaStream_t s)
{
    if (op == OP_HOLMF) return launch_holmf(p, a, s);
    const int vpt = vpt_for(prec, p->nvec, p->vpt);
    int grid = a.nitems;
    if (p->grid_cap > 0 && grid > p->grid_cap) grid = p->grid_cap;
    if (grid < 1) return CHEB_OK;
    const int th = p->threads;
    if (prec == CHEB_C128) {
        if (vpt == 2) launch_t<double, 2>(a, op, grid, th, s);
        else launch_t<double, 1>(a, op, grid, th, s);
    } else {
        if (vpt == 4) launch_t<float, 4>(a, op, grid, th, s);
        else if (vpt == 2) launch_t<float, 2>(a, op, grid, th, s);
        else launch_t<float, 1>(a, op, grid, th, s);
    }
    p->launches++;
    CHEB_CUDA(cudaGetLastError());
    return CHEB_OK;
}

// ---- diagonal scaling: d_i = 2 (H_ii - b)/a -------------------------------------------------
template <typename R>
__global__ void k_scale_diag(const WorkItem* items, int nitems, const DevBlock* blocks,
                             const double* onsite, int per_vec, int nvec, double diag_shift,
                             R* d)
{
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const WorkItem it = items[w];
        const DevBlock B = blocks[it.block];
        const int per = per_vec ? nvec : 1;
        const int64_t n = it.count * per;
        for (int64_t u = threadIdx.x; u < n; u += blockDim.x) {
            const int64_t idx = (B.offset + it.first) * per + u;
            const double hii = diag_shift + (onsite ? onsite[idx] : 0.0);
            d[idx] = (R)(2.0 * (hii - B.b) / B.a);
        }
    }
}

int launch_scale_diag(Plan* p, const double* onsite, cudaStream_t s)
{
    // 1D grid: H_ii = 1/dx^2 + V_i; ribbons: H_ii = eps_i
    const double shift = (p->desc.kind == CHEB_LAT1D) ? 1.0 / (p->desc.dx * p->desc.dx) : 0.0;
    const int grid = (int)std::min<int64_t>((int64_t)p->hitems.size(), 65535);
    if (p->prec == CHEB_C128)
        k_scale_diag<double><<<grid, 256, 0, s>>>(p->d_items, (int)p->hitems.size(), p->d_blocks,
                                                  onsite, p->desc.onsite_per_vec, p->nvec, shift,
                                                  static_cast<double*>(p->d_diag));
    else
        k_scale_diag<float><<<grid, 256, 0, s>>>(p->d_items, (int)p->hitems.size(), p->d_blocks,
                                                 onsite, p->desc.onsite_per_vec, p->nvec, shift,
                                                 static_cast<float*>(p->d_diag));
    p->launches++;
    CHEB_CUDA(cudaGetLastError());
    return CHEB_OK;
}

// ---- observables for the stencil kinds ------------------------------------------------------
// Per work item partials [nvec] of  norm2 | energy (<x|H x>) | probability of columns > param;
// then one CTA per (block) sums item partials in order.
template <typename R>
__global__ void k_obs_stencil(const WorkItem* items, int nitems, const DevBlock* blocks,
                              const void* psi_, const void* diag_, int diag_per_vec, int nvec,
                              int kind, double param, double* partials)
{
    using C = typename V2<R>::C;
    const C* psi = static_cast<const C*>(psi_);
    const R* diag = static_cast<const R*>(diag_);
    __shared__ double s_red[32];
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const WorkItem it = items[w];
        const DevBlock B = blocks[it.block];
        for (int v = 0; v < nvec; ++v) {
            double acc = 0.0;
            for (int64_t u = threadIdx.x; u < it.count; u += blockDim.x) {
                const int64_t sl = it.first + u;
                const int r = (int)(sl / B.L);
                const int c = (int)(sl - (int64_t)r * B.L);
                const int64_t gs = B.offset + sl;
                const C x = psi[gs * nvec + v];
                const double n2 = (double)x.x * x.x + (double)x.y * x.y;
                if (kind == CHEB_OBS_NORM2) {
                    acc += n2;
                } else if (kind == CHEB_OBS_PROB_COLS) {
                    if ((double)c > param) acc += n2;
                } else {  // energy: <x| 2H~ x>/2 * a + b |x|^2, with 2H~x from the stencil
                    const int vr = ((r + c) & 1) ? r - 1 : r + 1;
                    double sx = 0.0, sy = 0.0;
                    if (c > 0) { C y = psi[(gs - 1) * nvec + v]; sx += y.x; sy += y.y; }
                    if (c + 1 < B.L) { C y = psi[(gs + 1) * nvec + v]; sx += y.x; sy += y.y; }
                    if (vr >= 0 && vr < B.W) {
                        C y = psi[(gs + (int64_t)(vr - r) * B.L) * nvec + v];
                        sx += y.x;
                        sy += y.y;
                    }
                    const double d = (double)(diag_per_vec ? diag[gs * nvec + v] : diag[gs]);
                    const double hx = d * x.x + B.beta * sx, hy = d * x.y + B.beta * sy;
                    acc += 0.5 * B.a * ((double)x.x * hx + (double)x.y * hy) + B.b * n2;
                }
            }
            // block reduce (fixed order)
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_red[q];
                partials[(size_t)w * nvec + v] = t;
            }
            __syncthreads();
        }
    }
}

__global__ void k_obs_finalize(const double* partials, const int32_t* block_item_begin,
                               int nblocks, int nvec, double* out)
{
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < nblocks * nvec;
         slot += gridDim.x * blockDim.x) {
        const int q = slot / nvec, v = slot % nvec;
        double t = 0.0;
        for (int it = block_item_begin[q]; it < block_item_begin[q + 1]; ++it)
            t += partials[(size_t)it * nvec + v];
        out[slot] = t;
    }
}

// ---- FP64 records of ||psi||^2 and <psi|H|psi> (complex64 plans) -----------------------------
// cheb_evolve records the norm and energy of psi at the start of every obs_every-th step.
// complex128 plans take them from their first recurrence launch (FP64 throughout); complex64
// plans compute them here instead, with FP64 products and sums of the complex64 values, so
// that the first launch of a complex64 step keeps its FP32 per-thread sums (they feed only the
// divergence check |T_M|^2 <= 4 ||psi||^2) and unrecorded steps pay nothing.
// Stencil kinds: per work item and vector the two sums, then per (block, vec) in item order.
template <typename R>
__global__ void k_rec_obs_stencil(const WorkItem* items, int nitems, const DevBlock* blocks,
                                  const void* psi_, const void* diag_, int diag_per_vec, int nvec,
                                  double* partials)
{
    using C = typename V2<R>::C;
    const C* psi = static_cast<const C*>(psi_);
    const R* diag = static_cast<const R*>(diag_);
    __shared__ double s_red[32 * 2];
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const WorkItem it = items[w];
        const DevBlock B = blocks[it.block];
        for (int v = 0; v < nvec; ++v) {
            double n2 = 0.0, eh = 0.0;  // ||x||^2 and <x|2H~ x>
            for (int64_t u = threadIdx.x; u < it.count; u += blockDim.x) {
                const int64_t sl = it.first + u;
                const int r = (int)(sl / B.L);
                const int c = (int)(sl - (int64_t)r * B.L);
                const int64_t gs = B.offset + sl;
                const C x = psi[gs * nvec + v];
                const int vr = ((r + c) & 1) ? r - 1 : r + 1;
                double sx = 0.0, sy = 0.0;
                if (c > 0) { const C y = psi[(gs - 1) * nvec + v]; sx += y.x; sy += y.y; }
                if (c + 1 < B.L) { const C y = psi[(gs + 1) * nvec + v]; sx += y.x; sy += y.y; }
                if (vr >= 0 && vr < B.W) {
                    const C y = psi[(gs + (int64_t)(vr - r) * B.L) * nvec + v];
                    sx += y.x;
                    sy += y.y;
                }
                const double d = (double)(diag_per_vec ? diag[gs * nvec + v] : diag[gs]);
                const double hx = d * x.x + B.beta * sx, hy = d * x.y + B.beta * sy;
                n2 += (double)x.x * x.x + (double)x.y * x.y;
                eh += (double)x.x * hx + (double)x.y * hy;
            }
            for (int off = 16; off > 0; off >>= 1) {
                n2 += __shfl_xor_sync(0xffffffffu, n2, off);
                eh += __shfl_xor_sync(0xffffffffu, eh, off);
            }
            if ((threadIdx.x & 31) == 0) {
                s_red[(threadIdx.x >> 5) * 2 + 0] = n2;
                s_red[(threadIdx.x >> 5) * 2 + 1] = eh;
            }
            __syncthreads();
            if (threadIdx.x < 2) {
                double t = 0.0;
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_red[q * 2 + threadIdx.x];
                partials[((size_t)w * nvec + v) * 2 + threadIdx.x] = t;
            }
            __syncthreads();
        }
    }
}

// per (block, vec): one warp sums the block's item partials (lane-strided, fixed xor tree)
__global__ void k_rec_obs_finalize(const double* partials, const int32_t* block_item_begin,
                                   const DevBlock* blocks, int nblocks, int nvec, double* out)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int slot = warp; slot < nblocks * nvec; slot += nwarps) {
        const int q = slot / nvec, v = slot % nvec;
        double n2 = 0.0, eh = 0.0;
        for (int it = block_item_begin[q] + lane; it < block_item_begin[q + 1]; it += 32) {
            n2 += partials[((size_t)it * nvec + v) * 2 + 0];
            eh += partials[((size_t)it * nvec + v) * 2 + 1];
        }
        for (int off = 16; off > 0; off >>= 1) {
            n2 += __shfl_xor_sync(0xffffffffu, n2, off);
            eh += __shfl_xor_sync(0xffffffffu, eh, off);
        }
        if (lane == 0) {
            const DevBlock B = blocks[q];
            out[(size_t)slot * 2 + 0] = n2;
            out[(size_t)slot * 2 + 1] = 0.5 * B.a * eh + B.b * n2;  // <H> = (a/2) <2H~> + b n2
        }
    }
}

// out[v * 2 + 0] = n2[v], out[v * 2 + 1] = e[v]
__global__ void k_rec_obs_interleave(const double* n2, const double* e, int nvec, double* out)
{
    const int v = threadIdx.x;
    if (v < nvec) {
        out[v * 2 + 0] = n2[v];
        out[v * 2 + 1] = e[v];
    }
}

int launch_holstein_observable(Plan* p, const void* psi, int kind, double* out, cudaStream_t s);
int launch_holstein_energy(Plan* p, const void* psi, double* out, cudaStream_t s);

int record_prepare(Plan* p)
{
    const size_t need = std::max(p->hitems.size() * (size_t)p->nvec * 2, (size_t)p->nvec * 2);
    if (p->rec_scratch_cap < need) {
        if (p->d_rec_scratch) cudaFree(p->d_rec_scratch);
        p->d_rec_scratch = nullptr;
        p->rec_scratch_cap = 0;
        CHEB_CUDA(cudaMalloc(&p->d_rec_scratch, need * sizeof(double)));
        p->rec_scratch_cap = need;
    }
    return p->desc.kind == CHEB_HOLSTEIN ? obs_prepare(p) : CHEB_OK;
}

int launch_record(Plan* p, const void* psi, double* out, cudaStream_t s)
{
    int rc = record_prepare(p);
    if (rc) return rc;
    if (p->desc.kind == CHEB_HOLSTEIN) {  // one block: the two FP64 observables, interleaved
        double* n2 = p->d_rec_scratch;
        double* e = p->d_rec_scratch + p->nvec;
        rc = launch_observable(p, psi, CHEB_OBS_NORM2, 0.0, n2, s);
        if (!rc) rc = launch_observable(p, psi, CHEB_OBS_ENERGY, 0.0, e, s);
        if (rc) return rc;
        k_rec_obs_interleave<<<1, 32, 0, s>>>(n2, e, p->nvec, out);
        p->launches++;
        CHEB_CUDA(cudaGetLastError());
        return CHEB_OK;
    }
    const int nitems = (int)p->hitems.size();
    const int grid = std::min(nitems, 65535);
    if (p->prec == CHEB_C128)
        k_rec_obs_stencil<double><<<grid, 256, 0, s>>>(p->d_items, nitems, p->d_blocks, psi,
                                                       p->d_diag, p->desc.onsite_per_vec, p->nvec,
                                                       p->d_rec_scratch);
    else
        k_rec_obs_stencil<float><<<grid, 256, 0, s>>>(p->d_items, nitems, p->d_blocks, psi,
                                                      p->d_diag, p->desc.onsite_per_vec, p->nvec,
                                                      p->d_rec_scratch);
    const int slots = p->nblocks * p->nvec;
    k_rec_obs_finalize<<<std::min((slots + 7) / 8, 1024), 256, 0, s>>>(
        p->d_rec_scratch, p->d_block_item_begin, p->d_blocks, p->nblocks, p->nvec, out);
    p->launches += 2;
    CHEB_CUDA(cudaGetLastError());
    return CHEB_OK;
}


// allocate the stencil observables' partials ahead of a stream capture
int obs_prepare(Plan* p)
{
    const size_t need = p->hitems.size() * (size_t)p->nvec;
    if (p->obs_scratch_cap >= need) return CHEB_OK;
    if (p->d_obs_scratch) cudaFree(p->d_obs_scratch);
    p->d_obs_scratch = nullptr;
    p->obs_scratch_cap = 0;
    CHEB_CUDA(cudaMalloc(&p->d_obs_scratch, need * sizeof(double)));
    p->obs_scratch_cap = need;
    return CHEB_OK;
}

int launch_observable(Plan* p, const void* psi, int kind, double param, double* out,
                      cudaStream_t s)
{
    if (kind >= CHEB_OBS_HOL_DENSITY) {
        if (p->desc.kind != CHEB_HOLSTEIN)
            return fail(CHEB_ERR_UNSUPPORTED, "Holstein observable on a lattice plan");
        return launch_holstein_observable(p, psi, kind, out, s);
    }
    if (p->desc.kind == CHEB_HOLSTEIN) {
        if (kind == CHEB_OBS_PROB_COLS)
            return fail(CHEB_ERR_UNSUPPORTED, "column probability needs a lattice plan");
        if (kind == CHEB_OBS_ENERGY)
            return (p->op == OP_HOLMF) ? launch_holmf_energy(p, psi, out, s)
                                       : launch_holstein_energy(p, psi, out, s);
    }
    const int nitems = (int)p->hitems.size();
    const size_t need = (size_t)nitems * p->nvec;
    if (p->obs_scratch_cap < need) {
        if (p->d_obs_scratch) cudaFree(p->d_obs_scratch);
        p->d_obs_scratch = nullptr;
        p->obs_scratch_cap = 0;
        CHEB_CUDA(cudaMalloc(&p->d_obs_scratch, need * sizeof(double)));
        p->obs_scratch_cap = need;
    }
    const int grid = std::min(nitems, 65535);
    if (p->prec == CHEB_C128)
        k_obs_stencil<double><<<grid, 256, 0, s>>>(p->d_items, nitems, p->d_blocks, psi, p->d_diag,
                                                   p->desc.onsite_per_vec, p->nvec, kind, param,
                                                   p->d_obs_scratch);
    else
        k_obs_stencil<float><<<grid, 256, 0, s>>>(p->d_items, nitems, p->d_blocks, psi, p->d_diag,
                                                  p->desc.onsite_per_vec, p->nvec, kind, param,
                                                  p->d_obs_scratch);
    k_obs_finalize<<<1, 256, 0, s>>>(p->d_obs_scratch, p->d_block_item_begin, p->nblocks, p->nvec,
                                     out);
    p->launches += 2;
    CHEB_CUDA(cudaGetLastError());
    return CHEB_OK;
}

}  // namespace cheb
