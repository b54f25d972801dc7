// Temporally blocked Chebyshev recurrence with register-resident runs (Sec. 2.2, Eqs. U_1 and
// rec; brick-wall ribbons of Sec. 3.2, the 1D grid as W = 1), complex64.
//
// Same tiles, halos, validity rule and accumulator protocol as k_rec_tb (cheb_tb.cu): one
// launch forms orders ka..kb for every ribbon, a CTA owns the region of one tile and keeps the
// tile's interior valid for all orders.  What differs is how a CTA holds the region:
//
// * A CTA carries one plane element per site: a pair of vectors (float4, nvec 2 or 4; with 4
//   the two pairs of a tile go to two CTAs) or a single vector (float2, nvec 1).
// * Thread t owns the RUN consecutive positions t RUN .. t RUN + RUN - 1 of the region laid out
//   row-major with a padded row stride.  T_{k-1} and T_{k-2} of its own sites stay in
//   registers, so an order reads from shared memory only the vertical neighbour of each site
//   and the two neighbours beyond the run's ends, and stores each site's T_k once (the
//   neighbours of the next order read it).  Only T_{k-1} has a shared-memory plane (two planes,
//   read one / write the other).
// * Layout of a plane: site (rr, cc) of the RH x RW region is at position rr S + cc, where the
//   row stride S (from the tile builder) is RW + 1 rounded up to A = 4 for float4, 8 for
//   float2 (with boxes: the widest tile's, the same for every tile of a ribbon), so that the
//   S - RW >= 1 positions after every row are zero pads; one zero element follows the last
//   position (index NPOS = RUN TPB).  The pads make the neighbour left of column 0 and right of column RW - 1 a
//   zero read, which is the ribbon's open edge where the region ends at the ribbon border (where
//   it ends at an open side the site is outside the validity limit and its value unused).  A
//   vertical neighbour outside the region or the ribbon, and the left neighbour of position 0,
//   read the element at NPOS.
// * Bank conflicts: with RUN odd, the lanes of a quarter warp (float4) or half warp (float2)
//   address distinct bank groups for the same j; with S a multiple of A, the up and down
//   neighbours (+-S) of any two lanes still do.
// * A run is formed at an order if any of its sites is still valid.  Its pads are formed too,
//   with zero coupling, diagonal and values, so they stay exactly zero: no per-site branch in
//   the order loop (both planes are zeroed at every tile start, so every value read is finite).
//   The accumulation runs for every position and only interior sites are written out, and the
//   parity of the order, which decides how (-i)^k enters, is a compile-time constant.
// * A launch keeps its CTAs resident (one per SM), each working through tiles, and the inputs
//   of a CTA's next work item (T_{ka-1}, T_{ka-2}, d and the accumulator) stream into staging
//   buffers while the current item runs its orders, so the global-memory latency of a tile
//   start is hidden.  They are copied with cp.async, consecutive lanes on consecutive
//   positions, and published by a barrier after the wait; in the variant with boxes
//   (CHEB_TB_RUNS_TMA, pairs of vectors) T_{ka-1} and T_{ka-2} come as two tensor-memory-access
//   boxes of S x BH elements (BH = the ribbon's tallest region) whose shared-memory image is
//   exactly the plane layout above (box row rr, column cc at rr S + cc; columns and rows beyond
//   the ribbon read as zero).
// * The step's own vectors (the T pairs passed between launches, E, tail) are stored
//   pair-planar, element (site, pair) at pair x sites + site, so that a CTA, which owns one
//   pair, moves whole sectors; psi, read by the first launch and written by the last, keeps
//   its [site][vector] layout.
//
// Per formed site-order and plane element: one vertical load, 2 / RUN run-end loads, one store
// (k_rec_tb: own, three neighbours, T_{k-2} and the store).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "cheb_internal.cuh"

namespace cheb {

template <typename PT> struct TBRPlane;
template <> struct TBRPlane<float4> {
    static constexpr int A = 4;    // row-stride alignment (elements)
    static constexpr int PER = 2;  // vectors per element
};
template <> struct TBRPlane<float2> {
    static constexpr int A = 8;
    static constexpr int PER = 1;
};

// same validity limit as k_rec_tb (cheb_tb.cu)
__host__ __device__ __forceinline__ int tbr_limit(int rr, int cc, int RH, int RW, bool up,
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

__device__ __forceinline__ float4 tbr_zero(float4*) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float2 tbr_zero(float2*) { return make_float2(0.f, 0.f); }

// Packed two-float arithmetic on a complex value's (re, im) pair: one instruction for both
// components, each rounded as the scalar operation would be.
__device__ __forceinline__ unsigned long long tbr_pk(float2 v)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 tbr_upk(unsigned long long r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 tbr_add2(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(tbr_pk(a)), "l"(tbr_pk(b)));
    return tbr_upk(d);
}
__device__ __forceinline__ float2 tbr_fma2(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(tbr_pk(a)), "l"(tbr_pk(b)), "l"(tbr_pk(c)));
    return tbr_upk(d);
}

// h = beta (l + r + v) - p + d x, halved for T_1 = H~ T_0; beta is a float32 number in
// complex64 lattice plans (the plan chooses a so), zero at pads
__device__ __forceinline__ float2 tbr_h(float2 l, float2 r, float2 v, float2 p, float2 x, float d,
                                        float bh, bool half)
{
    const float2 s2 = tbr_add2(tbr_add2(l, r), v);
    float2 h = tbr_fma2(make_float2(bh, bh), s2, make_float2(-p.x, -p.y));
    h = tbr_fma2(make_float2(d, d), x, h);
    if (half) {
        h.x *= 0.5f;
        h.y *= 0.5f;
    }
    return h;
}
__device__ __forceinline__ float4 tbr_h(float4 l, float4 r, float4 v, float4 p, float4 x, float d,
                                        float bh, bool half)
{
    const float2 a = tbr_h(make_float2(l.x, l.y), make_float2(r.x, r.y), make_float2(v.x, v.y),
                           make_float2(p.x, p.y), make_float2(x.x, x.y), d, bh, half);
    const float2 b = tbr_h(make_float2(l.z, l.w), make_float2(r.z, r.w), make_float2(v.z, v.w),
                           make_float2(p.z, p.w), make_float2(x.z, x.w), d, bh, half);
    return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ float2 tbr_get(const float2& t, int) { return t; }
__device__ __forceinline__ float2 tbr_get(const float4& t, int c)
{
    return c ? make_float2(t.z, t.w) : make_float2(t.x, t.y);
}
__device__ __forceinline__ void tbr_put(float2& t, int, float2 v) { t = v; }
__device__ __forceinline__ void tbr_put(float4& t, int c, float2 v)
{
    if (c) {
        t.z = v.x;
        t.w = v.y;
    } else {
        t.x = v.x;
        t.y = v.y;
    }
}

// acc += (-i)^k q t with the sign of (-i)^k folded into q = (hi, lo); the parity of k is a
// compile-time constant in the order loop
template <bool ODD>
__device__ __forceinline__ void tbr_accum(float2& acc, const float2 q, const float2 t)
{
    if (!ODD) {
        acc = tbr_fma2(make_float2(q.y, q.y), t, acc);
        acc = tbr_fma2(make_float2(q.x, q.x), t, acc);
    } else {
        acc.x = fmaf(q.y, t.y, acc.x);
        acc.y = fmaf(-q.y, t.x, acc.y);
        acc.x = fmaf(q.x, t.y, acc.x);
        acc.y = fmaf(-q.x, t.x, acc.y);
    }
}

__device__ __forceinline__ float2 tbr_phase(const float2 a, const float2 ph, const float2 pl)
{
    float rx = fmaf(pl.x, a.x, -pl.y * a.y);
    float ry = fmaf(pl.x, a.y, pl.y * a.x);
    rx = fmaf(ph.x, a.x, fmaf(-ph.y, a.y, rx));
    ry = fmaf(ph.x, a.y, fmaf(ph.y, a.x, ry));
    return make_float2(rx, ry);
}

// asynchronous global -> shared copies of the next tile's inputs (all threads copy, with
// consecutive lanes on consecutive positions; a barrier after the wait publishes them)
__device__ __forceinline__ void tbr_cp16(void* sdst, const void* gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void tbr_cp8(void* sdst, const void* gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void tbr_cp4(void* sdst, const void* gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void tbr_cp(float4* sdst, const float4* gsrc) { tbr_cp16(sdst, gsrc); }
__device__ __forceinline__ void tbr_cp(float2* sdst, const float2* gsrc) { tbr_cp8(sdst, gsrc); }
__device__ __forceinline__ void tbr_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void tbr_cp_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Tensor-memory-access copies of a tile's T_{ka-1} / T_{ka-2}: one 3-D box (16-byte element,
// S columns, BH rows) per buffer from the ribbon's tensor map, issued by one thread against
// an mbarrier that expects the boxes' bytes; every thread waits on the barrier's phase before
// reading the staging buffers.  Waits are bounded: a wait that gives up raises bit 2 of the
// error flag (never expected: the copies always complete).
static constexpr int TBR_WAIT_TRIES = 1 << 22;

__device__ __forceinline__ unsigned tbr_smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tbr_mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tbr_smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void tbr_mbar_expect(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tbr_smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool tbr_mbar_wait(uint64_t* bar, unsigned parity)
{
    for (int i = 0; i < TBR_WAIT_TRIES; ++i) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(tbr_smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tbr_tma_box(void* sdst, const void* tmap, int c0, int c1, int c2,
                                            uint64_t* bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(tbr_smem_u32(sdst)),
                 "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2),
                 "r"(tbr_smem_u32(bar))
                 : "memory");
}
// generic-proxy accesses of the staging buffers (the previous tile's reads, ordered by a CTA
// barrier) before the async-proxy writes of the next boxes
__device__ __forceinline__ void tbr_fence_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Geometry of a work item (tile ti, plane element pr) as a thread sees it.
struct TBRTile {
    TBTile T;
    DevBlock B;
    int pr;
    int S;
    unsigned long long invS;  // q / S = (q * invS) >> 32, exact for q < 2^13
    bool live;                // the ribbon still has orders in this launch
};

// Descriptors of a work item staged in shared memory one item ahead: the ribbon's DevBlock
// (18 words, 8-byte aligned at word 0) and the tile (12 words); thread tid < 30 loads word
// tid.
constexpr int TBR_META_WORDS = 32;
constexpr int TBR_META_USED = 30;  // DevBlock (18 words) then TBTile (12 words)
static_assert(sizeof(DevBlock) == 18 * 4 && sizeof(TBTile) == 12 * 4, "descriptor words");

__device__ __forceinline__ int tbr_meta_load(const TBArgs& a, int w, int npairs, int tid)
{
    const int ti = w / npairs;
    if (tid < 18) return reinterpret_cast<const int*>(a.blocks + a.tiles[ti].block)[tid];
    return reinterpret_cast<const int*>(a.tiles + ti)[tid - 18];
}

__device__ __forceinline__ TBRTile tbr_tile(const int* meta, int w, int ka, int npairs)
{
    TBRTile t;
    const int ti = w / npairs;
    t.pr = w - ti * npairs;
    t.B = *reinterpret_cast<const DevBlock*>(meta);
    t.T = *reinterpret_cast<const TBTile*>(meta + 18);
    t.live = ka <= t.B.M;
    t.S = t.T.S;  // the ribbon's common stride (tile builder)
    t.invS = ((1ull << 32) + (unsigned)t.S - 1u) / (unsigned)t.S;
    return t;
}

// Walk over a thread's consecutive positions e0, e0 + 1, ...: region row rr and column cc of
// position e (site (rr, cc) is at e = rr S + cc) and the ribbon-relative site index
// rg = (R0 + rr) L + C0 + cc, advanced incrementally (one division per run, at its start).
// Columns RW .. S - 1 are pads.
struct TBRWalk {
    int rr, cc, rg;
    __device__ __forceinline__ TBRWalk(const TBRTile& t, int e0)
    {
        rr = (int)(((unsigned long long)e0 * t.invS) >> 32);
        cc = e0 - rr * t.S;
        rg = (t.T.R0 + rr) * t.B.L + t.T.C0 + cc;
    }
    __device__ __forceinline__ bool site(const TBRTile& t) const
    {
        return cc < t.T.C1 - t.T.C0 && rr < t.T.R1 - t.T.R0;
    }
    __device__ __forceinline__ bool interior(const TBRTile& t) const
    {
        const int r = t.T.R0 + rr, c = t.T.C0 + cc;
        return r >= t.T.r0 && r < t.T.r1 && c >= t.T.c0 && c < t.T.c1;
    }
    __device__ __forceinline__ void next(const TBRTile& t)
    {
        ++cc;
        ++rg;
        if (cc == t.S) {
            cc = 0;
            ++rr;
            rg += t.B.L - t.S;
        }
    }
};

// Issue the copies of a work item's inputs: T_{ka-1}, T_{ka-2} (not in the first launch), d,
// and for interior sites the accumulator the launch continues (E, or the tail when only the
// tail is read; when both are read the tail is loaded directly).  Thread tid copies positions
// tid, tid + TPB, ...
template <typename PT, int RUN, int TPB, bool FIRST, bool BOX>
__device__ __forceinline__ bool tbr_fetch(const TBArgs& a, const TBRTile& t, int npairs,
                                          PT* stX, PT* stP, PT* stA, float* stD, uint64_t* bar,
                                          bool box_ok)
{
    if (!t.live) return false;
    // boxes (kernel variant BOX, pairs of vectors) where the ribbon has tensor maps for this
    // launch's buffers and the staging buffers sit on 128-byte boundaries
    bool boxX = false, boxP = false;
    if constexpr (BOX) {
        const int mi = t.T.block * npairs + t.pr;
        boxX = box_ok && t.T.tma && a.tm_cur;
        boxP = box_ok && !FIRST && t.T.tma && a.tm_prev;
        if ((boxX || boxP) && threadIdx.x == 0) {
            tbr_fence_async();
            const unsigned box = (unsigned)t.S * (unsigned)t.T.BH * 16u;
            tbr_mbar_expect(bar, box * ((boxX ? 1u : 0u) + (boxP ? 1u : 0u)));
            if (boxX)
                tbr_tma_box(stX, static_cast<const CUtensorMap*>(a.tm_cur) + mi, 0, t.T.C0, t.T.R0,
                            bar);
            if (boxP)
                tbr_tma_box(stP, static_cast<const CUtensorMap*>(a.tm_prev) + mi, 0, t.T.C0,
                            t.T.R0, bar);
        }
    }
    const PT* in_prev = static_cast<const PT*>(a.in_prev);
    const PT* in_cur = static_cast<const PT*>(a.in_cur);
    const PT* accE = static_cast<const PT*>(a.acc_main);
    const PT* tail = static_cast<const PT*>(a.tail);
    const float* diag = static_cast<const float*>(a.diag);
    const bool done = min(a.kb, t.B.M) == t.B.M;
    const bool to_main = FIRST || (a.ka <= t.B.ksplit);
    const bool read_e = !FIRST && (to_main || done);
    const bool read_t = !FIRST && !to_main && a.prev_ka > t.B.ksplit;
    // this plane index of the ribbon's first site: psi [site][vector] (T_0 in the first
    // launch), the step's own vectors pair-planar
    const int64_t base_psi = t.B.offset * npairs + t.pr;
    const int64_t base_own = (int64_t)t.pr * a.nsites + t.B.offset;
    const PT* const accsrc = read_e ? accE : tail;
    // consecutive lanes on consecutive positions (position p = tid + k TPB): a warp's copies
    // cover a few contiguous lines of a region row, not 32 lines RUN sites apart
    const int RW = t.T.C1 - t.T.C0, RH = t.T.R1 - t.T.R0;
    const int ir0 = t.T.r0 - t.T.R0, ir1 = t.T.r1 - t.T.R0;
    const int ic0 = t.T.c0 - t.T.C0, ic1 = t.T.c1 - t.T.C0;
    const int rg0 = t.T.R0 * t.B.L + t.T.C0;
    const float* const dg = diag + t.B.offset;
#pragma unroll
    for (int k = 0; k < RUN; ++k) {
        const int p = (int)threadIdx.x + k * TPB;
        const int rr = (int)(((unsigned long long)p * t.invS) >> 32), cc = p - rr * t.S;
        if (rr < RH && cc < RW) {
            const int rg = rg0 + rr * t.B.L + cc;
            const int64_t go = base_own + rg;
            const int64_t gx = FIRST ? base_psi + (int64_t)rg * npairs : go;
            if (!boxX) tbr_cp(stX + p, in_cur + gx);
            if (!FIRST && !boxP) tbr_cp(stP + p, in_prev + go);
            tbr_cp4(stD + p, dg + rg);
            if ((read_e || read_t) && rr >= ir0 && rr < ir1 && cc >= ic0 && cc < ic1)
                tbr_cp(stA + p, accsrc + go);
        }
    }
    tbr_cp_commit();
    return boxX || boxP;
}

// One order k of parity ODD for the thread's run: dst <- 2 H~ src - dst at every position
// (src = T_{k-1}, dst = T_{k-2} in, T_k out), T_k stored to Pw, q_k T_k added to every
// position's accumulator (only interior ones are written out); HALF: the first order,
// T_1 = H~ T_0 (dst holds zeros).  Pads carry zero coupling, diagonal and values, so they
// stay exactly zero (every value read is finite: both planes are zeroed at each tile start).
// Reads Qr (T_{k-1}).
template <typename PT, int RUN, bool HALF, bool ODD>
__device__ __forceinline__ void tbr_order(const PT* __restrict__ Qr, PT* __restrict__ Pw,
                                          const PT (&src)[RUN], PT (&dst)[RUN],
                                          const float (&d)[RUN], const float (&bh)[RUN],
                                          const int (&vidx)[RUN], int zpos, int e0, bool active,
                                          float2 qk, float2 (&acc)[RUN][TBRPlane<PT>::PER])
{
    constexpr int PER = TBRPlane<PT>::PER;
    if (active) {
        PT V[RUN];
#pragma unroll
        for (int j = 0; j < RUN; ++j) V[j] = Qr[vidx[j]];
        const PT Lf = Qr[e0 > 0 ? e0 - 1 : zpos];
        const PT Rt = Qr[e0 + RUN];
#pragma unroll
        for (int j = 0; j < RUN; ++j) {
            const PT l = j > 0 ? src[j - 1] : Lf;
            const PT r = j < RUN - 1 ? src[j + 1] : Rt;
            const PT h = tbr_h(l, r, V[j], dst[j], src[j], d[j], bh[j], HALF);
#pragma unroll
            for (int c = 0; c < PER; ++c) tbr_accum<ODD>(acc[j][c], qk, tbr_get(h, c));
            dst[j] = h;
            Pw[e0 + j] = h;
        }
    }
    __syncthreads();
}

// orders k..ke, two per iteration (B <- 2 H~ A - B from plane qa into plane qb, then
// A <- 2 H~ B - A back); P0 = parity of k; a run is formed while rl >= (order - ka + 1)
template <typename PT, int RUN, bool P0>
__device__ __forceinline__ void tbr_orders_from(PT* qa, PT* qb, PT (&A)[RUN], PT (&Bv)[RUN],
                                                const float (&d)[RUN], const float (&bh)[RUN],
                                                const int (&vidx)[RUN], int zpos, int e0, int rl,
                                                int ka, int k, int ke,
                                                const float2* __restrict__ qc,
                                                float2 (&acc)[RUN][TBRPlane<PT>::PER])
{
    float2 qn = qc[k];
    for (;;) {
        float2 qk = qn;
        if (k < ke) qn = qc[k + 1];
        tbr_order<PT, RUN, false, P0>(qa, qb, A, Bv, d, bh, vidx, zpos, e0, rl >= k - ka + 1, qk,
                                      acc);
        if (k == ke) break;
        ++k;
        qk = qn;
        if (k < ke) qn = qc[k + 1];
        tbr_order<PT, RUN, false, !P0>(qb, qa, Bv, A, d, bh, vidx, zpos, e0, rl >= k - ka + 1, qk,
                                       acc);
        if (k == ke) break;
        ++k;
    }
}

// orders ka..ke: P <- 2 H~ X - P, then X <- 2 H~ P - X, ...; in the first launch (ka = 1)
// order 1 is peeled off (T_1 = H~ T_0, a compile-time halving) and the loop goes on from
// order 2 with the roles swapped
template <typename PT, int RUN, bool FIRST, bool P0>
__device__ __forceinline__ void tbr_orders(PT* plane0, PT* plane1, PT (&X)[RUN], PT (&P)[RUN],
                                           const float (&d)[RUN], const float (&bh)[RUN],
                                           const int (&vidx)[RUN], int zpos, int e0, int rl,
                                           int ka, int ke, const float2* __restrict__ qc,
                                           float2 (&acc)[RUN][TBRPlane<PT>::PER])
{
    if constexpr (FIRST) {
        tbr_order<PT, RUN, true, true>(plane0, plane1, X, P, d, bh, vidx, zpos, e0, rl >= 1,
                                       qc[ka], acc);
        if (ka < ke)
            tbr_orders_from<PT, RUN, false>(plane1, plane0, P, X, d, bh, vidx, zpos, e0, rl, ka,
                                            ka + 1, ke, qc, acc);
    } else {
        tbr_orders_from<PT, RUN, P0>(plane0, plane1, X, P, d, bh, vidx, zpos, e0, rl, ka, ka, ke,
                                     qc, acc);
    }
}

// Dynamic shared memory: two planes of NPOS + 1 elements (positions and the trailing zero),
// staging for T_{ka-1}, T_{ka-2}, the accumulator and d of the next tile; each part starts on a
// 128-byte boundary (the boxes' destinations).
template <typename PT, int RUN, int TPB> struct TBRLayout {
    static constexpr size_t NPOS = (size_t)RUN * TPB, E = sizeof(PT);
    static constexpr size_t up(size_t x) { return (x + 127) & ~(size_t)127; }
    static constexpr size_t plane1 = up((NPOS + 1) * E);
    static constexpr size_t stX = up(plane1 + (NPOS + 1) * E);
    static constexpr size_t stP = up(stX + NPOS * E);
    static constexpr size_t stA = up(stP + NPOS * E);
    static constexpr size_t stD = up(stA + NPOS * E);
    static constexpr size_t bytes = stD + NPOS * sizeof(float);
};
template <typename PT, int RUN, int TPB>
__host__ __device__ constexpr size_t tbr_smem_layout()
{
    return TBRLayout<PT, RUN, TPB>::bytes;
}

template <typename PT, int RUN, int TPB, bool FIRST, bool BOX>
__global__ void __launch_bounds__(TPB, 1) k_rec_tbr(TBArgs a)
{
    static_assert(!BOX || sizeof(PT) == 16, "boxes carry pairs of vectors");
    constexpr int PER = TBRPlane<PT>::PER;
    constexpr int NPOS = RUN * TPB;
    using LY = TBRLayout<PT, RUN, TPB>;
    extern __shared__ __align__(128) unsigned char tbr_smem_raw[];
    PT* const plane0 = reinterpret_cast<PT*>(tbr_smem_raw);
    PT* const plane1 = reinterpret_cast<PT*>(tbr_smem_raw + LY::plane1);
    PT* const stX = reinterpret_cast<PT*>(tbr_smem_raw + LY::stX);
    PT* const stP = reinterpret_cast<PT*>(tbr_smem_raw + LY::stP);
    PT* const stA = reinterpret_cast<PT*>(tbr_smem_raw + LY::stA);
    float* const stD = reinterpret_cast<float*>(tbr_smem_raw + LY::stD);
    // the boxes' destinations must start on 128-byte boundaries (else per-thread copies)
    const bool box_ok = (tbr_smem_u32(tbr_smem_raw) & 127u) == 0u;
    const PT zero = tbr_zero((PT*)nullptr);
    const int tid = threadIdx.x;
    const int e0 = tid * RUN;
    const int npairs = a.nvec / PER;  // plane elements per site in global memory
    const int nvec = a.nvec;

    PT* __restrict__ out_prev = static_cast<PT*>(a.out_prev);
    PT* __restrict__ out_cur = static_cast<PT*>(a.out_cur);
    PT* __restrict__ accE = static_cast<PT*>(a.acc_main);
    PT* __restrict__ tail = static_cast<PT*>(a.tail);
    PT* __restrict__ psi = static_cast<PT*>(a.psi);
    const float2* __restrict__ qc = static_cast<const float2*>(a.qcoef);
    __shared__ __align__(8) uint64_t s_bar;  // completion of the next tile's boxes
    unsigned bar_parity = 0;                  // parity of the next phase to wait for
    if (tid == 0) {
        plane0[NPOS] = zero;
        plane1[NPOS] = zero;
        if constexpr (BOX) tbr_mbar_init(&s_bar);
    }

    __shared__ __align__(16) int s_meta[2][TBR_META_WORDS];  // descriptors of items it, it + 1
    const int nwork = a.ntiles * npairs;
    int w = blockIdx.x;
    const bool any = w < nwork;
    if (any && tid < TBR_META_USED) s_meta[0][tid] = tbr_meta_load(a, w, npairs, tid);
    // the descriptors of the CTA's next item, loaded one item ahead (two dependent loads: the
    // tile, then its ribbon) so that later items find them arrived during the orders
    int meta_next = 0;
    if (tid < TBR_META_USED && w + (int)gridDim.x < nwork)
        meta_next = tbr_meta_load(a, w + (int)gridDim.x, npairs, tid);
    __syncthreads();
    TBRTile t;
    bool boxed = false;  // the fetched item's inputs come (partly) by boxes
    if (any) {
        t = tbr_tile(s_meta[0], w, a.ka, npairs);
        boxed = tbr_fetch<PT, RUN, TPB, FIRST, BOX>(a, t, npairs, stX, stP, stA, stD, &s_bar, box_ok);
    }
    for (int it = 0; w < nwork; w += gridDim.x, ++it) {
        const int wn = w + (int)gridDim.x;
        float n2[FIRST ? PER : 1];  // ||T_0||^2 of the interior (first launch)
#pragma unroll
        for (int q = 0; q < (FIRST ? PER : 1); ++q) n2[q] = 0.f;
        const TBRTile cur = t;
        const TBTile& T = cur.T;
        const DevBlock& B = cur.B;
        // this work item's inputs, copied during the previous item's orders by all threads;
        // the barrier also ends the previous item's reads of the planes
        tbr_cp_wait();
        if (BOX && boxed) {
            if (!tbr_mbar_wait(&s_bar, bar_parity)) {
                atomicOr(a.errflag, 2);
                tbr_mbar_wait(&s_bar, bar_parity);  // once more for the boxes in flight
            }
            bar_parity ^= 1u;
        }
        __syncthreads();
        PT X[RUN], P[RUN];
        float d[RUN], bh[RUN];
        int vidx[RUN];
        unsigned interm = 0;
        int rl = -1;  // last order index (1-based shrink) at which the run is formed
        float2 acc[RUN][PER];
        const int ke = min(a.kb, B.M);
        const bool done = (ke == B.M);
        const bool to_main = FIRST || (a.ka <= B.ksplit);
        const bool read_e = !FIRST && (to_main || done);
        const bool read_t = !FIRST && !to_main && a.prev_ka > B.ksplit;
        if (cur.live) {
            const int RW = T.C1 - T.C0, RH = T.R1 - T.R0;
            const bool open_t = T.R0 > 0, open_b = T.R1 < B.W, open_l = T.C0 > 0, open_r = T.C1 < B.L;
            const float bhi = (float)B.beta;  // exact: the plan chooses a so
            const int ir0 = T.r0 - T.R0, ir1 = T.r1 - T.R0, ic0 = T.c0 - T.C0, ic1 = T.c1 - T.C0;
            const bool ld_a = read_e || read_t;
            // Every position's staged inputs are loaded without conditions (all indexes lie in
            // the buffers) and kept only at sites, so the loads do not wait behind per-position
            // branches.  The vertical neighbour r +- 1 of a region row exists in the region
            // exactly when it exists in the ribbon, since the region never leaves the ribbon.
            int rr = (int)(((unsigned long long)e0 * cur.invS) >> 32), cc = e0 - rr * cur.S;
#pragma unroll
            for (int j = 0; j < RUN; ++j) {
                const int e = e0 + j;
                const PT xs = stX[e];
                const PT ps = FIRST ? zero : stP[e];
                const float ds = stD[e];
                const PT as = ld_a ? stA[e] : zero;
                const bool site = cc < RW && rr < RH;
                const bool inter = rr >= ir0 && rr < ir1 && cc >= ic0 && cc < ic1;  // a site
                const bool up = (T.R0 + rr + T.C0 + cc) & 1;  // vertical neighbour r - 1 (else r + 1)
                const int lim = tbr_limit(rr, cc, RH, RW, up, open_t, open_b, open_l, open_r);
                rl = site ? max(rl, lim) : rl;
                vidx[j] = !site ? NPOS : up ? (rr > 0 ? e - cur.S : NPOS) : (rr + 1 < RH ? e + cur.S : NPOS);
                X[j] = site ? xs : zero;
                P[j] = site ? ps : zero;
                d[j] = site ? ds : 0.f;
                bh[j] = site ? bhi : 0.f;
                interm |= inter ? (1u << j) : 0u;
                const PT ea = inter ? as : zero;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    acc[j][q] = tbr_get(ea, q);
                    if constexpr (FIRST) {  // ||T_0||^2 in FP32: feeds only the divergence check
                        const float2 x = tbr_get(inter ? xs : zero, q);
                        n2[q] = fmaf(x.x, x.x, fmaf(x.y, x.y, n2[q]));
                    }
                }
                if (++cc == cur.S) {
                    cc = 0;
                    ++rr;
                }
            }
            if (read_e && read_t) {  // E + tail at the ribbon's last order (the tail from global)
                TBRWalk wk(cur, e0);
#pragma unroll
                for (int j = 0; j < RUN; ++j, wk.next(cur)) {
                    if (!((interm >> j) & 1u)) continue;
                    const PT tv = tail[(int64_t)cur.pr * a.nsites + B.offset + wk.rg];
#pragma unroll
                    for (int q = 0; q < PER; ++q) {
                        const float2 y = tbr_get(tv, q);
                        acc[j][q].x += y.x;
                        acc[j][q].y += y.y;
                    }
                }
            }
            // T_{ka-1} of every position into plane 0, plane 1 zeroed (pads and all)
#pragma unroll
            for (int j = 0; j < RUN; ++j) {
                plane0[e0 + j] = X[j];
                plane1[e0 + j] = zero;
            }
            if (FIRST) {  // q_0 T_0
                const float2 q0 = qc[B.coef_off + 0];
#pragma unroll
                for (int j = 0; j < RUN; ++j)
#pragma unroll
                    for (int q = 0; q < PER; ++q) tbr_accum<false>(acc[j][q], q0, tbr_get(X[j], q));
            }
        }
        // plane 0 complete; the barrier also orders this tile's reads of the staging buffers
        // before the copies of the next item below overwrite them, and publishes the next
        // item's descriptors (slot (it + 1) & 1 was last read two items ago)
        if (tid < TBR_META_USED) s_meta[(it + 1) & 1][tid] = meta_next;
        __syncthreads();
        // the descriptors of the item after the next: loads in flight during this item's orders
        meta_next = 0;
        if (tid < TBR_META_USED && wn + (int)gridDim.x < nwork)
            meta_next = tbr_meta_load(a, wn + (int)gridDim.x, npairs, tid);
        // the next work item's inputs stream in while this one runs its orders
        boxed = false;
        if (wn < nwork) {
            t = tbr_tile(s_meta[(it + 1) & 1], wn, a.ka, npairs);
            boxed = tbr_fetch<PT, RUN, TPB, FIRST, BOX>(a, t, npairs, stX, stP, stA, stD, &s_bar, box_ok);
        }
        if (cur.live) {
            if (a.ka & 1)
                tbr_orders<PT, RUN, FIRST, true>(plane0, plane1, X, P, d, bh, vidx, NPOS, e0, rl,
                                                 a.ka, ke, qc + B.coef_off, acc);
            else
                tbr_orders<PT, RUN, FIRST, false>(plane0, plane1, X, P, d, bh, vidx, NPOS, e0, rl,
                                                  a.ka, ke, qc + B.coef_off, acc);
            // T_ke is in P when ke - ka is even (the last order ran the first half), else in X
            const bool last_in_p = ((ke - a.ka) & 1) == 0;
            float lim[PER];
#pragma unroll
            for (int c = 0; c < PER; ++c)
                lim[c] = done ? (float)(4.0 * a.norm2[((size_t)T.block * nvec + cur.pr * PER + c) * 2]) : 0.f;
            float2 ph, pl;
            ph.x = (float)B.ph_re;
            pl.x = (float)(B.ph_re - (double)ph.x);
            ph.y = (float)B.ph_im;
            pl.y = (float)(B.ph_im - (double)ph.y);
            if (!done) {
                // T_ke and T_{ke-1} of the interior straight from the planes (the last order's
                // barrier completed them; the next item's barrier ends these reads), consecutive
                // lanes on consecutive positions
                const PT* const planeK = last_in_p ? plane1 : plane0;
                const PT* const planeK1 = last_in_p ? plane0 : plane1;
                const int ir0 = T.r0 - T.R0, ir1 = T.r1 - T.R0;
                const int ic0 = T.c0 - T.C0, ic1 = T.c1 - T.C0;
                const int64_t gb = (int64_t)B.offset + (int64_t)T.R0 * B.L + T.C0;
#pragma unroll
                for (int k = 0; k < RUN; ++k) {
                    const int p = tid + k * TPB;
                    const int rr = (int)(((unsigned long long)p * cur.invS) >> 32);
                    const int cc = p - rr * cur.S;
                    if (rr >= ir0 && rr < ir1 && cc >= ic0 && cc < ic1) {
                        const int64_t g = (int64_t)cur.pr * a.nsites + gb + (int64_t)rr * B.L + cc;
                        out_cur[g] = planeK[p];
                        out_prev[g] = planeK1[p];
                    }
                }
            }
            TBRWalk wk(cur, e0);
#pragma unroll
            for (int j = 0; j < RUN; ++j, wk.next(cur)) {
                if (!((interm >> j) & 1u)) continue;
                PT aP;
#pragma unroll
                for (int c = 0; c < PER; ++c) tbr_put(aP, c, acc[j][c]);
                if (!done) {
                    const int64_t g = (int64_t)cur.pr * a.nsites + B.offset + wk.rg;
                    if (to_main) accE[g] = aP;
                    else tail[g] = aP;
                } else {
                    const PT tk = last_in_p ? P[j] : X[j];
                    PT oP;
#pragma unroll
                    for (int c = 0; c < PER; ++c) {
                        tbr_put(oP, c, tbr_phase(acc[j][c], ph, pl));  // E + tail + partial
                        // growth check |T_M|^2 <= 4 ||psi||^2, in FP32 (a divergence test)
                        const float2 tv = tbr_get(tk, c);
                        const float t2 = fmaf(tv.x, tv.x, tv.y * tv.y);
                        if (!(t2 <= lim[c])) atomicOr(a.errflag, 1);
                    }
                    psi[(B.offset + wk.rg) * npairs + cur.pr] = oP;
                }
            }
        }
        if constexpr (FIRST) {
            // ||psi||^2 per (ribbon, vector) for the growth check of the ribbon's last order:
            // FP32 warp sums added to the slot, which the step zeroes before its first launch
            // (summation order free: the check compares against 4 ||psi||^2)
            if (cur.live) {
                const int lane = tid & 31;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    float xs = n2[q];
                    for (int off = 16; off > 0; off >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, off);
                    if (lane == 0 && xs != 0.f)
                        atomicAdd(a.red_out + ((size_t)T.block * nvec + cur.pr * PER + q) * 2, (double)xs);
                }
            }
        }
    }
    tbr_cp_wait();  // no copy may be left in flight when the CTA exits
}

// ---- dispatch ---------------------------------------------------------------------------
// Compiled (vectors per plane element, run, threads): pairs of vectors (nvec 2 and 4) and single
// vectors (nvec 1); one CTA per SM (up to 1024 threads) or two.
#define CHEB_TBR_SHAPES(X)                                                             \
    X(float4, 3, 768) X(float4, 3, 512) X(float4, 5, 512) X(float4, 7, 384)             \
    X(float4, 9, 256)                                                                    \
    X(float2, 3, 1024) X(float2, 7, 512) X(float2, 5, 512)

static int tbr_elem_bytes(int nv) { return nv >= 2 ? 16 : 8; }

bool tbr_supported(int nv, int run, int tpb)
{
    const int eb = tbr_elem_bytes(nv);
#define CHEB_TBR_IS(PT, RUN, TPB) \
    if ((int)sizeof(PT) == eb && run == RUN && tpb == TPB) return true;
    CHEB_TBR_SHAPES(CHEB_TBR_IS)
#undef CHEB_TBR_IS
    return false;
}

size_t tbr_smem_bytes(int nv, int run, int tpb)
{
#define CHEB_TBR_SM(PT, RUN, TPB) \
    if ((int)sizeof(PT) == tbr_elem_bytes(nv) && run == RUN && tpb == TPB) return tbr_smem_layout<PT, RUN, TPB>();
    CHEB_TBR_SHAPES(CHEB_TBR_SM)
#undef CHEB_TBR_SM
    return 0;
}

// the variant with boxes exists for pairs of vectors only
template <typename PT> struct TBRBox {
    static constexpr bool value = sizeof(PT) == 16;
};

template <typename PT, int RUN, int TPB>
static int tbr_attr_t()
{
    const int smem = (int)tbr_smem_layout<PT, RUN, TPB>();
    CHEB_CUDA(cudaFuncSetAttribute(k_rec_tbr<PT, RUN, TPB, true, false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CHEB_CUDA(cudaFuncSetAttribute(k_rec_tbr<PT, RUN, TPB, false, false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    if constexpr (TBRBox<PT>::value) {
        CHEB_CUDA(cudaFuncSetAttribute(k_rec_tbr<PT, RUN, TPB, true, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        CHEB_CUDA(cudaFuncSetAttribute(k_rec_tbr<PT, RUN, TPB, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    }
    return CHEB_OK;
}

// resident CTAs per SM of a shape: the fewest over its variants (FIRST and not, with and
// without boxes)
template <typename PT, int RUN, int TPB>
static int tbr_occ_t()
{
    const size_t smem = tbr_smem_layout<PT, RUN, TPB>();
    int o[4] = {0, 0, 0, 0};
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[0], k_rec_tbr<PT, RUN, TPB, true, false>, TPB, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[1], k_rec_tbr<PT, RUN, TPB, false, false>, TPB, smem);
    o[2] = o[3] = o[1];
    if constexpr (TBRBox<PT>::value) {
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[2], k_rec_tbr<PT, RUN, TPB, true, true>, TPB, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[3], k_rec_tbr<PT, RUN, TPB, false, true>, TPB, smem);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return std::min(std::min(o[0], o[1]), std::min(o[2], o[3]));
}

int tbr_blocks_per_sm(int nv, int run, int tpb)
{
    const int eb = tbr_elem_bytes(nv);
#define CHEB_TBR_OCC(PT, RUN, TPB) \
    if ((int)sizeof(PT) == eb && run == RUN && tpb == TPB) return tbr_occ_t<PT, RUN, TPB>();
    CHEB_TBR_SHAPES(CHEB_TBR_OCC)
#undef CHEB_TBR_OCC
    return 0;
}

int tbr_configure(int nv, int run, int tpb)
{
    const int eb = tbr_elem_bytes(nv);
#define CHEB_TBR_ATTR(PT, RUN, TPB) \
    if ((int)sizeof(PT) == eb && run == RUN && tpb == TPB) return tbr_attr_t<PT, RUN, TPB>();
    CHEB_TBR_SHAPES(CHEB_TBR_ATTR)
#undef CHEB_TBR_ATTR
    return fail(CHEB_ERR_UNSUPPORTED, "run blocking: unsupported nvec / run / threads");
}

template <typename PT, int RUN, int TPB>
static void tbr_launch_t(const TBArgs& a, int grid, cudaStream_t s, bool box)
{
    const size_t smem = tbr_smem_layout<PT, RUN, TPB>();
    if constexpr (TBRBox<PT>::value) {
        if (box) {
            if (a.ka == 1) k_rec_tbr<PT, RUN, TPB, true, true><<<grid, TPB, smem, s>>>(a);
            else k_rec_tbr<PT, RUN, TPB, false, true><<<grid, TPB, smem, s>>>(a);
            return;
        }
    }
    if (a.ka == 1) k_rec_tbr<PT, RUN, TPB, true, false><<<grid, TPB, smem, s>>>(a);
    else k_rec_tbr<PT, RUN, TPB, false, false><<<grid, TPB, smem, s>>>(a);
}

int tbr_launch(Plan* p, const TBArgs& a, cudaStream_t s)
{
    const int per = p->nvec >= 2 ? 2 : 1;
    // persistent: as many CTAs as are resident (the caller's count if set), each looping over
    // work items, so that the copies of a CTA's next item overlap the orders of its current one
    int grid = a.ntiles * (p->nvec / per);
    const int cap = p->tb_grid_cap > 0 ? p->tb_grid_cap : p->tbr_resident;
    if (cap > 0 && grid > cap) grid = cap;
    if (grid < 1) return CHEB_OK;
    const int eb = tbr_elem_bytes(p->nvec), run = p->tb_spt, tpb = p->tb_tpb;
    // the variant with boxes when some ribbon of this launch has tensor maps
    const bool box = p->tb_kernel == CHEB_TB_RUNS_TMA && (a.tm_cur || a.tm_prev);
    bool ok = false;
#define CHEB_TBR_GO(PT, RUN, TPB)                                     \
    if (!ok && (int)sizeof(PT) == eb && run == RUN && tpb == TPB) {   \
        tbr_launch_t<PT, RUN, TPB>(a, grid, s, box);                  \
        ok = true;                                                    \
    }
    CHEB_TBR_SHAPES(CHEB_TBR_GO)
#undef CHEB_TBR_GO
    if (!ok) return fail(CHEB_ERR_UNSUPPORTED, "run blocking: unsupported nvec / run / threads");
    CHEB_CUDA(cudaGetLastError());
    p->launches++;
    return CHEB_OK;
}

// ---- tensor maps (host) ---------------------------------------------------------------------
// The CUDA driver API's tensor-map encoder, looked up once through the runtime (no link to
// libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tbr_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

bool tbr_tma_available() { return tbr_encoder() != nullptr; }

// Maps of one buffer (base: element 0 of the plan's [site][vec] complex64 vector) for the
// ribbons of a tile set: out[q * pairs + pr] views ribbon q's plane element pr as a 3-D tensor
// (4 floats, L columns of pairs * 16 bytes, W rows of L pairs * 16 bytes) with a box of
// (4, S, BH); columns and rows beyond the ribbon read as zero.  Ribbons without boxes keep a
// zeroed map that the kernel never uses.
static bool tbr_encode_buffer(const Plan* p, const TBSet& set, const void* base, bool planar,
                              CUtensorMap* out)
{
    const auto enc = tbr_encoder();
    const int npairs = p->nvec / 2;
    for (int q = 0; q < p->nblocks; ++q) {
        const TBTile& t = set.first[(size_t)q];
        const DevBlock& B = p->hblocks[q];
        for (int pr = 0; pr < npairs; ++pr) {
            CUtensorMap& m = out[(size_t)q * npairs + pr];
            std::memset(&m, 0, sizeof(m));
            if (!t.tma) continue;
            // psi: [site][vector], pair pr at 16 bytes per pair; the step's own vectors:
            // pair-planar, pair pr's sites contiguous
            const size_t first = planar ? (size_t)pr * p->n_sites + B.offset
                                        : (size_t)B.offset * npairs + pr;
            const size_t col = planar ? 16 : (size_t)npairs * 16;
            char* g = static_cast<char*>(const_cast<void*>(base)) + first * 16;
            const cuuint64_t dims[3] = {4, (cuuint64_t)B.L, (cuuint64_t)B.W};
            const cuuint64_t strides[2] = {(cuuint64_t)col, (cuuint64_t)B.L * col};
            const cuuint32_t box[3] = {4, (cuuint32_t)t.S, (cuuint32_t)t.BH};
            const cuuint32_t estr[3] = {1, 1, 1};
            if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, g, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
                CUDA_SUCCESS)
                return false;
        }
    }
    return true;
}

static bool tbr_boxes(const Plan* p)
{
    return p->tb_kernel == CHEB_TB_RUNS_TMA && p->nvec >= 2 && !p->tb_sched.empty() &&
           tbr_tma_available();
}

// Maps of the buffers of launches 1.. of the step (the two recurrence pairs; launch 0 reads
// psi, whose maps are made per psi pointer); psi slots invalidated.
int tbr_maps_prepare(Plan* p)
{
    for (Plan::TMPsi& t : p->tm_psi) t = Plan::TMPsi{};
    if (!tbr_boxes(p)) return CHEB_OK;
    const size_t nmap = (size_t)p->nblocks * (p->nvec / 2);
    p->tmap_array = nmap * sizeof(CUtensorMap);
    const size_t narrays = 2 * p->tb_sched.size() + Plan::kGraphSlots + 1;
    const size_t need = narrays * p->tmap_array;
    if (p->tmaps_cap < need) {
        if (p->d_tmaps) cudaFree(p->d_tmaps);
        p->d_tmaps = nullptr;
        p->tmaps_cap = 0;
        if (cudaMalloc(&p->d_tmaps, need) != cudaSuccess) return fail(CHEB_ERR_NOMEM, "tensor maps");
        p->tmaps_cap = need;
    }
    std::vector<CUtensorMap> h(narrays * nmap);
    std::memset(h.data(), 0, h.size() * sizeof(CUtensorMap));
    void* pairs[2][2] = {{p->d_A, p->d_B}, {p->d_C, p->d_D}};
    for (size_t i = 1; i < p->tb_sched.size(); ++i) {
        const TBSet& set = p->tb_sets[p->tb_sched[i].set];
        if (!tbr_encode_buffer(p, set, pairs[(i - 1) & 1][1], true, &h[(2 * i + 0) * nmap]) ||
            !tbr_encode_buffer(p, set, pairs[(i - 1) & 1][0], true, &h[(2 * i + 1) * nmap]))
            return fail(CHEB_ERR_CUDA, "tensor map encoding");
    }
    CHEB_CUDA(cudaMemcpy(p->d_tmaps, h.data(), need, cudaMemcpyHostToDevice));
    return CHEB_OK;
}

// psi's maps for launch 0 into psi slot `slot`, ordered on stream s (outside any capture)
int tbr_maps_psi(Plan* p, const void* psi, int slot, cudaStream_t s)
{
    if (!tbr_boxes(p) || !p->d_tmaps) return CHEB_OK;
    Plan::TMPsi& key = p->tm_psi[slot];
    if (key.psi == psi && key.epoch == p->shape_epoch) return CHEB_OK;
    const size_t nmap = (size_t)p->nblocks * (p->nvec / 2);
    std::vector<CUtensorMap> h(nmap);
    if (!tbr_encode_buffer(p, p->tb_sets[p->tb_sched[0].set], psi, false, h.data()))
        return fail(CHEB_ERR_CUDA, "tensor map encoding");
    char* dst = static_cast<char*>(p->d_tmaps) + (2 * p->tb_sched.size() + slot) * p->tmap_array;
    // pageable source: the call returns once the data is staged, and the copy is ordered on s
    CHEB_CUDA(cudaMemcpyAsync(dst, h.data(), p->tmap_array, cudaMemcpyHostToDevice, s));
    key.psi = psi;
    key.epoch = p->shape_epoch;
    return CHEB_OK;
}

// The map array a launch uses (which: 0 = T_{ka-1}, 1 = T_{ka-2}), or NULL for per-thread copies.
const void* tbr_maps_for(const Plan* p, int launch, int which, const void* psi, int slot)
{
    if (!tbr_boxes(p) || !p->d_tmaps) return nullptr;
    const char* base = static_cast<const char*>(p->d_tmaps);
    if (launch == 0) {
        if (slot < 0) return nullptr;
        const Plan::TMPsi& key = p->tm_psi[slot];
        if (which != 0 || key.psi != psi || key.epoch != p->shape_epoch) return nullptr;
        return base + (2 * p->tb_sched.size() + slot) * p->tmap_array;
    }
    return base + (2 * (size_t)launch + which) * p->tmap_array;
}

// Host work model of one launch of this kernel (cheb_plan_step_model)
void tbr_model_launch(const Plan* p, const std::vector<TBTile>& tiles, int ka, int kb,
                      int prev_ka, TBModel& m)
{
    const int nv = p->nvec;
    const int per = nv >= 2 ? 2 : 1;
    const double eb = tbr_elem_bytes(nv);
    const double nel = nv / per;  // plane elements per site (CTAs per tile)
    const int run = p->tb_spt, npos = p->tb_spt * p->tb_tpb;
    const bool first = ka == 1;
    for (const TBTile& T : tiles) {
        const DevBlock& B = p->hblocks[T.block];
        if (ka > B.M) continue;
        const int ke = std::min(kb, (int)B.M), ns = ke - ka + 1;
        const bool done = ke == B.M;
        const int RW = T.C1 - T.C0, RH = T.R1 - T.R0, S = T.S;  // the ribbon's stride
        const double inter = (double)(T.r1 - T.r0) * (T.c1 - T.c0);
        const bool ot = T.R0 > 0, ob = T.R1 < B.W, ol = T.C0 > 0, orr = T.C1 < B.L;
        // runs: positions t run .. t run + run - 1; a run is formed while any site is valid;
        // every non-pad position of a formed run is formed
        double formed = 0.0, run_orders = 0.0;
        for (int t = 0; t * run < npos; ++t) {
            int rl = -1, sites = 0;
            for (int j = 0; j < run; ++j) {
                const int q = t * run + j;
                const int rr = q / S, cc = q - rr * S;
                if (rr >= RH || cc >= RW) continue;
                ++sites;
                const bool up = ((T.R0 + rr) + (T.C0 + cc)) & 1;
                rl = std::max(rl, tbr_limit(rr, cc, RH, RW, up, ot, ob, ol, orr));
            }
            const int n = std::max(0, std::min(ns, rl));
            formed += (double)sites * n;
            run_orders += n;
        }
        m.useful += inter * ns;
        m.computed += formed;
        // per formed run-order: RUN vertical loads, two run-end loads and RUN stores (pads
        // included); per tile: both planes written over all positions, and the staging copies of
        // the inputs (T_{ka-1}, T_{ka-2}: the sites, or S x BH box elements; d and the interior's
        // accumulator), written once and read back once at the sites; all times the CTAs of the
        // tile (one per plane element)
        const double vin = first ? 1.0 : 2.0;
        const double staged = T.tma ? (double)T.S * T.BH : (double)RH * RW;
        const bool to_main = first || ka <= B.ksplit;
        const bool read_e = !first && (to_main || done);
        const bool read_t = !first && !to_main && prev_ka > B.ksplit;
        const double acc_in = (read_e ? 1.0 : 0.0) + (read_t ? 1.0 : 0.0);
        const double sites = (double)RH * RW;
        m.smem += nel * (eb * run_orders * (2.0 * run + 2.0) + 2.0 * eb * npos +
                         vin * eb * (staged + sites) + 2.0 * sites * 4.0 +
                         2.0 * inter * eb * (acc_in > 0 ? 1.0 : 0.0));
        const double outs = done ? 1.0 : 3.0;
        m.l2 += sites * (vin * nel * eb + 4.0 * nel) + inter * nel * eb * (acc_in + outs);
    }
}

}  // namespace cheb
