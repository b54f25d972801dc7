// Gradient of a real objective P(psi_n), psi_{s+1} = U(dt) psi_s, with respect to the on-site
// potential V_i (the diagonal of H).  The paper has no gradient; this is reverse-mode
// differentiation of Eqs. (U_1) and (rec) with a and b held fixed, so dH~/dV_i = e_i e_i^T/a.
//
// Convention: for real P, xbar = dP/d(conj x) and dP = 2 Re(xbar^+ dx).  With lambda = psibar
// of the step's output, the adjoints w_k of the recurrence vectors v_k obey (Clenshaw form)
//   w_M     = conj(C_M) lambda
//   w_{M-1} = conj(C_{M-1}) lambda + 2 H~ w_M
//   w_k     = conj(C_k) lambda + 2 H~ w_{k+1} - w_{k+2}          1 <= k <= M-2
//   w_0     = conj(C_0) lambda +   H~ w_1     - w_2
// and the step contributes  dP/dV_i += (4/a) sum_{k=1}^{M-1} Re(conj(w_{k+1,i}) v_{k,i})
//                                      + (2/a) Re(conj(w_{1,i}) v_{0,i});
// the input adjoint is psibar_s = w_0.  The forward vectors v_k of a step are needed in
// reverse order: the forward pass keeps ceil(sqrt(M+1)) checkpoint pairs (v_{jS}, v_{jS+1})
// and each segment is recomputed into a buffer of S vectors just before it is reversed.
// The step inputs psi_s are stored for every step of the trajectory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cheb_internal.cuh"

namespace cheb {

template <typename R> struct AV2;
template <> struct AV2<double> {
    using C = double2;
    static __device__ __forceinline__ C make(double x, double y) { return make_double2(x, y); }
};
template <> struct AV2<float> {
    using C = float2;
    static __device__ __forceinline__ C make(float x, float y) { return make_float2(x, y); }
};

// Geometry of the single ribbon (or 1D grid) of an adjoint plan.  The kernels run on a 2-D
// grid: threads over the columns c, grid rows over the ribbon rows r (grid-stride), and loop
// over the nvec vectors of a site, so no index needs a division.
struct AdjGeo {
    int32_t W, L, nvec;
    int32_t diag_per_vec;
    double beta;      // 2 h_offdiag / a
    const void* diag; // d_i = 2 (H_ii - b) / a, [site] or [site][vec]
};

// 2 H~ x of vector v at site (r, c), element index idx = site * nvec + v
template <typename R>
__device__ __forceinline__ typename AV2<R>::C adj_2h(const typename AV2<R>::C* __restrict__ x,
                                                   const AdjGeo& g, int r, int c, int64_t idx,
                                                   R d)
{
    const int vr = ((r + c) & 1) ? r - 1 : r + 1;
    const int64_t rowstep = (int64_t)g.L * g.nvec;
    R sx = 0, sy = 0;
    if (c > 0) { const auto y = x[idx - g.nvec]; sx += y.x; sy += y.y; }
    if (c + 1 < g.L) { const auto y = x[idx + g.nvec]; sx += y.x; sy += y.y; }
    if (vr >= 0 && vr < g.W) {
        const auto y = x[vr > r ? idx + rowstep : idx - rowstep];
        sx += y.x;
        sy += y.y;
    }
    const auto o = x[idx];
    const R beta = (R)g.beta;
    return AV2<R>::make(fma(d, o.x, beta * sx), fma(d, o.y, beta * sy));
}

// forward recurrence without accumulation: out = H~ cur (first) or 2 H~ cur - prev
template <typename R>
__global__ void k_adj_forward(AdjGeo g, const void* cur_, const void* prev_, void* out_, int first)
{
    using C = typename AV2<R>::C;
    const C* cur = static_cast<const C*>(cur_);
    const C* prev = static_cast<const C*>(prev_);
    C* out = static_cast<C*>(out_);
    const R* diag = static_cast<const R*>(g.diag);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.L) return;
    for (int r = blockIdx.y; r < g.W; r += gridDim.y) {
        const int64_t site = (int64_t)r * g.L + c;
        for (int v = 0; v < g.nvec; ++v) {
            const int64_t idx = site * g.nvec + v;
            const R d = g.diag_per_vec ? diag[idx] : diag[site];
            C h = adj_2h<R>(cur, g, r, c, idx, d);
            if (first) {
                h.x *= (R)0.5;
                h.y *= (R)0.5;
            } else {
                const C pv = prev[idx];
                h.x -= pv.x;
                h.y -= pv.y;
            }
            out[idx] = h;
        }
    }
}

// reverse step k: wk_out = conj(C_k) lam + f H~ w1 - w2 (f = 2, or 1 at k = 0; no matvec at
// k = M; no w2 for k >= M-1), grad += g Re(conj(w1) v_k) for k < M (g = 4/a, or 2/a at k = 0)
template <typename R>
__global__ void k_adj_reverse(AdjGeo g, int k, int M, const void* lam_, const void* w1_,
                              void* w2out_, const void* vk_, const void* qcoef_, int coef_off,
                              double ph_re, double ph_im, double a, double* grad)
{
    using C = typename AV2<R>::C;
    const C* lam = static_cast<const C*>(lam_);
    const C* w1 = static_cast<const C*>(w1_);
    C* w2out = static_cast<C*>(w2out_);
    const C* vk = static_cast<const C*>(vk_);
    const C* qc = static_cast<const C*>(qcoef_);  // (hi, lo) pairs
    const R* diag = static_cast<const R*>(g.diag);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.L) return;
    const C qq = qc[coef_off + k];
    // conj(C_k) = conj(ph) q_k (1 for even k, +i for odd k)
    const R pr = (R)ph_re, pim = -(R)ph_im;
    const double gfac = (k == 0 ? 2.0 : 4.0) / a;
    for (int r = blockIdx.y; r < g.W; r += gridDim.y) {
        const int64_t site = (int64_t)r * g.L + c;
        double gsum = 0.0;
        for (int v = 0; v < g.nvec; ++v) {
            const int64_t idx = site * g.nvec + v;
            const C l = lam[idx];
            C lp = AV2<R>::make(pr * l.x - pim * l.y, pr * l.y + pim * l.x);
            if (k & 1) lp = AV2<R>::make(-lp.y, lp.x);  // i * lp
            C wk = AV2<R>::make(fma(qq.x, lp.x, qq.y * lp.x), fma(qq.x, lp.y, qq.y * lp.y));
            if (k < M) {
                const R d = g.diag_per_vec ? diag[idx] : diag[site];
                const C h = adj_2h<R>(w1, g, r, c, idx, d);
                const R f = (k == 0) ? (R)0.5 : (R)1.0;
                wk.x += f * h.x;
                wk.y += f * h.y;
                if (k < M - 1) {
                    const C w2 = w2out[idx];
                    wk.x -= w2.x;
                    wk.y -= w2.y;
                }
                const C wn = w1[idx];
                const C vv = vk[idx];
                const double gv = gfac * ((double)wn.x * vv.x + (double)wn.y * vv.y);
                if (g.diag_per_vec) grad[idx] += gv;
                else gsum += gv;
            }
            w2out[idx] = wk;
        }
        if (!g.diag_per_vec && k < M) grad[site] += gsum;
    }
}

// lambda_n = Pi psi_n for the region of columns > region_col
template <typename R>
__global__ void k_adj_region_seed(AdjGeo g, const void* psi_, void* lam_, int64_t region_col)
{
    using C = typename AV2<R>::C;
    const C* psi = static_cast<const C*>(psi_);
    C* lam = static_cast<C*>(lam_);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.L) return;
    for (int r = blockIdx.y; r < g.W; r += gridDim.y) {
        const int64_t site = (int64_t)r * g.L + c;
        for (int v = 0; v < g.nvec; ++v)
            lam[site * g.nvec + v] = (c > region_col) ? psi[site * g.nvec + v] : AV2<R>::make(0, 0);
    }
}

// Enqueue the whole gradient computation on stream s (capturable: no allocation, no
// synchronisation).  ws holds the trajectory psi_0 .. psi_n, the checkpoints, two rolling
// vectors for the checkpoint pass, the segment, and three adjoint vectors (lambda of the step
// and the two w_k being formed, rotated from step to step instead of copied).
template <typename R>
static int adjoint_enqueue(Plan* p, cudaStream_t s, char* ws, const void* psi0, int nsteps,
                           const void* lambda_n, int64_t region_col, double* g, void* lambda0,
                           double* P)
{
    const size_t vb = p->vec_bytes();
    const DevBlock B = p->hblocks[0];
    const int M = B.M;
    const int S = (int)std::ceil(std::sqrt((double)(M + 1)));
    const int nseg = (M + 1 + S - 1) / S;
    AdjGeo geo{B.W, B.L, p->nvec, p->desc.onsite_per_vec, B.beta, p->d_diag};
    const int th = 256;
    const dim3 grid((unsigned)((B.L + th - 1) / th), (unsigned)std::min(B.W, 65535));
    auto V = [&](size_t i) { return static_cast<void*>(ws + i * vb); };
    const size_t o_traj = 0, o_ck = nsteps + 1, o_roll = o_ck + 2 * nseg, o_seg = o_roll + 2,
                 o_lw = o_seg + S;
    int rc = CHEB_OK;
    // forward trajectory with the fused propagator
    CHEB_CUDA(cudaMemcpyAsync(V(o_traj), psi0, vb, cudaMemcpyDeviceToDevice, s));
    for (int st = 0; st < nsteps; ++st) {
        CHEB_CUDA(cudaMemcpyAsync(V(o_traj + st + 1), V(o_traj + st), vb, cudaMemcpyDeviceToDevice, s));
        rc = plan_enqueue_step(p, V(o_traj + st + 1), s);
        if (rc) return rc;
    }
    // seed lambda_n in adjoint buffer li
    int li = 0;
    void* lam = V(o_lw + li);
    if (lambda_n) {
        CHEB_CUDA(cudaMemcpyAsync(lam, lambda_n, vb, cudaMemcpyDeviceToDevice, s));
    } else {
        k_adj_region_seed<R><<<grid, th, 0, s>>>(geo, V(o_traj + nsteps), lam, region_col);
        p->launches++;
        if (P) {
            rc = launch_observable(p, V(o_traj + nsteps), CHEB_OBS_PROB_COLS, (double)region_col, P, s);
            if (rc) return rc;
        }
    }
    const size_t gbytes = (size_t)p->n_sites * (p->desc.onsite_per_vec ? p->nvec : 1) * sizeof(double);
    CHEB_CUDA(cudaMemsetAsync(g, 0, gbytes, s));
    auto fwd = [&](const void* cur, const void* prev, void* out, int first) {
        k_adj_forward<R><<<grid, th, 0, s>>>(geo, cur, prev, out, first);
        p->launches++;
    };
    // vectors v_k needed by the reverse sweep: k <= M - 1; the checkpoint pass forms v_1 ..
    // v_kc, kc = the second vector of the last segment (or M - 1)
    const int kc = std::min(M - 1, (nseg - 1) * S + 1);
    for (int st = nsteps - 1; st >= 0; --st) {
        // where v_k lives during the checkpoint pass: v_0 is the trajectory's psi_st, the two
        // vectors v_{jS}, v_{jS+1} of every segment have their own slots, the others roll
        auto loc = [&](int k) -> void* {
            if (k == 0) return V(o_traj + st);
            const int j = k / S, m = k % S;
            if (m == 0) return V(o_ck + 2 * j);
            if (m == 1) return V(o_ck + 2 * j + 1);
            return V(o_roll + (k & 1));
        };
        if (kc >= 1) fwd(loc(0), nullptr, loc(1), 1);
        for (int k = 2; k <= kc; ++k) fwd(loc(k - 1), loc(k - 2), loc(k), 0);
        // reverse over segments; segment vector k: the checkpoints for k0, k0 + 1, else the
        // recomputed segment buffer
        void* const wb0 = V(o_lw + (li + 1) % 3);  // w_k of even k
        void* const wb1 = V(o_lw + (li + 2) % 3);  // w_k of odd k
        for (int j = nseg - 1; j >= 0; --j) {
            const int k0 = j * S, k1 = std::min(k0 + S - 1, M);
            auto seg = [&](int k) -> void* { return k - k0 < 2 ? loc(k) : V(o_seg + (k - k0)); };
            for (int k = k0 + 2; k <= std::min(k1, M - 1); ++k) fwd(seg(k - 1), seg(k - 2), seg(k), 0);
            for (int k = k1; k >= k0; --k) {
                void* wk = (k & 1) ? wb1 : wb0;               // w_k overwrites w_{k+2}
                const void* w1 = ((k + 1) & 1) ? wb1 : wb0;  // w_{k+1}
                k_adj_reverse<R><<<grid, th, 0, s>>>(geo, k, M, lam, w1, wk,
                                                     k < M ? seg(k) : nullptr, p->d_qcoef,
                                                     B.coef_off, B.ph_re, B.ph_im, B.a, g);
                p->launches++;
            }
        }
        // lambda_st = w_0: its buffer becomes the next step's lambda
        li = (li + 1) % 3;
        lam = V(o_lw + li);
    }
    if (lambda0) CHEB_CUDA(cudaMemcpyAsync(lambda0, lam, vb, cudaMemcpyDeviceToDevice, s));
    CHEB_CUDA(cudaGetLastError());
    return CHEB_OK;
}

// The gradient call is recorded once as a CUDA graph (about 3 M launches and one copy per
// time step, each too short to hide its own launch overhead) and replayed while the
// pointers, the number of steps and the plan's coefficients stay the same.
template <typename R>
static int adjoint_impl(Plan* p, const void* psi0, int nsteps, const void* lambda_n,
                        int64_t region_col, double* grad, void* lambda0, double* P)
{
    const size_t vb = p->vec_bytes();
    const int M = p->hblocks[0].M;
    const int S = (int)std::ceil(std::sqrt((double)(M + 1)));
    const int nseg = (M + 1 + S - 1) / S;
    const size_t nvecs = (size_t)(nsteps + 1) + 2 * (size_t)nseg + 2 + (size_t)S + 3;
    const size_t gbytes = (size_t)p->n_sites * (p->desc.onsite_per_vec ? p->nvec : 1) * sizeof(double);
    const size_t need = nvecs * vb + (grad ? 0 : gbytes);
    if (p->adj_ws_bytes < need) {
        if (p->adj_graph) {
            cudaGraphExecDestroy(p->adj_graph);
            p->adj_graph = nullptr;
        }
        if (p->adj_ws) cudaFree(p->adj_ws);
        p->adj_ws = nullptr;
        p->adj_ws_bytes = 0;
        if (cudaMalloc(&p->adj_ws, need) != cudaSuccess)
            return fail(CHEB_ERR_NOMEM, "adjoint workspace (trajectory of nsteps + 1 vectors)");
        p->adj_ws_bytes = need;
    }
    char* ws = static_cast<char*>(p->adj_ws);
    double* g = grad ? grad : reinterpret_cast<double*>(ws + nvecs * vb);
    int rc = obs_prepare(p);
    if (rc) return rc;
    Plan::AdjKey key;
    std::memset(&key, 0, sizeof(key));  // padding included, for the memcmp below
    key.psi0 = psi0;
    key.lambda_n = lambda_n;
    key.region_col = region_col;
    key.grad = grad;
    key.lambda0 = lambda0;
    key.P = P;
    key.nsteps = nsteps;
    key.dt = p->dt;
    key.epoch = p->shape_epoch;
    key.ws = p->adj_ws;
    const bool hit = p->adj_graph && std::memcmp(&key, &p->adj_key, sizeof(key)) == 0;
    if (!hit) {
        if (p->adj_graph) {
            cudaGraphExecDestroy(p->adj_graph);
            p->adj_graph = nullptr;
        }
        const bool timing = p->timing;
        p->timing = false;  // no per-launch events inside the graph
        const int64_t before = p->launches;
        cudaGraph_t graph = nullptr;
        CHEB_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = adjoint_enqueue<R>(p, p->cap_stream, ws, psi0, nsteps, lambda_n, region_col, g,
                                lambda0, P);
        cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &graph);
        p->timing = timing;
        p->adj_graph_kernels = (int)(p->launches - before);
        p->launches = before;
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "adjoint: cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&p->adj_graph, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(ce, "adjoint: cudaGraphInstantiate");
        p->adj_key = key;
    }
    CHEB_CUDA(cudaGraphLaunch(p->adj_graph, p->stream));
    p->launches += p->adj_graph_kernels;
    CHEB_CUDA(cudaStreamSynchronize(p->stream));
    return CHEB_OK;
}

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_adjoint_potential(cheb_plan* plan, const void* psi0, double dt, int nsteps,
                                      const void* lambda_n, int64_t region_col, double* grad,
                                      void* lambda0, double* P)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p || !psi0) return fail(CHEB_ERR_INVALID, "cheb_adjoint_potential: NULL argument");
    if (p->op != OP_STENCIL) return fail(CHEB_ERR_UNSUPPORTED, "adjoint needs a lattice plan");
    if (p->nblocks != 1) return fail(CHEB_ERR_UNSUPPORTED, "adjoint needs a single block");
    if (nsteps < 0) return fail(CHEB_ERR_INVALID, "nsteps < 0");
    const void* ptrs[] = {psi0, lambda_n, grad, lambda0, P};
    for (const void* q : ptrs)
        if (q && !aligned16(q)) return fail(CHEB_ERR_ALIGN, "adjoint: pointers must be 16-byte aligned");
    // a zero-step evolve sets dt (and the coefficients) without propagating
    int rc = cheb_evolve(plan, const_cast<void*>(psi0), dt, 0, 0, nullptr);
    if (rc) return rc;
    if (p->prec == CHEB_C128)
        return adjoint_impl<double>(p, psi0, nsteps, lambda_n, region_col, grad, lambda0, P);
    return adjoint_impl<float>(p, psi0, nsteps, lambda_n, region_col, grad, lambda0, P);
}
