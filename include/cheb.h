/*
 * cheb.h -- C ABI of the GB300 Chebyshev time-evolution library.
 *
 * The library propagates complex state vectors with the Chebyshev expansion of the time
 * evolution operator (Fehske et al., "Numerical approaches to time evolution of complex
 * quantum systems", Sec. 2.2):
 *
 *   U(dt) psi = e^{-i b dt} [ c_0 v_0 + 2 sum_{k=1}^{M} c_k v_k ],   c_k = (-i)^k J_k(a dt)
 *   v_0 = psi,  v_1 = H~ v_0,  v_{k+1} = 2 H~ v_k - v_{k-1},         H~ = (H - b)/a
 *
 * with a = (Emax - Emin)(1 + alpha)/2 and b = (Emax + Emin)/2 (Sec. 2.2, text after Eq. U_1),
 * and M the last order whose multiplier |(2 - delta_k0) c_k| reaches the tolerance (text after
 * Eq. dec_Bessel).  Every recurrence step is one fused CUDA kernel: it applies H~ to v_k,
 * forms v_{k+1}, and accumulates its weighted contribution into psi.
 *
 * Conventions for every entry point:
 *   - The return value is a status: CHEB_OK (0) or a negative CHEB_ERR_* code.  Nothing
 *     aborts or throws across this interface; cheb_last_error() gives a message for the
 *     calling thread's most recent failure.
 *   - "device" pointers are CUDA global-memory pointers on the plan's device, owned by the
 *     caller, 16-byte aligned (CHEB_ERR_ALIGN otherwise).  "host" pointers are ordinary
 *     memory, read during the call only.
 *   - State vectors are interleaved complex numbers: double2 (re, im) for CHEB_C128 and
 *     float2 for CHEB_C64.  With nvec vectors the layout is [site][vec]: the nvec values of
 *     one site are contiguous.  Observables and gradients are always double.
 *   - A plan is bound to one CUDA stream (given at creation; NULL = legacy default stream).
 *     All work is enqueued on it asynchronously; calls that return results to host memory
 *     synchronise that stream.  A plan is not thread-safe.
 *   - The plan owns its workspace (two recurrence vectors, coefficients, the scaled
 *     Hamiltonian data) and frees it in cheb_plan_destroy.
 */
#ifndef CHEB_H
#define CHEB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define CHEB_OK 0
#define CHEB_ERR_INVALID (-1)     /* bad argument (sizes, NULL, emin > emax, ...)          */
#define CHEB_ERR_ALIGN (-2)       /* a device pointer is not 16-byte aligned               */
#define CHEB_ERR_CUDA (-3)        /* a CUDA runtime call failed (message in last_error)    */
#define CHEB_ERR_NOMEM (-4)       /* device or host allocation failed                      */
#define CHEB_ERR_UNSUPPORTED (-5) /* operation not available for this operator kind        */
#define CHEB_ERR_ORDER (-6)       /* |c_k| did not fall below tol within max_order         */
#define CHEB_ERR_DIVERGED (-7)    /* recurrence grew: the spectral bounds do not enclose H */
#define CHEB_ERR_STATE (-8)       /* call out of order (e.g. no time step set)             */

/* ---- arithmetic of the state vectors ------------------------------------------------ */
typedef enum { CHEB_C128 = 0, CHEB_C64 = 1 } cheb_prec;

/* ---- operator kinds ----------------------------------------------------------------- */
typedef enum {
    /* 1D grid, Sec. 3.1: H = -(1/2) d^2/dx^2 + V(x) with the 3-point stencil (hbar = m = 1),
       psi = 0 outside the n grid points.  onsite = V_i. */
    CHEB_LAT1D = 0,
    /* Zigzag honeycomb ribbons, Sec. 3.2, Eq. (model): H = -t sum_<ij>(c_i^+ c_j + h.c.)
       + sum_j eps_j n_j.  Brick-wall indexing: site (r, c), r in [0, W) across, c in [0, L)
       along, index r*L + c; neighbours (r, c-1), (r, c+1) and (r+1, c) if r + c is even,
       (r-1, c) if odd; open at every border.  nblocks ribbons are stored one after another
       (ribbon q starts at site sum_{p<q} W_p L_p); each has its own a, b, c_k and M.
       onsite = eps_j.  The columns c = 0 and c = L-1 are armchair edges, so a ribbon with
       armchair edges along its length (Table 2: N_a dimer lines across) is the same operator
       with W = its length and L = N_a. */
    CHEB_HONEYCOMB_ZZ = 1,
    /* Holstein chain, Sec. 3.3, Eq. (ghm), one spinless electron:
       H = sum_i Delta_i n_i - t sum_i (c_i^+ c_{i+1} + h.c.) - sum_i g_i w0 (b_i^+ + b_i) n_i
       + w0 sum_i b_i^+ b_i, in the basis |e; n_0..n_{L-1}> with sum_i n_i <= nph (Sec. 3.3);
       Delta_i from onsite (device [L], NULL: 0), g_i from hol_g (NULL: g).
       Basis index = e * Dph + rank(n), Dph = C(nph + L, L), rank = position of n in the
       lexicographic order of all admissible tuples (n_0 most significant) -- see
       cheb_holstein_rank.  Stored as a SELL-C-sigma matrix built on the device, or, with
       hol_matrix_free = 1, applied without a stored matrix (Sec. 3.3). */
    CHEB_HOLSTEIN = 2
} cheb_kind;

typedef struct cheb_ham_desc {
    int32_t kind;            /* cheb_kind */
    /* CHEB_LAT1D */
    int64_t n;               /* grid points                                                */
    double dx;               /* grid spacing                                               */
    /* CHEB_HONEYCOMB_ZZ */
    int32_t nblocks;         /* ribbons (>= 1); also 1 for the other kinds                */
    const int32_t* W;        /* host [nblocks]: rows (zigzag chains) of each ribbon       */
    const int32_t* L;        /* host [nblocks]: columns of each ribbon                     */
    double hop;              /* transfer integral t (all kinds)                            */
    /* CHEB_LAT1D and CHEB_HONEYCOMB_ZZ: device, on-site energies (double).  Layout [site]
       when onsite_per_vec == 0 (shared by all nvec vectors), [site][vec] when 1 (one
       potential per vector, e.g. independent disorder realisations).  May be NULL (zero).
       Read once at plan creation (and by cheb_plan_set_onsite). */
    const double* onsite;
    int32_t onsite_per_vec;
    /* CHEB_HOLSTEIN */
    int32_t hol_sites;       /* L                                                          */
    int32_t hol_nph;         /* phonon cap                                                 */
    int32_t hol_periodic;    /* 1: bond (L-1, 0) present (needs L >= 3)                   */
    double omega0;           /* phonon frequency w0                                        */
    double g;                /* dimensionless coupling g                                   */
    int32_t sell_sigma;      /* CHEB_HOLSTEIN stored matrix: SELL-C-sigma window (C = 32):
                                rows sorted by decreasing length inside windows of sigma
                                rows (a multiple of 32, <= 2^20), so chunks pad little;
                                1 = no sorting; 0 = CHEB_SELL_SIGMA_DEFAULT_C128 / _C64   */
    /* CHEB_HOLSTEIN, optional: device [L] site couplings g_i (Eq. ghm,
       g_i = ((eps_p + eps_p,i)/w0)^{1/2}); NULL: g at every site.  With onsite = device [L]
       site potentials Delta_i (NULL: 0) this is the generalised model of Sec. 3.3. */
    const double* hol_g;
    /* CHEB_HOLSTEIN: 1 = matrix-free operator.  Sec. 3.3 recomputes the matrix elements in
       every multiplication so that its largest basis fits in memory; here each launch
       recomputes them from the basis indices (phonon ranks of n +- 1_e, see
       cheb_holstein_phonon_neighbors) and stores neither the matrix nor the diagonal.  Needs
       L <= 32 and nph <= 15 (CHEB_ERR_UNSUPPORTED otherwise); same basis, layout and results
       as the stored matrix.  0 = SELL-C matrix.  The CSR export needs the stored matrix. */
    int32_t hol_matrix_free;
} cheb_ham_desc;

/* sell_sigma = 0 selects these windows: complex128 plans are bound by the FP64 rate and gain
   from storing fewer padded entries (6.66 -> 6.41 ms per step at L = 12, nph <= 10, padding
   25.4 % -> 0.12 %); complex64 plans are bound by gather latency, and the row indirection
   sorting adds costs more than the padding it saves (3.86 -> 4.25 ms), so they keep the rows
   in basis order (1) */
#define CHEB_SELL_SIGMA_DEFAULT_C128 8192
#define CHEB_SELL_SIGMA_DEFAULT_C64 1

typedef struct cheb_plan cheb_plan;

/* ---- error text -------------------------------------------------------------------- */
/* Message of the calling thread's most recent failing call (static storage; never NULL). */
const char* cheb_last_error(void);
/* Fixed text of a status code. */
const char* cheb_strerror(int status);

/* ---- Sec. 2.2: rescaling and expansion coefficients (host, FP64) ---------------------- */
/* b = (emax + emin)/2, a = (emax - emin)(1 + alpha)/2 (Sec. 2.2, text after Eq. U_1). */
int cheb_rescale(double emin, double emax, double alpha, double* a, double* b);

/* Multipliers C_k = e^{-i b dt} (2 - delta_k0) (-i)^k J_k(a dt), k = 0..M, of Eq. (U_1)
   with Eq. (c_k); J_k by Miller's backward recurrence normalised with
   J_0 + 2 sum_k J_2k = 1.  M = largest k with |C_k| >= tol; M >= 2 always (an M of 1 is
   raised to 2).  c_re, c_im: host arrays of max_order + 1 doubles (caller-owned), filled
   for k = 0..M.  Returns CHEB_ERR_ORDER if |C_k| >= tol still holds at k = max_order. */
int cheb_coeffs(double a, double b, double dt, double tol, int max_order, double* c_re,
                double* c_im, int* M_out);

/* ---- plans ------------------------------------------------------------------------- */
/* Build a plan for nvec state vectors of the operator h, in precision prec (cheb_prec).
   emin, emax: host arrays [h->nblocks] of spectral bounds (one pair per ribbon; one pair
   for the other kinds); alpha: the safety margin of Sec. 2.2 (the paper uses 0.01).
   The plan scales the on-site data to d_i = 2 (H_ii - b)/a once, stores it in prec's real
   type, and allocates two recurrence vectors.  stream: a cudaStream_t or NULL.
   Holstein plans build the basis and the SELL matrix on the device. */
int cheb_plan_create(cheb_plan** out, const cheb_ham_desc* h, const double* emin,
                     const double* emax, double alpha, int prec, int nvec, void* stream);
void cheb_plan_destroy(cheb_plan* plan);

/* Tolerance and order cap used by the next cheb_step/cheb_evolve (defaults 1e-14, 100000). */
int cheb_plan_set_tol(cheb_plan* plan, double tol, int max_order);
/* Replace the on-site energies (device pointer, same layout as in the descriptor). */
int cheb_plan_set_onsite(cheb_plan* plan, const double* onsite);
/* Scalars of the plan: sites per vector (total over ribbons), number of vectors, blocks,
   and the a, b, M of block q (M for the last dt used, 0 before the first step).  Complex64
   lattice plans (CHEB_LAT1D, CHEB_HONEYCOMB_ZZ) enlarge the a of cheb_rescale by less than
   one part in 2^23 so that the scaled hopping 2 h / a is a float32 number. */
int cheb_plan_info(const cheb_plan* plan, int64_t* sites, int* nvec, int* nblocks);
int cheb_plan_block(const cheb_plan* plan, int q, double* a, double* b, int* M,
                    int64_t* offset, int* W, int* L);

/* ---- propagation ------------------------------------------------------------------- */
/* psi <- U(dt) psi for all nvec vectors (device, in place, [site][vec]).  Enqueues M fused
   recurrence kernels (M of the largest block) on the plan's stream and returns; the
   coefficients are recomputed on the host only when dt changes (Sec. 2.2: once per dt). */
int cheb_step(cheb_plan* plan, void* psi, double dt);

/* nsteps calls of cheb_step, replayed from one CUDA graph.  If obs_every > 0 and obs is not
   NULL, before every obs_every-th step s (s = 0, obs_every, ...) the plan records
   [||psi||^2, <psi|H|psi>] per (block, vec) into the device array obs (double, layout
   [record][block][vec][2], records = ceil(nsteps / obs_every)).  Both are FP64 reductions
   (FP64 products and sums): complex128 plans take them from the first recurrence kernel of
   that step (v_1 = H~ psi, no extra matvec); complex64 plans run one extra FP64 pass over
   psi before a recorded step (their first recurrence kernel sums its per-thread terms in
   FP32, which serve only the growth check below), so unrecorded steps cost nothing extra.
   Synchronises the stream and returns CHEB_ERR_DIVERGED if a recurrence vector exceeded
   the bound |v_k| <= ||psi|| that holds when the spectrum lies inside [emin, emax]. */
int cheb_evolve(cheb_plan* plan, void* psi, double dt, int nsteps, int obs_every,
                double* obs);

/* A batch of independent jobs from host memory: job j's state (n_sites x nvec complex values
   of the plan's precision, layout [site][vec]; vec_bytes = n_sites * nvec * 16 (complex128)
   or 8 (complex64) bytes) at (const char*)in + j * in_stride is copied to the device,
   propagated nsteps steps of dt and copied back to (char*)out + j * out_stride.  Strides are
   in bytes, 0 (every job reads / writes the same state) or >= vec_bytes.  The host-to-device
   copy of job j + 1 and the device-to-host copy of job j - 1 overlap the propagation of job j
   and each other (three device buffers of the plan; one stream per copy direction); the
   copies overlap only
   with pinned host memory (cudaHostAlloc / cudaHostRegister).  in and out may be the same
   buffer only with equal nonzero strides (CHEB_ERR_INVALID otherwise); other overlaps are the
   caller's error.  Host buffers are owned by the caller and must hold every addressed state.
   Synchronises before returning; CHEB_ERR_DIVERGED as cheb_evolve.  No counterpart in the
   paper (many initial states served from host memory). */
int cheb_evolve_host(cheb_plan* plan, const void* in, int64_t in_stride, void* out,
                     int64_t out_stride, int64_t njobs, double dt, int nsteps);

/* Time-dependent Hamiltonian (Sec. 2.2: the time variation of H(t) limits the step): nsteps
   steps of dt with H held constant over each step, step s using the on-site energies at
   onsite_seq + s * stride (device, double, in the layout of the descriptor's onsite array;
   stride in doubles, even, >= the array length).  Sampling V(t) at the step midpoints
   t_s + dt/2 makes the scheme second order in dt.  The rescaling a, b stays the one of the
   plan, so its bounds must enclose the spectrum of every H(t_s) (CHEB_ERR_DIVERGED
   otherwise).  obs_every / obs as cheb_evolve.  Afterwards the plan keeps the last step's
   on-site energies.  Lattice kinds only (CHEB_ERR_UNSUPPORTED for Holstein plans).
   Synchronises the plan's stream. */
int cheb_evolve_td(cheb_plan* plan, void* psi, double dt, int nsteps, const double* onsite_seq,
                   int64_t stride, int obs_every, double* obs);

/* Status of the work enqueued so far: synchronises the stream, returns CHEB_ERR_DIVERGED
   if the growth check fired since the last call (and clears it), CHEB_ERR_CUDA on an
   asynchronous CUDA error, else CHEB_OK. */
int cheb_sync(cheb_plan* plan);

/* ---- observables (device outputs, double) ------------------------------------------ */
typedef enum {
    CHEB_OBS_NORM2 = 0,     /* ||psi||^2 per (block, vec)                       [nblocks][nvec] */
    CHEB_OBS_ENERGY = 1,    /* <psi|H|psi> per (block, vec)                     [nblocks][nvec] */
    CHEB_OBS_PROB_COLS = 2, /* ribbons: sum_{c > param} |psi|^2 per (block,vec) [nblocks][nvec];
                               1D grid: sum over sites i > param                                 */
    CHEB_OBS_HOL_DENSITY = 3, /* Holstein <n_i>, Sec. 3.3 (Fig. 3)                  [L][nvec] */
    CHEB_OBS_HOL_PHONON = 4,  /* Holstein <b_i^+ b_i>                               [L][nvec] */
    CHEB_OBS_HOL_CHI = 5      /* Holstein chi_ii = <n_i (b_i + b_i^+)>              [L][nvec] */
} cheb_obs_kind;

/* Deterministic FP64 reductions of psi (device, plan layout) into out (device doubles). */
int cheb_observables(cheb_plan* plan, const void* psi, int kind, double param, double* out);

/* ---- plan-free region norm that allocates no device memory -------------------------- */
/* The paper has no counterpart: this serves callers that may not allocate device memory
   where they need a norm -- latency-critical loops that cannot take the device-wide
   synchronisation of cudaMalloc/cudaFree, and host programs whose own pool owns all device
   memory.  For one zigzag ribbon (or the 1D grid, L = n) held as psi (device, [site][vec],
   complex128 or complex64 by prec, n_sites = W * L), out[v] (device, nvec doubles) =
   sum over sites with column (site % L) > col_min of |psi_v|^2; col_min = -1 gives ||psi_v||^2.
   Same per-tile FP64 reduction as cheb_observables; its tile partials live in a static
   device array of CHEB_NOALLOC_MAX_PARTIALS doubles (512 KiB, held by every GPU that loads
   the library until exit), so ceil(n_sites / 1024) * nvec must not exceed that
   (CHEB_ERR_INVALID otherwise).  The array's device address is looked up on the first call
   made on each device, so make that first call before any stream capture.  Calls share the
   array: calls whose kernels may overlap on the GPU race.  Enqueued on stream (NULL =
   legacy default stream); no allocation of any kind. */
#define CHEB_NOALLOC_MAX_PARTIALS 65536
int cheb_region_norm_noalloc(const void* psi, int prec, int64_t n_sites, int32_t L, int nvec,
                             int64_t col_min, double* out, void* stream);

/* ---- gradient with respect to the on-site potential ---------------------------------- */
/* No counterpart in the paper: reverse-mode differentiation of Eqs. (U_1) and (rec) with
   a, b held fixed (dH~/dV_i = e_i e_i^T / a).  psi_n = U(dt)^nsteps psi0 is recomputed from
   psi0; the forward vectors of each step are regenerated from ceil(sqrt(M)) checkpoints.
   Objective: P = sum_{sites with column > region_col} |psi_n|^2 per vector (ribbons; for
   the 1D grid: index > region_col) when lambda_n is NULL; otherwise the caller supplies
   lambda_n = dP/d(conj psi_n) (device, plan layout) for an arbitrary real P.
   Outputs (device, caller-owned, may be NULL when not wanted):
     grad   : dP/dV_i, doubles, layout of the plan's onsite array ([site] summed over vecs
              when onsite_per_vec == 0, [site][vec] when 1);
     lambda0: dP/d(conj psi0), plan layout and precision;
     P      : doubles [nvec] (only with the region objective).
   The plan keeps the workspace (nsteps + 1 trajectory vectors plus about 3 sqrt(M) more)
   and records the whole computation as a CUDA graph that later calls with the same
   pointers, nsteps and dt replay.  Synchronises the plan's stream before returning.
   CHEB_ERR_UNSUPPORTED for Holstein plans and for plans with several ribbons. */
int cheb_adjoint_potential(cheb_plan* plan, const void* psi0, double dt, int nsteps,
                           const void* lambda_n, int64_t region_col, double* grad,
                           void* lambda0, double* P);

/* ---- Holstein basis (Sec. 3.3), host ------------------------------------------------ */
/* Number of phonon tuples with L sites and sum <= nph: C(nph + L, L). */
int64_t cheb_holstein_dim_phonon(int L, int nph);
/* rank of occ[0..L-1] (uint8) in the lexicographic order of admissible tuples, combined
   with the electron site e into idx = e * Dph + rank.  CHEB_ERR_INVALID if sum(occ) > nph. */
int cheb_holstein_rank(int L, int nph, const uint8_t* occ, int e, int64_t* idx);
/* Inverse of cheb_holstein_rank. */
int cheb_holstein_unrank(int L, int nph, int64_t idx, uint8_t* occ, int* e);
/* Phonon neighbours used by the matrix-free operator (Sec. 3.3): for the phonon
   configurations n of ranks p0 .. p0 + count - 1 (host arrays [count][L], row i for rank
   p0 + i) up[i][e] = rank(n + 1_e), or -1 when sum n = nph, and dn[i][e] = rank(n - 1_e), or
   -1 when n_e = 0.  Ranks are phonon ranks (the basis index minus e * Dph).  Computed on the
   host by the same routine the kernels run.  Needs 1 <= L <= 32, 0 <= nph <= 15,
   Dph < 2^31 and 0 <= p0, p0 + count <= Dph; CHEB_ERR_INVALID otherwise. */
int cheb_holstein_phonon_neighbors(int L, int nph, int64_t p0, int64_t count, int64_t* up,
                                   int64_t* dn);

/* ---- tuning --------------------------------------------------------------------------- */
/* Times the plan's recurrence over launch shapes on the plan's own workspace and keeps the
   fastest; the choice is kept in the plan.  Three passes: single-order launch shapes
   (threads per block, sites per thread, vectors per thread, grid size; the matrix-free
   Holstein variants), one launch timed as a captured graph of 16 when it is short, and the
   shapes of short steps (best launch x M < 2 ms) ranked again by whole steps; then temporal
   blocking (complex64 lattice plans) and cluster steps (small 1D grids) against single-order
   launches, by whole steps replayed from the step's CUDA graph.  Allocates one scratch
   vector for the duration of the call.  Needs a time step set (CHEB_ERR_STATE otherwise).
   Optional: plans start from a fixed default. */
int cheb_autotune(cheb_plan* plan);
/* Temporal blocking (complex64 lattice plans with nvec 1, 2 or 4 and a shared on-site
   array): orders_per_launch s > 0 makes each launch run s recurrence orders out of shared
   memory on 2-D tiles of each ribbon with a halo of s columns and ceil(s / 2) rows (a site d
   rows away is at least 2d - 1 bonds away on the brick wall); a CTA of `threads` threads
   holds a region of threads x sites_per_thread sites.  Compiled shapes (nvec: sites_per_thread x
   threads): 256 threads with 4, 6 or 8 (8 only for nvec <= 2); nvec 4 also 3, 4, 6 x 512 and
   2, 3 x 1024; nvec 2 also 6 x 1024; nvec 1 also 8 x 1024.  threads = 0 means 256.  s = 0
   returns to one order per launch.  CHEB_ERR_UNSUPPORTED for other plans, CHEB_ERR_INVALID
   for a shape that is not compiled.  cheb_autotune also chooses these. */
int cheb_plan_set_blocking(cheb_plan* plan, int orders_per_launch, int sites_per_thread,
                           int threads);
/* The blocked kernel, chosen with the shape:
     CHEB_TB_SITES  the kernel of cheb_plan_set_blocking: a thread's sites are `threads` apart
                    in the region, all recurrence vectors of the region in shared memory;
     CHEB_TB_RUNS   each thread owns a run of sites_per_thread consecutive sites (odd) whose
                    T_{k-1} and T_{k-2} stay in its registers; an order reads only the vertical
                    neighbours and the run-end neighbours from shared memory and stores T_k
                    once.  Region rows are padded to a multiple of 4 (pairs of vectors) or 8
                    (one vector) positions with at least one zero pad.  A CTA holds one pair of
                    vectors (nvec 2 and 4: the two pairs of a tile go to two CTAs) or one vector
                    (nvec 1).  The launch keeps its CTAs resident (one per SM), each working
                    through tiles, and copies its next tile's inputs into shared memory
                    while the current one runs.  Compiled (run x threads): pairs 3 x 768, 3 x 512,
                    5 x 512, 7 x 384, 9 x 256; single vectors 3 x 1024, 5 x 512, 7 x 512;
     CHEB_TB_RUNS_TMA  CHEB_TB_RUNS with the next tile's T_{k-1} and T_{k-2} staged by
                    tensor-memory-access boxes (one box per vector pair and buffer, completion
                    on an mbarrier) in place of per-thread copies; pairs of vectors only (nvec
                    2 and 4, CHEB_ERR_UNSUPPORTED otherwise).  All tiles of a ribbon share one
                    padded row stride S (its widest tile's) so that the box of S x (its
                    tallest region) lands as the plane layout; ribbons whose box exceeds
                    256 x 256, or a driver without the tensor-map encoder, fall back to the
                    per-thread copies.  Same compiled shapes as the pairs above.
   cheb_plan_set_blocking_kernel(plan, s, spt, threads, CHEB_TB_SITES) equals
   cheb_plan_set_blocking; errors as there.  cheb_plan_blocking_kernel reports the kernel of
   the blocking in use (CHEB_TB_SITES when blocking is off). */
typedef enum { CHEB_TB_SITES = 0, CHEB_TB_RUNS = 1, CHEB_TB_RUNS_TMA = 2 } cheb_tb_kernel;
int cheb_plan_set_blocking_kernel(cheb_plan* plan, int orders_per_launch, int sites_per_thread,
                                  int threads, int kernel);
int cheb_plan_blocking_kernel(const cheb_plan* plan, int* kernel);
/* CTAs of each blocked launch: at most `ctas`, every CTA working through the tiles (and vector
   pairs) i, i + ctas, ...; 0 (the default) means the strided-site kernel's one CTA per tile
   and the register-run kernel's resident CTAs (SMs x CTAs per SM), whose CTAs copy their next
   tile's inputs while the current one runs its orders.  Results do not depend on it.
   CHEB_ERR_INVALID for ctas < 0. */
int cheb_plan_set_blocking_grid(cheb_plan* plan, int ctas);

/* Whole steps on a thread-block cluster (1D grid plans, CHEB_LAT1D with nvec 1, a shared
   potential and at most 32768 points): ctas = 8 or 16 runs all M orders of a step in one
   launch of a cluster of that many CTAs that keep the recurrence vectors in shared memory and
   exchange the chunk borders through distributed shared memory, with one cluster barrier per
   order (the grid's single-order launches are latency-bound: M = 6353 at N = 2048,
   dt = 0.5); ctas = 0 returns to single-order launches.  CHEB_ERR_UNSUPPORTED for other plans
   or a cluster the device cannot schedule (16 CTAs is a non-portable size),
   CHEB_ERR_INVALID for other values.  cheb_plan_cluster reports the size in use (0: off).
   cheb_autotune also decides this. */
int cheb_plan_set_cluster(cheb_plan* plan, int ctas);
int cheb_plan_cluster(const cheb_plan* plan, int* ctas);

/* Launch shape chosen for the plan: threads per block, sites per thread, grid size, and
   vectors handled per thread (of the nvec at each site).  Matrix-free Holstein plans report
   phonon configurations per tile / threads as sites_per_thread and the configurations a
   thread advances together (1 or 2) in place of vectors per thread. */
int cheb_plan_launch(const cheb_plan* plan, int* threads, int* sites_per_thread, int* grid,
                     int* vecs_per_thread);
/* Orders per launch, sites per thread and threads per CTA of the temporal blocking in use
   (0, 0, 0: off). */
int cheb_plan_blocking(const cheb_plan* plan, int* orders_per_launch, int* sites_per_thread,
                       int* threads);

/* ---- introspection for tests ---------------------------------------------------------- */
/* The tiles temporal blocking uses for one W x L brick-wall ribbon with orders_per_launch
   orders per launch and region_sites sites per CTA (threads x sites_per_thread): per tile 8
   int32 (R0, R1, C0, C1, r0, r1, c0, c1), the region [R0, R1) x [C0, C1) and its interior
   [r0, r1) x [c0, c1) in ribbon rows and columns.  The halo is orders_per_launch columns and
   ceil(orders_per_launch / 2) rows on every side that is not a ribbon edge (Sec. 3.2
   lattice; the bound on the rows follows from the alternating vertical bonds).  *ntiles gets
   the count; up to `capacity` tiles are written to the caller's out (capacity 0: count only).
   Host-only, no device memory; CHEB_ERR_INVALID for bad arguments or a ribbon whose single
   interior column would not fit. */
int cheb_tb_tiles(int W, int L, int orders_per_launch, int region_sites, int32_t* out,
                  int64_t capacity, int64_t* ntiles);
/* The same for the register-run kernel's padded regions: region_positions = threads x run;
   10 int32 per tile: the 8 above, then the row stride S (the smallest multiple of align >=
   C1 - C0 + 1; align = 4 for pairs of vectors, 8 for one) and the box height BH.  With
   boxes = 0 (CHEB_TB_RUNS) S is the tile's own and BH = R1 - R0; with boxes = 1
   (CHEB_TB_RUNS_TMA) every tile of the ribbon takes the stride of its widest tile and BH =
   the most region rows of its tiles.  In both, 1 + BH x S <= region_positions. */
int cheb_tb_tiles_padded(int W, int L, int orders_per_launch, int region_positions, int align,
                         int boxes, int32_t* out, int64_t capacity, int64_t* ntiles);
/* Copies of the plan's device data to host memory, for checking the construction:
   the SELL matrix of a Holstein plan as CSR in original row order (rowptr [n+1] int64,
   col [nnz] int64, val [nnz] double with the unscaled H entries); nnz_out gets the count.
   Pass col = val = NULL to query nnz only.  Plans with more than 2^27 rows keep no
   unscaled copy of the matrix (CHEB_ERR_UNSUPPORTED). */
int cheb_plan_export_csr(cheb_plan* plan, int64_t* rowptr, int64_t* col, double* val,
                         int64_t* nnz_out);
/* Number of kernel launches the plan has enqueued since creation (graph replays count
   every kernel node). */
int64_t cheb_plan_launches(const cheb_plan* plan);

/* ---- kernel timing ------------------------------------------------------------------- */
/* enable != 0: cheb_step/cheb_evolve launch the recurrence kernels directly (no graph) and
   bracket each launch with a pair of CUDA events on the plan's stream; every launch also
   records its algorithmic DRAM bytes (each vector element read or written once, the on-site
   and SELL data read once).  cheb_plan_kernel_stats sums, over the launches since the last
   reset, the event times (ms), the launch count and the algorithmic bytes; it synchronises
   the stream.  reset != 0 clears the sums afterwards. */
int cheb_plan_set_timing(cheb_plan* plan, int enable);
int cheb_plan_kernel_stats(cheb_plan* plan, double* ms, int64_t* launches, double* bytes,
                           int reset);

/* SELL matrix of a Holstein plan: the sigma in use, the entries stored per chunk column
   (with padding) and the off-diagonal entries of the matrix (without padding).
   CHEB_ERR_UNSUPPORTED for plans without a stored matrix. */
int cheb_plan_sell_stats(const cheb_plan* plan, int* sigma, int64_t* stored, int64_t* offdiag);

/* ---- work model and peak probes (measurement; no counterpart in the paper) ----------- */
/* What one step of the plan's current launch schedule does, counted on the host from the
   launch shapes and tiles (no device work):
     useful_site_orders    sites x Chebyshev orders the step must form (a site carries all
                           nvec vectors), summed over blocks: sum_q W_q L_q M_q;
     computed_site_orders  the ones the kernels actually form: with temporal blocking the
                           halo sites of a tile are formed too, for as many orders as they
                           stay valid (equal to useful_site_orders for single-order launches);
     smem_bytes            shared-memory bytes the blocked kernel loads and stores (region
                           copies in, neighbour and own-site reads and the new values of every
                           order, interior read-back); 0 for single-order launches;
     dram_bytes            DRAM bytes if every operand crosses DRAM once per launch (halo
                           re-reads of a blocked launch served by L2);
     l2_bytes              bytes the launches move between L2 and the SMs (blocked: every
                           region's inputs including the halos; single-order: dram_bytes);
     launches              recurrence kernel launches per step.
   Needs a dt (after the first cheb_step / cheb_evolve).  Cluster steps report useful =
   computed and psi in and out as their traffic. */
typedef struct {
    double useful_site_orders;
    double computed_site_orders;
    double smem_bytes;
    double dram_bytes;
    double l2_bytes;
    int64_t launches;
} cheb_step_model;
int cheb_plan_step_model(const cheb_plan* plan, cheb_step_model* out);

/* Peak rates measured on the current device by the library's own micro-kernels, for
   rooflines that have no external reference figure: the shared-memory load bandwidth of all
   SMs (16-byte loads without bank conflicts, GB/s), and the FP64 and FP32 fused
   multiply-add rates (GFLOP/s, 2 flops per FMA).  Each probe runs on every SM, timed with
   CUDA events on stream (NULL = legacy default stream) after a warm-up launch, best of three;
   it allocates 64 bytes of device memory and synchronises.  CHEB_ERR_INVALID for an unknown
   kind. */
typedef enum {
    CHEB_PEAK_SMEM_LOAD_GBS = 0,
    CHEB_PEAK_FP64_GFLOPS = 1,
    CHEB_PEAK_FP32_GFLOPS = 2
} cheb_peak_kind;
int cheb_measure_peak(int kind, void* stream, double* value);

#ifdef __cplusplus
}
#endif
#endif /* CHEB_H */
