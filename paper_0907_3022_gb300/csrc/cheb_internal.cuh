// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cheb.h"

namespace cheb {

// ---- status plumbing -------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define CHEB_CUDA(call)                                        \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return ::cheb::cuda_fail(e_, #call); \
    } while (0)

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---- complex types ---------------------------------------------------------------------
template <typename R> struct CT;
template <> struct CT<double> { using type = double2; };
template <> struct CT<float> { using type = float2; };

// ---- operator geometry -------------------------------------------------------------------
enum OpKind : int { OP_STENCIL = 0, OP_SELL = 1, OP_HOLMF = 2 };

// One independent Hamiltonian block: a ribbon (W x L brick wall), the 1D grid (W = 1), or
// the whole Holstein matrix.  Device copy of the per-block scalars used by the kernels.
struct DevBlock {
    int64_t offset;   // first site of the block in the vector
    int32_t W, L;     // brick-wall rows/columns (1D grid: W = 1, L = n)
    int32_t M;        // truncation order for the current dt (>= 2)
    int32_t coef_off; // index of q_0 of this block in the coefficient table
    int32_t ksplit;   // orders k > ksplit accumulate into the tail vector (complex64 only)
    int32_t pad0;
    double beta;      // scaled off-diagonal 2 * h_offdiag / a (stencil kinds)
    double a, b;      // rescaling of Sec. 2.2
    double ph_re, ph_im; // e^{-i b dt}
};

// A tile of consecutive sites inside one block (work items never straddle blocks).
struct WorkItem {
    int32_t block;
    int32_t pad;
    int64_t first;  // first site, relative to the block
    int64_t count;  // sites in the tile
};

// Accumulation of psi in groups of orders (Eq. U_1).  The launch forming T_k adds to the
// accumulator only when k = 2 (mod 3) or k = M, and then adds every order formed since the
// previous such launch: T_{k-2}, T_{k-1}, T_k (the three recurrence vectors it holds), or
// the last one or two orders at k = M.  The terms are added in increasing order, so the sum
// is the same as adding each order when it is formed, for a third of the accumulator
// traffic.  complex64 plans keep the orders above ksplit (a value = 2 mod 3, or M) in the
// tail accumulator, so a group never straddles ksplit.
struct AccGroup {
    bool upd;            // this launch updates an accumulator
    bool last;           // k = M: psi receives its final value
    bool to_tail;        // the group goes to the tail accumulator
    bool read_acc;       // the accumulator already holds earlier groups
    bool read_psi_last;  // last group of a tail: psi + (tail + group)
    int n;               // orders in the group (1, 2 or 3)
    __host__ __device__ AccGroup(int k, int M, int ksplit) {
        last = (k == M);
        upd = (k >= 2) && (k % 3 == 2 || last);
        const int uprev = 3 * (k / 3) - 1;  // previous updating launch (-1: none)
        n = upd ? k - uprev : 0;
        to_tail = upd && uprev >= ksplit;
        read_acc = upd && (to_tail ? uprev >= ksplit + 3 : uprev >= 2);
        read_psi_last = last && to_tail;
    }
};

// Recurrence launch arguments (one launch = one order j, producing T_{j+1}).
enum RecMode : int { REC_FIRST = 0, REC_SECOND = 1, REC_GENERAL = 2 };

struct RecArgs {
    const WorkItem* items;
    int32_t nitems;
    int32_t nvec;
    const DevBlock* blocks;
    const void* diag;       // d_i = 2 (H_ii - b)/a in R; [site] or [site][vec]
    int32_t diag_per_vec;
    int32_t mode;
    int32_t j;              // this launch forms T_{j+1}
    const void* cur;        // T_j  (FIRST: psi)
    void* prev;             // T_{j-1} in, T_{j+1} out (FIRST: receives T_0)
    void* out1;             // FIRST only: receives T_1
    void* psi;              // accumulator (SECOND: written; GENERAL: read-modify-write)
    void* tail;             // accumulator of the small high orders (complex64 plans)
    const void* qcoef;      // R table: q_k = sign_k (2 - delta_k0) J_k(a dt), per block
    // SELL data (OP_SELL)
    const int32_t* sell_col;
    const void* sell_val;   // R, already multiplied by 2/a
    const int64_t* sell_chunk_off;
    const int32_t* sell_chunk_len;
    const int32_t* sell_perm;  // SELL-C-sigma: row of each storage position (NULL: identity)
    // reductions (FIRST): per work item [nvec][2] partial (norm2, <x|2H~x>/2)
    double* partials;
    unsigned int* done_counter;
    double* red_out;        // [nblocks][nvec][2]: norm2, <psi|H|psi>
    int32_t nblocks;
    const int32_t* block_item_begin; // [nblocks + 1]: items of block q are [begin_q, begin_{q+1})
    // growth check (last order of a block): |T_M,i|^2 <= 4 ||psi||^2 + tiny
    const double* norm2;    // [nblocks][nvec], from the FIRST launch of this step
    int* errflag;
};

// Temporal blocking (cheb_tb.cu): a tile of one ribbon with its halo region.
struct TBTile {
    int32_t block;
    int32_t R0, R1, C0, C1;  // region (ribbon rows/columns, half-open)
    int32_t r0, r1, c0, c1;  // interior
    // register-run kernel: the row stride of the ribbon's regions in shared memory (the same
    // for every tile of the ribbon), the most region rows of its tiles, and whether the
    // ribbon's inputs are copied by tensor-memory-access boxes of S x BH (1) or per thread (0)
    int32_t S, BH, tma;
};

struct TBArgs {
    const TBTile* tiles;
    int32_t ntiles;
    int32_t ka, kb;          // orders formed by this launch
    int32_t prev_ka;         // first order of the previous launch of the step (0: none)
    const DevBlock* blocks;
    int32_t nvec;            // vectors per site
    const void* diag;        // float d_i
    const void* in_prev;     // T_{ka-2} (unused when ka = 1)
    const void* in_cur;      // T_{ka-1} (psi when ka = 1)
    void* out_prev;          // T_{ke-1}
    void* out_cur;           // T_{ke}
    void* acc_main;          // E
    void* tail;
    void* psi;
    const void* qcoef;       // float2 (hi, lo) per order
    double* partials;        // first launch: [tile][nvec][2]
    unsigned int* done_counter;
    double* red_out;
    int32_t nblocks;
    const int32_t* block_tile_begin;
    const double* norm2;
    int* errflag;
    // register-run kernel: tensor maps [block * pairs + pair] of T_{ka-1} and T_{ka-2} for
    // the ribbons whose tiles are copied by boxes (NULL: per-thread copies)
    const void* tm_cur;
    const void* tm_prev;
    // register-run kernel: sites of the plan; its step-internal vectors (T pairs, E, tail) are
    // stored pair-planar, element (site, pair) at pair * nsites + site (psi keeps
    // [site][vector])
    int64_t nsites;
};

struct TBSet {
    int s = 0;
    TBTile* d_tiles = nullptr;
    int32_t* d_begin = nullptr;
    int ntiles = 0;
    std::vector<TBTile> first;  // host: the first tile of every ribbon (stride, box, tma flag)
};

struct Plan;

// temporal blocking (cheb_tb.cu)
size_t tb_smem_bytes(int nv, int spt, int tpb);
bool tb_supported(int nv, int spt, int tpb);
int tb_launch(Plan* p, const TBArgs& a, cudaStream_t s);
int tb_configure(int nv, int spt, int tpb);
bool tb_build_tiles(const Plan* p, int s, std::vector<TBTile>& tiles, std::vector<int32_t>& begin);
// the tiles of one W x L ribbon for s orders per launch and rmax region sites per CTA
// (appended to tiles); false if one interior column does not fit
// align > 0: padded rows of the register-run kernel (stride a multiple of align, >= 1 pad);
// uniform: one stride and box height for all tiles of the ribbon (tensor-memory-access boxes)
bool tb_tiles_of_ribbon(int W, int L, int s, int rmax, int block, std::vector<TBTile>& tiles,
                        int align = 0, bool uniform = false);
// host work model of one blocked launch over the given tiles (cheb_plan_step_model)
struct TBModel {
    double useful = 0.0, computed = 0.0, smem = 0.0, l2 = 0.0;
};
void tb_model_launch(const Plan* p, const std::vector<TBTile>& tiles, int ka, int kb,
                     int prev_ka, TBModel& m);
// temporal blocking with register-resident runs (cheb_tbr.cu), with or without boxes
inline bool tb_runs(int kernel) { return kernel == CHEB_TB_RUNS || kernel == CHEB_TB_RUNS_TMA; }
bool tbr_tma_available();
int tbr_maps_prepare(Plan* p);                               // maps of the internal buffers
int tbr_maps_psi(Plan* p, const void* psi, int slot, cudaStream_t s);  // psi maps into a slot
const void* tbr_maps_for(const Plan* p, int launch, int which, const void* psi, int slot);
bool tbr_supported(int nv, int run, int tpb);
size_t tbr_smem_bytes(int nv, int run, int tpb);
int tbr_configure(int nv, int run, int tpb);
int tbr_blocks_per_sm(int nv, int run, int tpb);  // resident CTAs per SM (0 on error)
int tbr_launch(Plan* p, const TBArgs& a, cudaStream_t s);
void tbr_model_launch(const Plan* p, const std::vector<TBTile>& tiles, int ka, int kb,
                      int prev_ka, TBModel& m);

// kernel launchers (cheb_kernels.cu)
int launch_recurrence(Plan* p, const RecArgs& a, int op, int prec, cudaStream_t s);
int launch_observable(Plan* p, const void* psi, int kind, double param, double* out,
                      cudaStream_t s);
int launch_scale_diag(Plan* p, const double* onsite, cudaStream_t s);
// FP64 record [block][vec][2] = (||psi||^2, <psi|H|psi>) of psi (complex64 plans' records)
int record_prepare(Plan* p);
int launch_record(Plan* p, const void* psi, double* out, cudaStream_t s);

// one step of a small 1D grid on a thread-block cluster (cheb_cluster.cu)
bool cluster_eligible(const Plan* p);
int cluster_configure(Plan* p, int ctas);
int cluster_launch(Plan* p, void* psi, cudaStream_t s);

// Holstein (cheb_holstein.cu: stored SELL matrix; cheb_holmf.cu: matrix-free operator)
int holstein_build(Plan* p);
int holmf_build(Plan* p);
int launch_holmf(Plan* p, const RecArgs& a, cudaStream_t s);
int launch_holmf_energy(Plan* p, const void* psi, double* out, cudaStream_t s);

// host Bessel (cheb_coeffs.cpp)
int bessel_j_seq(double z, int kmax, std::vector<double>& J);

// ---- the plan ----------------------------------------------------------------------------
struct Plan {
    cheb_ham_desc desc{};
    int prec = CHEB_C128;
    int nvec = 1;
    int op = OP_STENCIL;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    double alpha = 0.0;
    double tol = 1e-14;
    int max_order = 100000;
    double dt = 0.0;
    bool have_dt = false;

    int64_t n_sites = 0;
    int nblocks = 1;
    std::vector<double> emin, emax;
    std::vector<DevBlock> hblocks;
    std::vector<WorkItem> hitems;
    std::vector<int32_t> hblock_item_begin;
    int max_M = 0;

    // device data
    DevBlock* d_blocks = nullptr;
    WorkItem* d_items = nullptr;
    int32_t* d_block_item_begin = nullptr;
    void* d_diag = nullptr;     // R [site] or [site][vec]
    void* d_A = nullptr;        // recurrence vectors
    void* d_B = nullptr;
    void* d_tail = nullptr;     // second accumulator (complex64 plans)
    void* d_qcoef = nullptr;    // R
    size_t qcoef_cap = 0;
    double* d_partials = nullptr;
    unsigned int* d_counter = nullptr;
    double* d_red = nullptr;    // [nblocks][nvec][2]
    int* d_err = nullptr;
    double* d_obs_scratch = nullptr; // observable partials
    size_t obs_scratch_cap = 0;
    double* d_rec_scratch = nullptr; // partials of the FP64 records (complex64 plans)
    size_t rec_scratch_cap = 0;

    // SELL (Holstein)
    int64_t sell_nnz_stored = 0;
    int64_t sell_nchunks = 0;
    int32_t* d_sell_col = nullptr;
    void* d_sell_val = nullptr;
    int64_t* d_sell_chunk_off = nullptr;
    int32_t* d_sell_chunk_len = nullptr;
    int32_t* d_sell_perm = nullptr;   // row of each storage position (sigma sorting)
    int sell_sigma = 1;               // rows sorted by length inside windows of sigma rows
    int64_t sell_nnz_offdiag = 0;     // off-diagonal entries without padding
    double* d_hol_diag_raw = nullptr; // unscaled H_ii (double)
    double* d_sell_val_raw = nullptr; // unscaled off-diagonals (double), same layout
    int64_t hol_dph = 0;
    int64_t* d_binom = nullptr;       // binomial table for on-device ranking
    uint8_t* d_hol_rowlen = nullptr;  // true off-diagonal count per row (export, energy)

    // matrix-free Holstein operator
    int2* d_holmf_G = nullptr;        // tuple-count pairs (G(j, R - 1), G(j, R))
    void* d_holmf_dtab = nullptr;     // R [L][nph + 1] scaled diagonal by total phonon number
    void* d_holmf_qtab = nullptr;     // R [L][nph + 1] scaled phonon matrix elements
    double* d_holmf_partials = nullptr;
    size_t holmf_partials_cap = 0;
    int holmf_variant = 0;            // 0, 1: one phonon configuration per thread
                                      // (1: register cap); 2: two

    // launch shape
    int threads = 256;
    int spt = 1;         // sites per thread
    int grid_cap = 0;    // 0: one CTA per work item
    int vpt = 0;         // vectors per thread (0: default for the precision)
    int64_t tile = 256;
    bool tuned = false;

    // graphs of one step, one per psi pointer (a few kept; rebuilt when dt or the launch
    // shape change)
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        const void* psi = nullptr;
        int64_t epoch = -1;
        int kernels = 0;
        int64_t used = 0;
    };
    static constexpr int kGraphSlots = 4;
    StepGraph graphs[kGraphSlots];
    int64_t graph_clock = 0;
    cudaStream_t cap_stream = nullptr;
    int64_t shape_epoch = 0;  // bumped whenever items / launch shape / coefficients change

    // batches of jobs from host memory (cheb_evolve_host): three device buffers (one being
    // propagated while the next job's state arrives and the previous one's leaves), a stream
    // per copy direction and their events (created on first use)
    static constexpr int kJobBuffers = 3;
    static_assert(kJobBuffers <= kGraphSlots, "every job buffer needs its own step graph");
    void* d_job[kJobBuffers] = {};
    cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
    cudaEvent_t ev_in[kJobBuffers] = {}, ev_done[kJobBuffers] = {}, ev_out[kJobBuffers] = {};

    int64_t launches = 0;

    // temporal blocking (complex64 stencils): orders per launch (0: off), sites per thread
    int tb_s = 0;
    int cluster = 0;          // CTAs of the cluster running whole steps (small 1D grids); 0: off
    int tb_spt = 4;           // sites per thread (CHEB_TB_RUNS: the run length)
    int tb_tpb = 256;         // threads per CTA of the blocked kernel
    int tb_kernel = CHEB_TB_SITES;  // blocked kernel: strided sites or register runs (+ boxes)
    int tb_grid_cap = 0;      // CTAs of a blocked launch (cheb_plan_set_blocking_grid; 0: default)
    int tbr_resident = 0;     // resident CTAs of the register-run kernel's shape (SMs x per SM)
    void* d_C = nullptr;      // second recurrence pair and the main accumulator
    void* d_D = nullptr;
    void* d_E = nullptr;
    std::vector<TBSet> tb_sets;
    struct TBLaunch {
        int ka, kb, prev_ka, set;
    };
    std::vector<TBLaunch> tb_sched;   // launches of one step (rebuilt with dt / tb_s)
    // tensor maps of the register-run kernel (cheb_tbr.cu): per launch of the schedule the maps
    // of its T_{ka-1} and T_{ka-2} buffers, then kGraphSlots + 1 slots for psi (the graph slots,
    // then the slot of launches enqueued outside a capture); each map array holds
    // nblocks * pairs maps.  tm_psi_slot: the psi slot a capture in progress uses.
    void* d_tmaps = nullptr;
    size_t tmaps_cap = 0;
    size_t tmap_array = 0;            // bytes of one map array
    struct TMPsi {
        const void* psi = nullptr;
        int64_t epoch = -1;
    } tm_psi[kGraphSlots + 1];
    int tm_psi_slot = kGraphSlots;
    double* d_tb_partials = nullptr;
    size_t tb_partials_cap = 0;

    // adjoint: plan-owned workspace and the graph of the last gradient call
    void* adj_ws = nullptr;
    size_t adj_ws_bytes = 0;
    cudaGraphExec_t adj_graph = nullptr;
    struct AdjKey {
        const void* psi0;
        const void* lambda_n;
        int64_t region_col;
        const void* grad;
        const void* lambda0;
        const void* P;
        int nsteps;
        double dt;
        int64_t epoch;
        const void* ws;
    } adj_key{};
    int adj_graph_kernels = 0;

    // kernel timing (cheb_plan_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;               // events used since the last collection (pairs)
    std::vector<double> ev_bytes;     // algorithmic bytes of each timed launch
    double t_ms = 0.0, t_bytes = 0.0;
    int64_t t_launches = 0;

    size_t real_size() const { return prec == CHEB_C128 ? sizeof(double) : sizeof(float); }
    size_t cplx_size() const { return 2 * real_size(); }
    size_t vec_bytes() const { return (size_t)n_sites * (size_t)nvec * cplx_size(); }
};

int plan_build_items(Plan* p);
int plan_enqueue_step(Plan* p, void* psi, cudaStream_t s);
int obs_prepare(Plan* p);
int vpt_for(int prec, int nvec, int want);

}  // namespace cheb
