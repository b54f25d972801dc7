// Plan lifecycle, propagation (Sec. 2.2), observables and tuning behind the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cheb_internal.cuh"

namespace cheb {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    // a refused call (a launch configuration or an attribute the device does not accept) also
    // leaves its error as the runtime's last error; clear it so that the next launch check of
    // the plan does not report it again (sticky errors stay with the context regardless)
    cudaGetLastError();
    return CHEB_ERR_CUDA;
}

// Split every block into tiles of `tile` sites; Holstein tiles also never straddle two
// electron sites (blocks of Dph rows), so per-tile observables have a single slot.
int plan_build_items(Plan* p)
{
    const int nvg = p->nvec / vpt_for(p->prec, p->nvec, p->vpt);
    int64_t tile = (int64_t)p->threads * p->spt / nvg;
    if (tile < 1) tile = 1;
    p->tile = tile;
    p->hitems.clear();
    p->hblock_item_begin.assign(p->nblocks + 1, 0);
    for (int q = 0; q < p->nblocks; ++q) {
        p->hblock_item_begin[q] = (int32_t)p->hitems.size();
        const DevBlock& B = p->hblocks[q];
        const int64_t n = (p->desc.kind == CHEB_HOLSTEIN) ? p->n_sites : (int64_t)B.W * B.L;
        const int64_t seg = (p->desc.kind == CHEB_HOLSTEIN) ? p->hol_dph : n;
        for (int64_t s0 = 0; s0 < n; s0 += seg) {
            const int64_t s1 = std::min(n, s0 + seg);
            for (int64_t f = s0; f < s1; f += tile) {
                WorkItem it;
                it.block = q;
                it.pad = 0;
                it.first = f;
                it.count = std::min(tile, s1 - f);
                p->hitems.push_back(it);
            }
        }
    }
    p->hblock_item_begin[p->nblocks] = (int32_t)p->hitems.size();
    if (p->hitems.size() >= (size_t)INT32_MAX) return fail(CHEB_ERR_INVALID, "too many work items");
    if (p->d_items) cudaFree(p->d_items);
    if (p->d_block_item_begin) cudaFree(p->d_block_item_begin);
    if (p->d_partials) cudaFree(p->d_partials);
    p->d_items = nullptr;
    p->d_block_item_begin = nullptr;
    p->d_partials = nullptr;
    CHEB_CUDA(cudaMalloc(&p->d_items, p->hitems.size() * sizeof(WorkItem)));
    CHEB_CUDA(cudaMemcpy(p->d_items, p->hitems.data(), p->hitems.size() * sizeof(WorkItem),
                         cudaMemcpyHostToDevice));
    CHEB_CUDA(cudaMalloc(&p->d_block_item_begin, (p->nblocks + 1) * sizeof(int32_t)));
    CHEB_CUDA(cudaMemcpy(p->d_block_item_begin, p->hblock_item_begin.data(),
                         (p->nblocks + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    CHEB_CUDA(cudaMalloc(&p->d_partials, p->hitems.size() * p->nvec * 2 * sizeof(double)));
    p->shape_epoch++;
    return CHEB_OK;
}

static int upload_blocks(Plan* p)
{
    CHEB_CUDA(cudaMemcpy(p->d_blocks, p->hblocks.data(), p->hblocks.size() * sizeof(DevBlock),
                         cudaMemcpyHostToDevice));
    return CHEB_OK;
}

static int tb_prepare(Plan* p);

// Coefficients for a new dt: q_k = sign_k (2 - delta_k0) J_k(a dt) with sign_k = +1 for
// k mod 4 in {0, 1} and -1 for {2, 3}, so that (-i)^k (2 - delta_k0) J_k = q_k (1 or -i).
static int set_dt(Plan* p, double dt)
{
    if (p->have_dt && dt == p->dt) return CHEB_OK;
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(CHEB_ERR_INVALID, "dt must be >= 0");
    std::vector<double> table;
    int maxM = 0;
    for (int q = 0; q < p->nblocks; ++q) {
        DevBlock& B = p->hblocks[q];
        std::vector<double> cre((size_t)p->max_order + 1), cim((size_t)p->max_order + 1);
        int M = 0;
        int rc = cheb_coeffs(B.a, B.b, dt, p->tol, p->max_order, cre.data(), cim.data(), &M);
        if (rc) return rc;
        // recover q_k from C_k = e^{-i b dt} (-i)^k g_k: use the Bessel values directly
        std::vector<double> J;
        const long natural = (long)std::ceil(B.a * dt + 60.0 + 20.0 * std::cbrt(B.a * dt));
        const int kmax = (int)std::min<long>((long)p->max_order, std::max<long>(natural, M));
        if (bessel_j_seq(B.a * dt, kmax, J) != 0) return fail(CHEB_ERR_INVALID, "Bessel failed");
        B.M = M;
        B.coef_off = (int32_t)table.size();
        int ksplit = 2;
        for (int k = 0; k <= M; ++k) {
            const double g = (k == 0 ? 1.0 : 2.0) * J[(size_t)k];
            table.push_back(((k & 3) >= 2) ? -g : g);
            if (std::fabs(g) >= 1.0 / 256.0) ksplit = std::max(ksplit, k);
        }
        // complex64: orders with |q_k| < 2^-8 go to the tail accumulator; the split is raised
        // to the next order = 2 (mod 3) so that no group of the single-order launches
        // straddles it
        ksplit += ((2 - ksplit % 3) + 3) % 3;
        B.ksplit = (p->prec == CHEB_C64) ? std::min(ksplit, M) : M;
        B.ph_re = std::cos(B.b * dt);
        B.ph_im = -std::sin(B.b * dt);
        maxM = std::max(maxM, M);
    }
    // device table: (hi, lo) pairs in the plan's real type, q = hi + lo (lo = 0 for double)
    const size_t bytes = table.size() * 2 * p->real_size();
    if (p->qcoef_cap < bytes) {
        if (p->d_qcoef) cudaFree(p->d_qcoef);
        p->d_qcoef = nullptr;
        p->qcoef_cap = 0;
        CHEB_CUDA(cudaMalloc(&p->d_qcoef, bytes));
        p->qcoef_cap = bytes;
    }
    if (p->prec == CHEB_C128) {
        std::vector<double> t2(2 * table.size(), 0.0);
        for (size_t i = 0; i < table.size(); ++i) t2[2 * i] = table[i];
        CHEB_CUDA(cudaMemcpy(p->d_qcoef, t2.data(), bytes, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> t2(2 * table.size());
        for (size_t i = 0; i < table.size(); ++i) {
            const float hi = (float)table[i];
            t2[2 * i] = hi;
            t2[2 * i + 1] = (float)(table[i] - (double)hi);
        }
        CHEB_CUDA(cudaMemcpy(p->d_qcoef, t2.data(), bytes, cudaMemcpyHostToDevice));
    }
    int rc = upload_blocks(p);
    if (rc) return rc;
    p->max_M = maxM;
    p->dt = dt;
    p->have_dt = true;
    p->shape_epoch++;
    return tb_prepare(p);
}

static RecArgs base_args(Plan* p)
{
    RecArgs a;
    std::memset(&a, 0, sizeof(a));
    a.items = p->d_items;
    a.nitems = (int32_t)p->hitems.size();
    a.nvec = p->nvec;
    a.blocks = p->d_blocks;
    a.diag = p->d_diag;
    a.diag_per_vec = p->desc.onsite_per_vec;
    a.qcoef = p->d_qcoef;
    a.sell_col = p->d_sell_col;
    a.sell_val = p->d_sell_val;
    a.sell_chunk_off = p->d_sell_chunk_off;
    a.sell_chunk_len = p->d_sell_chunk_len;
    a.sell_perm = p->d_sell_perm;
    a.partials = p->d_partials;
    a.done_counter = p->d_counter;
    a.red_out = p->d_red;
    a.nblocks = p->nblocks;
    a.block_item_begin = p->d_block_item_begin;
    a.norm2 = p->d_red;
    a.errflag = p->d_err;
    a.tail = p->d_tail;
    return a;
}

// Algorithmic DRAM bytes of the launch forming T_k: every vector element the launch touches
// read or written once, the on-site data (and SELL entries) read once, for the sites of the
// blocks whose order reaches k.
static double launch_bytes(const Plan* p, int k)
{
    const double cs = (double)p->cplx_size() * p->nvec;
    // the matrix-free operator stores no diagonal
    const double ds = (p->op == OP_HOLMF) ? 0.0
                      : (double)p->real_size() * (p->desc.onsite_per_vec ? p->nvec : 1);
    double total = 0.0;
    for (const DevBlock& B : p->hblocks) {
        if (k > B.M) continue;
        const double sites = (p->op != OP_STENCIL) ? (double)p->n_sites : (double)B.W * B.L;
        double vecs;  // vectors read + written per site
        if (k == 1) {
            vecs = 2;                    // read psi; write T_1
        } else {
            const AccGroup ag(k, B.M, B.ksplit);
            vecs = 3;                    // read T_{k-1}, T_{k-2} (k = 2: psi); write T_k
            if (ag.upd) vecs += 1 + (ag.read_acc ? 1 : 0) + (ag.read_psi_last ? 1 : 0);
        }
        total += sites * (vecs * cs + ds);
    }
    if (p->op == OP_SELL) {
        total += (double)p->sell_nnz_stored * (4.0 + (double)p->real_size());
        if (p->d_sell_perm) total += 4.0 * (double)p->n_sites;  // row of each position
    }
    return total;
}

static int timed_launch(Plan* p, const RecArgs& a, cudaStream_t s)
{
    if (!p->timing) return launch_recurrence(p, a, p->op, p->prec, s);
    if (p->ev_used + 2 > p->ev_pool.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            CHEB_CUDA(cudaEventCreate(&e));
            p->ev_pool.push_back(e);
        }
    }
    CHEB_CUDA(cudaEventRecord(p->ev_pool[p->ev_used], s));
    int rc = launch_recurrence(p, a, p->op, p->prec, s);
    if (rc) return rc;
    CHEB_CUDA(cudaEventRecord(p->ev_pool[p->ev_used + 1], s));
    p->ev_used += 2;
    p->ev_bytes.push_back(launch_bytes(p, a.j + 1));
    return CHEB_OK;
}

// fold the recorded event pairs into the sums (synchronises)
static int collect_timing(Plan* p)
{
    if (p->ev_used == 0) return CHEB_OK;
    CHEB_CUDA(cudaEventSynchronize(p->ev_pool[p->ev_used - 1]));
    for (size_t i = 0; i < p->ev_used; i += 2) {
        float ms = 0.0f;
        CHEB_CUDA(cudaEventElapsedTime(&ms, p->ev_pool[i], p->ev_pool[i + 1]));
        p->t_ms += ms;
        p->t_bytes += p->ev_bytes[i / 2];
        p->t_launches++;
    }
    p->ev_used = 0;
    p->ev_bytes.clear();
    return CHEB_OK;
}

// ---- temporal blocking ---------------------------------------------------------------------
static bool tb_eligible(const Plan* p)
{
    return p->op == OP_STENCIL && p->prec == CHEB_C64 && !p->desc.onsite_per_vec &&
           (p->nvec == 1 || p->nvec == 2 || p->nvec == 4);
}

static int tb_set_for(Plan* p, int s)
{
    for (size_t i = 0; i < p->tb_sets.size(); ++i)
        if (p->tb_sets[i].s == s) return (int)i;
    std::vector<TBTile> tiles;
    std::vector<int32_t> begin;
    if (!tb_build_tiles(p, s, tiles, begin)) return -1;
    TBSet set;
    set.s = s;
    set.ntiles = (int)tiles.size();
    for (int q = 0; q < p->nblocks; ++q) set.first.push_back(tiles[(size_t)begin[q]]);
    if (cudaMalloc(&set.d_tiles, tiles.size() * sizeof(TBTile)) != cudaSuccess) return -2;
    if (cudaMalloc(&set.d_begin, begin.size() * sizeof(int32_t)) != cudaSuccess) {
        cudaFree(set.d_tiles);
        return -2;
    }
    cudaMemcpy(set.d_tiles, tiles.data(), tiles.size() * sizeof(TBTile), cudaMemcpyHostToDevice);
    cudaMemcpy(set.d_begin, begin.data(), begin.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    p->tb_sets.push_back(set);
    return (int)p->tb_sets.size() - 1;
}

// Launch schedule of one step with temporal blocking: orders 1..s0 (s0 < min M, so the first
// launch, which reads psi as T_0, never writes psi), then blocks of tb_s orders up to max M,
// the last block lengthened instead of followed by a short one.
// Builds the tile sets and buffers it needs (outside any stream capture).  On failure the
// plan falls back to single-order launches (tb_s = 0).
static int tb_prepare(Plan* p)
{
    p->tb_sched.clear();
    if (p->tb_s <= 0 || !tb_eligible(p) || !p->have_dt) return CHEB_OK;
    int minM = 1 << 30, maxM = 0;
    for (const DevBlock& B : p->hblocks) {
        minM = std::min(minM, (int)B.M);
        maxM = std::max(maxM, (int)B.M);
    }
    int rc0 = tb_runs(p->tb_kernel) ? tbr_configure(p->nvec, p->tb_spt, p->tb_tpb)
                                    : tb_configure(p->nvec, p->tb_spt, p->tb_tpb);
    if (rc0) {
        p->tb_s = 0;
        return rc0;
    }
    p->tbr_resident = tb_runs(p->tb_kernel)
                          ? tbr_blocks_per_sm(p->nvec, p->tb_spt, p->tb_tpb) * p->num_sms
                          : 0;
    const int s0 = std::max(1, std::min(p->tb_s, minM - 1));
    // order ranges [ka, kb] of the launches; a last range shorter than half a block is merged
    // into the one before (a launch costs its region loads and stores however few orders it
    // runs), unless that is the first launch, which must stay below min M
    std::vector<std::pair<int, int>> ranges;
    for (int ka = 1, kb = s0; ka <= maxM; ka = kb + 1, kb = std::min(ka + p->tb_s - 1, maxM))
        ranges.push_back({ka, kb});
    if (ranges.size() >= 3 && 2 * (ranges.back().second - ranges.back().first + 1) < p->tb_s) {
        const int len = ranges.back().second - ranges[ranges.size() - 2].first + 1;
        if (tb_set_for(p, len) >= 0) {  // else the ribbons do not fit the wider halo: keep both
            ranges[ranges.size() - 2].second = ranges.back().second;
            ranges.pop_back();
        }
    }
    std::vector<Plan::TBLaunch> sched;
    int prev = 0;
    for (const auto& rg : ranges) {
        const int set = tb_set_for(p, rg.second - rg.first + 1);
        if (set < 0) {
            p->tb_s = 0;
            return set == -2 ? fail(CHEB_ERR_NOMEM, "temporal blocking tiles") : CHEB_OK;
        }
        sched.push_back({rg.first, rg.second, prev, set});
        prev = rg.first;
    }
    const size_t vb = p->vec_bytes();
    for (void** b : {&p->d_C, &p->d_D, &p->d_E}) {
        if (!*b && cudaMalloc(b, vb) != cudaSuccess) return fail(CHEB_ERR_NOMEM, "temporal blocking buffers");
    }
    const size_t need = (size_t)p->tb_sets[sched[0].set].ntiles * p->nvec * 2;
    if (p->tb_partials_cap < need) {
        if (p->d_tb_partials) cudaFree(p->d_tb_partials);
        p->d_tb_partials = nullptr;
        p->tb_partials_cap = 0;
        if (cudaMalloc(&p->d_tb_partials, need * sizeof(double)) != cudaSuccess)
            return fail(CHEB_ERR_NOMEM, "temporal blocking partials");
        p->tb_partials_cap = need;
    }
    p->tb_sched = sched;
    p->shape_epoch++;
    return tbr_maps_prepare(p);
}

// algorithmic bytes of one blocked launch: region inputs counted once per interior site
static double tb_launch_bytes(const Plan* p, const Plan::TBLaunch& L)
{
    const double cs = (double)p->cplx_size() * p->nvec;
    const double ds = (double)p->real_size();
    double total = 0.0;
    for (const DevBlock& B : p->hblocks) {
        if (L.ka > B.M) continue;
        const double sites = (double)B.W * B.L;
        const bool first = L.ka == 1;
        const bool done = std::min(L.kb, (int)B.M) == B.M;
        const bool to_main = first || L.ka <= B.ksplit;
        const bool tail_has = L.prev_ka > B.ksplit;
        double v = (first ? 1 : 2);                  // T_{ka-1}, T_{ka-2}
        v += done ? 0 : 2;                           // T_{ke-1}, T_{ke} out
        if (!done) v += (to_main ? (first ? 0 : 1) : (tail_has ? 1 : 0)) + 1;  // acc in/out
        else v += (to_main ? 1 : (tail_has ? 2 : 1)) + 1;                    // E (+tail), psi
        total += sites * (v * cs + ds);
    }
    return total;
}

static int enqueue_step_tb(Plan* p, void* psi, cudaStream_t st);

// Enqueue the M_max fused kernels of one step on stream s.
// One step on the thread-block cluster (all M orders in one launch), timed like the others.
static int enqueue_step_cluster(Plan* p, void* psi, cudaStream_t s)
{
    if (p->timing) {
        if (p->ev_used + 2 > p->ev_pool.size()) {
            for (int e = 0; e < 64; ++e) {
                cudaEvent_t ev;
                CHEB_CUDA(cudaEventCreate(&ev));
                p->ev_pool.push_back(ev);
            }
        }
        CHEB_CUDA(cudaEventRecord(p->ev_pool[p->ev_used], s));
    }
    int rc = cluster_launch(p, psi, s);
    if (rc) return rc;
    if (p->timing) {
        CHEB_CUDA(cudaEventRecord(p->ev_pool[p->ev_used + 1], s));
        p->ev_used += 2;
        // DRAM operands of the whole step: psi in and out, the scaled diagonal
        p->ev_bytes.push_back((double)p->n_sites * (2.0 * p->cplx_size() + p->real_size()));
    }
    return CHEB_OK;
}

static int enqueue_step(Plan* p, void* psi, cudaStream_t s)
{
    if (p->cluster && cluster_eligible(p)) return enqueue_step_cluster(p, psi, s);
    if (!p->tb_sched.empty()) return enqueue_step_tb(p, psi, s);
    RecArgs a = base_args(p);
    if (p->timing && p->ev_used > 4096) {  // keep the event pool bounded
        int rc = collect_timing(p);
        if (rc) return rc;
    }
    for (int j = 0; j < p->max_M; ++j) {
        a.j = j;
        if (j == 0) {
            a.mode = REC_FIRST;
            a.cur = psi;
            a.prev = p->d_A;
            a.out1 = p->d_B;
            a.psi = nullptr;
        } else {
            a.mode = (j == 1) ? REC_SECOND : REC_GENERAL;
            a.cur = (j & 1) ? p->d_B : p->d_A;
            a.prev = (j & 1) ? p->d_A : p->d_B;
            a.out1 = nullptr;
            a.psi = psi;
        }
        int rc = timed_launch(p, a, s);
        if (rc) return rc;
    }
    return CHEB_OK;
}

static int enqueue_step_tb(Plan* p, void* psi, cudaStream_t st)
{
    void* pairs[2][2] = {{p->d_A, p->d_B}, {p->d_C, p->d_D}};
    // tensor maps of psi for the first launch (register-run kernel): the plan's own step-graph
    // capture uses the slot its graph prepared; launches enqueued directly use the last slot,
    // refreshed here; any other capture uses none (per-thread copies: a later call may rewrite
    // the last slot for another psi)
    int slot = p->tm_psi_slot;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CHEB_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
        slot = Plan::kGraphSlots;
        int rc = tbr_maps_psi(p, psi, slot, st);
        if (rc) return rc;
    } else if (slot == Plan::kGraphSlots) {
        slot = -1;
    }
    // the register-run kernel adds its first launch's ||psi||^2 into the (ribbon, vector)
    // slots of the growth check
    if (tb_runs(p->tb_kernel))
        CHEB_CUDA(cudaMemsetAsync(p->d_red, 0, (size_t)p->nblocks * p->nvec * 2 * sizeof(double), st));
    for (size_t i = 0; i < p->tb_sched.size(); ++i) {
        const Plan::TBLaunch& L = p->tb_sched[i];
        const TBSet& set = p->tb_sets[L.set];
        TBArgs a;
        std::memset(&a, 0, sizeof(a));
        a.tiles = set.d_tiles;
        a.ntiles = set.ntiles;
        a.ka = L.ka;
        a.kb = L.kb;
        a.prev_ka = L.prev_ka;
        a.blocks = p->d_blocks;
        a.nvec = p->nvec;
        a.diag = p->d_diag;
        if (i == 0) {
            a.in_prev = nullptr;
            a.in_cur = psi;
        } else {
            a.in_prev = pairs[(i - 1) & 1][0];
            a.in_cur = pairs[(i - 1) & 1][1];
        }
        a.out_prev = pairs[i & 1][0];
        a.out_cur = pairs[i & 1][1];
        a.acc_main = p->d_E;
        a.tail = p->d_tail;
        a.psi = psi;
        a.qcoef = p->d_qcoef;
        a.partials = p->d_tb_partials;
        a.done_counter = p->d_counter;
        a.red_out = p->d_red;
        a.nblocks = p->nblocks;
        a.block_tile_begin = set.d_begin;
        a.norm2 = p->d_red;
        a.errflag = p->d_err;
        a.tm_cur = tbr_maps_for(p, (int)i, 0, psi, slot);
        a.tm_prev = tbr_maps_for(p, (int)i, 1, psi, slot);
        a.nsites = p->n_sites;
        if (p->timing) {
            if (p->ev_used + 2 > p->ev_pool.size()) {
                for (int e = 0; e < 64; ++e) {
                    cudaEvent_t ev;
                    CHEB_CUDA(cudaEventCreate(&ev));
                    p->ev_pool.push_back(ev);
                }
            }
            CHEB_CUDA(cudaEventRecord(p->ev_pool[p->ev_used], st));
        }
        int rc = tb_runs(p->tb_kernel) ? tbr_launch(p, a, st) : tb_launch(p, a, st);
        if (rc) return rc;
        if (p->timing) {
            CHEB_CUDA(cudaEventRecord(p->ev_pool[p->ev_used + 1], st));
            p->ev_used += 2;
            p->ev_bytes.push_back(tb_launch_bytes(p, L));
        }
    }
    return CHEB_OK;
}

int plan_enqueue_step(Plan* p, void* psi, cudaStream_t s) { return enqueue_step(p, psi, s); }

// bytes of one record of cheb_evolve's obs array: [block][vec][2] doubles
static size_t rec_bytes(const Plan* p) { return (size_t)p->nblocks * p->nvec * 2 * sizeof(double); }

static int check_psi(const Plan* p, const void* psi)
{
    if (!psi) return fail(CHEB_ERR_INVALID, "psi is NULL");
    if (!aligned16(psi)) return fail(CHEB_ERR_ALIGN, "psi must be 16-byte aligned");
    return CHEB_OK;
}

// The step graph for this psi pointer: a cached one if dt and the launch shape are unchanged,
// else captured into the least recently used slot.
static int ensure_graph(Plan* p, void* psi, Plan::StepGraph** out)
{
    Plan::StepGraph* slot = nullptr;
    for (Plan::StepGraph& g : p->graphs)
        if (g.exec && g.psi == psi && g.epoch == p->shape_epoch) slot = &g;
    if (slot) {
        slot->used = ++p->graph_clock;
        *out = slot;
        return CHEB_OK;
    }
    slot = &p->graphs[0];
    for (Plan::StepGraph& g : p->graphs) {
        if (!g.exec) {
            slot = &g;
            break;
        }
        if (g.used < slot->used) slot = &g;
    }
    if (slot->exec) {
        cudaGraphExecDestroy(slot->exec);
        slot->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    // psi's tensor maps for this graph slot, ordered on the plan's stream before any replay
    const int gslot = (int)(slot - p->graphs);
    int rc0 = tbr_maps_psi(p, psi, gslot, p->stream);
    if (rc0) return rc0;
    p->tm_psi_slot = gslot;
    CHEB_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int64_t before = p->launches;
    int rc = enqueue_step(p, psi, p->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
    p->tm_psi_slot = Plan::kGraphSlots;
    const int64_t captured = p->launches - before;
    p->launches = before;  // captured launches are counted when the graph is replayed
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&slot->exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
    slot->psi = psi;
    slot->epoch = p->shape_epoch;
    slot->kernels = (int)captured;
    slot->used = ++p->graph_clock;
    *out = slot;
    return CHEB_OK;
}

static void free_plan(Plan* p)
{
    if (!p) return;
    for (Plan::StepGraph& g : p->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    for (int b = 0; b < Plan::kJobBuffers; ++b) {
        if (p->d_job[b]) cudaFree(p->d_job[b]);
        for (cudaEvent_t e : {p->ev_in[b], p->ev_done[b], p->ev_out[b]})
            if (e) cudaEventDestroy(e);
    }
    if (p->h2d_stream) cudaStreamDestroy(p->h2d_stream);
    if (p->d2h_stream) cudaStreamDestroy(p->d2h_stream);
    for (TBSet& t : p->tb_sets) {
        if (t.d_tiles) cudaFree(t.d_tiles);
        if (t.d_begin) cudaFree(t.d_begin);
    }
    for (void* q : {p->d_C, p->d_D, p->d_E, (void*)p->d_tb_partials, p->adj_ws, p->d_tmaps})
        if (q) cudaFree(q);
    if (p->adj_graph) cudaGraphExecDestroy(p->adj_graph);
    void* ptrs[] = {p->d_blocks, p->d_items, p->d_block_item_begin, p->d_diag, p->d_A, p->d_B,
                    p->d_tail,
                    p->d_qcoef, p->d_partials, p->d_counter, p->d_red, p->d_err,
                    p->d_obs_scratch, p->d_rec_scratch, p->d_sell_col, p->d_sell_val, p->d_sell_chunk_off,
                    p->d_sell_chunk_len, p->d_sell_perm, p->d_hol_diag_raw, p->d_sell_val_raw, p->d_binom,
                    p->d_hol_rowlen, p->d_holmf_G, p->d_holmf_dtab, p->d_holmf_qtab,
                    p->d_holmf_partials};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
}

}  // namespace cheb

using namespace cheb;

extern "C" const char* cheb_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* cheb_strerror(int status)
{
    switch (status) {
        case CHEB_OK: return "ok";
        case CHEB_ERR_INVALID: return "invalid argument";
        case CHEB_ERR_ALIGN: return "device pointer not 16-byte aligned";
        case CHEB_ERR_CUDA: return "CUDA runtime error";
        case CHEB_ERR_NOMEM: return "out of memory";
        case CHEB_ERR_UNSUPPORTED: return "unsupported for this operator";
        case CHEB_ERR_ORDER: return "expansion order limit reached";
        case CHEB_ERR_DIVERGED: return "recurrence diverged (spectral bounds too tight)";
        case CHEB_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

extern "C" int cheb_plan_create(cheb_plan** out, const cheb_ham_desc* h, const double* emin,
                                const double* emax, double alpha, int prec, int nvec,
                                void* stream)
{
    if (!out || !h || !emin || !emax) return fail(CHEB_ERR_INVALID, "cheb_plan_create: NULL argument");
    *out = nullptr;
    if (prec != CHEB_C128 && prec != CHEB_C64) return fail(CHEB_ERR_INVALID, "bad precision");
    if (nvec < 1 || nvec > 32 || (nvec & (nvec - 1)) != 0)
        return fail(CHEB_ERR_INVALID, "nvec must be a power of two in [1, 32]");
    if (!(alpha >= 0.0)) return fail(CHEB_ERR_INVALID, "alpha must be >= 0");
    Plan* p = new Plan();
    p->desc = *h;
    p->prec = prec;
    p->nvec = nvec;
    p->alpha = alpha;
    p->stream = static_cast<cudaStream_t>(stream);
    int rc = CHEB_OK;
    auto bail = [&](int code) {
        free_plan(p);
        return code;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) return bail(fail(CHEB_ERR_CUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(CHEB_ERR_CUDA, "stream creation failed"));

    if (h->onsite && !aligned16(h->onsite))
        return bail(fail(CHEB_ERR_ALIGN, "onsite must be 16-byte aligned"));
    if (h->kind == CHEB_HOLSTEIN && h->hol_g && !aligned16(h->hol_g))
        return bail(fail(CHEB_ERR_ALIGN, "hol_g must be 16-byte aligned"));
    if (h->sell_sigma < 0 || (h->sell_sigma > 1 && (h->sell_sigma % 32 != 0 || h->sell_sigma > (1 << 20))))
        return bail(fail(CHEB_ERR_INVALID, "sell_sigma must be 0, 1 or a multiple of 32 up to 2^20"));
    p->sell_sigma = h->sell_sigma != 0 ? h->sell_sigma
                    : (prec == CHEB_C128 ? CHEB_SELL_SIGMA_DEFAULT_C128 : CHEB_SELL_SIGMA_DEFAULT_C64);
    if (h->onsite_per_vec && h->kind == CHEB_HOLSTEIN)
        return bail(fail(CHEB_ERR_UNSUPPORTED, "per-vector on-site data needs a lattice kind"));
    switch (h->kind) {
        case CHEB_LAT1D: {
            if (h->n < 1 || h->n > INT32_MAX || !(h->dx > 0.0))
                return bail(fail(CHEB_ERR_INVALID, "LAT1D needs 1 <= n < 2^31 and dx > 0"));
            p->nblocks = 1;
            p->op = OP_STENCIL;
            DevBlock B{};
            B.offset = 0;
            B.W = 1;
            B.L = (int32_t)h->n;
            p->hblocks.push_back(B);
            p->n_sites = h->n;
            break;
        }
        case CHEB_HONEYCOMB_ZZ: {
            if (h->nblocks < 1 || !h->W || !h->L)
                return bail(fail(CHEB_ERR_INVALID, "HONEYCOMB_ZZ needs nblocks >= 1 and W, L arrays"));
            p->nblocks = h->nblocks;
            p->op = OP_STENCIL;
            int64_t off = 0;
            for (int q = 0; q < h->nblocks; ++q) {
                if (h->W[q] < 1 || h->L[q] < 1 || (int64_t)h->W[q] * h->L[q] > INT32_MAX)
                    return bail(fail(CHEB_ERR_INVALID, "ribbon sizes must be >= 1 and W*L < 2^31"));
                DevBlock B{};
                B.offset = off;
                B.W = h->W[q];
                B.L = h->L[q];
                p->hblocks.push_back(B);
                off += (int64_t)h->W[q] * h->L[q];
            }
            p->n_sites = off;
            break;
        }
        case CHEB_HOLSTEIN: {
            if (h->hol_sites < 1 || h->hol_sites > 64 || h->hol_nph < 0 || h->hol_nph > 255 ||
                (h->hol_periodic && h->hol_sites < 3))
                return bail(fail(CHEB_ERR_INVALID, "HOLSTEIN needs 1 <= L <= 64 (L >= 3 periodic), 0 <= nph <= 255"));
            if (h->hol_matrix_free &&
                (h->hol_sites > 32 || h->hol_nph > 15))
                return bail(fail(CHEB_ERR_UNSUPPORTED, "matrix-free Holstein needs L <= 32 and nph <= 15"));
            p->nblocks = 1;
            p->op = h->hol_matrix_free ? OP_HOLMF : OP_SELL;
            const int64_t dph = cheb_holstein_dim_phonon(h->hol_sites, h->hol_nph);
            if (dph < 1) return bail(fail(CHEB_ERR_INVALID, "Holstein basis too large"));
            p->hol_dph = dph;
            DevBlock B{};
            B.offset = 0;
            B.W = 1;
            B.L = 1;
            p->hblocks.push_back(B);
            p->n_sites = (int64_t)h->hol_sites * dph;
            if (p->n_sites >= ((int64_t)1 << 31) - 64)
                return bail(fail(CHEB_ERR_INVALID, "Holstein dimension >= 2^31"));
            if (h->hol_matrix_free && (uint64_t)p->n_sites * (uint64_t)nvec >= ((uint64_t)1 << 32))
                return bail(fail(CHEB_ERR_UNSUPPORTED, "matrix-free Holstein needs rows * nvec < 2^32"));
            break;
        }
        default:
            return bail(fail(CHEB_ERR_INVALID, "unknown operator kind"));
    }
    // rescaling per block (Sec. 2.2)
    for (int q = 0; q < p->nblocks; ++q) {
        double a = 0, b = 0;
        rc = cheb_rescale(emin[q], emax[q], alpha, &a, &b);
        if (rc) return bail(rc);
        DevBlock& B = p->hblocks[q];
        B.a = a;
        B.b = b;
        B.M = 0;
        B.ph_re = 1.0;
        B.ph_im = 0.0;
        // scaled off-diagonal: 1D grid -1/(2 dx^2); ribbons -t
        const double off = (h->kind == CHEB_LAT1D) ? -0.5 / (h->dx * h->dx) : -h->hop;
        B.beta = 2.0 * off / a;
        if (prec == CHEB_C64 && off != 0.0 && std::isfinite(B.beta)) {
            // complex64 lattice plans: a grows by less than one part in 2^23 so that the
            // scaled hopping is a float32 number (|beta| rounded toward zero), which the
            // kernels then apply with one multiply-add and no rounding bias; any a at least
            // the half width of the spectrum is valid (Sec. 2.2)
            float bf = (float)B.beta;
            if (std::fabs((double)bf) > std::fabs(B.beta)) bf = std::nextafterf(bf, 0.0f);
            if (bf != 0.0f) {
                B.a = 2.0 * off / (double)bf;
                B.beta = (double)bf;
            }
        }
        p->emin.push_back(emin[q]);
        p->emax.push_back(emax[q]);
    }
    // device allocations
    if (cudaMalloc(&p->d_blocks, p->hblocks.size() * sizeof(DevBlock)) != cudaSuccess)
        return bail(fail(CHEB_ERR_NOMEM, "cudaMalloc blocks"));
    rc = upload_blocks(p);
    if (rc) return bail(rc);
    const size_t per = (h->onsite_per_vec ? (size_t)nvec : 1);
    if ((p->op != OP_HOLMF &&
         cudaMalloc(&p->d_diag, (size_t)p->n_sites * per * p->real_size()) != cudaSuccess) ||
        cudaMalloc(&p->d_A, p->vec_bytes()) != cudaSuccess ||
        cudaMalloc(&p->d_B, p->vec_bytes()) != cudaSuccess ||
        (prec == CHEB_C64 && cudaMalloc(&p->d_tail, p->vec_bytes()) != cudaSuccess) ||
        cudaMalloc(&p->d_counter, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&p->d_red, (size_t)p->nblocks * nvec * 2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&p->d_err, sizeof(int)) != cudaSuccess)
        return bail(fail(CHEB_ERR_NOMEM, "cudaMalloc workspace"));
    if (cudaMemset(p->d_counter, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(p->d_red, 0, (size_t)p->nblocks * nvec * 2 * sizeof(double)) != cudaSuccess)
        return bail(fail(CHEB_ERR_CUDA, "cudaMemset workspace"));
    rc = plan_build_items(p);
    if (rc) return bail(rc);
    if (h->kind == CHEB_HOLSTEIN) {
        rc = (p->op == OP_HOLMF) ? holmf_build(p) : holstein_build(p);
        if (rc) return bail(rc);
    } else {
        rc = launch_scale_diag(p, h->onsite, p->stream);
        if (rc) return bail(rc);
    }
    if (cudaStreamSynchronize(p->stream) != cudaSuccess)
        return bail(fail(CHEB_ERR_CUDA, "plan setup kernels failed"));
    // the descriptor's host arrays are not kept
    p->desc.W = nullptr;
    p->desc.L = nullptr;
    *out = reinterpret_cast<cheb_plan*>(p);
    return CHEB_OK;
}

extern "C" void cheb_plan_destroy(cheb_plan* plan)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    free_plan(p);
}

extern "C" int cheb_plan_set_tol(cheb_plan* plan, double tol, int max_order)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p || !(tol > 0.0) || max_order < 2) return fail(CHEB_ERR_INVALID, "cheb_plan_set_tol");
    p->tol = tol;
    p->max_order = max_order;
    p->have_dt = false;
    return CHEB_OK;
}

extern "C" int cheb_plan_set_onsite(cheb_plan* plan, const double* onsite)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (p->desc.kind == CHEB_HOLSTEIN)
        return fail(CHEB_ERR_UNSUPPORTED, "on-site data of a Holstein plan is fixed at creation");
    if (onsite && !aligned16(onsite)) return fail(CHEB_ERR_ALIGN, "onsite must be 16-byte aligned");
    return launch_scale_diag(p, onsite, p->stream);
}

extern "C" int cheb_plan_info(const cheb_plan* plan, int64_t* sites, int* nvec, int* nblocks)
{
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (sites) *sites = p->n_sites;
    if (nvec) *nvec = p->nvec;
    if (nblocks) *nblocks = p->nblocks;
    return CHEB_OK;
}

extern "C" int cheb_plan_block(const cheb_plan* plan, int q, double* a, double* b, int* M,
                               int64_t* offset, int* W, int* L)
{
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!p || q < 0 || q >= p->nblocks) return fail(CHEB_ERR_INVALID, "cheb_plan_block");
    const DevBlock& B = p->hblocks[q];
    if (a) *a = B.a;
    if (b) *b = B.b;
    if (M) *M = p->have_dt ? B.M : 0;
    if (offset) *offset = B.offset;
    if (W) *W = B.W;
    if (L) *L = B.L;
    return CHEB_OK;
}

extern "C" int cheb_step(cheb_plan* plan, void* psi, double dt)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    int rc = check_psi(p, psi);
    if (rc) return rc;
    rc = set_dt(p, dt);
    if (rc) return rc;
    return enqueue_step(p, psi, p->stream);
}

extern "C" int cheb_sync(cheb_plan* plan)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    int flag = 0;
    CHEB_CUDA(cudaMemcpyAsync(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    CHEB_CUDA(cudaStreamSynchronize(p->stream));
    if (flag) {
        CHEB_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->stream));
        CHEB_CUDA(cudaStreamSynchronize(p->stream));
        return fail(CHEB_ERR_DIVERGED, "a recurrence vector exceeded ||psi||: spectral bounds too tight");
    }
    return CHEB_OK;
}

extern "C" int cheb_evolve(cheb_plan* plan, void* psi, double dt, int nsteps, int obs_every,
                           double* obs)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (nsteps < 0) return fail(CHEB_ERR_INVALID, "nsteps < 0");
    int rc = check_psi(p, psi);
    if (rc) return rc;
    if (obs && !aligned16(obs)) return fail(CHEB_ERR_ALIGN, "obs must be 16-byte aligned");
    rc = set_dt(p, dt);
    if (rc) return rc;
    if (nsteps == 0) return CHEB_OK;
    Plan::StepGraph* graph = nullptr;
    if (!p->timing) {
        rc = ensure_graph(p, psi, &graph);
        if (rc) return rc;
    }
    const bool recording = obs && obs_every > 0;
    if (recording && p->prec == CHEB_C64) {
        rc = record_prepare(p);
        if (rc) return rc;
    }
    for (int s = 0; s < nsteps; ++s) {
        const bool rec = recording && s % obs_every == 0;
        double* slot = rec ? obs + (size_t)(s / obs_every) * p->nblocks * p->nvec * 2 : nullptr;
        if (rec && p->prec == CHEB_C64) {
            rc = launch_record(p, psi, slot, p->stream);
            if (rc) return rc;
        }
        if (p->timing) {
            rc = enqueue_step(p, psi, p->stream);
            if (rc) return rc;
        } else {
            CHEB_CUDA(cudaGraphLaunch(graph->exec, p->stream));
            p->launches += graph->kernels;
        }
        if (rec && p->prec == CHEB_C128) {  // the first launch's FP64 sums of this step
            CHEB_CUDA(cudaMemcpyAsync(slot, p->d_red, rec_bytes(p), cudaMemcpyDeviceToDevice,
                                      p->stream));
        }
    }
    return cheb_sync(plan);
}

// Jobs from host memory: job j is copied in while job j-1 runs and copied out while job j+1
// runs (two device buffers; compute on the plan's stream, one stream per copy direction).
extern "C" int cheb_evolve_host(cheb_plan* plan, const void* in, int64_t in_stride, void* out,
                                int64_t out_stride, int64_t njobs, double dt, int nsteps)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (njobs < 0 || nsteps < 0) return fail(CHEB_ERR_INVALID, "njobs and nsteps must be >= 0");
    if (njobs > 0 && (!in || !out)) return fail(CHEB_ERR_INVALID, "cheb_evolve_host: NULL buffer");
    const size_t jb = p->vec_bytes();
    if ((in_stride != 0 && in_stride < (int64_t)jb) || (out_stride != 0 && out_stride < (int64_t)jb))
        return fail(CHEB_ERR_INVALID, "cheb_evolve_host: a stride is neither 0 nor >= one state");
    if (njobs > 1 && (const void*)out == in && (in_stride != out_stride || in_stride == 0))
        return fail(CHEB_ERR_INVALID,
                    "cheb_evolve_host: in and out alias but the jobs' states do not match up");
    int rc = set_dt(p, dt);
    if (rc) return rc;
    if (njobs == 0) return CHEB_OK;
    constexpr int NB = Plan::kJobBuffers;
    for (int b = 0; b < NB; ++b) {
        if (!p->d_job[b] && cudaMalloc(&p->d_job[b], jb) != cudaSuccess)
            return fail(CHEB_ERR_NOMEM, "cheb_evolve_host: job buffers");
        for (cudaEvent_t* e : {&p->ev_in[b], &p->ev_done[b], &p->ev_out[b]})
            if (!*e) CHEB_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    if (!p->h2d_stream) CHEB_CUDA(cudaStreamCreateWithFlags(&p->h2d_stream, cudaStreamNonBlocking));
    if (!p->d2h_stream) CHEB_CUDA(cudaStreamCreateWithFlags(&p->d2h_stream, cudaStreamNonBlocking));
    Plan::StepGraph* graph[NB] = {};
    if (!p->timing && nsteps > 0) {
        for (int b = 0; b < NB; ++b) {
            rc = ensure_graph(p, p->d_job[b], &graph[b]);
            if (rc) return rc;
        }
    }
    const char* src = static_cast<const char*>(in);
    char* dst = static_cast<char*>(out);
    auto copy_in = [&](int64_t j) -> int {
        const int b = (int)(j % NB);
        if (j >= NB) CHEB_CUDA(cudaStreamWaitEvent(p->h2d_stream, p->ev_out[b], 0));  // buffer free
        CHEB_CUDA(cudaMemcpyAsync(p->d_job[b], src + (size_t)j * (size_t)in_stride, jb,
                                  cudaMemcpyHostToDevice, p->h2d_stream));
        CHEB_CUDA(cudaEventRecord(p->ev_in[b], p->h2d_stream));
        return CHEB_OK;
    };
    rc = copy_in(0);
    if (rc) return rc;
    for (int64_t j = 0; j < njobs; ++j) {
        const int b = (int)(j % NB);
        if (j + 1 < njobs) {
            rc = copy_in(j + 1);
            if (rc) return rc;
        }
        CHEB_CUDA(cudaStreamWaitEvent(p->stream, p->ev_in[b], 0));
        for (int s = 0; s < nsteps; ++s) {
            if (graph[b]) {
                CHEB_CUDA(cudaGraphLaunch(graph[b]->exec, p->stream));
                p->launches += graph[b]->kernels;
            } else {
                rc = enqueue_step(p, p->d_job[b], p->stream);
                if (rc) return rc;
            }
        }
        CHEB_CUDA(cudaEventRecord(p->ev_done[b], p->stream));
        CHEB_CUDA(cudaStreamWaitEvent(p->d2h_stream, p->ev_done[b], 0));
        CHEB_CUDA(cudaMemcpyAsync(dst + (size_t)j * (size_t)out_stride, p->d_job[b], jb,
                                  cudaMemcpyDeviceToHost, p->d2h_stream));
        CHEB_CUDA(cudaEventRecord(p->ev_out[b], p->d2h_stream));
    }
    CHEB_CUDA(cudaStreamSynchronize(p->d2h_stream));
    return cheb_sync(plan);
}

// Time-dependent on-site energies: H held constant over each step (Sec. 2.2); step s first
// rescales the plan's diagonal from its own on-site array, then runs the M launches.
extern "C" int cheb_evolve_td(cheb_plan* plan, void* psi, double dt, int nsteps,
                              const double* onsite_seq, int64_t stride, int obs_every,
                              double* obs)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (p->desc.kind == CHEB_HOLSTEIN)
        return fail(CHEB_ERR_UNSUPPORTED, "cheb_evolve_td needs a lattice plan");
    if (nsteps < 0) return fail(CHEB_ERR_INVALID, "nsteps < 0");
    int rc = check_psi(p, psi);
    if (rc) return rc;
    if (nsteps == 0) return CHEB_OK;
    if (!onsite_seq) return fail(CHEB_ERR_INVALID, "cheb_evolve_td: onsite_seq is NULL");
    const int64_t per = (int64_t)p->n_sites * (p->desc.onsite_per_vec ? p->nvec : 1);
    if (nsteps > 1 && stride < per)
        return fail(CHEB_ERR_INVALID, "cheb_evolve_td: stride smaller than one on-site array");
    if (!aligned16(onsite_seq) || (nsteps > 1 && (stride & 1)))
        return fail(CHEB_ERR_ALIGN, "cheb_evolve_td: every step's array must be 16-byte aligned");
    if (obs && !aligned16(obs)) return fail(CHEB_ERR_ALIGN, "obs must be 16-byte aligned");
    rc = set_dt(p, dt);
    if (rc) return rc;
    const bool recording = obs && obs_every > 0;
    if (recording && p->prec == CHEB_C64) {
        rc = record_prepare(p);
        if (rc) return rc;
    }
    for (int s = 0; s < nsteps; ++s) {
        rc = launch_scale_diag(p, onsite_seq + (size_t)s * (size_t)stride, p->stream);
        if (rc) return rc;
        const bool rec = recording && s % obs_every == 0;
        double* slot = rec ? obs + (size_t)(s / obs_every) * p->nblocks * p->nvec * 2 : nullptr;
        if (rec && p->prec == CHEB_C64) {
            rc = launch_record(p, psi, slot, p->stream);
            if (rc) return rc;
        }
        rc = enqueue_step(p, psi, p->stream);
        if (rc) return rc;
        if (rec && p->prec == CHEB_C128) {
            CHEB_CUDA(cudaMemcpyAsync(slot, p->d_red, rec_bytes(p), cudaMemcpyDeviceToDevice,
                                      p->stream));
        }
    }
    return cheb_sync(plan);
}

extern "C" int cheb_observables(cheb_plan* plan, const void* psi, int kind, double param,
                                double* out)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p || !out) return fail(CHEB_ERR_INVALID, "cheb_observables: NULL argument");
    int rc = check_psi(p, psi);
    if (rc) return rc;
    if (!aligned16(out)) return fail(CHEB_ERR_ALIGN, "out must be 16-byte aligned");
    if (kind < CHEB_OBS_NORM2 || kind > CHEB_OBS_HOL_CHI) return fail(CHEB_ERR_INVALID, "bad kind");
    return launch_observable(p, psi, kind, param, out, p->stream);
}

extern "C" int cheb_plan_launch(const cheb_plan* plan, int* threads, int* spt, int* grid,
                                int* vpt)
{
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (threads) *threads = p->threads;
    if (spt) *spt = p->spt;
    if (p->op == OP_HOLMF) {  // tiles of threads * spt phonon configurations; NR per thread
        const int64_t units = p->hol_dph * p->nvec;
        const int64_t tile = (int64_t)p->threads * std::max(1, p->spt);
        const int64_t ntiles = (units + tile - 1) / tile;
        if (vpt) *vpt = p->holmf_variant == 2 ? 2 : 1;
        if (grid) *grid = (int)(p->grid_cap > 0 ? std::min<int64_t>(p->grid_cap, ntiles) : ntiles);
        return CHEB_OK;
    }
    if (vpt) *vpt = vpt_for(p->prec, p->nvec, p->vpt);
    if (grid) *grid = p->grid_cap > 0 ? std::min<int>(p->grid_cap, (int)p->hitems.size())
                                      : (int)p->hitems.size();
    return CHEB_OK;
}

extern "C" int64_t cheb_plan_launches(const cheb_plan* plan)
{
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    return p ? p->launches : -1;
}

// Autotuner: time one GENERAL-order launch per candidate (threads, sites/thread, grid cap)
// on the plan's own vectors and keep the fastest.
extern "C" int cheb_autotune(cheb_plan* plan)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (!p->have_dt) return fail(CHEB_ERR_STATE, "cheb_autotune: run a step (set dt) first");
    if (p->max_M < 3) return CHEB_OK;
    void* scratch = nullptr;
    CHEB_CUDA(cudaMalloc(&scratch, p->vec_bytes()));
    CHEB_CUDA(cudaMemsetAsync(scratch, 0, p->vec_bytes(), p->stream));
    CHEB_CUDA(cudaMemsetAsync(p->d_A, 0, p->vec_bytes(), p->stream));
    CHEB_CUDA(cudaMemsetAsync(p->d_B, 0, p->vec_bytes(), p->stream));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int th_c[] = {128, 256, 512};
    const int spt_c[] = {1, 2, 4};
    const int cap_c[] = {0, 4, 8, 16};
    std::vector<int> vpt_c;
    for (int v : {1, 2, 4})
        if (vpt_for(p->prec, p->nvec, v) == v && (p->op != OP_HOLMF || v == 1)) vpt_c.push_back(v);
    // matrix-free Holstein: its kernel variants (configurations per thread, register cap)
    std::vector<int> nr_c = {p->holmf_variant};
    if (p->op == OP_HOLMF) nr_c = {0, 1, 2};
    // mean time of one single-order launch: a warm-up launch timed with events; launches of
    // 0.2 ms or more are timed three more times with events, shorter ones (L2-resident
    // vectors, where launch gaps and event jitter dominate) as 16 launches captured in a graph
    // and replayed twice
    auto time_launch = [&](const RecArgs& a, float* out_ms) -> int {
        cudaEventRecord(e0, p->stream);
        int r = launch_recurrence(p, a, p->op, p->prec, p->stream);
        cudaEventRecord(e1, p->stream);
        if (r) return r;
        CHEB_CUDA(cudaEventSynchronize(e1));
        float ms0 = 0.0f;
        cudaEventElapsedTime(&ms0, e0, e1);
        if (ms0 >= 0.2f) {
            float tot = 0.0f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, p->stream);
                r = launch_recurrence(p, a, p->op, p->prec, p->stream);
                cudaEventRecord(e1, p->stream);
                if (r) return r;
                CHEB_CUDA(cudaEventSynchronize(e1));
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                tot += ms;
            }
            *out_ms = tot / 3.0f;
            return CHEB_OK;
        }
        constexpr int kRep = 16;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        CHEB_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < kRep && !r; ++i) r = launch_recurrence(p, a, p->op, p->prec, p->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
        if (!r && ce == cudaSuccess) ce = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        if (r) {
            if (ge) cudaGraphExecDestroy(ge);
            return r;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "autotune launch graph");
        cudaGraphLaunch(ge, p->stream);  // warm-up
        cudaEventRecord(e0, p->stream);
        cudaGraphLaunch(ge, p->stream);
        cudaGraphLaunch(ge, p->stream);
        cudaEventRecord(e1, p->stream);
        ce = cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaGraphExecDestroy(ge);
        if (ce != cudaSuccess) return cuda_fail(ce, "autotune launch graph");
        *out_ms = ms / (2.0f * kRep);
        return CHEB_OK;
    };
    float best = 1e30f;
    int bt = p->threads, bs = p->spt, bc = p->grid_cap, bv = p->vpt, bn = p->holmf_variant;
    struct Cand {
        float ms;
        int th, spt, cap, vpt, nr;
    };
    std::vector<Cand> cands;
    int rc = CHEB_OK;
    const int64_t launches0 = p->launches;
    for (int nr : nr_c) {
        p->holmf_variant = nr;
        for (int vpt : vpt_c) {
            for (int th : th_c) {
                if (p->op == OP_HOLMF && nr == 1 && th > 256) continue;
                for (int spt : spt_c) {
                    p->vpt = vpt;
                    p->threads = th;
                    p->spt = spt;
                    rc = plan_build_items(p);
                    if (rc) break;
                    for (int capm : cap_c) {
                        p->grid_cap = capm ? capm * p->num_sms : 0;
                        RecArgs a = base_args(p);
                        a.mode = REC_GENERAL;
                        a.j = 2;
                        a.cur = p->d_A;
                        a.prev = p->d_B;
                        a.psi = scratch;
                        float tot = 0.0f;
                        rc = time_launch(a, &tot);
                        if (rc) break;
                        cands.push_back({tot, th, spt, p->grid_cap, vpt, nr});
                        if (tot < best) {
                            best = tot;
                            bt = th;
                            bs = spt;
                            bc = p->grid_cap;
                            bv = vpt;
                            bn = nr;
                        }
                    }
                    if (rc) break;
                }
                if (rc) break;
            }
            if (rc) break;
        }
        if (rc) break;
    }
    // whole steps as cheb_evolve runs them: the step's graph replayed (one warm-up, 3 timed)
    auto time_steps = [&](float* out_ms) -> int {
        Plan::StepGraph* g = nullptr;
        int r = ensure_graph(p, scratch, &g);
        if (r) return r;
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        cudaGraphLaunch(g->exec, p->stream);
        cudaEventRecord(t0, p->stream);
        for (int rep = 0; rep < 3; ++rep) cudaGraphLaunch(g->exec, p->stream);
        cudaEventRecord(t1, p->stream);
        cudaError_t e = cudaEventSynchronize(t1);
        cudaEventElapsedTime(out_ms, t0, t1);
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        return e == cudaSuccess ? CHEB_OK : cuda_fail(e, "autotune step timing");
    };
    // a short step (small, L2-resident plans) mixes launch kinds whose best shapes differ and
    // lasts about as long as the launch gaps, and one launch's time ranks the shapes poorly:
    // there the shapes (at most 48, fastest single launch first) are compared as whole steps,
    // single-order launches only
    std::sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
    if (!rc && cands.size() > 1 && cands[0].ms * (float)p->max_M < 2.0f) {
        const int saved_s = p->tb_s, saved_cluster = p->cluster;
        p->tb_s = 0;
        p->tb_sched.clear();
        p->cluster = 0;
        float best_step = 1e30f;
        for (size_t i = 0; i < cands.size() && i < 48 && !rc; ++i) {
            const Cand& c = cands[i];
            p->threads = c.th;
            p->spt = c.spt;
            p->vpt = c.vpt;
            p->holmf_variant = c.nr;
            rc = plan_build_items(p);
            if (rc) break;
            p->grid_cap = c.cap;
            p->shape_epoch++;
            float ms = 0.0f;
            rc = time_steps(&ms);
            if (!rc && ms < best_step) {
                best_step = ms;
                bt = c.th;
                bs = c.spt;
                bc = c.cap;
                bv = c.vpt;
                bn = c.nr;
            }
        }
        p->tb_s = saved_s;
        p->cluster = saved_cluster;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->threads = bt;
    p->spt = bs;
    p->grid_cap = bc;
    p->vpt = bv;
    p->holmf_variant = bn;
    p->shape_epoch++;
    int rc2 = plan_build_items(p);
    if (rc) {
        cudaFree(scratch);
        return rc;
    }
    if (rc2) {
        cudaFree(scratch);
        return rc2;
    }
    // single-order launches against temporal blocking (complex64 stencils)
    if (tb_eligible(p)) {
        p->tb_s = 0;
        p->tb_sched.clear();
        p->shape_epoch++;
        float best_ms = 0.0f;
        rc = time_steps(&best_ms);
        int best_s = 0, best_spt = p->tb_spt, best_tpb = p->tb_tpb, best_kernel = p->tb_kernel;
        // (kernel, sites per thread, threads)
        const int shapes[][3] = {{CHEB_TB_SITES, 4, 256}, {CHEB_TB_SITES, 6, 256},
                                 {CHEB_TB_SITES, 8, 256}, {CHEB_TB_SITES, 3, 512},
                                 {CHEB_TB_SITES, 4, 512}, {CHEB_TB_SITES, 6, 512},
                                 {CHEB_TB_SITES, 2, 1024}, {CHEB_TB_SITES, 3, 1024},
                                 {CHEB_TB_SITES, 6, 1024}, {CHEB_TB_SITES, 8, 1024},
                                 {CHEB_TB_RUNS, 3, 768}, {CHEB_TB_RUNS, 3, 512},
                                 {CHEB_TB_RUNS, 5, 512}, {CHEB_TB_RUNS, 7, 384},
                                 {CHEB_TB_RUNS, 9, 256},
                                 {CHEB_TB_RUNS, 3, 1024}, {CHEB_TB_RUNS, 7, 512},
                                 {CHEB_TB_RUNS_TMA, 5, 512}, {CHEB_TB_RUNS_TMA, 7, 384},
                                 {CHEB_TB_RUNS_TMA, 9, 256}};
        for (const auto& sh : shapes) {
            if (rc) break;
            const int kern = sh[0], spt = sh[1], tpb = sh[2];
            if (tb_runs(kern) ? !tbr_supported(p->nvec, spt, tpb) : !tb_supported(p->nvec, spt, tpb))
                continue;
            if (kern == CHEB_TB_RUNS_TMA && (p->nvec < 2 || !tbr_tma_available())) continue;
            for (int s_try : {2, 3, 4, 5, 6, 7, 8, 10, 12}) {
                p->tb_s = s_try;
                p->tb_spt = spt;
                p->tb_tpb = tpb;
                p->tb_kernel = kern;
                for (TBSet& t : p->tb_sets) {  // tiles depend on the region budget (spt)
                    cudaFree(t.d_tiles);
                    cudaFree(t.d_begin);
                }
                p->tb_sets.clear();
                rc = tb_prepare(p);
                if (rc) break;
                if (p->tb_sched.empty()) continue;
                float ms = 0.0f;
                rc = time_steps(&ms);
                if (rc) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_s = s_try;
                    best_spt = spt;
                    best_tpb = tpb;
                    best_kernel = kern;
                }
            }
        }
        for (TBSet& t : p->tb_sets) {
            cudaFree(t.d_tiles);
            cudaFree(t.d_begin);
        }
        p->tb_sets.clear();
        p->tb_s = best_s;
        p->tb_spt = best_spt;
        p->tb_tpb = best_tpb;
        p->tb_kernel = best_kernel;
        int rc3 = tb_prepare(p);
        if (!rc) rc = rc3;
        CHEB_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->stream));
    }
    // whole steps: single-order launches against one cluster launch per step (small 1D grids)
    if (!rc && cluster_eligible(p)) {
        float best_ms = 0.0f;
        int best = 0;
        p->cluster = 0;
        p->shape_epoch++;
        rc = time_steps(&best_ms);
        for (int ctas : {8, 16}) {
            if (rc) break;
            if (cluster_configure(p, ctas) != CHEB_OK) continue;  // not schedulable here
            p->cluster = ctas;
            p->shape_epoch++;
            float ms = 0.0f;
            rc = time_steps(&ms);
            if (!rc && ms < best_ms) {
                best_ms = ms;
                best = ctas;
            }
        }
        p->cluster = best;
        if (!rc && best) rc = cluster_configure(p, best);  // attributes of the chosen size
        p->shape_epoch++;
        CHEB_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->stream));
    }
    p->launches = launches0;
    cudaStreamSynchronize(p->stream);
    for (Plan::StepGraph& g : p->graphs)  // graphs of the scratch buffer are not reused
        if (g.exec && g.psi == scratch) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            g.psi = nullptr;
        }
    cudaFree(scratch);
    if (rc) return rc;
    p->tuned = true;
    return CHEB_OK;
}

extern "C" int cheb_plan_sell_stats(const cheb_plan* plan, int* sigma, int64_t* stored,
                                    int64_t* offdiag)
{
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "cheb_plan_sell_stats: NULL plan");
    if (p->op != OP_SELL) return fail(CHEB_ERR_UNSUPPORTED, "cheb_plan_sell_stats: no SELL matrix");
    if (sigma) *sigma = p->sell_sigma;
    if (stored) *stored = p->sell_nnz_stored;
    if (offdiag) *offdiag = p->sell_nnz_offdiag;
    return CHEB_OK;
}

extern "C" int cheb_plan_step_model(const cheb_plan* plan, cheb_step_model* out)
{
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!p || !out) return fail(CHEB_ERR_INVALID, "cheb_plan_step_model: NULL argument");
    if (!p->have_dt) return fail(CHEB_ERR_STATE, "cheb_plan_step_model: no dt yet");
    std::memset(out, 0, sizeof(*out));
    double useful = 0.0;
    for (const DevBlock& B : p->hblocks) {
        const double sites = (p->op != OP_STENCIL) ? (double)p->n_sites : (double)B.W * B.L;
        useful += sites * B.M;
    }
    out->useful_site_orders = useful;
    if (p->cluster && cluster_eligible(p)) {
        out->computed_site_orders = useful;
        out->dram_bytes = out->l2_bytes = (double)p->n_sites * (2.0 * p->cplx_size() + p->real_size());
        out->launches = 1;
        return CHEB_OK;
    }
    if (!p->tb_sched.empty()) {
        TBModel m;
        double dram = 0.0;
        for (const Plan::TBLaunch& L : p->tb_sched) {
            std::vector<TBTile> tiles;
            std::vector<int32_t> begin;
            if (!tb_build_tiles(p, p->tb_sets[L.set].s, tiles, begin))
                return fail(CHEB_ERR_STATE, "cheb_plan_step_model: tiles");
            if (tb_runs(p->tb_kernel)) tbr_model_launch(p, tiles, L.ka, L.kb, L.prev_ka, m);
            else tb_model_launch(p, tiles, L.ka, L.kb, L.prev_ka, m);
            dram += tb_launch_bytes(p, L);
        }
        out->computed_site_orders = m.computed;
        out->smem_bytes = m.smem;
        out->l2_bytes = m.l2;
        out->dram_bytes = dram;
        out->launches = (int64_t)p->tb_sched.size();
        return CHEB_OK;
    }
    double dram = 0.0;
    for (int k = 1; k <= p->max_M; ++k) dram += launch_bytes(p, k);
    out->computed_site_orders = useful;
    out->dram_bytes = out->l2_bytes = dram;
    out->launches = p->max_M;
    return CHEB_OK;
}

extern "C" int cheb_tb_tiles(int W, int L, int orders_per_launch, int region_sites,
                             int32_t* out, int64_t capacity, int64_t* ntiles)
{
    if (!ntiles) return fail(CHEB_ERR_INVALID, "cheb_tb_tiles: NULL count");
    if (W < 1 || L < 1 || orders_per_launch < 1 || region_sites < 1)
        return fail(CHEB_ERR_INVALID, "cheb_tb_tiles: W, L, orders_per_launch, region_sites >= 1");
    if (capacity > 0 && !out) return fail(CHEB_ERR_INVALID, "cheb_tb_tiles: NULL out");
    std::vector<TBTile> tiles;
    if (!tb_tiles_of_ribbon(W, L, orders_per_launch, region_sites, 0, tiles))
        return fail(CHEB_ERR_INVALID, "cheb_tb_tiles: the ribbon does not fit the region budget");
    *ntiles = (int64_t)tiles.size();
    for (size_t i = 0; i < tiles.size() && (int64_t)i < capacity; ++i) {
        const TBTile& t = tiles[i];
        const int32_t v[8] = {t.R0, t.R1, t.C0, t.C1, t.r0, t.r1, t.c0, t.c1};
        std::memcpy(out + 8 * i, v, sizeof(v));
    }
    return CHEB_OK;
}

extern "C" int cheb_tb_tiles_padded(int W, int L, int orders_per_launch, int region_positions,
                                    int align, int boxes, int32_t* out, int64_t capacity,
                                    int64_t* ntiles)
{
    if (!ntiles) return fail(CHEB_ERR_INVALID, "cheb_tb_tiles_padded: NULL count");
    if (W < 1 || L < 1 || orders_per_launch < 1 || region_positions < 2 || (align != 4 && align != 8))
        return fail(CHEB_ERR_INVALID, "cheb_tb_tiles_padded: W, L, orders_per_launch >= 1, "
                                      "region_positions >= 2, align 4 or 8");
    if (capacity > 0 && !out) return fail(CHEB_ERR_INVALID, "cheb_tb_tiles_padded: NULL out");
    std::vector<TBTile> tiles;
    if (!tb_tiles_of_ribbon(W, L, orders_per_launch, region_positions, 0, tiles, align, boxes != 0))
        return fail(CHEB_ERR_INVALID, "cheb_tb_tiles_padded: the ribbon does not fit the region budget");
    *ntiles = (int64_t)tiles.size();
    for (size_t i = 0; i < tiles.size() && (int64_t)i < capacity; ++i) {
        const TBTile& t = tiles[i];
        const int32_t v[10] = {t.R0, t.R1, t.C0, t.C1, t.r0, t.r1, t.c0, t.c1, t.S, t.BH};
        std::memcpy(out + 10 * i, v, sizeof(v));
    }
    return CHEB_OK;
}

extern "C" int cheb_plan_export_csr(cheb_plan* plan, int64_t* rowptr, int64_t* col, double* val,
                                    int64_t* nnz_out)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p || !nnz_out) return fail(CHEB_ERR_INVALID, "cheb_plan_export_csr: NULL argument");
    if (p->op != OP_SELL) return fail(CHEB_ERR_UNSUPPORTED, "export needs a SELL (Holstein) plan");
    if (!p->d_sell_val_raw)
        return fail(CHEB_ERR_UNSUPPORTED, "plans above 2^27 rows keep no unscaled matrix copy");
    const int64_t n = p->n_sites;
    std::vector<uint8_t> rl(n);
    std::vector<double> diag(n);
    std::vector<int32_t> clen(p->sell_nchunks);
    std::vector<int64_t> coff(p->sell_nchunks + 1);
    CHEB_CUDA(cudaStreamSynchronize(p->stream));
    CHEB_CUDA(cudaMemcpy(rl.data(), p->d_hol_rowlen, n, cudaMemcpyDeviceToHost));
    CHEB_CUDA(cudaMemcpy(diag.data(), p->d_hol_diag_raw, n * sizeof(double), cudaMemcpyDeviceToHost));
    CHEB_CUDA(cudaMemcpy(clen.data(), p->d_sell_chunk_len, clen.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CHEB_CUDA(cudaMemcpy(coff.data(), p->d_sell_chunk_off, coff.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    int64_t nnz = n;
    for (int64_t i = 0; i < n; ++i) nnz += rl[i];
    *nnz_out = nnz;
    if (!rowptr || !col || !val) return CHEB_OK;
    std::vector<int32_t> scol(std::max<int64_t>(p->sell_nnz_stored, 1));
    std::vector<double> sval(std::max<int64_t>(p->sell_nnz_stored, 1));
    CHEB_CUDA(cudaMemcpy(scol.data(), p->d_sell_col, p->sell_nnz_stored * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CHEB_CUDA(cudaMemcpy(sval.data(), p->d_sell_val_raw, p->sell_nnz_stored * sizeof(double), cudaMemcpyDeviceToHost));
    // storage position of every row (the identity without sigma sorting)
    std::vector<int64_t> posof(n);
    if (p->d_sell_perm) {
        std::vector<int32_t> perm(n);
        CHEB_CUDA(cudaMemcpy(perm.data(), p->d_sell_perm, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
        for (int64_t q = 0; q < n; ++q) posof[perm[q]] = q;
    } else {
        for (int64_t q = 0; q < n; ++q) posof[q] = q;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        rowptr[i] = k;
        col[k] = i;
        val[k] = diag[i];
        ++k;
        const int64_t pos = posof[i];
        const int64_t off = coff[pos >> 5] + (pos & 31);
        for (int e = 0; e < rl[i]; ++e) {
            col[k] = scol[off + (int64_t)e * 32];
            val[k] = sval[off + (int64_t)e * 32];
            ++k;
        }
    }
    rowptr[n] = k;
    return CHEB_OK;
}

extern "C" int cheb_plan_set_timing(cheb_plan* plan, int enable)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (!enable) {
        int rc = collect_timing(p);
        if (rc) return rc;
    }
    p->timing = enable != 0;
    return CHEB_OK;
}

extern "C" int cheb_plan_kernel_stats(cheb_plan* plan, double* ms, int64_t* launches,
                                      double* bytes, int reset)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    int rc = collect_timing(p);
    if (rc) return rc;
    if (ms) *ms = p->t_ms;
    if (launches) *launches = p->t_launches;
    if (bytes) *bytes = p->t_bytes;
    if (reset) {
        p->t_ms = 0.0;
        p->t_bytes = 0.0;
        p->t_launches = 0;
    }
    return CHEB_OK;
}

extern "C" int cheb_plan_set_blocking(cheb_plan* plan, int s, int spt, int threads)
{
    return cheb_plan_set_blocking_kernel(plan, s, spt, threads, CHEB_TB_SITES);
}

extern "C" int cheb_plan_blocking_kernel(const cheb_plan* plan, int* kernel)
{
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!p || !kernel) return fail(CHEB_ERR_INVALID, "cheb_plan_blocking_kernel: NULL argument");
    *kernel = p->tb_sched.empty() ? CHEB_TB_SITES : p->tb_kernel;
    return CHEB_OK;
}

extern "C" int cheb_plan_set_blocking_kernel(cheb_plan* plan, int s, int spt, int threads,
                                             int kernel)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (s < 0 || s > 16) return fail(CHEB_ERR_INVALID, "orders_per_launch must be in [0, 16]");
    if (kernel != CHEB_TB_SITES && kernel != CHEB_TB_RUNS && kernel != CHEB_TB_RUNS_TMA)
        return fail(CHEB_ERR_INVALID,
                    "blocked kernel must be CHEB_TB_SITES, CHEB_TB_RUNS or CHEB_TB_RUNS_TMA");
    if (s > 0 && !tb_eligible(p))
        return fail(CHEB_ERR_UNSUPPORTED, "temporal blocking needs a complex64 lattice plan with "
                                          "nvec 1, 2 or 4 and a shared on-site array");
    if (s > 0 && kernel == CHEB_TB_RUNS_TMA && p->nvec < 2)
        return fail(CHEB_ERR_UNSUPPORTED, "CHEB_TB_RUNS_TMA needs pairs of vectors (nvec 2 or 4)");
    if (threads == 0) threads = 256;
    const bool ok = tb_runs(kernel) ? tbr_supported(p->nvec, spt, threads)
                                    : tb_supported(p->nvec, spt, threads);
    if (s > 0 && !ok)
        return fail(CHEB_ERR_INVALID, "temporal blocking: this (nvec, sites_per_thread, threads) "
                                      "shape is not compiled");
    for (TBSet& t : p->tb_sets) {
        cudaFree(t.d_tiles);
        cudaFree(t.d_begin);
    }
    p->tb_sets.clear();
    p->tb_s = s;
    if (s > 0) {
        p->tb_spt = spt;
        p->tb_tpb = threads;
        p->tb_kernel = kernel;
    }
    p->tb_sched.clear();
    p->shape_epoch++;
    int rc = tb_prepare(p);
    if (rc) return rc;
    if (s > 0 && p->have_dt && p->tb_sched.empty())
        return fail(CHEB_ERR_INVALID, "temporal blocking: a ribbon does not fit the tile budget");
    return CHEB_OK;
}

extern "C" int cheb_plan_set_blocking_grid(cheb_plan* plan, int ctas)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (ctas < 0) return fail(CHEB_ERR_INVALID, "cheb_plan_set_blocking_grid: ctas < 0");
    p->tb_grid_cap = ctas;
    p->shape_epoch++;  // the step graphs hold the launch shape
    return CHEB_OK;
}

extern "C" int cheb_plan_set_cluster(cheb_plan* plan, int ctas)
{
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    if (ctas != 0 && ctas != 8 && ctas != 16)
        return fail(CHEB_ERR_INVALID, "cheb_plan_set_cluster: ctas must be 0, 8 or 16");
    if (ctas && !cluster_eligible(p))
        return fail(CHEB_ERR_UNSUPPORTED, "cluster steps need a 1D grid plan (CHEB_LAT1D, nvec 1, "
                                          "shared potential) of at most 32768 points");
    if (ctas) {
        int rc = cluster_configure(p, ctas);
        if (rc) return rc;
    }
    p->cluster = ctas;
    p->shape_epoch++;
    return CHEB_OK;
}

extern "C" int cheb_plan_cluster(const cheb_plan* plan, int* ctas)
{
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!p || !ctas) return fail(CHEB_ERR_INVALID, "cheb_plan_cluster: NULL argument");
    *ctas = (p->cluster && cluster_eligible(p)) ? p->cluster : 0;
    return CHEB_OK;
}

extern "C" int cheb_plan_blocking(const cheb_plan* plan, int* s, int* spt, int* threads)
{
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!p) return fail(CHEB_ERR_INVALID, "NULL plan");
    const bool on = p->tb_s > 0 && tb_eligible(p);
    if (s) *s = on ? p->tb_s : 0;
    if (spt) *spt = on ? p->tb_spt : 0;
    if (threads) *threads = on ? p->tb_tpb : 0;
    return CHEB_OK;
}
