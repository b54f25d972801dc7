"""The register-run blocked kernel (CHEB_TB_RUNS, and CHEB_TB_RUNS_TMA with its inputs staged
by tensor-memory-access boxes) against the FP64 oracle and against single-order launches, at
every compiled shape, on ensembles with edge shapes: 1D chains (W = 1), a single site, ribbons
shorter than the halo, and widths and lengths that leave ragged last bands, columns and runs.
Interior sites of every tile keep all orders of a launch valid; halo sites, pads and runs that
straddle rows must never leak into them.

The two variants form every interior site's T_k from the same neighbour values in the same
order, whatever the tiles, so their results must be equal bit for bit."""
import numpy as np
import pytest

import workloads as wl
from _gpu_util import C64, dev_f64, dev_vec, host, oracle_ribbon, rel

pytestmark = pytest.mark.gpu

SIZES = [(1, 300), (1, 1), (3, 5), (50, 60), (97, 41), (7, 230), (130, 30), (2, 3), (61, 257)]
PAIR_SHAPES = [(3, 768), (3, 512), (5, 512), (7, 384), (9, 256)]
SINGLE_SHAPES = [(3, 1024), (5, 512), (7, 512)]


def _plan(cb, ens, nvec):
    W = [w for w, _ in ens.sizes]
    L = [l for _, l in ens.sizes]
    desc, keep = cb.desc_ribbons(W, L, ens.hop, dev_f64(ens.onsite()))
    lo, hi = ens.bounds()
    return cb.Plan(desc, lo, hi, 0.0, cb.CHEB_C64, nvec, keep=keep)


def _cases():
    out = []
    for nvec in (4, 2):
        for run, tpb in PAIR_SHAPES:
            out.append((nvec, run, tpb, 1))
            out.append((nvec, run, tpb, 2))
    for run, tpb in SINGLE_SHAPES:
        out.append((1, run, tpb, 1))
    return out


@pytest.mark.parametrize("s", [3, 6, 10])
@pytest.mark.parametrize("nvec,run,tpb,kernel", _cases())
def test_runs_match_oracle_and_single_order(nvec, run, tpb, kernel, s):
    import paper_0907_3022_gb300 as cb

    ens = wl.RibbonEnsemble(n_ribbons=len(SIZES), sizes=list(SIZES), sigma=4.0,
                            k0s=wl.ENSEMBLE_K0[:nvec])
    x = ens.packets()
    off = ens.offsets()
    # the last vector is a random state on every ribbon: every tile border carries amplitude
    for r in range(ens.n_ribbons):
        x[off[r]:off[r + 1], nvec - 1] = wl.random_state(int(off[r + 1] - off[r]), 99, r)
    nsteps = 6
    x0 = dev_vec(x, C64)
    ref_plan = _plan(cb, ens, nvec)
    a = x0.clone()
    ref_plan.evolve(a, ens.dt, nsteps)
    plan = _plan(cb, ens, nvec)
    plan.evolve(x0, ens.dt, 0)
    plan.set_blocking_kernel(s, run, tpb, kernel)
    assert plan.blocking_shape() == (s, run, tpb) and plan.blocking_kernel() == kernel
    b = x0.clone()
    plan.evolve(b, ens.dt, nsteps)
    out_a, out_b = host(a), host(b)
    assert rel(out_b, out_a) <= 2e-6
    if kernel == cb.CHEB_TB_RUNS_TMA:  # the same results as the per-thread copies, bit for bit
        plan.set_blocking_kernel(s, run, tpb, cb.CHEB_TB_RUNS)
        c = x0.clone()
        plan.evolve(c, ens.dt, nsteps)
        assert np.array_equal(host(c), out_b)
    import oracle

    for r in range(ens.n_ribbons):
        rb = ens.ribbon(r)
        H = oracle.honeycomb(rb.W, rb.L, rb.hop, rb.onsite())
        aa, bb = oracle.rescale(*rb.bounds(), 0.0)
        C, M = oracle.coeffs(aa, bb, rb.dt)
        for v in range(nvec):
            ref = H.evolve(aa, bb, C, nsteps, x[off[r]:off[r + 1], v])
            g = out_b[off[r]:off[r + 1], v]
            assert rel(g, ref) <= 1e-4, (r, v, rel(g, ref))
            assert np.max(np.abs(g - ref)) <= 1e-4 * np.max(np.abs(ref)), (r, v)
    plan.close()
    ref_plan.close()


@pytest.mark.parametrize("kernel,run,tpb", [(1, 7, 384), (2, 7, 384), (1, 3, 768), (0, 6, 512)])
def test_blocked_grid_does_not_change_results(kernel, run, tpb):
    """Every CTA of a blocked launch works through tiles i, i + grid, ...; with 1, 3 and 7
    CTAs each CTA runs many tiles in a row (the register-run kernel copying each next tile's
    inputs during the current one's orders), with the default grid the results must be the
    same bit for bit: a tile's arithmetic does not depend on which CTA runs it."""
    import paper_0907_3022_gb300 as cb

    ens = wl.RibbonEnsemble(n_ribbons=len(SIZES), sizes=list(SIZES), sigma=4.0,
                            k0s=wl.ENSEMBLE_K0[:4])
    x = ens.packets()
    off = ens.offsets()
    for r in range(ens.n_ribbons):
        x[off[r]:off[r + 1], 3] = wl.random_state(int(off[r + 1] - off[r]), 31, r)
    x0 = dev_vec(x, C64)
    plan = _plan(cb, ens, 4)
    plan.evolve(x0, ens.dt, 0)
    plan.set_blocking_kernel(6, run, tpb, kernel)
    outs = []
    for ctas in (0, 1, 3, 7):
        plan.set_blocking_grid(ctas)
        b = x0.clone()
        plan.evolve(b, ens.dt, 4)
        outs.append(host(b))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    with pytest.raises(cb.ChebError) as e:
        plan.set_blocking_grid(-1)
    assert e.value.status == cb.CHEB_ERR_INVALID
    plan.close()


def test_runs_small_orders_records_and_growth_check():
    """dt = 0.001 (M of about 5): the first launch is cut below min M and every ribbon ends
    inside the second; records every 10 steps; then bounds far too tight must trip the
    growth check."""
    import torch

    import paper_0907_3022_gb300 as cb

    ens = wl.RibbonEnsemble(n_ribbons=4, sizes=[(5, 40), (60, 33), (1, 70), (9, 9)], sigma=4.0,
                            dt=0.001)
    plan = _plan(cb, ens, 4)
    x0 = dev_vec(ens.packets(), C64)
    plan.evolve(x0, ens.dt, 0)
    plan.set_blocking_kernel(6, 3, 768, cb.CHEB_TB_RUNS)
    b = x0.clone()
    rec = torch.zeros((3, 4, 4, 2), dtype=torch.float64, device="cuda:0")
    plan.evolve(b, ens.dt, 30, 10, rec)
    out = host(b)
    off = ens.offsets()
    for r in range(4):
        W, L = ens.sizes[r]
        for v, k0 in enumerate(ens.k0s):
            ref, M = oracle_ribbon(W, L, ens.disorder(r), ens.seed, r, k0, 30, sigma=4.0,
                                   dt=ens.dt)
            assert rel(out[off[r]:off[r + 1], v], ref) <= 1e-4
    assert np.max(np.abs(rec.cpu().numpy()[:, :, :, 0] - 1.0)) <= 1e-5
    plan.close()
    # spectrum far outside the bounds: |T_M| grows like cosh, the check fires
    W, L = 8, 64
    rb = wl.Ribbon(W=W, L=L, sigma=4.0)
    desc, keep = cb.desc_ribbons([W], [L], 1.0, dev_f64(rb.onsite()))
    tight = cb.Plan(desc, [-1.0], [1.0], 0.0, cb.CHEB_C64, 2, keep=keep)
    x = dev_vec(np.stack([rb.packet(), rb.packet()], axis=1), C64)
    tight.evolve(x, 4.0, 0)
    tight.set_blocking_kernel(4, 3, 512, cb.CHEB_TB_RUNS)
    with pytest.raises(cb.ChebError) as e:
        tight.evolve(x, 4.0, 3)
    assert e.value.status == cb.CHEB_ERR_DIVERGED
    tight.close()


def test_runs_shape_errors():
    import paper_0907_3022_gb300 as cb

    ens = wl.RibbonEnsemble(n_ribbons=2, sizes=[(4, 10), (5, 12)])
    plan = _plan(cb, ens, 4)
    with pytest.raises(cb.ChebError) as e:  # run 3 with 1024 threads is compiled for nvec 1 only
        plan.set_blocking_kernel(4, 3, 1024, cb.CHEB_TB_RUNS)
    assert e.value.status == cb.CHEB_ERR_INVALID
    with pytest.raises(cb.ChebError) as e:
        plan.set_blocking_kernel(4, 3, 768, 7)
    assert e.value.status == cb.CHEB_ERR_INVALID
    plan.close()
    one = _plan(cb, ens, 1)
    with pytest.raises(cb.ChebError) as e:  # boxes carry pairs of vectors only
        one.set_blocking_kernel(4, 7, 512, cb.CHEB_TB_RUNS_TMA)
    assert e.value.status == cb.CHEB_ERR_UNSUPPORTED
    one.close()


def test_runs_tma_boxes_follow_the_state_vector():
    """The first launch of a step reads psi through tensor maps made for psi's address: direct
    steps (one map slot, rewritten when psi changes) and graph-replayed evolve calls on six
    vectors (more than the plan's four graph slots, so slots are evicted and their maps
    rewritten), interleaved, against the per-thread-copy kernel doing the same calls."""
    import paper_0907_3022_gb300 as cb

    ens = wl.RibbonEnsemble(n_ribbons=len(SIZES), sizes=list(SIZES), sigma=4.0,
                            k0s=wl.ENSEMBLE_K0[:4])
    off = ens.offsets()
    xs = []
    for j in range(6):
        x = ens.packets()
        for r in range(ens.n_ribbons):
            x[off[r]:off[r + 1], j % 4] = wl.random_state(int(off[r + 1] - off[r]), 500 + j, r)
        xs.append(x)
    calls = [(0, "e", 2), (1, "s", 1), (2, "e", 1), (0, "s", 1), (3, "e", 2), (4, "e", 1),
             (5, "e", 1), (1, "e", 2), (0, "e", 1), (2, "s", 1), (5, "s", 1), (3, "e", 1)]
    outs = {}
    for kernel in (cb.CHEB_TB_RUNS, cb.CHEB_TB_RUNS_TMA):
        plan = _plan(cb, ens, 4)
        psis = [dev_vec(x, C64) for x in xs]
        plan.evolve(psis[0], ens.dt, 0)
        plan.set_blocking_kernel(10, 7, 384, kernel)
        for j, kind, n in calls:
            if kind == "s":
                plan.step(psis[j], ens.dt)
            else:
                plan.evolve(psis[j], ens.dt, n)
        outs[kernel] = [host(p) for p in psis]
        plan.close()
    for j in range(6):
        assert np.array_equal(outs[cb.CHEB_TB_RUNS_TMA][j], outs[cb.CHEB_TB_RUNS][j]), j
