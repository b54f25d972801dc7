"""Temporally blocked recurrence (several orders per launch out of shared memory) against
the oracle and against single-order launches, on ensembles with edge shapes: 1D chains
(W = 1), single sites, ribbons shorter than the halo, widths above one 48-row band, and
per-ribbon orders M from 2 up."""
import numpy as np
import pytest

import workloads as wl
from _gpu_util import C64, dev_f64, dev_vec, host, oracle_ribbon, rel

pytestmark = pytest.mark.gpu

SIZES = [(1, 300), (1, 1), (3, 5), (50, 60), (97, 41), (7, 230), (130, 30), (2, 3)]


def _plan(cb, ens, nvec):
    W = [w for w, _ in ens.sizes]
    L = [l for _, l in ens.sizes]
    eps = dev_f64(ens.onsite())
    desc, keep = cb.desc_ribbons(W, L, ens.hop, eps)
    lo, hi = ens.bounds()
    return cb.Plan(desc, lo, hi, 0.0, cb.CHEB_C64, nvec, keep=keep)


@pytest.mark.parametrize("nvec", [4, 2, 1])
@pytest.mark.parametrize("s,spt", [(1, 4), (2, 4), (3, 6), (4, 4), (7, 4), (5, 8)])
def test_blocked_matches_oracle_and_single_order(nvec, s, spt):
    import paper_0907_3022_gb300 as cb

    if spt == 8 and nvec == 4:
        pytest.skip("sites_per_thread 8 needs nvec <= 2")
    ens = wl.RibbonEnsemble(n_ribbons=len(SIZES), sizes=list(SIZES), sigma=4.0,
                            k0s=wl.ENSEMBLE_K0[:nvec])
    nsteps = 7
    x0 = dev_vec(ens.packets(), C64)
    ref_plan = _plan(cb, ens, nvec)
    a = x0.clone()
    ref_plan.evolve(a, ens.dt, nsteps)
    plan = _plan(cb, ens, nvec)
    plan.evolve(x0, ens.dt, 0)
    plan.set_blocking(s, spt)
    assert plan.blocking() == (s, spt)
    b = x0.clone()
    plan.evolve(b, ens.dt, nsteps)
    out_a, out_b = host(a), host(b)
    assert rel(out_b, out_a) <= 2e-6
    off = ens.offsets()
    for r in range(ens.n_ribbons):
        W, L = ens.sizes[r]
        for v, k0 in enumerate(ens.k0s):
            ref, M = oracle_ribbon(W, L, ens.disorder(r), ens.seed, r, k0, nsteps, sigma=4.0)
            assert rel(out_b[off[r]:off[r + 1], v], ref) <= 1e-4, (r, v)


@pytest.mark.parametrize("nvec,spt,threads", [(4, 3, 512), (4, 4, 512), (4, 6, 512),
                                               (4, 2, 1024), (4, 3, 1024), (2, 6, 1024),
                                               (1, 8, 1024)])
@pytest.mark.parametrize("s", [3, 6])
def test_blocked_large_ctas(nvec, spt, threads, s):
    """CTAs of 512 and 1024 threads (one large region per SM): same results as single-order
    launches and the oracle on the edge-shape ensemble."""
    import paper_0907_3022_gb300 as cb

    ens = wl.RibbonEnsemble(n_ribbons=len(SIZES), sizes=list(SIZES), sigma=4.0,
                            k0s=wl.ENSEMBLE_K0[:nvec])
    nsteps = 5
    x0 = dev_vec(ens.packets(), C64)
    ref_plan = _plan(cb, ens, nvec)
    a = x0.clone()
    ref_plan.evolve(a, ens.dt, nsteps)
    plan = _plan(cb, ens, nvec)
    plan.evolve(x0, ens.dt, 0)
    plan.set_blocking(s, spt, threads)
    assert plan.blocking_shape() == (s, spt, threads)
    b = x0.clone()
    plan.evolve(b, ens.dt, nsteps)
    out_a, out_b = host(a), host(b)
    assert rel(out_b, out_a) <= 2e-6
    off = ens.offsets()
    for r in (0, 3, 4, 6):
        W, L = ens.sizes[r]
        ref, M = oracle_ribbon(W, L, ens.disorder(r), ens.seed, r, ens.k0s[0], nsteps, sigma=4.0)
        assert rel(out_b[off[r]:off[r + 1], 0], ref) <= 1e-4, r
    with pytest.raises(cb.ChebError) as e:  # a shape that is not compiled
        plan.set_blocking(s, 5, threads)
    assert e.value.status == cb.CHEB_ERR_INVALID


def test_blocked_small_orders_and_observables():
    """dt = 0.001 gives M of about 5 per ribbon: with 6 orders per launch the first launch is
    cut to M_min - 1 orders and every ribbon's last order falls inside the second launch."""
    import torch

    import paper_0907_3022_gb300 as cb

    ens = wl.RibbonEnsemble(n_ribbons=4, sizes=[(5, 40), (60, 33), (1, 70), (9, 9)], sigma=4.0,
                            dt=0.001)
    plan = _plan(cb, ens, 4)
    x0 = dev_vec(ens.packets(), C64)
    plan.evolve(x0, ens.dt, 0)
    Ms = [plan.block(q)["M"] for q in range(4)]
    assert min(Ms) <= 6
    plan.set_blocking(6, 4)
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
            assert M == Ms[r]
            assert rel(out[off[r]:off[r + 1], v], ref) <= 1e-4
    r = rec.cpu().numpy()
    assert np.max(np.abs(r[:, :, :, 0] - 1.0)) <= 1e-5


def test_blocking_rejected_where_unsupported():
    import paper_0907_3022_gb300 as cb

    ens = wl.RibbonEnsemble(n_ribbons=2, sizes=[(4, 10), (5, 12)])
    W = [w for w, _ in ens.sizes]
    L = [l for _, l in ens.sizes]
    eps = dev_f64(ens.onsite())
    desc, keep = cb.desc_ribbons(W, L, 1.0, eps)
    p128 = cb.Plan(desc, *ens.bounds(), 0.0, cb.CHEB_C128, 1, keep=keep)
    with pytest.raises(cb.ChebError) as e:
        p128.set_blocking(4, 4)
    assert e.value.status == cb.CHEB_ERR_UNSUPPORTED
    p64 = cb.Plan(desc, *ens.bounds(), 0.0, cb.CHEB_C64, 4, keep=keep)
    with pytest.raises(cb.ChebError) as e:
        p64.set_blocking(4, 8)
    assert e.value.status == cb.CHEB_ERR_INVALID
