"""Whole steps of a 1D grid on a thread-block cluster (all M orders of Eq. U_1 in one launch,
chunk borders through distributed shared memory) against single-order launches, the oracle
and full diagonalisation; sizes from 2 points to the 32768-point limit."""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu_util import C64, C128, dev_f64, dev_vec, host, rel

pytestmark = pytest.mark.gpu


def _grid(n):
    d = wl.DoubleWell1D(n=n, x_lo=-8.0, x_hi=8.0)
    return d


@pytest.mark.parametrize("ctas", [8, 16])
@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("n", [2, 5, 33, 257, 2048, 4100, 32768])
def test_cluster_steps_equal_single_order_launches(prec, n, ctas):
    import paper_0907_3022_gb300 as cb

    d = _grid(n)
    V = dev_f64(d.potential())
    lo, hi = d.bounds()
    dt = 0.002 if n > 1000 else 0.5  # keeps M (~ a dt, a ~ 1/dx^2) in the thousands
    nsteps = 3
    ref_plan = cb.Plan(cb.desc_lat1d(d.n, d.dx, V), [lo], [hi], 0.01, prec, 1, keep=(V,))
    a = dev_vec(d.packet(), prec)
    ref_plan.evolve(a, dt, nsteps)
    plan = cb.Plan(cb.desc_lat1d(d.n, d.dx, V), [lo], [hi], 0.01, prec, 1, keep=(V,))
    try:
        plan.set_cluster(ctas)
    except cb.ChebError as e:  # a 16-CTA cluster is a non-portable size
        assert ctas == 16 and e.status == cb.CHEB_ERR_UNSUPPORTED
        pytest.skip("16-CTA clusters cannot be scheduled on this device")
    assert plan.cluster() == ctas
    b = dev_vec(d.packet(), prec)
    n0 = plan.launches()
    plan.evolve(b, dt, nsteps)
    assert plan.launches() - n0 == nsteps  # one launch per step
    assert rel(host(b), host(a)) <= (1e-13 if prec == C128 else 2e-5)
    if n <= 4100:
        aa, bb = oracle.rescale(lo, hi, 0.01)
        C, M = oracle.coeffs(aa, bb, dt)
        ref = oracle.lattice1d(d.n, d.dx, d.potential()).evolve(aa, bb, C, nsteps, d.packet())
        assert plan.block(0)["M"] == M
        assert rel(host(b), ref) <= (1e-12 if prec == C128 else 1e-4)


def test_cluster_paper_double_well_and_step_observables():
    """Sec. 3.1 (1500 moments, t = 40) on the cluster path: within 2e-11 of full
    diagonalisation; the norm and energy recorded at the start of every step match the
    oracle's."""
    import torch
    from scipy.linalg import eigh_tridiagonal

    import paper_0907_3022_gb300 as cb

    d = wl.PaperDoubleWell()
    lo, hi = d.bounds()
    V = dev_f64(d.potential())
    plan = cb.Plan(cb.desc_lat1d(d.n, d.dx, V), [lo], [hi], 0.01, C128, 1, keep=(V,))
    plan.set_cluster(8)
    psi = dev_vec(d.packet(), C128)
    obs = torch.zeros((d.nsteps, 1, 1, 2), dtype=torch.float64, device="cuda:0")
    plan.evolve(psi, d.dt, d.nsteps, obs_every=1, obs=obs)
    dd, ee = d.tridiagonal()
    E, U = eigh_tridiagonal(dd, ee)
    ex = U @ (np.exp(-1j * E * d.t_end) * (U.T @ d.packet()))
    assert np.max(np.abs(host(psi) - ex)) / math.sqrt(d.dx) < 2e-11
    H = oracle.lattice1d(d.n, d.dx, d.potential())
    n2, e0 = H.norm_energy(d.packet())
    o = obs.cpu().numpy()
    assert abs(o[0, 0, 0, 0] - n2) <= 1e-13 and abs(o[0, 0, 0, 1] - e0) <= 1e-11
    assert np.max(np.abs(o[:, 0, 0, 1] - e0)) <= 1e-9  # energy conserved step to step


def test_cluster_unsupported_and_growth_check():
    import paper_0907_3022_gb300 as cb

    d = _grid(64)
    V = dev_f64(d.potential())
    lo, hi = d.bounds()
    p2 = cb.Plan(cb.desc_lat1d(d.n, d.dx, V), [lo], [hi], 0.01, C128, 2, keep=(V,))
    with pytest.raises(cb.ChebError) as e:
        p2.set_cluster(8)
    assert e.value.status == cb.CHEB_ERR_UNSUPPORTED
    big = _grid(32770)
    Vb = dev_f64(big.potential())
    pb = cb.Plan(cb.desc_lat1d(big.n, big.dx, Vb), [0.0], [1e5], 0.01, C128, 1, keep=(Vb,))
    with pytest.raises(cb.ChebError) as e:
        pb.set_cluster(8)
    assert e.value.status == cb.CHEB_ERR_UNSUPPORTED
    rb = wl.Ribbon(W=4, L=20)
    eps = dev_f64(rb.onsite())
    desc, keep = cb.desc_ribbons([rb.W], [rb.L], 1.0, eps)
    pr = cb.Plan(desc, [rb.bounds()[0]], [rb.bounds()[1]], 0.0, C128, 1, keep=keep)
    with pytest.raises(cb.ChebError) as e:
        pr.set_cluster(8)
    assert e.value.status == cb.CHEB_ERR_UNSUPPORTED
    with pytest.raises(cb.ChebError) as e:
        cb.Plan(cb.desc_lat1d(d.n, d.dx, V), [lo], [hi], 0.01, C128, 1, keep=(V,)).set_cluster(4)
    assert e.value.status == cb.CHEB_ERR_INVALID
    # bounds far too tight: the recurrence grows and the step reports it
    tight = cb.Plan(cb.desc_lat1d(d.n, d.dx, V), [lo], [lo + 0.1 * (hi - lo)], 0.0, C128, 1,
                    keep=(V,))
    tight.set_cluster(8)
    psi = dev_vec(d.packet(), C128)
    with pytest.raises(cb.ChebError) as e:
        tight.evolve(psi, 0.5, 2)
    assert e.value.status == cb.CHEB_ERR_DIVERGED


@pytest.mark.parametrize("prec", [C128, C64])
def test_cluster_after_autotune_and_switching_sizes(prec):
    """The tuner tries every cluster size; whatever it keeps, and any size set afterwards,
    must launch (the kernel attributes follow the size in use)."""
    import paper_0907_3022_gb300 as cb

    d = wl.PaperDoubleWell()
    lo, hi = d.bounds()
    V = dev_f64(d.potential())
    plan = cb.Plan(cb.desc_lat1d(d.n, d.dx, V), [lo], [hi], 0.01, prec, 1, keep=(V,))
    psi = dev_vec(d.packet(), prec)
    plan.evolve(psi, d.dt, 0)
    plan.autotune()
    plan.step(psi, d.dt)
    plan.evolve(psi, d.dt, 2)
    for c in (16, 8, 0, 8):
        try:
            plan.set_cluster(c)
        except cb.ChebError as e:
            assert c == 16 and e.status == cb.CHEB_ERR_UNSUPPORTED
            continue
        plan.evolve(psi, d.dt, 1)
        plan.step(psi, d.dt)
    plan.sync()
