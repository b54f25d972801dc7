"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Tolerances: complex128 relative L2 <= 1e-10 after the full evolution; complex64 relative L2
<= 1e-4 and norm drift <= 1e-5 (per vector, FP64 reduction); integer work (Holstein basis
and matrix structure) bit-exact.  Sizes span several work tiles with ragged tails, plus the
full configurations in the launch shapes the benchmark uses.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu_util import C64, C128, dev_f64, dev_vec, host, oracle_1d, oracle_ribbon, rel

pytestmark = pytest.mark.gpu


def _cb():
    import paper_0907_3022_gb300 as cb

    return cb


TOL = {C128: 1e-10, C64: 1e-4}


# ---------------------------------------------------------------------------------------
# 1D double well (Sec. 3.1): N = 256 (ED-checked size) and the full N = 2048 grid
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [256, 2048])
def test_double_well_1d(n):
    cb = _cb()
    d = wl.DoubleWell1D(n=n)
    lo, hi = d.bounds()
    V = dev_f64(d.potential())
    plan = cb.Plan(cb.desc_lat1d(n, d.dx, V), [lo], [hi], 0.01, cb.CHEB_C128, 1, keep=(V,))
    psi = dev_vec(d.packet(), C128)
    plan.evolve(psi, d.dt, d.nsteps)
    ref, M = oracle_1d(n)
    assert plan.block(0)["M"] == M
    assert rel(host(psi), ref) <= TOL[C128]


# ---------------------------------------------------------------------------------------
# zigzag ribbons (Sec. 3.2)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("W,L,nsteps", [(24, 100, 30), (1, 333, 20), (7, 1, 10), (5, 257, 25)])
def test_ribbon_small(prec, W, L, nsteps):
    cb = _cb()
    rb = wl.Ribbon(W=W, L=L, sigma=6.0)
    eps = dev_f64(rb.onsite())
    desc, keep = cb.desc_ribbons([W], [L], 1.0, eps)
    lo, hi = rb.bounds()
    plan = cb.Plan(desc, [lo], [hi], 0.0, prec, 1, keep=keep)
    psi = dev_vec(rb.packet(), prec)
    plan.evolve(psi, rb.dt, nsteps)
    ref, M = oracle_ribbon(W, L, rb.disorder, rb.seed, 0, rb.k0, nsteps, sigma=6.0)
    assert plan.block(0)["M"] == M
    assert rel(host(psi), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [C128, C64])
def test_ribbon_full_configuration(prec):
    """128 x 2048 zigzag ribbon, W = 1, packet sigma = 20, k0 = pi/3, dt = 1, 400 steps."""
    cb = _cb()
    import torch

    rb = wl.Ribbon()
    eps = dev_f64(rb.onsite())
    desc, keep = cb.desc_ribbons([rb.W], [rb.L], rb.hop, eps)
    lo, hi = rb.bounds()
    plan = cb.Plan(desc, [lo], [hi], 0.0, prec, 1, keep=keep)
    psi = dev_vec(rb.packet(), prec)
    obs = torch.zeros((rb.nsteps // 50, 1, 1, 2), dtype=torch.float64, device="cuda:0")
    plan.evolve(psi, rb.dt, rb.nsteps, 50, obs)
    ref, M = oracle_ribbon(rb.W, rb.L, rb.disorder, rb.seed, 0, rb.k0, rb.nsteps)
    assert rel(host(psi), ref) <= TOL[prec]
    n2 = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_NORM2, 0.0, n2)
    drift = abs(float(n2.item()) - 1.0)
    assert drift <= (1e-12 if prec == C128 else 1e-5)
    o = obs.cpu().numpy()[:, 0, 0]
    assert np.max(np.abs(o[:, 0] - 1.0)) <= (1e-12 if prec == C128 else 1e-5)
    assert np.max(np.abs(o[:, 1] - o[0, 1])) <= (1e-11 if prec == C128 else 1e-4)


# ---------------------------------------------------------------------------------------
# batched ensembles of uneven ribbons, several packets per ribbon
# ---------------------------------------------------------------------------------------
def _ensemble_run(ens, prec, nsteps, autotune=False):
    cb = _cb()
    W = [w for w, _ in ens.sizes]
    L = [l for _, l in ens.sizes]
    eps = dev_f64(ens.onsite())
    desc, keep = cb.desc_ribbons(W, L, ens.hop, eps)
    lo, hi = ens.bounds()
    plan = cb.Plan(desc, lo, hi, 0.0, prec, ens.nvec, keep=keep)
    psi = dev_vec(ens.packets(), prec)
    if autotune:
        plan.evolve(psi, ens.dt, 0)
        plan.autotune()
    plan.evolve(psi, ens.dt, nsteps)
    return plan, psi


@pytest.mark.parametrize("prec", [C128, C64])
def test_ensemble_small_all_ribbons(prec):
    ens = wl.RibbonEnsemble(n_ribbons=5, sizes=[(3, 40), (8, 71), (1, 130), (12, 33), (5, 5)],
                            sigma=5.0)
    nsteps = 15
    plan, psi = _ensemble_run(ens, prec, nsteps)
    out = host(psi)
    off = ens.offsets()
    for r in range(ens.n_ribbons):
        W, L = ens.sizes[r]
        for v, k0 in enumerate(ens.k0s):
            ref, M = oracle_ribbon(W, L, ens.disorder(r), ens.seed, r, k0, nsteps, sigma=5.0)
            assert plan.block(r)["M"] == M
            assert rel(out[off[r]:off[r + 1], v], ref) <= TOL[prec], (r, v)


def test_ensemble_full_configuration_sampled():
    """64 uneven ribbons x 4 packets, complex64, 200 steps, tuned launch shape: the two
    smallest ribbons against the oracle for every packet; every (ribbon, packet) norm."""
    cb = _cb()
    import torch

    ens = wl.RibbonEnsemble()
    plan, psi = _ensemble_run(ens, C64, ens.nsteps, autotune=True)
    n2 = torch.zeros((ens.n_ribbons, ens.nvec), dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_NORM2, 0.0, n2)
    assert float((n2 - 1.0).abs().max()) <= 1e-5
    out = host(psi)
    off = ens.offsets()
    order = np.argsort([w * l for w, l in ens.sizes])[:2]
    for r in order:
        W, L = ens.sizes[r]
        for v, k0 in enumerate(ens.k0s):
            ref, M = oracle_ribbon(W, L, ens.disorder(r), ens.seed, int(r), k0, ens.nsteps)
            assert plan.block(int(r))["M"] == M
            assert rel(out[off[r]:off[r + 1], v], ref) <= TOL[C64], (r, v)


# ---------------------------------------------------------------------------------------
# Holstein polaron (Sec. 3.3)
# ---------------------------------------------------------------------------------------
def _holstein_plan(hs, prec, nvec=1):
    cb = _cb()
    desc = cb.desc_holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g)
    lo, hi = hs.bounds()
    return cb.Plan(desc, [lo], [hi], hs.alpha, prec, nvec)


def _sorted_rows(rp, col, val):
    rows = []
    for i in range(len(rp) - 1):
        seg = sorted(zip(col[rp[i]:rp[i + 1]].tolist(), val[rp[i]:rp[i + 1]].tolist()))
        rows.append(seg)
    return rows


@pytest.mark.parametrize("L,nph,periodic", [(4, 3, True), (5, 4, False), (3, 6, True), (1, 7, False)])
def test_holstein_matrix_bit_exact(L, nph, periodic):
    hs = wl.Holstein(L=L, nph=nph, periodic=periodic)
    plan = _holstein_plan(hs, C128)
    rp, col, val = plan.export_csr()
    H = oracle.holstein(L, nph, periodic, hs.hop, hs.omega0, hs.g)
    orp, ocol, oval = H.csr()
    assert _sorted_rows(rp, col, val) == _sorted_rows(orp, ocol, oval)


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("L,nph,periodic,nsteps", [(4, 3, True, 40), (6, 4, True, 30), (5, 3, False, 20)])
def test_holstein_small(prec, L, nph, periodic, nsteps):
    cb = _cb()
    import torch

    hs = wl.Holstein(L=L, nph=nph, periodic=periodic)
    plan = _holstein_plan(hs, prec)
    psi = dev_vec(hs.initial_state(), prec)
    plan.evolve(psi, hs.dt, nsteps)
    H = oracle.holstein(L, nph, periodic, hs.hop, hs.omega0, hs.g)
    a, b = oracle.rescale(*hs.bounds(), hs.alpha)
    C, M = oracle.coeffs(a, b, hs.dt)
    ref = H.evolve(a, b, C, nsteps, hs.initial_state())
    assert plan.block(0)["M"] == M
    assert rel(host(psi), ref) <= TOL[prec]
    dens, phon, chi = H.observables(ref)
    tol = 1e-11 if prec == C128 else 1e-5
    for kind, r in ((cb.CHEB_OBS_HOL_DENSITY, dens), (cb.CHEB_OBS_HOL_PHONON, phon),
                    (cb.CHEB_OBS_HOL_CHI, chi)):
        out = torch.zeros(L, dtype=torch.float64, device="cuda:0")
        plan.observables(psi, kind, 0.0, out)
        assert np.max(np.abs(out.cpu().numpy() - r)) <= tol, kind
    e = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, e)
    assert abs(float(e.item()) - H.norm_energy(ref)[1]) <= (1e-10 if prec == C128 else 1e-4)


def test_holstein_full_configuration():
    """L = 12 periodic, nph <= 10 (D = 7,759,752): matrix bit-exact against the oracle's
    brute-force basis; one step in complex128 against the oracle; 200 steps conserve norm
    and energy; complex64 one step within 1e-4."""
    cb = _cb()
    import torch

    hs = wl.Holstein()
    plan = _holstein_plan(hs, C128)
    assert plan.sites == 7_759_752
    H = oracle.holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g)
    rp, col, val = plan.export_csr()
    orp, ocol, oval = H.csr()
    assert np.array_equal(rp, orp)
    # rows list entries in the same order in both codes: diagonal, hops, phonon up, down
    assert np.array_equal(col, ocol) and np.array_equal(val, oval)
    a, b = oracle.rescale(*hs.bounds(), hs.alpha)
    C, M = oracle.coeffs(a, b, hs.dt)
    ref1 = H.step(a, b, C, hs.initial_state())
    psi = dev_vec(hs.initial_state(), C128)
    plan.evolve(psi, hs.dt, 1)
    assert rel(host(psi), ref1) <= 1e-12
    e0 = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, e0)
    plan.evolve(psi, hs.dt, hs.nsteps - 1)
    n2 = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    e1 = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_NORM2, 0.0, n2)
    plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, e1)
    assert abs(float(n2.item()) - 1.0) <= 1e-11
    assert abs(float(e1.item()) - float(e0.item())) <= 1e-10
    dens = torch.zeros(hs.L, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_HOL_DENSITY, 0.0, dens)
    assert abs(float(dens.sum()) - 1.0) <= 1e-11
    plan.close()
    p64 = _holstein_plan(hs, C64)
    psi = dev_vec(hs.initial_state(), C64)
    p64.evolve(psi, hs.dt, 1)
    assert rel(host(psi), ref1) <= 1e-4


# ---------------------------------------------------------------------------------------
# observables, growth check, argument errors, graph/step equivalence, tuning
# ---------------------------------------------------------------------------------------
def test_ribbon_observables_match_oracle():
    cb = _cb()
    import torch

    rb = wl.Ribbon(W=16, L=90, sigma=5.0)
    epsn = rb.onsite()
    eps = dev_f64(epsn)
    desc, keep = cb.desc_ribbons([rb.W], [rb.L], 1.0, eps)
    plan = cb.Plan(desc, *[[x] for x in rb.bounds()], 0.0, cb.CHEB_C128, 1, keep=keep)
    x = rb.packet()
    psi = dev_vec(x, C128)
    H = oracle.honeycomb(rb.W, rb.L, 1.0, epsn)
    n2, e = H.norm_energy(x)
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_NORM2, 0.0, out)
    assert abs(out.item() - n2) < 1e-14
    plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, out)
    assert abs(out.item() - e) < 1e-13
    plan.observables(psi, cb.CHEB_OBS_PROB_COLS, 30.0, out)
    cols = np.arange(rb.W * rb.L) % rb.L
    assert abs(out.item() - np.sum(np.abs(x[cols > 30]) ** 2)) < 1e-14
    # the energy recorded by the first recurrence kernel of a step agrees
    rec = torch.zeros((1, 1, 1, 2), dtype=torch.float64, device="cuda:0")
    plan.evolve(psi, rb.dt, 1, 1, rec)
    assert abs(rec[0, 0, 0, 0].item() - n2) < 1e-13 and abs(rec[0, 0, 0, 1].item() - e) < 1e-12


def test_growth_check_flags_too_tight_bounds():
    cb = _cb()
    rb = wl.Ribbon(W=8, L=64, sigma=4.0)
    eps = dev_f64(rb.onsite())
    desc, keep = cb.desc_ribbons([rb.W], [rb.L], 1.0, eps)
    plan = cb.Plan(desc, [-1.0], [1.0], 0.0, cb.CHEB_C128, 1, keep=keep)  # true |E| up to ~3.5
    psi = dev_vec(rb.packet(), C128)
    with pytest.raises(cb.ChebError) as e:
        plan.evolve(psi, 4.0, 3)
    assert e.value.status == cb.CHEB_ERR_DIVERGED
    plan.sync()  # the flag is cleared once reported


def test_argument_errors():
    cb = _cb()
    import torch

    rb = wl.Ribbon(W=4, L=16)
    eps = dev_f64(rb.onsite())
    desc, keep = cb.desc_ribbons([4], [16], 1.0, eps)
    with pytest.raises(cb.ChebError) as e:
        cb.Plan(desc, [-3.5], [3.5], 0.0, cb.CHEB_C64, 3, keep=keep)
    assert e.value.status == cb.CHEB_ERR_INVALID
    with pytest.raises(cb.ChebError) as e:
        cb.Plan(desc, [3.5], [-3.5], 0.0, cb.CHEB_C64, 1, keep=keep)
    assert e.value.status == cb.CHEB_ERR_INVALID
    d0, k0 = cb.desc_ribbons([0], [16], 1.0, None)
    with pytest.raises(cb.ChebError):
        cb.Plan(d0, [-3.5], [3.5], 0.0, cb.CHEB_C64, 1, keep=k0)
    plan = cb.Plan(desc, [-3.5], [3.5], 0.0, cb.CHEB_C64, 1, keep=keep)
    buf = torch.zeros(4 * 16 + 1, dtype=torch.complex64, device="cuda:0")
    with pytest.raises(cb.ChebError) as e:
        plan.step(buf[1:], 1.0)  # 8-byte offset: not 16-byte aligned
    assert e.value.status == cb.CHEB_ERR_ALIGN
    with pytest.raises(cb.ChebError) as e:
        plan.step(buf[:64], -1.0)
    assert e.value.status == cb.CHEB_ERR_INVALID
    x = dev_vec(rb.packet(), C64)
    y = x.clone()
    plan.evolve(y, 1.0, 0)
    assert torch.equal(x, y)
    with pytest.raises(cb.ChebError) as e:  # periodic chain needs L >= 3
        cb.Plan(cb.desc_holstein(2, 2, True, 1.0, 1.0, 1.0), [-5.0], [5.0], 0.01, cb.CHEB_C128, 1)
    assert e.value.status == cb.CHEB_ERR_INVALID
    hp = cb.Plan(cb.desc_holstein(3, 2, True, 1.0, 1.0, 1.0), [-9.0], [9.0], 0.01, cb.CHEB_C128, 1)
    z = torch.zeros(hp.sites, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(cb.ChebError) as e:
        hp.adjoint_potential(z, 1.0, 1, region_col=0)
    assert e.value.status == cb.CHEB_ERR_UNSUPPORTED


def test_graph_replay_equals_single_steps_and_tuning_keeps_results():
    cb = _cb()
    ens = wl.RibbonEnsemble(n_ribbons=6, sizes=[(40, 500), (41, 777), (60, 501), (8, 4000),
                                                (160, 500), (3, 3)], sigma=8.0)
    W = [w for w, _ in ens.sizes]
    L = [l for _, l in ens.sizes]
    eps = dev_f64(ens.onsite())
    desc, keep = cb.desc_ribbons(W, L, 1.0, eps)
    lo, hi = ens.bounds()
    plan = cb.Plan(desc, lo, hi, 0.0, cb.CHEB_C64, 4, keep=keep)
    x0 = dev_vec(ens.packets(), C64)
    a = x0.clone()
    plan.evolve(a, 1.0, 5)
    b = x0.clone()
    for _ in range(5):
        plan.step(b, 1.0)
    plan.sync()
    assert bool((a == b).all())
    plan.autotune()
    c = x0.clone()
    plan.evolve(c, 1.0, 5)
    blk, _ = plan.blocking()
    if blk == 0:  # single-order launches: the launch shape does not change any result bit
        assert bool((a == c).all())
    else:  # temporal blocking: same recurrence vectors, partial sums added in another order
        assert rel(host(c), host(a)) <= 2e-6
    t, s, g, v = plan.launch_shape()
    assert t in (128, 256, 512) and s in (1, 2, 4) and g >= 1 and v in (1, 2, 4)
    n0 = plan.launches()
    plan.evolve(c, 1.0, 2)
    Ms = [plan.block(q)["M"] for q in range(6)]
    if blk == 0:
        expect = max(Ms)
    else:  # orders 1..s0, then blocks of blk; a last block shorter than blk/2 joins the one before
        s0 = min(blk, min(Ms) - 1)
        ranges = [(1, s0)]
        while ranges[-1][1] < max(Ms):
            ka = ranges[-1][1] + 1
            ranges.append((ka, min(ka + blk - 1, max(Ms))))
        if len(ranges) >= 3 and 2 * (ranges[-1][1] - ranges[-1][0] + 1) < blk:
            ranges[-2] = (ranges[-2][0], ranges[-1][1])
            ranges.pop()
        expect = len(ranges)
    assert plan.launches() - n0 == 2 * expect


# ---------------------------------------------------------------------------------------
# gradient with respect to the on-site potential
# ---------------------------------------------------------------------------------------
def _adjoint_case(W, L, nsteps, c0, r0, xR, seed=3022):
    rb = wl.Ribbon(W=W, L=L, disorder=1.0, seed=seed, sigma=20.0 if W >= 40 else 3.0, c0=c0,
                   r0=r0)
    eps = rb.onsite()
    mask = (np.arange(W * L) % L > xR).astype(np.uint8)
    return rb, eps, mask


@pytest.mark.parametrize("prec", [C128, C64])
def test_adjoint_small_matches_oracle(prec):
    cb = _cb()
    import torch

    rb, eps, mask = _adjoint_case(6, 24, 6, 6, 3, 12)
    H = oracle.honeycomb(rb.W, rb.L, 1.0, eps)
    a, b = oracle.rescale(*rb.bounds(), 0.0)
    C, M = oracle.coeffs(a, b, rb.dt)
    P, grad_ref, lam_ref = H.adjoint_region(a, b, C, 6, rb.packet(), mask)
    e = dev_f64(eps)
    desc, keep = cb.desc_ribbons([rb.W], [rb.L], 1.0, e)
    plan = cb.Plan(desc, *[[x] for x in rb.bounds()], 0.0, prec, 1, keep=keep)
    g = torch.zeros(rb.W * rb.L, dtype=torch.float64, device="cuda:0")
    Pd = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    lam0 = torch.zeros(rb.W * rb.L, dtype=torch.complex128 if prec == C128 else torch.complex64,
                       device="cuda:0")
    plan.adjoint_potential(dev_vec(rb.packet(), prec), rb.dt, 6, region_col=12, grad=g,
                           lambda0=lam0, P=Pd)
    tol = 1e-10 if prec == C128 else 2e-4
    assert abs(Pd.item() - P) <= tol * abs(P)
    assert rel(g.cpu().numpy(), grad_ref) <= tol
    assert rel(host(lam0), lam_ref) <= tol


def test_adjoint_full_configuration_fd_and_oracle():
    """60 x 1000 ribbon, W = 1, k0 = pi/3, T = 300 (dt = 1, M = 20): GPU gradient of P_R
    (x_R = 500) against the oracle's gradient and against central differences (h = 1e-6) of
    the GPU forward map on 32 random sites."""
    cb = _cb()
    import torch

    W, L, T, xR = 60, 1000, 300, 500
    rb, eps, mask = _adjoint_case(W, L, T, 250, 30, xR)
    e = dev_f64(eps)
    desc, keep = cb.desc_ribbons([W], [L], 1.0, e)
    lo, hi = rb.bounds()
    plan = cb.Plan(desc, [lo], [hi], 0.0, cb.CHEB_C128, 1, keep=keep)
    psi0 = dev_vec(rb.packet(), C128)
    g = torch.zeros(W * L, dtype=torch.float64, device="cuda:0")
    Pd = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.adjoint_potential(psi0, 1.0, T, region_col=xR, grad=g, P=Pd)
    grad = g.cpu().numpy()

    H = oracle.honeycomb(W, L, 1.0, eps)
    a, b = oracle.rescale(lo, hi, 0.0)
    C, M = oracle.coeffs(a, b, 1.0)
    P_ref, grad_ref, _ = H.adjoint_region(a, b, C, T, rb.packet(), mask)
    assert abs(Pd.item() - P_ref) <= 1e-10 * abs(P_ref)
    assert rel(grad, grad_ref) <= 1e-9

    def prob(epsv):
        e2 = dev_f64(epsv)
        plan.set_onsite(e2)
        x = psi0.clone()
        plan.evolve(x, 1.0, T)
        out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        plan.observables(x, cb.CHEB_OBS_PROB_COLS, float(xR), out)
        return out.item()

    rng = np.random.default_rng(32)
    sites = rng.choice(W * L, 32, replace=False)
    h = 1e-6
    for i in sites:
        ep, em = eps.copy(), eps.copy()
        ep[i] += h
        em[i] -= h
        fd = (prob(ep) - prob(em)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-4 * abs(grad[i]) + 1e-10, (i, fd, grad[i])
    plan.set_onsite(e)


def test_adjoint_batch_of_realisations_c64():
    """16 disorder realisations (one potential per vector), complex64: two realisations
    against the oracle's FP64 gradient.  Tolerances: P_R relative 1e-5 and the gradient
    relative L2 5e-5 -- the complex64 forward and adjoint states carry relative errors of a
    few 1e-6 after these 40 steps, and the gradient, a sum over steps and orders of products
    of the two, amplifies them by the sum's condition number (sum of |terms| / |sum|, about 3
    here), so its error is about 1e-5 at most (6e-6 measured)."""
    cb = _cb()
    import torch

    W, L, T, xR, nv = 20, 120, 40, 60, 16
    eps = np.stack([wl.anderson_disorder(W * L, 1.0, 3022, r) for r in range(nv)], axis=1)
    psi0 = wl.ribbon_packet(W, L, 8.0, math.pi / 3, 10, 30)
    e = dev_f64(eps)
    desc, keep = cb.desc_ribbons([W], [L], 1.0, e, onsite_per_vec=True)
    plan = cb.Plan(desc, [-3.5], [3.5], 0.0, cb.CHEB_C64, nv, keep=keep)
    x0 = dev_vec(np.repeat(psi0[:, None], nv, axis=1), C64)
    g = torch.zeros((W * L, nv), dtype=torch.float64, device="cuda:0")
    Pd = torch.zeros(nv, dtype=torch.float64, device="cuda:0")
    plan.adjoint_potential(x0, 1.0, T, region_col=xR, grad=g, P=Pd)
    mask = (np.arange(W * L) % L > xR).astype(np.uint8)
    for r in (0, 11):
        H = oracle.honeycomb(W, L, 1.0, eps[:, r])
        a, b = oracle.rescale(-3.5, 3.5, 0.0)
        C, M = oracle.coeffs(a, b, 1.0)
        P_ref, grad_ref, _ = H.adjoint_region(a, b, C, T, psi0, mask)
        assert abs(Pd[r].item() - P_ref) <= 1e-5 * P_ref
        assert rel(g[:, r].cpu().numpy(), grad_ref) <= 5e-5


def test_autograd_function_matches_adjoint():
    cb = _cb()
    import torch
    from paper_0907_3022_gb300.autograd import evolve_potential

    W, L, T = 6, 30, 5
    rb = wl.Ribbon(W=W, L=L, sigma=3.0, c0=8, r0=3)
    eps = rb.onsite()
    e = dev_f64(eps)
    desc, keep = cb.desc_ribbons([W], [L], 1.0, e)
    plan = cb.Plan(desc, *[[x] for x in rb.bounds()], 0.0, cb.CHEB_C128, 1, keep=keep)
    V = dev_f64(eps).requires_grad_(True)
    psi0 = dev_vec(rb.packet(), C128).requires_grad_(True)
    psi = evolve_potential(plan, V, psi0, 1.0, T)
    cols = torch.arange(W * L, device="cuda:0") % L
    Pt = (psi.abs() ** 2)[cols > 15].sum()
    gV, gpsi = torch.autograd.grad(Pt, (V, psi0))
    H = oracle.honeycomb(W, L, 1.0, eps)
    a, b = oracle.rescale(*rb.bounds(), 0.0)
    C, M = oracle.coeffs(a, b, 1.0)
    mask = (np.arange(W * L) % L > 15).astype(np.uint8)
    P_ref, grad_ref, lam_ref = H.adjoint_region(a, b, C, T, rb.packet(), mask)
    assert abs(Pt.item() - P_ref) <= 1e-12
    assert rel(gV.cpu().numpy(), grad_ref) <= 1e-10
    assert rel(host(gpsi), 2 * lam_ref) <= 1e-10
