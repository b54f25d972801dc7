"""The paper's own runs beyond the configurations: the double well of Sec. 3.1 against full
diagonalisation."""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu_util import C64, C128, dev_f64, dev_vec, host, rel

pytestmark = pytest.mark.gpu


def _exact_1d(d, t):
    from scipy.linalg import eigh_tridiagonal

    dd, ee = d.tridiagonal()
    E, U = eigh_tridiagonal(dd, ee)
    return U @ (np.exp(-1j * E * t) * (U.T @ d.packet()))


def test_paper_double_well_against_exact_diagonalisation():
    """Sec. 3.1: N = 2048, 1500 moments, dt = 0.4 to t = 40: complex128 within the paper's
    2e-11 (absolute, psi_i / sqrt(dx)) of full diagonalisation and within 1e-11 of the
    oracle; complex64 within 2e-3 relative."""
    import paper_0907_3022_gb300 as cb

    d = wl.PaperDoubleWell()
    lo, hi = d.bounds()
    V = dev_f64(d.potential())
    ex = _exact_1d(d, d.t_end)
    a, b = oracle.rescale(lo, hi, 0.01)
    C, M = oracle.coeffs(a, b, d.dt)
    ref = oracle.lattice1d(d.n, d.dx, d.potential()).evolve(a, b, C, d.nsteps, d.packet())
    for prec in (C128, C64):
        plan = cb.Plan(cb.desc_lat1d(d.n, d.dx, V), [lo], [hi], 0.01, prec, 1, keep=(V,))
        psi = dev_vec(d.packet(), prec)
        plan.evolve(psi, d.dt, d.nsteps)
        assert plan.block(0)["M"] == M == 1499
        out = host(psi)
        err = float(np.max(np.abs(out - ex)) / math.sqrt(d.dx))
        print(prec, "max abs err vs ED", err, "rel vs oracle", rel(out, ref))
        if prec == C128:
            assert err < 2e-11
            assert rel(out, ref) <= 1e-11
        else:
            assert rel(out, ex) <= 2e-3
        plan.close()


# ---------------------------------------------------------------------------------------
# time-dependent H(t), piecewise constant over each step (Sec. 2.2)
# ---------------------------------------------------------------------------------------
def _driven_well(n=96):
    d = wl.DoubleWell1D(n=n, x_lo=-6.0, x_hi=6.0)
    F, Om = 0.8, 1.3
    return d, (lambda t: d.potential() + F * math.sin(Om * t) * d.x), F * np.max(np.abs(d.x))


@pytest.mark.parametrize("prec", [C128, C64])
def test_time_dependent_1d_matches_oracle(prec):
    """Driven double well: the on-site energies at the step midpoints, 40 steps of 0.05;
    the GPU equals the oracle's piecewise-constant propagation (complex128 1e-12,
    complex64 1e-4)."""
    import paper_0907_3022_gb300 as cb

    d, Vt, vmax = _driven_well()
    dt, nsteps = 0.05, 40
    seq = np.stack([Vt((s + 0.5) * dt) for s in range(nsteps)])
    lo, hi = d.bounds()
    lo, hi = lo - vmax, hi + vmax
    a, b = oracle.rescale(lo, hi, 0.01)
    C, _ = oracle.coeffs(a, b, dt)
    ref = oracle.evolve_piecewise(lambda V: oracle.lattice1d(d.n, d.dx, V), seq, a, b, C,
                                  d.packet())
    V0 = dev_f64(d.potential())
    plan = cb.Plan(cb.desc_lat1d(d.n, d.dx, V0), [lo], [hi], 0.01, prec, 1, keep=(V0,))
    psi = dev_vec(d.packet(), prec)
    seq_dev = dev_f64(seq)
    plan.evolve_td(psi, dt, nsteps, seq_dev)
    assert rel(host(psi), ref) <= (1e-12 if prec == C128 else 1e-4)


def test_time_dependent_ensemble_uniform_shift_closed_form():
    """Three ribbons x 4 packets (complex64, temporal blocking and single-order launches)
    under a uniform shift v(t) = v0 + v1 t: the state is exp(-i(v0 T + v1 T^2/2)) times the
    unshifted evolution, exactly for midpoint sampling; complex128 single vector against the
    oracle."""
    import torch

    import paper_0907_3022_gb300 as cb

    rbs = [wl.Ribbon(W=12, L=60, sigma=4.0, stream=q) for q in range(3)]
    base = np.concatenate([rb.onsite() for rb in rbs])
    dt, nsteps, v0, v1 = 1.0, 12, 0.25, -0.05
    T = dt * nsteps
    vmin, vmax = min(v0, v0 + v1 * T), max(v0, v0 + v1 * T)
    lo = [rb.bounds()[0] + vmin for rb in rbs]
    hi = [rb.bounds()[1] + vmax for rb in rbs]
    seq = np.stack([base + v0 + v1 * (s + 0.5) * dt for s in range(nsteps)])
    phase = np.exp(-1j * (v0 * T + 0.5 * v1 * T * T))
    k0s = (np.pi / 6, np.pi / 4, np.pi / 3, np.pi / 2)
    X = np.concatenate([np.stack([rb.packet(k) for k in k0s], axis=1) for rb in rbs])
    eps = dev_f64(base)
    seq_dev = dev_f64(seq)
    for blocking in (0, 3):
        desc, keep = cb.desc_ribbons([rb.W for rb in rbs], [rb.L for rb in rbs], 1.0, eps)
        plan = cb.Plan(desc, lo, hi, 0.0, cb.CHEB_C64, 4, keep=keep)
        plan.evolve(dev_vec(X, C64), dt, 0)
        plan.set_blocking(blocking, 4)
        static = dev_vec(X, C64)
        plan.evolve(static, dt, nsteps)
        psi = dev_vec(X, C64)
        plan.evolve_td(psi, dt, nsteps, seq_dev)
        assert rel(host(psi), phase * host(static)) <= 2e-5
        plan.close()
    # complex128, one packet, against the oracle (each ribbon its own rescaling)
    desc, keep = cb.desc_ribbons([rb.W for rb in rbs], [rb.L for rb in rbs], 1.0, eps)
    plan = cb.Plan(desc, lo, hi, 0.0, C128, 1, keep=keep)
    x1 = X[:, 2].copy()
    psi = dev_vec(x1, C128)
    plan.evolve_td(psi, dt, nsteps, seq_dev)
    out = host(psi)
    off = np.cumsum([0] + [rb.W * rb.L for rb in rbs])
    for q, rb in enumerate(rbs):
        a, b = oracle.rescale(lo[q], hi[q], 0.0)
        C, _ = oracle.coeffs(a, b, dt)
        sl = slice(off[q], off[q + 1])
        ref = oracle.evolve_piecewise(lambda V: oracle.honeycomb(rb.W, rb.L, 1.0, V),
                                      [row[sl] for row in seq], a, b, C, x1[sl])
        assert rel(out[sl], ref) <= 1e-12
        assert rel(out[sl], phase * oracle.honeycomb(rb.W, rb.L, 1.0, base[sl]).evolve(
            a, b, C, nsteps, x1[sl])) <= 1e-12
    torch.cuda.synchronize()


def test_time_dependent_argument_errors():
    import torch

    import paper_0907_3022_gb300 as cb

    d = wl.DoubleWell1D(n=64, x_lo=-6.0, x_hi=6.0)
    V0 = dev_f64(d.potential())
    plan = cb.Plan(cb.desc_lat1d(d.n, d.dx, V0), [0.0], [400.0], 0.01, C128, 1, keep=(V0,))
    psi = dev_vec(d.packet(), C128)
    seq = torch.zeros((4, 66), dtype=torch.float64, device="cuda:0")
    for stride, status in ((63, cb.CHEB_ERR_INVALID), (65, cb.CHEB_ERR_ALIGN),
                           (67, cb.CHEB_ERR_ALIGN)):
        with pytest.raises(cb.ChebError) as e:
            plan.evolve_td(psi, 0.1, 3, seq, stride=stride)
        assert e.value.status == status
    plan.evolve_td(psi, 0.1, 3, seq, stride=66)  # padded rows
    hs = wl.Holstein(L=3, nph=2, periodic=True)
    hp = cb.Plan(cb.desc_holstein(3, 2, True, 1.0, 1.0, 1.0), [-9.0], [9.0], 0.01, C128, 1)
    hpsi = dev_vec(hs.initial_state(), C128)
    with pytest.raises(cb.ChebError) as e:
        hp.evolve_td(hpsi, 0.1, 1, seq)
    assert e.value.status == cb.CHEB_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------------------
# armchair ribbons of Table 2 (Sec. 3.2)
# ---------------------------------------------------------------------------------------
def _armchair_plan(cb, rbs, prec):
    eps = dev_f64(np.concatenate([rb.onsite() for rb in rbs]))
    desc, keep = cb.desc_armchair([rb.n_a for rb in rbs], [rb.length for rb in rbs], 1.0, eps)
    lo = [rb.bounds()[0] for rb in rbs]
    hi = [rb.bounds()[1] for rb in rbs]
    return cb.Plan(desc, lo, hi, 0.0, prec, 1, keep=keep)


def test_armchair_table2_against_exact_diagonalisation():
    """Table 2 set-up at reduced length (N_a = 10, 300 atoms per line), disorder W = 0.5 and
    4 in one two-ribbon plan, the state on one central site: t = 10^4 with dt = 1, 10 and 100
    agrees with exp(-iHt) from full diagonalisation of the oracle's matrix to 1e-9
    (complex128, absolute), whatever the step."""
    import paper_0907_3022_gb300 as cb

    rbs = [wl.ArmchairRibbon(length=300, disorder=w, stream=q) for q, w in enumerate((0.5, 4.0))]
    x0 = np.concatenate([rb.packet() for rb in rbs])
    off = np.cumsum([0] + [rb.n_sites for rb in rbs])
    exact = []
    for rb in rbs:
        E, U = np.linalg.eigh(oracle.honeycomb(rb.W, rb.L, 1.0, rb.onsite()).dense())
        exact.append(U @ (np.exp(-1j * E * rb.t_end) * (U.T @ rb.packet())))
    plan = _armchair_plan(cb, rbs, C128)
    for dt in (1.0, 10.0, 100.0):
        psi = dev_vec(x0, C128)
        plan.evolve(psi, dt, int(round(1e4 / dt)))
        out = host(psi)
        for q in range(2):
            assert np.max(np.abs(out[off[q]:off[q + 1]] - exact[q])) < 1e-9, (dt, q)
    # stronger disorder keeps the state closer to its start (Sec. 3.2: localisation)
    r = np.arange(300)

    def spread(x, rb):
        p = np.abs(x.reshape(rb.length, rb.n_a)) ** 2
        return float(np.sqrt(np.sum(p.sum(axis=1) * (r - rb.length // 2) ** 2)))

    assert spread(exact[1], rbs[1]) < spread(exact[0], rbs[0])


def test_armchair_table2_full_size():
    """The 10 x 1000 ribbons of Table 2 (W = 0.5 and 4): the states at t = 10^4 from dt = 1,
    10 and 100 agree to 1e-9, and dt = 100 matches the oracle to 1e-11 (complex128)."""
    import paper_0907_3022_gb300 as cb

    rbs = [wl.ArmchairRibbon(disorder=w, stream=q) for q, w in enumerate((0.5, 4.0))]
    x0 = np.concatenate([rb.packet() for rb in rbs])
    plan = _armchair_plan(cb, rbs, C128)
    outs = {}
    for dt in (1.0, 10.0, 100.0):
        psi = dev_vec(x0, C128)
        plan.evolve(psi, dt, int(round(1e4 / dt)))
        outs[dt] = host(psi)
    assert np.max(np.abs(outs[1.0] - outs[100.0])) < 1e-9
    assert np.max(np.abs(outs[10.0] - outs[100.0])) < 1e-9
    off = np.cumsum([0] + [rb.n_sites for rb in rbs])
    for q, rb in enumerate(rbs):
        a, b = oracle.rescale(*rb.bounds(), 0.0)
        C, M = oracle.coeffs(a, b, 100.0)
        assert plan.block(q)["M"] == M
        ref = oracle.honeycomb(rb.W, rb.L, 1.0, rb.onsite()).evolve(a, b, C, 100, rb.packet())
        assert rel(outs[100.0][off[q]:off[q + 1]], ref) <= 1e-11
