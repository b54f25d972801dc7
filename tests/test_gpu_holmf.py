"""Matrix-free Holstein operator (Sec. 3.3: matrix elements recomputed in every
multiplication) against the oracle and against the stored SELL matrix.

Both operators form each row's sum in the same order from the same scaled values, so their
states agree bit for bit; the oracle bounds both to the usual tolerances (complex128 1e-10,
complex64 1e-4 relative L2).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu_util import C64, C128, dev_f64, dev_vec, host, rel

pytestmark = pytest.mark.gpu

TOL = {C128: 1e-10, C64: 1e-4}


def _plan(cb, hs, prec, matrix_free, nvec=1):
    desc = cb.desc_holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g,
                            matrix_free=matrix_free)
    lo, hi = hs.bounds()
    return cb.Plan(desc, [lo], [hi], hs.alpha, prec, nvec)


def _polaron_plan(cb, pw, prec, matrix_free):
    d, g = dev_f64(pw.delta()), dev_f64(pw.gsite())
    desc = cb.desc_holstein(pw.L, pw.nph, pw.periodic, pw.hop, pw.omega0, 1.0, delta=d,
                            gsite=g, matrix_free=matrix_free)
    lo, hi = pw.bounds()
    return cb.Plan(desc, [lo], [hi], pw.alpha, prec, 1, keep=(d, g))


def _energy(cb, plan, psi, nvec=1):
    import torch

    e = torch.zeros(nvec, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, e)
    return e.cpu().numpy()


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("L,nph,periodic,nsteps", [(4, 3, True, 40), (6, 4, True, 30),
                                                   (5, 3, False, 20), (1, 7, False, 10),
                                                   (2, 5, False, 10), (7, 15, False, 3)])
def test_matrix_free_matches_oracle_and_sell(prec, L, nph, periodic, nsteps):
    import torch

    import paper_0907_3022_gb300 as cb

    hs = wl.Holstein(L=L, nph=nph, periodic=periodic)
    mf = _plan(cb, hs, prec, True)
    sell = _plan(cb, hs, prec, False)
    x0 = hs.initial_state()
    psi_mf, psi_sell = dev_vec(x0, prec), dev_vec(x0, prec)
    mf.evolve(psi_mf, hs.dt, nsteps)
    sell.evolve(psi_sell, hs.dt, nsteps)
    assert torch.equal(psi_mf, psi_sell)
    H = oracle.holstein(L, nph, periodic, hs.hop, hs.omega0, hs.g)
    a, b = oracle.rescale(*hs.bounds(), hs.alpha)
    C, M = oracle.coeffs(a, b, hs.dt)
    ref = H.evolve(a, b, C, nsteps, x0)
    assert mf.block(0)["M"] == M
    assert rel(host(psi_mf), ref) <= TOL[prec]
    e_ref = H.norm_energy(ref)[1]
    assert abs(_energy(cb, mf, psi_mf)[0] - e_ref) <= (1e-10 if prec == C128 else 1e-4)
    dens, phon, chi = H.observables(ref)
    tol = 1e-11 if prec == C128 else 1e-5
    for kind, r in ((cb.CHEB_OBS_HOL_DENSITY, dens), (cb.CHEB_OBS_HOL_PHONON, phon),
                    (cb.CHEB_OBS_HOL_CHI, chi)):
        out = torch.zeros(L, dtype=torch.float64, device="cuda:0")
        mf.observables(psi_mf, kind, 0.0, out)
        assert np.max(np.abs(out.cpu().numpy() - r)) <= tol, kind


@pytest.mark.parametrize("prec", [C128, C64])
def test_matrix_free_generalised_model(prec):
    """Site potentials (barrier) and site couplings of the polaron experiment, open chain."""
    import torch

    import paper_0907_3022_gb300 as cb

    pw = wl.Polaron(L=8, nph=5, barrier_site=5, packet_site=1, sigma=1.0)
    mf = _polaron_plan(cb, pw, prec, True)
    sell = _polaron_plan(cb, pw, prec, False)
    x0 = pw.initial_state()
    a_mf, a_sell = dev_vec(x0, prec), dev_vec(x0, prec)
    mf.evolve(a_mf, pw.dt, 16)
    sell.evolve(a_sell, pw.dt, 16)
    assert torch.equal(a_mf, a_sell)
    H = oracle.holstein(pw.L, pw.nph, pw.periodic, pw.hop, pw.omega0, 1.0,
                        Delta=pw.delta(), gsite=pw.gsite())
    a, b = oracle.rescale(*pw.bounds(), pw.alpha)
    C, M = oracle.coeffs(a, b, pw.dt)
    ref = H.evolve(a, b, C, 16, x0)
    assert rel(host(a_mf), ref) <= TOL[prec]
    e_mf, e_sell = _energy(cb, mf, a_mf)[0], _energy(cb, sell, a_sell)[0]
    e_ref = H.norm_energy(ref)[1]
    assert abs(e_mf - e_ref) <= (1e-10 if prec == C128 else 1e-4)
    assert abs(e_mf - e_sell) <= (1e-12 if prec == C128 else 1e-5) * max(1.0, abs(e_ref))


def test_matrix_free_several_vectors_and_step_observables():
    """nvec = 4 (one vector per thread, interleaved storage): every vector equals its own
    single-vector run; the norms and energies the first launch of each step records match
    the oracle's."""
    import torch

    import paper_0907_3022_gb300 as cb

    hs = wl.Holstein(L=5, nph=4, periodic=True)
    rng = np.random.default_rng(5)
    D = hs.dim
    X = (rng.standard_normal((D, 4)) + 1j * rng.standard_normal((D, 4)))
    X /= np.linalg.norm(X, axis=0)
    mf4 = _plan(cb, hs, C128, True, nvec=4)
    psi4 = dev_vec(X, C128)
    nsteps = 6
    obs = torch.zeros((nsteps, 1, 4, 2), dtype=torch.float64, device="cuda:0")
    mf4.evolve(psi4, hs.dt, nsteps, obs_every=1, obs=obs)
    H = oracle.holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g)
    a, b = oracle.rescale(*hs.bounds(), hs.alpha)
    C, M = oracle.coeffs(a, b, hs.dt)
    n2_0, e_0 = H.norm_energy(X[:, 2])
    o = obs.cpu().numpy()
    assert abs(o[0, 0, 2, 0] - n2_0) <= 1e-12 and abs(o[0, 0, 2, 1] - e_0) <= 1e-10
    out = host(psi4).reshape(D, 4)
    for v in range(4):
        ref = H.evolve(a, b, C, nsteps, X[:, v])
        assert rel(out[:, v], ref) <= 1e-10
    e = _energy(cb, mf4, psi4, 4)
    for v in range(4):
        assert abs(e[v] - H.norm_energy(out[:, v])[1]) <= 1e-10


def test_matrix_free_full_configuration_equals_sell():
    """L = 12 periodic, nph <= 10 (D = 7,759,752): the matrix-free complex64 and complex128
    plans reproduce the stored-matrix plans bit for bit over 3 steps; one complex128 step
    matches the oracle."""
    import torch

    import paper_0907_3022_gb300 as cb

    hs = wl.Holstein()
    H = oracle.holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g)
    a, b = oracle.rescale(*hs.bounds(), hs.alpha)
    C, M = oracle.coeffs(a, b, hs.dt)
    ref1 = H.step(a, b, C, hs.initial_state())
    for prec in (C128, C64):
        mf = _plan(cb, hs, prec, True)
        assert mf.sites == 7_759_752
        psi = dev_vec(hs.initial_state(), prec)
        mf.evolve(psi, hs.dt, 1)
        assert rel(host(psi), ref1) <= (1e-12 if prec == C128 else 1e-4)
        mf.autotune()
        mf.evolve(psi, hs.dt, 2)
        mf.close()
        sell = _plan(cb, hs, prec, False)
        q = dev_vec(hs.initial_state(), prec)
        sell.evolve(q, hs.dt, 3)
        sell.close()
        assert torch.equal(psi, q)


def test_matrix_free_limits_and_unsupported():
    import paper_0907_3022_gb300 as cb

    for L, nph in ((4, 16), (33, 2)):
        hs = wl.Holstein(L=L, nph=nph, periodic=False)
        with pytest.raises(cb.ChebError) as e:
            _plan(cb, hs, C128, True)
        assert e.value.status == cb.CHEB_ERR_UNSUPPORTED
    mf = _plan(cb, wl.Holstein(L=3, nph=2, periodic=True), C128, True)
    with pytest.raises(cb.ChebError) as e:
        mf.export_csr()
    assert e.value.status == cb.CHEB_ERR_UNSUPPORTED
