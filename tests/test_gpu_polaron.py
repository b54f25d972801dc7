"""Generalised Holstein model of the polaron experiment (Sec. 3.3, Fig. 3: site potentials
Delta_i, site couplings g_i, open chain, electron wave packet) against the oracle at reduced
sizes, and the paper's own basis (18 sites, at most 11 phonons, D = 622,751,220) built and
propagated on the GPU with its conservation laws checked."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu_util import C64, C128, dev_f64, dev_vec, host, rel

pytestmark = pytest.mark.gpu


def _plan(cb, pw, prec):
    d, g = dev_f64(pw.delta()), dev_f64(pw.gsite())
    desc = cb.desc_holstein(pw.L, pw.nph, pw.periodic, pw.hop, pw.omega0, 1.0, delta=d, gsite=g)
    lo, hi = pw.bounds()
    return cb.Plan(desc, [lo], [hi], pw.alpha, prec, 1, keep=(d, g))


def _oracle(pw):
    return oracle.holstein(pw.L, pw.nph, pw.periodic, pw.hop, pw.omega0, 1.0,
                           Delta=pw.delta(), gsite=pw.gsite())


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("L,nph,barrier,start,nsteps", [(6, 4, 4, 1, 30), (10, 6, 7, 2, 12)])
def test_generalised_holstein_matches_oracle(prec, L, nph, barrier, start, nsteps):
    import torch

    import paper_0907_3022_gb300 as cb

    pw = wl.Polaron(L=L, nph=nph, barrier_site=barrier, packet_site=start, sigma=1.0)
    plan = _plan(cb, pw, prec)
    H = _oracle(pw)
    if prec == C128:
        rp, col, val = plan.export_csr()
        orp, ocol, oval = H.csr()
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(val, oval)
    psi = dev_vec(pw.initial_state(), prec)
    plan.evolve(psi, pw.dt, nsteps)
    a, b = oracle.rescale(*pw.bounds(), pw.alpha)
    C, M = oracle.coeffs(a, b, pw.dt)
    ref = H.evolve(a, b, C, nsteps, pw.initial_state())
    assert plan.block(0)["M"] == M
    assert rel(host(psi), ref) <= (1e-10 if prec == C128 else 1e-4)
    dens, phon, chi = H.observables(ref)
    tol = 1e-11 if prec == C128 else 1e-5
    for kind, r in ((cb.CHEB_OBS_HOL_DENSITY, dens), (cb.CHEB_OBS_HOL_PHONON, phon),
                    (cb.CHEB_OBS_HOL_CHI, chi)):
        out = torch.zeros(L, dtype=torch.float64, device="cuda:0")
        plan.observables(psi, kind, 0.0, out)
        assert np.max(np.abs(out.cpu().numpy() - r)) <= tol
    e = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, e)
    assert abs(e.item() - H.norm_energy(ref)[1]) <= (1e-10 if prec == C128 else 1e-4)


def test_paper_polaron_basis_on_one_gpu():
    """D = 622,751,220 (the paper's run needed 18 processors and ~60 GB): the complex64
    plan is built on the device and two time steps keep the norm, the energy and
    sum_i <n_i> = 1."""
    import torch

    import paper_0907_3022_gb300 as cb

    pw = wl.Polaron()
    plan = _plan(cb, pw, C64)
    assert plan.sites == 622_751_220
    psi = torch.zeros(pw.dim, dtype=torch.complex64, device="cuda:0")
    idx = torch.from_numpy(pw.packet_indices()).to("cuda:0")
    psi[idx] = torch.from_numpy(pw.electron_packet().astype(np.complex64)).to("cuda:0")
    n2 = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    en = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, en)
    e0 = en.item()
    plan.evolve(psi, pw.dt, 2)
    plan.observables(psi, cb.CHEB_OBS_NORM2, 0.0, n2)
    plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, en)
    assert abs(n2.item() - 1.0) <= 1e-5
    assert abs(en.item() - e0) <= 1e-4 * max(1.0, abs(e0))
    dens = torch.zeros(pw.L, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_HOL_DENSITY, 0.0, dens)
    assert abs(float(dens.sum()) - 1.0) <= 1e-5
    # the packet moved right, towards the barrier
    d = dens.cpu().numpy()
    assert np.sum(np.arange(pw.L) * d) > pw.packet_site
