"""SELL-C-sigma storage of the Holstein matrix (Sec. 3.3, Eq. ghm): rows sorted by decreasing
off-diagonal count inside windows of sigma rows, chunks of 32 storage positions.  The matrix
exported back in row order is bit-identical to the oracle's for every sigma; propagation and
the energy observable through the sorted storage match the oracle; sorting cuts the padding
of the full configuration (L = 12, nph <= 10) from about 25 % to a few per cent."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu_util import C64, C128, dev_vec, host, rel

pytestmark = pytest.mark.gpu


def _plan(cb, hs, prec, sigma):
    desc = cb.desc_holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g, sell_sigma=sigma)
    lo, hi = hs.bounds()
    return cb.Plan(desc, [lo], [hi], hs.alpha, prec, 1)


def _sorted_rows(rp, col, val):
    return [sorted(zip(col[rp[i]:rp[i + 1]].tolist(), val[rp[i]:rp[i + 1]].tolist()))
            for i in range(len(rp) - 1)]


@pytest.mark.parametrize("sigma", [32, 64, 1024])
@pytest.mark.parametrize("L,nph,periodic", [(4, 3, True), (5, 4, False), (1, 7, False), (6, 5, True)])
def test_sigma_sorted_matrix_bit_exact(L, nph, periodic, sigma):
    import paper_0907_3022_gb300 as cb

    hs = wl.Holstein(L=L, nph=nph, periodic=periodic)
    plan = _plan(cb, hs, C128, sigma)
    st = plan.sell_stats()
    assert st["sigma"] == sigma
    rp, col, val = plan.export_csr()
    orp, ocol, oval = oracle.holstein(L, nph, periodic, hs.hop, hs.omega0, hs.g).csr()
    assert np.array_equal(rp, orp)
    assert _sorted_rows(rp, col, val) == _sorted_rows(orp, ocol, oval)
    assert st["offdiag"] == len(ocol) - plan.sites
    plan.close()


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("sigma", [64, 4096])
def test_sigma_sorted_propagation_and_energy(prec, sigma):
    import torch

    import paper_0907_3022_gb300 as cb

    hs = wl.Holstein(L=6, nph=5)
    plan = _plan(cb, hs, prec, sigma)
    x0 = wl.random_state(hs.dim, 11, 0)
    psi = dev_vec(x0, prec)
    nsteps = 20
    plan.evolve(psi, hs.dt, nsteps)
    H = oracle.holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g)
    a, b = oracle.rescale(*hs.bounds(), hs.alpha)
    C, M = oracle.coeffs(a, b, hs.dt)
    ref = H.evolve(a, b, C, nsteps, x0)
    assert rel(host(psi), ref) <= (1e-10 if prec == C128 else 1e-4)
    e = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, e)
    _, e_ref = H.norm_energy(ref)
    assert abs(e.item() - e_ref) <= (1e-10 if prec == C128 else 1e-4) * a
    plan.close()


def test_sigma_cuts_padding_of_the_full_configuration():
    import paper_0907_3022_gb300 as cb

    hs = wl.Holstein()
    unsorted = _plan(cb, hs, C64, 1).sell_stats()
    assert unsorted["stored"] / unsorted["offdiag"] > 1.2
    for sigma in (256, 1024):
        st = _plan(cb, hs, C64, sigma).sell_stats()
        assert st["offdiag"] == unsorted["offdiag"] == 22_573_824
        assert st["stored"] / st["offdiag"] < 1.05, (sigma, st)


def test_sigma_rejected():
    import paper_0907_3022_gb300 as cb

    hs = wl.Holstein(L=4, nph=3)
    for bad in (-1, 2, 48 + 1, 1 << 21):
        with pytest.raises(cb.ChebError) as e:
            _plan(cb, hs, C64, bad)
        assert e.value.status == cb.CHEB_ERR_INVALID
