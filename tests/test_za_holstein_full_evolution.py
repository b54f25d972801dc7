"""The full Holstein configuration (Sec. 3.3, Eq. ghm: L = 12 periodic, nph <= 10,
D = 7,759,752, t = 1, w0 = 1, g = 1.5, dt = 0.25, 200 steps from the electron on site 0 with
the phonon vacuum) against the FP64 oracle after the whole evolution, for the stored SELL
matrix and the matrix-free operator: complex128 relative L2 <= 1e-10; complex64 relative L2
<= 1e-4 and norm drift <= 1e-5 over the run.

The oracle's 3,800 sparse products take about five minutes of host time; the run is started
as a child process when the session begins (``tests/conftest.py``) and overlaps the other GPU
tests.  The file name makes pytest collect it after them.
"""
import numpy as np
import pytest

import workloads as wl
from _gpu_util import C64, C128, dev_vec, host, rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow, pytest.mark.holstein_full_oracle]


@pytest.mark.parametrize("matrix_free", [False, True])
@pytest.mark.parametrize("prec", [C128, C64])
def test_holstein_full_evolution_matches_oracle(holstein_full_reference, prec, matrix_free):
    import torch

    import paper_0907_3022_gb300 as cb

    ref = holstein_full_reference
    hs = wl.Holstein()
    desc = cb.desc_holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g,
                            matrix_free=matrix_free)
    lo, hi = hs.bounds()
    plan = cb.Plan(desc, [lo], [hi], hs.alpha, prec, 1)
    assert plan.sites == hs.dim
    psi = dev_vec(hs.initial_state(), prec)
    nrec = 10
    rec = torch.zeros((nrec, 1, 1, 2), dtype=torch.float64, device="cuda:0")
    plan.evolve(psi, hs.dt, hs.nsteps, hs.nsteps // nrec, rec)
    assert plan.block(0)["M"] == int(ref["M"])
    out = host(psi)
    err = rel(out, ref["psi"])
    n2 = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(psi, cb.CHEB_OBS_NORM2, 0.0, n2)
    r = rec.cpu().numpy()[:, 0, 0]
    drift = max(abs(float(n2.item()) - 1.0), float(np.max(np.abs(r[:, 0] - 1.0))))
    if prec == C128:
        assert err <= 1e-10, err
        assert drift <= 1e-11, drift
        # <H> of the start state is 0 (no phonon, no on-site energy) and is conserved: compare
        # on the scale of the spectrum's half width a
        e = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        plan.observables(psi, cb.CHEB_OBS_ENERGY, 0.0, e)
        a = plan.block(0)["a"]
        assert abs(float(e.item()) - float(ref["energy"])) <= 1e-10 * a
    else:
        assert err <= 1e-4, err
        assert drift <= 1e-5, drift
    plan.close()
