"""The allocation-free region norm (cheb_region_norm_noalloc) against cheb_observables.

cheb_region_norm_noalloc is for callers that may not allocate device memory (latency-critical
loops that cannot take cudaMalloc's device-wide synchronisation, hosts whose own pool owns all
device memory).  Its tile partials live in a static device array shared by every call, so the test
calls it twice in a row on different inputs and checks both results against the plan-based
entry point, which reduces the same quantity with plan-owned scratch.  This file is named to
be collected last.
"""
import numpy as np
import pytest

import workloads as wl
from _gpu_util import C64, C128, dev_f64, dev_vec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [C128, C64])
def test_noalloc_region_norm_matches_plan_observables(prec):
    import torch

    import paper_0907_3022_gb300 as cb

    rb = wl.Ribbon(W=48, L=700, sigma=15.0)
    eps = dev_f64(rb.onsite())
    desc, keep = cb.desc_ribbons([rb.W], [rb.L], rb.hop, eps)
    nvec = 4
    plan = cb.Plan(desc, *[[x] for x in rb.bounds()], 0.0, prec, nvec, keep=keep)
    packets = np.stack([rb.packet(k) for k in wl.ENSEMBLE_K0], axis=1)
    psi_a = dev_vec(packets, prec)
    psi_b = psi_a.clone()
    plan.evolve(psi_b, rb.dt, 30)  # a spread-out second input
    # regions that hold real probability (a complex64 packet's far tail is exactly zero)
    for psi, col in ((psi_a, 160), (psi_b, -1), (psi_b, 200)):
        for _ in range(2):  # two calls in a row on the shared static scratch
            got = torch.full((nvec,), -1.0, dtype=torch.float64, device="cuda:0")
            cb.cheb_region_norm_noalloc(psi, prec, rb.W * rb.L, rb.L, nvec, col, got)
            ref = torch.zeros(nvec, dtype=torch.float64, device="cuda:0")
            kind = cb.CHEB_OBS_NORM2 if col < 0 else cb.CHEB_OBS_PROB_COLS
            plan.observables(psi, kind, float(col), ref)
            torch.cuda.synchronize()
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            assert np.all(r > 1e-3)
            assert np.max(np.abs(g - r) / r) <= 1e-12, (col, g, r)


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    import torch

    import paper_0907_3022_gb300 as cb

    n_sites = 16384 * 1024 + 1  # 16385 tiles x 4 vectors > 65536 partials
    psi = torch.zeros(n_sites * 4, dtype=torch.complex64, device="cuda:0")
    out = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    with pytest.raises(cb.ChebError) as e:
        cb.cheb_region_norm_noalloc(psi, cb.CHEB_C64, n_sites, 1024, 4, -1, out)
    assert e.value.status == cb.CHEB_ERR_INVALID
    assert "CHEB_NOALLOC_MAX_PARTIALS" in cb.lib().cheb_last_error().decode()
    # the largest admissible size still works
    cb.cheb_region_norm_noalloc(psi, cb.CHEB_C64, 16384 * 1024, 1024, 4, -1, out)
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0
