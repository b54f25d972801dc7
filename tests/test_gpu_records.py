"""Recorded norms and energies of complex64 plans are FP64 reductions.

cheb_evolve records (||psi||^2, <psi|H|psi>) per (ribbon, packet) before every obs_every-th
step.  For complex64 plans the record comes from an FP64 pass over the complex64 state (the
first recurrence launch's FP32 sums only feed the divergence check), so it must agree with an
FP64 reduction of the same complex64 values on the host:
  - ||psi||^2: the products of float32 values are exact in FP64, so the two sums differ only
    by FP64 summation order: relative difference <= 1e-12;
  - <psi|H|psi>: the plan applies H through its scaled diagonal d_i = 2 (eps_i - b)/a rounded
    to float32 (and the hopping in FP64), with the plan's own a; the host reference is the
    oracle's operator with the on-site energies eps'_i = d_i a/2 + b that this rounded diagonal
    represents, so the two again differ by summation order only: |difference| <= 1e-12
    (a ||psi||^2).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu_util import C64, C128, dev_f64, dev_vec

pytestmark = pytest.mark.gpu

SIZES = [(158, 3177), (43, 700), (1, 300), (97, 41), (3, 5)]


def _ensemble():
    return wl.RibbonEnsemble(n_ribbons=len(SIZES), sizes=list(SIZES))


def _state(ens):
    x = ens.packets()
    off = ens.offsets()
    for r in range(ens.n_ribbons):
        x[off[r]:off[r + 1], 3] = wl.random_state(int(off[r + 1] - off[r]), 17, r)
    return x.astype(np.complex64)


@pytest.mark.parametrize("blocking", [(10, 6, 512), (0, 4, 256)])
def test_complex64_records_equal_fp64_host_reductions(blocking):
    import torch

    import paper_0907_3022_gb300 as cb

    ens = _ensemble()
    x32 = _state(ens)
    W = [w for w, _ in ens.sizes]
    L = [l for _, l in ens.sizes]
    eps = ens.onsite()
    desc, keep = cb.desc_ribbons(W, L, ens.hop, dev_f64(eps))
    lo, hi = ens.bounds()
    plan = cb.Plan(desc, lo, hi, 0.0, cb.CHEB_C64, ens.nvec, keep=keep)
    psi = dev_vec(x32, C64)
    plan.evolve(psi, ens.dt, 0)
    plan.set_blocking(*blocking)
    nrec = 3
    rec = torch.zeros((nrec, ens.n_ribbons, ens.nvec, 2), dtype=torch.float64, device="cuda:0")
    plan.evolve(psi, ens.dt, 2 * nrec, 2, rec)
    r = rec.cpu().numpy()
    # record 0 is the initial state, exactly known on the host
    x = x32.astype(np.complex128)
    off = ens.offsets()
    for q in range(ens.n_ribbons):
        rb = ens.ribbon(q)
        # the plan's own rescaling (complex64 lattice plans enlarge a by under one float32 ulp
        # so that the scaled hopping is a float32 number)
        a, b = plan.block(q)["a"], plan.block(q)["b"]
        a0, b0 = oracle.rescale(*rb.bounds(), 0.0)
        assert b == b0 and a0 <= a <= a0 * (1 + 2.0 ** -22)
        # 2 h / a (h = -1) is a float32 number, up to the double rounding of a itself
        assert abs(float(np.float32(-2.0 / a)) + 2.0 / a) <= 1e-15
        d32 = (2.0 * (rb.onsite() - b) / a).astype(np.float32)
        H = oracle.honeycomb(rb.W, rb.L, rb.hop, d32.astype(np.float64) * (a / 2.0) + b)
        for v in range(ens.nvec):
            xs = x[off[q]:off[q + 1], v]
            n2 = float(np.sum(xs.real ** 2 + xs.imag ** 2))
            _, e = H.norm_energy(xs)
            assert abs(r[0, q, v, 0] - n2) <= 1e-12 * n2, (q, v, r[0, q, v, 0], n2)
            assert abs(r[0, q, v, 1] - e) <= 1e-12 * a * n2, (q, v, r[0, q, v, 1], e)
    # later records: norm conserved within the complex64 tolerance
    assert np.max(np.abs(r[:, :, :, 0] / r[0:1, :, :, 0] - 1.0)) <= 1e-5
    plan.close()


@pytest.mark.parametrize("matrix_free", [False, True])
def test_complex64_holstein_record_norm_is_fp64(matrix_free):
    import torch

    import paper_0907_3022_gb300 as cb

    hs = wl.Holstein(L=6, nph=5)
    desc = cb.desc_holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g,
                            matrix_free=matrix_free)
    plan = cb.Plan(desc, [hs.bounds()[0]], [hs.bounds()[1]], hs.alpha, cb.CHEB_C64, 1)
    x32 = wl.random_state(hs.dim, 5, 0).astype(np.complex64)
    psi = dev_vec(x32, C64)
    rec = torch.zeros((2, 1, 1, 2), dtype=torch.float64, device="cuda:0")
    plan.evolve(psi, hs.dt, 2, 1, rec)
    x = x32.astype(np.complex128)
    n2 = float(np.sum(x.real ** 2 + x.imag ** 2))
    r = rec.cpu().numpy()
    assert abs(r[0, 0, 0, 0] - n2) <= 1e-12 * n2
    # the energy record equals cheb_observables' FP64 energy of the same state
    e = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    plan.observables(dev_vec(x32, C64), cb.CHEB_OBS_ENERGY, 0.0, e)
    assert abs(r[0, 0, 0, 1] - float(e.item())) <= 1e-12 * max(1.0, abs(float(e.item())))
    # and agrees with the oracle's FP64 energy within the float32 rounding of the matrix
    H = oracle.holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g)
    _, e_ref = H.norm_energy(x)
    a, _ = oracle.rescale(*hs.bounds(), hs.alpha)
    assert abs(r[0, 0, 0, 1] - e_ref) <= 1e-6 * a * n2
    plan.close()


def test_complex128_records_unchanged():
    """complex128 plans keep the first launch's FP64 sums as their record."""
    import torch

    import paper_0907_3022_gb300 as cb

    rb = wl.Ribbon(W=16, L=90, sigma=5.0)
    desc, keep = cb.desc_ribbons([rb.W], [rb.L], 1.0, dev_f64(rb.onsite()))
    plan = cb.Plan(desc, *[[v] for v in rb.bounds()], 0.0, cb.CHEB_C128, 1, keep=keep)
    x = rb.packet()
    rec = torch.zeros((1, 1, 1, 2), dtype=torch.float64, device="cuda:0")
    plan.evolve(dev_vec(x, C128), rb.dt, 1, 1, rec)
    n2, e = oracle.honeycomb(rb.W, rb.L, 1.0, rb.onsite()).norm_energy(x)
    assert abs(rec[0, 0, 0, 0].item() - n2) <= 1e-13 and abs(rec[0, 0, 0, 1].item() - e) <= 1e-12
    plan.close()
