"""The temporally blocked recurrence at the launch shapes the ensemble benchmark runs (8 to 12
orders per launch; the blocked kernels at their tuned CTA shapes, the register-run one with
per-thread copies and with tensor-memory-access boxes), element by
element against the FP64 oracle, on ribbons whose tiles need several row bands and several
column tiles, so that the row halo (ceil(s/2) rows), the column halo (s columns), ragged last
bands and columns and the merged last launch of a step are all exercised.

Inputs: the two widest and largest ribbons of the 64-ribbon ensemble (158 x 3177, 154 x 3426),
an odd-sized 131 x 1999 ribbon and small edge shapes, with Anderson disorder from the
ensemble's streams; packets 0-2 are the ensemble's Gaussian packets (k0 = pi/6, pi/4, pi/3),
packet 3 a seeded random state that occupies every site (so every tile border carries
amplitude).  Tolerance: complex64 relative L2 <= 1e-4 per (ribbon, packet) and every element
within 1e-4 of the packet's largest amplitude.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu_util import C64, dev_f64, dev_vec, host, rel

pytestmark = pytest.mark.gpu

SIZES = [(158, 3177), (154, 3426), (131, 1999), (1, 300), (3, 5), (97, 41), (7, 230), (130, 30),
         (2, 3), (1, 1)]
NSTEPS = 10
SITES, RUNS, RUNS_TMA = 0, 1, 2
# (orders per launch, sites per thread, threads, kernel): the strided-site kernel's tuned
# shapes and the register-run kernel's, with per-thread copies and with boxes
SHAPES = [(8, 6, 512, SITES), (10, 6, 512, SITES), (8, 3, 1024, SITES), (10, 3, 1024, SITES),
          (8, 7, 384, RUNS), (10, 7, 384, RUNS), (10, 9, 256, RUNS), (12, 9, 256, RUNS),
          (10, 3, 768, RUNS), (10, 7, 384, RUNS_TMA), (12, 9, 256, RUNS_TMA),
          (10, 5, 512, RUNS_TMA)]

_cache = {}


def _ensemble():
    return wl.RibbonEnsemble(n_ribbons=len(SIZES), sizes=list(SIZES),
                             k0s=wl.ENSEMBLE_K0[:4])


def _packets(ens):
    x = ens.packets()
    off = ens.offsets()
    for r in range(ens.n_ribbons):
        x[off[r]:off[r + 1], 3] = wl.random_state(int(off[r + 1] - off[r]), 4242, r)
    return x


def _oracle(ens, x0):
    """FP64 oracle after NSTEPS steps for every (ribbon, packet); computed once."""
    if "ref" not in _cache:
        off = ens.offsets()
        out = np.empty_like(x0)
        Ms = []
        for r in range(ens.n_ribbons):
            rb = ens.ribbon(r)
            H = oracle.honeycomb(rb.W, rb.L, rb.hop, rb.onsite())
            a, b = oracle.rescale(*rb.bounds(), 0.0)
            C, M = oracle.coeffs(a, b, rb.dt)
            Ms.append(M)
            for v in range(ens.nvec):
                out[off[r]:off[r + 1], v] = H.evolve(a, b, C, NSTEPS, x0[off[r]:off[r + 1], v])
        _cache["ref"] = (out, Ms)
    return _cache["ref"]


def _plan(cb, ens):
    W = [w for w, _ in ens.sizes]
    L = [l for _, l in ens.sizes]
    eps = dev_f64(ens.onsite())
    desc, keep = cb.desc_ribbons(W, L, ens.hop, eps)
    lo, hi = ens.bounds()
    return cb.Plan(desc, lo, hi, 0.0, cb.CHEB_C64, ens.nvec, keep=keep)


@pytest.mark.parametrize("s,spt,tpb,kernel", SHAPES)
def test_blocked_timed_shape_matches_oracle(s, spt, tpb, kernel):
    import paper_0907_3022_gb300 as cb

    ens = _ensemble()
    x0 = _packets(ens)
    ref, Ms = _oracle(ens, x0)
    plan = _plan(cb, ens)
    psi = dev_vec(x0, C64)
    plan.evolve(psi, ens.dt, 0)
    plan.set_blocking_kernel(s, spt, tpb, kernel)
    assert plan.blocking_shape() == (s, spt, tpb) and plan.blocking_kernel() == kernel
    assert [plan.block(q)["M"] for q in range(ens.n_ribbons)] == Ms
    plan.evolve(psi, ens.dt, NSTEPS)
    out = host(psi)
    off = ens.offsets()
    for r in range(ens.n_ribbons):
        for v in range(ens.nvec):
            g, e = out[off[r]:off[r + 1], v], ref[off[r]:off[r + 1], v]
            assert rel(g, e) <= 1e-4, (r, v, rel(g, e))
            assert np.max(np.abs(g - e)) <= 1e-4 * np.max(np.abs(e)), (r, v)
    # the same plan with single-order launches: same recurrence, partial sums in another order
    plan.set_blocking(0, 4, 256)
    psi2 = dev_vec(x0, C64)
    plan.evolve(psi2, ens.dt, NSTEPS)
    assert rel(out, host(psi2)) <= 2e-6
    plan.close()
