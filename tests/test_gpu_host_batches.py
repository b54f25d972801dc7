"""cheb_evolve_host: batches of independent states served from host memory, with the copies
overlapping the propagation.  Every job must equal the same propagation done on the device
with cheb_evolve (same kernels, same graphs: bit for bit)."""
import numpy as np
import pytest

import workloads as wl
from _gpu_util import C64, C128, dev_f64, dev_vec, host

pytestmark = pytest.mark.gpu


def _ensemble_plan(cb):
    rbs = [wl.Ribbon(W=14, L=70, sigma=4.0, stream=q) for q in range(3)]
    eps = dev_f64(np.concatenate([rb.onsite() for rb in rbs]))
    desc, keep = cb.desc_ribbons([rb.W for rb in rbs], [rb.L for rb in rbs], 1.0, eps)
    plan = cb.Plan(desc, [rb.bounds()[0] for rb in rbs], [rb.bounds()[1] for rb in rbs], 0.0,
                   C64, 4, keep=keep)
    k0s = (np.pi / 6, np.pi / 4, np.pi / 3, np.pi / 2)
    X = np.concatenate([np.stack([rb.packet(k) for k in k0s], axis=1) for rb in rbs])
    return plan, X


@pytest.mark.parametrize("blocking", [0, 3])
def test_host_jobs_equal_device_evolution(blocking):
    import torch

    import paper_0907_3022_gb300 as cb

    plan, X = _ensemble_plan(cb)
    plan.evolve(dev_vec(X, C64), 1.0, 0)
    plan.set_blocking(blocking, 4)
    rng = np.random.default_rng(11)
    jobs = [X * np.exp(1j * rng.uniform(0, 6.28)) * (1.0 + 0.1 * j) for j in range(3)]
    jobs[2] = jobs[2][::-1].copy()  # a different shape of state
    nsteps = 3
    ref = []
    for x in jobs:
        d = dev_vec(x, C64)
        plan.evolve(d, 1.0, nsteps)
        ref.append(host(d))
    hin = torch.from_numpy(np.stack(jobs).astype(np.complex64)).pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    plan.evolve_host(hin, hout, 3, 1.0, nsteps)
    for j in range(3):
        assert np.array_equal(hout[j].numpy().astype(np.complex128), ref[j])
    # in place (same buffer, same stride), pageable numpy buffers
    buf = np.stack(jobs).astype(np.complex64)
    plan.evolve_host(buf, buf, 3, 1.0, nsteps)
    for j in range(3):
        assert np.array_equal(buf[j].astype(np.complex128), ref[j])
    # stride 0: every job reads the same state and writes the same slot
    one_in = torch.from_numpy(jobs[1].astype(np.complex64)).pin_memory()
    one_out = torch.zeros_like(one_in).pin_memory()
    plan.evolve_host(one_in, one_out, 5, 1.0, nsteps, in_stride=0, out_stride=0)
    assert np.array_equal(one_out.numpy().astype(np.complex128), ref[1])
    # nsteps = 0 copies through; the plan's own graphs still work afterwards
    plan.evolve_host(one_in, one_out, 2, 1.0, 0, in_stride=0, out_stride=0)
    assert np.array_equal(one_out.numpy(), one_in.numpy())
    d = dev_vec(jobs[0], C64)
    plan.evolve(d, 1.0, nsteps)
    assert np.array_equal(host(d), ref[0])


def test_host_jobs_complex128_and_errors():
    import torch

    import paper_0907_3022_gb300 as cb

    dw = wl.DoubleWell1D(n=256)
    V = dev_f64(dw.potential())
    lo, hi = dw.bounds()
    plan = cb.Plan(cb.desc_lat1d(dw.n, dw.dx, V), [lo], [hi], 0.01, C128, 1, keep=(V,))
    x = dw.packet()
    d = dev_vec(x, C128)
    plan.evolve(d, dw.dt, 4)
    hin = torch.from_numpy(np.stack([x, x])).pin_memory()
    hout = torch.zeros_like(hin).pin_memory()
    plan.evolve_host(hin, hout, 2, dw.dt, 4)
    assert np.array_equal(hout[1].numpy(), host(d))
    with pytest.raises(cb.ChebError) as e:  # aliasing with stride 0
        plan.evolve_host(hin, hin, 2, dw.dt, 1, in_stride=0, out_stride=0)
    assert e.value.status == cb.CHEB_ERR_INVALID
    with pytest.raises(cb.ChebError) as e:  # stride shorter than a state
        plan.evolve_host(hin, hout, 2, dw.dt, 1, in_stride=16, out_stride=4096)
    assert e.value.status == cb.CHEB_ERR_INVALID
    with pytest.raises(ValueError):  # host buffer too small for the jobs
        plan.evolve_host(hin, hout, 3, dw.dt, 1)
