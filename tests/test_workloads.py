"""The seeded input generators: SplitMix64 against its published outputs, and the shapes of
the synthetic workloads."""
import math

import numpy as np

import workloads as wl


def test_splitmix64_published_outputs():
    """SplitMix64 (Steele, Lea, Flood 2014) seeded with 0 starts 0xE220A8397B1DCDAF,
    0x6E789E6AA1B965F4, 0x06C45D188009454F."""
    x = wl.splitmix64(0, 0, 3)
    assert [int(v) for v in x] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_and_uniforms():
    a = wl.splitmix64(907, 3, 5)
    b = wl.splitmix64(907 + (3 << 32), 0, 5)
    assert np.array_equal(a, b)
    u = wl.uniform01(1, 0, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    eps = wl.anderson_disorder(100000, 2.0, 5)
    assert eps.min() >= -1.0 and eps.max() < 1.0


def test_ensemble_shape():
    ens = wl.RibbonEnsemble()
    assert len(ens.sizes) == 64
    assert all(40 <= w <= 160 and 500 <= l <= 4000 for w, l in ens.sizes)
    assert ens.n_sites == 15_485_892
    assert ens.offsets()[-1] == ens.n_sites
    shifted = wl.RibbonEnsemble(stream0=64)
    assert shifted.sizes == ens.sizes
    assert not np.array_equal(shifted.ribbon(0).onsite(), ens.ribbon(0).onsite())


def test_packets_and_grid():
    rb = wl.Ribbon(W=16, L=64, sigma=5.0)
    p = rb.packet()
    assert abs(np.linalg.norm(p) - 1.0) < 1e-14
    d = wl.DoubleWell1D()
    assert abs(d.dx - 40 / 2048) < 1e-16 and d.nsteps == 100
    assert abs(np.linalg.norm(d.packet()) - 1.0) < 1e-14
    h = wl.Holstein()
    assert h.dim == 12 * math.comb(22, 10) == 7_759_752
    lo, hi = h.bounds()
    assert abs(lo + 4.7194) < 1e-4 and abs(hi - 20.2434) < 1e-4
