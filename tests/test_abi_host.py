"""C ABI checks that need no GPU: the library loads, exports every function include/cheb.h
declares, and its host-side arithmetic (Sec. 2.2 rescaling and coefficients, the Holstein
basis ranking of Sec. 3.3) agrees with the oracle."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import paper_0907_3022_gb300 as cb


def test_library_exports_every_declared_symbol():
    names = cb.header_functions()
    assert len(names) >= 20
    L = cb.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(cb._cheb._SIGS)


def test_rescale_matches_oracle():
    for emin, emax, alpha in [(-3.5, 3.5, 0.0), (0.9, 24461.8, 0.01), (-4.72, 20.24, 0.01)]:
        a1, b1 = cb.cheb_rescale(emin, emax, alpha)
        a2, b2 = oracle.rescale(emin, emax, alpha)
        assert abs(a1 - a2) <= 2e-16 * abs(a2) and abs(b1 - b2) <= 2e-16 * max(1, abs(b2))


def test_rescale_errors():
    with pytest.raises(cb.ChebError) as e:
        cb.cheb_rescale(1.0, 0.0, 0.01)
    assert e.value.status == cb.CHEB_ERR_INVALID
    assert "emin" in cb.lib().cheb_last_error().decode()


@pytest.mark.parametrize("a,b,dt", [(3.25, 0.0, 1.0), (3.5, 0.0, 1.0), (4.0, 0.0, 1.0),
                                    (12.6138, 7.76, 0.25), (40.0, -3.0, 0.9)])
def test_coeffs_match_oracle(a, b, dt):
    C1, M1 = cb.cheb_coeffs(a, b, dt, 1e-14)
    C2, M2 = oracle.coeffs(a, b, dt, 1e-14)
    assert M1 == max(M2, 2)
    assert np.max(np.abs(C1 - C2)) < 2e-15


def test_coeffs_large_argument_matches_oracle():
    """The 1D grid's z = a dt = 6176.4: Miller recurrence vs the oracle's quadrature."""
    import workloads as wl
    d = wl.DoubleWell1D()
    a, b = oracle.rescale(*d.bounds(), 0.01)
    C1, M1 = cb.cheb_coeffs(a, b, d.dt, 1e-14)
    C2, M2 = oracle.coeffs(a, b, d.dt, 1e-14)
    assert M1 == M2 == 6353
    assert np.max(np.abs(C1 - C2)) < 1e-13


def test_coeffs_errors():
    with pytest.raises(cb.ChebError) as e:
        cb.cheb_coeffs(6000.0, 0.0, 1.0, 1e-14, max_order=100)
    assert e.value.status == cb.CHEB_ERR_ORDER
    with pytest.raises(cb.ChebError):
        cb.cheb_coeffs(-1.0, 0.0, 1.0)


def test_coeffs_small_z_keeps_two_orders():
    C, M = cb.cheb_coeffs(1e-9, 0.0, 1.0, 1e-14)
    assert M == 2
    assert abs(C[0] - 1.0) < 1e-15


@pytest.mark.parametrize("L,nph", [(1, 5), (3, 2), (4, 3), (5, 4), (12, 2)])
def test_holstein_rank_bit_exact_vs_oracle_enumeration(L, nph):
    H = oracle.holstein(L, nph, False, 1.0, 1.0, 1.0)
    D = H.dim_phonon
    assert cb.cheb_holstein_dim_phonon(L, nph) == D == math.comb(nph + L, L)
    occ = H.occupations()
    for p in range(D):
        for e in (0, L - 1):
            idx = cb.cheb_holstein_rank(L, nph, occ[p], e)
            assert idx == e * D + p
            e2, o2 = cb.cheb_holstein_unrank(L, nph, idx)
            assert e2 == e and np.array_equal(o2, occ[p])


def test_holstein_rank_config_sizes():
    """L = 12, nph = 10: D = 12 * C(22, 10) = 7,759,752; the paper's 18 sites / 11 phonons
    give 622,751,220 (Sec. 3.3: D_tot = 6.2e8)."""
    assert 12 * cb.cheb_holstein_dim_phonon(12, 10) == 7_759_752
    assert 18 * cb.cheb_holstein_dim_phonon(18, 11) == 622_751_220
    # n_0 is the most significant entry: (0, ..., 0, v) are the first 11 tuples and
    # (10, 0, ..., 0) is the last one
    occ = np.zeros(12, np.uint8)
    occ[-1] = 10
    assert cb.cheb_holstein_rank(12, 10, occ, 0) == 10
    occ = np.zeros(12, np.uint8)
    occ[0] = 10
    assert cb.cheb_holstein_rank(12, 10, occ, 11) == 11 * 646_646 + 646_645


def test_holstein_rank_errors():
    with pytest.raises(cb.ChebError):
        cb.cheb_holstein_rank(3, 2, np.array([1, 1, 1], np.uint8), 0)
    with pytest.raises(cb.ChebError):
        cb.cheb_holstein_unrank(3, 2, 3 * 10, )
