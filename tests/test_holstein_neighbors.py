"""Phonon neighbours of the matrix-free Holstein operator (Sec. 3.3), checked on the host.

The matrix-free kernels address the phonon terms of row (e, n) through the ranks of n + 1_e
and n - 1_e, obtained from the budgets R_j without ranking the new tuple.  The host entry point
cheb_holstein_phonon_neighbors runs the same routine; here it is compared with the oracle's
own enumeration of the basis (lexicographic order, n_0 most significant), where the rank of a
tuple is its position among the sorted base-(nph + 1) keys, and on the paper's 18-site basis
with the library's ranking on sampled tuples.  A wrong offset would send the kernels to a
wrong (or out-of-range) row, so every admissible neighbour and every boundary (sum n = nph,
n_e = 0) is checked.
"""
import math

import numpy as np
import pytest

import oracle
import paper_0907_3022_gb300 as cb


def _expected(occ: np.ndarray, nph: int):
    """(up, dn) ranks from the oracle enumeration, -1 where n +- 1_e is not admissible."""
    D, L = occ.shape
    w = (nph + 1) ** np.arange(L - 1, -1, -1, dtype=np.int64)  # n_0 most significant
    keys = occ.astype(np.int64) @ w
    assert np.all(np.diff(keys) > 0)  # the enumeration is the lexicographic order
    tot = occ.sum(axis=1)
    up = np.full((D, L), -1, np.int64)
    dn = np.full((D, L), -1, np.int64)
    for e in range(L):
        ok = tot < nph
        k = keys[ok] + w[e]
        pos = np.searchsorted(keys, k)
        assert np.array_equal(keys[pos], k)
        up[ok, e] = pos
        ok = occ[:, e] > 0
        k = keys[ok] - w[e]
        pos = np.searchsorted(keys, k)
        assert np.array_equal(keys[pos], k)
        dn[ok, e] = pos
    return up, dn


@pytest.mark.parametrize("L,nph", [(1, 3), (1, 15), (2, 5), (3, 2), (4, 3), (6, 4), (5, 15),
                                   (8, 6), (3, 0)])
def test_neighbors_match_oracle_enumeration(L, nph):
    H = oracle.holstein(L, nph, False, 1.0, 1.0, 1.0)
    occ = H.occupations()
    D = occ.shape[0]
    assert D == math.comb(nph + L, L)
    up, dn = cb.cheb_holstein_phonon_neighbors(L, nph, 0, D)
    eu, ed = _expected(occ, nph)
    assert np.array_equal(up, eu)
    assert np.array_equal(dn, ed)
    # raising and lowering are inverse to each other
    for e in range(L):
        ok = up[:, e] >= 0
        assert np.array_equal(dn[up[ok, e], e], np.nonzero(ok)[0])


def test_neighbors_partial_ranges_agree():
    L, nph = 6, 5
    D = cb.cheb_holstein_dim_phonon(L, nph)
    up, dn = cb.cheb_holstein_phonon_neighbors(L, nph, 0, D)
    for p0, cnt in [(0, 1), (17, 40), (D - 5, 5), (D, 0)]:
        u, d = cb.cheb_holstein_phonon_neighbors(L, nph, p0, cnt)
        assert np.array_equal(u, up[p0:p0 + cnt]) and np.array_equal(d, dn[p0:p0 + cnt])


def test_neighbors_paper_basis_sampled():
    """Sec. 3.3: 18 sites, at most 11 phonons (Dph = 34,597,290): sampled phonon ranks and
    the two ends of the basis against the library's ranking of n +- 1_e."""
    L, nph = 18, 11
    D = cb.cheb_holstein_dim_phonon(L, nph)
    assert D == 34_597_290
    rng = np.random.default_rng(3022)
    starts = [0, D - 64] + [int(x) for x in rng.integers(0, D - 64, size=14)]
    for p0 in starts:
        up, dn = cb.cheb_holstein_phonon_neighbors(L, nph, p0, 64)
        for i in range(64):
            _, occ = cb.cheb_holstein_unrank(L, nph, p0 + i)
            tot = int(occ.sum())
            for e in range(L):
                o = occ.copy()
                if tot < nph:
                    o[e] += 1
                    assert up[i, e] == cb.cheb_holstein_rank(L, nph, o, 0)
                else:
                    assert up[i, e] == -1
                o = occ.copy()
                if occ[e] > 0:
                    o[e] -= 1
                    assert dn[i, e] == cb.cheb_holstein_rank(L, nph, o, 0)
                else:
                    assert dn[i, e] == -1


def test_neighbors_limits():
    # the matrix-free limits: L <= 32, nph <= 15, Dph < 2^31
    up, dn = cb.cheb_holstein_phonon_neighbors(32, 3, 0, 4)
    assert up.shape == (4, 32)
    assert np.all(up[0] >= 1)  # from the vacuum every site can be raised
    assert np.all(dn[0] == -1)
    for L, nph, p0, cnt in [(33, 2, 0, 1), (4, 16, 0, 1), (0, 2, 0, 1), (4, 3, -1, 1),
                            (4, 3, 30, 6), (20, 15, 0, 1)]:
        with pytest.raises(cb.ChebError) as ex:
            cb.cheb_holstein_phonon_neighbors(L, nph, p0, cnt)
        assert ex.value.status == cb.CHEB_ERR_INVALID
