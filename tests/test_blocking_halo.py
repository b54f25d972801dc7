"""The validity limit of the temporally blocked kernel on the brick wall (the ribbons of
Sec. 3.2): a site of a region may form order i of a launch only if every site it depends on
through i bonds lies inside the region.  The kernel takes, per site, the bond distance to the
region's open sides less one -- columns count one per site, rows 2d - 1 or 2d for d rows
depending on the direction of the site's vertical bond -- and cuts the row halo to ceil(s / 2).
Here that rule, restated, is checked against breadth-first search on random regions: it never
exceeds the exact distance to a site outside the region, and it changes by at most one along
a bond (so a site computed at order i reads neighbours valid at order i - 1)."""
import collections
import random

import pytest


def _neighbours(r, c, W, L):
    out = []
    if c > 0:
        out.append((r, c - 1))
    if c + 1 < L:
        out.append((r, c + 1))
    if (r + c) & 1:  # vertical bond up
        if r > 0:
            out.append((r - 1, c))
    elif r + 1 < W:
        out.append((r + 1, c))
    return out


def _limit(r, c, W, L, R0, R1, C0, C1):
    """The kernel's per-site limit (a large number where no side is open)."""
    rr, cc, up = r - R0, c - C0, (r + c) & 1
    RH, RW = R1 - R0, C1 - C0
    dl = 1 << 20
    if R0 > 0:
        dl = min(dl, 2 * rr + (0 if up else 1))
    if R1 < W:
        dl = min(dl, 2 * (RH - 1 - rr) + (1 if up else 0))
    if C0 > 0:
        dl = min(dl, cc)
    if C1 < L:
        dl = min(dl, RW - 1 - cc)
    return dl


def _random_region(rng):
    W, L = rng.randint(2, 24), rng.randint(2, 30)
    R0 = rng.randint(0, W - 1)
    R1 = rng.randint(R0 + 1, W)
    C0 = rng.randint(0, L - 1)
    C1 = rng.randint(C0 + 1, L)
    return W, L, R0, R1, C0, C1


def test_limit_never_exceeds_bond_distance():
    rng = random.Random(907)
    for _ in range(200):
        W, L, R0, R1, C0, C1 = _random_region(rng)
        dist, q = {}, collections.deque()
        for r in range(W):
            for c in range(L):
                if not (R0 <= r < R1 and C0 <= c < C1):
                    dist[(r, c)] = 0
                    q.append((r, c))
        while q:
            x = q.popleft()
            for y in _neighbours(*x, W, L):
                if y not in dist:
                    dist[y] = dist[x] + 1
                    q.append(y)
        for r in range(R0, R1):
            for c in range(C0, C1):
                lim = _limit(r, c, W, L, R0, R1, C0, C1)
                if (r, c) in dist:  # reachable from outside: limit <= distance - 1
                    assert lim <= dist[(r, c)] - 1, (W, L, R0, R1, C0, C1, r, c)


def test_limit_changes_by_at_most_one_along_a_bond():
    rng = random.Random(3022)
    for _ in range(200):
        W, L, R0, R1, C0, C1 = _random_region(rng)
        for r in range(R0, R1):
            for c in range(C0, C1):
                lim = _limit(r, c, W, L, R0, R1, C0, C1)
                for (a, b) in _neighbours(r, c, W, L):
                    if R0 <= a < R1 and C0 <= b < C1:
                        assert _limit(a, b, W, L, R0, R1, C0, C1) >= min(lim, 1 << 19) - 1
                    else:  # a site that is ever computed never reads outside the region
                        assert lim == 0 or lim >= 1 << 19


def test_row_halo_of_half_the_orders_suffices():
    """Interior rows sit ceil(s / 2) rows from an open row side: their limit is >= s."""
    for s in range(1, 17):
        hr = (s + 1) // 2
        W, L = 4 * hr + 3, 5
        R0, R1 = 1, W - 1  # both row sides open
        for r in range(R0 + hr, R1 - hr):
            for c in range(L):
                assert _limit(r, c, W, L, R0, R1, 0, L) >= s


# ---- the library's tile builder (host code, no GPU) -----------------------------------------
def _tiles(W, L, s, budget):
    import paper_0907_3022_gb300 as cb

    return cb.cheb_tb_tiles(W, L, s, budget)


def _check_tiles(W, L, s, budget):
    import numpy as np

    tiles = _tiles(W, L, s, budget)
    hr = (s + 1) // 2
    cover = np.zeros((W, L), dtype=np.int32)
    for R0, R1, C0, C1, r0, r1, c0, c1 in tiles.tolist():
        assert 0 <= R0 <= r0 < r1 <= R1 <= W and 0 <= C0 <= c0 < c1 <= C1 <= L
        assert (R1 - R0) * (C1 - C0) <= budget
        # halo: ceil(s/2) rows and s columns wherever the side is not a ribbon edge
        assert r0 - R0 == min(hr, r0) and R1 - r1 == min(hr, W - r1)
        assert c0 - C0 == min(s, c0) and C1 - c1 == min(s, L - c1)
        cover[r0:r1, c0:c1] += 1
        # every interior site keeps all s orders under the kernel's validity limit
        for r in range(r0, r1):
            for c in range(c0, c1):
                assert _limit(r, c, W, L, R0, R1, C0, C1) >= s
    assert (cover == 1).all()  # the interiors partition the ribbon
    return len(tiles)


def test_tiles_partition_the_ribbon_with_valid_interiors():
    for W, L in [(1, 1), (1, 300), (2, 3), (3, 5), (7, 230), (50, 60), (97, 41), (130, 30),
                 (160, 400), (77, 900), (40, 500)]:
        for s in (1, 2, 3, 5, 8, 10, 12):
            for budget in (1024, 3072, 8192):
                _check_tiles(W, L, s, budget)


def test_tiles_of_the_ensemble_ribbons():
    """All 64 ribbons of the default ensemble at the tuned shape (10 orders, 512 x 6 sites):
    the tile count the tuned launches process."""
    import workloads as wl

    ens = wl.RibbonEnsemble()
    total = 0
    for W, L in ens.sizes:
        total += len(_tiles(W, L, 10, 3072))
    for W, L in ens.sizes[:4]:  # the full per-site checks on a few of them
        _check_tiles(W, L, 10, 3072)
    assert total == 8445  # the first launch's CTA count in the DRAM capture of the profile


def test_tiles_rejected_when_one_column_does_not_fit():
    import paper_0907_3022_gb300 as cb

    with pytest.raises(cb.ChebError) as e:
        # a one-row band needs 1 + 2 x 5 rows and 1 + 2 x 10 columns: 231 > 100 sites
        cb.cheb_tb_tiles(300, 5000, 10, 100)
    assert e.value.status == cb.CHEB_ERR_INVALID
    with pytest.raises(cb.ChebError):
        cb.cheb_tb_tiles(0, 10, 4, 1024)


def test_tiles_span_row_bands_and_column_tiles():
    """At the shapes the ensemble benchmark times (8 or 10 orders; 6 x 512 or 3 x 1024 sites
    per region) the large ribbons of the GPU parity test are cut into >= 2 row bands and >= 2 column
    tiles (host-side tile builder of the library)."""
    import paper_0907_3022_gb300 as cb

    for s, spt, tpb in ((8, 6, 512), (10, 6, 512), (8, 3, 1024), (10, 3, 1024)):
        for W, L in ((158, 3177), (154, 3426), (131, 1999)):
            t = cb.cheb_tb_tiles(W, L, s, spt * tpb)
            assert len(set(t[:, 4].tolist())) >= 2, (s, spt, tpb, W, L)
            assert len(set(t[:, 6].tolist())) >= 2, (s, spt, tpb, W, L)


# ---- padded regions of the register-run kernel -----------------------------------------------
def _check_tiles_padded(W, L, s, positions, align, boxes):
    import numpy as np

    import paper_0907_3022_gb300 as cb

    tiles = cb.cheb_tb_tiles_padded(W, L, s, positions, align, boxes)
    hr = (s + 1) // 2
    cover = np.zeros((W, L), dtype=np.int32)
    if boxes:
        # one row stride and one box height for the whole ribbon: the widest tile's stride, the
        # tallest tile's rows, and together they fit the CTA's positions
        S_all, BH_all = set(tiles[:, 8].tolist()), set(tiles[:, 9].tolist())
        assert len(S_all) == 1 and len(BH_all) == 1
        S, BH = S_all.pop(), BH_all.pop()
        assert S % align == 0 and BH == max(tiles[:, 1] - tiles[:, 0])
        assert S == max((c1_ - c0_ + align) // align * align
                        for c0_, c1_ in zip(tiles[:, 2], tiles[:, 3]))
        assert 1 + BH * S <= positions
    for R0, R1, C0, C1, r0, r1, c0, c1, S, BH in tiles.tolist():
        assert 0 <= R0 <= r0 < r1 <= R1 <= W and 0 <= C0 <= c0 < c1 <= C1 <= L
        stride = (C1 - C0 + align) // align * align
        if not boxes:  # the tile's own stride and rows
            assert S == stride and BH == R1 - R0
        # at least one zero pad after every row, stride a multiple of align, and all rows plus
        # the trailing zero position fit the CTA's positions
        assert stride >= C1 - C0 + 1 and stride % align == 0 and stride - (C1 - C0) <= align
        assert 1 + (R1 - R0) * stride <= positions
        assert r0 - R0 == min(hr, r0) and R1 - r1 == min(hr, W - r1)
        assert c0 - C0 == min(s, c0) and C1 - c1 == min(s, L - c1)
        cover[r0:r1, c0:c1] += 1
        for r in range(r0, r1):
            for c in range(c0, c1):
                assert _limit(r, c, W, L, R0, R1, C0, C1) >= s
    assert (cover == 1).all()
    return len(tiles)


def test_padded_tiles_partition_the_ribbon_with_valid_interiors():
    for W, L in [(1, 1), (1, 300), (2, 3), (3, 5), (7, 230), (50, 60), (97, 41), (130, 30),
                 (160, 400), (40, 500)]:
        for s in (1, 3, 8, 10):
            for positions, align in ((1536, 4), (2304, 4), (2560, 4), (3072, 4), (5120, 8)):
                for boxes in (False, True):
                    _check_tiles_padded(W, L, s, positions, align, boxes)


def test_padded_tiles_rejected_when_one_column_does_not_fit():
    import paper_0907_3022_gb300 as cb

    with pytest.raises(cb.ChebError) as e:
        # rows of one interior column and a 10-column halo need a stride of 24: 11 x 24 + 1 > 200
        cb.cheb_tb_tiles_padded(300, 5000, 10, 200, 4)
    assert e.value.status == cb.CHEB_ERR_INVALID
    with pytest.raises(cb.ChebError):
        cb.cheb_tb_tiles_padded(10, 10, 4, 1024, 2)

