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
