"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper it pins and the independent fact it uses: a closed
form, an identity, a textbook special case, or a library routine (numpy/scipy LAPACK, scipy's
Bessel functions).  The set is chosen so that a dropped term, a wrong sign, a wrong index or a
transposed operand anywhere in the oracle fails at least one test.
"""
import math

import numpy as np
import pytest
from scipy.special import jv

import oracle
import workloads as wl


def ipow(k, sign=1):
    """Exact (sign*i)^k for an integer array k (numpy's complex power rounds for large k)."""
    tab = np.array([1, 1j, -1, -1j]) if sign > 0 else np.array([1, -1j, -1, 1j])
    return tab[np.asarray(k) % 4]


# --------------------------------------------------------------------------------------
# Sec. 2.2, rescaling: |E~| <= 1/(1+alpha) for the rescaled spectrum
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("alpha", [0.0, 0.01, 0.3])
def test_rescale_maps_spectrum_inside(alpha):
    rng = np.random.default_rng(1)
    E = np.sort(rng.normal(size=50) * 7 + 3)
    a, b = oracle.rescale(E[0], E[-1], alpha)
    Et = (E - b) / a
    assert np.max(np.abs(Et)) <= 1.0 / (1.0 + alpha) * (1 + 1e-15)
    assert np.isclose(np.max(np.abs(Et)), 1.0 / (1.0 + alpha), rtol=1e-14)
    assert np.isclose(Et[0], -Et[-1], rtol=1e-13)


def test_rescale_rejects_bad_bounds():
    with pytest.raises(ValueError):
        oracle.rescale(2.0, 1.0, 0.01)


# --------------------------------------------------------------------------------------
# Sec. 2.2, Eq. (c_k): c_k(z) = (-i)^k J_k(z)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("z", [0.0, 0.5, 3.25, 3.5, 4.0, 40.0])
def test_coeffs_match_library_bessel(z):
    km = oracle.default_kmax(z)
    c = oracle.bessel_coeffs(z, km)
    k = np.arange(km + 1)
    ref = ipow(k, -1) * jv(k, z)
    assert np.max(np.abs(c - ref)) < 2e-15


@pytest.mark.parametrize("z", [0.7, 3.5, 40.0, 600.0])
def test_coeffs_jacobi_anger(z):
    """e^{-izx} = c_0 + 2 sum_k c_k T_k(x) on [-1, 1] (the expansion Eq. (U_1) rests on)."""
    km = oracle.default_kmax(z)
    c = oracle.bessel_coeffs(z, km)
    x = np.cos(np.linspace(0, np.pi, 257))
    theta = np.arccos(x)
    k = np.arange(km + 1)
    T = np.cos(np.outer(theta, k))
    series = T @ (c * np.where(k == 0, 1.0, 2.0))
    assert np.max(np.abs(series - np.exp(-1j * z * x))) < 1e-13 * max(1.0, z / 40)


@pytest.mark.parametrize("z", [3.5, 600.0, 6176.385945851491])
def test_coeffs_bessel_sum_rules(z):
    """J_0 + 2 sum J_2k = 1 and J_0^2 + 2 sum J_k^2 = 1, at any z (incl. the 1D grid's z)."""
    km = oracle.default_kmax(z)
    c = oracle.bessel_coeffs(z, km)
    k = np.arange(km + 1)
    J = np.real(c * ipow(k))  # undo (-i)^k
    assert np.max(np.abs(np.imag(c * ipow(k)))) < 1e-15
    assert abs(J[0] + 2 * J[2::2].sum() - 1.0) < 1e-13
    assert abs(J[0] ** 2 + 2 * (J[1:] ** 2).sum() - 1.0) < 1e-13


@pytest.mark.parametrize("z", [3.5, 600.0, 6176.385945851491])
def test_coeffs_three_term_recurrence(z):
    """J_{k-1} + J_{k+1} = (2k/z) J_k."""
    km = oracle.default_kmax(z)
    c = oracle.bessel_coeffs(z, km)
    k = np.arange(km + 1)
    J = np.real(c * ipow(k))
    lhs = J[:-2] + J[2:]
    rhs = 2 * k[1:-1] / z * J[1:-1]
    assert np.max(np.abs(lhs - rhs)) < 2e-13 * max(1.0, math.sqrt(z) / 10)


def test_coeffs_asymptotic_decay():
    """Eq. (dec_Bessel): J_k(z) ~ (e z / 2k)^k / sqrt(2 pi k) for k >> z."""
    z = 2.0
    c = oracle.bessel_coeffs(z, 40)
    for k in range(8, 17):
        asym = (math.e * z / (2 * k)) ** k / math.sqrt(2 * math.pi * k)
        # leading-order form: relative corrections (z/2)^2/(k+1) and 1/(12k)
        assert abs(abs(c[k]) / asym - 1.0) < 1.5 * ((z / 2) ** 2 / (k + 1) + 1 / (12 * k))


def test_coeffs_truncation_rule_and_phase():
    """C_k = e^{-i b dt} (2 - delta_k0) (-i)^k J_k(a dt); M = last k with |C_k| >= tol."""
    a, b, dt, tol = 3.5, 0.7, 1.0, 1e-14
    C, M = oracle.coeffs(a, b, dt, tol)
    k = np.arange(M + 1)
    ref = np.exp(-1j * b * dt) * np.where(k == 0, 1, 2) * ipow(k, -1) * jv(k, a * dt)
    assert np.max(np.abs(C - ref)) < 3e-15
    assert abs(C[M]) >= tol
    tail = 2 * np.abs(jv(np.arange(M + 1, M + 40), a * dt))
    assert np.all(tail < tol)


def test_coeffs_1d_grid_order():
    """The double-well grid (N=2048 on [-20, 20), alpha = 0.01, dt = 0.5) needs M = 6353."""
    d = wl.DoubleWell1D()
    lo, hi = d.bounds()
    a, b = oracle.rescale(lo, hi, 0.01)
    C, M = oracle.coeffs(a, b, d.dt)
    assert M == 6353
    # the Bessel sum rule over the kept terms: sum |C_k / 2|^2 (k >= 1) + |C_0|^2 = 1
    assert abs(abs(C[0]) ** 2 + 0.5 * np.sum(np.abs(C[1:]) ** 2) - 1.0) < 1e-12


# --------------------------------------------------------------------------------------
# Sec. 3.1: 1D finite-difference Hamiltonian
# --------------------------------------------------------------------------------------
def test_lattice1d_free_spectrum_closed_form():
    """V = 0 with Dirichlet ends: E_j = (1 - cos(j pi/(N+1))) / dx^2, j = 1..N."""
    n, dx = 60, 0.3
    H = oracle.lattice1d(n, dx, np.zeros(n))
    E = np.linalg.eigvalsh(H.dense())
    j = np.arange(1, n + 1)
    ref = np.sort((1 - np.cos(j * np.pi / (n + 1))) / dx ** 2)
    assert np.max(np.abs(E - ref)) < 1e-12


def test_lattice1d_harmonic_levels():
    """V = x^2/2: lowest levels -> n + 1/2 up to the O(dx^2) error of the 3-point stencil."""
    n = 400
    x = np.linspace(-10, 10, n, endpoint=False)
    dx = x[1] - x[0]
    H = oracle.lattice1d(n, dx, 0.5 * x ** 2)
    E = np.linalg.eigvalsh(H.dense())[:5]
    assert np.max(np.abs(E - (np.arange(5) + 0.5))) < 0.5 * dx ** 2 * 5


def test_lattice1d_free_propagator_closed_form():
    """On the infinite grid with V = 0, <n|e^{-iHt}|m> = e^{-i t/dx^2} i^{n-m} J_{n-m}(t/dx^2).
    The packet stays far from the walls, so the finite grid agrees to the Chebyshev accuracy.
    This pins the sign of the time evolution (e^{-iHt}, a packet with k0 > 0 moves right)."""
    n, dx, t = 600, 1.0, 20.0
    x = np.arange(n) * dx
    psi0 = np.exp(-((x - 250) ** 2) / (2 * 8.0 ** 2) + 1j * 0.8 * x)
    psi0 /= np.linalg.norm(psi0)
    H = oracle.lattice1d(n, dx, np.zeros(n))
    a, b = oracle.rescale(0.0, 2.0 / dx ** 2, 0.01)
    C, M = oracle.coeffs(a, b, t / 4)
    psi = H.evolve(a, b, C, 4, psi0)
    lag = np.arange(-n + 1, n)
    kern = np.exp(-1j * t / dx ** 2) * ipow(lag) * jv(lag, t / dx ** 2)
    ref = np.array([np.sum(kern[i - np.arange(n) + n - 1] * psi0) for i in range(n)])
    assert np.linalg.norm(psi - ref) < 1e-12
    com0 = np.sum(x * np.abs(psi0) ** 2)
    com = np.sum(x * np.abs(psi) ** 2)
    assert com - com0 > 0.5 * t * math.sin(0.8)  # group velocity sin(k0)/dx^2 * dx^2


def test_propagator_matches_exact_diagonalisation_1d():
    """Sec. 2.1 vs Sec. 2.2 on the double-well grid at N = 256 (t = 50, 100 steps): the
    Chebyshev result reproduces exp(-iHt) psi within the paper's quoted 2e-11."""
    d = wl.DoubleWell1D(n=256)
    lo, hi = d.bounds()
    a, b = oracle.rescale(lo, hi, 0.01)
    C, M = oracle.coeffs(a, b, d.dt)
    H = oracle.lattice1d(d.n, d.dx, d.potential())
    psi = H.evolve(a, b, C, d.nsteps, d.packet())
    E, V = np.linalg.eigh(H.dense())
    ex = V @ (np.exp(-1j * E * d.t_end) * (V.T @ d.packet()))
    assert np.max(np.abs(psi - ex)) < 2e-11
    assert np.linalg.norm(psi - ex) / np.linalg.norm(ex) < 2e-11


def _tridiagonal_exact(d, e, psi0, t):
    """exp(-iHt) psi0 for the real symmetric tridiagonal H by full diagonalisation (LAPACK)."""
    from scipy.linalg import eigh_tridiagonal

    E, V = eigh_tridiagonal(d, e)
    return V @ (np.exp(-1j * E * t) * (V.T @ psi0))


def test_paper_double_well_accuracy_claim():
    """Sec. 3.1: N = 2048, M = 1500 moments at dt = 0.4, t = 40; the Chebyshev wave function
    agrees with full diagonalisation to an absolute error below 2e-11 (the paper's
    normalisation: psi_i / sqrt(dx)).  Also the physics of the set-up: the packet starts
    below the barrier and part of it tunnels to the right well."""
    d = wl.PaperDoubleWell()
    lo, hi = d.bounds()
    a, b = oracle.rescale(lo, hi, 0.01)
    C, M = oracle.coeffs(a, b, d.dt)
    assert M == 1499  # 1500 moments c_0 .. c_1499
    H = oracle.lattice1d(d.n, d.dx, d.potential())
    x0 = d.packet()
    psi = H.evolve(a, b, C, d.nsteps, x0)
    dd, ee = d.tridiagonal()
    ex = _tridiagonal_exact(dd, ee, x0, d.t_end)
    assert np.max(np.abs(psi - ex)) / math.sqrt(d.dx) < 2e-11
    n2, E0 = H.norm_energy(x0)
    assert abs(n2 - 1.0) < 1e-14 and 0.5 < E0 < d.V0  # below the barrier V(0) = V0
    assert np.min(d.potential()) > -1e-3 and abs(d.potential()[d.n // 2] - d.V0) < 1e-12
    right = np.sum(np.abs(ex[d.x > 0]) ** 2)
    assert 0.02 < right < 0.5


def test_piecewise_uniform_shift_closed_form():
    """H(t) = H_0 + v(t) 1 with v linear in t: exp(-i int v) exp(-i H_0 T) psi exactly, and
    the midpoint rule integrates a linear v without error, so the piecewise-constant
    propagation reproduces the closed form to rounding."""
    d = wl.DoubleWell1D(n=128, x_lo=-8.0, x_hi=8.0)
    V0 = d.potential()
    dt, nsteps, v0, v1 = 0.05, 40, 0.3, -0.7
    T = dt * nsteps
    tm = (np.arange(nsteps) + 0.5) * dt
    lo, hi = d.bounds()
    lo, hi = lo + min(v0, v0 + v1 * T), hi + max(v0, v0 + v1 * T)
    a, b = oracle.rescale(lo, hi, 0.01)
    C, _ = oracle.coeffs(a, b, dt)
    seq = [V0 + v0 + v1 * t for t in tm]
    psi = oracle.evolve_piecewise(lambda V: oracle.lattice1d(d.n, d.dx, V), seq, a, b, C,
                                  d.packet())
    dd, ee = d.tridiagonal()
    ex = np.exp(-1j * (v0 * T + 0.5 * v1 * T * T)) * _tridiagonal_exact(dd, ee, d.packet(), T)
    assert np.max(np.abs(psi - ex)) < 1e-12


def _driven_well(n=96):
    """Double well with a field F sin(Omega t) x switched on (does not commute with H_0)."""
    d = wl.DoubleWell1D(n=n, x_lo=-6.0, x_hi=6.0)
    F, Om = 0.8, 1.3
    return d, (lambda t: d.potential() + F * math.sin(Om * t) * d.x), F * np.max(np.abs(d.x))


def test_piecewise_midpoint_converges_to_schroedinger_solution():
    """The dt -> 0 limit of the piecewise-constant propagation is the solution of
    i dpsi/dt = H(t) psi, computed here by an unrelated integrator (scipy DOP853, rtol 1e-12);
    midpoint sampling makes the error fall by ~4x per halving of dt (second order)."""
    from scipy.integrate import solve_ivp

    d, Vt, vmax = _driven_well()
    T = 2.0
    dd, ee = d.tridiagonal()
    base = dd - d.potential()

    def rhs(t, y):
        psi = y[: d.n] + 1j * y[d.n:]
        h = (base + Vt(t)) * psi
        h[1:] += ee * psi[:-1]
        h[:-1] += ee * psi[1:]
        dpsi = -1j * h
        return np.concatenate([dpsi.real, dpsi.imag])

    x0 = d.packet()
    sol = solve_ivp(rhs, (0.0, T), np.concatenate([x0.real, x0.imag]), method="DOP853",
                    rtol=1e-12, atol=1e-13)
    ref = sol.y[: d.n, -1] + 1j * sol.y[d.n:, -1]
    lo, hi = d.bounds()
    a, b = oracle.rescale(lo - vmax, hi + vmax, 0.01)
    errs = []
    for nsteps in (20, 40, 80):
        dt = T / nsteps
        C, _ = oracle.coeffs(a, b, dt)
        seq = [Vt((s + 0.5) * dt) for s in range(nsteps)]
        psi = oracle.evolve_piecewise(lambda V: oracle.lattice1d(d.n, d.dx, V), seq, a, b, C,
                                      x0)
        errs.append(np.linalg.norm(psi - ref))
    assert errs[0] > 1e-6  # the driving matters at this step
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.5 < e1 / e2 < 4.5


def test_harmonic_coherent_state_returns_after_period():
    """V = x^2/2: a displaced ground state returns to itself after t = 2 pi (up to O(dx^2))."""
    n = 512
    x = np.linspace(-12, 12, n, endpoint=False)
    dx = x[1] - x[0]
    H = oracle.lattice1d(n, dx, 0.5 * x ** 2)
    psi0 = np.exp(-((x - 3.0) ** 2) / 2).astype(np.complex128)
    psi0 /= np.linalg.norm(psi0)
    Hd = H.dense()
    lo, hi = np.linalg.eigvalsh(Hd)[[0, -1]]
    a, b = oracle.rescale(lo, hi, 0.01)
    nsteps = 16
    C, M = oracle.coeffs(a, b, 2 * np.pi / nsteps)
    psi = H.evolve(a, b, C, nsteps, psi0)
    # global phase e^{-i pi} from the zero-point energy, up to the grid error
    assert abs(abs(np.vdot(psi0, psi)) - 1.0) < 5e-3
    half = H.evolve(a, b, C, nsteps // 2, psi0)
    com = np.sum(x * np.abs(half) ** 2)
    assert abs(com + 3.0) < 0.05  # at t = pi the packet sits at -x0


def test_norm_and_energy_conserved():
    d = wl.DoubleWell1D(n=256)
    lo, hi = d.bounds()
    a, b = oracle.rescale(lo, hi, 0.01)
    C, M = oracle.coeffs(a, b, d.dt)
    H = oracle.lattice1d(d.n, d.dx, d.potential())
    psi0 = d.packet()
    n0, e0 = H.norm_energy(psi0)
    psi = H.evolve(a, b, C, 20, psi0)
    n1, e1 = H.norm_energy(psi)
    assert abs(n1 - n0) < 1e-12
    assert abs(e1 - e0) < 1e-12 * abs(hi)


# --------------------------------------------------------------------------------------
# Sec. 3.2, Eq. (model): honeycomb ribbon
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("W,L", [(4, 8), (6, 12), (8, 6)])
def test_honeycomb_torus_spectrum_closed_form(W, L):
    """Periodic brick wall = honeycomb torus: E = +-t |1 + e^{-2 i k_c} + e^{i (k_r - k_c)}|,
    k_r = 2 pi m / W, k_c = 2 pi n / L, m < W, n < L/2 (two sites per cell)."""
    t = 1.3
    H = oracle.honeycomb(W, L, t, None, periodic=True)
    E = np.sort(np.linalg.eigvalsh(H.dense()))
    kr = 2 * np.pi * np.arange(W)[:, None] / W
    kc = 2 * np.pi * np.arange(L // 2)[None, :] / L
    f = np.abs(1 + np.exp(-2j * kc) + np.exp(1j * (kr - kc))).ravel()
    ref = np.sort(np.concatenate([t * f, -t * f]))
    assert np.max(np.abs(E - ref)) < 1e-12


def test_honeycomb_open_chain_and_dimer_limits():
    """W = 1: an open chain, E = -2t cos(j pi/(L+1)).  L = 1: isolated vertical dimers
    (0,1), (2,3), ... with E = +-t (and 0 for an odd W)."""
    t = 0.9
    L = 17
    E = np.linalg.eigvalsh(oracle.honeycomb(1, L, t).dense())
    ref = np.sort(-2 * t * np.cos(np.arange(1, L + 1) * np.pi / (L + 1)))
    assert np.max(np.abs(E - ref)) < 1e-13
    E = np.linalg.eigvalsh(oracle.honeycomb(7, 1, t).dense())
    ref = np.sort([t] * 3 + [-t] * 3 + [0.0])
    assert np.max(np.abs(E - ref)) < 1e-13


def test_honeycomb_open_ribbon_structure():
    """Open zigzag ribbon: bipartite (spectrum symmetric for eps = 0), bond count
    W (L-1) + #{(r, c): r < W-1, r + c even}, every degree <= 3, H symmetric, and the
    on-site energies on the diagonal."""
    W, L = 9, 14
    eps = wl.anderson_disorder(W * L, 2.0, seed=5)
    H = oracle.honeycomb(W, L, 1.0, eps).dense()
    assert np.allclose(H, H.T)
    assert np.allclose(np.diag(H), eps)
    off = H - np.diag(np.diag(H))
    nb = int((off != 0).sum()) // 2
    vert = sum(1 for r in range(W - 1) for c in range(L) if (r + c) % 2 == 0)
    assert nb == W * (L - 1) + vert
    assert (off != 0).sum(axis=1).max() == 3
    E = np.linalg.eigvalsh(oracle.honeycomb(W, L, 1.0).dense())
    assert np.allclose(E, -E[::-1], atol=1e-12)


@pytest.mark.parametrize("Na", [4, 5, 8, 10])
def test_honeycomb_armchair_ribbon_spectrum_closed_form(Na):
    """Armchair reading of the brick-wall (Sec. 3.2 ribbons with armchair edges): the
    columns are the N_a dimer lines; with the rows wrapped the ribbon is infinite along its
    length and its bands are E = +-t (1 + 4 cos^2 th_p + 4 cos th_p cos(phi/2))^(1/2),
    th_p = p pi/(N_a + 1), phi the Bloch phase per two rows; N_a = 3m - 1 is metallic."""
    W = 48
    H = oracle.honeycomb(W, Na, 1.0, periodic=2)
    E = np.sort(np.linalg.eigvalsh(H.dense()))
    th = np.arange(1, Na + 1) * np.pi / (Na + 1)
    phi = 2 * np.pi * np.arange(W // 2) / (W // 2)
    e = np.sqrt(np.maximum(0.0, 1 + 4 * np.cos(th)[:, None] ** 2
                           + 4 * np.cos(th)[:, None] * np.cos(phi / 2)[None, :])).ravel()
    ref = np.sort(np.concatenate([e, -e]))
    assert np.max(np.abs(E - ref)) < 1e-12
    gap = np.min(np.abs(E))
    assert (gap < 1e-12) == (Na % 3 == 2)


def test_propagator_matches_exact_diagonalisation_ribbon():
    rb = wl.Ribbon(W=8, L=32, disorder=1.0, seed=907, sigma=3.0, nsteps=40)
    eps = rb.onsite()
    H = oracle.honeycomb(rb.W, rb.L, rb.hop, eps)
    lo, hi = rb.bounds()
    a, b = oracle.rescale(lo, hi, 0.0)
    C, M = oracle.coeffs(a, b, rb.dt)
    psi0 = rb.packet()
    psi = H.evolve(a, b, C, rb.nsteps, psi0)
    E, V = np.linalg.eigh(H.dense())
    ex = V @ (np.exp(-1j * E * rb.dt * rb.nsteps) * (V.T @ psi0))
    assert np.linalg.norm(psi - ex) < 1e-12


# --------------------------------------------------------------------------------------
# Sec. 3.3, Eq. (ghm): Holstein chain in the truncated phonon basis
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("L,nph", [(1, 3), (3, 2), (4, 3), (2, 5), (5, 4)])
def test_holstein_basis_count_and_order(L, nph):
    """D = L * C(nph + L, L); occupations strictly increasing in lexicographic order; every
    tuple with sum <= nph appears (brute force over the box [0, nph]^L)."""
    H = oracle.holstein(L, nph, False, 1.0, 1.0, 1.0)
    assert H.n == L * math.comb(nph + L, L)
    occ = H.occupations()
    tuples = [tuple(int(v) for v in row) for row in occ]
    assert tuples == sorted(tuples) and len(set(tuples)) == len(tuples)
    import itertools
    allt = [t for t in itertools.product(range(nph + 1), repeat=L) if sum(t) <= nph]
    assert sorted(allt) == tuples
    for idx in range(H.n):
        e, o = H.state(idx)
        assert H.index(e, o) == idx


def test_holstein_paper_dimension():
    """Sec. 3.3: 18 sites with at most 11 phonons give D_tot = 6.2e8 (18 * C(29, 11))."""
    D = 18 * math.comb(11 + 18, 18)
    assert D == 622_751_220
    assert abs(D / 6.2e8 - 1) < 0.005


def test_holstein_no_coupling_spectrum():
    """g = 0 on a ring: E = -2t cos(2 pi q / L) + omega0 n with multiplicity C(n+L-1, L-1)."""
    L, nph, t, w0 = 5, 3, 0.8, 1.7
    E = np.sort(np.linalg.eigvalsh(oracle.holstein(L, nph, True, t, w0, 0.0).dense()))
    ref = []
    for n in range(nph + 1):
        mult = math.comb(n + L - 1, L - 1)
        for q in range(L):
            ref += [-2 * t * math.cos(2 * math.pi * q / L) + w0 * n] * mult
    assert np.max(np.abs(E - np.sort(ref))) < 1e-12


def test_holstein_single_site_displaced_oscillator():
    """t irrelevant, L = 1: H = w0 b^+b - g w0 (b + b^+), levels w0 (n - g^2)."""
    g, w0 = 1.0, 1.3
    E = np.linalg.eigvalsh(oracle.holstein(1, 60, False, 1.0, w0, g).dense())[:6]
    assert np.max(np.abs(E - w0 * (np.arange(6) - g ** 2))) < 1e-10


def test_holstein_coherent_dynamics_observables():
    """L = 1 from the phonon vacuum: <b^+b>(t) = 2 g^2 (1 - cos w0 t) and
    chi(t) = <n (b + b^+)> = 2 g (1 - cos w0 t) (a coherent state displaced toward +g),
    pinning the sign and the sqrt(n) factors of the coupling and the observables."""
    g, w0, nph = 1.5, 1.0, 60
    H = oracle.holstein(1, nph, False, 1.0, w0, g)
    lo, hi = np.linalg.eigvalsh(H.dense())[[0, -1]]
    a, b = oracle.rescale(lo, hi, 0.01)
    dt = 0.25
    C, M = oracle.coeffs(a, b, dt)
    psi = np.zeros(H.n, complex)
    psi[0] = 1.0
    for s in range(1, 13):
        psi = H.step(a, b, C, psi)
        dens, phon, chi = H.observables(psi)
        t = s * dt
        assert abs(dens[0] - 1.0) < 1e-12
        assert abs(phon[0] - 2 * g * g * (1 - math.cos(w0 * t))) < 1e-10
        assert abs(chi[0] - 2 * g * (1 - math.cos(w0 * t))) < 1e-10


def test_holstein_hermitian_and_row_structure():
    hs = wl.Holstein(L=4, nph=3)
    H = oracle.holstein(hs.L, hs.nph, True, hs.hop, hs.omega0, hs.g)
    Hd = H.dense()
    assert np.array_equal(Hd, Hd.T)
    lo, hi = hs.bounds()
    E = np.linalg.eigvalsh(Hd)
    assert lo <= E[0] and E[-1] <= hi


def test_propagator_matches_exact_diagonalisation_holstein():
    hs = wl.Holstein(L=4, nph=3, nsteps=40)
    H = oracle.holstein(hs.L, hs.nph, True, hs.hop, hs.omega0, hs.g)
    lo, hi = hs.bounds()
    a, b = oracle.rescale(lo, hi, hs.alpha)
    C, M = oracle.coeffs(a, b, hs.dt)
    psi0 = np.zeros(H.n, complex)
    psi0[0] = 1
    psi = H.evolve(a, b, C, hs.nsteps, psi0)
    E, V = np.linalg.eigh(H.dense())
    ex = V @ (np.exp(-1j * E * hs.dt * hs.nsteps) * (V.T @ psi0))
    assert np.linalg.norm(psi - ex) < 1e-12
    dens, phon, chi = H.observables(psi)
    assert abs(dens.sum() - 1) < 1e-12


# --------------------------------------------------------------------------------------
# Gradient of a region probability (no counterpart in the paper)
# --------------------------------------------------------------------------------------
def _ribbon_problem(W=6, L=20, nsteps=5):
    rb = wl.Ribbon(W=W, L=L, disorder=1.0, seed=3022, sigma=2.5, c0=6, r0=W // 2)
    eps = rb.onsite()
    a, b = oracle.rescale(*rb.bounds(), 0.0)
    C, M = oracle.coeffs(a, b, rb.dt)
    mask = np.zeros(W * L, np.uint8)
    mask.reshape(W, L)[:, L // 2 + 1:] = 1
    return rb, eps, a, b, C, mask, nsteps


def test_adjoint_matches_central_differences():
    rb, eps, a, b, C, mask, nsteps = _ribbon_problem()
    psi0 = rb.packet()
    H = oracle.honeycomb(rb.W, rb.L, rb.hop, eps)
    P, grad, _ = H.adjoint_region(a, b, C, nsteps, psi0, mask)

    def prob(e):
        psi = oracle.honeycomb(rb.W, rb.L, rb.hop, e).evolve(a, b, C, nsteps, psi0)
        return float(np.sum(np.abs(psi[mask == 1]) ** 2))

    assert abs(prob(eps) - P) < 1e-14
    rng = np.random.default_rng(0)
    h = 1e-6
    for i in rng.choice(rb.W * rb.L, 12, replace=False):
        ep, em = eps.copy(), eps.copy()
        ep[i] += h
        em[i] -= h
        fd = (prob(ep) - prob(em)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-4 * max(abs(fd), 1e-6) + 1e-9


def test_adjoint_matches_daleckii_krein():
    """Exact gradient of P(T) = |Pi e^{-iHT} psi0|^2: in the eigenbasis of H,
    d e^{-iHT}/dV_i = V (G o (V^T e_i e_i^T V)) V^T with G_mn = (e^{-iE_mT} - e^{-iE_nT})/(-i(E_m-E_n))
    ... written as the divided difference of f(E) = e^{-iET}; the truncated Chebyshev gradient
    agrees within its truncation error."""
    rb, eps, a, b, C, mask, nsteps = _ribbon_problem(W=4, L=12, nsteps=4)
    psi0 = rb.packet()
    H = oracle.honeycomb(rb.W, rb.L, rb.hop, eps)
    P, grad, _ = H.adjoint_region(a, b, C, nsteps, psi0, mask)
    E, V = np.linalg.eigh(H.dense())
    T = rb.dt * nsteps
    f = np.exp(-1j * E * T)
    dE = E[:, None] - E[None, :]
    same = np.abs(dE) < 1e-12
    G = np.where(same, -1j * T * f[:, None], (f[:, None] - f[None, :]) / np.where(same, 1, dE))
    psiT = V @ (f * (V.T @ psi0))
    Pi = mask.astype(float)
    c0 = V.T @ psi0
    lam = V.T @ (Pi * psiT)
    ref = np.empty(H.n)
    for i in range(H.n):
        Xi = np.outer(V[i], V[i])  # V^T e_i e_i^T V
        dpsi_eig = (G * Xi) @ c0
        ref[i] = 2 * np.real(np.vdot(lam, dpsi_eig))
    assert abs(P - float(np.sum(Pi * np.abs(psiT) ** 2))) < 1e-12
    assert np.max(np.abs(grad - ref)) < 1e-10


def test_holstein_site_dependent_terms_decoupled_limit():
    """t = 0 decouples the electron sites: with the electron at e the phonons at e form an
    oscillator displaced by g_e and the other site's phonons a free one, so the levels are
    Delta_e + w0 (m - g_e^2), m = 0, 1, ..., with multiplicity m + 1 (pins Delta_i and g_i of
    Eq. ghm per site; the cap of 30 phonons is invisible in the lowest levels)."""
    L, nph, w0 = 2, 30, 1.5
    Delta = np.array([0.0, 0.7])
    g = np.array([0.5, 0.9])
    H = oracle.holstein(L, nph, False, 0.0, w0, 1.0, Delta=Delta, gsite=g)
    E = np.sort(np.linalg.eigvalsh(H.dense()))
    ref = []
    for e in range(L):
        for m in range(6):
            ref += [Delta[e] + w0 * (m - g[e] ** 2)] * (m + 1)
    ref = np.sort(ref)[:12]
    assert np.max(np.abs(E[:12] - ref)) < 1e-9


def test_polaron_workload_shape():
    pw = wl.Polaron()
    assert pw.dim == 622_751_220
    g = pw.gsite()
    assert abs(g[0] - math.sqrt(0.5)) < 1e-15 and abs(g[11] - 1.0) < 1e-15
    assert pw.delta()[11] == 2.0 and pw.delta().sum() == 2.0
    assert abs(np.linalg.norm(pw.electron_packet()) - 1.0) < 1e-14
    small = wl.Polaron(L=5, nph=3, barrier_site=3, packet_site=1)
    H = oracle.holstein(small.L, small.nph, False, small.hop, small.omega0, 1.0,
                        Delta=small.delta(), gsite=small.gsite())
    lo, hi = small.bounds()
    E = np.linalg.eigvalsh(H.dense())
    assert lo <= E[0] and E[-1] <= hi
    psi0 = small.initial_state()
    dens, phon, chi = H.observables(psi0)
    assert np.allclose(dens, np.abs(small.electron_packet()) ** 2)
    assert np.allclose(phon, 0) and np.allclose(chi, 0)
