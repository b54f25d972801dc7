"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the Chebyshev method itself: it only produces the
Hamiltonian parameters (grids, on-site potentials, ribbon sizes), the initial wave packets
and the spectral bounds that both the oracle and the CUDA path take as inputs.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state <- state + 0x9E3779B97F4A7C15, then the
64-bit finaliser below.  Stream s of seed q starts at state q + (s << 32); one draw per site in
index order; u = (x >> 11) * 2**-53 in [0, 1).

Workloads (sizes follow the paper's three applications, Sec. 3):
  * 1D double well on a finite-difference grid (Sec. 3.1);
  * zigzag honeycomb ribbon with Anderson disorder (Sec. 3.2, Eq. "model");
  * batched ensemble of uneven ribbons (Sec. 3.2, many disorder realisations);
  * 1D Holstein polaron in a truncated phonon basis (Sec. 3.3, Eq. "ghm").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """n successive SplitMix64 outputs (uint64) of stream `stream` of seed `seed`."""
    state0 = np.uint64((int(seed) + (int(stream) << 32)) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = state0 + _GAMMA * np.arange(1, n + 1, dtype=np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """u = (x >> 11) * 2^-53 for n draws; exactly representable doubles in [0, 1)."""
    x = splitmix64(seed, stream, n)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def anderson_disorder(n_sites: int, W: float, seed: int, stream: int = 0) -> np.ndarray:
    """On-site energies eps_j uniform in [-W/2, W/2] (Sec. 3.2), one draw per site."""
    return W * (uniform01(seed, stream, n_sites) - 0.5)


# ----------------------------------------------------------------------------------------
# 1D double well (configuration: N=2048 on [-20, 20), V0=2, packet at -2 with k0=2)
# ----------------------------------------------------------------------------------------
@dataclass
class DoubleWell1D:
    n: int = 2048
    x_lo: float = -20.0
    x_hi: float = 20.0
    V0: float = 2.0
    x0: float = -2.0
    sigma: float = 0.5
    k0: float = 2.0
    dt: float = 0.5
    t_end: float = 50.0
    tol: float = 1e-14

    @property
    def dx(self) -> float:
        return (self.x_hi - self.x_lo) / self.n

    @property
    def x(self) -> np.ndarray:
        return self.x_lo + self.dx * np.arange(self.n)

    @property
    def nsteps(self) -> int:
        return int(round(self.t_end / self.dt))

    def potential(self) -> np.ndarray:
        x = self.x
        return self.V0 * (x * x / 4.0 - 1.0) ** 2

    def packet(self) -> np.ndarray:
        """exp(-(x-x0)^2/(2 sigma^2) + i k0 x), normalised to sum |psi_i|^2 = 1."""
        x = self.x
        psi = np.exp(-((x - self.x0) ** 2) / (2 * self.sigma ** 2) + 1j * self.k0 * x)
        return psi / np.linalg.norm(psi)

    def tridiagonal(self):
        """Diagonal and off-diagonal of the 3-point finite-difference H (hbar = m = 1)."""
        d = 1.0 / self.dx ** 2 + self.potential()
        e = np.full(self.n - 1, -0.5 / self.dx ** 2)
        return d, e

    def bounds(self):
        """Exact extreme eigenvalues of the grid Hamiltonian (LAPACK tridiagonal solver)."""
        from scipy.linalg import eigh_tridiagonal

        d, e = self.tridiagonal()
        lo = eigh_tridiagonal(d, e, eigvals_only=True, select="i", select_range=(0, 0))[0]
        hi = eigh_tridiagonal(d, e, eigvals_only=True, select="i",
                              select_range=(self.n - 1, self.n - 1))[0]
        return float(lo), float(hi)


@dataclass
class PaperDoubleWell:
    """The double well of Sec. 3.1: V(q) = V0 + (1/2) m w0^2 (-q^2 + a q^4) with m = 1,
    w0 = 0.4, a = 0.02, V0 = 1 (reference units; hbar = 1), minima V = 0 at q = +-5 and the
    barrier V = 1 at q = 0; the Gaussian of Eq. psi0, (2 pi sigma^2)^(-1/4)
    exp(-(q - q0)^2/(4 sigma^2) + i p0 q), with sigma = 1/sqrt(2), q0 = -5, p0 = 1; N = 2048
    grid points; dt = 0.4 to t = 40.  The grid extent is not stated: [-17.6, 17.6) is read,
    the extent at which the 1e-14 cutoff gives the paper's M = 1500 moments at dt = 0.4."""
    n: int = 2048
    q_lo: float = -17.6
    q_hi: float = 17.6
    m: float = 1.0
    omega0: float = 0.4
    a4: float = 0.02
    V0: float = 1.0
    q0: float = -5.0
    p0: float = 1.0
    sigma: float = 2.0 ** -0.5
    dt: float = 0.4
    t_end: float = 40.0

    @property
    def dx(self) -> float:
        return (self.q_hi - self.q_lo) / self.n

    @property
    def x(self) -> np.ndarray:
        return self.q_lo + self.dx * np.arange(self.n)

    @property
    def nsteps(self) -> int:
        return int(round(self.t_end / self.dt))

    def potential(self) -> np.ndarray:
        q = self.x
        return self.V0 + 0.5 * self.m * self.omega0 ** 2 * (-q * q + self.a4 * q ** 4)

    def packet(self) -> np.ndarray:
        """Eq. psi0 on the grid, scaled to a unit vector (sum |psi_i|^2 = 1; the continuum
        normalisation of the paper is psi_i / sqrt(dx))."""
        q = self.x
        s2 = self.sigma ** 2
        psi = (2 * np.pi * s2) ** -0.25 * np.exp(-((q - self.q0) ** 2) / (4 * s2)
                                                  + 1j * self.p0 * q)
        return psi / np.linalg.norm(psi)

    def tridiagonal(self):
        """Diagonal and off-diagonal of the 3-point H = -1/(2m) d^2/dq^2 + V (m = 1)."""
        d = 1.0 / self.dx ** 2 + self.potential()
        e = np.full(self.n - 1, -0.5 / self.dx ** 2)
        return d, e

    def bounds(self):
        """Exact extreme eigenvalues of the grid Hamiltonian (LAPACK tridiagonal solver)."""
        from scipy.linalg import eigh_tridiagonal

        d, e = self.tridiagonal()
        lo = eigh_tridiagonal(d, e, eigvals_only=True, select="i", select_range=(0, 0))[0]
        hi = eigh_tridiagonal(d, e, eigvals_only=True, select="i",
                              select_range=(self.n - 1, self.n - 1))[0]
        return float(lo), float(hi)


# ----------------------------------------------------------------------------------------
# Zigzag honeycomb ribbons (brick-wall indexing: site (r, c) -> r * L + c, r across, c along)
# ----------------------------------------------------------------------------------------
@dataclass
class Ribbon:
    W: int = 128            # zigzag chains across the ribbon (rows)
    L: int = 2048           # sites along the ribbon (columns)
    hop: float = 1.0
    disorder: float = 1.0   # Anderson W
    seed: int = 907
    stream: int = 0
    sigma: float = 20.0
    k0: float = math.pi / 3
    r0: int | None = None
    c0: int | None = None
    dt: float = 1.0
    nsteps: int = 400

    @property
    def n_sites(self) -> int:
        return self.W * self.L

    def onsite(self) -> np.ndarray:
        return anderson_disorder(self.n_sites, self.disorder, self.seed, self.stream)

    def bounds(self):
        """a = 3t + W/2, b = 0 (Gershgorin), passed as emin = -a, emax = a with alpha = 0."""
        a = 3.0 * self.hop + self.disorder / 2.0
        return -a, a

    def packet(self, k0: float | None = None) -> np.ndarray:
        return ribbon_packet(self.W, self.L, self.sigma, self.k0 if k0 is None else k0,
                             self.W // 2 if self.r0 is None else self.r0,
                             self.L // 4 if self.c0 is None else self.c0)


def ribbon_packet(W: int, L: int, sigma: float, k0: float, r0: int, c0: int) -> np.ndarray:
    """exp(-((c-c0)^2 + (r-r0)^2) / (2 sigma^2)) e^{i k0 c}, unit norm, flattened r * L + c."""
    r = np.arange(W)[:, None].astype(np.float64)
    c = np.arange(L)[None, :].astype(np.float64)
    psi = np.exp(-((c - c0) ** 2 + (r - r0) ** 2) / (2 * sigma ** 2) + 1j * k0 * c)
    psi = psi.reshape(-1)
    return psi / np.linalg.norm(psi)


def random_state(n_sites: int, seed: int, stream: int = 0) -> np.ndarray:
    """psi_j = (u - 1/2) + i (u' - 1/2) from 2 n_sites consecutive draws (u of site j at 2j,
    u' at 2j + 1), unit norm: every site occupied, every energy of the band present."""
    u = uniform01(seed, stream, 2 * n_sites)
    psi = (u[0::2] - 0.5) + 1j * (u[1::2] - 0.5)
    return psi / np.linalg.norm(psi)


ENSEMBLE_K0 = (math.pi / 6, math.pi / 4, math.pi / 3, math.pi / 2)
ENSEMBLE_DISORDER = (0.5, 1.0, 2.0)


@dataclass
class ArmchairRibbon:
    """Armchair ribbon of Sec. 3.2 / Table 2: N_a = 10 dimer lines across and 1000 atoms along
    each (10,000 atoms, 1.11 x 212.8 nm^2), Anderson disorder in [-W/2, W/2], the state
    localised on one site in the centre, propagated to t = 10^4 (units 1/t) with dt = 1, 10 or
    100.  In the brick-wall indexing the long direction runs across the rows: W_bw = length
    rows, L_bw = N_a columns, site (r, c) -> r * N_a + c."""
    n_a: int = 10
    length: int = 1000
    hop: float = 1.0
    disorder: float = 0.5
    seed: int = 907
    stream: int = 0
    dt: float = 1.0
    t_end: float = 1e4

    @property
    def W(self) -> int:  # brick-wall rows
        return self.length

    @property
    def L(self) -> int:  # brick-wall columns
        return self.n_a

    @property
    def n_sites(self) -> int:
        return self.length * self.n_a

    @property
    def nsteps(self) -> int:
        return int(round(self.t_end / self.dt))

    def onsite(self) -> np.ndarray:
        return anderson_disorder(self.n_sites, self.disorder, self.seed, self.stream)

    def bounds(self):
        """Gershgorin interval +-(3t + W/2)."""
        r = 3.0 * abs(self.hop) + 0.5 * self.disorder
        return -r, r

    def start_site(self) -> int:
        return (self.length // 2) * self.n_a + self.n_a // 2

    def packet(self) -> np.ndarray:
        psi = np.zeros(self.n_sites, dtype=np.complex128)
        psi[self.start_site()] = 1.0
        return psi


@dataclass
class RibbonEnsemble:
    """64 uneven zigzag ribbons; widths U{40..160}, lengths U{500..4000} from seed 0xC0FFEE,
    drawn W_0, L_0, W_1, L_1, ...; disorder cycled 0.5/1/2; per-ribbon disorder stream r of
    seed 907; 4 packets per ribbon with k0 = pi/6, pi/4, pi/3, pi/2."""
    n_ribbons: int = 64
    size_seed: int = 0xC0FFEE
    w_range: tuple = (40, 160)
    l_range: tuple = (500, 4000)
    seed: int = 907
    sigma: float = 20.0
    k0s: tuple = ENSEMBLE_K0
    dt: float = 1.0
    nsteps: int = 200
    hop: float = 1.0
    stream0: int = 0        # ribbon r draws its disorder from stream stream0 + r
    sizes: list = field(default_factory=list)

    def __post_init__(self):
        if not self.sizes:
            u = uniform01(self.size_seed, 0, 2 * self.n_ribbons)
            wl, wh = self.w_range
            ll, lh = self.l_range
            self.sizes = [(wl + int(math.floor((wh - wl + 1) * u[2 * i])),
                           ll + int(math.floor((lh - ll + 1) * u[2 * i + 1])))
                          for i in range(self.n_ribbons)]

    @property
    def nvec(self) -> int:
        return len(self.k0s)

    def disorder(self, r: int) -> float:
        return ENSEMBLE_DISORDER[r % len(ENSEMBLE_DISORDER)]

    def ribbon(self, r: int) -> Ribbon:
        W, L = self.sizes[r]
        return Ribbon(W=W, L=L, hop=self.hop, disorder=self.disorder(r), seed=self.seed,
                      stream=self.stream0 + r, sigma=self.sigma, dt=self.dt, nsteps=self.nsteps)

    def offsets(self) -> np.ndarray:
        n = np.array([W * L for W, L in self.sizes], dtype=np.int64)
        return np.concatenate([[0], np.cumsum(n)])

    @property
    def n_sites(self) -> int:
        return int(self.offsets()[-1])

    def onsite(self) -> np.ndarray:
        return np.concatenate([self.ribbon(r).onsite() for r in range(self.n_ribbons)])

    def bounds(self):
        lo, hi = zip(*(self.ribbon(r).bounds() for r in range(self.n_ribbons)))
        return np.array(lo), np.array(hi)

    def packets(self) -> np.ndarray:
        """[site][packet] complex array of shape (n_sites, nvec)."""
        out = np.empty((self.n_sites, self.nvec), dtype=np.complex128)
        off = self.offsets()
        for r in range(self.n_ribbons):
            rb = self.ribbon(r)
            for v, k0 in enumerate(self.k0s):
                out[off[r]:off[r + 1], v] = rb.packet(k0)
        return out


# ----------------------------------------------------------------------------------------
# Holstein polaron (Sec. 3.3): one electron, L sites, total phonon number <= nph
# ----------------------------------------------------------------------------------------
@dataclass
class Holstein:
    L: int = 12
    nph: int = 10
    periodic: bool = True
    hop: float = 1.0
    omega0: float = 1.0
    g: float = 1.5
    dt: float = 0.25
    nsteps: int = 200
    alpha: float = 0.01

    @property
    def dim_phonon(self) -> int:
        return math.comb(self.nph + self.L, self.L)

    @property
    def dim(self) -> int:
        return self.L * self.dim_phonon

    def bounds(self):
        """Gershgorin interval: rows with electron-site occupation k and total s carry
        diagonal omega0*s and off-diagonal radius z_hop*t + g*omega0*(sqrt(k+1)[s<nph] + sqrt(k))."""
        z_hop = 2 if self.periodic else min(2, self.L - 1)
        lo, hi = math.inf, -math.inf
        for s in range(self.nph + 1):
            for k in range(s + 1):
                rad = z_hop * abs(self.hop) + abs(self.g) * self.omega0 * (
                    (math.sqrt(k + 1) if s < self.nph else 0.0) + math.sqrt(k))
                lo = min(lo, self.omega0 * s - rad)
                hi = max(hi, self.omega0 * s + rad)
        return lo, hi

    def initial_state(self) -> np.ndarray:
        """Electron on site 0, phonon vacuum: basis index 0."""
        psi = np.zeros(self.dim, dtype=np.complex128)
        psi[0] = 1.0
        return psi


@dataclass
class Polaron:
    """Polaron formation and tunnelling (Sec. 3.3, Fig. 3): generalised Holstein model on an
    open chain of 18 sites with at most 11 phonons (D = 18 C(29, 11) = 622,751,220),
    eps_p = 1, w0 = 2, t = 1, barrier Delta = 2 at site 12 (index 11), and an electron wave
    packet at site 4 (index 3) with momentum pi/9 in the phonon vacuum.

    Values the paper does not state (readings): the extra coupling at the barrier site,
    eps_p,12 = eps_p (so g_12 = sqrt(2 eps_p / w0)); the packet width sigma = 2 sites."""
    L: int = 18
    nph: int = 11
    periodic: bool = False
    hop: float = 1.0
    omega0: float = 2.0
    eps_p: float = 1.0
    barrier_site: int = 11
    barrier: float = 2.0
    eps_p_barrier: float = 1.0
    packet_site: int = 3
    k: float = math.pi / 9
    sigma: float = 2.0
    dt: float = 0.25
    t_end: float = 20.0
    alpha: float = 0.01

    @property
    def dim_phonon(self) -> int:
        return math.comb(self.nph + self.L, self.L)

    @property
    def dim(self) -> int:
        return self.L * self.dim_phonon

    @property
    def nsteps(self) -> int:
        return int(round(self.t_end / self.dt))

    def delta(self) -> np.ndarray:
        d = np.zeros(self.L)
        if 0 <= self.barrier_site < self.L:
            d[self.barrier_site] = self.barrier
        return d

    def gsite(self) -> np.ndarray:
        """g_i = ((eps_p + eps_p,i) / w0)^{1/2} (Eq. ghm)."""
        extra = np.zeros(self.L)
        if 0 <= self.barrier_site < self.L:
            extra[self.barrier_site] = self.eps_p_barrier
        return np.sqrt((self.eps_p + extra) / self.omega0)

    def electron_packet(self) -> np.ndarray:
        """exp(-(i - i0)^2 / (2 sigma^2) + i k i) on the L sites, unit norm."""
        i = np.arange(self.L, dtype=np.float64)
        c = np.exp(-((i - self.packet_site) ** 2) / (2 * self.sigma ** 2) + 1j * self.k * i)
        return c / np.linalg.norm(c)

    def packet_indices(self) -> np.ndarray:
        """Basis indices |e; vacuum> = e * Dph (the vacuum has rank 0)."""
        return np.arange(self.L, dtype=np.int64) * self.dim_phonon

    def initial_state(self) -> np.ndarray:
        psi = np.zeros(self.dim, dtype=np.complex128)
        psi[self.packet_indices()] = self.electron_packet()
        return psi

    def bounds(self):
        """Gershgorin interval: rows with the electron at e, occupation k there and total s
        have diagonal Delta_e + w0 s and radius hops(e) t + g_e w0 (sqrt(k+1)[s<nph] + sqrt(k))."""
        d, g = self.delta(), self.gsite()
        lo, hi = math.inf, -math.inf
        for e in range(self.L):
            hops = 2 if self.periodic else (e > 0) + (e < self.L - 1)
            for s in range(self.nph + 1):
                for kk in range(s + 1):
                    rad = hops * abs(self.hop) + abs(g[e]) * self.omega0 * (
                        (math.sqrt(kk + 1) if s < self.nph else 0.0) + math.sqrt(kk))
                    lo = min(lo, d[e] + self.omega0 * s - rad)
                    hi = max(hi, d[e] + self.omega0 * s + rad)
        return lo, hi
