"""Python access to the FP64 CPU oracle (``cheb_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module; the library never does.  The oracle is a plain
single-threaded C implementation of the Chebyshev propagator of Sec. 2.2 of the paper
(Eqs. U_1, c_k, rec) and of the three model Hamiltonians of Sec. 3, sharing no code with the
CUDA library.

Every function that has no independent pin in ``tests/test_oracle_*.py`` would say
"parity unpinned" here; at present all of them are pinned (see the tests' docstrings).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cheb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_long)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_ubyte)
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, no fast-math.  -fcx-limited-range
    makes complex products use the textbook formula (ac - bd, ad + bc) inline instead of a
    library call whose only difference is the recovery of infinite/NaN operands."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fcx-limited-range",
               "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.oracle_rescale.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
            L.oracle_bessel_coeffs.argtypes = [ctypes.c_double, ctypes.c_int, _dp]
            L.oracle_coeffs.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, _dp, _ip]
            L.oracle_op_lattice1d.argtypes = [ctypes.c_long, ctypes.c_double, _dp]
            L.oracle_op_lattice1d.restype = _vp
            L.oracle_op_honeycomb.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp,
                                              ctypes.c_int]
            L.oracle_op_honeycomb.restype = _vp
            L.oracle_op_holstein.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             _dp, _dp]
            L.oracle_op_holstein.restype = _vp
            L.oracle_op_free.argtypes = [_vp]
            L.oracle_op_dim.argtypes = [_vp]
            L.oracle_op_dim.restype = ctypes.c_long
            L.oracle_op_nnz.argtypes = [_vp]
            L.oracle_op_nnz.restype = ctypes.c_long
            L.oracle_op_export.argtypes = [_vp, _lp, _lp, _dp]
            L.oracle_op_apply.argtypes = [_vp, _dp, _dp]
            L.oracle_holstein_dim_phonon.argtypes = [_vp]
            L.oracle_holstein_dim_phonon.restype = ctypes.c_long
            L.oracle_holstein_state.argtypes = [_vp, ctypes.c_long, _ip, _up]
            L.oracle_holstein_index.argtypes = [_vp, ctypes.c_int, _up]
            L.oracle_holstein_index.restype = ctypes.c_long
            L.oracle_holstein_observables.argtypes = [_vp, _dp, _dp, _dp, _dp]
            L.oracle_cheb_step.argtypes = [_vp, ctypes.c_double, ctypes.c_double, _dp,
                                           ctypes.c_int, _dp]
            L.oracle_cheb_evolve.argtypes = [_vp, ctypes.c_double, ctypes.c_double, _dp,
                                             ctypes.c_int, ctypes.c_int, _dp]
            L.oracle_norm_energy.argtypes = [_vp, _dp, _dp, _dp]
            L.oracle_adjoint_region.argtypes = [_vp, ctypes.c_double, ctypes.c_double, _dp,
                                                ctypes.c_int, ctypes.c_int, _dp, _up, _dp, _dp,
                                                _dp]
            _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.complex128)


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


# --------------------------------------------------------------------------------------
def rescale(emin: float, emax: float, alpha: float):
    """(a, b) of Sec. 2.2."""
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = lib().oracle_rescale(emin, emax, alpha, ctypes.byref(a), ctypes.byref(b))
    if rc:
        raise ValueError(f"oracle_rescale failed ({rc})")
    return a.value, b.value


def bessel_coeffs(z: float, kmax: int) -> np.ndarray:
    """c_k(z) = (-i)^k J_k(z), k = 0..kmax, from the integral of Eq. (c_k)."""
    out = np.empty(kmax + 1, dtype=np.complex128)
    rc = lib().oracle_bessel_coeffs(z, kmax, _d(out.view(np.float64)))
    if rc:
        raise ValueError(f"oracle_bessel_coeffs failed ({rc})")
    return out


def default_kmax(z: float) -> int:
    """Search bound for the truncation order: well past the Bessel turning point k ~ z."""
    return int(np.ceil(z + 60 + 20 * z ** (1.0 / 3.0)))


def coeffs(a: float, b: float, dt: float, tol: float = 1e-14, kmax: int | None = None):
    """(C_0..C_M, M): multipliers of T_k(H~) psi in Eq. (U_1), truncated at |C_k| < tol."""
    if kmax is None:
        kmax = default_kmax(a * dt)
    out = np.empty(kmax + 1, dtype=np.complex128)
    M = ctypes.c_int()
    rc = lib().oracle_coeffs(a, b, dt, tol, kmax, _d(out.view(np.float64)), ctypes.byref(M))
    if rc:
        raise ValueError(f"oracle_coeffs failed ({rc})")
    return out[: M.value + 1].copy(), M.value


class Operator:
    """An explicit CSR matrix held by the oracle."""

    def __init__(self, handle, keep=()):
        if not handle:
            raise ValueError("oracle operator construction failed (bad arguments)")
        self._h = ctypes.c_void_p(handle)
        self._keep = keep

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.oracle_op_free(self._h)
            self._h = None

    @property
    def n(self) -> int:
        return lib().oracle_op_dim(self._h)

    @property
    def nnz(self) -> int:
        return lib().oracle_op_nnz(self._h)

    def csr(self):
        n, nnz = self.n, self.nnz
        rp = np.empty(n + 1, dtype=np.int64)
        col = np.empty(nnz, dtype=np.int64)
        val = np.empty(nnz, dtype=np.float64)
        lib().oracle_op_export(self._h, rp.ctypes.data_as(_lp), col.ctypes.data_as(_lp), _d(val))
        return rp, col, val

    def dense(self) -> np.ndarray:
        rp, col, val = self.csr()
        H = np.zeros((self.n, self.n))
        for i in range(self.n):
            for p in range(rp[i], rp[i + 1]):
                H[i, col[p]] += val[p]
        return H

    def apply(self, x) -> np.ndarray:
        x = _c128(x)
        y = np.empty_like(x)
        lib().oracle_op_apply(self._h, _d(x.view(np.float64)), _d(y.view(np.float64)))
        return y

    # -- the Chebyshev propagator --------------------------------------------------
    def step(self, a: float, b: float, C: np.ndarray, psi) -> np.ndarray:
        psi = _c128(psi).copy()
        C = _c128(C)
        rc = lib().oracle_cheb_step(self._h, a, b, _d(C.view(np.float64)), len(C) - 1,
                                    _d(psi.view(np.float64)))
        if rc:
            raise ValueError(f"oracle_cheb_step failed ({rc})")
        return psi

    def evolve(self, a: float, b: float, C: np.ndarray, nsteps: int, psi) -> np.ndarray:
        psi = _c128(psi).copy()
        C = _c128(C)
        rc = lib().oracle_cheb_evolve(self._h, a, b, _d(C.view(np.float64)), len(C) - 1,
                                      nsteps, _d(psi.view(np.float64)))
        if rc:
            raise ValueError(f"oracle_cheb_evolve failed ({rc})")
        return psi

    def norm_energy(self, psi):
        psi = _c128(psi)
        nn, e = ctypes.c_double(), ctypes.c_double()
        lib().oracle_norm_energy(self._h, _d(psi.view(np.float64)), ctypes.byref(nn),
                                 ctypes.byref(e))
        return nn.value, e.value

    def adjoint_region(self, a: float, b: float, C: np.ndarray, nsteps: int, psi0, mask):
        """(P, dP/dV, lambda_0) for P = sum_{i in region} |psi_n(i)|^2."""
        psi0 = _c128(psi0)
        C = _c128(C)
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        grad = np.empty(self.n, dtype=np.float64)
        lam0 = np.empty(self.n, dtype=np.complex128)
        P = ctypes.c_double()
        rc = lib().oracle_adjoint_region(self._h, a, b, _d(C.view(np.float64)), len(C) - 1,
                                         nsteps, _d(psi0.view(np.float64)),
                                         mask.ctypes.data_as(_up), _d(grad), ctypes.byref(P),
                                         _d(lam0.view(np.float64)))
        if rc:
            raise ValueError(f"oracle_adjoint_region failed ({rc})")
        return P.value, grad, lam0


def lattice1d(n: int, dx: float, V) -> Operator:
    V = _f64(V)
    return Operator(lib().oracle_op_lattice1d(n, dx, _d(V)), keep=(V,))


def honeycomb(W: int, L: int, t: float, eps=None, periodic: bool | int = False) -> Operator:
    """Brick-wall honeycomb lattice: W rows (zigzag chains), L columns (dimer lines);
    periodic: False open, True / 1 a torus, 2 rows wrapped only (armchair ribbon made
    infinite along its length)."""
    e = _f64(eps) if eps is not None else None
    return Operator(lib().oracle_op_honeycomb(W, L, t, _d(e) if e is not None else None,
                                              int(periodic)), keep=(e,))


class HolsteinOperator(Operator):
    @property
    def dim_phonon(self) -> int:
        return lib().oracle_holstein_dim_phonon(self._h)

    def state(self, idx: int):
        L = self._L
        e = ctypes.c_int()
        occ = np.empty(L, dtype=np.uint8)
        rc = lib().oracle_holstein_state(self._h, idx, ctypes.byref(e), occ.ctypes.data_as(_up))
        if rc:
            raise IndexError(idx)
        return e.value, occ

    def index(self, e: int, occ) -> int:
        occ = np.ascontiguousarray(occ, dtype=np.uint8)
        return lib().oracle_holstein_index(self._h, e, occ.ctypes.data_as(_up))

    def occupations(self) -> np.ndarray:
        """[dim_phonon][L] occupations in basis order."""
        D = self.dim_phonon
        out = np.empty((D, self._L), dtype=np.uint8)
        e = ctypes.c_int()
        for p in range(D):
            lib().oracle_holstein_state(self._h, p, ctypes.byref(e),
                                        out[p].ctypes.data_as(_up))
        return out

    def observables(self, psi):
        psi = _c128(psi)
        L = self._L
        dens, phon, chi = (np.empty(L) for _ in range(3))
        rc = lib().oracle_holstein_observables(self._h, _d(psi.view(np.float64)), _d(dens),
                                               _d(phon), _d(chi))
        if rc:
            raise ValueError("oracle_holstein_observables failed")
        return dens, phon, chi


def holstein(L: int, nph: int, periodic: bool, t: float, omega0: float, g: float,
             Delta=None, gsite=None) -> HolsteinOperator:
    D = _f64(Delta) if Delta is not None else None
    G = _f64(gsite) if gsite is not None else None
    h = lib().oracle_op_holstein(L, nph, int(periodic), t, omega0, g,
                                 _d(D) if D is not None else None,
                                 _d(G) if G is not None else None)
    op = HolsteinOperator(h, keep=(D, G))
    op._L = L
    return op


def evolve_piecewise(make_op, onsite_seq, a: float, b: float, C: np.ndarray, psi) -> np.ndarray:
    """Time-dependent H(t) held constant over each step (Sec. 2.2: the time variation of H
    limits the step): for s = 0, 1, ..., psi <- exp(-i H_s dt) psi by the Chebyshev step of
    Eq. U_1 with H_s = make_op(onsite_seq[s]) and the fixed rescaling (a, b), which must
    enclose the spectrum of every H_s.  Sampling the on-site energies at the step midpoints
    makes the scheme second order in dt."""
    psi = _c128(psi).copy()
    for V in onsite_seq:
        psi = make_op(V).step(a, b, C, psi)
    return psi
