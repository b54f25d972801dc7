"""Helpers shared by the GPU tests: device copies, oracle runs cached per session."""
import functools

import numpy as np

import oracle
import workloads as wl

C128, C64 = 0, 1


def dev_vec(x, prec):
    import torch

    dt = np.complex128 if prec == C128 else np.complex64
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).astype(dt))).to("cuda:0")


def dev_f64(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float64))).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@functools.lru_cache(maxsize=None)
def oracle_1d(n, nsteps=None):
    d = wl.DoubleWell1D(n=n)
    a, b = oracle.rescale(*d.bounds(), 0.01)
    C, M = oracle.coeffs(a, b, d.dt)
    H = oracle.lattice1d(d.n, d.dx, d.potential())
    psi = H.evolve(a, b, C, d.nsteps if nsteps is None else nsteps, d.packet())
    return psi, M


@functools.lru_cache(maxsize=None)
def oracle_ribbon(W, L, disorder, seed, stream, k0, nsteps, sigma=20.0, r0=None, c0=None,
                  dt=1.0):
    rb = wl.Ribbon(W=W, L=L, disorder=disorder, seed=seed, stream=stream, sigma=sigma, r0=r0,
                   c0=c0, dt=dt)
    H = oracle.honeycomb(W, L, rb.hop, rb.onsite())
    a, b = oracle.rescale(*rb.bounds(), 0.0)
    C, M = oracle.coeffs(a, b, rb.dt)
    psi = H.evolve(a, b, C, nsteps, rb.packet(k0))
    return psi, M
