"""Runs the FP64 oracle over the full Holstein configuration (L = 12 periodic, nph <= 10,
D = 7,759,752, t = 1, w0 = 1, g = 1.5, dt = 0.25, 200 steps from the electron on site 0 with
the phonon vacuum; Sec. 3.3, Eq. ghm) and saves the final state, its norm and energy.

Test infrastructure: it calls only the oracle and the input module.  The GPU test of the full
evolution starts it as a child process at the beginning of the session, so that its five or
so minutes of host time overlap the other GPU tests.

Usage: python tests/holstein_oracle_run.py OUT.npz [NSTEPS]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402


def main(out: str, nsteps: int) -> None:
    hs = wl.Holstein()
    t0 = time.perf_counter()
    H = oracle.holstein(hs.L, hs.nph, hs.periodic, hs.hop, hs.omega0, hs.g)
    a, b = oracle.rescale(*hs.bounds(), hs.alpha)
    C, M = oracle.coeffs(a, b, hs.dt)
    psi = H.evolve(a, b, C, nsteps, hs.initial_state())
    n2, e = H.norm_energy(psi)
    tmp = out + ".tmp.npz"
    np.savez(tmp, psi=psi, norm2=n2, energy=e, M=M, nsteps=nsteps,
             seconds=time.perf_counter() - t0)
    os.replace(tmp, out)


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else wl.Holstein().nsteps)
