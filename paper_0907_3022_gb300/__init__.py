"""GB300 (sm_103a) Chebyshev time evolution: Python side of the C ABI in include/cheb.h.

ψ(t+Δt) = Σ_k C_k T_k(H̃) ψ(t) with the fused three-term recurrence of Sec. 2.2 of Fehske et
al., "Numerical approaches to time evolution of complex quantum systems", for the 1D grid
(Sec. 3.1), zigzag honeycomb ribbons and ensembles of them (Sec. 3.2) and the Holstein polaron
(Sec. 3.3).  See ``_cheb`` for the binding and ``autograd`` for the gradient with respect to
the on-site potential.
"""
from ._cheb import *  # noqa: F401,F403
from ._cheb import Plan, ChebError, lib  # noqa: F401
