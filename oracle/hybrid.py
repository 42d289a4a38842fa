"""Oracle hybrid start: RH92 iterations, then JFNK (test infrastructure only).

The paper proposes (Sect. 3.5) to run a few RH92 iterations before switching
to JFNK, to give the Newton iteration a starting point inside its domain of
convergence; it reports that JFNK started from LTE fails for its six-level
H I atom. Here RH92 runs from the initial guess until its population change
falls below ``switch_tol`` (or ``rh92_max`` iterations), then Algorithm 2
continues from there with RH92's last mean intensity as J^dagger_0. The RH92
corrections are limited per depth like the Newton corrections (see
``oracle.rh92``) whenever ``clamp`` is on for the Newton iteration.
"""
from __future__ import annotations

from .jfnk import jfnk
from .model import Model
from .rh92 import rh92


def hybrid(m: Model, n0, J0=None, switch_tol: float = 1e-2, rh92_max: int = 200, **jfnk_kwargs):
    warm = rh92(m, n0, J0=J0, ftol=switch_tol, maxiter=rh92_max,
                clamp=jfnk_kwargs.get("clamp", True))
    out = jfnk(m, warm.n, J0=warm.J, **jfnk_kwargs)
    out.rh92_iters = warm.iterations
    out.F_calls += warm.iterations
    return out
