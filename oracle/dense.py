"""Oracle dense Jacobian and dense Newton-Raphson (test infrastructure only).

Brute force for tiny grids: the full (N_l N_z) x (N_l N_z) Jacobian of
Fig. 1 assembled column by column from complex-step JVPs of unit vectors
(Eq. complex), and the plain Newton-Raphson iteration of Eq. newton_approx
solved with a dense LU. The paper's own Newton-Raphson reference curve
(Fig. 4) is exactly this method.
"""
from __future__ import annotations

import numpy as np

from .jfnk import SolveResult, depth_clamp, pop_change
from .model import Model, initial_J
from .residual import jvp_complex, jvp_fd, residual


def dense_jacobian(m: Model, n, Jdag, istar=None, method: str = "complex", eps=None) -> np.ndarray:
    n = np.asarray(n, dtype=float)
    N = n.size
    Jm = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        v = e.reshape(n.shape)
        if method == "complex":
            col = jvp_complex(m, n, Jdag, v, istar=istar)
        else:
            col = jvp_fd(m, n, Jdag, v, scheme=method, istar=istar, eps=eps)
        Jm[:, c] = col.ravel()
    return Jm


def dense_newton(m: Model, n0, J0=None, ftol: float = 1e-10, fdrop: float = 1e-2,
                 maxiter: int = 50, clamp: bool = True) -> SolveResult:
    n = np.array(n0, dtype=float)
    Jdag = initial_J(m) if J0 is None else np.array(J0, dtype=float)
    res = residual(m, n, Jdag)
    F0 = float(np.max(np.abs(res.F)))
    fnorm, err = F0, np.inf
    hist = [dict(iter=0, F_norm=F0, n=n.copy())]
    it = 0
    converged = False
    for it in range(1, maxiter + 1):
        Jm = dense_jacobian(m, n, Jdag, istar=res.istar)
        dn = np.linalg.solve(Jm, -res.F.ravel()).reshape(n.shape)
        n_prev = n
        n, _ = depth_clamp(n, dn) if clamp else (n + dn, None)
        Jdag = res.J
        res = residual(m, n, Jdag)
        fnorm = float(np.max(np.abs(res.F)))
        err = pop_change(n, n_prev)
        hist.append(dict(iter=it, F_norm=fnorm, dn_norm=err, n=n.copy()))
        if err <= ftol and fnorm <= fdrop * F0:
            converged = True
            break
    return SolveResult(n=n, J=res.J, converged=converged, newton_iters=it, F_calls=0,
                       jvp_calls=0, F_norm=fnorm, F_norm0=F0, dn_norm=err, history=hist,
                       I_emergent=res.I_emergent)
