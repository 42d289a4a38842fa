"""Oracle JFNK solver -- Algorithm 2 -- and the initial guesses (test infrastructure only).

Outer Newton-Raphson loop (Eq. newton_approx), inner left-preconditioned
Krylov solve (Eq. prec2) with JVPs by the complex step (Eq. complex) or by
finite differences, block-Jacobi preconditioner rebuilt at every base
evaluation (Algorithm 2, Sect. 2.5.2).

Readings where the paper leaves room:
  * J^dagger: each Newton step p uses one lagged mean intensity J^dagger_p
    for its base evaluation and all its JVPs; the base evaluation F(n^p)
    returns J(n^p), which becomes J^dagger_{p+1}. J^dagger_0 is the input
    estimate (B_nu(T) by default).
  * Conservation rows: chosen at the base point of each Newton step
    (argmax of n^p per depth, lowest index on ties) and kept for its JVPs.
  * Convergence (Sect. 3.1): ||dn/n||_inf = 1/2 ||(n_new - n_prev)/(n_new + n_prev)||_inf
    below ``ftol`` AND ||F||_inf at most ``fdrop`` times its initial value.
  * Per-depth limiting of the correction (Sect. 2.2.2): alpha_k =
    min(1, 0.9 min_{i: dn_i < 0} n_i/|dn_i|), n^k += alpha_k dn^k.
  * x_0 = 0 for the Krylov solver (Sect. 2.3).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import krylov
from .model import Model, initial_J
from .precond import apply_inverse, block_jacobi, dJ_dn, lu_factor_blocks
from .residual import COMPLEX_EPS, jvp_complex, jvp_fd, residual


@dataclass
class SolveResult:
    n: np.ndarray
    J: np.ndarray
    converged: bool
    newton_iters: int
    F_calls: int                 # base evaluations + JVP evaluations (F-class calls)
    jvp_calls: int
    F_norm: float
    F_norm0: float
    dn_norm: float
    history: List[dict] = field(default_factory=list)
    I_emergent: np.ndarray = None


def depth_clamp(n, dn, factor: float = 0.9):
    """Per-depth limiting that keeps populations positive (Sect. 2.2.2 reading)."""
    alpha = np.ones(n.shape[0])
    neg = dn < 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(neg, n / np.where(neg, -dn, 1.0), np.inf)
    lim = factor * ratio.min(axis=1)
    alpha = np.minimum(1.0, lim)
    return n + alpha[:, None] * dn, alpha


def pop_change(n_new, n_prev) -> float:
    return float(0.5 * np.max(np.abs((n_new - n_prev) / (n_new + n_prev))))


def zero_radiation_guess(m: Model) -> np.ndarray:
    """Populations of the rate equations with I = 0 (spontaneous rates only) plus conservation
    (Sect. 2.2.1). Pinned by the two-level closed form n_u/n_l = C_lu/(C_ul + A_ul) and by the
    Saha-Boltzmann limit of a six-level atom when collisions dominate."""
    from .residual import rates_from_J
    R_up, R_dn = rates_from_J(m, np.zeros((m.nq, m.nz)))
    n = np.zeros((m.nz, m.nl))
    for k in range(m.nz):
        A = np.zeros((m.nl, m.nl))
        for t, tr in enumerate(m.trans):
            i, j = tr.lo, tr.up
            up = m.Cmat[k, i, j] + R_up[t, k]
            dn = m.Cmat[k, j, i] + R_dn[t, k]
            A[i, i] += up
            A[i, j] -= dn
            A[j, i] -= up
            A[j, j] += dn
        rhs = np.zeros(m.nl)
        row = int(np.argmax(m.nstar[k]))
        A[row, :] = 1.0
        rhs[row] = m.ntot[k]
        n[k] = np.linalg.solve(A, rhs)
    return n


def jfnk(m: Model, n0, J0=None, ftol: float = 1e-4, fdrop: float = 1e-2, rtol: float = 1e-2,
         maxiter: int = 100, m_max: int = 50, max_restarts: int = 20, krylov_solver: str = "gmres",
         jvp: str = "complex", fd_choice: str = "eps1", precond: bool = True, clamp: bool = True,
         complex_eps: float = COMPLEX_EPS, line_search: bool = False,
         max_halvings: int = 12, precond_variant: int = 1) -> SolveResult:
    """Algorithm 2. ``precond_variant`` selects the solution of Sect. 2.5.2 the
    block-Jacobi preconditioner follows (1, 2 or 3; see ``precond.dJ_dn``); the
    lagged estimate of variant 2 starts at zero and is renewed at every base
    evaluation. ``line_search``: backtracking on ||F||_inf, alpha = 1, 1/2, 1/4,
    ... (at most ``max_halvings`` halvings, Sect. 2.2.2), each trial one F call."""
    n = np.array(n0, dtype=float)
    Jdag = initial_J(m) if J0 is None else np.array(J0, dtype=float)
    N = n.size
    res = residual(m, n, Jdag, want_lambda=precond)
    f = res.F
    fcalls, jvps = 1, 0
    F0 = float(np.max(np.abs(f)))
    fnorm = F0
    err = 1.0 + ftol
    hist = [dict(iter=0, F_norm=F0, dn_norm=np.nan, F_calls=1, n=n.copy())]
    niter = 0
    converged = False
    D_lag = None
    while niter < maxiter:
        if err <= ftol and fnorm <= fdrop * F0:
            converged = True
            break
        istar = res.istar
        if precond:
            Pb = block_jacobi(m, n, res, variant=precond_variant, D_prev=D_lag)
            if precond_variant == 2:
                D_lag = dJ_dn(m, n, res, 2, D_lag)
            lus = lu_factor_blocks(Pb)
            Pinv = lambda x: apply_inverse(lus, x).ravel()
        else:
            Pinv = lambda x: np.asarray(x).ravel()
        nbase = n.copy()
        Jd = Jdag

        def matvec(v, nbase=nbase, Jd=Jd, istar=istar, f0=f):
            vv = v.reshape(n.shape)
            if jvp == "complex":
                Jv = jvp_complex(m, nbase, Jd, vv, istar=istar, eps=complex_eps)
            else:
                Jv = jvp_fd(m, nbase, Jd, vv, scheme=jvp, choice=fd_choice, F0=f0, istar=istar)
            return Pinv(Jv)

        b = -Pinv(f)
        if krylov_solver == "gmres":
            kr = krylov.gmres(matvec, b, rtol, m_max=m_max, max_restarts=max_restarts)
        else:
            kr = krylov.bicgstab(matvec, b, rtol)
        calls_per_mv = 2 if jvp == "central" else 1
        jvps += kr.matvecs
        fcalls += kr.matvecs * calls_per_mv
        dn = kr.x.reshape(n.shape)
        n_prev = n
        Jdag = res.J                       # J(n^p) becomes J^dagger_{p+1}
        step = 1.0
        fnorm_prev = fnorm
        for _h in range(max_halvings + 1):
            # optional backtracking on ||F|| (Sect. 2.2.2): alpha = 1, 1/2, 1/4, ...
            n_try, _alpha = depth_clamp(n_prev, step * dn) if clamp else (n_prev + step * dn, None)
            with np.errstate(all="ignore"):
                res = residual(m, n_try, Jdag, want_lambda=precond)
            fcalls += 1
            fnorm = float(np.max(np.abs(res.F)))
            ok = np.isfinite(fnorm) and np.all(np.isfinite(res.J))
            if not line_search or (ok and fnorm < fnorm_prev):
                break
            step *= 0.5
        n = n_try
        f = res.F
        err = pop_change(n, n_prev)
        niter += 1
        hist.append(dict(iter=niter, F_norm=fnorm, dn_norm=err, F_calls=fcalls,
                         krylov_iters=kr.iterations, krylov_rel=kr.rel_residual, n=n.copy()))
        if not np.all(np.isfinite(n)):
            break
    else:
        converged = err <= ftol and fnorm <= fdrop * F0
    return SolveResult(n=n, J=res.J, converged=converged, newton_iters=niter, F_calls=fcalls,
                       jvp_calls=jvps, F_norm=fnorm, F_norm0=F0, dn_norm=err, history=hist,
                       I_emergent=res.I_emergent)
