"""Oracle RH92 iteration -- the paper's reference method (test infrastructure only).

Rybicki & Hummer (1992) linearisation with operator splitting and a local
(diagonal) approximate operator, with full preconditioning, as used by RH
(Uitenbroek 2001); the paper uses it as its reference (Sect. 3) but does not
restate its equations, so this is written from the published method:

  I = Psi* eta + I_eff,  I_eff = I^dagger - Psi* eta^dagger,
  Psi*_{mu nu}^k = dI^k/deta^k (the diagonal of the piecewise-linear
  Lambda operator divided by chi, App. A.2: a^k/chi^k for mu > 0,
  a^{k-1}/chi^k for mu < 0).

In the net radiative rate of transition t, n_lo R_lo,up - n_up R_up,lo =
int [chi_t I - eta_t], the product chi_t Psi* eta is preconditioned by taking
chi_t at the old populations (the cross-coupling terms), which leaves

  N_t(n') = int [chi_t(n') J_eff + chi_t(n) Psi*_avg eta(n') - eta_t(n')]

linear in the new populations n' (angle averages only, the atmosphere being
static). Together with the collision terms and the conservation row, one
N_l x N_l linear solve per depth gives n'. At the fixed point n' = n the rates
are exact, so RH92 and JFNK share the same solution.

Far from the solution (LTE start in a hot, strongly ionised layer) the solve
can return negative populations. With ``clamp`` the correction n' - n is then
limited per depth exactly like a Newton correction (Sect. 2.2.2, the same
``depth_clamp``): the paper states that limiting for the Newton step only, and
applying it to the RH92 correction is this implementation's reading; it leaves
every iteration that stays positive unchanged.

Pins (tests/test_oracle_solvers.py): the fixed point is JFNK's solution on a
column with background (which fixes the constant cross-coupling term), RH92
and JFNK reach the same populations and emergent spectrum, and on the
eps = 1e-4 slab RH92 ends orders of magnitude closer to the solution than the
same loop with Psi* = 0 (plain Lambda iteration), which a dropped or
mis-signed Psi* or cross-coupling term would reduce it to.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from .jfnk import depth_clamp, pop_change
from .model import FOURPI, H, Model, initial_J
from .residual import residual


@dataclass
class RH92Result:
    n: np.ndarray
    J: np.ndarray
    converged: bool
    iterations: int
    F_norm: float
    dn_norm: float
    history: List[dict] = field(default_factory=list)
    I_emergent: np.ndarray = None


def rh92_update(m: Model, n, res):
    """One preconditioned rate-equation solve per depth, from a residual evaluation at n."""
    if m.Vdir is not None:
        raise NotImplementedError("RH92 is written here for static columns (angle-averaged Psi*)")
    Wnu = FOURPI / (H * m.nu)
    psi = res.lam_eta                                   # [nq, nz] angle-averaged Psi*
    eta_bg = res.eta.copy()
    for t, tr in enumerate(m.trans):
        eta_bg = eta_bg - m.twohnu3c2[:, None] * m.g[t] * m.V[t] * n[:, tr.up][None, :]
    J_eff = res.J - psi * res.eta
    nl, nz = m.nl, m.nz
    M = np.zeros((nz, nl, nl))     # d(sum_t s_it N_t + collisions)/dn'_j
    c0 = np.zeros((nz, nl))        # constant part
    U = [m.twohnu3c2[:, None] * m.g[t] * m.V[t] for t in range(m.nt)]
    for t, tr in enumerate(m.trans):
        lo, up = tr.lo, tr.up
        W = m.omega[t][:, None] * Wnu[:, None]
        chi_old = m.V[t] * (n[:, lo][None, :] - m.g[t] * n[:, up][None, :])
        coef = np.zeros((nz, nl))
        coef[:, lo] += np.sum(W * m.V[t] * J_eff, axis=0)
        coef[:, up] -= np.sum(W * m.g[t] * m.V[t] * J_eff, axis=0)
        coef[:, up] -= np.sum(W * U[t], axis=0)
        wcp = W * chi_old * psi
        for s, ts in enumerate(m.trans):
            coef[:, ts.up] += np.sum(wcp * U[s], axis=0)
        const = np.sum(wcp * eta_bg, axis=0)
        coef[:, lo] += m.Cmat[:, lo, up]
        coef[:, up] -= m.Cmat[:, up, lo]
        M[:, lo, :] += coef
        M[:, up, :] -= coef
        c0[:, lo] += const
        c0[:, up] -= const
    n_new = np.zeros_like(n)
    for k in range(nz):
        A = M[k].copy()
        rhs = -c0[k].copy()
        row = res.istar[k]
        A[row, :] = 1.0
        rhs[row] = m.ntot[k]
        n_new[k] = np.linalg.solve(A, rhs)
    return n_new


def rh92(m: Model, n0, J0=None, ftol: float = 1e-4, maxiter: int = 500,
         clamp: bool = True) -> RH92Result:
    n = np.array(n0, dtype=float)
    Jdag = initial_J(m) if J0 is None else np.array(J0, dtype=float)
    hist = []
    err = np.inf
    converged = False
    it = 0
    res = residual(m, n, Jdag, want_lambda=True)
    for it in range(1, maxiter + 1):
        n_new = rh92_update(m, n, res)
        if clamp:
            n_new, _ = depth_clamp(n, n_new - n)
        err = pop_change(n_new, n)
        Jdag = res.J
        n = n_new
        res = residual(m, n, Jdag, want_lambda=True)
        hist.append(dict(iter=it, F_norm=float(np.max(np.abs(res.F))), dn_norm=err))
        if err < ftol:
            converged = True
            break
    return RH92Result(n=n, J=res.J, converged=converged, iterations=it,
                      F_norm=float(np.max(np.abs(res.F))), dn_norm=err, history=hist,
                      I_emergent=res.I_emergent)
