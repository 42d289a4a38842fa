"""Oracle Krylov solvers (test infrastructure only), Sect. 2.3.

GMRES (Saad & Schultz 1986): Arnoldi with modified Gram-Schmidt, Givens
rotations on the Hessenberg matrix, stop when ||r||_2 < delta ||r_0||_2 with
r_0 = b - A x_0 (Sect. 2.3), restart after ``m_max`` basis vectors.
BiCGSTAB (van der Vorst 1992): two matrix-vector products per iteration.

Both take the operator as a callable; with left preconditioning the caller
passes v -> P^{-1} J v and b = -P^{-1} F (Eq. prec2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class KrylovResult:
    x: np.ndarray
    matvecs: int
    converged: bool
    rel_residual: float
    iterations: int


def gmres(matvec, b, rtol: float, m_max: int = 50, max_restarts: int = 20, x0=None) -> KrylovResult:
    b = np.asarray(b, dtype=float)
    N = b.size
    x = np.zeros(N) if x0 is None else np.array(x0, dtype=float)
    nmv = 0
    if x0 is None:
        r = b.copy()
    else:
        r = b - matvec(x)
        nmv += 1
    r0norm = np.linalg.norm(r)
    if r0norm == 0.0:
        return KrylovResult(x, nmv, True, 0.0, 0)
    iters = 0
    resid = r0norm
    for _restart in range(max_restarts + 1):
        beta = np.linalg.norm(r)
        m = min(m_max, N)
        Vb = np.zeros((m + 1, N))
        Hh = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gv = np.zeros(m + 1)
        gv[0] = beta
        Vb[0] = r / beta
        j_done = 0
        converged = False
        for j in range(m):
            w = matvec(Vb[j])
            nmv += 1
            iters += 1
            for i in range(j + 1):                       # modified Gram-Schmidt
                Hh[i, j] = np.dot(w, Vb[i])
                w = w - Hh[i, j] * Vb[i]
            hnext = np.linalg.norm(w)
            Hh[j + 1, j] = hnext
            for i in range(j):                           # previous rotations
                hi, hi1 = Hh[i, j], Hh[i + 1, j]
                Hh[i, j] = cs[i] * hi + sn[i] * hi1
                Hh[i + 1, j] = -sn[i] * hi + cs[i] * hi1
            rr = np.hypot(Hh[j, j], Hh[j + 1, j])
            cs[j], sn[j] = (1.0, 0.0) if rr == 0.0 else (Hh[j, j] / rr, Hh[j + 1, j] / rr)
            breakdown = hnext == 0.0
            Hh[j, j] = rr
            Hh[j + 1, j] = 0.0
            gv[j + 1] = -sn[j] * gv[j]
            gv[j] = cs[j] * gv[j]
            j_done = j + 1
            resid = abs(gv[j + 1])
            if resid < rtol * r0norm or breakdown:
                converged = True
                break
            Vb[j + 1] = w / hnext
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):              # back substitution
            y[i] = (gv[i] - np.dot(Hh[i, i + 1:j_done], y[i + 1:])) / Hh[i, i]
        x = x + Vb[:j_done].T @ y
        if converged:
            return KrylovResult(x, nmv, True, resid / r0norm, iters)
        r = b - matvec(x)
        nmv += 1
        resid = np.linalg.norm(r)
        if resid < rtol * r0norm:
            return KrylovResult(x, nmv, True, resid / r0norm, iters)
    return KrylovResult(x, nmv, False, resid / r0norm, iters)


def bicgstab(matvec, b, rtol: float, max_iter: int = 200) -> KrylovResult:
    b = np.asarray(b, dtype=float)
    x = np.zeros_like(b)
    r = b.copy()
    r0n = np.linalg.norm(r)
    if r0n == 0.0:
        return KrylovResult(x, 0, True, 0.0, 0)
    rhat = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    nmv = 0
    for it in range(1, max_iter + 1):
        rho_new = np.dot(rhat, r)
        if rho_new == 0.0:
            break
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        v = matvec(p)
        nmv += 1
        alpha = rho / np.dot(rhat, v)
        s = r - alpha * v
        if np.linalg.norm(s) < rtol * r0n:
            x = x + alpha * p
            return KrylovResult(x, nmv, True, np.linalg.norm(s) / r0n, it)
        t = matvec(s)
        nmv += 1
        omega = np.dot(t, s) / np.dot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        if np.linalg.norm(r) < rtol * r0n:
            return KrylovResult(x, nmv, True, np.linalg.norm(r) / r0n, it)
        if omega == 0.0:
            break
    return KrylovResult(x, nmv, False, np.linalg.norm(r) / r0n, it)
