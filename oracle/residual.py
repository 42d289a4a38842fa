"""Oracle residual vector F(n) -- Algorithm 1 -- and Jacobian-vector products.

Test infrastructure only. Follows Algorithm 1 step by step:
  opacity chi and emissivity eta (Eqs. chi, eta) with the lagged mean
  intensity J^dagger in the background-scattering term; S = eta/chi; the
  formal solution along every (nu, mu) ray (Eqs. Iplus, Iminus); the mean
  intensity J = 1/2 sum_mu w_mu (I+ + I-); the radiative rates (Eqs. Rij, Rji);
  the per-transition net rates kappa added to F_i and subtracted from F_j;
  and the particle-conservation row on the most populated level of each
  depth (Eqs. residuals_1, residuals_2).

Reading of the rate integrals: the angle quadrature is normalised
(1/2 int dmu -> sum of Gauss-Legendre weights = 1), and the frequency integral
carries 4 pi / (h nu) so that R_ij = B_ij int phi J dnu with
(h nu / 4 pi) B_ij phi = V_ij (standard Einstein relations, RH92 notation).
The frequency quadrature of transition t is the trapezoid rule over the union
grid points inside its window.

JVPs: complex step J v = Im F(n + i eps v)/eps with eps = 1e-200 (Eq. complex),
the conservation rows and J^dagger taken from the real point; forward,
backward and central differences (Eqs. fordif-centdif) with the step choices
eps_1 and eps_2 of the Fig. 2 caption.

Pins (tests/test_oracle_residual.py): detailed balance at LTE populations with
J = B (every net rate vanishes), collision-only detailed balance, linearity of
the complex-step JVP, agreement with brute-force central differences, and the
exactness of the block-Jacobi blocks against the dense Jacobian. The
background terms of the opacity and emissivity are pinned by three physical
limits: Kirchhoff (isothermal LTE with J^dagger = B gives S = B_nu wherever
only continua and background are active, and at every line centre), pure
electron scattering (S = J^dagger for any J^dagger) and pure absorption (S
independent of J^dagger, S = B_nu for continuum absorption alone).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

from .formal import solve_rays
from .model import FOURPI, H, Model

COMPLEX_EPS = 1e-200


@dataclass
class ResidualResult:
    F: np.ndarray             # [nz, nl]
    J: np.ndarray             # [nq, nz] new mean intensity
    R_up: np.ndarray          # [nt, nz]
    R_dn: np.ndarray          # [nt, nz]
    istar: np.ndarray         # [nz] conservation row per depth
    chi: np.ndarray           # [nq, nz]
    eta: np.ndarray           # [nq, nz]
    I_emergent: np.ndarray    # [nq, nmu] outgoing intensity at the top
    lam_chi: Optional[np.ndarray] = None   # [nq, nz] 1/2 sum_mu w (dI^k/dchi^k) both hemispheres
    lam_eta: Optional[np.ndarray] = None   # [nq, nz] 1/2 sum_mu w (dI^k/deta^k)


def opacity_emissivity(m: Model, n, Jdag):
    """Eqs. chi and eta: chi = chi_c + chi_sca + sum V(n_i - g n_j); eta = eta_c + chi_sca J^dagger + sum (2 h nu^3/c^2) g V n_j."""
    chi = m.chi_c + m.chi_sca[None, :] + np.zeros((1, 1), dtype=n.dtype)
    eta = m.eta_c + m.chi_sca[None, :] * Jdag + np.zeros((1, 1), dtype=n.dtype)
    for t, tr in enumerate(m.trans):
        ni = n[:, tr.lo][None, :]
        nj = n[:, tr.up][None, :]
        chi = chi + m.V[t] * (ni - m.g[t] * nj)
        eta = eta + m.twohnu3c2[:, None] * m.g[t] * m.V[t] * nj
    return chi, eta


def conservation_rows(n) -> np.ndarray:
    """Most populated level per depth (lowest index on ties), from Re(n) (Algorithm 1, last loop)."""
    return np.argmax(np.real(n), axis=1)


def rates_from_J(m: Model, J):
    """Eqs. Rij / Rji with the angle integral already folded into J."""
    W = m.omega[:, :, None] * (FOURPI / (H * m.nu))[None, :, None] * m.V      # [nt, nq, nz]
    R_up = np.sum(W * J[None, :, :], axis=1)
    R_dn = np.sum(W * m.g * (m.twohnu3c2[None, :, None] + J[None, :, :]), axis=1)
    return R_up, R_dn


def assemble(m: Model, n, R_up, R_dn, istar):
    """Net rates per transition into F (Eq. residuals_1), then conservation rows (Eq. residuals_2)."""
    F = np.zeros_like(n, dtype=np.result_type(n, R_up))
    for t, tr in enumerate(m.trans):
        i, j = tr.lo, tr.up
        kappa = n[:, i] * (m.Cmat[:, i, j] + R_up[t]) - n[:, j] * (m.Cmat[:, j, i] + R_dn[t])
        F[:, i] += kappa
        F[:, j] -= kappa
    k = np.arange(m.nz)
    F[k, istar] = m.ntot - np.sum(n, axis=1)
    return F


def residual(m: Model, n, Jdag, istar=None, want_lambda: bool = False) -> ResidualResult:
    """Algorithm 1: F(n) given the lagged mean intensity J^dagger."""
    n = np.asarray(n)
    if istar is None:
        istar = conservation_rows(n)
    chi, eta = opacity_emissivity(m, n, Jdag)
    S = eta / chi
    out = solve_rays(chi, S, m.dz, m.mu, m.B[:, -1], want_derivs=want_lambda)
    I_up, I_dn = out[0], out[1]
    wmu = m.wmu[None, :, None]
    J = 0.5 * np.sum(wmu * (I_up + I_dn), axis=1)
    R_up, R_dn = rates_from_J(m, J)
    F = assemble(m, n, R_up, R_dn, istar)
    res = ResidualResult(F=F, J=J, R_up=R_up, R_dn=R_dn, istar=istar, chi=chi, eta=eta,
                         I_emergent=I_up[:, :, 0])
    if want_lambda:
        a_chi, a_eta, c_chi, c_eta = out[2]
        res.lam_chi = 0.5 * np.sum(wmu * (a_chi + c_chi), axis=1)
        res.lam_eta = 0.5 * np.sum(wmu * (a_eta + c_eta), axis=1)
    return res


def jvp_complex(m: Model, n, Jdag, v, istar=None, eps: float = COMPLEX_EPS):
    """J_F(n) v = Im F(n + i eps v) / eps (Eq. complex)."""
    n = np.asarray(n, dtype=float)
    if istar is None:
        istar = conservation_rows(n)
    res = residual(m, n + 1j * eps * np.asarray(v, dtype=float), Jdag, istar=istar)
    return res.F.imag / eps


def fd_step(n, v, scheme: str, choice: str) -> float:
    """Difference steps eps_1, eps_2 of the Fig. 2 caption."""
    vnorm = np.linalg.norm(v)
    if choice == "eps1":
        b = 1e-6
        return float(np.sum(b * np.abs(n)) / (n.size * vnorm) + b)
    r = 3.0 if scheme == "central" else 2.0
    return float(np.finfo(float).eps ** (1.0 / r) * np.sqrt(1.0 + np.linalg.norm(n)) / vnorm)


def jvp_fd(m: Model, n, Jdag, v, scheme: str = "forward", choice: str = "eps1",
           F0=None, istar=None, eps: Optional[float] = None):
    """Finite-difference JVPs (Eqs. fordif, backward, centdif)."""
    n = np.asarray(n, dtype=float)
    if istar is None:
        istar = conservation_rows(n)
    if eps is None:
        eps = fd_step(n, v, scheme, choice)
    if F0 is None and scheme != "central":
        F0 = residual(m, n, Jdag, istar=istar).F
    if scheme == "forward":
        return (residual(m, n + eps * v, Jdag, istar=istar).F - F0) / eps
    if scheme == "backward":
        return (F0 - residual(m, n - eps * v, Jdag, istar=istar).F) / eps
    Fp = residual(m, n + eps * v, Jdag, istar=istar).F
    Fm = residual(m, n - eps * v, Jdag, istar=istar).F
    return (Fp - Fm) / (2.0 * eps)
