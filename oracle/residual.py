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

A moving column (line-of-sight velocity, Sect. 3.4) takes the per-direction
path of ``_residual_moving``.

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
    # moving column: chi, eta are per direction [2 nmu, nq, nz]; the local
    # derivatives of each direction's intensity, not angle-averaged
    lam_chi_dir: Optional[np.ndarray] = None   # [2 nmu, nq, nz] dI_d^k/dchi_d^k
    lam_eta_dir: Optional[np.ndarray] = None   # [2 nmu, nq, nz] dI_d^k/deta_d^k


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


def opacity_emissivity_dir(m: Model, n, Jdag):
    """Eqs. chi and eta for a moving column, per direction d (the profile of
    transition t seen along mu_d is Vdir[t, d]): [2 nmu, nq, nz] each."""
    nd = 2 * m.nmu
    zero = np.zeros((nd, 1, 1), dtype=np.result_type(n, Jdag))
    chi = (m.chi_c + m.chi_sca[None, :])[None] + zero
    eta = (m.eta_c + m.chi_sca[None, :] * Jdag)[None] + zero
    for t, tr in enumerate(m.trans):
        ni = n[:, tr.lo][None, None, :]
        nj = n[:, tr.up][None, None, :]
        chi = chi + m.Vdir[t] * (ni - m.g[t][None] * nj)
        eta = eta + m.twohnu3c2[None, :, None] * m.g[t][None] * m.Vdir[t] * nj
    return chi, eta


def direction_weights(m: Model) -> np.ndarray:
    """1/2 w_mu of each direction (outgoing, then ingoing): J = sum_d h_d I_d."""
    return 0.5 * np.concatenate([m.wmu, m.wmu])


def _residual_moving(m: Model, n, Jdag, istar, want_lambda: bool) -> "ResidualResult":
    """Algorithm 1 for a moving column (Sect. 3.4): every direction carries its
    own opacity and source function, the formal solution runs per ray with
    them, J = sum_d h_d I_d feeds the background scattering, and the rate
    integrals weight each direction's intensity with the profile it sees:
    R_ij = sum_nu W sum_d h_d V_d I_d, R_ji = sum_nu W g sum_d h_d V_d (2 h nu^3/c^2 + I_d)."""
    chi, eta = opacity_emissivity_dir(m, n, Jdag)
    S = eta / chi
    nmu, nd = m.nmu, 2 * m.nmu
    dtype = np.result_type(chi, S, float)
    I = np.zeros((nd, m.nq, m.nz), dtype=dtype)
    lx = np.zeros_like(I) if want_lambda else None
    le = np.zeros_like(I) if want_lambda else None
    for a in range(nmu):
        mu_a = m.mu[a:a + 1]
        up = solve_rays(chi[a], S[a], m.dz, mu_a, m.B[:, -1], want_derivs=want_lambda)
        dn = solve_rays(chi[nmu + a], S[nmu + a], m.dz, mu_a, m.B[:, -1], want_derivs=want_lambda)
        I[a] = up[0][:, 0, :]
        I[nmu + a] = dn[1][:, 0, :]
        if want_lambda:
            lx[a], le[a] = up[2][0][:, 0, :], up[2][1][:, 0, :]
            lx[nmu + a], le[nmu + a] = dn[2][2][:, 0, :], dn[2][3][:, 0, :]
    h = direction_weights(m)
    J = np.einsum("d,dqk->qk", h, I)
    Wq = FOURPI / (H * m.nu)
    R_up = np.zeros((m.nt, m.nz), dtype=dtype)
    R_dn = np.zeros((m.nt, m.nz), dtype=dtype)
    for t in range(m.nt):
        W = m.omega[t][:, None] * Wq[:, None]                     # [nq, 1]
        hv = h[:, None, None] * m.Vdir[t]                         # [nd, nq, nz]
        R_up[t] = np.sum(W * np.sum(hv * I, axis=0), axis=0)
        R_dn[t] = np.sum(W * m.g[t] * np.sum(hv * (m.twohnu3c2[None, :, None] + I), axis=0), axis=0)
    F = assemble(m, n, R_up, R_dn, istar)
    res = ResidualResult(F=F, J=J, R_up=R_up, R_dn=R_dn, istar=istar, chi=chi, eta=eta,
                         I_emergent=np.stack([I[a][:, 0] for a in range(nmu)], axis=1))
    if want_lambda:
        res.lam_chi_dir, res.lam_eta_dir = lx, le
        res.lam_chi = np.einsum("d,dqk->qk", h, lx)
        res.lam_eta = np.einsum("d,dqk->qk", h, le)
    return res


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
    if m.Vdir is not None:
        return _residual_moving(m, n, Jdag, istar, want_lambda)
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
