"""Oracle block-Jacobi preconditioner (test infrastructure only).

The "first solution" of Sect. 2.5.2 (background-scattering derivatives
neglected), the choice the paper makes for its JFNK solvers: per depth k,

  P^k_ij = Gamma^k_ij + A^kk_ij          (Sect. 2.5.1)
  Gamma^k_ij = delta_ij sum_p (C_ip + R_ip) - (C_ji + R_ji)
  A^kk_ij    = sum_nu sum_t s_it W_t(nu) chi_t(nu) [beta_j dJ/dchi^k + gamma_j dJ/deta^k]

where chi_t = V_t (n_lo - g_t n_up) is the opacity of transition t, W_t the
rate quadrature weight omega_t 4 pi / (h nu), s_it = +1 (-1) when i is the
lower (upper) level of t, dJ/dchi^k and dJ/deta^k the angle averages of the
App. A.2 coefficients, and the conservation row replaced by -1 (Sect. 2.5.1).

The second and third solutions of Sect. 2.5.2 (``variant`` 2 and 3) add the
background-scattering term chi_sca d J/d n_j to d eta/d n_j: lagged from the
previous preconditioner build (2), or solved locally (3). ``dJ_dn`` holds the
three readings.

Reading of beta_j (the printed sum_{s>j} V_js (1 - g_js) is garbled):
beta_j = d chi / d n_j = sum_{t: lo=j} V_t - sum_{t: up=j} g_t V_t, derived from
Eq. chi; gamma_j = d eta / d n_j = sum_{t: up=j} (2 h nu^3 / c^2) g_t V_t.

With J^dagger frozen these blocks are exactly the diagonal blocks of the
Jacobian of F; tests/test_oracle_residual.py checks that against the dense
complex-step Jacobian.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .model import FOURPI, H, Model


def _alpha_beta_gamma(m: Model, n):
    """alpha_i = sum_t s_it W_t chi_t, beta_j = d chi/d n_j, gamma_j = d eta/d n_j, each [nl, nq, nz]."""
    nl, nq, nz = m.nl, m.nq, m.nz
    Wnu = FOURPI / (H * m.nu)
    alpha = np.zeros((nl, nq, nz))
    beta = np.zeros((nl, nq, nz))
    gamma = np.zeros((nl, nq, nz))
    for t, tr in enumerate(m.trans):
        lo, up = tr.lo, tr.up
        chi_t = m.V[t] * (n[:, lo][None, :] - m.g[t] * n[:, up][None, :])
        Wchi = m.omega[t][:, None] * Wnu[:, None] * chi_t
        alpha[lo] += Wchi
        alpha[up] -= Wchi
        beta[lo] += m.V[t]
        beta[up] -= m.g[t] * m.V[t]
        gamma[up] += m.twohnu3c2[:, None] * m.g[t] * m.V[t]
    return alpha, beta, gamma


def dJ_dn(m: Model, n, res, variant: int = 1, D_prev=None) -> np.ndarray:
    """Local estimate of d J_nu^k / d n_j^k, [nl, nq, nz], after one of the three
    solutions of Sect. 2.5.2 (Lchi, Leta: angle averages of dI^k/dchi^k, dI^k/deta^k):
      1: beta_j Lchi + gamma_j Leta (background-scattering derivative neglected);
      2: beta_j Lchi + (gamma_j + chi_sca D_prev_j) Leta, D_prev the previous
         estimate of d J/d n_j (lagged; zero when none);
      3: (beta_j Lchi + gamma_j Leta) / (1 - chi_sca Leta), the local terms of the
         self-consistent solution (coefficient r_k of Sect. 2.5.2)."""
    n = np.real(np.asarray(n))
    _, beta, gamma = _alpha_beta_gamma(m, n)
    lx, le = np.real(res.lam_chi)[None], np.real(res.lam_eta)[None]
    sca = m.chi_sca[None, None, :]
    if variant == 1:
        return beta * lx + gamma * le
    if variant == 2:
        Dp = np.zeros_like(beta) if D_prev is None else D_prev
        return beta * lx + (gamma + sca * Dp) * le
    if variant == 3:
        return (beta * lx + gamma * le) / (1.0 - sca * le)
    raise ValueError("variant must be 1, 2 or 3")


def _moving_radiative_block(m: Model, n, res) -> np.ndarray:
    """A^kk of a moving column: every direction d has its own opacity and
    profile, so sum_nu sum_d h_d alpha_{i,d} (beta_{j,d} dI_d/dchi_d + gamma_{j,d} dI_d/deta_d)
    with alpha_{i,d} = sum_t s_it W chi_{t,d} and beta, gamma from Vdir (first solution)."""
    from .residual import direction_weights
    nl, nq, nz, nd = m.nl, m.nq, m.nz, 2 * m.nmu
    Wnu = FOURPI / (H * m.nu)
    h = direction_weights(m)
    alpha = np.zeros((nl, nd, nq, nz))
    beta = np.zeros((nl, nd, nq, nz))
    gamma = np.zeros((nl, nd, nq, nz))
    for t, tr in enumerate(m.trans):
        lo, up = tr.lo, tr.up
        Vd = m.Vdir[t]
        chi_t = Vd * (n[:, lo][None, None, :] - m.g[t][None] * n[:, up][None, None, :])
        Wchi = (m.omega[t] * Wnu)[None, :, None] * chi_t
        alpha[lo] += Wchi
        alpha[up] -= Wchi
        beta[lo] += Vd
        beta[up] -= m.g[t][None] * Vd
        gamma[up] += m.twohnu3c2[None, :, None] * m.g[t][None] * Vd
    zeta = beta * np.real(res.lam_chi_dir)[None] + gamma * np.real(res.lam_eta_dir)[None]
    return np.einsum("d,idqk,jdqk->kij", h, alpha, zeta)


def block_jacobi(m: Model, n, res, variant: int = 1, D_prev=None) -> np.ndarray:
    """P[k] (nl x nl) from a residual evaluation made with ``want_lambda``."""
    n = np.real(np.asarray(n))
    nl, nz = m.nl, m.nz
    P = np.zeros((nz, nl, nl))
    if m.Vdir is not None and variant != 1:
        raise NotImplementedError("moving columns: the first solution of Sect. 2.5.2 only")
    alpha, _, _ = _alpha_beta_gamma(m, n)
    for t, tr in enumerate(m.trans):
        lo, up = tr.lo, tr.up
        # Gamma: direct dependence of kappa_t on n_lo, n_up
        up_rate = m.Cmat[:, lo, up] + res.R_up[t]
        dn_rate = m.Cmat[:, up, lo] + res.R_dn[t]
        P[:, lo, lo] += up_rate
        P[:, lo, up] -= dn_rate
        P[:, up, lo] -= up_rate
        P[:, up, up] += dn_rate
    if m.Vdir is not None:
        P += _moving_radiative_block(m, n, res)
    else:
        zeta = dJ_dn(m, n, res, variant, D_prev)
        P += np.einsum("iqk,jqk->kij", alpha, zeta)
    P[np.arange(nz), res.istar, :] = -1.0
    return P


def lu_factor_blocks(P):
    return [sla.lu_factor(P[k]) for k in range(P.shape[0])]


def apply_inverse(lus, x):
    """P^{-1} x, depth by depth."""
    x = np.asarray(x).reshape(len(lus), -1)
    return np.stack([sla.lu_solve(lus[k], x[k]) for k in range(len(lus))])
