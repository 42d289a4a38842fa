"""Oracle setup (test infrastructure only): grids, quadratures and tables.

Everything the residual needs that does not depend on the populations:
frequency and angle quadratures, LTE (Saha-Boltzmann) populations, Voigt
profiles, photo-ionisation cross-sections, the bound-free g_ij, Planck
functions, the background continuum and the collision rates. FP64 numpy,
one obvious loop or array expression per formula.

Pins (tests/test_oracle_model.py): Gauss-Legendre exactness, Voigt limits and
direct quadrature of the Voigt integral, Saha/Boltzmann ratios, detailed
balance of the collision rates, unit normalisation of the line profiles.

A moving column (line-of-sight velocity v, Sect. 3.4) gives every direction
of propagation mu_d its own line profile, centred at nu_0 (1 + mu_d v/c) and
renormalised on the line's window like the static one (reading: continua are
not shifted); ``Vdir`` holds them. Pins in tests/test_oracle_velocity.py.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np
from scipy.special import wofz

# cgs constants (CODATA 2018)
H = 6.62607015e-27
C = 2.99792458e10
KB = 1.380649e-16
ME = 9.1093837015e-28
QE = 4.80320471e-10
EV = 1.602176634e-12
AMU = 1.66053906660e-24
SIGMA_T = 6.6524587321e-25
FOURPI = 4.0 * np.pi


def gauss_legendre_01(n_mu: int):
    """Gauss-Legendre nodes and weights on ]0,1[ with sum(w) = 1 (Sect. 2.1.2)."""
    x, w = np.polynomial.legendre.leggauss(n_mu)
    return 0.5 * (x + 1.0), 0.5 * w


def line_offsets(n_nu: int, q_core: float, q_wing: float) -> np.ndarray:
    """Dimensionless line-grid offsets (grid rule documented in ``workloads``)."""
    u = 2.0 * np.arange(n_nu) / (n_nu - 1) - 1.0
    if q_wing <= 2.0 * q_core:
        return q_wing * u
    beta = 2.0 * np.arccosh(q_wing / (2.0 * q_core))
    return q_wing * np.sinh(beta * u) / np.sinh(beta)


def planck(nu, T):
    """B_nu(T) = (2 h nu^3 / c^2) / (exp(h nu / k T) - 1)."""
    return (2.0 * H * nu ** 3 / C ** 2) / np.expm1(H * nu / (KB * T))


def voigt_H(a, v):
    """Voigt function H(a, v) = Re w(v + i a), w the Faddeeva function (Sect. 3.1)."""
    return wofz(np.asarray(v) + 1j * np.asarray(a)).real


def saha_phi(gi, gj, Ei_eV, Ej_eV, T):
    """Saha-Boltzmann function Phi_ij(T) (Sect. 2.1.1, the equation after Eq. Vij2)."""
    return (gi / (2.0 * gj)) * (H ** 2 / (2.0 * np.pi * ME * KB * T)) ** 1.5 \
        * np.exp((Ej_eV - Ei_eV) * EV / (KB * T))


def lte_populations(atom, col) -> np.ndarray:
    """LTE populations n*[k, l] summing to n_tot (Saha-Boltzmann, Sect. 2.1.1).

    n*_l is proportional to g_l exp(-E_l/kT) [2 (2 pi m_e k T/h^2)^{3/2} / n_e]^(stage_l - stage_0),
    which reproduces n*_i/n*_j = n_e Phi_ij(T) across one ionisation stage and the
    Boltzmann ratio within a stage.
    """
    T = col.T[:, None]
    ne = col.ne[:, None]
    st = (atom.stage - atom.stage.min())[None, :]
    logw = (np.log(atom.g)[None, :] - atom.E_eV[None, :] * EV / (KB * T)
            + st * np.log(2.0 * (2.0 * np.pi * ME * KB * T / H ** 2) ** 1.5 / ne))
    logw -= logw.max(axis=1, keepdims=True)
    w = np.exp(logw)
    return col.ntot[:, None] * w / w.sum(axis=1, keepdims=True)


@dataclass
class Transition:
    kind: str          # "bb" or "bf"
    lo: int
    up: int
    q0: int            # first union-grid index of the window
    q1: int            # last union-grid index (inclusive)
    nu0: float         # line centre or edge frequency [Hz]


@dataclass
class Model:
    """All population-independent quantities of one column, FP64."""
    nz: int
    nl: int
    nt: int
    nq: int
    nmu: int
    nu: np.ndarray         # [nq] union frequency grid, ascending
    mu: np.ndarray         # [nmu]
    wmu: np.ndarray        # [nmu]
    z: np.ndarray          # [nz]
    dz: np.ndarray         # [nz-1] |z_k - z_{k+1}|
    T: np.ndarray
    ne: np.ndarray
    ntot: np.ndarray
    trans: List[Transition]
    omega: np.ndarray      # [nt, nq] quadrature weight of transition t at nu_q (0 outside window)
    V: np.ndarray          # [nt, nq, nz] V_ij (0 outside window), Eqs. Vij / Vij2
    g: np.ndarray          # [nt, nq, nz] g_ij, Eq. gij (bf) or g_i/g_j (bb)
    twohnu3c2: np.ndarray  # [nq]
    chi_c: np.ndarray      # [nq, nz] continuum absorption
    chi_sca: np.ndarray    # [nz] background scattering
    eta_c: np.ndarray      # [nq, nz] continuum emissivity
    B: np.ndarray          # [nq, nz] Planck function
    Cmat: np.ndarray       # [nz, nl, nl] collision rate i -> j
    nstar: np.ndarray      # [nz, nl] LTE populations
    active: np.ndarray     # [nt, nq] bool window mask
    vlos: np.ndarray = None    # [nz] line-of-sight velocity (> 0 upward), None for a static column
    mu_dir: np.ndarray = None  # [2 nmu] signed direction cosines: +mu (outgoing) then -mu (ingoing)
    Vdir: np.ndarray = None    # [nt, 2 nmu, nq, nz] V_ij seen by each direction (moving column only)

    @property
    def ray_points(self) -> int:
        return self.nq * 2 * self.nmu * self.nz


def _frequency_grids(atom):
    """Per-transition grids, merged into one ascending union grid."""
    per = []
    for ln in atom.lines:
        nu0 = (atom.E_eV[ln.j] - atom.E_eV[ln.i]) * EV / H
        x = line_offsets(ln.n_nu, ln.q_core, ln.q_wing)
        per.append(("bb", ln, nu0, nu0 * (1.0 + x * atom.vchar / C)))
    for ct in atom.conts:
        nue = (atom.E_eV[ct.j] - atom.E_eV[ct.i]) * EV / H
        s = np.arange(ct.n_nu) / (ct.n_nu - 1)
        per.append(("bf", ct, nue, nue * ct.y_max ** s))
    allnu = np.unique(np.concatenate([p[3] for p in per]))
    return per, allnu


def build_model(atom, col, n_mu: int = 5) -> Model:
    """Section 2.1 quantities for one atom on one column."""
    per, nu = _frequency_grids(atom)
    nq, nz, nl = len(nu), col.n_depth, atom.n_levels
    nt = len(per)
    mu, wmu = gauss_legendre_01(n_mu)
    T, ne = col.T, col.ne
    vturb = np.zeros(nz) if col.vturb is None else col.vturb
    trans, omega = [], np.zeros((nt, nq))
    V = np.zeros((nt, nq, nz))
    g = np.zeros((nt, nq, nz))
    active = np.zeros((nt, nq), dtype=bool)
    Cmat = np.zeros((nz, nl, nl))
    nstar = lte_populations(atom, col)
    for t, (kind, d, nu0, grid) in enumerate(per):
        q0 = int(np.searchsorted(nu, grid.min()))
        q1 = int(np.searchsorted(nu, grid.max()))
        trans.append(Transition(kind, d.i, d.j, q0, q1, nu0))
        win = nu[q0:q1 + 1]
        active[t, q0:q1 + 1] = True
        # trapezoid weights on the union points inside the window
        w = np.zeros(len(win))
        if len(win) > 1:
            dnu = np.diff(win)
            w[:-1] += 0.5 * dnu
            w[1:] += 0.5 * dnu
        omega[t, q0:q1 + 1] = w
        gi, gj = atom.g[d.i], atom.g[d.j]
        Ei, Ej = atom.E_eV[d.i], atom.E_eV[d.j]
        if kind == "bb":
            # Eq. Vij with (h nu / 4 pi) B_ij phi = (pi e^2 / m_e c) f phi
            dnud = nu0 / C * np.sqrt(2.0 * KB * T / (atom.mass_amu * AMU) + vturb ** 2)   # [nz]
            v = (win[:, None] - nu0) / dnud[None, :]
            phi = voigt_H(d.damping, v) / (np.sqrt(np.pi) * dnud[None, :])
            phi = phi / np.sum(w[:, None] * phi, axis=0, keepdims=True)   # sum_q omega phi = 1
            V[t, q0:q1 + 1, :] = (np.pi * QE ** 2 / (ME * C)) * d.f * phi
            g[t, q0:q1 + 1, :] = gi / gj
            # collisions (detailed balance with n*)
            hnu_kt = H * nu0 / (KB * T)
            if d.eps > 0.0:
                Aji = 8.0 * np.pi ** 2 * QE ** 2 * nu0 ** 2 / (ME * C ** 3) * (gi / gj) * d.f
                Cdown = d.eps * Aji / ((1.0 - d.eps) * (-np.expm1(-hnu_kt)))
            else:
                Cdown = 8.63e-6 * ne * d.upsilon / (gj * np.sqrt(T))
            Cmat[:, d.j, d.i] += Cdown
            Cmat[:, d.i, d.j] += Cdown * (gj / gi) * np.exp(-hnu_kt)
        else:
            # Eq. Vij2 and Eq. gij with hydrogenic alpha(nu) = alpha0 (nu_edge / nu)^3
            V[t, q0:q1 + 1, :] = (d.alpha0 * (nu0 / win) ** 3)[:, None]
            ratio = ne * saha_phi(gi, gj, Ei, Ej, T)            # n_i* / n_j*
            g[t, q0:q1 + 1, :] = ratio[None, :] * np.exp(-H * win[:, None] / (KB * T[None, :]))
            Cup = ne * d.q0 * np.sqrt(T) * np.exp(-(Ej - Ei) * EV / (KB * T))
            Cmat[:, d.i, d.j] += Cup
            Cmat[:, d.j, d.i] += Cup * ratio
    # a moving column: each direction sees its own Doppler-shifted line profile
    vlos = getattr(col, "vlos", None)
    Vdir, mu_dir = None, None
    if vlos is not None and np.any(vlos != 0.0):
        mu_dir = np.concatenate([mu, -mu])
        Vdir = np.zeros((nt, 2 * n_mu, nq, nz))
        for t, (kind, d, nu0, grid) in enumerate(per):
            tr = trans[t]
            if kind != "bb":
                Vdir[t] = V[t][None]                    # continua: no Doppler shift
                continue
            win = nu[tr.q0:tr.q1 + 1]
            w = omega[t, tr.q0:tr.q1 + 1]
            dnud = nu0 / C * np.sqrt(2.0 * KB * T / (atom.mass_amu * AMU) + vturb ** 2)
            for dd in range(2 * n_mu):
                # profile of the gas moving at vlos seen along direction mu_d:
                # centred at nu0 (1 + mu_d v / c), renormalised on the window
                v = (win[:, None] - nu0 * (1.0 + mu_dir[dd] * vlos[None, :] / C)) / dnud[None, :]
                phi = voigt_H(d.damping, v) / (np.sqrt(np.pi) * dnud[None, :])
                phi = phi / np.sum(w[:, None] * phi, axis=0, keepdims=True)
                Vdir[t, dd, tr.q0:tr.q1 + 1, :] = (np.pi * QE ** 2 / (ME * C)) * d.f * phi
    B = planck(nu[:, None], T[None, :])
    kap = np.full(nq, col.kappa)
    if col.kappa_power != 0.0:
        kap = col.kappa * np.minimum(col.kappa_max,
                                     np.maximum(1.0, (nu / col.kappa_nu_ref) ** col.kappa_power))
    chi_c = kap[:, None] * col.rho[None, :]
    chi_sca = SIGMA_T * ne if col.thomson else np.zeros(nz)
    eta_c = chi_c * B
    dz = np.abs(np.diff(col.z))
    return Model(nz=nz, nl=nl, nt=nt, nq=nq, nmu=n_mu, nu=nu, mu=mu, wmu=wmu,
                 z=col.z.copy(), dz=dz, T=T.copy(), ne=ne.copy(), ntot=col.ntot.copy(),
                 trans=trans, omega=omega, V=V, g=g,
                 twohnu3c2=2.0 * H * nu ** 3 / C ** 2, chi_c=chi_c, chi_sca=chi_sca,
                 eta_c=eta_c, B=B, Cmat=Cmat, nstar=nstar, active=active,
                 vlos=None if Vdir is None else np.array(vlos, dtype=float), mu_dir=mu_dir, Vdir=Vdir)


def initial_J(model: Model) -> np.ndarray:
    """Initial estimate of the mean intensity, J = B_nu(T) (LTE radiation field)."""
    return model.B.copy()
