"""Oracle formal solver (test infrastructure only).

Piecewise-linear short characteristics (Sect. 2.1.2, Eqs. Iplus/Iminus,
coefficients of App. A.1, Olson & Kunasz 1987) with the boundary conditions
I(bottom, mu>0) = B_nu(T_bottom) and I(top, mu<0) = 0, and the derivative
coefficients a_chi, a_eta, c_chi, c_eta of App. A.2.

Every routine accepts complex arrays (complex-step JVPs, Eq. complex): the
coefficient functions are analytic, using a Taylor series below
``DTAU_SERIES`` so that no cancellation spoils either the real or the
imaginary part (the paper asks for the perturbed equations to be
linearised for this reason, Sect. 2.4.2). Branches are chosen on Re(dtau).

Pins (tests/test_oracle_formal.py): exact reproduction of the closed-form
solution for a source function linear in optical depth, the constant-S slab,
agreement of the series and direct branches, and the analytic derivatives
against brute-force differences.
"""
from __future__ import annotations

import math

import numpy as np

DTAU_SERIES = 0.1
_NSER = 14
# a(x) = sum_{n>=1} (-1)^(n+1) x^n/(n+1)!, b(x) = sum_{n>=1} (-1)^(n+1) n x^n/(n+1)!
_A_COEF = [(-1.0) ** (n + 1) / math.factorial(n + 1) for n in range(1, _NSER + 1)]
_B_COEF = [(-1.0) ** (n + 1) * n / math.factorial(n + 1) for n in range(1, _NSER + 1)]


def _poly(coefs, x):
    """sum_i coefs[i] x^(i+1) by Horner (analytic, complex-safe)."""
    acc = np.zeros_like(x) + coefs[-1]
    for c in reversed(coefs[:-1]):
        acc = acc * x + c
    return acc * x


def pl_coefficients(dtau):
    """e = exp(-dtau), a = 1 - (1-e)/dtau, b = (1-e)/dtau - e, and b/dtau (App. A.1)."""
    dtau = np.asarray(dtau)
    e = np.exp(-dtau)
    small = dtau.real < DTAU_SERIES
    safe = np.where(small, 1.0, dtau)
    w = (1.0 - e) / safe
    a_dir = 1.0 - w
    b_dir = w - e
    bq_dir = b_dir / safe
    xs = np.where(small, dtau, 0.0)
    a_ser = _poly(_A_COEF, xs)
    b_ser = _poly(_B_COEF, xs)
    # b/dtau = sum_{n>=1} (-1)^(n+1) n x^(n-1)/(n+1)!
    bq_ser = _poly(_B_COEF[1:], xs) + _B_COEF[0]
    return (e, np.where(small, a_ser, a_dir), np.where(small, b_ser, b_dir),
            np.where(small, bq_ser, bq_dir))


def solve_rays(chi, S, dz, mu, I_bottom, want_derivs=False):
    """Intensities along all rays of one column.

    chi, S : [..., nz] opacity and source function (depth last, index 0 = top)
    dz     : [nz-1] |z_k - z_{k+1}|
    mu     : [nmu] positive direction cosines
    I_bottom : [...] incident intensity at the bottom for mu > 0 (B_nu(T_bottom))

    Returns I_up, I_dn of shape [..., nmu, nz]; with ``want_derivs`` also the
    local derivatives dI^k/dchi^k and dI^k/deta^k for both hemispheres
    (App. A.2: a_chi, a_eta for mu > 0 and c_chi, c_eta for mu < 0).
    """
    chi = chi[..., None, :]
    S = S[..., None, :]
    nz = chi.shape[-1]
    shape = np.broadcast_shapes(chi.shape[:-1], (len(mu),))
    dtype = np.result_type(chi, S, np.asarray(I_bottom), float)
    I_up = np.zeros(shape + (nz,), dtype=dtype)
    I_dn = np.zeros(shape + (nz,), dtype=dtype)
    if want_derivs:
        a_chi = np.zeros(shape + (nz,), dtype=dtype)
        a_eta = np.zeros(shape + (nz,), dtype=dtype)
        c_chi = np.zeros(shape + (nz,), dtype=dtype)
        c_eta = np.zeros(shape + (nz,), dtype=dtype)
    # outgoing rays, mu > 0: I^k = I^{k+1} e^{-dtau^k} + a^k S^k + b^k S^{k+1}  (Eq. Iplus)
    I_up[..., nz - 1] = np.asarray(I_bottom)[..., None]
    for k in range(nz - 2, -1, -1):
        h = dz[k] / (2.0 * mu)
        dtau = h * (chi[..., k] + chi[..., k + 1])
        e, a, b, bq = pl_coefficients(dtau)
        I_up[..., k] = I_up[..., k + 1] * e + a * S[..., k] + b * S[..., k + 1]
        if want_derivs:
            common = h * (e * (S[..., k + 1] - I_up[..., k + 1]) - (S[..., k + 1] - S[..., k]) * bq)
            a_chi[..., k] = -(S[..., k] / chi[..., k]) * a + common
            a_eta[..., k] = a / chi[..., k]
    # ingoing rays, mu < 0: I^k = I^{k-1} e^{-dtau^{k-1}} + a^{k-1} S^k + b^{k-1} S^{k-1}  (Eq. Iminus)
    I_dn[..., 0] = 0.0
    for k in range(1, nz):
        h = dz[k - 1] / (2.0 * mu)
        dtau = h * (chi[..., k - 1] + chi[..., k])
        e, a, b, bq = pl_coefficients(dtau)
        I_dn[..., k] = I_dn[..., k - 1] * e + a * S[..., k] + b * S[..., k - 1]
        if want_derivs:
            common = h * (e * (S[..., k - 1] - I_dn[..., k - 1]) - (S[..., k - 1] - S[..., k]) * bq)
            c_chi[..., k] = -(S[..., k] / chi[..., k]) * a + common
            c_eta[..., k] = a / chi[..., k]
    if want_derivs:
        return I_up, I_dn, (a_chi, a_eta, c_chi, c_eta)
    return I_up, I_dn
