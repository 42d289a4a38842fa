"""Pins of the oracle formal solver (no GPU)."""
import numpy as np
import pytest

from oracle import formal as OF


def _column(nz=40, seed=0):
    rng = np.random.default_rng(seed)
    dz = rng.uniform(0.5, 2.0, nz - 1)
    chi = 10.0 ** rng.uniform(-3, 1, nz)
    tau = np.concatenate([[0.0], np.cumsum(0.5 * dz * (chi[:-1] + chi[1:]))])
    return dz, chi, tau


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (0.3, 2.0), (5.0, -0.01)])
def test_linear_source_function_is_exact(alpha, beta):
    """For S linear in optical depth the piecewise-linear scheme is exact (App. A.1)."""
    dz, chi, tau = _column()
    S = alpha + beta * tau
    mu = np.array([0.1, 0.5, 1.0])
    Ib = 0.7
    I_up, I_dn = OF.solve_rays(chi, S, dz, mu, Ib)
    for m, mm in enumerate(mu):
        T = tau / mm
        TN = T[-1]
        E = np.exp(-(TN - T))
        up = alpha * (1 - E) + beta * mm * ((T + 1) - (TN + 1) * E) + Ib * E
        dn = alpha * (1 - np.exp(-T)) + beta * mm * (T - (1 - np.exp(-T)))
        np.testing.assert_allclose(I_up[m], up, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(I_dn[m], dn, rtol=1e-12, atol=1e-14)


def test_boundary_conditions_and_thick_slab():
    dz, chi, tau = _column(60, 3)
    S = np.full(60, 2.5)
    I_up, I_dn = OF.solve_rays(chi * 1e3, S, dz, np.array([0.3, 0.9]), 9.0)
    assert np.all(I_dn[:, 0] == 0.0)
    assert np.all(I_up[:, -1] == 9.0)
    np.testing.assert_allclose(I_up[:, 0], 2.5, rtol=1e-12)   # thick: emergent I = S


def test_series_and_direct_branches_agree():
    x = np.array([OF.DTAU_SERIES * (1 - 1e-12), OF.DTAU_SERIES * (1 + 1e-12)])
    e, a, b, bq = OF.pl_coefficients(x)
    assert a[0] == pytest.approx(a[1], rel=1e-13)
    assert b[0] == pytest.approx(b[1], rel=1e-13)
    assert bq[0] == pytest.approx(bq[1], rel=1e-12)
    # exact values from the definitions at a moderate argument, in extended precision
    from mpmath import mp, mpf, exp
    mp.dps = 40
    for xv in [1e-9, 1e-3, 0.05, 0.3, 7.0]:
        X = mpf(xv)
        w = (1 - exp(-X)) / X
        e, a, b, bq = OF.pl_coefficients(np.array([xv]))
        assert a[0] == pytest.approx(float(1 - w), rel=1e-14)
        assert b[0] == pytest.approx(float(w - exp(-X)), rel=1e-14)
        assert bq[0] == pytest.approx(float((w - exp(-X)) / X), rel=1e-14)


def test_complex_step_through_coefficients():
    x = np.array([1e-6, 0.05, 0.2, 3.0])
    h = 1e-200
    e, a, b, bq = OF.pl_coefficients(x + 1j * h)
    # d a / dx = b / x, d b / dx = e - b / x (derivatives of the App. A.1 coefficients)
    np.testing.assert_allclose(a.imag / h, bq.real, rtol=1e-13)
    np.testing.assert_allclose(b.imag / h, e.real - bq.real, rtol=1e-12)


def test_local_derivative_coefficients_against_differences():
    """App. A.2 a_chi, a_eta, c_chi, c_eta equal dI^k/dchi^k and dI^k/deta^k."""
    nz = 12
    dz, chi, tau = _column(nz, 5)
    eta = chi * (1.0 + np.linspace(0, 1, nz) ** 2)
    mu = np.array([0.25, 0.8])
    I_up, I_dn, (a_chi, a_eta, c_chi, c_eta) = OF.solve_rays(chi, eta / chi, dz, mu, 1.3, want_derivs=True)
    h = 1e-30
    for k in range(nz):
        for which in ("chi", "eta"):
            c2 = chi.astype(complex).copy()
            e2 = eta.astype(complex).copy()
            if which == "chi":
                c2[k] += 1j * h
            else:
                e2[k] += 1j * h
            Iu, Id = OF.solve_rays(c2, e2 / c2, dz, mu, 1.3)
            du, dd = Iu[:, k].imag / h, Id[:, k].imag / h
            ref_u = a_chi[:, k] if which == "chi" else a_eta[:, k]
            ref_d = c_chi[:, k] if which == "chi" else c_eta[:, k]
            np.testing.assert_allclose(ref_u, du, rtol=1e-10, atol=1e-14 * np.max(np.abs(du)))
            np.testing.assert_allclose(ref_d, dd, rtol=1e-10, atol=1e-14 * np.max(np.abs(dd)))
