"""Pins of the oracle setup against closed forms and brute force (no GPU)."""
import numpy as np
import pytest
from scipy import integrate

import workloads as W
from oracle import model as OM


@pytest.mark.parametrize("n_mu", [1, 2, 3, 5, 8])
def test_gauss_legendre_exact_moments(n_mu):
    mu, w = OM.gauss_legendre_01(n_mu)
    assert np.all((mu > 0) & (mu < 1))
    for p in range(2 * n_mu):
        assert abs(np.sum(w * mu ** p) - 1.0 / (p + 1)) < 1e-14


def _voigt_by_quadrature(a, v):
    # H(a, v) = a/pi int exp(-y^2) / ((v - y)^2 + a^2) dy, split at the Lorentz peak
    f = lambda y: np.exp(-y * y) / ((v - y) ** 2 + a * a)
    pts = sorted({-8.0, v - 50 * a, v, v + 50 * a, 8.0})
    pts = [p for p in pts if -8.0 <= p <= 8.0]
    total = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        val, _ = integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-13, limit=400)
        total += val
    # tails beyond |y| = 8 (exp(-64) ~ 1e-28) are negligible at these v
    return a / np.pi * total


@pytest.mark.parametrize("a,v", [(1e-3, 0.0), (1e-3, 2.5), (1e-2, 4.0), (0.1, 0.3), (0.1, 6.0), (0.05, 1.7)])
def test_voigt_matches_its_defining_integral(a, v):
    assert OM.voigt_H(a, v) == pytest.approx(_voigt_by_quadrature(a, v), rel=1e-9)


def test_voigt_limits():
    v = np.linspace(-5, 5, 41)
    np.testing.assert_allclose(OM.voigt_H(0.0, v), np.exp(-v * v), rtol=1e-14)
    a = 1e-3
    for vv in [40.0, 80.0]:
        lor = a / (np.sqrt(np.pi) * vv * vv) * (1 + 1.5 / vv ** 2)
        assert OM.voigt_H(a, vv) == pytest.approx(lor, rel=1e-5)
    # H(a, 0) = exp(a^2) erfc(a)
    from scipy.special import erfc
    for aa in [1e-3, 0.1, 0.5]:
        assert OM.voigt_H(aa, 0.0) == pytest.approx(np.exp(aa * aa) * erfc(aa), rel=1e-13)
    # unit area: int H dv = sqrt(pi)
    val, _ = integrate.quad(lambda x: OM.voigt_H(0.02, x), -np.inf, np.inf, limit=500)
    assert val == pytest.approx(np.sqrt(np.pi), rel=1e-8)


def test_planck_limits():
    T = 6000.0
    nu_rj = 1e10
    rj = 2 * nu_rj ** 2 * OM.KB * T / OM.C ** 2
    assert OM.planck(nu_rj, T) == pytest.approx(rj, rel=1e-5)
    nu_w = 3e16
    wien = 2 * OM.H * nu_w ** 3 / OM.C ** 2 * np.exp(-OM.H * nu_w / (OM.KB * T))
    assert OM.planck(nu_w, T) == pytest.approx(wien, rel=1e-12)


def test_lte_saha_boltzmann_ratios():
    atom = W.ca_like_atom(0)
    col = W.chromosphere(20)
    n = OM.lte_populations(atom, col)
    np.testing.assert_allclose(n.sum(axis=1), col.ntot, rtol=1e-14)
    kT = OM.KB * col.T
    # Boltzmann within the stage
    for i, j in [(0, 1), (0, 3), (2, 4)]:
        ratio = atom.g[j] / atom.g[i] * np.exp(-(atom.E_eV[j] - atom.E_eV[i]) * OM.EV / kT)
        np.testing.assert_allclose(n[:, j] / n[:, i], ratio, rtol=1e-12)
    # Saha across the stage, written out from the textbook form
    lam3 = (OM.H ** 2 / (2 * np.pi * OM.ME * kT)) ** 1.5
    for i in range(5):
        ratio_ci = 2.0 * atom.g[5] / atom.g[i] / (col.ne * lam3) * np.exp(-(atom.E_eV[5] - atom.E_eV[i]) * OM.EV / kT)
        np.testing.assert_allclose(n[:, 5] / n[:, i], ratio_ci, rtol=1e-11)


def test_profiles_normalised_and_collisions_in_detailed_balance():
    wl = W.config2(nu_scale=0.2, n_depth=12)
    m = OM.build_model(wl.atom, wl.columns[0], 3)
    for t, tr in enumerate(m.trans):
        if tr.kind == "bb":
            phi = m.V[t] / ((np.pi * OM.QE ** 2 / (OM.ME * OM.C)) * wl.atom.lines[t].f)
            np.testing.assert_allclose(np.sum(m.omega[t][:, None] * phi, axis=0), 1.0, rtol=1e-13)
        # quadrature weights cover the window exactly
        assert np.sum(m.omega[t]) == pytest.approx(m.nu[tr.q1] - m.nu[tr.q0], rel=1e-13)
        i, j = tr.lo, tr.up
        np.testing.assert_allclose(m.nstar[:, i] * m.Cmat[:, i, j], m.nstar[:, j] * m.Cmat[:, j, i], rtol=1e-12)


def test_union_grid_and_windows():
    wl = W.config3(nu_scale=0.2, n_depth=10)
    m = OM.build_model(wl.atom, wl.columns[0], 3)
    assert np.all(np.diff(m.nu) > 0)
    # every union point lies inside at least one window, and windows contain their own grid
    assert np.all(m.active.any(axis=0))
    nlines = len(wl.atom.lines)
    for t, tr in enumerate(m.trans):
        if t >= nlines:   # Lyman lines lie inside the Balmer continuum window (overlap)
            continue
    bal = m.trans[nlines + 1]
    lya = m.trans[0]
    assert bal.q0 <= lya.q0 and lya.q1 <= bal.q1


def test_line_grid_rule():
    x = OM.line_offsets(161, 3.0, 60.0)
    assert x[0] == pytest.approx(-60.0) and x[-1] == pytest.approx(60.0)
    assert x[80] == 0.0
    assert x[40] == pytest.approx(-3.0, rel=1e-12) and x[120] == pytest.approx(3.0, rel=1e-12)
    np.testing.assert_allclose(OM.line_offsets(41, 5.0, 5.0), np.linspace(-5, 5, 41), atol=1e-15)


def test_dense_overlap_workload_overlaps_more_transitions_than_a_packed_list():
    """The dense-overlap test atom has frequencies where all 12 lines are
    active at once (the kernels' packed per-frequency lists hold 8), so the
    GPU parity tests on it take the general transition lists."""
    wl = W.dense_overlap_workload()
    m = OM.build_model(wl.atom, wl.columns[0], wl.n_mu)
    active = np.zeros(m.nu.size, int)
    for t in m.trans:
        active[t.q0:t.q1 + 1] += 1
    assert active.max() == 12 > 8
