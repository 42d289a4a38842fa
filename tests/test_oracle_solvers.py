"""Pins of the oracle solvers: Krylov, Algorithm 2, RH92, dense Newton (no GPU)."""
import numpy as np
import pytest

import workloads as W
from oracle import krylov
from oracle import model as OM
from oracle.dense import dense_newton
from oracle.hybrid import hybrid
from oracle.jfnk import depth_clamp, jfnk, zero_radiation_guess
from oracle.residual import residual
from oracle.rh92 import rh92, rh92_update


def test_gmres_and_bicgstab_solve_linear_systems():
    rng = np.random.default_rng(0)
    A = np.eye(60) * 4 + rng.normal(size=(60, 60)) * 0.3
    b = rng.normal(size=60)
    x = np.linalg.solve(A, b)
    g = krylov.gmres(lambda v: A @ v, b, 1e-12, m_max=60)
    assert g.converged and np.allclose(g.x, x, rtol=1e-9, atol=1e-11)
    g = krylov.gmres(lambda v: A @ v, b, 1e-12, m_max=7, max_restarts=200)   # restarted
    assert g.converged and np.allclose(g.x, x, rtol=1e-8, atol=1e-10)
    bi = krylov.bicgstab(lambda v: A @ v, b, 1e-12)
    assert bi.converged and np.allclose(bi.x, x, rtol=1e-8, atol=1e-10)
    # GMRES residual never increases (Sect. 2.3)
    res = []
    for m in range(1, 30):
        r = krylov.gmres(lambda v: A @ v, b, 1e-30, m_max=m, max_restarts=0)
        res.append(np.linalg.norm(b - A @ r.x))
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(len(res) - 1))


@pytest.mark.slow
def test_sqrt_eps_law_under_depth_refinement():
    """Isothermal two-level atom: S(0) -> sqrt(eps) B as the depth grid is refined (config 1 physics)."""
    vals = []
    for nz in (101, 201, 401):
        atom = W.two_level_atom(n_nu=21)
        col = W.two_level_slab(atom, n_depth=nz, tau_max=1e6)
        m = OM.build_model(atom, col, 3)
        s = jfnk(m, m.nstar, rtol=1e-4, ftol=1e-9)
        assert s.converged
        r = residual(m, s.n, s.J)
        q0 = m.nq // 2
        vals.append((r.eta / r.chi)[q0, 0] / m.B[q0, 0] / 1e-2)
    assert vals[0] < vals[1] < vals[2] < 1.0
    # first-order convergence in the log-depth step: Richardson extrapolation hits sqrt(eps)
    extrap = 2 * vals[2] - vals[1]
    assert abs(extrap - 1.0) < 0.05


@pytest.mark.slow
def test_config1_solution_and_conservation_of_every_iterate():
    wl = W.config1()
    m = OM.build_model(wl.atom, wl.columns[0], wl.n_mu)
    s = jfnk(m, m.nstar, rtol=1e-2)
    assert s.converged and s.F_norm <= 1e-2 * s.F_norm0
    for h in s.history:
        np.testing.assert_allclose(h["n"].sum(axis=1), m.ntot, rtol=1e-12)
    r = residual(m, s.n, s.J)
    q0 = m.nq // 2
    ratio = (r.eta / r.chi)[q0, 0] / m.B[q0, 0]
    assert 0.006 < ratio < 0.01   # 101 log-spaced depths: ~0.73 sqrt(eps) (see refinement test)


def test_lte_limit_when_collisions_dominate():
    """Departures from Saha-Boltzmann vanish like 1/(collision scale) when collisions dominate."""
    wl = W.config2(nu_scale=0.1, n_depth=20)
    rng = np.random.default_rng(5)
    devs = []
    for scale in (1e12, 1e16, 1e20):
        m = OM.build_model(wl.atom, wl.columns[0], 3)
        m.Cmat *= scale
        n0 = W.perturbed_populations(m.nstar, rng, 0.3)
        n0 *= (m.ntot / n0.sum(axis=1))[:, None]
        s = jfnk(m, n0, rtol=1e-8, ftol=1e-10, J0=m.B)
        assert s.converged
        devs.append(np.max(np.abs(s.n / m.nstar - 1.0)))
    assert 3e2 < devs[0] / devs[1] < 3e4
    assert devs[2] < 1e-5


def test_jfnk_with_tight_krylov_tolerance_follows_dense_newton():
    """Fig. 4: JFNK approaches Newton-Raphson as r_tol -> 0."""
    wl = W.tiny_workload(n_depth=6, n_nu_line=9, n_nu_cont=4)
    m = OM.build_model(wl.atom, wl.columns[0], 2)
    dn = dense_newton(m, m.nstar, maxiter=4, ftol=0.0)
    jf = jfnk(m, m.nstar, rtol=1e-12, maxiter=4, ftol=0.0, fdrop=0.0)
    for it in range(1, 4):
        np.testing.assert_allclose(jf.history[it]["n"], dn.history[it]["n"], rtol=1e-7)


def test_rh92_fixed_point_is_the_jfnk_solution():
    """RH92's preconditioned rates are exact at n' = n: its fixed point is F(n) = 0 (Sect. 3.3)."""
    from oracle.rh92 import rh92_update
    wl = W.config2(nu_scale=0.1, n_depth=30)
    m = OM.build_model(wl.atom, wl.columns[0], 3)
    a = jfnk(m, m.nstar, rtol=1e-6, ftol=1e-11)
    assert a.converged
    res = residual(m, a.n, a.J, want_lambda=True)
    np.testing.assert_allclose(rh92_update(m, a.n, res), a.n, rtol=1e-10)


@pytest.mark.slow
def test_rh92_and_jfnk_converge_to_the_same_solution_and_spectrum():
    """Two-level slab (where RH92 converges): same populations and emergent spectrum (Figs. 9-10)."""
    wl = W.config1(n_depth=41, n_nu=21)
    m = OM.build_model(wl.atom, wl.columns[0], 3)
    a = jfnk(m, m.nstar, rtol=1e-8, ftol=1e-11)
    b = rh92(m, m.nstar, ftol=1e-11, maxiter=5000)
    assert a.converged and b.converged
    assert a.F_calls < b.iterations       # fewer formal solutions for JFNK
    np.testing.assert_allclose(a.n, b.n, rtol=1e-8)
    np.testing.assert_allclose(a.I_emergent, b.I_emergent, rtol=1e-8)


@pytest.mark.slow
def test_hybrid_start_converges_for_hydrogen():
    """Sect. 3.5 hybrid (RH92 then JFNK) on the H I-like atom, where JFNK from LTE fails."""
    wl = W.config3(nu_scale=0.1, n_depth=60)
    m = OM.build_model(wl.atom, wl.columns[0], 3)
    s = hybrid(m, m.nstar, rtol=1e-2)
    assert s.converged
    t = hybrid(m, m.nstar, rtol=1e-6, ftol=1e-10)
    assert t.converged
    np.testing.assert_allclose(s.n, t.n, rtol=1e-4)
    for h in t.history:
        np.testing.assert_allclose(h["n"].sum(axis=1), m.ntot, rtol=1e-11)


def _hot_top_column():
    """Coarse Ca II-like column whose LTE start sends the plain RH92 solve negative."""
    atom = W.ca_like_atom(0, 0.12)
    col = W.chromosphere(40, rng=np.random.default_rng(0), t_sigma=0.05, abundance=2.2e-6)
    return OM.build_model(atom, col, 3)


def test_limited_rh92_correction_stays_positive_and_conserves():
    """Sect. 2.2.2 per-depth limiting applied to the RH92 correction: alpha = 1
    exactly where no population falls below a tenth of its old value, every
    limited population keeps at least a tenth of it, and each depth still sums
    to its total particle density (both n and the plain update do)."""
    m = _hot_top_column()
    res = residual(m, m.nstar, OM.initial_J(m), want_lambda=True)
    raw = rh92_update(m, m.nstar, res)
    assert (raw <= 0).any()                      # the plain update leaves the domain
    np.testing.assert_allclose(raw.sum(axis=1), m.ntot, rtol=1e-10)
    lim, alpha = depth_clamp(m.nstar, raw - m.nstar)
    free = (raw >= 0.1 * m.nstar).all(axis=1)
    assert (alpha[free] == 1.0).all() and (alpha[~free] < 1.0).all()
    assert (lim >= 0.1 * m.nstar * (1 - 1e-12)).all()
    np.testing.assert_allclose(lim.sum(axis=1), m.ntot, rtol=1e-10)
    for k in range(1, 5):                        # every limited iterate stays positive
        w = rh92(m, m.nstar, ftol=0.0, maxiter=k)
        assert (w.n > 0).all()
        np.testing.assert_allclose(w.n.sum(axis=1), m.ntot, rtol=1e-10)


def test_limited_hybrid_start_reaches_the_jfnk_solution():
    """A capped, limited RH92 warm-up followed by Algorithm 2 lands on the same
    fixed point as Algorithm 2 from LTE (two different iterations, one solution)."""
    m = _hot_top_column()
    a = jfnk(m, m.nstar, rtol=1e-6, ftol=1e-10)
    b = hybrid(m, m.nstar, switch_tol=0.1, rh92_max=10, rtol=1e-6, ftol=1e-10)
    assert a.converged and b.converged and 0 < b.rh92_iters <= 10
    np.testing.assert_allclose(b.n, a.n, rtol=1e-8)


def test_zero_radiation_guess_solves_its_equations():
    wl = W.config2(nu_scale=0.1, n_depth=12)
    m = OM.build_model(wl.atom, wl.columns[0], 2)
    n = zero_radiation_guess(m)
    assert np.all(n > 0)
    np.testing.assert_allclose(n.sum(axis=1), m.ntot, rtol=1e-12)


def test_zero_radiation_guess_matches_the_two_level_closed_form():
    """With I = 0 a two-level atom balances collisional excitation against
    collisional de-excitation plus spontaneous emission:
    n_u / n_l = C_lu / (C_ul + A_ul), with A_ul from the Einstein relation
    A_ul = 8 pi^2 e^2 nu_0^2 / (m_e c^3) (g_l / g_u) f. The profile-weighted
    spontaneous rate differs from A_ul only by the (nu/nu_0)^2 variation across
    the Doppler core (< 1e-9)."""
    wl = W.config1(n_depth=15, n_nu=21)
    m = OM.build_model(wl.atom, wl.columns[0], 2)
    ln = wl.atom.lines[0]
    nu0 = m.trans[0].nu0
    A_ul = 8.0 * np.pi ** 2 * OM.QE ** 2 * nu0 ** 2 / (OM.ME * OM.C ** 3) \
        * (wl.atom.g[ln.i] / wl.atom.g[ln.j]) * ln.f
    C_lu, C_ul = m.Cmat[:, 0, 1], m.Cmat[:, 1, 0]
    n = zero_radiation_guess(m)
    np.testing.assert_allclose(n[:, 1] / n[:, 0], C_lu / (C_ul + A_ul), rtol=1e-8)
    np.testing.assert_allclose(n.sum(axis=1), m.ntot, rtol=1e-13)
    # eps = 1e-4: C_ul is about 1e-4 A_ul, so the guess lies far below LTE
    assert np.all(n[:, 1] / n[:, 0] < 1e-3 * m.nstar[:, 1] / m.nstar[:, 0])


def test_zero_radiation_guess_tends_to_lte_when_collisions_dominate():
    """Every row of the multi-level I = 0 rate equations (not only the one the
    conservation row leaves in a two-level atom): with collisions scaled up by
    1e12 the spontaneous rates are negligible and detailed balance of the
    collision rates gives back the Saha-Boltzmann populations, the departure
    shrinking like 1/scale (the ratio of spontaneous to collisional rates)."""
    wl = W.config2(nu_scale=0.1, n_depth=12)
    dev = []
    for scale in (1e12, 1e14, 1e16):
        m = OM.build_model(wl.atom, wl.columns[0], 2)
        m.Cmat *= scale
        dev.append(np.max(np.abs(zero_radiation_guess(m) / m.nstar - 1.0)))
    assert 50 < dev[0] / dev[1] < 200 and 50 < dev[1] / dev[2] < 200
    assert dev[2] < 1e-7


def test_rh92_operator_splitting_beats_lambda_iteration():
    """RH92 with its local operator Psi* against the same loop with Psi* = 0
    (plain Lambda iteration, no cross-coupling) on the eps = 1e-4 slab: after
    the same number of iterations RH92 is orders of magnitude closer to the
    solution, while Lambda iteration stalls with small population changes far
    from it (its classical false convergence). A dropped or mis-signed
    Psi* / cross-coupling term turns RH92 into the latter."""
    import oracle.rh92 as R
    wl = W.config1(n_depth=61, n_nu=21)
    m = OM.build_model(wl.atom, wl.columns[0], 3)
    ref = jfnk(m, m.nstar, rtol=1e-8, ftol=1e-12)
    assert ref.converged

    def iterate(k, lambda_only):
        n, Jd = m.nstar.copy(), OM.initial_J(m)
        changes = []
        for _ in range(k):
            res = residual(m, n, Jd, want_lambda=True)
            if lambda_only:
                res.lam_eta = np.zeros_like(res.lam_eta)
            n_new = R.rh92_update(m, n, res)
            changes.append(0.5 * np.max(np.abs((n_new - n) / (n_new + n))))
            n, Jd = n_new, res.J
        return np.max(np.abs(n / ref.n - 1.0)), changes

    e_rh, c_rh = iterate(160, False)
    e_la, c_la = iterate(160, True)
    assert e_rh < 0.05
    assert e_la > 1.0
    assert e_rh < 1e-2 * e_la
    # Lambda iteration's last changes are already small although it is a
    # factor of several away from the solution
    assert c_la[-1] < 2e-3
