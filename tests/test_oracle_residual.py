"""Pins of the oracle residual, JVPs and block-Jacobi preconditioner (no GPU)."""
import numpy as np
import pytest

import workloads as W
from oracle import model as OM
from oracle.dense import dense_jacobian
from oracle.precond import block_jacobi
from oracle.residual import assemble, jvp_complex, jvp_fd, opacity_emissivity, rates_from_J, residual


@pytest.fixture(scope="module")
def small_ca():
    wl = W.config2(nu_scale=0.1, n_depth=10)
    return OM.build_model(wl.atom, wl.columns[0], 2)


@pytest.fixture(scope="module")
def tiny():
    wl = W.tiny_workload(n_depth=5, n_nu_line=7, n_nu_cont=3)
    return OM.build_model(wl.atom, wl.columns[0], 2)


def test_detailed_balance_with_planck_radiation(small_ca):
    """At n = n* and J = B_nu(T) every radiative net rate vanishes (Kirchhoff + Einstein + Milne).

    Exact for bound-free (g_ij carries exp(-h nu/kT) per frequency); for a line
    the Boltzmann factor is taken at the line centre, so the balance holds up to
    the second order in (nu - nu_0)/nu_0 across the symmetric profile (~1e-9).
    """
    m = small_ca
    R_up, R_dn = rates_from_J(m, m.B)
    for t, tr in enumerate(m.trans):
        up = m.nstar[:, tr.lo] * R_up[t]
        dn = m.nstar[:, tr.up] * R_dn[t]
        np.testing.assert_allclose(up, dn, rtol=1e-12 if tr.kind == "bf" else 1e-8)
    F = assemble(m, m.nstar, R_up, R_dn, np.argmax(m.nstar, axis=1))
    gross = np.zeros_like(m.nstar)
    for t, tr in enumerate(m.trans):
        gross[:, tr.lo] += m.nstar[:, tr.lo] * R_up[t]
        gross[:, tr.up] += m.nstar[:, tr.lo] * R_up[t]
    assert np.all(np.abs(F) <= 1e-8 * gross + 1e-300)


def test_conservation_rows(small_ca):
    m = small_ca
    rng = np.random.default_rng(1)
    n = W.perturbed_populations(m.nstar, rng)
    r = residual(m, n, OM.initial_J(m))
    np.testing.assert_array_equal(r.istar, np.argmax(n, axis=1))
    np.testing.assert_allclose(r.F[np.arange(m.nz), r.istar], m.ntot - n.sum(axis=1), rtol=1e-14)
    # the other rows sum to minus the conservation row's net-rate content: sum_i F_i = 0 before replacement
    R_up, R_dn = r.R_up, r.R_dn
    Fraw = np.zeros_like(n)
    for t, tr in enumerate(m.trans):
        kap = n[:, tr.lo] * (m.Cmat[:, tr.lo, tr.up] + R_up[t]) - n[:, tr.up] * (m.Cmat[:, tr.up, tr.lo] + R_dn[t])
        Fraw[:, tr.lo] += kap
        Fraw[:, tr.up] -= kap
    assert np.max(np.abs(Fraw.sum(axis=1))) < 1e-12 * np.max(np.abs(Fraw))


def test_complex_step_jvp_is_linear(small_ca):
    m = small_ca
    rng = np.random.default_rng(2)
    n = W.perturbed_populations(m.nstar, rng, 0.2)
    Jd = OM.initial_J(m)
    v = rng.normal(size=n.shape) * n
    w = rng.normal(size=n.shape) * n
    Jv = jvp_complex(m, n, Jd, v)
    Jw = jvp_complex(m, n, Jd, w)
    Jc = jvp_complex(m, n, Jd, 2.5 * v - w)
    np.testing.assert_allclose(Jc, 2.5 * Jv - Jw, rtol=1e-10, atol=1e-12 * np.max(np.abs(Jc)))


def test_complex_step_matches_brute_force_differences(tiny):
    """Complex-step JVP vs central differences with a scanned step (well-scaled tiny case)."""
    m = tiny
    rng = np.random.default_rng(3)
    n = W.perturbed_populations(m.nstar, rng, 0.1)
    Jd = OM.initial_J(m)
    istar = np.argmax(n, axis=1)
    for trial in range(3):
        v = rng.normal(size=n.shape) * n
        ref = jvp_complex(m, n, Jd, v, istar=istar)
        best = np.inf
        for h in [1e-3, 3e-4, 1e-4, 3e-5, 1e-5, 3e-6]:
            cd = jvp_fd(m, n, Jd, v, scheme="central", istar=istar, eps=h)
            best = min(best, np.max(np.abs(cd - ref)) / np.max(np.abs(ref)))
        assert best < 1e-7


def test_block_jacobi_equals_dense_jacobian_diagonal_blocks(tiny):
    """With J^dagger frozen, P^k is exactly the k-th diagonal block of J_F (Sect. 2.5)."""
    m = tiny
    rng = np.random.default_rng(4)
    n = W.perturbed_populations(m.nstar, rng, 0.3)
    Jd = OM.initial_J(m) * 0.7
    res = residual(m, n, Jd, want_lambda=True)
    P = block_jacobi(m, n, res)
    Jm = dense_jacobian(m, n, Jd, istar=res.istar)
    nl = m.nl
    for k in range(m.nz):
        blk = Jm[k * nl:(k + 1) * nl, k * nl:(k + 1) * nl]
        np.testing.assert_allclose(P[k], blk, rtol=1e-9, atol=1e-11 * np.max(np.abs(blk)))
    # conservation rows: -1 on the own depth, 0 elsewhere
    for k in range(m.nz):
        row = Jm[k * nl + res.istar[k]]
        expect = np.zeros(m.nz * nl)
        expect[k * nl:(k + 1) * nl] = -1.0
        np.testing.assert_array_equal(row, expect)


def test_dense_jacobian_structure_is_nonlocal(tiny):
    """Off-diagonal blocks are nonzero (Fig. 1): the radiation couples all depths."""
    m = tiny
    n = m.nstar
    Jm = dense_jacobian(m, n, OM.initial_J(m))
    nl = m.nl
    off = Jm[0:nl, (m.nz - 1) * nl:m.nz * nl]
    assert np.max(np.abs(off)) > 0.0


def test_finite_differences_are_less_accurate_than_complex_step(small_ca):
    """Fig. 2: forward differences with eps_1 / eps_2 lose accuracy, the complex step does not."""
    m = small_ca
    n = m.nstar
    Jd = OM.initial_J(m)
    res = residual(m, n, Jd, want_lambda=True)
    P = block_jacobi(m, n, res)
    nl = m.nl
    errs = {}
    for scheme, choice in [("complex", None), ("forward", "eps1"), ("forward", "eps2")]:
        worst = 0.0
        for c in range(nl):
            k = m.nz // 2
            v = np.zeros_like(n)
            v[k, c] = 1.0
            if scheme == "complex":
                col = jvp_complex(m, n, Jd, v, istar=res.istar)
            else:
                col = jvp_fd(m, n, Jd, v, scheme=scheme, choice=choice, F0=res.F, istar=res.istar)
            ref = P[k][:, c]
            worst = max(worst, np.max(np.abs(col[k] - ref)) / np.max(np.abs(P[k])))
        errs[(scheme, choice)] = worst
    assert errs[("complex", None)] < 1e-10
    assert errs[("forward", "eps1")] > 1e3 * errs[("complex", None)]
    assert errs[("forward", "eps2")] > 1e3 * errs[("complex", None)]


def _isothermal_column(nz=12, T=6000.0, thomson=True, kappa=1.0, ntot_scale=1.0):
    """Isothermal column with the synthetic chromosphere's background law
    (power-law UV rise, Thomson scattering) at constant temperature."""
    base = W.chromosphere(nz, abundance=2.2e-6)
    ones = np.ones(nz)
    return W.replace(base, T=T * ones, ntot=ntot_scale * base.ntot, kappa=kappa, thomson=thomson)


def _line_centre_indices(m):
    out = []
    for tr in m.trans:
        if tr.kind == "bb":
            q = int(np.argmin(np.abs(m.nu - tr.nu0)))
            assert abs(m.nu[q] / tr.nu0 - 1.0) < 1e-15      # odd grids hold nu_0 itself
            out.append(q)
    return out


def test_source_function_is_planck_in_thermodynamic_equilibrium():
    """Kirchhoff (Eqs. chi, eta with the background of Sect. 2.1.1): on an
    isothermal column at LTE populations with J^dagger = B_nu(T), the source
    function equals B_nu at every frequency whose active transitions are
    continua or background only, and at every line centre (the line's g_ij is
    the Boltzmann ratio of its centre frequency). A dropped chi_sca in chi, a
    wrong eta_c or a mis-signed stimulated-emission term breaks this."""
    atom = W.ca_like_atom(0, 0.1)
    col = _isothermal_column()
    m = OM.build_model(atom, col, 2)
    chi, eta = opacity_emissivity(m, m.nstar, m.B)
    S = eta / chi
    bb = np.array([tr.kind == "bb" for tr in m.trans])
    no_line = ~m.active[bb].any(axis=0)
    assert no_line.sum() > 10
    np.testing.assert_allclose(S[no_line], m.B[no_line], rtol=1e-12)
    qc = _line_centre_indices(m)
    np.testing.assert_allclose(S[qc], m.B[qc], rtol=1e-12)
    # and off line centre the lines pull S away from B_nu (the test would pass
    # trivially if the line terms were missing)
    in_line = m.active[bb].any(axis=0)
    assert np.max(np.abs(S[in_line] / m.B[in_line] - 1.0)) > 1e-4


def test_pure_scattering_limit_gives_source_function_equal_to_J_dagger():
    """Pure electron scattering (no active atom, no continuum absorption):
    S = J^dagger at every (nu, k) for any lagged mean intensity, through the
    full residual evaluation (the scattering emissivity uses J^dagger, and
    chi_sca enters both chi and eta)."""
    atom = W.ca_like_atom(0, 0.1)
    col = _isothermal_column(kappa=0.0, thomson=True, ntot_scale=0.0)
    m = OM.build_model(atom, col, 2)
    rng = np.random.default_rng(9)
    Jd = m.B * np.exp(rng.normal(0.0, 1.0, m.B.shape))
    n0 = np.zeros((m.nz, m.nl))
    chi, eta = opacity_emissivity(m, n0, Jd)
    np.testing.assert_allclose(eta / chi, Jd, rtol=1e-14)
    r = residual(m, n0, Jd)
    np.testing.assert_allclose(r.eta / r.chi, Jd, rtol=1e-14)


def test_pure_absorption_limit_ignores_J_dagger():
    """Without Thomson scattering the source function does not depend on
    J^dagger, and continuum absorption alone (no active atom) gives S = B_nu."""
    atom = W.ca_like_atom(0, 0.1)
    m = OM.build_model(atom, _isothermal_column(thomson=False), 2)
    rng = np.random.default_rng(10)
    n = W.perturbed_populations(m.nstar, rng, 0.3)
    c1, e1 = opacity_emissivity(m, n, m.B)
    c2, e2 = opacity_emissivity(m, n, m.B * rng.uniform(0.1, 10.0, m.B.shape))
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(e1, e2)
    m0 = OM.build_model(atom, _isothermal_column(thomson=False, ntot_scale=0.0), 2)
    chi, eta = opacity_emissivity(m0, np.zeros((m0.nz, m0.nl)), m0.B * 3.0)
    np.testing.assert_allclose(eta / chi, m0.B, rtol=1e-14)


def test_preconditioner_variants_reduce_to_the_first_without_scattering(tiny):
    """Sect. 2.5.2: the second and third solutions differ from the first only
    through chi_sca; without background scattering all three give the same
    blocks (which equal the dense Jacobian's diagonal blocks, pinned above)."""
    from dataclasses import replace
    m = replace(tiny, chi_sca=np.zeros_like(tiny.chi_sca))
    rng = np.random.default_rng(5)
    n = W.perturbed_populations(m.nstar, rng, 0.3)
    res = residual(m, n, OM.initial_J(m), want_lambda=True)
    P1 = block_jacobi(m, n, res, variant=1)
    D = rng.normal(size=(m.nl, m.nq, m.nz))
    np.testing.assert_array_equal(block_jacobi(m, n, res, variant=2, D_prev=D), P1)
    np.testing.assert_array_equal(block_jacobi(m, n, res, variant=3), P1)


def test_lagged_scattering_estimate_converges_to_the_local_solution(tiny):
    """The lagged d J/d n of the second solution, renewed with fixed local
    operators, is a contraction (factor chi_sca Leta < 1) whose fixed point is
    the third solution's local self-consistent estimate."""
    from oracle.precond import dJ_dn
    from dataclasses import replace
    m = replace(tiny, chi_sca=tiny.chi_sca * 3e3)
    n = m.nstar
    res = residual(m, n, OM.initial_J(m), want_lambda=True)
    D3 = dJ_dn(m, n, res, 3)
    D = None
    for _ in range(80):
        D = dJ_dn(m, n, res, 2, D)
    np.testing.assert_allclose(D, D3, rtol=1e-12, atol=1e-14 * np.max(np.abs(D3)))


def test_local_scattering_solution_approaches_the_consistent_jacobian(tiny):
    """With J^dagger made self-consistent (J = Lambda[S(n, J)], iterated to
    convergence inside the residual), the diagonal blocks of the resulting
    dense complex-step Jacobian carry the scattering feedback that the first
    solution drops: on a strongly scattering column the third solution's
    blocks (local feedback kept) are several times closer to them."""
    from dataclasses import replace
    m = replace(tiny, chi_sca=tiny.chi_sca * 3e3)
    n = W.perturbed_populations(m.nstar, np.random.default_rng(4), 0.2)

    def consistent_J(nc, iters=150):
        J = OM.initial_J(m).astype(complex)
        for _ in range(iters):
            J = residual(m, nc, J).J
        return J

    Jc = consistent_J(n.astype(complex))
    np.testing.assert_allclose(residual(m, n, Jc).J, Jc, rtol=1e-12)   # converged
    res = residual(m, n, Jc.real, want_lambda=True)
    N, nl = n.size, m.nl
    Jm = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        nc = n + 1j * 1e-200 * e.reshape(n.shape)
        Jm[:, c] = (residual(m, nc, consistent_J(nc), istar=res.istar).F.imag / 1e-200).ravel()

    def dev(P):
        return max(np.max(np.abs(P[k] - Jm[k * nl:(k + 1) * nl, k * nl:(k + 1) * nl]))
                   / np.max(np.abs(Jm[k * nl:(k + 1) * nl, k * nl:(k + 1) * nl])) for k in range(m.nz))

    d1, d3 = dev(block_jacobi(m, n, res, variant=1)), dev(block_jacobi(m, n, res, variant=3))
    assert d1 > 0.02
    assert d3 < 0.25 * d1
