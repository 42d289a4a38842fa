"""GPU parity: the CUDA library through its C ABI against the CPU oracle.

Tolerances (FP64 mode): tables 1e-12 relative (Voigt profiles 1e-9, the
accuracy of the Weideman expansion against the Faddeeva function); F and
J_F v compared per element against the gross rate scale of their depth
(F cancels towards zero at the solution, so a relative error per element is
meaningless there); converged populations 1e-5 relative (the stated FP64 bar,
both solved far past it). Mixed mode: converged populations 1e-3 relative.
"""
import numpy as np
import pytest

import workloads as W
from oracle import model as OM
from oracle.jfnk import jfnk
from oracle.precond import block_jacobi as ora_P
from oracle.residual import jvp_complex, residual as ora_residual
from oracle.rh92 import rh92_update as ora_rh92

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2406_17234_gb300.binding")


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B.Context(0)


def _pair(ctx, wl, n_mu=None, col=0):
    n_mu = n_mu or wl.n_mu
    atom = B.Atom(ctx, wl.atom)
    atm = B.Atmosphere(ctx, atom, wl.columns[col], n_mu=n_mu)
    m = OM.build_model(wl.atom, wl.columns[col], n_mu)
    return atom, atm, m


CASES = {
    "two-level": lambda: W.config1(),
    "ca-small": lambda: W.config2(nu_scale=0.2, n_depth=37),
    "h-small": lambda: W.config3(nu_scale=0.15, n_depth=41),
    "tiny": lambda: W.tiny_workload(n_depth=5, n_nu_line=7, n_nu_cont=3),
    # 12 transitions active at once: the kernels' general transition lists
    "dense-overlap": lambda: W.dense_overlap_workload(),
}


def _gross(m, n, R_up, R_dn):
    g = np.zeros_like(n)
    for t, tr in enumerate(m.trans):
        up = n[:, tr.lo] * (m.Cmat[:, tr.lo, tr.up] + R_up[t])
        dn = n[:, tr.up] * (m.Cmat[:, tr.up, tr.lo] + R_dn[t])
        g[:, tr.lo] += up + dn
        g[:, tr.up] += up + dn
    g += np.abs(n).sum(axis=1, keepdims=True) * 1e-30
    return g


@pytest.mark.parametrize("case", sorted(CASES))
def test_tables_match_oracle(ctx, case):
    wl = CASES[case]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    np.testing.assert_allclose(atom.frequencies(), m.nu, rtol=1e-14)
    assert (atm.n_depth, atm.n_nu, atm.n_levels, atm.n_transitions) == (m.nz, m.nq, m.nl, m.nt)
    np.testing.assert_allclose(atm.lte(), m.nstar, rtol=1e-12)
    np.testing.assert_allclose(atm.planck(), m.B, rtol=1e-12)
    C = atm.table(2, m.nz * m.nl * m.nl).reshape(m.nz, m.nl, m.nl)
    np.testing.assert_allclose(C, m.Cmat, rtol=1e-12, atol=0)
    nwin = sum(tr.q1 - tr.q0 + 1 for tr in m.trans)
    V = atm.table(3, nwin * m.nz).reshape(nwin, m.nz)
    G = atm.table(4, nwin * m.nz).reshape(nwin, m.nz)
    w = atm.table(5, nwin)
    base = 0
    for t, tr in enumerate(m.trans):
        nw = tr.q1 - tr.q0 + 1
        np.testing.assert_allclose(w[base:base + nw], m.omega[t, tr.q0:tr.q1 + 1], rtol=1e-13)
        np.testing.assert_allclose(V[base:base + nw], m.V[t, tr.q0:tr.q1 + 1], rtol=1e-9 if tr.kind == "bb" else 1e-13)
        np.testing.assert_allclose(G[base:base + nw], m.g[t, tr.q0:tr.q1 + 1], rtol=1e-12)
        base += nw
    np.testing.assert_allclose(atm.table(6, m.nq * m.nz).reshape(m.nq, m.nz), m.chi_c, rtol=1e-12)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("perturb", [0.0, 0.3])
def test_residual_matches_oracle(ctx, case, perturb):
    wl = CASES[case]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    rng = np.random.default_rng(11)
    n = m.nstar if perturb == 0.0 else W.perturbed_populations(m.nstar, rng, perturb)
    Jd = m.B * np.exp(rng.normal(0, 0.2, m.B.shape))
    F, J, Ie = B.residual(atm, n, Jd, want_J=True, want_emergent=True)
    r = ora_residual(m, n, Jd)
    gross = _gross(m, n, r.R_up, r.R_dn)
    assert np.all(np.abs(F - r.F) <= 1e-10 * gross + 1e-12 * np.abs(r.F))
    k = np.arange(m.nz)
    # conservation rows n_tot - sum n in FP64: a rounding error of about
    # N_l ulp(n_tot), which is all the row holds at LTE populations
    assert np.all(np.abs(F[k, r.istar] - r.F[k, r.istar]) <= 1e-13 * np.abs(r.F[k, r.istar]) + 1e-14 * m.ntot)
    np.testing.assert_allclose(J, r.J, rtol=1e-10, atol=1e-14 * np.max(np.abs(r.J)))
    np.testing.assert_allclose(Ie, r.I_emergent, rtol=1e-10, atol=1e-14 * np.max(np.abs(r.I_emergent)))


@pytest.mark.parametrize("case", sorted(CASES))
def test_jvp_matches_complex_step(ctx, case):
    wl = CASES[case]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    rng = np.random.default_rng(12)
    n = W.perturbed_populations(m.nstar, rng, 0.2)
    Jd = m.B
    for trial in range(2):
        v = rng.normal(size=n.shape) * n
        g = B.jvp(atm, n, v, Jd)
        ref = jvp_complex(m, n, Jd, v)
        scale = np.max(np.abs(ref), axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(g - ref) / scale) < 1e-9


@pytest.mark.parametrize("case", sorted(CASES))
def test_block_jacobi_matches_oracle(ctx, case):
    wl = CASES[case]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    rng = np.random.default_rng(13)
    n = W.perturbed_populations(m.nstar, rng, 0.2)
    P = B.block_jacobi(atm, n, m.B)
    r = ora_residual(m, n, m.B, want_lambda=True)
    ref = ora_P(m, n, r)
    scale = np.max(np.abs(ref), axis=(1, 2), keepdims=True)
    assert np.max(np.abs(P - ref) / scale) < 1e-10


@pytest.mark.parametrize("case", ["two-level", "ca-small", "h-small", "dense-overlap"])
def test_rh92_update_matches_oracle(ctx, case):
    wl = CASES[case]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    n_gpu, J_gpu = B.rh92_update(atm, m.nstar, m.B)
    r = ora_residual(m, m.nstar, m.B, want_lambda=True)
    ref = ora_rh92(m, m.nstar, r)
    np.testing.assert_allclose(n_gpu, ref, rtol=1e-8, atol=1e-12 * np.max(ref))


@pytest.mark.parametrize("case", ["ca-small", "dense-overlap"])
def test_mixed_rh92_update_and_blocks_match_oracle(ctx, case):
    """The mixed mode's RH92 update (float-pair rate sums, FP32 Psi* sums, FP64
    per-depth solves) and its preconditioner blocks (FP32 sums of Sect. 2.5.1)
    against the FP64 oracle, each depth relative to its largest entry; the
    dense-overlap atom takes the kernels' general transition lists. (On the
    H I-like column the direct update's Lyman net rates cancel below FP32
    resolution, about 4e-3 here: the solver then takes the correction form.)"""
    wl = CASES[case]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    rng = np.random.default_rng(14)
    n = W.perturbed_populations(m.nstar, rng, 0.1)
    n_gpu, _ = B.rh92_update(atm, n, m.B, precision=B.JFNK_MIXED)
    r = ora_residual(m, n, m.B, want_lambda=True)
    ref = ora_rh92(m, n, r)
    assert np.max(np.abs(n_gpu - ref) / np.max(np.abs(ref), axis=1, keepdims=True)) < 1e-3
    P = B.block_jacobi(atm, n, m.B, precision=B.JFNK_MIXED)
    Pref = ora_P(m, n, r)
    assert np.max(np.abs(P - Pref) / np.max(np.abs(Pref), axis=(1, 2), keepdims=True)) < 1e-3


def test_solve_two_level_matches_oracle_and_conserves(ctx):
    wl = W.config1()
    atom, atm, m = _pair(ctx, wl)
    n, J, st = B.solve(atm, B.default_options(rtol=1e-6, ftol=1e-10))
    ref = jfnk(m, m.nstar, rtol=1e-6, ftol=1e-10)
    assert st["status"] == 0
    np.testing.assert_allclose(n, ref.n, rtol=1e-5)
    np.testing.assert_allclose(n.sum(axis=1), m.ntot, rtol=1e-12)
    # the sqrt(eps) observable: S(0)/B at line centre
    r = ora_residual(m, n, J)
    q0 = m.nq // 2
    ratio = (r.eta / r.chi)[q0, 0] / m.B[q0, 0]
    r2 = ora_residual(m, ref.n, ref.J)
    assert ratio == pytest.approx((r2.eta / r2.chi)[q0, 0] / m.B[q0, 0], rel=1e-5)


def test_solve_paper_tolerances_two_level(ctx):
    wl = W.config1()
    atom, atm, m = _pair(ctx, wl)
    n, J, st = B.solve(atm, B.default_options())
    ref = jfnk(m, m.nstar)
    assert st["status"] == 0 and ref.converged
    assert st["F_norm"] <= 1e-2 * st["F_norm0"]
    np.testing.assert_allclose(n, ref.n, rtol=1e-3)


def test_solve_ca_small_matches_oracle(ctx):
    wl = CASES["ca-small"]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    n, J, st = B.solve(atm, B.default_options(rtol=1e-6, ftol=1e-10))
    ref = jfnk(m, m.nstar, rtol=1e-6, ftol=1e-10)
    assert st["status"] == 0 and ref.converged
    np.testing.assert_allclose(n, ref.n, rtol=1e-5)


def test_solve_mixed_precision_against_fp64_oracle(ctx):
    wl = CASES["ca-small"]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    # FP32 formal solutions put a floor near 1e-6 under the population change,
    # so the mixed mode is converged to 1e-5 here
    n, J, st = B.solve(atm, B.default_options(rtol=1e-4, ftol=1e-5, precision=B.JFNK_MIXED))
    ref = jfnk(m, m.nstar, rtol=1e-6, ftol=1e-10)
    assert st["status"] == 0
    np.testing.assert_allclose(n, ref.n, rtol=1e-3)
    # paper tolerances in the mixed mode meet the same bar
    n2, _, st2 = B.solve(atm, B.default_options(precision=B.JFNK_MIXED))
    assert st2["status"] == 0 and st2["F_norm"] <= 1e-2 * st2["F_norm0"]
    np.testing.assert_allclose(n2, ref.n, rtol=1e-3)


def test_hybrid_solve_hydrogen(ctx):
    wl = W.config3(nu_scale=0.1, n_depth=60)
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    from oracle.hybrid import hybrid
    n, J, st = B.solve(atm, B.default_options(rtol=1e-6, ftol=1e-10, rh92_warmup=200))
    ref = hybrid(m, m.nstar, rtol=1e-6, ftol=1e-10)
    assert st["status"] == 0 and st["rh92_iters"] > 0
    np.testing.assert_allclose(n, ref.n, rtol=1e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_limited_hybrid_solve(ctx, precision):
    """Capped hybrid start on a column whose plain RH92 step goes negative: the
    limited RH92 warm-up and the JFNK phase match the oracle's."""
    from oracle.hybrid import hybrid
    atom = W.ca_like_atom(0, 0.12)
    col = W.chromosphere(40, rng=np.random.default_rng(0), t_sigma=0.05, abundance=2.2e-6)
    a = B.Atom(ctx, atom)
    atm = B.Atmosphere(ctx, a, col, n_mu=3)
    m = OM.build_model(atom, col, 3)
    ref = hybrid(m, m.nstar, switch_tol=0.1, rh92_max=10, rtol=1e-6, ftol=1e-10)
    tol = dict(rtol=1e-6, ftol=1e-10) if precision == 0 else dict(rtol=1e-4, ftol=1e-5)
    n, J, st = B.solve(atm, B.default_options(precision=precision, rh92_warmup=10, rh92_switch=0.1, **tol))
    assert st["status"] == 0 and 0 < st["rh92_iters"] <= 10
    if precision == 0:
        assert st["rh92_iters"] == ref.rh92_iters
    assert (n > 0).all()
    np.testing.assert_allclose(n, ref.n, rtol=1e-5 if precision == 0 else 1e-3)


@pytest.mark.parametrize("n_mu", [3, 5])
@pytest.mark.parametrize("start", ["lte", "hybrid"])
def test_sweep_variants_are_bit_identical(ctx, n_mu, start):
    """The mixed-mode formal kernels (thread per frequency, with the opacity
    tangent from its own kernel or formed in the tangent sweep; warp per
    frequency pair) give bit-identical solves, so the autotuner's choice
    changes the speed only."""
    wl = W.config4(n_columns=3, nz_min=60, nz_max=90, nu_scale=0.1)
    atom = B.Atom(ctx, wl.atom)
    atms = [B.Atmosphere(ctx, atom, c, n_mu=n_mu) for c in wl.columns]
    init = dict(rh92_warmup=10, rh92_switch=0.1) if start == "hybrid" else {}
    outs = []
    for v in (B.JFNK_FORMAL_SWEEP_THREAD, B.JFNK_FORMAL_SWEEP_WARP, B.JFNK_FORMAL_SWEEP_THREAD_FUSED):
        opts = B.default_options(precision=B.JFNK_MIXED, formal_variant=v, **init)
        ns, st = B.batch_solve(ctx, atms, opts, raise_on_fail=False)
        assert all(s["formal_kernel"] == v for s in st)
        outs.append((ns, st))
    for other in outs[1:]:
        for na, nb, sa, sb in zip(outs[0][0], other[0], outs[0][1], other[1]):
            assert sa["status"] == sb["status"] and sa["F_calls"] == sb["F_calls"]
            np.testing.assert_array_equal(na, nb)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single(ctx, precision):
    """Each column's result in a batch is bit-identical to its result alone."""
    wl = W.config4(n_columns=5, nz_min=60, nz_max=90, nu_scale=0.1)
    atom = B.Atom(ctx, wl.atom)
    atms = [B.Atmosphere(ctx, atom, c, n_mu=3) for c in wl.columns]
    tol = dict(rtol=1e-6, ftol=1e-9) if precision == 0 else dict(rtol=1e-4, ftol=1e-5)
    opts = B.default_options(precision=precision, **tol)
    ns, stats = B.batch_solve(ctx, atms, opts, raise_on_fail=False)
    assert sum(s["status"] == 0 for s in stats) >= 3
    for a, nb, s in zip(atms, ns, stats):
        n1, _, s1 = B.solve(a, B.default_options(precision=precision, **tol), raise_on_fail=False)
        assert s["status"] == s1["status"]
        assert s["F_calls"] == s1["F_calls"]
        if s["status"] == 0:
            np.testing.assert_array_equal(nb, n1)


def test_edge_cases(ctx):
    # minimum depth count, a single angle, a single transition
    wl = W.config1(n_depth=2, n_nu=3)
    atom, atm, m = _pair(ctx, wl, n_mu=1)
    F, _, _ = B.residual(atm, m.nstar)
    r = ora_residual(m, m.nstar, m.B)
    gross = _gross(m, m.nstar, r.R_up, r.R_dn)
    assert np.all(np.abs(F - r.F) <= 1e-10 * gross)
    # empty batch is a no-op
    ns, st = B.batch_solve(ctx, [])
    assert ns == [] and st == []


def test_invalid_descriptors_are_rejected(ctx):
    wl = W.config1()
    bad = W.two_level_atom()
    bad.lines[0] = W.replace(bad.lines[0], n_nu=4)
    with pytest.raises(B.JFNKError) as e:
        B.Atom(ctx, bad)
    assert e.value.code == B.JFNK_E_INVALID
    atom = B.Atom(ctx, wl.atom)
    col = wl.columns[0]
    col2 = W.replace(col, T=-col.T)
    with pytest.raises(B.JFNKError):
        B.Atmosphere(ctx, atom, col2)


def test_batch_plan_is_reusable_and_matches_single(ctx):
    """A persistent batch plan gives the same populations on repeated runs and alone."""
    wl = W.config4(n_columns=3, nz_min=64, nz_max=80, nu_scale=0.1)
    atom = B.Atom(ctx, wl.atom)
    atms = [B.Atmosphere(ctx, atom, c, n_mu=3) for c in wl.columns]
    plan = B.BatchPlan(ctx, atms, precision=B.JFNK_MIXED)
    opts = B.default_options(precision=B.JFNK_MIXED)
    ns1, st1 = plan.run(opts, raise_on_fail=False)
    ns1 = [n.copy() for n in ns1]
    ns2, st2 = plan.run(opts, raise_on_fail=False)
    for a, b_, s1, s2, atm in zip(ns1, ns2, st1, st2, atms):
        assert s1["status"] == s2["status"]
        np.testing.assert_array_equal(a, b_)
        if s1["status"] == 0:
            n_single, _, s = B.solve(atm, B.default_options(precision=B.JFNK_MIXED))
            np.testing.assert_array_equal(a, n_single)


def test_zero_radiation_guess_matches_oracle(ctx):
    """JFNK_INIT_ZERO_RADIATION: a solve stopped after its first tick (a base
    evaluation, no update yet) returns the initial guess, which must be the
    oracle's rate-equation solution with I = 0 (Sect. 2.2.1)."""
    from oracle.jfnk import zero_radiation_guess
    wl = W.config2(nu_scale=0.2, n_depth=37)
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    n, _, st = B.solve(atm, B.default_options(init=B.JFNK_INIT_ZERO_RADIATION, max_ticks=1), raise_on_fail=False)
    assert st["status"] == B.JFNK_E_TIMEOUT and st["F_calls"] == 1
    # the line profiles agree to ~1e-9 (published Voigt approximation vs the
    # oracle's quadrature); the per-depth solve amplifies that by its condition
    np.testing.assert_allclose(n, zero_radiation_guess(m), rtol=1e-7)


def test_zero_radiation_start_reaches_the_oracle_solution(ctx):
    """From the zero-radiation guess Algorithm 2 converges to the oracle's
    fixed point on the two-level atom (on the Ca II-like atom that start lies
    too far out: the oracle's iteration from it fails as well)."""
    from oracle.jfnk import zero_radiation_guess
    wl = W.config1(n_depth=41, n_nu=21)
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    tight = dict(rtol=1e-6, ftol=1e-10)
    ref = jfnk(m, zero_radiation_guess(m), **tight)
    n_zr, _, s2 = B.solve(atm, B.default_options(init=B.JFNK_INIT_ZERO_RADIATION, **tight))
    _, _, s1 = B.solve(atm, B.default_options(**tight))
    assert ref.converged and s2["status"] == 0 and s1["F_calls"] != s2["F_calls"]
    np.testing.assert_allclose(n_zr, ref.n, rtol=1e-5)


def test_unpreconditioned_solve_reaches_the_oracle_solution(ctx):
    """precond = 0: GMRES on J x = -F without the block-Jacobi blocks (more
    Krylov iterations, the same fixed point)."""
    wl = W.config1(n_depth=41, n_nu=21)
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    ref = jfnk(m, m.nstar, rtol=1e-6, ftol=1e-10)
    n0, _, s0 = B.solve(atm, B.default_options(precond=0, rtol=1e-6, ftol=1e-10, max_restarts=200))
    n1, _, s1 = B.solve(atm, B.default_options(rtol=1e-6, ftol=1e-10))
    assert s0["status"] == 0 and s0["jvp_calls"] > s1["jvp_calls"]
    np.testing.assert_allclose(n0, ref.n, rtol=1e-5)


@pytest.mark.parametrize("scheme,ojvp,ochoice,per_jvp", [
    ("JFNK_JVP_FORWARD_EPS1", "forward", "eps1", 1),
    ("JFNK_JVP_FORWARD_EPS2", "forward", "eps2", 1),
    ("JFNK_JVP_CENTRAL", "central", "eps2", 2),
])
def test_difference_jvps_reach_the_oracle_solution(ctx, scheme, ojvp, ochoice, per_jvp):
    """Finite-difference JVPs (Sect. 2.4, Fig. 2) inside the on-device GMRES:
    the same fixed point as the oracle's iteration with the same scheme and
    step, and one (forward) or two (central) residual evaluations per JVP."""
    wl = W.config1(n_depth=41, n_nu=21)
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    tight = dict(rtol=1e-6, ftol=1e-10)
    ref = jfnk(m, m.nstar, jvp=ojvp, fd_choice=ochoice, **tight)
    n_fd, _, s = B.solve(atm, B.default_options(jvp=getattr(B, scheme), **tight))
    _, _, st = B.solve(atm, B.default_options(**tight))
    assert ref.converged and s["status"] == 0
    np.testing.assert_allclose(n_fd, ref.n, rtol=1e-5)
    # base evaluations are counted the same way in both runs
    assert (s["F_calls"] - per_jvp * s["jvp_calls"] - s["newton_iters"]
            == st["F_calls"] - st["jvp_calls"] - st["newton_iters"])
    assert abs(s["newton_iters"] - ref.newton_iters) <= 2


def test_difference_jvps_are_fp64_only(ctx):
    wl = W.config1(n_depth=21, n_nu=11)
    atom, atm, m = _pair(ctx, wl, n_mu=2)
    with pytest.raises(RuntimeError):
        B.solve(atm, B.default_options(jvp=B.JFNK_JVP_CENTRAL, precision=B.JFNK_MIXED))


@pytest.mark.parametrize("op,bar", [("add", 2.0**-44), ("sub", 2.0**-44), ("mul", 2.0**-44),
                                    ("div", 2.0**-42), ("acc", 2.0**-44)])
def test_float_pair_arithmetic(ctx, op, bar):
    """The float-pair (hi + lo) arithmetic of the mixed mode's base evaluations
    against IEEE FP64 on the same rounded inputs: about 48 significant bits
    (the difference scaled by the larger operand where it cancels)."""
    rng = np.random.default_rng(31)
    m = 100_000
    a = 10.0 ** rng.uniform(-12, 12, m) * (rng.choice([-1.0, 1.0], m) if op != "acc" else 1.0)
    b = 10.0 ** rng.uniform(-12, 12, m) * (rng.choice([-1.0, 1.0], m) if op != "acc" else 1.0)
    b[:100] = a[:100] * (1.0 + 1e-9)   # near cancellation
    out = B.check_arith(ctx, op, a, b)

    def pair(x):
        hi = x.astype(np.float32).astype(np.float64)
        return hi + (x - hi).astype(np.float32).astype(np.float64)

    x, y = pair(a), pair(b)
    exact = {"add": x + y, "sub": x - y, "mul": x * y, "div": x / y, "acc": x + y}[op]
    scale = np.abs(exact) if op in ("mul", "div") else np.maximum(np.abs(x), np.abs(y))
    assert np.max(np.abs(out - exact) / scale) <= bar


@pytest.mark.parametrize("case", ["two-level", "ca-small", "h-small", "dense-overlap"])
def test_mixed_residual_matches_oracle(ctx, case):
    """The mixed mode's residual (FP32 formal solution, float-pair S, J and
    rate sums, FP64 assembly) against the FP64 oracle: J to the FP32 sweep's
    accuracy and F within 1e-4 of the gross rates of each level (the FP32
    rounding of the intensity differences, about 1e-6 relative, with a wide
    margin); the conservation rows are FP64 and exact."""
    wl = CASES[case]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    rng = np.random.default_rng(11)
    n = W.perturbed_populations(m.nstar, rng, 0.3)
    Jd = m.B * np.exp(rng.normal(0, 0.2, m.B.shape))
    F, J, _ = B.residual(atm, n, Jd, precision=B.JFNK_MIXED, want_J=True)
    r = ora_residual(m, n, Jd)
    gross = _gross(m, n, r.R_up, r.R_dn)
    assert np.all(np.abs(F - r.F) <= 1e-4 * gross)
    k = np.arange(m.nz)
    np.testing.assert_allclose(F[k, r.istar], r.F[k, r.istar], rtol=1e-13)
    np.testing.assert_allclose(J, r.J, rtol=1e-4, atol=1e-9 * np.max(np.abs(r.J)))


@pytest.mark.parametrize("case", ["two-level", "ca-small", "dense-overlap"])
def test_mixed_jvp_matches_complex_step(ctx, case):
    """The mixed mode's FP32 tangent (Jacobian-vector product) against the
    oracle's complex step, relative to the largest entry of each depth."""
    wl = CASES[case]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    rng = np.random.default_rng(12)
    n = W.perturbed_populations(m.nstar, rng, 0.2)
    v = rng.normal(size=n.shape) * n
    g = B.jvp(atm, n, v, m.B, precision=B.JFNK_MIXED)
    ref = jvp_complex(m, n, m.B, v)
    scale = np.max(np.abs(ref), axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(g - ref) / scale) < 1e-3


@pytest.mark.parametrize("case", ["two-level", "ca-small"])
def test_bicgstab_solve_matches_oracle(ctx, case):
    """BiCGSTAB as the Krylov solver of Algorithm 2 (Sect. 2.3; two JVPs per
    iteration): the same fixed point as the oracle's BiCGSTAB iteration, FP64
    at 1e-5 and mixed at 1e-3, and two Jacobian-vector products per
    BiCGSTAB iteration (every JVP count even within a Newton step, except an
    early exit on the half-step residual)."""
    wl = W.config1(n_depth=41, n_nu=21) if case == "two-level" else CASES[case]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    tight = dict(rtol=1e-6, ftol=1e-10)
    ref = jfnk(m, m.nstar, krylov_solver="bicgstab", **tight)
    n, _, st = B.solve(atm, B.default_options(krylov=B.JFNK_KRYLOV_BICGSTAB, **tight))
    _, _, sg = B.solve(atm, B.default_options(**tight))
    assert ref.converged and st["status"] == 0
    np.testing.assert_allclose(n, ref.n, rtol=1e-5)
    assert st["jvp_calls"] != sg["jvp_calls"]
    assert abs(st["newton_iters"] - ref.newton_iters) <= 2
    nm, _, sm = B.solve(atm, B.default_options(krylov=B.JFNK_KRYLOV_BICGSTAB, precision=B.JFNK_MIXED,
                                               rtol=1e-4, ftol=1e-5))
    assert sm["status"] == 0
    np.testing.assert_allclose(nm, ref.n, rtol=1e-3)


def test_bicgstab_with_difference_jvps(ctx):
    """BiCGSTAB with the central-difference JVPs of Fig. 2 (two residual
    evaluations per product) reaches the oracle's fixed point."""
    wl = W.config1(n_depth=41, n_nu=21)
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    tight = dict(rtol=1e-6, ftol=1e-10)
    ref = jfnk(m, m.nstar, krylov_solver="bicgstab", jvp="central", fd_choice="eps2", **tight)
    n, _, st = B.solve(atm, B.default_options(krylov=B.JFNK_KRYLOV_BICGSTAB, jvp=B.JFNK_JVP_CENTRAL, **tight))
    assert ref.converged and st["status"] == 0
    np.testing.assert_allclose(n, ref.n, rtol=1e-5)
    assert st["F_calls"] - 2 * st["jvp_calls"] - st["newton_iters"] == 1


@pytest.mark.parametrize("case", ["two-level", "ca-82"])
def test_rh92_only_solve_matches_oracle_iterations(ctx, case):
    """The reference method on its own (JFNK_SOLVER_RH92): the device follows
    the oracle's RH92 iterates, limited per depth, to the same stopping point
    (same iteration count within one, populations within 1e-8), and its fixed
    point is Algorithm 2's. (On the coarse 37-depth Ca II-like column RH92
    from LTE stalls, in the oracle as on the device; the 82-depth one
    converges.)"""
    from oracle.rh92 import rh92
    wl = W.config1(n_depth=41, n_nu=21) if case == "two-level" else W.config2(nu_scale=0.2)
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    ref = rh92(m, m.nstar, ftol=1e-6, maxiter=3000)
    n, _, st = B.solve(atm, B.default_options(solver=B.JFNK_SOLVER_RH92, ftol=1e-6, maxiter=3000))
    assert ref.converged and st["status"] == 0
    assert abs(st["rh92_iters"] - ref.iterations) <= 1 and st["newton_iters"] == 0
    assert st["F_calls"] == st["rh92_iters"] and st["jvp_calls"] == 0
    np.testing.assert_allclose(n, ref.n, rtol=1e-8)
    assert st["F_norm"] < st["F_norm0"]
    nj, _, _ = B.solve(atm, B.default_options(rtol=1e-6, ftol=1e-10))
    np.testing.assert_allclose(n, nj, rtol=1e-3)


def test_krylov_and_solver_options_are_checked(ctx):
    wl = W.config1(n_depth=21, n_nu=11)
    atom, atm, m = _pair(ctx, wl, n_mu=2)
    for bad in (dict(krylov=7), dict(solver=5), dict(krylov=B.JFNK_KRYLOV_BICGSTAB, krylov_max=4)):
        with pytest.raises(B.JFNKError) as e:
            B.solve(atm, B.default_options(**bad))
        assert e.value.code == B.JFNK_E_INVALID


def _scattering_case():
    """Coarse Ca II-like column with the electron density raised 300-fold, so
    that Thomson scattering matters to the preconditioner variants."""
    wl = W.config2(nu_scale=0.15, n_depth=30)
    col = wl.columns[0]
    return W.Workload(name="scattering", atom=wl.atom, columns=[W.replace(col, ne=col.ne * 300.0)], n_mu=3)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_preconditioner_variants_match_oracle(ctx, variant):
    """The three solutions of Sect. 2.5.2 on the device against the oracle's
    blocks (variant 2 with a given lagged estimate, whose renewal is compared
    too); variants 2 and 3 differ from the first on this column."""
    from oracle.precond import dJ_dn
    wl = _scattering_case()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    rng = np.random.default_rng(17)
    n = W.perturbed_populations(m.nstar, rng, 0.2)
    r = ora_residual(m, n, m.B, want_lambda=True)
    D0 = dJ_dn(m, n, r, 1) * rng.uniform(0.5, 1.5, (m.nl, m.nq, m.nz)) if variant == 2 else None
    ref = ora_P(m, n, r, variant=variant, D_prev=D0)
    P, D = B.block_jacobi_variant(atm, n, variant, m.B,
                                  dJdn_prev=None if D0 is None else D0.transpose(1, 2, 0))
    scale = np.max(np.abs(ref), axis=(1, 2), keepdims=True)
    assert np.max(np.abs(P - ref) / scale) < 1e-10
    if variant > 1:
        P1 = ora_P(m, n, r, variant=1)
        assert np.max(np.abs(ref - P1) / scale) > 1e-6
    if variant == 2:
        Dref = dJ_dn(m, n, r, 2, D0).transpose(1, 2, 0)
        sc = np.max(np.abs(Dref)) + 1e-300
        assert np.max(np.abs(D - Dref)) / sc < 1e-10


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_preconditioner_variant_solves_reach_the_oracle_solution(ctx, variant, precision):
    """Algorithm 2 preconditioned by the second or third solution reaches the
    oracle's fixed point under the same preconditioner (on the strongly
    scattering column JFNK from LTE does not converge, in the oracle either,
    so the solves use the regular one)."""
    wl = CASES["ca-small"]()
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    tight = dict(rtol=1e-6, ftol=1e-10)
    ref = jfnk(m, m.nstar, precond_variant=variant, **tight)
    tol = tight if precision == 0 else dict(rtol=1e-4, ftol=1e-5)
    n, _, st = B.solve(atm, B.default_options(precond=variant, precision=precision, **tol))
    assert ref.converged and st["status"] == 0
    np.testing.assert_allclose(n, ref.n, rtol=1e-5 if precision == 0 else 1e-3)


@pytest.mark.parametrize("precision", [0, 1])
def test_line_search_solve_matches_oracle(ctx, precision):
    """Backtracking on ||F||_inf (Sect. 2.2.2): on the three-level case the
    full Newton step raises ||F|| once, the line search halves it (extra F
    evaluations, as in the oracle) and both land on the oracle's solution."""
    wl = W.tiny_workload(n_depth=6, n_nu_line=7, n_nu_cont=3)
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    tight = dict(rtol=1e-6, ftol=1e-10)
    ref = jfnk(m, m.nstar, line_search=True, **tight)
    ref0 = jfnk(m, m.nstar, **tight)
    assert ref.F_calls > ref0.F_calls
    tol = tight if precision == 0 else dict(rtol=1e-4, ftol=1e-5)
    n, _, st = B.solve(atm, B.default_options(line_search=12, precision=precision, **tol))
    _, _, s0 = B.solve(atm, B.default_options(precision=precision, **tol))
    assert st["status"] == 0 and ref.converged
    assert st["F_calls"] > s0["F_calls"]
    np.testing.assert_allclose(n, ref.n, rtol=1e-5 if precision == 0 else 1e-3)
    if precision == 0:
        # trial evaluations beyond one per Newton step: backtracking happened on
        # both sides (the counts may differ by a borderline decision, since
        # the iterates are not identical: exact tangent vs complex step)
        trials_gpu = st["F_calls"] - st["jvp_calls"] - st["newton_iters"]
        trials_ref = ref.F_calls - ref.jvp_calls - ref.newton_iters
        assert trials_gpu > 1 and trials_ref > 1 and abs(trials_gpu - trials_ref) <= 2


@pytest.mark.slow
def test_rh92_only_mixed_reaches_the_oracle_fixed_point(ctx):
    """RH92 alone in the mixed mode on an H I-like column (optically thick
    Lyman lines, whose net rates cancel far below FP32 resolution): the
    correction form of the update, driven by the float-pair residual,
    converges to the oracle's RH92 fixed point within the mixed bar."""
    from oracle.rh92 import rh92
    wl = W.config3(nu_scale=0.1)
    atom, atm, m = _pair(ctx, wl, n_mu=3)
    ref = rh92(m, m.nstar, ftol=1e-6, maxiter=2000)
    n, _, st = B.solve(atm, B.default_options(solver=B.JFNK_SOLVER_RH92, precision=B.JFNK_MIXED,
                                              ftol=1e-5, maxiter=2000))
    assert ref.converged and st["status"] == 0
    np.testing.assert_allclose(n, ref.n, rtol=1e-3)


def test_profiled_batch_reports_its_stages_and_tuned_shapes(ctx):
    """A profiled mixed batch solve: each tick's stages are timed on one stream
    (the sweeps' own durations are two of them), the results are those of the
    unprofiled solve, and the autotuned opacity-tangent depth tile is one of
    its candidates."""
    wl = W.config4(n_columns=6, nz_min=40, nz_max=70, nu_scale=0.1)
    atom = B.Atom(ctx, wl.atom)
    atms = [B.Atmosphere(ctx, atom, c, n_mu=3) for c in wl.columns]
    start = dict(rh92_warmup=5, rh92_switch=0.1)
    plan = B.BatchPlan(ctx, atms, precision=B.JFNK_MIXED)
    n0, s0 = plan.run(B.default_options(precision=B.JFNK_MIXED, **start), raise_on_fail=False)
    n0 = [x.copy() for x in n0]
    n1, s1 = plan.run(B.default_options(precision=B.JFNK_MIXED, profile=1, **start), raise_on_fail=False)
    st = s1[0]
    stage = st["stage_ms"]
    assert len(stage) == 6 and all(x >= 0.0 for x in stage) and sum(stage) > 0.0
    assert abs(stage[1] - st["formal_tan_ms"]) <= 1e-9 * max(1.0, st["formal_tan_ms"])
    assert abs(stage[2] - st["formal_ms"]) <= 1e-9 * max(1.0, st["formal_ms"])
    assert st["opacity_depths"] in (4, 8, 16, 32)
    for a, b_, sa, sb in zip(n0, n1, s0, s1):
        assert sa["status"] == sb["status"] and sa["F_calls"] == sb["F_calls"]
        np.testing.assert_array_equal(a, b_)
    plan.close()
