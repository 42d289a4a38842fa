"""GPU parity of moving columns (line-of-sight velocity, Sect. 3.4) against
the oracle: per-direction profile tables, the residual with per-ray opacity,
formal solution and rate integrals, its exact tangent, the block-Jacobi
blocks, and converged solves (FP64, 1e-5 relative)."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import model as OM
from oracle.jfnk import jfnk
from oracle.precond import block_jacobi as ora_P
from oracle.residual import jvp_complex, residual as ora_residual

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2406_17234_gb300.binding")


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B.Context(0)


def _cases():
    tiny = W.tiny_workload(n_depth=6, n_nu_line=9, n_nu_cont=3)
    return {
        "tiny": (tiny.atom, replace(tiny.columns[0], vlos=np.linspace(3e5, -1e5, 6)), 2),
        "ca-gradient": (W.ca_like_atom(0, 0.15), W.velocity_chromosphere(40), 3),
        "two-level": (W.two_level_atom(n_nu=41),
                      replace(W.two_level_slab(W.two_level_atom(n_nu=41), n_depth=41, tau_max=1e3),
                              vlos=np.linspace(2e5, 0.0, 41)), 3),
    }


def _pair(ctx, atom, col, n_mu):
    a = B.Atom(ctx, atom)
    return a, B.Atmosphere(ctx, a, col, n_mu=n_mu), OM.build_model(atom, col, n_mu)


def _gross(m, n, R_up, R_dn):
    g = np.zeros_like(n)
    for t, tr in enumerate(m.trans):
        up = n[:, tr.lo] * (m.Cmat[:, tr.lo, tr.up] + R_up[t])
        dn = n[:, tr.up] * (m.Cmat[:, tr.up, tr.lo] + R_dn[t])
        g[:, tr.lo] += up + dn
        g[:, tr.up] += up + dn
    return g


@pytest.mark.parametrize("case", ["tiny", "ca-gradient", "two-level"])
def test_moving_tables_residual_jvp_and_blocks_match_oracle(ctx, case):
    atom, col, nmu = _cases()[case]
    a, atm, m = _pair(ctx, atom, col, nmu)
    assert m.Vdir is not None
    nwin = sum(tr.q1 - tr.q0 + 1 for tr in m.trans)
    Vd = atm.table(8, 2 * nmu * nwin * m.nz).reshape(2 * nmu, nwin, m.nz)
    base = 0
    for t, tr in enumerate(m.trans):
        nw = tr.q1 - tr.q0 + 1
        ref = m.Vdir[t, :, tr.q0:tr.q1 + 1]
        np.testing.assert_allclose(Vd[:, base:base + nw], ref, rtol=1e-9, atol=1e-12 * np.max(ref))
        base += nw
    rng = np.random.default_rng(31)
    n = W.perturbed_populations(m.nstar, rng, 0.3)
    Jd = m.B * np.exp(rng.normal(0, 0.2, m.B.shape))
    F, J, Ie = B.residual(atm, n, Jd, want_J=True, want_emergent=True)
    r = ora_residual(m, n, Jd, want_lambda=True)
    gross = _gross(m, n, r.R_up, r.R_dn)
    assert np.all(np.abs(F - r.F) <= 1e-10 * gross + 1e-12 * np.abs(r.F))
    np.testing.assert_allclose(J, r.J, rtol=1e-10, atol=1e-14 * np.max(r.J))
    np.testing.assert_allclose(Ie, r.I_emergent, rtol=1e-10, atol=1e-14 * np.max(r.I_emergent))
    v = rng.normal(size=n.shape) * n
    g = B.jvp(atm, n, v, Jd)
    ref = jvp_complex(m, n, Jd, v)
    assert np.max(np.abs(g - ref) / (np.max(np.abs(ref), axis=1, keepdims=True) + 1e-300)) < 1e-9
    P = B.block_jacobi(atm, n, Jd)
    Pr = ora_P(m, n, r)
    assert np.max(np.abs(P - Pr) / np.max(np.abs(Pr), axis=(1, 2), keepdims=True)) < 1e-10


@pytest.mark.parametrize("case", ["ca-gradient", "two-level"])
@pytest.mark.parametrize("krylov", ["JFNK_KRYLOV_GMRES", "JFNK_KRYLOV_BICGSTAB"])
def test_moving_solve_matches_oracle(ctx, case, krylov):
    atom, col, nmu = _cases()[case]
    a, atm, m = _pair(ctx, atom, col, nmu)
    tight = dict(rtol=1e-6, ftol=1e-10)
    ref = jfnk(m, m.nstar, krylov_solver="gmres" if krylov.endswith("GMRES") else "bicgstab", **tight)
    n, _, st = B.solve(atm, B.default_options(krylov=getattr(B, krylov), **tight))
    assert ref.converged and st["status"] == 0
    np.testing.assert_allclose(n, ref.n, rtol=1e-5)
    np.testing.assert_allclose(n.sum(axis=1), col.ntot, rtol=1e-12)


def test_moving_columns_reject_what_they_do_not_support(ctx):
    atom, col, nmu = _cases()["tiny"]
    a, atm, m = _pair(ctx, atom, col, nmu)
    for bad in (dict(precision=B.JFNK_MIXED), dict(rh92_warmup=5), dict(solver=B.JFNK_SOLVER_RH92),
                dict(precond=3)):
        with pytest.raises(B.JFNKError) as e:
            B.solve(atm, B.default_options(**bad))
        assert e.value.code == B.JFNK_E_INVALID
    with pytest.raises(B.JFNKError):
        B.rh92_update(atm, m.nstar)
    with pytest.raises(B.JFNKError):
        B.residual(atm, m.nstar, precision=B.JFNK_MIXED)
