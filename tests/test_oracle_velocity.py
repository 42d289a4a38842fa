"""Pins of the oracle's moving-column residual (line-of-sight velocity, Sect.
3.4): each direction of propagation sees its own Doppler-shifted profile, so
opacity, source function, intensity and the rate integrals are per ray."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import model as OM
from oracle.dense import dense_jacobian
from oracle.jfnk import jfnk
from oracle.precond import block_jacobi
from oracle.residual import jvp_complex, jvp_fd, residual


def _tiny_moving(v_top=3e5):
    wl = W.tiny_workload(n_depth=6, n_nu_line=9, n_nu_cont=3)
    col = replace(wl.columns[0], vlos=np.linspace(v_top, 0.0, 6))
    return OM.build_model(wl.atom, col, 2)


def _as_moving(m):
    """The static model run through the moving-column path: every direction
    carries the static profile."""
    nd = 2 * m.nmu
    return replace(m, Vdir=np.repeat(m.V[:, None], nd, axis=1), mu_dir=np.concatenate([m.mu, -m.mu]),
                   vlos=np.zeros(m.nz))


def test_moving_path_reduces_to_the_static_residual():
    wl = W.config2(nu_scale=0.1, n_depth=15)
    m = OM.build_model(wl.atom, wl.columns[0], 3)
    mv = _as_moving(m)
    rng = np.random.default_rng(3)
    n = W.perturbed_populations(m.nstar, rng, 0.3)
    Jd = m.B * np.exp(rng.normal(0, 0.2, m.B.shape))
    a, b = residual(m, n, Jd, want_lambda=True), residual(mv, n, Jd, want_lambda=True)
    scale = np.max(np.abs(a.F), axis=1, keepdims=True)
    assert np.max(np.abs(a.F - b.F) / scale) < 1e-12
    np.testing.assert_allclose(b.J, a.J, rtol=1e-12)
    np.testing.assert_allclose(b.I_emergent, a.I_emergent, rtol=1e-12)
    v = rng.normal(size=n.shape) * n
    ja, jb = jvp_complex(m, n, Jd, v), jvp_complex(mv, n, Jd, v)
    assert np.max(np.abs(ja - jb) / (np.max(np.abs(ja), axis=1, keepdims=True))) < 1e-12
    Pa, Pb = block_jacobi(m, n, a), block_jacobi(mv, n, b)
    np.testing.assert_allclose(Pb, Pa, rtol=1e-11, atol=1e-13 * np.max(np.abs(Pa)))


def test_vanishing_velocity_gives_the_static_profiles():
    wl = W.config2(nu_scale=0.1, n_depth=10)
    col = replace(wl.columns[0], vlos=np.full(10, 1e-9))
    m = OM.build_model(wl.atom, col, 2)
    ms = OM.build_model(wl.atom, wl.columns[0], 2)
    assert m.Vdir is not None
    for d in range(4):
        np.testing.assert_allclose(m.Vdir[:, d], ms.V, rtol=1e-9, atol=1e-12 * np.max(ms.V))


def test_moving_blocks_equal_the_dense_jacobian_diagonal_blocks():
    """With J^dagger frozen the per-direction block-Jacobi blocks are exactly
    the diagonal blocks of the complex-step Jacobian (Sect. 2.5)."""
    m = _tiny_moving()
    rng = np.random.default_rng(4)
    n = W.perturbed_populations(m.nstar, rng, 0.3)
    Jd = m.B * 0.7
    res = residual(m, n, Jd, want_lambda=True)
    P = block_jacobi(m, n, res)
    Jm = dense_jacobian(m, n, Jd, istar=res.istar)
    nl = m.nl
    for k in range(m.nz):
        blk = Jm[k * nl:(k + 1) * nl, k * nl:(k + 1) * nl]
        np.testing.assert_allclose(P[k], blk, rtol=1e-9, atol=1e-11 * np.max(np.abs(blk)))
    # and the velocity field matters: the static blocks differ
    mst = OM.build_model(W.tiny_workload(n_depth=6, n_nu_line=9, n_nu_cont=3).atom,
                         W.tiny_workload(n_depth=6, n_nu_line=9, n_nu_cont=3).columns[0], 2)
    Ps = block_jacobi(mst, n, residual(mst, n, Jd, want_lambda=True))
    assert np.max(np.abs(Ps - P) / np.max(np.abs(P), axis=(1, 2), keepdims=True)) > 1e-3


def test_moving_complex_step_matches_central_differences():
    m = _tiny_moving()
    rng = np.random.default_rng(5)
    n = W.perturbed_populations(m.nstar, rng, 0.1)
    Jd = OM.initial_J(m)
    istar = np.argmax(n, axis=1)
    v = rng.normal(size=n.shape) * n
    ref = jvp_complex(m, n, Jd, v, istar=istar)
    best = min(np.max(np.abs(jvp_fd(m, n, Jd, v, scheme="central", istar=istar, eps=h) - ref)) / np.max(np.abs(ref))
               for h in (1e-3, 3e-4, 1e-4, 3e-5, 1e-5))
    assert best < 1e-7


@pytest.mark.slow
def test_constant_velocity_only_shifts_the_spectrum():
    """A column moving as a whole (constant v) is the static column in the
    comoving frame: the populations are unchanged (to the quadrature of the
    shifted, renormalised profiles on the fixed grid) and each direction's
    emergent line is the static one shifted by nu_0 mu v/c."""
    atom = W.two_level_atom(n_nu=81)
    col = W.two_level_slab(atom, n_depth=41, tau_max=1e3)
    ms = OM.build_model(atom, col, 2)
    v0 = 0.3 * atom.vchar
    mv = OM.build_model(atom, replace(col, vlos=np.full(col.n_depth, v0)), 2)
    a = jfnk(ms, ms.nstar, rtol=1e-8, ftol=1e-11)
    b = jfnk(mv, mv.nstar, rtol=1e-8, ftol=1e-11)
    assert a.converged and b.converged
    np.testing.assert_allclose(b.n, a.n, rtol=3e-3)
    nu0 = ms.trans[0].nu0
    for j in range(ms.nmu):
        shifted = np.interp(ms.nu, ms.nu + nu0 * ms.mu[j] * v0 / OM.C, a.I_emergent[:, j])
        inner = np.abs(ms.nu / nu0 - 1.0) < 3.0 * atom.vchar / OM.C
        np.testing.assert_allclose(b.I_emergent[inner, j], shifted[inner], rtol=5e-2)   # linear interpolation


@pytest.mark.slow
def test_upward_flow_shifts_the_absorption_to_the_blue():
    """Gas rising in the upper layers (v > 0, towards the observer) absorbs at
    higher frequencies: in the emergent line the inner blue wing is darker than
    the mirrored red wing, while the static line is symmetric about nu_0 (a
    flipped sign of the Doppler shift darkens the red wing instead)."""
    atom = W.two_level_atom(n_nu=81)
    col = W.two_level_slab(atom, n_depth=41, tau_max=1e3)
    tau = np.logspace(-6, 3, 41)
    v = 1.5 * atom.vchar / (1.0 + (tau / 1e-1) ** 2)      # fast near the top, at rest deep down
    ms = OM.build_model(atom, col, 2)
    mv = OM.build_model(atom, replace(col, vlos=v), 2)
    a = jfnk(ms, ms.nstar, rtol=1e-8, ftol=1e-10)
    b = jfnk(mv, mv.nstar, rtol=1e-8, ftol=1e-10)
    assert a.converged and b.converged
    nu0 = ms.trans[0].nu0
    x = (ms.nu / nu0 - 1.0) * OM.C / atom.vchar             # offset in Doppler widths, symmetric grid
    j = ms.nmu - 1                                          # the direction closest to the vertical
    blue = (x > 0.9) & (x < 2.1)
    red = blue[::-1]
    np.testing.assert_allclose(a.I_emergent[blue, j], a.I_emergent[red, j][::-1], rtol=1e-3)
    assert np.all(b.I_emergent[blue, j] < 0.97 * b.I_emergent[red, j][::-1])
