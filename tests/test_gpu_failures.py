"""Failure detection without faulting the GPU: bad inputs and exhausted
limits made on the host, each reported through the C ABI as a status while
the context, the other columns of a batch and the other requests of a server
carry on unchanged.

  * a non-finite population in the initial guess: the first residual is
    non-finite, the column stops with JFNK_E_NAN (Algorithm 2 cannot proceed
    from it), and the next solve on the same context is unaffected;
  * the tick budget (max_ticks) and the Newton iteration limit (maxiter) stop
    a column with JFNK_E_TIMEOUT / JFNK_E_MAXITER;
  * in a batch, a failing column does not change the others' results
    (bit-identical to their solves alone);
  * in the server, a request that fails is retired with its status and the
    requests around it are served with their usual results;
  * a level that no transition touches makes every preconditioner block
    singular: the solve stops with an error status and the context serves the
    next solve as before.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2406_17234_gb300.binding")


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B.Context(0)


def _col(ctx, wl, n_mu=3):
    atom = B.Atom(ctx, wl.atom)
    return atom, B.Atmosphere(ctx, atom, wl.columns[0], n_mu=n_mu)


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_population_stops_the_column_with_nan_status(ctx, precision):
    wl = W.config2(nu_scale=0.15, n_depth=30)
    atom, atm = _col(ctx, wl)
    n0 = atm.lte().copy()
    n0[7, 2] = np.nan
    n, _, st = B.solve(atm, B.default_options(precision=precision), n0=n0, raise_on_fail=False)
    assert st["status"] == B.JFNK_E_NAN
    assert st["F_calls"] == 1 and st["newton_iters"] == 0
    with pytest.raises(B.JFNKError) as e:
        B.solve(atm, B.default_options(precision=precision), n0=n0)
    assert e.value.code == B.JFNK_E_NAN
    # the context and the column's buffers are still good
    n_ok, _, s_ok = B.solve(atm, B.default_options(precision=precision))
    n_ref, _, _ = B.solve(atm, B.default_options(precision=precision))
    assert s_ok["status"] == 0
    np.testing.assert_array_equal(n_ok, n_ref)


def test_tick_and_iteration_limits_report_their_status(ctx):
    wl = W.config1(n_depth=41, n_nu=21)
    atom, atm = _col(ctx, wl)
    _, _, st = B.solve(atm, B.default_options(max_ticks=5), raise_on_fail=False)
    assert st["status"] == B.JFNK_E_TIMEOUT and st["F_calls"] == 5
    _, _, st = B.solve(atm, B.default_options(maxiter=1), raise_on_fail=False)
    assert st["status"] == B.JFNK_E_MAXITER and st["newton_iters"] == 1
    _, _, st = B.solve(atm, B.default_options(solver=B.JFNK_SOLVER_RH92, maxiter=3), raise_on_fail=False)
    assert st["status"] == B.JFNK_E_MAXITER and st["rh92_iters"] == 3


@pytest.mark.parametrize("precision", [0, 1])
def test_a_failing_column_leaves_the_batch_unchanged(ctx, precision):
    """One column of a batch starts from a NaN population; it stops with
    JFNK_E_NAN after its first evaluation while the others converge exactly as
    they do alone."""
    import ctypes as C
    wl = W.config4(n_columns=4, nz_min=40, nz_max=60, nu_scale=0.1)
    atom = B.Atom(ctx, wl.atom)
    atms = [B.Atmosphere(ctx, atom, c, n_mu=3) for c in wl.columns]
    ns = [a.lte().copy() for a in atms]
    ns[2][5, 1] = np.nan
    start = dict(rh92_warmup=5, rh92_switch=0.1)     # the batch workload's hybrid start
    opts = B.default_options(precision=precision, init=B.JFNK_INIT_USER, **start)
    hs = (C.c_void_p * len(atms))(*[a.h for a in atms])
    nps = (C.c_void_p * len(atms))(*[n.ctypes.data for n in ns])
    stats = (B.jfnk_stats * len(atms))()
    rc = ctx.lib.jfnk_batch_solve(ctx.h, len(atms), hs, C.byref(opts), nps, None, stats, B.JFNK_MEM_HOST, None)
    assert rc == B.JFNK_E_NAN
    for i, (a, n, s) in enumerate(zip(atms, ns, stats)):
        if i == 2:
            assert s.status == B.JFNK_E_NAN and s.F_calls <= 2
            continue
        assert s.status == 0
        n1, _, s1 = B.solve(a, B.default_options(precision=precision, **start))
        assert s1["F_calls"] == s.F_calls
        np.testing.assert_array_equal(n, n1)


def test_server_retires_a_failing_request_and_serves_the_others(ctx):
    """A request whose own options leave it one Newton iteration is retired
    with JFNK_E_MAXITER; the requests before and after it are served with the
    results they get alone."""
    wls = [W.config2(nu_scale=0.12, n_depth=41), W.config1(n_depth=61, n_nu=41),
           W.config2(seed=2, nu_scale=0.1, n_depth=37)]
    cols = [_col(ctx, wl) for wl in wls]
    base = B.default_options(precision=B.JFNK_MIXED, rh92_warmup=10, rh92_switch=0.1)
    sv = B.Server(ctx, max_slots=2, max_depth=max(a.n_depth for _, a in cols),
                  max_freq=max(a.n_nu for _, a in cols), max_levels=6, max_trans=16, max_mu=3, opts=base)
    bad = B.default_options(precision=B.JFNK_MIXED, rh92_warmup=10, rh92_switch=0.1, maxiter=1)
    for i, (_, a) in enumerate(cols):
        sv.submit(a, i, bad if i == 1 else base)
    res = {}
    for _ in range(5000):
        sv.step()
        for r in sv.poll():
            res[r["id"]] = r
        if len(res) == len(cols):
            break
    sv.close()
    assert len(res) == len(cols)
    assert res[1]["status"] == B.JFNK_E_MAXITER and res[1]["stats"]["newton_iters"] == 1
    for i in (0, 2):
        assert res[i]["status"] == 0
        n1, _, s1 = B.solve(cols[i][1], base)
        np.testing.assert_array_equal(res[i]["n"], n1)


def test_singular_preconditioner_stops_with_a_status(ctx):
    """An atom with an isolated bound level (no line or continuum touches it):
    its rate-equation row is identically zero, so the block-Jacobi blocks of
    Sect. 2.5.1 are singular (the level is never the conservation row, being
    almost empty). The solve ends with an error status, not a hang or a
    wrong 'converged', and a regular column solves as before afterwards."""
    from dataclasses import replace
    base = W.tiny_workload(n_depth=12, n_nu_line=9, n_nu_cont=5)
    a = base.atom
    E = np.array([a.E_eV[0], a.E_eV[1], 6.0, a.E_eV[2]])
    g = np.array([a.g[0], a.g[1], 2.0, a.g[2]])
    stage = np.array([a.stage[0], a.stage[1], a.stage[1], a.stage[2]])
    lines = [replace(ln, j=ln.j) for ln in a.lines]                  # (0, 1)
    conts = [replace(c, j=3) for c in a.conts]                         # (0, 3), (1, 3)
    iso = replace(a, E_eV=E, g=g, stage=stage, lines=lines, conts=conts, name="isolated level")
    atom = B.Atom(ctx, iso)
    atm = B.Atmosphere(ctx, atom, base.columns[0], n_mu=base.n_mu)
    n, _, st = B.solve(atm, B.default_options(), raise_on_fail=False)
    assert st["status"] != 0
    assert st["status"] in (B.JFNK_E_NAN, B.JFNK_E_MAXITER, B.JFNK_E_TIMEOUT)
    # the context and a regular column are unaffected
    wl = W.config2(nu_scale=0.15, n_depth=30)
    atom2, atm2 = _col(ctx, wl)
    n1, _, s1 = B.solve(atm2, B.default_options())
    n2, _, s2 = B.solve(atm2, B.default_options())
    assert s1["status"] == 0
    np.testing.assert_array_equal(n1, n2)
