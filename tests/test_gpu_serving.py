"""GPU tests of the serving runtime (continuous batching, jfnk_server_*).

A column's result must not depend on the columns it shares the device with:
each request of a mixed stream (two-level, Ca II-like and H I-like atoms of
different sizes) is compared with the same column solved alone by jfnk_solve
with the same options. The stated tolerance is the mixed-mode bar (1e-3
relative); the per-column arithmetic is the same kernels in the same order,
so the test also asserts the stronger bit-identity it gets.
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


def _opts(hydrogen=False):
    """Per-request options: a short capped RH92 warm-up for the two-level and
    Ca II-like columns; the H I-like ones need a longer one (JFNK after ten
    RH92 iterations diverges for them, alone as in the mix)."""
    if hydrogen:
        return B.default_options(precision=B.JFNK_MIXED, rh92_warmup=200)
    return B.default_options(precision=B.JFNK_MIXED, rh92_warmup=10, rh92_switch=0.1)


def _mixed_columns(ctx):
    """(atom handle, atmosphere handle, options) of a small mixed stream."""
    wls = [(W.config1(n_depth=61, n_nu=41), False), (W.config2(nu_scale=0.15, n_depth=41), False),
           (W.config3(nu_scale=0.1, n_depth=37), True), (W.config2(seed=2, nu_scale=0.12, n_depth=53), False),
           (W.config3(seed=3, nu_scale=0.08, n_depth=45), True), (W.config1(n_depth=41, n_nu=31), False)]
    out = []
    for wl, h in wls:
        atom = B.Atom(ctx, wl.atom)
        out.append((atom, B.Atmosphere(ctx, atom, wl.columns[0], n_mu=wl.n_mu), _opts(h)))
    return out


def _drain(sv, n, max_active=None, max_steps=5000):
    res = []
    for _ in range(max_steps):
        active, _ = sv.step()
        if max_active is not None:
            assert active <= max_active
        res += sv.poll()
        if len(res) == n:
            return res
    raise AssertionError("server did not finish")


def _shape(cols):
    return dict(max_depth=max(a.n_depth for _, a, _ in cols), max_freq=max(a.n_nu for _, a, _ in cols),
                max_levels=max(a.n_levels for _, a, _ in cols),
                max_trans=max(a.n_transitions for _, a, _ in cols), max_mu=5)


def test_server_result_is_the_same_alone_and_in_the_mix(ctx):
    cols = _mixed_columns(ctx)
    sv = B.Server(ctx, max_slots=3, opts=_opts(), **_shape(cols))
    for i, (_, a, o) in enumerate(cols):
        sv.submit(a, i, o)
    res = {r["id"]: r for r in _drain(sv, len(cols))}
    sv.close()
    for i, (_, a, o) in enumerate(cols):
        r = res[i]
        assert r["status"] == 0, r
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        n_alone, _, st = B.solve(a, o)
        assert st["status"] == 0
        np.testing.assert_allclose(r["n"], n_alone, rtol=1e-3)
        np.testing.assert_array_equal(r["n"], n_alone)
        assert r["stats"]["F_calls"] == st["F_calls"]


def test_server_admits_by_free_memory(ctx):
    """A pool that holds only the largest request: one column in flight at a
    time, every request still served, results unchanged."""
    cols = _mixed_columns(ctx)[:3]
    probe = B.Server(ctx, max_slots=1, opts=_opts(), **_shape(cols))
    biggest = max(probe.bytes(a) for _, a, _ in cols)
    probe.close()
    sv = B.Server(ctx, max_slots=3, mem_bytes=biggest, opts=_opts(), **_shape(cols))
    for i, (_, a, o) in enumerate(cols):
        sv.submit(a, i, o)
    res = {r["id"]: r for r in _drain(sv, len(cols), max_active=1)}
    sv.close()
    for i, (_, a, o) in enumerate(cols):
        n_alone, _, _ = B.solve(a, o)
        np.testing.assert_array_equal(res[i]["n"], n_alone)
    # requests run one after another: each is admitted after the previous finished
    order = sorted(res.values(), key=lambda r: r["t_admit"])
    for prev, nxt in zip(order, order[1:]):
        assert nxt["t_admit"] >= prev["t_done"]


def test_server_rejects_columns_and_options_it_cannot_hold(ctx):
    cols = _mixed_columns(ctx)[:2]
    shape = _shape(cols)
    shape["max_depth"] = min(a.n_depth for _, a, _ in cols)
    sv = B.Server(ctx, max_slots=2, opts=_opts(), **shape)
    deepest = max(cols, key=lambda c: c[1].n_depth)[1]
    shallow = min(cols, key=lambda c: c[1].n_depth)[1]
    codes = []
    for atm, o in [(deepest, None), (shallow, B.default_options(precision=B.JFNK_FP64))]:
        try:
            sv.submit(atm, len(codes), o)
            codes.append(0)
        except B.JFNKError as err:
            codes.append(err.code)
    sv.close()
    assert codes == [B.JFNK_E_INVALID, B.JFNK_E_INVALID]
