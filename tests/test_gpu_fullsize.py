"""GPU parity at the full sizes of the five workloads, against the FP64 oracle.

Every case here runs at the size the benchmark times: 5 mu per hemisphere,
the full frequency grids (about 1,000 for the Ca II-like atom, 2,000 for the
H I-like one), 82 depths for the single columns, the 64- and 256-depth
extremes of the 4,096-column batch, and requests drawn from the serving
stream. The oracle's converged reference solves run in a spawn-started
process pool beside the GPU work (``oracle_jobs``).

Bars (per element, relative): converged populations 1e-5 in FP64 and 1e-3 in
the mixed mode, both against the oracle solved far past the stopping rule
(r_tol 1e-6, ||dn/n|| < 1e-10). Residuals and Jacobian-vector products are
compared per element against the gross rate scale of their depth, as in the
reduced-size parity tests. Each solve prints the residual norm it reached
(run with -s to see them).
"""
import numpy as np
import pytest

import oracle_jobs as J
import workloads as W
from oracle import model as OM
from oracle.residual import jvp_complex, residual as ora_residual

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

B = pytest.importorskip("paper_2406_17234_gb300.binding")

TIGHT = dict(rtol=1e-6, ftol=1e-10)          # FP64 GPU and every oracle reference
MIXED_TIGHT = dict(rtol=1e-4, ftol=1e-5)     # mixed mode: FP32 formal solutions floor dn/n near 1e-6
C3_START = dict(switch_tol=0.03, rh92_max=60)   # hybrid start of the H I-like columns
C4_START = dict(switch_tol=0.1, rh92_max=5)     # hybrid start of the batched Ca II-like columns
SERVE_START = {"H": C3_START, "other": dict(switch_tol=0.1, rh92_max=10)}


def _gpu_start(start):
    return dict(rh92_warmup=start["rh92_max"], rh92_switch=start["switch_tol"])


def _c4_indices(wl):
    """The shallowest and the deepest column of the batch and its first two."""
    nz = np.array([c.n_depth for c in wl.columns])
    out = [int(np.argmin(nz)), int(np.argmax(nz))]
    return out + [i for i in (0, 1) if i not in out]


def _c5_requests(wl):
    """The smallest request (N_nu x N_z) of each atom kind among the stream's first 300."""
    best = {}
    for r in range(300):
        a = wl.atoms[r]
        kind = a.name.split()[0].split("-")[0]
        cost = (sum(l.n_nu for l in a.lines) + sum(c.n_nu for c in a.conts)) * wl.columns[r].n_depth
        if kind not in best or cost < best[kind][0]:
            best[kind] = (cost, r)
    return sorted(r for _, r in best.values())


def _serve_start(atom):
    return SERVE_START["H" if atom.name.startswith("H") else "other"]


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B.Context(0)


@pytest.fixture(scope="module")
def wls():
    return {"c2": W.config2(), "c3": W.config3(), "c4": W.config4(), "c5": W.config5()}


@pytest.fixture(scope="module", autouse=True)
def references(wls):
    """Starts every oracle reference solve of this module at once."""
    c2, c3, c4, c5 = wls["c2"], wls["c3"], wls["c4"], wls["c5"]
    J.submit("c2", c2.atom, c2.columns[0], 5, "jfnk", **TIGHT)
    J.submit("c3", c3.atom, c3.columns[0], 5, "hybrid", **C3_START, **TIGHT)
    for i in _c4_indices(c4):
        J.submit(("c4", i), c4.atom, c4.columns[i], 5, "hybrid", **C4_START, **TIGHT)
    for r in _c5_requests(c5):
        J.submit(("c5", r), c5.atoms[r], c5.columns[r], 5, "hybrid", **_serve_start(c5.atoms[r]), **TIGHT)
    yield
    J.shutdown()


def _report(name, st, err):
    print(f"\nPARITY {name}: max rel err vs oracle {err:.2e}, ||F||inf {st['F_norm']:.3e} "
          f"(drop {st['F_norm'] / st['F_norm0']:.2e}), F_calls {st['F_calls']}, newton {st['newton_iters']}, "
          f"rh92 {st['rh92_iters']}")


def _rel(a, b):
    return float(np.max(np.abs(a / b - 1.0)))


def _gross(m, n, R_up, R_dn):
    g = np.zeros_like(n)
    for t, tr in enumerate(m.trans):
        up = n[:, tr.lo] * (m.Cmat[:, tr.lo, tr.up] + R_up[t])
        dn = n[:, tr.up] * (m.Cmat[:, tr.up, tr.lo] + R_dn[t])
        g[:, tr.lo] += up + dn
        g[:, tr.up] += up + dn
    return g


@pytest.mark.parametrize("cfg", ["c2", "c3"])
@pytest.mark.parametrize("precision", [0, 1])
def test_fullsize_residual_and_jvp(ctx, wls, cfg, precision):
    """F, J, the emergent intensity and J_F v of one full-size column at
    perturbed populations, per element against the oracle."""
    wl = wls[cfg]
    atom = B.Atom(ctx, wl.atom)
    atm = B.Atmosphere(ctx, atom, wl.columns[0], n_mu=5)
    m = OM.build_model(wl.atom, wl.columns[0], 5)
    rng = np.random.default_rng(21)
    n = W.perturbed_populations(m.nstar, rng, 0.3)
    Jd = m.B * np.exp(rng.normal(0, 0.2, m.B.shape))
    F, Jn, Ie = B.residual(atm, n, Jd, precision=precision, want_J=True, want_emergent=True)
    r = ora_residual(m, n, Jd)
    gross = _gross(m, n, r.R_up, r.R_dn)
    bar = 1e-10 if precision == 0 else 1e-4
    excess = np.abs(F - r.F) / (bar * gross + 1e-12 * np.abs(r.F))
    k, l = np.unravel_index(int(np.argmax(excess)), excess.shape)
    assert excess[k, l] <= 1.0, (f"depth {k} level {l}: F {F[k, l]:.6e} oracle {r.F[k, l]:.6e} "
                                 f"gross {gross[k, l]:.3e} istar {r.istar[k]} n {n[k].tolist()}")
    k = np.arange(m.nz)
    np.testing.assert_allclose(F[k, r.istar], r.F[k, r.istar], rtol=1e-13)
    np.testing.assert_allclose(Jn, r.J, rtol=bar, atol=(1e-14 if precision == 0 else 1e-9) * np.max(r.J))
    if precision == 0:
        np.testing.assert_allclose(Ie, r.I_emergent, rtol=1e-10, atol=1e-14 * np.max(r.I_emergent))
    v = rng.normal(size=n.shape) * n
    g = B.jvp(atm, n, v, Jd, precision=precision)
    ref = jvp_complex(m, n, Jd, v)
    scale = np.max(np.abs(ref), axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(g - ref) / scale) < (1e-9 if precision == 0 else 1e-3)


def test_config2_fullsize_fp64(ctx, wls):
    """Config 2 (Ca II-like, 82 depths, about 1,000 frequencies, FP64): the
    converged populations within 1e-5 of the oracle's, and the benchmark's
    paper-tolerance solve within 1e-3."""
    wl = wls["c2"]
    atom = B.Atom(ctx, wl.atom)
    atm = B.Atmosphere(ctx, atom, wl.columns[0], n_mu=5)
    n, _, st = B.solve(atm, B.default_options(**TIGHT))
    ref = J.result("c2")
    assert ref["converged"] and st["status"] == 0
    err = _rel(n, ref["n"])
    _report("config 2 FP64 (r_tol 1e-6, ftol 1e-10)", st, err)
    assert err < 1e-5
    np.testing.assert_allclose(n.sum(axis=1), wl.columns[0].ntot, rtol=1e-12)
    n2, _, st2 = B.solve(atm, B.default_options())
    err2 = _rel(n2, ref["n"])
    _report("config 2 FP64 (paper stopping rule)", st2, err2)
    assert st2["status"] == 0 and err2 < 1e-3


def test_config3_fullsize_mixed_and_fp64(ctx, wls):
    """Config 3 (H I-like, about 2,000 frequencies, hybrid start): the mixed
    mode within 1e-3 of the oracle (and of the FP64 GPU run), the FP64 mode
    within 1e-5."""
    wl = wls["c3"]
    atom = B.Atom(ctx, wl.atom)
    atm = B.Atmosphere(ctx, atom, wl.columns[0], n_mu=5)
    start = _gpu_start(C3_START)
    n64, _, s64 = B.solve(atm, B.default_options(**start, **TIGHT))
    nmx, _, smx = B.solve(atm, B.default_options(precision=B.JFNK_MIXED, **start, **MIXED_TIGHT))
    npp, _, spp = B.solve(atm, B.default_options(precision=B.JFNK_MIXED, **start))
    ref = J.result("c3")
    assert ref["converged"]
    assert s64["status"] == 0 and smx["status"] == 0 and spp["status"] == 0
    e64, emx, epp = _rel(n64, ref["n"]), _rel(nmx, ref["n"]), _rel(npp, ref["n"])
    _report("config 3 FP64 (tight)", s64, e64)
    _report("config 3 mixed (r_tol 1e-4, ftol 1e-5)", smx, emx)
    _report("config 3 mixed (paper stopping rule)", spp, epp)
    print(f"PARITY config 3 mixed vs FP64 GPU: {_rel(nmx, n64):.2e}")
    assert e64 < 1e-5
    assert emx < 1e-3 and epp < 1e-3
    assert _rel(nmx, n64) < 1e-3


@pytest.mark.parametrize("variant", ["JFNK_FORMAL_SWEEP_THREAD", "JFNK_FORMAL_SWEEP_WARP",
                                     "JFNK_FORMAL_SWEEP_THREAD_FUSED"])
def test_config4_batch_columns_against_oracle(ctx, wls, variant):
    """Columns of the 4,096-column batch (its 64- and 256-depth extremes and
    two more) solved together in one mixed batch plan with the benchmark's
    options (5 angles, hybrid start of at most 5 RH92 iterations, paper
    stopping rule), each within 1e-3 of the oracle; every sweep kernel."""
    wl = wls["c4"]
    idx = _c4_indices(wl)
    atom = B.Atom(ctx, wl.atom)
    atms = [B.Atmosphere(ctx, atom, wl.columns[i], n_mu=5) for i in idx]
    plan = B.BatchPlan(ctx, atms, precision=B.JFNK_MIXED)
    opts = B.default_options(precision=B.JFNK_MIXED, formal_variant=getattr(B, variant), **_gpu_start(C4_START))
    ns, stats = plan.run(opts)
    for i, n, st in zip(idx, ns, stats):
        ref = J.result(("c4", i))
        assert ref["converged"] and st["status"] == 0
        assert st["formal_kernel"] == getattr(B, variant)
        err = _rel(n, ref["n"])
        _report(f"config 4 column {i} (N_z {wl.columns[i].n_depth}, {variant})", st, err)
        assert err < 1e-3
    plan.close()


def test_config5_served_requests_against_oracle(ctx, wls):
    """One request of each atom kind taken from the serving stream, solved by
    the continuous-batching server among other requests, each within 1e-3 of
    the oracle."""
    wl = wls["c5"]
    picked = _c5_requests(wl)
    others = [r for r in range(8) if r not in picked][:3]
    ids = picked + others
    handles = {}
    for r in ids:
        a = B.Atom(ctx, wl.atoms[r])
        handles[r] = (a, B.Atmosphere(ctx, a, wl.columns[r], n_mu=5))
    atms = [h[1] for h in handles.values()]
    sv = B.Server(ctx, max_slots=3, max_depth=max(a.n_depth for a in atms), max_freq=max(a.n_nu for a in atms),
                  max_levels=max(a.n_levels for a in atms), max_trans=max(a.n_transitions for a in atms),
                  max_mu=5, opts=B.default_options(precision=B.JFNK_MIXED))
    for r in ids:
        sv.submit(handles[r][1], r, B.default_options(precision=B.JFNK_MIXED,
                                                      **_gpu_start(_serve_start(wl.atoms[r]))))
    res = {}
    for _ in range(20000):
        sv.step()
        for x in sv.poll():
            res[x["id"]] = x
        if len(res) == len(ids):
            break
    sv.close()
    assert len(res) == len(ids)
    for r in picked:
        ref = J.result(("c5", r))
        assert ref["converged"] and res[r]["status"] == 0, res[r]
        err = _rel(res[r]["n"], ref["n"])
        _report(f"config 5 request {r} ({wl.atoms[r].name}, N_z {wl.columns[r].n_depth})", res[r]["stats"], err)
        assert err < 1e-3
