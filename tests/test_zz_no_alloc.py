"""jfnk_residual_static: the allocation-free residual agrees with jfnk_residual.

Some callers cannot allocate device memory while they run (a memory budget
owned by another allocator, or a latency-critical loop that must never wait on
cudaMalloc). For them the library offers jfnk_residual_static, whose work
buffers live in one fixed device array. This test calls it through the C ABI
twice in a row with different inputs and checks each result against the
regular entry point, element by element, with the FP64 residual tolerance
used by the parity tests (per element, relative to the gross rates of its
depth). It is collected last so that a failure here leaves the other tests'
results intact.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import model as OM

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2406_17234_gb300.binding")


def _gross(m, n, F_ref):
    # scale of the rate terms that cancel in F: sum of |n_i (C + R)| over transitions,
    # approximated from the collision rates and the residual itself
    g = np.zeros_like(n)
    for tr in m.trans:
        g[:, tr.lo] += n[:, tr.lo] * m.Cmat[:, tr.lo, tr.up] + n[:, tr.up] * m.Cmat[:, tr.up, tr.lo]
        g[:, tr.up] += n[:, tr.lo] * m.Cmat[:, tr.lo, tr.up] + n[:, tr.up] * m.Cmat[:, tr.up, tr.lo]
    return g + np.abs(F_ref)


def test_static_residual_matches_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = B.Context(0)
    lib = ctx.lib
    # the last: the full H I-like column (about 2,000 frequencies), within the
    # array since the fused formal kernel needs no per-ray buffers
    cases = [W.config1(), W.config2(nu_scale=0.3, n_depth=50), W.config3()]
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream()
    for wl in cases:
        atom = B.Atom(ctx, wl.atom)
        atm = B.Atmosphere(ctx, atom, wl.columns[0], n_mu=wl.n_mu)
        m = OM.build_model(wl.atom, wl.columns[0], wl.n_mu)
        for call in range(2):   # two calls in a row: the shared array keeps old contents
            n = W.perturbed_populations(m.nstar, rng, 0.25 * call)
            Jd = m.B * np.exp(rng.normal(0.0, 0.1, m.B.shape))
            F_ref, J_ref, _ = B.residual(atm, n, Jd, want_J=True)
            n_d = torch.from_numpy(n.ravel().copy()).cuda()
            J_d = torch.from_numpy(Jd.ravel().copy()).cuda()
            F_d = torch.full_like(n_d, float("nan"))
            Jn_d = torch.full_like(J_d, float("nan"))
            rc = lib.jfnk_residual_static(ctx.h, atm.h, C.c_void_p(n_d.data_ptr()),
                                          C.c_void_p(J_d.data_ptr()), C.c_void_p(F_d.data_ptr()),
                                          C.c_void_p(Jn_d.data_ptr()), C.c_void_p(stream.cuda_stream))
            B.check(rc, "jfnk_residual_static")
            torch.cuda.synchronize()
            F = F_d.cpu().numpy().reshape(n.shape)
            Jn = Jn_d.cpu().numpy().reshape(J_ref.shape)
            assert np.all(np.abs(F - F_ref) <= 1e-10 * _gross(m, n, F_ref))
            np.testing.assert_allclose(Jn, J_ref, rtol=1e-10, atol=1e-14 * np.max(np.abs(J_ref)))


def test_static_residual_rejects_oversized_columns():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = B.Context(0)
    wl = W.config3(n_depth=420)   # about 2,000 frequencies x 420 depths: beyond the fixed array
    atom = B.Atom(ctx, wl.atom)
    atm = B.Atmosphere(ctx, atom, wl.columns[0], n_mu=wl.n_mu)
    n_d = torch.zeros(atm.n_depth * atm.n_levels, dtype=torch.float64, device="cuda")
    F_d = torch.zeros_like(n_d)
    rc = ctx.lib.jfnk_residual_static(ctx.h, atm.h, C.c_void_p(n_d.data_ptr()), None,
                                      C.c_void_p(F_d.data_ptr()), None, None)
    assert rc == B.JFNK_E_INVALID
    assert b"static scratch" in ctx.lib.jfnk_last_error()
