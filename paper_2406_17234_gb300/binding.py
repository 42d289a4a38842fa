"""Thin ctypes binding of ``libjfnk.so`` (include/jfnk.h): argument marshalling only.

Every computation happens in the library's CUDA kernels. Functions keep the
C names; the small classes below only own handles and convert the seeded
descriptors of ``workloads`` (or any object with the same fields) into the
C structures. Arrays are numpy (host memory) or torch CUDA tensors (device
memory, passed by ``data_ptr()`` with the current torch stream).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libjfnk.so")

JFNK_OK = 0
JFNK_E_INVALID = -1
JFNK_E_NOMEM = -2
JFNK_E_CUDA = -3
JFNK_E_DIVERGED = -4
JFNK_E_NAN = -5
JFNK_E_TIMEOUT = -6
JFNK_E_MAXITER = -7
JFNK_MEM_HOST = 0
JFNK_MEM_DEVICE = 1
JFNK_FP64 = 0
JFNK_MIXED = 1
JFNK_INIT_LTE = 0
JFNK_INIT_USER = 1
JFNK_INIT_ZERO_RADIATION = 2
JFNK_JVP_TANGENT = 0
JFNK_JVP_FORWARD_EPS1 = 1
JFNK_JVP_FORWARD_EPS2 = 2
JFNK_JVP_CENTRAL = 3
JFNK_KRYLOV_GMRES = 0
JFNK_KRYLOV_BICGSTAB = 1
JFNK_SOLVER_JFNK = 0
JFNK_SOLVER_RH92 = 1
JFNK_FORMAL_PER_RAY = 0
JFNK_FORMAL_FUSED = 1
JFNK_FORMAL_SWEEP_THREAD = 2
JFNK_FORMAL_SWEEP_WARP = 3
JFNK_FORMAL_MOVING = 4
JFNK_FORMAL_SWEEP_THREAD_FUSED = 5

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class jfnk_bb_desc(C.Structure):
    _fields_ = [("i", C.c_int), ("j", C.c_int), ("f", C.c_double), ("damping", C.c_double),
                ("upsilon", C.c_double), ("eps", C.c_double), ("n_nu", C.c_int),
                ("q_core", C.c_double), ("q_wing", C.c_double)]


class jfnk_bf_desc(C.Structure):
    _fields_ = [("i", C.c_int), ("j", C.c_int), ("alpha0", C.c_double), ("q0", C.c_double),
                ("n_nu", C.c_int), ("y_max", C.c_double)]


class jfnk_atom_desc(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("E_eV", _dp), ("g", _dp), ("stage", _ip),
                ("n_bb", C.c_int), ("bb", C.POINTER(jfnk_bb_desc)), ("n_bf", C.c_int),
                ("bf", C.POINTER(jfnk_bf_desc)), ("mass_amu", C.c_double), ("vchar", C.c_double)]


class jfnk_atmos_desc(C.Structure):
    _fields_ = [("n_depth", C.c_int), ("z", _dp), ("T", _dp), ("ne", _dp), ("ntot", _dp),
                ("rho", _dp), ("vturb", _dp), ("kappa", C.c_double), ("kappa_nu_ref", C.c_double),
                ("kappa_power", C.c_double), ("kappa_max", C.c_double), ("thomson", C.c_int),
                ("n_mu", C.c_int), ("vlos", _dp)]


class jfnk_options(C.Structure):
    _fields_ = [("ftol", C.c_double), ("fdrop", C.c_double), ("rtol", C.c_double),
                ("maxiter", C.c_int), ("krylov_max", C.c_int), ("max_restarts", C.c_int),
                ("precision", C.c_int), ("init", C.c_int), ("clamp", C.c_int),
                ("rh92_warmup", C.c_int), ("rh92_switch", C.c_double), ("max_ticks", C.c_int),
                ("profile", C.c_int), ("formal_variant", C.c_int), ("precond", C.c_int), ("jvp", C.c_int),
                ("krylov", C.c_int), ("solver", C.c_int), ("line_search", C.c_int)]


class jfnk_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int), ("rh92_iters", C.c_int),
                ("F_calls", C.c_int), ("jvp_calls", C.c_int), ("F_norm", C.c_double),
                ("F_norm0", C.c_double), ("dn_norm", C.c_double), ("ray_points", C.c_double),
                ("formal_ms", C.c_double), ("formal_launches", C.c_int), ("kernel_launches", C.c_int),
                ("formal_qb", C.c_int), ("formal_threads", C.c_int), ("formal_kernel", C.c_int),
                ("formal_tan_ms", C.c_double), ("formal_occ", C.c_int), ("formal_occ_base", C.c_int),
                ("formal_fuse", C.c_int), ("stage_ms", C.c_double * 6),
                ("opacity_depths", C.c_int)]

    def as_dict(self):
        return {f: (list(v) if isinstance(v, C.Array) else v)
                for f, v in ((f, getattr(self, f)) for f, _ in self._fields_)}


class jfnk_server_desc(C.Structure):
    _fields_ = [("max_slots", C.c_int), ("max_depth", C.c_int), ("max_freq", C.c_int),
                ("max_levels", C.c_int), ("max_trans", C.c_int), ("max_mu", C.c_int),
                ("mem_bytes", C.c_size_t), ("opts", jfnk_options)]


class jfnk_result(C.Structure):
    _fields_ = [("id", C.c_longlong), ("status", C.c_int), ("stats", jfnk_stats),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


# name -> (restype, argtypes)
_SIGNATURES = {
    "jfnk_last_error": (C.c_char_p, []),
    "jfnk_default_options": (None, [C.POINTER(jfnk_options)]),
    "jfnk_init": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "jfnk_destroy_ctx": (C.c_int, [C.c_void_p]),
    "jfnk_create_atom": (C.c_int, [C.c_void_p, C.POINTER(jfnk_atom_desc), C.POINTER(C.c_void_p)]),
    "jfnk_destroy_atom": (C.c_int, [C.c_void_p]),
    "jfnk_atom_info": (C.c_int, [C.c_void_p, _ip, _ip, _ip]),
    "jfnk_atom_frequencies": (C.c_int, [C.c_void_p, _dp]),
    "jfnk_create_atmosphere": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(jfnk_atmos_desc),
                                         C.POINTER(C.c_void_p)]),
    "jfnk_destroy_atmosphere": (C.c_int, [C.c_void_p]),
    "jfnk_atmos_info": (C.c_int, [C.c_void_p, _ip, _ip, _ip, _ip, _dp]),
    "jfnk_atmos_table": (C.c_int, [C.c_void_p, C.c_int, _dp, C.c_size_t]),
    "jfnk_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "jfnk_jvp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_int, C.c_void_p]),
    "jfnk_block_jacobi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int, C.c_void_p]),
    "jfnk_block_jacobi_variant": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "jfnk_rh92_update": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "jfnk_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(jfnk_options), C.c_void_p,
                             C.c_void_p, C.POINTER(jfnk_stats), C.c_int, C.c_void_p]),
    "jfnk_probe_alu": (C.c_int, [C.c_void_p, C.c_int, _dp]),
    "jfnk_check_arith": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "jfnk_batch_create": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.c_int, C.c_int,
                                    C.POINTER(C.c_void_p)]),
    "jfnk_batch_run": (C.c_int, [C.c_void_p, C.POINTER(jfnk_options), C.POINTER(C.c_void_p),
                                 C.POINTER(C.c_void_p), C.POINTER(jfnk_stats), C.c_int, C.c_void_p]),
    "jfnk_batch_destroy": (C.c_int, [C.c_void_p]),
    "jfnk_residual_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]),
    "jfnk_server_create": (C.c_int, [C.c_void_p, C.POINTER(jfnk_server_desc), C.POINTER(C.c_void_p)]),
    "jfnk_server_bytes": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "jfnk_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p,
                                     C.POINTER(jfnk_options)]),
    "jfnk_server_step": (C.c_int, [C.c_void_p, _ip, _ip]),
    "jfnk_server_poll": (C.c_int, [C.c_void_p, C.POINTER(jfnk_result), C.c_int, _ip]),
    "jfnk_server_clock": (C.c_double, [C.c_void_p]),
    "jfnk_server_destroy": (C.c_int, [C.c_void_p]),
    "jfnk_batch_solve": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p),
                                   C.POINTER(jfnk_options), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p), C.POINTER(jfnk_stats), C.c_int,
                                   C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads the shared library and declares every exported function."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libjfnk.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class JFNKError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().jfnk_last_error().decode()
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def check(code: int, where: str):
    if code != JFNK_OK:
        raise JFNKError(code, where)


def default_options(**kw) -> jfnk_options:
    o = jfnk_options()
    load().jfnk_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Context:
    def __init__(self, device: int = 0):
        self.lib = load()
        h = C.c_void_p()
        check(self.lib.jfnk_init(device, C.byref(h)), "jfnk_init")
        self.h = h

    def close(self):
        if self.h:
            self.lib.jfnk_destroy_ctx(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Atom:
    """Atom handle built from a ``workloads.Atom``-like descriptor."""

    def __init__(self, ctx: Context, atom):
        self.ctx = ctx
        lib = ctx.lib
        self._E = _f64(atom.E_eV)
        self._g = _f64(atom.g)
        self._st = np.ascontiguousarray(np.asarray(atom.stage, dtype=np.int32))
        bb = (jfnk_bb_desc * max(1, len(atom.lines)))()
        for k, l in enumerate(atom.lines):
            bb[k] = jfnk_bb_desc(l.i, l.j, l.f, l.damping, l.upsilon, l.eps, l.n_nu, l.q_core, l.q_wing)
        bf = (jfnk_bf_desc * max(1, len(atom.conts)))()
        for k, c in enumerate(atom.conts):
            bf[k] = jfnk_bf_desc(c.i, c.j, c.alpha0, c.q0, c.n_nu, c.y_max)
        self._bb, self._bf = bb, bf
        d = jfnk_atom_desc(len(self._E), self._E.ctypes.data_as(_dp), self._g.ctypes.data_as(_dp),
                           self._st.ctypes.data_as(_ip), len(atom.lines), bb, len(atom.conts), bf,
                           atom.mass_amu, atom.vchar)
        h = C.c_void_p()
        check(lib.jfnk_create_atom(ctx.h, C.byref(d), C.byref(h)), "jfnk_create_atom")
        self.h = h
        nl, nt, nq = C.c_int(), C.c_int(), C.c_int()
        lib.jfnk_atom_info(h, C.byref(nl), C.byref(nt), C.byref(nq))
        self.n_levels, self.n_transitions, self.n_nu = nl.value, nt.value, nq.value

    def frequencies(self) -> np.ndarray:
        nu = np.zeros(self.n_nu)
        check(self.ctx.lib.jfnk_atom_frequencies(self.h, nu.ctypes.data_as(_dp)), "jfnk_atom_frequencies")
        return nu

    def __del__(self):
        # a context finalized first (garbage cycles are finalized in any
        # order) has already gone: its handle must not be touched any more
        try:
            if self.h and self.ctx.h:
                self.ctx.lib.jfnk_destroy_atom(self.h)
        except Exception:
            pass


class Atmosphere:
    """Column handle built from a ``workloads.Column``-like descriptor."""

    def __init__(self, ctx: Context, atom: Atom, col, n_mu: int = 5):
        self.ctx, self.atom = ctx, atom
        lib = ctx.lib
        keep = [_f64(col.z), _f64(col.T), _f64(col.ne), _f64(col.ntot), _f64(col.rho)]
        vt = None if getattr(col, "vturb", None) is None else _f64(col.vturb)
        vl = None if getattr(col, "vlos", None) is None else _f64(col.vlos)
        self._keep = keep + [vt, vl]
        p = [k.ctypes.data_as(_dp) for k in keep]
        d = jfnk_atmos_desc(len(keep[0]), p[0], p[1], p[2], p[3], p[4],
                            vt.ctypes.data_as(_dp) if vt is not None else None,
                            col.kappa, getattr(col, "kappa_nu_ref", 0.0), getattr(col, "kappa_power", 0.0),
                            getattr(col, "kappa_max", 1.0), 1 if col.thomson else 0, n_mu,
                            vl.ctypes.data_as(_dp) if vl is not None else None)
        h = C.c_void_p()
        check(lib.jfnk_create_atmosphere(ctx.h, atom.h, C.byref(d), C.byref(h)), "jfnk_create_atmosphere")
        self.h = h
        nz, nq, nl, nt, rp = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_double()
        lib.jfnk_atmos_info(h, C.byref(nz), C.byref(nq), C.byref(nl), C.byref(nt), C.byref(rp))
        self.n_depth, self.n_nu, self.n_levels, self.n_transitions = nz.value, nq.value, nl.value, nt.value
        self.ray_points = rp.value
        self.n_mu = n_mu

    def table(self, which: int, count: int) -> np.ndarray:
        out = np.zeros(count)
        check(self.ctx.lib.jfnk_atmos_table(self.h, which, out.ctypes.data_as(_dp), count), "jfnk_atmos_table")
        return out

    def lte(self) -> np.ndarray:
        return self.table(0, self.n_depth * self.n_levels).reshape(self.n_depth, self.n_levels)

    def planck(self) -> np.ndarray:
        return self.table(1, self.n_nu * self.n_depth).reshape(self.n_nu, self.n_depth)

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                self.ctx.lib.jfnk_destroy_atmosphere(self.h)
        except Exception:
            pass


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()   # torch tensor


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    return int(stream) if isinstance(stream, int) else stream.cuda_stream


# ---- host-array conveniences (numpy in, numpy out) ---------------------------

def residual(atm: Atmosphere, n, Jdag=None, precision: int = JFNK_FP64, want_J: bool = False,
             want_emergent: bool = False):
    n = _f64(n)
    Jd = None if Jdag is None else _f64(Jdag)
    F = np.zeros_like(n)
    J = np.zeros((atm.n_nu, atm.n_depth)) if want_J else None
    Ie = np.zeros((atm.n_nu, atm.n_mu)) if want_emergent else None
    check(atm.ctx.lib.jfnk_residual(atm.ctx.h, atm.h, precision, _ptr(n), _ptr(Jd), _ptr(F), _ptr(J),
                                    _ptr(Ie), JFNK_MEM_HOST, None), "jfnk_residual")
    return F, J, Ie


def jvp(atm: Atmosphere, n, v, Jdag=None, precision: int = JFNK_FP64):
    n, v = _f64(n), _f64(v)
    Jd = None if Jdag is None else _f64(Jdag)
    out = np.zeros_like(n)
    check(atm.ctx.lib.jfnk_jvp(atm.ctx.h, atm.h, precision, _ptr(n), _ptr(Jd), _ptr(v), _ptr(out),
                               JFNK_MEM_HOST, None), "jfnk_jvp")
    return out


def block_jacobi(atm: Atmosphere, n, Jdag=None, precision: int = JFNK_FP64):
    n = _f64(n)
    Jd = None if Jdag is None else _f64(Jdag)
    P = np.zeros((atm.n_depth, atm.n_levels, atm.n_levels))
    check(atm.ctx.lib.jfnk_block_jacobi(atm.ctx.h, atm.h, precision, _ptr(n), _ptr(Jd), _ptr(P),
                                        JFNK_MEM_HOST, None), "jfnk_block_jacobi")
    return P


def block_jacobi_variant(atm: Atmosphere, n, variant: int, Jdag=None, dJdn_prev=None,
                         precision: int = JFNK_FP64):
    """Preconditioner blocks of solution ``variant`` of Sect. 2.5.2; returns
    (P [nz, nl, nl], the renewed lagged d J/d n [nq, nz, nl] for variant 2)."""
    n = _f64(n)
    P = np.zeros((atm.n_depth, atm.n_levels, atm.n_levels))
    D = np.zeros((atm.n_nu, atm.n_depth, atm.n_levels)) if variant == 2 else None
    Dp = None if dJdn_prev is None else _f64(dJdn_prev)
    check(atm.ctx.lib.jfnk_block_jacobi_variant(atm.ctx.h, atm.h, precision, variant, _ptr(n),
                                                _ptr(None if Jdag is None else _f64(Jdag)), _ptr(Dp),
                                                _ptr(P), _ptr(D), JFNK_MEM_HOST, None),
          "jfnk_block_jacobi_variant")
    return P, D


def rh92_update(atm: Atmosphere, n, Jdag=None, precision: int = JFNK_FP64):
    n = _f64(n)
    Jd = None if Jdag is None else _f64(Jdag)
    out = np.zeros_like(n)
    J = np.zeros((atm.n_nu, atm.n_depth))
    check(atm.ctx.lib.jfnk_rh92_update(atm.ctx.h, atm.h, precision, _ptr(n), _ptr(Jd), _ptr(out),
                                       _ptr(J), JFNK_MEM_HOST, None), "jfnk_rh92_update")
    return out, J


def solve(atm: Atmosphere, opts: Optional[jfnk_options] = None, n0=None, J0=None, raise_on_fail=True):
    """Algorithm 2 on the device; returns (n, J, stats). J0 defaults to B_nu(T)."""
    o = opts or default_options()
    n = np.zeros((atm.n_depth, atm.n_levels)) if n0 is None else _f64(n0).copy()
    if n0 is not None:
        o.init = JFNK_INIT_USER
    J = atm.planck() if J0 is None else _f64(J0).copy()
    st = jfnk_stats()
    rc = atm.ctx.lib.jfnk_solve(atm.ctx.h, atm.h, C.byref(o), _ptr(n), _ptr(J), C.byref(st),
                                JFNK_MEM_HOST, None)
    if raise_on_fail:
        check(rc, "jfnk_solve")
    return n, J, st.as_dict()


def probe_alu(ctx: Context, kind: int) -> float:
    v = C.c_double()
    check(ctx.lib.jfnk_probe_alu(ctx.h, kind, C.byref(v)), "jfnk_probe_alu")
    return v.value


ARITH_OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "acc": 4}


def check_arith(ctx: Context, op: str, a, b):
    """The library's float-pair arithmetic on a, b (its accuracy test)."""
    a, b = _f64(a).ravel(), _f64(b).ravel()
    out = np.zeros_like(a)
    check(ctx.lib.jfnk_check_arith(ctx.h, ARITH_OPS[op], _ptr(a), _ptr(b), _ptr(out), a.size),
          "jfnk_check_arith")
    return out


def batch_solve(ctx: Context, atms: Sequence[Atmosphere], opts: Optional[jfnk_options] = None,
                raise_on_fail=True):
    o = opts or default_options()
    nc = len(atms)
    ns = [np.zeros((a.n_depth, a.n_levels)) for a in atms]
    hs = (C.c_void_p * nc)(*[a.h for a in atms])
    nps = (C.c_void_p * nc)(*[n.ctypes.data for n in ns])
    stats = (jfnk_stats * nc)()
    rc = ctx.lib.jfnk_batch_solve(ctx.h, nc, hs, C.byref(o), nps, None, stats, JFNK_MEM_HOST, None)
    if raise_on_fail:
        check(rc, "jfnk_batch_solve")
    return ns, [s.as_dict() for s in stats]


class BatchPlan:
    """Persistent batch of columns (jfnk_batch_*): buffers, tuning and graph built once."""

    def __init__(self, ctx: Context, atms: Sequence[Atmosphere], precision: int = JFNK_FP64,
                 krylov_max: int = 50):
        self.ctx, self.atms, self.precision = ctx, list(atms), precision
        nc = len(self.atms)
        self._hs = (C.c_void_p * nc)(*[a.h for a in self.atms])
        h = C.c_void_p()
        check(ctx.lib.jfnk_batch_create(ctx.h, nc, self._hs, precision, krylov_max, C.byref(h)),
              "jfnk_batch_create")
        self.h = h
        self.ns = [np.zeros((a.n_depth, a.n_levels)) for a in self.atms]
        self._nps = (C.c_void_p * nc)(*[n.ctypes.data for n in self.ns])
        self.stats = (jfnk_stats * nc)()

    def run(self, opts: Optional[jfnk_options] = None, raise_on_fail: bool = True, stream=None):
        o = opts or default_options(precision=self.precision)
        o.precision = self.precision
        rc = self.ctx.lib.jfnk_batch_run(self.h, C.byref(o), self._nps, None, self.stats,
                                         JFNK_MEM_HOST, _stream(stream))
        if raise_on_fail:
            check(rc, "jfnk_batch_run")
        return self.ns, [s.as_dict() for s in self.stats]

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.lib.jfnk_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (jfnk_server_*): columns are submitted
    as they arrive, admitted into free slots when their work buffers fit in the
    server's device pool, and advanced together one captured tick graph per
    step. Results carry submission, admission and completion times on the
    server clock."""

    def __init__(self, ctx: Context, max_slots: int, max_depth: int, max_freq: int, max_levels: int = 6,
                 max_trans: int = 16, max_mu: int = 5, mem_bytes: int = 0,
                 opts: Optional[jfnk_options] = None):
        self.ctx = ctx
        d = jfnk_server_desc(max_slots=max_slots, max_depth=max_depth, max_freq=max_freq,
                             max_levels=max_levels, max_trans=max_trans, max_mu=max_mu,
                             mem_bytes=mem_bytes)
        d.opts = opts or default_options(precision=JFNK_MIXED)
        self.h = None
        h = C.c_void_p()
        check(ctx.lib.jfnk_server_create(ctx.h, C.byref(d), C.byref(h)), "jfnk_server_create")
        self.h = h
        self._pending = {}   # id -> (atmosphere, populations buffer)
        self._res = (jfnk_result * 256)()

    def bytes(self, atm: "Atmosphere") -> int:
        v = C.c_size_t()
        check(self.ctx.lib.jfnk_server_bytes(self.h, atm.h, C.byref(v)), "jfnk_server_bytes")
        return v.value

    def submit(self, atm: "Atmosphere", rid: int, opts: Optional[jfnk_options] = None) -> None:
        n = np.zeros((atm.n_depth, atm.n_levels))
        check(self.ctx.lib.jfnk_server_submit(self.h, atm.h, rid, n.ctypes.data,
                                              C.byref(opts) if opts is not None else None),
              "jfnk_server_submit")
        self._pending[rid] = (atm, n)

    def step(self):
        a, q = C.c_int(), C.c_int()
        check(self.ctx.lib.jfnk_server_step(self.h, C.byref(a), C.byref(q)), "jfnk_server_step")
        return a.value, q.value

    def poll(self):
        """Finished requests as dicts (id, status, stats, times, n)."""
        out = []
        while True:
            k = C.c_int()
            check(self.ctx.lib.jfnk_server_poll(self.h, self._res, len(self._res), C.byref(k)),
                  "jfnk_server_poll")
            for i in range(k.value):
                r = self._res[i]
                _, n = self._pending.pop(r.id)
                out.append(dict(id=r.id, status=r.status, stats=r.stats.as_dict(), t_submit=r.t_submit,
                                t_admit=r.t_admit, t_done=r.t_done, n=n))
            if k.value < len(self._res):
                return out

    def clock(self) -> float:
        return self.ctx.lib.jfnk_server_clock(self.h)

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.lib.jfnk_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
