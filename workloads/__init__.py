"""Seeded synthetic inputs shaped like the workloads of the paper (Sect. 3.1).

The paper solves its NLTE problems on the FAL-C atmosphere (82 depth points)
with model atoms of Ca II and H I (Sect. 3.1, Table 1). Neither data set is
available here, so this module builds seeded stand-ins with the same shapes:
chromosphere-like columns of 82 depths, six-level atoms with about 1,000 and
2,000 frequencies, the isothermal two-level slab of the sqrt(eps) law, a batch
of 4,096 perturbed columns and a Poisson stream of mixed column solves.

Only input recipes live here: level energies and weights, transition
parameters, frequency-grid parameters, collision parameters and the depth
structure of each column. Nothing of the residual, of the formal solution, of
the rate integrals or of the solvers is computed in this module; the CUDA
library and the CPU oracle each build their own tables from these
descriptors.

Frequency-grid rule shared by both consumers (a documented input convention,
implemented independently on each side):
  * bound-bound line with ``n_nu`` points (odd), ``q_core``, ``q_wing``:
    offsets x_s, s = 0..n_nu-1, u_s = 2 s/(n_nu-1) - 1 in [-1, 1];
    if q_wing <= 2 q_core: x = q_wing * u (uniform);
    else: beta = 2 acosh(q_wing / (2 q_core)), x = q_wing sinh(beta u)/sinh(beta)
    (half of the points then fall inside +-q_core);
    nu_s = nu_0 (1 + x_s * vchar / c).
  * bound-free continuum with ``n_nu`` points and ``y_max``:
    nu_s = nu_edge * y_max ** (s / (n_nu - 1)), s = 0..n_nu-1.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

# cgs constants used only to shape the inputs (thermal speeds, hydrostatics,
# the optical-depth scale of the two-level slab).
_KB = 1.380649e-16
_AMU = 1.66053906660e-24
_MH = 1.6735575e-24
_GSUN = 2.74e4
_H = 6.62607015e-27
_C = 2.99792458e10
_ME = 9.1093837015e-28
_QE = 4.80320471e-10
_EV = 1.602176634e-12


@dataclass(frozen=True)
class Line:
    """Bound-bound transition i -> j (0-based, i < j)."""
    i: int
    j: int
    f: float                 # absorption oscillator strength
    damping: float           # Voigt damping parameter a (depth independent)
    upsilon: float = 0.0     # effective collision strength
    eps: float = 0.0         # > 0: two-level thermalisation parameter (overrides upsilon)
    n_nu: int = 101          # frequency points (odd)
    q_core: float = 3.0      # core half-width [reference Doppler widths]
    q_wing: float = 30.0     # window half-width [reference Doppler widths]


@dataclass(frozen=True)
class Continuum:
    """Bound-free transition from bound level i to continuum level j."""
    i: int
    j: int
    alpha0: float            # photo-ionisation cross-section at the edge [cm^2]
    q0: float                # collisional ionisation coefficient [cm^3 s^-1 K^-1/2]
    n_nu: int = 40
    y_max: float = 2.0       # nu_max / nu_edge


@dataclass
class Atom:
    name: str
    E_eV: np.ndarray         # level energies above the ground level [eV]
    g: np.ndarray            # statistical weights
    stage: np.ndarray        # ionisation stage of each level
    lines: List[Line]
    conts: List[Continuum]
    mass_amu: float
    vchar: float             # reference velocity of the line grids [cm/s]

    @property
    def n_levels(self) -> int:
        return len(self.E_eV)

    @property
    def n_transitions(self) -> int:
        return len(self.lines) + len(self.conts)


@dataclass
class Column:
    """One plane-parallel column, depth index 0 at the top."""
    z: np.ndarray            # height [cm], strictly decreasing with index
    T: np.ndarray            # temperature [K]
    ne: np.ndarray           # electron density [cm^-3]
    ntot: np.ndarray         # total density of the active atom [cm^-3]
    rho: np.ndarray          # mass density [g cm^-3]
    kappa: float = 0.0       # continuum opacity per unit mass at nu <= kappa_nu_ref [cm^2 g^-1]
    kappa_nu_ref: float = 0.0   # above this frequency kappa rises as (nu/kappa_nu_ref)^kappa_power [Hz]
    kappa_power: float = 0.0    # 0: grey background
    kappa_max: float = 1.0      # cap on the UV rise factor
    thomson: bool = False    # add electron scattering sigma_T n_e
    vturb: Optional[np.ndarray] = None  # micro-turbulence [cm/s]; None = 0
    vlos: Optional[np.ndarray] = None   # line-of-sight velocity [cm/s], > 0 upward (towards the top); None = static

    @property
    def n_depth(self) -> int:
        return len(self.z)


@dataclass
class Workload:
    name: str
    atom: Atom
    columns: List[Column]
    n_mu: int = 5
    precision: str = "fp64"      # "fp64" or "mixed"
    init: str = "lte"            # "lte", "zero_radiation" or "hybrid" (RH92 iterations first)
    arrivals: Optional[np.ndarray] = None   # serving stream only [s]
    atoms: Optional[List[Atom]] = field(default=None)  # serving stream: atom per request


def _odd(n: int) -> int:
    n = int(max(3, n))
    return n if n % 2 == 1 else n + 1


def _thermal_speed(T: float, mass_amu: float) -> float:
    return float(np.sqrt(2.0 * _KB * T / (mass_amu * _AMU)))


# ---------------------------------------------------------------------------
# Config 1: isothermal two-level slab of the sqrt(eps) law.
# ---------------------------------------------------------------------------

def two_level_atom(n_nu: int = 41, eps: float = 1e-4, T: float = 5000.0,
                   lam_nm: float = 500.0, f: float = 0.5,
                   mass_amu: float = 40.0) -> Atom:
    """Two-level atom with a pure Doppler line sampled uniformly on +-5 widths."""
    E_u = _H * _C / (lam_nm * 1e-7) / _EV
    line = Line(i=0, j=1, f=f, damping=0.0, eps=eps, n_nu=_odd(n_nu),
                q_core=5.0, q_wing=5.0)
    return Atom(name="two-level", E_eV=np.array([0.0, E_u]), g=np.array([2.0, 4.0]),
                stage=np.array([0, 0]), lines=[line], conts=[],
                mass_amu=mass_amu, vchar=_thermal_speed(T, mass_amu))


def two_level_slab(atom: Atom, n_depth: int = 101, tau_min: float = 1e-6,
                   tau_max: float = 1e4, T: float = 5000.0,
                   ntot: float = 1e10, ne: float = 1e12) -> Column:
    """Isothermal slab whose line-centre LTE optical depth is log-spaced.

    The height scale is set from a Gaussian line-centre opacity estimate
    (unnormalised profile 1/(sqrt(pi) dnu_D)); only the shape of the tau grid
    matters for the sqrt(eps) law.
    """
    ln = atom.lines[0]
    nu0 = (atom.E_eV[ln.j] - atom.E_eV[ln.i]) * _EV / _H
    x = _H * nu0 / (_KB * T)
    gl, gu = atom.g[ln.i], atom.g[ln.j]
    nl = ntot * gl / (gl + gu * np.exp(-x))
    dnud = nu0 * atom.vchar / _C
    chi0 = (np.pi * _QE ** 2 / (_ME * _C)) * ln.f * nl * (1.0 - np.exp(-x)) / (np.sqrt(np.pi) * dnud)
    tau = np.logspace(np.log10(tau_min), np.log10(tau_max), n_depth)
    z = -tau / chi0
    ones = np.ones(n_depth)
    return Column(z=z, T=T * ones, ne=ne * ones, ntot=ntot * ones, rho=1e-12 * ones,
                  kappa=0.0, thomson=False)


def config1(n_depth: int = 101, n_nu: int = 41) -> Workload:
    atom = two_level_atom(n_nu=n_nu)
    return Workload(name="two-level isothermal slab (sqrt-eps)", atom=atom,
                    columns=[two_level_slab(atom, n_depth=n_depth)], n_mu=5,
                    precision="fp64", init="lte")


# ---------------------------------------------------------------------------
# Chromosphere-like column (stand-in for FAL-C).
# ---------------------------------------------------------------------------

_T_NODES = np.array([[-5.0, 1e5], [-4.6, 2.5e4], [-4.4, 8000.0], [-3.0, 6500.0],
                     [-0.7, 4400.0], [1.0, 9400.0]])


def chromosphere(n_depth: int = 82, m_top: float = 1e-5, m_bot: float = 10.0,
                 rng: Optional[np.random.Generator] = None, t_sigma: float = 0.0,
                 abundance: float = 2.2e-6, noise: str = "nodes") -> Column:
    """Hydrostatic column log-spaced in column mass.

    log T is piecewise linear in x = log10 m through fixed nodes (1e5 K at the
    top, a 4,400 K minimum, 9,400 K at the bottom). With t_sigma > 0 the
    profile is perturbed by exp(N(0, t_sigma^2)): on each node (``noise="nodes"``,
    a smooth perturbed profile) or on every depth point (``noise="depth"``);
    log10 n_e = 9 + (x + 5); p = g m;
    n_H = (p/kT - n_e)/1.1; rho = 1.4 m_H n_H; z from dz = dm / rho.

    Background continuum: kappa(nu) = 1 cm^2/g up to 400 nm, rising as
    (nu/nu_400)^6 into the UV and capped at 1e3 cm^2/g, a stand-in for the
    bound-free opacity of H- and metals that makes the UV continua form in the
    upper photosphere as they do in the Sun (a grey background leaves them
    optically thin down to the temperature minimum and gives departure
    coefficients of 1e5; an uncapped rise makes the 1e5 K top layers emit
    like a hot blackbody in the far UV).
    """
    m = np.logspace(np.log10(m_top), np.log10(m_bot), n_depth)
    x = np.log10(m)
    nodes_T = _T_NODES[:, 1].copy()
    if t_sigma > 0.0 and noise == "nodes":
        assert rng is not None
        nodes_T = nodes_T * np.exp(rng.normal(0.0, t_sigma, size=len(nodes_T)))
    logT = np.interp(x, _T_NODES[:, 0], np.log10(nodes_T))
    T = 10.0 ** logT
    if t_sigma > 0.0 and noise == "depth":
        assert rng is not None
        T = T * np.exp(rng.normal(0.0, t_sigma, size=n_depth))
    ne = 10.0 ** (9.0 + (x + 5.0))
    p = _GSUN * m
    nH = (p / (_KB * T) - ne) / 1.1
    rho = 1.4 * _MH * nH
    z = np.zeros(n_depth)
    for k in range(1, n_depth):
        z[k] = z[k - 1] - (m[k] - m[k - 1]) * 0.5 * (1.0 / rho[k - 1] + 1.0 / rho[k])
    return Column(z=z, T=T, ne=ne, ntot=abundance * nH, rho=rho, kappa=1.0,
                  kappa_nu_ref=_C / 400e-7, kappa_power=6.0, kappa_max=1e3, thomson=True)


def optimized_depth_grid(col: Column, n_depth: Optional[int] = None, wt_tau: float = 1.0,
                         wt_T: float = 1.0, wt_v: float = 1.0, v_scale: float = 2e5) -> Column:
    """Depth grid that places points where the column's structure changes
    (Sect. 3.4, after the depth optimisation of the Multi code extended to
    velocity gradients): the new points equidistribute the arc length of
    (wt_tau log10 m, wt_T log10 T, wt_v v / v_scale) along the old grid (m the
    column mass, standing in for the optical depth scale), with the same number
    of points unless ``n_depth`` is given; every quantity is interpolated
    linearly in the old depth index. An input recipe: both the library and the
    oracle receive the re-gridded column."""
    nz = col.n_depth if n_depth is None else int(n_depth)
    m = np.cumsum(np.concatenate([[0.0], 0.5 * (col.rho[1:] + col.rho[:-1]) * np.abs(np.diff(col.z))]))
    m = m + max(m[1], 1e-30)                       # strictly positive column mass
    v = np.zeros(col.n_depth) if col.vlos is None else col.vlos
    feats = np.stack([wt_tau * np.log10(m), wt_T * np.log10(col.T), wt_v * v / v_scale], axis=1)
    arc = np.concatenate([[0.0], np.cumsum(np.sqrt(np.sum(np.diff(feats, axis=0) ** 2, axis=1)))])
    target = np.linspace(0.0, arc[-1], nz)
    idx = np.interp(target, arc, np.arange(col.n_depth))    # fractional old index of each new point

    def lin(a):
        return None if a is None else np.interp(idx, np.arange(col.n_depth), a)

    return replace(col, z=lin(col.z), T=lin(col.T), ne=lin(col.ne), ntot=lin(col.ntot), rho=lin(col.rho),
                   vturb=lin(col.vturb), vlos=lin(col.vlos))


def velocity_chromosphere(n_depth: int = 82, v_top: float = 6e5, x_jump: float = -3.8, width: float = 0.08,
                          abundance: float = 2.2e-6, optimize: bool = True) -> Column:
    """The synthetic chromosphere with a sharp line-of-sight velocity gradient
    at the base of the chromosphere (Sect. 3.4: a jump near the lower
    chromosphere, positive velocity above it): v = v_top / (1 + exp((x - x_jump)
    / width)) with x = log10 column mass, zero below the jump; then re-gridded
    by ``optimized_depth_grid`` so that the jump is resolved by several points."""
    base = chromosphere(4 * n_depth, abundance=abundance)
    x = np.log10(np.logspace(-5, 1, 4 * n_depth))
    v = v_top / (1.0 + np.exp((x - x_jump) / width))
    col = replace(base, vlos=v)
    return optimized_depth_grid(col, n_depth) if optimize else chromosphere(n_depth, abundance=abundance)


def config2_velocity(seed: int = 0, n_depth: int = 82, nu_scale: float = 1.0) -> Workload:
    """Config 2 with the velocity gradient of Sect. 3.4 (FP64)."""
    atom = ca_like_atom(seed, nu_scale)
    return Workload(name="Ca II-like 6-level, 82-depth chromosphere with a velocity gradient", atom=atom,
                    columns=[velocity_chromosphere(n_depth)], n_mu=5, precision="fp64", init="lte")


def _line_window(a: float) -> float:
    return 300.0 * a + 30.0


def ca_like_atom(seed: int = 0, nu_scale: float = 1.0) -> Atom:
    """Six-level Ca II-like atom: 5 bound levels + continuum at 11.9 eV."""
    rng = np.random.default_rng(seed)
    E = np.zeros(6)
    E[1:3] = np.sort(rng.uniform(1.5, 2.0, size=2))
    E[3:5] = np.sort(rng.uniform(3.0, 3.3, size=2))
    E[5] = 11.9
    g = np.array([2.0, 4.0, 6.0, 2.0, 4.0, 1.0])
    stage = np.array([1, 1, 1, 1, 1, 2])
    pairs = [(0, 3), (0, 4), (1, 3), (2, 4), (1, 4)]
    lines = []
    for (i, j) in pairs:
        f = 10.0 ** rng.uniform(-2.0, 0.0)
        a = 10.0 ** rng.uniform(-3.0, -1.0)
        ups = rng.uniform(0.1, 1.0)
        lines.append(Line(i=i, j=j, f=f, damping=a, upsilon=ups,
                          n_nu=_odd(161 * nu_scale), q_core=3.0, q_wing=_line_window(a)))
    conts = []
    for i in range(5):
        alpha0 = rng.uniform(1e-19, 1e-17)
        q0 = 10.0 ** rng.uniform(-11.0, -10.0)
        conts.append(Continuum(i=i, j=5, alpha0=alpha0, q0=q0,
                               n_nu=max(2, int(round(40 * nu_scale))), y_max=2.0))
    return Atom(name="Ca II-like", E_eV=E, g=g, stage=stage, lines=lines, conts=conts,
                mass_amu=40.08, vchar=_thermal_speed(6000.0, 40.08))


def h_like_atom(seed: int = 1, nu_scale: float = 1.0) -> Atom:
    """Six-level H I-like atom: n = 1..5 + continuum, all 10 lines, 5 continua.

    Oscillator strengths and edge cross-sections follow Kramers' hydrogenic
    approximations, f_nm = 32/(3^1.5 pi) n^-5 m^-3 (1/n^2 - 1/m^2)^-3 and
    alpha_n = 7.91e-18 n cm^2, each scaled by a seeded factor U(0.8, 1.25), and
    effective collision strengths grow with the lower level as in hydrogen,
    Upsilon = U(0.5, 2) n^4 / (m - n)^2, so that the level structure stays
    hydrogen-like (random f-values and weak collisions among the upper levels
    make the Balmer and Paschen lines lase and no method converges).
    """
    rng = np.random.default_rng(seed)
    n = np.arange(1, 6)
    E = np.concatenate([13.6 * (1.0 - 1.0 / n ** 2), [13.6]])
    g = np.concatenate([2.0 * n ** 2, [1.0]])
    stage = np.array([0, 0, 0, 0, 0, 1])
    lines = []
    for i in range(5):
        for j in range(i + 1, 5):
            nl, nu_ = i + 1.0, j + 1.0
            f_kr = 32.0 / (3.0 ** 1.5 * np.pi) / (nl ** 5 * nu_ ** 3) * (1.0 / nl ** 2 - 1.0 / nu_ ** 2) ** -3
            f = f_kr * rng.uniform(0.8, 1.25)
            a = 10.0 ** rng.uniform(-3.0, -1.0)
            ups = rng.uniform(0.5, 2.0) * nl ** 4 / (nu_ - nl) ** 2
            lines.append(Line(i=i, j=j, f=f, damping=a, upsilon=ups,
                              n_nu=_odd(171 * nu_scale), q_core=3.0, q_wing=_line_window(a)))
    conts = []
    for i in range(5):
        alpha0 = 7.91e-18 * (i + 1) * rng.uniform(0.8, 1.25)
        q0 = 10.0 ** rng.uniform(-11.0, -10.0)
        conts.append(Continuum(i=i, j=5, alpha0=alpha0, q0=q0,
                               n_nu=max(2, int(round(60 * nu_scale))), y_max=4.0))
    return Atom(name="H I-like", E_eV=E, g=g, stage=stage, lines=lines, conts=conts,
                mass_amu=1.008, vchar=_thermal_speed(6000.0, 1.008))


def config2(seed: int = 0, n_depth: int = 82, nu_scale: float = 1.0) -> Workload:
    atom = ca_like_atom(seed, nu_scale)
    return Workload(name="Ca II-like 6-level, 82-depth chromosphere", atom=atom,
                    columns=[chromosphere(n_depth, abundance=2.2e-6)], n_mu=5,
                    precision="fp64", init="lte")


def config3(seed: int = 1, n_depth: int = 82, nu_scale: float = 1.0,
            precision: str = "mixed") -> Workload:
    atom = h_like_atom(seed, nu_scale)
    return Workload(name="H I-like 6-level, 82-depth chromosphere", atom=atom,
                    columns=[chromosphere(n_depth, abundance=1.0)], n_mu=5,
                    precision=precision, init="hybrid")


def config4(n_columns: int = 4096, seed: int = 20240624, nz_min: int = 64,
            nz_max: int = 256, nu_scale: float = 1.0, noise: str = "nodes") -> Workload:
    """Batch of independent columns: uniform depth counts, T noise sigma = 5 %
    (on the temperature nodes by default; per depth point with noise="depth")."""
    rng = np.random.default_rng(seed)
    atom = ca_like_atom(0, nu_scale)
    nzs = rng.integers(nz_min, nz_max + 1, size=n_columns)
    cols = [chromosphere(int(nz), rng=rng, t_sigma=0.05, abundance=2.2e-6, noise=noise) for nz in nzs]
    return Workload(name="batched 1.5D Ca II-like columns", atom=atom, columns=cols,
                    n_mu=5, precision="mixed", init="lte")


def _base_nu_count(atom: Atom) -> int:
    return sum(l.n_nu for l in atom.lines) + sum(c.n_nu for c in atom.conts)


def config5(n_requests: int = 10000, rate: float = 2000.0, seed: int = 20240624,
            nz_min: int = 48, nz_max: int = 300, nnu_min: int = 500,
            nnu_max: int = 2000) -> Workload:
    """Poisson stream of column solves: 20 % two-level, 40 % Ca II-like, 40 % H I-like."""
    rng = np.random.default_rng(seed + 1)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    arrivals = np.cumsum(gaps)
    kinds = rng.choice(3, size=n_requests, p=[0.2, 0.4, 0.4])
    nzs = rng.integers(nz_min, nz_max + 1, size=n_requests)
    nnus = rng.integers(nnu_min, nnu_max + 1, size=n_requests)
    atoms, cols = [], []
    base_ca = _base_nu_count(ca_like_atom(0))
    base_h = _base_nu_count(h_like_atom(1))
    for r in range(n_requests):
        nz = int(nzs[r])
        if kinds[r] == 0:
            atom = two_level_atom(n_nu=int(rng.integers(41, 201)))
            col = two_level_slab(atom, n_depth=nz)
        elif kinds[r] == 1:
            atom = ca_like_atom(0, nu_scale=nnus[r] / base_ca)
            col = chromosphere(nz, abundance=2.2e-6)
        else:
            atom = h_like_atom(1, nu_scale=nnus[r] / base_h)
            col = chromosphere(nz, abundance=1.0)
        atoms.append(atom)
        cols.append(col)
    return Workload(name="serving stream of mixed column solves", atom=atoms[0],
                    columns=cols, n_mu=5, precision="mixed", init="lte",
                    arrivals=arrivals, atoms=atoms)


def perturbed_populations(nstar: np.ndarray, rng: np.random.Generator,
                          rel: float = 0.3) -> np.ndarray:
    """Populations log-normally scattered around a reference (parity inputs)."""
    return nstar * np.exp(rng.normal(0.0, rel, size=nstar.shape))


def dense_overlap_workload(n_depth: int = 24, n_nu_line: int = 21, n_nu_cont: int = 8,
                           seed: int = 11) -> Workload:
    """An eight-level atom whose 12 lines all overlap: three nearly degenerate
    lower levels (1e-5 eV apart) and four nearly degenerate upper levels near
    3 eV, every lower-upper pair a line, so that at the lines' common centre
    12 transitions are active at once (more than the eight a frequency's packed
    transition list holds); 7 continua to an ionised level at 11.9 eV overlap
    among themselves above their edges. Not a physical ion: it exercises the
    general per-frequency transition lists of the kernels."""
    rng = np.random.default_rng(seed)
    E = np.array([0.0, 1e-5, 2e-5, 3.0, 3.0 + 1e-5, 3.0 + 2e-5, 3.0 + 3e-5, 11.9])
    g = np.array([2.0, 2.0, 2.0, 4.0, 4.0, 4.0, 4.0, 1.0])
    stage = np.array([1, 1, 1, 1, 1, 1, 1, 2])
    lines = []
    for i in range(3):
        for j in range(3, 7):
            a = 10.0 ** rng.uniform(-3.0, -2.0)
            lines.append(Line(i=i, j=j, f=10.0 ** rng.uniform(-2.0, -0.5), damping=a,
                              upsilon=rng.uniform(0.2, 1.0), n_nu=_odd(n_nu_line), q_core=3.0, q_wing=30.0))
    conts = [Continuum(i=i, j=7, alpha0=rng.uniform(1e-19, 1e-18), q0=10.0 ** rng.uniform(-11.0, -10.0),
                       n_nu=n_nu_cont, y_max=2.0) for i in range(7)]
    atom = Atom(name="dense-overlap", E_eV=E, g=g, stage=stage, lines=lines, conts=conts,
                mass_amu=40.08, vchar=_thermal_speed(6000.0, 40.08))
    col = chromosphere(n_depth, m_top=1e-4, m_bot=1.0, abundance=2.2e-6)
    return Workload(name="dense overlap", atom=atom, columns=[col], n_mu=3)


def tiny_workload(n_depth: int = 6, n_nu_line: int = 5, n_nu_cont: int = 3,
                  seed: int = 7, two_level: bool = False) -> Workload:
    """Very small three-level (or two-level) problem for brute-force checks."""
    if two_level:
        atom = two_level_atom(n_nu=n_nu_line, eps=1e-2)
        return Workload(name="tiny two-level", atom=atom,
                        columns=[two_level_slab(atom, n_depth=n_depth, tau_max=1e2)], n_mu=2)
    rng = np.random.default_rng(seed)
    E = np.array([0.0, 3.1, 11.9])
    g = np.array([2.0, 4.0, 1.0])
    stage = np.array([1, 1, 2])
    a = 10.0 ** rng.uniform(-3, -1)
    lines = [Line(i=0, j=1, f=0.3, damping=a, upsilon=0.5, n_nu=_odd(n_nu_line),
                  q_core=3.0, q_wing=10.0)]
    conts = [Continuum(i=0, j=2, alpha0=5e-18, q0=3e-11, n_nu=n_nu_cont, y_max=1.5),
             Continuum(i=1, j=2, alpha0=2e-18, q0=3e-11, n_nu=n_nu_cont, y_max=1.5)]
    atom = Atom(name="tiny Ca-like", E_eV=E, g=g, stage=stage, lines=lines, conts=conts,
                mass_amu=40.08, vchar=_thermal_speed(6000.0, 40.08))
    col = chromosphere(n_depth, m_top=1e-4, m_bot=1.0, abundance=2.2e-6)
    return Workload(name="tiny three-level", atom=atom, columns=[col], n_mu=2)


__all__ = ["Line", "Continuum", "Atom", "Column", "Workload", "config1", "config2", "config2_velocity",
           "velocity_chromosphere", "optimized_depth_grid",
           "config3", "config4", "config5", "two_level_atom", "two_level_slab",
           "chromosphere", "ca_like_atom", "h_like_atom", "perturbed_populations",
           "tiny_workload", "dense_overlap_workload", "replace"]
