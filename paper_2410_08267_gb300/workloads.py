"""Seeded synthetic workloads for relic-overdensity profiles.

This module only draws input parameters (cosmologies, halo masses and
concentrations, relic masses, radius lists, grid sizes, request arrival
times).  It contains none of the method's arithmetic: halo radii, the
background, the force, the integrator and the quadrature live in the CUDA
library and, independently, in the oracle.  Both consume the ``Problem``
records built here.

Workload recipes follow the shapes of the paper's use (Sec. II.D: a radius
list, a momentum grid and a direction grid per halo and relic mass; Sec. IV:
halo-growth, relic-distribution and coupling variants).  The paper uses no
public dataset; every input is synthetic and seeded.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# Halo-growth kinds (Eq. rhototal modulation xi(z), Sec. IV.A)
XI_STATIC, XI_LINEAR, XI_EXP = 0, 1, 2
# Coupling kinds (G -> kappa(z) G, Sec. IV.B)
KAPPA_ONE, KAPPA_POW1PZ, KAPPA_PAPER, KAPPA_CONST = 0, 1, 2, 3
# Relic distribution kinds (Sec. II.C, Sec. IV.B)
F_FD, F_FREEZEIN, F_TABLE = 0, 1, 2
# Radius units
RADII_KPC, RADII_R200 = 0, 1
# Precision modes
FP64, MIXED = 0, 1


@dataclass
class Problem:
    """One overdensity-profile request: one halo, one relic, one radius list."""
    Om: float = 0.31
    h: float = 0.67
    T0_K: float = 1.95
    M_h: float = 1e12
    c: float = 10.0
    z0: float = 0.0
    xi_kind: int = XI_LINEAR
    xi_p: tuple = (1.0, 0.0, 0.0)          # alpha, z_start (0 = z_i), z_stop (0 = z0)
    kappa_kind: int = KAPPA_ONE
    kappa_p: tuple = (0.0, 0.0, 0.0)
    m_eV: float = 0.1
    f_kind: int = F_FD
    f_p: tuple = (0.0, 0.0)                # FD chemical potential eta; table: q range
    f_table: tuple = ()                    # F_TABLE: f at log-spaced q from f_p[0] to f_p[1]
    radii: np.ndarray = field(default_factory=lambda: np.geomspace(1.0, 300.0, 10))
    radii_unit: int = RADII_KPC
    n_q: int = 50
    q_min: float = 0.01
    q_max: float = 10.0
    n_mu: int = 20
    n_steps: int = 400
    z_end: float = 4.0
    precision: int = MIXED
    masses: tuple = ()                     # mass reuse: relic masses read from the
                                           # trajectories of the fiducial m_eV

    @property
    def n_radii(self) -> int:
        return int(len(self.radii))

    @property
    def n_out(self) -> int:
        """Result values: radii x masses."""
        return self.n_radii * max(1, len(self.masses))

    @property
    def n_traj(self) -> int:
        return self.n_radii * self.n_q * self.n_mu

    @property
    def traj_steps(self) -> int:
        return self.n_traj * self.n_steps

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def c_of_M(M: float) -> float:
    """Concentration-mass power law used by the workload recipes: c = 9 (M/1e12)^-0.1."""
    return 9.0 * (M / 1e12) ** -0.1


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def plain_small(precision: int = FP64) -> List[Problem]:
    """Flat LCDM (Om=0.31, h=0.67), one static NFW halo 1e12 Msun with c=10,
    m=0.1 eV Fermi-Dirac relic, 10 radii log 1-300 kpc, 50 log q in 0.01-10,
    20 Gauss-Legendre mu, z 0->4 in 400 RK4 steps: 10^4 trajectories."""
    return [Problem(M_h=1e12, c=10.0, xi_kind=XI_STATIC, m_eV=0.1,
                    radii=np.geomspace(1.0, 300.0, 10), n_q=50, q_min=0.01, q_max=10.0,
                    n_mu=20, n_steps=400, z_end=4.0, precision=precision)]


PRECISION_SWEEP_MASSES = (0.01, 0.05, 0.1, 0.3)


def precision_sweep(precision: int = MIXED, masses=PRECISION_SWEEP_MASSES,
                    n_radii: int = 64, n_q: int = 200, n_mu: int = 64,
                    n_steps: int = 800) -> List[Problem]:
    """NFW halo 1e13 Msun, c from the c-M law, mass history M0 exp(-0.8 z),
    four relic masses, 64 radii log 1 kpc - 1 Mpc, 200 log q x 64 GL mu
    (about 3.3M trajectories), z 0->4 in 800 steps."""
    M = 1e13
    return [Problem(M_h=M, c=c_of_M(M), xi_kind=XI_EXP, xi_p=(0.8, 0.0, 0.0), m_eV=m,
                    radii=np.geomspace(1.0, 1000.0, n_radii), n_q=n_q, q_min=0.01,
                    q_max=10.0, n_mu=n_mu, n_steps=n_steps, z_end=4.0, precision=precision)
            for m in masses]


def precision_sweep_reuse(precision: int = MIXED, masses=PRECISION_SWEEP_MASSES,
                          n_radii: int = 64, n_mu: int = 64, n_steps: int = 800) -> Problem:
    """The precision sweep as ONE mass-reuse request (Sec. III): trajectories
    for the heaviest mass, read for every mass.  Each mass's own 0.01-10 k_B T0
    range maps to 0.01 (m_fid/m) .. 10 (m_fid/m) on the fiducial grid, so the
    grid spans the union, log-spaced at the per-mass density (200 nodes per
    three decades)."""
    m_fid = max(masses)
    q_min, q_max = 0.01, 10.0 * m_fid / min(masses)
    n_q = int(round(200 * np.log10(q_max / q_min) / 3.0))
    M = 1e13
    return Problem(M_h=M, c=c_of_M(M), xi_kind=XI_EXP, xi_p=(0.8, 0.0, 0.0), m_eV=m_fid,
                   radii=np.geomspace(1.0, 1000.0, n_radii), n_q=n_q, q_min=q_min,
                   q_max=q_max, n_mu=n_mu, n_steps=n_steps, z_end=4.0, precision=precision,
                   masses=tuple(masses))


def paper_production_grid(precision: int = MIXED, n_steps: int = 800) -> Problem:
    """The production grid of Sec. III as one mass-reuse request: 20 radii
    log 10 kpc - 50 Mpc, 200 momenta log 0.01-400 k_B T0 for the fiducial
    0.3 eV relic, 10 directions (Gauss-Legendre on [-1, 1] here) and 15 masses
    linear in 0.01-0.5 eV read from one trajectory set; a 1e12 Msun halo with
    the c-M law and linear growth, integrated back to z_i.  The step count is
    not stated in the paper (800 here)."""
    M = 1e12
    return Problem(M_h=M, c=c_of_M(M), xi_kind=XI_LINEAR, xi_p=(1.0, 0.0, 0.0), m_eV=0.3,
                   radii=np.geomspace(10.0, 50000.0, 20), n_q=200, q_min=0.01, q_max=400.0,
                   n_mu=10, n_steps=n_steps, z_end=0.0, precision=precision,
                   masses=tuple(float(m) for m in np.linspace(0.01, 0.5, 15)))


def batched_uneven(n_halos: int = 1024, seed: int = 2410, precision: int = MIXED,
                   n_steps: int = 400) -> List[Problem]:
    """1024 halos: log10 M ~ U[11,15], c lognormal (0.15 dex) about the c-M law,
    radius count ~ U{8..128} log-spaced 1e-3 r200 - 2 r200 (given in units of
    r200, converted by each implementation), n_q ~ U{32..256},
    n_mu ~ U{16..64}, m ~ U[0.01,0.3] eV, linear growth (paper default)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_halos):
        lgM = rng.uniform(11.0, 15.0)
        M = 10.0 ** lgM
        c = c_of_M(M) * 10.0 ** rng.normal(0.0, 0.15)
        nr = int(rng.integers(8, 129))
        nq = int(rng.integers(32, 257))
        nmu = int(rng.integers(16, 65))
        m = rng.uniform(0.01, 0.3)
        # Radii are given in units of r200, which only the implementations
        # compute; the recipe's 0.5 kpc inner end becomes a fixed 1e-3 r200
        # (0.15 kpc at 1e11 Msun, 3 kpc at 1e15 Msun).
        radii = np.geomspace(1e-3, 2.0, nr)
        out.append(Problem(M_h=M, c=c, xi_kind=XI_LINEAR, xi_p=(1.0, 0.0, 0.0), m_eV=m,
                           radii=radii, radii_unit=RADII_R200, n_q=nq, q_min=0.01,
                           q_max=10.0, n_mu=nmu, n_steps=n_steps, z_end=4.0,
                           precision=precision))
    return out


def new_physics(n_halos: int = 256, seed: int = 2411, precision: int = MIXED,
                n_radii: int = 128, n_q: int = 256, n_mu: int = 64,
                n_steps: int = 400) -> List[Problem]:
    """256 halos drawn as in the uneven batch; each halo gets one variant from
    {FD eta in {-1,0,1}, freeze-in q^-1/2 e^-q with m in [1,10] keV log-uniform}
    and a coupling G(a) = G0 a^-gamma with gamma in {0, 0.01, 0.05}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_halos):
        M = 10.0 ** rng.uniform(11.0, 15.0)
        c = c_of_M(M) * 10.0 ** rng.normal(0.0, 0.15)
        gamma = (0.0, 0.01, 0.05)[int(rng.integers(0, 3))]
        variant = int(rng.integers(0, 4))
        if variant < 3:
            f_kind, f_p, m = F_FD, (float(variant - 1), 0.0), rng.uniform(0.01, 0.3)
        else:
            f_kind, f_p, m = F_FREEZEIN, (0.0, 0.0), 10.0 ** rng.uniform(3.0, 4.0)
        out.append(Problem(M_h=M, c=c, xi_kind=XI_LINEAR, kappa_kind=KAPPA_POW1PZ,
                           kappa_p=(gamma, 0.0, 0.0), m_eV=m, f_kind=f_kind, f_p=f_p,
                           radii=np.geomspace(1e-3, 2.0, n_radii), radii_unit=RADII_R200,
                           n_q=n_q, q_min=0.01, q_max=10.0, n_mu=n_mu, n_steps=n_steps,
                           z_end=4.0, precision=precision))
    return out


def spectral_distortions(n_table: int = 512, q_first: float = 1e-3, q_last: float = 40.0):
    """Tabulated relic distributions of the kinds Sec. IV.B explores (the
    paper prints no formulas or parameters; these shapes are stand-ins):
    a thermal spectrum at 0.8 T0 with a Gaussian bump at q = 5, and a cold
    Fermi gas falling off faster than Fermi-Dirac above q = 3.  Returns
    {name: (f_p, f_table)} for the F_TABLE kind."""
    q = np.geomspace(q_first, q_last, n_table)
    bump = 1.0 / (1.0 + np.exp(q / 0.8)) + 0.05 * np.exp(-0.5 * (q - 5.0) ** 2)
    cold = 1.0 / (1.0 + np.exp((q - 3.0) / 0.3))
    return {"thermal_bump": ((q_first, q_last), tuple(float(v) for v in bump)),
            "cold_fermi_gas": ((q_first, q_last), tuple(float(v) for v in cold))}


SERVING_GRIDS = ((64, 16), (128, 32), (256, 64))


@dataclass
class Request:
    t_arrival: float          # seconds from stream start
    problem: Problem


def serving_stream(rate: float, n_requests: int, seed: int = 2412,
                   precision: int = MIXED, n_steps: int = 400,
                   max_radii: int = 256) -> List[Request]:
    """Poisson request stream: Om ~ U[.28,.34], h ~ U[.64,.72],
    log10 M ~ U[11,15] (c from the c-M law), m ~ U[0.01,0.5] eV,
    radius count ~ U{4..256} (log 1e-3..2 r200), grid from
    {64x16, 128x32, 256x64}."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate)
        M = 10.0 ** rng.uniform(11.0, 15.0)
        nq, nmu = SERVING_GRIDS[int(rng.integers(0, 3))]
        nr = int(rng.integers(4, max_radii + 1))
        p = Problem(Om=rng.uniform(0.28, 0.34), h=rng.uniform(0.64, 0.72), M_h=M,
                    c=c_of_M(M), xi_kind=XI_LINEAR, m_eV=rng.uniform(0.01, 0.5),
                    radii=np.geomspace(1e-3, 2.0, nr), radii_unit=RADII_R200,
                    n_q=nq, q_min=0.01, q_max=10.0, n_mu=nmu, n_steps=n_steps,
                    z_end=4.0, precision=precision)
        out.append(Request(t, p))
    return out


def subsample(problems: List[Problem], every: int) -> List[Problem]:
    """Every ``every``-th problem (seed-fixed subsample for oracle checks)."""
    return problems[::every]


def random_small(seed: int, n: int = 8, precision: int = FP64) -> List[Problem]:
    """Small mixed problems spanning every kind, for parity tests that must
    finish quickly on the oracle: a few radii, ragged grids, short step counts."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        M = 10.0 ** rng.uniform(11.0, 15.0)
        xi_kind = int(rng.integers(0, 3))
        xi_p = {XI_STATIC: (1.0, 0.0, 0.0), XI_LINEAR: (float(rng.choice([0.5, 1.0, 2.0])), 0.0, 0.0),
                XI_EXP: (0.8, 0.0, 0.0)}[xi_kind]
        kappa_kind = int(rng.integers(0, 4))
        kappa_p = {KAPPA_ONE: (0.0, 0.0, 0.0), KAPPA_POW1PZ: (0.05, 0.0, 0.0),
                   KAPPA_PAPER: (0.2, 1.5, 0.0), KAPPA_CONST: (1.1, 0.0, 0.0)}[kappa_kind]
        f_kind = int(rng.integers(0, 2))
        # the non-thermal shape is drawn at neutrino-like masses here (as in the
        # paper's freeze-in example at 0.3 eV), where a q grid of 0.01-10 T0
        # covers today's phase space
        m = rng.uniform(0.01, 0.5) if f_kind == F_FD else rng.uniform(0.05, 1.0)
        out.append(Problem(Om=rng.uniform(0.28, 0.34), h=rng.uniform(0.64, 0.72), M_h=M,
                           c=c_of_M(M) * 10.0 ** rng.normal(0.0, 0.15), xi_kind=xi_kind,
                           xi_p=xi_p, kappa_kind=kappa_kind, kappa_p=kappa_p, m_eV=m,
                           f_kind=f_kind, f_p=(float(rng.integers(-1, 2)), 0.0),
                           radii=np.geomspace(1e-3, 2.0, int(rng.integers(1, 6))),
                           radii_unit=RADII_R200, n_q=int(rng.integers(2, 40)),
                           q_min=0.01, q_max=10.0, n_mu=int(rng.integers(1, 24)),
                           n_steps=int(rng.integers(60, 200)), z_end=4.0,
                           precision=precision))
    return out
