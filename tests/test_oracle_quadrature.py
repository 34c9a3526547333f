"""Independent pin of the oracle's quadrature assembly (Eq. density_integral,
Eq. localdensity; Sec. III for mass reuse).

The oracle forms n/nbar as a trapezoid rule in ln q with weights w_j q_j^3
and Gauss-Legendre weights in mu, divided by twice the background on the same
grid.  Here the same ratio is formed by a different rule from its definition,

    n/nbar = int_{-1}^{1} dmu int dP P^2 f(P_i(P, mu))  /  (2 int dP P^2 f(P)),

with adaptive quadrature in linear P (scipy.integrate.quad) and numpy's own
Gauss-Legendre nodes in mu, over the same momentum range.  The final momenta
P_i come from the oracle's integrator (pinned on its own in
test_oracle_pins.py); only the assembly is under test.  A case with strong
clustering at a well-conditioned radius (0.3 eV relic, 1e12 Msun halo,
300 kpc) separates the candidates: a P^2-for-P^3 slip in the ln-q measure
moves n/nbar by 3 % and dropped direction weights by 0.2 %, both far above
the 1e-4 agreement required.
"""
import warnings

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2410_08267_gb300 import workloads as W

TOL = 1e-4
X0 = 300.0    # kpc: outside the core, where the discrete map is well conditioned


def _case():
    return W.plain_small(precision=W.FP64)[0].replace(m_eV=0.3, M_h=1e12, radii=np.array([X0]),
                                                       n_steps=200)


def _fd(q):
    # Fermi-Dirac in q = P/(k_B T0) with zero chemical potential (Sec. II.C)
    return 1.0 / (1.0 + np.exp(q))


def _final_q(pb, q, mu):
    s = oracle.initial_state(pb, X0, q, mu)
    s = oracle.integrate(pb, s, 0.0, -np.log1p(pb.z_end), pb.n_steps)
    return oracle.final_q(pb, s)


def _independent(pb, n_mu=16, p_power=2, mu_weights=True, scale=1.0, epsrel=1e-6):
    """n/nbar by adaptive quadrature in linear q and numpy Gauss-Legendre in mu.
    scale = s_a reads the fiducial trajectories for mass s_a m (Sec. III): the
    mass-a momentum is s_a q, so both integrals take f(s_a .) and the common
    factor s_a^3 cancels."""
    mu, w = np.polynomial.legendre.leggauss(n_mu)
    if not mu_weights:
        w = np.full(n_mu, 2.0 / n_mu)
    num = 0.0
    for m_k, w_k in zip(mu, w):
        # P_i(P) has kinks where trajectories start or stop crossing the NFW
        # edge, so quad may report that it reached its subdivision limit; its
        # result still agrees with the finest oracle grids to ~5e-6
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", integrate.IntegrationWarning)
            val = integrate.quad(lambda q: q ** p_power * _fd(scale * _final_q(pb, q, m_k)),
                                 pb.q_min, pb.q_max, epsabs=0.0, epsrel=epsrel, limit=100)[0]
        num += w_k * val
    den = integrate.quad(lambda q: q ** p_power * _fd(scale * q), pb.q_min, pb.q_max,
                         epsabs=0.0, epsrel=1e-12, limit=200)[0]
    return num / (2.0 * den)


@pytest.fixture(scope="module")
def independent_value():
    return _independent(_case())


def test_profile_assembly_matches_an_independent_quadrature(independent_value):
    pb = _case()
    errs = []
    for n_q, n_mu in ((100, 24), (400, 48), (800, 64)):
        got = oracle.profile(pb.replace(n_q=n_q, n_mu=n_mu))[0]
        errs.append(abs(got - independent_value) / independent_value)
    print("oracle vs independent quadrature, grids 100x24, 400x48, 800x64:", errs)
    assert independent_value > 1.1            # the case clusters strongly
    assert errs[-1] < TOL
    assert errs[-1] < errs[0]                 # refining the oracle's grid approaches it


def test_mass_reuse_assembly_matches_an_independent_quadrature():
    pb = _case().replace(n_q=800, n_mu=64)
    masses = [0.1, 0.01, 0.3]
    got = oracle.profile_masses(pb, masses)[:, 0]
    for m_a, g in zip(masses, got):
        ref = _independent(pb, scale=m_a / pb.m_eV)
        assert abs(g - ref) / ref < TOL, (m_a, g, ref)


def test_assembly_slips_are_caught(independent_value):
    """The pin has the power the module docstring claims: the assembly with a
    P^2-for-P^3 slip, or without the direction weights, lands far outside the
    tolerance of the correct oracle value."""
    pb = _case()
    good = oracle.profile(pb.replace(n_q=800, n_mu=64))[0]
    slip_q = _independent(pb, p_power=1, epsrel=1e-4)
    slip_mu = _independent(pb, mu_weights=False, epsrel=1e-4)
    assert abs(slip_q - good) / good > 30 * TOL
    assert abs(slip_mu - good) / good > 10 * TOL
