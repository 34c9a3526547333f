"""Pins of the FP64 oracle to things other than itself.

Each test ties one part of the oracle to a value the paper prints, a closed
form, an invariant of the equations of motion, a library routine, or an
independent formulation (the density profile instead of the enclosed-mass
closed form, the equations in z instead of ln a).  A dropped term, a wrong
sign, an index slip or a transposed operand anywhere in the oracle fails at
least one of them.
"""
import json
import math
import os

import mpmath
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2410_08267_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
C_KMS = 299792.458
G = 4.30091727e-6


def halo(**kw):
    base = dict(Om=0.31, h=0.67, M_h=1e12, c=10.0, xi_kind=W.XI_STATIC, m_eV=0.1)
    base.update(kw)
    return W.Problem(**base)


# --------------------------------------------------------------------------
# Sec. II.B: derived halo quantities
# --------------------------------------------------------------------------

def test_collapse_redshift_matches_printed_value():
    d = oracle.derive(halo())
    g = GOLD["one_plus_zi_over_one_plus_z0"]
    assert abs((1 + d["z_i"]) / g["value"] - 1) < g["rel_tol"]
    assert (1 + d["z_i"]) ** 3 == pytest.approx(200.0, rel=1e-13)


def test_critical_density_units():
    # pins G, H0 = 100 h km/s/Mpc and the kpc/Msun unit system
    for h in (0.5, 0.67, 0.8):
        d = oracle.derive(halo(h=h, Om=0.3))
        g = GOLD["rho_crit_over_h2_Msun_per_kpc3"]
        assert d["rho_bar0"] / (0.3 * h * h) == pytest.approx(g["value"], rel=g["rel_tol"])


def test_virial_mass_definition():
    # M_h = (4 pi/3) r200^3 * 200 rho_bar0: the halo is 200x the mean density today
    for M in (1e11, 1e13, 1e15):
        d = oracle.derive(halo(M_h=M, c=7.0))
        m200 = 4.0 / 3.0 * math.pi * d["r200"] ** 3 * 200.0 * d["rho_bar0"]
        assert m200 == pytest.approx(M, rel=1e-12)
        assert d["R"] == pytest.approx(d["r200"] * 200 ** (1 / 3), rel=1e-13)
        assert d["r_s"] == pytest.approx(d["r200"] / 7.0, rel=1e-14)


# --------------------------------------------------------------------------
# Sec. II.A, Sec. IV: background, growth, coupling
# --------------------------------------------------------------------------

def test_H_special_values():
    pb = halo(Om=0.31, h=0.67)
    assert oracle.H(pb, 0.0) == pytest.approx(0.067, rel=1e-15)
    # Einstein-de Sitter: H = H0 (1+z)^1.5
    eds = halo(Om=1.0)
    for z in (0.5, 3.0):
        assert oracle.H(eds, z) == pytest.approx(0.067 * (1 + z) ** 1.5, rel=1e-14)


def test_xi_limits_and_variants():
    pb = halo(xi_kind=W.XI_LINEAR)
    d = oracle.derive(pb)
    assert oracle.xi(pb, 0.0) == 1.0
    assert oracle.xi(pb, d["z_i"]) == 0.0
    assert oracle.xi(pb, d["z_i"] + 1.0) == 0.0
    assert oracle.xi(pb, d["z_i"] / 2) == pytest.approx(0.5, rel=1e-14)
    p2 = halo(xi_kind=W.XI_LINEAR, xi_p=(2.0, 0.0, 0.0))
    assert oracle.xi(p2, d["z_i"] / 2) == pytest.approx(0.25, rel=1e-14)
    # earlier onset and end: growth from z=8 to z=1
    p3 = halo(xi_kind=W.XI_LINEAR, xi_p=(1.0, 8.0, 1.0))
    assert oracle.xi(p3, 0.5) == 1.0 and oracle.xi(p3, 9.0) == 0.0
    assert oracle.xi(p3, 4.5) == pytest.approx(0.5, rel=1e-14)
    pe = halo(xi_kind=W.XI_EXP, xi_p=(0.8, 0.0, 0.0))
    assert oracle.xi(pe, 2.0) == pytest.approx(math.exp(-1.6), rel=1e-15)


def test_kappa_variants():
    assert oracle.kappa(halo(), 3.0) == 1.0
    pg = halo(kappa_kind=W.KAPPA_POW1PZ, kappa_p=(0.05, 0, 0))
    assert oracle.kappa(pg, 3.0) == pytest.approx(4.0 ** 0.05, rel=1e-15)   # a^-gamma at a=1/4
    pp = halo(kappa_kind=W.KAPPA_PAPER, kappa_p=(0.2, 1.5, 0))
    assert oracle.kappa(pp, 0.0) == 1.0                                     # decays to unity today
    assert oracle.kappa(pp, 1.0) == pytest.approx(1 + 0.2 * 0.5 ** 1.5, rel=1e-15)
    assert oracle.kappa(halo(kappa_kind=W.KAPPA_CONST, kappa_p=(1.1, 0, 0)), 2.0) == 1.1


# --------------------------------------------------------------------------
# Eq. nfw: I(y) against arbitrary precision
# --------------------------------------------------------------------------

@pytest.mark.parametrize("y", [1e-8, 3e-5, 9.99e-4, 1.0001e-3, 0.01, 0.02, 0.1, 0.5, 0.999, 1.0,
                               1.001, 3.0, 10.0, 40.0])
def test_I_against_mpmath(y):
    # a few ulp everywhere: the force enters a map that amplifies its errors
    mpmath.mp.dps = 40
    exact = mpmath.log1p(y) - mpmath.mpf(y) / (1 + mpmath.mpf(y))
    assert oracle.I(y) == pytest.approx(float(exact), rel=2e-15)


def test_I_dense_sweep_against_mpmath():
    mpmath.mp.dps = 40
    worst = 0.0
    for y in np.geomspace(1e-6, 50.0, 400):
        exact = float(mpmath.log1p(y) - mpmath.mpf(y) / (1 + mpmath.mpf(y)))
        worst = max(worst, abs(oracle.I(y) - exact) / exact)
    assert worst < 2e-15


# --------------------------------------------------------------------------
# App. A: closed-form gradient against the Poisson integral of Eq. rhototal
# --------------------------------------------------------------------------

def poisson_gradient(pb, d, r, z):
    """(4 pi G / (a r^2)) int_0^{r/(1+z)} r_p^2 [rho_tot - rho_bar] dr_p with
    rho_tot from Eq. rhototal and rho_NFW from Eq. nfw, integrated numerically.
    Sign: positive for an overdensity (attractive reading)."""
    zp1 = 1.0 + z
    xi = oracle.xi(pb, z)
    kap = oracle.kappa(pb, z)
    r_s, r200, Ic = d["r_s"], d["r200"], d["Ic"]
    rho_s = pb.M_h / (4 * math.pi * r_s ** 3 * Ic)
    rho_bar = d["rho_bar0"] * zp1 ** 3
    rp_max_halo = d["R"] / zp1

    def rho_tot(rp):
        if rp < r200:
            x = rp / r_s
            return rho_s / (x * (1 + x) ** 2) * xi + rho_bar * (1 - xi)
        if rp < rp_max_halo:
            return rho_bar * (1 - xi)
        return rho_bar

    rp = r / zp1
    pts = [p for p in (r200, rp_max_halo) if p < rp]
    val, _ = integrate.quad(lambda s: s * s * (rho_tot(s) - rho_bar), 0.0, rp,
                            points=pts or None, limit=400, epsabs=0, epsrel=1e-12)
    return 4 * math.pi * G * kap * zp1 * val / (r * r)


@pytest.mark.parametrize("kind", [W.XI_STATIC, W.XI_LINEAR, W.XI_EXP])
def test_force_equals_poisson_integral(kind):
    pb = halo(M_h=3e12, c=8.0, xi_kind=kind, xi_p=(1.0 if kind != W.XI_EXP else 0.8, 0, 0),
              kappa_kind=W.KAPPA_PAPER, kappa_p=(0.2, 1.5, 0))
    d = oracle.derive(pb)
    rng = np.random.default_rng(7)
    for _ in range(25):
        z = rng.uniform(0.0, 4.5)
        r = 10 ** rng.uniform(-1.0, math.log10(1.2 * d["R"]))
        ref = poisson_gradient(pb, d, r, z)
        got = oracle.dphidr(pb, r, z)
        scale = G * (1 + z) * pb.M_h / r ** 2       # point-mass gradient of the whole halo
        assert got == pytest.approx(ref, rel=1e-8, abs=1e-10 * scale)


def test_force_branches():
    pb = halo(M_h=1e13, c=6.0, xi_kind=W.XI_LINEAR)
    d = oracle.derive(pb)
    z = 1.3
    rb = d["r200"] * (1 + z)
    lo, hi = oracle.dphidr(pb, rb * (1 - 1e-12), z), oracle.dphidr(pb, rb * (1 + 1e-12), z)
    assert lo == pytest.approx(hi, rel=1e-9)                # continuous at the NFW edge
    assert oracle.dphidr(pb, d["R"] * (1 - 1e-9), z) == pytest.approx(0.0, abs=1e-9 * lo)
    assert oracle.dphidr(pb, d["R"] * 1.01, z) == 0.0        # compensated: zero beyond R
    assert oracle.dphidr(pb, 50.0, d["z_i"] + 0.1) == 0.0    # no halo before z_i
    assert oracle.dphidr(pb, 50.0, z) > 0.0                  # outward gradient: attractive
    # shell region is underdense: dPhi/dr decreases outward there
    r1, r2 = rb * 1.1, rb * 1.3
    assert oracle.dphidr(pb, r2, z) * r2 ** 2 < oracle.dphidr(pb, r1, z) * r1 ** 2


def test_mass_compensation_zero_total_perturbation():
    pb = halo(M_h=1e14, c=5.0, xi_kind=W.XI_LINEAR)
    d = oracle.derive(pb)
    for z in (0.0, 1.0, 3.0):
        assert poisson_gradient(pb, d, d["R"] * 0.999999, z) == pytest.approx(0.0, abs=1e-4 *
               poisson_gradient(pb, d, d["R"] * 0.5, z))


# --------------------------------------------------------------------------
# Eq. eoms: integrator invariants and an independent formulation
# --------------------------------------------------------------------------

def test_massless_halo_keeps_velocity_bitwise():
    pb = halo(M_h=0.0)
    s0 = np.array([30.0, 0.0, 120.0 * 0.3, 120.0 * math.sqrt(1 - 0.09)])
    s = oracle.integrate(pb, s0, 0.0, -math.log(5.0), 200)
    assert s[2] == s0[2] and s[3] == s0[3]


@pytest.mark.parametrize("Om", [1.0, 0.31])
def test_free_streaming_displacement(Om):
    # App. B: a free particle moves v * I_io, I_io = int_0^z (1+z') dz'/H(z').
    # Einstein-de Sitter has the closed form I_io = 2 [(1+z)^(1/2) - 1] / H0.
    pb = halo(M_h=0.0, Om=Om, h=0.7)
    z_end = 4.0
    H0 = 0.07
    if Om == 1.0:
        I_io = 2.0 * (math.sqrt(1 + z_end) - 1.0) / H0
    else:
        I_io, _ = integrate.quad(lambda z: (1 + z) / (H0 * math.sqrt(Om * (1 + z) ** 3 + 1 - Om)),
                                 0.0, z_end, epsabs=0, epsrel=1e-13)
    v = np.array([250.0, -80.0])
    s = oracle.integrate(pb, [100.0, 5.0, v[0], v[1]], 0.0, -math.log(1 + z_end), 400)
    # backward in time the particle sits behind its present position
    assert s[0] == pytest.approx(100.0 - v[0] * I_io, rel=1e-10)
    assert s[1] == pytest.approx(5.0 - v[1] * I_io, rel=1e-10)


def _smooth_orbit():
    # bound orbit inside the NFW region of a static 1e12 halo, far from r=0
    pb = halo(M_h=1e12, c=10.0, xi_kind=W.XI_STATIC)
    mu = 0.2
    s0 = [60.0, 0.0, 150.0 * mu, 150.0 * math.sqrt(1 - mu * mu)]
    return pb, np.array(s0)


def test_angular_momentum_conserved_to_order_h4():
    pb, s0 = _smooth_orbit()
    ell0 = s0[0] * s0[3] - s0[1] * s0[2]
    drift = []
    for n in (200, 400, 800):
        s = oracle.integrate(pb, s0, 0.0, -math.log(5.0), n)
        drift.append(abs((s[0] * s[3] - s[1] * s[2]) - ell0) / abs(ell0))
    assert drift[-1] < 1e-6
    # RK4 does not conserve ell exactly; its drift falls as h^4 (ratio -> 16
    # from above on this orbit, with the h^5 term still visible)
    assert 14.0 < drift[0] / drift[1] < 32.0 and 14.0 < drift[1] / drift[2] < 32.0


def test_time_reversibility():
    pb, s0 = _smooth_orbit()
    errs = []
    for n in (200, 400, 800):
        s = oracle.integrate(pb, s0, 0.0, -math.log(5.0), n)
        back = oracle.integrate(pb, s, -math.log(5.0), 0.0, n)
        errs.append(np.max(np.abs(back - s0) / np.abs(s0).max()))
    assert errs[-1] < 1e-5
    # the h^5 local-error terms of the backward and forward passes cancel, so
    # the round trip closes one order faster than the h^4 global error
    assert 26.0 < errs[0] / errs[1] < 38.0 and 26.0 < errs[1] / errs[2] < 38.0


def test_richardson_order_four():
    pb, s0 = _smooth_orbit()
    u1 = -math.log(5.0)
    v = [oracle.integrate(pb, s0, 0.0, u1, n) for n in (200, 400, 800, 1600)]
    ratios = [np.linalg.norm(v[i] - v[i + 1]) / np.linalg.norm(v[i + 1] - v[i + 2]) for i in range(2)]
    # fourth order: successive-difference ratio 2^4 = 16, approached from above
    assert all(14.0 < r < 30.0 for r in ratios) and ratios[1] < ratios[0]


def test_attractive_gravity_forward_in_time():
    # reading of the force sign: a particle at rest falls toward the halo
    pb = halo(M_h=1e13, c=6.0, xi_kind=W.XI_STATIC)
    s = oracle.integrate(pb, [200.0, 0.0, 0.0, 0.0], -math.log(2.0), -math.log(1.9), 50)
    assert s[0] < 200.0 and s[2] < 0.0
    # and backward in time from rest today it was moving outward
    s = oracle.integrate(pb, [200.0, 0.0, 0.0, 0.0], 0.0, -0.05, 50)
    assert s[2] > 0.0


def test_rk4_in_ln_a_matches_eoms_in_z():
    # Eq. eoms integrated in z (the paper's variable) with a high-order
    # adaptive library integrator, against the oracle's RK4 in ln a.
    pb = halo(M_h=2e12, c=9.0, xi_kind=W.XI_LINEAR, kappa_kind=W.KAPPA_POW1PZ,
              kappa_p=(0.05, 0, 0), Om=0.3, h=0.7)
    H0, Om = 0.07, 0.3

    def Hz(z):
        return H0 * math.sqrt(Om * (1 + z) ** 3 + 1 - Om)

    def rhs(z, s):
        x, y, vx, vy = s
        r = math.hypot(x, y)
        g = oracle.dphidr(pb, r, z) / r
        h = Hz(z)
        return [-vx * (1 + z) / h, -vy * (1 + z) / h,
                g * x / ((1 + z) * h), g * y / ((1 + z) * h)]

    s0 = [150.0, 0.0, 90.0, 140.0]
    z_end = 3.0
    sol = integrate.solve_ivp(rhs, (0.0, z_end), s0, method="DOP853", rtol=1e-12, atol=1e-12)
    ref = sol.y[:, -1]
    got = oracle.integrate(pb, s0, 0.0, -math.log(1 + z_end), 4000)
    assert np.allclose(got, ref, rtol=1e-7, atol=1e-7 * np.abs(ref).max())


# --------------------------------------------------------------------------
# Eq. localdensity quadrature
# --------------------------------------------------------------------------

def test_gauss_legendre_matches_library_and_is_exact():
    for n in (1, 2, 5, 20, 64, 100):
        x, w = oracle.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, xr, rtol=0, atol=1e-14)
        assert np.allclose(w, wr, rtol=0, atol=1e-14)
        for k in range(0, 2 * n, max(1, n // 4)):
            exact = 0.0 if k % 2 else 2.0 / (k + 1)
            assert np.dot(w, x ** k) == pytest.approx(exact, abs=1e-13)


def test_log_grid_trapezoid_weights():
    q, w = oracle.log_grid(50, 0.01, 10.0)
    assert q[0] == pytest.approx(0.01, rel=1e-15) and q[-1] == pytest.approx(10.0, rel=1e-14)
    lnq = np.log(q)
    fvals = q ** 3 / (1 + np.exp(q))
    assert np.dot(w, fvals) == pytest.approx(integrate.trapezoid(fvals, lnq), rel=1e-13)


def test_fermi_dirac_moment():
    g = GOLD["fd_moment_q2"]
    pb = halo()
    q, w = oracle.log_grid(4000, 1e-5, 60.0)
    fvals = np.array([oracle.f(pb, qq) for qq in q])
    assert np.dot(w, q ** 3 * fvals) == pytest.approx(g["value"], rel=g["rel_tol"])


def test_relic_distributions():
    assert oracle.f(halo(), 0.0) == 0.5
    eta = halo(f_p=(1.0, 0.0))
    assert oracle.f(eta, 1.0) == 0.5                                # chemical potential shift
    fi = halo(f_kind=W.F_FREEZEIN)
    assert oracle.f(fi, 4.0) == pytest.approx(math.exp(-4.0) / 2.0, rel=1e-15)


def test_massless_halo_gives_unit_overdensity():
    for kind in (W.F_FD, W.F_FREEZEIN):
        pb = W.plain_small()[0].replace(M_h=0.0, f_kind=kind, n_steps=40)
        out = oracle.profile(pb)
        assert np.all(np.abs(out - 1.0) < 1e-13)


def test_large_radius_returns_to_background_and_clusters_inside():
    pb = W.plain_small()[0].replace(M_h=1e12, xi_kind=W.XI_LINEAR, m_eV=0.3, n_q=30, n_mu=16,
                                    n_steps=200, radii=np.array([5.0, 150000.0]))
    out = oracle.profile(pb)
    assert out[0] > 1.05                  # clustered inside the halo (Fig. 2)
    assert abs(out[1] - 1.0) < 2e-3       # far outside R: background value


def test_radius_units_and_selection():
    pb = W.plain_small()[0].replace(n_steps=30, n_q=8, n_mu=6)
    d = oracle.derive(pb)
    full = oracle.profile(pb)
    sel = oracle.profile(pb, radius_sel=[3, 7])
    assert sel[3] == full[3] and sel[7] == full[7] and np.isnan(sel[0])
    pr = pb.replace(radii=np.asarray(pb.radii) / d["r200"], radii_unit=W.RADII_R200)
    assert np.allclose(oracle.profile(pr), full, rtol=1e-12)


def test_final_momenta_free_streaming_equal_initial():
    pb = W.plain_small()[0].replace(M_h=0.0, n_steps=20, n_q=7, n_mu=5)
    _, qi = oracle.profile(pb, radius_sel=[0, 4], return_qi=True)
    q, _ = oracle.log_grid(7, 0.01, 10.0)
    assert np.allclose(qi, q[None, :, None], rtol=1e-15)


def test_initial_speed_scale_matches_textbook_mean_speed():
    # <v> = int q^2 f v0(q) dq / int q^2 f dq for Fermi-Dirac relics of mass 1 eV
    g = GOLD["mean_relic_speed_kms_eV"]
    pb = halo(m_eV=1.0)
    q, w = oracle.log_grid(3000, 1e-5, 60.0)
    fq = np.array([oracle.f(pb, x) for x in q])
    v0 = np.array([oracle.initial_state(pb, 10.0, x, 0.0, )[3] for x in q])
    vmean = np.dot(w, q ** 3 * fq * v0) / np.dot(w, q ** 3 * fq)
    assert vmean == pytest.approx(g["value"], rel=g["rel_tol"])
    s = oracle.initial_state(pb, 10.0, 2.0, 0.6)
    assert s[0] == 10.0 and s[1] == 0.0 and s[2] / s[3] == pytest.approx(0.75, rel=1e-14)
    assert oracle.final_q(pb, s) == pytest.approx(2.0, rel=1e-15)
    # the equations are mass-free: (m, q) and (2m, 2q) start at the same velocity
    assert np.allclose(oracle.initial_state(halo(m_eV=0.2), 5.0, 3.0, 0.1),
                       oracle.initial_state(halo(m_eV=0.4), 5.0, 6.0, 0.1), rtol=1e-15)


# --------------------------------------------------------------------------
# Sec. III: one trajectory set read for many relic masses
# --------------------------------------------------------------------------

def test_mass_reuse_reads_the_fiducial_mass_bit_for_bit():
    pb = W.plain_small(precision=W.FP64)[0].replace(n_q=16, n_mu=6, n_steps=120)
    m = oracle.profile_masses(pb, [pb.m_eV, 0.3])
    assert np.array_equal(m[0], oracle.profile(pb))


def test_mass_reuse_equals_direct_runs_with_scaled_grids():
    # Mass m_a on the fiducial grid scaled by s_a = m_a/m starts every
    # trajectory at the fiducial velocity; a direct run at m_a on the scaled
    # q range must agree (exactly up to rounding where the map is well conditioned).
    pb = W.plain_small(precision=W.FP64)[0].replace(radii=np.array([100.0, 300.0]), n_q=24, n_mu=10)
    masses = [0.02, 0.05, 0.25, 0.6]
    m = oracle.profile_masses(pb, masses)
    for a, ma in enumerate(masses):
        s = ma / pb.m_eV
        b = oracle.profile(pb.replace(m_eV=ma, q_min=pb.q_min * s, q_max=pb.q_max * s))
        assert np.allclose(m[a], b, rtol=1e-6, atol=0), (ma, m[a], b)
    # heavier relics cluster more (Sec. III, Fig. 1)
    assert np.all(np.diff(m[:, 0]) > 0)


def test_mass_reuse_massless_halo_gives_background_for_every_mass():
    pb = W.plain_small(precision=W.FP64)[0].replace(M_h=0.0, n_q=20, n_mu=4, n_steps=40)
    m = oracle.profile_masses(pb, [0.01, 0.1, 0.5])
    assert np.allclose(m, 1.0, rtol=1e-13, atol=0)


# --------------------------------------------------------------------------
# Sec. IV.B: tabulated distributions
# --------------------------------------------------------------------------

def _table(fun, n=400, q0=1e-3, q1=40.0):
    q = np.geomspace(q0, q1, n)
    return q, tuple(float(v) for v in fun(q))


def test_table_interpolates_linearly_in_ln_q():
    q, tab = _table(lambda x: 2.0 + 0.5 * np.log(x), n=7, q0=0.01, q1=10.0)
    pb = halo(f_kind=W.F_TABLE, f_p=(0.01, 10.0), f_table=tab)
    for x in (0.0123, 0.5, 3.7, 9.99):
        assert oracle.f(pb, x) == pytest.approx(2.0 + 0.5 * math.log(x), rel=1e-13)
    assert oracle.f(pb, 1e-4) == tab[0]
    assert oracle.f(pb, 10.0) == pytest.approx(tab[-1], rel=1e-15)
    assert oracle.f(pb, 10.5) == 0.0


def test_dense_table_of_fermi_dirac_reproduces_the_closed_form():
    q, tab = _table(lambda x: 1.0 / (1.0 + np.exp(x)), n=3000, q0=1e-4, q1=60.0)
    base = W.plain_small(precision=W.FP64)[0].replace(n_q=24, n_mu=8, n_steps=200,
                                                       radii=np.array([10.0, 100.0]))
    a = oracle.profile(base)
    b = oracle.profile(base.replace(f_kind=W.F_TABLE, f_p=(1e-4, 60.0), f_table=tab))
    assert np.allclose(a, b, rtol=2e-5, atol=0)
    m0 = base.replace(M_h=0.0, f_kind=W.F_TABLE, f_p=(1e-4, 60.0), f_table=tab)
    assert np.allclose(oracle.profile(m0), 1.0, rtol=1e-13)


def test_conditioning_probe_force_error_is_a_relative_force_scale():
    """The probe's systematic force error (not part of the method) is a
    relative scale of every force evaluation: with eps = 0 it reproduces the
    oracle bit for bit, and with a constant coupling kappa (Sec. IV.B, which
    multiplies G in every evaluation) a force error of +eps (odd seed) or
    -eps (even seed) equals the run with kappa scaled by 1 +/- eps and the
    same seeded start-state noise, to rounding, at radii where the map is
    well conditioned."""
    pb = W.plain_small(precision=W.FP64)[0].replace(n_q=24, n_mu=8, n_steps=100,
                                                    kappa_kind=W.KAPPA_CONST,
                                                    kappa_p=(1.0, 0.0, 0.0))
    sel = [9]                       # 300 kpc: regular orbits, amplification ~1e3
    base = oracle.profile(pb, radius_sel=sel)[sel]
    same = oracle.profile_perturbed(pb, 0.0, 1, radius_sel=sel, force_noise=True)[sel]
    assert np.array_equal(same, base)
    eps = 1e-3
    for seed, k in ((1, 1.0 + eps), (2, 1.0 - eps)):
        got = oracle.profile_perturbed(pb, eps, seed, radius_sel=sel, force_noise=True)[sel]
        ref = oracle.profile_perturbed(pb.replace(kappa_p=(k, 0.0, 0.0)), eps, seed,
                                       radius_sel=sel)[sel]
        assert np.all(np.abs(got - ref) <= 1e-10 * np.abs(ref)), (seed, got, ref)
        assert np.all(np.abs(got - base) > 1e-7 * np.abs(base))      # it does move
