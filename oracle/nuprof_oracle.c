/*
 * nuprof_oracle.c -- plain, slow, FP64 CPU oracle for relic overdensity profiles
 * (Worku, Sabti & Kamionkowski, arXiv:2410.08267, "Rapid Methods for Modeling
 * Overdensities of Massive Neutrinos and Other Non-Cold Relics").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this file: it exists so that tests, the smoke check and the CPU-baseline leg of
 * the benchmark can compare the CUDA library against an obviously correct
 * restatement of the paper.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Every function follows one passage of the paper, cited beside it.  The method
 * is a discretised ODE plus a quadrature, so the oracle runs the same algorithm
 * (classical RK4 in u = ln a, the same grids and step count) in FP64, one
 * trajectory at a time, evaluating the background, the halo growth and the
 * force directly at every RK stage (no tables, nothing accumulated in time).
 *
 * Readings of passages that are silent, garbled or inconsistent (listed in full
 * in the design notes of the repository):
 *   R1  force sign: gravity is attractive.  dPhi/dr is taken POSITIVE for an
 *       overdensity (App. A printed with the opposite sign, which together with
 *       Eq. eoms would make gravity repulsive), used in dv/dz = gradPhi/((1+z)H).
 *   R2  dtau/dz = -1/H (Sec. II.A drops the minus sign; Eq. eoms is consistent
 *       with the minus sign).
 *   R3  f_FD(q) = 1/(1+exp(q - eta)), q = P/(k_B T0), T0 = 1.95 K (Sec. II.C
 *       prints "[1+exp(P/T]"; eta is an optional chemical potential).
 *   R4  mu = cos(psi) is integrated over [-1,1] with Gauss-Legendre nodes.
 *   R5  |P| quadrature: trapezoid rule in ln q on [q_min, q_max]; nbar uses the
 *       same grid, so a massless halo gives n/nbar = 1.
 *   R6  Newtonian P = m v throughout (no relativistic correction), as in the paper.
 *   R7  the backward integration ends at z_end (a parameter; the paper's z_i is
 *       the default), while xi(z) keeps the paper's z_i.
 *   R8  r -> 0: the force is set to zero when r^2 == 0 (never hit for x0 > 0 and
 *       Gauss-Legendre mu strictly inside (-1,1)).
 *   R9  I(y) = ln(1+y) - y/(1+y) is evaluated to a few ulp everywhere: by the
 *       positive-term series sum_{n>=2} t^n/n in t = y/(1+y) for y < 1, where
 *       the two terms cancel, and by log1p above.  The fixed-step map
 *       amplifies force errors by up to ~1e12 in halo cores, so the oracle's
 *       functions must carry no error beyond rounding.
 *
 * Units (a choice; the paper gives none): comoving length kpc, velocity km/s,
 * mass Msun, H in km/s/kpc, momentum q in units of k_B T0.
 *
 * Pins (tests/test_oracle_pins.py, tests/test_oracle_quadrature.py) tie every
 * function here to something other than itself: printed values, closed forms,
 * invariants, library routines, independent formulations.  The quadrature
 * assembly of or_profile and or_profile_masses (the q^3 measure in ln q, the
 * direction weights, the background, the mass scaling) is pinned against
 * adaptive quadrature in linear P at a well-conditioned radius with strong
 * clustering.  Parity unpinned: the absolute n/nbar at radii in halo cores,
 * where the fixed-step map is chaotic; the paper prints no such values and its
 * figures carry no recoverable data.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Physical constants (CODATA 2018 / IAU): the oracle's own copies. */
#define OR_G_KPC   4.30091727e-6       /* G in kpc (km/s)^2 / Msun */
#define OR_C_KMS   299792.458          /* speed of light, km/s      */
#define OR_KB_EVK  8.617333262e-5      /* Boltzmann constant, eV/K  */
#define OR_PI      3.14159265358979323846

/* Halo-growth and coupling kinds (same meaning as the library's enums). */
enum { OR_XI_STATIC = 0, OR_XI_LINEAR = 1, OR_XI_EXP = 2 };
enum { OR_KAPPA_ONE = 0, OR_KAPPA_POW1PZ = 1, OR_KAPPA_PAPER = 2, OR_KAPPA_CONST = 3 };
enum { OR_F_FD = 0, OR_F_FREEZEIN = 1, OR_F_TABLE = 2 };

typedef struct {
    double Om, h, T0_K;                 /* cosmology (Sec. II.A)               */
    double M_h, c, z0;                  /* halo (Sec. II.B)                    */
    int xi_kind, kappa_kind;
    double xi_p[3], kappa_p[3];
    double m_eV;                        /* relic mass                          */
    int f_kind, n_table;                /* n_table: nodes of a tabulated f     */
    double f_p[2];
    const double* f_table;              /* tabulated f values (kind 2)         */
} or_params;

typedef struct {
    double H0;          /* km/s/kpc                                         */
    double rho_bar0;    /* mean matter density today, Msun/kpc^3            */
    double R;           /* comoving radius of the collapsing region, kpc   */
    double z_i;         /* onset of collapse                                */
    double r200;        /* physical virial radius, kpc                      */
    double r_s;         /* NFW scale radius, kpc                            */
    double Ic;          /* I(c) = ln(1+c) - c/(1+c)                          */
    double xi_zs, xi_ze;/* linear-growth window actually used               */
    double force_scale; /* 1; the conditioning probe only: 1 + eps or 1 - eps */
} or_derived;

/* ---- Sec. II.B: halo parameters derived from (M_h, c, z0) --------------- */
int or_derive(const or_params* p, or_derived* d)
{
    if (!(p->Om > 0.0) || !(p->h > 0.0) || !(p->M_h >= 0.0) || !(p->c > 0.0))
        return -1;
    d->H0 = 0.1 * p->h;                                    /* 100h km/s/Mpc */
    double rho_crit0 = 3.0 * d->H0 * d->H0 / (8.0 * OR_PI * OR_G_KPC);
    d->rho_bar0 = p->Om * rho_crit0;                       /* mean *matter* density */
    /* M_h = (4 pi / 3) R^3 rho_bar(z0), with z0 = 0 */
    d->R = cbrt(3.0 * p->M_h / (4.0 * OR_PI * d->rho_bar0));
    /* (1+z_i)/(1+z0) = 200^(1/3) */
    d->z_i = cbrt(200.0) * (1.0 + p->z0) - 1.0;
    d->r200 = d->R / (1.0 + d->z_i);
    d->r_s = d->r200 / p->c;
    d->Ic = log1p(p->c) - p->c / (1.0 + p->c);
    d->xi_zs = (p->xi_p[1] > 0.0) ? p->xi_p[1] : d->z_i;
    d->xi_ze = (p->xi_p[2] > 0.0) ? p->xi_p[2] : p->z0;
    d->force_scale = 1.0;
    return 0;
}

/* ---- Sec. II.A: H(z) = H0 [Om (1+z)^3 + (1 - Om)]^(1/2) ----------------- */
double or_H(const or_params* p, const or_derived* d, double z)
{
    double zp1 = 1.0 + z;
    return d->H0 * sqrt(p->Om * zp1 * zp1 * zp1 + (1.0 - p->Om));
}

/* ---- Eq. rhototal modulation xi(z); Sec. IV.A variants ------------------- */
double or_xi(const or_params* p, const or_derived* d, double z)
{
    switch (p->xi_kind) {
    case OR_XI_STATIC:
        return 1.0;
    case OR_XI_LINEAR: {                 /* [(z_i - z)/(z_i - z0)]^alpha        */
        double alpha = (p->xi_p[0] > 0.0) ? p->xi_p[0] : 1.0;
        double t = (d->xi_zs - z) / (d->xi_zs - d->xi_ze);
        if (t <= 0.0) return 0.0;        /* before the onset: uniform universe */
        if (t >= 1.0) return 1.0;        /* after growth ends: NFW             */
        return pow(t, alpha);
    }
    case OR_XI_EXP:                      /* mass history M0 exp(-lambda z)      */
        return exp(-p->xi_p[0] * z);
    }
    return 0.0;
}

/* ---- Sec. IV.B: kappa(z) multiplying G ----------------------------------- */
double or_kappa(const or_params* p, double z)
{
    switch (p->kappa_kind) {
    case OR_KAPPA_ONE:    return 1.0;
    case OR_KAPPA_POW1PZ: return pow(1.0 + z, p->kappa_p[0]);          /* a^-gamma */
    case OR_KAPPA_PAPER:  return 1.0 + p->kappa_p[0] * pow(z / (1.0 + z), p->kappa_p[1]);
    case OR_KAPPA_CONST:  return p->kappa_p[0];
    }
    return 1.0;
}

/* ---- Eq. nfw: I(y) = ln(1+y) - y/(1+y), the NFW enclosed-mass shape ------
 * With t = y/(1+y) one has ln(1+y) = -ln(1-t), so I = -ln(1-t) - t is the
 * series sum_{n>=2} t^n / n of positive terms (no cancellation).  It is used
 * for t < 1/2 (y < 1), summed until the terms stop changing the sum; above,
 * the two terms differ by more than a factor 1.5 and are subtracted directly
 * (reading R9). */
double or_I(double y)
{
    double t = y / (1.0 + y);
    if (t < 0.5) {
        double s = 0.0, tn = t * t;
        for (int n = 2; n < 200; ++n) {
            double term = tn / (double)n;
            double next = s + term;
            if (next == s) break;
            s = next;
            tn *= t;
        }
        return s;
    }
    return log1p(y) - t;
}

/* ---- App. A: dPhi/dr at comoving radius r and redshift z ------------------
 * dPhi/dr = G kappa(z) (1+z) xi(z) M_h / r^2 * Mhat,
 *   Mhat = I(r/(r_s (1+z)))/I(c) - (r/R)^3   for r < r200 (1+z)   (NFW part)
 *        = 1 - (r/R)^3                        for r < R            (shell)
 *        = 0                                  otherwise
 * with R = r200 (1+z_i).  Positive = pointing outward (reading R1).          */
double or_dphidr(const or_params* p, const or_derived* d, double r, double z)
{
    if (r <= 0.0 || r >= d->R) return 0.0;
    double xi = or_xi(p, d, z);
    if (xi == 0.0) return 0.0;
    double zp1 = 1.0 + z;
    double rR3 = (r / d->R) * (r / d->R) * (r / d->R);
    double Mhat;
    if (r < d->r200 * zp1)
        Mhat = or_I(r / (d->r_s * zp1)) / d->Ic - rR3;
    else
        Mhat = 1.0 - rR3;
    return OR_G_KPC * or_kappa(p, z) * zp1 * xi * p->M_h * Mhat / (r * r) * d->force_scale;
}

/* ---- Eq. eoms rewritten in u = ln a (dz/du = -(1+z), reading R2):
 *   dx/du = (1+z)^2 v / H(z),   dv/du = -gradPhi / H(z),
 *   gradPhi = (dPhi/dr) x / r.                                              */
static void rhs(const or_params* p, const or_derived* d, double u,
                const double s[4], double ds[4])
{
    double z = exp(-u) - 1.0;
    double H = or_H(p, d, z);
    double zp1 = 1.0 + z;
    double A = zp1 * zp1 / H;
    ds[0] = A * s[2];
    ds[1] = A * s[3];
    double r2 = s[0] * s[0] + s[1] * s[1];
    double gx = 0.0, gy = 0.0;
    if (r2 > 0.0) {                                    /* reading R8 */
        double r = sqrt(r2);
        double g = or_dphidr(p, d, r, z) / r;
        gx = g * s[0];
        gy = g * s[1];
    }
    ds[2] = -gx / H;
    ds[3] = -gy / H;
}

/* ---- Sec. II.C / Sec. II.D: classical RK4 from u0 to u1 in n equal steps.
 * The stage times are u0 + (2k + j) du/2 computed from integers, never summed. */
void or_integrate(const or_params* p, const or_derived* d, double s[4],
                  double u0, double u1, int nsteps)
{
    double du = (u1 - u0) / (double)nsteps;
    double k1[4], k2[4], k3[4], k4[4], t[4];
    for (int k = 0; k < nsteps; ++k) {
        double ua = u0 + (double)k * du;
        double um = u0 + ((double)k + 0.5) * du;
        double ub = u0 + (double)(k + 1) * du;
        rhs(p, d, ua, s, k1);
        for (int i = 0; i < 4; ++i) t[i] = s[i] + 0.5 * du * k1[i];
        rhs(p, d, um, t, k2);
        for (int i = 0; i < 4; ++i) t[i] = s[i] + 0.5 * du * k2[i];
        rhs(p, d, um, t, k3);
        for (int i = 0; i < 4; ++i) t[i] = s[i] + du * k3[i];
        rhs(p, d, ub, t, k4);
        for (int i = 0; i < 4; ++i)
            s[i] += du / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
}

/* ---- Gauss-Legendre nodes and weights on [-1,1] (reading R4) -----------
 * Newton iteration on P_n(x) evaluated by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; w = 2 / ((1-x^2) P_n'(x)^2).      */
static void legendre_pair(int n, double x, double* pn, double* pnm1)
{
    double pk = x, pkm1 = 1.0;          /* P_1, P_0 */
    for (int k = 1; k < n; ++k) {
        double pkp1 = ((2.0 * k + 1.0) * x * pk - (double)k * pkm1) / (k + 1.0);
        pkm1 = pk;
        pk = pkp1;
    }
    *pn = pk;
    *pnm1 = pkm1;
}

int or_gauss_legendre(int n, double* x, double* w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; ++i) {
        double xi = cos(OR_PI * ((double)i + 0.75) / ((double)n + 0.5));
        double pn, pnm1, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_pair(n, xi, &pn, &pnm1);
            dp = (double)n * (xi * pn - pnm1) / (xi * xi - 1.0);   /* P_n'(x) */
            double dx = pn / dp;
            xi -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        legendre_pair(n, xi, &pn, &pnm1);
        dp = (double)n * (xi * pn - pnm1) / (xi * xi - 1.0);
        x[n - 1 - i] = xi;                       /* ascending order */
        w[n - 1 - i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
    }
    return 0;
}

/* ---- log-spaced q nodes with trapezoid weights in ln q (reading R5) ----- */
int or_log_grid(int n, double q_min, double q_max, double* q, double* wl)
{
    if (n < 2 || !(q_min > 0.0) || !(q_max > q_min)) return -1;
    double dl = log(q_max / q_min) / (double)(n - 1);
    for (int j = 0; j < n; ++j) {
        q[j] = exp(log(q_min) + (double)j * dl);
        wl[j] = (j == 0 || j == n - 1) ? 0.5 * dl : dl;
    }
    return 0;
}

/* ---- Sec. II.C, Sec. IV.B: initial phase-space distribution f(q) -------- */
double or_f(const or_params* p, double q)
{
    switch (p->f_kind) {
    case OR_F_FD:          /* Fermi-Dirac (reading R3) */
        return 1.0 / (1.0 + exp(q - p->f_p[0]));
    case OR_F_TABLE: {     /* tabulated f (Sec. IV.B distributions): nodes q_k log-spaced
                              from f_p[0] to f_p[1]; linear in ln q between nodes,
                              the first value below the range and 0 above it */
        int n = p->n_table;
        if (q <= p->f_p[0]) return p->f_table[0];
        if (q > p->f_p[1]) return 0.0;
        double pos = (double)(n - 1) * (log(q) - log(p->f_p[0])) / (log(p->f_p[1]) - log(p->f_p[0]));
        int k = (int)floor(pos);
        if (k >= n - 1) return p->f_table[n - 1];
        double frac = pos - (double)k;
        return (1.0 - frac) * p->f_table[k] + frac * p->f_table[k + 1];
    }
    case OR_F_FREEZEIN:    /* non-thermal q^(-1/2) e^(-q) */
        if (q < 1e-300) q = 1e-300;
        return exp(-q) / sqrt(q);
    }
    return 0.0;
}

/* ---- Sec. II.C initial conditions: x0 = (x0, 0), v0 = v0 (mu, sin psi),
 * with the comoving speed v0 = c P0 / m and P0 = q k_B T0 (Newtonian, R6). */
void or_initial_state(const or_params* p, double x0, double q, double mu, double s[4])
{
    double v0 = OR_C_KMS * q * (OR_KB_EVK * p->T0_K) / p->m_eV;
    s[0] = x0;
    s[1] = 0.0;
    s[2] = v0 * mu;
    s[3] = v0 * sqrt(1.0 - mu * mu);
}

/* Liouville map of Sec. II.C: final comoving momentum in units of k_B T0. */
double or_final_q(const or_params* p, const double s[4])
{
    return p->m_eV * sqrt(s[2] * s[2] + s[3] * s[3]) / (OR_C_KMS * OR_KB_EVK * p->T0_K);
}

/* Neumaier-compensated sum in index order (deterministic). */
static double csum(const double* a, long n)
{
    double s = 0.0, c = 0.0;
    for (long i = 0; i < n; ++i) {
        double t = s + a[i];
        if (fabs(s) >= fabs(a[i])) c += (s - t) + a[i];
        else                       c += (a[i] - t) + s;
        s = t;
    }
    return s + c;
}

/* ---- Eq. localdensity / Eq. density_integral: n/nbar at the given radii.
 * For each radius x0, momentum node q_j and direction node mu_k:
 *   start x = (x0, 0), v = v0 (mu, sqrt(1-mu^2)), v0 = c q_j k_B T0 / m
 *   (Sec. II.C initial conditions), integrate back from u = 0 to
 *   u = -ln(1+z_end) with nsteps RK4 steps, take q_i = m |v| / (c k_B T0)
 *   (Liouville: f0 = f_init(P_i)), and form
 *     n/nbar = sum_jk wl_j q_j^3 w_k f(q_i) / (2 sum_j wl_j q_j^3 f(q_j)).
 * radii_unit 0: radii are comoving kpc; 1: radii are in units of r200 (the
 * physical virial radius at z0 = 0, Sec. II.B).
 * radius_sel (length n_sel, may be NULL = all) chooses which radii to compute;
 * out[r] is written for the selected radii only.  qi_out, if not NULL, gets
 * q_i for every (selected radius, j, k) in that order.                       */
/* Counter-based uniform variate in [-1, 1) from splitmix64 (Steele, Lea &
 * Flood 2014) of (seed, radius index, trajectory index).  Used only to
 * measure the conditioning of the discrete method: see or_profile_perturbed. */
static double or_unit_noise(unsigned long long seed, long ir, long t)
{
    unsigned long long z = seed * 0x9E3779B97F4A7C15ULL + ((unsigned long long)ir << 32) + (unsigned long long)t;
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static int profile_impl(const or_params* p, const double* radii, int n_radii, int radii_unit,
                        const int* radius_sel, int n_sel, int n_q, double q_min, double q_max,
                        int n_mu, int nsteps, double z_end, int n_threads, double eps,
                        unsigned long long seed, int round_state, double* out, double* qi_out);

int or_profile(const or_params* p, const double* radii, int n_radii, int radii_unit,
               const int* radius_sel, int n_sel,
               int n_q, double q_min, double q_max, int n_mu,
               int nsteps, double z_end, int n_threads,
               double* out, double* qi_out)
{
    return profile_impl(p, radii, n_radii, radii_unit, radius_sel, n_sel, n_q, q_min, q_max,
                        n_mu, nsteps, z_end, n_threads, 0.0, 0ULL, 0, out, qi_out);
}

/* Conditioning probe (not part of the method): the same computation with every
 * trajectory's start state moved by eps u |x| (positions) and eps u |v|
 * (velocities), u uniform in [-1, 1) and independent per component and
 * trajectory; round_state bit 0 also rounds the state to IEEE single precision
 * after every RK4 step (what storing the state in FP32 does to an otherwise
 * FP64 computation) and bit 1, after every step, scales each component's
 * increment by (1 + eps u) and moves the component by eps u |x| or eps u |v|
 * (rounding-size noise at each step, as two FP64 codes with different
 * operation orders see it); bit 2 multiplies every force evaluation by
 * 1 + eps (odd seeds) or 1 - eps (even seeds), the systematic relative error
 * that evaluating the force in a given precision leaves (an FP32 force
 * carries a few 1e-7 in every evaluation, which rounding-size noise on the
 * state does not represent).  The spread of n/nbar over a
 * few seeds measures how strongly the discrete RK4 map amplifies rounding-size
 * differences; eps = 0 and round_state = 0 reproduce or_profile bit for bit. */
int or_profile_perturbed(const or_params* p, const double* radii, int n_radii, int radii_unit,
                         const int* radius_sel, int n_sel,
                         int n_q, double q_min, double q_max, int n_mu,
                         int nsteps, double z_end, int n_threads, double eps,
                         unsigned long long seed, int round_state, double* out, double* qi_out)
{
    return profile_impl(p, radii, n_radii, radii_unit, radius_sel, n_sel, n_q, q_min, q_max,
                        n_mu, nsteps, z_end, n_threads, eps, seed, round_state, out, qi_out);
}

/* round_state values for or_profile_perturbed */
#define OR_PROBE_ROUND_F32   1   /* round the state to float32 after every step          */
#define OR_PROBE_STEP_NOISE  2   /* rounding-size noise on each step's increments
                                    and on the state, every step                  */

static int profile_impl(const or_params* p, const double* radii, int n_radii, int radii_unit,
                        const int* radius_sel, int n_sel, int n_q, double q_min, double q_max,
                        int n_mu, int nsteps, double z_end, int n_threads, double eps,
                        unsigned long long seed, int round_state, double* out, double* qi_out)
{
    or_derived d;
    if (or_derive(p, &d) != 0) return -1;
    if (round_state & 4)                      /* probe: one relative force error per run */
        d.force_scale = (seed & 1ULL) ? 1.0 + eps : 1.0 - eps;
    if (z_end <= 0.0) z_end = d.z_i;          /* default end: the paper's z_i (R7) */
    if (n_radii < 1 || n_mu < 1 || nsteps < 1 || !(z_end > p->z0) || !(p->m_eV > 0.0))
        return -1;
    double* q = (double*)malloc(sizeof(double) * (size_t)n_q);
    double* wl = (double*)malloc(sizeof(double) * (size_t)n_q);
    double* mu = (double*)malloc(sizeof(double) * (size_t)n_mu);
    double* wmu = (double*)malloc(sizeof(double) * (size_t)n_mu);
    long ntr = (long)n_q * n_mu;
    double* contrib = (double*)malloc(sizeof(double) * (size_t)ntr);
    double* bg = (double*)malloc(sizeof(double) * (size_t)n_q);
    int rc = 0;
    if (!q || !wl || !mu || !wmu || !contrib || !bg) { rc = -2; goto done; }
    if (or_log_grid(n_q, q_min, q_max, q, wl) != 0) { rc = -1; goto done; }
    if (or_gauss_legendre(n_mu, mu, wmu) != 0) { rc = -1; goto done; }

    double u_end = -log1p(z_end);
    for (int j = 0; j < n_q; ++j)
        bg[j] = wl[j] * q[j] * q[j] * q[j] * or_f(p, q[j]);
    double nbar2 = 2.0 * csum(bg, n_q);

#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    int nsel = radius_sel ? n_sel : n_radii;
    for (int si = 0; si < nsel; ++si) {
        int ir = radius_sel ? radius_sel[si] : si;
        if (ir < 0 || ir >= n_radii) { rc = -1; goto done; }
        double x0 = (radii_unit == 1) ? radii[ir] * d.r200 : radii[ir];
        if (!(x0 > 0.0)) { rc = -1; goto done; }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
        for (long t = 0; t < ntr; ++t) {
            int j = (int)(t / n_mu), k = (int)(t % n_mu);
            double s[4];
            or_initial_state(p, x0, q[j], mu[k], s);
            if (eps != 0.0) {
                /* additive, scaled by |x| and |v|: also moves components that are 0 */
                double xn = sqrt(s[0] * s[0] + s[1] * s[1]), vn = sqrt(s[2] * s[2] + s[3] * s[3]);
                for (int c = 0; c < 4; ++c)
                    s[c] += eps * (c < 2 ? xn : vn) * or_unit_noise(seed * 8 + (unsigned long long)c, ir, t);
            }
            if (!(round_state & 3)) {      /* no per-step rounding or noise */
                or_integrate(p, &d, s, 0.0, u_end, nsteps);
            } else {
                double du = u_end / (double)nsteps;
                for (int k = 0; k < nsteps; ++k) {
                    double prev[4] = { s[0], s[1], s[2], s[3] };
                    or_integrate(p, &d, s, (double)k * du, (double)(k + 1) * du, 1);
                    if (round_state & 2) {
                        double xn = sqrt(s[0] * s[0] + s[1] * s[1]);
                        double vn = sqrt(s[2] * s[2] + s[3] * s[3]);
                        for (int c = 0; c < 4; ++c) {
                            unsigned long long key = (seed * 8 + 4 + (unsigned long long)c) * 65536ULL + (unsigned long long)k;
                            double inc = (s[c] - prev[c]) * (1.0 + eps * or_unit_noise(key, ir, t));
                            s[c] = prev[c] + inc + eps * (c < 2 ? xn : vn) * or_unit_noise(key ^ 0x5bd1e995ULL, ir, t);
                        }
                    }
                    if (round_state & 1)
                        for (int c = 0; c < 4; ++c) s[c] = (double)(float)s[c];
                }
            }
            double qi = or_final_q(p, s);
            if (qi_out) qi_out[(long)si * ntr + t] = qi;
            contrib[t] = wl[j] * q[j] * q[j] * q[j] * wmu[k] * or_f(p, qi);
        }
        out[ir] = csum(contrib, ntr) / nbar2;
    }
done:
    free(q); free(wl); free(mu); free(wmu); free(contrib); free(bg);
    return rc;
}

/* Sec. III (numerical methods): the equations of motion do not contain the
 * relic mass, so the trajectories are solved once, for the fiducial mass
 * p->m_eV, and read for every mass of a list.  A trajectory started with
 * momentum q_j (units of k_B T0) of the fiducial mass has the velocity of a
 * particle of mass m_a started with momentum s_a q_j, s_a = m_a / m_eV, and
 * ends with momentum s_a q_i.  The momentum grid of mass m_a is therefore the
 * fiducial grid times s_a, with the same trapezoid weights in ln q, and
 *   n/nbar_a = sum_jk w_j (s_a q_j)^3 w_k f(s_a q_i) / (2 sum_j w_j (s_a q_j)^3 f(s_a q_j)).
 * out holds [n_masses][n_radii] values (NaN-free only where computed). */
int or_profile_masses(const or_params* p, const double* radii, int n_radii, int radii_unit,
                      const int* radius_sel, int n_sel,
                      int n_q, double q_min, double q_max, int n_mu,
                      int nsteps, double z_end, int n_threads,
                      const double* masses, int n_masses, double* out)
{
    or_derived d;
    if (or_derive(p, &d) != 0) return -1;
    if (z_end <= 0.0) z_end = d.z_i;
    if (n_radii < 1 || n_mu < 1 || nsteps < 1 || n_masses < 1 || !(z_end > p->z0) ||
        !(p->m_eV > 0.0))
        return -1;
    for (int a = 0; a < n_masses; ++a)
        if (!(masses[a] > 0.0)) return -1;
    long ntr = (long)n_q * n_mu;
    double* q = (double*)malloc(sizeof(double) * (size_t)n_q);
    double* wl = (double*)malloc(sizeof(double) * (size_t)n_q);
    double* mu = (double*)malloc(sizeof(double) * (size_t)n_mu);
    double* wmu = (double*)malloc(sizeof(double) * (size_t)n_mu);
    double* qi = (double*)malloc(sizeof(double) * (size_t)ntr);
    double* contrib = (double*)malloc(sizeof(double) * (size_t)ntr);
    double* bg = (double*)malloc(sizeof(double) * (size_t)n_q);
    int rc = 0;
    if (!q || !wl || !mu || !wmu || !qi || !contrib || !bg) { rc = -2; goto done; }
    if (or_log_grid(n_q, q_min, q_max, q, wl) != 0) { rc = -1; goto done; }
    if (or_gauss_legendre(n_mu, mu, wmu) != 0) { rc = -1; goto done; }
    double u_end = -log1p(z_end);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    int nsel = radius_sel ? n_sel : n_radii;
    for (int si = 0; si < nsel; ++si) {
        int ir = radius_sel ? radius_sel[si] : si;
        if (ir < 0 || ir >= n_radii) { rc = -1; goto done; }
        double x0 = (radii_unit == 1) ? radii[ir] * d.r200 : radii[ir];
        if (!(x0 > 0.0)) { rc = -1; goto done; }
        /* the trajectories of the fiducial mass */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
        for (long t = 0; t < ntr; ++t) {
            int j = (int)(t / n_mu), k = (int)(t % n_mu);
            double st[4];
            or_initial_state(p, x0, q[j], mu[k], st);
            or_integrate(p, &d, st, 0.0, u_end, nsteps);
            qi[t] = or_final_q(p, st);
        }
        /* every mass reads them with momenta scaled by s_a */
        for (int a = 0; a < n_masses; ++a) {
            double sa = masses[a] / p->m_eV;
            for (int j = 0; j < n_q; ++j) {
                double qa = sa * q[j];
                bg[j] = wl[j] * qa * qa * qa * or_f(p, qa);
            }
            for (long t = 0; t < ntr; ++t) {
                int j = (int)(t / n_mu), k = (int)(t % n_mu);
                double qa = sa * q[j];
                contrib[t] = wl[j] * qa * qa * qa * wmu[k] * or_f(p, sa * qi[t]);
            }
            out[(long)a * n_radii + ir] = csum(contrib, ntr) / (2.0 * csum(bg, n_q));
        }
    }
done:
    free(q); free(wl); free(mu); free(wmu); free(qi); free(contrib); free(bg);
    return rc;
}

/* Number of OpenMP threads the oracle would use (1 without OpenMP). */
int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
