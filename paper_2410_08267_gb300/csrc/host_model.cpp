// Host-side FP64 model of the relic-overdensity library: input validation, the
// halo derivation of Sec. II.B, the background of Sec. II.A, the growth and
// coupling variants of Sec. IV, the per-step coefficient table consumed by the
// trajectory kernel, and the quadrature nodes of Eq. localdensity.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "nuprof_internal.h"

namespace nuprof {

void resolve_opts(const nu_opts* in, nu_opts& o)
{
    std::memset(&o, 0, sizeof(o));
    if (in) o = *in;
    if (o.n_steps == 0) o.n_steps = 400;
    if (o.block == 0) o.block = 256;
    if (o.tpt == 0) o.tpt = 1;
}

int validate(const nu_cosmo* cosmo, const nu_halo* halo, const nu_relic* relic,
             const double* radii, int n_radii, const nu_pgrid* g, const nu_opts* o)
{
    if (!cosmo || !halo || !relic || !radii || !g || !o) return NU_EINVAL;
    if (!(cosmo->Om > 0.0 && cosmo->Om <= 1.0) || !(cosmo->h > 0.0) || !(cosmo->T0_K > 0.0))
        return NU_EINVAL;
    if (!(halo->M_h >= 0.0) || !std::isfinite(halo->M_h) || !(halo->c > 0.0)) return NU_EINVAL;
    if (halo->z0 != 0.0) return NU_ENOTSUP;
    if (halo->xi_kind < NU_XI_STATIC || halo->xi_kind > NU_XI_EXP) return NU_EINVAL;
    if (halo->kappa_kind < NU_KAPPA_ONE || halo->kappa_kind > NU_KAPPA_CONST) return NU_EINVAL;
    if (halo->xi_kind == NU_XI_LINEAR) {
        double zs = halo->xi_p[1], ze = halo->xi_p[2];
        if (zs > 0.0 && ze > 0.0 && !(zs > ze)) return NU_EINVAL;
    }
    if (!(relic->m_eV > 0.0) || !std::isfinite(relic->m_eV)) return NU_EINVAL;
    if (relic->f_kind < NU_F_FD || relic->f_kind > NU_F_TABLE) return NU_EINVAL;
    if (relic->f_kind == NU_F_TABLE) {                // tabulated f (Sec. IV.B)
        if (!relic->f_table || relic->n_table < 2 || relic->n_table > NU_MAX_FTABLE) return NU_EINVAL;
        if (!(relic->f_p[0] > 0.0) || !(relic->f_p[1] > relic->f_p[0]) || !std::isfinite(relic->f_p[1]))
            return NU_EINVAL;
        for (int k = 0; k < relic->n_table; ++k)
            if (!(relic->f_table[k] >= 0.0) || !std::isfinite(relic->f_table[k])) return NU_EINVAL;
    }
    if (relic->n_masses < 0 || relic->n_masses > NU_MAX_MASSES) return NU_EINVAL;
    if (relic->n_masses > 0) {                        // mass reuse (Sec. III)
        if (!relic->masses_eV) return NU_EINVAL;
        for (int a = 0; a < relic->n_masses; ++a)
            if (!(relic->masses_eV[a] > 0.0) || !std::isfinite(relic->masses_eV[a])) return NU_EINVAL;
    }
    if (n_radii < 1) return NU_EINVAL;
    for (int i = 0; i < n_radii; ++i)
        if (!(radii[i] > 0.0) || !std::isfinite(radii[i])) return NU_EINVAL;
    if (g->n_q < 2 || g->n_mu < 1 || !(g->q_min > 0.0) || !(g->q_max > g->q_min)) return NU_EINVAL;
    if (o->n_steps < 1) return NU_EINVAL;
    if (o->n_steps > NU_MAX_STEPS) return NU_ENOTSUP;
    if (o->precision != NU_FP64 && o->precision != NU_MIXED) return NU_EINVAL;
    if ((o->flags & NU_FLAG_VERIFY) && o->precision != NU_MIXED) return NU_EINVAL;
    if (o->radii_unit != NU_RADII_KPC && o->radii_unit != NU_RADII_R200) return NU_EINVAL;
    if (o->radii_unit == NU_RADII_R200 && halo->M_h == 0.0) return NU_EINVAL;
    if (o->block < 64 || o->block > 512 || (o->block % 32) != 0) return NU_EINVAL;
    if (o->tpt != 1 && o->tpt != 2 && o->tpt != kTptPacked) return NU_EINVAL;
    if (o->tpt == kTptPacked && o->precision != NU_MIXED) return NU_EINVAL;
    long long ntraj = (long long)g->n_q * g->n_mu;
    if (ntraj > (1LL << 30) || (long long)n_radii * ntraj > (1LL << 40)) return NU_EINVAL;
    return NU_OK;
}

// Sec. II.B.  With rho_bar the mean matter density, the collapsing region of
// comoving radius R holds M_h = (4 pi / 3) R^3 rho_bar(z0); it starts to
// collapse at (1+z_i) = 200^(1/3) (1+z0) and ends as an NFW halo of physical
// radius r200 = R/(1+z_i) and scale radius r_s = r200/c.
int derive(const nu_cosmo& cosmo, const nu_halo& halo, const nu_opts& opts, Derived& d)
{
    d.H0 = 0.1 * cosmo.h;                                   // km/s/kpc
    const double rho_crit0 = 3.0 * d.H0 * d.H0 / (8.0 * kPi * kG);
    d.rho_bar0 = cosmo.Om * rho_crit0;
    d.R = std::cbrt(halo.M_h / (4.0 / 3.0 * kPi * d.rho_bar0));
    d.z_i = std::cbrt(200.0) * (1.0 + halo.z0) - 1.0;
    d.r200 = d.R / (1.0 + d.z_i);
    d.r_s = d.r200 / halo.c;
    d.Ic = std::log1p(halo.c) - halo.c / (1.0 + halo.c);
    d.xi_zs = halo.xi_p[1] > 0.0 ? halo.xi_p[1] : d.z_i;
    d.xi_ze = halo.xi_p[2] > 0.0 ? halo.xi_p[2] : halo.z0;
    d.z_end = opts.z_end > 0.0 ? opts.z_end : d.z_i;
    if (!(d.z_end > halo.z0)) return NU_EINVAL;
    return NU_OK;
}

// Sec. II.A: flat FRW without radiation.
double hubble(const nu_cosmo& cosmo, const Derived& d, double z)
{
    const double a3inv = (1.0 + z) * (1.0 + z) * (1.0 + z);
    return d.H0 * std::sqrt(cosmo.Om * a3inv + (1.0 - cosmo.Om));
}

// Eq. rhototal modulation and its Sec. IV.A variants.
double growth_xi(const nu_halo& halo, const Derived& d, double z)
{
    switch (halo.xi_kind) {
    case NU_XI_STATIC:
        return 1.0;
    case NU_XI_LINEAR: {
        const double t = (d.xi_zs - z) / (d.xi_zs - d.xi_ze);
        if (t <= 0.0) return 0.0;
        if (t >= 1.0) return 1.0;
        const double alpha = halo.xi_p[0] > 0.0 ? halo.xi_p[0] : 1.0;
        return alpha == 1.0 ? t : std::pow(t, alpha);
    }
    case NU_XI_EXP:
        return std::exp(-halo.xi_p[0] * z);
    default:
        return 0.0;
    }
}

// Sec. IV.B: G -> kappa(z) G.
double coupling_kappa(const nu_halo& halo, double z)
{
    switch (halo.kappa_kind) {
    case NU_KAPPA_POW1PZ: return std::pow(1.0 + z, halo.kappa_p[0]);
    case NU_KAPPA_PAPER:  return 1.0 + halo.kappa_p[0] * std::pow(z / (1.0 + z), halo.kappa_p[1]);
    case NU_KAPPA_CONST:  return halo.kappa_p[0];
    default:              return 1.0;
    }
}

// Initial distribution in q = P/(k_B T0): Fermi-Dirac with chemical potential
// (Sec. II.C) or the non-thermal q^(-1/2) e^(-q) shape.
double relic_f(const nu_relic& relic, double q)
{
    if (relic.f_kind == NU_F_TABLE) {
        // linear in ln q between log-spaced nodes; f_table[0] below, 0 above
        const int n = relic.n_table;
        if (!(q > relic.f_p[0])) return relic.f_table[0];
        if (q > relic.f_p[1]) return 0.0;
        const double u = std::log(q / relic.f_p[0]) * (n - 1) / std::log(relic.f_p[1] / relic.f_p[0]);
        if (u >= n - 1) return relic.f_table[n - 1];
        const int k = (int)u;
        const double w = u - k;
        return relic.f_table[k] + w * (relic.f_table[k + 1] - relic.f_table[k]);
    }
    if (relic.f_kind == NU_F_FREEZEIN) {
        const double qq = q > 1e-300 ? q : 1e-300;
        return std::exp(-qq) / std::sqrt(qq);
    }
    return 1.0 / (1.0 + std::exp(q - relic.f_p[0]));
}

// FP32 copy of the coefficient table, and with dup != nullptr the packed copy
// with every value stored twice.  The FP32 force tests the NFW edge on y, so
// the C_Q slots, which hold the squared edge for the FP64 force, carry in the
// FP32 tables the bound in y below which a lane takes the rational branch of
// I(y): min(c, kRationalYMax, (1 - 1e-3) R S) with S the stage's
// 1/((1+z) r_s).  The last term matters only while the NFW edge lies beyond R
// (before the collapse onset); its factor keeps every lane below the bound
// inside R whatever the rounding of y.
void fp32_table(const double* tab, int n_steps, const Derived& d, float* out, float* dup)
{
    const double c = d.r_s > 0.0 ? d.r200 / d.r_s : 0.0;
    const double ymax = std::min(c, kRationalYMax);
    for (int n = 0; n < n_steps; ++n) {
        const double* t = tab + (size_t)n * C_COUNT;
        for (int k = 0; k < C_COUNT; ++k) {
            double v = t[k];
            if (k >= C_Q0 && k <= C_Q2)
                v = std::min(ymax, (1.0 - 1e-3) * d.R * t[C_S0 + (k - C_Q0)]);
            const float f = (float)v;
            const size_t j = (size_t)n * C_COUNT + k;
            if (out) out[j] = f;
            if (dup) dup[2 * j] = dup[2 * j + 1] = f;
        }
    }
}

// Eq. eoms in u = ln a: dx/du = (1+z)^2 v / H, dv/du = -gradPhi / H with
// gradPhi = G kappa (1+z) xi M_h Mhat(r,z) x / r^3 (App. A, attractive sign).
// One RK4 step of size -h needs the stage redshifts at u = -n h, -(n+1/2) h and
// -(n+1) h; each is computed from the integer step index (1+z = e^{k h/2}),
// so no time variable is ever accumulated.
void coef_table_into(const nu_cosmo& cosmo, const nu_halo& halo, const Derived& d, int n_steps,
                     double* tab)
{
    const double h = std::log1p(d.z_end) / n_steps;
    auto stage = [&](long k, double& A, double& BF, double& S, double& Q) {
        const double zp1 = std::exp(0.5 * h * (double)k);
        const double z = std::expm1(0.5 * h * (double)k);
        const double H = hubble(cosmo, d, z);
        A = zp1 * zp1 / H;
        const double F = kG * coupling_kappa(halo, z) * zp1 * growth_xi(halo, d, z) * halo.M_h;
        BF = F / H;
        S = d.r_s > 0.0 ? 1.0 / (zp1 * d.r_s) : 0.0;
        // the NFW part ends at r200 (1+z), and nothing acts beyond R, so the
        // edge never exceeds R (it reaches R only at z >= z_i)
        const double rin = std::min(d.r200 * zp1, d.R);
        Q = rin * rin;
    };
    // the end stage of step n is the start stage of step n + 1: each of the
    // 2N + 1 half-step stages is evaluated once
    double Aa, BFa, Sa, Qa;
    stage(0L, Aa, BFa, Sa, Qa);
    for (int n = 0; n < n_steps; ++n) {
        double Am, BFm, Sm, Qm, Ab, BFb, Sb, Qb;
        stage(2L * n + 1, Am, BFm, Sm, Qm);
        stage(2L * n + 2, Ab, BFb, Sb, Qb);
        double* t = tab + (size_t)n * C_COUNT;
        t[C_MA1] = -0.5 * h * Aa;
        t[C_MA2] = -0.5 * h * Am;
        t[C_MA3] = -h * Am;
        t[C_B1] = 0.5 * h * BFa;
        t[C_B2] = 0.5 * h * BFm;
        t[C_B3] = h * BFm;
        t[C_B4] = h / 6.0 * BFb;
        t[C_W0] = -h / 6.0 * Aa;
        t[C_W1] = -h / 3.0 * Am;
        t[C_W2] = -h / 6.0 * Ab;
        t[C_S0] = Sa;
        t[C_S1] = Sm;
        t[C_S2] = Sb;
        t[C_Q0] = Qa;
        t[C_Q1] = Qm;
        t[C_Q2] = Qb;
        t[C_T0] = Sa / d.Ic;
        t[C_T1] = Sm / d.Ic;
        t[C_T2] = Sb / d.Ic;
        t[C_IREM] = h / 6.0 * (Aa + 4.0 * Am + Ab);    // this step's share, summed below
        Aa = Ab;
        BFa = BFb;
        Sa = Sb;
        Qa = Qb;
    }
    // remaining free-streaming distance per unit speed from each step to the end
    double rem = 0.0;
    for (int n = n_steps - 1; n >= 0; --n) {
        rem += tab[(size_t)n * C_COUNT + C_IREM];
        tab[(size_t)n * C_COUNT + C_IREM] = rem;
    }
}

// Requests of a scan often share their halo, background and step grid (a
// list of relic masses, a momentum-grid study): the last few tables are kept,
// keyed by every input the table depends on.
namespace {
struct TableKey {
    double v[14];
    int k[3];
    bool operator==(const TableKey& o) const
    {
        return std::memcmp(v, o.v, sizeof(v)) == 0 && std::memcmp(k, o.k, sizeof(k)) == 0;
    }
};
TableKey table_key(const nu_cosmo& cosmo, const nu_halo& halo, const Derived& d, int n_steps)
{
    TableKey key;
    std::memset(&key, 0, sizeof(key));
    const double v[14] = {cosmo.Om, cosmo.h, halo.M_h, halo.c, halo.z0, halo.xi_p[0],
                          halo.xi_p[1], halo.xi_p[2], halo.kappa_p[0], halo.kappa_p[1],
                          halo.kappa_p[2], d.z_end, 0.0, 0.0};
    std::memcpy(key.v, v, sizeof(v));
    key.k[0] = halo.xi_kind;
    key.k[1] = halo.kappa_kind;
    key.k[2] = n_steps;
    return key;
}
}  // namespace

void coef_table(const nu_cosmo& cosmo, const nu_halo& halo, const Derived& d, int n_steps,
                std::vector<double>& tab)
{
    constexpr size_t kKept = 8;
    static std::mutex mu;
    static std::vector<std::pair<TableKey, std::vector<double>>> kept;   // most recent last
    const TableKey key = table_key(cosmo, halo, d, n_steps);
    {
        std::lock_guard<std::mutex> g(mu);
        for (size_t i = 0; i < kept.size(); ++i) {
            if (kept[i].first == key) {
                tab = kept[i].second;
                std::rotate(kept.begin() + i, kept.begin() + i + 1, kept.end());
                return;
            }
        }
    }
    tab.assign((size_t)n_steps * C_COUNT, 0.0);
    coef_table_into(cosmo, halo, d, n_steps, tab.data());
    std::lock_guard<std::mutex> g(mu);
    if (kept.size() == kKept) kept.erase(kept.begin());
    kept.emplace_back(key, tab);
}

// |P| nodes: log-spaced on [q_min, q_max]; the integral of P^2 f dP is taken
// as the trapezoid rule in ln q of q^3 f, so the weight folded with q^3 is
// returned.  The coarse weights integrate the same range on every other node
// (with one fine interval at the top when n is even) and feed the error estimate.
void log_nodes_into(int n, double q_min, double q_max, double* q, double* wl, double* wlc)
{
    const double lmin = std::log(q_min);
    const double dl = (std::log(q_max) - lmin) / (n - 1);
    for (int j = 0; j < n; ++j) {
        q[j] = std::exp(lmin + dl * j);
        wl[j] = (j == 0 || j == n - 1) ? 0.5 * dl : dl;
        wlc[j] = 0.0;
    }
    if (n < 3) {
        for (int j = 0; j < n; ++j) wlc[j] = wl[j];
    } else {
        const int top = (n % 2 == 1) ? n - 1 : n - 2;   // last even node of the coarse rule
        for (int j = 0; j <= top; j += 2)
            wlc[j] = (j == 0 || j == top) ? dl : 2.0 * dl;
        if (top == n - 2) {                              // finish with one fine interval
            wlc[n - 2] += 0.5 * dl;
            wlc[n - 1] += 0.5 * dl;
        }
    }
    for (int j = 0; j < n; ++j) {
        const double q3 = q[j] * q[j] * q[j];
        wl[j] *= q3;
        wlc[j] *= q3;
    }
}

void log_nodes(int n, double q_min, double q_max, std::vector<double>& q,
               std::vector<double>& wl, std::vector<double>& wlc)
{
    q.assign(n, 0.0);
    wl.assign(n, 0.0);
    wlc.assign(n, 0.0);
    log_nodes_into(n, q_min, q_max, q.data(), wl.data(), wlc.data());
}

// Rules are cached per n (requests of a scan share a few direction grids).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w)
{
    static std::mutex mu;
    static std::map<int, std::pair<std::vector<double>, std::vector<double>>> cache;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(n);
        if (it != cache.end()) {
            x = it->second.first;
            w = it->second.second;
            return;
        }
    }
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    gauss_legendre_into(n, x.data(), w.data());
    std::lock_guard<std::mutex> g(mu);
    if (cache.size() < 4096) cache[n] = {x, w};
}

// Gauss-Legendre rule on [-1, 1]: roots of P_n from Tricomi's asymptotic
// estimate refined by Newton steps, with P_n and P_n' from the three-term
// recurrence; weights 2 / ((1 - x^2) P_n'(x)^2).  Nodes ascend.
void gauss_legendre_into(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) x[i] = w[i] = 0.0;
    const int half = (n + 1) / 2;
    for (int i = 0; i < half; ++i) {
        const double th = kPi * (4.0 * (i + 1) - 1.0) / (4.0 * n + 2.0);
        double r = (1.0 - (n - 1.0) / (8.0 * n * (double)n * n)) * std::cos(th);
        double dp = 1.0;
        for (int it = 0; it < 64; ++it) {
            double p0 = 1.0, p1 = r;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = (n == 1) ? r : p1;
            const double pm = (n == 1) ? 1.0 : p0;
            dp = n * (pm - r * pn) / (1.0 - r * r);
            const double step = pn / dp;
            r -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        double p0 = 1.0, p1 = r;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double pn = (n == 1) ? r : p1;
        const double pm = (n == 1) ? 1.0 : p0;
        dp = n * (pm - r * pn) / (1.0 - r * r);
        const double wi = 2.0 / ((1.0 - r * r) * dp * dp);
        x[n - 1 - i] = r;
        x[i] = -r;
        w[n - 1 - i] = wi;
        w[i] = wi;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

long long device_bytes(int precision, int n_steps, int n_radii, int n_q, int n_mu,
                       int tiles_per_seg, bool keep_qi, int n_mass, int n_ftab, long long* h2d_bytes)
{
    const size_t sz = precision == NU_FP64 ? sizeof(double) : sizeof(float);
    size_t b = 0;
    b += align256(4 * sizeof(unsigned));                       // control words
    b += align256(sizeof(DevProblem));
    b += align256(2 * sizeof(int));                             // tile prefix
    b += align256((size_t)n_steps * C_COUNT * sz);               // coefficient table
    if (precision == NU_MIXED) b += align256((size_t)n_steps * C_COUNT * 2 * sizeof(float));
    b += align256((size_t)n_radii * sz);                         // x0
    b += align256((size_t)n_q * sz);                             // v0
    b += 2 * align256((size_t)n_mu * sz);                        // mu, sin psi
    b += 2 * align256((size_t)n_q * sizeof(double));             // wq, wqc
    b += align256((size_t)n_mu * sizeof(double));                // wmu
    b += align256((size_t)n_mass * 3 * sizeof(double));          // mass scales, normalisations
    b += align256((size_t)(n_ftab > 0 ? n_ftab : 1) * sizeof(double));   // tabulated f (FP64)
    b += align256((size_t)n_radii * sizeof(unsigned));           // per-radius counters (zero)
    if (h2d_bytes) *h2d_bytes = (long long)b;                    // everything above is uploaded
    b += align256((size_t)n_radii * tiles_per_seg * 2 * n_mass * sizeof(double));
    b += 2 * align256((size_t)n_radii * n_mass * sizeof(double));   // out, err
    if (keep_qi) b += align256((size_t)n_radii * n_q * n_mu * sz);
    return (long long)b;
}

}  // namespace nuprof
