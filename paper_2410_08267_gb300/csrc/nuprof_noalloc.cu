// Overdensity profiles for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a framework that
// owns every device allocation through its own pool, real-time or embedded
// hosts that forbid allocation after start-up, or code that must not touch the
// allocator while another component is capturing work.  For them,
// nu_profile_compute_noalloc runs one request through the same trajectory
// kernel as nu_profile_run, but every device buffer the kernel needs (the
// request descriptor, the per-step coefficient table, the quadrature nodes and
// weights, the per-tile partial sums, the per-radius completion counters and
// the work counter) lives in one file-scope __device__ array of fixed size.
// Host-side tables are built in a static host buffer of the same size, so the
// call performs no heap allocation either.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "nuprof_internal.h"

namespace nuprof {
namespace {

constexpr size_t kArenaBytes = NU_NOALLOC_MAX_BYTES;
constexpr int kMaxDevices = 64;

// Device scratch shared by every call on a GPU; every GPU that loads the
// library holds it until the process exits.  In host code this name is only a
// host-side stand-in: the device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_arena[kArenaBytes];

// Host staging of the uploaded part of the arena (static: no heap allocation).
alignas(256) unsigned char g_stage[kArenaBytes];
std::mutex g_lock;
void* g_arena_dev[kMaxDevices];      // device address of g_arena, per device

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of the arena on the current device (looked up once per device).
int arena_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return NU_ENOTSUP;
    if (!g_arena_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_arena) != cudaSuccess || !p) {
            cudaGetLastError();
            return NU_ECUDA;
        }
        g_arena_dev[dev] = p;
    }
    *out = g_arena_dev[dev];
    return NU_OK;
}

// The per-step coefficient table, written into caller memory (the same
// stage definitions as the table of nu_profile_create: Eq. eoms in ln a with
// the App. A gradient at u = -n h, -(n+1/2) h, -(n+1) h).
void coef_table_into(const nu_cosmo& cosmo, const nu_halo& halo, const Derived& d, int n_steps,
                     double* tab)
{
    const double h = std::log1p(d.z_end) / n_steps;
    for (int n = 0; n < n_steps; ++n) {
        double A[3], BF[3], S[3], Q[3];
        for (int s = 0; s < 3; ++s) {
            const double k = 2.0 * n + s;
            const double zp1 = std::exp(0.5 * h * k);
            const double z = std::expm1(0.5 * h * k);
            const double H = hubble(cosmo, d, z);
            A[s] = zp1 * zp1 / H;
            BF[s] = kG * coupling_kappa(halo, z) * zp1 * growth_xi(halo, d, z) * halo.M_h / H;
            S[s] = d.r_s > 0.0 ? 1.0 / (zp1 * d.r_s) : 0.0;
            const double rin = std::min(d.r200 * zp1, d.R);   // edge never beyond R
            Q[s] = rin * rin;
        }
        double* t = tab + (size_t)n * C_COUNT;
        t[C_MA1] = -0.5 * h * A[0];
        t[C_MA2] = -0.5 * h * A[1];
        t[C_MA3] = -h * A[1];
        t[C_B1] = 0.5 * h * BF[0];
        t[C_B2] = 0.5 * h * BF[1];
        t[C_B3] = h * BF[1];
        t[C_B4] = h / 6.0 * BF[2];
        t[C_W0] = -h / 6.0 * A[0];
        t[C_W1] = -h / 3.0 * A[1];
        t[C_W2] = -h / 6.0 * A[2];
        t[C_S0] = S[0];
        t[C_S1] = S[1];
        t[C_S2] = S[2];
        t[C_Q0] = Q[0];
        t[C_Q1] = Q[1];
        t[C_Q2] = Q[2];
        t[C_T0] = S[0] / d.Ic;
        t[C_T1] = S[1] / d.Ic;
        t[C_T2] = S[2] / d.Ic;
        t[C_PAD] = 0.0;
    }
}

// Log-spaced q nodes with trapezoid-in-ln q weights times q^3 (fine and
// every-other-node rules), as in nu_profile_create.
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
        const int top = (n % 2 == 1) ? n - 1 : n - 2;
        for (int j = 0; j <= top; j += 2) wlc[j] = (j == 0 || j == top) ? dl : 2.0 * dl;
        if (top == n - 2) {
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

// Gauss-Legendre nodes (ascending) and weights on [-1, 1]: Newton iteration
// from Tricomi's estimate, as in nu_profile_create.
void gauss_legendre_into(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) x[i] = w[i] = 0.0;
    const int half = (n + 1) / 2;
    for (int i = 0; i < half; ++i) {
        const double th = kPi * (4.0 * (i + 1) - 1.0) / (4.0 * n + 2.0);
        double r = (1.0 - (n - 1.0) / (8.0 * n * (double)n * n)) * std::cos(th);
        for (int it = 0; it < 64; ++it) {
            double p0 = 1.0, p1 = r;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = (n == 1) ? r : p1;
            const double pm = (n == 1) ? 1.0 : p0;
            const double dp = n * (pm - r * pn) / (1.0 - r * r);
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
        const double dp = n * (pm - r * pn) / (1.0 - r * r);
        const double wi = 2.0 / ((1.0 - r * r) * dp * dp);
        x[n - 1 - i] = r;
        x[i] = -r;
        w[n - 1 - i] = wi;
        w[i] = wi;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

template <typename T>
void put_into(unsigned char* base, size_t off, const double* v, size_t n)
{
    T* p = reinterpret_cast<T*>(base + off);
    for (size_t i = 0; i < n; ++i) p[i] = (T)v[i];
}

}  // namespace
}  // namespace nuprof

using namespace nuprof;

extern "C" int nu_profile_compute_noalloc(const nu_cosmo* cosmo, const nu_halo* halo,
                                          const nu_relic* relic, const double* radii, int n_radii,
                                          const nu_pgrid* p_grid, const nu_opts* opts,
                                          double* n_over_nbar, double* err_est, void* stream)
{
    if (!n_over_nbar) return NU_EINVAL;
    nu_opts o;
    resolve_opts(opts, o);
    if (o.flags != 0) return NU_EINVAL;
    if (o.tpt == kTptPacked) return NU_ENOTSUP;   // the packed table is not staged here
    if (relic && relic->n_masses > 0) return NU_ENOTSUP;   // one mass per call
    if (relic && relic->f_kind == NU_F_TABLE) return NU_ENOTSUP;   // closed-form f only
    int rc = validate(cosmo, halo, relic, radii, n_radii, p_grid, &o);
    if (rc != NU_OK) return rc;
    Derived d;
    rc = derive(*cosmo, *halo, o, d);
    if (rc != NU_OK) return rc;

    const int nq = p_grid->n_q, nmu = p_grid->n_mu, N = o.n_steps;
    const long long seg = (long long)nq * nmu;
    const int tile = o.block * o.tpt;
    const long long tps_ll = (seg + tile - 1) / tile;
    const long long n_tiles_ll = tps_ll * n_radii;
    if (n_tiles_ll > (1LL << 30)) return NU_ETOOBIG;
    const int tps = (int)tps_ll, n_tiles = (int)n_tiles_ll;

    // arena layout (the same order as the buffers of nu_profile_create)
    const bool fp64 = o.precision == NU_FP64;
    const size_t sz = fp64 ? sizeof(double) : sizeof(float);
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t at = off; off += up256(bytes); return at; };
    const size_t o_ctrl = carve(4 * sizeof(unsigned));
    const size_t o_prob = carve(sizeof(DevProblem));
    const size_t o_pref = carve(2 * sizeof(int));
    const size_t o_coef = carve((size_t)N * C_COUNT * sz);
    const size_t o_x0 = carve((size_t)n_radii * sz);
    const size_t o_v0 = carve((size_t)nq * sz);
    const size_t o_mu = carve((size_t)nmu * sz);
    const size_t o_smu = carve((size_t)nmu * sz);
    const size_t o_wq = carve((size_t)nq * sizeof(double));
    const size_t o_wqc = carve((size_t)nq * sizeof(double));
    const size_t o_wmu = carve((size_t)nmu * sizeof(double));
    const size_t o_mass = carve(3 * sizeof(double));      // mass scale 1, two normalisations
    const size_t upload_end = off;
    const size_t o_part = carve((size_t)n_radii * tps * 2 * sizeof(double));
    const size_t o_cnt = carve((size_t)n_radii * sizeof(unsigned));
    const size_t o_out = carve((size_t)n_radii * sizeof(double));
    const size_t o_err = carve((size_t)n_radii * sizeof(double));
    // host scratch for the FP64 tables, placed after the uploaded image
    const size_t h_coef = carve((size_t)N * C_COUNT * sizeof(double));
    const size_t h_q = carve((size_t)nq * sizeof(double) * 3);
    const size_t h_mu = carve((size_t)nmu * sizeof(double) * 3);
    const size_t h_x0 = carve((size_t)n_radii * sizeof(double));
    const size_t h_out = carve((size_t)n_radii * 2 * sizeof(double));
    if (off > kArenaBytes) return NU_ETOOBIG;

    std::lock_guard<std::mutex> guard(g_lock);
    void* arena = nullptr;
    rc = arena_address(&arena);
    if (rc != NU_OK) return rc;
    unsigned char* dev = static_cast<unsigned char*>(arena);
    unsigned char* st = g_stage;
    std::memset(st, 0, upload_end);

    // ---- FP64 tables in the host scratch part of the static buffer ----
    double* coef = reinterpret_cast<double*>(st + h_coef);
    double* q = reinterpret_cast<double*>(st + h_q);
    double* wq = q + nq;
    double* wqc = q + 2 * nq;
    double* mu = reinterpret_cast<double*>(st + h_mu);
    double* wmu = mu + nmu;
    double* smu = mu + 2 * nmu;
    double* x0 = reinterpret_cast<double*>(st + h_x0);
    coef_table_into(*cosmo, *halo, d, N, coef);
    log_nodes_into(nq, p_grid->q_min, p_grid->q_max, q, wq, wqc);
    gauss_legendre_into(nmu, mu, wmu);
    const double kT0 = kKB * cosmo->T0_K;
    double nb = 0.0, nbc = 0.0;
    for (int j = 0; j < nq; ++j) {
        const double f = relic_f(*relic, q[j]);
        nb += wq[j] * f;
        nbc += wqc[j] * f;
        q[j] = kC * q[j] * kT0 / relic->m_eV;             // now the start speed v0 (km/s)
    }
    for (int k = 0; k < nmu; ++k) smu[k] = std::sqrt((1.0 - mu[k]) * (1.0 + mu[k]));
    for (int i = 0; i < n_radii; ++i)
        x0[i] = o.radii_unit == NU_RADII_R200 ? radii[i] * d.r200 : radii[i];

    DevProblem P;
    std::memset(&P, 0, sizeof(P));
    P.coef = dev + o_coef;
    P.x0 = dev + o_x0;
    P.v0 = dev + o_v0;
    P.mu = dev + o_mu;
    P.smu = dev + o_smu;
    P.wq = reinterpret_cast<const double*>(dev + o_wq);
    P.wqc = reinterpret_cast<const double*>(dev + o_wqc);
    P.wmu = reinterpret_cast<const double*>(dev + o_wmu);
    P.mass_s = reinterpret_cast<const double*>(dev + o_mass);
    P.norms = reinterpret_cast<const double*>(dev + o_mass) + 1;
    P.partials = reinterpret_cast<double*>(dev + o_part);
    P.seg_count = reinterpret_cast<unsigned*>(dev + o_cnt);
    P.out = reinterpret_cast<double*>(dev + o_out);
    P.err = reinterpret_cast<double*>(dev + o_err);
    P.qi = nullptr;
    P.status = reinterpret_cast<int*>(dev + o_ctrl + sizeof(unsigned));
    P.q_scale = relic->m_eV / (kC * kT0);
    P.invIc = 1.0 / d.Ic;
    P.invR3 = d.R > 0.0 ? 1.0 / (d.R * d.R * d.R) : 0.0;
    P.R2 = d.R * d.R;
    P.f_p0 = relic->f_p[0];
    P.f_kind = relic->f_kind;
    P.n_radii = n_radii;
    P.n_q = nq;
    P.n_mu = nmu;
    P.n_steps = N;
    P.tiles_per_seg = tps;
    P.tile = tile;
    P.precision = o.precision;
    P.n_mass = 1;

    // ---- uploaded image: control words (zero), descriptor, prefix, tables ----
    std::memcpy(st + o_prob, &P, sizeof(P));
    const int prefix[2] = {0, n_tiles};
    std::memcpy(st + o_pref, prefix, sizeof(prefix));
    if (fp64) {
        put_into<double>(st, o_coef, coef, (size_t)N * C_COUNT);
        put_into<double>(st, o_x0, x0, n_radii);
        put_into<double>(st, o_v0, q, nq);
        put_into<double>(st, o_mu, mu, nmu);
        put_into<double>(st, o_smu, smu, nmu);
    } else {
        put_into<float>(st, o_coef, coef, (size_t)N * C_COUNT);
        put_into<float>(st, o_x0, x0, n_radii);
        put_into<float>(st, o_v0, q, nq);
        put_into<float>(st, o_mu, mu, nmu);
        put_into<float>(st, o_smu, smu, nmu);
    }
    put_into<double>(st, o_wq, wq, nq);
    put_into<double>(st, o_wqc, wqc, nq);
    put_into<double>(st, o_wmu, wmu, nmu);
    const double mass[3] = {1.0, 1.0 / (2.0 * nb), 1.0 / (2.0 * nbc)};
    put_into<double>(st, o_mass, mass, 3);

    int per_sm = 0, sms = 0, devid = 0;
    const size_t smem = coef_smem_bytes(o.precision, N, o.tpt);
    rc = max_ctas_per_sm(o.precision, o.tpt, o.block, smem, &per_sm);
    if (rc != NU_OK) return rc;
    if (cudaGetDevice(&devid) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devid) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    const int grid = n_tiles < per_sm * sms ? n_tiles : per_sm * sms;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // The arena keeps the previous call's contents: the control words (work
    // counter, status) are part of the zeroed upload and the per-radius
    // completion counters are cleared explicitly.
    if (cudaMemcpyAsync(dev, st, upload_end, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(dev + o_cnt, 0, (size_t)n_radii * sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    rc = launch_traj(o.precision, o.tpt, o.block, grid, smem,
                     reinterpret_cast<const DevProblem*>(dev + o_prob),
                     reinterpret_cast<const int*>(dev + o_pref), 1, n_tiles,
                     reinterpret_cast<unsigned*>(dev + o_ctrl), stream);
    if (rc != NU_OK) {
        cudaGetLastError();
        return rc;
    }
    double* host_out = reinterpret_cast<double*>(st + h_out);
    if (cudaMemcpyAsync(host_out, dev + o_out, (size_t)n_radii * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(host_out + n_radii, dev + o_err, (size_t)n_radii * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    for (int i = 0; i < n_radii; ++i)
        if (!std::isfinite(host_out[i])) return NU_EDEVICE;
    std::memcpy(n_over_nbar, host_out, (size_t)n_radii * sizeof(double));
    if (err_est) std::memcpy(err_est, host_out + n_radii, (size_t)n_radii * sizeof(double));
    return NU_OK;
}
