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
// The host tables are built by the same routines as nu_profile_create, written
// into a static host buffer, so the call performs no heap allocation either.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>

#include "nuprof_internal.h"

namespace nuprof {
namespace {

constexpr size_t kArenaBytes = NU_NOALLOC_MAX_BYTES;
constexpr int kMaxDevices = 64;
constexpr double kDefaultTimeoutMs = 60000.0;

// Device scratch shared by every call on a GPU; every GPU that loads the
// library holds it until the process exits.  In host code this name is only a
// host-side stand-in: the device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_arena[kArenaBytes];

// Host side of a call: the staged upload image of the arena at the front,
// then the FP64 tables and the read-back results (static: no heap allocation).
alignas(256) unsigned char g_stage[kArenaBytes];
std::mutex g_lock;

// Per device: a call whose wait ran out left its work on `stream`; the array
// is not touched again until that stream has drained.
struct Pending {
    bool active = false;
    cudaStream_t stream = nullptr;
};
Pending g_pending[kMaxDevices];

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// Wait until every operation enqueued on `s` so far has finished, for at most
// timeout_ms: NU_OK, NU_ETIMEDOUT, or NU_ECUDA if the stream reports an error.
int wait_bounded(cudaStream_t s, double timeout_ms)
{
    using clock = std::chrono::steady_clock;
    const auto t0 = clock::now();
    for (int it = 0;; ++it) {
        const cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) return NU_OK;
        if (e != cudaErrorNotReady) {
            cudaGetLastError();
            return NU_ECUDA;
        }
        const double ms = std::chrono::duration<double, std::milli>(clock::now() - t0).count();
        if (ms >= timeout_ms) return NU_ETIMEDOUT;
        if (it < 2000)
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
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
    if (o.flags != 0 || o.timeout_ms < 0.0) return NU_EINVAL;
    if (o.tpt == kTptPacked) return NU_ENOTSUP;   // the packed table is not staged here
    if (relic && relic->n_masses > 0) return NU_ENOTSUP;   // one mass per call
    if (relic && relic->f_kind == NU_F_TABLE) return NU_ENOTSUP;   // closed-form f only
    int rc = validate(cosmo, halo, relic, radii, n_radii, p_grid, &o);
    if (rc != NU_OK) return rc;
    Derived d;
    rc = derive(*cosmo, *halo, o, d);
    if (rc != NU_OK) return rc;
    const double timeout_ms = o.timeout_ms > 0.0 ? o.timeout_ms : kDefaultTimeoutMs;

    const int nq = p_grid->n_q, nmu = p_grid->n_mu, N = o.n_steps;
    const long long seg = (long long)nq * nmu;
    const int tile = o.block * o.tpt;
    const long long tps_ll = (seg + tile - 1) / tile;
    const long long n_tiles_ll = tps_ll * n_radii;
    if (n_tiles_ll > (1LL << 30)) return NU_ETOOBIG;
    const int tps = (int)tps_ll, n_tiles = (int)n_tiles_ll;

    // Device layout (the same order as the buffers of nu_profile_create).
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
    if (off > kArenaBytes) return NU_ETOOBIG;             // the device array
    // Host layout of the static staging buffer: the upload image, then the
    // FP64 tables and the read-back results.
    size_t hoff = upload_end;
    auto hcarve = [&](size_t bytes) { size_t at = hoff; hoff += up256(bytes); return at; };
    const size_t h_coef = hcarve((size_t)N * C_COUNT * sizeof(double));
    const size_t h_q = hcarve((size_t)nq * sizeof(double) * 3);
    const size_t h_mu = hcarve((size_t)nmu * sizeof(double) * 3);
    const size_t h_x0 = hcarve((size_t)n_radii * sizeof(double));
    const size_t h_out = hcarve((size_t)n_radii * 2 * sizeof(double));
    if (hoff > kArenaBytes) return NU_ETOOBIG;            // the host buffer

    std::lock_guard<std::mutex> guard(g_lock);
    int dev_id = 0;
    if (cudaGetDevice(&dev_id) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    if (dev_id < 0 || dev_id >= kMaxDevices) return NU_ENOTSUP;
    Pending& pend = g_pending[dev_id];
    if (pend.active) {                                    // a timed-out call's work may still run
        rc = wait_bounded(pend.stream, timeout_ms);
        if (rc != NU_OK) return rc;
        pend.active = false;
    }
    // Device address of the array on the current device, looked up on every
    // call (a context re-created after a reset may place it elsewhere).
    void* arena = nullptr;
    if (cudaGetSymbolAddress(&arena, g_arena) != cudaSuccess || !arena) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    unsigned char* dev = static_cast<unsigned char*>(arena);
    unsigned char* st = g_stage;
    std::memset(st, 0, upload_end);

    // ---- FP64 tables (the routines of nu_profile_create) in the host part ----
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
        const double f = relic_f(*relic, 1.0 * q[j]);
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
    P.c_nfw = d.r_s > 0.0 ? d.r200 / d.r_s : 0.0;     // the NFW edge in y
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
        fp32_table(coef, N, d, reinterpret_cast<float*>(st + o_coef), nullptr);
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

    int per_sm = 0, sms = 0;
    const size_t smem = coef_smem_bytes(o.precision, N, o.tpt);
    rc = max_ctas_per_sm(o.precision, o.tpt, o.block, smem, &per_sm);
    if (rc != NU_OK) return rc;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    const int grid = n_tiles < per_sm * sms ? n_tiles : per_sm * sms;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: the control words (work
    // counter, status) are part of the zeroed upload and the per-radius
    // completion counters are cleared explicitly.
    if (cudaMemcpyAsync(dev, st, upload_end, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(dev + o_cnt, 0, (size_t)n_radii * sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        // nothing may still read the staging buffer or write the array
        if (wait_bounded(s, timeout_ms) != NU_OK) pend = {true, s};
        return NU_ECUDA;
    }
    rc = launch_traj(o.precision, o.tpt, o.block, grid, smem,
                     reinterpret_cast<const DevProblem*>(dev + o_prob),
                     reinterpret_cast<const int*>(dev + o_pref), 1, n_tiles,
                     reinterpret_cast<unsigned*>(dev + o_ctrl), stream);
    if (rc != NU_OK) cudaGetLastError();
    // Wait for this call's own work (bounded) before reading back: a copy
    // into the (pageable) static buffer would block until the kernel ends.
    // If the work does not finish in time, later calls wait for it before
    // they touch the array.
    int wrc = wait_bounded(s, timeout_ms);
    if (wrc == NU_ETIMEDOUT) pend = {true, s};
    if (rc != NU_OK) return rc;
    if (wrc != NU_OK) return wrc;
    double* host_out = reinterpret_cast<double*>(st + h_out);
    if (cudaMemcpyAsync(host_out, dev + o_out, (size_t)n_radii * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(host_out + n_radii, dev + o_err, (size_t)n_radii * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        cudaGetLastError();
        if (wait_bounded(s, timeout_ms) != NU_OK) pend = {true, s};
        return NU_ECUDA;
    }
    wrc = wait_bounded(s, timeout_ms);
    if (wrc == NU_ETIMEDOUT) pend = {true, s};
    if (wrc != NU_OK) return wrc;
    for (int i = 0; i < n_radii; ++i)
        if (!std::isfinite(host_out[i])) return NU_EDEVICE;
    std::memcpy(n_over_nbar, host_out, (size_t)n_radii * sizeof(double));
    if (err_est) std::memcpy(err_est, host_out + n_radii, (size_t)n_radii * sizeof(double));
    return NU_OK;
}
