// C-ABI of the relic-overdensity library: request handles, batches and the
// host side of every launch.  See include/nuprof.h for the contract of each
// entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "nuprof_internal.h"

using namespace nuprof;

namespace nuprof {
long long launches();
}

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device memory through the caller's allocator or cudaMalloc.
struct DeviceBlock {
    void* ptr = nullptr;
    size_t bytes = 0;
    nu_alloc_fn alloc = nullptr;
    nu_free_fn free = nullptr;
    void* ctx = nullptr;

    int allocate(size_t n, const nu_opts& o)
    {
        alloc = o.alloc;
        free = o.free;
        ctx = o.alloc_ctx;
        bytes = n;
        if (alloc) {
            ptr = alloc(n, ctx);
            return ptr ? NU_OK : NU_ENOMEM;
        }
        if (cudaMalloc(&ptr, n) != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
            return NU_ENOMEM;
        }
        return NU_OK;
    }
    void release()
    {
        if (!ptr) return;
        if (alloc) {
            if (free) free(ptr, bytes, ctx);
        } else {
            cudaFree(ptr);
        }
        ptr = nullptr;
    }
};

// An event shared by every handle that took part in one launch.
struct RunEvent {
    cudaEvent_t ev = nullptr;
    RunEvent() { cudaEventCreateWithFlags(&ev, cudaEventDisableTiming); }
    ~RunEvent()
    {
        if (ev) cudaEventDestroy(ev);
    }
};

int sm_count()
{
    static std::atomic<int> cached{0};
    int v = cached.load();
    if (v) return v;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cached.store(v);
    return v;
}

int persistent_grid(int precision, int tpt, int block, size_t smem, int n_tiles, int* grid,
                    bool gtab = false)
{
    int per_sm = 0;
    const int rc = max_ctas_per_sm(precision, tpt, block, smem, &per_sm, gtab);
    if (rc != NU_OK) return rc;
    const int sms = sm_count();
    if (per_sm < 1 || sms < 1) return NU_ECUDA;
    *grid = std::max(1, std::min(n_tiles, per_sm * sms));
    return NU_OK;
}

}  // namespace

struct nu_profile {
    nu_cosmo cosmo;
    nu_halo halo;
    nu_relic relic;
    nu_pgrid grid;
    nu_opts opts;
    Derived d;
    nu_plan_info info;
    int n_radii = 0;
    int tiles_per_seg = 0;
    int n_tiles = 0;
    size_t smem = 0;
    DeviceBlock mem;
    DevProblem hdp;                 // host copy (device pointers inside)
    DevProblem* d_prob = nullptr;
    int* d_prefix = nullptr;
    unsigned* d_ctrl = nullptr;     // [0] tile counter, [1] status
    std::shared_ptr<RunEvent> last;
    nu_profile* twin = nullptr;     // NU_FLAG_VERIFY: the same request in the FP64 mode
};

struct nu_batch {
    std::vector<nu_profile*> hs;
    int precision = NU_MIXED, tpt = 1, block = 256;
    int n_tiles = 0;
    size_t smem = 0;
    int grid = 0;
    DeviceBlock mem;
    DevProblem* d_probs = nullptr;
    int* d_prefix = nullptr;
    unsigned* d_ctrl = nullptr;
    long long h2d_bytes = 0;
    long long traj_steps = 0;
    unsigned long long* d_tallies = nullptr;   // [5], allocated at the first count
    bool use_graph = false;
    bool timing = false;
    bool gtab = false;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    bool timed_run = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    std::shared_ptr<RunEvent> ev;
};

namespace {

int plan_common(const nu_cosmo* cosmo, const nu_halo* halo, const nu_relic* relic,
                const double* radii, int n_radii, const nu_pgrid* grid, const nu_opts* opts_in,
                nu_opts& o, Derived& d, nu_plan_info& info, int& tiles_per_seg)
{
    resolve_opts(opts_in, o);
    int rc = validate(cosmo, halo, relic, radii, n_radii, grid, &o);
    if (rc != NU_OK) return rc;
    rc = derive(*cosmo, *halo, o, d);
    if (rc != NU_OK) return rc;
    const long long seg = (long long)grid->n_q * grid->n_mu;
    const int tile = o.block * traj_per_thread(o.tpt);
    tiles_per_seg = (int)((seg + tile - 1) / tile);
    std::memset(&info, 0, sizeof(info));
    info.R_kpc = d.R;
    info.r200_kpc = d.r200;
    info.r_s_kpc = d.r_s;
    info.z_i = d.z_i;
    info.Ic = d.Ic;
    info.rho_bar0 = d.rho_bar0;
    info.z_end = d.z_end;
    info.n_traj = seg * n_radii;
    info.traj_steps = info.n_traj * o.n_steps;
    const int tps_alloc = (int)((seg + kMinTile - 1) / kMinTile);
    info.device_bytes = device_bytes(o.precision, o.n_steps, n_radii, grid->n_q, grid->n_mu,
                                     tps_alloc, (o.flags & NU_FLAG_KEEP_QI) != 0,
                                     relic_n_mass(*relic),
                                     relic->f_kind == NU_F_TABLE ? relic->n_table : 0,
                                     &info.h2d_bytes);
    if (o.flags & NU_FLAG_VERIFY) {   // the FP64 twin's buffers come from the same allocator
        long long twin_h2d = 0;
        info.device_bytes += device_bytes(NU_FP64, o.n_steps, n_radii, grid->n_q, grid->n_mu,
                                          tps_alloc, false, relic_n_mass(*relic),
                                          relic->f_kind == NU_F_TABLE ? relic->n_table : 0,
                                          &twin_h2d);
        info.h2d_bytes += twin_h2d;
    }
    const long long nt = (long long)tiles_per_seg * n_radii;
    if (nt > (1LL << 30)) return NU_EINVAL;
    info.n_tiles = (int)nt;
    info.tile = tile;
    info.precision = o.precision;
    info.n_steps = o.n_steps;
    info.n_masses = relic_n_mass(*relic);
    return NU_OK;
}

// Append `n` values of type T (converted from double) to a staging buffer at offset off.
template <typename T>
void put(unsigned char* buf, size_t off, const double* v, size_t n)
{
    T* p = reinterpret_cast<T*>(buf + off);
    for (size_t i = 0; i < n; ++i) p[i] = (T)v[i];
}

// Page-locked host staging for the uploads of create and the reads of
// result: one process-wide buffer that grows to the largest request, held
// under a lock for one copy at a time (copies from page-locked memory run
// as true DMA, without the driver's intermediate bounce).  If page-locked
// memory cannot be had, an ordinary heap buffer is used instead.
class Stage {
public:
    explicit Stage(size_t bytes) : lk_(mu())
    {
        Buf& b = buf();
        if (b.cap < bytes) {
            if (b.p) cudaFreeHost(b.p);
            b.p = nullptr;
            b.cap = 0;
            const size_t want = bytes + bytes / 2;
            if (cudaHostAlloc(reinterpret_cast<void**>(&b.p), want, cudaHostAllocPortable) == cudaSuccess)
                b.cap = want;
            else
                cudaGetLastError();
        }
        if (b.p) {
            p_ = b.p;
        } else {
            heap_.resize(bytes);
            p_ = heap_.data();
        }
    }
    unsigned char* data() { return p_; }
    static size_t capacity()
    {
        std::lock_guard<std::mutex> g(mu());
        return buf().cap;
    }

private:
    struct Buf {
        unsigned char* p = nullptr;
        size_t cap = 0;
    };
    static std::mutex& mu()
    {
        static std::mutex m;
        return m;
    }
    static Buf& buf()
    {
        static Buf b;
        return b;
    }
    std::unique_lock<std::mutex> lk_;
    std::vector<unsigned char> heap_;
    unsigned char* p_ = nullptr;
};

// Enqueue one handle's own launch (work counter and status cleared first).
int launch_profile(nu_profile* h, cudaStream_t s)
{
    int grid = 0;
    const bool gtab = (h->opts.flags & NU_FLAG_GTAB) != 0;
    int rc = persistent_grid(h->opts.precision, h->opts.tpt, h->opts.block, h->smem, h->n_tiles, &grid,
                             gtab);
    if (rc != NU_OK) return rc;
    if (cudaMemsetAsync(h->d_ctrl, 0, 2 * sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    return launch_traj(h->opts.precision, h->opts.tpt, h->opts.block, grid, h->smem, h->d_prob,
                       h->d_prefix, 1, h->n_tiles, h->d_ctrl, s, gtab);
}

// err = |mixed - fp64| / |fp64| per result (0 where both are 0)
void verified_error(const double* mixed, const double* fp64, double* err, int n)
{
    for (int i = 0; i < n; ++i) {
        const double d = std::fabs(mixed[i] - fp64[i]);
        err[i] = d == 0.0 ? 0.0 : d / std::fabs(fp64[i]);
    }
}

}  // namespace

namespace nuprof {

size_t staging_capacity() { return Stage::capacity(); }
int staging_reserve(size_t bytes)
{
    { Stage st(bytes); }   // grows the buffer; its lock is released before the size is read
    return Stage::capacity() >= bytes ? NU_OK : NU_ENOMEM;
}

const DevProblem& profile_desc(const nu_profile* h) { return h->hdp; }
nu_profile* profile_twin(const nu_profile* h) { return h->twin; }
int profile_twin_run(nu_profile* h, void* stream)
{
    if (!h->twin) return NU_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rc = launch_profile(h->twin, s);
    if (rc != NU_OK) return rc;
    auto ev = std::make_shared<RunEvent>();
    if (!ev->ev || cudaEventRecord(ev->ev, s) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    h->twin->last = ev;
    return NU_OK;
}
int profile_twin_query(const nu_profile* h)
{
    if (!h->twin || !h->twin->last) return NU_EBUSY;
    const cudaError_t e = cudaEventQuery(h->twin->last->ev);
    if (e == cudaSuccess) return NU_OK;
    if (e == cudaErrorNotReady) return NU_EAGAIN;
    cudaGetLastError();
    return NU_ECUDA;
}
int profile_n_radii(const nu_profile* h) { return h->n_radii; }
int profile_n_out(const nu_profile* h) { return h->n_radii * h->hdp.n_mass; }
int profile_n_steps(const nu_profile* h) { return h->opts.n_steps; }
long long profile_n_traj(const nu_profile* h) { return h->info.n_traj; }

// Copy n/nbar and the error estimate of the last completed launch touching
// the handle (ordered on `stream`); the caller guarantees that launch is done.
int profile_read(const nu_profile* h, double* out, double* err, void* stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int n = profile_n_out(h);
    const size_t bytes = (size_t)n * sizeof(double);
    if (cudaMemcpyAsync(out, h->hdp.out, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (err && cudaMemcpyAsync(err, h->hdp.err, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(out[i])) return NU_EDEVICE;
    if (h->twin && err) {                 // verified: the error against the FP64 run
        std::vector<double> ref((size_t)n);
        if (cudaMemcpyAsync(ref.data(), h->twin->hdp.out, bytes, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return NU_ECUDA;
        }
        for (int i = 0; i < n; ++i)
            if (!std::isfinite(ref[i])) return NU_EDEVICE;
        verified_error(out, ref.data(), err, n);
    }
    return NU_OK;
}

}  // namespace nuprof

extern "C" {

int nu_version(void) { return NU_VERSION_MAJOR * 10000 + NU_VERSION_MINOR * 100 + NU_VERSION_PATCH; }

const char* nu_strerror(int code)
{
    switch (code) {
    case NU_OK: return "ok";
    case NU_EINVAL: return "invalid argument";
    case NU_ENOMEM: return "out of memory";
    case NU_ECUDA: return "CUDA runtime error";
    case NU_EBUSY: return "no run has been enqueued";
    case NU_ETIMEDOUT: return "timed out";
    case NU_EDEVICE: return "device reported a non-finite result";
    case NU_ENOTSUP: return "unsupported combination";
    case NU_ECANCELED: return "cancelled";
    case NU_EAGAIN: return "not finished yet";
    case NU_ETOOBIG: return "request exceeds the static scratch of the no-allocation entry point";
    default: return "unknown error";
    }
}

long long nu_kernel_launches(void) { return nuprof::launches(); }

int nu_profile_plan(const nu_cosmo* cosmo, const nu_halo* halo, const nu_relic* relic,
                    const double* radii, int n_radii, const nu_pgrid* p_grid,
                    const nu_opts* opts, nu_plan_info* info)
{
    if (!info) return NU_EINVAL;
    nu_opts o;
    Derived d;
    nu_plan_info tmp;
    int tps = 0;
    const int rc = plan_common(cosmo, halo, relic, radii, n_radii, p_grid, opts, o, d, tmp, tps);
    if (rc != NU_OK) return rc;
    *info = tmp;
    return NU_OK;
}

int nu_profile_create(const nu_cosmo* cosmo, const nu_halo* halo, const nu_relic* relic,
                      const double* radii, int n_radii, const nu_pgrid* p_grid,
                      const nu_opts* opts, nu_profile** out)
{
    if (!out) return NU_EINVAL;
    nu_opts o;
    Derived d;
    nu_plan_info info;
    int tps = 0;
    int rc = plan_common(cosmo, halo, relic, radii, n_radii, p_grid, opts, o, d, info, tps);
    if (rc != NU_OK) return rc;

    std::unique_ptr<nu_profile> h(new (std::nothrow) nu_profile());
    if (!h) return NU_ENOMEM;
    h->cosmo = *cosmo;
    h->halo = *halo;
    h->relic = *relic;
    h->relic.masses_eV = nullptr;                         // borrowed: not kept
    h->relic.f_table = nullptr;
    h->grid = *p_grid;
    h->opts = o;
    h->d = d;
    h->info = info;
    h->n_radii = n_radii;
    h->tiles_per_seg = tps;
    h->n_tiles = info.n_tiles;
    h->smem = coef_smem_bytes(o.precision, o.n_steps, o.tpt);

    // ---- host tables (FP64) ----
    const int nq = p_grid->n_q, nmu = p_grid->n_mu, N = o.n_steps;
    std::vector<double> coef, q, wq, wqc, mu, wmu;
    coef_table(*cosmo, *halo, d, N, coef);
    log_nodes(nq, p_grid->q_min, p_grid->q_max, q, wq, wqc);
    gauss_legendre(nmu, mu, wmu);
    const double kT0 = kKB * cosmo->T0_K;                 // eV
    std::vector<double> v0(nq), smu(nmu), x0(n_radii);
    for (int j = 0; j < nq; ++j) v0[j] = kC * q[j] * kT0 / relic->m_eV;   // Sec. II.C: P0 = m v0
    for (int k = 0; k < nmu; ++k) smu[k] = std::sqrt((1.0 - mu[k]) * (1.0 + mu[k]));
    for (int i = 0; i < n_radii; ++i)
        x0[i] = o.radii_unit == NU_RADII_R200 ? radii[i] * d.r200 : radii[i];
    // Masses read from the trajectories (Sec. III): scale s_a = m_a / m and the
    // background of each on the same (scaled) grid.
    const int nm = relic_n_mass(*relic);
    std::vector<double> mass_s(nm), norms(2 * (size_t)nm);
    for (int a = 0; a < nm; ++a) {
        mass_s[a] = relic->n_masses > 0 ? relic->masses_eV[a] / relic->m_eV : 1.0;
        double nb = 0.0, nbc = 0.0;
        for (int j = 0; j < nq; ++j) {
            const double f = relic_f(*relic, mass_s[a] * q[j]);
            nb += wq[j] * f;
            nbc += wqc[j] * f;
        }
        norms[2 * a] = 1.0 / (2.0 * nb);
        norms[2 * a + 1] = 1.0 / (2.0 * nbc);
    }

    // ---- device layout ----
    const bool fp64 = o.precision == NU_FP64;
    const size_t sz = fp64 ? sizeof(double) : sizeof(float);
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t at = off; off += align256(bytes); return at; };
    const size_t o_ctrl = carve(4 * sizeof(unsigned));
    const size_t o_prob = carve(sizeof(DevProblem));
    const size_t o_pref = carve(2 * sizeof(int));
    const size_t o_coef = carve((size_t)N * C_COUNT * sz);
    const size_t o_coef2 = fp64 ? 0 : carve((size_t)N * C_COUNT * 2 * sizeof(float));
    const size_t o_x0 = carve((size_t)n_radii * sz);
    const size_t o_v0 = carve((size_t)nq * sz);
    const size_t o_mu = carve((size_t)nmu * sz);
    const size_t o_smu = carve((size_t)nmu * sz);
    const size_t o_wq = carve((size_t)nq * sizeof(double));
    const size_t o_wqc = carve((size_t)nq * sizeof(double));
    const size_t o_wmu = carve((size_t)nmu * sizeof(double));
    const size_t o_mass = carve((size_t)nm * 3 * sizeof(double));   // scales, then norms
    const int nft = relic->f_kind == NU_F_TABLE ? relic->n_table : 0;
    const size_t o_ftab = carve((size_t)(nft > 0 ? nft : 1) * sizeof(double));   // tabulated f (FP64)
    const size_t o_cnt = carve((size_t)n_radii * sizeof(unsigned));   // zero in the upload image
    const size_t upload_end = off;                         // everything above is uploaded
    // tile sums sized for the smallest tile shape, so that any batch shape fits
    const size_t tps_alloc = (size_t)(((long long)nq * nmu + kMinTile - 1) / kMinTile);
    const size_t o_part = carve((size_t)n_radii * tps_alloc * 2 * nm * sizeof(double));
    const size_t o_out = carve((size_t)n_radii * nm * sizeof(double));
    const size_t o_err = carve((size_t)n_radii * nm * sizeof(double));
    const bool keep_qi = (o.flags & NU_FLAG_KEEP_QI) != 0;
    const size_t o_qi = keep_qi ? carve((size_t)n_radii * nq * nmu * sz) : 0;
    const size_t total = off;

    rc = h->mem.allocate(total, o);
    if (rc != NU_OK) return rc;
    unsigned char* base = static_cast<unsigned char*>(h->mem.ptr);

    DevProblem& P = h->hdp;
    std::memset(&P, 0, sizeof(P));
    P.coef = base + o_coef;
    P.coef2 = fp64 ? nullptr : base + o_coef2;
    P.x0 = base + o_x0;
    P.v0 = base + o_v0;
    P.mu = base + o_mu;
    P.smu = base + o_smu;
    P.wq = reinterpret_cast<const double*>(base + o_wq);
    P.wqc = reinterpret_cast<const double*>(base + o_wqc);
    P.wmu = reinterpret_cast<const double*>(base + o_wmu);
    P.mass_s = reinterpret_cast<const double*>(base + o_mass);
    P.norms = reinterpret_cast<const double*>(base + o_mass) + nm;
    P.partials = reinterpret_cast<double*>(base + o_part);
    P.seg_count = reinterpret_cast<unsigned*>(base + o_cnt);
    P.out = reinterpret_cast<double*>(base + o_out);
    P.err = reinterpret_cast<double*>(base + o_err);
    P.qi = keep_qi ? static_cast<void*>(base + o_qi) : nullptr;
    P.status = reinterpret_cast<int*>(base + o_ctrl + sizeof(unsigned));
    P.q_scale = relic->m_eV / (kC * kT0);                 // Liouville map: q_i = m |v| / (c k_B T0)
    P.invIc = 1.0 / d.Ic;
    P.invR3 = d.R > 0.0 ? 1.0 / (d.R * d.R * d.R) : 0.0;
    P.R2 = d.R * d.R;
    P.c_nfw = d.r_s > 0.0 ? d.r200 / d.r_s : 0.0;     // the NFW edge in y
    P.f_p0 = relic->f_p[0];
    P.f_kind = relic->f_kind;
    if (nft > 0) {
        P.n_ftab = nft;
        P.ftab = base + o_ftab;
        P.ftab_q0 = relic->f_p[0];
        P.ftab_q1 = relic->f_p[1];
        P.ftab_scale = (nft - 1) / std::log(relic->f_p[1] / relic->f_p[0]);
    }
    P.n_radii = n_radii;
    P.n_q = nq;
    P.n_mu = nmu;
    P.n_steps = N;
    P.tiles_per_seg = tps;
    P.tile = o.block * traj_per_thread(o.tpt);
    P.precision = o.precision;
    P.n_mass = nm;

    {   // the page-locked staging buffer is held (under its lock) only for the upload
        Stage staging(upload_end);
        unsigned char* stage = staging.data();
        std::memset(stage, 0, upload_end);
        std::memcpy(stage + o_prob, &P, sizeof(P));
        const int prefix[2] = {0, h->n_tiles};
        std::memcpy(stage + o_pref, prefix, sizeof(prefix));
        if (fp64) {
            put<double>(stage, o_coef, coef.data(), coef.size());
            put<double>(stage, o_x0, x0.data(), n_radii);
            put<double>(stage, o_v0, v0.data(), nq);
            put<double>(stage, o_mu, mu.data(), nmu);
            put<double>(stage, o_smu, smu.data(), nmu);
        } else {
            fp32_table(coef.data(), N, d, reinterpret_cast<float*>(stage + o_coef),
                       reinterpret_cast<float*>(stage + o_coef2));
            put<float>(stage, o_x0, x0.data(), n_radii);
            put<float>(stage, o_v0, v0.data(), nq);
            put<float>(stage, o_mu, mu.data(), nmu);
            put<float>(stage, o_smu, smu.data(), nmu);
        }
        put<double>(stage, o_wq, wq.data(), nq);
        put<double>(stage, o_wqc, wqc.data(), nq);
        put<double>(stage, o_wmu, wmu.data(), nmu);
        put<double>(stage, o_mass, mass_s.data(), nm);
        put<double>(stage, o_mass + nm * sizeof(double), norms.data(), 2 * (size_t)nm);
        if (nft > 0) {
            put<double>(stage, o_ftab, relic->f_table, nft);
        }

        cudaStream_t s = reinterpret_cast<cudaStream_t>(o.stream);
        // one copy and no kernel: a request can be created while a resident server
        // launch holds every SM
        if (cudaMemcpyAsync(base, stage, upload_end, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {   // the staging buffer is reused after this
            cudaGetLastError();
            h->mem.release();
            return NU_ECUDA;
        }
    }
    h->d_prob = reinterpret_cast<DevProblem*>(base + o_prob);
    h->d_prefix = reinterpret_cast<int*>(base + o_pref);
    h->d_ctrl = reinterpret_cast<unsigned*>(base + o_ctrl);
    if (o.flags & NU_FLAG_VERIFY) {       // the same request in the FP64 mode
        nu_opts o2 = o;
        o2.precision = NU_FP64;
        o2.flags = 0;
        o2.block = 256;
        o2.tpt = 1;
        rc = nu_profile_create(cosmo, halo, relic, radii, n_radii, p_grid, &o2, &h->twin);
        if (rc != NU_OK) {
            h->mem.release();
            return rc;
        }
    }
    *out = h.release();
    return NU_OK;
}

int nu_profile_run(nu_profile* h, void* stream)
{
    if (!h) return NU_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = launch_profile(h, s);
    if (rc == NU_OK && h->twin) rc = launch_profile(h->twin, s);
    if (rc != NU_OK) return rc;
    auto ev = std::make_shared<RunEvent>();
    if (!ev->ev || cudaEventRecord(ev->ev, s) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    h->last = ev;
    return NU_OK;
}

int nu_profile_result(nu_profile* h, double* n_over_nbar, double* err_est, int n_radii)
{
    if (!h || !n_over_nbar) return NU_EINVAL;
    if (n_radii != profile_n_out(h)) return NU_EINVAL;
    if (!h->last) return NU_EBUSY;
    if (cudaEventSynchronize(h->last->ev) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    // out and err are adjacent in the device layout: one copy brings both back
    Stage staging((size_t)2 * n_radii * sizeof(double));
    double* tmp = reinterpret_cast<double*>(staging.data());
    const size_t stride = (size_t)(reinterpret_cast<const char*>(h->hdp.err) -
                                   reinterpret_cast<const char*>(h->hdp.out));
    if (cudaMemcpy2D(tmp, n_radii * sizeof(double), h->hdp.out, stride,
                     n_radii * sizeof(double), err_est ? 2 : 1, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    for (int i = 0; i < n_radii; ++i)
        if (!std::isfinite(tmp[i])) return NU_EDEVICE;
    std::memcpy(n_over_nbar, tmp, n_radii * sizeof(double));
    if (err_est && h->twin) {             // verified: the error against the FP64 run
        if (cudaMemcpy(tmp + n_radii, h->twin->hdp.out, n_radii * sizeof(double),
                       cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return NU_ECUDA;
        }
        for (int i = 0; i < n_radii; ++i)
            if (!std::isfinite(tmp[n_radii + i])) return NU_EDEVICE;
        verified_error(n_over_nbar, tmp + n_radii, err_est, n_radii);
    } else if (err_est) {
        std::memcpy(err_est, tmp + n_radii, n_radii * sizeof(double));
    }
    return NU_OK;
}

int nu_profile_qi(nu_profile* h, double* qi, long long n)
{
    if (!h || !qi) return NU_EINVAL;
    if (!h->hdp.qi) return NU_EINVAL;
    const long long total = (long long)h->n_radii * h->grid.n_q * h->grid.n_mu;
    if (n != total) return NU_EINVAL;
    if (!h->last) return NU_EBUSY;
    if (cudaEventSynchronize(h->last->ev) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    if (h->opts.precision == NU_FP64) {
        if (cudaMemcpy(qi, h->hdp.qi, total * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return NU_ECUDA;
        }
        return NU_OK;
    }
    std::vector<float> tmp((size_t)total);
    if (cudaMemcpy(tmp.data(), h->hdp.qi, total * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    for (long long i = 0; i < total; ++i) qi[i] = tmp[(size_t)i];
    return NU_OK;
}

int nu_profile_force(nu_profile* h, int stage, const double* r, int n, double* m)
{
    if (!h || !r || !m || n < 1 || stage < 0 || stage > 2 * h->opts.n_steps) return NU_EINVAL;
    void* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)n * 2 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return NU_ENOMEM;
    }
    double* d_r = static_cast<double*>(buf);
    double* d_m = d_r + n;
    int rc = NU_OK;
    if (cudaMemcpy(d_r, r, (size_t)n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = NU_ECUDA;
    if (rc == NU_OK) rc = launch_force_probe(h->opts.precision, h->d_prob, stage, d_r, n, d_m, nullptr);
    if (rc == NU_OK && cudaMemcpy(m, d_m, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = NU_ECUDA;
    if (rc != NU_OK) cudaGetLastError();
    cudaFree(buf);
    return rc;
}

int nu_profile_info(const nu_profile* h, nu_plan_info* info)
{
    if (!h || !info) return NU_EINVAL;
    *info = h->info;
    return NU_OK;
}

void nu_profile_destroy(nu_profile* h)
{
    if (!h) return;
    if (h->last) cudaEventSynchronize(h->last->ev);
    h->last.reset();
    nu_profile_destroy(h->twin);
    h->mem.release();
    delete h;
}

int nu_batch_create(nu_profile* const* hs, int n, const nu_opts* opts, nu_batch** out)
{
    if (!hs || n < 1 || !out) return NU_EINVAL;
    std::unique_ptr<nu_batch> b(new (std::nothrow) nu_batch());
    if (!b) return NU_ENOMEM;
    // tile shape: opts->block / opts->tpt when given, else the requests' own
    // (which must then agree); precision must always agree
    const int want_block = opts ? opts->block : 0;
    const int want_tpt = opts ? opts->tpt : 0;
    if ((want_block != 0 && (want_block < 64 || want_block > 512 || want_block % 32 != 0)) ||
        (want_tpt != 0 && want_tpt != 1 && want_tpt != 2 && want_tpt != kTptPacked))
        return NU_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return NU_EINVAL;
        const nu_opts& o = hs[i]->opts;
        if (i == 0) {
            b->precision = o.precision;
            b->tpt = want_tpt ? want_tpt : o.tpt;
            b->block = want_block ? want_block : o.block;
        } else if (o.precision != b->precision || (!want_tpt && o.tpt != b->tpt) ||
                   (!want_block && o.block != b->block)) {
            return NU_EINVAL;
        }
        b->hs.push_back(hs[i]);
    }
    if (b->tpt == kTptPacked && b->precision != NU_MIXED) return NU_EINVAL;
    for (int i = 0; i < n; ++i) {
        b->smem = std::max(b->smem, coef_smem_bytes(b->precision, hs[i]->opts.n_steps, b->tpt));
    }
    const int tile = b->block * traj_per_thread(b->tpt);
    std::vector<DevProblem> descs(n);
    std::vector<int> prefix(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        descs[i] = hs[i]->hdp;
        const long long seg = (long long)hs[i]->grid.n_q * hs[i]->grid.n_mu;
        descs[i].tile = tile;
        descs[i].tiles_per_seg = (int)((seg + tile - 1) / tile);
        const long long next = (long long)prefix[i] + (long long)descs[i].tiles_per_seg * hs[i]->n_radii;
        if (next > (1LL << 30)) return NU_EINVAL;
        prefix[i + 1] = (int)next;
    }
    b->n_tiles = prefix[n];

    nu_opts o;
    resolve_opts(opts, o);
    if (opts) b->use_graph = (opts->flags & NU_FLAG_GRAPH) != 0;
    if (opts) b->timing = (opts->flags & NU_FLAG_TIMING) != 0;
    if (opts) b->gtab = (opts->flags & NU_FLAG_GTAB) != 0;
    if (b->timing && (cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess)) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t at = off; off += align256(bytes); return at; };
    const size_t o_ctrl = carve(4 * sizeof(unsigned));
    const size_t o_probs = carve((size_t)n * sizeof(DevProblem));
    const size_t o_pref = carve((size_t)(n + 1) * sizeof(int));
    int rc = b->mem.allocate(off, o);
    if (rc != NU_OK) return rc;
    Stage staging(off);
    unsigned char* stage = staging.data();
    std::memset(stage, 0, off);
    for (int i = 0; i < n; ++i)
        std::memcpy(stage + o_probs + i * sizeof(DevProblem), &descs[i], sizeof(DevProblem));
    std::memcpy(stage + o_pref, prefix.data(), (n + 1) * sizeof(int));
    unsigned char* base = static_cast<unsigned char*>(b->mem.ptr);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(o.stream);
    if (cudaMemcpyAsync(base, stage, off, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        b->mem.release();
        return NU_ECUDA;
    }
    b->h2d_bytes = (long long)off;
    for (int i = 0; i < n; ++i) b->traj_steps += hs[i]->info.traj_steps;
    b->d_ctrl = reinterpret_cast<unsigned*>(base + o_ctrl);
    b->d_probs = reinterpret_cast<DevProblem*>(base + o_probs);
    b->d_prefix = reinterpret_cast<int*>(base + o_pref);
    rc = persistent_grid(b->precision, b->tpt, b->block, b->smem, b->n_tiles, &b->grid, b->gtab);
    if (rc != NU_OK) {
        b->mem.release();
        return rc;
    }
    b->ev = std::make_shared<RunEvent>();
    *out = b.release();
    return NU_OK;
}

static int batch_enqueue(nu_batch* b, cudaStream_t s, bool timed)
{
    if (cudaMemsetAsync(b->d_ctrl, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return NU_ECUDA;
    if (timed && cudaEventRecord(b->t0, s) != cudaSuccess) return NU_ECUDA;
    int rc = launch_traj(b->precision, b->tpt, b->block, b->grid, b->smem, b->d_probs,
                         b->d_prefix, (int)b->hs.size(), b->n_tiles, b->d_ctrl, s, b->gtab);
    if (rc != NU_OK) return rc;
    if (timed && cudaEventRecord(b->t1, s) != cudaSuccess) return NU_ECUDA;
    for (nu_profile* h : b->hs)           // verified requests: their FP64 runs follow
        if (h->twin && (rc = launch_profile(h->twin, s)) != NU_OK) return rc;
    return NU_OK;
}

int nu_batch_run(nu_batch* b, void* stream)
{
    if (!b) return NU_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int rc = NU_OK;
    if (b->use_graph) {
        if (!b->exec) {
            // capture on a private stream (the legacy default stream cannot be
            // captured); the instantiated graph is then replayed on `s`
            if (!b->graph_stream &&
                cudaStreamCreateWithFlags(&b->graph_stream, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                b->graph_stream = nullptr;
                return NU_ECUDA;
            }
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(b->graph_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                cudaGetLastError();
                return NU_ECUDA;
            }
            rc = batch_enqueue(b, b->graph_stream, false);
            const cudaError_t e = cudaStreamEndCapture(b->graph_stream, &g);
            if (rc != NU_OK || e != cudaSuccess) {
                cudaGetLastError();
                if (g) cudaGraphDestroy(g);
                return NU_ECUDA;
            }
            const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                cudaGetLastError();
                b->exec = nullptr;
                return NU_ECUDA;
            }
        }
        if ((b->timing && cudaEventRecord(b->t0, s) != cudaSuccess) ||
            cudaGraphLaunch(b->exec, s) != cudaSuccess ||
            (b->timing && cudaEventRecord(b->t1, s) != cudaSuccess)) {
            cudaGetLastError();
            return NU_ECUDA;
        }
        count_launch();
    } else {
        rc = batch_enqueue(b, s, b->timing);
        if (rc != NU_OK) {
            cudaGetLastError();
            return rc;
        }
    }
    auto ev = std::make_shared<RunEvent>();
    if (!ev->ev || cudaEventRecord(ev->ev, s) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    b->ev = ev;
    b->timed_run = b->timing;
    for (nu_profile* h : b->hs) h->last = ev;
    return NU_OK;
}

int nu_batch_branch_counts(nu_batch* b, void* stream, long long* counts)
{
    if (!b || !counts) return NU_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    constexpr int kTallies = 6;
    if (!b->d_tallies &&
        cudaMalloc(&b->d_tallies, kTallies * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        b->d_tallies = nullptr;
        return NU_ENOMEM;
    }
    unsigned long long host[kTallies] = {0, 0, 0, 0, 0, 0};
    int rc = NU_OK;
    if (cudaMemsetAsync(b->d_tallies, 0, sizeof(host), s) != cudaSuccess ||
        cudaMemsetAsync(b->d_ctrl, 0, 2 * sizeof(unsigned), s) != cudaSuccess)
        rc = NU_ECUDA;
    if (rc == NU_OK)
        rc = launch_traj_tally(b->precision, b->tpt, b->block, b->grid, b->smem, b->d_probs,
                               b->d_prefix, (int)b->hs.size(), b->n_tiles, b->d_ctrl, b->d_tallies, s);
    if (rc == NU_OK && (cudaMemcpyAsync(host, b->d_tallies, sizeof(host), cudaMemcpyDeviceToHost, s) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        rc = NU_ECUDA;
    if (rc != NU_OK) {
        cudaGetLastError();
        return rc;
    }
    for (int k = 0; k < kTallies; ++k) counts[k] = (long long)host[k];
    return NU_OK;
}

int nu_batch_info(const nu_batch* b, int* n_tiles, long long* traj_steps, long long* h2d_bytes,
                  int* grid)
{
    if (!b) return NU_EINVAL;
    if (n_tiles) *n_tiles = b->n_tiles;
    if (traj_steps) *traj_steps = b->traj_steps;
    if (h2d_bytes) *h2d_bytes = b->h2d_bytes;
    if (grid) *grid = b->grid;
    return NU_OK;
}

int nu_batch_kernel_ms(nu_batch* b, float* ms)
{
    if (!b || !ms || !b->timing) return NU_EINVAL;
    if (!b->timed_run) return NU_EBUSY;
    if (cudaEventSynchronize(b->t1) != cudaSuccess || cudaEventElapsedTime(ms, b->t0, b->t1) != cudaSuccess) {
        cudaGetLastError();
        return NU_ECUDA;
    }
    return NU_OK;
}

void nu_batch_destroy(nu_batch* b)
{
    if (!b) return;
    if (b->ev && b->ev->ev) cudaEventSynchronize(b->ev->ev);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph_stream) cudaStreamDestroy(b->graph_stream);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->d_tallies) cudaFree(b->d_tallies);
    b->mem.release();
    delete b;
}

}  // extern "C"
