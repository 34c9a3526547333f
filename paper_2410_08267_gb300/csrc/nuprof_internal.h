// Internal declarations of the relic-overdensity library (not part of the C-ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "nuprof.h"

namespace nuprof {

// Physical constants (kpc, km/s, Msun, eV).
constexpr double kG = 4.30091727e-6;      // kpc (km/s)^2 / Msun
constexpr double kC = 299792.458;         // km/s
constexpr double kKB = 8.617333262e-5;    // eV / K
constexpr double kPi = 3.14159265358979323846;

// Entries of the per-step coefficient table (one RK4 step = 20 values).
// With h = ln(1+z_end)/N, stage redshifts z_a, z_m, z_b at u = -n h, -(n+1/2) h,
// -(n+1) h, A(z) = (1+z)^2/H, B(z) = 1/H and F(z) = G kappa (1+z) xi M_h:
enum CoefSlot {
    C_MA1 = 0,   // -(h/2) A(z_a)        X2 = x + C_MA1 v
    C_MA2,       // -(h/2) A(z_m)        X3 = x + C_MA2 V2
    C_MA3,       // -h A(z_m)            X4 = x + C_MA3 V3
    C_B1,        // (h/2) B F (z_a)      V2 = v + C_B1 m1 x
    C_B2,        // (h/2) B F (z_m)      V3 = v + C_B2 m2 X2
    C_B3,        // h B F (z_m)          V4 = v + C_B3 m3 X3
    C_B4,        // (h/6) B F (z_b)
    C_W0,        // -(h/6) A(z_a)        x' = x + W0 v + W1 (V2+V3) + W2 V4
    C_W1,        // -(h/3) A(z_m)
    C_W2,        // -(h/6) A(z_b)
    C_S0,        // 1/((1+z_a) r_s)      NFW argument scale
    C_S1,        // 1/((1+z_m) r_s)
    C_S2,        // 1/((1+z_b) r_s)
    C_Q0,        // min(r200 (1+z_a), R)^2   squared comoving edge of the NFW part
                 // (FP32 tables: the bound in y of the rational branch, fp32_table)
    C_Q1,
    C_Q2,
    C_T0,        // S(z_a) / I(c)        with rs = S/r: y = r^2 rs, S^2/(I(c) r) = rs T
    C_T1,
    C_T2,
    C_IREM,      // sum over steps k >= n of (h/6)(A_a + 4 A_m + A_b): the comoving
                 // distance per unit speed that a force-free trajectory covers from
                 // the start of step n to z_end (App. B's I_io, for the discrete map)
    C_COUNT
};
static_assert(C_COUNT == 20, "coefficient table layout");
static_assert(C_COUNT % 4 == 0, "a step of the FP32 table is whole 16-byte words");

// Largest dynamic shared memory of one CTA (GB300: 227 KB).  A table that does
// not fit is read through the L1 cache instead of being staged (same values,
// same results).
constexpr size_t kMaxStagedSmem = 232448;

// Halo and background quantities derived on the host in FP64 (Sec. II.B).
struct Derived {
    double H0, rho_bar0, R, z_i, r200, r_s, Ic;
    double xi_zs, xi_ze;   // growth window used by NU_XI_LINEAR
    double z_end;          // resolved end of the backward integration
};

int validate(const nu_cosmo* cosmo, const nu_halo* halo, const nu_relic* relic,
             const double* radii, int n_radii, const nu_pgrid* grid, const nu_opts* opts);
int derive(const nu_cosmo& cosmo, const nu_halo& halo, const nu_opts& opts, Derived& d);
double hubble(const nu_cosmo& cosmo, const Derived& d, double z);
double growth_xi(const nu_halo& halo, const Derived& d, double z);
double coupling_kappa(const nu_halo& halo, double z);
double relic_f(const nu_relic& relic, double q);
// Host tables, written into caller memory (no allocation) or into vectors.
void coef_table_into(const nu_cosmo& cosmo, const nu_halo& halo, const Derived& d, int n_steps,
                     double* table);   // [n_steps][C_COUNT]
// Largest y of the FP32 force's rational approximation of I(y)/y^2.
constexpr double kRationalYMax = 16.0;
// FP32 (and packed FP32) copies of a coefficient table; see host_model.cpp.
void fp32_table(const double* tab, int n_steps, const Derived& d, float* out, float* dup);
void coef_table(const nu_cosmo& cosmo, const nu_halo& halo, const Derived& d, int n_steps,
                std::vector<double>& table);
void log_nodes_into(int n, double q_min, double q_max, double* q, double* wl, double* wl_coarse);
void log_nodes(int n, double q_min, double q_max, std::vector<double>& q,
               std::vector<double>& wl, std::vector<double>& wl_coarse);
void gauss_legendre_into(int n, double* x, double* w);   // computed, not cached
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void resolve_opts(const nu_opts* in, nu_opts& out);
long long device_bytes(int precision, int n_steps, int n_radii, int n_q, int n_mu,
                       int tiles_per_seg, bool keep_qi, int n_mass, int n_ftab, long long* h2d_bytes);
// Number of masses read from one trajectory set (Sec. III mass reuse).
inline int relic_n_mass(const nu_relic& r) { return r.n_masses > 0 ? r.n_masses : 1; }

// Device-visible description of one request (POD, lives in device memory).
struct DevProblem {
    const void* coef;       // [n_steps][C_COUNT] float (mixed) or double (fp64)
    const void* coef2;      // [n_steps][C_COUNT][2] float, every value twice (mixed; packed path)
    const void* x0;         // [n_radii] start radius, kpc
    const void* v0;         // [n_q] start speed, km/s
    const void* mu;         // [n_mu] cos psi
    const void* smu;        // [n_mu] sin psi
    const double* wq;       // [n_q] trapezoid-in-ln q weight x q^3
    const double* wqc;      // [n_q] same on every other node (error estimate)
    const double* wmu;      // [n_mu] Gauss-Legendre weights
    const double* mass_s;   // [n_mass] mass scale s_a = m_a / m (1 for one mass)
    const double* norms;    // [n_mass][2] 1/(2 sum_j wq_j f(s_a q_j)), same with wqc
    double* partials;       // [n_radii][tiles_per_seg][n_mass][2] tile sums
    unsigned* seg_count;    // [n_radii] tiles finished (reset by the finisher)
    double* out;            // [n_mass][n_radii] n/nbar
    double* err;            // [n_mass][n_radii] relative quadrature-error estimate
    void* qi;               // [n_radii][n_q][n_mu] final q in the state precision (optional)
    int* status;            // bit 0: non-finite sum
    double q_scale;         // q_i = |v| * q_scale (fiducial mass)
    double invIc, invR3, R2;
    double c_nfw;           // concentration: the NFW edge in y = r / (r_s (1+z))
    double f_p0;
    int f_kind;
    int n_ftab;             // NU_F_TABLE: nodes of ftab
    const void* ftab;       // NU_F_TABLE: [n_ftab] f values (FP64)
    double ftab_q0;         // first node (k_B T0)
    double ftab_q1;         // last node
    double ftab_scale;      // (n_ftab - 1) / ln(q_last / q_first)
    int n_radii, n_q, n_mu, n_steps;
    int tiles_per_seg, tile;
    int precision;
    int n_mass;
    // Chunked integration (serving): when `state` is set, a launch advances
    // steps [step_begin, step_end) and keeps each trajectory's (x, y, vx, vy)
    // in `state` ([n_radii][n_q][n_mu] of 4 values in the state precision);
    // only the launch that reaches n_steps forms the quadrature.  step_end = 0
    // means n_steps (a whole run).
    void* state;
    int step_begin, step_end;
    // Early completion signal (serving): when set, the CTA that finishes the
    // last radius of the request writes 1 to done_flag (host-mapped memory)
    // after counting the radii in done_count (zeroed before the launch).
    unsigned* done_count;
    volatile unsigned* done_flag;
};

// Work queue of a resident server launch (page-locked host memory that the
// kernel reads through its device pointer).  The host appends requests to the
// launch's descriptor and tile-prefix arrays while it runs and publishes them;
// CTAs that claim a tile not yet published wait for it, each wait bounded.
// `word` holds (state << 32) | published tiles and is changed only by
// compare-and-swap, by the host (publish, close) and by a CTA whose wait ran
// out (expire): so no tile is ever published after a CTA has given up on it.
enum QueueState : unsigned { kQueueOpen = 0u, kQueueClosed = 1u, kQueueExpired = 2u };
struct QueueCtl {
    unsigned long long word;        // (state << 32) | published tiles
    unsigned n_probs;               // descriptors published (written before `word`)
    unsigned want_work;             // set by a CTA that found no published tile
    unsigned long long wait_limit_ns;   // bound on one CTA's wait for a tile
};

// Accessors used by the request server (api.cu).
const DevProblem& profile_desc(const nu_profile* h);
int profile_n_radii(const nu_profile* h);
int profile_n_out(const nu_profile* h);   // n_mass * n_radii result values
int profile_n_steps(const nu_profile* h);
long long profile_n_traj(const nu_profile* h);
int profile_read(const nu_profile* h, double* out, double* err, void* stream);
// The page-locked staging buffer of create and result: its size, and growing
// it (which may synchronize the device: not while a resident launch waits on
// the host).
size_t staging_capacity();
int staging_reserve(size_t bytes);
// NU_FLAG_VERIFY: the FP64 twin of a handle (nullptr without the flag), a
// launch of the twin alone with an event after it, and a query of that event
// (NU_OK done, NU_EAGAIN running, NU_EBUSY never run, NU_ECUDA).
nu_profile* profile_twin(const nu_profile* h);
int profile_twin_run(nu_profile* h, void* stream);
int profile_twin_query(const nu_profile* h);

// Kernel launch helpers (traj_kernel.cu).
int launch_traj(int precision, int tpt, int block, int grid, size_t smem_bytes,
                const DevProblem* d_probs, const int* d_tile_prefix, int n_probs, int n_tiles,
                unsigned* d_tile_counter, void* stream, bool gtab = false,
                QueueCtl* d_queue = nullptr);
int launch_traj_tally(int precision, int tpt, int block, int grid, size_t smem_bytes,
                      const DevProblem* d_probs, const int* d_tile_prefix, int n_probs, int n_tiles,
                      unsigned* d_tile_counter, unsigned long long* d_tallies, void* stream);
int max_ctas_per_sm(int precision, int tpt, int block, size_t smem_bytes, int* out,
                    bool gtab = false);
// Smallest tile (block 64 x 1 trajectory): request buffers of tile sums are
// sized for it, so a batch may run any tile shape over existing requests.
constexpr int kMinTile = 64;
size_t coef_smem_bytes(int precision, int n_steps, int tpt);
// Trajectories per thread of a tile shape: tpt 3 is two trajectories per
// thread in packed FP32x2 arithmetic (mixed precision only).
inline int traj_per_thread(int tpt) { return tpt == 3 ? 2 : tpt; }
constexpr int kTptPacked = 3;
int launch_force_probe(int precision, const DevProblem* d_prob, int stage, const double* d_r, int n,
                       double* d_out, void* stream);
void count_launch();

}  // namespace nuprof
