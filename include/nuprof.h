/*
 * nuprof.h -- C-ABI of the GB300 (sm_103a) relic-overdensity library.
 *
 * The library computes the present-day number-density profile n/nbar of a
 * non-cold relic (massive neutrinos by default) around a spherically symmetric,
 * growing, mass-compensated NFW dark-matter halo in a flat FRW background, by
 * the backward N-1-body method of Worku, Sabti & Kamionkowski (arXiv:2410.08267):
 *
 *   1. halo derivation: R, z_i, r200, r_s, I(c) from (M_h, c)        Sec. II.B
 *   2. one test-particle trajectory per (radius x0, momentum |P0|, direction
 *      mu = cos psi), started at x = (x0, 0), v = v0 (mu, sin psi)   Sec. II.C
 *   3. integration of the equations of motion backward from z0 = 0 to
 *      z_end through the closed-form potential gradient            Eq. eoms, App. A
 *      (classical RK4 in u = ln a with a fixed number of steps)
 *   4. Liouville map f0(x0, P0, mu) = f_init(P_i)                 Sec. II.C
 *   5. momentum/direction quadrature divided by the background    Eq. localdensity
 *
 * All work runs in hand-written CUDA kernels on one GPU.  There is no CPU
 * fallback: every entry point that needs the device returns NU_ECUDA when no
 * usable GPU is present.
 *
 * Conventions used by every entry point:
 *   - Units: comoving length in kpc, velocity in km/s, mass in Msun, relic
 *     mass in eV, momentum q in units of k_B T0.  Physical constants are fixed
 *     inside the library: G = 4.30091727e-6 kpc (km/s)^2/Msun,
 *     c = 299792.458 km/s, k_B = 8.617333262e-5 eV/K, H0 = 0.1 h km/s/kpc.
 *   - Gravity is attractive: the printed signs of the Poisson equation and of
 *     App. A are read as a typo (together with Eq. eoms they would repel).
 *   - Return values: NU_OK (0) on success, a negative NU_E* code otherwise;
 *     nu_strerror() names it.  On failure no output argument is written.
 *   - Ownership: every pointer argument is borrowed for the duration of the
 *     call only; the library copies what it keeps.  Handles returned through
 *     `out` arguments are owned by the caller and released by the matching
 *     *_destroy call.
 *   - Streams are passed as `void*` holding a cudaStream_t (NULL = the legacy
 *     default stream).  Calls on one handle must not overlap in time on
 *     different streams (they share the handle's device buffers).
 *   - Threading: distinct handles may be used from distinct host threads.
 */
#ifndef NUPROF_H
#define NUPROF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every entry point is exported from the shared library with default visibility. */
#if defined(__GNUC__)
#define NU_API __attribute__((visibility("default")))
#else
#define NU_API
#endif

#define NU_VERSION_MAJOR 1
#define NU_VERSION_MINOR 1
#define NU_VERSION_PATCH 0

/* ---- error codes ---------------------------------------------------------- */
#define NU_OK          0
#define NU_EINVAL     -1   /* an argument is out of range or inconsistent      */
#define NU_ENOMEM     -2   /* device or host allocation failed / over budget   */
#define NU_ECUDA      -3   /* a CUDA runtime call failed (no GPU, launch error) */
#define NU_EBUSY      -4   /* result asked for before any run was enqueued     */
#define NU_ETIMEDOUT  -5   /* a bounded wait ran out                           */
#define NU_EDEVICE    -6   /* the device status word reports a non-finite sum  */
#define NU_ENOTSUP    -7   /* valid but unsupported combination                */
#define NU_ECANCELED  -8   /* serving: the request was cancelled               */
#define NU_EAGAIN     -9   /* serving: the request is not finished yet         */
#define NU_ETOOBIG   -10   /* the request needs more than the static scratch
                              of nu_profile_compute_noalloc                    */

/* ---- halo growth xi(z) (Eq. rhototal; Sec. IV.A variants) ------------------ */
#define NU_XI_STATIC  0    /* xi = 1 at every z: the NFW halo exists throughout */
#define NU_XI_LINEAR  1    /* xi = clamp((z_s - z)/(z_s - z_e), 0, 1)^alpha;
                              xi_p = {alpha (<=0 -> 1), z_s (<=0 -> z_i), z_e (<=0 -> z0)} */
#define NU_XI_EXP     2    /* xi = exp(-lambda z); xi_p[0] = lambda (mass history M0 e^{-lambda z}) */

/* ---- coupling kappa(z) multiplying G (Sec. IV.B) --------------------------- */
#define NU_KAPPA_ONE    0  /* kappa = 1                                       */
#define NU_KAPPA_POW1PZ 1  /* kappa = (1+z)^gamma = a^-gamma; kappa_p[0] = gamma */
#define NU_KAPPA_PAPER  2  /* kappa = 1 + alpha (z/(1+z))^beta; kappa_p = {alpha, beta} */
#define NU_KAPPA_CONST  3  /* kappa = kappa_p[0]                              */

/* ---- initial relic distribution f(q), q = P / (k_B T0) (Sec. II.C, IV.B) -- */
#define NU_F_FD        0   /* Fermi-Dirac 1/(1+exp(q - eta)); f_p[0] = eta     */
#define NU_F_FREEZEIN  1   /* non-thermal q^(-1/2) exp(-q)                     */
#define NU_F_TABLE     2   /* tabulated f (the spectral distortions and other
                              relics of Sec. IV.B): f_table[k] = f(q_k) at
                              q_k = f_p[0] (f_p[1]/f_p[0])^(k/(n_table-1)),
                              k = 0 .. n_table-1; f is linear in ln q between
                              nodes, f_table[0] below f_p[0] and 0 above f_p[1] */
#define NU_MAX_FTABLE  4096

/* ---- precision modes ------------------------------------------------------ */
#define NU_FP64   0        /* state, force, f and sums in FP64                 */
#define NU_MIXED  1        /* FP32 state and force; time from an FP64-built
                              table; Liouville map, f and quadrature sums in
                              FP64                                             */

/* ---- radius units ---------------------------------------------------------- */
#define NU_RADII_KPC   0   /* comoving kpc                                     */
#define NU_RADII_R200  1   /* units of r200, the physical virial radius at z0  */

/* ---- option flags ---------------------------------------------------------- */
#define NU_FLAG_KEEP_QI  1 /* keep the final momentum q_i of every trajectory
                              (phase-space integrand, Fig. 3 of the paper)     */
#define NU_FLAG_GRAPH    2 /* batches: capture the launch in a CUDA graph      */
#define NU_FLAG_TIMING   4 /* batches: record CUDA events around the trajectory
                              kernel (read with nu_batch_kernel_ms)            */
#define NU_FLAG_GTAB     8 /* runs and batches: read the per-step coefficient
                              table in place through the L1 cache instead of
                              staging it in shared memory (frees shared memory,
                              so more CTAs fit on an SM); results are identical.
                              A table larger than 227 KB is always read this way */
#define NU_FLAG_VERIFY  16 /* mixed precision only: the request is also run in
                              the FP64 mode (same grids and steps) on the GPU,
                              and err_est then reports, per result, the error
                              against FP64, |mixed - FP64| / |FP64|, instead of
                              the quadrature self-estimate.  Costs an FP64 run
                              (about 100x the mixed kernel's time) and its
                              device memory; works for runs, batches and
                              served requests                                  */

typedef struct nu_cosmo {
    double Om;       /* matter density today; Omega_Lambda = 1 - Om (Sec. II.A) */
    double h;        /* H0 = 100 h km/s/Mpc                                    */
    double T0_K;     /* relic temperature today, 1.95 K for neutrinos          */
} nu_cosmo;

typedef struct nu_halo {
    double M_h;      /* halo mass, Msun (>= 0; 0 means no halo)                */
    double c;        /* concentration r200 / r_s (> 0)                          */
    double z0;       /* observation redshift; only 0 is supported              */
    int xi_kind;     /* NU_XI_*                                                */
    int kappa_kind;  /* NU_KAPPA_*                                             */
    double xi_p[3];
    double kappa_p[3];
} nu_halo;

/* Mass reuse (Sec. III): the equations of motion do not involve the relic
 * mass, so one set of trajectories serves many masses.  With n_masses = 0 the
 * request is for the single mass m_eV.  With n_masses >= 1, m_eV is the
 * fiducial mass that turns the momentum grid into start velocities
 * (v0 = c q k_B T0 / m_eV), and each of masses_eV[0 .. n_masses-1] reads the
 * same trajectories with momenta P = m v: for mass m_a the momentum nodes and
 * the final momenta are those of the fiducial mass times s_a = m_a / m_eV,
 * and the trapezoid weights in ln q are unchanged, so
 *   n/nbar_a = sum_jk w_j q_j^3 w_k f(s_a q_i) / (2 sum_j w_j q_j^3 f(s_a q_j)).
 * Results are then [n_masses][n_radii].  masses_eV is borrowed for the call. */
#define NU_MAX_MASSES 64

typedef struct nu_relic {
    double m_eV;     /* relic mass, eV (> 0); the fiducial mass if n_masses > 0 */
    int f_kind;      /* NU_F_*                                                 */
    int n_masses;    /* 0: one mass m_eV; 1 .. NU_MAX_MASSES: masses_eV        */
    double f_p[2];   /* FD: {eta, -}; table: {q_first, q_last} in k_B T0     */
    const double* masses_eV;   /* [n_masses] relic masses, eV (> 0)            */
    int n_table;     /* NU_F_TABLE: nodes (2 .. NU_MAX_FTABLE)                 */
    int reserved;
    const double* f_table;     /* NU_F_TABLE: [n_table] values >= 0, borrowed  */
} nu_relic;

typedef struct nu_pgrid {
    int n_q;         /* momentum nodes, log-spaced on [q_min, q_max] (>= 2);
                        trapezoid weights in ln q                              */
    int n_mu;        /* Gauss-Legendre nodes for mu on [-1, 1] (>= 1)          */
    double q_min;    /* > 0, units of k_B T0                                   */
    double q_max;    /* > q_min                                                */
} nu_pgrid;

/* Device allocator hooks: alloc returns a device pointer (NULL on failure),
 * free releases one.  With alloc == NULL the library calls cudaMalloc/cudaFree. */
typedef void* (*nu_alloc_fn)(size_t bytes, void* ctx);
typedef void  (*nu_free_fn)(void* ptr, size_t bytes, void* ctx);

typedef struct nu_opts {
    int n_steps;         /* RK4 steps from z0 to z_end (1 .. NU_MAX_STEPS)       */
    int precision;       /* NU_FP64 or NU_MIXED                                   */
    double z_end;        /* end of the backward integration; <= 0 -> the paper's z_i */
    int radii_unit;      /* NU_RADII_*                                            */
    int block;           /* threads per CTA: 0 (default 256) or 64..512, multiple of 32 */
    int tpt;             /* trajectories per thread: 0 (default 1), 1, 2, or 3 =
                            two per thread in packed FP32x2 arithmetic (mixed
                            precision; results bitwise those of 2).  The fastest
                            mixed-precision shape on GB300 is block 128, tpt 3
                            with NU_FLAG_GTAB; nu_autotune finds it            */
    int flags;           /* NU_FLAG_*                                             */
    nu_alloc_fn alloc;
    nu_free_fn free;
    void* alloc_ctx;
    void* stream;        /* cudaStream_t used for uploads during create           */
    double timeout_ms;   /* bound on the host's wait in synchronous calls
                            (nu_profile_compute_noalloc); 0 -> 60000 ms      */
} nu_opts;

#define NU_MAX_STEPS 3000  /* the per-step coefficient table (80 B per step in FP32,
                              160 B in FP64 and in the packed path) is staged in
                              shared memory when it fits in 227 KB and read
                              through the L1 cache otherwise                     */

typedef struct nu_profile nu_profile;
typedef struct nu_batch nu_batch;

/* Host-side summary of a request: derived halo quantities (Sec. II.B) and
 * sizes.  Filled by nu_profile_plan without touching the GPU. */
typedef struct nu_plan_info {
    double R_kpc;            /* comoving radius of the collapsing region      */
    double r200_kpc;         /* physical virial radius                        */
    double r_s_kpc;          /* NFW scale radius                              */
    double z_i;              /* onset redshift, (1+z_i) = 200^(1/3) (1+z0)    */
    double Ic;               /* ln(1+c) - c/(1+c)                             */
    double rho_bar0;         /* mean matter density today, Msun/kpc^3         */
    double z_end;            /* resolved end redshift                         */
    long long n_traj;        /* n_radii * n_q * n_mu                          */
    long long h2d_bytes;     /* bytes create() copies host -> device          */
    long long traj_steps;    /* n_traj * n_steps                              */
    long long device_bytes;  /* device memory create() will allocate          */
    int n_tiles;             /* work tiles of one run                         */
    int tile;                /* trajectories per tile (block * tpt)           */
    int precision;           /* NU_FP64 or NU_MIXED                           */
    int n_steps;             /* RK4 steps                                     */
    int n_masses;            /* masses read from the trajectories (>= 1)      */
    int reserved;
} nu_plan_info;

/* Fill *info for the request (validation + Sec. II.B derivation + sizing).
 * Needs no GPU.  Errors: NU_EINVAL for out-of-range inputs, NU_ENOTSUP for
 * z0 != 0 or n_steps > NU_MAX_STEPS. */
NU_API int nu_profile_plan(const nu_cosmo* cosmo, const nu_halo* halo, const nu_relic* relic,
                    const double* radii, int n_radii, const nu_pgrid* p_grid,
                    const nu_opts* opts, nu_plan_info* info);

/* Create a profile request (Sec. II.B-II.D).  Validates, derives the halo in
 * FP64 on the host, builds the per-step coefficient table (background H(z),
 * growth xi(z), coupling kappa(z) at every RK stage), the q and mu nodes and
 * weights and the background normalisation, allocates the device buffers
 * (through opts->alloc when given) and uploads them on opts->stream.
 * radii: n_radii values > 0 in opts->radii_unit.  *out is set only on success.
 * Errors: NU_EINVAL, NU_ENOTSUP, NU_ENOMEM, NU_ECUDA. */
NU_API int nu_profile_create(const nu_cosmo* cosmo, const nu_halo* halo, const nu_relic* relic,
                      const double* radii, int n_radii, const nu_pgrid* p_grid,
                      const nu_opts* opts, nu_profile** out);

/* Enqueue one evaluation of Eq. localdensity / nbar for every radius on
 * `stream` (asynchronous): backward RK4 trajectories (Eq. eoms with the
 * App. A gradient), Liouville map, f, and the quadrature reduction, in one
 * persistent kernel.  Re-running is idempotent.  Errors: NU_EINVAL (NULL
 * handle), NU_ECUDA (launch failure). */
NU_API int nu_profile_run(nu_profile* h, void* stream);

/* Wait for the last run of `h` and copy n/nbar (and, if err_est != NULL, an
 * estimate of the relative quadrature error of each value: the difference to
 * the same sum on a grid with every other q node, divided by 3; for a request
 * created with NU_FLAG_VERIFY, the relative difference to the same request in
 * the FP64 mode) into host arrays of n_radii doubles.  For a request with several masses (nu_relic
 * n_masses > 0) the arrays hold [n_masses][n_radii] values and n_radii must be
 * n_masses times the number of radii.  Errors: NU_EBUSY (never run), NU_EINVAL
 * (size mismatch), NU_EDEVICE (non-finite sum), NU_ECUDA. */
NU_API int nu_profile_result(nu_profile* h, double* n_over_nbar, double* err_est, int n_radii);

/* Copy the final momenta q_i (units of k_B T0) of every trajectory of the last
 * run, ordered [radius][q][mu], into a host array of n values
 * (n = n_radii * n_q * n_mu); they are kept on the device in the state
 * precision (FP64 or FP32).  Needs NU_FLAG_KEEP_QI at create; this is the
 * phase-space integrand of Sec. III (Fig. 3).  Errors: NU_EINVAL, NU_EBUSY,
 * NU_ECUDA. */
NU_API int nu_profile_qi(nu_profile* h, double* qi, long long n);

/* Verification of the force (App. A) exactly as the trajectory kernel computes
 * it: for each of n comoving radii r[i] (kpc, on the x axis) writes
 * m[i] = Mhat(r, z) / r^3 with Mhat = I(r/(r_s(1+z)))/I(c) - (r/R)^3 inside
 * r200(1+z), 1 - (r/R)^3 inside R and 0 beyond, evaluated in the handle's
 * precision at the redshift of RK stage `stage` (half-step index 0..2N:
 * 1+z = exp(stage * ln(1+z_end) / (2N))).  The gradient is
 * dPhi/dr = G kappa(z) (1+z) xi(z) M_h m r.  Host arrays; synchronous.
 * Errors: NU_EINVAL, NU_ENOMEM, NU_ECUDA. */
NU_API int nu_profile_force(nu_profile* h, int stage, const double* r, int n, double* m);

/* Plan numbers of an existing handle. */
NU_API int nu_profile_info(const nu_profile* h, nu_plan_info* info);

/* Release a handle and its device memory (waits for its last run). NULL-safe. */
NU_API void nu_profile_destroy(nu_profile* h);

/* Batch several requests into ONE persistent launch (uneven halos x radii x
 * grids drained from a shared work list).  All handles must have the same
 * precision and tile shape; each keeps its own outputs, read with
 * nu_profile_result.  The handles must outlive the batch.  opts may be NULL;
 * opts->flags & NU_FLAG_GRAPH captures the launch in a CUDA graph at the
 * first run and replays it afterwards; opts->block and opts->tpt (when non-zero)
 * set the batch's tile shape, else the requests' own shape is used (and must
 * agree).  Errors: NU_EINVAL, NU_ENOMEM, NU_ECUDA. */
NU_API int nu_batch_create(nu_profile* const* hs, int n, const nu_opts* opts, nu_batch** out);
NU_API int nu_batch_run(nu_batch* b, void* stream);
NU_API void nu_batch_destroy(nu_batch* b);

/* Device time in milliseconds of the trajectory kernel of the last
 * nu_batch_run of a batch created with NU_FLAG_TIMING (events recorded on the
 * launch stream around the kernel only; with NU_FLAG_GRAPH, around the graph
 * launch).  Waits for that run.  Errors: NU_EINVAL (no timing flag), NU_EBUSY
 * (never run), NU_ECUDA. */
NU_API int nu_batch_kernel_ms(nu_batch* b, float* ms);

/* Exact work statistics of one run of the batch, from a counting variant of
 * the trajectory kernel (launched once, synchronously, on `stream`; its
 * results are those of a normal run).  For unfinished trajectories only:
 * counts[0] force evaluations beyond R (gradient exactly zero), counts[1] in
 * the compensating shell, counts[2] in the NFW part with I(y) on its first
 * branch (FP32: the rational approximation, y < min(c, 16); FP64: the series,
 * y < 1), counts[3] on its logarithm branch, counts[4]
 * trajectory-steps integrated.  A trajectory is finished once its velocity
 * can no longer change (it lies beyond R on a line that does not re-enter
 * before z_end): its remaining steps are not needed work (its warp stops when
 * all of its lanes are finished; the test runs every 4 steps, so up to 3 steps
 * past the finish are counted).  counts[5] is every lane-step that the warps
 * ran, finished trajectories and padding lanes included, so counts[4] /
 * counts[5] is the fraction of lane-steps doing needed work.  The force is
 * data dependent (App. A has three branches), so these counts turn one run
 * into an exact algorithmic flop count.  counts must hold 6 values.  Errors:
 * NU_EINVAL, NU_ENOMEM, NU_ECUDA. */
NU_API int nu_batch_branch_counts(nu_batch* b, void* stream, long long* counts);

/* Launch-shape autotuner: times the batch of requests `hs` with each candidate
 * launch shape (threads per CTA x trajectories per thread x table source:
 * 256x1, 512x1, 256x2 staged in shared memory; 256x1, 384x1 through L1; and for
 * mixed precision the packed 256x3 and 128x3 through L1 and 256x3 staged; one
 * warm-up and the median of three runs) and reports the
 * fastest.  With cache_path != NULL, a JSON-lines cache keyed by GPU name,
 * precision, step-count and trajectory-count buckets (powers of two) is read
 * first and appended to after tuning.  Results of different shapes agree to
 * rounding, not bit for bit (the reduction order changes).  All requests must
 * share a precision.  Errors: NU_EINVAL, NU_ENOMEM, NU_ECUDA. */
typedef struct nu_tune_result {
    int block;               /* best threads per CTA                          */
    int tpt;                 /* best trajectories per thread                  */
    int flags;               /* best table source (0 or NU_FLAG_GTAB)         */
    float best_ms;           /* trajectory-kernel time of one run with it     */
    int from_cache;          /* 1 if read from the cache (no timing done)     */
    int n_candidates;
    int cand_block[8];
    int cand_tpt[8];
    int cand_flags[8];
    float cand_ms[8];
} nu_tune_result;
NU_API int nu_autotune(nu_profile* const* hs, int n, void* stream, const char* cache_path,
                       nu_tune_result* out);

/* Size of a batch: total work tiles, trajectory-steps of one run, bytes that
 * nu_batch_create copied host -> device, and the persistent grid (CTAs).
 * Any output pointer may be NULL.  Errors: NU_EINVAL. */
NU_API int nu_batch_info(const nu_batch* b, int* n_tiles, long long* traj_steps,
                         long long* h2d_bytes, int* grid);

/* ---- continuous-batching request server ------------------------------------
 * For rapid scans (the use the paper names: many cosmologies, halo and relic
 * masses and grids), requests are queued and served together: a worker thread
 * admits queued requests first come, first served while a device budget (one
 * arena, sub-allocated first fit) and a slot limit allow, and runs one
 * persistent trajectory launch per iteration over every admitted request,
 * advancing each by chunk_steps RK4 steps with its trajectories' state kept
 * on the device.  Requests arriving meanwhile join at the next launch; a
 * request that reaches its last step forms its quadrature (Eq. localdensity)
 * in that launch and leaves, freeing memory.  A request's result is bitwise
 * the one nu_profile_run gives it alone with the same tile shape.  Every wait
 * on the GPU is bounded by gpu_timeout_ms. */
typedef struct nu_server nu_server;
typedef struct nu_server_opts {
    size_t device_bytes;     /* device memory budget of the server (>= 1 MiB)     */
    int max_active;          /* requests on the GPU at once (0 -> 64: beyond that,
                                sharing launches among more requests only slows
                                each one down)                                  */
    int chunk_steps;         /* RK4 steps per launch (0: a request's whole run)   */
    int precision;           /* NU_FP64 or NU_MIXED: every request uses it        */
    int block, tpt, flags;   /* launch shape (0: 128 x 3 with NU_FLAG_GTAB for mixed,
                                256 x 1 for FP64)                                 */
    nu_alloc_fn alloc;       /* where the budget comes from (NULL: cudaMalloc)    */
    nu_free_fn free;
    void* alloc_ctx;
    double gpu_timeout_ms;   /* bound on one launch (<= 0 -> 60000)               */
    double step_budget;      /* trajectory-steps per launch (<= 0 -> 4e9): with many
                                requests active the chunk shrinks to fit it, which
                                bounds each launch's duration                      */
    int resident;            /* 1: requests that arrive while a launch runs join it
                                through a device work queue instead of waiting for
                                the next launch (whole runs: chunk_steps must be 0;
                                needs host-native atomics, else NU_ENOTSUP)        */
    double linger_ms;        /* resident: how long the queue stays open after it
                                runs dry, for arrivals to join (0: close at once)  */
    double queue_wait_ms;    /* resident: bound on one CTA's wait for queued work
                                (<= 0 -> 1000); when it runs out the launch ends
                                and the server counts it in queue_expired         */
} nu_server_opts;

typedef struct nu_serve_stats {
    long long submitted, admitted, completed, cancelled, rejected;
    long long iterations;    /* launches                                          */
    long long traj_steps;    /* trajectory-steps advanced                          */
    double busy_ms;          /* host-measured time of the launches                 */
    double p50_ms, p99_ms, mean_ms;   /* submit -> result latency of completed ones */
    int pending, active, max_active_seen;
    int status;              /* NU_OK, or the error that stopped the server        */
    long long arena_bytes, arena_peak;
    long long early;         /* results delivered while their last launch still ran */
    long long joined;        /* resident: requests admitted into a running launch    */
    long long queue_expired; /* resident: launches ended by a CTA's bounded queue wait */
} nu_serve_stats;

/* Start a server on the current device.  Errors: NU_EINVAL, NU_ENOMEM, NU_ECUDA. */
NU_API int nu_server_create(const nu_server_opts* opts, nu_server** out);
/* Queue a request (arguments as for nu_profile_create; opts may be NULL and
 * only its n_steps, z_end, radii_unit and NU_FLAG_VERIFY are used: a verified
 * request's FP64 run goes on a stream of its own, and the request is
 * delivered, with its error against FP64 in err_est, when both are done).  Returns a ticket at once;
 * the request is validated first (NU_EINVAL / NU_ENOTSUP), and a request that
 * can never fit the budget later completes with NU_ENOMEM. */
NU_API int nu_server_submit(nu_server* s, const nu_cosmo* cosmo, const nu_halo* halo,
                            const nu_relic* relic, const double* radii, int n_radii,
                            const nu_pgrid* p_grid, const nu_opts* opts, long long* ticket);
/* NU_EAGAIN while the request runs; when it is done, copies n/nbar, the error
 * estimate (may be NULL) and the submit-to-result latency (may be NULL) and
 * returns the request's status (NU_OK, NU_ECANCELED, NU_ENOMEM, NU_ETIMEDOUT ...)
 * once; NU_EINVAL for an unknown or already delivered ticket or a wrong n_radii
 * (for a mass-reuse request, n_masses times its number of radii; the server
 * keeps its own copies of the mass list and of a tabulated f). */
NU_API int nu_server_poll(nu_server* s, long long ticket, double* n_over_nbar, double* err_est,
                          int n_radii, double* latency_ms);
/* Cancel a queued or running request (it completes with NU_ECANCELED before
 * its next launch).  NU_EINVAL if the ticket is unknown or already done. */
NU_API int nu_server_cancel(nu_server* s, long long ticket);
NU_API int nu_server_stats(nu_server* s, nu_serve_stats* out);
/* Stop the worker (after the launch in flight) and release everything. */
NU_API void nu_server_destroy(nu_server* s);

/* Maximum device scratch of nu_profile_compute_noalloc (a static array). */
#define NU_NOALLOC_MAX_BYTES (4u << 20)

/* One request computed without allocating anything, for callers that cannot
 * call cudaMalloc (code whose device memory is owned by another framework's
 * pool, hosts that forbid allocation after start-up, code running while
 * another component captures work).  The paper has no counterpart: this is
 * nu_profile_create + nu_profile_run + nu_profile_result in one synchronous
 * call, with every device buffer the trajectory kernel needs (descriptor,
 * coefficient table, nodes and weights, tile sums, counters) placed in one
 * file-scope __device__ array of NU_NOALLOC_MAX_BYTES that every GPU loading
 * the library keeps until the process exits, and the host tables built (by
 * the same routines as nu_profile_create) in a static host buffer of the same
 * size.  It calls no cudaMalloc, cudaFree or other allocating routine.  The
 * results are bitwise those of nu_profile_create/run/result at the same
 * launch shape.
 *   Inputs are the same as nu_profile_create (opts may be NULL; opts->flags
 *   must be 0 and the allocator hooks are ignored; opts->timeout_ms bounds
 *   the wait); n_over_nbar and err_est (may be NULL) are host arrays of
 *   n_radii doubles.  The work runs on `stream`, which must not be capturing,
 *   and the call returns after it has finished.
 *   Set-up: every call looks up the array's device address
 *   (cudaGetSymbolAddress) with the current device; the first call on a
 *   device also loads the module there, so make it before any stream capture
 *   (other threads' captures must use the relaxed or thread-local mode).
 *   Sharing: all calls use the same array.  A process-wide lock serializes
 *   the calls and each waits for its own work, so calls from this library
 *   never overlap on the GPU; any other work that touched the array while a
 *   call ran would race with it.  The array keeps the last call's contents;
 *   each call clears the counters that must start at zero.
 *   Timeout: if the call's work has not finished within timeout_ms the call
 *   returns NU_ETIMEDOUT and its work keeps the array; later calls on that
 *   device first wait (again bounded) for that work, so keep its stream alive
 *   until a later call has returned something other than NU_ETIMEDOUT.
 *   Errors: NU_EINVAL, NU_ENOTSUP (the packed shape tpt = 3, a mass-reuse
 *   relic or a tabulated f: this entry point computes one closed-form
 *   distribution for one mass), NU_ETOOBIG (the request's device buffers, or
 *   its host tables, need more than NU_NOALLOC_MAX_BYTES, e.g. too many
 *   radii x tiles or steps), NU_ETIMEDOUT, NU_EDEVICE, NU_ECUDA. */
NU_API int nu_profile_compute_noalloc(const nu_cosmo* cosmo, const nu_halo* halo,
                                      const nu_relic* relic, const double* radii, int n_radii,
                                      const nu_pgrid* p_grid, const nu_opts* opts,
                                      double* n_over_nbar, double* err_est, void* stream);

/* Measured arithmetic throughput of the current GPU (the denominators of the
 * trajectory kernel's roofline, an FP32 ALU-bound path): scalar FP32 FMA and
 * packed FP32x2 FMA in TFLOP/s (FMA = 2 flops), and the special-function
 * unit's reciprocal square root and base-2 logarithm in Gop/s.  Each kernel
 * runs 8 independent chains per thread on 8 CTAs of 256 threads per SM, timed
 * with CUDA events on `stream` after one warm-up.  Errors: NU_EINVAL, NU_ECUDA. */
typedef struct nu_peaks {
    double ffma_tflops;
    double ffma2_tflops;
    double rsqrt_gops;
    double lg2_gops;
    int sm_count;
    int clock_mhz_nominal;   /* cudaDevAttrClockRate / 1000 */
    double dfma_tflops;      /* FP64 fused multiply-add (the FP64 mode's ALU peak) */
} nu_peaks;
NU_API int nu_measure_peaks(void* stream, nu_peaks* out);

/* Launch counters: kernels launched by the library since load (all handles). */
NU_API long long nu_kernel_launches(void);

NU_API const char* nu_strerror(int code);
NU_API int nu_version(void);   /* 10000*major + 100*minor + patch */

#ifdef __cplusplus
}
#endif

#endif /* NUPROF_H */
