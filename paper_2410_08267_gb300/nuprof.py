"""Python binding of the relic-overdensity C-ABI (include/nuprof.h).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libnuprof.so`` built in-tree by ``paper_2410_08267_gb300.build``.
There is no fallback: if the library is missing or cannot be loaded, the
import of the functions below raises.  PyTorch is used only for device memory
(the caching allocator, through the library's allocator hooks) and streams.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnuprof.so")

NU_OK, NU_EINVAL, NU_ENOMEM, NU_ECUDA, NU_EBUSY = 0, -1, -2, -3, -4
NU_ETIMEDOUT, NU_EDEVICE, NU_ENOTSUP, NU_ECANCELED, NU_EAGAIN = -5, -6, -7, -8, -9
NU_ETOOBIG = -10
NU_NOALLOC_MAX_BYTES = 4 << 20
NU_FP64, NU_MIXED = 0, 1
NU_RADII_KPC, NU_RADII_R200 = 0, 1
NU_FLAG_KEEP_QI, NU_FLAG_GRAPH, NU_FLAG_TIMING, NU_FLAG_GTAB, NU_FLAG_VERIFY = 1, 2, 4, 8, 16
NU_MAX_STEPS = 3000
NU_MAX_MASSES = 64
NU_MAX_FTABLE = 4096


class NuError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class nu_cosmo(C.Structure):
    _fields_ = [("Om", C.c_double), ("h", C.c_double), ("T0_K", C.c_double)]


class nu_halo(C.Structure):
    _fields_ = [("M_h", C.c_double), ("c", C.c_double), ("z0", C.c_double),
                ("xi_kind", C.c_int), ("kappa_kind", C.c_int),
                ("xi_p", C.c_double * 3), ("kappa_p", C.c_double * 3)]


class nu_relic(C.Structure):
    _fields_ = [("m_eV", C.c_double), ("f_kind", C.c_int), ("n_masses", C.c_int),
                ("f_p", C.c_double * 2), ("masses_eV", C.POINTER(C.c_double)),
                ("n_table", C.c_int), ("reserved", C.c_int), ("f_table", C.POINTER(C.c_double))]


class nu_pgrid(C.Structure):
    _fields_ = [("n_q", C.c_int), ("n_mu", C.c_int), ("q_min", C.c_double), ("q_max", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class nu_opts(C.Structure):
    _fields_ = [("n_steps", C.c_int), ("precision", C.c_int), ("z_end", C.c_double),
                ("radii_unit", C.c_int), ("block", C.c_int), ("tpt", C.c_int), ("flags", C.c_int),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("stream", C.c_void_p), ("timeout_ms", C.c_double)]


class nu_plan_info(C.Structure):
    _fields_ = [("R_kpc", C.c_double), ("r200_kpc", C.c_double), ("r_s_kpc", C.c_double),
                ("z_i", C.c_double), ("Ic", C.c_double), ("rho_bar0", C.c_double),
                ("z_end", C.c_double), ("n_traj", C.c_longlong), ("h2d_bytes", C.c_longlong),
                ("traj_steps", C.c_longlong),
                ("device_bytes", C.c_longlong), ("n_tiles", C.c_int), ("tile", C.c_int),
                ("precision", C.c_int), ("n_steps", C.c_int), ("n_masses", C.c_int),
                ("reserved", C.c_int)]


class nu_server_opts(C.Structure):
    _fields_ = [("device_bytes", C.c_size_t), ("max_active", C.c_int), ("chunk_steps", C.c_int),
                ("precision", C.c_int), ("block", C.c_int), ("tpt", C.c_int), ("flags", C.c_int),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("gpu_timeout_ms", C.c_double), ("step_budget", C.c_double),
                ("resident", C.c_int), ("linger_ms", C.c_double), ("queue_wait_ms", C.c_double)]


class nu_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("admitted", C.c_longlong),
                ("completed", C.c_longlong), ("cancelled", C.c_longlong),
                ("rejected", C.c_longlong), ("iterations", C.c_longlong),
                ("traj_steps", C.c_longlong), ("busy_ms", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("pending", C.c_int),
                ("active", C.c_int), ("max_active_seen", C.c_int), ("status", C.c_int),
                ("arena_bytes", C.c_longlong), ("arena_peak", C.c_longlong), ("early", C.c_longlong),
                ("joined", C.c_longlong), ("queue_expired", C.c_longlong)]


class nu_peaks(C.Structure):
    _fields_ = [("ffma_tflops", C.c_double), ("ffma2_tflops", C.c_double),
                ("rsqrt_gops", C.c_double), ("lg2_gops", C.c_double),
                ("sm_count", C.c_int), ("clock_mhz_nominal", C.c_int), ("dfma_tflops", C.c_double)]


class nu_tune_result(C.Structure):
    _fields_ = [("block", C.c_int), ("tpt", C.c_int), ("flags", C.c_int), ("best_ms", C.c_float),
                ("from_cache", C.c_int), ("n_candidates", C.c_int),
                ("cand_block", C.c_int * 8), ("cand_tpt", C.c_int * 8), ("cand_flags", C.c_int * 8),
                ("cand_ms", C.c_float * 8)]


_lib = None


def lib():
    """Load libnuprof.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "paper_2410_08267_gb300.build.build() (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    vp = C.c_void_p
    L.nu_profile_plan.argtypes = [P(nu_cosmo), P(nu_halo), P(nu_relic), P(C.c_double), C.c_int,
                                  P(nu_pgrid), P(nu_opts), P(nu_plan_info)]
    L.nu_profile_create.argtypes = [P(nu_cosmo), P(nu_halo), P(nu_relic), P(C.c_double), C.c_int,
                                    P(nu_pgrid), P(nu_opts), P(vp)]
    L.nu_profile_run.argtypes = [vp, vp]
    L.nu_profile_result.argtypes = [vp, P(C.c_double), P(C.c_double), C.c_int]
    L.nu_profile_qi.argtypes = [vp, P(C.c_double), C.c_longlong]
    L.nu_profile_info.argtypes = [vp, P(nu_plan_info)]
    L.nu_profile_force.argtypes = [vp, C.c_int, P(C.c_double), C.c_int, P(C.c_double)]
    L.nu_profile_destroy.argtypes = [vp]
    L.nu_profile_destroy.restype = None
    L.nu_batch_create.argtypes = [P(vp), C.c_int, P(nu_opts), P(vp)]
    L.nu_batch_run.argtypes = [vp, vp]
    L.nu_batch_kernel_ms.argtypes = [vp, P(C.c_float)]
    L.nu_batch_info.argtypes = [vp, P(C.c_int), P(C.c_longlong), P(C.c_longlong), P(C.c_int)]
    L.nu_batch_branch_counts.argtypes = [vp, vp, P(C.c_longlong)]
    L.nu_autotune.argtypes = [P(vp), C.c_int, vp, C.c_char_p, P(nu_tune_result)]
    L.nu_batch_destroy.argtypes = [vp]
    L.nu_batch_destroy.restype = None
    L.nu_profile_compute_noalloc.argtypes = [P(nu_cosmo), P(nu_halo), P(nu_relic), P(C.c_double),
                                             C.c_int, P(nu_pgrid), P(nu_opts), P(C.c_double),
                                             P(C.c_double), vp]
    L.nu_profile_compute_noalloc.restype = C.c_int
    L.nu_server_create.argtypes = [P(nu_server_opts), P(vp)]
    L.nu_server_submit.argtypes = [vp, P(nu_cosmo), P(nu_halo), P(nu_relic), P(C.c_double), C.c_int,
                                   P(nu_pgrid), P(nu_opts), P(C.c_longlong)]
    L.nu_server_poll.argtypes = [vp, C.c_longlong, P(C.c_double), P(C.c_double), C.c_int,
                                 P(C.c_double)]
    L.nu_server_cancel.argtypes = [vp, C.c_longlong]
    L.nu_server_stats.argtypes = [vp, P(nu_serve_stats)]
    L.nu_server_destroy.argtypes = [vp]
    L.nu_server_destroy.restype = None
    for name in ("nu_server_create", "nu_server_submit", "nu_server_poll", "nu_server_cancel",
                 "nu_server_stats"):
        getattr(L, name).restype = C.c_int
    L.nu_measure_peaks.argtypes = [vp, P(nu_peaks)]
    L.nu_measure_peaks.restype = C.c_int
    L.nu_kernel_launches.argtypes = []
    L.nu_kernel_launches.restype = C.c_longlong
    L.nu_strerror.argtypes = [C.c_int]
    L.nu_strerror.restype = C.c_char_p
    L.nu_version.argtypes = []
    for name in ("nu_profile_plan", "nu_profile_create", "nu_profile_run", "nu_profile_result",
                 "nu_profile_qi", "nu_profile_info", "nu_profile_force", "nu_batch_create",
                 "nu_batch_run",
                 "nu_batch_kernel_ms", "nu_batch_info", "nu_batch_branch_counts", "nu_autotune",
                 "nu_version"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != NU_OK:
        raise NuError(rc, where)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)       # torch.cuda.Stream


# ---------------------------------------------------------------------------
# PyTorch caching allocator as the library's device allocator
# ---------------------------------------------------------------------------

def _torch_alloc(nbytes, ctx):
    import torch
    return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                  torch.cuda.current_stream()))


def _torch_free(ptr, nbytes, ctx):
    import torch
    torch.cuda.caching_allocator_delete(int(ptr))


TORCH_ALLOC = ALLOC_FN(_torch_alloc)
TORCH_FREE = FREE_FN(_torch_free)


# ---------------------------------------------------------------------------
# Structs from a workload Problem
# ---------------------------------------------------------------------------

def structs(pb: "W.Problem", block: int = 0, tpt: int = 0, flags: int = 0, stream=None,
            torch_alloc: bool = True):
    cosmo = nu_cosmo(pb.Om, pb.h, pb.T0_K)
    halo = nu_halo()
    halo.M_h, halo.c, halo.z0 = pb.M_h, pb.c, pb.z0
    halo.xi_kind, halo.kappa_kind = int(pb.xi_kind), int(pb.kappa_kind)
    for i in range(3):
        halo.xi_p[i] = float(pb.xi_p[i])
        halo.kappa_p[i] = float(pb.kappa_p[i])
    relic = nu_relic()
    relic.m_eV, relic.f_kind = pb.m_eV, int(pb.f_kind)
    relic.f_p[0], relic.f_p[1] = float(pb.f_p[0]), float(pb.f_p[1])
    if len(pb.f_table):                     # tabulated f: f_p holds the node range
        relic._tab = np.ascontiguousarray(np.asarray(pb.f_table, dtype=np.float64))
        relic.n_table = len(relic._tab)
        relic.f_table = relic._tab.ctypes.data_as(C.POINTER(C.c_double))
    if len(pb.masses):                      # mass reuse: m_eV is the fiducial mass
        relic._masses = np.ascontiguousarray(np.asarray(pb.masses, dtype=np.float64))
        relic.n_masses = len(relic._masses)
        relic.masses_eV = relic._masses.ctypes.data_as(C.POINTER(C.c_double))
    grid = nu_pgrid(int(pb.n_q), int(pb.n_mu), float(pb.q_min), float(pb.q_max))
    opts = nu_opts()
    opts.n_steps, opts.precision, opts.z_end = int(pb.n_steps), int(pb.precision), float(pb.z_end)
    opts.radii_unit, opts.block, opts.tpt, opts.flags = int(pb.radii_unit), block, tpt, flags
    if torch_alloc:
        opts.alloc, opts.free = TORCH_ALLOC, TORCH_FREE
    opts.stream = _stream_ptr(stream)
    radii = np.ascontiguousarray(np.asarray(pb.radii, dtype=np.float64))
    return cosmo, halo, relic, radii, grid, opts


# ---------------------------------------------------------------------------
# C-ABI entry points (same names)
# ---------------------------------------------------------------------------

def nu_version() -> int:
    return lib().nu_version()


def strerror(code: int) -> str:
    return lib().nu_strerror(int(code)).decode()


nu_strerror = strerror


def nu_server_create(device_bytes: int, precision: int = NU_MIXED, max_active: int = 0,
                     chunk_steps: int = 100, block: int = 0, tpt: int = 0, flags: int = 0,
                     gpu_timeout_ms: float = 0.0, torch_alloc: bool = False,
                     step_budget: float = 0.0, resident: bool = False, linger_ms: float = 0.0,
                     queue_wait_ms: float = 0.0) -> C.c_void_p:
    o = nu_server_opts()
    o.step_budget = step_budget
    o.resident, o.linger_ms, o.queue_wait_ms = int(bool(resident)), linger_ms, queue_wait_ms
    o.device_bytes, o.max_active, o.chunk_steps, o.precision = device_bytes, max_active, chunk_steps, precision
    o.block, o.tpt, o.flags, o.gpu_timeout_ms = block, tpt, flags, gpu_timeout_ms
    if torch_alloc:
        o.alloc, o.free = TORCH_ALLOC, TORCH_FREE
    srv = C.c_void_p()
    _check(lib().nu_server_create(C.byref(o), C.byref(srv)), "nu_server_create")
    return srv


def nu_server_submit(srv, pb: "W.Problem", flags: int = 0) -> int:
    """Queue a request; flags may hold NU_FLAG_VERIFY."""
    cosmo, halo, relic, radii, grid, opts = structs(pb, torch_alloc=False, flags=flags)
    t = C.c_longlong()
    _check(lib().nu_server_submit(srv, C.byref(cosmo), C.byref(halo), C.byref(relic), _dptr(radii),
                                  len(radii), C.byref(grid), C.byref(opts), C.byref(t)),
           "nu_server_submit")
    return t.value


def nu_server_poll(srv, ticket: int, n_radii: int):
    """None while running; else (status, n/nbar, err, latency_ms)."""
    out = np.zeros(n_radii)
    err = np.zeros(n_radii)
    lat = C.c_double()
    rc = lib().nu_server_poll(srv, int(ticket), _dptr(out), _dptr(err), int(n_radii), C.byref(lat))
    if rc == NU_EAGAIN:
        return None
    if rc == NU_EINVAL:
        raise NuError(rc, "nu_server_poll")
    return rc, out, err, lat.value


def nu_server_cancel(srv, ticket: int):
    _check(lib().nu_server_cancel(srv, int(ticket)), "nu_server_cancel")


def nu_server_stats(srv) -> dict:
    st = nu_serve_stats()
    _check(lib().nu_server_stats(srv, C.byref(st)), "nu_server_stats")
    return {k: getattr(st, k) for k, _ in nu_serve_stats._fields_}


def nu_server_destroy(srv):
    if srv:
        lib().nu_server_destroy(srv)


def nu_measure_peaks(stream=None) -> dict:
    p = nu_peaks()
    _check(lib().nu_measure_peaks(_stream_ptr(stream), C.byref(p)), "nu_measure_peaks")
    return {k: getattr(p, k) for k, _ in nu_peaks._fields_}


def nu_kernel_launches() -> int:
    return lib().nu_kernel_launches()


def nu_profile_plan(cosmo, halo, relic, radii, grid, opts) -> dict:
    info = nu_plan_info()
    radii = np.ascontiguousarray(np.asarray(radii, dtype=np.float64))
    _check(lib().nu_profile_plan(C.byref(cosmo), C.byref(halo), C.byref(relic), _dptr(radii),
                                 len(radii), C.byref(grid), C.byref(opts), C.byref(info)),
           "nu_profile_plan")
    return {k: getattr(info, k) for k, _ in nu_plan_info._fields_}


def nu_profile_create(cosmo, halo, relic, radii, grid, opts) -> C.c_void_p:
    h = C.c_void_p()
    radii = np.ascontiguousarray(np.asarray(radii, dtype=np.float64))
    _check(lib().nu_profile_create(C.byref(cosmo), C.byref(halo), C.byref(relic), _dptr(radii),
                                   len(radii), C.byref(grid), C.byref(opts), C.byref(h)),
           "nu_profile_create")
    return h


def nu_profile_run(h, stream=None):
    _check(lib().nu_profile_run(h, _stream_ptr(stream)), "nu_profile_run")


def nu_profile_result(h, n_radii: int, with_err: bool = True):
    out = np.zeros(n_radii)
    err = np.zeros(n_radii) if with_err else None
    _check(lib().nu_profile_result(h, _dptr(out), _dptr(err) if with_err else None, int(n_radii)),
           "nu_profile_result")
    return (out, err) if with_err else out


def nu_profile_qi(h, n: int) -> np.ndarray:
    qi = np.zeros(n)
    _check(lib().nu_profile_qi(h, _dptr(qi), int(n)), "nu_profile_qi")
    return qi


def nu_profile_force(h, stage: int, r) -> np.ndarray:
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64))
    m = np.zeros_like(r)
    _check(lib().nu_profile_force(h, int(stage), _dptr(r), len(r), _dptr(m)), "nu_profile_force")
    return m


def nu_profile_compute_noalloc(cosmo, halo, relic, radii, grid, opts=None, stream=None):
    """One request without any allocation (static device scratch); returns
    (n/nbar, err_est) as host arrays."""
    radii = np.ascontiguousarray(np.asarray(radii, dtype=np.float64))
    out = np.zeros(len(radii))
    err = np.zeros(len(radii))
    _check(lib().nu_profile_compute_noalloc(C.byref(cosmo), C.byref(halo), C.byref(relic),
                                            _dptr(radii), len(radii), C.byref(grid),
                                            C.byref(opts) if opts is not None else None,
                                            _dptr(out), _dptr(err), _stream_ptr(stream)),
           "nu_profile_compute_noalloc")
    return out, err


def nu_profile_info(h) -> dict:
    info = nu_plan_info()
    _check(lib().nu_profile_info(h, C.byref(info)), "nu_profile_info")
    return {k: getattr(info, k) for k, _ in nu_plan_info._fields_}


def nu_profile_destroy(h):
    if h:
        lib().nu_profile_destroy(h)


def nu_batch_create(handles: Sequence, opts: Optional[nu_opts] = None) -> C.c_void_p:
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    b = C.c_void_p()
    _check(lib().nu_batch_create(arr, len(handles), C.byref(opts) if opts is not None else None,
                                 C.byref(b)), "nu_batch_create")
    return b


def nu_batch_run(b, stream=None):
    _check(lib().nu_batch_run(b, _stream_ptr(stream)), "nu_batch_run")


def nu_batch_kernel_ms(b) -> float:
    ms = C.c_float()
    _check(lib().nu_batch_kernel_ms(b, C.byref(ms)), "nu_batch_kernel_ms")
    return ms.value


def nu_batch_info(b) -> dict:
    nt, g = C.c_int(), C.c_int()
    ts, hb = C.c_longlong(), C.c_longlong()
    _check(lib().nu_batch_info(b, C.byref(nt), C.byref(ts), C.byref(hb), C.byref(g)), "nu_batch_info")
    return {"n_tiles": nt.value, "traj_steps": ts.value, "h2d_bytes": hb.value, "grid": g.value}


def nu_batch_branch_counts(b, stream=None):
    counts = (C.c_longlong * 6)()
    _check(lib().nu_batch_branch_counts(b, _stream_ptr(stream), counts), "nu_batch_branch_counts")
    return [int(v) for v in counts]


def nu_autotune(handles: Sequence, stream=None, cache_path: Optional[str] = None) -> dict:
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    r = nu_tune_result()
    _check(lib().nu_autotune(arr, len(handles), _stream_ptr(stream),
                             cache_path.encode() if cache_path else None, C.byref(r)), "nu_autotune")
    return {"block": r.block, "tpt": r.tpt, "flags": r.flags, "best_ms": r.best_ms,
            "from_cache": bool(r.from_cache),
            "candidates": [(r.cand_block[i], r.cand_tpt[i], r.cand_flags[i], r.cand_ms[i])
                           for i in range(r.n_candidates)]}


def nu_batch_destroy(b):
    if b:
        lib().nu_batch_destroy(b)


# ---------------------------------------------------------------------------
# Convenience wrappers over the same calls
# ---------------------------------------------------------------------------

def plan(pb: "W.Problem", **kw) -> dict:
    cosmo, halo, relic, radii, grid, opts = structs(pb, torch_alloc=False, **kw)
    return nu_profile_plan(cosmo, halo, relic, radii, grid, opts)


def create(pb: "W.Problem", **kw):
    cosmo, halo, relic, radii, grid, opts = structs(pb, **kw)
    return nu_profile_create(cosmo, halo, relic, radii, grid, opts)


def profile(pb: "W.Problem", stream=None, **kw):
    """Create, run, read and destroy one request: returns (n/nbar, err_est)."""
    h = create(pb, stream=stream, **kw)
    try:
        nu_profile_run(h, stream)
        return nu_profile_result(h, pb.n_out)
    finally:
        nu_profile_destroy(h)
