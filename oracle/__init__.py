"""FP64 CPU oracle for relic overdensity profiles (arXiv:2410.08267).

TEST INFRASTRUCTURE ONLY: imported by tests, by the smoke check and by the
benchmark's CPU-baseline leg.  The CUDA library never imports, links or calls
anything here.  The arithmetic lives in ``nuprof_oracle.c`` (plain C, FP64);
this module only marshals arguments through ctypes.

Functions and the passages they follow:
  derive        Sec. II.B (R, z_i, r200, r_s, I(c))
  H             Sec. II.A (flat FRW expansion rate)
  xi, kappa     Eq. rhototal modulation, Sec. IV.A / Sec. IV.B variants
  I             Eq. nfw (NFW enclosed-mass shape)
  dphidr        App. A (closed-form potential gradient; attractive sign)
  integrate     Eq. eoms in u = ln a, classical RK4
  gauss_legendre, log_grid   quadrature nodes for Eq. localdensity
  f             Sec. II.C / Sec. IV.B initial distributions
  initial_state, final_q     Sec. II.C initial conditions and Liouville map
  profile       Eq. localdensity divided by the background density
  profile_perturbed          conditioning probe (not part of the method)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrParams(C.Structure):
    _fields_ = [("Om", C.c_double), ("h", C.c_double), ("T0_K", C.c_double),
                ("M_h", C.c_double), ("c", C.c_double), ("z0", C.c_double),
                ("xi_kind", C.c_int), ("kappa_kind", C.c_int),
                ("xi_p", C.c_double * 3), ("kappa_p", C.c_double * 3),
                ("m_eV", C.c_double), ("f_kind", C.c_int), ("n_table", C.c_int),
                ("f_p", C.c_double * 2), ("f_table", C.POINTER(C.c_double))]


class OrDerived(C.Structure):
    _fields_ = [("H0", C.c_double), ("rho_bar0", C.c_double), ("R", C.c_double),
                ("z_i", C.c_double), ("r200", C.c_double), ("r_s", C.c_double),
                ("Ic", C.c_double), ("xi_zs", C.c_double), ("xi_ze", C.c_double),
                ("force_scale", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        P = C.POINTER(OrParams)
        D = C.POINTER(OrDerived)
        L.or_derive.argtypes = [P, D]
        L.or_derive.restype = C.c_int
        for name in ("or_H", "or_xi"):
            getattr(L, name).argtypes = [P, D, C.c_double]
            getattr(L, name).restype = C.c_double
        L.or_kappa.argtypes = [P, C.c_double]
        L.or_kappa.restype = C.c_double
        L.or_I.argtypes = [C.c_double]
        L.or_I.restype = C.c_double
        L.or_dphidr.argtypes = [P, D, C.c_double, C.c_double]
        L.or_dphidr.restype = C.c_double
        L.or_integrate.argtypes = [P, D, dp, C.c_double, C.c_double, C.c_int]
        L.or_integrate.restype = None
        L.or_gauss_legendre.argtypes = [C.c_int, dp, dp]
        L.or_gauss_legendre.restype = C.c_int
        L.or_log_grid.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp]
        L.or_log_grid.restype = C.c_int
        L.or_f.argtypes = [P, C.c_double]
        L.or_f.restype = C.c_double
        L.or_profile.argtypes = [P, dp, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int,
                                 C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                 C.c_double, C.c_int, dp, dp]
        L.or_profile.restype = C.c_int
        L.or_profile_perturbed.argtypes = [P, dp, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int,
                                           C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                           C.c_double, C.c_int, C.c_double, C.c_ulonglong, C.c_int,
                                           dp, dp]
        L.or_profile_perturbed.restype = C.c_int
        L.or_profile_masses.argtypes = [P, dp, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int,
                                        C.c_int, C.c_double, C.c_double, C.c_int,
                                        C.c_int, C.c_double, C.c_int, dp, C.c_int, dp]
        L.or_profile_masses.restype = C.c_int
        L.or_initial_state.argtypes = [P, C.c_double, C.c_double, C.c_double, dp]
        L.or_initial_state.restype = None
        L.or_final_q.argtypes = [P, dp]
        L.or_final_q.restype = C.c_double
        L.or_max_threads.argtypes = []
        L.or_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params(pb) -> OrParams:
    """Build the oracle's parameter record from a workload ``Problem``."""
    p = OrParams()
    p.Om, p.h, p.T0_K = pb.Om, pb.h, pb.T0_K
    p.M_h, p.c, p.z0 = pb.M_h, pb.c, pb.z0
    p.xi_kind, p.kappa_kind = int(pb.xi_kind), int(pb.kappa_kind)
    for i in range(3):
        p.xi_p[i] = float(pb.xi_p[i])
        p.kappa_p[i] = float(pb.kappa_p[i])
    p.m_eV = pb.m_eV
    p.f_kind = int(pb.f_kind)
    if len(getattr(pb, "f_table", ())):
        p._tab = np.ascontiguousarray(np.asarray(pb.f_table, dtype=np.float64))
        p.n_table = len(p._tab)
        p.f_table = p._tab.ctypes.data_as(C.POINTER(C.c_double))
    p.f_p[0], p.f_p[1] = float(pb.f_p[0]), float(pb.f_p[1])
    return p


def derive(pb) -> dict:
    p, d = params(pb), OrDerived()
    if lib().or_derive(C.byref(p), C.byref(d)) != 0:
        raise ValueError("invalid halo/cosmology parameters")
    return {k: getattr(d, k) for k, _ in OrDerived._fields_}


def _pd(pb):
    p, d = params(pb), OrDerived()
    if lib().or_derive(C.byref(p), C.byref(d)) != 0:
        raise ValueError("invalid halo/cosmology parameters")
    return p, d


def H(pb, z: float) -> float:
    p, d = _pd(pb)
    return lib().or_H(C.byref(p), C.byref(d), float(z))


def xi(pb, z: float) -> float:
    p, d = _pd(pb)
    return lib().or_xi(C.byref(p), C.byref(d), float(z))


def kappa(pb, z: float) -> float:
    p = params(pb)
    return lib().or_kappa(C.byref(p), float(z))


def I(y: float) -> float:
    return lib().or_I(float(y))


def dphidr(pb, r: float, z: float) -> float:
    p, d = _pd(pb)
    return lib().or_dphidr(C.byref(p), C.byref(d), float(r), float(z))


def integrate(pb, state, u0: float, u1: float, nsteps: int) -> np.ndarray:
    """RK4 in u = ln a from u0 to u1; state = (x, y, vx, vy) in kpc, km/s."""
    p, d = _pd(pb)
    s = np.ascontiguousarray(np.asarray(state, dtype=np.float64).copy())
    lib().or_integrate(C.byref(p), C.byref(d), _dptr(s), float(u0), float(u1), int(nsteps))
    return s


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().or_gauss_legendre(int(n), _dptr(x), _dptr(w)) != 0:
        raise ValueError("n must be >= 1")
    return x, w


def log_grid(n: int, q_min: float, q_max: float):
    q = np.zeros(n)
    w = np.zeros(n)
    if lib().or_log_grid(int(n), float(q_min), float(q_max), _dptr(q), _dptr(w)) != 0:
        raise ValueError("bad log grid")
    return q, w


def f(pb, q: float) -> float:
    p = params(pb)
    return lib().or_f(C.byref(p), float(q))


def initial_state(pb, x0: float, q: float, mu: float) -> np.ndarray:
    s = np.zeros(4)
    lib().or_initial_state(C.byref(params(pb)), float(x0), float(q), float(mu), _dptr(s))
    return s


def final_q(pb, state) -> float:
    s = np.ascontiguousarray(np.asarray(state, dtype=np.float64))
    return lib().or_final_q(C.byref(params(pb)), _dptr(s))


def max_threads() -> int:
    return lib().or_max_threads()


def profile(pb, radius_sel=None, n_threads: int = 0, return_qi: bool = False):
    """n/nbar for a workload ``Problem`` (all radii, or only ``radius_sel``).

    Returns an array of length n_radii (NaN where not computed); with
    ``return_qi`` also the final momenta q_i with shape (n_sel, n_q, n_mu).
    """
    p = params(pb)
    radii = np.ascontiguousarray(np.asarray(pb.radii, dtype=np.float64))
    n_r = len(radii)
    out = np.full(n_r, np.nan)
    if radius_sel is None:
        sel = None
        n_sel = n_r
        sel_ptr = None
    else:
        sel = np.ascontiguousarray(np.asarray(radius_sel, dtype=np.int32))
        n_sel = len(sel)
        sel_ptr = sel.ctypes.data_as(C.POINTER(C.c_int))
    qi = np.zeros((n_sel, pb.n_q, pb.n_mu)) if return_qi else None
    rc = lib().or_profile(C.byref(p), _dptr(radii), n_r, int(pb.radii_unit), sel_ptr, n_sel,
                          int(pb.n_q), float(pb.q_min), float(pb.q_max), int(pb.n_mu),
                          int(pb.n_steps), float(pb.z_end), int(n_threads), _dptr(out),
                          _dptr(qi) if qi is not None else None)
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (rc={rc})")
    return (out, qi) if return_qi else out


def profile_perturbed(pb, eps: float, seed: int, radius_sel=None, n_threads: int = 0,
                      return_qi: bool = False, round_state: bool = False,
                      step_noise: bool = False, force_noise: bool = False):
    """Conditioning probe: n/nbar with each trajectory's start velocity scaled by
    (1 + eps u), u ~ U[-1, 1) independent per trajectory (counter-based, seeded);
    with round_state the state is rounded to float32 after every RK4 step, with
    step_noise every state component is scaled by its own (1 + eps u) after
    every step, with force_noise every force evaluation is scaled by 1 + eps
    (odd seeds) or 1 - eps (even seeds).  Not part of the method; eps = 0
    without the options equals profile() exactly."""
    p = params(pb)
    radii = np.ascontiguousarray(np.asarray(pb.radii, dtype=np.float64))
    n_r = len(radii)
    out = np.full(n_r, np.nan)
    if radius_sel is None:
        sel_ptr, n_sel = None, n_r
    else:
        sel = np.ascontiguousarray(np.asarray(radius_sel, dtype=np.int32))
        sel_ptr, n_sel = sel.ctypes.data_as(C.POINTER(C.c_int)), len(sel)
    qi = np.zeros((n_sel, pb.n_q, pb.n_mu)) if return_qi else None
    rc = lib().or_profile_perturbed(C.byref(p), _dptr(radii), n_r, int(pb.radii_unit), sel_ptr,
                                    n_sel, int(pb.n_q), float(pb.q_min), float(pb.q_max),
                                    int(pb.n_mu), int(pb.n_steps), float(pb.z_end), int(n_threads),
                                    float(eps), int(seed),
                                    int(bool(round_state)) | (2 if step_noise else 0)
                                    | (4 if force_noise else 0), _dptr(out),
                                    _dptr(qi) if qi is not None else None)
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (rc={rc})")
    return (out, qi) if return_qi else out


def profile_masses(pb, masses, radius_sel=None, n_threads: int = 0):
    """Sec. III mass reuse: trajectories of the fiducial pb.m_eV read for every
    mass in ``masses``; returns an array [len(masses), n_radii] (NaN where not
    computed)."""
    p = params(pb)
    radii = np.ascontiguousarray(np.asarray(pb.radii, dtype=np.float64))
    m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64))
    n_r = len(radii)
    out = np.full((len(m), n_r), np.nan)
    if radius_sel is None:
        sel_ptr, n_sel = None, n_r
    else:
        sel = np.ascontiguousarray(np.asarray(radius_sel, dtype=np.int32))
        sel_ptr, n_sel = sel.ctypes.data_as(C.POINTER(C.c_int)), len(sel)
    rc = lib().or_profile_masses(C.byref(p), _dptr(radii), n_r, int(pb.radii_unit), sel_ptr, n_sel,
                                 int(pb.n_q), float(pb.q_min), float(pb.q_max), int(pb.n_mu),
                                 int(pb.n_steps), float(pb.z_end), int(n_threads), _dptr(m), len(m),
                                 _dptr(out))
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (rc={rc})")
    return out
