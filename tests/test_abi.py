"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/nuprof.h, and its host-side logic (validation, the
Sec. II.B halo derivation, sizing) agrees with the oracle."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2410_08267_gb300 import build as nbuild
from paper_2410_08267_gb300 import nuprof as nu
from paper_2410_08267_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    nbuild.build()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "nuprof.h")).read()
    return sorted(set(re.findall(r"NU_API\s+[\w\s\*]+?\b(nu_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert len(names) >= 12
    L = ctypes.CDLL(nu.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n


def test_version_and_strerror():
    assert nu.nu_version() == 10100
    for code in range(0, -10, -1):
        assert nu.strerror(code) != "unknown error"
    assert nu.strerror(-99) == "unknown error"


@pytest.mark.parametrize("pb", W.plain_small() + W.precision_sweep()[:2] + W.random_small(5, n=4))
def test_plan_matches_oracle_derivation(pb):
    info = nu.plan(pb)
    d = oracle.derive(pb)
    for k_lib, k_or in (("R_kpc", "R"), ("r200_kpc", "r200"), ("r_s_kpc", "r_s"), ("z_i", "z_i"),
                        ("Ic", "Ic"), ("rho_bar0", "rho_bar0")):
        assert info[k_lib] == pytest.approx(d[k_or], rel=1e-13), k_lib
    assert info["z_end"] == pb.z_end
    assert info["n_traj"] == pb.n_traj
    assert info["traj_steps"] == pb.traj_steps
    tile = 256
    assert info["tile"] == tile
    assert info["n_tiles"] == pb.n_radii * math.ceil(pb.n_q * pb.n_mu / tile)
    assert info["device_bytes"] > 0


def test_plan_tile_shapes():
    pb = W.plain_small()[0]
    for block, tpt in ((64, 1), (128, 2), (512, 1), (512, 2)):
        info = nu.plan(pb, block=block, tpt=tpt)
        assert info["tile"] == block * tpt
        assert info["n_tiles"] == 10 * math.ceil(1000 / (block * tpt))


BAD = [
    dict(Om=0.0), dict(Om=1.5), dict(h=-0.7), dict(T0_K=0.0), dict(M_h=-1.0), dict(M_h=float("nan")),
    dict(c=0.0), dict(m_eV=0.0), dict(n_q=1), dict(n_mu=0), dict(q_min=0.0), dict(q_max=0.005),
    dict(n_steps=-3), dict(radii=np.array([1.0, -2.0])), dict(radii=np.array([1.0, np.inf])),
    dict(precision=7), dict(radii_unit=5), dict(xi_kind=9), dict(kappa_kind=-1), dict(f_kind=4),
    dict(M_h=0.0, radii_unit=W.RADII_R200),
    dict(xi_kind=W.XI_LINEAR, xi_p=(1.0, 1.0, 2.0)),
]


@pytest.mark.parametrize("bad", BAD)
def test_plan_rejects_invalid_inputs(bad):
    pb = W.plain_small()[0].replace(**bad)
    with pytest.raises(nu.NuError) as e:
        nu.plan(pb)
    assert e.value.code in (nu.NU_EINVAL, nu.NU_ENOTSUP)


def test_packed_shape_rules():
    pb = W.plain_small(precision=W.MIXED)[0]
    info = nu.plan(pb, block=256, tpt=3)            # two trajectories per thread, packed
    assert info["tile"] == 512
    with pytest.raises(nu.NuError) as e:
        nu.plan(pb.replace(precision=W.FP64), block=256, tpt=3)
    assert e.value.code == nu.NU_EINVAL
    # a table too large to stage in shared memory is read through L1 instead
    assert nu.plan(pb.replace(n_steps=nu.NU_MAX_STEPS), block=256, tpt=3)["n_steps"] == nu.NU_MAX_STEPS


def test_plan_rejects_bad_launch_shape_and_unsupported():
    pb = W.plain_small()[0]
    for block, tpt in ((48, 1), (1024, 1), (100, 1), (256, 4)):
        with pytest.raises(nu.NuError) as e:
            nu.plan(pb, block=block, tpt=tpt)
        assert e.value.code == nu.NU_EINVAL
    with pytest.raises(nu.NuError) as e:
        nu.plan(pb.replace(z0=0.5))
    assert e.value.code == nu.NU_ENOTSUP
    with pytest.raises(nu.NuError) as e:
        nu.plan(pb.replace(n_steps=nu.NU_MAX_STEPS + 1))
    assert e.value.code == nu.NU_ENOTSUP


def test_default_end_redshift_is_collapse_onset():
    pb = W.plain_small()[0].replace(z_end=0.0)
    info = nu.plan(pb)
    assert info["z_end"] == pytest.approx(200 ** (1 / 3) - 1, rel=1e-14)


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cosmo, halo, relic, radii, grid, opts = nu.structs(W.plain_small()[0], torch_alloc=False)
    with pytest.raises(nu.NuError) as e:
        nu.nu_profile_create(cosmo, halo, relic, radii, grid, opts)
    assert e.value.code in (nu.NU_ECUDA, nu.NU_ENOMEM)


def test_mass_reuse_plan_and_validation():
    pb = W.plain_small(precision=W.MIXED)[0]
    one = nu.plan(pb)
    assert one["n_masses"] == 1
    many = nu.plan(pb.replace(masses=(0.01, 0.05, 0.3)))
    assert many["n_masses"] == 3 and many["n_traj"] == one["n_traj"]
    assert many["device_bytes"] > one["device_bytes"]
    for bad in ((0.1, 0.0), (0.1, -1.0), (float("nan"),), tuple([0.1] * (nu.NU_MAX_MASSES + 1))):
        with pytest.raises(nu.NuError) as e:
            nu.plan(pb.replace(masses=bad))
        assert e.value.code == nu.NU_EINVAL
    cosmo, halo, relic, radii, grid, opts = nu.structs(pb, torch_alloc=False)
    relic.n_masses = 2                      # a count without a list
    with pytest.raises(nu.NuError) as e:
        nu.nu_profile_plan(cosmo, halo, relic, radii, grid, opts)
    assert e.value.code == nu.NU_EINVAL


def test_noalloc_refuses_mass_reuse_before_touching_the_gpu():
    pb = W.plain_small(precision=W.MIXED)[0].replace(masses=(0.05, 0.1))
    cosmo, halo, relic, radii, grid, opts = nu.structs(pb, torch_alloc=False)
    with pytest.raises(nu.NuError) as e:
        nu.nu_profile_compute_noalloc(cosmo, halo, relic, radii, grid, None)
    assert e.value.code == nu.NU_ENOTSUP


def test_tabulated_distribution_validation():
    pb = W.plain_small(precision=W.MIXED)[0]
    (fp, tab) = W.spectral_distortions()["thermal_bump"]
    ok = pb.replace(f_kind=W.F_TABLE, f_p=fp, f_table=tab)
    assert nu.plan(ok)["device_bytes"] > nu.plan(pb)["device_bytes"]
    for bad in (ok.replace(f_table=tab[:1]), ok.replace(f_p=(0.0, 40.0)),
                ok.replace(f_p=(5.0, 1.0)), ok.replace(f_table=(-1.0,) + tab[1:]),
                ok.replace(f_table=(float("inf"),) + tab[1:])):
        with pytest.raises(nu.NuError) as e:
            nu.plan(bad)
        assert e.value.code == nu.NU_EINVAL
    cosmo, halo, relic, radii, grid, opts = nu.structs(ok, torch_alloc=False)
    with pytest.raises(nu.NuError) as e:
        nu.nu_profile_compute_noalloc(cosmo, halo, relic, radii, grid, None)
    assert e.value.code == nu.NU_ENOTSUP


def test_verify_rules():
    """NU_FLAG_VERIFY: the FP64 twin's memory is planned with the request, and
    the flag needs the mixed mode."""
    pb = W.plain_small(precision=W.MIXED)[0]
    plain = nu.plan(pb)
    verified = nu.plan(pb, flags=nu.NU_FLAG_VERIFY)
    fp64 = nu.plan(pb.replace(precision=W.FP64))
    assert verified["device_bytes"] > plain["device_bytes"] + 0.9 * fp64["device_bytes"]
    with pytest.raises(nu.NuError) as e:
        nu.plan(pb.replace(precision=W.FP64), flags=nu.NU_FLAG_VERIFY)
    assert e.value.code == nu.NU_EINVAL


def test_resident_server_needs_whole_runs():
    """A resident server runs whole requests: chunked launches are refused
    before any GPU work."""
    with pytest.raises(nu.NuError) as e:
        nu.nu_server_create(device_bytes=64 << 20, chunk_steps=100, resident=True)
    assert e.value.code == nu.NU_EINVAL
