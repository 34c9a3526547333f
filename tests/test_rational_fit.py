"""The FP32 force's rational approximations of I(y)/y^2 (Eq. nfw) in the
trajectory kernel are the ones the committed derivation produces, and they
meet their stated accuracy.

The derivation script fits each rational function. This test re-runs it and
compares its float32 coefficients with the literals in traj_kernel.cu, in
both the scalar and the packed evaluation. It then checks every fit against
I(y) computed independently in 40-digit arithmetic, on the whole range of
the fit."""
import importlib.util
import os
import re

import mpmath
import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2410_08267_gb300", "csrc")


def _fit_module():
    spec = importlib.util.spec_from_file_location("nfw_rational_fit",
                                                  os.path.join(CSRC, "nfw_rational_fit.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _kernel_horner(src, fname):
    """Coefficients of a Horner function in the kernel source, highest power first."""
    body = re.search(fname + r"\(float y\)\s*\{(.*?)\n\}", src, re.S).group(1)
    return [np.float32(v) for v in re.findall(r"(-?\d\.\d+e[-+]\d+)f", body)]


@pytest.fixture(scope="module")
def fits():
    mod = _fit_module()
    return {name: mod.fit(n, d, y) + (y,) for name, n, d, y in mod.FITS}


@pytest.mark.parametrize("name,nf,df", [("wide", "nfw_N16", "nfw_D16"), ("narrow", "nfw_N8", "nfw_D8")])
def test_kernel_coefficients_are_the_derived_ones(fits, name, nf, df):
    src = open(os.path.join(CSRC, "traj_kernel.cu")).read()
    _, a, b, _ = fits[name]
    n_k = _kernel_horner(src, nf)
    d_k = _kernel_horner(src, df)
    # The kernel lists N fully; D's constant term 1 is written as "1.0f". A
    # float32 coefficient may differ by an ulp when the least-squares solve
    # rounds differently on another machine.
    ulp2 = 2.0 ** -22
    assert np.allclose(n_k, a[::-1], rtol=ulp2, atol=0.0)
    assert np.allclose(d_k, b[:0:-1], rtol=ulp2, atol=0.0)
    assert b[0] == np.float32(1.0)
    # the packed evaluation uses the same literals as the scalar one
    for v in n_k + d_k:
        assert src.count(f"{float(v):.9e}f") == 2, v


def test_fits_meet_their_accuracy(fits):
    mpmath.mp.dps = 40
    for name, (e, a, b, y_max) in fits.items():
        assert e < 1e-7, (name, e)
        ys = np.linspace(0.0, y_max, 801)[1:]
        num = np.polyval(np.asarray(a, np.float64)[::-1], ys)
        den = np.polyval(np.asarray(b, np.float64)[::-1], ys)
        ref = np.array([float((mpmath.log1p(y) - y / (1 + mpmath.mpf(y))) / mpmath.mpf(y) ** 2)
                        for y in ys])
        # float32 coefficients evaluated exactly: the fit plus coefficient rounding
        assert np.max(np.abs(num / den / ref - 1.0)) < 3e-7, name
        assert np.all(den > 0.0)
