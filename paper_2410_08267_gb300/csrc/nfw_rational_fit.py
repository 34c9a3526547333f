"""Derivation of the FP32 rational functions for the NFW enclosed-mass shape.

The trajectory kernel's FP32 force evaluates I(y) = ln(1+y) - y/(1+y)
(Eq. nfw) inside the NFW part as y^2 g(y), where g(y) = I(y)/y^2 is
approximated by a rational function N(y)/D(y) with D(0) = 1. There are two
fits, and a request uses one of them for all of its evaluations:
* wide: numerator degree 4, denominator degree 5, on 0 <= y <= 16. It covers
  the whole NFW part of any halo with c <= 16 (halos with a larger c use the
  logarithm above y = 16);
* narrow: degrees 4 and 4 on 0 <= y <= 8, one fused multiply-add cheaper, for
  halos with c <= 8.
g is analytic except for a logarithmic branch point at y = -1. Rational
functions follow it far better than polynomials: a degree-9 polynomial reaches
the same accuracy only on [0, 1].

Fit: relative-error minimax by Lawson's iteration on linearised least squares.
Each step minimises sum_i w_i (N(y_i) - g_i D(y_i))^2 / (g_i D_prev(y_i))^2
over 2000 Chebyshev nodes of [0, Y], then multiplies each weight by its
relative error. The variable is scaled to [0, 1] for conditioning, and the
coefficients are scaled back by powers of Y, which is exact. Reference values
of g are computed in 30-digit arithmetic (mpmath).

Run:  python paper_2410_08267_gb300/csrc/nfw_rational_fit.py
It prints, for each fit, the coefficients in ascending powers of y (float32)
in the form used in traj_kernel.cu, the fit's relative error, and the error of
the float32 evaluation (Horner for N and D, then N / D) on a dense grid.
"""
import mpmath
import numpy as np

FITS = (("wide", 4, 5, 16.0), ("narrow", 4, 4, 8.0))
NODES = 2000
ITERS = 80


def g(y):
    y = mpmath.mpf(y)
    if y == 0:
        return mpmath.mpf(1) / 2
    return (mpmath.log1p(y) - y / (1 + y)) / y ** 2


def fit(n_deg, d_deg, y_max):
    mpmath.mp.dps = 30
    xs = 0.5 - 0.5 * np.cos(np.pi * (np.arange(NODES) + 0.5) / NODES)     # y / y_max
    gv = np.array([float(g(y_max * x)) for x in xs])
    w = np.full(NODES, 1.0 / NODES)
    d_prev = np.ones(NODES)
    best = None
    for _ in range(ITERS):
        A = np.hstack([np.vander(xs, n_deg + 1, increasing=True),
                       -gv[:, None] * np.vander(xs, d_deg + 1, increasing=True)[:, 1:]])
        s = np.sqrt(w) / (gv * np.abs(d_prev))
        cf = np.linalg.lstsq(A * s[:, None], gv * s, rcond=None)[0]
        a = cf[:n_deg + 1]
        b = np.concatenate([[1.0], cf[n_deg + 1:]])
        num = np.polyval(a[::-1], xs)
        den = np.polyval(b[::-1], xs)
        err = num / den / gv - 1.0
        e = float(np.max(np.abs(err)))
        if best is None or e < best[0]:
            best = (e, a.copy(), b.copy())
        w = w * np.abs(err)
        w /= w.sum()
        d_prev = den
    e, a, b = best
    scale_a = y_max ** -np.arange(n_deg + 1)
    scale_b = y_max ** -np.arange(d_deg + 1)
    return e, (a * scale_a).astype(np.float32), (b * scale_b).astype(np.float32)


def eval_f32(a, b, y):
    y = np.asarray(y, dtype=np.float32)
    num = np.full_like(y, a[-1])
    for c in a[-2::-1]:
        num = (num * y + c).astype(np.float32)
    den = np.full_like(y, b[-1])
    for c in b[-2::-1]:
        den = (den * y + c).astype(np.float32)
    return (num / den).astype(np.float32)


def f32_error(a, b, y_max, n=4001):
    ys = np.linspace(0.0, y_max, n).astype(np.float32)
    ex = np.array([float(g(float(v))) for v in ys])
    return float(np.max(np.abs(eval_f32(a, b, ys).astype(np.float64) / ex - 1.0)))


if __name__ == "__main__":
    for name, n_deg, d_deg, y_max in FITS:
        e, a, b = fit(n_deg, d_deg, y_max)
        print(f"{name}: degrees ({n_deg}, {d_deg}) on [0, {y_max:g}]")
        for j, v in enumerate(a):
            print(f"    N{j} = {float(v):.9e}f")
        for j, v in enumerate(b):
            print(f"    D{j} = {float(v):.9e}f")
        print("    fit relative error:", e)
        print("    max relative error (float32 evaluation):", f32_error(a, b, y_max))
