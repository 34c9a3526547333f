"""Derivation of the FP32 rational function for the NFW enclosed-mass shape.

The trajectory kernel's FP32 force evaluates I(y) = ln(1+y) - y/(1+y)
(Eq. nfw) inside the NFW part as y^2 g(y) with g(y) = I(y)/y^2 approximated
by a rational function N(y)/D(y), numerator degree 4 and denominator degree 5
(D(0) = 1), on 0 <= y <= 16: one formula for every y up to the NFW edge y = c
of any halo with c <= 16 (halos with a larger c use the logarithm above
y = 16).  g is analytic except for a logarithmic branch point at y = -1,
which rational functions follow far better than polynomials (a degree-9
polynomial reaches the same accuracy only on [0, 1]).

Fit: relative-error minimax by Lawson's iteration on linearised least squares
(minimise sum_i w_i (N(y_i) - g_i D(y_i))^2 / (g_i D_prev(y_i))^2 over 2000
Chebyshev nodes of [0, 16], then multiply each weight by its relative error),
with the variable scaled to [0, 1] for conditioning and the coefficients
scaled back by powers of 16 (exact).  Reference values of g in 30-digit
arithmetic (mpmath).

Run:  python paper_2410_08267_gb300/csrc/nfw_rational_fit.py
prints the coefficients (ascending powers of y, float32) in the form used in
traj_kernel.cu, the fit's relative error and the error of the float32
evaluation (Horner for N and D, then N / D) on a dense grid.
"""
import mpmath
import numpy as np

N_DEG, D_DEG = 4, 5
Y_MAX = 16.0
NODES = 2000
ITERS = 80


def g(y):
    y = mpmath.mpf(y)
    if y == 0:
        return mpmath.mpf(1) / 2
    return (mpmath.log1p(y) - y / (1 + y)) / y ** 2


def fit():
    mpmath.mp.dps = 30
    xs = 0.5 - 0.5 * np.cos(np.pi * (np.arange(NODES) + 0.5) / NODES)     # y / Y_MAX
    gv = np.array([float(g(Y_MAX * x)) for x in xs])
    w = np.full(NODES, 1.0 / NODES)
    d_prev = np.ones(NODES)
    best = None
    for _ in range(ITERS):
        A = np.hstack([np.vander(xs, N_DEG + 1, increasing=True),
                       -gv[:, None] * np.vander(xs, D_DEG + 1, increasing=True)[:, 1:]])
        s = np.sqrt(w) / (gv * np.abs(d_prev))
        cf = np.linalg.lstsq(A * s[:, None], gv * s, rcond=None)[0]
        a = cf[:N_DEG + 1]
        b = np.concatenate([[1.0], cf[N_DEG + 1:]])
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
    scale_a = Y_MAX ** -np.arange(N_DEG + 1)
    scale_b = Y_MAX ** -np.arange(D_DEG + 1)
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


def f32_error(a, b, n=4001):
    ys = np.linspace(0.0, Y_MAX, n).astype(np.float32)
    ex = np.array([float(g(float(v))) for v in ys])
    return float(np.max(np.abs(eval_f32(a, b, ys).astype(np.float64) / ex - 1.0)))


if __name__ == "__main__":
    e, a, b = fit()
    for j, v in enumerate(a):
        print(f"    N{j} = {float(v):.9e}f")
    for j, v in enumerate(b):
        print(f"    D{j} = {float(v):.9e}f")
    print("fit relative error:", e)
    print("max relative error (float32 evaluation):", f32_error(a, b))
