"""Derivation of the FP32 polynomial for the NFW enclosed-mass shape.

The trajectory kernel evaluates I(y) = ln(1+y) - y/(1+y) (Eq. nfw) for
0 <= y < 1 as y^2 P(y), where P is a degree-9 polynomial fitted here to
g(y) = I(y)/y^2 by least squares with relative weights on 400 Chebyshev
nodes of [0, 1], in 40-digit arithmetic (mpmath).  g is analytic on the disc
|y| < 1 around 0 with its nearest singularity at y = -1, so polynomials on
[0, 1] converge geometrically; degree 9 reaches about 3e-7 relative after
rounding the coefficients to float32 and evaluating by Horner in float32.
Above y = 1 the two terms of I differ by more than a factor 1.5 and the kernel
subtracts them directly.

Run:  python paper_2410_08267_gb300/csrc/nfw_poly_fit.py
prints the coefficients (ascending powers) in the form pasted into traj_kernel.cu
and the float32 error on a dense grid.
"""
import mpmath
import numpy as np

DEG = 9
Y_MAX = 1.0
NODES = 400


def g(y):
    y = mpmath.mpf(y)
    if y == 0:
        return mpmath.mpf(1) / 2
    return (mpmath.log1p(y) - y / (1 + y)) / y ** 2


def fit():
    mpmath.mp.dps = 40
    xs = [Y_MAX * (1 - mpmath.cos(mpmath.pi * (k + mpmath.mpf(1) / 2) / NODES)) / 2
          for k in range(NODES)]
    A = mpmath.matrix(NODES, DEG + 1)
    b = mpmath.matrix(NODES, 1)
    for i, x in enumerate(xs):
        gv = g(x)
        for j in range(DEG + 1):
            A[i, j] = x ** j / gv
        b[i] = 1
    c = mpmath.lu_solve(A.T * A, A.T * b)
    return np.array([float(v) for v in c], dtype=np.float32)


def max_rel_err(cf):
    ys = np.linspace(0.0, Y_MAX, 4001).astype(np.float32)
    p = np.full_like(ys, cf[-1])
    for j in range(DEG - 1, -1, -1):
        p = (p * ys + cf[j]).astype(np.float32)
    ex = np.array([float(g(float(v))) for v in ys])
    return float(np.max(np.abs(p.astype(np.float64) - ex) / ex))


if __name__ == "__main__":
    cf = fit()
    for j, v in enumerate(cf):
        print(f"    constexpr float kP{j} = {float(v):.9e}f;")
    print("max relative error (float32 Horner):", max_rel_err(cf))
