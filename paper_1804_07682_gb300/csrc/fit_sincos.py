"""Generate ff_consts.h: FP32 polynomial coefficients for sin and cos on the
reduced range |r| <= pi/2 (+ margin) and a 3-part split of pi for the
Cody-Waite reduction of the oscillation phase modulo pi.

Method: weighted least squares on Chebyshev-distributed points, iterated with
Lawson's reweighting toward the minimax solution, for
    sin r = r + r u (S1 + u (S2 + ... )),   u = r^2,
    cos r = 1 + u (C1 + u (C2 + ... )),
then the coefficients are rounded to float32 and the float32 Horner evaluation
is checked against the double-precision functions.

Run:  python fit_sincos.py > ff_consts.h
"""
import math
import sys
from fractions import Fraction

import numpy as np

R_MAX = math.pi / 2 + 2e-3
N_SIN = 4  # S1..S4: odd degree 9 (error ~5e-9)
N_COS = 4  # C1..C4: even degree 8 (error ~5e-8)

# pi to 60 digits (textbook value)
PI = Fraction("3.14159265358979323846264338327950288419716939937510582097494")


def lawson(basis, target, weight, iters=200):
    """minimise max |weight * (basis @ c - target)| by Lawson reweighting
    (weights floored so that no sample point drops out of the fit)."""
    lw = np.ones(target.size) / target.size
    c = None
    for _ in range(iters):
        sw = np.sqrt(lw)
        c, *_ = np.linalg.lstsq(basis * (sw * weight)[:, None], sw * weight * target, rcond=None)
        err = np.abs(weight * (basis @ c - target))
        lw = lw * (err / err.max()) + 1e-12
        lw /= lw.sum()
    return c


def fit_sequential(basis, target, weight):
    """Fit, round the lowest free coefficient to float32, refit the rest with
    it fixed; repeat.  Keeps the float32 rounding of the large low-order
    coefficients from dominating the error."""
    n = basis.shape[1]
    fixed = []
    for k in range(n):
        resid = target - (basis[:, :k] @ np.array(fixed) if k else 0.0)
        c = lawson(basis[:, k:], resid, weight)
        fixed.append(float(np.float32(c[0])))
    return np.array(fixed)


def fit():
    t = np.cos(np.linspace(0, np.pi, 6001))  # Chebyshev points on [-1, 1]
    r = 0.5 * (t + 1) * R_MAX
    r = r[r > 1e-3]
    u = r * r
    # sin: (sin r - r) / (r u) = S1 + S2 u + ...; absolute error weight r u
    fs = (np.sin(r) - r) / (r * u)
    Bs = np.stack([u ** k for k in range(N_SIN)], axis=1)
    cs = fit_sequential(Bs, fs, r * u)
    # cos: (cos r - 1) / u = C1 + C2 u + ...; absolute error weight u
    fc = (np.cos(r) - 1) / u
    Bc = np.stack([u ** k for k in range(N_COS)], axis=1)
    cc = fit_sequential(Bc, fc, u)
    return cs, cc


def f32(x):
    return np.float32(x)


def fma32(a, b, c):
    # a*b exact in double for float32 inputs; one rounding to float32
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def eval_sin32(r, cs):
    r = f32(r)
    u = f32(r * r)
    p = f32(cs[-1])
    for ck in cs[-2::-1]:
        p = fma32(p, u, f32(ck))
    ru = f32(r * u)
    return fma32(ru, p, r)


def eval_cos32(r, cc):
    r = f32(r)
    u = f32(r * r)
    p = f32(cc[-1])
    for ck in cc[-2::-1]:
        p = fma32(p, u, f32(ck))
    return fma32(u, p, f32(1.0))


def split_pi():
    """pi = A + B + C with A, B holding 12 significant bits each (so q*A and
    q*B are exact for integer q < 2^12) and C the float32 rounding of the rest."""
    def top_bits(x, bits):
        e = math.floor(math.log2(float(x)))
        scale = Fraction(2) ** (bits - 1 - e)
        return Fraction(math.floor(x * scale)) / scale
    A = top_bits(PI, 12)
    B = top_bits(PI - A, 12)
    C = float(np.float32(float(PI - A - B)))
    return float(A), float(B), C


def main():
    cs, cc = fit()
    cs32 = [f32(c) for c in cs]
    cc32 = [f32(c) for c in cc]
    rr = np.linspace(-R_MAX, R_MAX, 200001)
    es = max(abs(float(eval_sin32(x, cs32)) - math.sin(x)) for x in rr[::20])
    ec = max(abs(float(eval_cos32(x, cc32)) - math.cos(x)) for x in rr[::20])
    # polynomial error alone (double evaluation of the float32 coefficients)
    uu = rr * rr
    ps = rr + rr * uu * sum(float(c) * uu ** k for k, c in enumerate(cs32))
    pc = 1 + uu * sum(float(c) * uu ** k for k, c in enumerate(cc32))
    eps_s = np.abs(ps - np.sin(rr)).max()
    eps_c = np.abs(pc - np.cos(rr)).max()
    A, B, C = split_pi()
    assert A * 4096 == float(np.float32(A * 4096)) and A == float(np.float32(A))
    out = sys.stdout
    out.write("// Generated by fit_sincos.py -- do not edit.\n")
    out.write("// FP32 minimax-style polynomials on |r| <= %.6f (Lawson-weighted least squares).\n" % R_MAX)
    out.write("// Polynomial error (double evaluation): sin %.2e, cos %.2e.\n" % (eps_s, eps_c))
    out.write("// Float32 Horner evaluation error (sampled): sin %.2e, cos %.2e.\n" % (es, ec))
    out.write("#pragma once\n")
    for k, c in enumerate(cs32):
        out.write("#define GNA_SIN_C%d (%.9ef)\n" % (k + 1, float(c)))
    for k, c in enumerate(cc32):
        out.write("#define GNA_COS_C%d (%.9ef)\n" % (k + 1, float(c)))
    out.write("// pi = PI_A + PI_B + PI_C; PI_A and PI_B have 12 significant bits.\n")
    out.write("#define GNA_PI_A (%.17gf)\n" % A)
    out.write("#define GNA_PI_B (%.17gf)\n" % B)
    out.write("#define GNA_PI_C (%.9ef)\n" % C)
    # two-part split for the fused kernels: PI_B2 = float32(pi - PI_A)
    B2 = float(np.float32(float(PI - Fraction(A))))
    err2 = abs(float(PI - Fraction(A) - Fraction(B2)))
    out.write("// pi = PI_A + PI_B2 + e2 with PI_B2 the float32 rounding of pi - PI_A, |e2| = %.2e.\n" % err2)
    out.write("#define GNA_PI_B2 (%.9ef)\n" % B2)
    out.write("#define GNA_PI_E2 (%.3e)\n" % err2)
    out.write("#define GNA_INV_PI_F (%.9ef)\n" % float(np.float32(1 / math.pi)))
    # double-precision split for the FP64-phase variant: 26 + 26 bits + rest
    def top_bits(x, bits):
        e = math.floor(math.log2(float(x)))
        scale = Fraction(2) ** (bits - 1 - e)
        return Fraction(math.floor(x * scale)) / scale
    DA = top_bits(PI, 26)
    DB = top_bits(PI - DA, 26)
    DC = float(PI - DA - DB)
    out.write("// pi = PI_DA + PI_DB + PI_DC in double; PI_DA, PI_DB have 26 significant bits.\n")
    out.write("#define GNA_PI_DA (%.17g)\n" % float(DA))
    out.write("#define GNA_PI_DB (%.17g)\n" % float(DB))
    out.write("#define GNA_PI_DC (%.17g)\n" % DC)
    out.write("#define GNA_INV_PI_D (%.17g)\n" % (1 / math.pi))


if __name__ == "__main__":
    main()
