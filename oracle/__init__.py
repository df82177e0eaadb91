"""FP64 CPU oracle for the three-flavour vacuum oscillation chain.

TEST INFRASTRUCTURE ONLY.  This package may be used by the test-suite, by the
smoke check in ``__graft_entry__`` and by the benchmark's CPU-baseline leg.  The
CUDA library and its Python binding never import it; the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, double precision, sums in plain
index order); this module only loads it with ``ctypes`` and adds three steps
written in plain numpy/Python: the baseline weights, central finite
differences and the Levenberg-Marquardt fit loop.

Parity status of every function is pinned by ``tests/test_oracle_pins.py``
(closed forms, amplitude brute force, library quadrature, erf integrals,
finite differences), ``tests/test_oracle_pseudo.py`` (the generator's
known-answer vectors, the inversion's boundaries, the exact Poisson law) and
``tests/test_oracle_fit_pins.py`` (the fitter's iterates on designed linear
problems, derived by hand: the lambda schedule, rejections, ties, clamping);
nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fno-fast-math", _SRC,
            "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    lib.or_threads.restype = _I
    lib.or_set_threads.argtypes = [_I]
    lib.or_pmns.argtypes = [_D, _D, _D, _D, _PD, _PD]
    lib.or_prob.argtypes = [_I, _I, _D, _D, _D, _D, _D, _D, _D, _D, _I]
    lib.or_prob.restype = _D
    lib.or_pee.argtypes = [_PD, _I64, _D, _PD, _PD]
    lib.or_pee_grad.argtypes = [_PD, _I64, _D, _PD, _PD, _PD]
    lib.or_gl.argtypes = [_I, _PD, _PD]
    lib.or_gl.restype = _I
    lib.or_spectrum.argtypes = [_D, _D]
    lib.or_spectrum.restype = _D
    lib.or_binned.argtypes = [_I, _PD, _I, _PD, _PD, _I, _PD, _PD, _D, _PD, _PD]
    lib.or_binned.restype = _I
    lib.or_chi2.argtypes = [_I, _I, _PD, _PD, _PD, _D, _PD, _D, _PD, _I, _PD, _PD, _PD]
    lib.or_chi2.restype = _D
    lib.or_prob_grad.argtypes = [_I, _I, _PD, _D, _D, _I, _PD, _PD]
    lib.or_binned_general.argtypes = [_I, _PD, _I, _PD, _PD, _I, _PD, _PD, _I, _I, _I, _D, _PD, _PD]
    lib.or_binned_general.restype = _I
    _PU = ctypes.POINTER(ctypes.c_uint32)
    lib.or_philox4x32_10.argtypes = [_PU, _PU, _PU]
    lib.or_poisson_inv.argtypes = [_D, _D, _D]
    lib.or_poisson_inv.restype = _I64
    lib.or_pseudo_data.argtypes = [_PD, _PD, ctypes.POINTER(ctypes.c_int), _I, _I64, _I64, ctypes.c_uint64, _PD]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


class use_library:
    """Context manager that points this module at another build of oracle.c
    (used by the tests that plant mistakes in a copy of the oracle)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        _gl_cache.clear()
        _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        _gl_cache.clear()
        return False


def _p(a):
    return None if a is None else a.ctypes.data_as(_PD)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def threads() -> int:
    return _load().or_threads()


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def pmns(s12sq, s13sq, s23sq=0.5, delta=0.0) -> np.ndarray:
    """Complex 3x3 PMNS matrix U[alpha][i] (standard parameterisation)."""
    re = np.zeros(9)
    im = np.zeros(9)
    _load().or_pmns(s12sq, s13sq, s23sq, delta, _p(re), _p(im))
    return (re + 1j * im).reshape(3, 3)


def prob(alpha, beta, s12sq, s13sq, s23sq, delta, dm21, dm32, L_km, E_MeV, anti=False) -> float:
    """P(alpha -> beta), paper Sec. 4.1 general vacuum formula (alpha, beta in 0..2)."""
    return _load().or_prob(alpha, beta, s12sq, s13sq, s23sq, delta, dm21, dm32, L_km, E_MeV, int(anti))


def pee(E_MeV, L_km, osc) -> np.ndarray:
    """nue_bar survival probability on an energy array; osc = (s12^2, s13^2, dm21, dm32)."""
    E = _f64(E_MeV)
    o = _f64(osc)
    P = np.empty_like(E)
    _load().or_pee(_p(E), E.size, float(L_km), _p(o), _p(P))
    return P


def pee_grad(E_MeV, L_km, osc):
    """(P, dP/dtheta [n][4]) on an energy array."""
    E = _f64(E_MeV)
    o = _f64(osc)
    P = np.empty_like(E)
    dP = np.empty((E.size, 4))
    _load().or_pee_grad(_p(E), E.size, float(L_km), _p(o), _p(P), _p(dP))
    return P, dP


def gl(n: int):
    """n-point Gauss-Legendre nodes (ascending) and weights on [-1, 1]."""
    x = np.empty(n)
    w = np.empty(n)
    if _load().or_gl(int(n), _p(x), _p(w)) != 0:
        raise ValueError("n must be >= 1")
    return x, w


def spectrum(E_MeV, e_scale=1.0):
    return np.array([_load().or_spectrum(float(e), e_scale) for e in np.atleast_1d(E_MeV)])


def baseline_weights(L_km) -> np.ndarray:
    """omega_r = L_r^-2 / sum_s L_s^-2 (inverse-square flux weights)."""
    L = _f64(L_km)
    inv = 1.0 / (L * L)
    return inv / inv.sum()


_gl_cache: dict = {}


def _gl_cached(n):
    if n not in _gl_cache:
        _gl_cache[n] = gl(n)
    return _gl_cache[n]


def binned(edges, n, L_km, osc, e_scale=1.0, grad=False):
    """Per-baseline binned prediction mu[nL][nbins] (and d mu/d theta [nL][nbins][4])."""
    edges = _f64(edges)
    L = _f64(np.atleast_1d(L_km))
    o = _f64(osc)
    nb = edges.size - 1
    x, w = _gl_cached(int(n))
    mu = np.empty((L.size, nb))
    dmu = np.empty((L.size, nb, 4)) if grad else None
    _load().or_binned(nb, _p(edges), int(n), _p(x), _p(w), L.size, _p(L), _p(o), float(e_scale), _p(mu), _p(dmu))
    return (mu, dmu) if grad else mu


def chi2(omega, mu_rb, N, data, kind=0, eta=None, sigma=0.0, dmu_rb=None):
    """chi^2 of the combined prediction; returns dict(chi2, grad, J, mu)."""
    om = _f64(omega)
    mu_rb = _f64(mu_rb)
    nL, nb = mu_rb.shape
    d = _f64(data)
    e = None if eta is None else _f64(eta)
    dm = None if dmu_rb is None else _f64(dmu_rb)
    grad = np.empty(4 + nb) if dm is not None else None
    J = np.empty((nb, 4)) if dm is not None else None
    mu = np.empty(nb)
    c = _load().or_chi2(nb, nL, _p(om), _p(mu_rb), _p(dm), float(N), _p(e), float(sigma), _p(d), int(kind),
                        _p(grad), _p(J), _p(mu))
    return {"chi2": c, "grad": grad, "J": J, "mu": mu}


def chain(edges, n, L_km, osc, N, data, kind=0, eta=None, sigma=0.0, e_scale=1.0, omega=None, grad=True):
    """One full evaluation of the chain at one parameter point.

    Returns dict(chi2, grad[4+nbins], J[nbins][4], mu[nbins], mu_rb[nL][nbins],
    dmu_rb[nL][nbins][4]).
    """
    L = np.atleast_1d(_f64(L_km))
    om = baseline_weights(L) if omega is None else _f64(omega)
    if grad:
        mu_rb, dmu_rb = binned(edges, n, L, osc, e_scale, grad=True)
    else:
        mu_rb, dmu_rb = binned(edges, n, L, osc, e_scale, grad=False), None
    out = chi2(om, mu_rb, N, data, kind, eta, sigma, dmu_rb)
    out["mu_rb"] = mu_rb
    out["dmu_rb"] = dmu_rb
    out["omega"] = om
    return out


FLAVOUR = {"e": 0, "mu": 1, "tau": 2}


def prob_grad(alpha, beta, osc6, L_km, E_MeV, anti=False):
    """P(alpha -> beta) and dP / d(s12^2, s13^2, s23^2, delta, dm2_21, dm2_32) at one
    energy, from the Sec. 4.1 formula and the product rule on the mixing matrix."""
    P = ctypes.c_double()
    dP = np.empty(6)
    _load().or_prob_grad(FLAVOUR.get(alpha, alpha), FLAVOUR.get(beta, beta), _p(_f64(osc6)), float(L_km),
                         float(E_MeV), int(bool(anti)), ctypes.byref(P), _p(dP))
    return P.value, dP


def binned_general(edges, n, L_km, osc6, alpha, beta, anti=False, e_scale=1.0):
    """Per-baseline binned prediction of P(alpha -> beta): mu[nL][nbins] and
    d mu / d(six parameters) [nL][nbins][6]."""
    edges = _f64(edges)
    L = _f64(np.atleast_1d(L_km))
    nb = edges.size - 1
    x, w = _gl_cached(int(n))
    mu = np.empty((L.size, nb))
    dmu = np.empty((L.size, nb, 6))
    _load().or_binned_general(nb, _p(edges), int(n), _p(x), _p(w), L.size, _p(L), _p(_f64(osc6)),
                              FLAVOUR.get(alpha, alpha), FLAVOUR.get(beta, beta), int(bool(anti)),
                              float(e_scale), _p(mu), _p(dmu))
    return mu, dmu


def chain_general(edges, n, L_km, osc6, N, data, alpha, beta, anti=False, kind=0, eta=None, sigma=0.0,
                  e_scale=1.0, omega=None):
    """One evaluation of the chain for P(alpha -> beta) at one point of the six
    parameters.  The detector combination and chi^2 are the textbook ones of
    ``chi2`` (M_i = sum_r omega_r mu[r][i], mu_i = N (1 + eta_i) M_i, Pearson or
    Poisson, the nuisance penalty), written out here for six parameters.
    Returns dict(chi2, grad[6 + nbins], J[nbins][6] = d mu_i / d(parameters),
    mu[nbins], mu_rb, dmu_rb)."""
    L = np.atleast_1d(_f64(L_km))
    om = baseline_weights(L) if omega is None else _f64(omega)
    mu_rb, dmu_rb = binned_general(edges, n, L, osc6, alpha, beta, anti, e_scale)
    d = _f64(data)
    nb = d.size
    e = np.zeros(nb) if eta is None else _f64(eta)
    chi2v = 0.0
    grad = np.zeros(6 + nb)
    J = np.empty((nb, 6))
    mu = np.empty(nb)
    for i in range(nb):
        M = sum(om[r] * mu_rb[r, i] for r in range(L.size))
        dM = sum(om[r] * dmu_rb[r, i] for r in range(L.size))
        J[i] = N * (1.0 + e[i]) * dM
        m = N * (1.0 + e[i]) * M
        if kind == 0:
            term = (d[i] - m) ** 2 / m
            gi = 1.0 - d[i] * d[i] / (m * m)
        else:
            term = 2.0 * (m - d[i] + d[i] * np.log(d[i] / m)) if d[i] > 0 else 2.0 * m
            gi = 2.0 * (1.0 - d[i] / m)
        chi2v += term
        mu[i] = m
        grad[:6] += gi * N * (1.0 + e[i]) * dM
        grad[6 + i] = gi * N * M
        if eta is not None and sigma > 0:
            chi2v += e[i] * e[i] / (sigma * sigma)
            grad[6 + i] += 2.0 * e[i] / (sigma * sigma)
    return {"chi2": chi2v, "grad": grad, "J": J, "mu": mu, "mu_rb": mu_rb, "dmu_rb": dmu_rb, "omega": om}


def norm_for_total(edges, n, L_km, osc, total=1e5, e_scale=1.0, omega=None) -> float:
    """N such that sum_i N * sum_r omega_r mu[r][i] = total at the given point."""
    L = np.atleast_1d(_f64(L_km))
    om = baseline_weights(L) if omega is None else _f64(omega)
    mu_rb = binned(edges, n, L, osc, e_scale)
    return float(total / (om @ mu_rb).sum())


def fd_grad(f, theta, rel_h=1e-6):
    """Central finite differences of a scalar function, h = rel_h * |theta_q|."""
    theta = _f64(theta)
    g = np.empty_like(theta)
    for q in range(theta.size):
        h = rel_h * abs(theta[q]) if theta[q] != 0 else rel_h
        tp = theta.copy()
        tm = theta.copy()
        tp[q] += h
        tm[q] -= h
        g[q] = (f(tp) - f(tm)) / (2 * h)
    return g


FIT_BOX = {
    # (s2_12, s2_13, dm2_21, dm2_32)
    4: ((1e-6, 1e-6, 1e-7, 1e-7), (1 - 1e-6, 1 - 1e-6, np.inf, np.inf)),
    # (s2_12, s2_13, s2_23, delta_cp, dm2_21, dm2_32): delta_cp is free
    6: ((1e-6, 1e-6, 1e-6, -np.inf, 1e-7, 1e-7), (1 - 1e-6, 1 - 1e-6, 1 - 1e-6, np.inf, np.inf, np.inf)),
}


def fit_lm(evaluate, theta0, iters=20, lam0=1e-3, lo=None, hi=None):
    """Levenberg-Marquardt-damped Gauss-Newton, a fixed number of evaluations.

    The paper has no fitter; this is the textbook method in the order chosen for
    the batched fits: every iteration evaluates (chi2, g, J, mu) once at the
    trial point; if chi2 improved on the best point so far the trial becomes the
    current point and lambda /= 10, otherwise the trial is rejected and
    lambda *= 10; then H = sum_i (2/mu_i) J_i J_i^T (expected Fisher matrix),
    solve (H + lambda diag H) delta = -g at the current point and clamp the
    next trial into the box [lo, hi] (FIT_BOX for 4 or 6 parameters unless
    given).  ``evaluate(theta)`` must return a dict with chi2, grad (its first
    len(theta0) entries used), J [nbins][len(theta0)] and mu.  Returns
    (theta_best, chi2_best, history of chi2 per evaluation).
    """
    trial = _f64(theta0).copy()
    npar = trial.size
    lo = np.asarray(FIT_BOX[npar][0] if lo is None else lo, dtype=np.float64)
    hi = np.asarray(FIT_BOX[npar][1] if hi is None else hi, dtype=np.float64)
    best_theta = None
    best_chi2 = np.inf
    g = H = None
    lam = lam0
    hist = []
    for _ in range(iters):
        r = evaluate(trial)
        hist.append(r["chi2"])
        if r["chi2"] < best_chi2:
            best_chi2 = r["chi2"]
            best_theta = trial.copy()
            g = r["grad"][:npar].copy()
            Jm = r["J"]
            H = (Jm.T * (2.0 / r["mu"])) @ Jm
            lam = lam / 10.0
        else:
            lam = lam * 10.0
        A = H + lam * np.diag(np.diag(H))
        delta = np.linalg.solve(A, -g)
        trial = np.minimum(np.maximum(best_theta + delta, lo), hi)
    return best_theta, best_chi2, np.array(hist)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4 x 32-bit counter under a 2 x 32-bit key."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.empty(4, dtype=np.uint32)
    PU = ctypes.POINTER(ctypes.c_uint32)
    _load().or_philox4x32_10(c.ctypes.data_as(PU), k.ctypes.data_as(PU), out.ctypes.data_as(PU))
    return out


def poisson_inv(mu: float, u: float) -> int:
    """Poisson(mu) by inversion of one uniform (e^-mu from the host's libm)."""
    import math

    return int(_load().or_poisson_inv(float(mu), math.exp(-float(mu)), float(u)))


def pseudo_data(mu, nds: int, seed: int, j0: int = 0) -> np.ndarray:
    """Poisson pseudo-data sets j0 .. j0 + nds - 1 of the bin means mu: [nds][nbins].
    A mean is drawn as the sum of M = ceil(mu / 500) parts of mean mu / M."""
    import math

    m = _f64(mu)
    parts = np.array([max(1, math.ceil(v / 500.0)) for v in m], dtype=np.int32)
    mp = np.array([v / int(c) for v, c in zip(m, parts)])
    em = np.array([math.exp(-v) for v in mp])  # the C library's exp, as the product's host code uses
    out = np.empty((int(nds), m.size))
    _load().or_pseudo_data(_p(mp), _p(em), parts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), m.size, int(j0),
                           int(nds), ctypes.c_uint64(int(seed)), _p(out))
    return out
