"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the fact it uses: closed forms of the general vacuum formula
(paper Sec. 4.1), the plane-wave amplitude it is derived from, flavour
unitarity, the Jarlskog invariant, the textbook phase constant 1.267, library
quadrature (numpy leggauss, scipy erf, scipy eval_legendre), exact
Gauss-Legendre degrees, mpmath brute force at 50 digits, closed chi^2 cases and
central finite differences.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1804_07682_gb300 import workloads as wl

TRUTH = wl.TRUTH
# Textbook phase constant: dm2 L / (4E) = 1.2669326794 dm2[eV^2] L[km] / E[GeV]
# (hbar c = 197.3269804 MeV fm); the oracle forms the phase from hbar c itself.
K_GEV = 1.2669326794


def amplitude_prob(U, a, b, dm21, dm32, L_km, E_MeV, anti):
    """|sum_i V*_ai V_bi exp(-i m_i^2 L / 2E)|^2: the plane-wave amplitude that the
    paper's Sec. 4.1 formula expands (brute force, no trigonometric identities)."""
    V = U.conj() if anti else U
    m2 = np.array([0.0, dm21, dm21 + dm32])
    # m_i^2 L / (2E) with L / (hbar c) in 1/eV (hbar c = 197.3269804 MeV fm);
    # the value of the phase constant itself is pinned by the 1.267 tests below.
    ph = m2 * (L_km * 1e3 / 197.3269804e-9) / (2.0 * E_MeV * 1e6)
    amp = np.sum(V[a, :].conj() * V[b, :] * np.exp(-1j * ph))
    return abs(amp) ** 2


# ---------------------------------------------------------------- PMNS ----
def test_pmns_unitary_and_moduli():
    s12, s13, s23, d = 0.307, 0.0218, 0.45, 1.2 * np.pi
    U = oracle.pmns(s12, s13, s23, d)
    assert np.abs(U @ U.conj().T - np.eye(3)).max() < 1e-15
    # textbook moduli of the standard parameterisation
    assert abs(abs(U[0, 2]) ** 2 - s13) < 1e-15
    assert abs(abs(U[0, 1]) ** 2 - s12 * (1 - s13)) < 1e-15
    assert abs(abs(U[0, 0]) ** 2 - (1 - s12) * (1 - s13)) < 1e-15
    assert abs(abs(U[1, 2]) ** 2 - s23 * (1 - s13)) < 1e-15
    assert abs(abs(U[2, 2]) ** 2 - (1 - s23) * (1 - s13)) < 1e-15
    # Jarlskog invariant J = Im(U_mu3 U*_e3 U_e2 U*_mu2) = c12 s12 c23 s23 c13^2 s13 sin(delta)
    J = np.imag(U[1, 2] * U[0, 2].conj() * U[0, 1] * U[1, 1].conj())
    c12, c13, c23 = math.sqrt(1 - s12), math.sqrt(1 - s13), math.sqrt(1 - s23)
    Jref = c12 * math.sqrt(s12) * c23 * math.sqrt(s23) * c13 ** 2 * math.sqrt(s13) * math.sin(d)
    assert abs(J - Jref) < 1e-15


# --------------------------------------------------------- probability ----
@pytest.mark.parametrize("anti", [False, True])
def test_prob_equals_amplitude_brute_force(anti):
    s12, s13, s23, d = 0.307, 0.0218, 0.45, 1.2 * np.pi
    U = oracle.pmns(s12, s13, s23, d)
    rng = np.random.default_rng(5)
    for _ in range(40):
        L = rng.uniform(0.1, 1000.0)
        E = rng.uniform(0.5, 5000.0)
        for a, b in itertools.product(range(3), range(3)):
            p = oracle.prob(a, b, s12, s13, s23, d, 7.53e-5, 2.44e-3, L, E, anti)
            ref = amplitude_prob(U, a, b, 7.53e-5, 2.44e-3, L, E, anti)
            assert abs(p - ref) < 2e-12, (a, b, L, E, p, ref)


def test_prob_is_one_at_zero_baseline():
    for a, b in itertools.product(range(3), range(3)):
        p = oracle.prob(a, b, 0.307, 0.0218, 0.45, 1.2 * np.pi, 7.53e-5, 2.44e-3, 0.0, 3.0, False)
        assert p == (1.0 if a == b else 0.0)
    E = np.linspace(1.0, 10.0, 17)
    assert np.all(oracle.pee(E, 0.0, TRUTH) == 1.0)


def test_two_flavour_limits():
    E = np.linspace(1.8, 12.0, 301)
    L = 52.5
    s12, s13, dm21, dm32 = TRUTH
    # theta13 -> 0: P = 1 - sin^2(2 theta12) sin^2(1.267 dm21 L / E)
    p = oracle.pee(E, L, (s12, 0.0, dm21, dm32))
    ref = 1 - 4 * s12 * (1 - s12) * np.sin(K_GEV * dm21 * L / (E * 1e-3)) ** 2
    assert np.abs(p - ref).max() < 1e-7  # 1e-7: the constant is given to 9 digits
    # dm21 -> 0: P = 1 - sin^2(2 theta13) sin^2(1.267 dm31 L / E), dm31 = dm32
    p = oracle.pee(E, L, (s12, s13, 0.0, dm32))
    ref = 1 - 4 * s13 * (1 - s13) * np.sin(K_GEV * dm32 * L / (E * 1e-3)) ** 2
    assert np.abs(p - ref).max() < 1e-7


def test_phase_constant_textbook_1267():
    # two-flavour point where 1.267 dm2 L/E = pi/4: P = 1 - sin^2(2 theta)/2 and
    # dP/dphase = -sin^2(2 theta), so P pins the phase constant to first order.
    s13, dm = 0.1, 2.5e-3
    L = 1.0
    E_GeV = K_GEV * dm * L / (np.pi / 4)
    p = oracle.pee([E_GeV * 1e3], L, (0.0, s13, 0.0, dm))[0]
    sin22 = 4 * s13 * (1 - s13)
    assert abs(p - (1 - sin22 / 2)) < 1e-9
    # the value as printed to 4 digits (1.267) agrees to its own precision
    E4 = 1.267 * dm * L / (np.pi / 4)
    p4 = oracle.pee([E4 * 1e3], L, (0.0, s13, 0.0, dm))[0]
    assert abs(p4 - (1 - sin22 / 2)) < sin22 * (np.pi / 4) * 1e-3


@pytest.mark.parametrize("anti", [False, True])
def test_flavour_unitarity(anti):
    rng = np.random.default_rng(7)
    for _ in range(50):
        L = rng.uniform(1.0, 1500.0)
        E = rng.uniform(0.3, 8000.0)
        args = (0.31, 0.022, 0.55, 1.2 * np.pi, 7.4e-5, 2.5e-3, L, E, anti)
        P = np.array([[oracle.prob(a, b, *args) for b in range(3)] for a in range(3)])
        assert np.abs(P.sum(axis=1) - 1).max() < 1e-14
        assert np.abs(P.sum(axis=0) - 1).max() < 1e-14
        assert P.min() > -1e-15 and P.max() < 1 + 1e-15


def test_cpt_and_cp_violation():
    args = dict(s12sq=0.31, s13sq=0.022, s23sq=0.55, dm21=7.4e-5, dm32=2.5e-3, L_km=810.0, E_MeV=2000.0)
    d = 1.2 * np.pi
    for a, b in itertools.product(range(3), range(3)):
        p = oracle.prob(a, b, args["s12sq"], args["s13sq"], args["s23sq"], d, args["dm21"], args["dm32"],
                        args["L_km"], args["E_MeV"], False)
        pbar = oracle.prob(b, a, args["s12sq"], args["s13sq"], args["s23sq"], d, args["dm21"], args["dm32"],
                           args["L_km"], args["E_MeV"], True)
        assert abs(p - pbar) < 1e-14  # CPT: P(a->b) = P(bbar->abar)
    # CP asymmetry magnitude 16 |J| |sin x21 sin x31 sin x32| (textbook vacuum identity)
    U = oracle.pmns(args["s12sq"], args["s13sq"], args["s23sq"], d)
    J = np.imag(U[1, 2] * U[0, 2].conj() * U[0, 1] * U[1, 1].conj())
    p = oracle.prob(1, 0, 0.31, 0.022, 0.55, d, 7.4e-5, 2.5e-3, 810.0, 2000.0, False)
    pb = oracle.prob(1, 0, 0.31, 0.022, 0.55, d, 7.4e-5, 2.5e-3, 810.0, 2000.0, True)
    x = [K_GEV * dm * 810.0 / 2.0 for dm in (7.4e-5, 2.5e-3 + 7.4e-5, 2.5e-3)]
    assert abs(abs(p - pb) - 16 * abs(J) * abs(np.sin(x[0]) * np.sin(x[1]) * np.sin(x[2]))) < 1e-11  # constant given to 11 digits


def test_pee_equals_closed_form_coefficients():
    # Pee = 1 - sum_{i>j} 4|U_ei|^2|U_ej|^2 sin^2 x_ij with the moduli written out
    s12, s13, dm21, dm32 = TRUTH
    E = np.linspace(0.5, 15.0, 1001)
    L = 37.0
    A21 = 4 * s12 * (1 - s12) * (1 - s13) ** 2
    A31 = 4 * (1 - s12) * (1 - s13) * s13
    A32 = 4 * s12 * (1 - s13) * s13
    x = lambda dm: K_GEV * dm * L / (E * 1e-3)
    ref = 1 - A21 * np.sin(x(dm21)) ** 2 - A31 * np.sin(x(dm21 + dm32)) ** 2 - A32 * np.sin(x(dm32)) ** 2
    p = oracle.pee(E, L, TRUTH)
    assert np.abs(p - ref).max() < 2e-9  # constant to 9 digits, phase up to ~200 rad
    p2, _ = oracle.pee_grad(E, L, TRUTH)
    assert np.abs(p2 - p).max() < 1e-14


def test_pee_range_and_period():
    s12, s13, dm21, dm32 = TRUTH
    E = np.linspace(0.5, 15.0, 2001)
    for L in (0.5, 52.5, 60.0, 810.0):
        p = oracle.pee(E, L, TRUTH)
        assert p.min() >= 0 and p.max() <= 1
    # dm2 -> dm2 + pi/(K L/E) shifts every phase by pi: sin^2 unchanged (two-flavour limit)
    E0, L = 3.0, 52.5
    shift = np.pi / (K_GEV * L / (E0 * 1e-3))
    a = oracle.pee([E0], L, (s12, 0.0, dm21, dm32))[0]
    b = oracle.pee([E0], L, (s12, 0.0, dm21 + shift, dm32))[0]
    assert abs(a - b) < 1e-7


# ------------------------------------------------------ Gauss-Legendre ----
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 50, 128, 256])
def test_gl_matches_numpy_leggauss(n):
    x, w = oracle.gl(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.abs(x - xr).max() < 5e-15
    # leggauss's own edge weights carry ~1e-11 relative error at n = 128..256
    assert np.abs(w / wr - 1).max() < 5e-11


def test_gl_weights_mpmath():
    """Nodes and weights at 50 digits: secant iteration on P_n from mpmath's
    hypergeometric Legendre function, w = 2/((1-x^2) P_n'^2)."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    n = 128
    x, w = oracle.gl(n)
    for k in (0, 1, 2, 40, 64, 127):
        xk = mp.findroot(lambda t: mp.legendre(n, t), mp.mpf(x[k]), solver="secant", verify=False)
        assert abs(mp.legendre(n, xk)) < mp.mpf(10) ** -35
        dp = mp.diff(lambda t: mp.legendre(n, t), xk)
        wk = 2 / ((1 - xk ** 2) * dp ** 2)
        assert abs(float(xk) - x[k]) < 2e-16
        assert abs(float(wk) / w[k] - 1) < 1e-12


@pytest.mark.parametrize("n", [33, 50, 262, 524])
def test_gl_exact_to_degree_2n_minus_1(n):
    x, w = oracle.gl(n)
    # monomials x^m, m <= 2n-1, in the Chebyshev basis to stay well conditioned:
    # int_{-1}^{1} T_m = (1 + (-1)^m) / (1 - m^2), m != 1; = 0 for m = 1
    for m in list(range(0, 12)) + [2 * n - 3, 2 * n - 2, 2 * n - 1]:
        Tm = np.cos(m * np.arccos(np.clip(x, -1, 1)))
        exact = 0.0 if m == 1 else (1 + (-1) ** m) / (1 - m * m)
        assert abs(np.dot(w, Tm) - exact) < 1e-13, m
    # and fails at degree 2n (the rule is not exact there)
    T2n = np.cos(2 * n * np.arccos(np.clip(x, -1, 1)))
    assert abs(np.dot(w, T2n) - 2.0 / (1 - 4 * n * n)) > 1e-6


@pytest.mark.parametrize("n", [4096, 16384])
def test_gl_large_orders(n):
    from scipy.special import eval_legendre

    x, w = oracle.gl(n)
    assert abs(w.sum() - 2.0) < 1e-13
    assert np.all(np.diff(x) > 0)
    assert np.abs(x + x[::-1]).max() < 1e-15
    assert np.abs(w - w[::-1]).max() < 1e-15 * n
    # smooth integrands with closed forms (weights across the whole range)
    assert abs(np.dot(w, np.exp(x)) - (math.e - 1 / math.e)) < 1e-13
    assert abs(np.dot(w, np.cos(100 * x)) - np.sin(100.0) / 50) < 1e-13
    # nodes are zeros of P_n (library Legendre): P_n changes sign between midpoints
    mids = 0.5 * (x[1:] + x[:-1])
    sub = slice(0, n - 1, max(1, (n - 1) // 512))
    pm = eval_legendre(n, mids[sub])
    pm1 = eval_legendre(n, mids[sub.start + 1:][::sub.step][: pm.size]) if False else None
    idx = np.arange(0, n - 2, max(1, (n - 2) // 512))
    assert np.all(np.sign(eval_legendre(n, mids[idx])) != np.sign(eval_legendre(n, mids[idx + 1])))


def test_gl_edge_weights_mpmath_large_order():
    """Outermost nodes of the 16384-point rule (1 - x^2 ~ 5e-8).  The node must
    be the true root rounded to double (Newton in 30-digit arithmetic from the
    oracle's node), and the weight formula w = 2/((1-x^2) P_n'(x)^2) evaluated at
    that double node must match 30-digit arithmetic.  (At the true root the
    weight differs by ~4x/(1-x^2) times the node rounding, ~1e-8 relative.)"""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 30
    n = 16384
    x, w = oracle.gl(n)

    def leg(t):
        p0, p1 = mp.mpf(1), t
        for j in range(1, n):
            p0, p1 = p1, ((2 * j + 1) * t * p1 - j * p0) / (j + 1)
        return p1, p0

    def weight(t):
        pn, pn1 = leg(t)
        dp = n * (t * pn - pn1) / (t * t - 1)
        return 2 / ((1 - t * t) * dp * dp)

    for k in (0, 1):
        t = mp.mpf(x[k])
        for _ in range(2):
            pn, pn1 = leg(t)
            t = t - pn / (n * (t * pn - pn1) / (t * t - 1))
        assert abs(float(t - mp.mpf(x[k]))) <= 0.5 * np.spacing(abs(x[k]))
        # each of the n recurrence steps rounds ~4 times and w goes as 1/P_n'^2: bound 32 n eps
        assert abs(float(weight(mp.mpf(x[k]))) / w[k] - 1) < 32 * n * np.spacing(1.0)


# ---------------------------------------------------- binned prediction ----
def test_spectrum_closed_form():
    E = np.array([0.5, 1.8, 4.0, 12.0])
    assert np.allclose(oracle.spectrum(E), np.exp(0.87 - 0.16 * E - 0.091 * E * E), rtol=1e-15, atol=0)
    assert np.allclose(oracle.spectrum(E * 1e3, 1e-3), np.exp(0.87 - 0.16 * E - 0.091 * E * E), rtol=1e-15)


def _erf_integral(a, b, e_scale=1.0):
    # int_a^b exp(0.87 - 0.16 s E - 0.091 s^2 E^2) dE via completing the square
    # (erfc difference: both arguments are positive, so no cancellation)
    from scipy.special import erfc

    c2, c1, c0 = 0.091 * e_scale ** 2, 0.16 * e_scale, 0.87
    s = math.sqrt(c2)
    pref = math.exp(c0 + c1 * c1 / (4 * c2)) * math.sqrt(math.pi) / (2 * s)
    u = lambda E: s * (E + c1 / (2 * c2))
    assert u(a) > 0
    return pref * (erfc(u(a)) - erfc(u(b)))


@pytest.mark.parametrize("e_scale,edges", [(1.0, np.linspace(1.8, 12.0, 21)), (1e-3, np.linspace(500., 5000., 11))])
def test_binned_without_oscillation_is_spectrum_integral(e_scale, edges):
    mu = oracle.binned(edges, 50, [52.5, 3.0], (0.0, 0.0, 7.53e-5, 2.44e-3), e_scale)
    ref = np.array([_erf_integral(a, b, e_scale) for a, b in zip(edges[:-1], edges[1:])])
    assert np.abs(mu / ref[None, :] - 1).max() < 1e-13


def test_binned_brute_force_mpmath_tiny():
    """2 bins x 3 nodes x 2 baselines at 50 digits, 3-point rule in closed form
    (nodes 0, +-sqrt(3/5); weights 8/9, 5/9)."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    edges = [1.8, 3.1, 7.4]
    Ls = [52.5, 1.7]
    th = [0.307, 0.0218, 7.53e-5, 2.44e-3]
    xs = [-mp.sqrt(mp.mpf(3) / 5), mp.mpf(0), mp.sqrt(mp.mpf(3) / 5)]
    ws = [mp.mpf(5) / 9, mp.mpf(8) / 9, mp.mpf(5) / 9]
    hbarc = mp.mpf("197.3269804e-9")  # eV m

    def P(s12, s13, dm21, dm32, L, E):
        ue = [(1 - s12) * (1 - s13), s12 * (1 - s13), s13]
        m2 = [0, dm21, dm21 + dm32]
        p = mp.mpf(1)
        for i in range(3):
            for j in range(i):
                x = (m2[i] - m2[j]) * (L * 1000) / (4 * hbarc * E * 10 ** 6)
                p -= 4 * ue[i] * ue[j] * mp.sin(x) ** 2
        return p

    def mu_mp(thv, r, i):
        a, b = mp.mpf(edges[i]), mp.mpf(edges[i + 1])
        h, m = (b - a) / 2, (a + b) / 2
        s = 0
        for xk, wk in zip(xs, ws):
            E = m + h * xk
            s += h * wk * mp.exp(mp.mpf("0.87") - mp.mpf("0.16") * E - mp.mpf("0.091") * E * E) * \
                P(*thv, mp.mpf(Ls[r]), E)
        return s

    thm = [mp.mpf(t) for t in th]
    mu, dmu = oracle.binned(np.array(edges), 3, Ls, th, grad=True)
    for r in range(2):
        for i in range(2):
            ref = mu_mp(thm, r, i)
            assert abs(mu[r, i] / float(ref) - 1) < 1e-14
            for q in range(4):
                f = lambda t, q=q: mu_mp([t if k == q else thm[k] for k in range(4)], r, i)
                dref = mp.diff(f, thm[q])
                assert abs(dmu[r, i, q] - float(dref)) <= 1e-12 * abs(float(dref)) + 1e-30, (r, i, q)


# ---------------------------------------------------------------- chi^2 ----
def test_chi2_closed_cases():
    om = np.array([0.25, 0.75])
    mu_rb = np.array([[100.0, 50.0, 7.0], [80.0, 40.0, 9.0]])
    dmu = np.random.default_rng(0).normal(size=(2, 3, 4))
    M = om @ mu_rb
    N = 3.0
    for kind in (0, 1):
        r = oracle.chi2(om, mu_rb, N, N * M, kind, dmu_rb=dmu)
        assert abs(r["chi2"]) < 1e-12
        assert np.abs(r["grad"]).max() < 1e-12
        assert np.allclose(r["mu"], N * M, rtol=1e-15)
    # one bin, textbook values
    one = np.array([[5.0]])
    assert abs(oracle.chi2([1.0], one, 1.0, [7.0], 0)["chi2"] - 0.8) < 1e-15
    assert abs(oracle.chi2([1.0], one, 1.0, [7.0], 1)["chi2"] - 2 * (5 - 7 + 7 * math.log(7 / 5))) < 1e-14
    assert abs(oracle.chi2([1.0], one, 1.0, [0.0], 1)["chi2"] - 10.0) < 1e-15
    # nuisance: mu -> mu (1 + eta), penalty eta^2 / sigma^2
    r = oracle.chi2([1.0], one, 1.0, [7.0], 0, eta=[0.01], sigma=0.02)
    m = 5.0 * 1.01
    assert abs(r["chi2"] - ((7 - m) ** 2 / m + 0.25)) < 1e-14
    # transposed baselines change the answer (the combination is omega-weighted)
    a = oracle.chi2(om, mu_rb, N, [300.0, 120.0, 20.0], 0)["chi2"]
    b = oracle.chi2(om[::-1].copy(), mu_rb, N, [300.0, 120.0, 20.0], 0)["chi2"]
    assert abs(a - b) > 1e-3


@pytest.mark.parametrize("kind", [0, 1])
def test_gradient_matches_central_differences(kind):
    edges = np.linspace(0.5, 15.0, 41)
    L = np.array([52.5, 3.0, 17.0])
    n = 24
    theta = np.array(TRUTH) * np.array([1.03, 0.96, 1.02, 0.98])
    N = oracle.norm_for_total(edges, n, L, TRUTH)
    data = wl.poisson_data(N * (oracle.baseline_weights(L) @ oracle.binned(edges, n, L, TRUTH)), 3)
    eta = np.random.default_rng(2).normal(0, 0.02, 40)
    r = oracle.chain(edges, n, L, theta, N, data, kind, eta=eta, sigma=0.02)
    f = lambda t: oracle.chain(edges, n, L, t, N, data, kind, eta=eta, sigma=0.02, grad=False)["chi2"]
    g_fd = oracle.fd_grad(f, theta)
    assert np.linalg.norm(r["grad"][:4] - g_fd) <= 1e-5 * np.linalg.norm(g_fd)
    # nuisance gradient
    fe = lambda e: oracle.chain(edges, n, L, theta, N, data, kind, eta=e, sigma=0.02, grad=False)["chi2"]
    idx = [0, 7, 39]
    ge = []
    for i in idx:
        h = 1e-6
        ep, em = eta.copy(), eta.copy()
        ep[i] += h
        em[i] -= h
        ge.append((fe(ep) - fe(em)) / (2 * h))
    assert np.allclose(r["grad"][4 + np.array(idx)], ge, rtol=1e-6, atol=1e-6)


def test_lm_fit_recovers_truth_on_asimov_data():
    edges = np.linspace(0.5, 15.0, 101)
    L = np.array([52.5, 30.0, 8.0])
    n = 16
    N = oracle.norm_for_total(edges, n, L, TRUTH)
    data = N * (oracle.baseline_weights(L) @ oracle.binned(edges, n, L, TRUTH))
    start = np.array(TRUTH) * np.array([1.04, 0.95, 0.97, 1.03])
    ev = lambda t: oracle.chain(edges, n, L, t, N, data, 1)
    th, c2, hist = oracle.fit_lm(ev, start, iters=20)
    assert hist.size == 20
    assert c2 < 1e-8
    assert np.abs(th / np.array(TRUTH) - 1).max() < 1e-4


# ------------------------------------------------- any channel, gradient ----
TH6 = (0.307, 0.0218, 0.545, 1.2 * np.pi, 7.53e-5, 2.44e-3)


def fd6(f, th, rel_h=1e-6):
    g = np.empty(6)
    for q in range(6):
        h = rel_h * abs(th[q])
        tp, tm = list(th), list(th)
        tp[q] += h
        tm[q] -= h
        g[q] = (f(tp) - f(tm)) / (2 * h)
    return g


@pytest.mark.parametrize("a,b,anti,L,E", [("mu", "e", False, 810.0, 2000.0), ("mu", "mu", True, 810.0, 1500.0),
                                          ("e", "tau", False, 295.0, 600.0), ("tau", "mu", True, 1300.0, 3100.0),
                                          ("e", "e", True, 52.5, 4.0)])
def test_general_gradient_matches_central_differences(a, b, anti, L, E):
    # the analytic derivative of the Sec. 4.1 formula against differences of the
    # formula itself, in all six parameters
    P, dP = oracle.prob_grad(a, b, TH6, L, E, anti)
    fa, fb = oracle.FLAVOUR[a], oracle.FLAVOUR[b]
    assert P == oracle.prob(fa, fb, *TH6, L, E, anti)
    g = fd6(lambda t: oracle.prob(fa, fb, *t, L, E, anti), TH6)
    assert np.linalg.norm(dP - g) <= 1e-6 * np.linalg.norm(g)


def test_general_gradient_unitarity_and_cpt():
    # sum over final (or initial) flavours of P is 1 for any parameters, so the
    # derivatives sum to zero; CPT maps nu_bar a->b to nu b->a, derivatives too
    fl = ["e", "mu", "tau"]
    for E in (700.0, 2500.0):
        for a in fl:
            assert np.abs(sum(oracle.prob_grad(a, b, TH6, 810.0, E)[1] for b in fl)).max() < 1e-12 * 1e3
            assert np.abs(sum(oracle.prob_grad(b, a, TH6, 810.0, E, True)[1] for b in fl)).max() < 1e-12 * 1e3
            for b in fl:
                P1, d1 = oracle.prob_grad(a, b, TH6, 810.0, E, True)
                P2, d2 = oracle.prob_grad(b, a, TH6, 810.0, E, False)
                assert abs(P1 - P2) < 1e-14 and np.abs(d1 - d2).max() < 1e-10


def test_general_ee_gradient_is_the_closed_form():
    # for nue_bar survival the derivative in (s12^2, s13^2, dm21, dm32) equals
    # the closed-form moduli product rule, and theta23 and delta do not enter
    E = np.linspace(1.8, 12.0, 7)
    osc = (TH6[0], TH6[1], TH6[4], TH6[5])
    P, dP = oracle.pee_grad(E, 52.5, osc)
    for k, e in enumerate(E):
        p, d = oracle.prob_grad("e", "e", TH6, 52.5, e, True)
        assert abs(p - P[k]) < 1e-14
        assert np.abs(d[[0, 1, 4, 5]] - dP[k]).max() <= 1e-12 * (1 + np.abs(dP[k]).max())
        assert abs(d[2]) < 1e-13 and abs(d[3]) < 1e-13


def test_general_chain_reduces_to_the_ee_chain_and_matches_differences():
    edges = np.linspace(1.8, 9.0, 13)
    L = np.array([52.5, 20.0])
    n = 12
    osc = (TH6[0], TH6[1], TH6[4], TH6[5])
    N = oracle.norm_for_total(edges, n, L, osc)
    data = wl.poisson_data(N * (oracle.baseline_weights(L) @ oracle.binned(edges, n, L, osc)), 5)
    eta = np.random.default_rng(3).normal(0, 0.02, 12)
    g = oracle.chain_general(edges, n, L, TH6, N, data, "e", "e", True, 1, eta, 0.02)
    r = oracle.chain(edges, n, L, osc, N, data, 1, eta=eta, sigma=0.02)
    assert abs(g["chi2"] - r["chi2"]) <= 1e-12 * r["chi2"]
    assert np.abs(g["mu"] / r["mu"] - 1).max() < 1e-13
    assert np.linalg.norm(g["grad"][[0, 1, 4, 5]] - r["grad"][:4]) <= 1e-10 * np.linalg.norm(r["grad"][:4])
    assert np.abs(g["grad"][6:] - r["grad"][4:]).max() <= 1e-10 * np.abs(r["grad"][4:]).max()
    # numu -> nue at 810 km: the chi^2 gradient against central differences
    e2 = np.linspace(500.0, 5000.0, 11)
    N2 = 1e4
    d2 = wl.poisson_data(N2 * oracle.binned_general(e2, 10, [810.0], TH6, "mu", "e", e_scale=1e-3)[0][0], 6)
    th = (0.31, 0.0225, 0.52, 1.4 * np.pi, 7.4e-5, 2.5e-3)
    f = lambda t: oracle.chain_general(e2, 10, [810.0], t, N2, d2, "mu", "e", kind=1, e_scale=1e-3)["chi2"]
    gr = oracle.chain_general(e2, 10, [810.0], th, N2, d2, "mu", "e", kind=1, e_scale=1e-3)["grad"][:6]
    assert np.linalg.norm(gr - fd6(f, th)) <= 1e-5 * np.linalg.norm(gr)


def test_general_chain_jacobian_matches_central_differences():
    # J[i][q] = d mu_i / d p_q of the any-channel chain (the fits' Jacobian)
    # against central differences of mu itself, and the gradient identity
    # d chi2 / d p = sum_i (d chi2 / d mu_i) J_i for Poisson and Pearson
    edges = np.linspace(600.0, 4000.0, 9)
    th = np.array(TH6) * np.array([1.02, 0.97, 1.01, 0.95, 1.03, 0.99])
    data = np.array([31.0, 57.0, 60.0, 44.0, 38.0, 20.0, 14.0, 9.0])
    eta = np.random.default_rng(3).normal(0.0, 0.02, 8)
    for kind in (0, 1):
        r = oracle.chain_general(edges, 12, [810.0], th, 2e3, data, "mu", "e", False, kind, eta, 0.02, e_scale=1e-3)
        for q in range(6):
            h = 1e-6 * abs(th[q])
            tp, tm = th.copy(), th.copy()
            tp[q] += h
            tm[q] -= h
            mp = oracle.chain_general(edges, 12, [810.0], tp, 2e3, data, "mu", "e", False, kind, eta, 0.02,
                                      e_scale=1e-3)["mu"]
            mm = oracle.chain_general(edges, 12, [810.0], tm, 2e3, data, "mu", "e", False, kind, eta, 0.02,
                                      e_scale=1e-3)["mu"]
            fd = (mp - mm) / (2 * h)
            assert np.allclose(r["J"][:, q], fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max()), q
        mu = r["mu"]
        g_mu = (1 - data ** 2 / mu ** 2) if kind == 0 else 2 * (1 - data / mu)
        assert np.allclose(g_mu @ r["J"], r["grad"][:6], rtol=1e-12, atol=0.0)
