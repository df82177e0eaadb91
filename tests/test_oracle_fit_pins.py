"""Pins of the oracle's Levenberg-Marquardt fitter (``oracle.fit_lm``) on
designed problems whose iterates are known in closed form, and planted
mistakes in copies of the fitter, each caught by a pin.

The paper has no fitter; the batched fits use Levenberg-Marquardt-damped
Gauss-Newton as the textbook states it: one evaluation per iteration, the
trial is accepted when it lowers chi^2 strictly (then lambda / 10) and
rejected otherwise (lambda x 10), H = sum_i (2 / mu_i) J_i J_i^T, the next
trial is best + delta with (H + lambda diag H) delta = -g, clamped into a box.

The designed problems are linear least squares with a diagonal Jacobian,
chi^2(theta) = sum_q (d_q - a_q theta_q)^2 / v_q.  With mu = v the matrix H is
the exact Hessian 2 diag(a^2 / v), and one damped step shrinks every residual
r_q = d_q - a_q theta_q by the same factor, derived by hand:

    delta_q = -g_q / (H_qq (1 + lambda)) = r_q / (a_q (1 + lambda))
    r_q'    = r_q lambda / (1 + lambda).

A problem whose evaluation reports the Jacobian divided by c (a model with a
wrong slope estimate: H is c^2 too small, the step c^2 too long) overshoots:
r' = r (1 + lambda - c^2) / (1 + lambda), so trials are rejected until lambda
has grown past c^2 - 2, which fixes the accept / reject pattern.
"""
import inspect
import textwrap

import numpy as np
import pytest

import oracle

A_Q = np.array([1.0, 2.0, 0.5, 4.0])
V_Q = np.array([1.0, 4.0, 0.25, 2.0])


def linear_problem(d, a=A_Q, v=V_Q, c=1.0):
    """evaluate(theta) of the diagonal linear problem; the reported Jacobian is a / c."""
    d, a, v = (np.asarray(x, dtype=np.float64) for x in (d, a, v))

    def evaluate(theta):
        r = d - a * theta
        return {"chi2": float(np.sum(r * r / v)), "grad": -2.0 * a * r / v, "J": np.diag(a / c), "mu": v.copy()}

    return evaluate


NOBOX = dict(lo=(-np.inf,) * 4, hi=(np.inf,) * 4)


def test_fit_lm_accepted_steps_follow_the_lambda_schedule():
    # every trial improves: lambda goes lam0/10, lam0/100, ... and each step
    # multiplies all residuals by lambda / (1 + lambda)
    d = np.array([0.5, 0.3, 0.7, 2.0])
    th0 = np.array([0.1, 0.05, 0.2, 0.1])
    ev = linear_problem(d)
    th, c2, hist = oracle.fit_lm(ev, th0, iters=4, lam0=1.0, **NOBOX)
    r = d - A_Q * th0
    chi = [np.sum(r * r / V_Q)]
    for lam in (0.1, 0.01, 0.001):
        r = r * lam / (1.0 + lam)
        chi.append(np.sum(r * r / V_Q))
    assert hist.size == 4
    assert np.allclose(hist, chi, rtol=1e-9, atol=0.0)
    assert c2 == hist[-1]
    # the best point is the last trial: theta = (d - r) / a
    assert np.allclose(th, (d - r) / A_Q, rtol=1e-12, atol=1e-15)


def test_fit_lm_rejections_raise_lambda_and_ties_are_rejected():
    # reported Jacobian a / 2 (c = 2): r' = r (lambda - 3) / (1 + lambda).  From
    # lam0 = 1e-3: eval 1 accepted (lambda -> 1e-4); trials at 1e-4, 1e-3,
    # 1e-2, 0.1 overshoot (|r'| > |r|) and are rejected; at lambda = 1 the
    # trial lands on -r exactly (dyadic numbers), an equal chi^2, rejected
    # (strict improvement only); at lambda = 10 the residual shrinks by 7/11
    d = np.array([0.5, 0.25, 0.75, 0.25])
    th0 = np.array([0.25, 0.125, 0.5, 0.375])
    a = np.ones(4)
    v = np.ones(4)
    ev = linear_problem(d, a, v, c=2.0)
    th, c2, hist = oracle.fit_lm(ev, th0, iters=7, lam0=1e-3, **NOBOX)
    chi0 = np.sum((d - th0) ** 2)  # 0.0625 + 0.015625 + 0.0625 + 0.015625
    assert chi0 == 0.15625
    f = lambda lam: (lam - 3.0) / (1.0 + lam)
    expect = [chi0] + [chi0 * f(lam) ** 2 for lam in (1e-4, 1e-3, 1e-2, 0.1)] + [chi0, chi0 * (7.0 / 11.0) ** 2]
    assert np.allclose(hist, expect, rtol=1e-12, atol=0.0)
    assert hist[5] == chi0  # the tie, exactly
    assert c2 == hist[6]
    assert np.allclose(th, th0 + (d - th0) * 4.0 / 11.0, rtol=1e-14, atol=0.0)


def test_fit_lm_rejection_pattern_over_many_iterations():
    # c^2 = 3: r' = r (lambda - 2) / (1 + lambda); the pattern is
    # A R R R R A R A R A ... (lambda 1e-3 -> 1e-4 after eval 1, rejected up to
    # lambda = 1, then alternating between lambda = 0.1 (rejected, |r'| = 1.73 |r|)
    # and lambda = 1 (accepted, r' = -r / 2))
    d = np.array([0.5, 0.3, 0.7, 2.0])
    th0 = np.array([0.1, 0.05, 0.2, 0.1])
    ev = linear_problem(d, c=np.sqrt(3.0))
    th, c2, hist = oracle.fit_lm(ev, th0, iters=12, lam0=1e-3, **NOBOX)
    r0 = d - A_Q * th0
    chi0 = np.sum(r0 * r0 / V_Q)
    f = lambda lam: (lam - 2.0) / (1.0 + lam)
    expect = [chi0] + [chi0 * f(lam) ** 2 for lam in (1e-4, 1e-3, 1e-2, 0.1)]
    best = chi0
    for k in range(7):
        lam = 1.0 if k % 2 == 0 else 0.1
        trial = best * f(lam) ** 2
        expect.append(trial)
        if trial < best:
            best = trial
    assert np.allclose(hist, expect, rtol=1e-10, atol=0.0)
    accepted = [hist[0] < np.inf] + [hist[k] < min(hist[:k]) for k in range(1, 12)]
    assert accepted == [True, False, False, False, False, True, False, True, False, True, False, True]
    assert c2 == min(hist)


def test_fit_lm_clamps_trials_into_the_box():
    # the first parameter's least-squares value lies above the box (1.5 > 1 -
    # 1e-6): every trial is clamped to the bound, which then stays the best
    # value; the others follow the unconstrained schedule (diagonal problem)
    d = np.array([1.5, 0.3, 0.7, 2.0])
    th0 = np.array([0.9, 0.05, 0.2, 0.1])
    ev = linear_problem(d)
    th, c2, hist = oracle.fit_lm(ev, th0, iters=4, lam0=1.0)
    assert th[0] == 1.0 - 1e-6
    r = d - A_Q * th0
    tail = [np.sum(r[1:] ** 2 / V_Q[1:])]
    for lam in (0.1, 0.01, 0.001):
        r = r * lam / (1.0 + lam)
        tail.append(np.sum(r[1:] ** 2 / V_Q[1:]))
    r_clamped = d[0] - A_Q[0] * (1.0 - 1e-6)
    expect = [hist[0]] + [r_clamped ** 2 / V_Q[0] + t for t in tail[1:]]
    assert hist[0] == np.sum((d - A_Q * th0) ** 2 / V_Q)
    assert np.allclose(hist, expect, rtol=1e-9, atol=0.0)
    assert np.allclose(th[1:], (d[1:] - r[1:]) / A_Q[1:], rtol=1e-12, atol=1e-15)
    # and from below: a target under the lower bound of a mass splitting
    d2 = np.array([0.5, 0.3, -0.7, 2.0])
    th, _, _ = oracle.fit_lm(linear_problem(d2), th0, iters=3, lam0=1.0)
    assert th[2] == 1e-7


FIT_PINS = [test_fit_lm_accepted_steps_follow_the_lambda_schedule,
            test_fit_lm_rejections_raise_lambda_and_ties_are_rejected,
            test_fit_lm_rejection_pattern_over_many_iterations,
            test_fit_lm_clamps_trials_into_the_box]

# Planted mistakes in the fitter (old text -> new text, first occurrence).
FIT_MUTATIONS = {
    "H_without_factor_2": ('(2.0 / r["mu"])', '(1.0 / r["mu"])'),
    "lambda_down_on_reject": ("lam = lam * 10.0", "lam = lam / 10.0"),
    "lambda_up_on_accept": ("lam = lam / 10.0", "lam = lam * 10.0"),
    "accept_on_tie": ('if r["chi2"] < best_chi2:', 'if r["chi2"] <= best_chi2:'),
    "step_from_last_trial": ("best_theta + delta", "trial + delta"),
    "no_clamp": ("np.minimum(np.maximum(best_theta + delta, lo), hi)", "best_theta + delta"),
    "clamp_the_step": ("np.minimum(np.maximum(best_theta + delta, lo), hi)",
                       "best_theta + np.minimum(np.maximum(delta, lo), hi)"),
    "damping_identity": ("lam * np.diag(np.diag(H))", "lam * np.eye(4)"),
    "gradient_sign": ("np.linalg.solve(A, -g)", "np.linalg.solve(A, g)"),
    "hessian_not_weighted": ('(Jm.T * (2.0 / r["mu"])) @ Jm', "2.0 * Jm.T @ Jm"),
    "gradient_first_four_only": ('r["grad"][:npar]', 'r["grad"][:4]'),
}


@pytest.mark.parametrize("mut", sorted(FIT_MUTATIONS))
def test_fit_pins_catch_planted_mistake(mut, monkeypatch):
    old, new = FIT_MUTATIONS[mut]
    src = textwrap.dedent(inspect.getsource(oracle.fit_lm))
    assert src.count(old) >= 1, "mutation anchor not found: %s" % mut
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new, 1), "fit_lm_mutant", "exec"), ns)
    monkeypatch.setattr(oracle, "fit_lm", ns["fit_lm"])
    caught = []
    for pin in FIT_PINS:
        try:
            with np.errstate(all="ignore"):
                pin()
        except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError):
            caught.append(pin.__name__)
    assert caught, "no fitter pin failed for mutation %s" % mut


def test_fit_lm_six_parameters_box_and_free_phase():
    # six parameters in the any-channel order (s2_12, s2_13, s2_23, delta_cp,
    # dm2_21, dm2_32), diagonal linear problem: the default box clamps s2_23
    # (target 1.4 > 1 - 1e-6) and leaves delta_cp free (target -2.5); the
    # others follow the lambda schedule of the four-parameter pin
    a = np.array([1.0, 2.0, 1.0, 1.0, 0.5, 4.0])
    v = np.array([1.0, 4.0, 1.0, 2.0, 0.25, 2.0])
    d = np.array([0.5, 0.3, 1.4, -2.5, 0.7, 2.0])
    th0 = np.array([0.1, 0.05, 0.5, 1.0, 0.2, 0.1])
    th, c2, hist = oracle.fit_lm(linear_problem(d, a, v), th0, iters=4, lam0=1.0)
    assert th[2] == 1.0 - 1e-6
    free = [0, 1, 3, 4, 5]
    r = d - a * th0
    for lam in (0.1, 0.01, 0.001):
        r = r * lam / (1.0 + lam)
    assert np.allclose(th[free], ((d - r) / a)[free], rtol=1e-12, atol=1e-15)
    assert th[3] < 0.0  # delta_cp crossed zero
    r2 = (d[2] - a[2] * (1.0 - 1e-6)) ** 2 / v[2]
    assert np.isclose(c2, r2 + np.sum(r[free] ** 2 / v[free]), rtol=1e-9, atol=0.0)


FIT_PINS.append(test_fit_lm_six_parameters_box_and_free_phase)


def test_fit_sigma_is_the_inverse_fisher_diagonal():
    # the parity tests' statistical errors: J = [[1, 0], [0, 2], [1, 1]] and
    # mu = 2 give H = J^T J = [[2, 1], [1, 5]], H^-1 = [[5, -1], [-1, 2]] / 9
    import refs
    r = {"J": np.array([[1.0, 0.0], [0.0, 2.0], [1.0, 1.0]]), "mu": np.full(3, 2.0)}
    assert np.allclose(refs.fit_sigma(r), [np.sqrt(5.0 / 9.0), np.sqrt(2.0 / 9.0)], rtol=1e-14, atol=0.0)
    # halving every mu doubles H: the errors shrink by sqrt(2)
    r["mu"] = np.full(3, 1.0)
    assert np.allclose(refs.fit_sigma(r), [np.sqrt(5.0 / 18.0), np.sqrt(1.0 / 9.0)], rtol=1e-14, atol=0.0)
