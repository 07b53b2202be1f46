"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each test checks a closed form,
an exhaustive brute force, a printed value, an inequality the paper proves for
every iterate, or an algebraic identity derived independently.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2605_29291_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PHI = (1.0 + math.sqrt(5.0)) / 2.0


# --------------------------------------------------------------------------
# helpers: tiny random problems and an exhaustive box-QP minimiser
# --------------------------------------------------------------------------

def tiny_problem(n=4, m=2, seed=0, ridge=0.1, box=3.0):
    rng = np.random.default_rng(seed)
    Q = np.empty((m + 1, n, n))
    for i in range(m + 1):
        A = rng.standard_normal((n, n))
        Q[i] = A.T @ A / n
    Q[0] += ridge * np.eye(n)
    Q = Q.astype(np.float32).astype(np.float64)
    Q = 0.5 * (Q + np.swapaxes(Q, 1, 2))
    c = rng.standard_normal((m + 1, n))
    d = -rng.uniform(0.1, 1.0, size=m)
    lb, ub = -box * np.ones(n), box * np.ones(n)
    return O.Problem(Q, c, d, lb, ub)


def box_qp_bruteforce(H, lin, lb, ub):
    """min 0.5 x'Hx + lin'x over lb <= x <= ub for PD H, by trying every
    free / lower / upper pattern (3^n) and keeping the best feasible point."""
    n = len(lin)
    best, best_x = math.inf, None
    for pat in itertools.product((0, 1, 2), repeat=n):
        x = np.zeros(n)
        fixed = np.array([p != 0 for p in pat])
        for j, pj in enumerate(pat):
            if pj == 1:
                x[j] = lb[j]
            elif pj == 2:
                x[j] = ub[j]
        F = ~fixed
        if F.any():
            rhs = -(lin[F] + H[np.ix_(F, fixed)] @ x[fixed])
            x[F] = np.linalg.solve(H[np.ix_(F, F)], rhs)
        if np.all(x >= lb - 1e-12) and np.all(x <= ub + 1e-12):
            val = 0.5 * x @ H @ x + lin @ x
            if val < best:
                best, best_x = val, x
    return best_x, best


def lagrangian_pieces(prob, lam):
    H = prob.Q[0] + np.tensordot(lam, prob.Q[1:], axes=1)
    lin = prob.c[0] + lam @ prob.c[1:]
    const = lam @ prob.r
    return H, lin, const


def dual_value(prob, lam):
    """q(lam) = min_{x in X} L(x, lam) computed by exhaustive enumeration."""
    H, lin, const = lagrangian_pieces(prob, lam)
    _, v = box_qp_bruteforce(H, lin, prob.lb, prob.ub)
    return v + const


# --------------------------------------------------------------------------
# printed values
# --------------------------------------------------------------------------

def test_default_params_match_paper():
    gp = json.load(open(os.path.join(GOLDEN, "paper_params.json")))
    yx, xy = O.default_params("yx"), O.default_params("xy")
    assert yx.eta == gp["eta"]["value"] and xy.eta == gp["eta"]["value"]
    assert (yx.c_alpha, yx.delta, yx.c_beta) == (gp["yx"]["c_alpha"], gp["yx"]["delta"], 0.0)
    assert (xy.c_alpha, xy.c_beta, xy.delta) == (gp["xy"]["c_alpha"], gp["xy"]["c_beta"], gp["xy"]["delta"])
    assert yx.xi == gp["xi"]["value"] and yx.q == gp["q"]["value"]
    assert yx.gap_first == gp["gap_first"]["yx"] and xy.gap_first == gp["gap_first"]["xy"]


def test_nonmonotone_average_bound_printed_value():
    gp = json.load(open(os.path.join(GOLDEN, "paper_params.json")))
    assert abs(gp["phi"]["value"] - PHI) < 1e-15
    # (1 + log_{1/eta} phi) is "approximately 2" at eta = 0.6
    val = 1.0 + math.log(PHI) / math.log(1.0 / 0.6)
    assert abs(val - gp["nonmono_evals_per_iter_eta_0_6"]["value"]) < 0.1


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["yx", "xy"])
def test_first_iterate_closed_form(variant):
    """From (x, y) = (0, 0) with fixed step tau: x^1 = Pi_X(-tau q_0); yx gives
    y^1 = max(0, sigma r) = 0 (r < 0); xy gives y^1 = max(0, sigma g(x^1))."""
    prob = tiny_problem(n=5, m=3, seed=3)
    tau = 0.37
    p = O.default_params(variant, backtracking=False, tau_bar=tau, restart="none")
    st = O.start_routine(prob, np.zeros(5), np.zeros(3), p)
    O.apdb_iteration(prob, st, p)
    x1 = np.clip(-tau * prob.c[0], prob.lb, prob.ub)
    np.testing.assert_allclose(st.x, x1, rtol=0, atol=1e-15)
    if variant == "yx":
        np.testing.assert_array_equal(st.lam, np.zeros(3))
    else:
        g1 = np.array([0.5 * np.einsum("j,jk,k->", x1, prob.Q[i], x1) + prob.c[i] @ x1 + prob.r[i - 1]
                       for i in (1, 2, 3)])
        np.testing.assert_allclose(st.lam, np.maximum(0.0, p.gamma0 * tau * g1), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("variant", ["yx", "xy"])
def test_ball_constraint_closed_form(variant):
    """min c'x s.t. ||x||^2 <= rho^2 has x* = -rho c/||c||, lambda* = ||c||/(2 rho)."""
    rng = np.random.default_rng(11)
    cvec = rng.standard_normal(6).astype(np.float32)
    rho = 2.0
    prob = O.Problem.from_data(W.ball_qcqp(cvec, rho))
    # Q_0 = 0 makes this an LP over a ball: the yx variant (dual step first,
    # gamma_0 = 1) converges slowly here, so it is held to a looser tolerance.
    tol, atol = (1e-10, 1e-8) if variant == "xy" else (1e-7, 1e-5)
    p = O.default_params(variant, tol=tol, max_iter=20000, restart="fixed", restart_period=200)
    r = O.rapdb(prob, p=p)
    assert r.status == 0
    c64 = cvec.astype(np.float64)
    xs = -rho * c64 / np.linalg.norm(c64)
    ls = np.linalg.norm(c64) / (2 * rho)
    np.testing.assert_allclose(r.x, xs, atol=atol)
    np.testing.assert_allclose(r.lam, [ls], rtol=atol)


@pytest.mark.parametrize("m", [0, 1])
def test_interior_pd_qp_closed_form(m):
    """Q_0 PD with an interior minimiser and no active constraint:
    x* = -Q_0^{-1} q_0, lambda* = 0."""
    rng = np.random.default_rng(5)
    n = 8
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q0 = (U * rng.uniform(1.0, 5.0, n)) @ U.T
    Q = np.zeros((m + 1, n, n))
    Q[0] = Q0
    c = np.zeros((m + 1, n))
    c[0] = rng.standard_normal(n)
    d = np.zeros(m)
    if m:
        Q[1] = np.eye(n)
        d[:] = -50.0                      # ||x||^2/2 <= 50: slack at x*
    prob = O.Problem(Q, c, d, -10 * np.ones(n), 10 * np.ones(n))
    r = O.rapdb(prob, p=O.default_params("yx", tol=1e-11, restart="fixed"))
    xs = -np.linalg.solve(Q0, c[0])
    assert np.all(np.abs(xs) < 10)
    np.testing.assert_allclose(r.x, xs, atol=1e-9)
    if m:
        assert r.lam[0] < 1e-9


# --------------------------------------------------------------------------
# brute-force certificates
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("variant", ["yx", "xy"])
def test_weak_duality_certificate_bruteforce(seed, variant):
    """For any lam >= 0, q(lam) <= f* <= f(x) for feasible x.  The oracle's
    final pair closes that gap, with q computed by 3^n enumeration."""
    prob = tiny_problem(n=4, m=2, seed=seed)
    # The yx test function, evaluated literally from Phi differences, loses
    # its digits to cancellation once ||d||^2/tau nears eps*|Phi|; the literal
    # oracle therefore stalls near rel KKT 1e-8 in that variant.
    tol, slack = (1e-10, 1e-8) if variant == "xy" else (5e-8, 1e-7)
    r = O.rapdb(prob, p=O.default_params(variant, tol=tol, max_iter=50000))
    assert r.status == 0
    f = prob.f(r.x)
    g = prob.g(r.x)
    assert np.all(g <= slack)
    assert np.all(r.x >= prob.lb) and np.all(r.x <= prob.ub) and np.all(r.lam >= 0)
    qv = dual_value(prob, r.lam)
    assert qv <= f + slack
    assert f - qv <= 10 * slack * (1 + abs(f))


def test_gap_subproblem_matches_bruteforce():
    rng = np.random.default_rng(7)
    for seed in range(5):
        prob = tiny_problem(n=5, m=2, seed=seed, ridge=0.0)
        x = rng.uniform(-3, 3, 5)
        lam = rng.uniform(0, 2, 2)
        xi = 0.04
        xs = O.gap_x_subproblem(prob, x, lam, xi)
        H, lin, _ = lagrangian_pieces(prob, lam)
        H = H + 2 * xi * np.eye(5)
        lin = lin - 2 * xi * x
        xb, _ = box_qp_bruteforce(H, lin, prob.lb, prob.ub)
        np.testing.assert_allclose(xs, xb, atol=1e-9)


def test_smoothed_gap_zero_at_solution_and_nonnegative():
    prob = tiny_problem(n=4, m=2, seed=1)
    r = O.rapdb(prob, p=O.default_params("yx", tol=1e-11, max_iter=50000))
    assert abs(O.smoothed_gap(prob, r.x, r.lam, 0.04)) < 1e-8
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = rng.uniform(prob.lb, prob.ub)
        lam = rng.uniform(0, 3, prob.m)
        assert O.smoothed_gap(prob, x, lam, 0.04) >= -1e-10


# --------------------------------------------------------------------------
# KKT residual against hand-derived values
# --------------------------------------------------------------------------

def test_kkt_residual_ball_values():
    rng = np.random.default_rng(2)
    cvec = rng.standard_normal(5)
    rho = 1.5
    prob = O.Problem.from_data(W.ball_qcqp(cvec.astype(np.float32), rho))
    c64 = prob.c[0]
    xs = -rho * c64 / np.linalg.norm(c64)
    ls = np.linalg.norm(c64) / (2 * rho)
    rel, rs, rf = O.kkt_residual(prob, xs, [ls])
    assert rel < 1e-12
    eps = 1e-3
    rel, rs, rf = O.kkt_residual(prob, xs, [ls + eps])
    assert abs(rs - 2 * eps * rho) < 1e-12 and rf < 1e-12
    den = 1 + max(np.linalg.norm(c64), 2 * (ls + eps) * rho)
    assert abs(rel - 2 * eps * rho / den) < 1e-12
    # infeasible point with lambda = 0: r_feas = g(x) = ||x||^2 - rho^2
    x2 = 1.1 * xs
    rel, rs, rf = O.kkt_residual(prob, x2, [0.0])
    assert abs(rf - (np.sum(x2 ** 2) - rho ** 2)) < 1e-12
    assert abs(rs - np.linalg.norm(c64)) < 1e-12


def test_kkt_residual_box_normal_cone():
    """At a bound, a gradient pointing out of the box is fully absorbed by
    the normal cone; pointing inward it counts in full."""
    n = 3
    Q = np.zeros((1, n, n))
    c = np.array([[1.0, -1.0, 0.5]])
    prob = O.Problem(Q, c, np.zeros(0), -np.ones(n), np.ones(n))
    x = np.array([-1.0, 1.0, 0.0])          # grad = c: +1 at lb, -1 at ub, 0.5 interior
    rel, rs, rf = O.kkt_residual(prob, x, np.zeros(0))
    assert abs(rs - 0.5) < 1e-15
    x = np.array([1.0, -1.0, 0.0])          # wrong-way bounds: everything counts
    rel, rs, rf = O.kkt_residual(prob, x, np.zeros(0))
    assert abs(rs - np.linalg.norm(c[0])) < 1e-15


# --------------------------------------------------------------------------
# invariants the paper proves for every run
# --------------------------------------------------------------------------

def test_monotone_trial_count_identity():
    """c_nm = 0, mu = 0: tau_k^o = tau_{k-1}, so iteration k evaluates the
    test 1 + log_{1/eta}(tau_{k-1}/tau_k) times, tau is non-increasing, and
    the total is K + log_{1/eta}(tau_bar / tau_{K-1})."""
    prob = O.Problem.from_data(W.random_qcqp(30, 4, rows=15, seed=1))
    for variant in ("yx", "xy"):
        p = O.default_params(variant, c_nm=0, restart="none")
        log = {}
        O.apdb(prob, np.zeros(30), np.zeros(4), 150, p, log)
        tau = np.array(log["tau"])
        prev = np.concatenate([[p.tau_bar], tau[:-1]])
        assert np.all(tau <= prev * (1 + 1e-15))
        expect = 1 + np.round(np.log(prev / tau) / np.log(1 / p.eta))
        np.testing.assert_array_equal(np.array(log["trials"]), expect)
        total = sum(log["trials"])
        assert total == 150 + round(math.log(p.tau_bar / tau[-1]) / math.log(1 / p.eta))


def test_nonmonotone_ratio_and_count_bound():
    """c_nm = 1: tau_k / tau_{k-1} <= phi and the number of test evaluations
    is at most (1 + log_{1/eta} phi) K + log_{1/eta}(tau_bar / tau_min)."""
    prob = O.Problem.from_data(W.random_qcqp(30, 4, rows=15, seed=2))
    for variant in ("yx", "xy"):
        p = O.default_params(variant, c_nm=1, restart="none")
        log = {}
        K = 200
        O.apdb(prob, np.zeros(30), np.zeros(4), K, p, log)
        tau = np.array(log["tau"])
        prev = np.concatenate([[p.tau_bar], tau[:-1]])
        assert np.all(tau / prev <= PHI * (1 + 1e-12))
        L = 1 / p.eta
        bound = (1 + math.log(PHI, L)) * K + math.log(p.tau_bar / tau.min(), L)
        assert sum(log["trials"]) <= bound + 1e-9


def _ergodic_lhs_rhs(prob, st, p, x, y):
    """Both sides of the ergodic inequality of the lemma for the variant
    (eq. 4.16apd for xy, eq. 3.3apd for yx), with mu = 0 (gamma constant)."""
    xb, yb = st.x_cum / st.T, st.lam_cum / st.T
    dpK = 0.5 * np.sum((x - st.x) ** 2)
    ddK = 0.5 * np.sum((y - st.lam) ** 2)
    gap = prob.lagrangian(xb, y) - prob.lagrangian(x, yb)
    if p.variant == "xy":
        lhs = p.gamma0 * (1 - (p.c_alpha + p.c_beta)) / st.sigma0 * dpK + ddK / st.sigma0 + st.T * gap
    else:
        lhs = p.gamma0 / st.sigma0 * dpK + (1 - p.c_alpha) / st.sigma0 * ddK + st.T * gap
    rhs = 0.5 * np.sum((x - st.x0) ** 2) / st.tau0 + 0.5 * np.sum((y - st.lam0) ** 2) / st.sigma0
    return lhs, rhs


@pytest.mark.parametrize("variant", ["yx", "xy"])
@pytest.mark.parametrize("c_nm", [0, 1])
def test_ergodic_bound_at_random_points(variant, c_nm):
    """The lemma's bound holds for every (x, y) in X x Y and every K; a wrong
    sign, index or step in the iteration breaks it at some point."""
    prob = tiny_problem(n=6, m=3, seed=4, ridge=0.0)
    p = O.default_params(variant, c_nm=c_nm, restart="none")
    rng = np.random.default_rng(9)
    st = O.start_routine(prob, rng.uniform(-1, 1, 6), rng.uniform(0, 1, 3), p)
    for K in range(1, 121):
        O.apdb_iteration(prob, st, p)
        if K % 20 == 0:
            for _ in range(30):
                x = rng.uniform(prob.lb, prob.ub)
                y = rng.uniform(0, 4, 3)
                lhs, rhs = _ergodic_lhs_rhs(prob, st, p, x, y)
                assert lhs <= rhs + 1e-9 * (1 + abs(rhs))


def test_backtracking_accepts_below_psi_xy():
    """For tau <= Psi_1 the xy test always holds (lemma on APDB-xy bounds):
    started at tau_bar = Psi_1 (monotone, mu = 0) no trial is ever rejected."""
    prob = tiny_problem(n=5, m=2, seed=6, ridge=0.0)
    nrm = lambda A: np.linalg.norm(A, 2)
    Lg = math.sqrt(sum(nrm(prob.Q[i]) ** 2 for i in range(1, prob.m + 1)))
    rad = np.linalg.norm(np.maximum(np.abs(prob.lb), np.abs(prob.ub)))
    Bg = nrm(prob.c[1:].T) + rad * Lg
    p = O.default_params("xy", c_nm=0, restart="none")
    # bound the dual iterates first with a normal run, then use that bound
    st = O.start_routine(prob, np.zeros(5), np.zeros(2), p)
    ymax = 0.0
    for _ in range(300):
        O.apdb_iteration(prob, st, p)
        ymax = max(ymax, float(np.linalg.norm(st.lam)))
    Bbar = 2.0 * ymax + 1.0
    Lxx = nrm(prob.Q[0]) + Bbar * Lg
    psi1 = min(math.sqrt(p.c_alpha * (1 - p.delta)) / (Bg * math.sqrt(p.gamma0)),
               math.sqrt(p.c_beta * (1 - (p.c_alpha + p.c_beta + p.delta))) / Lxx)
    p.tau_bar = psi1
    log = {}
    st = O.start_routine(prob, np.zeros(5), np.zeros(2), p)
    for _ in range(300):
        O.apdb_iteration(prob, st, p, log)
        assert np.linalg.norm(st.lam) <= Bbar
    assert max(log["trials"]) == 1


def test_Ek_closed_form_identity():
    """For quadratics the yx test function equals
    0.5 d'Q(y)d - ||d||^2/(2 tau) + sigma/(2 c_a)||dg||^2 - (1-c_a)||dy||^2/(2 sigma)
    and the xy one equals
    tau/(2 c_a)||a||^2 + sigma/(2 g0 c_b)||Q(y^k)d||^2 - ||dy||^2/(2 sigma)
      - (1/tau - (c_a g_{k-1} + c_b g0)/sigma) ||d||^2 / 2,
    a = sum_i dy_i (Q_i x~ + q_i); derived by expanding the definitions."""
    prob = tiny_problem(n=6, m=3, seed=8, ridge=0.0)
    rng = np.random.default_rng(1)
    for variant in ("yx", "xy"):
        p = O.default_params(variant)
        for _ in range(10):
            st = O.start_routine(prob, rng.uniform(-2, 2, 6), rng.uniform(0, 1, 3), p)
            for _ in range(3):
                O.apdb_iteration(prob, st, p)
            tau = rng.uniform(0.01, 0.5)
            fn = O.yx_trial if variant == "yx" else O.xy_trial
            xn, ln, ok, aux = fn(prob, st, tau, p)
            sigma = st.gamma * tau
            d = xn - st.x
            dy = ln - st.lam
            if variant == "yx":
                Qy = prob.Q[0] + np.tensordot(ln, prob.Q[1:], axes=1)
                dg = np.array([d @ (prob.Q[i] @ st.x + prob.c[i]) + 0.5 * d @ prob.Q[i] @ d
                               for i in range(1, 4)])
                E = (0.5 * d @ Qy @ d - d @ d / (2 * tau) + sigma / (2 * p.c_alpha) * dg @ dg
                     - (1 - p.c_alpha) * dy @ dy / (2 * sigma))
            else:
                a = sum(dy[i - 1] * (prob.Q[i] @ xn + prob.c[i]) for i in range(1, 4))
                b = (prob.Q[0] + np.tensordot(st.lam, prob.Q[1:], axes=1)) @ d
                gprev = st.sigma_prev / st.tau_prev
                E = (tau / (2 * p.c_alpha) * a @ a + sigma / (2 * p.gamma0 * p.c_beta) * b @ b
                     - dy @ dy / (2 * sigma)
                     - (1 / tau - (p.c_alpha * gprev + p.c_beta * p.gamma0) / sigma) * (d @ d) / 2)
            assert abs(E - aux["E"]) <= 1e-9 * (1 + abs(E))


def test_iterates_stay_in_domain_and_restarts_reset():
    prob = O.Problem.from_data(W.random_qcqp(40, 5, rows=20, seed=3))
    p = O.default_params("yx", restart="fixed", restart_period=50, max_iter=160, tol=0.0)
    r = O.rapdb(prob, p=p, keep_iterates=160)
    for x, lam in r.log["iterates"]:
        assert np.all(x >= prob.lb) and np.all(x <= prob.ub) and np.all(lam >= 0)
    assert r.restarts == 3
    # the first trial of each run starts again at tau_bar
    ti = r.log["tau_init"]
    assert ti[0] == p.tau_bar and ti[50] == p.tau_bar and ti[100] == p.tau_bar and ti[150] == p.tau_bar
    assert ti[1] != p.tau_bar


def test_adaptive_restart_fires_only_on_halving():
    prob = O.Problem.from_data(W.random_qcqp(30, 4, rows=15, seed=4))
    p = O.default_params("yx", restart="gap", gap_first=20, gap_every=40, max_iter=400, tol=0.0)
    r = O.rapdb(prob, p=p)
    ref = None
    fired = 0
    for it, G, fire in r.log["gap"]:
        assert G >= -1e-10
        if ref is None:
            ref = G
            assert not fire
            continue
        assert fire == (G <= p.q * ref)
        if fire:
            ref = G
            fired += 1
    assert fired == r.restarts and fired >= 1


def test_warm_started_restart_takes_the_last_accepted_tau():
    """restart_warm_tau: the first trial after a restart is the last accepted
    tau of the previous run (tau_bar without the option)."""
    data = W.config("C1")
    prob = O.Problem.from_data(data)
    for warm in (False, True):
        p = O.default_params("yx", restart="fixed", restart_period=20, tol=0.0, max_iter=45,
                             restart_warm_tau=warm)
        r = O.rapdb(prob, p=p)
        ti, ta = r.log["tau_init"], r.log["tau"]
        assert ti[0] == p.tau_bar
        assert ti[20] == (ta[19] if warm else p.tau_bar)
        assert ti[40] == (ta[39] if warm else p.tau_bar)
