"""Pins of the oracle's restart bookkeeping that do not go through the oracle.

Two parts of rAPDB are checked here against quantities the test computes on
its own:

* The adaptive restart of eq. (ada_restart) with the schedule of Sec. 5.1:
  the smoothed gap G_xi is taken at k = gap_first and then every gap_every
  iterations, at the current iterate; a restart fires when G_xi <= q G_ref,
  and G_ref becomes the value at the new start point.  On a separable QCQP
  (every Q_i diagonal) both parts of G_xi (Def. of the smoothed duality gap)
  have closed forms: the y-part is a projection and the x-part a coordinatewise
  clamp, so the test recomputes every logged G from the kept iterates.
* The restart from the weighted average of Algorithm 2: after K^ iterations
  the new start point is sum_k t_k z^{k+1} / sum_k t_k with t_k = sigma_k /
  sigma_0 (Algorithm 1's averaging line), and the first iterate of the next
  run is one yx step from it, which for k = 0 has a closed form (theta
  multiplies g(x^0) - g(x^{-1}) = 0).

Each checker is also run on copies of the oracle with one planted mistake
(an off-by-one in the schedule, a reference that is not moved, the gap taken
at the previous iterate, unweighted or shifted averages); every planted
mistake must be reported.
"""
import inspect

import numpy as np
import pytest

import oracle as O
from oracle import rapdb_oracle as RO


# --------------------------------------------------------------------------
# a separable QCQP: Q_i = diag(q_i)
# --------------------------------------------------------------------------

def separable_problem(n=12, m=3, seed=0, box=4.0):
    rng = np.random.default_rng(seed)
    qd = np.empty((m + 1, n))
    qd[0] = rng.uniform(0.05, 2.0, n)          # Q_0 positive definite, ill conditioned
    qd[1:] = rng.uniform(0.0, 1.5, (m, n))
    qd = qd.astype(np.float32).astype(np.float64)
    Q = np.zeros((m + 1, n, n))
    for i in range(m + 1):
        Q[i][np.arange(n), np.arange(n)] = qd[i]
    c = rng.standard_normal((m + 1, n)).astype(np.float32).astype(np.float64)
    d = -rng.uniform(0.1, 1.0, m).astype(np.float32).astype(np.float64)
    lb, ub = -box * np.ones(n), box * np.ones(n)
    return O.Problem(Q, c, d, lb, ub), qd


def gap_closed_form(qd, c, r, lb, ub, x, lam, xi):
    """G_xi(x, lam) of a separable QCQP: y-part at lam' = max(0, lam + g/(2 xi)),
    x-part at x'_j = clamp(-(c(lam)_j - 2 xi x_j) / (q(lam)_j + 2 xi))."""
    def phi(z, l):
        f = 0.5 * np.sum(qd[0] * z * z) + c[0] @ z
        g = 0.5 * (qd[1:] * z * z).sum(axis=1) + c[1:] @ z + r
        return f + l @ g, g
    _, g = phi(x, lam)
    lp = np.maximum(0.0, lam + g / (2.0 * xi))
    y_part = phi(x, lp)[0] - xi * np.sum((lp - lam) ** 2)
    qlam = qd[0] + lam @ qd[1:]
    clam = c[0] + lam @ c[1:]
    xs = np.clip(-(clam - 2.0 * xi * x) / (qlam + 2.0 * xi), lb, ub)
    x_part = phi(xs, lam)[0] + xi * np.sum((xs - x) ** 2)
    return y_part - x_part


def iterate_at(result, prob, it, x0, lam0):
    """z^it: the start point for it = 0, else the kept iterate after it iterations."""
    if it == 0:
        return np.asarray(x0, np.float64), np.asarray(lam0, np.float64)
    return result.log["iterates"][it - 1]


def check_gap_schedule(result, prob, qd, p, x0, lam0):
    """Violations of the adaptive-restart schedule and bookkeeping (empty list
    when the run follows eq. (ada_restart) with the Sec. 5.1 schedule)."""
    bad = []
    log = result.log.get("gap", [])
    its = [e[0] for e in log]
    want = list(range(p.gap_first, result.iters, p.gap_every))
    if its != want:
        bad.append(f"evaluations at {its[:6]}..., expected {want[:6]}...")
        return bad
    ref = None
    fires = []
    for it, G, fire in log:
        x, lam = iterate_at(result, prob, it, x0, lam0)
        Gc = gap_closed_form(qd, prob.c, prob.r, prob.lb, prob.ub, x, lam, p.xi)
        if abs(G - Gc) > 1e-7 * (1.0 + abs(Gc)):
            bad.append(f"G at it={it}: logged {G}, closed form {Gc}")
        want_fire = ref is not None and Gc <= p.q * ref
        if bool(fire) != want_fire:
            bad.append(f"restart decision at it={it}: {fire}, expected {want_fire}")
        if ref is None or want_fire:
            ref = Gc          # the first value, then the value at each new start point
        if want_fire:
            fires.append(it)
    if result.restarts != len(fires):
        bad.append(f"{result.restarts} restarts counted, {len(fires)} expected")
    # a restart re-enters Algorithm 1 from its initialisation line: the first
    # trial of that iteration is tau_bar again, and only there
    ti = result.log["tau_init"]
    for it in range(1, result.iters):
        reset = ti[it] == p.tau_bar
        if (it in fires) and not reset:
            bad.append(f"no reset of tau at the restart it={it}")
    return bad


def mutated_oracle(fn, old, new):
    """A copy of oracle function `fn` with the source text `old` replaced by
    `new` (exactly one occurrence), compiled in the oracle module's namespace."""
    src = inspect.getsource(fn)
    assert src.count(old) == 1, (old, src.count(old))
    ns = dict(vars(RO))
    exec(compile(src.replace(old, new), RO.__file__, "exec"), ns)
    return ns[fn.__name__]


GAP_PARAMS = dict(restart="gap", gap_first=6, gap_every=4, max_iter=400, tol=1e-7, xi=0.04, q=0.1)


def run_gap(rapdb_fn, seed):
    prob, qd = separable_problem(seed=seed)
    p = O.default_params("yx", **GAP_PARAMS)
    x0, lam0 = np.zeros(prob.n), np.zeros(prob.m)
    r = rapdb_fn(prob, x0, lam0, p, keep_iterates=p.max_iter)
    return r, prob, qd, p, x0, lam0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gap_schedule_and_reference_follow_eq_ada_restart(seed):
    r, prob, qd, p, x0, lam0 = run_gap(O.rapdb, seed)
    assert r.status == 0                              # stopped on the tolerance
    assert check_gap_schedule(r, prob, qd, p, x0, lam0) == []
    fired = [e for e in r.log["gap"] if e[2]]
    kept = [e for e in r.log["gap"][1:] if not e[2]]
    assert len(fired) >= 1 and len(kept) >= 1      # both branches exercised


GAP_MUTATIONS = [
    ("schedule shifted by one", "(it - p.gap_first) % p.gap_every == 0", "(it - p.gap_first - 1) % p.gap_every == 0"),
    ("reference moved at every evaluation", "fire = G <= p.q * G_ref", "fire = G <= p.q * G_ref\n                G_ref = G"),
    ("reference not moved", "restarts += 1\n                    G_ref = G", "restarts += 1"),
    ("gap at the previous iterate", "xs, ls = st.x, st.lam\n            if it == p.gap_first",
     "xs, ls = st.x_prev, st.lam_prev\n            if it == p.gap_first"),
    ("restart keeps the run", "                    st = start_routine(prob, xs, ls, p, st.tau_prev if p.restart_warm_tau "
                              "else None)\n                    restarts += 1\n                    G_ref = G",
     "                    restarts += 1\n                    G_ref = G"),
]


@pytest.mark.parametrize("name,old,new", GAP_MUTATIONS, ids=[m[0] for m in GAP_MUTATIONS])
def test_gap_pin_catches_planted_mistakes(name, old, new):
    mutant = mutated_oracle(RO.rapdb, old, new)
    found = []
    for seed in (0, 1, 2):
        r, prob, qd, p, x0, lam0 = run_gap(mutant, seed)
        found += check_gap_schedule(r, prob, qd, p, x0, lam0)
    assert found, f"planted mistake '{name}' passed the pin"


# --------------------------------------------------------------------------
# restart from the weighted average (Algorithm 2)
# --------------------------------------------------------------------------

def yx_first_step(prob, xs, ls, tau, p):
    """The first iterate of an APDB-yx run started at (xs, ls) with accepted
    step tau: sigma = gamma_0 tau, and since x^{-1} = x^0 the momentum term
    vanishes: y^1 = max(0, ls + sigma g(xs)), x^1 = clamp(xs - tau grad_x L(xs, y^1))."""
    sigma = p.gamma0 * tau
    g = np.array([0.5 * xs @ prob.Q[i] @ xs + prob.c[i] @ xs + prob.r[i - 1] for i in range(1, prob.m + 1)])
    y1 = np.maximum(0.0, ls + sigma * g)
    grad = prob.Q[0] @ xs + prob.c[0] + sum(y1[i - 1] * (prob.Q[i] @ xs + prob.c[i]) for i in range(1, prob.m + 1))
    return np.clip(xs - tau * grad, prob.lb, prob.ub), y1


def check_average_restart(result, prob, p, x0, lam0):
    """Violations of Algorithm 2's restart line: at each restart (every K^
    iterations) the next run starts from sum t_k z^{k+1} / sum t_k over the
    finished run, t_k = sigma_k / sigma_0 from the logged sigma."""
    bad = []
    K = p.restart_period
    sig = result.log["sigma"]
    tau = result.log["tau"]
    its = result.log["iterates"]
    for start in range(0, result.iters - K, K):
        t = np.array(sig[start:start + K]) / sig[start]
        xs = sum(tk * its[start + k][0] for k, tk in enumerate(t)) / t.sum()
        ls = sum(tk * its[start + k][1] for k, tk in enumerate(t)) / t.sum()
        x1, y1 = yx_first_step(prob, xs, ls, tau[start + K], p)
        xg, yg = its[start + K]
        if not (np.allclose(xg, x1, rtol=1e-11, atol=1e-11) and np.allclose(yg, y1, rtol=1e-11, atol=1e-11)):
            bad.append(f"run starting at {start + K}: first iterate is not the step from the weighted average "
                       f"(|dx| = {np.max(np.abs(xg - x1)):.3e})")
        if result.log["tau_init"][start + K] != p.tau_bar:
            bad.append(f"no reset of tau at {start + K}")
    return bad


def run_average(rapdb_fn, seed, mu):
    from paper_2605_29291_gb300 import workloads as W
    prob = O.Problem.from_data(W.random_qcqp(24, 3, rows=12, seed=seed))
    p = O.default_params("yx", restart="fixed", restart_period=15, restart_from_average=True, max_iter=50,
                         tol=0.0, mu=mu)
    x0, lam0 = np.zeros(prob.n), np.zeros(prob.m)
    r = rapdb_fn(prob, x0, lam0, p, keep_iterates=p.max_iter)
    return r, prob, p, x0, lam0


@pytest.mark.parametrize("seed,mu", [(0, 0.0), (1, 0.0), (2, 0.05)])
def test_restart_from_weighted_average_follows_algorithm_2(seed, mu):
    r, prob, p, x0, lam0 = run_average(O.rapdb, seed, mu)
    assert r.restarts == 3
    sig = r.log["sigma"]
    assert max(sig[:15]) > 1.01 * min(sig[:15])      # the weights are not all equal
    assert check_average_restart(r, prob, p, x0, lam0) == []


AVG_MUTATIONS = [
    (RO.apdb_iteration, "unweighted average", "t_k = sigma / st.sigma0", "t_k = 1.0"),
    (RO.apdb_iteration, "average of the previous iterates", "st.x_cum = st.x_cum + t_k * x_new",
     "st.x_cum = st.x_cum + t_k * st.x"),
    (RO.apdb_iteration, "weights from tau", "t_k = sigma / st.sigma0", "t_k = tau / p.tau_bar"),
    (RO.rapdb, "restart from the last iterate",
     "if p.restart_from_average:\n                xs, ls = st.x_cum / st.T, st.lam_cum / st.T",
     "if p.restart_from_average:\n                xs, ls = st.x, st.lam"),
]


@pytest.mark.parametrize("fn,name,old,new", AVG_MUTATIONS, ids=[m[1] for m in AVG_MUTATIONS])
def test_average_pin_catches_planted_mistakes(fn, name, old, new):
    if fn is RO.apdb_iteration:
        mutant_iter = mutated_oracle(fn, old, new)
        ns = dict(vars(RO))
        ns["apdb_iteration"] = mutant_iter
        src = inspect.getsource(RO.rapdb)
        exec(compile(src, RO.__file__, "exec"), ns)
        rapdb_fn = ns["rapdb"]
    else:
        rapdb_fn = mutated_oracle(fn, old, new)
    found = []
    for seed, mu in ((0, 0.0), (1, 0.0), (2, 0.05)):
        r, prob, p, x0, lam0 = run_average(rapdb_fn, seed, mu)
        found += check_average_restart(r, prob, p, x0, lam0)
    assert found, f"planted mistake '{name}' passed the pin"
