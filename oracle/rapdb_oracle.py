"""Plain FP64 CPU implementation of APDB / rAPDB for box-constrained convex QCQPs.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU
arms use it.  It is deliberately slow and literal: every quantity the paper
defines is evaluated from its definition (Phi, grad_x Phi, g, the test function
E_k) with full float64 matrix-vector products; no algebraic shortcut, fusion or
reordering beyond what the paper's formulas state.

Sources (arXiv 2605.29291):
  * Problem, coupling Phi and its gradients: Sec. 2.1, eq. (QCQP) and the
    QCQP coupling function; Euclidean Bregman distances D = 0.5||.||^2
    (Sec. 2.2, remark after Def. of Bregman distances).
  * APDB-xy: Algorithm 1 with the test function of eq. (backtracking).
  * APDB-yx: Sec. 3.2, the modified parameter/update rules (eq. apdb-yx-y)
    and its test function E_k.  The dual ball B is not imposed (Sec. 5).
  * Step rule (monotone / non-monotone): Algorithm 1's tau update and
    Remark (non-monotone step sizes), eq. (nonmonotone-tau).
  * rAPDB fixed-frequency restart: Algorithm 2; restart from the last
    iterate as in the experiments (Sec. 5.1, implementation details), or from
    the weighted average as Algorithm 2 states.
  * Adaptive restart: eq. (ada_restart) with the schedule of Sec. 5.1/5.2
    (first evaluation at k=50 (yx) / k=100 (xy), then every gap_every).
  * Smoothed duality gap G_xi: Def. (smoothed duality gap) and the remark on
    computing it (y-part is a projection, x-part a strongly convex box QP).
  * KKT residual: the residual r(x, v, lambda) of Thm. (metric
    subregularity sufficient conditions) with the map G(z) of its proof; the
    normalisation into a relative residual is a reading (the paper is silent).
  * Dual on a simplex (the kernel-learning min-max problem of Sec. 5.2, eq.
    min-max-KML: y in {y >= 0, sum y = r}): the projection onto the simplex
    by the sort-and-threshold method of Held, Wolfe and Crowder (1974), the
    simplex normal cone in the KKT residual, and the simplex projection in
    the y-part of G_xi.
  * Linear equalities Ax = b (the paper's problem class with the equality
    block, eq. NCP; the kernel-learning constraint b'x = 0 of Sec. 5.2): the
    last n_eq rows of the constraint data are a_k'x - b_k with Q = 0 and a
    free (unprojected) multiplier; their KKT component is |a_k'x - b_k|.
  * A primal set with one hyperplane, X = {lb <= x <= ub, a'x = beta} (the
    kernel-learning problem of Sec. 5.2, eq. min-max-KML, minimises over
    {x >= 0, b'x = 0}: lb = 0, ub = +inf, a = b, beta = 0).  The Euclidean
    projection onto X is x = clamp(v - nu a) with the scalar nu that solves
    a'clamp(v - nu a) = beta (the optimality conditions of the projection;
    the left side is piecewise linear and non-increasing in nu, so nu is
    found exactly between two of its breakpoints).  The normal cone is
    N_X(x) = {t a + N_box(x)}, so r_stat = min over t of the box-cone
    residual of grad + t a (a convex piecewise quadratic, minimised piece by
    piece).  The gap's x-subproblem over X is the box QP with the term t a'x
    added, t found by bisection so that a'x(t) = beta (a'x(t) is
    non-increasing in t).

Parity pins (see tests/test_oracle_pins.py, tests/test_oracle_simplex_pins.py):
closed forms (ball constraint,
interior PD QP, one-step iterate), weak-duality certificates from an exact box
QP by exhaustive active-set enumeration, the ergodic bounds (Lemmas with eqs.
4.16apd / 3.3apd) at random points, step-size invariants (monotone identity of
the trial count, the golden-ratio bound of the non-monotone rule), the algebraic
identity of E_k for quadratics, G_xi(z*) = 0 and G_xi >= 0, and the
x-subproblem against brute-force active-set enumeration; the adaptive-restart
schedule, its decisions and reference value against closed-form gaps of a
separable QCQP, and the restart from the weighted average against the
independently formed average and the closed-form first step of the next run
(tests/test_oracle_restart_pins.py, each also run on planted mistakes).
Parity unpinned: absolute iteration counts of the paper's tables (different
instances and data).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Parameters (Sec. 5: eta = 0.7; yx c_alpha = 0.4, delta = 0.5; xy c_alpha = 0.25,
# c_beta = 0.3, delta = 0.4; xi = 0.04, q = 1/2).
# ---------------------------------------------------------------------------


@dataclass
class Params:
    variant: str = "yx"              # "yx" (Sec. 3.2) or "xy" (Algorithm 1)
    c_nm: int = 1                    # 0 monotone, 1 non-monotone (eq. nonmonotone-tau)
    backtracking: bool = True        # False: fixed step tau_bar, every trial accepted
    mu: float = 0.0
    c_alpha: float = 0.4
    c_beta: float = 0.0
    delta: float = 0.5
    eta: float = 0.7
    tau_bar: float = 1.0
    gamma0: float = 1.0
    restart: str = "fixed"           # "none" | "fixed" (Algorithm 2) | "gap" (eq. ada_restart)
    restart_period: int = 200
    restart_from_average: bool = False
    restart_warm_tau: bool = False   # a restart starts from the last accepted tau instead of tau_bar
    xi: float = 0.04
    q: float = 0.5
    gap_first: int = 50
    gap_every: int = 500
    max_iter: int = 50000
    max_trials: int = 60
    kkt_every: int = 1
    tol: float = 1e-6


def default_params(variant: str = "yx", **kw) -> Params:
    """The paper's experiment settings (Sec. 5.1) for the chosen variant."""
    if variant == "yx":
        p = Params(variant="yx", c_alpha=0.4, c_beta=0.0, delta=0.5, gap_first=50)
    elif variant == "xy":
        p = Params(variant="xy", c_alpha=0.25, c_beta=0.3, delta=0.4, gap_first=100)
    else:
        raise ValueError(variant)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class BacktrackError(RuntimeError):
    pass


# ---------------------------------------------------------------------------
# Problem: f(x) = 0.5 x'Q_0 x + q_0'x,  g_i(x) = 0.5 x'Q_i x + q_i'x + r_i,
# Phi(x, lam) = f(x) + lam'g(x)   (Sec. 2.1, QCQP coupling, p = 0).
# ---------------------------------------------------------------------------


def proj_simplex(v, r: float = 1.0):
    """Euclidean projection of v onto {y >= 0, sum y = r} (Held, Wolfe and
    Crowder, 1974): sort v in decreasing order, take the largest k with
    u_k > (sum_{j<=k} u_j - r) / k, then y = max(v - theta, 0) with theta =
    (sum_{j<=k} u_j - r) / k."""
    v = np.asarray(v, np.float64)
    u = np.sort(v)[::-1]
    css = np.cumsum(u) - r
    k = np.arange(1, v.size + 1)
    rho = int(np.nonzero(u - css / k > 0)[0][-1]) + 1
    theta = css[rho - 1] / rho
    return np.maximum(v - theta, 0.0)


def simplex_cone_distance(g, lam):
    """dist(g, N_Delta(lam)) for the simplex Delta = {y >= 0, sum y = r}:
    N_Delta(lam) = {t 1 - nu : nu >= 0, nu_i = 0 where lam_i > 0}, so the
    distance is min over t of sqrt(sum_{lam_i>0} (g_i - t)^2 +
    sum_{lam_i=0} max(g_i - t, 0)^2).  The function of t is convex and
    piecewise quadratic with breakpoints at the off-support g_i; on each
    piece its minimiser is the mean of g over the support and the off-support
    entries above the piece.  Returns (distance, the minimising t)."""
    g = np.asarray(g, np.float64)
    on = np.asarray(lam, np.float64) > 0.0
    off = np.sort(g[~on])
    best = (math.inf, 0.0)
    # pieces: t in (-inf, off_0], (off_0, off_1], ..., (off_last, +inf)
    edges = [-math.inf] + list(off) + [math.inf]
    for p in range(len(edges) - 1):
        lo, hi = edges[p], edges[p + 1]
        active = np.concatenate([g[on], off[p:]])     # off-support entries above the piece
        if active.size == 0:
            continue
        t = min(max(float(np.mean(active)), lo), hi)      # the piece's minimiser
        val = float(np.sum((g[on] - t) ** 2) + np.sum(np.maximum(g[~on] - t, 0.0) ** 2))
        if val < best[0]:
            best = (val, t)
    return math.sqrt(best[0]), best[1]


def hyperplane_phi(v, lb, ub, a, beta, nu):
    """a'clamp(v - nu a, lb, ub) - beta."""
    return float(a @ np.minimum(np.maximum(v - nu * a, lb), ub)) - beta


def proj_box_hyperplane(v, lb, ub, a, beta):
    """Euclidean projection of v onto {lb <= x <= ub, a'x = beta}.

    The projection is x = clamp(v - nu a, lb, ub) for the nu with
    a'x = beta.  phi(nu) = a'clamp(v - nu a) - beta is continuous, piecewise
    linear and non-increasing; its breakpoints are the nu at which some
    v_j - nu a_j reaches lb_j or ub_j.  The root lies between two adjacent
    breakpoints (found by bisection over the sorted breakpoints), or beyond the
    outermost one, and is the root of the linear piece there.  Returns
    (x, nu)."""
    v = np.asarray(v, np.float64)
    a = np.asarray(a, np.float64)
    nz = a != 0.0
    bps = []
    for bound in (lb, ub):
        bb = np.asarray(bound, np.float64)
        ok = nz & np.isfinite(bb)
        bps.append((v[ok] - bb[ok]) / a[ok])
    bp = np.unique(np.concatenate(bps))
    phi = lambda t: hyperplane_phi(v, lb, ub, a, beta, t)

    def slope_at(t0, t1):
        # phi is linear on [t0, t1]: its slope from two evaluations, or from
        # the free coordinates when the piece is unbounded
        mid = 0.5 * (t0 + t1) if np.isfinite(t0) and np.isfinite(t1) else (t1 - 1.0 if np.isfinite(t1) else t0 + 1.0)
        xm = v - mid * a
        free = (xm > lb) & (xm < ub)
        return -float(np.sum(a[free] ** 2))

    if bp.size == 0:
        sl = slope_at(-np.inf, np.inf)
        if sl == 0.0:
            raise ValueError("the hyperplane does not meet the box")
        nu = phi(0.0) / -sl
        return np.minimum(np.maximum(v - nu * a, lb), ub), nu
    lo_i, hi_i = 0, bp.size - 1
    f_lo, f_hi = phi(bp[lo_i]), phi(bp[hi_i])
    if f_lo < 0.0:          # root below the smallest breakpoint
        sl = slope_at(-np.inf, bp[0])
        if sl == 0.0:
            raise ValueError("the hyperplane does not meet the box")
        nu = bp[0] - f_lo / sl
    elif f_hi > 0.0:        # root above the largest breakpoint
        sl = slope_at(bp[-1], np.inf)
        if sl == 0.0:
            raise ValueError("the hyperplane does not meet the box")
        nu = bp[-1] - f_hi / sl
    else:
        # phi(bp[lo_i]) >= 0 >= phi(bp[hi_i]): bisect to adjacent breakpoints
        while hi_i - lo_i > 1:
            mid = (lo_i + hi_i) // 2
            fm = phi(bp[mid])
            if fm >= 0.0:
                lo_i, f_lo = mid, fm
            else:
                hi_i, f_hi = mid, fm
        if f_lo == 0.0:
            nu = bp[lo_i]
        elif f_hi == 0.0:
            nu = bp[hi_i]
        else:               # linear between the two: its root
            nu = bp[lo_i] + f_lo * (bp[hi_i] - bp[lo_i]) / (f_lo - f_hi)
    return np.minimum(np.maximum(v - nu * a, lb), ub), nu


def box_cone_residual(g, x, lb, ub):
    """Componentwise dist(0, g + N_box(x)): max(-g, 0) at a lower bound,
    max(g, 0) at an upper bound, |g| inside."""
    return np.where(x <= lb, np.maximum(-g, 0.0), np.where(x >= ub, np.maximum(g, 0.0), np.abs(g)))


def hyperplane_cone_distance(g, x, lb, ub, a):
    """dist(0, g + N_X(x)) for X = box with the hyperplane a'x = beta:
    N_X(x) = {t a + nu : nu in N_box(x)}, so the distance is the minimum over
    t of F(t) = ||box_cone_residual(g + t a)||.  F^2 is convex and piecewise
    quadratic; its breakpoints are the t at which g_j + t a_j = 0 for a
    coordinate at a bound.  On each piece the active terms are fixed and the
    minimiser is the least-squares t over them, clamped to the piece.
    Returns (distance, t)."""
    g = np.asarray(g, np.float64)
    a = np.asarray(a, np.float64)
    at_lo, at_hi = x <= lb, x >= ub
    bound = (at_lo | at_hi) & (a != 0.0)
    edges = np.unique(-g[bound] / a[bound])
    edges = np.concatenate([[-np.inf], edges, [np.inf]])
    best = (np.inf, 0.0)
    F2 = lambda t: float(np.sum(box_cone_residual(g + t * a, x, lb, ub) ** 2))
    for p in range(edges.size - 1):
        lo, hi = edges[p], edges[p + 1]
        mid = 0.5 * (lo + hi) if np.isfinite(lo) and np.isfinite(hi) else (hi - 1.0 if np.isfinite(hi) else
                                                                             (lo + 1.0 if np.isfinite(lo) else 0.0))
        gm = g + mid * a
        act = ~(at_lo | at_hi) | (at_lo & (gm < 0.0)) | (at_hi & (gm > 0.0))
        den = float(np.sum(a[act] ** 2))
        t = -float(np.sum(a[act] * g[act])) / den if den > 0.0 else mid
        t = min(max(t, lo), hi)
        val = F2(t)
        if val < best[0]:
            best = (val, t)
    return np.sqrt(best[0]), best[1]


class Problem:
    """Float64 copy of the canonical float32 data.  Q[0] is Q_0.  With
    dual_radius set, the dual set is the simplex {y >= 0, sum y = dual_radius}
    instead of the nonnegative orthant.  With hyperplane = (a, beta) the primal
    set is the box intersected with {a'x = beta}."""

    def __init__(self, Q, c, d, lb, ub, dual_radius=None, n_eq=0, hyperplane=None):
        self.dual_radius = None if dual_radius is None else float(dual_radius)
        self.hyp = None if hyperplane is None else (np.asarray(hyperplane[0], np.float64), float(hyperplane[1]))
        self.n_eq = int(n_eq)            # the last n_eq constraints are equalities (free multipliers)
        self.Q = np.asarray(Q, dtype=np.float64)
        self.c = np.asarray(c, dtype=np.float64)
        self.r = np.asarray(d, dtype=np.float64)
        self.lb = np.asarray(lb, dtype=np.float64)
        self.ub = np.asarray(ub, dtype=np.float64)
        self.n = self.Q.shape[1]
        self.m = self.Q.shape[0] - 1
        assert self.c.shape == (self.m + 1, self.n) and self.r.shape == (self.m,)
        assert 0 <= self.n_eq <= self.m
        self.m_ineq = self.m - self.n_eq
        assert not np.any(self.Q[1 + self.m_ineq:]), "equality rows carry no quadratic term"

    @classmethod
    def from_data(cls, data, dual_radius=None) -> "Problem":
        """The problem of a QCQPData; equalities A_eq x = b_eq (if any) become
        the last rows, a_k'x - b_k with a zero quadratic term."""
        h = data.numpy()
        if dual_radius is None:
            dual_radius = (data.meta or {}).get("dual_radius")
        hyp = None
        if getattr(data, "hyp_a", None) is not None:
            hyp = (np.asarray(data.numpy().hyp_a, np.float64), float(data.hyp_beta))
        Q, c, d = data.dense_q(), h.c, h.d
        p = 0
        if getattr(h, "A_eq", None) is not None:
            A = np.asarray(h.A_eq, np.float64).reshape(-1, data.n)
            p = A.shape[0]
            Q = np.concatenate([Q, np.zeros((p, data.n, data.n), Q.dtype)], axis=0)
            c = np.concatenate([np.asarray(c, np.float64), A], axis=0)
            d = np.concatenate([np.asarray(d, np.float64), -np.asarray(h.b_eq, np.float64)])
        return cls(Q, c, d, h.lb, h.ub, dual_radius, n_eq=p, hyperplane=hyp)

    # objective and constraints --------------------------------------------
    def f(self, x):
        return 0.5 * x @ (self.Q[0] @ x) + self.c[0] @ x

    def g(self, x):
        if self.m == 0:
            return np.zeros(0)
        return np.array([0.5 * x @ (self.Q[i] @ x) + self.c[i] @ x + self.r[i - 1]
                         for i in range(1, self.m + 1)])

    def phi(self, x, lam):
        """Phi(x, y) = f(x) + <lam, g(x)>."""
        return self.f(x) + lam @ self.g(x)

    def grad_x(self, x, lam):
        """grad_x Phi(x, y) = Q_0 x + q_0 + sum_i lam_i (Q_i x + q_i)."""
        gr = self.Q[0] @ x + self.c[0]
        for i in range(1, self.m + 1):
            gr = gr + lam[i - 1] * (self.Q[i] @ x + self.c[i])
        return gr

    def grad_y(self, x, lam):
        """grad_y Phi(x, y) = g(x) (independent of y for the lambda block)."""
        return self.g(x)

    def lagrangian(self, x, lam):
        """L(x, y) on X x Y (both inside their sets): equals Phi."""
        return self.phi(x, lam)

    def proj_x(self, x):
        if self.hyp is not None:
            return proj_box_hyperplane(x, self.lb, self.ub, self.hyp[0], self.hyp[1])[0]
        return np.minimum(np.maximum(x, self.lb), self.ub)

    def proj_y(self, lam):
        """Projection onto Y: the orthant or the simplex for the inequality
        multipliers, the identity for the equality multipliers."""
        lam = np.asarray(lam, np.float64)
        mi = self.m_ineq
        head = lam[:mi]
        if self.dual_radius is not None:
            head = proj_simplex(head, self.dual_radius) if mi > 0 else head
        else:
            head = np.maximum(head, 0.0)
        return np.concatenate([head, lam[mi:]])

    def default_lam0(self):
        """A dual start in Y: 0, or the simplex's centre (equality multipliers 0)."""
        lam = np.zeros(self.m)
        if self.dual_radius is not None and self.m_ineq > 0:
            lam[:self.m_ineq] = self.dual_radius / self.m_ineq
        return lam


def Dp(x, xk):
    """Euclidean Bregman distance 0.5||x - xk||^2 (Sec. 2.2)."""
    v = x - xk
    return 0.5 * float(v @ v)


Dd = Dp


# ---------------------------------------------------------------------------
# One APDB run (Algorithm 1 for xy; Sec. 3.2 rules for yx), as explicit state.
# ---------------------------------------------------------------------------


@dataclass
class RoutineState:
    x: np.ndarray
    x_prev: np.ndarray
    lam: np.ndarray
    lam_prev: np.ndarray
    tau_prev: float            # tau_{k-1}
    sigma_prev: float          # sigma_{k-1}
    gamma: float               # gamma_k
    tau_init: float            # first trial value of tau_k
    alpha_k: float             # alpha_k (set by the previous iteration)
    beta_k: float              # beta_k
    x0: np.ndarray = None
    lam0: np.ndarray = None
    tau0: float = None         # accepted tau_0 of this run
    sigma0: float = None       # accepted sigma_0 of this run
    k: int = 0
    x_cum: np.ndarray = None
    lam_cum: np.ndarray = None
    T: float = 0.0


def start_routine(prob: Problem, x0, lam0, p: Params, tau_start=None) -> RoutineState:
    """Initialisation line of Algorithm 1: (x^-1, y^-1) = (x^0, y^0),
    tau_-1 = tau_0 = tau_bar, sigma_-1 = gamma_0 tau_0, cumulative sums zero.
    alpha_0, beta_0 follow the recurrences at k = -1 (yx: alpha = c_alpha /
    sigma; xy: alpha = c_alpha / tau, beta = gamma_0 c_beta / sigma).
    tau_start replaces tau_bar (the warm-started restart option)."""
    t0 = p.tau_bar if tau_start is None else float(tau_start)
    sigma_m1 = p.gamma0 * t0
    if p.variant == "yx":
        a0, b0 = p.c_alpha / sigma_m1, 0.0
    else:
        a0, b0 = p.c_alpha / t0, p.gamma0 * p.c_beta / sigma_m1
    x0 = np.array(x0, dtype=np.float64)
    lam0 = np.array(lam0, dtype=np.float64)
    return RoutineState(x=x0.copy(), x_prev=x0.copy(), lam=lam0.copy(), lam_prev=lam0.copy(),
                        tau_prev=t0, sigma_prev=sigma_m1, gamma=p.gamma0,
                        tau_init=t0, alpha_k=a0, beta_k=b0, x0=x0.copy(),
                        lam0=lam0.copy(), x_cum=np.zeros_like(x0), lam_cum=np.zeros_like(lam0))


def yx_trial(prob: Problem, st: RoutineState, tau: float, p: Params):
    """One trial of APDB-yx (Sec. 3.2): dual step with momentum on grad_y Phi,
    then a projected primal step at the new dual point; returns the candidate
    and whether the test E_k <= -delta/tau D_p - delta/sigma D_d holds."""
    sigma = st.gamma * tau
    theta = st.sigma_prev / sigma
    alpha_next = p.c_alpha / sigma
    s = (1.0 + theta) * prob.grad_y(st.x, st.lam) - theta * prob.grad_y(st.x_prev, st.lam_prev)
    lam_new = prob.proj_y(st.lam + sigma * s)
    x_new = prob.proj_x(st.x - tau * prob.grad_x(st.x, lam_new))
    dp, dd = Dp(x_new, st.x), Dd(lam_new, st.lam)
    gy_diff = prob.grad_y(x_new, lam_new) - prob.grad_y(st.x, lam_new)
    E = (prob.phi(x_new, lam_new) - prob.phi(st.x, lam_new)
         - prob.grad_x(st.x, lam_new) @ (x_new - st.x) - dp / tau
         + (1.0 / (2.0 * alpha_next)) * float(gy_diff @ gy_diff)
         - (1.0 / sigma - theta * st.alpha_k) * dd)
    ok = E <= -p.delta / tau * dp - p.delta / sigma * dd
    return x_new, lam_new, ok, dict(sigma=sigma, theta=theta, alpha_next=alpha_next,
                                    beta_next=0.0, E=E)


def xy_trial(prob: Problem, st: RoutineState, tau: float, p: Params):
    """One trial of APDB-xy (Algorithm 1): primal step with momentum on
    grad_x Phi, dual projected ascent at the new primal point, and the test
    function of eq. (backtracking)."""
    sigma = st.gamma * tau
    theta = st.sigma_prev / sigma
    alpha_next = p.c_alpha / tau
    beta_next = p.gamma0 * p.c_beta / sigma
    s = (1.0 + theta) * prob.grad_x(st.x, st.lam) - theta * prob.grad_x(st.x_prev, st.lam_prev)
    x_new = prob.proj_x(st.x - tau * s)
    lam_new = prob.proj_y(st.lam + sigma * prob.grad_y(x_new, st.lam))
    dp, dd = Dp(x_new, st.x), Dd(lam_new, st.lam)
    a = prob.grad_x(x_new, lam_new) - prob.grad_x(x_new, st.lam)
    b = prob.grad_x(x_new, st.lam) - prob.grad_x(st.x, st.lam)
    E = ((1.0 / (2.0 * alpha_next)) * float(a @ a) - dd / sigma
         + ((1.0 / (2.0 * beta_next)) * float(b @ b) if beta_next > 0 else
            (0.0 if float(b @ b) == 0.0 else math.inf))
         - (1.0 / tau - theta * (st.alpha_k + st.beta_k)) * dp)
    ok = E <= -p.delta / tau * dp - p.delta / sigma * dd
    return x_new, lam_new, ok, dict(sigma=sigma, theta=theta, alpha_next=alpha_next,
                                    beta_next=beta_next, E=E)


def apdb_iteration(prob: Problem, st: RoutineState, p: Params, log: dict | None = None) -> int:
    """Iteration k of APDB: the backtracking loop (shrink tau by eta until the
    test holds), then the averaging line and the gamma / tau updates
    (Algorithm 1; eq. nonmonotone-tau when c_nm = 1).  Returns the number of
    test evaluations.  With backtracking off the first trial is accepted and
    tau stays at tau_bar."""
    trial_fn = yx_trial if p.variant == "yx" else xy_trial
    tau = st.tau_init
    for trial in range(1, p.max_trials + 1):
        x_new, lam_new, ok, aux = trial_fn(prob, st, tau, p)
        if ok or not p.backtracking:
            break
        tau = p.eta * tau
    else:
        raise BacktrackError(f"no step accepted after {p.max_trials} trials")
    sigma = aux["sigma"]
    if st.k == 0:
        st.tau0, st.sigma0 = tau, sigma
    t_k = sigma / st.sigma0
    st.x_cum = st.x_cum + t_k * x_new
    st.lam_cum = st.lam_cum + t_k * lam_new
    st.T += t_k
    if p.backtracking:
        gamma_next = st.gamma * (1.0 + p.mu * tau)
        tau_next = tau * math.sqrt(st.gamma / gamma_next * (1.0 + p.c_nm * tau / st.tau_prev))
    else:
        gamma_next, tau_next = st.gamma, tau
    if log is not None:
        log.setdefault("tau", []).append(tau)
        log.setdefault("tau_init", []).append(st.tau_init)
        log.setdefault("trials", []).append(trial)
        log.setdefault("sigma", []).append(sigma)
        log.setdefault("gamma", []).append(st.gamma)
    st.x_prev, st.x = st.x, x_new
    st.lam_prev, st.lam = st.lam, lam_new
    st.tau_prev, st.sigma_prev = tau, sigma
    st.alpha_k, st.beta_k = aux["alpha_next"], aux["beta_next"]
    st.gamma, st.tau_init = gamma_next, tau_next
    st.k += 1
    return trial


def apdb(prob: Problem, x0, lam0, K: int, p: Params, log: dict | None = None):
    """APDB(x^0, y^0, K): K iterations, returns the weighted averages
    (x_cum, y_cum) / T and the final state (Algorithm 1's return line)."""
    st = start_routine(prob, x0, lam0, p)
    for _ in range(K):
        apdb_iteration(prob, st, p, log)
    return st.x_cum / st.T, st.lam_cum / st.T, st


# ---------------------------------------------------------------------------
# KKT residual (reading of r(x, v, lambda) with relative normalisation).
# ---------------------------------------------------------------------------


def kkt_residual(prob: Problem, x, lam):
    """Returns (rel_kkt, r_stat, r_feas) with

      r_stat_j = dist(0, grad_x Phi(x, lam)_j + N_X(x)_j)   (box normal cone;
                 with the hyperplane, ||r_stat|| = dist(0, grad + N_X(x))),
      r_feas_i = dist(0, -g_i(x) + N_{R+}(lam_i)),
                 (simplex dual: ||r_feas|| = dist(g(x), N_Delta(lam)); an
                 equality row contributes |a_k'x - b_k|),
      rel_kkt = max(||r_stat|| / (1 + max(||Q_0x+q_0||, ||sum lam_i(Q_ix+q_i)||)),
                    ||r_feas|| / (1 + max(||r||, ||(g_i(x) - r_i)_i||))).
    """
    x = np.asarray(x, np.float64)
    lam = np.asarray(lam, np.float64)
    gf = prob.Q[0] @ x + prob.c[0]
    gc = np.zeros_like(x)
    for i in range(1, prob.m + 1):
        gc = gc + lam[i - 1] * (prob.Q[i] @ x + prob.c[i])
    grad = gf + gc
    if prob.hyp is not None:        # dist(0, grad + N_X(x)) with the hyperplane's direction
        r_stat = float(hyperplane_cone_distance(grad, x, prob.lb, prob.ub, prob.hyp[0])[0])
    else:
        r_stat = float(np.linalg.norm(box_cone_residual(grad, x, prob.lb, prob.ub)))
    g = prob.g(x)
    mi = prob.m_ineq
    if prob.dual_radius is not None and mi > 0:
        r_in = simplex_cone_distance(g[:mi], lam[:mi])[0]      # dist(0, -g + N_Delta(lam))
    else:
        r_in = float(np.linalg.norm(np.where(lam[:mi] > 0.0, np.abs(g[:mi]), np.maximum(g[:mi], 0.0))))
    r_feas = math.sqrt(r_in ** 2 + float(np.sum(g[mi:] ** 2)))   # equalities: |a_k'x - b_k|
    den_s = 1.0 + max(float(np.linalg.norm(gf)), float(np.linalg.norm(gc)))
    den_f = 1.0 + max(float(np.linalg.norm(prob.r)), float(np.linalg.norm(g - prob.r)))
    return max(r_stat / den_s, r_feas / den_f), r_stat, r_feas


# ---------------------------------------------------------------------------
# Smoothed duality gap G_xi(z) with D = 0.5||.||^2 (so 2 xi D = xi ||.||^2).
# ---------------------------------------------------------------------------


def gap_x_subproblem(prob: Problem, x, lam, xi):
    """argmin_{x' in X} Phi(x', lam) + xi ||x' - x||^2: a strongly convex box QP
    (Hessian Q(lam) + 2 xi I).  Solved exactly by bounded-variable least
    squares (an active-set method that terminates at the exact minimiser):
    with H = L L', 0.5 x'Hx + l'x = 0.5||L'x + L^{-1} l||^2 - const.  With
    the hyperplane a'x = beta in X, the equality's multiplier t is found by
    bisection on a'x(t) = beta, x(t) the box QP's minimiser with l + t a."""
    from scipy.linalg import cholesky, solve_triangular
    from scipy.optimize import lsq_linear
    H = prob.Q[0].copy()
    lin = prob.c[0].copy()
    for i in range(1, prob.m + 1):
        H += lam[i - 1] * prob.Q[i]
        lin += lam[i - 1] * prob.c[i]
    H = H + 2.0 * xi * np.eye(prob.n)
    lin = lin - 2.0 * xi * np.asarray(x, np.float64)
    L = cholesky(H, lower=True)
    lb, ub = prob.lb, prob.ub

    def box_qp(l):
        rhs = -solve_triangular(L, l, lower=True)
        res = lsq_linear(L.T, rhs, bounds=(lb, ub), method="bvls", tol=1e-15,
                         lsmr_tol=None, max_iter=None)
        return np.minimum(np.maximum(res.x, lb), ub)

    if prob.hyp is None:
        return box_qp(lin)
    # X with the hyperplane a'x = beta: the box QP with the multiplier term
    # t a'x; h(t) = a'x(t) - beta is non-increasing in t, bisected to the root
    a, beta = prob.hyp
    h = lambda t: float(a @ box_qp(lin + t * a)) - beta
    t_lo, t_hi = -1.0, 1.0
    while h(t_lo) < 0.0:
        t_lo *= 2.0
    while h(t_hi) > 0.0:
        t_hi *= 2.0
    for _ in range(200):
        t = 0.5 * (t_lo + t_hi)
        if t == t_lo or t == t_hi:
            break
        if h(t) > 0.0:
            t_lo = t
        else:
            t_hi = t
    return box_qp(lin + 0.5 * (t_lo + t_hi) * a)


def smoothed_gap(prob: Problem, x, lam, xi):
    """Self-centred smoothed gap G_xi(z) =
    [max_{lam' >= 0} Phi(x, lam') - xi||lam' - lam||^2]
      - [min_{x' in X} Phi(x', lam) + xi||x' - x||^2].
    The y-part is a projection: lam' = proj_Y(lam + g(x) / (2 xi)) (max(0, .)
    for the orthant, the simplex projection for a simplex dual)."""
    x = np.asarray(x, np.float64)
    lam = np.asarray(lam, np.float64)
    g = prob.g(x)
    lam_s = prob.proj_y(lam + g / (2.0 * xi))
    y_part = prob.phi(x, lam_s) - xi * float((lam_s - lam) @ (lam_s - lam))
    xs = gap_x_subproblem(prob, x, lam, xi)
    x_part = prob.phi(xs, lam) + xi * float((xs - x) @ (xs - x))
    return y_part - x_part


# ---------------------------------------------------------------------------
# rAPDB (Algorithm 2) with fixed-frequency or adaptive (G_xi) restarts.
# ---------------------------------------------------------------------------

STATUS_OK, STATUS_MAXITER, STATUS_BACKTRACK = 0, 5, 4


@dataclass
class Result:
    x: np.ndarray
    lam: np.ndarray
    iters: int
    trials: int
    restarts: int
    rel_kkt: float
    r_stat: float
    r_feas: float
    obj: float
    status: int
    log: dict = field(default_factory=dict)


def rapdb(prob: Problem, x0=None, lam0=None, p: Params | None = None, keep_iterates: int = 0):
    """rAPDB driver.  Iteration semantics (also followed by the CUDA path):

    at the top of global iteration `it` (iterate z^it):
      1. if kkt_every > 0 and it % kkt_every == 0: stop when rel_kkt <= tol;
      2. stop when it == max_iter;
      3. restart checks: fixed -- when the current run has done restart_period
         iterations; gap -- at it == gap_first store G_ref = G_xi(z^it); at
         it = gap_first + j * gap_every (j >= 1) restart when
         G_xi(candidate) <= q * G_ref and then set G_ref to that value;
         the candidate and the new start point are the last iterate, or the
         weighted average when restart_from_average;
      4. one APDB iteration (backtracking loop, averaging, step rule).
    """
    p = p or default_params()
    x0 = np.zeros(prob.n) if x0 is None else np.asarray(x0, np.float64)
    lam0 = prob.default_lam0() if lam0 is None else np.asarray(lam0, np.float64)
    st = start_routine(prob, x0, lam0, p)
    log: dict = {}
    it = trials = restarts = 0
    status = STATUS_OK
    G_ref = None
    rel = rs = rf = float("nan")
    iterates = []
    while True:
        if p.kkt_every > 0 and it % p.kkt_every == 0:
            rel, rs, rf = kkt_residual(prob, st.x, st.lam)
            if rel <= p.tol:
                break
        if it >= p.max_iter:
            status = STATUS_MAXITER
            break
        if p.restart == "fixed" and st.k == p.restart_period:
            if p.restart_from_average:
                xs, ls = st.x_cum / st.T, st.lam_cum / st.T
            else:
                xs, ls = st.x, st.lam
            st = start_routine(prob, xs, ls, p, st.tau_prev if p.restart_warm_tau else None)
            restarts += 1
        elif p.restart == "gap" and it >= p.gap_first:
            if st.k > 0 and p.restart_from_average:
                xs, ls = st.x_cum / st.T, st.lam_cum / st.T
            else:
                xs, ls = st.x, st.lam
            if it == p.gap_first:
                G_ref = smoothed_gap(prob, xs, ls, p.xi)
                log.setdefault("gap", []).append((it, G_ref, False))
            elif (it - p.gap_first) % p.gap_every == 0:
                G = smoothed_gap(prob, xs, ls, p.xi)
                fire = G <= p.q * G_ref
                log.setdefault("gap", []).append((it, G, bool(fire)))
                if fire:
                    st = start_routine(prob, xs, ls, p, st.tau_prev if p.restart_warm_tau else None)
                    restarts += 1
                    G_ref = G
        try:
            trials += apdb_iteration(prob, st, p, log)
        except BacktrackError:
            status = STATUS_BACKTRACK
            break
        it += 1
        if it <= keep_iterates:
            iterates.append((st.x.copy(), st.lam.copy()))
    if p.kkt_every <= 0 or status != STATUS_OK:
        rel, rs, rf = kkt_residual(prob, st.x, st.lam)
    if keep_iterates:
        log["iterates"] = iterates
    return Result(st.x.copy(), st.lam.copy(), it, trials, restarts, rel, rs, rf,
                  float(prob.f(st.x)), status, log)
