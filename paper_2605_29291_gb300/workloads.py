"""Seeded synthetic QCQP workloads.

This module builds problem data only; it holds none of the solver's arithmetic.
Both the FP64 oracle and the CUDA path consume the arrays it returns, so both
sides solve exactly the same problem: every array is rounded once to float32
here, and those float32 values are the canonical data.

Problem form (the paper's QCQP, Sec. 2.1, with a box as the simple set X):

    min_x 0.5 x'Q_0 x + c_0'x   s.t.  0.5 x'Q_i x + c_i'x + d_i <= 0 (i=1..m),
                                      lb <= x <= ub.

The paper writes q_i for c_i and r_i for d_i.  Arrays returned:

    Q   float32 (M, n, n), symmetric PSD, M = m+1 (Q_0 first) or m when Q_0
        is diagonal (``q0diag`` holds its diagonal) or zero
    c   float32 (m+1, n), row 0 = c_0
    d   float32 (m,)
    lb, ub float32 (n,) (ub may be +inf)
    hyp_a, hyp_beta  optional: the primal set is the box intersected with
        {hyp_a'x = hyp_beta}

Recipes:
  * ``random_qcqp``: Q_0 = A_0'A_0/n + ridge*I and Q_i = A_i'A_i/n with
    A_i in R^{rows x n} i.i.d. N(0,1); c_i ~ N(0,1); d_i = -U[0.1, 1] so that
    x = 0 is strictly feasible; box [-10, 10]^n.
  * ``paper_random_qcqp``: the construction of the paper's random QCQP
    experiment (Sec. 5.1): Q_i = L_i' S_i L_i with L_i orthonormal (QR of a
    Gaussian matrix) and S_i diagonal U[0,100] with its smallest entry set to
    0; q_i ~ N(0, I); -r_i ~ U[0, 1]; box [-10, 10]^n.
  * ``kml_qcqp``: a kernel-matrix-learning QCQP shaped like the paper's
    l2-soft-margin SVM experiment (Sec. 5.2), in epigraph form over
    z = (alpha, s):  min ||alpha||^2 - 2*1'alpha + m*s  s.t.
    alpha'H_i alpha <= s, 0 <= alpha <= C, 0 <= s <= s_max, where
    H_i = diag(b) G_i diag(b) and G_i is a kernel matrix normalised to unit
    diagonal.  Features: two Gaussian classes with means +-0.5*1, unit
    covariance, labels +-1, columns standardised.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

Q0_DENSE, Q0_DIAG, Q0_ZERO = 0, 1, 2


@dataclass
class QCQPData:
    """Canonical float32 problem data (host numpy or device torch tensors)."""

    n: int
    m: int
    Q: object                      # (M, n, n) float32
    c: object                      # (m+1, n) float32
    d: object                      # (m,) float32
    lb: object                     # (n,) float32
    ub: object                     # (n,) float32
    q0_kind: int = Q0_DENSE
    q0diag: object = None          # (n,) float32 when q0_kind == Q0_DIAG
    name: str = ""
    meta: dict = field(default_factory=dict)
    A_eq: object = None            # (p, n) float32: linear equalities A_eq x = b_eq (optional)
    b_eq: object = None            # (p,) float32
    hyp_a: object = None           # (n,) float32: primal set box and {hyp_a'x = hyp_beta} (optional)
    hyp_beta: float = 0.0

    @property
    def M(self) -> int:
        return self.m + 1 if self.q0_kind == Q0_DENSE else self.m

    def numpy(self) -> "QCQPData":
        """Host float32 numpy copy of the data."""
        def h(a):
            if a is None or isinstance(a, np.ndarray):
                return a
            return a.detach().cpu().numpy()
        return QCQPData(self.n, self.m, h(self.Q), h(self.c), h(self.d), h(self.lb),
                        h(self.ub), self.q0_kind, h(self.q0diag), self.name, dict(self.meta),
                        h(self.A_eq), h(self.b_eq), h(self.hyp_a), self.hyp_beta)

    def to(self, device) -> "QCQPData":
        """Copy of the data as contiguous float32 torch tensors on `device`."""
        import torch

        def t(a):
            if a is None:
                return None
            if isinstance(a, np.ndarray):
                a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
            return a.to(device=device, dtype=torch.float32).contiguous()
        return QCQPData(self.n, self.m, t(self.Q), t(self.c), t(self.d), t(self.lb), t(self.ub),
                        self.q0_kind, t(self.q0diag), self.name, dict(self.meta), t(self.A_eq), t(self.b_eq),
                        t(self.hyp_a), self.hyp_beta)

    def dense_q(self) -> np.ndarray:
        """(m+1, n, n) float32 host stack with Q_0 materialised (for the oracle)."""
        h = self.numpy()
        if self.q0_kind == Q0_DENSE:
            return h.Q
        q0 = np.zeros((self.n, self.n), np.float32)
        if self.q0_kind == Q0_DIAG:
            q0[np.arange(self.n), np.arange(self.n)] = h.q0diag
        return np.concatenate([q0[None], h.Q], axis=0)


def _sym32(q64: np.ndarray) -> np.ndarray:
    """Round to float32 and make exactly symmetric ((a+b)/2 is order-free)."""
    q = q64.astype(np.float32)
    return ((q + np.swapaxes(q, -1, -2)) * np.float32(0.5)).astype(np.float32)


def random_qcqp(n: int, m: int, rows: int | None = None, seed: int = 0,
                ridge: float = 1e-2, box: float = 10.0, device=None) -> QCQPData:
    """Gram-matrix QCQP: Q_0 = A_0'A_0/n + ridge*I, Q_i = A_i'A_i/n.

    ``rows`` defaults to n//2 (A_i in R^{n/2 x n}).  With ``device`` set to a
    CUDA device the Gram products run there in float64 through torch and the
    returned arrays stay on that device (used for the multi-GB stacks).
    """
    rows = n // 2 if rows is None else rows
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((m + 1, n)).astype(np.float32)
    d = (-rng.uniform(0.1, 1.0, size=m)).astype(np.float32)
    lb = np.full(n, -box, np.float32)
    ub = np.full(n, box, np.float32)
    if device is None:
        Q = np.empty((m + 1, n, n), np.float32)
        for i in range(m + 1):
            A = rng.standard_normal((rows, n))
            G = A.T @ A / n
            if i == 0:
                G[np.arange(n), np.arange(n)] += ridge
            Q[i] = _sym32(G)
        return QCQPData(n, m, Q, c, d, lb, ub, Q0_DENSE, None,
                        f"random_qcqp(n={n},m={m},rows={rows},seed={seed})")
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(rng.integers(0, 2**62)))
    Q = torch.empty((m + 1, n, n), dtype=torch.float32, device=device)
    eye = torch.eye(n, dtype=torch.float64, device=device)
    for i in range(m + 1):
        A = torch.randn((rows, n), generator=gen, dtype=torch.float64, device=device)
        G = A.T @ A / n
        if i == 0:
            G += ridge * eye
        g32 = G.to(torch.float32)
        Q[i] = (g32 + g32.T) * 0.5
        del A, G, g32
    t = lambda a: torch.from_numpy(a).to(device)
    return QCQPData(n, m, Q, t(c), t(d), t(lb), t(ub), Q0_DENSE, None,
                    f"random_qcqp(n={n},m={m},rows={rows},seed={seed},torch)")


def paper_random_qcqp(n: int, m: int, seed: int = 0, box: float = 10.0) -> QCQPData:
    """Random QCQP built as in the paper's first experiment (Sec. 5.1)."""
    rng = np.random.default_rng(seed)
    Q = np.empty((m + 1, n, n), np.float32)
    for i in range(m + 1):
        L, _ = np.linalg.qr(rng.standard_normal((n, n)))
        s = rng.uniform(0.0, 100.0, size=n)
        s[np.argmin(s)] = 0.0
        Q[i] = _sym32((L * s) @ L.T)
    c = rng.standard_normal((m + 1, n)).astype(np.float32)
    d = (-rng.uniform(0.0, 1.0, size=m)).astype(np.float32)
    lb = np.full(n, -box, np.float32)
    ub = np.full(n, box, np.float32)
    return QCQPData(n, m, Q, c, d, lb, ub, Q0_DENSE, None,
                    f"paper_random_qcqp(n={n},m={m},seed={seed})")


def kml_features(n: int, dfeat: int, seed: int):
    """Two Gaussian classes (means +-0.5*1, unit covariance), n/2 each,
    labels +-1, feature columns standardised."""
    rng = np.random.default_rng(seed)
    b = np.ones(n)
    b[n // 2:] = -1.0
    a = rng.standard_normal((n, dfeat)) + 0.5 * b[:, None]
    a = (a - a.mean(axis=0)) / a.std(axis=0)
    return a, b


def kml_kernel_specs(m: int) -> list:
    """Kernel list: the paper's three kernels (poly 2, RBF 0.1, linear) for
    m=3, the 8-kernel set (RBF 0.1,0.5,1,2,5; poly 2,3; linear) for m=8,
    otherwise m-4 log-spaced RBF widths in [0.05, 10], poly 2..4, linear."""
    if m == 3:
        return [("poly", 2), ("rbf", 0.1), ("linear", None)]
    if m == 8:
        return [("rbf", w) for w in (0.1, 0.5, 1.0, 2.0, 5.0)] + \
               [("poly", 2), ("poly", 3), ("linear", None)]
    nr = m - 4
    widths = np.exp(np.linspace(math.log(0.05), math.log(10.0), nr)) if nr > 1 else [1.0]
    return [("rbf", float(w)) for w in widths] + [("poly", 2), ("poly", 3), ("poly", 4),
                                                 ("linear", None)]


def _kml_h(A, B, kind, par, use_torch):
    """H(K) = diag(b) K diag(b) of one kernel, K normalised to a unit
    diagonal (float64)."""
    ip = A @ A.T
    if kind == "rbf":
        sq = (A * A).sum(1)
        dist2 = sq[:, None] + sq[None, :] - 2.0 * ip
        dist2 = dist2.clamp(min=0.0) if use_torch else np.maximum(dist2, 0.0)
        K = (-0.5 * dist2 / par).exp() if use_torch else np.exp(-0.5 * dist2 / par)
    elif kind == "poly":
        K = (1.0 + ip) ** par
    else:
        K = ip
    dg = K.diagonal().clone() if use_torch else K.diagonal().copy()
    dg = dg.clamp(min=1e-300) if use_torch else np.maximum(dg, 1e-300)
    s = dg.rsqrt() if use_torch else 1.0 / np.sqrt(dg)
    return K * (s * B)[:, None] * (s * B)[None, :]


def kml_qcqp(n: int, dfeat: int, m: int, seed: int = 0, C: float = 1.0,
             lam: float = 1.0, device=None) -> QCQPData:
    """Epigraph QCQP of the kernel-matrix-learning min-max problem.

    Variables z = (alpha, s) in R^{n+1}.  Q_0 = diag(2*lam*1_n, 0) (stored as
    a diagonal), c_0 = (-2*1_n, m); Q_i = blkdiag(2 H_i, 0), c_i = (0, -1),
    d_i = 0; box 0 <= alpha <= C, 0 <= s <= s_max with
    s_max = max_i sum_jk |H_i,jk| (alpha'H_i alpha cannot exceed it on the box).
    """
    a, b = kml_features(n, dfeat, seed)
    specs = kml_kernel_specs(m)
    assert len(specs) == m
    N = n + 1
    use_torch = device is not None
    if use_torch:
        import torch
        A = torch.from_numpy(a).to(device)
        B = torch.from_numpy(b).to(device)
        Q = torch.zeros((m, N, N), dtype=torch.float32, device=device)
    else:
        A, B = a, b
        Q = np.zeros((m, N, N), np.float32)
    smax = 0.0
    for i, (kind, par) in enumerate(specs):
        H = _kml_h(A, B, kind, par, use_torch)
        smax = max(smax, float(H.abs().sum()) if use_torch else float(np.abs(H).sum()))
        if use_torch:
            h32 = (2.0 * H).to(torch.float32)
            Q[i, :n, :n] = (h32 + h32.T) * 0.5
        else:
            Q[i, :n, :n] = _sym32(2.0 * H)
        del H
    c = np.zeros((m + 1, N), np.float32)
    c[0, :n] = -2.0
    c[0, n] = float(m)
    c[1:, n] = -1.0
    d = np.zeros(m, np.float32)
    lb = np.zeros(N, np.float32)
    ub = np.full(N, C, np.float32)
    ub[n] = np.float32(smax)
    q0diag = np.zeros(N, np.float32)
    q0diag[:n] = 2.0 * lam
    name = f"kml_qcqp(n={n},d={dfeat},m={m},seed={seed})"
    if use_torch:
        t = lambda v: torch.from_numpy(v).to(device)
        return QCQPData(N, m, Q, t(c), t(d), t(lb), t(ub), Q0_DIAG, t(q0diag), name)
    return QCQPData(N, m, Q, c, d, lb, ub, Q0_DIAG, q0diag, name)


def kml_minmax(n: int, dfeat: int, m: int, seed: int = 0, C: float = 1.0, lam: float = 1.0,
               device=None, bias: bool = False, primal_set: bool = False) -> QCQPData:
    """The kernel-learning min-max problem as the paper states it (Sec. 5.2,
    eq. min-max-KML), with the dual on the simplex:

        min_{0 <= x <= C} max_{y in Delta_m}  lam ||x||^2 - 2 1'x
                                              + sum_i (c / r_i) y_i x'H(K_i)x,

    r_i = trace(K_i) = n (unit-diagonal kernels), c = sum_i r_i, so
    c / r_i = m.  As QCQP data: Q_0 = 2 lam I (diagonal), c_0 = -2 1,
    Q_i = 2 m H(K_i), c_i = 0, d_i = 0; meta['dual_radius'] = 1.  With
    bias=True the paper's equality b'x = 0 (b the labels) is attached as
    A_eq = b', b_eq = 0 (a constraint with a free multiplier).  With
    primal_set=True the primal set is the paper's own, {x >= 0, b'x = 0}:
    lb = 0, ub = +inf and the hyperplane hyp_a = b, hyp_beta = 0 (no upper
    bound C).  Same features and kernels as kml_qcqp."""
    a, b = kml_features(n, dfeat, seed)
    specs = kml_kernel_specs(m)
    assert len(specs) == m
    use_torch = device is not None
    if use_torch:
        import torch
        A = torch.from_numpy(a).to(device)
        B = torch.from_numpy(b).to(device)
        Q = torch.zeros((m, n, n), dtype=torch.float32, device=device)
    else:
        A, B = a, b
        Q = np.zeros((m, n, n), np.float32)
    for i, (kind, par) in enumerate(specs):
        H = _kml_h(A, B, kind, par, use_torch)
        if use_torch:
            h32 = (2.0 * m * H).to(torch.float32)
            Q[i] = (h32 + h32.T) * 0.5
        else:
            Q[i] = _sym32(2.0 * m * H)
        del H
    c = np.zeros((m + 1, n), np.float32)
    c[0] = -2.0
    d = np.zeros(m, np.float32)
    lb = np.zeros(n, np.float32)
    ub = np.full(n, np.inf if primal_set else C, np.float32)
    q0diag = np.full(n, 2.0 * lam, np.float32)
    name = (f"kml_minmax(n={n},d={dfeat},m={m},seed={seed}{',bias' if bias else ''}"
            f"{',primal_set' if primal_set else ''})")
    meta = {"dual_radius": 1.0}
    A_eq = b.astype(np.float32).reshape(1, n) if bias else None
    b_eq = np.zeros(1, np.float32) if bias else None
    hyp_a = b.astype(np.float32) if primal_set else None
    if use_torch:
        t = lambda v: None if v is None else torch.from_numpy(v).to(device)
        return QCQPData(n, m, Q, t(c), t(d), t(lb), t(ub), Q0_DIAG, t(q0diag), name, meta, t(A_eq), t(b_eq),
                        t(hyp_a), 0.0)
    return QCQPData(n, m, Q, c, d, lb, ub, Q0_DIAG, q0diag, name, meta, A_eq, b_eq, hyp_a, 0.0)


def ball_qcqp(cvec: np.ndarray, rho: float, box: float = 10.0) -> QCQPData:
    """min c'x s.t. ||x||^2 <= rho^2 inside a box: Q_0 = 0, Q_1 = 2I,
    c_1 = 0, d_1 = -rho^2."""
    n = cvec.shape[0]
    Q = np.zeros((2, n, n), np.float32)
    Q[1] = 2.0 * np.eye(n, dtype=np.float32)
    c = np.zeros((2, n), np.float32)
    c[0] = cvec
    d = np.array([-rho * rho], np.float32)
    lb = np.full(n, -box, np.float32)
    ub = np.full(n, box, np.float32)
    return QCQPData(n, 1, Q, c, d, lb, ub, Q0_DENSE, None, f"ball(n={n},rho={rho})")


def batched_random_qcqp(count: int, seed: int = 0, n_lo: int = 64, n_hi: int = 1024,
                        m_lo: int = 2, m_hi: int = 32) -> list:
    """``count`` independent Gram-matrix QCQPs: n = round(n_lo*(n_hi/n_lo)^U)
    (log-uniform), m ~ U{m_lo..m_hi}, A_i in R^{floor(n/2) x n}."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(round(n_lo * (n_hi / n_lo) ** rng.uniform()))
        m = int(rng.integers(m_lo, m_hi + 1))
        out.append(random_qcqp(n, m, rows=n // 2, seed=int(rng.integers(0, 2**31))))
    return out


# Named workloads: the small oracle-sized case and the multi-GB cases.
def config(name: str, device=None, seed: int = 0) -> QCQPData:
    if name == "C1":
        return random_qcqp(200, 10, rows=100, seed=seed)
    if name == "C2":
        return random_qcqp(4096, 50, rows=2048, seed=seed, device=device)
    if name == "C3":
        return kml_qcqp(5000, 20, 8, seed=seed, device=device)
    if name == "C5":
        return kml_qcqp(16000, 32, 20, seed=seed, device=device)
    if name == "C3m":
        return kml_minmax(5000, 20, 8, seed=seed, device=device)
    if name == "C5m":
        return kml_minmax(16000, 32, 20, seed=seed, device=device)
    if name == "C3mb":
        return kml_minmax(5000, 20, 8, seed=seed, device=device, bias=True)
    if name == "C5mb":
        return kml_minmax(16000, 32, 20, seed=seed, device=device, bias=True)
    if name == "C3mx":       # the paper's primal set {x >= 0, b'x = 0}
        return kml_minmax(5000, 20, 8, seed=seed, device=device, primal_set=True)
    if name == "C5mx":
        return kml_minmax(16000, 32, 20, seed=seed, device=device, primal_set=True)
    if name == "P1":
        return paper_random_qcqp(1000, 10, seed=seed)
    raise KeyError(name)
