"""Oracle: Algorithm 1 (point-oriented Pareto computation) and its two
projections.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The norm is ||v|| = sqrt(v^T M v) for a symmetric positive-definite M
(Sec. 3.3 prints <v, v> without the square root; the square root is the
reading taken, default M = I).  Both projections are small convex QPs and are
handed to scipy's SLSQP as a library step.

Reading of the loop (Algorithm 1 and the worked example of Fig. 2): the
supporting point for w is added to Phi and Lambda, t_dn is projected when
w.r < w.t_dn, then t_up is refreshed from the enlarged Phi and the stopping
test ||t_dn - t_up|| <= eps is made on the refreshed t_up; otherwise the next
direction is w = M(t - t_up) / ||M(t - t_up)||_1.  The first direction is
e_1.  This is the paper's sequence of operations with the loop test placed
after the refresh, which is how the example counts its iterations.
"""

from __future__ import annotations

import numpy as np
from scipy.optimize import minimize


def mnorm(v, M):
    return float(np.sqrt(v @ M @ v))


def project_halfspaces(t, A, b, M):
    """argmin_z ||t - z||_M  s.t.  A z <= b   (Algorithm 1, the t_down step)."""
    t = np.asarray(t, np.float64)
    A = np.atleast_2d(np.asarray(A, np.float64))
    b = np.asarray(b, np.float64)
    if np.all(A @ t <= b):
        return t.copy()

    def f(z):
        d = z - t
        return 0.5 * d @ M @ d, M @ d

    cons = [{"type": "ineq", "fun": lambda z: b - A @ z, "jac": lambda z: -A}]
    res = minimize(f, t.copy(), jac=True, constraints=cons, method="SLSQP",
                   options={"ftol": 1e-16, "maxiter": 5000})
    return res.x


def project_down_hull(t, Phi, M):
    """argmin_x ||t - x||_M over x in down(conv Phi) (Algorithm 1, the t_up
    step): x <= sum_k lam_k phi_k with lam on the simplex."""
    t = np.asarray(t, np.float64)
    Phi = np.atleast_2d(np.asarray(Phi, np.float64))  # [m][n]
    m, n = Phi.shape
    # t itself if some convex combination dominates it (checked by the QP too)
    lam0 = np.full(m, 1.0 / m)
    x0 = np.minimum(t, Phi.T @ lam0)
    v0 = np.concatenate([x0, lam0])

    def f(v):
        d = v[:n] - t
        g = np.zeros(n + m)
        g[:n] = M @ d
        return 0.5 * d @ M @ d, g

    Jin = np.hstack([-np.eye(n), Phi.T])
    cons = [
        {"type": "ineq", "fun": lambda v: Phi.T @ v[n:] - v[:n], "jac": lambda v: Jin},
        {"type": "eq", "fun": lambda v: np.array([v[n:].sum() - 1.0]),
         "jac": lambda v: np.concatenate([np.zeros(n), np.ones(m)])[None, :]},
    ]
    bounds = [(None, None)] * n + [(0.0, None)] * m
    res = minimize(f, v0, jac=True, constraints=cons, bounds=bounds, method="SLSQP",
                   options={"ftol": 1e-16, "maxiter": 5000})
    x = res.x[:n]
    return np.minimum(x, t)


def alg1(supporting_point, t, M=None, eps=1e-6, max_iter=64, verify_only=False):
    """Algorithm 1.  supporting_point(w) -> r.  Returns a dict with the
    verdict (t_dn == t, Cor. (ii)), t_up, t_dn and the (w, r) history.

    verify_only: the verification-only setting of Sec. 5 (Experiment 2),
    where the outer-bound update is replaced by a break: the loop stops, with
    the verdict "not achievable", at the first point with w.r < w.t_dn."""
    t = np.asarray(t, np.float64)
    n = len(t)
    M = np.eye(n) if M is None else np.asarray(M, np.float64)
    w = np.zeros(n)
    w[0] = 1.0
    Phi, Lam = [], []
    t_dn = t.copy()
    moved = False
    t_up = None
    hist = []
    it = 0
    while True:
        r = np.asarray(supporting_point(w), np.float64)
        it += 1
        Phi.append(r)
        Lam.append((w.copy(), r))
        if w @ r < w @ t_dn:
            if verify_only:
                hist.append({"w": w.copy(), "r": r, "t_up": t_up, "t_dn": t_dn.copy()})
                t_up = t_up if t_up is not None else np.full(n, -np.inf)
                return {"feasible": False, "t_up": t_up, "t_dn": t_dn, "iterations": it, "history": hist,
                        "converged": True, "decided": True}
            A = np.array([wl for wl, _ in Lam])
            b = np.array([wl @ rl for wl, rl in Lam])
            t_dn = project_halfspaces(t, A, b, M)
            moved = True
        t_up = project_down_hull(t, np.array(Phi), M)
        hist.append({"w": w.copy(), "r": r, "t_up": t_up.copy(), "t_dn": t_dn.copy()})
        if mnorm(t_dn - t_up, M) <= eps or it >= max_iter:
            break
        d = M @ (t - t_up)
        w = d / np.abs(d).sum()
    return {"feasible": not moved, "t_up": t_up, "t_dn": t_dn, "iterations": it, "history": hist,
            "converged": mnorm(t_dn - t_up, M) <= eps}
