"""Oracle: Algorithm 1 (point-oriented Pareto computation) and its two
projections.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The norm is ||v|| = sqrt(v^T M v) for a symmetric positive-definite M
(Sec. 3.3 prints <v, v> without the square root; the square root is the
reading taken, default M = I).  With the Cholesky factor M = R^T R both
projections become Euclidean minimum-norm problems in y = R(x - t), and each
is solved by a finite active-set method whose last step is an exact dense
linear solve, so the result is exact up to rounding (no iteration tolerance
enters the answer):

  * the outer bound t_down (projection onto the polyhedron of the half-spaces
    {z : w_l . z <= w_l . r_l}) is a least-distance program
    min ||y|| s.t. G y >= h, solved through non-negative least squares
    (Lawson and Hanson, "Solving Least Squares Problems", 1974, Ch. 23,
    Algorithms NNLS and LDP);
  * the inner bound t_up (projection onto down(conv Phi) = conv Phi + R^n_-)
    is the minimum-norm point of conv{R(phi_k - t)} + cone{-R e_i}, found
    with Wolfe's algorithm ("Finding the nearest point in a polytope",
    Math. Programming 11, 1976) extended to the rays of the cone: the
    corral's affine minimiser is an exact KKT solve, and the convex weights
    of the points are the synthesis weights lambda (Sec. 3.3).

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


def mnorm(v, M):
    return float(np.sqrt(v @ M @ v))


def _chol_upper(M):
    """R with M = R^T R (R upper triangular)."""
    return np.linalg.cholesky(np.asarray(M, np.float64)).T


# ------------------------------------------------ non-negative least squares


def nnls(E, f, max_iter=None):
    """min ||E u - f||_2 subject to u >= 0 (Lawson-Hanson, Ch. 23, NNLS).

    Active-set method: the passive set P holds the free (positive)
    coordinates; each outer step frees the coordinate with the largest
    positive gradient w = E^T (f - E u), each inner step solves the
    unconstrained least-squares problem on P and, where that leaves P's
    coordinates non-positive, moves back to the boundary and drops them.
    The returned u is the exact least-squares solution on the final P."""
    E = np.asarray(E, np.float64)
    f = np.asarray(f, np.float64)
    m = E.shape[1]
    u = np.zeros(m)
    passive = np.zeros(m, bool)
    scale = max(np.abs(E).max(initial=0.0), 1e-300) * max(np.abs(f).max(initial=0.0), 1.0)
    tol = 1e-13 * scale * max(E.shape)
    max_iter = 30 * (m + 1) if max_iter is None else max_iter
    for _ in range(max_iter):
        w = E.T @ (f - E @ u)
        cand = np.where(~passive & (w > tol))[0]
        if len(cand) == 0:
            return u
        passive[cand[np.argmax(w[cand])]] = True
        while True:
            idx = np.where(passive)[0]
            z = np.zeros(m)
            z[idx] = np.linalg.lstsq(E[:, idx], f, rcond=None)[0]
            if np.all(z[idx] > 0):
                u = z
                break
            neg = idx[z[idx] <= 0]
            alpha = np.min(u[neg] / (u[neg] - z[neg]))
            u = u + alpha * (z - u)
            drop = idx[u[idx] <= 1e-15 * max(1.0, np.abs(u).max())]
            if len(drop) == 0:  # the blocking coordinate itself
                drop = neg[np.argmin(u[neg] / (u[neg] - z[neg]))][None]
            passive[drop] = False
            u[drop] = 0.0
    raise RuntimeError("nnls: iteration limit")


def ldp(G, h):
    """min ||x||_2 subject to G x >= h (Lawson-Hanson, Ch. 23, LDP).

    With E = [G^T; h^T] and f = e_{n+1}, the NNLS residual r = E u - f is
    zero iff the constraints are inconsistent; otherwise x = -r[:n] / r[n].
    Returns None when they are inconsistent."""
    G = np.atleast_2d(np.asarray(G, np.float64))
    h = np.asarray(h, np.float64)
    m, n = G.shape
    E = np.vstack([G.T, h[None, :]])
    f = np.zeros(n + 1)
    f[n] = 1.0
    u = nnls(E, f)
    r = E @ u - f
    if np.linalg.norm(r) <= 1e-13:
        return None
    return -r[:n] / r[n]


# ------------------------------------------------------------ the projections


def project_halfspaces(t, A, b, M):
    """argmin_z ||t - z||_M  s.t.  A z <= b   (Algorithm 1, the t_down step).

    With y = R (z - t): A z <= b  <=>  (-A R^-1) y >= A t - b, a least-distance
    program in y."""
    t = np.asarray(t, np.float64)
    A = np.atleast_2d(np.asarray(A, np.float64))
    b = np.asarray(b, np.float64)
    h = A @ t - b
    if np.all(h <= 0):
        return t.copy()
    R = _chol_upper(M)
    G = -np.linalg.solve(R.T, A.T).T  # -A R^-1
    y = ldp(G, h)
    if y is None:
        raise ValueError("project_halfspaces: the half-spaces have no common point")
    return t + np.linalg.solve(R, y)


def min_norm_point(P, Q=None, max_iter=None):
    """The point of least Euclidean norm in conv{P_k} + cone{Q_i} (rows of P
    and Q), with its coefficients: y = lam @ P + rho @ Q, lam on the simplex,
    rho >= 0.  Wolfe's algorithm with rays: the corral S (generators with
    positive coefficients, at least one point) is grown by the generator that
    most violates the optimality conditions (P_k . y >= y . y for every point,
    Q_i . y >= 0 for every ray) and shrunk, by the minor cycles, until its
    affine minimiser has positive coefficients."""
    P = np.atleast_2d(np.asarray(P, np.float64))
    m, n = P.shape
    Q = np.zeros((0, n)) if Q is None else np.atleast_2d(np.asarray(Q, np.float64)).reshape(-1, n)
    gens = np.vstack([P, Q])
    is_pt = np.arange(len(gens)) < m
    scale = max(np.abs(gens).max(initial=0.0), 1e-300)
    k0 = int(np.argmin(np.einsum("ij,ij->i", P, P)))
    S = [k0]
    coef = np.array([1.0])
    y = P[k0].copy()
    max_iter = 50 * (len(gens) + n + 1) if max_iter is None else max_iter
    for _ in range(max_iter):
        yy = y @ y
        test = gens @ y - np.where(is_pt, yy, 0.0)
        test[S] = np.inf
        j = int(np.argmin(test))
        # rounding in y . g is about 1e-16 |g| (|y| + |g|): stop once nothing
        # improves beyond it
        if test[j] >= -1e-13 * scale * (np.sqrt(yy) + 0.1 * scale) * max(n, 1):
            break
        S.append(j)
        coef = np.append(coef, 0.0)
        for _ in range(max_iter):
            Gs = gens[S]
            e = is_pt[S].astype(np.float64)
            s = len(S)
            K = np.zeros((s + 1, s + 1))
            K[:s, :s] = Gs @ Gs.T
            K[:s, s] = e
            K[s, :s] = e
            rhs = np.zeros(s + 1)
            rhs[s] = 1.0
            c = np.linalg.lstsq(K, rhs, rcond=None)[0][:s]
            if np.all(c > 0):
                coef = c
                break
            neg = np.where(c <= 0)[0]
            theta = np.min(coef[neg] / (coef[neg] - c[neg]))
            coef = coef + theta * (c - coef)
            keep = coef > 1e-15
            if np.all(keep):  # the blocking coefficient itself
                keep[neg[np.argmin(coef[neg] / (coef[neg] - c[neg]))]] = False
            if not np.any(keep & is_pt[S]):  # at least one point stays in the corral
                keep[int(np.argmax(np.where(is_pt[S], coef, -np.inf)))] = True
            S = [g for g, k in zip(S, keep) if k]
            coef = coef[keep]
            coef[is_pt[S]] /= coef[is_pt[S]].sum()
        y = coef @ gens[S]
        if j not in S:  # the new generator left the corral again: no progress beyond rounding
            break
    else:
        raise RuntimeError("min_norm_point: iteration limit")
    lam = np.zeros(m)
    rho = np.zeros(len(Q))
    for g, cg in zip(S, coef):
        if g < m:
            lam[g] = cg
        else:
            rho[g - m] = cg
    return y, lam, rho


def project_down_hull(t, Phi, M, return_lambda=False):
    """argmin_x ||t - x||_M over x in down(conv Phi) (Algorithm 1, the t_up
    step): down(conv Phi) = conv Phi + R^n_-, so with y = R (x - t) the
    projection is the minimum-norm point of conv{R(phi_k - t)} + cone{-R e_i}.
    With return_lambda, also the convex weights lam with x <= Phi^T lam."""
    t = np.asarray(t, np.float64)
    Phi = np.atleast_2d(np.asarray(Phi, np.float64))
    R = _chol_upper(M)
    P = (Phi - t[None, :]) @ R.T
    Q = -R.T  # rows: -R e_i
    y, lam, _ = min_norm_point(P, Q)
    x = t + np.linalg.solve(R, y)
    return (x, lam) if return_lambda else x


# ---------------------------------------------------------------- Algorithm 1


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
    lam = None
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
        t_up, lam = project_down_hull(t, np.array(Phi), M, return_lambda=True)
        hist.append({"w": w.copy(), "r": r, "t_up": t_up.copy(), "t_dn": t_dn.copy()})
        if mnorm(t_dn - t_up, M) <= eps or it >= max_iter:
            break
        d = M @ (t - t_up)
        w = d / np.abs(d).sum()
    return {"feasible": not moved, "t_up": t_up, "t_dn": t_dn, "iterations": it, "history": hist,
            "converged": mnorm(t_dn - t_up, M) <= eps, "lambda": lam}
