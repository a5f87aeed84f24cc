"""Oracle: the MORAP problem as one linear program, solved by a hand-written
dense simplex -- a second, independent decision of "is threshold t
achievable?" for tiny instances.  TEST INFRASTRUCTURE ONLY (see
oracle/__init__.py).

Sec. 3 (the discussion after Def. 1 and Fig. 1) notes that MORAP can be
written as a multi-objective LP with the construction that underlies
multi-objective verification of MDPs.  The achievable set is the downward
closure of the convex hull, over the task assignments f, of the points that
schedulers of the assigned products reach.  With occupation measures that
is linear:

  variables   mu[i][j] >= 0, the probability that agent i does task j, and
              per pair (i, j) and transient product state s
              z_ij(s, a) >= 0 (expected number of times action a is taken in
              s, already multiplied by mu[i][j]) and e_ij(s) >= 0 (mass that
              stays in s forever through a zero-reward self-loop);
  flow        sum_a z(s, a) + e(s) - sum_{s', a'} P(s | s', a') z(s', a')
                  = mu[i][j] [s = initial state]           for every s;
  objectives  sum_j sum rho_i z_ij  >= c_i          (costs),
              sum_i sum rho_{j+|I|} z_ij >= p_j     (probability, the
              pre-sink reward of Sec. 3.1);
  marginals   sum_j mu[i][j] <= 1, sum_i mu[i][j] <= 1.

By Lemma 2 (Birkhoff) the doubly substochastic matrices mu are exactly the
marginals of random assignments of the padded square problem, so the system
describes the achievable set of Def. 1.

t is achievable iff this system has a solution.  Zero-reward end
components other than self-loops are not modelled (the function checks that
there are none); the instances used have zero cost only on "stay".

The simplex is phase 1 of the textbook tableau method on A x = b, x >= 0,
b >= 0, with artificial variables: Dantzig's entering rule and the minimum
ratio test with the lexicographic tie rule, which cannot cycle.
"""

from __future__ import annotations

import numpy as np


def simplex_phase1(A, b, tol=1e-9, max_pivots=200_000, refresh=50):
    """Decide whether {x >= 0 : A x = b} is non-empty.  Returns
    (feasible, x, infeasibility), infeasibility = the phase-1 optimum (the
    smallest total violation, 0 when feasible).  Every `refresh` pivots the
    tableau is recomputed from the original data and the current basis
    (B^-1 by a dense solve), so that rounding does not accumulate."""
    A = np.array(A, np.float64)
    b = np.array(b, np.float64)
    m, n = A.shape
    neg = b < 0
    A[neg] *= -1.0
    b[neg] *= -1.0
    aug = np.hstack([A, np.eye(m), b[:, None]])  # [A | artificials | b]
    cost = np.concatenate([np.zeros(n), np.ones(m)])  # minimise the sum of the artificials
    basis = np.arange(n, n + m)
    T = np.zeros((m + 1, n + m + 1))

    def rebuild():
        T[:m] = np.linalg.solve(aug[:, basis], aug)
        T[m] = np.concatenate([cost, [0.0]]) - cost[basis] @ T[:m]

    rebuild()
    piv_tol = 1e-9
    for k in range(max_pivots):
        if k and k % refresh == 0:
            rebuild()
        red = T[m, :n + m]
        e = int(np.argmin(red))
        if red[e] >= -tol:
            break
        col = T[:m, e]
        rows = np.nonzero(col > piv_tol)[0]
        if len(rows) == 0:  # cannot happen in phase 1 (bounded below by 0) but for rounding
            T[m, e] = 0.0
            continue
        rhs = np.maximum(T[rows, -1], 0.0)
        ratios = rhs / col[rows]
        best = ratios.min()
        ties = rows[ratios <= best + 1e-12 * max(1.0, abs(best))]
        if len(ties) > 1:
            # lexicographic rule: the smallest row of [ratio | B^-1 row / pivot]
            # (no basis repeats, so the method terminates)
            R = T[ties, n:n + m] / col[ties, None]
            order = np.lexsort(R.T[::-1])
            r = int(ties[order[0]])
        else:
            r = int(ties[0])
        T[r] /= T[r, e]
        others = np.arange(m + 1) != r
        T[others] -= np.outer(T[others, e], T[r])
        basis[r] = e
    else:
        raise RuntimeError("simplex: pivot limit reached")
    rebuild()
    x = np.zeros(n + m)
    x[basis] = np.maximum(T[:m, -1], 0.0)
    infeas = float(x[n:].sum())
    feasible = infeas <= tol * max(1.0, float(np.abs(b).max(initial=0.0)))
    return bool(feasible), x[:n], infeas


def _pair_block(prod):
    """The flow structure of one product: transient states 0..n-2 (the last
    state is DONE), the variables (kind, s, a) with kind 'z' (a state-action)
    or 'e' (stay forever), and the columns of the flow matrix."""
    n_tr = prod.n - 1
    rho_c = prod.reward_cost()
    rho_p = prod.reward_prob()
    cols = []  # (kind, s, row, flow dict {state: coeff}, rho_c, rho_p)
    zero_edges = {}
    for s in range(n_tr):
        has_exit = False
        for a_row in range(prod.state_ptr[s], prod.state_ptr[s + 1]):
            succ = {}
            for t in range(prod.sa_ptr[a_row], prod.sa_ptr[a_row + 1]):
                u = int(prod.col[t])
                succ[u] = succ.get(u, 0.0) + float(prod.prob[t])
            zero_reward = rho_c[a_row] == 0.0 and rho_p[a_row] == 0.0
            if zero_reward and succ == {s: 1.0}:
                has_exit = True  # a free self-loop: replaced by the exit variable
                continue
            if succ.get(s, 0.0) >= 1.0 and rho_p[a_row] > 0.0:
                raise ValueError("a self-loop that earns probability reward (not reward-finite)")
            flow = {s: 1.0}
            for u, p in succ.items():
                if u < n_tr:
                    flow[u] = flow.get(u, 0.0) - p
            cols.append(("z", s, a_row, flow, float(rho_c[a_row]), float(rho_p[a_row])))
            if zero_reward:
                zero_edges.setdefault(s, set()).update(u for u in succ if u < n_tr and u != s)
        if has_exit:
            cols.append(("e", s, -1, {s: 1.0}, 0.0, 0.0))
    _check_no_zero_reward_cycle(n_tr, zero_edges)
    return cols


def _check_no_zero_reward_cycle(n, edges):
    colour = np.zeros(n, np.int8)  # 0 new, 1 on the stack, 2 done
    for root in range(n):
        if colour[root]:
            continue
        stack = [(root, iter(edges.get(root, ())))]
        colour[root] = 1
        while stack:
            v, it = stack[-1]
            u = next(it, None)
            if u is None:
                colour[v] = 2
                stack.pop()
            elif colour[u] == 1:
                raise ValueError("a zero-reward cycle other than a self-loop: not modelled by this LP")
            elif colour[u] == 0:
                colour[u] = 1
                stack.append((u, iter(edges.get(u, ()))))


def morap_feasible(prods, t, tol=1e-9, max_pivots=200_000):
    """Is threshold t = (c_1..c_|I|, p_1..p_|J|) achievable for the products
    prods[i][j]?  Returns (feasible, details) with the phase-1 infeasibility
    and, when feasible, the marginals mu and each pair's point.

    The random assignment enters through its marginals mu[i][j] = P(agent i
    does task j): by Lemma 2 (Birkhoff) the marginals of distributions over
    (padded) assignments are exactly the doubly substochastic matrices, so
    the LP carries one occupation-measure block per pair, scaled by mu[i][j],
    and the constraints sum_j mu[i][j] <= 1, sum_i mu[i][j] <= 1."""
    nI, nJ = len(prods), len(prods[0])
    t = np.asarray(t, np.float64)
    pairs = [(i, j) for i in range(nI) for j in range(nJ) if prods[i][j].init != prods[i][j].n - 1]
    blocks = {(i, j): _pair_block(prods[i][j]) for (i, j) in pairs}
    n_mu = nI * nJ
    flow_rows = [(i, j, s) for (i, j) in pairs for s in range(prods[i][j].n - 1)]
    row_of = {key: r for r, key in enumerate(flow_rows)}
    col_of = [(i, j, c) for (i, j) in pairs for c in blocks[(i, j)]]
    n_z = len(col_of)
    n_obj = nI + nJ
    n_marg = nI + nJ
    # columns: mu, z / e, objective slacks, marginal slacks
    n_var = n_mu + n_z + n_obj + n_marg
    r_obj = len(flow_rows)
    r_marg = r_obj + n_obj
    m = r_marg + n_marg
    A = np.zeros((m, n_var))
    bvec = np.zeros(m)
    for k, (i, j, (kind, s, a_row, flow, rc, rp)) in enumerate(col_of):
        col = n_mu + k
        for u, coef in flow.items():
            A[row_of[(i, j, u)], col] += coef
        A[r_obj + i, col] = rc
        A[r_obj + nI + j, col] = rp
    for (i, j) in pairs:
        A[row_of[(i, j, prods[i][j].init)], i * nJ + j] -= 1.0
    for i in range(nI):
        for j in range(nJ):
            A[r_marg + i, i * nJ + j] = 1.0  # agent i does at most one task
            A[r_marg + nI + j, i * nJ + j] = 1.0  # task j is done by at most one agent
    for q in range(n_obj):
        A[r_obj + q, n_mu + n_z + q] = -1.0  # objective - slack = threshold
        bvec[r_obj + q] = t[q]
    for q in range(n_marg):
        A[r_marg + q, n_mu + n_z + n_obj + q] = 1.0  # marginal + slack = 1
        bvec[r_marg + q] = 1.0
    feasible, x, infeas = simplex_phase1(A, bvec, tol=tol, max_pivots=max_pivots)
    details = {"infeasibility": infeas, "variables": n_var, "constraints": m}
    if feasible:
        details["mu"] = x[:n_mu].reshape(nI, nJ)
        points = {}
        for k, (i, j, (kind, s, a_row, flow, rc, rp)) in enumerate(col_of):
            pc, pp = points.get((i, j), (0.0, 0.0))
            points[(i, j)] = (pc + rc * x[n_mu + k], pp + rp * x[n_mu + k])
        details["pair_values"] = points
        details["achieved"] = A[r_obj:r_obj + n_obj, :n_mu + n_z] @ x[:n_mu + n_z]
    return feasible, details
