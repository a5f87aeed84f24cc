"""CPU checks of the precision arguments behind the engine's FP32 residual
corrections, for Algorithm 3's polish and for Algorithm 4's block
evaluation.  Evaluation: iterate E <- r + P E in
FP32 until the moves are within 2^-18 of the values (B), form
G = r + P B - B in FP64 and round it to FP32, iterate d <- G + P d in FP32
to the residual rule (moves below (slots + 1) 2^-23 |y| counted as 0), and
take E = B + d.  For a fixed scheduler E* = B + d* exactly, so the result
must match the scheduler's exact values (dense LU, oracle) to far inside the
1e-6 tolerance.  The polish is the same with a maximum over actions.  These
emulate the arithmetic with numpy float32; they do not run the engine."""

import numpy as np
import pytest
from scipy.sparse import csr_matrix

import instances as I
from oracle import core as O


def _policy_system(prod, mu):
    n = prod.n
    a = prod.state_ptr[:-1] + np.asarray(mu[:n])
    rows, cols, vals = [], [], []
    R = np.zeros((n, 2))
    rc, rp = prod.reward_cost(), prod.reward_prob()
    slots = 0
    for u in range(n - 1):
        t0, t1 = prod.sa_ptr[a[u]], prod.sa_ptr[a[u] + 1]
        slots = max(slots, t1 - t0)
        for t in range(t0, t1):
            rows.append(u)
            cols.append(int(prod.col[t]))
            vals.append(float(prod.prob[t]))
        R[u] = rc[a[u]], rp[a[u]]
    return csr_matrix((vals, (rows, cols)), shape=(n, n)), R, slots


def _residual_correction(P, R, slots, thr=1e-11, cap=200_000):
    P32, R32 = P.astype(np.float32), R.astype(np.float32)
    b = np.zeros_like(R32)
    for _ in range(cap):  # stage A
        y = (R32 + P32 @ b).astype(np.float32)
        moved = np.max(np.abs(y - b), axis=0)
        top = np.max(np.abs(y), axis=0)
        b = y
        if np.all(moved <= 2.0**-18 * top):
            break
    G = (R + P @ b.astype(np.float64) - b.astype(np.float64)).astype(np.float32)  # stage B
    d = np.zeros_like(R32)
    noise = (slots + 1) * 2.0**-23
    for _ in range(cap):  # stage C
        y = (G + P32 @ d).astype(np.float32)
        moved = np.abs(y - d)
        moved[moved <= noise * np.abs(y)] = 0.0
        d = y
        if np.max(moved) <= thr:
            break
    return b.astype(np.float64) + d.astype(np.float64)  # stage D


@pytest.mark.parametrize("case", ["tiny", "random"])
def test_residual_correction_reaches_the_exact_values(case):
    if case == "tiny":
        inst = I.config_tiny()
        agents, tasks, W = inst.agents, inst.tasks, inst.weights
    else:
        agents = [I.random_tiny_agent(7, 80 + i, n_states=300, n_actions=(1, 3), n_succ=(1, 4)) for i in range(2)]
        tasks = [I.random_tiny_task(7, 90 + j, n_locs=3) for j in range(2)]
        W = np.random.default_rng(3).dirichlet(np.ones(4), size=3)
    nI = len(agents)
    checked = 0
    for i in range(nI):
        for j in range(len(tasks)):
            prod = O.Product(agents[i], tasks[j])
            for k in range(len(W)):
                res = O.solve_pair(prod, W[k][i], W[k][nI + j])
                P, R, slots = _policy_system(prod, res["mu"])
                exact = np.stack([O.exact_policy_values(prod, prod.reward_cost(), res["mu"]),
                                  O.exact_policy_values(prod, prod.reward_prob(), res["mu"])], axis=1)
                if not np.all(np.isfinite(exact)):
                    continue  # a scheduler that never finishes and pays for it: no finite values
                E = _residual_correction(P, R, slots)
                assert np.max(np.abs(E - exact)) < 1e-8, (i, j, k)
                checked += 1
    assert checked >= 6


def _sa_system(prod, w_cost, w_prob):
    """Row-wise (state-action) transition matrix and scalarised rewards."""
    n, SA = prod.n, len(prod.sa_cost)
    rows = np.repeat(np.arange(SA), np.diff(prod.sa_ptr))
    P = csr_matrix((prod.prob.astype(np.float64), (rows, prod.col.astype(np.int64))), shape=(SA, n))
    return P, prod.reward_scalarised(w_cost, w_prob)


def _bellman_max(Q, starts):
    return np.maximum.reduceat(Q, starts)


def test_polish_residual_correction_reaches_the_fixed_point():
    """The optimisation's polish: from FP32 values B (here plain FP32 value
    iteration from 0, stopped at 2^-16 of w_p), the table
    G_a = r_a + P_a B - B(s) in FP64 rounded to FP32 and the correction
    d <- max_a (G_a + P_a d) iterated in FP32 to eps1 reach V = B + d within
    far less than the tolerance of the tightly converged oracle values."""
    inst = I.config_tiny()
    nI = len(inst.agents)
    checked = 0
    for i in range(nI):
        for j in range(len(inst.tasks)):
            prod = O.Product(inst.agents[i], inst.tasks[j])
            starts = prod.state_ptr[:-2]  # transient states (the last state is DONE)
            n_tr = prod.n - 1
            for k in range(len(inst.weights)):
                wc, wp = inst.weights[k][i], inst.weights[k][nI + j]
                if wp <= 0:
                    continue
                P, r = _sa_system(prod, wc, wp)
                P32, r32 = P.astype(np.float32), r.astype(np.float32)
                b = np.zeros(prod.n, np.float32)
                for _ in range(100_000):
                    y = b.copy()
                    y[:n_tr] = _bellman_max((r32 + P32 @ b).astype(np.float32), starts)
                    moved = np.max(np.abs(y - b))
                    b = y
                    if moved <= 2.0**-16 * wp:
                        break
                G = (r + P @ b.astype(np.float64) - b.astype(np.float64)[np.repeat(np.arange(prod.n),
                                                                                   np.diff(prod.state_ptr))]
                     ).astype(np.float32)
                d = np.zeros(prod.n, np.float32)
                for _ in range(100_000):
                    y = d.copy()
                    y[:n_tr] = _bellman_max((G + P32 @ d).astype(np.float32), starts)
                    moved = np.max(np.abs(y - d))
                    d = y
                    if moved <= 1e-8:
                        break
                V = b.astype(np.float64) + d.astype(np.float64)
                ref = O.solve_pair(prod, wc, wp, eps1=1e-13)
                assert np.max(np.abs(V - ref["x"])) < 1e-7, (i, j, k)
                checked += 1
    assert checked >= 6
