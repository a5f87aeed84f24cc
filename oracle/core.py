"""Oracle: products, Algorithms 2-4, exact evaluation and brute force.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64 throughout.

Product states follow oracle.c: u = k*S + s for the k-th non-done location,
plus one absorbing DONE state (the last index) with value 0.

Parity pins for each function live in tests/test_oracle_*.py.
"""

from __future__ import annotations

import ctypes
import itertools
import os

import numpy as np
from scipy.optimize import linear_sum_assignment
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

from . import dfa as _dfa

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def lib():
    """Load oracle/liboracle.so (built by oracle/build.py)."""
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "liboracle.so")
        if not os.path.exists(path):
            from .build import build as _build

            _build()
        L = ctypes.CDLL(path)
        L.orc_build_product.restype = ctypes.c_long
        L.orc_build_product.argtypes = [ctypes.c_int, _i32p, _i32p, _i32p, _f64p, _f64p, _i32p, ctypes.c_int,
                                        _i32p, _i32p, _i32p, ctypes.c_int, _i32p, _i32p, _i32p, _f64p, _f64p]
        L.orc_alg3.restype = ctypes.c_int
        L.orc_alg3.argtypes = [ctypes.c_int, _i32p, _i32p, _i32p, _f64p, _f64p, ctypes.c_double, ctypes.c_int,
                               _f64p, _i32p, ctypes.POINTER(ctypes.c_int)]
        L.orc_finalise_policy.restype = None
        L.orc_finalise_policy.argtypes = [ctypes.c_int, _i32p, _i32p, _i32p, _f64p, _f64p, _f64p, _i32p,
                                          ctypes.c_double, _i32p]
        L.orc_alg4.restype = ctypes.c_int
        L.orc_alg4.argtypes = [ctypes.c_int, _i32p, _i32p, _i32p, _f64p, _f64p, _i32p, ctypes.c_double,
                               ctypes.c_int, _f64p, ctypes.POINTER(ctypes.c_int)]
        _LIB = L
    return _LIB


class Product:
    """The agent-task product M_i (x) A_j with done_j collapsed to DONE."""

    def __init__(self, agent, task):
        d = _dfa.preprocess(task)
        let = _dfa.letters(agent, task)
        S, SA, T = agent.n_states, agent.n_sa, agent.n_trans
        n_nd = len(d["nd_loc"])
        self.S, self.n_nd, self.dfa = S, n_nd, d
        self.n = n_nd * S + 1
        self.done = n_nd * S
        state_ptr = np.zeros(n_nd * S + 2, np.int32)
        sa_ptr = np.zeros(n_nd * SA + 1, np.int32)
        col = np.zeros(max(n_nd * T, 1), np.int32)
        prob = np.zeros(max(n_nd * T, 1), np.float64)
        sa_cost = np.zeros(max(n_nd * SA, 1), np.float64)
        n_tr = lib().orc_build_product(
            S, agent.state_ptr.astype(np.int32), agent.sa_ptr.astype(np.int32), agent.succ.astype(np.int32),
            agent.prob.astype(np.float64), agent.cost.astype(np.float64), let, n_nd,
            np.ascontiguousarray(d["nd_loc"], np.int32), np.ascontiguousarray(d["nd_pos"], np.int32),
            np.ascontiguousarray(d["delta"].reshape(-1), np.int32), d["n_letters"],
            state_ptr, sa_ptr, col, prob, sa_cost)
        self.state_ptr = state_ptr[: self.n + 1]
        self.sa_ptr = sa_ptr[: n_nd * SA + 1]
        self.col = col[:n_tr]
        self.prob = prob[:n_tr]
        self.sa_cost = sa_cost[: n_nd * SA]
        # pre-sink flag per product state and per state-action row
        pre_state = np.zeros(self.n, bool)
        for k, q in enumerate(d["nd_loc"]):
            if d["pre"][q]:
                pre_state[k * S:(k + 1) * S] = True
        self.pre_state = pre_state
        self.sa_state = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.state_ptr))
        self.pre_sa = pre_state[self.sa_state].astype(np.float64)
        q0 = d["q0"]
        self.init = self.done if d["done"][q0] else int(d["nd_pos"][q0]) * S + agent.s0
        self.n_sa = len(self.sa_cost)
        self.n_trans = n_tr

    # rewards per state-action row ------------------------------------------
    def reward_cost(self):
        """rho_i(s, q, a) = -cost(s, a)."""
        return -self.sa_cost.astype(np.float64)

    def reward_prob(self):
        """rho_{j+|I|}(s, q, a) = 1 iff q is a pre-sink."""
        return self.pre_sa.copy()

    def reward_scalarised(self, w_cost, w_prob):
        """(w . rho)(s, q, a) restricted to this product's two objectives."""
        return w_cost * self.reward_cost() + w_prob * self.reward_prob()

    def key(self, u):
        """(agent state, DFA location) of product state u, or ('DONE',)."""
        if u == self.done:
            return ("DONE",)
        return (u % self.S, int(self.dfa["nd_loc"][u // self.S]))


def alg3(prod, rew, eps, max_sweeps=1_000_000, x0=None, a_rec0=None):
    x = np.zeros(prod.n) if x0 is None else np.array(x0, np.float64)
    a_rec = np.zeros(prod.n, np.int32) if a_rec0 is None else np.array(a_rec0, np.int32)
    sw = ctypes.c_int(0)
    rc = lib().orc_alg3(prod.n, prod.state_ptr, prod.sa_ptr, prod.col, prod.prob, np.ascontiguousarray(rew),
                        float(eps), int(max_sweeps), x, a_rec, ctypes.byref(sw))
    return x, a_rec, sw.value, rc == 0


def finalise(prod, rew, x, a_rec, tau=1e-9):
    mu = np.zeros(prod.n, np.int32)
    lib().orc_finalise_policy(prod.n, prod.state_ptr, prod.sa_ptr, prod.col, prod.prob, np.ascontiguousarray(rew),
                              np.ascontiguousarray(x, np.float64), np.ascontiguousarray(a_rec, np.int32),
                              float(tau), mu)
    return mu


def alg4(prod, rew, mu, eps, max_sweeps=10_000_000, x0=None):
    x = np.zeros(prod.n) if x0 is None else np.array(x0, np.float64)
    sw = ctypes.c_int(0)
    rc = lib().orc_alg4(prod.n, prod.state_ptr, prod.sa_ptr, prod.col, prod.prob, np.ascontiguousarray(rew),
                        np.ascontiguousarray(mu, np.int32), float(eps), int(max_sweeps), x, ctypes.byref(sw))
    return x, sw.value, rc == 0


def q_values(prod, rew, x):
    """Q(u, a) for every state-action row (numpy, for tests)."""
    contrib = prod.prob * x[prod.col]
    sums = np.zeros(prod.n_sa)
    rows = np.repeat(np.arange(prod.n_sa), np.diff(prod.sa_ptr))
    np.add.at(sums, rows, contrib)
    return rew + sums


def solve_pair(prod, w_cost, w_prob, eps1=1e-8, eps_eval=1e-11, tau=1e-9, max_sweeps=1_000_000,
               exact_eval=False):
    """Algorithm 3 on one product for the two weights that reach it, the
    returned scheduler, and Algorithm 4 for its cost and probability."""
    rew = prod.reward_scalarised(w_cost, w_prob)
    x, a_rec, sweeps, conv = alg3(prod, rew, eps1, max_sweeps)
    mu = finalise(prod, rew, x, a_rec, tau)
    if exact_eval:
        vc = exact_policy_values(prod, prod.reward_cost(), mu)
        vp = exact_policy_values(prod, prod.reward_prob(), mu)
        sc = sp = 0
    else:
        vc, sc, _ = alg4(prod, prod.reward_cost(), mu, eps_eval)
        vp, sp, _ = alg4(prod, prod.reward_prob(), mu, eps_eval)
    return {
        "c": float(x[prod.init]),
        "r_cost": float(vc[prod.init]),
        "r_prob": float(vp[prod.init]),
        "x": x,
        "a_rec": a_rec,
        "mu": mu,
        "sweeps": sweeps,
        "converged": conv,
        "eval_sweeps": (sc, sp),
        "rew": rew,
    }


def states_from_locations(prod, loc):
    """Oracle state index of each state of a product whose states are listed
    as pl * S + s over a list `loc` of non-done DFA locations (pl-th entry =
    the location), followed by one done state: for reading a scheduler
    computed on another layout of the same product."""
    S = prod.S
    pos = prod.dfa["nd_pos"]
    out = np.empty(len(loc) * S + 1, np.int64)
    for pl, q in enumerate(loc):
        out[pl * S:(pl + 1) * S] = int(pos[q]) * S + np.arange(S)
    out[-1] = prod.done
    return out


def scheduler_check(prod, w_cost, w_prob, mu, eps1=1e-8, eps_eval=1e-11, tau_gap=1e-9, r=None):
    """For a scheduler mu given in oracle state order: Algorithm 4 of its cost
    and probability (an exact solve when the product has at most 512
    states), and the number of states where the oracle's own scheduler has
    an action gap above tau_gap on its final values and mu differs from it.
    r: the oracle's solve_pair result for this pair, when already computed."""
    if r is None:
        r = solve_pair(prod, w_cost, w_prob, eps1=eps1, eps_eval=eps_eval)
    mu = np.asarray(mu, np.int32)
    if prod.n <= 512:
        vc = exact_policy_values(prod, prod.reward_cost(), mu)[prod.init]
        vp = exact_policy_values(prod, prod.reward_prob(), mu)[prod.init]
    else:
        vc = alg4(prod, prod.reward_cost(), mu, eps_eval, max_sweeps=1_000_000)[0][prod.init]
        vp = alg4(prod, prod.reward_prob(), mu, eps_eval, max_sweeps=1_000_000)[0][prod.init]
    # the action gap of the oracle's choice at every state (vectorised over rows)
    q = q_values(prod, r["rew"], r["x"])
    counts = np.diff(prod.state_ptr[: prod.n])
    states = np.repeat(np.arange(prod.n - 1), counts[: prod.n - 1])
    chosen = prod.state_ptr[: prod.n - 1] + r["mu"][: prod.n - 1]
    q_other = q.copy()
    q_other[chosen] = -np.inf
    best_other = np.full(prod.n - 1, -np.inf)
    np.maximum.at(best_other, states, q_other[: len(states)])
    gap = q[chosen] - best_other
    sel = gap > tau_gap
    checked = int(sel.sum())
    bad = sel & (mu[: prod.n - 1] != r["mu"][: prod.n - 1])
    mismatch = int(bad.sum())
    # at a mismatch: the oracle's gap, and how far mu's action falls below the
    # maximum on the oracle's values
    loss = q[chosen[bad]] - q[prod.state_ptr[: prod.n - 1][bad] + mu[: prod.n - 1][bad]]
    return {"c": r["c"], "r_cost": r["r_cost"], "r_prob": r["r_prob"], "mu_r_cost": float(vc), "mu_r_prob": float(vp),
            "gap_states": checked, "gap_mismatch": mismatch,
            "mismatch_max_gap": float(gap[bad].max()) if mismatch else 0.0,
            "mismatch_max_loss": float(loss.max()) if mismatch else 0.0}


def solve_pair_job(job):
    """One (agent, task, w_cost, w_prob, eps1[, loc, mu]) job, for process
    pools of the tests (spawned processes; the product is rebuilt in the
    worker).  Without a scheduler: (c, r_cost, r_prob) of solve_pair.  With
    another layout's location list `loc` and a scheduler `mu` on that
    layout: scheduler_check of mu."""
    agent, task, w_cost, w_prob, eps1 = job[:5]
    prod = Product(agent, task)
    if len(job) == 5:
        r = solve_pair(prod, w_cost, w_prob, eps1=eps1)
        return r["c"], r["r_cost"], r["r_prob"]
    loc, mu_other = job[5], np.asarray(job[6])
    idx = states_from_locations(prod, loc)
    mu = np.zeros(prod.n, np.int32)
    mu[idx[:-1]] = mu_other[: len(idx) - 1]
    return scheduler_check(prod, w_cost, w_prob, mu, eps1=eps1)


def solve_pairs_pooled(jobs, procs=None):
    """solve_pair_job over many jobs on every host core (spawn context, so
    it is safe in a process that already uses a GPU)."""
    import multiprocessing as mp

    procs = procs or len(os.sched_getaffinity(0))
    lib()  # built once here, not by every worker at once
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(solve_pair_job, jobs, chunksize=max(1, len(jobs) // (4 * procs)))


# ----------------------------------------------------------------------------
# exact values of a fixed scheduler and brute force over schedulers


def exact_policy_values(prod, rew, mu):
    """Expected total reward under the simple scheduler mu, exactly (dense
    LU).  States whose run under mu enters a closed class without DONE get 0
    if that class carries no reward and -inf/+inf otherwise."""
    n = prod.n
    a = prod.state_ptr[:-1] + np.asarray(mu[:n])
    rows, cols, vals = [], [], []
    r = np.zeros(n)
    for u in range(n):
        if u == prod.done:
            rows.append(u)
            cols.append(u)
            vals.append(1.0)
            continue
        r[u] = rew[a[u]]
        for t in range(prod.sa_ptr[a[u]], prod.sa_ptr[a[u] + 1]):
            rows.append(u)
            cols.append(int(prod.col[t]))
            vals.append(float(prod.prob[t]))
    P = csr_matrix((vals, (rows, cols)), shape=(n, n)).toarray()
    ncomp, comp = connected_components(csr_matrix(P > 0), directed=True, connection="strong")
    bottom = np.ones(ncomp, bool)
    for u in range(n):
        for v in np.flatnonzero(P[u] > 0):
            if comp[v] != comp[u]:
                bottom[comp[u]] = False
    in_bottom = bottom[comp]
    val = np.zeros(n)
    bad = np.zeros(n, bool)
    for c in range(ncomp):
        if not bottom[c]:
            continue
        members = np.flatnonzero(comp == c)
        tot = r[members]
        if np.any(tot != 0):
            val[members] = -np.inf if np.all(tot <= 0) else np.inf
            bad[members] = True
    # transient states that can reach a divergent class diverge as well
    changed = True
    while changed:
        changed = False
        for u in np.flatnonzero(~in_bottom & ~bad):
            nxt = np.flatnonzero(P[u] > 0)
            hit = nxt[bad[nxt]]
            if len(hit):
                bad[u] = True
                val[u] = -np.inf if np.any(val[hit] == -np.inf) else np.inf
                changed = True
    tr = np.flatnonzero(~in_bottom & ~bad)
    if len(tr):
        A = np.eye(len(tr)) - P[np.ix_(tr, tr)]
        val[tr] = np.linalg.solve(A, r[tr])
    return val


def enumerate_schedulers(prod):
    counts = np.diff(prod.state_ptr)
    ranges = [range(max(int(c), 1)) for c in counts]
    for choice in itertools.product(*ranges):
        yield np.asarray(choice, np.int32)


def brute_force(prod, w_cost, w_prob, limit=20000):
    """Every simple scheduler: its scalarised value and its (cost, prob) point
    at the initial state.  Returns (best value, list of (mu, value, point))."""
    counts = np.diff(prod.state_ptr)
    total = int(np.prod(np.maximum(counts, 1).astype(np.float64)))
    if total > limit:
        raise ValueError(f"{total} schedulers exceed the brute-force limit")
    out = []
    rc, rp = prod.reward_cost(), prod.reward_prob()
    for mu in enumerate_schedulers(prod):
        vc = exact_policy_values(prod, rc, mu)[prod.init]
        vp = exact_policy_values(prod, rp, mu)[prod.init]
        if not np.isfinite(vc):
            val = -np.inf if w_cost > 0 else w_prob * vp
        else:
            val = w_cost * vc + w_prob * vp
        out.append((mu, val, (vc, vp)))
    best = max(v for _, v, _ in out)
    return best, out


# ----------------------------------------------------------------------------
# Algorithm 2 (supporting point) and the assignment step


def assignment(C):
    """Hungarian step of Algorithm 2: the assignment f maximising
    sum_j C[f(j), j] (scipy's linear_sum_assignment).  C is square."""
    rows, cols = linear_sum_assignment(C, maximize=True)
    f = np.empty(C.shape[1], np.int64)
    f[cols] = rows
    return f


def pad_square(C):
    """|I| != |J|: pad with zero rows (dummy agents) or zero columns (dummy
    tasks) so the assignment is a permutation."""
    nI, nJ = C.shape
    n = max(nI, nJ)
    out = np.zeros((n, n))
    out[:nI, :nJ] = C
    return out


def products(inst_agents, inst_tasks):
    return [[Product(a, t) for t in inst_tasks] for a in inst_agents]


def supporting_point(prods, w, eps1=1e-8, eps_eval=1e-11, tau=1e-9):
    """Algorithm 2 for weight vector w over the product grid prods[i][j]."""
    nI, nJ = len(prods), len(prods[0])
    C = np.zeros((nI, nJ))
    RC = np.zeros((nI, nJ))
    RP = np.zeros((nI, nJ))
    for i in range(nI):
        for j in range(nJ):
            res = solve_pair(prods[i][j], w[i], w[nI + j], eps1, eps_eval, tau)
            C[i, j], RC[i, j], RP[i, j] = res["c"], res["r_cost"], res["r_prob"]
    f = assignment(pad_square(C))
    r = np.zeros(nI + nJ)
    for j in range(nJ):
        i = int(f[j])
        if i < nI:
            r[i] = RC[i, j]
            r[nI + j] = RP[i, j]
    return r, f[:nJ], C, RC, RP
