"""Seeded generators for agent MDPs, task DFAs, weight vectors and thresholds.

Formats (all numpy arrays, C-contiguous):

Agent (a labelled MDP, the paper's (S, s0, A, P, L) with a per-action cost):
    n_states            number of agent states
    s0                  initial state
    state_ptr[n+1]      int32, actions of state s are state-action (SA) rows
                        state_ptr[s] .. state_ptr[s+1]-1; the local action
                        index is the position inside that range
    sa_ptr[SA+1]        int32, successors of SA row a are sa_ptr[a] .. sa_ptr[a+1]-1
    succ[T]             int32 successor state of each transition (sorted and
                        distinct within an SA row)
    prob[T]             float64 transition probability (each SA row sums to 1)
    cost[SA]            float64 cost of taking the action (>= 0); the paper
                        uses it as the negative reward rho_i(s, a) = -cost
    label_ptr[n+1]      int32, atomic propositions holding in state s are
    label_ap[L]         label_ap[label_ptr[s] .. label_ptr[s+1]-1] (global AP ids)

Task (a DFA whose accepting locations are sinks):
    n_locs, q0, n_ap
    ap_ids[n_ap]        int32 global AP id of letter bit b
    delta[n_locs * 2^n_ap] int32, delta[q * 2^n_ap + letter]
    accepting[n_locs]   uint8

Grid semantics: actions stay=0, N=1, S=2, E=3, W=4; a move reaches the
intended neighbour with probability 1-slip and each perpendicular neighbour
with slip/2; a move into the border or an obstacle leaves the agent in place
(and still costs 1); stay costs 0.  Each cell carries the AP GRID_AP(x, y).
"""

from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

# Global atomic-proposition namespace: one AP per grid cell, one per region.
GRID_AP_STRIDE = 1024


def GRID_AP(x: int, y: int) -> int:
    return int(y) * GRID_AP_STRIDE + int(x)


def REGION_AP(r: int) -> int:
    return (1 << 22) + int(r)


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Counter-based generator (Philox) keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream)]))


@dataclass
class Agent:
    n_states: int
    s0: int
    state_ptr: np.ndarray
    sa_ptr: np.ndarray
    succ: np.ndarray
    prob: np.ndarray
    cost: np.ndarray
    label_ptr: np.ndarray
    label_ap: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_sa(self) -> int:
        return int(self.state_ptr[-1])

    @property
    def n_trans(self) -> int:
        return int(self.sa_ptr[-1])


@dataclass
class Task:
    n_locs: int
    q0: int
    n_ap: int
    ap_ids: np.ndarray
    delta: np.ndarray
    accepting: np.ndarray
    meta: dict = field(default_factory=dict)


@dataclass
class Instance:
    agents: list
    tasks: list
    weights: np.ndarray  # [K][|I|+|J|]
    thresholds: np.ndarray  # [n_points][|I|+|J|]: costs (negative) then probabilities
    name: str = ""
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# agents


def _pack_agent(rows, labels, s0, meta):
    """rows[s] = list of (cost, {succ: prob}); labels[s] = list of AP ids."""
    n = len(rows)
    state_ptr = np.zeros(n + 1, np.int32)
    sa_ptr = [0]
    succ, prob, cost = [], [], []
    for s, acts in enumerate(rows):
        state_ptr[s + 1] = state_ptr[s] + len(acts)
        for c, dist in acts:
            for t in sorted(dist):
                succ.append(t)
                prob.append(dist[t])
            sa_ptr.append(len(succ))
            cost.append(c)
    label_ptr = np.zeros(n + 1, np.int32)
    label_ap = []
    for s in range(n):
        label_ap.extend(sorted(set(labels[s])))
        label_ptr[s + 1] = len(label_ap)
    return Agent(
        n_states=n,
        s0=int(s0),
        state_ptr=state_ptr,
        sa_ptr=np.asarray(sa_ptr, np.int32),
        succ=np.asarray(succ, np.int32),
        prob=np.asarray(prob, np.float64),
        cost=np.asarray(cost, np.float64),
        label_ptr=label_ptr,
        label_ap=np.asarray(label_ap, np.int32),
        meta=meta,
    )


_DIRS = [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)]  # stay, N, S, E, W
_PERP = {1: (3, 4), 2: (3, 4), 3: (1, 2), 4: (1, 2)}


def _grid_index(W, H, blocked):
    idx = -np.ones((H, W), np.int64)
    k = 0
    for y in range(H):
        for x in range(W):
            if blocked is None or not blocked[y, x]:
                idx[y, x] = k
                k += 1
    return idx, k


def _region_labels(W, H, regions):
    lab = {}
    for ap, cells in regions or []:
        for (x, y) in cells:
            if 0 <= x < W and 0 <= y < H:
                lab.setdefault((x, y), []).append(ap)
    return lab


def grid_agent(W, H, slip, start, blocked=None, regions=None, move_cost=1.0):
    """Slippery grid robot (stay/N/S/E/W); `start` is an (x, y) cell."""
    idx, n = _grid_index(W, H, blocked)
    rlab = _region_labels(W, H, regions)
    rows, labels, cells = [], [], []
    for y in range(H):
        for x in range(W):
            s = idx[y, x]
            if s < 0:
                continue
            cells.append((x, y))

            def dest(d):
                nx, ny = x + _DIRS[d][0], y + _DIRS[d][1]
                if 0 <= nx < W and 0 <= ny < H and idx[ny, nx] >= 0:
                    return int(idx[ny, nx])
                return int(s)

            acts = [(0.0, {int(s): 1.0})]
            for d in (1, 2, 3, 4):
                dist = {}
                outs = [(dest(d), 1.0 - slip)]
                if slip > 0:
                    p1, p2 = _PERP[d]
                    outs += [(dest(p1), slip / 2.0), (dest(p2), slip / 2.0)]
                for t, p in outs:
                    dist[t] = dist.get(t, 0.0) + p
                acts.append((float(move_cost), dist))
            rows.append(acts)
            labels.append([GRID_AP(x, y)] + rlab.get((x, y), []))
    sx, sy = start
    assert idx[sy, sx] >= 0, "start cell is blocked"
    return _pack_agent(rows, labels, idx[sy, sx], {"W": W, "H": H, "slip": slip, "cells": cells, "kind": "grid"})


def moore_agent(W, H, start, seed, stream, blocked=None, regions=None, kmax=8, move_cost=1.0):
    """Grid robot whose moves have k ~ U{1..kmax} successors drawn from the
    3x3 Moore block around the cell (always including the intended
    neighbour), with Dirichlet(1) probabilities; stay is kept."""
    rng = _rng(seed, stream)
    idx, n = _grid_index(W, H, blocked)
    rlab = _region_labels(W, H, regions)
    block = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    rows, labels, cells = [], [], []
    for y in range(H):
        for x in range(W):
            s = idx[y, x]
            if s < 0:
                continue
            cells.append((x, y))

            def cell(dx, dy):
                nx, ny = x + dx, y + dy
                if 0 <= nx < W and 0 <= ny < H and idx[ny, nx] >= 0:
                    return int(idx[ny, nx])
                return int(s)

            acts = [(0.0, {int(s): 1.0})]
            for d in (1, 2, 3, 4):
                k = int(rng.integers(1, kmax + 1))
                intended = _DIRS[d]
                others = [b for b in block if b != intended]
                pick = rng.choice(len(others), size=k - 1, replace=False) if k > 1 else []
                outs = [intended] + [others[i] for i in pick]
                ps = rng.dirichlet(np.ones(k))
                dist = {}
                for (dx, dy), p in zip(outs, ps):
                    t = cell(dx, dy)
                    dist[t] = dist.get(t, 0.0) + float(p)
                acts.append((float(move_cost), dist))
            rows.append(acts)
            labels.append([GRID_AP(x, y)] + rlab.get((x, y), []))
    sx, sy = start
    return _pack_agent(rows, labels, idx[sy, sx], {"W": W, "H": H, "cells": cells, "kind": "moore"})


def corridor_agent(L, slip, start=0, stay=True):
    """1 x L corridor: E/W moves succeed with 1-slip, perpendicular slips
    are blocked (self-loops).  Used for closed-form checks."""
    return grid_agent(L, 1, slip, (start, 0))


def chain_agent(N, p_fwd, p_trap, cost=1.0):
    """States 0..N-1 plus a goal cell N and a trap cell N+1.  One 'go'
    action: forward with p_fwd, into the trap with p_trap, stay otherwise;
    plus a free 'stay' action (index 0).  The goal carries AP 1, the trap AP 2."""
    rows, labels = [], []
    for s in range(N):
        go = {}
        fwd = s + 1 if s + 1 < N else N
        go[fwd] = go.get(fwd, 0.0) + p_fwd
        go[N + 1] = go.get(N + 1, 0.0) + p_trap
        rest = 1.0 - p_fwd - p_trap
        if rest > 0:
            go[s] = go.get(s, 0.0) + rest
        rows.append([(0.0, {s: 1.0}), (float(cost), go)])
        labels.append([])
    rows.append([(0.0, {N: 1.0})])
    labels.append([1])
    rows.append([(0.0, {N + 1: 1.0})])
    labels.append([2])
    return _pack_agent(rows, labels, 0, {"kind": "chain", "N": N})


def fig2_agent():
    """The four-state agent of the paper's worked example (Fig. 2a):
    s0 -a-> {s0:.3, s1:.2, s2:.5}, s0 -b-> {s1:.9, s3:.1}, s2 -> s3,
    self-loops on s1 and s3, L(s1) = {x} (AP 0), L(s3) = {y} (AP 1),
    every action costs 1."""
    rows = [
        [(1.0, {0: 0.3, 1: 0.2, 2: 0.5}), (1.0, {1: 0.9, 3: 0.1})],
        [(1.0, {1: 1.0})],
        [(1.0, {3: 1.0})],
        [(1.0, {3: 1.0})],
    ]
    labels = [[], [0], [], [1]]
    return _pack_agent(rows, labels, 0, {"kind": "fig2"})


def fig2_task():
    """DFA of (not x) U y: q0 --y--> F, q0 --x and not y--> trap, else q0.
    Letter bit 0 = x, bit 1 = y."""
    delta = np.zeros((3, 4), np.int32)
    for letter in range(4):
        x, y = letter & 1, (letter >> 1) & 1
        delta[0, letter] = 1 if y else (2 if x else 0)
        delta[1, letter] = 1
        delta[2, letter] = 2
    return Task(3, 0, 2, np.array([0, 1], np.int32), delta.reshape(-1), np.array([0, 1, 0], np.uint8), {"kind": "fig2"})


def tie_drift_agent(delta=5e-9, s=0.5, s_far=1e-3):
    """Seven states built so that Algorithm 3's recorded action goes stale
    and two states tie.  From A (state 0, the start) the goal G (AP 0) is
    reached by X (one move, then G with 1 - delta, a dead end T otherwise) or
    by Y (a move that reaches G with probability s per try); B (state 1) can
    go to A or to X, and A to B.  Y's value overtakes X's only once its
    per-sweep increments are below 1e-8, while a far state Z (G with s_far
    per try) keeps the sweeps going, so A and B keep "go to X" recorded, and
    on the final values A -> B, B -> A and A -> Y all tie at probability 1.
    Every move costs 1; action 0 of every state is a free stay."""
    A, B, X, Y, Z, Gs, T = range(7)
    rows = [
        [(0.0, {A: 1.0}), (1.0, {B: 1.0}), (1.0, {X: 1.0}), (1.0, {Y: 1.0})],
        [(0.0, {B: 1.0}), (1.0, {A: 1.0}), (1.0, {X: 1.0})],
        [(0.0, {X: 1.0}), (1.0, {Gs: 1.0 - delta, T: delta})],
        [(0.0, {Y: 1.0}), (1.0, {Gs: s, Y: 1.0 - s})],
        [(0.0, {Z: 1.0}), (1.0, {Gs: s_far, Z: 1.0 - s_far})],
        [(0.0, {Gs: 1.0})],
        [(0.0, {T: 1.0})],
    ]
    labels = [[], [], [], [], [], [0], []]
    return _pack_agent(rows, labels, A, {"kind": "tie_drift"})


def sequence_task(target_aps, avoid_ap=None):
    """'Visit target_aps[0], then target_aps[1], ...' optionally with 'and never
    enter the region labelled avoid_ap before finishing' (a trap).
    Locations: 0..m-1 progress, m accept, m+1 trap (if avoid)."""
    m = len(target_aps)
    n_ap = m + (1 if avoid_ap is not None else 0)
    assert 1 <= n_ap <= 8
    n_locs = m + 1 + (1 if avoid_ap is not None else 0)
    acc, trap = m, m + 1
    nl = 1 << n_ap
    delta = np.zeros((n_locs, nl), np.int32)
    for q in range(n_locs):
        for letter in range(nl):
            if q >= m:
                delta[q, letter] = q
            elif avoid_ap is not None and (letter >> m) & 1:
                delta[q, letter] = trap
            elif (letter >> q) & 1:
                delta[q, letter] = q + 1
            else:
                delta[q, letter] = q
    accepting = np.zeros(n_locs, np.uint8)
    accepting[acc] = 1
    ap_ids = list(target_aps) + ([avoid_ap] if avoid_ap is not None else [])
    return Task(n_locs, 0, n_ap, np.asarray(ap_ids, np.int32), delta.reshape(-1), accepting,
                {"kind": "sequence", "m": m, "avoid": avoid_ap is not None})


def random_tiny_agent(seed, stream, n_states=4, n_actions=(1, 3), n_succ=(1, 3), n_ap=2, zero_cost_stay=True,
                      integer_probs=False):
    """Small random MDP for brute-force checks.  Action 0 is a zero-cost
    self-loop when zero_cost_stay is set."""
    rng = _rng(seed, stream)
    rows, labels = [], []
    for s in range(n_states):
        acts = []
        if zero_cost_stay:
            acts.append((0.0, {s: 1.0}))
        na = int(rng.integers(n_actions[0], n_actions[1] + 1))
        for _ in range(na):
            k = int(rng.integers(n_succ[0], min(n_succ[1], n_states) + 1))
            ts = rng.choice(n_states, size=k, replace=False)
            if integer_probs:
                w = rng.integers(1, 5, size=k).astype(np.float64)
                ps = w / w.sum()
            else:
                ps = rng.dirichlet(np.ones(k))
            acts.append((float(rng.integers(1, 4)), {int(t): float(p) for t, p in zip(ts, ps)}))
        rows.append(acts)
        labels.append([int(b) for b in range(n_ap) if rng.random() < 0.35])
    return _pack_agent(rows, labels, 0, {"kind": "tiny"})


def random_tiny_task(seed, stream, n_locs=3, n_ap=2):
    """Small random DFA with one accepting sink (last location) and
    arbitrary transitions among the others."""
    rng = _rng(seed, stream)
    nl = 1 << n_ap
    delta = np.zeros((n_locs, nl), np.int32)
    for q in range(n_locs - 1):
        delta[q] = rng.integers(0, n_locs, size=nl)
    delta[n_locs - 1] = n_locs - 1
    accepting = np.zeros(n_locs, np.uint8)
    accepting[n_locs - 1] = 1
    return Task(n_locs, 0, n_ap, np.arange(n_ap, dtype=np.int32), delta.reshape(-1), accepting, {"kind": "tiny"})


# ----------------------------------------------------------------------------
# weights and thresholds


def weight_vectors(n_agents, n_tasks, K, seed, stream=7):
    """K weight vectors on the simplex.  The first is e_1 (the Pareto
    loop's initial direction); the others put a random share a ~ 10^U[-3,0]
    on Dirichlet(1)-split cost weights and the rest on Dirichlet(1)-split
    probability weights, so some directions make tasks worth their cost and
    some do not (the spread a point-oriented Pareto run visits)."""
    rng = _rng(seed, stream)
    n = n_agents + n_tasks
    W = np.zeros((K, n), np.float64)
    if K > 0:
        W[0, 0] = 1.0
    for k in range(1, K):
        a = 10.0 ** rng.uniform(-3.0, 0.0)
        wc = rng.dirichlet(np.ones(n_agents)) * a
        wp = rng.dirichlet(np.ones(n_tasks))
        w = np.concatenate([wc, wp])
        W[k] = w / w.sum()
    return W


def dirichlet_weights(n, K, seed, stream=8):
    rng = _rng(seed, stream)
    return rng.dirichlet(np.ones(n), size=K)


def threshold_points(n_agents, n_tasks, n_points, seed, stream=9, cost_range=(5.0, 50.0), prob_range=(0.5, 0.99)):
    """Threshold points t = (c, p): c_i = -U[cost_range] (a cost bound as a
    negative reward), p_j = U[prob_range]."""
    rng = _rng(seed, stream)
    c = -rng.uniform(cost_range[0], cost_range[1], size=(n_points, n_agents))
    p = rng.uniform(prob_range[0], prob_range[1], size=(n_points, n_tasks))
    return np.concatenate([c, p], axis=1)


# ----------------------------------------------------------------------------
# workload configurations


def _largest_free_component(blocked):
    H, W = blocked.shape
    comp = -np.ones((H, W), np.int64)
    best, best_size, cid = -1, 0, 0
    for y in range(H):
        for x in range(W):
            if blocked[y, x] or comp[y, x] >= 0:
                continue
            stack, size = [(x, y)], 0
            comp[y, x] = cid
            while stack:
                cx, cy = stack.pop()
                size += 1
                for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    nx, ny = cx + dx, cy + dy
                    if 0 <= nx < W and 0 <= ny < H and not blocked[ny, nx] and comp[ny, nx] < 0:
                        comp[ny, nx] = cid
                        stack.append((nx, ny))
            if size > best_size:
                best, best_size = cid, size
            cid += 1
    return [(x, y) for y in range(H) for x in range(W) if comp[y, x] == best]


def config_tiny(seed=0):
    """2 agents on a 4x4 grid (slip 0.1), 3 tasks 'visit a then b',
    5 objectives, threshold cost <= 8 and probability >= 0.9 each."""
    rng = _rng(seed, 1)
    W = H = 4
    cells = [(x, y) for y in range(H) for x in range(W)]
    starts = [cells[i] for i in rng.choice(len(cells), size=2, replace=False)]
    free = [c for c in cells if c not in starts]
    tasks = []
    for j in range(3):
        a, b = (free[i] for i in rng.choice(len(free), size=2, replace=False))
        tasks.append(sequence_task([GRID_AP(*a), GRID_AP(*b)]))
    agents = [grid_agent(W, H, 0.1, st) for st in starts]
    t = np.array([[-8.0, -8.0, 0.9, 0.9, 0.9]])
    Wt = weight_vectors(2, 3, 4, seed)
    return Instance(agents, tasks, Wt, t, "tiny-4x4-2x3")


PARETO_WEIGHTS_GRID32 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                                     "grid32_pareto_weights.txt")


def config_grid32(seed=1, n_agents=10, n_tasks=20, side=32, K=16, obstacle_frac=0.15, pareto_weights=False):
    """10 agents on one 32x32 warehouse grid with 15% random obstacles,
    per-agent slip ~ U[0.05, 0.2]; 20 tasks of 3-6 DFA locations (sequenced
    visits, half of them with an avoid region that is a trap).

    pareto_weights: take the K = 16 weight vectors recorded from Algorithm 1
    runs on the seed-1 instance (the default sizes; data file written by
    the oracle's record_pareto_weights) instead of the synthetic draws.
    Other seeds of the same sizes reuse those directions."""
    rng = _rng(seed, 2)
    blocked = rng.random((side, side)) < obstacle_frac
    comp = _largest_free_component(blocked)
    comp_set = set(comp)
    blocked = np.ones((side, side), bool)
    for (x, y) in comp:
        blocked[y, x] = False
    starts = [comp[i] for i in rng.choice(len(comp), size=n_agents, replace=False)]
    start_set = set(starts)
    tasks, regions = [], []
    for j in range(n_tasks):
        n_locs = int(rng.integers(3, 7))
        avoid = bool(j % 2 == 1)
        m = n_locs - 1 - (1 if avoid else 0)
        m = max(m, 1)
        cand = [c for c in comp if c not in start_set]
        tg = [cand[i] for i in rng.choice(len(cand), size=m, replace=False)]
        avoid_ap = None
        if avoid:
            # a 3x3 block avoiding the targets and start cells
            for _ in range(100):
                cx, cy = int(rng.integers(1, side - 1)), int(rng.integers(1, side - 1))
                blk = [(cx + dx, cy + dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
                if not any(c in tg or c in start_set for c in blk):
                    break
            avoid_ap = REGION_AP(j)
            regions.append((avoid_ap, [c for c in blk if c in comp_set]))
        tasks.append(sequence_task([GRID_AP(*c) for c in tg], avoid_ap))
    slips = rng.uniform(0.05, 0.2, size=n_agents)
    agents = [grid_agent(side, side, float(slips[i]), starts[i], blocked, regions) for i in range(n_agents)]
    Wt = weight_vectors(n_agents, n_tasks, K, seed)
    if pareto_weights:
        if (n_agents, n_tasks, K) != (10, 20, 16):
            raise ValueError("the recorded Pareto-loop weights are 16 directions of 10 agents and 20 tasks")
        Wt = np.loadtxt(PARETO_WEIGHTS_GRID32, dtype=np.float64, comments="#").reshape(K, n_agents + n_tasks)
    t = threshold_points(n_agents, n_tasks, 4, seed)
    return Instance(agents, tasks, Wt, t, f"grid{side}-{n_agents}x{n_tasks}",
                    {"side": side, "obstacle_frac": obstacle_frac})


def config_uneven(seed=2, n_agents=50, n_tasks=100, K=64, side_range=(16, 64), loc_range=(2, 8), kmax=8,
                  common=16):
    """50 agents x 100 tasks: per-agent grid side ~ U{16..64} with Moore-block
    successors (1-8, Dirichlet(1)), DFAs of 2-8 locations whose targets lie in
    the 16x16 corner every grid contains; K Dirichlet(1) weights."""
    rng = _rng(seed, 3)
    corner = [(x, y) for y in range(common) for x in range(common)]
    tasks = []
    for j in range(n_tasks):
        n_locs = int(rng.integers(loc_range[0], loc_range[1] + 1))
        m = n_locs - 1
        tg = [corner[i] for i in rng.choice(len(corner), size=m, replace=False)]
        tasks.append(sequence_task([GRID_AP(*c) for c in tg]))
    agents = []
    target_cells = set()
    for t_ in tasks:
        for ap in t_.ap_ids:
            target_cells.add((int(ap) % GRID_AP_STRIDE, int(ap) // GRID_AP_STRIDE))
    for i in range(n_agents):
        side = int(rng.integers(side_range[0], side_range[1] + 1))
        while True:
            st = (int(rng.integers(0, side)), int(rng.integers(0, side)))
            if st not in target_cells:
                break
        agents.append(moore_agent(side, side, st, seed, 100 + i, kmax=kmax))
    Wt = np.concatenate([np.eye(1, n_agents + n_tasks), dirichlet_weights(n_agents + n_tasks, K - 1, seed)])
    t = threshold_points(n_agents, n_tasks, 4, seed)
    return Instance(agents, tasks, Wt, t, f"uneven-{n_agents}x{n_tasks}")


def config_large(seed=3, n_agents=20, n_tasks=50, side=128, K=32, n_targets=3):
    """20 agents x 50 tasks on 128x128 grids (slip ~ U[0.05,0.2]) with
    4-location DFAs (3 sequenced targets + accept)."""
    rng = _rng(seed, 4)
    cells_n = side * side
    starts = []
    for i in range(n_agents):
        c = int(rng.integers(0, cells_n))
        starts.append((c % side, c // side))
    start_set = set(starts)
    tasks = []
    for j in range(n_tasks):
        tg = []
        while len(tg) < n_targets:
            c = int(rng.integers(0, cells_n))
            xy = (c % side, c // side)
            if xy not in start_set and xy not in tg:
                tg.append(xy)
        tasks.append(sequence_task([GRID_AP(*c) for c in tg]))
    slips = rng.uniform(0.05, 0.2, size=n_agents)
    agents = [grid_agent(side, side, float(slips[i]), starts[i]) for i in range(n_agents)]
    Wt = weight_vectors(n_agents, n_tasks, K, seed)
    t = threshold_points(n_agents, n_tasks, 4, seed)
    return Instance(agents, tasks, Wt, t, f"large{side}-{n_agents}x{n_tasks}")


def instance_footprint(inst):
    """Agent-side sizes only (states, state-actions, transitions per agent)."""
    return [(a.n_states, a.n_sa, a.n_trans) for a in inst.agents]
