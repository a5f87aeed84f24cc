"""Algorithm 2 (and the Algorithm 1 loop on top of it) with the products of
one instance sharded over several processes, one GPU each.

The |I| x |J| product MDPs are independent until the assignment (Sec. 3.2),
so each product is a unit of work: products are dealt to ranks by a greedy
longest-processing-time rule on an estimate of their work (transitions x
expected sweeps), and each rank builds only its own products
(morap_select_pairs).  A batch of K weight vectors then runs as

  1. Algorithm 3 on every product the rank owns (morap_solve, no Algorithm 4);
  2. an all-gather of the c values, so that every rank holds c[K][|I|][|J|];
  3. the assignment, on every rank (the same host routine on the same input
     gives the same f everywhere, so nothing else needs to be exchanged);
  4. Algorithm 4 on the assigned pairs the rank owns (morap_evaluate);
  5. an all-reduce (sum) of the r vectors: each entry is written by exactly
     one rank and is 0 elsewhere, so the sum is exact.

Per (product, weight) pair the engine's result does not depend on the other
pairs in the batch, so the sharded supporting points are bit-identical to
those of one context holding every product.

The collectives go through torch.distributed (NCCL between GPUs, gloo on
the host).  The per-rank work is behind a small shard interface
(`optimise`, `evaluate`), which `EngineShard` implements with the C-ABI.
"""

from __future__ import annotations

import math
from typing import Callable, Sequence

import numpy as np

from . import morap as M


def product_loads(agents, tasks) -> np.ndarray:
    """Work estimate per product [|I|][|J|]: its transitions (the agent's
    transitions once per location of the task) times the sweeps value
    iteration needs, estimated as the longest expected path: the task's
    location count (targets visited in sequence) times the square root of
    the agent's state count (the side of a grid)."""
    L = np.zeros((len(agents), len(tasks)))
    for i, a in enumerate(agents):
        for j, t in enumerate(tasks):
            L[i, j] = float(len(a.succ)) * int(t.n_locs) * int(t.n_locs) * math.sqrt(int(a.n_states))
    return L


def partition_products(loads, world: int) -> list[list[tuple[int, int]]]:
    """Deal products (i, j) to `world` ranks: heaviest first, each to the rank
    with the least load so far (lowest rank on ties).  Deterministic, so
    every rank computes the same partition.  Returns each rank's pairs in
    (i, j) order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = np.asarray(loads, np.float64)
    nI, nJ = loads.shape
    order = sorted(((i, j) for i in range(nI) for j in range(nJ)), key=lambda ij: (-loads[ij], ij))
    total = [0.0] * world
    parts: list[list[tuple[int, int]]] = [[] for _ in range(world)]
    for ij in order:
        r = min(range(world), key=lambda q: (total[q], q))
        parts[r].append(ij)
        total[r] += float(loads[ij])
    return [sorted(p) for p in parts]


def assemble_c(parts: Sequence[np.ndarray], pairs_by_rank: Sequence[Sequence[tuple[int, int]]], n_agents: int,
               n_tasks: int) -> np.ndarray:
    """c[K][|I|][|J|] from the per-rank blocks c_r[K][n_r] (value e of rank r
    is product pairs_by_rank[r][e]; blocks may be padded beyond n_r)."""
    K = parts[0].shape[0]
    C = np.zeros((K, n_agents, n_tasks))
    for part, pairs in zip(parts, pairs_by_rank):
        for e, (i, j) in enumerate(pairs):
            C[:, i, j] = part[:, e]
    return C


def owned_pairs(assign: np.ndarray, pairs: Sequence[tuple[int, int]]):
    """(local product index, weight index, agent, task) of the assigned pairs
    a shard owns; the local index is the pair's position in `pairs`."""
    pos = {tuple(ij): e for e, ij in enumerate(pairs)}
    out = []
    for k in range(assign.shape[0]):
        for j in range(assign.shape[1]):
            i = int(assign[k, j])
            if i >= 0 and (i, j) in pos:
                out.append((pos[(i, j)], k, i, j))
    return out


class EngineShard:
    """Some products of one instance, on this process's GPU: a context with
    every agent and task, restricted to the shard's pairs."""

    def __init__(self, agents, tasks, pairs: Sequence[tuple[int, int]], cfg=None, stream=None):
        self.pairs = [tuple(p) for p in pairs]
        self.n_agents = len(agents)
        self.n_tasks = len(tasks)
        self.stream = stream
        self.ctx = None
        if self.pairs:
            self.ctx = M.Context(cfg)
            self.ctx.add(agents, tasks)
            self.ctx.select_pairs(self.pairs)
            self.ctx.build(stream)

    def optimise(self, W: np.ndarray):
        """Algorithm 3 for the shard's products: (c[K][n_pairs], not_converged)."""
        K = np.atleast_2d(W).shape[0]
        if self.ctx is None:
            return np.zeros((K, 0)), False
        out = self.ctx.solve(W, self.stream, evaluate=False)
        return out["c"], out["code"] == M.ENOTCONV

    def evaluate(self, assign: np.ndarray):
        """Algorithm 4 for the assigned pairs the shard owns: (r[K][|I|+|J|]
        with only those entries set, not_converged)."""
        K = assign.shape[0]
        r = np.zeros((K, self.n_agents + self.n_tasks))
        pairs = owned_pairs(assign, self.pairs)
        if not pairs:
            return r, False
        ev = M.morap_evaluate(self.ctx.h, [p for p, _, _, _ in pairs], [k for _, k, _, _ in pairs], self.stream)
        for e, (_, k, i, j) in enumerate(pairs):
            r[k, i] = ev["r_cost"][e]
            r[k, self.n_agents + j] = ev["r_prob"][e]
        return r, ev["code"] == M.ENOTCONV

    def stats(self):
        return self.ctx.stats() if self.ctx is not None else None

    def close(self):
        if self.ctx is not None:
            self.ctx.close()
            self.ctx = None


class TorchComm:
    """The two collectives over a torch.distributed process group."""

    def __init__(self, group=None, device=None):
        import torch
        import torch.distributed as dist

        self.torch, self.dist, self.group = torch, dist, group
        self.world = dist.get_world_size(group)
        self.device = device if device is not None else torch.device("cpu")

    def all_gather(self, a: np.ndarray) -> list[np.ndarray]:
        t = self.torch.from_numpy(np.ascontiguousarray(a)).to(self.device)
        out = [self.torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t, group=self.group)
        return [o.cpu().numpy() for o in out]

    def all_reduce_sum(self, a: np.ndarray) -> np.ndarray:
        t = self.torch.from_numpy(np.ascontiguousarray(a)).to(self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()


class ShardedSupportingPoints:
    """Algorithm 2 over a sharded instance: this rank's shard plus the
    collectives.  `pairs_by_rank` is the partition every rank agreed on."""

    def __init__(self, shard, pairs_by_rank: Sequence[Sequence[tuple[int, int]]], n_agents: int, n_tasks: int,
                 comm):
        self.shard = shard
        self.pairs_by_rank = [[tuple(p) for p in x] for x in pairs_by_rank]
        self.n_agents, self.n_tasks = n_agents, n_tasks
        self.comm = comm
        self.width = max(1, max(len(x) for x in self.pairs_by_rank))

    def __call__(self, W: np.ndarray) -> dict:
        W = np.atleast_2d(np.asarray(W, np.float64))
        K = W.shape[0]
        c, nc1 = self.shard.optimise(W)
        block = np.zeros((K, self.width))
        block[:, : c.shape[1]] = c
        C = assemble_c(self.comm.all_gather(block), self.pairs_by_rank, self.n_agents, self.n_tasks)
        assign = M.morap_assign_tasks(C)
        r_part, nc2 = self.shard.evaluate(assign)
        flags = np.zeros((K, self.n_agents + self.n_tasks + 1))
        flags[:, :-1] = r_part
        flags[0, -1] = 1.0 if (nc1 or nc2) else 0.0
        tot = self.comm.all_reduce_sum(flags)
        code = M.ENOTCONV if tot[0, -1] > 0 else M.OK
        return {"r": tot[:, :-1], "assign": assign, "c": C, "code": code}

    def query(self, t, Mnorm=None, eps=1e-6, max_iter=64, verify_only=False) -> dict:
        """Algorithm 1 for threshold t with these supporting points (or its
        verification-only form); every rank runs the same loop on the same
        numbers."""
        return run_alg1(lambda w: self(w[None, :]), t, Mnorm, eps, max_iter, verify_only)


def run_alg1(supporting_point: Callable[[np.ndarray], dict], t, Mnorm=None, eps=1e-6, max_iter=64,
             verify_only=False) -> dict:
    """Algorithm 1 (or its verification-only form) through morap_pareto_*,
    with supporting_point(w) -> {"r": [1][n], "code"}."""
    P = M.Pareto(t, Mnorm, eps, max_iter, verify_only)
    try:
        while True:
            w = P.next()
            if w is None:
                break
            out = supporting_point(w)
            P.step(np.asarray(out["r"])[0], out["code"])
        return P.result()
    finally:
        P.close()
