"""Algorithm 2 (and the Algorithm 1 loop on top of it) with the products of
one instance sharded over several processes, one GPU each.

The |I| x |J| product MDPs are independent until the assignment (Sec. 3.2):
agent i's products with every task go to one rank, chosen by a greedy
longest-processing-time rule on the agents' transition counts.  A batch of
K weight vectors then runs as

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

from typing import Callable, Sequence

import numpy as np

from . import morap as M


def partition_agents(loads: Sequence[float], world: int) -> list[list[int]]:
    """Deal agents to `world` ranks: heaviest first, each to the rank with the
    least load so far (lowest rank on ties).  Deterministic, so every rank
    computes the same partition.  Returns the sorted agent ids per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(loads)), key=lambda i: (-float(loads[i]), i))
    total = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (total[q], q))
        parts[r].append(i)
        total[r] += float(loads[i])
    return [sorted(p) for p in parts]


def agent_loads(agents, tasks) -> list[float]:
    """Work estimate per agent: its transitions times the summed location
    counts of the tasks (its products' transition count up to the trap and
    done pruning)."""
    locs = sum(int(t.n_locs) for t in tasks)
    return [float(len(a.succ)) * locs for a in agents]


def sub_weights(W: np.ndarray, agent_ids: Sequence[int], n_agents: int) -> np.ndarray:
    """The columns of W[K][|I|+|J|] that a shard with `agent_ids` uses."""
    W = np.atleast_2d(np.asarray(W, np.float64))
    cols = list(agent_ids) + list(range(n_agents, W.shape[1]))
    return np.ascontiguousarray(W[:, cols])


def assemble_c(parts: Sequence[np.ndarray], ids_by_rank: Sequence[Sequence[int]], n_agents: int) -> np.ndarray:
    """c[K][|I|][|J|] from the per-rank blocks c_r[K][rows_r][|J|] (blocks may be
    padded with extra rows beyond len(ids_by_rank[r]))."""
    K, _, nJ = parts[0].shape
    C = np.zeros((K, n_agents, nJ))
    for part, ids in zip(parts, ids_by_rank):
        for row, i in enumerate(ids):
            C[:, i, :] = part[:, row, :]
    return C


def owned_pairs(assign: np.ndarray, agent_ids: Sequence[int], n_tasks: int):
    """(local product index, weight index, agent, task) of the assigned pairs
    a shard owns; local product index = local agent row * |J| + j."""
    row = {i: r for r, i in enumerate(agent_ids)}
    out = []
    for k in range(assign.shape[0]):
        for j in range(n_tasks):
            i = int(assign[k, j])
            if i >= 0 and i in row:
                out.append((row[i] * n_tasks + j, k, i, j))
    return out


class EngineShard:
    """The products of some agents with every task, on this process's GPU."""

    def __init__(self, agents, tasks, agent_ids: Sequence[int], cfg=None, stream=None):
        self.agent_ids = list(agent_ids)
        self.n_agents = len(agents)
        self.n_tasks = len(tasks)
        self.stream = stream
        self.ctx = None
        if self.agent_ids:
            self.ctx = M.Context(cfg)
            self.ctx.add([agents[i] for i in self.agent_ids], tasks)
            self.ctx.build(stream)

    def optimise(self, W: np.ndarray):
        """Algorithm 3 for the shard's products: (c[K][rows][|J|], not_converged)."""
        K = np.atleast_2d(W).shape[0]
        if self.ctx is None:
            return np.zeros((K, 0, self.n_tasks)), False
        out = M.morap_solve(self.ctx.h, sub_weights(W, self.agent_ids, self.n_agents), len(self.agent_ids),
                            self.n_tasks, self.stream, evaluate=False)
        return out["c"], out["code"] == M.ENOTCONV

    def evaluate(self, assign: np.ndarray):
        """Algorithm 4 for the assigned pairs the shard owns: (r[K][|I|+|J|]
        with only those entries set, not_converged)."""
        K = assign.shape[0]
        r = np.zeros((K, self.n_agents + self.n_tasks))
        pairs = owned_pairs(assign, self.agent_ids, self.n_tasks)
        if not pairs:
            return r, False
        ev = M.morap_evaluate(self.ctx.h, [p for p, _, _, _ in pairs], [k for _, k, _, _ in pairs], self.stream)
        for e, (_, k, i, j) in enumerate(pairs):
            r[k, i] = ev["r_cost"][e]
            r[k, self.n_agents + j] = ev["r_prob"][e]
        return r, ev["code"] == M.ENOTCONV

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
    collectives.  `ids_by_rank` is the partition every rank agreed on."""

    def __init__(self, shard, ids_by_rank: Sequence[Sequence[int]], n_agents: int, n_tasks: int, comm):
        self.shard = shard
        self.ids_by_rank = [list(x) for x in ids_by_rank]
        self.n_agents, self.n_tasks = n_agents, n_tasks
        self.comm = comm
        self.rows = max(1, max(len(x) for x in self.ids_by_rank))

    def __call__(self, W: np.ndarray) -> dict:
        W = np.atleast_2d(np.asarray(W, np.float64))
        K = W.shape[0]
        c, nc1 = self.shard.optimise(W)
        block = np.zeros((K, self.rows, self.n_tasks))
        block[:, : c.shape[1], :] = c
        C = assemble_c(self.comm.all_gather(block), self.ids_by_rank, self.n_agents)
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
