"""The multi-process path (products of one instance dealt to ranks one by
one, Algorithm 2's c values all-gathered, the assignment replicated, the r
vectors summed) on CPU: world_size-2 and -3 gloo ranks (the latter with
ranks holding different numbers of products) whose per-rank solver is the
oracle.  The sharded supporting points and the Algorithm 1 loop built on
them must equal the oracle's unsharded ones on every rank."""

import os
import socket
import tempfile

import numpy as np
import pytest

import instances as I
from paper_2305_04397_gb300 import sharded as S


class OracleShard:
    """Per-rank work of the sharded driver done by the oracle (one FP64 CPU
    solve per product and weight)."""

    def __init__(self, agents, tasks, pairs):
        from oracle import core as O

        self.O = O
        self.agents, self.tasks = agents, tasks
        self.pairs = [tuple(p) for p in pairs]
        self.n_agents, self.n_tasks = len(agents), len(tasks)
        self.prods = {(i, j): O.Product(agents[i], tasks[j]) for i, j in self.pairs}
        self.last = {}

    def optimise(self, W):
        W = np.atleast_2d(W)
        K, nI = W.shape[0], self.n_agents
        c = np.zeros((K, len(self.pairs)))
        self.last = {}
        for k in range(K):
            for e, (i, j) in enumerate(self.pairs):
                res = self.O.solve_pair(self.prods[(i, j)], W[k][i], W[k][nI + j])
                c[k, e] = res["c"]
                self.last[(k, i, j)] = (res["r_cost"], res["r_prob"])
        return c, False

    def evaluate(self, assign):
        K = assign.shape[0]
        r = np.zeros((K, self.n_agents + self.n_tasks))
        for _, k, i, j in S.owned_pairs(assign, self.pairs):
            r[k, i], r[k, self.n_agents + j] = self.last[(k, i, j)]
        return r, False


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inst = I.config_tiny()
        nI, nJ = len(inst.agents), len(inst.tasks)
        parts = S.partition_products(S.product_loads(inst.agents, inst.tasks), world)
        shard = OracleShard(inst.agents, inst.tasks, parts[rank])
        sp = S.ShardedSupportingPoints(shard, parts, nI, nJ, S.TorchComm())
        out = sp(inst.weights[:3])
        q = sp.query(inst.thresholds[0], eps=1e-6, max_iter=12)
        v = sp.query(inst.thresholds[0], eps=1e-6, max_iter=12, verify_only=True)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), r=out["r"], assign=out["assign"], c=out["c"],
                 t_up=q["t_up"], t_down=q["t_down"], it=q["iterations"], feasible=q["feasible"],
                 w_hist=q["w_hist"], v_feasible=v["feasible"], v_it=v["iterations"])
    finally:
        dist.destroy_process_group()


def test_partition_covers_every_product_once_and_balances():
    rng = np.random.default_rng(4)
    loads = rng.uniform(1.0, 10.0, size=(4, 5))
    for world in (1, 2, 3, 7, 25):
        parts = S.partition_products(loads, world)
        assert len(parts) == world
        flat = sorted(ij for p in parts for ij in p)
        assert flat == [(i, j) for i in range(4) for j in range(5)]
        tot = [sum(loads[ij] for ij in p) for p in parts]
        # greedy LPT: no rank exceeds the lightest by more than the largest load
        assert max(tot) - min(tot) <= loads.max() + 1e-12
        assert parts == S.partition_products(loads, world)
    # 10 agents x 20 tasks on 8 ranks: a partition by agent would cap the
    # speed-up at 5 (2 agents on some rank); by product it is near even
    g = I.config_grid32()
    L = S.product_loads(g.agents, g.tasks)
    parts = S.partition_products(L, 8)
    tot = [sum(L[ij] for ij in p) for p in parts]
    assert max(tot) / (L.sum() / 8) < 1.05


def test_product_loads_follow_size():
    g = I.config_grid32()
    L = S.product_loads(g.agents[:2], [I.sequence_task([1]), I.sequence_task([1, 2, 3])])
    assert np.all(L[:, 1] > L[:, 0])  # more locations: more transitions and a longer horizon


def test_assemble_and_owned_pairs():
    pairs = [[(0, 0), (0, 2), (1, 1)], [(0, 1), (1, 0), (1, 2)]]
    parts = [np.array([[1.0, 2.0, 3.0, 0.0]]), np.array([[4.0, 5.0, 6.0, 0.0]])]  # padded to width 4
    C = S.assemble_c(parts, pairs, 2, 3)
    assert np.array_equal(C[0], np.array([[1.0, 4.0, 2.0], [5.0, 3.0, 6.0]]))
    assign = np.array([[1, -1, 0], [0, 1, -1]])
    assert S.owned_pairs(assign, pairs[0]) == [(1, 0, 0, 2), (0, 1, 0, 0), (2, 1, 1, 1)]
    assert S.owned_pairs(assign, pairs[1]) == [(1, 0, 1, 0)]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_gloo_matches_unsharded_oracle(oracle_lib, world):
    import torch.multiprocessing as mp

    from oracle import core as O
    from oracle import pareto as OP

    inst = I.config_tiny()
    parts = S.partition_products(S.product_loads(inst.agents, inst.tasks), world)
    assert sorted(ij for p in parts for ij in p) == [(i, j) for i in range(2) for j in range(3)]
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True, start_method="spawn")
        res = [dict(np.load(os.path.join(d, f"rank{r}.npz"))) for r in range(world)]
    # every rank holds the same numbers
    for r in range(1, world):
        for key in res[0]:
            assert np.array_equal(res[0][key], res[r][key]), key
    prods = O.products(inst.agents, inst.tasks)
    for k in range(3):
        r, f, C, _, _ = O.supporting_point(prods, inst.weights[k])
        assert np.max(np.abs(res[0]["c"][k] - C)) < 1e-12
        assert np.array_equal(res[0]["assign"][k], np.where(f < len(inst.agents), f, -1))
        assert np.max(np.abs(res[0]["r"][k] - r)) < 1e-12
    ref = OP.alg1(lambda w: O.supporting_point(prods, w)[0], inst.thresholds[0], eps=1e-6, max_iter=12)
    ver = OP.alg1(lambda w: O.supporting_point(prods, w)[0], inst.thresholds[0], eps=1e-6, max_iter=12,
                  verify_only=True)
    assert bool(res[0]["v_feasible"]) == ver["feasible"] and int(res[0]["v_it"]) == ver["iterations"]
    assert int(res[0]["it"]) == ref["iterations"]
    assert bool(res[0]["feasible"]) == ref["feasible"]
    assert np.max(np.abs(res[0]["t_up"] - ref["t_up"])) < 1e-6
    assert np.max(np.abs(res[0]["t_down"] - ref["t_dn"])) < 1e-6


def test_sharded_world1_equals_local_driver(oracle_lib):
    """One shard with every product and loop-back collectives gives the oracle's
    supporting point (the gather / reduce bookkeeping is the identity)."""

    class Loop:
        def all_gather(self, a):
            return [a]

        def all_reduce_sum(self, a):
            return a

    from oracle import core as O

    inst = I.config_tiny()
    nI, nJ = len(inst.agents), len(inst.tasks)
    every = [(i, j) for i in range(nI) for j in range(nJ)]
    sp = S.ShardedSupportingPoints(OracleShard(inst.agents, inst.tasks, every), [every], nI, nJ, Loop())
    out = sp(inst.weights[1:2])
    r, _, _, _, _ = O.supporting_point(O.products(inst.agents, inst.tasks), inst.weights[1])
    assert np.max(np.abs(out["r"][0] - r)) < 1e-12 and out["code"] == 0
