"""The sharded driver's per-rank steps on one GPU: two shards (products
dealt by the partition rule, each a context restricted to its pairs), their
c blocks assembled, the assignment taken once,
Algorithm 4 run per shard on the pairs it owns.  The result must be
bit-identical to one context holding every product (per-pair results do not
depend on the batch), and morap_evaluate must reject what it cannot do."""

import numpy as np
import pytest

import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch

    assert torch.cuda.is_available()
    from paper_2305_04397_gb300 import build

    build.build()
    from paper_2305_04397_gb300 import morap

    return morap


def test_two_shards_equal_one_context_bitwise(M):
    from paper_2305_04397_gb300 import sharded as S

    g = I.config_grid32()
    agents, tasks = g.agents[:4], g.tasks[:6]
    nI, nJ = len(agents), len(tasks)
    W = np.ascontiguousarray(g.weights[:5][:, list(range(4)) + list(range(10, 16))])
    W = W / W.sum(axis=1, keepdims=True)
    full = M.Context()
    full.add(agents, tasks)
    full.build()
    ref = full.supporting_points(W, want_c=True)
    parts = S.partition_products(S.product_loads(agents, tasks), 2)
    assert all(parts)
    shards = [S.EngineShard(agents, tasks, pairs) for pairs in parts]
    blocks = [s.optimise(W)[0] for s in shards]
    C = S.assemble_c(blocks, parts, nI, nJ)
    assert np.array_equal(C, ref["c"].reshape(C.shape))
    with pytest.raises(M.MorapError) as e:  # a context with a pair list has no assignment step
        shards[0].ctx.supporting_points(W)
    assert e.value.code == M.ESTATE
    assign = M.morap_assign_tasks(C)
    assert np.array_equal(assign, ref["assign"])
    r = sum(s.evaluate(assign)[0] for s in shards)
    assert np.array_equal(r, ref["r"])
    for s in shards:
        s.close()
    full.close()


def test_evaluate_errors(M):
    tiny = I.config_tiny()
    ctx = M.Context()
    ctx.add(tiny.agents, tiny.tasks)
    ctx.build()
    with pytest.raises(M.MorapError) as e:
        M.morap_evaluate(ctx.h, [0], [0])
    assert e.value.code == M.ESTATE
    ctx.solve(tiny.weights[:2], evaluate=False)
    with pytest.raises(M.MorapError) as e:
        M.morap_evaluate(ctx.h, [0], [2])
    assert e.value.code == M.EINVAL
    with pytest.raises(M.MorapError) as e:
        M.morap_evaluate(ctx.h, [6], [0])
    assert e.value.code == M.EINVAL
    got = M.morap_evaluate(ctx.h, [1, 4], [1, 0])
    full = ctx.solve(tiny.weights[:2], evaluate=True)
    assert got["r_cost"][0] == full["r_cost"][1].reshape(-1)[1]
    assert got["r_prob"][1] == full["r_prob"][0].reshape(-1)[4]
    ctx.close()


def test_sharded_driver_over_nccl_one_rank(M):
    """The driver's collectives over a real NCCL process group (one rank on
    this GPU): the points equal the unsharded context's bit for bit."""
    import os
    import socket

    import torch
    import torch.distributed as dist

    from paper_2305_04397_gb300 import sharded as S

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        g = I.config_grid32()
        agents, tasks = g.agents[:3], g.tasks[:4]
        W = np.ascontiguousarray(g.weights[:4][:, [0, 1, 2, 10, 11, 12, 13]])
        W = W / W.sum(axis=1, keepdims=True)
        parts = S.partition_products(S.product_loads(agents, tasks), 1)
        shard = S.EngineShard(agents, tasks, parts[0])
        sp = S.ShardedSupportingPoints(shard, parts, 3, 4, S.TorchComm(device=torch.device("cuda", 0)))
        got = sp(W)
        full = M.Context()
        full.add(agents, tasks)
        full.build()
        ref = full.supporting_points(W)
        assert np.array_equal(got["r"], ref["r"]) and np.array_equal(got["assign"], ref["assign"])
        q = sp.query(np.array([-30.0, -30.0, -30.0, 0.5, 0.5, 0.5, 0.5]), eps=1e-6, max_iter=20)
        q_ref = full.query(np.array([-30.0, -30.0, -30.0, 0.5, 0.5, 0.5, 0.5]), eps=1e-6, max_iter=20)
        assert q["feasible"] == q_ref["feasible"] and q["iterations"] == q_ref["iterations"]
        assert np.array_equal(q["t_up"], q_ref["t_up"])
        shard.close()
        full.close()
    finally:
        dist.destroy_process_group()
