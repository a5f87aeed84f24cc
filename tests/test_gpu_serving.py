"""Serving (morap_server_*): continuous batching of threshold-point queries
over several resident instances.  Each query's result is the same alone
(morap_query on the instance) and in the mix, and admission by device
footprint limits the queries in flight without changing any result."""

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


def _instances(M):
    tiny = I.config_tiny()
    g = I.config_grid32()
    pairs = [(tiny.agents, tiny.tasks), ([I.fig2_agent()], [I.fig2_task()]), (g.agents[:3], g.tasks[:4])]
    ctxs = []
    for a, t in pairs:
        c = M.Context()
        c.add(a, t)
        c.build()
        ctxs.append(c)
    return ctxs


def _queries(ctxs, n, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        i = int(rng.integers(0, len(ctxs)))
        nI, nJ = ctxs[i].n_agents, ctxs[i].n_tasks
        c = -rng.uniform(1.0, 12.0, size=nI)
        p = rng.uniform(0.1, 0.95, size=nJ)
        out.append((i, np.concatenate([c, p])))
    return out


@pytest.mark.parametrize("budget_slots,merge", [(0, 1), (1, 1), (0, 0), (1, 0)])
def test_results_same_alone_and_in_the_mix(M, budget_slots, merge):
    """Both batching modes: rounds across instances (merge = 1, one context
    holding every instance's products) and per-instance batches."""
    ctxs = _instances(M)
    qs = _queries(ctxs, 24)
    budget = 0
    if budget_slots:
        # room for about one weight slot of the largest instance at a time
        budget = max(sum(M.morap_product_info(c.h, p)["n_states"] for p in range(c.n_agents * c.n_tasks)) * 26
                     for c in ctxs)
    srv = M.Server(ctxs, max_batch=16, n_workers=3, eps=1e-6, max_iter=40, hbm_budget=budget, merge_instances=merge)
    tickets = [srv.submit(i, t) for i, t in qs]
    assert srv.wait(600.0) == M.OK
    mixed = [srv.poll(tk, i) for tk, (i, _) in zip(tickets, qs)]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(qs) and st["p99_ms"] >= st["p50_ms"] > 0
    if budget_slots:
        assert st["mean_batch"] <= 2.0
    else:
        assert st["mean_batch"] >= 1.0
    for (i, t), got in zip(qs, mixed):
        alone = ctxs[i].query(t, eps=1e-6, max_iter=40)
        assert got["feasible"] == alone["feasible"]
        assert got["iterations"] == alone["iterations"]
        assert np.max(np.abs(got["t_down"] - alone["t_down"])) < 1e-9
        assert np.max(np.abs(got["t_up"] - alone["t_up"])) < 1e-9
    for c in ctxs:
        c.close()
