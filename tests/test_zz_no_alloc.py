"""The allocation-free entry point (morap_plain_vi_noalloc) against the plain
per-model entry point (morap_solve_plain) and the FP64 oracle, through the
C-ABI.

Callers that may not allocate device memory (hosts whose own pool owns the
GPU, real-time loops that forbid allocation after start-up) hand in the
product's CSR and the output buffers themselves; the call keeps its scratch
in a static device array.  Two calls in a row must each match
morap_solve_plain and the oracle on the same product and weights, so
whatever the first call leaves in that array must not leak into the second,
and the device's free memory must not change across a call.  This file is
collected last on purpose.
"""

import numpy as np
import pytest

import instances as I
from oracle import core as O

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available()
    from paper_2305_04397_gb300 import build

    build.build()
    from paper_2305_04397_gb300 import morap as M

    inst = I.config_grid32()
    ctx = M.Context()
    ctx.add(inst.agents[:2], inst.tasks[:4])
    ctx.build()
    yield torch, M, ctx, inst
    ctx.close()


def _device_csr(torch, M, ctx, p):
    D = M.morap_product_download(ctx.h, p)
    info = D["info"]
    n = info["n_states"] - 1  # the done slot is index n
    t = {
        "state_sa": torch.from_numpy(D["state_sa"][: n + 1].astype(np.int32)).cuda(),
        "sa_tr": torch.from_numpy(D["sa_tr"].astype(np.int32)).cuda(),
        "col": torch.from_numpy(D["col"].astype(np.int32)).cuda(),
        "prob": torch.from_numpy(D["prob"].astype(np.float64)).cuda(),
        "cost": torch.from_numpy(D["cost"].astype(np.float64)).cuda(),
    }
    return info, n, t


def _call(M, cfg, info, n, t, wc, wp, values, policy, stream):
    return M.morap_plain_vi_noalloc(
        n, info["n_sa"], t["state_sa"].data_ptr(), t["sa_tr"].data_ptr(), t["col"].data_ptr(),
        t["prob"].data_ptr(), t["cost"].data_ptr(), info["pre_begin"], info["init_local"], wc, wp,
        cfg.eps_vi, cfg.tau_policy, cfg.max_sweeps, values, policy, stream)


def test_noalloc_matches_plain_and_oracle_on_two_calls_in_a_row(env):
    torch, M, ctx, inst = env
    nJ = 4
    cfg = M.morap_config_default()
    calls = [(0 * nJ + 1, 0.002, 0.3), (1 * nJ + 3, 0.0005, 0.05)]
    stream = torch.cuda.current_stream()
    # a warm-up call: the first use of the library's static array on a device
    # loads it (the module's globals), which the driver may place in fresh memory
    info, n, t = _device_csr(torch, M, ctx, calls[0][0])
    values = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    policy = torch.zeros(n, dtype=torch.int32, device="cuda")
    _call(M, cfg, info, n, t, 0.01, 0.5, values.data_ptr(), policy.data_ptr(), stream.cuda_stream)
    checked = 0
    for p, wc, wp in calls:
        info, n, t = _device_csr(torch, M, ctx, p)
        values = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
        policy = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        code, c, sweeps = _call(M, cfg, info, n, t, wc, wp, values.data_ptr(), policy.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before  # the call allocated nothing on the device
        assert code == M.OK
        ref = M.morap_solve_plain(ctx.h, [p], [(wc, wp)], stream.cuda_stream, evaluate=False)
        assert abs(c - ref["c"][0]) < TOL, (p, c, ref["c"][0])
        assert sweeps == int(ref["sweeps_vi"])
        v = values.cpu().numpy()
        assert np.all(np.isfinite(v)) and v[n] == 0.0 and v[info["init_local"]] == c
        # the oracle: the value at the initial state, and the scheduler
        # wherever the oracle's action gap exceeds 1e-9
        i, j = divmod(p, nJ)
        prod = O.Product(inst.agents[i], inst.tasks[j])
        r = O.solve_pair(prod, wc, wp)
        assert abs(c - r["c"]) < TOL
        mu = policy.cpu().numpy()
        assert np.all(mu >= 0) and np.all(mu < 5)
        q = O.q_values(prod, r["rew"], r["x"])
        for u in range(prod.n - 1):
            qa = q[prod.state_ptr[u]:prod.state_ptr[u + 1]]
            m = r["mu"][u]
            others = np.delete(qa, m)
            if len(others) and qa[m] - others.max() > 1e-9:
                assert mu[u] == m, (p, u)
                checked += 1
    assert checked > 100


def test_noalloc_rejects_sizes_over_the_limit(env):
    torch, M, ctx, inst = env
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MorapError) as e:
        M.morap_plain_vi_noalloc(200000, 10, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                 dummy.data_ptr(), 0, 0, 0.1, 0.9, 1e-8, 1e-9, 10, dummy.data_ptr(),
                                 dummy.data_ptr())
    assert e.value.code == M.EINVAL and "at most" in str(e.value)


def test_noalloc_rejects_host_buffers(env):
    """An output buffer that is not device memory of the current device is
    refused on the host, before any kernel could touch it."""
    torch, M, ctx, inst = env
    cfg = M.morap_config_default()
    info, n, t = _device_csr(torch, M, ctx, 0)
    policy = torch.zeros(n, dtype=torch.int32, device="cuda")
    host_values = np.zeros(n + 1)
    with pytest.raises(M.MorapError) as e:
        _call(M, cfg, info, n, t, 0.01, 0.5, host_values.ctypes.data, policy.data_ptr(), None)
    assert e.value.code == M.EINVAL and "values" in str(e.value)


def test_noalloc_refuses_a_capturing_stream(env):
    """The call synchronises after every sweep, so a stream under capture is
    refused before anything is enqueued on it."""
    torch, M, ctx, inst = env
    cfg = M.morap_config_default()
    info, n, t = _device_csr(torch, M, ctx, 0)
    values = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    policy = torch.zeros(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device="cuda")
    err = None
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        x.add_(1.0)
        try:
            _call(M, cfg, info, n, t, 0.01, 0.5, values.data_ptr(), policy.data_ptr(), s.cuda_stream)
        except M.MorapError as ex:
            err = ex
    assert err is not None and err.code == M.EINVAL and "captured" in str(err)
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 4.0
