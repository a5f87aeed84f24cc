"""The allocation-free entry point (morap_plain_vi_noalloc) against the plain
per-model entry point (morap_solve_plain), through the C-ABI.

Callers that may not allocate device memory (graph capture, hosts whose own
pool owns the GPU, real-time loops) hand in the product's CSR and the output
buffers themselves; the call keeps its scratch in a static device array.
Two calls in a row must each match morap_solve_plain on the same product and
weights, so whatever the first call leaves in that array must not leak into
the second.  This file is collected last on purpose.
"""

import numpy as np
import pytest

import instances as I

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


def test_noalloc_matches_plain_on_two_calls_in_a_row(env):
    torch, M, ctx, inst = env
    nJ = 4
    cfg = M.morap_config_default()
    calls = [(0 * nJ + 1, 0.002, 0.3), (1 * nJ + 3, 0.0005, 0.05)]
    stream = torch.cuda.current_stream()
    for p, wc, wp in calls:
        info, n, t = _device_csr(torch, M, ctx, p)
        values = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
        policy = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        code, c, sweeps = M.morap_plain_vi_noalloc(
            n, info["n_sa"], t["state_sa"].data_ptr(), t["sa_tr"].data_ptr(), t["col"].data_ptr(),
            t["prob"].data_ptr(), t["cost"].data_ptr(), info["pre_begin"], info["init_local"], wc, wp,
            cfg.eps_vi, cfg.tau_policy, cfg.max_sweeps, values.data_ptr(), policy.data_ptr(), stream.cuda_stream)
        assert code == M.OK
        ref = M.morap_solve_plain(ctx.h, [p], [(wc, wp)], stream.cuda_stream, evaluate=False)
        assert abs(c - ref["c"][0]) < TOL, (p, c, ref["c"][0])
        assert sweeps == int(ref["sweeps_vi"])
        v = values.cpu().numpy()
        assert np.all(np.isfinite(v)) and v[n] == 0.0 and v[info["init_local"]] == c
        mu = policy.cpu().numpy()
        assert np.all(mu >= 0) and np.all(mu < 5)


def test_noalloc_rejects_sizes_over_the_limit(env):
    torch, M, ctx, inst = env
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MorapError) as e:
        M.morap_plain_vi_noalloc(200000, 10, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                 dummy.data_ptr(), 0, 0, 0.1, 0.9, 1e-8, 1e-9, 10, dummy.data_ptr(),
                                 dummy.data_ptr())
    assert e.value.code == M.EINVAL and "at most" in str(e.value)
