"""Parity of the CUDA engine with the FP64 oracle, through the C-ABI.

Tolerances (the benchmark spec): per-objective values within 1e-6 absolute at
eps_vi = 1e-8; schedulers identical wherever the oracle's action gap
exceeds 1e-9; product CSRs identical (structure exact, probabilities
bit-exact).  Full-size checks run the 10 x 20 grid instance in the launch
configuration the benchmark times (one supporting-point batch of K = 16)
and compare sampled products one by one.
"""

import numpy as np
import pytest

import instances as I
from oracle import core as O
from oracle import pareto as OP

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def M():
    import torch

    assert torch.cuda.is_available()
    from paper_2305_04397_gb300 import build

    build.build()
    from paper_2305_04397_gb300 import morap

    return morap


def make_ctx(M, inst_or_pair, **cfg_kw):
    cfg = M.morap_config_default()
    for k, v in cfg_kw.items():
        setattr(cfg, k, v)
    ctx = M.Context(cfg)
    agents, tasks = (inst_or_pair.agents, inst_or_pair.tasks) if hasattr(inst_or_pair, "agents") else inst_or_pair
    ctx.add(agents, tasks)
    ctx.build()
    return ctx


@pytest.fixture(scope="module")
def tiny():
    return I.config_tiny()


@pytest.fixture(scope="module")
def tiny_prods(tiny):
    return O.products(tiny.agents, tiny.tasks)


def tiny_weights(tiny):
    extra = np.array([[0.01, 0.02, 0.5, 0.3, 0.17], [0.2, 0.2, 0.2, 0.2, 0.2], [0.0, 0.0, 1.0, 0.0, 0.0]])
    return np.vstack([tiny.weights, extra])


def canon_device(D):
    info = D["info"]
    S, n = info["S"], info["n_states"]
    done = n - 1
    out = {}
    for u in range(n - 1):
        key_s = (u % S, int(D["loc"][u // S]))
        for a in range(D["state_sa"][u + 1] - D["state_sa"][u]):
            sa = D["state_sa"][u] + a
            row = {}
            for t in range(D["sa_tr"][sa], D["sa_tr"][sa + 1]):
                c = int(D["col"][t])
                k = ("DONE",) if c == done else (c % S, int(D["loc"][c // S]))
                assert k not in row, ("a successor listed twice in one row", key_s, a, k)
                row[k] = float(D["prob"][t])
            out[key_s + (a,)] = (row, float(D["cost"][sa]))
    return out


def canon_oracle(p):
    out = {}
    for u in range(p.n - 1):
        ks = p.key(u)
        for a in range(p.state_ptr[u + 1] - p.state_ptr[u]):
            sa = p.state_ptr[u] + a
            row = {p.key(int(p.col[t])): float(p.prob[t]) for t in range(p.sa_ptr[sa], p.sa_ptr[sa + 1])}
            out[ks + (a,)] = (row, float(p.sa_cost[sa]))
    return out


# ------------------------------------------------------------- products


def test_product_csr_matches_oracle(M, tiny):
    """Product CSRs (Sec. 2, product MDP) equal the oracle's after a
    canonical sort: same rows, same successors (each listed once: those
    whose location is done merged into the done slot, probabilities summed),
    probabilities and costs bit for bit, the same transition count."""
    g = I.config_grid32()
    for agents, tasks in [(tiny.agents, tiny.tasks), ([I.fig2_agent()], [I.fig2_task()]),
                          (g.agents[:2], g.tasks[:3])]:
        ctx = make_ctx(M, (agents, tasks))
        for i, a in enumerate(agents):
            for j, t in enumerate(tasks):
                D = M.morap_product_download(ctx.h, i * len(tasks) + j)
                p = O.Product(a, t)
                assert D["info"]["n_states"] == p.n
                assert D["info"]["n_trans"] == p.n_trans  # duplicate successors merged, as in the oracle
                assert canon_device(D) == canon_oracle(p)
                assert p.key(p.init) == (("DONE",) if D["info"]["init_local"] == p.n - 1 else
                                         (D["info"]["init_local"] % D["info"]["S"],
                                          int(D["loc"][D["info"]["init_local"] // D["info"]["S"]])))
        ctx.close()


# ------------------------------------------------------------- Algorithm 3 / 4


def _oracle_pairs(prods, W, nI, nJ):
    K = len(W)
    c = np.zeros((K, nI, nJ))
    rc = np.zeros_like(c)
    rp = np.zeros_like(c)
    res = {}
    for k, w in enumerate(W):
        for i in range(nI):
            for j in range(nJ):
                r = O.solve_pair(prods[i][j], w[i], w[nI + j])
                c[k, i, j], rc[k, i, j], rp[k, i, j] = r["c"], r["r_cost"], r["r_prob"]
                res[k, i, j] = r
    return c, rc, rp, res


@pytest.mark.parametrize("precision,polish", [(0, 0), (0, 1), (1, 1)])
def test_solve_matches_oracle(M, tiny, tiny_prods, precision, polish):
    W = tiny_weights(tiny)
    nI, nJ = len(tiny.agents), len(tiny.tasks)
    ctx = make_ctx(M, tiny, precision=precision, polish=polish)
    out = ctx.solve(W)
    c, rc, rp, res = _oracle_pairs(tiny_prods, W, nI, nJ)
    assert np.all(out["status"] == 0)
    assert np.max(np.abs(out["c"] - c)) < TOL
    # A zero weight on one of the pair's two objectives leaves that objective
    # free among the optimal schedulers (ties), so only the weighted one and
    # the scalarised value are unique there; otherwise both must match.
    wc = W[:, :nI][:, :, None] * np.ones((1, 1, nJ))
    wp = W[:, nI:][:, None, :] * np.ones((1, nI, 1))
    both = (wc > 0) & (wp > 0)
    assert np.max(np.abs(out["r_cost"] - rc)[both | ((wc > 0) & (wp == 0))]) < TOL
    assert np.max(np.abs(out["r_prob"] - rp)[both | ((wp > 0) & (wc == 0))]) < TOL
    assert np.max(np.abs(wc * out["r_cost"] + wp * out["r_prob"] - c)) < TOL
    # schedulers: identical wherever the oracle's action gap exceeds 1e-9
    checked = 0
    for k in range(len(W)):
        for i in range(nI):
            for j in range(nJ):
                p = tiny_prods[i][j]
                r = res[k, i, j]
                mu, _ = M.morap_last_policy(ctx.h, k, i * nJ + j)
                q = O.q_values(p, r["rew"], r["x"])
                for u in range(p.n - 1):
                    a0, a1 = p.state_ptr[u], p.state_ptr[u + 1]
                    qa = q[a0:a1]
                    m = r["mu"][u]
                    others = np.delete(qa, m)
                    gap = qa[m] - (others.max() if len(others) else -np.inf)
                    if gap > 1e-9:
                        assert mu[u] == m, (k, i, j, u)
                        checked += 1
    assert checked > 20
    st = ctx.stats()
    if precision == 0:
        assert st["fp32_sweeps"] > 0 and st["polish"] == polish
    else:
        assert st["fp32_sweeps"] == 0 and st["polish"] == 1
    ctx.close()


def test_fp64_only_path_without_free_action(M):
    """The Fig. 2 agent has no zero-cost action, so the engine runs FP64 from
    0 (the FP32 lower-bound argument needs one); values match the oracle."""
    a, t = I.fig2_agent(), I.fig2_task()
    ctx = make_ctx(M, ([a], [t]))
    W = np.array([[1.0, 0.0], [0.4, 0.6], [0.0, 1.0], [0.2, 0.8]])
    out = ctx.solve(W)
    p = O.Product(a, t)
    for k, w in enumerate(W):
        r = O.solve_pair(p, w[0], w[1])
        assert out["c"][k, 0, 0] == pytest.approx(r["c"], abs=TOL)
        assert out["r_cost"][k, 0, 0] == pytest.approx(r["r_cost"], abs=TOL)
        assert out["r_prob"][k, 0, 0] == pytest.approx(r["r_prob"], abs=TOL)
    assert ctx.stats()["fp32_sweeps"] == 0
    # the paper's printed r1 for w = (1, 0)
    assert out["r_cost"][0, 0, 0] == pytest.approx(-1.1, abs=1e-9)
    assert out["r_prob"][0, 0, 0] == pytest.approx(0.1, abs=1e-9)
    ctx.close()


# ------------------------------------------------------------- Algorithm 2


def _check_supporting(out, prods, W, nI, nJ):
    for k, w in enumerate(W):
        r, f, C, RC, RP = O.supporting_point(prods, w)
        Cp = O.pad_square(C)
        fg = out["assign"][k]
        real = [i for i in fg if i >= 0]
        assert len(set(real)) == len(real)  # a (partial) permutation
        # the engine's assignment is optimal for the oracle's c matrix
        tot = sum(C[fg[j], j] for j in range(nJ) if fg[j] >= 0)
        best = sum(Cp[f[j], j] for j in range(nJ))
        assert tot == pytest.approx(best, abs=TOL)
        assert w @ out["r"][k] == pytest.approx(w @ r, abs=TOL)
        # r is the point of that assignment (both objectives are unique only
        # when both weights of the pair are positive)
        for j in range(nJ):
            i = fg[j]
            if i >= 0 and w[i] > 0 and w[nI + j] > 0:
                assert out["r"][k][nI + j] == pytest.approx(RP[i, j], abs=TOL)
                assert out["r"][k][i] == pytest.approx(RC[i, j], abs=TOL)


def test_supporting_points_match_oracle(M, tiny, tiny_prods):
    W = tiny_weights(tiny)
    ctx = make_ctx(M, tiny)
    out = ctx.supporting_points(W)
    _check_supporting(out, tiny_prods, W, len(tiny.agents), len(tiny.tasks))
    ctx.close()


# ------------------------------------------------------------- Algorithm 1


def test_query_matches_oracle_alg1(M, tiny, tiny_prods):
    """Algorithm 1 on the tiny instance for three thresholds.  Directions
    after the first have zero weights on the objectives t_up already meets,
    where the supporting point is not unique (tied assignments or
    schedulers; the two sides break ties differently), so two correct runs
    may take different paths.  Checked: every point of the engine's run is a
    supporting point (w.r equals the oracle's optimum for w, unique); the
    oracle's Algorithm 1 fed the engine's points reproduces the engine's
    directions, t_up, t_down, iteration count and verdict to 1e-6; the
    verdict equals the oracle's own run, and the two runs' final t_down lie
    within the distance Thm 3 allows (both bound the projection of t onto
    the achievable set); the synthesis is a valid random assignment."""
    ctx = make_ctx(M, tiny)
    for t in [tiny.thresholds[0], np.array([-12.0, -12.0, 0.6, 0.6, 0.6]), np.array([-1.0, -1.0, 0.2, 0.2, 0.2])]:
        got = ctx.query(t, eps=1e-6, max_iter=40)
        W, R = got["w_hist"], got["r_hist"]
        # every point is a supporting point of its direction
        for w, r in zip(W, R):
            best = O.supporting_point(tiny_prods, w)[0]
            assert abs(w @ r - w @ best) < TOL
        # the loop's arithmetic, fed the engine's points
        fed = iter(R)
        replay = OP.alg1(lambda w: next(fed), t, eps=1e-6, max_iter=40)
        assert replay["iterations"] == got["iterations"] and replay["feasible"] == got["feasible"]
        assert np.max(np.abs(np.array([h["w"] for h in replay["history"]]) - W)) < TOL
        assert np.max(np.abs(replay["t_dn"] - got["t_down"])) < TOL
        assert np.max(np.abs(replay["t_up"] - got["t_up"])) < TOL
        # the oracle's own run: same verdict; both final outer bounds are
        # within sqrt(2 eps d) + eps of the projection of t (d = |t - t_down|)
        own = OP.alg1(lambda w: O.supporting_point(tiny_prods, w)[0], t, eps=1e-6, max_iter=40)
        assert own["feasible"] == got["feasible"]
        d = max(np.linalg.norm(t - own["t_dn"]), np.linalg.norm(t - got["t_down"]))
        assert np.linalg.norm(own["t_dn"] - got["t_down"]) <= 2 * (np.sqrt(2e-6 * d) + 1e-6)
        # Lemma 6 on every direction the engine produced
        for w in W:
            assert np.all(w >= 0) and abs(w.sum() - 1) < 1e-9
        # the synthesis: a convex combination of the supporting points that
        # dominates t_up (and t itself when t is feasible), and a random
        # assignment in which no agent and no task is used more than once
        lam, F = got["lambda"], got["assign_hist"]
        assert np.all(lam >= 0) and abs(lam.sum() - 1) < 1e-12
        assert np.all(lam @ R >= got["t_up"] - 1e-7)
        if got["feasible"]:
            assert np.all(lam @ R >= t - 1e-7)
        P = M.random_assignment(lam, F, len(tiny.agents))
        assert np.all(P.sum(axis=0) <= 1 + 1e-12) and np.all(P.sum(axis=1) <= 1 + 1e-12)
        # the random assignment of the C-ABI is the sum of the convex weights
        # of the points that give task j to agent i (the weights behind t_up
        # are not unique when points are affinely dependent, so they are not
        # compared with the oracle's)
        P_sum = np.zeros_like(P)
        for l, f in enumerate(F):
            for j, i in enumerate(f):
                if i >= 0:
                    P_sum[i, j] += lam[l]
        assert np.max(np.abs(P - P_sum)) < 1e-15
        # the oracle's weights for the same points dominate the same t_up
        assert np.all(replay["lambda"] @ R >= got["t_up"] - 1e-7)
    ctx.close()


def test_verify_matches_query_and_oracle(M, tiny, tiny_prods):
    """The verification-only loop (Sec. 5, Exp. 2) through the C-ABI: the
    verdict of morap_query and of the oracle's verification-only loop, in no
    more iterations, with the same directions as the full loop up to its
    stop."""
    ctx = make_ctx(M, tiny)
    for t in [tiny.thresholds[0], np.array([-12.0, -12.0, 0.6, 0.6, 0.6]), np.array([-1.0, -1.0, 0.2, 0.2, 0.2])]:
        full = ctx.query(t, eps=1e-6, max_iter=40)
        ver = ctx.verify(t, eps=1e-6, max_iter=40)
        supp = lambda w: O.supporting_point(tiny_prods, w)[0]
        want = OP.alg1(supp, t, eps=1e-6, max_iter=40, verify_only=True)
        assert ver["feasible"] == full["feasible"] == want["feasible"] and ver["converged"]
        assert ver["iterations"] <= full["iterations"]
        assert np.array_equal(ver["w_hist"], full["w_hist"][: ver["iterations"]])
        # the oracle's verification-only loop fed the engine's points stops
        # at the same point with the same verdict
        fed = iter(ver["r_hist"])
        replay = OP.alg1(lambda w: next(fed), t, eps=1e-6, max_iter=40, verify_only=True)
        assert replay["iterations"] == ver["iterations"] and replay["feasible"] == ver["feasible"]
    ctx.close()


def test_query_verdicts_match_the_lp_oracle(M, tiny, tiny_prods):
    """The engine's Algorithm 1 verdicts (full and verification-only)
    against the LP formulation of MORAP solved by the oracle's simplex,
    which shares nothing with value iteration or Algorithm 1."""
    from oracle import lp as L

    ctx = make_ctx(M, tiny)
    rng = np.random.default_rng(17)
    ts = [np.array([-12.0, -12.0, 0.6, 0.6, 0.6]), np.array([-1.0, -1.0, 0.2, 0.2, 0.2])]
    ts += [np.concatenate([-rng.uniform(2, 14, 2), rng.uniform(0.1, 0.95, 3)]) for _ in range(4)]
    seen = set()
    for t in ts:
        full = ctx.query(t, eps=1e-7, max_iter=60)
        if not full["feasible"] and np.linalg.norm(full["t_down"] - t) < 1e-4:
            continue  # too close to the boundary to call
        ok, _ = L.morap_feasible(tiny_prods, t)
        assert full["feasible"] == ok, t
        assert ctx.verify(t, eps=1e-7, max_iter=60)["feasible"] == ok, t
        seen.add(ok)
    assert seen == {True, False}
    ctx.close()


def test_query_fig2(M):
    ctx = make_ctx(M, ([I.fig2_agent()], [I.fig2_task()]))
    prods = [[O.Product(I.fig2_agent(), I.fig2_task())]]
    supp = lambda w: O.supporting_point(prods, w)[0]
    for t in ([-1.8, 0.9], [-3.0, 0.5], [-2.5, 0.7]):
        got = ctx.query(np.array(t), eps=1e-7)
        want = OP.alg1(supp, np.array(t), eps=1e-7)
        assert got["feasible"] == want["feasible"] and got["iterations"] == want["iterations"]
        assert np.max(np.abs(got["t_down"] - want["t_dn"])) < TOL
        assert np.max(np.abs(got["t_up"] - want["t_up"])) < TOL
    ctx.close()


def test_query_grid32_subinstance_matches_oracle_alg1(M):
    """Algorithm 1 on a 3-agent x 4-task sub-instance of the 32x32 grid batch
    (12 products of ~3.5k states), for a threshold the loop finds achievable
    and one it does not.  After the first point every direction has zero
    weights on the objectives t_up already meets, so the supporting point of
    such a direction is not unique (the Hungarian step may pick any of the
    tied assignments, and both sides' tie-breaks differ), and two correct
    runs may take different paths.  So the run is checked part by part:
      * every point of the engine's run is a supporting point: w.r equals the
        oracle's optimum for that w (unique) to 1e-6;
      * the loop itself: the oracle's Algorithm 1 fed the engine's points
        reproduces the engine's directions, t_up, t_down, iteration count and
        verdict to 1e-6;
      * the verdict equals that of the oracle's own run."""
    inst = I.config_grid32()
    agents, tasks = inst.agents[:3], inst.tasks[:4]
    prods = O.products(agents, tasks)
    ctx = make_ctx(M, (agents, tasks))
    seen = set()
    for t in (np.array([-150.0, -150.0, -150.0, 0.3, 0.3, 0.3, 0.0]),
              np.array([-30.0, -30.0, -30.0, 0.95, 0.95, 0.95, 0.95])):
        got = ctx.query(t, eps=1e-6, max_iter=40)
        W, R = got["w_hist"], got["r_hist"]
        for w, r in zip(W, R):
            best = O.supporting_point(prods, w)[0]
            assert abs(w @ r - w @ best) < TOL
        fed = iter(R)
        replay = OP.alg1(lambda w: next(fed), t, eps=1e-6, max_iter=40)
        assert replay["iterations"] == got["iterations"] and replay["feasible"] == got["feasible"]
        assert np.max(np.abs(np.array([h["w"] for h in replay["history"]]) - W)) < TOL
        assert np.max(np.abs(replay["t_dn"] - got["t_down"])) < TOL
        assert np.max(np.abs(replay["t_up"] - got["t_up"])) < TOL
        own = OP.alg1(lambda w: O.supporting_point(prods, w)[0], t, eps=1e-6, max_iter=40)
        assert own["feasible"] == got["feasible"]
        seen.add(bool(got["feasible"]))
    assert seen == {True, False}
    ctx.close()


@pytest.mark.parametrize("precision,polish", [(0, 0), (0, 1), (1, 1)])
def test_tie_fallback_anchoring_matches_oracle(M, precision, polish):
    """A recorded action that went stale with a zero weight on the cost:
    on the final values "go to the neighbour" ties at two states, and the
    plain lowest-index fallback would send the run between them forever.
    The engine's scheduler (batched and plain paths) must reach the goal with
    the optimal probability, c and r as the oracle's."""
    a, t = I.tie_drift_agent(), I.sequence_task([0])
    p = O.Product(a, t)
    ctx = make_ctx(M, ([a], [t]), precision=precision, polish=polish)
    W = np.array([[0.0, 1.0], [0.0, 0.25], [0.01, 0.99]])
    out = ctx.solve(W)
    assert np.all(out["status"] == 0)
    for k, w in enumerate(W):
        r = O.solve_pair(p, w[0], w[1])
        assert out["c"][k, 0, 0] == pytest.approx(r["c"], abs=TOL)
        assert out["r_prob"][k, 0, 0] == pytest.approx(r["r_prob"], abs=TOL)
        assert out["r_prob"][k, 0, 0] == pytest.approx(1.0, abs=TOL)
        if w[0] > 0:
            assert out["r_cost"][k, 0, 0] == pytest.approx(r["r_cost"], abs=TOL)
        assert w[0] * out["r_cost"][k, 0, 0] + w[1] * out["r_prob"][k, 0, 0] == pytest.approx(out["c"][k, 0, 0],
                                                                                            abs=TOL)
    plain = M.morap_solve_plain(ctx.h, [0, 0], [(0.0, 1.0), (0.0, 0.25)])
    assert np.max(np.abs(plain["r_prob"] - 1.0)) < TOL
    assert np.max(np.abs(plain["c"] - out["c"][:2, 0, 0])) < TOL
    ctx.close()


@pytest.mark.parametrize("eval_block", [0, 1])
def test_tasks_done_at_the_start(M, eval_block):
    """A task whose initial location is accepting (every location done: the
    product has no non-done state) and one whose initial location is a trap
    (the product has non-done states the run never enters): every pair
    converges and c, r_cost and r_prob are 0, as in the oracle."""
    t_acc = I.Task(1, 0, 1, np.array([0], np.int32), np.array([0, 0], np.int32), np.array([1], np.uint8), {})
    delta = np.array([[0, 0], [1, 2], [2, 2]], np.int32).reshape(-1)
    t_trap = I.Task(3, 0, 1, np.array([0], np.int32), delta, np.array([0, 0, 1], np.uint8), {})
    a = I.grid_agent(4, 4, 0.1, (0, 0))
    ctx = make_ctx(M, ([a], [t_acc, t_trap, I.sequence_task([I.GRID_AP(3, 3)])]), eval_block=eval_block)
    W = np.array([[0.3, 0.7, 0.0, 0.0], [0.2, 0.0, 0.4, 0.4]])
    out = ctx.solve(W)
    assert np.all(out["status"] == 0)
    for j, t in enumerate((t_acc, t_trap)):
        r = O.solve_pair(O.Product(a, t), 0.3, 0.7)
        assert r["c"] == r["r_cost"] == r["r_prob"] == 0.0
        assert np.all(out["c"][:, 0, j] == 0.0) and np.all(out["r_cost"][:, 0, j] == 0.0)
        assert np.all(out["r_prob"][:, 0, j] == 0.0)
    sp = ctx.supporting_points(W)
    assert sp["r"][:, 1:3].max() == 0.0 and ctx.stats()["pairs_not_converged"] == 0
    ctx.close()


# ------------------------------------------------------------- full size


@pytest.fixture(scope="module")
def grid32():
    return I.config_grid32()


def test_grid32_full_size_sampled(M, grid32):
    """10 agents x 20 tasks (200 products of ~3.5k states) with K = 16 in one
    supporting-point batch (the benchmark's launch); sampled products are
    recomputed by the oracle one by one."""
    inst = grid32
    nI, nJ = len(inst.agents), len(inst.tasks)
    ctx = make_ctx(M, inst)
    W = inst.weights
    out = ctx.supporting_points(W, want_c=True)
    st = ctx.stats()
    assert st["pairs_not_converged"] == 0
    rng = np.random.default_rng(0)
    sample = [(int(i), int(j)) for i, j in zip(rng.integers(0, nI, 5), rng.integers(0, nJ, 5))]
    sample += [(int(out["assign"][k][j]), j) for k, j in [(3, 0), (7, 5), (11, 19)] if out["assign"][k][j] >= 0]
    checked = 0
    for n_s, (i, j) in enumerate(sample):
        p = O.Product(inst.agents[i], inst.tasks[j])
        for k in range(len(W)):
            r = O.solve_pair(p, W[k][i], W[k][nI + j])
            assert out["c"][k, i, j] == pytest.approx(r["c"], abs=TOL), (i, j, k)
            if out["assign"][k][j] == i:
                assert out["r"][k][i] == pytest.approx(r["r_cost"], abs=TOL), (i, j, k)
                assert out["r"][k][nI + j] == pytest.approx(r["r_prob"], abs=TOL), (i, j, k)
            if n_s < 3 and k in (2, 9):
                # the returned scheduler, wherever the oracle's action gap exceeds 1e-9
                mu, _ = M.morap_last_policy(ctx.h, k, i * nJ + j)
                q = O.q_values(p, r["rew"], r["x"])
                for u in range(p.n - 1):
                    qa = q[p.state_ptr[u]:p.state_ptr[u + 1]]
                    m = r["mu"][u]
                    others = np.delete(qa, m)
                    if len(others) and qa[m] - others.max() > 1e-9:
                        assert mu[u] == m, (i, j, k, u)
                        checked += 1
    assert checked > 1000
    # properties that hold at any size: probabilities in [0, 1], costs <= 0,
    # c consistent with w.r on the assigned products
    assert np.all(out["r"][:, nI:] >= -1e-12) and np.all(out["r"][:, nI:] <= 1 + 1e-12)
    assert np.all(out["r"][:, :nI] <= 1e-12)
    for k, w in enumerate(W):
        tot = sum(out["c"][k, out["assign"][k][j], j] for j in range(nJ) if out["assign"][k][j] >= 0)
        assert w @ out["r"][k] == pytest.approx(tot, abs=1e-5)
    ctx.close()


def test_grid32_every_c_matches_oracle(M, grid32):
    """Every c of the benchmark's batch (200 products x 16 weights, one
    supporting-point batch as the benchmark launches it) against the
    oracle, one pair per host process."""
    inst = grid32
    nI, nJ = len(inst.agents), len(inst.tasks)
    ctx = make_ctx(M, inst)
    W = inst.weights
    out = ctx.supporting_points(W, want_c=True)
    jobs = [(inst.agents[i], inst.tasks[j], float(W[k][i]), float(W[k][nI + j]), 1e-8)
            for k in range(len(W)) for i in range(nI) for j in range(nJ)]
    want = np.array([c for c, _, _ in O.solve_pairs_pooled(jobs)]).reshape(len(W), nI, nJ)
    err = np.abs(out["c"] - want)
    assert err.max() < TOL, (err.max(), np.unravel_index(err.argmax(), err.shape))
    ctx.close()


def test_host_driven_loop_matches_graph_loop(M, tiny):
    """launch_mode 1 (host-driven bodies, for profilers) runs the same
    kernels in the same order as the CUDA-graph while loop."""
    a = make_ctx(M, tiny)
    b = make_ctx(M, tiny, launch_mode=1)
    ra = a.supporting_points(tiny.weights, want_c=True)
    rb = b.supporting_points(tiny.weights, want_c=True)
    assert np.array_equal(ra["c"], rb["c"]) and np.array_equal(ra["r"], rb["r"])
    assert a.stats()["fp32_sweeps"] == b.stats()["fp32_sweeps"]
    a.close()
    b.close()


@pytest.mark.parametrize("polish", [0, 1])
def test_every_kernel_shape_gives_identical_results(M, grid32, polish):
    """The tuner only picks among kernel shapes that do the same arithmetic
    in the same order, so each forced shape must reproduce the tuned run
    bit for bit (and the stats must name the shape used), for both forms of
    the second phase."""
    pair = (grid32.agents[:3], grid32.tasks[:5])
    W = np.ascontiguousarray(grid32.weights[:8][:, [0, 1, 2, 10, 11, 12, 13, 14]])
    ref_ctx = make_ctx(M, pair, polish=polish)
    ref = ref_ctx.solve(W, evaluate=True)
    st = ref_ctx.stats()
    assert 0 <= st["variant_fp32"] < 4 and 0 <= st["variant_fp64"] < 4 and st["polish"] == polish
    ref_ctx.close()
    for v in range(4):
        ctx = make_ctx(M, pair, sweep_variant_fp32=v, sweep_variant_fp64=(v + 1) % 4, polish=polish)
        out = ctx.solve(W, evaluate=True)
        assert ctx.stats()["variant_fp32"] == v and ctx.stats()["variant_fp64"] == (v + 1) % 4
        for key in ("c", "r_cost", "r_prob"):
            assert np.array_equal(out[key], ref[key]), (v, key)
        ctx.close()


@pytest.mark.parametrize("polish", [0, 1])
def test_warps_per_item_give_identical_results(M, grid32, polish):
    """Short work lists split each item's states over several warps; the
    per-(state, weight) arithmetic is the same, so one warp per item
    (item_warps_max = 1) and the default must agree bit for bit, values,
    evaluations and schedulers, with the same sweep counts."""
    pair = (grid32.agents[:3], grid32.tasks[:6])
    W = np.ascontiguousarray(grid32.weights[:8][:, [0, 1, 2, 10, 11, 12, 13, 14, 15]])
    one = make_ctx(M, pair, polish=polish, item_warps_max=1)
    many = make_ctx(M, pair, polish=polish)
    a = one.solve(W, evaluate=True)
    st_one = one.stats()
    b = many.solve(W, evaluate=True)
    st_many = many.stats()
    for key in ("c", "r_cost", "r_prob"):
        assert np.array_equal(a[key], b[key]), key
    for k in range(len(W)):
        for p in range(3 * 6):
            assert np.array_equal(M.morap_last_policy(one.h, k, p)[0], M.morap_last_policy(many.h, k, p)[0])
    assert st_one["fp32_sweeps"] == st_many["fp32_sweeps"] and st_one["fp64_sweeps"] == st_many["fp64_sweeps"]
    assert st_one["skipped_fp32"] == st_many["skipped_fp32"] and st_one["computed_fp64"] == st_many["computed_fp64"]
    one.close()
    many.close()


@pytest.mark.parametrize("launch_mode", [0, 1])
@pytest.mark.parametrize("polish", [0, 1])
def test_tail_launch_gives_identical_results(M, grid32, polish, launch_mode):
    """The end of each sweep loop in one cooperative launch (a grid barrier
    between sweeps, each warp group keeping its item) against one launch per
    sweep to the end: the same values, evaluations, schedulers and sweep
    counts, bit for bit.  With the automatic threshold the tail launch takes
    the loop's last sweeps; with a threshold above every list length (capped
    at one item per warp of the launch) it takes all but the first body of six."""
    pair = (grid32.agents[:3], grid32.tasks[:6])
    W = np.ascontiguousarray(grid32.weights[:8][:, [0, 1, 2, 10, 11, 12, 13, 14, 15]])
    ctxs = {t: make_ctx(M, pair, polish=polish, launch_mode=launch_mode, tail_items=t) for t in (0, -1, 1 << 30)}
    out, st = {}, {}
    for t, ctx in ctxs.items():
        out[t] = ctx.solve(W, evaluate=True)
        st[t] = ctx.stats()
    for t in (-1, 1 << 30):
        for key in ("c", "r_cost", "r_prob"):
            assert np.array_equal(out[0][key], out[t][key]), (t, key)
        for k in range(len(W)):
            for p in range(3 * 6):
                assert np.array_equal(M.morap_last_policy(ctxs[0].h, k, p)[0], M.morap_last_policy(ctxs[t].h, k, p)[0])
        for key in ("fp32_sweeps", "fp64_sweeps", "skipped_fp32", "skipped_fp64", "computed_fp32", "computed_fp64",
                    "updates_fp32", "updates_fp64", "bytes_fp32", "bytes_fp64", "pairs_not_converged"):
            assert st[0][key] == st[t][key], (t, key)
        assert st[t]["tail_sweeps_fp32"] > 0 and st[t]["tail_sweeps_fp64"] > 0, t
        assert st[t]["kernel_launches"] < st[0]["kernel_launches"], t
    assert st[0]["tail_sweeps_fp32"] == 0 and st[0]["tail_sweeps_fp64"] == 0
    whole = st[1 << 30]
    assert whole["fp32_sweeps"] - whole["tail_sweeps_fp32"] == 6 and whole["fp64_sweeps"] - whole["tail_sweeps_fp64"] == 6
    for ctx in ctxs.values():
        ctx.close()


def test_tail_barrier_wait_is_bounded(M, tiny):
    """The grid barrier between a tail launch's sweeps waits about a second
    at most: in a launch where one block never arrives, the other blocks give
    up, report it and end; the device stays usable afterwards."""
    timed_out, ms = M.morap_barrier_selfcheck(0)
    assert timed_out and 900.0 <= ms <= 20000.0, (timed_out, ms)
    ctx = make_ctx(M, tiny)
    out = ctx.solve(tiny.weights)
    assert np.all(np.isfinite(out["c"]))
    ctx.close()


def test_tail_launch_at_full_size(M, grid32):
    """The 32x32-grid batch (200 products, 16 weights) with and without the
    tail launch, after the shape tuning of a first solve: the same c, the
    same sweep counts."""
    W = grid32.weights
    on = make_ctx(M, grid32)
    off = make_ctx(M, grid32, tail_items=0)
    for ctx in (on, off):
        ctx.solve(W)  # the first solve at this batch size tunes the kernel shapes (no tail launch)
    a, b = on.solve(W), off.solve(W)
    sa, sb = on.stats(), off.stats()
    assert np.array_equal(a["c"], b["c"])
    assert sa["fp32_sweeps"] == sb["fp32_sweeps"] and sa["fp64_sweeps"] == sb["fp64_sweeps"]
    assert sa["tail_sweeps_fp64"] > 0 and sb["tail_sweeps_fp64"] == 0
    on.close()
    off.close()


@pytest.mark.parametrize("polish", [0, 1])
def test_skipping_unchanged_items_is_exact(M, grid32, polish):
    """A sweep skips work items none of whose inputs changed in the previous
    sweep; the results must be those of recomputing everything, bit for bit,
    and some items must actually have been skipped."""
    pair = (grid32.agents[:3], grid32.tasks[:6])
    W = np.ascontiguousarray(grid32.weights[:8][:, [0, 1, 2, 10, 11, 12, 13, 14, 15]])
    on = make_ctx(M, pair, polish=polish)
    off = make_ctx(M, pair, skip_unchanged=0, polish=polish)
    a = on.solve(W, evaluate=True)
    st_on = on.stats()
    b = off.solve(W, evaluate=True)
    st_off = off.stats()
    for key in ("c", "r_cost", "r_prob"):
        assert np.array_equal(a[key], b[key]), key
    for k in range(len(W)):
        for p in range(3 * 6):
            assert np.array_equal(M.morap_last_policy(on.h, k, p)[0], M.morap_last_policy(off.h, k, p)[0])
    assert st_on["fp32_sweeps"] == st_off["fp32_sweeps"] and st_on["fp64_sweeps"] == st_off["fp64_sweeps"]
    assert st_on["skipped_fp32"] > 0 and st_off["skipped_fp32"] == 0 and st_off["skipped_fp64"] == 0
    on.close()
    off.close()


def test_skipping_with_scattered_successors(M):
    """Random MDPs whose actions jump anywhere: most work items have more
    input items than are recorded (so they are always recomputed), the rest
    have few.  Skipping must still be exact, and the values must match the
    oracle."""
    agents = [I.random_tiny_agent(3, 40 + i, n_states=1500, n_actions=(1, 3), n_succ=(1, 3)) for i in range(2)]
    tasks = [I.random_tiny_task(3, 50 + j, n_locs=3) for j in range(2)]
    rng = np.random.default_rng(8)
    W = rng.dirichlet(np.ones(4), size=4)
    on = make_ctx(M, (agents, tasks))
    off = make_ctx(M, (agents, tasks), skip_unchanged=0)
    a = on.solve(W, evaluate=True)
    b = off.solve(W, evaluate=True)
    for key in ("c", "r_cost", "r_prob"):
        assert np.array_equal(a[key], b[key]), key
    for i, j, k in [(0, 0, 0), (1, 1, 2), (0, 1, 3)]:
        r = O.solve_pair(O.Product(agents[i], tasks[j]), W[k][i], W[k][2 + j])
        assert a["c"][k, i, j] == pytest.approx(r["c"], abs=TOL)
    on.close()
    off.close()


def test_polish_forms_agree_at_full_size(M, grid32):
    """The FP32 residual correction on a double-float table and the
    double-float sweeps converge to the same fixed point: on the benchmark's
    batch (200 products, K = 16) the c values and points agree far inside
    the 1e-6 tolerance, with the same assignments and the same sweep counts."""
    inst = grid32
    out, st = {}, {}
    for polish in (0, 1):
        ctx = make_ctx(M, inst, polish=polish)
        out[polish] = ctx.supporting_points(inst.weights, want_c=True)
        st[polish] = ctx.stats()
        ctx.close()
    assert st[0]["polish"] == 0 and st[1]["polish"] == 1
    assert np.max(np.abs(out[0]["c"] - out[1]["c"])) < 1e-9
    assert np.max(np.abs(out[0]["r"] - out[1]["r"])) < 1e-9
    assert np.array_equal(out[0]["assign"], out[1]["assign"])
    assert st[0]["fp32_sweeps"] == st[1]["fp32_sweeps"]
    assert abs(st[0]["fp64_sweeps"] - st[1]["fp64_sweeps"]) <= 6


def test_block_evaluation_matches_sweep_loop(M, grid32):
    """Algorithm 4 with one block per pair (every sweep in one launch, FP32
    with a residual correction on a double-float table) and with the
    multi-launch double-float sweep loop: both stop at the same residual
    rule, so the points agree far inside the 1e-6 tolerance; the block
    path needs far fewer launches."""
    pair = (grid32.agents[:4], grid32.tasks[:8])
    W = np.ascontiguousarray(grid32.weights[:8][:, [0, 1, 2, 3, 10, 11, 12, 13, 14, 15, 16, 17]])
    out, st = {}, {}
    for eb in (1, 0):
        ctx = make_ctx(M, pair, eval_block=eb)
        out[eb] = ctx.solve(W, evaluate=True)
        st[eb] = ctx.stats()
        ctx.close()
    assert np.array_equal(out[0]["c"], out[1]["c"])
    for key in ("r_cost", "r_prob"):
        assert np.max(np.abs(out[0][key] - out[1][key])) < 1e-8, key
    assert out[1]["code"] == M.OK and st[1]["eval_sweeps"] > 0
    assert st[1]["kernel_launches"] < st[0]["kernel_launches"]


@pytest.mark.parametrize("n_succ", [(1, 3), (5, 7), (9, 12)])
def test_block_evaluation_any_row_length(M, n_succ):
    """The block evaluation has variants for rows of at most 4 and 8 slots
    and a general one; each must agree with the sweep loop and match the
    oracle."""
    agents = [I.random_tiny_agent(5, 60 + i, n_states=400, n_actions=(1, 3), n_succ=n_succ) for i in range(2)]
    tasks = [I.random_tiny_task(5, 70 + j, n_locs=3) for j in range(2)]
    W = np.random.default_rng(9).dirichlet(np.ones(4), size=3)
    out = {}
    for eb in (1, 0):
        ctx = make_ctx(M, (agents, tasks), eval_block=eb)
        out[eb] = ctx.solve(W, evaluate=True)
        ctx.close()
    assert out[1]["code"] == M.OK
    for key in ("r_cost", "r_prob"):
        assert np.max(np.abs(out[0][key] - out[1][key])) < 1e-8, key
    for i, j, k in [(0, 0, 0), (1, 1, 2)]:
        r = O.solve_pair(O.Product(agents[i], tasks[j]), W[k][i], W[k][2 + j])
        assert out[1]["r_cost"][k, i, j] == pytest.approx(r["r_cost"], abs=TOL)
        assert out[1]["r_prob"][k, i, j] == pytest.approx(r["r_prob"], abs=TOL)


@pytest.mark.parametrize("polish", [0, 1])
def test_in_place_sweeps(M, grid32, polish):
    """Algorithm 3 with values updated in place (the paper's printed loop)
    reaches the same fixed point as the synchronous sweeps, within the
    stopping error, in no more sweeps.  The recorded actions follow another
    trajectory, so where near-ties exist the returned scheduler may be
    another optimal one: its points agree in the scalarised value w.r = c,
    and the values match the oracle."""
    pair = (grid32.agents[:3], grid32.tasks[:6])
    W = np.ascontiguousarray(grid32.weights[:8][:, [0, 1, 2, 10, 11, 12, 13, 14, 15]])
    out, st = {}, {}
    for ip in (0, 1):
        ctx = make_ctx(M, pair, in_place=ip, polish=polish)
        out[ip] = ctx.solve(W, evaluate=True)
        st[ip] = ctx.stats()
        ctx.close()
    assert out[1]["code"] == M.OK
    # both stop at the same residual rule, each within its stopping error of
    # the fixed point
    assert np.max(np.abs(out[1]["c"] - out[0]["c"])) < TOL
    wc = W[:, :3][:, :, None]
    wp = W[:, 3:][:, None, :]
    for ip in (0, 1):
        assert np.max(np.abs(wc * out[ip]["r_cost"] + wp * out[ip]["r_prob"] - out[ip]["c"])) < TOL
    assert st[1]["fp32_sweeps"] + st[1]["fp64_sweeps"] <= st[0]["fp32_sweeps"] + st[0]["fp64_sweeps"]
    for i, j, k in [(0, 1, 2), (2, 5, 6)]:
        # the oracle converged far tighter than the rule, as the reference point
        r = O.solve_pair(O.Product(pair[0][i], pair[1][j]), W[k][i], W[k][3 + j], eps1=1e-12)
        assert out[1]["c"][k, i, j] == pytest.approx(r["c"], abs=TOL)


def test_batch_invariance(M, grid32):
    """Each pair runs exactly its own sweeps: a weight alone and inside the
    K = 16 batch gives bitwise-identical c and points."""
    inst = grid32
    ctx = make_ctx(M, inst)
    W = inst.weights
    full = ctx.solve(W, evaluate=True)
    for k in (0, 5, 13):
        one = ctx.solve(W[k:k + 1], evaluate=True)
        assert np.array_equal(one["c"][0], full["c"][k])
        assert np.array_equal(one["r_cost"][0], full["r_cost"][k])
        assert np.array_equal(one["r_prob"][0], full["r_prob"][k])
    ctx.close()


# ------------------------------------------------------------- edge cases


def test_edge_cases(M, tiny, tiny_prods):
    nI, nJ = len(tiny.agents), len(tiny.tasks)
    ctx = make_ctx(M, tiny)
    # K not a power of two, and K > 64 (two batches)
    rng = np.random.default_rng(4)
    W = rng.dirichlet(np.ones(nI + nJ), size=70)
    W[3] = 0.0
    out = ctx.solve(W)
    c, rc, rp, _ = _oracle_pairs(tiny_prods, W[[0, 3, 65, 69]], nI, nJ)
    got = out["c"][[0, 3, 65, 69]]
    assert np.max(np.abs(got - c)) < TOL
    assert np.all(out["c"][3] == 0.0)
    ctx.close()
    # task accepting at q0, and a task that can never be accomplished
    acc0 = I.Task(1, 0, 1, np.array([I.GRID_AP(0, 0)], np.int32), np.zeros(2, np.int32), np.array([1], np.uint8))
    never = I.sequence_task([I.GRID_AP(9, 9)])  # not on the 4x4 grid
    ctx = make_ctx(M, (tiny.agents, [acc0, never]))
    out = ctx.solve(np.array([[0.2, 0.2, 0.3, 0.3]]))
    assert np.all(out["c"] == 0.0) and np.all(out["r_prob"] == 0.0) and np.all(out["r_cost"] == 0.0)
    ctx.close()


def test_sweep_cap_reports_not_converged(M, grid32):
    ctx = make_ctx(M, grid32, max_sweeps=6)
    out = ctx.solve(grid32.weights[:4], check=False)
    assert out["code"] == M.ENOTCONV
    assert np.any(out["status"] == M.ENOTCONV)
    ctx.close()


def test_invalid_inputs(M, tiny):
    ctx = M.Context()
    a = tiny.agents[0]
    bad = a.prob.copy()
    bad[0] += 0.01
    with pytest.raises(M.MorapError) as e:
        M.morap_add_agent(ctx.h, a.n_states, a.s0, a.state_ptr, a.sa_ptr, a.succ, bad, a.cost, a.label_ptr,
                          a.label_ap)
    assert e.value.code == M.EINVAL
    with pytest.raises(M.MorapError) as e:
        ctx.solve(np.ones((1, 2)))
    assert e.value.code == M.ESTATE
    ctx.add(tiny.agents, tiny.tasks)
    ctx.build()
    W = tiny.weights.copy()
    W[0, 0] = -0.5
    with pytest.raises(M.MorapError) as e:
        ctx.solve(W)
    assert e.value.code == M.EINVAL
    ctx.close()
    for field, val in (("sweep_variant_fp32", 4), ("sweep_variant_fp64", -2), ("launch_mode", 2), ("polish", 2),
                       ("eval_block", 3), ("in_place", 2)):
        cfg = M.morap_config_default()
        setattr(cfg, field, val)
        with pytest.raises(M.MorapError) as e:
            M.Context(cfg)
        assert e.value.code == M.EINVAL, field


def test_hbm_budget_refuses_before_allocating(M, grid32):
    cfg = M.morap_config_default()
    cfg.hbm_budget = 1 << 20
    ctx = M.Context(cfg)
    ctx.add(grid32.agents, grid32.tasks)
    with pytest.raises(M.MorapError) as e:
        ctx.build()
    assert e.value.code == M.ENOMEM
    ctx.close()


# ------------------------------------------------------------- plain baseline


def test_plain_baseline_matches_oracle(M, tiny, tiny_prods):
    nI, nJ = len(tiny.agents), len(tiny.tasks)
    ctx = make_ctx(M, tiny)
    pairs = [(0, 0, 0.1, 0.9), (1, 2, 0.3, 0.7), (0, 1, 1.0, 0.0), (1, 0, 0.02, 0.98)]
    out = M.morap_solve_plain(ctx.h, [i * nJ + j for i, j, _, _ in pairs], [(a, b) for _, _, a, b in pairs])
    for e, (i, j, wc, wp) in enumerate(pairs):
        r = O.solve_pair(tiny_prods[i][j], wc, wp)
        assert out["c"][e] == pytest.approx(r["c"], abs=TOL)
        assert out["r_cost"][e] == pytest.approx(r["r_cost"], abs=TOL)
        assert out["r_prob"][e] == pytest.approx(r["r_prob"], abs=TOL)
        assert out["sweeps_vi"] > 0
    ctx.close()


def test_torch_allocator_and_stream(M, tiny):
    import torch

    cfg = M.morap_config_default()
    ctx = M.Context(cfg, use_torch_allocator=True)
    ctx.add(tiny.agents, tiny.tasks)
    s = torch.cuda.Stream()
    ctx.build(s.cuda_stream)
    a = ctx.solve(tiny.weights, stream=s.cuda_stream)
    ctx.close()
    ctx2 = make_ctx(M, tiny)
    b = ctx2.solve(tiny.weights)
    ctx2.close()
    assert np.array_equal(a["c"], b["c"])
