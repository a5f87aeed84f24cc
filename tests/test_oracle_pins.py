"""Pins for the FP64 oracle (CPU only).

Each test fixes a value the oracle must reproduce from something other than
itself: values printed in the paper's worked example (Fig. 2), closed forms,
exact linear solves, brute force over all simple schedulers, and the
invariants of Sec. 3 (VI from below, Lemma 7).  A dropped reward term, a
wrong sign, labels read on the source instead of the successor, or a wrong
tie rule each fail at least one of them.
"""

import json
import math
import os

import numpy as np
import pytest

import instances as I
from oracle import core as C
from oracle import dfa as D

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig2.json")))


@pytest.fixture(scope="module", autouse=True)
def _lib(oracle_lib):
    return oracle_lib


# ---------------------------------------------------------------- Fig. 2


def test_fig2_r1_printed_value():
    """Sec. 3.3 example: w = (1, 0) returns r1 = (-1.1, 0.1)."""
    p = C.Product(I.fig2_agent(), I.fig2_task())
    r = C.solve_pair(p, 1.0, 0.0, exact_eval=True)
    want = GOLD["printed"]["r1_for_w_1_0"]["value"]
    assert r["r_cost"] == pytest.approx(want[0], abs=1e-12)
    assert r["r_prob"] == pytest.approx(want[1], abs=1e-12)
    assert r["c"] == pytest.approx(want[0], abs=1e-9)


def test_fig2_scheduler_points():
    """The two simple schedulers at s0 give (-1.1, 0.1) and (-2/0.7, 0.5/0.7);
    the probability 0.714 is the one printed in Fig. 2b."""
    p = C.Product(I.fig2_agent(), I.fig2_task())
    _, out = C.brute_force(p, 0.5, 0.5)
    pts = sorted({(round(a, 12), round(b, 12)) for _, _, (a, b) in out})
    g = GOLD["pinned_under_presink_reading"]
    assert pts[0] == pytest.approx((g["scheduler_a_cost"]["value"], g["scheduler_a_prob"]["value"]), abs=1e-12)
    assert pts[1] == pytest.approx(tuple(g["scheduler_b_point"]["value"]), abs=1e-12)
    assert g["scheduler_a_prob"]["value"] == pytest.approx(0.714, abs=5e-4)


def test_fig2_probability_objective_picks_a():
    p = C.Product(I.fig2_agent(), I.fig2_task())
    r = C.solve_pair(p, 0.0, 1.0, exact_eval=True)
    assert r["r_prob"] == pytest.approx(0.5 / 0.7, abs=1e-12)
    assert r["mu"][p.init] == 0  # action a


# ---------------------------------------------------------------- closed forms


@pytest.mark.parametrize("L,slip,target", [(8, 0.2, 5), (12, 0.05, 11), (5, 0.0, 3)])
def test_corridor_expected_cost(L, slip, target):
    """1 x L corridor, target at distance d: E[cost] = d / (1 - slip), Pr = 1
    (perpendicular slips are blocked and cost a step; the pre-sink step is the
    free stay)."""
    a = I.corridor_agent(L, slip, 0)
    t = I.sequence_task([I.GRID_AP(target, 0)])
    p = C.Product(a, t)
    r = C.solve_pair(p, 0.001, 0.999, eps1=1e-13, exact_eval=True)
    assert r["r_cost"] == pytest.approx(-target / (1 - slip), abs=1e-9)
    assert r["r_prob"] == pytest.approx(1.0, abs=1e-12)


def test_corridor_two_targets():
    """'visit a then b': (d(s0,a) + d(a,b)) / (1 - slip)."""
    a = I.corridor_agent(10, 0.1, 2)
    t = I.sequence_task([I.GRID_AP(7, 0), I.GRID_AP(4, 0)])
    p = C.Product(a, t)
    r = C.solve_pair(p, 0.001, 0.999, eps1=1e-13, exact_eval=True)
    assert r["r_cost"] == pytest.approx(-(5 + 3) / 0.9, abs=1e-9)
    assert r["r_prob"] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("N,pf,pt", [(3, 0.6, 0.1), (5, 0.3, 0.05), (1, 0.5, 0.5)])
def test_chain_with_failure(N, pf, pt):
    """Chain: forward pf, trap pt, stay otherwise.  Pr = (pf/(pf+pt))^N and
    E[cost] = sum_{k<N} (pf/(pf+pt))^k / (pf+pt) (each stage costs a
    geometric number of steps and is reached with the product probability)."""
    a = I.chain_agent(N, pf, pt)
    t = I.sequence_task([1], avoid_ap=2)
    p = C.Product(a, t)
    r = C.solve_pair(p, 1e-6, 1.0, eps1=1e-14, exact_eval=True)
    ratio = pf / (pf + pt)
    assert r["r_prob"] == pytest.approx(ratio ** N, abs=1e-12)
    assert r["r_cost"] == pytest.approx(-sum(ratio ** k for k in range(N)) / (pf + pt), abs=1e-9)


def test_deterministic_grid_is_bfs_distance():
    """slip 0: the optimal cost to a single target is the BFS distance."""
    W = H = 6
    rng = np.random.default_rng(5)
    blocked = rng.random((H, W)) < 0.2
    blocked[0, 0] = False
    blocked[H - 1, W - 1] = False
    # BFS from the target
    from collections import deque

    tx, ty = W - 1, H - 1
    dist = -np.ones((H, W), int)
    dist[ty, tx] = 0
    dq = deque([(tx, ty)])
    while dq:
        x, y = dq.popleft()
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            nx, ny = x + dx, y + dy
            if 0 <= nx < W and 0 <= ny < H and not blocked[ny, nx] and dist[ny, nx] < 0:
                dist[ny, nx] = dist[y, x] + 1
                dq.append((nx, ny))
    a = I.grid_agent(W, H, 0.0, (0, 0), blocked)
    t = I.sequence_task([I.GRID_AP(tx, ty)])
    p = C.Product(a, t)
    r = C.solve_pair(p, 1e-3, 1.0, eps1=1e-13, exact_eval=True)
    if dist[0, 0] < 0:
        assert r["r_prob"] == 0.0
    else:
        assert r["r_cost"] == pytest.approx(-dist[0, 0], abs=1e-9)
        assert r["r_prob"] == pytest.approx(1.0, abs=1e-12)


def test_scalarised_value_is_weighted_objectives():
    """c_ij = w_i r_cost + w_p r_prob at the optimum (exact for the returned
    scheduler up to the VI stop error)."""
    inst = I.config_tiny()
    for a in inst.agents:
        for t in inst.tasks:
            p = C.Product(a, t)
            for wc, wp in [(0.2, 0.8), (0.05, 0.95), (0.5, 0.5)]:
                r = C.solve_pair(p, wc, wp, eps1=1e-13, exact_eval=True)
                assert r["c"] == pytest.approx(wc * r["r_cost"] + wp * r["r_prob"], abs=1e-9)


# ---------------------------------------------------------------- brute force


def _tiny_products(n=24):
    shapes = [(3, (1, 2), 2), (4, (1, 1), 2), (3, (1, 1), 3), (2, (1, 2), 3)]
    out = []
    for k in range(n):
        ns, na, nl = shapes[k % len(shapes)]
        a = I.random_tiny_agent(100 + k, 0, n_states=ns, n_actions=na, n_succ=(1, 3))
        t = I.random_tiny_task(100 + k, 1, n_locs=nl)
        p = C.Product(a, t)
        counts = np.maximum(np.diff(p.state_ptr), 1)
        if np.prod(counts.astype(float)) <= 4000:
            out.append(p)
    return out


@pytest.mark.parametrize("wc,wp", [(0.3, 0.7), (0.7, 0.3), (0.0, 1.0), (1.0, 0.0)])
def test_alg3_matches_brute_force_optimum(wc, wp):
    """Algorithm 3's value equals the best simple scheduler (exact LU per
    scheduler), and its returned scheduler attains it."""
    prods = _tiny_products()
    assert len(prods) >= 10
    for p in prods:
        best, out = C.brute_force(p, wc, wp)
        r = C.solve_pair(p, wc, wp, eps1=1e-13, exact_eval=True)
        assert r["c"] == pytest.approx(best, abs=1e-8)
        got = (wc * r["r_cost"] if wc else 0.0) + wp * r["r_prob"]
        assert got == pytest.approx(best, abs=1e-8)


def test_lemma7_no_achievable_point_above_hyperplane():
    """Lemma 7 on single products: w.r >= w.u for every simple scheduler's
    point u (r = the point Algorithm 2 returns for w)."""
    rng = np.random.default_rng(3)
    for p in _tiny_products(12):
        w = rng.dirichlet([1.0, 1.0])
        r = C.solve_pair(p, w[0], w[1], eps1=1e-13, exact_eval=True)
        _, out = C.brute_force(p, w[0], w[1])
        wr = w[0] * r["r_cost"] + w[1] * r["r_prob"]
        for _, _, (uc, up) in out:
            if np.isfinite(uc):
                assert wr >= w[0] * uc + w[1] * up - 1e-9


def test_alg4_matches_exact_solve():
    """Algorithm 4 to 1e-13 equals the dense solve of (I - P_mu) v = r_mu."""
    inst = I.config_tiny()
    for a in inst.agents:
        for t in inst.tasks:
            p = C.Product(a, t)
            r = C.solve_pair(p, 0.1, 0.9)
            for rew in (p.reward_cost(), p.reward_prob()):
                v_vi, _, ok = C.alg4(p, rew, r["mu"], 1e-14)
                v_ex = C.exact_policy_values(p, rew, r["mu"])
                assert ok
                assert np.max(np.abs(v_vi - v_ex)) < 1e-10


def test_vi_from_below_monotone_and_bounded():
    """From x = 0 with a free stay action the iterates never decrease and
    never exceed the optimum (the lower-bound property the engine's FP32
    phase relies on)."""
    inst = I.config_tiny()
    p = C.Product(inst.agents[0], inst.tasks[0])
    rew = p.reward_scalarised(0.05, 0.95)
    x_star, _, _, _ = C.alg3(p, rew, 1e-14)
    x = np.zeros(p.n)
    for _ in range(60):
        y, _, _, _ = C.alg3(p, rew, 0.0, max_sweeps=1, x0=x)
        assert np.all(y >= x - 1e-15)
        assert np.all(y <= x_star + 1e-12)
        x = y


def test_record_rule_avoids_stay_ties():
    """With a free stay action Q(stay) = V at the fixed point, so a greedy
    argmax with lowest-index ties would stay forever; the recorded action of
    Algorithm 3 keeps the progress move (probability objective)."""
    a = I.corridor_agent(6, 0.1, 0)
    t = I.sequence_task([I.GRID_AP(4, 0)])
    p = C.Product(a, t)
    r = C.solve_pair(p, 0.0, 1.0, eps1=1e-12, exact_eval=True)
    assert r["r_prob"] == pytest.approx(1.0, abs=1e-12)
    assert r["mu"][p.init] != 0
    greedy = C.q_values(p, r["rew"], r["x"])
    # the greedy lowest-index argmax at the initial state is 'stay' (action 0)
    a0, a1 = p.state_ptr[p.init], p.state_ptr[p.init + 1]
    assert int(np.argmax(greedy[a0:a1] >= greedy[a0:a1].max() - 1e-9)) == 0


def test_finalise_fallback_prefers_moving_over_self_loop():
    """When the recorded action is stale (more than tau below the maximum) the
    scheduler falls back to a near-maximiser that is not a self-loop: at a
    fixed point the free stay ties with the maximum, and choosing it would
    return "stay forever" where the value came from moving."""
    a = I.corridor_agent(6, 0.0, 0)
    t = I.sequence_task([I.GRID_AP(4, 0)])
    p = C.Product(a, t)
    rew = p.reward_scalarised(0.01, 0.99)
    x, a_rec, _, _ = C.alg3(p, rew, 1e-14)
    stale = np.full_like(a_rec, 4)  # W: away from the target
    mu = C.finalise(p, rew, x, stale)
    for s in range(4):  # states left of the target: the move towards it (E = 3)
        assert mu[s] == 3, (s, mu[s])
    v = C.exact_policy_values(p, p.reward_prob(), mu)
    assert v[p.init] == pytest.approx(1.0, abs=1e-12)


def test_tie_fallback_never_returns_a_two_state_cycle():
    """Zero weight on the cost (every move is free) and a stale recorded
    action: on the final values A -> B, B -> A and A -> Y all tie, and the
    lowest-index near-maximiser of A and of B would send the run between A
    and B forever (probability 0 instead of 1).  The returned scheduler
    must reach the goal with the optimal probability: the exact value of the
    scheduler (dense solve) equals c, which is 1."""
    a = I.tie_drift_agent()
    p = C.Product(a, I.sequence_task([0]))
    r = C.solve_pair(p, 0.0, 1.0, exact_eval=True)
    q = C.q_values(p, r["rew"], r["x"])
    A, B = p.init, p.init + 1
    qa = q[p.state_ptr[A]:p.state_ptr[A + 1]]
    assert qa[r["a_rec"][A]] < qa.max() - 1e-9  # the fallback branch is taken at A
    assert r["c"] == pytest.approx(1.0, abs=1e-9)
    assert r["r_prob"] == pytest.approx(r["c"], abs=1e-9)
    assert r["mu"][A] == 3 and r["mu"][B] == 1  # A -> Y, B -> A (and on to Y)
    # the planted mistake: lowest-index non-self-loop near-maximiser without
    # the anchoring rounds returns the A <-> B cycle, which this pin rejects
    mu_bad = r["mu"].copy()
    mu_bad[A], mu_bad[B] = 1, 1
    v_bad = C.exact_policy_values(p, p.reward_prob(), mu_bad)
    assert v_bad[A] == pytest.approx(0.0, abs=1e-12)


# ---------------------------------------------------------------- DFA and product


def test_dfa_presink_insertion_and_traps():
    t = I.fig2_task()
    d = D.preprocess(t)
    assert d["inserted_presink"]
    assert d["n_locs"] == 4
    assert list(d["trap"]) == [False, False, True, False]
    assert list(d["pre"]) == [False, False, False, True]
    assert list(d["nd_loc"]) == [0, 3]
    # a DFA whose only entry to F is already a pre-sink gets no new location
    delta = np.array([[1, 1], [2, 2], [2, 2]], np.int32).reshape(-1)
    t2 = I.Task(3, 0, 1, np.array([0], np.int32), delta, np.array([0, 0, 1], np.uint8))
    d2 = D.preprocess(t2)
    assert not d2["inserted_presink"] and list(d2["pre"]) == [False, True, False]


def test_dfa_rejects_non_sink_accepting():
    delta = np.array([[1, 1], [0, 1]], np.int32).reshape(-1)
    t = I.Task(2, 0, 1, np.array([0], np.int32), delta, np.array([0, 1], np.uint8))
    with pytest.raises(ValueError):
        D.preprocess(t)


def test_product_reads_labels_on_successor_and_sums_to_one():
    p = C.Product(I.fig2_agent(), I.fig2_task())
    # (s0,q0) -b-> s1 (label x -> trap) 0.9 and s3 (label y -> pre-sink P) 0.1
    a = p.state_ptr[p.init] + 1
    row = {p.key(int(c)): float(pr) for c, pr in zip(p.col[p.sa_ptr[a]:p.sa_ptr[a + 1]],
                                                       p.prob[p.sa_ptr[a]:p.sa_ptr[a + 1]])}
    assert row == {("DONE",): pytest.approx(0.9), (3, 3): pytest.approx(0.1)}
    sums = np.add.reduceat(p.prob, p.sa_ptr[:-1]) if len(p.sa_ptr) > 1 else []
    assert np.allclose(sums, 1.0)
    # size: |M| = |S| + |P| over non-done states (Sec. 2)
    assert p.n - 1 == 2 * 4


def test_initial_state_does_not_consume_start_label():
    """The product starts at (s0, q0): the label of s0 is not read then.  The
    first action's successor is read, so a free stay on the target cell
    advances the DFA (cost 0, probability 1), while the initial product state
    is still the (s0, q0) one."""
    a = I.corridor_agent(4, 0.0, 0)
    t = I.sequence_task([I.GRID_AP(0, 0)])  # target on the start cell
    p = C.Product(a, t)
    assert p.key(p.init) == (0, 0)
    r = C.solve_pair(p, 0.01, 0.99, eps1=1e-13, exact_eval=True)
    assert r["r_cost"] == pytest.approx(0.0, abs=1e-12)
    assert r["r_prob"] == pytest.approx(1.0, abs=1e-12)
    assert r["mu"][p.init] == 0
