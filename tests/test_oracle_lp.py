"""Pins of the LP oracle (oracle/lp.py): the hand-written simplex against
brute force over basic solutions and small systems with known answers, and
the MORAP LP (Sec. 3, Fig. 1; Lemma 2 for the random assignment) against
enumeration of deterministic schedulers and assignments and against
Algorithm 1 of the oracle.  CPU only."""

import itertools

import numpy as np
import pytest

import instances as I
from oracle import core as C
from oracle import lp as L
from oracle import pareto as P


def _brute_force_feasible(A, b):
    """{x >= 0 : A x = b} is non-empty iff a basic solution is (A of full row
    rank): try every choice of m columns."""
    m, n = A.shape
    for cols in itertools.combinations(range(n), m):
        B = A[:, cols]
        if abs(np.linalg.det(B)) < 1e-12:
            continue
        xb = np.linalg.solve(B, b)
        if np.all(xb >= -1e-10):
            return True
    return False


def test_simplex_small_known_systems():
    assert L.simplex_phase1([[1, 1]], [1])[0]
    assert not L.simplex_phase1([[1, 1], [1, -1]], [1, 2])[0]  # x = (1.5, -0.5)
    assert not L.simplex_phase1([[1, 1], [1, 0]], [1, 2])[0]
    # a degenerate system (several bases share the vertex x = (1, 0, 0, 0))
    A = np.array([[1.0, 1, 1, 1], [1, -1, 0, 2], [1, 0, -1, 3]])
    ok, x, infeas = L.simplex_phase1(A, [1, 1, 1])
    assert ok and np.allclose(A @ x, [1, 1, 1]) and np.all(x >= 0)
    # negative right-hand sides are handled by flipping rows
    ok, x, _ = L.simplex_phase1([[-1.0, -2.0]], [-4.0])
    assert ok and abs(x[0] + 2 * x[1] - 4) < 1e-12


@pytest.mark.parametrize("seed", range(12))
def test_simplex_matches_basic_solution_brute_force(seed):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(2, 4)), int(rng.integers(4, 7))
    A = rng.integers(-3, 4, size=(m, n)).astype(float)
    b = rng.integers(-3, 4, size=m).astype(float)
    if np.linalg.matrix_rank(A) < m:
        A[:, :m] += np.eye(m)
    ok, x, infeas = L.simplex_phase1(A, b)
    assert ok == _brute_force_feasible(A, b)
    if ok:
        assert np.all(x >= 0) and np.allclose(A @ x, b, atol=1e-9)
    else:
        assert infeas > 1e-9


def _tiny_instance(seed):
    agents = [I.random_tiny_agent(seed, k, n_states=3, n_actions=(1, 1), n_succ=(1, 2)) for k in range(2)]
    tasks = [I.random_tiny_task(seed, 10 + k, n_locs=2, n_ap=2) for k in range(2)]
    return C.products(agents, tasks)


def _achievable_points(prods):
    nI, nJ = len(prods), len(prods[0])
    pair_pts = {}
    for i in range(nI):
        for j in range(nJ):
            _, out = C.brute_force(prods[i][j], 0.5, 0.5)
            pair_pts[i, j] = sorted({(a, b) for _, _, (a, b) in out if np.isfinite(a)})
    n = max(nI, nJ)
    pts = []
    for perm in itertools.permutations(range(n)):
        pairs = [(perm[j], j) for j in range(nJ) if perm[j] < nI]
        for choice in itertools.product(*[pair_pts[p] for p in pairs]):
            r = np.zeros(nI + nJ)
            for (i, j), (c, pr) in zip(pairs, choice):
                r[i] = c
                r[nI + j] = pr
            pts.append(r)
    return np.unique(np.array(pts), axis=0)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_morap_lp_matches_enumeration(seed):
    """On instances small enough to enumerate every deterministic assignment
    and scheduler, t is achievable iff it lies in down(conv(points))."""
    prods = _tiny_instance(seed)
    pts = _achievable_points(prods)
    rng = np.random.default_rng(200 + seed)
    checked = 0
    for _ in range(12):
        t = pts.max(axis=0) + rng.uniform(-0.6, 0.3, size=4)
        dist = np.linalg.norm(t - P.project_down_hull(t, pts, np.eye(4)))
        if 1e-9 < dist < 1e-4:
            continue  # too close to the boundary to call
        ok, det = L.morap_feasible(prods, t)
        assert ok == (dist <= 1e-9), (t, dist, det["infeasibility"])
        if ok:
            assert np.all(det["achieved"] >= t - 1e-8)
            mu = det["mu"]
            assert np.all(mu.sum(axis=0) <= 1 + 1e-9) and np.all(mu.sum(axis=1) <= 1 + 1e-9)
        checked += 1
    assert checked >= 8


def test_morap_lp_fig2():
    prods = [[C.Product(I.fig2_agent(), I.fig2_task())]]
    supp = lambda w: C.supporting_point(prods, w, eps1=1e-12)[0]
    for t in ([-1.8, 0.9], [-3.0, 0.5], [-2.5, 0.7]):
        ref = P.alg1(supp, np.array(t), eps=1e-7)
        assert L.morap_feasible(prods, t)[0] == ref["feasible"], t


def test_morap_lp_matches_alg1_on_the_tiny_config():
    """2 agents x 3 tasks on a 4x4 grid (products of 49 states): too many
    schedulers to enumerate, so the LP is the independent check of the
    oracle's Algorithm 1 verdicts."""
    inst = I.config_tiny()
    prods = C.products(inst.agents, inst.tasks)
    supp = lambda w: C.supporting_point(prods, w)[0]
    rng = np.random.default_rng(5)
    ts = [inst.thresholds[0], np.array([-12.0, -12.0, 0.6, 0.6, 0.6]), np.array([-1.0, -1.0, 0.2, 0.2, 0.2])]
    ts += [np.concatenate([-rng.uniform(2, 14, 2), rng.uniform(0.1, 0.95, 3)]) for _ in range(3)]
    seen = set()
    for t in ts:
        ref = P.alg1(supp, t, eps=1e-7, max_iter=60)
        margin = np.linalg.norm(ref["t_dn"] - t)
        if not ref["feasible"] and margin < 1e-4:
            continue
        ok, det = L.morap_feasible(prods, t)
        assert ok == ref["feasible"], (t, margin, det["infeasibility"])
        seen.add(ok)
    assert seen == {True, False}
