"""Pins for the oracle's assignment step, projections and Algorithm 1 (CPU).

Assignment: brute force over all permutations.  Projections: closed forms
(one half-space, one dominating point, one LDP constraint), KKT certificates
that characterise each projection completely (to 1e-10, general metric M),
brute force over every active set in 2-4 dimensions, the non-negative least
squares step against brute force over supports, and a 1-D scan over
segments in 2-D.  Algorithm 1: Thm 3 / Cor. on
instances whose achievable set C is enumerable (all permutations x all
simple schedulers), and Lemma 6 on every direction it produces.
"""

import itertools

import numpy as np
import pytest
from scipy.optimize import nnls

import instances as I
from oracle import core as C
from oracle import pareto as P


@pytest.fixture(scope="module", autouse=True)
def _lib(oracle_lib):
    return oracle_lib


# ---------------------------------------------------------------- assignment


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_assignment_matches_permutation_brute_force(n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        Cm = rng.normal(size=(n, n))
        if n > 2:
            Cm[0, :] = Cm[1, :]  # some ties
        f = C.assignment(Cm)
        got = sum(Cm[f[j], j] for j in range(n))
        best = max(sum(Cm[p[j], j] for j in range(n)) for p in itertools.permutations(range(n)))
        assert got == pytest.approx(best, abs=1e-12)
        assert sorted(f.tolist()) == list(range(n))


def test_pad_square_dummy_agents():
    Cm = np.array([[1.0, 2.0, 3.0], [4.0, 0.5, 0.1]])
    S = C.pad_square(Cm)
    assert S.shape == (3, 3) and np.all(S[2] == 0)
    f = C.assignment(S)
    # best: agent 0 -> task 2 (3), agent 1 -> task 0 (4), dummy -> task 1
    assert f[2] == 0 and f[0] == 1 and f[1] == 2


# ---------------------------------------------------------------- projections
#
# Both projections are pinned to 1e-10 by conditions that characterise the
# answer completely (KKT certificates and brute force over every active
# set), and to closed forms where one exists.


def _rand_spd(rng, n):
    A = rng.normal(size=(n, n))
    return A @ A.T + n * np.eye(n)


def _nnls_brute(E, f):
    """min ||E u - f|| over u >= 0 by trying every support: the answer is the
    unconstrained least-squares solution on some support whose coordinates
    are positive and whose gradient is <= 0 off the support."""
    m = E.shape[1]
    best = None
    for k in range(m + 1):
        for S in itertools.combinations(range(m), k):
            u = np.zeros(m)
            if S:
                u[list(S)] = np.linalg.lstsq(E[:, list(S)], f, rcond=None)[0]
                if np.any(u[list(S)] <= 0):
                    continue
            g = E.T @ (f - E @ u)
            off = [j for j in range(m) if j not in S]
            if off and np.max(g[off]) > 1e-10:
                continue
            val = np.linalg.norm(E @ u - f)
            if best is None or val < best[0] - 1e-12:
                best = (val, u)
    return best


def test_nnls_kkt_and_brute_force():
    rng = np.random.default_rng(5)
    for _ in range(30):
        n, m = rng.integers(2, 6), rng.integers(1, 7)
        E = rng.normal(size=(n, m))
        f = rng.normal(size=n)
        u = P.nnls(E, f)
        g = E.T @ (f - E @ u)
        assert np.all(u >= 0)
        assert np.all(g <= 1e-12)
        assert np.all(np.abs(g[u > 0]) <= 1e-12)
        val, ub = _nnls_brute(E, f)
        assert np.linalg.norm(E @ u - f) == pytest.approx(val, abs=1e-12)
        assert np.max(np.abs(E @ u - E @ ub)) < 1e-10  # the fitted vector is unique


def test_ldp_closed_form():
    """One constraint g.x >= h with h > 0: x = h g / |g|^2; h <= 0: x = 0;
    inconsistent constraints are reported."""
    rng = np.random.default_rng(6)
    for _ in range(10):
        g = rng.normal(size=4)
        h = rng.uniform(0.1, 2.0)
        x = P.ldp(g[None, :], np.array([h]))
        assert np.max(np.abs(x - h * g / (g @ g))) < 1e-13
        assert np.max(np.abs(P.ldp(g[None, :], np.array([-h])))) < 1e-15
    g = np.array([[1.0, 0.0], [-1.0, 0.0]])
    assert P.ldp(g, np.array([1.0, 1.0])) is None  # x0 >= 1 and -x0 >= 1


def test_halfspace_projection_closed_form():
    rng = np.random.default_rng(0)
    for _ in range(10):
        n = 4
        M = _rand_spd(rng, n)
        w = rng.dirichlet(np.ones(n))
        t = rng.normal(size=n)
        b = w @ t - 0.7
        z = P.project_halfspaces(t, w[None, :], np.array([b]), M)
        Minv_w = np.linalg.solve(M, w)
        want = t - (w @ t - b) / (w @ Minv_w) * Minv_w
        assert np.max(np.abs(z - want)) < 1e-12


def _halfspace_instance(rng, n, m):
    Wt = rng.dirichlet(np.ones(n), size=m)
    R = rng.normal(size=(m, n))
    b = np.einsum("ij,ij->i", Wt, R)
    t = R.max(axis=0) + rng.uniform(0.1, 1.0, size=n)
    return Wt, b, t


def test_halfspace_projection_kkt():
    """z is feasible and M(t - z) = A_act^T mu with mu >= 0 on the active
    rows (the KKT conditions of a strictly convex QP: they fix z)."""
    rng = np.random.default_rng(1)
    for n, m in [(3, 2), (5, 6), (8, 12), (20, 30)]:
        for _ in range(4):
            Wt, b, t = _halfspace_instance(rng, n, m)
            M = _rand_spd(rng, n) if n <= 8 else np.eye(n)
            z = P.project_halfspaces(t, Wt, b, M)
            assert np.all(Wt @ z <= b + 1e-10)
            act = np.abs(Wt @ z - b) < 1e-9
            mu, res = nnls(Wt[act].T, M @ (t - z))
            assert res < 1e-10


def test_halfspace_projection_brute_force_active_sets():
    """Every subset S of at most n rows: z_S = argmin ||t - z||_M on
    A_S z = b_S (a KKT solve); the projection is the z_S that is feasible with
    non-negative multipliers, unique for a strictly convex objective."""
    rng = np.random.default_rng(3)
    for n, m in [(2, 3), (3, 4), (4, 6), (3, 7)]:
        for _ in range(5):
            Wt, b, t = _halfspace_instance(rng, n, m)
            M = _rand_spd(rng, n)
            Minv = np.linalg.inv(M)
            found = []
            for k in range(0, n + 1):
                for S in itertools.combinations(range(m), k):
                    S = list(S)
                    if S:
                        AS = Wt[S]
                        K = AS @ Minv @ AS.T
                        if np.linalg.matrix_rank(K) < len(S):
                            continue
                        mu = np.linalg.solve(K, AS @ t - b[S])
                        if np.any(mu < -1e-12):
                            continue
                        z = t - Minv @ AS.T @ mu
                    else:
                        z = t.copy()
                    if np.all(Wt @ z <= b + 1e-11):
                        found.append(z)
            assert found
            z = P.project_halfspaces(t, Wt, b, M)
            for zb in found:
                assert np.max(np.abs(z - zb)) < 1e-10


def _down_hull_certificate(t, Phi, M, x, lam):
    """x solves min ||t - x||_M over down(conv Phi) iff x <= Phi^T lam for some
    lam on the simplex, g = M (t - x) >= 0, and max_k g.phi_k <= g.x (the
    variational inequality over the generators: the points and the rays -e_i)."""
    g = M @ (t - x)
    sg = max(1.0, np.abs(g).max())  # tolerances relative to the scale of g and Phi
    sp = max(1.0, np.abs(Phi).max())
    assert np.all(lam >= -1e-15) and abs(lam.sum() - 1) < 1e-12
    assert np.all(x <= Phi.T @ lam + 1e-12 * sp)
    assert np.all(g >= -1e-12 * sg)
    assert np.max(Phi @ g) <= g @ x + 1e-10 * sg * sp


def test_down_hull_single_point_is_componentwise_min():
    t = np.array([-1.0, 0.9, 0.3])
    r = np.array([-2.0, 0.5, 0.8])
    x = P.project_down_hull(t, r[None, :], np.eye(3))
    assert np.max(np.abs(x - np.minimum(t, r))) < 1e-15


def test_down_hull_inside_returns_t():
    pts = np.array([[-1.0, 0.8], [-3.0, 0.95]])
    for t in ([-2.0, 0.8], [-1.5, 0.5], [-1.0, 0.8]):
        x = P.project_down_hull(np.array(t), pts, np.eye(2))
        assert np.max(np.abs(x - np.array(t))) < 1e-15


def _hull_instance(rng, n, m):
    Phi = np.column_stack([-rng.uniform(1, 5, size=(m, max(n // 2, 1))),
                           rng.uniform(0, 1, size=(m, n - max(n // 2, 1)))])
    t = Phi.max(axis=0) + rng.uniform(-0.5, 0.5, size=n)
    return Phi, t


def test_down_hull_certificate_general_metric():
    rng = np.random.default_rng(4)
    for n, m in [(2, 1), (2, 5), (3, 4), (5, 8), (9, 20), (30, 40)]:
        for _ in range(4):
            Phi, t = _hull_instance(rng, n, m)
            M = _rand_spd(rng, n) if n <= 9 else np.eye(n)
            x, lam = P.project_down_hull(t, Phi, M, return_lambda=True)
            _down_hull_certificate(t, Phi, M, x, lam)


def test_down_hull_brute_force_active_sets():
    """2-3 dimensions: every corral of at most n + 1 generators (points of Phi
    and the rays -e_i, at least one point): its affine minimiser, kept when
    its coefficients are non-negative and no generator improves on it.  The
    minimum-norm point is unique, so every kept candidate must be the
    oracle's projection (in y = R(x - t) coordinates, M = R^T R)."""
    rng = np.random.default_rng(8)
    for n, m in [(2, 3), (2, 5), (3, 4), (3, 5)]:
        for _ in range(4):
            Phi, t = _hull_instance(rng, n, m)
            M = _rand_spd(rng, n)
            R = np.linalg.cholesky(M).T
            gens = np.vstack([(Phi - t) @ R.T, -R.T])
            is_pt = np.arange(m + n) < m
            found = []
            for k in range(1, n + 2):
                for S in itertools.combinations(range(m + n), k):
                    S = list(S)
                    e = is_pt[S].astype(float)
                    if e.sum() == 0:
                        continue
                    Gs = gens[S]
                    K = np.block([[Gs @ Gs.T, e[:, None]], [e[None, :], np.zeros((1, 1))]])
                    if np.linalg.matrix_rank(K) < k + 1:
                        continue
                    c = np.linalg.solve(K, np.r_[np.zeros(k), 1.0])[:k]
                    if np.any(c < -1e-12):
                        continue
                    y = c @ Gs
                    test = gens @ y - np.where(is_pt, y @ y, 0.0)
                    if np.min(test) < -1e-10:
                        continue
                    found.append(t + np.linalg.solve(R, y))
            assert found
            x = P.project_down_hull(t, Phi, M)
            for xb in found:
                assert np.max(np.abs(x - xb)) < 1e-10


def _proj_down_2d_scan(t, pts):
    """2-D brute force: min over segments [a, b] of ||(t - y)_+||, y on the
    segment (convex in the segment parameter; golden-section search)."""
    best, best_x = np.inf, None
    for a, b in itertools.combinations_with_replacement(range(len(pts)), 2):
        pa, pb = pts[a], pts[b]

        def f(lam):
            y = lam * pa + (1 - lam) * pb
            return np.linalg.norm(np.maximum(t - y, 0)), np.minimum(t, y)

        lo, hi = 0.0, 1.0
        g = (np.sqrt(5) - 1) / 2
        for _ in range(200):
            m1, m2 = hi - g * (hi - lo), lo + g * (hi - lo)
            if f(m1)[0] <= f(m2)[0]:
                hi = m2
            else:
                lo = m1
        d, x = f(0.5 * (lo + hi))
        if d < best:
            best, best_x = d, x
    return best, best_x


def test_down_hull_2d_scan():
    rng = np.random.default_rng(2)
    for _ in range(10):
        pts = np.column_stack([-rng.uniform(1, 5, size=4), rng.uniform(0, 1, size=4)])
        t = np.array([-rng.uniform(0.5, 3), rng.uniform(0.3, 1.2)])
        d, x_scan = _proj_down_2d_scan(t, pts)
        x = P.project_down_hull(t, pts, np.eye(2))
        assert np.linalg.norm(t - x) == pytest.approx(d, abs=1e-12)
        assert np.max(np.abs(x - x_scan)) < 1e-6  # the scan's own resolution


def test_planted_mistakes_are_caught():
    """The certificates reject plausible wrong answers: a projection onto
    conv Phi alone (the rays of the down-closure dropped) and one in the
    Euclidean metric for a non-identity M."""
    rng = np.random.default_rng(9)
    Phi, _ = _hull_instance(rng, 3, 4)
    t = Phi.max(axis=0) + np.array([-10.0, 0.3, 0.3])  # far below every point in objective 0
    y, lam, _ = P.min_norm_point(Phi - t)
    with pytest.raises(AssertionError):
        _down_hull_certificate(t, Phi, np.eye(3), t + y, lam)
    # a point whose projection lies inside the segment between two points,
    # where the metric moves it
    Phi = np.array([[-1.0, 0.2], [-3.0, 0.9]])
    t = np.array([-1.5, 0.8])
    M = np.array([[1.0, 0.6], [0.6, 2.0]])
    x_e, lam_e = P.project_down_hull(t, Phi, np.eye(2), return_lambda=True)
    x, lam = P.project_down_hull(t, Phi, M, return_lambda=True)
    assert np.max(np.abs(x - x_e)) > 1e-3
    with pytest.raises(AssertionError):
        _down_hull_certificate(t, Phi, M, x_e, lam_e)
    _down_hull_certificate(t, Phi, M, x, lam)
    _down_hull_certificate(t, Phi, np.eye(2), x_e, lam_e)


# ---------------------------------------------------------------- Algorithm 1


def _achievable_points(prods):
    """All points reachable by a deterministic assignment and simple
    schedulers: C = down(conv of these) (Sec. 3.2)."""
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


def test_alg1_fig2_projects_onto_C():
    """Fig. 2 with t_u = (-1.8, 0.9): infeasible; t_down converges to the
    projection of t_u onto C (Thm 3 (iii), Cor. (iii))."""
    prods = [[C.Product(I.fig2_agent(), I.fig2_task())]]
    pts = _achievable_points(prods)
    t = np.array([-1.8, 0.9])
    supp = lambda w: C.supporting_point(prods, w, eps1=1e-12)[0]
    res = P.alg1(supp, t, eps=1e-7)
    d, x = _proj_down_2d_scan(t, pts)
    assert not res["feasible"]
    assert np.linalg.norm(res["t_dn"] - x) < 1e-5
    assert np.linalg.norm(res["t_up"] - x) < 1e-5
    # the first two directions: e_1, then straight up (M = I)
    assert np.allclose(res["history"][0]["w"], [1, 0])
    assert np.allclose(res["history"][1]["w"], [0, 1], atol=1e-7)


def test_alg1_fig2_feasible_point():
    prods = [[C.Product(I.fig2_agent(), I.fig2_task())]]
    t = np.array([-3.0, 0.5])
    supp = lambda w: C.supporting_point(prods, w, eps1=1e-12)[0]
    res = P.alg1(supp, t, eps=1e-7)
    assert res["feasible"]
    assert np.allclose(res["t_dn"], t)


def _tiny_instance(seed):
    agents = [I.random_tiny_agent(seed, k, n_states=3, n_actions=(1, 1), n_succ=(1, 2)) for k in range(2)]
    tasks = [I.random_tiny_task(seed, 10 + k, n_locs=2, n_ap=2) for k in range(2)]
    return C.products(agents, tasks)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_alg1_theorem3_on_enumerable_instances(seed):
    prods = _tiny_instance(seed)
    pts = _achievable_points(prods)
    rng = np.random.default_rng(seed)
    n = 4
    M = np.eye(n)
    for _ in range(3):
        hi = pts.max(axis=0)
        t = hi + rng.uniform(-0.6, 0.3, size=n)
        supp = lambda w: C.supporting_point(prods, w, eps1=1e-12)[0]
        res = P.alg1(supp, t, M=M, eps=1e-7)
        x_true = P.project_down_hull(t, pts, M)
        dist = np.linalg.norm(t - x_true)
        for h in res["history"]:
            w = h["w"]
            assert np.all(w >= -1e-12) and abs(w.sum() - 1) < 1e-9  # Lemma 6
            # Lemma 7 over the whole achievable set
            assert np.all(pts @ w <= w @ h["r"] + 1e-8)
            # Thm 3 (i) and (iii)
            assert np.linalg.norm(h["t_up"] - P.project_down_hull(h["t_up"], pts, M)) < 1e-6
            assert np.linalg.norm(t - h["t_dn"]) <= dist + 1e-6
            assert dist <= np.linalg.norm(t - h["t_up"]) + 1e-6
        assert np.linalg.norm(res["t_dn"] - x_true) < 1e-5
        feasible_true = dist < 1e-9
        assert res["feasible"] == feasible_true


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_alg1_verification_only_matches_full_loop(seed):
    """The verification-only loop (Sec. 5, Exp. 2: the outer-bound update
    replaced by a break) follows the full loop's directions and points until
    the first separating hyperplane, so its verdict is the full loop's and
    the true one (t inside the achievable set, by enumeration), and its run
    is a prefix of the full run."""
    prods = _tiny_instance(seed)
    pts = _achievable_points(prods)
    rng = np.random.default_rng(100 + seed)
    supp = lambda w: C.supporting_point(prods, w, eps1=1e-12)[0]
    for _ in range(4):
        t = pts.max(axis=0) + rng.uniform(-0.6, 0.3, size=4)
        full = P.alg1(supp, t, eps=1e-7)
        ver = P.alg1(supp, t, eps=1e-7, verify_only=True)
        truth = np.linalg.norm(t - P.project_down_hull(t, pts, np.eye(4))) < 1e-9
        assert ver["feasible"] == full["feasible"] == truth
        assert ver["iterations"] <= full["iterations"]
        for hv, hf in zip(ver["history"], full["history"]):
            assert np.array_equal(hv["w"], hf["w"]) and np.array_equal(hv["r"], hf["r"])
        if not truth:
            h = ver["history"][-1]
            assert h["w"] @ h["r"] < h["w"] @ t  # the separating hyperplane
            assert np.all(pts @ h["w"] <= h["w"] @ h["r"] + 1e-8)


def test_alg1_verification_only_fig2():
    prods = [[C.Product(I.fig2_agent(), I.fig2_task())]]
    supp = lambda w: C.supporting_point(prods, w, eps1=1e-12)[0]
    # t_u of Fig. 2 is not achievable: the second direction separates it
    res = P.alg1(supp, np.array([-1.8, 0.9]), eps=1e-7, verify_only=True)
    assert not res["feasible"] and res["iterations"] == 2
    res = P.alg1(supp, np.array([-3.0, 0.5]), eps=1e-7, verify_only=True)
    assert res["feasible"]
