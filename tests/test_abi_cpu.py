"""The C-ABI library on the CPU: it loads, exports every symbol include/morap.h
declares, and its host-side building blocks (task preprocessing, the
assignment of Algorithm 2, the two projections of Algorithm 1) agree with
the oracle.  No device call is made here."""

import itertools
import os
import re

import numpy as np
import pytest

import instances as I
from oracle import dfa as D
from oracle import core as C
from oracle import pareto as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def M():
    from paper_2305_04397_gb300 import build

    build.build()
    from paper_2305_04397_gb300 import morap

    morap.lib()
    return morap


def _declared():
    src = open(os.path.join(ROOT, "include", "morap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(morap_[a-z_0-9]+)\s*\(", src)) - {"morap_alloc_fn", "morap_free_fn"})


def test_exports_every_declared_symbol(M):
    import ctypes

    lib = ctypes.CDLL(M.LIB_PATH)
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(M.declared_symbols())


def test_config_default(M):
    cfg = M.morap_config_default()
    assert cfg.eps_vi == 1e-8 and cfg.eps_eval == 1e-11 and cfg.tau_policy == 1e-9
    assert cfg.precision == M.PREC_MIXED and cfg.max_sweeps == 100000
    assert cfg.polish == 0 and cfg.skip_unchanged == 1 and cfg.eval_block == 1 and cfg.in_place == 0
    assert cfg.sweep_variant_fp32 == -1 and cfg.sweep_variant_fp64 == -1 and cfg.item_warps_max == 0
    assert cfg.tail_items == -1


@pytest.mark.parametrize("field,val", [("polish", 2), ("in_place", 2), ("eval_block", 3), ("skip_unchanged", 2),
                                       ("launch_mode", 2), ("sweep_variant_fp32", 9), ("sweep_variant_fp64", -2),
                                       ("precision", 7), ("max_sweeps", 0), ("item_warps_max", 3),
                                       ("item_warps_max", 16), ("tail_items", -2)])
def test_config_validation_needs_no_device(M, field, val):
    """Invalid configurations are refused (EINVAL) before any CUDA call."""
    cfg = M.morap_config_default()
    setattr(cfg, field, val)
    with pytest.raises(M.MorapError) as e:
        M.morap_ctx_create(cfg)
    assert e.value.code == M.EINVAL, field


@pytest.mark.parametrize("n", [1, 2, 4, 6, 7])
def test_assignment_vs_brute_force(M, n):
    rng = np.random.default_rng(10 + n)
    for _ in range(4):
        Cm = rng.normal(size=(n, n))
        f = M.morap_assign_max(Cm)
        got = sum(Cm[f[j], j] for j in range(n))
        best = max(sum(Cm[p[j], j] for j in range(n)) for p in itertools.permutations(range(n)))
        assert got == pytest.approx(best, abs=1e-12)
        assert sorted(f) == list(range(n))


def test_assignment_large_vs_oracle(M):
    rng = np.random.default_rng(1)
    Cm = rng.normal(size=(60, 60))
    f = M.morap_assign_max(Cm)
    fo = C.assignment(Cm)
    assert sum(Cm[f[j], j] for j in range(60)) == pytest.approx(sum(Cm[fo[j], j] for j in range(60)), abs=1e-9)


def test_halfspace_projection_vs_oracle(M):
    """The engine's outer-bound projection (interior point with an exact
    active-set finish) against the oracle's least-distance program, to
    1e-10, for the identity and a general metric."""
    rng = np.random.default_rng(2)
    for n, m in [(2, 1), (3, 3), (5, 6), (8, 10), (25, 40)]:
        for _ in range(3):
            Wt = rng.dirichlet(np.ones(n), size=m)
            R = rng.normal(size=(m, n))
            b = np.einsum("ij,ij->i", Wt, R)
            t = R.max(axis=0) + rng.uniform(0.1, 1.0, size=n)
            A = rng.normal(size=(n, n))
            Mm = A @ A.T + n * np.eye(n)
            for MM in (None, Mm):
                z = M.morap_project_halfspaces(t, Wt, b, MM)
                zo = P.project_halfspaces(t, Wt, b, np.eye(n) if MM is None else MM)
                assert np.all(Wt @ z <= b + 1e-9)
                assert np.max(np.abs(z - zo)) < 1e-10, (n, m)


def test_down_hull_projection_vs_oracle(M):
    """The engine's inner-bound projection against the oracle's minimum-norm
    point (Wolfe's algorithm), to 1e-10, for the identity and a general
    metric; t inside, on and outside the down-closure."""
    rng = np.random.default_rng(3)
    for n, m in [(2, 1), (2, 3), (3, 4), (5, 6), (6, 9), (20, 30)]:
        for _ in range(3):
            Phi = np.column_stack([-rng.uniform(1, 5, size=(m, max(n // 2, 1))),
                                   rng.uniform(0, 1, size=(m, n - max(n // 2, 1)))])
            A = rng.normal(size=(n, n))
            for t, MM in ((Phi.max(axis=0) + rng.uniform(-0.5, 0.5, size=n), None),
                          (Phi.max(axis=0) + rng.uniform(-0.5, 0.5, size=n), A @ A.T + n * np.eye(n)),
                          (Phi[0] - 0.01, None), (Phi.mean(axis=0), None)):
                x = M.morap_project_down_hull(t, Phi, MM)
                xo = P.project_down_hull(t, Phi, np.eye(n) if MM is None else MM)
                assert np.max(np.abs(x - xo)) < 1e-10, (n, m)


def test_random_assignment_by_hand(M):
    """Three points with weights 0.5 / 0.3 / 0.2 over two agents and three
    tasks (-1: no agent): P[i][j] sums the weights of the points that give
    task j to agent i (Sec. 3.3, the synthesis)."""
    lam = np.array([0.5, 0.3, 0.2])
    F = np.array([[0, 1, -1], [1, -1, 0], [0, 1, -1]], np.int32)
    P = M.random_assignment(lam, F, 2)
    want = np.array([[0.7, 0.0, 0.3], [0.3, 0.7, 0.0]])
    assert np.max(np.abs(P - want)) < 1e-15
    with pytest.raises(M.MorapError) as e:
        M.random_assignment(lam, np.array([[0, 2, -1]] * 3, np.int32), 2)
    assert e.value.code == M.EINVAL
    with pytest.raises(M.MorapError) as e:
        M.random_assignment(np.array([0.5, -0.1, 0.6]), F, 2)
    assert e.value.code == M.EINVAL


def test_random_assignment_is_doubly_substochastic(M):
    """Convex weights over partial permutations (each agent does at most one
    task, each task at most one agent) give row and column sums <= 1; with
    as many agents as tasks and full permutations, exactly 1 (Birkhoff)."""
    rng = np.random.default_rng(11)
    for nI, nJ in [(3, 5), (4, 4), (6, 2)]:
        m = 7
        lam = rng.dirichlet(np.ones(m))
        F = np.full((m, nJ), -1, np.int32)
        for l in range(m):
            perm = rng.permutation(max(nI, nJ))
            F[l] = [perm[j] if perm[j] < nI else -1 for j in range(nJ)]
        P = M.random_assignment(lam, F, nI)
        assert np.all(P >= 0) and np.all(P.sum(axis=0) <= 1 + 1e-12) and np.all(P.sum(axis=1) <= 1 + 1e-12)
        if nI == nJ:
            assert np.max(np.abs(P.sum(axis=0) - 1)) < 1e-12 and np.max(np.abs(P.sum(axis=1) - 1)) < 1e-12


def test_task_preprocess_vs_oracle(M):
    tasks = [I.fig2_task(), I.sequence_task([1, 2, 3]), I.sequence_task([4, 5], avoid_ap=9)]
    tasks += [I.random_tiny_task(7, k, n_locs=4, n_ap=2) for k in range(6)]
    for t in tasks:
        n, flags = M.morap_task_preprocess(t.n_locs, t.q0, t.n_ap, t.delta, t.accepting)
        d = D.preprocess(t)
        assert n == d["n_locs"]
        assert [bool(f & 1) for f in flags] == list(d["accepting"])
        assert [bool(f & 2) for f in flags] == list(d["trap"])
        assert [bool(f & 4) for f in flags] == list(d["pre"])
        assert [bool(f & 8) for f in flags] == list(d["done"])


def test_task_preprocess_rejects_non_sink_accepting(M):
    delta = np.array([[1, 1], [0, 1]], np.int32).reshape(-1)
    with pytest.raises(M.MorapError) as e:
        M.morap_task_preprocess(2, 0, 1, delta, np.array([0, 1], np.uint8))
    assert e.value.code == M.EINVAL
    assert "not a sink" in str(e.value)


def test_pareto_stepper_synthesis_on_a_known_set(M):
    """Algorithm 1 fed from a known achievable set (the down-closure of the
    convex hull of four points, supporting points found by enumeration): the
    loop decides feasibility as the geometry says, and its convex weights
    reproduce a point that dominates t_up (t itself when feasible)."""
    pts = np.array([[-1.0, 0.2], [-2.0, 0.6], [-4.0, 0.9], [-3.0, 0.5]])

    def support(w):
        return pts[int(np.argmax(pts @ w))]

    # (-3, 0.7) needs a mix: half of (-2, 0.6) and half of (-4, 0.9) gives (-3, 0.75)
    for t, feasible in (([-2.5, 0.6], True), ([-3.0, 0.7], True), ([-2.5, 0.7], False), ([-3.5, 0.95], False)):
        P = M.Pareto(t, eps=1e-9, max_iter=30)
        while True:
            w = P.next()
            if w is None:
                break
            P.step(support(w))
        res = P.result()
        P.close()
        lam = res["lambda"]
        assert res["feasible"] == feasible
        assert np.all(lam >= 0) and abs(lam.sum() - 1) < 1e-12
        assert np.all(lam @ res["r_hist"] >= res["t_up"] - 1e-9)
        if feasible:
            assert np.all(lam @ res["r_hist"] >= np.array(t) - 1e-9)


def test_pareto_stepper_verification_only(M):
    """The verification-only stepper on the same known set: the verdicts of
    the full loop, never more points, and its points a prefix of the full
    loop's; the oracle's verification-only loop gives the same run."""
    from oracle import pareto as OP

    pts = np.array([[-1.0, 0.2], [-2.0, 0.6], [-4.0, 0.9], [-3.0, 0.5]])

    def support(w):
        return pts[int(np.argmax(pts @ w))]

    def run(t, verify_only):
        P = M.Pareto(t, eps=1e-9, max_iter=30, verify_only=verify_only)
        while True:
            w = P.next()
            if w is None:
                break
            P.step(support(w))
        res = P.result()
        P.close()
        return res

    for t, feasible in (([-2.5, 0.6], True), ([-3.0, 0.7], True), ([-2.5, 0.7], False), ([-3.5, 0.95], False)):
        full, ver = run(t, False), run(t, True)
        assert ver["feasible"] == full["feasible"] == feasible and ver["converged"]
        assert ver["iterations"] <= full["iterations"]
        assert np.array_equal(ver["r_hist"], full["r_hist"][: ver["iterations"]])
        ref = OP.alg1(support, np.array(t), eps=1e-9, max_iter=30, verify_only=True)
        assert ref["feasible"] == feasible and ref["iterations"] == ver["iterations"]
        if not feasible:
            assert np.array_equal(ver["t_down"], np.array(t))  # the outer bound is never projected
