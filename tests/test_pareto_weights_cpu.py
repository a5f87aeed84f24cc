"""The 32x32-grid batch's weight vectors are Algorithm 1 directions (Sec. 3.3)
recorded by the oracle (oracle/record_pareto_weights.py).  Check the data
file against what it claims: 16 distinct directions on the simplex, the
first e_1 (Algorithm 1's initial direction), and the second the direction
Algorithm 1 takes after the first supporting point, recomputed here from
one oracle supporting point at e_1 and the down-hull projection."""

import numpy as np

import instances as I
from oracle import core as O
from oracle import pareto as PA


def test_recorded_directions_are_algorithm1_directions():
    inst = I.config_grid32(pareto_weights=True)
    W = inst.weights
    nI, nJ = len(inst.agents), len(inst.tasks)
    assert W.shape == (16, nI + nJ)
    assert np.all(W >= 0) and np.allclose(W.sum(axis=1), 1.0, atol=1e-12)
    assert len({tuple(w) for w in W}) == 16
    e1 = np.zeros(nI + nJ)
    e1[0] = 1.0
    assert np.array_equal(W[0], e1)
    # one supporting point at e_1 (Algorithm 2 by the oracle, pairs on the host cores)
    jobs = [(inst.agents[i], inst.tasks[j], float(e1[i]), float(e1[nI + j]), 1e-8)
            for i in range(nI) for j in range(nJ)]
    res = O.solve_pairs_pooled(jobs)
    C = np.array([r[0] for r in res]).reshape(nI, nJ)
    RC = np.array([r[1] for r in res]).reshape(nI, nJ)
    RP = np.array([r[2] for r in res]).reshape(nI, nJ)
    f = O.assignment(O.pad_square(C))
    r = np.zeros(nI + nJ)
    for j in range(nJ):
        if int(f[j]) < nI:
            r[int(f[j])] = RC[int(f[j]), j]
            r[nI + j] = RP[int(f[j]), j]
    t = inst.thresholds[0]
    t_up = PA.project_down_hull(t, r[None, :], np.eye(nI + nJ))
    d = t - t_up
    assert np.allclose(W[1], np.maximum(d, 0.0) / np.abs(d).sum(), atol=1e-9)
