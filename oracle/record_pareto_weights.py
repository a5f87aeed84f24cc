"""Record the weight vectors of the 32x32-grid batch from Algorithm 1 runs
(Sec. 3.3) computed by the oracle: the batch's "weight vectors from the
Pareto loop".  Test and benchmark infrastructure: it runs only the oracle
(FP64 C Algorithms 2-4 per pair, the exact projections of oracle/pareto.py)
on the seeded instance and writes the directions to
instances/data/grid32_pareto_weights.txt, which the benchmark reads as data.

Algorithm 1 starts every run at w = e_1 and then points each direction from
the current inner point t_up towards the threshold t (entries that rounding
makes slightly negative are weights of 0).  The runs start from
the instance's threshold points in turn; directions already recorded (the
repeated e_1) are not repeated; the first K distinct directions are kept.

    python -m oracle.record_pareto_weights
"""

from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

from instances import gen as G  # noqa: E402
from oracle import core as O  # noqa: E402
from oracle import pareto as PA  # noqa: E402

OUT = os.path.join(ROOT, "instances", "data", "grid32_pareto_weights.txt")


def supporting_point_pooled(inst, procs=None):
    """Algorithm 2 for one direction: Algorithm 3 and 4 for every pair on the
    host cores, then the assignment (as oracle.core.supporting_point)."""
    nI, nJ = len(inst.agents), len(inst.tasks)

    def sp(w):
        jobs = [(inst.agents[i], inst.tasks[j], float(w[i]), float(w[nI + j]), 1e-8)
                for i in range(nI) for j in range(nJ)]
        res = O.solve_pairs_pooled(jobs, procs)
        C = np.array([r[0] for r in res]).reshape(nI, nJ)
        RC = np.array([r[1] for r in res]).reshape(nI, nJ)
        RP = np.array([r[2] for r in res]).reshape(nI, nJ)
        f = O.assignment(O.pad_square(C))
        r = np.zeros(nI + nJ)
        for j in range(nJ):
            i = int(f[j])
            if i < nI:
                r[i] = RC[i, j]
                r[nI + j] = RP[i, j]
        return r

    return sp


def record(K=16, seed=1, procs=None):
    inst = G.config_grid32(seed=seed)
    sp = supporting_point_pooled(inst, procs)
    dirs = []
    for t in inst.thresholds:
        run = PA.alg1(sp, t, eps=1e-6, max_iter=K)
        for h in run["history"]:
            # t_up lies below t, so M (t - t_up) >= 0 up to the projections'
            # rounding (entries of -1e-13 on the objectives t_up meets): those
            # are weights of 0, as the engine's Algorithm 1 forms them
            w = np.maximum(np.asarray(h["w"], np.float64), 0.0)
            if not any(np.array_equal(w, d) for d in dirs):
                dirs.append(w)
        print(f"threshold run: {run['iterations']} iterations, feasible={run['feasible']}, "
              f"{len(dirs)} distinct directions so far", flush=True)
        if len(dirs) >= K:
            break
    return np.array(dirs[:K])


def main():
    W = record()
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as f:
        f.write("# Weight vectors of the 32x32-grid batch (config_grid32, seed 1): the first 16\n")
        f.write("# distinct directions of Algorithm 1 runs (Sec. 3.3) from the instance's threshold\n")
        f.write("# points in turn, computed by the oracle (written by oracle/record_pareto_weights.py).\n")
        f.write(f"# {W.shape[0]} rows x {W.shape[1]} columns (10 agent costs, then 20 task probabilities)\n")
        for w in W:
            f.write(" ".join(repr(float(x)) for x in w) + "\n")
    print(f"wrote {W.shape[0]} directions to {OUT}")


if __name__ == "__main__":
    main()
