"""Oracle: task-DFA preprocessing (test infrastructure only).

Follows Sec. 2 ("Deterministic Finite Automata": sinks, successors, traps
Q_R) and Sec. 3.1 (done_j holds on Q_F u Q_R; the probability reward
rho_{j+|I|}(s,q,a) = 1 iff q is not accepting and every successor of q is
accepting, a "pre-sink"; when no such location exists the DFA is extended
with one without changing its language).

Reading taken where the paper is brief: every transition into an accepting
location must leave from a pre-sink, otherwise the one-off reward would not
count every accomplishment.  So each transition delta(q, W) in Q_F from a
non-accepting location q that is not a pre-sink is redirected to one new
location P whose every letter leads to an accepting location.  P is then a
pre-sink and the accepted words are unchanged apart from one extra step.
"""

from __future__ import annotations

import numpy as np


def preprocess(task):
    nl = 1 << int(task.n_ap)
    n = int(task.n_locs)
    delta = np.asarray(task.delta, np.int64).reshape(n, nl).copy()
    acc = np.asarray(task.accepting).astype(bool).copy()
    if not (0 <= int(task.q0) < n):
        raise ValueError("q0 out of range")
    if delta.min() < 0 or delta.max() >= n:
        raise ValueError("delta target out of range")
    for q in range(n):
        if acc[q] and np.any(delta[q] != q):
            raise ValueError(f"accepting location {q} is not a sink")

    def is_pre(q):
        return (not acc[q]) and bool(np.all(acc[delta[q]]))

    pre_orig = [is_pre(q) for q in range(n)]
    redirect = [(q, W) for q in range(n) if not acc[q] and not pre_orig[q]
                for W in range(nl) if acc[delta[q, W]]]
    if redirect:
        f = int(np.flatnonzero(acc)[0])
        P = n
        delta = np.vstack([delta, np.full((1, nl), f, np.int64)])
        acc = np.append(acc, False)
        for q, W in redirect:
            delta[q, W] = P
        n += 1
    pre = np.array([is_pre(q) for q in range(n)], bool)

    # traps: no run reaches an accepting location
    reach = acc.copy()
    changed = True
    while changed:
        changed = False
        for q in range(n):
            if not reach[q] and np.any(reach[delta[q]]):
                reach[q] = True
                changed = True
    trap = ~reach
    done = acc | trap
    nd_loc = np.flatnonzero(~done).astype(np.int32)
    nd_pos = -np.ones(n, np.int32)
    nd_pos[nd_loc] = np.arange(len(nd_loc), dtype=np.int32)
    return {
        "n_locs": n,
        "n_letters": nl,
        "q0": int(task.q0),
        "delta": delta.astype(np.int32),
        "accepting": acc,
        "trap": trap,
        "done": done,
        "pre": pre,
        "nd_loc": nd_loc,
        "nd_pos": nd_pos,
        "inserted_presink": bool(redirect),
    }


def letters(agent, task):
    """The letter of task `task` read on each agent state: bit b is set when
    the task's b-th atomic proposition is in L(s)."""
    ap_bit = {int(ap): b for b, ap in enumerate(task.ap_ids)}
    out = np.zeros(agent.n_states, np.int32)
    for s in range(agent.n_states):
        v = 0
        for k in range(agent.label_ptr[s], agent.label_ptr[s + 1]):
            b = ap_bit.get(int(agent.label_ap[k]))
            if b is not None:
                v |= 1 << b
        out[s] = v
    return out
