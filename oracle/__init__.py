"""Independent FP64 CPU oracle for the MORAP hot path (arxiv 2305.04397).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import, call, link or execute
anything under oracle/.  The engine (paper_2305_04397_gb300) never does, and
the two share no code: the only common module is `instances`, which
generates seeded inputs and holds none of the method's arithmetic.

Contents, each following the passage cited in its docstring:
  dfa.py     task-DFA preprocessing: traps, done_j, pre-sinks (Sec. 2, 3.1)
  oracle.c   product MDP (Sec. 2), Algorithm 3, the scheduler reading,
             Algorithm 4 (Appendix A.4) -- plain C loops, FP64
  core.py    ctypes wrappers, exact fixed-scheduler values (dense LU),
             brute force over simple schedulers, Algorithm 2 with the
             assignment step (scipy's linear_sum_assignment)
  pareto.py  Algorithm 1 and its two projections (scipy SLSQP)
  lp.py      the MORAP problem as one linear program (occupation measures,
             Lemma 2 for the random assignment) and a hand-written dense
             simplex: a second decision of "is t achievable?" for tiny
             instances

Every function is pinned by tests/test_oracle_*.py against closed forms,
brute force, exact linear solves, invariants of Sec. 3 (Lemmas 6-7, Thm 3)
and the values printed for the worked example of Fig. 2.
"""
