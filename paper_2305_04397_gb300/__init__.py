"""GB300-native engine for multi-objective random task assignment and
planning (arxiv 2305.04397): batched weighted-sum value iteration over all
agent x task product MDPs, per-objective policy evaluation, the assignment
step and the point-oriented Pareto loop, behind the C-ABI of
include/morap.h (libmorap.so).  `morap` is the thin ctypes binding.
"""

from . import morap  # noqa: F401
