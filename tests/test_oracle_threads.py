"""The oracle's node loops run on several threads (OpenMP): every node is
computed on its own, so the state after a few steps is bit-identical for
any thread count."""
import numpy as np

import oracle as O
from paper_2002_04353_gb300 import inputs as I


def test_oracle_state_does_not_depend_on_the_thread_count():
    case = I.plunge_case(ni=64, nj=20, chord=200.0)
    states = []
    n0 = O.threads()
    try:
        for n in (1, 3):
            assert O.threads(n) == n
            o = O.Oracle(case.mesh, case.motion, case.flow)
            o.step(5)
            states.append(o.state())
    finally:
        O.threads(n0)
    for k in ("f", "g", "rho", "ux", "uy", "T"):
        assert np.array_equal(states[0][k], states[1][k]), k
