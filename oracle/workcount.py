"""Operation counts of the oracle's pointwise routines, for the roofline numerator.

TEST INFRASTRUCTURE, like the rest of this package: the CUDA library never runs
it. The oracle's C++ routines are instantiated on an operation-counting dual
number (``Cnt`` in ift_oracle.cpp: one count per +, -, *, /, sqrt, exp; a
derivative that is structurally zero costs nothing), and this module evaluates
them at one representative state of the benchmark's Euler problem:

* the Euler flux f(U) (Eq. p2r-flux with the Euler flux of Sec. 4.2): its value
  and one forward-mode derivative along a state direction;
* the Roe flux H(U+, U-; n): its value and one derivative along U+ and along U-,
  at a face where no wave speed lies within the entropy-fix width (the fixed
  branch costs a few operations more and is not counted);
* the Burgers Roe flux: value and one derivative along u+.

``python -m oracle.workcount`` prints the constants that
paper_2305_15661_gb300/perfmodel.py stores; a CPU test checks that the two agree.
"""

from __future__ import annotations

import numpy as np

from . import PROB_BURGERS1D, PROB_EULER2D, Oracle, freestream


def _tiny_oracle(problem):
    if problem == PROB_EULER2D:
        X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
        ev = np.array([[0, 1, 2]], dtype=np.int32)
    else:
        X = np.array([0.0, 1.0])
        ev = np.array([[0, 1]], dtype=np.int32)
    return Oracle(problem, 1, X, ev)


def euler_counts(gamma: float = 1.4) -> dict:
    O = _tiny_oracle(PROB_EULER2D)
    Um = freestream(gamma, np.array([2.0, 0.0]))
    Up = freestream(gamma, np.array([2.0, 0.01])) * (1.0 + 1e-2 * np.array([1.0, -1.0, 1.0, -1.0]))
    n = 0.01 * np.array([0.6, 0.8])
    d = np.array([1.0, 0.5, -0.25, 2.0])
    fv, ft = O.count_pointwise(0, Up, Up, n, d)
    hv, hp = O.count_pointwise(1, Up, Um, n, d)
    _, hm = O.count_pointwise(4, Up, Um, n, d)
    return {"flux": (fv, ft), "roe": (hv, hp, hm)}


def burgers_counts() -> dict:
    O = _tiny_oracle(PROB_BURGERS1D)
    hv, hp = O.count_pointwise(2, np.array([1.2]), np.array([1.0]), np.array([1.0]), np.array([1.0]))
    return {"roe": (hv, hp)}


if __name__ == "__main__":
    e = euler_counts()
    b = burgers_counts()
    print(f"EULER_FLUX = {e['flux']}")
    print(f"EULER_ROE = {e['roe']}")
    print(f"BURGERS_ROE = {b['roe']}")
