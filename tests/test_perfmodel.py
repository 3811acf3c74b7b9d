"""The work model behind the roofline numerator (paper_2305_15661_gb300/perfmodel.py).

* The operation-counting dual number of the oracle is checked against counts done
  by hand on two routines: the Euler flux f(U) (19 value operations; 41 for the
  derivative along a direction that seeds all four state components) and the
  Burgers Roe flux (17 value operations; 15 for the derivative along u+, with the
  structurally zero terms of u- and n costing nothing).
* The constants the model stores are the ones oracle/workcount.py counts.
* The model's residual and per-column counts do not exceed what the oracle's own
  element routine performs (the oracle is written for clarity, not economy, so
  its counts are upper bounds of the minimal work).
"""

import numpy as np

import oracle as orc
from oracle import workcount
from paper_2305_15661_gb300 import perfmodel as P
from paper_2305_15661_gb300 import workloads as W


def test_counter_against_hand_counts():
    e = workcount.euler_counts()
    assert e["flux"] == (19, 41)
    b = workcount.burgers_counts()
    assert b["roe"] == (17, 15)


def test_stored_constants_are_the_counted_ones():
    e = workcount.euler_counts()
    assert P.EULER_FLUX == e["flux"]
    assert P.EULER_ROE == e["roe"]
    assert P.BURGERS_ROE == workcount.burgers_counts()["roe"]


def test_model_does_not_exceed_the_oracles_own_operations():
    wl = W.euler_workload(n=6, p=2, k_u=20, k_x=4, seed=2)
    O = orc.Oracle.from_workload(wl)
    U = wl.Phi @ wl.w_eval
    x = wl.X.ravel() + wl.Psi @ wl.tau_eval
    e = 17
    Ue, Up, xe = O.gather(U, x, e)
    Phie, Phip, Psie = O.gather_rows(wl.Phi, wl.Psi, e)
    value, _ = O.count_element(e, Ue, Up, xe, wl.mus[0])
    _, along_state = O.count_element(e, Ue, Up, xe, wl.mus[0], dUe=Phie[:, 0], dUp=Phip[:, 0])
    _, along_mesh = O.count_element(e, Ue, Up, xe, wl.mus[0], dxe=Psie[:, 0])
    m = P.flops_per_element(2, 2, 20, 4)
    assert m["residual"] <= value
    assert m["state_columns"] / 20 <= along_state
    assert m["mesh_columns"] / 4 <= along_mesh
    # the full assembly: every part counted once, the total their sum
    parts = ("reconstruction", "residual", "objective", "pointwise_jacobians", "state_columns",
             "mesh_columns", "contraction")
    assert m["total"] == sum(m[k] for k in parts)
    assert m["element"] + m["reduction"] == m["total"]
