"""The stored oracle Newton solutions of the slab workloads (written by
tests/golden/newton_truth.py, which calls only the oracle) still belong to
the current input generators and still solve the oracle's equations."""
import os
import sys

import numpy as np
import pytest

from oracle.assembly import FEProblem
from workloads import slab_config

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
from newton_truth import WORKLOADS, input_digest, load_truth, truth_path  # noqa: E402


@pytest.mark.parametrize("name", WORKLOADS)
def test_stored_newton_solution_solves_the_oracle_equations(name):
    assert os.path.exists(truth_path(name))
    d, digest, log = load_truth(name)
    prob = slab_config(name)
    assert digest == input_digest(prob)
    fe = FEProblem(prob)
    assert d.shape == (fe.n_free,)
    # Newton stopped at 1e-11 of the last load step's initial residual,
    # which is below the residual of the full load at d = 0
    r = fe.residual(d, 1.0)
    r0 = fe.residual(np.zeros(fe.n_free), 1.0)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(r0)
    assert fe.min_jacobian(d) > 0.0
    # every load level reached without halving, each one converged to 1e-11
    lams = sorted({rec["lam"] for rec in log})
    assert lams == [0.25, 0.5, 0.75, 1.0]
    for lam in lams:
        last = [rec for rec in log if rec["lam"] == lam][-1]
        assert last["res_new"] <= 1e-11 * last["r0"]
