"""The fit workload's synthetic outputs (fitbench.synthetic_times, plain
NumPy from the models' term lists) equal the oracle's evaluation of the same
model expressions at the same parameters, so the oracle and the GPU fits
calibrate on data neither of them produced."""
import numpy as np

import pm_inputs
from oracle.model import Model as OModel
from paper_1904_09538_gb300.fitbench import TRUTH, features, model_expr, synthetic_times


def test_synthetic_times_match_oracle_model_evaluation():
    K = 64
    oms = [OModel("f_wall_time", model_expr(k)) for k in range(K)]
    Xs, ls = features(K, lambda k: len(oms[k].features))
    assert {len(om.params) for om in oms} == set(range(4, 13))
    for k, (om, X) in enumerate(zip(oms, Xs)):
        t = synthetic_times(k, om.features, X)
        g = np.array([om.eval(TRUTH, dict(zip(om.features, row))) for row in X])
        want = g * (1 + 1e-2 * pm_inputs.noise((len(X),), 9900 + k))
        assert np.max(np.abs(t / want - 1)) <= 1e-14, k
