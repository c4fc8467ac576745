"""Estimators computed from the GPU's int64 accumulators equal those of the oracle run.

The accumulators are bit-exact with the oracle after every sweep, so every host-side
estimator (batch means, error bars, autocorrelation times, rates) read from a sequence of
GPU observations must equal, element for element, the one read from the oracle's."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1004_0023_gb300 import estimators, instances, pt

pytestmark = pytest.mark.gpu


def _equal(a, b, what):
    if isinstance(a, dict):
        assert a.keys() == b.keys(), what
        for k in a:
            _equal(a[k], b[k], what + "." + k)
    else:
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b), err_msg=what)


@pytest.mark.parametrize("name,window,windows", [("regular3_n16_p32_r16", 100, 20), ("regular3_n256_p64_r64", 25, 8)])
def test_estimators_from_gpu_accumulators_equal_the_oracle_runs(libpt, name, window, windows):
    prob = instances.workload(name, 4)
    g = pt.PT.from_problem(prob)
    o = Oracle.from_problem(prob, threads=8)
    hg, ho = [g.obs()], [o.obs()]
    for _ in range(windows):
        g.run(window, 1)
        o.run(window, 1)
        hg.append(g.obs())
        ho.append(o.obs())
    g.close()
    o.close()
    args = (prob.n, prob.P, prob.T, prob.gamma)
    _equal(estimators.autocorrelation(hg, *args), estimators.autocorrelation(ho, *args), "autocorrelation")
    _equal(estimators.rate_errors(hg), estimators.rate_errors(ho), "rate_errors")
    _equal(estimators.quantum_energy(hg[-1], *args, since=hg[0]), estimators.quantum_energy(ho[-1], *args, since=ho[0]),
           "quantum_energy")
    _equal(estimators.round_trips([h["replica_at"] for h in hg]), estimators.round_trips([h["replica_at"] for h in ho]),
           "round_trips")
