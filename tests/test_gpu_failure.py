"""Failure detection on the GPU without a fault: the bounded waits give up and
report, and the context keeps working afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_21242_gb300 import capi, flows
from paper_2602_21242_gb300.lattice import Lattice

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_times_out_and_context_survives(oracle, which):
    status, secs = capi.lbm_selftest_timeout(which)
    assert status == capi.LBM_ETIMEOUT
    assert 0.2 < secs < 10.0
    # the context is still usable: a small run still matches the oracle
    f0 = flows.random_populations(16, 12, seed=77)
    with Lattice(16, 12, 0.35, 0.8, "complete") as lat:
        lat.set_state(torch.from_numpy(f0).cuda())
        lat.step(5)
        got = lat.state().cpu().numpy()
    ref = oracle.run(f0, 0.35, 0.8, 3, 5)
    assert np.max(np.abs(got - ref) / np.abs(ref).max(axis=0)) <= 1e-12


def test_host_side_faults_are_reported():
    """Errors made on the host: bad sizes, stepping before init, a NaN state."""
    with pytest.raises(capi.LBMError):
        Lattice(0, 4, 0.3, 0.6)
    with Lattice(8, 8, 0.3, 0.6, "oreg") as lat:
        with pytest.raises(capi.LBMError) as e:
            lat.step(1)
        assert e.value.status == capi.LBM_ESTATE
        f = flows.random_populations(8, 8, seed=2)
        f[0, 0, 0] = np.inf
        lat.set_state(torch.from_numpy(f).cuda())
        lat.set_diagnostics_interval(1)
        lat.step(2)
        with pytest.raises(capi.LBMError) as e:
            lat.sync()
        assert e.value.status == capi.LBM_ENONFINITE
