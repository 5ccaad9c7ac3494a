"""Failure detection without a GPU fault: a bounded device wait that runs out is reported to
the host as HAMR_ERR_TIMEOUT, and the device context stays usable afterwards.  The wait is
made to run out by a test hook that withholds one arrival on a staging barrier (nothing is
left unset that the hardware would wait on forever, and nothing faults)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_02236_gb300 import build
    build.build()
    from paper_2502_02236_gb300 import hamr, inputs as I
    return hamr, I


@pytest.mark.parametrize("periodic", [(False, False, False), (True, True, False)])
def test_bounded_wait_reports_timeout_and_context_survives(env, periodic):
    hamr, I = env
    dims = (40, 36, 10)
    n = int(np.prod(dims))
    S0 = I.initial_state(n, "tilt", seed=3, tilt_deg=20)
    with hamr.Lattice([dims], [5], precision="fp32", a=0.25e-9, periodic=periodic, mu_s=I.MU_S, ku=I.KU_SC,
                      alpha=0.1, dt=1e-16) as lat:
        lat.set_neighbour_shells([I.J_SC])
        lat.set_temperature_profile(0, 300.0)
        lat.set_moments(0, S0)
        lat.inject_wait_timeout(4096)
        with pytest.raises(hamr.HamrError) as e:
            lat.sllg_heun_steps(1)
        assert e.value.code == hamr.ERR_TIMEOUT
        # the hook is spent; the handle and the device context still work
        lat.step = 0
        lat.set_moments(0, S0)
        lat.sllg_heun_steps(20)
        assert lat.check_finite()
        S = lat.read_moments(0)
        assert np.allclose(np.linalg.norm(S, axis=1), 1.0, atol=1e-5)
