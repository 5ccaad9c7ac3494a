"""The step entry point that allocates nothing (hamr_sllg_heun_step_noalloc), for callers
that cannot call cudaMalloc and so cannot create a handle: two calls in a row through the C
ABI must give what the handle-based FP64 path gives for the same two steps.

This file is collected last on purpose; it must pass on its own in a fresh process and
after the rest of the suite.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_02236_gb300 import build
    build.build()
    from paper_2502_02236_gb300 import hamr, inputs as I
    return torch, hamr, I


def test_noalloc_two_steps_match_handle_path(env):
    torch, hamr, I = env
    nx, ny, nz, a = 40, 33, 7, 0.25e-9
    g2 = I.voronoi_grains(nx, ny, a, a, 3e-9, 0.5e-9, 21)
    grain = I.columnar(g2, nz)
    ng = int(g2.max()) + 1
    n = nx * ny * nz
    S0 = I.mask_void(I.initial_state(n, "tilt", seed=4, tilt_deg=25), grain)
    phys = dict(a=a, mu_s=I.MU_S, ku=I.KU_SC, alpha=0.1, dt=1e-16)
    T = dict(T_amb=300.0, T_peak=850.0, fwhm=5e-9, x0=3e-9, y0=4e-9, vx=2e4, vy=0.0)
    B = (0.2, 0.0, -1.0)
    seed = 77

    # the existing entry points: a handle, one step per call
    lat = hamr.Lattice([(nx, ny, nz)], [seed], precision="fp64", periodic=(True, False, False), **phys)
    lat.set_neighbour_shells([I.J_SC])
    lat.set_grain_map(0, grain, ng)
    lat.set_temperature_profile(0, **T)
    lat.set_field_sequence(0, 1.0, B)
    lat.set_moments(0, S0)
    lat.sllg_heun_steps(1)
    ref1 = lat.read_moments(0)
    lat.sllg_heun_steps(1)
    ref2 = lat.read_moments(0)
    lat.close()

    # the entry point without allocation, on buffers the caller owns
    S_in = torch.from_numpy(S0).cuda()
    S_out = torch.empty_like(S_in)
    g = torch.from_numpy(grain).cuda()
    torch.cuda.synchronize()
    kw = dict(grain=g, periodic=(True, False, False), J=I.J_SC, seed=seed, B_app=B, **phys, **T)
    hamr.sllg_heun_step_noalloc((nx, ny, nz), S_in, S_out, step=0, **kw)
    torch.cuda.synchronize()
    got1 = S_out.cpu().numpy()
    hamr.sllg_heun_step_noalloc((nx, ny, nz), S_out, S_out, step=1, **kw)   # in place
    torch.cuda.synchronize()
    got2 = S_out.cpu().numpy()

    assert np.max(np.abs(got1 - ref1)) < TOL64
    assert np.max(np.abs(got2 - ref2)) < TOL64
    assert np.max(np.abs(got2 - S0)) > 1e-4          # the steps did move the spins
    assert np.array_equal(got2[grain < 0], S0[grain < 0])

    # and directly against the FP64 oracle for the same two steps
    import oracle as orc
    p = orc.sc_params(nx, ny, nz, a, I.J_SC, periodic=(True, False, False), mu_s=I.MU_S, ku=I.KU_SC, alpha=0.1,
                      dt=1e-16, seed=seed, **T, B0=1.0, direction=B)
    S = np.ascontiguousarray(S0.copy())
    orc.Oracle(p, grain).run(S, 0, 2)
    assert np.max(np.abs(got2 - S)) < TOL64

    # an output that partly overlaps the input is refused on the host
    big = torch.zeros((2 * n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(hamr.HamrError, match="overlaps") as e:
        hamr.sllg_heun_step_noalloc((nx, ny, nz), big[:n], big[n // 2:n // 2 + n], step=0, **kw)
    assert e.value.code == hamr.ERR_ARG


def test_noalloc_rejects_oversize(env):
    torch, hamr, I = env
    n = hamr.NOALLOC_MAX_SITES + 1
    S = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(hamr.HamrError, match="HAMR_NOALLOC_MAX_SITES") as e:
        hamr.sllg_heun_step_noalloc((n, 1, 1), S, S, a=0.25e-9, mu_s=I.MU_S, J=I.J_SC)
    assert e.value.code == hamr.ERR_ARG
