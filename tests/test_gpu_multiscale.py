"""The multiscale write window on the GPU (hamr_ms_*, FP64) against the FP64 oracle: same
seeded inputs, element-by-element comparison of the micromagnetic cells and the window spins
within 1e-9 (FP64) or 2e-4 (FP32).  Cases: a stationary window with the laser spot and write field on, a window
moving with a fast spot through several shifts, the 1 nm / 0.25 nm geometry of the full
track at reduced size, the full 500 x 60 x 10 nm track for two steps, and call-order errors."""
import numpy as np
import pytest

import oracle as orc
from paper_2502_02236_gb300 import inputs as I
from paper_2502_02236_gb300.hamr import ERR_ARG, ERR_STATE, HamrError, Multiscale

TOL = {"fp64": 1e-9, "fp32": 2e-4}
PRECISIONS = ["fp64", "fp32"]


def pair(w, precision="fp64", profile=None, demag=False, margin=-1):
    """The oracle and the GPU handle for one multiscale input description."""
    T, F = w["T"], w["field"]
    p = orc.MsParams(w["ncx"], w["ncy"], w["ncz"], w["cell"], w["ratio"], w["wx"], J=w["J"], mu_s=w["mu_s"],
                     ku=w["ku"], lam=w["lam"], T_C=w["T_C"], Ms0=w["Ms0"], A0=w["A0"], K0=w["K0"], dt=w["dt"],
                     seed=w["seed"], **T, B0=F["B0"], direction=F["direction"], bits=F["bits"],
                     bit_len=F["bit_len"], ramp_len=F["ramp_len"], head_x0=F["head_x0"], head_v=F["head_v"],
                     profile=profile, demag=demag, margin=margin)
    O = orc.MsOracle(p, w["grain"])
    G = Multiscale(w["ncx"], w["ncy"], w["ncz"], w["cell"], w["ratio"], w["wx"], J=w["J"], mu_s=w["mu_s"],
                   ku=w["ku"], Ms0=w["Ms0"], A0=w["A0"], K0=w["K0"], lam=w["lam"], T_C=w["T_C"], dt=w["dt"],
                   seed=w["seed"], precision=precision)
    G.set_grain_map(w["grain"])
    G.set_temperature_profile(**T)
    G.set_field_sequence(**F)
    if profile:
        G.set_head_profile(**profile)
    if demag:
        G.set_demag(True)
    if margin >= 0:
        G.set_region(margin)
    return p, O, G


def params(w, T=None, F=None, profile=None, demag=False):
    """Oracle parameters of an input description with the drivers T, F (those of w by default)."""
    T, F = T or w["T"], F or w["field"]
    return orc.MsParams(w["ncx"], w["ncy"], w["ncz"], w["cell"], w["ratio"], w["wx"], J=w["J"], mu_s=w["mu_s"],
                        ku=w["ku"], lam=w["lam"], T_C=w["T_C"], Ms0=w["Ms0"], A0=w["A0"], K0=w["K0"], dt=w["dt"],
                        seed=w["seed"], **T, B0=F["B0"], direction=F["direction"], bits=F["bits"],
                        bit_len=F["bit_len"], ramp_len=F["ramp_len"], head_x0=F["head_x0"], head_v=F["head_v"],
                        profile=profile, demag=demag)


def tilted_cells(w, seed=3, deg=35.0):
    n = w["ncx"] * w["ncy"] * w["ncz"]
    S = I.initial_state(n, "tilt", seed=seed, tilt_deg=deg)
    return I.mask_void(S, w["grain"])


def start(w, p, O, G, ox):
    m = tilted_cells(w)
    O.set_cells(m)
    G.set_cells(m)
    O.set_window(ox)
    G.set_window(ox)


def compare(O, G):
    dm = np.abs(G.read_cells() - O.cells()).max()
    dS = np.abs(G.read_moments() - O.moments()).max()
    return dm, dS


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_stationary_window_matches_oracle(prec):
    w = I.multiscale_track(ncx=20, ncy=6, ncz=2, cell=1e-9, ratio=2, wx=6, grain_d=5e-9, boundary=1e-9, seed=21,
                           v=0.0, x_spot=10e-9)
    p, O, G = pair(w, prec)
    tol = TOL[prec]
    with G:
        start(w, p, O, G, 7)
        dm, dS = compare(O, G)
        # placement: the same thermalised spins (FP32 stores them rounded)
        assert dm < tol and dS < (1e-12 if prec == "fp64" else 1e-7)
        O.run(200)
        G.steps(200)
        dm, dS = compare(O, G)
        assert dm < tol and dS < tol, (dm, dS)
        assert G.window() == (7, 200)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_moving_window_matches_oracle(prec):
    # a spot fast enough to move the window about five cells in 200 steps; its start is off
    # the cell grid, so that no step puts it exactly on a column boundary (a tie that two
    # equally correct roundings may break either way)
    w = I.multiscale_track(ncx=24, ncy=5, ncz=2, cell=1e-9, ratio=2, wx=6, grain_d=5e-9, boundary=1e-9, seed=22,
                           v=2.5e5, x_spot=6.013e-9)
    p, O, G = pair(w, prec)
    with G:
        ox = orc.ms_target(p, 0.0)
        start(w, p, O, G, ox)
        for block in (70, 130):
            O.run(block, follow=True)
            G.steps(block, follow=True)
            dm, dS = compare(O, G)
            assert dm < TOL[prec] and dS < TOL[prec], (block, dm, dS)
            assert G.window()[0] == O.window
        assert O.window >= ox + 4


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_track_geometry_reduced_matches_oracle(prec):
    """1 nm cells with 0.25 nm sites (4 per cell edge, the full track's geometry), 8 nm
    grains, laser over T_C in the window, a few window moves."""
    w = I.multiscale_track(ncx=40, ncy=12, ncz=4, cell=1e-9, ratio=4, wx=10, seed=23, v=5e5, x_spot=9.013e-9)
    p, O, G = pair(w, prec)
    with G:
        start(w, p, O, G, orc.ms_target(p, 0.0))
        ox = O.window
        O.run(60, follow=True)
        G.steps(60, follow=True)
        dm, dS = compare(O, G)
        assert dm < TOL[prec] and dS < TOL[prec], (dm, dS)
        assert G.window()[0] == O.window >= ox + 2


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_full_track_two_steps_matches_oracle(prec):
    """The full multiscale track: 500 x 60 x 10 cells of 1 nm and a 60 nm window of
    240 x 240 x 40 sites (2.3 M), two coupled steps."""
    w = I.multiscale_track()
    p, O, G = pair(w, prec)
    with G:
        ox = orc.ms_target(p, 0.0)
        start(w, p, O, G, ox)
        O.run(2)
        G.steps(2)
        dm, dS = compare(O, G)
        assert dm < TOL[prec] and dS < TOL[prec], (dm, dS)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_head_profile_matches_oracle(prec):
    """The write field as tanh profiles following a moving head over a bit pattern, in both
    regions and in m_e(T), with the window following the spot."""
    w = I.multiscale_track(ncx=40, ncy=6, ncz=2, cell=1e-9, ratio=2, wx=8, grain_d=5e-9, seed=26, v=1.2e5,
                           x_spot=12.013e-9)
    w["field"].update(bit_len=4e-9, ramp_len=0.5e-9, head_x0=12.4e-9, head_v=1.2e5, B0=1.5)
    prof = dict(Bx0=0.6, wz=3e-9, dz=1e-9, wx=2e-9, dx=-1e-9)
    p, O, G = pair(w, prec, profile=prof)
    with G:
        start(w, p, O, G, orc.ms_target(p, 0.0))
        ox = O.window
        O.run(150, follow=True)
        G.steps(150, follow=True)
        dm, dS = compare(O, G)
        assert dm < TOL[prec] and dS < TOL[prec], (dm, dS)
        assert G.window()[0] == O.window >= ox + 1
        G.set_head_profile(wz=0.0)          # back to the uniform field
        with pytest.raises(HamrError) as e:
            G.set_head_profile(Bx0=0.1, wz=1e-9, wx=0.0)
        assert e.value.code == ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_demag_matches_oracle(prec):
    """The demagnetising field of Eq. 7 (FFT convolution on the GPU, direct summation in the
    oracle) in both regions, with the laser on and the window following the spot."""
    w = I.multiscale_track(ncx=24, ncy=6, ncz=3, cell=1e-9, ratio=2, wx=6, grain_d=5e-9, seed=27, v=1.5e5,
                           x_spot=9.013e-9)
    p, O, G = pair(w, prec, demag=True)
    with G:
        start(w, p, O, G, orc.ms_target(p, 0.0))
        ox = O.window
        O.run(100, follow=True)
        G.steps(100, follow=True)
        dm, dS = compare(O, G)
        assert dm < TOL[prec] and dS < TOL[prec], (dm, dS)
        assert G.window()[0] == O.window >= ox + 1
        G.set_demag(False)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("demag,margin", [(False, -1), (True, -1), (False, 4), (True, 4)])
def test_two_stream_step_is_deterministic(prec, demag, margin):
    """A step runs Eq. 6, the m_e solve and RK4 stages 0-2 on a second stream beside the
    window step: two runs of the same sequence (steps, a window move, steps) give bitwise the
    same cells and spins, so no kernel reads what the other stream has not yet written."""
    w = I.multiscale_track(ncx=30, ncy=6, ncz=3, cell=1e-9, ratio=4, wx=6, grain_d=5e-9, seed=43, v=2.5e5,
                           x_spot=8.013e-9)
    out = []
    for _ in range(2):
        p, O, G = pair(w, prec, demag=demag, margin=margin)
        with G:
            start(w, p, O, G, orc.ms_target(p, 0.0))
            G.steps(40, follow=True)
            G.steps(40, follow=True)
            out.append((G.read_cells(), G.read_moments(), G.window()))
    assert out[0][2] == out[1][2]
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("ncz", [1, 3, 10, 11])
def test_demag_field_matches_direct_sum(prec, ncz):
    """Eq. 7 alone: B_d of a given magnetisation by the GPU's convolution (in-plane FFTs on the
    padded grid, direct sum along z; 1 to 10 planes take the register-blocked sum in FP32, 11
    the general one) against the oracle's direct summation over every pair of cells, element
    by element.  Odd column and row counts give ragged transforms; a fifth of the cells carry
    no magnetisation."""
    w = I.multiscale_track(ncx=17, ncy=5, ncz=ncz, cell=1e-9, ratio=2, wx=4, grain_d=5e-9, seed=41, v=0.0,
                           x_spot=8e-9)
    p, O, G = pair(w, prec, demag=True)
    n = w["ncx"] * w["ncy"] * ncz
    rng = np.random.default_rng(400 + ncz)
    M = rng.normal(size=(n, 3))
    M *= (w["Ms0"] * rng.uniform(0.2, 1.0, size=n) / np.linalg.norm(M, axis=1))[:, None]
    M[rng.random(n) < 0.2] = 0.0
    want = orc.demag_field(p, M)
    with G:
        got = G.demag_field(M)
        scale = np.abs(want).max()
        err = np.abs(got - want).max() / scale
        assert err < (1e-11 if prec == "fp64" else 2e-6), err
        # the field changes sign with M (a linear map)
        assert np.abs(G.demag_field(-M) + got).max() <= 1e-12 * scale * (1 if prec == "fp64" else 1e5)
        G.set_demag(False)
        assert np.array_equal(G.demag_field(M), got)   # the grid stays built
    _, _, G2 = pair(w, prec)
    with G2:
        with pytest.raises(HamrError) as e:
            G2.demag_field(M)
        assert e.value.code == ERR_STATE


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_read_track_matches_oracle(prec):
    """Read-back of the track: a written pattern of +z / -z bit regions reads back exactly; after
    a coupled run the per-bit signals match the oracle's."""
    w = I.multiscale_track(ncx=60, ncy=8, ncz=2, cell=1e-9, ratio=2, wx=8, grain_d=5e-9, seed=25, v=0.0,
                           x_spot=30.2e-9)
    p, O, G = pair(w, prec)
    L, pattern = 6e-9, [0, 1, 1, 0, 1, 0, 0, 1, 1, 0]
    n = w["ncx"] * w["ncy"] * w["ncz"]
    m = np.zeros((w["ncz"], w["ncy"], w["ncx"], 3))
    for b, v in enumerate(pattern):
        m[:, :, b * 6:(b + 1) * 6, 2] = -1.0 if v else 1.0
    m = I.mask_void(m.reshape(n, 3), w["grain"])
    with G:
        G.set_cells(m)
        O.set_cells(m)
        sig, bits = G.read_track(0.0, L, len(pattern), 1, 7)
        osig, obits = O.read_track(0.0, L, len(pattern), 1, 7)
        assert list(bits) == pattern == list(obits)
        assert np.abs(sig - osig).max() < 1e-12
        # after a coupled run with the window over the track
        m2 = tilted_cells(w)
        G.set_cells(m2)
        O.set_cells(m2)
        G.set_window(11)
        O.set_window(11)
        G.steps(50)
        O.run(50)
        sig, bits = G.read_track(0.0, L, len(pattern), 0, 8)
        osig, obits = O.read_track(0.0, L, len(pattern), 0, 8)
        assert np.abs(sig - osig).max() < TOL[prec], np.abs(sig - osig).max()


@pytest.mark.gpu
def test_call_order_and_arguments():
    w = I.multiscale_track(ncx=12, ncy=3, ncz=2, cell=1e-9, ratio=2, wx=4, grain_d=3e-9, seed=24)
    with Multiscale(12, 3, 2, 1e-9, 2, 4, J=w["J"], mu_s=w["mu_s"], ku=w["ku"], Ms0=w["Ms0"], A0=w["A0"],
                    K0=w["K0"], lam=0.1, T_C=w["T_C"]) as G:
        with pytest.raises(HamrError) as e:
            G.steps(1)
        assert e.value.code == ERR_STATE
        with pytest.raises(HamrError) as e:
            G.set_window(0)
        assert e.value.code == ERR_STATE
        G.set_cells(tilted_cells(w))
        with pytest.raises(HamrError) as e:
            G.set_window(9)
        assert e.value.code == ERR_ARG
        G.set_window(8)
        G.steps(0)
        assert G.window() == (8, 0)
        bad = np.zeros(12 * 3 * 2, np.int32)
        bad[3] = -2
        with pytest.raises(HamrError) as e:
            G.set_grain_map(bad)
        assert e.value.code == ERR_ARG
        for args in ((0.0, 0.0, 3), (0.0, 1e-9, 3, 2, 2), (0.0, 1e-9, 3, 0, 4)):
            with pytest.raises(HamrError) as e:
                G.read_track(*args)
            assert e.value.code == ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_head_profile_switched_off_mid_run(prec):
    """After the head profile is switched off, every column's m_e(T) is solved again with the
    uniform field: no column keeps an m_e from its profile field, including those far from the
    spot whose temperature has not changed (steps after the switch against the oracle)."""
    w = I.multiscale_track(ncx=40, ncy=6, ncz=2, cell=1e-9, ratio=2, wx=8, grain_d=5e-9, seed=28, v=1.2e5,
                           x_spot=12.013e-9)
    w["field"].update(bit_len=4e-9, ramp_len=0.5e-9, head_x0=12.4e-9, head_v=1.2e5, B0=1.5)
    prof = dict(Bx0=0.6, wz=3e-9, dz=1e-9, wx=2e-9, dx=-1e-9)
    p, O, G = pair(w, prec, profile=prof)
    with G:
        start(w, p, O, G, orc.ms_target(p, 0.0))
        O.run(60, follow=True)
        G.steps(60, follow=True)
        G.set_head_profile(wz=0.0)
        O.set_drivers(params(w))
        O.run(80, follow=True)
        G.steps(80, follow=True)
        dm, dS = compare(O, G)
        assert dm < TOL[prec] and dS < TOL[prec], (dm, dS)
        assert G.window()[0] == O.window


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_zero_field_columns_cool_through_tc(prec):
    """No write field: the passing spot heats columns above T_C (m_e = 0) and they cool below it
    again, where m_e(T) must return to the largest root of the mean-field equation, not stay at
    the unstable root 0 its last solve started from (against the oracle's bisection)."""
    w = I.multiscale_track(ncx=30, ncy=4, ncz=2, cell=1e-9, ratio=2, wx=6, grain_d=5e-9, seed=29, v=4e5,
                           x_spot=7.013e-9)
    w["T"].update(T_peak=1500.0, fwhm=6e-9)
    w["field"].update(B0=0.0)
    p, O, G = pair(w, prec)
    with G:
        start(w, p, O, G, orc.ms_target(p, 0.0))
        ox = O.window
        for block in (150, 150):
            O.run(block, follow=True)
            G.steps(block, follow=True)
            dm, dS = compare(O, G)
            assert dm < TOL[prec] and dS < TOL[prec], (block, dm, dS)
        assert O.window >= ox + 8


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
def test_parallel_track_second_pass_matches_oracle(prec):
    """Two tracks written side by side (Sec. III): a first pass with the spot and the head over
    one row band, then a second pass with the spot centre moved across the track by 15 nm
    scaled to this mesh (new temperature profile, spot and head restarted at the current time,
    the window placed back at the new spot, handing the old one back by Eq. 6).  Cells and
    window spins against the oracle after each pass, and both bands read back the same."""
    dt, v = 1e-16, 2e5
    w = I.multiscale_track(ncx=40, ncy=16, ncz=2, cell=1e-9, ratio=2, wx=8, grain_d=5e-9, seed=30, v=v,
                           x_spot=8.013e-9)
    w["T"].update(y0=4.5e-9, fwhm=6e-9, T_peak=1100.0)
    w["field"].update(bit_len=4e-9, ramp_len=0.5e-9, head_x0=8.4e-9, head_v=v, B0=2.0)
    p, O, G = pair(w, prec)
    n1 = 120
    with G:
        start(w, p, O, G, orc.ms_target(p, 0.0))
        O.run(n1, follow=True)
        G.steps(n1, follow=True)
        dm, dS = compare(O, G)
        assert dm < TOL[prec] and dS < TOL[prec], ("first pass", dm, dS)
        t1 = n1 * dt
        T2 = dict(w["T"], x0=w["T"]["x0"] - v * t1, y0=11.5e-9)
        F2 = dict(w["field"], head_x0=w["field"]["head_x0"] - v * t1, bits=I.bits_of("1011001"))
        G.set_temperature_profile(**T2)
        G.set_field_sequence(**F2)
        p2 = params(w, T2, F2)
        O.set_drivers(p2)
        ox2 = orc.ms_target(p2, t1)
        assert ox2 < O.window
        O.set_window(ox2)
        G.set_window(ox2)
        dm, dS = compare(O, G)
        assert dm < TOL[prec] and dS < TOL[prec], ("re-placed", dm, dS)
        O.run(n1, follow=True)
        G.steps(n1, follow=True)
        dm, dS = compare(O, G)
        assert dm < TOL[prec] and dS < TOL[prec], ("second pass", dm, dS)
        assert G.window()[0] == O.window
        for band in ((0, 8), (8, 16)):
            sig, bits = G.read_track(0.0, 4e-9, 9, *band)
            osig, obits = O.read_track(0.0, 4e-9, 9, *band)
            assert np.abs(sig - osig).max() < TOL[prec]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("demag", [False, True])
def test_simulated_region_matches_oracle(prec, demag):
    """The simulated region (Sec. II, Fig. 1): only the window and three cell columns on each
    side evolve, the rest of the track is frozen (m and the m_e of its last evolved step, which
    enter Eq. 7); the region moves with the window through several moves."""
    w = I.multiscale_track(ncx=36, ncy=5, ncz=2, cell=1e-9, ratio=2, wx=6, grain_d=5e-9, seed=31, v=2.5e5,
                           x_spot=8.013e-9)
    p, O, G = pair(w, prec, demag=demag, margin=3)
    with G:
        start(w, p, O, G, orc.ms_target(p, 0.0))
        ox = O.window
        m0 = O.cells().copy()
        for block in (90, 110):
            O.run(block, follow=True)
            G.steps(block, follow=True)
            dm, dS = compare(O, G)
            assert dm < TOL[prec] and dS < TOL[prec], (block, dm, dS)
            assert G.window()[0] == O.window
        assert O.window >= ox + 4
        ahead = np.arange(36) >= O.window + 6 + 3
        cells = G.read_cells().reshape(2, 5, 36, 3)[:, :, ahead]
        want = m0.reshape(2, 5, 36, 3)[:, :, ahead]
        assert np.abs(cells - want).max() < (1e-15 if prec == "fp64" else 1e-7)   # frozen cells stay put
