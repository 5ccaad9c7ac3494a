"""Pins of the multiscale-window oracle (oracle/hamr_ms_oracle.c) to what the paper and the
mathematics fix: limits of the equilibrium magnetisation m_e(T), the printed values of the
thermalisation cone law, the cone's polar-angle distribution, Eq. 6 by brute force, the
micromagnetic LLG in closed form for an isolated cell, and the equivalence of the
micromagnetic and atomistic equations of motion when a cell holds one site (Eq. 9).
Sections and equations refer to arXiv 2502.02236.
"""
import math

import numpy as np

import oracle as o

A = 0.25e-9
MU_S = 3 * o.C_MU_B
J_SC = 6.7e-21
KU = 1.0e-22
G = o.C_GAMMA
KB = o.C_KB


# ----------------------------------------------------------------------------- m_e(T)
def check_langevin_branches():
    """L(x) = coth x - 1/x: the small-x series and the closed form agree where they meet,
    L is odd, and L(x) -> 1 - 1/x for large x."""
    for x in (9.99e-4, 1.001e-3):
        assert abs(o.langevin(x) - (1 / math.tanh(x) - 1 / x)) < 1e-12
        assert abs(o.langevin(x) - x / 3) < x ** 3 / 40
    assert o.langevin(-0.7) == -o.langevin(0.7)
    assert abs(o.langevin(50.0) - (1 - 1 / 50.0)) < 1e-15


def check_me_limits():
    """m_e(T) (Sec. II): 1 at T -> 0 with the low-temperature slope 1 - T/3T_C; 0 above T_C
    without a field; the mean-field critical law m_e^2 = (5/3)(T_C/T - 1)(T/T_C)^3 just
    below T_C; the Curie-Weiss response (mu_s B / 3 kB T) / (1 - T_C/T) well above T_C."""
    Tc = 700.0
    assert o.me(Tc, 0.0, MU_S, 0.0) == 1.0
    for T in (1.0, 5.0):
        assert abs(o.me(Tc, T, MU_S, 0.0) - (1 - T / (3 * Tc))) < 2 * (T / Tc) ** 2
    # at T_C the residual is cubic in m, so bisection stops near 1e-8
    assert o.me(Tc, Tc, MU_S, 0.0) < 1e-6
    for T in (1.2 * Tc, 3 * Tc):
        assert o.me(Tc, T, MU_S, 0.0) < 1e-12
    T = 0.999 * Tc
    want = math.sqrt(5.0 / 3.0 * (Tc / T - 1) * (T / Tc) ** 3)
    assert abs(o.me(Tc, T, MU_S, 0.0) / want - 1) < 5e-3
    T, B = 4 * Tc, 1.0
    cw = (MU_S * B / (3 * KB * T)) / (1 - Tc / T)
    assert abs(o.me(Tc, T, MU_S, B) / cw - 1) < 1e-3
    # a field raises m_e; heating lowers it
    assert o.me(Tc, 500.0, MU_S, 2.0) > o.me(Tc, 500.0, MU_S, 0.0) > o.me(Tc, 600.0, MU_S, 0.0)


def check_micromagnetic_damping_law():
    """alpha(T) = lambda (1 - T / 3 T_C) below T_C (Sec. II): lambda at 0 K, 2 lambda / 3 at T_C."""
    p = o.MsParams(4, 1, 1, A, 1, 1, J=J_SC, lam=0.1)
    assert o.ms_alpha(p, 0.0) == 0.1
    assert abs(o.ms_alpha(p, p.T_C) - 0.2 / 3) < 1e-15
    assert abs(o.ms_alpha(p, 0.5 * p.T_C) - 0.1 * (1 - 1 / 6)) < 1e-15


# ----------------------------------------------------------------------------- thermalisation
def check_theta_max_printed_values():
    """theta_max = (5 pi / 9) sqrt(1 - sqrt(1 + 6 (M/Ms0 - 1)/5)) (Sec. II): 0 for a fully
    ordered cell, 5 pi / 9 at M/Ms0 = 1/6 where the inner root vanishes, and decreasing in
    between; below 1/6 the root's argument is held at 0."""
    assert o.theta_max(1.0) == 0.0
    assert abs(o.theta_max(1 / 6) - 5 * math.pi / 9) < 1e-15
    assert o.theta_max(0.05) == o.theta_max(1 / 6)
    xs = np.linspace(1 / 6, 1, 50)
    th = [o.theta_max(x) for x in xs]
    assert all(a > b for a, b in zip(th, th[1:]))
    assert abs(o.theta_max(0.5) - 5 * math.pi / 9 * math.sqrt(1 - math.sqrt(0.4))) < 1e-15


def check_cone_distribution():
    """Thermalised spins are unit vectors within theta_max of the cell direction, with the
    polar angle uniform in [0, theta_max] (its mean is theta_max / 2 and the mean spin is
    e3 sin(theta_max)/theta_max, the azimuth averaging the transverse part away)."""
    from scipy import stats
    rng = np.random.default_rng(5)
    for e3 in (np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.0, -1.0]), rng.normal(size=3)):
        e3 = e3 / np.linalg.norm(e3)
        thm = 1.1
        S = np.array([o.cone_sample(e3, thm, 9, s, 2) for s in range(6000)])
        assert np.all(np.abs(np.linalg.norm(S, axis=1) - 1) < 1e-14)
        th = np.arccos(np.clip(S @ e3, -1, 1))
        assert th.max() <= thm + 1e-12
        assert stats.kstest(th / thm, "uniform").pvalue > 1e-4
        mean = S.mean(axis=0)
        assert np.linalg.norm(mean - e3 * math.sin(thm) / thm) < 0.03
    # theta_max = 0 returns the cell direction itself
    e3 = np.array([0.6, 0.0, 0.8])
    assert np.allclose(o.cone_sample(e3, 0.0, 1, 2, 3), e3, atol=1e-15)


# ----------------------------------------------------------------------------- coupled window
def _uniform_cells(p, v=(0.0, 0.0, 1.0)):
    m = np.zeros((p.n_cells, 3))
    m[:] = v
    return m


def check_eq6_average_brute_force():
    """Eq. 6: after a zero-step run every window cell holds the direction of the sum of the
    spins inside it (brute force over the cell's sites); cells outside keep their m."""
    p = o.MsParams(9, 3, 2, 2 * A, 2, 4, J=J_SC, ku=KU, seed=4)
    grain = np.zeros(p.n_cells, np.int32)
    grain[5] = -1
    O = o.MsOracle(p, grain)
    m0 = _uniform_cells(p, (0.0, 0.6, 0.8))
    O.set_cells(m0)
    O.set_window(3)
    rng = np.random.default_rng(2)
    S = rng.normal(size=(O.nw, 3))
    S /= np.linalg.norm(S, axis=1)[:, None]
    nxw, nyw, nzw = p.window_dims
    r = p.ratio
    for k in range(nzw):
        for j in range(nyw):
            for i in range(nxw):
                q = (3 + i // r) + p.ncx * (j // r + p.ncy * (k // r))
                if grain[q] < 0:
                    S[i + nxw * (j + nyw * k)] = 0.0
    O.set_moments(S)
    O.run(0)
    m = O.cells()
    for q in range(p.n_cells):
        cx, cy, cz = q % p.ncx, (q // p.ncx) % p.ncy, q // (p.ncx * p.ncy)
        if not 3 <= cx < 7:
            want = m0[q] if grain[q] >= 0 else np.zeros(3)
        elif grain[q] < 0:
            want = np.zeros(3)
        else:
            s = np.zeros(3)
            for dk in range(r):
                for dj in range(r):
                    for di in range(r):
                        i, j, k = (cx - 3) * r + di, cy * r + dj, cz * r + dk
                        s += S[i + nxw * (j + nyw * k)]
            want = s / np.linalg.norm(s)
        assert np.allclose(m[q], want, atol=1e-14), q


def check_uniform_state_stationary_through_shifts():
    """A uniform state along the field at T = 0 feels no torque on either side of the
    interface, and a window moving with the spot thermalises with theta_max = 0 (m_e = 1):
    every spin and every cell stays exactly along z through several shifts."""
    p = o.MsParams(14, 2, 2, 2 * A, 2, 4, J=J_SC, ku=KU, dt=1e-16, seed=3, B0=0.5,
                   direction=(0, 0, 1), fwhm=0.0, x0=6 * 2 * A, vx=2 * A / (10 * 1e-16))
    O = o.MsOracle(p)
    O.set_cells(_uniform_cells(p))
    O.set_window(o.ms_target(p, 0.0))
    w0 = O.window
    O.run(45, follow=True)
    assert w0 == 4 and O.window == o.ms_target(p, 45 * 1e-16) == 9
    S = O.moments()
    assert np.array_equal(S, np.tile([0.0, 0.0, 1.0], (O.nw, 1)))
    assert np.array_equal(O.cells(), _uniform_cells(p))


def check_isolated_cell_llg():
    """One micromagnetic cell with no magnetic neighbour, uniform T, field B along z
    (Eq. 1 without thermal field, Eq. 5 with K(T)/Ms(T) = K0 m_e^2 / Ms0, Sec. II):
    without damping it precesses at gamma (B + (2 K0 m_e^2 / Ms0) cos theta) at constant
    theta; with damping and no anisotropy, tan(theta/2) decays as
    exp(-alpha gamma B t / (1 + alpha^2)) with alpha = lambda (1 - T / 3 T_C)."""
    B0, T, dt, n = 1.0, 350.0, 2e-15, 400
    for lam, ku in ((0.0, KU), (0.1, 0.0)):
        p = o.MsParams(6, 1, 1, A, 1, 1, J=J_SC, ku=ku, lam=lam, dt=dt, T_amb=T, B0=B0, direction=(0, 0, 1))
        grain = np.array([-1, -1, -1, -1, 0, -1], np.int32)
        O = o.MsOracle(p, grain)
        th0 = 0.4
        m = np.zeros((6, 3))
        m[4] = (math.sin(th0), 0.0, math.cos(th0))
        O.set_cells(m)
        O.set_window(0)
        O.run(n)
        got = O.cells()[4]
        t = n * dt
        me = o.me(p.T_C, T, MU_S, B0)
        if lam == 0.0:
            w = G * (B0 + 2 * p.K0 * me ** 2 / p.Ms0 * math.cos(th0))
            want = np.array([math.sin(th0) * math.cos(w * t), math.sin(th0) * math.sin(w * t), math.cos(th0)])
        else:
            al = lam * (1 - T / (3 * p.T_C))
            th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-al * G * B0 * t / (1 + al * al)))
            ph = G * B0 * t / (1 + al * al)
            want = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        assert np.linalg.norm(got - want) < 1e-8, (lam, got, want)


def check_mm_standing_spin_wave():
    """Micromagnetic exchange at temperature (Eq. 4 with A(T)/Ms(T) = A0 m_e / Ms0, Eq. 5
    with K(T)/Ms(T) = K0 m_e^2 / Ms0): on an open chain of N cells, the small standing wave
    m_x + i m_y = eps cos(pi n (i + 1/2) / N) precesses without damping at
    gamma [B + 2 K0 m_e^2 / Ms0 + (2 A0 m_e / Ms0) (2 - 2 cos(pi n / N)) / c^2], the
    eigenvalue of the 6-point Laplacian with missing neighbours left out."""
    N, c, T, B0, eps = 16, 1e-9, 400.0, 0.5, 1e-4
    p = o.MsParams(N + 1, 1, 1, c, 4, 1, J=J_SC, ku=KU, lam=0.0, dt=1e-16, T_amb=T, B0=B0,
                   direction=(0, 0, 1), A0=J_SC / (2 * A), Ms0=MU_S / A ** 3, K0=KU / A ** 3)
    grain = np.zeros(N + 1, np.int32)
    grain[0] = -1                       # the window's cell: no atomistic sites
    me = o.me(p.T_C, T, MU_S, B0)
    for n in (1, 3):
        O = o.MsOracle(p, grain)
        i = np.arange(N)
        amp = eps * np.cos(np.pi * n * (i + 0.5) / N)
        m = np.zeros((N + 1, 3))
        m[1:, 0] = amp
        m[1:, 2] = np.sqrt(1 - amp ** 2)
        O.set_cells(m)
        O.set_window(0)
        steps = 300
        O.run(steps)
        got = O.cells()[1:]
        w = G * (B0 + 2 * p.K0 * me ** 2 / p.Ms0 + 2 * p.A0 * me / p.Ms0 * (2 - 2 * math.cos(math.pi * n / N)) / c ** 2)
        ph = np.arctan2(got[:, 1], got[:, 0])
        k = int(np.argmax(amp))
        want = w * steps * p.drv.dt
        assert abs((ph[k] - want + math.pi) % (2 * math.pi) - math.pi) < 1e-4 * want, (n, ph[k], want)


def _tilted(n, seed, deg):
    rng = np.random.default_rng(seed)
    th = np.deg2rad(deg) * rng.random(n)
    ph = 2 * np.pi * rng.random(n)
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)


def _coupled_vs_atomistic(dt, n_steps):
    """Largest spin difference between the multiscale run with one site per cell and the
    atomistic oracle on the whole lattice, from the same tilted state, at T = 0."""
    ncx, ncy, ncz, wx, ox = 12, 5, 3, 4, 4
    grain = np.zeros(ncx * ncy * ncz, np.int32)
    grain.reshape(ncz, ncy, ncx)[:, :, 9] = -1      # a void column: an interface of its own
    grain.reshape(ncz, ncy, ncx)[:, :, 10:] = 1     # and a second grain behind it
    kw = dict(ku=KU, dt=dt, B0=0.7, direction=(0.3, 0.0, -1.0), T_amb=0.0, seed=5)
    p = o.MsParams(ncx, ncy, ncz, A, 1, wx, J=J_SC, lam=0.1, **kw)
    S0 = _tilted(p.n_cells, 1, 40.0)
    S0[grain < 0] = 0.0
    O = o.MsOracle(p, grain)
    O.set_cells(S0)
    O.set_window(ox)
    win = S0.reshape(ncz, ncy, ncx, 3)[:, :, ox:ox + wx].reshape(-1, 3)
    O.set_moments(np.ascontiguousarray(win))
    O.run(n_steps)
    ms = O.cells()
    pa = o.sc_params(ncx, ncy, ncz, A, J_SC, mu_s=MU_S, alpha=0.1, **kw)
    Oa = o.Oracle(pa, grain)
    S = np.ascontiguousarray(S0.copy())
    Oa.run(S, 0, n_steps)
    return np.abs(ms - S).max()


def check_ratio_one_window_matches_atomistic_lattice():
    """With one site per cell (cell edge = a), Ms0 = mu_s / a^3, K0 = ku / a^3 (Appendix A)
    and A0 = J / 2a (Eq. 9), at T = 0 (m_e = 1, alpha = lambda), the micromagnetic field
    (2A0/Ms0) lap(m) + (2K0/Ms0) m_z z differs from the atomistic one of Eq. 2-3 only by a
    term along m, so the coupled window and the plain atomistic lattice solve the same
    equations.  They differ only in how they are integrated: RK4 outside, Heun inside, and
    each region stepped with the other's interface values frozen at t_n, a splitting of
    first order in dt.  So the difference must shrink in proportion to dt; a wrong interface
    bond on either side leaves a difference that does not shrink."""
    T_end = 2e-14
    e = [_coupled_vs_atomistic(dt, int(round(T_end / dt))) for dt in (2e-16, 1e-16, 5e-17)]
    assert e[2] < 2.5e-3, e
    assert 1.8 < e[0] / e[1] < 2.2 and 1.8 < e[1] / e[2] < 2.2, e


def check_full_window_equals_atomistic_oracle():
    """A window covering the whole track with one site per cell leaves no micromagnetic
    cell to evolve; its sites then follow the atomistic oracle exactly (same Philox stream:
    the track site index equals the lattice site index), with thermal noise, laser spot and
    granular decoupling on."""
    ncx, ncy, ncz = 7, 5, 3
    grain = np.zeros(ncx * ncy * ncz, np.int32)
    grain.reshape(ncz, ncy, ncx)[:, 2, :] = -1
    grain.reshape(ncz, ncy, ncx)[:, 3:, :] = 1
    kw = dict(ku=KU, dt=1e-16, B0=0.8, direction=(0.0, 0.0, -1.0), T_amb=300.0, T_peak=800.0,
              fwhm=1e-9, x0=0.8e-9, y0=0.5e-9, vx=1e4, seed=11)
    p = o.MsParams(ncx, ncy, ncz, A, 1, ncx, J=J_SC, lam=0.1, **kw)
    S0 = _tilted(p.n_cells, 4, 30.0)
    S0[grain < 0] = 0.0
    O = o.MsOracle(p, grain)
    O.set_cells(S0)
    O.set_window(0)
    O.set_moments(S0)
    O.run(60)
    pa = o.sc_params(ncx, ncy, ncz, A, J_SC, mu_s=MU_S, alpha=0.1, **kw)
    S = np.ascontiguousarray(S0.copy())
    o.Oracle(pa, grain).run(S, 0, 60)
    assert np.abs(O.moments() - S).max() < 1e-13


def check_shift_moves_spins():
    """One window move (Fig. 1): the sites shift back by one cell column, the trailing
    column is handed to the micromagnetic side by Eq. 6 and the new leading column is
    thermalised from its cells (at T = 0, theta_max = 0: the cell direction itself).  The
    step before it is made negligibly short."""
    ncx, ncy, ncz, r, wx = 10, 2, 1, 2, 4
    p = o.MsParams(ncx, ncy, ncz, 2 * A, r, wx, J=J_SC, ku=KU, dt=1e-28, T_amb=0.0,
                   x0=5 * 2 * A, vx=0.6 * 2 * A / 1e-28, seed=2)
    O = o.MsOracle(p)
    m0 = _tilted(p.n_cells, 6, 60.0)
    O.set_cells(m0)
    O.set_window(3)
    S0 = _tilted(O.nw, 7, 60.0)
    O.set_moments(S0)
    O.run(1, follow=True)
    assert O.window == 4
    nxw, nyw, nzw = p.window_dims
    S = O.moments().reshape(nzw, nyw, nxw, 3)
    S0 = S0.reshape(nzw, nyw, nxw, 3)
    assert np.abs(S[:, :, :nxw - r] - S0[:, :, r:]).max() < 1e-9
    m = O.cells().reshape(ncz, ncy, ncx, 3)
    m0 = m0.reshape(ncz, ncy, ncx, 3)
    for cy in range(ncy):
        lead = m0[0, cy, 7]
        assert np.abs(S[:, cy * r:(cy + 1) * r, nxw - r:] - lead).max() < 1e-12
        s = S0[:, cy * r:(cy + 1) * r, :r].reshape(-1, 3).sum(axis=0)
        assert np.abs(m[0, cy, 3] - s / np.linalg.norm(s)).max() < 1e-9


def check_read_track():
    """Read-back: cells set to +z / -z by bit regions read back as the written pattern with
    signals of exactly +1 / -1; non-magnetic cells and rows outside the band do not count;
    a bit window with no magnetic cell reads 0."""
    ncx, ncy, ncz, L = 40, 6, 2, 5
    p = o.MsParams(ncx, ncy, ncz, 1e-9, 1, 4, J=J_SC)
    grain = np.zeros(ncx * ncy * ncz, np.int32)
    g3 = grain.reshape(ncz, ncy, ncx)
    g3[:, :, 17] = -1
    g3[:, :, 30:35] = -1                          # bit 6 has no magnetic cell
    pattern = [0, 1, 1, 0, 1, 0, 0, 1]
    m = np.zeros((ncz, ncy, ncx, 3))
    for b, v in enumerate(pattern):
        m[:, :, b * L:(b + 1) * L, 2] = -1.0 if v else 1.0
    m[:, 0, :, 2] = 1.0                           # a row outside the band, along +z everywhere
    m[:, :, 17, 2] = -1.0                         # a non-magnetic cell (set to 0 by set_cells)
    O = o.MsOracle(p, grain)
    O.set_cells(m.reshape(-1, 3))
    sig, bits = O.read_track(0.0, L * 1e-9, len(pattern), cy0=1, cy1=ncy)
    want = np.array([-1.0 if v else 1.0 for v in pattern])
    want[6] = 0.0
    assert np.array_equal(sig, want), sig
    assert list(bits) == [v if b != 6 else 0 for b, v in enumerate(pattern)]
    # the band including row 0 averages it in: bit 1 reads -1 over 5 rows and +1 over 1
    sig2, _ = O.read_track(0.0, L * 1e-9, 2, cy0=0, cy1=ncy)
    assert abs(sig2[1] - (-5 + 1) / 6) < 1e-15


PROFILE = dict(wz=3e-9, dz=2e-9, Bx0=0.3, wx=2e-9, dx=-1e-9)


def check_head_profile_shape():
    """Write field with the head profile (a reading of the tanh profiles of Sec. III, Fig. 2):
    the full field B0 s(t) dir and Bx0 s(t) x far upstream of the head, half of each at its
    offset from the head, none far downstream; the polarity s(t) of the bit pattern flips both
    components; without the profile the field is uniform."""
    kw = dict(J=J_SC, B0=0.8, direction=(0, 0, -1), head_x0=10e-9, head_v=1e3, bits=[0, 1], bit_len=15e-9,
              ramp_len=1e-12)
    p = o.MsParams(30, 1, 1, 1e-9, 1, 2, profile=PROFILE, **kw)
    xh = 10e-9
    B = o.ms_field(p, xh - 1e-6, 0.0)
    assert np.allclose(B, [0.3, 0.0, -0.8], atol=1e-12)
    assert abs(o.ms_field(p, xh + 2e-9, 0.0)[2] + 0.4) < 1e-15
    assert abs(o.ms_field(p, xh - 1e-9, 0.0)[0] - 0.15) < 1e-15
    assert np.allclose(o.ms_field(p, xh + 1e-6, 0.0), 0.0, atol=1e-15)
    # the head has moved into bit 1 (polarity -1) at t = 10 ns
    t = 10e-9
    assert o.field_polarity(p.drv, t) == -1.0
    assert np.allclose(o.ms_field(p, xh + 1e3 * t - 1e-6, t), [-0.3, 0.0, 0.8], atol=1e-12)
    pu = o.MsParams(30, 1, 1, 1e-9, 1, 2, **kw)
    for x in (0.0, 12e-9, 1e-6):
        assert np.array_equal(o.ms_field(pu, x, 0.0), o.applied_field(pu.drv, 0.0))


def _rotate(v, axis, ang):
    k = axis / np.linalg.norm(axis)
    return v * math.cos(ang) + np.cross(k, v) * math.sin(ang) + k * (k @ v) * (1 - math.cos(ang))


def check_isolated_cell_and_site_in_head_profile():
    """An isolated micromagnetic cell and an isolated window site (no magnetic neighbour, no
    anisotropy, no damping, T = 0) precess about the local profile field B(x) at gamma |B(x)|:
    both sides of the window evaluate the field where they sit."""
    dt, n = 2e-16, 500
    p = o.MsParams(12, 1, 1, A, 1, 2, J=J_SC, ku=0.0, lam=0.0, dt=dt, T_amb=0.0, B0=1.0, direction=(0, 0, 1),
                   head_x0=6 * A, head_v=0.0, profile=dict(wz=2 * A, dz=0.0, Bx0=0.6, wx=3 * A, dx=A))
    grain = np.full(12, -1, np.int32)
    grain[3] = 0          # a cell outside the window
    grain[8] = 1          # the window's one site (window at columns 8, 9)
    O = o.MsOracle(p, grain)
    m0 = np.zeros((12, 3))
    m0[3] = m0[8] = (math.sin(0.5), 0.0, math.cos(0.5))
    O.set_cells(m0)
    O.set_window(8)
    O.set_moments(np.array([[math.sin(0.5), 0.0, math.cos(0.5)], [0.0, 0.0, 0.0]]))
    O.run(n)
    t = n * dt
    for x, got in (((3 + 0.5) * A, O.cells()[3]), ((8 + 0.5) * A, O.moments()[0])):
        B = o.ms_field(p, x, 0.0)
        want = _rotate(np.array([math.sin(0.5), 0.0, math.cos(0.5)]), B, G * np.linalg.norm(B) * t)
        assert np.linalg.norm(got - want) < 1e-8, (x, got, want)


MU0 = 1.25663706212e-6


def check_demag_tensor_limits():
    """Demagnetising tensor of cuboid cells (Eq. 7, Newell et al. 1993): the self-term of a
    cube is 1/3 on each axis with no off-diagonal part; every self-term has trace 1; a flat
    cell tends to N_zz = 1 and a needle to N_zz = 0, N_xx = 1/2; the tensor is even in the
    offset, N_xy odd in X; far away it is the point-dipole tensor -(V/4 pi r^3)(3 rr/r^2 - I)."""
    a = 1e-9
    N = o.demag_tensor(0, 0, 0, a, a, a)
    assert np.allclose(N[:3], 1 / 3, atol=1e-14) and np.allclose(N[3:], 0, atol=1e-14)
    for d in ((a, 2 * a, 0.5 * a), (3 * a, a, a), (a, a, 7 * a)):
        assert abs(o.demag_tensor(0, 0, 0, *d)[:3].sum() - 1) < 1e-12
    assert o.demag_tensor(0, 0, 0, 30 * a, 30 * a, 0.1 * a)[2] > 0.98
    nd = o.demag_tensor(0, 0, 0, 0.05 * a, 0.05 * a, 20 * a)
    assert nd[2] < 0.01 and abs(nd[0] - 0.5) < 0.01
    r = np.array([2.3, -1.1, 0.7]) * a
    assert np.allclose(o.demag_tensor(*r, a, a, a), o.demag_tensor(*(-r), a, a, a), rtol=1e-12, atol=0)
    Nm = o.demag_tensor(-r[0], r[1], r[2], a, a, a)
    assert abs(Nm[3] + o.demag_tensor(*r, a, a, a)[3]) < 1e-14
    for k in (12.0, 30.0, 60.0):
        X, Y, Z = k * a * 0.48, k * a * 0.6, k * a * 0.64
        R = math.sqrt(X * X + Y * Y + Z * Z)
        pre = -a ** 3 / (4 * math.pi * R ** 3)
        want = [pre * (3 * X * X / R ** 2 - 1), pre * (3 * Y * Y / R ** 2 - 1), pre * (3 * Z * Z / R ** 2 - 1),
                pre * 3 * X * Y / R ** 2, pre * 3 * X * Z / R ** 2, pre * 3 * Y * Z / R ** 2]
        assert np.allclose(o.demag_tensor(X, Y, Z, a, a, a), want, rtol=2e-3 if k == 12.0 else 3e-4, atol=0)
    # on either side of the cutoff of 40 cell edges the tensor is the dipole tensor at that point
    for X, rtol in ((39.99 * a, 1e-4), (40.01 * a, 1e-12)):
        want = -a ** 3 / (4 * math.pi * X ** 3) * np.array([2.0, -1.0, -1.0])
        assert np.allclose(o.demag_tensor(X, 0, 0, a, a, a)[:3], want, rtol=rtol, atol=0)


def check_demag_uniform_film():
    """A uniformly magnetised film of 40 x 40 x 1 cells: at its centre the field is close to
    -mu0 M for M normal to the film and close to 0 for M in its plane (the thin-film limits of
    Eq. 7)."""
    p = o.MsParams(40, 40, 1, 1e-9, 1, 1, J=J_SC)
    Ms = 1e6
    for Mdir, want in (((0, 0, 1), (0, 0, -MU0 * Ms)), ((1, 0, 0), (0, 0, 0))):
        M = np.tile(np.array(Mdir, float) * Ms, (p.n_cells, 1))
        Bd = o.demag_field(p, M)
        c = 20 + 40 * 20
        assert np.linalg.norm(Bd[c] - want) < 0.06 * MU0 * Ms, (Mdir, Bd[c])


def check_demag_in_coupled_step():
    """With the demagnetising field on and every other field off (J = 0, no anisotropy, no
    applied field, T = 0, no damping), one short step turns each cell and window site by
    -gamma m x B_d dt, with B_d = -mu0 N * M from the magnetisation assembled here: window cells
    M = (mu_s / V) sum of their spins (Eq. 6), the other cells Ms0 m (m_e = 1 at T = 0)."""
    dt = 1e-19
    p = o.MsParams(6, 3, 2, 1e-9, 2, 2, J=0.0, ku=0.0, lam=0.0, dt=dt, T_amb=0.0, B0=0.0, seed=3, demag=True,
                   Ms0=1.2e6, T_C=700.0)
    grain = np.zeros(p.n_cells, np.int32)
    grain[5] = -1
    O = o.MsOracle(p, grain)
    m0 = _tilted(p.n_cells, 8, 70.0)
    m0[grain < 0] = 0.0
    O.set_cells(m0)
    O.set_window(2)
    S0 = _tilted(O.nw, 9, 70.0)
    nxw, nyw, nzw = p.window_dims
    cell_of = lambda i, j, k: (2 + i // 2) + 6 * (j // 2 + 3 * (k // 2))
    for k in range(nzw):
        for j in range(nyw):
            for i in range(nxw):
                if grain[cell_of(i, j, k)] < 0:
                    S0[i + nxw * (j + nyw * k)] = 0.0
    O.set_moments(S0)
    M = p.Ms0 * m0.copy()
    V = 1e-27
    for q in range(p.n_cells):
        if 2 <= q % 6 < 4:
            M[q] = 0.0
    for k in range(nzw):
        for j in range(nyw):
            for i in range(nxw):
                M[cell_of(i, j, k)] += p.mu_s / V * S0[i + nxw * (j + nyw * k)]
    Bd = o.demag_field(p, M)
    O.run(1)
    dm = O.cells() - m0
    for q in range(p.n_cells):
        if grain[q] < 0 or 2 <= q % 6 < 4:
            continue
        want = -G * np.cross(m0[q], Bd[q]) * dt
        assert np.linalg.norm(dm[q] - want) < 1e-4 * np.linalg.norm(want) + 1e-16, q
    dS = O.moments() - S0
    for k in range(nzw):
        for j in range(nyw):
            for i in range(nxw):
                s = i + nxw * (j + nyw * k)
                if grain[cell_of(i, j, k)] < 0:
                    continue
                want = -G * np.cross(S0[s], Bd[cell_of(i, j, k)]) * dt
                assert np.linalg.norm(dS[s] - want) < 1e-4 * np.linalg.norm(want) + 1e-16, s


def check_window_target():
    """The window is centred on the laser spot and stays on the track."""
    p = o.MsParams(20, 1, 1, 1e-9, 4, 6, J=J_SC, x0=10.2e-9, vx=1.0)
    assert o.ms_target(p, 0.0) == 7
    assert o.ms_target(p, 5e-9) == 12
    assert o.ms_target(p, 1.0) == 14
    p2 = o.MsParams(20, 1, 1, 1e-9, 4, 6, J=J_SC, x0=-3e-9)
    assert o.ms_target(p2, 0.0) == 0


def check_set_drivers_continues_run():
    """Replacing the drivers between steps by the same ones leaves the run bitwise what an
    uninterrupted run gives (the step count, window and state are kept: the laser keeps moving
    and the noise keeps its counters); drivers for another track are refused."""
    kw = dict(J=J_SC, ku=KU, dt=1e-16, T_amb=300.0, T_peak=1200.0, fwhm=4e-9, x0=4.2e-9, y0=1e-9,
              vx=2e5, B0=1.0, direction=(0.0, 0.0, -1.0), seed=5)
    p = o.MsParams(16, 2, 1, 2 * A, 2, 4, **kw)
    a, b = o.MsOracle(p), o.MsOracle(p)
    m0 = _tilted(p.n_cells, 3, 40.0)
    for O in (a, b):
        O.set_cells(m0)
        O.set_window(o.ms_target(p, 0.0))
    a.run(30, follow=True)
    b.run(13, follow=True)
    b.set_drivers(o.MsParams(16, 2, 1, 2 * A, 2, 4, **kw))
    b.run(17, follow=True)
    assert a.step == b.step == 30 and a.window == b.window
    assert np.array_equal(a.cells(), b.cells()) and np.array_equal(a.moments(), b.moments())
    try:
        b.set_drivers(o.MsParams(17, 2, 1, 2 * A, 2, 4, **kw))
        raise AssertionError("drivers of another track accepted")
    except ValueError:
        pass


def check_second_pass_keeps_written_tracks():
    """Two passes along parallel tracks (Sec. III): at T = 0 with no write field, every spin
    along +z or -z stays exactly there (its field is along z, so there is no torque and no
    noise), Eq. 6 of a uniform cell returns its direction and a cone of half-angle 0 returns
    the cell's direction.  So after a first pass along one row band, then new drivers (spot
    centre on the other band, spot and head restarted at the current time) and a second pass,
    both written patterns read back exactly and the window follows the new spot."""
    ncx, ncy, ncz, r, wx, L = 36, 10, 1, 2, 6, 4
    cell = 2 * A
    v = 4 * cell / (60 * 1e-16)        # four cells per 60 steps
    kw = dict(J=J_SC, ku=KU, dt=1e-16, T_amb=0.0, vx=v, B0=0.0, seed=9)
    p1 = o.MsParams(ncx, ncy, ncz, cell, r, wx, x0=3.2 * cell, y0=2 * cell, **kw)
    pat1 = [0, 1, 1, 0, 1, 0, 0, 1, 0]
    pat2 = [1, 1, 0, 0, 1, 0, 1, 1, 0]
    m = np.zeros((ncz, ncy, ncx, 3))
    m[..., 2] = 1.0
    for b in range(len(pat1)):
        m[:, 0:4, b * L:(b + 1) * L, 2] = -1.0 if pat1[b] else 1.0
        m[:, 6:10, b * L:(b + 1) * L, 2] = -1.0 if pat2[b] else 1.0
    m = m.reshape(-1, 3)
    O = o.MsOracle(p1)
    O.set_cells(m)
    O.set_window(o.ms_target(p1, 0.0))
    O.run(240, follow=True)
    assert O.window == o.ms_target(p1, 240e-16) > 15
    t1 = O.step * 1e-16
    p2 = o.MsParams(ncx, ncy, ncz, cell, r, wx, x0=3.2 * cell - v * t1, y0=8 * cell, **kw)
    O.set_drivers(p2)
    O.set_window(o.ms_target(p2, t1))
    assert O.window == o.ms_target(p1, 0.0)
    O.run(240, follow=True)
    assert O.window == o.ms_target(p2, O.step * 1e-16) > 15
    assert np.array_equal(O.cells()[O.window * 0:], O.cells())
    cells = O.cells().reshape(ncz, ncy, ncx, 3)
    outside = np.ones(ncx, bool)
    outside[O.window:O.window + wx] = False
    assert np.array_equal(cells[:, :, outside], m.reshape(ncz, ncy, ncx, 3)[:, :, outside])
    for (c0, c1), pat in (((0, 4), pat1), ((6, 10), pat2)):
        sig, bits = O.read_track(0.0, L * cell, len(pat), c0, c1)
        assert list(bits) == pat
        assert np.array_equal(np.abs(sig), np.ones(len(pat)))
    S = O.moments()
    assert np.array_equal(np.abs(S[:, 2]), np.ones(len(S))) and not S[:, :2].any()


def check_window_replacement_hands_back():
    """Placing a window elsewhere first hands the old window's sites back to their cells by
    Eq. 6 (brute force over each cell's sites), as the trailing column of a move is; after
    set_cells the old sites are stale, and a re-placement hands nothing back."""
    ncx, ncy, ncz, r, wx = 12, 2, 1, 2, 4
    p = o.MsParams(ncx, ncy, ncz, 2 * A, r, wx, J=J_SC, ku=KU, dt=1e-16, T_amb=200.0, seed=3)
    O = o.MsOracle(p)
    m0 = _tilted(p.n_cells, 4, 50.0)
    O.set_cells(m0)
    O.set_window(2)
    S = _tilted(O.nw, 5, 70.0)
    O.set_moments(S)
    O.set_window(7)
    cells = O.cells().reshape(ncz, ncy, ncx, 3)
    Sw = S.reshape(ncz * r, ncy * r, wx * r, 3)
    for cy in range(ncy):
        for cx in range(2, 2 + wx):
            s = Sw[:, cy * r:(cy + 1) * r, (cx - 2) * r:(cx - 1) * r].reshape(-1, 3).sum(axis=0)
            assert np.abs(cells[0, cy, cx] - s / np.linalg.norm(s)).max() < 1e-14
    rest = np.ones(ncx, bool)
    rest[2:2 + wx] = False
    assert np.array_equal(cells[:, :, rest], m0.reshape(ncz, ncy, ncx, 3)[:, :, rest])
    O.set_cells(m0)
    O.set_window(1)
    assert np.array_equal(O.cells(), m0)


def check_region_frozen_end_spin_wave():
    """Simulated region (Sec. II, Fig. 1): cells beyond it are frozen, so the region's edge
    cell sees a neighbour that does not move.  A chain of N region cells with a free end (a
    non-magnetic cell) and a frozen end (cells held along +z) carries small standing waves
    m_x + i m_y = eps cos(th (j + 1/2)), th = (2n - 1) pi / (2N + 1), the modes of the
    Laplacian with one missing and one fixed neighbour (eigenvalue 2 - 2 cos th), precessing
    at gamma [B + 2 K0 m_e^2 / Ms0 + (2 A0 m_e / Ms0)(2 - 2 cos th) / c^2]."""
    N, F, c, T, B0, eps = 12, 6, 1e-9, 400.0, 0.5, 1e-4
    p = o.MsParams(N + F + 1, 1, 1, c, 4, 1, J=J_SC, ku=KU, lam=0.0, dt=1e-16, T_amb=T, B0=B0,
                   direction=(0, 0, 1), A0=J_SC / (2 * A), Ms0=MU_S / A ** 3, K0=KU / A ** 3, margin=N)
    grain = np.zeros(N + F + 1, np.int32)
    grain[0] = -1                       # the window's cell: no atomistic sites
    me = o.me(p.T_C, T, MU_S, B0)
    for n in (1, 2):
        th = (2 * n - 1) * math.pi / (2 * N + 1)
        O = o.MsOracle(p, grain)
        j = np.arange(N)
        amp = eps * np.cos(th * (j + 0.5))
        m = np.zeros((N + F + 1, 3))
        m[:, 2] = 1.0
        m[1:N + 1, 0] = amp
        m[1:N + 1, 2] = np.sqrt(1 - amp ** 2)
        O.set_cells(m)
        O.set_window(0)
        steps = 300
        O.run(steps)
        got = O.cells()
        assert np.array_equal(got[N + 1:], m[N + 1:])      # the frozen cells did not move
        w = G * (B0 + 2 * p.K0 * me ** 2 / p.Ms0 + 2 * p.A0 * me / p.Ms0 * (2 - 2 * math.cos(th)) / c ** 2)
        ph = np.arctan2(got[1:N + 1, 1], got[1:N + 1, 0])
        want = w * steps * p.drv.dt
        assert abs((ph[0] - want + math.pi) % (2 * math.pi) - math.pi) < 1e-4 * want, (n, ph[0], want)


def _region_pair(margin, demag, steps, seed=3):
    """The same moving-window run with the whole track evolved and with a simulated region."""
    kw = dict(J=J_SC, ku=KU, dt=1e-16, T_amb=300.0, T_peak=1300.0, fwhm=5e-9, x0=7.3e-9, y0=2e-9, vx=2.5e5,
              B0=1.2, direction=(0.1, 0.0, -1.0), seed=seed, demag=demag)
    grain = np.zeros(30 * 4 * 2, np.int32)
    grain.reshape(2, 4, 30)[:, :, 17] = -1
    out = []
    for g in (-1, margin):
        p = o.MsParams(30, 4, 2, 1e-9, 2, 6, margin=g, **kw)
        O = o.MsOracle(p, grain)
        O.set_cells(_tilted(p.n_cells, seed, 30.0) * (grain >= 0)[:, None])
        O.set_window(o.ms_target(p, 0.0))
        O.run(steps, follow=True)
        out.append(O)
    return out


def check_region_covering_track_is_whole_track():
    """A simulated region at least as long as the track evolves every cell: bitwise the
    whole-track run, window moves and the demagnetising field included."""
    a, b = _region_pair(40, True, 40)
    assert a.window == b.window > o.ms_target(a.p, 0.0)
    assert np.array_equal(a.cells(), b.cells()) and np.array_equal(a.moments(), b.moments())


def check_region_first_step_and_frozen_cells():
    """One coupled step with a simulated region: the window and the region's cells at least
    four columns inside its edges are bitwise the whole-track step (an edge cell sees a frozen
    neighbour's m in the four RK4 stages, the whole track a moving one, and that difference
    moves one column per stage; the demagnetising field of the frozen cells uses the m_e stored
    at the placement, the current one on the first step), and the frozen cells do not move;
    over a longer run the cells ahead of the region stay as they were."""
    a, b = _region_pair(6, True, 1)
    ox, cols = b.window, np.arange(30)
    region = (cols >= ox - 6) & (cols < ox + 6 + 6)
    inner = (cols >= ox - 2) & (cols < ox + 6 + 2)
    ca, cb = a.cells().reshape(2, 4, 30, 3), b.cells().reshape(2, 4, 30, 3)
    assert np.array_equal(ca[:, :, inner], cb[:, :, inner])
    assert np.array_equal(a.moments(), b.moments())
    c0 = _tilted(30 * 4 * 2, 3, 30.0).reshape(2, 4, 30, 3)
    mag = np.ones((2, 4, 30), bool)
    mag[:, :, 17] = False
    out = ~region
    assert np.array_equal(cb[:, :, out][mag[:, :, out]], c0[:, :, out][mag[:, :, out]])
    assert not np.array_equal(ca[:, :, out], cb[:, :, out])
    a, b = _region_pair(3, False, 40)
    ahead = cols >= b.window + 6 + 3
    cb = b.cells().reshape(2, 4, 30, 3)
    assert ahead.any() and np.array_equal(cb[:, :, ahead][mag[:, :, ahead]], c0[:, :, ahead][mag[:, :, ahead]])


FAST_CHECKS = [
    check_langevin_branches, check_me_limits, check_micromagnetic_damping_law,
    check_theta_max_printed_values, check_cone_distribution, check_eq6_average_brute_force,
    check_uniform_state_stationary_through_shifts, check_isolated_cell_llg, check_mm_standing_spin_wave,
    check_ratio_one_window_matches_atomistic_lattice, check_full_window_equals_atomistic_oracle,
    check_shift_moves_spins, check_window_target, check_read_track, check_head_profile_shape,
    check_isolated_cell_and_site_in_head_profile, check_demag_tensor_limits, check_demag_uniform_film,
    check_demag_in_coupled_step, check_set_drivers_continues_run, check_second_pass_keeps_written_tracks,
    check_window_replacement_hands_back, check_region_frozen_end_spin_wave,
    check_region_covering_track_is_whole_track, check_region_first_step_and_frozen_cells,
]
