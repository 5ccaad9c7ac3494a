"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each check raises AssertionError when the oracle departs from a closed form, an
invariant, a value printed in the paper or a published test vector.  They are plain
functions so that the mutation test can run them against an oracle with a planted
mistake.  Sections and equations refer to arXiv 2502.02236.
"""
import math
import os

import numpy as np

import oracle as o

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
A = 0.25e-9
MU_S = 3 * o.C_MU_B
G = o.C_GAMMA


def golden_params():
    out = {}
    with open(os.path.join(GOLDEN, "paper_parameters.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = v
    return out


# ----------------------------------------------------------------------------- RNG
def check_philox_kat():
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        got = o.philox4x32_10(w[0:4], w[4:6])
        assert list(got) == w[6:10], (r, [hex(x) for x in got])


def check_normals_statistics():
    """Box-Muller normals: zero mean, unit variance, no cross-correlation, normal shape."""
    from scipy import stats
    n = 20000
    xi = np.array([o.thermal_normals(7, i, 3) for i in range(n)])
    assert np.all(np.abs(xi.mean(axis=0)) < 5 / math.sqrt(n))
    assert np.all(np.abs(xi.var(axis=0) - 1) < 5 * math.sqrt(2 / n))
    c = np.corrcoef(xi.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 5 / math.sqrt(n))
    for d in range(3):
        assert stats.kstest(xi[:, d], "norm").pvalue > 1e-4
    # different steps and seeds give different streams
    assert not np.allclose(o.thermal_normals(7, 5, 3), o.thermal_normals(7, 5, 4))
    assert not np.allclose(o.thermal_normals(7, 5, 3), o.thermal_normals(8, 5, 3))


# ----------------------------------------------------------------------------- single spin
def _single(alpha, B0, ku=0.0, dt=1e-15, **kw):
    p = o.sc_params(1, 1, 1, A, 0.0, alpha=alpha, dt=dt, B0=B0, direction=(0, 0, 1), ku=ku,
                    mu_s=MU_S, **kw)
    return p, o.Oracle(p)


def _phase_track(orc, S, n_steps, chunk):
    """Unwrapped azimuth after each chunk of steps."""
    phis = [math.atan2(S[0, 1], S[0, 0])]
    step = 0
    for _ in range(n_steps // chunk):
        orc.run(S, step, chunk)
        step += chunk
        phis.append(math.atan2(S[0, 1], S[0, 0]))
    return np.unwrap(phis)


def check_larmor():
    """alpha = 0, T = 0, B = B0 z: phi(t) = phi0 + gamma B0 t, theta fixed (Eq. 1)."""
    B0, dt, th0 = 1.0, 1e-15, 0.7
    p, orc = _single(0.0, B0, dt=dt)
    S = np.array([[math.sin(th0), 0.0, math.cos(th0)]])
    ph = _phase_track(orc, S, 4000, 100)
    w = (ph[-1] - ph[0]) / (4000 * dt)
    assert abs(w / (G * B0) - 1) < 1e-7, w / (G * B0)
    assert abs(math.acos(S[0, 2]) - th0) < 1e-10


def check_anisotropy_precession():
    """alpha = 0: omega = gamma (B0 + 2 ku cos(theta) / mu_s) (Eq. 1 with Eq. 3)."""
    B0, ku, dt, th0 = 0.5, 1e-22, 1e-16, 0.4
    p, orc = _single(0.0, B0, ku=ku, dt=dt)
    S = np.array([[math.sin(th0), 0.0, math.cos(th0)]])
    ph = _phase_track(orc, S, 20000, 200)
    w = (ph[-1] - ph[0]) / (20000 * dt)
    want = G * (B0 + 2 * ku / MU_S * math.cos(th0))
    assert abs(w / want - 1) < 1e-7, w / want


def check_damped_relaxation():
    """alpha > 0: tan(theta/2) = tan(theta0/2) exp(-alpha gamma B0 t/(1+alpha^2)),
    dphi/dt = gamma B0 / (1 + alpha^2) (Eq. 1, Landau-Lifshitz form)."""
    al, B0, dt, th0, N = 0.1, 1.0, 1e-15, 2.5, 30000
    p, orc = _single(al, B0, dt=dt)
    S = np.array([[math.sin(th0), 0.0, math.cos(th0)]])
    ph = _phase_track(orc, S, N, 100)
    t = N * dt
    th = math.acos(S[0, 2])
    want = 2 * math.atan(math.tan(th0 / 2) * math.exp(-al * G * B0 * t / (1 + al * al)))
    assert abs(th - want) < 1e-7, (th, want)
    w = (ph[-1] - ph[0]) / t
    assert abs(w / (G * B0 / (1 + al * al)) - 1) < 1e-7


def check_heun_second_order():
    """Global error of the deterministic Heun step falls as dt^2."""
    al, B0, th0, T = 0.3, 10.0, 2.0, 20e-12
    want = 2 * math.atan(math.tan(th0 / 2) * math.exp(-al * G * B0 * T / (1 + al * al)))
    errs = []
    for dt in (4e-14, 2e-14, 1e-14):
        p, orc = _single(al, B0, dt=dt)
        S = np.array([[math.sin(th0), 0.0, math.cos(th0)]])
        orc.run(S, 0, int(round(T / dt)))
        errs.append(abs(math.acos(S[0, 2]) - want))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


# ----------------------------------------------------------------------------- lattice
def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def check_conservation_alpha0():
    """alpha = 0, T = 0, fields along z: energy and sum S_z are constants of motion; the
    Heun drift falls as dt^2; |S_i| = 1 after every step."""
    drifts = []
    for dt in (2e-16, 1e-16):
        p = o.sc_params(6, 5, 4, A, 6.7e-21, periodic=(True, True, True), ku=1e-22,
                        alpha=0.0, dt=dt, B0=-1.0, direction=(0, 0, 1))
        orc = o.Oracle(p)
        S = _random_state(p.n, 3)
        S[:, 2] = np.abs(S[:, 2]) + 1.0
        S /= np.linalg.norm(S, axis=1, keepdims=True)
        E0, Z0 = orc.energy(S, 0), S[:, 2].sum()
        n = int(round(2e-14 / dt))
        orc.run(S, 0, n)
        assert np.max(np.abs(np.linalg.norm(S, axis=1) - 1)) < 1e-14
        drifts.append((abs(orc.energy(S, n) - E0) / abs(E0), abs(S[:, 2].sum() - Z0) / p.n))
    (e1, z1), (e2, z2) = drifts
    assert e1 < 2e-4 and z1 < 5e-5, drifts
    # a first-order scheme would only halve the drift
    assert e1 / e2 > 3.5 and z1 / z2 > 3.5, drifts


def check_uniform_state_no_exchange_torque():
    """A uniform state on a periodic lattice feels an exchange field parallel to itself:
    with no other field it does not move (Eq. 2)."""
    p = o.sc_params(4, 4, 4, A, 6.7e-21, periodic=(True, True, True), alpha=0.1, dt=1e-16)
    orc = o.Oracle(p)
    v = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    S = np.tile(v, (p.n, 1))
    orc.run(S, 0, 50)
    assert np.max(np.abs(S - v)) < 1e-14


def check_energy_dissipation():
    """alpha > 0, T = 0, static field: the energy never increases (Eq. 1 damping term)."""
    p = o.sc_params(5, 4, 3, A, 6.7e-21, ku=1e-22, alpha=0.5, dt=1e-16, B0=-1.0,
                    direction=(0, 0, 1))
    orc = o.Oracle(p)
    S = _random_state(p.n, 4)
    E = [orc.energy(S, 0)]
    for k in range(20):
        orc.run(S, 10 * k, 10)
        E.append(orc.energy(S, 10 * k + 10))
    assert np.all(np.diff(E) <= 1e-12 * abs(E[0])), np.diff(E)
    assert E[-1] < E[0]


def _shell_offsets_l10(a, c):
    ap = a / math.sqrt(2)
    J1 = [(ap, 0, 0), (-ap, 0, 0), (0, ap, 0), (0, -ap, 0)]
    J2 = [(0, 0, c), (0, 0, -c)]
    J3 = [(ap, ap, 0), (ap, -ap, 0), (-ap, ap, 0), (-ap, -ap, 0)]
    return [J1, J2, J3]


def heun_phase_rate(w, dt):
    """Angular rate that Heun's scheme gives the linear oscillator dpsi/dt = i w psi: one
    step multiplies psi by 1 + i w dt - (w dt)^2 / 2."""
    th = w * dt
    return math.atan2(th, 1 - th * th / 2) / dt


def _measure_omega(p, k, n_steps, chunk, eps=1e-3):
    """Excite a small-amplitude plane wave of wavevector k about +z (alpha = 0, T = 0) and
    return the precession frequency of its Fourier amplitude."""
    orc = o.Oracle(p)
    ix, iy, iz = np.meshgrid(np.arange(p.nx), np.arange(p.ny), np.arange(p.nz), indexing="ij")
    ax, ay, az = p.spacing
    r = np.stack([(ix.T.ravel() + 0.5) * ax, (iy.T.ravel() + 0.5) * ay,
                  (iz.T.ravel() + 0.5) * az], axis=1)
    kr = r @ np.asarray(k)
    S = np.stack([eps * np.cos(kr), eps * np.sin(kr), np.ones_like(kr)], axis=1)
    S /= np.linalg.norm(S, axis=1, keepdims=True)
    S = np.ascontiguousarray(S)
    phase = np.exp(-1j * kr)
    ph = [np.angle(np.sum((S[:, 0] + 1j * S[:, 1]) * phase))]
    for s in range(n_steps // chunk):
        orc.run(S, s * chunk, chunk)
        ph.append(np.angle(np.sum((S[:, 0] + 1j * S[:, 1]) * phase)))
    ph = np.unwrap(ph)
    return (ph[-1] - ph[0]) / (n_steps * p.dt)


def check_spin_waves_sc():
    """Linear spin waves on a periodic SC lattice about +z, alpha = 0:
    omega(k) = gamma [B0 + 2 ku/mu_s + (J/mu_s) sum_d 2 (1 - cos k_d a)]."""
    J, ku, B0, dt = 6.7e-21, 1e-22, 1.0, 1e-16
    p = o.sc_params(16, 8, 4, A, J, periodic=(True, True, True), ku=ku, alpha=0.0, dt=dt,
                    B0=B0, direction=(0, 0, 1))
    for m in [(1, 0, 0), (3, 2, 0), (8, 0, 2), (5, 4, 1)]:
        k = (2 * math.pi * m[0] / (16 * A), 2 * math.pi * m[1] / (8 * A), 2 * math.pi * m[2] / (4 * A))
        want = G * (B0 + 2 * ku / MU_S + J / MU_S * sum(2 * (1 - math.cos(kd * A)) for kd in k))
        got = _measure_omega(p, k, 600, 20)
        assert abs(got / heun_phase_rate(want, dt) - 1) < 1e-5, (m, got / want)


def check_spin_waves_l10_shells():
    """L1_0 Fe sublattice with three shells J1, J2, J3:
    omega(k) = gamma [B0 + 2 ku/mu_s + sum_s (J_s/mu_s) sum_{delta in s} (1 - cos k.delta)]."""
    a, c = 0.385e-9, 0.371e-9
    J1 = 6.7e-21
    Js = (J1, 0.5 * J1, 0.1 * J1)
    ku, B0, dt = 2.6e-22, 1.0, 1e-16
    nx, ny, nz = 12, 8, 4
    p = o.l10_params(nx, ny, nz, a, c, *Js, periodic=(True, True, True), ku=ku, alpha=0.0,
                     dt=dt, B0=B0, direction=(0, 0, 1))
    ap = a / math.sqrt(2)
    shells = _shell_offsets_l10(a, c)
    for m in [(1, 0, 0), (2, 3, 0), (0, 0, 1), (5, 2, 2), (6, 4, 0)]:
        k = (2 * math.pi * m[0] / (nx * ap), 2 * math.pi * m[1] / (ny * ap), 2 * math.pi * m[2] / (nz * c))
        ex = sum(Js[s] * sum(1 - math.cos(np.dot(k, dl)) for dl in shells[s]) for s in range(3))
        want = G * (B0 + 2 * ku / MU_S + ex / MU_S)
        got = _measure_omega(p, k, 600, 20)
        assert abs(got / heun_phase_rate(want, dt) - 1) < 1e-5, (m, got / want)


def check_spin_wave_stiffness_eq9_eq10():
    """Long-wave limit reproduces Eq. 11 with A_SC = J/(2a) (Eq. 9) and, with one J for all
    ten L1_0 neighbours, A_L10 = 3J/(2a) (Eq. 10), using the paper's mu_s = Ms a^3 (SC) and
    Ms a^3 / 2 (L1_0) and its printed J values (Sec. III, Appendix A)."""
    gp = golden_params()
    Ms = float(gp["Ms_A_per_m"])
    # SC, a = 0.5 nm, J = 6.8e-21 J
    a, J = float(gp["a_SC_m"]), float(gp["J_SC_J"])
    mu = Ms * a ** 3
    nx = 128
    p = o.sc_params(nx, 1, 1, a, J, periodic=(True, True, True), mu_s=mu, alpha=0.0, dt=2e-16,
                    B0=1.0, direction=(0, 0, 1))
    w0 = G * 1.0
    A_sc = J / (2 * a)
    for m in (1, 2):
        k = 2 * math.pi * m / (nx * a)
        got = _measure_omega(p, (k, 0, 0), 2000, 50) - w0
        want = (2 * A_sc / Ms) * G * k ** 2      # lambda_ex gamma Ms k^2 with B = mu0 H
        assert abs(got / want - 1) < 1e-3 + (k * a) ** 2 / 12 * 1.5, (m, got / want)
    # L1_0, a = 0.385 nm, c = 0.371 nm, uniform J = 3.77e-21 J over all ten neighbours
    a, c, J = 0.385e-9, 0.371e-9, float(gp["J_L10_J"])
    mu = Ms * a ** 3 / 2
    ap = a / math.sqrt(2)
    p = o.l10_params(nx, 1, 1, a, c, J, J, J, periodic=(True, True, True), mu_s=mu, alpha=0.0,
                     dt=2e-16, B0=1.0, direction=(0, 0, 1))
    A_l10 = 3 * J / (2 * a)
    for m in (1, 2):
        k = 2 * math.pi * m / (nx * ap)
        got = _measure_omega(p, (k, 0, 0), 2000, 50) - w0
        want = (2 * A_l10 / Ms) * G * k ** 2
        assert abs(got / want - 1) < 1e-3 + (k * ap) ** 2 / 12 * 1.5, (m, got / want)


# ----------------------------------------------------------------------------- neighbours
def check_neighbour_geometry():
    """Bond counts from geometry: SC 6 (3 at an open corner), L1_0 Fe 10 = 4 nearest + 6
    next-nearest (Sec. II); bonds are symmetric with equal shells; the bond set of an
    open lattice equals the brute-force set of site pairs at a shell distance."""
    p = o.sc_params(5, 4, 3, A, 1.0)
    rp, col, sh = o.Oracle(p).neighbours()
    deg = np.diff(rp)
    assert deg[0] == 3 and deg.max() == 6 and deg[1 + 5 * (1 + 4 * 1)] == 6
    p = o.sc_params(5, 4, 3, A, 1.0, periodic=(True, True, True))
    rp, col, sh = o.Oracle(p).neighbours()
    assert np.all(np.diff(rp) == 6)
    p = o.l10_params(6, 5, 4, 0.385e-9, 0.371e-9, 1.0, 0.5, 0.1, periodic=(True, True, True))
    rp, col, sh = o.Oracle(p).neighbours()
    assert np.all(np.diff(rp) == 10)
    assert all(np.bincount(sh[rp[i]:rp[i + 1]], minlength=3).tolist() == [4, 2, 4] for i in range(p.n))
    for lat in (o.sc_params(4, 3, 3, A, 1.0),
                o.l10_params(4, 4, 3, 0.385e-9, 0.371e-9, 1.0, 0.5, 0.1)):
        rp, col, sh = o.Oracle(lat).neighbours()
        got = {(i, int(col[k]), int(sh[k])) for i in range(lat.n) for k in range(rp[i], rp[i + 1])}
        assert all((j, i, s) in got for (i, j, s) in got)
        ii, jj, kk = np.meshgrid(np.arange(lat.nx), np.arange(lat.ny), np.arange(lat.nz), indexing="ij")
        pos = np.stack([ii.T.ravel() * lat.spacing[0], jj.T.ravel() * lat.spacing[1],
                        kk.T.ravel() * lat.spacing[2]], axis=1)
        brute = set()
        for i in range(lat.n):
            d = np.linalg.norm(pos - pos[i], axis=1)
            for s, ds in enumerate(lat.shells):
                for j in np.nonzero(np.abs(d - ds) <= 1e-6 * ds)[0]:
                    if j != i:
                        brute.add((i, int(j), s))
        assert got == brute


def check_grain_decoupling():
    """No exchange bond crosses a grain boundary or touches a non-magnetic site, and a
    non-magnetic site (S = 0) stays zero (Sec. II: exchange-decoupled grains)."""
    p = o.sc_params(6, 4, 2, A, 6.7e-21, ku=1e-22, alpha=0.1, dt=1e-16, T_amb=300.0)
    grain = np.zeros(p.n, dtype=np.int32)
    ix = np.arange(p.n) % 6
    grain[ix >= 3] = 1
    grain[ix == 3] = -1
    orc = o.Oracle(p, grain)
    rp, col, sh = orc.neighbours()
    for i in range(p.n):
        for k in range(rp[i], rp[i + 1]):
            assert grain[col[k]] == grain[i] >= 0
    assert np.all(np.diff(rp)[grain < 0] == 0)
    S = _random_state(p.n, 5)
    S[grain < 0] = 0
    orc.run(S, 0, 20)
    assert np.all(S[grain < 0] == 0)
    assert np.max(np.abs(np.linalg.norm(S[grain >= 0], axis=1) - 1)) < 1e-14


# ----------------------------------------------------------------------------- drivers
def check_drivers():
    """Gaussian laser spot and trapezoidal bit-pattern write field (Sec. III, Fig. 2)."""
    gp = golden_params()
    bits = [int(ch) for ch in gp["bit_pattern"]]
    L = float(gp["bit_len_m"])
    v = float(gp["head_v_m_per_s"])
    p = o.sc_params(1, 1, 1, A, 0.0, T_amb=300.0, T_peak=800.0, fwhm=50e-9, x0=10e-9, y0=20e-9,
                    vx=v, bits=bits, bit_len=L, ramp_len=2e-9, head_x0=0.0, head_v=v, B0=0.8,
                    direction=(0, 0, 1))
    assert abs(o.temperature(p, 10e-9, 20e-9, 0.0) - 800.0) < 1e-12
    assert abs(o.temperature(p, 10e-9 + 25e-9, 20e-9, 0.0) - 550.0) < 1e-9    # r = FWHM/2
    assert abs(o.temperature(p, 10e-9 + v * 1e-9, 20e-9 + 25e-9, 1e-9) - 550.0) < 1e-9
    assert abs(o.temperature(p, 42e-9, 20e-9, 0.0) - 460.6) < 0.05           # r = 32 nm
    t_at = lambda xh: xh / v
    assert o.field_polarity(p, t_at(10e-9)) == 1.0                        # bit 0 = '0'
    assert o.field_polarity(p, t_at(45e-9)) == -1.0                       # bit 2 = '1'
    assert abs(o.field_polarity(p, t_at(41e-9))) < 1e-6                   # mid-ramp 0 -> 1
    assert abs(o.field_polarity(p, t_at(40.5e-9)) - 0.5) < 1e-6
    assert o.field_polarity(p, t_at(-5e-9)) == 1.0                        # before bit 0
    assert o.field_polarity(p, t_at(600e-9)) == -1.0                      # after last bit '1'
    for b, bit in enumerate(bits):
        want = -1.0 if bit else 1.0
        assert o.field_polarity(p, t_at((b + 0.5) * L)) == want
    B = o.applied_field(p, t_at(45e-9))
    assert np.allclose(B, [0, 0, -0.8])
    q = o.sc_params(1, 1, 1, A, 0.0, B0=1.0, direction=(0, 0, -1))        # static field
    assert np.allclose(o.applied_field(q, 123e-12), [0, 0, -1.0])


def check_eq8_parameter_law():
    """Eq. 8, J = 3 kB Tc/(eps z), reproduces the printed J_SC and J_L10 (Sec. III)."""
    gp = golden_params()
    Tc = float(gp["Tc_K"])
    for tag in ("SC", "L10"):
        eps, z, Jp = float(gp["eps_" + tag]), float(gp["z_" + tag]), float(gp["J_%s_J" % tag])
        J = 3 * o.C_KB * Tc / (eps * z)
        mant, ex = gp["J_%s_J" % tag].split("e")
        decimals = len(mant.split(".")[1]) if "." in mant else 0
        half_unit = 0.5 * 10.0 ** (-decimals) * 10.0 ** int(ex)   # rounding of the printed value
        assert abs(J - Jp) <= half_unit, (tag, J, Jp)


# ----------------------------------------------------------------------------- thermal
def _ensemble(n, alpha, B0, ku, T, dt, burn, sample, every):
    """Independent spins (no exchange) at temperature T; returns sampled S_z values."""
    p = o.sc_params(n, 1, 1, A, 0.0, alpha=alpha, dt=dt, B0=B0, direction=(0, 0, 1), ku=ku,
                    T_amb=T, seed=11)
    orc = o.Oracle(p)
    S = np.zeros((n, 3))
    S[:, 2] = 1.0
    orc.run(S, 0, burn)
    zs = []
    for k in range(sample // every):
        orc.run(S, burn + k * every, every)
        zs.append(S[:, 2].copy())
    return np.array(zs)


def _langevin(x):
    return 1 / math.tanh(x) - 1 / x


def check_boltzmann_field():
    """Single spins in a field at temperature T: <S_z> = L(mu_s B / kB T), the Langevin
    function (Sec. II), to within statistics and the O(dt) Heun bias."""
    T, x = 300.0, 2.0
    B0 = x * o.C_KB * T / MU_S
    z = _ensemble(2048, 1.0, B0, 0.0, T, 1e-16, 3000, 6000, 100)
    want = _langevin(x)
    err = z.std() / math.sqrt(z.size / 4)
    assert abs(z.mean() - want) < 5 * err + 0.01, (z.mean(), want, err)


def check_boltzmann_anisotropy():
    """Single spins with uniaxial anisotropy: P(S_z) ~ exp(s S_z^2), s = ku/kB T, so
    <S_z^2> = e^s/(s Z) - 1/(2 s) with Z = 2 int_0^1 exp(s x^2) dx (Eq. 3 at equilibrium)."""
    from scipy import integrate
    T, s = 300.0, 3.0
    ku = s * o.C_KB * T
    z = _ensemble(2048, 1.0, 0.0, ku, T, 1e-16, 3000, 6000, 100)
    Z = 2 * integrate.quad(lambda x: math.exp(s * x * x), 0, 1)[0]
    want = math.exp(s) / (s * Z) - 1 / (2 * s)
    z2 = z ** 2
    err = z2.std() / math.sqrt(z2.size / 4)
    assert abs(z2.mean() - want) < 5 * err + 0.01, (z2.mean(), want, err)


def check_isotropic_thermal():
    """No field and no anisotropy: the thermal field alone spreads spins uniformly over
    the sphere, <S_z> = 0 and <S_z^2> = 1/3."""
    z = _ensemble(2048, 1.0, 0.0, 0.0, 300.0, 1e-16, 3000, 6000, 100)
    err = 1 / math.sqrt(3 * z.size / 4)
    assert abs(z.mean()) < 5 * err + 0.01
    assert abs((z ** 2).mean() - 1 / 3) < 5 * err + 0.01


# checks the mutation test runs (fast ones first)
# ----------------------------------------------------------------------------- reductions
def check_energy_closed_form():
    """Uniform state v: every bond contributes -J_s (v.v = 1) once, so on a lattice with
    n_s bonds in shell s, E = -sum_s J_s n_s - N ku v_z^2 - N mu_s B.v (Eqs. 2, 3 as an
    energy).  SC, periodic x,y and open z: 3N - nx ny bonds.  L1_0 fully periodic: per
    site 2 in-plane nearest, 1 out-of-plane and 2 in-plane diagonal bonds."""
    v = np.array([0.36, -0.48, 0.8])
    B0, d = 0.7, np.array([0.6, 0.0, -0.8])
    nx, ny, nz, J, ku = 5, 4, 3, 6.7e-21, 1e-22
    p = o.sc_params(nx, ny, nz, A, J, periodic=(True, True, False), ku=ku, mu_s=MU_S, B0=B0,
                    direction=tuple(d))
    N = nx * ny * nz
    want = -J * (3 * N - nx * ny) - N * ku * v[2] ** 2 - N * MU_S * B0 * (d @ v)
    got = o.Oracle(p).energy(np.tile(v, (N, 1)), 0)
    assert abs(got - want) < 1e-12 * abs(want), (got, want)
    J1, J2, J3 = 6.7e-21, 3.35e-21, 0.67e-21
    p = o.l10_params(6, 6, 4, 0.385e-9, 0.371e-9, J1, J2, J3, periodic=(True, True, True), ku=0.0,
                     mu_s=MU_S)
    N = 6 * 6 * 4
    got = o.Oracle(p).energy(np.tile(v, (N, 1)), 0)
    want = -N * (2 * J1 + J2 + 2 * J3)
    assert abs(got - want) < 1e-12 * abs(want), (got, want)


def check_magnetisation_and_grain_sums():
    """M averages the magnetic sites only and the per-grain sums add each grain's spins
    (Eq. 6 as an average): against brute-force sums on a tiny lattice with voids; a +z
    state with voids has M = z exactly."""
    p = o.sc_params(5, 4, 3, A, 6.7e-21)
    rng = np.random.default_rng(5)
    grain = rng.integers(-1, 4, size=p.n).astype(np.int32)
    S = _random_state(p.n, 9)
    S[grain < 0] = 0.0
    orc = o.Oracle(p, grain)
    mag = grain >= 0
    assert np.allclose(orc.magnetisation(S), S[mag].sum(axis=0) / mag.sum(), rtol=0, atol=1e-15)
    sums, counts = orc.grain_sums(S, 4)
    for g in range(4):
        assert counts[g] == (grain == g).sum()
        assert np.allclose(sums[g], S[grain == g].sum(axis=0), rtol=0, atol=1e-14)
    up = np.zeros_like(S)
    up[mag, 2] = 1.0
    assert np.array_equal(orc.magnetisation(up), [0.0, 0.0, 1.0])


def check_step_sites_matches_full_step():
    """The site-by-site step used on full-size lattices gives what the whole-lattice step
    gives, at every site (granular, periodic in x, laser and write field on)."""
    p = o.sc_params(7, 6, 4, A, 6.7e-21, periodic=(True, False, False), ku=1e-22, alpha=0.1,
                    dt=1e-16, T_amb=300.0, T_peak=800.0, fwhm=2e-9, x0=1e-9, y0=0.7e-9, vx=2e4,
                    B0=0.8, direction=(0, 0, -1), seed=3)
    rng = np.random.default_rng(8)
    grain = rng.integers(-1, 3, size=p.n).astype(np.int32)
    S = _random_state(p.n, 10)
    S[grain < 0] = 0.0
    want = S.copy()
    o.Oracle(p, grain).step(want, 5)
    got = o.step_sites(p, grain, S, 5, np.arange(p.n))
    assert np.max(np.abs(got - want)) < 1e-15


FAST_CHECKS = [
    check_philox_kat, check_larmor, check_damped_relaxation, check_anisotropy_precession,
    check_uniform_state_no_exchange_torque, check_drivers, check_neighbour_geometry,
    check_grain_decoupling, check_spin_waves_sc, check_spin_waves_l10_shells,
    check_conservation_alpha0, check_normals_statistics, check_boltzmann_field,
    check_boltzmann_anisotropy, check_energy_closed_form, check_magnetisation_and_grain_sums,
    check_step_sites_matches_full_step,
]
