"""FP64 CPU oracle for the stochastic LLG Heun step (arXiv 2502.02236, Sec. II).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline leg
of the benchmark are the only callers.  The oracle is a plain C program
(hamr_oracle.c) reached through ctypes; it shares no code with the CUDA library.

Geometry helpers here state the lattices of the paper from their definitions:
  * simple cubic, spacing a, one exchange shell at distance a (6 neighbours, Sec. II);
  * L1_0 FePt, Fe sites only (Appendix A): Fe planes are square nets of spacing
    a' = a/sqrt(2) stacked at c; exchange shells at a' (4 in-plane), c (2 out of
    plane) and a (4 in-plane diagonals), i.e. 4 nearest + 6 next-nearest (Sec. II).
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

C_MU_B = 9.2740100783e-24          # Bohr magneton [J/T]
C_GAMMA = 1.76085963023e11         # electron gyromagnetic ratio [rad/(s T)]
C_KB = 1.380649e-23                # Boltzmann constant [J/K]

_lib = None


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3),
        ("ax", ctypes.c_double), ("ay", ctypes.c_double), ("az", ctypes.c_double),
        ("n_shells", ctypes.c_int32),
        ("shell_dist", ctypes.c_double * 4),
        ("J", ctypes.c_double * 4),
        ("mu_s", ctypes.c_double), ("ku", ctypes.c_double), ("alpha", ctypes.c_double),
        ("dt", ctypes.c_double), ("gamma", ctypes.c_double),
        ("T_amb", ctypes.c_double), ("T_peak", ctypes.c_double), ("fwhm", ctypes.c_double),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("vx", ctypes.c_double),
        ("vy", ctypes.c_double),
        ("B0", ctypes.c_double), ("dir", ctypes.c_double * 3),
        ("n_bits", ctypes.c_int32),
        ("bits", ctypes.POINTER(ctypes.c_uint8)),
        ("bit_len", ctypes.c_double), ("ramp_len", ctypes.c_double),
        ("head_x0", ctypes.c_double), ("head_v", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class OrcMsParams(ctypes.Structure):
    _fields_ = [
        ("ncx", ctypes.c_int32), ("ncy", ctypes.c_int32), ("ncz", ctypes.c_int32),
        ("cell", ctypes.c_double), ("ratio", ctypes.c_int32), ("wx", ctypes.c_int32),
        ("J", ctypes.c_double), ("mu_s", ctypes.c_double), ("ku", ctypes.c_double),
        ("Ms0", ctypes.c_double), ("A0", ctypes.c_double), ("K0", ctypes.c_double),
        ("lambda_", ctypes.c_double), ("T_C", ctypes.c_double),
        ("drv", OrcParams),
        ("profile", ctypes.c_int32), ("prof_wz", ctypes.c_double), ("prof_dz", ctypes.c_double),
        ("prof_Bx0", ctypes.c_double), ("prof_wx", ctypes.c_double), ("prof_dx", ctypes.c_double),
        ("demag", ctypes.c_int32), ("margin", ctypes.c_int32),
    ]


def _dp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i64, i32, u64, d = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_uint64, ctypes.c_double)
        P = ctypes.POINTER(OrcParams)
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_thermal_normals.argtypes = [u64, u64, u64, vp]
        L.orc_temperature.argtypes = [P, d, d, d]
        L.orc_temperature.restype = d
        L.orc_field_polarity.argtypes = [P, d]
        L.orc_field_polarity.restype = d
        L.orc_applied_field.argtypes = [P, d, vp]
        L.orc_llg_rhs.argtypes = [P, vp, vp, vp]
        L.orc_site_neighbours.argtypes = [P, vp, i64, vp, vp, ctypes.c_int]
        L.orc_site_neighbours.restype = ctypes.c_int
        L.orc_create.argtypes = [P, vp]
        L.orc_create.restype = vp
        L.orc_destroy.argtypes = [vp]
        L.orc_n_sites.argtypes = [vp]
        L.orc_n_sites.restype = i64
        L.orc_nnz.argtypes = [vp]
        L.orc_nnz.restype = i64
        L.orc_get_neighbours.argtypes = [vp, vp, vp, vp]
        L.orc_set_drivers.argtypes = [vp, d, d, d, d, d, d, d]
        L.orc_heun_step.argtypes = [vp, vp, i64]
        L.orc_heun_step.restype = ctypes.c_int
        L.orc_magnetisation.argtypes = [vp, vp, vp]
        L.orc_run.argtypes = [vp, vp, i64, i64, i32, vp]
        L.orc_run.restype = i64
        L.orc_grain_sums.argtypes = [vp, vp, i32, vp, vp]
        L.orc_energy.argtypes = [vp, vp, i64]
        L.orc_energy.restype = d
        L.orc_step_sites.argtypes = [P, vp, vp, i64, i64, vp, vp]
        L.orc_step_sites.restype = ctypes.c_int
        # multiscale window (hamr_ms_oracle.c)
        MP = ctypes.POINTER(OrcMsParams)
        L.orc_langevin.argtypes = [d]
        L.orc_langevin.restype = d
        L.orc_me.argtypes = [d, d, d, d]
        L.orc_me.restype = d
        L.orc_theta_max.argtypes = [d]
        L.orc_theta_max.restype = d
        L.orc_ms_alpha.argtypes = [MP, d]
        L.orc_ms_alpha.restype = d
        L.orc_cone_sample.argtypes = [vp, d, u64, u64, u64, vp]
        L.orc_ms_window_sites.argtypes = [MP]
        L.orc_ms_window_sites.restype = i64
        L.orc_ms_create.argtypes = [MP, vp]
        L.orc_ms_create.restype = vp
        L.orc_ms_destroy.argtypes = [vp]
        L.orc_ms_set_drivers.argtypes = [vp, MP]
        L.orc_ms_set_drivers.restype = ctypes.c_int
        L.orc_ms_set_cells.argtypes = [vp, vp]
        L.orc_ms_get_cells.argtypes = [vp, vp]
        L.orc_ms_get_moments.argtypes = [vp, vp]
        L.orc_ms_set_moments.argtypes = [vp, vp]
        L.orc_ms_window.argtypes = [vp]
        L.orc_ms_window.restype = i32
        L.orc_ms_step_count.argtypes = [vp]
        L.orc_ms_step_count.restype = i64
        L.orc_ms_set_window.argtypes = [vp, i32]
        L.orc_ms_set_window.restype = ctypes.c_int
        L.orc_ms_target.argtypes = [MP, d]
        L.orc_ms_target.restype = i32
        L.orc_ms_run.argtypes = [vp, i64, i32]
        L.orc_ms_run.restype = ctypes.c_int
        L.orc_ms_read_track.argtypes = [vp, d, d, i32, i32, i32, vp, vp]
        L.orc_ms_field.argtypes = [MP, d, d, vp]
        L.orc_newell_f.argtypes = [d, d, d]
        L.orc_newell_f.restype = d
        L.orc_newell_g.argtypes = [d, d, d]
        L.orc_newell_g.restype = d
        L.orc_demag_tensor.argtypes = [d, d, d, d, d, d, vp]
        L.orc_demag_field.argtypes = [MP, vp, vp]
        _lib = L
    return _lib


# --------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key):
    """Philox4x32-10 block: four 32-bit counter words and two key words -> four words."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_dp(c), _dp(k), _dp(out))
    return out


def thermal_normals(seed, site, step):
    """The three standard normals of (seed, site, step)."""
    xi = np.zeros(3)
    lib().orc_thermal_normals(int(seed), int(site), int(step), _dp(xi))
    return xi


# --------------------------------------------------------------------------- params
class Params:
    """Physical and driver parameters of one replica (plain attributes, SI units)."""

    def __init__(self, nx, ny, nz, spacing, shells, J, *, periodic=(False, False, False),
                 mu_s=3 * C_MU_B, ku=0.0, alpha=0.1, dt=1e-16, gamma=C_GAMMA, seed=1,
                 T_amb=0.0, T_peak=0.0, fwhm=0.0, x0=0.0, y0=0.0, vx=0.0, vy=0.0,
                 B0=0.0, direction=(0.0, 0.0, 1.0), bits=(), bit_len=1.0, ramp_len=0.0,
                 head_x0=0.0, head_v=0.0):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.spacing = tuple(float(s) for s in spacing)
        self.shells = tuple(float(s) for s in shells)
        self.J = tuple(float(j) for j in J)
        assert len(self.shells) == len(self.J) <= 4
        self.periodic = tuple(bool(p) for p in periodic)
        self.mu_s, self.ku, self.alpha, self.dt, self.gamma = mu_s, ku, alpha, dt, gamma
        self.seed = int(seed)
        self.T_amb, self.T_peak, self.fwhm = T_amb, T_peak, fwhm
        self.x0, self.y0, self.vx, self.vy = x0, y0, vx, vy
        self.B0, self.direction = B0, tuple(direction)
        self.bits = np.asarray(bits, dtype=np.uint8)
        self.bit_len, self.ramp_len, self.head_x0, self.head_v = bit_len, ramp_len, head_x0, head_v

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def struct(self):
        s = OrcParams()
        s.nx, s.ny, s.nz = self.nx, self.ny, self.nz
        for d in range(3):
            s.periodic[d] = int(self.periodic[d])
            s.dir[d] = self.direction[d]
        s.ax, s.ay, s.az = self.spacing
        s.n_shells = len(self.shells)
        for k in range(len(self.shells)):
            s.shell_dist[k] = self.shells[k]
            s.J[k] = self.J[k]
        s.mu_s, s.ku, s.alpha, s.dt, s.gamma = self.mu_s, self.ku, self.alpha, self.dt, self.gamma
        s.T_amb, s.T_peak, s.fwhm = self.T_amb, self.T_peak, self.fwhm
        s.x0, s.y0, s.vx, s.vy = self.x0, self.y0, self.vx, self.vy
        s.B0 = self.B0
        s.n_bits = len(self.bits)
        self._bits_keep = np.ascontiguousarray(self.bits)
        s.bits = self._bits_keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        s.bit_len, s.ramp_len, s.head_x0, s.head_v = (self.bit_len, self.ramp_len,
                                                      self.head_x0, self.head_v)
        s.seed = self.seed
        return s


def sc_params(nx, ny, nz, a, J, **kw):
    """Simple cubic lattice of spacing a with one exchange shell at distance a."""
    return Params(nx, ny, nz, (a, a, a), (a,), (J,), **kw)


def l10_params(nx, ny, nz, a, c, J1, J2, J3, **kw):
    """L1_0 Fe sublattice: square nets of spacing a/sqrt(2) stacked at c; shells at
    a/sqrt(2) (J1), c (J2) and a (J3)."""
    ap = a / math.sqrt(2.0)
    return Params(nx, ny, nz, (ap, ap, c), (ap, c, a), (J1, J2, J3), **kw)


# --------------------------------------------------------------------------- driver functions
def temperature(p, x, y, t):
    s = p.struct()
    return lib().orc_temperature(ctypes.byref(s), float(x), float(y), float(t))


def field_polarity(p, t):
    s = p.struct()
    return lib().orc_field_polarity(ctypes.byref(s), float(t))


def applied_field(p, t):
    s = p.struct()
    B = np.zeros(3)
    lib().orc_applied_field(ctypes.byref(s), float(t), _dp(B))
    return B


def llg_rhs(p, S, B):
    s = p.struct()
    S = np.ascontiguousarray(S, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    f = np.zeros(3)
    lib().orc_llg_rhs(ctypes.byref(s), _dp(S), _dp(B), _dp(f))
    return f


# --------------------------------------------------------------------------- lattice runs
class Oracle:
    """One replica: parameters, grain map (int32, -1 = non-magnetic) and neighbour list."""

    def __init__(self, p, grain=None):
        self.p = p
        self._s = p.struct()
        if grain is None:
            grain = np.zeros(p.n, dtype=np.int32)
        self.grain = np.ascontiguousarray(grain, dtype=np.int32).reshape(-1)
        assert self.grain.size == p.n
        self._h = lib().orc_create(ctypes.byref(self._s), _dp(self.grain))
        if not self._h:
            raise MemoryError("oracle context allocation failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    @property
    def n(self):
        return self.p.n

    def neighbours(self):
        """CSR of the bond list: row_ptr[n+1], col[nnz], shell[nnz] (int64, int64, int32)."""
        L = lib()
        nnz = L.orc_nnz(self._h)
        rp = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(max(nnz, 1), dtype=np.int64)
        sh = np.zeros(max(nnz, 1), dtype=np.int32)
        L.orc_get_neighbours(self._h, _dp(rp), _dp(col), _dp(sh))
        return rp, col[:nnz], sh[:nnz]

    def set_drivers(self, T_amb, T_peak=0.0, fwhm=0.0, x0=0.0, y0=0.0, vx=0.0, vy=0.0):
        lib().orc_set_drivers(self._h, T_amb, T_peak, fwhm, x0, y0, vx, vy)

    def step(self, S, step):
        """One Heun step in place on S (float64 array of shape (n, 3))."""
        assert S.dtype == np.float64 and S.flags.c_contiguous and S.size == 3 * self.n
        if lib().orc_heun_step(self._h, _dp(S), int(step)) != 0:
            raise MemoryError("oracle step allocation failed")
        return S

    def run(self, S, step0, n_steps, record_every=0):
        """n_steps steps in place; returns the magnetisation records, shape (n_rec, 3)."""
        assert S.dtype == np.float64 and S.flags.c_contiguous and S.size == 3 * self.n
        n_rec = (step0 + n_steps) // record_every - step0 // record_every if record_every > 0 else 0
        M = np.zeros((max(n_rec, 1), 3))
        got = lib().orc_run(self._h, _dp(S), int(step0), int(n_steps), int(record_every), _dp(M))
        if got < 0:
            raise MemoryError("oracle step allocation failed")
        return M[:got]

    def magnetisation(self, S):
        M = np.zeros(3)
        lib().orc_magnetisation(self._h, _dp(np.ascontiguousarray(S, dtype=np.float64)), _dp(M))
        return M

    def grain_sums(self, S, n_grains):
        sums = np.zeros((max(n_grains, 1), 3))
        counts = np.zeros(max(n_grains, 1), dtype=np.int64)
        lib().orc_grain_sums(self._h, _dp(np.ascontiguousarray(S, dtype=np.float64)),
                             int(n_grains), _dp(sums), _dp(counts))
        return sums[:n_grains], counts[:n_grains]

    def energy(self, S, step):
        return lib().orc_energy(self._h, _dp(np.ascontiguousarray(S, dtype=np.float64)), int(step))


def step_sites(p, grain, S, step, sites):
    """State after step `step` at the listed sites only, from the full pre-step state."""
    s = p.struct()
    grain = np.ascontiguousarray(grain, dtype=np.int32).reshape(-1)
    S = np.ascontiguousarray(S, dtype=np.float64)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.zeros((sites.size, 3))
    rc = lib().orc_step_sites(ctypes.byref(s), _dp(grain), _dp(S), int(step), sites.size,
                              _dp(sites), _dp(out))
    if rc != 0:
        raise RuntimeError("oracle neighbour list overflow")
    return out


# --------------------------------------------------------------------------- multiscale window
def langevin(x):
    """L(x) = coth x - 1/x (Sec. II)."""
    return lib().orc_langevin(float(x))


def me(T_C, T, mu_s, B):
    """Equilibrium magnetisation m_e(T): the root of m = L(3 T_C m / T + mu_s B / kB T)."""
    return lib().orc_me(float(T_C), float(T), float(mu_s), float(B))


def theta_max(mr):
    """Half-angle of the thermalisation cone for M / Ms0 = mr (Sec. II)."""
    return lib().orc_theta_max(float(mr))


def cone_sample(e3, th_max, seed, site, event):
    out = np.zeros(3)
    e3 = np.ascontiguousarray(e3, dtype=np.float64)
    lib().orc_cone_sample(_dp(e3), float(th_max), int(seed), int(site), int(event), _dp(out))
    return out


class MsParams:
    """Multiscale window: ncx x ncy x ncz micromagnetic cells of edge `cell`, an atomistic
    simple-cubic window of spacing cell/ratio covering wx cell columns (all of y and z).
    The micromagnetic constants default to the atomistic ones per unit volume: Ms0 =
    mu_s / a^3, K0 = ku / a^3 (Appendix A) and A0 = J / 2a (Eq. 9)."""

    def __init__(self, ncx, ncy, ncz, cell, ratio, wx, *, J, mu_s=3 * C_MU_B, ku=0.0, lam=0.1,
                 T_C=None, Ms0=None, A0=None, K0=None, dt=1e-16, gamma=C_GAMMA, seed=1,
                 T_amb=0.0, T_peak=0.0, fwhm=0.0, x0=0.0, y0=0.0, vx=0.0, vy=0.0,
                 B0=0.0, direction=(0.0, 0.0, 1.0), bits=(), bit_len=1.0, ramp_len=0.0,
                 head_x0=0.0, head_v=0.0, profile=None, demag=False, margin=-1):
        self.ncx, self.ncy, self.ncz = int(ncx), int(ncy), int(ncz)
        self.demag = bool(demag)
        # simulated region: the window and `margin` cell columns on each side are evolved, the
        # rest of the track is frozen (margin < 0: the whole track is evolved)
        self.margin = int(margin)
        # head profile: dict(wz=, dz=, Bx0=, wx=, dx=) or None for a uniform field
        self.profile = dict(profile) if profile else None
        self.cell, self.ratio, self.wx = float(cell), int(ratio), int(wx)
        a = self.cell / self.ratio
        self.a = a
        self.J, self.mu_s, self.ku, self.lam = J, mu_s, ku, lam
        self.T_C = 1.443 * J / C_KB if T_C is None else T_C
        self.Ms0 = mu_s / a ** 3 if Ms0 is None else Ms0
        self.A0 = J / (2 * a) if A0 is None else A0
        self.K0 = ku / a ** 3 if K0 is None else K0
        # the drivers, time step, gyromagnetic ratio and seed ride in an atomistic Params
        self.drv = Params(1, 1, 1, (a, a, a), (a,), (J,), mu_s=mu_s, ku=ku, alpha=lam, dt=dt,
                          gamma=gamma, seed=seed, T_amb=T_amb, T_peak=T_peak, fwhm=fwhm, x0=x0,
                          y0=y0, vx=vx, vy=vy, B0=B0, direction=direction, bits=bits,
                          bit_len=bit_len, ramp_len=ramp_len, head_x0=head_x0, head_v=head_v)

    @property
    def n_cells(self):
        return self.ncx * self.ncy * self.ncz

    @property
    def window_dims(self):
        r = self.ratio
        return (self.wx * r, self.ncy * r, self.ncz * r)

    def struct(self):
        s = OrcMsParams()
        s.ncx, s.ncy, s.ncz = self.ncx, self.ncy, self.ncz
        s.cell, s.ratio, s.wx = self.cell, self.ratio, self.wx
        s.J, s.mu_s, s.ku = self.J, self.mu_s, self.ku
        s.Ms0, s.A0, s.K0 = self.Ms0, self.A0, self.K0
        s.lambda_, s.T_C = self.lam, self.T_C
        s.drv = self.drv.struct()
        s.demag = int(self.demag)
        s.margin = self.margin
        if self.profile:
            s.profile = 1
            s.prof_wz, s.prof_dz = self.profile["wz"], self.profile["dz"]
            s.prof_Bx0, s.prof_wx, s.prof_dx = self.profile["Bx0"], self.profile["wx"], self.profile["dx"]
        self._keep = self.drv
        return s


def ms_alpha(p, T):
    s = p.struct()
    return lib().orc_ms_alpha(ctypes.byref(s), float(T))


def ms_field(p, x, t):
    """The write field at track position x and time t."""
    s = p.struct()
    B = np.zeros(3)
    lib().orc_ms_field(ctypes.byref(s), float(x), float(t), _dp(B))
    return B


def demag_tensor(X, Y, Z, dx, dy, dz):
    """(Nxx, Nyy, Nzz, Nxy, Nxz, Nyz) between cuboid cells at offset (X, Y, Z) (Eq. 7)."""
    N = np.zeros(6)
    lib().orc_demag_tensor(float(X), float(Y), float(Z), float(dx), float(dy), float(dz), _dp(N))
    return N


def demag_field(p, M):
    """B_d = -mu0 N * M on every cell of the track of p, by direct summation (M: (n_cells, 3) A/m)."""
    s = p.struct()
    M = np.ascontiguousarray(M, dtype=np.float64).reshape(-1)
    Bd = np.zeros((p.n_cells, 3))
    lib().orc_demag_field(ctypes.byref(s), _dp(M), _dp(Bd))
    return Bd


def ms_target(p, t):
    s = p.struct()
    return lib().orc_ms_target(ctypes.byref(s), float(t))


class MsOracle:
    """The multiscale window on the CPU: cells' grain ids (int32, -1 = non-magnetic),
    micromagnetic directions m (n_cells, 3) and the window spins S (n_window, 3)."""

    def __init__(self, p, cell_grain=None):
        self.p = p
        self._s = p.struct()
        if cell_grain is None:
            cell_grain = np.zeros(p.n_cells, dtype=np.int32)
        self.grain = np.ascontiguousarray(cell_grain, dtype=np.int32).reshape(-1)
        assert self.grain.size == p.n_cells
        self._h = lib().orc_ms_create(ctypes.byref(self._s), _dp(self.grain))
        if not self._h:
            raise MemoryError("oracle context allocation failed")
        self.nw = int(np.prod(p.window_dims))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_ms_destroy(h)
            self._h = None

    def set_drivers(self, p):
        """New drivers (laser spot, write field, head profile, demagnetising switch) from the
        MsParams p of the same track, material, time step and seed, from the next step on."""
        s = p.struct()
        if lib().orc_ms_set_drivers(self._h, ctypes.byref(s)) != 0:
            raise ValueError("the parameters describe another track or material")
        self.p = p
        self._s = s

    def set_cells(self, m):
        m = np.ascontiguousarray(m, dtype=np.float64).reshape(-1)
        assert m.size == 3 * self.p.n_cells
        lib().orc_ms_set_cells(self._h, _dp(m))

    def cells(self):
        m = np.zeros((self.p.n_cells, 3))
        lib().orc_ms_get_cells(self._h, _dp(m))
        return m

    def moments(self):
        S = np.zeros((self.nw, 3))
        lib().orc_ms_get_moments(self._h, _dp(S))
        return S

    def set_moments(self, S):
        S = np.ascontiguousarray(S, dtype=np.float64).reshape(-1)
        assert S.size == 3 * self.nw
        lib().orc_ms_set_moments(self._h, _dp(S))

    @property
    def window(self):
        return lib().orc_ms_window(self._h)

    @property
    def step(self):
        return lib().orc_ms_step_count(self._h)

    def set_window(self, ox):
        if lib().orc_ms_set_window(self._h, int(ox)) != 0:
            raise ValueError("window outside the track")

    def run(self, n_steps, follow=False):
        if lib().orc_ms_run(self._h, int(n_steps), int(bool(follow))) != 0:
            raise MemoryError("oracle step allocation failed")

    def read_track(self, x_start, bit_len, n_bits, cy0=0, cy1=None):
        """Mean m_z of the magnetic cells of each bit window and the bits it reads as."""
        cy1 = self.p.ncy if cy1 is None else cy1
        sig = np.zeros(max(n_bits, 1))
        bits = np.zeros(max(n_bits, 1), dtype=np.uint8)
        lib().orc_ms_read_track(self._h, float(x_start), float(bit_len), int(n_bits), int(cy0), int(cy1),
                                _dp(sig), _dp(bits))
        return sig[:n_bits], bits[:n_bits]
