"""Seeded synthetic inputs shared by the library's tests, the benchmark and the oracle runs.

This module holds none of the sLLG arithmetic: it only draws inputs (granular grain
maps, initial spin states, replica sizes and temperatures, bit patterns) and names the
workloads.  Both the CUDA path and the FP64 oracle consume the same arrays.

Granular media (Sec. II-III of arXiv 2502.02236): exchange-decoupled columnar FePt grains
from a Voronoi construction, separated by non-magnetic boundaries.  The paper gives the
mean grain size (7, 8 or 9 nm) but no distribution; the grains here come from a jittered
hexagonal seed lattice whose jitter gives equivalent-circle diameters with a log-normal
spread of about 0.15, and a site is non-magnetic when it lies within half the boundary
width of a Voronoi edge.
"""
import math

import numpy as np

MU_B = 9.2740100783e-24          # Bohr magneton [J/T]
KB = 1.380649e-23               # Boltzmann constant [J/K]
GAMMA = 1.76085963023e11         # electron gyromagnetic ratio [rad/(s T)]

#: The bit pattern written in the paper's track simulations (Sec. III, Fig. 3).
PAPER_BIT_PATTERN = "0010111100101101100100001"

# hexagonal-lattice pitch per unit mean equivalent-circle diameter and the seed jitter
# (in units of the pitch) that give a log-normal diameter spread of about 0.15
_HEX_ECD = math.sqrt(2.0 * math.sqrt(3.0) / math.pi)
_JITTER = 0.27


def voronoi_grains(nx, ny, dx, dy, mean_diameter, boundary, seed, jitter=_JITTER):
    """Columnar grain map of an nx x ny site grid (spacing dx, dy [m]): int32 [ny, nx] with
    grain ids 0..G-1 and -1 on the non-magnetic boundaries.  Grain ids are renumbered
    densely in order of first appearance (x fastest)."""
    rng = np.random.default_rng(seed)
    pitch = mean_diameter / _HEX_ECD
    Lx, Ly = nx * dx, ny * dy
    rows = int(math.ceil(Ly / (pitch * math.sqrt(3) / 2))) + 3
    cols = int(math.ceil(Lx / pitch)) + 3
    jj, ii = np.meshgrid(np.arange(-1, rows - 1), np.arange(-1, cols - 1), indexing="ij")
    sx = (ii + 0.5 * (jj % 2)) * pitch
    sy = jj * pitch * math.sqrt(3) / 2
    seeds = np.stack([sx.ravel(), sy.ravel()], axis=1)
    seeds += rng.normal(scale=jitter * pitch, size=seeds.shape)
    # random global offset so that grid edges do not align with the seed lattice
    seeds += rng.uniform(0, pitch, size=2)
    px = (np.arange(nx) + 0.5) * dx
    py = (np.arange(ny) + 0.5) * dy
    P = np.stack(np.meshgrid(px, py, indexing="xy"), axis=-1).reshape(-1, 2)
    d2 = ((P[:, None, :] - seeds[None, :, :]) ** 2).sum(-1)
    nearest = np.argmin(d2, axis=1)
    d1 = d2[np.arange(P.shape[0]), nearest]
    # distance of each point to the bisector between its nearest seed and every other seed
    sep = np.linalg.norm(seeds[None, :, :] - seeds[nearest][:, None, :], axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        bis = (d2 - d1[:, None]) / (2.0 * sep)
    bis[np.arange(P.shape[0]), nearest] = np.inf
    edge = bis.min(axis=1)
    g = nearest.copy()
    g[edge < 0.5 * boundary] = -1
    # dense renumbering in order of first appearance
    out = np.full(g.shape, -1, dtype=np.int32)
    ids = {}
    for k, v in enumerate(g):
        if v >= 0:
            out[k] = ids.setdefault(int(v), len(ids))
    return out.reshape(ny, nx)


def columnar(grain2d, nz):
    """Per-site grain ids (x fastest, then y, then z) of columnar grains."""
    return np.ascontiguousarray(np.tile(grain2d.reshape(-1), nz).astype(np.int32))


def grain_diameters(grain2d, dx, dy):
    """Equivalent-circle diameters of the magnetic part of each grain [m]."""
    counts = np.bincount(grain2d[grain2d >= 0].ravel())
    return np.sqrt(4.0 * counts * dx * dy / math.pi)


def initial_state(n, kind="+z", seed=0, tilt_deg=10.0):
    """Unit spins, float64 [n, 3]: '+z' (all up), 'tilt' (polar angle uniform in
    [0, tilt_deg], random azimuth) or 'random' (uniform on the sphere)."""
    rng = np.random.default_rng(seed)
    S = np.zeros((n, 3))
    if kind == "+z":
        S[:, 2] = 1.0
    elif kind == "tilt":
        th = np.deg2rad(tilt_deg) * rng.uniform(size=n)
        ph = rng.uniform(0, 2 * np.pi, size=n)
        S[:] = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    elif kind == "random":
        v = rng.normal(size=(n, 3))
        S[:] = v / np.linalg.norm(v, axis=1, keepdims=True)
    else:
        raise ValueError(kind)
    return S


def mask_void(S, grain):
    """Zero the spins of non-magnetic sites (grain id < 0)."""
    S = np.array(S, dtype=np.float64, copy=True)
    S[np.asarray(grain).reshape(-1) < 0] = 0.0
    return S


def bits_of(pattern):
    return np.array([int(c) for c in pattern], dtype=np.uint8)


# ----------------------------------------------------------------------------- workloads
def sc_track_replica(nx, ny, nz, a=0.25e-9, grain_d=8e-9, boundary=1e-9, seed=11):
    """Granular simple-cubic track piece: dims and per-site grain ids."""
    g2 = voronoi_grains(nx, ny, a, a, grain_d, boundary, seed)
    return columnar(g2, nz), int(g2.max()) + 1


def ensemble_replicas(R=256, seed=13, side=(32, 96), layers=(8, 32), T=(500.0, 900.0),
                      a=0.25e-9, grain_d=8e-9, boundary=1e-9):
    """Batched ensemble of independent simple-cubic grain arrays of uneven size: per
    replica (nx, ny, nz), uniform temperature, grain map (list of int32 arrays), grain
    count and Philox seed."""
    rng = np.random.default_rng(seed)
    dims = np.stack([rng.integers(side[0], side[1] + 1, size=R),
                     rng.integers(side[0], side[1] + 1, size=R),
                     rng.integers(layers[0], layers[1] + 1, size=R)], axis=1).astype(np.int32)
    temps = rng.uniform(T[0], T[1], size=R)
    grains, ngr = [], []
    for r in range(R):
        g2 = voronoi_grains(int(dims[r, 0]), int(dims[r, 1]), a, a, grain_d, boundary,
                            seed * 100003 + r)
        grains.append(columnar(g2, int(dims[r, 2])))
        ngr.append(int(g2.max()) + 1)
    seeds = (np.uint64(seed) << np.uint64(32)) + np.arange(R, dtype=np.uint64)
    return dims, temps, grains, ngr, seeds


# ----------------------------------------------------------------------------- named workloads
J_SC = 6.7e-21           # nearest-neighbour exchange of the workloads [J]
KU_SC = 1.0e-22          # uniaxial anisotropy per atom of the SC workloads [J]
KU_L10 = 2.6e-22         # uniaxial anisotropy per atom of the L1_0 workload [J]
MU_S = 3 * MU_B          # atomic moment of all workloads [J/T]


def workload(name, **over):
    """Parameters of the named workloads.  A workload is a dict with the lattice kind,
    precision, per-replica dims/seeds/grains/drivers, the physical constants and the run
    length; `over` replaces top-level keys.

    sc32_pbc   plain FP64 SC 32x32x8, periodic x,y, open z, uniform 300 K, 1 T along -z,
               initial +z, 2000 steps, Philox seed 1, M every 10 steps;
    sc_track   granular SC track 256x256x32 at a = 0.25 nm (64x64x8 nm), 8 nm Voronoi grains
               with 1 nm boundaries, 50 nm FWHM laser 800 K peak over 300 K moving at 20 m/s,
               +/-0.8 T trapezoidal field with 20 nm bits, 1e5 steps of 0.1 fs, FP32;
    l10_window L1_0 Fe sublattice of the fct cell a = 0.385 nm, c = 0.371 nm over a
               60x100x10 nm window (220x367x27 sites), J1 = 6.7e-21 J, J2 = J1/2, J3 = J1/10,
               ku = 2.6e-22 J, 7 nm grains, laser and field as sc_track, FP32, on the
               implicit three-shell stencil (neighbours="csr" gives the list path);
    ensemble256 256 independent SC grain arrays, sides 32..96, 8..32 layers, uniform T in
               500..900 K, 0.8 T along -z, 8 nm grains, FP32, 1e5 steps.
    """
    a = 0.25e-9
    base = dict(lattice="sc", precision="fp32", neighbours="stencil", a=a, c=0.0,
                periodic=(False, False, False), mu_s=MU_S, ku=KU_SC, alpha=0.1, dt=1e-16,
                J=[J_SC], record_every=10)
    if name == "sc32_pbc":
        w = dict(base, precision="fp64", periodic=(True, True, False), steps=2000,
                 replicas=[dict(dims=(32, 32, 8), seed=1, grain=None, n_grains=1,
                                T=dict(T_amb=300.0), field=dict(B0=1.0, direction=(0, 0, -1)),
                                init="+z")])
    elif name == "sc_track":
        nx, ny, nz = 256, 256, 32
        g, ng = sc_track_replica(nx, ny, nz, a=a, grain_d=8e-9, boundary=1e-9, seed=11)
        w = dict(base, steps=100000, replicas=[dict(
            dims=(nx, ny, nz), seed=11, grain=g, n_grains=ng,
            T=dict(T_amb=300.0, T_peak=800.0, fwhm=50e-9, x0=nx * a / 2, y0=ny * a / 2, vx=20.0),
            field=dict(B0=0.8, direction=(0, 0, 1), bits=bits_of(PAPER_BIT_PATTERN), bit_len=20e-9,
                       ramp_len=2e-9, head_x0=nx * a / 2, head_v=20.0),
            init="+z")])
    elif name == "l10_window":
        la, lc = 0.385e-9, 0.371e-9
        ap = la / math.sqrt(2.0)
        nx, ny, nz = int(60e-9 / ap), int(100e-9 / ap), int(round(10e-9 / lc))
        g2 = voronoi_grains(nx, ny, ap, ap, 7e-9, 1e-9, 12)
        w = dict(base, lattice="l10", neighbours="stencil", a=la, c=lc, ku=KU_L10,
                 J=[J_SC, 0.5 * J_SC, 0.1 * J_SC], steps=100000, replicas=[dict(
                     dims=(nx, ny, nz), seed=12, grain=columnar(g2, nz), n_grains=int(g2.max()) + 1,
                     T=dict(T_amb=300.0, T_peak=800.0, fwhm=50e-9, x0=nx * ap / 2, y0=ny * ap / 2, vx=20.0),
                     field=dict(B0=0.8, direction=(0, 0, 1), bits=bits_of(PAPER_BIT_PATTERN),
                                bit_len=20e-9, ramp_len=2e-9, head_x0=nx * ap / 2, head_v=20.0),
                     init="+z")])
    elif name == "ensemble256":
        R = over.pop("R", 256)
        dims, temps, grains, ngr, seeds = ensemble_replicas(R=R, seed=13)
        w = dict(base, steps=100000, replicas=[dict(
            dims=tuple(int(v) for v in dims[r]), seed=int(seeds[r]), grain=grains[r], n_grains=ngr[r],
            T=dict(T_amb=float(temps[r])), field=dict(B0=0.8, direction=(0, 0, -1)), init="+z")
            for r in range(R)])
    else:
        raise KeyError(name)
    w.update(over)
    w["name"] = name
    return w


def multiscale_track(ncx=500, ncy=60, ncz=10, cell=1e-9, ratio=4, wx=60, grain_d=8e-9, boundary=1e-9, seed=14,
                     T_peak=800.0, v=20.0, x_spot=None):
    """The multiscale track: ncx x ncy x ncz micromagnetic cells of edge `cell` (by default
    500 x 60 x 10 nm at 1 nm) with an atomistic simple-cubic window of spacing cell / ratio
    (0.25 nm) wx cells long (60 nm: 240 x 240 x 40 sites) over the hot spot; Voronoi grains
    of mean diameter grain_d at cell resolution with `boundary`-wide non-magnetic borders;
    50 nm FWHM laser, T_peak over 300 K, moving at v; +/-0.8 T write field of 20 nm bits with
    the paper's pattern.  The micromagnetic constants are the atomistic ones per unit volume
    (Ms0 = mu_s / a^3, K0 = ku / a^3) and A0 = J / 2a; T_C = 1.443 J / kB.  Returns a dict
    of these inputs; cells start along +z."""
    a = cell / ratio
    g2 = voronoi_grains(ncx, ncy, cell, cell, grain_d, boundary, seed)
    grain = columnar(g2, ncz)
    xs = (wx / 2.0 + 1.0) * cell if x_spot is None else x_spot
    return dict(ncx=ncx, ncy=ncy, ncz=ncz, cell=cell, ratio=ratio, wx=wx, grain=grain,
                J=J_SC, mu_s=MU_S, ku=KU_SC, Ms0=MU_S / a ** 3, A0=J_SC / (2 * a), K0=KU_SC / a ** 3,
                lam=0.1, T_C=1.443 * J_SC / KB, dt=1e-16, seed=seed,
                T=dict(T_amb=300.0, T_peak=T_peak, fwhm=50e-9, x0=xs, y0=ncy * cell / 2, vx=v, vy=0.0),
                field=dict(B0=0.8, direction=(0.0, 0.0, 1.0), bits=bits_of(PAPER_BIT_PATTERN), bit_len=20e-9,
                           ramp_len=2e-9, head_x0=xs, head_v=v))
