"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 path 1e-9 on every spin component (spins are unit vectors, so this is
relative); FP32 path 2e-4 on every spin component over up to 1000 steps.  Both hold at
T = 0 and at T > 0 because the thermal field is drawn from the same Philox stream on both
sides; only rounding differs.
"""
import os

import numpy as np
import pytest

import oracle as orc
from common import gpu_lattice, initial, max_abs, oracle_for, oracle_params
from paper_2502_02236_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 2e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2502_02236_gb300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def run_both(w, n_steps, S0=None, precision=None, neighbours=None, record_every=0, tile=None):
    """Advance GPU and oracle by n_steps from the same state; returns per-replica
    (gpu spins, oracle spins, gpu records, oracle records)."""
    R = len(w["replicas"])
    S0 = S0 if S0 is not None else [initial(rep) for rep in w["replicas"]]
    lat = gpu_lattice(w, precision=precision, neighbours=neighbours, S0=S0)
    if tile:
        lat.set_tile(*tile)
    lat.sllg_heun_steps(n_steps, record_every)
    out = []
    for r in range(R):
        o = oracle_for(w, r)
        S = np.ascontiguousarray(S0[r], dtype=np.float64).copy()
        Mo = o.run(S, 0, n_steps, record_every)
        Mg, steps, _ = lat.read_magnetisation(r)
        out.append((lat.read_moments(r), S, Mg, Mo))
    lat.close()
    return out


def tiny_track(nx=45, ny=37, nz=9, seed=5, T=True, field=True, grains=True, a=0.25e-9):
    """A granular SC piece with a fast laser and a fast head so that both drivers change
    within a few hundred steps."""
    g2 = I.voronoi_grains(nx, ny, a, a, 3e-9, 0.5e-9, seed) if grains else np.zeros((ny, nx), np.int32)
    rep = dict(dims=(nx, ny, nz), seed=1000 + seed, grain=I.columnar(g2, nz), n_grains=int(g2.max()) + 1,
               init="tilt")
    if T:
        rep["T"] = dict(T_amb=300.0, T_peak=900.0, fwhm=6e-9, x0=2e-9, y0=nx * a / 3, vx=2e4, vy=1e3)
    if field:
        rep["field"] = dict(B0=2.0, direction=(0.1, 0.0, 1.0), bits=I.bits_of("0110100"), bit_len=0.3e-9,
                            ramp_len=0.05e-9, head_x0=-0.2e-9, head_v=2e4)
    return rep


def workload_of(reps, precision="fp32", **over):
    w = dict(lattice="sc", precision=precision, neighbours="stencil", a=0.25e-9, c=0.0,
             periodic=(False, False, False), mu_s=I.MU_S, ku=I.KU_SC, alpha=0.1, dt=1e-16, J=[I.J_SC],
             replicas=reps)
    w.update(over)
    return w


# --------------------------------------------------------------------------- FP64 plain path
def test_fp64_sc32_pbc_T0_tilt():
    w = I.workload("sc32_pbc")
    w["replicas"][0]["T"] = dict(T_amb=0.0)
    S0 = [I.initial_state(32 * 32 * 8, "tilt", seed=2, tilt_deg=30)]
    (g, o, Mg, Mo), = run_both(w, 200, S0=S0, record_every=10)
    assert max_abs(g, o) < TOL64
    assert Mg.shape == Mo.shape == (20, 3)
    assert max_abs(Mg, Mo) < TOL64


def test_fp64_sc32_pbc_workload():
    """The plain FP64 workload as specified: 32x32x8, 300 K, 1 T along -z, +z start, 2000
    steps, M every 10 steps."""
    w = I.workload("sc32_pbc")
    (g, o, Mg, Mo), = run_both(w, 2000, record_every=10)
    assert max_abs(g, o) < TOL64
    assert Mg.shape == (200, 3)
    assert max_abs(Mg, Mo) < TOL64


def test_fp64_granular_drivers():
    w = workload_of([tiny_track()], precision="fp64")
    (g, o, Mg, Mo), = run_both(w, 400, record_every=50)
    assert max_abs(g, o) < TOL64
    assert max_abs(Mg, Mo) < TOL64


# --------------------------------------------------------------------------- FP32 fused path
def test_fp32_sc32_pbc_T0_tilt_1000():
    w = I.workload("sc32_pbc", precision="fp32")
    w["replicas"][0]["T"] = dict(T_amb=0.0)
    S0 = [I.initial_state(32 * 32 * 8, "tilt", seed=2, tilt_deg=30)]
    (g, o, Mg, Mo), = run_both(w, 1000, S0=S0, record_every=100)
    assert max_abs(g, o) < TOL32
    assert max_abs(Mg, Mo) < TOL32


def test_fp32_sc32_pbc_thermal_1000():
    w = I.workload("sc32_pbc", precision="fp32")
    (g, o, Mg, Mo), = run_both(w, 1000, record_every=10)
    assert max_abs(g, o) < TOL32
    assert max_abs(Mg, Mo) < TOL32


TILES = [(512, 36 * 24), (1024, 68 * 24), (256, 36 * 14), (256, 36 * 24)]


@pytest.mark.parametrize("tile", TILES)
def test_fp32_granular_drivers_every_tile(tile):
    w = workload_of([tiny_track()])
    (g, o, Mg, Mo), = run_both(w, 500, record_every=100, tile=tile)
    assert max_abs(g, o) < TOL32
    assert max_abs(Mg, Mo) < TOL32


@pytest.mark.parametrize("lattice,periodic", [("sc", (False, False, False)), ("sc", (True, False, True)),
                                              ("l10", (False, False, True)), ("l10", (False, True, False))])
def test_plane_ranges_bitwise_equal_to_whole_columns(lattice, periodic):
    """Work items over plane ranges (the split used when a batch has too few column blocks for
    the GPU) give bitwise the spins and records of whole-column items: the predictor on a
    range's boundary planes recomputes the neighbouring range's S' with the same noise.  The
    work model splits this small batch by itself."""
    reps = [tiny_track(45, 37, 13, seed=5), tiny_track(23, 30, 9, seed=7),
            dict(dims=(40, 30, 7), seed=8, init="random", T=dict(T_amb=700.0), field=dict(B0=0.8, direction=(0, 0, -1)))]
    if lattice == "sc":
        w = workload_of(reps, periodic=periodic)
    else:
        w = dict(lattice="l10", precision="fp32", neighbours="stencil", a=0.385e-9, c=0.371e-9, periodic=periodic,
                 mu_s=I.MU_S, ku=I.KU_L10, alpha=0.1, dt=1e-16, J=[I.J_SC, 0.5 * I.J_SC, 0.1 * I.J_SC], replicas=reps)
    S0 = [initial(rep) for rep in reps]
    got = {}
    for planes in (0, 13, 4, 5):
        lat = gpu_lattice(w, S0=S0)
        lat.set_plane_range(planes)
        used = lat.query(6)
        assert used == (planes or used) and 4 <= used <= 13, (planes, used)
        if planes == 0:
            assert used < 13 and lat.query(5) > 2 * 3   # split by the work model
        lat.sllg_heun_steps(41, 20)
        got[planes] = ([lat.read_moments(r) for r in range(len(reps))],
                       [lat.read_magnetisation(r)[0] for r in range(len(reps))])
        lat.close()
    for planes in (0, 4, 5):
        for r in range(len(reps)):
            assert np.array_equal(got[planes][0][r], got[13][0][r]), (planes, r)
            assert np.array_equal(got[planes][1][r], got[13][1][r]), (planes, r)
    o = oracle_for(w, 1)
    S = S0[1].copy()
    o.run(S, 0, 41, 0)
    assert max_abs(got[0][0][1], S) < TOL32


def uneven_replicas():
    """Uneven batch: a single spin, thin slabs, a ragged granular piece, a replica with no
    magnetic site, and one with adjacent different grains (bonds that must be cut)."""
    reps = [
        dict(dims=(1, 1, 1), seed=11, init="tilt", T=dict(T_amb=500.0), field=dict(B0=1.0, direction=(0, 0, -1))),
        dict(dims=(3, 70, 5), seed=12, init="random", T=dict(T_amb=700.0)),
        dict(dims=(33, 2, 17), seed=13, init="tilt", T=dict(T_amb=100.0), field=dict(B0=0.5, direction=(1, 0, 0))),
        tiny_track(40, 29, 8, seed=7),
        dict(dims=(5, 4, 3), seed=15, grain=np.full(60, -1, np.int32), n_grains=0, init="+z"),
    ]
    g = np.zeros((9, 10), np.int32)
    g[:, 5:] = 1
    reps.append(dict(dims=(10, 9, 4), seed=16, grain=I.columnar(g, 4), n_grains=2, init="random",
                     T=dict(T_amb=400.0)))
    return reps


def test_fp32_batched_uneven():
    w = workload_of(uneven_replicas())
    for r, (g, o, Mg, Mo) in enumerate(run_both(w, 300, record_every=30)):
        assert max_abs(g, o) < TOL32, r
        assert max_abs(Mg, Mo) < TOL32, r


def test_fp64_batched_uneven():
    w = workload_of(uneven_replicas(), precision="fp64")
    for r, (g, o, Mg, Mo) in enumerate(run_both(w, 300, record_every=30)):
        assert max_abs(g, o) < TOL64, r
        assert max_abs(Mg, Mo) < TOL64, r


@pytest.mark.parametrize("periodic", [(False, False, False), (True, True, False), (True, False, True)])
def test_fp32_multi_tile_splits(periodic):
    """Replicas wider than one column block in x and y, open and periodic, so that halos
    between blocks and across periodic edges are exercised."""
    reps = [tiny_track(150, 140, 6, seed=31), tiny_track(70, 66, 5, seed=32, grains=False),
            dict(dims=(97, 3, 4), seed=33, init="random", T=dict(T_amb=600.0))]
    w = workload_of(reps, periodic=periodic)
    for r, (g, o, Mg, Mo) in enumerate(run_both(w, 120, record_every=40)):
        assert max_abs(g, o) < TOL32, r
        assert max_abs(Mg, Mo) < TOL32, r


def test_fp32_non_columnar_grains():
    """Grains that change along z, touching grains (bonds cut by the grain mask) and scattered
    non-magnetic sites."""
    nx, ny, nz = 37, 29, 11
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    g = ((x // 9 + y // 7 + z // 3) % 4).transpose(2, 1, 0).reshape(-1).astype(np.int32)
    rng = np.random.default_rng(5)
    g[rng.uniform(size=g.size) < 0.1] = -1
    rep = dict(dims=(nx, ny, nz), seed=41, grain=g, n_grains=4, init="random",
               T=dict(T_amb=350.0, T_peak=700.0, fwhm=4e-9, x0=4e-9, y0=3e-9, vx=1e4))
    for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
        w = workload_of([rep], precision=prec)
        (gg, o, Mg, Mo), = run_both(w, 150, record_every=50)
        assert max_abs(gg, o) < tol, prec
        assert max_abs(Mg, Mo) < tol, prec


@pytest.mark.parametrize("tile", TILES)
def test_fp32_many_items_per_cta(tile):
    """More column blocks than resident CTAs, so that every persistent CTA runs several work
    items in a row (open edges: TMA staging), mixed with a replica that needs the exchange mask
    (per-position staging) in the same launch."""
    rng = np.random.default_rng(9)
    reps = []
    for r in range(200):
        nx, ny, nz = (int(v) for v in rng.integers([10, 10, 2], [23, 23, 7]))
        reps.append(dict(dims=(nx, ny, nz), seed=500 + r, init="random", T=dict(T_amb=float(rng.uniform(100, 900))),
                         field=dict(B0=0.7, direction=(0, 0, -1))))
    g = np.zeros((12, 14), np.int32)
    g[:, 7:] = 1
    reps.append(dict(dims=(14, 12, 3), seed=777, grain=I.columnar(g, 3), n_grains=2, init="random",
                     T=dict(T_amb=300.0)))
    w = workload_of(reps)
    for r, (gg, o, Mg, Mo) in enumerate(run_both(w, 40, record_every=20, tile=tile)):
        assert max_abs(gg, o) < TOL32, r
        assert max_abs(Mg, Mo) < TOL32, r


def test_periodic_tiny_lattices_both_precisions():
    """Periodic lattices smaller than a tile, down to 1 x 1 x 1 (a site is its own neighbour)."""
    reps = [dict(dims=d, seed=20 + k, init="random", T=dict(T_amb=300.0), field=dict(B0=1.0, direction=(0, 0, 1)))
            for k, d in enumerate([(1, 1, 1), (2, 2, 2), (3, 1, 2), (2, 5, 1), (7, 3, 3)])]
    for prec, tol in (("fp64", TOL64), ("fp32", TOL32)):
        w = workload_of(reps, precision=prec, periodic=(True, True, True))
        for r, (g, o, Mg, Mo) in enumerate(run_both(w, 200, record_every=20)):
            assert max_abs(g, o) < tol, (prec, r)


# --------------------------------------------------------------------------- neighbour lists
def l10_piece(nx=24, ny=20, nz=6, seed=3):
    la, lc = 0.385e-9, 0.371e-9
    ap = la / np.sqrt(2)
    g2 = I.voronoi_grains(nx, ny, ap, ap, 3e-9, 0.5e-9, seed)
    rep = dict(dims=(nx, ny, nz), seed=300 + seed, grain=I.columnar(g2, nz), n_grains=int(g2.max()) + 1,
               init="tilt", T=dict(T_amb=400.0, T_peak=800.0, fwhm=4e-9, x0=3e-9, y0=3e-9, vx=1e4),
               field=dict(B0=1.0, direction=(0, 0, -1)))
    return dict(lattice="l10", precision="fp64", neighbours="csr", a=la, c=lc, periodic=(False, True, False),
                mu_s=I.MU_S, ku=I.KU_L10, alpha=0.1, dt=1e-16, J=[I.J_SC, 0.5 * I.J_SC, 0.1 * I.J_SC],
                replicas=[rep])


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_l10_three_shells(prec, tol):
    w = l10_piece()
    (g, o, Mg, Mo), = run_both(w, 300, precision=prec, record_every=50)
    assert max_abs(g, o) < tol
    assert max_abs(Mg, Mo) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_l10_stencil_three_shells(prec, tol):
    """The implicit L1_0 stencil (the fused kernel in FP32, the two-pass path in FP64)
    against the oracle's geometric shells: granular, laser, field, periodic in y."""
    w = l10_piece(30, 26, 7, seed=5)
    (g, o, Mg, Mo), = run_both(w, 300, precision=prec, neighbours="stencil", record_every=50)
    assert max_abs(g, o) < tol
    assert max_abs(Mg, Mo) < tol


@pytest.mark.parametrize("tile", TILES + ["fp64"])
def test_l10_stencil_every_tile_touching_grains(tile):
    """The fused L1_0 kernel in every compiled shape (and the FP64 two-pass stencil), open and
    fully periodic lattices, with grains that touch (no boundary layer, so the exchange mask
    decides every bond)."""
    prec, tol = ("fp64", TOL64) if tile == "fp64" else ("fp32", TOL32)
    for periodic in ((False, False, False), (True, True, True)):
        la, lc = 0.385e-9, 0.371e-9
        ap = la / np.sqrt(2)
        g2 = I.voronoi_grains(40, 34, ap, ap, 2.5e-9, 0.0, 8)
        rep = dict(dims=(40, 34, 5), seed=77, grain=I.columnar(g2, 5), n_grains=int(g2.max()) + 1, init="random",
                   T=dict(T_amb=500.0), field=dict(B0=0.5, direction=(0.3, 0, -1)))
        w = dict(lattice="l10", precision=prec, neighbours="stencil", a=la, c=lc, periodic=periodic,
                 mu_s=I.MU_S, ku=I.KU_L10, alpha=0.1, dt=1e-16, J=[I.J_SC, 0.5 * I.J_SC, 0.1 * I.J_SC],
                 replicas=[rep])
        (g, o, _, _), = run_both(w, 60, tile=None if tile == "fp64" else tile)
        assert max_abs(g, o) < tol, (tile, periodic)


def test_l10_list_matches_stencil():
    w = l10_piece(22, 18, 5, seed=6)
    (gs, o, _, _), = run_both(w, 100, neighbours="stencil")
    (gc, _, _, _), = run_both(w, 100, neighbours="csr")
    assert max_abs(gs, gc) < 1e-12
    assert max_abs(gc, o) < TOL64


def test_sc_list_matches_stencil():
    w = workload_of([tiny_track(31, 22, 7, seed=9)], precision="fp64", periodic=(True, False, True))
    (gs, o, _, _), = run_both(w, 100)
    (gc, _, _, _), = run_both(w, 100, neighbours="csr")
    assert max_abs(gs, gc) < 1e-12
    assert max_abs(gc, o) < TOL64


def test_external_list_same_as_built():
    """A list given through hamr_set_csr (here the geometric bond list) gives the same
    trajectory as the list the library builds."""
    w = l10_piece(12, 10, 4)
    rep = w["replicas"][0]
    o = oracle_for(w, 0)
    rp, col, sh = o.neighbours()
    S0 = [initial(rep)]
    ref = gpu_lattice(w, S0=S0)
    ref.sllg_heun_steps(100)
    lat = gpu_lattice(w, S0=S0)
    lat.set_csr(0, rp.astype(np.int32), col.astype(np.int32), sh.astype(np.uint8))
    lat.set_moments(0, S0[0])
    lat.sllg_heun_steps(100)
    assert max_abs(lat.read_moments(0), ref.read_moments(0)) < 1e-12


# --------------------------------------------------------------------------- reductions, energy
@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_grain_averages_and_energy(prec, tol):
    rep = tiny_track(48, 40, 6, seed=4)
    w = workload_of([rep], precision=prec)
    S0 = [initial(rep)]
    lat = gpu_lattice(w, S0=S0)
    lat.sllg_heun_steps(120, 40)
    o = oracle_for(w, 0)
    S = S0[0].copy()
    o.run(S, 0, 120)
    M, steps, Mg = lat.read_magnetisation(0, rep["n_grains"])
    assert list(steps) == [40, 80, 120]
    sums, counts = o.grain_sums(S, rep["n_grains"])
    want = np.where(counts[:, None] > 0, sums / np.maximum(counts[:, None], 1), 0.0)
    assert max_abs(Mg, want) < tol
    assert max_abs(M[-1], o.magnetisation(S)) < tol
    E = lat.read_energy(0)
    Eo = o.energy(S, 120)
    assert abs(E - Eo) <= (1e-9 if prec == "fp64" else 2e-4) * abs(Eo)


def test_fp32_grain_records_batched_and_after_grain_change():
    """Per-grain record sums of the FP32 fused path over a batch: granular replicas, one
    replica of a single grain (rows of 70 sites, so runs of 32, 32 and 6 slots, and one grain
    spanning many warp items), then again after one replica's grain map changes between record
    points (the runs are rebuilt)."""
    reps = [tiny_track(48, 40, 6, seed=4), tiny_track(70, 33, 4, seed=6, grains=False), tiny_track(45, 37, 5, seed=8)]
    w = workload_of(reps)
    S = [initial(rep) for rep in reps]
    lat = gpu_lattice(w, S0=S)

    def check(step0, n):
        for r, rep in enumerate(w["replicas"]):
            o = oracle_for(w, r)
            o.run(S[r], step0, n)
            M, steps, Mg = lat.read_magnetisation(r, rep["n_grains"])
            assert steps[-1] == step0 + n
            sums, counts = o.grain_sums(S[r], rep["n_grains"])
            want = np.where(counts[:, None] > 0, sums / np.maximum(counts[:, None], 1), 0.0)
            assert max_abs(Mg, want) < TOL32, (r, max_abs(Mg, want))
            assert max_abs(M[-1], o.magnetisation(S[r])) < TOL32

    lat.sllg_heun_steps(40, 20)
    check(0, 40)
    a = w["a"]
    g2 = I.voronoi_grains(45, 37, a, a, 4e-9, 0.5e-9, 99)
    grain = I.columnar(g2, 5)
    w["replicas"][2] = dict(reps[2], grain=grain, n_grains=int(g2.max()) + 1)
    lat.set_grain_map(2, grain, int(g2.max()) + 1)
    # sites that turn magnetic had no spin: give them +z on both sides
    S2 = S[2].reshape(-1, 3).copy()
    S2[np.all(S2 == 0.0, axis=1)] = (0.0, 0.0, 1.0)
    S[2] = np.ascontiguousarray(I.mask_void(S2, grain).reshape(S[2].shape))
    lat.set_moments(2, S[2])
    lat.sllg_heun_steps(40, 20)
    check(40, 40)


# --------------------------------------------------------------------------- state handling
def test_checkpoint_resume_bitwise(tmp_path):
    w = workload_of(uneven_replicas()[:4])
    lat = gpu_lattice(w)
    lat.sllg_heun_steps(60, 20)
    path = str(tmp_path / "state.bin")
    lat.save_state(path)
    lat.sllg_heun_steps(45, 0)
    want = [lat.read_moments(r) for r in range(4)]
    assert lat.step == 105
    other = gpu_lattice(w)
    other.load_state(path)
    assert other.step == 60
    other.sllg_heun_steps(20, 0)
    other.sllg_heun_steps(25, 7)       # split differently, with records on the way
    for r in range(4):
        assert np.array_equal(other.read_moments(r), want[r])


def test_autotune_keeps_state():
    w = workload_of(uneven_replicas())
    lat = gpu_lattice(w)
    lat.sllg_heun_steps(10)
    before = [lat.read_moments(r) for r in range(len(w["replicas"]))]
    tile = lat.autotune(3)
    assert lat.step == 10
    assert tile in TILES
    for r, b in enumerate(before):
        assert np.array_equal(lat.read_moments(r), b)


def test_finite_check_flags_injected_nan():
    w = workload_of([dict(dims=(8, 8, 4), seed=1, init="+z")])
    lat = gpu_lattice(w)
    assert lat.check_finite()
    S = initial(w["replicas"][0])
    S[17, 1] = np.nan
    lat.set_moments(0, S)
    assert not lat.check_finite()


def test_device_pointer_roundtrip():
    import torch
    w = workload_of([tiny_track(20, 18, 5, seed=8)], precision="fp64")
    rep = w["replicas"][0]
    lat = gpu_lattice(w)
    S0 = initial(rep, "random", seed=3)
    t = torch.from_numpy(S0).cuda()
    lat.set_moments_device(0, t)
    out = torch.empty_like(t)
    lat.read_moments_device(0, out)
    torch.cuda.synchronize()
    want = I.mask_void(S0, rep["grain"])
    assert np.array_equal(out.cpu().numpy(), want)


# --------------------------------------------------------------------------- full sizes, sampled
def sample_sites(w, r, k, seed):
    rep = w["replicas"][r]
    n = int(np.prod(rep["dims"]))
    rng = np.random.default_rng(seed)
    nx, ny, nz = rep["dims"]
    edges = [0, nx - 1, nx * (ny - 1), n - 1, n // 2]
    return np.unique(np.concatenate([rng.integers(0, n, size=k), edges]))


@pytest.mark.parametrize("name", ["sc_track", "l10_window"])
def test_full_size_one_step_sampled(name):
    """One step of the full-size workload, compared at sampled sites that the oracle
    computes one by one from the same pre-step state."""
    w = I.workload(name)
    S0 = [initial(rep) for rep in w["replicas"]]
    lat = gpu_lattice(w, S0=S0)
    lat.sllg_heun_steps(1, 1)
    g = lat.read_moments(0)
    sites = sample_sites(w, 0, 3000, 1)
    want = orc.step_sites(oracle_params(w, 0), w["replicas"][0]["grain"], S0[0], 0, sites)
    assert max_abs(g[sites], want) < TOL32
    assert np.abs(g[sites] - S0[0][sites]).max() > 1e-3     # the step did move the spins


def test_full_size_ensemble_sampled():
    """The batched 256-replica workload in its benchmark launch configuration: one step,
    sampled sites of every replica against the oracle."""
    w = I.workload("ensemble256")
    S0 = [initial(rep) for rep in w["replicas"]]
    lat = gpu_lattice(w, S0=S0)
    lat.autotune(2)
    lat.sllg_heun_steps(1, 1)
    worst = 0.0
    for r in range(len(w["replicas"])):
        sites = sample_sites(w, r, 40, r)
        want = orc.step_sites(oracle_params(w, r), w["replicas"][r]["grain"], S0[r], 0, sites)
        worst = max(worst, max_abs(lat.read_moments(r)[sites], want))
    assert worst < TOL32


# --------------------------------------------------------------------------- degenerate inputs
@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_all_void_replica_zero_steps_and_ragged_batch(prec, tol):
    """A batch holding a replica with no magnetic site at all and a 1-site-thick one: zero
    steps change nothing; after steps the void replica stays zero with M = 0, and the others
    match the oracle."""
    reps = uneven_replicas()[:3]
    void = dict(dims=(9, 7, 3), seed=5, grain=np.full(9 * 7 * 3, -1, dtype=np.int32), n_grains=1, init="random",
                T=dict(T_amb=300.0))
    thin = dict(dims=(13, 1, 1), seed=6, init="random", T=dict(T_amb=300.0), field=dict(B0=1.0, direction=(0, 0, 1)))
    reps = [void] + reps + [thin]
    w = workload_of(reps, precision=prec)
    S0 = [initial(rep) for rep in reps]
    lat = gpu_lattice(w, S0=S0)
    lat.sllg_heun_steps(0, 5)
    for r in range(len(reps)):
        assert np.array_equal(lat.read_moments(r), S0[r].astype(np.float32).astype(np.float64)
                              if prec == "fp32" else S0[r])
    lat.close()
    outs = run_both(w, 40, S0=S0, record_every=20)
    g, o, Mg, Mo = outs[0]
    assert not np.any(g) and not np.any(o)           # void: nothing to move
    assert np.array_equal(Mg, np.zeros((2, 3)))      # M of a replica without magnetic sites
    for r, (g, o, Mg, Mo) in enumerate(outs[1:], 1):
        assert max_abs(g, o) < tol, r
        assert max_abs(Mg, Mo) < tol, r


def test_call_order_and_list_checks():
    """Stepping before the exchange shells are set is a STATE error; a neighbour list whose
    bonds have no partner is rejected with ARG and leaves the handle usable."""
    from paper_2502_02236_gb300 import hamr
    rep = tiny_track(12, 10, 4, seed=3)
    w = workload_of([rep], precision="fp64", neighbours="csr")
    lat = gpu_lattice(w)
    o = oracle_for(w, 0)
    rp, col, sh = o.neighbours()
    bad = sh.astype(np.uint8).copy()
    bad[0] = (bad[0] + 1) % 2                       # one bond in another shell than its partner
    with pytest.raises(hamr.HamrError) as e:
        lat.set_csr(0, rp.astype(np.int32), col.astype(np.int32), bad)
    assert e.value.code == hamr.ERR_ARG
    lat.set_csr(0, rp.astype(np.int32), col.astype(np.int32), sh.astype(np.uint8))
    lat.sllg_heun_steps(5)
    lat.close()
    from paper_2502_02236_gb300.hamr import Lattice
    with Lattice([(8, 8, 2)], [1], precision="fp32", a=0.25e-9, mu_s=I.MU_S, ku=I.KU_SC, alpha=0.1, dt=1e-16) as fresh:
        with pytest.raises(hamr.HamrError) as e:
            fresh.sllg_heun_steps(1)
        assert e.value.code == hamr.ERR_STATE
