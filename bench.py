#!/usr/bin/env python
"""Throughput of the stochastic-LLG Heun step on one node: atomistic spin-steps/s.

Default workload: the batched ensemble of 256 independent simple-cubic grain arrays of
uneven size (sides 32..96, 8..32 layers, ~2.1e7 sites in total), FP32 state with FP64
reductions, M(t) recorded every 10 steps, advanced by the fused persistent kernel.  A step
is one Heun step of every replica.  Beside it: the plain FP64 GPU path on the same workload,
the end-to-end rate through the C ABI with host buffers, and the FP64 CPU oracle on a
bounded sample of the same workload (the CPU baseline).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own ensemble (seeds offset by rank, no collective on the
data path): weak scaling.  Rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_SITE_FP32 = 26   # read S 12 B + write S 12 B + 2-byte grain code
BYTES_PER_SITE_FP64 = 50   # read S 24 B + write S 24 B + 2-byte grain code
METRIC = "atomistic spin-steps/s (FP32 batched vs FP64 plain, same GB300)"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--warmup", type=int, default=50)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="ensemble256")
    p.add_argument("--fp64-steps", type=int, default=30)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-ms", action="store_true", help="skip the multiscale-track line")
    p.add_argument("--ms-steps", type=int, default=20)
    p.add_argument("--ms-margin", type=int, default=-1,
                   help="multiscale_track: evolve only the window and this many cell columns on each side")
    p.add_argument("--ms-ncx", type=int, default=500, help="multiscale_track: track length in cells")
    p.add_argument("--ms-demag", action="store_true",
                   help="with --workload multiscale_track: the demagnetising field on")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--tile", default=None, help="fused-kernel shape THREADSxSTAGED instead of autotuning")
    p.add_argument("--planes", type=int, default=0,
                   help="planes per work item of the fused kernel (0: the library's work model)")
    return p.parse_args()


# ----------------------------------------------------------------------------- distributed
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v):
        if not self.pg:
            return v
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([float(v)], device=dev, dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[4]) for r in rows if r[4].replace(".", "").isdigit()]
        load = [s for s, p in zip(sm, pw)] if sm else []
        # samples under load: power above the midpoint of the observed range
        if pw:
            cut = min(pw) + 0.5 * (max(pw) - min(pw))
            load = [s for s, p in zip(sm, pw) if p >= cut] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "samples_under_load": len(load),
                "reasons": reasons}


# ----------------------------------------------------------------------------- helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_sources_sha256():
    """Hash of the fused kernel's sources (the template, its simple-cubic instantiation and
    the device helpers it includes)."""
    h = hashlib.sha256()
    for f in ("kernels_fused.cuh", "kernels_fused_sc.cu", "device_common.cuh"):
        with open(os.path.join(ROOT, "paper_2502_02236_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kernel_counters():
    """DRAM bytes and warp instructions per fused launch from the committed ncu summary, if
    it was taken on the kernel sources as they are now (else None)."""
    path = os.path.join(ROOT, "profiles", "fused_ensemble256_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        if t.get("kernel_sha256") == kernel_sources_sha256():
            return t
    except (OSError, ValueError):
        pass
    return None


def issue_roof(warp_inst, avg_launch_ms, sm_mhz):
    """The instruction-issue roof of a launch: its warp instructions over every SM's four
    schedulers issuing one instruction per cycle at the sampled SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    if not warp_inst or not sm_mhz:
        return None
    roof_ms = warp_inst / (sms * 4 * sm_mhz * 1e6) * 1e3
    return {"warp_inst_per_launch": warp_inst, "sms": sms, "issue_per_clk": 4 * sms, "sm_mhz": sm_mhz,
            "roof_ms": roof_ms, "frac": roof_ms / avg_launch_ms}


def oracle_error(lat, w, reps, n_per=40):
    """Largest |S_gpu - S_oracle| over sampled sites of the given replicas after one step of the
    handle from its current state; the FP64 oracle steps each sampled site from the same
    pre-step state (edges and random sites of every replica)."""
    import oracle as orc
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from common import oracle_params
    S0 = {r: lat.read_moments(r) for r in reps}
    step = lat.step
    lat.sllg_heun_steps(1, 0)
    worst, count = 0.0, 0
    for r in reps:
        rep = w["replicas"][r]
        nx, ny, nz = rep["dims"]
        n = nx * ny * nz
        rng = np.random.default_rng(r)
        sites = np.unique(np.concatenate([rng.integers(0, n, size=n_per), [0, nx - 1, nx * (ny - 1), n - 1]]))
        want = orc.step_sites(oracle_params(w, r), rep.get("grain"), S0[r], step, sites)
        worst = max(worst, float(np.abs(lat.read_moments(r)[sites] - want).max()))
        count += len(sites)
    return {"max_abs_spin": worst, "sites": count, "replicas": len(reps),
            "what": "one step from the handle's state, every sampled site against the FP64 oracle"}


def l2_note(n_sites):
    import torch
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    mb = 12 * n_sites / 1e6
    if 12 * n_sites > l2:
        return "inputs larger than L2 (two %.0f MB FP32 state buffers, L2 %.0f MB); no flush" % (mb, l2 / 1e6)
    return "state fits in L2 (two %.0f MB FP32 buffers, L2 %.0f MB): L2-resident, not flushed" % (mb, l2 / 1e6)


def rank_seeds(reps, rank):
    """Philox keys of one rank's replicas: each rank runs its own ensemble (the workload's
    seeds with the rank in the top 16 bits), so ranks share no random stream."""
    return [int(rep["seed"]) ^ (rank << 48) for rep in reps]


def aggregate(n_sites, steps, world, ms):
    """Whole-job spin-steps/s: every rank advanced n_sites sites by `steps` steps, and the
    job took the slowest rank's time `ms`."""
    return n_sites * steps * world / (ms / 1e3)


def build_lattice(w, precision, rank=0):
    from paper_2502_02236_gb300.hamr import Lattice
    reps = w["replicas"]
    seeds = rank_seeds(reps, rank)
    lat = Lattice([rep["dims"] for rep in reps], seeds, lattice=w["lattice"], precision=precision,
                  neighbours=w["neighbours"], a=w["a"], c=w["c"], periodic=w["periodic"], mu_s=w["mu_s"],
                  ku=w["ku"], alpha=w["alpha"], dt=w["dt"])
    lat.set_neighbour_shells(w["J"])
    for r, rep in enumerate(reps):
        if rep.get("grain") is not None:
            lat.set_grain_map(r, rep["grain"], rep["n_grains"])
        if rep.get("T"):
            lat.set_temperature_profile(r, **rep["T"])
        if rep.get("field"):
            lat.set_field_sequence(r, **rep["field"])
    return lat


def prime(lat, K, record_every):
    """Capture, untimed, the CUDA graphs of every block size that a timed call of K steps
    will replay, and leave the step count aligned to record_every."""
    if record_every > 0:
        r = K % record_every
        if r:
            lat.sllg_heun_steps(r, record_every)
            lat.sllg_heun_steps(record_every - r, record_every)
    else:
        lat.sllg_heun_steps(64 + K % 64, 0)


def timed(lat, dist, K, record_every):
    import torch
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    lat.sllg_heun_steps_async(K, record_every)
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    lat.synchronize()
    return e0.elapsed_time(e1)


def cpu_baseline(w, seconds):
    """The FP64 oracle as it stands on this host's cores (OpenMP over sites, all cores), over a
    bounded sample of the workload: the first replicas, whose oracle contexts (neighbour lists)
    are built before timing, stepped together until about `seconds` have passed."""
    import oracle as orc
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from common import initial, oracle_params
    reps, n = [], 0
    for r, rep in enumerate(w["replicas"]):
        reps.append(r)
        n += int(np.prod(rep["dims"]))
        if n >= 300000:
            break
    orcs = [orc.Oracle(oracle_params(w, r), w["replicas"][r].get("grain")) for r in reps]
    S = [initial(w["replicas"][r]) for r in reps]
    for o, s in zip(orcs, S):  # one untimed step
        o.step(s, 0)
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for o, s in zip(orcs, S):
            o.step(s, 1 + steps)
        steps += 1
    el = time.perf_counter() - t0
    return n * steps / el, reps, n, steps, el


def cpu_baseline_one_core(workload, seconds):
    """The same oracle timing on one host core (OpenMP limited to one thread in a child
    process); None if the child fails."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; from paper_2502_02236_gb300 import inputs as I; "
            "v, reps, n, steps, el = bench.cpu_baseline(I.workload(%r), %r); "
            "print(json.dumps({'value': v, 'unit': 'spin-steps/s', 'cores': 1, "
            "'sample': 'replicas 0..%%d (%%d sites), %%d steps in %%.1f s' %% (reps[-1], n, steps, el)}))"
            % (ROOT, workload, float(seconds)))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        return json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        return None


def ms_rate(w, precision, K, dist, demag=False, margin=-1):
    """ms per coupled step of the multiscale track w from +z cells, the window following the
    spot (CUDA events on the library's stream, max over ranks), after 3 untimed steps."""
    import torch
    from paper_2502_02236_gb300.hamr import Multiscale
    G = Multiscale(w["ncx"], w["ncy"], w["ncz"], w["cell"], w["ratio"], w["wx"], J=w["J"], mu_s=w["mu_s"],
                   ku=w["ku"], Ms0=w["Ms0"], A0=w["A0"], K0=w["K0"], lam=w["lam"], T_C=w["T_C"], dt=w["dt"],
                   seed=w["seed"] ^ (dist.rank << 48), precision=precision)
    G.set_grain_map(w["grain"])
    G.set_temperature_profile(**w["T"])
    G.set_field_sequence(**w["field"])
    m = np.zeros((w["ncx"] * w["ncy"] * w["ncz"], 3))
    m[:, 2] = 1.0
    G.set_cells(m)
    G.set_region(margin)
    G.set_window(int(np.floor(w["T"]["x0"] / w["cell"] - w["wx"] / 2 + 0.5)))
    if demag:
        G.set_demag(True)
    G.steps(3, follow=True)
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    G.steps(K, follow=True)
    e1.record()
    torch.cuda.synchronize()
    ms = dist.max(e0.elapsed_time(e1))
    G.close()
    return ms / K


def multiscale_line(args, dist):
    """The full multiscale track (500 x 60 x 10 nm of 1 nm micromagnetic cells with a 60 nm
    atomistic window of 240 x 240 x 40 sites at 0.25 nm, window following the laser), FP32
    with the FP64 rate beside it: coupled steps per second, as atomistic spin-steps/s of the
    window and cell-steps/s of the track, timed with CUDA events on the library's stream;
    beside them the FP64 oracle's coupled step on the host cores (rank 0, one process only)."""
    import torch
    from paper_2502_02236_gb300 import inputs as I
    from paper_2502_02236_gb300.hamr import Multiscale
    w = I.multiscale_track()
    m = np.zeros((w["ncx"] * w["ncy"] * w["ncz"], 3))
    m[:, 2] = 1.0
    ox = int(np.floor(w["T"]["x0"] / w["cell"] - w["wx"] / 2 + 0.5))

    def make(precision):
        G = Multiscale(w["ncx"], w["ncy"], w["ncz"], w["cell"], w["ratio"], w["wx"], J=w["J"], mu_s=w["mu_s"],
                       ku=w["ku"], Ms0=w["Ms0"], A0=w["A0"], K0=w["K0"], lam=w["lam"], T_C=w["T_C"], dt=w["dt"],
                       seed=w["seed"] ^ (dist.rank << 48), precision=precision)
        G.set_grain_map(w["grain"])
        G.set_temperature_profile(**w["T"])
        G.set_field_sequence(**w["field"])
        return G

    def rate(precision, K, demag=False):
        G = make(precision)
        G.set_cells(m)
        G.set_window(ox)
        if demag:
            G.set_demag(True)
        G.steps(3, follow=True)
        dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        G.steps(K, follow=True)
        e1.record()
        torch.cuda.synchronize()
        ms = dist.max(e0.elapsed_time(e1))
        G.close()
        return ms / K, G.n_window, G.n_cells

    K = max(1, args.ms_steps)
    t32, nw, nc = rate("fp32", 5 * K)
    t64, _, _ = rate("fp64", K)
    t32d, _, _ = rate("fp32", K, demag=True)
    line = {"workload": "multiscale_track", "dtype": "f32", "window_sites": nw, "cells": nc, "steps": 5 * K,
            "ms_per_step": t32, "window_spin_steps_per_s": nw * dist.world / (t32 / 1e3),
            "cell_steps_per_s": nc * dist.world / (t32 / 1e3),
            "fp64": {"ms_per_step": t64, "window_spin_steps_per_s": nw * dist.world / (t64 / 1e3), "steps": K},
            "speedup_fp32_over_fp64": t64 / t32,
            "fp32_with_demag": {"ms_per_step": t32d, "window_spin_steps_per_s": nw * dist.world / (t32d / 1e3),
                                "steps": K, "note": "Eq. 7: in-plane FFTs on the 1000 x 120 padded grid, direct "
                                                    "sum over the 10 planes"},
            "launches_per_step": 7, "streams": 2,
            "note": "1 nm cells, 0.25 nm sites, 8 nm grains, window follows the spot; Eq. 6, the m_e solve and "
                    "RK4 stages 0-2 on a second stream beside the window step"}
    # the simulated region (Sec. II, Fig. 1): the window and 60 cell columns on each side evolve,
    # the rest of the track is frozen; the step's cost follows the region, not the track
    reg = {}
    for ncx in (500, 2000):
        wt = I.multiscale_track(ncx=ncx)
        reg[str(ncx)] = {"ms_per_step": ms_rate(wt, "fp32", 5 * K, dist, margin=60),
                         "ms_per_step_demag": ms_rate(wt, "fp32", K, dist, demag=True, margin=60),
                         "cells": ncx * wt["ncy"] * wt["ncz"]}
    line["region"] = {"margin_cells": 60, "dtype": "f32", "tracks_by_ncx": reg,
                      "note": "track lengths of 500 and 2000 cells; Eq. 7 with the region's own field on a "
                              "360-column padded grid each step and the frozen track's field kept between moves"}
    if not args.no_cpu and dist.rank == 0 and dist.world == 1:
        import oracle as orc
        T, F = w["T"], w["field"]
        p = orc.MsParams(w["ncx"], w["ncy"], w["ncz"], w["cell"], w["ratio"], w["wx"], J=w["J"], mu_s=w["mu_s"],
                         ku=w["ku"], lam=w["lam"], T_C=w["T_C"], Ms0=w["Ms0"], A0=w["A0"], K0=w["K0"], dt=w["dt"],
                         seed=w["seed"], **T, B0=F["B0"], direction=F["direction"], bits=F["bits"],
                         bit_len=F["bit_len"], ramp_len=F["ramp_len"], head_x0=F["head_x0"], head_v=F["head_v"])
        O = orc.MsOracle(p, w["grain"])
        O.set_cells(m)
        O.set_window(ox)
        O.run(1, follow=True)
        t0 = time.perf_counter()
        O.run(2, follow=True)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nw * 2 / el, "unit": "window spin-steps/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": "2 coupled steps of the full track in %.1f s" % el}
        # the same three coupled steps on the GPU in both precisions, against the oracle
        for prec, key in (("fp32", None), ("fp64", "fp64")):
            G = make(prec)
            G.set_cells(m)
            G.set_window(ox)
            G.steps(3, follow=True)
            err = {"max_abs_cell": float(np.abs(G.read_cells() - O.cells()).max()),
                   "max_abs_spin": float(np.abs(G.read_moments() - O.moments()).max()),
                   "what": "3 coupled steps of the full track from the same state, every cell and window spin"}
            G.close()
            (line[key] if key else line)["oracle_err"] = err
        line["region"]["oracle_err"] = ms_oracle_err(w, "fp32", margin=60)
        line["region"]["oracle_err"]["what"] = "3 coupled steps of the full track, 60 columns each side evolved"
        # Eq. 7: the oracle sums over every pair of cells, so its error is taken on a shorter,
        # thinner track that runs the same kernels (the in-plane transforms and the sum along z)
        ws = I.multiscale_track(ncx=40, ncy=8, ncz=4, ratio=4, wx=10, grain_d=5e-9, seed=33, x_spot=20.2e-9)
        for margin, tgt in ((-1, line["fp32_with_demag"]), (8, line["region"])):
            e = ms_oracle_err(ws, "fp32", margin=margin, demag=True)
            e["what"] = ("3 coupled steps of a 40 x 8 x 4-cell track (0.25 nm sites, a 10-cell window%s) with "
                         "Eq. 7" % (", 8 columns each side evolved" if margin >= 0 else ""))
            tgt["oracle_err_demag" if margin >= 0 else "oracle_err"] = e
    return line


def ms_oracle_err(w, precision, margin=-1, demag=False, steps=3):
    """Largest difference of every cell and window spin to the FP64 oracle after `steps`
    coupled steps of the multiscale track w from +z cells, the window following the spot."""
    import oracle as orc
    from paper_2502_02236_gb300.hamr import Multiscale
    T, F = w["T"], w["field"]
    p = orc.MsParams(w["ncx"], w["ncy"], w["ncz"], w["cell"], w["ratio"], w["wx"], J=w["J"], mu_s=w["mu_s"],
                     ku=w["ku"], lam=w["lam"], T_C=w["T_C"], Ms0=w["Ms0"], A0=w["A0"], K0=w["K0"], dt=w["dt"],
                     seed=w["seed"], **T, B0=F["B0"], direction=F["direction"], bits=F["bits"],
                     bit_len=F["bit_len"], ramp_len=F["ramp_len"], head_x0=F["head_x0"], head_v=F["head_v"],
                     demag=demag, margin=margin)
    m = np.zeros((w["ncx"] * w["ncy"] * w["ncz"], 3))
    m[:, 2] = 1.0
    ox = orc.ms_target(p, 0.0)
    O = orc.MsOracle(p, w["grain"])
    O.set_cells(m)
    O.set_window(ox)
    O.run(steps, follow=True)
    G = Multiscale(w["ncx"], w["ncy"], w["ncz"], w["cell"], w["ratio"], w["wx"], J=w["J"], mu_s=w["mu_s"],
                   ku=w["ku"], Ms0=w["Ms0"], A0=w["A0"], K0=w["K0"], lam=w["lam"], T_C=w["T_C"], dt=w["dt"],
                   seed=w["seed"], precision=precision)
    G.set_grain_map(w["grain"])
    G.set_temperature_profile(**T)
    G.set_field_sequence(**F)
    G.set_cells(m)
    if margin >= 0:
        G.set_region(margin)
    if demag:
        G.set_demag(True)
    G.set_window(ox)
    G.steps(steps, follow=True)
    err = {"max_abs_cell": float(np.abs(G.read_cells() - O.cells()).max()),
           "max_abs_spin": float(np.abs(G.read_moments() - O.moments()).max())}
    G.close()
    return err


def multiscale_only(args, dist):
    """bench.py --workload multiscale_track: the multiscale track alone, FP32, K = --steps
    coupled steps after --warmup (the demagnetising field on with --ms-demag); one JSON line."""
    import torch
    from paper_2502_02236_gb300 import inputs as I
    from paper_2502_02236_gb300.hamr import Multiscale
    w = I.multiscale_track(ncx=args.ms_ncx)
    G = Multiscale(w["ncx"], w["ncy"], w["ncz"], w["cell"], w["ratio"], w["wx"], J=w["J"], mu_s=w["mu_s"], ku=w["ku"],
                   Ms0=w["Ms0"], A0=w["A0"], K0=w["K0"], lam=w["lam"], T_C=w["T_C"], dt=w["dt"],
                   seed=w["seed"] ^ (dist.rank << 48), precision="fp32")
    G.set_grain_map(w["grain"])
    G.set_temperature_profile(**w["T"])
    G.set_field_sequence(**w["field"])
    m = np.zeros((G.n_cells, 3))
    m[:, 2] = 1.0
    G.set_cells(m)
    G.set_region(args.ms_margin)
    G.set_window(int(np.floor(w["T"]["x0"] / w["cell"] - w["wx"] / 2 + 0.5)))
    if args.ms_demag:
        G.set_demag(True)
    G.steps(max(3, args.warmup), follow=True)
    K = max(1, args.steps)
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    G.steps(K, follow=True)
    e1.record()
    torch.cuda.synchronize()
    ms = dist.max(e0.elapsed_time(e1))
    nw = G.n_window
    G.close()
    out = {"metric": "window spin-steps/s (multiscale track, FP32)", "value": nw * K * dist.world / (ms / 1e3),
           "unit": "spin-steps/s", "n_gpus": dist.world, "steps": K, "warmup": max(3, args.warmup),
           "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": {"workload": "multiscale_track", "demag": bool(args.ms_demag),
                                           "window_sites": nw, "cells": G.n_cells, "margin": args.ms_margin}}
    if dist.rank == 0:
        print(json.dumps(out), flush=True)
    dist.close()


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        return reference_arm(args, dist)
    import torch
    from paper_2502_02236_gb300 import build
    from paper_2502_02236_gb300 import inputs as I
    if dist.rank == 0:
        build.build()
    dist.barrier()
    build.build()
    torch.cuda.set_device(dist.local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)     # the library runs on (and is timed on) this stream
    if args.workload == "multiscale_track":
        return multiscale_only(args, dist)
    W = max(3, args.warmup)
    K = args.steps
    w = I.workload(args.workload)
    rec = int(w.get("record_every", 10))
    n_sites = sum(int(np.prod(rep["dims"])) for rep in w["replicas"])
    n_mag = sum(int((np.asarray(rep["grain"]) >= 0).sum()) if rep.get("grain") is not None
                else int(np.prod(rep["dims"])) for rep in w["replicas"])

    lat = build_lattice(w, "fp32", dist.rank)
    if args.planes:
        lat.set_plane_range(args.planes)
    if args.tile:
        lat.set_tile(*(int(v) for v in args.tile.split("x")))
        tile = lat.get_tile()
    else:
        tile = lat.autotune(5)
    lat.sllg_heun_steps(W - W % rec + rec, rec)
    prime(lat, K, rec)
    prime(lat, K, 0)
    clocks = Clocks(dist.local)
    clocks.start()
    ms = timed(lat, dist, K, rec)
    clk = clocks.stop()
    ms = dist.max(ms)
    value = aggregate(n_sites, K, dist.world, ms)
    # the dominant kernel alone: the same K steps without records (one fused launch per step
    # plus one bookkeeping launch per 64 steps)
    ms_k = dist.max(timed(lat, dist, K, 0))
    t_launch = ms_k / K / 1e3
    achieved = BYTES_PER_SITE_FP32 * n_sites / t_launch / 1e9
    peak, peak_kind = peaks()
    counters = kernel_counters() if args.workload == "ensemble256" and tile == (512, 864) else None
    traffic = counters.get("dram_bytes_per_launch") if counters else None
    assert lat.check_finite()
    launches = K + K // rec

    out = {"metric": METRIC, "value": value, "unit": "spin-steps/s", "n_gpus": dist.world, "steps": K,
           "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "replicas": len(w["replicas"]), "lattice_sites": n_sites,
                      "magnetic_sites": n_mag, "record_every": rec, "tile": list(tile),
                      "plane_range": lat.query(6), "work_items": lat.query(5),
                      "l2": l2_note(n_sites),
                      "parallelism": "replica batches per GPU, no collective"},
           "magnetic_spin_steps_per_s": n_mag * K * dist.world / (ms / 1e3),
           "gpu_launches": launches,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": traffic,
                        "traffic_gbs": traffic / t_launch / 1e9 if traffic else None,
                        "frac_magnetic": BYTES_PER_SITE_FP32 * n_mag / t_launch / 1e9 / peak,
                        "peak_source": peak_kind, "kernel": "k_fused", "avg_launch_ms": t_launch * 1e3,
                        "bytes_per_site": BYTES_PER_SITE_FP32,
                        "issue": issue_roof(counters.get("warp_inst_per_launch") if counters else None,
                                            t_launch * 1e3, (clk or {}).get("sm_mhz"))},
           "clocks": clk}

    # plain FP64 path on the same workload (the speedup denominator)
    if not args.no_fp64:
        lat64 = build_lattice(w, "fp64", dist.rank)
        K64 = max(1, args.fp64_steps)
        lat64.sllg_heun_steps(rec, rec)
        prime(lat64, K64, rec)
        ms64 = dist.max(timed(lat64, dist, K64, rec))
        v64 = n_sites * K64 * dist.world / (ms64 / 1e3)
        out["fp64_plain"] = {"value": v64, "unit": "spin-steps/s", "steps": K64, "ms_per_step": ms64 / K64,
                             "launches_per_step": 2, "dtype": "f64"}
        out["speedup_fp32_over_fp64"] = value / v64
        if args.no_cpu or dist.rank != 0 or dist.world != 1:
            lat64.close()
            lat64 = None

    # end to end through the C ABI with host buffers: upload all spins from pinned memory,
    # K steps with records, read the records and all spins back
    if not args.no_e2e:
        S_host = [torch.empty((int(np.prod(rep["dims"])), 3), dtype=torch.float64).pin_memory()
                  for rep in w["replicas"]]
        for t in S_host:
            t[:, 2] = 1.0
        hb = sum(t.numel() * 8 for t in S_host)
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r, t in enumerate(S_host):
            lat.set_moments(r, t.numpy())
        lat.sllg_heun_steps(K, rec)
        d2h = 0
        for r, t in enumerate(S_host):
            M, st, _ = lat.read_magnetisation(r)
            d2h += M.nbytes
            lat.read_moments(r, t.numpy())
        el = dist.max(time.perf_counter() - t0)
        d2h += hb
        out["e2e"] = {"value": n_sites * K * dist.world / el, "unit": "spin-steps/s",
                      "h2d_bytes_per_step": hb / K, "d2h_bytes_per_step": d2h / K,
                      "note": "per call: H2D of all spins, K steps, D2H of M(t) and all spins; bytes / K"}

    if not args.no_ms and args.workload == "ensemble256":
        out["multiscale"] = multiscale_line(args, dist)

    if not args.no_cpu and dist.rank == 0 and dist.world == 1:
        # the error against the FP64 oracle beside every reported rate (this leg runs the oracle)
        chk = list(range(0, len(w["replicas"]), max(1, len(w["replicas"]) // 32)))
        out["oracle_err"] = oracle_error(lat, w, chk)
        if not args.no_fp64:
            out["fp64_plain"]["oracle_err"] = oracle_error(lat64, w, chk[:8])
            lat64.close()
        v, reps, n, steps, el = cpu_baseline(w, args.cpu_seconds)
        out["cpu_baseline"] = {"value": v, "unit": "spin-steps/s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": "FP64 oracle, replicas 0..%d of the workload (%d sites), %d steps in %.1f s"
                                         % (reps[-1], n, steps, el)}
        one = cpu_baseline_one_core(args.workload, max(3.0, args.cpu_seconds / 3))
        if one:
            out["cpu_baseline"]["one_core"] = one
    lat.close()
    if dist.rank == 0:
        print(json.dumps(out), flush=True)
    dist.close()


def reference_arm(args, dist):
    """The FP64 CPU oracle timed on this host's cores on the same workload, metric and unit."""
    if dist.rank != 0:
        dist.close()
        return
    from paper_2502_02236_gb300 import inputs as I
    import oracle as orc
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from common import initial, oracle_params
    w = I.workload(args.workload)
    # sample: the first replicas of the ensemble up to ~3e5 sites, stepped K + W times
    reps, n = [], 0
    for r, rep in enumerate(w["replicas"]):
        reps.append(r)
        n += int(np.prod(rep["dims"]))
        if n >= 300000:
            break
    orcs = [orc.Oracle(oracle_params(w, r), w["replicas"][r].get("grain")) for r in reps]
    S = [initial(w["replicas"][r]) for r in reps]
    W, K = max(3, args.warmup), args.steps
    budget = 150.0
    t_start = time.perf_counter()
    for k in range(min(W, 3)):
        for o, s in zip(orcs, S):
            o.step(s, k)
    t0 = time.perf_counter()
    done = 0
    for k in range(K):
        for o, s in zip(orcs, S):
            o.step(s, W + k)
        done += 1
        if time.perf_counter() - t_start > budget:
            break
    el = time.perf_counter() - t0
    v = n * done / el
    out = {"metric": METRIC, "value": v, "unit": "spin-steps/s", "n_gpus": dist.world, "steps": done,
           "warmup": W, "ms_per_step": el / done * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "sample_replicas": len(reps), "sample_sites": n},
           "cpu_baseline": {"value": v, "unit": "spin-steps/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "replicas 0..%d (%d sites), %d steps" % (reps[-1], n, done)},
           "e2e": {"value": v, "unit": "spin-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    dist.close()


if __name__ == "__main__":
    main()
