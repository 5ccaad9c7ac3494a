"""Builds the CUDA handle and the FP64 oracle from one workload description, so that a
parity test feeds both sides the same seeded inputs."""
import math

import numpy as np

import oracle as orc
from paper_2502_02236_gb300 import inputs as I


def initial(rep, kind=None, seed=0):
    n = int(np.prod(rep["dims"]))
    S = I.initial_state(n, kind or rep.get("init", "+z"), seed=seed)
    if rep.get("grain") is not None:
        S = I.mask_void(S, rep["grain"])
    return S


def oracle_params(w, r):
    rep = w["replicas"][r]
    nx, ny, nz = rep["dims"]
    T = dict(T_amb=0.0, T_peak=0.0, fwhm=0.0, x0=0.0, y0=0.0, vx=0.0, vy=0.0)
    T.update(rep.get("T", {}))
    F = dict(B0=0.0, direction=(0.0, 0.0, 1.0), bits=(), bit_len=1.0, ramp_len=0.0, head_x0=0.0,
             head_v=0.0)
    F.update(rep.get("field", {}))
    kw = dict(periodic=w["periodic"], mu_s=w["mu_s"], ku=w["ku"], alpha=w["alpha"], dt=w["dt"],
              seed=rep["seed"], **T, B0=F["B0"], direction=F["direction"], bits=F["bits"],
              bit_len=F["bit_len"], ramp_len=F["ramp_len"], head_x0=F["head_x0"], head_v=F["head_v"])
    if w["lattice"] == "sc":
        return orc.sc_params(nx, ny, nz, w["a"], w["J"][0], **kw)
    return orc.l10_params(nx, ny, nz, w["a"], w["c"], *w["J"], **kw)


def oracle_for(w, r):
    rep = w["replicas"][r]
    g = rep.get("grain")
    return orc.Oracle(oracle_params(w, r), None if g is None else np.asarray(g, dtype=np.int32))


def gpu_lattice(w, precision=None, neighbours=None, S0=None):
    from paper_2502_02236_gb300.hamr import Lattice
    reps = w["replicas"]
    lat = Lattice([rep["dims"] for rep in reps], [rep["seed"] for rep in reps], lattice=w["lattice"],
                  precision=precision or w["precision"], neighbours=neighbours or w["neighbours"],
                  a=w["a"], c=w["c"], periodic=w["periodic"], mu_s=w["mu_s"], ku=w["ku"],
                  alpha=w["alpha"], dt=w["dt"])
    lat.set_neighbour_shells(w["J"])
    for r, rep in enumerate(reps):
        if rep.get("grain") is not None:
            lat.set_grain_map(r, rep["grain"], rep["n_grains"])
        T = rep.get("T")
        if T:
            lat.set_temperature_profile(r, **T)
        F = rep.get("field")
        if F:
            lat.set_field_sequence(r, **F)
        lat.set_moments(r, S0[r] if S0 is not None else initial(rep))
    return lat


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) if np.asarray(a).size else 0.0
