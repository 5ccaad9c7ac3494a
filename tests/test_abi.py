"""The C-ABI library loads and exports every symbol hamr.h declares, and rejects bad
arguments on the host before touching a device (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hlib():
    from paper_2502_02236_gb300 import build, hamr
    build.build()
    return hamr.lib()


def declared():
    txt = open(os.path.join(ROOT, "include", "hamr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hamr_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(hlib):
    from paper_2502_02236_gb300 import hamr
    names = declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(hlib, n), n
    assert sorted(hamr.EXPORTS) == names


def _desc(**over):
    from paper_2502_02236_gb300.hamr import Desc
    dims = np.array(over.pop("dims", [4, 4, 4]), dtype=np.int32)
    seeds = np.array(over.pop("seeds", [1]), dtype=np.uint64)
    d = Desc()
    d.lattice, d.precision, d.neighbours = 0, 0, 0
    d.n_replicas = len(seeds)
    d.dims = dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.seeds = seeds.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    d.a, d.c = 0.25e-9, 0.0
    d.mu_s, d.ku, d.alpha, d.dt, d.gamma = 2.78e-23, 1e-22, 0.1, 1e-16, 1.76e11
    for k, v in over.items():
        setattr(d, k, v)
    d._keep = (dims, seeds)
    return d


@pytest.mark.parametrize("bad", [
    dict(lattice=7), dict(precision=3), dict(neighbours=5), dict(lattice=1, neighbours=0),
    dict(a=0.0), dict(a=-1e-9), dict(mu_s=0.0), dict(dt=0.0), dict(gamma=-1.0), dict(alpha=-0.1),
    dict(lattice=1, neighbours=1, c=0.0), dict(dims=[0, 4, 4]), dict(dims=[4, 4, -1]),
    dict(dims=[70000, 1, 1]), dict(n_replicas=0),
])
def test_create_rejects_bad_descriptor(hlib, bad):
    d = _desc(**bad)
    h = ctypes.c_void_p()
    rc = hlib.hamr_lattice_create(ctypes.byref(h), ctypes.byref(d))
    assert rc == -1, hlib.hamr_last_error(None)
    assert not h.value
    assert len(hlib.hamr_last_error(None)) > 0


def test_create_null_arguments(hlib):
    h = ctypes.c_void_p()
    assert hlib.hamr_lattice_create(None, None) == -1
    assert hlib.hamr_lattice_create(ctypes.byref(h), None) == -1


def test_null_handle_calls_are_errors(hlib):
    assert hlib.hamr_sllg_heun_steps(None, 10, 0) == -1
    assert hlib.hamr_set_step(None, 0) == -1
    assert hlib.hamr_get_step(None, None) == -1
    assert hlib.hamr_synchronize(None) == -1
    assert hlib.hamr_set_grain_map(None, 0, None, 0) == -1
    hlib.hamr_destroy(None)


def test_create_without_device_fails_cleanly(hlib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    d = _desc()
    h = ctypes.c_void_p()
    rc = hlib.hamr_lattice_create(ctypes.byref(h), ctypes.byref(d))
    assert rc == -3 and not h.value
    assert b"device" in hlib.hamr_last_error(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2502_02236_gb300 import hamr
    monkeypatch.setattr(hamr, "_lib", None)
    monkeypatch.setattr(hamr, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hamr.lib()
