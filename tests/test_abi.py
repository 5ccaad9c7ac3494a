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


def _ms_desc(**over):
    from paper_2502_02236_gb300.hamr import MsDesc
    d = MsDesc()
    d.ncx, d.ncy, d.ncz, d.cell, d.ratio, d.wx = 20, 4, 2, 1e-9, 2, 6
    d.J, d.mu_s, d.ku = 6.7e-21, 2.78e-23, 1e-22
    d.Ms0, d.A0, d.K0 = 1.78e6, 1.34e-11, 6.4e6
    d.lambda_, d.T_C, d.gamma, d.dt, d.seed = 0.1, 700.0, 1.76e11, 1e-16, 1
    d.precision = 1
    for k, v in over.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad", [
    dict(ncx=0), dict(ncy=-1), dict(ratio=0), dict(wx=0), dict(wx=21), dict(cell=0.0), dict(mu_s=0.0),
    dict(dt=-1e-16), dict(T_C=0.0), dict(Ms0=0.0), dict(lambda_=-0.1), dict(J=float("nan")), dict(precision=2),
    dict(ncz=70000, ratio=1),
])
def test_multiscale_create_rejects_bad_descriptor(hlib, bad):
    """The multiscale window's descriptor is checked before any device work."""
    d = _ms_desc(**bad)
    h = ctypes.c_void_p()
    assert hlib.hamr_ms_create(ctypes.byref(h), ctypes.byref(d)) == -1
    assert not h.value
    assert hlib.hamr_ms_last_error(None)


def test_multiscale_null_arguments(hlib):
    d = _ms_desc()
    assert hlib.hamr_ms_create(None, ctypes.byref(d)) == -1
    h = ctypes.c_void_p()
    assert hlib.hamr_ms_create(ctypes.byref(h), None) == -1
    for f, args in (("hamr_ms_steps", (1, 0)), ("hamr_ms_set_window", (0,)), ("hamr_ms_read_cells", (None,)),
                    ("hamr_ms_set_cells", (None,))):
        assert getattr(hlib, f)(None, *args) == -1
