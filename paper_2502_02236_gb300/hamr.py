"""Python binding of the C ABI in include/hamr.h (argument marshalling only).

Every step of the stochastic-LLG Heun path runs in the CUDA library libhamr.so; this
module only converts arguments.  There is no CPU fallback: importing works without the
library, but the first call raises if libhamr.so has not been built.
"""
import ctypes
import os

import numpy as np

from .inputs import GAMMA

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhamr.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_TIMEOUT, ERR_NUMERIC, ERR_IO = 0, -1, -2, -3, -4, -5, -6, -7
LATTICE = {"sc": 0, "l10": 1}
PRECISION = {"fp32": 0, "fp64": 1}
NEIGHBOURS = {"stencil": 0, "csr": 1}
EXPORTS = [
    "hamr_lattice_create", "hamr_set_neighbour_shells", "hamr_set_csr", "hamr_set_grain_map",
    "hamr_set_temperature_profile", "hamr_set_field_sequence", "hamr_set_moments",
    "hamr_set_moments_device", "hamr_sllg_heun_steps", "hamr_sllg_heun_steps_async",
    "hamr_synchronize", "hamr_read_moments", "hamr_read_moments_device",
    "hamr_read_magnetisation", "hamr_clear_records", "hamr_read_energy", "hamr_get_step",
    "hamr_set_step", "hamr_check_finite", "hamr_save_state", "hamr_load_state", "hamr_set_tile",
    "hamr_get_tile", "hamr_set_plane_range", "hamr_autotune", "hamr_query", "hamr_last_error", "hamr_destroy",
    "hamr_sllg_heun_step_noalloc", "hamr_inject_wait_timeout",
    "hamr_ms_create", "hamr_ms_set_grain_map", "hamr_ms_set_temperature_profile",
    "hamr_ms_set_field_sequence", "hamr_ms_set_cells", "hamr_ms_set_window", "hamr_ms_set_moments",
    "hamr_ms_steps", "hamr_ms_read_cells", "hamr_ms_read_moments", "hamr_ms_get_window", "hamr_ms_read_track",
    "hamr_ms_set_head_profile", "hamr_ms_set_demag", "hamr_ms_demag_field", "hamr_ms_set_region",
    "hamr_ms_last_error", "hamr_ms_destroy",
]
NOALLOC_MAX_SITES = 131072


class HamrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hamr error %d: %s" % (code, msg))
        self.code = code


class Desc(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("precision", ctypes.c_int32), ("neighbours", ctypes.c_int32),
        ("n_replicas", ctypes.c_int32),
        ("dims", ctypes.POINTER(ctypes.c_int32)), ("seeds", ctypes.POINTER(ctypes.c_uint64)),
        ("a", ctypes.c_double), ("c", ctypes.c_double),
        ("periodic", ctypes.c_int32 * 3),
        ("mu_s", ctypes.c_double), ("ku", ctypes.c_double), ("alpha", ctypes.c_double),
        ("dt", ctypes.c_double), ("gamma", ctypes.c_double),
        ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
    ]


class NoallocParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3),
        ("a", ctypes.c_double), ("mu_s", ctypes.c_double), ("J", ctypes.c_double),
        ("ku", ctypes.c_double), ("alpha", ctypes.c_double), ("dt", ctypes.c_double),
        ("gamma", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("T_amb", ctypes.c_double), ("T_peak", ctypes.c_double), ("fwhm", ctypes.c_double),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("vx", ctypes.c_double),
        ("vy", ctypes.c_double), ("B_app", ctypes.c_double * 3),
    ]


class MsDesc(ctypes.Structure):
    _fields_ = [
        ("ncx", ctypes.c_int32), ("ncy", ctypes.c_int32), ("ncz", ctypes.c_int32),
        ("cell", ctypes.c_double), ("ratio", ctypes.c_int32), ("wx", ctypes.c_int32),
        ("J", ctypes.c_double), ("mu_s", ctypes.c_double), ("ku", ctypes.c_double),
        ("Ms0", ctypes.c_double), ("A0", ctypes.c_double), ("K0", ctypes.c_double),
        ("lambda_", ctypes.c_double), ("T_C", ctypes.c_double),
        ("gamma", ctypes.c_double), ("dt", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int32), ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
    ]


_lib = None


def lib():
    """The loaded libhamr.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhamr.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_2502_02236_gb300.build" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "hamr_lattice_create": [vp, vp],
            "hamr_set_neighbour_shells": [vp, i32, vp],
            "hamr_set_csr": [vp, i32, vp, vp, vp],
            "hamr_set_grain_map": [vp, i32, vp, i32],
            "hamr_set_temperature_profile": [vp, i32, d, d, d, d, d, d, d],
            "hamr_set_field_sequence": [vp, i32, d, vp, vp, i32, d, d, d, d],
            "hamr_set_moments": [vp, i32, vp],
            "hamr_set_moments_device": [vp, i32, vp],
            "hamr_sllg_heun_steps": [vp, i64, i32],
            "hamr_sllg_heun_steps_async": [vp, i64, i32],
            "hamr_synchronize": [vp],
            "hamr_read_moments": [vp, i32, vp],
            "hamr_read_moments_device": [vp, i32, vp],
            "hamr_read_magnetisation": [vp, i32, vp, i64, vp, vp, vp],
            "hamr_clear_records": [vp],
            "hamr_read_energy": [vp, i32, vp],
            "hamr_get_step": [vp, vp],
            "hamr_set_step": [vp, i64],
            "hamr_check_finite": [vp],
            "hamr_save_state": [vp, ctypes.c_char_p],
            "hamr_load_state": [vp, ctypes.c_char_p],
            "hamr_set_tile": [vp, i32, i32],
            "hamr_get_tile": [vp, vp, vp],
            "hamr_set_plane_range": [vp, i32],
            "hamr_autotune": [vp, i32],
            "hamr_query": [vp, i32, vp],
            "hamr_sllg_heun_step_noalloc": [vp, vp, vp, vp, i64, vp],
            "hamr_inject_wait_timeout": [vp, i32],
            "hamr_ms_create": [vp, vp],
            "hamr_ms_set_grain_map": [vp, vp],
            "hamr_ms_set_temperature_profile": [vp, d, d, d, d, d, d, d],
            "hamr_ms_set_field_sequence": [vp, d, vp, vp, i32, d, d, d, d],
            "hamr_ms_set_cells": [vp, vp],
            "hamr_ms_set_window": [vp, i32],
            "hamr_ms_set_moments": [vp, vp],
            "hamr_ms_steps": [vp, i64, i32],
            "hamr_ms_read_cells": [vp, vp],
            "hamr_ms_read_moments": [vp, vp],
            "hamr_ms_get_window": [vp, vp, vp],
            "hamr_ms_read_track": [vp, d, d, i32, i32, i32, vp, vp],
            "hamr_ms_set_head_profile": [vp, d, d, d, d, d],
            "hamr_ms_set_demag": [vp, i32],
            "hamr_ms_demag_field": [vp, vp, vp],
            "hamr_ms_set_region": [vp, i32],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.hamr_last_error.argtypes = [vp]
        L.hamr_last_error.restype = ctypes.c_char_p
        L.hamr_destroy.argtypes = [vp]
        L.hamr_destroy.restype = None
        L.hamr_ms_last_error.argtypes = [vp]
        L.hamr_ms_last_error.restype = ctypes.c_char_p
        L.hamr_ms_destroy.argtypes = [vp]
        L.hamr_ms_destroy.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _torch_current():
    """(device ordinal, stream handle) of torch's current CUDA stream, or (0, None).  The
    legacy default stream (handle 0) cannot be graph-captured: the library then makes its
    own stream, and device-pointer calls must be ordered by the caller."""
    try:
        import torch
        if torch.cuda.is_available():
            s = torch.cuda.current_stream()
            return torch.cuda.current_device(), (s.cuda_stream or None)
    except Exception:
        pass
    return 0, None


class Lattice:
    """One hamr_t handle: n_replicas independent lattices advanced together."""

    def __init__(self, dims, seeds, *, lattice="sc", precision="fp32", neighbours="stencil",
                 a=0.25e-9, c=0.0, periodic=(False, False, False), mu_s, ku=0.0, alpha=0.1,
                 dt=1e-16, gamma=GAMMA, device=None, stream="torch"):
        L = lib()
        self.dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
        self.R = self.dims.shape[0]
        self.seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64).reshape(-1))
        if self.seeds.size != self.R:
            raise ValueError("one seed per replica")
        self.precision = precision
        d = Desc()
        d.lattice = LATTICE[lattice]
        d.precision = PRECISION[precision]
        d.neighbours = NEIGHBOURS[neighbours]
        d.n_replicas = self.R
        d.dims = self.dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.seeds = self.seeds.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        d.a, d.c = a, c
        for k in range(3):
            d.periodic[k] = int(bool(periodic[k]))
        d.mu_s, d.ku, d.alpha, d.dt, d.gamma = mu_s, ku, alpha, dt, gamma
        tdev, tstream = _torch_current()
        d.device = tdev if device is None else device
        self.stream = tstream if stream == "torch" else stream
        d.stream = self.stream
        h = ctypes.c_void_p()
        rc = L.hamr_lattice_create(ctypes.byref(h), ctypes.byref(d))
        if rc != OK:
            raise HamrError(rc, L.hamr_last_error(None).decode())
        self._h = h

    # -------------------------------------------------------------------- plumbing
    def _ck(self, rc):
        if rc != OK:
            raise HamrError(rc, lib().hamr_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            lib().hamr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def n_sites(self, r):
        nx, ny, nz = self.dims[r]
        return int(nx) * int(ny) * int(nz)

    # -------------------------------------------------------------------- setters
    def set_neighbour_shells(self, J):
        J = np.ascontiguousarray(np.asarray(J, dtype=np.float64).reshape(-1))
        self._ck(lib().hamr_set_neighbour_shells(self._h, J.size, _p(J)))

    def set_csr(self, replica, row_ptr, col, shell):
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        sh = np.ascontiguousarray(shell, dtype=np.uint8)
        self._ck(lib().hamr_set_csr(self._h, replica, _p(rp), _p(cl), _p(sh)))

    def set_grain_map(self, replica, grain, n_grains):
        g = np.ascontiguousarray(np.asarray(grain, dtype=np.int32).reshape(-1))
        if g.size != self.n_sites(replica):
            raise ValueError("grain map size %d != %d sites" % (g.size, self.n_sites(replica)))
        self._ck(lib().hamr_set_grain_map(self._h, replica, _p(g), int(n_grains)))

    def set_temperature_profile(self, replica, T_amb, T_peak=0.0, fwhm=0.0, x0=0.0, y0=0.0, vx=0.0, vy=0.0):
        self._ck(lib().hamr_set_temperature_profile(self._h, replica, T_amb, T_peak, fwhm, x0, y0, vx, vy))

    def set_field_sequence(self, replica, B0, direction=(0.0, 0.0, 1.0), bits=(), bit_len=1.0,
                           ramp_len=0.0, head_x0=0.0, head_v=0.0):
        dr = np.ascontiguousarray(np.asarray(direction, dtype=np.float64))
        b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8).reshape(-1))
        bp = _p(b) if b.size else None
        self._ck(lib().hamr_set_field_sequence(self._h, replica, B0, _p(dr), bp, b.size, bit_len,
                                               ramp_len, head_x0, head_v))

    def set_moments(self, replica, S):
        S = np.ascontiguousarray(np.asarray(S, dtype=np.float64))
        if S.size != 3 * self.n_sites(replica):
            raise ValueError("spin array must hold 3 x %d values" % self.n_sites(replica))
        self._ck(lib().hamr_set_moments(self._h, replica, _p(S)))

    def set_moments_device(self, replica, S):
        """S: a contiguous float64 CUDA tensor of shape (n, 3) on the handle's device."""
        if S.dtype != __import__("torch").float64 or not S.is_cuda or not S.is_contiguous():
            raise ValueError("need a contiguous float64 CUDA tensor")
        if S.numel() != 3 * self.n_sites(replica):
            raise ValueError("spin tensor must hold 3 x %d values" % self.n_sites(replica))
        self._ck(lib().hamr_set_moments_device(self._h, replica, ctypes.c_void_p(S.data_ptr())))

    # -------------------------------------------------------------------- stepping
    def sllg_heun_steps(self, n_steps, record_every=0):
        self._ck(lib().hamr_sllg_heun_steps(self._h, int(n_steps), int(record_every)))

    def sllg_heun_steps_async(self, n_steps, record_every=0):
        self._ck(lib().hamr_sllg_heun_steps_async(self._h, int(n_steps), int(record_every)))

    def synchronize(self):
        self._ck(lib().hamr_synchronize(self._h))

    # -------------------------------------------------------------------- readers
    def read_moments(self, replica, out=None):
        n = self.n_sites(replica)
        if out is None:
            out = np.empty((n, 3))
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 3 * n
        self._ck(lib().hamr_read_moments(self._h, replica, _p(out)))
        return out

    def read_moments_device(self, replica, out):
        if out.numel() != 3 * self.n_sites(replica) or not out.is_contiguous():
            raise ValueError("need a contiguous float64 CUDA tensor of 3 x n values")
        self._ck(lib().hamr_read_moments_device(self._h, replica, ctypes.c_void_p(out.data_ptr())))
        return out

    def read_magnetisation(self, replica, n_grains=0):
        """(M_t [n_rec, 3], steps [n_rec], M_grain [n_grains, 3] or None)."""
        n = ctypes.c_int64()
        self._ck(lib().hamr_read_magnetisation(self._h, replica, None, 0, ctypes.byref(n), None, None))
        M = np.zeros((max(n.value, 1), 3))
        st = np.zeros(max(n.value, 1), dtype=np.int64)
        G = np.zeros((max(n_grains, 1), 3)) if n_grains > 0 else None
        self._ck(lib().hamr_read_magnetisation(self._h, replica, _p(M), n.value, ctypes.byref(n),
                                               _p(G) if G is not None else None, _p(st)))
        return M[:n.value], st[:n.value], (G[:n_grains] if G is not None else None)

    def clear_records(self):
        self._ck(lib().hamr_clear_records(self._h))

    def read_energy(self, replica):
        E = ctypes.c_double()
        self._ck(lib().hamr_read_energy(self._h, replica, ctypes.byref(E)))
        return E.value

    @property
    def step(self):
        s = ctypes.c_int64()
        self._ck(lib().hamr_get_step(self._h, ctypes.byref(s)))
        return s.value

    @step.setter
    def step(self, value):
        self._ck(lib().hamr_set_step(self._h, int(value)))

    def check_finite(self):
        rc = lib().hamr_check_finite(self._h)
        if rc == ERR_NUMERIC:
            return False
        self._ck(rc)
        return True

    def save_state(self, path):
        self._ck(lib().hamr_save_state(self._h, os.fsencode(path)))

    def load_state(self, path):
        self._ck(lib().hamr_load_state(self._h, os.fsencode(path)))

    def set_tile(self, tx, ty):
        self._ck(lib().hamr_set_tile(self._h, tx, ty))

    def get_tile(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        self._ck(lib().hamr_get_tile(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_plane_range(self, planes):
        """Planes per work item of the fused FP32 kernel (0: chosen by the work model)."""
        self._ck(lib().hamr_set_plane_range(self._h, int(planes)))

    def autotune(self, steps_per_trial=20):
        self._ck(lib().hamr_autotune(self._h, int(steps_per_trial)))
        return self.get_tile()

    def inject_wait_timeout(self, polls):
        """Failure-detection test: the next step call has one bounded device wait run out
        after `polls` polls and raises HamrError with code ERR_TIMEOUT."""
        self._ck(lib().hamr_inject_wait_timeout(self._h, int(polls)))

    def query(self, key):
        v = ctypes.c_int64()
        self._ck(lib().hamr_query(self._h, int(key), ctypes.byref(v)))
        return v.value


def sllg_heun_step_noalloc(dims, S_in, S_out, *, grain=None, step=0, periodic=(False, False, False),
                           a, mu_s, J, ku=0.0, alpha=0.1, dt=1e-16, gamma=GAMMA, seed=0, T_amb=0.0,
                           T_peak=0.0, fwhm=0.0, x0=0.0, y0=0.0, vx=0.0, vy=0.0, B_app=(0.0, 0.0, 0.0),
                           stream=None):
    """One FP64 Heun step through hamr_sllg_heun_step_noalloc on caller-owned device
    tensors: S_in, S_out float64 (n, 3) (the same tensor or disjoint), grain int32 (n,) or None.
    The library allocates nothing; the call is stream-ordered on `stream` (a raw handle,
    None = the legacy default stream)."""
    p = NoallocParams()
    p.nx, p.ny, p.nz = (int(v) for v in dims)
    for k in range(3):
        p.periodic[k] = int(bool(periodic[k]))
        p.B_app[k] = float(B_app[k])
    p.a, p.mu_s, p.J, p.ku, p.alpha, p.dt, p.gamma = a, mu_s, J, ku, alpha, dt, gamma
    p.seed = int(seed)
    p.T_amb, p.T_peak, p.fwhm, p.x0, p.y0, p.vx, p.vy = T_amb, T_peak, fwhm, x0, y0, vx, vy
    g = ctypes.c_void_p(grain.data_ptr()) if grain is not None else None
    rc = lib().hamr_sllg_heun_step_noalloc(ctypes.byref(p), ctypes.c_void_p(S_in.data_ptr()),
                                           ctypes.c_void_p(S_out.data_ptr()), g, int(step), stream)
    if rc != OK:
        raise HamrError(rc, lib().hamr_last_error(None).decode())


class Multiscale:
    """One hamr_ms_t handle: the multiscale write window (an atomistic simple-cubic window
    in a micromagnetic track, FP64 or FP32).  Cell arrays are (ncx*ncy*ncz, 3), window spins
    (nxw*nyw*nzw, 3), x fastest."""

    def __init__(self, ncx, ncy, ncz, cell, ratio, wx, *, J, mu_s, ku, Ms0, A0, K0, lam, T_C,
                 dt=1e-16, gamma=GAMMA, seed=1, precision="fp64", device=None, stream="torch"):
        L = lib()
        d = MsDesc()
        d.ncx, d.ncy, d.ncz, d.cell, d.ratio, d.wx = ncx, ncy, ncz, cell, ratio, wx
        d.J, d.mu_s, d.ku, d.Ms0, d.A0, d.K0 = J, mu_s, ku, Ms0, A0, K0
        d.lambda_, d.T_C, d.gamma, d.dt, d.seed = lam, T_C, gamma, dt, int(seed)
        d.precision = PRECISION[precision]
        tdev, tstream = _torch_current()
        d.device = tdev if device is None else device
        d.stream = tstream if stream == "torch" else stream
        self.n_cells = ncx * ncy * ncz
        self.ncy = ncy
        self.window_dims = (wx * ratio, ncy * ratio, ncz * ratio)
        self.n_window = int(np.prod(self.window_dims))
        h = ctypes.c_void_p()
        rc = L.hamr_ms_create(ctypes.byref(h), ctypes.byref(d))
        if rc != OK:
            raise HamrError(rc, L.hamr_ms_last_error(None).decode())
        self._h = h

    def _ck(self, rc):
        if rc != OK:
            raise HamrError(rc, lib().hamr_ms_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            lib().hamr_ms_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_grain_map(self, cell_grain):
        g = np.ascontiguousarray(np.asarray(cell_grain, dtype=np.int32).reshape(-1))
        if g.size != self.n_cells:
            raise ValueError("one grain id per cell")
        self._ck(lib().hamr_ms_set_grain_map(self._h, _p(g)))

    def set_temperature_profile(self, T_amb, T_peak=0.0, fwhm=0.0, x0=0.0, y0=0.0, vx=0.0, vy=0.0):
        self._ck(lib().hamr_ms_set_temperature_profile(self._h, T_amb, T_peak, fwhm, x0, y0, vx, vy))

    def set_field_sequence(self, B0, direction=(0.0, 0.0, 1.0), bits=(), bit_len=1.0, ramp_len=0.0,
                           head_x0=0.0, head_v=0.0):
        dr = np.ascontiguousarray(np.asarray(direction, dtype=np.float64))
        b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
        self._ck(lib().hamr_ms_set_field_sequence(self._h, B0, _p(dr), _p(b) if b.size else None, b.size,
                                                  bit_len, ramp_len, head_x0, head_v))

    def set_head_profile(self, Bx0=0.0, wz=0.0, dz=0.0, wx=1.0, dx=0.0):
        """tanh profiles of the write field along the track following the head (wz <= 0: a
        spatially uniform field)."""
        self._ck(lib().hamr_ms_set_head_profile(self._h, Bx0, wz, dz, wx, dx))

    def set_region(self, margin):
        """Evolve only the window and `margin` cell columns on each side; the rest of the track
        is frozen (margin < 0: the whole track)."""
        self._ck(lib().hamr_ms_set_region(self._h, int(margin)))

    def set_demag(self, on=True):
        """The demagnetising field of Eq. 7 in both regions (FFT convolution in x and y, direct
        sum along z)."""
        self._ck(lib().hamr_ms_set_demag(self._h, int(bool(on))))

    def demag_field(self, M):
        """B_d = -mu0 N * M [T] of Eq. 7 on every cell for the given magnetisation M [A/m]
        ((n_cells, 3)); needs set_demag(True)."""
        M = np.ascontiguousarray(np.asarray(M, dtype=np.float64).reshape(-1))
        if M.size != 3 * self.n_cells:
            raise ValueError("three components per cell")
        B = np.zeros((self.n_cells, 3))
        self._ck(lib().hamr_ms_demag_field(self._h, _p(M), _p(B)))
        return B

    def set_cells(self, m):
        m = np.ascontiguousarray(np.asarray(m, dtype=np.float64).reshape(-1))
        if m.size != 3 * self.n_cells:
            raise ValueError("three components per cell")
        self._ck(lib().hamr_ms_set_cells(self._h, _p(m)))

    def set_window(self, x0_cells):
        self._ck(lib().hamr_ms_set_window(self._h, int(x0_cells)))

    def set_moments(self, S):
        S = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(-1))
        if S.size != 3 * self.n_window:
            raise ValueError("three components per window site")
        self._ck(lib().hamr_ms_set_moments(self._h, _p(S)))

    def steps(self, n_steps, follow=False):
        self._ck(lib().hamr_ms_steps(self._h, int(n_steps), int(bool(follow))))

    def read_cells(self):
        m = np.zeros((self.n_cells, 3))
        self._ck(lib().hamr_ms_read_cells(self._h, _p(m)))
        return m

    def read_moments(self):
        S = np.zeros((self.n_window, 3))
        self._ck(lib().hamr_ms_read_moments(self._h, _p(S)))
        return S

    def read_track(self, x_start, bit_len, n_bits, cy0=0, cy1=None):
        """Mean m_z of the magnetic cells in each bit window of the track (rows cy0..cy1-1)
        and the bits it reads as (1 where negative)."""
        cy1 = self.ncy if cy1 is None else cy1
        sig = np.zeros(max(int(n_bits), 1))
        bits = np.zeros(max(int(n_bits), 1), dtype=np.uint8)
        self._ck(lib().hamr_ms_read_track(self._h, float(x_start), float(bit_len), int(n_bits), int(cy0), int(cy1),
                                          _p(sig), _p(bits)))
        return sig[:n_bits], bits[:n_bits]

    def window(self):
        ox = ctypes.c_int32()
        st = ctypes.c_int64()
        self._ck(lib().hamr_ms_get_window(self._h, ctypes.byref(ox), ctypes.byref(st)))
        return ox.value, st.value
