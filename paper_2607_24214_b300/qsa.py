"""Python binding of the QS-PIC C ABI (include/qsa.h): argument marshalling only.

Every step of the hot path runs in the CUDA kernels of libqsa.so.  PyTorch supplies device
memory (its caching allocator, through the ABI's allocator callbacks) and the CUDA stream.
There is no fallback: if the library is missing or no GPU is present, construction raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import config

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libqsa.so")
# the bounds-checked debug build (build.build(bounds=True)); QSA_LIBRARY selects another file
BOUNDS_LIB_PATH = os.path.join(_HERE, "_lib", "libqsa_bounds.so")

QSA_OK = 0
QSA_ERR_ARG = -1
QSA_ERR_CUDA = -2
QSA_ERR_OOM = -3
QSA_ERR_TIMEOUT = -4
QSA_ERR_NONFINITE = -5
QSA_ERR_STATE = -6
QSA_WARN_PSI_FLOOR = 1

FIELDS = ("Wx", "Wy", "Ez", "Bx", "By", "Bz")   # Wx = E_x - B_y, Wy = E_y + B_x
SOURCES = ("Sb", "Jz", "Jx", "Jy")

EXPORTS = ("qsa_init", "qsa_set_beam", "qsa_get_beam", "qsa_plasma_sweep", "qsa_beam_step",
           "qsa_diagnostics", "qsa_copy_field", "qsa_copy_source", "qsa_field_solve",
           "qsa_phase_times", "qsa_launch_count", "qsa_device_bytes", "qsa_last_error",
           "qsa_destroy", "qsa_field_solve_static", "qsa_advance", "qsa_launch_times",
           "qsa_eq5_march", "qsa_advance_batch", "qsa_bounds_check", "qsa_grad_forward",
           "qsa_grad_backward", "qsa_rehome", "qsa_rehome_count", "qsa_batch_graphs")


class QsaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qsa error {code}: {msg}")
        self.code = code


class Species(ct.Structure):
    _fields_ = [("Z", ct.c_double), ("M", ct.c_double), ("alpha", ct.c_double),
                ("gamma_b", ct.c_double), ("gamma_spread_rel", ct.c_double),
                ("uperp_spread", ct.c_double), ("noise_rel", ct.c_double),
                ("ppc_x", ct.c_int32), ("ppc_y", ct.c_int32), ("ppc_xi", ct.c_int32),
                ("seeded", ct.c_int32), ("xi_front", ct.c_double), ("xi_back", ct.c_double)]


class Mode(ct.Structure):
    _fields_ = [("mx", ct.c_int32), ("my", ct.c_int32), ("amplitude", ct.c_double),
                ("phase", ct.c_double)]


class KVec(ct.Structure):
    _fields_ = [("mx", ct.c_int32), ("my", ct.c_int32)]


class ParamsC(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nxi", ct.c_int32),
                ("ppc_plasma_x", ct.c_int32), ("ppc_plasma_y", ct.c_int32),
                ("n_species", ct.c_int32), ("n_modes", ct.c_int32), ("precision", ct.c_int32),
                ("n_pc_iter", ct.c_int32), ("pipeline_depth", ct.c_int32),
                ("Lx", ct.c_double), ("Ly", ct.c_double), ("Lxi", ct.c_double),
                ("dt", ct.c_double), ("psi_floor", ct.c_double), ("seed", ct.c_uint64),
                ("spin_limit", ct.c_int64), ("species", Species * 4), ("modes", Mode * 16),
                ("n_diag_modes", ct.c_int32), ("_pad", ct.c_int32), ("diag_modes", KVec * 16),
                ("pc_tol", ct.c_double), ("rehome_frac", ct.c_double)]


_DP = ct.POINTER(ct.c_double)


class Diag(ct.Structure):
    _fields_ = [("energy", _DP), ("psi0", _DP), ("ez0", _DP), ("jz_mean", _DP),
                ("kappa2", _DP), ("opp_min", _DP), ("n_floor", _DP), ("invariant", _DP),
                ("charge", _DP), ("pc_residual", _DP), ("beam_lost", ct.c_int64),
                ("sweeps", ct.c_int64), ("rms", _DP), ("seg_width", ct.c_double),
                ("rms_seg", _DP), ("mode_amp", _DP), ("beam_moments", _DP),
                ("pc_iters", _DP)]


ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)
FREE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)

_lib = None


def load_library(path: str = None):
    """Load libqsa.so (built by paper_2607_24214_b300.build) and declare its signatures.
    The environment variable QSA_LIBRARY, when set, names the file instead (for example the
    bounds-checked debug build)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("QSA_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m "
                          f"paper_2607_24214_b300.build` (nvcc, sm_103a)")
    lib = ct.CDLL(path)
    P = ct.c_void_p
    lib.qsa_init.argtypes = [ct.POINTER(ParamsC), P, ALLOC_FN, FREE_FN, P, ct.POINTER(P)]
    lib.qsa_init.restype = ct.c_int
    lib.qsa_set_beam.argtypes = [P, ct.c_int, ct.c_int64] + [_DP] * 7
    lib.qsa_set_beam.restype = ct.c_int
    lib.qsa_get_beam.argtypes = [P, ct.c_int, ct.c_int64] + [_DP] * 7 + [ct.POINTER(ct.c_int64)]
    lib.qsa_get_beam.restype = ct.c_int
    for name in ("qsa_plasma_sweep", "qsa_beam_step"):
        getattr(lib, name).argtypes = [P]
        getattr(lib, name).restype = ct.c_int
    lib.qsa_advance.argtypes = [P, ct.c_int32]
    lib.qsa_advance.restype = ct.c_int
    lib.qsa_advance_batch.argtypes = [ct.POINTER(P), ct.c_int32, ct.c_int32]
    lib.qsa_advance_batch.restype = ct.c_int
    lib.qsa_batch_graphs.argtypes = [P, ct.c_int32, ct.POINTER(ct.c_int64)]
    lib.qsa_batch_graphs.restype = ct.c_int
    lib.qsa_bounds_check.argtypes = [ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64)]
    lib.qsa_bounds_check.restype = ct.c_int
    lib.qsa_rehome.argtypes = [P]
    lib.qsa_rehome.restype = ct.c_int
    lib.qsa_rehome_count.argtypes = [P]
    lib.qsa_rehome_count.restype = ct.c_int64
    lib.qsa_grad_forward.argtypes = [P, ct.c_int32, ct.c_int32, _DP]
    lib.qsa_grad_forward.restype = ct.c_int
    lib.qsa_grad_backward.argtypes = [P, ct.c_double, _DP, _DP]
    lib.qsa_grad_backward.restype = ct.c_int
    lib.qsa_launch_times.argtypes = [P, ct.POINTER(ct.c_float), ct.c_int,
                                     ct.POINTER(ct.c_int)]
    lib.qsa_launch_times.restype = ct.c_int
    lib.qsa_diagnostics.argtypes = [P, ct.POINTER(Diag)]
    lib.qsa_diagnostics.restype = ct.c_int
    lib.qsa_copy_field.argtypes = [P, ct.c_int, ct.c_int, ct.c_int, _DP]
    lib.qsa_copy_field.restype = ct.c_int
    lib.qsa_copy_source.argtypes = [P, ct.c_int, ct.c_int, ct.c_int, _DP]
    lib.qsa_copy_source.restype = ct.c_int
    lib.qsa_field_solve.argtypes = [P] + [_DP] * 6 + [ct.c_double, _DP]
    lib.qsa_field_solve.restype = ct.c_int
    lib.qsa_field_solve_static.argtypes = ([ct.c_int32, ct.c_int32, ct.c_double, ct.c_double,
                                            ct.c_double, ct.c_int32] + [P] * 8)
    lib.qsa_field_solve_static.restype = ct.c_int
    lib.qsa_eq5_march.argtypes = ([ct.c_int32, ct.c_int32, ct.c_double] + [_DP] * 3 +
                                  [ct.c_double, ct.c_int32, ct.c_int32, _DP, P])
    lib.qsa_eq5_march.restype = ct.c_int
    lib.qsa_phase_times.argtypes = [P, ct.POINTER(ct.c_int64), ct.c_int]
    lib.qsa_phase_times.restype = ct.c_int
    lib.qsa_launch_count.argtypes = [P]
    lib.qsa_launch_count.restype = ct.c_int64
    lib.qsa_device_bytes.argtypes = [P]
    lib.qsa_device_bytes.restype = ct.c_int64
    lib.qsa_last_error.argtypes = [P]
    lib.qsa_last_error.restype = ct.c_char_p
    lib.qsa_destroy.argtypes = [P]
    lib.qsa_destroy.restype = None
    _lib = lib
    return lib


def to_c_params(p: config.Params) -> ParamsC:
    c = ParamsC()
    c.nx, c.ny, c.nxi = p.nx, p.ny, p.nxi
    c.ppc_plasma_x, c.ppc_plasma_y = p.ppc_plasma_x, p.ppc_plasma_y
    c.n_species = len(p.species)
    c.n_modes = len(p.modes)
    c.precision = 0 if p.precision == "fp64" else 1
    c.n_pc_iter = p.n_pc_iter
    c.pc_tol = p.pc_tol
    c.rehome_frac = p.rehome_frac
    c.pipeline_depth = p.pipeline_depth
    c.Lx, c.Ly, c.Lxi, c.dt = p.Lx, p.Ly, p.Lxi, p.dt
    c.psi_floor = p.psi_floor
    c.seed = p.seed
    c.spin_limit = p.spin_limit
    for i, s in enumerate(p.species):
        cs = c.species[i]
        cs.Z, cs.M, cs.alpha, cs.gamma_b = s.Z, s.M, s.alpha, s.gamma_b
        cs.gamma_spread_rel, cs.uperp_spread, cs.noise_rel = (s.gamma_spread_rel,
                                                              s.uperp_spread, s.noise_rel)
        cs.ppc_x, cs.ppc_y, cs.ppc_xi = s.ppc_x, s.ppc_y, s.ppc_xi
        cs.seeded = 1 if s.seeded else 0
        cs.xi_front, cs.xi_back = s.xi_front, s.xi_back
    for i, m in enumerate(p.modes):
        c.modes[i].mx, c.modes[i].my = m.mx, m.my
        c.modes[i].amplitude, c.modes[i].phase = m.amplitude, m.phase
    c.n_diag_modes = len(p.diag_modes)
    for i, (mx, my) in enumerate(p.diag_modes):
        c.diag_modes[i].mx, c.diag_modes[i].my = mx, my
    return c


def _ptr(a):
    return a.ctypes.data_as(_DP)


def eq5_march(gamma, psi0, dpsi0, dxi, tau_end, n_tau, n_out=1, stream=None):
    """Eq. 5 marched on the GPU for a batch of modes (qsa_eq5_march): gamma [m], psi0 and
    dpsi0 [m, n_xi] at tau = 0 on xi_i = i dxi.  Returns psi [n_out, m, n_xi] at
    tau = tau_end (o + 1) / n_out."""
    lib = load_library()
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    a = np.ascontiguousarray(psi0, dtype=np.float64)
    b = np.ascontiguousarray(dpsi0, dtype=np.float64)
    m, n = a.shape
    out = np.empty((n_out, m, n))
    strm = ct.c_void_p(stream.cuda_stream) if stream is not None else None
    rc = lib.qsa_eq5_march(m, n, float(dxi), _ptr(g), _ptr(a), _ptr(b), float(tau_end),
                           int(n_tau), int(n_out), _ptr(out), strm)
    if rc != QSA_OK:
        raise QsaError(rc, lib.qsa_last_error(None).decode())
    return out


def bounds_check():
    """(enabled, first failing source line, failures) of the bounds-checked debug build's
    index checks on the current device; enabled is False for the release build."""
    lib = load_library()
    first, count = ct.c_int64(), ct.c_int64()
    rc = lib.qsa_bounds_check(ct.byref(first), ct.byref(count))
    if rc < 0:
        raise QsaError(rc, "bounds counters could not be read")
    return rc == 1, first.value, count.value


def advance_batch(instances, n_steps: int):
    """n_steps beam steps of every QSA instance (same precision, n_pc_iter and stream), up to
    16 instances per persistent launch (qsa_advance_batch)."""
    lib = load_library()
    arr = (ct.c_void_p * len(instances))(*[q.h for q in instances])
    rc = lib.qsa_advance_batch(arr, len(instances), int(n_steps))
    if rc < 0:
        raise QsaError(rc, lib.qsa_last_error(instances[0].h if instances else None).decode())
    return rc


def batch_graphs(lead, enable=None) -> int:
    """CUDA graphs of the batched steps led by QSA instance `lead` (qsa_batch_graphs):
    enable True/False switches them, None leaves them; returns the steps run as graphs so far
    (negative, -1 - that number, when graphs are off or a capture failed)."""
    lib = load_library()
    n = ct.c_int64(0)
    e = -1 if enable is None else (1 if enable else 0)
    rc = lib.qsa_batch_graphs(lead.h, e, ct.byref(n))
    if rc < 0:
        raise QsaError(rc, lib.qsa_last_error(lead.h).decode())
    return int(n.value)


class QSA:
    """One QS-PIC instance on the current CUDA device and stream."""

    def __init__(self, p: config.Params, stream=None, torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("QSA needs a CUDA device")
        self.lib = load_library()
        self.p = p
        self.device = torch.cuda.current_device()
        self._torch_stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream = ct.c_void_p(self._torch_stream.cuda_stream)
        if torch_allocator:
            dev = self.device

            def _alloc(nbytes, ctx, strm):
                try:
                    return torch.cuda.caching_allocator_alloc(nbytes, dev, strm)
                except Exception:
                    return None

            def _free(ptr, nbytes, ctx, strm):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc = ALLOC_FN(_alloc)
            self._free = FREE_FN(_free)
        else:
            self._alloc = ALLOC_FN()
            self._free = FREE_FN()
        self._cp = to_c_params(p)
        h = ct.c_void_p()
        rc = self.lib.qsa_init(ct.byref(self._cp), self.stream, self._alloc, self._free, None,
                               ct.byref(h))
        if rc != QSA_OK:
            raise QsaError(rc, self.lib.qsa_last_error(None).decode())
        self.h = h
        self.nk = p.nxi + 1

    # -- helpers
    def _check(self, rc):
        if rc < 0:
            raise QsaError(rc, self.lib.qsa_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.qsa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the hot path
    def sweep(self):
        return self._check(self.lib.qsa_plasma_sweep(self.h))

    def beam_step(self):
        return self._check(self.lib.qsa_beam_step(self.h))

    def advance(self, n_steps: int):
        """n_steps x (sweep, beam step); pipelined launches when p.pipeline_depth >= 2."""
        return self._check(self.lib.qsa_advance(self.h, int(n_steps)))

    def rehome(self):
        """Move every beam particle into a storage slot of the cell it occupies (qsa_rehome)."""
        return self._check(self.lib.qsa_rehome(self.h))

    def rehome_count(self) -> int:
        return int(self.lib.qsa_rehome_count(self.h))

    def launch_times(self) -> np.ndarray:
        """Device ms of each persistent launch of the last pipelined advance()."""
        out = np.zeros(64, dtype=np.float32)
        n = ct.c_int()
        self._check(self.lib.qsa_launch_times(
            self.h, out.ctypes.data_as(ct.POINTER(ct.c_float)), out.size, ct.byref(n)))
        return out[:n.value].copy()

    # -- gradients (discrete adjoint, FP64 handles)
    def grad_forward(self, n_steps: int, step_ckpt: int = 10) -> float:
        """n_steps beam steps and the final sweep from the beam qsa_init built, recorded for
        grad_backward (qsa_grad_forward); returns 1/2 sum (B_x^2 + B_y^2) dx dy dxi of the
        final sweep."""
        loss = ct.c_double()
        self._check(self.lib.qsa_grad_forward(self.h, int(n_steps), int(step_ckpt),
                                              ct.byref(loss)))
        return loss.value

    def grad_backward(self, dloss: float = 1.0):
        """dloss times the gradient of the recorded loss with respect to the seeded mode
        amplitudes [n_modes] and each species' alpha [n_species] (qsa_grad_backward)."""
        dm = np.zeros(max(len(self.p.modes), 1))
        da = np.zeros(max(len(self.p.species), 1))
        self._check(self.lib.qsa_grad_backward(self.h, float(dloss), _ptr(dm), _ptr(da)))
        return dm[:len(self.p.modes)], da[:len(self.p.species)]

    # -- data in / out
    def set_beam(self, si: int, b: dict):
        arrs = [np.ascontiguousarray(b[k], dtype=np.float64)
                for k in ("x", "y", "xi", "ux", "uy", "uz", "w")]
        n = arrs[0].size
        return self._check(self.lib.qsa_set_beam(self.h, si, n, *[_ptr(a) for a in arrs]))

    def get_beam(self, si: int, n: int) -> dict:
        keys = ("x", "y", "xi", "ux", "uy", "uz", "w")
        arrs = [np.empty(n) for _ in keys]
        nout = ct.c_int64()
        self._check(self.lib.qsa_get_beam(self.h, si, n, *[_ptr(a) for a in arrs],
                                          ct.byref(nout)))
        return dict(zip(keys, arrs))

    def diagnostics(self, seg_width: float = 2.0) -> dict:
        """Per-slice diagnostics of the last sweep (see qsa_diag).  Adds "beam_rms_u":
        [species, xi cell, 3] weighted rms spread of u_x, u_y, u_z, and "beam_weight":
        [species, xi cell] sum of w/wbar, both derived from the raw moment sums."""
        nk, p = self.nk, self.p
        out = {k: np.zeros(nk) for k in ("psi0", "ez0", "jz_mean", "kappa2", "opp_min",
                                          "n_floor", "invariant", "charge", "pc_residual",
                                          "pc_iters")}
        out["energy"] = np.zeros((nk, 6))
        out["rms"] = np.zeros((nk, 6))
        nseg = max(1, int(np.ceil(p.Lxi / seg_width - 1e-12)))
        out["rms_seg"] = np.zeros((nseg, 6))
        out["mode_amp"] = np.zeros((nk, max(len(p.diag_modes), 1), 5, 2))
        out["beam_moments"] = np.zeros((max(len(p.species), 1), max(p.nxi, 1), 7))
        d = Diag()
        d.seg_width = seg_width
        for k, v in out.items():
            setattr(d, k, _ptr(v))
        rc = self.lib.qsa_diagnostics(self.h, ct.byref(d))
        out["status"] = rc
        out["beam_lost"] = d.beam_lost
        out["sweeps"] = d.sweeps
        self._check(rc)
        m = out["beam_moments"]
        wsum = m[..., 0]
        with np.errstate(invalid="ignore", divide="ignore"):
            mean = m[..., 1:4] / wsum[..., None]
            var = m[..., 4:7] / wsum[..., None] - mean ** 2
        out["beam_weight"] = wsum
        out["beam_rms_u"] = np.sqrt(np.maximum(var, 0.0))
        return out

    def field(self, f, j0=0, j1=None) -> np.ndarray:
        j1 = self.nk if j1 is None else j1
        fi = FIELDS.index(f) if isinstance(f, str) else int(f)
        out = np.empty((j1 - j0, self.p.ny, self.p.nx))
        self._check(self.lib.qsa_copy_field(self.h, fi, j0, j1, _ptr(out)))
        return out

    def slab(self, j0=0, j1=None) -> np.ndarray:
        """Fields of slices j0..j1-1 as [j, 6, ny, nx] (Wx, Wy, Ez, Bx, By, Bz)."""
        return np.stack([self.field(f, j0, j1) for f in range(6)], axis=1)

    def source(self, q, j0=0, j1=None) -> np.ndarray:
        j1 = self.nk if j1 is None else j1
        qi = SOURCES.index(q) if isinstance(q, str) else int(q)
        out = np.empty((j1 - j0, self.p.ny, self.p.nx))
        self._check(self.lib.qsa_copy_source(self.h, qi, j0, j1, _ptr(out)))
        return out

    def field_solve(self, S, Jx, Jy, Jz, Dx, Dy, kappa2=0.0) -> dict:
        ins = [np.ascontiguousarray(a, dtype=np.float64) for a in (S, Jx, Jy, Jz, Dx, Dy)]
        out = np.empty((7, self.p.ny, self.p.nx))
        self._check(self.lib.qsa_field_solve(self.h, *[_ptr(a) for a in ins], kappa2, _ptr(out)))
        return dict(zip(("psi", "gpx", "gpy", "Ez", "Bz", "Bx", "By"), out))

    def phase_times(self) -> np.ndarray:
        """[8 slices, 32 phases, 2] globaltimer stamps (ns) of the last sweep: last arrival
        at each phase's closing barrier, and block 0's exit from it (0 = not recorded)."""
        out = np.zeros(8 * 32 * 2, dtype=np.int64)
        self._check(self.lib.qsa_phase_times(self.h, out.ctypes.data_as(ct.POINTER(ct.c_int64)),
                                             out.size))
        return out.reshape(8, 32, 2)

    def launch_count(self) -> int:
        return int(self.lib.qsa_launch_count(self.h))

    def device_bytes(self) -> int:
        return int(self.lib.qsa_device_bytes(self.h))
