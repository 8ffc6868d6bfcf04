"""GB300-native long-range step of Ewald summation with prolates (ESP).

Thin ctypes binding of the C ABI in ``include/esp.h`` (libesp.so, built in-tree by
``paper_2601_00161_gb300/build.py``).  Every step of the computation runs in the library's
CUDA kernels and cuFFT; this module only marshals arguments.  PyTorch supplies device
memory and streams.  There is no CPU fallback: importing the binding fails loudly when
the shared library is missing.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libesp.so")

ESP_OK = 0
ESP_ERR_ARG = -1
ESP_ERR_CELL = -2
ESP_ERR_GRID = -3
ESP_ERR_SUPPORT = -4
ESP_ERR_NONFINITE = -5
ESP_ERR_CUDA = -6
ESP_ERR_CUFFT = -7
ESP_ERR_TIMEOUT = -8
ESP_ERR_STATE = -9

ESP_FP64 = 0
ESP_FP32 = 1
ESP_IO_F64 = 16
ESP_BF16_GRID = 32
ESP_ACCUM_LEN = 16

# every symbol include/esp.h declares
EXPORTS = (
    "esp_plan", "esp_set_cell", "esp_set_stream", "esp_step", "esp_energy_pressure",
    "esp_forces", "esp_forces_from_spectrum", "esp_compute_host", "esp_result_from_accum",
    "esp_copy_grid", "esp_copy_spectrum", "esp_plan_info", "esp_destroy", "esp_last_error",
    "esp_c_from_tolerance", "esp_profile", "esp_profile_read", "esp_spread_noalloc",
    "esp_cell_gradient", "esp_near", "esp_forces_ik", "esp_local_virial", "esp_atom_energy",
    "esp_pressure_coupling",
)

ESP_COUPLE_ISO, ESP_COUPLE_SEMI, ESP_COUPLE_ANISO, ESP_COUPLE_FLEXIBLE = 0, 1, 2, 3

ESP_NOALLOC_MAX_ATOMS = 65536
ESP_NOALLOC_MAX_TILES = 4096

STAGES = ("memset", "bin", "scan", "scatter", "zero_grid", "spread", "fft_fwd", "xfft_scale",
          "fft_inv", "gather")


class esp_result(ctypes.Structure):
    _fields_ = [
        ("energy_recip", ctypes.c_double),
        ("energy_self", ctypes.c_double),
        ("energy_bg", ctypes.c_double),
        ("virial_recip", ctypes.c_double * 9),
        ("pressure_recip", ctypes.c_double * 9),
        ("pressure_bg", ctypes.c_double),
        ("volume", ctypes.c_double),
        ("qsum", ctypes.c_double),
        ("q2sum", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {
            "energy_recip": self.energy_recip,
            "energy_self": self.energy_self,
            "energy_bg": self.energy_bg,
            "virial_recip": np.array(self.virial_recip).reshape(3, 3),
            "pressure_recip": np.array(self.pressure_recip).reshape(3, 3),
            "pressure_bg": self.pressure_bg,
            "volume": self.volume,
            "qsum": self.qsum,
            "q2sum": self.q2sum,
        }


class ESPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ESP error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python paper_2601_00161_gb300/build.py` "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    dptr = ctypes.POINTER(ctypes.c_double)
    sig = {
        "esp_plan": (ci, [ctypes.POINTER(vp), dptr, i64, ctypes.POINTER(ci), ci, cd, cd, ci, vp]),
        "esp_set_cell": (ci, [vp, dptr]),
        "esp_set_stream": (ci, [vp, vp]),
        "esp_step": (ci, [vp, vp, vp, vp, vp]),
        "esp_energy_pressure": (ci, [vp, vp, vp, ctypes.POINTER(esp_result)]),
        "esp_forces": (ci, [vp, vp, vp, vp]),
        "esp_forces_from_spectrum": (ci, [vp, vp]),
        "esp_compute_host": (ci, [vp, vp, vp, vp, ctypes.POINTER(esp_result)]),
        "esp_result_from_accum": (ci, [vp, dptr, ctypes.POINTER(esp_result)]),
        "esp_copy_grid": (ci, [vp, vp]),
        "esp_copy_spectrum": (ci, [vp, vp]),
        "esp_plan_info": (ci, [vp, dptr, ci]),
        "esp_destroy": (ci, [vp]),
        "esp_last_error": (ctypes.c_char_p, [vp]),
        "esp_c_from_tolerance": (cd, [cd]),
        "esp_pressure_coupling": (ci, [dptr, ci, dptr]),
        "esp_profile": (ci, [vp, ci]),
        "esp_profile_read": (ci, [vp, dptr, ci]),
        "esp_spread_noalloc": (ci, [dptr, i64, ctypes.POINTER(ci), ci, cd, ci, vp, vp, vp, vp]),
        "esp_cell_gradient": (ci, [vp, vp, vp, vp, vp]),
        "esp_near": (ci, [vp, vp, vp, vp, ci, vp]),
        "esp_forces_ik": (ci, [vp, vp, vp, vp]),
        "esp_local_virial": (ci, [vp, vp, vp, vp]),
        "esp_atom_energy": (ci, [vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _check(code: int, plan=None):
    if code != ESP_OK:
        msg = _lib.esp_last_error(plan)
        raise ESPError(code, msg.decode() if msg else "")


def _cell_colmajor(cell) -> ctypes.Array:
    h = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    return (ctypes.c_double * 9)(*h.T.ravel())  # columns of h = cell vectors


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# ---- the C ABI, same names ---------------------------------------------------------------
def esp_plan(cell, n, grid, w, c, alpha, precision=ESP_FP64, stream=None):
    h = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    code = _lib.esp_plan(ctypes.byref(h), _cell_colmajor(cell), int(n), g, int(w), float(c),
                         float(alpha), int(precision), ctypes.c_void_p(stream) if stream else None)
    _check(code, None)
    return h


def esp_set_cell(plan, cell):
    _check(_lib.esp_set_cell(plan, _cell_colmajor(cell)), plan)


def esp_set_stream(plan, stream):
    _check(_lib.esp_set_stream(plan, ctypes.c_void_p(stream) if stream else None), plan)


def esp_step(plan, pos, q, forces=None, accum=None):
    _check(_lib.esp_step(plan, _ptr(pos), _ptr(q), _ptr(forces), _ptr(accum)), plan)


def esp_energy_pressure(plan, pos, q) -> esp_result:
    out = esp_result()
    _check(_lib.esp_energy_pressure(plan, _ptr(pos), _ptr(q), ctypes.byref(out)), plan)
    return out


def esp_forces(plan, pos, q, forces):
    _check(_lib.esp_forces(plan, _ptr(pos), _ptr(q), _ptr(forces)), plan)


def esp_forces_from_spectrum(plan, forces):
    _check(_lib.esp_forces_from_spectrum(plan, _ptr(forces)), plan)


def esp_cell_gradient(plan, pos, forces, accum, grad):
    _check(_lib.esp_cell_gradient(plan, _ptr(pos), _ptr(forces), _ptr(accum), _ptr(grad)), plan)


def esp_forces_ik(plan, pos, q, forces):
    _check(_lib.esp_forces_ik(plan, _ptr(pos), _ptr(q), _ptr(forces)), plan)


def esp_local_virial(plan, pos, q, virial):
    _check(_lib.esp_local_virial(plan, _ptr(pos), _ptr(q), _ptr(virial)), plan)


def esp_atom_energy(plan, pos, q, energy):
    _check(_lib.esp_atom_energy(plan, _ptr(pos), _ptr(q), _ptr(energy)), plan)


def esp_near(plan, pos, q, forces, add, out):
    _check(_lib.esp_near(plan, _ptr(pos), _ptr(q), _ptr(forces), int(add), _ptr(out)), plan)


def esp_compute_host(plan, pos: np.ndarray, q: np.ndarray, forces: np.ndarray | None):
    out = esp_result()
    fp = forces.ctypes.data_as(ctypes.c_void_p) if forces is not None else None
    _check(_lib.esp_compute_host(plan, pos.ctypes.data_as(ctypes.c_void_p),
                                 q.ctypes.data_as(ctypes.c_void_p), fp, ctypes.byref(out)), plan)
    return out


def esp_result_from_accum(plan, accum_host) -> esp_result:
    a = np.ascontiguousarray(accum_host, dtype=np.float64)
    out = esp_result()
    _check(_lib.esp_result_from_accum(plan, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ctypes.byref(out)), plan)
    return out


def esp_copy_grid(plan, dst: np.ndarray):
    _check(_lib.esp_copy_grid(plan, dst.ctypes.data_as(ctypes.c_void_p)), plan)


def esp_copy_spectrum(plan, dst: np.ndarray):
    _check(_lib.esp_copy_spectrum(plan, dst.ctypes.data_as(ctypes.c_void_p)), plan)


def esp_plan_info(plan) -> dict:
    v = (ctypes.c_double * 18)()
    _check(_lib.esp_plan_info(plan, v, 18), plan)
    keys = ["c", "rc", "psi0_at_0", "C0", "lambda0", "deg", "rdeg", "fit_err", "rfit_err",
            "ntiles", "T1", "T2", "T3", "launches", "Xbg", "box_mode", "nb1", "nb2"]
    return dict(zip(keys, list(v)))


def esp_destroy(plan):
    _lib.esp_destroy(plan)


def esp_last_error(plan=None) -> str:
    m = _lib.esp_last_error(plan)
    return m.decode() if m else ""


def esp_c_from_tolerance(delta: float) -> float:
    c = _lib.esp_c_from_tolerance(float(delta))
    if c < 0:
        raise ESPError(ESP_ERR_ARG, "delta must lie in (0, 1)")
    return c


def esp_pressure_coupling(P, mode: int):
    """The pressure a barostat's cell coupling sees (ESP_COUPLE_*) from a 3x3 tensor."""
    import numpy as np

    a = np.ascontiguousarray(np.asarray(P, dtype=np.float64).reshape(9))
    out = np.zeros(6)
    k = _lib.esp_pressure_coupling(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(mode),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if k < 0:
        raise ESPError(k, esp_last_error(None))
    return out[:k].copy()


def esp_profile(plan, enable: bool):
    _check(_lib.esp_profile(plan, 1 if enable else 0), plan)


def esp_profile_read(plan) -> dict:
    v = (ctypes.c_double * len(STAGES))()
    _check(_lib.esp_profile_read(plan, v, len(STAGES)), plan)
    return dict(zip(STAGES, list(v)))


def esp_spread_noalloc(cell, n, grid, w, c, precision, pos, q, grid_out, stream=None):
    """Spreading with the library's static scratch (no device allocation); see esp.h."""
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    _check(_lib.esp_spread_noalloc(_cell_colmajor(cell), int(n), g, int(w), float(c),
                                   int(precision), _ptr(pos), _ptr(q), _ptr(grid_out),
                                   ctypes.c_void_p(stream) if stream else None), None)


# ---- convenience wrapper over torch tensors ----------------------------------------------
class Plan:
    """Owns an esp_plan_t.  Positions / charges / forces are torch CUDA tensors."""

    def __init__(self, cell, n, grid, P, c, rc, precision="fp64", io_double=None, stream=None):
        """precision: "fp64", "fp32", or "fp32_bf16grid" (FP32 with the potential grid
        stored in BF16 between the inverse transform and the force gather)."""
        import torch

        if precision not in ("fp64", "fp32", "fp32_bf16grid"):
            raise ValueError("precision must be fp64, fp32 or fp32_bf16grid")
        self.torch = torch
        self.fp64 = precision == "fp64"
        self.io_double = self.fp64 if io_double is None else bool(io_double)
        flags = ESP_FP64 if self.fp64 else ESP_FP32
        if not self.fp64 and self.io_double:
            flags |= ESP_IO_F64
        if precision == "fp32_bf16grid":
            flags |= ESP_BF16_GRID
        self.io_dtype = torch.float64 if self.io_double else torch.float32
        self.n = int(n)
        self.grid = tuple(int(x) for x in grid)
        self.P, self.c, self.rc = int(P), float(c), float(rc)
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        self.handle = esp_plan(cell, n, grid, P, c, rc, flags, st)
        self.cell = np.array(cell, dtype=np.float64).reshape(3, 3)

    def close(self):
        if getattr(self, "handle", None):
            esp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _in(self, pos, q):
        t = self.torch
        pos = t.as_tensor(pos, dtype=self.io_dtype, device="cuda").contiguous()
        q = t.as_tensor(q, dtype=self.io_dtype, device="cuda").contiguous()
        if pos.shape != (self.n, 3) or q.shape != (self.n,):
            raise ValueError("pos must be [n, 3] and q [n]")
        return pos, q

    def set_cell(self, cell):
        esp_set_cell(self.handle, cell)
        self.cell = np.array(cell, dtype=np.float64).reshape(3, 3)

    def energy_pressure(self, pos, q) -> dict:
        pos, q = self._in(pos, q)
        return esp_energy_pressure(self.handle, pos, q).as_dict()

    def forces(self, pos, q, out=None):
        pos, q = self._in(pos, q)
        if out is None:
            out = self.torch.empty((self.n, 3), dtype=self.io_dtype, device="cuda")
        esp_forces(self.handle, pos, q, out)
        return out

    def step(self, pos, q, forces=None, accum=None):
        esp_step(self.handle, pos, q, forces, accum)

    def compute(self, pos, q) -> tuple[dict, "object"]:
        """Energy, pressure and forces (one full step)."""
        pos, q = self._in(pos, q)
        F = self.torch.empty((self.n, 3), dtype=self.io_dtype, device="cuda")
        acc = self.torch.zeros(ESP_ACCUM_LEN, dtype=self.torch.float64, device="cuda")
        esp_step(self.handle, pos, q, F, acc)
        res = esp_result_from_accum(self.handle, acc.cpu().numpy()).as_dict()
        return res, F

    def near(self, pos, q, forces=None, add=False):
        """Near part of the split: (U_N, W_N 3x3, forces).  ``forces`` is overwritten, or
        added to when ``add``."""
        pos, q = self._in(pos, q)
        if forces is None:
            forces = self.torch.zeros((self.n, 3), dtype=self.io_dtype, device="cuda")
        out = self.torch.empty(7, dtype=self.torch.float64, device="cuda")
        esp_near(self.handle, pos, q, forces, add, out)
        o = out.cpu().numpy()
        W = np.array([[o[1], o[4], o[5]], [o[4], o[2], o[6]], [o[5], o[6], o[3]]])
        return float(o[0]), W, forces

    def forces_ik(self, pos, q):
        """Forces by ik-differentiation (momentum-conserving variant)."""
        pos, q = self._in(pos, q)
        out = self.torch.empty((self.n, 3), dtype=self.io_dtype, device="cuda")
        esp_forces_ik(self.handle, pos, q, out)
        return out

    def local_virial(self, pos, q):
        """Per-atom long-range virial [n, 6] (xx yy zz xy xz yz); divide by V for pressure."""
        pos, q = self._in(pos, q)
        out = self.torch.empty((self.n, 6), dtype=self.io_dtype, device="cuda")
        esp_local_virial(self.handle, pos, q, out)
        return out

    def atom_energy(self, pos, q):
        """Per-atom Fourier energy [n]; sums to the reciprocal energy."""
        pos, q = self._in(pos, q)
        out = self.torch.empty(self.n, dtype=self.io_dtype, device="cuda")
        esp_atom_energy(self.handle, pos, q, out)
        return out

    def info(self) -> dict:
        return esp_plan_info(self.handle)

    def grid_values(self) -> np.ndarray:
        a = np.empty(self.grid, dtype=np.float64 if self.fp64 else np.float32)
        esp_copy_grid(self.handle, a)
        return a

    def spectrum(self) -> np.ndarray:
        shp = (self.grid[0], self.grid[1], self.grid[2] // 2 + 1)
        a = np.empty(shp, dtype=np.complex128 if self.fp64 else np.complex64)
        esp_copy_spectrum(self.handle, a)
        return a


from .autograd import LongRangeEnergy, long_range_energy  # noqa: E402,F401
