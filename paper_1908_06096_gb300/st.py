"""Thin ctypes binding over the C ABI in include/st.h and include/st_stages.h.

Argument marshalling only: every step of the transform runs in the CUDA
library (libst.so next to this file).  PyTorch supplies device memory and
streams.  There is no fallback: if the library is missing or fails to load,
the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libst.so")

ST_GRID_REGULAR, ST_GRID_OCTAHEDRAL = 0, 1
ST_FP64, ST_FP32_TC, ST_BF16X3, ST_FP32_SIMT = 0, 1, 2, 3
PRECISIONS = {"fp64": ST_FP64, "tf32x3": ST_FP32_TC, "bf16x3": ST_BF16X3, "fp32": ST_FP32_SIMT}
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
          4: "device-side wait timed out", 5: "unsupported", 6: "busy"}


class STError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)}" + (f" ({detail})" if detail else ""))


class _GridDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nlat", ctypes.c_int), ("nlon", ctypes.c_int)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("nlat", ctypes.c_int), ("kind", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_fields", ctypes.c_int), ("max_m", ctypes.c_int),
                ("spec_elems", ctypes.c_size_t), ("grid_points", ctypes.c_size_t),
                ("element_bytes", ctypes.c_size_t), ("device_bytes", ctypes.c_size_t),
                ("table_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t),
                ("launch_shape", ctypes.c_int * 6)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("direction", ctypes.c_int), ("spec_in", ctypes.c_void_p),
                ("grid", ctypes.c_void_p), ("spec_out", ctypes.c_void_p), ("nfields", ctypes.c_int)]


class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double),
                ("timed", ctypes.c_longlong)]


_lib = None

# (name, argtypes) of every exported entry point; the ABI test checks this
# list against the declarations in include/*.h.
_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "st_plan_create": [ctypes.POINTER(_VP), _I, ctypes.POINTER(_GridDesc), _I, _I, _VP],
    "st_plan_destroy": [_VP],
    "st_plan_create_shared": [ctypes.POINTER(_VP), _VP, _I, _VP],
    "st_plan_inject": [_VP, _I, ctypes.c_uint],
    "st_plan_autotune": [_VP, _I, ctypes.c_char_p, _VP],
    "st_plan_query": [_VP, ctypes.POINTER(_PlanInfo)],
    "st_plan_row_lengths": [_VP, ctypes.POINTER(ctypes.c_int)],
    "st_plan_nodes": [_VP, _D, _D],
    "st_inv_trans": [_VP, _VP, _VP, _I, _VP],
    "st_dir_trans": [_VP, _VP, _VP, _I, _VP],
    "st_plan_sync": [_VP, _VP],
    "st_status_string": [_I],
    "st_last_error": [],
    "st_gauss_nodes": [_I, _VP, _VP, _VP],
    "st_legendre_values": [_I, _VP, _I, _VP, _VP],
    "st_inv_legendre": [_VP, _VP, _I, _VP],
    "st_inv_fft": [_VP, _VP, _I, _VP],
    "st_dir_fft": [_VP, _VP, _I, _VP],
    "st_dir_legendre": [_VP, _VP, _I, _VP],
    "st_fourier_export": [_VP, _I, _I, _VP, _VP],
    "st_plan_set_timing": [_VP, _I],
    "st_plan_timings": [_VP, ctypes.POINTER(_KernelTime), _I, ctypes.POINTER(ctypes.c_int)],
    "st_plan_reset_timings": [_VP],
    "st_inv_trans_static": [_VP, _VP, _VP, _I, _VP],
    "st_batch_create": [ctypes.POINTER(_VP), ctypes.POINTER(_BatchItem), _I],
    "st_batch_run": [_VP, _VP, _I],
    "st_batch_destroy": [_VP],
    "st_static_scratch_bytes": [],
    "st_build_info": [ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "st_plan_save_tables": [_VP, ctypes.c_char_p],
    "st_plan_load_tables": [_VP, ctypes.c_char_p],
    "st_plan_enable_derivatives": [_VP, _VP],
    "st_inv_trans_deriv": [_VP, _VP, _VP, _I, _VP],
    "st_inv_trans_uv": [_VP, _VP, _VP, _I, _VP],
    "st_dir_trans_vordiv": [_VP, _VP, _VP, _I, _VP],
}


def ensure_built():
    """Compile the library if it is missing or stale (nvcc, sm_103a)."""
    from . import build
    build.build()
    return load()


def load():
    """Load libst.so (raises if it is not there)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.st_static_scratch_bytes.restype = ctypes.c_size_t
    lib.st_status_string.restype = ctypes.c_char_p
    lib.st_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != 0:
        raise STError(rc, what, load().st_last_error().decode())


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t: torch.Tensor) -> int:
    return int(t.data_ptr())


def build_info():
    """(compute capability major, minor, kernel binary version) from st_build_info."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().st_build_info(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "st_build_info")
    return a.value, b.value, c.value


def gauss_nodes(nlat: int, stream=None):
    """Device FP64 Gauss-Legendre nodes and weights (north to south)."""
    mu = torch.empty(nlat, dtype=torch.float64, device="cuda")
    w = torch.empty(nlat, dtype=torch.float64, device="cuda")
    _check(load().st_gauss_nodes(nlat, _ptr(mu), _ptr(w), _stream_handle(stream)), "st_gauss_nodes")
    return mu, w


def legendre_values(T: int, mu: torch.Tensor, stream=None):
    """Device FP64 Pbar_n^m(mu_i) for all (m, n <= T): [len(mu), (T+1)(T+2)/2]."""
    mu = mu.to(device="cuda", dtype=torch.float64).contiguous()
    out = torch.empty((mu.numel(), (T + 1) * (T + 2) // 2), dtype=torch.float64, device="cuda")
    _check(load().st_legendre_values(T, _ptr(mu), mu.numel(), _ptr(out), _stream_handle(stream)),
           "st_legendre_values")
    return out


class Plan:
    """A transform plan: st.Plan(T, "regular"|"octahedral", nlat, nlon, precision, max_fields).

    ``inv(spec)`` takes [nfields, nspec, 2] (re, im) and returns
    [nfields, grid_points]; ``dir(grid)`` the reverse.  Element type is
    float64 for precision "fp64" and float32 otherwise.  Both run
    asynchronously on the current (or given) torch stream.
    """

    def __init__(self, T: int, grid: str = "regular", nlat: int | None = None, nlon: int | None = None,
                 precision: str = "bf16x3", max_fields: int = 1, stream=None, share_with: "Plan | None" = None):
        lib = load()
        if share_with is not None:
            src = share_with
            self.T, self.grid, self.nlat, self.nlon = src.T, src.grid, src.nlat, src.nlon
            self.precision, self.prec_code, self.max_fields = src.precision, src.prec_code, max_fields
            h = _VP()
            _check(lib.st_plan_create_shared(ctypes.byref(h), src.handle, max_fields, _stream_handle(stream)),
                   "st_plan_create_shared")
            self._h = h
            info = _PlanInfo()
            _check(lib.st_plan_query(h, ctypes.byref(info)), "st_plan_query")
            self.info = info
            self.nspec = int(info.spec_elems)
            self.npts = int(info.grid_points)
            self.dtype = src.dtype
            return
        if nlat is None:
            nlat = T + 1 if grid == "regular" else 2 * (T + 1)
            nlat += nlat & 1
        if nlon is None:
            nlon = 2 * nlat if grid == "regular" else 0
        self.T, self.grid, self.nlat, self.nlon = T, grid, nlat, nlon
        self.precision = precision
        self.prec_code = PRECISIONS[precision]
        self.max_fields = max_fields
        desc = _GridDesc(ST_GRID_REGULAR if grid == "regular" else ST_GRID_OCTAHEDRAL, nlat, nlon)
        h = _VP()
        _check(lib.st_plan_create(ctypes.byref(h), T, ctypes.byref(desc), self.prec_code, max_fields,
                                  _stream_handle(stream)), "st_plan_create")
        self._h = h
        info = _PlanInfo()
        _check(lib.st_plan_query(h, ctypes.byref(info)), "st_plan_query")
        self.info = info
        self.nspec = int(info.spec_elems)
        self.npts = int(info.grid_points)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().st_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def row_lengths(self):
        arr = (ctypes.c_int * self.nlat)()
        _check(load().st_plan_row_lengths(self._h, arr), "st_plan_row_lengths")
        return list(arr)

    def nodes(self):
        import numpy as np
        mu = np.zeros(self.nlat)
        w = np.zeros(self.nlat)
        _check(load().st_plan_nodes(self._h, mu.ctypes.data_as(_D), w.ctypes.data_as(_D)), "st_plan_nodes")
        return mu, w

    def _nf(self, t: torch.Tensor, per: int) -> int:
        assert t.is_cuda and t.dtype == self.dtype and t.is_contiguous(), (t.device, t.dtype)
        assert t.numel() % per == 0, (t.shape, per)
        return t.numel() // per

    def inv(self, spec: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        nf = self._nf(spec, self.nspec * 2)
        if out is None:
            out = torch.empty((nf, self.npts), dtype=self.dtype, device=spec.device)
        _check(load().st_inv_trans(self._h, _ptr(spec), _ptr(out), nf, _stream_handle(stream)), "st_inv_trans")
        return out

    def inv_static(self, spec: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Inverse transform through st_inv_trans_static (scratch in the
        library's fixed device array; no allocation inside the call)."""
        nf = self._nf(spec, self.nspec * 2)
        if out is None:
            out = torch.empty((nf, self.npts), dtype=self.dtype, device=spec.device)
        _check(load().st_inv_trans_static(self._h, _ptr(spec), _ptr(out), nf, _stream_handle(stream)),
               "st_inv_trans_static")
        return out

    def dir(self, grid: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        nf = self._nf(grid, self.npts)
        if out is None:
            out = torch.empty((nf, self.nspec, 2), dtype=self.dtype, device=grid.device)
        _check(load().st_dir_trans(self._h, _ptr(grid), _ptr(out), nf, _stream_handle(stream)), "st_dir_trans")
        return out

    def save_tables(self, path: str):
        _check(load().st_plan_save_tables(self._h, path.encode()), "st_plan_save_tables")

    def load_tables(self, path: str):
        _check(load().st_plan_load_tables(self._h, path.encode()), "st_plan_load_tables")

    # -- derivative and wind transforms (unit sphere; U = u cos(phi), V = v cos(phi))
    def enable_derivatives(self, stream=None):
        _check(load().st_plan_enable_derivatives(self._h, _stream_handle(stream)), "st_plan_enable_derivatives")

    def inv_deriv(self, spec: torch.Tensor, stream=None):
        """(dF/dlambda, cos(phi) dF/dphi), each [nfields, grid_points]."""
        nf = self._nf(spec, self.nspec * 2)
        out = torch.empty((2 * nf, self.npts), dtype=self.dtype, device=spec.device)
        _check(load().st_inv_trans_deriv(self._h, _ptr(spec), _ptr(out), nf, _stream_handle(stream)),
               "st_inv_trans_deriv")
        return out[:nf], out[nf:]

    def inv_uv(self, vor: torch.Tensor, div: torch.Tensor, stream=None):
        """Wind images (U, V), each [nfields, grid_points], from vorticity and divergence spectra."""
        nf = self._nf(vor, self.nspec * 2)
        vd = torch.cat([vor.reshape(nf, self.nspec, 2), div.reshape(nf, self.nspec, 2)]).contiguous()
        out = torch.empty((2 * nf, self.npts), dtype=self.dtype, device=vor.device)
        _check(load().st_inv_trans_uv(self._h, _ptr(vd), _ptr(out), nf, _stream_handle(stream)), "st_inv_trans_uv")
        return out[:nf], out[nf:]

    def dir_vordiv(self, U: torch.Tensor, V: torch.Tensor, stream=None):
        """(vorticity, divergence) spectra [nfields, nspec, 2] from wind images U, V."""
        nf = self._nf(U, self.npts)
        uv = torch.cat([U.reshape(nf, self.npts), V.reshape(nf, self.npts)]).contiguous()
        out = torch.empty((2 * nf, self.nspec, 2), dtype=self.dtype, device=U.device)
        _check(load().st_dir_trans_vordiv(self._h, _ptr(uv), _ptr(out), nf, _stream_handle(stream)),
               "st_dir_trans_vordiv")
        return out[:nf], out[nf:]

    def autotune(self, nfields: int | None = None, cache_path: str | None = None, stream=None):
        """Time candidate launch shapes on this plan and keep the fastest
        (st_plan_autotune); optionally append the choice to cache_path."""
        nf = self.max_fields if nfields is None else nfields
        _check(load().st_plan_autotune(self._h, nf, cache_path.encode() if cache_path else None,
                                       _stream_handle(stream)), "st_plan_autotune")

    def launch_shape(self):
        info = _PlanInfo()
        _check(load().st_plan_query(self._h, ctypes.byref(info)), "st_plan_query")
        return list(info.launch_shape)

    def set_timing(self, enable: bool):
        _check(load().st_plan_set_timing(self._h, 1 if enable else 0), "st_plan_set_timing")

    def reset_timings(self):
        _check(load().st_plan_reset_timings(self._h), "st_plan_reset_timings")

    def timings(self) -> dict:
        """{kernel name: {"launches", "timed", "total_ms"}} since the last reset."""
        arr = (_KernelTime * 16)()
        n = ctypes.c_int()
        _check(load().st_plan_timings(self._h, arr, 16, ctypes.byref(n)), "st_plan_timings")
        return {arr[i].name.decode(): {"launches": int(arr[i].launches), "timed": int(arr[i].timed),
                                       "total_ms": float(arr[i].total_ms)} for i in range(min(n.value, 16))}

    def sync(self, stream=None):
        _check(load().st_plan_sync(self._h, _stream_handle(stream)), "st_plan_sync")

    # -- stages
    def inv_legendre(self, spec, stream=None):
        nf = self._nf(spec, self.nspec * 2)
        _check(load().st_inv_legendre(self._h, _ptr(spec), nf, _stream_handle(stream)), "st_inv_legendre")
        return nf

    def inv_fft(self, nf, out=None, stream=None):
        if out is None:
            out = torch.empty((nf, self.npts), dtype=self.dtype, device="cuda")
        _check(load().st_inv_fft(self._h, _ptr(out), nf, _stream_handle(stream)), "st_inv_fft")
        return out

    def dir_fft(self, grid, stream=None):
        nf = self._nf(grid, self.npts)
        _check(load().st_dir_fft(self._h, _ptr(grid), nf, _stream_handle(stream)), "st_dir_fft")
        return nf

    def dir_legendre(self, nf, out=None, stream=None):
        if out is None:
            out = torch.empty((nf, self.nspec, 2), dtype=self.dtype, device="cuda")
        _check(load().st_dir_legendre(self._h, _ptr(out), nf, _stream_handle(stream)), "st_dir_legendre")
        return out

    def fourier_export(self, direction: int, nf: int, stream=None) -> torch.Tensor:
        """Fourier buffer as complex128 [2, T+1, nlat/2, nf]."""
        J = self.nlat // 2
        out = torch.empty((2, self.T + 1, J, nf, 2), dtype=torch.float64, device="cuda")
        _check(load().st_fourier_export(self._h, direction, nf, _ptr(out), _stream_handle(stream)),
               "st_fourier_export")
        return torch.view_as_complex(out)


class Batch:
    """Many transforms in one set of launches (st_batch_*).

    items: list of (plan, direction, spec_in, grid, spec_out) with direction
    "inv", "dir" or "round" and torch tensors (None where unused).  The
    tensors must stay alive as long as the batch.
    """

    DIRS = {"inv": 0, "dir": 1, "round": 2}

    def __init__(self, items):
        lib = load()
        arr = (_BatchItem * len(items))()
        self._keep = []
        for i, (plan, direction, spec_in, grid, spec_out) in enumerate(items):
            nf = grid.numel() // plan.npts
            arr[i] = _BatchItem(plan.handle.value, self.DIRS[direction],
                                spec_in.data_ptr() if spec_in is not None else None, grid.data_ptr(),
                                spec_out.data_ptr() if spec_out is not None else None, nf)
            self._keep.append((plan, spec_in, grid, spec_out))
        h = _VP()
        _check(lib.st_batch_create(ctypes.byref(h), arr, len(items)), "st_batch_create")
        self._h = h

    def run(self, stream=None, graph: bool = True, persistent: bool = False):
        """persistent: the whole batch in one cooperative launch (use_graph 2);
        raises STError (ST_ERR_UNSUPPORTED) for a batch that does not qualify."""
        mode = 2 if persistent else (1 if graph else 0)
        _check(load().st_batch_run(self._h, _stream_handle(stream), mode), "st_batch_run")

    def close(self):
        if getattr(self, "_h", None):
            load().st_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
