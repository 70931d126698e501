"""Thin ctypes binding of ``include/mbir.h``: argument marshalling only.

Every computation runs in the CUDA library ``libmbir.so``; torch supplies device
memory and streams.  There is no CPU fallback: if the library was not built,
:func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MBIR_LIBRARY selects another build of the library (e.g. a tuning variant)
LIB_PATH = os.environ.get("MBIR_LIBRARY") or os.path.join(HERE, "libmbir.so")

FP32, FP32_COMPENSATED, FP64 = 0, 1, 2
PENALTY_L1, PENALTY_DB4 = 0, 1
PENALTY_TV = 2
PENALTIES = {"l1": PENALTY_L1, "db4": PENALTY_DB4, "tv": PENALTY_TV}
BACKPROJECTIONS = {"transpose": 0, "hilbert": 1}

STATUS = {0: "MBIR_OK", -1: "MBIR_ERR_INVALID", -2: "MBIR_ERR_UNSUPPORTED_SIZE",
          -3: "MBIR_ERR_OOM", -4: "MBIR_ERR_CUDA", -5: "MBIR_ERR_TIMEOUT",
          -6: "MBIR_ERR_NOT_CONVERGED"}


class MbirError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class Geometry(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("nz", C.c_int32), ("m", C.c_int32),
        ("k", C.POINTER(C.c_double)), ("source", C.POINTER(C.c_double)),
        ("dx_um", C.c_double), ("dz_um", C.c_double),
        ("na", C.c_double), ("z_focus_um", C.c_double),
        ("disp_a", C.c_double), ("disp_b", C.c_double), ("k0", C.c_double),
        ("falloff_half_um", C.c_double),
        ("kb_width", C.c_int32), ("kb_oversamp", C.c_double), ("kb_alpha", C.c_double),
        ("precision", C.c_int32),
    ]


class SolveOpts(C.Structure):
    _fields_ = [
        ("penalty", C.c_int32), ("lam", C.c_double), ("lambda_is_relative", C.c_int32),
        ("max_iter", C.c_int32), ("min_iter", C.c_int32), ("rel_tol", C.c_double),
        ("power_iters", C.c_int32), ("step", C.c_double), ("warm_start", C.c_int32),
        ("tv_iters", C.c_int32), ("backprojection", C.c_int32),
    ]


class LambdaSearchInfo(C.Structure):
    _fields_ = [
        ("lambda_rel", C.c_double), ("lam", C.c_double), ("ncc", C.c_double), ("step", C.c_double),
        ("evaluations", C.c_int32), ("trace_lambda_rel", C.POINTER(C.c_double)),
        ("trace_ncc", C.POINTER(C.c_double)),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("iters", C.c_int32), ("status", C.c_int32), ("objective", C.c_double),
        ("lipschitz", C.c_double), ("step", C.c_double), ("lambda_used", C.c_double),
        ("objective_trace", C.POINTER(C.c_double)), ("trace_len", C.c_int32),
    ]


class ProfileEntry(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_int64), ("total_ms", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("tile_c", C.c_int32), ("lateral_order", C.c_int32), ("adjoint_kernel", C.c_int32),
                ("pair_ms", C.c_double)]


_lib = None

# name -> (restype, argtypes)
_SIGNATURES = {
    "mbir_plan_create": (C.c_int, [C.POINTER(Geometry), C.c_void_p, C.POINTER(C.c_void_p)]),
    "mbir_plan_destroy": (None, [C.c_void_p]),
    "mbir_volume_plan_create": (C.c_int, [C.POINTER(Geometry), C.c_int32, C.c_double, C.c_void_p,
                                          C.POINTER(C.c_void_p)]),
    "mbir_volume_dims": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "mbir_plan_dims": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mbir_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mbir_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mbir_adjoint_hilbert": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mbir_isam_interpolated": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mbir_ncc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "mbir_lambda_search": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                     C.POINTER(LambdaSearchInfo), C.c_void_p]),
    "mbir_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveOpts), C.c_void_p,
                             C.POINTER(SolveInfo), C.c_void_p]),
    "mbir_solve_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                   C.POINTER(SolveOpts), C.POINTER(C.c_void_p), C.POINTER(SolveInfo), C.c_void_p]),
    "mbir_server_create": (C.c_int, [C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]),
    "mbir_server_destroy": (None, [C.c_void_p]),
    "mbir_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveOpts),
                                     C.c_void_p, C.POINTER(C.c_int64)]),
    "mbir_server_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mbir_server_poll": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.POINTER(SolveInfo),
                                   C.POINTER(C.c_double)]),
    "mbir_server_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                    C.POINTER(C.c_int64)]),
    "mbir_server_request_bytes": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    "mbir_admission_simulate": (C.c_int, [C.c_size_t, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int64)]),
    "mbir_lipschitz": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.c_void_p]),
    "mbir_prox": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    "mbir_prox_tv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p]),
    "mbir_wavelet": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mbir_wavelet_static": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mbir_profile_begin": (C.c_int, [C.c_void_p, C.c_int32]),
    "mbir_profile_only": (C.c_int, [C.c_void_p, C.c_char_p]),
    "mbir_plan_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]),
    "mbir_plan_get_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mbir_plan_set_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mbir_profile_end": (C.c_int, [C.c_void_p, C.POINTER(ProfileEntry), C.c_int32, C.POINTER(C.c_int32)]),
    "mbir_status_string": (C.c_char_p, [C.c_int]),
    "mbir_last_error": (C.c_char_p, []),
}


def lib() -> C.CDLL:
    """Load libmbir.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def _check(rc: int, where: str) -> None:
    if rc != 0:
        detail = lib().mbir_last_error().decode() if rc == -4 or rc == -3 else ""
        raise MbirError(rc, where, detail)


def _stream_handle(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


@dataclass
class _HostArrays:
    k: np.ndarray
    source: np.ndarray | None


def make_geometry(d: dict, precision: int = FP32) -> tuple[Geometry, _HostArrays]:
    """C geometry from a workload's plain-number description (keeps the host arrays alive)."""
    k = np.ascontiguousarray(d["k"], dtype=np.float64)
    src = d.get("source")
    src = None if src is None else np.ascontiguousarray(src, dtype=np.float64)
    g = Geometry()
    g.nx, g.nz, g.m = int(d["nx"]), int(d["nz"]), int(d["m"])
    g.k = k.ctypes.data_as(C.POINTER(C.c_double))
    g.source = src.ctypes.data_as(C.POINTER(C.c_double)) if src is not None else None
    g.dx_um = float(d["dx_um"])
    g.dz_um = float(d.get("dz_um", 0.0))
    g.na = float(d.get("na", 0.0))
    g.z_focus_um = float(d.get("z_focus_um", 0.0))
    g.disp_a = float(d.get("disp_a", 0.0))
    g.disp_b = float(d.get("disp_b", 0.0))
    g.k0 = float(d.get("k0", 0.0))
    g.falloff_half_um = float(d.get("falloff_half_um", 0.0))
    g.kb_width = int(d.get("kb_width", 6))
    g.kb_oversamp = float(d.get("kb_oversamp", 2.0))
    g.kb_alpha = float(d.get("kb_alpha", 0.0))
    g.precision = int(precision)
    return g, _HostArrays(k, src)


class Plan:
    """One B-scan geometry on the current CUDA device (mbir_plan_create)."""

    def __init__(self, geometry: dict, precision: int = FP32, stream=None):
        import torch
        self.geometry = geometry
        self.precision = precision
        self.nx, self.nz, self.m = int(geometry["nx"]), int(geometry["nz"]), int(geometry["m"])
        self.real_dtype = torch.float64 if precision == FP64 else torch.float32
        self.complex_dtype = torch.complex128 if precision == FP64 else torch.complex64
        g, keep = make_geometry(geometry, precision)
        h = C.c_void_p()
        _check(lib().mbir_plan_create(C.byref(g), _stream_handle(stream), C.byref(h)), "mbir_plan_create")
        self._h = h
        del keep

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().mbir_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- argument checks -------------------------------------------------
    def _image(self, t, name):
        if t.dtype != self.complex_dtype or tuple(t.shape) != (self.nx, self.nz) or not t.is_cuda \
                or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {self.complex_dtype} tensor "
                             f"of shape ({self.nx}, {self.nz})")

    def _meas(self, t, name):
        if t.dtype != self.real_dtype or tuple(t.shape) != (self.nx, self.m) or not t.is_cuda \
                or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {self.real_dtype} tensor "
                             f"of shape ({self.nx}, {self.m})")

    def _mask(self, t):
        import torch
        if t is None:
            return None
        if t.dtype != torch.uint8 or tuple(t.shape) != (self.nx, self.m) or not t.is_cuda \
                or not t.is_contiguous():
            raise ValueError(f"mask must be a contiguous CUDA uint8 tensor of shape ({self.nx}, {self.m})")
        return t

    # -- operators -------------------------------------------------------
    def forward(self, x, mask=None, out=None, stream=None):
        import torch
        self._image(x, "x")
        mask = self._mask(mask)
        if out is None:
            out = torch.empty((self.nx, self.m), dtype=self.real_dtype, device=x.device)
        self._meas(out, "out")
        _check(lib().mbir_forward(self._h, _ptr(x), _ptr(mask), _ptr(out), _stream_handle(stream)),
               "mbir_forward")
        return out

    def adjoint(self, y, mask=None, out=None, stream=None):
        import torch
        self._meas(y, "y")
        mask = self._mask(mask)
        if out is None:
            out = torch.empty((self.nx, self.nz), dtype=self.complex_dtype, device=y.device)
        self._image(out, "out")
        _check(lib().mbir_adjoint(self._h, _ptr(y), _ptr(mask), _ptr(out), _stream_handle(stream)),
               "mbir_adjoint")
        return out

    def adjoint_hilbert(self, y, mask=None, out=None, stream=None):
        """The paper's back-projection Phi*(y) = B^H A(s y) (mbir_adjoint_hilbert)."""
        import torch
        self._meas(y, "y")
        mask = self._mask(mask)
        if out is None:
            out = torch.empty((self.nx, self.nz), dtype=self.complex_dtype, device=y.device)
        self._image(out, "out")
        _check(lib().mbir_adjoint_hilbert(self._h, _ptr(y), _ptr(mask), _ptr(out), _stream_handle(stream)),
               "mbir_adjoint_hilbert")
        return out

    def isam_interpolated(self, y, mask=None, out=None, stream=None):
        """The direct-ISAM baseline on linearly interpolated measurements (mbir_isam_interpolated)."""
        import torch
        self._meas(y, "y")
        mask = self._mask(mask)
        if out is None:
            out = torch.empty((self.nx, self.nz), dtype=self.complex_dtype, device=y.device)
        self._image(out, "out")
        _check(lib().mbir_isam_interpolated(self._h, _ptr(y), _ptr(mask), _ptr(out), _stream_handle(stream)),
               "mbir_isam_interpolated")
        return out

    def ncc(self, x, z, stream=None) -> float:
        """NCC of magnitudes (Eq. ncc) of two images of the plan (mbir_ncc)."""
        self._image(x, "x")
        self._image(z, "z")
        r = C.c_double()
        _check(lib().mbir_ncc(self._h, _ptr(x), _ptr(z), C.byref(r), _stream_handle(stream)), "mbir_ncc")
        return r.value

    def lambda_search(self, y, mask, z_true, *, lo: float = -4.0, hi: float = 0.0, n_eval: int = 10,
                      penalty: str = "db4", iters: int = 100, power_iters: int = 30, step: float = 0.0,
                      tv_iters: int = 0, backprojection: str = "transpose", out=None, stream=None):
        """Golden-section search of log10(relative lambda) in [lo, hi] maximising the NCC with
        z_true (mbir_lambda_search).  Returns (best x, info dict with the evaluation trace)."""
        import torch
        self._meas(y, "y")
        mask = self._mask(mask)
        self._image(z_true, "z_true")
        if out is None:
            out = torch.empty((self.nx, self.nz), dtype=self.complex_dtype, device=y.device)
        self._image(out, "out")
        o = SolveOpts(PENALTIES[penalty], 0.0, 1, int(iters), 0, 0.0, int(power_iters), float(step), 0,
                      int(tv_iters), BACKPROJECTIONS[backprojection])
        tl = (C.c_double * n_eval)()
        tn = (C.c_double * n_eval)()
        info = LambdaSearchInfo()
        info.trace_lambda_rel = C.cast(tl, C.POINTER(C.c_double))
        info.trace_ncc = C.cast(tn, C.POINTER(C.c_double))
        _check(lib().mbir_lambda_search(self._h, _ptr(y), _ptr(mask), _ptr(z_true), C.byref(o), float(lo),
                                        float(hi), int(n_eval), _ptr(out), C.byref(info),
                                        _stream_handle(stream)), "mbir_lambda_search")
        n = info.evaluations
        return out, dict(lambda_rel=info.lambda_rel, lam=info.lam, ncc=info.ncc, step=info.step,
                         evaluations=n, trace_lambda_rel=np.array(tl[:n]), trace_ncc=np.array(tn[:n]))

    def autotune(self, reps: int = 5, stream=None) -> dict:
        """Time the candidate launch choices (mbir_plan_autotune); keep and return the fastest."""
        t, n = Tuning(), C.c_int32()
        _check(lib().mbir_plan_autotune(self._h, int(reps), C.byref(t), C.byref(n), _stream_handle(stream)),
               "mbir_plan_autotune")
        return dict(tile_c=t.tile_c, lateral_order=t.lateral_order, adjoint_kernel=t.adjoint_kernel,
                    pair_ms=t.pair_ms, tried=n.value)

    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().mbir_plan_get_tuning(self._h, C.byref(t)), "mbir_plan_get_tuning")
        return dict(tile_c=t.tile_c, lateral_order=t.lateral_order, adjoint_kernel=t.adjoint_kernel)

    def set_tuning(self, tile_c: int, lateral_order: int = 0, adjoint_kernel: int = -1) -> None:
        t = Tuning(int(tile_c), int(lateral_order), int(adjoint_kernel), 0.0)
        _check(lib().mbir_plan_set_tuning(self._h, C.byref(t)), "mbir_plan_set_tuning")

    def lipschitz(self, mask=None, iters: int = 30, stream=None) -> float:
        mask = self._mask(mask)
        v = C.c_double()
        _check(lib().mbir_lipschitz(self._h, _ptr(mask), int(iters), C.byref(v), _stream_handle(stream)),
               "mbir_lipschitz")
        return v.value

    def profile_begin(self, capacity: int = 1 << 16) -> None:
        """Record a CUDA event pair around every later kernel launch on this plan."""
        _check(lib().mbir_profile_begin(self._h, int(capacity)), "mbir_profile_begin")

    def profile_only(self, kernel_class: str | None) -> None:
        """While recording, record only launches of one kernel class (None: all)."""
        _check(lib().mbir_profile_only(self._h, None if kernel_class is None else kernel_class.encode()),
               "mbir_profile_only")

    def profile_end(self) -> dict:
        """Stop recording; returns {kernel class: (launches, total_ms)}."""
        buf = (ProfileEntry * 32)()
        n = C.c_int32()
        _check(lib().mbir_profile_end(self._h, buf, 32, C.byref(n)), "mbir_profile_end")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
                for i in range(min(n.value, 32))}

    def prox(self, v, tau: float, penalty: str = "l1", out=None, stream=None):
        import torch
        self._image(v, "v")
        if out is None:
            out = torch.empty_like(v)
        self._image(out, "out")
        _check(lib().mbir_prox(self._h, PENALTIES[penalty], _ptr(v), float(tau), _ptr(out),
                               _stream_handle(stream)), "mbir_prox")
        return out

    def prox_tv(self, v, tau: float, iters: int = 20, out=None, stream=None):
        """prox of tau * TV by `iters` dual projected-gradient steps (mbir_prox_tv); out != v."""
        import torch
        self._image(v, "v")
        if out is None:
            out = torch.empty_like(v)
        self._image(out, "out")
        _check(lib().mbir_prox_tv(self._h, _ptr(v), float(tau), int(iters), _ptr(out), _stream_handle(stream)),
               "mbir_prox_tv")
        return out

    def wavelet(self, x, inverse: bool = False, out=None, stream=None):
        import torch
        self._image(x, "x")
        if out is None:
            out = torch.empty_like(x)
        self._image(out, "out")
        _check(lib().mbir_wavelet(self._h, int(bool(inverse)), _ptr(x), _ptr(out), _stream_handle(stream)),
               "mbir_wavelet")
        return out

    def solve(self, y, mask=None, *, penalty: str = "l1", lam: float = 0.01, relative: bool = True,
              iters: int = 100, min_iter: int = 0, rel_tol: float = 0.0, power_iters: int = 30,
              step: float = 0.0, x0=None, out=None, trace: bool = False, tv_iters: int = 0,
              backprojection: str = "transpose", stream=None):
        """FISTA (mbir_solve).  Returns (x, info dict).  tv_iters: dual steps per TV prox (0: 20);
        backprojection: "transpose" (Phi^H) or "hilbert" (the paper's Phi*)."""
        import torch
        self._meas(y, "y")
        mask = self._mask(mask)
        if out is None:
            out = torch.zeros((self.nx, self.nz), dtype=self.complex_dtype, device=y.device) \
                if x0 is None else x0.clone()
        elif x0 is not None:
            out.copy_(x0)
        self._image(out, "out")
        o = SolveOpts(PENALTIES[penalty], float(lam), int(bool(relative)), int(iters), int(min_iter),
                      float(rel_tol), int(power_iters), float(step), int(x0 is not None), int(tv_iters),
                      BACKPROJECTIONS[backprojection])
        info = SolveInfo()
        tr = None
        if trace:
            tr = (C.c_double * iters)()
            info.objective_trace = C.cast(tr, C.POINTER(C.c_double))
            info.trace_len = iters
        rc = lib().mbir_solve(self._h, _ptr(y), _ptr(mask), C.byref(o), _ptr(out), C.byref(info),
                              _stream_handle(stream))
        if rc not in (0, -6):
            _check(rc, "mbir_solve")
        d = dict(iters=info.iters, status=info.status, objective=info.objective,
                 lipschitz=info.lipschitz, step=info.step, lambda_used=info.lambda_used)
        if trace:
            d["trace"] = np.array(tr[: info.iters])
        return out, d


class VolumePlan:
    """One 3-D volume geometry (mbir_volume_plan_create): the B-scan geometry plus a
    second lateral axis of ny pixels.  Image [nx, ny, nz], measurements and mask
    [nx, ny, m]; forward, adjoint and the l1 FISTA solve."""

    def __init__(self, geometry: dict, ny: int, dy_um: float = 0.0, precision: int = FP32, stream=None):
        import torch
        self.geometry = geometry
        self.precision = precision
        self.nx, self.nz, self.m = int(geometry["nx"]), int(geometry["nz"]), int(geometry["m"])
        self.ny = int(ny)
        self.real_dtype = torch.float64 if precision == FP64 else torch.float32
        self.complex_dtype = torch.complex128 if precision == FP64 else torch.complex64
        g, keep = make_geometry(geometry, precision)
        h = C.c_void_p()
        _check(lib().mbir_volume_plan_create(C.byref(g), self.ny, float(dy_um), _stream_handle(stream),
                                             C.byref(h)), "mbir_volume_plan_create")
        self._h = h
        del keep

    handle = Plan.handle
    close = Plan.close
    __del__ = Plan.__del__

    def _check_t(self, t, name, dtype, last):
        shape = (self.nx, self.ny, last)
        if t.dtype != dtype or tuple(t.shape) != shape or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of shape {shape}")

    def forward(self, x, mask=None, out=None, stream=None):
        import torch
        self._check_t(x, "x", self.complex_dtype, self.nz)
        if mask is not None:
            self._check_t(mask, "mask", torch.uint8, self.m)
        if out is None:
            out = torch.empty((self.nx, self.ny, self.m), dtype=self.real_dtype, device=x.device)
        self._check_t(out, "out", self.real_dtype, self.m)
        _check(lib().mbir_forward(self._h, _ptr(x), _ptr(mask), _ptr(out), _stream_handle(stream)),
               "mbir_forward")
        return out

    def adjoint(self, y, mask=None, out=None, stream=None):
        import torch
        self._check_t(y, "y", self.real_dtype, self.m)
        if mask is not None:
            self._check_t(mask, "mask", torch.uint8, self.m)
        if out is None:
            out = torch.empty((self.nx, self.ny, self.nz), dtype=self.complex_dtype, device=y.device)
        self._check_t(out, "out", self.complex_dtype, self.nz)
        _check(lib().mbir_adjoint(self._h, _ptr(y), _ptr(mask), _ptr(out), _stream_handle(stream)),
               "mbir_adjoint")
        return out


    def solve(self, y, mask=None, *, lam: float = 0.01, relative: bool = True, iters: int = 100,
              power_iters: int = 30, step: float = 0.0, x0=None, out=None, stream=None):
        """FISTA with the l1 penalty on the volume (mbir_solve).  Returns (x, info dict)."""
        import torch
        self._check_t(y, "y", self.real_dtype, self.m)
        if mask is not None:
            self._check_t(mask, "mask", torch.uint8, self.m)
        if out is None:
            out = torch.zeros((self.nx, self.ny, self.nz), dtype=self.complex_dtype, device=y.device) \
                if x0 is None else x0.clone()
        elif x0 is not None:
            out.copy_(x0)
        self._check_t(out, "out", self.complex_dtype, self.nz)
        o = SolveOpts(PENALTIES["l1"], float(lam), int(bool(relative)), int(iters), 0, 0.0, int(power_iters),
                      float(step), int(x0 is not None), 0, BACKPROJECTIONS["transpose"])
        info = SolveInfo()
        _check(lib().mbir_solve(self._h, _ptr(y), _ptr(mask), C.byref(o), _ptr(out), C.byref(info),
                                _stream_handle(stream)), "mbir_solve")
        return out, dict(iters=info.iters, status=info.status, objective=info.objective,
                         lipschitz=info.lipschitz, step=info.step, lambda_used=info.lambda_used)


def solve_batch(plans, ys, masks=None, *, penalties="l1", lams=0.01, relative=True, iters=100,
                power_iters=30, steps=0.0, outs=None, stream=None):
    """FISTA on several B-scans in one batched, graph-captured run (mbir_solve_batch).

    plans, ys, masks, outs: sequences (masks entries may be None); penalties, lams and
    steps: one value for all or one per scan.  Returns (xs, infos)."""
    import torch
    n = len(plans)
    as_list = lambda v: list(v) if isinstance(v, (list, tuple)) else [v] * n
    penalties, lams, steps = as_list(penalties), as_list(lams), as_list(steps)
    masks = [None] * n if masks is None else list(masks)
    if outs is None:
        outs = [torch.zeros((p.nx, p.nz), dtype=p.complex_dtype, device=y.device) for p, y in zip(plans, ys)]
    for p, y, m, o in zip(plans, ys, masks, outs):
        p._meas(y, "y")
        p._mask(m)
        p._image(o, "out")
    H = (C.c_void_p * n)(*[p.handle.value for p in plans])
    Y = (C.c_void_p * n)(*[y.data_ptr() for y in ys])
    M = (C.c_void_p * n)(*[(m.data_ptr() if m is not None else None) for m in masks])
    X = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    O = (SolveOpts * n)(*[SolveOpts(PENALTIES[pen], float(lam), int(bool(relative)), int(iters), 0, 0.0,
                                    int(power_iters), float(st), 0)
                          for pen, lam, st in zip(penalties, lams, steps)])
    I = (SolveInfo * n)()
    _check(lib().mbir_solve_batch(H, n, Y, M, O, X, I, _stream_handle(stream)), "mbir_solve_batch")
    infos = [dict(iters=I[i].iters, status=I[i].status, lipschitz=I[i].lipschitz, step=I[i].step,
                  lambda_used=I[i].lambda_used) for i in range(n)]
    return outs, infos


def admission_simulate(budget: int, bytes_: list[int], arrive: list[int], service: list[int]):
    """Host-only replay of the server's admission rule; returns (admit_tick, done_tick, peak)."""
    n = len(bytes_)
    B = (C.c_int64 * n)(*bytes_)
    A = (C.c_int32 * n)(*arrive)
    S = (C.c_int32 * n)(*service)
    adm = (C.c_int32 * n)()
    done = (C.c_int32 * n)()
    peak = C.c_int64()
    _check(lib().mbir_admission_simulate(int(budget), n, B, A, S, adm, done, C.byref(peak)),
           "mbir_admission_simulate")
    return list(adm), list(done), peak.value


class Server:
    """Continuous-batching reconstruction server (mbir_server_*)."""

    def __init__(self, hbm_budget_bytes: int, stream=None):
        self._stream = stream
        h = C.c_void_p()
        _check(lib().mbir_server_create(int(hbm_budget_bytes), _stream_handle(stream), C.byref(h)),
               "mbir_server_create")
        self._h = h
        self._keep = {}

    def submit(self, plan: Plan, y, mask=None, out=None, *, penalty="l1", lam=0.01, relative=True,
               iters=100, min_iter=0, rel_tol=0.0, power_iters=30, step=0.0) -> int:
        import torch
        plan._meas(y, "y")
        plan._mask(mask)
        if out is None:
            out = torch.zeros((plan.nx, plan.nz), dtype=plan.complex_dtype, device=y.device)
        plan._image(out, "out")
        o = SolveOpts(PENALTIES[penalty], float(lam), int(bool(relative)), int(iters), int(min_iter),
                      float(rel_tol), int(power_iters), float(step), 0)
        t = C.c_int64()
        _check(lib().mbir_server_submit(self._h, plan.handle, _ptr(y), _ptr(mask), C.byref(o), _ptr(out),
                                        C.byref(t)), "mbir_server_submit")
        self._keep[t.value] = (plan, y, mask, out)
        return t.value

    def step(self):
        a, p, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().mbir_server_step(self._h, C.byref(a), C.byref(p), C.byref(c)), "mbir_server_step")
        return a.value, p.value, c.value

    def poll(self, ticket: int):
        """None while running, else (out tensor, info dict, latency seconds)."""
        d = C.c_int32()
        info = SolveInfo()
        lat = C.c_double()
        _check(lib().mbir_server_poll(self._h, int(ticket), C.byref(d), C.byref(info), C.byref(lat)),
               "mbir_server_poll")
        if not d.value:
            return None
        plan, y, mask, out = self._keep.pop(ticket)
        return out, dict(iters=info.iters, status=info.status, objective=info.objective,
                         lipschitz=info.lipschitz, step=info.step, lambda_used=info.lambda_used), lat.value

    def stats(self):
        u, pk, c = C.c_size_t(), C.c_size_t(), C.c_int64()
        _check(lib().mbir_server_stats(self._h, C.byref(u), C.byref(pk), C.byref(c)), "mbir_server_stats")
        return dict(bytes_in_use=u.value, peak_bytes=pk.value, completed=c.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().mbir_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def request_bytes(plan: Plan, penalty: str = "l1", iters: int = 100) -> int:
    b = C.c_size_t()
    _check(lib().mbir_server_request_bytes(plan.handle, PENALTIES[penalty], int(iters), C.byref(b)),
           "mbir_server_request_bytes")
    return b.value
