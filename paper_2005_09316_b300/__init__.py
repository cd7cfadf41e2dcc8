"""Python binding of libwoden_b300 (the C ABI in include/woden_b300.h).

Argument marshalling only: every step of the prediction, peel and adjoint runs in the library's
CUDA kernels.  PyTorch provides device memory and streams.  There is no CPU fallback: if the
library cannot be loaded, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwoden_b300.so")
_lib = None
_lock = threading.Lock()

WN_OK, WN_EINVAL, WN_ENOMEM, WN_ECUDA, WN_ETIMEOUT, WN_EBUSY, WN_ENOTFOUND = range(7)
WN_PREC_MIXED, WN_PREC_FP64, WN_PREC_FP64_UNTUNED = 0, 1, 2
WN_SHAPE_BF16X3, WN_SHAPE_BF16X1, WN_SHAPE_LUT_BF16X3, WN_SHAPE_TF32, WN_SHAPE_TF32X3 = 0, 1, 2, 3, 4
WN_DEVERR_ANTENNA, WN_DEVERR_TIMEOUT, WN_DEVERR_SKY, WN_DEVERR_CALIB = 0x1, 0x2, 0x4, 0x8

EXPORTED = ("wn_create", "wn_destroy", "wn_last_error", "wn_version", "wn_set_precision", "wn_device_errors",
            "wn_sky_upload", "wn_sky_free", "wn_sky_bytes", "wn_predict", "wn_peel", "wn_peel_model",
            "wn_predict_grad", "wn_predict_static", "wn_server_create", "wn_server_destroy", "wn_server_submit",
            "wn_server_poll", "wn_server_wait", "wn_server_copy", "wn_server_release", "wn_server_cancel",
            "wn_server_stats", "wn_server_set_policy", "wn_server_set_order", "wn_calibrate", "wn_fit_shapelets", "wn_pipe_rates",
            "wn_phasor_loop_rate", "wn_sky_shapelet_operand", "wn_selftest_timeout", "wn_mma_rate", "wn_mma_rate_tf32", "wn_set_trace", "wn_debug_fail_allocs",
            "wn_sky_shapelet_operand_tf32", "wn_sky_update")


class WnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"woden_b300 error {code}: {msg}")
        self.code = code


_P = ctypes.c_void_p


class WnObs(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int32), ("n_base", ctypes.c_int32), ("n_time", ctypes.c_int32),
                ("n_chan", ctypes.c_int32), ("uvw", _P), ("freq_hz", _P), ("ant1", _P), ("ant2", _P),
                ("dec0", ctypes.c_double), ("chan_spacing_hz", ctypes.c_double), ("freq0_hz", ctypes.c_double)]


class WnSky(ctypes.Structure):
    _fields_ = [("n_point", ctypes.c_int32), ("n_gauss", ctypes.c_int32), ("n_shape", ctypes.c_int32)] + \
               [(n, _P) for n in ("l", "m", "flux", "alpha", "nu_ref", "g_maj", "g_min", "g_pa", "s_beta1",
                                  "s_beta2", "s_pa", "s_nmax", "s_off", "s_n1", "s_n2", "s_coeff")]


GRAD_FIELDS = ("flux", "alpha", "l", "m", "g_maj", "g_min", "g_pa", "s_beta1", "s_beta2", "s_pa", "s_coeff")


class WnSkyGrad(ctypes.Structure):
    _fields_ = [(n, _P) for n in GRAD_FIELDS]


def load(build_if_missing: bool = True):
    """Load (building first if sources are newer) the in-tree libwoden_b300.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if build_if_missing and _build.stale():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libwoden_b300.so not found at {LIB_PATH}; run paper_2005_09316_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        i, P = ctypes.c_int, ctypes.c_void_p
        L.wn_create.argtypes = [ctypes.POINTER(P), i]
        L.wn_destroy.argtypes = [P]
        L.wn_destroy.restype = None
        L.wn_last_error.restype = ctypes.c_char_p
        L.wn_version.restype = ctypes.c_char_p
        L.wn_set_precision.argtypes = [P, i, i]
        L.wn_device_errors.argtypes = [P, ctypes.POINTER(ctypes.c_uint32)]
        L.wn_sky_upload.argtypes = [P, ctypes.POINTER(WnSky), ctypes.POINTER(i), P]
        L.wn_sky_free.argtypes = [P, i]
        L.wn_sky_update.argtypes = [P, i, ctypes.POINTER(WnSky), P]
        L.wn_sky_bytes.argtypes = [P, i, ctypes.POINTER(ctypes.c_size_t)]
        L.wn_sky_shapelet_operand.argtypes = [P, i, i, P, ctypes.c_size_t, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.wn_predict.argtypes = [P, ctypes.POINTER(WnObs), i, P, i, P]
        L.wn_predict_static.argtypes = [P, ctypes.POINTER(WnObs), i, P, i, P]
        L.wn_peel.argtypes = [P, ctypes.POINTER(WnObs), i, P, i, i, P, P, P]
        L.wn_peel_model.argtypes = [P, ctypes.POINTER(WnObs), P, i, i, P, P, P, P]
        L.wn_predict_grad.argtypes = [P, ctypes.POINTER(WnObs), i, P, i, i, P, P, ctypes.POINTER(WnSkyGrad),
                                      P, P]
        u64, dbl = ctypes.c_uint64, ctypes.c_double
        L.wn_server_create.argtypes = [P, i, ctypes.c_size_t, i, i, i, ctypes.POINTER(P)]
        L.wn_server_destroy.argtypes = [P]
        L.wn_server_destroy.restype = None
        L.wn_server_submit.argtypes = [P, ctypes.POINTER(WnObs), i, i, P, i, i, P, ctypes.POINTER(u64)]
        L.wn_server_poll.argtypes = [P, u64, ctypes.POINTER(i), ctypes.POINTER(P), ctypes.POINTER(dbl)]
        L.wn_server_wait.argtypes = [P, u64, dbl, ctypes.POINTER(P), ctypes.POINTER(dbl)]
        L.wn_server_copy.argtypes = [P, u64, P, P]
        L.wn_server_release.argtypes = [P, u64]
        L.wn_server_cancel.argtypes = [P, u64]
        L.wn_server_stats.argtypes = [P, ctypes.POINTER(dbl)]
        L.wn_server_set_policy.argtypes = [P, i, dbl]
        L.wn_server_set_order.argtypes = [P, i]
        L.wn_calibrate.argtypes = [P, ctypes.POINTER(WnObs), P, P, P, i, P]
        L.wn_fit_shapelets.argtypes = [P, ctypes.POINTER(WnObs), i, P, i, i, P, i, dbl, P, ctypes.POINTER(dbl), P]
        L.wn_pipe_rates.argtypes = [P, ctypes.POINTER(dbl)]
        L.wn_phasor_loop_rate.argtypes = [P, ctypes.POINTER(dbl)]
        L.wn_selftest_timeout.argtypes = [P, dbl]
        L.wn_mma_rate.argtypes = [P, ctypes.POINTER(dbl)]
        L.wn_mma_rate_tf32.argtypes = [P, ctypes.POINTER(dbl)]
        L.wn_set_trace.argtypes = [P, ctypes.c_int]
        L.wn_debug_fail_allocs.argtypes = [ctypes.c_int]
        L.wn_sky_shapelet_operand_tf32.argtypes = L.wn_sky_shapelet_operand.argtypes
        for name in EXPORTED:
            if name not in ("wn_destroy", "wn_last_error", "wn_version", "wn_server_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(code: int):
    if code != WN_OK:
        raise WnError(code, load().wn_last_error().decode())


def _torch():
    import torch
    return torch


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream_handle(stream) -> int | None:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclass
class DeviceObs:
    """An observation resident on the device (torch tensors) plus its host scalars."""
    n_ant: int
    n_time: int
    n_chan: int
    uvw: object      # [T, B, 3] float64 cuda
    freq: object     # [F] float64 cuda
    ant1: object     # [B] int32 cuda
    ant2: object     # [B] int32 cuda
    dec0: float
    chan_spacing: float
    freq0: float

    @property
    def n_base(self) -> int:
        return int(self.ant1.shape[0])

    @property
    def n_rows(self) -> int:
        return self.n_time * self.n_base

    @property
    def n_vis(self) -> int:
        return self.n_rows * self.n_chan

    def struct(self) -> WnObs:
        return WnObs(self.n_ant, self.n_base, self.n_time, self.n_chan, self.uvw.data_ptr(), self.freq.data_ptr(),
                     self.ant1.data_ptr(), self.ant2.data_ptr(), float(self.dec0), float(self.chan_spacing),
                     float(self.freq0))


def channel_spacing(freq) -> float:
    """The uniform spacing of a channel list, or 0.0 if it is not uniform to 1e-9 relative."""
    f = np.asarray(freq, dtype=np.float64)
    if f.size < 2:
        return 0.0
    df = (f[-1] - f[0]) / (f.size - 1)
    if df <= 0:
        return 0.0
    ideal = f[0] + df * np.arange(f.size)
    return float(df) if np.all(np.abs(f - ideal) <= 1e-12 * np.abs(f)) and np.all(f[1:] - f[:-1] == df) else 0.0


def obs_to_device(obs, device="cuda") -> DeviceObs:
    """Copy a host observation (uvw [T,B,3], freq [F], ant1/ant2 [B]) to the device."""
    torch = _torch()
    uvw = torch.as_tensor(np.ascontiguousarray(obs.uvw, dtype=np.float64)).to(device)
    freq_np = np.ascontiguousarray(obs.freq, dtype=np.float64)
    return DeviceObs(int(obs.n_ant), int(obs.uvw.shape[0]), int(freq_np.size), uvw,
                     torch.as_tensor(freq_np).to(device),
                     torch.as_tensor(np.ascontiguousarray(obs.ant1, dtype=np.int32)).to(device),
                     torch.as_tensor(np.ascontiguousarray(obs.ant2, dtype=np.int32)).to(device),
                     float(obs.dec0), channel_spacing(freq_np), float(freq_np[0]))


SKY_F64 = ("l", "m", "flux", "alpha", "nu_ref", "g_maj", "g_min", "g_pa", "s_beta1", "s_beta2", "s_pa", "s_coeff")
SKY_I32 = ("s_nmax", "s_off", "s_n1", "s_n2")


def sky_to_device(sky, device="cuda") -> dict:
    """Device tensors of a host sky table (any object with the wn_sky field names)."""
    torch = _torch()
    out = {"n_point": int(sky.n_point), "n_gauss": int(sky.n_gauss), "n_shape": int(sky.n_shape)}
    for n in SKY_F64:
        out[n] = torch.as_tensor(np.ascontiguousarray(getattr(sky, n), dtype=np.float64)).to(device)
    for n in SKY_I32:
        out[n] = torch.as_tensor(np.ascontiguousarray(getattr(sky, n), dtype=np.int32)).to(device)
    return out


def _sky_struct(d: dict) -> WnSky:
    s = WnSky(d["n_point"], d["n_gauss"], d["n_shape"])
    for n in SKY_F64 + SKY_I32:
        t = d[n]
        setattr(s, n, t.data_ptr() if t.numel() else None)
    return s


class Model:
    def __init__(self, ctx: "Context", mid: int, n_point: int, n_gauss: int, n_shape: int, nnz: int):
        self.ctx, self.id = ctx, mid
        self.n_point, self.n_gauss, self.n_shape, self.nnz = n_point, n_gauss, n_shape, nnz

    @property
    def n_comp(self) -> int:
        return self.n_point + self.n_gauss + self.n_shape

    def update(self, sky, stream=None):
        """Re-pack this resident model in place from new parameter values (a device sky dict or a host sky
        table with this model's counts and shapelet structure); nothing is allocated on the device."""
        d = sky if isinstance(sky, dict) else sky_to_device(sky, f"cuda:{self.ctx.device}")
        if (d["n_point"], d["n_gauss"], d["n_shape"]) != (self.n_point, self.n_gauss, self.n_shape):
            raise ValueError("component counts differ from the resident model's")
        s = _sky_struct(d)
        _check(load().wn_sky_update(self.ctx.h, self.id, ctypes.byref(s), _stream_handle(stream)))

    def nbytes(self) -> int:
        v = ctypes.c_size_t()
        _check(load().wn_sky_bytes(self.ctx.h, self.id, ctypes.byref(v)))
        return int(v.value)

    def shapelet_operand(self, q: int):
        """Shapelet q's packed coefficient operand as raw bf16 bit patterns (uint16 hi, lo, each k_pad x n_pad
        in the canonical K-major core-matrix order) with k_pad and n_pad."""
        kp, npd = ctypes.c_int(), ctypes.c_int()
        _check(load().wn_sky_shapelet_operand(self.ctx.h, self.id, q, None, 0, ctypes.byref(kp), ctypes.byref(npd)))
        buf = np.empty(2 * kp.value * npd.value, dtype=np.uint16)
        _check(load().wn_sky_shapelet_operand(self.ctx.h, self.id, q, buf.ctypes.data, buf.nbytes, ctypes.byref(kp),
                                              ctypes.byref(npd)))
        half = kp.value * npd.value
        return buf[:half], buf[half:], kp.value, npd.value

    def shapelet_operand_tf32(self, q: int, with_lo: bool = False):
        """Shapelet q's tf32 operand as raw FP32 bit patterns (uint32, k_pad x n_pad in the K-major order of
        8 x 4 core matrices) with k_pad and n_pad; with_lo: (hi, lo, k_pad, n_pad), lo being the tf32
        remainder operand of WN_SHAPE_TF32X3."""
        kp, npd = ctypes.c_int(), ctypes.c_int()
        f = load().wn_sky_shapelet_operand_tf32
        _check(f(self.ctx.h, self.id, q, None, 0, ctypes.byref(kp), ctypes.byref(npd)))
        n = kp.value * npd.value
        buf = np.empty(2 * n if with_lo else n, dtype=np.uint32)
        _check(f(self.ctx.h, self.id, q, buf.ctypes.data, buf.nbytes, ctypes.byref(kp), ctypes.byref(npd)))
        if with_lo:
            return buf[:n], buf[n:], kp.value, npd.value
        return buf, kp.value, npd.value

    def free(self):
        if self.id:
            _check(load().wn_sky_free(self.ctx.h, self.id))
            self.id = 0


class Context:
    """A library context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = device
        h = ctypes.c_void_p()
        _check(load().wn_create(ctypes.byref(h), device))
        self.h = h

    def close(self):
        if self.h:
            load().wn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: int = WN_PREC_MIXED, shape_mode: int = WN_SHAPE_BF16X3):
        _check(load().wn_set_precision(self.h, precision, shape_mode))

    def device_errors(self) -> int:
        v = ctypes.c_uint32()
        _check(load().wn_device_errors(self.h, ctypes.byref(v)))
        return int(v.value)

    def calibrate(self, obs: DeviceObs, model_vis, data, gains=None, n_iter: int = 10, stream=None):
        """Per-(time, channel) antenna gains fitted by n_iter iterations of the linearised least squares
        (Sec. 5.1); gains [T][F][A] complex64 are updated in place (ones if not given) and returned."""
        torch = _torch()
        if gains is None:
            gains = torch.ones((obs.n_time, obs.n_chan, obs.n_ant), dtype=torch.complex64,
                               device=f"cuda:{self.device}")
        for t, shape in ((model_vis, (obs.n_time, obs.n_base, obs.n_chan)), (data, (obs.n_time, obs.n_base, obs.n_chan)),
                         (gains, (obs.n_time, obs.n_chan, obs.n_ant))):
            if t.dtype != torch.complex64 or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"expected a contiguous complex64 tensor of shape {shape}")
        o = obs.struct()
        _check(load().wn_calibrate(self.h, ctypes.byref(o), model_vis.data_ptr(), data.data_ptr(), gains.data_ptr(),
                                   int(n_iter), _stream_handle(stream)))
        return gains

    def fit_shapelets(self, obs: DeviceObs, model: Model, gains, data, coeff=None, n_iter: int = 200,
                      tol: float = 1e-6, stream=None):
        """Least-squares shapelet coefficients of `model` for `data` (visibility space, CGLS); returns
        (coefficients as a float64 device tensor in upload order, info dict).  The model keeps them."""
        torch = _torch()
        if coeff is None:
            coeff = torch.zeros(model.nnz, dtype=torch.float64, device=f"cuda:{self.device}")
        if coeff.dtype != torch.float64 or coeff.numel() != model.nnz or not coeff.is_contiguous():
            raise ValueError("coeff must be a contiguous float64 tensor of the model's nnz")
        info = (ctypes.c_double * 4)()
        o = obs.struct()
        _check(load().wn_fit_shapelets(self.h, ctypes.byref(o), model.id, gains.data_ptr(), int(gains.shape[0]),
                                       int(gains.shape[1]), data.data_ptr(), int(n_iter), float(tol),
                                       coeff.data_ptr(), info, _stream_handle(stream)))
        return coeff, {"iterations": int(info[0]), "rel_grad": info[1], "resid2": info[2], "resid2_start": info[3]}

    def pipe_rates(self) -> dict:
        """Measured lane operations per second of the FP32 FMA, packed FFMA2, MUFU ex2 and FP64 FMA pipes."""
        r = (ctypes.c_double * 4)()
        _check(load().wn_pipe_rates(self.h, r))
        return {"ffma": r[0], "ffma2": r[1], "mufu_ex2": r[2], "dfma": r[3]}

    def selftest_timeout(self, seconds: float = 0.5):
        """Run a kernel whose bounded wait cannot complete; it must give up after `seconds` and flag it."""
        _check(load().wn_selftest_timeout(self.h, float(seconds)))

    def set_trace(self, on: bool = True):
        """NVTX ranges around the context's compute calls (for profilers that record NVTX)."""
        _check(load().wn_set_trace(self.h, 1 if on else 0))

    def mma_rate(self) -> dict:
        """SM clocks per tcgen05 MMA (M = 128, K = 16, bf16) at N = 128 and 64, and of TMEM loads."""
        r = (ctypes.c_double * 4)()
        _check(load().wn_mma_rate(self.h, r))
        return {"clk_per_mma_n128": r[0], "clk_per_mma_n64": r[1], "clk_tmem_ld16": r[2], "clk_tmem_ld16_x8": r[3]}

    def mma_rate_tf32(self) -> dict:
        """SM clocks per tcgen05 MMA (M = 128, K = 8, tf32) at N = 128 and 64."""
        r = (ctypes.c_double * 2)()
        _check(load().wn_mma_rate_tf32(self.h, r))
        return {"clk_per_mma_n128": r[0], "clk_per_mma_n64": r[1]}

    def phasor_loop_rate(self) -> float:
        """Evaluations per second the point/Gaussian kernel's channel loop sustains by itself."""
        r = ctypes.c_double()
        _check(load().wn_phasor_loop_rate(self.h, ctypes.byref(r)))
        return r.value

    def upload(self, sky, stream=None) -> Model:
        d = sky if isinstance(sky, dict) else sky_to_device(sky, f"cuda:{self.device}")
        s = _sky_struct(d)
        mid = ctypes.c_int()
        _check(load().wn_sky_upload(self.h, ctypes.byref(s), ctypes.byref(mid), _stream_handle(stream)))
        return Model(self, mid.value, d["n_point"], d["n_gauss"], d["n_shape"], int(d["s_coeff"].numel()))

    def _vis(self, obs: DeviceObs, out):
        torch = _torch()
        if out is None:
            return torch.empty((obs.n_time, obs.n_base, obs.n_chan), dtype=torch.complex64,
                               device=f"cuda:{self.device}")
        return out

    def predict(self, obs: DeviceObs, model: Model, out=None, accumulate: bool = False, stream=None):
        out = self._vis(obs, out)
        o = obs.struct()
        _check(load().wn_predict(self.h, ctypes.byref(o), model.id, out.data_ptr(), int(accumulate),
                                 _stream_handle(stream)))
        return out

    def predict_static(self, obs: DeviceObs, model: Model, out=None, accumulate: bool = False, stream=None):
        """wn_predict_static: the same prediction without any device allocation (fixed-size scratch)."""
        out = self._vis(obs, out)
        o = obs.struct()
        _check(load().wn_predict_static(self.h, ctypes.byref(o), model.id, out.data_ptr(), int(accumulate),
                                        _stream_handle(stream)))
        return out

    def peel(self, obs: DeviceObs, model: Model, gains, data, out=None, stream=None):
        out = self._vis(obs, out)
        o = obs.struct()
        _check(load().wn_peel(self.h, ctypes.byref(o), model.id, gains.data_ptr(), int(gains.shape[0]),
                              int(gains.shape[1]), data.data_ptr(), out.data_ptr(), _stream_handle(stream)))
        return out

    def peel_model(self, obs: DeviceObs, gains, data, model_vis, out=None, stream=None):
        out = self._vis(obs, out)
        o = obs.struct()
        _check(load().wn_peel_model(self.h, ctypes.byref(o), gains.data_ptr(), int(gains.shape[0]),
                                    int(gains.shape[1]), data.data_ptr(), model_vis.data_ptr(), out.data_ptr(),
                                    _stream_handle(stream)))
        return out

    def predict_grad(self, obs: DeviceObs, model: Model, gains, data, resid=None, want_loss: bool = True,
                     stream=None) -> dict:
        torch = _torch()
        dev = f"cuda:{self.device}"
        resid = self._vis(obs, resid)
        sizes = dict(flux=model.n_comp, alpha=model.n_comp, l=model.n_comp, m=model.n_comp, g_maj=model.n_gauss,
                     g_min=model.n_gauss, g_pa=model.n_gauss, s_beta1=model.n_shape, s_beta2=model.n_shape,
                     s_pa=model.n_shape, s_coeff=model.nnz)
        grads = {k: torch.empty(v, dtype=torch.float64, device=dev) for k, v in sizes.items()}
        g = WnSkyGrad(*[grads[k].data_ptr() if grads[k].numel() else None for k in GRAD_FIELDS])
        loss = torch.empty(1, dtype=torch.float64, device=dev) if want_loss else None
        o = obs.struct()
        _check(load().wn_predict_grad(self.h, ctypes.byref(o), model.id, gains.data_ptr(), int(gains.shape[0]),
                                      int(gains.shape[1]), data.data_ptr(), resid.data_ptr(), ctypes.byref(g),
                                      _ptr(loss), _stream_handle(stream)))
        grads["loss"] = loss
        grads["resid"] = resid
        return grads


def version() -> str:
    return load().wn_version().decode()


def debug_fail_allocs(n: int):
    """Make the library's next n device allocations fail as out-of-memory (host-side fault injection)."""
    _check(load().wn_debug_fail_allocs(int(n)))
