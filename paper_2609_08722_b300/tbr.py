"""Python binding of the TBR C ABI (``include/tbr.h``): argument marshalling only.

Every step of the render and of the replay adjoint runs in the CUDA kernels of
``libtbr.so``; this module only turns torch CUDA tensors into the pointers and
structs the C entry points take, and raises on a non-OK status.  If the library
is missing the import of any entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtbr.so")

TBR_OK, TBR_ERR_INVALID_ARG, TBR_ERR_OOM, TBR_ERR_CUDA, TBR_ERR_TIMEOUT = 0, 1, 2, 3, 4
TBR_ERR_ADMISSION, TBR_ERR_OVERFLOW, TBR_ERR_NOT_FOUND = 5, 6, 7
_STATUS_NAMES = {0: "TBR_OK", 1: "TBR_ERR_INVALID_ARG", 2: "TBR_ERR_OOM", 3: "TBR_ERR_CUDA",
                 4: "TBR_ERR_TIMEOUT", 5: "TBR_ERR_ADMISSION", 6: "TBR_ERR_OVERFLOW",
                 7: "TBR_ERR_NOT_FOUND"}

# Every entry point include/tbr.h declares (checked by the ABI test).
EXPORTED = ["tbr_render_hard", "tbr_render_hard_transport", "tbr_render_hard_noalloc", "tbr_compensate", "tbr_render_soft", "tbr_render_backward", "tbr_ctx_status",
            "tbr_ctx_bytes", "tbr_ctx_destroy", "tbr_loss_mse", "tbr_render_soft_adjoint_mse", "tbr_fit_default_config",
            "tbr_fit_create", "tbr_fit_step", "tbr_fit_get_program", "tbr_fit_iteration",
            "tbr_fit_destroy", "tbr_serve_default_config", "tbr_serve_create", "tbr_serve_load_program",
            "tbr_serve_submit", "tbr_serve_poll", "tbr_serve_wait", "tbr_serve_request_times",
            "tbr_serve_release", "tbr_serve_stats", "tbr_serve_destroy", "tbr_profile_enable", "tbr_profile_read", "tbr_profile_reset",
            "tbr_measure_peak", "tbr_last_error", "tbr_version"]


class TbrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class TbrProgram(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("k", ctypes.c_int32),
                ("cx", ctypes.c_void_p), ("cy", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("length", ctypes.c_void_p), ("half_width", ctypes.c_void_p),
                ("logits", ctypes.c_void_p), ("palette", ctypes.c_void_p),
                ("background", ctypes.c_float * 3), ("color_temp", ctypes.c_float),
                ("coupling", ctypes.c_void_p)]


class TbrHardStats(ctypes.Structure):
    _fields_ = [("band_steps", ctypes.c_int64), ("background_pixels", ctypes.c_int64),
                ("visited_steps", ctypes.c_int64)]


class TbrSoftOpts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("tau_min", ctypes.c_float),
                ("checkpoint_every", ctypes.c_int32), ("record_capacity", ctypes.c_int32),
                ("inert", ctypes.c_int32), ("drift_tolerance", ctypes.c_float),
                ("repair_capacity", ctypes.c_int32), ("transport", ctypes.c_int32),
                ("early_exit", ctypes.c_float)]


TRANSPORTS = {"capsule": 0, "drops": 1}


class TbrCtxStats(ctypes.Structure):
    _fields_ = [("records", ctypes.c_int64), ("max_records", ctypes.c_int64),
                ("overflow_pixels", ctypes.c_int64), ("drift_resets", ctypes.c_int64),
                ("timeouts", ctypes.c_int64), ("invalid_params", ctypes.c_int64),
                ("repaired_pixels", ctypes.c_int64), ("repair_overflow", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load libtbr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_2609_08722_b300/build.py "
                                   "(or __graft_entry__.build()) first; there is no fallback")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            st = ctypes.c_int
            L.tbr_render_hard.argtypes = [ctypes.POINTER(TbrProgram), i32, i32, i32, i32, P, P,
                                          ctypes.POINTER(TbrHardStats), P]
            L.tbr_render_hard_transport.argtypes = [ctypes.POINTER(TbrProgram), i32, i32, i32, i32, i32, P, P,
                                                    ctypes.POINTER(TbrHardStats), P]
            L.tbr_compensate.argtypes = [ctypes.POINTER(TbrProgram), i32, i32, P, P, P, P, P,
                                         ctypes.POINTER(ctypes.c_int64), P]
            L.tbr_render_soft.argtypes = [ctypes.POINTER(TbrProgram), i32, i32,
                                          ctypes.POINTER(TbrSoftOpts), P, ctypes.POINTER(P), P]
            L.tbr_render_backward.argtypes = [P, P, P, P, P, P, P, P, P, P]
            L.tbr_ctx_status.argtypes = [P, ctypes.POINTER(TbrCtxStats)]
            L.tbr_ctx_bytes.argtypes = [P]
            L.tbr_ctx_bytes.restype = ctypes.c_size_t
            L.tbr_ctx_destroy.argtypes = [P]
            L.tbr_ctx_destroy.restype = None
            L.tbr_loss_mse.argtypes = [P, P, i64, P, P, P]
            L.tbr_last_error.restype = ctypes.c_char_p
            L.tbr_version.restype = ctypes.c_char_p
            for f in ("tbr_render_hard", "tbr_render_hard_transport", "tbr_compensate", "tbr_render_soft", "tbr_render_backward",
                      "tbr_ctx_status", "tbr_loss_mse"):
                getattr(L, f).restype = st
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != TBR_OK:
        raise TbrError(status, lib().tbr_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t: torch.Tensor, device, dtype=torch.float32) -> torch.Tensor:
    return torch.as_tensor(t).to(device=device, dtype=dtype).contiguous()


@dataclasses.dataclass
class DeviceProgram:
    """A stroke program resident on the GPU (float32, contiguous)."""
    cx: torch.Tensor
    cy: torch.Tensor
    theta: torch.Tensor
    length: torch.Tensor
    half_width: torch.Tensor
    logits: torch.Tensor      # [n, k]
    palette: torch.Tensor     # [k, 3]
    background: tuple = (1.0, 1.0, 1.0)
    color_temp: float = 1.0
    coupling: Optional[torch.Tensor] = None  # [n, 3] profile c_1..c_3 of the coupling variant, or None

    @property
    def n(self) -> int:
        return int(self.cx.shape[0])

    @property
    def k(self) -> int:
        return int(self.palette.shape[0])

    @classmethod
    def from_host(cls, prog, device="cuda") -> "DeviceProgram":
        """From any object with numpy arrays (``inputs.Program``)."""
        t = lambda a: torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(device)
        cpl = getattr(prog, "coupling", None)
        return cls(cx=t(prog.cx), cy=t(prog.cy), theta=t(prog.theta), length=t(prog.length),
                   half_width=t(prog.half_width), logits=t(prog.logits), palette=t(prog.palette),
                   background=tuple(float(v) for v in np.asarray(prog.background)),
                   color_temp=float(prog.color_temp), coupling=None if cpl is None else t(cpl))

    def struct(self) -> TbrProgram:
        for name in ("cx", "cy", "theta", "length", "half_width", "logits", "palette"):
            v = getattr(self, name)
            if not (v.is_cuda and v.dtype == torch.float32 and v.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
        if self.logits.shape != (self.n, self.k) or self.palette.shape != (self.k, 3):
            raise ValueError("logits must be [n, k] and palette [k, 3]")
        s = TbrProgram()
        s.n, s.k = self.n, self.k
        s.cx, s.cy, s.theta = _ptr(self.cx), _ptr(self.cy), _ptr(self.theta)
        s.length, s.half_width = _ptr(self.length), _ptr(self.half_width)
        s.logits, s.palette = _ptr(self.logits), _ptr(self.palette)
        s.background = (ctypes.c_float * 3)(*self.background)
        s.color_temp = float(self.color_temp)
        if self.coupling is not None:
            c = self.coupling
            if not (c.is_cuda and c.dtype == torch.float32 and c.is_contiguous() and c.shape == (self.n, 3)):
                raise ValueError("coupling must be a contiguous float32 CUDA tensor [n, 3]")
            s.coupling = _ptr(c)
        return s


def render_hard(prog: DeviceProgram, W: int, H: int, n_prefix: int = -1, snap: bool = False,
                with_idx: bool = True, stats: bool = False, out_rgb=None, out_idx=None, stream=None,
                transport: str = "capsule"):
    """tbr_render_hard (transport "capsule") or tbr_render_hard_transport;
    returns (rgb [H,W,3], idx [H,W] or None, stats dict or None)."""
    dev = prog.cx.device
    rgb = out_rgb if out_rgb is not None else torch.empty((H, W, 3), device=dev, dtype=torch.float32)
    idx = out_idx if out_idx is not None else (
        torch.empty((H, W), device=dev, dtype=torch.int32) if with_idx else None)
    st = TbrHardStats() if stats else None
    s = prog.struct()
    if transport == "capsule":
        check(lib().tbr_render_hard(ctypes.byref(s), W, H, n_prefix, int(bool(snap)), _ptr(rgb), _ptr(idx),
                                    ctypes.byref(st) if st is not None else None, _stream(stream)))
    else:
        check(lib().tbr_render_hard_transport(ctypes.byref(s), W, H, n_prefix, int(bool(snap)),
                                              TRANSPORTS[transport], _ptr(rgb), _ptr(idx),
                                              ctypes.byref(st) if st is not None else None, _stream(stream)))
    sd = None
    if st is not None:
        sd = {"band_steps": st.band_steps, "background_pixels": st.background_pixels,
              "visited_steps": st.visited_steps}
    return rgb, idx, sd


def compensate(prog: DeviceProgram, endpoint: bool = False, skip_blocked: bool = False, stream=None) -> dict:
    """tbr_compensate: the one-pass closed-form compensation of a program
    (anchor variant, or endpoint with endpoint=True); returns dict cx, cy,
    theta, length [n] float32, blocked [n] int32 and n_blocked (int)."""
    dev = prog.cx.device
    out = {k: torch.empty(prog.n, device=dev, dtype=torch.float32) for k in ("cx", "cy", "theta", "length")}
    out["blocked"] = torch.empty(prog.n, device=dev, dtype=torch.int32)
    nb = ctypes.c_int64(0)
    s = prog.struct()
    check(lib().tbr_compensate(ctypes.byref(s), int(bool(endpoint)), int(bool(skip_blocked)), _ptr(out["cx"]),
                               _ptr(out["cy"]), _ptr(out["theta"]), _ptr(out["length"]), _ptr(out["blocked"]),
                               ctypes.byref(nb), _stream(stream)))
    out["n_blocked"] = int(nb.value)
    return out


class SoftContext:
    """A replay context (tbr_ctx*): what the adjoint needs from one soft forward."""

    def __init__(self, handle: int, prog: DeviceProgram, W: int, H: int):
        self.handle = handle
        self.n, self.k, self.W, self.H = prog.n, prog.k, W, H
        self.device = prog.cx.device

    def backward(self, dL_drgb: torch.Tensor, want_palette: bool = True, stream=None) -> dict:
        """tbr_render_backward; returns the gradient tensors."""
        if self.handle is None:
            raise RuntimeError("context already destroyed")
        d = dL_drgb.contiguous()
        if d.shape != (self.H, self.W, 3) or d.dtype != torch.float32 or not d.is_cuda:
            raise ValueError("dL_drgb must be a [H, W, 3] float32 CUDA tensor")
        e = lambda *sh: torch.empty(sh, device=self.device, dtype=torch.float32)
        g = {"cx": e(self.n), "cy": e(self.n), "theta": e(self.n), "length": e(self.n),
             "half_width": e(self.n), "logits": e(self.n, self.k)}
        g["palette"] = e(self.k, 3) if want_palette else None
        check(lib().tbr_render_backward(ctypes.c_void_p(self.handle), _ptr(d), _ptr(g["cx"]),
                                        _ptr(g["cy"]), _ptr(g["theta"]), _ptr(g["length"]),
                                        _ptr(g["half_width"]), _ptr(g["logits"]), _ptr(g["palette"]),
                                        _stream(stream)))
        return g

    def status(self, raise_on_error: bool = True) -> dict:
        """tbr_ctx_status (synchronises)."""
        st = TbrCtxStats()
        code = lib().tbr_ctx_status(ctypes.c_void_p(self.handle), ctypes.byref(st))
        out = {f: getattr(st, f) for f, _ in TbrCtxStats._fields_}
        out["status"] = code
        if raise_on_error:
            check(code)
        return out

    def nbytes(self) -> int:
        return int(lib().tbr_ctx_bytes(ctypes.c_void_p(self.handle)))

    def destroy(self) -> None:
        if self.handle is not None:
            lib().tbr_ctx_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def render_soft(prog: DeviceProgram, W: int, H: int, tau: float, tau_min: float, record: bool = False,
                checkpoint_every: int = 0, record_capacity: int = 0, inert: bool = False,
                out_rgb=None, stream=None, reuse: Optional["SoftContext"] = None,
                drift_tolerance: float = 0.0, repair_capacity: int = 0, transport: str = "capsule",
                early_exit: float = 0.0):
    """tbr_render_soft; returns (rgb [H,W,3], SoftContext or None).  ``reuse``
    overwrites an existing context of the same shape instead of allocating.
    ``transport="drops"`` renders with the sixteen-drop transport (forward only).
    ``early_exit`` > 0 (forward only) stops a pixel once T < early_exit."""
    dev = prog.cx.device
    rgb = out_rgb if out_rgb is not None else torch.empty((H, W, 3), device=dev, dtype=torch.float32)
    opts = TbrSoftOpts(float(tau), float(tau_min), int(checkpoint_every), int(record_capacity),
                       int(bool(inert)), float(drift_tolerance), int(repair_capacity), TRANSPORTS[transport],
                       float(early_exit))
    handle = ctypes.c_void_p(reuse.handle if reuse is not None else None)
    s = prog.struct()
    check(lib().tbr_render_soft(ctypes.byref(s), W, H, ctypes.byref(opts), _ptr(rgb),
                                ctypes.byref(handle) if (record or reuse is not None) else None,
                                _stream(stream)))
    if reuse is not None:
        return rgb, reuse
    ctx = SoftContext(handle.value, prog, W, H) if record else None
    return rgb, ctx


def loss_mse(rgb: torch.Tensor, target: torch.Tensor, want_grad: bool = True, stream=None):
    """tbr_loss_mse; returns (loss [1] device tensor, dL/drgb or None)."""
    rgb = rgb.contiguous()
    target = target.contiguous()
    if rgb.shape != target.shape or rgb.shape[-1] != 3:
        raise ValueError("rgb and target must both be [..., 3]")
    loss = torch.empty(1, device=rgb.device, dtype=torch.float32)
    d = torch.empty_like(rgb) if want_grad else None
    check(lib().tbr_loss_mse(_ptr(rgb), _ptr(target), rgb.numel() // 3, _ptr(loss), _ptr(d),
                             _stream(stream)))
    return loss, d


def version() -> str:
    return lib().tbr_version().decode()


# ---------------------------------------------------------------------------
# Fit (tbr_fit_*) and per-kernel timing (tbr_profile_*)
# ---------------------------------------------------------------------------
class TbrFitConfig(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("tau_start", ctypes.c_float),
                ("tau_end", ctypes.c_float), ("tau_min", ctypes.c_float),
                ("color_temp_start", ctypes.c_float), ("color_temp_end", ctypes.c_float),
                ("lr_center", ctypes.c_float), ("lr_angle", ctypes.c_float),
                ("lr_length", ctypes.c_float), ("lr_width", ctypes.c_float),
                ("lr_logits", ctypes.c_float), ("lr_palette", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float),
                ("length_max", ctypes.c_float), ("width_lo", ctypes.c_float),
                ("width_hi", ctypes.c_float), ("length_weight", ctypes.c_float),
                ("train_palette", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
                ("record_capacity", ctypes.c_int32)]


class TbrKernelTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


KERNELS = {"pack": 0, "hard": 1, "soft": 2, "backward": 3, "epilogue": 4, "loss": 5, "update": 6,
           "serve": 7, "compensate": 8}


def _fit_lib():
    L = lib()
    if not getattr(L, "_fit_typed", False):
        P = ctypes.c_void_p
        L.tbr_fit_default_config.argtypes = [ctypes.POINTER(TbrFitConfig)]
        L.tbr_fit_default_config.restype = None
        L.tbr_fit_create.argtypes = [ctypes.POINTER(TbrProgram), P, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(TbrFitConfig), ctypes.POINTER(P), P]
        L.tbr_fit_step.argtypes = [P, ctypes.POINTER(ctypes.c_float), P]
        L.tbr_fit_get_program.argtypes = [P, ctypes.POINTER(TbrProgram)]
        L.tbr_fit_iteration.argtypes = [P]
        L.tbr_fit_iteration.restype = ctypes.c_int32
        L.tbr_fit_destroy.argtypes = [P]
        L.tbr_fit_destroy.restype = None
        for f in ("tbr_fit_create", "tbr_fit_step", "tbr_fit_get_program", "tbr_profile_enable",
                  "tbr_profile_read"):
            getattr(L, f).restype = ctypes.c_int
        L.tbr_profile_enable.argtypes = [ctypes.c_int32]
        L.tbr_profile_read.argtypes = [ctypes.c_int32, ctypes.POINTER(TbrKernelTime)]
        L.tbr_profile_reset.argtypes = []
        L.tbr_profile_reset.restype = None
        L.tbr_measure_peak.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), P]
        L.tbr_measure_peak.restype = ctypes.c_int
        L._fit_typed = True
    return L


def default_fit_config(**overrides) -> TbrFitConfig:
    c = TbrFitConfig()
    _fit_lib().tbr_fit_default_config(ctypes.byref(c))
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


class _DeviceArray:
    """Exposes a library-owned float32 device buffer to torch (no copy)."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f4", "data": (ptr, False),
                                         "version": 2, "strides": None}


class Fit:
    """tbr_fit_*: Adam on a stroke program against a target image."""

    def __init__(self, init: DeviceProgram, target: torch.Tensor, config: Optional[TbrFitConfig] = None,
                 stream=None):
        L = _fit_lib()
        t = target.contiguous()
        H, W = int(t.shape[0]), int(t.shape[1])
        if t.shape != (H, W, 3) or t.dtype != torch.float32 or not t.is_cuda:
            raise ValueError("target must be a [H, W, 3] float32 CUDA tensor")
        self.W, self.H, self.n, self.k = W, H, init.n, init.k
        self.device = init.cx.device
        self.config = config if config is not None else default_fit_config()
        h = ctypes.c_void_p()
        s = init.struct()
        check(L.tbr_fit_create(ctypes.byref(s), _ptr(t), W, H, ctypes.byref(self.config), ctypes.byref(h),
                               _stream(stream)))
        self.handle = h.value

    def step(self, stream=None) -> float:
        loss = ctypes.c_float()
        check(_fit_lib().tbr_fit_step(ctypes.c_void_p(self.handle), ctypes.byref(loss), _stream(stream)))
        return float(loss.value)

    @property
    def iteration(self) -> int:
        return int(_fit_lib().tbr_fit_iteration(ctypes.c_void_p(self.handle)))

    def program(self) -> DeviceProgram:
        """A copy of the current program as torch tensors."""
        v = TbrProgram()
        check(_fit_lib().tbr_fit_get_program(ctypes.c_void_p(self.handle), ctypes.byref(v)))
        n, k = self.n, self.k
        # the view's arrays are consecutive slices of one device buffer of 5n + nk + 3k floats
        total = 5 * n + n * k + 3 * k
        buf = torch.as_tensor(_DeviceArray(v.cx, total), device=self.device)
        sl = lambda a, b: buf[a:b].clone()
        cpl = None
        if v.coupling:  # the fixed coupling profile, [n, 3]
            cpl = torch.as_tensor(_DeviceArray(v.coupling, 3 * n), device=self.device).clone().view(n, 3)
        return DeviceProgram(cx=sl(0, n), cy=sl(n, 2 * n), theta=sl(2 * n, 3 * n), length=sl(3 * n, 4 * n),
                             half_width=sl(4 * n, 5 * n), logits=sl(5 * n, 5 * n + n * k).view(n, k),
                             palette=sl(5 * n + n * k, total).view(k, 3),
                             background=tuple(v.background), color_temp=float(v.color_temp), coupling=cpl)

    def destroy(self):
        if self.handle is not None:
            _fit_lib().tbr_fit_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def profile_enable(on: bool = True) -> None:
    check(_fit_lib().tbr_profile_enable(int(bool(on))))


def profile_reset() -> None:
    _fit_lib().tbr_profile_reset()


def profile_read(kernel: str) -> tuple[int, float]:
    """(launches, total device ms) of one kernel since the last reset."""
    t = TbrKernelTime()
    check(_fit_lib().tbr_profile_read(KERNELS[kernel], ctypes.byref(t)))
    return int(t.launches), float(t.total_ms)


PEAK_KINDS = {"ffma2": 0, "ffma": 1, "ex2": 2, "rcp": 3}


def measure_peak(kind: str, iters: int = 200000, stream=None) -> tuple[float, float]:
    """tbr_measure_peak: (operations per second, timed launch ms) of one chain
    microbenchmark on every SM -- FLOPs for "ffma2" / "ffma" (a fused
    multiply-add counts 2 per lane), MUFU results for "ex2" / "rcp"."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    check(_fit_lib().tbr_measure_peak(PEAK_KINDS[kind], int(iters), ctypes.byref(rate), ctypes.byref(ms),
                                      _stream(stream)))
    return float(rate.value), float(ms.value)


# ---------------------------------------------------------------------------
# torch.autograd wrapper: soft render forward, replay adjoint backward
# ---------------------------------------------------------------------------
class SoftRender(torch.autograd.Function):
    """R = soft render of (cx, cy, theta, length, half_width, logits, palette);
    backward runs the replay adjoint (tbr_render_backward)."""

    @staticmethod
    def forward(fctx, cx, cy, theta, length, half_width, logits, palette, W, H, tau, tau_min,
                background, color_temp, checkpoint_every, record_capacity):
        dp = DeviceProgram(cx.detach().contiguous(), cy.detach().contiguous(), theta.detach().contiguous(),
                           length.detach().contiguous(), half_width.detach().contiguous(),
                           logits.detach().contiguous(), palette.detach().contiguous(),
                           tuple(float(b) for b in background), float(color_temp))
        rgb, sctx = render_soft(dp, W, H, tau, tau_min, record=True, checkpoint_every=checkpoint_every,
                                record_capacity=record_capacity)
        fctx.sctx = sctx
        return rgb

    @staticmethod
    def backward(fctx, grad_rgb):
        sctx = fctx.sctx
        g = sctx.backward(grad_rgb.contiguous().float())
        sctx.status()
        sctx.destroy()
        fctx.sctx = None
        return (g["cx"], g["cy"], g["theta"], g["length"], g["half_width"], g["logits"], g["palette"],
                None, None, None, None, None, None, None, None)


def soft_render(cx, cy, theta, length, half_width, logits, palette, W, H, tau, tau_min,
                background=(1.0, 1.0, 1.0), color_temp=1.0, checkpoint_every=0, record_capacity=0):
    """Differentiable soft render (the replay adjoint provides the gradients)."""
    return SoftRender.apply(cx, cy, theta, length, half_width, logits, palette, W, H, tau, tau_min,
                            background, color_temp, checkpoint_every, record_capacity)


def soft_adjoint_mse(prog: DeviceProgram, target: torch.Tensor, tau: float, tau_min: float,
                     checkpoint_every: int = 0, record_capacity: int = 0, want_rgb: bool = False,
                     want_palette: bool = True, stats: bool = False, stream=None):
    """tbr_render_soft_adjoint_mse: loss-fused soft forward + replay adjoint.
    Returns (loss [1] device tensor, gradients dict, rgb or None, stats dict or None)."""
    L = lib()
    if not getattr(L, "_fused_typed", False):
        P = ctypes.c_void_p
        L.tbr_render_soft_adjoint_mse.argtypes = [ctypes.POINTER(TbrProgram), ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.POINTER(TbrSoftOpts), P, P, P, P, P, P, P, P, P, P,
                                                  ctypes.POINTER(TbrCtxStats), P]
        L.tbr_render_soft_adjoint_mse.restype = ctypes.c_int
        L._fused_typed = True
    t = target.contiguous()
    H, W = int(t.shape[0]), int(t.shape[1])
    dev = prog.cx.device
    e = lambda *sh: torch.empty(sh, device=dev, dtype=torch.float32)
    n, k = prog.n, prog.k
    g = {"cx": e(n), "cy": e(n), "theta": e(n), "length": e(n), "half_width": e(n), "logits": e(n, k),
         "palette": e(k, 3) if want_palette else None}
    loss = e(1)
    rgb = e(H, W, 3) if want_rgb else None
    opts = TbrSoftOpts(float(tau), float(tau_min), int(checkpoint_every), int(record_capacity), 0)
    st = TbrCtxStats() if stats else None
    s = prog.struct()
    check(L.tbr_render_soft_adjoint_mse(ctypes.byref(s), W, H, ctypes.byref(opts), _ptr(t), _ptr(rgb), _ptr(loss),
                                        _ptr(g["cx"]), _ptr(g["cy"]), _ptr(g["theta"]), _ptr(g["length"]),
                                        _ptr(g["half_width"]), _ptr(g["logits"]), _ptr(g["palette"]),
                                        ctypes.byref(st) if st is not None else None, _stream(stream)))
    sd = {f: getattr(st, f) for f, _ in TbrCtxStats._fields_} if st is not None else None
    return loss, g, rgb, sd


# ---------------------------------------------------------------------------
# Serving (tbr_serve_*)
# ---------------------------------------------------------------------------
REQ_HARD, REQ_SOFT_ADJOINT, REQ_RECOLOUR, REQ_REORDER, REQ_INSERT = 0, 1, 2, 3, 4


class TbrServeConfig(ctypes.Structure):
    _fields_ = [("memory_cap_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32),
                ("max_strokes", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
                ("record_capacity", ctypes.c_int32), ("idle_exit_us", ctypes.c_int32),
                ("ready_wait_us", ctypes.c_int32)]


class TbrRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("program", ctypes.c_uint64), ("W", ctypes.c_int32),
                ("H", ctypes.c_int32), ("n_prefix", ctypes.c_int32), ("snap", ctypes.c_int32),
                ("tau", ctypes.c_float), ("tau_min", ctypes.c_float), ("target", ctypes.c_void_p),
                ("out_rgb", ctypes.c_void_p), ("out_idx", ctypes.c_void_p), ("out_loss", ctypes.c_void_p),
                ("out_grad", ctypes.c_void_p), ("edit_a", ctypes.c_int32), ("edit_b", ctypes.c_int32),
                ("edit_start", ctypes.c_int32), ("insert_palette", ctypes.c_int32),
                ("insert_stroke", ctypes.c_float * 5), ("ready", ctypes.c_void_p)]


class TbrServeCounters(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("refused", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("inflight", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("fixed_bytes", ctypes.c_int64),
                ("persistent_ctas", ctypes.c_int32)]


def _serve_lib():
    L = lib()
    if not getattr(L, "_serve_typed", False):
        P = ctypes.c_void_p
        L.tbr_serve_default_config.argtypes = [ctypes.POINTER(TbrServeConfig)]
        L.tbr_serve_default_config.restype = None
        L.tbr_serve_create.argtypes = [ctypes.POINTER(TbrServeConfig), ctypes.POINTER(P)]
        L.tbr_serve_load_program.argtypes = [P, ctypes.POINTER(TbrProgram), ctypes.POINTER(ctypes.c_uint64)]
        L.tbr_serve_submit.argtypes = [P, ctypes.POINTER(TbrRequest), ctypes.POINTER(ctypes.c_uint64), P]
        L.tbr_serve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int)]
        L.tbr_serve_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int)]
        L.tbr_serve_request_times.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]
        L.tbr_serve_release.argtypes = [P, ctypes.c_uint64]
        L.tbr_serve_stats.argtypes = [P, ctypes.POINTER(TbrServeCounters)]
        L.tbr_serve_destroy.argtypes = [P]
        L.tbr_serve_destroy.restype = None
        for f in ("tbr_serve_create", "tbr_serve_load_program", "tbr_serve_submit", "tbr_serve_poll",
                  "tbr_serve_wait", "tbr_serve_request_times", "tbr_serve_release", "tbr_serve_stats"):
            getattr(L, f).restype = ctypes.c_int
        L._serve_typed = True
    return L


def default_serve_config(**overrides) -> TbrServeConfig:
    c = TbrServeConfig()
    _serve_lib().tbr_serve_default_config(ctypes.byref(c))
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


class Server:
    """tbr_serve_*: continuous-batching server on the current device."""

    def __init__(self, config: Optional[TbrServeConfig] = None):
        L = _serve_lib()
        self.config = config if config is not None else default_serve_config()
        h = ctypes.c_void_p()
        check(L.tbr_serve_create(ctypes.byref(self.config), ctypes.byref(h)))
        self.handle = h.value
        self._keep = {}

    def load_program(self, prog: DeviceProgram) -> int:
        pid = ctypes.c_uint64()
        s = prog.struct()
        check(_serve_lib().tbr_serve_load_program(ctypes.c_void_p(self.handle), ctypes.byref(s), ctypes.byref(pid)))
        return int(pid.value)

    def submit(self, kind: int, program: int, W: int, H: int, out_rgb=None, out_idx=None, target=None,
               out_loss=None, out_grad=None, tau=0.0, tau_min=1.0, snap=False, edit_a=0, edit_b=0,
               edit_start=0, insert_palette=0, insert_stroke=(0.5, 0.5, 0.0, 0.0, 0.05), stream=None,
               ready=None) -> int:
        """ready: optional int32 tensor (device memory) whose first word the
        request's work items wait to become nonzero (tbr_request.ready)."""
        r = TbrRequest()
        r.kind, r.program, r.W, r.H, r.n_prefix, r.snap = kind, program, W, H, -1, int(bool(snap))
        r.tau, r.tau_min = float(tau), float(tau_min)
        r.target, r.out_rgb, r.out_idx = _ptr(target), _ptr(out_rgb), _ptr(out_idx)
        r.out_loss, r.out_grad = _ptr(out_loss), _ptr(out_grad)
        r.edit_a, r.edit_b, r.edit_start, r.insert_palette = edit_a, edit_b, edit_start, insert_palette
        r.insert_stroke = (ctypes.c_float * 5)(*[float(v) for v in insert_stroke])
        if ready is not None and ready.dtype != torch.int32:
            raise TypeError("ready must be an int32 tensor")
        r.ready = _ptr(ready)
        rid = ctypes.c_uint64()
        check(_serve_lib().tbr_serve_submit(ctypes.c_void_p(self.handle), ctypes.byref(r), ctypes.byref(rid),
                                            _stream(stream)))
        # keep the caller's buffers alive until the request is released
        self._keep[int(rid.value)] = (target, out_rgb, out_idx, out_loss, out_grad, ready)
        return int(rid.value)

    def poll(self, rid: int) -> tuple[bool, int]:
        done, res = ctypes.c_int32(), ctypes.c_int()
        check(_serve_lib().tbr_serve_poll(ctypes.c_void_p(self.handle), rid, ctypes.byref(done), ctypes.byref(res)))
        return bool(done.value), int(res.value)

    def wait(self, rid: int, timeout_ms: int = 60000) -> int:
        res = ctypes.c_int()
        check(_serve_lib().tbr_serve_wait(ctypes.c_void_p(self.handle), rid, timeout_ms, ctypes.byref(res)))
        return int(res.value)

    def times(self, rid: int) -> tuple[float, float]:
        q, l = ctypes.c_double(), ctypes.c_double()
        check(_serve_lib().tbr_serve_request_times(ctypes.c_void_p(self.handle), rid, ctypes.byref(q),
                                                   ctypes.byref(l)))
        return float(q.value), float(l.value)

    def release(self, rid: int) -> None:
        check(_serve_lib().tbr_serve_release(ctypes.c_void_p(self.handle), rid))
        self._keep.pop(rid, None)

    def stats(self) -> dict:
        c = TbrServeCounters()
        check(_serve_lib().tbr_serve_stats(ctypes.c_void_p(self.handle), ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in TbrServeCounters._fields_}

    def destroy(self) -> None:
        if self.handle is not None:
            _serve_lib().tbr_serve_destroy(ctypes.c_void_p(self.handle))
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
