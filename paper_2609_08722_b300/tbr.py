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
EXPORTED = ["tbr_render_hard", "tbr_render_soft", "tbr_render_backward", "tbr_ctx_status",
            "tbr_ctx_bytes", "tbr_ctx_destroy", "tbr_loss_mse", "tbr_last_error", "tbr_version"]


class TbrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class TbrProgram(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("k", ctypes.c_int32),
                ("cx", ctypes.c_void_p), ("cy", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("length", ctypes.c_void_p), ("half_width", ctypes.c_void_p),
                ("logits", ctypes.c_void_p), ("palette", ctypes.c_void_p),
                ("background", ctypes.c_float * 3), ("color_temp", ctypes.c_float)]


class TbrHardStats(ctypes.Structure):
    _fields_ = [("band_steps", ctypes.c_int64), ("background_pixels", ctypes.c_int64),
                ("visited_steps", ctypes.c_int64)]


class TbrSoftOpts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("tau_min", ctypes.c_float),
                ("checkpoint_every", ctypes.c_int32), ("record_capacity", ctypes.c_int32),
                ("inert", ctypes.c_int32)]


class TbrCtxStats(ctypes.Structure):
    _fields_ = [("records", ctypes.c_int64), ("max_records", ctypes.c_int64),
                ("overflow_pixels", ctypes.c_int64), ("drift_resets", ctypes.c_int64),
                ("timeouts", ctypes.c_int64), ("invalid_params", ctypes.c_int64)]


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
            for f in ("tbr_render_hard", "tbr_render_soft", "tbr_render_backward", "tbr_ctx_status",
                      "tbr_loss_mse"):
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
        return cls(cx=t(prog.cx), cy=t(prog.cy), theta=t(prog.theta), length=t(prog.length),
                   half_width=t(prog.half_width), logits=t(prog.logits), palette=t(prog.palette),
                   background=tuple(float(v) for v in np.asarray(prog.background)),
                   color_temp=float(prog.color_temp))

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
        return s


def render_hard(prog: DeviceProgram, W: int, H: int, n_prefix: int = -1, snap: bool = False,
                with_idx: bool = True, stats: bool = False, out_rgb=None, out_idx=None, stream=None):
    """tbr_render_hard; returns (rgb [H,W,3], idx [H,W] or None, stats dict or None)."""
    dev = prog.cx.device
    rgb = out_rgb if out_rgb is not None else torch.empty((H, W, 3), device=dev, dtype=torch.float32)
    idx = out_idx if out_idx is not None else (
        torch.empty((H, W), device=dev, dtype=torch.int32) if with_idx else None)
    st = TbrHardStats() if stats else None
    s = prog.struct()
    check(lib().tbr_render_hard(ctypes.byref(s), W, H, n_prefix, int(bool(snap)), _ptr(rgb), _ptr(idx),
                                ctypes.byref(st) if st is not None else None, _stream(stream)))
    sd = None
    if st is not None:
        sd = {"band_steps": st.band_steps, "background_pixels": st.background_pixels,
              "visited_steps": st.visited_steps}
    return rgb, idx, sd


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
                out_rgb=None, stream=None):
    """tbr_render_soft; returns (rgb [H,W,3], SoftContext or None)."""
    dev = prog.cx.device
    rgb = out_rgb if out_rgb is not None else torch.empty((H, W, 3), device=dev, dtype=torch.float32)
    opts = TbrSoftOpts(float(tau), float(tau_min), int(checkpoint_every), int(record_capacity),
                       int(bool(inert)))
    handle = ctypes.c_void_p()
    s = prog.struct()
    check(lib().tbr_render_soft(ctypes.byref(s), W, H, ctypes.byref(opts), _ptr(rgb),
                                ctypes.byref(handle) if record else None, _stream(stream)))
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
