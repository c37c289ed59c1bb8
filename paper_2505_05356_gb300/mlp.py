"""Deformation MLP on the tensor cores (Sec. 4, "MLP"): binding of
gftorf_mlp_forward / gftorf_mlp_backward.

delta[b][g] = MLP(gamma(means[g] * inv_scale), gamma(times[b])); its output is
the renderer's per-frame displacement input (``params["delta"]``), and the
renderer's ``grads["delta"]`` is the backward's input.  Parameters are one
packed float32 vector (layout in include/gftorf.h; ``scenes.init_mlp_params``
draws the paper's initialisation).
"""
from __future__ import annotations

import ctypes
from typing import Sequence, Tuple

import torch

from . import gftorf

WIDTH, DEPTH, INPUT = 256, 8, 128
C_LIGHT = 299792458.0


def unambiguous_range(freq_hz: float) -> float:
    """d_u = c / (2 f): the positions are divided by it before encoding."""
    return C_LIGHT / (2.0 * freq_hz)


def _lib():
    L = gftorf.load()
    if not getattr(L, "_mlp_typed", False):
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        L.gftorf_mlp_param_count.restype = sz
        L.gftorf_mlp_param_count.argtypes = []
        L.gftorf_mlp_workspace_size.restype = sz
        L.gftorf_mlp_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int32]
        L.gftorf_mlp_forward.restype = ctypes.c_int
        L.gftorf_mlp_forward.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, vp,
                                         ctypes.POINTER(ctypes.c_float), ctypes.c_float, vp, vp,
                                         sz, vp]
        L.gftorf_mlp_backward.restype = ctypes.c_int
        L.gftorf_mlp_backward.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, vp,
                                          ctypes.POINTER(ctypes.c_float), ctypes.c_float, vp, vp,
                                          vp, vp, sz, vp]
        L.gftorf_mlp_infer_workspace_size.restype = sz
        L.gftorf_mlp_infer_workspace_size.argtypes = []
        L.gftorf_mlp_infer.restype = ctypes.c_int
        L.gftorf_mlp_infer.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, vp,
                                       ctypes.POINTER(ctypes.c_float), ctypes.c_float, vp, vp,
                                       sz, vp]
        L.gftorf_mlp_export.restype = ctypes.c_int
        L.gftorf_mlp_export.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, vp, vp, sz, vp]
        L.gftorf_mlp_debug_inject.restype = None
        L.gftorf_mlp_debug_inject.argtypes = [ctypes.c_int32]
        L.gftorf_mlp_read_status.restype = ctypes.c_int
        L.gftorf_mlp_read_status.argtypes = [vp, sz, vp]
        L._mlp_typed = True
    return L


def param_count() -> int:
    return int(_lib().gftorf_mlp_param_count())


class DeformationMLP:
    """Workspace for one (N Gaussians, B frames) shape."""

    def __init__(self, n_gaussians: int, n_frames: int, inv_scale: float, device="cuda"):
        gftorf._require_cuda()
        self.lib = _lib()
        self.N, self.B, self.inv_scale = int(n_gaussians), int(n_frames), float(inv_scale)
        nbytes = self.lib.gftorf_mlp_workspace_size(self.N, self.B)
        if nbytes == 0:
            raise gftorf.GftorfError(gftorf.ERR_ARG, "gftorf_mlp_workspace_size")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_ptr = ctypes.c_void_p(self.ws.data_ptr() + off)
        self.ws_bytes = nbytes
        self.device = torch.device(device)

    def _times(self, times: Sequence[float]):
        if len(times) != self.B:
            raise ValueError("expected %d times" % self.B)
        return (ctypes.c_float * self.B)(*[float(t) for t in times])

    def _check_f32(self, **ts):
        for k, t in ts.items():
            if t is not None and (t.dtype != torch.float32 or not t.is_contiguous()):
                raise ValueError("%s must be contiguous float32" % k)

    def forward(self, theta: torch.Tensor, means: torch.Tensor, times: Sequence[float],
                delta: torch.Tensor = None) -> torch.Tensor:
        self._check_f32(theta=theta, means=means)
        if delta is None:
            delta = torch.empty((self.B, self.N, 3), dtype=torch.float32, device=self.device)
        self._keep = self._times(times)
        gftorf._check(self.lib.gftorf_mlp_forward(self.N, self.B, gftorf._ptr(theta),
                                                  gftorf._ptr(means), self._keep,
                                                  self.inv_scale, gftorf._ptr(delta),
                                                  self.ws_ptr, self.ws_bytes, gftorf._stream()),
                      "gftorf_mlp_forward")
        return delta

    def infer(self, theta: torch.Tensor, means: torch.Tensor, times: Sequence[float],
              delta: torch.Tensor = None) -> torch.Tensor:
        """Forward without keeping activations (one fused kernel; bit-identical
        to forward())."""
        self._check_f32(theta=theta, means=means)
        if delta is None:
            delta = torch.empty((self.B, self.N, 3), dtype=torch.float32, device=self.device)
        self._keep_i = self._times(times)
        gftorf._check(self.lib.gftorf_mlp_infer(self.N, self.B, gftorf._ptr(theta),
                                                gftorf._ptr(means), self._keep_i, self.inv_scale,
                                                gftorf._ptr(delta), self.ws_ptr, self.ws_bytes,
                                                gftorf._stream()),
                      "gftorf_mlp_infer")
        return delta

    def backward(self, theta, means, times, d_delta, d_theta=None,
                 d_means=None) -> Tuple[torch.Tensor, torch.Tensor]:
        self._check_f32(theta=theta, means=means, d_delta=d_delta)
        if d_theta is None:
            d_theta = torch.empty_like(theta)
        if d_means is None:
            d_means = torch.empty_like(means)
        self._keep_b = self._times(times)
        gftorf._check(self.lib.gftorf_mlp_backward(self.N, self.B, gftorf._ptr(theta),
                                                   gftorf._ptr(means), self._keep_b,
                                                   self.inv_scale, gftorf._ptr(d_delta),
                                                   gftorf._ptr(d_theta), gftorf._ptr(d_means),
                                                   self.ws_ptr, self.ws_bytes, gftorf._stream()),
                      "gftorf_mlp_backward")
        return d_theta, d_means

    def export(self, what: str, layer: int = 0) -> torch.Tensor:
        """An intermediate of the last forward / backward as float32
        (B N rows): 'enc', 'H' (layer), 'dZ' (layer), 'd_enc'."""
        code = {"enc": 0, "H": 1, "dZ": 2, "d_enc": 3}[what]
        M = self.N * self.B
        cols = INPUT if code in (0, 3) else WIDTH
        if code == 3:
            out = torch.empty((M, cols), dtype=torch.float32, device=self.device)
        else:
            out = torch.empty((M, cols), dtype=torch.int16, device=self.device)
        gftorf._check(self.lib.gftorf_mlp_export(self.N, self.B, code, layer, gftorf._ptr(out),
                                                 self.ws_ptr, self.ws_bytes, gftorf._stream()),
                      "gftorf_mlp_export")
        if code == 3:
            return out
        return (out.to(torch.int32) << 16).view(torch.float32)

    def read_status(self) -> int:
        return int(self.lib.gftorf_mlp_read_status(self.ws_ptr, self.ws_bytes, gftorf._stream()))

    def check(self):
        code = self.read_status()
        if code != gftorf.OK:
            raise gftorf.GftorfError(code, "device status")


def debug_inject(mode: int):
    """Test hooks: 1 = the kernels' load warps issue nothing, so their bounded
    waits run out (GFTORF_ERR_TIMEOUT, no GPU fault); 2 = the training
    forward and the backward's dZ chain run one GEMM per layer instead of
    fused; 0 = normal."""
    _lib().gftorf_mlp_debug_inject(int(mode))
