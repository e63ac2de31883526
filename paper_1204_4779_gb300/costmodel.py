"""Learned cost model of the variant tuner: a 3-layer MLP (width 64, FP32) trained and
evaluated on the GPU by the library's own kernels (hydro_mlp_* of the C ABI).  This module only
marshals arguments; torch holds the device arrays.

The model maps a feature vector of (kernel variant, grid) to the standardised logarithm of
the measured time per cell-update; the tuner uses it to rank candidate variants before
benchmarking them.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import hydro


class MLP:
    def __init__(self, d: int, hidden: int = 64, seed: int = 0, device=None):
        self.lib = hydro.load_library()
        self.d, self.hidden = int(d), int(hidden)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        n = ctypes.c_int64()
        hydro._check(self.lib.hydro_mlp_sizes(self.d, self.hidden, 1, ctypes.byref(n), None),
                     "hydro_mlp_sizes")
        self.n_params = int(n.value)
        rng = np.random.default_rng(seed)
        p = np.empty(self.n_params, dtype=np.float32)
        H, dd = self.hidden, self.d
        o = 0
        for fan_in, rows, cols in ((dd, H, dd), (H, H, H), (H, 1, H)):
            w = rng.normal(0.0, 1.0 / np.sqrt(fan_in), rows * cols)
            p[o:o + rows * cols] = w
            o += rows * cols
            p[o:o + rows] = 0.0
            o += rows
        self.params = torch.from_numpy(p).to(self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = 0
        self._ws = None
        self._ws_n = 0

    def _workspace(self, n: int):
        if self._ws is None or self._ws_n < n:
            b = ctypes.c_size_t()
            hydro._check(self.lib.hydro_mlp_sizes(self.d, self.hidden, int(n), None, ctypes.byref(b)),
                         "hydro_mlp_sizes")
            self._ws = torch.empty(int(b.value), dtype=torch.uint8, device=self.device)
            self._ws_n = n
        return self._ws

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def _xt(self, X, t=None):
        X = torch.as_tensor(np.asarray(X, dtype=np.float32)).to(self.device).contiguous()
        if X.dim() != 2 or X.shape[1] != self.d:
            raise ValueError(f"inputs must be (n, {self.d})")
        tt = None
        if t is not None:
            tt = torch.as_tensor(np.asarray(t, dtype=np.float32)).to(self.device).contiguous()
        return X, tt

    def predict(self, X) -> np.ndarray:
        X, _ = self._xt(X)
        n = X.shape[0]
        y = torch.empty(n, dtype=torch.float32, device=self.device)
        hydro._check(self.lib.hydro_mlp_forward(self.params.data_ptr(), self.d, self.hidden,
                                                X.data_ptr(), n, y.data_ptr(),
                                                self._workspace(n).data_ptr(), self._stream()),
                     "hydro_mlp_forward")
        return y.cpu().numpy()

    def gradient(self, X, t):
        """(gradient of the mean squared loss w.r.t. the flat parameters, loss)."""
        X, tt = self._xt(X, t)
        n = X.shape[0]
        g = torch.empty_like(self.params)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        hydro._check(self.lib.hydro_mlp_gradient(self.params.data_ptr(), self.d, self.hidden,
                                                 X.data_ptr(), tt.data_ptr(), n,
                                                 self._workspace(n).data_ptr(), g.data_ptr(),
                                                 loss.data_ptr(), self._stream()),
                     "hydro_mlp_gradient")
        return g.cpu().numpy(), float(loss.item())

    def adam(self, grad, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        g = torch.as_tensor(np.asarray(grad, dtype=np.float32)).to(self.device).contiguous()
        self.step_count += 1
        hydro._check(self.lib.hydro_mlp_adam(self.params.data_ptr(), self.m.data_ptr(),
                                             self.v.data_ptr(), g.data_ptr(), self.n_params,
                                             self.step_count, lr, beta1, beta2, eps,
                                             self._stream()), "hydro_mlp_adam")

    def train(self, X, t, epochs: int, lr: float = 3e-3):
        """Full-batch Adam on the GPU; returns the loss history (one value per epoch)."""
        X, tt = self._xt(X, t)
        n = X.shape[0]
        losses = torch.empty(max(epochs, 1), dtype=torch.float32, device=self.device)
        hydro._check(self.lib.hydro_mlp_train(self.params.data_ptr(), self.m.data_ptr(),
                                              self.v.data_ptr(), self.d, self.hidden,
                                              X.data_ptr(), tt.data_ptr(), n, int(epochs),
                                              self.step_count, lr,
                                              self._workspace(n).data_ptr(), losses.data_ptr(),
                                              self._stream()), "hydro_mlp_train")
        self.step_count += int(epochs)
        return losses[:epochs].cpu().numpy()

    def get_params(self) -> np.ndarray:
        return self.params.cpu().numpy().astype(np.float64)

    def set_params(self, p):
        self.params.copy_(torch.as_tensor(np.asarray(p, dtype=np.float32)))
