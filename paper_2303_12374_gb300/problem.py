"""Host-side marshalling for one grid: padded device buffers in the layout
kl_layout() recommends, and copies of interior blocks in and out.

This file only moves data (numpy <-> torch, interior <-> padded buffer); all
stencil work runs in libkl's kernels.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import kl

TORCH_DTYPES = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16, 3: torch.float16}


class Problem:
    """Layout and scalars of one grid; buffers are 1D torch tensors of `extent` elements."""

    def __init__(self, nx, ny, nz, *, g, dtype, walls, dx=None, dy=None, dz=None, zh=None,
                 nu=0.0, device="cuda", xybc=False):
        self.nx, self.ny, self.nz, self.g = nx, ny, nz, g
        self.dtype = kl.DTYPES[dtype] if isinstance(dtype, str) else dtype
        self.tdtype = TORCH_DTYPES[self.dtype]
        self.device = device
        self.sj, self.sk, self.origin, self.extent = kl.kl_layout(nx, ny, nz, g, self.dtype)
        self._zh = None
        zh_ptr = None
        if zh is not None:
            self._zh = np.ascontiguousarray(zh, dtype=np.float64)
            zh_ptr = self._zh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.grid = kl.Grid(nx, ny, nz, g, self.sj, self.sk, self.origin, self.extent,
                            1 if walls else 0, 1 if xybc else 0,
                            dx if dx else 1.0 / nx, dy if dy else 1.0 / ny,
                            dz if dz else (0.0 if zh is not None else 1.0 / nz), nu, zh_ptr)

    # ---------------------------------------------------------- buffers
    def empty(self, dtype=None) -> torch.Tensor:
        return torch.zeros(self.extent, dtype=dtype or self.tdtype, device=self.device)

    def view(self, buf: torch.Tensor) -> torch.Tensor:
        """(nz, ny, nx) strided view of the interior of a padded buffer."""
        return buf.as_strided((self.nz, self.ny, self.nx), (self.sk, self.sj, 1), self.origin)

    def padded_view(self, buf: torch.Tensor) -> torch.Tensor:
        g = self.g
        return buf.as_strided((self.nz + 2 * g, self.ny + 2 * g, self.nx + 2 * g),
                              (self.sk, self.sj, 1), self.origin - g * (1 + self.sj + self.sk))

    def upload(self, a: np.ndarray, dtype=None) -> torch.Tensor:
        buf = self.empty(dtype)
        self.view(buf).copy_(torch.from_numpy(np.ascontiguousarray(a)).to(buf.dtype))
        return buf

    def download(self, buf: torch.Tensor) -> np.ndarray:
        return self.view(buf).to(torch.float64).cpu().numpy()

    def rounded(self, a: np.ndarray) -> np.ndarray:
        """Values of `a` after rounding to the storage type (what the kernels see)."""
        return torch.from_numpy(np.ascontiguousarray(a)).to(self.tdtype).to(torch.float64).numpy()
