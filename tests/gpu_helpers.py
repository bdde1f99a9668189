"""Helpers for the GPU parity tests: run the CUDA path through the C ABI."""
from __future__ import annotations

import numpy as np
import torch

from paper_2104_07526_gb300 import pcr

U64_EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def ensure_built():
    from paper_2104_07526_gb300 import build
    build.build()
    pcr.lib()


class Renderer:
    """One pcr context on torch's current stream, plus device buffers."""

    def __init__(self, device: int = 0):
        ensure_built()
        self.ctx = pcr.Context(device, stream=torch.cuda.current_stream())
        self.h = self.ctx.handle
        self.points = None
        self.n = 0
        self.fb = None
        self.size = None

    def close(self):
        self.ctx.close()

    def upload(self, cloud) -> torch.Tensor:
        t = cloud if isinstance(cloud, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(cloud))
        self.points = t.to("cuda").contiguous()
        self.n = self.points.shape[0]
        pcr.pcr_upload_points(self.h, self.points if self.n else None, self.n)
        return self.points

    def view(self, m, width: int, height: int):
        pcr.pcr_set_matrix(self.h, np.asarray(m, dtype=np.float32))
        pcr.pcr_set_viewport(self.h, width, height)
        if self.size != (width, height):
            self.fb = pcr.alloc_framebuffer(width, height)
            self.size = (width, height)
            pcr.pcr_set_framebuffer(self.h, self.fb["keys"], self.fb["hq_depth"], self.fb["hq_rg"], self.fb["hq_ba"])
            pcr.pcr_set_hq1r_buffer(self.h, self.fb["hq1r_primary"])
            pcr.pcr_set_lock_buffer(self.h, self.fb["locks"], 0)

    def render_basic(self, variant: int, clear: bool = True) -> np.ndarray:
        pcr.pcr_render_basic(self.h, variant, clear)
        return self.keys()

    def render_rgb(self, variant: int, clear: bool = True) -> np.ndarray:
        pcr.pcr_render_rgb(self.h, variant, clear)
        return self.keys()

    def keys(self) -> np.ndarray:
        torch.cuda.synchronize()
        return self.fb["keys"].cpu().numpy().view(np.uint64)

    def render_hq(self, variant: int, factor: float = 1.01, clear: bool = True):
        pcr.pcr_render_hq(self.h, factor, variant, clear)
        torch.cuda.synchronize()
        return (self.fb["hq_depth"].cpu().numpy().view(np.uint32), self.fb["hq_rg"].cpu().numpy().view(np.uint64),
                self.fb["hq_ba"].cpu().numpy().view(np.uint64))

    def render_hq1r_sums(self, variant: int, factor: float = 1.01):
        """HQS1R render; returns (depth, r, g, b, count) with the primary
        word's fields (r 14 bits at 50, g 14 at 36, b 14 at 22, count 22 at
        0) added to the 32-bit fallback sums."""
        pcr.pcr_render_hq1r(self.h, factor, variant, True)
        torch.cuda.synchronize()
        p = self.fb["hq1r_primary"].cpu().numpy().view(np.uint64)
        rg = self.fb["hq_rg"].cpu().numpy().view(np.uint64)
        ba = self.fb["hq_ba"].cpu().numpy().view(np.uint64)
        m14, m22, m32 = np.uint64(0x3FFF), np.uint64(0x3FFFFF), np.uint64(0xFFFFFFFF)
        r = (rg >> np.uint64(32)) + ((p >> np.uint64(50)) & m14)
        g = (rg & m32) + ((p >> np.uint64(36)) & m14)
        b = (ba >> np.uint64(32)) + ((p >> np.uint64(22)) & m14)
        c = (ba & m32) + (p & m22)
        d = self.fb["hq_depth"].cpu().numpy().view(np.uint32)
        return d, r, g, b, c

    def resolve(self, mode: int, background: int = 0) -> np.ndarray:
        pcr.pcr_resolve(self.h, mode, self.fb["image"], background)
        torch.cuda.synchronize()
        return self.fb["image"].cpu().numpy().view(np.uint32)


def reorder_gpu(h: int, cloud_dev: torch.Tensor, seed: int, mode: int):
    """Reorder a device cloud in place; returns perm[new] = old (numpy)."""
    n = cloud_dev.shape[0]
    ws = torch.empty(max(pcr.pcr_reorder_workspace_size(n), 1), dtype=torch.uint8, device="cuda")
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    pcr.pcr_reorder_morton_shuffle128(h, cloud_dev if n else None, n, seed, mode, ws, perm if n else None)
    torch.cuda.synchronize()
    return perm[:n].cpu().numpy().view(np.uint32)
