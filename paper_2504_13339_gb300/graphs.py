"""CUDA-graph capture of whole rendering / training steps.

Every library call enqueues kernels on the caller's stream with no host
synchronisation (instance counts stay on the device), so a complete step --
projection, binning, sort, compositing of all views and TFs, loss and
backward -- can be captured once and replayed, removing the per-launch host
cost.  Buffer addresses are baked into the graph: replays must reuse the same
tensors (update their contents in place).
"""
from __future__ import annotations

import torch

from . import _lib


class CapturedStep:
    """Captures `fn()` (which must only enqueue work on the current stream)
    after `warmup` eager runs on a side stream; `replay()` re-executes it.
    `launches` is the number of library kernels in one replay."""

    def __init__(self, fn, warmup=2):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                fn()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        before = _lib.veg_kernel_launches()
        with torch.cuda.graph(self.graph):
            fn()
        self.launches = _lib.veg_kernel_launches() - before
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()
